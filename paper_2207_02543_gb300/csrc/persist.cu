// Persistent PCG iterations (an option for small problems): one cooperative launch runs up to
// `iters` whole iterations of Algorithm 3 (PCG preconditioned by one two-grid cycle
// AMG(0; K, r, r1, r2) of Algorithm 2 with P = Phi_r, Section 3.3; damped Jacobi,
// r1 = r2 = 1) for the ACTIVE lanes of a batch. Where the matrix and vectors of all
// slots are a few MB, the eight kernels per iteration of the graph path are bound by
// their launch and drain latency, not by bytes; here the phases of an iteration are
// separated by grid-wide barriers instead of kernel boundaries. (Measured, it reaches
// parity with the graph at a few thousand unknowns and loses above; the autotuner
// decides.)
//
// Phases of one iteration (| = grid barrier):
//   A  p = s + beta p                                                          |
//   B  q = K p (double-float), partial p^T q                                   |
//   C  alpha per slot, x += alpha p, r -= alpha q                              |
//   D  y1 = omega D^-1 r, r1 = r - K y1, partial ||r||^2 and Phi^T r1           |
//   E  convergence test, e_c = L^-T L^-1 Phi^T r1 for the slots this CTA owns  |
//   F  s = y1 + Phi e_c + omega D^-1 (r1 - (K Phi) e_c), partial r^T s         |
//      (the post-smoothing from K Phi: K y2 = (r - r1) + (K Phi) e_c)
//   beta per slot
// Every CTA forms the per-slot scalars itself from the same partial sums, added in the
// same fixed order, so all CTAs hold identical copies (in shared memory) and take the
// same decisions; CTA 0 writes them back at the end. Arithmetic per element follows
// the graph path's kernels (double-float outer vectors, FP32 preconditioner, FP64
// scalars and coarse solve); only the grouping of the partial sums differs.
//
// Vectors written during the launch by another CTA are read through L2
// (ld.global.cg), never through the non-coherent read-only path. A barrier wait is
// bounded: when it expires the CTA sets *err = 3 and returns, and every other CTA
// gives up at its next barrier (bounded as well), so the launch always ends.
#include "common.cuh"
#include "lanes.cuh"

namespace {

constexpr int PERSIST_OUT = 16;                 // restriction outputs per thread (Bp * kp <= 16 * 256)
constexpr unsigned PERSIST_POLLS = 1u << 24;    // bound on the polls of one barrier wait (>= ~1 s)

struct PersistArgs {
    int nb, n, Bp, lgBp, k, kp, stat, pr, iters;
    float omega;
    const int32_t* row_ptr;
    const int32_t* col_idx;
    const float* vals;   // [nnzb][bs*bs][Bp]
    const float* dinv;   // [n][Bp]
    const float* phi;    // [n][kp]
    const float* W;      // K Phi per slot, mode-major [kp][n][Bp]
    const double* Lc;    // Cholesky factors [Bp][k][k]
    float2* x;
    float2* r;
    float2* p;
    float2* q;
    float* s;
    float* r1;
    float* ec;           // [Bp][kp]
    double* part;        // [G][2 Bp]
    double* tot;         // [2 Bp] per-slot totals of part, written by the last CTA to arrive
    double* cpart;       // [G][Bp][kp]
    SlotScalars* sc;
    unsigned* bar;       // bar[0] arrivals, bar[1] the latest released summing barrier; zero at launch
    int* err;
};

// Per-slot total over the G partial rows part[g * 2 Bp + off + slot], in the same fixed
// order in every CTA; returned in threads t < Bp.
__device__ __forceinline__ double slot_total(const double* part, int G, int Bp, int off, double* s_tmp) {
    const int Q = blockDim.x / Bp;
    const int b = threadIdx.x % Bp, qd = threadIdx.x / Bp;
    const int g0 = (int)((long long)G * qd / Q), g1 = (int)((long long)G * (qd + 1) / Q);
    double s = 0.0;
    int g = g0;
    for (; g + 8 <= g1; g += 8) {   // eight loads in flight, added in order
        double v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = __ldcg(part + (long long)(g + j) * 2 * Bp + off + b);
#pragma unroll
        for (int j = 0; j < 8; ++j) s += v[j];
    }
    for (; g < g1; ++g) s += __ldcg(part + (long long)g * 2 * Bp + off + b);
    __syncthreads();
    s_tmp[threadIdx.x] = s;
    __syncthreads();
    double tot = 0.0;
    if ((int)threadIdx.x < Bp)
        for (int qq = 0; qq < Q; ++qq) tot += s_tmp[qq * Bp + threadIdx.x];
    return tot;
}

// Grid-wide barrier: every CTA adds one arrival and waits until all G arrivals of this
// barrier are in (the count is cumulative over the launch: barrier j completes at j G).
// False if the wait ran out or another CTA gave up.
__device__ __forceinline__ bool grid_barrier(const PersistArgs& A, unsigned& epoch) {
    __shared__ int s_ok;
    epoch += gridDim.x;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(A.bar, 1u);
        int ok = 0;
        for (unsigned t = 0; t < PERSIST_POLLS; ++t) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(A.bar) : "memory");
            if (v >= epoch) { ok = 1; break; }
            if (*(volatile int*)A.err) break;
            __nanosleep(64);
        }
        if (!ok) atomicCAS(A.err, 0, 3);
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Grid-wide barrier that also sums the partial rows: the last CTA to arrive (it sees the
// arrival count reach the target) adds part[g][j Bp + b] over g in the fixed order of
// slot_total into tot[j Bp + b] (j < nsum), then releases the others through bar[1]; the
// others wait for the release and read the totals. One CTA reads the G partial rows instead
// of every CTA. False if the wait ran out or another CTA gave up.
__device__ __forceinline__ bool grid_barrier_sum(const PersistArgs& A, unsigned& epoch, int nsum, double* s_tmp) {
    __shared__ int s_last, s_ok;
    epoch += gridDim.x;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned before = atomicAdd(A.bar, 1u);
        s_last = before + 1u == epoch;
        __threadfence();
    }
    __syncthreads();
    if (s_last) {
        for (int j = 0; j < nsum; ++j) {
            const double t = slot_total(A.part, gridDim.x, A.Bp, j * A.Bp, s_tmp);
            if ((int)threadIdx.x < A.Bp) A.tot[j * A.Bp + threadIdx.x] = t;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            asm volatile("st.release.gpu.global.u32 [%0], %1;" :: "l"(A.bar + 1), "r"(epoch) : "memory");
            s_ok = 1;
        }
    } else if (threadIdx.x == 0) {
        int ok = 0;
        for (unsigned t = 0; t < PERSIST_POLLS; ++t) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(A.bar + 1) : "memory");
            if (v >= epoch) { ok = 1; break; }
            if (*(volatile int*)A.err) break;
            __nanosleep(64);
        }
        if (!ok) atomicCAS(A.err, 0, 3);
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// The CTA's per-slot sums (cta_lane_sum order) into its partial row, at offset `off`.
__device__ __forceinline__ void put_partial(const PersistArgs& A, double v, int off, double* s_tmp, double* s_out) {
    cta_lane_sum(v, A.Bp, s_tmp, s_out);
    if ((int)threadIdx.x < A.Bp) A.part[(long long)blockIdx.x * 2 * A.Bp + off + threadIdx.x] = s_out[threadIdx.x];
}

template <int BS>
__global__ void __launch_bounds__(POD2G_THREADS, 2) k_persist(const PersistArgs A) {
    extern __shared__ float s_ec[];  // [Bp][kp + 1]
    __shared__ SlotScalars s_sc[64];
    __shared__ double s_tmp[POD2G_THREADS];
    __shared__ double s_out[64];
    __shared__ double s_cv[POD2G_MAX_K];
    __shared__ int s_any;
    const int Bp = A.Bp, kp = A.kp, G = gridDim.x, tid = threadIdx.x;
    const int lane = tid & (Bp - 1);
    const float w = A.omega;
    for (int b = tid; b < Bp; b += blockDim.x) s_sc[b] = A.sc[b];
    const long long items = (long long)A.nb << A.lgBp;   // (block row, slot) pairs
    const long long elems = (long long)A.n * Bp;         // (unknown, slot) pairs
    const long long stride = (long long)G * blockDim.x;
    const long long first = (long long)blockIdx.x * blockDim.x + tid;
    unsigned epoch = 0;
    bool ok = true;
    for (int iter = 0; iter < A.iters; ++iter) {
        __syncthreads();
        if (tid == 0) {
            int any = 0;
            for (int b = 0; b < Bp; ++b) any |= s_sc[b].state == SLOT_ACTIVE;
            s_any = any;
        }
        __syncthreads();
        if (!s_any) break;  // the same in every CTA
        // ---- A: p = s + beta p (each thread's own elements)
        bool on = s_sc[lane].state == SLOT_ACTIVE;
        if (on) {
            const float2 beta = df_from_double(s_sc[lane].beta);
            for (long long e = first; e < elems; e += stride) A.p[e] = df_add(df_of(A.s[e]), df_mul(beta, A.p[e]));
        }
        if (!(ok = grid_barrier(A, epoch))) break;
        // ---- B: q = K p, partial p^T q
        {
            float dh = 0.f, dl = 0.f;
            if (on) {
                for (long long it = first; it < items; it += stride) {
                    const int i = (int)(it >> A.lgBp);
                    float ah[BS], al[BS];
#pragma unroll
                    for (int a = 0; a < BS; ++a) { ah[a] = 0.f; al[a] = 0.f; }
                    const int b1 = __ldg(A.row_ptr + i + 1);
#pragma unroll 2
                    for (int blk = __ldg(A.row_ptr + i); blk < b1; ++blk) {
                        const int j = __ldg(A.col_idx + blk);
                        const float* vb = A.vals + (long long)blk * BS * BS * Bp + lane;
                        float v[BS * BS];
                        float2 pj[BS];
#pragma unroll
                        for (int e = 0; e < BS * BS; ++e) v[e] = __ldg(vb + e * Bp);
#pragma unroll
                        for (int cc = 0; cc < BS; ++cc) pj[cc] = __ldcg(A.p + ((long long)j * BS + cc) * Bp + lane);
#pragma unroll
                        for (int a = 0; a < BS; ++a)
#pragma unroll
                            for (int cc = 0; cc < BS; ++cc) df_acc_fma(ah[a], al[a], v[a * BS + cc], pj[cc].x, pj[cc].y);
                    }
#pragma unroll
                    for (int a = 0; a < BS; ++a) {
                        const long long o = ((long long)i * BS + a) * Bp + lane;
                        const float2 qv = df_norm(ah[a], al[a]);
                        A.q[o] = qv;
                        const float2 pv = __ldcg(A.p + o);
                        df_acc_fma(dh, dl, pv.x, qv.x, qv.y);
                        dl = __fmaf_rn(pv.y, qv.x, dl);
                    }
                }
            }
            put_partial(A, (double)dh + (double)dl, 0, s_tmp, s_out);
        }
        if (!(ok = grid_barrier_sum(A, epoch, 1, s_tmp))) break;
        // ---- C: alpha, x += alpha p, r -= alpha q
        {
            const double pq = tid < Bp ? __ldcg(A.tot + tid) : 0.0;
            if (tid < Bp) {
                SlotScalars& S = s_sc[tid];
                if (S.state == SLOT_ACTIVE) {
                    if (S.iters >= S.maxit) {
                        S.state = SLOT_DONE; S.result = POD2G_NOT_CONVERGED; S.alpha = 0.0;
                    } else if (!(pq > 0.0) || !isfinite(pq)) {
                        S.state = SLOT_DONE; S.result = isfinite(pq) ? POD2G_BREAKDOWN : POD2G_NONFINITE; S.alpha = 0.0;
                    } else {
                        S.alpha = A.stat ? 1.0 : S.rs / pq;
                        S.iters += 1;
                    }
                }
            }
            __syncthreads();
            on = s_sc[lane].state == SLOT_ACTIVE;
            if (on) {
                const float2 al = df_from_double(s_sc[lane].alpha), nal = df_neg(al);
                for (long long e = first; e < elems; e += stride) {
                    A.x[e] = df_add(A.x[e], df_mul(al, A.p[e]));
                    A.r[e] = df_add(A.r[e], df_mul(nal, __ldcg(A.q + e)));
                }
            }
        }
        if (!(ok = grid_barrier(A, epoch))) break;
        // ---- D: r1 = r - K (omega D^-1 r), partial ||r||^2, partial Phi^T r1 over the CTA's rows
        {
            float rr = 0.f;
            if (on) {
                for (long long it = first; it < items; it += stride) {
                    const int i = (int)(it >> A.lgBp);
                    float acc[BS];
#pragma unroll
                    for (int a = 0; a < BS; ++a) acc[a] = 0.f;
                    const int b1 = __ldg(A.row_ptr + i + 1);
#pragma unroll 2
                    for (int blk = __ldg(A.row_ptr + i); blk < b1; ++blk) {
                        const int j = __ldg(A.col_idx + blk);
                        const float* vb = A.vals + (long long)blk * BS * BS * Bp + lane;
                        float v[BS * BS], y[BS];
#pragma unroll
                        for (int e = 0; e < BS * BS; ++e) v[e] = __ldg(vb + e * Bp);
#pragma unroll
                        for (int cc = 0; cc < BS; ++cc) {
                            const long long o = ((long long)j * BS + cc) * Bp + lane;
                            y[cc] = w * __ldg(A.dinv + o) * __ldcg(reinterpret_cast<const float*>(A.r + o));
                        }
#pragma unroll
                        for (int a = 0; a < BS; ++a)
#pragma unroll
                            for (int cc = 0; cc < BS; ++cc) acc[a] = __fmaf_rn(v[a * BS + cc], y[cc], acc[a]);
                    }
#pragma unroll
                    for (int a = 0; a < BS; ++a) {
                        const long long o = ((long long)i * BS + a) * Bp + lane;
                        const float rv = __ldcg(reinterpret_cast<const float*>(A.r + o));
                        A.r1[o] = rv - acc[a];
                        rr = __fmaf_rn(rv, rv, rr);
                    }
                }
            }
            put_partial(A, (double)rr, 0, s_tmp, s_out);   // ends with __syncthreads: r1 of the CTA's rows visible
            if (kp > 0) {
                // c[b][m] += Phi[d][m] r1[d][b] over the unknowns d of the block rows this CTA
                // covered, in increasing d; thread t owns outputs o = t + 256 u (NO > 256), or
                // output t % NO over every Q-th unknown (NO <= 256, Q = 256 / NO groups,
                // combined in group order)
                const int NO = Bp * kp;
                const int Q = NO >= (int)blockDim.x ? 1 : (int)blockDim.x / NO;
                const int qd = NO >= (int)blockDim.x ? 0 : tid / NO;
                float cacc[PERSIST_OUT];
#pragma unroll
                for (int u = 0; u < PERSIST_OUT; ++u) cacc[u] = 0.f;
                if (qd < Q) {
                    for (long long it0 = (long long)blockIdx.x * blockDim.x; it0 < items; it0 += stride) {
                        const long long d0 = (it0 >> A.lgBp) * BS;
                        const long long d1 = min((it0 + blockDim.x) >> A.lgBp, (long long)A.nb) * BS;
                        for (long long d = d0 + qd; d < d1; d += Q) {
#pragma unroll
                            for (int u = 0; u < PERSIST_OUT; ++u) {
                                const int o = (NO >= (int)blockDim.x ? tid + u * (int)blockDim.x : tid % NO);
                                if ((u == 0 || NO >= (int)blockDim.x) && o < NO) {
                                    const int b = o / kp, m = o - b * kp;
                                    cacc[u] = __fmaf_rn(__ldg(A.phi + d * kp + m), __ldcg(A.r1 + d * Bp + b), cacc[u]);
                                }
                            }
                        }
                    }
                }
                double* cp = A.cpart + (long long)blockIdx.x * NO;
                if (NO >= (int)blockDim.x) {
#pragma unroll
                    for (int u = 0; u < PERSIST_OUT; ++u) {
                        const int o = tid + u * (int)blockDim.x;
                        if (o < NO) cp[o] = (double)cacc[u];
                    }
                } else {
                    s_tmp[tid] = (double)cacc[0];
                    __syncthreads();
                    if (tid < NO) {
                        double t = 0.0;
                        for (int qq = 0; qq < Q; ++qq) t += s_tmp[qq * NO + tid];
                        cp[tid] = t;
                    }
                }
            }
        }
        if (!(ok = grid_barrier_sum(A, epoch, 1, s_tmp))) break;
        // ---- E: convergence test on ||r||^2, coarse solve for the slots b = blockIdx.x (mod G)
        {
            const double rr = tid < Bp ? __ldcg(A.tot + tid) : 0.0;
            if (tid < Bp) {
                SlotScalars& S = s_sc[tid];
                if (S.state == SLOT_ACTIVE) {
                    S.rr = rr;
                    if (!isfinite(rr)) {
                        S.state = SLOT_DONE; S.result = POD2G_NONFINITE;
                    } else if (rr <= S.tol2) {
                        S.state = SLOT_DONE; S.result = POD2G_OK;
                    }
                }
            }
            __syncthreads();
            if (A.k > 0) {
                const int k = A.k;
                for (int b = blockIdx.x; b < Bp; b += G) {
                    if (s_sc[b].state != SLOT_ACTIVE) continue;
                    // c[m] = sum_g cpart[g][b][m]: thread (m, qd) sums a contiguous range of g
                    const int Q = blockDim.x / kp;
                    const int m = tid % kp, qd = tid / kp;
                    double cs = 0.0;
                    if (qd < Q) {
                        const int g0 = (int)((long long)G * qd / Q), g1 = (int)((long long)G * (qd + 1) / Q);
                        int g = g0;
                        for (; g + 8 <= g1; g += 8) {   // eight loads in flight, added in order
                            double v[8];
#pragma unroll
                            for (int j = 0; j < 8; ++j) v[j] = __ldcg(A.cpart + ((long long)(g + j) * Bp + b) * kp + m);
#pragma unroll
                            for (int j = 0; j < 8; ++j) cs += v[j];
                        }
                        for (; g < g1; ++g) cs += __ldcg(A.cpart + ((long long)g * Bp + b) * kp + m);
                    }
                    __syncthreads();
                    s_tmp[tid] = cs;
                    __syncthreads();
                    if (tid < kp) {
                        double t = 0.0;
                        for (int qq = 0; qq < Q; ++qq) t += s_tmp[qq * kp + tid];
                        s_cv[tid] = t;
                    }
                    __syncthreads();
                    const double* L = A.Lc + (long long)b * k * k;
                    if (tid < 32) {
                        for (int i = 0; i < k; ++i) {
                            const double yi = s_cv[i] / L[i * k + i];
                            __syncwarp();
                            if (tid == 0) s_cv[i] = yi;
                            for (int j = i + 1 + tid; j < k; j += 32) s_cv[j] -= L[j * k + i] * yi;
                            __syncwarp();
                        }
                        for (int i = k - 1; i >= 0; --i) {
                            const double ei = s_cv[i] / L[i * k + i];
                            __syncwarp();
                            if (tid == 0) s_cv[i] = ei;
                            for (int j = tid; j < i; j += 32) s_cv[j] -= L[i * k + j] * ei;
                            __syncwarp();
                        }
                        for (int mm = tid; mm < kp; mm += 32) A.ec[(long long)b * kp + mm] = mm < k ? (float)s_cv[mm] : 0.f;
                    }
                    __syncthreads();
                }
            }
        }
        if (!(ok = grid_barrier(A, epoch))) break;
        // ---- F: s = y1 + Phi e_c + omega D^-1 (r1 - (K Phi) e_c), partial r^T s (and r^T s_old)
        {
            for (int e = tid; e < Bp * kp; e += blockDim.x)
                s_ec[(e / kp) * (kp + 1) + e % kp] = s_sc[e / kp].state == SLOT_ACTIVE ? __ldcg(A.ec + e) : 0.f;
            __syncthreads();
            on = s_sc[lane].state == SLOT_ACTIVE;
            float h = 0.f, l = 0.f, xh = 0.f, xl = 0.f;
            if (on) {
                const float* el = s_ec + lane * (kp + 1);
                const long long mstride = (long long)A.n * Bp;
                for (long long e = first; e < elems; e += stride) {
                    const long long d = e >> A.lgBp;
                    const float2 rv = A.r[e];
                    const float dv = __ldg(A.dinv + e);
                    const float so = A.pr ? A.s[e] : 0.f;
                    float y = w * dv * rv.x, y2 = 0.f, t = __ldcg(A.r1 + e), t2 = 0.f;
                    const float* ph = A.phi + d * kp;
                    const float* wr = A.W + e;
                    int m = 0;
                    for (; m + 2 <= kp; m += 2) {
                        const float e0 = el[m], e1 = el[m + 1];
                        y = __fmaf_rn(__ldg(ph + m), e0, y);
                        y2 = __fmaf_rn(__ldg(ph + m + 1), e1, y2);
                        t = __fmaf_rn(-__ldg(wr + m * mstride), e0, t);
                        t2 = __fmaf_rn(-__ldg(wr + (m + 1) * mstride), e1, t2);
                    }
                    for (; m < kp; ++m) {
                        y = __fmaf_rn(__ldg(ph + m), el[m], y);
                        t = __fmaf_rn(-__ldg(wr + m * mstride), el[m], t);
                    }
                    const float sv = __fmaf_rn(w * dv, t + t2, y + y2);
                    if (A.pr) df_acc_fma(xh, xl, so, rv.x, rv.y);
                    A.s[e] = sv;
                    df_acc_fma(h, l, sv, rv.x, rv.y);
                }
            }
            put_partial(A, (double)h + (double)l, 0, s_tmp, s_out);
            if (A.pr) put_partial(A, (double)xh + (double)xl, Bp, s_tmp, s_out);
        }
        if (!(ok = grid_barrier_sum(A, epoch, A.pr ? 2 : 1, s_tmp))) break;
        // ---- beta
        {
            const double rs = tid < Bp ? __ldcg(A.tot + tid) : 0.0;
            const double rsx = A.pr && tid < Bp ? __ldcg(A.tot + Bp + tid) : 0.0;
            if (tid < Bp) {
                SlotScalars& S = s_sc[tid];
                if (S.state == SLOT_ACTIVE) {
                    if (!(rs > 0.0) || !isfinite(rs)) {
                        S.state = SLOT_DONE;
                        S.result = isfinite(rs) ? POD2G_BREAKDOWN : POD2G_NONFINITE;
                    } else {
                        S.beta = (S.first || A.stat) ? 0.0 : (A.pr ? (rs - rsx) / S.rs : rs / S.rs);
                        S.rs = rs;
                        S.first = 0;
                    }
                }
            }
        }
    }
    __syncthreads();
    if (blockIdx.x == 0)
        for (int b = tid; b < Bp; b += blockDim.x) A.sc[b] = s_sc[b];
}

const void* persist_fn(int bs) {
    if (bs == 1) return (const void*)k_persist<1>;
    if (bs == 2) return (const void*)k_persist<2>;
    if (bs == 3) return (const void*)k_persist<3>;
    return nullptr;
}

size_t persist_smem(const pod2g_ctx* c) { return sizeof(float) * (size_t)c->Bp * (c->kp + 1); }

}  // namespace

// The persistent form applies to the mixed-precision assembled Jacobi cycle (r1 = r2 = 1)
// with at most 64 slot lanes, with K Phi stored for the post-smoothing (or no coarse space).
bool persist_applies(const pod2g_ctx* c) {
    return c->precision != POD2G_FP64 && !c->elem && c->smoother == POD2G_SMOOTHER_JACOBI && c->pre == 1 &&
           c->post == 1 && c->Bp <= 64 && c->bs >= 1 && c->bs <= 3 && c->kp <= POD2G_MAX_K &&
           (c->kp == 0 || c->d_W32 != nullptr) && c->Bp * c->kp <= PERSIST_OUT * POD2G_THREADS;
}

// Largest cooperative grid: resident CTAs per SM times the SMs (0 where it does not apply).
int persist_max_grid(pod2g_ctx* c) {
    if (!persist_applies(c)) return 0;
    const void* fn = persist_fn(c->bs);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, POD2G_THREADS, persist_smem(c)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return occ * c->num_sms;
}

// One cooperative launch of up to `iters` iterations for the ACTIVE lanes on c->stream,
// with c->grid_persist CTAs (all resident at once).
int persist_launch(pod2g_ctx* c, int iters) {
    if (!persist_applies(c) || c->grid_persist < 1) return POD2G_INVALID_ARG;
    PersistArgs A;
    A.nb = c->nb;
    A.n = c->n;
    A.Bp = c->Bp;
    A.lgBp = 0;
    while ((1 << A.lgBp) < c->Bp) ++A.lgBp;
    A.k = c->k;
    A.kp = c->kp;
    A.stat = c->method == POD2G_STATIONARY;
    A.pr = c->beta_pr;
    A.iters = iters;
    A.omega = (float)c->omega;
    A.row_ptr = c->d_row_ptr;
    A.col_idx = c->d_col_idx;
    A.vals = c->d_vals32;
    A.dinv = c->d_dinv32;
    A.phi = c->d_phi32;
    A.W = c->d_W32;
    A.Lc = c->d_Lc;
    A.x = c->d_xdf;
    A.r = c->d_rdf;
    A.p = c->d_pdf;
    A.q = c->d_qdf;
    A.s = c->d_s32;
    A.r1 = c->d_y32;
    A.ec = c->d_ec;
    A.part = c->d_part;
    A.tot = c->d_part + (size_t)2 * c->Bp * 4 * c->num_sms;   // after the partial rows of 4 * SMs CTAs
    A.cpart = c->d_cpart;
    A.sc = c->d_sc;
    A.bar = c->d_counters + CNT_PERSIST;
    A.err = c->d_err;
    P2G_CUDA(cudaMemsetAsync(A.bar, 0, 2 * sizeof(unsigned), c->stream));
    void* args[] = {&A};
    P2G_CUDA(cudaLaunchCooperativeKernel(persist_fn(c->bs), dim3(c->grid_persist), dim3(POD2G_THREADS), args,
                                         persist_smem(c), c->stream));
    return POD2G_OK;
}
