// Batched mixed-precision POD-2G-PCG: up to Bp parameter instances ("slots")
// iterate in lockstep over one shared sparsity pattern.
//
// Method: Algorithm 3 of arXiv 2207.02543 (PCG preconditioned by one cycle
// AMG(0; K, r, r1, r2) of the two-grid scheme of Algorithm 2 with P = Phi_r,
// Section 3.3), damped-Jacobi relaxation, r1, r2 in {0, 1}.
//
// Layout: every per-instance vector and the matrix values are slot-interleaved
// (element (row, slot) at row * Bp + slot), so one warp reads 32 instances of the
// same row in one coalesced transaction and the column indices are read once for
// all instances. A thread owns one block row of one slot; the slot of a thread is
// fixed (threadIdx.x % Bp, Bp | blockDim), so a slot's reduction order does not
// depend on the other slots: a result is bit-identical alone and in a mix.
//
// Precision: x, r, p and q = K p are double-float (pairs of FP32, ~48-bit
// significand), because GB300 executes FP64 at ~1/70 of its FP32 rate; the
// preconditioner (smoothing, restriction, prolongation) is FP32; per-slot
// scalars, cross-CTA sums and the coarse Cholesky solve are FP64.
//
// One PCG iteration = 7 kernels, captured `chunk` times in one CUDA graph:
//   k_p      p = s + beta p
//   k_spmv   q = K p, p^T q             (last CTA: alpha = r^T s / p^T q, maxit, breakdown)
//   k_upd    x += alpha p, r -= alpha q
//   k_pre    y1 = omega D^-1 r, r1 = r - K y1, partials of Phi^T r1 and ||r||^2
//   k_coarse per slot: ||r|| test, c = Phi^T r1, e_c = L^-T L^-1 c
//   k_prol   y2 = y1 + Phi e_c
//   k_post   s = y2 + omega D^-1 (r - K y2), r^T s  (last CTA: beta)
#include "common.cuh"

#include <chrono>
#include <cmath>

namespace {

struct Dims {
    int nb, Bp, lgBp, k, kp, G;
    double omega;
};

// p[g0*stride] + ... + p[(g1-1)*stride], added in increasing g (so the result is
// that of the plain serial loop); loads are issued eight at a time.
__device__ __forceinline__ double ordered_sum(const double* __restrict__ p, int g0, int g1, long long stride) {
    double s = 0.0;
    int g = g0;
    for (; g + 8 <= g1; g += 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = p[(long long)(g + u) * stride];
#pragma unroll
        for (int u = 0; u < 8; ++u) s += v[u];
    }
    for (; g < g1; ++g) s += p[(long long)g * stride];
    return s;
}

// sum over the threads of this CTA that own `lane` (thread t owns lane t % Bp),
// in thread order; result to out[lane] for lane < Bp. smem must hold blockDim doubles.
__device__ __forceinline__ void cta_lane_sum(double v, int Bp, double* smem, double* out) {
    __syncthreads();
    smem[threadIdx.x] = v;
    __syncthreads();
    if ((int)threadIdx.x < Bp) {
        double s = 0.0;
        for (int t = threadIdx.x; t < (int)blockDim.x; t += Bp) s += smem[t];
        out[threadIdx.x] = s;
    }
}

// total over CTAs g = 0..G-1 of part[g * stride + lane] (fixed order), computed by
// all threads of one CTA; returns the total in threads t < Bp (t = lane).
__device__ __forceinline__ double grid_lane_total(const double* part, int G, int stride, int Bp, double* smem) {
    const int Q = blockDim.x / Bp;
    const int b = threadIdx.x % Bp, q = threadIdx.x / Bp;
    const int g0 = (int)((long long)G * q / Q), g1 = (int)((long long)G * (q + 1) / Q);
    double s = ordered_sum(part + b, g0, g1, stride);
    __syncthreads();
    smem[threadIdx.x] = s;
    __syncthreads();
    double tot = 0.0;
    if ((int)threadIdx.x < Bp)
        for (int qq = 0; qq < Q; ++qq) tot += smem[qq * Bp + threadIdx.x];
    return tot;
}

__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 df_of(float a) { return make_float2(a, 0.f); }

// ---------------------------------------------------------------------------- load / store / residual
// Joining lanes: b -> bdf, x0 -> xdf (zero if absent), p = q = 0.
__global__ void k_load(const double* __restrict__ b, const double* __restrict__ x0, const int* __restrict__ slots,
                       int nslots, int n, int Bp, float2* __restrict__ bdf, float2* __restrict__ xdf,
                       float2* __restrict__ pdf, float2* __restrict__ qdf, float* __restrict__ s32) {
    long long total = (long long)nslots * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e / n);
        long long d = e - (long long)r * n;
        long long o = d * Bp + slots[r];
        bdf[o] = df_from_double(b[e]);
        xdf[o] = x0 ? df_from_double(x0[e]) : make_float2(0.f, 0.f);
        pdf[o] = make_float2(0.f, 0.f);
        qdf[o] = make_float2(0.f, 0.f);
        s32[o] = 0.f;
    }
}

// x (double-float, lanes) -> FP64 [nslots][n]; zero for b = 0 instances.
__global__ void k_store(double* __restrict__ x, const int* __restrict__ slots, int nslots, int n, int Bp,
                        const float2* __restrict__ xdf, const SlotScalars* __restrict__ sc) {
    long long total = (long long)nslots * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e / n);
        long long d = e - (long long)r * n;
        int lane = slots[r];
        x[e] = sc[lane].bb == 0.0 ? 0.0 : df_to_double(xdf[d * Bp + lane]);
    }
}

// r = b - K x in double-float for masked lanes. init: writes r, sums ||b||^2 and
// sets tol2 = tol^2 ||b||^2 (b = 0 or non-finite -> DONE). final: sums
// ||b - K x||^2 into relres.
template <int BS>
__global__ void __launch_bounds__(POD2G_THREADS) k_resid(Dims D, int final_mode, const int* __restrict__ mask,
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx, const float* __restrict__ vals,
    const float2* __restrict__ x, const float2* __restrict__ b, float2* __restrict__ r, double* part,
    unsigned* counter, SlotScalars* sc) {
    __shared__ double smem[POD2G_THREADS];
    const int lane = threadIdx.x & (D.Bp - 1);
    const bool on = mask[lane] != 0;
    float bh = 0.f, bl = 0.f, rh = 0.f, rl = 0.f;
    if (on) {
        const long long items = (long long)D.nb << D.lgBp;
        for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
             it += (long long)gridDim.x * blockDim.x) {
            const int i = (int)(it >> D.lgBp);
            float ah[BS], al[BS];
#pragma unroll
            for (int a = 0; a < BS; ++a) { ah[a] = 0.f; al[a] = 0.f; }
            for (int blk = row_ptr[i]; blk < row_ptr[i + 1]; ++blk) {
                const int j = col_idx[blk];
                float2 xj[BS];
#pragma unroll
                for (int cc = 0; cc < BS; ++cc) xj[cc] = x[((long long)j * BS + cc) * D.Bp + lane];
#pragma unroll
                for (int a = 0; a < BS; ++a)
#pragma unroll
                    for (int cc = 0; cc < BS; ++cc)
                        df_acc_fma(ah[a], al[a], vals[((long long)blk * BS * BS + a * BS + cc) * D.Bp + lane],
                                   xj[cc].x, xj[cc].y);
            }
#pragma unroll
            for (int a = 0; a < BS; ++a) {
                const long long o = ((long long)i * BS + a) * D.Bp + lane;
                float2 bv = b[o];
                float2 rv = df_add(bv, df_neg(df_norm(ah[a], al[a])));
                if (!final_mode) r[o] = rv;
                df_acc_fma(bh, bl, bv.x, bv.x, 2.f * bv.y);
                df_acc_fma(rh, rl, rv.x, rv.x, 2.f * rv.y);
            }
        }
    }
    double* pg = part + (long long)blockIdx.x * D.Bp * 2;
    cta_lane_sum((double)bh + (double)bl, D.Bp, smem, pg);
    cta_lane_sum((double)rh + (double)rl, D.Bp, smem, pg + D.Bp);
    if (!last_cta_arrive(counter)) return;
    double bb = grid_lane_total(part, D.G, 2 * D.Bp, D.Bp, smem);
    double rr = grid_lane_total(part + D.Bp, D.G, 2 * D.Bp, D.Bp, smem);
    if ((int)threadIdx.x < D.Bp && mask[threadIdx.x]) {
        SlotScalars& s = sc[threadIdx.x];
        if (final_mode) {
            s.relres = s.bb > 0.0 ? sqrt(rr / s.bb) : 0.0;
        } else {
            s.bb = bb;
            s.tol2 = s.tol2 * bb;  // host stored tol^2
            if (bb == 0.0) {
                s.state = SLOT_DONE; s.result = POD2G_OK; s.iters = 0;
            } else if (!isfinite(bb) || !isfinite(rr)) {
                s.state = SLOT_DONE; s.result = POD2G_NONFINITE;
            }
        }
    }
    last_cta_reset(counter);
}

// ---------------------------------------------------------------------------- PCG kernels
// p = s + beta p (double-float)
__global__ void k_p(Dims D, int want, const float* __restrict__ s, float2* __restrict__ p,
                    const SlotScalars* __restrict__ sc, long long total) {
    const int lane = threadIdx.x & (D.Bp - 1);
    if (sc[lane].state != want) return;
    const float2 beta = df_from_double(sc[lane].beta);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x)
        p[e] = df_add(df_of(s[e]), df_mul(beta, p[e]));
}

// q = K p (double-float), partial p^T q; last CTA: alpha per slot.
template <int BS>
__global__ void __launch_bounds__(POD2G_THREADS) k_spmv(Dims D, int want,
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx, const float* __restrict__ vals,
    const float2* __restrict__ p, float2* __restrict__ q, double* part, unsigned* counter, SlotScalars* sc) {
    __shared__ double smem[POD2G_THREADS];
    const int lane = threadIdx.x & (D.Bp - 1);
    const bool on = sc[lane].state == want;
    float dh = 0.f, dl = 0.f;
    if (on) {
        const long long items = (long long)D.nb << D.lgBp;
        for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
             it += (long long)gridDim.x * blockDim.x) {
            const int i = (int)(it >> D.lgBp);
            float ah[BS], al[BS];
#pragma unroll
            for (int a = 0; a < BS; ++a) { ah[a] = 0.f; al[a] = 0.f; }
            const int b0 = row_ptr[i], b1 = row_ptr[i + 1];
            for (int blk = b0; blk < b1; ++blk) {
                const int j = col_idx[blk];
                float2 pj[BS];
#pragma unroll
                for (int cc = 0; cc < BS; ++cc) pj[cc] = p[((long long)j * BS + cc) * D.Bp + lane];
                const float* vb = vals + (long long)blk * BS * BS * D.Bp + lane;
#pragma unroll
                for (int a = 0; a < BS; ++a)
#pragma unroll
                    for (int cc = 0; cc < BS; ++cc)
                        df_acc_fma(ah[a], al[a], vb[(a * BS + cc) * D.Bp], pj[cc].x, pj[cc].y);
            }
#pragma unroll
            for (int a = 0; a < BS; ++a) {
                const long long o = ((long long)i * BS + a) * D.Bp + lane;
                float2 qv = df_norm(ah[a], al[a]);
                q[o] = qv;
                float2 pv = p[o];
                // p^T q: exact pv.x * qv.x plus the cross terms
                df_acc_fma(dh, dl, pv.x, qv.x, qv.y);
                dl = __fmaf_rn(pv.y, qv.x, dl);
            }
        }
    }
    cta_lane_sum((double)dh + (double)dl, D.Bp, smem, part + (long long)blockIdx.x * D.Bp * 2);
    if (!last_cta_arrive(counter)) return;
    double pq = grid_lane_total(part, D.G, 2 * D.Bp, D.Bp, smem);
    if ((int)threadIdx.x < D.Bp) {
        SlotScalars& s = sc[threadIdx.x];
        if (s.state == want) {
            if (s.iters >= s.maxit) {
                s.state = SLOT_DONE; s.result = POD2G_NOT_CONVERGED; s.alpha = 0.0;
            } else if (!(pq > 0.0) || !isfinite(pq)) {
                s.state = SLOT_DONE; s.result = isfinite(pq) ? POD2G_BREAKDOWN : POD2G_NONFINITE; s.alpha = 0.0;
            } else {
                s.alpha = s.rs / pq;
                s.iters += 1;
            }
        }
    }
    last_cta_reset(counter);
}

// x += alpha p, r -= alpha q (double-float, elementwise)
__global__ void k_upd(Dims D, int want, float2* __restrict__ x, float2* __restrict__ r,
                      const float2* __restrict__ p, const float2* __restrict__ q,
                      const SlotScalars* __restrict__ sc, long long total) {
    const int lane = threadIdx.x & (D.Bp - 1);
    if (sc[lane].state != want) return;
    const float2 al = df_from_double(sc[lane].alpha);
    const float2 nal = df_neg(al);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        x[e] = df_add(x[e], df_mul(al, p[e]));
        r[e] = df_add(r[e], df_mul(nal, q[e]));
    }
}

// Pre-relaxation from zero and restriction: y1 = omega D^-1 r (r1 = 1) or 0 (r1 = 0),
// r1 = r - K y1, partial sums of c = Phi^T r1 and of ||r||^2.
template <int BS, int KP>
__global__ void __launch_bounds__(POD2G_THREADS) k_pre(Dims D, int want, int PRE,
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx, const float* __restrict__ vals,
    const float* __restrict__ dinv, const float2* __restrict__ r, const float* __restrict__ phi,
    double* part, double* cpart, const SlotScalars* __restrict__ sc) {
    extern __shared__ float red[];  // [blockDim][kp + 1]
    __shared__ double smem[POD2G_THREADS];
    const int lane = threadIdx.x & (D.Bp - 1);
    const bool on = sc[lane].state == want;
    const int kp = KP, ks = KP + 1;
    float cacc[KP > 0 ? KP : 1];
#pragma unroll
    for (int m = 0; m < (KP > 0 ? KP : 1); ++m) cacc[m] = 0.f;
    float rr = 0.f;
    const float w = (float)D.omega;
    if (on) {
        const long long items = (long long)D.nb << D.lgBp;
        for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
             it += (long long)gridDim.x * blockDim.x) {
            const int i = (int)(it >> D.lgBp);
            float acc[BS];
#pragma unroll
            for (int a = 0; a < BS; ++a) acc[a] = 0.f;
            if (PRE) {
                for (int blk = row_ptr[i]; blk < row_ptr[i + 1]; ++blk) {
                    const int j = col_idx[blk];
                    float yj[BS];
#pragma unroll
                    for (int cc = 0; cc < BS; ++cc) {
                        const long long o = ((long long)j * BS + cc) * D.Bp + lane;
                        yj[cc] = w * dinv[o] * r[o].x;
                    }
                    const float* vb = vals + (long long)blk * BS * BS * D.Bp + lane;
#pragma unroll
                    for (int a = 0; a < BS; ++a)
#pragma unroll
                        for (int cc = 0; cc < BS; ++cc) acc[a] = __fmaf_rn(vb[(a * BS + cc) * D.Bp], yj[cc], acc[a]);
                }
            }
#pragma unroll
            for (int a = 0; a < BS; ++a) {
                const long long d = (long long)i * BS + a;
                const float2 rv = r[d * D.Bp + lane];
                const float r1 = rv.x - acc[a];
                rr = __fmaf_rn(rv.x, rv.x, rr);
                const float4* ph = reinterpret_cast<const float4*>(phi + d * KP);
#pragma unroll
                for (int m4 = 0; m4 < KP / 4; ++m4) {
                    float4 f = ph[m4];
                    cacc[4 * m4 + 0] = __fmaf_rn(f.x, r1, cacc[4 * m4 + 0]);
                    cacc[4 * m4 + 1] = __fmaf_rn(f.y, r1, cacc[4 * m4 + 1]);
                    cacc[4 * m4 + 2] = __fmaf_rn(f.z, r1, cacc[4 * m4 + 2]);
                    cacc[4 * m4 + 3] = __fmaf_rn(f.w, r1, cacc[4 * m4 + 3]);
                }
            }
        }
    }
    // per-slot CTA sums: ||r||^2 and the kp restriction components
    cta_lane_sum((double)rr, D.Bp, smem, part + (long long)blockIdx.x * D.Bp * 2);
    if (KP == 0) return;
#pragma unroll
    for (int m = 0; m < (KP > 0 ? KP : 1); ++m) red[threadIdx.x * ks + m] = cacc[m];
    __syncthreads();
    double* cp = cpart + (long long)blockIdx.x * D.Bp * kp;
    for (int o = threadIdx.x; o < D.Bp * kp; o += blockDim.x) {
        const int b = o / kp, m = o - b * kp;
        double s = 0.0;
        for (int t = b; t < (int)blockDim.x; t += D.Bp) s += (double)red[t * ks + m];
        cp[o] = s;
    }
}

// One CTA per slot: convergence test on ||r||^2, coarse right-hand side
// c = Phi^T r1 (sum over CTAs in order), e_c = L^-T L^-1 c in FP64.
__global__ void k_coarse(Dims D, int want, int init, const double* __restrict__ part,
                         const double* __restrict__ cpart, const double* __restrict__ Lc, float* __restrict__ ec,
                         SlotScalars* sc) {
    __shared__ double smem[POD2G_THREADS];
    __shared__ double cv[POD2G_MAX_K];
    __shared__ int go;
    const int b = blockIdx.x;
    if (sc[b].state != want) return;
    // ||r||^2 over CTAs: contiguous ranges per thread, then a fixed tree
    {
        const int T = blockDim.x;
        const int g0 = (int)((long long)D.G * threadIdx.x / T), g1 = (int)((long long)D.G * (threadIdx.x + 1) / T);
        smem[threadIdx.x] = ordered_sum(part + b, g0, g1, (long long)D.Bp * 2);
        __syncthreads();
        for (int h = T / 2; h > 0; h >>= 1) {
            if ((int)threadIdx.x < h) smem[threadIdx.x] += smem[threadIdx.x + h];
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        double rr = smem[0];
        SlotScalars& S = sc[b];
        S.rr = rr;
        go = 1;
        if (!isfinite(rr)) {
            S.state = SLOT_DONE; S.result = POD2G_NONFINITE; go = 0;
        } else if (rr <= S.tol2) {
            S.state = SLOT_DONE; S.result = POD2G_OK; go = 0;
        }
    }
    __syncthreads();
    if (!go || D.k == 0) return;
    // c[m] = sum_g cpart[g][b][m]: thread (m, q) sums a contiguous range of g
    const int kp = D.kp;
    const int Q = blockDim.x / kp;
    const int m = threadIdx.x % kp, q = threadIdx.x / kp;
    double cs = 0.0;
    if (q < Q) {
        const int g0 = (int)((long long)D.G * q / Q), g1 = (int)((long long)D.G * (q + 1) / Q);
        cs = ordered_sum(cpart + (long long)b * kp + m, g0, g1, (long long)D.Bp * kp);
    }
    __syncthreads();
    smem[threadIdx.x] = cs;
    __syncthreads();
    if ((int)threadIdx.x < kp) {
        double t = 0.0;
        for (int qq = 0; qq < Q; ++qq) t += smem[qq * kp + threadIdx.x];
        cv[threadIdx.x] = t;
    }
    __syncthreads();
    const int k = D.k;
    const double* L = Lc + (long long)b * k * k;
    if (threadIdx.x < 32) {
        const int l = threadIdx.x;
        for (int i = 0; i < k; ++i) {
            double yi = cv[i] / L[i * k + i];
            __syncwarp();
            if (l == 0) cv[i] = yi;
            for (int j = i + 1 + l; j < k; j += 32) cv[j] -= L[j * k + i] * yi;
            __syncwarp();
        }
        for (int i = k - 1; i >= 0; --i) {
            double ei = cv[i] / L[i * k + i];
            __syncwarp();
            if (l == 0) cv[i] = ei;
            for (int j = l; j < i; j += 32) cv[j] -= L[i * k + j] * ei;
            __syncwarp();
        }
        for (int mm = l; mm < kp; mm += 32) ec[(long long)b * kp + mm] = mm < k ? (float)cv[mm] : 0.f;
    }
    (void)init;
}

// y2 = y1 + Phi e_c with y1 = omega D^-1 r (r1 = 1) or 0
template <int PRE>
__global__ void k_prol(Dims D, int want, const float* __restrict__ dinv, const float2* __restrict__ r,
                       const float* __restrict__ phi, const float* __restrict__ ec, float* __restrict__ y,
                       const SlotScalars* __restrict__ sc, long long n) {
    extern __shared__ float s_ec[];  // [Bp][kp + 1] (odd row stride: no bank conflicts across slots)
    for (int e = threadIdx.x; e < D.Bp * D.kp; e += blockDim.x) s_ec[(e / D.kp) * (D.kp + 1) + e % D.kp] = ec[e];
    __syncthreads();
    const int lane = threadIdx.x & (D.Bp - 1);
    if (sc[lane].state != want) return;
    const float w = (float)D.omega;
    const int kp = D.kp;
    const float* el = s_ec + lane * (kp + 1);
    const long long items = n << D.lgBp;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
         it += (long long)gridDim.x * blockDim.x) {
        const long long d = it >> D.lgBp;
        float v = PRE ? w * dinv[it] * r[it].x : 0.f;
        const float4* ph = reinterpret_cast<const float4*>(phi + d * kp);
        for (int m4 = 0; m4 < kp / 4; ++m4) {
            float4 f = ph[m4];
            v = __fmaf_rn(f.x, el[4 * m4 + 0], v);
            v = __fmaf_rn(f.y, el[4 * m4 + 1], v);
            v = __fmaf_rn(f.z, el[4 * m4 + 2], v);
            v = __fmaf_rn(f.w, el[4 * m4 + 3], v);
        }
        y[it] = v;
    }
}

// s = y2 + omega D^-1 (r - K y2) (r2 = 1) or y2 (r2 = 0); partial r^T s (and
// r^T s_old for Polak-Ribiere); last CTA: beta, JOINING -> ACTIVE.
template <int BS, int POST>
__global__ void __launch_bounds__(POD2G_THREADS) k_post(Dims D, int want, int pr,
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx, const float* __restrict__ vals,
    const float* __restrict__ dinv, const float2* __restrict__ r, const float* __restrict__ y, float* __restrict__ s,
    double* part, unsigned* counter, SlotScalars* sc) {
    __shared__ double smem[POD2G_THREADS];
    const int lane = threadIdx.x & (D.Bp - 1);
    const bool on = sc[lane].state == want;
    float h = 0.f, l = 0.f, xh = 0.f, xl = 0.f;
    const float w = (float)D.omega;
    if (on) {
        const long long items = (long long)D.nb << D.lgBp;
        for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
             it += (long long)gridDim.x * blockDim.x) {
            const int i = (int)(it >> D.lgBp);
            float acc[BS];
#pragma unroll
            for (int a = 0; a < BS; ++a) acc[a] = 0.f;
            if (POST) {
                for (int blk = row_ptr[i]; blk < row_ptr[i + 1]; ++blk) {
                    const int j = col_idx[blk];
                    float yj[BS];
#pragma unroll
                    for (int cc = 0; cc < BS; ++cc) yj[cc] = y[((long long)j * BS + cc) * D.Bp + lane];
                    const float* vb = vals + (long long)blk * BS * BS * D.Bp + lane;
#pragma unroll
                    for (int a = 0; a < BS; ++a)
#pragma unroll
                        for (int cc = 0; cc < BS; ++cc) acc[a] = __fmaf_rn(vb[(a * BS + cc) * D.Bp], yj[cc], acc[a]);
                }
            }
#pragma unroll
            for (int a = 0; a < BS; ++a) {
                const long long o = ((long long)i * BS + a) * D.Bp + lane;
                const float2 rv = r[o];
                const float yv = y[o];
                const float sv = POST ? __fmaf_rn(w * dinv[o], rv.x - acc[a], yv) : yv;
                if (pr) {
                    const float so = s[o];
                    df_acc_fma(xh, xl, so, rv.x, rv.y);
                }
                s[o] = sv;
                df_acc_fma(h, l, sv, rv.x, rv.y);
            }
        }
    }
    double* pg = part + (long long)blockIdx.x * D.Bp * 2;
    cta_lane_sum((double)h + (double)l, D.Bp, smem, pg);
    if (pr) cta_lane_sum((double)xh + (double)xl, D.Bp, smem, pg + D.Bp);
    if (!last_cta_arrive(counter)) return;
    double rs = grid_lane_total(part, D.G, 2 * D.Bp, D.Bp, smem);
    double rsx = pr ? grid_lane_total(part + D.Bp, D.G, 2 * D.Bp, D.Bp, smem) : 0.0;
    if ((int)threadIdx.x < D.Bp) {
        SlotScalars& S = sc[threadIdx.x];
        if (S.state == want) {
            if (!(rs > 0.0) || !isfinite(rs)) {
                S.state = SLOT_DONE;
                S.result = isfinite(rs) ? POD2G_BREAKDOWN : POD2G_NONFINITE;
            } else {
                S.beta = S.first ? 0.0 : (pr ? (rs - rsx) / S.rs : rs / S.rs);
                S.rs = rs;
                S.first = 0;
                if (want == SLOT_JOINING) S.state = SLOT_ACTIVE;
            }
        }
    }
    last_cta_reset(counter);
}

}  // namespace

// ---------------------------------------------------------------------------- host side
static Dims dims_of(pod2g_ctx* c) {
    Dims D;
    D.nb = c->nb;
    D.Bp = c->Bp;
    D.lgBp = 0;
    while ((1 << D.lgBp) < c->Bp) ++D.lgBp;
    D.k = c->k;
    D.kp = c->kp;
    D.G = c->grid_rows;
    D.omega = c->omega;
    return D;
}

#define LAUNCH_BS(KERNEL, ...)                                                         \
    do {                                                                               \
        if (c->bs == 1) KERNEL<1> __VA_ARGS__;                                         \
        else if (c->bs == 2) KERNEL<2> __VA_ARGS__;                                    \
        else KERNEL<3> __VA_ARGS__;                                                    \
    } while (0)

#define KP_LIST(X, BS) X(BS, 0) X(BS, 8) X(BS, 16) X(BS, 24) X(BS, 32) X(BS, 40) X(BS, 48) X(BS, 64)

template <int BS, int KP>
static const void* pre_fn() { return (const void*)k_pre<BS, KP>; }

template <int BS>
static void launch_pre(pod2g_ctx* c, Dims D, int want) {
    dim3 g(D.G), t(POD2G_THREADS);
    size_t sm = c->smem_pre;
#define CASE_KP(BS_, KP_)                                                                                  \
    case KP_:                                                                                              \
        k_pre<BS_, KP_><<<g, t, sm, c->stream>>>(D, want, c->pre, c->d_row_ptr, c->d_col_idx, c->d_vals32, \
                                                 c->d_dinv32, c->d_rdf, c->d_phi32, c->d_part, c->d_cpart,  \
                                                 c->d_sc);                                                 \
        break;
    switch (c->kp) { KP_LIST(CASE_KP, BS) }
#undef CASE_KP
}

template <int BS>
static void launch_post(pod2g_ctx* c, Dims D, int want) {
    dim3 g(D.G), t(POD2G_THREADS);
    if (c->post)
        k_post<BS, 1><<<g, t, 0, c->stream>>>(D, want, c->beta_pr, c->d_row_ptr, c->d_col_idx, c->d_vals32,
                                              c->d_dinv32, c->d_rdf, c->d_y32, c->d_s32, c->d_part,
                                              c->d_counters + CNT_POST, c->d_sc);
    else
        k_post<BS, 0><<<g, t, 0, c->stream>>>(D, want, c->beta_pr, c->d_row_ptr, c->d_col_idx, c->d_vals32,
                                              c->d_dinv32, c->d_rdf, c->d_y32, c->d_s32, c->d_part,
                                              c->d_counters + CNT_POST, c->d_sc);
}

// Event-record node after a kernel of a captured iteration (timing mode only).
static int mark(pod2g_ctx* c) {
    P2G_TRY(pod2g_check_launch(c));
    if (c->cap_ev) P2G_CUDA(cudaEventRecordWithFlags(c->cap_ev[c->cap_idx++], c->stream, cudaEventRecordExternal));
    return POD2G_OK;
}

// the preconditioner s = AMG(0; K, r, r1, r2) for lanes in state `want`
static int enqueue_precond(pod2g_ctx* c, Dims D, int want) {
    const long long n = c->n;
    if (c->bs == 1) launch_pre<1>(c, D, want);
    else if (c->bs == 2) launch_pre<2>(c, D, want);
    else launch_pre<3>(c, D, want);
    P2G_TRY(mark(c));
    k_coarse<<<c->Bp, POD2G_THREADS, 0, c->stream>>>(D, want, want == SLOT_JOINING, c->d_part, c->d_cpart, c->d_Lc,
                                                     c->d_ec, c->d_sc);
    P2G_TRY(mark(c));
    size_t sm = sizeof(float) * c->Bp * (c->kp + 1);
    int gp = std::max(1, std::min(D.G, ceil_div(n * c->Bp, POD2G_THREADS)));
    if (c->pre)
        k_prol<1><<<gp, POD2G_THREADS, sm, c->stream>>>(D, want, c->d_dinv32, c->d_rdf, c->d_phi32, c->d_ec, c->d_y32,
                                                        c->d_sc, n);
    else
        k_prol<0><<<gp, POD2G_THREADS, sm, c->stream>>>(D, want, c->d_dinv32, c->d_rdf, c->d_phi32, c->d_ec, c->d_y32,
                                                        c->d_sc, n);
    P2G_TRY(mark(c));
    if (c->bs == 1) launch_post<1>(c, D, want);
    else if (c->bs == 2) launch_post<2>(c, D, want);
    else launch_post<3>(c, D, want);
    P2G_TRY(mark(c));
    return POD2G_OK;
}

// one PCG iteration (Algorithm 3 loop body) for ACTIVE lanes
static int enqueue_iteration(pod2g_ctx* c, Dims D) {
    const long long total = (long long)c->n * c->Bp;
    const int ge = std::max(1, std::min(D.G, ceil_div(total, POD2G_THREADS)));
    if (c->cap_ev) P2G_CUDA(cudaEventRecordWithFlags(c->cap_ev[c->cap_idx++], c->stream, cudaEventRecordExternal));
    k_p<<<ge, POD2G_THREADS, 0, c->stream>>>(D, SLOT_ACTIVE, c->d_s32, c->d_pdf, c->d_sc, total);
    P2G_TRY(mark(c));
    LAUNCH_BS(k_spmv, <<<D.G, POD2G_THREADS, 0, c->stream>>>(D, SLOT_ACTIVE, c->d_row_ptr, c->d_col_idx, c->d_vals32,
                                                             c->d_pdf, c->d_qdf, c->d_part,
                                                             c->d_counters + CNT_SPMV, c->d_sc));
    P2G_TRY(mark(c));
    k_upd<<<ge, POD2G_THREADS, 0, c->stream>>>(D, SLOT_ACTIVE, c->d_xdf, c->d_rdf, c->d_pdf, c->d_qdf, c->d_sc, total);
    P2G_TRY(mark(c));
    return enqueue_precond(c, D, SLOT_ACTIVE);
}

int batched_alloc(pod2g_ctx* c) {
    int dev = c->device;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    c->num_sms = sms > 0 ? sms : 152;
    const long long items = (long long)c->nb * c->Bp;
    c->grid_rows = std::max(1, std::min(ceil_div(items, POD2G_THREADS), 4 * c->num_sms));
    c->smem_pre = POD2G_THREADS * (c->kp + 1) * (int)sizeof(float);
    if (c->precision != POD2G_FP64) {
        const void* f = nullptr;
#define FN_KP(BS_, KP_) if (c->bs == BS_ && c->kp == KP_) f = pre_fn<BS_, KP_>();
        KP_LIST(FN_KP, 1) KP_LIST(FN_KP, 2) KP_LIST(FN_KP, 3)
#undef FN_KP
        if (!f) return POD2G_INVALID_ARG;
        P2G_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, c->smem_pre));
    }
    return POD2G_OK;
}

// Load nslots right-hand sides (and optional x0) into the given lanes, set the
// per-slot scalars and run r0 = b - K x0 plus the first preconditioner pass.
int batched_load(pod2g_ctx* c, int nslots, const int* slots, const double* b_dev, const double* x0_dev,
                 const double* tol, const int* maxit) {
    Dims D = dims_of(c);
    int* d_slots = (int*)(c->d_mask + c->Bp);
    P2G_CUDA(cudaMemcpyAsync(d_slots, slots, sizeof(int) * nslots, cudaMemcpyHostToDevice, c->stream));
    std::vector<int> mask(c->Bp, 0);
    for (int i = 0; i < nslots; ++i) mask[slots[i]] = 1;
    // per-slot scalars: host mirror is the source for the joining lanes
    P2G_CUDA(cudaMemcpyAsync(c->h_sc, c->d_sc, sizeof(SlotScalars) * c->Bp, cudaMemcpyDeviceToHost, c->stream));
    P2G_CUDA(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < nslots; ++i) {
        SlotScalars& s = c->h_sc[slots[i]];
        s = SlotScalars();
        s.state = SLOT_JOINING;
        s.result = POD2G_NOT_CONVERGED;
        s.tol2 = tol[i] * tol[i];
        s.maxit = maxit[i];
        s.first = 1;
    }
    P2G_CUDA(cudaMemcpyAsync(c->d_mask, mask.data(), sizeof(int) * c->Bp, cudaMemcpyHostToDevice, c->stream));
    P2G_CUDA(cudaMemcpyAsync(c->d_sc, c->h_sc, sizeof(SlotScalars) * c->Bp, cudaMemcpyHostToDevice, c->stream));
    const long long tot = (long long)nslots * c->n;
    k_load<<<std::max(1, std::min(ceil_div(tot, POD2G_THREADS), 8 * c->num_sms)), POD2G_THREADS, 0, c->stream>>>(
        b_dev, x0_dev, d_slots, nslots, c->n, c->Bp, c->d_bdf, c->d_xdf, c->d_pdf, c->d_qdf, c->d_s32);
    P2G_TRY(pod2g_check_launch(c));
    LAUNCH_BS(k_resid, <<<D.G, POD2G_THREADS, 0, c->stream>>>(D, 0, c->d_mask, c->d_row_ptr, c->d_col_idx,
                                                              c->d_vals32, c->d_xdf, c->d_bdf, c->d_rdf, c->d_part,
                                                              c->d_counters + CNT_RESID, c->d_sc));
    P2G_TRY(pod2g_check_launch(c));
    // s0 = AMG(0; K, r0, r1, r2), convergence test at k = 0, rs0; JOINING -> ACTIVE
    return enqueue_precond(c, D, SLOT_JOINING);
}

static int build_graph(pod2g_ctx* c) {
    if (c->graph_exec) return POD2G_OK;
    Dims D = dims_of(c);
    cudaGraph_t g;
    if (c->timing && c->tev.empty()) {
        c->tev.resize((size_t)c->chunk * 8);
        for (auto& ev : c->tev) P2G_CUDA(cudaEventCreate(&ev));
    }
    P2G_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int st = POD2G_OK;
    for (int it = 0; it < c->chunk && st == POD2G_OK; ++it) {
        c->cap_ev = c->timing ? &c->tev[(size_t)it * 8] : nullptr;
        c->cap_idx = 0;
        st = enqueue_iteration(c, D);
    }
    c->cap_ev = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (st != POD2G_OK) return st;
    P2G_CUDA(e);
    e = cudaGraphInstantiate(&c->graph_exec, g, 0);
    cudaGraphDestroy(g);
    P2G_CUDA(e);
    c->launches -= (int64_t)7 * c->chunk;  // captured, not launched; counted at each replay
    return POD2G_OK;
}

// One CUDA-graph launch (`chunk` PCG iterations for the ACTIVE lanes), then the
// per-slot scalars are copied back to the host mirror.
int batched_chunk(pod2g_ctx* c) {
    P2G_TRY(build_graph(c));
    P2G_CUDA(cudaGraphLaunch(c->graph_exec, c->stream));
    c->launches += (int64_t)7 * c->chunk;
    P2G_CUDA(cudaMemcpyAsync(c->h_sc, c->d_sc, sizeof(SlotScalars) * c->Bp, cudaMemcpyDeviceToHost, c->stream));
    P2G_CUDA(cudaStreamSynchronize(c->stream));
    if (c->timing) {
        for (int it = 0; it < c->chunk; ++it)
            for (int j = 0; j < 7; ++j) {
                float ms = 0.f;
                P2G_CUDA(cudaEventElapsedTime(&ms, c->tev[(size_t)it * 8 + j], c->tev[(size_t)it * 8 + j + 1]));
                c->kt_ms[j] += ms;
                c->kt_n[j] += 1;
            }
    }
    return POD2G_OK;
}

// Per-kernel timing of the captured iterations: on/off (rebuilds the graph).
int batched_set_timing(pod2g_ctx* c, int on) {
    if (c->precision == POD2G_FP64) return POD2G_INVALID_ARG;
    if (c->graph_exec) {
        cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = nullptr;
    }
    c->timing = on != 0;
    for (int j = 0; j < 8; ++j) { c->kt_ms[j] = 0.0; c->kt_n[j] = 0; }
    return POD2G_OK;
}

// Run chunks until every lane in `lanes` is DONE. Bounded: each ACTIVE lane
// finishes within maxit iterations, so at most max(maxit)/chunk + 1 launches.
int batched_run(pod2g_ctx* c, const std::vector<int>& lanes) {
    P2G_CUDA(cudaMemcpyAsync(c->h_sc, c->d_sc, sizeof(SlotScalars) * c->Bp, cudaMemcpyDeviceToHost, c->stream));
    P2G_CUDA(cudaStreamSynchronize(c->stream));
    int64_t bound = 2;
    for (int b : lanes) bound = std::max<int64_t>(bound, (int64_t)c->h_sc[b].maxit / c->chunk + 2);
    if (c->spin_limit > 0) bound = std::min<int64_t>(bound, c->spin_limit);
    for (int64_t polls = 0;; ++polls) {
        bool all = true;
        for (int b : lanes) all = all && c->h_sc[b].state == SLOT_DONE;
        if (all) return POD2G_OK;
        if (polls >= bound) return POD2G_TIMEOUT;
        P2G_TRY(batched_chunk(c));
    }
}

// true residual for the finished lanes, x out, per-slot results
int batched_finalize(pod2g_ctx* c, int nslots, const int* slots, double* x_dev, int* iters, double* relres,
                     int* status) {
    Dims D = dims_of(c);
    std::vector<int> mask(c->Bp, 0);
    for (int i = 0; i < nslots; ++i) mask[slots[i]] = 1;
    int* d_slots = (int*)(c->d_mask + c->Bp);
    P2G_CUDA(cudaMemcpyAsync(c->d_mask, mask.data(), sizeof(int) * c->Bp, cudaMemcpyHostToDevice, c->stream));
    P2G_CUDA(cudaMemcpyAsync(d_slots, slots, sizeof(int) * nslots, cudaMemcpyHostToDevice, c->stream));
    LAUNCH_BS(k_resid, <<<D.G, POD2G_THREADS, 0, c->stream>>>(D, 1, c->d_mask, c->d_row_ptr, c->d_col_idx,
                                                              c->d_vals32, c->d_xdf, c->d_bdf, c->d_rdf, c->d_part,
                                                              c->d_counters + CNT_RESID, c->d_sc));
    P2G_TRY(pod2g_check_launch(c));
    const long long tot = (long long)nslots * c->n;
    k_store<<<std::max(1, std::min(ceil_div(tot, POD2G_THREADS), 8 * c->num_sms)), POD2G_THREADS, 0, c->stream>>>(
        x_dev, d_slots, nslots, c->n, c->Bp, c->d_xdf, c->d_sc);
    P2G_TRY(pod2g_check_launch(c));
    P2G_CUDA(cudaMemcpyAsync(c->h_sc, c->d_sc, sizeof(SlotScalars) * c->Bp, cudaMemcpyDeviceToHost, c->stream));
    P2G_CUDA(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < nslots; ++i) {
        const SlotScalars& s = c->h_sc[slots[i]];
        if (iters) iters[i] = s.iters;
        if (relres) relres[i] = s.relres;
        if (status) status[i] = s.state == SLOT_DONE ? s.result : POD2G_NOT_CONVERGED;
    }
    return POD2G_OK;
}
