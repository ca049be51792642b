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
// The sparse row kernels are memory-latency bound unless many loads are in
// flight: each thread fetches the column indices, values and gathered vector
// entries of UNROLL blocks before using any of them, and the grids fill every
// SM. Per-slot partial sums are first combined across an 8-CTA thread-block
// cluster through distributed shared memory, so the last cluster to finish sums
// G/8 partial rows instead of G.
//
// The stationary method (Algorithm 2 iterated: u <- u + AMG(0; K, r), r <- r - K AMG(0; K, r))
// runs the same kernels with alpha = 1 and beta = 0.
//
// One PCG iteration = 8 kernels, captured `chunk` times in one CUDA graph:
//   k_p      p = s + beta p
//   k_spmv   q = K p, p^T q             (last cluster: alpha = r^T s / p^T q, maxit, breakdown)
//   k_upd    x += alpha p, r -= alpha q
//   k_smooth1 y1 = omega D^-1 r, r1 = r - K y1 (stored), partials of ||r||^2
//   k_restrict partials of c = Phi^T r1
//   k_coarse per slot: ||r|| test, c, e_c = L^-T L^-1 c
//   k_prol   y2 = y1 + Phi e_c
//   k_post   s = y2 + omega D^-1 (r - K y2), r^T s  (last cluster: beta)
#include "common.cuh"
#include "lanes.cuh"

#include <cooperative_groups.h>

#include <type_traits>

#include <chrono>
#include <cstring>
#include <cmath>

namespace cg = cooperative_groups;

#define CLUSTER 8   // CTAs per thread-block cluster of the row kernels
#ifndef UNROLL
#define UNROLL 2    // blocks of a row fetched ahead (FP32 smoother row kernels)
#endif
#ifndef ROW_MINB
#define ROW_MINB 5  // minimum resident CTAs per SM requested for the FP32 smoother row kernels
#endif
#ifndef UNROLL_DF
#define UNROLL_DF 2    // the same for the double-float row kernels (outer SpMV, residual)
#endif
#ifndef ROW_MINB_DF
#define ROW_MINB_DF 5
#endif
// 3 x 3 blocks keep twice the operands of a 2 x 2 block in flight: their row kernels
// request fewer resident CTAs (64 registers) so that nothing spills
#ifndef ROW_MINB_BS3
#define ROW_MINB_BS3 4
#endif
#define MINB(BS, M) ((BS) == 3 ? ROW_MINB_BS3 : (M))
// L2 bulk prefetch of the row stream `ROW_PF` grid-stride passes ahead (0: off; measured
// slower than no prefetch on the 2D elasticity workload at distance 1)
#ifndef ROW_PF
#define ROW_PF 0
#endif

namespace {

struct Dims {
    int nb, Bp, lgBp, k, kp, G, NP;  // NP = G / CLUSTER partial-sum rows of the row kernels
    int NPc;                         // partial-sum rows of the restriction
    int NPs;                         // partial-sum rows of the outer SpMV (its own grid)
    int stat;                        // 1: stationary two-grid iteration (alpha = 1, beta = 0)
    double omega;
};

// The cluster's rank-0 CTA sums s_vals[0..nv) of all CTAs of its cluster (rank
// order, read through distributed shared memory) into out[0..nv).
__device__ __forceinline__ void cluster_store(const double* s_vals, int nv, double* out) {
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    if (cl.block_rank() == 0) {
        const int nr = (int)cl.num_blocks();
        for (int e = threadIdx.x; e < nv; e += blockDim.x) {
            double s = 0.0;
            for (int r = 0; r < nr; ++r) s += cl.map_shared_rank(const_cast<double*>(s_vals), r)[e];
            out[e] = s;
        }
    }
    cl.sync();
}

// After cluster_store: true in exactly one CTA, the rank-0 CTA of the last
// cluster to arrive, which may then read all NP partial rows. No CTA waits on
// another cluster, so nothing can hang. The counter is reset by that CTA.
__device__ __forceinline__ bool last_cluster_arrive(unsigned* counter, int nclusters) {
    __shared__ bool am_last;
    if (cg::this_cluster().block_rank() != 0) return false;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(counter, 1u);
        am_last = (prev == (unsigned)nclusters - 1);
    }
    __syncthreads();
    if (am_last) __threadfence();
    return am_last;
}

// Prefetching loop over the blocks b0..b1 of one block row: for each group of
// UNROLL blocks, `fetch_blk(u, blk)` issues the loads that depend only on the block
// index (per-slot values, element descriptors) together with the column indices, then
// `fetch_vec(u, j)` the gathers of vector entries at column j, then `use(u)` consumes
// slot u. The value stream (the bulk of the bytes) thus never waits for a column index.
// Blocks past the row end are skipped.
template <int U = UNROLL, class FetchBlk, class FetchVec, class Use>
__device__ __forceinline__ void row_blocks(const int32_t* __restrict__ col_idx, int b0, int b1, FetchBlk fetch_blk,
                                           FetchVec fetch_vec, Use use) {
    for (int blk0 = b0; blk0 < b1; blk0 += U) {
        int jj[U];
#pragma unroll
        for (int u = 0; u < U; ++u) jj[u] = (blk0 + u < b1) ? __ldg(col_idx + blk0 + u) : -1;
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (blk0 + u < b1) fetch_blk(u, blk0 + u);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (jj[u] >= 0) fetch_vec(u, jj[u]);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (jj[u] >= 0) use(u);
    }
}

// Element kernels (MF = 1) stage the FP32 reference sub-blocks in shared memory
// (read with warp-uniform addresses); assembled kernels read per-slot values.
#define ELEM_SMEM_KREF(MF, E)                                                    \
    __shared__ float s_kref[(MF) ? POD2G_KREF_MAX : 1];                          \
    if (MF) {                                                                    \
        for (int t_ = threadIdx.x; t_ < (E).nk; t_ += blockDim.x) s_kref[t_] = (E).kref[t_]; \
        __syncthreads();                                                         \
    }

// ---------------------------------------------------------------------------- bulk copies (cp.async.bulk + mbarrier)
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// global -> own shared memory, completion counted in bytes on `bar`; 16-byte
// aligned addresses and a size that is a multiple of 16
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
// Wait for the phase with the given parity to complete, at most `limit` polls;
// false if it did not.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned limit) {
    const uint32_t a = smem_addr(bar);
    for (unsigned t = 0; t < limit; ++t) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
#define MBAR_POLLS (1u << 22)  // bound on the polls of one wait (each poll may suspend briefly)

// ---------------------------------------------------------------------------- L2 prefetch of row streams
// Bytes [b0, b1) of a device allocation (rounded out to 16 bytes; allocations are
// 256-byte aligned and sized in multiples of 256, so the rounded range stays inside)
// are requested into L2 by the bulk-copy engine: fire and forget, nothing waits on it.
__device__ __forceinline__ void l2_prefetch_range(const void* base, long long b0, long long b1) {
    b0 &= ~15LL;
    b1 = (b1 + 15) & ~15LL;
    const char* p = static_cast<const char*>(base);
    for (long long o = b0; o < b1; o += 32768) {
        const unsigned sz = (unsigned)min(32768LL, b1 - o);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p + o), "r"(sz) : "memory");
    }
}

// Row kernels walk items it = (block row << lgBp) + slot lane in grid-stride passes, so a
// warp's 32 items are consecutive and cover one or more whole block rows (Bp <= 32) or
// part of one (Bp > 32). The block data of those rows (column indices, and per-slot
// values `bpb` bytes per block, or element descriptors) is one contiguous range. Lane 0
// of the first warp of a row group prefetches into L2 the range the warp will read `ahead`
// passes later (ahead = 0: the current pass), so that its dependent loads hit L2.
__device__ __forceinline__ void prefetch_rows(const Dims& D, long long it, int ahead,
                                              const int32_t* __restrict__ row_ptr, const int32_t* col_idx,
                                              const void* bdata, long long bpb) {
    const long long wbase = it - (threadIdx.x & 31);
    if ((threadIdx.x & 31) != 0 || (wbase & (D.Bp - 1)) != 0) return;
    const long long nxt = wbase + (long long)ahead * gridDim.x * blockDim.x;
    const long long i_lo = nxt >> D.lgBp;
    if (i_lo >= D.nb) return;
    const long long i_hi = min((long long)D.nb - 1, (nxt + 31) >> D.lgBp);
    const long long k0 = __ldg(row_ptr + i_lo), k1 = __ldg(row_ptr + i_hi + 1);
    l2_prefetch_range(col_idx, 4 * k0, 4 * k1);
    if (bdata) l2_prefetch_range(bdata, bpb * k0, bpb * k1);
}

// ---------------------------------------------------------------------------- load / store / residual
// Joining lanes: b -> bdf, x0 -> xdf (zero if absent), p = q = 0.
__global__ void k_load(const double* __restrict__ b, const double* __restrict__ x0, const int* __restrict__ slots,
                       int nslots, int n, int Bp, float2* __restrict__ bdf, double* __restrict__ b64,
                       float2* __restrict__ xdf, float2* __restrict__ pdf, float2* __restrict__ qdf,
                       float* __restrict__ s32) {
    long long total = (long long)nslots * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e / n);
        long long d = e - (long long)r * n;
        long long o = d * Bp + slots[r];
        bdf[o] = df_from_double(b[e]);
        b64[o] = b[e];
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

// r = b - K x in double-float for masked lanes: writes r, sums ||b||^2 and sets
// tol2 = tol^2 ||b||^2 (b = 0 or non-finite -> DONE).
template <int BS, int MF>
__global__ void __cluster_dims__(CLUSTER, 1, 1) __launch_bounds__(POD2G_THREADS, MINB(BS, ROW_MINB_DF))
k_resid(Dims D, const int* __restrict__ mask, const int32_t* __restrict__ row_ptr,
        const int32_t* __restrict__ col_idx, const float* __restrict__ vals, ElemOp E, const float2* __restrict__ x,
        const float2* __restrict__ b, float2* __restrict__ r, double* part, unsigned* counter, SlotScalars* sc) {
    __shared__ double s_tmp[POD2G_THREADS];
    __shared__ double s_out[2 * POD2G_MAX_BP];
    ELEM_SMEM_KREF(MF, E);
    const int lane = threadIdx.x & (D.Bp - 1);
    const bool on = mask[lane] != 0;
    float bh = 0.f, bl = 0.f, rh = 0.f, rl = 0.f;
    const long long items = (long long)D.nb << D.lgBp;
    const bool warp_on = __any_sync(0xffffffffu, on);
    const void* bdata = MF ? (const void*)E.desc : (const void*)vals;  // per-block data streamed with the rows
    const long long bpb = MF ? 8LL : (long long)BS * BS * D.Bp * 4;
    bool first = true;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
         it += (long long)gridDim.x * blockDim.x) {
        if (ROW_PF > 0 && warp_on) {
            if (first) prefetch_rows(D, it, 0, row_ptr, col_idx, bdata, bpb);
            prefetch_rows(D, it, ROW_PF, row_ptr, col_idx, bdata, bpb);
            first = false;
        }
        if (on) {
            const int i = (int)(it >> D.lgBp);
            float ah[BS], al[BS];
#pragma unroll
            for (int a = 0; a < BS; ++a) { ah[a] = 0.f; al[a] = 0.f; }
            float2 xj[UNROLL_DF][BS];
            float v[UNROLL_DF][BS * BS];
            uint64_t dsc[UNROLL_DF];
            float ce[MF ? POD2G_ELEM_RE : 1];
            if constexpr (MF) elem_row_coefs(E, i, lane, D.Bp, ce);
            row_blocks<UNROLL_DF>(col_idx, row_ptr[i], row_ptr[i + 1],
                [&](int u, int blk) {
                    if constexpr (MF) {
                        dsc[u] = __ldg(E.desc + blk);
                    } else {
                        const float* vb = vals + (long long)blk * BS * BS * D.Bp + lane;
#pragma unroll
                        for (int e = 0; e < BS * BS; ++e) v[u][e] = vb[e * D.Bp];
                    }
                },
                [&](int u, int j) {
#pragma unroll
                    for (int cc = 0; cc < BS; ++cc) xj[u][cc] = x[((long long)j * BS + cc) * D.Bp + lane];
                },
                [&](int u) {
                    if constexpr (MF) elem_block_values<BS>(dsc[u], ce, s_kref, v[u]);
#pragma unroll
                    for (int a = 0; a < BS; ++a)
#pragma unroll
                        for (int cc = 0; cc < BS; ++cc)
                            df_acc_fma(ah[a], al[a], v[u][a * BS + cc], xj[u][cc].x, xj[u][cc].y);
                });
#pragma unroll
            for (int a = 0; a < BS; ++a) {
                const long long o = ((long long)i * BS + a) * D.Bp + lane;
                float2 bv = b[o];
                float2 rv = df_add(bv, df_neg(df_norm(ah[a], al[a])));
                r[o] = rv;
                df_acc_fma(bh, bl, bv.x, bv.x, 2.f * bv.y);
                df_acc_fma(rh, rl, rv.x, rv.x, 2.f * rv.y);
            }
        }
    }
    cta_lane_sum((double)bh + (double)bl, D.Bp, s_tmp, s_out);
    cta_lane_sum((double)rh + (double)rl, D.Bp, s_tmp, s_out + D.Bp);
    cluster_store(s_out, 2 * D.Bp, part + (long long)(blockIdx.x / CLUSTER) * D.Bp * 2);
    if (!last_cluster_arrive(counter, D.NP)) return;
    double bb = grid_lane_total(part, D.NP, 2 * D.Bp, D.Bp, s_tmp);
    double rr = grid_lane_total(part + D.Bp, D.NP, 2 * D.Bp, D.Bp, s_tmp);
    if ((int)threadIdx.x < D.Bp && mask[threadIdx.x]) {
        SlotScalars& s = sc[threadIdx.x];
        s.bb = bb;
        s.tol2 = s.tol2 * bb;  // host stored tol^2
        if (bb == 0.0) {
            s.state = SLOT_DONE; s.result = POD2G_OK; s.iters = 0;
        } else if (!isfinite(bb) || !isfinite(rr)) {
            s.state = SLOT_DONE; s.result = POD2G_NONFINITE;
        }
    }
    if (threadIdx.x == 0) *counter = 0u;
}

// The reported final residual ||b - K x||_2 / ||b||_2 in FP64 for masked lanes: the
// stored FP32 values (exact in FP64) times x (the double-float iterate, hi + lo exact
// in FP64) accumulated with FP64 fused multiply-adds, b the caller's FP64 right-hand
// side, and FP64 sums of squares reduced in a fixed order.
template <int BS, int MF>
__global__ void __cluster_dims__(CLUSTER, 1, 1) __launch_bounds__(POD2G_THREADS)
k_resid64(Dims D, const int* __restrict__ mask, const int32_t* __restrict__ row_ptr,
          const int32_t* __restrict__ col_idx, const float* __restrict__ vals, ElemOp E, const float2* __restrict__ x,
          const double* __restrict__ b64, double* part, unsigned* counter, SlotScalars* sc) {
    __shared__ double s_tmp[POD2G_THREADS];
    __shared__ double s_out[2 * POD2G_MAX_BP];
    ELEM_SMEM_KREF(MF, E);
    const int lane = threadIdx.x & (D.Bp - 1);
    const bool on = mask[lane] != 0;
    double bb = 0.0, rr = 0.0;
    if (on) {
        const long long items = (long long)D.nb << D.lgBp;
        for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
             it += (long long)gridDim.x * blockDim.x) {
            const int i = (int)(it >> D.lgBp);
            double acc[BS];
#pragma unroll
            for (int a = 0; a < BS; ++a) acc[a] = 0.0;
            float ce[MF ? POD2G_ELEM_RE : 1];
            if constexpr (MF) elem_row_coefs(E, i, lane, D.Bp, ce);
            for (int blk = row_ptr[i]; blk < row_ptr[i + 1]; ++blk) {
                const int j = __ldg(col_idx + blk);
                float v[BS * BS];
                if constexpr (MF) {
                    elem_block_values<BS>(__ldg(E.desc + blk), ce, s_kref, v);
                } else {
                    const float* vb = vals + (long long)blk * BS * BS * D.Bp + lane;
#pragma unroll
                    for (int e = 0; e < BS * BS; ++e) v[e] = vb[e * D.Bp];
                }
                double xj[BS];
#pragma unroll
                for (int cc = 0; cc < BS; ++cc) {
                    const float2 t = x[((long long)j * BS + cc) * D.Bp + lane];
                    xj[cc] = (double)t.x + (double)t.y;
                }
#pragma unroll
                for (int a = 0; a < BS; ++a)
#pragma unroll
                    for (int cc = 0; cc < BS; ++cc) acc[a] = fma((double)v[a * BS + cc], xj[cc], acc[a]);
            }
#pragma unroll
            for (int a = 0; a < BS; ++a) {
                const double bv = b64[((long long)i * BS + a) * D.Bp + lane];
                const double rv = bv - acc[a];
                bb = fma(bv, bv, bb);
                rr = fma(rv, rv, rr);
            }
        }
    }
    cta_lane_sum(bb, D.Bp, s_tmp, s_out);
    cta_lane_sum(rr, D.Bp, s_tmp, s_out + D.Bp);
    cluster_store(s_out, 2 * D.Bp, part + (long long)(blockIdx.x / CLUSTER) * D.Bp * 2);
    if (!last_cluster_arrive(counter, D.NP)) return;
    const double btot = grid_lane_total(part, D.NP, 2 * D.Bp, D.Bp, s_tmp);
    const double rtot = grid_lane_total(part + D.Bp, D.NP, 2 * D.Bp, D.Bp, s_tmp);
    if ((int)threadIdx.x < D.Bp && mask[threadIdx.x]) sc[threadIdx.x].relres = btot > 0.0 ? sqrt(rtot / btot) : 0.0;
    if (threadIdx.x == 0) *counter = 0u;
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

// q = K p (double-float), partial p^T q; last cluster: alpha per slot.
template <int BS, int MF>
__global__ void __cluster_dims__(CLUSTER, 1, 1) __launch_bounds__(POD2G_THREADS, MINB(BS, ROW_MINB_DF))
k_spmv(Dims D, int want, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
       const float* __restrict__ vals, ElemOp E, const float2* __restrict__ p, float2* __restrict__ q, double* part,
       unsigned* counter, SlotScalars* sc) {
    __shared__ double s_tmp[POD2G_THREADS];
    __shared__ double s_out[POD2G_MAX_BP];
    ELEM_SMEM_KREF(MF, E);
    const int lane = threadIdx.x & (D.Bp - 1);
    const bool on = sc[lane].state == want;
    float dh = 0.f, dl = 0.f;
    const long long items = (long long)D.nb << D.lgBp;
    const bool warp_on = __any_sync(0xffffffffu, on);
    const void* bdata = MF ? (const void*)E.desc : (const void*)vals;  // per-block data streamed with the rows
    const long long bpb = MF ? 8LL : (long long)BS * BS * D.Bp * 4;
    bool first = true;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
         it += (long long)gridDim.x * blockDim.x) {
        if (ROW_PF > 0 && warp_on) {
            if (first) prefetch_rows(D, it, 0, row_ptr, col_idx, bdata, bpb);
            prefetch_rows(D, it, ROW_PF, row_ptr, col_idx, bdata, bpb);
            first = false;
        }
        if (on) {
            const int i = (int)(it >> D.lgBp);
            float ah[BS], al[BS];
#pragma unroll
            for (int a = 0; a < BS; ++a) { ah[a] = 0.f; al[a] = 0.f; }
            float2 pj[UNROLL_DF][BS];
            float v[UNROLL_DF][BS * BS];
            uint64_t dsc[UNROLL_DF];
            float ce[MF ? POD2G_ELEM_RE : 1];
            if constexpr (MF) elem_row_coefs(E, i, lane, D.Bp, ce);
            row_blocks<UNROLL_DF>(col_idx, row_ptr[i], row_ptr[i + 1],
                [&](int u, int blk) {
                    if constexpr (MF) {
                        dsc[u] = __ldg(E.desc + blk);
                    } else {
                        const float* vb = vals + (long long)blk * BS * BS * D.Bp + lane;
#pragma unroll
                        for (int e = 0; e < BS * BS; ++e) v[u][e] = vb[e * D.Bp];
                    }
                },
                [&](int u, int j) {
#pragma unroll
                    for (int cc = 0; cc < BS; ++cc) pj[u][cc] = p[((long long)j * BS + cc) * D.Bp + lane];
                },
                [&](int u) {
                    if constexpr (MF) elem_block_values<BS>(dsc[u], ce, s_kref, v[u]);
#pragma unroll
                    for (int a = 0; a < BS; ++a)
#pragma unroll
                        for (int cc = 0; cc < BS; ++cc)
                            df_acc_fma(ah[a], al[a], v[u][a * BS + cc], pj[u][cc].x, pj[u][cc].y);
                });
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
    cta_lane_sum((double)dh + (double)dl, D.Bp, s_tmp, s_out);
    cluster_store(s_out, D.Bp, part + (long long)(blockIdx.x / CLUSTER) * D.Bp * 2);
    if (!last_cluster_arrive(counter, D.NPs)) return;
    double pq = grid_lane_total(part, D.NPs, 2 * D.Bp, D.Bp, s_tmp);
    if ((int)threadIdx.x < D.Bp) {
        SlotScalars& s = sc[threadIdx.x];
        if (s.state == want) {
            if (s.iters >= s.maxit) {
                s.state = SLOT_DONE; s.result = POD2G_NOT_CONVERGED; s.alpha = 0.0;
            } else if (!(pq > 0.0) || !isfinite(pq)) {
                s.state = SLOT_DONE; s.result = isfinite(pq) ? POD2G_BREAKDOWN : POD2G_NONFINITE; s.alpha = 0.0;
            } else {
                s.alpha = D.stat ? 1.0 : s.rs / pq;
                s.iters += 1;
            }
        }
    }
    if (threadIdx.x == 0) *counter = 0u;
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

// Pre-relaxation from zero and the residual it leaves: y1 = omega D^-1 r (PRE = 1),
// 0 (PRE = 0) or a stored y1 (PRE = 2, Gauss-Seidel), r1 = r - K y1, written to
// out (FP32); cluster partial sums of ||r||^2 go to part[cluster][slot].
template <int BS, int MF>
__global__ void __cluster_dims__(CLUSTER, 1, 1) __launch_bounds__(POD2G_THREADS, MINB(BS, ROW_MINB))
k_smooth1(Dims D, int want, int PRE, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
          const float* __restrict__ vals, ElemOp E, const float* __restrict__ dinv, const float2* __restrict__ r,
          const float* __restrict__ y1, float* __restrict__ out, double* part, const SlotScalars* __restrict__ sc) {
    __shared__ double s_tmp[POD2G_THREADS];
    __shared__ double s_out[POD2G_MAX_BP];
    ELEM_SMEM_KREF(MF, E);
    const int lane = threadIdx.x & (D.Bp - 1);
    const bool on = sc[lane].state == want;
    float rr = 0.f;
    const float w = (float)D.omega;
    const long long items = (long long)D.nb << D.lgBp;
    const bool warp_on = __any_sync(0xffffffffu, on);
    const void* bdata = MF ? (const void*)E.desc : (const void*)vals;  // per-block data streamed with the rows
    const long long bpb = MF ? 8LL : (long long)BS * BS * D.Bp * 4;
    bool first = true;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
         it += (long long)gridDim.x * blockDim.x) {
        if (ROW_PF > 0 && warp_on) {
            if (PRE && first) prefetch_rows(D, it, 0, row_ptr, col_idx, bdata, bpb);
            if (PRE) prefetch_rows(D, it, ROW_PF, row_ptr, col_idx, bdata, bpb);
            first = false;
        }
        if (on) {
            const int i = (int)(it >> D.lgBp);
            float acc[BS];
#pragma unroll
            for (int a = 0; a < BS; ++a) acc[a] = 0.f;
            if (PRE) {
                // gathered r.hi and D^-1 (or the stored y1) stay as loaded until the block is used,
                // so that all loads of the group are in flight together
                float yj[UNROLL][BS], dj[UNROLL][BS], v[UNROLL][BS * BS];
                uint64_t dsc[UNROLL];
                float ce[MF ? POD2G_ELEM_RE : 1];
                if constexpr (MF) elem_row_coefs(E, i, lane, D.Bp, ce);
                row_blocks(col_idx, row_ptr[i], row_ptr[i + 1],
                    [&](int u, int blk) {
                        if constexpr (MF) {
                            dsc[u] = __ldg(E.desc + blk);
                        } else {
                            const float* vb = vals + (long long)blk * BS * BS * D.Bp + lane;
#pragma unroll
                            for (int e = 0; e < BS * BS; ++e) v[u][e] = vb[e * D.Bp];
                        }
                    },
                    [&](int u, int j) {
#pragma unroll
                        for (int cc = 0; cc < BS; ++cc) {
                            const long long o = ((long long)j * BS + cc) * D.Bp + lane;
                            if (PRE == 2) {
                                yj[u][cc] = y1[o];
                            } else {
                                yj[u][cc] = r[o].x;
                                dj[u][cc] = dinv[o];
                            }
                        }
                    },
                    [&](int u) {
                        if constexpr (MF) elem_block_values<BS>(dsc[u], ce, s_kref, v[u]);
                        float y[BS];
#pragma unroll
                        for (int cc = 0; cc < BS; ++cc) y[cc] = PRE == 2 ? yj[u][cc] : w * dj[u][cc] * yj[u][cc];
#pragma unroll
                        for (int a = 0; a < BS; ++a)
#pragma unroll
                            for (int cc = 0; cc < BS; ++cc) acc[a] = __fmaf_rn(v[u][a * BS + cc], y[cc], acc[a]);
                    });
            }
#pragma unroll
            for (int a = 0; a < BS; ++a) {
                const long long o = ((long long)i * BS + a) * D.Bp + lane;
                const float rv = r[o].x;
                out[o] = rv - acc[a];
                rr = __fmaf_rn(rv, rv, rr);
            }
        }
    }
    cta_lane_sum((double)rr, D.Bp, s_tmp, s_out);
    cluster_store(s_out, D.Bp, part + (long long)(blockIdx.x / CLUSTER) * D.Bp * 2);
}

// Restriction c = Phi^T r1 for every slot: a tall-skinny product of Phi (row-major
// [n][KP]) and r1 (slot-interleaved [n][Bp]), register-tiled as an outer product:
// a thread owns LB consecutive slots x 8 consecutive modes, and per row loads
// LB values of r1 (one vector load) and 8 of Phi (two float4, shared by the warp)
// for 8*LB FMAs. A team of (Bp/LB) * (KP/8) threads covers all Bp x KP outputs;
// the CTA's teams split its contiguous chunk of rows (two rows in flight per
// thread) and their partials are summed in team order. Cluster partial rows go
// to cpart[cluster][slot][KP].
template <int KP, int LB>
__global__ void __cluster_dims__(CLUSTER, 1, 1) __launch_bounds__(POD2G_THREADS)
k_restrict(Dims D, int want, long long n, const float* __restrict__ phi, const float* __restrict__ r1,
           double* cpart, const SlotScalars* __restrict__ sc) {
    extern __shared__ double s_c[];  // [Bp * KP] doubles, then [teams][Bp * KP] floats
    const int Bp = D.Bp;
    const int NOUT = Bp * KP;
    const int quads = Bp / LB, groups = KP / 8;
    const int team_size = quads * groups;
    const int teams = POD2G_THREADS / team_size;
    const int team = threadIdx.x / team_size, w = threadIdx.x - team * team_size;
    const int q = w % quads, g = w / quads;
    const int b0 = q * LB, m0 = g * 8;
    float* s_team = (float*)(s_c + NOUT);
    // every slot of the quad is accumulated: outputs of slots that are not in
    // state `want` are never read (each slot has its own accumulators)
    const bool on = team < teams;
    (void)sc;
    (void)want;
    float acc[LB][8];
#pragma unroll
    for (int l = 0; l < LB; ++l)
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[l][m] = 0.f;
    const long long per = (n + gridDim.x - 1) / gridDim.x;
    const long long d_begin = blockIdx.x * per, d_end = min(n, d_begin + per);
    auto load_r = [&](long long d, float* x) {
        const float* p = r1 + d * Bp + b0;
        if (LB == 4) { const float4 v = *reinterpret_cast<const float4*>(p); x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w; }
        else if (LB == 8) {
            const float4 v0 = *reinterpret_cast<const float4*>(p), v1 = *reinterpret_cast<const float4*>(p + 4);
            x[0] = v0.x; x[1] = v0.y; x[2] = v0.z; x[3] = v0.w; x[4] = v1.x; x[5] = v1.y; x[6] = v1.z; x[7] = v1.w;
        } else if (LB == 2) { const float2 v = *reinterpret_cast<const float2*>(p); x[0] = v.x; x[1] = v.y; }
        else x[0] = p[0];
    };
    auto fma_row = [&](const float* x, float4 f0, float4 f1) {
        const float f[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
#pragma unroll
        for (int l = 0; l < LB; ++l)
#pragma unroll
            for (int m = 0; m < 8; ++m) acc[l][m] = __fmaf_rn(f[m], x[l], acc[l][m]);
    };
    if (on) {
        long long d = d_begin + team;
        for (; d + teams < d_end; d += 2 * teams) {
            float xa[LB], xb[LB];
            load_r(d, xa);
            load_r(d + teams, xb);
            const float4* pa = reinterpret_cast<const float4*>(phi + d * KP + m0);
            const float4* pb = reinterpret_cast<const float4*>(phi + (d + teams) * KP + m0);
            const float4 a0 = __ldg(pa), a1 = __ldg(pa + 1), c0 = __ldg(pb), c1 = __ldg(pb + 1);
            fma_row(xa, a0, a1);
            fma_row(xb, c0, c1);
        }
        if (d < d_end) {
            float xa[LB];
            load_r(d, xa);
            const float4* pa = reinterpret_cast<const float4*>(phi + d * KP + m0);
            fma_row(xa, __ldg(pa), __ldg(pa + 1));
        }
    }
    if (team < teams) {
#pragma unroll
        for (int l = 0; l < LB; ++l)
#pragma unroll
            for (int m = 0; m < 8; ++m) s_team[team * NOUT + (b0 + l) * KP + m0 + m] = on ? acc[l][m] : 0.f;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < NOUT; o += blockDim.x) {
        double s = 0.0;
        for (int t = 0; t < teams; ++t) s += (double)s_team[t * NOUT + o];
        s_c[o] = s;
    }
    __syncthreads();
    cluster_store(s_c, NOUT, cpart + (long long)(blockIdx.x / CLUSTER) * NOUT);
}

// The same restriction with the CTA's contiguous rows of r1 ([n][Bp]) and Phi
// ([n][KP]) staged through shared memory: chunks of R rows are copied with
// cp.async.bulk into a ring of RS_STAGES buffers (one mbarrier each) while the
// teams consume earlier chunks, so the loads of a thread no longer wait on HBM
// latency. A wait that exceeds its poll bound sets *err, waits (bounded) for the
// copies still in flight and skips the rest of the work; every CTA still takes
// part in the cluster reduction, so nothing waits forever.
#define RS_STAGES 3
template <int KP, int LB>
__global__ void __cluster_dims__(CLUSTER, 1, 1) __launch_bounds__(POD2G_THREADS)
k_restrict_bulk(Dims D, long long n, int R, const float* __restrict__ phi, const float* __restrict__ r1,
                double* cpart, int* err) {
    extern __shared__ __align__(16) unsigned char s_raw[];
    __shared__ int s_bad;
    const int Bp = D.Bp;
    const int NOUT = Bp * KP;
    const int quads = Bp / LB, groups = KP / 8;
    const int team_size = quads * groups;
    const int teams = POD2G_THREADS / team_size;
    const int team = threadIdx.x / team_size, w = threadIdx.x - team * team_size;
    const int q = w % quads, g = w / quads;
    const int b0 = q * LB, m0 = g * 8;
    double* s_c = reinterpret_cast<double*>(s_raw);
    float* s_team = reinterpret_cast<float*>(s_c + NOUT);
    float* s_r = s_team + teams * NOUT;
    float* s_p = s_r + RS_STAGES * R * Bp;
    uint64_t* bars = reinterpret_cast<uint64_t*>(s_p + RS_STAGES * R * KP);
    const long long per = (n + gridDim.x - 1) / gridDim.x;
    const long long d_begin = blockIdx.x * per, d_end = min(n, d_begin + per);
    const int nchunks = d_end > d_begin ? (int)((d_end - d_begin + R - 1) / R) : 0;
    if (threadIdx.x == 0) {
        s_bad = 0;
        for (int st = 0; st < RS_STAGES; ++st) mbar_init(bars + st, 1);
        mbar_fence_init();
    }
    __syncthreads();
    int issued = 0;  // meaningful in thread 0
    auto issue = [&](int ch) {
        const int st = ch % RS_STAGES;
        const long long d0 = d_begin + (long long)ch * R;
        const int rows = (int)min((long long)R, d_end - d0);
        const unsigned br = (unsigned)rows * Bp * 4u, bq = (unsigned)rows * KP * 4u;
        mbar_expect_tx(bars + st, br + bq);
        bulk_load(s_r + (size_t)st * R * Bp, r1 + d0 * Bp, br, bars + st);
        bulk_load(s_p + (size_t)st * R * KP, phi + d0 * KP, bq, bars + st);
    };
    if (threadIdx.x == 0)
        for (; issued < min(nchunks, RS_STAGES); ++issued) issue(issued);
    float acc[LB][8];
#pragma unroll
    for (int l = 0; l < LB; ++l)
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[l][m] = 0.f;
    int bad_chunk = -1;
    for (int ch = 0; ch < nchunks; ++ch) {
        const int st = ch % RS_STAGES;
        if (!mbar_wait(bars + st, (unsigned)(ch / RS_STAGES) & 1u, MBAR_POLLS)) s_bad = 1;
        const int rows = (int)min((long long)R, d_end - (d_begin + (long long)ch * R));
        if (team < teams) {
            const float* rb = s_r + (size_t)st * R * Bp + b0;
            const float* pb = s_p + (size_t)st * R * KP + m0;
            for (int t = team; t < rows; t += teams) {
                float x[LB];
                if (LB == 4) {
                    const float4 v = *reinterpret_cast<const float4*>(rb + (size_t)t * Bp);
                    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
                } else if (LB == 8) {
                    const float4 v0 = *reinterpret_cast<const float4*>(rb + (size_t)t * Bp);
                    const float4 v1 = *reinterpret_cast<const float4*>(rb + (size_t)t * Bp + 4);
                    x[0] = v0.x; x[1] = v0.y; x[2] = v0.z; x[3] = v0.w;
                    x[4] = v1.x; x[5] = v1.y; x[6] = v1.z; x[7] = v1.w;
                } else {
#pragma unroll
                    for (int l = 0; l < LB; ++l) x[l] = rb[(size_t)t * Bp + l];
                }
                const float4 f0 = *reinterpret_cast<const float4*>(pb + (size_t)t * KP);
                const float4 f1 = *reinterpret_cast<const float4*>(pb + (size_t)t * KP + 4);
                const float f[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
#pragma unroll
                for (int l = 0; l < LB; ++l)
#pragma unroll
                    for (int m = 0; m < 8; ++m) acc[l][m] = __fmaf_rn(f[m], x[l], acc[l][m]);
            }
        }
        __syncthreads();  // buffer st is free again
        if (s_bad) {
            bad_chunk = ch;
            break;
        }
        if (threadIdx.x == 0 && issued < nchunks) issue(issued++);
    }
    if (bad_chunk >= 0) {
        // a copy did not complete in time: report, let the copies in flight land, skip the rest
        if (threadIdx.x == 0) {
            atomicExch(err, 2);
            for (int ch = bad_chunk; ch < issued; ++ch)
                mbar_wait(bars + ch % RS_STAGES, (unsigned)(ch / RS_STAGES) & 1u, MBAR_POLLS);
        }
        __syncthreads();
    }
    if (team < teams) {
#pragma unroll
        for (int l = 0; l < LB; ++l)
#pragma unroll
            for (int m = 0; m < 8; ++m) s_team[team * NOUT + (b0 + l) * KP + m0 + m] = acc[l][m];
    }
    __syncthreads();
    for (int o = threadIdx.x; o < NOUT; o += blockDim.x) {
        double sum = 0.0;
        for (int t = 0; t < teams; ++t) sum += (double)s_team[t * NOUT + o];
        s_c[o] = sum;
    }
    __syncthreads();
    cluster_store(s_c, NOUT, cpart + (long long)(blockIdx.x / CLUSTER) * NOUT);
}

// One CTA per slot: convergence test on ||r||^2, coarse right-hand side
// c = Phi^T r1 (sum over partial rows in order), e_c = L^-T L^-1 c in FP64.
__global__ void k_coarse(Dims D, int want, const double* __restrict__ part, const double* __restrict__ cpart,
                         const double* __restrict__ Lc, float* __restrict__ ec, SlotScalars* sc) {
    __shared__ double smem[POD2G_THREADS];
    __shared__ double cv[POD2G_MAX_K];
    __shared__ int go;
    const int b = blockIdx.x;
    if (sc[b].state != want) return;
    const int kp = D.kp;
    const long long nv = (long long)D.Bp * kp;
    // ||r||^2 over partial rows: contiguous ranges per thread, then a fixed tree
    {
        const int T = blockDim.x;
        const int g0 = (int)((long long)D.NP * threadIdx.x / T), g1 = (int)((long long)D.NP * (threadIdx.x + 1) / T);
        smem[threadIdx.x] = ordered_sum(part + b, g0, g1, 2LL * D.Bp);
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
    const int Q = blockDim.x / kp;
    const int m = threadIdx.x % kp, q = threadIdx.x / kp;
    double cs = 0.0;
    if (q < Q) {
        const int g0 = (int)((long long)D.NPc * q / Q), g1 = (int)((long long)D.NPc * (q + 1) / Q);
        cs = ordered_sum(cpart + (long long)b * kp + m, g0, g1, nv);  // rows of the restriction grid
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
}

// y2 = y1 + Phi e_c with y1 = omega D^-1 r (PRE = 1), 0 (PRE = 0) or stored
// (PRE = 2; y may alias y1, each element is read before it is written); KP a
// compile-time width so that a row's Phi loads are all issued before they are used.
template <int PRE, int KP>
__global__ void __launch_bounds__(POD2G_THREADS)
k_prol(Dims D, int want, const float* __restrict__ dinv, const float2* __restrict__ r, const float* y1,
       const float* __restrict__ phi, const float* __restrict__ ec, float* y, const SlotScalars* __restrict__ sc,
       long long n) {
    extern __shared__ float s_ec[];  // [Bp][KP + 1] (odd row stride: no bank conflicts across slots)
    if constexpr (KP > 0)
        for (int e = threadIdx.x; e < D.Bp * KP; e += blockDim.x) s_ec[(e / KP) * (KP + 1) + e % KP] = ec[e];
    __syncthreads();
    const int lane = threadIdx.x & (D.Bp - 1);
    if (sc[lane].state != want) return;
    const float w = (float)D.omega;
    constexpr int KA = KP > 0 ? KP : 4;
    float e_l[KA];
#pragma unroll
    for (int m = 0; m < KP; ++m) e_l[m] = s_ec[lane * (KP + 1) + m];
    const long long items = n << D.lgBp;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
         it += (long long)gridDim.x * blockDim.x) {
        const long long d = it >> D.lgBp;
        const float4* ph = reinterpret_cast<const float4*>(phi + d * KP);
        float4 f[KA / 4];
#pragma unroll
        for (int m4 = 0; m4 < KP / 4; ++m4) f[m4] = __ldg(ph + m4);
        float v = PRE == 2 ? y1[it] : (PRE ? w * dinv[it] * r[it].x : 0.f);
        float v2 = 0.f;
#pragma unroll
        for (int m4 = 0; m4 < KP / 4; ++m4) {
            v = __fmaf_rn(f[m4].x, e_l[4 * m4 + 0], v);
            v2 = __fmaf_rn(f[m4].y, e_l[4 * m4 + 1], v2);
            v = __fmaf_rn(f[m4].z, e_l[4 * m4 + 2], v);
            v2 = __fmaf_rn(f[m4].w, e_l[4 * m4 + 3], v2);
        }
        y[it] = v + v2;
    }
}

// One Gauss-Seidel step over the nodes of one colour (eq. GaussSeidel, pointwise):
// for each node i of the colour and each component a in order (reverse order if
// BWD), y_ia += D_ia^-1 (r - K y)_ia, in place. Nodes of one colour share no
// stored block, so their threads are independent; inside a node the components
// are updated in sequence, the later rows corrected through the diagonal block.
// FROM0: the forward sweep from y = 0, where nodes of this and later colours
// still read as 0 (their memory is not read).
template <int BS, int MF, int BWD>
__global__ void __launch_bounds__(POD2G_THREADS, MINB(BS, ROW_MINB))
k_gs(Dims D, int want, int from0, int colour, const int32_t* __restrict__ cnodes, int cnt,
     const uint8_t* __restrict__ col_of, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
     const float* __restrict__ vals, ElemOp E, const float* __restrict__ dinv, const float2* __restrict__ r,
     float* y, const SlotScalars* __restrict__ sc) {
    ELEM_SMEM_KREF(MF, E);
    const int lane = threadIdx.x & (D.Bp - 1);
    if (sc[lane].state != want) return;
    const long long items = (long long)cnt << D.lgBp;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
         it += (long long)gridDim.x * blockDim.x) {
        const int i = cnodes[it >> D.lgBp];
        float acc[BS], vd[BS * BS];
#pragma unroll
        for (int a = 0; a < BS; ++a) acc[a] = 0.f;
#pragma unroll
        for (int e = 0; e < BS * BS; ++e) vd[e] = 0.f;
        float yj[UNROLL][BS], v[UNROLL][BS * BS];
        int jj[UNROLL];
        uint64_t dsc[UNROLL];
        float ce[MF ? POD2G_ELEM_RE : 1];
        if constexpr (MF) elem_row_coefs(E, i, lane, D.Bp, ce);
        row_blocks(col_idx, row_ptr[i], row_ptr[i + 1],
            [&](int u, int blk) {
                if constexpr (MF) {
                    dsc[u] = __ldg(E.desc + blk);
                } else {
                    const float* vb = vals + (long long)blk * BS * BS * D.Bp + lane;
#pragma unroll
                    for (int e = 0; e < BS * BS; ++e) v[u][e] = vb[e * D.Bp];
                }
            },
            [&](int u, int j) {
                jj[u] = j;
                const bool zero = from0 && (j == i || (int)col_of[j] >= colour);
#pragma unroll
                for (int cc = 0; cc < BS; ++cc) yj[u][cc] = zero ? 0.f : y[((long long)j * BS + cc) * D.Bp + lane];
            },
            [&](int u) {
                if constexpr (MF) elem_block_values<BS>(dsc[u], ce, s_kref, v[u]);
#pragma unroll
                for (int a = 0; a < BS; ++a)
#pragma unroll
                    for (int cc = 0; cc < BS; ++cc) acc[a] = __fmaf_rn(v[u][a * BS + cc], yj[u][cc], acc[a]);
                if (jj[u] == i) {
#pragma unroll
                    for (int e = 0; e < BS * BS; ++e) vd[e] = v[u][e];
                }
            });
#pragma unroll
        for (int t = 0; t < BS; ++t) {
            const int a = BWD ? BS - 1 - t : t;
            const long long o = ((long long)i * BS + a) * D.Bp + lane;
            const float yo = from0 ? 0.f : y[o];
            const float dy = dinv[o] * (r[o].x - acc[a]);
            y[o] = yo + dy;
#pragma unroll
            for (int b = 0; b < BS; ++b)
                if (BWD ? b < a : b > a) acc[b] = __fmaf_rn(vd[b * BS + a], dy, acc[b]);
        }
    }
}

// s = y2 + omega D^-1 (r - K y2) (r2 = 1) or y2 (r2 = 0); partial r^T s (and
// r^T s_old for Polak-Ribiere); last cluster: beta, JOINING -> ACTIVE.
template <int BS, int POST, int MF>
__global__ void __cluster_dims__(CLUSTER, 1, 1) __launch_bounds__(POD2G_THREADS, MINB(BS, ROW_MINB))
k_post(Dims D, int want, int pr, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
       const float* __restrict__ vals, ElemOp E, const float* __restrict__ dinv, const float2* __restrict__ r,
       const float* __restrict__ y, float* __restrict__ s, double* part, unsigned* counter, SlotScalars* sc) {
    __shared__ double s_tmp[POD2G_THREADS];
    __shared__ double s_out[2 * POD2G_MAX_BP];
    ELEM_SMEM_KREF(MF && POST, E);
    const int lane = threadIdx.x & (D.Bp - 1);
    const bool on = sc[lane].state == want;
    float h = 0.f, l = 0.f, xh = 0.f, xl = 0.f;
    const float w = (float)D.omega;
    const long long items = (long long)D.nb << D.lgBp;
    const bool warp_on = __any_sync(0xffffffffu, on);
    const void* bdata = MF ? (const void*)E.desc : (const void*)vals;  // per-block data streamed with the rows
    const long long bpb = MF ? 8LL : (long long)BS * BS * D.Bp * 4;
    bool first = true;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
         it += (long long)gridDim.x * blockDim.x) {
        if (ROW_PF > 0 && warp_on) {
            if (POST && first) prefetch_rows(D, it, 0, row_ptr, col_idx, bdata, bpb);
            if (POST) prefetch_rows(D, it, ROW_PF, row_ptr, col_idx, bdata, bpb);
            first = false;
        }
        if (on) {
            const int i = (int)(it >> D.lgBp);
            float acc[BS];
#pragma unroll
            for (int a = 0; a < BS; ++a) acc[a] = 0.f;
            if (POST) {
                float yj[UNROLL][BS], v[UNROLL][BS * BS];
                uint64_t dsc[UNROLL];
                float ce[MF ? POD2G_ELEM_RE : 1];
                if constexpr (MF) elem_row_coefs(E, i, lane, D.Bp, ce);
                row_blocks(col_idx, row_ptr[i], row_ptr[i + 1],
                    [&](int u, int blk) {
                        if constexpr (MF) {
                            dsc[u] = __ldg(E.desc + blk);
                        } else {
                            const float* vb = vals + (long long)blk * BS * BS * D.Bp + lane;
#pragma unroll
                            for (int e = 0; e < BS * BS; ++e) v[u][e] = vb[e * D.Bp];
                        }
                    },
                    [&](int u, int j) {
#pragma unroll
                        for (int cc = 0; cc < BS; ++cc) yj[u][cc] = y[((long long)j * BS + cc) * D.Bp + lane];
                    },
                    [&](int u) {
                        if constexpr (MF) elem_block_values<BS>(dsc[u], ce, s_kref, v[u]);
#pragma unroll
                        for (int a = 0; a < BS; ++a)
#pragma unroll
                            for (int cc = 0; cc < BS; ++cc) acc[a] = __fmaf_rn(v[u][a * BS + cc], yj[u][cc], acc[a]);
                    });
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
    cta_lane_sum((double)h + (double)l, D.Bp, s_tmp, s_out);
    cta_lane_sum((double)xh + (double)xl, D.Bp, s_tmp, s_out + D.Bp);
    cluster_store(s_out, 2 * D.Bp, part + (long long)(blockIdx.x / CLUSTER) * D.Bp * 2);
    if (!last_cluster_arrive(counter, D.NP)) return;
    double rs = grid_lane_total(part, D.NP, 2 * D.Bp, D.Bp, s_tmp);
    double rsx = pr ? grid_lane_total(part + D.Bp, D.NP, 2 * D.Bp, D.Bp, s_tmp) : 0.0;
    if ((int)threadIdx.x < D.Bp) {
        SlotScalars& S = sc[threadIdx.x];
        if (S.state == want) {
            if (!(rs > 0.0) || !isfinite(rs)) {
                S.state = SLOT_DONE;
                S.result = isfinite(rs) ? POD2G_BREAKDOWN : POD2G_NONFINITE;
            } else {
                S.beta = (S.first || D.stat) ? 0.0 : (pr ? (rs - rsx) / S.rs : rs / S.rs);
                S.rs = rs;
                S.first = 0;
                if (want == SLOT_JOINING) S.state = SLOT_ACTIVE;
            }
        }
    }
    if (threadIdx.x == 0) *counter = 0u;
}

// ---------------------------------------------------------------------------- single-instance row kernels
// For one slot lane (Bp = 1) a block row's values are one contiguous run ([block][bs*bs]); a
// thread per row would walk it alone with strided, uncoalesced loads. Here a group of LPR lanes
// owns a row: lane t takes blocks beg + t, beg + t + LPR, ..., so a group reads the row's values
// as coalesced runs and its gathers are in flight at once; the bs partial sums are then combined
// across the group by a fixed butterfly of shuffles, and lane a < bs writes output a. LPR = 8:
// each lane takes several blocks of a row between butterfly steps (the SpMV's steps add
// double-float pairs, ~30 instructions each), measured faster than 32 lanes with a block each
// for the SpMV and the smoothing passes. KIND as k_rows_ws.
template <int BS, int KIND>
__global__ void __cluster_dims__(CLUSTER, 1, 1) __launch_bounds__(POD2G_THREADS)
k_rows_v1(Dims D, int want, int pr, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
          const float* __restrict__ vals, const float* __restrict__ dinv, const float2* __restrict__ vin,
          const float* __restrict__ yin, float2* __restrict__ qout, float* __restrict__ out, double* part,
          unsigned* counter, SlotScalars* sc) {
    constexpr int LPR = 8;
    constexpr int BB = BS * BS;
    __shared__ double s_tmp[POD2G_THREADS];
    __shared__ double s_out[2 * POD2G_MAX_BP];
    const int sub = threadIdx.x & (LPR - 1);
    const unsigned gmask = LPR == 32 ? 0xffffffffu : (((1u << LPR) - 1u) << (threadIdx.x & (32 - LPR)));
    const bool on = sc[0].state == want;
    const float w = (float)D.omega;
    float d1h = 0.f, d1l = 0.f, d2h = 0.f, d2l = 0.f;
    const long long groups = (long long)gridDim.x * (POD2G_THREADS / LPR);
    if (on) {
        for (long long i = (long long)blockIdx.x * (POD2G_THREADS / LPR) + threadIdx.x / LPR; i < D.nb; i += groups) {
            const int beg = __ldg(row_ptr + i), end = __ldg(row_ptr + i + 1);
            float ah[BS], al[BS];
#pragma unroll
            for (int a = 0; a < BS; ++a) { ah[a] = 0.f; al[a] = 0.f; }
#pragma unroll 2
            for (int blk = beg + sub; blk < end; blk += LPR) {
                const int j = __ldg(col_idx + blk);
                float v[BB];
                const float* vb = vals + (long long)blk * BB;
#pragma unroll
                for (int e = 0; e < BB; ++e) v[e] = __ldg(vb + e);
                if constexpr (KIND == 0) {
                    float2 pj[BS];
#pragma unroll
                    for (int cc = 0; cc < BS; ++cc) pj[cc] = vin[(long long)j * BS + cc];
#pragma unroll
                    for (int a = 0; a < BS; ++a)
#pragma unroll
                        for (int cc = 0; cc < BS; ++cc) df_acc_fma(ah[a], al[a], v[a * BS + cc], pj[cc].x, pj[cc].y);
                } else {
                    float yj[BS];
#pragma unroll
                    for (int cc = 0; cc < BS; ++cc) {
                        const long long o = (long long)j * BS + cc;
                        yj[cc] = KIND == 1 ? w * dinv[o] * vin[o].x : yin[o];
                    }
#pragma unroll
                    for (int a = 0; a < BS; ++a)
#pragma unroll
                        for (int cc = 0; cc < BS; ++cc) ah[a] = __fmaf_rn(v[a * BS + cc], yj[cc], ah[a]);
                }
            }
            // combine the group's partial sums (fixed butterfly; every lane ends with the totals)
#pragma unroll
            for (int off = LPR / 2; off > 0; off >>= 1) {
#pragma unroll
                for (int a = 0; a < BS; ++a) {
                    const float oh = __shfl_xor_sync(gmask, ah[a], off);
                    if constexpr (KIND == 0) {
                        const float ol = __shfl_xor_sync(gmask, al[a], off);
                        const float2 t = df_add(df_norm(ah[a], al[a]), df_norm(oh, ol));
                        ah[a] = t.x;
                        al[a] = t.y;
                    } else {
                        ah[a] = __fadd_rn(ah[a], oh);
                    }
                }
            }
            if (sub < BS) {
                float h = ah[0], l = al[0];
#pragma unroll
                for (int a = 1; a < BS; ++a)
                    if (sub == a) { h = ah[a]; l = al[a]; }
                const long long o = (long long)i * BS + sub;
                if constexpr (KIND == 0) {
                    const float2 qv = df_norm(h, l);
                    qout[o] = qv;
                    const float2 pv = vin[o];
                    df_acc_fma(d1h, d1l, pv.x, qv.x, qv.y);
                    d1l = __fmaf_rn(pv.y, qv.x, d1l);
                } else if constexpr (KIND == 1) {
                    const float rv = vin[o].x;
                    out[o] = rv - h;
                    d1h = __fmaf_rn(rv, rv, d1h);
                } else {
                    const float2 rv = vin[o];
                    const float sv = __fmaf_rn(w * dinv[o], rv.x - h, yin[o]);
                    if (pr) df_acc_fma(d2h, d2l, out[o], rv.x, rv.y);
                    out[o] = sv;
                    df_acc_fma(d1h, d1l, sv, rv.x, rv.y);
                }
            }
        }
    }
    cta_lane_sum((double)d1h + (double)d1l, 1, s_tmp, s_out);
    if constexpr (KIND == 2) cta_lane_sum((double)d2h + (double)d2l, 1, s_tmp, s_out + 1);
    cluster_store(s_out, KIND == 2 ? 2 : 1, part + (long long)(blockIdx.x / CLUSTER) * 2);
    if constexpr (KIND == 1) return;
    if (!last_cluster_arrive(counter, KIND == 0 ? D.NPs : D.NP)) return;
    if constexpr (KIND == 0) {
        const double pq = grid_lane_total(part, D.NPs, 2, 1, s_tmp);
        if (threadIdx.x == 0) {
            SlotScalars& S = sc[0];
            if (S.state == want) {
                if (S.iters >= S.maxit) {
                    S.state = SLOT_DONE; S.result = POD2G_NOT_CONVERGED; S.alpha = 0.0;
                } else if (!(pq > 0.0) || !isfinite(pq)) {
                    S.state = SLOT_DONE; S.result = isfinite(pq) ? POD2G_BREAKDOWN : POD2G_NONFINITE; S.alpha = 0.0;
                } else {
                    S.alpha = D.stat ? 1.0 : S.rs / pq;
                    S.iters += 1;
                }
            }
        }
    } else {
        const double rs = grid_lane_total(part, D.NP, 2, 1, s_tmp);
        const double rsx = pr ? grid_lane_total(part + 1, D.NP, 2, 1, s_tmp) : 0.0;
        if (threadIdx.x == 0) {
            SlotScalars& S = sc[0];
            if (S.state == want) {
                if (!(rs > 0.0) || !isfinite(rs)) {
                    S.state = SLOT_DONE;
                    S.result = isfinite(rs) ? POD2G_BREAKDOWN : POD2G_NONFINITE;
                } else {
                    S.beta = (S.first || D.stat) ? 0.0 : (pr ? (rs - rsx) / S.rs : rs / S.rs);
                    S.rs = rs;
                    S.first = 0;
                    if (want == SLOT_JOINING) S.state = SLOT_ACTIVE;
                }
            }
        }
    }
    if (threadIdx.x == 0) *counter = 0u;
}

// ---------------------------------------------------------------------------- prolongation + post-smoothing from K Phi
// With W = K Phi of each slot stored (FP32, mode-major [KP][n][Bp], so that a warp reads one mode of
// consecutive unknowns and slots in one coalesced run; formed at set-up with K_c), the product
// K y2 of the post-smoothing needs no pass over the matrix: y2 = y1 + Phi e_c, and
// K y2 = K y1 + W e_c = (r - r1) + W e_c, since the pre-smoothing pass left r1 = r - K y1. Hence
//     s = y2 + omega D^-1 (r - K y2) = y2 + omega D^-1 (r1 - W e_c),
// one elementwise pass reading Phi (shared by the slots), W, r1, r and D^-1 instead of the
// prolongation pass plus a sweep over the slot's matrix values: 4 n KP bytes of W per slot
// against 4 bs^2 nnzb of values. Partial r^T s (and r^T s_old for Polak-Ribiere) per cluster; the
// last cluster forms beta exactly as the post-smoothing row kernel does (Jacobi, r1 = r2 = 1).
template <int KP>
__global__ void __cluster_dims__(CLUSTER, 1, 1) __launch_bounds__(POD2G_THREADS, 4)
k_postw(Dims D, int want, int pr, const float* __restrict__ dinv, const float2* __restrict__ r,
        const float* __restrict__ r1, const float* __restrict__ phi, const float* __restrict__ W,
        const float* __restrict__ ec, float* __restrict__ s, double* part, unsigned* counter, SlotScalars* sc,
        long long n) {
    extern __shared__ float s_ec[];  // [Bp][KP + 1]
    __shared__ double s_tmp[POD2G_THREADS];
    __shared__ double s_out[2 * POD2G_MAX_BP];
    for (int e = threadIdx.x; e < D.Bp * KP; e += blockDim.x) s_ec[(e / KP) * (KP + 1) + e % KP] = ec[e];
    __syncthreads();
    const int lane = threadIdx.x & (D.Bp - 1);
    const bool on = sc[lane].state == want;
    const float w = (float)D.omega;
    float h = 0.f, l = 0.f, xh = 0.f, xl = 0.f;
    if (on) {
        const float* el = s_ec + lane * (KP + 1);   // the slot's e_c (odd row stride: no bank conflicts)
        const long long items = n << D.lgBp;
        for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
             it += (long long)gridDim.x * blockDim.x) {
            const long long d = it >> D.lgBp;
            const float4* ph = reinterpret_cast<const float4*>(phi + d * KP);
            const float* wr = W + d * D.Bp + lane;   // W[m][d][slot]: mode m at wr + m * n * Bp
            const long long mstride = n * D.Bp;
            const float2 rv = r[it];
            const float dv = dinv[it];
            const float r1v = r1[it];
            const float so = pr ? s[it] : 0.f;
            float y = w * dv * rv.x, y2 = 0.f, t = r1v, t2 = 0.f;
#pragma unroll
            for (int m4 = 0; m4 < KP / 4; ++m4) {
                const float4 f = __ldg(ph + m4);
                const float w0 = __ldg(wr + (4 * m4 + 0) * mstride), w1 = __ldg(wr + (4 * m4 + 1) * mstride);
                const float w2 = __ldg(wr + (4 * m4 + 2) * mstride), w3 = __ldg(wr + (4 * m4 + 3) * mstride);
                const float e0 = el[4 * m4], e1 = el[4 * m4 + 1], e2 = el[4 * m4 + 2], e3 = el[4 * m4 + 3];
                y = __fmaf_rn(f.x, e0, y);
                y2 = __fmaf_rn(f.y, e1, y2);
                y = __fmaf_rn(f.z, e2, y);
                y2 = __fmaf_rn(f.w, e3, y2);
                t = __fmaf_rn(-w0, e0, t);
                t2 = __fmaf_rn(-w1, e1, t2);
                t = __fmaf_rn(-w2, e2, t);
                t2 = __fmaf_rn(-w3, e3, t2);
            }
            const float sv = __fmaf_rn(w * dv, t + t2, y + y2);
            if (pr) df_acc_fma(xh, xl, so, rv.x, rv.y);
            s[it] = sv;
            df_acc_fma(h, l, sv, rv.x, rv.y);
        }
    }
    cta_lane_sum((double)h + (double)l, D.Bp, s_tmp, s_out);
    cta_lane_sum((double)xh + (double)xl, D.Bp, s_tmp, s_out + D.Bp);
    cluster_store(s_out, 2 * D.Bp, part + (long long)(blockIdx.x / CLUSTER) * D.Bp * 2);
    if (!last_cluster_arrive(counter, D.NP)) return;
    const double rs = grid_lane_total(part, D.NP, 2 * D.Bp, D.Bp, s_tmp);
    const double rsx = pr ? grid_lane_total(part + D.Bp, D.NP, 2 * D.Bp, D.Bp, s_tmp) : 0.0;
    if ((int)threadIdx.x < D.Bp) {
        SlotScalars& S = sc[threadIdx.x];
        if (S.state == want) {
            if (!(rs > 0.0) || !isfinite(rs)) {
                S.state = SLOT_DONE;
                S.result = isfinite(rs) ? POD2G_BREAKDOWN : POD2G_NONFINITE;
            } else {
                S.beta = (S.first || D.stat) ? 0.0 : (pr ? (rs - rsx) / S.rs : rs / S.rs);
                S.rs = rs;
                S.first = 0;
                if (want == SLOT_JOINING) S.state = SLOT_ACTIVE;
            }
        }
    }
    if (threadIdx.x == 0) *counter = 0u;
}

// ---------------------------------------------------------------------------- warp-staged row kernels
// The outer SpMV, the pre-smoothing pass and the post-smoothing pass of assembled
// operators with 4 <= Bp <= 64 slot lanes and damped-Jacobi relaxation, restructured
// so that no thread waits on the value stream (the bulk of their bytes):
//   * a warp owns RPW = 32 / LR consecutive block rows (a "row group"; LR = Bp / SPT
//     lanes per row, SPT slots per lane, so that a lane reads SPT consecutive slots
//     with one vector access) and walks its groups in grid-stride order, so that the
//     rows in flight across the GPU form one front and gathered entries are reused
//     from L2;
//   * a group is processed in chunks of WS_U blocks per row. The values of a row's
//     chunk are contiguous ([block][bs*bs][Bp]); one lane per row copies them with
//     cp.async.bulk into the warp's ring of WS_STAGES shared-memory buffers (one
//     mbarrier each), two chunks ahead of the one being used;
//   * the gathered vector entries of the next chunk are loaded into registers before
//     the current chunk is used, with column indices loaded one chunk earlier still.
// Arithmetic and per-slot reduction order are fixed per slot (a lane always owns the
// same slots), so a result does not depend on the other slots. A bounded mbarrier
// wait that expires sets *err to 2, waits (bounded) for the copies the warp still has
// in flight and skips the warp's remaining rows; every CTA still joins the reductions.
#define WS_STAGES 3
template <int BS> struct WsU { static constexpr int U = BS == 1 ? 9 : 3; };

// floats per row slot of a stage buffer: the chunk's values, padded so that the RPW
// rows of a warp read disjoint banks (row stride / LR odd)
__host__ __device__ constexpr int ws_row_stride(int bs, int Bp, int spt) {
    return (32 / (Bp / spt) > 1 && ((bs == 1 ? 9 : 3) * bs * bs) % 2 == 0) ? (bs == 1 ? 9 : 3) * bs * bs * Bp + Bp / spt
                                                                          : (bs == 1 ? 9 : 3) * bs * bs * Bp;
}

template <int SPT>
__device__ __forceinline__ void ws_ld2(const float2* p, float2 (&o)[SPT]) {
    if constexpr (SPT == 1) {
        o[0] = *p;
    } else if constexpr (SPT == 2) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        o[0] = make_float2(v.x, v.y); o[1] = make_float2(v.z, v.w);
    } else {
        static_assert(SPT <= 2, "one or two slots per lane");
    }
}
template <int SPT>
__device__ __forceinline__ void ws_ld1(const float* p, float (&o)[SPT]) {
    if constexpr (SPT == 1) {
        o[0] = *p;
    } else if constexpr (SPT == 2) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        o[0] = v.x; o[1] = v.y;
    } else {
        static_assert(SPT <= 2, "one or two slots per lane");
    }
}

// Position of a warp in its walk: row group g (chunk c of nch), and the block range of
// the lane's row in that group.
struct WsCur {
    int g, c, nch, beg, len;
};

// KIND 0: q = K p (double-float), partial p^T q, last cluster alpha (as k_spmv).
// KIND 1: r1 = r - K (omega D^-1 r), partial ||r||^2 (as k_smooth1 with PRE = 1).
// KIND 2: s = y2 + omega D^-1 (r - K y2), partial r^T s (and r^T s_old), last cluster
//         beta (as k_post with POST = 1).
template <int BS, int SPT, int KIND>
__global__ void __cluster_dims__(CLUSTER, 1, 1) __launch_bounds__(POD2G_THREADS, (BS == 3 && SPT == 2) ? 1 : 2)
k_rows_ws(Dims D, int want, int pr, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
          const float* __restrict__ vals, const float* __restrict__ dinv, const float2* __restrict__ vin,
          const float* __restrict__ yin, float2* __restrict__ qout, float* __restrict__ out, double* part,
          unsigned* counter, SlotScalars* sc, int* err) {
    constexpr int U = WsU<BS>::U;
    constexpr int BB = BS * BS;
    extern __shared__ __align__(16) float s_ws[];
    __shared__ double s_tmp[POD2G_THREADS * SPT];
    __shared__ double s_out[2 * POD2G_MAX_BP];
    const int Bp = D.Bp;
    const int LR = Bp / SPT, RPW = 32 / LR;
    const int RS = ws_row_stride(BS, Bp, SPT);
    const int SF = RPW * RS;  // floats per stage buffer
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = lane / LR, slot0 = (lane % LR) * SPT;
    const int NG = (D.nb + RPW - 1) / RPW;
    const int TW = gridDim.x * (POD2G_THREADS / 32);
    float* ring = s_ws + (size_t)warp * WS_STAGES * SF;
    uint64_t* bars = reinterpret_cast<uint64_t*>(s_ws + (size_t)(POD2G_THREADS / 32) * WS_STAGES * SF) +
                     warp * WS_STAGES;
    bool on[SPT];
    bool any_on = false, all_on = true;
#pragma unroll
    for (int s = 0; s < SPT; ++s) {
        on[s] = sc[slot0 + s].state == want;
        any_on |= on[s];
        all_on &= on[s];
    }
    const bool work = __any_sync(0xffffffffu, any_on);  // uniform over the grid (all warps see all slots)
    if (lane == 0) {
        for (int st = 0; st < WS_STAGES; ++st) mbar_init(bars + st, 1);
        mbar_fence_init();
    }
    __syncwarp();
    const float w = (float)D.omega;
    // per-slot partial sums (double-float pairs accumulated in FP32)
    float d1h[SPT], d1l[SPT], d2h[SPT], d2l[SPT];
#pragma unroll
    for (int s = 0; s < SPT; ++s) { d1h[s] = 0.f; d1l[s] = 0.f; d2h[s] = 0.f; d2l[s] = 0.f; }

    auto load_group = [&](WsCur& q) {
        const int i = q.g * RPW + r;
        q.beg = 0;
        q.len = 0;
        if (q.g < NG && i < D.nb) {
            q.beg = __ldg(row_ptr + i);
            q.len = __ldg(row_ptr + i + 1) - q.beg;
        }
        const unsigned mx = __reduce_max_sync(0xffffffffu, (unsigned)q.len);
        q.nch = (int)((mx + U - 1) / U);
    };
    auto next = [&](WsCur q) {
        if (q.g >= NG) return q;
        if (++q.c >= q.nch) {
            q.g += TW;
            q.c = 0;
            load_group(q);
        }
        return q;
    };
    auto nblk = [&](const WsCur& q) { return q.g < NG ? min(U, max(0, q.len - q.c * U)) : 0; };
    // copies of the chunk of state q into stage buffer st (all lanes call)
    auto issue = [&](const WsCur& q, int st) {
        if (q.g >= NG) return;
        const int nbk = nblk(q);
        const unsigned bytes = (unsigned)nbk * BB * Bp * 4u;
        const unsigned total = __reduce_add_sync(0xffffffffu, (lane % LR) == 0 ? bytes : 0u);
        if (lane == 0) mbar_expect_tx(bars + st, total);
        __syncwarp();
        if ((lane % LR) == 0 && nbk > 0)
            bulk_load(ring + (size_t)st * SF + r * RS, vals + ((long long)q.beg + q.c * U) * BB * Bp, bytes, bars + st);
    };
    auto load_cols = [&](const WsCur& q, int (&cj)[U]) {
        const int nbk = nblk(q);
#pragma unroll
        for (int u = 0; u < U; ++u) cj[u] = u < nbk ? __ldg(col_idx + q.beg + q.c * U + u) : -1;
    };
    // gathered entries of the chunk, held as loaded until the chunk is used (so that no thread
    // waits on them a chunk early): KIND 0 p (double-float); KIND 1 (r.hi, D^-1); KIND 2 y
    using GT = typename std::conditional<KIND == 2, float, float2>::type;
    auto gather = [&](const int (&cj)[U], GT (&G)[U][BS][SPT]) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (cj[u] < 0) continue;
#pragma unroll
            for (int cc = 0; cc < BS; ++cc) {
                const long long o = ((long long)cj[u] * BS + cc) * Bp + slot0;
                if constexpr (KIND == 0) {
                    ws_ld2<SPT>(vin + o, G[u][cc]);
                } else if constexpr (KIND == 1) {
                    float2 rv[SPT];
                    float dv[SPT];
                    ws_ld2<SPT>(vin + o, rv);
                    ws_ld1<SPT>(dinv + o, dv);
#pragma unroll
                    for (int s = 0; s < SPT; ++s) G[u][cc][s] = make_float2(rv[s].x, dv[s]);
                } else {
                    ws_ld1<SPT>(yin + o, G[u][cc]);
                }
            }
        }
    };

    WsCur C{(int)blockIdx.x * (POD2G_THREADS / 32) + warp, 0, 0, 0, 0};
    if (!work) C.g = NG;
    load_group(C);
    int t = 0, issued = 0;
    issue(C, 0);
    issued = C.g < NG ? 1 : 0;
    WsCur Gs = next(C);
    issue(Gs, 1);
    issued += Gs.g < NG ? 1 : 0;
    WsCur P = next(Gs);
    int cj[U], cjn[U];
    GT G[U][BS][SPT], Gn[U][BS][SPT];
    load_cols(C, cj);
    gather(cj, G);
    load_cols(Gs, cjn);
    // accumulators of the lane's row and its own-row operands (loaded at the group's first chunk)
    float ah[BS][SPT], al[BS][SPT];
    float bh[BS], bl[BS];      // KIND 0, one slot per lane, bs >= 2: the accumulators of the second column
    float2 own2[BS][SPT];      // KIND 0: p; KIND 1, 2: r
    float owny[BS][SPT], ownd[BS][SPT], owns[BS][SPT];
    bool bad = false;
    while (C.g < NG) {
        // 1. gathers of the next chunk
        gather(cjn, Gn);
        // 2. copies two chunks ahead, and their column indices
        issue(P, (t + 2) % WS_STAGES);
        issued += P.g < NG ? 1 : 0;
        int cjp[U];
        load_cols(P, cjp);
        // 3. this chunk
        if (C.c == 0) {
#pragma unroll
            for (int a = 0; a < BS; ++a)
#pragma unroll
                for (int s = 0; s < SPT; ++s) { ah[a][s] = 0.f; al[a][s] = 0.f; }
#pragma unroll
            for (int a = 0; a < BS; ++a) { bh[a] = 0.f; bl[a] = 0.f; }
            const int i = C.g * RPW + r;
            if (i < D.nb) {
#pragma unroll
                for (int a = 0; a < BS; ++a) {
                    const long long o = ((long long)i * BS + a) * Bp + slot0;
                    ws_ld2<SPT>(vin + o, own2[a]);
                    if constexpr (KIND == 2) {
                        ws_ld1<SPT>(yin + o, owny[a]);
                        ws_ld1<SPT>(dinv + o, ownd[a]);
                        if (pr) ws_ld1<SPT>(out + o, owns[a]);
                    }
                }
            }
        }
        const int st = t % WS_STAGES;
        bad = __any_sync(0xffffffffu, !mbar_wait(bars + st, (unsigned)(t / WS_STAGES) & 1u, MBAR_POLLS));
        if (bad) break;
        const float* vb = ring + (size_t)st * SF + r * RS + slot0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (cj[u] < 0) continue;
            if constexpr (KIND == 0 && SPT == 2 && BS >= 2) {
                // the lane's two slots in packed instructions (each accumulator sees the same
                // operations in the same order as below)
#pragma unroll
                for (int cc = 0; cc < BS; ++cc) {
                    const float2 h2 = make_float2(G[u][cc][0].x, G[u][cc][1].x);
                    const float2 l2 = make_float2(G[u][cc][0].y, G[u][cc][1].y);
                    const float2 nh2 = f2_mul(h2, make_float2(-1.f, -1.f));
#pragma unroll
                    for (int a = 0; a < BS; ++a) {
                        float v[2];
                        ws_ld1<2>(vb + (u * BB + a * BS + cc) * Bp, v);
                        float2 hi = make_float2(ah[a][0], ah[a][1]), lo = make_float2(al[a][0], al[a][1]);
                        df_acc_fma2(hi, lo, make_float2(v[0], v[1]), h2, nh2, l2);
                        ah[a][0] = hi.x; ah[a][1] = hi.y;
                        al[a][0] = lo.x; al[a][1] = lo.y;
                    }
                }
            } else if constexpr (KIND == 0 && SPT == 1 && BS >= 2) {
                // columns 0 and 1 of the block in packed instructions, into two accumulators per
                // row (column 2 of a 3x3 block goes to the first, scalar); the two are added in
                // double-float at the end of the row
                const float2 h2 = make_float2(G[u][0][0].x, G[u][1][0].x);
                const float2 l2 = make_float2(G[u][0][0].y, G[u][1][0].y);
                const float2 nh2 = f2_mul(h2, make_float2(-1.f, -1.f));
#pragma unroll
                for (int a = 0; a < BS; ++a) {
                    const float* va = vb + (u * BB + a * BS) * Bp;
                    float2 hi = make_float2(ah[a][0], bh[a]), lo = make_float2(al[a][0], bl[a]);
                    df_acc_fma2(hi, lo, make_float2(va[0], va[Bp]), h2, nh2, l2);
                    ah[a][0] = hi.x; bh[a] = hi.y;
                    al[a][0] = lo.x; bl[a] = lo.y;
                    if constexpr (BS == 3) df_acc_fma(ah[a][0], al[a][0], va[2 * Bp], G[u][2][0].x, G[u][2][0].y);
                }
            } else {
#pragma unroll
                for (int a = 0; a < BS; ++a)
#pragma unroll
                    for (int cc = 0; cc < BS; ++cc) {
                        float v[SPT];
                        ws_ld1<SPT>(vb + (u * BB + a * BS + cc) * Bp, v);
#pragma unroll
                        for (int s = 0; s < SPT; ++s) {
                            if constexpr (KIND == 0) df_acc_fma(ah[a][s], al[a][s], v[s], G[u][cc][s].x, G[u][cc][s].y);
                            else if constexpr (KIND == 1)
                                ah[a][s] = __fmaf_rn(v[s], w * G[u][cc][s].y * G[u][cc][s].x, ah[a][s]);
                            else ah[a][s] = __fmaf_rn(v[s], G[u][cc][s], ah[a][s]);
                        }
                    }
            }
        }
        if (C.c == C.nch - 1) {
            const int i = C.g * RPW + r;
            if (i < D.nb && any_on) {
#pragma unroll
                for (int a = 0; a < BS; ++a) {
                    const long long o = ((long long)i * BS + a) * Bp + slot0;
                    if constexpr (KIND == 0) {
                        float2 qv[SPT];
#pragma unroll
                        for (int s = 0; s < SPT; ++s) {
                            if constexpr (SPT == 1 && BS >= 2)
                                qv[s] = df_add(df_norm(ah[a][s], al[a][s]), df_norm(bh[a], bl[a]));
                            else
                                qv[s] = df_norm(ah[a][s], al[a][s]);
                            if (on[s]) {
                                const float2 pv = own2[a][s];
                                df_acc_fma(d1h[s], d1l[s], pv.x, qv[s].x, qv[s].y);
                                d1l[s] = __fmaf_rn(pv.y, qv[s].x, d1l[s]);
                            }
                        }
                        if (SPT == 2 && all_on) {
                            *reinterpret_cast<float4*>(qout + o) = make_float4(qv[0].x, qv[0].y, qv[1].x, qv[1].y);
                        } else {
#pragma unroll
                            for (int s = 0; s < SPT; ++s)
                                if (on[s]) qout[o + s] = qv[s];
                        }
                    } else if constexpr (KIND == 1) {
#pragma unroll
                        for (int s = 0; s < SPT; ++s) {
                            if (!on[s]) continue;
                            const float rv = own2[a][s].x;
                            out[o + s] = rv - ah[a][s];
                            d1h[s] = __fmaf_rn(rv, rv, d1h[s]);
                        }
                    } else {
#pragma unroll
                        for (int s = 0; s < SPT; ++s) {
                            if (!on[s]) continue;
                            const float2 rv = own2[a][s];
                            const float sv = __fmaf_rn(w * ownd[a][s], rv.x - ah[a][s], owny[a][s]);
                            if (pr) df_acc_fma(d2h[s], d2l[s], owns[a][s], rv.x, rv.y);
                            out[o + s] = sv;
                            df_acc_fma(d1h[s], d1l[s], sv, rv.x, rv.y);
                        }
                    }
                }
            }
        }
        // 4. advance
        __syncwarp();  // every lane is done with buffer st before it is refilled
        C = Gs;
        Gs = P;
        P = next(P);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            cj[u] = cjn[u];
            cjn[u] = cjp[u];
#pragma unroll
            for (int cc = 0; cc < BS; ++cc)
#pragma unroll
                for (int s = 0; s < SPT; ++s) G[u][cc][s] = Gn[u][cc][s];
        }
        ++t;
    }
    if (bad) {
        // a copy did not complete in time: report, let the copies in flight land, skip the rest
        if (lane == 0) {
            atomicExch(err, 2);
            for (int k = t; k < issued; ++k)
                mbar_wait(bars + k % WS_STAGES, (unsigned)(k / WS_STAGES) & 1u, MBAR_POLLS);
        }
        __syncwarp();
    }
    // per-slot CTA sums (entry tid*SPT + s belongs to slot (tid*SPT + s) mod Bp)
    auto cta_sum = [&](const float* h, const float* l, double* dst) {
        __syncthreads();
#pragma unroll
        for (int s = 0; s < SPT; ++s) s_tmp[threadIdx.x * SPT + s] = (double)h[s] + (double)l[s];
        __syncthreads();
        if ((int)threadIdx.x < Bp) {
            double acc = 0.0;
            for (int e = threadIdx.x; e < POD2G_THREADS * SPT; e += Bp) acc += s_tmp[e];
            dst[threadIdx.x] = acc;
        }
        __syncthreads();
    };
    cta_sum(d1h, d1l, s_out);
    if constexpr (KIND == 2) cta_sum(d2h, d2l, s_out + Bp);
    cluster_store(s_out, KIND == 2 ? 2 * Bp : Bp, part + (long long)(blockIdx.x / CLUSTER) * Bp * 2);
    if constexpr (KIND == 1) return;
    if (!last_cluster_arrive(counter, KIND == 0 ? D.NPs : D.NP)) return;
    if constexpr (KIND == 0) {
        const double pq = grid_lane_total(part, D.NPs, 2 * Bp, Bp, s_tmp);
        if ((int)threadIdx.x < Bp) {
            SlotScalars& S = sc[threadIdx.x];
            if (S.state == want) {
                if (S.iters >= S.maxit) {
                    S.state = SLOT_DONE; S.result = POD2G_NOT_CONVERGED; S.alpha = 0.0;
                } else if (!(pq > 0.0) || !isfinite(pq)) {
                    S.state = SLOT_DONE; S.result = isfinite(pq) ? POD2G_BREAKDOWN : POD2G_NONFINITE; S.alpha = 0.0;
                } else {
                    S.alpha = D.stat ? 1.0 : S.rs / pq;
                    S.iters += 1;
                }
            }
        }
    } else {
        const double rs = grid_lane_total(part, D.NP, 2 * Bp, Bp, s_tmp);
        const double rsx = pr ? grid_lane_total(part + Bp, D.NP, 2 * Bp, Bp, s_tmp) : 0.0;
        if ((int)threadIdx.x < Bp) {
            SlotScalars& S = sc[threadIdx.x];
            if (S.state == want) {
                if (!(rs > 0.0) || !isfinite(rs)) {
                    S.state = SLOT_DONE;
                    S.result = isfinite(rs) ? POD2G_BREAKDOWN : POD2G_NONFINITE;
                } else {
                    S.beta = (S.first || D.stat) ? 0.0 : (pr ? (rs - rsx) / S.rs : rs / S.rs);
                    S.rs = rs;
                    S.first = 0;
                    if (want == SLOT_JOINING) S.state = SLOT_ACTIVE;
                }
            }
        }
    }
    if (threadIdx.x == 0) *counter = 0u;
}

}  // namespace

// ---------------------------------------------------------------------------- host side
static int restrict_grid(pod2g_ctx* c);

static Dims dims_of(pod2g_ctx* c) {
    Dims D;
    D.nb = c->nb;
    D.Bp = c->Bp;
    D.lgBp = 0;
    while ((1 << D.lgBp) < c->Bp) ++D.lgBp;
    D.k = c->k;
    D.kp = c->kp;
    D.G = c->grid_rows;
    D.NP = c->grid_rows / CLUSTER;
    D.NPs = c->grid_spmv / CLUSTER;
    D.NPc = restrict_grid(c) / CLUSTER;
    D.stat = c->method == POD2G_STATIONARY;
    D.omega = c->omega;
    return D;
}

// grid of the row kernels: a multiple of the cluster size, at most 8 CTAs per SM
int batched_grid(int num_sms, long long items) {
    int g = ceil_div(items, POD2G_THREADS);
    g = std::max(CLUSTER, std::min(g, 8 * num_sms));
    return ceil_div(g, CLUSTER) * CLUSTER;
}

// KERNEL<BS, MF> for the context's block size and operator form (MF = 1: element-factored)
#define LAUNCH_BS(KERNEL, ...)                                                         \
    do {                                                                               \
        if (c->elem) {                                                                 \
            if (c->bs == 1) KERNEL<1, 1> __VA_ARGS__;                                  \
            else if (c->bs == 2) KERNEL<2, 1> __VA_ARGS__;                             \
            else KERNEL<3, 1> __VA_ARGS__;                                             \
        } else {                                                                       \
            if (c->bs == 1) KERNEL<1, 0> __VA_ARGS__;                                  \
            else if (c->bs == 2) KERNEL<2, 0> __VA_ARGS__;                             \
            else KERNEL<3, 0> __VA_ARGS__;                                             \
        }                                                                              \
    } while (0)

#define KP_LIST(X) X(8) X(16) X(24) X(32) X(40) X(48) X(64)

// Jacobi: y1 = omega D^-1 r on the fly (PRE = r1). Gauss-Seidel: y1 stored in s (PRE = 2) or 0.
template <int BS, int MF>
static void launch_smooth1(pod2g_ctx* c, Dims D, int want) {
    const int pre = c->smoother == POD2G_SMOOTHER_SGS ? (c->pre ? 2 : 0) : c->pre;
    k_smooth1<BS, MF><<<D.G, POD2G_THREADS, 0, c->stream>>>(D, want, pre, c->d_row_ptr, c->d_col_idx,
                                                             c->d_vals32, elem_op(c), c->d_dinv32, c->d_rdf,
                                                             c->d_s32, c->d_y32, c->d_part, c->d_sc);
}

// Gauss-Seidel sweep over all colours (forward from zero, or backward in place) on s.
template <int BS, int MF>
static int launch_gs(pod2g_ctx* c, Dims D, int want, int backward) {
    const ElemOp E = elem_op(c);
    for (int t = 0; t < c->ncolours; ++t) {
        const int col = backward ? c->ncolours - 1 - t : t;
        const int cnt = c->coff[col + 1] - c->coff[col];
        if (cnt == 0) continue;
        const int g = std::max(1, std::min(ceil_div((long long)cnt << D.lgBp, POD2G_THREADS), 8 * c->num_sms));
        if (backward)
            k_gs<BS, MF, 1><<<g, POD2G_THREADS, 0, c->stream>>>(D, want, 0, col, c->d_cnodes + c->coff[col], cnt,
                                                                 c->d_colour, c->d_row_ptr, c->d_col_idx,
                                                                 c->d_vals32, E, c->d_dinv32, c->d_rdf, c->d_s32,
                                                                 c->d_sc);
        else
            k_gs<BS, MF, 0><<<g, POD2G_THREADS, 0, c->stream>>>(D, want, 1, col, c->d_cnodes + c->coff[col], cnt,
                                                                 c->d_colour, c->d_row_ptr, c->d_col_idx,
                                                                 c->d_vals32, E, c->d_dinv32, c->d_rdf, c->d_s32,
                                                                 c->d_sc);
        P2G_TRY(pod2g_check_launch(c));
    }
    return POD2G_OK;
}

// slots per thread of the restriction: 4 (vector loads), more when Bp x kp needs it
static int restrict_lb(int Bp, int kp) {
    int lb = std::min(4, Bp);
    while ((Bp / lb) * (kp / 8) > POD2G_THREADS) lb *= 2;
    return lb;
}
static size_t restrict_smem(int Bp, int kp) {
    if (kp == 0) return 0;
    const int lb = restrict_lb(Bp, kp);
    const int teams = POD2G_THREADS / ((Bp / lb) * (kp / 8));
    return (size_t)Bp * kp * sizeof(double) + (size_t)teams * Bp * kp * sizeof(float);
}
static int restrict_grid(pod2g_ctx* c) { return c->grid_restrict; }

// Bulk-staged restriction: rows per chunk (~24 KB of r1 and Phi per stage, a
// multiple of 4) and its shared memory; 0 when it does not apply (Bp < 4: rows
// of r1 are not 16-byte multiples) or does not fit.
static int restrict_bulk_rows_default(int Bp, int kp) {
    if (kp == 0 || Bp < 4) return 0;
    int R = 24576 / ((Bp + kp) * 4);
    R = std::max(8, std::min(128, R)) / 4 * 4;
    return R;
}
static size_t restrict_bulk_smem_rows(int Bp, int kp, int R) {
    if (R == 0) return 0;
    const size_t sz = restrict_smem(Bp, kp) + (size_t)RS_STAGES * R * (Bp + kp) * sizeof(float) +
                      RS_STAGES * sizeof(uint64_t);
    return sz <= 200 * 1024 ? sz : 0;
}
// the context's rows per chunk (a tuning setting; 0 = the default)
static int restrict_bulk_rows(const pod2g_ctx* c) {
    if (c->kp == 0 || c->Bp < 4) return 0;
    return c->restrict_rows > 0 ? c->restrict_rows : restrict_bulk_rows_default(c->Bp, c->kp);
}
static size_t restrict_bulk_smem(const pod2g_ctx* c) {
    return restrict_bulk_smem_rows(c->Bp, c->kp, restrict_bulk_rows(c));
}

#define LB_LIST(X, KP) X(KP, 1) X(KP, 2) X(KP, 4) X(KP, 8)
static void launch_restrict(pod2g_ctx* c, Dims D, int want) {
    const size_t smb = restrict_bulk_smem(c);
    const size_t sm = smb ? smb : restrict_smem(c->Bp, c->kp);
    const int R = restrict_bulk_rows(c);
    const int g = D.NPc * CLUSTER;
    const int lb = restrict_lb(c->Bp, c->kp);
#define CASE_LB(KP_, LB_)                                                                                          \
    if (c->kp == KP_ && lb == LB_) {                                                                               \
        if (smb)                                                                                                   \
            k_restrict_bulk<KP_, LB_><<<g, POD2G_THREADS, sm, c->stream>>>(D, c->n, R, c->d_phi32, c->d_y32,       \
                                                                           c->d_cpart, c->d_err);                  \
        else                                                                                                       \
            k_restrict<KP_, LB_><<<g, POD2G_THREADS, sm, c->stream>>>(D, want, c->n, c->d_phi32, c->d_y32,         \
                                                                      c->d_cpart, c->d_sc);                        \
    }
#define CASE_KP(KP_) LB_LIST(CASE_LB, KP_)
    KP_LIST(CASE_KP)
#undef CASE_KP
#undef CASE_LB
}

// y2 = y1 + Phi e_c. Jacobi: y1 recomputed from r (or 0), y2 -> y. Gauss-Seidel: y1
// stored in s (or 0), y2 -> s in place.
static void launch_prol(pod2g_ctx* c, Dims D, int want) {
    const size_t sm = sizeof(float) * c->Bp * (c->kp + 1);
    const long long n = c->n;
    const int gp = std::max(1, std::min(ceil_div(n * c->Bp, POD2G_THREADS), c->grid_prol));
    const bool gs = c->smoother == POD2G_SMOOTHER_SGS;
    const int pre = gs ? (c->pre ? 2 : 0) : (c->pre ? 1 : 0);
    float* out = gs ? c->d_s32 : c->d_y32;
#define PROL(PRE_, KP_)                                                                                     \
    k_prol<PRE_, KP_><<<gp, POD2G_THREADS, sm, c->stream>>>(D, want, c->d_dinv32, c->d_rdf, c->d_s32,      \
                                                            c->d_phi32, c->d_ec, out, c->d_sc, n)
#define CASE_KP(KP_)                                     \
    case KP_:                                            \
        if (pre == 2) PROL(2, KP_);                      \
        else if (pre == 1) PROL(1, KP_);                 \
        else PROL(0, KP_);                               \
        break;
    switch (c->kp) {
        KP_LIST(CASE_KP)
        CASE_KP(0)
    }
#undef CASE_KP
#undef PROL
}

template <int BS, int MF>
static void launch_post(pod2g_ctx* c, Dims D, int want) {
    dim3 g(D.G), t(POD2G_THREADS);
    // Gauss-Seidel: s is already final in place; k_post without its SpMV only forms r^T s and
    // beta. Its y and s then name the same buffer: each element is read and written back with
    // the same value by the same thread (beta_pr is 0, so s is not read), nothing else touches it.
    if (c->smoother == POD2G_SMOOTHER_SGS)
        k_post<BS, 0, MF><<<g, t, 0, c->stream>>>(D, want, 0, c->d_row_ptr, c->d_col_idx, c->d_vals32, elem_op(c),
                                                  c->d_dinv32, c->d_rdf, c->d_s32, c->d_s32, c->d_part,
                                                  c->d_counters + CNT_POST, c->d_sc);
    else if (c->post)
        k_post<BS, 1, MF><<<g, t, 0, c->stream>>>(D, want, c->beta_pr, c->d_row_ptr, c->d_col_idx, c->d_vals32,
                                                  elem_op(c), c->d_dinv32, c->d_rdf, c->d_y32, c->d_s32, c->d_part,
                                                  c->d_counters + CNT_POST, c->d_sc);
    else
        k_post<BS, 0, MF><<<g, t, 0, c->stream>>>(D, want, c->beta_pr, c->d_row_ptr, c->d_col_idx, c->d_vals32,
                                                  elem_op(c), c->d_dinv32, c->d_rdf, c->d_y32, c->d_s32, c->d_part,
                                                  c->d_counters + CNT_POST, c->d_sc);
}

// ---- warp-staged row kernels (k_rows_ws): applicability, shared memory, launch
// slots per lane: two above 32 slot lanes (a warp covers at most 32 lanes of a row)
static int ws_spt(const pod2g_ctx* c) { return c->Bp > 32 ? 2 : 1; }
// the staged kernels apply to assembled operators with 4 <= Bp <= 64 and Jacobi relaxation
static bool ws_applies(const pod2g_ctx* c) {
    return !c->elem && c->precision != POD2G_FP64 && c->Bp >= 4 && c->Bp <= 64 &&
           c->smoother == POD2G_SMOOTHER_JACOBI;
}
static size_t ws_smem(int bs, int Bp, int spt) {
    const int rpw = 32 / (Bp / spt);
    return (size_t)(POD2G_THREADS / 32) * WS_STAGES * ((size_t)rpw * ws_row_stride(bs, Bp, spt) * 4 + 8);
}
static bool ws_spmv(const pod2g_ctx* c) { return ws_applies(c) && (c->rows_kernel & 2); }
static bool ws_smooth(const pod2g_ctx* c) { return ws_applies(c) && (c->rows_kernel & 1); }
// single-instance contexts (Bp = 1): the group-per-row kernels are the alternative form
static bool v1_applies(const pod2g_ctx* c) {
    return !c->elem && c->precision != POD2G_FP64 && c->Bp == 1 && c->smoother == POD2G_SMOOTHER_JACOBI;
}
static bool v1_spmv(const pod2g_ctx* c) { return v1_applies(c) && (c->rows_kernel & 2); }
static bool v1_smooth(const pod2g_ctx* c) { return v1_applies(c) && (c->rows_kernel & 1); }
#define V1_DISPATCH(KIND, ...)                                                             \
    do {                                                                                   \
        if (c->bs == 1) k_rows_v1<1, KIND> __VA_ARGS__;                                    \
        else if (c->bs == 2) k_rows_v1<2, KIND> __VA_ARGS__;                               \
        else k_rows_v1<3, KIND> __VA_ARGS__;                                               \
    } while (0)
static void launch_spmv_v1(pod2g_ctx* c, Dims D, int want) {
    V1_DISPATCH(0, <<<c->grid_spmv, POD2G_THREADS, 0, c->stream>>>(
                       D, want, 0, c->d_row_ptr, c->d_col_idx, c->d_vals32, c->d_dinv32, c->d_pdf, nullptr,
                       c->d_qdf, nullptr, c->d_part, c->d_counters + CNT_SPMV, c->d_sc));
}
static void launch_smooth1_v1(pod2g_ctx* c, Dims D, int want) {
    V1_DISPATCH(1, <<<D.G, POD2G_THREADS, 0, c->stream>>>(
                       D, want, 0, c->d_row_ptr, c->d_col_idx, c->d_vals32, c->d_dinv32, c->d_rdf, nullptr,
                       nullptr, c->d_y32, c->d_part, nullptr, c->d_sc));
}
static void launch_post_v1(pod2g_ctx* c, Dims D, int want) {
    V1_DISPATCH(2, <<<D.G, POD2G_THREADS, 0, c->stream>>>(
                       D, want, c->beta_pr, c->d_row_ptr, c->d_col_idx, c->d_vals32, c->d_dinv32, c->d_rdf,
                       c->d_y32, nullptr, c->d_s32, c->d_part, c->d_counters + CNT_POST, c->d_sc));
}

#define WS_DISPATCH(KIND, ...)                                                            \
    do {                                                                                   \
        const bool two_ = ws_spt(c) == 2;                                                   \
        if (c->bs == 1) {                                                                  \
            if (two_) k_rows_ws<1, 2, KIND> __VA_ARGS__;                                   \
            else k_rows_ws<1, 1, KIND> __VA_ARGS__;                                        \
        } else if (c->bs == 2) {                                                           \
            if (two_) k_rows_ws<2, 2, KIND> __VA_ARGS__;                                   \
            else k_rows_ws<2, 1, KIND> __VA_ARGS__;                                        \
        } else {                                                                           \
            if (two_) k_rows_ws<3, 2, KIND> __VA_ARGS__;                                   \
            else k_rows_ws<3, 1, KIND> __VA_ARGS__;                                        \
        }                                                                                  \
    } while (0)

static void launch_spmv_ws(pod2g_ctx* c, Dims D, int want) {
    const size_t sm = ws_smem(c->bs, c->Bp, ws_spt(c));
    WS_DISPATCH(0, <<<c->grid_spmv, POD2G_THREADS, sm, c->stream>>>(
                       D, want, 0, c->d_row_ptr, c->d_col_idx, c->d_vals32, c->d_dinv32, c->d_pdf, nullptr,
                       c->d_qdf, nullptr, c->d_part, c->d_counters + CNT_SPMV, c->d_sc, c->d_err));
}
static void launch_smooth1_ws(pod2g_ctx* c, Dims D, int want) {
    const size_t sm = ws_smem(c->bs, c->Bp, ws_spt(c));
    WS_DISPATCH(1, <<<D.G, POD2G_THREADS, sm, c->stream>>>(
                       D, want, 0, c->d_row_ptr, c->d_col_idx, c->d_vals32, c->d_dinv32, c->d_rdf, nullptr,
                       nullptr, c->d_y32, c->d_part, nullptr, c->d_sc, c->d_err));
}
static void launch_post_ws(pod2g_ctx* c, Dims D, int want) {
    const size_t sm = ws_smem(c->bs, c->Bp, ws_spt(c));
    WS_DISPATCH(2, <<<D.G, POD2G_THREADS, sm, c->stream>>>(
                       D, want, c->beta_pr, c->d_row_ptr, c->d_col_idx, c->d_vals32, c->d_dinv32, c->d_rdf,
                       c->d_y32, nullptr, c->d_s32, c->d_part, c->d_counters + CNT_POST, c->d_sc, c->d_err));
}
static int ws_set_attributes(pod2g_ctx* c) {
    const void* fns[3] = {nullptr, nullptr, nullptr};
#define WS_FN(BS_, SPT_)                                                   \
    if (c->bs == BS_ && ws_spt(c) == SPT_) {                               \
        fns[0] = (const void*)k_rows_ws<BS_, SPT_, 0>;                     \
        fns[1] = (const void*)k_rows_ws<BS_, SPT_, 1>;                     \
        fns[2] = (const void*)k_rows_ws<BS_, SPT_, 2>;                     \
    }
    WS_FN(1, 1) WS_FN(1, 2) WS_FN(2, 1) WS_FN(2, 2) WS_FN(3, 1) WS_FN(3, 2)
#undef WS_FN
    for (const void* f : fns) {
        if (!f) return POD2G_INVALID_ARG;
        P2G_TRY(allow_max_smem(f));
    }
    return POD2G_OK;
}

// Prolongation + post-smoothing from K Phi (k_postw): available when the context stores W (Jacobi
// relaxation with r1 = r2 = 1), selected by bit 2 of rows_kernel.
static bool kphi_post(const pod2g_ctx* c) { return c->d_W32 && (c->rows_kernel & 4); }
static void launch_postw(pod2g_ctx* c, Dims D, int want) {
    const size_t sm = sizeof(float) * c->Bp * (c->kp + 1);
#define POSTW(KP_)                                                                                          \
    case KP_:                                                                                               \
        k_postw<KP_><<<D.G, POD2G_THREADS, sm, c->stream>>>(D, want, c->beta_pr, c->d_dinv32, c->d_rdf,   \
                                                            c->d_y32, c->d_phi32, c->d_W32, c->d_ec,      \
                                                            c->d_s32, c->d_part, c->d_counters + CNT_POST,  \
                                                            c->d_sc, c->n);                                \
        break;
    switch (c->kp) { KP_LIST(POSTW) }
#undef POSTW
}

// Event-record node after a kernel of a captured iteration (timing mode only).
static int mark(pod2g_ctx* c) {
    P2G_TRY(pod2g_check_launch(c));
    if (c->cap_ev) P2G_CUDA(cudaEventRecordWithFlags(c->cap_ev[c->cap_idx++], c->stream, cudaEventRecordExternal));
    return POD2G_OK;
}

static int elementwise_grid(pod2g_ctx* c, long long total) {
    return std::max(1, std::min(ceil_div(total, POD2G_THREADS), 8 * c->num_sms));
}

// the preconditioner s = AMG(0; K, r, r1, r2) for lanes in state `want`
static int enqueue_precond(pod2g_ctx* c, Dims D, int want) {
    const bool gs = c->smoother == POD2G_SMOOTHER_SGS;
    int st = POD2G_OK;
    if (gs && c->pre) LAUNCH_BS(st = launch_gs, (c, D, want, 0));   // y1: forward sweep from zero, into s
    P2G_TRY(st);
    if (ws_smooth(c) && c->pre == 1) launch_smooth1_ws(c, D, want);
    else if (v1_smooth(c) && c->pre == 1) launch_smooth1_v1(c, D, want);
    else LAUNCH_BS(launch_smooth1, (c, D, want));
    P2G_TRY(mark(c));
    if (c->kp > 0) launch_restrict(c, D, want);
    P2G_TRY(mark(c));
    k_coarse<<<c->Bp, POD2G_THREADS, 0, c->stream>>>(D, want, c->d_part, c->d_cpart, c->d_Lc, c->d_ec, c->d_sc);
    P2G_TRY(mark(c));
    if (kphi_post(c)) {
        // prolongation and post-smoothing in one pass from K Phi (timed as the post-smoothing)
        if (c->cap_ev) P2G_CUDA(cudaEventRecordWithFlags(c->cap_ev[c->cap_idx++], c->stream, cudaEventRecordExternal));
        launch_postw(c, D, want);
        P2G_TRY(mark(c));
        return POD2G_OK;
    }
    launch_prol(c, D, want);
    P2G_TRY(mark(c));
    if (gs && c->post) LAUNCH_BS(st = launch_gs, (c, D, want, 1));  // backward sweep on s in place
    P2G_TRY(st);
    if (ws_smooth(c) && c->post == 1) launch_post_ws(c, D, want);
    else if (v1_smooth(c) && c->post == 1) launch_post_v1(c, D, want);
    else LAUNCH_BS(launch_post, (c, D, want));
    P2G_TRY(mark(c));
    return POD2G_OK;
}

// one PCG iteration (Algorithm 3 loop body) for ACTIVE lanes
static int enqueue_iteration(pod2g_ctx* c, Dims D) {
    const long long total = (long long)c->n * c->Bp;
    const int ge = std::max(1, std::min(ceil_div(total, POD2G_THREADS), c->grid_vec));
    if (c->cap_ev) P2G_CUDA(cudaEventRecordWithFlags(c->cap_ev[c->cap_idx++], c->stream, cudaEventRecordExternal));
    k_p<<<ge, POD2G_THREADS, 0, c->stream>>>(D, SLOT_ACTIVE, c->d_s32, c->d_pdf, c->d_sc, total);
    P2G_TRY(mark(c));
    const ElemOp E = elem_op(c);
    if (ws_spmv(c))
        launch_spmv_ws(c, D, SLOT_ACTIVE);
    else if (v1_spmv(c))
        launch_spmv_v1(c, D, SLOT_ACTIVE);
    else
        LAUNCH_BS(k_spmv, <<<c->grid_spmv, POD2G_THREADS, 0, c->stream>>>(D, SLOT_ACTIVE, c->d_row_ptr, c->d_col_idx,
                                                                 c->d_vals32, E, c->d_pdf, c->d_qdf, c->d_part,
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
    c->grid_rows = batched_grid(c->num_sms, (long long)c->nb * c->Bp);
    c->grid_spmv = c->grid_rows;
    c->grid_restrict = batched_grid(c->num_sms, (long long)2 * c->num_sms * POD2G_THREADS);
    c->grid_prol = 8 * c->num_sms;
    c->grid_vec = 8 * c->num_sms;
    c->rows_kernel = c->d_W32 ? 4 : 0;
    if (v1_applies(c)) {
        // single instance: the group-per-row smoothing kernels by default, and the group-per-row SpMV
        // for 3 x 3 blocks (measured faster than one thread per block row there, slower for 2 x 2
        // blocks); the autotuner compares both forms
        int occ = 0;
        if (c->bs == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_rows_v1<1, 0>, POD2G_THREADS, 0);
        else if (c->bs == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_rows_v1<2, 0>, POD2G_THREADS, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_rows_v1<3, 0>, POD2G_THREADS, 0);
        cudaGetLastError();
        if (occ > 0) {
            c->rows_kernel |= c->bs == 3 ? 3 : 1;
            c->ws_occ = occ;
            // no more CTAs than rows to cover (a group of lanes per row, 256 / LPR rows per CTA)
            const int lpr = 8;
            const int need = ceil_div(c->nb, POD2G_THREADS / lpr);
            c->grid_rows = std::max(CLUSTER, std::min(std::min(8 * c->num_sms, occ * c->num_sms),
                                                      ceil_div(need, CLUSTER) * CLUSTER) / CLUSTER * CLUSTER);
            c->grid_spmv = c->grid_rows;
        }
    }
    if (ws_applies(c)) {
        // staged row kernels by default: one wave of resident CTAs for the row kernels
        P2G_TRY(ws_set_attributes(c));
        int occ = 0;
        const int sm = (int)ws_smem(c->bs, c->Bp, ws_spt(c));
#define WS_OCC(BS_, SPT_)                                                                                   \
        if (c->bs == BS_ && ws_spt(c) == SPT_)                                                              \
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_rows_ws<BS_, SPT_, 0>, POD2G_THREADS, sm);
        WS_OCC(1, 1) WS_OCC(1, 2) WS_OCC(2, 1) WS_OCC(2, 2) WS_OCC(3, 1) WS_OCC(3, 2)
#undef WS_OCC
        cudaGetLastError();
        if (occ > 0) {
            // four waves of resident CTAs (measured faster than one: the hardware keeps every SM
            // fed as 8-CTA clusters retire)
            c->rows_kernel |= 3;
            c->ws_occ = occ;
            // no more CTAs than row groups to cover (8 warps of 32 / LR rows per CTA)
            const int rpw = 32 / (c->Bp / ws_spt(c));
            const int need = ceil_div(c->nb, (POD2G_THREADS / 32) * rpw);
            c->grid_rows = std::max(CLUSTER, std::min(std::min(8 * c->num_sms, 4 * occ * c->num_sms),
                                                      ceil_div(need, CLUSTER) * CLUSTER) / CLUSTER * CLUSTER);
            c->grid_spmv = c->grid_rows;
        }
    }
    // whole iterations in one launch (rows_kernel bit 3): as many CTAs as the rows need (256
    // row-slot items each), all resident at once. Not the default: on the problems measured it was
    // at best at parity with the graph of kernels (a few thousand unknowns) and slower above that;
    // the autotuner selects it where it measures faster
    const int pmax = std::min(persist_max_grid(c), 4 * c->num_sms);
    if (pmax > 0) c->grid_persist = std::max(1, std::min(pmax, ceil_div((long long)c->nb * c->Bp, POD2G_THREADS)));
    if (c->precision != POD2G_FP64 && c->kp > 0) {
        const int sm_r = (int)(restrict_bulk_smem(c) ? restrict_bulk_smem(c) : restrict_smem(c->Bp, c->kp));
        const int lb = restrict_lb(c->Bp, c->kp);
        const int sm_p = c->Bp * (c->kp + 1) * (int)sizeof(float);
        const void* fr = nullptr;
        const void* fp2 = nullptr;
        const void* fp1 = nullptr;
        const void* fp0 = nullptr;
#define FN_LB(KP_, LB_)                                                                    \
        if (c->kp == KP_ && lb == LB_)                                                     \
            fr = restrict_bulk_smem(c) ? (const void*)k_restrict_bulk<KP_, LB_> \
                                       : (const void*)k_restrict<KP_, LB_>;
#define FN_KP(KP_)                                                      \
        LB_LIST(FN_LB, KP_)                                              \
        if (c->kp == KP_) {                                              \
            fp2 = (const void*)k_prol<2, KP_>;                           \
            fp1 = (const void*)k_prol<1, KP_>;                           \
            fp0 = (const void*)k_prol<0, KP_>;                           \
        }
        KP_LIST(FN_KP)
#undef FN_KP
#undef FN_LB
        if (!fr) return POD2G_INVALID_ARG;
        if (sm_r > 227 * 1024 || sm_p > 227 * 1024) return POD2G_INVALID_ARG;
        const void* fw = nullptr;
#define FW_KP(KP_) if (c->kp == KP_) fw = (const void*)k_postw<KP_>;
        KP_LIST(FW_KP)
#undef FW_KP
        if (fw) P2G_TRY(allow_max_smem(fw));
        P2G_TRY(allow_max_smem(fr));
        P2G_TRY(allow_max_smem(fp2));
        P2G_TRY(allow_max_smem(fp1));
        P2G_TRY(allow_max_smem(fp0));
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
    k_load<<<elementwise_grid(c, tot), POD2G_THREADS, 0, c->stream>>>(
        b_dev, x0_dev, d_slots, nslots, c->n, c->Bp, c->d_bdf, c->d_b64, c->d_xdf, c->d_pdf, c->d_qdf, c->d_s32);
    P2G_TRY(pod2g_check_launch(c));
    const ElemOp E = elem_op(c);
    LAUNCH_BS(k_resid, <<<D.G, POD2G_THREADS, 0, c->stream>>>(D, c->d_mask, c->d_row_ptr, c->d_col_idx,
                                                              c->d_vals32, E, c->d_xdf, c->d_bdf, c->d_rdf, c->d_part,
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
        c->tev.resize((size_t)c->chunk * 9);
        for (auto& ev : c->tev) P2G_CUDA(cudaEventCreate(&ev));
    }
    const int64_t l0 = c->launches;
    P2G_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int st = POD2G_OK;
    for (int it = 0; it < c->chunk && st == POD2G_OK; ++it) {
        c->cap_ev = c->timing ? &c->tev[(size_t)it * 9] : nullptr;
        c->cap_idx = 0;
        st = enqueue_iteration(c, D);
    }
    c->cap_ev = nullptr;
    c->iter_launches = (c->launches - l0) / c->chunk;
    c->launches = l0;  // captured, not launched; counted at each replay
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (st != POD2G_OK) return st;
    P2G_CUDA(e);
    e = cudaGraphInstantiate(&c->graph_exec, g, 0);
    cudaGraphDestroy(g);
    P2G_CUDA(e);
    return POD2G_OK;
}

// Whole iterations in one cooperative launch (rows_kernel bit 3; not in per-kernel timing mode).
static bool persist_on(const pod2g_ctx* c) {
    return (c->rows_kernel & 8) && !c->timing && c->grid_persist > 0 && persist_applies(c);
}

// `chunk` PCG iterations for the ACTIVE lanes: one persistent launch, or one replay of
// the captured graph.
static int launch_iterations(pod2g_ctx* c) {
    if (persist_on(c)) {
        P2G_TRY(persist_launch(c, c->chunk));
        c->launches += 1;
        return POD2G_OK;
    }
    P2G_TRY(build_graph(c));
    P2G_CUDA(cudaGraphLaunch(c->graph_exec, c->stream));
    c->launches += c->iter_launches * c->chunk;
    return POD2G_OK;
}

// One launch of `chunk` PCG iterations for the ACTIVE lanes, then the per-slot
// scalars are copied back to the host mirror.
int batched_chunk(pod2g_ctx* c) {
    P2G_TRY(launch_iterations(c));
    P2G_CUDA(cudaMemcpyAsync(c->h_sc, c->d_sc, sizeof(SlotScalars) * c->Bp, cudaMemcpyDeviceToHost, c->stream));
    P2G_CUDA(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    P2G_CUDA(cudaStreamSynchronize(c->stream));
    if (*c->h_err) return POD2G_TIMEOUT;  // a bounded device wait expired
    if (c->timing) {
        for (int it = 0; it < c->chunk; ++it)
            for (int j = 0; j < 8; ++j) {
                float ms = 0.f;
                P2G_CUDA(cudaEventElapsedTime(&ms, c->tev[(size_t)it * 9 + j], c->tev[(size_t)it * 9 + j + 1]));
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
// finishes within maxit iterations, so at most max(maxit)/chunk + 2 launches.
int batched_run(pod2g_ctx* c, const std::vector<int>& lanes) {
    P2G_CUDA(cudaMemcpyAsync(c->h_sc, c->d_sc, sizeof(SlotScalars) * c->Bp, cudaMemcpyDeviceToHost, c->stream));
    P2G_CUDA(cudaStreamSynchronize(c->stream));
    int64_t bound = 2;
    for (int b : lanes) bound = std::max<int64_t>(bound, (int64_t)c->h_sc[b].maxit / c->chunk + 2);
    if (c->spin_limit > 0) bound = std::min<int64_t>(bound, c->spin_limit);
    auto all_done = [&](const SlotScalars* hs) {
        for (int b : lanes)
            if (hs[b].state != SLOT_DONE) return false;
        return true;
    };
    if (c->timing || !c->h_sc2) {
        for (int64_t polls = 0;; ++polls) {
            if (all_done(c->h_sc)) return POD2G_OK;
            if (polls >= bound) return POD2G_TIMEOUT;
            P2G_TRY(batched_chunk(c));
        }
    }
    // One chunk of lookahead: launch k + 1 is queued before the lane states after
    // launch k are examined, so the GPU does not idle during the host's check. Lanes
    // that finished are frozen on the device, so the extra launch changes nothing.
    if (all_done(c->h_sc)) return POD2G_OK;
    SlotScalars* hb[2] = {c->h_sc, c->h_sc2};
    int* he[2] = {c->h_err, c->h_err2};
    auto enqueue = [&](int64_t k) -> int {
        P2G_TRY(launch_iterations(c));
        P2G_CUDA(cudaMemcpyAsync(hb[k & 1], c->d_sc, sizeof(SlotScalars) * c->Bp, cudaMemcpyDeviceToHost, c->stream));
        P2G_CUDA(cudaMemcpyAsync(he[k & 1], c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        P2G_CUDA(cudaEventRecord(c->la_ev[k & 1], c->stream));
        return POD2G_OK;
    };
    P2G_TRY(enqueue(0));
    for (int64_t k = 0;; ++k) {
        const bool ahead = k + 1 < bound;
        if (ahead) P2G_TRY(enqueue(k + 1));
        P2G_CUDA(cudaEventSynchronize(c->la_ev[k & 1]));
        const bool err = *he[k & 1] != 0, done = all_done(hb[k & 1]);
        if (err || done || !ahead) {
            P2G_CUDA(cudaStreamSynchronize(c->stream));
            const int64_t last = ahead ? k + 1 : k;   // the latest copy holds the final states
            if (hb[last & 1] != c->h_sc) std::memcpy(c->h_sc, hb[last & 1], sizeof(SlotScalars) * c->Bp);
            if (err || *he[last & 1]) return POD2G_TIMEOUT;
            return done ? POD2G_OK : POD2G_TIMEOUT;
        }
    }
}

// Lanes that are still iterating when the host gives up (its bounded wait expired) are
// marked DONE with `result`: later launches skip them and their last iterate can be stored.
int batched_retire(pod2g_ctx* c, const std::vector<int>& lanes, int result) {
    P2G_CUDA(cudaStreamSynchronize(c->stream));
    P2G_CUDA(cudaMemcpyAsync(c->h_sc, c->d_sc, sizeof(SlotScalars) * c->Bp, cudaMemcpyDeviceToHost, c->stream));
    P2G_CUDA(cudaStreamSynchronize(c->stream));
    for (int b : lanes)
        if (c->h_sc[b].state != SLOT_DONE) {
            c->h_sc[b].state = SLOT_DONE;
            c->h_sc[b].result = result;
        }
    P2G_CUDA(cudaMemcpyAsync(c->d_sc, c->h_sc, sizeof(SlotScalars) * c->Bp, cudaMemcpyHostToDevice, c->stream));
    P2G_CUDA(cudaStreamSynchronize(c->stream));
    return POD2G_OK;
}

// true FP64 residual for the finished lanes, x out, per-slot results
int batched_finalize(pod2g_ctx* c, int nslots, const int* slots, double* x_dev, int* iters, double* relres,
                     int* status) {
    Dims D = dims_of(c);
    std::vector<int> mask(c->Bp, 0);
    for (int i = 0; i < nslots; ++i) mask[slots[i]] = 1;
    int* d_slots = (int*)(c->d_mask + c->Bp);
    P2G_CUDA(cudaMemcpyAsync(c->d_mask, mask.data(), sizeof(int) * c->Bp, cudaMemcpyHostToDevice, c->stream));
    P2G_CUDA(cudaMemcpyAsync(d_slots, slots, sizeof(int) * nslots, cudaMemcpyHostToDevice, c->stream));
    const ElemOp E = elem_op(c);
    LAUNCH_BS(k_resid64, <<<D.G, POD2G_THREADS, 0, c->stream>>>(D, c->d_mask, c->d_row_ptr, c->d_col_idx,
                                                                c->d_vals32, E, c->d_xdf, c->d_b64, c->d_part,
                                                                c->d_counters + CNT_RESID, c->d_sc));
    P2G_TRY(pod2g_check_launch(c));
    const long long tot = (long long)nslots * c->n;
    k_store<<<elementwise_grid(c, tot), POD2G_THREADS, 0, c->stream>>>(x_dev, d_slots, nslots, c->n, c->Bp, c->d_xdf,
                                                                        c->d_sc);
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

// ---------------------------------------------------------------------------- launch shapes
int batched_set_tuning(pod2g_ctx* c, const pod2g_tuning* t) {
    const int sms = c->num_sms;
    if (t->grid_rows < CLUSTER || t->grid_rows % CLUSTER || t->grid_rows > 8 * sms) return POD2G_INVALID_ARG;
    if (t->grid_spmv < CLUSTER || t->grid_spmv % CLUSTER || t->grid_spmv > 8 * sms) return POD2G_INVALID_ARG;
    if (t->grid_restrict < CLUSTER || t->grid_restrict % CLUSTER || t->grid_restrict > 4 * sms) return POD2G_INVALID_ARG;
    if (t->grid_prol < 1 || t->grid_prol > 8 * sms || t->grid_vec < 1 || t->grid_vec > 8 * sms) return POD2G_INVALID_ARG;
    if (t->rows_kernel < 0 || t->rows_kernel > 15 ||
        ((t->rows_kernel & 3) && !((ws_applies(c) || v1_applies(c)) && c->ws_occ > 0)) ||
        ((t->rows_kernel & 4) && !c->d_W32))
        return POD2G_INVALID_ARG;
    const int pmax = std::min(persist_max_grid(c), 4 * sms);
    if (t->grid_persist < 0 || t->grid_persist > pmax || ((t->rows_kernel & 8) && t->grid_persist < 1))
        return POD2G_INVALID_ARG;
    if (t->restrict_rows != 0 &&
        (t->restrict_rows < 4 || t->restrict_rows > 256 || t->restrict_rows % 4 || c->Bp < 4 || c->kp == 0 ||
         !restrict_bulk_smem_rows(c->Bp, c->kp, t->restrict_rows)))
        return POD2G_INVALID_ARG;
    // a bulk-staged restriction stays bulk-staged (its kernel and attributes were chosen at creation)
    if (t->restrict_rows == 0 && c->Bp >= 4 && c->kp > 0 &&
        !restrict_bulk_smem_rows(c->Bp, c->kp, restrict_bulk_rows_default(c->Bp, c->kp)))
        return POD2G_INVALID_ARG;
    c->restrict_rows = t->restrict_rows;
    c->rows_kernel = t->rows_kernel;
    if (t->grid_persist > 0) c->grid_persist = t->grid_persist;
    c->grid_rows = t->grid_rows;
    c->grid_spmv = t->grid_spmv;
    c->grid_restrict = t->grid_restrict;
    c->grid_prol = t->grid_prol;
    c->grid_vec = t->grid_vec;
    if (c->graph_exec) {
        cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = nullptr;
    }
    return POD2G_OK;
}

// Autotuner: run `iters` iterations of the given (set-up) slots for each of a few
// candidate launch shapes, timing every kernel with CUDA events inside the graph,
// and keep per kernel group the fastest shape: outer SpMV, smoother row kernels
// (k_smooth1 + k_post), restriction, prolongation, vector updates (k_p + k_upd). The slots are
// left idle. The result depends on measured times; a given shape gives
// deterministic results, and shapes differ only in the summation order of partials.
int batched_autotune(pod2g_ctx* c, int nslots, const int* slots, const double* b_dev, int iters) {
    const int sms = c->num_sms;
    const int NC = 5;
    auto r8 = [&](int g, int cap) { return std::max(CLUSTER, std::min(cap, g) / CLUSTER * CLUSTER); };
    const int need_rows = batched_grid(sms, (long long)c->nb * c->Bp);
    const int need_vec = std::max(1, ceil_div((long long)c->n * c->Bp, POD2G_THREADS));
    const int row_f[NC] = {3, 4, 5, 6, 8}, res_f[NC] = {1, 2, 3, 4, 4}, vec_f[NC] = {2, 3, 4, 6, 8};
    pod2g_tuning cand[NC];
    for (int j = 0; j < NC; ++j) {
        cand[j] = pod2g_tuning();
        cand[j].restrict_rows = 0;
        cand[j].grid_rows = r8(row_f[j] * sms, need_rows);
        cand[j].grid_spmv = cand[j].grid_rows;
        cand[j].grid_restrict = r8(res_f[j] * sms, 4 * sms);
        cand[j].grid_prol = std::min(vec_f[j] * sms, need_vec);
        cand[j].grid_vec = std::min(vec_f[j] * sms, need_vec);
    }
    // the warp-staged row kernels (where they apply) with one to eight waves of resident CTAs
    const bool ws = (ws_applies(c) || v1_applies(c)) && c->ws_occ > 0;
    const int wave = c->ws_occ * sms;
    const int ws_f[NC] = {1, 2, 3, 4, 8};
    pod2g_tuning cand_ws[NC];
    const int kbit = c->rows_kernel & 4;   // the K Phi form of the post-smoothing is kept as set
    const int gpers = c->grid_persist;
    for (int j = 0; j < NC; ++j) {
        cand[j].rows_kernel = kbit;
        cand[j].grid_persist = gpers;
        cand_ws[j] = cand[j];
        cand_ws[j].rows_kernel = 3 | kbit;
        cand_ws[j].grid_rows = r8(ws_f[j] * wave, 8 * sms);
        cand_ws[j].grid_spmv = cand_ws[j].grid_rows;
    }
    const bool timing0 = c->timing;
    std::vector<double> tol(nslots, 0.0);
    std::vector<int> maxit(nslots, iters + 16 * c->chunk);
    std::vector<int> lanes(slots, slots + nslots);
    double t_rows[2 * NC], t_spmv[2 * NC], t_res[NC], t_prol[NC], t_vec[NC];
    for (int j = 0; j < 2 * NC; ++j) t_rows[j] = t_spmv[j] = 1e300;
    for (int j = 0; j < NC && ws; ++j) {
        P2G_TRY(batched_set_tuning(c, &cand_ws[j]));
        P2G_TRY(batched_set_timing(c, 1));
        P2G_TRY(batched_load(c, nslots, slots, b_dev, nullptr, tol.data(), maxit.data()));
        for (int it = 0; it < iters; it += c->chunk) P2G_TRY(batched_chunk(c));
        auto per = [&](int k) { return c->kt_n[k] ? c->kt_ms[k] / (double)c->kt_n[k] : 0.0; };
        t_spmv[NC + j] = per(1);
        t_rows[NC + j] = per(3) + per(7);
    }
    for (int j = 0; j < NC; ++j) {
        P2G_TRY(batched_set_tuning(c, &cand[j]));
        P2G_TRY(batched_set_timing(c, 1));
        P2G_TRY(batched_load(c, nslots, slots, b_dev, nullptr, tol.data(), maxit.data()));
        for (int it = 0; it < iters; it += c->chunk) P2G_TRY(batched_chunk(c));
        auto per = [&](int k) { return c->kt_n[k] ? c->kt_ms[k] / (double)c->kt_n[k] : 0.0; };
        t_vec[j] = per(0) + per(2);               // k_p, k_upd
        t_spmv[j] = per(1);                       // k_spmv
        t_rows[j] = per(3) + per(7);              // k_smooth1, k_post
        t_res[j] = per(4);                        // k_restrict
        t_prol[j] = per(6);                       // k_prol
    }
    auto best = [&](const double* t, int m) {
        int b = 0;
        for (int j = 1; j < m; ++j)
            if (t[j] < t[b]) b = j;
        return b;
    };
    auto row_cand = [&](int j) -> const pod2g_tuning& { return j < NC ? cand[j] : cand_ws[j - NC]; };
    pod2g_tuning pick = pod2g_tuning();
    const int br = best(t_rows, 2 * NC), bsp = best(t_spmv, 2 * NC);
    pick.grid_rows = row_cand(br).grid_rows;
    pick.grid_spmv = row_cand(bsp).grid_spmv;
    pick.rows_kernel = (br >= NC ? 1 : 0) | (bsp >= NC ? 2 : 0) | (c->rows_kernel & 4);
    pick.grid_restrict = cand[best(t_res, NC)].grid_restrict;
    pick.grid_prol = cand[best(t_prol, NC)].grid_prol;
    pick.grid_vec = cand[best(t_vec, NC)].grid_vec;
    pick.restrict_rows = 0;
    // the restriction's rows per staged chunk (its Phi / r1 tile): half, the default and twice
    const int R0 = restrict_bulk_rows_default(c->Bp, c->kp);
    if (R0 > 0) {
        double best_t = t_res[best(t_res, NC)];
        for (int f = 0; f < 2; ++f) {
            const int R = f == 0 ? std::max(4, R0 / 2 / 4 * 4) : std::min(256, R0 * 2);
            if (R == R0 || !restrict_bulk_smem_rows(c->Bp, c->kp, R)) continue;
            pod2g_tuning tr = pick;
            tr.restrict_rows = R;
            P2G_TRY(batched_set_tuning(c, &tr));
            P2G_TRY(batched_set_timing(c, 1));
            P2G_TRY(batched_load(c, nslots, slots, b_dev, nullptr, tol.data(), maxit.data()));
            for (int it = 0; it < iters; it += c->chunk) P2G_TRY(batched_chunk(c));
            const double tr_ms = c->kt_n[4] ? c->kt_ms[4] / (double)c->kt_n[4] : 1e300;
            if (tr_ms < best_t) {
                best_t = tr_ms;
                pick.restrict_rows = R;
            }
        }
    }
    // whole launches: the graph of the chosen shape against the persistent launch at up to
    // four grid sizes (the rows' need, one and two CTAs per SM, every resident CTA), each timed
    // over `iters` iterations with CUDA events around the launches
    const int pmax = std::min(persist_max_grid(c), 4 * sms);
    pick.grid_persist = pmax > 0 ? c->grid_persist : 0;
    if (pmax > 0) {
        cudaEvent_t e0, e1;
        P2G_CUDA(cudaEventCreate(&e0));
        P2G_CUDA(cudaEventCreate(&e1));
        auto per_iter = [&](const pod2g_tuning& t, double* ms) -> int {
            P2G_TRY(batched_set_tuning(c, &t));
            P2G_TRY(batched_set_timing(c, 0));
            P2G_TRY(batched_load(c, nslots, slots, b_dev, nullptr, tol.data(), maxit.data()));
            P2G_TRY(batched_chunk(c));  // warm-up (graph instantiation)
            P2G_CUDA(cudaEventRecord(e0, c->stream));
            int n_it = 0;
            for (int it = 0; it < iters; it += c->chunk, n_it += c->chunk) P2G_TRY(batched_chunk(c));
            P2G_CUDA(cudaEventRecord(e1, c->stream));
            P2G_CUDA(cudaEventSynchronize(e1));
            float f = 0.f;
            P2G_CUDA(cudaEventElapsedTime(&f, e0, e1));
            *ms = (double)f / std::max(1, n_it);
            return POD2G_OK;
        };
        int st = POD2G_OK;
        double t_best = 1e300;
        pod2g_tuning tg = pick;
        tg.rows_kernel &= 7;
        st = per_iter(tg, &t_best);
        const int need = std::max(1, ceil_div((long long)c->nb * c->Bp, POD2G_THREADS));
        const int gp[4] = {std::min(need, pmax), std::min(sms, pmax), std::min(2 * sms, pmax), pmax};
        for (int j = 0; j < 4 && st == POD2G_OK; ++j) {
            bool seen = false;
            for (int i = 0; i < j; ++i) seen |= gp[i] == gp[j];
            if (seen) continue;
            pod2g_tuning tp = tg;
            tp.rows_kernel |= 8;
            tp.grid_persist = gp[j];
            double ms = 1e300;
            st = per_iter(tp, &ms);
            if (st == POD2G_OK && ms < t_best) {
                t_best = ms;
                pick = tp;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        P2G_TRY(st);
    }
    P2G_TRY(batched_set_tuning(c, &pick));
    P2G_TRY(batched_set_timing(c, timing0 ? 1 : 0));
    // leave the slots idle
    P2G_CUDA(cudaMemcpyAsync(c->h_sc, c->d_sc, sizeof(SlotScalars) * c->Bp, cudaMemcpyDeviceToHost, c->stream));
    P2G_CUDA(cudaStreamSynchronize(c->stream));
    for (int b : lanes) c->h_sc[b].state = SLOT_IDLE;
    P2G_CUDA(cudaMemcpyAsync(c->d_sc, c->h_sc, sizeof(SlotScalars) * c->Bp, cudaMemcpyHostToDevice, c->stream));
    P2G_CUDA(cudaStreamSynchronize(c->stream));
    return POD2G_OK;
}
