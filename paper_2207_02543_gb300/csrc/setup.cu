// Per-instance set-up (one slot): matrix values into the solver's layout, the
// Jacobi diagonal D^{-1}, the Galerkin coarse matrix K_c = Phi^T K Phi
// (arXiv 2207.02543, Section 3.3, eq. POD_ROM) symmetrised, and its Cholesky
// factor in FP64 (the k x k coarse solve of Algorithm 2 with P = Phi_r).
//
// Mixed paths: K Phi is formed in double-float from FP32 values and the FP32 (or
// BF16-rounded) basis, whose products are exact; the contraction Phi^T (K Phi)
// accumulates double-float per thread and FP64 across threads and CTAs. K Phi
// of a smooth mode is ~h^2 smaller than |K||Phi|, so FP32 accumulation would lose
// most digits of K_c; double-float keeps ~14.
// FP64 path: the same steps in FP64.
#include "common.cuh"

namespace {

// values (FP64, one instance, [nnzb][bs*bs]) -> FP32 contiguous copy and (vals32
// not null) the slot's lane of the interleaved array [nnzb*bs*bs][Bp]
__global__ void k_convert_values(const double* __restrict__ v64, float* __restrict__ v32_stage,
                                 float* __restrict__ vals32, long long total, int Bp, int slot) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        float v = __double2float_rn(v64[e]);
        v32_stage[e] = v;
        if (vals32) vals32[e * Bp + slot] = v;
    }
}

// D^{-1}: one thread per unknown. status[0] set to NOT_SPD on a non-positive or
// non-finite diagonal entry.
template <typename V>
__global__ void k_dinv(const V* __restrict__ vals, const int32_t* __restrict__ diag_blk, int nb, int bs,
                       double* __restrict__ dinv64, float* __restrict__ dinv32, int Bp, int slot,
                       int* __restrict__ status) {
    int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= nb * bs) return;
    int i = d / bs, rr = d - i * bs;
    double a = (double)vals[(long long)diag_blk[i] * bs * bs + rr * bs + rr];
    if (!(a > 0.0) || !isfinite(a)) {
        atomicCAS(status, (int)POD2G_OK, (int)POD2G_NOT_SPD);
        a = 1.0;
    }
    if (dinv64) dinv64[d] = 1.0 / a;
    if (dinv32) dinv32[(long long)d * Bp + slot] = (float)(1.0 / a);
}

// Several instances at once (more than 8): FP64 values [nslots][tot] -> FP32 lanes slots[i] of the
// interleaved array, through a 32 x 32 shared-memory tile so that both the reads
// (along entries) and the writes (along slots) are coalesced.
__global__ void k_interleave(const double* __restrict__ v64, long long tot, int nslots, const int* __restrict__ slots,
                             int Bp, float* __restrict__ vals32) {
    __shared__ float tile[32][33];
    const long long e0 = (long long)blockIdx.x * 32;
    const int s0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int i = s0 + k;
        const long long e = e0 + threadIdx.x;
        if (i < nslots && e < tot) tile[k][threadIdx.x] = __double2float_rn(v64[(long long)i * tot + e]);
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int i = s0 + threadIdx.x;
        const long long e = e0 + k;
        if (i < nslots && e < tot) vals32[e * Bp + slots[i]] = tile[threadIdx.x][k];
    }
}

// Few instances (<= 8): FP64 values [nslots][tot] -> FP32 lanes, a thread per entry e reading the
// instances' e-th values (coalesced along e) and writing them to its lanes of row e.
__global__ void k_interleave_few(const double* __restrict__ v64, long long tot, int nslots,
                                 const int* __restrict__ slots, int Bp, float* __restrict__ vals32) {
    int sl[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) sl[i] = i < nslots ? slots[i] : 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (i < nslots) v[i] = __double2float_rn(v64[(long long)i * tot + e]);
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (i < nslots) vals32[e * Bp + sl[i]] = v[i];
    }
}

// W = K Phi, double-float, one thread per (unknown row, group of 8 modes): the row's
// values are read once for the 8 modes; each output accumulates in the same order as
// a thread per output would.
__global__ void k_w_df8(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                        const float* __restrict__ v32, const float* __restrict__ phi, int nb, int bs, int kp,
                        float2* __restrict__ W) {
    const int groups = kp / 8;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long total = (long long)nb * bs * groups;
    if (t >= total) return;
    const int g = (int)(t % groups);
    const long long d = t / groups;
    const int i = (int)(d / bs), rr = (int)(d - (long long)i * bs);
    float hi[8], lo[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) { hi[m] = 0.f; lo[m] = 0.f; }
    for (int blk = row_ptr[i]; blk < row_ptr[i + 1]; ++blk) {
        const int j = col_idx[blk];
        const float* vb = v32 + (long long)blk * bs * bs + rr * bs;
        for (int cc = 0; cc < bs; ++cc) {
            const float v = vb[cc];
            const float4* ph = reinterpret_cast<const float4*>(phi + ((long long)j * bs + cc) * kp + 8 * g);
            const float4 f0 = __ldg(ph), f1 = __ldg(ph + 1);
            const float f[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
#pragma unroll
            for (int m = 0; m < 8; ++m) df_acc_fma(hi[m], lo[m], v, f[m], 0.f);
        }
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) W[d * kp + 8 * g + m] = df_norm(hi[m], lo[m]);
}

// W = K Phi in FP64.
__global__ void k_w_f64(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                        const double* __restrict__ v64, const double* __restrict__ phi, int nb, int bs, int kp,
                        double* __restrict__ W) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long total = (long long)nb * bs * kp;
    if (t >= total) return;
    int m = (int)(t % kp);
    long long d = t / kp;
    int i = (int)(d / bs), rr = (int)(d - (long long)i * bs);
    double acc = 0.0;
    for (int blk = row_ptr[i]; blk < row_ptr[i + 1]; ++blk) {
        int j = col_idx[blk];
        const double* vb = v64 + (long long)blk * bs * bs + rr * bs;
        for (int cc = 0; cc < bs; ++cc) acc = fma(vb[cc], phi[((long long)j * bs + cc) * kp + m], acc);
    }
    W[d * kp + m] = acc;
}

// W = K Phi (double-float [n][kp]) -> the slot's lane of the FP32 copy, mode-major [kp][n][Bp], used by
// the post-smoothing pass that forms K y2 from it. A CTA transposes tiles of 64 unknowns through shared
// memory: it reads their rows of W as one contiguous run and writes each mode's 64 entries together.
__global__ void k_w32(const float2* __restrict__ W, long long n, int kp, int Bp, int slot, float* __restrict__ W32) {
    __shared__ float tile[64][POD2G_MAX_K + 1];
    for (long long d0 = (long long)blockIdx.x * 64; d0 < n; d0 += (long long)gridDim.x * 64) {
        const int rows = (int)min(64LL, n - d0);
        __syncthreads();
        for (int e = threadIdx.x; e < rows * kp; e += blockDim.x) {
            const float2 w = W[d0 * kp + e];
            tile[e / kp][e % kp] = __fadd_rn(w.x, w.y);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < rows * kp; e += blockDim.x) {
            const int m = e / rows, dd = e - m * rows;
            W32[((long long)m * n + d0 + dd) * Bp + slot] = tile[dd][m];
        }
    }
}

// Element coefficients (FP64, one instance) -> the slot's lane of the FP32
// interleaved array; status NONFINITE on a NaN or Inf.
__global__ void k_coef_convert(const double* __restrict__ c64, float* __restrict__ coef32, int n_el, int Bp,
                               int slot, int* __restrict__ status) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_el; e += gridDim.x * blockDim.x) {
        const double v = c64[e];
        if (!isfinite(v)) atomicCAS(status, (int)POD2G_OK, (int)POD2G_NONFINITE);
        coef32[(long long)e * Bp + slot] = __double2float_rn(v);
    }
}

// Parametrized coefficients of one instance: c_e = exp(mu + sigma * (modes[e] . theta))
// (lognormal) or mu + sigma * (modes[e] . theta), in FP64, into the slot's FP32 lane.
// status: NONFINITE for a non-finite c_e, NOT_SPD for c_e <= 0 (first error kept).
__global__ void k_field_coef(const double* __restrict__ modes, const double* __restrict__ theta, int m, double mu,
                             double sigma, int lognormal, float* __restrict__ coef32, int n_el, int Bp, int slot,
                             int* __restrict__ status) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_el; e += gridDim.x * blockDim.x) {
        double g = 0.0;
        for (int j = 0; j < m; ++j) g = fma(modes[(long long)e * m + j], theta[j], g);
        const double v = lognormal ? exp(mu + sigma * g) : mu + sigma * g;
        if (!isfinite(v)) atomicCAS(status, (int)POD2G_OK, (int)POD2G_NONFINITE);
        else if (!(v > 0.0)) atomicCAS(status, (int)POD2G_OK, (int)POD2G_NOT_SPD);
        coef32[(long long)e * Bp + slot] = __double2float_rn(v);
    }
}

// The FP32 values of one slot's element operator, contiguous [nnzb][bs*bs]
// (one thread per block row), from the same block-value routine the solver's
// row kernels use.
template <int BS>
__global__ void k_elem_stage(ElemOp E, const int32_t* __restrict__ row_ptr, int nb, int Bp, int slot,
                             float* __restrict__ stage32) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
        float ce[POD2G_ELEM_RE];
        elem_row_coefs(E, i, slot, Bp, ce);
        for (int blk = row_ptr[i]; blk < row_ptr[i + 1]; ++blk) {
            float v[BS * BS];
            elem_block_values<BS>(E.desc[blk], ce, E.kref, v);
#pragma unroll
            for (int e = 0; e < BS * BS; ++e) stage32[(long long)blk * BS * BS + e] = v[e];
        }
    }
}

// Last CTA of a K_c contraction: sum the nparts partial k x k matrices in part order
// (deterministic), symmetrise into Lout, and factor it in place (lower triangle) in FP64.
// A pivot below 64 eps times its original diagonal entry means K_c is numerically singular
// (e.g. linearly dependent modes) and is reported as not SPD.
__device__ void ac_reduce_factor(const double* part, int nparts, int k, double* Ac, double* Lout, int* status) {
    const int npairs = k * k;
    for (int pr = threadIdx.x; pr < npairs; pr += blockDim.x) {
        double s = 0.0;
        for (int g = 0; g < nparts; ++g) s += part[(long long)g * npairs + pr];
        Ac[pr] = s;
    }
    __syncthreads();
    // symmetrise into L (lower triangle used)
    for (int pr = threadIdx.x; pr < npairs; pr += blockDim.x) {
        int i = pr / k, j = pr - i * k;
        Lout[pr] = 0.5 * (Ac[i * k + j] + Ac[j * k + i]);
    }
    __syncthreads();
    // right-looking Cholesky in place (lower triangle), FP64
    __shared__ int fail;
    __shared__ double diag0[POD2G_MAX_K];
    if (threadIdx.x == 0) fail = 0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) diag0[j] = Lout[j * k + j];
    __syncthreads();
    for (int j = 0; j < k; ++j) {
        if (threadIdx.x == 0) {
            double d = Lout[j * k + j];
            if (!(d > 64.0 * 2.220446049250313e-16 * diag0[j]) || !isfinite(d)) { fail = 1; d = 1.0; }
            Lout[j * k + j] = sqrt(d);
        }
        __syncthreads();
        double ljj = Lout[j * k + j];
        for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) Lout[i * k + j] /= ljj;
        __syncthreads();
        int m = k - j - 1;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            int i = j + 1 + e / m, t = j + 1 + e % m;
            if (t <= i) Lout[i * k + t] -= Lout[i * k + j] * Lout[t * k + j];
        }
        __syncthreads();
    }
    for (int pr = threadIdx.x; pr < npairs; pr += blockDim.x) {
        int i = pr / k, j = pr - i * k;
        if (j > i) Lout[pr] = 0.0;
    }
    if (threadIdx.x == 0 && fail) atomicCAS(status, (int)POD2G_OK, (int)POD2G_NOT_SPD);
}

#define AC_TILE 32

// Contraction K_c = Phi^T W (k x k), split over CTAs along the n rows; the last
// CTA sums the partials in CTA order (deterministic), symmetrises, and factors
// K_c = L L^T in FP64. status gets NOT_SPD if a pivot is not positive.
template <bool DF>
__global__ void k_ac(const void* __restrict__ phi_v, const void* __restrict__ W_v, long long n, int k, int kp,
                     double* __restrict__ part, unsigned* counter, double* __restrict__ Ac,
                     double* __restrict__ Lout, int* __restrict__ status) {
    // tile of AC_TILE rows of Phi and W in shared memory; FP64 path uses s_d*,
    // double-float path s_f* (Phi as float, W as (hi, lo) floats)
    __shared__ double s_dphi[DF ? 1 : AC_TILE][POD2G_MAX_K];
    __shared__ double s_dw[DF ? 1 : AC_TILE][POD2G_MAX_K];
    __shared__ float s_fphi[DF ? AC_TILE : 1][POD2G_MAX_K];
    __shared__ float2 s_fw[DF ? AC_TILE : 1][POD2G_MAX_K];
    const int npairs = k * k;
    const int per = (npairs + blockDim.x - 1) / blockDim.x;  // pairs per thread (<= 16)
    double acc[16];
    float acc_hi[16], acc_lo[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) { acc[q] = 0.0; acc_hi[q] = 0.f; acc_lo[q] = 0.f; }
    long long rows_per_cta = (n + gridDim.x - 1) / gridDim.x;
    long long r0 = blockIdx.x * rows_per_cta, r1 = min(n, r0 + rows_per_cta);
    for (long long base = r0; base < r1; base += AC_TILE) {
        int cnt = (int)min((long long)AC_TILE, r1 - base);
        __syncthreads();
        for (int e = threadIdx.x; e < AC_TILE * k; e += blockDim.x) {
            int rr = e / k, m = e - rr * k;
            long long idx = (base + rr) * kp + m;
            if (DF) {
                s_fphi[rr][m] = rr < cnt ? ((const float*)phi_v)[idx] : 0.f;
                s_fw[rr][m] = rr < cnt ? ((const float2*)W_v)[idx] : make_float2(0.f, 0.f);
            } else {
                s_dphi[rr][m] = rr < cnt ? ((const double*)phi_v)[idx] : 0.0;
                s_dw[rr][m] = rr < cnt ? ((const double*)W_v)[idx] : 0.0;
            }
        }
        __syncthreads();
        for (int q = 0; q < per; ++q) {
            int pr = threadIdx.x + q * blockDim.x;
            if (pr >= npairs) break;
            int m1 = pr / k, m2 = pr - m1 * k;
            if (DF) {
                // products Phi (FP32) x W (double-float) accumulated in double-float
                float hi = acc_hi[q], lo = acc_lo[q];
                for (int rr = 0; rr < cnt; ++rr) {
                    float2 w = s_fw[rr][m2];
                    df_acc_fma(hi, lo, s_fphi[rr][m1], w.x, w.y);
                }
                acc_hi[q] = hi;
                acc_lo[q] = lo;
            } else {
                double a = acc[q];
                for (int rr = 0; rr < cnt; ++rr) a = fma(s_dphi[rr][m1], s_dw[rr][m2], a);
                acc[q] = a;
            }
        }
    }
    for (int q = 0; q < per; ++q) {
        int pr = threadIdx.x + q * blockDim.x;
        if (pr >= npairs) break;
        part[(long long)blockIdx.x * npairs + pr] = DF ? ((double)acc_hi[q] + (double)acc_lo[q]) : acc[q];
    }
    if (!last_cta_arrive(counter)) return;
    ac_reduce_factor(part, gridDim.x, k, Ac, Lout, status);
    last_cta_reset(counter);
}


// ---------------------------------------------------------------------------- K_c on the tensor cores
// K_c = Phi^T W (W = K Phi, double-float) as a dense contraction over the n rows on the
// 5th-generation tensor cores (tcgen05.mma, BF16 operands, FP32 accumulation in tensor
// memory). Each FP32 operand is split into three BF16 pieces, x = x1 + x2 + x3 exactly
// (8 significant bits each; for W the high word, its low word being below the kept
// terms); the products x_p y_q with p + q <= 2 (six per K-step) carry every bit down to
// ~2^-24 of each term, as the split-precision tensor-core products of Ootomo and Yokota
// (2022) do. Per CTA: a contiguous range of rows, in stages of TC_KT rows; the threads
// load a stage (issued while the previous one is being stored), split it and store the
// pieces into shared memory in the no-swizzle K-major layout (8 x 16-byte core matrices),
// one thread issues the MMAs of the stage
// (TC_KT / 16 K-steps x 6 products) into one 128 x N FP32 accumulator in tensor memory
// and commits them to an mbarrier, and the stage buffer is refilled only after that
// barrier fires (two buffers). At the end each warp reads its 32 accumulator rows
// (tcgen05.ld), the CTA writes its FP64 partial and the last CTA reduces and factors as
// k_ac does. The accumulator sums at most rows-per-CTA terms in FP32.
#define TC_KT 64                // rows per stage
#define TC_M 128                // MMA rows (modes of Phi; rows >= k are zero)
#define TC_THREADS 128          // four warps: one per 32-lane quarter of tensor memory
#define TC_NP 3                 // BF16 pieces per operand

__device__ __forceinline__ uint32_t s_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, K-major; lbo = byte distance of core
// matrices adjacent along K, sbo = along M / N
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of tcgen05
    return d;                // base offset 0, layout type 0 (no swizzle)
}
// instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major, M x N
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool tc_wait(uint64_t* bar, unsigned parity) {
    const uint32_t a = s_addr(bar);
    for (unsigned t = 0; t < (1u << 22); ++t) {
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
// three BF16 pieces of an FP32 value (exact: x = p0 + p1 + p2)
__device__ __forceinline__ void bf16_split3(float x, __nv_bfloat16 (&p)[TC_NP]) {
    p[0] = __float2bfloat16_rn(x);
    const float r1 = __fsub_rn(x, __bfloat162float(p[0]));
    p[1] = __float2bfloat16_rn(r1);
    p[2] = __float2bfloat16_rn(__fsub_rn(r1, __bfloat162float(p[1])));
}

// shared-memory bytes of k_ac_tc for N accumulator columns
__host__ __device__ constexpr size_t tc_smem_a() { return (size_t)TC_NP * TC_KT * TC_M * 2; }
__host__ __device__ constexpr size_t tc_smem_b(int N) { return (size_t)TC_NP * TC_KT * N * 2; }
static size_t tc_smem(int N) { return 2 * (tc_smem_a() + tc_smem_b(N)) + 64; }

__global__ void __launch_bounds__(TC_THREADS)
k_ac_tc(const float* __restrict__ phi, const float2* __restrict__ W, long long n, int k, int kp, int N,
        double* __restrict__ part, unsigned* counter, double* __restrict__ Ac, double* __restrict__ Lout,
        int* __restrict__ status) {
    extern __shared__ __align__(128) unsigned char tc_raw[];
    // [buffer][piece][K/8][M/8][8 rows x 16 B] for A = Phi^T, [buffer][piece][K/8][N/8][128 B] for B = W
    unsigned char* sA = tc_raw;
    unsigned char* sB = tc_raw + 2 * tc_smem_a();
    uint64_t* bars = reinterpret_cast<uint64_t*>(tc_raw + 2 * (tc_smem_a() + tc_smem_b(N)));
    uint32_t* s_taddr = reinterpret_cast<uint32_t*>(bars + 2);
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t LBO_A = (TC_M / 8) * 128, LBO_B = (uint32_t)(N / 8) * 128;
    const size_t PIECE_A = (size_t)(TC_KT / 8) * LBO_A, PIECE_B = (size_t)(TC_KT / 8) * LBO_B;
    // zero both buffers once: rows of A beyond k and columns of B beyond k stay zero
    for (size_t e = tid; e < 2 * (tc_smem_a() + tc_smem_b(N)) / 16; e += TC_THREADS)
        reinterpret_cast<uint4*>(tc_raw)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_addr(bars)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_addr(bars + 1)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(s_addr(s_taddr))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *s_taddr;
    const uint32_t idesc = tc_idesc(TC_M, N);
    const long long per = (n + gridDim.x - 1) / gridDim.x;
    const long long r0 = min(n, (long long)blockIdx.x * per), r1 = min(n, r0 + per);
    const int nst = (int)((r1 - r0 + TC_KT - 1) / TC_KT);
    bool bad = false;
    // two consecutive rows of one mode per item (a 32-bit word, two K positions, per piece); a
    // thread's items of the next stage are loaded into registers while the current one is stored
    constexpr int TC_ITEMS = (TC_KT / 2) * POD2G_MAX_K / TC_THREADS;
    const int nitems = (TC_KT / 2) * kp;
    float pf[TC_ITEMS][4];
    auto load_stage = [&](int st) {
        const long long base = r0 + (long long)st * TC_KT;
#pragma unroll
        for (int u = 0; u < TC_ITEMS; ++u) {
            const int e = tid + u * TC_THREADS;
            const int q = e / kp, m = e - q * kp;
            const long long i0 = base + 2 * q, i1 = i0 + 1;
            const bool ok = e < nitems && m < k;
            pf[u][0] = ok && i0 < r1 ? __ldg(phi + i0 * kp + m) : 0.f;
            pf[u][1] = ok && i1 < r1 ? __ldg(phi + i1 * kp + m) : 0.f;
            pf[u][2] = ok && i0 < r1 ? W[i0 * kp + m].x : 0.f;
            pf[u][3] = ok && i1 < r1 ? W[i1 * kp + m].x : 0.f;
        }
    };
    if (nst > 0) load_stage(0);
    for (int st = 0; st < nst; ++st) {
        const int buf = st & 1;
        if (st >= 2 && !tc_wait(bars + buf, (unsigned)((st - 2) >> 1) & 1u)) bad = true;
        unsigned char* A = sA + buf * tc_smem_a();
        unsigned char* B = sB + buf * tc_smem_b(N);
#pragma unroll
        for (int u = 0; u < TC_ITEMS; ++u) {
            const int e = tid + u * TC_THREADS;
            const int q = e / kp, m = e - q * kp;
            if (e >= nitems || m >= k) continue;
            const int kk = 2 * q;
            const float f0 = pf[u][0], f1 = pf[u][1], w0 = pf[u][2], w1 = pf[u][3];
            __nv_bfloat16 a0[TC_NP], a1[TC_NP], b0[TC_NP], b1[TC_NP];
            bf16_split3(f0, a0);
            bf16_split3(f1, a1);
            bf16_split3(w0, b0);
            bf16_split3(w1, b1);
            const uint32_t in_core = (uint32_t)((m & 7) * 16 + (kk & 7) * 2);
            const size_t offA = (size_t)(kk >> 3) * LBO_A + (size_t)(m >> 3) * 128 + in_core;
            const size_t offB = (size_t)(kk >> 3) * LBO_B + (size_t)(m >> 3) * 128 + in_core;
#pragma unroll
            for (int p = 0; p < TC_NP; ++p) {
                __nv_bfloat162 va, vb;
                va.x = a0[p]; va.y = a1[p];
                vb.x = b0[p]; vb.y = b1[p];
                *reinterpret_cast<__nv_bfloat162*>(A + p * PIECE_A + offA) = va;
                *reinterpret_cast<__nv_bfloat162*>(B + p * PIECE_B + offB) = vb;
            }
        }
        if (st + 1 < nst) load_stage(st + 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = s_addr(A), b0 = s_addr(B);
#pragma unroll
            for (int ks = 0; ks < TC_KT / 16; ++ks) {
#pragma unroll
                for (int p = 0; p < TC_NP; ++p)
#pragma unroll
                    for (int q = 0; q + p < TC_NP; ++q) {
                        const uint64_t da = tc_desc(a0 + (uint32_t)(p * PIECE_A) + 2 * ks * LBO_A, LBO_A, 128);
                        const uint64_t db = tc_desc(b0 + (uint32_t)(q * PIECE_B) + 2 * ks * LBO_B, LBO_B, 128);
                        tc_mma(tmem, da, db, idesc, (st > 0 || ks > 0 || p > 0 || q > 0) ? 1u : 0u);
                    }
            }
            tc_commit(bars + buf);
        }
    }
    // wait for the last stage's MMAs (a commit tracks every earlier MMA of the thread)
    if (nst > 0 && !tc_wait(bars + ((nst - 1) & 1), (unsigned)((nst - 1) >> 1) & 1u)) bad = true;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // accumulator rows 32*warp .. 32*warp+31 (modes m1), columns m2 < N
    const int m1 = warp * 32 + (tid & 31);
    double* prt = part + (long long)blockIdx.x * k * k;
    for (int c0 = 0; c0 < N; c0 += 16) {
        uint32_t v[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
            "%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (m1 < k)
            for (int j = 0; j < 16 && c0 + j < k; ++j)
                prt[(long long)m1 * k + c0 + j] = nst > 0 ? (double)__uint_as_float(v[j]) : 0.0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
    if (bad && tid == 0) atomicCAS(status, (int)POD2G_OK, (int)POD2G_TIMEOUT);
    if (!last_cta_arrive(counter)) return;
    ac_reduce_factor(part, gridDim.x, k, Ac, Lout, status);
    last_cta_reset(counter);
}
}  // namespace

// Mixed paths: D^-1, K Phi, K_c and its Cholesky factor from the slot's FP32 values in d_stage32.
static int setup_from_stage32(pod2g_ctx* c, int slot, int* st) {
    const int T = POD2G_THREADS;
    const int n = c->n;
    const float* stage32 = c->d_stage32;
    double* L = c->d_Lc + (size_t)slot * c->k * c->k;
    k_dinv<float><<<ceil_div(n, T), T, 0, c->stream>>>(stage32, c->d_diag_blk, c->nb, c->bs, nullptr, c->d_dinv32,
                                                        c->Bp, slot, st);
    P2G_TRY(pod2g_check_launch(c));
    if (c->k > 0) {
        long long tw = (long long)n * (c->kp / 8);
        k_w_df8<<<ceil_div(tw, T), T, 0, c->stream>>>(c->d_row_ptr, c->d_col_idx, stage32, c->d_phi32, c->nb,
                                                      c->bs, c->kp, (float2*)c->d_W);
        P2G_TRY(pod2g_check_launch(c));
        if (c->d_W32) {
            k_w32<<<std::max(1, std::min(ceil_div(n, 64), 8 * c->num_sms)), T, 0, c->stream>>>(
                (const float2*)c->d_W, (long long)n, c->kp, c->Bp, slot, c->d_W32);
            P2G_TRY(pod2g_check_launch(c));
        }
        if (c->coarse_tc) {
            // tensor cores: one CTA per SM (at least 4 stages each), N = k rounded up to 16
            const int N = (c->k + 15) / 16 * 16;
            const int ga = std::max(1, std::min(c->num_sms, ceil_div(n, 4 * TC_KT)));
            k_ac_tc<<<ga, TC_THREADS, tc_smem(N), c->stream>>>(c->d_phi32, (const float2*)c->d_W, n, c->k, c->kp, N,
                                                               c->d_ac_part, c->d_counters + CNT_AC, c->d_Ac, L, st);
        } else {
            const int ga = std::max(1, std::min(2 * c->num_sms, ceil_div(n, 256)));
            k_ac<true><<<ga, T, 0, c->stream>>>(c->d_phi32, c->d_W, n, c->k, c->kp, c->d_ac_part,
                                                c->d_counters + CNT_AC, c->d_Ac, L, st);
        }
        P2G_TRY(pod2g_check_launch(c));
    }
    return POD2G_OK;
}

// Element contexts: coefficients (FP64, device) -> the slot's FP32 lane, the FP32
// operator values of that slot, then the common set-up.
static int setup_elem_tail(pod2g_ctx* c, int slot, int* st);

int setup_coeffs(pod2g_ctx* c, int slot, const double* coef_dev) {
    const int T = POD2G_THREADS;
    P2G_CUDA(cudaMemsetAsync(c->d_setup_status + slot, 0, sizeof(int), c->stream));
    int* st = c->d_setup_status + slot;
    k_coef_convert<<<std::min(ceil_div(c->n_el, T), 8 * c->num_sms), T, 0, c->stream>>>(
        coef_dev, c->d_coef32, c->n_el, c->Bp, slot, st);
    P2G_TRY(pod2g_check_launch(c));
    return setup_elem_tail(c, slot, st);
}

// Element contexts with a registered field: c_e(theta) on the device, then the same set-up.
int setup_theta(pod2g_ctx* c, int slot, const double* theta_dev) {
    const int T = POD2G_THREADS;
    P2G_CUDA(cudaMemsetAsync(c->d_setup_status + slot, 0, sizeof(int), c->stream));
    int* st = c->d_setup_status + slot;
    k_field_coef<<<std::min(ceil_div(c->n_el, T), 8 * c->num_sms), T, 0, c->stream>>>(
        c->d_modes, theta_dev, c->field_m, c->field_mu, c->field_sigma, c->field_log, c->d_coef32, c->n_el, c->Bp,
        slot, st);
    P2G_TRY(pod2g_check_launch(c));
    return setup_elem_tail(c, slot, st);
}

// FP32 operator values of the slot from its coefficients, then D^-1, K_c and its factor.
static int setup_elem_tail(pod2g_ctx* c, int slot, int* st) {
    const int T = POD2G_THREADS;
    const ElemOp E = elem_op(c);
    const int g = std::min(ceil_div(c->nb, T), 8 * c->num_sms);
    if (c->bs == 1) k_elem_stage<1><<<g, T, 0, c->stream>>>(E, c->d_row_ptr, c->nb, c->Bp, slot, c->d_stage32);
    else if (c->bs == 2) k_elem_stage<2><<<g, T, 0, c->stream>>>(E, c->d_row_ptr, c->nb, c->Bp, slot, c->d_stage32);
    else k_elem_stage<3><<<g, T, 0, c->stream>>>(E, c->d_row_ptr, c->nb, c->Bp, slot, c->d_stage32);
    P2G_TRY(pod2g_check_launch(c));
    return setup_from_stage32(c, slot, st);
}

int setup_values(pod2g_ctx* c, int slot, const double* vals_dev, bool lane_done);

// Set-up of several slots (values_dev: nslots consecutive instances): on the mixed
// paths the interleaved lanes of all of them are written by one tiled kernel first.
int setup_values_batch(pod2g_ctx* c, int nslots, const int* slots, const double* values_dev) {
    const long long tot = (long long)c->nnzb * c->bs * c->bs;
    const bool batch = c->precision != POD2G_FP64 && nslots > 1;
    if (batch) {
        int* d_slots = (int*)(c->d_mask + c->Bp);
        P2G_CUDA(cudaMemcpyAsync(d_slots, slots, sizeof(int) * nslots, cudaMemcpyHostToDevice, c->stream));
        if (nslots <= 8) {
            k_interleave_few<<<std::max(1, std::min(ceil_div(tot, 256), 8 * c->num_sms)), 256, 0, c->stream>>>(
                values_dev, tot, nslots, d_slots, c->Bp, c->d_vals32);
        } else {
            dim3 grid((unsigned)((tot + 31) / 32), (unsigned)((nslots + 31) / 32)), block(32, 8);
            k_interleave<<<grid, block, 0, c->stream>>>(values_dev, tot, nslots, d_slots, c->Bp, c->d_vals32);
        }
        P2G_TRY(pod2g_check_launch(c));
    }
    for (int i = 0; i < nslots; ++i) P2G_TRY(setup_values(c, slots[i], values_dev + (size_t)i * tot, batch));
    return POD2G_OK;
}

int setup_values(pod2g_ctx* c, int slot, const double* vals_dev) { return setup_values(c, slot, vals_dev, false); }

// lane_done: the slot's lane of the interleaved values was already written
int setup_values(pod2g_ctx* c, int slot, const double* vals_dev, bool lane_done) {
    const long long total = (long long)c->nnzb * c->bs * c->bs;
    const int T = POD2G_THREADS;
    const int n = c->n;
    const int32_t* diag_blk = c->d_diag_blk;
    P2G_CUDA(cudaMemsetAsync(c->d_setup_status + slot, 0, sizeof(int), c->stream));
    int* st = c->d_setup_status + slot;
    double* L = c->d_Lc + (size_t)slot * c->k * c->k;
    if (c->precision == POD2G_FP64) {
        double* v = c->d_vals64 + (size_t)slot * total;
        if (v != vals_dev)
            P2G_CUDA(cudaMemcpyAsync(v, vals_dev, total * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        k_dinv<double><<<ceil_div(n, T), T, 0, c->stream>>>(v, diag_blk, c->nb, c->bs,
                                                             c->d_dinv64 + (size_t)slot * n, nullptr, 1, 0, st);
        P2G_TRY(pod2g_check_launch(c));
        if (c->k > 0) {
            long long tw = (long long)n * c->kp;
            k_w_f64<<<ceil_div(tw, T), T, 0, c->stream>>>(c->d_row_ptr, c->d_col_idx, v, c->d_phi64, c->nb, c->bs,
                                                          c->kp, c->d_W);
            P2G_TRY(pod2g_check_launch(c));
            int g = std::max(1, std::min(2 * c->num_sms, ceil_div(n, 256)));
            k_ac<false><<<g, T, 0, c->stream>>>(c->d_phi64, c->d_W, n, c->k, c->kp, c->d_ac_part,
                                                c->d_counters + CNT_AC, c->d_Ac, L, st);
            P2G_TRY(pod2g_check_launch(c));
        }
    } else {
        int g = std::min(ceil_div(total, T), 8 * c->num_sms);
        k_convert_values<<<g, T, 0, c->stream>>>(vals_dev, c->d_stage32, lane_done ? nullptr : c->d_vals32, total,
                                                 c->Bp, slot);
        P2G_TRY(pod2g_check_launch(c));
        P2G_TRY(setup_from_stage32(c, slot, st));
    }
    return POD2G_OK;
}

// dynamic shared memory of the tensor-core contraction (once per context)
int setup_tc_attributes(pod2g_ctx* c) {
    (void)c;
    return allow_max_smem((const void*)k_ac_tc);
}
