// Shared definitions of the POD-2G-PCG library: context layout, error handling,
// double-float arithmetic and block-reduction helpers.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/pod2g.h"

#define POD2G_THREADS 256      // threads per CTA of the row kernels
#define POD2G_MAX_K 64         // largest supported number of POD modes
#define POD2G_MAX_BP 256       // largest slot-lane count
#define POD2G_ELEM_RE 8        // element positions per block row (elements adjacent to one node)
#define POD2G_KREF_MAX 576     // reference-matrix entries, (npe * bs)^2 with npe * bs <= 24
#define POD2G_PERSIST_ITEMS (1LL << 20)  // unknowns x slot lanes up to which K Phi is kept for the persistent launch

// ---------------------------------------------------------------------------- slot states
enum SlotState : int { SLOT_IDLE = 0, SLOT_JOINING = 1, SLOT_ACTIVE = 2, SLOT_DONE = 3 };

// Per-slot scalars of the batched PCG (device memory, one entry per slot lane).
struct SlotScalars {
    double rs;      // r_k^T s_k
    double alpha;
    double beta;
    double bb;      // ||b||^2
    double tol2;    // tol^2 ||b||^2
    double rr;      // ||r_k||^2 (recurrence residual)
    double relres;  // final true relative residual
    int state;      // SlotState
    int result;     // POD2G_* status once DONE
    int iters;
    int maxit;
    int first;      // 1 while the initial preconditioner pass runs (beta forced to 0)
    int pad;
};

// ---------------------------------------------------------------------------- context
struct ServeRequest;

struct pod2g_ctx {
    int device = 0;
    int nb = 0, bs = 0, n = 0, nnzb = 0, k = 0, kp = 0;   // kp: k padded to a multiple of 4
    int precision = 0, pre = 1, post = 1, beta_pr = 0, B = 1, Bp = 1, chunk = 8;
    int method = 0;                     // POD2G_PCG or POD2G_STATIONARY
    int smoother = 0;                   // POD2G_SMOOTHER_JACOBI or POD2G_SMOOTHER_SGS
    bool coarse_tc = false;             // K_c = Phi^T (K Phi) contracted on the tensor cores (mixed paths)
    // multicolour order of the Gauss-Seidel smoother
    int ncolours = 0;
    std::vector<int> coff;              // [ncolours + 1] offsets into d_cnodes
    int32_t* d_cnodes = nullptr;        // [nb] nodes sorted by colour
    uint8_t* d_colour = nullptr;        // [nb] colour of each node
    int64_t iter_launches = 8;          // kernels per captured iteration
    double omega = 2.0 / 3.0;
    size_t hbm_budget = 0, allocated = 0;
    int64_t spin_limit = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::atomic<int64_t> launches{0};
    int num_sms = 152;

    // pattern
    int32_t* d_row_ptr = nullptr;
    int32_t* d_col_idx = nullptr;
    int32_t* d_diag_blk = nullptr;      // [nb] index of each block row's diagonal block

    // POD basis, row-major [n][kp] (entries beyond k are zero)
    double* d_phi64 = nullptr;          // FP64 path
    float* d_phi32 = nullptr;           // mixed paths (BF16-rounded values, widened, for MIXED_BF16PHI)

    // element-factored operator (pod2g_create_elements; elem = 1)
    int elem = 0, n_el = 0, npe = 0;
    uint64_t* d_desc = nullptr;         // [nnzb] block descriptors (see ElemOp)
    int32_t* d_rowel = nullptr;         // [nb][POD2G_ELEM_RE] adjacent elements, ascending, -1 padded
    float* d_kref32 = nullptr;          // [npe*npe][bs*bs] FP32 reference sub-blocks
    float* d_coef32 = nullptr;          // [n_el][Bp] FP32 coefficients, slot-interleaved
    // parametrized coefficients c_e(theta) (pod2g_set_field)
    int field_m = 0, field_log = 1;
    double field_mu = 0.0, field_sigma = 1.0;
    double* d_modes = nullptr;          // [n_el][m]
    double* d_theta = nullptr;          // [B][m] staging of parameter vectors

    // per-slot set-up results
    double* d_Lc = nullptr;             // [B][k][k] Cholesky factors (FP64)
    int* d_setup_status = nullptr;      // [B]
    std::vector<int> setup_ok;          // host copy: slot has a valid set-up

    // set-up scratch (one instance at a time)
    double* d_stage = nullptr;          // [nnzb*bs*bs] FP64 values staging
    float* d_stage32 = nullptr;         // [nnzb*bs*bs] FP32-rounded values (mixed paths)
    double* d_W = nullptr;              // [n][kp]: K Phi (FP64 accumulate)
    double* d_ac_part = nullptr;        // [G][k][k] contraction partials
    double* d_Ac = nullptr;             // [k][k]
    unsigned* d_counters = nullptr;     // last-CTA counters (several)

    // ---- plain FP64 path (slot-major)
    double* d_vals64 = nullptr;         // [B][nnzb][bs*bs]
    double* d_dinv64 = nullptr;         // [B][n]
    double *d_x64 = nullptr, *d_r64 = nullptr, *d_s64 = nullptr, *d_p64 = nullptr, *d_q64 = nullptr,
           *d_y64 = nullptr, *d_t64 = nullptr, *d_w64 = nullptr;
    double* d_c64 = nullptr;            // [kp] restriction / coarse vector
    double* d_part64 = nullptr;         // [G * (kp+4)] reduction partials
    double* d_scal64 = nullptr;         // [16] plain-path scalars
    double* h_scal64 = nullptr;         // pinned host mirror

    // ---- batched mixed path (slot-interleaved: element (row, slot) at row*Bp + slot)
    float* d_vals32 = nullptr;          // [nnzb][bs*bs][Bp]
    float* d_dinv32 = nullptr;          // [n][Bp]
    float2* d_xdf = nullptr;            // [n][Bp] double-float
    float2* d_rdf = nullptr;
    float2* d_pdf = nullptr;
    float2* d_qdf = nullptr;
    float2* d_bdf = nullptr;
    double* d_b64 = nullptr;            // [n][Bp] the right-hand sides in FP64 (final residual)
    float* d_s32 = nullptr;             // [n][Bp]
    float* d_y32 = nullptr;             // [n][Bp]
    float* d_W32 = nullptr;             // [kp][n][Bp] K Phi per slot (FP32), when the post-smoothing uses it
    float* d_ec = nullptr;              // [Bp][kp] coarse corrections
    double* d_part = nullptr;           // reduction partials [G][Bp][2] (scalars)
    double* d_cpart = nullptr;          // restriction partials [G][Bp][kp]
    SlotScalars* d_sc = nullptr;        // [Bp]
    SlotScalars* h_sc = nullptr;        // pinned host mirror
    int* d_err = nullptr;               // device error word: set when a bounded device wait expires
    int* h_err = nullptr;               // pinned host mirror
    SlotScalars* h_sc2 = nullptr;       // second pinned mirror and error word for the lookahead launch
    int* h_err2 = nullptr;
    cudaEvent_t la_ev[2] = {nullptr, nullptr};
    int* d_mask = nullptr;              // [2 Bp] lane mask and slot list for load / finalize
    double* d_iob = nullptr;            // [B][n] staging of right-hand sides (host-buffer entry points)
    double* d_iox = nullptr;            // [B][n] staging of x0 / x
    int grid_rows = 0;                  // CTAs of the row kernels (multiple of the cluster size 8)
    int grid_spmv = 0;                  // CTAs of the outer SpMV (multiple of 8)
    int grid_restrict = 0;              // CTAs of the restriction (multiple of 8)
    int grid_prol = 0;                  // CTAs of the prolongation
    int grid_vec = 0;                   // CTAs of the vector updates (p, x/r)
    int rows_kernel = 0;                // bit 0: staged smoother row kernels, bit 1: staged outer SpMV
    int ws_occ = 0;                     // resident CTAs per SM of the staged row kernels (0: not available)
    int restrict_rows = 0;              // rows per staged chunk of the restriction (0: default)
    int grid_persist = 0;               // CTAs of the persistent launch (rows_kernel bit 3)
    cudaGraphExec_t graph_exec = nullptr;
    // per-kernel timing (event-record nodes around each kernel of the captured iterations)
    bool timing = false;
    std::vector<cudaEvent_t> tev;       // [chunk][9]
    cudaEvent_t* cap_ev = nullptr;      // events of the iteration being captured
    int cap_idx = 0;
    double kt_ms[8] = {0};
    long long kt_n[8] = {0};

    // serving
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool serving = false, stop = false;
    int max_queue = 0;
    uint64_t next_ticket = 1;
    std::deque<ServeRequest*> queue;
    std::map<uint64_t, ServeRequest*> finished;
    std::map<uint64_t, ServeRequest*> inflight;
};

struct ServeRequest {
    uint64_t ticket;
    std::vector<double> values, b, x0, x;   // values: block values, coefficients, or theta
    bool has_x0 = false;
    bool theta = false;                     // values holds the parameters theta
    double tol = 1e-8;
    int maxit = 1000;
    int iters = 0, status = POD2G_PENDING;
    double relres = 0.0;
    double t_submit = 0.0, t_done = 0.0;
    int slot = -1;
};

// ---------------------------------------------------------------------------- errors
#define P2G_CUDA(call)                                                          \
    do {                                                                        \
        cudaError_t e__ = (call);                                               \
        if (e__ != cudaSuccess) {                                               \
            pod2g_set_last_cuda_error(e__);                                     \
            pod2g_trace(__FILE__, __LINE__, POD2G_CUDA_ERROR);                  \
            return POD2G_CUDA_ERROR;                                            \
        }                                                                       \
    } while (0)

#define P2G_TRY(call)                                                           \
    do {                                                                        \
        int s__ = (call);                                                       \
        if (s__ != POD2G_OK) {                                                  \
            pod2g_trace(__FILE__, __LINE__, s__);                               \
            return s__;                                                         \
        }                                                                       \
    } while (0)

// With POD2G_DEBUG set in the environment, failing calls are traced to stderr.
void pod2g_trace(const char* file, int line, int status);

void pod2g_set_last_cuda_error(cudaError_t e);
int pod2g_check_launch(pod2g_ctx* c);  // counts a launch, checks cudaGetLastError

static inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------------------- double-float
// Unevaluated sums hi + lo of two FP32 numbers (|lo| <= ulp(hi)/2): a ~48-bit
// significand carried in FP32 arithmetic. Built from the error-free
// transformations TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and TwoProd via FMA, and the
// double-word algorithms of Joldes, Muller and Popescu (ACM TOMS 44(2), 2017).
// Operations are written so that no multiply-add pair can be contracted.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ float2 df_norm(float hi, float lo) {
    float s, e;
    fast_two_sum(hi, lo, s, e);
    return make_float2(s, e);
}
// a + b, both double-float ("AccurateDWPlusDW")
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    float sh, sl, th, tl;
    two_sum(a.x, b.x, sh, sl);
    two_sum(a.y, b.y, th, tl);
    sl = __fadd_rn(sl, th);
    fast_two_sum(sh, sl, sh, sl);
    sl = __fadd_rn(sl, tl);
    return df_norm(sh, sl);
}
// a * b, both double-float ("DWTimesDW")
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
    float ph = __fmul_rn(a.x, b.x);
    float pl = __fmaf_rn(a.x, b.x, -ph);
    pl = __fmaf_rn(a.x, b.y, pl);
    pl = __fmaf_rn(a.y, b.x, pl);
    return df_norm(ph, pl);
}
// accumulator (hi, lo) += v * (ph + pl) for an FP32 v: the product v*ph is
// split exactly, its high part added with TwoSum, all low parts gathered in lo.
__device__ __forceinline__ void df_acc_fma(float& hi, float& lo, float v, float ph, float pl) {
    float p = __fmul_rn(v, ph);
    float pe = __fmaf_rn(v, ph, -p);
    float s, e;
    two_sum(hi, p, s, e);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, pe));
    lo = __fmaf_rn(v, pl, lo);
}
// ---- packed FP32 pairs: the f32x2 instructions of the sm_100 family apply one FP32 operation
// (IEEE, round to nearest even, no flush to zero) to both halves of a 64-bit register pair,
// in one instruction; each half is rounded exactly as the scalar operation rounds it.
__device__ __forceinline__ unsigned long long f2_bits(float2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 f2_of(unsigned long long r) {
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_of(d);
}
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_of(d);
}
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_of(d);
}
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
    return f2_of(d);
}
// df_acc_fma on two accumulators at once, in packed instructions: (hi.x, lo.x) += v.x (ph.x + pl.x)
// and (hi.y, lo.y) += v.y (ph.y + pl.y), every operation rounded as in df_acc_fma (the sign
// flips are exact: -(v ph) is formed as v (-ph), and p - bb as -((-p) + bb)). nph = -ph.
__device__ __forceinline__ void df_acc_fma2(float2& hi, float2& lo, float2 v, float2 ph, float2 nph, float2 pl) {
    const float2 np = f2_mul(v, nph);      // -p, p = v ph rounded
    const float2 pe = f2_fma(v, ph, np);   // v ph - p, exact
    const float2 s = f2_sub(hi, np);       // TwoSum(hi, p)
    const float2 bb = f2_sub(s, hi);
    const float2 t2 = f2_sub(hi, f2_sub(s, bb));
    const float2 e = f2_sub(t2, f2_add(np, bb));
    hi = s;
    lo = f2_add(lo, f2_add(e, pe));
    lo = f2_fma(v, pl, lo);
}
__device__ __forceinline__ float2 df_from_double(double d) {
    float hi = __double2float_rn(d);
    float lo = __double2float_rn(d - (double)hi);
    return make_float2(hi, lo);
}
__device__ __forceinline__ double df_to_double(float2 a) { return (double)a.x + (double)a.y; }

// ---------------------------------------------------------------------------- last-CTA pattern
// Every CTA calls this after writing its partial results; it returns true in
// exactly one CTA (the last to arrive), which may then read all partials. No
// CTA waits for another, so nothing can hang. The counter is reset by the last CTA.
__device__ __forceinline__ bool last_cta_arrive(unsigned* counter) {
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(counter, 1u);
        am_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (am_last) __threadfence();
    return am_last;
}
__device__ __forceinline__ void last_cta_reset(unsigned* counter) {
    if (threadIdx.x == 0) *counter = 0u;
}

// ---------------------------------------------------------------------------- element-factored operator
// K = sum_e c_e K_ref on the stored block pattern. One 64-bit descriptor per
// stored block, shared by all slots: for each position p < 8 of the block row's
// element list, bit 48 + p says that element holds the block, and bits 6p..6p+5
// give its reference sub-block s = a * npe + b (a, b the local indices of the
// row and column nodes). Bit 62: zero block (a fixed node's row or column); bit
// 63: identity block (a fixed node's diagonal block).
struct ElemOp {
    const uint64_t* desc;     // [nnzb]
    const int32_t* rowel;     // [nb][POD2G_ELEM_RE]
    const float* coef;        // [n_el][Bp]
    const float* kref;        // [npe*npe][bs*bs]
    int nk;                   // floats in kref
};

static inline ElemOp elem_op(const pod2g_ctx* c) {
    ElemOp E;
    E.desc = c->d_desc;
    E.rowel = c->d_rowel;
    E.coef = c->d_coef32;
    E.kref = c->d_kref32;
    E.nk = c->npe * c->npe * c->bs * c->bs;
    return E;
}

// The coefficients c_e of block row i's elements for one slot lane (0 where no element).
__device__ __forceinline__ void elem_row_coefs(const ElemOp& E, int i, int lane, int Bp, float* ce) {
    int el[POD2G_ELEM_RE];
#pragma unroll
    for (int p = 0; p < POD2G_ELEM_RE; ++p) el[p] = __ldg(E.rowel + (long long)i * POD2G_ELEM_RE + p);
#pragma unroll
    for (int p = 0; p < POD2G_ELEM_RE; ++p) ce[p] = el[p] >= 0 ? E.coef[(long long)el[p] * Bp + lane] : 0.f;
}

// Values of one block from its descriptor: the FP32 sum, in element order, of the
// rounded products c_e * K_ref[s] (no contraction into FMA).
template <int BS>
__device__ __forceinline__ void elem_block_values(uint64_t d, const float* ce, const float* kref, float* v) {
    if (d >> 62) {
        const float dg = (d >> 63) ? 1.f : 0.f;
#pragma unroll
        for (int e = 0; e < BS * BS; ++e) v[e] = (e % (BS + 1) == 0) ? dg : 0.f;
        return;
    }
#pragma unroll
    for (int e = 0; e < BS * BS; ++e) v[e] = 0.f;
#pragma unroll
    for (int p = 0; p < POD2G_ELEM_RE; ++p) {
        if ((d >> (48 + p)) & 1ull) {
            const float* K = kref + (int)((d >> (6 * p)) & 63ull) * (BS * BS);
#pragma unroll
            for (int e = 0; e < BS * BS; ++e) v[e] = __fadd_rn(v[e], __fmul_rn(ce[p], K[e]));
        }
    }
}

// counters used by the last-CTA reductions (indices into ctx->d_counters)
enum { CNT_SPMV = 0, CNT_POST = 1, CNT_RESID = 2, CNT_PLAIN = 3, CNT_AC = 4, CNT_W = 5, CNT_PERSIST = 6 /* and 7 */, CNT_N = 16 };

// ---------------------------------------------------------------------------- internal entry points
int plain_solve(pod2g_ctx* c, int slot, const double* b_dev, const double* x0_dev, double tol, int maxit,
                double* x_dev, int* iters, double* relres, int* status);
int setup_values(pod2g_ctx* c, int slot, const double* vals_dev);
int setup_values_batch(pod2g_ctx* c, int nslots, const int* slots, const double* values_dev);
int setup_coeffs(pod2g_ctx* c, int slot, const double* coef_dev);
int setup_theta(pod2g_ctx* c, int slot, const double* theta_dev);
int setup_tc_attributes(pod2g_ctx* c);
// Allow a kernel the device's largest dynamic shared memory per block. The attribute belongs to the
// function, not to a context, so every context sets the same value: a context that needs less can
// never lower the limit below what another context's launches of the same kernel request.
int allow_max_smem(const void* fn);
// doubles describing one instance: matrix values, or element coefficients
static inline size_t instance_len(const pod2g_ctx* c) {
    return c->elem ? (size_t)c->n_el : (size_t)c->nnzb * c->bs * c->bs;
}
static inline int setup_instance(pod2g_ctx* c, int slot, const double* dev) {
    return c->elem ? setup_coeffs(c, slot, dev) : setup_values(c, slot, dev);
}
int batched_load(pod2g_ctx* c, int nslots, const int* slots, const double* b_dev, const double* x0_dev,
                 const double* tol, const int* maxit);
int batched_run(pod2g_ctx* c, const std::vector<int>& lanes);
int batched_retire(pod2g_ctx* c, const std::vector<int>& lanes, int result);
int batched_chunk(pod2g_ctx* c);
int batched_set_timing(pod2g_ctx* c, int on);
int batched_grid(int num_sms, long long items);
int batched_finalize(pod2g_ctx* c, int nslots, const int* slots, double* x_dev, int* iters, double* relres,
                     int* status);
int batched_alloc(pod2g_ctx* c);
int rom_solution(pod2g_ctx* c, int nslots, const int* slots, const double* b_dev, double* x_dev);
int batched_set_tuning(pod2g_ctx* c, const pod2g_tuning* t);
int batched_autotune(pod2g_ctx* c, int nslots, const int* slots, const double* b_dev, int iters);
// persistent launch of whole iterations (persist.cu)
bool persist_applies(const pod2g_ctx* c);
int persist_max_grid(pod2g_ctx* c);
int persist_launch(pod2g_ctx* c, int iters);
void batched_free(pod2g_ctx* c);
int dev_alloc(pod2g_ctx* c, void** p, size_t bytes);
