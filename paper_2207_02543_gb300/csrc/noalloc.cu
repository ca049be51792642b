// A solve entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code running under an allocator that owns
// all device memory (a framework's caching allocator, a memory pool sized at
// start-up), callers that must not synchronise the device as cudaMalloc/cudaFree
// may do, or embedders that only hand the library pointers they already own.
// pod2g_solve_noalloc serves them: it is the single-instance FP64 solve of an FP64
// context (same kernels, same results), but every scratch buffer it needs lives in
// one file-scope static __device__ array of fixed size, which each GPU that loads
// the library holds until the process exits. The caller passes inputs and outputs
// as device pointers; nothing is allocated or freed.
#include "common.cuh"

#include <cstring>
#include <mutex>

namespace {

constexpr long long NA_MAX_N = POD2G_NOALLOC_MAX_N;   // unknowns
constexpr int NA_MAX_K = POD2G_NOALLOC_MAX_K;         // POD modes
constexpr int NA_MAX_KP = NA_MAX_K;                   // padded modes (k <= 32 pads to <= 32)
constexpr int NA_MAX_G = 1024;                        // partial-sum slots (>= CTAs of any kernel used)
constexpr int NA_MAX_DEV = 64;

// byte offsets of the sub-buffers inside the scratch array (each 256-byte aligned)
constexpr size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }
constexpr size_t OFF_PHI = 0;
constexpr size_t OFF_W = OFF_PHI + align256(sizeof(double) * NA_MAX_N * NA_MAX_KP);
constexpr size_t OFF_DINV = OFF_W + align256(sizeof(double) * NA_MAX_N * NA_MAX_KP);
constexpr size_t OFF_VEC = OFF_DINV + align256(sizeof(double) * NA_MAX_N);
constexpr size_t OFF_ACP = OFF_VEC + 8 * align256(sizeof(double) * NA_MAX_N);
constexpr size_t OFF_PART = OFF_ACP + align256(sizeof(double) * 64 * NA_MAX_K * NA_MAX_K);
constexpr size_t OFF_AC = OFF_PART + align256(sizeof(double) * NA_MAX_G * (NA_MAX_KP + 8));
constexpr size_t OFF_LC = OFF_AC + align256(sizeof(double) * NA_MAX_K * NA_MAX_K);
constexpr size_t OFF_C = OFF_LC + align256(sizeof(double) * NA_MAX_K * NA_MAX_K);
constexpr size_t OFF_SCAL = OFF_C + align256(sizeof(double) * NA_MAX_KP);
constexpr size_t OFF_CNT = OFF_SCAL + align256(sizeof(double) * 16);
constexpr size_t OFF_STAT = OFF_CNT + align256(sizeof(unsigned) * CNT_N);
constexpr size_t OFF_DIAG = OFF_STAT + align256(sizeof(int) * 2);
constexpr size_t SCRATCH_BYTES = OFF_DIAG + align256(sizeof(int32_t) * NA_MAX_N);

// The scratch memory (10,503,168 bytes). Device code below only receives pointers
// into it; host code obtains its device address with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_pod2g_scratch[SCRATCH_BYTES];

// Validates the pattern and finds each block row's diagonal block. err[0] != 0
// flags an invalid pattern (rows read only inside validated bounds).
__global__ void k_check_pattern(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx, int nb,
                                int nnzb, int32_t* __restrict__ diag, int* __restrict__ err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    int a = row_ptr[i], b = row_ptr[i + 1];
    if ((i == 0 && a != 0) || (i == nb - 1 && b != nnzb) || a < 0 || b < a || b > nnzb) {
        atomicExch(err, 1);
        return;
    }
    int d = -1, prev = -1;
    for (int t = a; t < b; ++t) {
        int j = col_idx[t];
        if (j < 0 || j >= nb || j <= prev) { atomicExch(err, 1); return; }
        if (j == i) d = t;
        prev = j;
    }
    if (d < 0) atomicExch(err, 1);
    diag[i] = d < 0 ? 0 : d;
}

// column-major Phi [k][n] -> row-major [n][kp] (zero padding beyond k)
__global__ void k_phi_rows(const double* __restrict__ phi_cm, long long n, int k, int kp, double* __restrict__ out) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= n * kp) return;
    long long d = t / kp;
    int m = (int)(t - d * kp);
    out[t] = m < k ? phi_cm[(long long)m * n + d] : 0.0;
}

std::mutex g_mu;                                // serialises calls within the process
pod2g_ctx g_ctx[NA_MAX_DEV];                    // host-side state, constructed at library load
double g_scal_host[NA_MAX_DEV][16];             // host mirror of the per-solve scalars

int pick_kp_small(int k) {
    const int list[] = {0, 8, 16, 24, 32};
    for (int v : list)
        if (v >= k) return v;
    return -1;
}

}  // namespace

extern "C" int pod2g_solve_noalloc(int32_t n_brows, int32_t bs, int32_t nnzb, const int32_t* row_ptr_dev,
                                   const int32_t* col_idx_dev, const double* values_dev, const double* phi_dev,
                                   int k, const pod2g_opts* opts, const double* b_dev, const double* x0_dev,
                                   double tol, int maxit, double* x_dev, int* iters, double* relres, int* status,
                                   void* stream) {
    if (n_brows <= 0 || bs < 1 || bs > 3 || nnzb < n_brows || !row_ptr_dev || !col_idx_dev || !values_dev ||
        !b_dev || !x_dev || !(tol >= 0.0) || maxit < 0 || k < 0 || (k > 0 && !phi_dev))
        return POD2G_INVALID_ARG;
    const long long n = (long long)n_brows * bs;
    if (n > NA_MAX_N || k > NA_MAX_K) return POD2G_TOO_LARGE;  // beyond the scratch array's capacity
    pod2g_opts o;
    if (opts) o = *opts; else pod2g_default_opts(&o);
    if (!(o.omega > 0.0) || o.pre < 0 || o.post < 0 || o.pre > 8 || o.post > 8) return POD2G_INVALID_ARG;
    // only the damped-Jacobi PCG solve is offered here
    if (o.method != POD2G_PCG || o.smoother != POD2G_SMOOTHER_JACOBI) return POD2G_INVALID_ARG;

    std::lock_guard<std::mutex> lock(g_mu);
    int dev = 0;
    P2G_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEV) return POD2G_INVALID_ARG;
    // The device address of the array in the current device's context, looked up on every
    // call (a cheap host query), so that a context torn down and re-created since the last
    // call is never written through a stale pointer.
    void* addr = nullptr;
    P2G_CUDA(cudaGetSymbolAddress(&addr, g_pod2g_scratch));
    unsigned char* S = (unsigned char*)addr;
    pod2g_ctx* c = &g_ctx[dev];
    // On every return path, including errors, the caller's stream is drained before the lock
    // is released, so that the next call never overwrites scratch that queued work still uses.
    struct DrainOnExit {
        cudaStream_t s;
        ~DrainOnExit() { cudaStreamSynchronize(s); }
    } drain{(cudaStream_t)stream};
    c->device = dev;
    c->nb = n_brows; c->bs = bs; c->n = (int)n; c->nnzb = nnzb; c->k = k; c->kp = pick_kp_small(k);
    c->precision = POD2G_FP64; c->pre = o.pre; c->post = o.post; c->beta_pr = o.beta_pr ? 1 : 0;
    c->B = 1; c->Bp = 1; c->omega = o.omega;
    c->stream = (cudaStream_t)stream;
    int sms = 0;
    P2G_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    c->num_sms = std::max(1, std::min(sms, 256));
    c->d_row_ptr = const_cast<int32_t*>(row_ptr_dev);
    c->d_col_idx = const_cast<int32_t*>(col_idx_dev);
    c->d_vals64 = const_cast<double*>(values_dev);  // read only
    c->d_phi64 = (double*)(S + OFF_PHI);
    c->d_W = (double*)(S + OFF_W);
    c->d_dinv64 = (double*)(S + OFF_DINV);
    double** vecs[] = {&c->d_x64, &c->d_r64, &c->d_s64, &c->d_p64, &c->d_q64, &c->d_y64, &c->d_t64, &c->d_w64};
    for (int v = 0; v < 8; ++v) *vecs[v] = (double*)(S + OFF_VEC + v * align256(sizeof(double) * NA_MAX_N));
    c->d_ac_part = (double*)(S + OFF_ACP);
    c->d_part64 = (double*)(S + OFF_PART);
    c->d_Ac = (double*)(S + OFF_AC);
    c->d_Lc = (double*)(S + OFF_LC);
    c->d_c64 = (double*)(S + OFF_C);
    c->d_scal64 = (double*)(S + OFF_SCAL);
    c->d_counters = (unsigned*)(S + OFF_CNT);
    c->d_setup_status = (int*)(S + OFF_STAT);
    int* d_err = (int*)(S + OFF_STAT) + 1;
    c->d_diag_blk = (int32_t*)(S + OFF_DIAG);
    c->h_scal64 = g_scal_host[dev];

    // the array keeps the previous call's contents: counters and flags start at zero
    P2G_CUDA(cudaMemsetAsync(c->d_counters, 0, sizeof(unsigned) * CNT_N, c->stream));
    P2G_CUDA(cudaMemsetAsync(c->d_setup_status, 0, sizeof(int) * 2, c->stream));
    k_check_pattern<<<ceil_div(n_brows, 256), 256, 0, c->stream>>>(row_ptr_dev, col_idx_dev, n_brows, nnzb,
                                                                   c->d_diag_blk, d_err);
    P2G_TRY(pod2g_check_launch(c));
    int h_err = 0;
    P2G_CUDA(cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    P2G_CUDA(cudaStreamSynchronize(c->stream));
    if (h_err) return POD2G_INVALID_ARG;
    if (c->kp > 0) {
        k_phi_rows<<<ceil_div(n * c->kp, 256), 256, 0, c->stream>>>(phi_dev, n, k, c->kp, c->d_phi64);
        P2G_TRY(pod2g_check_launch(c));
    }
    // per-instance set-up (D^-1, K_c, Cholesky), then the FP64 solve
    P2G_TRY(setup_values(c, 0, values_dev));
    int st_setup = 0;
    P2G_CUDA(cudaMemcpyAsync(&st_setup, c->d_setup_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    P2G_CUDA(cudaStreamSynchronize(c->stream));
    if (st_setup != POD2G_OK) {
        if (status) *status = st_setup;
        return st_setup;
    }
    int st = POD2G_OK, it = 0;
    double rr = 0.0;
    P2G_TRY(plain_solve(c, 0, b_dev, x0_dev, tol, maxit, x_dev, &it, &rr, &st));
    if (iters) *iters = it;
    if (relres) *relres = rr;
    if (status) *status = st;
    return st;
}
