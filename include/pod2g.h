/*
 * pod2g.h — C ABI of a GB300 (sm_103a) solver for parametrized sparse SPD systems
 *           K(theta) u = f(theta) by POD-2G-preconditioned conjugate gradients.
 *
 * Method: arXiv 2207.02543 (Nikolopoulos et al.), Algorithm 3 (PCG whose
 * preconditioner is one cycle of an algebraic two-grid scheme) with the cycle of
 * Algorithm 2 and the POD basis Phi_r as prolongation operator (Section 3.3).
 * The preconditioner applied to a residual r is s = AMG(0; K, r, r1, r2):
 *     y  <- 0;  r1 damped-Jacobi sweeps  y <- y + omega D^{-1} (r - K y)
 *     e_c = (Phi^T K Phi)^{-1} Phi^T (r - K y);   y <- y + Phi e_c
 *     r2 damped-Jacobi sweeps;                    s = y
 * with D = diag(K) (or forward / backward multicolour Gauss-Seidel sweeps, see
 * pod2g_opts.smoother). The outer iteration is Algorithm 1 with T^{-1} r := s,
 * or, as the stationary method, u <- u + s(f - K u) (Algorithm 2 iterated).
 *
 * Conventions
 *   - n_brows block rows of size bs (1, 2 or 3); n = n_brows * bs unknowns.
 *   - Pattern: block CSR, int32 row_ptr[n_brows+1], col_idx[nnzb]; columns sorted
 *     ascending within a row, every diagonal block present, pattern symmetric.
 *     One pattern is shared by every parameter instance ("slot") of a context.
 *   - Values of one instance: double values[nnzb * bs * bs], block after block,
 *     each block row-major.
 *   - Phi: double phi[n * k], column-major (column j = POD mode j), any
 *     full-column-rank basis (orthonormality is not required).
 *   - Vectors (b, x0, x) are double[n] per instance.
 *   - Stopping rule: ||r_k||_2 <= tol * ||b||_2 on the recurrence residual,
 *     tested before every iteration (k = 0 included). iters = number of alpha
 *     updates. final relative residual = ||b - K x||_2 / ||b||_2 recomputed at
 *     exit in FP64 on every path: the stored matrix values (FP32-rounded on the
 *     mixed paths, exact in FP64) times the returned x, accumulated with FP64
 *     fused multiply-adds against the caller's FP64 b, FP64 sums of squares.
 *     b = 0 gives x = 0, iters = 0, relres = 0.
 *   - Precision modes:
 *       POD2G_FP64          values, vectors, Phi and arithmetic in FP64; one
 *                           instance at a time, kernel by kernel, convergence
 *                           checked on the host every iteration (the plain path);
 *       POD2G_MIXED_FP32PHI batched path: values stored in FP32 (the system solved
 *                           is the one with FP32-rounded values), preconditioner
 *                           (smoothing, restriction, prolongation) in FP32 with
 *                           FP32 Phi, K_c = Phi^T (K Phi) formed in double-float,
 *                           outer recurrences (x, r, p, K p, dot products) in
 *                           double-float (~48-bit significand, pairs of FP32,
 *                           error-free transformations), scalars and the k x k
 *                           Cholesky factor in FP64;
 *       POD2G_MIXED_BF16PHI as above with Phi rounded to BF16.
 *   - Ownership: the library copies every input; callers keep their buffers.
 *     Output buffers belong to the caller. Functions whose name ends in _dev take
 *     device pointers, read and written in the context's stream.
 *   - Thread safety: a context is used by one host thread at a time, except that
 *     pod2g_submit / pod2g_poll may be called from any thread while the serving
 *     worker runs (they take the context's queue lock).
 *   - All functions return a status code (POD2G_OK = 0) unless noted.
 */
#ifndef POD2G_H
#define POD2G_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define POD2G_OK             0  /* success / converged */
#define POD2G_NOT_CONVERGED  1  /* maxit reached; x holds the last iterate */
#define POD2G_BREAKDOWN      2  /* p^T K p <= 0 or r^T s <= 0: matrix or preconditioner not SPD */
#define POD2G_NOT_SPD        3  /* coarse matrix Phi^T K Phi not SPD, or a non-positive diagonal */
#define POD2G_INVALID_ARG    4  /* bad argument (null pointer, size, slot index, pattern) */
#define POD2G_ADMISSION      5  /* request refused: over the context's HBM budget / no free slot */
#define POD2G_OOM            6  /* device allocation failed */
#define POD2G_CUDA_ERROR     7  /* a CUDA call failed */
#define POD2G_TIMEOUT        8  /* a bounded device or host wait expired */
#define POD2G_NONFINITE      9  /* NaN or Inf in an input or an iterate */
#define POD2G_PENDING       10  /* pod2g_poll: request not finished yet */
#define POD2G_TOO_LARGE     11  /* pod2g_solve_noalloc: size beyond its fixed scratch capacity */

/* precision modes */
#define POD2G_FP64           0
#define POD2G_MIXED_FP32PHI  1
#define POD2G_MIXED_BF16PHI  2

/* relaxation schemes of the two-grid cycle */
#define POD2G_SMOOTHER_JACOBI 0  /* damped Jacobi u <- u + omega D^-1 (f - K u), pre and post */
#define POD2G_SMOOTHER_SGS    1  /* pointwise Gauss-Seidel (eq. GaussSeidel) in a multicolour order:
                                    forward sweeps before, backward sweeps after the coarse
                                    correction (omega is not used) */

/* contraction K_c = Phi^T (K Phi) of the per-instance set-up on the mixed paths (K Phi is
 * always formed in double-float on the CUDA cores) */
#define POD2G_COARSE_DF      0  /* double-float on the CUDA cores (~14 significant digits) */
#define POD2G_COARSE_TENSOR  1  /* tensor cores (tcgen05, BF16 operands, FP32 accumulation): each
                                   operand split into three BF16 pieces, the six products whose
                                   pieces reach down to ~2^-24 of the term, FP32 partial sums per
                                   CTA added in FP64 (K_c to ~1e-7 of its largest entry) */

/* solution methods */
#define POD2G_PCG            0  /* PCG preconditioned by one POD-2G cycle from zero (Algorithm 3) */
#define POD2G_STATIONARY     1  /* the POD-2G two-grid cycle itself as the iteration (Algorithm 2,
                                   Section 3.3): u <- u + AMG(0; K, f - K u, r1, r2) */

typedef struct pod2g_ctx* pod2g_t;

/* Shared sparsity pattern (host arrays, copied by pod2g_create). */
typedef struct {
    int32_t n_brows;          /* number of block rows (= block columns) */
    int32_t bs;               /* block size: 1, 2 or 3 */
    const int32_t* row_ptr;   /* [n_brows + 1], row_ptr[0] = 0 */
    const int32_t* col_idx;   /* [row_ptr[n_brows]] */
} pod2g_pattern;

/* Per-context options; fill with pod2g_default_opts and override. */
typedef struct {
    double omega;             /* damped-Jacobi weight (default 2/3); needs omega * rho(D^-1 K) < 2 */
    int pre;                  /* r1: pre-relaxation sweeps (default 1; 0..8 FP64, 0 or 1 mixed) */
    int post;                 /* r2: post-relaxation sweeps (default 1; 0..8 FP64, 0 or 1 mixed) */
    int precision;            /* POD2G_FP64 / POD2G_MIXED_FP32PHI / POD2G_MIXED_BF16PHI */
    int beta_pr;              /* 0: beta = r_{k+1}^T s_{k+1} / r_k^T s_k (Algorithm 1); 1: Polak-Ribiere */
    int max_batch;            /* number of instance slots (1..256) */
    size_t hbm_budget;        /* bytes the context may allocate; 0 = no limit */
    int64_t spin_limit;       /* bound on the host's polls of a batched solve (one poll per CUDA-graph
                                 launch of `chunk` iterations; 0 = maxit / chunk + 2). When it runs
                                 out, the unfinished instances stop with status POD2G_TIMEOUT and
                                 their last iterate; the context stays usable. */
    int chunk;                /* PCG iterations per CUDA-graph launch in the batched path (default 8) */
    void* stream;             /* cudaStream_t to run on; NULL = a stream owned by the context */
    int method;               /* POD2G_PCG (default) or POD2G_STATIONARY; iters then counts cycles */
    int smoother;             /* POD2G_SMOOTHER_JACOBI (default) or POD2G_SMOOTHER_SGS. Nodes are
                                 coloured greedily in index order (smallest colour no lower-index
                                 neighbour holds); a sweep visits colour 0, 1, .. and within a node
                                 its components in order (backward: all reversed). Mixed precision
                                 with SGS: beta_pr must be 0. */
    int coarse;               /* POD2G_COARSE_TENSOR (default) or POD2G_COARSE_DF: how the mixed
                                 paths contract K_c = Phi^T (K Phi); ignored by POD2G_FP64 */
} pod2g_opts;

/* Fill *opts with defaults. Never fails. */
void pod2g_default_opts(pod2g_opts* opts);

/* Create a context for one pattern and one POD basis (Section 3.3: Phi_r is the
 * prolongation, Phi_r^T the restriction). k may be 0 (no coarse correction: the
 * preconditioner reduces to r1 + r2 damped-Jacobi sweeps). Allocates all device
 * memory for max_batch slots. Returns POD2G_ADMISSION if that exceeds hbm_budget. */
int pod2g_create(const pod2g_pattern* pattern, const double* phi, int k,
                 const pod2g_opts* opts, pod2g_t* out);

/* Load the matrix values of one parameter instance into a slot and run the
 * per-instance set-up: D^{-1}, K_c = Phi^T K Phi (eq. POD_ROM) symmetrised, and
 * its FP64 Cholesky factor. values: nnzb*bs*bs doubles, host memory if
 * on_device == 0, device memory otherwise. Returns POD2G_NOT_SPD for a
 * non-positive diagonal entry or an indefinite K_c (the slot is then unusable
 * until values are set again). Not for element contexts (POD2G_INVALID_ARG). */
int pod2g_set_values(pod2g_t ctx, int slot, const double* values, int on_device);

/* Same for several slots at once: values_dev points to nslots consecutive
 * instances (nslots * nnzb*bs*bs doubles, device memory). status[i] (host) gets
 * each slot's set-up status; the return value is the first non-OK status. A slot
 * listed twice returns POD2G_INVALID_ARG. */
int pod2g_set_values_batch_dev(pod2g_t ctx, int nslots, const int* slots,
                               const double* values_dev, int* status);

/* ---- Element-factored operator.
 * The finite-element systems of the paper (Section 4.1, Section 4.2) have a
 * material coefficient constant over each element, so K(theta) = sum_e c_e(theta)
 * K_ref scattered to the element's nodes, with one reference element matrix K_ref
 * on a uniform mesh. A context created from this description stores per instance
 * only the n_elems coefficients c_e instead of nnzb*bs*bs matrix values; its
 * kernels form each block's values when they read it. Block (i, j) sums, over the
 * elements e holding both node i (local index a) and node j (local index b), in
 * ascending element index, the FP32 products c_e * K_ref[a, b] (c_e and K_ref
 * rounded to FP32; each product and each partial sum rounded, no fused
 * multiply-add). A fixed node's block row and column hold the identity on its
 * diagonal block and zero elsewhere. The set-up (D^-1, K_c, Cholesky) uses these
 * same FP32 values. */
typedef struct {
    int32_t n_elems;          /* number of elements */
    int32_t npe;              /* nodes per element, 2..8; npe * bs <= 24 */
    const int32_t* conn;      /* [n_elems][npe] block row (node) of each local node; -1 = no node */
    const double* k_ref;      /* [(npe*bs) x (npe*bs)] row-major reference element matrix */
    const uint8_t* fixed;     /* [n_brows] 1 = fixed node (identity row/column); NULL = none */
} pod2g_elements;

/* Like pod2g_create, for a pattern whose blocks hold element contributions as
 * described above (host arrays, copied). Mixed precision modes only (FP64 returns
 * POD2G_INVALID_ARG), and so is a node with more than 8 adjacent elements, an
 * element whose node pair has no stored block, a node listed twice in one
 * element, or a non-symmetric K_ref. */
int pod2g_create_elements(const pod2g_pattern* pattern, const pod2g_elements* elements,
                          const double* phi, int k, const pod2g_opts* opts, pod2g_t* out);

/* Element contexts: load one instance's n_elems coefficients c_e into a slot
 * (host memory if on_device == 0, else device memory) and run its set-up, with
 * the same status rules as pod2g_set_values (non-finite c_e: POD2G_NONFINITE). */
int pod2g_set_coeffs(pod2g_t ctx, int slot, const double* coeffs, int on_device);

/* Several slots at once: coeffs_dev holds nslots * n_elems doubles (device). */
int pod2g_set_coeffs_batch_dev(pod2g_t ctx, int nslots, const int* slots,
                               const double* coeffs_dev, int* status);

/* Element contexts: a registered parametrization of the element coefficients,
 *     c_e(theta) = exp(mu + sigma * sum_j modes[e][j] * theta_j)   (lognormal != 0)
 *     c_e(theta) = mu + sigma * sum_j modes[e][j] * theta_j        (lognormal == 0),
 * the form of a truncated Karhunen-Loeve expansion of the material field evaluated
 * at the elements (the paper's random material properties, Section 4.1, Section 4.2).
 * modes: host [n_elems][m] doubles (copied), 1 <= m <= 64. */
int pod2g_set_field(pod2g_t ctx, const double* modes, int m, double mu, double sigma, int lognormal);

/* Instance set-up from the parameters theta (host, m doubles): c_e(theta) is
 * evaluated on the device (FP64, then rounded to FP32 like pod2g_set_coeffs), then
 * the set-up of pod2g_set_coeffs. A non-finite c_e gives POD2G_NONFINITE, c_e <= 0
 * POD2G_NOT_SPD. POD2G_INVALID_ARG without a registered field. */
int pod2g_set_theta(pod2g_t ctx, int slot, const double* theta);
/* Several slots: theta holds nslots * m doubles (host). */
int pod2g_set_theta_batch(pod2g_t ctx, int nslots, const int* slots, const double* theta, int* status);

/* Solve one instance (Algorithm 3). b, x0 (NULL: zero) and x are host arrays of
 * n doubles. iters / relres may be NULL. *relres is the true relative residual
 * ||b - K x||_2 / ||b||_2 of the returned x, recomputed in FP64 at exit (see
 * Conventions), not the recurrence residual of the stopping test. */
int pod2g_solve(pod2g_t ctx, int slot, const double* b, const double* x0, double tol,
                int maxit, double* x, int* iters, double* relres);

/* Solve nslots instances together (host arrays: b[i], x0[i] (x0 or x0[i] may be
 * NULL), x[i], each n doubles). iters/relres/status: host arrays of nslots (may
 * be NULL). Returns the first non-OK per-slot status, or OK. */
int pod2g_solve_batch(pod2g_t ctx, int nslots, const int* slots, const double* const* b,
                      const double* const* x0, double tol, int maxit, double* const* x,
                      int* iters, double* relres, int* status);

/* Device-memory variant: b_dev, x0_dev (NULL: zero) and x_dev hold nslots
 * consecutive vectors of n doubles. iters/relres/status are host arrays. */
int pod2g_solve_batch_dev(pod2g_t ctx, int nslots, const int* slots, const double* b_dev,
                          const double* x0_dev, double tol, int maxit, double* x_dev,
                          int* iters, double* relres, int* status);

/* POD reduced-order solution (Section 3.3, steps 3-4): x_i = Phi K_c^{-1} Phi^T b_i
 * for set-up slots, with the coarse matrix of each slot's set-up; the
 * reduced-order approximation that the paper's surrogate stands in for, to be
 * passed as x0. b_dev, x_dev: nslots consecutive vectors of n doubles (device).
 * k = 0 gives x = 0. Blocks until done. */
int pod2g_rom_solution_dev(pod2g_t ctx, int nslots, const int* slots, const double* b_dev,
                           double* x_dev);

/* Serving. A request carries one instance's values (host, nnzb*bs*bs doubles),
 * its right-hand side and an optional x0 (host, n doubles each); the library
 * copies them. Requests are admitted into free slots of the context's batch as
 * slots free up (continuous batching: converged instances retire and waiting
 * requests join the running batch between CUDA-graph launches). Returns
 * POD2G_ADMISSION if the waiting queue already holds max_queue requests
 * (pod2g_serve_start). *ticket identifies the request. */
int pod2g_serve_start(pod2g_t ctx, int max_queue);
int pod2g_submit(pod2g_t ctx, const double* values, const double* b, const double* x0,
                 double tol, int maxit, uint64_t* ticket);
/* (For a context from pod2g_create_elements, `values` holds the request's n_elems
 * coefficients.)
 * Non-blocking: POD2G_PENDING until the request finishes; then copies x (host, n
 * doubles; may be NULL), iters, relres, status (may be NULL), returns OK and
 * forgets the ticket. latency_s (may be NULL) = submit-to-completion seconds. */
int pod2g_poll(pod2g_t ctx, uint64_t ticket, double* x, int* iters, double* relres,
               int* status, double* latency_s);
int pod2g_serve_stop(pod2g_t ctx);
/* Serving by parameters (element contexts with a registered field): a request
 * carries theta (host, m doubles) instead of coefficients; otherwise as pod2g_submit. */
int pod2g_submit_theta(pod2g_t ctx, const double* theta, const double* b, const double* x0,
                       double tol, int maxit, uint64_t* ticket);

/* Query sizes: n, nnzb, k, max_batch (any pointer may be NULL). */
int pod2g_info(pod2g_t ctx, int* n, int* nnzb, int* k, int* max_batch);

/* Number of kernel launches the context has issued (for launch accounting). */
int64_t pod2g_launch_count(pod2g_t ctx);

/* Device memory held by the context, in bytes (what pod2g_create allocated and
 * checked against hbm_budget); 0 for NULL. Serving front ends use it to admit
 * further problems under a shared HBM budget. */
int64_t pod2g_device_bytes(pod2g_t ctx);

/* Per-kernel timing of the batched PCG iteration (mixed contexts only). With
 * on != 0, CUDA events are recorded around each of the 8 kernels of every
 * iteration inside the CUDA graph, and accumulated after each graph launch;
 * switching resets the totals. pod2g_kernel_times copies, for kernel j =
 * 0..7 (p update, K p, x/r update, pre-smoothing, restriction, coarse solve,
 * prolongation, post-smoothing), the total milliseconds ms[j] and the number of
 * timed launches launches[j] (arrays of 8; either may be NULL). */
int pod2g_kernel_timing(pod2g_t ctx, int on);
int pod2g_kernel_times(pod2g_t ctx, double* ms, int64_t* launches);

/* The coarse matrix of a set-up slot (Section 3.3, eq. POD_ROM): copies its k x k
 * lower-triangular Cholesky factor L, K_c = L L^T with K_c = (Phi^T K Phi +
 * (Phi^T K Phi)^T) / 2, row-major into L (host, k*k doubles; the strict upper triangle
 * is zero). POD2G_INVALID_ARG for a slot without a valid set-up. */
int pod2g_coarse_factor(pod2g_t ctx, int slot, double* L);

/* ---- Surrogate initial guess (Section 3.2): u_sur(theta) = s * decoder(FFNN(theta)).
 * FFNN: h1 = tanh(W1 theta + b1), h2 = tanh(W2 h1 + b2), o = W3 h2 + b3 (FP64 on the device),
 * latent z = z_mean + z_std * o; decoder: u = Psi z with ks modes Psi (stored in FP32, the
 * product accumulated in FP32); s = the query's load factor. The solver accepts any x0: pass the
 * prediction as x0_dev of pod2g_solve_batch_dev. The object is independent of any solver
 * context. */
typedef struct pod2g_sur* pod2g_sur_t;
/* Copies all arrays (host): psi [n x ks] column-major; w1 [hidden x m], w2 [hidden x hidden],
 * w3 [ks x hidden] row-major; b1, b2 [hidden]; b3, z_mean, z_std [ks]. Limits: 1 <= m <= 64,
 * 1 <= hidden <= 256, 1 <= ks <= 256 (POD2G_INVALID_ARG otherwise). stream: the cudaStream_t the
 * predictions run in (NULL = a stream owned by the object). */
int pod2g_surrogate_create(int64_t n, int m, int ks, int hidden, const double* psi, const double* w1,
                           const double* b1, const double* w2, const double* b2, const double* w3,
                           const double* b3, const double* z_mean, const double* z_std, void* stream,
                           pod2g_sur_t* out);
/* x_dev (device, nq consecutive vectors of n doubles) = the predictions for theta (host, nq x m
 * row-major) and scale (host, nq load factors; NULL = 1). Queued in the object's stream; returns
 * once queued (the host arrays may be reused at return). */
int pod2g_surrogate_predict_dev(pod2g_sur_t sur, int nq, const double* theta, const double* scale,
                                double* x_dev);
void pod2g_surrogate_destroy(pod2g_sur_t sur);

/* Free all device memory of the context. NULL is ignored. */
void pod2g_destroy(pod2g_t ctx);

/* Solve without allocating device memory (the paper has no counterpart: this is
 * a deployment variant of pod2g_solve on a POD2G_FP64 context).
 *
 * For callers that cannot call cudaMalloc: code whose device memory is owned by
 * another allocator (a framework's caching allocator, a pool reserved at start-up),
 * callers that must not trigger the device-wide synchronisation that cudaMalloc /
 * cudaFree can imply, and embedders that only hand over buffers they already own.
 * It runs the same kernels as pod2g_solve on an FP64 context (same results), but
 * every scratch buffer lives in one file-scope static device array of about
 * 10.5 MB, which each GPU that loads the library holds until the process exits.
 * Nothing is allocated or freed; no context is needed.
 *
 * Inputs (device pointers, read only): the block-CSR pattern (row_ptr_dev
 * [n_brows+1], col_idx_dev [nnzb], sorted columns, diagonal present), values_dev
 * (nnzb*bs*bs doubles, row-major blocks), phi_dev (n*k doubles, column-major, may
 * be NULL when k = 0), b_dev and x0_dev (n doubles; x0_dev NULL = zero). opts:
 * omega, pre, post, beta_pr are used (NULL = defaults); method must be POD2G_PCG and
 * smoother POD2G_SMOOTHER_JACOBI (anything else returns POD2G_INVALID_ARG); precision,
 * max_batch, hbm_budget, spin_limit, chunk and stream are ignored. Output: x_dev (n doubles, device);
 * iters, relres, status (host, may be NULL) as for pod2g_solve. stream: the
 * cudaStream_t to run on (NULL = the legacy default stream).
 *
 * Limits: n = n_brows*bs <= POD2G_NOALLOC_MAX_N and k <= POD2G_NOALLOC_MAX_K;
 * larger sizes return POD2G_TOO_LARGE before any device work. An invalid pattern
 * returns POD2G_INVALID_ARG.
 *
 * Set-up: every call looks up the device address of the static array in the current
 * device's context (cudaGetSymbolAddress, a host query; the first such query on a
 * device may initialise the module there, so make the first call before any CUDA
 * stream capture). Every call shares the array and overwrites what the previous call
 * left there; the counters that must start at zero are cleared at the start of each
 * call. Calls that overlap on the GPU would race on the array: the library
 * serialises calls made from one process with a lock, and each call, on every return
 * path including errors, waits for the work it queued on `stream` before it returns.
 * Returns the solve status (POD2G_OK when converged), or an error code. */
#define POD2G_NOALLOC_MAX_N 16384
#define POD2G_NOALLOC_MAX_K 32
int pod2g_solve_noalloc(int32_t n_brows, int32_t bs, int32_t nnzb, const int32_t* row_ptr_dev,
                        const int32_t* col_idx_dev, const double* values_dev, const double* phi_dev, int k,
                        const pod2g_opts* opts, const double* b_dev, const double* x0_dev, double tol,
                        int maxit, double* x_dev, int* iters, double* relres, int* status, void* stream);

/* ---- Launch shapes of the batched (mixed-precision) path: CTAs per grid of each
 * kernel group. A shape changes only the grouping of partial sums, so results are
 * deterministic for a given shape and differ between shapes at rounding level. */
typedef struct {
    int32_t grid_rows;      /* smoother / residual row kernels: multiple of 8, 8..8*SMs */
    int32_t grid_restrict;  /* restriction Phi^T r: multiple of 8, 8..4*SMs */
    int32_t grid_prol;      /* prolongation: 1..8*SMs */
    int32_t grid_vec;       /* vector updates (p; x and r): 1..8*SMs */
    int32_t grid_spmv;      /* outer SpMV q = K p: multiple of 8, 8..8*SMs */
    int32_t rows_kernel;    /* form of the sparse row kernels: bit 0 the smoother passes, bit 1 the
                               outer SpMV use the warp-staged kernels (each warp copies the matrix
                               values of its rows into shared memory with bulk asynchronous copies
                               ahead of use; assembled operators with 4..64 slot lanes and Jacobi
                               relaxation) or, with one slot lane, the kernels that give each block row
                               a group of 8 lanes; bit 2: the prolongation and post-smoothing run as one
                               pass that forms K y2 = (r - r1) + (K Phi) e_c from K Phi stored per slot
                               at set-up, without a sweep over the matrix (contexts that store K Phi:
                               assembled, Jacobi with r1 = r2 = 1, K Phi smaller than the values and
                               within the HBM budget). 0 = one thread per block row and slot, and the
                               post-smoothing as a sweep. Bit 3: whole iterations run in one
                               cooperative launch of grid_persist CTAs with grid-wide barriers between
                               the phases (assembled, Jacobi with r1 = r2 = 1, at most 64 slot lanes,
                               K Phi stored or no coarse space; K Phi is kept for this where n * lanes
                               <= 2^20); not a default (it measured at best at parity with the graph
                               path), the autotuner selects it where it is faster. Default: bits 0, 1
                               and 2 where the context supports them, except bit 1 with one slot lane
                               and 1x1 or 2x2 blocks (one thread per row measured faster there). */
    int32_t restrict_rows;  /* rows of Phi and r1 per shared-memory chunk of the bulk-staged
                               restriction (its tile; multiple of 4, 4..256, within 200 KB of shared
                               memory; 4 or more slot lanes); 0 = the default (~24 KB per chunk) */
    int32_t grid_persist;   /* CTAs of the persistent launch (rows_kernel bit 3): 1..the number that
                               fit on the GPU at once, at most 4*SMs; 0 where the form does not apply */
} pod2g_tuning;

/* Current shape (mixed contexts; FP64 contexts return POD2G_INVALID_ARG). */
int pod2g_get_tuning(pod2g_t ctx, pod2g_tuning* out);
/* Set a shape; POD2G_INVALID_ARG if a field is out of range or the context is serving. */
int pod2g_set_tuning(pod2g_t ctx, const pod2g_tuning* t);
/* Autotuner: for five candidate shapes (and, where they apply, five grid sizes of the
 * warp-staged row kernels, then half and twice the restriction's default chunk, then the
 * persistent launch at up to four grid sizes against the graph of the chosen shape, timed
 * per launch), solve the given set-up slots with right-hand
 * sides b_dev (nslots consecutive vectors of n doubles, device) for `iters`
 * iterations (rounded up to whole graph launches), timing each kernel with CUDA
 * events, and keep per kernel group the fastest candidate (kernel form and grid). The slots are left idle
 * (their set-up stays valid). *out (may be NULL) receives the chosen shape. Not
 * while serving. */
int pod2g_autotune(pod2g_t ctx, int nslots, const int* slots, const double* b_dev, int iters,
                   pod2g_tuning* out);

/* Static message for a status code. Never NULL. */
const char* pod2g_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* POD2G_H */
