// Plain FP64 path: one instance at a time, one kernel per step, convergence
// checked on the host after every iteration, no CUDA graphs. It is the direct
// statement of Algorithm 3 (arXiv 2207.02543, Section 3.4) with the two-grid
// cycle of Algorithm 2 (P = Phi_r, Section 3.3) and damped-Jacobi relaxation, in
// FP64 throughout (or, as the stationary method, the two-grid cycle iterated on
// its own); it serves the FP64 workloads and is the baseline that the
// batched mixed-precision path is measured against.
#include "common.cuh"

#include <algorithm>
#include <cmath>

namespace {

enum { S_RS = 0, S_PQ = 1, S_RR = 2, S_BB = 3, S_RSNEW = 4, S_RSX = 5, S_ALPHA = 6, S_BETA = 7, S_N = 16 };
enum RowMode { ROW_AX = 0, ROW_RES = 1, ROW_SMOOTH = 2 };

// Block-sum of one double per thread in fixed order; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    return s;
}

// Finish a scalar reduction: CTA partial -> part[blockIdx]; the last CTA sums the
// partials in CTA order into *out.
__device__ __forceinline__ void finish_scalar(double v, double* part, unsigned* counter, double* out) {
    double s = block_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
    if (!last_cta_arrive(counter)) return;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int g = 0; g < (int)gridDim.x; ++g) t += part[g];
        *out = t;
    }
    last_cta_reset(counter);
}

// One row of K x for unknown d (block row i, component rr).
__device__ __forceinline__ double row_dot(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                                          const double* __restrict__ vals, const double* __restrict__ x, int bs,
                                          int i, int rr) {
    double acc = 0.0;
    for (int blk = row_ptr[i]; blk < row_ptr[i + 1]; ++blk) {
        int j = col_idx[blk];
        const double* vb = vals + (long long)blk * bs * bs + rr * bs;
        for (int cc = 0; cc < bs; ++cc) acc = fma(vb[cc], x[j * bs + cc], acc);
    }
    return acc;
}

// out = K x (AX), f - K x (RES) or x + omega D^{-1} (f - K x) (SMOOTH).
// Optional dot: *dot_out = x^T out (AX, gives p^T K p) or f^T f (RES, gives b^T b).
__global__ void k_row(int mode, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                      const double* __restrict__ vals, const double* __restrict__ dinv, double omega,
                      const double* __restrict__ x, const double* __restrict__ f, double* __restrict__ out, int nb,
                      int bs, double* part, unsigned* counter, double* dot_out) {
    int n = nb * bs;
    double d_acc = 0.0;
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < n; d += gridDim.x * blockDim.x) {
        int i = d / bs, rr = d - i * bs;
        double kx = x ? row_dot(row_ptr, col_idx, vals, x, bs, i, rr) : 0.0;
        double v;
        if (mode == ROW_AX) {
            v = kx;
            if (dot_out) d_acc = fma(x[d], v, d_acc);
        } else if (mode == ROW_RES) {
            v = f[d] - kx;
            if (dot_out) d_acc = fma(f[d], f[d], d_acc);
        } else {
            v = (x ? x[d] : 0.0) + omega * dinv[d] * (f[d] - kx);
        }
        out[d] = v;
    }
    if (dot_out) finish_scalar(d_acc, part, counter, dot_out);
}

// x += alpha p; r -= alpha q with alpha = rs / pq; *rr_out = r^T r.
__global__ void k_update_xr(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                            const double* __restrict__ q, int n, double* scal, double* part, unsigned* counter) {
    double pq = scal[S_PQ];
    if (!(pq > 0.0) || !isfinite(pq)) return;  // breakdown: the host stops on the previous iterate
    double alpha = scal[S_RS] / pq;
    double acc = 0.0;
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < n; d += gridDim.x * blockDim.x) {
        x[d] = fma(alpha, p[d], x[d]);
        double rv = fma(-alpha, q[d], r[d]);
        r[d] = rv;
        acc = fma(rv, rv, acc);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) scal[S_ALPHA] = alpha;
    finish_scalar(acc, part, counter, scal + S_RR);
}

// dot products r^T s (and r^T s_old for Polak-Ribiere)
__global__ void k_dot2(const double* __restrict__ r, const double* __restrict__ s, const double* __restrict__ s_old,
                       int n, double* part, unsigned* counter, double* out, double* part2, unsigned* counter2,
                       double* out2) {
    double a = 0.0, b = 0.0;
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < n; d += gridDim.x * blockDim.x) {
        a = fma(r[d], s[d], a);
        if (s_old) b = fma(r[d], s_old[d], b);
    }
    finish_scalar(a, part, counter, out);
    if (s_old) finish_scalar(b, part2, counter2, out2);
}

// p = s + beta p with beta = rs_new / rs (Fletcher-Reeves form of Algorithm 1)
// or (rs_new - rs_cross) / rs (Polak-Ribiere); then rs <- rs_new. first: p = s.
__global__ void k_update_p(double* __restrict__ p, const double* __restrict__ s, int n, double* scal, int first,
                           int pr) {
    double beta = first ? 0.0 : (pr ? (scal[S_RSNEW] - scal[S_RSX]) / scal[S_RS] : scal[S_RSNEW] / scal[S_RS]);
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < n; d += gridDim.x * blockDim.x)
        p[d] = fma(beta, p[d], s[d]);
    if (blockIdx.x == 0 && threadIdx.x == 0) scal[S_BETA] = beta;
}

// One Gauss-Seidel step over the nodes of one colour (FP64, pointwise, eq.
// GaussSeidel): for each node and each component in order (reverse if bwd),
// y_d += (f - K y)_d / K_dd with the current y. Nodes of one colour do not couple.
__global__ void k_gs64(const int32_t* __restrict__ cnodes, int cnt, const int32_t* __restrict__ row_ptr,
                       const int32_t* __restrict__ col_idx, const double* __restrict__ vals,
                       const double* __restrict__ dinv, const double* __restrict__ f, double* y, int bs, int bwd) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
        const int i = cnodes[t];
        for (int q = 0; q < bs; ++q) {
            const int a = bwd ? bs - 1 - q : q;
            const int d = i * bs + a;
            const double kx = row_dot(row_ptr, col_idx, vals, y, bs, i, a);
            y[d] += dinv[d] * (f[d] - kx);
        }
    }
}

// x += s (the correction of one stationary two-grid cycle)
__global__ void k_add(double* __restrict__ x, const double* __restrict__ s, int n) {
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < n; d += gridDim.x * blockDim.x) x[d] += s[d];
}

__global__ void k_copy_scalar(double* scal, int dst, int src) {
    if (threadIdx.x == 0 && blockIdx.x == 0) scal[dst] = scal[src];
}

// Restriction c = Phi^T t (Phi row-major [n][kp]) split over CTAs; the last CTA
// sums partials in CTA order and solves L L^T e_c = c (forward, then backward
// substitution, column-oriented, one warp). e_c overwrites c.
__global__ void k_restrict_solve(const double* __restrict__ phi, const double* __restrict__ t, int n, int k, int kp,
                                 const double* __restrict__ L, double* part, unsigned* counter, double* c) {
    __shared__ double sh[POD2G_THREADS / 32][POD2G_MAX_K];
    double acc[POD2G_MAX_K];
    for (int m = 0; m < k; ++m) acc[m] = 0.0;
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < n; d += gridDim.x * blockDim.x) {
        double tv = t[d];
        const double* pr = phi + (long long)d * kp;
        for (int m = 0; m < k; ++m) acc[m] = fma(pr[m], tv, acc[m]);
    }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int m = 0; m < k; ++m) {
        double v = acc[m];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (l == 0) sh[w][m] = v;
    }
    __syncthreads();
    for (int m = threadIdx.x; m < k; m += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i][m];
        part[(long long)blockIdx.x * kp + m] = s;
    }
    if (!last_cta_arrive(counter)) return;
    __shared__ double cv[POD2G_MAX_K];
    for (int m = threadIdx.x; m < k; m += blockDim.x) {
        double s = 0.0;
        for (int g = 0; g < (int)gridDim.x; ++g) s += part[(long long)g * kp + m];
        cv[m] = s;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        // forward: L y = c
        for (int i = 0; i < k; ++i) {
            double yi = cv[i] / L[i * k + i];
            __syncwarp();
            if (l == 0) cv[i] = yi;
            for (int j = i + 1 + l; j < k; j += 32) cv[j] -= L[j * k + i] * yi;
            __syncwarp();
        }
        // backward: L^T e = y
        for (int i = k - 1; i >= 0; --i) {
            double ei = cv[i] / L[i * k + i];
            __syncwarp();
            if (l == 0) cv[i] = ei;
            for (int j = l; j < i; j += 32) cv[j] -= L[i * k + j] * ei;
            __syncwarp();
        }
        for (int m = l; m < k; m += 32) c[m] = cv[m];
    }
    last_cta_reset(counter);
}

// y += Phi e_c
__global__ void k_prolong(double* __restrict__ y, const double* __restrict__ phi, const double* __restrict__ ec, int n,
                          int k, int kp) {
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < n; d += gridDim.x * blockDim.x) {
        const double* pr = phi + (long long)d * kp;
        double v = y[d];
        for (int m = 0; m < k; ++m) v = fma(pr[m], ec[m], v);
        y[d] = v;
    }
}

}  // namespace

// one application of the preconditioner s = AMG(0; K, r, r1, r2) (Algorithm 3)
static int plain_precond(pod2g_ctx* c, int slot, const double* r, double* s) {
    const int T = POD2G_THREADS, n = c->n;
    const int G = std::max(1, std::min(ceil_div(n, T), 4 * c->num_sms));
    const double* vals = c->d_vals64 + (size_t)slot * c->nnzb * c->bs * c->bs;
    const double* dinv = c->d_dinv64 + (size_t)slot * n;
    double* y = c->d_y64;
    double* t = c->d_t64;
    const bool gs = c->smoother == POD2G_SMOOTHER_SGS;
    auto sweep = [&](int bwd) -> int {
        for (int q = 0; q < c->ncolours; ++q) {
            const int col = bwd ? c->ncolours - 1 - q : q;
            const int cnt = c->coff[col + 1] - c->coff[col];
            if (cnt == 0) continue;
            k_gs64<<<std::max(1, std::min(ceil_div(cnt, T), 4 * c->num_sms)), T, 0, c->stream>>>(
                c->d_cnodes + c->coff[col], cnt, c->d_row_ptr, c->d_col_idx, vals, dinv, r, y, c->bs, bwd);
            P2G_TRY(pod2g_check_launch(c));
        }
        return POD2G_OK;
    };
    // pre-relaxation from y = 0
    if (gs) {
        P2G_CUDA(cudaMemsetAsync(y, 0, sizeof(double) * n, c->stream));
        for (int it = 0; it < c->pre; ++it) P2G_TRY(sweep(0));
    } else if (c->pre == 0) {
        P2G_CUDA(cudaMemsetAsync(y, 0, sizeof(double) * n, c->stream));
    } else {
        k_row<<<G, T, 0, c->stream>>>(ROW_SMOOTH, c->d_row_ptr, c->d_col_idx, vals, dinv, c->omega, nullptr, r, y,
                                      c->nb, c->bs, nullptr, nullptr, nullptr);
        P2G_TRY(pod2g_check_launch(c));
        for (int it = 1; it < c->pre; ++it) {
            k_row<<<G, T, 0, c->stream>>>(ROW_SMOOTH, c->d_row_ptr, c->d_col_idx, vals, dinv, c->omega, y, r, t,
                                          c->nb, c->bs, nullptr, nullptr, nullptr);
            P2G_TRY(pod2g_check_launch(c));
            std::swap(y, t);
        }
    }
    if (c->k > 0) {
        // residual, restriction, coarse solve, prolongation + correction
        k_row<<<G, T, 0, c->stream>>>(ROW_RES, c->d_row_ptr, c->d_col_idx, vals, dinv, c->omega, y, r, t, c->nb,
                                      c->bs, nullptr, nullptr, nullptr);
        P2G_TRY(pod2g_check_launch(c));
        const int Gr = std::max(1, std::min(ceil_div(n, T), 2 * c->num_sms));
        k_restrict_solve<<<Gr, T, 0, c->stream>>>(c->d_phi64, t, n, c->k, c->kp,
                                                  c->d_Lc + (size_t)slot * c->k * c->k, c->d_part64,
                                                  c->d_counters + CNT_PLAIN, c->d_c64);
        P2G_TRY(pod2g_check_launch(c));
        k_prolong<<<G, T, 0, c->stream>>>(y, c->d_phi64, c->d_c64, n, c->k, c->kp);
        P2G_TRY(pod2g_check_launch(c));
    }
    // post-relaxation; the last sweep writes s
    if (gs) {
        for (int it = 0; it < c->post; ++it) P2G_TRY(sweep(1));
        P2G_CUDA(cudaMemcpyAsync(s, y, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    } else if (c->post == 0) {
        P2G_CUDA(cudaMemcpyAsync(s, y, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    } else {
        for (int it = 0; it < c->post; ++it) {
            double* out = (it == c->post - 1) ? s : t;
            k_row<<<G, T, 0, c->stream>>>(ROW_SMOOTH, c->d_row_ptr, c->d_col_idx, vals, dinv, c->omega, y, r, out,
                                          c->nb, c->bs, nullptr, nullptr, nullptr);
            P2G_TRY(pod2g_check_launch(c));
            if (out == t) std::swap(y, t);
        }
    }
    if (y != c->d_y64) std::swap(c->d_y64, c->d_t64);
    return POD2G_OK;
}

static int read_scalars(pod2g_ctx* c) {
    P2G_CUDA(cudaMemcpyAsync(c->h_scal64, c->d_scal64, sizeof(double) * S_N, cudaMemcpyDeviceToHost, c->stream));
    P2G_CUDA(cudaStreamSynchronize(c->stream));
    return POD2G_OK;
}

int plain_solve(pod2g_ctx* c, int slot, const double* b_dev, const double* x0_dev, double tol, int maxit,
                double* x_dev, int* iters_out, double* relres_out, int* status_out) {
    const int T = POD2G_THREADS, n = c->n;
    const int G = std::max(1, std::min(ceil_div(n, T), 4 * c->num_sms));
    const double* vals = c->d_vals64 + (size_t)slot * c->nnzb * c->bs * c->bs;
    const double* dinv = c->d_dinv64 + (size_t)slot * n;
    double* part = c->d_part64;
    unsigned* cnt = c->d_counters + CNT_PLAIN;
    double* sc = c->d_scal64;
    double *x = c->d_x64, *r = c->d_r64, *s = c->d_s64, *p = c->d_p64, *q = c->d_q64;
    // u0, r0 = f - K u0, ||f||^2
    if (x0_dev) {
        P2G_CUDA(cudaMemcpyAsync(x, x0_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    } else {
        P2G_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, c->stream));
    }
    k_row<<<G, T, 0, c->stream>>>(ROW_RES, c->d_row_ptr, c->d_col_idx, vals, dinv, c->omega, x, b_dev, r, c->nb,
                                  c->bs, part, cnt, sc + S_BB);
    P2G_TRY(pod2g_check_launch(c));
    k_dot2<<<G, T, 0, c->stream>>>(r, r, nullptr, n, part, cnt, sc + S_RR, nullptr, nullptr, nullptr);
    P2G_TRY(pod2g_check_launch(c));
    P2G_TRY(read_scalars(c));
    const double bb = c->h_scal64[S_BB];
    int status = POD2G_NOT_CONVERGED, k = 0;
    if (bb == 0.0) {
        P2G_CUDA(cudaMemsetAsync(x_dev, 0, sizeof(double) * n, c->stream));
        P2G_CUDA(cudaStreamSynchronize(c->stream));
        if (iters_out) *iters_out = 0;
        if (relres_out) *relres_out = 0.0;
        if (status_out) *status_out = POD2G_OK;
        return POD2G_OK;
    }
    if (!std::isfinite(bb) || !std::isfinite(c->h_scal64[S_RR])) {
        status = POD2G_NONFINITE;
    } else if (c->method == POD2G_STATIONARY) {
        // Algorithm 2 as the solver: u <- u + AMG(0; K, f - K u, r1, r2), which is one
        // two-grid cycle applied to u; the residual is recomputed from u every cycle.
        const double tol2 = tol * tol * bb;
        double rr = c->h_scal64[S_RR];
        while (true) {
            if (rr <= tol2) { status = POD2G_OK; break; }
            if (k >= maxit) { status = POD2G_NOT_CONVERGED; break; }
            P2G_TRY(plain_precond(c, slot, r, s));
            k_add<<<G, T, 0, c->stream>>>(x, s, n);
            P2G_TRY(pod2g_check_launch(c));
            k_row<<<G, T, 0, c->stream>>>(ROW_RES, c->d_row_ptr, c->d_col_idx, vals, dinv, c->omega, x, b_dev, r,
                                          c->nb, c->bs, nullptr, nullptr, nullptr);
            P2G_TRY(pod2g_check_launch(c));
            k_dot2<<<G, T, 0, c->stream>>>(r, r, nullptr, n, part, cnt, sc + S_RR, nullptr, nullptr, nullptr);
            P2G_TRY(pod2g_check_launch(c));
            P2G_TRY(read_scalars(c));
            ++k;
            rr = c->h_scal64[S_RR];
            if (!std::isfinite(rr)) { status = POD2G_NONFINITE; break; }
        }
    } else {
        const double tol2 = tol * tol * bb;
        double rr = c->h_scal64[S_RR];
        // s0 = AMG(0; K, r0, r1, r2); p0 = s0; rs = r0^T s0
        P2G_TRY(plain_precond(c, slot, r, s));
        k_dot2<<<G, T, 0, c->stream>>>(r, s, nullptr, n, part, cnt, sc + S_RSNEW, nullptr, nullptr, nullptr);
        P2G_TRY(pod2g_check_launch(c));
        k_update_p<<<G, T, 0, c->stream>>>(p, s, n, sc, 1, 0);
        P2G_TRY(pod2g_check_launch(c));
        k_copy_scalar<<<1, 32, 0, c->stream>>>(sc, S_RS, S_RSNEW);
        P2G_TRY(pod2g_check_launch(c));
        P2G_TRY(read_scalars(c));
        double rs = c->h_scal64[S_RS];
        while (true) {
            if (rr <= tol2) { status = POD2G_OK; break; }
            if (k >= maxit) { status = POD2G_NOT_CONVERGED; break; }
            if (!(rs > 0.0) || !std::isfinite(rs)) { status = POD2G_BREAKDOWN; break; }
            // q = K p; p^T q
            k_row<<<G, T, 0, c->stream>>>(ROW_AX, c->d_row_ptr, c->d_col_idx, vals, dinv, c->omega, p, nullptr, q,
                                          c->nb, c->bs, part, cnt, sc + S_PQ);
            P2G_TRY(pod2g_check_launch(c));
            k_update_xr<<<G, T, 0, c->stream>>>(x, r, p, q, n, sc, part, cnt);
            P2G_TRY(pod2g_check_launch(c));
            P2G_TRY(read_scalars(c));  // host convergence check every iteration
            double pq = c->h_scal64[S_PQ];
            if (!(pq > 0.0) || !std::isfinite(pq)) {  // x, r were left unchanged on the device
                status = POD2G_BREAKDOWN;
                break;
            }
            ++k;
            rr = c->h_scal64[S_RR];
            if (!std::isfinite(rr)) { status = POD2G_NONFINITE; break; }
            if (rr <= tol2) { status = POD2G_OK; break; }
            // s = AMG(0; K, r, r1, r2); beta; p = s + beta p
            if (c->beta_pr)
                P2G_CUDA(cudaMemcpyAsync(c->d_w64, s, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
            P2G_TRY(plain_precond(c, slot, r, s));
            k_dot2<<<G, T, 0, c->stream>>>(r, s, c->beta_pr ? c->d_w64 : nullptr, n, part, cnt, sc + S_RSNEW,
                                           part + 4 * c->num_sms, c->d_counters + CNT_PLAIN + 1, sc + S_RSX);
            P2G_TRY(pod2g_check_launch(c));
            k_update_p<<<G, T, 0, c->stream>>>(p, s, n, sc, 0, c->beta_pr);
            P2G_TRY(pod2g_check_launch(c));
            k_copy_scalar<<<1, 32, 0, c->stream>>>(sc, S_RS, S_RSNEW);
            P2G_TRY(pod2g_check_launch(c));
            P2G_TRY(read_scalars(c));
            rs = c->h_scal64[S_RS];
        }
    }
    // true residual ||b - K x|| / ||b||
    k_row<<<G, T, 0, c->stream>>>(ROW_RES, c->d_row_ptr, c->d_col_idx, vals, dinv, c->omega, x, b_dev, q, c->nb,
                                  c->bs, nullptr, nullptr, nullptr);
    P2G_TRY(pod2g_check_launch(c));
    k_dot2<<<G, T, 0, c->stream>>>(q, q, nullptr, n, part, cnt, sc + S_RR, nullptr, nullptr, nullptr);
    P2G_TRY(pod2g_check_launch(c));
    P2G_CUDA(cudaMemcpyAsync(x_dev, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    P2G_TRY(read_scalars(c));
    if (iters_out) *iters_out = k;
    if (relres_out) *relres_out = std::sqrt(c->h_scal64[S_RR] / bb);
    if (status_out) *status_out = status;
    return POD2G_OK;
}
