// POD reduced-order solution x = Phi K_c^{-1} Phi^T b (arXiv 2207.02543,
// Section 3.3, steps 3-4: the Galerkin projection onto the POD basis, solved
// with the coarse matrix K_c = Phi^T K Phi of the slot's set-up). It is the
// reduced-order approximation that the paper's surrogate replaces; the solver
// takes it as an initial guess.
//
// Three kernels per call, all slots of the call at once: per-CTA partials of
// Phi^T b in FP64 (FP32 or FP64 basis), one CTA per slot summing them in CTA
// order and solving L L^T e = c, and the prolongation Phi e in FP64.
#include "common.cuh"

namespace {

// partial[i][g][m] = sum over the rows of chunk g of Phi[d][m] * b_i[d]
template <typename PHI>
__global__ void k_rom_restrict(const PHI* __restrict__ phi, const double* __restrict__ b, int n, int kp,
                               double* __restrict__ partial) {
    extern __shared__ double s_red[];  // [blockDim.x]
    const int g = blockIdx.x, i = blockIdx.y, G = gridDim.x;
    const int groups = blockDim.x / kp;
    const int m = threadIdx.x % kp, q = threadIdx.x / kp;
    const long long per = (n + G - 1) / G;
    const long long d0 = g * per, d1 = min((long long)n, d0 + per);
    double acc = 0.0;
    if (q < groups)
        for (long long d = d0 + q; d < d1; d += groups) acc = fma((double)phi[d * kp + m], b[(long long)i * n + d], acc);
    s_red[threadIdx.x] = acc;
    __syncthreads();
    if ((int)threadIdx.x < kp) {
        double s = 0.0;
        for (int t = 0; t < groups; ++t) s += s_red[t * kp + threadIdx.x];
        partial[((long long)i * G + g) * kp + threadIdx.x] = s;
    }
}

// e_i = L_i^{-T} L_i^{-1} c_i with c_i = sum over chunks (in order); one CTA per slot.
__global__ void k_rom_solve(const double* __restrict__ partial, int G, int k, int kp, const int* __restrict__ slots,
                            const double* __restrict__ Lc, double* __restrict__ e) {
    __shared__ double cv[POD2G_MAX_K];
    const int i = blockIdx.x;
    for (int m = threadIdx.x; m < kp; m += blockDim.x) {
        double s = 0.0;
        for (int g = 0; g < G; ++g) s += partial[((long long)i * G + g) * kp + m];
        cv[m] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double* L = Lc + (long long)slots[i] * k * k;
        for (int r = 0; r < k; ++r) {
            double v = cv[r];
            for (int t = 0; t < r; ++t) v -= L[r * k + t] * cv[t];
            cv[r] = v / L[r * k + r];
        }
        for (int r = k - 1; r >= 0; --r) {
            double v = cv[r];
            for (int t = r + 1; t < k; ++t) v -= L[t * k + r] * cv[t];
            cv[r] = v / L[r * k + r];
        }
    }
    __syncthreads();
    for (int m = threadIdx.x; m < kp; m += blockDim.x) e[(long long)i * kp + m] = m < k ? cv[m] : 0.0;
}

// x_i[d] = sum_m Phi[d][m] e_i[m]
template <typename PHI>
__global__ void k_rom_prolong(const PHI* __restrict__ phi, const double* __restrict__ e, int n, int kp, int nslots,
                              double* __restrict__ x) {
    const long long total = (long long)nslots * n;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / n);
        const long long d = t - (long long)i * n;
        double v = 0.0;
        for (int m = 0; m < kp; ++m) v = fma((double)phi[d * kp + m], e[(long long)i * kp + m], v);
        x[t] = v;
    }
}

}  // namespace

static int rom_group(pod2g_ctx* c, int nslots, const int* slots, const double* b_dev, double* x_dev) {
    const int n = c->n, kp = c->kp, T = POD2G_THREADS;
    // scratch in the set-up buffer W ([n][kp] doubles): partials [nslots][G][kp],
    // then e [nslots][kp], then the slot list
    const long long cap_rows = (long long)n / nslots - 2;
    const int G = (int)std::max(1LL, std::min({(long long)2 * c->num_sms, cap_rows, (long long)ceil_div(n, T)}));
    double* partial = c->d_W;
    double* e = c->d_W + (size_t)nslots * G * kp;
    int* dsl = reinterpret_cast<int*>(e + (size_t)nslots * kp);
    P2G_CUDA(cudaMemcpyAsync(dsl, slots, sizeof(int) * nslots, cudaMemcpyHostToDevice, c->stream));
    dim3 gr(G, nslots);
    const size_t sm = sizeof(double) * T;
    const int gp = std::max(1, std::min(ceil_div((long long)nslots * n, T), 8 * c->num_sms));
    if (c->precision == POD2G_FP64) {
        k_rom_restrict<double><<<gr, T, sm, c->stream>>>(c->d_phi64, b_dev, n, kp, partial);
        P2G_TRY(pod2g_check_launch(c));
        k_rom_solve<<<nslots, 64, 0, c->stream>>>(partial, G, c->k, kp, dsl, c->d_Lc, e);
        P2G_TRY(pod2g_check_launch(c));
        k_rom_prolong<double><<<gp, T, 0, c->stream>>>(c->d_phi64, e, n, kp, nslots, x_dev);
    } else {
        k_rom_restrict<float><<<gr, T, sm, c->stream>>>(c->d_phi32, b_dev, n, kp, partial);
        P2G_TRY(pod2g_check_launch(c));
        k_rom_solve<<<nslots, 64, 0, c->stream>>>(partial, G, c->k, kp, dsl, c->d_Lc, e);
        P2G_TRY(pod2g_check_launch(c));
        k_rom_prolong<float><<<gp, T, 0, c->stream>>>(c->d_phi32, e, n, kp, nslots, x_dev);
    }
    return pod2g_check_launch(c);
}

int rom_solution(pod2g_ctx* c, int nslots, const int* slots, const double* b_dev, double* x_dev) {
    const int n = c->n;
    if (c->k == 0) {
        P2G_CUDA(cudaMemsetAsync(x_dev, 0, sizeof(double) * (size_t)nslots * n, c->stream));
    } else {
        // as many slots per group as the scratch holds (at least one: W has n*kp >= 2*kp + 1 doubles
        // for n >= 3; smaller systems go one slot at a time with one chunk)
        const int per = std::max(1, std::min(nslots, n / 3));
        for (int i0 = 0; i0 < nslots; i0 += per) {
            const int m = std::min(per, nslots - i0);
            P2G_TRY(rom_group(c, m, slots + i0, b_dev + (size_t)i0 * n, x_dev + (size_t)i0 * n));
        }
    }
    P2G_CUDA(cudaStreamSynchronize(c->stream));
    return POD2G_OK;
}
