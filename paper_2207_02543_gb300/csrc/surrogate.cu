// Surrogate initial guess on the device (arXiv 2207.02543, Section 3.2, online phase):
// u_sur(theta) = s * decoder(FFNN(theta)), where FFNN is a feed-forward network with two
// tanh hidden layers whose output o gives the latent z = z_mean + z_std * o, and the
// decoder is the tall-skinny product u = Psi z with ks POD modes Psi. The solver accepts any
// x0; this object produces one per query from its parameters, in the caller's stream, so that
// "surrogate prediction, then POD-2G-PCG" runs on the device end to end.
//
//   k_sur_ffnn   one CTA per query: the network in FP64 (a few thousand operations), then
//                z * s in FP32 for the decoder
//   k_sur_decode thread per unknown i: x[q][i] = sum_j Psi[j][i] z[q][j] for a tile of QT
//                queries held in registers; Psi (FP32, mode-major [ks][n]) is read once per
//                tile, coalesced across threads; z comes from shared memory (broadcast)
#include "common.cuh"

#define SUR_MAX_M 64
#define SUR_MAX_H 256
#define SUR_MAX_KS 256
#define SUR_QT 16          // queries per decoder pass

struct pod2g_sur {
    long long n = 0;
    int m = 0, ks = 0, H = 0;
    int device = 0, num_sms = 152;
    float* d_psi = nullptr;       // [ks][n]
    double* d_par = nullptr;      // w1 [H][m], b1 [H], w2 [H][H], b2 [H], w3 [ks][H], b3 [ks], z_mean [ks], z_std [ks]
    double* d_in = nullptr;       // [SUR_QT][m + 1]: theta, scale
    float* d_z = nullptr;         // [SUR_QT][ks]
    double* h_in = nullptr;       // pinned staging of d_in
    cudaStream_t stream = nullptr;
    bool own_stream = false;
};

namespace {

__global__ void k_sur_ffnn(const double* __restrict__ par, const double* __restrict__ in, int m, int H, int ks,
                           float* __restrict__ z) {
    __shared__ double h1[SUR_MAX_H], h2[SUR_MAX_H];
    const int q = blockIdx.x;
    const double* th = in + (long long)q * (m + 1);
    const double s = th[m];
    const double* w1 = par;
    const double* b1 = w1 + (long long)H * m;
    const double* w2 = b1 + H;
    const double* b2 = w2 + (long long)H * H;
    const double* w3 = b2 + H;
    const double* b3 = w3 + (long long)ks * H;
    const double* zm = b3 + ks;
    const double* zs = zm + ks;
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        double a = b1[i];
        for (int j = 0; j < m; ++j) a = fma(w1[(long long)i * m + j], th[j], a);
        h1[i] = tanh(a);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        double a = b2[i];
        for (int j = 0; j < H; ++j) a = fma(w2[(long long)i * H + j], h1[j], a);
        h2[i] = tanh(a);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ks; i += blockDim.x) {
        double a = b3[i];
        for (int j = 0; j < H; ++j) a = fma(w3[(long long)i * H + j], h2[j], a);
        z[(long long)q * ks + i] = (float)(s * (zm[i] + zs[i] * a));
    }
}

template <int QT>
__global__ void __launch_bounds__(256) k_sur_decode(const float* __restrict__ psi, const float* __restrict__ z,
                                                    long long n, int ks, int nq, double* __restrict__ x) {
    __shared__ float s_z[SUR_MAX_KS * QT];   // [j][q]
    for (int e = threadIdx.x; e < ks * QT; e += blockDim.x) {
        const int j = e / QT, q = e - j * QT;
        s_z[e] = q < nq ? z[(long long)q * ks + j] : 0.f;
    }
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float acc[QT];
#pragma unroll
        for (int q = 0; q < QT; ++q) acc[q] = 0.f;
        for (int j = 0; j < ks; ++j) {
            const float p = __ldg(psi + (long long)j * n + i);
#pragma unroll
            for (int q = 0; q < QT; ++q) acc[q] = __fmaf_rn(p, s_z[j * QT + q], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < QT; ++q)
            if (q < nq) x[(long long)q * n + i] = (double)acc[q];
    }
}

__global__ void k_sur_psi(const double* __restrict__ psi64, float* __restrict__ psi32, long long total) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x)
        psi32[e] = __double2float_rn(psi64[e]);
}

}  // namespace

static void sur_free(pod2g_sur* s) {
    if (!s) return;
    cudaFree(s->d_psi);
    cudaFree(s->d_par);
    cudaFree(s->d_in);
    cudaFree(s->d_z);
    if (s->h_in) cudaFreeHost(s->h_in);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

int pod2g_surrogate_create(int64_t n, int m, int ks, int hidden, const double* psi, const double* w1,
                           const double* b1, const double* w2, const double* b2, const double* w3, const double* b3,
                           const double* z_mean, const double* z_std, void* stream, pod2g_sur_t* out) {
    if (!out) return POD2G_INVALID_ARG;
    *out = nullptr;
    if (n <= 0 || m < 1 || m > SUR_MAX_M || ks < 1 || ks > SUR_MAX_KS || hidden < 1 || hidden > SUR_MAX_H)
        return POD2G_INVALID_ARG;
    if (!psi || !w1 || !b1 || !w2 || !b2 || !w3 || !b3 || !z_mean || !z_std) return POD2G_INVALID_ARG;
    pod2g_sur* s = new pod2g_sur();
    s->n = n; s->m = m; s->ks = ks; s->H = hidden;
    cudaGetDevice(&s->device);
    cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
    if (stream) {
        s->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) { sur_free(s); return POD2G_CUDA_ERROR; }
        s->own_stream = true;
    }
    const size_t npar = (size_t)hidden * m + hidden + (size_t)hidden * hidden + hidden + (size_t)ks * hidden + 3 * (size_t)ks;
    std::vector<double> par;
    par.reserve(npar);
    par.insert(par.end(), w1, w1 + (size_t)hidden * m);
    par.insert(par.end(), b1, b1 + hidden);
    par.insert(par.end(), w2, w2 + (size_t)hidden * hidden);
    par.insert(par.end(), b2, b2 + hidden);
    par.insert(par.end(), w3, w3 + (size_t)ks * hidden);
    par.insert(par.end(), b3, b3 + ks);
    par.insert(par.end(), z_mean, z_mean + ks);
    par.insert(par.end(), z_std, z_std + ks);
    double* d_psi64 = nullptr;
    bool ok = cudaMalloc(&s->d_psi, sizeof(float) * (size_t)ks * n) == cudaSuccess &&
              cudaMalloc(&s->d_par, sizeof(double) * npar) == cudaSuccess &&
              cudaMalloc(&s->d_in, sizeof(double) * SUR_QT * (m + 1)) == cudaSuccess &&
              cudaMalloc(&s->d_z, sizeof(float) * SUR_QT * ks) == cudaSuccess &&
              cudaMallocHost(&s->h_in, sizeof(double) * SUR_QT * (m + 1)) == cudaSuccess &&
              cudaMalloc(&d_psi64, sizeof(double) * (size_t)n) == cudaSuccess;
    if (!ok) {
        cudaFree(d_psi64);
        sur_free(s);
        return POD2G_OOM;
    }
    ok = cudaMemcpy(s->d_par, par.data(), sizeof(double) * npar, cudaMemcpyHostToDevice) == cudaSuccess;
    // Psi column by column (n x ks column-major on the host = mode-major), rounded to FP32
    for (int j = 0; ok && j < ks; ++j) {
        ok = cudaMemcpy(d_psi64, psi + (size_t)j * n, sizeof(double) * n, cudaMemcpyHostToDevice) == cudaSuccess;
        if (ok) {
            k_sur_psi<<<std::max(1, std::min(ceil_div(n, 256), 8 * s->num_sms)), 256>>>(d_psi64, s->d_psi + (size_t)j * n, n);
            ok = cudaGetLastError() == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess;
        }
    }
    cudaFree(d_psi64);
    if (!ok) {
        sur_free(s);
        return POD2G_CUDA_ERROR;
    }
    *out = s;
    return POD2G_OK;
}

int pod2g_surrogate_predict_dev(pod2g_sur_t s, int nq, const double* theta, const double* scale, double* x_dev) {
    if (!s || nq < 0 || (nq > 0 && (!theta || !x_dev))) return POD2G_INVALID_ARG;
    const int m = s->m;
    for (int q0 = 0; q0 < nq; q0 += SUR_QT) {
        const int cnt = std::min(SUR_QT, nq - q0);
        // the pinned staging buffer is reused: wait for the previous tile's copy
        P2G_CUDA(cudaStreamSynchronize(s->stream));
        for (int q = 0; q < cnt; ++q) {
            for (int j = 0; j < m; ++j) s->h_in[q * (m + 1) + j] = theta[(size_t)(q0 + q) * m + j];
            s->h_in[q * (m + 1) + m] = scale ? scale[q0 + q] : 1.0;
        }
        P2G_CUDA(cudaMemcpyAsync(s->d_in, s->h_in, sizeof(double) * cnt * (m + 1), cudaMemcpyHostToDevice, s->stream));
        k_sur_ffnn<<<cnt, 128, 0, s->stream>>>(s->d_par, s->d_in, m, s->H, s->ks, s->d_z);
        P2G_CUDA(cudaGetLastError());
        const int g = std::max(1, std::min(ceil_div(s->n, 256), 4 * s->num_sms));
        k_sur_decode<SUR_QT><<<g, 256, 0, s->stream>>>(s->d_psi, s->d_z, s->n, s->ks, cnt, x_dev + (size_t)q0 * s->n);
        P2G_CUDA(cudaGetLastError());
    }
    return POD2G_OK;
}

void pod2g_surrogate_destroy(pod2g_sur_t s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    sur_free(s);
}
