// C ABI of the POD-2G-PCG library (declared in include/pod2g.h): context
// creation and device memory, per-instance set-up, solves, and the serving worker
// that admits requests into free slots of the running batch (continuous batching).
#include "common.cuh"

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

static thread_local cudaError_t g_last_cuda = cudaSuccess;
void pod2g_set_last_cuda_error(cudaError_t e) { g_last_cuda = e; }

void pod2g_trace(const char* file, int line, int status) {
    static const bool on = getenv("POD2G_DEBUG") != nullptr;
    if (on)
        fprintf(stderr, "pod2g: %s:%d -> status %d (%s)\n", file, line, status,
                status == POD2G_CUDA_ERROR ? cudaGetErrorString(g_last_cuda) : "");
}

int pod2g_check_launch(pod2g_ctx* c) {
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_last_cuda = e;
        return POD2G_CUDA_ERROR;
    }
    return POD2G_OK;
}

int dev_alloc(pod2g_ctx* c, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return POD2G_OK;
    bytes = (bytes + 255) & ~(size_t)255;
    if (c->hbm_budget && c->allocated + bytes > c->hbm_budget) return POD2G_ADMISSION;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return POD2G_OOM;
    }
    c->allocated += bytes;
    return POD2G_OK;
}

// FP64 -> nearest BF16 (round to nearest even on the FP64 significand), as FP32.
static float round_bf16(double v) {
    uint64_t u;
    std::memcpy(&u, &v, 8);
    if (((u >> 52) & 0x7ff) == 0x7ff) return (float)v;
    uint64_t r = u + 0x00001FFFFFFFFFFFull + ((u >> 45) & 1ull);
    r &= ~0x00001FFFFFFFFFFFull;
    double d;
    std::memcpy(&d, &r, 8);
    return (float)d;
}

static int pick_kp(int k) {
    const int list[] = {0, 8, 16, 24, 32, 40, 48, 64};
    for (int v : list)
        if (v >= k) return v;
    return -1;
}

int allow_max_smem(const void* fn) {
    int dev = 0, mx = 0;
    P2G_CUDA(cudaGetDevice(&dev));
    P2G_CUDA(cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    P2G_CUDA(cudaFuncGetAttributes(&fa, fn));
    P2G_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - (int)fa.sharedSizeBytes));
    return POD2G_OK;
}

extern "C" {

void pod2g_default_opts(pod2g_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->omega = 2.0 / 3.0;
    o->pre = 1;
    o->post = 1;
    o->precision = POD2G_MIXED_FP32PHI;
    o->beta_pr = 0;
    o->max_batch = 1;
    o->hbm_budget = 0;
    o->spin_limit = 0;
    o->chunk = 8;
    o->stream = nullptr;
    o->method = POD2G_PCG;
    o->coarse = POD2G_COARSE_TENSOR;
}

const char* pod2g_strerror(int s) {
    switch (s) {
        case POD2G_OK: return "ok";
        case POD2G_NOT_CONVERGED: return "not converged (maxit reached)";
        case POD2G_BREAKDOWN: return "breakdown (p^T K p <= 0 or r^T s <= 0)";
        case POD2G_NOT_SPD: return "not SPD (coarse matrix or diagonal)";
        case POD2G_INVALID_ARG: return "invalid argument";
        case POD2G_ADMISSION: return "admission refused (HBM budget or queue full)";
        case POD2G_OOM: return "device out of memory";
        case POD2G_CUDA_ERROR: return g_last_cuda != cudaSuccess ? cudaGetErrorString(g_last_cuda) : "CUDA error";
        case POD2G_TIMEOUT: return "timeout";
        case POD2G_NONFINITE: return "non-finite value";
        case POD2G_PENDING: return "pending";
        case POD2G_TOO_LARGE: return "size exceeds the fixed scratch capacity of pod2g_solve_noalloc";
        default: return "unknown status";
    }
}

static void free_all(pod2g_ctx* c) {
    void* ptrs[] = {c->d_row_ptr, c->d_col_idx, c->d_diag_blk, c->d_phi64, c->d_phi32, c->d_Lc,
                    c->d_setup_status, c->d_stage, c->d_stage32, c->d_W, c->d_ac_part, c->d_Ac, c->d_counters,
                    c->d_vals64, c->d_dinv64, c->d_x64, c->d_r64, c->d_s64, c->d_p64, c->d_q64, c->d_y64, c->d_t64,
                    c->d_w64, c->d_c64, c->d_part64, c->d_scal64, c->d_vals32, c->d_dinv32, c->d_xdf, c->d_rdf,
                    c->d_pdf, c->d_qdf, c->d_bdf, c->d_b64, c->d_s32, c->d_y32, c->d_W32, c->d_ec, c->d_part, c->d_cpart, c->d_sc,
                    c->d_mask, c->d_iob, c->d_iox, c->d_err, c->d_desc, c->d_rowel, c->d_kref32, c->d_coef32, c->d_cnodes, c->d_colour, c->d_modes, c->d_theta};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->h_scal64) cudaFreeHost(c->h_scal64);
    if (c->h_sc) cudaFreeHost(c->h_sc);
    if (c->h_err) cudaFreeHost(c->h_err);
    if (c->h_sc2) cudaFreeHost(c->h_sc2);
    if (c->h_err2) cudaFreeHost(c->h_err2);
    for (auto ev : c->la_ev)
        if (ev) cudaEventDestroy(ev);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    for (auto ev : c->tev) cudaEventDestroy(ev);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

void pod2g_destroy(pod2g_ctx* c) {
    if (!c) return;
    pod2g_serve_stop(c);
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

#define ALLOC(ptr, bytes)                                                      \
    do {                                                                       \
        int s_ = dev_alloc(c, (void**)&(ptr), (bytes));                        \
        if (s_ != POD2G_OK) { free_all(c); delete c; return s_; }              \
    } while (0)

}  // extern "C"

// Host tables of the element-factored operator (see ElemOp): per block row its
// adjacent elements in ascending index, per stored block its descriptor, and the
// FP32 reference sub-blocks. Returns INVALID_ARG for a description the solver
// cannot represent.
static int build_element_tables(const pod2g_pattern* pat, const pod2g_elements* el, std::vector<int32_t>& rowel,
                                std::vector<uint64_t>& desc, std::vector<float>& kref) {
    const int nb = pat->n_brows, bs = pat->bs, npe = el->npe;
    if (el->n_elems < 1 || npe < 2 || npe > 8 || npe * bs > 24 || !el->conn || !el->k_ref) return POD2G_INVALID_ARG;
    const int nk = npe * bs;
    double kmax = 0.0;
    for (int t = 0; t < nk * nk; ++t) {
        if (!std::isfinite(el->k_ref[t])) return POD2G_NONFINITE;
        kmax = std::max(kmax, std::fabs(el->k_ref[t]));
    }
    for (int r = 0; r < nk; ++r)
        for (int q = 0; q < r; ++q)
            if (std::fabs(el->k_ref[r * nk + q] - el->k_ref[q * nk + r]) > 1e-12 * kmax) return POD2G_INVALID_ARG;
    rowel.assign((size_t)nb * POD2G_ELEM_RE, -1);
    std::vector<int> cnt(nb, 0);
    for (int e = 0; e < el->n_elems; ++e) {
        const int32_t* cn = el->conn + (size_t)e * npe;
        for (int a = 0; a < npe; ++a) {
            const int i = cn[a];
            if (i < -1 || i >= nb) return POD2G_INVALID_ARG;
            if (i < 0) continue;
            for (int b = 0; b < a; ++b)
                if (cn[b] == i) return POD2G_INVALID_ARG;  // a node listed twice
            if (cnt[i] >= POD2G_ELEM_RE) return POD2G_INVALID_ARG;
            rowel[(size_t)i * POD2G_ELEM_RE + cnt[i]++] = e;  // e ascends: lists are sorted
        }
    }
    const int64_t nnzb = pat->row_ptr[nb];
    desc.assign((size_t)nnzb, 0ull);
    for (int i = 0; i < nb; ++i) {
        const int32_t* cols = pat->col_idx + pat->row_ptr[i];
        const int ncol = pat->row_ptr[i + 1] - pat->row_ptr[i];
        for (int p = 0; p < cnt[i]; ++p) {
            const int e = rowel[(size_t)i * POD2G_ELEM_RE + p];
            const int32_t* cn = el->conn + (size_t)e * npe;
            int a = 0;
            while (cn[a] != i) ++a;
            for (int b = 0; b < npe; ++b) {
                const int j = cn[b];
                if (j < 0) continue;
                const int32_t* hit = std::lower_bound(cols, cols + ncol, j);
                if (hit == cols + ncol || *hit != j) return POD2G_INVALID_ARG;  // coupling without a stored block
                uint64_t& d = desc[(size_t)(pat->row_ptr[i] + (hit - cols))];
                d |= (1ull << (48 + p)) | ((uint64_t)(a * npe + b) << (6 * p));
            }
        }
    }
    if (el->fixed) {
        for (int i = 0; i < nb; ++i)
            for (int t = pat->row_ptr[i]; t < pat->row_ptr[i + 1]; ++t) {
                const int j = pat->col_idx[t];
                if (el->fixed[i] || el->fixed[j]) desc[t] = (i == j && el->fixed[i]) ? (1ull << 63) : (1ull << 62);
            }
    }
    kref.assign((size_t)npe * npe * bs * bs, 0.f);
    for (int a = 0; a < npe; ++a)
        for (int b = 0; b < npe; ++b)
            for (int r = 0; r < bs; ++r)
                for (int q = 0; q < bs; ++q)
                    kref[((size_t)(a * npe + b) * bs + r) * bs + q] = (float)el->k_ref[(a * bs + r) * nk + b * bs + q];
    return POD2G_OK;
}

static int create_impl(const pod2g_pattern* pat, const pod2g_elements* el, const double* phi, int k,
                       const pod2g_opts* opts_in, pod2g_t* out) {
    if (!out) return POD2G_INVALID_ARG;
    *out = nullptr;
    pod2g_opts o;
    if (opts_in) o = *opts_in; else pod2g_default_opts(&o);
    if (!pat || !pat->row_ptr || !pat->col_idx || pat->n_brows <= 0 || pat->bs < 1 || pat->bs > 3)
        return POD2G_INVALID_ARG;
    if (k < 0 || k > POD2G_MAX_K || (k > 0 && !phi)) return POD2G_INVALID_ARG;
    if (o.precision < 0 || o.precision > 2 || o.max_batch < 1 || o.max_batch > POD2G_MAX_BP) return POD2G_INVALID_ARG;
    if (!(o.omega > 0.0) || o.pre < 0 || o.post < 0 || o.pre > 8 || o.post > 8) return POD2G_INVALID_ARG;
    if (o.precision != POD2G_FP64 && (o.pre > 1 || o.post > 1)) return POD2G_INVALID_ARG;
    if (o.method != POD2G_PCG && o.method != POD2G_STATIONARY) return POD2G_INVALID_ARG;
    if (o.smoother != POD2G_SMOOTHER_JACOBI && o.smoother != POD2G_SMOOTHER_SGS) return POD2G_INVALID_ARG;
    if (o.smoother == POD2G_SMOOTHER_SGS && o.precision != POD2G_FP64 && o.beta_pr) return POD2G_INVALID_ARG;
    if (o.coarse != POD2G_COARSE_DF && o.coarse != POD2G_COARSE_TENSOR) return POD2G_INVALID_ARG;
    if (o.chunk <= 0) o.chunk = 8;
    // pattern checks: monotone row_ptr, columns in range and sorted, diagonal present
    const int nb = pat->n_brows;
    if (pat->row_ptr[0] != 0) return POD2G_INVALID_ARG;
    std::vector<int32_t> diag(nb, -1);
    for (int i = 0; i < nb; ++i) {
        int a = pat->row_ptr[i], b = pat->row_ptr[i + 1];
        if (b < a) return POD2G_INVALID_ARG;
        for (int t = a; t < b; ++t) {
            int j = pat->col_idx[t];
            if (j < 0 || j >= nb) return POD2G_INVALID_ARG;
            if (t > a && j <= pat->col_idx[t - 1]) return POD2G_INVALID_ARG;
            if (j == i) diag[i] = t;
        }
        if (diag[i] < 0) return POD2G_INVALID_ARG;
    }
    const int bs = pat->bs;
    const long long n = (long long)nb * bs;
    const long long nnzb = pat->row_ptr[nb];
    if (k > 0) {
        for (long long e = 0; e < n * k; ++e)
            if (!std::isfinite(phi[e])) return POD2G_NONFINITE;
    }
    std::vector<int32_t> h_rowel;
    std::vector<uint64_t> h_desc;
    std::vector<float> h_kref;
    if (el) {
        if (o.precision == POD2G_FP64) return POD2G_INVALID_ARG;
        int st = build_element_tables(pat, el, h_rowel, h_desc, h_kref);
        if (st != POD2G_OK) return st;
    }

    pod2g_ctx* c = new pod2g_ctx();
    cudaGetDevice(&c->device);
    c->nb = nb; c->bs = bs; c->n = (int)n; c->nnzb = (int)nnzb; c->k = k; c->kp = pick_kp(k);
    c->precision = o.precision; c->pre = o.pre; c->post = o.post; c->beta_pr = o.beta_pr ? 1 : 0;
    c->B = o.max_batch; c->omega = o.omega; c->hbm_budget = o.hbm_budget; c->spin_limit = o.spin_limit;
    c->chunk = o.chunk;
    c->method = o.method;
    c->smoother = o.smoother;
    c->coarse_tc = o.precision != POD2G_FP64 && o.coarse == POD2G_COARSE_TENSOR;
    std::vector<int32_t> h_cnodes;
    std::vector<uint8_t> h_colour;
    if (c->smoother == POD2G_SMOOTHER_SGS) {
        // greedy colouring in node order: smallest colour held by no lower-index neighbour
        std::vector<int> col(nb, -1);
        int ncol = 0;
        for (int i = 0; i < nb; ++i) {
            std::vector<char> taken(ncol + 1, 0);
            for (int t = pat->row_ptr[i]; t < pat->row_ptr[i + 1]; ++t) {
                const int j = pat->col_idx[t];
                if (j < i) taken[col[j]] = 1;
            }
            int cc = 0;
            while (taken[cc]) ++cc;
            col[i] = cc;
            ncol = std::max(ncol, cc + 1);
        }
        if (ncol > 255) { delete c; return POD2G_INVALID_ARG; }
        c->ncolours = ncol;
        c->coff.assign(ncol + 1, 0);
        for (int i = 0; i < nb; ++i) c->coff[col[i] + 1]++;
        for (int q = 0; q < ncol; ++q) c->coff[q + 1] += c->coff[q];
        h_cnodes.resize(nb);
        std::vector<int> fill(c->coff.begin(), c->coff.end() - 1);
        for (int i = 0; i < nb; ++i) h_cnodes[fill[col[i]]++] = i;
        h_colour.assign(col.begin(), col.end());
    }
    if (el) {
        c->elem = 1;
        c->n_el = el->n_elems;
        c->npe = el->npe;
    }
    int Bp = 1;
    while (Bp < o.max_batch) Bp <<= 1;
    c->Bp = c->precision == POD2G_FP64 ? 1 : Bp;
    if (o.stream) {
        c->stream = (cudaStream_t)o.stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return POD2G_CUDA_ERROR; }
        c->own_stream = true;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    c->num_sms = sms > 0 ? sms : 152;
    const int kp = c->kp;
    const long long tot = nnzb * bs * bs;
    const int Gmax = 4 * c->num_sms;

    ALLOC(c->d_row_ptr, sizeof(int32_t) * (nb + 1));
    ALLOC(c->d_col_idx, sizeof(int32_t) * nnzb);
    ALLOC(c->d_diag_blk, sizeof(int32_t) * nb);
    ALLOC(c->d_Lc, sizeof(double) * std::max(1, c->B * k * k));
    ALLOC(c->d_setup_status, sizeof(int) * c->B);
    ALLOC(c->d_stage, sizeof(double) * std::max(tot, (long long)c->n_el));
    ALLOC(c->d_W, sizeof(double) * (std::max(3LL, n) * std::max(kp, 1) + 64));
    ALLOC(c->d_ac_part, sizeof(double) * std::max(1, 2 * c->num_sms * k * k));
    ALLOC(c->d_Ac, sizeof(double) * std::max(1, k * k));
    ALLOC(c->d_counters, sizeof(unsigned) * CNT_N);
    if (c->smoother == POD2G_SMOOTHER_SGS) {
        ALLOC(c->d_cnodes, sizeof(int32_t) * nb);
        ALLOC(c->d_colour, sizeof(uint8_t) * nb);
    }
    ALLOC(c->d_iob, sizeof(double) * n * c->B);
    ALLOC(c->d_iox, sizeof(double) * n * c->B);
    if (c->precision == POD2G_FP64) {
        ALLOC(c->d_phi64, sizeof(double) * std::max(1LL, n * kp));
        ALLOC(c->d_vals64, sizeof(double) * tot * c->B);
        ALLOC(c->d_dinv64, sizeof(double) * n * c->B);
        double** vecs[] = {&c->d_x64, &c->d_r64, &c->d_s64, &c->d_p64, &c->d_q64, &c->d_y64, &c->d_t64, &c->d_w64};
        for (double** v : vecs) ALLOC(*v, sizeof(double) * n);
        ALLOC(c->d_c64, sizeof(double) * std::max(1, kp));
        ALLOC(c->d_part64, sizeof(double) * (size_t)Gmax * (kp + 8));
        ALLOC(c->d_scal64, sizeof(double) * 16);
        if (cudaMallocHost(&c->h_scal64, sizeof(double) * 16) != cudaSuccess) { free_all(c); delete c; return POD2G_OOM; }
    } else {
        ALLOC(c->d_phi32, sizeof(float) * std::max(1LL, n * kp));
        ALLOC(c->d_stage32, sizeof(float) * tot);
        if (c->elem) {
            ALLOC(c->d_desc, sizeof(uint64_t) * nnzb);
            ALLOC(c->d_rowel, sizeof(int32_t) * nb * POD2G_ELEM_RE);
            ALLOC(c->d_kref32, sizeof(float) * h_kref.size());
            ALLOC(c->d_coef32, sizeof(float) * (size_t)c->n_el * Bp);
        } else {
            ALLOC(c->d_vals32, sizeof(float) * tot * Bp);
        }
        ALLOC(c->d_dinv32, sizeof(float) * n * Bp);
        ALLOC(c->d_xdf, sizeof(float2) * n * Bp);
        ALLOC(c->d_rdf, sizeof(float2) * n * Bp);
        ALLOC(c->d_pdf, sizeof(float2) * n * Bp);
        ALLOC(c->d_qdf, sizeof(float2) * n * Bp);
        ALLOC(c->d_bdf, sizeof(float2) * n * Bp);
        ALLOC(c->d_b64, sizeof(double) * n * Bp);
        ALLOC(c->d_s32, sizeof(float) * n * Bp);
        ALLOC(c->d_y32, sizeof(float) * n * Bp);
        // K Phi per slot, for the post-smoothing without a matrix sweep (k_postw and the persistent
        // launch), when it is smaller than the slot's matrix values or the problem is small enough for
        // the persistent launch, and it fits the budget; otherwise the context does without it
        if (!c->elem && c->smoother == POD2G_SMOOTHER_JACOBI && c->pre == 1 && c->post == 1 && kp > 0 &&
            ((long long)n * kp < tot || (long long)n * Bp <= POD2G_PERSIST_ITEMS)) {
            if (dev_alloc(c, (void**)&c->d_W32, sizeof(float) * n * kp * Bp) != POD2G_OK) c->d_W32 = nullptr;
        }
        ALLOC(c->d_ec, sizeof(float) * std::max(1, Bp * kp));
        ALLOC(c->d_part, sizeof(double) * (Gmax + 1) * Bp * 2);   // + the persistent launch's totals
        ALLOC(c->d_cpart, sizeof(double) * (size_t)Gmax * Bp * std::max(1, kp));
        ALLOC(c->d_sc, sizeof(SlotScalars) * Bp);
        ALLOC(c->d_mask, sizeof(int) * 2 * Bp);
        ALLOC(c->d_err, sizeof(int));
        if (cudaMallocHost(&c->h_err, sizeof(int)) != cudaSuccess) { free_all(c); delete c; return POD2G_OOM; }
        *c->h_err = 0;
        if (cudaMallocHost(&c->h_sc, sizeof(SlotScalars) * Bp) != cudaSuccess) { free_all(c); delete c; return POD2G_OOM; }
        std::memset(c->h_sc, 0, sizeof(SlotScalars) * Bp);
        if (cudaMallocHost(&c->h_sc2, sizeof(SlotScalars) * Bp) != cudaSuccess ||
            cudaMallocHost(&c->h_err2, sizeof(int)) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->la_ev[0], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->la_ev[1], cudaEventDisableTiming) != cudaSuccess) {
            free_all(c);
            delete c;
            return POD2G_OOM;
        }
        std::memset(c->h_sc2, 0, sizeof(SlotScalars) * Bp);
        *c->h_err2 = 0;
        if (batched_alloc(c) != POD2G_OK) { free_all(c); delete c; return POD2G_INVALID_ARG; }
        if (c->coarse_tc && c->k > 0 && setup_tc_attributes(c) != POD2G_OK) {
            free_all(c);
            delete c;
            return POD2G_CUDA_ERROR;
        }
    }
    c->setup_ok.assign(c->B, 0);
    // uploads (synchronous, once)
    auto up = [&](void* dst, const void* src, size_t bytes) {
        return cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    bool ok = up(c->d_row_ptr, pat->row_ptr, sizeof(int32_t) * (nb + 1)) &&
              up(c->d_col_idx, pat->col_idx, sizeof(int32_t) * nnzb) &&
              up(c->d_diag_blk, diag.data(), sizeof(int32_t) * nb) &&
              cudaMemset(c->d_counters, 0, sizeof(unsigned) * CNT_N) == cudaSuccess;
    if (ok && kp > 0) {
        if (c->precision == POD2G_FP64) {
            std::vector<double> h(n * kp, 0.0);
            for (long long d = 0; d < n; ++d)
                for (int m = 0; m < k; ++m) h[d * kp + m] = phi[(long long)m * n + d];
            ok = up(c->d_phi64, h.data(), sizeof(double) * n * kp);
        } else {
            std::vector<float> h(n * kp, 0.f);
            for (long long d = 0; d < n; ++d)
                for (int m = 0; m < k; ++m) {
                    double v = phi[(long long)m * n + d];
                    h[d * kp + m] = c->precision == POD2G_MIXED_BF16PHI ? round_bf16(v) : (float)v;
                }
            ok = up(c->d_phi32, h.data(), sizeof(float) * n * kp);
        }
    }
    if (ok && c->smoother == POD2G_SMOOTHER_SGS) {
        ok = up(c->d_cnodes, h_cnodes.data(), sizeof(int32_t) * nb) &&
             up(c->d_colour, h_colour.data(), sizeof(uint8_t) * nb);
    }
    if (ok && c->elem) {
        ok = up(c->d_desc, h_desc.data(), sizeof(uint64_t) * nnzb) &&
             up(c->d_rowel, h_rowel.data(), sizeof(int32_t) * nb * POD2G_ELEM_RE) &&
             up(c->d_kref32, h_kref.data(), sizeof(float) * h_kref.size()) &&
             cudaMemset(c->d_coef32, 0, sizeof(float) * (size_t)c->n_el * Bp) == cudaSuccess;
    }
    if (ok && c->precision != POD2G_FP64) {
        ok = cudaMemset(c->d_sc, 0, sizeof(SlotScalars) * Bp) == cudaSuccess &&
             cudaMemset(c->d_err, 0, sizeof(int)) == cudaSuccess &&
             (c->elem || cudaMemset(c->d_vals32, 0, sizeof(float) * tot * Bp) == cudaSuccess) &&
             cudaMemset(c->d_dinv32, 0, sizeof(float) * n * Bp) == cudaSuccess &&
             cudaMemset(c->d_xdf, 0, sizeof(float2) * n * Bp) == cudaSuccess &&
             cudaMemset(c->d_rdf, 0, sizeof(float2) * n * Bp) == cudaSuccess &&
             cudaMemset(c->d_pdf, 0, sizeof(float2) * n * Bp) == cudaSuccess &&
             cudaMemset(c->d_qdf, 0, sizeof(float2) * n * Bp) == cudaSuccess &&
             cudaMemset(c->d_bdf, 0, sizeof(float2) * n * Bp) == cudaSuccess &&
             cudaMemset(c->d_b64, 0, sizeof(double) * n * Bp) == cudaSuccess &&
             cudaMemset(c->d_s32, 0, sizeof(float) * n * Bp) == cudaSuccess &&
             cudaMemset(c->d_y32, 0, sizeof(float) * n * Bp) == cudaSuccess;
    }
    if (!ok) {
        g_last_cuda = cudaGetLastError();
        free_all(c);
        delete c;
        return POD2G_CUDA_ERROR;
    }
    *out = c;
    return POD2G_OK;
}

extern "C" {

int pod2g_create(const pod2g_pattern* pat, const double* phi, int k, const pod2g_opts* opts, pod2g_t* out) {
    return create_impl(pat, nullptr, phi, k, opts, out);
}

int pod2g_create_elements(const pod2g_pattern* pat, const pod2g_elements* el, const double* phi, int k,
                          const pod2g_opts* opts, pod2g_t* out) {
    if (out) *out = nullptr;
    if (!el) return POD2G_INVALID_ARG;
    return create_impl(pat, el, phi, k, opts, out);
}

int pod2g_info(pod2g_t c, int* n, int* nnzb, int* k, int* max_batch) {
    if (!c) return POD2G_INVALID_ARG;
    if (n) *n = c->n;
    if (nnzb) *nnzb = c->nnzb;
    if (k) *k = c->k;
    if (max_batch) *max_batch = c->B;
    return POD2G_OK;
}

int64_t pod2g_launch_count(pod2g_t c) { return c ? (int64_t)c->launches : 0; }

int64_t pod2g_device_bytes(pod2g_t c) { return c ? (int64_t)c->allocated : 0; }

int pod2g_coarse_factor(pod2g_t c, int slot, double* L) {
    if (!c || !L || slot < 0 || slot >= c->B) return POD2G_INVALID_ARG;
    if (!c->setup_ok[slot]) return POD2G_INVALID_ARG;
    if (c->k == 0) return POD2G_OK;
    P2G_CUDA(cudaMemcpyAsync(L, c->d_Lc + (size_t)slot * c->k * c->k, sizeof(double) * c->k * c->k,
                             cudaMemcpyDeviceToHost, c->stream));
    P2G_CUDA(cudaStreamSynchronize(c->stream));
    return POD2G_OK;
}

int pod2g_kernel_timing(pod2g_t c, int on) {
    if (!c || c->serving) return POD2G_INVALID_ARG;
    return batched_set_timing(c, on);
}

static int check_slots(pod2g_ctx* c, int nslots, const int* slots);

int pod2g_get_tuning(pod2g_t c, pod2g_tuning* out) {
    if (!c || !out || c->precision == POD2G_FP64) return POD2G_INVALID_ARG;
    out->grid_rows = c->grid_rows;
    out->grid_restrict = c->grid_restrict;
    out->grid_prol = c->grid_prol;
    out->grid_vec = c->grid_vec;
    out->grid_spmv = c->grid_spmv;
    out->rows_kernel = c->rows_kernel;
    out->restrict_rows = c->restrict_rows;
    out->grid_persist = c->grid_persist;
    return POD2G_OK;
}

int pod2g_set_tuning(pod2g_t c, const pod2g_tuning* t) {
    if (!c || !t || c->precision == POD2G_FP64 || c->serving) return POD2G_INVALID_ARG;
    return batched_set_tuning(c, t);
}

int pod2g_autotune(pod2g_t c, int nslots, const int* slots, const double* b_dev, int iters, pod2g_tuning* out) {
    if (!c || !b_dev || iters < 1 || c->precision == POD2G_FP64 || c->serving) return POD2G_INVALID_ARG;
    P2G_TRY(check_slots(c, nslots, slots));
    P2G_TRY(batched_autotune(c, nslots, slots, b_dev, iters));
    return out ? pod2g_get_tuning(c, out) : POD2G_OK;
}

int pod2g_kernel_times(pod2g_t c, double* ms, int64_t* launches) {
    if (!c) return POD2G_INVALID_ARG;
    for (int j = 0; j < 8; ++j) {
        if (ms) ms[j] = c->kt_ms[j];
        if (launches) launches[j] = c->kt_n[j];
    }
    return POD2G_OK;
}

static int finish_setup(pod2g_ctx* c, int nslots, const int* slots, int* status) {
    std::vector<int> st(c->B, 0);
    cudaError_t e = cudaMemcpyAsync(st.data(), c->d_setup_status, sizeof(int) * c->B, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) { g_last_cuda = e; return POD2G_CUDA_ERROR; }
    int first = POD2G_OK;
    for (int i = 0; i < nslots; ++i) {
        int s = st[slots[i]];
        c->setup_ok[slots[i]] = (s == POD2G_OK);
        if (status) status[i] = s;
        if (s != POD2G_OK && first == POD2G_OK) first = s;
    }
    return first;
}

int pod2g_set_values(pod2g_t c, int slot, const double* values, int on_device) {
    if (!c || !values || slot < 0 || slot >= c->B) return POD2G_INVALID_ARG;
    if (c->serving || c->elem) return POD2G_INVALID_ARG;
    const size_t bytes = sizeof(double) * (size_t)c->nnzb * c->bs * c->bs;
    const double* src = values;
    if (!on_device) {
        P2G_CUDA(cudaMemcpyAsync(c->d_stage, values, bytes, cudaMemcpyHostToDevice, c->stream));
        src = c->d_stage;
    }
    c->setup_ok[slot] = 0;
    P2G_TRY(setup_values(c, slot, src));
    return finish_setup(c, 1, &slot, nullptr);
}

int pod2g_set_coeffs(pod2g_t c, int slot, const double* coeffs, int on_device) {
    if (!c || !coeffs || slot < 0 || slot >= c->B) return POD2G_INVALID_ARG;
    if (c->serving || !c->elem) return POD2G_INVALID_ARG;
    const double* src = coeffs;
    if (!on_device) {
        P2G_CUDA(cudaMemcpyAsync(c->d_stage, coeffs, sizeof(double) * c->n_el, cudaMemcpyHostToDevice, c->stream));
        src = c->d_stage;
    }
    c->setup_ok[slot] = 0;
    P2G_TRY(setup_coeffs(c, slot, src));
    return finish_setup(c, 1, &slot, nullptr);
}

int pod2g_set_coeffs_batch_dev(pod2g_t c, int nslots, const int* slots, const double* coeffs_dev, int* status) {
    if (!c || !slots || !coeffs_dev || nslots < 1 || nslots > c->B) return POD2G_INVALID_ARG;
    if (c->serving || !c->elem) return POD2G_INVALID_ARG;
    for (int i = 0; i < nslots; ++i) {
        if (slots[i] < 0 || slots[i] >= c->B) return POD2G_INVALID_ARG;
        c->setup_ok[slots[i]] = 0;
        P2G_TRY(setup_coeffs(c, slots[i], coeffs_dev + (size_t)i * c->n_el));
    }
    return finish_setup(c, nslots, slots, status);
}

int pod2g_set_field(pod2g_t c, const double* modes, int m, double mu, double sigma, int lognormal) {
    if (!c || !modes || !c->elem || c->serving || m < 1 || m > 64) return POD2G_INVALID_ARG;
    if (!std::isfinite(mu) || !std::isfinite(sigma)) return POD2G_NONFINITE;
    for (long long t = 0; t < (long long)c->n_el * m; ++t)
        if (!std::isfinite(modes[t])) return POD2G_NONFINITE;
    if (c->d_modes) {  // replace an earlier field
        cudaStreamSynchronize(c->stream);
        cudaFree(c->d_modes);
        cudaFree(c->d_theta);
        c->d_modes = c->d_theta = nullptr;
        c->allocated -= ((sizeof(double) * (size_t)c->n_el * c->field_m + 255) & ~(size_t)255) +
                        ((sizeof(double) * (size_t)c->B * c->field_m + 255) & ~(size_t)255);
        c->field_m = 0;
    }
    int st = dev_alloc(c, (void**)&c->d_modes, sizeof(double) * (size_t)c->n_el * m);
    if (st == POD2G_OK) st = dev_alloc(c, (void**)&c->d_theta, sizeof(double) * (size_t)c->B * m);
    if (st != POD2G_OK) {
        if (c->d_modes) {
            cudaFree(c->d_modes);
            c->allocated -= (sizeof(double) * (size_t)c->n_el * m + 255) & ~(size_t)255;
        }
        c->d_modes = nullptr;
        return st;
    }
    P2G_CUDA(cudaMemcpy(c->d_modes, modes, sizeof(double) * (size_t)c->n_el * m, cudaMemcpyHostToDevice));
    c->field_m = m;
    c->field_mu = mu;
    c->field_sigma = sigma;
    c->field_log = lognormal ? 1 : 0;
    return POD2G_OK;
}

int pod2g_set_theta_batch(pod2g_t c, int nslots, const int* slots, const double* theta, int* status) {
    if (!c || !slots || !theta || nslots < 1 || nslots > c->B) return POD2G_INVALID_ARG;
    if (c->serving || !c->elem || c->field_m == 0) return POD2G_INVALID_ARG;
    for (int i = 0; i < nslots; ++i)
        if (slots[i] < 0 || slots[i] >= c->B) return POD2G_INVALID_ARG;
    const int m = c->field_m;
    P2G_CUDA(cudaMemcpyAsync(c->d_theta, theta, sizeof(double) * (size_t)nslots * m, cudaMemcpyHostToDevice,
                             c->stream));
    for (int i = 0; i < nslots; ++i) {
        c->setup_ok[slots[i]] = 0;
        P2G_TRY(setup_theta(c, slots[i], c->d_theta + (size_t)i * m));
    }
    return finish_setup(c, nslots, slots, status);
}

int pod2g_set_theta(pod2g_t c, int slot, const double* theta) {
    int st = POD2G_OK;
    int rc = pod2g_set_theta_batch(c, 1, &slot, theta, &st);
    return rc;
}

int pod2g_set_values_batch_dev(pod2g_t c, int nslots, const int* slots, const double* values_dev, int* status) {
    if (!c || !slots || !values_dev || nslots < 1 || nslots > c->B) return POD2G_INVALID_ARG;
    if (c->serving || c->elem) return POD2G_INVALID_ARG;
    std::vector<char> seen(c->B, 0);
    for (int i = 0; i < nslots; ++i) {
        if (slots[i] < 0 || slots[i] >= c->B || seen[slots[i]]) return POD2G_INVALID_ARG;
        seen[slots[i]] = 1;
        c->setup_ok[slots[i]] = 0;
    }
    P2G_TRY(setup_values_batch(c, nslots, slots, values_dev));
    return finish_setup(c, nslots, slots, status);
}

static int check_slots(pod2g_ctx* c, int nslots, const int* slots) {
    if (nslots < 1 || nslots > c->B || !slots) return POD2G_INVALID_ARG;
    std::vector<char> seen(c->B, 0);
    for (int i = 0; i < nslots; ++i) {
        int s = slots[i];
        if (s < 0 || s >= c->B || seen[s] || !c->setup_ok[s]) {
            if (getenv("POD2G_DEBUG"))
                fprintf(stderr, "pod2g: slot %d (index %d) rejected: B=%d seen=%d setup_ok=%d\n", s, i, c->B,
                        (s >= 0 && s < c->B) ? (int)seen[s] : -1, (s >= 0 && s < c->B) ? c->setup_ok[s] : -1);
            return POD2G_INVALID_ARG;
        }
        seen[s] = 1;
    }
    return POD2G_OK;
}

int pod2g_solve_batch_dev(pod2g_t c, int nslots, const int* slots, const double* b_dev, const double* x0_dev,
                          double tol, int maxit, double* x_dev, int* iters, double* relres, int* status) {
    if (!c || !b_dev || !x_dev || !(tol >= 0.0) || maxit < 0) return POD2G_INVALID_ARG;
    if (c->serving) return POD2G_INVALID_ARG;
    P2G_TRY(check_slots(c, nslots, slots));
    std::vector<int> st(nslots, POD2G_OK);
    if (c->precision == POD2G_FP64) {
        for (int i = 0; i < nslots; ++i) {
            int it = 0;
            double rr = 0.0;
            P2G_TRY(plain_solve(c, slots[i], b_dev + (size_t)i * c->n, x0_dev ? x0_dev + (size_t)i * c->n : nullptr,
                                tol, maxit, x_dev + (size_t)i * c->n, &it, &rr, &st[i]));
            if (iters) iters[i] = it;
            if (relres) relres[i] = rr;
        }
    } else {
        // lane = slot index: slots >= Bp cannot occur (B <= Bp)
        std::vector<double> tols(nslots, tol);
        std::vector<int> maxits(nslots, maxit);
        P2G_TRY(batched_load(c, nslots, slots, b_dev, x0_dev, tols.data(), maxits.data()));
        std::vector<int> lanes(slots, slots + nslots);
        const int rr = batched_run(c, lanes);
        if (rr == POD2G_TIMEOUT) P2G_TRY(batched_retire(c, lanes, POD2G_TIMEOUT));
        else P2G_TRY(rr);
        P2G_TRY(batched_finalize(c, nslots, slots, x_dev, iters, relres, st.data()));
    }
    int first = POD2G_OK;
    for (int i = 0; i < nslots; ++i) {
        if (status) status[i] = st[i];
        if (st[i] != POD2G_OK && first == POD2G_OK) first = st[i];
    }
    return first;
}

int pod2g_rom_solution_dev(pod2g_t c, int nslots, const int* slots, const double* b_dev, double* x_dev) {
    if (!c || !b_dev || !x_dev || c->serving) return POD2G_INVALID_ARG;
    P2G_TRY(check_slots(c, nslots, slots));
    return rom_solution(c, nslots, slots, b_dev, x_dev);
}

int pod2g_solve_batch(pod2g_t c, int nslots, const int* slots, const double* const* b, const double* const* x0,
                      double tol, int maxit, double* const* x, int* iters, double* relres, int* status) {
    if (!c || !b || !x) return POD2G_INVALID_ARG;
    P2G_TRY(check_slots(c, nslots, slots));
    const size_t n = c->n;
    bool any_x0 = false;
    for (int i = 0; i < nslots; ++i) {
        if (!b[i] || !x[i]) return POD2G_INVALID_ARG;
        if (x0 && x0[i]) any_x0 = true;
    }
    for (int i = 0; i < nslots; ++i) {
        P2G_CUDA(cudaMemcpyAsync(c->d_iob + i * n, b[i], sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
        if (any_x0) {
            if (x0[i]) {
                P2G_CUDA(cudaMemcpyAsync(c->d_iox + i * n, x0[i], sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
            } else {
                P2G_CUDA(cudaMemsetAsync(c->d_iox + i * n, 0, sizeof(double) * n, c->stream));
            }
        }
    }
    // x is written into d_iob's rows after b has been consumed: use a separate region
    int rc = pod2g_solve_batch_dev(c, nslots, slots, c->d_iob, any_x0 ? c->d_iox : nullptr, tol, maxit, c->d_iox,
                                   iters, relres, status);
    if (rc == POD2G_INVALID_ARG || rc == POD2G_CUDA_ERROR || rc == POD2G_TIMEOUT) return rc;
    for (int i = 0; i < nslots; ++i)
        P2G_CUDA(cudaMemcpyAsync(x[i], c->d_iox + i * n, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    P2G_CUDA(cudaStreamSynchronize(c->stream));
    return rc;
}

int pod2g_solve(pod2g_t c, int slot, const double* b, const double* x0, double tol, int maxit, double* x, int* iters,
                double* relres) {
    const double* bb[1] = {b};
    const double* xx0[1] = {x0};
    double* xx[1] = {x};
    int st = 0;
    int rc = pod2g_solve_batch(c, 1, &slot, bb, x0 ? xx0 : nullptr, tol, maxit, xx, iters, relres, &st);
    return rc;
}

}  // extern "C"
