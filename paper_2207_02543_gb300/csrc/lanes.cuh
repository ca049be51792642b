// Per-slot reductions shared by the batched kernels (slot-interleaved layout: thread t
// of a CTA works for slot t % Bp, Bp a power of two dividing the CTA size). Every sum
// is taken in a fixed order, so a slot's result does not depend on the other slots.
#pragma once

#include "common.cuh"

namespace {

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

// Per-slot CTA sum: thread t contributes v to slot t % Bp; the sums (in thread
// order) land in s_out[slot]. Ends with a barrier.
__device__ __forceinline__ void cta_lane_sum(double v, int Bp, double* s_tmp, double* s_out) {
    __syncthreads();
    s_tmp[threadIdx.x] = v;
    __syncthreads();
    if ((int)threadIdx.x < Bp) {
        double s = 0.0;
        for (int t = threadIdx.x; t < (int)blockDim.x; t += Bp) s += s_tmp[t];
        s_out[threadIdx.x] = s;
    }
    __syncthreads();
}

// total over partial rows g = 0..NP-1 of part[g * stride + slot] (fixed order),
// computed by all threads of one CTA; the total is returned in threads t < Bp.
__device__ __forceinline__ double grid_lane_total(const double* part, int NP, int stride, int Bp, double* s_tmp) {
    const int Q = blockDim.x / Bp;
    const int b = threadIdx.x % Bp, q = threadIdx.x / Bp;
    const int g0 = (int)((long long)NP * q / Q), g1 = (int)((long long)NP * (q + 1) / Q);
    double s = ordered_sum(part + b, g0, g1, stride);
    __syncthreads();
    s_tmp[threadIdx.x] = s;
    __syncthreads();
    double tot = 0.0;
    if ((int)threadIdx.x < Bp)
        for (int qq = 0; qq < Q; ++qq) tot += s_tmp[qq * Bp + threadIdx.x];
    return tot;
}

__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 df_of(float a) { return make_float2(a, 0.f); }

}  // namespace
