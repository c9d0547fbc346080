// flb_kernels.cuh -- lattice kernels: fused pull-stream + collide (+ sampling),
// correlation reduction and finalisation, conservation sums, state I/O.
//
// A buffer holds the post-collision populations f*_i(x, t-1) (layout and ghost
// frame: flb_layout.cuh); the step kernel pulls g_i(x) = f*_i(x - v_i), which is
// the pre-collision state f_i(x, t) of Eq. LBE1, collides it and writes
// f*_i(x, t) to the other buffer.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "flb_collide.cuh"
#include "flb_device.cuh"
#include "flb_layout.cuh"

namespace flb {

constexpr int kSums = 54;          // 9 first moments + 45 unique second moments
constexpr int kStepThreads = 256;

struct DevError {
    int code;        // 0 = none, else kStatus*
    int pad;
    long long node;
    long long step;
};

struct Vec9 {
    double v[9];
};

template <class T>
struct StepArgs {
    const T* src;
    T* dst;
    Geometry geo;
    uint32_t step;
    uint32_t node0;     // noise counter of node (0, 0): Lx y0 for a slab starting at row y0
    double* partials;   // [gridDim.x][kSums] when sampling
    DevError* err;
    const T* lut;       // velocity table (look-up-table f-norm only)
    T ref[9];           // c = f^0(rho0, u0), subtracted before sampling
};

__device__ __forceinline__ void record_error(DevError* err, int code, long long node,
                                             long long step) {
    if (atomicCAS(&err->code, 0, code) == 0) {
        err->node = node;
        err->step = step;
    }
}

// Accumulation type of the per-thread correlation sums: FP32 for the FP32
// path (a thread sums a few hundred nodes at most), FP64 otherwise; per-block
// partials and everything after them are FP64.
template <class T>
struct AccType { using type = T; };

template <class A>
__device__ __forceinline__ void block_reduce_sums(A (&s)[kSums], double* out) {
    __shared__ double red[kStepThreads / 32][kSums];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kSums; ++k) {
        A v = s[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][k] = (double)v;
    }
    __syncthreads();
    if (threadIdx.x < kSums) {
        double t = 0.0;
        for (int w = 0; w < kStepThreads / 32; ++w) t += red[w][threadIdx.x];
        out[threadIdx.x] = t;
    }
}

// Fused step: pull-stream, (sample), collide with noise, store.
template <class T, int BASIS, bool SAMPLE>
__global__ void __launch_bounds__(kStepThreads)
step_kernel(StepArgs<T> a, CollideConst<T> cc) {
    using A = typename AccType<T>::type;
    const int Lx = a.geo.Lx;
    const long long N = (long long)Lx * a.geo.Ly;
    A s[kSums];
    if (SAMPLE) {
#pragma unroll
        for (int k = 0; k < kSums; ++k) s[k] = A(0);
    }
    // N < 2^31 (checked at creation): 32-bit node indices
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < (int)N; n += gridDim.x * blockDim.x) {
        const int y = n / Lx;
        const int x = n - y * Lx;
        T g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = a.src[at(a.geo, i, x - cvx(i), y - cvy(i))];
        if (SAMPLE) {
            A d[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) d[i] = A(g[i]) - A(a.ref[i]);
            int k = 9;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                s[i] += d[i];
#pragma unroll
                for (int j = i; j < 9; ++j) s[k++] += d[i] * d[j];
            }
        }
        T f[9];
        const uint32_t st = collide_basis<T, BASIS>(
            g, NodeNoise{cc.key, a.node0 + (uint32_t)n, a.step},
            [&](T* gg) {
#pragma unroll
                for (int i = 0; i < 9; ++i) gg[i] = g[i];
            },
            a.lut, cc, f);
        if (st != kStatusOk) record_error(a.err, (int)(st & 0xFF), (long long)a.node0 + n, a.step);
        store_node(a.dst, a.geo, x, y, f);
    }
    if (SAMPLE) block_reduce_sums<A>(s, a.partials + (long long)blockIdx.x * kSums);
}

// Sum over blocks of partials[b * kSums + q], computed by one warp: lane l adds
// blocks l, l + 32, ... in order, then a fixed butterfly combines the lanes, so
// the result does not depend on timing. All lanes return the total.
__device__ __forceinline__ double reduce_partials(const double* partials, int q, int nblocks,
                                                  int lane) {
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += __ldcg(&partials[(size_t)b * kSums + q]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Adds the per-block partials into the running FP64 sums; block q, one warp,
// handles sum q.
__global__ void accumulate_partials_kernel(const double* partials, int nblocks, double* acc);

// C = S2/n - m m^T, m = S1/n, and CM = B C B^T for the measurement basis B.
__global__ void finalize_kernel(const double* acc, long long nsamp, const double* basis,
                                double* out /* Cff[81], CMM[81], mean[9] */);

}  // namespace flb
