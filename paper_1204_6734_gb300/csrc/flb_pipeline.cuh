// flb_pipeline.cuh -- pieces shared by the pipelined FP32 step kernels (one
// lattice: flb_step_tma.cu; many lattices: flb_batch.cu): tile shape of the
// shared-memory ring, storing a packed node pair, and the CTA/grid reduction of
// correlation sums.
#pragma once

#include <cuda_runtime.h>

#include "flb_collide.cuh"
#include "flb_internal.h"
#include "flb_kernels.cuh"
#include "flb_layout.cuh"
#include "flb_tma.cuh"

namespace flb {

constexpr int kTW = 128;               // tile width (nodes)
constexpr int kBoxW = kTW + 8;         // TMA box width: x0 - 4 .. x0 + 131
constexpr int kDefaultNW = 8;
constexpr int kSamplers = 4;   // sampler warps: one per SM sub-partition
constexpr int kDefaultSampling = 1;   // kSamplerWarps

// Tile of 128 x TH nodes, TH = NW / 2; the ring holds STAGES tiles. The ring
// must be deep: a stage is in flight from HBM only between its refill and its
// arrival, and consumers keep their stage until they have finished the tile.
template <int NW>
struct TileShape {
    static constexpr int TH = NW / 2;                                  // rows per tile
    static constexpr int SPLANE = (TH * kBoxW + 31) / 32 * 32;         // floats per plane box
    static constexpr int STAGE = 9 * SPLANE;                           // floats per stage
    static constexpr int STAGES = NW <= 8 ? 8 : (NW <= 12 ? 6 : 5);   // 157 / 176 / 173 / 196 KB
    static constexpr int RED = NW > kSamplers ? NW : kSamplers;        // warps reducing
    static constexpr size_t smem_bytes() {
        return sizeof(float) * (size_t)STAGES * STAGE + 2 * STAGES * sizeof(uint64_t) +
               sizeof(double) * RED * kSums;
    }
};

// Store lane k of a node pair, interior node (x, y) whose cell in plane 0 is
// pa, with the ghost copies it needs (store_node_ghosts).
__device__ __forceinline__ void store_lane_ghosts(float* pa, const Geometry& geo, int x, int y,
                                                  const f2 f[9], int k) {
    float v[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) v[i] = lane(f[i], k);
    store_node_ghosts(pa, geo, x, y, v);
}

// CTA reduction of per-thread correlation sums held by `group` threads (warps
// [w0, w0 + group/32)): warp shuffles, FP64 across warps in warp order, then
// one FP64 atomic add per sum and CTA into the running sums. The order in which
// CTAs add is not fixed, so the last bits of the FP64 sums may differ between
// runs; a deterministic last-CTA reduction was measured to hold one SM for
// 15-25 us at the end of every sampled step.
__device__ __forceinline__ void publish_sums(const float (&v)[kSums], int w0, int group,
                                             double* red, const TmaArgs& a) {
    const int warp = threadIdx.x >> 5, lane_id = threadIdx.x & 31;
    const int nw = group / 32, c = threadIdx.x - 32 * w0;
#pragma unroll
    for (int q = 0; q < kSums; ++q) {
        float x = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane_id == 0) red[(warp - w0) * kSums + q] = (double)x;
    }
    named_sync(1, group);
    if (c < kSums) {
        double tot = 0.0;
        for (int w = 0; w < nw; ++w) tot += red[w * kSums + c];
        atomicAdd(&a.acc[c], tot);
    }
}

}  // namespace flb
