// flb_gram.cuh -- the equal-time correlation sums of the nodes a warp collides,
// accumulated on the tensor cores.
//
// The sums S1_i = sum_x d_i(x) and S2_ij = sum_x d_i(x) d_j(x) of the centred
// pre-collision populations d = f - f^0(rho0, u0) (Eqs. dfdef, efif0) are one
// Gram matrix: with H the 16 x K matrix whose rows 0..8 hold d_i / s over K
// nodes and row 9 holds ones, C = H H^T has C_ij = S2_ij / s^2 and
// C_i9 = S1_i / s. A warp stages its 64 nodes (two per thread) as FP16 (round
// to nearest) in rows 0..9 of a shared-memory block (gram_stage), loads 16
// rows back in the fragment layout of mma.m16n8k16 with ldmatrix and
// accumulates C in FP32 registers, 8 per thread (gram_mma); every
// kGramFlushTiles tiles the FP32 partials of rows and columns 0..9 are added
// to an FP64 16 x 16 matrix in shared memory (gram_flush). Rows 10..15 of H
// only reach rows and columns 10..15 of C, which nothing reads: they are not
// allocated, and the ldmatrix lanes of rows 10..15 read the warp's own rows
// 2..7 (finite values the warp staged itself; rows 8, 9 and 2..7 fall in
// distinct shared-memory banks).
//
// The scale s (sqrt(kT rho0)) makes the thermal fluctuations of order one in
// FP16, whose rounding (relative 2^-12, unbiased) enters the sums as noise
// far below their statistical error; it is chosen by the host only where
// every deviation a valid state can hold stays in FP16's range, and the
// sampler-warp path (FP32 products) is used otherwise.
#pragma once

#include <cuda_fp16.h>

#include <cstdint>

#include "flb_tma.cuh"
#include "flb_vec.cuh"

namespace flb {

constexpr int kGramRowHalves = 72;                       // 64 nodes + 8 halves: 144-byte rows
constexpr int kGramRows = 10;                            // rows of H a warp stages
constexpr int kGramWarpHalves = kGramRows * kGramRowHalves;   // one warp's block: 1440 bytes
constexpr int kGramFlushTiles = 16;                      // FP32 partials of <= 1024 products

// The constant row of a warp's block: row 9, ones.
__device__ __forceinline__ void gram_init(__half* blk) {
    const int lane = threadIdx.x & 31;
    reinterpret_cast<uint32_t*>(blk)[9 * (kGramRowHalves / 2) + lane] = 0x3C003C00u;
}
// A block with all 16 rows (row 9 ones, rows 10..15 zeros), for the batched
// kernel, which has shared memory to spare: measured 1 % faster there than
// ten-row blocks (the one-lattice kernel needs the room for its fifth stage).
constexpr int kGramFullHalves = 16 * kGramRowHalves;
__device__ __forceinline__ void gram_init_full(__half* blk) {
    const int lane = threadIdx.x & 31;
    uint32_t* w = reinterpret_cast<uint32_t*>(blk);
#pragma unroll
    for (int r = 9; r < 16; ++r) w[r * (kGramRowHalves / 2) + lane] = r == 9 ? 0x3C003C00u : 0u;
}

__device__ __forceinline__ void mma16816(float (&c)[8], int o, uint32_t a0, uint32_t a1,
                                         uint32_t a2, uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[o]), "+f"(c[o + 1]), "+f"(c[o + 2]), "+f"(c[o + 3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Shared addresses of one thread in its warp's block, computed once: the
// word it stages (column pair 2 lane, 2 lane + 1 of row 0) and the row its
// ldmatrix lanes address (threads 8m..8m+7 give the rows of matrix m; the
// matrices (rows 0-7, k 0-7), (rows 8-15, k 0-7), (rows 0-7, k 8-15),
// (rows 8-15, k 8-15) of a 16-node step are the A fragment of
// mma.m16n8k16, and H^T's B fragments of the column blocks 0-7 and 8-15 are
// matrices (0, 2) and (1, 3)).
struct GramLane {
    uint32_t st, ld;
    // rows: the rows the block holds (kGramRows, or 16 for a full block)
    __device__ __forceinline__ GramLane(uint32_t blk, int rows) {
        const int lane = threadIdx.x & 31, m = lane >> 3, r = lane & 7;
        const int row = (m & 1) * 8 + r;
        st = blk + 4u * lane;
        ld = blk + 2u * ((row < rows ? row : row - 8) * kGramRowHalves + (m >> 1) * 8);
    }
};

template <int I>
__device__ __forceinline__ void gram_store(uint32_t st, f2 h) {
    const __half2 v = __floats2half2_rn(h.v.x, h.v.y);
    asm volatile("st.shared.b32 [%0+%1], %2;" ::"r"(st), "n"(2 * kGramRowHalves * I),
                 "r"(*reinterpret_cast<const uint32_t*>(&v)));
}

template <int S>
__device__ __forceinline__ void gram_step(uint32_t ld, float (&c)[8]) {
    uint32_t d0, d1, d2, d3;
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4+%5];"
                 : "=r"(d0), "=r"(d1), "=r"(d2), "=r"(d3)
                 : "r"(ld), "n"(32 * S));
    mma16816(c, 0, d0, d1, d2, d3, d0, d2);
    mma16816(c, 4, d0, d1, d2, d3, d1, d3);
}

// Stage the 64 nodes of this warp (h: node A of the thread in .x, node B in .y,
// already scaled by 1/s and zero for nodes outside the lattice). The warp must
// have finished reading the block's previous contents.
__device__ __forceinline__ void gram_stage(const GramLane& g, const f2 (&h)[9]) {
    __syncwarp();
    gram_store<0>(g.st, h[0]);
    gram_store<1>(g.st, h[1]);
    gram_store<2>(g.st, h[2]);
    gram_store<3>(g.st, h[3]);
    gram_store<4>(g.st, h[4]);
    gram_store<5>(g.st, h[5]);
    gram_store<6>(g.st, h[6]);
    gram_store<7>(g.st, h[7]);
    gram_store<8>(g.st, h[8]);
}

// Add the staged block to c: four 16-node steps of two mma.m16n8k16 each.
__device__ __forceinline__ void gram_mma(const GramLane& g, float (&c)[8]) {
    __syncwarp();
    gram_step<0>(g.ld, c);
    gram_step<1>(g.ld, c);
    gram_step<2>(g.ld, c);
    gram_step<3>(g.ld, c);
}

// Add the FP32 partials to the FP64 matrix cm[16][16] (rows and columns 0..9
// only) and clear them. Fragment of thread (g, q) = (lane / 4, lane % 4):
// c[0..3] = C[g][2q], C[g][2q+1], C[g+8][2q], C[g+8][2q+1]; c[4..7] the same
// with the columns + 8.
__device__ __forceinline__ void gram_flush(float (&c)[8], double* cm) {
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int row = g + ((k & 2) ? 8 : 0);
        const int col = 2 * q + (k & 1) + ((k & 4) ? 8 : 0);
        if (row < 10 && col < 10) atomicAdd(&cm[row * 16 + col], (double)c[k]);
        c[k] = 0.f;
    }
}

// Sum q of the kSums layout (9 first moments, then the upper triangle of the
// second moments row by row) from the FP64 Gram matrix: S1_i = s C[i][9],
// S2_ij = s^2 C[i][j].
__device__ __forceinline__ double gram_sum(const double* cm, int q, double s) {
    if (q < 9) return s * cm[q * 16 + 9];
    int k = q - 9, i = 0;
    while (k >= 9 - i) {
        k -= 9 - i;
        ++i;
    }
    return s * s * cm[i * 16 + i + k];
}

}  // namespace flb
