// flb_step_tma.cu -- the pipelined FP32 fused step for sm_103a.
//
// Persistent CTAs walk the lattice in tiles of 128 x TH nodes (TH = NW / 2).
// For every tile and every plane i, the box of 136 x TH populations that the
// pull g_i(x) = f*_i(x - v_i) of the tile needs (shifted by v_iy rows; 4 extra
// columns on each side cover v_ix = +-1) streams from HBM into a ring of
// shared-memory stages with 2D TMA copies, signalling mbarriers. NW consumer
// warps take two nodes per thread -- node A at tile column r, node B at
// r + 64 -- read their nine shifted populations from shared memory, collide
// both nodes at once in packed FP32x2 arithmetic (flb_collide.cuh with
// V = f2), release the stage and store straight to HBM, rows coalesced, with
// the ghost copies of edge nodes (flb_layout.cuh).
//
// Who refills a stage: a producer warp beside 8 to 14 consumer warps; with 16
// consumer warps (no room for a 17th) the last warp to release a stage.
//
// Correlation sums on sampling steps: by default each consumer warp stages its
// nodes' deviations in FP16 and adds them to a Gram matrix on the tensor cores
// (flb_gram.cuh); otherwise sampler warps read the same stage and accumulate
// the 9 + 45 sums in packed FP32x2 registers, or the consumers accumulate their
// own nodes. At the end the CTA reduces the sums to FP64 and adds them to the
// running sums with FP64 atomics: no separate reduction launch and no serial
// tail.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>

#include "flb_collide.cuh"
#include "flb_gram.cuh"
#include "flb_internal.h"
#include "flb_pipeline.cuh"
#include "flb_tma.cuh"

namespace flb {

// Tile coordinates (tx, ty) of t = blockIdx.x + k gridDim.x, k = 0, 1, ...,
// advanced without a division per tile.
struct TileWalk {
    int tx, ty, dx, dy, nx;
    __device__ __forceinline__ TileWalk(int t0, int step, int tiles_x) : nx(tiles_x) {
        ty = t0 / nx;
        tx = t0 - ty * nx;
        dy = step / nx;
        dx = step - dy * nx;
    }
    __device__ __forceinline__ void next() {
        tx += dx;
        ty += dy;
        if (tx >= nx) {
            tx -= nx;
            ++ty;
        }
    }
};

// Issue the nine TMA box loads of tile (tx, ty) into stage s (one thread).
template <int NW>
__device__ __forceinline__ void issue_tile(float* smem, const CUtensorMap* map, const TmaArgs& a,
                                           int tx, int ty, int s, uint64_t* full) {
    using TS = TileShape<NW>;
    mbar_arrive_expect_tx(&full[s], 9u * TS::TH * kBoxW * sizeof(float));
    const int x0 = tx * kTW, y0 = ty * TS::TH;
    float* st = smem + s * TS::STAGE;
#pragma unroll
    for (int i = 0; i < 9; ++i)
        tma_load_2d(st + i * TS::SPLANE, map, x0 + kXO - 4,
                    i * (a.geo.Ly + 2) + y0 + 1 - cvy(i), &full[s]);
}

// Producer state of an elected thread that refills each stage once every warp
// has released it. Stage s holds tiles s, s + STAGES, ... of this CTA; the
// tile coordinates advance by TileWalk, without a division per tile.
template <int NW>
struct Producer {
    int issued = 0;
    bool ok = true;
    TileWalk walk;   // the next tile to issue

    __device__ __forceinline__ explicit Producer(const TmaArgs& a)
        : walk(blockIdx.x, gridDim.x, a.tiles_x) {}

    __device__ __forceinline__ void issue(float* smem, const CUtensorMap* map, const TmaArgs& a,
                                          int s, uint64_t* full) {
        issue_tile<NW>(smem, map, a, walk.tx, walk.ty, s, full);
        walk.next();
    }

    __device__ __forceinline__ void prologue(float* smem, const CUtensorMap* map,
                                             const TmaArgs& a, uint64_t* full) {
        prefetch_tensormap(map);
        for (int t = blockIdx.x; t < a.ntiles && issued < TileShape<NW>::STAGES;
             t += gridDim.x, ++issued)
            issue(smem, map, a, issued, full);
    }
    // after this CTA's k-th tile (stage s, use n) was released by the caller
    __device__ __forceinline__ void refill(float* smem, const CUtensorMap* map, const TmaArgs& a,
                                           uint64_t* full, uint64_t* empty, int s, int n) {
        if (!ok) return;
        const int tn = blockIdx.x + issued * gridDim.x;
        if (tn >= a.ntiles) return;
        if (!mbar_wait_sleep(&empty[s], n & 1)) {
            record_error(a.err, kStatusTimeout, -1, a.step);
            ok = false;
            return;
        }
        issue(smem, map, a, s, full);
        ++issued;
    }
    // no copy may be in flight when the CTA exits: wait for tiles issued but not
    // consumed by the caller's loop (only after a timeout)
    __device__ __forceinline__ void drain(const TmaArgs& a, uint64_t* full, int consumed) {
        constexpr int S = TileShape<NW>::STAGES;
        for (int j = issued > S ? issued - S : 0; j < issued; ++j)
            if (j >= consumed && !mbar_wait(&full[j % S], (j / S) & 1)) {
                record_error(a.err, kStatusTimeout, -1, a.step);
                break;
            }
    }
};

// Correlation sums of two nodes (lanes of d, already centred and masked).
__device__ __forceinline__ void add_sums(float (&v)[kSums], const f2 (&d)[9]) {
    int q = 9;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        v[i] += d[i].v.x + d[i].v.y;
#pragma unroll
        for (int j = i; j < 9; ++j, ++q) v[q] = fmaf(d[i].v.x, d[j].v.x, fmaf(d[i].v.y, d[j].v.y, v[q]));
    }
}

// Sampling modes of the pipelined step.
enum : int { kNoSampling = 0, kSamplerWarps = 1, kFusedSampling = 2, kTensorSampling = 3 };

// With 16 colliding warps there is no producer warp (a 17th warp would cap
// every thread at 96 registers: one sub-partition would hold five warps):
// thread 0 issues the first STAGES tiles, and after that the last warp to
// release a stage refills it (a counter per stage in place of the empty
// barrier), so no thread waits for the others.
template <int NW, int MODE>
constexpr bool embedded_producer() {
    return NW >= 16 && (MODE == kNoSampling || MODE == kTensorSampling);
}

template <int MODE>
struct WarpCount {
    template <int NW>
    static constexpr int extra() {
        return MODE == kSamplerWarps ? kSamplers
                                     : (MODE == kFusedSampling || embedded_producer<NW, MODE>() ? 0 : 1);
    }
};

// Shared memory of the tensor-sampling mode beyond the ring and the reduction
// buffer: one Gram block per colliding warp.
template <int NW>
constexpr size_t gram_smem_bytes() {
    return (size_t)NW * kGramWarpHalves * sizeof(__half);
}

// Every shape fits the 227 KB of shared memory a CTA may take.
constexpr size_t kMaxSmem = 227 * 1024;
static_assert(TileShape<8>::smem_bytes() + gram_smem_bytes<8>() <= kMaxSmem, "8 warps");
static_assert(TileShape<12>::smem_bytes() + gram_smem_bytes<12>() <= kMaxSmem, "12 warps");
static_assert(TileShape<14>::smem_bytes() + gram_smem_bytes<14>() <= kMaxSmem, "14 warps");
static_assert(TileShape<16>::smem_bytes() + gram_smem_bytes<16>() <= kMaxSmem, "16 warps");

// Warp roles. kNoSampling: NW consumer warps + one producer warp.
// kSamplerWarps: NW consumers + kSamplers sampler warps (sampler w reads rows
// w, w + kSamplers, ... of each tile from the same stage and accumulates the
// sums in packed registers); the first sampler lane produces.
// kFusedSampling: NW consumers that also accumulate the sums of their own
// nodes; lane 0 of warp 0 produces.
// kTensorSampling: NW consumers that accumulate the sums of their own nodes as
// a Gram matrix on the tensor cores (flb_gram.cuh) + one producer warp.
template <int BASIS, int MODE, int NW>
__global__ void __launch_bounds__((NW + WarpCount<MODE>::template extra<NW>()) * 32, 1)
step_tma_kernel(const __grid_constant__ CUtensorMap map, const TmaArgs a,
                const CollideConst<float> cc) {
    using TS = TileShape<NW>;
    constexpr int TH = TS::TH;
    constexpr int kStages = TS::STAGES;
    constexpr int NX = WarpCount<MODE>::template extra<NW>();
    extern __shared__ __align__(128) float smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * TS::STAGE);
    uint64_t* empty = full + kStages;
    double* red = reinterpret_cast<double*>(empty + kStages);
    constexpr bool kTensor = MODE == kTensorSampling;
    // tensor sampling: FP64 Gram matrix (16 x 16) in red, the warps' blocks after it
    __half* gram = reinterpret_cast<__half*>(red + TS::RED * kSums);

    const int warp = threadIdx.x >> 5, lane_id = threadIdx.x & 31;
    constexpr bool kEmbed = embedded_producer<NW, MODE>();
    static_assert(!kEmbed || (NW & (NW - 1)) == 0, "release counts wrap at 2^32");
    // kEmbed: the empty barriers' words count the releases of each stage
    uint32_t* released = reinterpret_cast<uint32_t*>(empty);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            if (kEmbed)
                released[s] = 0u;
            else
                mbar_init(&empty[s], NW + (MODE == kSamplerWarps ? NX : 0));
        }
        fence_mbar_init();
    }
    if (kTensor) {
        if (threadIdx.x < 256) red[threadIdx.x] = 0.0;
        if (warp < NW) gram_init(gram + warp * kGramWarpHalves);
    }
    __syncthreads();

    const int Lx = a.geo.Lx, Ly = a.geo.Ly;

    if ((MODE == kNoSampling || kTensor) && !kEmbed && warp == NW) {
        // ---------------- producer warp
        if (lane_id == 0) {
            Producer<NW> prod(a);
            prod.prologue(smem, &map, a, full);
            int s = 0, n = 0;
            for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
                prod.refill(smem, &map, a, full, empty, s, n);
                if (++s == kStages) {
                    s = 0;
                    ++n;
                }
            }
            prod.drain(a, full, prod.issued);
        }
        return;
    }

    if (MODE == kSamplerWarps && warp >= NW) {
        // ---------------- sampler warps
        const int sw = warp - NW;
        const bool producer = sw == 0 && lane_id == 0;
        Producer<NW> prod(a);
        if (producer) prod.prologue(smem, &map, a, full);
        f2 s1[9], s2[45];
#pragma unroll
        for (int q = 0; q < 9; ++q) s1[q] = f2(0.f);
#pragma unroll
        for (int q = 0; q < 45; ++q) s2[q] = f2(0.f);
        int k = 0, s = 0, n = 0;
        TileWalk w(blockIdx.x, gridDim.x, a.tiles_x);
        for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++k, w.next()) {
            if (!mbar_wait_sleep(&full[s], n & 1)) {
                record_error(a.err, kStatusTimeout, -1, a.step);
                break;
            }
            const int x0 = w.tx * kTW;
            for (int row = sw; row < TH; row += NX) {
                const int y = w.ty * TH + row;
                const float* st = smem + s * TS::STAGE + row * kBoxW + 4 + lane_id;
                f2 d[2][9];
#pragma unroll
                for (int p = 0; p < 2; ++p)
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        const float* q = st + i * TS::SPLANE - cvx(i) + 64 * p;
                        d[p][i] = f2(q[0], q[32]);
                    }
                if (row + NX >= TH) warp_arrive(&empty[s], lane_id);   // last row: release first
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const int xA = x0 + lane_id + 64 * p;
                    const bool inA = xA < Lx && y < Ly, inB = xA + 32 < Lx && y < Ly;
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        f2 e = d[p][i] - f2(a.ref[i]);
                        if (!(inA && inB)) e = f2(inA ? e.v.x : 0.f, inB ? e.v.y : 0.f);
                        d[p][i] = e;
                    }
                    int q = 0;
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        s1[i] += d[p][i];
#pragma unroll
                        for (int j = i; j < 9; ++j, ++q) s2[q] = mad(d[p][i], d[p][j], s2[q]);
                    }
                }
            }
            if (sw >= TH) warp_arrive(&empty[s], lane_id);   // a sampler without a row here
            if (producer) prod.refill(smem, &map, a, full, empty, s, n);
            if (++s == kStages) {
                s = 0;
                ++n;
            }
        }
        if (producer) prod.drain(a, full, k);
        float v[kSums];
#pragma unroll
        for (int q = 0; q < kSums; ++q) {
            const f2 x = q < 9 ? s1[q] : s2[q - 9];
            v[q] = x.v.x + x.v.y;
        }
        publish_sums(v, NW, NX * 32, red, a);
        return;
    }

    // ---------------- consumers: two nodes per thread, packed FP32x2
    const int c = threadIdx.x;          // 0 .. 32 NW - 1
    const int ty = c >> 6, r = c & 63;
    constexpr bool kFused = MODE == kFusedSampling;
    const bool producer = (kFused || kEmbed) && c == 0;
    Producer<NW> prod(a);
    if (producer) prod.prologue(smem, &map, a, full);
    float v[kFused ? kSums : 1];
    if (kFused) {
#pragma unroll
        for (int q = 0; q < kSums; ++q) v[q] = 0.f;
    }
    float gc[kTensor ? 8 : 1];
    if (kTensor) {
#pragma unroll
        for (int q = 0; q < 8; ++q) gc[q] = 0.f;
    }
    int gtiles = 0;
    const GramLane gblk(smem_u32(gram + warp * kGramWarpHalves), kGramRows);
    int k = 0, s = 0, n = 0;   // tile count, its stage and the stage's use
    bool timed_out = false;
    TileWalk w(blockIdx.x, gridDim.x, a.tiles_x);
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++k, w.next()) {
        if (!mbar_wait(&full[s], n & 1)) {
            record_error(a.err, kStatusTimeout, -1, a.step);
            timed_out = true;
            break;
        }
        const float* st = smem + s * TS::STAGE + ty * kBoxW + 4 + r;
        auto load = [&](f2* g) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const float* p = st + i * TS::SPLANE - cvx(i);
                g[i] = f2(p[0], p[64]);
            }
        };
        f2 g[9];
        load(g);

        // tile origin (the same for every thread, so the tests on it below
        // are uniform branches) and this thread's nodes
        const int x0 = w.tx * kTW, y0 = w.ty * TH;
        const int y = y0 + ty;
        const int xA = x0 + r, xB = xA + 64;
        const bool inA = xA < Lx && y < Ly, inB = xB < Lx && y < Ly;
        const bool whole = x0 + kTW <= Lx && y0 + TH <= Ly;   // every node of the tile
        if (a.fields) {
            // structure-factor sample of this state: drho, dj_x, dj_y of both
            // nodes from the deviations f_i - ref_i, summed in the order the
            // separate field kernel uses (the same FP32 values)
            f2 d[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) d[i] = g[i] - f2(a.ref[i]);
            const f2 fr = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
            const f2 fx = (d[1] - d[3]) + ((d[5] - d[6]) + (d[8] - d[7]));
            const f2 fy = (d[2] - d[4]) + ((d[5] + d[6]) - (d[7] + d[8]));
            const size_t N = (size_t)Lx * Ly;
            float* o = a.fields + (size_t)y * Lx + xA;
            if (whole || inA) {
                o[0] = fr.v.x;
                o[N] = fx.v.x;
                o[2 * N] = fy.v.x;
            }
            if (whole || inB) {
                o[64] = fr.v.y;
                o[N + 64] = fx.v.y;
                o[2 * N + 64] = fy.v.y;
            }
        }
        if (kFused) {
            f2 d[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                f2 e = g[i] - f2(a.ref[i]);
                if (!whole) e = f2(inA ? e.v.x : 0.f, inB ? e.v.y : 0.f);
                d[i] = e;
            }
            add_sums(reinterpret_cast<float(&)[kSums]>(v), d);
        }
        // tensor sampling: stage this tile's nodes when the collision reads
        // them a second time
        auto stage = [&](const f2* gs) {
            f2 hs[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) hs[i] = mad(gs[i], f2(a.sinv), f2(a.snref[i]));
            if (!whole) {
#pragma unroll
                for (int i = 0; i < 9; ++i) hs[i] = f2(inA ? hs[i].v.x : 0.f, inB ? hs[i].v.y : 0.f);
            }
            gram_stage(gblk, hs);
        };
        auto refetch = [&](f2* gg) {
            load(gg);
            if (kTensor) stage(gg);
        };
        const uint32_t nodeA = a.node0 + (uint32_t)xA + (uint32_t)Lx * (uint32_t)y;
        f2 f[9];
        const uint32_t stt = collide_basis<f2, BASIS>(
            g, PairNoise{cc.key, nodeA, nodeA + 64u, a.step}, refetch, a.lut,
            cc, f);
        if (kTensor) {
            gram_mma(gblk, reinterpret_cast<float(&)[8]>(gc));
            if (++gtiles == kGramFlushTiles) {
                gram_flush(reinterpret_cast<float(&)[8]>(gc), red);
                gtiles = 0;
            }
        }
        // the stage is held until g was read the second time
        if constexpr (kEmbed) {
            // the NW-th release of this use of the stage refills it with the
            // CTA's tile kStages later (the counter is never reset: NW divides
            // 2^32)
            __syncwarp();
            if (lane_id == 0 && ((release_count(&released[s]) + 1u) & (NW - 1)) == 0) {
                const int tn = t + kStages * gridDim.x;
                if (tn < a.ntiles) {
                    fence_proxy_async_smem();
                    const int nty = tn / a.tiles_x;
                    issue_tile<NW>(smem, &map, a, tn - nty * a.tiles_x, nty, s, full);
                }
            }
        } else {
            warp_arrive(&empty[s], lane_id);
        }
        if (stt) {
            if (inA && (stt & 0xFF)) record_error(a.err, (int)(stt & 0xFF), nodeA, a.step);
            if (inB && (stt >> 8)) record_error(a.err, (int)(stt >> 8), nodeA + 64u, a.step);
        }
        // an inner tile stores without edge tests; on an edge tile each lane
        // tests its node and adds the ghost copies it needs
        const bool inner = x0 > 0 && y0 > 0 && x0 + kTW < Lx && y0 + TH < Ly;
        float* pa = a.dst + at(a.geo, 0, xA, y);
        if (inner) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                pa[i * a.geo.plane] = f[i].v.x;
                pa[i * a.geo.plane + 64] = f[i].v.y;
            }
        } else {
            if (inA) store_lane_ghosts(pa, a.geo, xA, y, f, 0);
            if (inB) store_lane_ghosts(pa + 64, a.geo, xB, y, f, 1);
        }
        if (producer && !kEmbed) prod.refill(smem, &map, a, full, empty, s, n);
        if (++s == kStages) {
            s = 0;
            ++n;
        }
    }
    if (kEmbed && timed_out && lane_id == 0) {
        // copies this warp did not consume may still be in flight: wait (with
        // the bound of every wait) for the next kStages tiles
        for (int j = k; j < k + kStages && blockIdx.x + j * gridDim.x < a.ntiles; ++j)
            if (!mbar_wait(&full[j % kStages], (j / kStages) & 1)) break;
    }
    if (kFused) {
        if (producer) prod.drain(a, full, k);
        publish_sums(reinterpret_cast<float(&)[kSums]>(v), 0, NW * 32, red, a);
    }
    if (kTensor) {
        gram_flush(reinterpret_cast<float(&)[8]>(gc), red);
        named_sync(1, NW * 32);
        if (c < kSums) atomicAdd(&a.acc[c], gram_sum(red, c, a.s));
    }
}

// The bounded wait the pipelined kernels rely on, exercised alone: a warp
// waits on an mbarrier that nothing completes, gives up after `limit` cycles
// and records a timeout as a step kernel would (no fault, no hang).
__global__ void wait_probe_kernel(long long limit, DevError* err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const bool done = mbar_wait_for(&bar, 0, limit);
    if (!done && threadIdx.x == 0) record_error(err, kStatusTimeout, -1, 0);
}

cudaError_t wait_probe(long long limit, DevError* err, cudaStream_t s) {
    if (limit < 0 || limit > kWaitCycles) return cudaErrorInvalidValue;
    wait_probe_kernel<<<1, 32, 0, s>>>(limit, err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

namespace {

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                              const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                              const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
    static EncodeFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

template <int NW, int MODE>
const void* kernel_ptr_m(int basis) {
    if (basis == 0) return (const void*)step_tma_kernel<0, MODE, NW>;
    if (basis == 1) return (const void*)step_tma_kernel<1, MODE, NW>;
    return (const void*)step_tma_kernel<2, MODE, NW>;
}

template <int NW>
const void* kernel_ptr(int basis, int mode) {
    if (mode == kTensorSampling) return kernel_ptr_m<NW, kTensorSampling>(basis);
    if constexpr (NW > 12) {
        return mode == kNoSampling ? kernel_ptr_m<NW, kNoSampling>(basis) : nullptr;
    } else {
        if (mode == kSamplerWarps) return kernel_ptr_m<NW, kSamplerWarps>(basis);
        if (mode == kFusedSampling) return kernel_ptr_m<NW, kFusedSampling>(basis);
        return kernel_ptr_m<NW, kNoSampling>(basis);
    }
}

const void* kernel_for(int nw, int basis, int mode) {
    switch (nw) {
        case 8: return kernel_ptr<8>(basis, mode);
        case 12: return kernel_ptr<12>(basis, mode);
        case 14: return kernel_ptr<14>(basis, mode);
        case 16: return kernel_ptr<16>(basis, mode);
        default: return nullptr;
    }
}

int warps_for(int nw, int mode) {
    if (mode == kSamplerWarps) return nw + kSamplers;
    if (mode == kFusedSampling || nw >= 16) return nw;
    return nw + 1;
}

// Dynamic shared memory of a plan (the largest of its modes).
size_t smem_for(int nw) {
    switch (nw) {
        case 8: return TileShape<8>::smem_bytes() + gram_smem_bytes<8>();
        case 12: return TileShape<12>::smem_bytes() + gram_smem_bytes<12>();
        case 14: return TileShape<14>::smem_bytes() + gram_smem_bytes<14>();
        case 16: return TileShape<16>::smem_bytes() + gram_smem_bytes<16>();
        default: return 0;
    }
}

}  // namespace

cudaError_t tma_encode_planes(CUtensorMap* map, void* buf, const Geometry& g, int box_w, int th,
                              int elem_bytes) {
    EncodeFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)g.pitch, (cuuint64_t)(9 * (long long)(g.Ly + 2))};
    if (elem_bytes != 4 && elem_bytes != 2) return cudaErrorInvalidValue;
    const cuuint64_t strides[1] = {(cuuint64_t)g.pitch * (cuuint64_t)elem_bytes};
    const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)th};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType dt =
        elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const CUresult rc = enc(map, dt, 2, buf, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return rc == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t tma_plan(TmaPlan* plan, void* buf0, void* buf1, const Geometry& g, int nw) {
    plan->ready = false;
    if (nw == 0) nw = kDefaultNW;
    if (!kernel_for(nw, 0, kNoSampling)) return cudaErrorInvalidValue;
    const int th = nw / 2;
    void* bufs[2] = {buf0, buf1};
    for (int b = 0; b < 2; ++b) {
        const cudaError_t e = tma_encode_planes(&plan->map[b], bufs[b], g, kBoxW, th);
        if (e != cudaSuccess) return e;
    }
    const size_t smem = smem_for(nw);
    int dev = 0, sms = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = 2;
    for (int basis = 0; basis < 3 && ce == cudaSuccess; ++basis)
        for (int mode = 0; mode < 4 && ce == cudaSuccess; ++mode) {
            const void* fn = kernel_for(nw, basis, mode);
            if (!fn) continue;
            ce = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            int n = 0;
            if (ce == cudaSuccess)
                ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, warps_for(nw, mode) * 32,
                                                                   smem);
            if (n < per_sm) per_sm = n;
        }
    if (ce != cudaSuccess) return ce;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    plan->nw = nw;
    plan->smem = smem;
    plan->tiles_x = (g.Lx + kTW - 1) / kTW;
    plan->ntiles = plan->tiles_x * ((g.Ly + th - 1) / th);
    int grid = sms * per_sm;
    if (grid > plan->ntiles) grid = plan->ntiles;
    plan->grid = grid < 1 ? 1 : grid;
    if (plan->sample_mode != kSamplerWarps && plan->sample_mode != kFusedSampling &&
        plan->sample_mode != kTensorSampling)
        plan->sample_mode = kDefaultSampling;
    if (!kernel_for(nw, 0, plan->sample_mode)) plan->sample_mode = kTensorSampling;
    plan->ready = true;
    return cudaSuccess;
}

cudaError_t tma_step(const TmaPlan& plan, int src, const TmaArgs& a,
                     const CollideConst<float>& cc, int basis, bool sample, cudaStream_t s) {
    const int mode = sample ? plan.sample_mode : kNoSampling;
    const void* fn = kernel_for(plan.nw, basis, mode);
    if (!fn || !plan.ready) return cudaErrorInvalidValue;
    TmaArgs args = a;
    args.tiles_x = plan.tiles_x;
    args.ntiles = plan.ntiles;
    void* params[3] = {(void*)&plan.map[src], (void*)&args, (void*)&cc};
    return cudaLaunchKernel(fn, dim3(plan.grid), dim3(warps_for(plan.nw, mode) * 32), params,
                            plan.smem, s);
}

}  // namespace flb
