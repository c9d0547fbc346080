// flb_batch_kernel.cuh -- the pipelined FP32 fused step over many independent
// lattices ("replicas") of different sizes and parameters in one launch.
//
// Every replica has its own two population buffers (ghost-frame layout,
// flb_layout.cuh) and a descriptor in device memory: the TMA tensor maps of
// its two buffers and a 448-byte "hot" block (collision constants, reference
// equilibrium, geometry, pointers, time and sampling schedule). The tiles of
// all replicas form one table; CTA b walks the contiguous range
// [b T / G, (b + 1) T / G) of it, so it meets each replica in one run.
//
// For every tile the producer thread reads the tile's code and its replica's
// time from global memory, writes a small tile record (origin, time, live) into
// the stage and loads the nine population boxes plus the hot block into the
// same stage; consumers and samplers take everything they need from the stage.
// A replica whose time has reached its end (tend) is skipped: its stage gets
// only the record. The batch step counter and the tile count live in device
// memory (BatchCtl) and the last CTA to finish advances the step, so a CUDA
// graph of k launches can be replayed while the host changes the membership
// between replays: replica r is at time t_r = t0_r + (step - join_r).
//
// Tile shapes (the autotuner's choices): TW x TH nodes, NW consumer warps,
// NPT nodes per consumer thread (2: packed FP32x2 pairs at columns r and
// r + TW/2; 1: scalar), TH = NW * 32 * NPT / TW. The register file bounds the
// warp count: with 8 consumers (about 160 registers each in the f-norm) the
// correlation sums come from 4 sampler warps (108 registers for their packed
// sums); with 12 consumers (at most 128 registers) the consumers add their own
// nodes to a Gram matrix on the tensor cores (flb_gram.cuh), flushed per run
// of tiles of one replica into FP64 sums in shared memory (the first
// kRunSlots runs of the CTA) or straight into the replica's FP64 sums.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "flb_gram.cuh"
#include "flb_pipeline.cuh"

namespace flb {

struct __align__(16) ReplicaHot {
    CollideConst<float> cc;   // -omega, amplitudes, Philox round keys
    float ref[9];             // f^0(rho0, u0), subtracted before sampling
    int Lx, Ly, tiles_x;
    float gram_inv;           // 1 / s of the tensor-core sums (0: not allowed)
    int t0, join;             // replica time t0 at batch step `join`
    int warmup, every;        // sampling schedule (every = 0: off)
    long long pitch, plane;
    float* buf[2];            // buffer (t & 1) holds f*(t - 1), the source of step t
    double* acc;              // kSums running sums
    DevError* err;
    int tend;                 // the replica stops before time tend
    float gram_s;             // s = sqrt(kT rho0): nodes are staged as (f - ref) / s
    // packed pairs {c, c} of the constants the node-pair consumers use
    CollidePairs pc;          // -omega_a, -amp_a
    float2 sinv;              // 1 / s
    float2 snref[9];          // -ref_i / s: staged value (f_i - ref_i) / s = f_i / s + snref_i
    // mixed tiling: tiles of kind 0 (tiles_x columns), of kinds 0 and 1, and
    // the x origins of the kind-1 and kind-2 columns
    int kt0, kt01, kx1, kx2;
};
static_assert(sizeof(ReplicaHot) == 448, "the hot block is copied as 448 bytes");
static_assert(offsetof(ReplicaHot, pc) == 256 && offsetof(ReplicaHot, snref) % 8 == 0,
              "packed pairs start on 8-byte boundaries");

// Mixed tiling (tile width kMixedTW): a replica is cut into column bands of
// three tile kinds of 768 nodes each, kind k = (128 >> k) x (6 << k) nodes:
// 128-wide columns, then at most one 64-wide and one 32-wide column for the
// rest of the width, so that no band pads more than 31 columns. Every kind
// keeps two nodes per thread and 12 consumer warps.
constexpr int kMixedTW = 0;
constexpr int kKinds = 3;
__host__ __device__ constexpr int kind_tw(int k) { return 128 >> k; }
__host__ __device__ constexpr int kind_th(int k) { return 6 << k; }
__host__ __device__ constexpr int kind_bw(int k) { return (128 >> k) + 8; }

struct __align__(128) ReplicaDesc {
    CUtensorMap map[2 * kKinds];   // tensor map of (kind k, buffer b) at 2 k + b
    ReplicaHot hot;
};

struct BatchCtl {
    unsigned int step;        // launches completed
    unsigned int ticket;      // CTAs finished in the current launch
    int ntiles;               // entries of the tile table in use
    int pad;
};

struct BatchArgs {
    const ReplicaDesc* desc;
    const uint32_t* tiles;    // (replica << kLocalBits) | tile index within the replica
    BatchCtl* ctl;
    const float* lut;         // velocity table of the look-up-table f-norm (BASIS 2)
};

constexpr int kLocalBits = 18;
constexpr uint32_t kLocalMask = (1u << kLocalBits) - 1u;
constexpr int kMaxBatchReplicas = 1 << (32 - kLocalBits);

constexpr int kBatchNW = 8;       // consumer warps beside sampler warps
constexpr int kBatchNWTensor = 12;  // consumer warps with the tensor-core sums
constexpr int kRunSlots = 4;        // runs of one replica whose sums a CTA keeps in shared memory

template <int TW_, int NPT, int NW_ = kBatchNW>
struct BatchShape {
    static constexpr int NW = NW_;
    static constexpr bool MIXED = TW_ == kMixedTW;
    static_assert(!MIXED || (NPT == 2 && NW == kBatchNWTensor), "mixed tiling: 12 warps, node pairs");
    static constexpr bool TENSOR = NW > kBatchNW;
    static constexpr int TW = MIXED ? kind_tw(0) : TW_;           // (mixed: of kind 0)
    static constexpr int TH = NW * 32 * NPT / TW;                // rows per tile
    static constexpr int BW = TW + 8;                            // box width: x0 - 4 .. x0 + TW + 3
    static constexpr int RW = TW / NPT;                          // consumer threads per row
    static constexpr int PAIRS = TW / 64;                        // node pairs per sampler lane and row
    // floats per plane box (mixed: room for the largest box, kind 2's)
    static constexpr int SPLANE = MIXED ? kind_th(2) * kind_bw(2) : (TH * BW + 31) / 32 * 32;
    static constexpr int HOT = sizeof(ReplicaHot) / 4;           // floats of the hot block
    static constexpr int INFO = 32;                              // tile record, padded to 128 B
    // a multiple of 32 floats, so that every plane box of every stage starts
    // on the 128-byte boundary a tensor copy into shared memory needs
    static constexpr int STAGE = (9 * SPLANE + HOT + INFO + 31) / 32 * 32;
    static_assert(SPLANE % 32 == 0 && STAGE % 32 == 0, "128-byte aligned boxes");
    static constexpr int FIT = (MIXED ? 180000 : 163840) / (4 * STAGE);   // 160-176 KB of stages
    static constexpr int STAGES = FIT < 16 ? FIT : 16;
    static constexpr size_t GRAM =
        TENSOR ? (size_t)NW * kGramFullHalves * 2 + kRunSlots * 256 * 8 + kRunSlots * 16 + NW * 16 : 0;
    static constexpr size_t smem_bytes() {
        return sizeof(float) * (size_t)STAGES * STAGE + 2 * STAGES * sizeof(uint64_t) + 16 + GRAM;
    }
};

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Fill stage s with global tile t (one thread). The tile record {x0, y0, t_r,
// live} is written with a plain shared store before the arrival on the full
// barrier, whose release makes it visible to the waiting warps.
struct TileFetch {
    const ReplicaDesc* d;
    int x0, y0, tr, Ly, kind, rep;
    bool live, sampled;
};

// The global reads behind one tile (its code, then its replica's time and
// geometry): done one tile ahead of the issue, so their latency overlaps the
// producer's wait for the stage.
template <int TW, int NPT, int NW>
__device__ __forceinline__ TileFetch batch_fetch(const BatchArgs& a, unsigned step, int t) {
    using BS = BatchShape<TW, NPT, NW>;
    TileFetch f;
    const uint32_t code = __ldg(&a.tiles[t]);
    f.rep = (int)(code >> kLocalBits);
    f.d = a.desc + f.rep;
    const int local = (int)(code & kLocalMask);
    f.tr = __ldg(&f.d->hot.t0) + (int)(step - (unsigned)__ldg(&f.d->hot.join));
    const int tiles_x = __ldg(&f.d->hot.tiles_x);
    f.Ly = __ldg(&f.d->hot.Ly);
    f.live = f.tr < __ldg(&f.d->hot.tend);
    // the sampling schedule, decided once per tile here rather than by every
    // thread that reads the tile
    const int every = __ldg(&f.d->hot.every), warmup = __ldg(&f.d->hot.warmup);
    f.sampled = every > 0 && f.tr >= warmup && ((f.tr - warmup) % every) == 0;
    f.kind = 0;
    if (BS::MIXED) {
        const int kt0 = __ldg(&f.d->hot.kt0), kt01 = __ldg(&f.d->hot.kt01);
        if (local >= kt01) {
            f.kind = 2;
            f.x0 = __ldg(&f.d->hot.kx2);
            f.y0 = (local - kt01) * kind_th(2);
            return f;
        }
        if (local >= kt0) {
            f.kind = 1;
            f.x0 = __ldg(&f.d->hot.kx1);
            f.y0 = (local - kt0) * kind_th(1);
            return f;
        }
    }
    const int ty = local / tiles_x;
    f.x0 = (local - ty * tiles_x) * BS::TW;
    f.y0 = ty * BS::TH;
    return f;
}

template <int TW, int NPT, int NW>
__device__ __forceinline__ void batch_issue(float* smem, const TileFetch& f, int s, uint64_t* full) {
    using BS = BatchShape<TW, NPT, NW>;
    float* st = smem + s * BS::STAGE;
    // record: origin, replica time, and (0 for a tile not stepped) bit 0 set,
    // bit 1 sampled at this time, bits 2-3 the tile kind, bits 4.. the replica
    *reinterpret_cast<int4*>(st + 9 * BS::SPLANE + BS::HOT) =
        make_int4(f.x0, f.y0, f.tr, f.live ? 1 | (f.sampled ? 2 : 0) | (f.kind << 2) | (f.rep << 4) : 0);
    if (!f.live) {
        mbar_arrive(&full[s]);
        return;
    }
    const uint32_t box = BS::MIXED ? (uint32_t)(kind_th(f.kind) * kind_bw(f.kind)) : (uint32_t)(BS::TH * BS::BW);
    mbar_arrive_expect_tx(&full[s], 9u * box * sizeof(float) + sizeof(ReplicaHot));
    const CUtensorMap* map = &f.d->map[2 * f.kind + (f.tr & 1)];
#pragma unroll
    for (int i = 0; i < 9; ++i)
        tma_load_2d(st + i * BS::SPLANE, map, f.x0 + kXO - 4, i * (f.Ly + 2) + f.y0 + 1 - cvy(i),
                    &full[s]);
    bulk_load(st + 9 * BS::SPLANE, &f.d->hot, sizeof(ReplicaHot), &full[s]);
}

// Add a thread's Gram partials (gram_flush's fragment) straight to a
// replica's FP64 sums, scaled by s (first moments) and s^2 (second moments).
__device__ __forceinline__ void gram_flush_global(float (&c)[8], double* acc, double sc) {
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int row = g + ((k & 2) ? 8 : 0);
        const int col = 2 * q + (k & 1) + ((k & 4) ? 8 : 0);
        if (row < 9 && col == 9)
            atomicAdd(&acc[row], sc * (double)c[k]);
        else if (row <= col && col < 9)
            atomicAdd(&acc[9 + row * 9 - row * (row - 1) / 2 + (col - row)], sc * sc * (double)c[k]);
        c[k] = 0.f;
    }
}

// Warp roles: NW consumer warps, then one producer warp (SAMPLE = false, or
// the tensor-core sums) or kSamplers sampler warps whose first lane also
// produces (SAMPLE = true with 8 consumer warps).
template <int BASIS, bool SAMPLE, int TW, int NPT, int NWC = kBatchNW>
__global__ void __launch_bounds__((NWC + (SAMPLE && NWC == kBatchNW ? kSamplers : 1)) * 32, 1)
batch_step_kernel(const BatchArgs a) {
    using BS = BatchShape<TW, NPT, NWC>;
    constexpr int NW = NWC;
    constexpr bool kTensor = SAMPLE && BS::TENSOR;
    constexpr int BW = BS::BW;
    constexpr int TH = BS::TH;
    constexpr int S = BS::STAGES;
    constexpr int NX = SAMPLE && !kTensor ? kSamplers : 1;
    extern __shared__ __align__(128) float smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * BS::STAGE);
    uint64_t* empty = full + S;
    // tensor-core sums: per-run FP64 Gram matrices (16 x 16, rows and columns
    // 0..9 used), their replicas and scales, then the consumer warps' blocks
    double* run_cm = reinterpret_cast<double*>(empty + S + 2);
    double** run_acc = reinterpret_cast<double**>(run_cm + kRunSlots * 256);
    double* run_s = reinterpret_cast<double*>(run_acc + kRunSlots);
    // each consumer warp's current run: its replica's sums and scale
    double** cur_acc = reinterpret_cast<double**>(run_s + kRunSlots);
    double* cur_s = reinterpret_cast<double*>(cur_acc + NW);
    __half* gram = reinterpret_cast<__half*>(cur_s + NW);

    const int warp = threadIdx.x >> 5, lane_id = threadIdx.x & 31;
    const unsigned step = __ldcg(&a.ctl->step);
    const int ntiles = __ldcg(&a.ctl->ntiles);
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NW + (SAMPLE && !kTensor ? NX : 0));
        }
        fence_mbar_init();
    }
    if (kTensor) {
        for (int k = threadIdx.x; k < kRunSlots * 256; k += blockDim.x) run_cm[k] = 0.0;
        if (warp < NW) gram_init_full(gram + warp * kGramFullHalves);
    }
    __syncthreads();

    const int tbeg = (int)((long long)blockIdx.x * ntiles / gridDim.x);
    const int ntile = (int)((long long)(blockIdx.x + 1) * ntiles / gridDim.x) - tbeg;
    // the replica an error without a node belongs to
    auto first_err = [&]() { return a.desc[__ldg(&a.tiles[tbeg]) >> kLocalBits].hot.err; };

    if (warp >= NW) {
        const bool producer = warp == NW && lane_id == 0;
        int issued = 0, k = 0;
        bool ok = true;
        TileFetch nxt{};
        if (producer) {
            for (; issued < S && issued < ntile; ++issued)
                batch_issue<TW, NPT, NWC>(smem, batch_fetch<TW, NPT, NWC>(a, step, tbeg + issued), issued, full);
            if (issued < ntile) nxt = batch_fetch<TW, NPT, NWC>(a, step, tbeg + issued);
        }
        if (!SAMPLE || kTensor) {
            if (producer) {
                for (; k < ntile && issued < ntile; ++k) {
                    const int s = k % S;
                    if (!mbar_wait_sleep(&empty[s], (k / S) & 1)) {
                        ok = false;
                        break;
                    }
                    batch_issue<TW, NPT, NWC>(smem, nxt, s, full);
                    if (++issued < ntile) nxt = batch_fetch<TW, NPT, NWC>(a, step, tbeg + issued);
                }
                if (!ok) {
                    record_error(first_err(), kStatusTimeout, -1, step);
                    // let the copies still in flight land before the CTA exits
                    for (int j = issued > S ? issued - S : 0; j < issued; ++j)
                        if (!mbar_wait(&full[j % S], (j / S) & 1)) break;
                }
            }
            return;
        }
        // ---------------- samplers: warp sw takes rows sw, sw + kSamplers, ...
        const int sw = warp - NW;
        f2 s1[9], s2[45];
#pragma unroll
        for (int q = 0; q < 9; ++q) s1[q] = f2(0.f);
#pragma unroll
        for (int q = 0; q < 45; ++q) s2[q] = f2(0.f);
        double* run_acc = nullptr;   // replica whose sums the registers hold
        auto flush = [&]() {
            if (!run_acc) return;
#pragma unroll
            for (int q = 0; q < kSums; ++q) {
                f2& x2 = q < 9 ? s1[q] : s2[q - 9];
                float v = x2.v.x + x2.v.y;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane_id == 0) atomicAdd(&run_acc[q], (double)v);
                x2 = f2(0.f);
            }
            run_acc = nullptr;
        };
        for (; k < ntile && ok; ++k) {
            const int s = k % S, n = k / S;
            if (!mbar_wait_sleep(&full[s], n & 1)) {
                ok = false;
                break;
            }
            const float* stg = smem + s * BS::STAGE;
            const int4 info = *reinterpret_cast<const int4*>(stg + 9 * BS::SPLANE + BS::HOT);
            const ReplicaHot& h = *reinterpret_cast<const ReplicaHot*>(stg + 9 * BS::SPLANE);
            bool released = false;
            if (info.w & 2) {
                double* acc = h.acc;
                float ref[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) ref[i] = h.ref[i];
                const int Lx = h.Lx, Ly = h.Ly;
                if (run_acc != acc) flush();
                run_acc = acc;
                for (int row = sw; row < TH; row += kSamplers) {
                    const int y = info.y + row;
                    const float* st = stg + row * BW + 4 + lane_id;
#pragma unroll
                    for (int p = 0; p < BS::PAIRS; ++p) {
                        f2 d[9];
#pragma unroll
                        for (int i = 0; i < 9; ++i) {
                            const float* q = st + i * BS::SPLANE - cvx(i) + 64 * p;
                            d[i] = f2(q[0], q[32]);
                        }
                        if (row + kSamplers >= TH && p == BS::PAIRS - 1) {
                            // last read of the stage: release before the arithmetic
                            warp_arrive(&empty[s], lane_id);
                            released = true;
                        }
                        const int xA = info.x + lane_id + 64 * p;
                        const bool inA = xA < Lx && y < Ly, inB = xA + 32 < Lx && y < Ly;
#pragma unroll
                        for (int i = 0; i < 9; ++i) {
                            f2 e = d[i] - f2(ref[i]);
                            if (!(inA && inB)) e = f2(inA ? e.v.x : 0.f, inB ? e.v.y : 0.f);
                            d[i] = e;
                        }
                        int q = 0;
#pragma unroll
                        for (int i = 0; i < 9; ++i) {
                            s1[i] += d[i];
#pragma unroll
                            for (int j = i; j < 9; ++j, ++q) s2[q] = mad(d[i], d[j], s2[q]);
                        }
                    }
                }
            }
            if (!released) warp_arrive(&empty[s], lane_id);
            if (producer && issued < ntile) {
                if (!mbar_wait_sleep(&empty[s], n & 1)) {
                    ok = false;
                    break;
                }
                batch_issue<TW, NPT, NWC>(smem, nxt, s, full);
                if (++issued < ntile) nxt = batch_fetch<TW, NPT, NWC>(a, step, tbeg + issued);
            }
        }
        flush();
        if (!ok) {
            record_error(first_err(), kStatusTimeout, -1, step);
            if (producer)
                for (int j = k; j < issued; ++j)
                    if (!mbar_wait(&full[j % S], (j / S) & 1)) break;
        }
        return;
    }

    // ---------------- consumers
    const int c = threadIdx.x;
    const int ty = c / BS::RW, r = c % BS::RW;
    // tensor-core sums: this warp's FP32 partials belong to run `run` (the
    // run-th replica this CTA samples; every warp sees the same sequence)
    float gc[kTensor ? 8 : 1];
    if (kTensor) {
#pragma unroll
        for (int q = 0; q < 8; ++q) gc[q] = 0.f;
    }
    int run = -1, gtiles = 0, run_rep = -1;
    const int wc = c >> 5;
    const GramLane gl(kTensor ? smem_u32(gram + wc * kGramFullHalves) : 0u, 16);
    auto gram_out = [&]() {
        if (run < 0) return;
        if (run < kRunSlots)
            gram_flush(reinterpret_cast<float(&)[8]>(gc), run_cm + run * 256);
        else
            gram_flush_global(reinterpret_cast<float(&)[8]>(gc), cur_acc[wc], cur_s[wc]);
        gtiles = 0;
    };
    for (int k = 0; k < ntile; ++k) {
        const int s = k % S;
        if (!mbar_wait(&full[s], (k / S) & 1)) {
            record_error(first_err(), kStatusTimeout, -1, step);
            break;
        }
        const float* stg = smem + s * BS::STAGE;
        const int4 info = *reinterpret_cast<const int4*>(stg + 9 * BS::SPLANE + BS::HOT);
        if (!info.w) {
            warp_arrive(&empty[s], lane_id);
            continue;
        }
        const ReplicaHot& hs = *reinterpret_cast<const ReplicaHot*>(stg + 9 * BS::SPLANE);
        const uint32_t tr = (uint32_t)info.z;
        const int rep = info.w >> 4;
        if (NPT == 2) {
            const int Lx = hs.Lx, Ly = hs.Ly;
            // this thread's node pair: A at (ax, ay) of the tile, B at
            // (ax + dx, ay + dy); the tile is tw x th nodes in boxes bw wide
            int tw = BS::TW, th = BS::TH, bw = BW, ax = r, ay = ty, dx = BS::TW / 2, dy = 0;
            if constexpr (BS::MIXED) {
                // kind 0: two warps a row, each 64 columns wide; kind 1: a
                // warp a row; kind 2: a warp two rows. B lies 32 columns
                // right of A (kinds 0 and 1) or under it (kind 2).
                const int kind = (info.w >> 2) & 3, w = c >> 5;
                const bool vert = kind == 2;
                tw = kind_tw(kind);
                th = kind_th(kind);
                bw = tw + 8;
                ay = (w << 1) >> (2 - kind);
                ax = lane_id + (kind == 0 ? (w & 1) << 6 : 0);
                dx = vert ? 0 : 32;
                dy = vert ? 1 : 0;
            }
            const float* sa = stg + ay * bw + ax + 4;   // node A's cell in plane 0
            const int sb = dy * bw + dx;                // node B's offset from A
            auto load = [&](f2* g) {
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const float* p = sa + i * BS::SPLANE - cvx(i);
                    g[i] = f2(p[0], p[sb]);
                }
            };
            f2 g[9];
            load(g);
            const int xA = info.x + ax, yA = info.y + ay, xB = xA + dx, yB = yA + dy;
            const bool inA = xA < Lx && yA < Ly, inB = xB < Lx && yB < Ly;
            const uint32_t nodeA = (uint32_t)xA + (uint32_t)Lx * (uint32_t)yA;
            const uint32_t nodeB = (uint32_t)xB + (uint32_t)Lx * (uint32_t)yB;
            const bool smp = kTensor && (info.w & 2);
            if (smp && rep != run_rep) {   // a new run of sampled tiles
                gram_out();
                ++run;
                run_rep = rep;
                __syncwarp();   // every lane has flushed with the previous run's record
                if (lane_id == 0) {
                    const double sc = (double)hs.gram_s;
                    cur_acc[wc] = hs.acc;
                    cur_s[wc] = sc;
                    if (run < kRunSlots) {
                        run_acc[run] = hs.acc;
                        run_s[run] = sc;
                    }
                }
                __syncwarp();
            }
            // every node of the tile lies in the replica (a uniform test)
            const bool whole = info.x + tw <= Lx && info.y + th <= Ly;
            // stage the nodes when the collision reads them a second time
            auto stage = [&](const f2* gs) {
                f2 hv[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) hv[i] = mad(gs[i], f2(hs.sinv), f2(hs.snref[i]));
                if (!whole) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) hv[i] = f2(inA ? hv[i].v.x : 0.f, inB ? hv[i].v.y : 0.f);
                }
                gram_stage(gl, hv);
            };
            auto refetch = [&](f2* gg) {
                load(gg);
                if (kTensor && smp) stage(gg);
            };
            f2 f[9];
            const uint32_t stt = collide_basis<f2, BASIS>(
                g, PairNoise{hs.cc.key, nodeA, nodeB, tr}, refetch, a.lut, hs.pc, f);
            if (kTensor && smp) {
                gram_mma(gl, reinterpret_cast<float(&)[8]>(gc));
                if (++gtiles == kGramFlushTiles) gram_out();
            }
            // what the stores need, read before the stage is released
            Geometry geo;
            geo.Lx = Lx;
            geo.Ly = Ly;
            geo.pitch = hs.pitch;
            geo.plane = hs.plane;
            float* dst = hs.buf[(tr + 1u) & 1u];
            warp_arrive(&empty[s], lane_id);
            if (stt) {
                DevError* err = a.desc[rep].hot.err;
                if (inA && (stt & 0xFF)) record_error(err, (int)(stt & 0xFF), nodeA, tr);
                if (inB && (stt >> 8)) record_error(err, (int)(stt >> 8), nodeB, tr);
            }
            // an inner tile stores without edge tests; on an edge tile each lane
            // tests its node and adds the ghost copies it needs
            const bool inner = info.x > 0 && info.y > 0 && info.x + tw < geo.Lx && info.y + th < geo.Ly;
            float* pa = dst + at(geo, 0, xA, yA);
            const long long gb = dy * geo.pitch + dx;   // B's offset from A
            if (inner) {
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    pa[i * geo.plane] = f[i].v.x;
                    pa[i * geo.plane + gb] = f[i].v.y;
                }
            } else {
                if (inA) store_lane_ghosts(pa, geo, xA, yA, f, 0);
                if (inB) store_lane_ghosts(pa + gb, geo, xB, yB, f, 1);
            }
        } else {
            Geometry geo;
            geo.Lx = hs.Lx;
            geo.Ly = hs.Ly;
            geo.pitch = hs.pitch;
            geo.plane = hs.plane;
            float* dst = hs.buf[(tr + 1u) & 1u];
            DevError* err = hs.err;
            const int y = info.y + ty;
            const float* st = stg + ty * BW + 4 + r;
            auto load = [&](float* g) {
#pragma unroll
                for (int i = 0; i < 9; ++i) g[i] = st[i * BS::SPLANE - cvx(i)];
            };
            float g[9];
            load(g);
            const int x = info.x + r;
            const bool in = x < geo.Lx && y < geo.Ly;
            const uint32_t node = (uint32_t)x + (uint32_t)geo.Lx * (uint32_t)y;
            float f[9];
            const uint32_t stt = collide_basis<float, BASIS>(
                g, NodeNoise{hs.cc.key, node, tr}, load, a.lut, hs.cc, f);
            warp_arrive(&empty[s], lane_id);
            if (in) {
                if (stt & 0xFF) record_error(err, (int)(stt & 0xFF), node, tr);
                store_node(dst, geo, x, y, f);
            }
        }
    }
    if (kTensor) {
        gram_out();
        named_sync(1, NW * 32);
        const int nrun = run + 1 < kRunSlots ? run + 1 : kRunSlots;
        for (int k = c; k < nrun * kSums; k += NW * 32) {
            const int j = k / kSums, q = k - j * kSums;
            atomicAdd(&run_acc[j][q], gram_sum(run_cm + j * 256, q, run_s[j]));
        }
    }
    // the last CTA to finish advances the batch step (every CTA read it at its start)
    if (c == 0) {
        __threadfence();
        if (atomicAdd(&a.ctl->ticket, 1u) == gridDim.x - 1) {
            a.ctl->step = step + 1u;
            a.ctl->ticket = 0u;
        }
    }
}

// Tile shapes the batch can run; index = FLB_TILE_* of flb.h. Shapes with 12
// consumer warps take their correlation sums on the tensor cores.
struct BatchVariant {
    int tw, npt, nw;   // tw = kMixedTW: the mixed tiling
    __host__ __device__ constexpr bool mixed() const { return tw == kMixedTW; }
    __host__ __device__ constexpr int th() const { return mixed() ? kind_th(0) : nw * 32 * npt / tw; }
    __host__ __device__ constexpr bool tensor() const { return nw > kBatchNW; }
};
constexpr BatchVariant kBatchVariants[6] = {{128, 2, kBatchNW},       {64, 2, kBatchNW},
                                            {128, 1, kBatchNW},       {128, 2, kBatchNWTensor},
                                            {64, 2, kBatchNWTensor},  {kMixedTW, 2, kBatchNWTensor}};
constexpr int kNumBatchVariants = 6;

// Kernel of (variant, basis, sampling), instantiated in flb_batch_k<basis>.cu.
const void* batch_kernel_std(int variant, bool sample);
const void* batch_kernel_loc(int variant, bool sample);
const void* batch_kernel_lut(int variant, bool sample);
size_t batch_smem_bytes(int variant);

}  // namespace flb
