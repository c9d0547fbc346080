// flb_step_tma.cu -- the pipelined FP32 fused step for sm_103a.
//
// Persistent CTAs walk the lattice in tiles of 128 x TH nodes (TH = NW / 2).
// One producer warp streams, for every tile and every plane i, the box of
// 136 x TH populations that the pull g_i(x) = f*_i(x - v_i) of the tile needs
// (shifted by v_iy rows; 4 extra columns on each side cover v_ix = +-1) from
// HBM into a ring of shared-memory stages with 2D TMA copies, signalling
// mbarriers. NW consumer warps take two nodes per thread -- node A at tile
// column r, node B at r + 64 -- read their nine shifted populations from shared
// memory, release the stage, and collide both nodes at once in packed FP32x2
// arithmetic (flb_collide.cuh with V = f2). Stores go straight to HBM, rows
// coalesced, with the ghost copies of boundary nodes (flb_layout.cuh).
//
// With sampling on, TH sampler warps (one per tile row) read the same stage and
// accumulate the 9 + 45 correlation sums in packed FP32x2 registers while the
// consumers collide; the first sampler lane also issues the TMA loads. At the
// end the CTA reduces the sums to FP64 partials and the last CTA to finish adds
// all partials, in CTA order, to the running sums: deterministic, with no
// separate reduction launch.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>

#include "flb_collide.cuh"
#include "flb_internal.h"
#include "flb_tma.cuh"

namespace flb {

constexpr int kTW = 128;               // tile width (nodes)
constexpr int kBoxW = kTW + 8;         // TMA box width: x0 - 4 .. x0 + 131
constexpr int kStages = 4;
constexpr int kDefaultNW = 8;

template <int NW>
struct TileShape {
    static constexpr int TH = NW / 2;                                  // rows per tile
    static constexpr int SPLANE = (TH * kBoxW + 31) / 32 * 32;         // floats per plane box
    static constexpr int STAGE = 9 * SPLANE;                           // floats per stage
    static constexpr size_t smem_bytes() {
        return sizeof(float) * (size_t)kStages * STAGE + 2 * kStages * sizeof(uint64_t) +
               sizeof(double) * TH * kSums + 16;
    }
};

__device__ __forceinline__ void store_lane(const TmaArgs& a, int x, int y, const f2 f[9], int k) {
    float v[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) v[i] = lane(f[i], k);
    store_node(a.dst, a.geo, x, y, v);
}

// Issue the nine TMA box loads of tile t into stage s (one thread).
template <int NW>
__device__ __forceinline__ void issue_tile(float* smem, const CUtensorMap* map, const TmaArgs& a,
                                           int t, int s, uint64_t* full) {
    using TS = TileShape<NW>;
    mbar_arrive_expect_tx(&full[s], 9u * TS::TH * kBoxW * sizeof(float));
    const int x0 = (t % a.tiles_x) * kTW, y0 = (t / a.tiles_x) * TS::TH;
    float* st = smem + s * TS::STAGE;
#pragma unroll
    for (int i = 0; i < 9; ++i)
        tma_load_2d(st + i * TS::SPLANE, map, x0 + kXO - 4,
                    i * (a.geo.Ly + 2) + y0 + 1 - cvy(i), &full[s]);
}

// Warp roles: warps [0, NW) collide (consumers); warps [NW, NW + NS) are the
// producer (NS = 1, no sampling) or, with sampling, NS = TH sampler warps --
// sampler w accumulates the correlation sums of row w of every tile -- whose
// first lane is also the producer.
template <int BASIS, bool SAMPLE, int NW>
__global__ void __launch_bounds__((NW + (SAMPLE ? NW / 2 : 1)) * 32, 1)
step_tma_kernel(const __grid_constant__ CUtensorMap map, const TmaArgs a,
                const CollideConst<float> cc) {
    using TS = TileShape<NW>;
    constexpr int TH = TS::TH;
    constexpr int NS = SAMPLE ? TH : 1;
    extern __shared__ __align__(128) float smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * TS::STAGE);
    uint64_t* empty = full + kStages;
    double* red = reinterpret_cast<double*>(empty + kStages);
    int* flag = reinterpret_cast<int*>(red + TH * kSums);

    const int warp = threadIdx.x >> 5, lane_id = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NW + (SAMPLE ? NS : 0));
        }
        fence_mbar_init();
    }
    __syncthreads();

    const int Lx = a.geo.Lx, Ly = a.geo.Ly;

    if (!SAMPLE && warp == NW) {
        // ---------------- producer warp
        if (lane_id == 0) {
            prefetch_tensormap(&map);
            int k = 0;
            for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++k) {
                const int s = k % kStages, n = k / kStages;
                if (n > 0 && !mbar_wait(&empty[s], (n - 1) & 1)) {
                    record_error(a.err, kStatusTimeout, -1, a.step);
                    break;
                }
                issue_tile<NW>(smem, &map, a, t, s, full);
            }
            // no copy may still be in flight when the CTA exits
            for (int j = k > kStages ? k - kStages : 0; j < k; ++j)
                if (!mbar_wait(&full[j % kStages], (j / kStages) & 1)) {
                    record_error(a.err, kStatusTimeout, -1, a.step);
                    break;
                }
        }
        return;
    }

    if (SAMPLE && warp >= NW) {
        // ---------------- samplers (first lane of the first one also produces)
        const int row = warp - NW;
        const bool producer = row == 0 && lane_id == 0;
        int issued = 0;
        bool ok = true;
        if (producer) {
            prefetch_tensormap(&map);
            for (int t = blockIdx.x; t < a.ntiles && issued < kStages; t += gridDim.x, ++issued)
                issue_tile<NW>(smem, &map, a, t, issued, full);
        }
        f2 s1[9], s2[45];
#pragma unroll
        for (int q = 0; q < 9; ++q) s1[q] = f2(0.f);
#pragma unroll
        for (int q = 0; q < 45; ++q) s2[q] = f2(0.f);
        int k = 0;
        for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++k) {
            const int s = k % kStages, n = k / kStages;
            if (!mbar_wait(&full[s], n & 1)) {
                record_error(a.err, kStatusTimeout, -1, a.step);
                ok = false;
                break;
            }
            const int x0 = (t % a.tiles_x) * kTW, y = (t / a.tiles_x) * TH + row;
            const float* st = smem + s * TS::STAGE + row * kBoxW + 4 + lane_id;
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const int xA = x0 + lane_id + 64 * p;
                const bool inA = xA < Lx && y < Ly, inB = xA + 32 < Lx && y < Ly;
                f2 d[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const float* q = st + i * TS::SPLANE - cvx(i) + 64 * p;
                    d[i] = f2(q[0], q[32]) - f2(a.ref[i]);
                }
                if (!(inA && inB)) {
#pragma unroll
                    for (int i = 0; i < 9; ++i)
                        d[i] = f2(inA ? d[i].v.x : 0.f, inB ? d[i].v.y : 0.f);
                }
                int q = 0;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    s1[i] += d[i];
#pragma unroll
                    for (int j = i; j < 9; ++j, ++q) s2[q] = mad(d[i], d[j], s2[q]);
                }
            }
            __syncwarp();
            if (lane_id == 0) mbar_arrive(&empty[s]);
            if (producer && ok) {
                // refill this stage with the tile kStages ahead once every warp released it
                const int tn = blockIdx.x + issued * gridDim.x;
                if (tn < a.ntiles) {
                    if (!mbar_wait(&empty[s], n & 1)) {
                        record_error(a.err, kStatusTimeout, -1, a.step);
                        ok = false;
                    } else {
                        issue_tile<NW>(smem, &map, a, tn, s, full);
                        ++issued;
                    }
                }
            }
        }
        if (producer)   // no copy may still be in flight when the CTA exits
            for (int j = issued > kStages ? issued - kStages : 0; j < issued; ++j)
                if (j >= k && !mbar_wait(&full[j % kStages], (j / kStages) & 1)) {
                    record_error(a.err, kStatusTimeout, -1, a.step);
                    break;
                }

        // CTA reduction: lanes (warp shuffles), then samplers in FP64
#pragma unroll
        for (int q = 0; q < kSums; ++q) {
            const f2 v2 = q < 9 ? s1[q] : s2[q - 9];
            float v = v2.v.x + v2.v.y;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane_id == 0) red[row * kSums + q] = (double)v;
        }
        const int c = threadIdx.x - NW * 32;   // 0 .. 32 NS - 1
        named_sync(1, NS * 32);
        if (c < kSums) {
            double tot = 0.0;
            for (int w = 0; w < NS; ++w) tot += red[w * kSums + c];
            a.partials[(size_t)blockIdx.x * kSums + c] = tot;
        }
        // grid: the last CTA to finish adds every CTA's partial, in CTA order
        __threadfence();
        named_sync(1, NS * 32);
        if (c == 0) *flag = (atomicAdd(a.ticket, 1u) == gridDim.x - 1) ? 1 : 0;
        named_sync(1, NS * 32);
        if (*flag) {
            __threadfence();
            if (c < kSums) {
                double tot = 0.0;
                for (unsigned b = 0; b < gridDim.x; ++b)
                    tot += __ldcg(&a.partials[(size_t)b * kSums + c]);
                a.acc[c] += tot;
            }
            if (c == 0) *a.ticket = 0u;
        }
        return;
    }

    // ---------------- consumers: two nodes per thread, packed FP32x2
    const int c = threadIdx.x;          // 0 .. 32 NW - 1
    const int ty = c >> 6, r = c & 63;
    int k = 0;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++k) {
        const int s = k % kStages, n = k / kStages;
        if (!mbar_wait(&full[s], n & 1)) {
            record_error(a.err, kStatusTimeout, -1, a.step);
            break;
        }
        const float* st = smem + s * TS::STAGE + ty * kBoxW + 4 + r;
        f2 g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const float* p = st + i * TS::SPLANE - cvx(i);
            g[i] = f2(p[0], p[64]);
        }
        __syncwarp();
        if (lane_id == 0) mbar_arrive(&empty[s]);

        const int x0 = (t % a.tiles_x) * kTW, y = (t / a.tiles_x) * TH + ty;
        const int xA = x0 + r, xB = xA + 64;
        const bool inA = xA < Lx && y < Ly, inB = xB < Lx && y < Ly;
        const uint32_t nodeA = (uint32_t)xA + (uint32_t)Lx * (uint32_t)y;
        f2 f[9];
        const uint32_t stt = collide<f2, BASIS>(
            g, [&](f2* N) { node_normals(cc.key, nodeA, nodeA + 64u, a.step, N); }, cc, f);
        if (inA) {
            if (stt & 0xFF) record_error(a.err, (int)(stt & 0xFF), nodeA, a.step);
            store_lane(a, xA, y, f, 0);
        }
        if (inB) {
            if (stt >> 8) record_error(a.err, (int)(stt >> 8), nodeA + 64u, a.step);
            store_lane(a, xB, y, f, 1);
        }
    }
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

template <int NW>
const void* kernel_ptr(int basis, bool sample) {
    if (basis == 0)
        return sample ? (const void*)step_tma_kernel<0, true, NW>
                      : (const void*)step_tma_kernel<0, false, NW>;
    return sample ? (const void*)step_tma_kernel<1, true, NW>
                  : (const void*)step_tma_kernel<1, false, NW>;
}

const void* kernel_for(int nw, int basis, bool sample) {
    switch (nw) {
        case 4: return kernel_ptr<4>(basis, sample);
        case 8: return kernel_ptr<8>(basis, sample);
        default: return nullptr;
    }
}

size_t smem_for(int nw) {
    switch (nw) {
        case 4: return TileShape<4>::smem_bytes();
        case 8: return TileShape<8>::smem_bytes();
        default: return 0;
    }
}

}  // namespace

int tma_max_grid(int sms) { return sms * 2; }

cudaError_t tma_plan(TmaPlan* plan, void* buf0, void* buf1, const Geometry& g, int nw) {
    plan->ready = false;
    if (nw == 0) nw = kDefaultNW;
    if (!kernel_for(nw, 0, false)) return cudaErrorInvalidValue;
    EncodeFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const int th = nw / 2;
    const cuuint64_t dims[2] = {(cuuint64_t)g.pitch, (cuuint64_t)(9 * (long long)(g.Ly + 2))};
    const cuuint64_t strides[1] = {(cuuint64_t)g.pitch * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)kBoxW, (cuuint32_t)th};
    const cuuint32_t estr[2] = {1, 1};
    void* bufs[2] = {buf0, buf1};
    for (int b = 0; b < 2; ++b) {
        const CUresult rc = enc(&plan->map[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, bufs[b], dims,
                                strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (rc != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    const size_t smem = smem_for(nw);
    int dev = 0, sms = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int basis = 0; basis < 2 && ce == cudaSuccess; ++basis)
        for (int sample = 0; sample < 2 && ce == cudaSuccess; ++sample)
            ce = cudaFuncSetAttribute(kernel_for(nw, basis, sample != 0),
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (ce == cudaSuccess)
        ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel_for(nw, 1, true),
                                                           (nw + nw / 2) * 32, smem);
    if (ce != cudaSuccess) return ce;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (per_sm > 2) per_sm = 2;
    plan->nw = nw;
    plan->smem = smem;
    plan->tiles_x = (g.Lx + kTW - 1) / kTW;
    plan->ntiles = plan->tiles_x * ((g.Ly + th - 1) / th);
    int grid = sms * per_sm;
    if (grid > plan->ntiles) grid = plan->ntiles;
    plan->grid = grid < 1 ? 1 : grid;
    plan->ready = true;
    return cudaSuccess;
}

cudaError_t tma_step(const TmaPlan& plan, int src, const TmaArgs& a,
                     const CollideConst<float>& cc, int basis, bool sample, cudaStream_t s) {
    const void* fn = kernel_for(plan.nw, basis, sample);
    if (!fn || !plan.ready) return cudaErrorInvalidValue;
    TmaArgs args = a;
    args.tiles_x = plan.tiles_x;
    args.ntiles = plan.ntiles;
    void* params[3] = {(void*)&plan.map[src], (void*)&args, (void*)&cc};
    const int warps = plan.nw + (sample ? plan.nw / 2 : 1);
    return cudaLaunchKernel(fn, dim3(plan.grid), dim3(warps * 32), params, plan.smem, s);
}

}  // namespace flb
