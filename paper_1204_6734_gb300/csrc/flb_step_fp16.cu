// flb_step_fp16.cu -- the pipelined fused step with the FP16 deviation store.
//
// The state is kept as h_i = (f_i - c_i) / sqrt(kT) in FP16, with c = f^0(rho0,
// u0) in FP32: the thermal deviations are O(sqrt(kT f^0)), so h is O(1) and
// FP16's 11-bit significand resolves it to about 2.4e-4 of a standard
// deviation. A buffer then holds 18 bytes per node instead of 36 (36 bytes per
// node and step moved instead of 72). The collision itself is the FP32 one of
// flb_collide.cuh: each node decodes f = c + sqrt(kT) h, collides in packed
// FP32x2, and encodes h* = (f* - c) / sqrt(kT) with round-to-nearest.
//
// Structure as in flb_step_tma.cu: persistent CTAs, 128 x 4 tiles, 2D TMA
// boxes into a ring of shared-memory stages, 8 colliding warps with two nodes
// per thread, and on sampling steps 4 sampler warps (one tile row each) whose
// first lane also produces. Boxes start 8 columns left of the tile (a TMA box
// of 16-bit elements must start at a multiple of 8 elements) and are 144 wide.
// The samplers accumulate h_i and h_i h_j directly (h is already the
// deviation from c) and scale by sqrt(kT) and kT when they publish.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "flb_collide.cuh"
#include "flb_internal.h"
#include "flb_pipeline.cuh"
#include "flb_tma.cuh"

namespace flb {

namespace {

constexpr int kHBoxW = kTW + 16;   // x0 - 8 .. x0 + 135
constexpr int kHOff = 8;           // column of x0 in a box
constexpr int kHNW = 8;            // colliding warps
constexpr int kHTH = kHNW / 2;     // rows per tile

struct HShape {
    static constexpr int SPLANE = kHTH * kHBoxW;   // halves per plane box (1152 B)
    static constexpr int STAGE = 9 * SPLANE;      // halves per stage (10368 B)
    static constexpr int STAGES = 16;
    static constexpr size_t smem_bytes() {
        return sizeof(__half) * (size_t)STAGES * STAGE + 2 * STAGES * sizeof(uint64_t) +
               sizeof(double) * kSamplers * kSums;
    }
};
static_assert((HShape::SPLANE * sizeof(__half)) % 128 == 0, "plane boxes stay 128-byte aligned");

__device__ __forceinline__ void issue_tile16(__half* smem, const CUtensorMap* map, const HArgs& a,
                                             int t, int s, uint64_t* full) {
    mbar_arrive_expect_tx(&full[s], 9u * kHTH * kHBoxW * sizeof(__half));
    const int x0 = (t % a.tiles_x) * kTW, y0 = (t / a.tiles_x) * kHTH;
    __half* st = smem + s * HShape::STAGE;
#pragma unroll
    for (int i = 0; i < 9; ++i)
        tma_load_2d(st + i * HShape::SPLANE, map, x0 + kXO - kHOff,
                    i * (a.geo.Ly + 2) + y0 + 1 - cvy(i), &full[s]);
}

// The elected producer thread (as in flb_step_tma.cu).
struct Producer16 {
    int issued = 0;
    bool ok = true;

    __device__ __forceinline__ void prologue(__half* smem, const CUtensorMap* map, const HArgs& a,
                                             uint64_t* full) {
        prefetch_tensormap(map);
        for (int t = blockIdx.x; t < a.ntiles && issued < HShape::STAGES; t += gridDim.x, ++issued)
            issue_tile16(smem, map, a, t, issued, full);
    }
    __device__ __forceinline__ void refill(__half* smem, const CUtensorMap* map, const HArgs& a,
                                           uint64_t* full, uint64_t* empty, int s, int n) {
        if (!ok) return;
        const int tn = blockIdx.x + issued * gridDim.x;
        if (tn >= a.ntiles) return;
        if (!mbar_wait_sleep(&empty[s], n & 1)) {
            record_error(a.err, kStatusTimeout, -1, a.step);
            ok = false;
            return;
        }
        issue_tile16(smem, map, a, tn, s, full);
        ++issued;
    }
    __device__ __forceinline__ void drain(const HArgs& a, uint64_t* full, int consumed) {
        constexpr int S = HShape::STAGES;
        for (int j = issued > S ? issued - S : 0; j < issued; ++j)
            if (j >= consumed && !mbar_wait(&full[j % S], (j / S) & 1)) {
                record_error(a.err, kStatusTimeout, -1, a.step);
                break;
            }
    }
};

__device__ __forceinline__ f2 h2f(const __half* p, int off) {
    return f2(__half2float(p[0]), __half2float(p[off]));
}

template <int BASIS, bool SAMPLE>
__global__ void __launch_bounds__((kHNW + (SAMPLE ? kSamplers : 1)) * 32, 1)
step_fp16_kernel(const __grid_constant__ CUtensorMap map, const HArgs a,
                 const CollideConst<float> cc) {
    constexpr int S = HShape::STAGES;
    constexpr int NW = kHNW, TH = kHTH;
    constexpr int NX = SAMPLE ? kSamplers : 1;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __half* smem = reinterpret_cast<__half*>(smem_raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * HShape::STAGE);
    uint64_t* empty = full + S;
    double* red = reinterpret_cast<double*>(empty + S);

    const int warp = threadIdx.x >> 5, lane_id = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NW + (SAMPLE ? NX : 0));
        }
        fence_mbar_init();
    }
    __syncthreads();
    const int Lx = a.geo.Lx, Ly = a.geo.Ly;

    if (!SAMPLE && warp == NW) {
        // ---------------- producer warp
        if (lane_id == 0) {
            Producer16 prod;
            prod.prologue(smem, &map, a, full);
            int k = 0;
            for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++k)
                prod.refill(smem, &map, a, full, empty, k % S, k / S);
            prod.drain(a, full, prod.issued);
        }
        return;
    }

    if (SAMPLE && warp >= NW) {
        // ---------------- sampler warps: sums of h_i and h_i h_j, scaled at the end
        const int sw = warp - NW;
        const bool producer = sw == 0 && lane_id == 0;
        Producer16 prod;
        if (producer) prod.prologue(smem, &map, a, full);
        f2 s1[9], s2[45];
#pragma unroll
        for (int q = 0; q < 9; ++q) s1[q] = f2(0.f);
#pragma unroll
        for (int q = 0; q < 45; ++q) s2[q] = f2(0.f);
        int k = 0;
        for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++k) {
            const int s = k % S, n = k / S;
            if (!mbar_wait_sleep(&full[s], n & 1)) {
                record_error(a.err, kStatusTimeout, -1, a.step);
                break;
            }
            const int x0 = (t % a.tiles_x) * kTW;
            for (int row = sw; row < TH; row += NX) {
                const int y = (t / a.tiles_x) * TH + row;
                const __half* st = smem + s * HShape::STAGE + row * kHBoxW + kHOff + lane_id;
                f2 d[2][9];
#pragma unroll
                for (int p = 0; p < 2; ++p)
#pragma unroll
                    for (int i = 0; i < 9; ++i) d[p][i] = h2f(st + i * HShape::SPLANE - cvx(i) + 64 * p, 32);
                if (row + NX >= TH) {   // last row: release before the arithmetic
                    __syncwarp();
                    if (lane_id == 0) mbar_arrive(&empty[s]);
                }
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const int xA = x0 + lane_id + 64 * p;
                    const bool inA = xA < Lx && y < Ly, inB = xA + 32 < Lx && y < Ly;
                    if (!(inA && inB)) {
#pragma unroll
                        for (int i = 0; i < 9; ++i)
                            d[p][i] = f2(inA ? d[p][i].v.x : 0.f, inB ? d[p][i].v.y : 0.f);
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
            if (sw >= TH) {
                __syncwarp();
                if (lane_id == 0) mbar_arrive(&empty[s]);
            }
            if (producer) prod.refill(smem, &map, a, full, empty, s, n);
        }
        if (producer) prod.drain(a, full, k);
        float v[kSums];
#pragma unroll
        for (int q = 0; q < kSums; ++q) {
            const f2 x = q < 9 ? s1[q] : s2[q - 9];
            v[q] = (x.v.x + x.v.y) * (q < 9 ? a.scale : a.scale * a.scale);
        }
        TmaArgs pa;
        pa.acc = a.acc;
        publish_sums(v, NW, NX * 32, red, pa);
        return;
    }

    // ---------------- colliding warps: decode, collide in FP32x2, encode
    const int c = threadIdx.x;
    const int ty = c >> 6, r = c & 63;
    int k = 0;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++k) {
        const int s = k % S, n = k / S;
        if (!mbar_wait(&full[s], n & 1)) {
            record_error(a.err, kStatusTimeout, -1, a.step);
            break;
        }
        const __half* st = smem + s * HShape::STAGE + ty * kHBoxW + kHOff + r;
        auto load = [&](f2* g) {
#pragma unroll
            for (int i = 0; i < 9; ++i)
                g[i] = mad(h2f(st + i * HShape::SPLANE - cvx(i), 64), f2(a.scale), f2(a.ref[i]));
        };
        f2 g[9];
        load(g);
        const int x0 = (t % a.tiles_x) * kTW, y = (t / a.tiles_x) * TH + ty;
        const int xA = x0 + r, xB = xA + 64;
        const bool inA = xA < Lx && y < Ly, inB = xB < Lx && y < Ly;
        const uint32_t nodeA = a.node0 + (uint32_t)xA + (uint32_t)Lx * (uint32_t)y;
        f2 f[9];
        const uint32_t stt = collide_basis<f2, BASIS>(
            g, PairNoise{cc.key, nodeA, nodeA + 64u, a.step}, load, a.lut, cc, f);
        __syncwarp();
        if (lane_id == 0) mbar_arrive(&empty[s]);
        if (stt) {
            if (inA && (stt & 0xFF)) record_error(a.err, (int)(stt & 0xFF), nodeA, a.step);
            if (inB && (stt >> 8)) record_error(a.err, (int)(stt >> 8), nodeA + 64u, a.step);
        }
        // h* = (f* - c) / sqrt(kT) = f* inv_scale + nref
        __half hA[9], hB[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const f2 h = mad(f[i], f2(a.inv_scale), f2(a.nref[i]));
            hA[i] = __float2half_rn(h.v.x);
            hB[i] = __float2half_rn(h.v.y);
        }
        __half* pa = a.dst + at(a.geo, 0, xA, y);
        if (x0 > 0 && y - ty > 0 && x0 + kTW < Lx && y - ty + TH < Ly) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                pa[i * a.geo.plane] = hA[i];
                pa[i * a.geo.plane + 64] = hB[i];
            }
        } else {
            if (inA) store_node_ghosts(pa, a.geo, xA, y, hA);
            if (inB) store_node_ghosts(pa + 64, a.geo, xB, y, hB);
        }
    }
}

const void* fp16_kernel(int basis, bool sample) {
    if (basis == 0) return sample ? (const void*)step_fp16_kernel<0, true> : (const void*)step_fp16_kernel<0, false>;
    if (basis == 1) return sample ? (const void*)step_fp16_kernel<1, true> : (const void*)step_fp16_kernel<1, false>;
    return sample ? (const void*)step_fp16_kernel<2, true> : (const void*)step_fp16_kernel<2, false>;
}

}  // namespace

cudaError_t fp16_plan(TmaPlan* plan, void* buf0, void* buf1, const Geometry& g) {
    plan->ready = false;
    void* bufs[2] = {buf0, buf1};
    for (int b = 0; b < 2; ++b) {
        const cudaError_t e = tma_encode_planes(&plan->map[b], bufs[b], g, kHBoxW, kHTH, 2);
        if (e != cudaSuccess) return e;
    }
    const size_t smem = HShape::smem_bytes();
    int dev = 0, sms = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int basis = 0; basis < 3 && ce == cudaSuccess; ++basis)
        for (int smp = 0; smp < 2 && ce == cudaSuccess; ++smp)
            ce = cudaFuncSetAttribute(fp16_kernel(basis, smp),
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ce != cudaSuccess) return ce;
    plan->nw = kHNW;
    plan->smem = smem;
    plan->tiles_x = (g.Lx + kTW - 1) / kTW;
    plan->ntiles = plan->tiles_x * ((g.Ly + kHTH - 1) / kHTH);
    plan->grid = sms < plan->ntiles ? sms : plan->ntiles;
    if (plan->grid < 1) plan->grid = 1;
    plan->ready = true;
    return cudaSuccess;
}

cudaError_t fp16_step(const TmaPlan& plan, int src, const HArgs& a, const CollideConst<float>& cc,
                      int basis, bool sample, cudaStream_t s) {
    if (!plan.ready) return cudaErrorInvalidValue;
    HArgs args = a;
    args.tiles_x = plan.tiles_x;
    args.ntiles = plan.ntiles;
    void* params[3] = {(void*)&plan.map[src], (void*)&args, (void*)&cc};
    return cudaLaunchKernel(fp16_kernel(basis, sample), dim3(plan.grid),
                            dim3((kHNW + (sample ? kSamplers : 1)) * 32), params, plan.smem, s);
}

}  // namespace flb
