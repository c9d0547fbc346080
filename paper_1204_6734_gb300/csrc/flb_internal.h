// flb_internal.h -- interface between the C-ABI translation unit and the
// pipelined FP32 step kernel (flb_step_tma.cu).
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "flb_kernels.cuh"

namespace flb {

struct TmaArgs {
    float* dst;             // buffer receiving f*(t)
    Geometry geo;
    uint32_t step;
    uint32_t node0;         // noise counter of node (0, 0) (slabs: Lx y0)
    int tiles_x, ntiles;    // 128 x TH tiles of the lattice
    double* acc;            // running FP64 sums (sampling)
    DevError* err;
    const float* lut;       // velocity table (look-up-table f-norm only)
    float ref[9];           // f^0(rho0, u0) subtracted before sampling
    // tensor-core sampling: nodes are staged as h = (f - ref) / s in FP16
    float sinv;             // 1 / s
    float snref[9];         // -ref / s
    double s;               // s (the sums are rescaled in FP64)
    // structure-factor sampling of this step's pre-collision state: the fields
    // drho, dj_x, dj_y of every node into fields[f Lx Ly + y Lx + x] (nullptr: none)
    float* fields;
};

constexpr int kPlanTensorSampling = 3;   // TmaPlan::sample_mode of the tensor-core sums
constexpr int kTensorNW = 12;            // colliding warps of the tensor-sampling plan

struct TmaPlan {
    CUtensorMap map[2];     // source tensor maps of buffer 0 and buffer 1
    int nw;                 // consumer warps per CTA (tile = 128 x nw/2 nodes)
    int grid;               // persistent CTAs
    size_t smem;            // dynamic shared memory per CTA
    int tiles_x, ntiles;
    int sample_mode;        // sampling steps: 1 sampler warps, 2 fused into the consumers,
                            // 3 tensor-core Gram sums in the consumers
    bool ready;
};

// Encode the tensor maps and choose the launch shape for a lattice whose two
// population buffers are buf0 and buf1. nw = 0 picks the default. Returns
// cudaSuccess or the error that prevents the pipelined kernel.
cudaError_t tma_plan(TmaPlan* plan, void* buf0, void* buf1, const Geometry& g, int nw);

// Tensor map of the nine planes of one buffer (ghost-frame layout), seen as
// one 2D array of pitch x 9 (Ly + 2) elements of elem_bytes (4: FP32, 2: FP16),
// for boxes of box_w x th.
cudaError_t tma_encode_planes(CUtensorMap* map, void* buf, const Geometry& g, int box_w, int th,
                              int elem_bytes = 4);

// Arguments of the FP16-deviation-store step (flb_step_fp16.cu): the buffer
// holds h = (f - ref) / scale in FP16, scale = sqrt(kT).
struct HArgs {
    __half* dst;            // buffer receiving h*(t)
    Geometry geo;
    uint32_t step;
    uint32_t node0;         // noise counter of node (0, 0) (slabs: Lx y0)
    int tiles_x, ntiles;
    double* acc;            // running FP64 sums of f - ref (sampling)
    DevError* err;
    float ref[9];           // f^0(rho0, u0)
    float nref[9];          // -ref / scale
    float scale, inv_scale;
    const float* lut;       // velocity table (look-up-table f-norm only)
};

// One warp waits on an mbarrier nothing completes, for at most `limit` cycles
// (<= the kernels' own bound), and records the timeout in err.
cudaError_t wait_probe(long long limit, DevError* err, cudaStream_t s);

// Tensor maps and launch shape of the FP16-store kernel; one step of it.
cudaError_t fp16_plan(TmaPlan* plan, void* buf0, void* buf1, const Geometry& g);
cudaError_t fp16_step(const TmaPlan& plan, int src, const HArgs& a, const CollideConst<float>& cc,
                      int basis, bool sample, cudaStream_t s);

// One fused step from buffer `src` into a.dst. basis: 0 Hermite, 1 f-norm,
// 2 look-up-table f-norm.
cudaError_t tma_step(const TmaPlan& plan, int src, const TmaArgs& a,
                     const CollideConst<float>& cc, int basis, bool sample, cudaStream_t s);

}  // namespace flb
