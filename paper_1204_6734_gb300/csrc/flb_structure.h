// flb_structure.h -- static structure factors of a lattice's hydrodynamic
// fields (Eqs. sfactorr, sfactoru, rcorrelator), sampled on the device.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "flb_io.cuh"
#include "flb_layout.cuh"

namespace flb {

struct StructSampler;

// Device buffers for an Lx x Ly lattice at transform precision rbytes (4:
// FP32, 8: FP64); FLB_ERR_ARG when a row or column of complex values does not
// fit one CTA's shared memory (sides above 20480 in FP32, 10240 in FP64);
// FLB_ERR_OOM when an allocation fails.
// fused: the FP32 step kernel will form the fields itself (structure_fields,
// structure_sample_fields), which needs a 3 Lx Ly FP32 field buffer.
int structure_create(StructSampler** out, int Lx, int Ly, int rbytes, bool fused);
void structure_destroy(StructSampler* s);
cudaError_t structure_reset(StructSampler* s, cudaStream_t st);
// One sample of the pre-collision state the pull from `buf` gives:
// accumulates |drho(k)|^2, |dj_x(k)|^2 and dj_x(k) conj(dj_y(k)); ref[9] is
// f^0(rho0, u0), the fields being sums of f_i - ref_i.
cudaError_t structure_sample(StructSampler* s, const void* buf, int precision, const Geometry& geo,
                             const DevCodec& codec, const double* ref, cudaStream_t st);
// The field buffer ([f][y][x], f = drho, dj_x, dj_y, FP32) a step kernel fills
// on a sampling step when the sampler was created fused and both sides are
// powers of two; nullptr otherwise (structure_sample is used then).
float* structure_fields(StructSampler* s);
// One sample from the fields a step kernel has written to structure_fields(s)
// (the same sums as structure_sample of that step's pre-collision state).
cudaError_t structure_sample_fields(StructSampler* s, cudaStream_t st);
// The four FP64 sums S_rho, S_jx, Re R, Im R, each Ly x Lx ([m_y][m_x]),
// times `scale`, into the host arrays out[0..3] (a NULL entry is skipped);
// synchronises the stream. FLB_OK, FLB_ERR_OOM or FLB_ERR_CUDA.
int structure_read(StructSampler* s, double* const out[4], double scale, cudaStream_t st);
int64_t structure_samples(const StructSampler* s);

}  // namespace flb
