// flb_lut.cu -- the velocity table of the look-up-table f-norm (Section 4):
// for each of the 51 x 51 table velocities u_g = ((k_x - 25)/50, (k_y - 25)/50)
// the Cholesky factor of the f-norm Schur complement at u_g (the form the
// collision applies it in: below-diagonal entries negated, reciprocal diagonal),
// u_g itself and a validity flag, in FP64 and FP32 (layout: flb_collide.cuh,
// kLutStride per entry). Built once per device, on first use, by one kernel
// that factors at every table velocity in FP64 (the FP32 table holds the FP64
// values rounded); kept in this file's device memory (0.7 MB per device) for
// the life of the process.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/flb.h"
#include "flb_basis.cuh"
#include "flb_runtime.h"

namespace flb {
namespace {

constexpr int kLutCells = kLutN * kLutN;

static __device__ __align__(16) float g_lut32[kLutCells * kLutStride];
static __device__ __align__(16) double g_lut64[kLutCells * kLutStride];

__global__ void lut_build_kernel(float* t32, double* t64) {
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= kLutCells) return;
    const int kx = cell % kLutN, ky = cell / kLutN;
    const double ux = (kx - 25.0) / 50.0, uy = (ky - 25.0) / 50.0;
    double W[9];
    feq_unit_fp64(ux, uy, W);
    bool ok = true;
    for (int i = 0; i < 9; ++i) ok = ok && W[i] > 0.0;
    const double uxx = ux * ux, uyy = uy * uy, uxy = ux * uy, usq = uxx + uyy;
    double Ln[6][6], inv[6];
    fnorm_factor<double>(ux, uy, uxx, uyy, uxy, usq, uxx - uyy, usq * -1.5, Ln, inv);
    for (int j = 0; j < 6; ++j) ok = ok && isfinite(inv[j]);
    double* e = t64 + (size_t)cell * kLutStride;
    for (int i = 1; i < 6; ++i)
        for (int j = 0; j < i; ++j) e[lut_ln_index(i, j)] = ok ? Ln[i][j] : 0.0;
    for (int j = 0; j < 6; ++j) e[kLutInv + j] = ok ? inv[j] : (double)INFINITY;
    e[kLutU] = ux;
    e[kLutU + 1] = uy;
    e[kLutFlag] = ok ? 1.0 : 0.0;
    float* e32 = t32 + (size_t)cell * kLutStride;
    for (int k = 0; k < kLutStride; ++k) e32[k] = (float)e[k];
}

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
const float* g_t32[kMaxDevices];
const double* g_t64[kMaxDevices];

}  // namespace

int lut_tables(const float** t32, const double** t64) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return FLB_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_t32[dev]) {
        void *p32 = nullptr, *p64 = nullptr;
        cudaError_t ce = cudaGetSymbolAddress(&p32, g_lut32);
        if (ce == cudaSuccess) ce = cudaGetSymbolAddress(&p64, g_lut64);
        if (ce == cudaSuccess) {
            // on a stream of its own, then waited for: callers may be capturing
            // theirs; this runs once per device
            cudaStream_t s;
            ce = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
            if (ce == cudaSuccess) {
                lut_build_kernel<<<(kLutCells + 63) / 64, 64, 0, s>>>((float*)p32, (double*)p64);
                ce = cudaGetLastError();
                const cudaError_t e2 = cudaStreamSynchronize(s);
                if (ce == cudaSuccess) ce = e2;
                cudaStreamDestroy(s);
            }
        }
        if (ce != cudaSuccess) {
            cudaGetLastError();
            return FLB_ERR_CUDA;
        }
        g_t32[dev] = (const float*)p32;
        g_t64[dev] = (const double*)p64;
    }
    if (t32) *t32 = g_t32[dev];
    if (t64) *t64 = g_t64[dev];
    return FLB_OK;
}

}  // namespace flb
