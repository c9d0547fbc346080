// flb_io.cuh -- state I/O between the public host layout f[i][y][x]
// (pre-collision f_i(x, t)) and a device buffer in the ghost-frame layout,
// which holds f*_i(z) = f_i(z + v_i) for the next pull; and a uniform fill.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "flb_kernels.cuh"
#include "flb_layout.cuh"

namespace flb {

template <class T>
__global__ void scatter_state_kernel(const double* in, Geometry geo, T* buf) {
    const long long N = (long long)geo.Lx * geo.Ly;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < (int)N; n += gridDim.x * blockDim.x) {
        const int y = n / geo.Lx, x = n - y * geo.Lx;
        for (int i = 0; i < 9; ++i) {
            // the buffer holds f*_i(z) = f_i(z + v_i): write f_i(x) at z = x - v_i,
            // with the ghost copy the pull of f_i(x) will read
            const int zx = wrap(x - cvx(i), geo.Lx), zy = wrap(y - cvy(i), geo.Ly);
            store_pop(buf, geo, i, zx, zy, (T)in[i * N + n]);
        }
    }
}

template <class T>
__global__ void gather_state_kernel(const T* buf, Geometry geo, double* out) {
    const long long N = (long long)geo.Lx * geo.Ly;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < (int)N; n += gridDim.x * blockDim.x) {
        const int y = n / geo.Lx, x = n - y * geo.Lx;
        for (int i = 0; i < 9; ++i) out[i * N + n] = (double)buf[pull_at(geo, i, x, y)];
    }
}

template <class T>
__global__ void fill_kernel(T* buf, Geometry geo, Vec9 v) {
    const long long total = 9 * geo.plane;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x)
        buf[k] = (T)v.v[k / geo.plane];
}

// FP16 deviation store: a buffer holds h_i = (f_i - ref_i) / scale.
struct DevCodec {
    float ref[9];
    float scale;
};

__device__ __forceinline__ double dev_decode(const DevCodec& c, int i, __half h) {
    return (double)c.ref[i] + (double)c.scale * (double)__half2float(h);
}

static __global__ void scatter_dev_kernel(const double* in, Geometry geo, DevCodec c, __half* buf) {
    const long long N = (long long)geo.Lx * geo.Ly;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < (int)N; n += gridDim.x * blockDim.x) {
        const int y = n / geo.Lx, x = n - y * geo.Lx;
        for (int i = 0; i < 9; ++i) {
            const int zx = wrap(x - cvx(i), geo.Lx), zy = wrap(y - cvy(i), geo.Ly);
            const double h = (in[i * N + n] - (double)c.ref[i]) / (double)c.scale;
            store_pop(buf, geo, i, zx, zy, __double2half(h));
        }
    }
}

static __global__ void gather_dev_kernel(const __half* buf, Geometry geo, DevCodec c, double* out) {
    const long long N = (long long)geo.Lx * geo.Ly;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < (int)N; n += gridDim.x * blockDim.x) {
        const int y = n / geo.Lx, x = n - y * geo.Lx;
        for (int i = 0; i < 9; ++i) out[i * N + n] = dev_decode(c, i, buf[pull_at(geo, i, x, y)]);
    }
}

}  // namespace flb
