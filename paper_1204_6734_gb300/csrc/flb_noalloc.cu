// flb_noalloc.cu -- flb_step_noalloc: the FP64 fused step with correlation
// sampling for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc: plugins whose host application owns
// every device allocation through its own pool, and real-time or serving loops
// that plan their memory ahead of time and cannot take the implicit
// synchronisation of an allocation. This entry point takes the two population
// buffers from the caller and keeps its own scratch (per-block partial sums,
// the running sums, the error record) in a fixed array in this file's device
// memory. It ends by copying the sums to the host and synchronising the stream,
// so it is not a call for a stream that is being captured: such a stream is
// refused before anything is queued on it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/flb.h"
#include "flb_collide.cuh"
#include "flb_host.h"
#include "flb_kernels.cuh"

namespace flb {
namespace {

constexpr int kNoallocThreads = 256;
constexpr int kNoallocMaxBlocks = 1024;   // one node per thread: 262144 nodes at most

struct NoallocScratch {
    double partials[kNoallocMaxBlocks * kSums];
    double acc[kSums];
    DevError err;
};

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
NoallocScratch* g_scratch_addr[kMaxDevices];   // device address of the array, per device

// Device address of the scratch on the current device (host code may not use
// the symbol itself: on the host it names a stand-in, not device memory).
int scratch_on_current_device(NoallocScratch** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return FLB_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return FLB_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<NoallocScratch*>(ptr);
    }
    *out = g_scratch_addr[dev];
    return FLB_OK;
}

// Variant of the generic step kernel on the caller's buffers in the public
// layout f[i][y][x] (pre-collision state): one node per thread, the node's
// pre-collision populations are sampled into per-block FP64 partials, then
// collided and pushed to x + v_i (periodic) in the output buffer.
template <int BASIS>
__global__ void __launch_bounds__(kNoallocThreads)
noalloc_step_kernel(const double* fin, double* fout, int Lx, int Ly, uint32_t step,
                    CollideConst<double> cc, Vec9 ref, NoallocScratch* scratch) {
    const long long N = (long long)Lx * Ly;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    double s[kSums];
#pragma unroll
    for (int k = 0; k < kSums; ++k) s[k] = 0.0;
    if (n < N) {
        const int y = n / Lx, x = n - y * Lx;
        double g[9], f[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = fin[i * N + n];
        double d[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) d[i] = g[i] - ref.v[i];
        int k = 9;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            s[i] = d[i];
#pragma unroll
            for (int j = i; j < 9; ++j) s[k++] = d[i] * d[j];
        }
        const uint32_t st = collide<double, BASIS>(
            g, NodeNoise{cc.key, (uint32_t)n, step}, cc, f);
        if (st != kStatusOk) record_error(&scratch->err, (int)(st & 0xFF), n, step);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int xd = wrap(x + cvx(i), Lx), yd = wrap(y + cvy(i), Ly);
            fout[i * N + xd + (long long)Lx * yd] = f[i];
        }
    }
    block_reduce_sums<double>(s, scratch->partials + (size_t)blockIdx.x * kSums);
}

__global__ void noalloc_accumulate_kernel(NoallocScratch* scratch, int nblocks) {
    const double v = reduce_partials(scratch->partials, blockIdx.x, nblocks, threadIdx.x);
    if (threadIdx.x == 0) scratch->acc[blockIdx.x] += v;
}

}  // namespace
}  // namespace flb

using namespace flb;

extern "C" int flb_step_noalloc(const flb_params* p, double* dev_f, double* dev_work,
                                int64_t t0, int64_t nsteps, double* host_S1, double* host_S2,
                                void* stream) {
    // the checks flb_create makes, then this entry point's own limits
    if (!valid_params(p)) return FLB_ERR_ARG;
    if (!dev_f || !dev_work || dev_f == dev_work || t0 < 0 || nsteps < 0) return FLB_ERR_ARG;
    if (p->precision != FLB_FP64 || (p->basis != FLB_BASIS_STANDARD && p->basis != FLB_BASIS_LOCAL))
        return FLB_ERR_ARG;
    const long long N = (long long)p->Lx * p->Ly;
    if (N > (long long)kNoallocThreads * kNoallocMaxBlocks) return FLB_ERR_ARG;
    if (t0 + nsteps > 0xFFFFFFFFLL) return FLB_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    // the call reads its results back and synchronises: refuse a stream under
    // capture before queueing anything, so that the caller's capture survives
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        return FLB_ERR_CUDA;
    }
    if (cap != cudaStreamCaptureStatusNone) return FLB_ERR_ARG;

    NoallocScratch* scratch = nullptr;
    int rc = scratch_on_current_device(&scratch);
    if (rc) return rc;

    const CollideConst<double> cc = collide_const<double>(p);
    Vec9 ref;
    feq_host(p->rho0, p->ux0, p->uy0, ref.v);

    // the array keeps the previous call's contents: clear the sums and the error
    cudaError_t ce = cudaMemsetAsync(scratch->acc, 0, sizeof(scratch->acc), s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(&scratch->err, 0, sizeof(DevError), s);
    const int blocks = (int)((N + kNoallocThreads - 1) / kNoallocThreads);
    double* in = dev_f;
    double* out = dev_work;
    for (int64_t k = 0; k < nsteps && ce == cudaSuccess; ++k) {
        const uint32_t step = (uint32_t)(t0 + k);
        if (p->basis == FLB_BASIS_STANDARD)
            noalloc_step_kernel<0><<<blocks, kNoallocThreads, 0, s>>>(in, out, p->Lx, p->Ly, step,
                                                                      cc, ref, scratch);
        else
            noalloc_step_kernel<1><<<blocks, kNoallocThreads, 0, s>>>(in, out, p->Lx, p->Ly, step,
                                                                      cc, ref, scratch);
        ce = cudaGetLastError();
        if (ce == cudaSuccess) {
            noalloc_accumulate_kernel<<<kSums, 32, 0, s>>>(scratch, blocks);
            ce = cudaGetLastError();
        }
        double* t = in;
        in = out;
        out = t;
    }
    // the final state belongs in dev_f
    if (ce == cudaSuccess && in != dev_f)
        ce = cudaMemcpyAsync(dev_f, in, (size_t)9 * N * sizeof(double), cudaMemcpyDeviceToDevice, s);
    double acc[kSums];
    DevError err;
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(acc, scratch->acc, sizeof(acc), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(&err, &scratch->err, sizeof(err), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return FLB_ERR_CUDA;
    }
    if (err.code == kStatusInvalidVelocity) return FLB_ERR_INVALID_VELOCITY;
    if (err.code == kStatusNonfinite) return FLB_ERR_NONFINITE;
    if (host_S1)
        for (int i = 0; i < 9; ++i) host_S1[i] = acc[i];
    if (host_S2) {
        int k = 9;
        for (int i = 0; i < 9; ++i)
            for (int j = i; j < 9; ++j, ++k) host_S2[i * 9 + j] = host_S2[j * 9 + i] = acc[k];
    }
    return FLB_OK;
}
