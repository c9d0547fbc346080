// flb_capi.cu -- the C ABI declared in include/flb.h: lattice handles, device
// memory, kernel launches, correlation/conservation reductions, state I/O.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/flb.h"
#include "flb_basis.cuh"
#include "flb_host.h"
#include "flb_runtime.h"
#include "flb_internal.h"
#include "flb_io.cuh"
#include "flb_structure.h"
#include "flb_kernels.cuh"

namespace flb {

// ---------------------------------------------------------------------------
// Reduction kernels
// ---------------------------------------------------------------------------

__global__ void accumulate_partials_kernel(const double* partials, int nblocks, double* acc) {
    const double v = reduce_partials(partials, blockIdx.x, nblocks, threadIdx.x);
    if (threadIdx.x == 0) acc[blockIdx.x] += v;
}

// Rows of the basis the correlations are measured in: the Hermite rows
// (Eq. d2q93a), or the f-norm basis at (ux0, uy0) -- Cholesky of the full 9x9
// Gram matrix sum_i p^a_i p^b_i f_i^0(1,u0), m~ = L^{-1} P. One thread.
__global__ void measure_basis_kernel(int basis, double ux0, double uy0, double* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (basis == FLB_BASIS_STANDARD) {
        double P[9][9];
        hermite_rows_fp64(P);
        for (int a = 0; a < 9; ++a)
            for (int i = 0; i < 9; ++i) out[a * 9 + i] = P[a][i];
        return;
    }
    fnorm_basis_fp64(ux0, uy0, out);
}

__global__ void finalize_kernel(const double* acc, long long nsamp, const double* B,
                                double* out) {
    __shared__ double C[81];
    __shared__ double mean[9];
    const int t = threadIdx.x;
    const double inv = 1.0 / (double)nsamp;
    if (t < 9) mean[t] = acc[t] * inv;
    __syncthreads();
    if (t < 81) {
        const int i = t / 9, j = t % 9;
        const int a = i < j ? i : j, b = i < j ? j : i;
        // index of (a, b), a <= b, in the packed upper triangle after S1
        const int k = 9 + a * 9 - a * (a - 1) / 2 + (b - a);
        C[t] = acc[k] * inv - mean[i] * mean[j];
        out[t] = C[t];
    }
    __syncthreads();
    if (t < 81) {
        const int a = t / 9, b = t % 9;
        double s = 0.0;
        for (int i = 0; i < 9; ++i)
            for (int j = 0; j < 9; ++j) s += B[a * 9 + i] * C[i * 9 + j] * B[b * 9 + j];
        out[81 + t] = s;
    }
    if (t < 9) out[162 + t] = mean[t];
}

// Total mass and momentum of the pre-collision state, FP64 per block.
__device__ __forceinline__ double pop_value(const double* src, long long k, int, const DevCodec&) {
    return src[k];
}
__device__ __forceinline__ double pop_value(const float* src, long long k, int, const DevCodec&) {
    return (double)src[k];
}
__device__ __forceinline__ double pop_value(const __half* src, long long k, int i,
                                            const DevCodec& c) {
    return dev_decode(c, i, src[k]);
}

template <class T>
__global__ void __launch_bounds__(kStepThreads)
conservation_kernel(const T* src, Geometry geo, double* partials, DevCodec codec) {
    const long long N = (long long)geo.Lx * geo.Ly;
    double r = 0.0, jx = 0.0, jy = 0.0;
    // the pre-collision state f_i(x) = f*_i(x - v_i)
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < (int)N; n += gridDim.x * blockDim.x) {
        const int y = n / geo.Lx, x = n - y * geo.Lx;
        for (int i = 0; i < 9; ++i) {
            const double v = pop_value(src, pull_at(geo, i, x, y), i, codec);
            r += v;
            jx += v * cvx(i);
            jy += v * cvy(i);
        }
    }
    __shared__ double red[3][kStepThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        r += __shfl_xor_sync(0xffffffffu, r, o);
        jx += __shfl_xor_sync(0xffffffffu, jx, o);
        jy += __shfl_xor_sync(0xffffffffu, jy, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][warp] = r;
        red[1][warp] = jx;
        red[2][warp] = jy;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int w = 0; w < kStepThreads / 32; ++w) t += red[threadIdx.x][w];
        partials[blockIdx.x * 3 + threadIdx.x] = t;
    }
}

__global__ void sum3_kernel(const double* partials, int nblocks, double* out) {
    const int k = threadIdx.x;
    if (k >= 3) return;
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += partials[b * 3 + k];
    out[k] = t;
}

// Max |f_a - f_b|, sum of (f_a - f_b)^2 and max |f_b| over the pre-collision
// states of two lattices of the same size (any storage precisions), per block.
struct StateView {
    const void* buf;
    int prec;   // FLB_FP64, FLB_FP32 or FLB_FP16_DEV
    Geometry geo;
    DevCodec codec;
    __device__ __forceinline__ double get(int i, int x, int y) const {
        const long long k = pull_at(geo, i, x, y);
        if (prec == FLB_FP64) return ((const double*)buf)[k];
        if (prec == FLB_FP32) return (double)((const float*)buf)[k];
        return dev_decode(codec, i, ((const __half*)buf)[k]);
    }
};

__global__ void __launch_bounds__(kStepThreads)
state_difference_kernel(StateView a, StateView b, double* partials) {
    const int Lx = a.geo.Lx;
    const long long N = (long long)Lx * a.geo.Ly;
    double mx = 0.0, ss = 0.0, mb = 0.0;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < (int)N; n += gridDim.x * blockDim.x) {
        const int y = n / Lx, x = n - y * Lx;
        for (int i = 0; i < 9; ++i) {
            const double fa = a.get(i, x, y), fb = b.get(i, x, y);
            const double d = fa - fb;
            mx = fmax(mx, fabs(d));
            ss += d * d;
            mb = fmax(mb, fabs(fb));
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
        mb = fmax(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    }
    __shared__ double red[3][kStepThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][warp] = mx;
        red[1][warp] = ss;
        red[2][warp] = mb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kStepThreads / 32; ++w) {
            red[0][0] = fmax(red[0][0], red[0][w]);
            red[1][0] += red[1][w];
            red[2][0] = fmax(red[2][0], red[2][w]);
        }
        partials[blockIdx.x * 3 + 0] = red[0][0];
        partials[blockIdx.x * 3 + 1] = red[1][0];
        partials[blockIdx.x * 3 + 2] = red[2][0];
    }
}

// ---------------------------------------------------------------------------
// Test hooks
// ---------------------------------------------------------------------------

template <class T>
__global__ void noise_draws_kernel(uint64_t seed, uint32_t replica, uint32_t step,
                                   const uint32_t* nodes, int n, uint32_t* fields,
                                   double* normals) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const NoiseKey key = make_noise_key(seed, replica);   // per-thread copy, test hook only
    uint32_t f[6];
    node_fields(key, nodes[k], step, f);
    T z[6];
    box_muller(f, z);
    for (int q = 0; q < 6; ++q) {
        fields[k * 6 + q] = f[q];
        normals[k * 6 + q] = (double)z[q];
    }
}

template <class T, int BASIS>
__global__ void collide_nodes_kernel(const double* g, const uint32_t* ids, uint32_t step,
                                     int n, CollideConst<T> cc, const T* lut, double* fs,
                                     int* status) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    T gg[9], ff[9];
    for (int i = 0; i < 9; ++i) gg[i] = (T)g[k * 9 + i];
    const uint32_t id = ids[k];
    const int st = (int)(collide_basis<T, BASIS>(
                             gg, NodeNoise{cc.key, id, step},
                             [&](T* g2) {
                                 for (int i = 0; i < 9; ++i) g2[i] = gg[i];
                             },
                             lut, cc, ff) &
                         0xFF);
    for (int i = 0; i < 9; ++i) fs[k * 9 + i] = (double)ff[i];
    status[k] = st;
}

}  // namespace flb

// ===========================================================================
// Handle and C ABI
// ===========================================================================

using namespace flb;

// Halo of a slab (flb_set_slab): the populations that cross its y boundaries.
// Moving up (v_y = +1): 2, 5, 6; moving down (v_y = -1): 4, 7, 8.
__device__ __constant__ int kHaloUp[3] = {2, 5, 6};
__device__ __constant__ int kHaloDown[3] = {4, 7, 8};

// lo: f*_i(x, 0) for i moving down (to the slab below); hi: f*_i(x, Ly - 1) for
// i moving up (to the slab above); each 3 rows of Lx values.
template <class T>
__global__ void halo_pack_kernel(const T* buf, Geometry geo, T* lo, T* hi) {
    const int Lx = geo.Lx;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 6 * Lx; k += gridDim.x * blockDim.x) {
        const int q = k / Lx, x = k - q * Lx;
        if (q < 3)
            lo[k] = buf[at(geo, kHaloDown[q], x, 0)];
        else
            hi[k - 3 * Lx] = buf[at(geo, kHaloUp[q - 3], x, geo.Ly - 1)];
    }
}

// The ghost rows the next pull reads across the y boundaries: row -1 (i moving
// up) from the slab below's hi, row Ly (i moving down) from the slab above's
// lo, columns -1 .. Lx with the lattice's periodicity in x.
template <class T>
__global__ void halo_unpack_kernel(T* buf, Geometry geo, const T* lo, const T* hi) {
    const int Lx = geo.Lx, W = Lx + 2;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 6 * W; k += gridDim.x * blockDim.x) {
        const int q = k / W, c = k - q * W - 1;
        const int x = wrap(c, Lx);
        if (q < 3)
            buf[at(geo, kHaloUp[q], c, -1)] = lo[q * Lx + x];
        else
            buf[at(geo, kHaloDown[q - 3], c, geo.Ly)] = hi[(q - 3) * Lx + x];
    }
}

struct flb_lattice_s {
    flb_params p;
    int elem;            // bytes per population value
    Geometry geo;
    char* ws;
    bool own_ws;
    size_t ws_bytes;
    void* buf[2];
    int cur;             // buf[cur] holds f*(t-1), the source of the next pull
    double* partials;
    int nblocks;         // grid of the step kernel
    double* acc;         // kSums running sums
    double* small;       // basis (81) + finalize output (171) + conservation (3)
    DevError* err;
    cudaStream_t stream;
    int64_t t, warmup, every, nsamp;
    int sticky;
    int variant;           // FLB_KERNEL_*
    TmaPlan tma;           // pipelined FP32 kernel (tensor maps, launch shape)
    TmaPlan tma_quiet;     // the same for steps without sampling, when it differs
    const float* lut32 = nullptr;    // velocity tables (look-up-table f-norm)
    const double* lut64 = nullptr;
    double ref[9];
    StructSampler* sk = nullptr;      // structure factors (allocated on demand)
    int64_t sk_warmup = 0, sk_every = 0;
    // slab of a larger periodic lattice (flb_set_slab): rows y0 .. y0 + Ly - 1
    // of Ly_total; node0 = Lx y0 offsets the noise counters
    bool slab = false;
    int slab_y0 = 0, slab_Ly_total = 0;
    uint32_t node0 = 0;
};

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

int elem_size(int prec) { return prec == FLB_FP64 ? 8 : (prec == FLB_FP16_DEV ? 2 : 4); }

Geometry make_geometry(const flb_params* p) { return flb::make_geometry(p->Lx, p->Ly); }

int device_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

int step_grid(const Geometry& g, int sms) {
    const long long N = (long long)g.Lx * g.Ly;
    long long blocks = (N + kStepThreads - 1) / kStepThreads;
    const long long cap = (long long)(sms > 0 ? sms : 1) * 8;
    if (blocks > cap) blocks = cap;
    return (int)(blocks < 1 ? 1 : blocks);
}

struct Layout {
    size_t buf_bytes, partial_off, acc_off, small_off, err_off, total;
    int nblocks, npartials;
};

Layout layout(const flb_params* p, int sms) {
    Layout L;
    const Geometry g = make_geometry(p);
    L.nblocks = step_grid(g, sms);
    L.buf_bytes = align_up((size_t)(9 * g.plane) * elem_size(p->precision));
    size_t off = 2 * L.buf_bytes;
    L.npartials = L.nblocks;
    L.partial_off = off;
    off += align_up(sizeof(double) * (size_t)L.npartials * kSums);
    L.acc_off = off;
    off += align_up(sizeof(double) * kSums);
    L.small_off = off;
    off += align_up(sizeof(double) * (81 + 171 + 3 + 3 * (size_t)L.nblocks));
    L.err_off = off;
    off += align_up(sizeof(DevError));
    L.total = off;
    return L;
}

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? FLB_OK : FLB_ERR_CUDA; }


template <class T, int BASIS, bool SAMPLE>
cudaError_t launch_step_t(flb_lattice h) {
    StepArgs<T> a;
    a.src = (const T*)h->buf[h->cur];
    a.dst = (T*)h->buf[h->cur ^ 1];
    a.geo = h->geo;
    a.step = (uint32_t)h->t;
    a.node0 = h->node0;
    a.partials = h->partials;
    a.err = h->err;
    a.lut = (const T*)(sizeof(T) == 8 ? (const void*)h->lut64 : (const void*)h->lut32);
    for (int i = 0; i < 9; ++i) a.ref[i] = (T)h->ref[i];
    step_kernel<T, BASIS, SAMPLE><<<h->nblocks, kStepThreads, 0, h->stream>>>(
        a, collide_const<T>(&h->p));
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_step_p(flb_lattice h, bool sample) {
    if (h->p.basis == FLB_BASIS_STANDARD)
        return sample ? launch_step_t<T, 0, true>(h) : launch_step_t<T, 0, false>(h);
    if (h->p.basis == FLB_BASIS_LOCAL)
        return sample ? launch_step_t<T, 1, true>(h) : launch_step_t<T, 1, false>(h);
    return sample ? launch_step_t<T, 2, true>(h) : launch_step_t<T, 2, false>(h);
}

// Pipelined FP32 kernel: also reduces the sampled sums into h->acc itself.
cudaError_t launch_step_tma(flb_lattice h, bool sample, float* fields) {
    TmaArgs a;
    a.fields = fields;
    a.dst = (float*)h->buf[h->cur ^ 1];
    a.geo = h->geo;
    a.step = (uint32_t)h->t;
    a.node0 = h->node0;
    a.tiles_x = a.ntiles = 0;
    a.acc = h->acc;
    a.err = h->err;
    a.lut = h->lut32;
    for (int i = 0; i < 9; ++i) a.ref[i] = (float)h->ref[i];
    a.s = tensor_sampling_ok(&h->p) ? gram_scale(&h->p) : 1.0;
    a.sinv = (float)(1.0 / a.s);
    for (int i = 0; i < 9; ++i) a.snref[i] = (float)(-h->ref[i] / a.s);
    const TmaPlan& plan = !sample && h->tma_quiet.ready ? h->tma_quiet : h->tma;
    return tma_step(plan, h->cur, a, collide_const<float>(&h->p), h->p.basis, sample, h->stream);
}

bool uses_tma(flb_lattice h) {
    return h->p.precision == FLB_FP32 && h->variant != FLB_KERNEL_GENERIC;
}

// The pipelined kernels (FP32, FP16 store) add their sums to h->acc themselves.
bool reduces_in_kernel(flb_lattice h) { return uses_tma(h) || h->p.precision == FLB_FP16_DEV; }

DevCodec dev_codec(flb_lattice h) {
    DevCodec c;
    for (int i = 0; i < 9; ++i) c.ref[i] = (float)h->ref[i];
    c.scale = (float)std::sqrt(h->p.kT);
    return c;
}

// FP16 deviation store: h = (f - ref) / sqrt(kT), collision in FP32.
cudaError_t launch_step_fp16(flb_lattice h, bool sample) {
    HArgs a;
    a.dst = (__half*)h->buf[h->cur ^ 1];
    a.geo = h->geo;
    a.step = (uint32_t)h->t;
    a.node0 = h->node0;
    a.tiles_x = a.ntiles = 0;
    a.acc = h->acc;
    a.err = h->err;
    a.lut = h->lut32;
    const DevCodec c = dev_codec(h);
    a.scale = c.scale;
    a.inv_scale = 1.0f / c.scale;
    for (int i = 0; i < 9; ++i) {
        a.ref[i] = c.ref[i];
        a.nref[i] = -c.ref[i] * a.inv_scale;
    }
    return fp16_step(h->tma, h->cur, a, collide_const<float>(&h->p), h->p.basis, sample, h->stream);
}

// fields: where the pipelined FP32 kernel writes the structure-factor fields
// of this step's pre-collision state (nullptr: not sampled by the step).
cudaError_t launch_step(flb_lattice h, bool sample, float* fields = nullptr) {
    if (h->p.precision == FLB_FP64) return launch_step_p<double>(h, sample);
    if (h->p.precision == FLB_FP16_DEV) return launch_step_fp16(h, sample);
    if (uses_tma(h)) return launch_step_tma(h, sample, fields);
    return launch_step_p<float>(h, sample);
}

int check_device_error(flb_lattice h) {
    DevError e;
    cudaError_t ce = cudaMemcpyAsync(&e, h->err, sizeof(e), cudaMemcpyDeviceToHost, h->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
    if (ce != cudaSuccess) return FLB_ERR_CUDA;
    if (e.code != 0 && h->sticky == 0) h->sticky = map_status(e.code);
    return h->sticky;
}

}  // namespace

namespace flb {

int lattice_create(const flb_params* p, void* dev_workspace, size_t workspace_bytes,
                   cudaStream_t stream, bool sync, flb_lattice* out) {
    if (!out) return FLB_ERR_ARG;
    *out = nullptr;
    if (!valid_params(p)) return FLB_ERR_ARG;
    const int sms = device_sms();
    if (sms <= 0) return FLB_ERR_CUDA;
    const Layout L = layout(p, sms);
    flb_lattice h = new (std::nothrow) flb_lattice_s();
    if (!h) return FLB_ERR_OOM;
    h->p = *p;
    h->elem = elem_size(p->precision);
    h->geo = flb::make_geometry(p->Lx, p->Ly);
    h->stream = stream;
    if (dev_workspace) {
        if (workspace_bytes < L.total || ((uintptr_t)dev_workspace % kAlign) != 0) {
            delete h;
            return FLB_ERR_OOM;
        }
        h->ws = (char*)dev_workspace;
        h->own_ws = false;
    } else {
        void* ptr = nullptr;
        if (cudaMalloc(&ptr, L.total) != cudaSuccess) {
            cudaGetLastError();
            delete h;
            return FLB_ERR_OOM;
        }
        h->ws = (char*)ptr;
        h->own_ws = true;
    }
    h->ws_bytes = L.total;
    h->buf[0] = h->ws;
    h->buf[1] = h->ws + L.buf_bytes;
    h->partials = (double*)(h->ws + L.partial_off);
    h->acc = (double*)(h->ws + L.acc_off);
    h->small = (double*)(h->ws + L.small_off);
    h->err = (DevError*)(h->ws + L.err_off);
    h->nblocks = L.nblocks;
    h->variant = FLB_KERNEL_AUTO;
    h->cur = 0;
    feq_host(p->rho0, p->ux0, p->uy0, h->ref);

    cudaError_t ce = cudaMemsetAsync(h->ws + L.partial_off, 0, L.total - L.partial_off, h->stream);
    Vec9 v;
    for (int i = 0; i < 9; ++i) v.v[i] = h->ref[i];
    if (ce == cudaSuccess) {
        if (p->precision == FLB_FP64)
            fill_kernel<double><<<grid_for(9 * h->geo.plane), 256, 0, h->stream>>>(
                (double*)h->buf[0], h->geo, v);
        else if (p->precision == FLB_FP32)
            fill_kernel<float><<<grid_for(9 * h->geo.plane), 256, 0, h->stream>>>(
                (float*)h->buf[0], h->geo, v);
        else   // FP16 deviation store: f = ref everywhere is h = 0
            cudaMemsetAsync(h->buf[0], 0, L.buf_bytes, h->stream);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess && sync) ce = cudaStreamSynchronize(h->stream);
    // sampling steps: the correlation sums on the tensor cores, where the
    // parameters allow it, with 16 colliding warps in the f-norm bases (4096^2:
    // f-norm 54.8 against 54.6 GLUPS with 12, table f-norm 55.5 against 50.4)
    // and 12 in the Hermite norm (77.9 against 71.4 with 16); otherwise the
    // sampler warps beside 8 colliding warps. 16 warps make 128 x 8 tiles: a
    // lattice with fewer than 8 of them per SM keeps 12 (more CTAs busy).
    const bool tensor = tensor_sampling_ok(p);
    const bool tall = (long long)((p->Lx + 127) / 128) * ((p->Ly + 7) / 8) >= 8LL * (sms > 0 ? sms : 1);
    const int fnorm_nw = tall ? 16 : kTensorNW;
    const int tensor_nw = p->basis == FLB_BASIS_STANDARD ? kTensorNW : fnorm_nw;
    h->tma.sample_mode = tensor ? kPlanTensorSampling : 0;
    if (ce == cudaSuccess && p->basis == FLB_BASIS_LOCAL_LUT &&
        lut_tables(&h->lut32, &h->lut64) != FLB_OK)
        ce = cudaErrorUnknown;
    h->tma_quiet.ready = false;
    if (ce == cudaSuccess && p->precision == FLB_FP32) {
        ce = tma_plan(&h->tma, h->buf[0], h->buf[1], h->geo, tensor ? tensor_nw : 0);
        // steps without sampling: 16 colliding warps in the f-norm bases
        // (4096^2: f-norm 64.6 against 60.6 GLUPS with 12, table f-norm 63.8
        // against 61.8; 12 on small lattices), 8 in the Hermite norm (85.0
        // against 74.4 with 12)
        const int quiet_nw = p->basis == FLB_BASIS_STANDARD ? 8 : fnorm_nw;
        if (ce == cudaSuccess && quiet_nw != h->tma.nw &&
            tma_plan(&h->tma_quiet, h->buf[0], h->buf[1], h->geo, quiet_nw) != cudaSuccess) {
            cudaGetLastError();
            h->tma_quiet.ready = false;
        }
    }
    if (ce == cudaSuccess && p->precision == FLB_FP16_DEV)
        ce = fp16_plan(&h->tma, h->buf[0], h->buf[1], h->geo);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        if (h->own_ws) cudaFree(h->ws);
        delete h;
        return FLB_ERR_CUDA;
    }
    *out = h;
    return FLB_OK;
}

int lattice_enqueue_readout(flb_lattice h, double* acc_out, DevError* err_out) {
    if (!h) return FLB_ERR_ARG;
    cudaError_t ce = cudaMemcpyAsync(acc_out, h->acc, sizeof(double) * kSums,
                                     cudaMemcpyDeviceToHost, h->stream);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(err_out, h->err, sizeof(DevError), cudaMemcpyDeviceToHost, h->stream);
    return cuda_rc(ce);
}

int64_t lattice_samples(flb_lattice h) { return h ? h->nsamp : 0; }

int64_t lattice_time(flb_lattice h) { return h ? h->t : -1; }

void lattice_forget(flb_lattice h) {
    if (h && !h->own_ws) delete h;
}

}  // namespace flb

namespace flb {

int finalize_sums(const double* acc, int64_t nsamp, int32_t measure_basis, double ux0, double uy0,
                  cudaStream_t st, double* Cff, double* CMM, double* mean_dev) {
    if (measure_basis != FLB_BASIS_STANDARD && measure_basis != FLB_BASIS_LOCAL) return FLB_ERR_ARG;
    if (nsamp <= 0) return FLB_ERR_STATE;
    double* dev = nullptr;   // sums, basis, results
    if (cudaMalloc(&dev, sizeof(double) * (kSums + 81 + 171)) != cudaSuccess) {
        cudaGetLastError();
        return FLB_ERR_OOM;
    }
    double host[171];
    cudaError_t ce = cudaMemcpyAsync(dev, acc, sizeof(double) * kSums, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) {
        measure_basis_kernel<<<1, 32, 0, st>>>(measure_basis, ux0, uy0, dev + kSums);
        finalize_kernel<<<1, 96, 0, st>>>(dev, nsamp, dev + kSums, dev + kSums + 81);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(host, dev + kSums + 81, sizeof(host), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    cudaFree(dev);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return FLB_ERR_CUDA;
    }
    if (Cff) std::memcpy(Cff, host, 81 * sizeof(double));
    if (CMM) std::memcpy(CMM, host + 81, 81 * sizeof(double));
    if (mean_dev) std::memcpy(mean_dev, host + 162, 9 * sizeof(double));
    return FLB_OK;
}

}  // namespace flb

namespace {
template <class T>
cudaError_t halo_call(flb_lattice h, bool pack, void* lo, void* hi) {
    const int n = 6 * (h->p.Lx + 2);
    const int grid = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
    if (pack)
        halo_pack_kernel<T><<<grid, 256, 0, h->stream>>>((const T*)h->buf[h->cur], h->geo, (T*)lo,
                                                          (T*)hi);
    else
        halo_unpack_kernel<T><<<grid, 256, 0, h->stream>>>((T*)h->buf[h->cur], h->geo,
                                                            (const T*)lo, (const T*)hi);
    return cudaGetLastError();
}
int halo(flb_lattice h, bool pack, void* lo, void* hi) {
    if (!h || !lo || !hi || !h->slab) return FLB_ERR_ARG;
    if (h->sticky) return h->sticky;
    cudaError_t ce;
    if (h->p.precision == FLB_FP64)
        ce = halo_call<double>(h, pack, lo, hi);
    else if (h->p.precision == FLB_FP32)
        ce = halo_call<float>(h, pack, lo, hi);
    else
        ce = halo_call<__half>(h, pack, lo, hi);
    return cuda_rc(ce);
}
}  // namespace

extern "C" {

int flb_version(void) { return 100; }

const char* flb_error_string(int code) {
    switch (code) {
        case FLB_OK: return "ok";
        case FLB_ERR_ARG: return "invalid argument";
        case FLB_ERR_OOM: return "out of device memory or workspace too small";
        case FLB_ERR_INVALID_VELOCITY: return "a node velocity left the region where all f_i^0(1,u) > 0";
        case FLB_ERR_NONFINITE: return "non-finite or non-positive density at a node";
        case FLB_ERR_TIMEOUT: return "a bounded device wait timed out";
        case FLB_ERR_CUDA: return "CUDA runtime error";
        case FLB_ERR_STATE: return "call not valid in the current state";
        default: return "unknown error";
    }
}

size_t flb_workspace_bytes(const flb_params* p) {
    if (!valid_params(p)) return 0;
    return layout(p, device_sms()).total;
}

int flb_create(const flb_params* p, void* dev_workspace, size_t workspace_bytes, void* stream,
               flb_lattice* out) {
    return lattice_create(p, dev_workspace, workspace_bytes, (cudaStream_t)stream, true, out);
}

int flb_destroy(flb_lattice h) {
    if (!h) return FLB_OK;
    cudaError_t ce = cudaStreamSynchronize(h->stream);
    structure_destroy(h->sk);
    if (h->own_ws) {
        cudaError_t fe = cudaFree(h->ws);
        if (ce == cudaSuccess) ce = fe;
    }
    delete h;
    return cuda_rc(ce);
}

int flb_reset_statistics(flb_lattice h) {
    if (!h) return FLB_ERR_ARG;
    h->nsamp = 0;
    return cuda_rc(cudaMemsetAsync(h->acc, 0, sizeof(double) * kSums, h->stream));
}

int flb_set_sampling(flb_lattice h, int64_t warmup, int64_t every) {
    if (!h || warmup < 0 || every < 0) return FLB_ERR_ARG;
    h->warmup = warmup;
    h->every = every;
    return flb_reset_statistics(h);
}

int flb_set_structure_sampling(flb_lattice h, int64_t warmup, int64_t every) {
    if (!h || warmup < 0 || every < 0) return FLB_ERR_ARG;
    if (h->slab && every > 0) return FLB_ERR_ARG;   // the transform spans the whole lattice
    if (h->sticky) return h->sticky;
    if (every > 0 && !h->sk) {
        const int rc = structure_create(&h->sk, h->p.Lx, h->p.Ly,
                                        h->p.precision == FLB_FP64 ? 8 : 4, h->p.precision == FLB_FP32);
        if (rc) return rc;
    }
    h->sk_warmup = warmup;
    h->sk_every = every;
    return h->sk ? cuda_rc(structure_reset(h->sk, h->stream)) : FLB_OK;
}

int flb_structure_factors(flb_lattice h, double* S_rho, double* S_jx, double* R_re, double* R_im,
                          int64_t* n_samples) {
    if (!h) return FLB_ERR_ARG;
    const int64_t ns = structure_samples(h->sk);
    if (n_samples) *n_samples = ns;
    if (!S_rho && !S_jx && !R_re && !R_im) return FLB_OK;
    if (!h->sk || ns == 0) return FLB_ERR_STATE;
    double* const out[4] = {S_rho, S_jx, R_re, R_im};
    return structure_read(h->sk, out, 1.0 / ((double)ns * h->p.rho0), h->stream);
}

int flb_step(flb_lattice h, int64_t n) {
    if (!h || n < 0) return FLB_ERR_ARG;
    if (h->sticky) return h->sticky;
    const long long N = (long long)h->p.Lx * h->p.Ly;
    for (int64_t s = 0; s < n; ++s) {
        const bool sample =
            h->every > 0 && h->t >= h->warmup && ((h->t - h->warmup) % h->every) == 0;
        cudaError_t ce = cudaSuccess;
        // a structure-factor sample of the state this step starts from: the
        // pipelined FP32 kernel forms its fields while it collides, else the
        // sampler reads the populations before the step
        const bool sk_due =
            h->sk_every > 0 && h->t >= h->sk_warmup && ((h->t - h->sk_warmup) % h->sk_every) == 0;
        float* fields = sk_due && uses_tma(h) ? structure_fields(h->sk) : nullptr;
        if (sk_due && !fields)
            ce = structure_sample(h->sk, h->buf[h->cur], h->p.precision, h->geo, dev_codec(h), h->ref,
                                  h->stream);
        if (ce == cudaSuccess) ce = launch_step(h, sample, fields);
        if (ce == cudaSuccess && fields) ce = structure_sample_fields(h->sk, h->stream);
        if (ce == cudaSuccess && sample && !reduces_in_kernel(h)) {
            accumulate_partials_kernel<<<kSums, 32, 0, h->stream>>>(h->partials, h->nblocks,
                                                                     h->acc);
            ce = cudaGetLastError();
        }
        if (sample) h->nsamp += N;
        if (ce != cudaSuccess) return FLB_ERR_CUDA;
        h->t += 1;
        h->cur ^= 1;
    }
    return FLB_OK;
}

int flb_set_option(flb_lattice h, int32_t option, int32_t value) {
    if (!h) return FLB_ERR_ARG;
    if (option == FLB_OPT_KERNEL) {
        if (value != FLB_KERNEL_AUTO && value != FLB_KERNEL_GENERIC && value != FLB_KERNEL_PIPELINED)
            return FLB_ERR_ARG;
        if (value == FLB_KERNEL_PIPELINED && h->p.precision != FLB_FP32) return FLB_ERR_ARG;
        if (value == FLB_KERNEL_GENERIC && h->p.precision == FLB_FP16_DEV) return FLB_ERR_ARG;
        h->variant = value;
        return FLB_OK;
    }
    if (option == FLB_OPT_PIPELINE_SAMPLING) {
        if (h->p.precision != FLB_FP32 || value < 1 || value > 3) return FLB_ERR_ARG;
        if (value == kPlanTensorSampling && !tensor_sampling_ok(&h->p)) return FLB_ERR_ARG;
        TmaPlan plan = h->tma;
        plan.sample_mode = value;
        cudaError_t ce = tma_plan(&plan, h->buf[0], h->buf[1], h->geo, h->tma.nw);
        if (ce == cudaSuccess && plan.sample_mode != value && h->tma.nw > kTensorNW) {
            // 16 colliding warps take only the tensor-core sums: the other
            // modes run with 12
            plan.sample_mode = value;
            ce = tma_plan(&plan, h->buf[0], h->buf[1], h->geo, kTensorNW);
        }
        if (ce != cudaSuccess || plan.sample_mode != value) {
            cudaGetLastError();
            return FLB_ERR_ARG;
        }
        h->tma = plan;
        return FLB_OK;
    }
    if (option == FLB_OPT_PIPELINE_WARPS) {
        if (h->p.precision != FLB_FP32) return FLB_ERR_ARG;
        TmaPlan plan;
        plan.sample_mode = h->tma.sample_mode;
        const cudaError_t ce = tma_plan(&plan, h->buf[0], h->buf[1], h->geo, value);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            return FLB_ERR_ARG;
        }
        if (plan.sample_mode == kPlanTensorSampling && !tensor_sampling_ok(&h->p)) return FLB_ERR_ARG;
        h->tma = plan;
        h->tma_quiet.ready = false;   // the given count for every step
        return FLB_OK;
    }
    return FLB_ERR_ARG;
}

int flb_set_slab(flb_lattice h, int32_t Ly_total, int32_t y0) {
    if (!h || y0 < 0 || Ly_total < 1 || (long long)y0 + h->p.Ly > Ly_total) return FLB_ERR_ARG;
    if ((long long)h->p.Lx * Ly_total > 0xFFFFFFFFLL) return FLB_ERR_ARG;
    if (h->sk_every > 0) return FLB_ERR_ARG;   // structure factors are whole-lattice quantities
    h->slab = true;
    h->slab_y0 = y0;
    h->slab_Ly_total = Ly_total;
    h->node0 = (uint32_t)h->p.Lx * (uint32_t)y0;
    return FLB_OK;
}

size_t flb_halo_bytes(flb_lattice h) {
    if (!h) return 0;
    return (size_t)3 * h->p.Lx * elem_size(h->p.precision);
}

int flb_halo_pack(flb_lattice h, void* dev_lo, void* dev_hi) { return halo(h, true, dev_lo, dev_hi); }

int flb_halo_unpack(flb_lattice h, const void* dev_lo, const void* dev_hi) {
    return halo(h, false, const_cast<void*>(dev_lo), const_cast<void*>(dev_hi));
}

int flb_sync(flb_lattice h) {
    if (!h) return FLB_ERR_ARG;
    return check_device_error(h);
}

int flb_time(flb_lattice h, int64_t* t) {
    if (!h || !t) return FLB_ERR_ARG;
    *t = h->t;
    return FLB_OK;
}

int flb_set_time(flb_lattice h, int64_t t) {
    if (!h || t < 0 || t > (int64_t)UINT32_MAX) return FLB_ERR_ARG;
    h->t = t;
    return FLB_OK;
}

int flb_set_raw_sums(flb_lattice h, const double* S1, const double* S2, int64_t n_samples) {
    if (!h || !S1 || !S2 || n_samples < 0) return FLB_ERR_ARG;
    double acc[kSums];
    int k = 0;
    for (int i = 0; i < 9; ++i) acc[k++] = S1[i];
    for (int i = 0; i < 9; ++i)
        for (int j = i; j < 9; ++j) acc[k++] = S2[i * 9 + j];
    cudaError_t ce = cudaMemcpyAsync(h->acc, acc, sizeof(acc), cudaMemcpyHostToDevice, h->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
    if (ce != cudaSuccess) return FLB_ERR_CUDA;
    h->nsamp = n_samples;
    return FLB_OK;
}

int flb_error_location(flb_lattice h, int64_t* node, int64_t* step) {
    if (!h) return FLB_ERR_ARG;
    DevError e;
    cudaError_t ce = cudaMemcpyAsync(&e, h->err, sizeof(e), cudaMemcpyDeviceToHost, h->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
    if (ce != cudaSuccess) return FLB_ERR_CUDA;
    if (node) *node = e.code ? e.node : -1;
    if (step) *step = e.code ? e.step : -1;
    return FLB_OK;
}

int flb_reset_error(flb_lattice h) {
    if (!h) return FLB_ERR_ARG;
    h->sticky = 0;
    cudaError_t ce = cudaMemsetAsync(h->err, 0, sizeof(DevError), h->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
    return cuda_rc(ce);
}

int flb_raw_sums(flb_lattice h, double* S1, double* S2, int64_t* n_samples) {
    if (!h) return FLB_ERR_ARG;
    double acc[kSums];
    cudaError_t ce = cudaMemcpyAsync(acc, h->acc, sizeof(acc), cudaMemcpyDeviceToHost, h->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
    if (ce != cudaSuccess) return FLB_ERR_CUDA;
    const int rc = check_device_error(h);
    if (rc) return rc;
    if (S1)
        for (int i = 0; i < 9; ++i) S1[i] = acc[i];
    if (S2) {
        int k = 9;
        for (int i = 0; i < 9; ++i)
            for (int j = i; j < 9; ++j, ++k) S2[i * 9 + j] = S2[j * 9 + i] = acc[k];
    }
    if (n_samples) *n_samples = h->nsamp;
    return FLB_OK;
}


int flb_correlations(flb_lattice h, int32_t measure_basis, double* Cff, double* CMM,
                     double* mean_dev, int64_t* n_samples) {
    if (!h) return FLB_ERR_ARG;
    if (measure_basis != FLB_BASIS_STANDARD && measure_basis != FLB_BASIS_LOCAL)
        return FLB_ERR_ARG;
    int rc = check_device_error(h);
    if (rc) return rc;
    if (n_samples) *n_samples = h->nsamp;
    if (h->nsamp <= 0) return FLB_ERR_STATE;
    double* basis = h->small;
    double* res = h->small + 81;
    measure_basis_kernel<<<1, 32, 0, h->stream>>>(measure_basis, h->p.ux0, h->p.uy0, basis);
    finalize_kernel<<<1, 96, 0, h->stream>>>(h->acc, h->nsamp, basis, res);
    double host[171];
    cudaError_t ce = cudaGetLastError();
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(host, res, sizeof(host), cudaMemcpyDeviceToHost, h->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
    if (ce != cudaSuccess) return FLB_ERR_CUDA;
    if (Cff) std::memcpy(Cff, host, 81 * sizeof(double));
    if (CMM) std::memcpy(CMM, host + 81, 81 * sizeof(double));
    if (mean_dev) std::memcpy(mean_dev, host + 162, 9 * sizeof(double));
    return FLB_OK;
}

int flb_conservation(flb_lattice h, double sums[3]) {
    if (!h || !sums) return FLB_ERR_ARG;
    double* part = h->small + 81 + 171 + 3;
    double* res = h->small + 81 + 171;
    if (h->p.precision == FLB_FP64)
        conservation_kernel<double><<<h->nblocks, kStepThreads, 0, h->stream>>>(
            (const double*)h->buf[h->cur], h->geo, part, DevCodec());
    else if (h->p.precision == FLB_FP32)
        conservation_kernel<float><<<h->nblocks, kStepThreads, 0, h->stream>>>(
            (const float*)h->buf[h->cur], h->geo, part, DevCodec());
    else
        conservation_kernel<__half><<<h->nblocks, kStepThreads, 0, h->stream>>>(
            (const __half*)h->buf[h->cur], h->geo, part, dev_codec(h));
    sum3_kernel<<<1, 32, 0, h->stream>>>(part, h->nblocks, res);
    cudaError_t ce = cudaGetLastError();
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(sums, res, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
    if (ce != cudaSuccess) return FLB_ERR_CUDA;
    return check_device_error(h);
}

int flb_state_difference(flb_lattice a, flb_lattice b, double out[3]) {
    if (!a || !b || !out || a->p.Lx != b->p.Lx || a->p.Ly != b->p.Ly) return FLB_ERR_ARG;
    StateView va{a->buf[a->cur], a->p.precision, a->geo, dev_codec(a)};
    StateView vb{b->buf[b->cur], b->p.precision, b->geo, dev_codec(b)};
    const int grid = grid_for((long long)a->p.Lx * a->p.Ly);
    double* part = nullptr;
    if (cudaMalloc(&part, sizeof(double) * 3 * grid) != cudaSuccess) {
        cudaGetLastError();
        return FLB_ERR_OOM;
    }
    // both lattices' pending steps first
    cudaError_t ce = cudaStreamSynchronize(b->stream);
    if (ce == cudaSuccess) {
        state_difference_kernel<<<grid, kStepThreads, 0, a->stream>>>(va, vb, part);
        ce = cudaGetLastError();
    }
    std::vector<double> host(3 * (size_t)grid);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(host.data(), part, sizeof(double) * host.size(),
                             cudaMemcpyDeviceToHost, a->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(a->stream);
    cudaFree(part);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return FLB_ERR_CUDA;
    }
    double mx = 0.0, ss = 0.0, mb = 0.0;
    for (int k = 0; k < grid; ++k) {
        mx = std::max(mx, host[3 * k]);
        ss += host[3 * k + 1];
        mb = std::max(mb, host[3 * k + 2]);
    }
    out[0] = mx;
    out[1] = std::sqrt(ss / (9.0 * (double)a->p.Lx * (double)a->p.Ly));
    out[2] = mb;
    return FLB_OK;
}

// The device address of page-locked host memory, or null for other memory:
// the state I/O kernels then read or write the caller's host array themselves
// (one pass over the host link, no device staging buffer).
static double* pinned_view(const void* host) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? static_cast<double*>(a.devicePointer) : nullptr;
}

int flb_get_populations(flb_lattice h, double* host_out) {
    if (!h || !host_out) return FLB_ERR_ARG;
    const size_t n = (size_t)9 * h->p.Lx * h->p.Ly;
    double* direct = pinned_view(host_out);
    double* tmp = direct;
    if (!direct && cudaMalloc(&tmp, n * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return FLB_ERR_OOM;
    }
    const int grid = grid_for((long long)h->p.Lx * h->p.Ly);
    if (h->p.precision == FLB_FP64)
        gather_state_kernel<double><<<grid, 256, 0, h->stream>>>((const double*)h->buf[h->cur],
                                                                 h->geo, tmp);
    else if (h->p.precision == FLB_FP32)
        gather_state_kernel<float><<<grid, 256, 0, h->stream>>>((const float*)h->buf[h->cur],
                                                                h->geo, tmp);
    else
        gather_dev_kernel<<<grid, 256, 0, h->stream>>>((const __half*)h->buf[h->cur], h->geo,
                                                       dev_codec(h), tmp);
    cudaError_t ce = cudaGetLastError();
    if (ce == cudaSuccess && !direct)
        ce = cudaMemcpyAsync(host_out, tmp, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
    if (!direct) cudaFree(tmp);
    if (ce != cudaSuccess) return FLB_ERR_CUDA;
    return check_device_error(h);
}

int flb_set_populations(flb_lattice h, const double* host_in) {
    if (!h || !host_in) return FLB_ERR_ARG;
    const size_t n = (size_t)9 * h->p.Lx * h->p.Ly;
    double* direct = pinned_view(host_in);
    double* tmp = direct;
    if (!direct && cudaMalloc(&tmp, n * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return FLB_ERR_OOM;
    }
    cudaError_t ce = direct ? cudaSuccess
                            : cudaMemcpyAsync(tmp, host_in, n * sizeof(double),
                                              cudaMemcpyHostToDevice, h->stream);
    const int grid = grid_for((long long)h->p.Lx * h->p.Ly);
    if (ce == cudaSuccess) {
        if (h->p.precision == FLB_FP64)
            scatter_state_kernel<double><<<grid, 256, 0, h->stream>>>(tmp, h->geo,
                                                                      (double*)h->buf[h->cur]);
        else if (h->p.precision == FLB_FP32)
            scatter_state_kernel<float><<<grid, 256, 0, h->stream>>>(tmp, h->geo,
                                                                     (float*)h->buf[h->cur]);
        else
            scatter_dev_kernel<<<grid, 256, 0, h->stream>>>(tmp, h->geo, dev_codec(h),
                                                            (__half*)h->buf[h->cur]);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) ce = cudaMemsetAsync(h->err, 0, sizeof(DevError), h->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
    if (!direct) cudaFree(tmp);
    h->sticky = 0;
    return cuda_rc(ce);
}

int flb_run_host(const flb_params* p, const double* f_in, int64_t nsteps, int64_t warmup,
                 int64_t every, double* f_out, double* S1, double* S2, int64_t* n_samples) {
    if (!p || nsteps < 0) return FLB_ERR_ARG;
    flb_lattice h = nullptr;
    int rc = flb_create(p, nullptr, 0, nullptr, &h);
    if (rc) return rc;
    if (f_in) rc = flb_set_populations(h, f_in);
    if (!rc) rc = flb_set_sampling(h, warmup, every);
    if (!rc) rc = flb_step(h, nsteps);
    if (!rc) rc = flb_sync(h);
    if (!rc && f_out) rc = flb_get_populations(h, f_out);
    if (!rc && (S1 || S2 || n_samples)) rc = flb_raw_sums(h, S1, S2, n_samples);
    const int drc = flb_destroy(h);
    return rc ? rc : drc;
}

int flb_noise_draws(uint64_t seed, uint32_t replica, uint32_t step, const uint32_t* nodes,
                    int32_t n, int32_t precision, uint32_t* fields, double* normals) {
    if (n < 0 || (n > 0 && (!nodes || !fields || !normals))) return FLB_ERR_ARG;
    if (precision != FLB_FP64 && precision != FLB_FP32) return FLB_ERR_ARG;
    if (n == 0) return FLB_OK;
    uint32_t *d_nodes = nullptr, *d_fields = nullptr;
    double* d_normals = nullptr;
    cudaError_t ce = cudaMalloc(&d_nodes, n * sizeof(uint32_t));
    if (ce == cudaSuccess) ce = cudaMalloc(&d_fields, 6 * (size_t)n * sizeof(uint32_t));
    if (ce == cudaSuccess) ce = cudaMalloc(&d_normals, 6 * (size_t)n * sizeof(double));
    if (ce == cudaSuccess)
        ce = cudaMemcpy(d_nodes, nodes, n * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) {
        const int grid = (n + 127) / 128;
        if (precision == FLB_FP64)
            noise_draws_kernel<double><<<grid, 128>>>(seed, replica, step, d_nodes, n, d_fields,
                                                      d_normals);
        else
            noise_draws_kernel<float><<<grid, 128>>>(seed, replica, step, d_nodes, n, d_fields,
                                                     d_normals);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess)
        ce = cudaMemcpy(fields, d_fields, 6 * (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (ce == cudaSuccess)
        ce = cudaMemcpy(normals, d_normals, 6 * (size_t)n * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(d_nodes);
    cudaFree(d_fields);
    cudaFree(d_normals);
    return cuda_rc(ce);
}

int flb_collide_nodes(const flb_params* p, const double* g, const uint32_t* node_ids,
                      uint32_t step, int32_t n, double* fstar, int32_t* status) {
    if (!p || n < 0 || (n > 0 && (!g || !node_ids || !fstar))) return FLB_ERR_ARG;
    flb_params q = *p;
    q.Lx = q.Ly = 1;
    if (!valid_params(&q)) return FLB_ERR_ARG;
    if (n == 0) return FLB_OK;
    double *d_g = nullptr, *d_f = nullptr;
    uint32_t* d_ids = nullptr;
    int* d_st = nullptr;
    cudaError_t ce = cudaMalloc(&d_g, 9 * (size_t)n * sizeof(double));
    if (ce == cudaSuccess) ce = cudaMalloc(&d_f, 9 * (size_t)n * sizeof(double));
    if (ce == cudaSuccess) ce = cudaMalloc(&d_ids, (size_t)n * sizeof(uint32_t));
    if (ce == cudaSuccess) ce = cudaMalloc(&d_st, (size_t)n * sizeof(int));
    if (ce == cudaSuccess)
        ce = cudaMemcpy(d_g, g, 9 * (size_t)n * sizeof(double), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess)
        ce = cudaMemcpy(d_ids, node_ids, (size_t)n * sizeof(uint32_t), cudaMemcpyHostToDevice);
    const float* l32 = nullptr;
    const double* l64 = nullptr;
    if (ce == cudaSuccess && p->basis == FLB_BASIS_LOCAL_LUT && lut_tables(&l32, &l64) != FLB_OK)
        ce = cudaErrorUnknown;
    if (ce == cudaSuccess) {
        const int grid = (n + 127) / 128;
        if (p->precision == FLB_FP64) {
            const CollideConst<double> cc = collide_const<double>(p);
            if (p->basis == FLB_BASIS_STANDARD)
                collide_nodes_kernel<double, 0><<<grid, 128>>>(d_g, d_ids, step, n, cc, l64, d_f, d_st);
            else if (p->basis == FLB_BASIS_LOCAL)
                collide_nodes_kernel<double, 1><<<grid, 128>>>(d_g, d_ids, step, n, cc, l64, d_f, d_st);
            else
                collide_nodes_kernel<double, 2><<<grid, 128>>>(d_g, d_ids, step, n, cc, l64, d_f, d_st);
        } else {
            const CollideConst<float> cc = collide_const<float>(p);
            if (p->basis == FLB_BASIS_STANDARD)
                collide_nodes_kernel<float, 0><<<grid, 128>>>(d_g, d_ids, step, n, cc, l32, d_f, d_st);
            else if (p->basis == FLB_BASIS_LOCAL)
                collide_nodes_kernel<float, 1><<<grid, 128>>>(d_g, d_ids, step, n, cc, l32, d_f, d_st);
            else
                collide_nodes_kernel<float, 2><<<grid, 128>>>(d_g, d_ids, step, n, cc, l32, d_f, d_st);
        }
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess)
        ce = cudaMemcpy(fstar, d_f, 9 * (size_t)n * sizeof(double), cudaMemcpyDeviceToHost);
    int* st = nullptr;
    if (ce == cudaSuccess && status) {
        st = new (std::nothrow) int[n];
        if (st) {
            ce = cudaMemcpy(st, d_st, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost);
            for (int k = 0; k < n && ce == cudaSuccess; ++k) status[k] = map_status(st[k]);
            delete[] st;
        }
    }
    cudaFree(d_g);
    cudaFree(d_f);
    cudaFree(d_ids);
    cudaFree(d_st);
    return cuda_rc(ce);
}

int flb_wait_probe(int64_t limit_cycles) {
    if (limit_cycles < 0 || limit_cycles > 4000000000LL) return FLB_ERR_ARG;
    DevError* err = nullptr;
    if (cudaMalloc(&err, sizeof(DevError)) != cudaSuccess) {
        cudaGetLastError();
        return FLB_ERR_OOM;
    }
    DevError e;
    cudaError_t ce = cudaMemset(err, 0, sizeof(DevError));
    if (ce == cudaSuccess) ce = wait_probe(limit_cycles, err, 0);
    if (ce == cudaSuccess) ce = cudaMemcpy(&e, err, sizeof(e), cudaMemcpyDeviceToHost);
    cudaFree(err);
    if (ce != cudaSuccess) return FLB_ERR_CUDA;
    return map_status(e.code);
}

}  // extern "C"
