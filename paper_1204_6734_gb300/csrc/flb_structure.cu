// flb_structure.cu -- static structure factors of the hydrodynamic fields
// (Eqs. sfactorr, sfactoru, rcorrelator): on a sampling step,
//   delta rho(x), delta j_x(x), delta j_y(x) of the pre-collision state,
//   their 2D transforms a(k) = sum_x a(x) exp(-i k.x), k = 2 pi (m_x/Lx, m_y/Ly),
//   and the FP64 sums of |drho(k)|^2, |dj_x(k)|^2 and dj_x(k) conj(dj_y(k)).
// The fields are formed from the deviations f_i - c_i, c = f^0(rho0, u0), whose
// moments are rho - rho0 and j - rho0 u0 exactly (c has moments rho0, rho0 u0).
//
// Two paths compute the transform, FP64 for FP64 lattices, FP32 otherwise:
//  * both sides powers of two (the fast path, two launches): one CTA per pair
//    of rows forms the fields from the pulled populations and transforms
//    them along x as one complex sequence per field (row y in the real part,
//    row y+1 in the imaginary part), then splits the two rows' spectra by
//    Hermitian symmetry and keeps m_x = 0..Lx/2; one CTA per column of that
//    half spectrum transforms along y and adds the three products to the
//    half-plane sums. The other half follows from S(-k) = S(k),
//    R(-k) = conj R(k) (real fields), applied when the sums are read.
//  * other sides: fields, row transforms, column transforms and the sums as
//    separate launches over the full plane, with a direct O(L^2) transform
//    for a side that is not a power of two.
// Each radix-2 transform runs in shared memory, input in bit-reversed order,
// with one padding element every 2^ps elements so that the bit-reversed
// scatter does not put a warp's 32 elements on one bank.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "../../include/flb.h"
#include "flb_io.cuh"
#include "flb_layout.cuh"
#include "flb_structure.h"

namespace flb {

namespace {

template <class R>
struct Cx {
    R re, im;
};

template <class R>
struct Ref9 {
    R v[9];
};

template <class R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

// f_i - c_i of one stored value, in the transform precision R.
template <class R>
__device__ __forceinline__ R pop_dev(const double* b, long long k, int i, const DevCodec&,
                                     const Ref9<R>& c) {
    return (R)b[k] - c.v[i];
}
template <class R>
__device__ __forceinline__ R pop_dev(const float* b, long long k, int i, const DevCodec&,
                                     const Ref9<R>& c) {
    return (R)b[k] - c.v[i];
}
template <class R>
__device__ __forceinline__ R pop_dev(const __half* b, long long k, int i, const DevCodec& d,
                                     const Ref9<R>& c) {
    return ((R)d.ref[i] - c.v[i]) + (R)d.scale * (R)__half2float(b[k]);
}

// delta rho, delta j_x, delta j_y at node (x, y) of the pre-collision state,
// f_i(x) = buf at x - v_i (pull).
template <class T, class R>
__device__ __forceinline__ void node_fields(const T* buf, const Geometry& geo, const DevCodec& codec,
                                            const Ref9<R>& c, int x, int y, R& r, R& jx, R& jy) {
    R d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int xs = wrap(x - cvx(i), geo.Lx), ys = wrap(y - cvy(i), geo.Ly);
        d[i] = pop_dev(buf, at(geo, i, xs, ys), i, codec, c);
    }
    r = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
    jx = (d[1] - d[3]) + ((d[5] - d[6]) + (d[8] - d[7]));
    jy = (d[2] - d[4]) + ((d[5] + d[6]) - (d[7] + d[8]));
}

__host__ __device__ __forceinline__ int log2i(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

__device__ __forceinline__ int bitrev(int v, int bits) { return (int)(__brev((unsigned)v) >> (32 - bits)); }

__device__ __forceinline__ int pad(int i, int ps) { return i + (i >> ps); }

// In-place radix-2 decimation-in-time transform of `count` sequences of
// length 2^bits in shared memory, sequence q at s + q * seq, element i at
// pad(i); input in bit-reversed order, output in natural order.
// tw[m] = exp(-2 pi i m / L), m < L / 2.
template <class R>
__device__ __forceinline__ void fft_pow2(Cx<R>* s, int bits, int count, int seq, int ps,
                                         const Cx<R>* __restrict__ tw) {
    const int hb = bits - 1;
    const int nb = count << hb;
    for (int lh = 0; lh < bits; ++lh) {
        const int half = 1 << lh;
        for (int j = threadIdx.x; j < nb; j += blockDim.x) {
            const int q = j >> hb, b = j & ((1 << hb) - 1);
            const int pos = b & (half - 1);
            const int i1 = ((b >> lh) << (lh + 1)) + pos, i2 = i1 + half;
            Cx<R>* x = s + q * seq;
            const Cx<R> w = tw[pos << (hb - lh)];
            const Cx<R> t = cmul(w, x[pad(i2, ps)]);
            const Cx<R> u = x[pad(i1, ps)];
            x[pad(i1, ps)] = {u.re + t.re, u.im + t.im};
            x[pad(i2, ps)] = {u.re - t.re, u.im - t.im};
        }
        __syncthreads();
    }
}

constexpr int kThreads = 512;

// ---- fast path: both sides powers of two ----------------------------------

// One CTA per row pair (y0, y0 + 1): H[f][y][m], m = 0..Lx/2 (row pitch Hx),
// the x-transform of field f (0: drho, 1: dj_x, 2: dj_y) of row y.
template <class T, class R>
__global__ void __launch_bounds__(kThreads) rows_pair_kernel(const T* __restrict__ buf, Geometry geo,
                                                             DevCodec codec, Ref9<R> c, int bits,
                                                             int ps, const Cx<R>* __restrict__ tw,
                                                             Cx<R>* __restrict__ H, int Hx) {
    extern __shared__ __align__(16) unsigned char raw[];
    Cx<R>* s = reinterpret_cast<Cx<R>*>(raw);
    const int Lx = geo.Lx, Ly = geo.Ly;
    const int seq = pad(Lx, ps) + 1;
    const int y0 = 2 * blockIdx.x, y1 = y0 + 1;
    for (int x = threadIdx.x; x < Lx; x += blockDim.x) {
        R r0, a0, b0, r1, a1, b1;
        node_fields(buf, geo, codec, c, x, y0, r0, a0, b0);
        node_fields(buf, geo, codec, c, x, y1, r1, a1, b1);
        const int p = pad(bitrev(x, bits), ps);
        s[p] = {r0, r1};
        s[seq + p] = {a0, a1};
        s[2 * seq + p] = {b0, b1};
    }
    __syncthreads();
    fft_pow2(s, bits, 3, seq, ps, tw);
    // z = a + i b with a, b real: A(m) = (Z(m) + conj Z(-m)) / 2,
    // B(m) = (Z(m) - conj Z(-m)) / (2i)
    for (int f = 0; f < 3; ++f) {
        const Cx<R>* z = s + f * seq;
        Cx<R>* out0 = H + ((size_t)f * Ly + y0) * Hx;
        Cx<R>* out1 = out0 + Hx;
        for (int m = threadIdx.x; m < Hx; m += blockDim.x) {
            const Cx<R> u = z[pad(m, ps)], w = z[pad((Lx - m) & (Lx - 1), ps)];
            out0[m] = {R(0.5) * (u.re + w.re), R(0.5) * (u.im - w.im)};
            out1[m] = {R(0.5) * (u.im + w.im), R(0.5) * (w.re - u.re)};
        }
    }
}

// One CTA per block of C columns (C a power of two) of the half spectrum: the
// y-transform of each, then acc[q][m_x][m_y] += |drho|^2 (q = 0), |dj_x|^2
// (1), Re and Im of dj_x conj(dj_y) (2, 3); acc[q] is Hx x Ly, m_y fastest.
template <class R>
__global__ void __launch_bounds__(kThreads) cols_acc_kernel(const Cx<R>* __restrict__ H, int Ly,
                                                            int Hx, int bits, int ps, int lc,
                                                            const Cx<R>* __restrict__ tw,
                                                            double* __restrict__ acc) {
    extern __shared__ __align__(16) unsigned char raw[];
    Cx<R>* s = reinterpret_cast<Cx<R>*>(raw);
    const int C = 1 << lc;
    const int seq = pad(Ly, ps) + 1;
    const int c0 = blockIdx.x * C;
    constexpr int kBatch = 4;
    for (int f = 0; f < 3; ++f) {
        const Cx<R>* src = H + (size_t)f * Ly * Hx + c0;
        Cx<R>* dst = s + f * C * seq;
        // kBatch independent loads in flight per thread before the stores
        for (int j0 = threadIdx.x; j0 < (Ly << lc); j0 += kBatch * blockDim.x) {
            Cx<R> v[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int j = j0 + u * blockDim.x;
                const int y = j >> lc, cc = j & (C - 1);
                v[u] = (j < (Ly << lc) && c0 + cc < Hx) ? src[(size_t)y * Hx + cc] : Cx<R>{R(0), R(0)};
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int j = j0 + u * blockDim.x;
                if (j < (Ly << lc)) {
                    const int y = j >> lc, cc = j & (C - 1);
                    dst[cc * seq + pad(bitrev(y, bits), ps)] = v[u];
                }
            }
        }
    }
    __syncthreads();
    fft_pow2(s, bits, 3 * C, seq, ps, tw);
    for (int j = threadIdx.x; j < (Ly << lc); j += blockDim.x) {
        const int cc = j >> bits, m = j & (Ly - 1);
        const int col = c0 + cc;
        if (col >= Hx) continue;
        const Cx<R> a = s[cc * seq + pad(m, ps)];
        const Cx<R> b = s[(C + cc) * seq + pad(m, ps)];
        const Cx<R> d = s[(2 * C + cc) * seq + pad(m, ps)];
        const size_t k = (size_t)col * Ly + m, Q = (size_t)Hx * Ly;
        const double ar = a.re, ai = a.im, br = b.re, bi = b.im, dr = d.re, di = d.im;
        acc[k] += ar * ar + ai * ai;
        acc[Q + k] += br * br + bi * bi;
        acc[2 * Q + k] += br * dr + bi * di;
        acc[3 * Q + k] += bi * dr - br * di;
    }
}

// ---- general path: any sides -----------------------------------------------

template <class T, class R>
__global__ void fields_kernel(const T* __restrict__ buf, Geometry geo, DevCodec codec, Ref9<R> c,
                              Cx<R>* A, Cx<R>* B, Cx<R>* D) {
    const int N = geo.Lx * geo.Ly;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        const int y = n / geo.Lx, x = n - y * geo.Lx;
        R r, jx, jy;
        node_fields(buf, geo, codec, c, x, y, r, jx, jy);
        A[n] = {r, R(0)};
        B[n] = {jx, R(0)};
        D[n] = {jy, R(0)};
    }
}

// One CTA per row of each field (blockIdx.y): in-place radix-2 transform.
template <class R>
__global__ void fft_rows_kernel(Cx<R>* F, int Lx, int Ly, int ps, const Cx<R>* tw) {
    extern __shared__ __align__(16) unsigned char raw[];
    Cx<R>* s = reinterpret_cast<Cx<R>*>(raw);
    Cx<R>* row = F + ((size_t)blockIdx.y * Ly + blockIdx.x) * Lx;
    const int bits = log2i(Lx);
    for (int i = threadIdx.x; i < Lx; i += blockDim.x) s[pad(bitrev(i, bits), ps)] = row[i];
    __syncthreads();
    fft_pow2(s, bits, 1, 0, ps, tw);
    for (int i = threadIdx.x; i < Lx; i += blockDim.x) row[i] = s[pad(i, ps)];
}

// One CTA per column of each field: in-place radix-2 transform.
template <class R>
__global__ void fft_cols_kernel(Cx<R>* F, int Lx, int Ly, int ps, const Cx<R>* tw) {
    extern __shared__ __align__(16) unsigned char raw[];
    Cx<R>* s = reinterpret_cast<Cx<R>*>(raw);
    Cx<R>* col = F + (size_t)blockIdx.y * Ly * Lx + blockIdx.x;
    const int bits = log2i(Ly);
    for (int y = threadIdx.x; y < Ly; y += blockDim.x) s[pad(bitrev(y, bits), ps)] = col[(size_t)y * Lx];
    __syncthreads();
    fft_pow2(s, bits, 1, 0, ps, tw);
    for (int y = threadIdx.x; y < Ly; y += blockDim.x) col[(size_t)y * Lx] = s[pad(y, ps)];
}

// Direct transform of one row of each field (any L):
// out[m] = sum_x in[x] tw[(m x) mod L], tw[m] = exp(-2 pi i m / L), m < L.
template <class R>
__global__ void dft_rows_kernel(Cx<R>* F, int Lx, int Ly, const Cx<R>* tw) {
    extern __shared__ __align__(16) unsigned char raw[];
    Cx<R>* s = reinterpret_cast<Cx<R>*>(raw);
    Cx<R>* row = F + ((size_t)blockIdx.y * Ly + blockIdx.x) * Lx;
    for (int i = threadIdx.x; i < Lx; i += blockDim.x) s[i] = row[i];
    __syncthreads();
    for (int m = threadIdx.x; m < Lx; m += blockDim.x) {
        R re = 0, im = 0;
        int idx = 0;
        for (int x = 0; x < Lx; ++x) {
            const Cx<R> v = cmul(s[x], tw[idx]);
            re += v.re;
            im += v.im;
            idx += m;
            if (idx >= Lx) idx -= Lx;
        }
        row[m] = {re, im};
    }
}

// Direct transform of one column of each field (any L).
template <class R>
__global__ void dft_cols_kernel(Cx<R>* F, int Lx, int Ly, const Cx<R>* tw) {
    extern __shared__ __align__(16) unsigned char raw[];
    Cx<R>* s = reinterpret_cast<Cx<R>*>(raw);
    Cx<R>* col = F + (size_t)blockIdx.y * Ly * Lx + blockIdx.x;
    for (int y = threadIdx.x; y < Ly; y += blockDim.x) s[y] = col[(size_t)y * Lx];
    __syncthreads();
    for (int m = threadIdx.x; m < Ly; m += blockDim.x) {
        R re = 0, im = 0;
        int idx = 0;
        for (int y = 0; y < Ly; ++y) {
            const Cx<R> v = cmul(s[y], tw[idx]);
            re += v.re;
            im += v.im;
            idx += m;
            if (idx >= Ly) idx -= Ly;
        }
        col[(size_t)m * Lx] = {re, im};
    }
}

template <class R>
__global__ void accumulate_kernel(const Cx<R>* A, const Cx<R>* B, const Cx<R>* D, int N, double* acc) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        const double ar = A[k].re, ai = A[k].im, br = B[k].re, bi = B[k].im;
        const double dr = D[k].re, di = D[k].im;
        acc[k] += ar * ar + ai * ai;
        acc[N + k] += br * br + bi * bi;
        acc[2 * (size_t)N + k] += br * dr + bi * di;   // Re(b conj(d))
        acc[3 * (size_t)N + k] += bi * dr - br * di;   // Im(b conj(d))
    }
}

bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Padding shift for a transform of length L: one element every L / 32, so
// that 32 consecutive bit-reversed indices land on distinct banks; none for
// L < 32 (those indices are already distinct modulo 32).
int pad_shift(int L) {
    const int b = log2i(L);
    return b >= 5 ? b - 5 : b;
}

size_t padded(int L, int ps) { return (size_t)L + ((size_t)L >> ps) + 1; }

constexpr size_t kGeneralSmem = 160 * 1024;

}  // namespace

struct StructSampler {
    int Lx = 0, Ly = 0, rbytes = 8;   // transform precision: 8 FP64, 4 FP32
    bool fast = false;                // both sides powers of two, fused launches
    int Hx = 0;                       // fast: columns of the half spectrum, Lx/2 + 1
    int lc = 0;                       // fast: log2 of the columns per CTA
    size_t smem_rows = 0, smem_cols = 0;
    void* fields = nullptr;           // general: 3 Lx Ly complex; fast: 3 Ly Hx complex
    double* acc = nullptr;            // general: 4 x [Ly][Lx]; fast: 4 x [Hx][Ly]
    size_t acc_count = 0;             // doubles in acc
    void* twx = nullptr;              // twiddles along x and y
    void* twy = nullptr;
    int64_t nsamp = 0;
};

namespace {

template <class R>
cudaError_t upload_twiddles(int L, void** out) {
    // power of two: exp(-2 pi i m / L) for m < L/2; otherwise all m < L
    const int n = pow2(L) ? std::max(1, L / 2) : L;
    std::vector<Cx<R>> h(n);
    for (int m = 0; m < n; ++m) {
        const double a = -2.0 * M_PI * (double)m / (double)L;
        h[m] = {(R)std::cos(a), (R)std::sin(a)};
    }
    cudaError_t ce = cudaMalloc(out, sizeof(Cx<R>) * n);
    if (ce == cudaSuccess)
        ce = cudaMemcpy(*out, h.data(), sizeof(Cx<R>) * n, cudaMemcpyHostToDevice);
    return ce;
}

template <class T, class R>
cudaError_t sample_fast(StructSampler* s, const T* buf, const Geometry& geo, const DevCodec& codec,
                        const Ref9<R>& c, cudaStream_t st) {
    Cx<R>* H = (Cx<R>*)s->fields;
    const int bx = log2i(s->Lx), by = log2i(s->Ly);
    cudaError_t ce = cudaFuncSetAttribute(rows_pair_kernel<T, R>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->smem_rows);
    if (ce != cudaSuccess) return ce;
    rows_pair_kernel<T, R><<<s->Ly / 2, kThreads, s->smem_rows, st>>>(
        buf, geo, codec, c, bx, pad_shift(s->Lx), (const Cx<R>*)s->twx, H, s->Hx);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return ce;
    ce = cudaFuncSetAttribute(cols_acc_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)s->smem_cols);
    if (ce != cudaSuccess) return ce;
    const int C = 1 << s->lc;
    cols_acc_kernel<R><<<(s->Hx + C - 1) / C, kThreads, s->smem_cols, st>>>(
        H, s->Ly, s->Hx, by, pad_shift(s->Ly), s->lc, (const Cx<R>*)s->twy, s->acc);
    return cudaGetLastError();
}

template <class T, class R>
cudaError_t sample_general(StructSampler* s, const T* buf, const Geometry& geo,
                           const DevCodec& codec, const Ref9<R>& c, cudaStream_t st) {
    const int Lx = s->Lx, Ly = s->Ly, N = Lx * Ly;
    Cx<R>* F = (Cx<R>*)s->fields;
    const Cx<R>* tx = (const Cx<R>*)s->twx;
    const Cx<R>* ty = (const Cx<R>*)s->twy;
    fields_kernel<T, R><<<std::min(4096, (N + 255) / 256), 256, 0, st>>>(buf, geo, codec, c, F, F + N,
                                                                        F + 2 * (size_t)N);
    cudaError_t ce = cudaGetLastError();
    if (ce == cudaSuccess && Lx > 1) {
        if (pow2(Lx)) {
            const int ps = pad_shift(Lx);
            const size_t sm = sizeof(Cx<R>) * padded(Lx, ps);
            ce = cudaFuncSetAttribute(fft_rows_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (ce == cudaSuccess) fft_rows_kernel<R><<<dim3(Ly, 3), kThreads, sm, st>>>(F, Lx, Ly, ps, tx);
        } else {
            const size_t sm = sizeof(Cx<R>) * Lx;
            ce = cudaFuncSetAttribute(dft_rows_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (ce == cudaSuccess) dft_rows_kernel<R><<<dim3(Ly, 3), 256, sm, st>>>(F, Lx, Ly, tx);
        }
        if (ce == cudaSuccess) ce = cudaGetLastError();
    }
    if (ce == cudaSuccess && Ly > 1) {
        if (pow2(Ly)) {
            const int ps = pad_shift(Ly);
            const size_t sm = sizeof(Cx<R>) * padded(Ly, ps);
            ce = cudaFuncSetAttribute(fft_cols_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (ce == cudaSuccess) fft_cols_kernel<R><<<dim3(Lx, 3), kThreads, sm, st>>>(F, Lx, Ly, ps, ty);
        } else {
            const size_t sm = sizeof(Cx<R>) * Ly;
            ce = cudaFuncSetAttribute(dft_cols_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (ce == cudaSuccess) dft_cols_kernel<R><<<dim3(Lx, 3), 256, sm, st>>>(F, Lx, Ly, ty);
        }
        if (ce == cudaSuccess) ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) {
        accumulate_kernel<R><<<std::min(4096, (N + 255) / 256), 256, 0, st>>>(F, F + N, F + 2 * (size_t)N,
                                                                              N, s->acc);
        ce = cudaGetLastError();
    }
    return ce;
}

template <class T, class R>
cudaError_t sample_typed(StructSampler* s, const void* buf, const Geometry& geo, const DevCodec& codec,
                         const double* ref, cudaStream_t st) {
    Ref9<R> c;
    for (int i = 0; i < 9; ++i) c.v[i] = (R)ref[i];
    return s->fast ? sample_fast<T, R>(s, (const T*)buf, geo, codec, c, st)
                   : sample_general<T, R>(s, (const T*)buf, geo, codec, c, st);
}

}  // namespace

int structure_create(StructSampler** out, int Lx, int Ly, int rbytes) {
    *out = nullptr;
    if ((rbytes != 4 && rbytes != 8) || Lx < 1 || Ly < 1) return FLB_ERR_ARG;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return FLB_ERR_CUDA;
    const size_t cb = 2 * (size_t)rbytes;   // bytes of one complex value
    StructSampler* s = new (std::nothrow) StructSampler();
    if (!s) return FLB_ERR_OOM;
    s->Lx = Lx;
    s->Ly = Ly;
    s->rbytes = rbytes;
    if (pow2(Lx) && pow2(Ly) && Lx >= 2 && Ly >= 2) {
        s->smem_rows = 3 * cb * padded(Lx, pad_shift(Lx));
        // columns per CTA: the most that leave room for two CTAs per SM, else one
        const size_t col = 3 * cb * padded(Ly, pad_shift(Ly));
        s->lc = 0;
        while (s->lc < 2 && col << (s->lc + 1) <= (size_t)optin / 2) ++s->lc;
        s->smem_cols = col << s->lc;
        s->fast = s->smem_rows <= (size_t)optin && s->smem_cols <= (size_t)optin;
    }
    // the general path holds one row (column) of complex values per CTA
    if (!s->fast && ((size_t)Lx * cb > kGeneralSmem || (size_t)Ly * cb > kGeneralSmem)) {
        delete s;
        return FLB_ERR_ARG;
    }
    const size_t N = (size_t)Lx * Ly;
    s->Hx = Lx / 2 + 1;
    const size_t nfield = s->fast ? 3 * (size_t)Ly * s->Hx : 3 * N;
    s->acc_count = s->fast ? 4 * (size_t)Ly * s->Hx : 4 * N;
    cudaError_t ce = cudaMalloc(&s->fields, nfield * cb);
    if (ce == cudaSuccess) ce = cudaMalloc(&s->acc, s->acc_count * sizeof(double));
    if (ce == cudaSuccess) ce = cudaMemset(s->acc, 0, s->acc_count * sizeof(double));
    if (ce == cudaSuccess)
        ce = rbytes == 8 ? upload_twiddles<double>(Lx, &s->twx) : upload_twiddles<float>(Lx, &s->twx);
    if (ce == cudaSuccess)
        ce = rbytes == 8 ? upload_twiddles<double>(Ly, &s->twy) : upload_twiddles<float>(Ly, &s->twy);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        structure_destroy(s);
        return FLB_ERR_OOM;
    }
    *out = s;
    return FLB_OK;
}

void structure_destroy(StructSampler* s) {
    if (!s) return;
    cudaFree(s->fields);
    cudaFree(s->acc);
    cudaFree(s->twx);
    cudaFree(s->twy);
    delete s;
}

cudaError_t structure_reset(StructSampler* s, cudaStream_t st) {
    s->nsamp = 0;
    return cudaMemsetAsync(s->acc, 0, s->acc_count * sizeof(double), st);
}

cudaError_t structure_sample(StructSampler* s, const void* buf, int precision, const Geometry& geo,
                             const DevCodec& codec, const double* ref, cudaStream_t st) {
    cudaError_t ce;
    if (s->rbytes == 8)
        ce = precision == FLB_FP64   ? sample_typed<double, double>(s, buf, geo, codec, ref, st)
             : precision == FLB_FP32 ? sample_typed<float, double>(s, buf, geo, codec, ref, st)
                                     : sample_typed<__half, double>(s, buf, geo, codec, ref, st);
    else
        ce = precision == FLB_FP64   ? sample_typed<double, float>(s, buf, geo, codec, ref, st)
             : precision == FLB_FP32 ? sample_typed<float, float>(s, buf, geo, codec, ref, st)
                                     : sample_typed<__half, float>(s, buf, geo, codec, ref, st);
    if (ce == cudaSuccess) s->nsamp += 1;
    return ce;
}

int structure_read(StructSampler* s, double* out, cudaStream_t st) {
    const size_t N = (size_t)s->Lx * s->Ly;
    if (!s->fast) {
        cudaError_t ce = cudaMemcpyAsync(out, s->acc, 4 * N * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        return ce == cudaSuccess ? FLB_OK : FLB_ERR_CUDA;
    }
    std::vector<double> half;
    try {
        half.resize(s->acc_count);
    } catch (const std::bad_alloc&) {
        return FLB_ERR_OOM;
    }
    cudaError_t ce = cudaMemcpyAsync(half.data(), s->acc, s->acc_count * sizeof(double),
                                     cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return FLB_ERR_CUDA;
    const int Lx = s->Lx, Ly = s->Ly, Hx = s->Hx;
    const size_t Q = (size_t)Hx * Ly;
    for (int q = 0; q < 4; ++q)
        for (int my = 0; my < Ly; ++my)
            for (int mx = 0; mx < Lx; ++mx) {
                // m_x > Lx/2: the value at -k; Im R changes sign there
                const bool mirror = mx >= Hx;
                const int hx = mirror ? Lx - mx : mx, hy = mirror ? (Ly - my) & (Ly - 1) : my;
                const double v = half[q * Q + (size_t)hx * Ly + hy];
                out[q * N + (size_t)my * Lx + mx] = (mirror && q == 3) ? -v : v;
            }
    return FLB_OK;
}

int64_t structure_samples(const StructSampler* s) { return s ? s->nsamp : 0; }

}  // namespace flb
