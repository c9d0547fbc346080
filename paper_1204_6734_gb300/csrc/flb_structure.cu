// flb_structure.cu -- static structure factors of the hydrodynamic fields
// (Eqs. sfactorr, sfactoru, rcorrelator): on a sampling step,
//   delta rho(x), delta j_x(x), delta j_y(x) of the pre-collision state,
//   their 2D transforms a(k) = sum_x a(x) exp(-i k.x), k = 2 pi (m_x/Lx, m_y/Ly),
//   and the FP64 sums of |drho(k)|^2, |dj_x(k)|^2 and dj_x(k) conj(dj_y(k)).
// The fields are formed from the deviations f_i - c_i, c = f^0(rho0, u0), whose
// moments are rho - rho0 and j - rho0 u0 exactly (c has moments rho0, rho0 u0).
//
// Two paths compute the transform, FP64 for FP64 lattices, FP32 otherwise:
//  * both sides powers of two up to 4096 (the fast path, two launches): one
//    CTA per pair of rows forms the fields from the pulled populations and
//    transforms them along x as one complex sequence per field (row y in the
//    real part, row y+1 in the imaginary part), then splits the two rows'
//    spectra by Hermitian symmetry and keeps m_x = 0..Lx/2, written
//    column-major; one CTA per column of that half spectrum transforms along
//    y and adds the three products to the half-plane sums. The other half
//    follows from S(-k) = S(k), R(-k) = conj R(k) (real fields), applied when
//    the sums are read.
//  * other sides: fields, row transforms, column transforms and the sums as
//    separate launches over the full plane, with a direct O(L^2) transform
//    for a side that is not a power of two.
// The power-of-two transforms are in-place Stockham passes in shared memory
// (radix 8 or 16 in registers, natural order in and out).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <utility>
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

// Twiddle-table reads, in FP32 marked to stay in L1 (a pass touches at most a
// few KB of the table, while the transformed data streams past).
__device__ __forceinline__ Cx<float> ld_twiddle(const Cx<float>* p) {
    float2 v;
    asm("ld.global.nc.L1::evict_last.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return {v.x, v.y};
}
__device__ __forceinline__ Cx<double> ld_twiddle(const Cx<double>* p) { return *p; }

// Reads of data used once (spectra, partial sums): not kept in L1.
__device__ __forceinline__ float4 ld_stream(const float4* p) {
    float4 v;
    asm volatile("ld.global.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
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
    for (int i = 0; i < 9; ++i) d[i] = pop_dev(buf, pull_at(geo, i, x, y), i, codec, c);
    r = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
    jx = (d[1] - d[3]) + ((d[5] - d[6]) + (d[8] - d[7]));
    jy = (d[2] - d[4]) + ((d[5] + d[6]) - (d[7] + d[8]));
}

__host__ __device__ __forceinline__ int log2i(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

// Radix-R DFT of v[0..R-1] in registers (R = 2, 4, 8, 16), in place:
// v[k] <- sum_n v[n] exp(-2 pi i n k / R), as log2 R radix-2 stages on
// bit-reversed input; the twiddles are roots of unity of order 16, known
// constants, and the ones equal to 1 and -i cost no multiply.
__host__ __device__ constexpr double cos16(int e) {
    // cos(2 pi e / 16) for any integer e
    e &= 15;
    return e == 0 ? 1.0 : e == 1 || e == 15 ? 0.92387953251128675613 : e == 2 || e == 14 ? 0.70710678118654752440
         : e == 3 || e == 13 ? 0.38268343236508977173 : e == 4 || e == 12 ? 0.0
         : e == 5 || e == 11 ? -0.38268343236508977173 : e == 6 || e == 10 ? -0.70710678118654752440
         : e == 7 || e == 9 ? -0.92387953251128675613 : -1.0;
}

template <int R>
__host__ __device__ constexpr int rev_bits(int i) {
    int r = 0;
    for (int b = 1; b < R; b <<= 1) r = (r << 1) | ((i & b) ? 1 : 0);
    return r;
}

template <int R, class RT>
__device__ __forceinline__ void dft_reg(Cx<RT>* v) {
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int j = rev_bits<R>(i);
        if (i < j) {
            const Cx<RT> t = v[i];
            v[i] = v[j];
            v[j] = t;
        }
    }
#pragma unroll
    for (int h = 1; h < R; h <<= 1) {
#pragma unroll
        for (int g = 0; g < R; g += 2 * h) {
#pragma unroll
            for (int p = 0; p < h; ++p) {
                const int e = p * (8 / h);   // w = exp(-2 pi i p / (2h)) = exp(-2 pi i e / 16)
                const Cx<RT> b = v[g + p + h];
                Cx<RT> t;
                if (e == 0) {
                    t = b;
                } else if (e == 4) {
                    t = {b.im, -b.re};
                } else {
                    const RT c = (RT)cos16(e), sn = (RT)cos16(e - 4);   // sin(2 pi e / 16)
                    t = {b.re * c + b.im * sn, b.im * c - b.re * sn};
                }
                const Cx<RT> a = v[g + p];
                v[g + p] = {a.re + t.re, a.im + t.im};
                v[g + p + h] = {a.re - t.re, a.im - t.im};
            }
        }
    }
}

// Shared-memory position of element i of a sequence transformed with E
// elements per thread and pass. E = 8: a permutation within each aligned block
// of 128 elements, bits 4-6 of i XORed into bits 0-2 and bit 6 into bit 3, so
// that every access pattern of the radix-8 passes is free of bank conflicts
// for 8-byte elements (the 16 lanes of a half warp reach 16 distinct bank
// pairs): consecutive elements (the reads, the loads, the stores), stride 8
// (the first pass's writes) and runs of 8 a stride 64 apart (the second
// pass's writes); no padding. E = 16: one padding element every 16.
__host__ __device__ constexpr int spos8(int i) { return i ^ ((i >> 4) & 7) ^ (((i >> 6) & 1) << 3); }

template <int E>
__device__ __forceinline__ int spos(int i) {
    if constexpr (E == 16)
        return i + (i >> 4);
    else
        return spos8(i);
}

template <int E>
__host__ __device__ constexpr int padded_len(int L) {
    return E == 16 ? L + (L >> 4) + 1 : L;
}

// One Stockham pass of radix R (the autosort formulation of Govindaraju et
// al., SC'08) over `count` sequences of length L = 2^lgL, sequence q at
// s + q * seq: sub-transforms of size Ns = 2^lgNs become size Ns R. Butterfly
// j of a sequence reads elements j + r L/R, applies the twiddles
// exp(-2 pi i r (j mod Ns) / (Ns R)) from the table T[m] = exp(-2 pi i m / L),
// transforms them in registers and writes them to (j div Ns) Ns R +
// (j mod Ns) + r Ns. In place: a round of whole sequences is read into
// registers, the block synchronises, then writes. blockDim.x must be a
// multiple of the threads per sequence, L / min(E, L).
template <int E, int R, class RT>
__device__ __forceinline__ void stockham_pass(Cx<RT>* s, int lgL, int lgNs, int count, int seq,
                                              const Cx<RT>* __restrict__ T) {
    constexpr int lgR = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4;
    const int L = 1 << lgL;
    const int per = min(E, L) / R;           // butterflies per thread
    const int nj = L >> lgR;                 // butterflies per sequence
    const int tps = nj / per;                // threads per sequence
    const int spr = blockDim.x / tps;        // sequences per round
    const int Ns = 1 << lgNs;
    const int tsh = lgL - lgNs - lgR;        // twiddle index scale L / (Ns R)
    constexpr int PMAX = E / R;
    for (int q0 = 0; q0 < count; q0 += spr) {
        const int q = q0 + (int)threadIdx.x / tps;
        const int t = (int)threadIdx.x % tps;
        const bool active = q < count;
        Cx<RT>* x = s + q * seq;
        Cx<RT> v[PMAX][R];
        if (active) {
#pragma unroll
            for (int b = 0; b < PMAX; ++b) {
                if (b >= per) break;
                const int j = t + b * tps, k = j & (Ns - 1);
#pragma unroll
                for (int r = 0; r < R; ++r) v[b][r] = x[spos<E>(j + r * nj)];
                if (lgNs > 0) {
                    // w_r = exp(-2 pi i r k / (Ns R)) = w_1^r: w_1 read from the
                    // table (consecutive lanes read consecutive entries), the
                    // powers of two by squaring, the others as w_hi w_(r - hi),
                    // hi the largest power of two below r (at most four
                    // roundings deep)
                    Cx<RT> w[R];
                    w[1] = ld_twiddle(T + (k << tsh));
                    v[b][1] = cmul(v[b][1], w[1]);
#pragma unroll
                    for (int r = 2; r < R; ++r) {
                        const int hi = r >= 8 ? 8 : r >= 4 ? 4 : 2;
                        w[r] = hi == r ? cmul(w[r / 2], w[r / 2]) : cmul(w[hi], w[r - hi]);
                        v[b][r] = cmul(v[b][r], w[r]);
                    }
                }
                dft_reg<R>(v[b]);
            }
        }
        __syncthreads();
        if (active) {
#pragma unroll
            for (int b = 0; b < PMAX; ++b) {
                if (b >= per) break;
                const int j = t + b * tps, k = j & (Ns - 1);
                const int d = ((j >> lgNs) << (lgNs + lgR)) + k;
#pragma unroll
                for (int r = 0; r < R; ++r) x[spos<E>(d + r * Ns)] = v[b][r];
            }
        }
        __syncthreads();
    }
}

// Forward transform of `count` sequences of length 2^lgL in shared memory
// (natural order in and out, element i at spos<E>(i)): passes of radix E
// (8 or 16), then one of the remainder.
template <int E, class RT>
__device__ __forceinline__ void fft_seqs(Cx<RT>* s, int lgL, int count, int seq,
                                         const Cx<RT>* __restrict__ T) {
    constexpr int lgE = E == 16 ? 4 : 3;
    int lgNs = 0;
    for (; lgNs + lgE <= lgL; lgNs += lgE) stockham_pass<E, E, RT>(s, lgL, lgNs, count, seq, T);
    switch (lgL - lgNs) {
        case 1: stockham_pass<E, 2, RT>(s, lgL, lgNs, count, seq, T); break;
        case 2: stockham_pass<E, 4, RT>(s, lgL, lgNs, count, seq, T); break;
        case 3: stockham_pass<E, 8, RT>(s, lgL, lgNs, count, seq, T); break;
        default: break;
    }
}

// Elements per thread and pass: 8 in the fused kernels (two 512-thread CTAs
// per SM at 64 registers, no spills); in the general line transform 16 in
// FP32 and 8 in FP64 (lines up to 16384 and 8192 in 1024 threads).
constexpr int kEfast = 8;
template <class R>
struct Elines {
    static constexpr int E = sizeof(R) == 4 ? 16 : 8;
};

constexpr int kThreads = 512;
// Shared memory a column CTA may take so that two fit one SM (half of the
// 227 KB a CTA can opt into on sm_100 / sm_103).
constexpr int kColsSmemBudget = 232448 / 2;

// ---- the same radix-8 passes with the length 2^LG known at compile time ----
// (the FP32 kernels of the fused-field path): loop bounds, strides and the
// twiddle scale are constants, and the positions of a butterfly's elements
// come from one swizzled base per butterfly, spos8 being linear over XOR
// (spos8(a ^ b) = spos8(a) ^ spos8(b)) and a + b = a ^ b for the disjoint bit
// ranges of j and r nj (reads) and of d and r Ns (writes).
template <int LG, int R, int LGNS>
__device__ __forceinline__ void pass_c(Cx<float>* s, int count, int seq, const Cx<float>* __restrict__ T) {
    constexpr int lgR = R == 2 ? 1 : R == 4 ? 2 : 3;
    constexpr int L = 1 << LG;
    constexpr int per = (L < kEfast ? L : kEfast) / R;   // butterflies per thread
    constexpr int nj = L >> lgR;                         // butterflies per sequence
    constexpr int tps = nj / per;                        // threads per sequence
    constexpr int spr = kThreads / tps;                  // sequences per round
    constexpr int Ns = 1 << LGNS;
    constexpr int tsh = LG - LGNS - lgR;
    const int t = (int)threadIdx.x % tps, qt = (int)threadIdx.x / tps;
    for (int q0 = 0; q0 < count; q0 += spr) {
        const int q = q0 + qt;
        const bool active = q < count;
        Cx<float>* x = s + q * seq;
        Cx<float> v[per][R];
        if (active) {
#pragma unroll
            for (int b = 0; b < per; ++b) {
                const int j = t + b * tps;
                const int pj = spos8(j);
#pragma unroll
                for (int r = 0; r < R; ++r) v[b][r] = x[pj ^ spos8(r * nj)];
                if constexpr (LGNS > 0) {
                    // w_r = w_1^r as in stockham_pass
                    Cx<float> w[R];
                    w[1] = ld_twiddle(T + ((j & (Ns - 1)) << tsh));
                    v[b][1] = cmul(v[b][1], w[1]);
#pragma unroll
                    for (int r = 2; r < R; ++r) {
                        const int hi = r >= 4 ? 4 : 2;
                        w[r] = hi == r ? cmul(w[r / 2], w[r / 2]) : cmul(w[hi], w[r - hi]);
                        v[b][r] = cmul(v[b][r], w[r]);
                    }
                }
                dft_reg<R>(v[b]);
            }
        }
        __syncthreads();
        if (active) {
#pragma unroll
            for (int b = 0; b < per; ++b) {
                const int j = t + b * tps;
                const int pd = spos8(((j >> LGNS) << (LGNS + lgR)) + (j & (Ns - 1)));
#pragma unroll
                for (int r = 0; r < R; ++r) x[pd ^ spos8(r * Ns)] = v[b][r];
            }
        }
        __syncthreads();
    }
}

// Forward transform of `count` sequences of length 2^LG (element i at spos8(i)).
template <int LG, int LGNS = 0>
__device__ __forceinline__ void fft_c(Cx<float>* s, int count, int seq, const Cx<float>* __restrict__ T) {
    if constexpr (LGNS + 3 <= LG) {
        pass_c<LG, 8, LGNS>(s, count, seq, T);
        fft_c<LG, LGNS + 3>(s, count, seq, T);
    } else if constexpr (LG - LGNS == 2) {
        pass_c<LG, 4, LGNS>(s, count, seq, T);
    } else if constexpr (LG - LGNS == 1) {
        pass_c<LG, 2, LGNS>(s, count, seq, T);
    }
}

// ---- fast path: both sides powers of two ----------------------------------

// Two adjacent complex values as one vector store (16 B in FP32, 2 x 16 B in
// FP64); p is aligned to twice the element size.
__device__ __forceinline__ void store_pair(Cx<float>* p, Cx<float> a, Cx<float> b) {
    *reinterpret_cast<float4*>(p) = make_float4(a.re, a.im, b.re, b.im);
}
__device__ __forceinline__ void store_pair(Cx<double>* p, Cx<double> a, Cx<double> b) {
    reinterpret_cast<double2*>(p)[0] = make_double2(a.re, a.im);
    reinterpret_cast<double2*>(p)[1] = make_double2(b.re, b.im);
}

// Layout of the half spectrum H[f]: columns m = 0..Lx/2 in pairs (2p, 2p + 1),
// each pair stored y by y with its two values side by side, (m, y) at
// (p Ly + y) 2 + (m & 1); a field holds hx2(Hx) pairs. A row-pair CTA then
// writes whole 32-byte sectors ((2p, y), (2p + 1, y), (2p, y + 1), (2p + 1,
// y + 1) in FP32), and a column's values are every other one of its pair's.
__host__ __device__ constexpr int hx2(int Hx) { return (Hx + 1) / 2; }
__device__ __forceinline__ size_t h_index(int m, int y, int Ly) {
    return ((size_t)(m >> 1) * Ly + y) * 2 + (m & 1);
}

// The x-transform of the three fields of the row pair (y0, y0 + 1), staged in
// shared memory s as one complex sequence per field (row y0 in the real part,
// row y0 + 1 in the imaginary part, element x at spos(x)), and the store of
// the half spectrum: H[f][m][y], m = 0..Lx/2 (Hx columns of Ly values), the
// x-transform of field f (0: drho, 1: dj_x, 2: dj_y) of row y, column-major so
// that the y-transforms read contiguous columns.
template <class R>
__device__ __forceinline__ void rows_transform_store(Cx<R>* s, int seq, int lgLx, int Lx, int Ly,
                                                     int y0, const Cx<R>* __restrict__ tw,
                                                     Cx<R>* __restrict__ H, int Hx) {
    __syncthreads();
    fft_seqs<kEfast>(s, lgLx, 3, seq, tw);
    // z = a + i b with a, b real: A(m) = (Z(m) + conj Z(-m)) / 2,
    // B(m) = (Z(m) - conj Z(-m)) / (2i)
    const int np = hx2(Hx);
    for (int f = 0; f < 3; ++f) {
        const Cx<R>* z = s + f * seq;
        Cx<R>* out = H + (size_t)f * np * Ly * 2;
        for (int p = threadIdx.x; p < np; p += blockDim.x) {
            Cx<R> a[2], b[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = 2 * p + h;
                const Cx<R> u = z[spos<kEfast>(m & (Lx - 1))], w = z[spos<kEfast>((Lx - m) & (Lx - 1))];
                a[h] = {R(0.5) * (u.re + w.re), R(0.5) * (u.im - w.im)};
                b[h] = {R(0.5) * (u.im + w.im), R(0.5) * (w.re - u.re)};
            }
            Cx<R>* o = out + ((size_t)p * Ly + y0) * 2;   // (2p, y0), (2p + 1, y0), then row y0 + 1
            store_pair(o, a[0], a[1]);
            store_pair(o + 2, b[0], b[1]);
        }
    }
}

// One CTA per row pair (y0, y0 + 1): the fields formed from the pulled
// populations, then rows_transform_store.
template <class T, class R>
__global__ void __launch_bounds__(kThreads, 2) rows_pair_kernel(const T* __restrict__ buf, Geometry geo,
                                                             DevCodec codec, Ref9<R> c, int lgLx,
                                                             const Cx<R>* __restrict__ tw,
                                                             Cx<R>* __restrict__ H, int Hx) {
    extern __shared__ __align__(16) unsigned char raw[];
    Cx<R>* s = reinterpret_cast<Cx<R>*>(raw);
    const int Lx = geo.Lx, Ly = geo.Ly;
    const int seq = padded_len<kEfast>(Lx);
    const int y0 = 2 * blockIdx.x, y1 = y0 + 1;
    for (int x = threadIdx.x; x < Lx; x += blockDim.x) {
        R r0, a0, b0, r1, a1, b1;
        node_fields(buf, geo, codec, c, x, y0, r0, a0, b0);
        node_fields(buf, geo, codec, c, x, y1, r1, a1, b1);
        const int p = spos<kEfast>(x);
        s[p] = {r0, r1};
        s[seq + p] = {a0, a1};
        s[2 * seq + p] = {b0, b1};
    }
    rows_transform_store(s, seq, lgLx, Lx, Ly, y0, tw, H, Hx);
}

// One CTA per row pair (y0, y0 + 1) of the FP32 fields F[f][y][x] that the
// step kernel wrote on this sampling step (bit-identical to the fields
// node_fields forms from the same state), Lx = 2^LG: the x-transform of the
// three fields as in rows_transform_store, with the compile-time passes.
template <int LG>
__global__ void __launch_bounds__(kThreads, 2) rows_fields_kernel(const float* __restrict__ F, int Ly,
                                                               const Cx<float>* __restrict__ tw,
                                                               Cx<float>* __restrict__ H, int Hx) {
    constexpr int Lx = 1 << LG;
    extern __shared__ __align__(16) unsigned char raw[];
    Cx<float>* s = reinterpret_cast<Cx<float>*>(raw);
    const int y0 = 2 * blockIdx.x;
    const size_t N = (size_t)Lx * Ly;
    const float* r0 = F + (size_t)y0 * Lx;
    if constexpr (LG >= 3) {
        // the first radix-8 pass straight from the field rows: butterfly t of
        // field q takes x = t + r Lx/8 (r = 0..7; consecutive lanes, coalesced
        // loads), transforms in registers and writes its outputs 8 t + r to
        // their swizzled positions spos8(8 t) ^ r, so the values do not pass
        // through shared memory on their way in
        constexpr int nj = Lx / 8, spr = kThreads / nj;
        const int t = (int)threadIdx.x % nj, qt = (int)threadIdx.x / nj;
        const int pd = spos8(8 * t);
        for (int q0 = 0; q0 < 3; q0 += spr) {
            const int q = q0 + qt;
            if (q < 3) {
                const float* rf = r0 + q * N + t;
                Cx<float> v[8];
#pragma unroll
                for (int r = 0; r < 8; ++r) v[r] = {__ldcs(rf + r * nj), __ldcs(rf + Lx + r * nj)};
                dft_reg<8>(v);
                Cx<float>* z = s + q * Lx;
#pragma unroll
                for (int r = 0; r < 8; ++r) z[pd ^ r] = v[r];
            }
        }
        __syncthreads();
        fft_c<LG, 3>(s, 3, Lx, tw);
    } else {
        for (int x = threadIdx.x; x < Lx; x += kThreads)
#pragma unroll
            for (int f = 0; f < 3; ++f) s[f * Lx + spos8(x)] = {r0[f * N + x], r0[f * N + Lx + x]};
        __syncthreads();
        fft_c<LG>(s, 3, Lx, tw);
    }
    // z = a + i b with a, b real: A(m) = (Z(m) + conj Z(-m)) / 2,
    // B(m) = (Z(m) - conj Z(-m)) / (2i); H[f][m][y], column-major
    constexpr int np = hx2(Lx / 2 + 1);
    for (int f = 0; f < 3; ++f) {
        const Cx<float>* z = s + f * Lx;
        Cx<float>* out = H + (size_t)f * np * Ly * 2;
        for (int p = threadIdx.x; p < np; p += kThreads) {
            Cx<float> a[2], b[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = 2 * p + h;
                const Cx<float> u = z[spos8(m & (Lx - 1))], w = z[spos8((Lx - m) & (Lx - 1))];
                a[h] = {0.5f * (u.re + w.re), 0.5f * (u.im - w.im)};
                b[h] = {0.5f * (u.im + w.im), 0.5f * (w.re - u.re)};
            }
            Cx<float>* o = out + ((size_t)p * Ly + y0) * 2;   // one 32-byte sector
            store_pair(o, a[0], a[1]);
            store_pair(o + 2, b[0], b[1]);
        }
    }
}

// The sums a column kernel adds to: FP64 for FP64 transforms (the products
// formed in FP64, cols_acc_kernel), FP32 partials of at most kPartialSamples
// samples for FP32 transforms (the products formed in FP32, cols_part_kernel)
// that flush_part4_kernel adds to the FP64 sums; GB300's FP64 rate makes FP64
// products the cost of the column kernel otherwise.
constexpr int kPartialSamples = 16;

// One CTA per block of C = 2^lc columns of the half spectrum H[f][m][y]: the
// y-transform of each, then acc[q][m_x][m_y] += |drho|^2 (q = 0), |dj_x|^2
// (1), Re and Im of dj_x conj(dj_y) (2, 3); acc[q] is Hx x Ly, m_y fastest
// (instantiated for FP64 transforms and sums).
template <class R, class A>
__global__ void __launch_bounds__(kThreads, 2) cols_acc_kernel(const Cx<R>* __restrict__ H, int lgLy,
                                                            int Hx, int lc,
                                                            const Cx<R>* __restrict__ tw,
                                                            A* __restrict__ acc) {
    extern __shared__ __align__(16) unsigned char raw[];
    Cx<R>* s = reinterpret_cast<Cx<R>*>(raw);
    const int Ly = 1 << lgLy, C = 1 << lc;
    const int seq = padded_len<kEfast>(Ly);
    const int c0 = blockIdx.x * C;
    const int n = Ly << lc;
    const int lgn = lgLy + lc;
    const size_t Q = (size_t)Hx * Ly;
    const size_t QH = (size_t)hx2(Hx) * Ly * 2;   // values of H per field
    // kLoad independent loads in flight per thread before the stores
    constexpr int kLoad = 8;
    for (int j0 = threadIdx.x; j0 < 3 * n; j0 += kLoad * blockDim.x) {
        Cx<R> v[kLoad];
#pragma unroll
        for (int u = 0; u < kLoad; ++u) {
            const int j = j0 + u * blockDim.x;
            const int f = j >> lgn, cc = (j >> lgLy) & (C - 1), y = j & (Ly - 1);
            v[u] = (j < 3 * n && c0 + cc < Hx) ? H[(size_t)f * QH + h_index(c0 + cc, y, Ly)]
                                               : Cx<R>{R(0), R(0)};
        }
#pragma unroll
        for (int u = 0; u < kLoad; ++u) {
            const int j = j0 + u * blockDim.x;
            const int f = j >> lgn, cc = (j >> lgLy) & (C - 1), y = j & (Ly - 1);
            if (j < 3 * n) s[(f * C + cc) * seq + spos<kEfast>(y)] = v[u];
        }
    }
    __syncthreads();
    fft_seqs<kEfast>(s, lgLy, 3 * C, seq, tw);
    // kAcc sites per thread at a time: their 4 kAcc sums are read before any
    // is written back
    constexpr int kAcc = 2;
    for (int j0 = threadIdx.x; j0 < n; j0 += kAcc * blockDim.x) {
        A old[kAcc][4];
#pragma unroll
        for (int u = 0; u < kAcc; ++u) {
            const int j = j0 + u * blockDim.x;
            const int col = c0 + (j >> lgLy);
            const size_t k = (size_t)col * Ly + (j & (Ly - 1));
            const bool ok = j < n && col < Hx;
#pragma unroll
            for (int q = 0; q < 4; ++q) old[u][q] = ok ? acc[q * Q + k] : A(0);
        }
#pragma unroll
        for (int u = 0; u < kAcc; ++u) {
            const int j = j0 + u * blockDim.x;
            const int cc = j >> lgLy, m = j & (Ly - 1);
            const int col = c0 + cc;
            if (j >= n || col >= Hx) continue;
            const Cx<R> a = s[cc * seq + spos<kEfast>(m)];
            const Cx<R> b = s[(C + cc) * seq + spos<kEfast>(m)];
            const Cx<R> d = s[(2 * C + cc) * seq + spos<kEfast>(m)];
            const size_t k = (size_t)col * Ly + m;
            const A ar = a.re, ai = a.im, br = b.re, bi = b.im, dr = d.re, di = d.im;
            acc[k] = old[u][0] + (ar * ar + ai * ai);
            acc[Q + k] = old[u][1] + (br * br + bi * bi);
            acc[2 * Q + k] = old[u][2] + (br * dr + bi * di);
            acc[3 * Q + k] = old[u][3] + (bi * dr - br * di);
        }
    }
}

// Columns per CTA of the column kernels: the most (up to 4) whose three
// sequences of 2^LG FP32 values leave room for two CTAs per SM.
__host__ __device__ constexpr int cols_lc(int lg) {
    return (24 << lg) * 4 <= kColsSmemBudget ? 2 : (24 << lg) * 2 <= kColsSmemBudget ? 1 : 0;
}

// The FP32 column kernel of the fused-field path, Ly = 2^LG, C = 2^cols_lc(LG)
// columns per CTA: the y-transforms with the compile-time passes, then the
// four partial sums of each half-plane point side by side (part[k] =
// (|drho|^2, |dj_x|^2, Re, Im of dj_x conj dj_y), k = m_x Ly + m_y), one
// 16-byte read and one 16-byte write per point; spectra and partial sums are
// streamed past L1, where the twiddles are kept. With Ly >= 128 the swizzle
// of the CTA's value i (column i >> LG, element i mod Ly) is spos8(i).
template <int LG>
__global__ void __launch_bounds__(kThreads, 2) cols_part_kernel(const Cx<float>* __restrict__ H, int Hx,
                                                             const Cx<float>* __restrict__ tw,
                                                             float4* __restrict__ part) {
    constexpr int Ly = 1 << LG, LC = cols_lc(LG), C = 1 << LC;
    constexpr int n = Ly << LC;        // values per field in this CTA
    extern __shared__ __align__(16) unsigned char raw[];
    Cx<float>* s = reinterpret_cast<Cx<float>*>(raw);
    const int c0 = blockIdx.x * C;
    const size_t QH = (size_t)hx2(Hx) * Ly * 2;   // values of H per field
    const int nvalid = min(C, Hx - c0) * Ly;     // values of columns that exist
    auto pos = [](int i) { return Ly >= 128 ? spos8(i) : (i & ~(Ly - 1)) + spos8(i & (Ly - 1)); };
    constexpr int U = n > kThreads ? n / kThreads : 1;
    const int i0 = threadIdx.x;
    if constexpr (LG >= 3) {
        // the first radix-8 pass straight from H: butterfly t of sequence q
        // (field q / C, column c0 + q mod C) takes y = t + r Ly/8 (consecutive
        // lanes read consecutive y of the column), transforms in registers and
        // writes its outputs 8 t + r to spos8(8 t) ^ r of the sequence
        constexpr int nj = Ly / 8, spr = kThreads / nj;
        const int t = (int)threadIdx.x % nj, qt = (int)threadIdx.x / nj;
        const int pd = spos8(8 * t);
        for (int q0 = 0; q0 < 3 * C; q0 += spr) {
            const int q = q0 + qt;
            if (q < 3 * C) {
                const int f = q >> LC, c = c0 + (q & (C - 1));
                Cx<float> v[8];
                if (c < Hx) {
                    const Cx<float>* col = H + (size_t)f * QH;
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        const float2 w = __ldcs(reinterpret_cast<const float2*>(col + h_index(c, t + r * nj, Ly)));
                        v[r] = {w.x, w.y};
                    }
                    dft_reg<8>(v);
                } else {
#pragma unroll
                    for (int r = 0; r < 8; ++r) v[r] = {0.f, 0.f};
                }
                Cx<float>* z = s + q * Ly;
#pragma unroll
                for (int r = 0; r < 8; ++r) z[pd ^ r] = v[r];
            }
        }
        __syncthreads();
        fft_c<LG, 3>(s, 3 * C, Ly, tw);
    } else {
        // all of a field's loads in flight; the C columns of a field: column
        // pairs, both columns' y values as one 16-byte load
        if (i0 < n) {
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                const Cx<float>* Hf = H + (size_t)f * QH + (size_t)c0 * Ly;   // pair c0 / 2 (c0 even when C > 1)
                constexpr int U2 = U / 2 > 0 ? U / 2 : 1;
                float4 v[U2];
#pragma unroll
                for (int u = 0; u < U2; ++u) {
                    const int q = i0 + u * kThreads;   // < n / 2
                    v[u] = q < n / 2 && 2 * (q >> LG) < min(C, Hx - c0)
                               ? __ldcs(reinterpret_cast<const float4*>(Hf + 2 * q))
                               : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < U2; ++u) {
                    const int q = i0 + u * kThreads;
                    if (q < n / 2) {
                        const int cp = q >> LG, y = q & (Ly - 1);   // columns 2 cp, 2 cp + 1 of the CTA
                        s[f * n + pos(2 * cp * Ly + y)] = {v[u].x, v[u].y};
                        s[f * n + pos((2 * cp + 1) * Ly + y)] = {v[u].z, v[u].w};
                    }
                }
            }
        }
        __syncthreads();
        fft_c<LG>(s, 3 * C, Ly, tw);
    }
    float4* pc = part + (size_t)c0 * Ly;   // the CTA's columns, contiguous
    constexpr int kAcc = U < 4 ? U : 4;
    if (i0 < n) {
#pragma unroll
        for (int u0 = 0; u0 < U; u0 += kAcc) {
            float4 old[kAcc];
#pragma unroll
            for (int u = 0; u < kAcc; ++u) {
                const int i = i0 + (u0 + u) * kThreads;
                old[u] = i < nvalid ? ld_stream(pc + i) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < kAcc; ++u) {
                const int i = i0 + (u0 + u) * kThreads;
                if (i >= nvalid) continue;
                const int p = pos(i);
                const Cx<float> a = s[p], b = s[n + p], d = s[2 * n + p];
                float4 o = old[u];
                o.x += a.re * a.re + a.im * a.im;
                o.y += b.re * b.re + b.im * b.im;
                o.z += b.re * d.re + b.im * d.im;
                o.w += b.im * d.re - b.re * d.im;
                pc[i] = o;
            }
        }
    }
}

// acc[q Q + k] += part[k].q in FP64, part[k] = 0 (Q half-plane points).
__global__ void flush_part4_kernel(float4* __restrict__ part, double* __restrict__ acc, size_t Q) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < Q;
         k += (size_t)gridDim.x * blockDim.x) {
        const float4 v = part[k];
        acc[k] += (double)v.x;
        acc[Q + k] += (double)v.y;
        acc[2 * Q + k] += (double)v.z;
        acc[3 * Q + k] += (double)v.w;
        part[k] = make_float4(0.f, 0.f, 0.f, 0.f);
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

// In-place transform of line blockIdx.x of each field (blockIdx.y) with a
// power-of-two length 2^lgL: rows (elements `step` = 1 apart, lines Lx apart)
// or columns (elements Lx apart, lines 1 apart).
template <class R>
__global__ void __launch_bounds__(1024) fft_lines_kernel(Cx<R>* F, int lgL, size_t step, size_t line,
                                                         size_t field, const Cx<R>* __restrict__ tw) {
    extern __shared__ __align__(16) unsigned char raw[];
    Cx<R>* s = reinterpret_cast<Cx<R>*>(raw);
    Cx<R>* p = F + blockIdx.y * field + blockIdx.x * line;
    const int L = 1 << lgL;
    for (int i = threadIdx.x; i < L; i += blockDim.x) s[spos<Elines<R>::E>(i)] = p[i * step];
    __syncthreads();
    fft_seqs<Elines<R>::E>(s, lgL, 1, 0, tw);
    for (int i = threadIdx.x; i < L; i += blockDim.x) p[i * step] = s[spos<Elines<R>::E>(i)];
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

// Threads of a transform CTA: at least the threads one sequence takes.
template <class R>
int fft_threads(int L) {
    return std::max(kThreads, L / Elines<R>::E);
}

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
    float* part = nullptr;            // fast FP32 transforms: FP32 partials of acc
    float* fin = nullptr;             // fast, fused: 3 Lx Ly FP32 fields from the step kernel
    int pending = 0;                  // samples held in part
    void* twx = nullptr;              // twiddles along x and y
    void* twy = nullptr;
    int64_t nsamp = 0;
};

namespace {

template <class R>
cudaError_t upload_twiddles(int L, void** out) {
    // exp(-2 pi i m / L), m < L
    std::vector<Cx<R>> h(L);
    for (int m = 0; m < L; ++m) {
        const double a = -2.0 * M_PI * (double)m / (double)L;
        h[m] = {(R)std::cos(a), (R)std::sin(a)};
    }
    cudaError_t ce = cudaMalloc(out, sizeof(Cx<R>) * L);
    if (ce == cudaSuccess) ce = cudaMemcpy(*out, h.data(), sizeof(Cx<R>) * L, cudaMemcpyHostToDevice);
    return ce;
}

cudaError_t flush_partials(StructSampler* s, cudaStream_t st) {
    s->pending = 0;
    if (!s->part) return cudaSuccess;
    const size_t Q = s->acc_count / 4;
    const int grid = (int)std::min<size_t>(4096, (Q + 255) / 256);
    flush_part4_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<float4*>(s->part), s->acc, Q);
    return cudaGetLastError();
}

// The compile-time-length kernels by log2 of the length (1..12).
using RowsFieldsFn = void (*)(const float*, int, const Cx<float>*, Cx<float>*, int);
using ColsPartFn = void (*)(const Cx<float>*, int, const Cx<float>*, float4*);
template <int LG>
constexpr RowsFieldsFn rows_fields_at() { return rows_fields_kernel<LG>; }
template <int LG>
constexpr ColsPartFn cols_part_at() { return cols_part_kernel<LG>; }
template <int... LG>
RowsFieldsFn rows_fields_fn(int lg, std::integer_sequence<int, LG...>) {
    const RowsFieldsFn t[] = {rows_fields_at<LG + 1>()...};
    return lg >= 1 && lg <= (int)sizeof...(LG) ? t[lg - 1] : nullptr;
}
template <int... LG>
ColsPartFn cols_part_fn(int lg, std::integer_sequence<int, LG...>) {
    const ColsPartFn t[] = {cols_part_at<LG + 1>()...};
    return lg >= 1 && lg <= (int)sizeof...(LG) ? t[lg - 1] : nullptr;
}
constexpr int kMaxFastLg = 12;   // sides up to 4096
RowsFieldsFn rows_fields_for(int lg) { return rows_fields_fn(lg, std::make_integer_sequence<int, kMaxFastLg>{}); }
ColsPartFn cols_part_for(int lg) { return cols_part_fn(lg, std::make_integer_sequence<int, kMaxFastLg>{}); }

// The column launch of the power-of-two path and the partial-sum flush.
template <class R>
cudaError_t cols_accumulate(StructSampler* s, cudaStream_t st) {
    const Cx<R>* H = (const Cx<R>*)s->fields;
    const int C = 1 << s->lc;
    cudaError_t ce;
    if constexpr (sizeof(R) == 4) {
        const ColsPartFn k = cols_part_for(log2i(s->Ly));
        ce = cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)s->smem_cols);
        if (ce != cudaSuccess) return ce;
        k<<<(s->Hx + C - 1) / C, kThreads, s->smem_cols, st>>>(H, s->Hx, (const Cx<R>*)s->twy,
                                                               reinterpret_cast<float4*>(s->part));
        ce = cudaGetLastError();
        if (ce == cudaSuccess && ++s->pending == kPartialSamples) ce = flush_partials(s, st);
        return ce;
    } else {
        ce = cudaFuncSetAttribute(cols_acc_kernel<R, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)s->smem_cols);
        if (ce != cudaSuccess) return ce;
        cols_acc_kernel<R, double><<<(s->Hx + C - 1) / C, kThreads, s->smem_cols, st>>>(
            H, log2i(s->Ly), s->Hx, s->lc, (const Cx<R>*)s->twy, s->acc);
        return cudaGetLastError();
    }
}

template <class T, class R>
cudaError_t sample_fast(StructSampler* s, const T* buf, const Geometry& geo, const DevCodec& codec,
                        const Ref9<R>& c, cudaStream_t st) {
    cudaError_t ce = cudaFuncSetAttribute(rows_pair_kernel<T, R>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->smem_rows);
    if (ce != cudaSuccess) return ce;
    rows_pair_kernel<T, R><<<s->Ly / 2, kThreads, s->smem_rows, st>>>(
        buf, geo, codec, c, log2i(s->Lx), (const Cx<R>*)s->twx, (Cx<R>*)s->fields, s->Hx);
    ce = cudaGetLastError();
    return ce == cudaSuccess ? cols_accumulate<R>(s, st) : ce;
}

template <class R>
cudaError_t fft_lines(Cx<R>* F, int L, size_t step, size_t line, int nlines, size_t field,
                      const Cx<R>* tw, cudaStream_t st) {
    const size_t sm = sizeof(Cx<R>) * padded_len<Elines<R>::E>(L);
    cudaError_t ce = cudaFuncSetAttribute(fft_lines_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (ce == cudaSuccess) {
        fft_lines_kernel<R><<<dim3(nlines, 3), fft_threads<R>(L), sm, st>>>(F, log2i(L), step, line, field, tw);
        ce = cudaGetLastError();
    }
    return ce;
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
            ce = fft_lines<R>(F, Lx, 1, Lx, Ly, N, tx, st);
        } else {
            const size_t sm = sizeof(Cx<R>) * Lx;
            ce = cudaFuncSetAttribute(dft_rows_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (ce == cudaSuccess) dft_rows_kernel<R><<<dim3(Ly, 3), 256, sm, st>>>(F, Lx, Ly, tx);
            if (ce == cudaSuccess) ce = cudaGetLastError();
        }
    }
    if (ce == cudaSuccess && Ly > 1) {
        if (pow2(Ly)) {
            ce = fft_lines<R>(F, Ly, Lx, 1, Lx, N, ty, st);
        } else {
            const size_t sm = sizeof(Cx<R>) * Ly;
            ce = cudaFuncSetAttribute(dft_cols_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (ce == cudaSuccess) dft_cols_kernel<R><<<dim3(Lx, 3), 256, sm, st>>>(F, Lx, Ly, ty);
            if (ce == cudaSuccess) ce = cudaGetLastError();
        }
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

int structure_create(StructSampler** out, int Lx, int Ly, int rbytes, bool fused) {
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
    // fast path: one sequence's threads (L / E) fit one 512-thread CTA
    if (pow2(Lx) && pow2(Ly) && Lx >= 2 && Ly >= 2 && Lx / kEfast <= kThreads && Ly / kEfast <= kThreads) {
        s->smem_rows = 3 * cb * padded_len<kEfast>(Lx);
        // columns per CTA: the most that leave room for two CTAs per SM, else one
        const size_t col = 3 * cb * padded_len<kEfast>(Ly);
        s->lc = 0;
        if (rbytes == 4)   // the FP32 column kernel's fixed count (two CTAs per SM on sm_103)
            s->lc = cols_lc(log2i(Ly));
        else
            while (s->lc < 2 && col << (s->lc + 1) <= (size_t)optin / 2) ++s->lc;
        s->smem_cols = col << s->lc;
        s->fast = s->smem_rows <= (size_t)optin && s->smem_cols <= (size_t)optin;
    }
    // the general path holds one row (column) of complex values per CTA
    const auto fits = [&](int L) {
        if (!pow2(L)) return (size_t)L * cb <= kGeneralSmem;
        return rbytes == 4 ? L / Elines<float>::E <= 1024 && padded_len<Elines<float>::E>(L) * cb <= (size_t)optin
                           : L / Elines<double>::E <= 1024 && padded_len<Elines<double>::E>(L) * cb <= (size_t)optin;
    };
    if (!s->fast && !(fits(Lx) && fits(Ly))) {
        delete s;
        return FLB_ERR_ARG;
    }
    const size_t N = (size_t)Lx * Ly;
    s->Hx = Lx / 2 + 1;
    const size_t nfield = s->fast ? 3 * (size_t)Ly * 2 * hx2(s->Hx) : 3 * N;
    s->acc_count = s->fast ? 4 * (size_t)Ly * s->Hx : 4 * N;
    cudaError_t ce = cudaMalloc(&s->fields, nfield * cb);
    if (ce == cudaSuccess) ce = cudaMalloc(&s->acc, s->acc_count * sizeof(double));
    if (ce == cudaSuccess) ce = cudaMemset(s->acc, 0, s->acc_count * sizeof(double));
    if (ce == cudaSuccess && s->fast && rbytes == 4) {
        ce = cudaMalloc(&s->part, s->acc_count * sizeof(float));
        if (ce == cudaSuccess) ce = cudaMemset(s->part, 0, s->acc_count * sizeof(float));
        if (ce == cudaSuccess && fused) ce = cudaMalloc(&s->fin, 3 * N * sizeof(float));
    }
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
    cudaFree(s->part);
    cudaFree(s->fin);
    cudaFree(s->twx);
    cudaFree(s->twy);
    delete s;
}

cudaError_t structure_reset(StructSampler* s, cudaStream_t st) {
    s->nsamp = 0;
    s->pending = 0;
    cudaError_t ce = cudaMemsetAsync(s->acc, 0, s->acc_count * sizeof(double), st);
    if (ce == cudaSuccess && s->part) ce = cudaMemsetAsync(s->part, 0, s->acc_count * sizeof(float), st);
    return ce;
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

float* structure_fields(StructSampler* s) { return s ? s->fin : nullptr; }

cudaError_t structure_sample_fields(StructSampler* s, cudaStream_t st) {
    if (!s->fin) return cudaErrorInvalidValue;
    const RowsFieldsFn k = rows_fields_for(log2i(s->Lx));
    cudaError_t ce = cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)s->smem_rows);
    if (ce != cudaSuccess) return ce;
    k<<<s->Ly / 2, kThreads, s->smem_rows, st>>>(s->fin, s->Ly, (const Cx<float>*)s->twx,
                                                  (Cx<float>*)s->fields, s->Hx);
    ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cols_accumulate<float>(s, st);
    if (ce == cudaSuccess) s->nsamp += 1;
    return ce;
}

int structure_read(StructSampler* s, double* const out[4], double scale, cudaStream_t st) {
    const size_t N = (size_t)s->Lx * s->Ly;
    if (s->pending > 0 && flush_partials(s, st) != cudaSuccess) {
        cudaGetLastError();
        return FLB_ERR_CUDA;
    }
    if (!s->fast) {
        cudaError_t ce = cudaSuccess;
        for (int q = 0; q < 4 && ce == cudaSuccess; ++q)
            if (out[q])
                ce = cudaMemcpyAsync(out[q], s->acc + q * N, N * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) return FLB_ERR_CUDA;
        for (int q = 0; q < 4; ++q)
            if (out[q])
                for (size_t n = 0; n < N; ++n) out[q][n] *= scale;
        return FLB_OK;
    }
    // half plane [q][m_x][m_y], m_x = 0..Lx/2, one q at a time
    const int Lx = s->Lx, Ly = s->Ly, Hx = s->Hx;
    const size_t Q = (size_t)Hx * Ly;
    std::vector<double> half;
    try {
        half.resize(Q);
    } catch (const std::bad_alloc&) {
        return FLB_ERR_OOM;
    }
    for (int q = 0; q < 4; ++q) {
        if (!out[q]) continue;
        cudaError_t ce = cudaMemcpyAsync(half.data(), s->acc + q * Q, Q * sizeof(double),
                                         cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) return FLB_ERR_CUDA;
        // m_x > Lx/2: the value at -k; Im R changes sign there
        const double sm = q == 3 ? -scale : scale;
        for (int my = 0; my < Ly; ++my) {
            double* row = out[q] + (size_t)my * Lx;
            for (int mx = 0; mx < Hx; ++mx) row[mx] = half[(size_t)mx * Ly + my] * scale;
            const int ny = (Ly - my) & (Ly - 1);
            for (int mx = Hx; mx < Lx; ++mx) row[mx] = half[(size_t)(Lx - mx) * Ly + ny] * sm;
        }
    }
    return FLB_OK;
}

int64_t structure_samples(const StructSampler* s) { return s ? s->nsamp : 0; }

}  // namespace flb
