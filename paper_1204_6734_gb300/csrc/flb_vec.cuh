// flb_vec.cuh -- arithmetic types of the collision.
//
// The collision is written once, over a "lane type" V:
//   double  -- FP64 (parity mode), IEEE division and square roots;
//   float   -- FP32, SFU reciprocal / square roots;
//   f2      -- two FP32 nodes per thread in Blackwell's packed FP32x2
//              instructions (add/sub/mul/fma .f32x2, sm_100+): one issue slot
//              for the same operation on two nodes. The kernel is bound by
//              instruction issue, so this halves the cost of the arithmetic.
// Every type provides +, -, *, mad(a,b,c) = a*b + c, construction from a
// scalar constant, and the per-lane functions rcp, rsq (1/sqrt), sqr.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace flb {

__device__ __forceinline__ double mad(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float mad(float a, float b, float c) { return fmaf(a, b, c); }

__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ double rsq(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ double sqr(double x) { return sqrt(x); }

__device__ __forceinline__ float rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsq(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sqr(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// SFU base-2 logarithm, sine and cosine with denormals flushed: the noise
// draws never pass a denormal (u1 >= 2^-21, |angle| = 0 or >= 2 pi 2^-21), so
// these give the values of the non-flushing forms without their fix-ups.
__device__ __forceinline__ float lg2_ftz(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void sincos_ftz(float x, float* s, float* c) {
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(*s) : "f"(x));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(*c) : "f"(x));
}

// Two FP32 lanes (node A in .x, node B in .y).
struct f2 {
    float2 v;
    __device__ __forceinline__ f2() {}
    __device__ __forceinline__ explicit f2(float2 a) : v(a) {}
    __device__ __forceinline__ f2(float s) : v(make_float2(s, s)) {}
    __device__ __forceinline__ f2(float a, float b) : v(make_float2(a, b)) {}
};

__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return f2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 mad(f2 a, f2 b, f2 c) { return f2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) {
    uint64_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r)
        : "l"(*reinterpret_cast<const uint64_t*>(&a.v)), "l"(*reinterpret_cast<const uint64_t*>(&b.v)));
    return f2(*reinterpret_cast<const float2*>(&r));
}
__device__ __forceinline__ f2& operator+=(f2& a, f2 b) { return a = a + b; }

__device__ __forceinline__ f2 rcp(f2 a) { return f2(rcp(a.v.x), rcp(a.v.y)); }
__device__ __forceinline__ f2 rsq(f2 a) { return f2(rsq(a.v.x), rsq(a.v.y)); }
__device__ __forceinline__ f2 sqr(f2 a) { return f2(sqr(a.v.x), sqr(a.v.y)); }

// Lane access (lanes = 1 for the scalar types).
template <class V> struct Lanes { static constexpr int n = 1; };
template <> struct Lanes<f2> { static constexpr int n = 2; };

__device__ __forceinline__ double lane(double a, int) { return a; }
__device__ __forceinline__ float lane(float a, int) { return a; }
__device__ __forceinline__ float lane(f2 a, int k) { return k ? a.v.y : a.v.x; }

// Scalar element type of a lane type.
template <class V> struct Elem { using type = V; };
template <> struct Elem<f2> { using type = float; };

}  // namespace flb
