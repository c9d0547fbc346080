// flb_device.cuh -- per-node device math of the fluctuating D2Q9 step.
//
// Kaehler & Wagner, arXiv:1204.6734. Everything here runs on one node in
// registers: the noise draw (Philox4x32-10 + Box-Muller), the Hermite transforms
// of the appendix (Eqs. d2q93a, d2q93b, d2q94), and the collision of Eq. LBEMRT
// in either the Hermite norm (Eq. fluctf5) or the f-norm of Section 4, whose
// basis is rebuilt at every node from the node's own velocity.
//
// f-norm basis. Gram-Schmidt of the Hermite rows p^0..p^8 in order under
// <a,b> = sum_i a_i W_i b_i, W_i = f_i^0(1,u) (Eqs. fnorm, gramschmidt, gsortho),
// is the same as m~ = L^{-1} P with L the Cholesky factor (positive diagonal)
// of the Gram matrix G(u) = P diag(W) P^T. Here:
//  * G(u) is evaluated in closed form. W = w (.) (P^T e(u)) with e(u) the
//    Hermite equilibrium moments at rho = 1 (Eq. d2q94), so every entry of G is
//    a short polynomial in u (the lattice sums of D2Q9 cancel most terms).
//  * The first three columns of L are analytic: L_CC = [[1,0,0],[sqrt3 ux,1,0],
//    [sqrt3 uy,0,1]] (m~^0 = 1, m~^1 = sqrt3 (v_x - u_x), m~^2 = sqrt3 (v_y - u_y)),
//    and the rows of L below them are l_a = (e_a, k1_a, k2_a) with
//    k1_a = G_a1 - sqrt3 ux e_a, k2_a = G_a2 - sqrt3 uy e_a.
//  * What remains is the 6x6 Cholesky L' of the Schur complement
//    S = G_NN - l l^T over the non-conserved moments N = {3..8}.
//  * With u = j/rho the conserved f-norm moments are rho, 0, 0, so the
//    non-conserved moments are M~_N = L'^{-1} (M_N - rho e_N): the Hermite
//    non-equilibrium moments, whitened by L'.
//  * The back transform n^a_i = m~^a_i W_i (below Eq. fluctf2) of a change D~_N
//    of the non-conserved moments is f* - g = W (.) (P^T D) with
//    D_N = L'^{-T} D~_N and D_C = (-E + sqrt3 (ux K1 + uy K2), -K1, -K2),
//    E = e.D_N, K1 = k1.D_N, K2 = k2.D_N.
// The Hermite-norm collision is the special case L = I, W = w.
#pragma once

#include <cstdint>

#include "flb_vec.cuh"

namespace flb {

// ---------------------------------------------------------------------------
// Constants
// ---------------------------------------------------------------------------

constexpr double kSqrt3 = 1.7320508075688772935274463415059;
constexpr double kSqrt3h = 1.2247448713915890490986420373529;   // sqrt(3/2)
constexpr double kSqrt6 = 2.4494897427831780981972840747059;
constexpr double kSqrt6h = 1.2247448713915890490986420373529;   // sqrt(6)/2
constexpr double kSqrt2x3h = 2.1213203435596425732025330863145;  // 3 sqrt(2)/2
constexpr double kSqrt2x3 = 4.2426406871192851464050661726291;   // 3 sqrt(2)
constexpr double kTwoPi = 6.283185307179586476925286766559;

// velocities (order of the j rows of Eq. d2q93a)
__host__ __device__ constexpr int cvx(int i) {
    return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
}
__host__ __device__ constexpr int cvy(int i) {
    return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
}

// ---------------------------------------------------------------------------
// Noise: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and Box-Muller
// ---------------------------------------------------------------------------

struct Draw {
    uint32_t x0, x1, x2, x3;
};

// The six 21-bit fields k_q = (X >> 21q) mod 2^21 of X = x0 + 2^32 x1 + 2^64 x2 + 2^96 x3.
__device__ __forceinline__ void draw_fields(const Draw& d, uint32_t k[6]) {
    const uint32_t m = 0x1FFFFFu;
    k[0] = d.x0 & m;
    k[1] = (d.x0 >> 21) | ((d.x1 & 0x3FFu) << 11);
    k[2] = (d.x1 >> 10) & m;
    k[3] = (d.x1 >> 31) | ((d.x2 & 0xFFFFFu) << 1);
    k[4] = (d.x2 >> 20) | ((d.x3 & 0x1FFu) << 12);
    k[5] = (d.x3 >> 9) & m;
}

// Box-Muller: u1 = (k_{2p}+1) 2^-21 in (0,1], u2 = k_{2p+1} 2^-21 in [0,1),
// N_{2p} = sqrt(-2 ln u1) cos(2 pi u2), N_{2p+1} = sqrt(-2 ln u1) sin(2 pi u2).
__device__ __forceinline__ void box_muller(const uint32_t k[6], double n[6]) {
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const double u1 = ((double)k[2 * p] + 1.0) * 0x1p-21;
        const double u2 = (double)k[2 * p + 1] * 0x1p-21;
        const double r = sqrt(-2.0 * log(u1));
        double s, c;
        sincos(kTwoPi * u2, &s, &c);
        n[2 * p] = r * c;
        n[2 * p + 1] = r * s;
    }
}

// FP32 form with the SFU: ln u1 = ln2 * log2(u1) (MUFU.LG2, absolute error
// 2^-22.6 on [0.5, 2], 2 ulp elsewhere); the angle is moved to [-pi, pi) where
// the SFU sine and cosine are accurate to 2^-21.4, using
// cos(t + pi) = -cos t, sin(t + pi) = -sin t.
__device__ __forceinline__ void box_muller(const uint32_t k[6], float n[6]) {
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const float u1 = (float)(k[2 * p] + 1u) * 0x1p-21f;
        const float r2 = -1.3862943611198906f * lg2_ftz(u1);   // -2 ln u1
        float r;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(r2));
        const float t = (float)((int)k[2 * p + 1] - (1 << 20)) * (float)(kTwoPi * 0x1p-21);
        float s, c;
        sincos_ftz(t, &s, &c);
        n[2 * p] = -r * c;
        n[2 * p + 1] = -r * s;
    }
}

// ---------------------------------------------------------------------------
// Per-launch constants
// ---------------------------------------------------------------------------

// Noise key of one lattice: Philox round keys precomputed from the seed.
struct NoiseKey {
    uint32_t rk[20];   // (k0 + r W0, k1 + r W1) mod 2^32, r = 0..9; (k0, k1) = seed
    uint32_t replica;  // third counter word
};

template <class T>
struct CollideConst {
    T nomega[6];   // -omega_a, a = 3..8
    T amp[6];      // sqrt(kT omega_a (2 - omega_a)); times sqrt(rho) gives xi^a
    NoiseKey key;
};

// The FP32 relaxation and noise constants as packed pairs {c, c}: a kernel that
// reads its constants from shared memory then loads each FP32x2 operand with one
// 64-bit load instead of a load and two moves. The Philox key stays in
// CollideConst.
struct CollidePairs {
    float2 nomega[6];   // -omega_a
    float2 namp[6];     // -sqrt(kT omega_a (2 - omega_a))
};

__host__ __device__ inline NoiseKey make_noise_key(uint64_t seed, uint32_t replica) {
    NoiseKey k;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        k.rk[2 * r] = k0;
        k.rk[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    k.replica = replica;
    return k;
}

enum : int { kStatusOk = 0, kStatusInvalidVelocity = 1, kStatusNonfinite = 2, kStatusTimeout = 3 };

}  // namespace flb
