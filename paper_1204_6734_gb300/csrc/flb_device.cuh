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

__device__ __forceinline__ Draw philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                              uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t y0 = hi1 ^ c1 ^ k0;
        const uint32_t y2 = hi0 ^ c3 ^ k1;
        c0 = y0;
        c1 = lo1;
        c2 = y2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return Draw{c0, c1, c2, c3};
}

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

__device__ __forceinline__ Draw node_draw(uint64_t seed, uint32_t replica, uint32_t node,
                                          uint32_t step) {
    return philox4x32_10(node, step, replica, 0u, (uint32_t)seed, (uint32_t)(seed >> 32));
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
        const float r2 = -1.3862943611198906f * __log2f(u1);   // -2 ln u1
        float r;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(r2));
        const float t = (float)((int)k[2 * p + 1] - (1 << 20)) * (float)(kTwoPi * 0x1p-21);
        float s, c;
        __sincosf(t, &s, &c);
        n[2 * p] = -r * c;
        n[2 * p + 1] = -r * s;
    }
}

// ---------------------------------------------------------------------------
// Precision-dependent helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rsq(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double sqr_root(double x) { return sqrt(x); }
__device__ __forceinline__ float sqr_root(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Per-launch collision constants (a = 3..8 stored at [a-3]).
template <class T>
struct CollideConst {
    T omega[6];   // omega_a
    T amp[6];     // sqrt(kT omega_a (2 - omega_a)); times sqrt(rho) gives xi^a
    uint64_t seed;
    uint32_t replica;
};

enum : int { kStatusOk = 0, kStatusInvalidVelocity = 1, kStatusNonfinite = 2 };

// ---------------------------------------------------------------------------
// Hermite transforms (Eq. d2q93a rows, Eq. d2q93b = w (.) P^T)
// ---------------------------------------------------------------------------

// Non-conserved Hermite moments M^3..M^8 of g.
template <class T>
__device__ __forceinline__ void hermite_moments_N(const T g[9], T M[6]) {
    const T s13 = g[1] + g[3], s24 = g[2] + g[4];
    const T d13 = g[3] - g[1], d42 = g[4] - g[2];
    const T c = g[5] + g[6] + g[7] + g[8];
    const T p58 = g[5] + g[8], p67 = g[6] + g[7];
    const T p56 = g[5] + g[6], p78 = g[7] + g[8];
    M[0] = T(1.5) * (s13 - s24);                                  // Pi_xx-yy
    M[1] = T(3) * ((g[5] + g[7]) - (g[6] + g[8]));                // Pi_xy
    M[2] = -g[0] + T(0.5) * (s13 + s24) + T(2) * c;               // Pi_xx+yy
    M[3] = T(kSqrt3h) * d13 + T(kSqrt6) * (p58 - p67);            // q_x
    M[4] = T(kSqrt3h) * d42 + T(kSqrt6) * (p56 - p78);            // q_y
    M[5] = T(0.5) * g[0] - (s13 + s24) + T(2) * c;                // epsilon
}

// h = P^T D: h_i = sum_a p^a_i D_a.
template <class T>
__device__ __forceinline__ void hermite_back(const T D[9], T h[9]) {
    const T base0 = D[0] - D[5] + T(0.5) * D[8];
    const T axis = D[0] + T(0.5) * D[5] - D[8];          // common to i = 1..4
    const T diag = D[0] + T(2) * D[5] + T(2) * D[8];     // common to i = 5..8
    const T jx = T(kSqrt3) * D[1], jy = T(kSqrt3) * D[2];
    const T px = T(1.5) * D[3], pxy = T(3) * D[4];
    const T qxa = T(kSqrt3h) * D[6], qya = T(kSqrt3h) * D[7];
    const T qxd = T(kSqrt6) * D[6], qyd = T(kSqrt6) * D[7];
    h[0] = base0;
    h[1] = axis + jx + px - qxa;
    h[3] = axis - jx + px + qxa;
    h[2] = axis + jy - px - qya;
    h[4] = axis - jy - px + qya;
    const T a = diag + pxy, b = diag - pxy;
    const T xpy = jx + jy + qxd + qyd;   // +x+y corner
    const T xmy = jx - jy + qxd - qyd;   // +x-y corner
    h[5] = a + xpy;
    h[7] = a - xpy;
    h[8] = b + xmy;
    h[6] = b - xmy;
}

// ---------------------------------------------------------------------------
// Collision of one node (Eq. LBEMRT)
// ---------------------------------------------------------------------------

// Hermite norm: relaxation of M^a - M^{a,0} (Eq. d2q94) at rate omega_a plus
// noise xi^a N^a on a = 3..8, back transform with n = w (.) P^T.
template <class T>
__device__ __forceinline__ int collide_standard(const T g[9], const T N[6],
                                                const CollideConst<T>& cc, T f[9]) {
    const T rho = ((g[0] + (g[1] + g[3])) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8]));
    if (!(rho > T(0)) || !isfinite(rho)) {
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = g[i];
        return kStatusNonfinite;
    }
    const T jx = (g[1] - g[3]) + ((g[5] + g[8]) - (g[6] + g[7]));
    const T jy = (g[2] - g[4]) + ((g[5] + g[6]) - (g[7] + g[8]));
    const T ir = rcp(rho);
    const T ux = jx * ir, uy = jy * ir;
    const T uxx = ux * ux, uyy = uy * uy;
    T M[6];
    hermite_moments_N(g, M);
    M[0] -= rho * T(1.5) * (uxx - uyy);
    M[1] -= rho * T(3) * (ux * uy);
    M[2] -= rho * T(1.5) * (uxx + uyy);
    const T sr = sqr_root(rho);
    T D[9];
    D[0] = D[1] = D[2] = T(0);
#pragma unroll
    for (int a = 0; a < 6; ++a) D[3 + a] = -cc.omega[a] * M[a] + cc.amp[a] * sr * N[a];
    T h[9];
    hermite_back(D, h);
    const T w0 = T(4.0 / 9.0), w1 = T(1.0 / 9.0), w5 = T(1.0 / 36.0);
    f[0] = g[0] + w0 * h[0];
#pragma unroll
    for (int i = 1; i <= 4; ++i) f[i] = g[i] + w1 * h[i];
#pragma unroll
    for (int i = 5; i <= 8; ++i) f[i] = g[i] + w5 * h[i];
    return kStatusOk;
}

// f-norm (Section 4): basis orthonormal under W = f^0(1,u) of this node.
template <class T>
__device__ __forceinline__ int collide_local(const T g[9], const T N[6],
                                             const CollideConst<T>& cc, T f[9]) {
    const T rho = ((g[0] + (g[1] + g[3])) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8]));
    if (!(rho > T(0)) || !isfinite(rho)) {
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = g[i];
        return kStatusNonfinite;
    }
    const T jx = (g[1] - g[3]) + ((g[5] + g[8]) - (g[6] + g[7]));
    const T jy = (g[2] - g[4]) + ((g[5] + g[6]) - (g[7] + g[8]));
    const T ir = rcp(rho);
    const T ux = jx * ir, uy = jy * ir;
    const T uxx = ux * ux, uyy = uy * uy, uxy = ux * uy;
    const T usq = uxx + uyy;

    // W_i = f_i^0(1, u) (Eq. d2q9f0)
    T W[9];
    {
        const T base = T(1) - T(1.5) * usq;
        const T ax = base + T(4.5) * uxx, ay = base + T(4.5) * uyy;
        const T dp = base + T(4.5) * (usq + T(2) * uxy);   // (u.v)^2 for v = +-(1,1)
        const T dm = base + T(4.5) * (usq - T(2) * uxy);   // v = +-(1,-1)
        const T sx = T(3) * ux, sy = T(3) * uy;
        W[0] = T(4.0 / 9.0) * base;
        W[1] = T(1.0 / 9.0) * (ax + sx);
        W[3] = T(1.0 / 9.0) * (ax - sx);
        W[2] = T(1.0 / 9.0) * (ay + sy);
        W[4] = T(1.0 / 9.0) * (ay - sy);
        W[5] = T(1.0 / 36.0) * (dp + (sx + sy));
        W[7] = T(1.0 / 36.0) * (dp - (sx + sy));
        W[8] = T(1.0 / 36.0) * (dm + (sx - sy));
        W[6] = T(1.0 / 36.0) * (dm - (sx - sy));
    }
    bool valid = true;
#pragma unroll
    for (int i = 0; i < 9; ++i) valid = valid && (W[i] > T(0));

    // conserved block of L: rows l_a = (e_a, k1_a, k2_a), a = 3..8
    const T e3 = T(1.5) * (uxx - uyy), e4 = T(3) * uxy, e5 = T(1.5) * usq;
    const T s3x = T(kSqrt3) * ux, s3y = T(kSqrt3) * uy;
    T k1[6], k2[6];
    k1[0] = s3x * (T(1) - e3);
    k1[1] = s3y * (T(1) - T(3) * uxx);
    k1[2] = s3x * (T(1) - e5);
    k1[3] = T(kSqrt2x3h) * uyy;
    k1[4] = T(kSqrt2x3) * uxy;
    k1[5] = T(0);
    k2[0] = -s3y * (T(1) + e3);
    k2[1] = s3x * (T(1) - T(3) * uyy);
    k2[2] = s3y * (T(1) - e5);
    k2[3] = T(kSqrt2x3) * uxy;
    k2[4] = T(kSqrt2x3h) * uxx;
    k2[5] = T(0);
    const T e[6] = {e3, e4, e5, T(0), T(0), T(0)};

    // Gram matrix G_NN(u) = sum_i p^a_i p^b_i W_i, a, b = 3..8 (upper triangle)
    T S[6][6];
    {
        const T r6x = T(kSqrt6h) * ux, r6y = T(kSqrt6h) * uy;     // sqrt6/2 u
        S[0][0] = T(1) + T(0.75) * usq;
        S[0][1] = T(0);
        S[0][2] = T(0.75) * (uxx - uyy);
        S[0][3] = -r6x;
        S[0][4] = r6y;
        S[0][5] = -T(1.5) * (uxx - uyy);
        S[1][1] = T(1) + T(3) * usq;
        S[1][2] = T(6) * uxy;
        S[1][3] = T(kSqrt6) * uy;
        S[1][4] = T(kSqrt6) * ux;
        S[1][5] = T(6) * uxy;
        S[2][2] = T(1) + T(0.75) * usq;
        S[2][3] = r6x;
        S[2][4] = r6y;
        S[2][5] = T(1.5) * usq;
        S[3][3] = T(1) + T(3) * uxx + T(1.5) * uyy;
        S[3][4] = T(6) * uxy;
        S[3][5] = T(kSqrt6) * ux;
        S[4][4] = T(1) + T(1.5) * uxx + T(3) * uyy;
        S[4][5] = T(kSqrt6) * uy;
        S[5][5] = T(1) + T(1.5) * usq;
    }
    // Schur complement S = G_NN - e e^T - k1 k1^T - k2 k2^T
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
        for (int b = a; b < 6; ++b) S[a][b] -= e[a] * e[b] + k1[a] * k1[b] + k2[a] * k2[b];

    // Cholesky S = L' L'^T (lower factor stored in the lower triangle of L)
    T L[6][6], inv[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        T d = S[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
        valid = valid && (d > T(0));
        inv[j] = rsq(d);
#pragma unroll
        for (int i = j + 1; i < 6; ++i) {
            T s = S[j][i];
#pragma unroll
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            L[i][j] = s * inv[j];
        }
    }
    if (!valid) {
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = g[i];
        return kStatusInvalidVelocity;
    }

    // non-conserved f-norm moments M~_N = L'^{-1} (M_N - rho e_N)
    T M[6];
    hermite_moments_N(g, M);
    M[0] -= rho * e3;
    M[1] -= rho * e4;
    M[2] -= rho * e5;
    T y[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        T s = M[j];
#pragma unroll
        for (int k = 0; k < j; ++k) s -= L[j][k] * y[k];
        y[j] = s * inv[j];
    }
    // change of each moment: relaxation towards M~^{a,0} = 0 (Eq. fnormmeq) + noise
    const T sr = sqr_root(rho);
    T z[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) z[a] = -cc.omega[a] * y[a] + cc.amp[a] * sr * N[a];
    // D_N = L'^{-T} z
#pragma unroll
    for (int j = 5; j >= 0; --j) {
        T s = z[j];
#pragma unroll
        for (int k = j + 1; k < 6; ++k) s -= L[k][j] * z[k];
        z[j] = s * inv[j];
    }
    T E = T(0), K1 = T(0), K2 = T(0);
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        E += e[a] * z[a];
        K1 += k1[a] * z[a];
        K2 += k2[a] * z[a];
    }
    T D[9];
    D[0] = -E + (s3x * K1 + s3y * K2);
    D[1] = -K1;
    D[2] = -K2;
#pragma unroll
    for (int a = 0; a < 6; ++a) D[3 + a] = z[a];
    T h[9];
    hermite_back(D, h);
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = g[i] + W[i] * h[i];
    return kStatusOk;
}

template <class T, int BASIS>
__device__ __forceinline__ int collide(const T g[9], uint32_t node, uint32_t step,
                                       const CollideConst<T>& cc, T f[9]) {
    uint32_t k[6];
    draw_fields(node_draw(cc.seed, cc.replica, node, step), k);
    T N[6];
    box_muller(k, N);
    if (BASIS == 0) return collide_standard<T>(g, N, cc, f);
    return collide_local<T>(g, N, cc, f);
}

}  // namespace flb
