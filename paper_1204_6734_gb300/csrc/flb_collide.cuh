// flb_collide.cuh -- the collision of Eq. LBEMRT for one node (V = double,
// float) or two nodes (V = f2), in the Hermite norm (BASIS 0) or the f-norm
// (BASIS 1). The algebra is described at the top of flb_device.cuh; here it is
// arranged so that every subtraction folds into a fused multiply-add:
//  * the Schur complement S of the conserved block is evaluated negated
//    (Sn = -S), each entry a closed-form polynomial in the velocity;
//  * the Cholesky factor is stored negated (Ln = -L'): the products Ln Ln = L L
//    keep their sign, so the factorisation and both triangular solves are
//    chains of fma(Ln, ., .) followed by one scaling with 1/L'_jj.
// Validity (Fig. 11): the Gram matrix P diag(W) P^T is positive definite iff
// every W_i = f_i^0(1,u) > 0; its leading 3x3 block is always positive definite,
// so this holds iff every pivot of S is positive, i.e. iff all six 1/sqrt(pivot)
// are finite. The kernel checks their sum.
#pragma once

#include <type_traits>

#include "flb_device.cuh"
#include "flb_vec.cuh"

namespace flb {

// Philox4x32-10 (Salmon et al., SC'11) with the round keys precomputed.
__device__ __forceinline__ Draw philox_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                          const NoiseKey& key) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t y0 = (uint32_t)(p1 >> 32) ^ c1 ^ key.rk[2 * r];
        const uint32_t y2 = (uint32_t)(p0 >> 32) ^ c3 ^ key.rk[2 * r + 1];
        c0 = y0;
        c1 = (uint32_t)p1;
        c2 = y2;
        c3 = (uint32_t)p0;
    }
    return Draw{c0, c1, c2, c3};
}

// Counter (node, step, replica, 0), key = seed.
__device__ __forceinline__ void node_fields(const NoiseKey& key, uint32_t node, uint32_t step,
                                            uint32_t k[6]) {
    draw_fields(philox_rk(node, step, key.replica, 0u, key), k);
}

template <class T>
__device__ __forceinline__ void node_normals(const NoiseKey& key, uint32_t node, uint32_t step,
                                             T n[6]) {
    uint32_t k[6];
    node_fields(key, node, step, k);
    box_muller(k, n);
}

__device__ __forceinline__ void node_normals(const NoiseKey& key, uint32_t nodeA, uint32_t nodeB,
                                             uint32_t step, f2 n[6]) {
    float a[6], b[6];
    node_normals(key, nodeA, step, a);
    node_normals(key, nodeB, step, b);
#pragma unroll
    for (int q = 0; q < 6; ++q) n[q] = f2(a[q], b[q]);
}

// The six noise increments xi^a N^a = sqrt(rho) amp_a N^a (Eqs. FDT, noiseamp)
// of the FP32 collisions, with sqrt(rho) and amp_a folded into the Box-Muller
// radius: r = sqrt(rho (-2 ln2) log2(u1)), u1 = (k + 1) 2^-21 formed exactly,
// so that log2 is taken where the SFU is accurate in absolute terms (near
// u1 = 1, the draws with the smallest radius; u1 = 1 gives r = 0 exactly). One
// node (scalar lanes) or a node pair (packed lanes) take the same operations
// per lane, so both give bit-identical increments. FP64 uses unit normals
// (operator()).
// The offsets ride in fused multiply-adds on the exact conversions of the
// 21-bit fields k: fma(k, 2^-21, 2^-21) is (k + 1) 2^-21 exactly, and
// fma(k, c, -2^20 c) is (k - 2^20) c rounded once, as the product of the
// exact difference would be (2^20 c is exact).
constexpr float kLn2x2 = 1.3862943611198906f;
constexpr float kAngle = (float)(kTwoPi * 0x1p-21);   // 2 pi 2^-21, the angle of one step of k

// -omega_a and -amp_a as operands of type V, from the constants in either form
// (CollideConst: scalars broadcast to the lanes; CollidePairs: packed pairs).
template <class V, class T>
__device__ __forceinline__ V nomega_of(const CollideConst<T>& cc, int a) { return V(cc.nomega[a]); }
template <class V>
__device__ __forceinline__ V nomega_of(const CollidePairs& cc, int a) { return V(cc.nomega[a]); }
__device__ __forceinline__ f2 namp_of(const CollideConst<float>& cc, int a) { return f2(-cc.amp[a]); }
__device__ __forceinline__ f2 namp_of(const CollidePairs& cc, int a) { return f2(cc.namp[a]); }

struct NodeNoise {
    const NoiseKey& key;
    uint32_t node, step;
    template <class T>
    __device__ __forceinline__ void operator()(T n[6]) const {
        node_normals(key, node, step, n);
    }
    __device__ __forceinline__ void scaled(float rho, const CollideConst<float>& cc, float n[6]) const {
        uint32_t k[6];
        node_fields(key, node, step, k);
        const float nr = rho * -kLn2x2;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const float u1 = mad((float)k[2 * p], 0x1p-21f, 0x1p-21f);
            const float r = sqr(lg2_ftz(u1) * nr);
            const float t = mad((float)k[2 * p + 1], kAngle, -0x1p20f * kAngle);
            float s, c;
            sincos_ftz(t, &s, &c);
            // cos(t + pi) = -cos t, sin(t + pi) = -sin t
            n[2 * p] = (r * -cc.amp[2 * p]) * c;
            n[2 * p + 1] = (r * -cc.amp[2 * p + 1]) * s;
        }
    }
};

struct PairNoise {
    const NoiseKey& key;
    uint32_t nodeA, nodeB, step;
    template <class CC>
    __device__ __forceinline__ void scaled(f2 rho, const CC& cc, f2 n[6]) const {
        uint32_t ka[6], kb[6];
        node_fields(key, nodeA, step, ka);
        node_fields(key, nodeB, step, kb);
        const f2 nr = rho * f2(-kLn2x2);
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const f2 u1 = mad(f2((float)ka[2 * p], (float)kb[2 * p]), f2(0x1p-21f), f2(0x1p-21f));
            const f2 r = sqr(f2(lg2_ftz(u1.v.x), lg2_ftz(u1.v.y)) * nr);
            const f2 t = mad(f2((float)ka[2 * p + 1], (float)kb[2 * p + 1]), f2(kAngle),
                             f2(-0x1p20f * kAngle));
            float sa, ca, sb, cb;
            sincos_ftz(t.v.x, &sa, &ca);
            sincos_ftz(t.v.y, &sb, &cb);
            n[2 * p] = (r * namp_of(cc, 2 * p)) * f2(ca, cb);
            n[2 * p + 1] = (r * namp_of(cc, 2 * p + 1)) * f2(sa, sb);
        }
    }
};

// xi^a N^a, a = 3..8: FP32 folds the amplitudes into the draw (NodeNoise,
// PairNoise); FP64 scales unit normals (the arithmetic of the oracle's order).
template <class V, class Noise, class CC>
__device__ __forceinline__ void noise_increments(Noise& noise, V rho, const CC& cc, V xi[6]) {
    if constexpr (!std::is_same<V, double>::value) {
        noise.scaled(rho, cc, xi);
    } else {
        V N[6];
        noise(N);
        const V sr = sqr(rho);
#pragma unroll
        for (int a = 0; a < 6; ++a) xi[a] = (sr * N[a]) * V(cc.amp[a]);
    }
}

// True when every lane has a finite positive density and (f-norm) a basis:
// the common case, decided with one test instead of per-lane status codes.
__device__ __forceinline__ bool all_ok(double rho, double invsum) {
    return rho > 0 && rho < INFINITY && invsum < INFINITY;
}
__device__ __forceinline__ bool all_ok(float rho, float invsum) {
    return rho > 0.f && rho < INFINITY && invsum < INFINITY;
}
__device__ __forceinline__ bool all_ok(f2 rho, f2 invsum) {
    return fminf(rho.v.x, rho.v.y) > 0.f && fmaxf(rho.v.x, rho.v.y) < INFINITY &&
           invsum.v.x + invsum.v.y < INFINITY;
}

__device__ __forceinline__ double rsq_neg(double x) { return rsq(-x); }
__device__ __forceinline__ float rsq_neg(float x) { return rsq(-x); }
__device__ __forceinline__ f2 rsq_neg(f2 a) { return f2(rsq(-a.v.x), rsq(-a.v.y)); }

// Status per lane: bits [8k, 8k+8) hold the kStatus* code of lane k.
template <class V>
__device__ __forceinline__ uint32_t lane_status(V rho, V invsum, bool local) {
    uint32_t st = 0;
#pragma unroll
    for (int k = 0; k < Lanes<V>::n; ++k) {
        const auto r = lane(rho, k);
        uint32_t s = kStatusOk;
        if (!(r > 0) || !isfinite(r)) {
            s = kStatusNonfinite;
        } else if (local) {
            const auto q = lane(invsum, k);
            if (!isfinite(q)) s = kStatusInvalidVelocity;
        }
        st |= s << (8 * k);
    }
    return st;
}

// Lanes whose status is not ok keep their pre-collision populations.
__device__ __forceinline__ void keep_invalid(uint32_t st, const double g[9], double f[9]) {
    if (st)
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = g[i];
}
__device__ __forceinline__ void keep_invalid(uint32_t st, const float g[9], float f[9]) {
    if (st)
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = g[i];
}
__device__ __forceinline__ void keep_invalid(uint32_t st, const f2 g[9], f2 f[9]) {
    if (st) {
        const bool a = (st & 0xFF) != 0, b = (st >> 8) != 0;
#pragma unroll
        for (int i = 0; i < 9; ++i)
            f[i] = f2(a ? g[i].v.x : f[i].v.x, b ? g[i].v.y : f[i].v.y);
    }
}

// f* - g for the given non-conserved increments (Hermite coefficients D of
// P^T D, with D_1 = -K1, D_2 = -K2 folded into the constants).
template <class V, bool CONS>
__device__ __forceinline__ void hermite_back(V D0, V K1, V K2, const V Dn[6], V h[9]) {
    using S = typename Elem<V>::type;
    const V D3 = Dn[0], D4 = Dn[1], D5 = Dn[2], D6 = Dn[3], D7 = Dn[4], D8 = Dn[5];
    V base0, axis, diag, jxt, jyt;
    if (CONS) {
        base0 = mad(D8, V(S(0.5)), D0 - D5);
        axis = mad(D5, V(S(0.5)), D0 - D8);
        diag = mad(D5 + D8, V(S(2)), D0);
        jxt = K1 * V(S(-kSqrt3));
        jyt = K2 * V(S(-kSqrt3));
    } else {   // D0 = D1 = D2 = 0
        base0 = mad(D8, V(S(0.5)), V(S(0)) - D5);
        axis = mad(D5, V(S(0.5)), V(S(0)) - D8);
        diag = (D5 + D8) * V(S(2));
    }
    const V px = D3 * V(S(1.5)), pxy = D4 * V(S(3));
    const V qxa = D6 * V(S(kSqrt3h)), qya = D7 * V(S(kSqrt3h));
    const V ap = axis + px, am = axis - px;
    const V jq = CONS ? jxt - qxa : V(S(0)) - qxa;
    const V jqy = CONS ? jyt - qya : V(S(0)) - qya;
    h[0] = base0;
    h[1] = ap + jq;
    h[3] = ap - jq;
    h[2] = am + jqy;
    h[4] = am - jqy;
    const V a = diag + pxy, b = diag - pxy;
    // sqrt6 = 2 sqrt(3/2)
    const V ex = CONS ? mad(qxa, V(S(2)), jxt) : qxa * V(S(2));
    const V ey = CONS ? mad(qya, V(S(2)), jyt) : qya * V(S(2));
    const V xpy = ex + ey, xmy = ex - ey;
    h[5] = a + xpy;
    h[7] = a - xpy;
    h[8] = b + xmy;
    h[6] = b - xmy;
}

// Density, velocity and the non-equilibrium Hermite moments M^a - rho e_a(u),
// a = 3..8 (Eqs. d2q93a, d2q94), of the populations g, u = j / rho.
template <class V>
__device__ __forceinline__ void hermite_moments(const V g[9], V& rho, V& ux, V& uy, V (&M)[6]) {
    using S = typename Elem<V>::type;
    const V s13 = g[1] + g[3], s24 = g[2] + g[4];
    const V d13 = g[1] - g[3], d24 = g[2] - g[4];
    const V c58 = g[5] + g[8], c67 = g[6] + g[7];
    const V c56 = g[5] + g[6], c78 = g[7] + g[8];
    const V cx = c58 - c67, cy = c56 - c78;
    const V c = c58 + c67;
    const V s1234 = s13 + s24;
    rho = (g[0] + s1234) + c;
    const V jx = d13 + cx, jy = d24 + cy;
    const V ir = rcp(rho);
    ux = jx * ir;
    uy = jy * ir;
    const V uxx = ux * ux, uyy = uy * uy, uxy = ux * uy;
    const V usq = uxx + uyy;
    const V t3 = uxx - uyy;
    // Hermite equilibrium moments at rho = 1 (Eq. d2q94), negated: ne_a = -e_a
    const V ne3 = t3 * V(S(-1.5)), ne4 = uxy * V(S(-3)), ne5 = usq * V(S(-1.5));
    M[0] = mad(rho, ne3, (s13 - s24) * V(S(1.5)));
    M[1] = mad(rho, ne4, ((g[5] - g[6]) + (g[7] - g[8])) * V(S(3)));
    M[2] = mad(rho, ne5, mad(s1234, V(S(0.5)), c * V(S(2))) - g[0]);
    M[3] = mad(cx, V(S(kSqrt6)), d13 * V(S(-kSqrt3h)));
    M[4] = mad(cy, V(S(kSqrt6)), d24 * V(S(-kSqrt3h)));
    M[5] = mad(g[0], V(S(0.5)), c * V(S(2))) - s1234;
}

// The Cholesky factor of the f-norm Schur complement at a velocity u (the
// basis velocity), stored negated: Ln = -L' below the diagonal and inv_j =
// 1/L'_jj (infinite where a pivot is not positive: u outside the valid
// region). Inputs: u, its products and ne5 = -3/2 |u|^2.
//  * Sn = -S, S = G_NN - e e^T - k1 k1^T - k2 k2^T (upper triangle), in closed
//    form: with X = ux^2, Y = uy^2, Z = ux uy, Q = X + Y, D = X - Y the entries
//    are short polynomials (the rank-3 update cancels most terms of G_NN),
//    e.g. S_00 = 1 - 9Q/4 + 27/4 D^2 (1 - Q), S_22 = 1 - 9Q/4 + 27/4 Q^2 (1 - Q),
//    S_01 = 27/2 Z D (1 - Q), S_55 = 1 + 3Q/2.
//  * the factorisation and both triangular solves are chains of
//    fma(Ln, ., .) followed by one scaling with 1/L'_jj.
template <class V>
__device__ __forceinline__ void fnorm_factor(V ux, V uy, V uxx, V uyy, V uxy, V usq, V t3, V ne5,
                                             V (&Ln)[6][6], V (&inv)[6]) {
    using S = typename Elem<V>::type;
    V Sn[6][6];
    {
        const V Z2 = uxy * uxy, D2 = t3 * t3, Q2 = usq * usq;
        const V nv = mad(usq, V(S(6.75)), V(S(-6.75)));      // -27/4 (1 - Q)
        const V nv2 = mad(usq, V(S(13.5)), V(S(-13.5)));     // -27/2 (1 - Q)
        const V nc1 = mad(usq, V(S(2.25)), V(S(-1)));        // -(1 - 9Q/4)
        const V nw = mad(usq, V(S(-27)), V(S(18)));
        const V ax = ux * V(S(kSqrt6 / 4)), ay = uy * V(S(kSqrt6 / 4));
        Sn[0][0] = mad(D2, nv, nc1);
        Sn[2][2] = mad(Q2, nv, nc1);
        Sn[0][1] = (uxy * t3) * nv2;
        Sn[1][1] = mad(Z2 + Z2, nv2, V(S(-1)));
        Sn[1][2] = (uxy * usq) * nv2;
        Sn[0][2] = (t3 * V(S(2.25))) * mad(mad(usq, V(S(3)), V(S(-3))), usq, V(S(1)));
        Sn[0][5] = t3 * V(S(1.5));
        Sn[1][5] = uxy * V(S(-6));
        Sn[2][5] = ne5;
        Sn[3][5] = ux * V(S(-kSqrt6));
        Sn[4][5] = uy * V(S(-kSqrt6));
        Sn[5][5] = mad(usq, V(S(-1.5)), V(S(-1)));
        Sn[3][4] = uxy * mad(usq, V(S(9)), V(S(-6)));
        Sn[3][3] = mad(uyy, mad(uyy, V(S(4.5)), mad(uxx, V(S(18)), V(S(-1.5)))),
                       mad(uxx, V(S(-3)), V(S(-1))));
        Sn[4][4] = mad(uxx, mad(uxx, V(S(4.5)), mad(uyy, V(S(18)), V(S(-1.5)))),
                       mad(uyy, V(S(-3)), V(S(-1))));
        Sn[0][3] = ax * mad(uyy, mad(t3, V(S(-27)), V(S(-6))), V(S(2)));
        Sn[0][4] = ay * mad(uxx, mad(t3, V(S(-27)), V(S(6))), V(S(-2)));
        Sn[1][3] = ay * mad(Z2, V(S(-54)), mad(uxx, V(S(12)), mad(uyy, V(S(6)), V(S(-4)))));
        Sn[1][4] = ax * mad(Z2, V(S(-54)), mad(uyy, V(S(12)), mad(uxx, V(S(6)), V(S(-4)))));
        Sn[2][3] = ax * mad(uyy, nw, V(S(-2)));
        Sn[2][4] = ay * mad(uxx, nw, V(S(-2)));
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        V dn = Sn[j][j];                       // -(pivot)
#pragma unroll
        for (int k = 0; k < j; ++k) dn = mad(Ln[j][k], Ln[j][k], dn);
        inv[j] = rsq_neg(dn);
#pragma unroll
        for (int i = j + 1; i < 6; ++i) {
            V s = Sn[j][i];
#pragma unroll
            for (int k = 0; k < j; ++k) s = mad(Ln[i][k], Ln[j][k], s);
            Ln[i][j] = s * inv[j];
        }
    }
}

// The f-norm collision given the non-equilibrium Hermite moments M (of the
// node's own velocity) and the factor (Ln, inv) of the basis velocity u =
// (ux, uy), here the table velocity u_g of the look-up-table variant. The
// fully local collision (collide) takes the same steps with the node's own
// velocity written out in one body: split into this function it measured 3 %
// slower at 4096^2 (a different schedule of the same operations).
//  * M~_N = L'^{-1} M, relaxation towards M~^{a,0} = 0 (Eq. fnormmeq) plus
//    noise, D_N = L'^{-T} of the increments;
//  * the conserved increments from the rows of L below the conserved block at
//    u: -e, k1, k2 (zero entries omitted; cheap to rebuild from u, so they are
//    computed here rather than kept in registers across the factorisation);
//  * f* = g + W (.) P^T D, W_i = f_i^0(1, u) (Eq. d2q9f0). refetch(gg)
//    supplies g again. Returns the status (invsum infinite: no basis at u).
template <class V, class Noise, class Refetch, class CC>
__device__ __forceinline__ uint32_t fnorm_update(const V (&M)[6], const V (&Ln)[6][6], const V (&inv)[6],
                                                 V rho, V ux, V uy, Noise& noise, Refetch& refetch,
                                                 const CC& cc, V invsum, V f[9]) {
    using S = typename Elem<V>::type;
    const V uxx = ux * ux, uyy = uy * uy, uxy = ux * uy;
    const V usq = uxx + uyy;
    const V t3 = uxx - uyy;
    const V ne3 = t3 * V(S(-1.5)), ne4 = uxy * V(S(-3)), ne5 = usq * V(S(-1.5));
    const V s3x = ux * V(S(kSqrt3)), s3y = uy * V(S(kSqrt3));
    // M~_N = L'^{-1} (M_N - rho e_N)
    V y[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        V s = M[j];
#pragma unroll
        for (int k = 0; k < j; ++k) s = mad(Ln[j][k], y[k], s);
        y[j] = s * inv[j];
    }
    // increments: relaxation towards M~^{a,0} = 0 (Eq. fnormmeq) plus noise
    V z[6];
    noise_increments(noise, rho, cc, z);
#pragma unroll
    for (int a = 0; a < 6; ++a) z[a] = mad(nomega_of<V>(cc, a), y[a], z[a]);
    // D_N = L'^{-T} z
#pragma unroll
    for (int j = 5; j >= 0; --j) {
        V s = z[j];
#pragma unroll
        for (int k = j + 1; k < 6; ++k) s = mad(Ln[k][j], z[k], s);
        z[j] = s * inv[j];
    }
    const V nE = mad(ne3, z[0], mad(ne4, z[1], ne5 * z[2]));
    V k1[5], k2[5];
    {
        const V base = mad(usq, V(S(-1.5)), V(S(1)));   // 1 - e5
        k1[0] = s3x * mad(t3, V(S(-1.5)), V(S(1)));
        k1[1] = s3y * mad(uxx, V(S(-3)), V(S(1)));
        k1[2] = s3x * base;
        k1[3] = uyy * V(S(kSqrt2x3h));
        k1[4] = uxy * V(S(kSqrt2x3));
        k2[0] = s3y * mad(t3, V(S(-1.5)), V(S(-1)));
        k2[1] = s3x * mad(uyy, V(S(-3)), V(S(1)));
        k2[2] = s3y * base;
        k2[3] = k1[4];
        k2[4] = uxx * V(S(kSqrt2x3h));
    }
    const V K1 = mad(k1[0], z[0], mad(k1[1], z[1], mad(k1[2], z[2], mad(k1[3], z[3], k1[4] * z[4]))));
    const V K2 = mad(k2[0], z[0], mad(k2[1], z[1], mad(k2[2], z[2], mad(k2[3], z[3], k2[4] * z[4]))));
    const V D0 = mad(s3x, K1, mad(s3y, K2, nE));
    V h[9];
    hermite_back<V, true>(D0, K1, K2, z, h);
    // W_i = f_i^0(1, u) (Eq. d2q9f0)
    V W[9];
    {
        const V base = mad(usq, V(S(-1.5)), V(S(1)));
        const V b45 = mad(usq, V(S(4.5)), base);
        const V ax = mad(uxx, V(S(4.5)), base), ay = mad(uyy, V(S(4.5)), base);
        const V dp = mad(uxy, V(S(9)), b45), dm = mad(uxy, V(S(-9)), b45);
        const V spy = ux + uy, smy = ux - uy;
        W[0] = base * V(S(4.0 / 9.0));
        const V tx = ax * V(S(1.0 / 9.0)), ty = ay * V(S(1.0 / 9.0));
        W[1] = mad(ux, V(S(1.0 / 3.0)), tx);
        W[3] = mad(ux, V(S(-1.0 / 3.0)), tx);
        W[2] = mad(uy, V(S(1.0 / 3.0)), ty);
        W[4] = mad(uy, V(S(-1.0 / 3.0)), ty);
        const V tp = dp * V(S(1.0 / 36.0)), tm = dm * V(S(1.0 / 36.0));
        W[5] = mad(spy, V(S(1.0 / 12.0)), tp);
        W[7] = mad(spy, V(S(-1.0 / 12.0)), tp);
        W[8] = mad(smy, V(S(1.0 / 12.0)), tm);
        W[6] = mad(smy, V(S(-1.0 / 12.0)), tm);
    }

    V gg[9];
    refetch(gg);
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = mad(W[i], h[i], gg[i]);
    if (all_ok(rho, invsum)) return 0;
    const uint32_t st = lane_status(rho, invsum, true);
    keep_invalid(st, gg, f);
    return st;
}

// One collision. g: pre-collision populations; noise(N) fills the normals
// N^3..N^8 (called once, after the basis is built, to keep registers free);
// f: output.
template <class V, int BASIS, class Noise, class CC>
__device__ __forceinline__ uint32_t collide(const V g[9], Noise noise, const CC& cc, V f[9]) {
    return collide<V, BASIS>(g, noise, [&](V* gg) {
#pragma unroll
        for (int i = 0; i < 9; ++i) gg[i] = g[i];
    }, cc, f);
}

// As above; refetch(gg) supplies g again for the final f = g + W h, so the
// caller may drop g from registers in between (the pipelined kernel re-reads
// it from shared memory).
template <class V, int BASIS, class Noise, class Refetch, class CC>
__device__ __forceinline__ uint32_t collide(const V g[9], Noise noise, Refetch refetch,
                                            const CC& cc, V f[9]) {
    using S = typename Elem<V>::type;
    // density, momentum, velocity
    const V s13 = g[1] + g[3], s24 = g[2] + g[4];
    const V d13 = g[1] - g[3], d24 = g[2] - g[4];
    const V c58 = g[5] + g[8], c67 = g[6] + g[7];
    const V c56 = g[5] + g[6], c78 = g[7] + g[8];
    const V cx = c58 - c67, cy = c56 - c78;
    const V c = c58 + c67;
    const V s1234 = s13 + s24;
    const V rho = (g[0] + s1234) + c;
    const V jx = d13 + cx, jy = d24 + cy;
    const V ir = rcp(rho);
    const V ux = jx * ir, uy = jy * ir;
    const V uxx = ux * ux, uyy = uy * uy, uxy = ux * uy;
    const V usq = uxx + uyy;
    const V t3 = uxx - uyy;
    // Hermite equilibrium moments at rho = 1 (Eq. d2q94), negated: ne_a = -e_a
    const V ne3 = t3 * V(S(-1.5)), ne4 = uxy * V(S(-3)), ne5 = usq * V(S(-1.5));
    // non-equilibrium Hermite moments M^a - rho e_a, a = 3..8
    V M[6];
    M[0] = mad(rho, ne3, (s13 - s24) * V(S(1.5)));
    M[1] = mad(rho, ne4, ((g[5] - g[6]) + (g[7] - g[8])) * V(S(3)));
    M[2] = mad(rho, ne5, mad(s1234, V(S(0.5)), c * V(S(2))) - g[0]);
    M[3] = mad(cx, V(S(kSqrt6)), d13 * V(S(-kSqrt3h)));
    M[4] = mad(cy, V(S(kSqrt6)), d24 * V(S(-kSqrt3h)));
    M[5] = mad(g[0], V(S(0.5)), c * V(S(2))) - s1234;

    if (BASIS == 0) {
        // Hermite norm: D_a = -omega_a (M^a - M^{a,0}) + xi^a N^a, f* = g + w (.) P^T D
        V Dn[6];
        noise_increments(noise, rho, cc, Dn);
#pragma unroll
        for (int a = 0; a < 6; ++a) Dn[a] = mad(nomega_of<V>(cc, a), M[a], Dn[a]);
        V h[9];
        hermite_back<V, false>(V(S(0)), V(S(0)), V(S(0)), Dn, h);
        V gg[9];
        refetch(gg);
        f[0] = mad(h[0], V(S(4.0 / 9.0)), gg[0]);
#pragma unroll
        for (int i = 1; i <= 4; ++i) f[i] = mad(h[i], V(S(1.0 / 9.0)), gg[i]);
#pragma unroll
        for (int i = 5; i <= 8; ++i) f[i] = mad(h[i], V(S(1.0 / 36.0)), gg[i]);
        if (all_ok(rho, V(S(0)))) return 0;
        const uint32_t st = lane_status(rho, rho, false);
        keep_invalid(st, gg, f);
        return st;
    }

    // rows of L below the conserved block: -e, k1, k2 (zero entries omitted);
    // cheap to rebuild from u, so they are recomputed where needed instead of
    // being kept in registers across the factorisation
    const V s3x = ux * V(S(kSqrt3)), s3y = uy * V(S(kSqrt3));
    auto rows = [&](V k1[5], V k2[5]) {
        const V base = mad(usq, V(S(-1.5)), V(S(1)));   // 1 - e5
        k1[0] = s3x * mad(t3, V(S(-1.5)), V(S(1)));
        k1[1] = s3y * mad(uxx, V(S(-3)), V(S(1)));
        k1[2] = s3x * base;
        k1[3] = uyy * V(S(kSqrt2x3h));
        k1[4] = uxy * V(S(kSqrt2x3));
        k2[0] = s3y * mad(t3, V(S(-1.5)), V(S(-1)));
        k2[1] = s3x * mad(uyy, V(S(-3)), V(S(1)));
        k2[2] = s3y * base;
        k2[3] = k1[4];
        k2[4] = uxx * V(S(kSqrt2x3h));
    };

    V Ln[6][6], inv[6];
    fnorm_factor(ux, uy, uxx, uyy, uxy, usq, t3, ne5, Ln, inv);
    const V invsum = ((inv[0] + inv[1]) + (inv[2] + inv[3])) + (inv[4] + inv[5]);

    // M~_N = L'^{-1} (M_N - rho e_N)
    V y[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        V s = M[j];
#pragma unroll
        for (int k = 0; k < j; ++k) s = mad(Ln[j][k], y[k], s);
        y[j] = s * inv[j];
    }
    // increments: relaxation towards M~^{a,0} = 0 (Eq. fnormmeq) plus noise
    V z[6];
    noise_increments(noise, rho, cc, z);
#pragma unroll
    for (int a = 0; a < 6; ++a) z[a] = mad(nomega_of<V>(cc, a), y[a], z[a]);
    // D_N = L'^{-T} z
#pragma unroll
    for (int j = 5; j >= 0; --j) {
        V s = z[j];
#pragma unroll
        for (int k = j + 1; k < 6; ++k) s = mad(Ln[k][j], z[k], s);
        z[j] = s * inv[j];
    }
    const V nE = mad(ne3, z[0], mad(ne4, z[1], ne5 * z[2]));
    V k1[5], k2[5];
    rows(k1, k2);
    const V K1 = mad(k1[0], z[0], mad(k1[1], z[1], mad(k1[2], z[2], mad(k1[3], z[3], k1[4] * z[4]))));
    const V K2 = mad(k2[0], z[0], mad(k2[1], z[1], mad(k2[2], z[2], mad(k2[3], z[3], k2[4] * z[4]))));
    const V D0 = mad(s3x, K1, mad(s3y, K2, nE));
    V h[9];
    hermite_back<V, true>(D0, K1, K2, z, h);
    // W_i = f_i^0(1, u) (Eq. d2q9f0)
    V W[9];
    {
        const V base = mad(usq, V(S(-1.5)), V(S(1)));
        const V b45 = mad(usq, V(S(4.5)), base);
        const V ax = mad(uxx, V(S(4.5)), base), ay = mad(uyy, V(S(4.5)), base);
        const V dp = mad(uxy, V(S(9)), b45), dm = mad(uxy, V(S(-9)), b45);
        const V spy = ux + uy, smy = ux - uy;
        W[0] = base * V(S(4.0 / 9.0));
        const V tx = ax * V(S(1.0 / 9.0)), ty = ay * V(S(1.0 / 9.0));
        W[1] = mad(ux, V(S(1.0 / 3.0)), tx);
        W[3] = mad(ux, V(S(-1.0 / 3.0)), tx);
        W[2] = mad(uy, V(S(1.0 / 3.0)), ty);
        W[4] = mad(uy, V(S(-1.0 / 3.0)), ty);
        const V tp = dp * V(S(1.0 / 36.0)), tm = dm * V(S(1.0 / 36.0));
        W[5] = mad(spy, V(S(1.0 / 12.0)), tp);
        W[7] = mad(spy, V(S(-1.0 / 12.0)), tp);
        W[8] = mad(smy, V(S(1.0 / 12.0)), tm);
        W[6] = mad(smy, V(S(-1.0 / 12.0)), tm);
    }

    V gg[9];
    refetch(gg);
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = mad(W[i], h[i], gg[i]);
    if (all_ok(rho, invsum)) return 0;
    const uint32_t st = lane_status(rho, invsum, true);
    keep_invalid(st, gg, f);
    return st;
}

// ---------------------------------------------------------------------------
// Look-up-table f-norm (Section 4, the paper's practical variant): the basis at
// the nearest velocity u_g of a 51 x 51 table, u_g = ((k_x - 25)/50,
// (k_y - 25)/50), k = floor(50 u + 25.5) in 0..50. The collision projects
// g - f^0(rho, u) (the node's own equilibrium, taken exactly) on the f-norm
// basis at u_g, Y^a = m~^a(u_g) . (g - f^0(rho, u)), relaxes and adds noise,
// D^a = -omega_a Y^a + xi^a N^a, and returns f* = g + W(u_g) (.) sum_a m~^a D^a.
// Since g - f^0(rho, u) carries no mass or momentum, Y_N = L'(u_g)^{-1} (M_N -
// rho e_N(u)) with the Hermite moments of the node: the local f-norm update
// (fnorm_update) with the factor of u_g in place of the node's. A table entry
// therefore holds that factor: Ln (the 15 entries below the diagonal, row by
// row), inv (6), u_g (2) and a validity flag (0 where some W_i(u_g) <= 0, with
// inv infinite there), 24 values, built in FP64.
// ---------------------------------------------------------------------------
constexpr int kLutN = 51;
constexpr int kLutStride = 24;   // values per entry
constexpr int kLutInv = 15;
constexpr int kLutU = 21;
constexpr int kLutFlag = 23;

__host__ __device__ constexpr int lut_ln_index(int i, int j) { return i * (i - 1) / 2 + j; }   // i > j

__device__ __forceinline__ double lut_coord(double u) {
    return floor(__dadd_rn(__dmul_rn(50.0, u), 25.5));
}
__device__ __forceinline__ float lut_coord(float u) {
    return floorf(__fadd_rn(__fmul_rn(50.0f, u), 25.5f));
}

// Table cell of velocity u, or -1 off the table (NaN included).
template <class S>
__device__ __forceinline__ int lut_cell(S ux, S uy) {
    const S kx = lut_coord(ux), ky = lut_coord(uy);
    if (!(kx >= S(0) && kx <= S(kLutN - 1) && ky >= S(0) && ky <= S(kLutN - 1))) return -1;
    return (int)ky * kLutN + (int)kx;
}

// One table entry (16-byte aligned) through the read-only path.
__device__ __forceinline__ void lut_load_entry(const float* p, float (&r)[kLutStride]) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int k = 0; k < kLutStride / 4; ++k) {
        const float4 v = __ldg(q + k);
        r[4 * k] = v.x;
        r[4 * k + 1] = v.y;
        r[4 * k + 2] = v.z;
        r[4 * k + 3] = v.w;
    }
}
__device__ __forceinline__ void lut_load_entry(const double* p, double (&r)[kLutStride]) {
    const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int k = 0; k < kLutStride / 2; ++k) {
        const double2 v = __ldg(q + k);
        r[2 * k] = v.x;
        r[2 * k + 1] = v.y;
    }
}

template <class V, class Noise, class Refetch, class CC>
__device__ __forceinline__ uint32_t collide_lut(const V g[9], Noise noise, Refetch refetch,
                                                const typename Elem<V>::type* lut, const CC& cc,
                                                V f[9]) {
    using S = typename Elem<V>::type;
    constexpr int NL = Lanes<V>::n;
    V rho, ux, uy, M[6];
    hermite_moments(g, rho, ux, uy, M);
    // the factor of each lane's table velocity; off the table or at an
    // invalid cell, inv is infinite (the status then keeps the lane's g)
    S e[NL][kLutStride];
    bool on[NL];
#pragma unroll
    for (int k = 0; k < NL; ++k) {
        const int cell = lut_cell(lane(ux, k), lane(uy, k));
        on[k] = cell >= 0;
        lut_load_entry(lut + (size_t)(cell < 0 ? 0 : cell) * kLutStride, e[k]);
    }
    auto val = [&](int q) {
        if constexpr (NL == 1)
            return V(e[0][q]);
        else
            return V(e[0][q], e[NL - 1][q]);
    };
    V Ln[6][6], inv[6];
#pragma unroll
    for (int i = 1; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < i; ++j) Ln[i][j] = val(lut_ln_index(i, j));
#pragma unroll
    for (int j = 0; j < 6; ++j) inv[j] = val(kLutInv + j);
    V invsum = ((inv[0] + inv[1]) + (inv[2] + inv[3])) + (inv[4] + inv[5]);
    if (!(on[0] && on[NL - 1])) {
        if constexpr (NL == 1)
            invsum = V(S(INFINITY));
        else
            invsum = V(on[0] ? lane(invsum, 0) : S(INFINITY), on[1] ? lane(invsum, 1) : S(INFINITY));
    }
    return fnorm_update<V>(M, Ln, inv, rho, val(kLutU), val(kLutU + 1), noise, refetch, cc, invsum, f);
}

// The collision of basis BASIS: 0 Hermite norm, 1 f-norm, 2 look-up-table
// f-norm (lut: the velocity table, unused otherwise).
template <class V, int BASIS, class Noise, class Refetch, class CC>
__device__ __forceinline__ uint32_t collide_basis(const V g[9], Noise noise, Refetch refetch,
                                                  const typename Elem<V>::type* lut, const CC& cc,
                                                  V f[9]) {
    if constexpr (BASIS == 2)
        return collide_lut<V>(g, noise, refetch, lut, cc, f);
    else
        return collide<V, BASIS>(g, noise, refetch, cc, f);
}

}  // namespace flb
