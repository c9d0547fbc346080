/*
 * flb_oracle.c -- plain FP64 CPU oracle of the fluctuating D2Q9 lattice-Boltzmann
 * method of Kaehler & Wagner (arXiv:1204.6734).
 *
 * TEST INFRASTRUCTURE. Loaded only by the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark; never by the product. Shares no code with
 * the CUDA path. Compiled with -ffp-contract=off so that x86-64 and aarch64
 * hosts round every operation the same way.
 *
 * Every function cites the passage it follows. Where the paper is silent or
 * garbled the reading taken is stated at the point of use.
 */
#include "flb_oracle.h"

#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* D2Q9 tables (Appendix "Hermite norm D2Q9")                                */
/* ------------------------------------------------------------------------- */

/* Fig. 1 (the velocity diagram) is not available; the order of the v_i is the
 * one implied by the j_x and j_y rows of Eq. d2q93a, which equal sqrt(3) v_x
 * and sqrt(3) v_y. */
static const int VX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int VY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

/* Eq. d2q9w */
static double weight(int i) {
    if (i == 0) return 4.0 / 9.0;
    if (i <= 4) return 1.0 / 9.0;
    return 1.0 / 36.0;
}

/* Eq. d2q93a, forward transform m[a][i], entries as printed. */
static void hermite_m(double m[9][9]) {
    const double s3 = sqrt(3.0), s32 = sqrt(1.5), s6 = sqrt(6.0);
    const double rows[9][9] = {
        {1, 1, 1, 1, 1, 1, 1, 1, 1},
        {0, s3, 0, -s3, 0, s3, -s3, -s3, s3},
        {0, 0, s3, 0, -s3, s3, s3, -s3, -s3},
        {0, 1.5, -1.5, 1.5, -1.5, 0, 0, 0, 0},
        {0, 0, 0, 0, 0, 3, -3, 3, -3},
        {-1, 0.5, 0.5, 0.5, 0.5, 2, 2, 2, 2},
        {0, -s32, 0, s32, 0, s6, -s6, -s6, s6},
        {0, 0, -s32, 0, s32, s6, s6, -s6, -s6},
        {0.5, -1, -1, -1, -1, 2, 2, 2, 2},
    };
    memcpy(m, rows, sizeof(rows));
}

/* Eq. d2q93b, back transform n[i][a], entries as printed. */
static void hermite_n(double n[9][9]) {
    const double a = 1.0 / (3.0 * sqrt(3.0));   /* 1/(3 sqrt3)  */
    const double b = 1.0 / (3.0 * sqrt(6.0));   /* 1/(3 sqrt6)  */
    const double c = 1.0 / (12.0 * sqrt(3.0));  /* 1/(12 sqrt3) */
    const double d = 1.0 / (6.0 * sqrt(6.0));   /* 1/(6 sqrt6)  */
    const double rows[9][9] = {
        {4.0 / 9, 0, 0, 0, 0, -4.0 / 9, 0, 0, 2.0 / 9},
        {1.0 / 9, a, 0, 1.0 / 6, 0, 1.0 / 18, -b, 0, -1.0 / 9},
        {1.0 / 9, 0, a, -1.0 / 6, 0, 1.0 / 18, 0, -b, -1.0 / 9},
        {1.0 / 9, -a, 0, 1.0 / 6, 0, 1.0 / 18, b, 0, -1.0 / 9},
        {1.0 / 9, 0, -a, -1.0 / 6, 0, 1.0 / 18, 0, b, -1.0 / 9},
        {1.0 / 36, c, c, 0, 1.0 / 12, 1.0 / 18, d, d, 1.0 / 18},
        {1.0 / 36, -c, c, 0, -1.0 / 12, 1.0 / 18, -d, d, 1.0 / 18},
        {1.0 / 36, -c, -c, 0, 1.0 / 12, 1.0 / 18, -d, -d, 1.0 / 18},
        {1.0 / 36, c, -c, 0, -1.0 / 12, 1.0 / 18, d, -d, 1.0 / 18},
    };
    memcpy(n, rows, sizeof(rows));
}

void orc_tables(int vx[9], int vy[9], double w[9], double m[81], double n[81]) {
    double mm[9][9], nn[9][9];
    hermite_m(mm);
    hermite_n(nn);
    for (int i = 0; i < 9; ++i) {
        if (vx) vx[i] = VX[i];
        if (vy) vy[i] = VY[i];
        if (w) w[i] = weight(i);
    }
    if (m) memcpy(m, mm, sizeof(mm));
    if (n) memcpy(n, nn, sizeof(nn));
}

/* Eq. d2q9f0 (Eq. f0 with theta = 1/3):
 * f_i^0 = rho w_i [1 + 3 u.v_i + 9/2 (u.v_i)^2 - 3/2 u.u] */
void orc_feq(double rho, double ux, double uy, double f0[9]) {
    const double uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        const double uv = ux * VX[i] + uy * VY[i];
        f0[i] = rho * weight(i) * (1.0 + 3.0 * uv + 4.5 * uv * uv - 1.5 * uu);
    }
}

/* Eq. d2q94: equilibrium moments in the Hermite norm. */
void orc_hermite_meq(double rho, double ux, double uy, double meq[9]) {
    const double s3 = sqrt(3.0);
    meq[0] = rho;
    meq[1] = s3 * rho * ux;
    meq[2] = s3 * rho * uy;
    meq[3] = 1.5 * rho * (ux * ux - uy * uy);
    meq[4] = 3.0 * rho * ux * uy;
    meq[5] = 1.5 * rho * (ux * ux + uy * uy);
    meq[6] = 0.0;
    meq[7] = 0.0;
    meq[8] = 0.0;
}

/* ------------------------------------------------------------------------- */
/* f-norm basis (Section 4, Eqs. fnorm, fnormsp, gramschmidt, gsortho)        */
/* ------------------------------------------------------------------------- */

/* Readings taken (the paper is ambiguous here):
 *  - the scalar product weight is W_i = f_i^0(1, u) (Eq. fnorm), so that the
 *    basis depends on u only and Eq. fnormmeq holds; Eq. fnormsp writes f_i^0,
 *    which differs by the factor rho;
 *  - Eq. gsortho divides by the squared norm; orthonormality (Eq. fnorm)
 *    requires the square root, which is what is done here;
 *  - the paper lists the six physical start vectors rho, j_x, j_y, Pi_xx-yy,
 *    Pi_xy, Pi_xx+yy; the three ghost rows q_x, q_y, epsilon of Eq. d2q93a
 *    follow them in that order.
 * The projection coefficients are taken against the unmodified start vector,
 * as Eq. gramschmidt writes them (classical Gram-Schmidt). */
int orc_local_basis(double ux, double uy, double mt[81]) {
    double p[9][9], W[9];
    hermite_m(p);
    orc_feq(1.0, ux, uy, W);
    for (int i = 0; i < 9; ++i)
        if (!(W[i] > 0.0)) return ORC_ERR_INVALID_VELOCITY;

    for (int a = 0; a < 9; ++a) {
        double mhat[9];
        for (int i = 0; i < 9; ++i) mhat[i] = p[a][i];
        for (int b = 0; b < a; ++b) {
            double proj = 0.0; /* sum_j mt^b_j f^0_j m^a_j */
            for (int j = 0; j < 9; ++j) proj += mt[b * 9 + j] * W[j] * p[a][j];
            for (int i = 0; i < 9; ++i) mhat[i] -= mt[b * 9 + i] * proj;
        }
        double nrm2 = 0.0;
        for (int j = 0; j < 9; ++j) nrm2 += mhat[j] * W[j] * mhat[j];
        if (!(nrm2 > 0.0)) return ORC_ERR_INVALID_VELOCITY;
        const double nrm = sqrt(nrm2);
        for (int i = 0; i < 9; ++i) mt[a * 9 + i] = mhat[i] / nrm;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Random numbers                                                            */
/* ------------------------------------------------------------------------- */

/* Philox4x32-10 as defined by Salmon, Moraes, Dror and Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64-bit
 * products, the key bumped by the Weyl constants between rounds. */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        const uint64_t p0 = (uint64_t)PHILOX_M0 * x0;
        const uint64_t p1 = (uint64_t)PHILOX_M1 * x2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t y0 = hi1 ^ x1 ^ k0;
        const uint32_t y1 = lo1;
        const uint32_t y2 = hi0 ^ x3 ^ k1;
        const uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Noise draw of one node-step. Counter (node, step, replica, 0), key = seed.
 * The 128 output bits X = out0 + 2^32 out1 + 2^64 out2 + 2^96 out3 are cut
 * into six 21-bit fields k_q = (X >> 21 q) mod 2^21, q = 0..5. */
void orc_draw_fields(uint64_t seed, uint32_t replica, uint32_t node, uint32_t step,
                     uint32_t fields[6]) {
    const uint32_t ctr[4] = {node, step, replica, 0u};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    for (int q = 0; q < 6; ++q) {
        uint32_t k = 0;
        for (int b = 0; b < 21; ++b) {
            const int bit = 21 * q + b;            /* bit index in X */
            const uint32_t v = (out[bit / 32] >> (bit % 32)) & 1u;
            k |= v << b;
        }
        fields[q] = k;
    }
}

/* Box-Muller on the pairs (k_0,k_1), (k_2,k_3), (k_4,k_5):
 *   u1 = (k_{2p} + 1) / 2^21 in (0,1],  u2 = k_{2p+1} / 2^21 in [0,1),
 *   N_{2p} = sqrt(-2 ln u1) cos(2 pi u2),  N_{2p+1} = sqrt(-2 ln u1) sin(2 pi u2). */
void orc_normals(uint64_t seed, uint32_t replica, uint32_t node, uint32_t step,
                 double nrm[6]) {
    uint32_t k[6];
    orc_draw_fields(seed, replica, node, step, k);
    const double scale = 1.0 / 2097152.0; /* 2^-21 */
    const double two_pi = 6.283185307179586476925286766559;
    for (int p = 0; p < 3; ++p) {
        const double u1 = ((double)k[2 * p] + 1.0) * scale;
        const double u2 = (double)k[2 * p + 1] * scale;
        const double r = sqrt(-2.0 * log(u1));
        nrm[2 * p] = r * cos(two_pi * u2);
        nrm[2 * p + 1] = r * sin(two_pi * u2);
    }
}

/* ------------------------------------------------------------------------- */
/* Collision (Eq. LBEMRT)                                                    */
/* ------------------------------------------------------------------------- */

/* Eq. noiseamp with 1/tau^a = omega_a and the variance scale k_B T:
 *   xi^a = (1/tau^a) sqrt(kT rho (2 tau^a - 1)) = sqrt(kT rho omega_a (2 - omega_a)),
 * so that <dM^a dM^b> = kT rho delta^{ab} (Eq. fluctf4 with Poisson statistics
 * scaled by kT); rho is the density of the colliding node. */
static double noise_amplitude(double kT, double rho, double omega) {
    const double v = kT * rho * omega * (2.0 - omega);
    return v > 0.0 ? sqrt(v) : 0.0;
}

/* Standard (Hermite norm) collision: forward transform with m (Eq. d2q93a),
 * relaxation towards the moments of Eq. d2q94 with Lambda^{ab} = -omega_a
 * delta^{ab}, noise xi^a N^a on the non-conserved moments a = 3..8, back
 * transform with n (Eq. d2q93b). */
static int collide_standard(const orc_params* p, const double g[9], const double N[6],
                            double fstar[9]) {
    double m[9][9], n[9][9];
    hermite_m(m);
    hermite_n(n);
    double M[9];
    for (int a = 0; a < 9; ++a) {
        M[a] = 0.0;
        for (int i = 0; i < 9; ++i) M[a] += m[a][i] * g[i];
    }
    const double rho = M[0];
    const double ux = M[1] / (sqrt(3.0) * rho);
    const double uy = M[2] / (sqrt(3.0) * rho);
    double Meq[9];
    orc_hermite_meq(rho, ux, uy, Meq);
    /* Eq. LBEMRT in its increment form: f* - f = sum_a n^a_i dM^a with
     * dM^a = -omega_a (M^a - M^{a,0}) + xi^a N^a for a = 3..8 and dM^a = 0 for
     * the conserved a = 0, 1, 2. */
    double dM[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int a = 3; a < 9; ++a)
        dM[a] = -p->omega[a] * (M[a] - Meq[a]) +
                noise_amplitude(p->kT, rho, p->omega[a]) * N[a - 3];
    for (int i = 0; i < 9; ++i) {
        double df = 0.0;
        for (int a = 0; a < 9; ++a) df += n[i][a] * dM[a];
        fstar[i] = g[i] + df;
    }
    return ORC_OK;
}

/* Local (f-norm) collision of Section 4: rho and u of the node, the basis
 * mt(u) by Gram-Schmidt, moments Mt^a = sum_i mt^a_i g_i (Eq. Mtilde),
 * relaxation towards Mt^{a,0} = rho delta^{a0} (Eq. fnormmeq) plus noise for
 * a = 3..8, and the back transform with n^a_i = mt^a_i f_i^0(rho,u)/rho
 * (the choice made below Eq. fluctf2). The conserved moments a = 0, 1, 2 are
 * passed through unchanged: their increment is zero. */
static int collide_local(const orc_params* p, const double g[9], const double N[6],
                         double fstar[9]) {
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) {
        rho += g[i];
        jx += g[i] * VX[i];
        jy += g[i] * VY[i];
    }
    if (!(rho > 0.0) || !isfinite(jx) || !isfinite(jy)) return ORC_ERR_NONFINITE;
    const double ux = jx / rho, uy = jy / rho;
    double mt[81];
    const int rc = orc_local_basis(ux, uy, mt);
    if (rc != ORC_OK) return rc;
    double W[9];
    orc_feq(1.0, ux, uy, W);

    double Mt[9];
    for (int a = 0; a < 9; ++a) {
        Mt[a] = 0.0;
        for (int i = 0; i < 9; ++i) Mt[a] += mt[a * 9 + i] * g[i];
    }
    /* increment form of Eq. LBEMRT, as for the Hermite norm */
    double dM[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int a = 3; a < 9; ++a) {
        const double Meq = 0.0; /* Eq. fnormmeq */
        dM[a] = -p->omega[a] * (Mt[a] - Meq) +
                noise_amplitude(p->kT, rho, p->omega[a]) * N[a - 3];
    }
    for (int i = 0; i < 9; ++i) {
        double df = 0.0;
        for (int a = 0; a < 9; ++a) df += mt[a * 9 + i] * W[i] * dM[a];
        fstar[i] = g[i] + df;
    }
    return ORC_OK;
}

/* Look-up-table f-norm (the practical variant of Section 4): the basis is not
 * formed at the node's own velocity u but at the nearest velocity u_g of a
 * 51 x 51 table, u_g = ((k_x - 25)/50, (k_y - 25)/50), k = 0..50 (spacing
 * 0.02, |u_g| <= 0.5 per component), k = floor(50 u + 25.5). A velocity off the
 * table, or a table velocity where some f_i^0(1, u_g) <= 0 (the corners, Fig.
 * 11), has no basis: the paper's run fails there. */
int orc_lut_velocity(double ux, double uy, double* ugx, double* ugy) {
    const double kx = floor(50.0 * ux + 25.5), ky = floor(50.0 * uy + 25.5);
    if (!(kx >= 0.0 && kx <= 50.0 && ky >= 0.0 && ky <= 50.0)) return ORC_ERR_INVALID_VELOCITY;
    *ugx = (kx - 25.0) / 50.0;
    *ugy = (ky - 25.0) / 50.0;
    return ORC_OK;
}

/* The collision with the table basis mt(u_g): moments Mt^a = sum_i mt^a_i g_i;
 * the equilibrium moments in that basis are no longer rho delta^{a0} (Eq.
 * fnormmeq holds only at u_g = u) but the projection Mt^{a,eq} = sum_i mt^a_i
 * f_i^0(rho, u) of the node's equilibrium (the paper keeps that projection to
 * O(u_g^3); here it is taken exactly); relaxation towards it with
 * Lambda = -omega_a and noise xi^a N^a for a = 3..8, and the back transform
 * with n^a_i = mt^a_i f_i^0(1, u_g). The conserved moments pass through. */
static int collide_lut(const orc_params* p, const double g[9], const double N[6],
                       double fstar[9]) {
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) {
        rho += g[i];
        jx += g[i] * VX[i];
        jy += g[i] * VY[i];
    }
    if (!(rho > 0.0) || !isfinite(jx) || !isfinite(jy)) return ORC_ERR_NONFINITE;
    const double ux = jx / rho, uy = jy / rho;
    double ugx, ugy;
    int rc = orc_lut_velocity(ux, uy, &ugx, &ugy);
    if (rc != ORC_OK) return rc;
    double mt[81];
    rc = orc_local_basis(ugx, ugy, mt);
    if (rc != ORC_OK) return rc;
    double Wg[9], f0[9];
    orc_feq(1.0, ugx, ugy, Wg);
    orc_feq(rho, ux, uy, f0);

    double Mt[9], Mteq[9];
    for (int a = 0; a < 9; ++a) {
        Mt[a] = 0.0;
        Mteq[a] = 0.0;
        for (int i = 0; i < 9; ++i) {
            Mt[a] += mt[a * 9 + i] * g[i];
            Mteq[a] += mt[a * 9 + i] * f0[i];
        }
    }
    double dM[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int a = 3; a < 9; ++a)
        dM[a] = -p->omega[a] * (Mt[a] - Mteq[a]) +
                noise_amplitude(p->kT, rho, p->omega[a]) * N[a - 3];
    for (int i = 0; i < 9; ++i) {
        double df = 0.0;
        for (int a = 0; a < 9; ++a) df += mt[a * 9 + i] * Wg[i] * dM[a];
        fstar[i] = g[i] + df;
    }
    return ORC_OK;
}

int orc_collide_node(const orc_params* p, const double g[9], uint32_t node,
                     uint32_t step, double fstar[9]) {
    double N[6];
    orc_normals(p->seed, p->replica, node, step, N);
    int rc;
    if (p->basis == ORC_BASIS_STANDARD)
        rc = collide_standard(p, g, N, fstar);
    else if (p->basis == ORC_BASIS_LOCAL)
        rc = collide_local(p, g, N, fstar);
    else if (p->basis == ORC_BASIS_LOCAL_LUT)
        rc = collide_lut(p, g, N, fstar);
    else
        return ORC_ERR_ARG;
    if (rc != ORC_OK) return rc;
    for (int i = 0; i < 9; ++i)
        if (!isfinite(fstar[i])) return ORC_ERR_NONFINITE;
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Lattice update (Eq. LBE1) and sampling                                    */
/* ------------------------------------------------------------------------- */

void orc_init_equilibrium(const orc_params* p, double* f) {
    double f0[9];
    orc_feq(p->rho0, p->ux0, p->uy0, f0);
    const size_t nn = (size_t)p->Lx * (size_t)p->Ly;
    for (int i = 0; i < 9; ++i)
        for (size_t k = 0; k < nn; ++k) f[(size_t)i * nn + k] = f0[i];
}

static int wrap(int a, int L) {
    a %= L;
    return a < 0 ? a + L : a;
}

/* One time step of Eq. LBE1 at every node: collide at x, then move the result
 * to x + v_i with periodic wrap-around (push form of the streaming). The
 * equal-time statistics use the pre-collision f_i(x, t) and the reference
 * c = f^0(rho0, u0) of Eq. efif0. */
int orc_run(const orc_params* p, double* f, int64_t step0, int64_t nsteps,
            int64_t warmup, int64_t every, double* S1, double* S2, int64_t* nsamp,
            int64_t* err_node, int64_t* err_step) {
    if (!p || !f || p->Lx <= 0 || p->Ly <= 0 || nsteps < 0) return ORC_ERR_ARG;
    const int Lx = p->Lx, Ly = p->Ly;
    const size_t nn = (size_t)Lx * (size_t)Ly;
    double c[9];
    orc_feq(p->rho0, p->ux0, p->uy0, c);

    /* the next state, on the C heap */
    double* next = (double*)malloc(sizeof(double) * 9 * nn);
    if (!next) return ORC_ERR_ARG;

    int rc = ORC_OK;
    for (int64_t s = 0; s < nsteps && rc == ORC_OK; ++s) {
        const int64_t t = step0 + s;
        const int sample = every > 0 && t >= warmup && ((t - warmup) % every) == 0;
        for (int y = 0; y < Ly && rc == ORC_OK; ++y) {
            for (int x = 0; x < Lx; ++x) {
                const size_t node = (size_t)x + (size_t)Lx * (size_t)y;
                double g[9], fs[9];
                for (int i = 0; i < 9; ++i) g[i] = f[(size_t)i * nn + node];
                if (sample) {
                    double d[9];
                    for (int i = 0; i < 9; ++i) d[i] = g[i] - c[i];
                    for (int i = 0; i < 9; ++i) {
                        S1[i] += d[i];
                        for (int j = 0; j < 9; ++j) S2[i * 9 + j] += d[i] * d[j];
                    }
                }
                rc = orc_collide_node(p, g, (uint32_t)node, (uint32_t)t, fs);
                if (rc != ORC_OK) {
                    if (err_node) *err_node = (int64_t)node;
                    if (err_step) *err_step = t;
                    break;
                }
                for (int i = 0; i < 9; ++i) {
                    const int xd = wrap(x + VX[i], Lx), yd = wrap(y + VY[i], Ly);
                    next[(size_t)i * nn + (size_t)xd + (size_t)Lx * (size_t)yd] = fs[i];
                }
            }
        }
        if (rc == ORC_OK) {
            memcpy(f, next, sizeof(double) * 9 * nn);
            if (sample && nsamp) *nsamp += (int64_t)nn;
        }
    }
    free(next);
    return rc;
}
