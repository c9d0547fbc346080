// flb_basis.cuh -- explicit basis matrices in FP64 (one thread): the Hermite
// rows P (Eq. d2q93a) and the f-norm basis m~(u) = L^{-1} P at a velocity u,
// L the Cholesky factor of the Gram matrix G = P diag(W) P^T, W = f^0(1, u)
// (Eqs. fnorm, gramschmidt). Used where the basis itself is needed: the
// measurement basis of the correlations and the velocity table of the
// look-up-table f-norm. The collision kernels never form it.
#pragma once

#include "flb_collide.cuh"

namespace flb {

__device__ __forceinline__ void hermite_rows_fp64(double P[9][9]) {
    // row a of P = P^T applied to the unit vector e_a (D_1 = -K1, D_2 = -K2)
    for (int a = 0; a < 9; ++a) {
        double Dn[6];
        for (int b = 0; b < 6; ++b) Dn[b] = (a == 3 + b) ? 1.0 : 0.0;
        double h[9];
        hermite_back<double, true>(a == 0 ? 1.0 : 0.0, a == 1 ? -1.0 : 0.0, a == 2 ? -1.0 : 0.0,
                                   Dn, h);
        for (int i = 0; i < 9; ++i) P[a][i] = h[i];
    }
}

__device__ __forceinline__ void feq_unit_fp64(double ux, double uy, double W[9]) {
    const double usq = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        const double uv = ux * cvx(i) + uy * cvy(i);
        const double wi = i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
        W[i] = wi * (1.0 + 3.0 * uv + 4.5 * uv * uv - 1.5 * usq);
    }
}

// m~ rows (out[a * 9 + i]) at u; false (and NaN rows) if some W_i <= 0.
__device__ __forceinline__ bool fnorm_basis_fp64(double ux, double uy, double out[81]) {
    double P[9][9], W[9];
    hermite_rows_fp64(P);
    feq_unit_fp64(ux, uy, W);
    bool ok = true;
    for (int i = 0; i < 9; ++i) ok = ok && W[i] > 0.0;
    double L[9][9];
    for (int a = 0; a < 9; ++a)
        for (int b = 0; b < 9; ++b) {
            double s = 0.0;
            for (int i = 0; i < 9; ++i) s += P[a][i] * W[i] * P[b][i];
            L[a][b] = s;
        }
    for (int j = 0; j < 9; ++j) {
        double d = L[j][j];
        for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
        d = sqrt(d);
        L[j][j] = d;
        for (int i = j + 1; i < 9; ++i) {
            double s = L[i][j];
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            L[i][j] = s / d;
        }
    }
    for (int i = 0; i < 9; ++i)          // forward substitution per column of P
        for (int a = 0; a < 9; ++a) {
            double s = P[a][i];
            for (int k = 0; k < a; ++k) s -= L[a][k] * out[k * 9 + i];
            out[a * 9 + i] = s / L[a][a];
        }
    return ok;
}

}  // namespace flb
