// flb_host.h -- host-side helpers shared by the C-ABI translation units:
// parameter validation, the reference equilibrium, the collision constants,
// grid sizing of the plain element-wise kernels and error-code mapping.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "../../include/flb.h"
#include "flb_device.cuh"
#include "flb_kernels.cuh"

namespace flb {

// f_i^0(rho, u) of Eq. d2q9f0.
inline void feq_host(double rho, double ux, double uy, double f[9]) {
    const double usq = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        const double uv = ux * cvx(i) + uy * cvy(i);
        const double wi = i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
        f[i] = rho * wi * (1.0 + 3.0 * uv + 4.5 * uv * uv - 1.5 * usq);
    }
}

// 1 if p describes a lattice flb_create accepts.
inline int valid_params(const flb_params* p) {
    if (!p) return 0;
    if (p->Lx < 1 || p->Ly < 1) return 0;
    if ((long long)p->Lx * p->Ly >= (1LL << 31)) return 0;
    if (!(p->rho0 > 0) || !std::isfinite(p->rho0)) return 0;
    if (!(p->kT >= 0) || !std::isfinite(p->kT)) return 0;
    if (!std::isfinite(p->ux0) || !std::isfinite(p->uy0)) return 0;
    for (int a = 3; a < 9; ++a)
        if (!(p->omega[a] > 0 && p->omega[a] < 2)) return 0;
    if (p->basis != FLB_BASIS_STANDARD && p->basis != FLB_BASIS_LOCAL &&
        p->basis != FLB_BASIS_LOCAL_LUT)
        return 0;
    if (p->precision != FLB_FP64 && p->precision != FLB_FP32 && p->precision != FLB_FP16_DEV)
        return 0;
    if (p->precision == FLB_FP16_DEV && !(p->kT > 0)) return 0;   // the store scale is sqrt(kT)
    if (p->reserved != 0) return 0;
    // the mean velocity must leave every f_i^0(1,u0) > 0 (Fig. 11)
    const double usq = p->ux0 * p->ux0 + p->uy0 * p->uy0;
    for (int i = 0; i < 9; ++i) {
        const double uv = p->ux0 * cvx(i) + p->uy0 * cvy(i);
        if (!(1.0 + 3.0 * uv + 4.5 * uv * uv - 1.5 * usq > 0.0)) return 0;
    }
    return 1;
}

// -omega_a and the noise amplitudes sqrt(kT omega_a (2 - omega_a)), a = 3..8.
template <class T>
CollideConst<T> collide_const(const flb_params* p) {
    CollideConst<T> cc;
    for (int a = 0; a < 6; ++a) {
        const double om = p->omega[3 + a];
        cc.nomega[a] = (T)(-om);
        const double v = p->kT * om * (2.0 - om);
        cc.amp[a] = (T)(v > 0 ? std::sqrt(v) : 0.0);
    }
    cc.key = make_noise_key(p->seed, p->replica);
    return cc;
}

// Scale s of the tensor-core correlation sums (the nodes are staged as
// (f - f^0(rho0, u0)) / s in FP16): s = sqrt(kT rho0) makes the thermal
// fluctuations of order one. Used only where a deviation as large as a few
// rho0 stays far inside FP16's range (|d| / s <= 4 sqrt(rho0 / kT) <= 16000);
// otherwise, and at kT = 0, the sums are taken with FP32 products.
inline bool tensor_sampling_ok(const flb_params* p) {
    return p->kT > 0 && std::sqrt(p->rho0 / p->kT) <= 4000.0;
}
inline double gram_scale(const flb_params* p) { return std::sqrt(p->kT * p->rho0); }

inline int grid_for(long long n) {
    long long b = (n + 255) / 256;
    if (b > 4096) b = 4096;
    return (int)(b < 1 ? 1 : b);
}

inline int map_status(int code) {
    if (code == kStatusInvalidVelocity) return FLB_ERR_INVALID_VELOCITY;
    if (code == kStatusNonfinite) return FLB_ERR_NONFINITE;
    if (code == kStatusTimeout) return FLB_ERR_TIMEOUT;
    return code ? FLB_ERR_STATE : FLB_OK;
}

}  // namespace flb
