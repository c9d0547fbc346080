/*
 * flb_oracle.h -- plain FP64 CPU oracle of the fluctuating D2Q9 lattice-Boltzmann
 * method of Kaehler & Wagner, "A fluctuating lattice-Boltzmann method with
 * improved Galilean invariance" (arXiv:1204.6734).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load this library. The product (the CUDA library under
 * paper_1204_6734_gb300/) never includes, links or calls it, and this oracle
 * shares no code, header, table or constant with it.
 *
 * Everything here is double precision and written for clarity, not speed: the
 * equations are evaluated in the paper's order and notation, one node at a time.
 *
 * Conventions (shared by contract, not by code, with the CUDA path):
 *  - velocities v_i, i = 0..8, in the order read off the j_x, j_y rows of the
 *    printed Hermite matrix (Eq. d2q93a): 0 rest, 1 (+x), 2 (+y), 3 (-x), 4 (-y),
 *    5 (+x+y), 6 (-x+y), 7 (-x-y), 8 (+x-y);
 *  - populations in SoA layout f[i][y][x] (index i*Lx*Ly + y*Lx + x);
 *  - the state is the pre-collision (post-streaming) f_i(x, t) of Eq. LBE1;
 *  - node index n = x + Lx*y, time step t counts collisions performed;
 *  - noise: Philox4x32-10 block with counter (n, t, replica, 0) and key
 *    (seed low word, seed high word) -> six 21-bit fields -> three Box-Muller
 *    pairs -> standard normals N^a for a = 3..8 in order.
 */
#ifndef FLB_ORACLE_H
#define FLB_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BASIS_STANDARD = 0, ORC_BASIS_LOCAL = 1, ORC_BASIS_LOCAL_LUT = 2 };

enum {
    ORC_OK = 0,
    ORC_ERR_ARG = -1,
    ORC_ERR_INVALID_VELOCITY = -3, /* some f_i^0(1,u) <= 0: the f-norm has no basis */
    ORC_ERR_NONFINITE = -4
};

typedef struct {
    int32_t Lx, Ly;
    double rho0, ux0, uy0, kT;
    double omega[9];   /* relaxation rate 1/tau^a per moment; 0..2 are ignored */
    int32_t basis;     /* ORC_BASIS_STANDARD (Hermite norm), ORC_BASIS_LOCAL (f-norm) or
                          ORC_BASIS_LOCAL_LUT (f-norm from the velocity table) */
    uint32_t replica;  /* third Philox counter word */
    uint64_t seed;     /* Philox key */
} orc_params;

/* Tables of the appendix: velocities, weights (Eq. d2q9w), forward m[a][i]
 * (Eq. d2q93a) and back n[i][a] (Eq. d2q93b) Hermite matrices as printed. */
void orc_tables(int vx[9], int vy[9], double w[9], double m[81], double n[81]);

/* Eq. d2q9f0: Qian's second-order equilibrium with theta = 1/3. */
void orc_feq(double rho, double ux, double uy, double f0[9]);

/* Eq. d2q94: Hermite equilibrium moments M^{a,0}. */
void orc_hermite_meq(double rho, double ux, double uy, double meq[9]);

/* Section 4: f-norm basis mt[a][i] by Gram-Schmidt (Eqs. gramschmidt, gsortho,
 * normalised by the square root) under the scalar product sum_i a_i W_i b_i,
 * W_i = f_i^0(1, u). Returns ORC_ERR_INVALID_VELOCITY if some W_i <= 0. */
int orc_local_basis(double ux, double uy, double mt[81]);

/* Section 4, look-up-table variant: the table velocity u_g = ((k_x - 25)/50,
 * (k_y - 25)/50) nearest to u, k = floor(50 u + 25.5) in 0..50; returns
 * ORC_ERR_INVALID_VELOCITY off the table. */
int orc_lut_velocity(double ux, double uy, double* ugx, double* ugy);

/* Salmon et al. (SC'11) Philox4x32 with 10 rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* The six 21-bit integer fields of one node-step block and the six standard
 * normals built from them (Box & Muller 1958). */
void orc_draw_fields(uint64_t seed, uint32_t replica, uint32_t node, uint32_t step,
                     uint32_t fields[6]);
void orc_normals(uint64_t seed, uint32_t replica, uint32_t node, uint32_t step,
                 double nrm[6]);

/* One collision (Eq. LBEMRT) of the pre-collision populations g at one node.
 * Writes the post-collision populations fstar. */
int orc_collide_node(const orc_params* p, const double g[9], uint32_t node,
                     uint32_t step, double fstar[9]);

/* Uniform initial state f_i = f_i^0(rho0, u0) at every node. */
void orc_init_equilibrium(const orc_params* p, double* f);

/* Advance the state f (pre-collision, SoA) by nsteps updates of Eq. LBE1,
 * starting at time step0: for each t, collide every node then push-stream.
 * Before the collision of step t, when t >= warmup and (t - warmup) % every == 0
 * (every > 0), the pre-collision state is sampled:
 *   S1[i] += sum_x (f_i - c_i),  S2[i*9+j] += sum_x (f_i - c_i)(f_j - c_j),
 * c = f^0(rho0, u0), nsamp += Lx*Ly. S1/S2/nsamp may be NULL when every <= 0.
 * Returns 0 or the first error; on error the node and step are written to
 * *err_node / *err_step when those pointers are non-NULL. */
int orc_run(const orc_params* p, double* f, int64_t step0, int64_t nsteps,
            int64_t warmup, int64_t every, double* S1, double* S2, int64_t* nsamp,
            int64_t* err_node, int64_t* err_step);

#ifdef __cplusplus
}
#endif
#endif
