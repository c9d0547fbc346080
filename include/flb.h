/*
 * flb.h -- C ABI of the GB300 (sm_103a) fluctuating D2Q9 lattice-Boltzmann library.
 *
 * The library implements the fused stream-collide-noise step of Kaehler & Wagner,
 * "A fluctuating lattice-Boltzmann method with improved Galilean invariance"
 * (arXiv:1204.6734), with either the standard Hermite-norm moment basis
 * (Section 2, Eqs. fluctf5, d2q93a, d2q93b, d2q94) or the paper's f-norm basis
 * orthogonalised at every node against the local equilibrium (Section 4,
 * Eqs. fnorm, gramschmidt, gsortho, Mtilde, fnormmeq), plus the reduction of the
 * equal-time correlations <df_i df_j> and <dM^a dM^b> (Eqs. dfdef, efif0,
 * dfidfj2dmadmb).
 *
 * Conventions used by every entry point:
 *  - Return value: FLB_OK (0) or a negative FLB_ERR_* code. No entry point
 *    aborts, traps or prints. flb_error_string() names a code.
 *  - Velocities i = 0..8: 0 rest, 1 (+x), 2 (+y), 3 (-x), 4 (-y), 5 (+x+y),
 *    6 (-x+y), 7 (-x-y), 8 (+x-y) -- the order the j_x, j_y rows of Eq. d2q93a
 *    imply. Moments a = 0..8: rho, j_x, j_y, Pi_xx-yy, Pi_xy, Pi_xx+yy, q_x,
 *    q_y, epsilon (Eq. d2q93a).
 *  - Host population arrays are double, SoA, f[i][y][x] at index
 *    i*Lx*Ly + y*Lx + x, and hold the pre-collision (post-streaming) state
 *    f_i(x, t) of Eq. LBE1.
 *  - Noise: Philox4x32-10 (Salmon et al., SC'11) with counter
 *    (node = x + Lx*y, step t, replica, 0) and key (seed low, seed high);
 *    the 128 output bits give six 21-bit fields, three Box-Muller pairs, and
 *    the normals N^a of a = 3..8 in order. The variance scale is k_B T:
 *    xi^a = sqrt(kT rho omega_a (2 - omega_a)) (Eq. noiseamp with 1/tau = omega),
 *    rho the density of the colliding node.
 *  - Ownership: the caller owns every host pointer passed in; the library copies
 *    what it needs before returning. A lattice handle owns its device memory
 *    unless the caller passed a device workspace to flb_create.
 *  - Streams: all device work of a handle is ordered on the stream given to
 *    flb_create (NULL = the legacy default stream). Calls on one handle must
 *    not be made concurrently from several host threads.
 *  - Errors found on the device (a node whose velocity leaves the region where
 *    every f_i^0(1,u) > 0, Fig. 11; a non-finite density) are recorded by the
 *    kernel, which leaves that node uncollided; they are reported by the next
 *    flb_sync / flb_get_populations / flb_correlations / flb_conservation and
 *    make the handle refuse further steps until flb_set_populations or
 *    flb_reset_error.
 */
#ifndef FLB_H
#define FLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FLB_OK 0
#define FLB_ERR_ARG (-1)              /* invalid argument or parameter */
#define FLB_ERR_OOM (-2)              /* device allocation failed or workspace too small */
#define FLB_ERR_INVALID_VELOCITY (-3) /* some f_i^0(1,u) <= 0 at a node (Fig. 11) */
#define FLB_ERR_NONFINITE (-4)        /* non-finite or non-positive density at a node */
#define FLB_ERR_TIMEOUT (-5)          /* a bounded device wait gave up */
#define FLB_ERR_CUDA (-6)             /* a CUDA runtime call failed */
#define FLB_ERR_STATE (-7)            /* call not valid in the handle's state (e.g. no samples) */

/* Bases of the collision: the Hermite norm of the appendix (fixed weights
 * w_i), the f-norm of Section 4 (weights f_i^0(1, u) at the node's own u,
 * orthogonalised per node), and the f-norm from the paper's 51 x 51 velocity
 * table (Section 4: the basis at the nearest table velocity u_g, spacing
 * 0.02, |u_g| <= 0.5; equilibrium moments projected onto it exactly; velocity
 * off the table or at a table point where some f_i^0(1, u_g) <= 0 is
 * FLB_ERR_INVALID_VELOCITY). Every precision takes every basis; batches and
 * the server (FP32) take all three. */
typedef enum { FLB_BASIS_STANDARD = 0, FLB_BASIS_LOCAL = 1, FLB_BASIS_LOCAL_LUT = 2 } flb_basis;
typedef enum { FLB_FP64 = 0, FLB_FP32 = 1, FLB_FP16_DEV = 2 } flb_precision;

/* Parameters of one periodic lattice. */
typedef struct {
    int32_t Lx, Ly;      /* lattice sides, 1 <= Lx, Ly and Lx*Ly < 2^31 */
    double rho0;         /* mean density (> 0); initial state f^0(rho0, u0) */
    double ux0, uy0;     /* mean velocity u0; f_i^0(1,u0) > 0 for all i required */
    double kT;           /* k_B T, the variance scale of the noise (>= 0) */
    double omega[9];     /* relaxation rate 1/tau^a of moment a; entries 0..2
                            (conserved) are ignored, 3..8 must lie in (0, 2) */
    int32_t basis;       /* flb_basis */
    int32_t precision;   /* flb_precision: FP64 and FP32 store and compute in
                            that type; FP16_DEV stores h_i = (f_i - f_i^0(rho0,
                            u0)) / sqrt(kT) in FP16 (kT > 0 required) and
                            computes in FP32 */
    uint64_t seed;       /* Philox key */
    uint32_t replica;    /* third Philox counter word */
    uint32_t reserved;   /* must be 0 */
} flb_params;

typedef struct flb_lattice_s* flb_lattice;

/* Device bytes a lattice with these parameters needs (populations, two
 * buffers, plus reduction scratch); 0 if the parameters are invalid. */
size_t flb_workspace_bytes(const flb_params* p);

/* Create a lattice on the current CUDA device, initialised to the uniform
 * equilibrium f_i = f_i^0(rho0, u0) (Eq. d2q9f0) at time t = 0.
 *  dev_workspace: NULL to let the library allocate, or a device pointer to at
 *                 least flb_workspace_bytes(p) bytes, 256-byte aligned, that the
 *                 caller keeps alive until flb_destroy.
 *  stream:        a cudaStream_t (as void*), or NULL for the default stream.
 * Errors: FLB_ERR_ARG (parameters), FLB_ERR_OOM, FLB_ERR_CUDA. */
int flb_create(const flb_params* p, void* dev_workspace, size_t workspace_bytes,
               void* stream, flb_lattice* out);

/* Release the lattice and, if the library allocated it, its device memory.
 * Waits for the handle's stream. NULL is accepted. */
int flb_destroy(flb_lattice h);

/* Sample the pre-collision state of every step t with t >= warmup and
 * (t - warmup) % every == 0 into the equal-time correlation sums (every = 0
 * switches sampling off). Also clears the sums. */
int flb_set_sampling(flb_lattice h, int64_t warmup, int64_t every);

/* Clear the correlation sums and the sample count. */
int flb_reset_statistics(flb_lattice h);

/* Enqueue n time steps of Eq. LBE1 (pull streaming, collision with noise) on
 * the handle's stream; returns without waiting. Errors: FLB_ERR_ARG (n < 0),
 * a recorded device error (sticky), FLB_ERR_CUDA. */
int flb_step(flb_lattice h, int64_t n);

/* Wait for the handle's stream and report any device error recorded so far. */
int flb_sync(flb_lattice h);

/* Current time step t (number of collisions performed). */
int flb_time(flb_lattice h, int64_t* t);

/* Checkpoint and resume. A run continues exactly (the same noise draws, the
 * same sampling schedule, the same sums up to FP64 rounding order) from its
 * state f_i(x, t) (flb_get_populations), its time t (flb_time) and its raw
 * sums (flb_raw_sums): on a new handle with the same parameters call
 * flb_set_sampling (which clears the sums), then flb_set_raw_sums,
 * flb_set_time and flb_set_populations. flb_set_time sets t, the step
 * counter of the noise (0 <= t < 2^32); flb_set_raw_sums sets S1[9],
 * S2[81] (the entries i <= j are used) and the node-sample count.
 * Errors: FLB_ERR_ARG, FLB_ERR_CUDA. Structure-factor sums are not covered. */
int flb_set_time(flb_lattice h, int64_t t);
int flb_set_raw_sums(flb_lattice h, const double* S1, const double* S2, int64_t n_samples);

/* Node and step of the first recorded device error (-1, -1 if none). */
int flb_error_location(flb_lattice h, int64_t* node, int64_t* step);

/* Forget a recorded device error (the state is left as it is). */
int flb_reset_error(flb_lattice h);

/* Equal-time correlations of the sampled pre-collision populations (the step
 * kernels accumulate FP64 sums; they are finalised on the device):
 *  Cff[81]   <df_i df_j> = centred covariance of f_i over nodes and samples
 *            (Eqs. dfdef, efif0; the mean is the sample mean);
 *  CMM[81]   <dM^a dM^b> = sum_ij m^a_i m^b_j <df_i df_j> (Eq. dfidfj2dmadmb),
 *            m = the Hermite rows (measure_basis = FLB_BASIS_STANDARD) or the
 *            f-norm basis at the mean velocity u0 (FLB_BASIS_LOCAL, the choice
 *            made after Eq. fidjx); orthonormal under w resp. f^0(1,u0), so the
 *            ideal gas gives CMM = kT rho0 I;
 *  mean_dev[9]  mean of f_i - f_i^0(rho0, u0);
 *  n_samples    number of node samples (nodes x sampled steps).
 * Any output pointer may be NULL. Errors: FLB_ERR_STATE when nothing was
 * sampled, device errors. Synchronises the handle's stream. */
int flb_correlations(flb_lattice h, int32_t measure_basis, double* Cff, double* CMM,
                     double* mean_dev, int64_t* n_samples);

/* Raw FP64 sums S1[i] = sum (f_i - c_i), S2[i*9+j] = sum (f_i - c_i)(f_j - c_j),
 * c = f^0(rho0, u0), over all samples. Any pointer may be NULL. */
int flb_raw_sums(flb_lattice h, double* S1, double* S2, int64_t* n_samples);

/* Total mass and momentum of the current state, sum_x (rho, j_x, j_y), reduced
 * in FP64 on the device. Synchronises. */
int flb_conservation(flb_lattice h, double sums[3]);

/* Copy the current pre-collision state f_i(x, t) to host memory
 * (9*Lx*Ly doubles, layout above). Page-locked host memory (cudaHostAlloc,
 * cudaHostRegister) is written by the device directly, in one pass; other
 * host memory through a device staging buffer of the same size (FLB_ERR_OOM
 * if it cannot be allocated). Synchronises. */
int flb_get_populations(flb_lattice h, double* host_out);

/* Replace the current pre-collision state f_i(x, t) by host data (9*Lx*Ly
 * doubles, layout above; converted to the handle's precision). Page-locked
 * host memory is read by the device directly; other memory through a device
 * staging buffer. Clears a recorded device error. Synchronises. */
int flb_set_populations(flb_lattice h, const double* host_in);

/* Difference of the current pre-collision states of two lattices of the same
 * size, in any precisions, computed on the device: out[0] = max |f_a - f_b|,
 * out[1] = root mean square of f_a - f_b over all 9 Lx Ly values, out[2] =
 * max |f_b|. No counterpart in the paper: it serves the precision study.
 * Synchronises both handles' streams. Errors: FLB_ERR_ARG (sizes differ). */
int flb_state_difference(flb_lattice a, flb_lattice b, double out[3]);

/* Static structure factors (Eqs. sfactorr, sfactoru, rcorrelator).
 * flb_set_structure_sampling samples the pre-collision state of every step t
 * with t >= warmup and (t - warmup) % every == 0 (every = 0: off) and clears
 * the sums. On a sampling step, before the step's collision, the device forms
 * delta rho(x) = rho(x) - rho0, delta j(x) = j(x) - rho0 u0, transforms them,
 * a(k) = sum_x a(x) exp(-i k.x) with k = 2 pi (m_x / Lx, m_y / Ly), and adds
 * |drho(k)|^2, |dj_x(k)|^2 and dj_x(k) conj(dj_y(k)) to FP64 sums. The
 * transform runs in FP64 for FP64 lattices, in FP32 otherwise: FFTs (Stockham
 * passes in shared memory) for power-of-two sides, a direct O(L^2) transform
 * per row or column for other sides; when both sides are powers of two up to
 * 4096, two launches per sample and sums over half the k plane (the other
 * half follows from S(-k) = S(k), R(-k) = conj R(k)); an FP32 lattice on the
 * pipelined kernel then has the step kernel itself write the three fields of
 * the state it starts from (the same FP32 values), and the two launches
 * transform them. The first call with every > 0 allocates the library's own
 * device buffers (at most 3 complex and 4 double arrays of Lx*Ly values; FP32
 * power-of-two lattices also 4 float arrays of partial sums and 3 float field
 * arrays), freed by flb_destroy. Errors: FLB_ERR_ARG (negative arguments; a
 * side above 20480 in FP32 or 10240 in FP64), FLB_ERR_OOM, a recorded device
 * error (sticky). */
int flb_set_structure_sampling(flb_lattice h, int64_t warmup, int64_t every);

/* The sampled factors, each an Ly x Lx array indexed [m_y][m_x] (host memory,
 * caller-owned): S_rho = <|drho(k)|^2> / rho0, S_jx = <|dj_x(k)|^2> / rho0 and
 * R = <dj_x(k) conj(dj_y(k))> / rho0 = R_re + i R_im, averages over the
 * samples. At rest (u0 = 0) every k != 0 mode of S_rho approaches Lx Ly kT
 * and of S_jx Lx Ly kT / 3, the per-site variances kT rho0 and kT rho0 / 3 of
 * the fluctuating equilibrium; R approaches 0. Any array pointer may be NULL;
 * *n_samples (may be NULL) receives the number of samples. Synchronises.
 * Errors: FLB_ERR_STATE when an array is asked for and nothing was sampled,
 * FLB_ERR_OOM, FLB_ERR_CUDA. */
int flb_structure_factors(flb_lattice h, double* S_rho, double* S_jx, double* R_re, double* R_im,
                          int64_t* n_samples);

/* Whole-job entry point with host buffers: create a lattice, upload the
 * initial state (or start from equilibrium when f_in is NULL), run nsteps
 * with sampling (warmup, every), and copy back the final state (f_out may be
 * NULL) and the correlation sums (S1[9], S2[81], n_samples; may be NULL).
 * Host-device copies are part of the call. */
int flb_run_host(const flb_params* p, const double* f_in, int64_t nsteps, int64_t warmup,
                 int64_t every, double* f_out, double* S1, double* S2, int64_t* n_samples);

/* Failure detection, for testing: every wait of the pipelined kernels is
 * bounded (about 2 s), after which the kernel records a timeout that the next
 * flb_sync reports as FLB_ERR_TIMEOUT, and exits. Here one warp waits on a
 * barrier that nothing completes, for limit_cycles (0 .. 4e9) SM cycles, on
 * the legacy default stream: the call returns FLB_ERR_TIMEOUT without a
 * fault or a hang, and the context stays usable. Synchronous. */
int flb_wait_probe(int64_t limit_cycles);

/* Noise draws of the device code, for testing: for each of n nodes, the six
 * 21-bit Philox fields and the six standard normals N^3..N^8 the step kernel
 * of the given precision (FLB_FP64 or FLB_FP32) uses at (seed, replica, node,
 * step). nodes, fields (6n) and normals (6n) are host arrays. Synchronous. */
int flb_noise_draws(uint64_t seed, uint32_t replica, uint32_t step, const uint32_t* nodes,
                    int32_t n, int32_t precision, uint32_t* fields, double* normals);

/* One collision (Eq. LBEMRT) of n independent nodes by the device code, for
 * testing: g (9n, node-major g[k*9+i]) in, fstar (9n) out, with node index
 * node_ids[k] and time step `step` for the noise. Computes in p->precision;
 * p->Lx, p->Ly are ignored. status[k] (may be NULL) receives 0 or an FLB_ERR_*
 * code per node. Synchronous. */
int flb_collide_nodes(const flb_params* p, const double* g, const uint32_t* node_ids,
                      uint32_t step, int32_t n, double* fstar, int32_t* status);

/* ---------------------------------------------------------------------------
 * Batches: many independent FP32 lattices ("replicas") of different sizes and
 * parameters, stepped together by one persistent launch per step of the
 * pipelined kernel (the tiles of all replicas in one table). Each replica has
 * its own state, noise stream (its seed and replica id), time, sampling
 * schedule and sums, and error record; its populations are those of a lattice
 * handle created with the same parameters and stepped as often, and its sums
 * equal the handle's up to the summation order. The paper runs one lattice at
 * a time and has no counterpart of batches: they exist to fill the GPU with
 * many small lattices.
 *
 * Replicas join and leave between steps: flb_batch_add takes a slot and pool
 * memory, flb_batch_remove gives them back. All replicas of a batch share the
 * basis given at open time. Population buffers come from one device pool
 * allocated at open time (its size is the batch's HBM budget); adding and
 * removing replicas never allocates device memory. Threading: one thread per
 * batch. All calls are asynchronous on the batch's stream unless noted.
 * ------------------------------------------------------------------------- */
typedef struct flb_batch_s* flb_batch;

/* Tile shapes of the batched kernel (flb_batch_set_tile, flb_batch_autotune):
 * 128 x 4 nodes, 2 nodes per thread (default);
 * 64 x 8 nodes, 2 nodes per thread (wastes less on narrow lattices);
 * 128 x 2 nodes, 1 node per thread;
 *   (these three: 8 colliding warps per CTA beside 4 sampler warps on
 *   sampling steps, FP32 products)
 * 128 x 6 and 64 x 12 nodes, 2 nodes per thread, 12 colliding warps that add
 *   their own nodes to the correlation sums on the tensor cores (deviations
 *   staged in FP16, as FLB_OPT_PIPELINE_SAMPLING 3 of a lattice): only when
 *   every replica has kT > 0 and sqrt(rho0 / kT) <= 4000 (FLB_ERR_ARG from
 *   flb_batch_set_tile otherwise, and from flb_batch_add of a replica that
 *   breaks it; flb_batch_autotune skips them and reports -1 for their time);
 * mixed: as 128 x 6, with each replica cut into columns of three tile kinds of
 *   768 nodes (128 x 6, 64 x 12, 32 x 24): 128-wide columns, then one 64- or
 *   32-wide column, or one of each, for the rest of the width, so that no
 *   column pads more than 31 nodes of a row (the tensor-core conditions above).
 * One CTA per SM. */
#define FLB_TILE_128x4 0
#define FLB_TILE_64x8 1
#define FLB_TILE_128x2 2
#define FLB_TILE_128x6 3
#define FLB_TILE_64x12 4
#define FLB_TILE_MIXED 5
#define FLB_TILE_COUNT 6

/* Open an empty batch for replicas in `basis` (flb_basis): at most
 * max_replicas (1 .. 16384) at a time, population buffers carved from one
 * device pool of pool_bytes. stream as for flb_create. Synchronous.
 * Errors: FLB_ERR_ARG, FLB_ERR_OOM (the pool cannot be allocated), FLB_ERR_CUDA. */
int flb_batch_open(int32_t basis, int32_t max_replicas, size_t pool_bytes, void* stream,
                   flb_batch* out);

/* Pool bytes one replica takes (its two FP32 buffers); 0 if p is not valid
 * for a batch (flb_create's rules, FP32, each side <= 8192). */
size_t flb_batch_replica_bytes(const flb_params* p);

/* Add a replica at its equilibrium f^0(rho0, u0) and time 0; it runs for
 * nsteps steps (0 = until removed) and then stays at time nsteps, skipped by
 * the kernel, until removed. Sampling is off until flb_batch_set_sampling.
 * *slot receives its index (the lowest free one). Errors: FLB_ERR_ARG
 * (parameters, basis differs from the batch's), FLB_ERR_OOM (no free slot or
 * no pool range large enough: retry after a removal), FLB_ERR_CUDA. */
int flb_batch_add(flb_batch b, const flb_params* p, int64_t nsteps, int32_t* slot);

/* Free a slot and its pool memory. Steps already enqueued still complete. */
int flb_batch_remove(flb_batch b, int32_t slot);

/* Convenience: open a batch sized for the n replicas p[0..n-1] (one basis)
 * and add them as slots 0..n-1 with no step limit. Synchronous. */
int flb_batch_create(const flb_params* p, int32_t n, void* stream, flb_batch* out);

/* Pool bytes flb_batch_create needs for these replicas; 0 if any is invalid. */
size_t flb_batch_workspace_bytes(const flb_params* p, int32_t n);

/* Waits for the stream, frees all device memory of the batch. */
int flb_batch_destroy(flb_batch b);

/* Sampling schedule of one slot (slot = -1: every slot), as flb_set_sampling
 * with times counted from the replica's time 0; clears its sums. */
int flb_batch_set_sampling(flb_batch b, int32_t slot, int64_t warmup, int64_t every);

/* Enqueue n steps of the batch (one launch each): every live replica below
 * its step limit advances by one time step per launch. With graphs on
 * (flb_batch_set_graph), whole chunks are replayed from a captured CUDA graph.
 * Errors: FLB_ERR_ARG, FLB_ERR_CUDA. Device errors surface in sync/status. */
int flb_batch_step(flb_batch b, int64_t n);

/* Capture chunks of `steps` launches into a CUDA graph, replayed by
 * flb_batch_step (0 = launch every step directly; at most 100000). The graph
 * stays valid across membership changes. Must not be called while the
 * batch's stream is being captured by the caller. */
int flb_batch_set_graph(flb_batch b, int32_t steps);

/* Tile shape (FLB_TILE_*), and the autotuner: runs trial_steps real steps of
 * the batch in every shape (plus 2 warm-up steps each), times them with CUDA
 * events, keeps the fastest and reports it in *tile (may be NULL) and the
 * milliseconds per step of each shape in ms_per_step[FLB_TILE_COUNT] (may be
 * NULL). The trial steps advance the replicas like any others. Synchronous. */
int flb_batch_set_tile(flb_batch b, int32_t tile);
int flb_batch_get_tile(flb_batch b, int32_t* tile);
int flb_batch_autotune(flb_batch b, int32_t trial_steps, int32_t* tile, double* ms_per_step);

/* Wait for the batch's stream; FLB_OK or the error of the lowest slot that
 * recorded one. flb_batch_status: the same for one slot. Synchronous. */
int flb_batch_sync(flb_batch b);
int flb_batch_status(flb_batch b, int32_t slot);

/* Steps enqueued on the batch so far, and the time of one replica. */
int flb_batch_time(flb_batch b, int64_t* step);
int flb_batch_replica_time(flb_batch b, int32_t slot, int64_t* t);

/* Live replicas, their tiles in the current shape, pool bytes in use and the
 * pool size (any pointer may be NULL). */
int flb_batch_info(flb_batch b, int32_t* replicas, int64_t* tiles, size_t* pool_used,
                   size_t* pool_size);

/* Per-replica results and state, as their lattice-handle counterparts
 * (flb_raw_sums, flb_get_populations, flb_set_populations: 9 * Lx * Ly
 * doubles of that slot's lattice). Synchronous. */
int flb_batch_raw_sums(flb_batch b, int32_t slot, double* S1, double* S2, int64_t* n_samples);

/* Equal-time correlations pooled over the n replicas slots[0..n-1] (e.g. the
 * same parameters with different seeds): their FP64 sums and sample counts
 * are added, then finalised as flb_correlations does (Eqs. dfdef, efif0,
 * dfidfj2dmadmb), the measurement basis at their common u0. The replicas
 * must share rho0 and u0, since each one's sums are taken relative to
 * f^0(rho0, u0). Synchronous. Errors: FLB_ERR_ARG (bad slot, rho0 or u0
 * differ, measure_basis), FLB_ERR_STATE (no samples), a replica's recorded
 * device error, FLB_ERR_OOM, FLB_ERR_CUDA. */
int flb_batch_correlations(flb_batch b, int32_t n, const int32_t* slots, int32_t measure_basis,
                           double* Cff, double* CMM, double* mean_dev, int64_t* n_samples);
int flb_batch_get_populations(flb_batch b, int32_t slot, double* host_out);
int flb_batch_set_populations(flb_batch b, int32_t slot, const double* host_in);

/* ---------------------------------------------------------------------------
 * Request server: continuous batching of simulation requests. A request is
 * one FP32 periodic lattice (flb_params), run for nsteps steps with the given
 * sampling schedule; its result is its correlation sums. Requests queue in
 * submission order and are admitted, in that order, as soon as a slot and a
 * range of the device pool (pool_bytes: the HBM budget) are free; admitted
 * requests run together and leave when done, while others wait or arrive.
 * The host enqueues work up to two chunks of `chunk_steps` steps ahead of the
 * GPU. Like batches, this has no counterpart in the paper.
 *
 * Modes: FLB_SERVE_BATCHED runs all admitted requests as one batch (one
 * launch per step, chunks replayed from a CUDA graph); FLB_SERVE_PER_LATTICE
 * gives each its own lattice handle (one launch per lattice and step), for
 * comparison. A request's result does not depend on the mode or on the other
 * requests, up to the summation order of its sums.
 * Threading: one thread per server. The stream is the server's.
 * ------------------------------------------------------------------------- */
typedef struct flb_server_s* flb_server;

#define FLB_SERVE_BATCHED 0
#define FLB_SERVE_PER_LATTICE 1

typedef struct {
    int64_t id;            /* from flb_server_submit */
    int32_t status;        /* FLB_OK or the request's device error */
    int32_t reserved;
    int64_t steps;         /* steps run */
    int64_t n_samples;     /* sampled node-steps */
    double S1[9];          /* sums as flb_raw_sums */
    double S2[81];
    double t_submit, t_admit, t_done;   /* seconds on the server clock */
} flb_result;

typedef struct {
    int64_t submitted, queued;
    int64_t running;         /* admitted and stepping */
    int64_t finishing;       /* at their last step, result not yet retired */
    int64_t completed, pending_results;
    int64_t chunks;          /* chunks retired */
    int64_t replica_steps;   /* request-steps in retired chunks */
    int64_t node_steps;      /* lattice-node updates in retired chunks */
    int64_t pool_used, pool_size;   /* bytes */
    double gpu_busy_s;       /* device time of retired chunks (CUDA events) */
    double clock_s;          /* server clock now: seconds since creation */
} flb_serve_stats;

/* Errors: FLB_ERR_ARG, FLB_ERR_OOM (pool or page-locked memory), FLB_ERR_CUDA.
 * max_slots: requests running at once (1 .. 16384). Synchronous. */
int flb_server_create(int32_t mode, int32_t basis, size_t pool_bytes, int32_t max_slots,
                      int32_t chunk_steps, void* stream, flb_server* out);
/* Waits for the stream; results not yet polled are dropped. */
int flb_server_destroy(flb_server s);

/* Queue a request (p: FP32, the server's basis; nsteps >= 1). *id receives
 * its id. FLB_ERR_OOM if it could never fit the pool. Returns at once. */
int flb_server_submit(flb_server s, const flb_params* p, int64_t nsteps, int64_t warmup,
                      int64_t every, int64_t* id);

/* Make progress: retire completed chunks, admit queued requests, enqueue
 * chunks; then copy up to max_results finished requests into results and
 * their count into *n_results. wait != 0: if no result is ready and work is
 * in flight, block until the oldest chunk completes first. */
int flb_server_poll(flb_server s, int32_t wait, int32_t max_results, flb_result* results,
                    int32_t* n_results);

int flb_server_stats(flb_server s, flb_serve_stats* out);

/* Tile shape of a batched server (FLB_TILE_*; default FLB_TILE_64x8).
 * FLB_ERR_STATE for a per-lattice server. */
int flb_server_set_tile(flb_server s, int32_t tile);

/* Tuning and testing options of a lattice handle.
 *  FLB_OPT_KERNEL: which step kernel runs -- FLB_KERNEL_AUTO (default: the
 *    pipelined TMA kernel for FP32, the generic kernel for FP64),
 *    FLB_KERNEL_GENERIC (one node per thread, plain loads) or
 *    FLB_KERNEL_PIPELINED (FP32 only). All give the same results up to rounding.
 *  FLB_OPT_PIPELINE_WARPS: colliding warps per CTA of the pipelined kernel
 *    (8, 12, 14 or 16; the tile is 128 x value/2 nodes) for every step. By
 *    default the f-norm bases use 16 on lattices of at least 8 such tiles
 *    per SM and 12 below that, the Hermite norm 12 on sampling steps and 8
 *    without sampling; with sampler warps, 8. 14 and 16 exist with the
 *    tensor-core sums and without sampling only (16 without a producer warp:
 *    the last warp to release a stage refills it); choosing sampling mode 1
 *    or 2 then falls back to 12. FP32 only.
 *  FLB_OPT_PIPELINE_SAMPLING: how the pipelined kernel accumulates the
 *    correlation sums on sampling steps -- 1: dedicated sampler warps read the
 *    staged tile (FP32 products; the default where 3 is not allowed); 2: the colliding warps accumulate their own nodes
 *    (FP32 products); 3 (default): the colliding warps stage their nodes'
 *    deviations (f - f^0(rho0, u0)) / sqrt(kT rho0) in FP16 and add them to a
 *    Gram matrix on the tensor cores, FP32 partials of at most 1024 products
 *    summed in FP64 (each sum within (2^-10 + 2^-14) sqrt(S2_ii S2_jj), resp.
 *    (2^-11 + 2^-14) sqrt(n S2_ii), of the exact one). 3 requires kT > 0 and
 *    sqrt(rho0 / kT) <= 4000 (every deviation a valid state holds stays far
 *    inside FP16's range).
 * Errors: FLB_ERR_ARG for an unknown option or value. */
#define FLB_OPT_KERNEL 0
#define FLB_OPT_PIPELINE_WARPS 1
#define FLB_OPT_PIPELINE_SAMPLING 2
#define FLB_KERNEL_AUTO 0
#define FLB_KERNEL_GENERIC 1
#define FLB_KERNEL_PIPELINED 2
int flb_set_option(flb_lattice h, int32_t option, int32_t value);

/* Slab decomposition of one periodic lattice along y (the step is local plus
 * streaming, Eq. LBE1, so a lattice of Lx x Ly_total nodes splits into slabs
 * of whole rows that exchange only the populations crossing their y
 * boundaries). flb_set_slab makes handle h (of Lx x Ly nodes) hold rows
 * y0 .. y0 + Ly - 1 of such a lattice: its noise counters and error locations
 * use the global node x + Lx (y0 + y), so a decomposed run draws exactly what
 * the whole lattice does, and its y boundaries are open to the caller's halo
 * exchange instead of periodic within the handle. Call it before the first
 * step; Lx Ly_total <= 2^32. A slab samples the correlations and the
 * conservation sums of its own nodes (the slabs' sums add up to the lattice's);
 * structure factors are not available on a slab. Errors: FLB_ERR_ARG.
 *
 * The exchange, after every step (the state from flb_create or
 * flb_set_populations needs none), for every slab:
 *   flb_halo_pack(h, lo, hi)   -- writes f*_i of the slab's row 0 for the
 *       populations moving down (i = 4, 7, 8) to the device buffer lo, and of
 *       its row Ly - 1 for those moving up (i = 2, 5, 6) to hi: each buffer 3
 *       rows of Lx values of the state's precision, flb_halo_bytes(h) bytes;
 *   the caller moves the slab below's hi and the slab above's lo (periodic in
 *       y) into this slab's receive buffers (a device copy, or a send and a
 *       receive between GPUs);
 *   flb_halo_unpack(h, lo, hi) -- lo (the slab below's hi) fills the ghost row
 *       the slab's row 0 pulls from, hi (the slab above's lo) the one its row
 *       Ly - 1 pulls from, with the lattice's periodicity in x.
 * Both are enqueued on the handle's stream; the buffers are the caller's
 * device memory. Errors: FLB_ERR_ARG (not a slab, null buffer), FLB_ERR_CUDA. */
int flb_set_slab(flb_lattice h, int32_t Ly_total, int32_t y0);
size_t flb_halo_bytes(flb_lattice h);
int flb_halo_pack(flb_lattice h, void* dev_lo, void* dev_hi);
int flb_halo_unpack(flb_lattice h, const void* dev_lo, const void* dev_hi);

/* The FP64 fused step with correlation sampling, for callers that cannot
 * allocate device memory. (The paper has no counterpart: this is an interface
 * for such callers.) Plugins whose host application owns every device
 * allocation through its own pool, and loops that plan their memory ahead and
 * cannot take the synchronisation of cudaMalloc, fall in this group. The entry
 * point calls no cudaMalloc, cudaFree or allocating library routine. It copies
 * its sums to the host and synchronises the stream before it returns, so it
 * cannot be recorded into a CUDA graph: a stream that is being captured is
 * refused with FLB_ERR_ARG before anything is queued on it.
 *  p        parameters, checked as flb_create checks them; precision must be
 *           FLB_FP64, basis FLB_BASIS_STANDARD or FLB_BASIS_LOCAL; Lx*Ly <= 262144 nodes
 *           (larger lattices are rejected with FLB_ERR_ARG: the scratch below
 *           holds the partial sums of at most 1024 blocks of 256 nodes).
 *  dev_f    device array of 9*Lx*Ly doubles: on entry the pre-collision state
 *           f_i(x, t0) in the layout f[i][y][x] above; on return f_i(x, t0+nsteps).
 *  dev_work device array of the same size, overwritten (the caller's second
 *           buffer; distinct from dev_f).
 *  t0       time of the state in dev_f (the noise counter of the first step).
 *  nsteps   number of steps; the pre-collision state of every one of them is
 *           sampled.
 *  host_S1, host_S2  (may be NULL) host arrays of 9 and 81 doubles receiving the
 *           sums of f_i - c_i and (f_i - c_i)(f_j - c_j), c = f^0(rho0, u0), over
 *           the nodes and steps of this call only (as flb_raw_sums).
 *  stream   cudaStream_t (as void*) or NULL; the call synchronises it.
 * Scratch: a fixed array of about 432 KB in this library's device memory, held
 * by every GPU that loads the library until the process exits. The first call
 * on a device looks up its address there (cudaGetSymbolAddress) with that
 * device current. Every call shares the array and clears
 * the sums it needs at its start; calls that overlap on the GPU (other streams,
 * other host threads) race on it and must not be issued.
 * Errors: FLB_ERR_ARG (bad parameters, buffers, sizes, or a capturing stream),
 * FLB_ERR_INVALID_VELOCITY / FLB_ERR_NONFINITE (a node left the valid region;
 * it was not collided), FLB_ERR_CUDA. */
int flb_step_noalloc(const flb_params* p, double* dev_f, double* dev_work, int64_t t0,
                     int64_t nsteps, double* host_S1, double* host_S2, void* stream);

const char* flb_error_string(int code);

/* Library version as major*10000 + minor*100 + patch. */
int flb_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FLB_H */
