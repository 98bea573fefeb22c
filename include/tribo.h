/*
 * tribo.h -- C ABI of the GB300 (sm_103a) library for the data-parallel hot
 * path of point-particle triboelectric charging in a turbulent channel
 * (Wilms & Grosshans, "Effect of Reynolds number on triboelectric particle
 * charging in turbulent channel flow").
 *
 * One coupled particle step (Sec. 2.2 and Sec. 2.3.1 of the paper):
 *   1. locate each particle's cell and deposit its charge to the cell
 *      (charge density = sum of charges in a cell / cell volume, Sec. 2.2);
 *   2. solve laplacian(phi) = -rho/eps with grounded walls (Sec. 2.2; second
 *      order finite volumes, Sec. 3.1): DFT in the periodic x, z directions,
 *      tridiagonal solve in the wall-normal y direction; E = -grad(phi);
 *   3. interpolate the gas velocity u and E trilinearly at each particle;
 *   4. integrate du_p/dt = f_ad + f_el (Eq. particle-motion) with
 *      Schiller-Naumann (or Stokes) drag and f_el = q E / m_p;
 *   5. hard-sphere wall impacts (wall-normal velocity flips, Sec. 2.2) with
 *      the condenser-model charge dq_w = dq_c + dq_t (Eqs. particle-wall-
 *      exchange, capacity-capacitor, charge-contact-area, charge-contact-
 *      area-alpha2, precharge-surface).
 *
 * Conventions
 *   - All functions return tribo_status (0 = OK); no exception crosses the ABI.
 *   - SI units throughout.
 *   - Arrays are C-contiguous.  Lattice arrays are indexed [k][jn][i][c]
 *     (z slowest, x fastest); cell arrays [k][j][i].
 *   - "real" means double when params.precision == TRIBO_FP64 and float when
 *     params.precision == TRIBO_MIXED.
 *   - Device pointers are CUDA device (or managed) pointers on the device that
 *     was current at tribo_init; host pointers are ordinary (preferably
 *     pinned) host memory.
 *   - Calls are stream-ordered on the context's stream unless stated
 *     otherwise; errors detected on the device set a sticky error word that
 *     the next synchronising call (tribo_sync, tribo_stats, any host-pointer
 *     call) reports as TRIBO_ERR_DEVICE.
 *   - Nothing falls back to the CPU.
 */
#ifndef TRIBO_H
#define TRIBO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t tribo_status;

#define TRIBO_OK              0
#define TRIBO_ERR_ARG         1  /* invalid argument (null pointer, size, layout) */
#define TRIBO_ERR_UNSUPPORTED 2  /* e.g. an FFT length that is not 2^a 3^b */
#define TRIBO_ERR_CUDA        3  /* CUDA runtime error (tribo_last_error has it) */
#define TRIBO_ERR_OOM         4  /* device allocation failed */
#define TRIBO_ERR_DEVICE      5  /* the device error word is set */
#define TRIBO_ERR_CAPACITY    6  /* more particles than the context was sized for */

/* bits of the device error word (tribo_error_bits) */
#define TRIBO_DEV_ESCAPED   0x1u /* a particle was still outside the contact planes after one reflection */
#define TRIBO_DEV_NONFINITE 0x2u /* a particle state became NaN or Inf */
#define TRIBO_DEV_OUTSIDE   0x4u /* a particle position was outside the channel before a step */
#define TRIBO_DEV_TIMEOUT   0x8u /* a bounded wait between the tasks of a persistent kernel ran out
                                    (the results of that call are not valid) */

#define TRIBO_FP64  0   /* everything in FP64 */
#define TRIBO_MIXED 1   /* FP32 particle state, interpolation, force math, FFT
                           and fields; FP64-class y-tridiagonal solve (FP64
                           factors, double-single sweeps); FP64 cell charge
                           sums, wall-impact charge, time of flight and
                           per-particle charges */

#define TRIBO_DRAG_STOKES           0
#define TRIBO_DRAG_SCHILLER_NAUMANN 1
#define TRIBO_DRAG_OFF              2

#define TRIBO_IMPACT_SPEED  0   /* |u_i| = full particle speed at impact */
#define TRIBO_IMPACT_NORMAL 1   /* |u_i| = wall-normal speed at impact */

typedef struct tribo_ctx tribo_ctx;

/* Channel grid (Sec. 3.1): periodic in x (length lx) and z (length lz), walls
 * at y = y_faces[0] = 0 and y = y_faces[ny].  x and z cells are uniform.
 * y_faces: HOST array of ny+1 strictly increasing faces, copied at init.
 * nx, nz must be 2^a 3^b with 4 <= n <= 1024; nx even; 2 <= ny <= 1024. */
typedef struct {
    int32_t nx, ny, nz;
    double lx, lz;
    const double* y_faces;
} tribo_grid;

/* Physical parameters (Table 1) and switches.
 * eps: gas permittivity in Poisson's equation and in C = eps A / h;
 * eps0: vacuum permittivity in T_w = eps_w eps0 phi_p;
 * U_c: particle-wall contact potential [V] (not given in the paper);
 * kappa_A: factor on the Hertz contact area (1 in the paper).
 * dq_t: 1 to include the pre-charge transfer dq_t = -(A_iw / (pi d^2)) q
 *       (Eq. precharge-surface read as contact-area fraction), 0 to omit it.
 * electrostatics: 1 to deposit, solve and apply q E / m each step, 0 for none.
 * sort_every: re-sort particles by cell every this many steps (0 = never);
 *       sorting permutes all particle arrays, including id.
 * coulomb: 1 to add the near field of the hybrid electrostatics (Sec. 2.2):
 *       Coulomb's law between particles that share a cell, on top of the mesh
 *       field (needs electrostatics = 1 and max_particles >= n; not available
 *       in tribo_adjoint or a batch).
 * collisions: 1 for 4-way coupling: hard-sphere particle-particle collisions
 *       (Sec. 2.2) of particles that share a cell at the end of a step, with
 *       the condenser-model charge exchange of the contact (Sec. 2.3.1); a
 *       pair collides when the spheres overlap, approach each other and each
 *       is the other's nearest such partner (needs max_particles >= n; not
 *       available in tribo_adjoint or a batch). */
typedef struct {
    double mu_p, E_p, phi_p, k_e, mu_w, E_w, eps_w, h, eps, eps0;
    double nu, rho, rho_p;
    double U_c, kappa_A;
    int32_t drag_law, impact_vel, dq_t, electrostatics, precision;
    int32_t sort_every;
    int32_t coulomb;
    int32_t collisions;
} tribo_params;

/* Gas velocity on the wall-extended lattice (Nz, Ny+2, Nx, 3) of "real":
 * node (k, jn, i) sits at x = (i + 1/2) dx, z = (k + 1/2) dz and
 * y = 0 (jn = 0), cell centre jn - 1 (1 <= jn <= ny), 2 delta (jn = ny + 1).
 * Copied into the context's own lattice (the caller keeps ownership). */
typedef struct {
    const void* u;
    int32_t on_host;          /* 1: u is a host pointer, 0: device pointer */
} tribo_fluid;

/* Particle ensemble, structure of arrays, caller-owned.  Borrowed for the
 * duration of a call (host pointers) or until the stream reaches the end of
 * the call's work (device pointers).
 *   x, y, z, vx, vy, vz, d : n "real"
 *   q, q_wall              : n double (charge; cumulative charge received in
 *                            wall impacts)
 *   n_imp                  : n uint32 cumulative wall-impact count
 *   id                     : n uint32, optional (NULL): permuted with the
 *                            particles when they are re-sorted
 *   cell                   : n uint32, optional (NULL) output: cell key
 *                            (k * ny + j) * nx + i of each final position
 *   site                   : n double, optional (NULL): the charging-site
 *                            density c/c0 in [0, 1] of the stochastic scaling
 *                            model (Sec. 2.3.2), updated by each wall impact
 *                            while the SSM is set (tribo_set_ssm) and
 *                            permuted with the particles by a sort; NULL
 *                            holds c/c0 = 1 */
typedef struct {
    int64_t n;
    void *x, *y, *z, *vx, *vy, *vz, *d;
    double* q;
    double* q_wall;
    uint32_t* n_imp;
    uint32_t* id;
    uint32_t* cell;
    int32_t on_host;          /* 1: all pointers are host pointers */
    double* site;
} tribo_particles;

/* Create a context on the current device.  stream: a cudaStream_t to order
 * all work on (NULL = the legacy default stream).  max_particles sizes the
 * context's staging and sort buffers.  On failure *out is NULL. */
tribo_status tribo_init(tribo_ctx** out, const tribo_grid* grid, const tribo_fluid* fluid,
                        const tribo_params* params, int64_t max_particles, void* stream);

/* Replace the gas-velocity lattice (e.g. a time-varying field). */
tribo_status tribo_set_fluid(tribo_ctx* ctx, const tribo_fluid* fluid);

/* Synthetic time-varying gas field, evaluated on the device at every step.
 * It stands in for the paper's DNS/LES gas field (Sec. 2.1), which is not
 * available; the paper has no counterpart for this recipe.  At lattice node
 * (x, y, z) and time t:
 *   u(x, t) = ubar(y) e_x + damp(y) sum_m amp_m cos(k_x,m (x - ubar(y) t)
 *                                                  + ky_m y + k_z,m z + phase_m)
 * with k_x,m = 2 pi nxi_m / lx and k_z,m = 2 pi nzi_m / lz: random Fourier
 * modes advected with the local mean velocity.  All arrays are HOST arrays,
 * copied by the call:
 *   nxi, nzi : n_modes int32 integer wavenumbers, |nxi| < nx/2, |nzi| < nz/2
 *   ky, phase: n_modes double [1/m], [rad]
 *   amp      : (n_modes, 3) double amplitude vectors [m/s]
 *   ubar, damp: ny+2 double at the lattice y nodes (wall nodes: ubar = damp = 0)
 * t0 is the field time of the particle state at the next tribo_step; each
 * step evaluates the field at the current time, then advances it by dt.
 * 1 <= n_modes <= 4096.  Passing NULL switches back to the frozen lattice. */
typedef struct {
    int32_t n_modes;
    const int32_t* nxi;
    const int32_t* nzi;
    const double* ky;
    const double* amp;
    const double* phase;
    const double* ubar;
    const double* damp;
    double t0;
} tribo_modes;

tribo_status tribo_set_modes(tribo_ctx* ctx, const tribo_modes* modes);

/* Evaluate the mode field of tribo_set_modes at time t.  u_out: device
 * (3, Nz, Ny+2, Nx) "real" planes u_x, u_y, u_z, or NULL to write the
 * context's own gas lattice.  TRIBO_ERR_ARG if no modes are set.
 * Asynchronous. */
tribo_status tribo_eval_modes(tribo_ctx* ctx, double t, void* u_out);

/* Stochastic scaling model (SSM) of wall-impact charging (Sec. 2.3.2), with
 * the reference impact of Sec. 3.1 (r0 = 2e-4 m, un0 = 0.925 m/s,
 * mu0 = -4.12e-15 C, sigma0 = 6.49e-15 C, gamma0 = -0.191,
 * dq0_min = -2.19e-14 C; c_sat = C_sat = 5e-4 C/m^2).  An impact gives
 * dq = mu_w - Y with mu_w = dq0_min (A/A0) chi_w and Y skew-normal with mean
 * (dq0_min - mu0)(A/A0) chi_i, deviation sigma0 sqrt((A/A0) chi_i) and
 * skewness -gamma0 / ((A/A0) chi_i) (clipped to [-0.99, 0.99]), where
 * A, A0 are the Hertz contact areas of the impact and of the reference
 * impact and chi_w = 1 - sgn(dq0_min) 4 q/(c_sat d^2),
 * chi_i = 1 + sgn(dq0_min - mu0) 4 q/(c_sat d^2), both clipped to [0, 1],
 * and N_i/N_0 carries the particle's charging-site density c/c0 (the
 * particles' site array; 1 where it is NULL).  Each impact then uses up the
 * fraction a = (A/(pi d^2)) chi_i (q/q_max) of the remaining sites,
 * c/c0 <- c/c0 (1 - a) clipped to [0, 1], with q the charge before the
 * impact and q_max = sgn(dq0_min) c_sat d^2/4 (the paper's sum over earlier
 * contacts, taken one contact at a time).  The random numbers are
 * Philox4x32-10 with counter (particle id, impact count before the impact,
 * 0, 0) and key (seed low word, seed high word): results do not depend on
 * the particle order.  Needs the particles' id arrays in tribo_step; not
 * available in tribo_adjoint or a batch.  ssm NULL: back to the condenser
 * model. */
typedef struct {
    double r0, un0, mu0, sigma0, gamma0, dq0_min, c_sat;
    uint64_t seed;
} tribo_ssm;

tribo_status tribo_set_ssm(tribo_ctx* ctx, const tribo_ssm* ssm);

/* Momentum source of the particles on the gas, F_s of the momentum equation
 * (Eq. ns, Sec. 2.1): the aerodynamic forces of the particles of a control
 * volume summed, per unit gas mass,
 *   F_s[c] = -(1 / (rho V_c)) sum_{p in c} m_p dv_p / dt,
 * where dv_p = (u - v) phi1 - a tau phi2 is the velocity change the drag
 * gives the particle over the step under the exponential integrator (u, the
 * electric acceleration a and tau frozen; phi1 = 1 - e^-s, phi2 = s - phi1,
 * s = dt / tau), and c is the particle's cell at the start of the step (where
 * u was gathered).  Wall and particle-particle impulses are not aerodynamic
 * and are not included; drag off gives zero.
 * F_s: device (3, Nz, Ny, Nx) "real" planes F_x, F_y, F_z in m/s^2 (cell
 * key (k Ny + j) Nx + i within a plane), aligned to the real type,
 * caller-owned and borrowed until replaced; NULL switches the source off.
 * Every tribo_step with nsteps >= 1 overwrites it with the mean of F_s over
 * its steps (stream-ordered; zero when there are no particles), so a gas
 * solver stepping once per call receives the source of that step.
 * tribo_adjoint and batches do not write it.  TRIBO_ERR_ARG for a misaligned
 * pointer. */
tribo_status tribo_set_momentum_source(tribo_ctx* ctx, void* F_s);

/* Replace the physical parameters and switches (precision must not change). */
tribo_status tribo_set_params(tribo_ctx* ctx, const tribo_params* params);

/* Advance the particles nsteps coupled steps of length dt [s].  Device
 * pointers: asynchronous on the context's stream.  Host pointers: copies in,
 * steps, copies out and synchronises before returning; every host array then
 * holds the new state.  A host call that does not re-sort (and has no pair
 * interactions) sends back the positions and velocities of all particles
 * and q, q_wall, n_imp only of those whose impact count changed: the others'
 * values are unchanged, and the caller's arrays already hold them. */
tribo_status tribo_step(tribo_ctx* ctx, tribo_particles* p, double dt, int32_t nsteps);

/* Bytes the host-pointer calls of this context have moved across the host
 * link since tribo_init: host to device and device to host (the sum of the
 * copies issued).  Either pointer may be NULL; TRIBO_ERR_ARG if ctx is NULL.
 * The paper has no counterpart: it measures the interface, not the method. */
tribo_status tribo_transfer_bytes(tribo_ctx* ctx, uint64_t* h2d, uint64_t* d2h);

/* Standalone Poisson solve and field (step 2 above).  rho: device
 * (Nz, Ny, Nx) double charge density [C/m^3].  phi: device (Nz, Ny, Nx)
 * double, may be NULL.  E: device (3, Nz, Ny+2, Nx) "real", the planes
 * E_x, E_y, E_z on the wall-extended lattice; the wall nodes hold E_x = E_z = 0
 * and the one-sided E_y.  rho, phi and E must be 16-byte aligned;
 * TRIBO_ERR_ARG otherwise.  In TRIBO_MIXED the transforms are FP32: the
 * first pass reads the FP64 rho and rounds each value as it transforms it.
 * Asynchronous. */
tribo_status tribo_poisson(tribo_ctx* ctx, const double* rho, double* phi, void* E);

/* Reverse-mode derivative of the mean particle charge after nsteps coupled
 * steps, J = (1/n) sum_p q_p(T) (the quantity behind the charging-rate
 * statistics of Sec. 4.1), with respect to the condenser model's contact
 * potential U_c and contact-area factor kappa_A (Sec. 2.3.1) and to each
 * particle's diameter d_p (which enters the drag and the mass of Sec. 2.2 and
 * the impact charge of Sec. 2.3.1).  It is the derivative of the discrete step
 * map with every discrete decision (cell, interpolation stencil, wall
 * contact) held at its forward value.
 *   p: DEVICE particle arrays (on_host = 0), n >= 1; they are advanced
 *      nsteps steps exactly as tribo_step would, except that they are never
 *      re-sorted (sort_every is ignored), and the statistics accumulate.
 *   ckpt_every >= 1: the forward pass stores the state every ckpt_every
 *      steps; the backward pass recomputes each segment from its stored
 *      state, keeping that segment's states (and field lattices) in a
 *      workspace the context owns and keeps for later calls.  The field
 *      lattice of every forward step is also kept when it fits in the budget
 *      of tribo_set_adjoint_memory; the recomputed segments then take it
 *      instead of solving again.
 *   J, dJ_dUc, dJ_dkappaA: HOST doubles, each may be NULL.
 *   dJ_dd: DEVICE array of n doubles (dJ/dd_p), may be NULL.
 * Synchronises; TRIBO_ERR_OOM if the workspace cannot be allocated. */
tribo_status tribo_adjoint(tribo_ctx* ctx, tribo_particles* p, double dt, int32_t nsteps, int32_t ckpt_every,
                           double* J, double* dJ_dUc, double* dJ_dkappaA, double* dJ_dd);

/* Device memory the adjoint may take for the field lattices of every forward
 * step (nsteps x 3 x Nz x (Ny+2) x Nx reals): max_bytes < 0 (the default)
 * half of the free device memory at the call, 0 never (each recomputed
 * segment solves its fields again), > 0 at most that many bytes.  The results
 * do not depend on it beyond rounding. */
tribo_status tribo_set_adjoint_memory(tribo_ctx* ctx, int64_t max_bytes);

/* Statistics since the last tribo_reset_stats (Sec. 4.1): sum of the current
 * particle charges of p (may be NULL: sum_q is then not written), total wall
 * impacts, total charge received from the walls, and the per-y-cell particle
 * counts summed over the steps (hist_y: host, ny doubles, may be NULL);
 * n_samples: number of steps summed.  Synchronises. */
tribo_status tribo_stats(tribo_ctx* ctx, const tribo_particles* p, double* sum_q,
                         uint64_t* n_impacts, double* sum_wall, double* hist_y,
                         int64_t* n_samples);
tribo_status tribo_reset_stats(tribo_ctx* ctx);

/* Wait for the context's stream; report the sticky device error word. */
tribo_status tribo_sync(tribo_ctx* ctx);
uint32_t     tribo_error_bits(const tribo_ctx* ctx);
tribo_status tribo_clear_error(tribo_ctx* ctx);

/* Testing aid for the bounded waits of the pipelined inverse transform (the
 * persistent launch whose tasks wait on one another): from the next solve on,
 * the consumer tasks of node plane `plane` wait for one producer task more than
 * exists, so each of their waits runs out after its iteration limit (about a
 * second), sets TRIBO_DEV_TIMEOUT in the device error word and returns; the
 * launch still ends and the context stays usable (tribo_clear_error), but that
 * solve's field is not valid.  plane = -1 (the default) clears it.  Grids
 * solved without the pipeline ignore it.  TRIBO_ERR_ARG for ctx NULL or
 * plane < -1. */
tribo_status tribo_test_pipeline_wait(tribo_ctx* ctx, int32_t plane);

/* Number of kernel launches the library issued since the context was made. */
int64_t      tribo_launch_count(const tribo_ctx* ctx);

/* Per-kernel timing with CUDA events recorded on the context's stream around
 * each launch.  tribo_timing_enable(ctx, 1) clears and starts the
 * accumulators, 0 stops them.  tribo_timing_read synchronises and returns,
 * for phases 0..nphases-1, the summed device time [ms] and the launch count
 * since the last enable (ms, counts: host arrays of nphases entries).
 * tribo_phase_name gives the phase's kernel name (NULL past the last). */
#define TRIBO_NPHASES 12
tribo_status tribo_timing_enable(tribo_ctx* ctx, int32_t on);
tribo_status tribo_timing_read(tribo_ctx* ctx, double* ms, int64_t* counts, int32_t nphases);
const char*  tribo_phase_name(int32_t phase);

/* The Poisson solve of tribo_poisson without a context and without any device
 * allocation, for callers that cannot allocate device memory while they run
 * (an embedding whose caching allocator already holds the device's memory, a
 * real-time loop that must not wait on or fail in an allocation, a plug-in
 * that is only handed pre-allocated buffers).  The paper has no counterpart;
 * it is an interface convenience.  rho, phi (may be NULL) and E have the
 * layouts and meaning of tribo_poisson; grid as for tribo_init; eps is the
 * gas permittivity; precision TRIBO_FP64 or TRIBO_MIXED selects the "real"
 * type of E; stream: a cudaStream_t (NULL = legacy default).  Asynchronous:
 * the grid tables are built on the device by the call's first kernel from
 * values passed by value, so the call copies nothing from host memory and
 * does not wait for earlier work on the stream.  All scratch lives in one
 * static device array of 32 MiB that the library reserves on every device it
 * is loaded on until the process exits.  Grids that need more, or more than
 * 256 cells in any direction, are rejected with TRIBO_ERR_CAPACITY
 * (tribo_last_error gives the sizes); the largest cubes that fit are 96^3 in
 * TRIBO_MIXED (27.9 MiB with phi) and 72^3 in TRIBO_FP64 (19.4 MiB with phi),
 * and e.g. 256 x 64 x 64 in TRIBO_MIXED fits without phi (28.6 MiB) but not
 * with it (32.8 MiB).  A grid whose transforms need more shared memory per
 * block than the device offers is rejected with TRIBO_ERR_UNSUPPORTED.  The
 * first call on a device looks up that array's address (so make it before any
 * stream capture).  Calls share the array: calls whose GPU work overlaps race. */
tribo_status tribo_poisson_noalloc(const tribo_grid* grid, double eps, int32_t precision,
                                   const double* rho, double* phi, void* E, void* stream);

/* Batched ensemble: many independent channels (each made by tribo_init with
 * its own grid, gas lattice, parameters and max_particles >= its particle
 * count) advanced together, as in the paper's sweeps over Re_tau and particle
 * size (Sec. 4).  Every step forks one branch per channel (cell sort when
 * due, Poisson solve and field) and joins in ONE persistent particle kernel
 * over all channels' particles; steps are captured into a CUDA graph and
 * replayed.  Mixed-precision channels that share a grid whose transform
 * lengths are compiled in solve together: each pass of their Poisson solves
 * is one launch over all of them.  The channels must share precision and device and use frozen
 * gas lattices (no tribo_set_modes).  While a batch exists, its channels must
 * not be stepped or solved (tribo_step, tribo_poisson, tribo_adjoint) on their
 * own concurrently with it: they share the channel's work arrays.  sort_every: re-sort each
 * channel's particles by cell every this many batch steps (0 = never).
 * stream: a cudaStream_t (NULL = legacy default) on which the batch joins. */
typedef struct tribo_batch tribo_batch;
tribo_status tribo_batch_create(tribo_batch** out, int32_t n_channels, tribo_ctx* const* channels,
                                int32_t sort_every, void* stream);

/* Time the candidate shapes of the particle kernel (threads per block,
 * particles per tile, blocks per SM) on scratch copies of the particles and
 * keep the fastest; choice (3 int32, may be NULL) receives it.  The particles
 * are not changed.  tribo_batch_step tunes on its first call if this was not
 * called.  particles: host array of n_channels pointers to ensembles of DEVICE
 * arrays; dt: host array of n_channels step lengths.  Synchronises. */
tribo_status tribo_batch_autotune(tribo_batch* b, tribo_particles* const* particles, const double* dt,
                                  int32_t* choice);

/* Advance every channel nsteps steps (channel i with dt[i]); arguments as for
 * tribo_batch_autotune.  Asynchronous on the batch's stream; statistics and
 * error words accumulate in each channel's context. */
tribo_status tribo_batch_step(tribo_batch* b, tribo_particles* const* particles, const double* dt, int32_t nsteps);

/* Wait for the batch's stream; report any channel's device error word. */
tribo_status tribo_batch_sync(tribo_batch* b);

/* Kernels the batch has executed (direct launches plus the kernels of each
 * graph replay). */
int64_t      tribo_batch_launch_count(const tribo_batch* b);

/* Time the batch's particle kernel (the step of Sec. 2.1-2.3 over all
 * channels): enable != 0 starts an empty record, 0 stops recording.  While it
 * is on, tribo_batch_step issues every step as direct launches (no graph
 * replay) and brackets each particle-kernel launch with CUDA events on the
 * batch's stream.  TRIBO_ERR_ARG for b NULL; TRIBO_ERR_CUDA if events cannot
 * be made. */
tribo_status tribo_batch_timing(tribo_batch* b, int32_t enable);

/* Wait for the timed launches and read the record: *total_ms, the summed
 * device time of the particle-kernel launches since tribo_batch_timing (or the
 * last read), and *launches, their number; the record restarts empty.
 * TRIBO_ERR_ARG for a NULL argument. */
tribo_status tribo_batch_kernel_time(tribo_batch* b, double* total_ms, int64_t* launches);
void         tribo_batch_destroy(tribo_batch* b);

const char*  tribo_strerror(tribo_status s);
const char*  tribo_last_error(void);      /* thread-local detail of the last failure */
void         tribo_destroy(tribo_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* TRIBO_H */
