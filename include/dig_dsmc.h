/*
 * dig_dsmc.h -- C ABI of the GB300 (sm_103a) DSMC / DIG hot-path library.
 *
 * The library runs the data-parallel hot path of the DIG method of
 * "Multiscale simulation of rarefied polyatomic gas flow via DIG method"
 * (arXiv 2501.10965): the DSMC time step of a polyatomic gas with continuous
 * rotational energy (Sec. 2.2), the cell sampling of Eq. (DSMC_macroscopic),
 * the higher-order terms of Eq. (hot_constitutive) with the adaptive Kn_GLL
 * mask of Sec. 3.1, the steady synthetic equations of Eq. (macroscopic_equation)
 * (Sec. 3 step 3) and the particle modification of Sec. 3.2.
 *
 * Conventions for every entry point:
 *  - Plain C types only.  "dev" pointers are CUDA device pointers on the
 *    device that was current when dsmc_init ran; "host" pointers are CPU
 *    memory.  Arrays are dense, row-major, FP64 unless stated.
 *  - The caller owns every buffer it passes, including the workspace given to
 *    dsmc_init; the library never frees caller memory and allocates no device
 *    memory at run time.  The library owns the opaque handle (host memory)
 *    and one fixed device array used only by synth_solve_noalloc.
 *  - Work is queued on the CUDA stream given to dsmc_init.  Calls that return
 *    host values (counts, iterations, statistics) synchronise that stream.
 *  - Return value: DSMC_OK (0) or a negative DSMC_ERR_* code; no exception or
 *    longjmp crosses the ABI.  dsmc_last_error() describes the last failure
 *    on a handle.  On DSMC_ERR_ARG, DSMC_ERR_CAPACITY and DSMC_ERR_NUMERIC the
 *    simulation state is left unchanged unless stated otherwise.
 *  - A handle must not be used from two host threads at once.
 *
 * Units (Sec. 2): lengths in L0, density in rho0, temperature in T0, speed in
 * sqrt(R T0); a particle has unit mass; I_r is the rotational energy of one
 * molecule per unit mass in units of R T0, so <I_r> = (d_r/2) T_r.
 */
#ifndef DIG_DSMC_H
#define DIG_DSMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DSMC_ABI_VERSION 2

#define DSMC_OK 0
#define DSMC_ERR_ARG (-1)           /* invalid argument or configuration */
#define DSMC_ERR_CAPACITY (-2)      /* particle count would exceed the workspace */
#define DSMC_ERR_NUMERIC (-3)       /* non-finite or non-positive rho / T input */
#define DSMC_ERR_NOT_CONVERGED (-4) /* synth_solve hit n_m iterations; outputs written */
#define DSMC_ERR_TIMEOUT (-5)       /* a bounded device wait gave up */
#define DSMC_ERR_CUDA (-6)          /* a CUDA runtime call failed */

#define DSMC_PREC_FP64_DET 0 /* FP64 particles, oracle-identical event order */
#define DSMC_PREC_FP32 1     /* FP32 particles in padded cell bins, FP64 moments */

#define DSMC_WALL_DIFFUSE 0  /* full accommodation at wall_t, wall_u (Sec. 4) */
#define DSMC_WALL_SPECULAR 1 /* mirror reflection */

#define DSMC_NFIELDS 18 /* rho, u(3), T_t, T_r, sigma(xx yy zz xy xz yz), q_t(3), q_r(3) */
#define DSMC_NHOT 12    /* HoT of sigma (6), q_t (3), q_r (3) */
#define DSMC_NTARGET 6  /* rho, u(3), T_t, T_r */
#define DSMC_NMOM 17    /* raw sums per cell, see dsmc_get_accumulators */

/* Simulation description.  Walls: 0 at x = 0, 1 at x = lx, 2 at y = 0,
 * 3 at y = ly (2D only).  A 1D slab has walls 0 and 1 only and ignores ny, ly. */
typedef struct dsmc_config {
  int32_t version;   /* DSMC_ABI_VERSION */
  int32_t dim;       /* 1 or 2 */
  int32_t nx, ny;    /* uniform Cartesian cells */
  int32_t ppc;       /* initial particles per cell */
  int32_t precision; /* DSMC_PREC_* */
  double lx, ly;     /* domain lengths */
  double kn;         /* global Knudsen number, Sec. 2: mu_ref = Kn sqrt(2/pi) */
  double omega;      /* VHS viscosity index (Sec. 4: 0.74) */
  double alpha;      /* VSS scattering exponent, 0 < alpha <= 2 (1: VHS, isotropic) */
  double z_rot;      /* rotational collision number Z, Eq. (P_inelastic) */
  double d_r;        /* rotational degrees of freedom: 2 (linear) or 3 (non-linear molecules) */
  double a_matrix[4]; /* A_tt, A_tr, A_rt, A_rr of Eq. (heat_flux_relaxation) */
  double dt;          /* time step */
  int32_t wall_kind[4];
  double wall_t[4];
  double wall_u[4][3]; /* wall velocity; its normal component must be 0 */
  double init_rho, init_tt, init_tr; /* initial uniform equilibrium state */
  double init_u[3];
  int32_t collisions; /* 1: collide (normal); 0: collisionless gas */
  int32_t n_s;        /* DSMC steps per DIG iteration (informational) */
  int32_t n_m;        /* maximum synth_solve iterations (Sec. 3 step 3) */
  int32_t pad0;
  double kn_ref;      /* Kn_GLL threshold of Sec. 3.1 */
  double synth_tol;   /* synth_solve stops when the relative change is below this */
  uint64_t seed;      /* Philox4x32-10 key */
  int64_t capacity;   /* maximum particles; 0 = chosen from ppc and bin_slack */
  double bin_slack;   /* FP32 layout: a cell's bin holds slack x its count (+32) */
  /* Mesh (DSMC_MESH_*).  DSMC_MESH_ANNULUS is the flow past a cylinder of
   * Sec. 4.2: r_in <= r <= r_out, nx angular x ny radial cells (cell j nx + k,
   * sector k between the rays at 2 pi k / nx and 2 pi (k+1) / nx, ring j
   * between R_j and R_{j+1}, R_j = r_in + (r_out - r_in) (q^j - 1) /
   * (q^ny - 1) with q = stretch, uniform for q = 1); wall 0 is the cylinder
   * (at rest; walls 1-3 are unused); particles leave through the outer
   * circle and the freestream (fs_rho, fs_t, fs_u) enters through it with
   * the one-sided flux of a drifting Maxwellian.  lx, ly are not used; ppc
   * is the mean number of particles per cell, the weight F = init_rho x
   * (annulus area / cells) / ppc, and cell c starts with Iround(init_rho
   * V_c / F) particles.  Single case only; dsmc_hot, dig_correct and the
   * HoT network work on its polar gradients and cell volumes, synth_solve
   * with synth2d = 1 (nx >= 5 sectors, ny >= 3 rings).
   * DSMC_MESH_REFINED is the wall-refined 2D box of Sec. 4.1: the box's
   * walls, nx x ny cells whose widths grow geometrically by the factor q =
   * stretch from both walls of each axis to the middle (widths proportional
   * to q^min(i, n-1-i), summing to lx or ly); ppc is the mean per cell, F
   * = init_rho lx ly / (nx ny ppc), cell c starts with Iround(init_rho V_c
   * / F) particles.  Single case only; synth_solve works on it with
   * synth2d = 1 (differences over the distances between cell centres, each
   * balance divided by its cell's width, the total mass weighted by V_c). */
  int32_t mesh;
  /* 1: reserve workspace for the 2D synthetic solve of a single box case
   * (synth_solve on dim 2; min(nx, ny) <= 500).  Its banded factorisation
   * takes about 8 N (20 m + 158) bytes, N = 5 nx ny unknowns,
   * m = min(nx, ny) (15 MB at 24 x 24, 0.86 GB at 100 x 100); 0 leaves it
   * out (synth_solve on a 2D handle then returns DSMC_ERR_ARG). */
  int32_t synth2d;
  double r_in, r_out, stretch;
  double fs_rho, fs_t, fs_u[3];
} dsmc_config;

#define DSMC_MESH_BOX 0
#define DSMC_MESH_ANNULUS 1
#define DSMC_MESH_REFINED 2

typedef struct dsmc_handle dsmc_handle;

/* Workspace bytes dsmc_init needs for cfg (device memory, 256-byte aligned,
 * any contents).  Returns DSMC_ERR_ARG for an unsupported configuration. */
int dsmc_workspace_size(const dsmc_config *cfg, size_t *bytes);

/* Create a simulation in the caller's workspace (dev, >= dsmc_workspace_size
 * bytes) on stream (a cudaStream_t, or NULL for the legacy default stream) and
 * fill it with the uniform equilibrium state of cfg: in every cell, ppc
 * particles uniform in the cell with Maxwellian velocities at (init_u,
 * init_tt) and rotational energies I_r with I_r / init_tr Gamma(d_r / 2)
 * distributed (exponential for d_r = 2) (Sec. 3 step 1: particles
 * initialised from an equilibrium distribution).
 * The workspace must stay allocated until dsmc_destroy. */
int dsmc_init(const dsmc_config *cfg, void *dev_workspace, size_t bytes, void *stream,
              dsmc_handle **out);

/* A batch: ncases independent simulations (cfgs[0..ncases-1], same dim and
 * precision; each with its own cells, gas, walls, time step, particles per
 * cell and seed) held by one handle and advanced together, one kernel launch
 * per stage for all of them.  Cells are numbered case after case: case k owns
 * the cfgs[k].nx * ny cells that follow those of cases 0..k-1, and every
 * array argument of the calls below (fields, HoT, targets, accumulators,
 * (sigma g)_max) uses that numbering.  Random streams are keyed by each
 * case's seed and its own cell numbers, so in FP64-deterministic mode a case
 * evolves exactly as it would alone.  synth_solve solves every slab;
 * dsmc_set_particles is not available for a batch.  The paper has no batch
 * mode: it is how dozens of uneven cases (or replicas for ensemble averages)
 * share the GPU. */
int dsmc_batch_workspace_size(const dsmc_config *cfgs, int ncases, size_t *bytes);
int dsmc_batch_init(const dsmc_config *cfgs, int ncases, void *dev_workspace, size_t bytes,
                    void *stream, dsmc_handle **out);

/* Release the handle (host memory only; the workspace stays the caller's). */
int dsmc_destroy(dsmc_handle *h);

/* Text of the last error on h (never NULL). */
const char *dsmc_last_error(const dsmc_handle *h);

/* Advance nsteps DSMC time steps (Sec. 2.2), each in the order: free flight
 * with wall interaction, cell indexing and sort, No-Time-Counter collisions
 * with VHS cross-section and Borgnakke-Larsen exchange (Eq. P_inelastic),
 * and, if sample != 0, accumulation of the cell sums behind
 * Eq. (DSMC_macroscopic); on the annulus the freestream enters after the
 * flight.  Asynchronous, except that the FP32 layout reads a few words back
 * at the end to decide whether its cell bins must be rebuilt, and the FP64
 * layout on the annulus synchronises every step to learn its particle
 * count.  DSMC_ERR_TIMEOUT: a cell's bulk copy did not complete in time.
 * DSMC_ERR_CAPACITY (unlike elsewhere, the steps have run): particles did
 * not fit (the FP32 overflow list was full, or on the annulus the freestream
 * entries exceeded the workspace) and those particles are lost. */
int dsmc_step(dsmc_handle *h, int nsteps, int sample);

/* Time-averaged cell fields of Eq. (DSMC_macroscopic) from the sums
 * accumulated since the last reset: dev_fields is ncells x DSMC_NFIELDS.
 * Central moments are taken about the time-averaged velocity; T_r =
 * 2 sum(I_r)/(d_r N); empty cells give zeros.  reset != 0 clears the sums
 * afterwards. */
int dsmc_sample(dsmc_handle *h, double *dev_fields, int reset);

/* Higher-order terms, Eq. (hot_constitutive): dev_hot (ncells x DSMC_NHOT) =
 * sampled stress and heat fluxes minus the NSF relations of
 * Eq. (ns_constitutive) evaluated with the sampled fields (kappa from
 * Eq. (kappa_A)); dev_kngll (ncells) = Kn_GLL of Sec. 3.1; dev_mask (ncells,
 * uint8) = 1 where Kn_GLL >= kn_ref.  HoT is set to 0 where mask = 0.
 * Any of dev_kngll / dev_mask may be NULL. */
int dsmc_hot(dsmc_handle *h, const double *dev_fields, double *dev_hot, double *dev_kngll,
             uint8_t *dev_mask);

/* Steady synthetic equations (Eq. macroscopic_equation with the
 * constitutive relations of Eq. full_constitutive), Sec. 3 step 3, solved
 * by Newton's method from dev_fields (ncells x DSMC_NFIELDS) with the
 * higher-order terms dev_hot (ncells x DSMC_NHOT) until the largest relative
 * update is below synth_tol or n_m iterations.
 *
 * 1D slab: u_x = 0; the first and last cell keep the sampled u_y, u_z, T_t,
 * T_r (Dirichlet); total mass equals the sampled mass.  Block cyclic
 * reduction of the block-tridiagonal Newton system.
 *
 * 2D box, uniform or wall-refined (single case with synth2d = 1; nx, ny >=
 * 3): unknowns rho, u_x, u_y, T_t, T_r per cell (u_z keeps its sampled
 * value); cells next to a wall keep the sampled u_x, u_y, T_t, T_r and
 * balance their mass; the four corner cells keep their sampled state and
 * exchange no flux; cell (1, 0)'s mass balance is replaced by the total mass
 * (sum rho V_c); face fluxes carry a fourth-difference dissipation of the
 * conserved variables (1/32 of the face's |u_n| + sound speed).
 *
 * Annulus around a cylinder (single case with synth2d = 1; nx >= 5 sectors,
 * ny >= 3 rings): the same equations by finite volumes on the sector cells
 * (face vectors the integrals of the faces' normals, so a uniform state is
 * exact; velocities Cartesian, each face's flux in its own normal frame);
 * both boundary rings (next to the cylinder and on the freestream side)
 * keep their whole sampled state; no total-mass row.
 *
 * Residual and central-difference Jacobian in
 * FP64; each Newton step solves with a blocked banded LU factorisation
 * (partial pivoting) of the Jacobian in FP32 and iterative refinement with
 * FP64 residuals; later Newton steps reuse the factorisation while the
 * updates keep halving.  At most min(n_m, 100) Newton iterations.
 *
 * dev_out is ncells x DSMC_NTARGET.  host_iters / host_resid (may be NULL)
 * receive the iteration count and the final max |residual|.  Returns
 * DSMC_ERR_ARG on a 2D handle without synth2d;
 * DSMC_ERR_NOT_CONVERGED (outputs written) when the iteration limit is
 * reached; DSMC_ERR_NUMERIC when no Newton update keeps rho > 0 and T > 0
 * (noisy HoT can make rho = (P - HoT_xx) / T_t negative in 1D, and a
 * singular 2D system admits no update) or, in 2D, when positivity cuts a
 * Newton step below 1/1024 of itself (no solution near the state, e.g. a
 * shock the central differences cannot carry), in which case the output is the
 * sampled fields, so that it can still serve as a dig_correct target;
 * DSMC_ERR_TIMEOUT when a bounded wait of the 2D substitution gave up (its
 * CTAs wait on one another; no result is written then).  In a batch the
 * worst status of the slabs is returned. */
int synth_solve(dsmc_handle *h, const double *dev_fields, const double *dev_hot, double *dev_out,
                int *host_iters, double *host_resid);

/* 2D synthetic solve across calls (Sec. 3: each DIG iteration solves the
 * same grid's equations again, for fields that change little from one
 * iteration to the next).  Bit 0 of `on`: each synth_solve starts from the
 * factorisation of the Jacobian that the handle's previous synth_solve left
 * in the workspace (none before the first call), and refactorises only when
 * the Newton updates stop halving.  Bit 1: Newton starts from the previous
 * call's solution (when that call converged) instead of the sampled fields
 * (the boundary rows' equations pin their cells to the new sampled values
 * in the first step).  A solve that does not converge this way is repeated
 * from a fresh factorisation and the sampled fields, so the converged
 * solution is the same as with on = 0 up to the tolerance.  on = 0 (the
 * default) factorises in every call and starts from the sampled fields.
 * DSMC_ERR_ARG unless the handle is a single 2D case with synth2d = 1. */
int dsmc_synth_reuse(dsmc_handle *h, int on);

/* Particle modification of Sec. 3.2 to the target dev_target (ncells x
 * DSMC_NTARGET = rho, u, T_t, T_r): (i) N_new = Iround(rho V / F); (ii) remove
 * uniformly chosen particles, or add copies of uniformly chosen existing ones
 * placed uniformly in the cell (an empty cell draws from the target
 * Maxwellian); (iii) sample u*, T_t*, T_r* of the result; (iv) v <- a v + b,
 * I_r <- c I_r with a = sqrt(T_t/T_t*), b = u - a u*, c = T_r/T_r*.
 * DSMC_ERR_NUMERIC (nothing changed) if a target is non-finite, rho < 0 or,
 * where rho > 0, a temperature <= 0 (a cell with rho = 0, such as an
 * unsampled cell's fields, empties and its temperatures are not used);
 * DSMC_ERR_CAPACITY (nothing changed) if the new total does not fit. */
int dig_correct(dsmc_handle *h, const double *dev_target);

/* Largest slab synth_solve_noalloc accepts. */
#define DSMC_SYNTH_NOALLOC_MAX_CELLS 2048

/* synth_solve for callers that cannot allocate device memory.  The paper has
 * no counterpart: this is a library convenience.  Callers such as a host code
 * whose device memory is owned by another allocator (a pool it may not grow
 * or bypass), or one that runs under a device-memory budget fixed at
 * start-up, where a new allocation is not permitted, cannot create a handle,
 * because dsmc_init needs a workspace they would have to allocate.  This
 * call needs no handle and no workspace: it reads the configuration from
 * cfg (dim must be 1, nx >= 3) and solves the same
 * discrete equations as synth_solve, from the same kind of inputs
 * (dev_fields ncells x DSMC_NFIELDS, dev_hot ncells x DSMC_NHOT) into
 * dev_out (ncells x DSMC_NTARGET), all caller-owned device arrays, on
 * stream (a cudaStream_t or NULL).  It calls no cudaMalloc, cudaFree or
 * allocating library routine.
 *  - Scratch: the solver's Newton scratch lives in one fixed device array in
 *    the library (about 1.8 MB, enough for DSMC_SYNTH_NOALLOC_MAX_CELLS
 *    cells); every GPU that loads the library holds it until the process
 *    exits.  nx above DSMC_SYNTH_NOALLOC_MAX_CELLS returns DSMC_ERR_CAPACITY
 *    and launches nothing.
 *  - The first call on a device looks up the array's device address on the
 *    current device (once per device); make that first call before any
 *    stream capture on that device.
 *  - Every call uses the same array, which keeps the last call's contents;
 *    the solver writes each scratch word before it reads it.  Calls that
 *    overlap on the GPU (other streams, other host threads) race on the
 *    array and corrupt each other's results: serialise them.
 *  - Waits on stream between batches of Newton iterations (it reads the
 *    convergence count back) and synchronises it before returning, so it
 *    cannot be captured into a CUDA graph: on a stream that is capturing
 *    (or the legacy stream while another stream captures) it returns
 *    DSMC_ERR_ARG and launches nothing;
 *    host_iters / host_resid (may be NULL) receive the iteration count and
 *    the final max |residual|.  Returns DSMC_OK,
 *    DSMC_ERR_NOT_CONVERGED (outputs written), DSMC_ERR_NUMERIC,
 *    DSMC_ERR_ARG, DSMC_ERR_CAPACITY or DSMC_ERR_CUDA. */
int synth_solve_noalloc(const dsmc_config *cfg, const double *dev_fields, const double *dev_hot,
                        double *dev_out, void *stream, int *host_iters, double *host_resid);

/* ---- state access (tests, checkpoints, diagnostics) ---------------------- */

/* Number of particles (synchronises). */
int dsmc_num_particles(dsmc_handle *h, int64_t *host_n);

/* Copy the particles out, cell by cell (cell index order; within a cell the
 * current storage order), converted to FP64: six dev arrays of length
 * capacity_out (x, y, vx, vy, vz, I_r; y = 0 in 1D) and dev_cell (int32).
 * host_n receives the count; DSMC_ERR_CAPACITY if capacity_out is too small. */
int dsmc_get_particles(dsmc_handle *h, double *dev_x, double *dev_y, double *dev_vx, double *dev_vy,
                       double *dev_vz, double *dev_ir, int32_t *dev_cell, int64_t capacity_out,
                       int64_t *host_n);

/* Replace the particles by n given ones (dev FP64 arrays; y ignored in 1D);
 * they are binned by position keeping their given order within a cell. */
int dsmc_set_particles(dsmc_handle *h, int64_t n, const double *dev_x, const double *dev_y,
                       const double *dev_vx, const double *dev_vy, const double *dev_vz,
                       const double *dev_ir);

/* Raw per-cell sums (dev, ncells x DSMC_NMOM): N, sum v_i (3), sum v_i v_j
 * (xx yy zz xy xz yz), sum v_i |v|^2 (3), sum I_r, sum I_r v_i (3), over the
 * sampled steps since the last reset; host_nsamples receives their number. */
int dsmc_get_accumulators(dsmc_handle *h, double *dev_out, int64_t *host_nsamples);

/* Per-cell (sigma g)_max (dev, ncells), read or overwritten. */
int dsmc_get_sgmax(dsmc_handle *h, double *dev_out);
int dsmc_set_sgmax(dsmc_handle *h, const double *dev_in);

/* Step counter (keys the random streams of the DSMC step) and DIG iteration
 * counter (keys those of dig_correct). */
int dsmc_get_counters(dsmc_handle *h, uint32_t *host_step, uint32_t *host_dig_iter);
int dsmc_set_counters(dsmc_handle *h, uint32_t step, uint32_t dig_iter);

/* Event counters since dsmc_init (host, 8 entries): candidate pairs, accepted
 * collisions, accepted pairs with sigma g > (sigma g)_max, Borgnakke-Larsen
 * events, wall hits, flights cut after 8 wall hits, particles that did not fit
 * their cell bin (FP32 layout, kept in an overflow list until the next
 * rebuild), bin rebuilds. */
int dsmc_get_stats(dsmc_handle *h, int64_t *host_out8);

/* Annulus: particles that entered through the outer circle and particles
 * that left through it since dsmc_init (host, 2 entries), so that the count
 * is the initial one + entered - left; an entering particle whose partial
 * flight ends outside never entered and is in neither.  Zero on the box. */
int dsmc_get_flow(dsmc_handle *h, int64_t *host_out2);

/* Cell volumes (areas per unit depth in 2D, lengths in 1D) of every cell
 * (host, ncells doubles).  Fields from dsmc_sample use them for rho. */
int dsmc_get_volumes(dsmc_handle *h, double *host_out);

/* Wall tallies since dsmc_init (host, 4 walls x 5): hits, momentum (3) and
 * energy (translational + rotational) delivered to the wall, per unit mass
 * of a simulated particle (multiply by F = rho V / N for physical units). */
int dsmc_get_wall_tally(dsmc_handle *h, double *host_out20);

/* Launch shape of the FP32 fused step (host): warps (= cells) per CTA, 2
 * or 4.  A handle times four shapes -- 4 warps with the tile sized from the
 * particles per cell, 2 warps, and 4 warps with the tile 32 particles
 * smaller and larger -- on real steps of its first dsmc_step call of at
 * least 20 steps and keeps the fastest (the first unless another is faster
 * by more than 1 %); 0 before that call and in the FP64-deterministic mode.
 * The paper has no counterpart. */
int dsmc_get_launch_config(dsmc_handle *h, int *host_warps_per_cta);

/* The same launch shape with its tile: particles staged per warp in shared
 * memory (cells above it take the chunked path); 0, 0 before the tuning
 * call and in the FP64-deterministic mode. */
int dsmc_get_launch_shape(dsmc_handle *h, int *host_warps_per_cta, int *host_tile);

/* Derived constants (host, 8 entries): dx, dy, cell volume V, particle weight
 * F, mu_ref, K (nu = K p / mu), C_sigma (sigma g = C_sigma g^(2-2 omega)),
 * P_inelastic. */
int dsmc_get_constants(dsmc_handle *h, double *host_out8);

/* ------------------------------------------------------------------------
 * HoT surrogate network (an extension; the paper has no counterpart: it
 * takes the higher-order terms of Eq. (hot_constitutive) from the DSMC
 * moments alone).  Each handle owns one network, 12 -> 64 -> 64 -> 64 -> 5
 * with tanh hidden layers, FP32 master weights and bfloat16 copies that the
 * forward and backward kernels use with FP32 accumulation.
 *
 * Inputs per cell (12): the gradients of rho, u_x, u_y, T_t, T_r along x and
 * y, scaled by the local mean free path lambda = mu(T)/(rho T) sqrt(pi T/2)
 * and by rho, sqrt(T), sqrt(T), T, T respectively, then Kn_GLL and T_r/T_t.
 * Outputs (5): HoT sigma_xx, sigma_xy, sigma_yy divided by p = rho T, and the
 * components of HoT q_t and q_r along grad T (x where grad T = 0) divided
 * by p sqrt(T).  The cells with mask = 1 (Kn_GLL >= kn_ref, as returned by
 * dsmc_hot) are the training set and the cells where the network replaces
 * those components; every other HoT component comes from DSMC.
 *
 * Parameters (DSMC_MLP_NPARAM floats, host memory): for each layer k = 1..4
 * the weights W_k (n_out x n_in, row major) then the biases b_k.  dsmc_init
 * sets them as hot_mlp_init does with the configuration's seed. */
#define DSMC_MLP_NPARAM 9477

/* Glorot-uniform weights and zero biases from a seeded generator on the
 * host; resets the Adam state. */
int hot_mlp_init(dsmc_handle *h, uint64_t seed);
/* Copy the FP32 master parameters in / out (host memory); set resets the
 * Adam state and rejects non-finite values (DSMC_ERR_NUMERIC). */
int hot_mlp_set_params(dsmc_handle *h, const float *host_params);
int hot_mlp_get_params(dsmc_handle *h, float *host_params);

/* Loss (mean over the mask = 1 cells of the mean squared error of the 5
 * normalised outputs against the DSMC HoT) and its gradient with respect to
 * the parameters (host_grad, DSMC_MLP_NPARAM floats, may be NULL), for the
 * fields / HoT / Kn_GLL / mask of dsmc_sample and dsmc_hot (device).  The
 * parameters are not changed.  DSMC_ERR_ARG if no cell has mask = 1. */
int hot_mlp_grad(dsmc_handle *h, const double *dev_fields, const double *dev_hot, const double *dev_kngll,
                 const uint8_t *dev_mask, float *host_grad, double *host_loss);

/* nsteps full-batch Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, step size
 * lr) on the same data; host_loss (may be NULL) receives the loss before the
 * last step. */
int hot_mlp_train(dsmc_handle *h, const double *dev_fields, const double *dev_hot, const double *dev_kngll,
                  const uint8_t *dev_mask, int nsteps, double lr, double *host_loss);

/* HoT for the synthetic equations: dev_hot_out (ncells x DSMC_NHOT) = the
 * network's sigma_xx, sigma_xy, sigma_yy and q_t, q_r along grad T where
 * mask = 1, the DSMC HoT (dev_hot) everywhere else and for every other
 * component; a cell whose prediction is not finite keeps the DSMC HoT.  The
 * network runs on the tensor cores (bfloat16 weights and layer inputs,
 * mma.sync with FP32 sums).
 * host_judge (may be NULL) receives the mean squared difference between the
 * network and the DSMC HoT over the mask = 1 cells (normalised units).
 * dev_hot_out may equal dev_hot. */
int hot_mlp_apply(dsmc_handle *h, const double *dev_fields, const double *dev_hot, const double *dev_kngll,
                  const uint8_t *dev_mask, double *dev_hot_out, double *host_judge);

/* hot_mlp_apply with the DSMC terms as the judge of the network, cell by
 * cell: each call adds, for every network cell (mask = 1), the residual r =
 * network - DSMC of its 5 normalised outputs, r^2 and the DSMC terms Y to
 * the running sums of its group (dev_group: ncells int32 ids in [0,
 * ncells), or NULL for one group per cell; e.g. the same cell of every
 * replica of a batch), and a network cell takes the network's HoT only if
 * its group holds at least min_samples (>= 2) residuals and, for every
 * output, |mean r| + z SE(r) <= rel |mean Y| (z > 0, rel > 0: the network's
 * bias is bounded, with z standard errors of confidence, by the fraction
 * rel of the DSMC terms); otherwise it keeps the DSMC HoT.  The sums
 * persist across calls (a DIG run's iterations) until hot_mlp_judge_reset
 * or a change of the parameters.  The inference runs on the tensor cores
 * (bfloat16 weights and inputs of every layer, FP32 sums).  host_nnet (may
 * be NULL) receives the number of cells given the network's HoT; host_judge
 * as in hot_mlp_apply. */
int hot_mlp_apply_judged(dsmc_handle *h, const double *dev_fields, const double *dev_hot, const double *dev_kngll,
                         const uint8_t *dev_mask, const int32_t *dev_group, double z, int min_samples, double rel,
                         double *dev_hot_out, double *host_judge, int64_t *host_nnet);

/* Clear the judge's running sums (hot_mlp_apply_judged). */
int hot_mlp_judge_reset(dsmc_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* DIG_DSMC_H */
