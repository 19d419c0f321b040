/*
 * evd.h -- C ABI of libevd, a GB300 (sm_103a) implementation of the forced
 * explicit velocity-difference (EVD) multicomponent lattice Boltzmann step of
 * Lourenco, Constantino & Tavares, "Forcing mass transfer approach in
 * multicomponent miscible mixtures using the lattice Boltzmann method",
 * Chem. Eng. Sci. 2025 (arXiv 2504.07059).
 *
 * One time step (Sec. 2 and 3 of the paper), per species i and lattice node x:
 *   1. streaming with the species' own lattice speed c_i = sqrt(M_1/M_i)
 *      (Eq. speed_DLS, Eq. discrete_velocity_DLS) and second-order spatial
 *      interpolation back to the nodes (Eq. Second_order_spatial_interpolation),
 *      closed at impermeable walls by the mass-conserving scheme of App. A and
 *      periodic elsewhere;
 *   2. moments rho_i, forced equilibrium velocity u_i^eq (Eq.
 *      first_order_moment_force), mixture rho and u, number density n and ideal
 *      pressure p = n M_1 c_s1^2 (Sec. 4.1);
 *   3. cross relaxation times tau_ij from the Maxwell-Stefan diffusivities
 *      (Eq. Luo&Girimaji_tau for two species, the closed forms of Sec. 4.1 for
 *      three);
 *   4. BGK self collision (Eq. BGK_self_collision) about f^{i(0)} (Eq. feqi0),
 *      the velocity-difference cross collision (Eq. Cross_collision_Sirovich)
 *      and the forcing term (Eq. CE_forcing_term_discretized) with
 *      F_i = rho_i g, combined as in Eq. (LBE_forcing).
 *
 * Conventions.
 *   - Sites are ordered x fastest: site = x + nx*(y + ny*z).  D2Q9 has nz = 1.
 *   - Species are given in non-decreasing molar mass; species 0 is the lightest
 *     and has lattice speed c = 1 (the paper's species 1).
 *   - Lattice units throughout, dt = dx = 1.
 *   - D2Q9 directions follow Eq. (discrete_velocity_DLS): 0 rest, 1 (+x),
 *     2 (+y), 3 (-x), 4 (-y), 5 (+x+y), 6 (-x+y), 7 (-x-y), 8 (+x-y).
 *     D3Q19 (an extension; the paper is two-dimensional): 0 rest, 1..6 =
 *     +x -x +y -y +z -z, then (+x+y) (-x-y) (+x-y) (-x+y) (+x+z) (-x-z)
 *     (+x-z) (-x+z) (+y+z) (-y-z) (+y-z) (-y+z).
 *   - Host arrays are owned by the caller and copied.  Device arrays are
 *     owned by the caller and must stay valid until the stream has consumed
 *     them.  Every "_device" call is asynchronous on the context's stream;
 *     every host-array readout synchronises that stream.
 *   - No call aborts or exits.  Each returns a status; evd_last_error() gives
 *     a message.  After EVD_ERR_CUDA the context must be destroyed.
 *   - A context is not thread-safe; calls on one context must be serialised.
 */
#ifndef EVD_H
#define EVD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EVD_API_VERSION 1

typedef enum {
    EVD_OK = 0,
    EVD_ERR_ARG = 1,       /* invalid argument or configuration                      */
    EVD_ERR_CUDA = 2,      /* a CUDA runtime call failed; the context is unusable     */
    EVD_ERR_UNSTABLE = 3,  /* a kernel saw rho_i <= 0, a NaN, or a non-positive tau_ij */
    EVD_ERR_TIMEOUT = 4,   /* a bounded device-side wait gave up                      */
    EVD_ERR_STATE = 5      /* call out of order (e.g. step before set_fields)         */
} evd_status;

typedef enum { EVD_D2Q9 = 0, EVD_D3Q19 = 1 } evd_lattice;

/* Storage and arithmetic of the populations.
 *   EVD_FP64       double storage, double arithmetic.
 *   EVD_FP32       float storage of deviations, float arithmetic on them, in
 *                  one of two encodings (evd_set_reference_mode):
 *                  - one reference per species: f - w_a rho_ref_i with
 *                    rho_ref_i the mean initial density of species i;
 *                  - the node's own density: the rest plane holds the
 *                    species density rho_i(x) and the other planes
 *                    f_a - w_a rho_i(x); the rest deviation is minus the sum
 *                    of the others (the deviations of a post-collision state
 *                    sum to zero), so it costs no extra bytes.  A stencil
 *                    value from node X enters node O as
 *                    g(X) + w_a (rho(X) - rho(O)), and the moments and the
 *                    collision work on deviations from rho(O): a species
 *                    depleted a thousandfold somewhere keeps the precision of
 *                    its own density there.
 *   EVD_FP16_STORE half storage of the deviation f - w_a rho~_i(x) from the
 *                  node's own species density, which is stored too (as a
 *                  half, one extra plane per species); float arithmetic on
 *                  deviations from the node's own density, as above.
 *                  Each stored value decodes with the density stored at its
 *                  own node, so interpolation still conserves mass and the
 *                  deviations stay small where densities differ strongly.
 * Per-species mass reductions are double in every mode. */
typedef enum { EVD_FP64 = 0, EVD_FP32 = 1, EVD_FP16_STORE = 2 } evd_precision;

/* wall_mask bits; a dimension is either periodic (both bits clear) or closed
 * by impermeable walls at both ends (both bits set). */
#define EVD_WALL_XM 0x01u
#define EVD_WALL_XP 0x02u
#define EVD_WALL_YM 0x04u
#define EVD_WALL_YP 0x08u
#define EVD_WALL_ZM 0x10u
#define EVD_WALL_ZP 0x20u

/* Species per lattice: up to 6 for D2Q9 in the general kernel (the cross
 * relaxation times then come from a dense solve of Eq.
 * relation_tauij_diff_coeff at every node); up to 3 for D3Q19, for batch
 * members, with the corrective forcing terms and for the adjoint (which use
 * the closed forms of Sec. 4.1). */
#define EVD_MAX_SPECIES 6
#define EVD_MAX_SPECIES_D3Q19 3

typedef struct {
    int lattice;          /* evd_lattice                                           */
    int precision;        /* evd_precision                                         */
    int nx, ny, nz;       /* nodes per dimension, >= 1; nz = 1 for D2Q9;          */
                          /* nx*ny*nz < 2^31                                       */
    unsigned wall_mask;   /* EVD_WALL_* bits                                       */
} evd_grid;

/* Corrective forcing terms of Eq. (improved_forcing_scheme), added to the
 * standard forcing term (Sec. 3; the paper finds them negligible in its cases,
 * Sec. 4.3):
 *   EVD_FORCE_S_DIFF  w [(e e - cs2 I)/cs2^2 . u] . Theta_i dt/(2 tau_i - dt)
 *   EVD_FORCE_S_P     - w [(e e - cs2 I)/cs2^2 . u] . grad(rho_i cs2)
 *   EVD_FORCE_S_RHO   w [(e e - cs2 I)/cs2 . u_i^eq] . (w_i grad rho)
 * Gradients: the isotropic lattice gradient (1/cs0^2) sum_a w_a e_a phi(x+e_a)
 * of the densities of f_t (the paper does not give one), a neighbour beyond a
 * wall taking the node's value.  D2Q9 only (EVD_ERR_ARG for D3Q19); the
 * gradient terms add one density pass over the populations per step. */
#define EVD_FORCE_S_DIFF 1u
#define EVD_FORCE_S_P 2u
#define EVD_FORCE_S_RHO 4u

typedef struct {
    int n_species;             /* 1 .. EVD_MAX_SPECIES (3 for D3Q19)                */
    const double* molar_mass;  /* [n_species], > 0, non-decreasing                  */
    const double* diffusivity; /* [n_species*n_species], symmetric Maxwell-Stefan   */
                               /* D_ij > 0 in lattice units; diagonal ignored        */
    double tau1;               /* self relaxation time of species 0, > 1/2; the     */
                               /* others follow from equal kinematic viscosity       */
    double g[3];               /* specific body force, F_i = rho_i g (gravity)       */
    unsigned flags;            /* EVD_FORCE_* corrective forcing terms, or 0          */
} evd_species;

typedef struct evd_ctx evd_ctx;

/* Library ABI version (EVD_API_VERSION). */
int evd_version(void);

/* Bytes of ONE population buffer for this configuration (the step ping-pongs
 * between two).  Returns 0 for an invalid configuration. */
size_t evd_required_bytes(const evd_grid* grid, const evd_species* species);

/* Create a context on the current CUDA device.  cuda_stream is a cudaStream_t
 * (NULL = legacy default stream); all work of the context is ordered on it.
 * The library allocates the two population buffers and small scratch.
 * On failure *out is NULL and evd_last_error(NULL) describes the problem. */
evd_status evd_create(const evd_grid* grid, const evd_species* species,
                      void* cuda_stream, evd_ctx** out);

/* As evd_create, but the two population buffers are caller-owned device
 * memory of at least evd_required_bytes() each, 256-byte aligned, and must
 * outlive the context.  Small scratch is still allocated by the library. */
evd_status evd_create_with_buffers(const evd_grid* grid, const evd_species* species,
                                   void* cuda_stream, void* pop_a, void* pop_b,
                                   size_t bytes_each, evd_ctx** out);

/* Change the stream later calls are ordered on. */
evd_status evd_set_stream(evd_ctx* ctx, void* cuda_stream);

/* Initial state (Sec. 4.1, 4.2): rho_i = x_i M_i n, zero velocities, and
 * populations f = f^{i(0)} of Eq. (feqi0) with the equilibrium velocity
 * replaced by u_i0 = -g dt/2, so that the first moments give u_i^eq = 0.
 * x: [n_species][sites] mole fractions (> 0); n: [sites] total number
 * density, or NULL for 1.  Resets the time to 0.  The host version
 * synchronises; the device version is asynchronous apart from one small
 * readback of the mean species densities. */
evd_status evd_set_fields(evd_ctx* ctx, const double* x_host, const double* n_host);
evd_status evd_set_fields_device(evd_ctx* ctx, const double* x_dev, const double* n_dev);

/* Replace the state by arbitrary post-stream populations f_t, host array
 * [n_species][Q][sites].  Keeps the time counter.  Synchronises. */
evd_status evd_set_populations(evd_ctx* ctx, const double* f_host);

/* Advance nsteps >= 0 time steps, asynchronously on the stream. */
evd_status evd_step(evd_ctx* ctx, long long nsteps);

/* Observables of the current state f_t, asynchronously, into device arrays
 * (any may be NULL):
 *   x   [n_species][sites]      mole fraction x_i = rho_i/(n M_i)
 *   rho [n_species][sites]      species density (Eq. zeroth_order_moment)
 *   u   [D][sites]              mixture velocity (Eq. Sirovich_mixture_velocity)
 *   ui  [n_species][D][sites]   species velocity u_i = u_i^eq - Theta_i/(2 rho_i)
 *                               (Eq. CE_EQ83), D = 2 or 3 by lattice. */
evd_status evd_readout_device(evd_ctx* ctx, double* x, double* rho, double* u, double* ui);

/* Host-array readouts (synchronise the stream). */
evd_status evd_get_mole_fractions(evd_ctx* ctx, double* x_host);
evd_status evd_get_densities(evd_ctx* ctx, double* rho_host);
evd_status evd_get_velocities(evd_ctx* ctx, double* u_mix_host, double* u_species_host);

/* Per-species total mass sum_x rho_i(x) of the current state, reduced in
 * double precision in a fixed order (bitwise reproducible run to run).
 * The device version writes [n_species] doubles asynchronously. */
evd_status evd_get_species_mass(evd_ctx* ctx, double* m_host);
evd_status evd_species_mass_device(evd_ctx* ctx, double* m_dev);

/* Post-stream populations f_t as doubles, host array [n_species][Q][sites]
 * (a test hook; allocates a temporary device buffer of that size). */
evd_status evd_get_populations(evd_ctx* ctx, double* f_host);

/* Time steps taken since the last evd_set_fields. */
long long evd_time(const evd_ctx* ctx);

/* Synchronise and report the device error flag: EVD_ERR_UNSTABLE if any
 * kernel since evd_set_fields saw a non-positive or NaN species density or a
 * non-positive or non-finite cross relaxation time, else EVD_OK.  (tau_ij
 * below 1/2 is a legitimate outcome of the ternary relation for trace
 * species and is not flagged.) */
evd_status evd_check(evd_ctx* ctx);

/* Number of kernels this context has launched so far (launch accounting). */
long long evd_launch_count(const evd_ctx* ctx);

/* Step kernel.  EVD_KERNEL_TMA stages the interpolation stencil of every
 * population plane in shared memory with TMA tile copies (D3Q19, FP32 with
 * one reference per species or FP16 storage, walls in x and y, rows a
 * multiple of 16 bytes); it is the default where it applies (the FP32
 * node-reference encoding runs the general kernel, and evd_get_kernel then
 * reports EVD_KERNEL_GENERAL).  EVD_KERNEL_GENERAL handles every configuration
 * (one thread per node, stencil read through the caches).  Both compute the
 * same step.  EVD_KERNEL_AUTO picks the first that applies; asking for
 * EVD_KERNEL_TMA where it does not apply is EVD_ERR_ARG. */
#define EVD_KERNEL_AUTO 0
#define EVD_KERNEL_GENERAL 1
#define EVD_KERNEL_TMA 2
evd_status evd_set_kernel(evd_ctx* ctx, int kernel);
int evd_get_kernel(const evd_ctx* ctx);

/* Reference of the EVD_FP32 encoding (not in the paper; a precision device).
 * EVD_REF_SPECIES: one reference density per species (the TMA-staged step
 * implements it).  EVD_REF_NODE: the node's own density (general kernel).
 * EVD_REF_AUTO (default): per node where some species' density varies by
 * more than a factor 2 over the initial field, per species otherwise.  The
 * choice is made by the next evd_set_fields / evd_set_fields_device /
 * evd_set_populations.  evd_get_reference_mode returns the encoding in
 * effect: EVD_REF_SPECIES or EVD_REF_NODE for EVD_FP32, EVD_REF_NODE for
 * EVD_FP16_STORE, EVD_REF_AUTO (0) for EVD_FP64, -1 for a NULL ctx. */
#define EVD_REF_AUTO 0
#define EVD_REF_SPECIES 1
#define EVD_REF_NODE 2
evd_status evd_set_reference_mode(evd_ctx* ctx, int mode);
int evd_get_reference_mode(const evd_ctx* ctx);

/* Per-node specific body force field k(x) added to the uniform g:
 * F_i(x) = rho_i (g + k(x)) in the moments, the forcing term and the initial
 * velocities (Eq. first_order_moment_force, Eq. CE_forcing_term_discretized;
 * the centrifugal force rho_i omega^2 r of Sec. 4.2 Case II is such a field).
 * k_host: host [D][sites] doubles (component-major, x fastest), finite;
 * copied to the device in the arithmetic type of the precision.  NULL removes
 * the field.  Set it before evd_set_fields, whose initial state uses it; it
 * applies to every later step and readout.  While a field is set the general
 * kernel runs the step (the TMA-staged step takes a uniform g only):
 * evd_get_kernel reports EVD_KERNEL_GENERAL and evd_set_kernel(EVD_KERNEL_TMA)
 * returns EVD_ERR_ARG.  Synchronises. */
evd_status evd_set_force_field(evd_ctx* ctx, const double* k_host);

/* Discrete adjoint of the step (D2Q9, FP64 storage, uniform g, no corrective
 * terms, mass correction off; EVD_ERR_ARG otherwise).  From the initial
 * state x0 (host [ns][sites] mole fractions) and n0 (host [sites] or NULL,
 * as evd_set_fields), runs nsteps steps and returns the loss
 *   L = sum_i sum_y (xbar_i(y) - target_i(y))^2,
 * xbar_i(y) the mean over x of the mole fractions after nsteps steps,
 * target host [ns][ny]; and its exact gradient with respect to the
 * Maxwell-Stefan diffusivities (dL_dD host [ns][ns], symmetric, zero
 * diagonal; NULL to skip) and the body force (dL_dg host [3], z entry 0;
 * NULL to skip).  The reverse sweep applies the transpose of each step:
 * the transposed Jacobian of the node-local collision of Eq. LBE_forcing
 * with tau_ij of Eq. relation_tauij_diff_coeff (exact; by hand-written
 * reverse mode or by dual numbers, as evd_set_adjoint_mode selects) and the
 * transposed gather (Eq. Second_order_spatial_interpolation and App. A).  States are recomputed from
 * checkpoints stored every checkpoint_every steps (0: about sqrt(nsteps));
 * memory: (nsteps / checkpoint_every + checkpoint_every + 3) population
 * buffers.  Leaves the context at t = nsteps of this run (FP64 forward).
 * Synchronises. */
evd_status evd_loss_gradient(evd_ctx* ctx, const double* x0, const double* n0, long long nsteps,
                             const double* target, int checkpoint_every, double* loss, double* dL_dD,
                             double* dL_dg);

/* How evd_loss_gradient applies the transpose of each node's collision
 * Jacobian.  EVD_ADJOINT_REVERSE (the default): reverse mode written out by
 * hand through the moments, tau_ij, V_i, the equilibria and the forcing term
 * of Eq. LBE_forcing (only the small Jacobian of the closed-form tau_ij is
 * taken in forward mode).  EVD_ADJOINT_DUAL: the Jacobian from forward-mode
 * dual numbers through the same collision code as the step, one tangent per
 * node moment (rho_i, J_i) and per parameter; slower, kept as a cross-check.
 * Both are exact up to rounding.  EVD_ERR_ARG for any other mode. */
#define EVD_ADJOINT_REVERSE 0
#define EVD_ADJOINT_DUAL 1
evd_status evd_set_adjoint_mode(evd_ctx* ctx, int mode);

/* Storage of evd_loss_gradient's forward pass.  EVD_FP64 (the default): the
 * context's own double-precision steps.  EVD_FP32: an internal float context
 * (node-reference encoding, no mass correction) runs the forward pass and
 * the checkpoint recomputation, reproducing each step's dithered rounding;
 * every state the reverse sweep needs is decoded to doubles, and the reverse
 * sweep (the transposed collision and gather) runs in FP64 as before.  The
 * gradient is then that of the FP32 trajectory, whose distance from the FP64
 * one the FP32 accuracy bounds.  In this mode the context itself stays at
 * t = 0 of the run.  EVD_ERR_ARG for another precision. */
evd_status evd_set_adjoint_forward(evd_ctx* ctx, int precision);

/* Rows per tile of the TMA-staged step: 1 (the default; four CTAs of 3 warps
 * per SM for three species, each synchronising only the species of its
 * row), 2 (two CTAs of 6 warps) or 4 (one CTA of 12 warps).  Same results;
 * a tuning knob.  Synchronises.  EVD_ERR_ARG where the TMA step does not
 * apply. */
evd_status evd_set_tile_rows(evd_ctx* ctx, int rows);

/* Poll limit of the TMA-staged step's waits for its tile copies (not in the
 * paper; the failure-detection path).  Every wait of a step for the
 * mbarrier that completes a tile copy polls at most `polls` times; a wait
 * that gives up makes every CTA that saw it stop stepping, wait (with the
 * default limit) for the copies it still has in flight, and set
 * EVD_ERR_TIMEOUT, which the next evd_check returns.  The output buffer is
 * then partly written and the context should be re-initialised (set_fields
 * or set_populations) or destroyed.  polls < 0 restores the default 2^22
 * (far longer than any copy takes); 0 makes every wait give up at once, which
 * is how the timeout path is tested.  Applies to the TMA step only.
 * EVD_ERR_ARG for a NULL ctx. */
evd_status evd_set_wait_limit(evd_ctx* ctx, int polls);

/* FP64 species-mass correction (not in the paper; a precision device for
 * FP32/FP16 storage).  Every `every` steps the step kernel also reduces the
 * per-species mass of f_t in double precision; the deficit from the initial
 * masses (the target, computed in double at evd_set_fields) is re-injected in
 * the next step in proportion to each node's density, f_a += w_a c_i rho_i(x)
 * with c_i = (m0_i - m_i)/m_i, so that a species is corrected where it is
 * present rather than by the same amount at nodes where it is a trace.  0 turns it
 * off.  Default: off for EVD_FP64, every 8 steps for EVD_FP32, every step for
 * EVD_FP16_STORE (its storage rounding drifts the mass faster). */
evd_status evd_set_mass_correction(evd_ctx* ctx, int every);

/* The FP64 target masses [n_species] (initial species masses).  Synchronises. */
evd_status evd_get_target_mass(evd_ctx* ctx, double* m_host);

/* Per-species total mass of a population array, without allocating.
 * The paper has no counterpart; this is a service for callers that cannot
 * call cudaMalloc: code whose device memory is owned by another allocator
 * (a framework's caching pool or an application's fixed budget), and loops
 * that must not pay the device-wide synchronisation cudaMalloc may cause.
 * Such callers can compute the mass of a state they hold, for instance the
 * output of evd_get_populations copied to their own device memory.
 *   f_dev  device array [n_species][q][nsites] of doubles (dense, caller-owned)
 *   n_species 1..3, q 9 (D2Q9) or 19 (D3Q19), nsites 1..2^40
 *   m_dev  device array [n_species] receiving sum over directions and sites
 * Asynchronous on cuda_stream (NULL = legacy default stream); sums in double
 * in a fixed order.  Allocates nothing: the block partial sums live in a
 * file-scope device array of 1024 x 3 doubles (24 KiB), present on every
 * device that loads the library until the process exits.  Its address is
 * looked up on the first call on each device (with that device current),
 * and again on the first call after that device's context was torn down
 * and created anew (cudaDeviceReset); make such a first call before any
 * stream capture.  All calls share the
 * array: calls that overlap on the GPU (different streams, or several host
 * threads) race and give wrong sums; serialise them.  Returns EVD_ERR_ARG
 * for sizes beyond the limits above and EVD_ERR_CUDA if a launch fails;
 * evd_last_error(NULL) then describes the problem. */
evd_status evd_population_mass_noalloc(const double* f_dev, int n_species, int q,
                                       long long nsites, double* m_dev, void* cuda_stream);

/* Arithmetic throughput of the current GPU (not in the paper; the roofline
 * of the FP64 step, which double-precision arithmetic bounds on this part):
 * 8 independent fused multiply-add chains per thread, iters links each, on 8
 * blocks of 256 threads per SM, timed with CUDA events on cuda_stream after
 * one warm-up launch.  kind 0: double FMA; 1: float FMA; 2: float pairs
 * (f32x2 FMA).  Returns the flops of the timed launch (2 per FMA and lane)
 * and its milliseconds; the rate at the clock the GPU ran is flops / ms.
 * Allocates and frees a small output array.  EVD_ERR_ARG for an unknown
 * kind or iters outside 1 .. 2^24; evd_last_error(NULL) describes errors. */
evd_status evd_fma_rate(int kind, int iters, double* flops, double* ms, void* cuda_stream);

/* Release the context and all memory the library allocated for it. */
evd_status evd_destroy(evd_ctx* ctx);

/* Message of the last failed call on ctx, or of the last failed evd_create*
 * on this thread when ctx is NULL.  Never NULL. */
const char* evd_last_error(const evd_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* EVD_H */
