/* evd_batch.h -- many independent lattices advanced together.
 *
 * A batch holds N independent members: lattices of one lattice type and one
 * storage precision, each with its own extents, walls and species table
 * (molar masses, Maxwell-Stefan diffusivities, tau_1, body force).  One step
 * of the batch advances every member by exactly the time step evd_step
 * performs for a single lattice (gather with the second-order interpolation
 * of Eq. Second_order_spatial_interpolation and the App. A walls, moments,
 * tau_ij, collision with forcing of Eq. LBE_forcing): the paper defines one
 * lattice at a time and has no counterpart of the batch, which exists only to
 * keep a GPU busy with many small problems (for instance a sweep of Loschmidt
 * tubes of uneven length, mass ratio, diffusivity and gravity).
 *
 * Execution: the members are cut into work items (ranges of consecutive sites
 * of one member).  A step is ONE kernel launch over all items of all members,
 * persistent by default (a grid of a few CTAs per SM looping over the items),
 * and runs of steps are replayed from a captured CUDA graph.  The item size
 * and the CTAs per SM are the schedule; evd_batch_autotune times candidate
 * schedules on the live state and keeps the fastest.
 *
 * Concatenated layouts.  Host and device field arrays hold the members one
 * after another in member order; inside member m (sites_m = nx*ny*nz, x
 * fastest) the layout is that of the single-lattice API:
 *   x, rho  : [ns_m][sites_m]           total  sum_m ns_m * sites_m
 *   n       : [sites_m]                 total  sum_m sites_m
 *   u       : [D][sites_m]              total  D * sum_m sites_m
 *   ui      : [ns_m][D][sites_m]        total  D * sum_m ns_m * sites_m
 *   mass    : [N][EVD_MAX_SPECIES]      (unused species slots are 0)
 * evd_batch_sizes returns these totals.
 *
 * Errors and streams follow evd.h: every call returns a status and sets the
 * batch's last error; steps are stream-ordered on the batch's stream; host
 * readouts synchronise it.  A batch is not thread-safe. */
#ifndef EVD_BATCH_H
#define EVD_BATCH_H

#include "evd.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct evd_batch evd_batch;

/* One member: extents (nz = 1 for D2Q9), EVD_WALL_* mask, species table.  The
 * same preconditions as evd_grid / evd_species in evd_create; the species
 * arrays are copied at evd_batch_create. */
typedef struct {
    int nx, ny, nz;
    unsigned wall_mask;
    evd_species species;
} evd_member;

/* Creates a batch of n_members >= 1 members of one lattice (EVD_D2Q9 or
 * EVD_D3Q19) and one precision (EVD_FP64, EVD_FP32, EVD_FP16_STORE) on the
 * current device.  Reduced storage keeps deviations from each node's own
 * density (EVD_FP32: in the rest plane, as evd_set_reference_mode's
 * EVD_REF_NODE; EVD_FP16_STORE: in an extra half plane) and rounds its last
 * operation with a dither seeded per step from a device step counter (so
 * graph replays draw fresh seeds; evd_batch_set_fields resets it and
 * evd_batch_autotune restores it).  Allocates two population buffers holding
 * every member (each member's planes padded to 64 elements) plus small
 * tables.
 * EVD_ERR_ARG if a member is invalid (the message names it), EVD_ERR_CUDA if
 * an allocation fails.  *out is NULL on failure. */
evd_status evd_batch_create(int lattice, int precision, const evd_member* members, int n_members,
                            void* cuda_stream, evd_batch** out);

/* Totals of the concatenated layouts above: sites (sum of sites_m) and
 * species_sites (sum of ns_m * sites_m).  Either pointer may be NULL. */
evd_status evd_batch_sizes(const evd_batch* b, long long* sites, long long* species_sites);

/* Initial state of every member (as evd_set_fields, Sec. 4.2 initialisation):
 * x host [species_sites] mole fractions, n host [sites] number densities or
 * NULL for 1.  Values must be > 0.  Sets t = 0 and the FP64 species-mass
 * targets.  Synchronises. */
evd_status evd_batch_set_fields(evd_batch* b, const double* x, const double* n);

/* Advances every member nsteps >= 0 steps.  Asynchronous on the stream.
 * EVD_ERR_STATE before evd_batch_set_fields. */
evd_status evd_batch_step(evd_batch* b, long long nsteps);

/* Observables of the current state of every member into DEVICE arrays laid
 * out as above (any of them NULL to skip), as evd_readout_device.
 * Asynchronous. */
evd_status evd_batch_readout_device(evd_batch* b, double* x, double* rho, double* u, double* ui);

/* The same into HOST arrays; synchronise and check the device error word
 * (EVD_ERR_UNSTABLE if a member went unstable). */
evd_status evd_batch_get_mole_fractions(evd_batch* b, double* x);
evd_status evd_batch_get_densities(evd_batch* b, double* rho);
evd_status evd_batch_get_velocities(evd_batch* b, double* u, double* ui);

/* Per-member species masses sum_x rho_i of the current state in FP64, host
 * [n_members][EVD_MAX_SPECIES].  Synchronises. */
evd_status evd_batch_get_species_mass(evd_batch* b, double* mass);

/* Schedule: sites per work item (a multiple of 128, 128..65536) and
 * persistent CTAs per SM (1..32), or 0 for one CTA per work item.
 * Rebuilds the work list; the results do not depend on it. */
evd_status evd_batch_set_schedule(evd_batch* b, int item_sites, int ctas_per_sm);
evd_status evd_batch_get_schedule(const evd_batch* b, int* item_sites, int* ctas_per_sm);

/* Times every candidate schedule (item sizes 128..2048, 2..16 persistent
 * CTAs per SM or one CTA per item) for steps_per_trial steps (even, 2..64)
 * on a copy of the current state, restores the state, keeps the fastest
 * schedule and returns it (either pointer may be NULL).  Needs
 * evd_batch_set_fields first and room for one more copy of the populations.
 * Synchronises. */
evd_status evd_batch_autotune(evd_batch* b, int steps_per_trial, int* item_sites, int* ctas_per_sm);

/* Runs of steps_per_graph steps (even, 2..1024, and a multiple of the
 * mass-correction interval when that is on) are captured once into a CUDA
 * graph and replayed; 0 launches every step directly.  Default 8.  The
 * results do not depend on it. */
evd_status evd_batch_set_graph(evd_batch* b, int steps_per_graph);

/* FP64 species-mass correction of every member, as evd_set_mass_correction:
 * every `every` steps (0 = off; default off for EVD_FP64, 8 for EVD_FP32, 1
 * for EVD_FP16_STORE). */
evd_status evd_batch_set_mass_correction(evd_batch* b, int every);

/* Steps taken since evd_batch_set_fields; -1 for NULL. */
long long evd_batch_time(const evd_batch* b);

/* Kernels launched on the device by this batch so far, those inside graph
 * replays included; -1 for NULL. */
long long evd_batch_launch_count(const evd_batch* b);

/* Synchronises and reads the device error word: EVD_ERR_UNSTABLE if any
 * member reached rho_i <= 0 or a non-positive / non-finite tau_ij. */
evd_status evd_batch_check(evd_batch* b);

/* Frees everything; NULL is a no-op returning EVD_OK. */
evd_status evd_batch_destroy(evd_batch* b);

/* Message of the last failed call on b (NULL: of the last failed
 * evd_batch_create on this thread). */
const char* evd_batch_last_error(const evd_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* EVD_BATCH_H */
