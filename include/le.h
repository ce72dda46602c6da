/*
 * le.h — C ABI of the GB300 (sm_103a) Lees-Edwards shear-flow MD library.
 *
 * The method is Lees-Edwards (LE) sheared periodic boundaries for short-range
 * molecular dynamics, after Xu et al., "Implementation and Parallel
 * Optimization of the Lees-Edwards Boundary Condition in ESPResSo++"
 * (arXiv 2109.11083).  One simulation handle holds one sheared box resident
 * in GPU memory; every step of the method runs in this library's CUDA kernels.
 *
 * Geometry and conventions (Sec. 2.1 of the paper):
 *   - flow along x, velocity gradient along z, vorticity along y;
 *   - box [0,Lx) x [0,Ly) x [0,Lz); streaming profile v_s(z) =
 *     shear_rate * (z - Lz/2) (Eq. 1);
 *   - the image box above is displaced along x by
 *     dX(t) = (shear_rate * Lz * t) mod Lx (Eq. 4, Fig. 1), with t = n * dt
 *     taken from the integer step n;
 *   - a particle leaving through the top face re-enters at the bottom with
 *     x -= dX and vx -= shear_rate * Lz; through the bottom face the mirror
 *     image (Eq. 4 with the sign of Fig. 1);
 *   - reduced LJ units (Sec. 2.4): positions in sigma, energies in eps.
 *
 * Memory and threads: every pointer argument is a HOST pointer owned by the
 * caller; the library copies inputs in and writes outputs into the caller's
 * buffers (pinned buffers make the copies faster).  The library owns all of
 * its device memory.  A handle must be used by one host thread at a time.
 * Particle arrays are in the caller's order (particle id = row index) even
 * though the library keeps particles sorted by cell internally.
 *
 * Errors: every call returns an le_status and never aborts.  le_last_error()
 * describes the last failure on a handle.  When le_step fails with
 * LE_ERR_BOND_BROKEN, LE_ERR_NONFINITE, LE_ERR_RANGE or LE_ERR_CAPACITY the
 * state is rolled back to what it was when that le_step call began.
 */
#ifndef LE_H
#define LE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define LE_API __attribute__((visibility("default")))
#else
#define LE_API
#endif

typedef struct le_sim le_sim; /* opaque, library-owned */

typedef enum le_status {
    LE_OK = 0,
    LE_ERR_INVALID_ARG = 1,   /* a null pointer, a size out of range, ... */
    LE_ERR_CUDA = 2,          /* a CUDA runtime call failed (message in le_last_error) */
    LE_ERR_OOM = 3,           /* device memory could not be allocated */
    LE_ERR_BOX_TOO_SMALL = 4, /* rc + skin must be below half of every box edge */
    LE_ERR_BOND_BROKEN = 5,   /* a FENE bond reached R0 (Eq. 11: infinite energy) */
    LE_ERR_NONFINITE = 6,     /* a force or velocity became NaN or infinite */
    LE_ERR_CAPACITY = 7,      /* the neighbour list overflowed and could not grow */
    LE_ERR_TIMEOUT = 8,       /* a bounded device-side wait gave up */
    LE_ERR_STATE = 9,         /* call order: e.g. le_step before le_set_particles */
    LE_ERR_RANGE = 10         /* a sampled |vx| > 1000 or m vy^2 > 2000: beyond the
                                 fixed-point range of the profile sums */
} le_status;

typedef enum le_precision {
    LE_FP64 = 0,              /* every quantity in FP64 */
    LE_FP32 = 1               /* FP32 pair forces and velocities; positions kept
                                 to FP64-class precision (see le_create) */
} le_precision;

typedef enum le_thermostat {
    LE_THERMO_NONE = 0,
    LE_THERMO_PECULIAR = 1,   /* Langevin on the peculiar velocity v - v_s(z) e_x (Eq. 5) */
    LE_THERMO_ABSOLUTE = 2,   /* the comparison variant of Sec. 2.2 (Fig. 3, xi_abs): the same
                                 friction and noise acting on the lab-frame velocity v */
    LE_THERMO_DPD = 3         /* DPD (Eqs. 6-8, read as the fluctuation-dissipation form):
                                 F_ij = [-xi w^2 (r^.v_ij) + sqrt(24 kT xi/dt) theta_ij w] r^,
                                 w = 1 - r/rc, for every pair within rc, v_ij against the
                                 image j refers to (moving at +-shear_rate*Lz across the
                                 face), theta_ij in U(-1/2,1/2) from Philox4x64-10 at counter
                                 (step, min id, max id, 1); momentum-conserving */
} le_thermostat;

typedef struct le_params {
    double eps, sigma;        /* LJ parameters (Eq. 9) */
    double mass;              /* particle mass m */
    double kT;                /* target temperature k_B T */
    double xi;                /* Langevin friction rate (Eq. 5): F = -xi m (v - v_s) + random */
    double dt;                /* time step */
    int    lj_shift;          /* 1: energy shift of Eq. 10 (does not change forces) */
    int    thermostat;        /* le_thermostat */
    double fene_k, fene_R0;   /* FENE bond (Eq. 11); used only when bonds are set */
    int    precision;         /* le_precision */
    uint64_t seed;            /* random-force stream: Philox4x64-10 with key (seed, system_id) */
    uint64_t system_id;       /*   and counter (step, particle id, 0, 0)                       */
    int    sample_every;      /* >0: accumulate stress and profile every this many steps */
    int    profile_bins;      /* number of z bins of the velocity profile (1..1024) */
    double angle_k;           /* k_a of the chain bending term (Eq. 12, read as
                                 k_a (1 + cos theta), theta the angle at the middle
                                 bead of two bonds); 0: none; used only with bonds */
    double force_cap;         /* > 0: each LJ pair force is limited to this magnitude
                                 (the push-off of overlapping random-walk chains
                                 before a melt is integrated; not part of Eqs. 9-13);
                                 LE_FP64 only; 0: none */
} le_params;

/* Fills *p with defaults: eps = sigma = mass = kT = xi = 1, dt = 0.005,
 * lj_shift = 1, thermostat = LE_THERMO_PECULIAR, fene_k = 30, fene_R0 = 1.5,
 * precision = LE_FP64, seed = 0, system_id = 0, sample_every = 1,
 * profile_bins = 20, angle_k = 0, force_cap = 0. */
LE_API void le_default_params(le_params *p);

/* Creates a handle for the box [0,box[0]) x [0,box[1]) x [0,box[2]) sheared at
 * shear_rate (Eq. 1), with LJ cut-off rc (strict r < rc) and Verlet skin
 * `skin`.  The cell grid has edge >= rc + skin.  cuda_stream is a cudaStream_t
 * (may be NULL for the legacy default stream); all device work of the handle
 * is ordered on it.  In LE_FP32 mode positions are stored as an FP64 cell
 * reference plus an FP32 (hi, lo) pair for the displacement from it, which
 * keeps ~48 significant bits near the reference.
 * Errors: LE_ERR_INVALID_ARG (null out/params, non-positive box, rc, dt or
 * mass, negative skin, bins out of range), LE_ERR_BOX_TOO_SMALL
 * (rc + skin >= half of an edge), LE_ERR_CUDA. */
LE_API le_status le_create(const double box[3], double shear_rate, double rc, double skin,
                           const le_params *p, void *cuda_stream, le_sim **out);

/* Bonds for the FENE potential (Eq. 11): nb pairs of particle ids (nb x 2,
 * row-major).  At most 8 bonds per particle.  Call before le_set_particles;
 * calling it afterwards re-initialises the forces from the current state.
 * Errors: LE_ERR_INVALID_ARG (id out of range once particles are set, a
 * self-bond, more than 8 bonds on a particle). */
LE_API le_status le_set_bonds(le_sim *s, int64_t nb, const int32_t *pairs);

/* Loads n particles: pos (n x 3, row-major, any real coordinates; they are
 * wrapped into the box as images at step 0, where dX = 0) and lab-frame vel
 * (n x 3).  Resets the step counter to 0, the samples and the counters, builds
 * the cell/Verlet lists and computes the initial total force.  1 <= n <= 2^24 (16,777,216).
 * Errors: LE_ERR_INVALID_ARG, LE_ERR_OOM, LE_ERR_BOND_BROKEN, LE_ERR_CUDA. */
LE_API le_status le_set_particles(le_sim *s, int64_t n, const double *pos, const double *vel);

/* Advances nsteps >= 0 velocity-Verlet steps (kick, drift, LE wrap and
 * velocity jump, rebuild when the skin-displacement + image-shift trigger
 * fires, LJ/FENE forces under the LE minimum image, Langevin on the peculiar
 * velocity, kick, samples).  Returns when the work has finished.
 * Errors (state rolled back to the start of the call): LE_ERR_BOND_BROKEN,
 * LE_ERR_NONFINITE, LE_ERR_RANGE, LE_ERR_CAPACITY (after growing the list
 * failed); also LE_ERR_STATE, LE_ERR_INVALID_ARG, LE_ERR_TIMEOUT, LE_ERR_CUDA. */
LE_API le_status le_step(le_sim *s, int64_t nsteps);

/* Conservative forces (LJ + FENE) of the current step, n x 3 row-major. */
LE_API le_status le_forces(le_sim *s, double *out);

/* Current positions wrapped into the box (LE image at the current dX) and
 * the matching lab-frame velocities, n x 3 each; either pointer may be NULL. */
LE_API le_status le_positions(le_sim *s, double *pos, double *vel);

/* out9: instantaneous Eq. 15 stress tensor of the current state, row-major
 * (sigma = -(1/V)[sum m (v - v_s)(v - v_s) + sum_{i<j} r_ij F_ij]);
 * xz_avg: mean of sigma_xz over the samples taken since the last reset;
 * nsamples: how many.  Any pointer may be NULL.  Viscosity (Eq. 14) is
 * xz_avg / shear_rate. */
LE_API le_status le_stress(le_sim *s, double out9[9], double *xz_avg, int64_t *nsamples);

/* Mean lab-frame vx in each of the nbins z-bins over the samples since the
 * last reset (NaN for an empty bin), and the particle counts per bin.
 * nbins must equal params.profile_bins. */
LE_API le_status le_velocity_profile(le_sim *s, int nbins, double *vx_mean, int64_t *counts);

/* The z-profiles of Sec. 3.1 (Fig. 3) over the same samples and bins as
 * le_velocity_profile (bin b = floor(z / Lz * nbins), z wrapped into [0, Lz),
 * full-step velocities):
 *   vx_mean[b]  mean lab-frame vx,
 *   t_y[b]      mean m vy^2 (the temperature from the vorticity component,
 *               which the shear flow does not carry),
 *   density[b]  mean particle count / bin volume (Lx Ly Lz / nbins),
 *   counts[b]   particle samples in the bin.
 * Any output pointer may be NULL; host arrays of nbins entries, owned by the
 * caller.  nbins must equal le_params.profile_bins (else
 * LE_ERR_INVALID_ARG).  Empty bins give NaN means. */
LE_API le_status le_profiles(le_sim *s, int nbins, double *vx_mean, double *t_y, double *density,
                             int64_t *counts);

/* Mean peculiar temperature (3N - 3 degrees of freedom) over the samples. */
LE_API le_status le_temperature(le_sim *s, double *tpec_avg);

/* Clears the running samples (stress, profile, temperature). */
LE_API le_status le_reset_samples(le_sim *s);

typedef struct le_counters {
    int64_t step;             /* current integer step n */
    int64_t particles;
    int64_t rebuilds;         /* list rebuilds since le_set_particles */
    int64_t image_rebuilds;   /* rebuilds the displacement alone would not have needed */
    int64_t list_capacity;    /* neighbour slots per particle */
    int64_t list_max;         /* largest neighbour count seen at a rebuild */
    int64_t cells[3];         /* cell grid */
    double  dX;               /* current image offset */
    double  list_mean;        /* mean neighbour count of the last build */
    int32_t force_threads;    /* launch shape of the pair kernel (threads per block) */
    int32_t list_threads;     /* launch shape of the list build */
} le_counters;

LE_API le_status le_get_counters(le_sim *s, le_counters *out);

/* Launch shapes.  The pair kernel sums each particle's forces in its own
 * thread in list order, the list build is one thread per particle and every
 * sample is a fixed-point integer sum, so the threads per block of these two
 * kernels change no result (trajectories are bit-identical); they only
 * change speed.
 *
 * le_set_launch: force_threads in {32, 64, ..., 256}, list_threads in
 * {32, 64, ..., 256} (multiples of 32; else LE_ERR_INVALID_ARG).  Takes
 * effect at the next step (captured graphs are dropped).
 *
 * le_tune: the autotuner.  Times every pair of force_threads in {128, 256}
 * and list_threads in {64, 128, 256} on this system with its own step graph
 * (list builds included): one 16-step warm-up chunk, then steps_per_trial
 * steps (rounded down to whole 16-step chunks, at least one), restoring the
 * state before and after every trial.  Two sweeps over the shapes; each
 * shape is scored by its faster trial and the fastest shape is kept.  The state after le_tune is the state
 * before it.  best_force / best_list (nullable) receive the choice;
 * ms_per_step (nullable) its measured time per step. */
LE_API le_status le_set_launch(le_sim *s, int force_threads, int list_threads);
LE_API le_status le_tune(le_sim *s, int steps_per_trial, int *best_force, int *best_list,
                         double *ms_per_step);

/* Checkpoint: an opaque copy of the whole dynamical state in the library's
 * internal (cell-sorted) layout: positions, velocities, forces, the integer
 * step, the last list-build record and the running samples.  With
 * buf == NULL, *bytes receives the size needed.  le_set_state accepts a blob
 * from a handle with the same box, parameters and particle count; stepping
 * after it reproduces the uninterrupted run bit for bit (the random force is
 * a pure function of seed, system id, step and particle id). */
LE_API le_status le_get_state(le_sim *s, void *buf, size_t *bytes);
LE_API le_status le_set_state(le_sim *s, const void *buf, size_t bytes);

/* Runs nsteps like le_step, as ONE launch of a graph captured for exactly
 * that many steps, with CUDA events around every launch of the pair-force
 * kernel and of the integrate kernel.  Returns the summed device time of each
 * (milliseconds) and the whole graph's device time.  Meant for measurement. */
LE_API le_status le_step_profiled(le_sim *s, int64_t nsteps, double *force_ms,
                                  double *integrate_ms, double *total_ms);

/* eager != 0: launch every kernel directly on the stream instead of through
 * CUDA graphs; the host reads the rebuild decision back after each step.
 * The kernels and the results are identical.  Profilers that cannot look
 * inside graphs with conditional nodes need this mode; it is slower. */
LE_API le_status le_set_eager(le_sim *s, int eager);

/* Device memory (bytes) a handle with these parameters and n particles
 * (nbonds bonds) would hold after le_set_particles, including the rollback
 * snapshot taken by le_step: for admission against a memory budget. */
LE_API le_status le_estimate_device_bytes(const double box[3], double shear_rate, double rc,
                                          double skin, const le_params *p, int64_t n,
                                          int64_t nbonds, size_t *bytes);

/* ---------------------------------------------------------------- batches
 * A batch advances many independent handles (boxes of uneven size, shear
 * rates, parameters) with ONE CUDA-graph launch per 16 steps.  Members that
 * share precision, bonds and thermostat kind form a group, and each kernel
 * of a step (drift, decide, the rebuild kernels, pair forces) is ONE launch
 * for the whole group: each block finds its member in a prefix table of
 * block counts and runs that member's own kernel code on its own data; the
 * rebuild kernels run every step, and blocks of members whose trigger did
 * not fire return at once.  A group launches with its first member's launch
 * shapes.  Each member's trajectory is bit-identical to stepping it alone
 * with le_step.  Members remain ordinary handles (their
 * outputs are read with le_forces, le_stress, ...), must have particles,
 * must not be stepped on their own while in a batch, and stay owned by the
 * caller.  The memory budget (0: none) bounds the sum of the members'
 * device memory; le_batch_add refuses a member beyond it with LE_ERR_OOM. */
typedef struct le_batch le_batch;

LE_API le_status le_batch_create(size_t budget_bytes, void *cuda_stream, le_batch **out);
LE_API le_status le_batch_add(le_batch *b, le_sim *s);
LE_API le_status le_batch_remove(le_batch *b, le_sim *s);
/* Advances every member nsteps.  On a member's error every member is rolled
 * back to the start of the call (list overflows are grown and retried). */
LE_API le_status le_batch_step(le_batch *b, int64_t nsteps);

/* The autotuner for a batch: every candidate shape of le_tune, applied to all
 * members, times the batch itself over 2 x 16-step chunks (as le_batch_step
 * runs it: all members' kernels together), every member rolled back to its
 * state before each trial; the fastest is kept.  Results are unchanged (see
 * le_set_launch).  best_force / best_list / ms_per_step (nullable) receive
 * the choice and its time per batch step. */
LE_API le_status le_batch_tune(le_batch *b, int steps_per_trial, int *best_force, int *best_list,
                               double *ms_per_step);
LE_API le_status le_batch_destroy(le_batch *b);
LE_API const char *le_batch_last_error(const le_batch *b);

/* Conservative LJ forces (Eq. 9/10, no bonds) on n particles at positions
 * pos (n x 3, host, caller order; any real coordinates, taken as images at
 * step `step`, whose image offset is dX(step) of Eq. 4) written to forces
 * (n x 3, host), for the box, shear rate, rc, skin and parameters of
 * le_create (precision selects FP64 or FP32 arithmetic; the thermostat,
 * bond, sampling and force_cap fields are ignored).  No handle is needed.
 * The paper has no counterpart to this entry point.  It exists for callers
 * that cannot call cudaMalloc where they need forces: a loop that must not
 * allocate device memory (or meet an out-of-memory error) once it runs, or a
 * host program whose device memory belongs to another pool.  It allocates
 * nothing: all of its device buffers are carved out of one static device
 * array of 32 MiB that every device loading this library holds until exit,
 * which bounds n to 16,384 (fewer for very dense boxes; LE_ERR_INVALID_ARG
 * beyond).  The first call in each CUDA context of a device (its primary
 * context, or a new one after a reset) looks the array's address up; make
 * the first call on a device before any stream capture.  Calls share the array, serialise on a lock and
 * return after their device work (on cuda_stream, NULL for the default
 * stream) has finished; work that overlapped a call on the array would race.
 * Errors: LE_ERR_INVALID_ARG, LE_ERR_BOX_TOO_SMALL, LE_ERR_CAPACITY,
 * LE_ERR_NONFINITE, LE_ERR_TIMEOUT (a bounded wait on a bulk copy in the
 * pair kernel gave up), LE_ERR_CUDA. */
LE_API le_status le_forces_noalloc(const double box[3], double shear_rate, double rc, double skin,
                                   const le_params *p, int64_t step, int64_t n, const double *pos,
                                   double *forces, void *cuda_stream);

/* The resort step (Sec. 2.3: particles re-binned into cells; Sec. 3.3: its
 * cost under shear) on its own: a stable least-significant-digit radix sort
 * of n cell keys (host array, each below 2^bits, 1 <= bits <= 32), the same
 * device code a handle runs at every list build.  order (n, host) receives
 * the permutation that sorts the keys, equal keys kept in input order;
 * sorted_keys (n, host, may be NULL) the sorted keys.  Device buffers are
 * allocated and freed inside the call, which returns after its work (on
 * cuda_stream, NULL for the default stream) has finished.  1 <= n <= 2^24.
 * Errors: LE_ERR_INVALID_ARG (sizes, a key of more than `bits` bits),
 * LE_ERR_OOM, LE_ERR_CUDA. */
LE_API le_status le_sort_cell_keys(int64_t n, const uint32_t *keys, int bits, uint32_t *order,
                                   uint32_t *sorted_keys, void *cuda_stream);

/* Measurement aid, not a step of the method: the FP32 arithmetic peak of the
 * CUDA cores of the current device in TFLOP/s, an FMA counted as 2 flops,
 * for scalar FMAs (tflops_fma) and for the paired fma.rn.f32x2 form
 * (tflops_fma2) that the pair kernel uses.  Best of three timed rounds of
 * independent FMA chains on 8 blocks per SM (about 40 GFLOP each, well under
 * a second).  It allocates and frees a small device buffer and synchronises
 * the default stream.  It backs the arithmetic cross-check of the pair
 * kernel, whose roofline is HBM.  Errors: LE_ERR_INVALID_ARG (a NULL
 * output), LE_ERR_CUDA. */
LE_API le_status le_fp32_peak(double *tflops_fma, double *tflops_fma2);

/* Failure-detection self-test, not a step of the method (the paper has no
 * counterpart).  One warp waits, through the same bounded mbarrier wait that
 * the pair kernel uses for its bulk copies of list rows, on a barrier that
 * nothing completes.  The wait gives up after about one second (or 2^22
 * polls, whichever comes first) and the call returns LE_ERR_TIMEOUT, the
 * expected outcome, with the time the probe took in waited_ms (nullable):
 * a copy that never lands in the pair kernel ends as a status the host reads,
 * not as a hang, and the device stays usable.  Work runs on cuda_stream (NULL:
 * the default stream); a small device buffer is allocated and freed inside.
 * LE_OK would mean the wait completed, which cannot happen; LE_ERR_CUDA on a
 * CUDA failure. */
LE_API le_status le_wait_selftest(void *cuda_stream, double *waited_ms);

LE_API le_status le_destroy(le_sim *s);
LE_API const char *le_last_error(const le_sim *s);
LE_API const char *le_status_string(le_status st);

#ifdef __cplusplus
}
#endif
#endif /* LE_H */
