/*
 * sph.h -- C ABI of the GB300 SPH hot path (libsph).
 *
 * The library implements one global time step of the SPH method of
 * Meier, Potter, Reinhardt & Stadel, "Smoothed Particle Hydrodynamics in
 * pkdgrav3 for Shock Physics Simulations. I. Hydrodynamics" (arXiv:2511.11425),
 * for ideal gases without gravity, on one GPU:
 *
 *   sph_build_cells       curve sort + bucket bounds (Sec. 2.1 tree order,
 *                         Sec. 2.3.2 cell bounds and box-of-balls bounds)
 *   sph_density_h         rho_i = sum_j m_j W_ij(h_i) (Eq. Density_estimate) with
 *                         h_i from Newton-Raphson on the constant kernel mass
 *                         4/3 pi h_i^3 rho_i = N_ngb m_i, and the grad-h term
 *                         Omega_i (Sec. 2.3.3)
 *   sph_forces            predictor + ideal-gas EOS (Sec. 2.3.6 step 2,
 *                         Sec. 2.3.1), momentum / PdV / Monaghan viscosity
 *                         equations (Sec. 2.3.5, Eq. AV_heating) and the
 *                         per-particle time-step criteria (Sec. 2.3.6,
 *                         Eq. courant_condition)
 *   sph_kdk_step          closing kick, global step choice, opening kick and
 *                         drift (Sec. 2.3.6 steps 4-5, one global step size)
 *   sph_reduce_conserved  mass, momentum, angular momentum, kinetic and
 *                         internal energy totals
 *
 * Conventions shared by every call
 *   - Pointers inside sph_particles are DEVICE pointers of the current CUDA
 *     device, owned by the caller; each array has n elements (x, v, a are
 *     arrays of three separate component arrays).  The library never frees
 *     them.  sph_build_cells permutes every array of the struct in place
 *     into curve order; `id` travels with the particles so callers can map
 *     back to their own order.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is queued on it; every call returns after a
 *     device-to-host read of the library's status word on that stream, so
 *     a returned SPH_OK means the queued work has completed without a
 *     detected error.
 *   - The context owns all scratch memory (keys, buckets, tree, interaction
 *     lists, staged particle records); it is sized by `capacity` at
 *     sph_create and grown on demand only for interaction lists.
 *   - Errors are status codes; nothing aborts, traps or throws across the
 *     ABI.  sph_last_error returns a human-readable message for the last
 *     non-OK status of a context.
 *   - h is the kernel's support radius: W(r,h) = w(r/h)/h^3 vanishes for r >= h.
 */
#ifndef SPH_H
#define SPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPH_OK = 0,
    SPH_ERR_ARG = 1,        /* invalid argument (NULL pointer, n > capacity, h >= L/2 ...) */
    SPH_ERR_CUDA = 2,       /* a CUDA runtime call failed                                  */
    SPH_ERR_CAPACITY = 3,   /* a fixed-size internal buffer would overflow                 */
    SPH_ERR_NOCONV = 4,     /* Newton iteration on h did not converge within max_newton    */
    SPH_ERR_NONFINITE = 5,  /* a NaN / Inf was produced or found in the inputs             */
                            /* 6 is unused: no kernel of the library waits on another   */
    SPH_ERR_STATE = 7       /* calls made out of order (e.g. forces before density)        */
} sph_status;

/* opaque context: scratch memory, bounds tree, integration state */
typedef struct sph_ctx sph_ctx;

/* smoothing kernels named in Sec. 2.3 (support radius h) */
enum { SPH_KERNEL_WC2 = 0, SPH_KERNEL_WC4 = 1, SPH_KERNEL_WC6 = 2, SPH_KERNEL_M4 = 3 };
/* internal-energy update: PdV equation (Sec. 2.3.5) or entropy-conserving
 * rescale u <- u (rho/rho_old)^(gamma-1) plus viscous heating only */
enum { SPH_ENERGY_PDV = 0, SPH_ENERGY_ISENTROPIC = 1 };
/* space-filling curve that orders the particles into buckets (Sec. 2.1 sorts
 * along a curve so that cells are contiguous; both curves visit the octree
 * cells depth first, the Hilbert curve without jumps between cells) */
enum { SPH_CURVE_HILBERT = 0, SPH_CURVE_MORTON = 1 };
/* arithmetic of the pair sums: the mixed-precision form (FP32 pairs on
 * positions relative to their bucket, FP64 positions and integration) or
 * FP64 throughout the pair sums (the per-particle arrays of sph_particles
 * keep their types in both) */
enum { SPH_PRECISION_MIXED = 0, SPH_PRECISION_FP64 = 1 };
/* the density the forces use (Sec. 2.3.3): the kernel sum (Eq.
 * Density_estimate), or the variant in which rho is state integrated with
 * the mass conservation equation drho/dt = -rho div v.  In the evolved mode
 * the density pass still finds h and Omega (its kernel sum goes to context
 * scratch, not to p->rho); p->rho holds the evolved density between steps,
 * started from the kernel sum by the first density pass of the context;
 * sph_forces uses rho_pred = rho (1 - dt_old/2 div v_old) (the predictor,
 * with the div v of the last force pass) and sph_kdk_step kicks rho with
 * the rate -rho_pred div v like u. */
enum { SPH_DENSITY_SUMMED = 0, SPH_DENSITY_EVOLVED = 1 };

typedef struct {
    int32_t kernel;        /* SPH_KERNEL_*                                       */
    int32_t energy_mode;   /* SPH_ENERGY_*                                       */
    double  n_ngb;         /* target 4/3 pi h^3 rho / m (self included)          */
    double  gamma;         /* ideal-gas adiabatic index                          */
    double  alpha, beta;   /* Monaghan viscosity parameters                      */
    double  eps_av;        /* epsilon of the mu_ij denominator                   */
    double  eta_courant;   /* eta_C of Eq. courant_condition                     */
    double  eta_acc;       /* eta_a of the acceleration criterion                */
    double  box_lo[3];     /* domain; positions on periodic axes stay inside     */
    double  box_hi[3];
    int32_t periodic[3];   /* 1 = periodic axis (minimum image), 0 = open        */
    int32_t max_newton;    /* Newton iteration cap per particle (<= 255)         */
    double  h_rel_tol;     /* error of the reported h relative to the root of the
                              Newton iteration; see sph_density_h              */
    double  list_margin;   /* density lists gather within h (1 + list_margin)    */
    int32_t curve;         /* particle order: SPH_CURVE_HILBERT or SPH_CURVE_MORTON */
    int32_t group_log;     /* buckets per list walk = 2^group_log (1..3); 0 = 3  */
    double  bucket_cell;   /* a bucket stays inside one key cell of side <=
                              bucket_cell h (>= 1; 0 = 3)                        */
    double  group_cell;    /* a walk group stays inside one key cell of side <=
                              group_cell h (>= bucket_cell; 0 = 6)               */
    int32_t resort_period; /* sph_step / graph replays re-sort the particles every
                              resort_period steps and only refit the buckets'
                              bounds to the moved particles in between (1..64;
                              0 = 1); taken from the first instance of a batch  */
    int32_t precision;     /* SPH_PRECISION_MIXED (0, default): FP32 pair
                              arithmetic on cell-relative offsets with compensated
                              sums; SPH_PRECISION_FP64: every pair sum, the h
                              iteration and the force accumulators in FP64 (the
                              plain form); must agree across a batch            */
    int32_t density_mode;  /* SPH_DENSITY_SUMMED (0, default): rho from the kernel
                              sum; SPH_DENSITY_EVOLVED: rho integrated with the
                              mass conservation equation (needs SPH_ENERGY_PDV);
                              must agree across a batch                         */
    int32_t interface_correction; /* 1: the interface correction of Sec. 2.3.4
                              (mixed precision, summed density; must agree
                              across a batch); 0: off                         */
    double  ic_alpha;      /* normalisation of the kernel imbalance (Eq.
                              Kernel_imbalance); 0 = the kernel's own value, at
                              which a particle on a flat interface between two
                              uniform materials has I = 1                     */
    double  r_gas[4];      /* gas constant of materials 0..3 (ideal gases with
                              the instance's gamma: T = (gamma-1) u / R,
                              rho = P / (R T)); used by the interface correction */
} sph_params;

typedef struct {
    int64_t   n;           /* number of particles                                */
    double   *x[3];        /* positions x_i (FP64)                               */
    double   *v[3];        /* velocities v_{i-1/2} between steps (FP64)          */
    double   *u;           /* specific internal energy u_{i-1/2} (FP64)          */
    float    *m;           /* masses                                             */
    float    *h;           /* smoothing length (support radius); input seed,     */
                           /* output of sph_density_h                            */
    float    *rho;         /* density (output of sph_density_h)                  */
    float    *omega;       /* grad-h term Omega (output of sph_density_h)        */
    float    *a[3];        /* acceleration a_i (output of sph_forces)            */
    float    *dudt_h;      /* du/dt|H, PdV term (output of sph_forces)           */
    float    *dudt_av;     /* du/dt|Pi, viscous heating (output of sph_forces)   */
    float    *divv;        /* velocity divergence (output of sph_forces)         */
    float    *dt_i;        /* per-particle time-step limit (output of sph_forces)*/
    uint16_t *nngb;        /* neighbours j != i with r_ij < h_i (sph_density_h)  */
    uint8_t  *iters;       /* Newton iterations taken (sph_density_h)            */
    int64_t  *id;          /* caller's particle ids, permuted with the particles */
    uint8_t  *mat;         /* material of each particle (index into
                              sph_params.r_gas), permuted with the particles;
                              read only with the interface correction on (may
                              be NULL otherwise)                               */
} sph_particles;

/* Host-side view of the same state for sph_step_host: HOST pointers, same
 * layout and meaning as sph_particles. */
typedef sph_particles sph_host_particles;

/* phases timed per launch group while sph_set_profiling is on (index into
 * sph_stats.phase_ms / phase_launches) */
enum {
    SPH_PHASE_KEYS = 0,      /* bounding boxes + curve keys                       */
    SPH_PHASE_SORT = 1,      /* radix-sort passes                                 */
    SPH_PHASE_PERMUTE = 2,   /* gather + copy-back of every particle array        */
    SPH_PHASE_LAYOUT = 3,    /* bucket layout scan                                */
    SPH_PHASE_BUCKETS = 4,   /* bucket origins, relative positions, leaf bounds   */
    SPH_PHASE_TREE = 5,      /* bottom-up bounds refit                            */
    SPH_PHASE_BOB_REFIT = 6, /* box-of-balls refresh after the density pass       */
    SPH_PHASE_WALK = 7,      /* interaction-list walks                            */
    SPH_PHASE_DENSITY = 8,   /* Newton kernel (all passes, re-walk rounds)        */
    SPH_PHASE_PREDICT = 9,   /* predictor + EOS                                   */
    SPH_PHASE_FORCES = 10,   /* pair-force kernel                                 */
    SPH_PHASE_FINALIZE = 11, /* finalize sums, time-step limits                   */
    SPH_PHASE_KDK = 12,      /* step choice, kicks and drift                      */
    SPH_PHASE_CONSERVED = 13,/* conserved totals                                  */
    SPH_PHASE_COUNT = 14
};

typedef struct {
    uint64_t density_pairs;      /* sum over Newton passes of sum_i n_i (last density call) */
    uint64_t force_pairs;        /* unordered pairs with r < max(h_i,h_j) (last force call)  */
    uint64_t density_candidates; /* candidate pair tests in the density pass                 */
    uint64_t force_candidates;   /* candidate pair tests in the force pass                   */
    int32_t  max_newton_iters;   /* largest Newton iteration count of the last density call  */
    int32_t  relists;            /* buckets re-walked because h left the list margin         */
    int64_t  list_entries_density; /* source buckets in the density lists                    */
    int64_t  list_entries_force;   /* source buckets in the force lists                      */
    double   dt_old;             /* step size of the last sph_kdk_step (0 before the first)  */
    float    ms_build, ms_density, ms_forces, ms_kdk; /* last call durations (CUDA events)    */
    float    ms_walk;            /* interaction-list walks of the last density + force calls */
    float    ms_density_kernel;  /* Newton kernel alone, all passes of the last density call */
    float    ms_force_kernel;    /* pair-force kernel alone, last force call                 */
    int32_t  pad_;
    uint64_t force_av_pairs;     /* pairs of the last force call with v_ij.r_ij < 0          */
    uint64_t launches;           /* kernels launched by this context since sph_create        */
    double   phase_ms[16];       /* per SPH_PHASE_*: device time accumulated while profiling */
    uint64_t phase_launches[16]; /* per SPH_PHASE_*: timed launch groups                     */
} sph_stats;

/*
 * sph_create: allocate a context for up to `capacity` particles on the current
 * CUDA device.  `params` is copied.  Fails with SPH_ERR_ARG for capacity < 0,
 * an unknown kernel, gamma <= 1, n_ngb <= 0, an empty box or max_newton not in
 * [1,255]; SPH_ERR_CUDA if device memory cannot be allocated.
 * On success *out receives the context (caller destroys it with sph_destroy).
 */
sph_status sph_create(const sph_params *params, int64_t capacity, sph_ctx **out);

/*
 * sph_batch_create: a context for `ninst` INDEPENDENT problems stepped
 * together (the batched form): instance k owns particles
 * [offsets[k], offsets[k+1]) of every array (offsets: host array of ninst+1,
 * offsets[0] = 0), has its own box, periodicity, gamma, viscosity parameters
 * and time step, and never interacts with another instance.  Every phase is
 * one kernel launch over all instances.  params: host array of ninst structs;
 * kernel, energy_mode, max_newton, h_rel_tol and list_margin must agree
 * (SPH_ERR_ARG otherwise).  All calls below accept a batch context with
 * p->n = offsets[ninst]; sph_kdk_step's dt_used reports instance 0 (all steps:
 * sph_batch_get_dt), sph_reduce_conserved writes 9 totals per instance.
 */
sph_status sph_batch_create(const sph_params *params, int32_t ninst, const int64_t *offsets,
                            sph_ctx **out);

/* sph_destroy: free the context and its device memory (NULL is ignored). */
void sph_destroy(sph_ctx *ctx);

/*
 * sph_build_cells (Sec. 2.1: particles reordered so that cells are contiguous;
 * Sec. 2.3.2: cell bound and box-of-balls bound per cell).  Computes
 * space-filling-curve keys of x (per instance: the box cut into near-cubes
 * in snake order, params.curve inside each cube, 30 bits), stably sorts
 * them, permutes EVERY array of *p in place, cuts the order into buckets of
 * at most 32 consecutive particles that stay inside one key cell of side
 * <= bucket_cell h (walk groups inside one of side <= group_cell h) and
 * builds the bounds tree over the buckets from x and the current h.  Positions on
 * periodic axes must lie in [box_lo, box_hi).  SPH_ERR_ARG if p->n > capacity
 * or a required pointer is NULL; SPH_ERR_NONFINITE for non-finite x or h.
 */
sph_status sph_build_cells(sph_ctx *ctx, sph_particles *p, void *stream);

/*
 * sph_density_h (Sec. 2.3.3).  For every particle solves
 * 4/3 pi h^3 rho(h) = N_ngb m by Newton-Raphson with a bisection safeguard,
 * starting from h_seed (device array of n floats, curve order) or, if
 * h_seed is NULL, from p->h.  Writes p->h, p->rho, p->omega, p->nngb,
 * p->iters; h is the Newton update h + dh of the last evaluation.  Newton
 * converges quadratically: that update lies |g''/(2 g')| dh^2 from the root
 * (g'' from the same kernel sums), and the iteration ends once this is below
 * h_rel_tol h with |dh| < sqrt(h_rel_tol) h (at most 1e-2 h), or once
 * |dh| < h_rel_tol h.  rho, Omega and nngb are reported at the updated h
 * (the evaluated sums moved to first order in dh, nngb counted from the
 * hits within sqrt(h_rel_tol) h of the support radius).  With the interface correction
 * on, the step itself must be below h_rel_tol h and rho, Omega and nngb are
 * those of the evaluated h.  In SPH_ENERGY_ISENTROPIC mode it also moves u along its adiabat
 * to the new density, u <- u (rho/rho_old)^(gamma-1), using the rho left in
 * p->rho by the previous call.  Then refreshes the box-of-balls bounds with
 * the new h (Sec. 2.3.3, bounds updated after the density pass).
 * Requires sph_build_cells since the last change of positions
 * (SPH_ERR_STATE otherwise).  SPH_ERR_NOCONV if a particle needs more than
 * max_newton iterations; SPH_ERR_ARG if a converged h reaches half a
 * periodic box length.
 */
sph_status sph_density_h(sph_ctx *ctx, sph_particles *p, const float *h_seed, void *stream);

/*
 * sph_density_at: rho, Omega and the neighbour count at the GIVEN h (device
 * array, curve order), without iterating; optionally lists neighbour ids.
 * When ids != NULL it must hold n*cap int64 and receives, for particle i, the
 * `id` values of its neighbours j != i (r_ij < h_i) in slots [i*cap, i*cap+cap);
 * count[i] (device uint32, may be NULL) receives the full count even when it
 * exceeds cap.  Outputs rho, omega and nngb go to *p.  Test and diagnostic
 * entry point for neighbour-set checks.
 */
sph_status sph_density_at(sph_ctx *ctx, sph_particles *p, const float *h, int64_t cap,
                          uint32_t *count, int64_t *ids, void *stream);

/*
 * sph_forces (Sec. 2.3.5, 2.3.6).  Predicts v, u to the current time with the
 * previous derivatives and half the previous step (step 2 of the substep),
 * evaluates P = (gamma-1) rho u and c, then accumulates over every unordered
 * pair with r_ij < max(h_i, h_j), each pair evaluated once with equal and
 * opposite contributions: the pressure acceleration (gather + scatter
 * terms), du/dt|H, the Monaghan viscosity (acceleration and heating, averaged
 * kernel), div v, and the Courant limit.  Writes p->a, p->dudt_h,
 * p->dudt_av, p->divv, p->dt_i (= min(eta_a sqrt(h/|a|), Courant limit)).
 * Requires sph_density_h since sph_build_cells (SPH_ERR_STATE otherwise).
 */
sph_status sph_forces(sph_ctx *ctx, sph_particles *p, void *stream);

/*
 * sph_kdk_step (Sec. 2.3.6 steps 4-5 with one global step size).  Closing
 * kick of v and u over half the previous step with a and du/dt from
 * sph_forces; new step = dt_fixed if dt_fixed > 0, else min_i dt_i (device
 * reduction); opening kick over half the new step; drift x over the new
 * step; periodic wrap.  The smoothing length is advanced with the drift,
 * h <- h exp(dt div v / 3) (continuity equation, factor clamped to [1/2, 2]),
 * so p->h holds the seed of the next density pass.  If dt_used != NULL the
 * new step is written there
 * (this needs no extra synchronisation: every call already waits for its
 * status).  Positions change, so the next sph_density_h needs
 * sph_build_cells first.
 */
sph_status sph_kdk_step(sph_ctx *ctx, sph_particles *p, double dt_fixed, double *dt_used,
                        void *stream);

/*
 * sph_step: one whole step = sph_build_cells, sph_density_h (seeded with the
 * current h), sph_forces, sph_kdk_step.  Same arguments and errors.  With
 * params.resort_period = k > 1 only every k-th step re-sorts; the steps in
 * between keep the buckets and refit their bounds to the moved particles
 * (the results are the same up to summation order).
 */
sph_status sph_step(sph_ctx *ctx, sph_particles *p, double dt_fixed, double *dt_used,
                    void *stream);

/*
 * sph_step_rungs: one global step dt0 with hierarchical power-of-two time
 * steps (Sec. 2.3.6, Time integration).  The step is cut into 2^max_rung
 * substeps of dt0 / 2^max_rung; a particle on rung r steps 2^(max_rung - r)
 * substeps at a time and is active on the substeps that its period
 * divides.  Every substep runs the density pass, predicts
 * every particle's v and u to the substep time (v + (tau - T/2) a, tau the
 * time since its last step boundary, T its period; v, u are half-step
 * values), evaluates the forces (all pairs that have an active particle take
 * effect: inactive particles keep their derivatives), kicks the active
 * particles (closing kick over T/2, new rung r = ceil(log2(dt0 / dt_i))
 * clamped to [0, max_rung] and raised to (largest rung of the particle's
 * force partners) - 2, a lower rung only to one whose period divides the
 * substep, opening kick over half the new period) and drifts every particle.
 * Rungs start at 0 and persist across calls (sph_get_rungs reads them, in
 * the particles' current order); a run uses one max_rung (SPH_ERR_STATE
 * otherwise) and either only hierarchical or only global steps
 * (sph_set_dt_old(ctx, 0) does not reset the rungs).  The first substep
 * re-sorts the particles, the others refit the bounds.  Mixed precision and
 * summed density only (SPH_ERR_ARG); not with the learned seed
 * (SPH_ERR_STATE).  A failed substep leaves x, v, u as they were after the
 * substeps before it.  Synchronous (one status read at the end).
 * FastGas (on by default, sph_set_fastgas): after each substep's density
 * walk the groups holding an active particle or a listed neighbour of one
 * are marked (from the density lists, both directions), and the density
 * pass, the force walk and the force pass run over the marked groups only;
 * the other particles keep h, rho and Omega of their last pass.  Off, every
 * substep solves every particle's density and sums every pair.
 */
sph_status sph_step_rungs(sph_ctx *ctx, sph_particles *p, double dt0, int32_t max_rung,
                          void *stream);

/* sph_set_fastgas: on != 0 restricts the substeps of sph_step_rungs to the
 * active particles' neighbourhoods (FastGas, Sec. 2.3.6); 0 solves every
 * particle on every substep.  Takes effect at the next call. */
sph_status sph_set_fastgas(sph_ctx *ctx, int32_t on);

/* sph_get_rungs: rung of each of the first n particles (HOST array, current
 * particle order); zeros before the first sph_step_rungs.  Synchronous. */
sph_status sph_get_rungs(sph_ctx *ctx, uint8_t *out, int64_t n);

/*
 * sph_step_host: sph_step on HOST arrays.  Copies the arrays a step reads
 * (x, v, u, m, h, a, dudt_h, dudt_av, id, and rho in SPH_ENERGY_ISENTROPIC
 * mode) to device buffers owned by the context (allocated on first use for
 * the context's capacity), runs the step there and copies every array it
 * changes back (in curve order, like sph_step).  If sph_step_host_capture
 * recorded a step for this context with the same dt_fixed and n, the step is
 * that graph's replay (as sph_graph_launch), else sph_step.
 * Memory: host arrays may be pageable or pinned and must hold n elements.
 * Pinned arrays that the GPU can address are read and written by one copy
 * kernel per direction (all such arrays in one launch), the others by
 * cudaMemcpyAsync.
 * Overlap: the inputs no kernel reads before the end of the density phase
 * (v, u, a, dudt_h, dudt_av) are copied by the copy engines on a stream of
 * the context while the step's first phases run (in a step that re-sorts,
 * before it: the re-sort permutes every array).  In a replay, the density
 * and force outputs are copied back while the rest of the step runs; a
 * replay that only refits neither reads id nor changes m and id, so id is
 * not copied in and m and id are not copied back.  On an error status of a
 * replay the host arrays hold what the failed step left (x, v, u as they
 * were).
 * h2d_bytes / d2h_bytes (when non-NULL) receive the bytes copied in and out.
 */
sph_status sph_step_host(sph_ctx *ctx, sph_host_particles *hp, double dt_fixed, double *dt_used,
                         int64_t *h2d_bytes, int64_t *d2h_bytes, void *stream);

/*
 * sph_step_host_capture (no counterpart in the paper, like sph_step_host):
 * copy the step inputs of *hp into the context's
 * device buffers and record one step on them as sph_graph_capture does
 * (same rules: non-default stream, finite dt_fixed, isentropic mode after
 * one plain step); later sph_step_host calls with this dt_fixed and n
 * replay it.  *hp is not modified.  Replaces any graph the context held.
 */
sph_status sph_step_host_capture(sph_ctx *ctx, sph_host_particles *hp, double dt_fixed,
                                 void *stream);

/*
 * sph_reduce_conserved: out[9k .. 9k+8] = M, P_x, P_y, P_z, L_x, L_y, L_z,
 * E_kin, E_int of instance k (one instance unless the context is a batch),
 * from m, x, v, u of *p, summed in FP64 in a fixed order (bit-identical from
 * run to run).  out is a HOST array of 9 doubles per instance.
 */
sph_status sph_reduce_conserved(sph_ctx *ctx, const sph_particles *p, double *out, void *stream);

/*
 * sph_graph_capture: record one whole sph_step (build, density with its
 * re-walk rounds, forces, kick-drift-kick and the status read-back) on
 * `stream` into a CUDA graph owned by the context, without running it.  The
 * graph is bound to the arrays of *p and to dt_fixed; stream must not be the
 * legacy default stream.  In SPH_ENERGY_ISENTROPIC mode capture after one
 * plain sph_step, so the previous density exists.  A new capture replaces
 * the old graph.
 * The graph also reduces the conserved totals of the stepped state (as
 * sph_reduce_conserved).  With resort_period > 1 a second graph (refit
 * instead of re-sort) is captured and replays follow sph_step's schedule.
 * sph_graph_launch: replay the captured step on `stream`, wait, and report
 * the status like sph_step (dt_used: new step of instance 0, may be NULL).
 * sph_graph_totals: the totals of the last successful replay (HOST array of 9
 * doubles per instance); SPH_ERR_STATE before the first replay.
 */
sph_status sph_graph_capture(sph_ctx *ctx, sph_particles *p, double dt_fixed, void *stream);
sph_status sph_graph_launch(sph_ctx *ctx, double *dt_used, void *stream);
sph_status sph_graph_totals(const sph_ctx *ctx, double *out);

/* sph_batch_get_dt: the step size each instance used in the last
 * kick-drift-kick (host array of one double per instance). */
sph_status sph_batch_get_dt(const sph_ctx *ctx, double *out);

/*
 * sph_reduce_conserved_noalloc: the totals of sph_reduce_conserved without a
 * context and without allocating device memory.  The paper has no
 * counterpart; this entry point exists for callers that cannot call
 * cudaMalloc: applications whose pool allocator owns all device memory, hooks
 * that run inside another library's time step (where an allocation would
 * synchronise the device or fail under memory pressure), code that must keep
 * the process's device footprint fixed.
 *   p      device arrays x, v, u, m of p->n particles (other members ignored)
 *   out    DEVICE array of 9 doubles owned by the caller; receives M, P_x,
 *          P_y, P_z, L_x, L_y, L_z, E_kin, E_int (fixed summation order)
 *   stream cudaStream_t as void*; the call only queues work and returns, so
 *          synchronise the stream before reading out
 * Partial sums live in a fixed file-scope device array of 576 KiB that every
 * GPU loading the library keeps until exit; n is therefore limited to
 * 8,388,608 particles and larger n returns SPH_ERR_CAPACITY without launching.
 * The array's device address is looked up in the CUDA context current at
 * the call (afresh on every call whose stream is not being captured, and
 * cached per context for calls made during a stream capture): make the first
 * call in each context before any stream capture.  All calls on a device
 * share the array: calls that overlap on the GPU race and give wrong totals.
 * n = 0 writes nine zeros to out.
 * Errors: SPH_ERR_ARG (NULL pointer, n < 0); SPH_ERR_CAPACITY (n > 8,388,608,
 * nothing launched); SPH_ERR_CUDA (a CUDA error was already pending from the
 * caller's earlier work: it is left pending and nothing is launched; or the
 * address lookup or a launch of this call failed; or the first call in a
 * context was made during a stream capture).  There is no context, so
 * sph_last_error does not apply.
 */
sph_status sph_reduce_conserved_noalloc(const sph_particles *p, double *out, void *stream);

/* ---- learned smoothing-length seed --------------------------------------
 * The Newton iteration for h (Sec. 2.3.3) needs a starting value; the paper
 * does not say where it starts.  By default sph_kdk_step leaves each
 * particle's h at the continuity estimate h exp(dt divv / 3).  The paper has
 * no counterpart for the alternative below: a 4-32-32-1 ReLU network, run
 * on the tensor cores with bfloat16 weights and FP32 accumulation inside the
 * kick-drift-kick, proposes a correction y, and
 *     h_seed = h exp(phi0 + y / 100), factor clamped to [1/2, 2],
 * except where |phi0| and |phi2| are both below h_rel_tol (the last seed was
 * within the Newton tolerance and the continuity estimate moves h by less)
 * or where |y| / 100 is below the root-mean-square residual of the last
 * training call (the network's own fit error): there y is not applied.
 * The iteration still runs to h_rel_tol from that seed, so the converged h
 * does not depend on the network.
 * Features of particle i at the end of a step (dt = new step, dt_old = last):
 *     phi0 = dt divv_i / 3,  phi1 = nngb_i / n_ngb - 1,
 *     phi2 = ln(h_i / seed_i) (seed_i = start of this step's iteration),
 *     phi3 = ln(dt / dt_old) (0 on the first step);
 * network inputs x = (100 phi0, 4 phi1, 100 phi2, 10 phi3).  Training
 * samples (x, y*) pair the inputs with y* = 100 (ln(h_new / h) - phi0),
 * h_new being what the next density pass converges to.
 * Parameters: SPH_MLP_NPARAM floats in the order W1 (32 x 4, row-major by
 * hidden unit), b1 (32), W2 (32 x 32), b2 (32), W3 (32), b3 (1); the master
 * copy is FP32, the inference copy bfloat16 (round to nearest even).  One
 * network per context (shared by the instances of a batch).
 */
#define SPH_MLP_NPARAM 1249
enum { SPH_SEED_ANALYTIC = 0, SPH_SEED_MLP = 1 };

/* sph_mlp_set_weights / sph_mlp_get_weights: copy the FP32 master
 * parameters from / to a HOST array of count == SPH_MLP_NPARAM floats
 * (SPH_ERR_ARG otherwise).  Setting resets the Adam moments and step count
 * and refreshes the bfloat16 copy.  Both synchronise the device. */
sph_status sph_mlp_set_weights(sph_ctx *ctx, const float *w, int64_t count);
sph_status sph_mlp_get_weights(sph_ctx *ctx, float *w, int64_t count);

/* sph_mlp_set_seed_mode: SPH_SEED_ANALYTIC (default) or SPH_SEED_MLP for
 * the seeds written by later kick-drift-kick steps (a captured graph keeps
 * the mode it was captured with). */
sph_status sph_mlp_set_seed_mode(sph_ctx *ctx, int32_t mode);

/* sph_mlp_record: on != 0 starts collecting training samples from the
 * steps that follow: every kick-drift-kick stores the inputs x of its
 * particles (they move with the particles), and the next density pass turns
 * those particles whose hash of (index, step) is 0 modulo `stride` into
 * samples.  Samples whose |ln(h_new / h)| exceeds ln 2 are skipped.  The
 * device ring buffer holds `capacity` samples (the oldest are overwritten);
 * it is allocated here (synchronous).  on == 0 stops recording and keeps the
 * samples.  SPH_ERR_ARG for capacity < 1 or stride < 1 when on != 0. */
sph_status sph_mlp_record(sph_ctx *ctx, int32_t on, int64_t capacity, int32_t stride);

/* sph_mlp_samples: number of samples held (synchronises the device). */
sph_status sph_mlp_samples(sph_ctx *ctx, int64_t *count);

/* sph_mlp_get_samples: copy the first n samples held into HOST arrays x
 * (n x 4 floats) and y (n floats); SPH_ERR_ARG if fewer are held.  The ring
 * buffer keeps no order beyond the slots the recording passes wrote. */
sph_status sph_mlp_get_samples(sph_ctx *ctx, float *x, float *y, int64_t n);

/* sph_mlp_load_samples: replace the samples by n DEVICE pairs: x (n x 4
 * floats, row-major), y (n floats).  The buffer grows to n if needed. */
sph_status sph_mlp_load_samples(sph_ctx *ctx, const float *x, const float *y, int64_t n,
                                void *stream);

/* sph_mlp_train: `iters` Adam steps (beta1 0.9, beta2 0.999, eps 1e-8,
 * learning rate lr) on the mean squared error over minibatches of `batch`
 * samples drawn uniformly with replacement from the samples held (counter-
 * based SplitMix64 on seed); batch <= 0 or >= the number held takes every
 * sample in order (full batch).  Gradients come from FP32 forward and
 * backward kernels and are summed in a fixed order.  Refreshes the bfloat16
 * copy at the end and synchronises; loss_first / loss_last (HOST, may be
 * NULL) receive the minibatch loss of the first and the last step, and
 * sqrt(last loss) / 100 becomes the dead zone of the correction
 * (sph_mlp_set_weights resets it to 0).
 * SPH_ERR_STATE when no samples are held. */
sph_status sph_mlp_train(sph_ctx *ctx, int32_t iters, int32_t batch, double lr, uint64_t seed,
                         double *loss_first, double *loss_last, void *stream);

/* sph_mlp_grad: mean squared error of the FP32 master network over n DEVICE
 * samples (x: n x 4 floats row-major, y: n floats) and its gradient, into
 * HOST arrays grad (SPH_MLP_NPARAM floats) and loss (1 double); sums in a
 * fixed order, synchronous.  Changes no state. */
sph_status sph_mlp_grad(sph_ctx *ctx, const float *x, const float *y, int64_t n, float *grad,
                        double *loss, void *stream);

/* sph_mlp_infer: network outputs y (n DEVICE floats) for inputs x (n x 4
 * DEVICE floats, row-major) through the bfloat16 tensor-core path the seed
 * uses.  Asynchronous on stream. */
sph_status sph_mlp_infer(sph_ctx *ctx, const float *x, int64_t n, float *y, void *stream);

/* sph_bucket_layout: the bucket slots of the last sph_build_cells, for
 * inspection.  Slot b holds particles [first[b], first[b + 1]) (in the order
 * sph_build_cells left them; an empty range is a padding slot); slots of
 * instance k are contiguous, groups are runs of 2^group_log slots.  first
 * is a HOST array of cap entries; *nslots receives the number of slots
 * (first needs nslots + 1 entries, SPH_ERR_ARG otherwise).  Synchronous.
 * The paper has no counterpart (it is a view of the data layout). */
sph_status sph_bucket_layout(sph_ctx *ctx, int32_t *first, int64_t cap, int64_t *nslots);

/* sph_set_list_arena: size of the shared overflow arena that holds the
 * interaction lists of walk groups whose lists outgrow their 1024 fixed slots
 * (a group whose h spans most of its problem: a very heavy particle, one
 * leaving a free surface).  The default is max(2^23, 16 x groups) entries of
 * 4 bytes.  A walk that finds the arena full fails the call with
 * SPH_ERR_CAPACITY (a failed step leaves x, v, u as they were); a larger arena
 * lets such problems run, a smaller one caps the memory.  Shrinking only
 * lowers the limit; growing past the allocated size reallocates the list
 * buffer (synchronous) and drops a step recorded by sph_graph_capture or
 * sph_step_host_capture (record it again).  SPH_ERR_ARG for entries < 0,
 * SPH_ERR_CAPACITY if the lists would pass 2^32 entries.  The paper has no
 * counterpart (it is a memory-budget setting of this library). */
sph_status sph_set_list_arena(sph_ctx *ctx, int64_t entries);

/* sph_set_profiling: on != 0 starts timing every phase of the calls that
 * follow (CUDA events around each launch group of a plain call; steps
 * replayed from a captured graph and calls made during a capture are not
 * timed) and clears the accumulated times in sph_stats.phase_ms; on == 0
 * stops.  Costs two event records per launch group.  The paper has no
 * counterpart (instrumentation of this library). */
sph_status sph_set_profiling(sph_ctx *ctx, int32_t on);

/* sph_set_dt_old: set the previous step size used by the predictor and the
 * closing kick (0 restarts the integration as at t = 0). */
sph_status sph_set_dt_old(sph_ctx *ctx, double dt_old);

/* sph_get_stats: counters and timings of the last calls (host struct). */
sph_status sph_get_stats(const sph_ctx *ctx, sph_stats *out);

/* sph_last_error: message of the last non-OK status ("" if none); the
 * string is owned by the context. */
const char *sph_last_error(const sph_ctx *ctx);

/* sph_version: library version string. */
const char *sph_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SPH_H */
