/*
 * steps.h -- C ABI of libsteps, a GB300 (sm_103a) direct-summation gravity
 * engine for StePS-style compactified N-body simulations (Racz, Szapudi,
 * Dobos, Csabai & Szalay, "StePS: A Multi-GPU Cosmological N-body Code for
 * Compactified Simulations").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Units are the caller's; G is taken from steps_config.  H0 and time share
 *    one unit (the Friedmann equation, Eq. 1, is evaluated as written).
 *  - Arrays of 3-vectors are row-major [n][3] float64.  Scalars are float64.
 *  - Any array argument may be a host pointer or a device pointer on the
 *    context's device; the library classifies it with cudaPointerGetAttributes
 *    and copies as needed.  The caller keeps ownership of every buffer it
 *    passes; the library copies inputs before the call returns.
 *  - Particle order at the boundary is always the caller's order.  The
 *    library keeps its state spatially sorted internally; the permutation
 *    never leaks.
 *  - Every entry point returns a steps_status and never aborts.  On failure
 *    steps_last_error() returns a thread-local, human-readable reason.
 *  - Work is issued on the stream given at steps_init.  With NULL the context
 *    creates and owns a private non-blocking stream.  Calls that return data
 *    (forces, state, diagnostics, checkpoints) synchronise that stream before
 *    returning; steps_kdk_step without a_out and steps_kdk_run's graph
 *    replays are asynchronous until the next synchronising call.
 */
#ifndef STEPS_H
#define STEPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    STEPS_OK = 0,
    STEPS_EINVAL = 1,       /* bad argument: NULL where required, n <= 0, non-finite input, h <= 0 */
    STEPS_ENOMEM = 2,       /* device allocation failed or exceeds the context's cap */
    STEPS_ECUDA = 3,        /* a CUDA runtime call failed; see steps_last_error() */
    STEPS_ETIMEOUT = 4,     /* a bounded device-side wait ran out; the kernel exited cleanly */
    STEPS_ENONFINITE = 5,   /* a result contained NaN or Inf */
    STEPS_EUNSUPPORTED = 6  /* option not built into this library */
} steps_status;

typedef enum {
    STEPS_STATIC = 0,   /* static, non-comoving Newtonian background (the paper's proper-coordinate mode) */
    STEPS_COMOVING = 1, /* spherical comoving equation of motion, Eq. 8 */
    STEPS_COMOVING_REVERSED = 2, /* Eq. 8 with gravity reversed, as for relaxing a glass (Sec. 3.1): the
                                   pair term and the background term both change sign, so a uniform
                                   sphere stays in equilibrium; a(t) still follows Eq. 1 (an
                                   Einstein-de Sitter background: Om = 1, OL = 0).  Single
                                   simulations only; steps_forces then returns the repulsive term. */
    STEPS_PERIODIC = 3  /* periodic comoving equation of motion, Eq. 2: pair term / a^3 - 2 H v with
                           the image sum of Eq. 5 in a cubic box of side `box` (every image n with
                           |x_i - x_j - nL| < 2.6 L, or with images = 1 only the leading one, the n
                           with x_i - x_j - nL in [-L/2, L/2)^3); positions are wrapped into
                           [0, L)^3.  STEPS_F32_COMP or STEPS_F64 only; single simulations only;
                           steps_forces_subset and the potential energy are not available. */
} steps_mode;

typedef enum {
    STEPS_F32_COMP = 0,  /* FP32 pair arithmetic, tile-relative coordinates, compensated per-target sums */
    STEPS_F32_NAIVE = 1, /* FP32 pair arithmetic, one plain FP32 running sum per target */
    STEPS_F64 = 2        /* FP64 pair arithmetic and sums on the GPU */
} steps_prec;

typedef struct {
    double G;                 /* gravitational constant */
    double H0;                /* Hubble constant (1/time unit) */
    double Om, OL, Or, Ok;    /* density parameters of Eq. 1 (present-day values) */
    int mode;                 /* steps_mode */
    int prec;                 /* steps_prec */
    int resort_every;         /* re-sort particles spatially every this many steps (<=0: default 8) */
    int tile_override;        /* 0 = autotuned force-kernel variant (STEPS_PERIODIC: 64-particle tiles,
                                 not tuned); k>0 selects variant k-1 (its tile size in periodic mode) */
    double box;               /* STEPS_PERIODIC: side L of the periodic box */
    int images;               /* STEPS_PERIODIC: 0 = image sum cut at 2.6 L (Eq. 5), 1 = quasi-periodic */
} steps_config;

typedef struct steps_ctx steps_ctx;

/* Default configuration: G = H0 = 1, Om = 0.3, OL = 0.7, static mode, STEPS_F32_COMP. */
steps_config steps_default_config(void);

/*
 * steps_init -- create a simulation context holding n particles on the
 * current CUDA device.
 *   pos  [n][3]  positions (comoving in STEPS_COMOVING mode)
 *   vel  [n][3]  velocities dx/dt (NULL = zero)
 *   mass [n]     particle masses, > 0
 *   soft [n]     per-particle softening lengths h_i (> 0), or NULL to derive
 *                them from the masses by Eq. 7, h_i = (m_i/m_min)^(1/3) h_min
 *   h_min        softening of the lightest particle; used only when soft == NULL
 *   t0, a0       initial cosmic time and scale factor (a0 ignored in static mode)
 *   cfg          configuration (NULL = steps_default_config())
 *   cuda_stream  cudaStream_t to issue work on (NULL = a private stream)
 * Each pair (i, j) uses the softening support h_i + h_j (Eq. 2, Eq. 8).
 * The pair term at the initial positions is computed before returning.
 * Errors: EINVAL (n <= 0, NULL pos/mass/out, non-finite values, m <= 0,
 * h <= 0), ENOMEM, ECUDA.  On error *out is set to NULL.
 */
steps_status steps_init(steps_ctx **out, int64_t n, const double *pos, const double *vel,
                        const double *mass, const double *soft, double h_min, double t0,
                        double a0, const steps_config *cfg, void *cuda_stream);

/*
 * steps_forces -- evaluate the softened pair term of Eq. 8 at the current
 * positions (Eq. 3 with the spline kernel of Eq. 4, summed over all j != i):
 *   acc_i = -G sum_{j != i} m_j F(|x_i - x_j|, h_i + h_j) (x_i - x_j)/|x_i - x_j|
 * i.e. the pair acceleration before the 1/a^3 factor, in the precision chosen
 * by cfg.prec.  acc_out [n][3] (host or device, caller order) may be NULL, in
 * which case the result only refreshes the context's stored acceleration.
 */
steps_status steps_forces(steps_ctx *ctx, double *acc_out);

/*
 * steps_kdk_step -- advance one kick-drift-kick step of length dt
 * (Eq. 9-11, one force evaluation per step).  In STEPS_COMOVING mode each
 * half-kick applies A = acc/a^3 - 2 (adot/a) v + (4 pi G/3) Om rho_crit x / a^3
 * (Eq. 8; rho_crit = 3 H0^2/(8 pi G)), with a and adot/a taken at that
 * half-kick's time point and v at kick entry; a(t) advances by one RK4 step
 * of Eq. 1 with the same dt.  In STEPS_STATIC mode A = acc.
 * a_out (host, may be NULL) receives the new scale factor; passing it
 * synchronises the stream.  All state stays on the device (FP64).
 */
steps_status steps_kdk_step(steps_ctx *ctx, double dt, double *a_out);

/*
 * steps_kdk_run -- nsteps KDK steps with per-step lengths dts[nsteps] (host
 * array), issued as a replayed CUDA graph.  Equivalent to calling
 * steps_kdk_step for each dts[k], bit for bit.
 */
steps_status steps_kdk_run(steps_ctx *ctx, int nsteps, const double *dts);

/*
 * Eq. 12 (Sec. 2.3): adaptive step length of the KDK integrator,
 *   dt = min(dt_max, min_i sqrt(2 eta_i eps / |A_i|)),   eta_i = 2.8 h_i,
 * with eps the accuracy parameter and A_i the acceleration the next kick
 * applies at the current state (comoving mode: the pair term / a^3 - 2 H v +
 * the background term of Eq. 8; static mode: the pair term).  A particle with
 * A_i = 0 sets no limit.  When t_end is finite the step is also limited to
 * t_end - t (never below 0); pass +INFINITY for no limit.  eta_i = 2.8 h_i is
 * taken as printed (the paper calls it the Plummer-equivalent softening; the
 * spline's own Plummer equivalent is h_i / 2.8, which is the same criterion
 * with eps divided by 7.84).
 * steps_timestep computes dt on the device from the forces of the last
 * evaluation, makes it the length of the next device-resident step and, if
 * dt_out is not NULL, synchronises and returns it (the caller then passes it
 * to steps_kdk_step).  EINVAL unless eps and dt_max are finite and > 0 and
 * t_end is not NaN.
 */
steps_status steps_timestep(steps_ctx *ctx, double eps, double dt_max, double t_end, double *dt_out);

/*
 * nsteps KDK steps (Eq. 11), each of the length Eq. 12 gives at its start,
 * computed and applied on the device (non-sorting steps replay one CUDA
 * graph; no host synchronisation between steps).  Steps taken after t has
 * reached t_end have length 0 and move nothing.  *t_out (may be NULL)
 * receives the final t.  Same argument checks as steps_timestep.
 */
steps_status steps_kdk_run_adaptive(steps_ctx *ctx, int nsteps, double eps, double dt_max, double t_end,
                                    double *t_out);

/*
 * steps_get_state -- copy the FP64 state out in caller order.  Any pointer
 * may be NULL to skip it.  pos/vel/acc are [n][3]; acc is the pair term at the
 * current positions.  Synchronises the stream.
 */
steps_status steps_get_state(steps_ctx *ctx, double *pos, double *vel, double *acc, double *t,
                             double *a);

/*
 * steps_set_state -- overwrite positions and velocities (caller order,
 * [n][3], host or device) and the time/scale factor, then re-sort and
 * recompute the pair term.  Masses and softening are kept.
 */
steps_status steps_set_state(steps_ctx *ctx, const double *pos, const double *vel, double t,
                             double a);

/*
 * Exact checkpoint/resume.  steps_checkpoint_size gives the byte size of an
 * opaque blob holding the full internal state (sorted FP64 arrays, the
 * permutation, the stored pair term, t, a, step count).  Restoring it into a
 * context created with the same n, masses, softening and config continues the
 * run bit-identically to an uninterrupted one.  buf is host memory.
 */
steps_status steps_checkpoint_size(steps_ctx *ctx, size_t *bytes);
steps_status steps_checkpoint_save(steps_ctx *ctx, void *buf);
steps_status steps_checkpoint_load(steps_ctx *ctx, const void *buf);

/*
 * steps_forces_subset -- the pair term of Eq. 8 (same definition as
 * steps_forces) for nt selected targets only, always summed in FP64 on the
 * GPU over all n sources, at the current positions.  targets [nt] are caller
 * indices (host or device int64); acc_out [nt][3] (host or device) receives
 * the rows in the order given.  Used for accuracy checks and the FP64
 * comparison timing.  EINVAL for an index outside [0, n).
 */
steps_status steps_forces_subset(steps_ctx *ctx, int64_t nt, const int64_t *targets, double *acc_out);

/*
 * steps_diagnostics -- FP64 diagnostics at the current state:
 *   ekin = 1/2 sum m v^2,  p = sum m v,  epot = 1/2 sum_i sum_{j != i} G m_i m_j W(r_ij, h_i+h_j)
 * where W is the pair potential of the spline kernel (W' = F of Eq. 4,
 * W = -1/r for r >= h, W(0) = -2.8/h).  Any output pointer (host) may be
 * NULL; epot costs an O(N^2) FP64 pass, so pass NULL to skip it.
 */
steps_status steps_diagnostics(steps_ctx *ctx, double *ekin, double *epot, double p[3]);

/* Number of particles in the context. */
int64_t steps_size(const steps_ctx *ctx);

/* Release the context and all its device memory.  NULL is ignored. */
void steps_free(steps_ctx *ctx);

const char *steps_strerror(steps_status s);
const char *steps_last_error(void);

/*
 * Testing hook: bound, in nanoseconds, for every device-side wait of the
 * force kernels of this context (default 2e9).  A wait that runs out makes the
 * kernel record STEPS_ETIMEOUT, drain its own copies and exit; the next
 * synchronising call returns STEPS_ETIMEOUT.  0 makes the first wait give up.
 */
steps_status steps_set_wait_limit(steps_ctx *ctx, int64_t ns);

/*
 * Process-wide cap, in bytes, on the device memory this library allocates
 * (0 = no cap, the default).  An allocation that would exceed it fails with
 * STEPS_ENOMEM before cudaMalloc is called; used to exercise the out-of-memory
 * path without exhausting the GPU.
 */
steps_status steps_set_memory_limit(size_t bytes);

/*
 * Kernel timing for benchmarks.  While enabled, the context records CUDA
 * events around every pair-force kernel launch on its stream.
 * steps_profile_read synchronises and returns the summed device time of those
 * launches (ms), their count, and the number of kernels of this library the
 * context launched since the last reset.  Any output pointer may be NULL.
 */
steps_status steps_profile_enable(steps_ctx *ctx, int on);
steps_status steps_profile_read(steps_ctx *ctx, double *force_ms, int64_t *force_launches,
                                int64_t *kernel_launches, int reset);
/*
 * The far-field kernel alone (FP32 modes): summed device time (ms) of the
 * far-field launches recorded since the last steps_profile_read reset, and
 * their count.  Read it before the reset; it does not reset anything itself.
 */
steps_status steps_profile_read_far(steps_ctx *ctx, double *far_ms, int64_t *far_launches);

/*
 * steps_forces_noalloc -- the same pair term and FP32 compensated arithmetic
 * as steps_forces (64-particle tiles, caller order) for a system of at most
 * STEPS_NOALLOC_MAX_N particles, without allocating any device memory.  The
 * paper has no counterpart: this entry point exists for callers that cannot
 * allocate around a force evaluation, e.g. code running inside an application
 * whose caching allocator already owns the device memory, or a per-step loop
 * that must not take the implicit device synchronisation of cudaMalloc and
 * cudaFree.  All scratch lives in one fixed array of about 6.7 MiB compiled
 * into this library; every device that loads the library holds it until exit.
 *   pos [n][3], mass [n], soft [n] (or NULL: derived from h_min as in steps_init), acc_out [n][3]:
 *   device pointers on the current device, caller order, caller-owned.
 *   cuda_stream: stream to run on (NULL = legacy default stream); the call
 *   synchronises it before returning.
 * Errors: EINVAL for n outside [1, STEPS_NOALLOC_MAX_N], NULL or host
 * pointers, or pointers to another device's memory (all checked before any
 * GPU work), or non-finite / non-positive inputs (found on the GPU and
 * reported after the call's one synchronisation; acc_out then holds no
 * result); ECUDA; ETIMEOUT as for steps_forces.
 * The first call on a device looks up the scratch array's device address and
 * caches it; make that first call before any stream capture begins.
 * Every call shares the scratch array, which keeps the previous call's
 * contents (the call clears what must start at zero): calls that overlap on
 * the GPU -- different streams or host threads on one device -- race and must
 * be serialised by the caller.
 */
#define STEPS_NOALLOC_MAX_N 8192
steps_status steps_forces_noalloc(int64_t n, const double *pos, const double *mass,
                                  const double *soft, double h_min, double G, double *acc_out,
                                  void *cuda_stream);

/*
 * Spherical-glass initial conditions (Sec. 3.1, Eq. 14-18).  The real space is
 * compactified onto the 3-sphere of diameter D_s by the inverse stereographic
 * projection (Eq. 14: omega = 2 arctan(r / D_s)); the compactified space is
 * cut into shells along omega, n_shell particles are placed uniformly in the
 * compact volume of each shell and mapped back by Eq. 15, and each shell's
 * particles carry m = rho_bar V_shell / n_shell (Eq. 16, V_shell the
 * real-space volume).  Two slicings:
 *   STEPS_GLASS_CONST_DOMEGA  -- n_radial shells of equal width in omega from
 *       omega_c = 2 arctan(r_c / D_s) to omega_max = 2 arctan(R_sim / D_s);
 *       the ball r < r_c holds N_inner = floor((4 pi / 3) r_c^3 rho_bar / m_inner)
 *       equal-mass particles (Eq. 17), m_inner = the first shell's particle
 *       mass, placed uniformly in real space;
 *   STEPS_GLASS_CONST_VOLUME  -- n_radial shells of equal compact volume from
 *       omega = 0 to omega_max, edges from Eq. 18 solved numerically.
 * The glass itself is made by relaxing these positions under reversed gravity
 * (steps_init with mode STEPS_COMOVING_REVERSED, Om = 1, OL = 0).
 */
typedef enum { STEPS_GLASS_CONST_DOMEGA = 0, STEPS_GLASS_CONST_VOLUME = 1 } steps_glass_scheme;

typedef struct {
    int scheme;       /* steps_glass_scheme */
    double D_s;       /* diameter of the hypersphere (Eq. 14-15) */
    double R_sim;     /* real-space radius of the simulated volume */
    int n_radial;     /* shells (outside the inner ball for STEPS_GLASS_CONST_DOMEGA) */
    int64_t n_shell;  /* particles per shell */
    double r_c;       /* STEPS_GLASS_CONST_DOMEGA: radius of the united inner ball, 0 < r_c < R_sim */
    double rho_bar;   /* mean matter density Om rho_crit of Eq. 16 */
} steps_glass_spec;

/*
 * The layout of a spec: total particle count, inner-ball count and mass (0
 * for STEPS_GLASS_CONST_VOLUME), shell edges in omega [n_radial + 1] and the
 * particle mass of each shell [n_radial].  Host outputs, any may be NULL.
 * EINVAL for a non-positive or non-finite size, an unknown scheme, or r_c
 * outside (0, R_sim) in the constant delta-omega scheme.
 */
steps_status steps_glass_layout(const steps_glass_spec *spec, int64_t *n_total, int64_t *n_inner,
                                double *m_inner, double *omega_edges, double *shell_mass);

/*
 * Place the n = n_total particles of a spec from the caller's uniform random
 * numbers u [n][3] in [0, 1): u[k][0] picks omega inside the particle's shell
 * (by the compact-volume law) or the radius inside the inner ball, u[k][1] the
 * cosine of the polar angle (1 - 2u), u[k][2] the azimuth (2 pi u).  Writes
 * pos [n][3] and mass [n]: the inner ball's particles first, then n_shell per
 * shell, innermost first.  u, pos and mass may be host or device pointers;
 * the call allocates device scratch of 7n + 2 n_radial + 1 doubles for its
 * duration and synchronises the stream.  EINVAL as steps_glass_layout, or if
 * n is not the layout's count.
 */
steps_status steps_glass_place(const steps_glass_spec *spec, int64_t n, const double *u, double *pos,
                               double *mass, void *cuda_stream);

/*
 * Ensembles: many independent simulations of uneven N and differing
 * cosmologies advanced together (batched runs for parameter studies, the use
 * the paper names for fast low-resolution simulations in its abstract).  Each member is
 * a system of its own -- its particles interact only with each other -- with
 * its own steps_config (G, H0, Om, OL, Or, Ok, mode; precision, re-sort period
 * and tile_override are taken from cfgs[0]), t0, a0 and softening (soft[s], or
 * NULL / soft == NULL: Eq. 7 with h_min[s]).  All members share one force
 * launch per step (the far-field grid walks every member's tile pairs) and
 * one CUDA graph per step.  Members are padded to multiples of 1,024
 * particles; unless tile_override names a variant, init times every force
 * variant of the summation mode whose target block fits that padding on the
 * members' initial state (median of three evaluations) and keeps the fastest.
 *   n [nsims], pos/vel/mass/soft: arrays of nsims pointers (host or device),
 *   each [n_s][3] or [n_s] in the member's caller order; vel may be NULL.
 * steps_ensemble_run: nsteps KDK steps (Eq. 9-11), dts [nsims][nsteps] host,
 * row-major (member s uses dts[s*nsteps + k] at step k).
 * steps_ensemble_get_state: member s's state in its caller order (any output
 * pointer may be NULL).  steps_ensemble_stats: padded particle total and the
 * near/all tile pairs since the last call.  steps_ensemble_variant: index of
 * the force variant in use (steps_variant_name).
 */
typedef struct steps_ens steps_ens;
steps_status steps_ensemble_init(steps_ens **out, int nsims, const int64_t *n,
                                 const double *const *pos, const double *const *vel,
                                 const double *const *mass, const double *const *soft,
                                 const double *h_min, const double *t0, const double *a0,
                                 const steps_config *cfgs, void *cuda_stream);
steps_status steps_ensemble_run(steps_ens *e, int nsteps, const double *dts);
steps_status steps_ensemble_get_state(steps_ens *e, int sim, double *pos, double *vel, double *acc,
                                      double *t, double *a);
steps_status steps_ensemble_variant(steps_ens *e, int *k);
steps_status steps_ensemble_stats(steps_ens *e, int64_t *total_particles, uint64_t *near_pairs,
                                  uint64_t *all_pairs);
void steps_ensemble_free(steps_ens *e);

/*
 * steps_paircount -- exact pair counts DD of nsets point sets in one launch.
 * The statistics of the density field are what the simulations are run for
 * (Sec. 1; opening of Sec. 3); the central sphere's two-point correlation
 * function xi(r) = DD/RR - 1 (natural estimator, RR analytic for a uniform
 * ball) is the target of the emulator.  The paper gives no counting
 * algorithm: this is the exact pair count by definition.  Set s is pos[offsets[s] .. offsets[s+1]) of
 * pos [N][3] (host or device).  Coordinates are quantised about the set's
 * centre (centres [nsets][3]) to integers q = llround((x - c) * (1/step));
 * |x - c| / step must stay below 2^29 (else EINVAL), so that |q_i - q_j|^2
 * fits in int64.  A pair i < j falls in bin b when
 * edge2[b] <= |q_i - q_j|^2 < edge2[b+1] (edge2 [nbins+1], squared edges in
 * units of step^2, non-negative and non-decreasing; nbins <= 64).
 * dd_out [nsets][nbins] (host or device) receives the counts.  Integer
 * arithmetic throughout: counts are exact and independent of the order of
 * the additions.  Allocates scratch for the call; synchronises the stream.
 */
steps_status steps_paircount(int nsets, const int64_t *offsets, const double *pos,
                             const double *centres, double step, int nbins, const int64_t *edge2,
                             uint64_t *dd_out, void *cuda_stream);

/*
 * Near-field threshold of the FP32 path (default 1/32): a source tile is
 * summed with the compensated near-field method when its bounding box comes
 * closer to the target tile than alpha x (centre distance + both extents);
 * pairs inside h_i + h_j and tiles larger than their distance always are.
 * Larger alpha moves more work to the (slower, more exact) near field.
 */
steps_status steps_set_near_alpha(steps_ctx *ctx, double alpha);

/*
 * Tile-pair statistics of the FP32 path since the last call (reset on read):
 * how many target-tile x source-tile pairs were classified near field
 * (summed with the compensated/spline path) out of all pairs visited.
 * Synchronises the stream.
 */
steps_status steps_force_stats(steps_ctx *ctx, uint64_t *near_pairs, uint64_t *all_pairs);

/* Force-kernel variants built into the library (for tile_override and tuning). */
int steps_num_variants(void);
const char *steps_variant_name(int k);
/* The variant (0-based) the context's FP32 path uses, as chosen by
 * tile_override or the autotuner; -1 for STEPS_F64. */
steps_status steps_get_variant(steps_ctx *ctx, int *k);

#ifdef __cplusplus
}
#endif

#endif /* STEPS_H */
