/*
 * sidm.h -- C ABI of the GB300 (sm_103a) SIDM scattering pass.
 *
 * The pass is the per-step self-interaction step of the N-body method of
 * Fischer, Yu & Dolag (2025), "Accurately simulating core-collapse
 * self-interacting dark matter halos":
 *   (a) kernel sizes h_i from the N_ngb nearest neighbours (Sect. 2),
 *   (b) pair interaction probabilities over kernel overlaps
 *       P_ij = (sigma(v_ij)/m) m_j |v_ij| Lambda_ij dt (Sect. 3.5, Eq. vel_dep),
 *   (c) scatter draws and isotropic, energy- and momentum-conserving velocity
 *       updates (Sect. 2, Sect. 5), with a deterministic order for particles
 *       hit more than once in a step.
 *
 * Conventions for every call
 *   - All pointers named *_dev are device pointers on the context's device;
 *     pointers without that suffix are host pointers.  Particle arrays are SoA:
 *     a "[3][N]" array holds x[0..N), then y[0..N), then z[0..N).
 *   - The caller owns every particle array and every output.  The context owns
 *     only its scratch, allocated once by sidm_create; no other call allocates.
 *   - Calls are asynchronous on the given stream (0 = legacy default stream)
 *     unless stated otherwise.  A call that returns non-zero has enqueued
 *     nothing that writes a caller array.
 *   - Return value: 0 on success, a negative SIDM_E* code otherwise;
 *     sidm_last_error() gives a one-line message.
 *   - Failures found on the device (capacity, round limit, bad input) set bits
 *     of a device-side status word, read by sidm_status().  Nothing traps, and
 *     every wait inside a kernel is bounded.
 *   - Halo layout: particles of halo h are [halo_off[h], halo_off[h+1]) of the
 *     particle arrays.  Every particle of a halo has the same mass, ids are
 *     unique within a halo and smaller than 2^27; at most 1024 halos.
 */
#ifndef SIDM_H
#define SIDM_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define SIDM_OK          0
#define SIDM_EINVAL     -1   /* bad argument or call order                        */
#define SIDM_ECAPACITY  -2   /* a capacity given to sidm_create is too small      */
#define SIDM_ECUDA      -3   /* a CUDA runtime call failed                        */
#define SIDM_EROUNDS    -4   /* the resolve round limit was hit (see sidm_status) */
#define SIDM_EDEVICE    -5   /* the device status word is non-zero               */

/* device status word bits (sidm_status) */
#define SIDM_DEV_EVENT_OVERFLOW  0x1u  /* more events than event_cap: velocities untouched */
#define SIDM_DEV_ROUNDS          0x2u  /* resolve stopped at max_rounds                     */
#define SIDM_DEV_STACK           0x4u  /* tree traversal stack overflow (results invalid)   */
#define SIDM_DEV_BAD_INPUT       0x8u  /* id >= 2^27 or non-finite position                 */
#define SIDM_DEV_WAIT_TIMEOUT    0x10u /* a bounded wait on an async copy gave up           */

/* precision forms */
#define SIDM_MIXED 0   /* FP32 offsets/velocities/probabilities, FP64 reductions */
#define SIDM_FP64  1   /* every step in FP64                                     */

/* sidm_config.flags */
#define SIDM_FLAG_SUM_P   0x1  /* accumulate sum_j P_ij per particle (diagnostic) */
#define SIDM_FLAG_TIMING  0x2  /* time hot kernels with CUDA events (sidm_kernel_times) */
#define SIDM_FLAG_LOCAL_DIAG 0x4 /* keep scratch for sidm_local_diagnostics (40 B/particle) */
#define SIDM_FLAG_DRAG    0x8  /* keep scratch for forward-dominated halos (sidm_xs.angular = 1):
                                  per-particle interaction lists, 64 B per event_cap */

typedef struct sidm_ctx sidm_ctx;

typedef struct {
    int64_t n_max;       /* particle capacity (all halos together), >= 1            */
    int32_t halo_max;    /* halo capacity, 1..1024                                  */
    int32_t ngb_max;     /* largest N_ngb of any halo, 1..128                       */
    int64_t event_cap;   /* scatter events kept per step, >= 1                      */
    int32_t precision;   /* SIDM_MIXED or SIDM_FP64                                 */
    int32_t device;      /* CUDA device ordinal                                      */
    int32_t knn_warps;   /* warps per CTA of the neighbour kernel, 0..16, 0 = 8      */
    int32_t pair_warps;  /* warps per CTA of the pair kernel, 0..8, 0 = 8            */
    int32_t max_rounds;  /* resolve round limit, 0 = default (256)                   */
    int32_t flags;       /* SIDM_FLAG_*                                              */
    int32_t grid_ctas;   /* persistent CTAs per kernel, 0 = SM count x occupancy     */
    int32_t use_tma;     /* 1: stage candidate tiles with bulk async copies (TMA)    */
    /* launch knobs of the hot kernels; none changes a result (0 = default) */
    int32_t knn_groups;  /* kernel-size search: lane groups of the candidate mask,   */
                         /*   2, 4 or 8 (default 2; plain-load path)                 */
    int32_t knn_chains;  /*   independent distance chains, 4 or 8 (default 4; 8     */
                         /*   with knn_groups 4 only)                                */
    int32_t knn_flush;   /*   pending keys per lane that trigger a heap merge before */
                         /*   a tree node's tests, 1..32 (default 32)                */
    float   knn_slack;   /*   warm-start bound / previous kernel size, 1..2 (1.07)   */
    int32_t pair_per_round; /* pair kernel: pairs a lane queues per round, 1..4 (4; mixed-form draws) */
    int32_t knn_batch;   /* kernel-size search: 1 loops over each staged leaf's      */
                         /*   candidates, 2 over compacted batches of them, 3 as 2    */
                         /*   with warm-started searches in the fixed-bound kernel    */
                         /*   (default 3; bulk copies and neighbour lists take 1)     */
} sidm_config;

/* Cross-section per unit mass of one halo (Sect. 3.8, Eq. vel_dep), given as
 * the viscosity cross-section sigma_V of App. A (normalised to the total
 * cross-section for isotropic scattering):
 *   kind 0: sigma_V/m = s0 (velocity independent);
 *   kind 1: sigma_V/m = s0 / (1 + (v/w)^2)^2, v = |v_i - v_j| the pair speed.
 * angular 0: isotropic scattering (sigma = sigma_V): a pair scatters with
 *   probability P_ij = (sigma/m) m_j v Lambda_ij dt into an isotropic direction.
 * angular 1: forward-dominated (Sect. 3.8: the limit of a vanishing angle at
 *   constant momentum transfer): every in-range pair interacts every step; its
 *   relative velocity u (i the smaller id) turns by alpha, cos(alpha) = 1 - D,
 *   sin(alpha) = sqrt(D (2 - D)) (alpha = pi for D >= 2), with
 *   D = (sigma_V/m) / 3 |u| m_j Lambda_ij dt (the momentum-transfer cross-section
 *   of that limit is sigma_V / 3), towards the projection onto u's normal
 *   plane of the isotropic direction of Philox words 1 and 2 (as an isotropic
 *   scatter draws it), uniform in azimuth about u; |u| and the centre-of-mass
 *   velocity are kept.  Pairs apply in ascending key order from the current
 *   velocities, with Lambda, m_j and dt of the step start.  Needs a context
 *   created with SIDM_FLAG_DRAG and an event_cap that holds every in-range
 *   pair (about 2 N_ngb per particle).
 * Code units. */
typedef struct {
    int32_t kind;
    int32_t angular;
    double s0;
    double w;
} sidm_xs;

/* A fixed analytic host galaxy (Sect. 4.1: the satellite moves in an external
 * potential of six parts, each given by its Eq. there), about `center`, with
 * r = |x - center| and R, z the cylindrical radius and height about it:
 *   NFW halo        Phi = -4 pi G rho_s r_s^3 ln(1 + r/r_s) / r        (rho_s = 0: none)
 *   Hernquist bulge Phi = -G M_H / (r + a_H)                          (M_H = 0: none)
 *   n_disks Miyamoto-Nagai disks
 *                   Phi = -G M_d / sqrt(R^2 + (a_d + sqrt(z^2 + b_d^2))^2)
 * Code units; every length > 0 (b_d > 0), every mass >= 0, 0 <= n_disks <= 4. */
#define SIDM_HOST_MAX_DISKS 4
typedef struct {
    double G;
    double center[3];
    double rho_s;
    double r_s;
    double M_H;
    double a_H;
    int32_t n_disks;
    int32_t pad_;
    double M_d[SIDM_HOST_MAX_DISKS];
    double a_d[SIDM_HOST_MAX_DISKS];
    double b_d[SIDM_HOST_MAX_DISKS];
} sidm_host;

/* Per-step statistics, written by sidm_scatter_step (device memory). */
typedef struct {
    unsigned long long n_pairs;   /* in-range pairs whose P was formed            */
    unsigned long long n_events;  /* accepted events (can exceed event_cap)       */
    unsigned long long n_p_gt1;   /* pairs with P > 1 (no clamp; always fire)     */
    unsigned long long n_near;    /* pairs with |P - u| < 1e-6                   */
    unsigned long long n_multi;   /* particles in more than one event            */
    unsigned int rounds;          /* resolve rounds used                          */
    unsigned int status;          /* SIDM_DEV_* bits raised by this step          */
    double d_energy;              /* sum over events of the change of the pair's  */
                                  /* kinetic energy from the stored velocities    */
                                  /* (FP64, exact fixed-point accumulation)       */
    float max_sum_p;              /* max_i sum_j P_ij (SIDM_FLAG_SUM_P only)      */
    float pad_;
    unsigned long long n_tested;  /* candidate pairs given the in-range test      */
} sidm_step_stats;

/* One accepted scatter event, as kept for the current step. */
typedef struct {
    unsigned long long key;       /* halo<<54 | min id<<27 | max id               */
    uint32_t i, j;                /* particle indices (i has the smaller id)      */
    uint32_t x1, x2;              /* Philox words 1, 2 (scattering direction)     */
    float P;                      /* interaction probability                      */
    uint32_t x0;                  /* Philox word 0 (u = x0 * 2^-32)               */
} sidm_event;

/* Create a context on cfg->device: checks the configuration, allocates all
 * scratch for n_max particles / halo_max halos / event_cap events, and fills
 * the Lambda lookup table (FP64 quadrature of the spline overlap, Sect. 3.5).
 * Synchronous.  On failure *ctx is NULL. */
int sidm_create(sidm_ctx** ctx, const sidm_config* cfg);

/* Free the context and all its scratch (synchronous). NULL is a no-op. */
int sidm_destroy(sidm_ctx* ctx);

/* Message of the last failed call on this context (never NULL). */
const char* sidm_last_error(const sidm_ctx* ctx);

/* Message of the last failed sidm_create (thread-local). */
const char* sidm_create_error(void);

/* (a0) Cell build.  Sorts the particles of every halo by a 3 x 17-bit Morton
 * key of a power-of-two cube around the halo, permutes pos/vel/id in place
 * into that order, and builds leaves of 32 consecutive particles with FP32
 * offsets to power-of-two cell origins, bounding boxes and a bounding-volume
 * tree.  Replaces the neighbour-search structure of Sect. 2.
 *   n_halos    : 1..halo_max
 *   halo_off   : host int64[n_halos+1], non-decreasing, halo_off[0] == 0,
 *                halo_off[n_halos] <= n_max.  A changed layout is uploaded by
 *                this call (host -> device copy); an unchanged one is not.
 *   pos_dev    : f64 [3][N] positions (reordered in place)
 *   vel_dev    : [3][N] velocities, f32 (SIDM_MIXED) or f64 (SIDM_FP64)
 *                (reordered in place)
 *   id_dev     : u32 [N] particle ids (reordered in place)
 * Must be called again after any change of the positions. */
int sidm_build_cells(sidm_ctx* ctx, int32_t n_halos, const int64_t* halo_off,
                     double* pos_dev, void* vel_dev, uint32_t* id_dev, cudaStream_t stream);

/* (a1) Kernel sizes (Sect. 2; Eq. hDl): h_i = distance to the N_ngb-th nearest
 * other particle of the same halo, in the precision form's distance (FP32
 * canonical offset distance or FP64).
 *   n_ngb   : host int32[n_halos], 1 <= n_ngb[h] <= ngb_max and
 *             n_ngb[h] < particles of halo h (empty halos are skipped)
 *   h_dev   : out, f32 (SIDM_MIXED) or f64 (SIDM_FP64) [N], in the order left
 *             by sidm_build_cells
 * Requires a preceding sidm_build_cells. */
int sidm_kernel_sizes(sidm_ctx* ctx, const int32_t* n_ngb, void* h_dev, cudaStream_t stream);

/* (a2-a4) Scatter step.  For every unordered pair of a halo with
 * d_ij < h_i + h_j: Lambda_ij, P_ij = (sigma(v_ij)/m) m |v_ij| Lambda_ij dt
 * from the step-start velocities, u = Philox4x32-10(key = seed,
 * counter = (step mod 2^32, min id, max id, halo)) word 0 times 2^-32, event iff
 * u < P.  Events are applied in ascending (halo, min id, max id) order, each
 * from the current velocities: v_cm +- (m_j/M)|dv| n, n isotropic from Philox
 * words 1 and 2 (cos theta = 2 u1 - 1, phi = 2 pi u2); the smaller id gets +.
 *   seed, step  : Philox key and counter word 0
 *   xs_dev      : device sidm_xs[n_halos]
 *   dt_dev      : device f64[n_halos] time step per halo
 *   mass_dev    : device f64[n_halos] particle mass per halo
 *   vel_dev     : [3][N] velocities (f32 or f64 by precision), updated in place
 *   stats_dev   : device sidm_step_stats, overwritten (may be NULL)
 * If more than event_cap events are drawn, no velocity is changed and
 * SIDM_DEV_EVENT_OVERFLOW is raised.  Requires sidm_kernel_sizes. */
int sidm_scatter_step(sidm_ctx* ctx, uint64_t seed, uint64_t step, const sidm_xs* xs_dev,
                      const double* dt_dev, const double* mass_dev, void* vel_dev,
                      sidm_step_stats* stats_dev, cudaStream_t stream);

/* (a5) Per-halo kinetic energy and momentum, E = sum 1/2 m |v|^2,
 * p = sum m v (the paper tracks energy conservation throughout, Sect. 3.4).
 * FP32 velocities are summed exactly as 128-bit integers per chunk of 16384
 * particles (bits below 2^-94 of the chunk's largest term may drop), FP64
 * velocities with compensated (two-sum) FP64 accumulation; chunk sums are
 * merged as double-doubles in a fixed order and scaled by the mass once, so
 * repeated calls give identical bits.
 *   mass_dev : device f64[n_halos]
 *   vel_dev  : [3][N] velocities (f32 or f64 by precision)
 *   out_dev  : device f64[n_halos][4] = (E, px, py, pz)
 *   comp_dev : device f64[n_halos][4] residual compensation terms, or NULL
 * Requires sidm_build_cells (for the halo layout). */
int sidm_energy_momentum(sidm_ctx* ctx, const double* mass_dev, const void* vel_dev,
                         double* out_dev, double* comp_dev, cudaStream_t stream);

/* Synchronise the stream, return the device status word (SIDM_DEV_* bits
 * raised since the last sidm_status) in *status and clear it.  Returns
 * SIDM_EDEVICE if it was non-zero, SIDM_ECUDA on a CUDA error. */
int sidm_status(sidm_ctx* ctx, cudaStream_t stream, uint32_t* status);

/* ---- harness and test entry points -------------------------------------- */

/* Permutation of the last sidm_build_cells: perm_dev[s] = index, before that
 * call, of the particle now at position s.  device u32[N]. */
int sidm_get_perm(sidm_ctx* ctx, uint32_t* perm_dev, cudaStream_t stream);

/* Neighbour ids of the last kernel-size pass (mixed form only): for particle s
 * the ids of its n_ngb nearest others in ascending (canonical d^2, id) order.
 *   nbr_dev : device u32[N][k_stride], k_stride >= max n_ngb. */
int sidm_neighbours(sidm_ctx* ctx, const int32_t* n_ngb, int32_t k_stride,
                    uint32_t* nbr_dev, cudaStream_t stream);

/* Copy the events kept by the last sidm_scatter_step, in the order they were
 * drawn (not sorted), to ev_dev[0..min(cap, n)); *n_host receives the event
 * count (synchronises the stream). */
int sidm_get_events(sidm_ctx* ctx, int64_t cap, sidm_event* ev_dev, int64_t* n_host,
                    cudaStream_t stream);

/* Evaluate the device Lambda(d; h_i, h_j) (lookup table of the context's
 * precision) for n triples; all device f64 arrays. */
int sidm_lambda_eval(sidm_ctx* ctx, int64_t n, const double* d_dev, const double* hi_dev,
                     const double* hj_dev, double* out_dev, cudaStream_t stream);

/* Ballistic drift x += v dt per halo (harness for multi-step runs):
 * dt_dev device f64[n_halos]; pos f64 [3][N]; vel f32/f64 [3][N]. */
int sidm_drift(sidm_ctx* ctx, const double* dt_dev, double* pos_dev, const void* vel_dev,
               cudaStream_t stream);

/* Reflecting spherical boundary (Sect. 2: the isolated halos are kept inside
 * a sphere of 200 kpc that turns outward-moving particles back, leaving the
 * energy unchanged).  Reading: a particle of halo h with |x - c_h| > R_h and
 * v . (x - c_h) > 0 has the radial part of its velocity reversed,
 *   v <- v - 2 (v . d) d / |d|^2,  d = x - c_h   (speed kept; FP64, then
 * rounded to the velocity's type).  Call it after sidm_drift.
 *   bound_dev : device f64 [n_halos][4] = (c_x, c_y, c_z, R); R <= 0: no boundary
 *   pos_dev   : f64 [3][N];  vel_dev : [3][N] f32/f64 by precision, updated
 * Arrays in the order left by sidm_build_cells (which must come first). */
int sidm_reflect_boundary(sidm_ctx* ctx, const double* bound_dev, const double* pos_dev, void* vel_dev,
                          cudaStream_t stream);

/* Per-particle sum_j P_ij of the last scatter step (SIDM_FLAG_SUM_P), f32 [N]. */
int sidm_get_sum_p(sidm_ctx* ctx, float* out_dev, cudaStream_t stream);

/* Kernels launched by the calls above since the context was created. */
int64_t sidm_launch_count(const sidm_ctx* ctx);

/* Device time of the hot kernels, measured with CUDA events recorded on the
 * launching stream around each launch (contexts created with
 * SIDM_FLAG_TIMING; at most 4096 launches are recorded between resets).
 *   ms_out[4]    : milliseconds of {cell build (whole a0 sequence), kernel-size
 *                  kernel, pair kernel, resolve kernel} since the last reset
 *   count_out[4] : launches recorded per slot (may be NULL)
 *   reset        : non-zero clears the record afterwards
 * Synchronises the device. */
int sidm_kernel_times(sidm_ctx* ctx, double* ms_out, int64_t* count_out, int32_t reset);

/* Work counters of the kernel-size and pair kernels since the last reset
 * (synchronises the device): out[0] candidate leaves staged by the kernel-size
 * kernel, out[1] lane-level candidate distances, out[2] heap insertions,
 * out[3] largest number of leaves staged for one query leaf, out[4] candidate
 * leaves staged by the pair kernel, out[5] its largest per query leaf,
 * out[6] in-range pairs whose Lambda was looked up (all of them under
 * SIDM_FLAG_SUM_P; otherwise only those whose draw fell below the upper bound
 * of P), out[7] particles whose warm-started kernel-size search found fewer
 * than N_ngb candidates inside the guessed bound and was redone cold.
 * reset != 0 clears them afterwards. */
int sidm_diagnostics(sidm_ctx* ctx, uint64_t* out, int32_t reset);

/* Local diagnostics of every particle (Sect. 3.5 Eq. hDl, Sect. 3.6
 * Eq. knudsen_number, App. C Eq. effective_cross_section), from one traversal
 * of the in-range pairs fused with the kernel sums (no draws, no velocity
 * change):
 *   rho_i = sum over j with d_ij < h_i, i itself included, of m W(d_ij, h_i)
 *           (SPH density over the particle's own kernel);
 *   nu_i  = 1-D velocity dispersion of the same kernel-weighted moments,
 *           nu^2 = (<|v|^2> - |<v>|^2) / 3;
 *   sigma_eff_i / m = <v^5 sigma(v)> / <v^5> over the relative-speed
 *           Maxwellian of two particles of dispersion nu_i (sigma_V = sigma
 *           for isotropic scattering);
 *   (h/l)_i = (sigma_eff/m) rho^(2/3) (3 m N_ngb / (pi sqrt 2))^(1/3);
 *   Kn_i    = sqrt(4 pi G / (rho nu^2)) / (sigma_eff/m).
 *   xs_dev   : device sidm_xs[n_halos] (the cross-section law of each halo)
 *   mass_dev : device f64[n_halos] particle mass per halo
 *   vel_dev  : [3][N] velocities (f32 or f64 by precision), read only
 *   G        : gravitational constant in code units
 *   out_dev  : out, f32 (SIDM_MIXED) or f64 (SIDM_FP64) [5][N]: rho, nu,
 *              sigma_eff/m, h/l, Kn, in the order left by sidm_build_cells
 * Requires SIDM_FLAG_LOCAL_DIAG at creation and a preceding
 * sidm_kernel_sizes; uses the kernel sizes and N_ngb of that call.  The
 * moments are summed with FP64 atomics, so the last bits of rho and nu may
 * differ between runs. */
int sidm_local_diagnostics(sidm_ctx* ctx, const sidm_xs* xs_dev, const double* mass_dev, const void* vel_dev,
                           double G, void* out_dev, cudaStream_t stream);

/* Scatter step on individual power-of-two time steps (the individual time
 * steps of Sect. 3.1).  Particle u of bin b = bin_dev[u] has the step
 * dt_max / 2^b; the 2^(n_bins-1) sub-steps of a big step dt_max are numbered
 * 0 .., and bin b opens a step at sub-step s iff s is a multiple of
 * 2^(n_bins-1-b).  At sub-step `substep` only pairs whose particles both open
 * a step are tested, with P formed on the longer of the two steps,
 * dt_max / 2^min(b_i, b_j); everything else is sidm_scatter_step.  Under
 * SIDM_FLAG_SUM_P the per-particle sums hold P scaled to dt_max (a rate times
 * dt_max), so sidm_timestep_criterion takes dt_max as the step of every halo.
 *   dt_max    : the longest step (bin 0), > 0
 *   n_bins    : 1..16;  substep : 0 .. 2^(n_bins-1) - 1
 *   bin_dev   : device int32[N], bins in 0 .. n_bins-1, in the order left by
 *               sidm_build_cells (the caller permutes its bins with the
 *               particles, e.g. through sidm_get_perm)
 * Other arguments and behaviour as sidm_scatter_step. */
int sidm_scatter_step_binned(sidm_ctx* ctx, uint64_t seed, uint64_t step, const sidm_xs* xs_dev, double dt_max,
                             int32_t n_bins, int32_t substep, const int32_t* bin_dev, const double* mass_dev,
                             void* vel_dev, sidm_step_stats* stats_dev, cudaStream_t stream);

/* Kick by the analytic host (kick-drift-kick on individual steps): every
 * particle whose step opens at sub-step `substep` (phase 0, before the drift)
 * or closes after it (phase 1, after the drift of that sub-step) gets
 * v += a(x) dt_b / 2, dt_b = dt_max / 2^b, with the acceleration a = -grad Phi
 * of `host` evaluated in FP64 at its FP64 position (zero from the spherical
 * parts at the centre itself).
 *   host      : host-memory sidm_host
 *   bin_dev   : device int32[N] or NULL (every particle in bin 0)
 *   pos_dev   : f64 [3][N];  vel_dev : [3][N] f32 or f64 by precision, updated
 * Arrays in the order left by sidm_build_cells (which must come first). */
int sidm_host_kick(sidm_ctx* ctx, const sidm_host* host, double dt_max, int32_t n_bins, int32_t substep,
                   int32_t phase, const int32_t* bin_dev, const double* pos_dev, void* vel_dev, cudaStream_t stream);

/* Potential of the analytic host at every particle (for the energy of a
 * satellite run, E = sum_i m (v_i^2 / 2 + Phi(x_i))), FP64.
 *   host    : host-memory sidm_host (as sidm_host_kick)
 *   pos_dev : f64 [3][N] in the order left by sidm_build_cells (which must come first)
 *   phi_dev : device f64 [N], written
 * Errors: SIDM_EINVAL for a null argument or a bad host. */
int sidm_host_potential(sidm_ctx* ctx, const sidm_host* host, const double* pos_dev, double* phi_dev,
                        cudaStream_t stream);

/* SIDM time-step criterion (Sect. 2: a separate time-step criterion for the
 * self-interactions; tau = 0.04 in every SIDM run of the simulation table;
 * Sect. 3.6: a minimum allowed time step).  From the per-particle sums of the
 * last sidm_scatter_step (SIDM_FLAG_SUM_P), the step on which the particle
 * expects tau scatterings:
 *   dt_i = tau * dt_h / sum_j P_ij, raised to dt_min and capped at dt_max
 *          (dt_max for a particle without partners),
 * and its power-of-two bin: the largest dt_max / 2^b not above dt_i,
 * b in [0, n_bins - 1] (the smallest bin if even that is too long).
 *   tau, dt_min, dt_max : 0 < tau, 0 <= dt_min <= dt_max, dt_max > 0
 *   n_bins              : 1..32
 *   dt_dev              : device f64[n_halos], the dt the sums were formed with
 *   dt_out_dev          : out, device f64[N] (may be NULL)
 *   bin_out_dev         : out, device int32[N] (may be NULL)
 *   dt_halo_min_dev     : out, device f64[n_halos], the smallest dt_i of each
 *                         halo (dt_max for an empty halo; may be NULL)
 * Outputs follow the order left by sidm_build_cells.  Requires
 * SIDM_FLAG_SUM_P at creation and a preceding sidm_scatter_step. */
int sidm_timestep_criterion(sidm_ctx* ctx, double tau, double dt_min, double dt_max, int32_t n_bins,
                            const double* dt_dev, double* dt_out_dev, int32_t* bin_out_dev,
                            double* dt_halo_min_dev, cudaStream_t stream);

/* Warm start of the kernel-size search (enabled by default).  When enabled,
 * sidm_build_cells seeds every particle's search with its kernel size from the
 * last sidm_kernel_sizes call (carried through the permutation, so the
 * caller's arrays must still be in the order that call left them, with the
 * same halo layout and N_ngb).  The search then only admits candidates within
 * knn_slack times that size (1.07 by default); a particle with fewer than
 * N_ngb of them is redone from scratch by a second, per-lane launch on the
 * same stream.  The result is the exact k-th distance in
 * every case -- a stale or wrong guess costs time, never accuracy -- so this
 * is the usual SPH practice of starting from the previous smoothing length
 * (Sect. 2: h follows the N_ngb nearest neighbours as particles move).
 *   enable : 0 disables it (every search starts cold), non-zero enables it
 * Host-only; takes effect at the next sidm_build_cells. */
int sidm_warm_start(sidm_ctx* ctx, int32_t enable);


/* ---- allocation-free variant -------------------------------------------- */

/* Limits of sidm_energy_momentum_static. */
#define SIDM_STATIC_MAX_HALOS   64     /* halos per call                                */
#define SIDM_STATIC_MAX_CHUNKS  4096   /* chunks of 16384 particles per call (~67 M)    */

/* Per-halo kinetic energy and momentum, like sidm_energy_momentum, for callers
 * that must not allocate device memory.  (The paper has no counterpart: this
 * is a deployment variant, not a step of the method.)
 *
 * Who needs it: code running inside a host application that owns all device
 * memory of the process -- a framework with its own caching allocator, or a
 * fixed memory budget -- where a library may not call cudaMalloc/cudaFree.
 * This call needs no context and allocates nothing: it calls no cudaMalloc,
 * cudaFree or allocating library routine.  Its scratch (two FP64 words per
 * quantity per chunk and per group of 32 chunks, 268 KiB in all) is a fixed
 * file-scope device array,
 * which every GPU that loads libsidm holds until the process exits.
 *
 * Every call outside stream capture looks up the device address of the
 * scratch array on the current device (cudaGetSymbolAddress, which allocates
 * nothing) and remembers it for that device; a call made while its stream is
 * being captured uses the remembered address, so the first call on a device
 * must come before any stream capture.  Every call shares the same scratch
 * and overwrites what it uses (nothing has to start at zero), so calls that
 * overlap on the GPU -- on different streams, or from different threads --
 * race and must be serialised by the caller.
 *
 * The arithmetic and its order are those of sidm_energy_momentum, so both give
 * the same bits on the same inputs.
 *   n_halos   : 1..SIDM_STATIC_MAX_HALOS
 *   halo_off  : host int64[n_halos+1], halo_off[0] == 0, non-decreasing; the
 *               halos may hold at most SIDM_STATIC_MAX_CHUNKS chunks of 16384
 *               particles together (SIDM_ECAPACITY otherwise)
 *   precision : SIDM_MIXED (vel f32) or SIDM_FP64 (vel f64)
 *   mass_dev  : device f64[n_halos]
 *   vel_dev   : device [3][N] velocities, N = halo_off[n_halos]
 *   out_dev   : device f64[n_halos][4] = (E, px, py, pz)
 *   comp_dev  : device f64[n_halos][4] residual compensation terms, or NULL
 * Returns SIDM_OK, SIDM_EINVAL (bad argument, or a first call on a device
 * made during stream capture), SIDM_ECAPACITY (too many chunks) or
 * SIDM_ECUDA (device lookup or launch failed); sidm_static_last_error() gives
 * the reason.  Asynchronous on the stream. */
int sidm_energy_momentum_static(int32_t n_halos, const int64_t* halo_off, int32_t precision,
                                const double* mass_dev, const void* vel_dev, double* out_dev,
                                double* comp_dev, cudaStream_t stream);

/* Message of the last failed sidm_energy_momentum_static call of the calling
 * thread ("" after a successful call; never NULL). */
const char* sidm_static_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SIDM_H */
