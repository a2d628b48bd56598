/*
 * evol.h -- C ABI of the GB300 (sm_103a) tree + SPH force step of EvoL
 * (Merlin et al., arXiv:0912.1786, "EvoL: the new Padova T-SPH parallel code").
 *
 * One call of evol_step computes, for N particles of which the first n_gas are SPH gas:
 *   - the Barnes-Hut oct-tree of cubes with monopole + quadrupole node moments (Sect. 2.2),
 *   - adaptive softening lengths eps_i = eta n_i^{-1/3} with the correction terms Upsilon, X
 *     (Sect. 2.1, Eqs. rho0, etan, zeta; App. B),
 *   - smoothing lengths h_i = eta n_i^{-1/3} from the gas number density, the mass density
 *     rho_i and the variable-mass grad-h terms Omega*_i, zeta_i (Sect. 3, Eqs. hn, nsum,
 *     densitySPH, drhodr),
 *   - the gravitational acceleration by a tree walk with the opening criterion
 *     r > l/theta + delta (Eq. opcrit), symmetrised softened pair forces and the adaptive
 *     softening correction (Eq. dLgravdr; App. B),
 *   - the SPH pressure + artificial-viscosity acceleration and du/dt (Eqs. motionvarmass1,
 *     thermalvarmass1, mu_visc; App. B), with the Thomas-Couchman kernel gradient (Sect. 3
 *     footnote) and nearest-image periodic axes (Sect. 4.3),
 *   - optionally periodic gravity in a cube by the Ewald method (Sect. 4.3),
 *   - optionally the other dissipation terms of Sect. 3.3.3: the signal-velocity viscosity
 *     (Eqs. pvsig, vsig), the Balsara limiter, per-particle alpha with its time derivative
 *     (Eq. alphaswitch) and the artificial conductivity with per-particle alpha^u.
 *
 * Conventions common to every entry point:
 *   - All particle and output pointers are DEVICE pointers (cudaMalloc'd or torch tensors),
 *     float32, structure-of-arrays, in the caller's order, owned by the caller.  The one
 *     exception is evol_step_host, which takes host pointers.
 *   - Gas particles are the first n_gas entries of every per-particle array.
 *   - Calls are asynchronous on the stream given to evol_create.  A call returns EVOL_OK or
 *     an argument / launch error at once; errors found on the device (list overflow,
 *     no root for a length, NaN) are recorded in the context and returned by evol_sync.
 *   - A context is not thread-safe.  There is no host (CPU) fallback: a context can only be
 *     created on a CUDA device.
 */
#ifndef EVOL_H
#define EVOL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------ */
#define EVOL_OK          0
#define EVOL_EINVAL     -1   /* bad argument (NULL pointer, n out of range, bad parameter) */
#define EVOL_ENOMEM     -2   /* n exceeds the context capacity, or device allocation failed */
#define EVOL_ECUDA      -3   /* a CUDA runtime call failed */
#define EVOL_EOVERFLOW  -4   /* a fixed-capacity device list (nodes, neighbour candidates) overflowed */
#define EVOL_ENOCONV    -5   /* a smoothing/softening length has no root or did not converge */
#define EVOL_ETIMEOUT   -6   /* a bounded device wait gave up */
#define EVOL_ENAN       -7   /* a non-finite value was produced */
#define EVOL_ESTATE     -8   /* call order violated (e.g. forces before density) */

/* ---- dissipation variants (Sect. 3.3.3) ------------------------------------------------ */
#define EVOL_VISC_MONAGHAN        0  /* Pi = (-alpha cbar mu + beta mu^2) / rhobar (Eq. mu_visc) */
#define EVOL_VISC_SIGNAL          1  /* Pi = -alpha v^sig w / rhobar (Eqs. pvsig, vsig) */
#define EVOL_COND_VSIG_SOUND      0  /* conductivity signal speed: v^sig of Eq. vsig */
#define EVOL_COND_VSIG_PRESSURE   1  /* sqrt(|P_i - P_j| / rhobar) */
#define EVOL_COND_SRC_SQRTU       0  /* conductivity switch source h |lap u| / sqrt(u) */
#define EVOL_COND_SRC_LINEAR      1  /* 0.1 h |lap u| */

/* ---- SPH schemes (Sect. 3) ------------------------------------------------------------ */
#define EVOL_SPH_LAGRANGIAN       0  /* h from the n-h relation h^3 n(h) = eta^3, grad-h terms kept */
#define EVOL_SPH_STANDARD         1  /* h with N = n_nei_sph (rounded) gas particles, the particle
                                        itself included, inside 2h: h = (r_(N) + r_(N+1)) / 4 from
                                        the N-th and (N+1)-th smallest gas distances; grad-h terms
                                        dropped (Omega* = 1, zeta = 0) */

/* ---- precision forms -------------------------------------------------------------- */
#define EVOL_FP32_PLAIN  0   /* FP32 moments and FP32 accumulation of per-particle sums */
#define EVOL_FP32_MIXED  1   /* FP64 multipole/centre-of-mass accumulation; the gravity totals
                                compensated (TwoSum of blocked FP32 partial sums, read out in
                                FP64); the walk arithmetic stays FP32 */

typedef struct evol_ctx evol_ctx;   /* opaque; owns every device scratch buffer */

/* Particles (Sect. 1: each particle carries mass, position, velocity, plus for gas the
 * internal energy; Sect. 3.2: gas carries both eps and h).  Length n (u: n_gas). */
typedef struct {
    int64_t n;             /* number of particles, 0 <= n <= the context capacity */
    int64_t n_gas;         /* the first n_gas particles are gas, 0 <= n_gas <= n */
    const float *x, *y, *z;
    const float *vx, *vy, *vz;
    const float *m;        /* masses, > 0 */
    const float *u;        /* specific internal energy of gas particles (length n_gas) */
    float *h;              /* in: starting guess (> 0) for gas; out: solved smoothing length */
    float *eps;            /* in: softening (fixed) or starting guess (adaptive); out: solved */
    const float *alpha;    /* per-particle viscosity alpha_i (length n_gas); read only with
                              variable_alpha, required then */
    const float *alpha_u;  /* per-particle conductivity alpha^u_i (length n_gas); read only with
                              conduction, required then */
} evol_particles;

/* Parameters (Sect. 5 lists the paper's choices: eta, alpha, beta, gamma, theta). */
typedef struct {
    float theta;               /* opening angle of Eq. opcrit; 0 opens every node (direct sum) */
    float n_nei_sph;           /* target neighbour number N_nei = 4/3 pi (2 eta)^3 for h */
    float n_nei_grav;          /* target neighbour number for the adaptive eps */
    float gamma;               /* adiabatic index of P = (gamma - 1) rho u */
    float alpha, beta;         /* Monaghan viscosity parameters (Eq. mu_visc) */
    float G;                   /* gravitational constant */
    int gravity;               /* 1: compute gravity */
    int sph;                   /* 1: compute SPH density and forces for the gas */
    int adaptive_softening;    /* 1: eps solved with correction terms; 0: eps fixed as given */
    int use_tc_gradient;       /* 1: Thomas-Couchman gradient in the SPH force and du/dt */
    int periodic_mask;         /* bit a set: axis a periodic.  SPH: any axes (nearest image).  With
                                  gravity only 7, a cube (equal lengths): periodic gravity by the
                                  Ewald method (Sect. 4.3) -- nearest images plus the replicas'
                                  correction, tabulated on a 65^3 octant grid and interpolated
                                  trilinearly, for every pair and every far node's monopole; the
                                  potential includes the zero-mean periodic term and the particle's
                                  own replicas; a node is taken at the nearest image of its centre
                                  of mass (direct + correction is periodic: any image serves), and
                                  nodes of side above L/8 are opened; not with evol_step_batched */
    float periodic_lo[3], periodic_hi[3];
    int precision;             /* EVOL_FP32_PLAIN or EVOL_FP32_MIXED */
    int leaf_size;             /* a cube is split while it holds more than leaf_size particles
                                  (1..64; 0 = default 8).  Changes cost, not the definition. */
    int group_size;            /* particles per warp group in the walks: 0 or 32 */
    /* Dissipation variants (Sect. 3.3.3).  A zeroed block is the Monaghan viscosity with the
     * constant alpha and beta above.  Every variant uses, per pair, w_ij = v_ij.r_ij/|r_ij| and
     * the signal velocity v^sig_ij = c_i + c_j - min(w_ij, 0) (Eq. vsig; the min keeps it >= c_i + c_j
     * for receding pairs), and per particle v^sig_i = max(2 c_i, max_j v^sig_ij). */
    int visc_form;             /* EVOL_VISC_MONAGHAN or EVOL_VISC_SIGNAL */
    int balsara;               /* 1: Pi_ij times (f_i + f_j)/2, f_i = |div v| / (|div v| + |curl v|
                                  + balsara_eta c_i/h_i) (0 where that denominator is 0) */
    float balsara_eta;         /* >= 0; the paper's value is about 1e-4 */
    int variable_alpha;        /* 1: alpha_ij = (alpha_i + alpha_j)/2 from p->alpha (either form),
                                  and out->dalpha = -(alpha_i - alpha_min)/tau_i
                                  + alpha_source f_i max(0, -div v_i), tau_i = alpha_tau h_i/v^sig_i */
    float alpha_min, alpha_tau, alpha_source;   /* paper: 0.01, 0.1, 0.75; alpha_tau > 0 */
    int conduction;            /* 1: du_i/dt += sum_j m_j Pi^u_ij |gradbar W_ij| with
                                  Pi^u_ij = -(alpha^u_i + alpha^u_j)/2 v^u (u_i - u_j) / rhobar_ij,
                                  and out->dalpha_u = -(alpha^u_i - alpha_u_min)/tau_i + S^u_i */
    int cond_vsig;             /* v^u: EVOL_COND_VSIG_SOUND or EVOL_COND_VSIG_PRESSURE */
    int cond_source;           /* S^u from Brookshaw's lap u_i = sum_j 2 m_j (u_i - u_j)/rho_j
                                  |gradbar W_ij|/r_ij: EVOL_COND_SRC_SQRTU or EVOL_COND_SRC_LINEAR */
    float alpha_u_min;         /* paper: 0 */
    int sph_scheme;            /* EVOL_SPH_LAGRANGIAN (0) or EVOL_SPH_STANDARD; the standard scheme
                                  needs 1 <= n_nei_sph (rounded) <= 335 */
    int length_group;          /* particles per group walk of the length solves (they share one
                                  tree walk listing the leaves near them): 0 = 8, or 1..32.
                                  Changes cost, not the definition. */
} evol_params;

/* Outputs, caller order.  Any pointer may be NULL (not written). */
typedef struct {
    float *ax, *ay, *az;       /* length n: total acceleration (gravity + SPH) */
    float *pot;                /* length n: Phi_i = G sum_j m_j phi(r_ij, eps_i), self term included */
    float *rho;                /* length n_gas: mass density (Eq. densitySPH) */
    float *P, *c;              /* length n_gas: pressure and sound speed */
    float *omega, *zeta;       /* length n_gas: Omega*_i and zeta_i (Eq. drhodr) */
    float *dudt;               /* length n_gas: du/dt (Eq. thermalvarmass1) */
    float *ups, *X;            /* length n: Upsilon_i and X_i (adaptive softening) */
    float *dalpha;             /* length n_gas: d alpha_i / dt (variable_alpha; else not written) */
    float *dalpha_u;           /* length n_gas: d alpha^u_i / dt (conduction; else not written) */
} evol_outputs;

/* Create a context for up to max_n particles on the current CUDA device; every device
 * buffer is allocated here (about 1 KB per particle of capacity).  stream: a cudaStream_t
 * (NULL = the legacy default stream).  Returns EVOL_EINVAL, EVOL_ENOMEM or EVOL_ECUDA on
 * failure, with *ctx set to NULL. */
int evol_create(evol_ctx **ctx, int64_t max_n, void *stream);
int evol_destroy(evol_ctx *ctx);

/* Tree build (Sect. 2.2): root cube, 63-bit Morton keys (21 bits per axis), stable radix sort,
 * pre-order node list (a cube is split into its non-empty octants while it holds more than
 * leaf_size particles, down to level 21), node moments (mass, centre of mass, traceless
 * quadrupole about it, delta = |geometric centre - centre of mass|, particle bounding box). */
int evol_build_tree(evol_ctx *ctx, const evol_particles *p, const evol_params *prm);

/* SPH density (Sect. 3, Eqs. hn, nsum, densitySPH, drhodr; Sect. 3.1 gather view): solves
 * h_i^3 n_i(h_i) = eta^3 for every gas particle by Newton iteration with a bisection bracket
 * on a cached candidate list, then rho, Omega*, zeta, P and c.  Builds the tree first if
 * evol_build_tree was not called for these particles.  Writes p->h and the density outputs. */
int evol_sph_density(evol_ctx *ctx, evol_particles *p, const evol_params *prm, evol_outputs *out);

/* Gravity (Sect. 2.1-2.2; App. B): with adaptive softening solves eps for every particle and
 * Upsilon, X; then the tree walk.  OVERWRITES ax, ay, az and pot. */
int evol_gravity(evol_ctx *ctx, evol_particles *p, const evol_params *prm, evol_outputs *out);

/* SPH forces (Eqs. motionvarmass1, thermalvarmass1; App. B): pairs with
 * r_ij < 2 max(h_i, h_j).  ADDS the SPH acceleration to ax, ay, az and writes dudt.
 * Requires evol_sph_density on the same particles first (else EVOL_ESTATE). */
int evol_sph_forces(evol_ctx *ctx, const evol_particles *p, const evol_params *prm, evol_outputs *out);

/* The whole force step: build + eps solve + h solve + one fused walk for gravity and SPH
 * forces (Sect. 3.1: "the gravitational force is evaluated together with the construction
 * of the neighbour list").  Recorded once into a CUDA graph per (pointers, n, parameters)
 * and replayed afterwards; no host synchronisation inside. */
int evol_step(evol_ctx *ctx, evol_particles *p, const evol_params *prm, evol_outputs *out);

/* Batched step over nsys independent systems (no forces between systems): the particles of
 * system k are positions [sys_offsets[k], sys_offsets[k+1]) of every per-particle array
 * (sys_offsets: HOST array of nsys + 1 values, 0 = sys_offsets[0] <= ... <= sys_offsets[nsys] = n;
 * gas still means the first n_gas particles overall).  Each system gets its own root cube and
 * tree, exactly as evol_step would build for it alone; all systems go through the same kernel
 * launches (one per phase, CUDA-graph captured per nsys).  1 <= nsys <= 65536, else EVOL_EINVAL.
 * Synchronises the context stream on entry when the offsets differ from those of the previous
 * step on this context (they are staged in pinned host memory); repeated steps of one batch do
 * not synchronise. */
int evol_step_batched(evol_ctx *ctx, const int64_t *sys_offsets, int nsys, evol_particles *p,
                      const evol_params *prm, evol_outputs *out);

/* Kick-drift-kick leapfrog with a fixed step dt (Sect. 4.1): one force step at the start, then
 * nsteps times: v += a dt/2 (and u += du/dt dt/2 for gas); x += v dt (periodic axes wrapped
 * into [periodic_lo, periodic_hi)); force step; v += a dt/2, u += du/dt dt/2.  The particle
 * arrays x, y, z, vx, vy, vz and u are updated IN PLACE, so they must be writable device
 * memory despite their const qualifiers (so are alpha and alpha_u, kicked with their time
 * derivatives like u, when variable_alpha / conduction is on); h and eps carry over as the next step's starting
 * guesses.  out receives the outputs of the last force step (any field may be NULL).  One KDK
 * step (kicks, drift and the force phases) is recorded into CUDA graphs once and replayed
 * nsteps times.  Returns EVOL_EINVAL for nsteps < 0 or dt not finite. */
int evol_kdk(evol_ctx *ctx, evol_particles *p, const evol_params *prm, evol_outputs *out, float dt, int nsteps);

/* Global time step of the integrator (Sect. 4.2).  Each eta scales one per-particle criterion;
 * 0 leaves the criterion out.  With L = min(eps_i, h_i) (eps alone for non-gas particles):
 *   eta_acc sqrt(L/|a|),  eta_vel L/|v|,  eta_av |v|/|a|,
 *   eta_courant h / (h |div v| + c + 1.2 (alpha c + beta max_j |mu_ij|))     (gas; alpha_i
 *                                                        with variable_alpha, in both forms),
 *   eta_u |u / (du/dt)|                                                     (gas).
 * (The paper prints the second and third criteria under square roots that do not give a time;
 * they are taken as written here.)  dt is the smallest criterion over all particles, clamped to
 * [dt_min, dt_max] (dt_max where no criterion applies). */
typedef struct {
    float eta_acc, eta_vel, eta_av, eta_courant, eta_u;
    float dt_min, dt_max;           /* 0 <= dt_min <= dt_max, dt_max > 0 */
    int predicted_velocity;         /* 1: SPH terms use v_n + a_n dt and u_n + (du/dt)_n dt (Sect. 4.1) */
    int predict_lengths;            /* 1: each solve starts from L exp(div v dt / 3), the continuity
                                       equation's prediction (Sect. 2.1); changes cost, not results */
} evol_integrator;

/* Kick-drift-kick leapfrog with the global time step (Sect. 4.1-4.2), entirely on the device:
 * one force step at the start, then nsteps times: dt from the criteria of the last force step
 * (a device minimum over all particles), v += a dt/2 (u += du/dt dt/2 for gas), x += v dt (periodic
 * axes wrapped), the predicted starting lengths, a force step (velocity divergences and the
 * largest |mu| per gas particle included), v += a dt/2, u += du/dt dt/2.  One step is recorded
 * into a CUDA graph once and replayed nsteps times; dt never leaves the device.  x, y, z, vx, vy,
 * vz, u, h and eps are updated IN PLACE (writable device memory despite the const qualifiers).
 * *time (host, in/out, may be NULL) advances by the sum of the steps; *last_dt (may be NULL)
 * receives the last step.  out receives the outputs of the last force step.  Synchronises the
 * stream before returning.  EVOL_EINVAL for nsteps < 0, negative etas or a bad dt range. */
int evol_run(evol_ctx *ctx, evol_particles *p, const evol_params *prm, const evol_integrator *ip,
             evol_outputs *out, int nsteps, double *time, float *last_dt);

/* Individual power-of-two time steps (Sect. 4.2.1).  Steps are dt_max / 2^k, 0 <= k <= max_bin, on an
 * integer timeline of T = 2^max_bin ticks per largest step.  Each particle's step [tb, te] has a
 * power-of-two length that divides tb; the step is the largest power of two not longer than the
 * particle's criterion (those of evol_integrator; the finest where a criterion is below one tick),
 * and it can grow only where the current time is a multiple of the new length, so that everyone is
 * synchronised at the end of every largest step. */
typedef struct {
    evol_integrator crit;           /* criteria (etas), predicted_velocity, and dt_max = the largest
                                       step; dt_min and predict_lengths are not used */
    int max_bin;                    /* 0 <= max_bin <= 30 */
    float wake_factor;              /* 0: no wake-up; else > 1 (the paper suggests 4 to 8) */
} evol_bins;

/* KDK leapfrog with individual steps (Sect. 4.1, 4.2.1), entirely on the device, for nlargest
 * largest steps from a synchronised start.  A force step of all particles starts the run; then
 * each system step: t_next = the earliest step end; every particle drifts to t_next with its
 * half-kicked velocity; the particles whose step ends there (active) are the only ones evaluated --
 * tree of all particles at their drifted positions, eps and h solves, density and force walks over
 * the active list -- while the others keep the lengths, densities and accelerations of their last
 * evaluation (their velocity and u predicted to t_next for the SPH terms when predicted_velocity);
 * active particles get their second half kick, a new step and its first half kick.  With
 * wake_factor > 1, an inactive gas particle whose step exceeds wake_factor times the step just
 * completed by an active SPH neighbour ends its step at the first multiple of the largest power of
 * two <= wake_factor x that step, and the part of its first half kick beyond it is taken back.
 * One system step is a CUDA graph recorded once and replayed; the host reads the system time
 * after each (one stream synchronisation per system step).  x, y, z, vx, vy, vz, u, h, eps (and
 * alpha, alpha_u with their switches) are updated IN PLACE.  *time (may be NULL) advances by
 * nlargest * dt_max; stats (may be NULL): [0] system steps, [1] particle evaluations including the
 * start, [2] wake-ups, [3] new steps whose criterion was below one tick.  out receives the last
 * force step's outputs (every particle is active in it).  Single system only (no evol_step_batched
 * offsets).  EVOL_EINVAL for bad parameters. */
int evol_run_bins(evol_ctx *ctx, evol_particles *p, const evol_params *prm, const evol_bins *bp, evol_outputs *out,
                  int nlargest, double *time, int64_t stats[4]);

/* evol_step on HOST buffers: copies the inputs host -> device into context-owned buffers,
 * runs the step and copies every non-NULL output (and h, eps) back, then synchronises.
 * The particle and output pointers of this call are host pointers (pinned memory is
 * fastest).  Returns the step status (as evol_sync). */
int evol_step_host(evol_ctx *ctx, evol_particles *p_host, const evol_params *prm, evol_outputs *out_host);

/* Autotuner for the cost parameters of the step (never theta or the neighbour numbers): times
 * evol_step on these particles for each candidate leaf size and returns the fastest in
 * *best_leaf.  candidates: host array of ncand leaf sizes in 1..64 (NULL: {4, 8, 12, 16, 24, 32});
 * after one untimed step (clock ramp-up) each candidate gets one untimed step (graph recording)
 * and reps >= 1 timed steps, each started from the caller's h and eps as passed in (restored
 * before every step, outside the timed interval); ms_out (host, ncand floats, may be NULL)
 * receives each candidate's median step time.  On return h and eps hold the caller's starting
 * values again; out receives the last run's results.  Synchronous. */
int evol_autotune(evol_ctx *ctx, evol_particles *p, const evol_params *prm, evol_outputs *out,
                  const int *candidates, int ncand, int reps, int *best_leaf, float *ms_out);

/* The same autotuner for the length solves' group size (prm->length_group), at the parameters
 * given (leaf size included): candidates in 1..32 (NULL: {4, 8, 16, 32}); *best receives the fastest,
 * ms_out (may be NULL) each candidate's median step time.  Same timing protocol as evol_autotune. */
int evol_autotune_length_group(evol_ctx *ctx, evol_particles *p, const evol_params *prm, evol_outputs *out,
                               const int *candidates, int ncand, int reps, int *best, float *ms_out);

/* The autotuners for a batch of independent systems: the same protocol, timing
 * evol_step_batched with these offsets (same rules as evol_step_batched; a bad offset array
 * returns its EVOL_EINVAL from the first step).  which = EVOL_TUNE_LEAF_SIZE (candidates in 1..64,
 * NULL: {4, 8, 12, 16, 24, 32}) or EVOL_TUNE_LENGTH_GROUP (candidates in 1..32, NULL:
 * {4, 8, 16, 32}); any other value is EVOL_EINVAL.  *best receives the fastest candidate, ms_out
 * (may be NULL) each candidate's median step time.  Synchronous. */
#define EVOL_TUNE_LEAF_SIZE    0
#define EVOL_TUNE_LENGTH_GROUP 1
int evol_autotune_batched(evol_ctx *ctx, const int64_t *sys_offsets, int nsys, evol_particles *p,
                          const evol_params *prm, evol_outputs *out, int which, const int *candidates, int ncand,
                          int reps, int *best, float *ms_out);

/* Wait for the context stream and return the first device-side error recorded since the
 * previous evol_sync (then clear it), or EVOL_OK. */
int evol_sync(evol_ctx *ctx);

/* FP64 totals of the last step (valid after evol_sync): [0..2] sum m v, [3..5] sum m a,
 * [6] kinetic energy, [7] thermal energy sum m u, [8] potential energy 1/2 sum m Phi,
 * [9] sum m (v.a + du/dt) over gas (SPH energy balance), [10] sum m, [11] node count,
 * [12] far-node interactions, [13] particle-particle pairs, [14] SPH pairs,
 * [15] length-solve iterations (sum over particles). */
int evol_get_diagnostics(evol_ctx *ctx, double out[16]);

/* Work counters of the last step (valid after evol_sync), 32 values:
 *   [0] far-node interactions   [1] particle pairs (all)   [2] SPH pairs
 *   [3] length-solve iterations (sum over particles)
 *   [4] [5] [6] work-queue positions of the walk, the h solve and the eps solve
 *   [7] nonzero if a traversal hit its pop or climb cap
 *   [8] gravity pairs inside 2 max(eps_i, eps_j) (softened; the rest are Newtonian)
 *   [9] lane slots of the far-node loop, [10] of the pair loop's first pass, [11] of its second
 *       pass (32 per entry or trip: interactions / slots is the fraction of busy lanes)
 *   [12] nodes popped by the force walk's groups, [13] of them tested lane by lane (neither
 *        accepted nor opened for the whole group), [14] leaves opened, [15] internal nodes opened
 *   length solves, eps at [16..19] and h at [20..23]: [+0] neighbour gathers from a group's leaf
 *        list, [+1] gathers by a particle's own tree walk, [+2] neighbour lists that overflowed,
 *        [+3] group leaf lists that overflowed
 *   [24] eps-solve and [25] h-solve Newton iterations (sum over particles)
 *   [26..31] zero */
int evol_get_counters(evol_ctx *ctx, uint64_t out[32]);

/* Debug copies of internal state (valid after evol_sync), into host memory of cap bytes.
 * Returns the number of ELEMENTS available (whatever cap), or a negative status.
 *   EVOL_DBG_KEYS   uint64[n]   Morton keys in sorted order
 *   EVOL_DBG_PERM   int32[n]    sorted position -> caller index
 *   EVOL_DBG_NODES  int32[5*nn] begin[nn], end[nn], level[nn], next[nn], nchild[nn] (pre-order)
 *   EVOL_DBG_CUBE   double[4]   root corner x, y, z and side
 *   EVOL_DBG_MOMENTS float[20*nn] per node: M, com xyz, Q xx yy zz xy xz yz, delta,
 *                              bbox min xyz, bbox max xyz, 2 epsmax, 2 hmax (-1: no gas),
 *                              (l/theta + delta)^2
 *   EVOL_DBG_HASHES uint64[3*n] caller order: far-node set, near-leaf set, SPH neighbour set
 *   EVOL_DBG_COUNTS int32[3*n]  caller order: far nodes, particle pairs, SPH pairs
 *   EVOL_DBG_FLOW   float[3*n]  caller order: div v with the softening kernel, div v with the
 *                               smoothing kernel (gas), largest |mu_ij| of the viscosity (gas)
 *   EVOL_DBG_DISS   float[5*n]  caller order, gas: div v and |curl v| with the smoothing kernel,
 *                               Balsara f_i, v^sig_i, Brookshaw lap u_i (as printed, with
 *                               |gradbar W|; conduction only)
 *   EVOL_DBG_BINS   int64[2*n]  caller order: step start tb and end te (ticks) after evol_run_bins
 * Hashes and per-particle counts are written only while check mode is on; the divergences only
 * by evol_run's force steps or when a dissipation variant needs them (Balsara, variable alpha);
 * EVOL_DBG_DISS only by steps with a dissipation variant on. */
#define EVOL_DBG_KEYS     1
#define EVOL_DBG_PERM     2
#define EVOL_DBG_NODES    3
#define EVOL_DBG_CUBE     4
#define EVOL_DBG_MOMENTS  5
#define EVOL_DBG_HASHES   6
#define EVOL_DBG_COUNTS   7
#define EVOL_DBG_FLOW     8
#define EVOL_DBG_DISS     9
#define EVOL_DBG_BINS    10
int64_t evol_get_debug(evol_ctx *ctx, int what, void *host_dst, int64_t cap_bytes);

/* Check mode (0/1): the walks also record, per particle, order-independent 64-bit hashes
 * (splitmix64 of the id, summed) of the accepted-node set, the opened-leaf set and the SPH
 * neighbour set, and their sizes.  Slower; off by default. */
int evol_set_check_mode(evol_ctx *ctx, int on);

/* Per-warp traversal-stack capacity of the tree walks, in entries: 32 <= entries <= the
 * capacity evol_create allocated (4096); 0 restores that capacity.  A walk that would need more
 * stops before writing past it and the step reports EVOL_EOVERFLOW.  Lowering it serves to test
 * that path.  Takes effect from the next call.  Returns EVOL_EINVAL out of range. */
int evol_set_stack_limit(evol_ctx *ctx, int64_t entries);

/* Event timings (ms) of the phases of the last evol_step: [0] build, [1] eps solve,
 * [2] h solve, [3] force walk, [4] total. Valid after evol_sync. */
int evol_get_timings(evol_ctx *ctx, float out[5]);

/* Allocation-free key + sort stage (the paper has no counterpart: this is a service for callers
 * that may not allocate device memory where they call us, e.g. from a host callback or a
 * framework hook that must not re-enter the device allocator, or in a process whose device
 * memory is fixed at start-up).  Computes the root cube, the 63-bit Morton keys and the stable
 * radix sort exactly as evol_build_tree does and returns the sorted keys and the permutation
 * (sorted position -> caller index).  x, y, z, keys_sorted (n) and perm (n) are DEVICE pointers
 * owned by the caller; keys_sorted and perm are also used as working space.  cube (device,
 * 4 doubles: corner x, y, z, side) may be NULL.  stream: a cudaStream_t (NULL = legacy stream).
 * Allocates nothing: its scratch is a static device array of EVOL_NOALLOC_MAX_N * 12 bytes
 * (768 KiB) held by every GPU that loads the library until the process exits.
 * Set-up: the array lives in the library's device module, which the CUDA runtime loads on a
 * device at its first use there -- that load is what places the array in device memory.  A call
 * with n == 0 (pointers may be NULL) does this set-up for the current device and launches
 * nothing; evol_create also does it for its device.  Make that call at start-up, where
 * allocating is still allowed, before any stream capture, and again after a cudaDeviceReset
 * (which unloads the module).  Without it, the first call with n > 0 on a device does the set-up.
 * All calls share the array: calls that overlap on the GPU race.  Returns EVOL_EINVAL if n < 0
 * or n > EVOL_NOALLOC_MAX_N, or a pointer is NULL (n > 0); EVOL_ECUDA if the set-up fails;
 * asynchronous otherwise. */
#define EVOL_NOALLOC_MAX_N 65536
int evol_sort_keys_noalloc(int64_t n, const float *x, const float *y, const float *z, uint64_t *keys_sorted,
                           int32_t *perm, double *cube, void *stream);

/* Measurement helper (not part of the paper's method): the device's FP32 throughput, measured
 * by kernels in which every thread runs eight independent chains of `iters` x 64 fused
 * multiply-adds (2 operations each) over 2048 resident threads per SM, on the current device:
 * once with scalar FP32 FMAs (*tflops) and once with packed two-wide FMAs (fma.rn.f32x2;
 * *tflops_packed, may be NULL).  *ms (may be NULL) receives the scalar kernel's duration.
 * Synchronous; allocates a few bytes of device memory for the duration of the call.  The larger
 * rate is the peak the force walk's FP32 roofline fraction is quoted against. */
int evol_fp32_peak(int iters, double *tflops, double *tflops_packed, float *ms);

const char *evol_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* EVOL_H */
