// Internal declarations of the GB300 force-step library: context layout, FP32 kernel
// functions and small device helpers.  Not part of the C ABI (see include/evol.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/evol.h"

#define EVOL_MAXLEVEL 21          // 21 bits per axis, 63-bit Morton keys
#define EVOL_WARP 32
#define EVOL_NCOUNTERS 32
#define EVOL_PI_F 3.14159265358979f

// ---- device error word: first error wins ------------------------------------------------
__device__ __forceinline__ void evol_flag(int *err, int code)
{
    atomicCAS(err, 0, code);
}

// ---- sorted per-particle state packed for the walks --------------------------------------
// pos  : x, y, z, m
// grav : 1/eps, X/Upsilon, h (0 for non-gas), zeta/Omega* (0 for non-gas)
// hydro: vx, vy, vz, P/rho^2
// snd  : c, rho, 1/h (0 for non-gas), P
// diss : alpha, Balsara f, u, alpha^u (gas, only with a dissipation variant on)
struct evol_dev {
    // particles, sorted order
    float4 *pos, *vel, *grav, *hydro, *snd;
    float *vah;              // v . a_hyd per particle (energy balance diagnostic)
    int32_t *orig;           // sorted -> caller index
    int32_t *inv;            // caller -> sorted index
    float *len_h, *len_eps;  // solved lengths, sorted
    float *nh, *omega, *zeta, *rho;     // gas outputs (sorted; n entries, non-gas unused)
    float *neps, *ups, *X;              // softening outputs (sorted)
    float4 *acc;             // ax, ay, az, pot (sorted)
    float *divv_h, *divv_e;  // velocity divergence with the smoothing / softening kernel (sorted)
    float *mumax;            // largest |mu_ij| of the viscosity per gas particle (sorted)
    float4 *diss;            // dissipation operands: alpha_i, Balsara f_i, u_i, alpha^u_i (sorted, gas)
    float *curlv_h;          // |curl v| with the smoothing kernel (sorted)
    float *vsig, *lapu;      // v^sig_i and Brookshaw lap u_i of the last walk (sorted)
    float *dalpha, *dalpha_u;    // d alpha/dt and d alpha^u/dt (sorted)
    // individual time steps (caller order unless noted)
    unsigned long long *tb, *te;    // step [tb, te] of each particle, in ticks
    int32_t *bact;                  // 1: the particle is active in the current system step
    float *pred_tau;                // t_now - (tb + te)/2 (time units): prediction of v and u
    float *pers;                    // last evaluation: rho, Omega*, zeta, Upsilon, X, div v, |curl v| (7 x cap)
    int32_t *actf, *acts, *act;     // sorted: active flags, their exclusive scan (+ total), the list
    // force walk: per super-group (8 groups of 32 list entries) the nodes its bounds accept for all
    // its particles (EVOL_SG_ACAP each), the frontier its groups start from (EVOL_SG_FCAP each), and
    // their counts (-1: walk from the root)
    int32_t *sg_acc, *sg_front;
    int2 *sg_info;
    unsigned *nbmin;                // sorted: smallest active-neighbour step (wake-up)
    unsigned long long *bt;         // [0] t_sys [1] t_next (ticks); [2..5] run counts
    float4 *ewald;                  // periodic gravity: correction table (f, g) for L = 1
    float *dt;               // integrator scalars: [0] time step, [1] criterion minimum (as bits)
    double *time;            // integrator time
    float *dudt;             // sorted
    // sort
    uint64_t *keys_a, *keys_b;
    int32_t *vals_a, *vals_b;
    uint32_t *hist;          // 256 * nblocks
    // tree construction
    int8_t *lcp;             // d_i: common octal digits of keys i-1, i (-1: i starts a system)
    int32_t *cnt, *base;     // nodes beginning at each sorted position, and its exclusive scan
    int32_t *scan_part;      // scan block partials
    // nodes (pre-order)
    int32_t *nbeg, *nend, *nlev, *nnext, *nparent, *nnch, *narrive;
    float4 *nA;              // com x, y, z, ropen^2 with ropen = l/theta + delta (Eq. opcrit)
    float4 *nB;              // bbox centre x, y, z, 2 hmax (-1: no gas; 0 until lengths are known)
    float4 *nC;              // bbox half widths x, y, z, 2 epsmax
    float4 *nQ0;             // Qxx, Qyy, Qzz, M
    float4 *nQ1;             // Qxy, Qxz, Qyz, delta
    double *nM64, *nC64, *nQ64;         // FP64 moments (mixed precision): M, com[3], Q[6]
    float4 *nBmin, *nBmax;              // particle bounding box (w of nBmin: node holds gas)
    float4 *nCoff;                      // FP32 moments: centre of mass - geometric centre, M
    int4 *nI;                           // walk copy: level | leaf << 8, next, begin, end
    int4 *nK0, *nK1;                    // child ids (up to 8, -1 padded) of internal nodes
    int2 *wstack;                       // per-warp traversal stacks of the force walk
    // length solve scratch: per-lane (distance, mass) neighbour lists of every warp slot
    int32_t *cand_leaf;
    uint32_t *cand_mask;     // unused
    // reductions / counters
    double *diag_part;       // per-block partials of diagnostics
    double *diag;            // 16
    unsigned long long *counters;   // EVOL_NCOUNTERS; indices as evol_get_counters documents
    int *err;
    int32_t *nnodes;         // device node count
    double *cube;            // corner x, y, z, side of every system (4 per system)
    float *fcube;            // the same in float
    int32_t *sys_off;        // system offsets (nsys + 1), sorted order keeps systems contiguous
    int32_t *sys_sorted;     // system of each sorted position
    int32_t *sys_root;       // root node of each system
    float *bbox_part;        // per-block min/max partials
    // check mode
    unsigned long long *hash3;   // 3 per particle (sorted)
    int32_t *cnt3;               // 3 per particle (sorted)
};

struct evol_ctx {
    int64_t cap;             // particle capacity
    int64_t node_cap;
    int device, num_sms;
    cudaStream_t stream;
    evol_dev d;
    int64_t sort_blocks;
    int64_t bbox_blocks;
    int64_t cand_slots, cand_cap;
    int64_t wstack_slots, wstack_cap;
    int64_t wstack_lim;      // entries the walks may use per warp (<= wstack_cap)
    int64_t diag_blocks;
    int host_err;            // first error seen on the host side
    int check_mode;
    int want_divv;           // the length solves also form div v (integrator)
    const float *pred_dt;    // device time step of the predicted pack (integrator), or NULL
    const float *pred_tau;   // per-particle prediction times (individual steps), or NULL
    int persist;             // the un-permute also keeps the last-evaluation state (d.pers)
    int bins_active;         // the walks being recorded take the active list
    int bins_wake;           // and the force walk records the wake-up minimum
    unsigned long long bins_t_end;   // end of the current individual-step run (ticks)
    // state of the last build / density
    int64_t built_n, built_ngas;
    int nsys;                // systems of the current particle set (1 unless batched)
    int nsys_cap;
    int staged_nsys;         // systems whose offsets d.sys_off holds from h_sys_off (0: none)
    int32_t *h_sys_off;      // pinned host staging of the system offsets
    const void *built_x;
    int density_done, eps_done;
    // graph cache for evol_step
    cudaGraphExec_t graph_exec[8];   // one per phase of evol_step
    uint64_t graph_sig;
    // events for phase timings
    cudaEvent_t ev[6];
    // host staging for evol_step_host (device buffers)
    float *stage;            // 12 * cap floats (inputs) + 14 * cap floats (outputs)
    // leapfrog: accelerations and du/dt in caller order, and the recorded KDK step
    float *kdk_acc;
    cudaGraphExec_t kdk_exec;
    uint64_t kdk_sig;
    cudaGraphExec_t run_exec;        // one global-step KDK step (evol_run)
    uint64_t run_sig;
    cudaGraphExec_t bins_exec;       // one system step of evol_run_bins
    uint64_t bins_sig;
    unsigned long long *h_bt;        // pinned host copy of the system time
    int ewald_ready;                 // the Ewald table has been computed
};

// ---- host-side launch helpers (defined in evol_api.cu / tree.cu / walks) ------------------
int evol_launch_build(evol_ctx *c, const evol_particles *p, const evol_params *prm);   // uses c->nsys
int evol_launch_lengths(evol_ctx *c, const evol_particles *p, const evol_params *prm, int mode);
int evol_launch_walk(evol_ctx *c, const evol_particles *p, const evol_params *prm, int do_grav, int do_sph);
int evol_launch_node_lengths(evol_ctx *c, const evol_params *prm, int n_gas);
int evol_launch_unpermute(evol_ctx *c, const evol_particles *p, const evol_outputs *o, int what);
int evol_launch_diagnostics(evol_ctx *c, const evol_particles *p, const evol_params *prm);
int evol_launch_integrator_step(evol_ctx *c, const evol_particles *p, const evol_params *prm, const evol_integrator *ip,
                                int stage);
int evol_launch_bins(evol_ctx *c, const evol_particles *p, const evol_params *prm, const evol_bins *bp, int stage);
int evol_launch_active_list(evol_ctx *c, int n);
int evol_ewald_prepare(evol_ctx *c);

#define EVOL_UNPERM_LENGTHS 1
#define EVOL_UNPERM_DENSITY 2
#define EVOL_UNPERM_ACC     4
#define EVOL_UNPERM_DUDT    8
#define EVOL_UNPERM_EPSOUT  16
#define EVOL_UNPERM_DALPHA  32
#define EVOL_UNPERM_DALPHA_U 64
#define EVOL_UNPERM_ACTIVE  128   // only particles flagged in d.bact
#define EVOL_UNPERM_PERSIST 256   // the persistent last-evaluation state d.pers (individual steps)

// Any dissipation variant of Sect. 3.3.3 on (they act on SPH pairs only).
static inline bool evol_diss_on(const evol_params *prm)
{
    return prm->sph &&
           (prm->visc_form != EVOL_VISC_MONAGHAN || prm->balsara || prm->variable_alpha || prm->conduction);
}
// The switch rates a step writes out (variable alpha, conduction).
static inline int evol_unperm_switches(const evol_params *prm)
{
    return (prm->sph && prm->variable_alpha ? EVOL_UNPERM_DALPHA : 0) |
           (prm->sph && prm->conduction ? EVOL_UNPERM_DALPHA_U : 0);
}
// The Balsara factor (limiter, alpha source) needs div v and |curl v| from the h solve.
static inline bool evol_needs_curl(const evol_params *prm) { return prm->sph && (prm->balsara || prm->variable_alpha); }

static inline int evol_cuda_ok(cudaError_t e) { return e == cudaSuccess ? EVOL_OK : EVOL_ECUDA; }

// ---- FP32 kernel functions (Eqs. spline, softforce, softphi, dphidh; TC gradient) -------
// M4 spline w(u) = 1/4 (2-u)_+^3 - (1-u)_+^3 and its derivative dw/du; W = w / (pi h^3).
__device__ __forceinline__ void evol_w_dw(float u, float &w, float &dw)
{
    float a = fmaxf(2.f - u, 0.f), b = fmaxf(1.f - u, 0.f);
    float a2 = a * a, b2 = b * b;
    w = 0.25f * a2 * a - b2 * b;
    dw = -0.75f * a2 + 3.f * b2;
}

// Softened force kernel divided by r, times eps^3:  eps^3 phi'(r, eps) / r, for u < 2.
__device__ __forceinline__ float evol_gsoft_over_r(float u)
{
    float u2 = u * u;
    if (u < 1.f) return 4.f / 3.f - 1.2f * u2 + 0.5f * u2 * u;
    float u3 = u2 * u;
    return 8.f / 3.f - 3.f * u + 1.2f * u2 - u3 / 6.f - 1.f / (15.f * u3);
}

// Softened potential times eps: eps phi(r, eps), for u < 2.
__device__ __forceinline__ float evol_phisoft(float u)
{
    float u2 = u * u;
    if (u < 1.f) return (2.f / 3.f) * u2 - 0.3f * u2 * u2 + 0.1f * u2 * u2 * u - 1.4f;
    return (4.f / 3.f) * u2 - u2 * u + 0.3f * u2 * u2 - u2 * u2 * u / 30.f - 1.6f + 1.f / (15.f * u);
}

// dphi/deps times eps^2, for u < 2 (Eq. dphidh with the -3/2 u^4 sign of the outer branch).
__device__ __forceinline__ float evol_dphideps(float u)
{
    float u2 = u * u;
    if (u < 1.f) return -2.f * u2 + 1.5f * u2 * u2 - 0.6f * u2 * u2 * u + 1.4f;
    if (u < 2.f) return -4.f * u2 + 4.f * u2 * u - 1.5f * u2 * u2 + 0.2f * u2 * u2 * u + 1.6f;
    return 0.f;
}

// (dW/dr) / r times pi h^5, exact spline derivative: w'(u)/u.
__device__ __forceinline__ float evol_dw_over_u(float u)
{
    if (u < 1.f) return -3.f + 2.25f * u;
    float a = fmaxf(2.f - u, 0.f);
    return -0.75f * a * a / u;
}

// Thomas-Couchman gradient: (dW/dr)/r times pi h^5 (Sect. 3 footnote).
__device__ __forceinline__ float evol_tc_over_u(float u)
{
    if (u < 2.f / 3.f) return -1.f / u;
    if (u < 1.f) return -0.75f * (4.f - 3.f * u);
    float a = fmaxf(2.f - u, 0.f);
    return -0.75f * a * a / u;
}

// splitmix64 finaliser (Steele, Lea & Flood 2014), for interaction-set hashes in check mode.
__device__ __forceinline__ unsigned long long evol_mix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float evol_wrap(float d, float len, int periodic)
{
    return periodic ? d - len * rintf(d / len) : d;
}

// ---- force-walk super-groups: groups of 32 list entries per super-group, list capacities -----
#define EVOL_SG_GROUPS 8
#define EVOL_SG_ACAP 3072
#define EVOL_SG_FCAP 768

// ---- periodic gravity (Ewald, Sect. 4.3) ----------------------------------------------------
// Correction table for a cube of side 1: (f_x, f_y, f_z, g) at the grid points (i, j, k) / (2 N) of the
// octant [0, 1/2]^3, 0 <= i, j, k <= N; entry ((i M + j) M + k), M = N + 1.
#define EVOL_EWALD_N 64
#define EVOL_EWALD_M (EVOL_EWALD_N + 1)

// Walk parameters passed by value to kernels.
struct evol_kparams {
    float theta, G, gamma, alpha, beta;
    float eta_h, eta_e;
    int gravity, sph, adaptive, use_tc, periodic_mask, mixed;
    float plen[3];
    int n, n_gas, leaf;
    int stack_cap;           // traversal-stack entries a warp may use
    int stack_stride;        // entries allocated per warp (>= stack_cap)
    int nsys;
    int want_divv;           // length solves also form div v
    int want_curl;           // the h solve also forms |curl v| (Balsara limiter, alpha switch)
    int standard, nstd;      // h solve by the standard scheme with nstd neighbours inside 2h
    // individual time steps: the walks take only the particles of the active list d.act (sorted
    // positions, ascending; its length at d.acts[n]); the force walk also records, per SPH
    // neighbour, the smallest step (ticks) of an active particle next to it (wake-up)
    int active, wake;
    int super;               // the force walk's groups start from their super-group's lists
    int lsub;                // particles per group walk of the length solves (1..32)
    // periodic gravity (Ewald): cube side, 2 N / L for the table lookup, the table (L = 1)
    int ewald;
    float ewald_L, ewald_sc;
    const float4 *ewald_tab;
    // dissipation variants (Sect. 3.3.3); diss = any of them on
    int diss, visc_form, balsara, var_alpha, conduction, cond_vsig, cond_source;
    float alpha_min, alpha_tau, alpha_source, alpha_u_min;
};
