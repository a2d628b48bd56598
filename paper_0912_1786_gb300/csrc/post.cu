// Per-particle packing between the phases (equation of state, walk operands), un-permutation
// of results into the caller's order, and FP64 global diagnostics.
#include <cuda_runtime.h>
#include <stdint.h>

#include "evol_internal.cuh"

namespace {

// Dissipation operands of the pack (Sect. 3.3.3): per-particle alpha and alpha^u in the caller's
// order (NULL: the constant alpha, alpha^u = 0) and the Balsara limiter's constant.
struct DissPack {
    const float *alpha, *alpha_u;
    float alpha_const, balsara_eta;
    int on, need_f;
};

// Walk operands.  grav = (1/eps, X/Upsilon, h, zeta/Omega*), hydro = (v, P/rho^2),
// snd = (c, rho, 1/h, P).  Ideal gas (App. B): P = (gamma-1) rho u, c = sqrt(gamma (gamma-1) u).
// With a dissipation variant on, diss = (alpha_i, f_i, u_i, alpha^u_i) with the Balsara factor
// f_i = |div v| / (|div v| + |curl v| + eta_B c/h), 0 where that denominator is 0.
__global__ void k_pack(int n, int n_gas, int do_grav, int adaptive, int do_sph, float gamma, evol_dev d, DissPack dp)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    if (do_grav) {
        float e = d.len_eps[s];
        g.x = 1.f / e;
        if (adaptive) {
            g.y = d.X[s] / d.ups[s];
        } else {
            d.ups[s] = 1.f;
            d.X[s] = 0.f;
        }
    }
    float4 v = d.vel[s];
    float4 hy = make_float4(v.x, v.y, v.z, 0.f);
    float4 sn = make_float4(0.f, 0.f, 0.f, 0.f);
    if (do_sph && d.orig[s] < n_gas) {
        float h = d.len_h[s], rho = d.rho[s], u = v.w;
        float P = (gamma - 1.f) * rho * u;
        g.z = h;
        g.w = d.zeta[s] / d.omega[s];
        hy.w = P / (rho * rho);
        sn = make_float4(sqrtf(gamma * (gamma - 1.f) * u), rho, 1.f / h, P);
        if (dp.on) {
            const int j = d.orig[s];
            float f = 0.f;
            if (dp.need_f) {
                const float dv = fabsf(d.divv_h[s]);
                const float den = dv + d.curlv_h[s] + dp.balsara_eta * sn.x * sn.z;
                f = den > 0.f ? dv / den : 0.f;
            }
            d.diss[s] = make_float4(dp.alpha ? dp.alpha[j] : dp.alpha_const, f, u, dp.alpha_u ? dp.alpha_u[j] : 0.f);
        }
    }
    d.grav[s] = g;
    d.hydro[s] = hy;
    d.snd[s] = sn;
}

// Results into the caller's order: thread j gathers caller index j's values from its sorted
// position (so the writes, the larger share of the traffic, are coalesced).  Every value written
// is checked: a non-finite one is flagged as EVOL_ENAN (the first error recorded wins, so a length
// that had no root reports ENOCONV).
__global__ void k_unpermute(int n, int n_gas, int what, int add_acc, evol_dev d, float *h, float *eps, float *ax,
                            float *ay, float *az, float *pot, float *rho, float *P, float *c, float *omega,
                            float *zeta, float *dudt, float *ups, float *X, float *dalpha, float *dalpha_u,
                            int64_t stride)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    if ((what & EVOL_UNPERM_ACTIVE) && !d.bact[j]) return;     // individual steps: evaluated ones only
    const int s = d.inv[j];
    const bool gas = j < n_gas;
    bool fin = true;
    auto put = [&](float *dst, float v) {
        fin = fin && isfinite(v);
        if (dst) dst[j] = v;
    };
    if (what & EVOL_UNPERM_LENGTHS) {
        if (gas) put(h, d.len_h[s]);
    }
    if (what & EVOL_UNPERM_EPSOUT) {
        put(eps, d.len_eps[s]);
        put(ups, d.ups[s]);
        put(X, d.X[s]);
    }
    if ((what & EVOL_UNPERM_DENSITY) && gas) {
        float4 sn = d.snd[s];
        put(rho, d.rho[s]);
        put(P, sn.w);
        put(c, sn.x);
        put(omega, d.omega[s]);
        put(zeta, d.zeta[s]);
    }
    if (what & EVOL_UNPERM_ACC) {
        float4 a = d.acc[s];
        if (add_acc) {
            fin = fin && isfinite(a.x) && isfinite(a.y) && isfinite(a.z);
            if (ax) ax[j] += a.x;
            if (ay) ay[j] += a.y;
            if (az) az[j] += a.z;
        } else {
            put(ax, a.x);
            put(ay, a.y);
            put(az, a.z);
            put(pot, a.w);
        }
    }
    if ((what & EVOL_UNPERM_DUDT) && gas) put(dudt, d.dudt[s]);
    if ((what & EVOL_UNPERM_DALPHA) && gas && dalpha) put(dalpha, d.dalpha[s]);
    if ((what & EVOL_UNPERM_DALPHA_U) && gas && dalpha_u) put(dalpha_u, d.dalpha_u[s]);
    if (what & EVOL_UNPERM_PERSIST) {
        // the last evaluation of the particle, kept for the system steps in which it is inactive
        float *q = d.pers + j;
        if (gas) {
            q[0] = d.rho[s];
            q[stride] = d.omega[s];
            q[2 * stride] = d.zeta[s];
            q[5 * stride] = d.divv_h[s];
            q[6 * stride] = d.curlv_h[s];
        }
        q[3 * stride] = d.ups[s];
        q[4 * stride] = d.X[s];
    }
    if (!fin) evol_flag(d.err, EVOL_ENAN);
}

constexpr int DG_THREADS = 256;
constexpr int DG_N = 11;

__global__ void k_diag_partial(int n, int n_gas, int have_sph, evol_dev d, double *part)
{
    double v[DG_N];
    for (int k = 0; k < DG_N; ++k) v[k] = 0.0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        float4 p = d.pos[s], ve = d.vel[s], a = d.acc[s];
        double m = p.w;
        v[0] += m * ve.x; v[1] += m * ve.y; v[2] += m * ve.z;
        v[3] += m * a.x; v[4] += m * a.y; v[5] += m * a.z;
        v[6] += 0.5 * m * ((double)ve.x * ve.x + (double)ve.y * ve.y + (double)ve.z * ve.z);
        bool gas = d.orig[s] < n_gas;
        if (gas) v[7] += m * ve.w;
        v[8] += 0.5 * m * a.w;
        if (gas && have_sph) v[9] += m * ((double)d.vah[s] + (double)d.dudt[s]);
        v[10] += m;
    }
    __shared__ double sh[DG_THREADS / 32][DG_N];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = 0; k < DG_N; ++k) {
        double x = v[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sh[w][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < DG_N) {
        double x = 0.0;
        for (int k = 0; k < DG_THREADS / 32; ++k) x += sh[k][threadIdx.x];
        part[blockIdx.x * DG_N + threadIdx.x] = x;
    }
}

__global__ void k_diag_final(int nparts, const double *part, const int32_t *nnodes,
                             const unsigned long long *counters, double *diag)
{
    int k = threadIdx.x;
    if (k < DG_N) {
        double x = 0.0;
        for (int b = 0; b < nparts; ++b) x += part[b * DG_N + k];
        diag[k] = x;
    }
    if (k == 0) {
        diag[11] = (double)*nnodes;
        diag[12] = (double)counters[0];
        diag[13] = (double)counters[1];
        diag[14] = (double)counters[2];
        diag[15] = (double)counters[3];
    }
}

// Leapfrog pieces (Sect. 4.1, KDK): half kick of v (and u for gas), drift of x with periodic
// wrapping, in the caller's order.
// Per-particle switches advanced with the kicks, like u (caller order, gas): alpha by d alpha/dt
// and alpha^u by d alpha^u/dt, each only where both pointers are set.
struct SwitchKick {
    float *alpha, *alpha_u;
    const float *dalpha, *dalpha_u;
};

__device__ __forceinline__ void kick_switches(const SwitchKick &sk, int i, float hdt)
{
    if (sk.alpha && sk.dalpha) sk.alpha[i] += hdt * sk.dalpha[i];
    if (sk.alpha_u && sk.dalpha_u) sk.alpha_u[i] += hdt * sk.dalpha_u[i];
}

__global__ void k_kick(int n, int n_gas, float half_dt, float *vx, float *vy, float *vz, float *u, const float *ax,
                       const float *ay, const float *az, const float *dudt, SwitchKick sk)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    vx[i] += half_dt * ax[i];
    vy[i] += half_dt * ay[i];
    vz[i] += half_dt * az[i];
    if (u && dudt && i < n_gas) u[i] += half_dt * dudt[i];
    if (i < n_gas) kick_switches(sk, i, half_dt);
}

__global__ void k_drift(int n, float dt, float *x, float *y, float *z, const float *vx, const float *vy,
                        const float *vz, int pmask, float lo0, float lo1, float lo2, float len0, float len1, float len2)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float p[3] = {x[i] + dt * vx[i], y[i] + dt * vy[i], z[i] + dt * vz[i]};
    const float lo[3] = {lo0, lo1, lo2}, len[3] = {len0, len1, len2};
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if ((pmask >> a) & 1) {
            float t = p[a] - lo[a];
            t -= len[a] * floorf(t / len[a]);
            if (t >= len[a]) t -= len[a];       // rounding can land exactly on the upper edge
            if (t < 0.f) t = 0.f;
            p[a] = lo[a] + t;
        }
    x[i] = p[0];
    y[i] = p[1];
    z[i] = p[2];
}

// ---- global time step (Sect. 4.2) ------------------------------------------------------
// Per particle, in the caller's order, the smallest of the criteria
//   eta_acc sqrt(L/|a|), eta_vel L/|v|, eta_av |v|/|a|          (L = min(eps, h), eps without gas)
//   eta_C h / (h |div v| + c + 1.2 (alpha c + beta max |mu|)),  eta_u |u / (du/dt)|     (gas)
// (a criterion with eta = 0, or without a finite positive value, is left out); the minimum over
// all particles is folded into *dtbits (the bits of a non-negative float order like the float).
// The sorted-order quantities (c, div v, max |mu|) are read through the inverse permutation.
struct TsParams {
    float eta_acc, eta_vel, eta_av, eta_c, eta_u, alpha, beta;
    int gravity, sph;
    int var_alpha;           // the Courant term takes alpha_i (packed with the dissipation operands)
};

// The smallest of the criteria for caller index j (INFINITY where none applies).
__device__ float particle_criterion(int j, int n_gas, const evol_dev &d, const TsParams &tp, const float *vx,
                                    const float *vy, const float *vz, const float *u, const float *acc,
                                    int64_t stride, const float *h, const float *eps)
{
    const float ax = acc[j], ay = acc[stride + j], az = acc[2 * stride + j];
    const float a = sqrtf(ax * ax + ay * ay + az * az);
    const float v = sqrtf(vx[j] * vx[j] + vy[j] * vy[j] + vz[j] * vz[j]);
    const bool gas = tp.sph && j < n_gas;
    float L = tp.gravity ? eps[j] : INFINITY;
    if (gas) L = fminf(L, h[j]);
    float c[5] = {INFINITY, INFINITY, INFINITY, INFINITY, INFINITY};
    if (tp.eta_acc > 0.f) c[0] = tp.eta_acc * sqrtf(L / a);
    if (tp.eta_vel > 0.f) c[1] = tp.eta_vel * L / v;
    if (tp.eta_av > 0.f) c[2] = tp.eta_av * v / a;
    if (gas) {
        const int s = d.inv[j];
        const float cs = d.snd[s].x, hj = h[j];
        const float al = tp.var_alpha ? d.diss[s].x : tp.alpha;
        if (tp.eta_c > 0.f)
            c[3] = tp.eta_c * hj / (hj * fabsf(d.divv_h[s]) + cs + 1.2f * (al * cs + tp.beta * d.mumax[s]));
        if (tp.eta_u > 0.f) c[4] = tp.eta_u * fabsf(u[j] / acc[3 * stride + j]);
    }
    float dt = INFINITY;
#pragma unroll
    for (int k = 0; k < 5; ++k)
        if (c[k] > 0.f && c[k] < INFINITY) dt = fminf(dt, c[k]);      // NaN and 0 are left out
    return dt;
}

__global__ void k_dt_criteria(int n, int n_gas, evol_dev d, TsParams tp, const float *vx, const float *vy,
                              const float *vz, const float *u, const float *acc, int64_t stride, const float *h,
                              const float *eps, unsigned *dtbits)
{
    float dt = INFINITY;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        dt = fminf(dt, particle_criterion(j, n_gas, d, tp, vx, vy, vz, u, acc, stride, h, eps));
    for (int o = 16; o > 0; o >>= 1) dt = fminf(dt, __shfl_xor_sync(0xffffffffu, dt, o));
    if ((threadIdx.x & 31) == 0) atomicMin(dtbits, __float_as_uint(dt));
}

// dt = the criteria's minimum clamped to [dt_min, dt_max] (dt_max where no criterion applies);
// the integrator time advances by dt.
__global__ void k_dt_final(float *dt, const unsigned *dtbits, double *time, float dt_min, float dt_max)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    float v = __uint_as_float(*dtbits);
    v = fminf(v, dt_max);
    v = fmaxf(v, dt_min);
    dt[0] = v;
    *time += (double)v;
}

// Kick with the device time step: v += f dt a (u += f dt du/dt and the switches for gas), caller order.
__global__ void k_kick_dev(int n, int n_gas, const float *dtp, float f, float *vx, float *vy, float *vz, float *u,
                           const float *acc, int64_t stride, SwitchKick sk)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float hdt = f * *dtp;
    vx[i] += hdt * acc[i];
    vy[i] += hdt * acc[stride + i];
    vz[i] += hdt * acc[2 * stride + i];
    if (u && i < n_gas) u[i] += hdt * acc[3 * stride + i];
    if (i < n_gas) kick_switches(sk, i, hdt);
}

__global__ void k_drift_dev(int n, const float *dtp, float *x, float *y, float *z, const float *vx, const float *vy,
                            const float *vz, int pmask, float lo0, float lo1, float lo2, float len0, float len1,
                            float len2)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float dt = *dtp;
    float p[3] = {x[i] + dt * vx[i], y[i] + dt * vy[i], z[i] + dt * vz[i]};
    const float lo[3] = {lo0, lo1, lo2}, len[3] = {len0, len1, len2};
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if ((pmask >> a) & 1) {
            float t = p[a] - lo[a];
            t -= len[a] * floorf(t / len[a]);
            if (t >= len[a]) t -= len[a];
            if (t < 0.f) t = 0.f;
            p[a] = lo[a] + t;
        }
    x[i] = p[0];
    y[i] = p[1];
    z[i] = p[2];
}

// Starting lengths of the next solve from the continuity equation (Sect. 2.1): dn/dt = -n div v
// and L ~ n^(-1/3) give L(t + dt) = L exp(div v dt / 3), applied to the solved lengths the caller's
// arrays hold; div v comes from the last solve (sorted order, through the inverse permutation).
__global__ void k_predict_lengths(int n, int n_gas, evol_dev d, const float *dtp, float *h, float *eps, int do_h,
                                  int do_eps)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float k = *dtp * (1.f / 3.f);
    const int s = d.inv[j];
    if (do_eps) eps[j] *= __expf(d.divv_e[s] * k);
    if (do_h && j < n_gas) h[j] *= __expf(d.divv_h[s] * k);
}

// ---- individual power-of-two time steps (Sect. 4.2.1) -----------------------------------------
// Integer timeline: T = 2^K ticks per largest step dt_max, tick = dt_max / T.  Particle j's step is
// [tb_j, te_j]; d.bt holds t_sys, t_next and the run counts (system steps, active evaluations,
// wake-ups, criteria below one tick).
struct BinsParams {
    unsigned long long T, t_end;
    float tick, wake;
    int n, n_gas, periodic_mask;
    float lo[3], len[3];
};

// The largest power-of-two step (ticks) not longer than dt, in [1, T].
__device__ __forceinline__ unsigned long long step_for(float dt, const BinsParams &bp)
{
    unsigned long long L = 1ull;
    while (2ull * L <= bp.T && (float)(2ull * L) * bp.tick <= dt) L *= 2ull;
    return L;
}

// t_next = the smallest step end (d.bt[1] must hold all bits set on entry)
__global__ void k_bins_next(BinsParams bp, evol_dev d)
{
    unsigned long long m = ~0ull;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < bp.n; j += gridDim.x * blockDim.x)
        m = min(m, d.te[j]);
    for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMin(&d.bt[1], m);
}

// Everyone drifts to t_next with its half-kicked velocity; the particles whose step ends there are
// flagged active; each particle's prediction time t_next - (tb + te)/2 for v and u.
__global__ void k_bins_drift(BinsParams bp, evol_dev d, float *x, float *y, float *z, const float *vx, const float *vy,
                             const float *vz)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= bp.n) return;
    const unsigned long long tn = d.bt[1], ts = d.bt[0];
    const float dt = (float)(tn - ts) * bp.tick;
    float p[3] = {x[j] + dt * vx[j], y[j] + dt * vy[j], z[j] + dt * vz[j]};
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if ((bp.periodic_mask >> a) & 1) {
            float t = p[a] - bp.lo[a];
            t -= bp.len[a] * floorf(t / bp.len[a]);
            if (t >= bp.len[a]) t -= bp.len[a];
            if (t < 0.f) t = 0.f;
            p[a] = bp.lo[a] + t;
        }
    x[j] = p[0];
    y[j] = p[1];
    z[j] = p[2];
    const unsigned long long tb = d.tb[j], te = d.te[j];
    d.bact[j] = te == tn ? 1 : 0;
    // t_next - (tb + te)/2 in ticks: exact in integers (times two), then to time units
    d.pred_tau[j] = (float)((long long)(2ull * tn) - (long long)(tb + te)) * 0.5f * bp.tick;
}

// Inactive particles: the lengths and densities of their last evaluation, into sorted order.
__global__ void k_bins_fill(BinsParams bp, evol_dev d, int64_t stride)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= bp.n) return;
    const int j = d.orig[s];
    if (d.bact[j]) return;
    const float *q = d.pers + j;
    if (j < bp.n_gas) {
        d.rho[s] = q[0];
        d.omega[s] = q[stride];
        d.zeta[s] = q[2 * stride];
        d.divv_h[s] = q[5 * stride];
        d.curlv_h[s] = q[6 * stride];
    }
    d.ups[s] = q[3 * stride];
    d.X[s] = q[4 * stride];
}

// A kick of the flagged particles (caller order): v += f a, u += f du/dt, switches alike, with
// f = fac * (te - tb) * tick (second half kick: fac = 1/2).
__global__ void k_bins_kick2(BinsParams bp, evol_dev d, float *vx, float *vy, float *vz, float *u, const float *acc,
                             int64_t stride, SwitchKick sk)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= bp.n || !d.bact[j]) return;
    const float f = 0.5f * (float)(d.te[j] - d.tb[j]) * bp.tick;
    vx[j] += f * acc[j];
    vy[j] += f * acc[stride + j];
    vz[j] += f * acc[2 * stride + j];
    if (j < bp.n_gas) {
        if (u) u[j] += f * acc[3 * stride + j];
        kick_switches(sk, j, f);
    }
}

// Active particles, unless t_next ends the run: the step from the criteria, longer than before only
// where t_next is a multiple of it; [tb, te] = [t_next, t_next + L]; first half kick v += a L/2.
__global__ void k_bins_newstep(BinsParams bp, evol_dev d, TsParams tp, float *vx, float *vy, float *vz, float *u,
                               const float *acc, int64_t stride, const float *h, const float *eps, SwitchKick sk)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= bp.n || !d.bact[j]) return;
    const unsigned long long tn = d.bt[1];
    if (tn >= bp.t_end) return;
    const float dt = particle_criterion(j, bp.n_gas, d, tp, vx, vy, vz, u, acc, stride, h, eps);
    unsigned long long L = step_for(dt, bp);
    if (!((float)bp.tick <= dt)) atomicAdd(&d.bt[5], 1ull);       // below one tick (or none): finest step
    if (tn > 0) L = min(L, tn & (~tn + 1ull));                      // the largest power of two dividing t_next
    d.tb[j] = tn;
    d.te[j] = tn + L;
    const float f = 0.5f * (float)L * bp.tick;
    vx[j] += f * acc[j];
    vy[j] += f * acc[stride + j];
    vz[j] += f * acc[2 * stride + j];
    if (j < bp.n_gas) {
        if (u) u[j] += f * acc[3 * stride + j];
        kick_switches(sk, j, f);
    }
}

// Wake-up: an inactive gas particle whose step exceeds wake times the step just completed by an
// active SPH neighbour (d.nbmin, sorted) ends its step at the first multiple of L' > t_next, L' the
// largest power of two <= wake x that step; the part of its first half kick beyond the shortened
// step is taken back.
__global__ void k_bins_wake(BinsParams bp, evol_dev d, float *vx, float *vy, float *vz, float *u, const float *acc,
                            int64_t stride, SwitchKick sk)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= bp.n_gas || d.bact[j]) return;
    const unsigned m = d.nbmin[d.inv[j]];
    if (m == 0xffffffffu) return;
    const unsigned long long tb = d.tb[j], te = d.te[j], Lj = te - tb, tn = d.bt[1];
    const float lim = bp.wake * (float)m;
    if (!((float)Lj > lim)) return;
    unsigned long long Lw = 1ull;
    while (2ull * Lw <= bp.T && (float)(2ull * Lw) <= lim) Lw *= 2ull;
    if (Lw >= Lj) return;
    const unsigned long long ten = (tn / Lw + 1ull) * Lw;
    if (ten >= te) return;
    const float f = -0.5f * (float)(Lj - (ten - tb)) * bp.tick;
    vx[j] += f * acc[j];
    vy[j] += f * acc[stride + j];
    vz[j] += f * acc[2 * stride + j];
    if (u) u[j] += f * acc[3 * stride + j];
    kick_switches(sk, j, f);
    d.te[j] = ten;
    atomicAdd(&d.bt[4], 1ull);
}

// t_sys = t_next; counts
__global__ void k_bins_advance(BinsParams bp, evol_dev d)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    d.bt[0] = d.bt[1];
    d.bt[2] += 1ull;
    d.bt[3] += (unsigned long long)d.acts[bp.n];
}

// Start of a run: every particle active at t = 0 (its first step is chosen by k_bins_newstep).
__global__ void k_bins_start(BinsParams bp, evol_dev d)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < bp.n) {
        d.tb[j] = 0ull;
        d.te[j] = 0ull;
        d.bact[j] = 1;
    }
    if (j < 6) d.bt[j] = 0ull;
}

}  // namespace

static SwitchKick switch_kick(const evol_particles *p, const evol_params *prm, const float *dalpha,
                              const float *dalpha_u)
{
    SwitchKick sk{};
    if (prm->sph && prm->variable_alpha) {
        sk.alpha = (float *)p->alpha;
        sk.dalpha = dalpha;
    }
    if (prm->sph && prm->conduction) {
        sk.alpha_u = (float *)p->alpha_u;
        sk.dalpha_u = dalpha_u;
    }
    return sk;
}

int evol_launch_kick(evol_ctx *c, const evol_particles *p, const evol_params *prm, float half_dt, const float *ax,
                     const float *ay, const float *az, const float *dudt, const float *dalpha, const float *dalpha_u)
{
    int n = (int)p->n;
    k_kick<<<(n + 255) / 256, 256, 0, c->stream>>>(n, (int)p->n_gas, half_dt, (float *)p->vx, (float *)p->vy,
                                                   (float *)p->vz, (float *)p->u, ax, ay, az, dudt,
                                                   switch_kick(p, prm, dalpha, dalpha_u));
    return evol_cuda_ok(cudaGetLastError());
}

int evol_launch_drift(evol_ctx *c, const evol_particles *p, const evol_params *prm, float dt)
{
    int n = (int)p->n;
    k_drift<<<(n + 255) / 256, 256, 0, c->stream>>>(
        n, dt, (float *)p->x, (float *)p->y, (float *)p->z, p->vx, p->vy, p->vz, prm->periodic_mask,
        prm->periodic_lo[0], prm->periodic_lo[1], prm->periodic_lo[2], prm->periodic_hi[0] - prm->periodic_lo[0],
        prm->periodic_hi[1] - prm->periodic_lo[1], prm->periodic_hi[2] - prm->periodic_lo[2]);
    return evol_cuda_ok(cudaGetLastError());
}

int evol_launch_pack(evol_ctx *c, const evol_particles *p, const evol_params *prm, int do_grav, int do_sph)
{
    int n = (int)p->n;
    DissPack dp{};
    dp.on = do_sph && evol_diss_on(prm);
    dp.need_f = evol_needs_curl(prm);
    dp.alpha = prm->variable_alpha ? p->alpha : nullptr;
    dp.alpha_u = prm->conduction ? p->alpha_u : nullptr;
    dp.alpha_const = prm->alpha;
    dp.balsara_eta = prm->balsara_eta;
    k_pack<<<(n + 255) / 256, 256, 0, c->stream>>>(n, (int)p->n_gas, do_grav, prm->adaptive_softening, do_sph,
                                                   prm->gamma, c->d, dp);
    return evol_cuda_ok(cudaGetLastError());
}

int evol_launch_unpermute_ex(evol_ctx *c, const evol_particles *p, const evol_outputs *o, int what, int add_acc)
{
    int n = (int)p->n;
    evol_outputs z{};
    const evol_outputs *q = o ? o : &z;
    k_unpermute<<<(n + 255) / 256, 256, 0, c->stream>>>(n, (int)p->n_gas, what, add_acc, c->d, p->h, p->eps, q->ax,
                                                        q->ay, q->az, q->pot, q->rho, q->P, q->c, q->omega, q->zeta,
                                                        q->dudt, q->ups, q->X, q->dalpha, q->dalpha_u, c->cap);
    return evol_cuda_ok(cudaGetLastError());
}

int evol_launch_unpermute(evol_ctx *c, const evol_particles *p, const evol_outputs *o, int what)
{
    return evol_launch_unpermute_ex(c, p, o, what, 0);
}

int evol_launch_diagnostics(evol_ctx *c, const evol_particles *p, const evol_params *prm)
{
    int nb = (int)c->diag_blocks;
    k_diag_partial<<<nb, DG_THREADS, 0, c->stream>>>((int)p->n, (int)p->n_gas, prm->sph, c->d, c->d.diag_part);
    k_diag_final<<<1, 32, 0, c->stream>>>(nb, c->d.diag_part, c->d.nnodes, c->d.counters, c->d.diag);
    return evol_cuda_ok(cudaGetLastError());
}

// One global-step KDK step around a force step: stage 0 = time step, first half kick, drift and
// the predicted starting lengths; stage 1 = the second half kick.  The accelerations and du/dt of
// the last force step are c->kdk_acc (caller order: ax | ay | az | du/dt | d alpha/dt | d alpha^u/dt,
// c->cap apart).
int evol_launch_integrator_step(evol_ctx *c, const evol_particles *p, const evol_params *prm, const evol_integrator *ip,
                                int stage)
{
    const int n = (int)p->n, ng = (int)p->n_gas;
    const int tb = 256, gb = (n + tb - 1) / tb;
    const int64_t cap = c->cap;
    unsigned *dtbits = reinterpret_cast<unsigned *>(c->d.dt + 1);
    const SwitchKick sk = switch_kick(p, prm, c->kdk_acc + 4 * cap, c->kdk_acc + 5 * cap);
    if (stage == 0) {
        TsParams tp{ip->eta_acc, ip->eta_vel, ip->eta_av, ip->eta_courant, ip->eta_u, prm->alpha, prm->beta,
                    prm->gravity, prm->sph && p->n_gas > 0, prm->sph && prm->variable_alpha};
        // all bits set: above every non-negative float's bits, so the first criterion replaces it
        cudaMemsetAsync(dtbits, 0xff, sizeof(unsigned), c->stream);
        k_dt_criteria<<<c->num_sms * 4, 256, 0, c->stream>>>(n, ng, c->d, tp, p->vx, p->vy, p->vz, p->u, c->kdk_acc,
                                                              cap, p->h, p->eps, dtbits);
        k_dt_final<<<1, 32, 0, c->stream>>>(c->d.dt, dtbits, c->d.time, ip->dt_min, ip->dt_max);
        k_kick_dev<<<gb, tb, 0, c->stream>>>(n, ng, c->d.dt, 0.5f, (float *)p->vx, (float *)p->vy, (float *)p->vz,
                                             (float *)p->u, c->kdk_acc, cap, sk);
        k_drift_dev<<<gb, tb, 0, c->stream>>>(
            n, c->d.dt, (float *)p->x, (float *)p->y, (float *)p->z, p->vx, p->vy, p->vz, prm->periodic_mask,
            prm->periodic_lo[0], prm->periodic_lo[1], prm->periodic_lo[2], prm->periodic_hi[0] - prm->periodic_lo[0],
            prm->periodic_hi[1] - prm->periodic_lo[1], prm->periodic_hi[2] - prm->periodic_lo[2]);
        if (ip->predict_lengths)
            k_predict_lengths<<<gb, tb, 0, c->stream>>>(n, ng, c->d, c->d.dt, p->h, p->eps,
                                                        prm->sph && ng > 0 && p->h != nullptr,
                                                        prm->gravity && prm->adaptive_softening);
    } else {
        k_kick_dev<<<gb, tb, 0, c->stream>>>(n, ng, c->d.dt, 0.5f, (float *)p->vx, (float *)p->vy, (float *)p->vz,
                                             (float *)p->u, c->kdk_acc, cap, sk);
    }
    return evol_cuda_ok(cudaGetLastError());
}

// Individual time steps (Sect. 4.2.1): the kernels of one stage of a system step (see evol_run_bins).
//   stage 0: start (every particle active at t = 0, first steps and first half kicks)
//   stage 1: t_next, drift, active flags, prediction times
//   stage 2: inactive particles' last evaluation into sorted order
//   stage 3: second half kicks, new steps and first half kicks, wake-up, t_sys = t_next
int evol_launch_bins(evol_ctx *c, const evol_particles *p, const evol_params *prm, const evol_bins *bp, int stage)
{
    const int n = (int)p->n, ng = (int)p->n_gas;
    const int tb = 256, gb = (n + tb - 1) / tb;
    const int64_t cap = c->cap;
    BinsParams b{};
    b.T = 1ull << bp->max_bin;
    b.tick = (float)((double)bp->crit.dt_max / (double)b.T);
    b.wake = bp->wake_factor;
    b.n = n;
    b.n_gas = ng;
    b.periodic_mask = prm->periodic_mask;
    for (int a = 0; a < 3; ++a) {
        b.lo[a] = prm->periodic_lo[a];
        b.len[a] = prm->periodic_hi[a] - prm->periodic_lo[a];
    }
    b.t_end = c->bins_t_end;
    const SwitchKick sk = switch_kick(p, prm, c->kdk_acc + 4 * cap, c->kdk_acc + 5 * cap);
    const evol_integrator *ip = &bp->crit;
    TsParams tp{ip->eta_acc, ip->eta_vel, ip->eta_av, ip->eta_courant, ip->eta_u, prm->alpha, prm->beta,
                prm->gravity, prm->sph && ng > 0, prm->sph && prm->variable_alpha};
    float *vx = (float *)p->vx, *vy = (float *)p->vy, *vz = (float *)p->vz, *u = (float *)p->u;
    switch (stage) {
    case 0:
        k_bins_start<<<gb, tb, 0, c->stream>>>(b, c->d);
        k_bins_newstep<<<gb, tb, 0, c->stream>>>(b, c->d, tp, vx, vy, vz, u, c->kdk_acc, cap, p->h, p->eps, sk);
        break;
    case 1:
        cudaMemsetAsync(c->d.bt + 1, 0xff, sizeof(unsigned long long), c->stream);
        k_bins_next<<<c->num_sms * 4, 256, 0, c->stream>>>(b, c->d);
        k_bins_drift<<<gb, tb, 0, c->stream>>>(b, c->d, (float *)p->x, (float *)p->y, (float *)p->z, p->vx, p->vy,
                                               p->vz);
        break;
    case 2:
        k_bins_fill<<<gb, tb, 0, c->stream>>>(b, c->d, cap);
        break;
    case 3:
        k_bins_kick2<<<gb, tb, 0, c->stream>>>(b, c->d, vx, vy, vz, u, c->kdk_acc, cap, sk);
        k_bins_newstep<<<gb, tb, 0, c->stream>>>(b, c->d, tp, vx, vy, vz, u, c->kdk_acc, cap, p->h, p->eps, sk);
        if (bp->wake_factor > 0.f && ng > 0)
            k_bins_wake<<<(ng + tb - 1) / tb, tb, 0, c->stream>>>(b, c->d, vx, vy, vz, u, c->kdk_acc, cap, sk);
        k_bins_advance<<<1, 32, 0, c->stream>>>(b, c->d);
        break;
    default:
        return EVOL_EINVAL;
    }
    return evol_cuda_ok(cudaGetLastError());
}

// ---- periodic gravity: the Ewald correction table (Sect. 4.3) ----------------------------------
namespace {

// One grid point of the table for a cube of side 1 (w = 2): the correction f of the acceleration
// by the replicas beyond the nearest image and its zero-mean potential g,
//   f(x) = x/|x|^3 - sum_{|n|<5} (x - n)/r_n^3 (erfc(w r_n) + 2 w r_n/sqrt(pi) e^{-w^2 r_n^2})
//          - 2 sum_{0<|h|<5} h/h^2 e^{-pi^2 h^2/w^2} sin(2 pi h.x),
//   g(x) = 1/|x| - sum_n erfc(w r_n)/r_n - 1/pi sum_h e^{-pi^2 h^2/w^2}/h^2 cos(2 pi h.x) + pi/w^2,
// in FP64 (the n = 0 terms combined with the direct ones, by series near x = 0).
__global__ void k_ewald_table(float4 *tab)
{
    const int N = EVOL_EWALD_N, M = EVOL_EWALD_M;
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= M * M * M) return;
    const int k = id % M, j = (id / M) % M, i = id / (M * M);
    const double x[3] = {0.5 * i / N, 0.5 * j / N, 0.5 * k / N};
    const double w = 2.0, pi = 3.14159265358979323846, sqpi = sqrt(pi);
    double F[3] = {0.0, 0.0, 0.0}, g = 0.0;
    for (int a = -4; a <= 4; ++a)
        for (int b = -4; b <= 4; ++b)
            for (int c = -4; c <= 4; ++c) {
                const int n2 = a * a + b * b + c * c;
                if (n2 >= 25) continue;
                const double d[3] = {x[0] - a, x[1] - b, x[2] - c};
                const double rn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                const double z = w * rn;
                if (n2 == 0) {
                    if (z < 1e-3) {
                        const double z2 = z * z;
                        const double k3 = 4.0 / (3.0 * sqpi) * w * w * w * (1.0 - 0.6 * z2);
                        for (int q = 0; q < 3; ++q) F[q] += x[q] * k3;
                        g += 2.0 * w / sqpi * (1.0 - z2 / 3.0);
                    } else {
                        const double kk = (erf(z) - 2.0 * z / sqpi * exp(-z * z)) / (rn * rn * rn);
                        for (int q = 0; q < 3; ++q) F[q] += x[q] * kk;
                        g += erf(z) / rn;
                    }
                    continue;
                }
                const double kk = (erfc(z) + 2.0 * z / sqpi * exp(-z * z)) / (rn * rn * rn);
                for (int q = 0; q < 3; ++q) F[q] -= d[q] * kk;
                g -= erfc(z) / rn;
            }
    for (int a = -4; a <= 4; ++a)
        for (int b = -4; b <= 4; ++b)
            for (int c = -4; c <= 4; ++c) {
                const int h2 = a * a + b * b + c * c;
                if (h2 == 0 || h2 >= 25) continue;
                const double e = exp(-pi * pi * h2 / (w * w));
                const double ph = 2.0 * pi * (a * x[0] + b * x[1] + c * x[2]);
                const double ks = 2.0 * e / h2 * sin(ph);
                F[0] -= ks * a;
                F[1] -= ks * b;
                F[2] -= ks * c;
                g -= e / (pi * h2) * cos(ph);
            }
    g += pi / (w * w);
    tab[id] = make_float4((float)F[0], (float)F[1], (float)F[2], (float)g);
}

}  // namespace

// Build the Ewald table once per context (outside any stream capture: the entry points call this
// before recording their graphs).
int evol_ewald_prepare(evol_ctx *c)
{
    if (c->ewald_ready) return EVOL_OK;
    const int cnt = EVOL_EWALD_M * EVOL_EWALD_M * EVOL_EWALD_M;
    k_ewald_table<<<(cnt + 127) / 128, 128, 0, c->stream>>>(c->d.ewald);
    if (cudaGetLastError() != cudaSuccess) return EVOL_ECUDA;
    c->ewald_ready = 1;
    return EVOL_OK;
}
