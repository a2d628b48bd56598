// Force walk: gravity (Sect. 2.1-2.2, App. B) and SPH pressure + viscosity forces and du/dt
// (Sect. 3, Eqs. motionvarmass1, thermalvarmass1, mu_visc) in one traversal of the tree, as
// the paper does its second walk (Sect. 3.1).
//
// A warp owns 32 consecutive particles in key order (a compact group).  Node A is a far node
// for particle i iff
//     |r_i - com_A| > l_A/theta + delta_A                                     (Eq. opcrit)
// and A's particle box lies farther than R_iA = 2 max(eps_i, epsmax_A) (and, for gas i and a
// node holding gas, farther than 2 max(h_i, hmax_A)); otherwise it is opened.  The warp keeps a
// stack of (node, mask of lanes that still need the node) and pops up to 32 entries at a time,
// one per lane, so the node loads of a batch are issued together.  Each popped node is first
// classified against the group's bounding box: if every lane must accept it, or every lane must
// open it, by bounds that hold with a relative margin of 1e-5 over the FP32 rounding of the
// per-lane test, the decision is taken for the whole mask; only the remaining ("mixed") nodes
// are tested lane by lane.  The per-particle decisions are therefore exactly those of a
// per-particle walk.  Accepted nodes (with their accept mask) and the particles of opened leaves
// (with their open mask) are staged in shared memory and evaluated in batches: far nodes by
// monopole + traceless quadrupole about the centre of mass, near particles by the symmetrised
// softened pair force plus the adaptive-softening correction, and, for gas pairs with
// r < 2 max(h_i, h_j), the SPH terms.
#include <cuda_runtime.h>
#include <stdint.h>

#include "evol_internal.cuh"

namespace {

constexpr int WK_THREADS = 128;
constexpr int WK_WARPS = WK_THREADS / 32;
constexpr int FARCAP = 64;
constexpr int NEARCAP = 64;

constexpr float TAU = 1e-5f;      // safety margin of the group-level bounds

struct WalkSmem {
    float4 bA[WK_WARPS][32];      // popped batch: com, ropen^2
    float4 bB[WK_WARPS][32];      // box centre, 2 hmax
    float4 bC[WK_WARPS][32];      // box half widths, 2 epsmax
    int far_id[WK_WARPS][FARCAP];
    unsigned far_mask[WK_WARPS][FARCAP];
    float4 fA[WK_WARPS][FARCAP];
    float4 fQ0[WK_WARPS][FARCAP];
    float4 fQ1[WK_WARPS][FARCAP];
    int near_j[WK_WARPS][NEARCAP];
    unsigned near_mask[WK_WARPS][NEARCAP];
    float4 np[WK_WARPS][NEARCAP];
    float4 ng[WK_WARPS][NEARCAP];
    float4 nh[WK_WARPS][NEARCAP];
    float4 ns[WK_WARPS][NEARCAP];
    int norig[WK_WARPS][NEARCAP];
    float4 gbox[WK_WARPS][3];     // group bounds: centre, 0 | half widths, 0 | emax, emin, hmax, hmin
};

// The kernel functions of the pair loop in a division-free form: each takes u and iu = 1/u (iu is
// read only where u >= 1, and where u < 2/3 for the Thomas-Couchman gradient), with 1/u formed
// from quantities already at hand (eps/r, h/r).  Same polynomials as the FP32 kernel functions:
//   gsoft_over_r: eps^3 phi'(r)/r,  phisoft: eps phi(r),  dw_over_u: pi h^5 (dW/dr)/r,
//   tc_over_u: the Thomas-Couchman form of the latter.
// The two branches share one Horner form in u whose coefficients are selected by u < 1; the
// outer branch's 1/u terms are selected, not multiplied by zero, so that a huge 1/u (a pair far
// closer than the softening length) cannot turn into 0 * inf.
__device__ __forceinline__ float gsoft_over_r_u(float u, float iu)
{
    // u < 1: 4/3 - 6/5 u^2 + 1/2 u^3;   1 <= u < 2: 8/3 - 3u + 6/5 u^2 - 1/6 u^3 - 1/(15 u^3)
    const bool in = u < 1.f;
    const float c1 = in ? 0.f : -3.f, c2 = in ? -1.2f : 1.2f, c3 = in ? 0.5f : -1.f / 6.f;
    const float c0 = in ? 4.f / 3.f : 8.f / 3.f;
    const float tail = in ? 0.f : (-1.f / 15.f) * (iu * iu * iu);
    return fmaf(u, fmaf(u, fmaf(u, c3, c2), c1), c0) + tail;
}

__device__ __forceinline__ float phisoft_u(float u, float iu)
{
    // u < 1: -7/5 + 2/3 u^2 - 3/10 u^4 + 1/10 u^5
    // 1 <= u < 2: -8/5 + 4/3 u^2 - u^3 + 3/10 u^4 - 1/30 u^5 + 1/(15 u)
    const bool in = u < 1.f;
    const float c2 = in ? 2.f / 3.f : 4.f / 3.f, c3 = in ? 0.f : -1.f, c4 = in ? -0.3f : 0.3f;
    const float c5 = in ? 0.1f : -1.f / 30.f, c0 = in ? -1.4f : -1.6f;
    const float tail = in ? 0.f : (1.f / 15.f) * iu;
    const float u2 = u * u;
    return fmaf(u2, fmaf(u, fmaf(u, fmaf(u, c5, c4), c3), c2), c0) + tail;
}

__device__ __forceinline__ float dw_over_u_u(float u, float iu)
{
    const float a = fmaxf(2.f - u, 0.f);
    return u < 1.f ? -3.f + 2.25f * u : -0.75f * a * a * iu;
}

__device__ __forceinline__ float tc_over_u_u(float u, float iu)
{
    const float a = fmaxf(2.f - u, 0.f);
    return u < 2.f / 3.f ? -iu : (u < 1.f ? -0.75f * (4.f - 3.f * u) : -0.75f * a * a * iu);
}

// 1/x from the hardware reciprocal (about 1 ulp), for operands of the pair loop
__device__ __forceinline__ float rcp_fast(float x) { return __fdividef(1.f, x); }

template <bool MIXED>
struct Acc {
    float ax = 0.f, ay = 0.f, az = 0.f, pot = 0.f;      // gravity (without G)
    float hx = 0.f, hy = 0.f, hz = 0.f, du = 0.f;       // SPH
};

// Register budgets: the plain gravity + SPH walk (the production form) fits five blocks per SM
// (at most 102 registers) without spilling; every other variant carries a minimum of one block
// per SM, so that the compiler keeps its state in registers instead of spilling to local memory.
template <bool GRAV, bool SPH, bool MIXED, bool CHECK>
__global__ void __launch_bounds__(WK_THREADS, (GRAV && SPH && !MIXED && !CHECK) ? 5 : 1) k_walk(evol_dev d, evol_kparams kp, unsigned long long *queue)
{
    __shared__ WalkSmem sm;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int n = kp.n;
    const int ngroups = (n + 31) >> 5;
    const int pm = SPH ? kp.periodic_mask : 0;
    const float plen0 = kp.plen[0], plen1 = kp.plen[1], plen2 = kp.plen[2];
    const float inv_pi = 1.f / EVOL_PI_F;

    for (;;) {
        int g = 0;
        if (lane == 0) g = (int)atomicAdd(queue, 1ull);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= ngroups) break;
        const int s = g * 32 + lane;
        const bool valid = s < n;
        const float4 pi = valid ? d.pos[s] : make_float4(0.f, 0.f, 0.f, 0.f);
        // this lane's hydro operands (v, P/rho^2, c, rho, 1/h, zeta/Omega*) are read where they are
        // used, in the SPH pass, which keeps them out of the traversal's live registers
        const float4 g0 = valid ? d.grav[s] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float xu_i = g0.y;                   // X/Upsilon (adaptive-softening correction)
        const bool gas_i = SPH && valid && g0.z > 0.f;
        const bool active = valid && (GRAV || gas_i);
        const float ie_i = g0.x, two_eps_i = GRAV && active ? 2.f / g0.x : 0.f;
        const float two_h_i = gas_i ? 2.f * g0.z : 0.f;
        const float inv_mi = valid ? 1.f / pi.w : 0.f;
        const float eps_i = GRAV && valid ? 1.f / ie_i : 0.f;

        Acc<MIXED> acc;
        double tax = 0, tay = 0, taz = 0, tpot = 0, thx = 0, thy = 0, thz = 0, tdu = 0;
        unsigned long long hfar = 0, hnear = 0, hsph = 0;
        int cfar = 0, cpp = 0, csph = 0;
        // interaction counts of this lane (one group's counts fit 32 bits)
        unsigned wfar = 0, wpp = 0, wsph = 0, wsoft = 0;
        // lane slots issued (32 per entry or per loop trip; kept by lane 0): fill of the far loop,
        // of pass 1 and of pass 2 of the near loop
        unsigned wfar_slots = 0, wnear_slots = 0, wpass2_slots = 0;

        auto fold = [&]() {
            if (MIXED) {
                tax += acc.ax; tay += acc.ay; taz += acc.az; tpot += acc.pot;
                thx += acc.hx; thy += acc.hy; thz += acc.hz; tdu += acc.du;
                acc = Acc<MIXED>();
            }
        };

        int nfar = 0, nnear = 0;

        auto flush_far = [&]() {
            __syncwarp();
            // pad to a multiple of 4 with empty-mask entries (node 0 is always valid)
            const int padded = (nfar + 3) & ~3;
            if (lane < padded - nfar) {
                sm.far_id[w][nfar + lane] = 0;
                sm.far_mask[w][nfar + lane] = 0u;
            }
            __syncwarp();
            for (int l = lane; l < padded; l += 32) {
                const int id = sm.far_id[w][l];
                sm.fA[w][l] = d.nA[id];
                sm.fQ0[w][l] = d.nQ0[id];
                sm.fQ1[w][l] = d.nQ1[id];
                wfar += __popc(sm.far_mask[w][l]);     // interaction count (this lane's share)
            }
            if (lane == 0) wfar_slots += 32u * (unsigned)padded;
            __syncwarp();
            for (int e = 0; e < padded; e += 4) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const unsigned msk = sm.far_mask[w][e + u];
                    const float4 A = sm.fA[w][e + u], Q0 = sm.fQ0[w][e + u], Q1 = sm.fQ1[w][e + u];
                    const float dx = pi.x - A.x, dy = pi.y - A.y, dz = pi.z - A.z;
                    const float d2 = dx * dx + dy * dy + dz * dz;
                    // lanes outside the mask get rinv = 0, so every term below vanishes for them
                    const float rinv = ((msk >> lane) & 1u) ? rsqrtf(d2) : 0.f;
                    const float rinv2 = rinv * rinv;
                    const float r3 = rinv * rinv2, r5 = r3 * rinv2, r7 = r5 * rinv2;
                    const float qx = Q0.x * dx + Q1.x * dy + Q1.y * dz;
                    const float qy = Q1.x * dx + Q0.y * dy + Q1.z * dz;
                    const float qz = Q1.y * dx + Q1.z * dy + Q0.z * dz;
                    const float dqd = dx * qx + dy * qy + dz * qz;
                    const float c1 = -Q0.w * r3 - 2.5f * dqd * r7;
                    acc.ax += c1 * dx + r5 * qx;
                    acc.ay += c1 * dy + r5 * qy;
                    acc.az += c1 * dz + r5 * qz;
                    acc.pot += -Q0.w * rinv - 0.5f * dqd * r5;
                }
            }
            fold();
            nfar = 0;
            __syncwarp();
        };

        auto flush_near = [&]() {
            __syncwarp();
            for (int l = lane; l < nnear; l += 32) {
                const int j = sm.near_j[w][l];
                {
                    // interaction count (this lane's share): the entry's lanes, less the particle itself
                    const unsigned msk = sm.near_mask[w][l];
                    const int sl = j - g * 32;
                    const unsigned self = (sl >= 0 && sl < 32) ? ((msk >> sl) & 1u) : 0u;
                    wpp += __popc(msk) - self;
                }
                sm.np[w][l] = d.pos[j];
                sm.ng[w][l] = d.grav[j];
                if (SPH) {
                    sm.nh[w][l] = d.hydro[j];
                    sm.ns[w][l] = d.snd[j];
                }
                if (CHECK) sm.norig[w][l] = d.orig[j];
            }
            if (lane == 0) wnear_slots += 32u * (unsigned)((nnear + 1) & ~1);
            __syncwarp();
            // Pass 1, every entry, two at a time and branch-free.  A gravity pair farther apart than
            // 2 max(eps_i, eps_j) is Newtonian: both softened kernels equal their point-mass forms there
            // (Eqs. softforce, softphi) and the correction term vanishes with dW/dr; it is summed here.
            // Pairs inside that distance, and gas pairs inside 2 max(h_i, h_j), are marked per lane
            // (bit t of sbits) and evaluated in pass 2, each lane taking its own marked pairs, so that
            // the warp runs the softened and SPH terms about as often as its busiest lane has such pairs.
            unsigned long long sbits = 0ull;
            for (int t = 0; t < nnear; t += 2) {
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const bool ok = t + hh < nnear;
                    const int tt = ok ? t + hh : t;
                    const unsigned msk = ok ? sm.near_mask[w][tt] : 0u;
                    const int j = sm.near_j[w][tt];
                    const bool mine = ((msk >> lane) & 1u) && j != s;
                    if (CHECK && mine) ++cpp;
                    const float4 pj = sm.np[w][tt];
                    const float4 gj = sm.ng[w][tt];
                    const float dx = evol_wrap(pi.x - pj.x, plen0, pm & 1);
                    const float dy = evol_wrap(pi.y - pj.y, plen1, pm & 2);
                    const float dz = evol_wrap(pi.z - pj.z, plen2, pm & 4);
                    const float r2 = dx * dx + dy * dy + dz * dz;
                    bool mark = false;
                    if (GRAV) {
                        const float iem = fminf(ie_i, gj.x);               // 1 / max(eps_i, eps_j)
                        const bool soft = r2 * (iem * iem) < 4.f;
                        const float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
                        const float mr = (mine && !soft) ? pj.w * rinv : 0.f;      // m_j / r
                        const float mr3 = mr * (rinv * rinv);
                        acc.ax = fmaf(-mr3, dx, acc.ax);
                        acc.ay = fmaf(-mr3, dy, acc.ay);
                        acc.az = fmaf(-mr3, dz, acc.az);
                        acc.pot -= mr;
                        mark = mine && soft;
                        wsoft += mark ? 1u : 0u;
                    }
                    if (SPH && mine && gas_i && gj.z > 0.f) {
                        const float two_h = fmaxf(two_h_i, 2.f * gj.z);
                        if (r2 < two_h * two_h) {
                            if (CHECK) {
                                ++csph;
                                hsph += evol_mix64((unsigned long long)sm.norig[w][tt]);
                            }
                            ++wsph;
                            if (r2 > 0.f) mark = true;
                        }
                    }
                    if (mark) sbits |= 1ull << tt;
                }
            }
            // Pass 2: the marked pairs of each lane.  Every lane of the warp runs this loop; lanes past
            // the end of the particle array have no marks and read nothing.
            if (__any_sync(0xffffffffu, sbits != 0ull)) {
                const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 gi = (SPH && valid) ? d.grav[s] : z4;
                const float4 hi = (SPH && valid) ? d.hydro[s] : z4;
                const float4 si = (SPH && valid) ? d.snd[s] : z4;
                while (__any_sync(0xffffffffu, sbits != 0ull)) {
                    if (lane == 0) wpass2_slots += 32u;
                    if (sbits) {
                        const int t = __ffsll((long long)sbits) - 1;
                        sbits &= sbits - 1ull;
                        const float4 pj = sm.np[w][t];
                        const float4 gj = sm.ng[w][t];
                        const float dx = evol_wrap(pi.x - pj.x, plen0, pm & 1);
                        const float dy = evol_wrap(pi.y - pj.y, plen1, pm & 2);
                        const float dz = evol_wrap(pi.z - pj.z, plen2, pm & 4);
                        const float r2 = dx * dx + dy * dy + dz * dz;
                        // r and 1/r from one reciprocal square root (coincident particles: both 0)
                        const float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
                        const float r = r2 * rinv;
                        if (GRAV) {
                            const float iem = fminf(ie_i, gj.x);
                            if (r2 * (iem * iem) < 4.f) {          // the same test as pass 1
                                // symmetrised softened pair force and potential (App. B), each side
                                // softened where u < 2 and Newtonian beyond
                                const float mj = pj.w;
                                const float ui = r * ie_i, uj = r * gj.x;
                                const float iui = rinv * eps_i, iuj = rinv * rcp_fast(gj.x);
                                const float rinv3 = rinv * rinv * rinv;
                                const float fi = ui < 2.f ? gsoft_over_r_u(ui, iui) * ie_i * ie_i * ie_i : rinv3;
                                const float fj = uj < 2.f ? gsoft_over_r_u(uj, iuj) * gj.x * gj.x * gj.x : rinv3;
                                float f = -0.5f * mj * (fi + fj);
                                acc.pot += mj * (ui < 2.f ? phisoft_u(ui, iui) * ie_i : -rinv);
                                if (kp.adaptive) {
                                    // adaptive-softening correction (Eq. dLgravdr, mass-weighted reading)
                                    const float ie2 = ie_i * ie_i, je2 = gj.x * gj.x;
                                    const float ci = ui < 2.f ? xu_i * dw_over_u_u(ui, iui) * ie2 * ie2 * ie_i : 0.f;
                                    const float cj = uj < 2.f ? gj.y * dw_over_u_u(uj, iuj) * je2 * je2 * gj.x : 0.f;
                                    f += -0.5f * inv_pi * (ci + mj * inv_mi * cj);
                                }
                                acc.ax += f * dx;
                                acc.ay += f * dy;
                                acc.az += f * dz;
                            }
                        }
                        if (SPH && gas_i && gj.z > 0.f && r2 > 0.f) {
                            const float two_h = fmaxf(two_h_i, 2.f * gj.z);
                            if (r2 < two_h * two_h) {                // the same test as pass 1
                                const float4 hj = sm.nh[w][t];
                                const float4 sj = sm.ns[w][t];
                                const float ihi = si.z, ihj = sj.z;
                                const float uhi = r * ihi, uhj = r * ihj;
                                const float iuhi = rinv * gi.z, iuhj = rinv * gj.z;     // h / r
                                const float ihi2 = ihi * ihi, ihj2 = ihj * ihj;
                                const float kgi = (kp.use_tc ? tc_over_u_u(uhi, iuhi) : dw_over_u_u(uhi, iuhi)) * ihi2 * ihi2 * ihi * inv_pi;
                                const float kgj = (kp.use_tc ? tc_over_u_u(uhj, iuhj) : dw_over_u_u(uhj, iuhj)) * ihj2 * ihj2 * ihj * inv_pi;
                                const float fi = 1.f + gi.w * rcp_fast(pj.w);     // 1 + zeta_i / (m_j Omega*_i)
                                const float fj = 1.f + gj.w * inv_mi;             // 1 + zeta_j / (m_i Omega*_j)
                                const float vx = hi.x - hj.x, vy = hi.y - hj.y, vz = hi.z - hj.z;
                                const float vr = vx * dx + vy * dy + vz * dz;
                                float visc = 0.f;
                                if (vr < 0.f) {
                                    const float hb = 0.5f * (gi.z + gj.z);
                                    const float mu = hb * vr * rcp_fast(r2 + 0.01f * hb * hb);
                                    const float cb = 0.5f * (si.x + sj.x);
                                    const float rb = 0.5f * (si.y + sj.y);
                                    visc = (-kp.alpha * cb * mu + kp.beta * mu * mu) * rcp_fast(rb);
                                }
                                const float gbar = 0.5f * (kgi * fi + kgj * fj);
                                const float pterm_i = hi.w * fi * kgi;
                                const float sc = -pj.w * (pterm_i + hj.w * fj * kgj + visc * gbar);
                                acc.hx += sc * dx;
                                acc.hy += sc * dy;
                                acc.hz += sc * dz;
                                acc.du += pj.w * (pterm_i + 0.5f * visc * gbar) * vr;
                            }
                        }
                    }
                }
            }
            fold();
            nnear = 0;
            __syncwarp();
        };

        const unsigned rootmask = __ballot_sync(0xffffffffu, active);
        const unsigned ltmask = (1u << lane) - 1u;
        // group bounds: particle box, extreme interaction radii
        float gx0 = active ? pi.x : INFINITY, gy0 = active ? pi.y : INFINITY, gz0 = active ? pi.z : INFINITY;
        float gx1 = active ? pi.x : -INFINITY, gy1 = active ? pi.y : -INFINITY, gz1 = active ? pi.z : -INFINITY;
        float emax = (GRAV && active) ? two_eps_i : 0.f, emin = (GRAV && active) ? two_eps_i : INFINITY;
        float hmax = gas_i ? two_h_i : -1.f, hmin = gas_i ? two_h_i : INFINITY;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            gx0 = fminf(gx0, __shfl_xor_sync(0xffffffffu, gx0, o));
            gy0 = fminf(gy0, __shfl_xor_sync(0xffffffffu, gy0, o));
            gz0 = fminf(gz0, __shfl_xor_sync(0xffffffffu, gz0, o));
            gx1 = fmaxf(gx1, __shfl_xor_sync(0xffffffffu, gx1, o));
            gy1 = fmaxf(gy1, __shfl_xor_sync(0xffffffffu, gy1, o));
            gz1 = fmaxf(gz1, __shfl_xor_sync(0xffffffffu, gz1, o));
            emax = fmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, o));
            emin = fminf(emin, __shfl_xor_sync(0xffffffffu, emin, o));
            hmax = fmaxf(hmax, __shfl_xor_sync(0xffffffffu, hmax, o));
            hmin = fminf(hmin, __shfl_xor_sync(0xffffffffu, hmin, o));
        }
        const bool all_gas = SPH && __all_sync(0xffffffffu, !active || gas_i);
        if (!GRAV) emin = 0.f;
        // the group bounds live in shared memory for the traversal (read as broadcasts), which keeps
        // them out of the registers the pair loops need
        if (lane == 0) {
            sm.gbox[w][0] = make_float4(0.5f * (gx0 + gx1), 0.5f * (gy0 + gy1), 0.5f * (gz0 + gz1), 0.f);
            sm.gbox[w][1] = make_float4(0.5f * (gx1 - gx0), 0.5f * (gy1 - gy0), 0.5f * (gz1 - gz0), 0.f);
            sm.gbox[w][2] = make_float4(emax, emin, hmax, hmin);
        }
        __syncwarp();

        int2 *stk = d.wstack + (size_t)(blockIdx.x * WK_WARPS + w) * kp.stack_stride;
        // one stack entry per system present in the group: its root with the mask of its lanes
        int top = 0;
        {
            const int myroot = active ? d.sys_root[d.sys_sorted[s]] : -1;
            const unsigned peers = __match_any_sync(0xffffffffu, myroot);
            const bool leader = active && (__ffs(peers) - 1) == lane;
            const unsigned leaders = __ballot_sync(0xffffffffu, leader);
            if (leader) stk[__popc(leaders & ltmask)] = make_int2(myroot, (int)peers);
            top = __popc(leaders);
        }
        __syncwarp();
        // a traversal pops every node at most once; a larger count can only come from a corrupt
        // tree: stop, flag it and report where
        long long pops = 0;
        const long long pop_cap = 2ll * (long long)(*d.nnodes) + 64;
        while (top > 0) {
            if (++pops > pop_cap) {
                if (lane == 0) {
                    evol_flag(d.err, EVOL_ETIMEOUT);
                    atomicMax(&d.counters[7], 1ull);
                }
                break;
            }
            const int k = min(top, 32);
            top -= k;
            int node = -1;
            unsigned M = 0;
            if (lane < k) {
                const int2 e = stk[top + lane];
                node = e.x;
                M = (unsigned)e.y;
            }
            __syncwarp();
            int4 I = make_int4(0, 0, 0, 0);
            int cls = 0;                     // 0 none, 1 accept all, 2 open all, 3 mixed
            unsigned Ak = 0, Ok = 0;
            if (lane < k) {
                I = d.nI[node];
                const float4 B = d.nB[node];
                const float4 C = d.nC[node];
                const float4 A = GRAV ? d.nA[node] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 G0 = sm.gbox[w][0], G1 = sm.gbox[w][1], G2 = sm.gbox[w][2];
                const float gcx = G0.x, gcy = G0.y, gcz = G0.z, gwx = G1.x, gwy = G1.y, gwz = G1.z;
                const float emax = G2.x, emin = G2.y, hmax = G2.z, hmin = G2.w;
                const float dx = fabsf(evol_wrap(B.x - gcx, plen0, pm & 1));
                const float dy = fabsf(evol_wrap(B.y - gcy, plen1, pm & 2));
                const float dz = fabsf(evol_wrap(B.z - gcz, plen2, pm & 4));
                // nearest and farthest distance of a group point from the node box
                const float nx = fmaxf(dx - (C.x + gwx), 0.f), ny = fmaxf(dy - (C.y + gwy), 0.f),
                            nz = fmaxf(dz - (C.z + gwz), 0.f);
                const float fx = fmaxf(dx + gwx - C.x, 0.f), fy = fmaxf(dy + gwy - C.y, 0.f),
                            fz = fmaxf(dz + gwz - C.z, 0.f);
                const float bnear2 = nx * nx + ny * ny + nz * nz, bfar2 = fx * fx + fy * fy + fz * fz;
                float rup = GRAV ? fmaxf(emax, C.w) : 0.f;
                float rlo = GRAV ? fmaxf(emin, C.w) : 0.f;
                if (SPH && B.w >= 0.f && hmax >= 0.f) {
                    rup = fmaxf(rup, fmaxf(hmax, B.w));
                    if (all_gas) rlo = fmaxf(rlo, fmaxf(hmin, B.w));
                }
                bool acc_all = bnear2 > rup * rup * (1.f + TAU);
                bool open_all = bfar2 < rlo * rlo * (1.f - TAU);
                if (GRAV) {
                    const float ax = fabsf(A.x - gcx), ay = fabsf(A.y - gcy), az = fabsf(A.z - gcz);
                    const float mx = fmaxf(ax - gwx, 0.f), my = fmaxf(ay - gwy, 0.f), mz = fmaxf(az - gwz, 0.f);
                    const float Mx = ax + gwx, My = ay + gwy, Mz = az + gwz;
                    acc_all = acc_all && (mx * mx + my * my + mz * mz > A.w * (1.f + TAU));
                    open_all = open_all || (Mx * Mx + My * My + Mz * Mz < A.w * (1.f - TAU));
                }
                if (acc_all) {
                    cls = 1;
                    Ak = M;
                } else if (open_all) {
                    cls = 2;
                    Ok = M;
                } else {
                    cls = 3;
                }
                sm.bA[w][lane] = A;
                sm.bB[w][lane] = B;
                sm.bC[w][lane] = C;
            }
            __syncwarp();
            // mixed nodes: every lane in the mask applies its own test
            unsigned mm = __ballot_sync(0xffffffffu, cls == 3);
            while (mm) {
                const int kk = __ffs(mm) - 1;
                mm &= mm - 1u;
                const unsigned Mk = __shfl_sync(0xffffffffu, M, kk);
                bool far = false;
                if ((Mk >> lane) & 1u) {
                    const float4 B = sm.bB[w][kk];
                    const float4 C = sm.bC[w][kk];
                    float ex = fabsf(evol_wrap(pi.x - B.x, plen0, pm & 1)) - C.x;
                    float ey = fabsf(evol_wrap(pi.y - B.y, plen1, pm & 2)) - C.y;
                    float ez = fabsf(evol_wrap(pi.z - B.z, plen2, pm & 4)) - C.z;
                    ex = fmaxf(ex, 0.f); ey = fmaxf(ey, 0.f); ez = fmaxf(ez, 0.f);
                    const float bd2 = ex * ex + ey * ey + ez * ez;
                    float R = GRAV ? fmaxf(two_eps_i, C.w) : 0.f;
                    if (SPH && gas_i && B.w >= 0.f) R = fmaxf(R, fmaxf(two_h_i, B.w));
                    far = bd2 > R * R;
                    if (GRAV && far) {
                        const float4 A = sm.bA[w][kk];
                        const float dx = pi.x - A.x, dy = pi.y - A.y, dz = pi.z - A.z;
                        far = dx * dx + dy * dy + dz * dz > A.w;
                    }
                }
                const unsigned Af = __ballot_sync(0xffffffffu, far);
                if (lane == kk) {
                    Ak = Af;
                    Ok = Mk & ~Af;
                }
            }
            // accepted nodes
            const unsigned fa = __ballot_sync(0xffffffffu, Ak != 0u);
            if (CHECK) {
                unsigned f2 = fa;
                while (f2) {
                    const int kk = __ffs(f2) - 1;
                    f2 &= f2 - 1u;
                    const int nk = __shfl_sync(0xffffffffu, node, kk);
                    const unsigned ak = __shfl_sync(0xffffffffu, Ak, kk);
                    if ((ak >> lane) & 1u) {
                        ++cfar;
                        hfar += evol_mix64((unsigned long long)nk);
                    }
                }
            }
            if (GRAV && fa) {
                const int cnt = __popc(fa);
                if (nfar + cnt > FARCAP - 3) flush_far();
                if (Ak) {
                    const int pos = nfar + __popc(fa & ltmask);
                    sm.far_id[w][pos] = node;
                    sm.far_mask[w][pos] = Ak;
                }
                nfar += cnt;
            }
            // opened leaves: their particles go to the near list
            const bool isleaf = (I.x >> 8) & 1;
            unsigned lm = __ballot_sync(0xffffffffu, Ok != 0u && isleaf);
            while (lm) {
                const int kk = __ffs(lm) - 1;
                lm &= lm - 1u;
                const unsigned ok = __shfl_sync(0xffffffffu, Ok, kk);
                const int b0 = __shfl_sync(0xffffffffu, I.z, kk);
                const int e0 = __shfl_sync(0xffffffffu, I.w, kk);
                if (CHECK) {
                    const int ln = __shfl_sync(0xffffffffu, node, kk);
                    if ((ok >> lane) & 1u) hnear += evol_mix64((unsigned long long)ln);
                }
                for (int b = b0; b < e0; b += 32) {
                    const int kc = min(32, e0 - b);
                    if (nnear + kc > NEARCAP) flush_near();
                    if (lane < kc) {
                        sm.near_j[w][nnear + lane] = b + lane;
                        sm.near_mask[w][nnear + lane] = ok;
                    }
                    nnear += kc;
                }
            }
            // opened internal nodes: push their children with the open mask
            const bool io = Ok != 0u && !isleaf;
            int nch = 0;
            int ch[8];
            if (io) {
                const int4 K0 = d.nK0[node], K1 = d.nK1[node];
                ch[0] = K0.x; ch[1] = K0.y; ch[2] = K0.z; ch[3] = K0.w;
                ch[4] = K1.x; ch[5] = K1.y; ch[6] = K1.z; ch[7] = K1.w;
#pragma unroll
                for (int q = 0; q < 8; ++q) nch += ch[q] >= 0 ? 1 : 0;
            }
            int incl = nch;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            if (top + total > kp.stack_cap) {
                if (lane == 0) evol_flag(d.err, EVOL_EOVERFLOW);
                break;
            }
            if (io) {
                int pos = top + incl - nch;
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (q < nch) stk[pos + q] = make_int2(ch[q], (int)Ok);
            }
            top += total;
            __syncwarp();
        }
        if (GRAV && nfar) flush_far();
        if (nnear) flush_near();

        if (!MIXED) {
            tax = acc.ax; tay = acc.ay; taz = acc.az; tpot = acc.pot;
            thx = acc.hx; thy = acc.hy; thz = acc.hz; tdu = acc.du;
        }
        if (valid) {
            float ax = 0.f, ay = 0.f, az = 0.f, pot = 0.f;
            if (GRAV) {
                // self term of the potential: m_i phi(0, eps_i) = -7/5 m_i / eps_i
                const double G = kp.G;
                ax = (float)(G * tax);
                ay = (float)(G * tay);
                az = (float)(G * taz);
                pot = (float)(G * (tpot - 1.4 * (double)pi.w * (double)ie_i));
            }
            ax += (float)thx;
            ay += (float)thy;
            az += (float)thz;
            d.acc[s] = make_float4(ax, ay, az, pot);
            if (SPH) {
                d.dudt[s] = gas_i ? (float)tdu : 0.f;
                const float4 hv = d.hydro[s];
                d.vah[s] = gas_i ? (float)(hv.x * thx + hv.y * thy + hv.z * thz) : 0.f;
            }
            if (CHECK) {
                d.hash3[3 * s + 0] = hfar;
                d.hash3[3 * s + 1] = hnear;
                d.hash3[3 * s + 2] = hsph;
                d.cnt3[3 * s + 0] = cfar;
                d.cnt3[3 * s + 1] = cpp;
                d.cnt3[3 * s + 2] = csph;
            }
        }
        // interaction counters, per lane: summed over the warp
        unsigned long long wf = wfar, wp = wpp, ws = wsph, wo = wsoft;   // warp sums in 64 bits
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            wf += __shfl_xor_sync(0xffffffffu, wf, o);
            wp += __shfl_xor_sync(0xffffffffu, wp, o);
            ws += __shfl_xor_sync(0xffffffffu, ws, o);
            wo += __shfl_xor_sync(0xffffffffu, wo, o);
        }
        if (lane == 0) {
            atomicAdd(&d.counters[0], wf);
            atomicAdd(&d.counters[1], wp);
            atomicAdd(&d.counters[2], ws);
            atomicAdd(&d.counters[8], wo);
            atomicAdd(&d.counters[9], (unsigned long long)wfar_slots);
            atomicAdd(&d.counters[10], (unsigned long long)wnear_slots);
            atomicAdd(&d.counters[11], (unsigned long long)wpass2_slots);
        }
    }
}

template <bool GRAV, bool SPH, bool MIXED, bool CHECK>
void launch_walk(evol_ctx *c, const evol_kparams &kp)
{
    static int blocks_per_sm = -1;
    if (blocks_per_sm < 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_walk<GRAV, SPH, MIXED, CHECK>, WK_THREADS, 0);
        if (blocks_per_sm < 1) blocks_per_sm = 1;
        if (blocks_per_sm > 8) blocks_per_sm = 8;          // stack slots exist for 32 warps per SM
    }
    unsigned long long *q = c->d.counters + 4;
    cudaMemsetAsync(q, 0, sizeof(unsigned long long), c->stream);
    k_walk<GRAV, SPH, MIXED, CHECK><<<c->num_sms * blocks_per_sm, WK_THREADS, 0, c->stream>>>(c->d, kp, q);
}

template <bool GRAV, bool SPH>
void launch_walk_pc(evol_ctx *c, const evol_kparams &kp, bool mixed, bool check)
{
    if (mixed) {
        if (check) launch_walk<GRAV, SPH, true, true>(c, kp);
        else launch_walk<GRAV, SPH, true, false>(c, kp);
    } else {
        if (check) launch_walk<GRAV, SPH, false, true>(c, kp);
        else launch_walk<GRAV, SPH, false, false>(c, kp);
    }
}

}  // namespace

int evol_launch_walk(evol_ctx *c, const evol_particles *p, const evol_params *prm, int do_grav, int do_sph)
{
    evol_kparams kp{};
    kp.n = (int)p->n;
    kp.n_gas = (int)p->n_gas;
    kp.theta = prm->theta;
    kp.G = prm->G;
    kp.gamma = prm->gamma;
    kp.alpha = prm->alpha;
    kp.beta = prm->beta;
    kp.adaptive = prm->adaptive_softening;
    kp.use_tc = prm->use_tc_gradient;
    kp.periodic_mask = prm->periodic_mask;
    for (int a = 0; a < 3; ++a) kp.plen[a] = prm->periodic_hi[a] - prm->periodic_lo[a];
    kp.stack_cap = (int)c->wstack_lim;
    kp.stack_stride = (int)c->wstack_cap;
    bool mixed = prm->precision == EVOL_FP32_MIXED;
    bool check = c->check_mode != 0;
    if (do_grav && do_sph) launch_walk_pc<true, true>(c, kp, mixed, check);
    else if (do_grav) launch_walk_pc<true, false>(c, kp, mixed, check);
    else if (do_sph) launch_walk_pc<false, true>(c, kp, mixed, check);
    return evol_cuda_ok(cudaGetLastError());
}
