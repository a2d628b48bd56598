// Force walk: gravity (Sect. 2.1-2.2, App. B) and SPH pressure + viscosity forces and du/dt
// (Sect. 3, Eqs. motionvarmass1, thermalvarmass1, mu_visc) in one traversal of the tree, as
// the paper does its second walk (Sect. 3.1).
//
// A warp owns 32 consecutive particles in key order and walks the pre-order node list once.
// Every lane applies its own opening test to each node the warp visits, so the result is the
// per-particle tree walk: node A is a far node for particle i iff
//     |r_i - com_A| > l_A/theta + delta_A                                     (Eq. opcrit)
// and A's particle box lies farther than R_iA = 2 max(eps_i, epsmax_A) (and, for gas i and a
// node holding gas, farther than 2 max(h_i, hmax_A)); otherwise it is opened.  A ballot gives
// the accept mask and the open mask; the open mask of each level is kept in lane `level` of a
// register so that descending and skipping need no stack.  Far nodes (with their accept mask)
// and the particles of opened leaves (with their open mask) are staged in shared memory and
// evaluated in batches: far nodes by monopole + traceless quadrupole about the centre of mass,
// near particles by the symmetrised softened pair force plus the adaptive-softening
// correction, and, for gas pairs with r < 2 max(h_i, h_j), the SPH terms.
#include <cuda_runtime.h>
#include <stdint.h>

#include "evol_internal.cuh"

namespace {

constexpr int WK_THREADS = 128;
constexpr int WK_WARPS = WK_THREADS / 32;
constexpr int FARCAP = 64;
constexpr int NEARCAP = 64;

struct WalkSmem {
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
};

template <bool MIXED>
struct Acc {
    float ax = 0.f, ay = 0.f, az = 0.f, pot = 0.f;      // gravity (without G)
    float hx = 0.f, hy = 0.f, hz = 0.f, du = 0.f;       // SPH
};

template <bool GRAV, bool SPH, bool MIXED, bool CHECK>
__global__ void __launch_bounds__(WK_THREADS) k_walk(evol_dev d, evol_kparams kp, unsigned long long *queue)
{
    __shared__ WalkSmem sm;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int n = kp.n;
    const int ngroups = (n + 31) >> 5;
    const int nn = *d.nnodes;
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
        const float4 gi = valid ? d.grav[s] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 hi = (valid && SPH) ? d.hydro[s] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 si = (valid && SPH) ? d.snd[s] : make_float4(0.f, 0.f, 0.f, 0.f);
        const bool gas_i = SPH && valid && gi.z > 0.f;
        const bool active = valid && (GRAV || gas_i);
        const float ie_i = gi.x, two_eps_i = GRAV && active ? 2.f / gi.x : 0.f;
        const float two_h_i = gas_i ? 2.f * gi.z : 0.f;
        const float inv_mi = valid ? 1.f / pi.w : 0.f;

        Acc<MIXED> acc;
        double tax = 0, tay = 0, taz = 0, tpot = 0, thx = 0, thy = 0, thz = 0, tdu = 0;
        unsigned long long hfar = 0, hnear = 0, hsph = 0;
        int cfar = 0, cpp = 0, csph = 0;
        unsigned long long wfar = 0, wpp = 0, wsph = 0;

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
            for (int l = lane; l < nfar; l += 32) {
                const int id = sm.far_id[w][l];
                sm.fA[w][l] = d.nA[id];
                sm.fQ0[w][l] = d.nQ0[id];
                sm.fQ1[w][l] = d.nQ1[id];
            }
            __syncwarp();
            for (int e = 0; e < nfar; ++e) {
                const unsigned msk = sm.far_mask[w][e];
                wfar += __popc(msk);
                if ((msk >> lane) & 1u) {
                    const float4 A = sm.fA[w][e], Q0 = sm.fQ0[w][e], Q1 = sm.fQ1[w][e];
                    const float dx = pi.x - A.x, dy = pi.y - A.y, dz = pi.z - A.z;
                    const float d2 = dx * dx + dy * dy + dz * dz;
                    const float rinv = rsqrtf(d2);
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
                sm.np[w][l] = d.pos[j];
                sm.ng[w][l] = d.grav[j];
                if (SPH) {
                    sm.nh[w][l] = d.hydro[j];
                    sm.ns[w][l] = d.snd[j];
                }
                if (CHECK) sm.norig[w][l] = d.orig[j];
            }
            __syncwarp();
            for (int t = 0; t < nnear; ++t) {
                const unsigned msk = sm.near_mask[w][t];
                const int j = sm.near_j[w][t];
                const bool mine = ((msk >> lane) & 1u) && j != s;
                {
                    const int sl = j - g * 32;
                    const unsigned self = (sl >= 0 && sl < 32) ? ((msk >> sl) & 1u) : 0u;
                    wpp += __popc(msk) - self;
                }
                if (!mine) continue;
                if (CHECK) ++cpp;
                const float4 pj = sm.np[w][t];
                const float4 gj = sm.ng[w][t];
                const float dx = evol_wrap(pi.x - pj.x, plen0, pm & 1);
                const float dy = evol_wrap(pi.y - pj.y, plen1, pm & 2);
                const float dz = evol_wrap(pi.z - pj.z, plen2, pm & 4);
                const float r2 = dx * dx + dy * dy + dz * dz;
                const float r = sqrtf(r2);
                if (GRAV) {
                    const float rinv = rsqrtf(r2);
                    const float ui = r * ie_i, uj = r * gj.x;
                    const float rinv3 = rinv * rinv * rinv;
                    const float fi = ui < 2.f ? evol_gsoft_over_r(ui) * ie_i * ie_i * ie_i : rinv3;
                    const float fj = uj < 2.f ? evol_gsoft_over_r(uj) * gj.x * gj.x * gj.x : rinv3;
                    float f = -0.5f * pj.w * (fi + fj);
                    acc.pot += pj.w * (ui < 2.f ? evol_phisoft(ui) * ie_i : -rinv);
                    if (kp.adaptive) {
                        const float ie2 = ie_i * ie_i, je2 = gj.x * gj.x;
                        const float ci = ui < 2.f ? gi.y * evol_dw_over_u(ui) * ie2 * ie2 * ie_i : 0.f;
                        const float cj = uj < 2.f ? gj.y * evol_dw_over_u(uj) * je2 * je2 * gj.x : 0.f;
                        f += -0.5f * inv_pi * (ci + pj.w * inv_mi * cj);
                    }
                    acc.ax += f * dx;
                    acc.ay += f * dy;
                    acc.az += f * dz;
                }
                if (SPH && gas_i && gj.z > 0.f) {
                    const float two_h = fmaxf(two_h_i, 2.f * gj.z);
                    if (r2 < two_h * two_h) {
                        if (CHECK) {
                            ++csph;
                            hsph += evol_mix64((unsigned long long)sm.norig[w][t]);
                        }
                        ++wsph;
                        if (r2 > 0.f) {
                            const float4 hj = sm.nh[w][t];
                            const float4 sj = sm.ns[w][t];
                            const float ihi = si.z, ihj = sj.z;
                            const float uhi = r * ihi, uhj = r * ihj;
                            const float ihi2 = ihi * ihi, ihj2 = ihj * ihj;
                            const float kgi = (kp.use_tc ? evol_tc_over_u(uhi) : evol_dw_over_u(uhi)) * ihi2 * ihi2 * ihi * inv_pi;
                            const float kgj = (kp.use_tc ? evol_tc_over_u(uhj) : evol_dw_over_u(uhj)) * ihj2 * ihj2 * ihj * inv_pi;
                            const float fi = 1.f + gi.w / pj.w;       // 1 + zeta_i / (m_j Omega*_i)
                            const float fj = 1.f + gj.w * inv_mi;     // 1 + zeta_j / (m_i Omega*_j)
                            const float vx = hi.x - hj.x, vy = hi.y - hj.y, vz = hi.z - hj.z;
                            const float vr = vx * dx + vy * dy + vz * dz;
                            float visc = 0.f;
                            if (vr < 0.f) {
                                const float hb = 0.5f * (gi.z + gj.z);
                                const float mu = hb * vr / (r2 + 0.01f * hb * hb);
                                const float cb = 0.5f * (si.x + sj.x);
                                const float rb = 0.5f * (si.y + sj.y);
                                visc = (-kp.alpha * cb * mu + kp.beta * mu * mu) / rb;
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
            fold();
            nnear = 0;
            __syncwarp();
        };

        const unsigned rootmask = __ballot_sync(0xffffffffu, active);
        int node = rootmask ? 0 : nn;
        unsigned lvlmask = 0;
        while (node < nn) {
            const int4 I = d.nI[node];
            const int lev = I.x & 255;
            const unsigned M = lev == 0 ? rootmask : __shfl_sync(0xffffffffu, lvlmask, lev - 1);
            bool far = false;
            if ((M >> lane) & 1u) {
                const float4 B = d.nB[node];
                const float4 C = d.nC[node];
                float ex = fabsf(evol_wrap(pi.x - B.x, plen0, pm & 1)) - C.x;
                float ey = fabsf(evol_wrap(pi.y - B.y, plen1, pm & 2)) - C.y;
                float ez = fabsf(evol_wrap(pi.z - B.z, plen2, pm & 4)) - C.z;
                ex = fmaxf(ex, 0.f); ey = fmaxf(ey, 0.f); ez = fmaxf(ez, 0.f);
                const float bd2 = ex * ex + ey * ey + ez * ez;
                float R = GRAV ? fmaxf(two_eps_i, C.w) : 0.f;
                if (SPH && gas_i && B.w >= 0.f) R = fmaxf(R, fmaxf(two_h_i, B.w));
                far = bd2 > R * R;
                if (GRAV && far) {
                    const float4 A = d.nA[node];
                    const float dx = pi.x - A.x, dy = pi.y - A.y, dz = pi.z - A.z;
                    far = dx * dx + dy * dy + dz * dz > A.w;
                }
            }
            const unsigned Af = __ballot_sync(0xffffffffu, far);
            const unsigned O = M & ~Af;
            if (CHECK && ((Af >> lane) & 1u)) {
                ++cfar;
                hfar += evol_mix64((unsigned long long)node);
            }
            if (GRAV && Af) {
                if (lane == 0) {
                    sm.far_id[w][nfar] = node;
                    sm.far_mask[w][nfar] = Af;
                }
                if (++nfar == FARCAP) flush_far();
            }
            if (O) {
                if (I.x >> 8) {
                    if (CHECK && ((O >> lane) & 1u)) hnear += evol_mix64((unsigned long long)node);
                    for (int b = I.z; b < I.w; b += 32) {
                        const int k = min(32, I.w - b);
                        if (nnear + k > NEARCAP) flush_near();
                        if (lane < k) {
                            sm.near_j[w][nnear + lane] = b + lane;
                            sm.near_mask[w][nnear + lane] = O;
                        }
                        nnear += k;
                    }
                    node = I.y;
                } else {
                    if (lane == lev) lvlmask = O;
                    node = node + 1;
                }
            } else {
                node = I.y;
            }
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
                d.vah[s] = gas_i ? (float)(hi.x * thx + hi.y * thy + hi.z * thz) : 0.f;
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
        // interaction counters: wfar / wpp are warp-uniform; wsph is per lane
        unsigned long long ws = wsph;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ws += __shfl_xor_sync(0xffffffffu, ws, o);
        if (lane == 0) {
            atomicAdd(&d.counters[0], wfar);
            atomicAdd(&d.counters[1], wpp);
            atomicAdd(&d.counters[2], ws);
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
    bool mixed = prm->precision == EVOL_FP32_MIXED;
    bool check = c->check_mode != 0;
    if (do_grav && do_sph) launch_walk_pc<true, true>(c, kp, mixed, check);
    else if (do_grav) launch_walk_pc<true, false>(c, kp, mixed, check);
    else if (do_sph) launch_walk_pc<false, true>(c, kp, mixed, check);
    return evol_cuda_ok(cudaGetLastError());
}
