// Smoothing and softening lengths (Sect. 2.1 Eqs. rho0, etan, iter; Sect. 3 Eqs. hn, nsum,
// densitySPH, drhodr; Sect. 3.1 "gather" view with an enlarged search radius).
//
// A warp owns a group of 32 consecutive particles in key order.  It walks the tree once with
// per-lane search radii R_i = 2 L_i (1 + 0.1) and records every leaf that any lane must open,
// with the mask of those lanes, in a per-warp candidate list.  Each lane then solves
//     F(L) = L^3 n(L) - eta^3 = 0,   n(L) = sum_j W(r_ij, L)  (self term included)
// by Newton steps kept inside a bisection bracket, re-using the list while 2L stays inside
// the cached radius and walking again otherwise.  F is non-decreasing in L, so the root is
// unique; with w(u) = pi L^3 W the sums are kept dimensionless:
//     F = Sw/pi - eta^3,  F' = -Suw/(pi L),  Sw = sum w(u),  Suw = sum u w'(u).
// Outputs (mode 0, gas h):   rho = Smw/(pi h^3), Omega* = -Suw/(3 Sw),
//                           zeta = (3 Smw + Smuw)/(3 Sw)          (Sect. 3, Eq. drhodr)
// Outputs (mode 1, eps):     Upsilon = -Suw/(3 Sw),
//                           X = -(pi eps^2/(3 Sw)) sum_k m_k eps^2 dphi/deps   (Sect. 2.1)
#include <cuda_runtime.h>
#include <stdint.h>

#include "evol_internal.cuh"

namespace {

constexpr int LW_THREADS = 128;
constexpr int LW_WARPS = LW_THREADS / 32;
constexpr int MAX_ITERS = 60;
constexpr int MAX_WALKS = 24;
constexpr float SEARCH_MARGIN = 1.1f;
constexpr float CONV_TOL = 1e-6f;     // relative step below which one last evaluation is taken

enum { ST_DONE = 0, ST_ACTIVE = 1, ST_LAST = 2 };

template <int MODE>
__global__ void __launch_bounds__(LW_THREADS) k_lengths(evol_dev d, evol_kparams kp, int cand_cap,
                                                        unsigned long long *queue)
{
    const int lane = threadIdx.x & 31;
    const int wslot = blockIdx.x * LW_WARPS + (threadIdx.x >> 5);
    int2 *cl = reinterpret_cast<int2 *>(d.cand_leaf) + (size_t)wslot * cand_cap;
    uint32_t *cm = d.cand_mask + (size_t)wslot * cand_cap;
    const int n = kp.n;
    const int ngroups = (n + 31) >> 5;
    const int nn = *d.nnodes;
    const float eta = MODE == 0 ? kp.eta_h : kp.eta_e;
    const float eta3 = eta * eta * eta;
    const float inv_pi = 1.f / EVOL_PI_F;
    float plen[3] = {kp.plen[0], kp.plen[1], kp.plen[2]};
    const int pm = kp.periodic_mask;
    const float side = d.fcube[3];

    for (;;) {
        int g = 0;
        if (lane == 0) g = (int)atomicAdd(queue, 1ull);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= ngroups) break;
        const int s = g * 32 + lane;
        const bool valid = s < n;
        float4 pi4 = valid ? d.pos[s] : make_float4(0.f, 0.f, 0.f, 0.f);
        const bool gas_i = valid && d.orig[s] < kp.n_gas;
        const bool act = MODE == 0 ? gas_i : valid;
        float L = 0.f;
        if (act) {
            L = MODE == 0 ? d.len_h[s] : d.len_eps[s];
            if (!(L > 0.f) || !(L < 1e30f)) L = side / cbrtf((float)n);
        }
        float lo = 0.f, hi = INFINITY;
        int status = act ? ST_ACTIVE : ST_DONE;
        bool stale = act;                  // needs a (re)walk before its sums are valid
        float Rc = 0.f;
        int iters = 0, walks = 0;

        while (__any_sync(0xffffffffu, status != ST_DONE)) {
            // ---- walk: collect the leaves any stale lane must open ----
            if (__any_sync(0xffffffffu, stale)) {
                if (stale) Rc = 2.f * L * SEARCH_MARGIN;
                ++walks;
                const unsigned rootmask = __ballot_sync(0xffffffffu, status != ST_DONE);
                const float R2 = Rc * Rc;
                int node = 0, nc = 0;
                unsigned lvlmask = 0;
                bool overflow = false;
                while (node < nn) {
                    const int4 I = d.nI[node];
                    const int lev = I.x & 255;
                    const unsigned M = lev == 0 ? rootmask : __shfl_sync(0xffffffffu, lvlmask, lev - 1);
                    bool open = false;
                    if ((M >> lane) & 1u) {
                        const float4 B = d.nB[node];
                        if (MODE == 1 || B.w >= 0.f) {
                            const float4 C = d.nC[node];
                            float ex = fabsf(evol_wrap(pi4.x - B.x, plen[0], pm & 1)) - C.x;
                            float ey = fabsf(evol_wrap(pi4.y - B.y, plen[1], pm & 2)) - C.y;
                            float ez = fabsf(evol_wrap(pi4.z - B.z, plen[2], pm & 4)) - C.z;
                            ex = fmaxf(ex, 0.f); ey = fmaxf(ey, 0.f); ez = fmaxf(ez, 0.f);
                            open = ex * ex + ey * ey + ez * ez < R2;
                        }
                    }
                    const unsigned O = __ballot_sync(0xffffffffu, open);
                    if (O == 0u) {
                        node = I.y;
                    } else if (I.x >> 8) {
                        if (nc < cand_cap) {
                            if (lane == 0) {
                                cl[nc] = make_int2(I.z, I.w);
                                cm[nc] = O;
                            }
                            ++nc;
                        } else {
                            overflow = true;
                        }
                        node = I.y;
                    } else {
                        if (lane == lev) lvlmask = O;
                        node = node + 1;
                    }
                }
                __syncwarp();
                if (overflow) {
                    if (lane == 0) evol_flag(d.err, EVOL_EOVERFLOW);
                    break;
                }
                stale = false;
                // ---- Newton / bisection on the cached list ----
                for (;;) {
                    const bool need = (status == ST_ACTIVE || status == ST_LAST) && !stale;
                    if (!__any_sync(0xffffffffu, need)) break;
                    float Sw = 0.f, Suw = 0.f, Smw = 0.f, Smuw = 0.f;
                    const float Linv = need ? 1.f / L : 0.f;
                    const float L2x4 = 4.f * L * L;
                    for (int e = 0; e < nc; ++e) {
                        const int2 rg = cl[e];
                        const unsigned msk = cm[e];
                        const bool mine = need && ((msk >> lane) & 1u);
                        if (!__any_sync(0xffffffffu, mine)) continue;
                        for (int j = rg.x; j < rg.y; ++j) {
                            const float4 pj = d.pos[j];
                            if (MODE == 0 && d.orig[j] >= kp.n_gas) continue;
                            if (!mine) continue;
                            float dx = evol_wrap(pi4.x - pj.x, plen[0], pm & 1);
                            float dy = evol_wrap(pi4.y - pj.y, plen[1], pm & 2);
                            float dz = evol_wrap(pi4.z - pj.z, plen[2], pm & 4);
                            const float r2 = dx * dx + dy * dy + dz * dz;
                            if (r2 < L2x4) {
                                const float u = sqrtf(r2) * Linv;
                                float w, dw;
                                evol_w_dw(u, w, dw);
                                Sw += w;
                                Suw += u * dw;
                                if (MODE == 0) {
                                    Smw += pj.w * w;
                                    Smuw += pj.w * u * dw;
                                } else {
                                    Smw += pj.w * evol_dphideps(u);
                                }
                            }
                        }
                    }
                    if (status == ST_LAST && !stale) {
                        const float nsum = Sw * inv_pi * Linv * Linv * Linv;
                        if (MODE == 0) {
                            d.len_h[s] = L;
                            d.nh[s] = nsum;
                            d.rho[s] = Smw * inv_pi * Linv * Linv * Linv;
                            d.omega[s] = -Suw / (3.f * Sw);
                            d.zeta[s] = (3.f * Smw + Smuw) / (3.f * Sw);
                        } else {
                            d.len_eps[s] = L;
                            d.neps[s] = nsum;
                            d.ups[s] = -Suw / (3.f * Sw);
                            d.X[s] = -EVOL_PI_F * L * L * Smw / (3.f * Sw);
                        }
                        status = ST_DONE;
                    } else if (status == ST_ACTIVE && !stale) {
                        ++iters;
                        const float F = Sw * inv_pi - eta3;
                        const float Fp = -Suw * inv_pi * Linv;
                        if (F < 0.f) lo = L;
                        if (F > 0.f) hi = L;
                        float Ln;
                        if (F == 0.f) {
                            Ln = L;
                        } else {
                            Ln = Fp > 0.f ? L - F / Fp : (hi < INFINITY ? 0.5f * (lo + hi) : 2.f * L);
                            if (!(Ln > lo && Ln < hi)) Ln = hi < INFINITY ? 0.5f * (lo + hi) : 2.f * L;
                        }
                        const bool conv = fabsf(Ln - L) <= CONV_TOL * L || (hi < INFINITY && hi - lo <= 1e-7f * hi);
                        L = Ln;
                        if (conv) status = ST_LAST;
                        if (iters >= MAX_ITERS) {
                            evol_flag(d.err, EVOL_ENOCONV);
                            status = ST_LAST;
                        }
                        if (2.f * L >= Rc) stale = true;
                        if (L > 4.f * side) {             // no root: fewer neighbours than required
                            evol_flag(d.err, EVOL_ENOCONV);
                            status = ST_DONE;
                            stale = false;
                            if (MODE == 0) d.len_h[s] = L; else d.len_eps[s] = L;
                        }
                    }
                }
            }
            if (walks >= MAX_WALKS && __any_sync(0xffffffffu, status != ST_DONE)) {
                if (status != ST_DONE) evol_flag(d.err, EVOL_ENOCONV);
                break;
            }
        }
        // iteration count for the diagnostics
        int it = iters;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) it += __shfl_xor_sync(0xffffffffu, it, o);
        if (lane == 0) atomicAdd(&d.counters[3], (unsigned long long)it);
    }
}

}  // namespace

int evol_launch_lengths(evol_ctx *c, const evol_particles *p, const evol_params *prm, int mode)
{
    evol_kparams kp{};
    kp.n = (int)p->n;
    kp.n_gas = (int)p->n_gas;
    kp.eta_h = 0.5f * cbrtf(3.f * prm->n_nei_sph / (4.f * EVOL_PI_F));
    kp.eta_e = 0.5f * cbrtf(3.f * prm->n_nei_grav / (4.f * EVOL_PI_F));
    kp.periodic_mask = prm->periodic_mask;
    for (int a = 0; a < 3; ++a) kp.plen[a] = prm->periodic_hi[a] - prm->periodic_lo[a];
    unsigned long long *q = c->d.counters + (mode == 0 ? 5 : 6);
    cudaMemsetAsync(q, 0, sizeof(unsigned long long), c->stream);
    int blocks = (int)(c->cand_slots / LW_WARPS);
    if (mode == 0)
        k_lengths<0><<<blocks, LW_THREADS, 0, c->stream>>>(c->d, kp, (int)c->cand_cap, q);
    else
        k_lengths<1><<<blocks, LW_THREADS, 0, c->stream>>>(c->d, kp, (int)c->cand_cap, q);
    return evol_cuda_ok(cudaGetLastError());
}

int evol_lengths_warps_per_block() { return LW_WARPS; }
