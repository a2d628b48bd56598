// Smoothing and softening lengths (Sect. 2.1 Eqs. rho0, etan, iter; Sect. 3 Eqs. hn, nsum,
// densitySPH, drhodr; Sect. 3.1 "gather" view with an enlarged search radius).
//
// A warp owns a group of 32 consecutive particles in key order.  Each lane needs the particles
// within its search radius R_i = 2 L_i (1 + 0.1).  The warp walks the tree once for all lanes,
// popping up to 32 nodes at a time and classifying each against the group's bounding box (skip
// for every lane / open for every lane / test lane by lane, with a 1e-5 relative margin over
// FP32 rounding).  The particles of the opened leaves are gathered: each lane keeps those within
// its own radius, as (distance, mass) pairs, in a private list.  Each lane then solves
//     F(L) = L^3 n(L) - eta^3 = 0,   n(L) = sum_j W(r_ij, L)  (self term included)
// by Newton steps kept inside a bisection bracket on its list, gathering again when 2L leaves
// the cached radius.  F is non-decreasing in L, so the root is unique.  With w(u) = pi L^3 W
// the sums are dimensionless:
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
constexpr float TAU = 1e-5f;          // safety margin of the group-level bounds

enum { ST_DONE = 0, ST_ACTIVE = 1, ST_LAST = 2 };

constexpr int GCAP = 64;              // staged leaf particles per warp

struct LenSmem {
    float4 bB[LW_WARPS][32];
    float4 bC[LW_WARPS][32];
    int gj[LW_WARPS][GCAP];           // staged particle index
    unsigned gmask[LW_WARPS][GCAP];   // lanes that opened its leaf
    float4 gp[LW_WARPS][GCAP];        // position, mass (mass < 0: excluded species)
};

template <int MODE>
__global__ void __launch_bounds__(LW_THREADS, 6) k_lengths(evol_dev d, evol_kparams kp, int list_cap,
                                                        unsigned long long *queue)
{
    __shared__ LenSmem sm;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int wslot = blockIdx.x * LW_WARPS + w;
    float2 *lst = reinterpret_cast<float2 *>(d.cand_leaf) + (size_t)wslot * list_cap * 32;
    int2 *stk = d.wstack + (size_t)wslot * kp.stack_cap;
    const int n = kp.n;
    const int ngroups = (n + 31) >> 5;
    const float eta = MODE == 0 ? kp.eta_h : kp.eta_e;
    const float eta3 = eta * eta * eta;
    const float inv_pi = 1.f / EVOL_PI_F;
    const float plen0 = kp.plen[0], plen1 = kp.plen[1], plen2 = kp.plen[2];
    const int pm = kp.periodic_mask;

    for (;;) {
        int g = 0;
        if (lane == 0) g = (int)atomicAdd(queue, 1ull);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= ngroups) break;
        const int s = g * 32 + lane;
        const bool valid = s < n;
        const float4 pi4 = valid ? d.pos[s] : make_float4(0.f, 0.f, 0.f, 0.f);
        const bool gas_i = valid && d.orig[s] < kp.n_gas;
        const bool act = MODE == 0 ? gas_i : valid;
        const float side = valid ? d.fcube[4 * d.sys_sorted[s] + 3] : 1.f;     // the system's root cube
        float L = 0.f;
        if (act) {
            L = MODE == 0 ? d.len_h[s] : d.len_eps[s];
            if (!(L > 0.f) || !(L < 1e30f)) L = side / cbrtf((float)n);
        }
        float lo = 0.f, hi = INFINITY;
        int status = act ? ST_ACTIVE : ST_DONE;
        bool stale = act;                  // needs a (re)gather before its sums are valid
        float Rc = 0.f;
        int cnt = 0;                        // entries in this lane's list
        int iters = 0, walks = 0;
        // group box of the lanes' positions (fixed for the group)
        float gx0 = act ? pi4.x : INFINITY, gy0 = act ? pi4.y : INFINITY, gz0 = act ? pi4.z : INFINITY;
        float gx1 = act ? pi4.x : -INFINITY, gy1 = act ? pi4.y : -INFINITY, gz1 = act ? pi4.z : -INFINITY;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            gx0 = fminf(gx0, __shfl_xor_sync(0xffffffffu, gx0, o));
            gy0 = fminf(gy0, __shfl_xor_sync(0xffffffffu, gy0, o));
            gz0 = fminf(gz0, __shfl_xor_sync(0xffffffffu, gz0, o));
            gx1 = fmaxf(gx1, __shfl_xor_sync(0xffffffffu, gx1, o));
            gy1 = fmaxf(gy1, __shfl_xor_sync(0xffffffffu, gy1, o));
            gz1 = fmaxf(gz1, __shfl_xor_sync(0xffffffffu, gz1, o));
        }
        const float gcx = 0.5f * (gx0 + gx1), gcy = 0.5f * (gy0 + gy1), gcz = 0.5f * (gz0 + gz1);
        const float gwx = 0.5f * (gx1 - gx0), gwy = 0.5f * (gy1 - gy0), gwz = 0.5f * (gz1 - gz0);

        while (__any_sync(0xffffffffu, status != ST_DONE)) {
            if (walks >= MAX_WALKS) {
                if (status != ST_DONE) evol_flag(d.err, EVOL_ENOCONV);
                break;
            }
            // ---- gather: the stale lanes collect the particles within their radius ----
            if (__any_sync(0xffffffffu, stale)) {
                ++walks;
                if (stale) {
                    Rc = 2.f * L * SEARCH_MARGIN;
                    cnt = 0;
                }
                const bool coll = stale;
                const float R2 = coll ? Rc * Rc : 0.f;
                float rmax = coll ? Rc : 0.f, rmin = coll ? Rc : INFINITY;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
                    rmin = fminf(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
                }
                bool over = false;
                bool broken = false;
                int ng = 0;
                auto gather_flush = [&]() {
                    __syncwarp();
                    for (int l = lane; l < ng; l += 32) {
                        const int j = sm.gj[w][l];
                        float4 p = d.pos[j];
                        if (MODE == 0 && d.orig[j] >= kp.n_gas) p.w = -1.f;
                        sm.gp[w][l] = p;
                    }
                    __syncwarp();
                    for (int t = 0; t < ng; ++t) {
                        const float4 pj = sm.gp[w][t];
                        if (((sm.gmask[w][t] >> lane) & 1u) && pj.w >= 0.f) {
                            const float dx = evol_wrap(pi4.x - pj.x, plen0, pm & 1);
                            const float dy = evol_wrap(pi4.y - pj.y, plen1, pm & 2);
                            const float dz = evol_wrap(pi4.z - pj.z, plen2, pm & 4);
                            const float r2 = dx * dx + dy * dy + dz * dz;
                            if (r2 < R2) {
                                if (cnt < list_cap) lst[(size_t)cnt * 32 + lane] = make_float2(sqrtf(r2), pj.w);
                                else over = true;
                                ++cnt;
                            }
                        }
                    }
                    ng = 0;
                    __syncwarp();
                };
                // one stack entry per system present among the collecting lanes
                int top = 0;
                {
                    const int myroot = coll ? d.sys_root[d.sys_sorted[s]] : -1;
                    const unsigned peers = __match_any_sync(0xffffffffu, myroot);
                    const bool leader = coll && (__ffs(peers) - 1) == lane;
                    const unsigned leaders = __ballot_sync(0xffffffffu, leader);
                    if (leader) stk[__popc(leaders & ((1u << lane) - 1u))] = make_int2(myroot, (int)peers);
                    top = __popc(leaders);
                }
                __syncwarp();
                long long pops = 0;
                const long long pop_cap = 2ll * (long long)(*d.nnodes) + 64;
                while (top > 0) {
                    if (++pops > pop_cap) {        // corrupt tree: stop, flag and report where
                        if (lane == 0) {
                            evol_flag(d.err, EVOL_ETIMEOUT);
                            atomicMax(&d.counters[7], 2ull);
                        }
                        broken = true;
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
                    int cls = 0;              // 0 none/skip, 2 open all, 3 mixed
                    unsigned Ok = 0;
                    if (lane < k) {
                        I = d.nI[node];
                        const float4 B = d.nB[node];
                        const float4 C = d.nC[node];
                        if (MODE == 1 || B.w >= 0.f) {
                            const float dx = fabsf(evol_wrap(B.x - gcx, plen0, pm & 1));
                            const float dy = fabsf(evol_wrap(B.y - gcy, plen1, pm & 2));
                            const float dz = fabsf(evol_wrap(B.z - gcz, plen2, pm & 4));
                            const float nx = fmaxf(dx - (C.x + gwx), 0.f), ny = fmaxf(dy - (C.y + gwy), 0.f),
                                        nz = fmaxf(dz - (C.z + gwz), 0.f);
                            const float fx = fmaxf(dx + gwx - C.x, 0.f), fy = fmaxf(dy + gwy - C.y, 0.f),
                                        fz = fmaxf(dz + gwz - C.z, 0.f);
                            const float bnear2 = nx * nx + ny * ny + nz * nz, bfar2 = fx * fx + fy * fy + fz * fz;
                            if (bnear2 >= rmax * rmax * (1.f + TAU)) {
                                cls = 0;
                            } else if (bfar2 < rmin * rmin * (1.f - TAU)) {
                                cls = 2;
                                Ok = M;
                            } else {
                                cls = 3;
                            }
                        }
                        sm.bB[w][lane] = B;
                        sm.bC[w][lane] = C;
                    }
                    __syncwarp();
                    unsigned mm = __ballot_sync(0xffffffffu, cls == 3);
                    while (mm) {
                        const int kk = __ffs(mm) - 1;
                        mm &= mm - 1u;
                        const unsigned Mk = __shfl_sync(0xffffffffu, M, kk);
                        bool open = false;
                        if ((Mk >> lane) & 1u) {
                            const float4 B = sm.bB[w][kk];
                            const float4 C = sm.bC[w][kk];
                            float ex = fabsf(evol_wrap(pi4.x - B.x, plen0, pm & 1)) - C.x;
                            float ey = fabsf(evol_wrap(pi4.y - B.y, plen1, pm & 2)) - C.y;
                            float ez = fabsf(evol_wrap(pi4.z - B.z, plen2, pm & 4)) - C.z;
                            ex = fmaxf(ex, 0.f); ey = fmaxf(ey, 0.f); ez = fmaxf(ez, 0.f);
                            open = ex * ex + ey * ey + ez * ez < R2;
                        }
                        const unsigned Of = __ballot_sync(0xffffffffu, open);
                        if (lane == kk) Ok = Of;
                    }
                    // opened leaves: stage their particles, then each lane keeps those within its radius
                    const bool isleaf = (I.x >> 8) & 1;
                    unsigned lm = __ballot_sync(0xffffffffu, Ok != 0u && isleaf);
                    while (lm) {
                        const int kk = __ffs(lm) - 1;
                        lm &= lm - 1u;
                        const unsigned ok = __shfl_sync(0xffffffffu, Ok, kk);
                        const int b0 = __shfl_sync(0xffffffffu, I.z, kk);
                        const int e0 = __shfl_sync(0xffffffffu, I.w, kk);
                        for (int b = b0; b < e0; b += 32) {
                            const int kc = min(32, e0 - b);
                            if (ng + kc > GCAP) gather_flush();
                            if (lane < kc) {
                                sm.gj[w][ng + lane] = b + lane;
                                sm.gmask[w][ng + lane] = ok;
                            }
                            ng += kc;
                        }
                    }
                    // opened internal nodes: push children
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
                        broken = true;
                        break;
                    }
                    if (io) {
                        const int pos = top + incl - nch;
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            if (q < nch) stk[pos + q] = make_int2(ch[q], (int)Ok);
                    }
                    top += total;
                    __syncwarp();
                }
                if (broken) break;
                if (ng) gather_flush();
                stale = false;
                if (over) {
                    // more neighbours than the list holds: the radius is too large; shrink, gather again
                    float Ln = 0.75f * L;
                    if (Ln <= lo) Ln = 0.5f * (lo + L);
                    L = Ln;
                    stale = true;
                    cnt = 0;
                }
            }
            // ---- Newton / bisection on the private lists ----
            for (int sweep = 0;; ++sweep) {
                const bool need = (status == ST_ACTIVE || status == ST_LAST) && !stale;
                if (!__any_sync(0xffffffffu, need)) break;
                if (sweep > 2 * MAX_ITERS + 8) {   // cannot happen: every active lane converges or stops
                    if (lane == 0) {
                        evol_flag(d.err, EVOL_ETIMEOUT);
                        atomicMax(&d.counters[7], 3ull);
                    }
                    status = ST_DONE;
                    stale = false;
                    break;
                }
                float Sw = 0.f, Suw = 0.f, Smw = 0.f, Smuw = 0.f;
                const float Linv = need ? 1.f / L : 0.f;
                const float twoL = 2.f * L;
                const int my = need ? cnt : 0;
                int mx = my;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                for (int e = 0; e < mx; ++e) {
                    if (e < my) {
                        const float2 rm = lst[(size_t)e * 32 + lane];
                        if (rm.x < twoL) {
                            const float u = rm.x * Linv;
                            float wv, dw;
                            evol_w_dw(u, wv, dw);
                            Sw += wv;
                            Suw += u * dw;
                            if (MODE == 0) {
                                Smw += rm.y * wv;
                                Smuw += rm.y * u * dw;
                            } else {
                                Smw += rm.y * evol_dphideps(u);
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
    kp.stack_cap = (int)c->wstack_cap;
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
