// Smoothing and softening lengths (Sect. 2.1 Eqs. rho0, etan, iter; Sect. 3 Eqs. hn, nsum,
// densitySPH, drhodr; Sect. 3.1 "gather" view with an enlarged search radius).
//
// Each particle i needs the particles within its search radius R_i = 2 L_i (1 + 0.1).  A warp
// takes SUB consecutive particles in key order (evol_params.length_group, 8 by default) and
// solves them one after the other, all 32 lanes on one particle.  For the SUB particles the warp
// first walks the tree once, popping up to 32 nodes at a time and opening those whose particle box
// comes within R_g = max R_i of the particles' bounding box; the leaves reached are listed in
// shared memory (where they do not fit, the walk is repeated for halves of the particles).
// A particle then tests the listed leaves against its own ball, and the particles of the leaves
// that pass, 32 at a time across leaves.  A particle whose radius grows beyond R_g, or whose
// group list overflowed, walks the tree on its own (same walk, from the particle's root).  The
// neighbours found are appended, as (distance, mass) pairs, to a shared-memory list.
// On that list the particle solves
//     F(L) = L^3 n(L) - eta^3 = 0,   n(L) = sum_j W(r_ij, L)  (self term included)
// by Newton steps in L^3 kept inside a bisection bracket, gathering again when 2L leaves the gathered
// radius.  F is non-decreasing in L, so the root is unique.  With w(u) = pi L^3 W the sums are
// dimensionless:
//     F = Sw/pi - eta^3,  F' = -Suw/(pi L),  Sw = sum w(u),  Suw = sum u w'(u).
// Each lane sums every 32nd entry of the list; the partial sums are combined across the warp.
// Outputs (mode 0, gas h):   rho = Smw/(pi h^3), Omega* = -Suw/(3 Sw),
//                           zeta = (3 Smw + Smuw)/(3 Sw)          (Sect. 3, Eq. drhodr)
// Outputs (mode 1, eps):     Upsilon = -Suw/(3 Sw),
//                           X = -(pi eps^2/(3 Sw)) sum_k m_k eps^2 dphi/deps   (Sect. 2.1)
// On request, either mode:   div v = 3 sum_j ((v_i - v_j).(r_i - r_j)/r_ij) w'(u) / (L Suw)
//                           (the discretised continuity equation of Sect. 2.1)
// Standard SPH scheme (Sect. 3, mode 0 on request): no root is solved.  Once a gathered ball holds
// at least N + 1 gas particles (the particle itself included), h = (r_(N) + r_(N+1)) / 4 from the
// N-th and (N+1)-th smallest distances, so that exactly N lie inside 2h; then one evaluation with
// Omega* = 1, zeta = 0 (the grad-h terms are dropped) and div v, curl v normalised by n alone.
#include <cuda_runtime.h>
#include <stdint.h>

#include "evol_internal.cuh"

namespace {

constexpr int LW_THREADS = 128;
constexpr int LW_WARPS = LW_THREADS / 32;
constexpr int HCAP = 96;              // leaves listed per pass of a particle's gather
constexpr int PCAP = 336;             // neighbour entries of the particle being solved
constexpr int SUB_DEFAULT = 8;        // particles sharing one group walk (evol_params.length_group = 0)
constexpr int GCAP = 240;             // leaves in a group walk's list
constexpr int MAX_ITERS = 60;
constexpr int MAX_WALKS = 24;
constexpr float SEARCH_MARGIN = 1.1f;
// Relative step below which one last evaluation is taken: a Newton step that small leaves an
// error of the order of its square (the iteration converges quadratically), far below FP32
// resolution; a bisection step must be smaller, as it halves the error only.
constexpr float NEWTON_TOL = 1e-4f;
constexpr float CONV_TOL = 1e-6f;

enum { ST_DONE = 0, ST_ACTIVE = 1, ST_LAST = 2 };

struct LenSmem {
    float4 gc[LW_WARPS][GCAP];        // group list: leaf box centre; w: first particle (int bits)
    float4 gh[LW_WARPS][GCAP];        // leaf box half widths; w: end of its particle range (int bits)
    int hb[LW_WARPS][HCAP + 1];       // listed leaves: exclusive prefix of their particle counts
    int hs[LW_WARPS][HCAP];           // and the first particle of each
    float2 nb[LW_WARPS][PCAP];        // neighbours of the particle solved: (distance, index bits), or
                                      // (distance, mass) when no velocity divergence is wanted
    unsigned lc[LW_WARPS][4];         // work counts of the warp's current item (kept by lane 0)
};

// The k-th smallest (k >= 1) of the cnt <= PCAP listed distances: the smallest x with at least k
// distances <= x, by bisection on the bit patterns (non-negative floats order like their bits).
__device__ __forceinline__ float kth_distance(const float2 *nb, int cnt, int k, int lane)
{
    unsigned lo = 0u, hi = 0x7f800000u;
    while (lo < hi) {
        const unsigned mid = lo + ((hi - lo) >> 1);
        int c = 0;
        for (int e = lane; e < cnt; e += 32) c += __float_as_uint(nb[e].x) <= mid ? 1 : 0;
        c = __reduce_add_sync(0xffffffffu, c);
        if (c >= k) hi = mid;
        else lo = mid + 1u;
    }
    return __uint_as_float(lo);
}

// Particles of the listed leaves against the particle at (px, py, pz), 32 at a time across
// leaves: those within R2 (gas only in mode 0) are appended to the neighbour list with their
// index (their mass when no velocity divergence is wanted, which spares the last evaluation its
// reads).  Returns the new count (entries beyond PCAP are counted but not stored).
template <int MODE, bool PER>
__device__ __forceinline__ int gather_listed(const evol_dev &d, const evol_kparams &kp, const int *hb, const int *hs,
                                             int nh, float2 *nb, int cnt, float px, float py, float pz, float R2,
                                             int lane)
{
    const unsigned ltmask = (1u << lane) - 1u;
    const float p0 = kp.plen[0], p1 = kp.plen[1], p2 = kp.plen[2];
    const int pm = PER ? kp.periodic_mask : 0;   // PER: periodic axes present
    const int total = hb[nh];
    constexpr int U = 1;              // chunks whose loads are issued together (more costs occupancy)
    // the listed leaf holding the chunk's first flattened index; leaves are never empty, so the
    // leaves starting inside a 32-index chunk are among the next 32, and each start offset is
    // distinct: one bit per offset (a warp OR) gives every lane its leaf by a population count
    int k0 = 0;
    for (int c0 = 0; c0 < total; c0 += 32 * U) {
        int jj[U];
#pragma unroll
        for (int h = 0; h < U; ++h) {
            const int x0 = c0 + 32 * h;
            const int kb = k0 + 1 + lane;
            const int p = kb < nh ? hb[kb] - x0 : 32;
            const unsigned starts = __reduce_or_sync(0xffffffffu, (p > 0 && p < 32) ? (1u << p) : 0u);
            const int x = x0 + lane;
            jj[h] = -1;
            if (x < total) {
                const int k = k0 + __popc(starts & ((2u << lane) - 1u));
                jj[h] = hs[k] + (x - hb[k]);
            }
            // the leaf holding x0 + 32
            k0 += __popc(starts);
            if (k0 + 1 < nh && hb[k0 + 1] == x0 + 32) ++k0;
        }
        float4 pj[U];
        bool gas[U];
#pragma unroll
        for (int h = 0; h < U; ++h) {
            pj[h] = jj[h] >= 0 ? d.pos[jj[h]] : make_float4(0.f, 0.f, 0.f, -1.f);
            gas[h] = MODE == 1 || (jj[h] >= 0 && d.orig[jj[h]] < kp.n_gas);
        }
#pragma unroll
        for (int h = 0; h < U; ++h) {
            const float dx = evol_wrap(px - pj[h].x, p0, pm & 1);
            const float dy = evol_wrap(py - pj[h].y, p1, pm & 2);
            const float dz = evol_wrap(pz - pj[h].z, p2, pm & 4);
            const float r2 = dx * dx + dy * dy + dz * dz;
            const bool in = jj[h] >= 0 && r2 < R2 && gas[h];
            const unsigned bal = __ballot_sync(0xffffffffu, in);
            if (in) {
                const int e = cnt + __popc(bal & ltmask);
                if (e < PCAP) nb[e] = make_float2(sqrtf(r2), kp.want_divv ? __int_as_float(jj[h]) : pj[h].w);
            }
            cnt += __popc(bal);
        }
    }
    return cnt;
}

// The particles within sqrt(R2) of (px, py, pz): a walk from `root` opening the nodes whose
// particle box comes within the radius; the leaves reached are listed (HCAP at a time) and their
// particles gathered into the neighbour list.  Returns the neighbour count, or -1 when the walk
// had to stop (corrupt tree or stack overflow; the error word is set).
template <int MODE, bool PER>
__device__ int gather_ball(const evol_dev &d, const evol_kparams &kp, int *hb, int *hs, float2 *nb, int lane,
                           int *stk, int stack_cap, long long pop_cap, int root, float px, float py, float pz,
                           float R2)
{
    const unsigned ltmask = (1u << lane) - 1u;
    const float p0 = kp.plen[0], p1 = kp.plen[1], p2 = kp.plen[2];
    const int pm = PER ? kp.periodic_mask : 0;   // PER: periodic axes present
    if (lane == 0) {
        stk[0] = root;
        hb[0] = 0;
    }
    int top = 1, nh = 0, cnt = 0;
    __syncwarp();
    long long pops = 0;
    while (top > 0) {
        if (++pops > pop_cap) {
            if (lane == 0) {
                evol_flag(d.err, EVOL_ETIMEOUT);
                atomicMax(&d.counters[7], 2ull);
            }
            return -1;
        }
        const int k = min(top, 32);
        top -= k;
        const int node = lane < k ? stk[top + lane] : -1;
        __syncwarp();
        bool open = false, leaf = false;
        int4 I = make_int4(0, 0, 0, 0);
        if (lane < k) {
            I = d.nI[node];
            const float4 B = d.nB[node];
            const float4 C = d.nC[node];
            if (MODE == 1 || B.w >= 0.f) {
                const float ex = fmaxf(fabsf(evol_wrap(B.x - px, p0, pm & 1)) - C.x, 0.f);
                const float ey = fmaxf(fabsf(evol_wrap(B.y - py, p1, pm & 2)) - C.y, 0.f);
                const float ez = fmaxf(fabsf(evol_wrap(B.z - pz, p2, pm & 4)) - C.z, 0.f);
                open = ex * ex + ey * ey + ez * ez < R2;
            }
            leaf = (I.x >> 8) & 1;
        }
        // leaves reached: list them (flush the list through the gather when it is full)
        const unsigned lv = __ballot_sync(0xffffffffu, open && leaf);
        const int nl = __popc(lv);
        if (nl) {
            if (nh + nl > HCAP) {
                __syncwarp();
                cnt = gather_listed<MODE, PER>(d, kp, hb, hs, nh, nb, cnt, px, py, pz, R2, lane);
                __syncwarp();
                nh = 0;
            }
            // exclusive prefix of the leaves' particle counts within this batch
            int c = (open && leaf) ? I.w - I.z : 0;
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const int base = nh == 0 ? 0 : hb[nh];
            __syncwarp();
            if (open && leaf) {
                const int e = nh + __popc(lv & ltmask);
                hs[e] = I.z;
                hb[e] = base + incl - c;
            }
            if (lane == 31) hb[nh + nl] = base + incl;
            nh += nl;
            __syncwarp();
        }
        // opened internal nodes: push their children
        const bool io = open && !leaf;
        int nch = 0;
        int ch[8];
        if (io) {
            const int4 K0 = d.nK0[node], K1 = d.nK1[node];
            ch[0] = K0.x; ch[1] = K0.y; ch[2] = K0.z; ch[3] = K0.w;
            ch[4] = K1.x; ch[5] = K1.y; ch[6] = K1.z; ch[7] = K1.w;
#pragma unroll
            for (int t = 0; t < 8; ++t) nch += ch[t] >= 0 ? 1 : 0;
        }
        int incl = nch;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        if (top + total > stack_cap) {
            if (lane == 0) evol_flag(d.err, EVOL_EOVERFLOW);
            return -1;
        }
        if (io) {
            const int pos = top + incl - nch;
#pragma unroll
            for (int t = 0; t < 8; ++t)
                if (t < nch) stk[pos + t] = ch[t];
        }
        top += total;
        __syncwarp();
    }
    if (nh) cnt = gather_listed<MODE, PER>(d, kp, hb, hs, nh, nb, cnt, px, py, pz, R2, lane);
    __syncwarp();
    return cnt;
}

// Group walk: the leaves whose particle box comes within sqrt(R2) of the box (c, hw) (gas
// leaves only in mode 0), from one root per system present among the `seed` lanes.  The
// leaves go to the group list; returns their number, GCAP + 1 when they do not fit, or -1 when
// the walk had to stop (corrupt tree or stack overflow; the error word is set).
template <int MODE, bool PER>
__device__ int collect_leaves(const evol_dev &d, const evol_kparams &kp, float4 *gc, float4 *gh, int lane,
                              int *stk, int stack_cap, long long pop_cap, float cx, float cy, float cz, float hx,
                              float hy, float hz, float R2, int myroot, bool seed)
{
    const unsigned ltmask = (1u << lane) - 1u;
    const float p0 = kp.plen[0], p1 = kp.plen[1], p2 = kp.plen[2];
    const int pm = PER ? kp.periodic_mask : 0;   // PER: periodic axes present
    int top = 0;
    {
        const unsigned peers = __match_any_sync(0xffffffffu, seed ? myroot : -1);
        const bool leader = seed && (__ffs(peers) - 1) == lane;
        const unsigned leaders = __ballot_sync(0xffffffffu, leader);
        if (leader) stk[__popc(leaders & ltmask)] = myroot;
        top = __popc(leaders);
    }
    __syncwarp();
    int count = 0;
    long long pops = 0;
    while (top > 0) {
        if (++pops > pop_cap) {
            if (lane == 0) {
                evol_flag(d.err, EVOL_ETIMEOUT);
                atomicMax(&d.counters[7], 2ull);
            }
            return -1;
        }
        const int k = min(top, 32);
        top -= k;
        const int node = lane < k ? stk[top + lane] : -1;
        __syncwarp();
        bool open = false, leaf = false;
        int4 I = make_int4(0, 0, 0, 0);
        float4 B = make_float4(0.f, 0.f, 0.f, 0.f), C = B;
        if (lane < k) {
            I = d.nI[node];
            B = d.nB[node];
            C = d.nC[node];
            if (MODE == 1 || B.w >= 0.f) {
                const float ex = fmaxf(fabsf(evol_wrap(B.x - cx, p0, pm & 1)) - (C.x + hx), 0.f);
                const float ey = fmaxf(fabsf(evol_wrap(B.y - cy, p1, pm & 2)) - (C.y + hy), 0.f);
                const float ez = fmaxf(fabsf(evol_wrap(B.z - cz, p2, pm & 4)) - (C.z + hz), 0.f);
                open = ex * ex + ey * ey + ez * ez < R2;
            }
            leaf = (I.x >> 8) & 1;
        }
        const unsigned lv = __ballot_sync(0xffffffffu, open && leaf);
        if (open && leaf) {
            const int e = count + __popc(lv & ltmask);
            if (e < GCAP) {
                gc[e] = make_float4(B.x, B.y, B.z, __int_as_float(I.z));
                gh[e] = make_float4(C.x, C.y, C.z, __int_as_float(I.w));
            }
        }
        count += __popc(lv);
        if (count > GCAP) return GCAP + 1;
        // opened internal nodes: push their children
        const bool io = open && !leaf;
        int nch = 0;
        int ch[8];
        if (io) {
            const int4 K0 = d.nK0[node], K1 = d.nK1[node];
            ch[0] = K0.x; ch[1] = K0.y; ch[2] = K0.z; ch[3] = K0.w;
            ch[4] = K1.x; ch[5] = K1.y; ch[6] = K1.z; ch[7] = K1.w;
#pragma unroll
            for (int t = 0; t < 8; ++t) nch += ch[t] >= 0 ? 1 : 0;
        }
        int incl = nch;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        if (top + total > stack_cap) {
            if (lane == 0) evol_flag(d.err, EVOL_EOVERFLOW);
            return -1;
        }
        if (io) {
            const int pos = top + incl - nch;
#pragma unroll
            for (int t = 0; t < 8; ++t)
                if (t < nch) stk[pos + t] = ch[t];
        }
        top += total;
        __syncwarp();
    }
    return count;
}

// A particle's gather from its group list: the listed leaves of its own system (particle range
// inside [sbeg, send)) whose box comes within sqrt(R2) of (px, py, pz), then their particles.
template <int MODE, bool PER>
__device__ int gather_from_list(const evol_dev &d, const evol_kparams &kp, const float4 *gc, const float4 *gh,
                                int nleaf, int *hb, int *hs, float2 *nb, int lane, float px, float py,
                                float pz, float R2, int sbeg, int send)
{
    const unsigned ltmask = (1u << lane) - 1u;
    const float p0 = kp.plen[0], p1 = kp.plen[1], p2 = kp.plen[2];
    const int pm = PER ? kp.periodic_mask : 0;   // PER: periodic axes present
    int cnt = 0, nh = 0;
    for (int base = 0; base < nleaf; base += 32) {
        const int l = base + lane;
        bool hit = false;
        int2 r = make_int2(0, 0);
        if (l < nleaf) {
            const float4 B = gc[l], C = gh[l];
            r = make_int2(__float_as_int(B.w), __float_as_int(C.w));
            const float ex = fmaxf(fabsf(evol_wrap(B.x - px, p0, pm & 1)) - C.x, 0.f);
            const float ey = fmaxf(fabsf(evol_wrap(B.y - py, p1, pm & 2)) - C.y, 0.f);
            const float ez = fmaxf(fabsf(evol_wrap(B.z - pz, p2, pm & 4)) - C.z, 0.f);
            hit = r.x >= sbeg && r.x < send && ex * ex + ey * ey + ez * ez < R2;
        }
        const unsigned hm = __ballot_sync(0xffffffffu, hit);
        const int nl = __popc(hm);
        if (nl) {
            if (nh + nl > HCAP) {
                __syncwarp();
                cnt = gather_listed<MODE, PER>(d, kp, hb, hs, nh, nb, cnt, px, py, pz, R2, lane);
                __syncwarp();
                nh = 0;
            }
            const int c = hit ? r.y - r.x : 0;
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const int base_cnt = nh == 0 ? 0 : hb[nh];
            __syncwarp();
            if (hit) {
                const int e = nh + __popc(hm & ltmask);
                hs[e] = r.x;
                hb[e] = base_cnt + incl - c;
            }
            if (lane == 31) hb[nh + nl] = base_cnt + incl;
            nh += nl;
            __syncwarp();
        }
    }
    if (nh) cnt = gather_listed<MODE, PER>(d, kp, hb, hs, nh, nb, cnt, px, py, pz, R2, lane);
    __syncwarp();
    return cnt;
}

// Variants: STD the standard scheme (mode 0), ACT the active list of individual time steps, CURL
// |curl v| in the last evaluation (mode 0), PER periodic axes; each a template parameter, so that
// the default solve's code carries none of them.  Five blocks per SM (at most 102 registers); the
// curl variants, which need more registers, four.
template <int MODE, bool STD, bool ACT, bool CURL, bool PER>
__global__ void __launch_bounds__(LW_THREADS, CURL ? 4 : 5) k_lengths(evol_dev d, evol_kparams kp, unsigned long long *queue)
{
    __shared__ LenSmem sm;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int wslot = blockIdx.x * LW_WARPS + w;
    // the warp's stack: node ids, two per int2 slot of the shared traversal-stack buffer
    int *stk = reinterpret_cast<int *>(d.wstack + (size_t)wslot * kp.stack_stride);
    const int stack_cap = 2 * kp.stack_cap;
    const int n = kp.n;
    // items of SUB consecutive entries of the particle list (individual time steps: the active list)
    const int SUB = kp.lsub;
    const int nlist = ACT ? d.acts[n] : n;
    const int ngroups = (nlist + SUB - 1) / SUB;   // the queue hands out SUB particles at a time
    const float eta = MODE == 0 ? kp.eta_h : kp.eta_e;
    const float eta3 = eta * eta * eta;
    const float inv_pi = 1.f / EVOL_PI_F;
    const int nn = *d.nnodes;
    const long long pop_cap = 2ll * (long long)nn + 64;
    float2 *nb = sm.nb[w];

    for (;;) {
        int g = 0;
        if (lane == 0) g = (int)atomicAdd(queue, 1ull);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= ngroups) break;
        const int e = g * SUB + lane;                 // lanes 0 .. SUB-1 hold the particles
        const bool valid = lane < SUB && e < nlist;
        const int s = ACT ? (valid ? d.act[e] : 0) : e;
        const float4 pi4 = valid ? d.pos[s] : make_float4(0.f, 0.f, 0.f, 0.f);
        const bool gas_i = valid && d.orig[s] < kp.n_gas;
        const bool act = MODE == 0 ? gas_i : valid;
        const unsigned todo0 = __ballot_sync(0xffffffffu, act);
        if (!todo0) continue;
        const int sys = valid ? d.sys_sorted[s] : 0;
        const float side = valid ? d.fcube[4 * sys + 3] : 1.f;     // the system's root cube
        const int root = act ? d.sys_root[sys] : -1;
        // the system's particles in key order: [sbeg, send)
        const int sbeg = act ? d.nbeg[root] : 0, send = act ? d.nend[root] : 0;
        float L0 = 0.f;
        if (act) {
            L0 = MODE == 0 ? d.len_h[s] : d.len_eps[s];
            if (!(L0 > 0.f) || !(L0 < 1e30f)) L0 = side / cbrtf((float)n);
        }
        int iters_total = 0;
        // gathers from the group list [0], by the particle's own walk [1], list overflows [2],
        // group-list overflows [3]
        unsigned *lc = sm.lc[w];
        if (lane < 4) lc[lane] = 0u;
        __syncwarp();
        bool broken = false;

        // one group walk for the SUB particles; where their leaves do not fit one list, walks for
        // the first half of them and then for the rest
        unsigned pending = todo0, subm = todo0;
        while (pending && !broken) {
          // the walk's particles: their box and largest search radius
          const bool insub = (subm >> lane) & 1u;
          float gx0 = insub ? pi4.x : INFINITY, gy0 = insub ? pi4.y : INFINITY, gz0 = insub ? pi4.z : INFINITY;
          float gx1 = insub ? pi4.x : -INFINITY, gy1 = insub ? pi4.y : -INFINITY, gz1 = insub ? pi4.z : -INFINITY;
          float Rg = insub ? 2.f * L0 * SEARCH_MARGIN : 0.f;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
              gx0 = fminf(gx0, __shfl_xor_sync(0xffffffffu, gx0, o));
              gy0 = fminf(gy0, __shfl_xor_sync(0xffffffffu, gy0, o));
              gz0 = fminf(gz0, __shfl_xor_sync(0xffffffffu, gz0, o));
              gx1 = fmaxf(gx1, __shfl_xor_sync(0xffffffffu, gx1, o));
              gy1 = fmaxf(gy1, __shfl_xor_sync(0xffffffffu, gy1, o));
              gz1 = fmaxf(gz1, __shfl_xor_sync(0xffffffffu, gz1, o));
              Rg = fmaxf(Rg, __shfl_xor_sync(0xffffffffu, Rg, o));
          }
          const int nleaf = collect_leaves<MODE, PER>(d, kp, sm.gc[w], sm.gh[w], lane, stk, stack_cap, pop_cap,
                                                 0.5f * (gx0 + gx1), 0.5f * (gy0 + gy1), 0.5f * (gz0 + gz1),
                                                 0.5f * (gx1 - gx0), 0.5f * (gy1 - gy0), 0.5f * (gz1 - gz0), Rg * Rg,
                                                 root, insub);
          if (nleaf < 0) {
              broken = true;
              break;
          }
          const bool glist = nleaf <= GCAP;
          if (lane == 0 && !glist) ++lc[3];
          if (!glist && __popc(subm) > 1) {
              unsigned upper = subm;                  // subm less its lowest popc/2 particles
              for (int q = __popc(subm) / 2; q > 0; --q) upper &= upper - 1u;
              subm &= ~upper;
              continue;
          }
          unsigned todo = subm;
          while (todo && !broken) {
            const int t = __ffs(todo) - 1;
            todo &= todo - 1u;
            const float px = __shfl_sync(0xffffffffu, pi4.x, t);
            const float py = __shfl_sync(0xffffffffu, pi4.y, t);
            const float pz = __shfl_sync(0xffffffffu, pi4.z, t);
            const float sd = __shfl_sync(0xffffffffu, side, t);
            const int rt = __shfl_sync(0xffffffffu, root, t);
            const int sb = __shfl_sync(0xffffffffu, sbeg, t);
            const int se = __shfl_sync(0xffffffffu, send, t);
            float L = __shfl_sync(0xffffffffu, L0, t);
            // every lane holds the same solver state for particle t
            float lo = 0.f, hi = INFINITY, Rc = 0.f;
            // after a neighbour-list overflow at search radius Rlim no length with 2 L >= Rlim can
            // be evaluated: the bracket's upper end is kept below Rlim / 2 and every later gather
            // radius below Rlim
            float Rlim = INFINITY;
            int status = ST_ACTIVE;
            bool stale = true;
            int cnt = 0, iters = 0, walks = 0;
            // a particle whose length cannot be found still gets every output written: its length
            // as reached, NaN for the quantities derived from the (missing) root
            auto give_up = [&](int code) {
                if (lane == 0) evol_flag(d.err, code);
                if (lane == t) {
                    const int si = ACT ? s : g * SUB + t;   // lane t holds particle t
                    const float qnan = __int_as_float(0x7fc00000);
                    if (MODE == 0) {
                        d.len_h[si] = L;
                        d.nh[si] = qnan; d.rho[si] = qnan; d.omega[si] = qnan; d.zeta[si] = qnan;
                    } else {
                        d.len_eps[si] = L;
                        d.neps[si] = qnan; d.ups[si] = qnan; d.X[si] = qnan;
                    }
                }
                status = ST_DONE;
            };
            while (status != ST_DONE) {
                if (stale) {
                    if (walks >= MAX_WALKS) {
                        give_up(EVOL_ENOCONV);
                        break;
                    }
                    ++walks;
                    // gather radius: 2 L (1 + margin), and strictly between 2 L and Rlim
                    Rc = fminf(2.f * L * SEARCH_MARGIN, L + 0.5f * Rlim);
                    const float R2 = Rc * Rc;
                    cnt = 0;
                    __syncwarp();
                    if (glist && Rc <= Rg) {
                        if (lane == 0) ++lc[0];
                        cnt = gather_from_list<MODE, PER>(d, kp, sm.gc[w], sm.gh[w], nleaf, sm.hb[w], sm.hs[w], nb,
                                                     lane, px, py, pz, R2, sb, se);
                    } else {
                        if (lane == 0) ++lc[1];
                        cnt = gather_ball<MODE, PER>(d, kp, sm.hb[w], sm.hs[w], nb, lane, stk, stack_cap, pop_cap, rt, px,
                                                py, pz, R2);
                    }
                    if (cnt < 0) {
                        broken = true;
                        break;
                    }
                    __syncwarp();
                    stale = false;
                    if (cnt > PCAP) {
                        // more neighbours than the list holds: the radius is too large; shrink, gather again
                        if (lane == 0) ++lc[2];
                        Rlim = fminf(Rlim, Rc);
                        hi = fminf(hi, 0.5f * Rlim * (1.f - 1e-6f));
                        float Ln = 0.75f * L;
                        if (Ln <= lo) Ln = 0.5f * (lo + fminf(L, hi));
                        if (!(Ln > lo && Ln < hi)) {          // nothing left to evaluate
                            give_up(EVOL_EOVERFLOW);
                            break;
                        }
                        L = Ln;
                        stale = true;
                        status = ST_ACTIVE;                    // a converged length is solved again
                        continue;
                    }
                }
                if (MODE == 0 && STD && status == ST_ACTIVE) {
                    // standard scheme: widen the ball until it holds N + 1 gas particles, then h
                    // from the N-th and (N+1)-th distances (every particle closer than the
                    // (N+1)-th is in the list: the list holds the whole ball)
                    if (cnt < kp.nstd + 1) {
                        if (Rc > 8.f * sd) {                  // fewer gas particles than N + 1
                            give_up(EVOL_ENOCONV);
                            break;
                        }
                        L = Rc;
                        stale = true;
                        continue;
                    }
                    const float rN = kth_distance(nb, cnt, kp.nstd, lane);
                    const float rN1 = kth_distance(nb, cnt, kp.nstd + 1, lane);
                    L = 0.25f * (rN + rN1);
                    status = ST_LAST;
                }
                // Sums over the list (lane l takes entries l, l + 32, ...), combined across the warp.
                // A Newton iteration needs Sw and Suw; the last evaluation also needs the
                // mass-weighted sums of the outputs.
                const bool last = status == ST_LAST;
                float Sw = 0.f, Suw = 0.f, S3 = 0.f, S4 = 0.f, S5 = 0.f;
                float S6x = 0.f, S6y = 0.f, S6z = 0.f;       // curl sums (h solve, on request)
                const float Linv = 1.f / L;
                if (!last) {
                    for (int e = lane; e < cnt; e += 32) {
                        const float u = nb[e].x * Linv;
                        const float aa = fmaxf(2.f - u, 0.f), bb = fmaxf(1.f - u, 0.f);
                        const float a2 = aa * aa, b2 = bb * bb;
                        Sw += 0.25f * a2 * aa - b2 * bb;                    // w(u)
                        Suw += u * (-0.75f * a2 + 3.f * b2);                // u w'(u)
                    }
                } else {
                    // the neighbours' masses are in the list, or (for the continuity equation) read
                    // with their positions and velocities from the sorted particle state
                    const int st = ACT ? __shfl_sync(0xffffffffu, s, t) : g * SUB + t;
                    const float4 vi = kp.want_divv ? d.vel[st] : make_float4(0.f, 0.f, 0.f, 0.f);
                    for (int e = lane; e < cnt; e += 32) {
                        const float2 rj = nb[e];
                        const int j = kp.want_divv ? __float_as_int(rj.y) : 0;
                        const float4 pj = kp.want_divv ? d.pos[j] : make_float4(0.f, 0.f, 0.f, rj.y);
                        const float u = rj.x * Linv;
                        float wv, dw;
                        evol_w_dw(u, wv, dw);      // zero for u >= 2
                        Sw += wv;
                        Suw += u * dw;
                        if (MODE == 0) {
                            S3 += pj.w * wv;                               // Smw
                            S4 += pj.w * u * dw;                           // Smuw
                        } else {
                            S3 += pj.w * evol_dphideps(u);                 // sum m eps^2 dphi/deps
                        }
                        if (kp.want_divv && rj.x > 0.f) {
                            // (v_i - v_j).(r_i - r_j) / r  w'(u)  (Sect. 2.1, continuity equation)
                            const float4 vj = d.vel[j];
                            const int pmk = PER ? kp.periodic_mask : 0;
                            const float dx = evol_wrap(px - pj.x, kp.plen[0], pmk & 1);
                            const float dy = evol_wrap(py - pj.y, kp.plen[1], pmk & 2);
                            const float dz = evol_wrap(pz - pj.z, kp.plen[2], pmk & 4);
                            S5 += ((vi.x - vj.x) * dx + (vi.y - vj.y) * dy + (vi.z - vj.z) * dz) / rj.x * dw;
                            if (MODE == 0 && CURL) {
                                // (v_i - v_j) x (r_i - r_j) / r  w'(u)
                                const float ux = vi.x - vj.x, uy = vi.y - vj.y, uz = vi.z - vj.z;
                                const float q = dw / rj.x;
                                S6x += (uy * dz - uz * dy) * q;
                                S6y += (uz * dx - ux * dz) * q;
                                S6z += (ux * dy - uy * dx) * q;
                            }
                        }
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    Sw += __shfl_xor_sync(0xffffffffu, Sw, o);
                    Suw += __shfl_xor_sync(0xffffffffu, Suw, o);
                    if (last) {
                        S3 += __shfl_xor_sync(0xffffffffu, S3, o);
                        if (MODE == 0) S4 += __shfl_xor_sync(0xffffffffu, S4, o);
                        if (kp.want_divv) S5 += __shfl_xor_sync(0xffffffffu, S5, o);
                        if (MODE == 0 && CURL) {
                            S6x += __shfl_xor_sync(0xffffffffu, S6x, o);
                            S6y += __shfl_xor_sync(0xffffffffu, S6y, o);
                            S6z += __shfl_xor_sync(0xffffffffu, S6z, o);
                        }
                    }
                }
                // identical on every lane up to the order of the additions; take lane 0's values
                Sw = __shfl_sync(0xffffffffu, Sw, 0);
                Suw = __shfl_sync(0xffffffffu, Suw, 0);
                if (last) {
                    S3 = __shfl_sync(0xffffffffu, S3, 0);
                    if (MODE == 0) S4 = __shfl_sync(0xffffffffu, S4, 0);
                    if (kp.want_divv) S5 = __shfl_sync(0xffffffffu, S5, 0);
                    if (MODE == 0 && CURL) {
                        S6x = __shfl_sync(0xffffffffu, S6x, 0);
                        S6y = __shfl_sync(0xffffffffu, S6y, 0);
                        S6z = __shfl_sync(0xffffffffu, S6z, 0);
                    }
                }
                const float Smw = S3, Smuw = S4;
                if (status == ST_LAST) {
                    if (lane == t) {
                        const int si = ACT ? s : g * SUB + t;   // lane t holds particle t
                        const float nsum = Sw * inv_pi * Linv * Linv * Linv;
                        if (MODE == 0) {
                            d.len_h[si] = L;
                            d.nh[si] = nsum;
                            d.rho[si] = Smw * inv_pi * Linv * Linv * Linv;
                            d.omega[si] = STD ? 1.f : -Suw / (3.f * Sw);
                            d.zeta[si] = STD ? 0.f : (3.f * Smw + Smuw) / (3.f * Sw);
                        } else {
                            d.len_eps[si] = L;
                            d.neps[si] = nsum;
                            d.ups[si] = -Suw / (3.f * Sw);
                            d.X[si] = -EVOL_PI_F * L * L * Smw / (3.f * Sw);
                        }
                        // div v = -1/(n C) sum_j (v_i - v_j).grad_i W = 3 S5 / (L Suw), C = Upsilon
                        // or Omega* = -Suw/(3 Sw), n = Sw/(pi L^3), grad W = r_ij/r w'(u)/(pi L^4)
                        // (the standard scheme takes C = 1: div v = -S5 / (L Sw))
                        const bool stdc = MODE == 0 && STD;
                        if (kp.want_divv)
                            (MODE == 0 ? d.divv_h : d.divv_e)[si] = stdc ? -S5 / (L * Sw) : 3.f * S5 / (L * Suw);
                        // |curl v| = |1/(n C) sum_j (v_i - v_j) x grad_i W| = 3 |S6| / (L |Suw|)
                        if (MODE == 0 && CURL) {
                            const float s6 = sqrtf(S6x * S6x + S6y * S6y + S6z * S6z);
                            d.curlv_h[si] = stdc ? s6 / (L * Sw) : 3.f * s6 / (L * fabsf(Suw));
                        }
                    }
                    status = ST_DONE;
                } else {
                    ++iters;
                    const float F = Sw * inv_pi - eta3;
                    if (F < 0.f) lo = L;
                    if (F > 0.f) hi = L;
                    float Ln;
                    bool newton = false;
                    if (F == 0.f) {
                        Ln = L;
                    } else {
                        // Newton step in y = L^3, on which F = n y - eta^3 depends almost linearly
                        // (n varies slowly with L): dF/dy = F'/(3 L^2) with F' = -Suw/(pi L), so
                        // y' = y (1 + 3 pi F / Suw); bisection where it leaves the bracket
                        const float q = 1.f + 3.f * EVOL_PI_F * F / Suw;
                        newton = Suw < 0.f && q > 0.f;
                        Ln = newton ? L * cbrtf(q) : (hi < INFINITY ? 0.5f * (lo + hi) : 2.f * L);
                        if (newton && fabsf(Ln - L) <= NEWTON_TOL * L) {
                            // converged: a step this small goes towards the root (F' > 0), and one
                            // below FP32 resolution leaves L on the bracket's end
                            if (Ln < lo || Ln > hi) Ln = L;
                        } else {
                            // below the root with no upper bracket yet, F' counts only the few
                            // neighbours inside the kernel and the step can overshoot by orders of
                            // magnitude: grow by at most a factor 2 until the root is bracketed
                            if (hi == INFINITY && Ln > 2.f * L) {
                                Ln = 2.f * L;
                                newton = false;
                            }
                            if (!(Ln > lo && Ln < hi)) {
                                Ln = hi < INFINITY ? 0.5f * (lo + hi) : 2.f * L;
                                newton = false;
                            }
                        }
                    }
                    const bool conv = fabsf(Ln - L) <= (newton ? NEWTON_TOL : CONV_TOL) * L ||
                                      (hi < INFINITY && hi - lo <= 1e-7f * hi);
                    L = Ln;
                    if (conv) status = ST_LAST;
                    if (iters >= MAX_ITERS) {
                        if (lane == 0) evol_flag(d.err, EVOL_ENOCONV);
                        status = ST_LAST;
                    }
                    if (2.f * L >= Rc) stale = true;
                    if (L > 4.f * sd)                 // no root: fewer neighbours than required
                        give_up(EVOL_ENOCONV);
                    else if (stale && 2.f * L >= Rlim)   // the next gather would overflow again
                        give_up(EVOL_EOVERFLOW);
                }
            }
            iters_total += iters;
          }
          pending &= ~subm;
          subm = pending;
        }
        if (lane == 0) {
            atomicAdd(&d.counters[3], (unsigned long long)iters_total);
            unsigned long long *c4 = d.counters + (MODE == 1 ? 16 : 20);
            for (int q = 0; q < 4; ++q) atomicAdd(c4 + q, (unsigned long long)lc[q]);
            atomicAdd(&d.counters[MODE == 1 ? 24 : 25], (unsigned long long)iters_total);
        }
        if (broken) break;
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
    kp.active = c->bins_active;
    kp.want_curl = mode == 0 && evol_needs_curl(prm);
    kp.standard = mode == 0 && prm->sph_scheme == EVOL_SPH_STANDARD;
    kp.nstd = (int)lrintf(prm->n_nei_sph);
    kp.want_divv = c->want_divv || kp.want_curl;
    kp.lsub = prm->length_group > 0 ? prm->length_group : SUB_DEFAULT;
    kp.stack_cap = (int)c->wstack_lim;
    kp.stack_stride = (int)c->wstack_cap;
    unsigned long long *q = c->d.counters + (mode == 0 ? 5 : 6);
    cudaMemsetAsync(q, 0, sizeof(unsigned long long), c->stream);
    int blocks = (int)(c->cand_slots / LW_WARPS);
    // variant = standard scheme | active list << 1 | curl << 2 | periodic << 3 (mode 0);
    // 16 + active list | periodic << 1 (mode 1)
    const int per = prm->periodic_mask ? 1 : 0;
    const int var = mode == 0 ? ((kp.standard ? 1 : 0) | (kp.active ? 2 : 0) | (kp.want_curl ? 4 : 0) | (per << 3))
                              : 16 + ((kp.active ? 1 : 0) | (per << 1));
#define EVOL_LEN(M, S, A, C, P) \
    k_lengths<M, S, A, C, P><<<blocks, LW_THREADS, 0, c->stream>>>(c->d, kp, q); break
    switch (var) {
    case 0: EVOL_LEN(0, false, false, false, false);
    case 1: EVOL_LEN(0, true, false, false, false);
    case 2: EVOL_LEN(0, false, true, false, false);
    case 3: EVOL_LEN(0, true, true, false, false);
    case 4: EVOL_LEN(0, false, false, true, false);
    case 5: EVOL_LEN(0, true, false, true, false);
    case 6: EVOL_LEN(0, false, true, true, false);
    case 7: EVOL_LEN(0, true, true, true, false);
    case 8: EVOL_LEN(0, false, false, false, true);
    case 9: EVOL_LEN(0, true, false, false, true);
    case 10: EVOL_LEN(0, false, true, false, true);
    case 11: EVOL_LEN(0, true, true, false, true);
    case 12: EVOL_LEN(0, false, false, true, true);
    case 13: EVOL_LEN(0, true, false, true, true);
    case 14: EVOL_LEN(0, false, true, true, true);
    case 15: EVOL_LEN(0, true, true, true, true);
    case 16: EVOL_LEN(1, false, false, false, false);
    case 17: EVOL_LEN(1, false, true, false, false);
    case 18: EVOL_LEN(1, false, false, false, true);
    default: EVOL_LEN(1, false, true, false, true);
    }
#undef EVOL_LEN
    return evol_cuda_ok(cudaGetLastError());
}

int evol_lengths_warps_per_block() { return LW_WARPS; }
int evol_lengths_list_cap() { return PCAP; }
