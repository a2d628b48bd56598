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
#ifndef EVOL_WALK_MINB
#define EVOL_WALK_MINB 5           // resident blocks per SM the production walk is compiled for
#endif
#ifndef EVOL_FAR_UNROLL
#define EVOL_FAR_UNROLL 4          // entry pairs per trip of the far-node loop
#endif
constexpr int WK_WARPS = WK_THREADS / 32;
constexpr int FARCAP = 64;
constexpr int NEARCAP = 64;
constexpr int SG_GROUPS = EVOL_SG_GROUPS;   // groups per super-group (see k_super)

constexpr float TAU = 1e-5f;      // safety margin of the group-level bounds

struct WalkSmem {
    float4 bA[WK_WARPS][32];      // popped batch: com, ropen^2
    float4 bB[WK_WARPS][32];      // box centre, 2 hmax
    float4 bC[WK_WARPS][32];      // box half widths, 2 epsmax
    int far_id[WK_WARPS][FARCAP];
    unsigned far_mask[WK_WARPS][FARCAP];
    // far nodes in pairs for the packed two-wide evaluation: for the pair of entries (2p, 2p + 1),
    // component c of entry 2p + k sits at fpair[p][2c + k], c = x, y, z, -M, Qxx, Qyy, Qzz, Qxy,
    // Qxz, Qyz (centre of mass, mass and traceless quadrupole)
    __align__(16) float fpair[WK_WARPS][FARCAP / 2][20];
    int near_j[WK_WARPS][NEARCAP];
    unsigned near_mask[WK_WARPS][NEARCAP];       // lanes that opened the entry's leaf, less its own lane
    // near entries in pairs for the two-wide first pass: component c of entry 2q + k sits at
    // npair[q][2c + k], c = x, y, z, m, E = (2 eps)^2, H = (2 h)^2 (-1: not gas)
    __align__(16) float npair[WK_WARPS][NEARCAP / 2][12];
    float4 ng[WK_WARPS][NEARCAP];
    float4 nh[WK_WARPS][NEARCAP];
    float4 ns[WK_WARPS][NEARCAP];
    float4 gbox[WK_WARPS][3];     // group bounds: centre, 0 | half widths, 0 | emax, emin, hmax, hmin
    unsigned wc[WK_WARPS][8];     // per-group work counts kept by lane 0 (see the end of k_walk)
    float mum[WK_WARPS][32];      // largest |mu_ij| of each lane's particle (viscosity)
    int gs[WK_WARPS][32];         // active list: the sorted position of each lane's particle
    unsigned gself[WK_WARPS][32]; // active list: the lane whose particle is a leaf chunk's entry
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

// Position of the k-th (0-based) set bit of m (k < popc(m)), by halving with population counts.
__device__ __forceinline__ int nth_bit(unsigned m, int k)
{
    int p = 0;
#pragma unroll
    for (int h = 16; h > 0; h >>= 1) {
        const int c = __popc(m & ((1u << h) - 1u));
        if (k >= c) {
            k -= c;
            m >>= h;
            p += h;
        }
    }
    return p;
}

// Packed two-wide FP32 arithmetic (add/mul/fma .rn.f32x2): one instruction computes the same
// operation, rounded the same way, on two independent FP32 values held in a 64-bit register.
// The far-node loop evaluates two accepted nodes per lane with it, which halves the issue slots
// its arithmetic needs.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk2(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float lo2(f32x2 v)
{
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    (void)b;
    return a;
}
__device__ __forceinline__ float hi2(f32x2 v)
{
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    (void)a;
    return b;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Periodic gravity: trilinear interpolation in the Ewald table (Sect. 4.3).  f is odd in its own
// coordinate and even in the others, g is even, so the table holds the octant [0, L/2]^3 only; the
// four components are interpolated as two packed pairs, (f_x, f_y) and (f_z, g), and the caller
// applies the octant signs.  sc = 2 N / L.
struct Ew2 {
    f32x2 xy, zw;
};
__device__ __forceinline__ Ew2 ewald_lookup2(const float4 *__restrict__ tab, float dx, float dy, float dz, float sc)
{
    const int M = EVOL_EWALD_M;
    const float nm1 = (float)(EVOL_EWALD_N - 1);
    const float ux = fabsf(dx) * sc, uy = fabsf(dy) * sc, uz = fabsf(dz) * sc;
    // the cell, clamped in float before the conversion (fminf returns nm1 for a NaN offset), so that
    // every index stays inside the table; truncation is the floor for the non-negative values
    const int i = __float2int_rz(fminf(ux, nm1)), j = __float2int_rz(fminf(uy, nm1)), k = __float2int_rz(fminf(uz, nm1));
    const float tx = ux - (float)i, ty = uy - (float)j, tz = uz - (float)k;
    const ulonglong2 *b = reinterpret_cast<const ulonglong2 *>(tab + ((i * M + j) * M + k));
    const ulonglong2 c000 = b[0], c001 = b[1], c010 = b[M], c011 = b[M + 1];
    const ulonglong2 c100 = b[M * M], c101 = b[M * M + 1], c110 = b[M * M + M], c111 = b[M * M + M + 1];
    const f32x2 TZ = pk2(tz, tz), TY = pk2(ty, ty), TX = pk2(tx, tx);
    auto L = [](f32x2 a, f32x2 c, f32x2 t) { return fma2(t, sub2(c, a), a); };
    const f32x2 a0 = L(c000.x, c001.x, TZ), b0 = L(c000.y, c001.y, TZ);
    const f32x2 a1 = L(c010.x, c011.x, TZ), b1 = L(c010.y, c011.y, TZ);
    const f32x2 a2 = L(c100.x, c101.x, TZ), b2 = L(c100.y, c101.y, TZ);
    const f32x2 a3 = L(c110.x, c111.x, TZ), b3 = L(c110.y, c111.y, TZ);
    const f32x2 e0 = L(a0, a1, TY), g0 = L(b0, b1, TY), e1 = L(a2, a3, TY), g1 = L(b2, b3, TY);
    return Ew2{L(e0, e1, TX), L(g0, g1, TX)};
}


// Per-particle sums of one flush (a block of at most FARCAP far nodes or NEARCAP near entries).
struct Acc {
    float ax = 0.f, ay = 0.f, az = 0.f, pot = 0.f;      // gravity (without G)
    float hx = 0.f, hy = 0.f, hz = 0.f, du = 0.f;       // SPH
};

// Error-free sum of two floats (Knuth's TwoSum): s + e == a + b exactly, s = fl(a + b).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bp = s - a, ap = s - bp;
    e = (a - ap) + (b - bp);
}

// Mixed form: the gravity totals (acceleration and potential, sums over thousands of far nodes and
// near particles) are compensated sums.  Each flush block's sum is added to the running FP32 total
// with TwoSum and the rounding error of that addition kept in a separate compensation term, so the
// totals carry the blocks' own FP32 rounding only (a few ulps of at most 64 terms), not that of
// thousands of successive additions.  The hydro sums (about N_nei pair terms, one or two flushes)
// gain nothing from compensation at this granularity and are summed as in the plain form.  The
// running totals are the plain form's registers (parked in shared memory while the pair loop sums
// a block in them); the compensation terms sit in shared memory (one per lane and component), which
// keeps the mixed walk at the plain walk's register count and residency.
template <bool MIXED>
struct MixSmem {
    // [0, 4): compensation terms of ax, ay, az, pot; [4, 8): the running totals, parked here while
    // the pair loop sums its flush block in their registers
    float c[WK_WARPS][8][32];
};
template <>
struct MixSmem<false> {
};

// Dissipation operands staged per near entry (alpha, Balsara f, u, alpha^u of the neighbour) and
// each lane's running v^sig maximum and Brookshaw sum: only the DISS variants hold them.
template <bool DISS>
struct DissSmem {
    float4 nd[WK_WARPS][NEARCAP];
    float vs[WK_WARPS][32];
    float lap[WK_WARPS][32];
};
template <>
struct DissSmem<false> {
};

// Check mode: each lane's SPH neighbour count and set hash, accumulated by whichever lane
// evaluates the pair (integer sums, so the order does not matter).
template <bool CHECK>
struct CheckSmem {
    int cs[WK_WARPS][32];
    unsigned long long hs[WK_WARPS][32];
    int norig[WK_WARPS][NEARCAP];                 // original index of each near entry
};
template <>
struct CheckSmem<false> {
};

// Register budgets, chosen so that no variant spills to local memory: the gravity + SPH walk (the
// production form, plain or mixed) and the SPH-only walk fit five blocks per SM (at most 102
// registers), the walks with the dissipation variants (DISS) and the plain gravity-only periodic
// (EWALD) walk four (128 registers), the other gravity-only, periodic and mixed DISS walks three;
// the check-mode variants one.
template <bool GRAV, bool SPH, bool MIXED, bool CHECK, bool DISS, bool EWALD>
__global__ void __launch_bounds__(WK_THREADS, CHECK ? 1 : (EWALD && !SPH && !MIXED) ? 4 : (EWALD || (GRAV && !SPH) || (MIXED && DISS)) ? 3 : DISS ? 4 : EVOL_WALK_MINB) k_walk(evol_dev d, evol_kparams kp, unsigned long long *queue)
{
    __shared__ WalkSmem sm;
    __shared__ DissSmem<DISS> ds;
    __shared__ CheckSmem<CHECK> cks;
    __shared__ MixSmem<MIXED> mx;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int n = kp.n;
    // individual time steps: groups of 32 consecutive entries of the active list
    const int nlist = kp.active ? d.acts[n] : n;
    const int ngroups = (nlist + 31) >> 5;
    // periodic axes: SPH alone, or gravity in a periodic cube (EWALD: nearest images plus the
    // tabulated correction of the replicas, Sect. 4.3); pmg: the periodic axes of the gravity tests
    const int pm = ((SPH && !GRAV) || EWALD) ? kp.periodic_mask : 0;
    const int pmg = EWALD ? kp.periodic_mask : 0;
    const float iL = EWALD ? 1.f / kp.ewald_L : 0.f;
    const float side0 = EWALD ? d.fcube[3] : 0.f;     // root cube side (periodic gravity: one system)
    const float plen0 = kp.plen[0], plen1 = kp.plen[1], plen2 = kp.plen[2];
    const float inv_pi = 1.f / EVOL_PI_F;

    for (;;) {
        int g = 0;
        if (lane == 0) g = (int)atomicAdd(queue, 1ull);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= ngroups) break;
        const int e = g * 32 + lane;
        const bool valid = e < nlist;
        const int s = kp.active ? (valid ? d.act[e] : 0) : e;
        const float4 pi = valid ? d.pos[s] : make_float4(0.f, 0.f, 0.f, 0.f);
        // the group's sorted positions, for the self test of the near list (active list only)
        if (kp.active) sm.gs[w][lane] = valid ? s : -1;
        // this lane's hydro operands (v, P/rho^2, c, rho, 1/h, zeta/Omega*) are read where they are
        // used, in the SPH pass, which keeps them out of the traversal's live registers
        const float4 g0 = valid ? d.grav[s] : make_float4(0.f, 0.f, 0.f, 0.f);
        const bool gas_i = SPH && valid && g0.z > 0.f;
        const bool active = valid && (GRAV || gas_i);
        const float ie_i = g0.x, two_eps_i = GRAV && active ? 2.f / g0.x : 0.f;
        const float two_h_i = gas_i ? 2.f * g0.z : 0.f;
        // squared near radii of the pair tests: softened gravity inside max(E_i, E_j), SPH inside
        // max(H_i, H_j) when both are gas (H = -1 marks a particle that is not)
        const float E_i = two_eps_i * two_eps_i;
        const float H_i = gas_i ? two_h_i * two_h_i : -1.f;

        Acc acc;
        unsigned long long hfar = 0, hnear = 0;
        int cfar = 0, cpp = 0;
        // interaction counts of this lane (one group's counts fit 32 bits)
        unsigned wfar = 0, wpp = 0, wsph = 0, wsoft = 0;
        // per-group counts kept by lane 0 in shared memory: lane slots issued (32 per entry or per
        // loop trip) by the far loop [0], pass 1 [1] and pass 2 [2] of the pair loop; nodes popped
        // [3], tested lane by lane [4]; leaves [5] and internal nodes [6] opened
        unsigned *wc = sm.wc[w];
        if (lane < 8) wc[lane] = 0u;
        if (SPH) sm.mum[w][lane] = 0.f;
        if constexpr (DISS) {
            ds.vs[w][lane] = 0.f;
            ds.lap[w][lane] = 0.f;
        }
        if constexpr (CHECK) {
            cks.cs[w][lane] = 0;
            cks.hs[w][lane] = 0ull;
        }
        if constexpr (MIXED) {
#pragma unroll
            for (int k = 0; k < 4; ++k) mx.c[w][k][lane] = 0.f;
        }
        __syncwarp();

        // adds a block sum b to gravity component k of this lane's total (compensated in the mixed
        // form)
        auto add_to = [&](float &total, int k, float b) {
            if constexpr (MIXED) {
                float t, e;
                two_sum(total, b, t, e);
                total = t;
                mx.c[w][k][lane] += e;
            } else {
                total += b;
            }
        };

        int nfar = 0, nnear = 0;

        auto flush_far = [&]() {
            __syncwarp();
            // pad to a whole trip of the loop with empty-mask entries (node 0 is always valid)
            constexpr int TRIP = 2 * EVOL_FAR_UNROLL;
            const int padded = (nfar + TRIP - 1) / TRIP * TRIP;
            if (lane < padded - nfar) {
                sm.far_id[w][nfar + lane] = 0;
                sm.far_mask[w][nfar + lane] = 0u;
            }
            __syncwarp();
            for (int l = lane; l < padded; l += 32) {
                const int id = sm.far_id[w][l];
                const float4 A = d.nA[id], Q0 = d.nQ0[id], Q1 = d.nQ1[id];
                float *f = sm.fpair[w][l >> 1] + (l & 1);
                f[0] = A.x; f[2] = A.y; f[4] = A.z; f[6] = -Q0.w;
                f[8] = Q0.x; f[10] = Q0.y; f[12] = Q0.z; f[14] = Q1.x; f[16] = Q1.y; f[18] = Q1.z;
                wfar += __popc(sm.far_mask[w][l]);     // interaction count (this lane's share)
            }
            if (lane == 0) wc[0] += 32u * (unsigned)padded;
            __syncwarp();
            // monopole + traceless quadrupole about the centre of mass, d = r_i - com:
            //   a += -M d/d^3 + Q d/d^5 - 5/2 (d.Q.d) d/d^7,  phi += -M/d - 1/2 (d.Q.d)/d^5
            // two entries per packed operation; lanes outside an entry's mask take 1/d = 0 for it,
            // so every term vanishes for them
            const f32x2 PX = pk2(pi.x, pi.x), PY = pk2(pi.y, pi.y), PZ = pk2(pi.z, pi.z);
            const f32x2 KM25 = pk2(-2.5f, -2.5f), KM05 = pk2(-0.5f, -0.5f);
            f32x2 fax = 0ull, fay = 0ull, faz = 0ull, fpot = 0ull;      // +0.0f in both halves
            f32x2 ewxy = 0ull, ewzw = 0ull;                             // Ewald corrections (x M)
            for (int e = 0; e < padded; e += TRIP) {
#pragma unroll
                for (int u = 0; u < EVOL_FAR_UNROLL; ++u) {
                    const int pp = (e >> 1) + u;
                    const uint2 mk = *reinterpret_cast<const uint2 *>(&sm.far_mask[w][2 * pp]);
                    const ulonglong2 *F = reinterpret_cast<const ulonglong2 *>(sm.fpair[w][pp]);
                    const ulonglong2 v0 = F[0], v1 = F[1], v2 = F[2], v3 = F[3], v4 = F[4];
                    // v0 = (x, y), v1 = (z, -M), v2 = (Qxx, Qyy), v3 = (Qzz, Qxy), v4 = (Qxz, Qyz)
                    f32x2 dx = sub2(PX, v0.x), dy = sub2(PY, v0.y), dz = sub2(PZ, v1.x);
                    if constexpr (EWALD) {
                        // nearest image of the centre of mass, and the node's replicas beyond it
                        // (monopole: its mass at the centre of mass)
                        dx = pk2(evol_wrap(lo2(dx), plen0, pmg & 1), evol_wrap(hi2(dx), plen0, pmg & 1));
                        dy = pk2(evol_wrap(lo2(dy), plen1, pmg & 2), evol_wrap(hi2(dy), plen1, pmg & 2));
                        dz = pk2(evol_wrap(lo2(dz), plen2, pmg & 4), evol_wrap(hi2(dz), plen2, pmg & 4));
                        if ((mk.x >> lane) & 1u) {
                            const float ex = lo2(dx), ey = lo2(dy), ez = lo2(dz);
                            const Ew2 c = ewald_lookup2(kp.ewald_tab, ex, ey, ez, kp.ewald_sc);
                            // octant signs folded into the mass: f_a odd in its own coordinate
                            const float Mn = -lo2(v1.y);
                            ewxy = fma2(pk2(ex < 0.f ? -Mn : Mn, ey < 0.f ? -Mn : Mn), c.xy, ewxy);
                            ewzw = fma2(pk2(ez < 0.f ? -Mn : Mn, Mn), c.zw, ewzw);
                        }
                        if ((mk.y >> lane) & 1u) {
                            const float ex = hi2(dx), ey = hi2(dy), ez = hi2(dz);
                            const Ew2 c = ewald_lookup2(kp.ewald_tab, ex, ey, ez, kp.ewald_sc);
                            const float Mn = -hi2(v1.y);
                            ewxy = fma2(pk2(ex < 0.f ? -Mn : Mn, ey < 0.f ? -Mn : Mn), c.xy, ewxy);
                            ewzw = fma2(pk2(ez < 0.f ? -Mn : Mn, Mn), c.zw, ewzw);
                        }
                    }
                    const f32x2 d2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
                    const float r0 = ((mk.x >> lane) & 1u) ? rsqrtf(lo2(d2)) : 0.f;
                    const float r1 = ((mk.y >> lane) & 1u) ? rsqrtf(hi2(d2)) : 0.f;
                    const f32x2 rinv = pk2(r0, r1);
                    const f32x2 rinv2 = mul2(rinv, rinv);
                    const f32x2 r3 = mul2(rinv, rinv2), r5 = mul2(r3, rinv2);
                    const f32x2 qx = fma2(v4.x, dz, fma2(v3.y, dy, mul2(v2.x, dx)));
                    const f32x2 qy = fma2(v4.y, dz, fma2(v2.y, dy, mul2(v3.y, dx)));
                    const f32x2 qz = fma2(v3.x, dz, fma2(v4.y, dy, mul2(v4.x, dx)));
                    const f32x2 dqd = fma2(dz, qz, fma2(dy, qy, mul2(dx, qx)));
                    const f32x2 t5 = mul2(dqd, r5);                      // (d.Q.d)/d^5
                    // c1 = -M/d^3 - 5/2 (d.Q.d)/d^7
                    const f32x2 c1 = fma2(mul2(t5, rinv2), KM25, mul2(v1.y, r3));
                    fax = fma2(c1, dx, fma2(r5, qx, fax));
                    fay = fma2(c1, dy, fma2(r5, qy, fay));
                    faz = fma2(c1, dz, fma2(r5, qz, faz));
                    fpot = fma2(v1.y, rinv, fma2(t5, KM05, fpot));
                }
            }
            add_to(acc.ax, 0, lo2(fax) + hi2(fax));
            add_to(acc.ay, 1, lo2(fay) + hi2(fay));
            add_to(acc.az, 2, lo2(faz) + hi2(faz));
            add_to(acc.pot, 3, lo2(fpot) + hi2(fpot));
            if constexpr (EWALD) {
                // the table is for a cube of side 1: f scales as 1/L^2, g as 1/L
                add_to(acc.ax, 0, lo2(ewxy) * iL * iL);
                add_to(acc.ay, 1, hi2(ewxy) * iL * iL);
                add_to(acc.az, 2, lo2(ewzw) * iL * iL);
                add_to(acc.pot, 3, hi2(ewzw) * iL);
            }
            nfar = 0;
            __syncwarp();
        };

        auto flush_near = [&]() {
            __syncwarp();
            // an odd list gets an empty partner entry (no lanes, finite zeros) for the two-wide pass
            if ((nnear & 1) && lane == 0) {
                sm.near_mask[w][nnear] = 0u;
                float *f = sm.npair[w][nnear >> 1] + 1;
#pragma unroll
                for (int c = 0; c < 6; ++c) f[2 * c] = 0.f;
            }
            for (int l = lane; l < nnear; l += 32) {
                const int j = sm.near_j[w][l];
                wpp += __popc(sm.near_mask[w][l]);         // interaction count (this lane's share)
                const float4 pj = d.pos[j];
                const float4 gj = d.grav[j];
                float *f = sm.npair[w][l >> 1] + (l & 1);
                const float te = GRAV ? 2.f / gj.x : 0.f, th = 2.f * gj.z;
                f[0] = pj.x; f[2] = pj.y; f[4] = pj.z; f[6] = pj.w;
                f[8] = te * te;
                f[10] = gj.z > 0.f ? th * th : -1.f;
                sm.ng[w][l] = gj;
                if (SPH) {
                    sm.nh[w][l] = d.hydro[j];
                    sm.ns[w][l] = d.snd[j];
                }
                if constexpr (DISS) ds.nd[w][l] = d.diss[j];     // read only for gas pairs
                if constexpr (CHECK) cks.norig[w][l] = d.orig[j];
            }
            if (lane == 0) wc[1] += 32u * (unsigned)((nnear + 1) & ~1);
            if constexpr (MIXED && GRAV) {
                // park the running gravity totals; the pair loop sums this flush's block from zero
                mx.c[w][4][lane] = acc.ax;
                mx.c[w][5][lane] = acc.ay;
                mx.c[w][6][lane] = acc.az;
                mx.c[w][7][lane] = acc.pot;
                acc.ax = acc.ay = acc.az = acc.pot = 0.f;
            }
            __syncwarp();
            // Pass 1, every entry, two at a time in packed form.  A gravity pair farther apart than
            // 2 max(eps_i, eps_j) is Newtonian: both softened kernels equal their point-mass forms
            // there (Eqs. softforce, softphi) and the correction term vanishes with dW/dr; it is summed
            // here (as +m/r^3 d and +m/r, subtracted at the end).  Pairs inside that distance, and gas
            // pairs inside 2 max(h_i, h_j), are marked per lane (bit t of sbits) and evaluated in
            // pass 2, where the warp's marked pairs are shared out 32 at a time.
            unsigned long long sbits = 0ull;
            {
                const f32x2 PX = pk2(pi.x, pi.x), PY = pk2(pi.y, pi.y), PZ = pk2(pi.z, pi.z);
                f32x2 nax = 0ull, nay = 0ull, naz = 0ull, npot = 0ull;
                f32x2 ewnxy = 0ull, ewnzw = 0ull;
                for (int q = 0; q < (nnear + 1) >> 1; ++q) {
                    const uint2 mk = *reinterpret_cast<const uint2 *>(&sm.near_mask[w][2 * q]);
                    const ulonglong2 *F = reinterpret_cast<const ulonglong2 *>(sm.npair[w][q]);
                    const ulonglong2 v0 = F[0], v1 = F[1], v2 = F[2];   // (x, y), (z, m), (E, H)
                    f32x2 dx = sub2(PX, v0.x), dy = sub2(PY, v0.y), dz = sub2(PZ, v1.x);
                    if (pm) {
                        dx = pk2(evol_wrap(lo2(dx), plen0, pm & 1), evol_wrap(hi2(dx), plen0, pm & 1));
                        dy = pk2(evol_wrap(lo2(dy), plen1, pm & 2), evol_wrap(hi2(dy), plen1, pm & 2));
                        dz = pk2(evol_wrap(lo2(dz), plen2, pm & 4), evol_wrap(hi2(dz), plen2, pm & 4));
                    }
                    const f32x2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
                    const float ra = lo2(r2), rb = hi2(r2);
                    const bool mine_a = (mk.x >> lane) & 1u, mine_b = (mk.y >> lane) & 1u;
                    if constexpr (EWALD) {
                        // every pair, softened or not: the replicas of j beyond its nearest image
                        if (mine_a) {
                            const float ex = lo2(dx), ey = lo2(dy), ez = lo2(dz);
                            const Ew2 c = ewald_lookup2(kp.ewald_tab, ex, ey, ez, kp.ewald_sc);
                            const float mj = lo2(v1.y);
                            ewnxy = fma2(pk2(ex < 0.f ? -mj : mj, ey < 0.f ? -mj : mj), c.xy, ewnxy);
                            ewnzw = fma2(pk2(ez < 0.f ? -mj : mj, mj), c.zw, ewnzw);
                        }
                        if (mine_b) {
                            const float ex = hi2(dx), ey = hi2(dy), ez = hi2(dz);
                            const Ew2 c = ewald_lookup2(kp.ewald_tab, ex, ey, ez, kp.ewald_sc);
                            const float mj = hi2(v1.y);
                            ewnxy = fma2(pk2(ex < 0.f ? -mj : mj, ey < 0.f ? -mj : mj), c.xy, ewnxy);
                            ewnzw = fma2(pk2(ez < 0.f ? -mj : mj, mj), c.zw, ewnzw);
                        }
                    }
                    if (CHECK) cpp += (mine_a ? 1 : 0) + (mine_b ? 1 : 0);
                    bool mark_a = false, mark_b = false;
                    if (GRAV) {
                        const bool soft_a = ra < fmaxf(E_i, lo2(v2.x)), soft_b = rb < fmaxf(E_i, hi2(v2.x));
                        const float ia = (mine_a && !soft_a) ? rsqrtf(ra) : 0.f;
                        const float ib = (mine_b && !soft_b) ? rsqrtf(rb) : 0.f;
                        const f32x2 rinv = pk2(ia, ib);
                        const f32x2 mr = mul2(v1.y, rinv);                   // m_j / r
                        const f32x2 mr3 = mul2(mr, mul2(rinv, rinv));
                        nax = fma2(mr3, dx, nax);
                        nay = fma2(mr3, dy, nay);
                        naz = fma2(mr3, dz, naz);
                        npot = add2(npot, mr);
                        mark_a = mine_a && soft_a;
                        mark_b = mine_b && soft_b;
                    }
                    if (SPH) {
                        const float Ha = lo2(v2.y), Hb = hi2(v2.y);
                        mark_a = mark_a || (mine_a && fminf(H_i, Ha) >= 0.f && ra < fmaxf(H_i, Ha));
                        mark_b = mark_b || (mine_b && fminf(H_i, Hb) >= 0.f && rb < fmaxf(H_i, Hb));
                    }
                    sbits |= ((unsigned long long)(mark_a ? 1u : 0u) | ((unsigned long long)(mark_b ? 1u : 0u) << 1)) << (2 * q);
                }
                if (GRAV) {
                    acc.ax -= lo2(nax) + hi2(nax);
                    acc.ay -= lo2(nay) + hi2(nay);
                    acc.az -= lo2(naz) + hi2(naz);
                    acc.pot -= lo2(npot) + hi2(npot);
                }
                if constexpr (EWALD) {
                    acc.ax += lo2(ewnxy) * iL * iL;
                    acc.ay += hi2(ewnxy) * iL * iL;
                    acc.az += lo2(ewnzw) * iL * iL;
                    acc.pot += hi2(ewnzw) * iL;
                }
            }
            // Pass 2: the marked pairs, shared out over the warp.  The marks are enumerated lane by
            // lane (each lane's in entry order) and taken 32 at a time, item k of a batch by lane k,
            // which reads its pair's owner (the lane whose particle is i) from the sorted state.  The
            // items of one owner are consecutive: a segmented scan sums each batch's results per
            // owner, and the owner adds the total; maxima go to shared memory as atomic maxima (the
            // values are non-negative, so their bit patterns order like the floats).
            {
                const int nm = __popcll(sbits);
                int incl = nm;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                const int excl = incl - nm;               // this lane's first item
                const int nitems = __shfl_sync(0xffffffffu, incl, 31);
                const unsigned sb_lo = (unsigned)sbits, sb_hi = (unsigned)(sbits >> 32);
                const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
                // this lane's operands as an owner, formed once per flush and handed to the items by
                // shuffles (as at the top of the group: 1/eps, eps, X/Upsilon, h, zeta/Omega*, 1/m)
                const float4 gl = (nitems > 0 && valid) ? d.grav[s] : z4;
                const float eps_l = GRAV && valid ? 1.f / gl.x : 0.f;
                const float inv_ml = valid ? 1.f / pi.w : 0.f;
                for (int base = 0; base < nitems; base += 32) {
                    if (lane == 0) wc[2] += 32u;
                    const int item = base + lane;
                    // the owner: the last lane whose items start at or before this one
                    int o = 0;
#pragma unroll
                    for (int st = 16; st > 0; st >>= 1) {
                        const int ex = __shfl_sync(0xffffffffu, excl, o + st);
                        if (ex <= item) o += st;
                    }
                    const unsigned olo = __shfl_sync(0xffffffffu, sb_lo, o);
                    const unsigned ohi = __shfl_sync(0xffffffffu, sb_hi, o);
                    const int k = item - __shfl_sync(0xffffffffu, excl, o);    // the owner's k-th mark
                    const int so = __shfl_sync(0xffffffffu, s, o);
                    // the owner's operands
                    const float4 po = make_float4(__shfl_sync(0xffffffffu, pi.x, o), __shfl_sync(0xffffffffu, pi.y, o),
                                                  __shfl_sync(0xffffffffu, pi.z, o), 0.f);
                    const float4 go = make_float4(__shfl_sync(0xffffffffu, gl.x, o), __shfl_sync(0xffffffffu, gl.y, o),
                                                  __shfl_sync(0xffffffffu, gl.z, o), __shfl_sync(0xffffffffu, gl.w, o));
                    const float E_o = __shfl_sync(0xffffffffu, E_i, o), H_o = __shfl_sync(0xffffffffu, H_i, o);
                    const float eps_o = __shfl_sync(0xffffffffu, eps_l, o);
                    const float inv_mo = __shfl_sync(0xffffffffu, inv_ml, o);
                    const float ie_o = go.x, xu_o = go.y;
                    float sum[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                    if (item < nitems) {
                        const int nlo = __popc(olo);
                        const int t = k < nlo ? nth_bit(olo, k) : 32 + nth_bit(ohi, k - nlo);
                        const float *f = sm.npair[w][t >> 1] + (t & 1);
                        const float mj = f[6], Ej = f[8], Hj = f[10];
                        const float dx = evol_wrap(po.x - f[0], plen0, pm & 1);
                        const float dy = evol_wrap(po.y - f[2], plen1, pm & 2);
                        const float dz = evol_wrap(po.z - f[4], plen2, pm & 4);
                        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));     // as in pass 1
                        // r and 1/r from one reciprocal square root (coincident particles: both 0)
                        const float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
                        const float r = r2 * rinv;
                        const float4 gj = sm.ng[w][t];
                        if (GRAV && r2 < fmaxf(E_o, Ej)) {              // the same test as pass 1
                            ++wsoft;
                            // symmetrised softened pair force and potential (App. B), each side
                            // softened where u < 2 and Newtonian beyond
                            const float ui = r * ie_o, uj = r * gj.x;
                            const float iui = rinv * eps_o, iuj = rinv * rcp_fast(gj.x);
                            const float rinv3 = rinv * rinv * rinv;
                            const float fi = ui < 2.f ? gsoft_over_r_u(ui, iui) * ie_o * ie_o * ie_o : rinv3;
                            const float fj = uj < 2.f ? gsoft_over_r_u(uj, iuj) * gj.x * gj.x * gj.x : rinv3;
                            float fg = -0.5f * mj * (fi + fj);
                            sum[3] = mj * (ui < 2.f ? phisoft_u(ui, iui) * ie_o : -rinv);
                            if (kp.adaptive) {
                                // adaptive-softening correction (Eq. dLgravdr, mass-weighted reading)
                                const float ie2 = ie_o * ie_o, je2 = gj.x * gj.x;
                                const float ci = ui < 2.f ? xu_o * dw_over_u_u(ui, iui) * ie2 * ie2 * ie_o : 0.f;
                                const float cj = uj < 2.f ? gj.y * dw_over_u_u(uj, iuj) * je2 * je2 * gj.x : 0.f;
                                fg += -0.5f * inv_pi * (ci + mj * inv_mo * cj);
                            }
                            sum[0] = fg * dx;
                            sum[1] = fg * dy;
                            sum[2] = fg * dz;
                        }
                        if (SPH && fminf(H_o, Hj) >= 0.f && r2 < fmaxf(H_o, Hj)) {   // as in pass 1
                            ++wsph;
                            if constexpr (CHECK) {
                                atomicAdd(&cks.cs[w][o], 1);
                                atomicAdd(&cks.hs[w][o], evol_mix64((unsigned long long)cks.norig[w][t]));
                            }
                            if (kp.wake) {
                                // wake-up: the owner's step (ticks), recorded at its SPH neighbour
                                const int jo = d.orig[so];
                                atomicMin(&d.nbmin[sm.near_j[w][t]], (unsigned)(d.te[jo] - d.tb[jo]));
                            }
                            if (r2 > 0.f) {
                                const float4 gi = go;
                                const float4 hi = d.hydro[so];
                                const float4 si = d.snd[so];
                                const float4 di = DISS ? d.diss[so] : z4;
                                const float4 hj = sm.nh[w][t];
                                const float4 sj = sm.ns[w][t];
                                const float ihi = si.z, ihj = sj.z;
                                const float uhi = r * ihi, uhj = r * ihj;
                                const float iuhi = rinv * gi.z, iuhj = rinv * gj.z;     // h / r
                                const float ihi2 = ihi * ihi, ihj2 = ihj * ihj;
                                const float kgi = (kp.use_tc ? tc_over_u_u(uhi, iuhi) : dw_over_u_u(uhi, iuhi)) * ihi2 * ihi2 * ihi * inv_pi;
                                const float kgj = (kp.use_tc ? tc_over_u_u(uhj, iuhj) : dw_over_u_u(uhj, iuhj)) * ihj2 * ihj2 * ihj * inv_pi;
                                const float fi = 1.f + gi.w * rcp_fast(mj);       // 1 + zeta_i / (m_j Omega*_i)
                                const float fj = 1.f + gj.w * inv_mo;             // 1 + zeta_j / (m_i Omega*_j)
                                const float vx = hi.x - hj.x, vy = hi.y - hj.y, vz = hi.z - hj.z;
                                const float vr = vx * dx + vy * dy + vz * dz;
                                float visc = 0.f;
                                // dissipation variants: w_ij = v_ij . r_ij / r and the signal velocity
                                // v^sig_ij = c_i + c_j - min(w_ij, 0) (Eq. vsig)
                                float4 dj = z4;
                                float wij = 0.f, vsig = 0.f;
                                if constexpr (DISS) {
                                    dj = ds.nd[w][t];
                                    wij = vr * rinv;
                                    vsig = si.x + sj.x - fminf(wij, 0.f);
                                    atomicMax(reinterpret_cast<int *>(&ds.vs[w][o]), __float_as_int(vsig));
                                }
                                if (vr < 0.f) {
                                    const float hb = 0.5f * (gi.z + gj.z);
                                    const float mu = hb * vr * rcp_fast(r2 + 0.01f * hb * hb);
                                    atomicMax(reinterpret_cast<int *>(&sm.mum[w][o]), __float_as_int(-mu));   // |mu|
                                    const float cb = 0.5f * (si.x + sj.x);
                                    const float rb = 0.5f * (si.y + sj.y);
                                    if constexpr (!DISS) {
                                        visc = (-kp.alpha * cb * mu + kp.beta * mu * mu) * rcp_fast(rb);
                                    } else {
                                        // alpha_ij = (alpha_i + alpha_j)/2 (Eq. alphaswitch); Monaghan
                                        // (Eq. mu_visc) or signal-velocity form (Eq. pvsig); Balsara
                                        // limiter (f_i + f_j)/2
                                        const float al = kp.var_alpha ? 0.5f * (di.x + dj.x) : kp.alpha;
                                        visc = (kp.visc_form == EVOL_VISC_SIGNAL ? -al * vsig * wij
                                                                                  : (-al * cb * mu + kp.beta * mu * mu)) *
                                               rcp_fast(rb);
                                        if (kp.balsara) visc *= 0.5f * (di.y + dj.y);
                                    }
                                }
                                const float gbar = 0.5f * (kgi * fi + kgj * fj);
                                const float pterm_i = hi.w * fi * kgi;
                                const float sc = -mj * (pterm_i + hj.w * fj * kgj + visc * gbar);
                                sum[4] = sc * dx;
                                sum[5] = sc * dy;
                                sum[6] = sc * dz;
                                sum[7] = mj * (pterm_i + 0.5f * visc * gbar) * vr;
                                if constexpr (DISS) {
                                    if (kp.conduction) {
                                        // artificial conductivity: du_i/dt += m_j Pi^u_ij |gradbar W_ij| with
                                        // Pi^u = -alphabar^u v^u (u_i - u_j) / rhobar (gbar is the mean
                                        // gradient over r); Brookshaw's sum 2 m_j (u_i - u_j)/rho_j |gradbar W|/r
                                        const float irb = rcp_fast(0.5f * (si.y + sj.y));
                                        const float duij = di.z - dj.z;
                                        const float vu = kp.cond_vsig == EVOL_COND_VSIG_PRESSURE
                                                             ? sqrtf(fabsf(si.w - sj.w) * irb)
                                                             : vsig;
                                        const float ag = fabsf(gbar);
                                        sum[7] -= mj * (0.5f * (di.w + dj.w)) * vu * duij * irb * ag * r;
                                        sum[8] = 2.f * mj * duij * rcp_fast(sj.y) * ag;
                                    }
                                }
                            }
                        }
                    }
                    // segmented inclusive scan over the batch: a segment starts where the owner changes
                    const int oprev = __shfl_up_sync(0xffffffffu, o, 1);     // every lane takes part
                    int head = (lane == 0 || oprev != o) ? 1 : 0;
#pragma unroll
                    for (int dd = 1; dd < 32; dd <<= 1) {
                        const int hu = __shfl_up_sync(0xffffffffu, head, dd);
#pragma unroll
                        for (int q = 0; q < 9; ++q) {
                            if ((q < 4 && !GRAV) || (q >= 4 && q < 8 && !SPH) || (q == 8 && !DISS)) continue;
                            const float vu = __shfl_up_sync(0xffffffffu, sum[q], dd);
                            if (lane >= dd && !head) sum[q] += vu;
                        }
                        if (lane >= dd) head |= hu;
                    }
                    // each owner takes its segment's total from the segment's last item
                    const bool mine = nm > 0 && excl < base + 32 && excl + nm > base;
                    const int tail = (min(excl + nm, base + 32) - 1 - base) & 31;
                    float tot_[9];
#pragma unroll
                    for (int q = 0; q < 9; ++q) {
                        tot_[q] = 0.f;
                        if ((q < 4 && !GRAV) || (q >= 4 && q < 8 && !SPH) || (q == 8 && !DISS)) continue;
                        const float tv = __shfl_sync(0xffffffffu, sum[q], tail);
                        if (mine) tot_[q] = tv;
                    }
                    if (mine) {
                        acc.ax += tot_[0];
                        acc.ay += tot_[1];
                        acc.az += tot_[2];
                        acc.pot += tot_[3];
                        acc.hx += tot_[4];
                        acc.hy += tot_[5];
                        acc.hz += tot_[6];
                        acc.du += tot_[7];
                        if constexpr (DISS) ds.lap[w][lane] += tot_[8];
                    }
                }
            }
            if constexpr (MIXED && GRAV) {
                // the block's sums into the parked totals, compensated
                float b = acc.ax;
                acc.ax = mx.c[w][4][lane];
                add_to(acc.ax, 0, b);
                b = acc.ay;
                acc.ay = mx.c[w][5][lane];
                add_to(acc.ay, 1, b);
                b = acc.az;
                acc.az = mx.c[w][6][lane];
                add_to(acc.az, 2, b);
                b = acc.pot;
                acc.pot = mx.c[w][7][lane];
                add_to(acc.pot, 3, b);
            }
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
        int top = 0;
        // nodes accepted for all by the super-group, taken 32 at a time before the stack: [apos, aend)
        const int *alist = d.sg_acc;
        int apos = 0, aend = 0;
        // (not in the periodic gravity walk, which opens every node above L/8 and keeps its registers
        // for the Ewald lookups)
        const int2 sgi = (!EWALD && kp.super) ? d.sg_info[g / SG_GROUPS] : make_int2(-1, -1);
        if (sgi.x >= 0 && sgi.y <= kp.stack_cap) {
            // the super-group's lists (k_super), with the mask of every active lane: its frontier on
            // the stack, the nodes it accepted for all as batches that skip the node tests (they
            // count only as far nodes, and as accepted nodes in check mode)
            const size_t sgb = (size_t)(g / SG_GROUPS);
            for (int k = lane; k < sgi.y; k += 32)
                stk[k] = make_int2(d.sg_front[sgb * EVOL_SG_FCAP + k], (int)rootmask);
            top = sgi.y;
            alist = d.sg_acc + sgb * EVOL_SG_ACAP;
            aend = (GRAV || CHECK) ? sgi.x : 0;
        } else {
            // one stack entry per system present in the group: its root with the mask of its lanes
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
        while (top > 0 || apos < aend) {
            if (++pops > pop_cap) {
                if (lane == 0) {
                    evol_flag(d.err, EVOL_ETIMEOUT);
                    atomicMax(&d.counters[7], 1ull);
                }
                break;
            }
            int node = -1;
            unsigned M = 0;
            const bool pre = apos < aend;    // a batch of the super-group's accepted nodes
            int k;
            if (pre) {
                k = min(aend - apos, 32);
                if (lane < k) {
                    node = alist[apos + lane];
                    M = rootmask;
                }
                apos += k;
            } else {
                k = min(top, 32);
                top -= k;
                if (lane < k) {
                    const int2 e = stk[top + lane];
                    node = e.x;
                    M = (unsigned)e.y;
                }
            }
            __syncwarp();
            int4 I = make_int4(0, 0, 0, 0);
            int cls = 0;                     // 0 none, 1 accept all, 2 open all, 3 mixed
            unsigned Ak = 0, Ok = 0;
            if (pre) {
                if (lane < k) {
                    cls = 1;
                    Ak = M;
                }
            } else if (lane < k) {
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
                if (EWALD && !(ldexpf(side0, -(I.x & 0xff)) <= 0.125f * kp.ewald_L)) {
                    // periodic gravity: nodes of side above L/8 are always opened (their replicas'
                    // correction is taken as a monopole, whose error grows as (l/L)^2)
                    acc_all = false;
                    open_all = true;
                }
                if (GRAV) {
                    const float ax = fabsf(evol_wrap(A.x - gcx, plen0, pmg & 1)), ay = fabsf(evol_wrap(A.y - gcy, plen1, pmg & 2)),
                                az = fabsf(evol_wrap(A.z - gcz, plen2, pmg & 4));
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
            unsigned mm = pre ? 0u : __ballot_sync(0xffffffffu, cls == 3);
            if (lane == 0 && !pre) {
                wc[3] += (unsigned)k;
                wc[4] += (unsigned)__popc(mm);
            }
            while (mm) {
                const int kk = __ffs(mm) - 1;
                mm &= mm - 1u;
                const unsigned Mk = __shfl_sync(0xffffffffu, M, kk);
                bool far = false;
                if ((Mk >> lane) & 1u) {
                    const float4 B = sm.bB[w][kk];
                    const float4 C = sm.bC[w][kk];
                    const float qx = fabsf(evol_wrap(pi.x - B.x, plen0, pm & 1));
                    const float qy = fabsf(evol_wrap(pi.y - B.y, plen1, pm & 2));
                    const float qz = fabsf(evol_wrap(pi.z - B.z, plen2, pm & 4));
                    const float ex = fmaxf(qx - C.x, 0.f), ey = fmaxf(qy - C.y, 0.f), ez = fmaxf(qz - C.z, 0.f);
                    const float bd2 = ex * ex + ey * ey + ez * ez;
                    float R = GRAV ? fmaxf(two_eps_i, C.w) : 0.f;
                    if (SPH && gas_i && B.w >= 0.f) R = fmaxf(R, fmaxf(two_h_i, B.w));
                    far = bd2 > R * R;
                    if (GRAV && far) {
                        const float4 A = sm.bA[w][kk];
                        const float dx = evol_wrap(pi.x - A.x, plen0, pmg & 1), dy = evol_wrap(pi.y - A.y, plen1, pmg & 2),
                                    dz = evol_wrap(pi.z - A.z, plen2, pmg & 4);
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
                if (nfar + cnt > FARCAP - 2 * EVOL_FAR_UNROLL + 1) flush_far();
                if (Ak) {
                    const int pos = nfar + __popc(fa & ltmask);
                    sm.far_id[w][pos] = node;
                    sm.far_mask[w][pos] = Ak;
                }
                nfar += cnt;
            }
            if (pre) continue;               // nothing opened
            // opened leaves: their particles go to the near list
            const bool isleaf = (I.x >> 8) & 1;
            unsigned lm = __ballot_sync(0xffffffffu, Ok != 0u && isleaf);
            {
                const unsigned im = __ballot_sync(0xffffffffu, Ok != 0u && !isleaf);
                if (lane == 0) {
                    wc[5] += (unsigned)__popc(lm);
                    wc[6] += (unsigned)__popc(im);
                }
            }
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
                    if (!kp.active) {
                        if (lane < kc) {
                            // the particle itself never pairs with itself: its lane leaves the mask
                            const int j = b + lane, sl = j - g * 32;
                            sm.near_j[w][nnear + lane] = j;
                            sm.near_mask[w][nnear + lane] = ok & ~((sl >= 0 && sl < 32) ? (1u << sl) : 0u);
                        }
                    } else {
                        // active list: the group's lanes hold arbitrary sorted positions; the lane
                        // whose particle is entry b + q marks slot q, and that bit leaves the mask
                        if (lane < kc) sm.gself[w][lane] = 0u;
                        __syncwarp();
                        const int mine = sm.gs[w][lane];
                        if (mine >= b && mine < b + kc) sm.gself[w][mine - b] = 1u << lane;
                        __syncwarp();
                        if (lane < kc) {
                            sm.near_j[w][nnear + lane] = b + lane;
                            sm.near_mask[w][nnear + lane] = ok & ~sm.gself[w][lane];
                        }
                        __syncwarp();
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

        double tax = acc.ax, tay = acc.ay, taz = acc.az, tpot = acc.pot;
        double thx = acc.hx, thy = acc.hy, thz = acc.hz, tdu = acc.du;
        if constexpr (MIXED) {
            // total = running sum + compensation, in FP64
            tax += (double)mx.c[w][0][lane]; tay += (double)mx.c[w][1][lane];
            taz += (double)mx.c[w][2][lane]; tpot += (double)mx.c[w][3][lane];
        }
        if (valid) {
            float ax = 0.f, ay = 0.f, az = 0.f, pot = 0.f;
            if (GRAV) {
                // self term of the potential: m_i phi(0, eps_i) = -7/5 m_i / eps_i
                const double G = kp.G;
                ax = (float)(G * tax);
                ay = (float)(G * tay);
                az = (float)(G * taz);
                double self_img = 0.0;
                if (EWALD) self_img = (double)pi.w * (double)kp.ewald_tab[0].w * (double)iL;   // own replicas
                pot = (float)(G * (tpot - 1.4 * (double)pi.w * (double)ie_i + self_img));
            }
            ax += (float)thx;
            ay += (float)thy;
            az += (float)thz;
            d.acc[s] = make_float4(ax, ay, az, pot);
            if (SPH) {
                d.dudt[s] = gas_i ? (float)tdu : 0.f;
                d.mumax[s] = gas_i ? sm.mum[w][lane] : 0.f;
                const float4 hv = d.hydro[s];
                d.vah[s] = gas_i ? (float)(hv.x * thx + hv.y * thy + hv.z * thz) : 0.f;
            }
            if constexpr (DISS) {
                if (gas_i) {
                    // v^sig_i = max(2 c_i, max_j v^sig_ij) (the self pair has w = 0); tau_i =
                    // alpha_tau h_i / v^sig_i; the switches of alpha (Eq. alphaswitch) and alpha^u
                    const float4 sn = d.snd[s], di = d.diss[s];
                    const float h_i = g0.z;
                    const float vs = fmaxf(ds.vs[w][lane], 2.f * sn.x);
                    const float lap = ds.lap[w][lane];
                    const float itau = vs / (kp.alpha_tau * h_i);
                    d.vsig[s] = vs;
                    d.lapu[s] = lap;
                    if (kp.var_alpha)
                        d.dalpha[s] = -(di.x - kp.alpha_min) * itau + kp.alpha_source * di.y * fmaxf(0.f, -d.divv_h[s]);
                    if (kp.conduction) {
                        const float src = kp.cond_source == EVOL_COND_SRC_LINEAR ? 0.1f * h_i * fabsf(lap)
                                                                                 : h_i * fabsf(lap) * rsqrtf(di.z);
                        d.dalpha_u[s] = -(di.w - kp.alpha_u_min) * itau + src;
                    }
                }
            }
            if constexpr (CHECK) {
                d.hash3[3 * s + 0] = hfar;
                d.hash3[3 * s + 1] = hnear;
                d.hash3[3 * s + 2] = cks.hs[w][lane];
                d.cnt3[3 * s + 0] = cfar;
                d.cnt3[3 * s + 1] = cpp;
                d.cnt3[3 * s + 2] = cks.cs[w][lane];
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
            for (int q = 0; q < 7; ++q) atomicAdd(&d.counters[9 + q], (unsigned long long)wc[q]);
        }
    }
}

// Super-groups: 8 consecutive groups (256 consecutive entries of the particle list) walk the top of
// the tree once for all 8.  A node that the super-group's bounds accept for every one of its
// particles is accepted by each particle's own test (the bounds hold with the same margin as the
// group bounds, and a group's particles are a subset), and every particle reaches it (each of its
// ancestors was opened for all of them); such nodes are listed once and go to each group's far
// list with the mask of all its lanes.  Nodes the bounds leave undecided, and the leaves they open
// for all, form the frontier from which each group's own traversal starts.  A super-group with
// particles of more than one system, or whose lists do not fit, is marked, and its groups walk
// from the root.
template <bool GRAV, bool SPH, bool EWALD>
__global__ void __launch_bounds__(32, 24) k_super(evol_dev d, evol_kparams kp, int nsg)
{
    const int lane = threadIdx.x;
    const int n = kp.n;
    const int nlist = kp.active ? d.acts[n] : n;
    const int pm = ((SPH && !GRAV) || EWALD) ? kp.periodic_mask : 0;
    const int pmg = EWALD ? kp.periodic_mask : 0;
    const float plen0 = kp.plen[0], plen1 = kp.plen[1], plen2 = kp.plen[2];
    const float side0 = EWALD ? d.fcube[3] : 0.f;
    int *stk = reinterpret_cast<int *>(d.wstack + (size_t)blockIdx.x * kp.stack_stride);
    const int stack_cap = 2 * kp.stack_cap;
    const unsigned ltmask = (1u << lane) - 1u;
    const long long pop_cap = 2ll * (long long)(*d.nnodes) + 64;
    for (int sg = blockIdx.x; sg < nsg; sg += gridDim.x) {
        // bounds over the super-group's active particles (as the group bounds of the walk)
        float gx0 = INFINITY, gy0 = INFINITY, gz0 = INFINITY, gx1 = -INFINITY, gy1 = -INFINITY, gz1 = -INFINITY;
        float emax = 0.f, emin = INFINITY, hmax = -1.f, hmin = INFINITY;
        int rmin = 0x7fffffff, rmax = -1;
        bool all_gas = true;
#pragma unroll 1
        for (int q = 0; q < 32 * SG_GROUPS; q += 32) {
            const int e = sg * 32 * SG_GROUPS + q + lane;
            if (e >= nlist) continue;
            const int s = kp.active ? d.act[e] : e;
            const float4 p = d.pos[s];
            const float4 g0 = d.grav[s];
            const bool gas = SPH && g0.z > 0.f;
            if (!(GRAV || gas)) continue;           // not active in this walk
            gx0 = fminf(gx0, p.x); gy0 = fminf(gy0, p.y); gz0 = fminf(gz0, p.z);
            gx1 = fmaxf(gx1, p.x); gy1 = fmaxf(gy1, p.y); gz1 = fmaxf(gz1, p.z);
            if (GRAV) {
                const float te = 2.f / g0.x;
                emax = fmaxf(emax, te);
                emin = fminf(emin, te);
            }
            if (gas) {
                hmax = fmaxf(hmax, 2.f * g0.z);
                hmin = fminf(hmin, 2.f * g0.z);
            } else {
                all_gas = false;
            }
            const int r = d.sys_root[d.sys_sorted[s]];
            rmin = min(rmin, r);
            rmax = max(rmax, r);
        }
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
            rmin = min(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
            rmax = max(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
        }
        all_gas = SPH && __all_sync(0xffffffffu, all_gas);
        if (!GRAV) emin = 0.f;
        int2 info = make_int2(-1, -1);
        if (rmax >= 0 && rmin == rmax) {
            const float gcx = 0.5f * (gx0 + gx1), gcy = 0.5f * (gy0 + gy1), gcz = 0.5f * (gz0 + gz1);
            const float gwx = 0.5f * (gx1 - gx0), gwy = 0.5f * (gy1 - gy0), gwz = 0.5f * (gz1 - gz0);
            int *acc = d.sg_acc + (size_t)sg * EVOL_SG_ACAP;
            int *front = d.sg_front + (size_t)sg * EVOL_SG_FCAP;
            int na = 0, nf = 0, top = 1;
            bool ok = true;
            if (lane == 0) stk[0] = rmin;
            __syncwarp();
            long long pops = 0;
            while (top > 0) {
                if (++pops > pop_cap) {
                    ok = false;
                    break;
                }
                const int k = min(top, 32);
                top -= k;
                const int node = lane < k ? stk[top + lane] : -1;
                __syncwarp();
                int cls = 0;                 // 0 none, 1 accept all, 2 open all, 3 mixed
                bool leaf = false;
                int4 I = make_int4(0, 0, 0, 0);
                if (lane < k) {
                    I = d.nI[node];
                    const float4 B = d.nB[node];
                    const float4 C = d.nC[node];
                    const float4 A = GRAV ? d.nA[node] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float dx = fabsf(evol_wrap(B.x - gcx, plen0, pm & 1));
                    const float dy = fabsf(evol_wrap(B.y - gcy, plen1, pm & 2));
                    const float dz = fabsf(evol_wrap(B.z - gcz, plen2, pm & 4));
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
                    if (EWALD && !(ldexpf(side0, -(I.x & 0xff)) <= 0.125f * kp.ewald_L)) {
                        acc_all = false;
                        open_all = true;
                    }
                    if (GRAV) {
                        const float ax = fabsf(evol_wrap(A.x - gcx, plen0, pmg & 1)), ay = fabsf(evol_wrap(A.y - gcy, plen1, pmg & 2)),
                                    az = fabsf(evol_wrap(A.z - gcz, plen2, pmg & 4));
                        const float mx = fmaxf(ax - gwx, 0.f), my = fmaxf(ay - gwy, 0.f), mz = fmaxf(az - gwz, 0.f);
                        const float Mx = ax + gwx, My = ay + gwy, Mz = az + gwz;
                        acc_all = acc_all && (mx * mx + my * my + mz * mz > A.w * (1.f + TAU));
                        open_all = open_all || (Mx * Mx + My * My + Mz * Mz < A.w * (1.f - TAU));
                    }
                    cls = acc_all ? 1 : (open_all ? 2 : 3);
                    leaf = (I.x >> 8) & 1;
                }
                // accepted for all: listed (far nodes of the gravity walks; the SPH-only walks read
                // them only in check mode, which records every accepted node)
                const unsigned am = __ballot_sync(0xffffffffu, cls == 1);
                if (am) {
                    if (na + __popc(am) > EVOL_SG_ACAP) {
                        ok = false;
                        break;
                    }
                    if (cls == 1) acc[na + __popc(am & ltmask)] = node;
                    na += __popc(am);
                }
                // undecided, or a leaf opened for all: the groups' frontier
                const bool fr = cls == 3 || (cls == 2 && leaf);
                const unsigned fm = __ballot_sync(0xffffffffu, fr);
                if (fm) {
                    if (nf + __popc(fm) > EVOL_SG_FCAP) {
                        ok = false;
                        break;
                    }
                    if (fr) front[nf + __popc(fm & ltmask)] = node;
                    nf += __popc(fm);
                }
                // internal nodes opened for all: push their children
                const bool io = cls == 2 && !leaf;
                int nch = 0;
                int ch[8];
                if (io) {
                    const int4 K0 = d.nK0[node], K1 = d.nK1[node];
                    ch[0] = K0.x; ch[1] = K0.y; ch[2] = K0.z; ch[3] = K0.w;
                    ch[4] = K1.x; ch[5] = K1.y; ch[6] = K1.z; ch[7] = K1.w;
#pragma unroll
                    for (int u = 0; u < 8; ++u) nch += ch[u] >= 0 ? 1 : 0;
                }
                int incl = nch;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                const int total = __shfl_sync(0xffffffffu, incl, 31);
                if (top + total > stack_cap) {
                    ok = false;
                    break;
                }
                if (io) {
                    const int pos = top + incl - nch;
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (u < nch) stk[pos + u] = ch[u];
                }
                top += total;
                __syncwarp();
            }
            if (ok) info = make_int2(na, nf);
        }
        if (lane == 0) d.sg_info[sg] = info;
        __syncwarp();
    }
}

template <bool GRAV, bool SPH, bool MIXED, bool CHECK, bool DISS, bool EWALD>
void launch_walk(evol_ctx *c, const evol_kparams &kp)
{
    static int blocks_per_sm = -1;
    if (blocks_per_sm < 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_walk<GRAV, SPH, MIXED, CHECK, DISS, EWALD>,
                                                      WK_THREADS, 0);
        if (blocks_per_sm < 1) blocks_per_sm = 1;
        if (blocks_per_sm > 8) blocks_per_sm = 8;          // stack slots exist for 32 warps per SM
    }
    unsigned long long *q = c->d.counters + 4;
    cudaMemsetAsync(q, 0, sizeof(unsigned long long), c->stream);
    k_walk<GRAV, SPH, MIXED, CHECK, DISS, EWALD><<<c->num_sms * blocks_per_sm, WK_THREADS, 0, c->stream>>>(c->d, kp, q);
}

template <bool GRAV, bool SPH, bool DISS, bool EWALD>
void launch_walk_pcd(evol_ctx *c, const evol_kparams &kp, bool mixed, bool check)
{
    if (mixed) {
        if (check) launch_walk<GRAV, SPH, true, true, DISS, EWALD>(c, kp);
        else launch_walk<GRAV, SPH, true, false, DISS, EWALD>(c, kp);
    } else {
        if (check) launch_walk<GRAV, SPH, false, true, DISS, EWALD>(c, kp);
        else launch_walk<GRAV, SPH, false, false, DISS, EWALD>(c, kp);
    }
}

template <bool GRAV, bool SPH, bool EWALD>
void launch_walk_pce(evol_ctx *c, const evol_kparams &kp, bool mixed, bool check)
{
    // the super-groups' top-of-tree walk first (one warp per block, 16 blocks per SM)
    const int nsg = (kp.n + 32 * SG_GROUPS - 1) / (32 * SG_GROUPS);
    if (!EWALD && kp.super && nsg > 0) k_super<GRAV, SPH, EWALD><<<c->num_sms * 24, 32, 0, c->stream>>>(c->d, kp, nsg);
    if constexpr (SPH) {
        if (kp.diss) {
            launch_walk_pcd<GRAV, SPH, true, EWALD>(c, kp, mixed, check);
            return;
        }
    }
    launch_walk_pcd<GRAV, SPH, false, EWALD>(c, kp, mixed, check);
}

template <bool GRAV, bool SPH>
void launch_walk_pc(evol_ctx *c, const evol_kparams &kp, bool mixed, bool check)
{
    if constexpr (GRAV) {
        if (kp.ewald) {
            launch_walk_pce<GRAV, SPH, true>(c, kp, mixed, check);
            return;
        }
    }
    launch_walk_pce<GRAV, SPH, false>(c, kp, mixed, check);
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
    kp.active = c->bins_active;
    kp.wake = c->bins_active && do_sph && c->d.nbmin != nullptr && c->bins_wake;
    kp.ewald = do_grav && prm->periodic_mask == 7;
    if (kp.ewald) {
        kp.ewald_L = prm->periodic_hi[0] - prm->periodic_lo[0];
        kp.ewald_sc = 2.f * EVOL_EWALD_N / kp.ewald_L;
        kp.ewald_tab = c->d.ewald;
    }
    kp.diss = do_sph && evol_diss_on(prm);
    kp.visc_form = prm->visc_form;
    kp.balsara = prm->balsara;
    kp.var_alpha = prm->variable_alpha;
    kp.conduction = prm->conduction;
    kp.cond_vsig = prm->cond_vsig;
    kp.cond_source = prm->cond_source;
    kp.alpha_min = prm->alpha_min;
    kp.alpha_tau = prm->alpha_tau;
    kp.alpha_source = prm->alpha_source;
    kp.alpha_u_min = prm->alpha_u_min;
    kp.super = 1;
    bool mixed = prm->precision == EVOL_FP32_MIXED;
    bool check = c->check_mode != 0;
    if (do_grav && do_sph) launch_walk_pc<true, true>(c, kp, mixed, check);
    else if (do_grav) launch_walk_pc<true, false>(c, kp, mixed, check);
    else if (do_sph) launch_walk_pc<false, true>(c, kp, mixed, check);
    return evol_cuda_ok(cudaGetLastError());
}
