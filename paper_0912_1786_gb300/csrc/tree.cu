// Tree build on the GPU (Sect. 2.2 of the paper): root cube, 63-bit Morton keys, stable LSD
// radix sort, particle permutation, pre-order octree from the sorted keys, and node moments
// reduced bottom-up.
//
// Node construction does not insert particles one by one.  With keys sorted, the cells of
// level l are the maximal runs of keys sharing their top 3l bits; a cell is a node iff its
// parent cell holds more than `leaf` particles (the root always is).  Writing d_i for the
// number of leading octal digits that keys i-1 and i share, position i begins a level-l cell
// iff d_i < l, so the nodes beginning at i are the levels d_i+1 .. (last level whose parent
// holds > leaf particles).  Counting them per position and scanning gives every node its
// pre-order index directly (pre-order = sorted by (begin, level)); the first child of an
// internal node is the next index and the subtree skip pointer is the first node beginning
// at the node's end.
#include <cuda_runtime.h>
#include <stdint.h>

#include "evol_internal.cuh"

namespace {

constexpr int BB_THREADS = 256;
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int SC_THREADS = 1024;
constexpr int SC_ITEMS = 4;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;

// ---------------------------------------------------------------------------------------
// Root cube
// ---------------------------------------------------------------------------------------
// A non-finite position is flagged as EVOL_ENAN (the min/max below ignore NaN, and every later
// phase keeps its loops bounded on such input, so the step completes and reports the error).
__global__ void k_bbox_partial(int n, const float *__restrict__ x, const float *__restrict__ y,
                               const float *__restrict__ z, float *__restrict__ part, int *err)
{
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float v[3] = {x[i], y[i], z[i]};
        if (!(isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]))) evol_flag(err, EVOL_ENAN);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], v[a]);
            hi[a] = fmaxf(hi[a], v[a]);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    }
    __shared__ float s[BB_THREADS / 32][6];
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0)
        for (int a = 0; a < 3; ++a) { s[w][a] = lo[a]; s[w][3 + a] = hi[a]; }
    __syncthreads();
    if (threadIdx.x < 6) {
        float r = s[0][threadIdx.x];
        for (int k = 1; k < BB_THREADS / 32; ++k)
            r = threadIdx.x < 3 ? fminf(r, s[k][threadIdx.x]) : fmaxf(r, s[k][threadIdx.x]);
        part[blockIdx.x * 6 + threadIdx.x] = r;
    }
}

// corner = per-axis minimum; side = smallest power of two >= extent * (1 + 2^-20) (1 if 0)
__global__ void k_bbox_final(int nparts, const float *__restrict__ part, double *cube, float *fcube)
{
    if (threadIdx.x != 0) return;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = 0; b < nparts; ++b)
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], part[b * 6 + a]);
            hi[a] = fmaxf(hi[a], part[b * 6 + 3 + a]);
        }
    double ext = 0.0;
    for (int a = 0; a < 3; ++a) {
        double e = (double)hi[a] - (double)lo[a];
        ext = e > ext ? e : ext;
    }
    double target = ext * (1.0 + ldexp(1.0, -20));
    double s = 1.0;
    if (target > 0.0) {
        int ex;
        double fr = frexp(target, &ex);
        s = (fr == 0.5) ? ldexp(1.0, ex - 1) : ldexp(1.0, ex);
    }
    for (int a = 0; a < 3; ++a) {
        cube[a] = (double)lo[a];
        fcube[a] = lo[a];
    }
    cube[3] = s;
    fcube[3] = (float)s;
}

// ---------------------------------------------------------------------------------------
// Morton keys: q_a = clamp(floor((x_a - corner_a) * 2^21 / side), 0, 2^21 - 1), FP64 (the scale
// is a power of two, so the result is the exact floor of the double difference), interleaved
// with x the most significant bit of each triplet.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t spread3(uint64_t v)
{
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

// 2^21 / side for a power-of-two side (exact, without a double division)
__device__ __forceinline__ double key_scale(double side)
{
    int e;
    frexp(side, &e);                 // side = 2^(e-1)
    return ldexp(1.0, EVOL_MAXLEVEL + 1 - e);
}

__global__ void k_keys(int n, const float *__restrict__ x, const float *__restrict__ y, const float *__restrict__ z,
                       const double *__restrict__ cube, uint64_t *__restrict__ keys, int32_t *__restrict__ vals)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double scale = key_scale(cube[3]);
    float v[3] = {x[i], y[i], z[i]};
    uint64_t q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double s = floor(__dmul_rn(__dsub_rn((double)v[a], cube[a]), scale));
        s = s < 0.0 ? 0.0 : s;
        s = s > 2097151.0 ? 2097151.0 : s;
        q[a] = (uint64_t)s;
    }
    keys[i] = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
    vals[i] = i;
}

// ---------------------------------------------------------------------------------------
// Exclusive scan of int32 (reduce / top / down-sweep).  Used for the radix histograms and the
// per-position node counts.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t *sh, int32_t &total)
{
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int32_t s = lane < nw ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        if (lane < nw) sh[lane] = s;
    }
    __syncthreads();
    int32_t pre = (w > 0 ? sh[w - 1] : 0) + x - v;
    total = sh[nw - 1];
    __syncthreads();
    return pre;
}

__global__ void k_scan_reduce(int n, const int32_t *__restrict__ in, int32_t *__restrict__ part)
{
    __shared__ int32_t sh[32];
    int base = blockIdx.x * SC_TILE;
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k) {
        int i = base + k * SC_THREADS + threadIdx.x;
        if (i < n) s += in[i];
    }
    int32_t tot;
    block_excl_scan(s, sh, tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void k_scan_top(int nparts, int32_t *__restrict__ part)
{
    __shared__ int32_t sh[32];
    int32_t carry = 0;
    for (int b = 0; b < nparts; b += blockDim.x) {
        int i = b + threadIdx.x;
        int32_t v = i < nparts ? part[i] : 0, tot;
        int32_t pre = block_excl_scan(v, sh, tot);
        if (i < nparts) part[i] = carry + pre;
        carry += tot;
    }
    if (threadIdx.x == 0) part[nparts] = carry;
}

// out may alias in.  out[n] receives the grand total when write_total is set.
__global__ void k_scan_down(int n, const int32_t *in, int32_t *out, const int32_t *__restrict__ part, int nparts,
                            int write_total)
{
    __shared__ int32_t sh[32];
    int base = blockIdx.x * SC_TILE + threadIdx.x * SC_ITEMS;
    int32_t v[SC_ITEMS], s = 0;
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k) {
        int i = base + k;
        v[k] = i < n ? in[i] : 0;
        s += v[k];
    }
    int32_t tot;
    int32_t pre = block_excl_scan(s, sh, tot) + part[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k) {
        int i = base + k;
        if (i < n) out[i] = pre;
        pre += v[k];
    }
    if (write_total && blockIdx.x == 0 && threadIdx.x == 0) out[n] = part[nparts];
}

// ---------------------------------------------------------------------------------------
// Stable LSD radix sort, 8-bit digits, 64-bit keys with int32 values.
// ---------------------------------------------------------------------------------------
__global__ void k_rs_hist(int n, const uint64_t *__restrict__ keys, int shift, int32_t *__restrict__ hist, int nblocks)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int base = blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int k = 0; k < RS_ITEMS; ++k) {
        int i = base + k * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * nblocks + blockIdx.x] = (int32_t)h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(int n, const uint64_t *__restrict__ kin,
                                                           const int32_t *__restrict__ vin, uint64_t *__restrict__ kout,
                                                           int32_t *__restrict__ vout, int shift,
                                                           const int32_t *__restrict__ offs, int nblocks)
{
    constexpr int NW = RS_THREADS / 32;
    __shared__ uint32_t wcnt[NW][256];
    __shared__ uint32_t run[256];
    __shared__ uint32_t goff[256];
    int t = threadIdx.x, lane = t & 31, w = t >> 5;
    goff[t] = (uint32_t)offs[t * nblocks + blockIdx.x];
    run[t] = 0;
    unsigned lt = (1u << lane) - 1u;
    int base = blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ITEMS; ++r) {
#pragma unroll
        for (int k = 0; k < NW; ++k) wcnt[k][t] = 0;
        __syncthreads();
        int i = base + r * RS_THREADS + t;
        bool valid = i < n;
        uint64_t key = valid ? kin[i] : 0ull;
        int32_t val = valid ? vin[i] : 0;
        unsigned d = valid ? ((unsigned)(key >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned rank = __popc(peers & lt);
        if (valid && (__ffs(peers) - 1) == lane) wcnt[w][d] = __popc(peers);
        __syncthreads();
        uint32_t acc = run[t];
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            uint32_t c = wcnt[k][t];
            wcnt[k][t] = acc;
            acc += c;
        }
        run[t] = acc;
        __syncthreads();
        if (valid) {
            uint32_t pos = goff[d] + wcnt[w][d] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------
// Permutation into sorted order.
// ---------------------------------------------------------------------------------------
__global__ void k_permute(int n, int n_gas, const int32_t *__restrict__ perm, const float *__restrict__ x,
                          const float *__restrict__ y, const float *__restrict__ z, const float *__restrict__ vx,
                          const float *__restrict__ vy, const float *__restrict__ vz, const float *__restrict__ m,
                          const float *__restrict__ u, const float *__restrict__ h, const float *__restrict__ eps,
                          float4 *__restrict__ pos, float4 *__restrict__ vel, float *__restrict__ lh,
                          float *__restrict__ le, int32_t *__restrict__ orig, int32_t *__restrict__ inv,
                          const float *__restrict__ pred_dt, const float *__restrict__ pred_acc, int64_t stride,
                          const float *__restrict__ pred_tau)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int j = perm[s];
    bool gas = j < n_gas;
    pos[s] = make_float4(x[j], y[j], z[j], m[j]);
    float4 v = make_float4(vx ? vx[j] : 0.f, vy ? vy[j] : 0.f, vz ? vz[j] : 0.f, (gas && u) ? u[j] : 0.f);
    if (pred_dt || pred_tau) {
        // integrator: the force step sees the velocity and internal energy predicted to the end of
        // the step, v_n + a_n dt and u_n + (du/dt)_n dt (Sect. 4.1); the caller's arrays hold the
        // half-kicked values, so half a step of the previous accelerations (pred_acc: ax | ay | az |
        // du/dt in the caller's order, `stride` apart) is added -- with individual steps each
        // particle's own time since the middle of its step, pred_tau[j]
        const float hdt = pred_tau ? pred_tau[j] : 0.5f * *pred_dt;
        v.x += hdt * pred_acc[j];
        v.y += hdt * pred_acc[stride + j];
        v.z += hdt * pred_acc[2 * stride + j];
        if (gas && u) v.w += hdt * pred_acc[3 * stride + j];
    }
    vel[s] = v;
    lh[s] = (gas && h) ? h[j] : 0.f;
    le[s] = eps ? eps[j] : 0.f;
    orig[s] = j;
    inv[j] = s;
}

// ---------------------------------------------------------------------------------------
// Node construction.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int sys_of_pos(const int32_t *__restrict__ sys_off, int nsys, int s)
{
    // largest k with sys_off[k] <= s
    int lo = 0, hi = nsys;           // sys_off[0] = 0 <= s < sys_off[nsys]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (sys_off[mid] <= s) lo = mid; else hi = mid;
    }
    return lo;
}

// d_i = common leading octal digits of keys i-1 and i; -1 where i starts a system (a forest of
// independent trees, one per system, in one pre-order list).
__global__ void k_lcp(int n, const uint64_t *__restrict__ keys, const int32_t *__restrict__ sys_off, int nsys,
                      int8_t *__restrict__ lcp, int32_t *__restrict__ sys_sorted)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int sy = sys_of_pos(sys_off, nsys, i);
    sys_sorted[i] = sy;
    if (i == sys_off[sy]) {
        lcp[i] = -1;
        return;
    }
    uint64_t x = keys[i - 1] ^ keys[i];
    lcp[i] = x == 0 ? (int8_t)EVOL_MAXLEVEL : (int8_t)((__clzll((long long)x) - 1) / 3);
}

// Does the level-lam run containing position i hold more than `leaf` particles?
__device__ __forceinline__ bool run_exceeds(int n, const int8_t *__restrict__ lcp, int i, int lam, int leaf)
{
    int c = 1;
    for (int t = i; c <= leaf && t > 0 && lcp[t] >= lam; --t) ++c;
    for (int t = i + 1; c <= leaf && t < n && lcp[t] >= lam; ++t) ++c;
    return c > leaf;
}

__device__ __forceinline__ int nodes_at(int n, const int8_t *__restrict__ lcp, int i, int leaf, int &lo)
{
    lo = lcp[i] + 1;                  // 0 where a system starts (lcp = -1)
    int c = 0;
    for (int l = lo; l <= EVOL_MAXLEVEL; ++l) {
        if (l > 0 && !run_exceeds(n, lcp, i, l - 1, leaf)) break;
        ++c;
    }
    return c;
}

__global__ void k_count(int n, const int8_t *__restrict__ lcp, int leaf, int32_t *__restrict__ cnt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo;
    cnt[i] = nodes_at(n, lcp, i, leaf, lo);
}

// end of the level-l run beginning at position i; nend = end of i's system
__device__ __forceinline__ int run_end(int nend, const uint64_t *__restrict__ keys, const int8_t *__restrict__ lcp,
                                       int i, int l, int leaf)
{
    int t = i + 1;
    for (int k = 0; k <= leaf && t < nend; ++k, ++t)
        if (lcp[t] < l) return t;
    if (t >= nend) return nend;
    if (l == 0) return nend;
    int sh = 3 * (EVOL_MAXLEVEL - l);
    uint64_t upper = keys[i] | ((1ull << sh) - 1ull);
    // gallop then bisect for the first index with key > upper
    int lo = t - 1, step = 1, hi = t;
    while (hi < nend && keys[hi] <= upper) {
        lo = hi;
        step <<= 1;
        hi = t - 1 + step;
    }
    if (hi > nend) hi = nend;
    while (hi - lo > 1) {
        int mid = lo + ((hi - lo) >> 1);
        if (keys[mid] <= upper) lo = mid; else hi = mid;
    }
    return hi;
}

__global__ void k_fill(int n, const uint64_t *__restrict__ keys, const int8_t *__restrict__ lcp,
                       const int32_t *__restrict__ sys_off, const int32_t *__restrict__ sys_sorted,
                       const int32_t *__restrict__ base, int leaf, int64_t node_cap, int32_t *__restrict__ nbeg,
                       int32_t *__restrict__ nend, int32_t *__restrict__ nlev, int32_t *__restrict__ nnext,
                       int32_t *__restrict__ nnodes, int *err)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int total = base[n];
    if (i == 0) {
        *nnodes = total > node_cap ? (int)node_cap : total;
        if (total > node_cap) evol_flag(err, EVOL_EOVERFLOW);
    }
    if (i >= n) return;
    int lo;
    int c = nodes_at(n, lcp, i, leaf, lo);
    int b = base[i];
    const int send = sys_off[sys_sorted[i] + 1];
    for (int k = 0; k < c; ++k) {
        int id = b + k;
        if (id >= node_cap) return;
        int l = lo + k;
        int e = run_end(send, keys, lcp, i, l, leaf);
        nbeg[id] = i;
        nend[id] = e;
        nlev[id] = l;
        int nx = e < n ? base[e] : total;
        nnext[id] = nx > node_cap ? (int)node_cap : nx;
    }
}

__global__ void k_link(const int32_t *__restrict__ nnodes, int leaf, const int32_t *__restrict__ nbeg,
                       const int32_t *__restrict__ nend, const int32_t *__restrict__ nlev,
                       const int32_t *__restrict__ nnext, int32_t *__restrict__ nparent, int32_t *__restrict__ nnch,
                       int32_t *__restrict__ narrive, int4 *__restrict__ nI, int4 *__restrict__ nK0,
                       int4 *__restrict__ nK1)
{
    int nn = *nnodes;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < nn; id += gridDim.x * blockDim.x) {
        narrive[id] = 0;
        if (nlev[id] == 0) nparent[id] = -1;     // the root of a system
        int e = nend[id];
        bool internal = (e - nbeg[id] > leaf) && nlev[id] < EVOL_MAXLEVEL;
        int k = 0;
        int ch[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
        if (internal) {
            int c = id + 1;
            while (c < nn && nbeg[c] < e && k < 8) {
                nparent[c] = id;
                ch[k] = c;
                ++k;
                c = nnext[c];
            }
        }
        nK0[id] = make_int4(ch[0], ch[1], ch[2], ch[3]);
        nK1[id] = make_int4(ch[4], ch[5], ch[6], ch[7]);
        nnch[id] = k;
        nI[id] = make_int4(nlev[id] | ((internal ? 0 : 1) << 8), nnext[id], nbeg[id], e);
    }
}

// ---------------------------------------------------------------------------------------
// Moments, leaf-up.  A leaf sums its particles; the last child to finish a parent (atomic
// arrival count) combines the children with the parallel-axis shift of the quadrupole.
//
// FP32 (plain) moments take every position relative to the node's geometric centre (exact in
// double: a dyadic point of the root cube), so the centre of mass and the quadrupole carry
// rounding on the scale of the node, not of the coordinates; a parent combines its children's
// centre-of-mass offsets shifted by the (power-of-two) difference of the two centres, which is
// exact in float.  The absolute centre of mass is formed once, in double, when the node is
// written.  FP64 (mixed) moments use absolute coordinates.
// ---------------------------------------------------------------------------------------
template <typename T>
struct Mom {
    T M, c[3], q[6];       // mass, centre of mass (FP32: offset from the node centre), traceless
                           // quadrupole about it (xx yy zz xy xz yz)
};

struct NodeOut {
    float4 *nA, *nB, *nC, *nQ0, *nQ1, *bmin, *bmax, *coff;
    double *M64, *C64, *Q64;
};

// geometric centre of the node whose first key is key0 at level lev (exact in double)
__device__ __forceinline__ void node_centre(const double *__restrict__ cube, uint64_t key0, int lev, double cg[3])
{
    double side = ldexp(cube[3], -lev);
    uint64_t qa[3] = {0, 0, 0};
    for (int l = 1; l <= lev; ++l) {
        unsigned dg = (unsigned)(key0 >> (3 * (EVOL_MAXLEVEL - l))) & 7u;
        qa[0] = (qa[0] << 1) | ((dg >> 2) & 1u);
        qa[1] = (qa[1] << 1) | ((dg >> 1) & 1u);
        qa[2] = (qa[2] << 1) | (dg & 1u);
    }
    for (int a = 0; a < 3; ++a) cg[a] = cube[a] + ((double)qa[a] + 0.5) * side;
}

template <typename T>
__device__ void write_node(const NodeOut &o, int id, const Mom<T> &mm, float3 lo, float3 hi, int hasgas, int lev,
                           const double cg[3], double side, float theta, bool mixed)
{
    constexpr bool rel = sizeof(T) == sizeof(float);
    double com[3], dd = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double off = rel ? (double)mm.c[a] : (double)mm.c[a] - cg[a];
        com[a] = rel ? cg[a] + off : (double)mm.c[a];
        dd += off * off;
    }
    float delta = (float)sqrt(dd);
    float l = (float)side;
    float ropen = theta > 0.f ? l / theta + delta : INFINITY;
    o.nA[id] = make_float4((float)com[0], (float)com[1], (float)com[2], ropen * ropen);
    float4 bb = make_float4(0.5f * (lo.x + hi.x), 0.5f * (lo.y + hi.y), 0.5f * (lo.z + hi.z), hasgas ? 0.f : -1.f);
    o.nB[id] = bb;
    o.nC[id] = make_float4(0.5f * (hi.x - lo.x), 0.5f * (hi.y - lo.y), 0.5f * (hi.z - lo.z), 0.f);
    o.nQ0[id] = make_float4((float)mm.q[0], (float)mm.q[1], (float)mm.q[2], (float)mm.M);
    o.nQ1[id] = make_float4((float)mm.q[3], (float)mm.q[4], (float)mm.q[5], delta);
    o.bmin[id] = make_float4(lo.x, lo.y, lo.z, (float)hasgas);
    o.bmax[id] = make_float4(hi.x, hi.y, hi.z, 0.f);
    if (rel) o.coff[id] = make_float4((float)mm.c[0], (float)mm.c[1], (float)mm.c[2], (float)mm.M);
    if (mixed) {
        o.M64[id] = (double)mm.M;
        for (int a = 0; a < 3; ++a) o.C64[3 * id + a] = (double)mm.c[a];
        for (int a = 0; a < 6; ++a) o.Q64[6 * id + a] = (double)mm.q[a];
    }
}

template <typename T>
__device__ void leaf_moments(int b, int e, int n_gas, const float4 *__restrict__ pos, const int32_t *__restrict__ orig,
                             const double cg[3], Mom<T> &mm, float3 &lo, float3 &hi, int &hasgas)
{
    constexpr bool rel = sizeof(T) == sizeof(float);
    T M = 0, s0 = 0, s1 = 0, s2 = 0;
    lo = make_float3(INFINITY, INFINITY, INFINITY);
    hi = make_float3(-INFINITY, -INFINITY, -INFINITY);
    hasgas = 0;
    auto coord = [&](float x, int a) -> T { return rel ? (T)((double)x - cg[a]) : (T)x; };
    for (int s = b; s < e; ++s) {
        float4 p = pos[s];
        M += (T)p.w;
        s0 += (T)p.w * coord(p.x, 0);
        s1 += (T)p.w * coord(p.y, 1);
        s2 += (T)p.w * coord(p.z, 2);
        lo.x = fminf(lo.x, p.x); lo.y = fminf(lo.y, p.y); lo.z = fminf(lo.z, p.z);
        hi.x = fmaxf(hi.x, p.x); hi.y = fmaxf(hi.y, p.y); hi.z = fmaxf(hi.z, p.z);
        if (orig[s] < n_gas) hasgas = 1;
    }
    mm.M = M;
    if (M > 0) {
        mm.c[0] = s0 / M; mm.c[1] = s1 / M; mm.c[2] = s2 / M;
    } else {
        mm.c[0] = coord(0.5f * (lo.x + hi.x), 0);
        mm.c[1] = coord(0.5f * (lo.y + hi.y), 1);
        mm.c[2] = coord(0.5f * (lo.z + hi.z), 2);
    }
    for (int a = 0; a < 6; ++a) mm.q[a] = 0;
    for (int s = b; s < e; ++s) {
        float4 p = pos[s];
        T d0 = coord(p.x, 0) - mm.c[0], d1 = coord(p.y, 1) - mm.c[1], d2 = coord(p.z, 2) - mm.c[2];
        T r2 = d0 * d0 + d1 * d1 + d2 * d2, w = (T)p.w;
        mm.q[0] += w * (3 * d0 * d0 - r2);
        mm.q[1] += w * (3 * d1 * d1 - r2);
        mm.q[2] += w * (3 * d2 * d2 - r2);
        mm.q[3] += w * 3 * d0 * d1;
        mm.q[4] += w * 3 * d0 * d2;
        mm.q[5] += w * 3 * d1 * d2;
    }
}

// child c's moments; FP32: its centre-of-mass offset re-expressed about the parent's centre.  A
// child cell is one level below its parent (a cell with one non-empty octant still has that octant
// as its child), so its centre is the parent's centre moved by a quarter of the parent's side
// along each axis, in the direction the child's octal digit gives: a power of two, exact in float.
template <typename T>
__device__ void load_child(const NodeOut &o, int c, float side_p, const uint64_t *__restrict__ keys,
                           const int32_t *__restrict__ nbeg, const int32_t *__restrict__ nlev, Mom<T> &mm,
                           float3 &lo, float3 &hi, int &hasgas, bool mixed)
{
    constexpr bool rel = sizeof(T) == sizeof(float);
    float4 bl = __ldcg(&o.bmin[c]), bh = __ldcg(&o.bmax[c]);
    lo = make_float3(bl.x, bl.y, bl.z);
    hi = make_float3(bh.x, bh.y, bh.z);
    hasgas = bl.w != 0.f;
    float4 Q0, Q1;
    if (mixed) {
        mm.M = (T)__ldcg(&o.M64[c]);
        for (int a = 0; a < 3; ++a) mm.c[a] = (T)__ldcg(&o.C64[3 * c + a]);
        for (int a = 0; a < 6; ++a) mm.q[a] = (T)__ldcg(&o.Q64[6 * c + a]);
        return;
    }
    Q0 = __ldcg(&o.nQ0[c]);
    Q1 = __ldcg(&o.nQ1[c]);
    mm.q[0] = (T)Q0.x; mm.q[1] = (T)Q0.y; mm.q[2] = (T)Q0.z;
    mm.q[3] = (T)Q1.x; mm.q[4] = (T)Q1.y; mm.q[5] = (T)Q1.z;
    if (rel) {
        const float4 co = __ldcg(&o.coff[c]);
        const int lc = __ldcg(&nlev[c]);
        const unsigned dg = (unsigned)(__ldcg(&keys[__ldcg(&nbeg[c])]) >> (3 * (EVOL_MAXLEVEL - lc))) & 7u;
        const float q = 0.25f * side_p;
        mm.M = (T)co.w;
        mm.c[0] = (T)co.x + (T)((dg & 4u) ? q : -q);
        mm.c[1] = (T)co.y + (T)((dg & 2u) ? q : -q);
        mm.c[2] = (T)co.z + (T)((dg & 1u) ? q : -q);
    } else {
        const float4 A = __ldcg(&o.nA[c]);
        mm.M = (T)Q0.w;
        mm.c[0] = (T)A.x; mm.c[1] = (T)A.y; mm.c[2] = (T)A.z;
    }
}

template <typename T>
__device__ void combine(const NodeOut &o, int id, int nch, const int32_t *__restrict__ nnext, const double cgp[3],
                        float side_p, const uint64_t *__restrict__ keys, const int32_t *__restrict__ nbeg,
                        const int32_t *__restrict__ nlev, Mom<T> &mm, float3 &lo, float3 &hi, int &hasgas, bool mixed)
{
    constexpr bool rel = sizeof(T) == sizeof(float);
    Mom<T> ch[8];
    lo = make_float3(INFINITY, INFINITY, INFINITY);
    hi = make_float3(-INFINITY, -INFINITY, -INFINITY);
    hasgas = 0;
    T M = 0, s[3] = {0, 0, 0};
    int c = id + 1;
    for (int k = 0; k < nch; ++k) {
        float3 cl, chh;
        int cg;
        load_child(o, c, side_p, keys, nbeg, nlev, ch[k], cl, chh, cg, mixed);
        lo.x = fminf(lo.x, cl.x); lo.y = fminf(lo.y, cl.y); lo.z = fminf(lo.z, cl.z);
        hi.x = fmaxf(hi.x, chh.x); hi.y = fmaxf(hi.y, chh.y); hi.z = fmaxf(hi.z, chh.z);
        hasgas |= cg;
        M += ch[k].M;
        for (int a = 0; a < 3; ++a) s[a] += ch[k].M * ch[k].c[a];
        c = nnext[c];
    }
    mm.M = M;
    float cen[3] = {0.5f * (lo.x + hi.x), 0.5f * (lo.y + hi.y), 0.5f * (lo.z + hi.z)};
    for (int a = 0; a < 3; ++a) mm.c[a] = M > 0 ? s[a] / M : (rel ? (T)((double)cen[a] - cgp[a]) : (T)cen[a]);
    for (int a = 0; a < 6; ++a) mm.q[a] = 0;
    for (int j = 0; j < nch; ++j) {
        T d0 = ch[j].c[0] - mm.c[0], d1 = ch[j].c[1] - mm.c[1], d2 = ch[j].c[2] - mm.c[2];
        T r2 = d0 * d0 + d1 * d1 + d2 * d2, w = ch[j].M;
        mm.q[0] += ch[j].q[0] + w * (3 * d0 * d0 - r2);
        mm.q[1] += ch[j].q[1] + w * (3 * d1 * d1 - r2);
        mm.q[2] += ch[j].q[2] + w * (3 * d2 * d2 - r2);
        mm.q[3] += ch[j].q[3] + w * 3 * d0 * d1;
        mm.q[4] += ch[j].q[4] + w * 3 * d0 * d2;
        mm.q[5] += ch[j].q[5] + w * 3 * d1 * d2;
    }
}

template <typename T>
__global__ void k_moments(const int32_t *__restrict__ nnodes, int n_gas, const int32_t *__restrict__ nbeg,
                          const int32_t *__restrict__ nend, const int32_t *__restrict__ nlev,
                          const int32_t *__restrict__ nnext, const int32_t *__restrict__ nparent,
                          const int32_t *__restrict__ nnch, int32_t *__restrict__ narrive,
                          const float4 *__restrict__ pos, const int32_t *__restrict__ orig,
                          const uint64_t *__restrict__ keys, const double *__restrict__ cube,
                          const int32_t *__restrict__ sys_sorted, float theta, NodeOut o, int mixed, int *err)
{
    int nn = *nnodes;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < nn; id += gridDim.x * blockDim.x) {
        if (nnch[id] != 0) continue;
        Mom<T> mm;
        float3 lo, hi;
        int hg;
        const double *cb = cube + 4 * sys_sorted[nbeg[id]];
        double cg[3];
        node_centre(cb, keys[nbeg[id]], nlev[id], cg);
        leaf_moments<T>(nbeg[id], nend[id], n_gas, pos, orig, cg, mm, lo, hi, hg);
        write_node<T>(o, id, mm, lo, hi, hg, nlev[id], cg, ldexp(cb[3], -nlev[id]), theta, mixed != 0);
        __threadfence();
        int p = nparent[id];
        for (int climb = 0; p >= 0 && p < nn; ++climb) {
            if (climb > EVOL_MAXLEVEL + 1) {     // deeper than the tree can be: corrupt parents
                evol_flag(err, EVOL_ETIMEOUT);
                break;
            }
            int old = atomicAdd(&narrive[p], 1);
            if (old != nnch[p] - 1) break;
            __threadfence();
            const double *cbp = cube + 4 * sys_sorted[nbeg[p]];
            double cgp[3];
            node_centre(cbp, keys[nbeg[p]], nlev[p], cgp);
            combine<T>(o, p, nnch[p], nnext, cgp, (float)ldexp(cbp[3], -nlev[p]), keys, nbeg, nlev, mm, lo, hi, hg,
                       mixed != 0);
            write_node<T>(o, p, mm, lo, hi, hg, nlev[p], cgp, ldexp(cbp[3], -nlev[p]), theta, mixed != 0);
            __threadfence();
            p = nparent[p];
        }
    }
}

// Node maxima of 2 eps (all particles) and 2 h (gas), leaf-up like the moments.
__device__ __forceinline__ void leaf_len(int b, int e, int n_gas, const int32_t *__restrict__ orig,
                                         const float *__restrict__ le, const float *__restrict__ lh, float &em,
                                         float &hm)
{
    em = 0.f;
    hm = -1.f;
    for (int s = b; s < e; ++s) {
        em = fmaxf(em, le[s]);
        if (orig[s] < n_gas) hm = fmaxf(hm, lh[s]);
    }
}

__global__ void k_node_lengths(const int32_t *__restrict__ nnodes, int n_gas, const int32_t *__restrict__ nbeg,
                               const int32_t *__restrict__ nend, const int32_t *__restrict__ nnext,
                               const int32_t *__restrict__ nparent, const int32_t *__restrict__ nnch,
                               int32_t *__restrict__ narrive, const int32_t *__restrict__ orig,
                               const float *__restrict__ le, const float *__restrict__ lh, float4 *nB, float4 *nC,
                               int *err)
{
    int nn = *nnodes;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < nn; id += gridDim.x * blockDim.x) {
        if (nnch[id] != 0) continue;
        float em, hm;
        leaf_len(nbeg[id], nend[id], n_gas, orig, le, lh, em, hm);
        nC[id].w = 2.f * em;
        nB[id].w = hm >= 0.f ? 2.f * hm : -1.f;
        __threadfence();
        int p = nparent[id];
        for (int climb = 0; p >= 0 && p < nn; ++climb) {
            if (climb > EVOL_MAXLEVEL + 1) {     // deeper than the tree can be: corrupt parents
                evol_flag(err, EVOL_ETIMEOUT);
                break;
            }
            int old = atomicAdd(&narrive[p], 1);
            if (old != nnch[p] - 1) break;
            __threadfence();
            float e2 = 0.f, h2 = -1.f;
            for (int c = p + 1; c < nn && __ldcg(&nbeg[c]) < nend[p]; c = __ldcg(&nnext[c])) {
                e2 = fmaxf(e2, __ldcg(&nC[c].w));
                h2 = fmaxf(h2, __ldcg(&nB[c].w));
            }
            nC[p].w = e2;
            nB[p].w = h2;
            __threadfence();
            p = nparent[p];
        }
    }
}

// ---- several independent systems (batched): per-system cube and keys ----------------------
__global__ void k_set_single(int n, int32_t *sys_off)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        sys_off[0] = 0;
        sys_off[1] = n;
    }
}

// one block per system: its cube from its own particles
__global__ void k_bbox_sys(const int32_t *__restrict__ sys_off, const float *__restrict__ x,
                           const float *__restrict__ y, const float *__restrict__ z, double *cube, float *fcube,
                           int *err)
{
    const int k = blockIdx.x;
    const int b = sys_off[k], e = sys_off[k + 1];
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = b + threadIdx.x; i < e; i += blockDim.x) {
        float v[3] = {x[i], y[i], z[i]};
        if (!(isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]))) evol_flag(err, EVOL_ENAN);
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], v[a]);
            hi[a] = fmaxf(hi[a], v[a]);
        }
    }
    for (int a = 0; a < 3; ++a)
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    __shared__ float sred[BB_THREADS / 32][6];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0)
        for (int a = 0; a < 3; ++a) {
            sred[w][a] = lo[a];
            sred[w][3 + a] = hi[a];
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ext = 0.0;
        float L[3], H[3];
        for (int a = 0; a < 3; ++a) {
            L[a] = sred[0][a];
            H[a] = sred[0][3 + a];
            for (int q = 1; q < BB_THREADS / 32; ++q) {
                L[a] = fminf(L[a], sred[q][a]);
                H[a] = fmaxf(H[a], sred[q][3 + a]);
            }
            double ee = (double)H[a] - (double)L[a];
            ext = ee > ext ? ee : ext;
        }
        double target = ext * (1.0 + ldexp(1.0, -20)), side = 1.0;
        if (target > 0.0) {
            int ex;
            double fr = frexp(target, &ex);
            side = (fr == 0.5) ? ldexp(1.0, ex - 1) : ldexp(1.0, ex);
        }
        for (int a = 0; a < 3; ++a) {
            cube[4 * k + a] = (double)L[a];
            fcube[4 * k + a] = L[a];
        }
        cube[4 * k + 3] = side;
        fcube[4 * k + 3] = (float)side;
    }
}

__device__ __forceinline__ uint64_t key_of(float x, float y, float z, const double *__restrict__ cb)
{
    const double scale = key_scale(cb[3]);
    const float v[3] = {x, y, z};
    uint64_t q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double t = floor(__dmul_rn(__dsub_rn((double)v[a], cb[a]), scale));
        t = t < 0.0 ? 0.0 : (t > 2097151.0 ? 2097151.0 : t);
        q[a] = (uint64_t)t;
    }
    return (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
}

// keys in the caller's order, each relative to its own system's cube
__global__ void k_keys_sys(int n, const float *__restrict__ x, const float *__restrict__ y,
                           const float *__restrict__ z, const int32_t *__restrict__ sys_off, int nsys,
                           const double *__restrict__ cube, uint64_t *__restrict__ keys, int32_t *__restrict__ vals)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int sy = sys_of_pos(sys_off, nsys, i);
    keys[i] = key_of(x[i], y[i], z[i], cube + 4 * sy);
    vals[i] = i;
}

// system id of the particle at each position of the current order (digit source of the last passes)
__global__ void k_gather_sys(int n, const int32_t *__restrict__ vals, const int32_t *__restrict__ sys_off, int nsys,
                             uint64_t *__restrict__ skey)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    skey[i] = (uint64_t)sys_of_pos(sys_off, nsys, vals[i]);
}

// Morton keys again, in the final order (the system passes carried only the system digit)
__global__ void k_keys_sorted(int n, const float *__restrict__ x, const float *__restrict__ y,
                              const float *__restrict__ z, const int32_t *__restrict__ vals,
                              const int32_t *__restrict__ sys_off, int nsys, const double *__restrict__ cube,
                              uint64_t *__restrict__ keys, int32_t *__restrict__ vals_out)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int j = vals[s];
    const int sy = sys_of_pos(sys_off, nsys, j);
    keys[s] = key_of(x[j], y[j], z[j], cube + 4 * sy);
    if (vals_out) vals_out[s] = j;
}

__global__ void k_sys_root(int nsys, const int32_t *__restrict__ sys_off, const int32_t *__restrict__ base,
                           int32_t *__restrict__ sys_root)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nsys) sys_root[k] = base[sys_off[k]];
}

__global__ void k_zero_i32(const int32_t *__restrict__ nnodes, int32_t *a)
{
    int nn = *nnodes;
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < nn; id += gridDim.x * blockDim.x) a[id] = 0;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------
static int scan_i32(evol_ctx *c, int n, const int32_t *in, int32_t *out, int write_total)
{
    int nparts = (n + SC_TILE - 1) / SC_TILE;
    if (nparts < 1) nparts = 1;
    k_scan_reduce<<<nparts, SC_THREADS, 0, c->stream>>>(n, in, c->d.scan_part);
    k_scan_top<<<1, SC_THREADS, 0, c->stream>>>(nparts, c->d.scan_part);
    k_scan_down<<<nparts, SC_THREADS, 0, c->stream>>>(n, in, out, c->d.scan_part, nparts, write_total);
    return evol_cuda_ok(cudaGetLastError());
}

namespace {
__global__ void k_active_flags(int n, const int32_t *__restrict__ orig, const int32_t *__restrict__ bact,
                               int32_t *__restrict__ actf)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) actf[s] = bact[orig[s]];
}

__global__ void k_active_scatter(int n, const int32_t *__restrict__ actf, const int32_t *__restrict__ acts,
                                 int32_t *__restrict__ act)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n && actf[s]) act[acts[s]] = s;
}
}  // namespace

// The active list of an individual-time-step system step: the sorted positions of the flagged
// particles in ascending order (so that consecutive entries stay close in space), and their
// number at d.acts[n].
int evol_launch_active_list(evol_ctx *c, int n)
{
    evol_dev &d = c->d;
    int tb = 256, gb = (n + tb - 1) / tb;
    k_active_flags<<<gb, tb, 0, c->stream>>>(n, d.orig, d.bact, d.actf);
    int rc = scan_i32(c, n, d.actf, d.acts, 1);
    if (rc) return rc;
    k_active_scatter<<<gb, tb, 0, c->stream>>>(n, d.actf, d.acts, d.act);
    return evol_cuda_ok(cudaGetLastError());
}

int evol_launch_build(evol_ctx *c, const evol_particles *p, const evol_params *prm)
{
    evol_dev &d = c->d;
    int n = (int)p->n;
    const int nsys = c->nsys > 0 ? c->nsys : 1;
    int leaf = prm->leaf_size > 0 ? prm->leaf_size : 8;
    cudaStream_t st = c->stream;
    int tb = 256, gb = (n + tb - 1) / tb;
    if (nsys == 1) {
        int nb = (int)c->bbox_blocks;
        k_set_single<<<1, 32, 0, st>>>(n, d.sys_off);
        k_bbox_partial<<<nb, BB_THREADS, 0, st>>>(n, p->x, p->y, p->z, d.bbox_part, d.err);
        k_bbox_final<<<1, 32, 0, st>>>(nb, d.bbox_part, d.cube, d.fcube);
        k_keys<<<gb, tb, 0, st>>>(n, p->x, p->y, p->z, d.cube, d.keys_a, d.vals_a);
    } else {
        // the offsets were copied into d.sys_off by the caller of this launcher
        k_bbox_sys<<<nsys, BB_THREADS, 0, st>>>(d.sys_off, p->x, p->y, p->z, d.cube, d.fcube, d.err);
        k_keys_sys<<<gb, tb, 0, st>>>(n, p->x, p->y, p->z, d.sys_off, nsys, d.cube, d.keys_a, d.vals_a);
    }
    int rsb = (n + RS_TILE - 1) / RS_TILE;
    uint64_t *ka = d.keys_a, *kb = d.keys_b;
    int32_t *va = d.vals_a, *vb = d.vals_b;
    for (int shift = 0; shift < 64; shift += 8) {
        k_rs_hist<<<rsb, RS_THREADS, 0, st>>>(n, ka, shift, (int32_t *)d.hist, rsb);
        int rc = scan_i32(c, 256 * rsb, (int32_t *)d.hist, (int32_t *)d.hist, 0);
        if (rc) return rc;
        k_rs_scatter<<<rsb, RS_THREADS, 0, st>>>(n, ka, va, kb, vb, shift, (int32_t *)d.hist, rsb);
        uint64_t *tk = ka; ka = kb; kb = tk;
        int32_t *tv = va; va = vb; vb = tv;
    }
    // 8 passes: sorted keys and permutation are back in keys_a / vals_a
    if (nsys > 1) {
        // stable passes on the system id make the order (system, key); then the keys are recomputed
        k_gather_sys<<<gb, tb, 0, st>>>(n, d.vals_a, d.sys_off, nsys, d.keys_b);
        ka = d.keys_b; kb = d.keys_a; va = d.vals_a; vb = d.vals_b;
        for (int shift = 0; (1ll << shift) < (long long)nsys; shift += 8) {
            k_rs_hist<<<rsb, RS_THREADS, 0, st>>>(n, ka, shift, (int32_t *)d.hist, rsb);
            int rc = scan_i32(c, 256 * rsb, (int32_t *)d.hist, (int32_t *)d.hist, 0);
            if (rc) return rc;
            k_rs_scatter<<<rsb, RS_THREADS, 0, st>>>(n, ka, va, kb, vb, shift, (int32_t *)d.hist, rsb);
            uint64_t *tk = ka; ka = kb; kb = tk;
            int32_t *tv = va; va = vb; vb = tv;
        }
        // va holds the final permutation; rebuild keys_a / vals_a from it
        k_keys_sorted<<<gb, tb, 0, st>>>(n, p->x, p->y, p->z, va, d.sys_off, nsys, d.cube, d.keys_a,
                                         va == d.vals_a ? nullptr : d.vals_a);
    }
    k_permute<<<gb, tb, 0, st>>>(n, (int)p->n_gas, d.vals_a, p->x, p->y, p->z, p->vx, p->vy, p->vz, p->m, p->u,
                                 p->h, p->eps, d.pos, d.vel, d.len_h, d.len_eps, d.orig, d.inv,
                                 c->pred_dt, c->kdk_acc, c->cap, c->pred_tau);
    k_lcp<<<gb, tb, 0, st>>>(n, d.keys_a, d.sys_off, nsys, d.lcp, d.sys_sorted);
    k_count<<<gb, tb, 0, st>>>(n, d.lcp, leaf, d.cnt);
    int rc = scan_i32(c, n, d.cnt, d.base, 1);
    if (rc) return rc;
    k_fill<<<gb, tb, 0, st>>>(n, d.keys_a, d.lcp, d.sys_off, d.sys_sorted, d.base, leaf, c->node_cap, d.nbeg, d.nend,
                              d.nlev, d.nnext, d.nnodes, d.err);
    k_sys_root<<<(nsys + 255) / 256, 256, 0, st>>>(nsys, d.sys_off, d.base, d.sys_root);
    int ng = c->num_sms * 8;
    k_link<<<ng, 256, 0, st>>>(d.nnodes, leaf, d.nbeg, d.nend, d.nlev, d.nnext, d.nparent, d.nnch, d.narrive, d.nI,
                               d.nK0, d.nK1);
    NodeOut o{d.nA, d.nB, d.nC, d.nQ0, d.nQ1, d.nBmin, d.nBmax, d.nCoff, d.nM64, d.nC64, d.nQ64};
    float theta = prm->theta;
    if (prm->precision == EVOL_FP32_MIXED)
        k_moments<double><<<ng, 128, 0, st>>>(d.nnodes, (int)p->n_gas, d.nbeg, d.nend, d.nlev, d.nnext, d.nparent,
                                              d.nnch, d.narrive, d.pos, d.orig, d.keys_a, d.cube, d.sys_sorted, theta,
                                              o, 1, d.err);
    else
        k_moments<float><<<ng, 128, 0, st>>>(d.nnodes, (int)p->n_gas, d.nbeg, d.nend, d.nlev, d.nnext, d.nparent,
                                             d.nnch, d.narrive, d.pos, d.orig, d.keys_a, d.cube, d.sys_sorted, theta,
                                             o, 0, d.err);
    return evol_cuda_ok(cudaGetLastError());
}

int evol_launch_node_lengths(evol_ctx *c, const evol_params *prm, int n_gas)
{
    evol_dev &d = c->d;
    int ng = c->num_sms * 8;
    (void)prm;
    k_zero_i32<<<ng, 256, 0, c->stream>>>(d.nnodes, d.narrive);
    k_node_lengths<<<ng, 128, 0, c->stream>>>(d.nnodes, n_gas, d.nbeg, d.nend, d.nnext, d.nparent,
                                              d.nnch, d.narrive, d.orig, d.len_eps, d.len_h, d.nB, d.nC, d.err);
    return evol_cuda_ok(cudaGetLastError());
}
