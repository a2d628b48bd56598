// Allocation-free variant of the key + sort stage of the tree build: root cube, 63-bit Morton
// keys and the stable radix sort, done by one thread block whose scratch lives in a file-scope
// static device array instead of memory obtained from cudaMalloc.
//
// Who needs this: callers that may not allocate device memory at the point where they call
// the library -- for example code running inside a host callback or a framework hook that must
// not re-enter the device allocator, or a process whose device memory is partitioned once at
// start-up and may not grow.  Such callers pass their own input and output buffers and this
// entry point allocates nothing: no cudaMalloc, no cudaFree, no library routine that allocates.
//
// The static array belongs to this file's device module.  The CUDA runtime loads a module on a
// device lazily, at its first use there, and loading it is what places the array (and the
// kernel's code) in device memory.  So the set-up -- loading the module and looking up the
// array's device address with cudaGetSymbolAddress, with the device current -- is done by a
// call with n == 0 (which launches nothing), by evol_create for its device, or else by the first
// call on each device.  A caller that may not allocate later makes the n == 0 call at start-up,
// before any stream capture; after a cudaDeviceReset it makes it again (the reset unloads the
// module and with it the array).  All calls share the one array, which keeps whatever the
// previous call left in it; calls whose executions overlap on the GPU therefore race and must be
// ordered by the caller (for example by using one stream).
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "evol_internal.cuh"

namespace {

constexpr int NA_THREADS = 1024;
constexpr int NA_WARPS = NA_THREADS / 32;
constexpr int NA_MAX_DEVICES = 64;

// Scratch: the ping-pong keys and indices of the sort.  Every byte is written before it is read
// within a call, so nothing has to be cleared between calls.
constexpr size_t NA_SCRATCH_BYTES = (size_t)EVOL_NOALLOC_MAX_N * (sizeof(uint64_t) + sizeof(int32_t));
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_SCRATCH_BYTES];

std::mutex g_setup_mutex;
void *g_scratch_addr[NA_MAX_DEVICES];      // device address of g_noalloc_scratch, per device
bool g_scratch_ready[NA_MAX_DEVICES];

__device__ __forceinline__ uint64_t na_spread3(uint64_t v)
{
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

// One block.  keys/perm (caller buffers) and the scratch pair serve as the sort's ping-pong
// buffers; 8 passes leave the result in the caller's buffers.
__global__ void __launch_bounds__(NA_THREADS) k_sort_keys_single_block(int n, const float *__restrict__ x,
                                                                       const float *__restrict__ y,
                                                                       const float *__restrict__ z,
                                                                       uint64_t *keys, int32_t *perm,
                                                                       unsigned char *scratch, double *cube_out)
{
    __shared__ float s_red[NA_WARPS][6];
    __shared__ double s_cube[4];
    __shared__ uint32_t s_hist[256];
    __shared__ uint32_t s_off[256];
    __shared__ uint32_t s_wcnt[NA_WARPS][256];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    uint64_t *kb = reinterpret_cast<uint64_t *>(scratch);
    int32_t *vb = reinterpret_cast<int32_t *>(scratch + (size_t)EVOL_NOALLOC_MAX_N * sizeof(uint64_t));

    // root cube: per-axis min corner, side = smallest power of two >= extent (1 + 2^-20)
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = t; i < n; i += NA_THREADS) {
        float v[3] = {x[i], y[i], z[i]};
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
    if (lane == 0)
        for (int a = 0; a < 3; ++a) {
            s_red[w][a] = lo[a];
            s_red[w][3 + a] = hi[a];
        }
    __syncthreads();
    if (t == 0) {
        float l[3], h[3];
        for (int a = 0; a < 3; ++a) {
            l[a] = s_red[0][a];
            h[a] = s_red[0][3 + a];
            for (int k = 1; k < NA_WARPS; ++k) {
                l[a] = fminf(l[a], s_red[k][a]);
                h[a] = fmaxf(h[a], s_red[k][3 + a]);
            }
        }
        double ext = 0.0;
        for (int a = 0; a < 3; ++a) {
            double e = (double)h[a] - (double)l[a];
            ext = e > ext ? e : ext;
        }
        double target = ext * (1.0 + ldexp(1.0, -20)), side = 1.0;
        if (target > 0.0) {
            int ex;
            double fr = frexp(target, &ex);
            side = (fr == 0.5) ? ldexp(1.0, ex - 1) : ldexp(1.0, ex);
        }
        for (int a = 0; a < 3; ++a) s_cube[a] = (double)l[a];
        s_cube[3] = side;
        if (cube_out)
            for (int a = 0; a < 4; ++a) cube_out[a] = s_cube[a];
    }
    __syncthreads();

    // keys into the caller's buffers (pass 0 reads them)
    const double scale = ldexp(1.0, EVOL_MAXLEVEL) / s_cube[3];
    for (int i = t; i < n; i += NA_THREADS) {
        float v[3] = {x[i], y[i], z[i]};
        uint64_t q[3];
        for (int a = 0; a < 3; ++a) {
            double s = floor(__dmul_rn(__dsub_rn((double)v[a], s_cube[a]), scale));
            s = s < 0.0 ? 0.0 : (s > 2097151.0 ? 2097151.0 : s);
            q[a] = (uint64_t)s;
        }
        keys[i] = (na_spread3(q[0]) << 2) | (na_spread3(q[1]) << 1) | na_spread3(q[2]);
        perm[i] = i;
    }
    __syncthreads();

    // stable LSD radix sort, 8 passes of 8 bits
    const unsigned lt = (1u << lane) - 1u;
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 8 * pass;
        uint64_t *ksrc = (pass & 1) ? kb : keys, *kdst = (pass & 1) ? keys : kb;
        int32_t *vsrc = (pass & 1) ? vb : perm, *vdst = (pass & 1) ? perm : vb;
        if (t < 256) s_hist[t] = 0;
        __syncthreads();
        for (int i = t; i < n; i += NA_THREADS) atomicAdd(&s_hist[(unsigned)(ksrc[i] >> shift) & 255u], 1u);
        __syncthreads();
        if (t == 0) {
            uint32_t acc = 0;
            for (int d = 0; d < 256; ++d) {
                s_off[d] = acc;
                acc += s_hist[d];
            }
        }
        __syncthreads();
        for (int base = 0; base < n; base += NA_THREADS) {
            for (int d = t; d < NA_WARPS * 256; d += NA_THREADS) (&s_wcnt[0][0])[d] = 0;
            __syncthreads();
            const int i = base + t;
            const bool valid = i < n;
            const uint64_t key = valid ? ksrc[i] : 0ull;
            const int32_t val = valid ? vsrc[i] : 0;
            const unsigned dg = valid ? ((unsigned)(key >> shift) & 255u) : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, dg);
            const unsigned rank = __popc(peers & lt);
            if (valid && (__ffs(peers) - 1) == lane) s_wcnt[w][dg] = __popc(peers);
            __syncthreads();
            if (t < 256) {
                uint32_t acc = s_off[t];
                for (int k = 0; k < NA_WARPS; ++k) {
                    uint32_t c = s_wcnt[k][t];
                    s_wcnt[k][t] = acc;
                    acc += c;
                }
                s_off[t] = acc;
            }
            __syncthreads();
            if (valid) {
                const uint32_t pos = s_wcnt[w][dg] + rank;
                kdst[pos] = key;
                vdst[pos] = val;
            }
            __syncthreads();
        }
    }
}

// Device address of the static scratch on the current device, looked up once per device (or
// again when `refresh` is set).
int scratch_for_current_device(void **out, bool refresh)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return EVOL_ECUDA;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return EVOL_EINVAL;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ready[dev] || refresh) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return EVOL_ECUDA;
        }
        g_scratch_addr[dev] = p;
        g_scratch_ready[dev] = true;
    }
    *out = g_scratch_addr[dev];
    return EVOL_OK;
}

}  // namespace

// Set-up for the current device (module load + address lookup); evol_create calls it.
int evol_noalloc_setup_current_device()
{
    void *p = nullptr;
    return scratch_for_current_device(&p, false);
}

extern "C" int evol_sort_keys_noalloc(int64_t n, const float *x, const float *y, const float *z, uint64_t *keys_sorted,
                                      int32_t *perm, double *cube, void *stream)
{
    if (n < 0 || n > EVOL_NOALLOC_MAX_N) return EVOL_EINVAL;
    void *scratch = nullptr;
    if (n == 0) return scratch_for_current_device(&scratch, true);     // set-up call: nothing launched
    if (!x || !y || !z || !keys_sorted || !perm) return EVOL_EINVAL;
    int rc = scratch_for_current_device(&scratch, false);
    if (rc) return rc;
    k_sort_keys_single_block<<<1, NA_THREADS, 0, (cudaStream_t)stream>>>(
        (int)n, x, y, z, keys_sorted, perm, static_cast<unsigned char *>(scratch), cube);
    return cudaGetLastError() == cudaSuccess ? EVOL_OK : EVOL_ECUDA;
}
