// C ABI of the force-step library (include/evol.h): context management, argument checks,
// phase sequencing, CUDA-graph capture of the whole step, host-buffer step, diagnostics and
// debug copies.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "evol_internal.cuh"

int evol_launch_pack(evol_ctx *c, const evol_particles *p, const evol_params *prm, int do_grav, int do_sph);
int evol_launch_unpermute_ex(evol_ctx *c, const evol_particles *p, const evol_outputs *o, int what, int add_acc);
int evol_lengths_warps_per_block();
int evol_lengths_list_cap();
int evol_launch_kick(evol_ctx *c, const evol_particles *p, const evol_params *prm, float half_dt, const float *ax,
                     const float *ay, const float *az, const float *dudt, const float *dalpha, const float *dalpha_u);
int evol_launch_drift(evol_ctx *c, const evol_particles *p, const evol_params *prm, float dt);
int evol_noalloc_setup_current_device();

namespace {

constexpr int64_t NODE_FACTOR = 3;       // node capacity = 3 * particles + 64
constexpr int64_t WSTACK_CAP = 4096;     // traversal stack entries per warp in the force walk
constexpr int NSYS_CAP = 65536;          // independent systems per batched call

template <typename T>
int dalloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void **)p, count * sizeof(T)) == cudaSuccess ? EVOL_OK : EVOL_ENOMEM;
}

void free_all(evol_ctx *c)
{
    evol_dev &d = c->d;
    void *ptrs[] = {d.pos, d.vel, d.grav, d.hydro, d.snd, d.vah, d.orig, d.inv, d.divv_h, d.divv_e, d.mumax, d.dt, d.time, d.len_h, d.len_eps, d.nh, d.omega,
                    d.diss, d.curlv_h, d.vsig, d.lapu, d.dalpha, d.dalpha_u, d.tb, d.te, d.bact, d.pred_tau,
                    d.pers, d.actf, d.acts, d.act, d.sg_acc, d.sg_front, d.sg_info, d.nbmin, d.bt, d.ewald,
                    d.zeta, d.rho, d.neps, d.ups, d.X, d.acc, d.dudt, d.keys_a, d.keys_b, d.vals_a, d.vals_b,
                    d.hist, d.lcp, d.cnt, d.base, d.scan_part, d.nbeg, d.nend, d.nlev, d.nnext, d.nparent,
                    d.nnch, d.narrive, d.nA, d.nB, d.nC, d.nQ0, d.nQ1, d.nM64, d.nC64, d.nQ64, d.nBmin,
                    d.nBmax, d.nCoff, d.nI, d.nK0, d.nK1, d.wstack, d.cand_leaf, d.cand_mask, d.diag_part, d.diag, d.counters, d.err, d.nnodes,
                    d.cube, d.fcube, d.bbox_part, d.hash3, d.cnt3, c->stage, c->kdk_acc, d.sys_off, d.sys_root, d.sys_sorted};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (int k = 0; k < 6; ++k)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    if (c->h_sys_off) cudaFreeHost(c->h_sys_off);
    for (int k = 0; k < 8; ++k)
        if (c->graph_exec[k]) cudaGraphExecDestroy(c->graph_exec[k]);
    if (c->kdk_exec) cudaGraphExecDestroy(c->kdk_exec);
    if (c->run_exec) cudaGraphExecDestroy(c->run_exec);
    if (c->bins_exec) cudaGraphExecDestroy(c->bins_exec);
    if (c->h_bt) cudaFreeHost(c->h_bt);
}

int check_args(evol_ctx *c, const evol_particles *p, const evol_params *prm)
{
    if (!c || !p || !prm) return EVOL_EINVAL;
    if (p->n < 0 || p->n_gas < 0 || p->n_gas > p->n) return EVOL_EINVAL;
    if (p->n > c->cap) return EVOL_ENOMEM;
    if (p->n == 0) return EVOL_OK;
    if (!p->x || !p->y || !p->z || !p->m) return EVOL_EINVAL;
    if (!(prm->theta >= 0.f)) return EVOL_EINVAL;
    if (prm->leaf_size < 0 || prm->leaf_size > 64) return EVOL_EINVAL;
    if (prm->group_size != 0 && prm->group_size != 32) return EVOL_EINVAL;
    if (prm->precision != EVOL_FP32_PLAIN && prm->precision != EVOL_FP32_MIXED) return EVOL_EINVAL;
    if (prm->gravity) {
        if (!p->eps) return EVOL_EINVAL;
        // periodic gravity (Ewald): a cube periodic on all three axes
        if (prm->periodic_mask) {
            if (prm->periodic_mask != 7) return EVOL_EINVAL;
            const float L = prm->periodic_hi[0] - prm->periodic_lo[0];
            if (!(L > 0.f) || prm->periodic_hi[1] - prm->periodic_lo[1] != L ||
                prm->periodic_hi[2] - prm->periodic_lo[2] != L)
                return EVOL_EINVAL;
        }
        if (prm->adaptive_softening && !(prm->n_nei_grav > 0.f)) return EVOL_EINVAL;
    }
    if (prm->sph && p->n_gas > 0) {
        if (!p->u || !p->h) return EVOL_EINVAL;
        if (!(prm->n_nei_sph > 0.f) || !(prm->gamma > 1.f)) return EVOL_EINVAL;
    }
    if (prm->periodic_mask & ~7) return EVOL_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (((prm->periodic_mask >> a) & 1) && !(prm->periodic_hi[a] > prm->periodic_lo[a])) return EVOL_EINVAL;
    // dissipation variants (Sect. 3.3.3)
    if (prm->visc_form != EVOL_VISC_MONAGHAN && prm->visc_form != EVOL_VISC_SIGNAL) return EVOL_EINVAL;
    if (prm->cond_vsig != EVOL_COND_VSIG_SOUND && prm->cond_vsig != EVOL_COND_VSIG_PRESSURE) return EVOL_EINVAL;
    if (prm->cond_source != EVOL_COND_SRC_SQRTU && prm->cond_source != EVOL_COND_SRC_LINEAR) return EVOL_EINVAL;
    if (prm->balsara && !(prm->balsara_eta >= 0.f)) return EVOL_EINVAL;
    if ((prm->variable_alpha || prm->conduction) && !(prm->alpha_tau > 0.f)) return EVOL_EINVAL;
    if (prm->sph_scheme != EVOL_SPH_LAGRANGIAN && prm->sph_scheme != EVOL_SPH_STANDARD) return EVOL_EINVAL;
    if (prm->length_group < 0 || prm->length_group > 32) return EVOL_EINVAL;
    if (prm->sph && prm->sph_scheme == EVOL_SPH_STANDARD) {
        const long nstd = lrintf(prm->n_nei_sph);
        if (nstd < 1 || nstd + 1 > evol_lengths_list_cap()) return EVOL_EINVAL;
    }
    if (prm->sph && p->n_gas > 0) {
        if (prm->variable_alpha && !p->alpha) return EVOL_EINVAL;
        if (prm->conduction && !p->alpha_u) return EVOL_EINVAL;
    }
    return EVOL_OK;
}

// FNV-1a over the bytes that define a captured step
uint64_t fnv(uint64_t h, const void *data, size_t len)
{
    const unsigned char *b = (const unsigned char *)data;
    for (size_t i = 0; i < len; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

void reset_counters(evol_ctx *c)
{
    cudaMemsetAsync(c->d.counters, 0, EVOL_NCOUNTERS * sizeof(unsigned long long), c->stream);
}

int ensure_tree(evol_ctx *c, const evol_particles *p, const evol_params *prm)
{
    if (c->built_n == p->n && c->built_ngas == p->n_gas && c->built_x == (const void *)p->x && c->nsys == 1)
        return EVOL_OK;
    c->nsys = 1;
    c->staged_nsys = 0;
    int rc = evol_launch_build(c, p, prm);
    if (rc) return rc;
    c->built_n = p->n;
    c->built_ngas = p->n_gas;
    c->built_x = p->x;
    c->density_done = 0;
    c->eps_done = 0;
    return EVOL_OK;
}

int set_err(evol_ctx *c, int rc)
{
    if (rc && !c->host_err) c->host_err = rc;
    return rc;
}

// The phases of one full step; each is captured into its own graph so that the timing
// events can be recorded between graph launches.
constexpr int NPHASE = 5;   // build | eps solve | h solve + pack + node maxima | walk | un-permute + diagnostics

int record_phase(evol_ctx *c, int k, evol_particles *p, const evol_params *prm, evol_outputs *out)
{
    int rc = EVOL_OK;
    const bool grav = prm->gravity != 0, sph = prm->sph != 0 && p->n_gas > 0;
    switch (k) {
    case 0:
        reset_counters(c);
        rc = evol_launch_build(c, p, prm);
        break;
    case 1:
        if (grav && prm->adaptive_softening) rc = evol_launch_lengths(c, p, prm, 1);
        break;
    case 2:
        if (sph) rc = evol_launch_lengths(c, p, prm, 0);
        if (!rc) rc = evol_launch_pack(c, p, prm, grav, sph);
        if (!rc) rc = evol_launch_node_lengths(c, prm, (int)p->n_gas);
        break;
    case 3:
        rc = evol_launch_walk(c, p, prm, grav, sph);
        break;
    case 4: {
        int what = EVOL_UNPERM_ACC | (grav ? EVOL_UNPERM_EPSOUT : 0) |
                   (sph ? (EVOL_UNPERM_LENGTHS | EVOL_UNPERM_DENSITY | EVOL_UNPERM_DUDT) : 0) |
                   (sph ? evol_unperm_switches(prm) : 0) | (c->persist ? EVOL_UNPERM_PERSIST : 0) |
                   (c->bins_active ? EVOL_UNPERM_ACTIVE : 0);
        rc = evol_launch_unpermute(c, p, out, what);
        if (!rc) rc = evol_launch_diagnostics(c, p, prm);
        break;
    }
    }
    return rc;
}

}  // namespace

namespace {
// Times the step (step(q) runs one: evol_step or evol_step_batched) for each candidate value of one
// cost parameter (set(q, v) writes it into a copy of the parameters) and returns the fastest; see
// evol_autotune for the protocol.
template <typename Set, typename Step>
int tune_param(evol_ctx *c, evol_particles *p, const evol_params *prm, const int *candidates, int ncand, int reps,
               int *best_out, float *ms_out, Set set, Step step)
{
    int rc = EVOL_OK;
    if (p->n == 0) {
        *best_out = candidates[0];
        return EVOL_OK;
    }
    // Every timed step starts from the caller's starting lengths, as a step of the caller's run
    // does: they are kept in the host-step staging buffer and restored before each step (outside
    // the timed interval).
    const int64_t n = p->n, ng = p->n_gas;
    float *save_h = c->stage, *save_e = c->stage + c->cap;
    auto restore = [&]() {
        if (p->h && ng > 0) cudaMemcpyAsync(p->h, save_h, ng * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
        if (p->eps) cudaMemcpyAsync(p->eps, save_e, n * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
    };
    if (p->h && ng > 0) cudaMemcpyAsync(save_h, p->h, ng * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
    if (p->eps) cudaMemcpyAsync(save_e, p->eps, n * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return EVOL_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return EVOL_ECUDA;
    }
    float best = 3.0e38f;
    int best_k = 0;
    std::vector<float> t(reps);
    // one untimed step first, so that the first candidate does not pay the clocks' ramp-up
    {
        evol_params q = *prm;
        set(q, candidates[0]);
        restore();
        rc = step(q);
        if (!rc) rc = evol_sync(c);
    }
    for (int k = 0; k < ncand && !rc; ++k) {
        evol_params q = *prm;
        set(q, candidates[k]);
        restore();
        if ((rc = step(q))) break;                           // records the graphs for this value
        if ((rc = evol_sync(c))) break;
        for (int r = 0; r < reps && !rc; ++r) {
            restore();
            cudaEventRecord(e0, c->stream);
            rc = step(q);
            cudaEventRecord(e1, c->stream);
            if (!rc) rc = evol_sync(c);
            if (!rc && cudaEventElapsedTime(&t[r], e0, e1) != cudaSuccess) rc = EVOL_ECUDA;
        }
        if (rc) break;
        std::vector<float> srt(t);
        std::sort(srt.begin(), srt.end());
        const float med = (reps & 1) ? srt[reps / 2] : 0.5f * (srt[reps / 2 - 1] + srt[reps / 2]);
        if (ms_out) ms_out[k] = med;
        if (med < best) {
            best = med;
            best_k = k;
        }
    }
    restore();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!rc) *best_out = candidates[best_k];
    return rc;
}

}  // namespace

extern "C" {

const char *evol_strerror(int code)
{
    switch (code) {
    case EVOL_OK: return "ok";
    case EVOL_EINVAL: return "invalid argument";
    case EVOL_ENOMEM: return "capacity exceeded or device allocation failed";
    case EVOL_ECUDA: return "CUDA runtime error";
    case EVOL_EOVERFLOW: return "fixed-capacity device list overflowed";
    case EVOL_ENOCONV: return "smoothing/softening length has no root or did not converge";
    case EVOL_ETIMEOUT: return "bounded device wait gave up";
    case EVOL_ENAN: return "non-finite value produced";
    case EVOL_ESTATE: return "call order violated";
    default: return "unknown status";
    }
}

int evol_create(evol_ctx **out, int64_t max_n, void *stream)
{
    if (!out) return EVOL_EINVAL;
    *out = nullptr;
    if (max_n < 1 || max_n > (int64_t)0x3fffffff) return EVOL_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return EVOL_ECUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return EVOL_ECUDA;
    evol_ctx *c = (evol_ctx *)calloc(1, sizeof(evol_ctx));
    if (!c) return EVOL_ENOMEM;
    c->cap = max_n;
    c->node_cap = NODE_FACTOR * max_n + 64;
    c->device = dev;
    c->num_sms = prop.multiProcessorCount;
    c->stream = (cudaStream_t)stream;
    c->sort_blocks = (max_n + 4095) / 4096;
    c->bbox_blocks = c->num_sms * 2;
    c->diag_blocks = c->num_sms * 2;
    c->cand_cap = 0;
    c->cand_slots = (int64_t)c->num_sms * 6 * evol_lengths_warps_per_block();   // length-solve warps
    c->wstack_slots = (int64_t)c->num_sms * 32;      // the walk and length grids use at most 32 warps per SM
    c->wstack_cap = WSTACK_CAP;
    c->wstack_lim = WSTACK_CAP;
    int64_t n = max_n, nn = c->node_cap;
    int64_t scan_parts = (256 * c->sort_blocks > n + 1 ? 256 * c->sort_blocks : n + 1) / 4096 + 2;
    evol_dev &d = c->d;
    int rc = 0;
    rc |= dalloc(&d.pos, n); rc |= dalloc(&d.vel, n); rc |= dalloc(&d.grav, n); rc |= dalloc(&d.hydro, n);
    rc |= dalloc(&d.snd, n); rc |= dalloc(&d.vah, n); rc |= dalloc(&d.orig, n); rc |= dalloc(&d.inv, n);
    rc |= dalloc(&d.len_h, n); rc |= dalloc(&d.len_eps, n); rc |= dalloc(&d.nh, n); rc |= dalloc(&d.omega, n);
    rc |= dalloc(&d.zeta, n); rc |= dalloc(&d.rho, n); rc |= dalloc(&d.neps, n); rc |= dalloc(&d.ups, n);
    rc |= dalloc(&d.X, n); rc |= dalloc(&d.acc, n); rc |= dalloc(&d.dudt, n);
    rc |= dalloc(&d.divv_h, n); rc |= dalloc(&d.divv_e, n); rc |= dalloc(&d.mumax, n);
    rc |= dalloc(&d.diss, n); rc |= dalloc(&d.curlv_h, n); rc |= dalloc(&d.vsig, n); rc |= dalloc(&d.lapu, n);
    rc |= dalloc(&d.dalpha, n); rc |= dalloc(&d.dalpha_u, n);
    rc |= dalloc(&d.tb, n); rc |= dalloc(&d.te, n); rc |= dalloc(&d.bact, n); rc |= dalloc(&d.pred_tau, n);
    rc |= dalloc(&d.pers, 7 * n); rc |= dalloc(&d.actf, n); rc |= dalloc(&d.acts, n + 1); rc |= dalloc(&d.act, n);
    {
        const int64_t nsg = n / (32 * EVOL_SG_GROUPS) + 2;     // super-groups of the force walk
        rc |= dalloc(&d.sg_acc, nsg * EVOL_SG_ACAP); rc |= dalloc(&d.sg_front, nsg * EVOL_SG_FCAP);
        rc |= dalloc(&d.sg_info, nsg);
    }
    rc |= dalloc(&d.nbmin, n); rc |= dalloc(&d.bt, 8);
    rc |= dalloc(&d.ewald, (int64_t)EVOL_EWALD_M * EVOL_EWALD_M * EVOL_EWALD_M);
    if (!rc && cudaMallocHost((void **)&c->h_bt, 8 * sizeof(unsigned long long)) != cudaSuccess) rc = EVOL_ENOMEM;
    rc |= dalloc(&d.dt, 4); rc |= dalloc(&d.time, 1);
    rc |= dalloc(&d.keys_a, n); rc |= dalloc(&d.keys_b, n); rc |= dalloc(&d.vals_a, n); rc |= dalloc(&d.vals_b, n);
    rc |= dalloc(&d.hist, 256 * c->sort_blocks + 1);
    rc |= dalloc(&d.lcp, n); rc |= dalloc(&d.cnt, n + 1); rc |= dalloc(&d.base, n + 1);
    rc |= dalloc(&d.scan_part, scan_parts);
    rc |= dalloc(&d.nbeg, nn); rc |= dalloc(&d.nend, nn); rc |= dalloc(&d.nlev, nn); rc |= dalloc(&d.nnext, nn);
    rc |= dalloc(&d.nparent, nn); rc |= dalloc(&d.nnch, nn); rc |= dalloc(&d.narrive, nn);
    rc |= dalloc(&d.nA, nn); rc |= dalloc(&d.nB, nn); rc |= dalloc(&d.nC, nn); rc |= dalloc(&d.nQ0, nn);
    rc |= dalloc(&d.nQ1, nn); rc |= dalloc(&d.nM64, nn); rc |= dalloc(&d.nC64, 3 * nn); rc |= dalloc(&d.nQ64, 6 * nn);
    rc |= dalloc(&d.nBmin, nn); rc |= dalloc(&d.nBmax, nn); rc |= dalloc(&d.nCoff, nn); rc |= dalloc(&d.nI, nn);
    rc |= dalloc(&d.nK0, nn); rc |= dalloc(&d.nK1, nn);
    rc |= dalloc(&d.wstack, c->wstack_slots * c->wstack_cap);
    rc |= dalloc(&d.cand_leaf, 1);                                      // unused
    rc |= dalloc(&d.cand_mask, 1);
    rc |= dalloc(&d.diag_part, 16 * c->diag_blocks); rc |= dalloc(&d.diag, 16);
    rc |= dalloc(&d.counters, EVOL_NCOUNTERS); rc |= dalloc(&d.err, 1); rc |= dalloc(&d.nnodes, 1);
    c->nsys_cap = NSYS_CAP;
    rc |= dalloc(&d.cube, 4 * (int64_t)NSYS_CAP); rc |= dalloc(&d.fcube, 4 * (int64_t)NSYS_CAP);
    rc |= dalloc(&d.bbox_part, 6 * c->bbox_blocks);
    rc |= dalloc(&d.sys_off, NSYS_CAP + 1); rc |= dalloc(&d.sys_root, NSYS_CAP); rc |= dalloc(&d.sys_sorted, n);
    if (!rc && cudaMallocHost((void **)&c->h_sys_off, (NSYS_CAP + 1) * sizeof(int32_t)) != cudaSuccess) rc = EVOL_ENOMEM;
    rc |= dalloc(&d.hash3, 3 * n); rc |= dalloc(&d.cnt3, 3 * n);
    rc |= dalloc(&c->stage, 26 * n);
    rc |= dalloc(&c->kdk_acc, 6 * n);
    for (int k = 0; k < 6 && !rc; ++k)
        if (cudaEventCreate(&c->ev[k]) != cudaSuccess) rc = EVOL_ECUDA;
    if (!rc) {
        cudaMemset(d.err, 0, sizeof(int));
        cudaMemset(d.counters, 0, EVOL_NCOUNTERS * sizeof(unsigned long long));
        cudaMemset(d.nnodes, 0, sizeof(int32_t));
        cudaMemset(d.diag, 0, 16 * sizeof(double));
        if (cudaDeviceSynchronize() != cudaSuccess) rc = EVOL_ECUDA;
    }
    if (rc) {
        cudaGetLastError();
        free_all(c);
        free(c);
        return rc < 0 ? (rc == EVOL_ECUDA ? EVOL_ECUDA : EVOL_ENOMEM) : EVOL_ENOMEM;
    }
    c->built_n = -1;
    // the allocation-free entry point's static scratch: placed and looked up on this device now,
    // while allocating is allowed (a failure here is retried by that entry point's own set-up)
    evol_noalloc_setup_current_device();
    cudaGetLastError();
    *out = c;
    return EVOL_OK;
}

int evol_destroy(evol_ctx *c)
{
    if (!c) return EVOL_EINVAL;
    cudaStreamSynchronize(c->stream);
    free_all(c);
    free(c);
    return EVOL_OK;
}

int evol_set_check_mode(evol_ctx *c, int on)
{
    if (!c) return EVOL_EINVAL;
    c->check_mode = on ? 1 : 0;
    return EVOL_OK;
}

int evol_set_stack_limit(evol_ctx *c, int64_t entries)
{
    if (!c) return EVOL_EINVAL;
    if (entries == 0) entries = c->wstack_cap;
    if (entries < 32 || entries > c->wstack_cap) return EVOL_EINVAL;
    c->wstack_lim = entries;
    return EVOL_OK;
}

int evol_build_tree(evol_ctx *c, const evol_particles *p, const evol_params *prm)
{
    int rc = check_args(c, p, prm);
    if (rc || p->n == 0) return rc;
    c->built_n = -1;
    reset_counters(c);
    return set_err(c, ensure_tree(c, p, prm));
}

int evol_sph_density(evol_ctx *c, evol_particles *p, const evol_params *prm, evol_outputs *out)
{
    int rc = check_args(c, p, prm);
    if (rc || p->n == 0) return rc;
    if (!prm->sph) return EVOL_EINVAL;
    if ((rc = ensure_tree(c, p, prm))) return set_err(c, rc);
    if (p->n_gas == 0) return EVOL_OK;
    if ((rc = evol_launch_lengths(c, p, prm, 0))) return set_err(c, rc);
    if ((rc = evol_launch_pack(c, p, prm, c->eps_done, 1))) return set_err(c, rc);
    if ((rc = evol_launch_unpermute(c, p, out, EVOL_UNPERM_LENGTHS | EVOL_UNPERM_DENSITY))) return set_err(c, rc);
    c->density_done = 1;
    return EVOL_OK;
}

int evol_gravity(evol_ctx *c, evol_particles *p, const evol_params *prm, evol_outputs *out)
{
    int rc = check_args(c, p, prm);
    if (rc || p->n == 0) return rc;
    if (!prm->gravity) return EVOL_EINVAL;
    if (prm->periodic_mask == 7 && (rc = evol_ewald_prepare(c))) return set_err(c, rc);
    if ((rc = ensure_tree(c, p, prm))) return set_err(c, rc);
    if (prm->adaptive_softening)
        if ((rc = evol_launch_lengths(c, p, prm, 1))) return set_err(c, rc);
    c->eps_done = 1;
    if ((rc = evol_launch_pack(c, p, prm, 1, c->density_done))) return set_err(c, rc);
    if ((rc = evol_launch_node_lengths(c, prm, (int)p->n_gas))) return set_err(c, rc);
    if ((rc = evol_launch_walk(c, p, prm, 1, 0))) return set_err(c, rc);
    if ((rc = evol_launch_unpermute(c, p, out, EVOL_UNPERM_ACC | EVOL_UNPERM_EPSOUT))) return set_err(c, rc);
    return EVOL_OK;
}

int evol_sph_forces(evol_ctx *c, const evol_particles *p, const evol_params *prm, evol_outputs *out)
{
    int rc = check_args(c, p, prm);
    if (rc || p->n == 0) return rc;
    if (!prm->sph) return EVOL_EINVAL;
    if (c->built_n != p->n || c->built_x != (const void *)p->x || !c->density_done) return EVOL_ESTATE;
    if (p->n_gas == 0) return EVOL_OK;
    if ((rc = evol_launch_node_lengths(c, prm, (int)p->n_gas))) return set_err(c, rc);
    if ((rc = evol_launch_walk(c, p, prm, 0, 1))) return set_err(c, rc);
    if ((rc = evol_launch_unpermute_ex(c, p, out,
                                       EVOL_UNPERM_ACC | EVOL_UNPERM_DUDT | evol_unperm_switches(prm),
                                       1)))
        return set_err(c, rc);
    return EVOL_OK;
}

static int run_step(evol_ctx *c, evol_particles *p, const evol_params *prm, evol_outputs *out)
{
    evol_outputs zero{};
    if (!out) out = &zero;
    if (prm->gravity && prm->periodic_mask == 7) {
        int erc = evol_ewald_prepare(c);
        if (erc) return set_err(c, erc);
    }
    uint64_t sig = 1469598103934665603ull;
    sig = fnv(sig, &c->nsys, sizeof c->nsys);
    sig = fnv(sig, p, sizeof *p);
    sig = fnv(sig, prm, sizeof *prm);
    sig = fnv(sig, out, sizeof *out);
    sig = fnv(sig, &c->check_mode, sizeof c->check_mode);
    sig = fnv(sig, &c->wstack_lim, sizeof c->wstack_lim);
    sig = fnv(sig, &c->want_divv, sizeof c->want_divv);
    sig = fnv(sig, &c->pred_dt, sizeof c->pred_dt);
    sig = fnv(sig, &c->persist, sizeof c->persist);
    sig = fnv(sig, &c->stream, sizeof c->stream);
    if (!c->graph_exec[0] || sig != c->graph_sig) {
        for (int k = 0; k < NPHASE; ++k)
            if (c->graph_exec[k]) {
                cudaGraphExecDestroy(c->graph_exec[k]);
                c->graph_exec[k] = nullptr;
            }
        cudaStream_t cap_stream = c->stream;
        bool own = false;
        if (!cap_stream) {          // the legacy stream cannot be captured: record on a private stream
            if (cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking) != cudaSuccess)
                return set_err(c, EVOL_ECUDA);
            own = true;
        }
        cudaStream_t saved = c->stream;
        c->stream = cap_stream;
        int prc = EVOL_OK;
        for (int k = 0; k < NPHASE && !prc; ++k) {
            cudaGraph_t graph = nullptr;
            if (cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                prc = EVOL_ECUDA;
                break;
            }
            int rrc = record_phase(c, k, p, prm, out);
            cudaError_t e = cudaStreamEndCapture(cap_stream, &graph);
            if (rrc || e != cudaSuccess || !graph) {
                prc = rrc ? rrc : EVOL_ECUDA;
            } else if (cudaGraphInstantiate(&c->graph_exec[k], graph, 0) != cudaSuccess) {
                c->graph_exec[k] = nullptr;
                prc = EVOL_ECUDA;
            }
            if (graph) cudaGraphDestroy(graph);
        }
        c->stream = saved;
        if (own) cudaStreamDestroy(cap_stream);
        if (prc) {
            cudaGetLastError();
            for (int k = 0; k < NPHASE; ++k)
                if (c->graph_exec[k]) {
                    cudaGraphExecDestroy(c->graph_exec[k]);
                    c->graph_exec[k] = nullptr;
                }
            return set_err(c, prc);
        }
        c->graph_sig = sig;
    }
    for (int k = 0; k < NPHASE; ++k) {
        cudaEventRecord(c->ev[k], c->stream);
        if (cudaGraphLaunch(c->graph_exec[k], c->stream) != cudaSuccess) return set_err(c, EVOL_ECUDA);
    }
    cudaEventRecord(c->ev[NPHASE], c->stream);
    c->built_n = p->n;
    c->built_ngas = p->n_gas;
    c->built_x = p->x;
    c->density_done = prm->sph && p->n_gas > 0;
    c->eps_done = prm->gravity;
    return EVOL_OK;
}

int evol_step(evol_ctx *c, evol_particles *p, const evol_params *prm, evol_outputs *out)
{
    int rc = check_args(c, p, prm);
    if (rc || p->n == 0) return rc;
    c->nsys = 1;
    c->staged_nsys = 0;
    return run_step(c, p, prm, out);
}

int evol_step_batched(evol_ctx *c, const int64_t *sys_offsets, int nsys, evol_particles *p, const evol_params *prm,
                      evol_outputs *out)
{
    int rc = check_args(c, p, prm);
    if (rc) return rc;
    if (!sys_offsets || nsys < 1 || nsys > c->nsys_cap) return EVOL_EINVAL;
    if (prm->gravity && prm->periodic_mask) return EVOL_EINVAL;     // periodic gravity: one system
    if (sys_offsets[0] != 0 || sys_offsets[nsys] != p->n) return EVOL_EINVAL;
    for (int k = 0; k < nsys; ++k)
        if (sys_offsets[k + 1] < sys_offsets[k]) return EVOL_EINVAL;
    if (p->n == 0) return EVOL_OK;
    // offsets already on the device from the previous step on this context, itself a step of this
    // batch (every single-system entry point sets nsys = 1 before its kernels rewrite the offsets),
    // are not staged again, so that repeated steps of one batch need no host synchronisation
    bool staged = c->staged_nsys == nsys && c->nsys == nsys;
    for (int k = 0; staged && k <= nsys; ++k) staged = c->h_sys_off[k] == (int32_t)sys_offsets[k];
    if (!staged) {
        // the previous call's copy may still be in flight from the pinned staging buffer
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return set_err(c, EVOL_ECUDA);
        for (int k = 0; k <= nsys; ++k) c->h_sys_off[k] = (int32_t)sys_offsets[k];
        if (cudaMemcpyAsync(c->d.sys_off, c->h_sys_off, (nsys + 1) * sizeof(int32_t), cudaMemcpyHostToDevice,
                            c->stream) != cudaSuccess) {
            c->staged_nsys = 0;
            return set_err(c, EVOL_ECUDA);
        }
        c->staged_nsys = nsys;
    }
    c->nsys = nsys;
    return run_step(c, p, prm, out);
}

int evol_kdk(evol_ctx *c, evol_particles *p, const evol_params *prm, evol_outputs *out, float dt, int nsteps)
{
    int rc = check_args(c, p, prm);
    if (rc || (p && p->n == 0)) return rc;
    if (nsteps < 0 || !(dt == dt) || dt > 3.0e38f || dt < -3.0e38f) return EVOL_EINVAL;
    if (!p->vx || !p->vy || !p->vz) return EVOL_EINVAL;
    const int64_t cap = c->cap;
    evol_outputs o = out ? *out : evol_outputs{};
    o.ax = c->kdk_acc;
    o.ay = c->kdk_acc + cap;
    o.az = c->kdk_acc + 2 * cap;
    o.dudt = c->kdk_acc + 3 * cap;
    o.dalpha = c->kdk_acc + 4 * cap;
    o.dalpha_u = c->kdk_acc + 5 * cap;
    // forces at the starting positions
    if ((rc = evol_step(c, p, prm, &o))) return rc;
    if (nsteps > 0) {
        uint64_t sig = 88172645463325252ull;
        sig = fnv(sig, p, sizeof *p);
        sig = fnv(sig, prm, sizeof *prm);
        sig = fnv(sig, &o, sizeof o);
        sig = fnv(sig, &dt, sizeof dt);
        sig = fnv(sig, &c->check_mode, sizeof c->check_mode);
        sig = fnv(sig, &c->wstack_lim, sizeof c->wstack_lim);
        sig = fnv(sig, &c->stream, sizeof c->stream);
        if (!c->kdk_exec || sig != c->kdk_sig) {
            if (c->kdk_exec) {
                cudaGraphExecDestroy(c->kdk_exec);
                c->kdk_exec = nullptr;
            }
            cudaStream_t cap_stream = c->stream;
            bool own = false;
            if (!cap_stream) {
                if (cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking) != cudaSuccess)
                    return set_err(c, EVOL_ECUDA);
                own = true;
            }
            cudaStream_t saved = c->stream;
            c->stream = cap_stream;
            cudaGraph_t graph = nullptr;
            int prc = EVOL_OK;
            if (cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                prc = EVOL_ECUDA;
            } else {
                prc = evol_launch_kick(c, p, prm, 0.5f * dt, o.ax, o.ay, o.az, o.dudt, o.dalpha, o.dalpha_u);
                if (!prc) prc = evol_launch_drift(c, p, prm, dt);
                for (int k = 0; k < NPHASE && !prc; ++k) prc = record_phase(c, k, p, prm, &o);
                if (!prc) prc = evol_launch_kick(c, p, prm, 0.5f * dt, o.ax, o.ay, o.az, o.dudt, o.dalpha, o.dalpha_u);
                cudaError_t e = cudaStreamEndCapture(cap_stream, &graph);
                if (!prc && (e != cudaSuccess || !graph)) prc = EVOL_ECUDA;
                if (!prc && cudaGraphInstantiate(&c->kdk_exec, graph, 0) != cudaSuccess) {
                    c->kdk_exec = nullptr;
                    prc = EVOL_ECUDA;
                }
            }
            if (graph) cudaGraphDestroy(graph);
            c->stream = saved;
            if (own) cudaStreamDestroy(cap_stream);
            if (prc) {
                cudaGetLastError();
                return set_err(c, prc);
            }
            c->kdk_sig = sig;
        }
        for (int k = 0; k < nsteps; ++k)
            if (cudaGraphLaunch(c->kdk_exec, c->stream) != cudaSuccess) return set_err(c, EVOL_ECUDA);
    }
    // hand the last accelerations, du/dt and switch rates to the caller
    const int64_t n = p->n, ng = p->n_gas;
    float *dst[6] = {out ? out->ax : nullptr, out ? out->ay : nullptr, out ? out->az : nullptr,
                     out ? out->dudt : nullptr, out && prm->variable_alpha ? out->dalpha : nullptr,
                     out && prm->conduction ? out->dalpha_u : nullptr};
    const float *src[6] = {o.ax, o.ay, o.az, o.dudt, o.dalpha, o.dalpha_u};
    const int64_t len[6] = {n, n, n, ng, ng, ng};
    for (int k = 0; k < 6; ++k)
        if (dst[k] && len[k] > 0)
            cudaMemcpyAsync(dst[k], src[k], len[k] * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
    return EVOL_OK;
}

int evol_run(evol_ctx *c, evol_particles *p, const evol_params *prm, const evol_integrator *ip, evol_outputs *out,
             int nsteps, double *time, float *last_dt)
{
    int rc = check_args(c, p, prm);
    if (rc || (p && p->n == 0)) return rc;
    if (!ip || nsteps < 0) return EVOL_EINVAL;
    const float et[5] = {ip->eta_acc, ip->eta_vel, ip->eta_av, ip->eta_courant, ip->eta_u};
    for (float e : et)
        if (!(e >= 0.f)) return EVOL_EINVAL;
    if (!(ip->dt_min >= 0.f) || !(ip->dt_max > 0.f) || !(ip->dt_min <= ip->dt_max) || ip->dt_max > 3.0e38f)
        return EVOL_EINVAL;
    if (!p->vx || !p->vy || !p->vz) return EVOL_EINVAL;
    const int64_t cap = c->cap;
    evol_outputs o = out ? *out : evol_outputs{};
    o.ax = c->kdk_acc;
    o.ay = c->kdk_acc + cap;
    o.az = c->kdk_acc + 2 * cap;
    o.dudt = c->kdk_acc + 3 * cap;
    o.dalpha = c->kdk_acc + 4 * cap;
    o.dalpha_u = c->kdk_acc + 5 * cap;
    const double t0 = time ? *time : 0.0;
    if (cudaMemcpyAsync(c->d.time, &t0, sizeof(double), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
        return set_err(c, EVOL_ECUDA);
    // forces, velocity divergences and the largest |mu| at the starting positions
    c->want_divv = 1;
    c->pred_dt = nullptr;
    if ((rc = evol_step(c, p, prm, &o))) {
        c->want_divv = 0;
        return rc;
    }
    if (nsteps > 0) {
        uint64_t sig = 6364136223846793005ull;
        sig = fnv(sig, p, sizeof *p);
        sig = fnv(sig, prm, sizeof *prm);
        sig = fnv(sig, ip, sizeof *ip);
        sig = fnv(sig, &o, sizeof o);
        sig = fnv(sig, &c->check_mode, sizeof c->check_mode);
        sig = fnv(sig, &c->wstack_lim, sizeof c->wstack_lim);
        sig = fnv(sig, &c->stream, sizeof c->stream);
        if (!c->run_exec || sig != c->run_sig) {
            if (c->run_exec) {
                cudaGraphExecDestroy(c->run_exec);
                c->run_exec = nullptr;
            }
            cudaStream_t cap_stream = c->stream;
            bool own = false;
            if (!cap_stream) {
                if (cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
                    c->want_divv = 0;
                    return set_err(c, EVOL_ECUDA);
                }
                own = true;
            }
            cudaStream_t saved = c->stream;
            c->stream = cap_stream;
            cudaGraph_t graph = nullptr;
            int prc = EVOL_OK;
            if (cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                prc = EVOL_ECUDA;
            } else {
                prc = evol_launch_integrator_step(c, p, prm, ip, 0);
                c->pred_dt = ip->predicted_velocity ? c->d.dt : nullptr;
                for (int k = 0; k < NPHASE && !prc; ++k) prc = record_phase(c, k, p, prm, &o);
                c->pred_dt = nullptr;
                if (!prc) prc = evol_launch_integrator_step(c, p, prm, ip, 1);
                cudaError_t e = cudaStreamEndCapture(cap_stream, &graph);
                if (!prc && (e != cudaSuccess || !graph)) prc = EVOL_ECUDA;
                if (!prc && cudaGraphInstantiate(&c->run_exec, graph, 0) != cudaSuccess) {
                    c->run_exec = nullptr;
                    prc = EVOL_ECUDA;
                }
            }
            if (graph) cudaGraphDestroy(graph);
            c->stream = saved;
            if (own) cudaStreamDestroy(cap_stream);
            if (prc) {
                cudaGetLastError();
                c->want_divv = 0;
                return set_err(c, prc);
            }
            c->run_sig = sig;
        }
        for (int k = 0; k < nsteps; ++k)
            if (cudaGraphLaunch(c->run_exec, c->stream) != cudaSuccess) {
                c->want_divv = 0;
                return set_err(c, EVOL_ECUDA);
            }
    }
    c->want_divv = 0;
    // hand the last accelerations, du/dt and switch rates to the caller
    const int64_t n = p->n, ng = p->n_gas;
    float *dst[6] = {out ? out->ax : nullptr, out ? out->ay : nullptr, out ? out->az : nullptr,
                     out ? out->dudt : nullptr, out && prm->variable_alpha ? out->dalpha : nullptr,
                     out && prm->conduction ? out->dalpha_u : nullptr};
    const float *src[6] = {o.ax, o.ay, o.az, o.dudt, o.dalpha, o.dalpha_u};
    const int64_t len[6] = {n, n, n, ng, ng, ng};
    for (int k = 0; k < 6; ++k)
        if (dst[k] && len[k] > 0)
            cudaMemcpyAsync(dst[k], src[k], len[k] * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
    double tt = t0;
    float dt = 0.f;
    cudaMemcpyAsync(&tt, c->d.time, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(&dt, c->d.dt, sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return set_err(c, EVOL_ECUDA);
    if (time) *time = tt;
    if (last_dt) *last_dt = nsteps > 0 ? dt : 0.f;
    return EVOL_OK;
}

int evol_run_bins(evol_ctx *c, evol_particles *p, const evol_params *prm, const evol_bins *bp, evol_outputs *out,
                  int nlargest, double *time, int64_t stats[4])
{
    int rc = check_args(c, p, prm);
    if (rc || (p && p->n == 0)) return rc;
    if (!bp || nlargest < 0 || bp->max_bin < 0 || bp->max_bin > 30) return EVOL_EINVAL;
    const evol_integrator *ip = &bp->crit;
    const float et[5] = {ip->eta_acc, ip->eta_vel, ip->eta_av, ip->eta_courant, ip->eta_u};
    for (float e : et)
        if (!(e >= 0.f)) return EVOL_EINVAL;
    if (!(ip->dt_max > 0.f) || ip->dt_max > 3.0e38f) return EVOL_EINVAL;
    if (!(bp->wake_factor == 0.f || bp->wake_factor > 1.f) || !(bp->wake_factor < 3.0e38f)) return EVOL_EINVAL;
    if (!p->vx || !p->vy || !p->vz) return EVOL_EINVAL;
    const int64_t cap = c->cap, n = p->n, ng = p->n_gas;
    const unsigned long long t_end = (unsigned long long)nlargest << bp->max_bin;
    // every evaluation's accelerations, du/dt and switch rates go to kdk_acc (caller order)
    evol_outputs o = out ? *out : evol_outputs{};
    o.ax = c->kdk_acc;
    o.ay = c->kdk_acc + cap;
    o.az = c->kdk_acc + 2 * cap;
    o.dudt = c->kdk_acc + 3 * cap;
    o.dalpha = c->kdk_acc + 4 * cap;
    o.dalpha_u = c->kdk_acc + 5 * cap;
    auto reset = [&]() {
        c->want_divv = 0;
        c->persist = 0;
        c->bins_active = 0;
        c->bins_wake = 0;
        c->pred_tau = nullptr;
        c->pred_dt = nullptr;
    };
    // the start: every particle evaluated, its state kept for the steps in which it is inactive
    reset();
    c->want_divv = 1;
    c->persist = 1;
    c->bins_t_end = t_end;
    if ((rc = evol_step(c, p, prm, &o))) {
        reset();
        return rc;
    }
    const bool wake = bp->wake_factor > 0.f && prm->sph && ng > 0;
    if (t_end > 0) {
        if ((rc = evol_launch_bins(c, p, prm, bp, 0))) {
            reset();
            return set_err(c, rc);
        }
        uint64_t sig = 0x9e3779b97f4a7c15ull;
        sig = fnv(sig, p, sizeof *p);
        sig = fnv(sig, prm, sizeof *prm);
        sig = fnv(sig, bp, sizeof *bp);
        sig = fnv(sig, &o, sizeof o);
        sig = fnv(sig, &t_end, sizeof t_end);
        sig = fnv(sig, &c->check_mode, sizeof c->check_mode);
        sig = fnv(sig, &c->wstack_lim, sizeof c->wstack_lim);
        sig = fnv(sig, &c->stream, sizeof c->stream);
        if (!c->bins_exec || sig != c->bins_sig) {
            if (c->bins_exec) {
                cudaGraphExecDestroy(c->bins_exec);
                c->bins_exec = nullptr;
            }
            cudaStream_t cap_stream = c->stream;
            bool own = false;
            if (!cap_stream) {
                if (cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
                    reset();
                    return set_err(c, EVOL_ECUDA);
                }
                own = true;
            }
            cudaStream_t saved = c->stream;
            c->stream = cap_stream;
            cudaGraph_t graph = nullptr;
            int prc = EVOL_OK;
            if (cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                prc = EVOL_ECUDA;
            } else {
                const bool grav = prm->gravity != 0, sph = prm->sph != 0 && ng > 0;
                // t_next, drift, active flags, prediction times
                prc = evol_launch_bins(c, p, prm, bp, 1);
                // tree of every particle (velocities and u predicted per particle)
                c->pred_tau = ip->predicted_velocity ? c->d.pred_tau : nullptr;
                if (!prc) prc = record_phase(c, 0, p, prm, &o);
                if (!prc) prc = evol_launch_active_list(c, (int)n);
                // solves and walk over the active list; the inactive keep their last evaluation
                c->bins_active = 1;
                c->bins_wake = wake;
                if (!prc && grav && prm->adaptive_softening) prc = evol_launch_lengths(c, p, prm, 1);
                if (!prc && sph) prc = evol_launch_lengths(c, p, prm, 0);
                if (!prc) prc = evol_launch_bins(c, p, prm, bp, 2);
                if (!prc) prc = evol_launch_pack(c, p, prm, grav, sph);
                if (!prc) prc = evol_launch_node_lengths(c, prm, (int)ng);
                if (!prc && wake && cudaMemsetAsync(c->d.nbmin, 0xff, n * sizeof(unsigned), cap_stream) != cudaSuccess)
                    prc = EVOL_ECUDA;
                if (!prc) prc = record_phase(c, 3, p, prm, &o);
                if (!prc) prc = record_phase(c, 4, p, prm, &o);
                // kicks, new steps, wake-up, t_sys = t_next
                if (!prc) prc = evol_launch_bins(c, p, prm, bp, 3);
                cudaError_t e = cudaStreamEndCapture(cap_stream, &graph);
                if (!prc && (e != cudaSuccess || !graph)) prc = EVOL_ECUDA;
                if (!prc && cudaGraphInstantiate(&c->bins_exec, graph, 0) != cudaSuccess) {
                    c->bins_exec = nullptr;
                    prc = EVOL_ECUDA;
                }
            }
            if (graph) cudaGraphDestroy(graph);
            c->stream = saved;
            if (own) cudaStreamDestroy(cap_stream);
            if (prc) {
                cudaGetLastError();
                reset();
                return set_err(c, prc);
            }
            c->bins_sig = sig;
        }
        // system steps until the end; each advances the time by at least one tick
        unsigned long long tsys = 0;
        for (unsigned long long it = 0; it < t_end && tsys < t_end; ++it) {
            if (cudaGraphLaunch(c->bins_exec, c->stream) != cudaSuccess ||
                cudaMemcpyAsync(c->h_bt, c->d.bt, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream) !=
                    cudaSuccess ||
                cudaStreamSynchronize(c->stream) != cudaSuccess) {
                reset();
                return set_err(c, EVOL_ECUDA);
            }
            // a system step that did not advance the time would repeat forever: stop
            if (c->h_bt[0] <= tsys) {
                reset();
                return set_err(c, EVOL_ESTATE);
            }
            tsys = c->h_bt[0];
        }
    }
    reset();
    // hand the last accelerations, du/dt and switch rates to the caller
    float *dst[6] = {out ? out->ax : nullptr, out ? out->ay : nullptr, out ? out->az : nullptr,
                     out ? out->dudt : nullptr, out && prm->variable_alpha ? out->dalpha : nullptr,
                     out && prm->conduction ? out->dalpha_u : nullptr};
    const float *src[6] = {o.ax, o.ay, o.az, o.dudt, o.dalpha, o.dalpha_u};
    const int64_t len[6] = {n, n, n, ng, ng, ng};
    for (int k = 0; k < 6; ++k)
        if (dst[k] && len[k] > 0)
            cudaMemcpyAsync(dst[k], src[k], len[k] * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
    if (cudaMemcpyAsync(c->h_bt, c->d.bt, 6 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return set_err(c, EVOL_ECUDA);
    if (stats) {
        const bool ran = t_end > 0;
        stats[0] = ran ? (int64_t)c->h_bt[2] : 0;
        stats[1] = (ran ? (int64_t)c->h_bt[3] : 0) + n;
        stats[2] = ran ? (int64_t)c->h_bt[4] : 0;
        stats[3] = ran ? (int64_t)c->h_bt[5] : 0;
    }
    if (time) *time += (double)nlargest * (double)ip->dt_max;
    return EVOL_OK;
}

int evol_step_host(evol_ctx *c, evol_particles *ph, const evol_params *prm, evol_outputs *oh)
{
    int rc = check_args(c, ph, prm);
    if (rc || ph->n == 0) return rc;
    int64_t n = ph->n, ng = ph->n_gas;
    float *st = c->stage;
    constexpr int NIN = 12, NOUT = 14;
    float *in[NIN];
    for (int k = 0; k < NIN; ++k) in[k] = st + (int64_t)k * c->cap;
    const float *src[NIN] = {ph->x, ph->y, ph->z, ph->vx, ph->vy, ph->vz, ph->m, ph->u, ph->h, ph->eps,
                             ph->alpha, ph->alpha_u};
    int64_t len[NIN] = {n, n, n, n, n, n, n, ng, ng, n, ng, ng};
    for (int k = 0; k < NIN; ++k)
        if (src[k] && len[k] > 0)
            if (cudaMemcpyAsync(in[k], src[k], len[k] * sizeof(float), cudaMemcpyHostToDevice, c->stream) !=
                cudaSuccess)
                return set_err(c, EVOL_ECUDA);
    evol_particles pd = *ph;
    pd.x = in[0]; pd.y = in[1]; pd.z = in[2];
    pd.vx = ph->vx ? in[3] : nullptr; pd.vy = ph->vy ? in[4] : nullptr; pd.vz = ph->vz ? in[5] : nullptr;
    pd.m = in[6];
    pd.u = ph->u ? in[7] : nullptr;
    pd.h = ph->h ? in[8] : nullptr;
    pd.eps = ph->eps ? in[9] : nullptr;
    pd.alpha = ph->alpha ? in[10] : nullptr;
    pd.alpha_u = ph->alpha_u ? in[11] : nullptr;
    evol_outputs zero{};
    if (!oh) oh = &zero;
    float *outp[NOUT];
    for (int k = 0; k < NOUT; ++k) outp[k] = st + (int64_t)(NIN + k) * c->cap;
    float *hdst[NOUT] = {oh->ax, oh->ay, oh->az, oh->pot, oh->rho, oh->P, oh->c, oh->omega, oh->zeta, oh->dudt,
                         oh->ups, oh->X, oh->dalpha, oh->dalpha_u};
    int64_t olen[NOUT] = {n, n, n, n, ng, ng, ng, ng, ng, ng, n, n, ng, ng};
    evol_outputs od{};
    float **odp[NOUT] = {&od.ax, &od.ay, &od.az, &od.pot, &od.rho, &od.P, &od.c, &od.omega, &od.zeta, &od.dudt,
                         &od.ups, &od.X, &od.dalpha, &od.dalpha_u};
    for (int k = 0; k < NOUT; ++k) *odp[k] = hdst[k] ? outp[k] : nullptr;
    if ((rc = evol_step(c, &pd, prm, &od))) return rc;
    for (int k = 0; k < NOUT; ++k)
        if (hdst[k] && olen[k] > 0)
            cudaMemcpyAsync(hdst[k], outp[k], olen[k] * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    if (ph->h && ng > 0) cudaMemcpyAsync(ph->h, in[8], ng * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    if (ph->eps) cudaMemcpyAsync(ph->eps, in[9], n * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    return evol_sync(c);
}

int evol_autotune(evol_ctx *c, evol_particles *p, const evol_params *prm, evol_outputs *out,
                  const int *candidates, int ncand, int reps, int *best_leaf, float *ms_out)
{
    static const int defaults[6] = {4, 8, 12, 16, 24, 32};
    int rc = check_args(c, p, prm);
    if (rc) return rc;
    if (!best_leaf || reps < 1 || (candidates && ncand < 1)) return EVOL_EINVAL;
    if (!candidates) {
        candidates = defaults;
        ncand = 6;
    }
    for (int k = 0; k < ncand; ++k)
        if (candidates[k] < 1 || candidates[k] > 64) return EVOL_EINVAL;
    return tune_param(c, p, prm, candidates, ncand, reps, best_leaf, ms_out,
                      [](evol_params &q, int v) { q.leaf_size = v; },
                      [&](const evol_params &q) { return evol_step(c, p, &q, out); });
}

int evol_autotune_length_group(evol_ctx *c, evol_particles *p, const evol_params *prm, evol_outputs *out,
                               const int *candidates, int ncand, int reps, int *best, float *ms_out)
{
    static const int defaults[4] = {4, 8, 16, 32};
    int rc = check_args(c, p, prm);
    if (rc) return rc;
    if (!best || reps < 1 || (candidates && ncand < 1)) return EVOL_EINVAL;
    if (!candidates) {
        candidates = defaults;
        ncand = 4;
    }
    for (int k = 0; k < ncand; ++k)
        if (candidates[k] < 1 || candidates[k] > 32) return EVOL_EINVAL;
    return tune_param(c, p, prm, candidates, ncand, reps, best, ms_out,
                      [](evol_params &q, int v) { q.length_group = v; },
                      [&](const evol_params &q) { return evol_step(c, p, &q, out); });
}

int evol_autotune_batched(evol_ctx *c, const int64_t *sys_offsets, int nsys, evol_particles *p,
                          const evol_params *prm, evol_outputs *out, int which, const int *candidates, int ncand,
                          int reps, int *best, float *ms_out)
{
    static const int leaf_defaults[6] = {4, 8, 12, 16, 24, 32};
    static const int group_defaults[4] = {4, 8, 16, 32};
    int rc = check_args(c, p, prm);
    if (rc) return rc;
    if (!sys_offsets || !best || reps < 1 || (candidates && ncand < 1)) return EVOL_EINVAL;
    if (which != EVOL_TUNE_LEAF_SIZE && which != EVOL_TUNE_LENGTH_GROUP) return EVOL_EINVAL;
    const bool leaf = which == EVOL_TUNE_LEAF_SIZE;
    if (!candidates) {
        candidates = leaf ? leaf_defaults : group_defaults;
        ncand = leaf ? 6 : 4;
    }
    for (int k = 0; k < ncand; ++k)
        if (candidates[k] < 1 || candidates[k] > (leaf ? 64 : 32)) return EVOL_EINVAL;
    auto step = [&](const evol_params &q) { return evol_step_batched(c, sys_offsets, nsys, p, &q, out); };
    if (leaf)
        return tune_param(c, p, prm, candidates, ncand, reps, best, ms_out,
                          [](evol_params &q, int v) { q.leaf_size = v; }, step);
    return tune_param(c, p, prm, candidates, ncand, reps, best, ms_out,
                      [](evol_params &q, int v) { q.length_group = v; }, step);
}

int evol_sync(evol_ctx *c)
{
    if (!c) return EVOL_EINVAL;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        return EVOL_ECUDA;
    }
    int e = 0;
    if (cudaMemcpy(&e, c->d.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return EVOL_ECUDA;
    if (e) cudaMemset(c->d.err, 0, sizeof(int));
    int h = c->host_err;
    c->host_err = 0;
    return h ? h : e;
}

int evol_get_diagnostics(evol_ctx *c, double out[16])
{
    if (!c || !out) return EVOL_EINVAL;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return EVOL_ECUDA;
    return cudaMemcpy(out, c->d.diag, 16 * sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess ? EVOL_OK
                                                                                                 : EVOL_ECUDA;
}

int evol_get_counters(evol_ctx *c, uint64_t out[32])
{
    if (!c || !out) return EVOL_EINVAL;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return EVOL_ECUDA;
    unsigned long long v[EVOL_NCOUNTERS];
    if (cudaMemcpy(v, c->d.counters, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess) return EVOL_ECUDA;
    for (int k = 0; k < 32; ++k) out[k] = k < EVOL_NCOUNTERS ? (uint64_t)v[k] : 0;
    return EVOL_OK;
}

int evol_get_timings(evol_ctx *c, float out[5])
{
    if (!c || !out) return EVOL_EINVAL;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return EVOL_ECUDA;
    // build | eps solve | h solve (+ pack, node maxima) | walk | total
    const int pairs[5][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 4}, {0, 5}};
    for (int k = 0; k < 5; ++k) {
        float ms = -1.f;
        if (cudaEventElapsedTime(&ms, c->ev[pairs[k][0]], c->ev[pairs[k][1]]) != cudaSuccess) {
            cudaGetLastError();
            ms = -1.f;
        }
        out[k] = ms;
    }
    return EVOL_OK;
}

int64_t evol_get_debug(evol_ctx *c, int what, void *dst, int64_t cap)
{
    if (!c) return EVOL_EINVAL;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return EVOL_ECUDA;
    int64_t n = c->built_n > 0 ? c->built_n : 0;
    int32_t nn = 0;
    cudaMemcpy(&nn, c->d.nnodes, sizeof nn, cudaMemcpyDeviceToHost);
    auto copy = [&](const void *src, int64_t bytes) -> bool {
        if (!dst || cap < bytes) return false;
        return cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost) == cudaSuccess;
    };
    switch (what) {
    case EVOL_DBG_KEYS:
        copy(c->d.keys_a, n * 8);
        return n;
    case EVOL_DBG_PERM:
        copy(c->d.orig, n * 4);
        return n;
    case EVOL_DBG_CUBE:
        copy(c->d.cube, 32);
        return 4;
    case EVOL_DBG_NODES: {
        if (dst && cap >= (int64_t)nn * 20) {
            int32_t *o = (int32_t *)dst;
            cudaMemcpy(o, c->d.nbeg, nn * 4, cudaMemcpyDeviceToHost);
            cudaMemcpy(o + nn, c->d.nend, nn * 4, cudaMemcpyDeviceToHost);
            cudaMemcpy(o + 2 * nn, c->d.nlev, nn * 4, cudaMemcpyDeviceToHost);
            cudaMemcpy(o + 3 * nn, c->d.nnext, nn * 4, cudaMemcpyDeviceToHost);
            cudaMemcpy(o + 4 * nn, c->d.nnch, nn * 4, cudaMemcpyDeviceToHost);
        }
        return (int64_t)nn * 5;
    }
    case EVOL_DBG_MOMENTS: {
        if (dst && cap >= (int64_t)nn * 80) {
            std::vector<float4> A(nn), B(nn), C(nn), Q0(nn), Q1(nn), bl(nn), bh(nn);
            cudaMemcpy(A.data(), c->d.nA, nn * 16, cudaMemcpyDeviceToHost);
            cudaMemcpy(B.data(), c->d.nB, nn * 16, cudaMemcpyDeviceToHost);
            cudaMemcpy(C.data(), c->d.nC, nn * 16, cudaMemcpyDeviceToHost);
            cudaMemcpy(Q0.data(), c->d.nQ0, nn * 16, cudaMemcpyDeviceToHost);
            cudaMemcpy(Q1.data(), c->d.nQ1, nn * 16, cudaMemcpyDeviceToHost);
            cudaMemcpy(bl.data(), c->d.nBmin, nn * 16, cudaMemcpyDeviceToHost);
            cudaMemcpy(bh.data(), c->d.nBmax, nn * 16, cudaMemcpyDeviceToHost);
            float *o = (float *)dst;
            for (int32_t i = 0; i < nn; ++i) {
                float v[20] = {Q0[i].w, A[i].x,  A[i].y,  A[i].z,  Q0[i].x, Q0[i].y, Q0[i].z,
                               Q1[i].x, Q1[i].y, Q1[i].z, Q1[i].w, bl[i].x, bl[i].y, bl[i].z,
                               bh[i].x, bh[i].y, bh[i].z, C[i].w,  B[i].w,  A[i].w};
                memcpy(o + 20 * (int64_t)i, v, sizeof v);
            }
        }
        return (int64_t)nn * 20;
    }
    case EVOL_DBG_FLOW: {
        if (dst && cap >= 3 * n * 4) {
            std::vector<int32_t> orig(n);
            std::vector<float> a(n), b(n), m(n);
            cudaMemcpy(orig.data(), c->d.orig, n * 4, cudaMemcpyDeviceToHost);
            cudaMemcpy(a.data(), c->d.divv_e, n * 4, cudaMemcpyDeviceToHost);
            cudaMemcpy(b.data(), c->d.divv_h, n * 4, cudaMemcpyDeviceToHost);
            cudaMemcpy(m.data(), c->d.mumax, n * 4, cudaMemcpyDeviceToHost);
            float *o = (float *)dst;
            for (int64_t s = 0; s < n; ++s) {
                o[orig[s]] = a[s];
                o[n + orig[s]] = b[s];
                o[2 * n + orig[s]] = m[s];
            }
        }
        return 3 * n;
    }
    case EVOL_DBG_BINS: {
        if (dst && cap >= 2 * n * 8) {
            cudaMemcpy(dst, c->d.tb, n * 8, cudaMemcpyDeviceToHost);
            cudaMemcpy((char *)dst + n * 8, c->d.te, n * 8, cudaMemcpyDeviceToHost);
        }
        return 2 * n;
    }
    case EVOL_DBG_DISS: {
        if (dst && cap >= 5 * n * 4) {
            std::vector<int32_t> orig(n);
            cudaMemcpy(orig.data(), c->d.orig, n * 4, cudaMemcpyDeviceToHost);
            const float *src[5] = {c->d.divv_h, c->d.curlv_h, nullptr, c->d.vsig, c->d.lapu};
            std::vector<float> a(n);
            std::vector<float4> ds(n);
            cudaMemcpy(ds.data(), c->d.diss, n * 16, cudaMemcpyDeviceToHost);
            float *o = (float *)dst;
            for (int k = 0; k < 5; ++k) {
                if (src[k]) cudaMemcpy(a.data(), src[k], n * 4, cudaMemcpyDeviceToHost);
                for (int64_t s = 0; s < n; ++s) o[k * n + orig[s]] = src[k] ? a[s] : ds[s].y;
            }
        }
        return 5 * n;
    }
    case EVOL_DBG_HASHES:
    case EVOL_DBG_COUNTS: {
        int64_t esz = what == EVOL_DBG_HASHES ? 8 : 4;
        if (dst && cap >= 3 * n * esz) {
            std::vector<int32_t> orig(n);
            cudaMemcpy(orig.data(), c->d.orig, n * 4, cudaMemcpyDeviceToHost);
            if (what == EVOL_DBG_HASHES) {
                std::vector<unsigned long long> hs(3 * n);
                cudaMemcpy(hs.data(), c->d.hash3, 3 * n * 8, cudaMemcpyDeviceToHost);
                unsigned long long *o = (unsigned long long *)dst;
                for (int64_t s = 0; s < n; ++s)
                    for (int k = 0; k < 3; ++k) o[3 * (int64_t)orig[s] + k] = hs[3 * s + k];
            } else {
                std::vector<int32_t> hs(3 * n);
                cudaMemcpy(hs.data(), c->d.cnt3, 3 * n * 4, cudaMemcpyDeviceToHost);
                int32_t *o = (int32_t *)dst;
                for (int64_t s = 0; s < n; ++s)
                    for (int k = 0; k < 3; ++k) o[3 * (int64_t)orig[s] + k] = hs[3 * s + k];
            }
        }
        return 3 * n;
    }
    default:
        return EVOL_EINVAL;
    }
}

}  // extern "C"
