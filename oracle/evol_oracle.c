/*
 * FP64 CPU oracle for the EvoL Tree+SPH force step (Merlin et al., arXiv:0912.1786).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct reference
 * that the CUDA library is checked against.  It shares no code, header, table or helper
 * with the CUDA path and must never be linked into it.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark load it.
 *
 * Everything is double precision.  Inputs arrive as the same float arrays the GPU sees
 * and are promoted to double on entry.  Each routine states the passage of the paper it
 * follows; where the paper is ambiguous or garbled the reading taken is stated at the
 * routine ("Reading: ...").
 *
 * Notation follows the paper: W is the M4 spline kernel (Eq. spline), phi the softened
 * potential kernel (Eq. softphi), phi' its radial derivative (Eq. softforce), dphi/deps
 * its softening derivative (Eq. dphidh), n the number density (Eq. rho0 / Eq. nsum),
 * eps = eta n^{-1/3} (Eq. etan), h = eta n^{-1/3} (Eq. hn), Upsilon/xi the adaptive
 * softening correction terms (Sect. 2.1), Omega* and zeta the variable-mass grad-h terms
 * (Sect. 3, Eq. drhodr), Pi the Monaghan artificial viscosity (Eq. mu_visc) or its signal-velocity
 * form (Eqs. pvsig, vsig) with the Balsara limiter and per-particle alpha, Pi^u the artificial
 * conductivity (Sect. 3.3.3).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXLEVEL 21          /* 21 bits per axis -> 63-bit keys */
#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------------------ */
/* Kernel functions                                                                      */
/* ------------------------------------------------------------------------------------ */

/* Eq. spline: W(r,h) = 1/(pi h^3) * {1 - 3/2 u^2 + 3/4 u^3 ; 1/4 (2-u)^3 ; 0}, u = r/h. */
double orc_W(double r, double h)
{
    double u = r / h, w;
    if (u < 1.0)
        w = 1.0 - 1.5 * u * u + 0.75 * u * u * u;
    else if (u < 2.0)
        w = 0.25 * (2.0 - u) * (2.0 - u) * (2.0 - u);
    else
        w = 0.0;
    return w / (ORC_PI * h * h * h);
}

/* dW/dr of Eq. spline at fixed h (exact derivative of the spline). */
double orc_dWdr(double r, double h)
{
    double u = r / h, dw;
    if (u < 1.0)
        dw = -3.0 * u + 2.25 * u * u;
    else if (u < 2.0)
        dw = -0.75 * (2.0 - u) * (2.0 - u);
    else
        dw = 0.0;
    return dw / (ORC_PI * h * h * h * h);
}

/* dW/dh of Eq. spline at fixed r: -(3 w(u) + u w'(u)) / (pi h^4). */
double orc_dWdh(double r, double h)
{
    double u = r / h, w, dw;
    if (u < 1.0) {
        w = 1.0 - 1.5 * u * u + 0.75 * u * u * u;
        dw = -3.0 * u + 2.25 * u * u;
    } else if (u < 2.0) {
        w = 0.25 * (2.0 - u) * (2.0 - u) * (2.0 - u);
        dw = -0.75 * (2.0 - u) * (2.0 - u);
    } else {
        return 0.0;
    }
    return -(3.0 * w + u * dw) / (ORC_PI * h * h * h * h);
}

/* Thomas & Couchman modified kernel gradient (Sect. 3, footnote to Eqs. motionvarmass and
 * thermalvarmass): dW/dr = -1/(4 pi h^4) * {4 ; 3u(4-3u) ; 3(2-u)^2 ; 0} with the branch
 * points u = 2/3, 1, 2.  Reading: the printed form lacks the 1/h^4 factor; it is restored so
 * that the expression equals the exact dW/dr for u >= 2/3. */
double orc_dWdr_tc(double r, double h)
{
    double u = r / h, g;
    if (u < 2.0 / 3.0)
        g = 4.0;
    else if (u < 1.0)
        g = 3.0 * u * (4.0 - 3.0 * u);
    else if (u < 2.0)
        g = 3.0 * (2.0 - u) * (2.0 - u);
    else
        g = 0.0;
    return -g / (4.0 * ORC_PI * h * h * h * h);
}

/* Eq. softphi: softened potential kernel phi(r, eps); phi -> -1/r for u >= 2. */
double orc_phi(double r, double eps)
{
    double u = r / eps;
    if (u < 1.0) {
        double u2 = u * u;
        return (2.0 / 3.0 * u2 - 0.3 * u2 * u2 + 0.1 * u2 * u2 * u - 1.4) / eps;
    } else if (u < 2.0) {
        double u2 = u * u;
        return (4.0 / 3.0 * u2 - u2 * u + 0.3 * u2 * u2 - u2 * u2 * u / 30.0 - 1.6 + 1.0 / (15.0 * u)) / eps;
    }
    return -1.0 / r;
}

/* Eq. softforce: phi'(r, eps) = dphi/dr; equals 1/r^2 for u >= 2. */
double orc_dphidr(double r, double eps)
{
    double u = r / eps;
    if (u < 1.0) {
        double u2 = u * u;
        return (4.0 / 3.0 * u - 1.2 * u2 * u + 0.5 * u2 * u2) / (eps * eps);
    } else if (u < 2.0) {
        double u2 = u * u;
        return (8.0 / 3.0 * u - 3.0 * u2 + 1.2 * u2 * u - u2 * u2 / 6.0 - 1.0 / (15.0 * u2)) / (eps * eps);
    }
    return 1.0 / (r * r);
}

/* Eq. dphidh: dphi/deps at fixed r.  Reading: the 1 <= u < 2 branch is printed with +3/2 u^4;
 * the sign is taken as -3/2 u^4, the only choice for which dphi/deps = -(f + u f')/eps^2 with
 * f = eps*phi, which is continuous at u = 1 and vanishes at u = 2. */
double orc_dphideps(double r, double eps)
{
    double u = r / eps;
    if (u < 1.0) {
        double u2 = u * u;
        return (-2.0 * u2 + 1.5 * u2 * u2 - 0.6 * u2 * u2 * u + 1.4) / (eps * eps);
    } else if (u < 2.0) {
        double u2 = u * u;
        return (-4.0 * u2 + 4.0 * u2 * u - 1.5 * u2 * u2 + 0.2 * u2 * u2 * u + 1.6) / (eps * eps);
    }
    return 0.0;
}

/* eta from the ideal neighbour number, N_nei = 4/3 pi (2 eta)^3 (Sect. 2.1, below Eq. etan). */
double orc_eta_from_nnei(double n_nei)
{
    return 0.5 * cbrt(3.0 * n_nei / (4.0 * ORC_PI));
}

/* splitmix64 finaliser (Steele, Lea & Flood 2014), used only to form order-independent
 * hashes of interaction sets. */
static uint64_t orc_mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t orc_hash_id(uint64_t id) { return orc_mix64(id); }

/* ------------------------------------------------------------------------------------ */
/* Tree (Sect. 2.2): cubes halved recursively; built here from sorted 63-bit Morton keys.  */
/* ------------------------------------------------------------------------------------ */

typedef struct orc_tree {
    int64_t n, n_gas;
    int leaf;                            /* a node is split while count > leaf and level < 21 */
    double *x, *y, *z, *m;               /* original order, promoted to double */
    double corner[3], side;              /* root cube [corner, corner + side)^3 */
    uint64_t *key;                       /* original order */
    int32_t *perm;                       /* sorted position -> original index */
    int64_t nnodes, cap;
    int32_t *nbeg, *nend, *nlev, *nnext, *nnch;
    double *M, *com, *Q, *cgeo, *l, *delta, *bmin, *bmax;   /* com/cgeo/bmin/bmax: 3 per node; Q: 6 */
    double *epsmax, *hmax;
    int32_t *hasgas;
    /* per-particle lengths used by the force walk (original order) */
    double *eps, *h;
} orc_tree;

/* Root cube (Sect. 2.2 "sequence of cubes"): corner = per-axis minimum of the positions,
 * side = smallest power of two >= (largest extent) * (1 + 2^-20); side = 1 if all particles
 * coincide.  Computed from the float inputs exactly (float min/max, double difference). */
static void orc_root_cube(orc_tree *t, const float *x, const float *y, const float *z)
{
    const float *p[3] = {x, y, z};
    double ext = 0.0;
    for (int a = 0; a < 3; ++a) {
        float lo = p[a][0], hi = p[a][0];
        for (int64_t i = 1; i < t->n; ++i) {
            if (p[a][i] < lo) lo = p[a][i];
            if (p[a][i] > hi) hi = p[a][i];
        }
        t->corner[a] = (double)lo;
        double e = (double)hi - (double)lo;
        if (e > ext) ext = e;
    }
    double target = ext * (1.0 + ldexp(1.0, -20));
    double s = 1.0;
    if (target > 0.0) {
        int ex;
        double fr = frexp(target, &ex);      /* target = fr * 2^ex, fr in [0.5, 1) */
        s = (fr == 0.5) ? ldexp(1.0, ex - 1) : ldexp(1.0, ex);
    }
    t->side = s;
}

/* Morton key: q_a = clamp(floor((x_a - corner_a) * 2^21 / side), 0, 2^21 - 1); bits interleaved
 * with x the most significant of each triplet.  Level-l cell digit = bits [3(21-l), 3(21-l)+3). */
static uint64_t orc_key_of(const orc_tree *t, double x, double y, double z)
{
    double v[3] = {x, y, z};
    uint64_t q[3];
    for (int a = 0; a < 3; ++a) {
        double s = floor((v[a] - t->corner[a]) * ldexp(1.0, ORC_MAXLEVEL) / t->side);
        if (s < 0.0) s = 0.0;
        if (s > (double)((1u << ORC_MAXLEVEL) - 1)) s = (double)((1u << ORC_MAXLEVEL) - 1);
        q[a] = (uint64_t)s;
    }
    uint64_t k = 0;
    for (int b = ORC_MAXLEVEL - 1; b >= 0; --b) {
        k = (k << 3) | (((q[0] >> b) & 1u) << 2) | (((q[1] >> b) & 1u) << 1) | ((q[2] >> b) & 1u);
    }
    return k;
}

static const uint64_t *orc_sort_keys_ref;
static int orc_cmp_perm(const void *pa, const void *pb)
{
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    uint64_t ka = orc_sort_keys_ref[a], kb = orc_sort_keys_ref[b];
    if (ka < kb) return -1;
    if (ka > kb) return 1;
    return (a > b) - (a < b);       /* ties by original index: a stable sort */
}

static int orc_digit(uint64_t key, int level)   /* octant of the level-`level` cell, level >= 1 */
{
    return (int)((key >> (3 * (ORC_MAXLEVEL - level))) & 7u);
}

/* Recursive subdivision in pre-order (Sect. 2.2): a cube is split into its non-empty octants
 * while it holds more than `leaf` particles and is above the finest level. */
static int orc_split(orc_tree *t, int level, int64_t b, int64_t e)
{
    if (t->nnodes >= t->cap) return -1;
    int64_t id = t->nnodes++;
    t->nbeg[id] = (int32_t)b;
    t->nend[id] = (int32_t)e;
    t->nlev[id] = level;
    t->nnch[id] = 0;
    if (e - b > t->leaf && level < ORC_MAXLEVEL) {
        int64_t s = b;
        while (s < e) {
            int d = orc_digit(t->key[t->perm[s]], level + 1);
            int64_t u = s;
            while (u < e && orc_digit(t->key[t->perm[u]], level + 1) == d) ++u;
            if (orc_split(t, level + 1, s, u) != 0) return -1;
            t->nnch[id] += 1;
            s = u;
        }
    }
    t->nnext[id] = (int32_t)t->nnodes;     /* first node after this subtree */
    return 0;
}

/* Node moments by direct summation over the node's particles (Sect. 2.2: mass, centre of
 * mass and quadrupole; Eq. opcrit: delta = |geometric centre - centre of mass|).
 * Q_ab = sum m (3 d_a d_b - d^2 delta_ab), d = x - com; order xx, yy, zz, xy, xz, yz. */
static void orc_moments(orc_tree *t, int64_t id)
{
    int64_t b = t->nbeg[id], e = t->nend[id];
    double M = 0, cx = 0, cy = 0, cz = 0;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    int hg = 0;
    for (int64_t s = b; s < e; ++s) {
        int64_t j = t->perm[s];
        double p[3] = {t->x[j], t->y[j], t->z[j]};
        M += t->m[j];
        cx += t->m[j] * p[0];
        cy += t->m[j] * p[1];
        cz += t->m[j] * p[2];
        for (int a = 0; a < 3; ++a) {
            if (p[a] < lo[a]) lo[a] = p[a];
            if (p[a] > hi[a]) hi[a] = p[a];
        }
        if (j < t->n_gas) hg = 1;
    }
    double com[3];
    if (M > 0) {
        com[0] = cx / M; com[1] = cy / M; com[2] = cz / M;
    } else {   /* massless node: use the particle box centre */
        for (int a = 0; a < 3; ++a) com[a] = 0.5 * (lo[a] + hi[a]);
    }
    double q[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t s = b; s < e; ++s) {
        int64_t j = t->perm[s];
        double d[3] = {t->x[j] - com[0], t->y[j] - com[1], t->z[j] - com[2]};
        double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        q[0] += t->m[j] * (3 * d[0] * d[0] - d2);
        q[1] += t->m[j] * (3 * d[1] * d[1] - d2);
        q[2] += t->m[j] * (3 * d[2] * d[2] - d2);
        q[3] += t->m[j] * 3 * d[0] * d[1];
        q[4] += t->m[j] * 3 * d[0] * d[2];
        q[5] += t->m[j] * 3 * d[1] * d[2];
    }
    double side = ldexp(t->side, -t->nlev[id]);
    uint64_t k = t->key[t->perm[b]];
    double dd = 0;
    for (int a = 0; a < 3; ++a) {
        /* integer cell coordinate of this node along axis a */
        uint64_t qa = 0;
        for (int lev = 1; lev <= t->nlev[id]; ++lev) {
            int dig = orc_digit(k, lev);
            qa = (qa << 1) | (uint64_t)((dig >> (2 - a)) & 1);
        }
        t->cgeo[3 * id + a] = t->corner[a] + ((double)qa + 0.5) * side;
        t->com[3 * id + a] = com[a];
        t->bmin[3 * id + a] = lo[a];
        t->bmax[3 * id + a] = hi[a];
        dd += (com[a] - t->cgeo[3 * id + a]) * (com[a] - t->cgeo[3 * id + a]);
    }
    t->M[id] = M;
    memcpy(&t->Q[6 * id], q, sizeof q);
    t->l[id] = side;
    t->delta[id] = sqrt(dd);
    t->hasgas[id] = hg;
}

void orc_free(orc_tree *t)
{
    if (!t) return;
    void *ptrs[] = {t->x, t->y, t->z, t->m, t->key, t->perm, t->nbeg, t->nend, t->nlev, t->nnext,
                    t->nnch, t->M, t->com, t->Q, t->cgeo, t->l, t->delta, t->bmin, t->bmax,
                    t->epsmax, t->hmax, t->hasgas, t->eps, t->h};
    for (size_t i = 0; i < sizeof ptrs / sizeof ptrs[0]; ++i) free(ptrs[i]);
    free(t);
}

/* Build keys, the sorted permutation, the pre-order node list and every node's moments.
 * Returns NULL on bad arguments or allocation failure. */
orc_tree *orc_build(int64_t n, int64_t n_gas, const float *x, const float *y, const float *z,
                    const float *m, int leaf)
{
    if (n <= 0 || n_gas < 0 || n_gas > n || leaf < 1 || n > 0x7fffffff) return NULL;
    orc_tree *t = (orc_tree *)calloc(1, sizeof *t);
    if (!t) return NULL;
    t->n = n;
    t->n_gas = n_gas;
    t->leaf = leaf;
    t->x = malloc(n * sizeof(double));
    t->y = malloc(n * sizeof(double));
    t->z = malloc(n * sizeof(double));
    t->m = malloc(n * sizeof(double));
    t->key = malloc(n * sizeof(uint64_t));
    t->perm = malloc(n * sizeof(int32_t));
    t->eps = calloc(n, sizeof(double));
    t->h = calloc(n, sizeof(double));
    if (!t->x || !t->y || !t->z || !t->m || !t->key || !t->perm || !t->eps || !t->h) goto fail;
    for (int64_t i = 0; i < n; ++i) {
        t->x[i] = x[i]; t->y[i] = y[i]; t->z[i] = z[i]; t->m[i] = m[i];
    }
    orc_root_cube(t, x, y, z);
    for (int64_t i = 0; i < n; ++i) {
        t->key[i] = orc_key_of(t, t->x[i], t->y[i], t->z[i]);
        t->perm[i] = (int32_t)i;
    }
    orc_sort_keys_ref = t->key;
    qsort(t->perm, (size_t)n, sizeof(int32_t), orc_cmp_perm);

    t->cap = 22 * n + 1;   /* every particle lies in at most 22 nodes */
    t->nbeg = malloc(t->cap * sizeof(int32_t));
    t->nend = malloc(t->cap * sizeof(int32_t));
    t->nlev = malloc(t->cap * sizeof(int32_t));
    t->nnext = malloc(t->cap * sizeof(int32_t));
    t->nnch = malloc(t->cap * sizeof(int32_t));
    if (!t->nbeg || !t->nend || !t->nlev || !t->nnext || !t->nnch) goto fail;
    if (orc_split(t, 0, 0, n) != 0) goto fail;
    int64_t nn = t->nnodes;
    t->M = malloc(nn * sizeof(double));
    t->com = malloc(3 * nn * sizeof(double));
    t->Q = malloc(6 * nn * sizeof(double));
    t->cgeo = malloc(3 * nn * sizeof(double));
    t->l = malloc(nn * sizeof(double));
    t->delta = malloc(nn * sizeof(double));
    t->bmin = malloc(3 * nn * sizeof(double));
    t->bmax = malloc(3 * nn * sizeof(double));
    t->epsmax = calloc(nn, sizeof(double));
    t->hmax = calloc(nn, sizeof(double));
    t->hasgas = malloc(nn * sizeof(int32_t));
    if (!t->M || !t->com || !t->Q || !t->cgeo || !t->l || !t->delta || !t->bmin || !t->bmax ||
        !t->epsmax || !t->hmax || !t->hasgas) goto fail;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t id = 0; id < nn; ++id) orc_moments(t, id);
    return t;
fail:
    orc_free(t);
    return NULL;
}

/* ---- accessors for the tests ---------------------------------------------------------- */
int64_t orc_nnodes(const orc_tree *t) { return t->nnodes; }
void orc_get_cube(const orc_tree *t, double *corner, double *side)
{
    memcpy(corner, t->corner, 3 * sizeof(double));
    *side = t->side;
}
void orc_get_keys(const orc_tree *t, uint64_t *out) { memcpy(out, t->key, t->n * sizeof(uint64_t)); }
void orc_get_perm(const orc_tree *t, int32_t *out) { memcpy(out, t->perm, t->n * sizeof(int32_t)); }
void orc_get_nodes(const orc_tree *t, int32_t *beg, int32_t *end, int32_t *lev, int32_t *next, int32_t *nch)
{
    int64_t nn = t->nnodes;
    memcpy(beg, t->nbeg, nn * 4);
    memcpy(end, t->nend, nn * 4);
    memcpy(lev, t->nlev, nn * 4);
    memcpy(next, t->nnext, nn * 4);
    memcpy(nch, t->nnch, nn * 4);
}
void orc_get_moments(const orc_tree *t, double *M, double *com, double *Q, double *delta,
                     double *bmin, double *bmax, double *cgeo, double *l)
{
    int64_t nn = t->nnodes;
    memcpy(M, t->M, nn * 8);
    memcpy(com, t->com, 3 * nn * 8);
    memcpy(Q, t->Q, 6 * nn * 8);
    memcpy(delta, t->delta, nn * 8);
    memcpy(bmin, t->bmin, 3 * nn * 8);
    memcpy(bmax, t->bmax, 3 * nn * 8);
    memcpy(cgeo, t->cgeo, 3 * nn * 8);
    memcpy(l, t->l, nn * 8);
}

/* ------------------------------------------------------------------------------------ */
/* Geometry with optional periodic axes (Sect. 4.3: SPH periodicity by nearest image).    */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    int mask;            /* bit a set: axis a periodic */
    double lo[3], len[3];
} orc_period;

static double orc_wrap(const orc_period *pp, int a, double d)
{
    if (pp && (pp->mask >> a) & 1) d -= pp->len[a] * nearbyint(d / pp->len[a]);
    return d;
}

/* Squared distance from point p to the node's particle bounding box (nearest image on
 * periodic axes). */
static double orc_box_dist2(const orc_tree *t, const orc_period *pp, int64_t id, const double *p)
{
    double s = 0;
    for (int a = 0; a < 3; ++a) {
        double c = 0.5 * (t->bmin[3 * id + a] + t->bmax[3 * id + a]);
        double w = 0.5 * (t->bmax[3 * id + a] - t->bmin[3 * id + a]);
        double d = fabs(orc_wrap(pp, a, p[a] - c)) - w;
        if (d > 0) s += d * d;
    }
    return s;
}

/* Collect every particle j (species filter: gas_only) with |r_ij| < R by a tree range search
 * (Sect. 2.2, last paragraph: neighbour lists from the tree walk).  Returns the count, or -1
 * if cap is exceeded. */
static int64_t orc_gather(const orc_tree *t, const orc_period *pp, const double *p, double R,
                          int gas_only, int64_t *out, double *out_r, int64_t cap)
{
    int64_t cnt = 0, id = 0, nn = t->nnodes;
    while (id < nn) {
        if (orc_box_dist2(t, pp, id, p) >= R * R || (gas_only && !t->hasgas[id])) {
            id = t->nnext[id];
            continue;
        }
        if (t->nnch[id] == 0) {
            for (int64_t s = t->nbeg[id]; s < t->nend[id]; ++s) {
                int64_t j = t->perm[s];
                if (gas_only && j >= t->n_gas) continue;
                double dx = orc_wrap(pp, 0, p[0] - t->x[j]);
                double dy = orc_wrap(pp, 1, p[1] - t->y[j]);
                double dz = orc_wrap(pp, 2, p[2] - t->z[j]);
                double r = sqrt(dx * dx + dy * dy + dz * dz);
                if (r < R) {
                    if (cnt >= cap) return -1;
                    out[cnt] = j;
                    out_r[cnt] = r;
                    ++cnt;
                }
            }
            id = t->nnext[id];
        } else {
            id = id + 1;
        }
    }
    return cnt;
}

/* ------------------------------------------------------------------------------------ */
/* Smoothing / softening length (Eqs. rho0, etan, hn, nsum, iter).                        */
/* ------------------------------------------------------------------------------------ */

/* The length is the root of F(L) = L^3 n(L) - eta^3, n(L) = sum_j W(r_ij, L) including j = i.
 * F is non-decreasing (L^3 W(r, L) = w(r/L)/pi), so the root is unique; it is found by
 * bisection to |dL| <= 1e-13 L.  Reading: the paper's f = |n_i - n_sum| (Eq. iter) has the
 * same root; its tolerance 1e-2..1e-3 is replaced by a tight one for reference use.
 *
 * mode 0: h of a gas particle from gas neighbours; outputs n, rho = sum m_j W (Eq. densitySPH),
 *         Omega* = 1 - (dh/dn) sum dW/dh, zeta = (dh/dn) sum m_j dW/dh (Sect. 3, Eq. drhodr).
 * mode 1: eps of any particle from all neighbours; outputs n, Upsilon = 1 - (deps/dn) sum dW/deps
 *         (Sect. 2.1) and X = (deps/dn) sum_k m_k dphi_ik/deps, self term included.
 *         Reading: the paper's xi (Eq. zeta) carries no mass; re-deriving the equation of motion
 *         from L_grav (Eq. Lgrav) for unequal masses gives the mass-weighted X, which equals
 *         m * xi for equal masses.  The double sum in L_grav includes k = j, so X does too.
 * Returns 0, or -2 if no root exists (too few particles), -3 on neighbour overflow. */
static int orc_cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* The "standard SPH scheme" of Sect. 3 (the alternative to the n-h relation): h is chosen so that
 * a fixed number N of gas particles, the particle itself included, lies inside the kernel's
 * support sphere r < 2h, and the grad-h terms are dropped (Omega* = 1, zeta = 0).  Reading: the
 * sphere is the kernel support 2h, which keeps N the same neighbour number as in
 * N = 4/3 pi (2 eta)^3 of the n-h scheme; any 2h in (r_(N), r_(N+1)] holds exactly N particles
 * (r_(k): the k-th smallest distance, r_(1) = 0 the particle itself), and the midpoint
 * h = (r_(N) + r_(N+1)) / 4 is taken, the choice farthest from changing the count.  Then n and rho
 * are the usual kernel sums at that h.  out as orc_solve_one, mode 0. */
static int orc_solve_standard(const orc_tree *t, const orc_period *pp, int nstd, int64_t i, double guess,
                              double *out, int64_t *scratch, double *rscr, int64_t cap)
{
    double p[3] = {t->x[i], t->y[i], t->z[i]};
    double R = (guess > 0 ? 2.0 * guess * 1.25 : 2.0 * t->side / cbrt((double)t->n));
    double span = t->side * 4.0;
    int64_t cnt;
    for (;;) {
        cnt = orc_gather(t, pp, p, R, 1, scratch, rscr, cap);
        if (cnt < 0) return -3;
        if (cnt >= nstd + 1) break;
        if (R > span) return -2;         /* fewer than N + 1 gas particles in reach */
        R *= 2.0;
    }
    /* every particle closer than the (N+1)-th is inside R: sort the distances (indices follow) */
    double *rs = malloc(cnt * sizeof(double));
    if (!rs) return -3;
    memcpy(rs, rscr, cnt * sizeof(double));
    qsort(rs, cnt, sizeof(double), orc_cmp_double);
    double L = 0.25 * (rs[nstd - 1] + rs[nstd]);
    free(rs);
    double nsum = 0, rho = 0;
    for (int64_t k = 0; k < cnt; ++k) {
        nsum += orc_W(rscr[k], L);
        rho += t->m[scratch[k]] * orc_W(rscr[k], L);
    }
    out[0] = L;
    out[1] = nsum;
    out[2] = rho;
    out[3] = 1.0;      /* Omega*: grad-h terms dropped */
    out[4] = 0.0;      /* zeta */
    return 0;
}

static int orc_solve_one(const orc_tree *t, const orc_period *pp, int mode, double eta, int64_t i,
                         double guess, double *out /* [5] */, int64_t *scratch, double *rscr, int64_t cap)
{
    double p[3] = {t->x[i], t->y[i], t->z[i]};
    double eta3 = eta * eta * eta;
    int gas_only = (mode == 0);
    double R = (guess > 0 ? 2.0 * guess * 1.25 : 2.0 * t->side / cbrt((double)t->n));
    double span = t->side * 4.0;
    int64_t cnt;
    double lo = 0.0;
    for (;;) {
        cnt = orc_gather(t, pp, p, R, gas_only, scratch, rscr, cap);
        if (cnt < 0) return -3;
        double hi = 0.5 * R, F = -eta3;
        for (int64_t k = 0; k < cnt; ++k) F += orc_W(rscr[k], hi) * hi * hi * hi;
        if (F >= 0) break;
        lo = hi;
        if (R > span) return -2;
        R *= 2.0;
    }
    double hi = 0.5 * R;
    while (hi - lo > 1e-13 * hi) {
        double mid = 0.5 * (lo + hi), F = -eta3;
        for (int64_t k = 0; k < cnt; ++k) F += orc_W(rscr[k], mid) * mid * mid * mid;
        if (F >= 0) hi = mid; else lo = mid;
    }
    double L = 0.5 * (lo + hi);
    double nsum = 0, s_dW = 0, s_mdW = 0, rho = 0, s_mdphi = 0;
    for (int64_t k = 0; k < cnt; ++k) {
        int64_t j = scratch[k];
        double r = rscr[k];
        nsum += orc_W(r, L);
        s_dW += orc_dWdh(r, L);
        s_mdW += t->m[j] * orc_dWdh(r, L);
        rho += t->m[j] * orc_W(r, L);
        s_mdphi += t->m[j] * orc_dphideps(r, L);
    }
    double dLdn = -L / (3.0 * nsum);      /* derivative of Eq. etan / Eq. hn */
    out[0] = L;
    out[1] = nsum;
    if (mode == 0) {
        out[2] = rho;
        out[3] = 1.0 - dLdn * s_dW;      /* Omega* */
        out[4] = dLdn * s_mdW;           /* zeta   */
    } else {
        out[2] = 1.0 - dLdn * s_dW;      /* Upsilon */
        out[3] = dLdn * s_mdphi;         /* X       */
        out[4] = 0.0;
    }
    return 0;
}

/* Solve for the particles listed in idx (all particles of the mode's species if idx == NULL).
 * mode 0: gas h from the n-h relation; 1: eps; 2: gas h of the standard scheme with
 * N = n_nei (rounded) neighbours.  guess: original-order float array of starting lengths (may be
 * NULL).  Outputs are written at the particle's original index in out0..out4 (arrays of length
 * n).  Returns 0 or the first error code met. */
int orc_solve_lengths(const orc_tree *t, int mode, double n_nei, const int64_t *idx, int64_t nidx,
                      const float *guess, int periodic_mask, const double *plo, const double *phi_,
                      double *out0, double *out1, double *out2, double *out3, double *out4)
{
    double eta = orc_eta_from_nnei(n_nei);
    orc_period per = {periodic_mask, {0, 0, 0}, {1, 1, 1}};
    for (int a = 0; a < 3; ++a)
        if ((periodic_mask >> a) & 1) { per.lo[a] = plo[a]; per.len[a] = phi_[a] - plo[a]; }
    int64_t count = idx ? nidx : (mode != 1 ? t->n_gas : t->n);
    int nstd = (int)nearbyint(n_nei);
    int err = 0;
#pragma omp parallel
    {
        int64_t cap = 1 << 16;
        int64_t *scr = malloc(cap * sizeof(int64_t));
        double *rs = malloc(cap * sizeof(double));
#pragma omp for schedule(dynamic, 64)
        for (int64_t q = 0; q < count; ++q) {
            int64_t i = idx ? idx[q] : q;
            double o[5];
            double gs = guess ? guess[i] : 0.0;
            int rc = !(scr && rs) ? -3
                     : mode == 2  ? orc_solve_standard(t, &per, nstd, i, gs, o, scr, rs, cap)
                                  : orc_solve_one(t, &per, mode, eta, i, gs, o, scr, rs, cap);
            if (rc != 0) {
#pragma omp critical
                if (!err) err = rc;
                continue;
            }
            out0[i] = o[0]; out1[i] = o[1]; out2[i] = o[2]; out3[i] = o[3];
            if (out4) out4[i] = o[4];
        }
        free(scr);
        free(rs);
    }
    return err;
}

/* Velocity divergence at every listed particle from the discretised continuity equation
 * (Sect. 2.1, the equations below Eq. continuity): with n_i = sum_j W(r_ij, L_i),
 *     div v_i = -1/(n_i C_i) sum_j (v_i - v_j) . grad_i W(r_ij, L_i),
 * and, when curl != NULL, the magnitude of the curl from the same neighbour sum (the rotational
 * part of the velocity field that the Balsara limiter of Sect. 3.3.3 needs):
 *     curl v_i = +1/(n_i C_i) sum_j (v_i - v_j) x grad_i W(r_ij, L_i)
 * (for v = w x r the sum gives 2 w, for v = k r it gives -3 k in div v; the signs follow from
 * the kernel's second moment, sum_j (1/n) x_a x_b dW/dr / r = -delta_ab),
 * where L is the particle's solved length and C its correction factor: Upsilon for the softening
 * (mode 1, all species) and Omega* for the smoothing length (mode 0, gas neighbours of gas).
 * grad_i W = (r_i - r_j)/r dW/dr with the exact spline derivative.  L, nsum, corr: original order
 * (as orc_solve_lengths returns them); idx: particles to evaluate (all of the mode's species if
 * NULL).  Returns 0, or -3 on neighbour overflow. */
int orc_divv(const orc_tree *t, int mode, const double *L, const double *nsum, const double *corr,
             const double *vx, const double *vy, const double *vz, const int64_t *idx, int64_t nidx,
             int periodic_mask, const double *plo, const double *phi_, double *divv, double *curl)
{
    orc_period per = {periodic_mask, {0, 0, 0}, {1, 1, 1}};
    for (int a = 0; a < 3; ++a)
        if ((periodic_mask >> a) & 1) { per.lo[a] = plo[a]; per.len[a] = phi_[a] - plo[a]; }
    int64_t count = idx ? nidx : (mode == 0 ? t->n_gas : t->n);
    int err = 0;
#pragma omp parallel
    {
        int64_t cap = 1 << 16;
        int64_t *scr = malloc(cap * sizeof(int64_t));
        double *rs = malloc(cap * sizeof(double));
#pragma omp for schedule(dynamic, 64)
        for (int64_t q = 0; q < count; ++q) {
            int64_t i = idx ? idx[q] : q;
            double p[3] = {t->x[i], t->y[i], t->z[i]};
            int64_t cnt = (scr && rs) ? orc_gather(t, &per, p, 2.0 * L[i], mode == 0, scr, rs, cap) : -1;
            if (cnt < 0) {
#pragma omp critical
                if (!err) err = -3;
                continue;
            }
            double s = 0.0, cv[3] = {0.0, 0.0, 0.0};
            for (int64_t k = 0; k < cnt; ++k) {
                int64_t j = scr[k];
                double r = rs[k];
                if (j == i || r <= 0.0) continue;
                double rv[3] = {orc_wrap(&per, 0, p[0] - t->x[j]), orc_wrap(&per, 1, p[1] - t->y[j]),
                                orc_wrap(&per, 2, p[2] - t->z[j])};
                double dv[3] = {vx[i] - vx[j], vy[i] - vy[j], vz[i] - vz[j]};
                double g = orc_dWdr(r, L[i]) / r;           /* grad_i W = r_vec g */
                s += (dv[0] * rv[0] + dv[1] * rv[1] + dv[2] * rv[2]) * g;
                cv[0] += (dv[1] * rv[2] - dv[2] * rv[1]) * g;
                cv[1] += (dv[2] * rv[0] - dv[0] * rv[2]) * g;
                cv[2] += (dv[0] * rv[1] - dv[1] * rv[0]) * g;
            }
            divv[i] = -s / (nsum[i] * corr[i]);
            if (curl) curl[i] = sqrt(cv[0] * cv[0] + cv[1] * cv[1] + cv[2] * cv[2]) / (nsum[i] * corr[i]);
        }
        free(scr);
        free(rs);
    }
    return err;
}

/* ------------------------------------------------------------------------------------ */
/* Periodic gravity by the Ewald method (Sect. 4.3).                                        */
/* ------------------------------------------------------------------------------------ */

#define ORC_EWALD_N 64           /* table intervals per axis over the octant [0, L/2] */
#define ORC_EWALD_LMAX 0.125    /* nodes of side above this fraction of L are opened */

/* Ewald correction for a unit mass in a periodic cube of side L (Sect. 4.3, the series of
 * Hernquist et al. 1991 and Springel 2001 as printed), x = r_i - r_j (nearest image):
 *   f(x) = x/|x|^3 - sum_{|n|<5} (x - nL)/r_n^3 (erfc(w r_n) + 2 w r_n/sqrt(pi) exp(-w^2 r_n^2))
 *          - 2/L^2 sum_{0<|h|<5} h/h^2 exp(-pi^2 h^2/(w^2 L^2)) sin(2 pi h.x/L),      w = 2/L,
 * r_n = |x - nL|, n and h integer triplets; i receives G m_j f(x) beyond the nearest-image force.
 * Reading: the paper prints the acceleration only; the potential is the matching zero-mean
 * periodic one, g(x) = 1/|x| - psi(x) with
 *   psi(x) = sum_n erfc(w r_n)/r_n + 1/(pi L) sum_h exp(-pi^2 h^2/(w^2 L^2))/h^2 cos(2 pi h.x/L)
 *            - pi/(w^2 L^3),
 * so that f = -grad g and the potential of i gains G m_j g(x) (g(0), the images of i itself, is
 * finite).  Reading: |n| < 5 and |h| < 5 are Euclidean norms. */
void orc_ewald_exact(const double *x, double L, double f[3], double *g)
{
    const double w = 2.0 / L, sqpi = sqrt(ORC_PI);
    double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    double F[3] = {0, 0, 0}, psi = 0.0;
    for (int a = -4; a <= 4; ++a)
        for (int b = -4; b <= 4; ++b)
            for (int c = -4; c <= 4; ++c) {
                int n2 = a * a + b * b + c * c;
                if (n2 >= 25) continue;
                double d[3] = {x[0] - a * L, x[1] - b * L, x[2] - c * L};
                double rn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                if (n2 == 0) {
                    /* with the direct term: x/r^3 (1 - erfc - 2 w r/sqrt(pi) e^{-w^2 r^2}) and
                     * 1/r - erfc/r = erf/r; for small w r by their series */
                    double z = w * rn;
                    if (z < 1e-3) {
                        double z2 = z * z;
                        double k3 = 4.0 / (3.0 * sqpi) * w * w * w * (1.0 - 0.6 * z2);
                        for (int q = 0; q < 3; ++q) F[q] += x[q] * k3;
                        psi += 2.0 * w / sqpi * (1.0 - z2 / 3.0);
                    } else {
                        double k = (erf(z) - 2.0 * z / sqpi * exp(-z * z)) / (rn * rn * rn);
                        for (int q = 0; q < 3; ++q) F[q] += x[q] * k;
                        psi += erf(z) / rn;
                    }
                    continue;
                }
                double z = w * rn;
                double k = (erfc(z) + 2.0 * z / sqpi * exp(-z * z)) / (rn * rn * rn);
                for (int q = 0; q < 3; ++q) F[q] -= d[q] * k;
                psi -= erfc(z) / rn;
            }
    /* here F = x/r^3 - (real-space sum) and psi (accumulating g) = 1/r - (real-space sum) */
    for (int a = -4; a <= 4; ++a)
        for (int b = -4; b <= 4; ++b)
            for (int c = -4; c <= 4; ++c) {
                int h2 = a * a + b * b + c * c;
                if (h2 == 0 || h2 >= 25) continue;
                double e = exp(-ORC_PI * ORC_PI * h2 / (w * w * L * L));
                double ph = 2.0 * ORC_PI * (a * x[0] + b * x[1] + c * x[2]) / L;
                double ks = 2.0 / (L * L) * e / h2 * sin(ph);
                F[0] -= ks * a;
                F[1] -= ks * b;
                F[2] -= ks * c;
                psi -= e / (ORC_PI * L * h2) * cos(ph);
            }
    psi += ORC_PI / (w * w * L * L * L);
    (void)r;
    f[0] = F[0];
    f[1] = F[1];
    f[2] = F[2];
    *g = psi;
}

/* The table of the method (Sect. 4.3): f and g for L = 1 at the grid points (i, j, k) / (2N) of the
 * octant [0, 1/2]^3, 0 <= i, j, k <= N = ORC_EWALD_N, four values each; built once per process. */
static double *orc_ewald_tab = NULL;

const double *orc_ewald_table(void)
{
    if (orc_ewald_tab) return orc_ewald_tab;
    const int N = ORC_EWALD_N, M = N + 1;
    double *tab = malloc((size_t)M * M * M * 4 * sizeof(double));
    if (!tab) return NULL;
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j)
            for (int k = 0; k < M; ++k) {
                double x[3] = {0.5 * i / N, 0.5 * j / N, 0.5 * k / N};
                double *o = tab + 4 * (((size_t)i * M + j) * M + k);
                orc_ewald_exact(x, 1.0, o, o + 3);
            }
    orc_ewald_tab = tab;
    return tab;
}

/* Trilinear interpolation in the table (Sect. 4.3) for a nearest-image x (|x_a| <= L/2) in a cube of
 * side L: each component of f is odd in its own coordinate and even in the others, g is even, so
 * the octant table serves every x: f_a(x) = sign(x_a) F_a(|x|) / L^2, g(x) = G(|x|) / L. */
void orc_ewald_interp(double L, const double *x, double f[3], double *g)
{
    const double *tab = orc_ewald_table();
    const int N = ORC_EWALD_N, M = N + 1;
    int i0[3];
    double t[3];
    for (int a = 0; a < 3; ++a) {
        double u = fabs(x[a]) / L * 2.0 * N;
        int i = (int)floor(u);
        if (i > N - 1) i = N - 1;
        if (i < 0) i = 0;
        i0[a] = i;
        t[a] = u - i;
    }
    double v[4] = {0, 0, 0, 0};
    for (int c = 0; c < 8; ++c) {
        int di = c >> 2 & 1, dj = c >> 1 & 1, dk = c & 1;
        double wgt = (di ? t[0] : 1 - t[0]) * (dj ? t[1] : 1 - t[1]) * (dk ? t[2] : 1 - t[2]);
        const double *o = tab + 4 * (((size_t)(i0[0] + di) * M + (i0[1] + dj)) * M + (i0[2] + dk));
        for (int q = 0; q < 4; ++q) v[q] += wgt * o[q];
    }
    for (int a = 0; a < 3; ++a) f[a] = (x[a] < 0 ? -v[a] : v[a]) / (L * L);
    *g = v[3] / L;
}

/* ------------------------------------------------------------------------------------ */
/* Forces: tree walk with the Dubinski opening criterion, far nodes by monopole +          */
/* quadrupole, near particles by the softened symmetric pair force with the adaptive      */
/* softening correction, and SPH pressure + viscosity + du/dt on the same near list.       */
/* ------------------------------------------------------------------------------------ */

/* Dissipation variants of Sect. 3.3.3 (all off: the standard Monaghan viscosity with constant
 * alpha and beta).  Per-particle inputs in original order. */
typedef struct {
    int form;             /* 0: Monaghan (Eq. mu_visc); 1: signal velocity (Eqs. pvsig, vsig) */
    int balsara;          /* 1: Pi_ij multiplied by (f_i + f_j)/2, the Balsara limiter */
    int var_alpha;        /* 1: alpha_ij = (alpha_i + alpha_j)/2 (Eq. alphaswitch) */
    int conduction;       /* 1: the artificial conductivity Pi^u_ij */
    int cond_vsig;        /* signal speed of Pi^u: 0 as Eq. vsig, 1 sqrt(|P_i - P_j| / rho_ij) */
    const double *f;      /* Balsara factor f_i (balsara) */
    const double *alpha;  /* alpha_i (var_alpha) */
    const double *alpha_u;/* alpha^u_i (conduction) */
    const double *u;      /* specific internal energy u_i (conduction) */
} orc_diss;

typedef struct {
    double theta, G, gamma, alpha, beta;
    int gravity, sph, adaptive, use_tc;
    orc_diss ds;
    double ewald_L;       /* > 0: periodic gravity in a cube of this side (Ewald, Sect. 4.3) */
} orc_params;

/* Per-particle state needed by the force pass (original order, length n).  Fields of species
 * that do not apply (SPH fields of dark matter) are ignored. */
typedef struct {
    const double *vx, *vy, *vz;
    const double *eps, *ups, *X;          /* gravity: eps, Upsilon, X */
    const double *h, *rho, *P, *c, *om, *zeta;  /* SPH: h, rho, P, sound speed, Omega*, zeta */
} orc_state;

/* Node maxima of eps (all particles) and h (gas particles) used by the near test. */
void orc_set_node_lengths(orc_tree *t, const double *eps, const double *h)
{
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t id = 0; id < t->nnodes; ++id) {
        double em = 0, hm = 0;
        for (int64_t s = t->nbeg[id]; s < t->nend[id]; ++s) {
            int64_t j = t->perm[s];
            if (eps && eps[j] > em) em = eps[j];
            if (h && j < t->n_gas && h[j] > hm) hm = h[j];
        }
        t->epsmax[id] = em;
        t->hmax[id] = hm;
    }
}

typedef struct {
    double a[3], pot, dudt;
    double ahyd[3];
    uint64_t hfar, hnear, hsph;
    int64_t nfar, npp, nsph;
    double margin;      /* smallest distance of any decision from its threshold, relative to
                           (threshold + coordinate scale of the particle) */
    double scale;       /* max |coordinate| of the particle: the scale of FP32 position rounding */
    double aabs, duabs; /* sums of the magnitudes of the individual contributions to a and du/dt */
    double mumax;       /* largest |mu_ij| of the viscosity over the SPH neighbours */
    double vsig;        /* largest signal velocity v^sig_ij over the SPH neighbours */
    double lapu;        /* Brookshaw estimate of the Laplacian of u (conduction only) */
    double lapabs;      /* sum of the magnitudes of its terms */
} orc_result;

/* Distance of one decision (value v against threshold thr) from its threshold.  It is taken
 * relative to thr + the particle's coordinate scale: an FP32 evaluation of the same test rounds
 * positions, centres of mass and box bounds on the scale of the coordinates and the threshold on
 * its own scale, so a decision closer than a few FP32 ulps of that sum can go either way. */
static void orc_margin(orc_result *res, double v, double thr)
{
    if (thr > 0 && isfinite(thr)) {
        double mg = fabs(v - thr) / (thr + res->scale);
        if (mg < res->margin) res->margin = mg;
    }
}

/* One pair (i, j), j != i, with r_vec = r_i - r_j (nearest image). */
static void orc_pair(const orc_tree *t, const orc_params *pr, const orc_state *st, int64_t i, int64_t j,
                     const double *rv, orc_result *res)
{
    double r2 = rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2];
    double r = sqrt(r2);
    double mi = t->m[i], mj = t->m[j];
    if (pr->gravity) {
        double ei = st->eps[i], ej = st->eps[j];
        res->pot += pr->G * mj * orc_phi(r, ei);
        orc_margin(res, r, 2.0 * (ei > ej ? ei : ej));
        if (r > 0) {
            /* App. B, first line: symmetrised softened force. */
            double f = -pr->G * mj * 0.5 * (orc_dphidr(r, ei) + orc_dphidr(r, ej)) / r;
            if (pr->adaptive) {
                /* App. B second line, mass-weighted reading (see orc_solve_one). */
                f += -0.5 * pr->G * (st->X[i] / st->ups[i] * orc_dWdr(r, ei) +
                                     (mj / mi) * st->X[j] / st->ups[j] * orc_dWdr(r, ej)) / r;
            }
            for (int a = 0; a < 3; ++a) res->a[a] += f * rv[a];
            res->aabs += fabs(f) * r;
        }
        if (pr->ewald_L > 0) {
            /* the replicas of j beyond its nearest image (Sect. 4.3, tabulated correction) */
            double fe[3], ge;
            orc_ewald_interp(pr->ewald_L, rv, fe, &ge);
            for (int a = 0; a < 3; ++a) res->a[a] += pr->G * mj * fe[a];
            res->aabs += pr->G * mj * sqrt(fe[0] * fe[0] + fe[1] * fe[1] + fe[2] * fe[2]);
            res->pot += pr->G * mj * ge;
        }
    }
    if (pr->sph && i < t->n_gas && j < t->n_gas) {
        double hi = st->h[i], hj = st->h[j];
        double R = 2.0 * (hi > hj ? hi : hj);
        orc_margin(res, r, R);
        if (r < R) {
            res->nsph += 1;
            res->hsph += orc_hash_id((uint64_t)j);
            if (r > 0) {
                double gi = pr->use_tc ? orc_dWdr_tc(r, hi) : orc_dWdr(r, hi);
                double gj = pr->use_tc ? orc_dWdr_tc(r, hj) : orc_dWdr(r, hj);
                double fi = 1.0 + st->zeta[i] / (mj * st->om[i]);   /* (1 + zeta_i/(m_j Omega*_i)) */
                double fj = 1.0 + st->zeta[j] / (mi * st->om[j]);   /* (1 + zeta_j/(m_i Omega*_j)) */
                double Pi_ = st->P[i] / (st->rho[i] * st->rho[i]);
                double Pj_ = st->P[j] / (st->rho[j] * st->rho[j]);
                double v[3] = {st->vx[i] - st->vx[j], st->vy[i] - st->vy[j], st->vz[i] - st->vz[j]};
                double vr = v[0] * rv[0] + v[1] * rv[1] + v[2] * rv[2];
                const orc_diss *ds = &pr->ds;
                double w = vr / r;                                  /* w_ij = v_ij . r_ij / |r_ij| */
                double cb = 0.5 * (st->c[i] + st->c[j]);
                double rb = 0.5 * (st->rho[i] + st->rho[j]);
                /* Eq. vsig, v^sig = 2 cbar - w.  Reading: w enters only where the pair approaches
                 * (w < 0), so that v^sig >= c_i + c_j for every pair; for approaching pairs, the only
                 * ones the viscosity acts on, this is the printed form. */
                double vsig = 2.0 * cb - (w < 0 ? w : 0.0);
                if (vsig > res->vsig) res->vsig = vsig;
                double al = ds->var_alpha ? 0.5 * (ds->alpha[i] + ds->alpha[j]) : pr->alpha;
                /* Monaghan viscosity (Eq. mu_visc): mu = hbar v.r / (r^2 + 0.01 hbar^2); mu is formed
                 * in both forms, its largest |mu| enters the Courant criterion. */
                double Pi_visc = 0;
                if (vr < 0) {
                    double hb = 0.5 * (hi + hj);
                    double mu = hb * vr / (r2 + 0.01 * hb * hb);
                    if (fabs(mu) > res->mumax) res->mumax = fabs(mu);
                    if (ds->form == 0)
                        Pi_visc = (-al * cb * mu + pr->beta * mu * mu) / rb;
                    else
                        Pi_visc = -al * vsig * w / rb;              /* Eq. pvsig */
                    if (ds->balsara) Pi_visc *= 0.5 * (ds->f[i] + ds->f[j]);
                }
                /* grad_i W_ij(h) = dW/dr * r_vec / r; mean gradient with grad-h factors. */
                double gbar = 0.5 * (gi * fi + gj * fj);
                /* Reading: Eq. motionvarmass needs a leading minus for a repulsive pressure
                 * (re-derived from Eq. dvdt and Eq. drhodr). */
                double s = -mj * (Pi_ * fi * gi + Pj_ * fj * gj + Pi_visc * gbar) / r;
                for (int a = 0; a < 3; ++a) {
                    res->a[a] += s * rv[a];
                    res->ahyd[a] += s * rv[a];
                }
                res->aabs += fabs(s) * r;
                /* Reading: Eq. thermalvarmass with (v_i - v_j) so that compression heats;
                 * viscous heating 1/2 Pi v_ij . gradbar W >= 0. */
                res->dudt += mj * (Pi_ * fi * gi + 0.5 * Pi_visc * gbar) * vr / r;
                res->duabs += fabs(mj * (Pi_ * fi * gi + 0.5 * Pi_visc * gbar) * vr / r);
                if (ds->conduction) {
                    /* Artificial conductivity (Sect. 3.3.3):
                     *   Pi^u_ij = -alphabar^u_ij v^u_sig (u_i - u_j) / rhobar_ij,
                     * added to du_i/dt as m_j Pi^u_ij |gradbar W_ij|.  Reading: the printed factor
                     * w_ij on Pi^u is left out; with it the term would not have the units of du/dt
                     * (Pi^u carries a velocity cubed over a density), and heat would flow from cold to
                     * hot for approaching pairs.  Without it the term moves heat from the hotter
                     * particle of a pair to the colder one and conserves sum_i m_i u_i. */
                    double du_ = ds->u[i] - ds->u[j];
                    double vu = ds->cond_vsig == 0 ? vsig : sqrt(fabs(st->P[i] - st->P[j]) / rb);
                    double au = 0.5 * (ds->alpha_u[i] + ds->alpha_u[j]);
                    double Piu = -au * vu * du_ / rb;
                    res->dudt += mj * Piu * fabs(gbar);
                    res->duabs += fabs(mj * Piu * gbar);
                    /* Brookshaw's Laplacian, as printed: sum_j 2 m_j (u_i - u_j)/rho_j |gradbar W_ij| / r */
                    res->lapu += 2.0 * mj * du_ / st->rho[j] * fabs(gbar) / r;
                    res->lapabs += fabs(2.0 * mj * du_ / st->rho[j] * gbar / r);
                }
            }
        }
    }
}

/* Far node: Newtonian monopole + traceless quadrupole about the centre of mass,
 * d = r_i - com: a = -G M d/d^3 + G [Q d / d^5 - 5/2 (d.Q.d) d / d^7],
 * phi = -G M / d - G/2 (d.Q.d) / d^5. */
static void orc_far(const orc_tree *t, const orc_params *pr, const orc_period *pp, int64_t id, const double *p,
                    orc_result *res)
{
    const double *c = &t->com[3 * id], *q = &t->Q[6 * id];
    /* periodic gravity: the nearest image of the centre of mass */
    double d[3] = {p[0] - c[0], p[1] - c[1], p[2] - c[2]};
    if (pr->ewald_L > 0)
        for (int a = 0; a < 3; ++a) d[a] = orc_wrap(pp, a, d[a]);
    double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double di = 1.0 / sqrt(d2), di2 = di * di;
    double di3 = di * di2, di5 = di3 * di2, di7 = di5 * di2;
    double Qd[3] = {q[0] * d[0] + q[3] * d[1] + q[4] * d[2],
                    q[3] * d[0] + q[1] * d[1] + q[5] * d[2],
                    q[4] * d[0] + q[5] * d[1] + q[2] * d[2]};
    double dQd = d[0] * Qd[0] + d[1] * Qd[1] + d[2] * Qd[2];
    double M = t->M[id], mag = 0;
    for (int a = 0; a < 3; ++a) {
        double c = pr->G * (-M * d[a] * di3 + Qd[a] * di5 - 2.5 * dQd * d[a] * di7);
        res->a[a] += c;
        mag += c * c;
    }
    res->aabs += sqrt(mag);
    res->pot += pr->G * (-M * di - 0.5 * dQd * di5);
    if (pr->ewald_L > 0) {
        /* replicas of the node: its mass at the centre of mass (reading: the correction is taken
         * for the monopole; the quadrupole's replicas are left out) */
        double fe[3], ge;
        orc_ewald_interp(pr->ewald_L, d, fe, &ge);
        for (int a = 0; a < 3; ++a) res->a[a] += pr->G * M * fe[a];
        res->aabs += pr->G * M * sqrt(fe[0] * fe[0] + fe[1] * fe[1] + fe[2] * fe[2]);
        res->pot += pr->G * M * ge;
    }
}

/* Opening test of node id for particle i (Sect. 2.2, Eq. opcrit plus the near test).
 * Reading: a node is accepted as a far node iff |r_i - com| > l/theta + delta AND its particle
 * box lies farther than R_i = 2 max(eps_i, epsmax_node) (and, for gas i and a node holding
 * gas, farther than 2 max(h_i, hmax_node)).  Accepted nodes therefore never need softening
 * (the softened-node branch of Sect. 2.2 is not needed), and no neighbour is missed. */
static int orc_accept(const orc_tree *t, const orc_params *pr, const orc_period *pp, const orc_state *st,
                      int64_t i, int64_t id, const double *p, orc_result *res)
{
    double R = 0;
    if (pr->gravity) {
        double e = st->eps[i] > t->epsmax[id] ? st->eps[i] : t->epsmax[id];
        R = 2.0 * e;
    }
    if (pr->sph && i < t->n_gas && t->hasgas[id]) {
        double hh = st->h[i] > t->hmax[id] ? st->h[i] : t->hmax[id];
        if (2.0 * hh > R) R = 2.0 * hh;
    }
    double bd = sqrt(orc_box_dist2(t, pp, id, p));
    orc_margin(res, bd, R);
    int far = bd > R;
    if (pr->gravity) {
        const double *c = &t->com[3 * id];
        double dv[3] = {p[0] - c[0], p[1] - c[1], p[2] - c[2]};
        if (pr->ewald_L > 0)
            for (int a = 0; a < 3; ++a) dv[a] = orc_wrap(pp, a, dv[a]);
        double d = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
        double ropen = (pr->theta > 0) ? t->l[id] / pr->theta + t->delta[id] : INFINITY;
        orc_margin(res, d, ropen);
        far = far && (d > ropen);
        /* Periodic gravity: the node is taken at the nearest image of its centre of mass, whatever
         * images its particles' own nearest ones are: the direct force of the node there plus the
         * correction of its replicas is the full periodic force of its mass, and that force is
         * periodic, so any one image serves.  The correction is taken for the node's mass at the
         * centre of mass; its error grows as (l/L)^2.  Reading: nodes of side l > L/8 are opened
         * (the paper states no rule; with it the tree error at theta = 0.5 stays near the
         * non-periodic one). */
        if (pr->ewald_L > 0) far = far && (t->l[id] <= ORC_EWALD_LMAX * pr->ewald_L);
    }
    return far;
}

static void orc_force_one(const orc_tree *t, const orc_params *pr, const orc_period *pp, const orc_state *st,
                          int64_t i, orc_result *res)
{
    memset(res, 0, sizeof *res);
    res->margin = INFINITY;
    double p[3] = {t->x[i], t->y[i], t->z[i]};
    res->scale = fmax(fabs(p[0]), fmax(fabs(p[1]), fabs(p[2])));
    int64_t id = 0, nn = t->nnodes;
    /* Pre-order walk; nnext skips a subtree. */
    while (id < nn) {
        if (orc_accept(t, pr, pp, st, i, id, p, res)) {
            if (pr->gravity) orc_far(t, pr, pp, id, p, res);
            res->nfar += 1;
            res->hfar += orc_hash_id((uint64_t)id);
            id = t->nnext[id];
        } else if (t->nnch[id] == 0) {
            res->hnear += orc_hash_id((uint64_t)id);
            for (int64_t s = t->nbeg[id]; s < t->nend[id]; ++s) {
                int64_t j = t->perm[s];
                if (j == i) continue;
                double rv[3] = {orc_wrap(pp, 0, p[0] - t->x[j]), orc_wrap(pp, 1, p[1] - t->y[j]),
                                orc_wrap(pp, 2, p[2] - t->z[j])};
                res->npp += 1;
                orc_pair(t, pr, st, i, j, rv, res);
            }
            id = t->nnext[id];
        } else {
            id = id + 1;
        }
    }
    /* self term of the potential, phi(0, eps_i) (the double sum of Eq. Lgrav includes k = j) */
    if (pr->gravity) res->pot += pr->G * t->m[i] * orc_phi(0.0, st->eps[i]);
    /* periodic gravity: the particle's own replicas */
    if (pr->gravity && pr->ewald_L > 0) {
        double z[3] = {0, 0, 0}, fe[3], ge;
        orc_ewald_interp(pr->ewald_L, z, fe, &ge);
        res->pot += pr->G * t->m[i] * ge;
    }
}

/* Force pass for the particles in idx (all if idx == NULL).  Outputs at original index. */
void orc_forces(orc_tree *t, double theta, double G, double gamma, double alpha, double beta,
                int gravity, int sph, int adaptive, int use_tc,
                int periodic_mask, const double *plo, const double *phi_,
                const double *vx, const double *vy, const double *vz,
                const double *eps, const double *ups, const double *X,
                const double *h, const double *rho, const double *P, const double *c,
                const double *om, const double *zeta,
                const int64_t *idx, int64_t nidx,
                double *ax, double *ay, double *az, double *pot, double *dudt,
                uint64_t *hfar, uint64_t *hnear, uint64_t *hsph,
                int64_t *nfar, int64_t *npp, int64_t *nsph, double *margin,
                double *aabs, double *duabs, double *mumax,
                const orc_diss *diss, double *vsig, double *lapu, double *lapabs)
{
    orc_params pr = {theta, G, gamma, alpha, beta, gravity, sph, adaptive, use_tc, {0}, 0.0};
    if (diss) pr.ds = *diss;
    orc_state st = {vx, vy, vz, eps, ups, X, h, rho, P, c, om, zeta};
    orc_period per = {periodic_mask, {0, 0, 0}, {1, 1, 1}};
    for (int a = 0; a < 3; ++a)
        if ((periodic_mask >> a) & 1) { per.lo[a] = plo[a]; per.len[a] = phi_[a] - plo[a]; }
    /* periodic gravity: a cube periodic in all three axes (Sect. 4.3); the table is built first */
    if (gravity && periodic_mask == 7) {
        pr.ewald_L = per.len[0];
        orc_ewald_table();
    }
    orc_set_node_lengths(t, gravity ? eps : NULL, sph ? h : NULL);
    int64_t count = idx ? nidx : t->n;
#pragma omp parallel for schedule(dynamic, 32)
    for (int64_t q = 0; q < count; ++q) {
        int64_t i = idx ? idx[q] : q;
        orc_result res;
        orc_force_one(t, &pr, &per, &st, i, &res);
        ax[i] = res.a[0]; ay[i] = res.a[1]; az[i] = res.a[2];
        pot[i] = res.pot;
        dudt[i] = res.dudt;
        if (hfar) hfar[i] = res.hfar;
        if (hnear) hnear[i] = res.hnear;
        if (hsph) hsph[i] = res.hsph;
        if (nfar) nfar[i] = res.nfar;
        if (npp) npp[i] = res.npp;
        if (nsph) nsph[i] = res.nsph;
        if (margin) margin[i] = res.margin;
        if (aabs) aabs[i] = res.aabs;
        if (duabs) duabs[i] = res.duabs;
        if (mumax) mumax[i] = res.mumax;
        /* the self pair (w = 0) bounds v^sig_i from below by 2 c_i, also for a particle without
         * neighbours */
        if (vsig) vsig[i] = (sph && i < t->n_gas && c) ? fmax(res.vsig, 2.0 * c[i]) : 0.0;
        if (lapu) lapu[i] = res.lapu;
        if (lapabs) lapabs[i] = res.lapabs;
    }
}

/* Wake-up input of the individual time steps (Sect. 4.2.1): for every gas particle j, the smallest
 * key[i] over the listed gas particles i (the active ones) that are its SPH neighbours, i.e. with
 * r_ij < 2 max(h_i, h_j), i != j.  out (length n) must hold +inf on entry; entries without such a
 * neighbour keep it.  h: original order (gas entries used).  Returns 0, or -3 on overflow. */
int orc_sph_nbmin(const orc_tree *t, const double *h, const int64_t *idx, int64_t nidx, const double *key,
                  int periodic_mask, const double *plo, const double *phi_, double *out)
{
    orc_period per = {periodic_mask, {0, 0, 0}, {1, 1, 1}};
    for (int a = 0; a < 3; ++a)
        if ((periodic_mask >> a) & 1) { per.lo[a] = plo[a]; per.len[a] = phi_[a] - plo[a]; }
    double hmax = 0;
    for (int64_t j = 0; j < t->n_gas; ++j)
        if (h[j] > hmax) hmax = h[j];
    int64_t cap = 1 << 16;
    int64_t *scr = malloc(cap * sizeof(int64_t));
    double *rs = malloc(cap * sizeof(double));
    int err = (scr && rs) ? 0 : -3;
    for (int64_t q = 0; q < nidx && !err; ++q) {
        int64_t i = idx[q];
        if (i >= t->n_gas) continue;
        double p[3] = {t->x[i], t->y[i], t->z[i]};
        int64_t cnt = orc_gather(t, &per, p, 2.0 * (h[i] > hmax ? h[i] : hmax), 1, scr, rs, cap);
        if (cnt < 0) {
            err = -3;
            break;
        }
        for (int64_t k = 0; k < cnt; ++k) {
            int64_t j = scr[k];
            double R = 2.0 * (h[i] > h[j] ? h[i] : h[j]);
            if (j != i && rs[k] < R && key[i] < out[j]) out[j] = key[i];
        }
    }
    free(scr);
    free(rs);
    return err;
}

/* Ideal-gas equation of state (App. B; Sect. 3.3.1): P = (gamma-1) rho u, c = sqrt(gamma(gamma-1)u). */
void orc_eos(int64_t n, double gamma, const double *rho, const double *u, double *P, double *c)
{
    for (int64_t i = 0; i < n; ++i) {
        P[i] = (gamma - 1.0) * rho[i] * u[i];
        c[i] = sqrt(gamma * (gamma - 1.0) * u[i]);
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
