/*
 * CPU FP64 oracle of the DENSER hot path in plain C -- TEST INFRASTRUCTURE ONLY.
 *
 * The same restatement of the paper as oracle/denser_oracle.py, written out in C so
 * that the oracle can run maps of millions of voxels and thousands of iterations:
 *   - block allocation of the hashing voxel grid (Section III-A, "Fusing Data");
 *   - projective TSDF fusion (Section III-A, Eq. 1);
 *   - Omega = {allocated, w > 0} and the Omega-aware gradient and divergence
 *     (Section III-B, Eq. 3 and Eq. 4);
 *   - the Chambolle-Pock iteration (Section III-C, steps 1-4; Table I);
 *   - the primal and dual energies (Eq. 2 and the saddle form of Section III-C).
 * Readings R1-R10 are those listed in oracle/denser_oracle.py.
 *
 * Every expression is evaluated in the operation order of the numpy oracle, one IEEE
 * double operation at a time (compiled with -ffp-contract=off: no fused multiply-add),
 * so allocation, fusion and the iterates equal the numpy oracle's bit for bit; only the
 * energy sums differ in their summation order.  The iteration is Jacobi: every voxel
 * is updated from the previous iterate, so the per-block OpenMP loops give the same
 * result for any thread count.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference arm use
 * this library (through oracle/oracle_c.py).  It shares no code with the CUDA path.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define BV 512 /* voxels per 8^3 block */

typedef struct {
    double s, mu, lam, sigma, tau, theta;
    int64_t cap;       /* block capacity */
    int64_t nb;        /* allocated blocks */
    int64_t *key;      /* [cap][4] segment, bx, by, bz in block-index order */
    double *f, *w, *u, *ub, *p; /* [cap][512]; p [3][cap][512] */
    /* open-addressing table of block keys -> block index */
    uint64_t hmask;
    int64_t *hidx;     /* -1 = empty */
} omap;

/* ------------------------------------------------------------- key table */
static uint64_t mix(const int64_t *k) {
    uint64_t h = 0x9e3779b97f4a7c15ull;
    for (int i = 0; i < 4; ++i) {
        h ^= (uint64_t)k[i] + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
        h *= 0xbf58476d1ce4e5b9ull;
        h ^= h >> 31;
    }
    return h;
}

static int same(const int64_t *a, const int64_t *b) { return a[0] == b[0] && a[1] == b[1] && a[2] == b[2] && a[3] == b[3]; }

static int64_t lookup(const omap *m, const int64_t *k) {
    for (uint64_t h = mix(k) & m->hmask;; h = (h + 1) & m->hmask) {
        const int64_t i = m->hidx[h];
        if (i < 0) return -1;
        if (same(m->key + 4 * i, k)) return i;
    }
}

static void insert(omap *m, int64_t i) {
    uint64_t h = mix(m->key + 4 * i) & m->hmask;
    while (m->hidx[h] >= 0) h = (h + 1) & m->hmask;
    m->hidx[h] = i;
}

omap *ocl_new(double s, double mu, double lam, double sigma, double tau, double theta, int64_t cap) {
    omap *m = (omap *)calloc(1, sizeof(omap));
    if (!m) return NULL;
    m->s = s, m->mu = mu, m->lam = lam, m->sigma = sigma, m->tau = tau, m->theta = theta;
    m->cap = cap;
    uint64_t slots = 1;
    while (slots < (uint64_t)(2 * cap + 2)) slots <<= 1;
    m->hmask = slots - 1;
    m->hidx = (int64_t *)malloc(sizeof(int64_t) * slots);
    m->key = (int64_t *)malloc(sizeof(int64_t) * 4 * cap);
    m->f = (double *)calloc((size_t)cap * BV, sizeof(double));
    m->w = (double *)calloc((size_t)cap * BV, sizeof(double));
    m->u = (double *)calloc((size_t)cap * BV, sizeof(double));
    m->ub = (double *)calloc((size_t)cap * BV, sizeof(double));
    m->p = (double *)calloc((size_t)3 * cap * BV, sizeof(double));
    if (!m->hidx || !m->key || !m->f || !m->w || !m->u || !m->ub || !m->p) return NULL;
    for (uint64_t i = 0; i < slots; ++i) m->hidx[i] = -1;
    return m;
}

void ocl_free(omap *m) {
    if (!m) return;
    free(m->hidx), free(m->key), free(m->f), free(m->w), free(m->u), free(m->ub), free(m->p);
    free(m);
}

int64_t ocl_num_blocks(const omap *m) { return m->nb; }

/* Threads of every parallel loop that follows (n <= 0: the OpenMP default). */
void ocl_set_threads(int n) { omp_set_num_threads(n > 0 ? n : omp_get_num_procs()); }

/* p is stored [3][cap][512]; the three components of voxel v are p[a*cap*512 + v] */
static double *pc(omap *m, int a) { return m->p + (size_t)a * m->cap * BV; }

/* Appends blocks in the given order with zero state (coords [n][4]); f, w may be NULL.
 * Returns the number appended, or -1 when a key is already present or the capacity
 * would be exceeded. */
int64_t ocl_load_blocks(omap *m, const int64_t *coords, const double *f, const double *w, int64_t n) {
    if (m->nb + n > m->cap) return -1;
    for (int64_t i = 0; i < n; ++i)
        if (lookup(m, coords + 4 * i) >= 0) return -1;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t b = m->nb++;
        memcpy(m->key + 4 * b, coords + 4 * i, 4 * sizeof(int64_t));
        insert(m, b);
        if (f) memcpy(m->f + (size_t)b * BV, f + (size_t)i * BV, BV * sizeof(double));
        if (w) memcpy(m->w + (size_t)b * BV, w + (size_t)i * BV, BV * sizeof(double));
    }
    return n;
}

/* --------------------------------------------------------------- allocation */
static int key_less(const int64_t *a, const int64_t *b) {
    /* ascending (segment, bz, by, bx) */
    if (a[0] != b[0]) return a[0] < b[0];
    if (a[3] != b[3]) return a[3] < b[3];
    if (a[2] != b[2]) return a[2] < b[2];
    return a[1] < b[1];
}

static int key_cmp(const void *x, const void *y) {
    const int64_t *a = (const int64_t *)x, *b = (const int64_t *)y;
    return key_less(a, b) ? -1 : (key_less(b, a) ? 1 : 0);
}

typedef struct {
    int64_t *k; /* [cap][4] */
    int64_t n, cap;
    uint64_t mask;
    int64_t *slot;
} keyset;

static int ks_init(keyset *s, int64_t cap) {
    s->n = 0, s->cap = cap;
    uint64_t slots = 1;
    while (slots < (uint64_t)(2 * cap + 2)) slots <<= 1;
    s->mask = slots - 1;
    s->k = (int64_t *)malloc(sizeof(int64_t) * 4 * cap);
    s->slot = (int64_t *)malloc(sizeof(int64_t) * slots);
    if (!s->k || !s->slot) return -1;
    for (uint64_t i = 0; i < slots; ++i) s->slot[i] = -1;
    return 0;
}

static int ks_grow(keyset *s) {
    keyset t;
    if (ks_init(&t, 2 * s->cap)) return -1;
    for (int64_t i = 0; i < s->n; ++i) {
        uint64_t h = mix(s->k + 4 * i) & t.mask;
        while (t.slot[h] >= 0) h = (h + 1) & t.mask;
        memcpy(t.k + 4 * t.n, s->k + 4 * i, 4 * sizeof(int64_t));
        t.slot[h] = t.n++;
    }
    free(s->k), free(s->slot);
    *s = t;
    return 0;
}

static int ks_add(keyset *s, const int64_t *k) {
    uint64_t h = mix(k) & s->mask;
    for (;; h = (h + 1) & s->mask) {
        const int64_t i = s->slot[h];
        if (i < 0) break;
        if (same(s->k + 4 * i, k)) return 0;
    }
    if (s->n == s->cap) {
        if (ks_grow(s)) return -1;
        return ks_add(s, k);
    }
    memcpy(s->k + 4 * s->n, k, 4 * sizeof(int64_t));
    s->slot[h] = s->n++;
    return 0;
}

/* Allocation rule of Section III-A under reading R1: for every valid pixel (finite
 * d > 0) and n = -N..N, N = ceil(mu/h - 1e-9), h = s/2:
 *     z = d + n h (skipped when z <= 0);  X = (((x + 0.5) - cx) z) / fx, Y likewise, Z = z
 *     g_r = ((R_r0 X + R_r1 Y) + R_r2 Z) + t_r;  key = floor(g / (8 s))
 * New keys are appended in ascending (segment, bz, by, bx) order.  Returns the number of
 * new blocks, or -1 when the capacity is exceeded. */
int64_t ocl_alloc(omap *m, const float *depth, int W, int H, double fx, double fy, double cx, double cy,
                  const double *T, int64_t segment) {
    const double h = 0.5 * m->s, bs = 8.0 * m->s;
    const int N = (int)ceil(m->mu / h - 1e-9);
    const int nt = omp_get_max_threads();
    keyset *part = (keyset *)calloc((size_t)nt, sizeof(keyset));
    int fail = part == NULL;
    /* each thread collects the new keys of its rows; the union is then sorted, so the
     * result does not depend on how rows were shared out */
#pragma omp parallel num_threads(nt) reduction(| : fail)
    {
        keyset *ks = part + omp_get_thread_num();
        if (fail || ks_init(ks, 1 << 16)) fail = 1;
#pragma omp for schedule(dynamic, 4)
        for (int y = 0; y < H; ++y) {
            if (fail) continue;
            const double vv = ((double)y + 0.5) - cy;
            for (int x = 0; x < W; ++x) {
                const float d32 = depth[(size_t)y * W + x];
                if (!(isfinite(d32) && d32 > 0.0f)) continue;
                const double d = (double)d32;
                const double uu = ((double)x + 0.5) - cx;
                for (int n = -N; n <= N; ++n) {
                    const double z = d + (double)n * h;
                    if (!(z > 0.0)) continue;
                    const double X = (uu * z) / fx, Y = (vv * z) / fy, Z = z;
                    int64_t k[4];
                    k[0] = segment;
                    for (int r = 0; r < 3; ++r) {
                        const double g = ((T[4 * r + 0] * X + T[4 * r + 1] * Y) + T[4 * r + 2] * Z) + T[4 * r + 3];
                        k[1 + r] = (int64_t)floor(g / bs);
                    }
                    if (lookup(m, k) >= 0) continue;
                    if (ks_add(ks, k)) fail = 1;
                }
            }
        }
    }
    keyset all;
    int64_t total = 0;
    for (int t = 0; t < nt && !fail; ++t) total += part[t].n;
    if (!fail && ks_init(&all, total + 1)) fail = 1;
    for (int t = 0; t < nt && !fail; ++t)
        for (int64_t i = 0; i < part[t].n; ++i) ks_add(&all, part[t].k + 4 * i);
    if (part)
        for (int t = 0; t < nt; ++t) free(part[t].k), free(part[t].slot);
    free(part);
    if (fail) return -1;
    qsort(all.k, (size_t)all.n, 4 * sizeof(int64_t), key_cmp);
    const int64_t added = all.n;
    const int64_t rc = ocl_load_blocks(m, all.k, NULL, NULL, all.n);
    free(all.k), free(all.slot);
    return rc < 0 ? -1 : added;
}

/* ------------------------------------------------------------------- fusion */
/* Projective fusion (Section III-A, steps 1-4, Eq. 1) of one depth map into every
 * allocated voxel of `segment`:
 *     p_c = R^T p_g + (-R^T t);  skip z_c <= 0
 *     px = floor((fx x_c) / z_c + cx), py likewise (reading R3); skip outside / invalid
 *     u_SDF = d - z_c; skip u_SDF < -mu;  u_TSDF = min(1, u_SDF / mu) (reading R2)
 *     w' = w + 1;  f' = (u_TSDF + w f) / w'                                  (Eq. 1) */
void ocl_fuse(omap *m, const float *depth, int W, int H, double fx, double fy, double cx, double cy,
              const double *T, int64_t segment) {
    double Ri[9], ti[3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Ri[3 * r + c] = T[4 * c + r];
    for (int r = 0; r < 3; ++r) ti[r] = -((T[0 * 4 + r] * T[3] + T[1 * 4 + r] * T[7]) + T[2 * 4 + r] * T[11]);
    const double s = m->s, mu = m->mu;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t b = 0; b < m->nb; ++b) {
        const int64_t *k = m->key + 4 * b;
        if (k[0] != segment) continue;
        double *fb = m->f + (size_t)b * BV, *wb = m->w + (size_t)b * BV;
        for (int l = 0; l < BV; ++l) {
            const int64_t i = k[1] * 8 + (l & 7), j = k[2] * 8 + ((l >> 3) & 7), kk = k[3] * 8 + (l >> 6);
            const double gx = ((double)i + 0.5) * s, gy = ((double)j + 0.5) * s, gz = ((double)kk + 0.5) * s;
            const double xc = ((Ri[0] * gx + Ri[1] * gy) + Ri[2] * gz) + ti[0];
            const double yc = ((Ri[3] * gx + Ri[4] * gy) + Ri[5] * gz) + ti[1];
            const double zc = ((Ri[6] * gx + Ri[7] * gy) + Ri[8] * gz) + ti[2];
            if (!(zc > 0.0)) continue;
            const double pxf = floor((fx * xc) / zc + cx), pyf = floor((fy * yc) / zc + cy);
            if (!(pxf >= 0.0 && pxf < (double)W && pyf >= 0.0 && pyf < (double)H)) continue;
            const double d = (double)depth[(size_t)pyf * W + (size_t)pxf];
            if (!(isfinite(d) && d > 0.0)) continue;
            const double usdf = d - zc;
            if (!(usdf >= -mu)) continue;
            const double q = usdf / mu;
            const double utsdf = q < 1.0 ? q : 1.0;
            const double w_old = wb[l], w_new = w_old + 1.0;
            fb[l] = (utsdf + w_old * fb[l]) / w_new;
            wb[l] = w_new;
        }
    }
}

/* ---------------------------------------------------- neighbours, grad, div */
/* Block-level neighbour table: nbr[b][a] (a = 0,1,2 for +x,+y,+z; 3,4,5 for -x,-y,-z),
 * -1 where that block is not allocated (reading R5: Omega-bar, the role of i = V_x). */
static int64_t *neighbour_table(const omap *m) {
    int64_t *nbr = (int64_t *)malloc(sizeof(int64_t) * 6 * (m->nb ? m->nb : 1));
    if (!nbr) return NULL;
    for (int64_t b = 0; b < m->nb; ++b)
        for (int a = 0; a < 6; ++a) {
            int64_t q[4];
            memcpy(q, m->key + 4 * b, sizeof q);
            q[1 + (a % 3)] += a < 3 ? 1 : -1;
            nbr[6 * b + a] = lookup(m, q);
        }
    return nbr;
}

/* Flat index of the neighbour of voxel (b, l) along axis a (dir +1 or -1), -1 if none. */
static int64_t voxel_nb(const int64_t *nbr, int64_t b, int l, int a, int dir) {
    const int stride = a == 0 ? 1 : (a == 1 ? 8 : 64);
    const int c = (l / stride) & 7;
    if ((dir > 0 && c < 7) || (dir < 0 && c > 0)) return b * BV + l + dir * stride;
    const int64_t nb = nbr[6 * b + a + (dir > 0 ? 0 : 3)];
    if (nb < 0) return -1;
    return nb * BV + l - dir * 7 * stride;
}

/* Eq. 3 edge e_a(v): v and v + a both in Omega. */
static int edge(const omap *m, const int64_t *nbr, int64_t b, int l, int a, int64_t *fwd) {
    const int64_t v = b * BV + l;
    *fwd = voxel_nb(nbr, b, l, a, +1);
    return m->w[v] > 0.0 && *fwd >= 0 && m->w[*fwd] > 0.0;
}

/* (div p)_v = sum_a [e_a(v) p^a_v - e_a(v - a) p^a_{v-a}], Eq. 4 as the negative adjoint
 * of Eq. 3 (reading R6), summed over a = x, y, z left to right. */
static double divergence(omap *m, const int64_t *nbr, int64_t b, int l) {
    const int64_t v = b * BV + l;
    double d = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double *pa = pc(m, a);
        int64_t f;
        const double own = edge(m, nbr, b, l, a, &f) ? pa[v] : 0.0;
        double back = 0.0;
        const int64_t vb = voxel_nb(nbr, b, l, a, -1);
        if (vb >= 0) {
            int64_t f2;
            if (edge(m, nbr, vb / BV, (int)(vb % BV), a, &f2)) back = pa[vb];
        }
        d = d + (own - back);
    }
    return d;
}

/* ----------------------------------------------------------- primal-dual */
/* Chambolle-Pock iterations (Section III-C, steps 2-4; readings R7, R8), Jacobi:
 *     p~ = p + sigma grad_Omega(u^);  p = p~ / max(1, |p~|_2)
 *     u~ = u + tau div_Omega(p);  u = (u~ + tau lam w f) / (1 + tau lam w) on Omega
 *     u^ = u + theta (u - u_old)
 * threads <= 0 uses the OpenMP default.  Returns 0, or -1 when memory runs out. */
int ocl_iterate(omap *m, int iters, int threads) {
    int64_t *nbr = neighbour_table(m);
    if (!nbr) return -1;
    const double sg = m->sigma, tau = m->tau, lam = m->lam, th = m->theta;
    double *p0 = pc(m, 0), *p1 = pc(m, 1), *p2 = pc(m, 2);
    double *dv = (double *)malloc(sizeof(double) * (size_t)(m->nb ? m->nb : 1) * BV);
    if (!dv) {
        free(nbr);
        return -1;
    }
    const int nt = threads > 0 ? threads : omp_get_max_threads();
    for (int it = 0; it < iters; ++it) {
        /* dual step: reads u^ at v and v + a, writes p at v only */
#pragma omp parallel for schedule(static) num_threads(nt)
        for (int64_t b = 0; b < m->nb; ++b)
            for (int l = 0; l < BV; ++l) {
                const int64_t v = b * BV + l;
                double g[3];
                for (int a = 0; a < 3; ++a) {
                    int64_t f;
                    g[a] = edge(m, nbr, b, l, a, &f) ? m->ub[f] - m->ub[v] : 0.0;
                }
                const double q0 = p0[v] + sg * g[0], q1 = p1[v] + sg * g[1], q2 = p2[v] + sg * g[2];
                const double nrm = sqrt((q0 * q0 + q1 * q1) + q2 * q2);
                const double sc = nrm > 1.0 ? nrm : 1.0;
                p0[v] = q0 / sc, p1[v] = q1 / sc, p2[v] = q2 / sc;
            }
        /* divergence of the new p (reads p at v and v - a) */
#pragma omp parallel for schedule(static) num_threads(nt)
        for (int64_t b = 0; b < m->nb; ++b)
            for (int l = 0; l < BV; ++l) dv[b * BV + l] = divergence(m, nbr, b, l);
        /* primal step and relaxation (reads and writes voxel v only) */
#pragma omp parallel for schedule(static) num_threads(nt)
        for (int64_t b = 0; b < m->nb; ++b)
            for (int l = 0; l < BV; ++l) {
                const int64_t v = b * BV + l;
                const double u_old = m->u[v];
                double u = u_old;
                if (m->w[v] > 0.0) {
                    const double ut = u_old + tau * dv[v];
                    u = (ut + ((tau * lam) * m->w[v]) * m->f[v]) / (1.0 + (tau * lam) * m->w[v]);
                }
                m->u[v] = u;
                m->ub[v] = u + th * (u - u_old);
            }
    }
    free(dv);
    free(nbr);
    return 0;
}

/* Primal P(u) = sum_Omega |grad u|_2 + (lam/2) w (u - f)^2 and dual
 * D(p) = sum_Omega [-f div p - (div p)^2 / (2 lam w)] (reading R10). */
int ocl_energies(omap *m, double *P, double *D) {
    int64_t *nbr = neighbour_table(m);
    if (!nbr) return -1;
    double sp = 0.0, sd = 0.0;
    const double lam = m->lam;
#pragma omp parallel for schedule(static) reduction(+ : sp, sd)
    for (int64_t b = 0; b < m->nb; ++b)
        for (int l = 0; l < BV; ++l) {
            const int64_t v = b * BV + l;
            if (!(m->w[v] > 0.0)) continue;
            double g[3];
            for (int a = 0; a < 3; ++a) {
                int64_t f;
                g[a] = edge(m, nbr, b, l, a, &f) ? m->u[f] - m->u[v] : 0.0;
            }
            const double tv = sqrt((g[0] * g[0] + g[1] * g[1]) + g[2] * g[2]);
            const double r = m->u[v] - m->f[v];
            sp += tv + ((0.5 * lam) * m->w[v]) * (r * r);
            const double d = divergence(m, nbr, b, l);
            sd += -m->f[v] * d - (d * d) / ((2.0 * lam) * m->w[v]);
        }
    free(nbr);
    *P = sp, *D = sd;
    return 0;
}

/* ------------------------------------------------------------- state I/O */
/* Copies the map out in block-index order (any output may be NULL): coords [nb][4];
 * f, w, u, ub [nb][512]; p [3][nb][512]. */
void ocl_get(const omap *m, int64_t *coords, double *f, double *w, double *u, double *ub, double *p) {
    const size_t n = (size_t)m->nb * BV;
    if (coords) memcpy(coords, m->key, sizeof(int64_t) * 4 * m->nb);
    if (f) memcpy(f, m->f, sizeof(double) * n);
    if (w) memcpy(w, m->w, sizeof(double) * n);
    if (u) memcpy(u, m->u, sizeof(double) * n);
    if (ub) memcpy(ub, m->ub, sizeof(double) * n);
    if (p)
        for (int a = 0; a < 3; ++a) memcpy(p + a * n, m->p + (size_t)a * m->cap * BV, sizeof(double) * n);
}

/* Overwrites u, u^ [nb][512] and p [3][nb][512] (NULL = zeros). */
void ocl_set_state(omap *m, const double *u, const double *ub, const double *p) {
    const size_t n = (size_t)m->nb * BV;
    if (u) memcpy(m->u, u, sizeof(double) * n); else memset(m->u, 0, sizeof(double) * n);
    if (ub) memcpy(m->ub, ub, sizeof(double) * n); else memset(m->ub, 0, sizeof(double) * n);
    for (int a = 0; a < 3; ++a) {
        double *dst = m->p + (size_t)a * m->cap * BV;
        if (p) memcpy(dst, p + a * n, sizeof(double) * n); else memset(dst, 0, sizeof(double) * n);
    }
}
