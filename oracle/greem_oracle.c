/*
 * greem_oracle.c -- plain, slow FP64 CPU oracle for the periodic short-range (PP)
 * tree force of GreeM (Ishiyama, Fukushige & Makino 2009, "GreeM: Massively
 * Parallel TreePM Code for Large Cosmological N-body Simulations").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline / reference leg of bench.py load this library.  It shares no source,
 * header, table or constant generator with the CUDA library; both sides are
 * written from the paper and from the readings stated below.
 *
 * Build: gcc -O2 -std=c11 -fopenmp -ffp-contract=off -fPIC -shared -lm.
 * -ffp-contract=off matters: every integer-deciding comparison below is a plain
 * IEEE FP64 product or quotient, and no a*b+c may be fused on any host.
 *
 * What is computed, step by step (paper sections in brackets):
 *   wrap + 63-bit Morton key            [Sec. 3.2.5: "morton key", 12 B/particle]
 *   stable sort on the key               [reading: ties broken by input index]
 *   octree over sorted ranges            [Sec. 2.2 step 2; Sec. 3.1.2: N_leaf rule]
 *   monopole moments (mass, COM)         [Sec. 3.1.2: center-of-mass approximation]
 *   groups of <= n_crit particles        [Sec. 2.2 step 5; Sec. 3.1.2: N_crit]
 *   interaction lists (Barnes 1990)      [Sec. 2.2 steps 3 and 5: opening criterion,
 *                                         r_cut pruning]
 *   list force with g_P3M                [Eq. 1 and Eq. 2]
 *   brute-force minimum-image sum        [Eq. 1, Eq. 2; Sec. 1: image particles]
 *
 * Readings of points the paper leaves open; the tag in brackets is the reading's
 * number (C1-C19, R1-R4), the same on the CUDA side:
 *   - [C9, R2] wrap: r = x - L*floor(x/L); r<0 -> r+L; r>=L -> r-L; anything outside [0,L) -> 0.
 *   - [C9] key: ix = min(floor((r/L)*2^21), 2^21-1) per axis, 21 bits per axis, the x bit
 *     is the most significant bit of each 3-bit digit.
 *   - [C4] l_min = smallest level k with L*2^-k < L/2 - r_cut; nodes above l_min are always
 *     split and never accepted, groups live at level >= l_min.  This keeps every
 *     per-node image shift equal to the per-pair minimum image for pairs within r_cut.
 *   - [C5] leaf iff count < n_leaf or level 21 (levels < l_min always split).
 *   - [C6] group = first node in preorder with level >= l_min and (count <= n_crit or leaf).
 *   - [C1, C2] integer geometry in units u = L/2^22: a level-k cell with index i has centre
 *     (2i+1)*2^(21-k) and half side 2^(21-k); the period is 2^22.
 *   - [C4] node-to-group offset wrapped into [-2^21, 2^21).
 *   - [C2] prune iff (double)S_gap * (u*u) > r_cut*r_cut, S_gap = sum of squared per-axis
 *     gaps (exact integers) between the node's cell and the group's particle box: the
 *     smallest box of finest-level (level 21) cells that holds every particle of the
 *     group.  A particle of an opened leaf is tested the same way with its own finest
 *     cell and is left out when the test holds.  Either way the left-out mass lies
 *     farther than r_cut from every particle of the group, where Eq. 2 is exactly 0.
 *   - [C17] distance-dependent opening angle (Sec. 4.1, Eq. 12), when selected: theta(d) =
 *     min(theta_max, theta0 / sqrt(R g(R))) with R = d/eta (the distance in units of eta,
 *     which makes theta0 dimensionless) and theta(d) = theta_max where R g(R) = 0; the
 *     accept test below then uses theta(d)^2 in place of theta^2.
 *   - [C1] accept iff level >= l_min and (double)(l*l) < (theta*theta) * (double)S_d,
 *     l = node side, S_d = squared distance from node centre to the nearest point of
 *     the group cell (both in u).  Prune is tested first.
 *   - [C7, C8] Plummer softening: acc = m g(r/eta) d / (r^2+eps^2)^(3/2); pairs with r^2 == 0
 *     are skipped.  eps = 0 gives Eq. 1 exactly.
 *   - [C4] minimum image per pair: d -= L while d > L/2; d += L while d < -L/2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXLEVEL 21

/* ------------------------------------------------------------------------- */
/* Eq. 2: the Hockney & Eastwood S2 cutoff function, both branches written out. */
double or_g_p3m(double R)
{
    if (R < 0.0) R = -R;
    double R2 = R * R, R3 = R2 * R, R4 = R3 * R, R5 = R4 * R, R6 = R5 * R, R7 = R6 * R, R8 = R7 * R;
    if (R < 1.0)
        return 1.0 - (224.0 * R3 - 224.0 * R5 + 70.0 * R6 + 48.0 * R7 - 21.0 * R8) / 140.0;
    if (R < 2.0)
        return 1.0 - (12.0 - 224.0 * R2 + 896.0 * R3 - 840.0 * R4 + 224.0 * R5 + 70.0 * R6 - 48.0 * R7 +
                      7.0 * R8) / 140.0;
    return 0.0;
}

/* First and second derivatives of Eq. 2 in R, term by term from the printed branches
 * (the quadrupole terms of Sec. 4.1 need the cutoff function's derivatives). */
double or_g_p3m_d1(double R)
{
    if (R < 0.0) R = -R;
    double R2 = R * R, R3 = R2 * R, R4 = R3 * R, R5 = R4 * R, R6 = R5 * R, R7 = R6 * R;
    if (R < 1.0) return -(3.0 * 224.0 * R2 - 5.0 * 224.0 * R4 + 6.0 * 70.0 * R5 + 7.0 * 48.0 * R6 - 8.0 * 21.0 * R7) / 140.0;
    if (R < 2.0)
        return -(-2.0 * 224.0 * R + 3.0 * 896.0 * R2 - 4.0 * 840.0 * R3 + 5.0 * 224.0 * R4 + 6.0 * 70.0 * R5 -
                 7.0 * 48.0 * R6 + 8.0 * 7.0 * R7) / 140.0;
    return 0.0;
}

double or_g_p3m_d2(double R)
{
    if (R < 0.0) R = -R;
    double R2 = R * R, R3 = R2 * R, R4 = R3 * R, R5 = R4 * R, R6 = R5 * R;
    if (R < 1.0)
        return -(6.0 * 224.0 * R - 20.0 * 224.0 * R3 + 30.0 * 70.0 * R4 + 42.0 * 48.0 * R5 - 56.0 * 21.0 * R6) / 140.0;
    if (R < 2.0)
        return -(-2.0 * 224.0 + 6.0 * 896.0 * R - 12.0 * 840.0 * R2 + 20.0 * 224.0 * R3 + 30.0 * 70.0 * R4 -
                 42.0 * 48.0 * R5 + 56.0 * 7.0 * R6) / 140.0;
    return 0.0;
}

/* Quadrupole part of the acceleration from a mass distribution with second moments
 * q = (xx, yy, zz, xy, xz, yz) about its COM at separation d = COM - x (Sec. 4.1).  With
 * the pair force m f(r) d/r, f(r) = g(r/eta)/r^2, and Phi' = f, the second-order Taylor
 * term of sum_j m_j grad Phi(d + s_j) is
 *   1/2 B tr(Q) d + 1/2 C (d.Q.d) d + B Q d,
 *   A = f/r, B = A'/r = g'/(eta r^4) - 3 g/r^5, C = B'/r = g''/(eta^2 r^5) - 7 g'/(eta r^6) + 15 g/r^7,
 * which for g = 1 is the Newtonian quadrupole.  eps must be 0. */
void or_quad_accel(const double d[3], const double q[6], double eta, double out[3])
{
    out[0] = out[1] = out[2] = 0.0;
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 == 0.0) return;
    double r = sqrt(r2), R = r / eta;
    double g = or_g_p3m(R), g1 = or_g_p3m_d1(R) / eta, g2 = or_g_p3m_d2(R) / (eta * eta);
    double r4 = r2 * r2, r5 = r4 * r, r6 = r4 * r2, r7 = r6 * r;
    double B = g1 / r4 - 3.0 * g / r5;
    double C = g2 / r5 - 7.0 * g1 / r6 + 15.0 * g / r7;
    double Qd[3] = {q[0] * d[0] + q[3] * d[1] + q[4] * d[2], q[3] * d[0] + q[1] * d[1] + q[5] * d[2],
                    q[4] * d[0] + q[5] * d[1] + q[2] * d[2]};
    double dQd = d[0] * Qd[0] + d[1] * Qd[1] + d[2] * Qd[2];
    double tr = q[0] + q[1] + q[2];
    for (int c = 0; c < 3; c++) out[c] = 0.5 * B * tr * d[c] + 0.5 * C * dQd * d[c] + B * Qd[c];
}

/* Eq. 1: acceleration on the evaluation point from a particle of mass m at
 * separation d = x_j - x_i (already the image to use).  G = 1.  eta = r_cut/2. */
void or_pair_accel(const double d[3], double m, double eta, double eps, double out[3])
{
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    out[0] = out[1] = out[2] = 0.0;
    if (r2 == 0.0) return;
    double r = sqrt(r2);
    double g = or_g_p3m(r / eta);
    if (g == 0.0) return;
    double s2 = r2 + eps * eps;
    double f = m * g / (s2 * sqrt(s2));
    out[0] = f * d[0];
    out[1] = f * d[1];
    out[2] = f * d[2];
}

/* Periodic wrap into [0, L) (reading stated in the header). */
double or_wrap(double x, double L)
{
    double r = x - L * floor(x / L);
    if (r < 0.0) r = r + L;
    if (r >= L) r = r - L;
    if (!(r >= 0.0 && r < L)) r = 0.0;
    return r;
}

/* Integer cell index along one axis at the finest level (21). */
int64_t or_cell_index(double r, double L)
{
    double q = (r / L) * 2097152.0;
    double f = floor(q);
    int64_t i = (int64_t)f;
    if (i < 0) i = 0;
    if (i > 2097151) i = 2097151;
    return i;
}

/* 63-bit Morton key, one bit at a time (the x bit is the high bit of each triplet). */
uint64_t or_morton(int64_t ix, int64_t iy, int64_t iz)
{
    uint64_t k = 0;
    for (int b = 0; b < 21; b++) {
        k |= (uint64_t)((ix >> b) & 1) << (3 * b + 2);
        k |= (uint64_t)((iy >> b) & 1) << (3 * b + 1);
        k |= (uint64_t)((iz >> b) & 1) << (3 * b + 0);
    }
    return k;
}

/* Smallest level whose cell side is below L/2 - r_cut; -1 if no level <= 21 qualifies. */
int or_lmin(double L, double r_cut)
{
    double lim = 0.5 * L - r_cut;
    double s = L;
    for (int k = 0; k <= OR_MAXLEVEL; k++) {
        if (s < lim) return k;
        s = s * 0.5;
    }
    return -1;
}

/* ------------------------------------------------------------------------- */
/* Brute-force minimum-image direct sum (the plain definition the tree approximates). */
static double min_image(double d, double L)
{
    double h = 0.5 * L;
    while (d > h) d -= L;
    while (d < -h) d += L;
    return d;
}

/* Eq. 1 summed over every other particle j (minimum image, index order) for particle i
 * of the wrapped positions w. */
static void direct_one(const double *w, const float *mass, int64_t N, double L, double eta, double eps, int64_t i,
                       double *out)
{
    double a[3] = {0, 0, 0};
    for (int64_t j = 0; j < N; j++) {
        if (j == i) continue;
        double d[3], f[3];
        for (int c = 0; c < 3; c++) d[c] = min_image(w[3 * j + c] - w[3 * i + c], L);
        or_pair_accel(d, (double)mass[j], eta, eps, f);
        a[0] += f[0];
        a[1] += f[1];
        a[2] += f[2];
    }
    out[0] = a[0];
    out[1] = a[1];
    out[2] = a[2];
}

int or_direct(const double *pos, const float *mass, int64_t N, double L, double r_cut, double eps,
              double *acc, int nthreads)
{
    if (N < 1 || !(L > 0) || !(r_cut > 0) || !(r_cut < 0.5 * L)) return -1;
    double eta = 0.5 * r_cut;
    double *w = (double *)malloc(sizeof(double) * 3 * N);
    if (!w) return -3;
    for (int64_t i = 0; i < 3 * N; i++) w[i] = or_wrap(pos[i], L);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t i = 0; i < N; i++) direct_one(w, mass, N, L, eta, eps, i, acc + 3 * i);
    free(w);
    return 0;
}

/* The same sum for the particles idx[0..nt) only (acc [nt,3]): O(N) per particle, for the
 * tree-against-direct error on sets too large for the whole O(N^2) sum. */
int or_direct_at(const double *pos, const float *mass, int64_t N, double L, double r_cut, double eps,
                 const int64_t *idx, int64_t nt, double *acc, int nthreads)
{
    if (N < 1 || nt < 0 || !(L > 0) || !(r_cut > 0) || !(r_cut < 0.5 * L)) return -1;
    for (int64_t k = 0; k < nt; k++)
        if (idx[k] < 0 || idx[k] >= N) return -1;
    double eta = 0.5 * r_cut;
    double *w = (double *)malloc(sizeof(double) * 3 * N);
    if (!w) return -3;
    for (int64_t i = 0; i < 3 * N; i++) w[i] = or_wrap(pos[i], L);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t k = 0; k < nt; k++) direct_one(w, mass, N, L, eta, eps, idx[k], acc + 3 * k);
    free(w);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Tree state.  Nodes are numbered in DFS preorder. */
typedef struct {
    int64_t N;
    double L, r_cut, eta, u;
    int n_leaf, n_crit, lmin;
    /* particles in sorted order */
    double *x, *y, *z;
    float *m;
    uint64_t *key;
    int64_t *perm; /* sorted position -> input index */
    /* nodes */
    int64_t nn, ncap;
    int32_t *lvl;
    int64_t *ix, *iy, *iz; /* cell index at the node's own level */
    int64_t *beg, *end, *skip;
    int8_t *leaf;
    double *M, *cx, *cy, *cz;
    double *Q;  /* [nn][6] second moments about the COM: xx, yy, zz, xy, xz, yz (Sec. 4.1) */
    /* groups (node indices, preorder) */
    int64_t ng;
    int64_t *grp;
    /* lists for a set of groups, CSR over the set */
    int64_t nlg;      /* number of groups with lists */
    int64_t *lgrp;    /* which groups */
    int64_t *loff;    /* nlg+1 offsets */
    int64_t nent, ecap;
    int8_t *ekind;    /* 0 particle, 1 node */
    int64_t *eidx;    /* sorted particle index or node index */
    int8_t *esh;      /* 3 per entry: image shift in units of L, -1/0/+1 */
    double theta;
} or_tree;

typedef struct {
    uint64_t key;
    int64_t idx;
} kv_t;

static int kv_cmp(const void *a, const void *b)
{
    const kv_t *p = (const kv_t *)a, *q = (const kv_t *)b;
    if (p->key < q->key) return -1;
    if (p->key > q->key) return 1;
    if (p->idx < q->idx) return -1;
    if (p->idx > q->idx) return 1;
    return 0;
}

static int grow_nodes(or_tree *t)
{
    int64_t nc = t->ncap ? 2 * t->ncap : 1024;
#define RE(p, T)                                                 \
    do {                                                         \
        void *q = realloc(t->p, sizeof(T) * (size_t)nc);         \
        if (!q) return -3;                                       \
        t->p = (T *)q;                                           \
    } while (0)
    RE(lvl, int32_t); RE(ix, int64_t); RE(iy, int64_t); RE(iz, int64_t);
    RE(beg, int64_t); RE(end, int64_t); RE(skip, int64_t); RE(leaf, int8_t);
    RE(M, double); RE(cx, double); RE(cy, double); RE(cz, double);
    {
        void *q = realloc(t->Q, sizeof(double) * 6 * (size_t)nc);
        if (!q) return -3;
        t->Q = (double *)q;
    }
#undef RE
    t->ncap = nc;
    return 0;
}

/* Digit (octant) of a key at level k (1..21): bits 3*(21-k) .. 3*(21-k)+2. */
static int digit_at(uint64_t key, int k) { return (int)((key >> (3 * (21 - k))) & 7u); }

static int build_rec(or_tree *t, int level, int64_t b, int64_t e, int64_t ix, int64_t iy, int64_t iz)
{
    if (t->nn == t->ncap && grow_nodes(t)) return -3;
    int64_t n = t->nn++;
    t->lvl[n] = level;
    t->ix[n] = ix;
    t->iy[n] = iy;
    t->iz[n] = iz;
    t->beg[n] = b;
    t->end[n] = e;
    /* monopole moments, summed sequentially in sorted order (Sec. 3.1.2) */
    double M = 0, sx = 0, sy = 0, sz = 0;
    for (int64_t j = b; j < e; j++) {
        double mj = (double)t->m[j];
        M += mj;
        sx += mj * t->x[j];
        sy += mj * t->y[j];
        sz += mj * t->z[j];
    }
    t->M[n] = M;
    if (M > 0) {
        t->cx[n] = sx / M;
        t->cy[n] = sy / M;
        t->cz[n] = sz / M;
    } else { /* massless node: use the cell centre */
        double side = t->L / (double)(1LL << level);
        t->cx[n] = ((double)ix + 0.5) * side;
        t->cy[n] = ((double)iy + 0.5) * side;
        t->cz[n] = ((double)iz + 0.5) * side;
    }
    /* second moments about the COM, by their definition (Sec. 4.1: second-order terms) */
    {
        double q[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t j = b; j < e; j++) {
            double mj = (double)t->m[j];
            double dx = t->x[j] - t->cx[n], dy = t->y[j] - t->cy[n], dz = t->z[j] - t->cz[n];
            q[0] += mj * dx * dx;
            q[1] += mj * dy * dy;
            q[2] += mj * dz * dz;
            q[3] += mj * dx * dy;
            q[4] += mj * dx * dz;
            q[5] += mj * dy * dz;
        }
        for (int c = 0; c < 6; c++) t->Q[6 * n + c] = q[c];
    }
    int64_t cnt = e - b;
    int split = level < OR_MAXLEVEL && (level < t->lmin || cnt >= t->n_leaf);
    t->leaf[n] = (int8_t)!split;
    if (split) {
        int64_t s = b;
        for (int o = 0; o < 8; o++) {
            int64_t f = s;
            while (f < e && digit_at(t->key[f], level + 1) == o) f++;
            if (f > s) {
                int rc = build_rec(t, level + 1, s, f, 2 * ix + ((o >> 2) & 1), 2 * iy + ((o >> 1) & 1),
                                   2 * iz + (o & 1));
                if (rc) return rc;
            }
            s = f;
        }
    }
    t->skip[n] = t->nn;
    return 0;
}

static int groups_rec(or_tree *t, int64_t n, int64_t *cap)
{
    int64_t cnt = t->end[n] - t->beg[n];
    if (t->lvl[n] >= t->lmin && (cnt <= t->n_crit || t->leaf[n])) {
        if (t->ng == *cap) {
            *cap = *cap ? 2 * *cap : 1024;
            int64_t *q = (int64_t *)realloc(t->grp, sizeof(int64_t) * (size_t)*cap);
            if (!q) return -3;
            t->grp = q;
        }
        t->grp[t->ng++] = n;
        return 0;
    }
    for (int64_t c = n + 1; c < t->skip[n]; c = t->skip[c]) {
        int rc = groups_rec(t, c, cap);
        if (rc) return rc;
    }
    return 0;
}

void or_tree_free(or_tree *t)
{
    if (!t) return;
    free(t->x); free(t->y); free(t->z); free(t->m); free(t->key); free(t->perm);
    free(t->lvl); free(t->ix); free(t->iy); free(t->iz); free(t->beg); free(t->end);
    free(t->skip); free(t->leaf); free(t->M); free(t->cx); free(t->cy); free(t->cz); free(t->Q);
    free(t->grp); free(t->lgrp); free(t->loff); free(t->ekind); free(t->eidx); free(t->esh);
    free(t);
}

/* Steps 1-4: wrap, keys, stable sort, tree + moments, groups.  Returns NULL on bad
 * arguments or allocation failure; *err gets the reason (-1 argument, -3 memory). */
or_tree *or_tree_build(const double *pos, const float *mass, int64_t N, double L, double r_cut, int n_leaf,
                       int n_crit, int *err)
{
    *err = -1;
    if (N < 1 || !(L > 0) || !(r_cut > 0) || !(r_cut < 0.5 * L) || n_leaf < 1 || n_crit < 1) return NULL;
    int lmin = or_lmin(L, r_cut);
    if (lmin < 0) return NULL;
    for (int64_t i = 0; i < 3 * N; i++)
        if (!isfinite(pos[i])) return NULL;
    *err = -3;
    or_tree *t = (or_tree *)calloc(1, sizeof(or_tree));
    if (!t) return NULL;
    t->N = N;
    t->L = L;
    t->r_cut = r_cut;
    t->eta = 0.5 * r_cut;
    t->u = L / 4194304.0;
    t->n_leaf = n_leaf;
    t->n_crit = n_crit;
    t->lmin = lmin;
    kv_t *kv = (kv_t *)malloc(sizeof(kv_t) * (size_t)N);
    double *w = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    t->x = (double *)malloc(sizeof(double) * (size_t)N);
    t->y = (double *)malloc(sizeof(double) * (size_t)N);
    t->z = (double *)malloc(sizeof(double) * (size_t)N);
    t->m = (float *)malloc(sizeof(float) * (size_t)N);
    t->key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    t->perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    if (!kv || !w || !t->x || !t->y || !t->z || !t->m || !t->key || !t->perm) {
        free(kv); free(w); or_tree_free(t);
        return NULL;
    }
    for (int64_t i = 0; i < N; i++) {
        for (int c = 0; c < 3; c++) w[3 * i + c] = or_wrap(pos[3 * i + c], L);
        kv[i].key = or_morton(or_cell_index(w[3 * i], L), or_cell_index(w[3 * i + 1], L),
                              or_cell_index(w[3 * i + 2], L));
        kv[i].idx = i;
    }
    qsort(kv, (size_t)N, sizeof(kv_t), kv_cmp);
    for (int64_t s = 0; s < N; s++) {
        int64_t i = kv[s].idx;
        t->key[s] = kv[s].key;
        t->perm[s] = i;
        t->x[s] = w[3 * i];
        t->y[s] = w[3 * i + 1];
        t->z[s] = w[3 * i + 2];
        t->m[s] = mass[i];
    }
    free(kv);
    free(w);
    if (build_rec(t, 0, 0, N, 0, 0, 0)) { or_tree_free(t); return NULL; }
    int64_t gcap = 0;
    if (groups_rec(t, 0, &gcap)) { or_tree_free(t); return NULL; }
    *err = 0;
    return t;
}

int64_t or_tree_n_nodes(const or_tree *t) { return t->nn; }
int64_t or_tree_n_groups(const or_tree *t) { return t->ng; }
int or_tree_lmin(const or_tree *t) { return t->lmin; }

void or_tree_get_sorted(const or_tree *t, uint64_t *key, int64_t *perm, double *xyz, float *m)
{
    for (int64_t s = 0; s < t->N; s++) {
        if (key) key[s] = t->key[s];
        if (perm) perm[s] = t->perm[s];
        if (xyz) { xyz[3 * s] = t->x[s]; xyz[3 * s + 1] = t->y[s]; xyz[3 * s + 2] = t->z[s]; }
        if (m) m[s] = t->m[s];
    }
}

/* nodes: [nn, 9] int64 = level, ix, iy, iz, begin, end, skip, leaf, 0 */
void or_tree_get_nodes(const or_tree *t, int64_t *out)
{
    for (int64_t n = 0; n < t->nn; n++) {
        int64_t *o = out + 9 * n;
        o[0] = t->lvl[n]; o[1] = t->ix[n]; o[2] = t->iy[n]; o[3] = t->iz[n];
        o[4] = t->beg[n]; o[5] = t->end[n]; o[6] = t->skip[n]; o[7] = t->leaf[n]; o[8] = 0;
    }
}

/* moments: [nn, 4] double = M, cx, cy, cz */
void or_tree_get_moments(const or_tree *t, double *out)
{
    for (int64_t n = 0; n < t->nn; n++) {
        out[4 * n] = t->M[n]; out[4 * n + 1] = t->cx[n]; out[4 * n + 2] = t->cy[n]; out[4 * n + 3] = t->cz[n];
    }
}

/* second moments: [nn, 6] double = xx, yy, zz, xy, xz, yz about the COM */
void or_tree_get_quadrupoles(const or_tree *t, double *out)
{
    for (int64_t n = 0; n < 6 * t->nn; n++) out[n] = t->Q[n];
}

void or_tree_get_groups(const or_tree *t, int64_t *out)
{
    for (int64_t g = 0; g < t->ng; g++) out[g] = t->grp[g];
}

/* ------------------------------------------------------------------------- */
/* Step 5: interaction list of one group, DFS preorder over the tree. */
typedef struct {
    or_tree *t;
    int64_t cg[3], hg; /* group cell centre and half side, units of u */
    int64_t cb[3], hb[3]; /* centre and half sides of the group's particle box, units of u */
    double uu, rc2, th2;
    int eq12;              /* distance-dependent theta (Eq. 12) */
    double t02, tmax2;     /* theta0^2, theta_max^2 */
    double u_over_eta;
} walk_t;

/* theta^2 of the accept test at squared distance sd (units of u^2). */
static double walk_theta2(const walk_t *W, int64_t sd)
{
    if (!W->eq12) return W->th2;
    double R = sqrt((double)sd) * W->u_over_eta;
    double rg = R * or_g_p3m(R);
    if (!(rg > 0.0)) return W->tmax2;
    double t2 = W->t02 / rg;
    return t2 < W->tmax2 ? t2 : W->tmax2;
}

/* r_cut test of a box (centre d relative to the group cell centre, already the image
 * to use; half side h, all in u) against the group's particle box. */
static int beyond_rcut(const walk_t *W, const int64_t d[3], int64_t h)
{
    int64_t sgap = 0;
    for (int c = 0; c < 3; c++) {
        int64_t e = d[c] - (W->cb[c] - W->cg[c]);
        if (e < 0) e = -e;
        int64_t gap = e - h - W->hb[c];
        if (gap < 0) gap = 0;
        sgap += gap * gap;
    }
    return (double)sgap * W->uu > W->rc2;
}

static int push_entry(or_tree *t, int kind, int64_t idx, const int sh[3])
{
    if (t->nent == t->ecap) {
        int64_t nc = t->ecap ? 2 * t->ecap : 4096;
        int8_t *k = (int8_t *)realloc(t->ekind, (size_t)nc);
        if (!k) return -3;
        t->ekind = k;
        int64_t *x = (int64_t *)realloc(t->eidx, sizeof(int64_t) * (size_t)nc);
        if (!x) return -3;
        t->eidx = x;
        int8_t *s = (int8_t *)realloc(t->esh, 3 * (size_t)nc);
        if (!s) return -3;
        t->esh = s;
        t->ecap = nc;
    }
    t->ekind[t->nent] = (int8_t)kind;
    t->eidx[t->nent] = idx;
    for (int c = 0; c < 3; c++) t->esh[3 * t->nent + c] = (int8_t)sh[c];
    t->nent++;
    return 0;
}

static int walk_rec(walk_t *W, int64_t n)
{
    or_tree *t = W->t;
    int k = t->lvl[n];
    int64_t hn = (int64_t)1 << (21 - k);
    int64_t cn[3] = {(2 * t->ix[n] + 1) * hn, (2 * t->iy[n] + 1) * hn, (2 * t->iz[n] + 1) * hn};
    const int64_t P = (int64_t)1 << 22, H = (int64_t)1 << 21;
    int64_t sd = 0, dn[3];
    int sh[3];
    for (int c = 0; c < 3; c++) {
        int64_t d = cn[c] - W->cg[c];
        sh[c] = 0;
        if (d >= H) { d -= P; sh[c] = -1; }
        else if (d < -H) { d += P; sh[c] = 1; }
        dn[c] = d;
        int64_t ad = d < 0 ? -d : d;
        int64_t e = ad - W->hg;
        if (e < 0) e = 0;
        sd += e * e;
    }
    /* r_cut pruning: the whole node lies farther than r_cut from the group's particles */
    if (beyond_rcut(W, dn, hn)) return 0;
    /* opening criterion (Barnes-Hut on cell side, distance to the group cell) */
    int64_t l = 2 * hn;
    if (k >= t->lmin && (double)(l * l) < walk_theta2(W, sd) * (double)sd) return push_entry(t, 1, n, sh);
    if (t->leaf[n]) {
        for (int64_t j = t->beg[n]; j < t->end[n]; j++) {
            /* the particle's finest cell, in the node's image */
            int64_t dj[3] = {2 * or_cell_index(t->x[j], t->L) + 1 - W->cg[0],
                             2 * or_cell_index(t->y[j], t->L) + 1 - W->cg[1],
                             2 * or_cell_index(t->z[j], t->L) + 1 - W->cg[2]};
            for (int c = 0; c < 3; c++) dj[c] += (int64_t)sh[c] * P;
            if (beyond_rcut(W, dj, 1)) continue;
            int rc = push_entry(t, 0, j, sh);
            if (rc) return rc;
        }
        return 0;
    }
    for (int64_t c = n + 1; c < t->skip[n]; c = t->skip[c]) {
        int rc = walk_rec(W, c);
        if (rc) return rc;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Local essential tree for one receiving domain (Sec. 2.2 step 3): walk the tree in
 * preorder; a node whose cell lies farther than r_cut from the domain box is skipped, a
 * node that satisfies the opening criterion from the box (level >= l_min, l^2 < theta^2 d^2
 * with d the distance from its cell centre to the nearest point of the box) is sent as
 * one item, a leaf that is opened sends its particles whose finest cell lies within r_cut
 * of the box, and any other node is opened.  The same tests as the list walk (readings C1,
 * C2, C4) with the box in place of the group's cell and particle box.  The box is
 * [lo, hi) per axis in finest cells, i.e. [2 lo, 2 hi) in u; distances are periodic. */
typedef struct {
    const or_tree *t;
    int64_t cb[3], hb[3]; /* box centre and half sides, units u */
    double uu, rc2, th2;
    int64_t *kind, *idx;  /* output: kind 1 node / 0 particle, index */
    int64_t n, cap;
} let_t;

static int64_t per_gap(int64_t cbox, int64_t c, int64_t hsum)
{
    const int64_t P = (int64_t)1 << 22, H = (int64_t)1 << 21;
    int64_t d = cbox - c;
    if (d >= H) d -= P;
    else if (d < -H) d += P;
    if (d < 0) d = -d;
    d -= hsum;
    return d > 0 ? d : 0;
}

static int let_push(let_t *W, int64_t kind, int64_t idx)
{
    if (W->n < W->cap) {
        W->kind[W->n] = kind;
        W->idx[W->n] = idx;
    }
    W->n++;
    return 0;
}

static void let_rec(let_t *W, int64_t n)
{
    const or_tree *t = W->t;
    int k = t->lvl[n];
    int64_t hn = (int64_t)1 << (21 - k);
    int64_t cn[3] = {(2 * t->ix[n] + 1) * hn, (2 * t->iy[n] + 1) * hn, (2 * t->iz[n] + 1) * hn};
    int64_t sgap = 0, sd = 0;
    for (int c = 0; c < 3; c++) {
        int64_t g = per_gap(W->cb[c], cn[c], hn + W->hb[c]);
        int64_t e = per_gap(W->cb[c], cn[c], W->hb[c]);
        sgap += g * g;
        sd += e * e;
    }
    if ((double)sgap * W->uu > W->rc2) return;
    int64_t l = 2 * hn;
    if (k >= t->lmin && (double)(l * l) < W->th2 * (double)sd) {
        let_push(W, 1, n);
        return;
    }
    if (t->leaf[n]) {
        for (int64_t j = t->beg[n]; j < t->end[n]; j++) {
            int64_t cj[3] = {2 * or_cell_index(t->x[j], t->L) + 1, 2 * or_cell_index(t->y[j], t->L) + 1,
                             2 * or_cell_index(t->z[j], t->L) + 1};
            int64_t s2 = 0;
            for (int c = 0; c < 3; c++) {
                int64_t g = per_gap(W->cb[c], cj[c], 1 + W->hb[c]);
                s2 += g * g;
            }
            if ((double)s2 * W->uu > W->rc2) continue;
            let_push(W, 0, j);
        }
        return;
    }
    for (int64_t c = n + 1; c < t->skip[n]; c = t->skip[c]) let_rec(W, c);
}

/* Items of the LET for box[6] at opening angle theta: kind/idx [cap]; returns the number
 * of items (those beyond cap are counted, not written), or -1 for a bad box. */
int64_t or_let_export(const or_tree *t, const int32_t box[6], double theta, int64_t *kind, int64_t *idx, int64_t cap)
{
    if (!(theta >= 0)) return -1;
    let_t W;
    W.t = t;
    for (int c = 0; c < 3; c++) {
        int64_t lo = box[2 * c], hi = box[2 * c + 1];
        if (lo < 0 || hi > ((int64_t)1 << 21) || lo > hi) return -1;
        if (lo == hi) return 0;
        W.cb[c] = lo + hi;
        W.hb[c] = hi - lo;
    }
    W.uu = t->u * t->u;
    W.rc2 = t->r_cut * t->r_cut;
    W.th2 = theta * theta;
    W.kind = kind;
    W.idx = idx;
    W.n = 0;
    W.cap = cap;
    let_rec(&W, 0);
    return W.n;
}

/* Build lists for groups gsel[0..ns) (all groups when gsel == NULL). */
static int lists_build(or_tree *t, double theta, int eq12, double theta0, const int64_t *gsel, int64_t ns);

/* Lists with the constant opening angle theta. */
int or_lists_build(or_tree *t, double theta, const int64_t *gsel, int64_t ns)
{
    return lists_build(t, theta, 0, 0.0, gsel, ns);
}

/* Lists with the distance-dependent opening angle of Eq. 12 (theta0), capped at theta_max. */
int or_lists_build_eq12(or_tree *t, double theta0, double theta_max, const int64_t *gsel, int64_t ns)
{
    if (!(theta0 >= 0)) return -1;
    return lists_build(t, theta_max, 1, theta0, gsel, ns);
}

static int lists_build(or_tree *t, double theta, int eq12, double theta0, const int64_t *gsel, int64_t ns)
{
    if (!(theta >= 0)) return -1;
    if (!gsel) ns = t->ng;
    free(t->lgrp); free(t->loff);
    t->lgrp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ns > 0 ? ns : 1));
    t->loff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ns + 1));
    if (!t->lgrp || !t->loff) return -3;
    t->nlg = ns;
    t->nent = 0;
    t->theta = theta;
    walk_t W;
    W.t = t;
    W.uu = t->u * t->u;
    W.rc2 = t->r_cut * t->r_cut;
    W.th2 = theta * theta;
    W.eq12 = eq12;
    W.t02 = theta0 * theta0;
    W.tmax2 = theta * theta;
    W.u_over_eta = t->u / t->eta;
    for (int64_t s = 0; s < ns; s++) {
        int64_t g = gsel ? gsel[s] : s;
        if (g < 0 || g >= t->ng) return -1;
        int64_t n = t->grp[g];
        int k = t->lvl[n];
        W.hg = (int64_t)1 << (21 - k);
        W.cg[0] = (2 * t->ix[n] + 1) * W.hg;
        W.cg[1] = (2 * t->iy[n] + 1) * W.hg;
        W.cg[2] = (2 * t->iz[n] + 1) * W.hg;
        {
            const double *xs[3] = {t->x, t->y, t->z};
            for (int c = 0; c < 3; c++) {
                int64_t lo = 2097151, hi = 0;
                for (int64_t j = t->beg[n]; j < t->end[n]; j++) {
                    int64_t q = or_cell_index(xs[c][j], t->L);
                    if (q < lo) lo = q;
                    if (q > hi) hi = q;
                }
                /* finest cells lo..hi span [2 lo, 2 hi + 2] in u */
                W.cb[c] = lo + hi + 1;
                W.hb[c] = hi - lo + 1;
            }
        }
        t->lgrp[s] = g;
        t->loff[s] = t->nent;
        int rc = walk_rec(&W, 0);
        if (rc) return rc;
    }
    t->loff[ns] = t->nent;
    return 0;
}

int64_t or_lists_n_entries(const or_tree *t) { return t->nent; }

/* offsets: nlg+1; kind: nent; idx: nent; shift: 3*nent */
void or_lists_get(const or_tree *t, int64_t *offsets, int8_t *kind, int64_t *idx, int8_t *shift)
{
    for (int64_t s = 0; s <= t->nlg; s++) offsets[s] = t->loff[s];
    for (int64_t e = 0; e < t->nent; e++) {
        kind[e] = t->ekind[e];
        idx[e] = t->eidx[e];
        for (int c = 0; c < 3; c++) shift[3 * e + c] = t->esh[3 * e + c];
    }
}

/* Step 6: FP64 force from the lists, Eq. 1-2, per-pair minimum image against the
 * entry position (particle or node centre of mass).  acc_sorted gets [N,3] in
 * sorted order; only particles of groups with lists are written (others zero). */
static int list_force(const or_tree *t, double eps, int quad, double *acc_sorted, int nthreads);

int or_list_force(const or_tree *t, double eps, double *acc_sorted, int nthreads)
{
    return list_force(t, eps, 0, acc_sorted, nthreads);
}

/* The same with the second-order terms of Sec. 4.1 added for node entries (eps = 0). */
int or_list_force_quad(const or_tree *t, double *acc_sorted, int nthreads)
{
    return list_force(t, 0.0, 1, acc_sorted, nthreads);
}

static int list_force(const or_tree *t, double eps, int quad, double *acc_sorted, int nthreads)
{
    memset(acc_sorted, 0, sizeof(double) * 3 * (size_t)t->N);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t s = 0; s < t->nlg; s++) {
        int64_t n = t->grp[t->lgrp[s]];
        for (int64_t i = t->beg[n]; i < t->end[n]; i++) {
            double a[3] = {0, 0, 0};
            double xi[3] = {t->x[i], t->y[i], t->z[i]};
            for (int64_t e = t->loff[s]; e < t->loff[s + 1]; e++) {
                double xj[3], mj;
                int64_t j = t->eidx[e];
                if (t->ekind[e] == 0) {
                    xj[0] = t->x[j]; xj[1] = t->y[j]; xj[2] = t->z[j];
                    mj = (double)t->m[j];
                } else {
                    xj[0] = t->cx[j]; xj[1] = t->cy[j]; xj[2] = t->cz[j];
                    mj = t->M[j];
                }
                double d[3], f[3];
                for (int c = 0; c < 3; c++) d[c] = min_image(xj[c] - xi[c], t->L);
                or_pair_accel(d, mj, t->eta, eps, f);
                a[0] += f[0];
                a[1] += f[1];
                a[2] += f[2];
                if (quad && t->ekind[e] == 1) {
                    or_quad_accel(d, t->Q + 6 * j, t->eta, f);
                    a[0] += f[0];
                    a[1] += f[1];
                    a[2] += f[2];
                }
            }
            acc_sorted[3 * i] = a[0];
            acc_sorted[3 * i + 1] = a[1];
            acc_sorted[3 * i + 2] = a[2];
        }
    }
    return 0;
}

/* Convenience: whole pipeline, acceleration in input order ([N,3] FP64). */
int or_short_force(const double *pos, const float *mass, int64_t N, double L, double r_cut, double theta,
                   int n_crit, int n_leaf, double eps, double *acc, int nthreads)
{
    int err;
    or_tree *t = or_tree_build(pos, mass, N, L, r_cut, n_leaf, n_crit, &err);
    if (!t) return err;
    int rc = or_lists_build(t, theta, NULL, 0);
    if (rc) { or_tree_free(t); return rc; }
    double *as = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    if (!as) { or_tree_free(t); return -3; }
    or_list_force(t, eps, as, nthreads);
    for (int64_t s = 0; s < N; s++)
        for (int c = 0; c < 3; c++) acc[3 * t->perm[s] + c] = as[3 * s + c];
    free(as);
    or_tree_free(t);
    return 0;
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
