/*
 * pt_oracle.c -- plain CPU oracle for the P3T long-range force.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or helper
 * with the CUDA library; the two meet only through the seeded input arrays.
 *
 * Everything is float64, written to be read against the paper:
 *   Wang, Iwasawa, Nitadori & Makino (2020), "PeTar: a high-performance
 *   N-body code for modelling massive collisional stellar systems".
 *
 *   Sec. 5.1, Eq. 11   Hamiltonian split: H_L carries G m_i m_j (1 - W)/r_ij
 *   Sec. 6.1, Eq. 15   potential changeover W(x)
 *   Sec. 6.1, Eq. 16   helper f(x), x = (r - r_in)/(r_out - r_in), Lambda
 *   Sec. 6.1, Eq. 17   force changeover K(x)
 *   Sec. 6.1, Eq. 18   W = f - f(1) r / r_out,  K = f - (x + r_in/(r_out-r_in)) f'
 *   Sec. 4, Sec. 5.1 (Fig. 2)  Barnes-Hut tree; a cell "inside theta" acts
 *                      as a super-particle (centre of mass + multipoles)
 *   Sec. 6.4.2, Eqs. 30-31  quadrupole tensor and its traceless form
 *   Sec. 6 (Fig. 3 schedule, step 2)  tree neighbour search within r_out
 *   Sec. 6.3.1, Eq. 24 orbit-dependent neighbour radius, pericentre stage
 *
 * Functions:
 *   orc_f / orc_W / orc_K      changeover functions exactly as printed
 *   orc_direct                 direct O(N^2) long-range acc and pot
 *   orc_direct_short           direct short-range part (split-identity pin)
 *   orc_neighbours_*           brute-force r_out neighbour sets
 *   orc_pericentre, orc_rnb,   orbit-dependent neighbour radius (Eq. 24) and
 *   orc_orbit_*                the two-stage pericentre selection (Sec. 6.3.1)
 *   orc_tree_*                 keys, stable sort, octree, moments, groups,
 *                              group-wise walk and tree force
 *
 * Readings where the paper is silent (the tree definition, the opening rule,
 * the key scheme, the treatment of r <= r_in for the potential) are stated
 * at each function.  Parity status: the changeover functions, the direct
 * sum, the neighbour sets, keys/sort/topology and the theta = 0 tree are
 * pinned by tests against closed forms, identities and brute force; a
 * cell's potential and acceleration are pinned by the Legendre expansion of
 * two point masses, by acceleration = -grad(potential) and by their
 * truncation orders; the size of the tree-versus-direct truncation error has
 * no printed value in the paper (parity unpinned for that magnitude; only
 * its scaling is pinned).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_BITS 21                      /* grid bits per dimension       */
#define ORC_GRID (1u << ORC_BITS)        /* 2^21 cells per dimension      */

/* ------------------------------------------------------------------------ */
/* Changeover functions, Sec. 6.1                                           */
/* ------------------------------------------------------------------------ */

/* Eq. 16: f(x) = 1 + Lambda x^5 (14 - 28 x + 20 x^2 - 5 x^3). */
double orc_f(double x, double lam)
{
    double x5 = x * x * x * x * x;
    return 1.0 + lam * x5 * (14.0 - 28.0 * x + 20.0 * x * x - 5.0 * x * x * x);
}

/* Eq. 15: W(x) = Lambda (1 - 2x) for x <= 0, Lambda (1 - 2x) - 1 + f(x)
 * for 0 < x < 1, and 0 for x >= 1. */
double orc_W(double x, double lam)
{
    if (x <= 0.0) return lam * (1.0 - 2.0 * x);
    if (x < 1.0) return lam * (1.0 - 2.0 * x) - 1.0 + orc_f(x, lam);
    return 0.0;
}

/* Eq. 17: K(x) = 1 for x <= 0, (x-1)^4 (1 + 4x + 10x^2 + 20x^3 + 35 Lambda x^4)
 * for 0 < x < 1, and 0 for x >= 1. */
double orc_K(double x, double lam)
{
    if (x <= 0.0) return 1.0;
    if (x < 1.0) {
        double t = x - 1.0;
        return t * t * t * t *
               (1.0 + 4.0 * x + 10.0 * x * x + 20.0 * x * x * x + 35.0 * lam * x * x * x * x);
    }
    return 0.0;
}

/* Long-range pull of particle j (mass mj at xj) on the point xi, Eq. 11 with
 * Eqs. 15-17, without the factor G:
 *   acc += mj (xj - xi) (1 - K) / r^3,   pot += -mj (1 - W) / r.
 * For r <= r_in (x <= 0) K = 1, so the force vanishes, and with
 * W = Lambda (1 - 2x) the identity 1 - Lambda + 2 Lambda x = 2 r / (r_out + r_in)
 * gives the constant (1 - W)/r = 2/(r_out + r_in); it is used in that form so
 * that coincident particles (r = 0) give a finite potential. */
static void pair_longrange(const double *xi, const double *xj, double mj,
                           double r_in, double r_out, double *acc, double *pot)
{
    double dx = xj[0] - xi[0], dy = xj[1] - xi[1], dz = xj[2] - xi[2];
    double r2 = dx * dx + dy * dy + dz * dz;
    double r = sqrt(r2);
    double lam = (r_out - r_in) / (r_out + r_in);
    double x = (r - r_in) / (r_out - r_in);
    if (x <= 0.0) {
        *pot += -mj * 2.0 / (r_out + r_in);
        return;
    }
    double K = orc_K(x, lam), W = orc_W(x, lam);
    double r3 = r2 * r;
    acc[0] += mj * dx * (1.0 - K) / r3;
    acc[1] += mj * dy * (1.0 - K) / r3;
    acc[2] += mj * dz * (1.0 - K) / r3;
    *pot += -mj * (1.0 - W) / r;
}

/* Short-range part (the H_S side of Eq. 11): acc += mj dx K / r^3,
 * pot += -mj W / r, for r > 0.  Used only to pin the split identity. */
static void pair_shortrange(const double *xi, const double *xj, double mj,
                            double r_in, double r_out, double *acc, double *pot)
{
    double dx = xj[0] - xi[0], dy = xj[1] - xi[1], dz = xj[2] - xi[2];
    double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 == 0.0) return;
    double r = sqrt(r2);
    double lam = (r_out - r_in) / (r_out + r_in);
    double x = (r - r_in) / (r_out - r_in);
    double K = orc_K(x, lam), W = orc_W(x, lam);
    double r3 = r2 * r;
    acc[0] += mj * dx * K / r3;
    acc[1] += mj * dy * K / r3;
    acc[2] += mj * dz * K / r3;
    *pot += -mj * W / r;
}

/* ------------------------------------------------------------------------ */
/* Direct summation (the plain definition the tree approximates)            */
/* ------------------------------------------------------------------------ */

/* For each target t (original index targets[t], or t itself when targets is
 * NULL): a = G sum_{j != i} m_j (x_j - x_i)(1 - K)/r^3 and
 * phi = -G sum_{j != i} m_j (1 - W)/r, j in ascending order. */
/* Mass-dependent changeover (Sec. 6.1, Eq. 12): particle i has radii
 * s_i (r_in, r_out) and a pair uses the larger of the two (Eq. 16:
 * r_in,ij = max(r_in,i, r_in,j), same for r_out).  scale == NULL means s = 1. */
static double pair_scale(const double *scale, int64_t i, int64_t j)
{
    if (!scale) return 1.0;
    return scale[i] > scale[j] ? scale[i] : scale[j];
}

/* Eq. 12: s_i = max(1, m_i / <m>)^(1/3), <m> the mean mass (summed in index order). */
void orc_radius_scale(int64_t n, const double *mass, double *scale)
{
    double M = 0.0;
    for (int64_t i = 0; i < n; i++) M += mass[i];
    double mean = M / (double)n;
    for (int64_t i = 0; i < n; i++) {
        double q = mass[i] / mean;
        scale[i] = cbrt(q > 1.0 ? q : 1.0);
    }
}

void orc_direct(int64_t n, const double *pos, const double *mass, double G,
                double r_in, double r_out, int64_t nt, const int64_t *targets,
                double *acc, double *pot, int shortrange, const double *scale)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; t++) {
        int64_t i = targets ? targets[t] : t;
        double a[3] = {0.0, 0.0, 0.0}, p = 0.0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double sij = pair_scale(scale, i, j);
            if (shortrange)
                pair_shortrange(pos + 3 * i, pos + 3 * j, mass[j], sij * r_in, sij * r_out, a, &p);
            else
                pair_longrange(pos + 3 * i, pos + 3 * j, mass[j], sij * r_in, sij * r_out, a, &p);
        }
        acc[3 * t + 0] = G * a[0];
        acc[3 * t + 1] = G * a[1];
        acc[3 * t + 2] = G * a[2];
        pot[t] = G * p;
    }
}

/* ------------------------------------------------------------------------ */
/* Neighbour sets: j != i with r^2 < r_out^2, r^2 = dx*dx + dy*dy + dz*dz    */
/* summed left to right (this file is compiled without FMA contraction).    */
/* ------------------------------------------------------------------------ */

static int is_neighbour(const double *xi, const double *xj, double rout2)
{
    double dx = xj[0] - xi[0], dy = xj[1] - xi[1], dz = xj[2] - xi[2];
    double r2 = dx * dx + dy * dy + dz * dz;
    return r2 < rout2;
}

/* The pair's r_out squared: (s_ij r_out)^2 with s_ij = max(s_i, s_j). */
static double pair_rout2(const double *scale, int64_t i, int64_t j, double r_out)
{
    double ro = r_out * pair_scale(scale, i, j);
    return ro * ro;
}

/* counts[t] = number of neighbours of target t. */
void orc_neighbours_count(int64_t n, const double *pos, double r_out, int64_t nt,
                          const int64_t *targets, int64_t *counts, const double *scale)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; t++) {
        int64_t i = targets ? targets[t] : t, c = 0;
        for (int64_t j = 0; j < n; j++)
            if (j != i && is_neighbour(pos + 3 * i, pos + 3 * j, pair_rout2(scale, i, j, r_out))) c++;
        counts[t] = c;
    }
}

/* Fill idx[offsets[t] ..] with the neighbours of target t, ascending. */
void orc_neighbours_fill(int64_t n, const double *pos, double r_out, int64_t nt,
                         const int64_t *targets, const int64_t *offsets, int32_t *idx,
                         const double *scale)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; t++) {
        int64_t i = targets ? targets[t] : t, c = offsets[t];
        for (int64_t j = 0; j < n; j++)
            if (j != i && is_neighbour(pos + 3 * i, pos + 3 * j, pair_rout2(scale, i, j, r_out)))
                idx[c++] = (int32_t)j;
    }
}

/* ------------------------------------------------------------------------ */
/* Tree.  The paper uses the Barnes-Hut tree of FDPS without defining it;   */
/* the definition below is this project's reading, fixed so that every      */
/* structural decision is exactly reproducible:                             */
/*   root box: o = per-dimension minimum, S = largest extent (1 if 0);       */
/*   grid:     q_d = clamp(floor((x_d - o_d) * (2^21 / S)), 0, 2^21 - 1);     */
/*   key:      21 bits per dimension interleaved, bit 3b+2 from q_x,         */
/*             3b+1 from q_y, 3b from q_z;                                    */
/*   order:    ascending key, equal keys by ascending original index;       */
/*   nodes:    the root is all particles (level 0); a node of level l with   */
/*             more than n_leaf particles and l < 21 is split into the       */
/*             non-empty runs that share the top 3(l+1) key bits; otherwise  */
/*             it is a leaf;                                                */
/*   moments:  M, centre of mass, Q = sum m (3 d d^T - |d|^2 I) about the    */
/*             centre of mass (Eq. 31 gives A' = Q / 2), and the tight box   */
/*             of the particles' grid cells.                                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t begin, count;       /* particle range in sorted order           */
    int level, leaf;
    int64_t first_child;        /* children are stored contiguously         */
    int nchild;
    uint32_t qmin[3], qmax[3];  /* tight box in grid cells (inclusive)      */
    double M, com[3], Q[6];     /* Q order: xx, yy, zz, xy, xz, yz          */
    double smax;                /* largest radius scale of its particles    */
} orc_node;

typedef struct {
    int64_t begin, count;
    uint32_t qmin[3], qmax[3];
    double smax;
} orc_group;

typedef struct {
    int64_t n;
    double origin[3], S, scale;
    uint64_t *key;              /* per original index                       */
    uint32_t *q;                /* per original index, 3 each               */
    int64_t *perm;              /* sorted slot -> original index            */
    double *spos, *smass;       /* sorted copies                            */
    double *sscale;             /* sorted radius scales (all 1 if none)     */
    uint32_t *sq;               /* sorted grid coordinates                  */
    uint64_t *skey;
    orc_node *node;
    int64_t nnodes, cap;
    orc_group *group;
    int64_t ngroups, gcap;
    int n_leaf, n_group;
} orc_tree;

static uint64_t interleave(uint32_t qx, uint32_t qy, uint32_t qz)
{
    uint64_t k = 0;
    for (int b = 0; b < ORC_BITS; b++) {
        k |= (uint64_t)((qx >> b) & 1u) << (3 * b + 2);
        k |= (uint64_t)((qy >> b) & 1u) << (3 * b + 1);
        k |= (uint64_t)((qz >> b) & 1u) << (3 * b);
    }
    return k;
}

/* Root box and grid coordinates (this project's key scheme, see above). */
static void compute_keys(orc_tree *t, const double *pos)
{
    int64_t n = t->n;
    double lo[3], hi[3];
    for (int d = 0; d < 3; d++) { lo[d] = pos[d]; hi[d] = pos[d]; }
    for (int64_t i = 1; i < n; i++)
        for (int d = 0; d < 3; d++) {
            double v = pos[3 * i + d];
            if (v < lo[d]) lo[d] = v;
            if (v > hi[d]) hi[d] = v;
        }
    double S = 0.0;
    for (int d = 0; d < 3; d++) {
        t->origin[d] = lo[d];
        if (hi[d] - lo[d] > S) S = hi[d] - lo[d];
    }
    if (S == 0.0) S = 1.0;
    t->S = S;
    t->scale = (double)ORC_GRID / S;
    for (int64_t i = 0; i < n; i++) {
        for (int d = 0; d < 3; d++) {
            double u = floor((pos[3 * i + d] - t->origin[d]) * t->scale);
            if (u < 0.0) u = 0.0;
            if (u > (double)(ORC_GRID - 1)) u = (double)(ORC_GRID - 1);
            t->q[3 * i + d] = (uint32_t)u;
        }
        t->key[i] = interleave(t->q[3 * i], t->q[3 * i + 1], t->q[3 * i + 2]);
    }
}

static const uint64_t *g_sort_keys;     /* comparator context (single thread) */
static int cmp_key_then_index(const void *a, const void *b)
{
    int64_t ia = *(const int64_t *)a, ib = *(const int64_t *)b;
    uint64_t ka = g_sort_keys[ia], kb = g_sort_keys[ib];
    if (ka != kb) return ka < kb ? -1 : 1;
    return ia < ib ? -1 : (ia > ib ? 1 : 0);
}

static int64_t node_alloc(orc_tree *t, int64_t k)
{
    if (t->nnodes + k > t->cap) {
        int64_t nc = t->cap * 2 + k + 16;
        t->node = (orc_node *)realloc(t->node, (size_t)nc * sizeof(orc_node));
        t->cap = nc;
    }
    int64_t first = t->nnodes;
    t->nnodes += k;
    return first;
}

/* Moments of one node straight from its particles (two passes). */
static void node_moments(orc_tree *t, orc_node *v)
{
    double M = 0.0, s[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < 3; d++) { v->qmin[d] = ORC_GRID; v->qmax[d] = 0; }
    v->smax = 0.0;
    for (int64_t p = v->begin; p < v->begin + v->count; p++) {
        double m = t->smass[p];
        if (t->sscale[p] > v->smax) v->smax = t->sscale[p];
        M += m;
        for (int d = 0; d < 3; d++) {
            s[d] += m * t->spos[3 * p + d];
            uint32_t qd = t->sq[3 * p + d];
            if (qd < v->qmin[d]) v->qmin[d] = qd;
            if (qd > v->qmax[d]) v->qmax[d] = qd;
        }
    }
    v->M = M;
    for (int d = 0; d < 3; d++)
        v->com[d] = (M > 0.0) ? s[d] / M : t->spos[3 * v->begin + d];
    for (int k = 0; k < 6; k++) v->Q[k] = 0.0;
    for (int64_t p = v->begin; p < v->begin + v->count; p++) {
        double m = t->smass[p];
        double d0 = t->spos[3 * p] - v->com[0];
        double d1 = t->spos[3 * p + 1] - v->com[1];
        double d2 = t->spos[3 * p + 2] - v->com[2];
        double dd = d0 * d0 + d1 * d1 + d2 * d2;
        v->Q[0] += m * (3.0 * d0 * d0 - dd);
        v->Q[1] += m * (3.0 * d1 * d1 - dd);
        v->Q[2] += m * (3.0 * d2 * d2 - dd);
        v->Q[3] += m * (3.0 * d0 * d1);
        v->Q[4] += m * (3.0 * d0 * d2);
        v->Q[5] += m * (3.0 * d1 * d2);
    }
}

/* The key digit (0..7) of sorted particle p at level l+1. */
static int digit_at(const orc_tree *t, int64_t p, int l)
{
    return (int)((t->skey[p] >> (3 * (ORC_BITS - 1 - l))) & 7u);
}

/* Split node v (index vi) recursively per the node rule above. */
static void build_node(orc_tree *t, int64_t vi)
{
    orc_node *v = &t->node[vi];
    node_moments(t, v);
    if (v->count <= t->n_leaf || v->level >= ORC_BITS) {
        v->leaf = 1;
        v->nchild = 0;
        v->first_child = -1;
        return;
    }
    int64_t b[9];
    int64_t p = v->begin, end = v->begin + v->count;
    int nch = 0;
    int64_t cb[8], cc[8];
    for (int c = 0; c < 8; c++) {
        b[c] = p;
        while (p < end && digit_at(t, p, v->level) == c) p++;
        if (p > b[c]) { cb[nch] = b[c]; cc[nch] = p - b[c]; nch++; }
    }
    int64_t first = node_alloc(t, nch);
    v = &t->node[vi];                     /* realloc may have moved it */
    v->leaf = 0;
    v->nchild = nch;
    v->first_child = first;
    int lev = v->level + 1;
    for (int k = 0; k < nch; k++) {
        orc_node *c = &t->node[first + k];
        memset(c, 0, sizeof(*c));
        c->begin = cb[k];
        c->count = cc[k];
        c->level = lev;
    }
    for (int k = 0; k < nch; k++) build_node(t, first + k);
}

/* Groups (this project's reading of "group-wise walk"): going down from the
 * root, a node with at most n_group particles, or a leaf, is one group;
 * otherwise its children are taken in key order and each child with more
 * than n_group particles is handled recursively (a leaf that large is a
 * group of its own).  The smaller children of a node with at most
 * 8 n_group particles form runs of consecutive children, each cut in key
 * order into groups of exactly n_group particles (the last one of a run
 * smaller); those of a larger node are packed whole and greedily into
 * groups of at most n_group (cutting there could join sparse children of a
 * wide node into one group whose box reaches far).  A group's box is the
 * tight box of its particles' grid cells. */
static void group_emit(orc_tree *t, int64_t begin, int64_t count,
                       const uint32_t *qmin, const uint32_t *qmax, double smax)
{
    if (t->ngroups == t->gcap) {
        t->gcap = t->gcap * 2 + 16;
        t->group = (orc_group *)realloc(t->group, (size_t)t->gcap * sizeof(orc_group));
    }
    orc_group *g = &t->group[t->ngroups++];
    g->begin = begin;
    g->count = count;
    for (int d = 0; d < 3; d++) { g->qmin[d] = qmin[d]; g->qmax[d] = qmax[d]; }
    g->smax = smax;
}

/* one group over sorted particles [b, b + c): box and largest radius scale
 * straight from the particles */
static void group_of_range(orc_tree *t, int64_t b, int64_t c)
{
    uint32_t mn[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, mx[3] = {0, 0, 0};
    double sm = 0.0;
    for (int64_t i = b; i < b + c; i++) {
        for (int d = 0; d < 3; d++) {
            uint32_t q = t->sq[3 * i + d];
            if (q < mn[d]) mn[d] = q;
            if (q > mx[d]) mx[d] = q;
        }
        if (t->sscale[i] > sm) sm = t->sscale[i];
    }
    group_emit(t, b, c, mn, mx, sm);
}

/* a run of consecutive small children, [b, b + c): cut into n_group pieces */
static void group_run(orc_tree *t, int64_t b, int64_t c)
{
    for (int64_t o = 0; o < c; o += t->n_group)
        group_of_range(t, b + o, c - o < t->n_group ? c - o : t->n_group);
}

static void build_groups(orc_tree *t, int64_t vi)
{
    const orc_node *v = &t->node[vi];
    if (v->count <= t->n_group || v->leaf) {
        group_emit(t, v->begin, v->count, v->qmin, v->qmax, v->smax);
        return;
    }
    const int cut = v->count <= 8 * (int64_t)t->n_group;   /* cut runs, else pack children */
    int64_t rb = 0, rc = 0;                 /* the current run (or pack) of small children */
    for (int k = 0; k < v->nchild; k++) {
        const orc_node *c = &t->node[v->first_child + k];
        if (c->count > t->n_group) {
            if (rc) { if (cut) group_run(t, rb, rc); else group_of_range(t, rb, rc); }
            rc = 0;
            build_groups(t, v->first_child + k);
            continue;
        }
        if (!cut && rc && rc + c->count > t->n_group) {
            group_of_range(t, rb, rc);
            rc = 0;
        }
        if (rc == 0) rb = c->begin;
        rc += c->count;
    }
    if (rc) { if (cut) group_run(t, rb, rc); else group_of_range(t, rb, rc); }
}

static int cmp_group_begin(const void *a, const void *b)
{
    int64_t x = ((const orc_group *)a)->begin, y = ((const orc_group *)b)->begin;
    return x < y ? -1 : (x > y ? 1 : 0);
}

orc_tree *orc_tree_build(int64_t n, const double *pos, const double *mass,
                         int n_leaf, int n_group, const double *scale)
{
    orc_tree *t = (orc_tree *)calloc(1, sizeof(orc_tree));
    t->n = n;
    t->n_leaf = n_leaf;
    t->n_group = n_group;
    t->key = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    t->q = (uint32_t *)malloc((size_t)n * 3 * sizeof(uint32_t));
    t->perm = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    t->spos = (double *)malloc((size_t)n * 3 * sizeof(double));
    t->smass = (double *)malloc((size_t)n * sizeof(double));
    t->sscale = (double *)malloc((size_t)n * sizeof(double));
    t->sq = (uint32_t *)malloc((size_t)n * 3 * sizeof(uint32_t));
    t->skey = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    compute_keys(t, pos);
    for (int64_t i = 0; i < n; i++) t->perm[i] = i;
    g_sort_keys = t->key;
    qsort(t->perm, (size_t)n, sizeof(int64_t), cmp_key_then_index);
    for (int64_t s = 0; s < n; s++) {
        int64_t i = t->perm[s];
        for (int d = 0; d < 3; d++) {
            t->spos[3 * s + d] = pos[3 * i + d];
            t->sq[3 * s + d] = t->q[3 * i + d];
        }
        t->smass[s] = mass[i];
        t->sscale[s] = scale ? scale[i] : 1.0;
        t->skey[s] = t->key[i];
    }
    int64_t root = node_alloc(t, 1);
    memset(&t->node[root], 0, sizeof(orc_node));
    t->node[root].begin = 0;
    t->node[root].count = n;
    t->node[root].level = 0;
    build_node(t, root);
    build_groups(t, root);
    /* depth-first emission is already in key order; sorting makes it explicit */
    qsort(t->group, (size_t)t->ngroups, sizeof(orc_group), cmp_group_begin);
    return t;
}

void orc_tree_free(orc_tree *t)
{
    if (!t) return;
    free(t->key); free(t->q); free(t->perm); free(t->spos); free(t->smass); free(t->sscale);
    free(t->sq); free(t->skey); free(t->node); free(t->group);
    free(t);
}

/* info[0] = n, info[1] = nodes, info[2] = groups, info[3] = max level;
 * box[0..2] = origin, box[3] = S, box[4] = scale. */
void orc_tree_info(const orc_tree *t, int64_t *info, double *box)
{
    int maxl = 0;
    for (int64_t v = 0; v < t->nnodes; v++)
        if (t->node[v].level > maxl) maxl = t->node[v].level;
    info[0] = t->n; info[1] = t->nnodes; info[2] = t->ngroups; info[3] = maxl;
    for (int d = 0; d < 3; d++) box[d] = t->origin[d];
    box[3] = t->S; box[4] = t->scale;
}

void orc_tree_keys(const orc_tree *t, uint64_t *key, uint32_t *q, int64_t *perm)
{
    memcpy(key, t->key, (size_t)t->n * sizeof(uint64_t));
    memcpy(q, t->q, (size_t)t->n * 3 * sizeof(uint32_t));
    memcpy(perm, t->perm, (size_t)t->n * sizeof(int64_t));
}

/* Node table: ints[v*8 + {0..7}] = begin, count, level, leaf, first_child,
 * nchild, -, -; q[v*6 + ...] = qmin xyz, qmax xyz; mom[v*10 + ...] = M,
 * com xyz, Q xx yy zz xy xz yz. */
void orc_tree_nodes(const orc_tree *t, int64_t *ints, uint32_t *q, double *mom)
{
    for (int64_t v = 0; v < t->nnodes; v++) {
        const orc_node *c = &t->node[v];
        int64_t *o = ints + 8 * v;
        o[0] = c->begin; o[1] = c->count; o[2] = c->level; o[3] = c->leaf;
        o[4] = c->first_child; o[5] = c->nchild; o[6] = 0; o[7] = 0;
        for (int d = 0; d < 3; d++) { q[6 * v + d] = c->qmin[d]; q[6 * v + 3 + d] = c->qmax[d]; }
        mom[10 * v] = c->M;
        for (int d = 0; d < 3; d++) mom[10 * v + 1 + d] = c->com[d];
        for (int k = 0; k < 6; k++) mom[10 * v + 4 + k] = c->Q[k];
    }
}

/* groups: g[k*8 + {0..7}] = begin, count, qmin xyz, qmax xyz. */
void orc_tree_groups(const orc_tree *t, int64_t *g)
{
    for (int64_t k = 0; k < t->ngroups; k++) {
        const orc_group *p = &t->group[k];
        int64_t *o = g + 8 * k;
        o[0] = p->begin; o[1] = p->count;
        for (int d = 0; d < 3; d++) { o[2 + d] = p->qmin[d]; o[5 + d] = p->qmax[d]; }
    }
}

/* ------------------------------------------------------------------------ */
/* Group-wise walk.  A cell C is used as a super-particle for group G when   */
/* both hold:                                                               */
/*   (opening angle, Sec. 4 and Sec. 5.1) s^2 < theta^2 d^2, with s the side */
/*   of C's geometric cube and d the distance from G's box to the cube's    */
/*   centre, both in units of half a grid cell (so exact integers), and the */
/*   product theta^2 d^2 formed in float64;                                  */
/*   (changeover, Sec. 5.1, Eq. 11) every particle of C is at least r_out    */
/*   from every particle of G, tested conservatively on grid cells: the     */
/*   squared gap between the two boxes, in whole cells, is at least         */
/*   floor((r_out * scale)^2) + 2.                                           */
/* Otherwise a leaf's particles go to the particle-particle (PP) list and   */
/* an internal cell is opened.  Children are visited in key order.         */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t *cells, ncells, ccap;
    int64_t *pp, npp, pcap;
} walk_out;

/* Gap threshold for radius scale s: floor(((r_out s) scale)^2) + 2 whole
 * grid cells squared.  The pair radius is the larger of the two scales, and
 * the threshold grows with s, so a cell is tested against the larger of the
 * group's and the cell's thresholds. */
static int64_t rout_threshold(const orc_tree *t, double r_out, double s)
{
    double R = (r_out * s) * t->scale;
    double R2 = R * R;
    if (R2 > 4.0e18) return (int64_t)4000000000000000000LL;  /* no gap that large */
    return (int64_t)floor(R2) + 2;
}

static int accept_cell(const orc_tree *t, const orc_group *G, const orc_node *C, double theta2,
                       double r_out)
{
    int sh = ORC_BITS - C->level;
    int64_t d2 = 0, gap2 = 0;
    for (int d = 0; d < 3; d++) {
        int64_t p = (int64_t)(C->qmin[d] >> sh);
        int64_t c2 = (2 * p + 1) << sh;                 /* centre, half cells */
        int64_t lo = 2 * (int64_t)G->qmin[d], hi = 2 * ((int64_t)G->qmax[d] + 1);
        int64_t dd = 0;
        if (lo - c2 > dd) dd = lo - c2;
        if (c2 - hi > dd) dd = c2 - hi;
        d2 += dd * dd;
        int64_t g = 0;
        int64_t g1 = (int64_t)C->qmin[d] - (int64_t)G->qmax[d] - 1;
        int64_t g2 = (int64_t)G->qmin[d] - (int64_t)C->qmax[d] - 1;
        if (g1 > g) g = g1;
        if (g2 > g) g = g2;
        gap2 += g * g;
    }
    double s = (double)((int64_t)1 << (ORC_BITS + 1 - C->level));  /* side, half cells */
    if (!(s * s < theta2 * (double)d2)) return 0;
    int64_t tg = rout_threshold(t, r_out, G->smax), tc = rout_threshold(t, r_out, C->smax);
    return gap2 >= (tg > tc ? tg : tc);
}

static void walk_visit(const orc_tree *t, const orc_group *G, int64_t vi,
                       double theta2, double r_out, walk_out *w)
{
    const orc_node *C = &t->node[vi];
    if (accept_cell(t, G, C, theta2, r_out)) {
        if (w->cells && w->ncells < w->ccap) w->cells[w->ncells] = vi;
        w->ncells++;
        return;
    }
    if (C->leaf) {
        for (int64_t p = C->begin; p < C->begin + C->count; p++) {
            if (w->pp && w->npp < w->pcap) w->pp[w->npp] = p;
            w->npp++;
        }
        return;
    }
    for (int k = 0; k < C->nchild; k++)
        walk_visit(t, G, C->first_child + k, theta2, r_out, w);
}

/* Lists of group g: cells (node indices) and PP (sorted particle indices).
 * Returns 0, or 1 if a capacity was too small (counts are still complete). */
int orc_tree_walk(const orc_tree *t, int64_t g, double theta, double r_out,
                  int64_t *cells, int64_t ccap, int64_t *pp, int64_t pcap,
                  int64_t *ncells, int64_t *npp)
{
    walk_out w = {cells, 0, ccap, pp, 0, pcap};
    walk_visit(t, &t->group[g], 0, theta * theta, r_out, &w);
    *ncells = w.ncells;
    *npp = w.npp;
    return (w.ncells > ccap || w.npp > pcap) ? 1 : 0;
}

/* Newtonian pull of a cell on point xi, monopole plus (order 2) quadrupole
 * about the centre of mass, without G; with d = xi - com, r = |d|:
 *   phi = -M/r - d.Q.d / (2 r^5)
 *   a   = -M d/r^3 + Q d / r^5 - (5/2) (d.Q.d) d / r^7. */
static void cell_pull(const orc_node *C, const double *xi, int order, double *acc, double *pot)
{
    double d[3] = {xi[0] - C->com[0], xi[1] - C->com[1], xi[2] - C->com[2]};
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double r = sqrt(r2);
    double r3 = r2 * r;
    for (int k = 0; k < 3; k++) acc[k] += -C->M * d[k] / r3;
    *pot += -C->M / r;
    if (order >= 2) {
        const double *Q = C->Q;     /* xx yy zz xy xz yz */
        double Qd[3] = {Q[0] * d[0] + Q[3] * d[1] + Q[4] * d[2],
                        Q[3] * d[0] + Q[1] * d[1] + Q[5] * d[2],
                        Q[4] * d[0] + Q[5] * d[1] + Q[2] * d[2]};
        double dQd = d[0] * Qd[0] + d[1] * Qd[1] + d[2] * Qd[2];
        double r5 = r3 * r2, r7 = r5 * r2;
        for (int k = 0; k < 3; k++) acc[k] += Qd[k] / r5 - 2.5 * dQd * d[k] / r7;
        *pot += -dQd / (2.0 * r5);
    }
}

/* Exposed for the cell pins (truncation orders, Legendre closed form,
 * -grad phi): pull of node v on point xi. */
void orc_cell_pull(const orc_tree *t, int64_t v, const double *xi, int order,
                   double *acc, double *pot)
{
    acc[0] = acc[1] = acc[2] = 0.0;
    *pot = 0.0;
    cell_pull(&t->node[v], xi, order, acc, pot);
}

/* Tree force on sorted particle s of group g, given g's lists. */
static void tree_force_one(const orc_tree *t, int64_t s, const walk_out *w,
                           double r_in, double r_out, double G, int order,
                           double *acc, double *pot)
{
    double a[3] = {0.0, 0.0, 0.0}, p = 0.0;
    const double *xi = t->spos + 3 * s;
    for (int64_t k = 0; k < w->ncells; k++)
        cell_pull(&t->node[w->cells[k]], xi, order, a, &p);
    for (int64_t k = 0; k < w->npp; k++) {
        int64_t j = w->pp[k];
        if (j == s) continue;
        double sij = t->sscale[s] > t->sscale[j] ? t->sscale[s] : t->sscale[j];
        pair_longrange(xi, t->spos + 3 * j, t->smass[j], sij * r_in, sij * r_out, a, &p);
    }
    for (int k = 0; k < 3; k++) acc[k] = G * a[k];
    *pot = G * p;
}

static int64_t group_of(const orc_tree *t, int64_t s)
{
    int64_t lo = 0, hi = t->ngroups - 1;
    while (lo < hi) {   /* last group with begin <= s (groups sorted by begin) */
        int64_t mid = (lo + hi + 1) / 2;
        if (t->group[mid].begin <= s) lo = mid; else hi = mid - 1;
    }
    return lo;
}


static void walk_alloc(const orc_tree *t, int64_t g, double theta, double r_out, walk_out *w)
{
    walk_out c = {NULL, 0, 0, NULL, 0, 0};
    walk_visit(t, &t->group[g], 0, theta * theta, r_out, &c);
    w->ccap = c.ncells; w->pcap = c.npp;
    w->cells = (int64_t *)malloc((size_t)(c.ncells + 1) * sizeof(int64_t));
    w->pp = (int64_t *)malloc((size_t)(c.npp + 1) * sizeof(int64_t));
    w->ncells = 0; w->npp = 0;
    walk_visit(t, &t->group[g], 0, theta * theta, r_out, w);
}

/* Tree force.  With targets == NULL every particle is computed (one walk per
 * group) and results are written per ORIGINAL index; otherwise target t is
 * original index targets[t] and results go to slot t.  stats (optional):
 * [0] cell interactions, [1] PP interactions (list entries times targets). */
void orc_tree_force(orc_tree *t, double theta, double r_in, double r_out, double G,
                    int order, int64_t nt, const int64_t *targets,
                    double *acc, double *pot, int64_t *stats)
{
    int64_t ci = 0, pi = 0;
    if (!targets) {
        int64_t *inv = (int64_t *)malloc((size_t)t->n * sizeof(int64_t));
        for (int64_t s = 0; s < t->n; s++) inv[s] = t->perm[s];
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : ci, pi)
        for (int64_t g = 0; g < t->ngroups; g++) {
            walk_out w;
            walk_alloc(t, g, theta, r_out, &w);
            const orc_group *grp = &t->group[g];
            for (int64_t s = grp->begin; s < grp->begin + grp->count; s++) {
                int64_t i = inv[s];
                tree_force_one(t, s, &w, r_in, r_out, G, order, acc + 3 * i, pot + i);
            }
            ci += w.ncells * grp->count;
            pi += w.npp * grp->count;
            free(w.cells); free(w.pp);
        }
        free(inv);
    } else {
        int64_t *slot = (int64_t *)malloc((size_t)t->n * sizeof(int64_t));
        for (int64_t s = 0; s < t->n; s++) slot[t->perm[s]] = s;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : ci, pi)
        for (int64_t k = 0; k < nt; k++) {
            int64_t s = slot[targets[k]];
            int64_t g = group_of(t, s);
            walk_out w;
            walk_alloc(t, g, theta, r_out, &w);
            tree_force_one(t, s, &w, r_in, r_out, G, order, acc + 3 * k, pot + k);
            ci += w.ncells;
            pi += w.npp;
            free(w.cells); free(w.pp);
        }
        free(slot);
    }
    if (stats) { stats[0] = ci; stats[1] = pi; }
}

/* ------------------------------------------------------------------------ */
/* Orbit-dependent neighbour criterion, Sec. 6.3.1, Eq. 24                   */
/*                                                                          */
/* Stage 1 (candidates): particle i searches within                         */
/*     r_nb,i = r_out,i + C_r |v_i| dt_L        (Eq. 24; r_out,i = s_i r_out) */
/* and j != i is a candidate of i when r_ij < r_nb,ij = max(r_nb,i, r_nb,j)  */
/* (the larger radius, as for the pair radii of Eq. 12, so the relation is   */
/* symmetric).  Stage 2 keeps candidate j when the pericentre distance of    */
/* the two-body Kepler orbit of (i, j) is below C_v R_ij.  As printed,       */
/* R_ij = r_nb,i; but a pericentre is never larger than the current         */
/* separation, so with C_v >= 1 that test keeps every candidate.  The        */
/* reading used by default is R_ij = r_out,ij = max(r_out,i, r_out,j): a     */
/* candidate is kept if its orbit brings it (within the safety factor C_v)  */
/* into the changeover region; mode 1 applies the printed R_ij = r_nb,ij.   */
/* Every operation below is a single IEEE operation in the order written    */
/* (no contraction), so each decision is reproducible bit for bit.          */
/* ------------------------------------------------------------------------ */

/* Pericentre of the relative Kepler orbit with separation dx, relative
 * velocity dv and mu = G (m_i + m_j): with h = |dx x dv| and the
 * eccentricity vector mu e = (v^2 - mu/r) dx - (dx . dv) dv, the pericentre
 * is r_p = (h^2 / mu) / (1 + |e|).  (The eccentricity vector is used rather
 * than e^2 = 1 + 2 E h^2 / mu^2, which cancels to half the digits for nearly
 * circular orbits.)  Limits: dv = 0 gives r; mu = 0 (straight-line motion)
 * gives the impact parameter h / |dv|; h = 0 with motion gives 0. */
double orc_pericentre(const double *dx, const double *dv, double mu)
{
    double r2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
    double v2 = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2];
    if (v2 == 0.0) return sqrt(r2);
    double cx = dx[1] * dv[2] - dx[2] * dv[1];
    double cy = dx[2] * dv[0] - dx[0] * dv[2];
    double cz = dx[0] * dv[1] - dx[1] * dv[0];
    double h2 = cx * cx + cy * cy + cz * cz;
    if (mu == 0.0) return sqrt(h2 / v2);
    double r = sqrt(r2);
    double a = v2 - mu / r;
    double b = dx[0] * dv[0] + dx[1] * dv[1] + dx[2] * dv[2];
    double ex = a * dx[0] - b * dv[0];
    double ey = a * dx[1] - b * dv[1];
    double ez = a * dx[2] - b * dv[2];
    double e = sqrt(ex * ex + ey * ey + ez * ez) / mu;
    return (h2 / mu) / (1.0 + e);
}

/* Eq. 24 for every particle: r_nb[i] = s_i r_out + C_r (|v_i| dt). */
void orc_rnb(int64_t n, const double *vel, const double *scale, double r_out, double dt,
             double C_r, double *rnb)
{
    for (int64_t i = 0; i < n; i++) {
        const double *v = vel + 3 * i;
        double sp = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        double ro = r_out * (scale ? scale[i] : 1.0);
        rnb[i] = ro + C_r * (sp * dt);
    }
}

/* 0: not a candidate, 1: candidate dropped by stage 2, 2: neighbour. */
static int orbit_pair(const double *pos, const double *vel, const double *mass,
                      const double *scale, const double *rnb, double r_out, double G,
                      double C_v, int mode, int64_t i, int64_t j)
{
    double dx[3] = {pos[3 * j] - pos[3 * i], pos[3 * j + 1] - pos[3 * i + 1],
                    pos[3 * j + 2] - pos[3 * i + 2]};
    double r2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
    double R = rnb[i] > rnb[j] ? rnb[i] : rnb[j];
    if (!(r2 < R * R)) return 0;
    if (mode == 2) return 2;
    double dv[3] = {vel[3 * j] - vel[3 * i], vel[3 * j + 1] - vel[3 * i + 1],
                    vel[3 * j + 2] - vel[3 * i + 2]};
    double rp = orc_pericentre(dx, dv, G * (mass[i] + mass[j]));
    double Rs = mode == 1 ? R : r_out * pair_scale(scale, i, j);
    return rp < C_v * Rs ? 2 : 1;
}

/* counts[t] (neighbours of target t after the chosen stage) and the number
 * of stage-1 candidates in ncand[t]. */
void orc_orbit_count(int64_t n, const double *pos, const double *vel, const double *mass,
                     const double *scale, const double *rnb, double r_out, double G, double C_v,
                     int mode, int64_t nt, const int64_t *targets, int64_t *counts, int64_t *ncand)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; t++) {
        int64_t i = targets ? targets[t] : t, c = 0, k = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            int s = orbit_pair(pos, vel, mass, scale, rnb, r_out, G, C_v, mode, i, j);
            k += s > 0;
            c += s == 2;
        }
        counts[t] = c;
        if (ncand) ncand[t] = k;
    }
}

/* Fill idx[offsets[t] ..] with the neighbours of target t, ascending. */
void orc_orbit_fill(int64_t n, const double *pos, const double *vel, const double *mass,
                    const double *scale, const double *rnb, double r_out, double G, double C_v,
                    int mode, int64_t nt, const int64_t *targets, const int64_t *offsets,
                    int32_t *idx)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; t++) {
        int64_t i = targets ? targets[t] : t, c = offsets[t];
        for (int64_t j = 0; j < n; j++)
            if (j != i && orbit_pair(pos, vel, mass, scale, rnb, r_out, G, C_v, mode, i, j) == 2)
                idx[c++] = (int32_t)j;
    }
}

int orc_abi_version(void) { return 1; }
