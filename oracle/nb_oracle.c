/*
 * nb_oracle.c - FP64 CPU oracle for the short-range non-bonded evaluation of
 * ACEMD (Harvey, Giupponi & De Fabritiis 2009, section "Molecular dynamics on
 * the GPU"): Lennard-Jones 12-6 with a switching function, real-space Ewald
 * Coulomb (erfc) under a cutoff, minimum-image orthorhombic periodic box,
 * excluded pairs and scaled 1-4 pairs, the cell binning that drives it, and
 * the adjoint used for force-field fitting.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle.so, which
 * only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * load.  It shares no code, header or table with the CUDA library.
 *
 * The paper states no force-field formulas; the functional forms below are the
 * readings recorded in the design notes:
 *   U_LJ(r)  = A/r^12 - B/r^6, A = 4 eps sig^12, B = 4 eps sig^6,
 *              Lorentz-Berthelot: sig_ab = (sig_a + sig_b)/2, eps_ab = sqrt(eps_a eps_b)
 *              (CHARMM force field, section "Molecular dynamics on the GPU").
 *   S(r)     = 1 (r <= rs); (rc^2-r^2)^2 (rc^2+2r^2-3rs^2)/(rc^2-rs^2)^3 (rs < r < rc)
 *              CHARMM energy switch on LJ only ("switched at 7.5 A", section
 *              "Performance").
 *   U_C(r)   = ke qi qj erfc(alpha r)/r, truncated at rc; alpha = 0 gives ke qi qj / r.
 *   weights  : excluded (1-2, 1-3) pairs contribute nothing; 1-4 pairs are
 *              scaled by s14_lj (LJ) and s14_c (Coulomb) (section "Molecular
 *              dynamics on the GPU", exclusion bitmaps).
 *   in(i,j)  : r2_f32 < rc_f32*rc_f32 with r2_f32 computed in FP32 from the
 *              FP32 coordinates, per axis s = xj - xi; s > L/2 -> d = (xj-L)-xi;
 *              s < -L/2 -> d = xj-(xi-L); else d = s; r2 = fma(dz,dz,fma(dy,dy,dx*dx)).
 *   binning  : 2-D columns (x, y), atoms z-sorted inside a column, columns padded
 *              to whole clusters of CLUSTER atoms (cell list of section
 *              "Molecular dynamics on the GPU", one particle per thread).
 * All values are FP64 over the exactly up-cast FP32 inputs.  Compile with
 * -ffp-contract=off so that the FP32 predicates round exactly as written.
 *
 * Parity unpinned: orc_binning, a specification of the sorted data layout
 * (no result depends on it; the pair set it induces is pinned by brute
 * force), and the conventions above that the paper does not fix (switch
 * form, ke, the 1-4/exclusion weights under Ewald, the combination rule).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_CLUSTER 8

/* ------------------------------------------------------------------ */
/* FP32 predicates (the decision side of the method, taken in FP32).   */
/* ------------------------------------------------------------------ */

/* Wrap one FP32 coordinate into [0, L) with FP32 IEEE operations. */
static float wrap1(float x, float L)
{
    if (x >= 0.0f && x < L) return x;
    float k = floorf(x / L);
    x = fmaf(-k, L, x);
    if (x < 0.0f) x = x + L;
    if (x >= L) x = x - L;
    return x;
}

void orc_wrap_f32(int64_t n, float *pos, const float *box)
{
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) pos[3 * i + a] = wrap1(pos[3 * i + a], box[a]);
}

/* Minimum-image FP32 displacement d = x_j - x_i (exact-shift form) and its
 * squared length.  img[a] is the integer image offset of j along axis a
 * (d_a = x_j + img*L - x_i). */
static float min_image_f32(const float *xi, const float *xj, const float *box, int *img, float *d)
{
    for (int a = 0; a < 3; ++a) {
        float L = box[a], h = 0.5f * L;
        float s = xj[a] - xi[a];
        if (s > h) { d[a] = (xj[a] - L) - xi[a]; img[a] = -1; }
        else if (s < -h) { d[a] = xj[a] - (xi[a] - L); img[a] = 1; }
        else { d[a] = s; img[a] = 0; }
    }
    return fmaf(d[2], d[2], fmaf(d[1], d[1], d[0] * d[0]));
}

/* ------------------------------------------------------------------ */
/* Topology lookup: per-atom partner lists (excluded = 1, scaled 1-4 = 2). */
/* ------------------------------------------------------------------ */
typedef struct { int64_t n; int64_t *start; int32_t *partner; int8_t *kind; } topo_t;

static void topo_build(topo_t *t, int64_t n, int64_t nex, const int32_t *ex, int64_t n14, const int32_t *p14)
{
    t->n = n;
    t->start = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t k = 0; k < nex; ++k) { t->start[ex[2 * k] + 1]++; t->start[ex[2 * k + 1] + 1]++; }
    for (int64_t k = 0; k < n14; ++k) { t->start[p14[2 * k] + 1]++; t->start[p14[2 * k + 1] + 1]++; }
    for (int64_t i = 0; i < n; ++i) t->start[i + 1] += t->start[i];
    int64_t m = t->start[n];
    t->partner = (int32_t *)malloc((size_t)(m ? m : 1) * sizeof(int32_t));
    t->kind = (int8_t *)malloc((size_t)(m ? m : 1));
    int64_t *fill = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) fill[i] = t->start[i];
    for (int64_t k = 0; k < nex; ++k) {
        int32_t a = ex[2 * k], b = ex[2 * k + 1];
        t->partner[fill[a]] = b; t->kind[fill[a]++] = 1;
        t->partner[fill[b]] = a; t->kind[fill[b]++] = 1;
    }
    for (int64_t k = 0; k < n14; ++k) {
        int32_t a = p14[2 * k], b = p14[2 * k + 1];
        t->partner[fill[a]] = b; t->kind[fill[a]++] = 2;
        t->partner[fill[b]] = a; t->kind[fill[b]++] = 2;
    }
    free(fill);
}

static int topo_kind(const topo_t *t, int64_t i, int64_t j)
{
    for (int64_t k = t->start[i]; k < t->start[i + 1]; ++k)
        if (t->partner[k] == j) return t->kind[k];
    return 0;
}

static void topo_free(topo_t *t) { free(t->start); free(t->partner); free(t->kind); }

/* ------------------------------------------------------------------ */
/* Parameters.                                                         */
/* ------------------------------------------------------------------ */
/* Tabulated radial functions (section "Molecular dynamics on the GPU": the
 * radial parts of the van der Waals and electrostatic terms linearly
 * interpolated from lookup tables; n = 4096 in the paper's error figure).
 * Six functions of r: E12 = S r^-12, E6 = S r^-6, Ec = erfc(alpha r)/r (1/r
 * for alpha = 0) and their -r d/dr: F12, F6, Fc.  Table point k sits at
 * r_k = k rc / n (k = 0..n), evaluated at max(r_k, TAB_RFLOOR); the table
 * holds, per interval k < n, the FP32 rounding of f(r_k) and of
 * f(r_{k+1}) - f(r_k).  A distance r uses interval k = min(floor(r n / rc),
 * n - 1), t = r n / rc - k and f = T_k + t D_k. */
#define TAB_RFLOOR 0.5
static int g_tab_n = 0; /* 0: direct evaluation (set by orc_set_table) */

typedef struct {
    int n;
    double inv_h;
    float *T, *D; /* [n][6] values and differences: E12, E6, Ec, F12, F6, Fc */
} tab_t;

typedef struct {
    float box[3];
    float rc_f, rc2_f;           /* FP32 cutoff and its FP32 square (membership) */
    double rc, rs, alpha, ke;    /* FP64 values of the FP32 parameters */
    double s14_lj, s14_c;
    int switched;
    int ntypes;
    const double *A, *B;         /* [T*T] A_ab = 4 eps sig^12, B_ab = 4 eps sig^6 */
    tab_t *tab;                  /* tabulated radial functions, or NULL */
} prm_t;

void orc_set_table(int n) { g_tab_n = n; }

static void prm_init(prm_t *p, const float *box, float rc, float rs, float alpha, float ke,
                     float s14_lj, float s14_c, int ntypes, const double *A, const double *B)
{
    for (int a = 0; a < 3; ++a) p->box[a] = box[a];
    p->rc_f = rc;
    p->rc2_f = rc * rc;
    p->rc = rc; p->rs = rs; p->alpha = alpha; p->ke = ke;
    p->s14_lj = s14_lj; p->s14_c = s14_c;
    p->switched = rs < rc;
    p->ntypes = ntypes; p->A = A; p->B = B;
    p->tab = NULL;
}

static void switch_fn(const prm_t *p, double r, double *S, double *S1, double *S2);

/* The six radial functions at r (see tab_t). */
static void radial_fns(const prm_t *p, double r, double f[6])
{
    double S, S1, S2;
    switch_fn(p, r, &S, &S1, &S2);
    double ir = 1.0 / r, ir6 = ir * ir * ir * ir * ir * ir, ir12 = ir6 * ir6;
    f[0] = S * ir12;
    f[1] = S * ir6;
    f[3] = 12.0 * S * ir12 - r * S1 * ir12;
    f[4] = 6.0 * S * ir6 - r * S1 * ir6;
    if (p->alpha > 0.0) {
        f[2] = erfc(p->alpha * r) * ir;
        f[5] = f[2] + 2.0 * p->alpha / sqrt(M_PI) * exp(-p->alpha * p->alpha * r * r);
    } else {
        f[2] = ir;
        f[5] = ir;
    }
}

static void tab_build(prm_t *p, int n)
{
    tab_t *t = (tab_t *)malloc(sizeof(tab_t));
    t->n = n;
    t->inv_h = (double)n / p->rc;
    t->T = (float *)malloc(sizeof(float) * 6 * (size_t)n);
    t->D = (float *)malloc(sizeof(float) * 6 * (size_t)n);
    double f0[6], f1[6];
    for (int k = 0; k < n; ++k) {
        double r0 = (double)k * p->rc / n, r1 = (double)(k + 1) * p->rc / n;
        radial_fns(p, r0 > TAB_RFLOOR ? r0 : TAB_RFLOOR, f0);
        radial_fns(p, r1 > TAB_RFLOOR ? r1 : TAB_RFLOOR, f1);
        for (int c = 0; c < 6; ++c) {
            t->T[6 * k + c] = (float)f0[c];
            t->D[6 * k + c] = (float)(f1[c] - f0[c]);
        }
    }
    p->tab = t;
}

static void prm_free(prm_t *p)
{
    if (!p->tab) return;
    free(p->tab->T);
    free(p->tab->D);
    free(p->tab);
    p->tab = NULL;
}

/* Lorentz-Berthelot combination on the type-pair table (CHARMM rule). */
void orc_combine_lb(int ntypes, const float *sigma, const float *eps, double *sig_tab, double *eps_tab,
                    double *A, double *B)
{
    for (int a = 0; a < ntypes; ++a)
        for (int b = 0; b < ntypes; ++b) {
            double s = 0.5 * ((double)sigma[a] + (double)sigma[b]);
            double e = sqrt((double)eps[a] * (double)eps[b]);
            sig_tab[a * ntypes + b] = s;
            eps_tab[a * ntypes + b] = e;
            double s6 = s * s * s * s * s * s;
            A[a * ntypes + b] = 4.0 * e * s6 * s6;
            B[a * ntypes + b] = 4.0 * e * s6;
        }
}

/* Pair terms at distance r for one weighted pair.
 * U: energy parts; du: dU/dr; d2u: d2U/dr2; dA, dB: dU/dA, dU/dB and their
 * r-derivatives; dqq: dU/d(qi qj) and its r-derivative. */
typedef struct {
    double e_lj, e_c, du, d2u;
    double uA, uA_r, uB, uB_r;
    double uqq, uqq_r;
} pterm_t;

static void switch_fn(const prm_t *p, double r, double *S, double *S1, double *S2)
{
    if (!p->switched || r <= p->rs) { *S = 1.0; *S1 = 0.0; *S2 = 0.0; return; }
    double rc2 = p->rc * p->rc, rs2 = p->rs * p->rs, r2 = r * r;
    double D = (rc2 - rs2) * (rc2 - rs2) * (rc2 - rs2);
    *S = (rc2 - r2) * (rc2 - r2) * (rc2 + 2.0 * r2 - 3.0 * rs2) / D;
    *S1 = 12.0 * r * (rc2 - r2) * (rs2 - r2) / D;
    *S2 = 12.0 * ((rc2 - r2) * (rs2 - r2) - 2.0 * r2 * (rs2 - r2) - 2.0 * r2 * (rc2 - r2)) / D;
}

static void pair_terms(const prm_t *p, double r, double A, double B, double qq, double wlj, double wc,
                       pterm_t *t)
{
    double ir = 1.0 / r, ir2 = ir * ir, ir6 = ir2 * ir2 * ir2;
    /* LJ pieces V = A r^-12 - B r^-6 and its derivatives. */
    double r12 = ir6 * ir6;
    double V = A * r12 - B * ir6;
    double V1 = -12.0 * A * r12 * ir + 6.0 * B * ir6 * ir;
    double V2 = 156.0 * A * r12 * ir2 - 42.0 * B * ir6 * ir2;
    double S, S1, S2;
    switch_fn(p, r, &S, &S1, &S2);
    t->e_lj = wlj * S * V;
    double dlj = wlj * (S1 * V + S * V1);
    double d2lj = wlj * (S2 * V + 2.0 * S1 * V1 + S * V2);
    t->uA = wlj * S * r12;
    t->uA_r = wlj * (S1 * r12 - 12.0 * S * r12 * ir);
    t->uB = -wlj * S * ir6;
    t->uB_r = -wlj * (S1 * ir6 - 6.0 * S * ir6 * ir);
    /* Coulomb phi(r) = erfc(alpha r)/r. */
    double phi, phi1, phi2;
    if (p->alpha > 0.0) {
        double ar = p->alpha * r;
        double ec = erfc(ar);
        double c = 2.0 * p->alpha / sqrt(M_PI);
        double g = exp(-ar * ar);
        phi = ec * ir;
        phi1 = -c * g * ir - ec * ir2;
        phi2 = 2.0 * p->alpha * p->alpha * c * g + 2.0 * c * g * ir2 + 2.0 * ec * ir2 * ir;
    } else {
        phi = ir; phi1 = -ir2; phi2 = 2.0 * ir2 * ir;
    }
    t->uqq = wc * p->ke * phi;
    t->uqq_r = wc * p->ke * phi1;
    t->e_c = qq * t->uqq;
    t->du = dlj + qq * t->uqq_r;
    t->d2u = d2lj + qq * wc * p->ke * phi2;
}

/* Weights from the topology kind; returns 0 for an excluded pair. */
static int pair_weights(const prm_t *p, int kind, double *wlj, double *wc)
{
    if (kind == 1) return 0;
    if (kind == 2) { *wlj = p->s14_lj; *wc = p->s14_c; }
    else { *wlj = 1.0; *wc = 1.0; }
    return 1;
}

/* ------------------------------------------------------------------ */
/* Forward: energy, forces, virial.                                    */
/* ------------------------------------------------------------------ */

/* Accumulate one in-range pair (i, j) with FP64 displacement d = x_j^img - x_i. */
static void accum_pair(const prm_t *p, const double *d, double r, double A, double B, double qq,
                       double wlj, double wc, double *Fi, double *Fj, double *E, double *W)
{
    pterm_t t;
    if (p->tab) {
        /* interpolated radial functions; du = dU/dr = -(-r dU/dr) / r */
        const tab_t *tb = p->tab;
        double x = r * tb->inv_h;
        int k = (int)floor(x);
        if (k > tb->n - 1) k = tb->n - 1;
        double u = x - (double)k, f[6];
        for (int c = 0; c < 6; ++c) f[c] = (double)tb->T[6 * k + c] + u * (double)tb->D[6 * k + c];
        t.e_lj = wlj * (A * f[0] - B * f[1]);
        t.e_c = qq * wc * p->ke * f[2];
        t.du = -(wlj * (A * f[3] - B * f[4]) + qq * wc * p->ke * f[5]) / r;
    } else {
        pair_terms(p, r, A, B, qq, wlj, wc, &t);
    }
    E[2] += fabs(t.e_lj); E[3] += fabs(t.e_c);
    E[4] += t.e_lj * t.e_lj; E[5] += t.e_c * t.e_c;
    double h = t.du / r; /* F_i = h d, F_j = -h d */
    for (int a = 0; a < 3; ++a) { Fi[a] += h * d[a]; if (Fj) Fj[a] -= h * d[a]; }
    E[0] += t.e_lj; E[1] += t.e_c;
    /* W_ab = sum d_ij,a f_ij,b with d_ij = x_i - x_j = -d and f_ij = h d. */
    W[0] -= h * d[0] * d[0]; W[1] -= h * d[1] * d[1]; W[2] -= h * d[2] * d[2];
    W[3] -= h * d[0] * d[1]; W[4] -= h * d[0] * d[2]; W[5] -= h * d[1] * d[2];
}

static void disp64(const float *xi, const float *xj, const float *box, const int *img, double *d, double *r)
{
    double s = 0.0;
    for (int a = 0; a < 3; ++a) {
        d[a] = ((double)xj[a] + (double)img[a] * (double)box[a]) - (double)xi[a];
        s += d[a] * d[a];
    }
    *r = sqrt(s);
}

/* Plain O(N^2) sum over unique pairs i < j.  F [n*3], E [6] (LJ, Coulomb,
 * then the sums of |pair energy| of each part: the scale against which the
 * rounding error of a summed energy is measured, then the sums of squared
 * pair energies: the scale of the random part of that error), W [6] (xx, yy,
 * zz, xy, xz, yz).  Returns the number of pairs in range. */
int64_t orc_forces_allpairs(int64_t n, const float *pos, const float *q, const int32_t *type,
                            int ntypes, const double *A, const double *B, const float *box,
                            float rc, float rs, float alpha, float ke, float s14_lj, float s14_c,
                            int64_t nex, const int32_t *ex, int64_t n14, const int32_t *p14,
                            double *F, double *E, double *W)
{
    prm_t p;
    prm_init(&p, box, rc, rs, alpha, ke, s14_lj, s14_c, ntypes, A, B);
    if (g_tab_n > 0) tab_build(&p, g_tab_n);
    topo_t t;
    topo_build(&t, n, nex, ex, n14, p14);
    memset(F, 0, sizeof(double) * 3 * (size_t)n);
    for (int a = 0; a < 6; ++a) E[a] = 0.0;
    for (int a = 0; a < 6; ++a) W[a] = 0.0;
    int64_t npairs = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            int img[3];
            float df[3];
            float r2 = min_image_f32(pos + 3 * i, pos + 3 * j, box, img, df);
            if (!(r2 < p.rc2_f)) continue;
            double wlj, wc;
            if (!pair_weights(&p, topo_kind(&t, i, j), &wlj, &wc)) continue;
            double d[3], r;
            disp64(pos + 3 * i, pos + 3 * j, box, img, d, &r);
            int ab = type[i] * ntypes + type[j];
            accum_pair(&p, d, r, A[ab], B[ab], (double)q[i] * (double)q[j], wlj, wc,
                       F + 3 * i, F + 3 * j, E, W);
            ++npairs;
        }
    prm_free(&p);
    topo_free(&t);
    return npairs;
}

/* ------------------------------------------------------------------ */
/* Cell-list traversal (the paper's cell-list scheme) for large systems. */
/* Cells of width >= rc; every atom visits the 27 surrounding cells and  */
/* keeps its own force and half of each pair energy.  Membership is the  */
/* same FP32 predicate, so the pair set equals the all-pairs one.       */
/* ------------------------------------------------------------------ */
typedef struct { int nc[3]; int64_t *start; int64_t *atom; } grid_t;

static int grid_build(grid_t *g, int64_t n, const float *pos, const float *box, double rc)
{
    for (int a = 0; a < 3; ++a) {
        g->nc[a] = (int)floor((double)box[a] / rc);
        if (g->nc[a] < 3) return 0;
    }
    int64_t ncell = (int64_t)g->nc[0] * g->nc[1] * g->nc[2];
    g->start = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    g->atom = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    int64_t *cell = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        int c[3];
        for (int a = 0; a < 3; ++a) {
            c[a] = (int)floor((double)pos[3 * i + a] * g->nc[a] / (double)box[a]);
            if (c[a] >= g->nc[a]) c[a] = g->nc[a] - 1;
            if (c[a] < 0) c[a] = 0;
        }
        cell[i] = ((int64_t)c[2] * g->nc[1] + c[1]) * g->nc[0] + c[0];
        g->start[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) g->start[c + 1] += g->start[c];
    int64_t *fill = (int64_t *)malloc((size_t)ncell * sizeof(int64_t));
    for (int64_t c = 0; c < ncell; ++c) fill[c] = g->start[c];
    for (int64_t i = 0; i < n; ++i) g->atom[fill[cell[i]]++] = i;
    free(fill);
    free(cell);
    return 1;
}

static void grid_free(grid_t *g) { free(g->start); free(g->atom); }

static int64_t grid_cell_of(const grid_t *g, const float *x, const float *box, int *c)
{
    for (int a = 0; a < 3; ++a) {
        c[a] = (int)floor((double)x[a] * g->nc[a] / (double)box[a]);
        if (c[a] >= g->nc[a]) c[a] = g->nc[a] - 1;
        if (c[a] < 0) c[a] = 0;
    }
    return ((int64_t)c[2] * g->nc[1] + c[1]) * g->nc[0] + c[0];
}

/* Per-atom accumulation for atom i over all its neighbours j != i (both
 * orders are visited across atoms, so each atom keeps half the pair energy). */
static int64_t atom_sum(const prm_t *p, const topo_t *t, const grid_t *g, int64_t n, const float *pos,
                        const float *q, const int32_t *type, int64_t i, double *Fi, double *Ei, double *Wi)
{
    int64_t cnt = 0;
    int c[3];
    Fi[0] = Fi[1] = Fi[2] = 0.0;
    for (int a = 0; a < 6; ++a) Ei[a] = 0.0;
    for (int a = 0; a < 6; ++a) Wi[a] = 0.0;
    if (g) grid_cell_of(g, pos + 3 * i, p->box, c);
    int64_t jlist_n = g ? 27 : 1;
    for (int64_t nb = 0; nb < jlist_n; ++nb) {
        int64_t jb, je;
        const int64_t *idx = NULL;
        if (g) {
            int cc[3] = {c[0] + (int)(nb % 3) - 1, c[1] + (int)((nb / 3) % 3) - 1, c[2] + (int)(nb / 9) - 1};
            for (int a = 0; a < 3; ++a) cc[a] = (cc[a] + g->nc[a]) % g->nc[a];
            int64_t cell = ((int64_t)cc[2] * g->nc[1] + cc[1]) * g->nc[0] + cc[0];
            jb = g->start[cell]; je = g->start[cell + 1]; idx = g->atom;
        } else { jb = 0; je = n; }
        for (int64_t k = jb; k < je; ++k) {
            int64_t j = idx ? idx[k] : k;
            if (j == i) continue;
            int img[3];
            float df[3];
            float r2 = min_image_f32(pos + 3 * i, pos + 3 * j, p->box, img, df);
            if (!(r2 < p->rc2_f)) continue;
            double wlj, wc;
            if (!pair_weights(p, topo_kind(t, i, j), &wlj, &wc)) continue;
            double d[3], r;
            disp64(pos + 3 * i, pos + 3 * j, p->box, img, d, &r);
            int ab = type[i] * p->ntypes + type[j];
            double e2[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, w6[6] = {0, 0, 0, 0, 0, 0};
            accum_pair(p, d, r, p->A[ab], p->B[ab], (double)q[i] * (double)q[j], wlj, wc, Fi, NULL, e2, w6);
            /* each pair is visited from both atoms: half of every sum here */
            for (int a = 0; a < 6; ++a) Ei[a] += 0.5 * e2[a];
            for (int a = 0; a < 6; ++a) Wi[a] += 0.5 * w6[a];
            ++cnt;
        }
    }
    return cnt;
}

/* Cell-list forward over all atoms (OpenMP over atoms; deterministic: per-atom
 * partials are summed in atom order).  Returns the number of unique pairs. */
int64_t orc_forces_cells(int64_t n, const float *pos, const float *q, const int32_t *type,
                         int ntypes, const double *A, const double *B, const float *box,
                         float rc, float rs, float alpha, float ke, float s14_lj, float s14_c,
                         int64_t nex, const int32_t *ex, int64_t n14, const int32_t *p14,
                         double *F, double *E, double *W)
{
    prm_t p;
    prm_init(&p, box, rc, rs, alpha, ke, s14_lj, s14_c, ntypes, A, B);
    if (g_tab_n > 0) tab_build(&p, g_tab_n);
    topo_t t;
    topo_build(&t, n, nex, ex, n14, p14);
    grid_t g;
    int have_grid = grid_build(&g, n, pos, box, (double)rc);
    double *Ep = (double *)malloc(sizeof(double) * 12 * (size_t)(n ? n : 1));
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i)
        cnt[i] = atom_sum(&p, &t, have_grid ? &g : NULL, n, pos, q, type, i, F + 3 * i, Ep + 12 * i, Ep + 12 * i + 6);
    for (int a = 0; a < 6; ++a) E[a] = 0.0;
    for (int a = 0; a < 6; ++a) W[a] = 0.0;
    int64_t tot = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int a = 0; a < 6; ++a) E[a] += Ep[12 * i + a];
        for (int a = 0; a < 6; ++a) W[a] += Ep[12 * i + 6 + a];
        tot += cnt[i];
    }
    free(Ep); free(cnt);
    if (have_grid) grid_free(&g);
    prm_free(&p);
    topo_free(&t);
    return tot / 2;
}

/* Forces on a subset of atoms only (plain loop over all j), for sampled checks
 * of systems too large for the full sum.  F [m*3]; E4 [m*6] half pair energies
 * (LJ, Coulomb, |LJ|, |Coulomb|, LJ^2, Coulomb^2). */
void orc_forces_subset(int64_t n, const float *pos, const float *q, const int32_t *type,
                       int ntypes, const double *A, const double *B, const float *box,
                       float rc, float rs, float alpha, float ke, float s14_lj, float s14_c,
                       int64_t nex, const int32_t *ex, int64_t n14, const int32_t *p14,
                       int64_t m, const int64_t *atoms, double *F, double *E4, int64_t *npair)
{
    prm_t p;
    prm_init(&p, box, rc, rs, alpha, ke, s14_lj, s14_c, ntypes, A, B);
    if (g_tab_n > 0) tab_build(&p, g_tab_n);
    topo_t t;
    topo_build(&t, n, nex, ex, n14, p14);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < m; ++k) {
        double W[6];
        npair[k] = atom_sum(&p, &t, NULL, n, pos, q, type, atoms[k], F + 3 * k, E4 + 6 * k, W);
    }
    prm_free(&p);
    topo_free(&t);
}

/* FP64 terms of m given pairs with unit weights (no exclusion or 1-4
 * scaling), for pair-by-pair comparison with the kernel's FP32 pair
 * arithmetic: d = x_j - x_i exactly as given (the caller applies the periodic
 * image), r = |d| in FP64.  out [m*4]: (E_LJ (switched), E_Coul, dU/dr,
 * A r^-12 + B r^-6, an LJ magnitude that vanishes neither where E_LJ changes
 * sign nor where the switch reaches zero).  Same pair_terms as the forward
 * sums. */
void orc_pair_terms(int64_t m, const float *xi, const float *xj, const float *qi, const float *qj,
                    const int32_t *ti, const int32_t *tj, int ntypes, const double *A, const double *B,
                    float rc, float rs, float alpha, float ke, double *out)
{
    prm_t p;
    const float box[3] = {0.0f, 0.0f, 0.0f};
    prm_init(&p, box, rc, rs, alpha, ke, 1.0f, 1.0f, ntypes, A, B);
    for (int64_t k = 0; k < m; ++k) {
        double r2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double d = (double)xj[3 * k + a] - (double)xi[3 * k + a];
            r2 += d * d;
        }
        const double r = sqrt(r2);
        const int ab = ti[k] * ntypes + tj[k];
        pterm_t t;
        pair_terms(&p, r, A[ab], B[ab], (double)qi[k] * (double)qj[k], 1.0, 1.0, &t);
        const double ir6 = 1.0 / (r2 * r2 * r2);
        out[4 * k] = t.e_lj;
        out[4 * k + 1] = t.e_c;
        out[4 * k + 2] = t.du;
        out[4 * k + 3] = A[ab] * ir6 * ir6 + B[ab] * ir6;
    }
    prm_free(&p);
}

/* Unique in-range, non-excluded pairs (i < j) written to ij [cap*2].
 * Returns the total count (which may exceed cap). */
int64_t orc_pairs(int64_t n, const float *pos, const float *box, float rc,
                  int64_t nex, const int32_t *ex, int64_t n14, const int32_t *p14,
                  int64_t cap, int32_t *ij)
{
    topo_t t;
    topo_build(&t, n, nex, ex, n14, p14);
    float rc2 = rc * rc;
    grid_t g;
    int have_grid = grid_build(&g, n, pos, box, (double)rc);
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; ++i) {
        int c[3];
        int64_t nbn = have_grid ? 27 : 1;
        if (have_grid) grid_cell_of(&g, pos + 3 * i, box, c);
        for (int64_t nb = 0; nb < nbn; ++nb) {
            int64_t jb = i + 1, je = n;
            const int64_t *idx = NULL;
            if (have_grid) {
                int cc[3] = {c[0] + (int)(nb % 3) - 1, c[1] + (int)((nb / 3) % 3) - 1, c[2] + (int)(nb / 9) - 1};
                for (int a = 0; a < 3; ++a) cc[a] = (cc[a] + g.nc[a]) % g.nc[a];
                int64_t cell = ((int64_t)cc[2] * g.nc[1] + cc[1]) * g.nc[0] + cc[0];
                jb = g.start[cell]; je = g.start[cell + 1]; idx = g.atom;
            }
            for (int64_t k = jb; k < je; ++k) {
                int64_t j = idx ? idx[k] : k;
                if (j <= i) continue;
                int img[3];
                float df[3];
                if (!(min_image_f32(pos + 3 * i, pos + 3 * j, box, img, df) < rc2)) continue;
                if (topo_kind(&t, i, j) == 1) continue;
                if (cnt < cap) { ij[2 * cnt] = (int32_t)i; ij[2 * cnt + 1] = (int32_t)j; }
                ++cnt;
            }
        }
    }
    if (have_grid) grid_free(&g);
    topo_free(&t);
    return cnt;
}

/* ------------------------------------------------------------------ */
/* Adjoint.  L = sum_i G_i . F_i + gE * (E_LJ + E_C).                  */
/* Outputs dL/dx [n*3] (the Hessian-vector product -H G plus -gE F),   */
/* dL/dq [n], dL/dA_ab and dL/dB_ab [T*T] (symmetric: each unordered    */
/* type pair's value is stored in both [a][b] and [b][a]) and, when     */
/* non-null, the sums of |pair contribution| of each table entry.      */
/* ------------------------------------------------------------------ */
int64_t orc_backward_allpairs(int64_t n, const float *pos, const float *q, const int32_t *type,
                              int ntypes, const double *A, const double *B, const float *box,
                              float rc, float rs, float alpha, float ke, float s14_lj, float s14_c,
                              int64_t nex, const int32_t *ex, int64_t n14, const int32_t *p14,
                              const double *G, double gE,
                              double *dx, double *dq, double *dA, double *dB, double *dAabs, double *dBabs)
{
    prm_t p;
    prm_init(&p, box, rc, rs, alpha, ke, s14_lj, s14_c, ntypes, A, B);
    topo_t t;
    topo_build(&t, n, nex, ex, n14, p14);
    memset(dx, 0, sizeof(double) * 3 * (size_t)n);
    memset(dq, 0, sizeof(double) * (size_t)n);
    memset(dA, 0, sizeof(double) * (size_t)ntypes * ntypes);
    memset(dB, 0, sizeof(double) * (size_t)ntypes * ntypes);
    if (dAabs) memset(dAabs, 0, sizeof(double) * (size_t)ntypes * ntypes);
    if (dBabs) memset(dBabs, 0, sizeof(double) * (size_t)ntypes * ntypes);
    int64_t npairs = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            int img[3];
            float df[3];
            float r2 = min_image_f32(pos + 3 * i, pos + 3 * j, box, img, df);
            if (!(r2 < p.rc2_f)) continue;
            double wlj, wc;
            if (!pair_weights(&p, topo_kind(&t, i, j), &wlj, &wc)) continue;
            double d[3], r;
            disp64(pos + 3 * i, pos + 3 * j, box, img, d, &r);
            int ab = type[i] * ntypes + type[j];
            double qi = q[i], qj = q[j];
            pterm_t pt;
            pair_terms(&p, r, A[ab], B[ab], qi * qj, wlj, wc, &pt);
            /* F_i = h d, F_j = -h d with h = U'/r; g = G_i - G_j. */
            double h = pt.du / r;
            double h1 = (pt.d2u * r - pt.du) / (r * r); /* dh/dr */
            double g[3], gd = 0.0;
            for (int a = 0; a < 3; ++a) { g[a] = G[3 * i + a] - G[3 * j + a]; gd += g[a] * d[a]; }
            for (int a = 0; a < 3; ++a) {
                double v = h * g[a] + (h1 / r) * gd * d[a] + gE * h * d[a];
                dx[3 * i + a] -= v;
                dx[3 * j + a] += v;
            }
            /* charges: U_C = qi qj uqq(r), h_C = qi qj uqq_r / r */
            dq[i] += qj * (pt.uqq_r / r * gd + gE * pt.uqq);
            dq[j] += qi * (pt.uqq_r / r * gd + gE * pt.uqq);
            double gA = pt.uA_r / r * gd + gE * pt.uA;
            double gB = pt.uB_r / r * gd + gE * pt.uB;
            int ba = type[j] * ntypes + type[i];
            dA[ab] += gA; dB[ab] += gB;
            if (ba != ab) { dA[ba] += gA; dB[ba] += gB; }
            /* summation scale of each table entry (sum of |contribution|) */
            if (dAabs) { dAabs[ab] += fabs(gA); if (ba != ab) dAabs[ba] += fabs(gA); }
            if (dBabs) { dBabs[ab] += fabs(gB); if (ba != ab) dBabs[ba] += fabs(gB); }
            ++npairs;
        }
    topo_free(&t);
    return npairs;
}

/* Chain rule from the symmetric (A, B) table gradient to the type-pair
 * (sigma_ab, eps_ab) table and then to per-type Lorentz-Berthelot
 * parameters.  dsig/deps [T] per type; the per-type eps derivative is
 * undefined (NaN) for a type with eps = 0 that pairs with a nonzero eps. */
void orc_lb_chain(int T, const double *sig_tab, const double *eps_tab, const double *dA, const double *dB,
                  const float *eps, double *dsig_tab, double *deps_tab, double *dsig, double *deps)
{
    for (int k = 0; k < T * T; ++k) {
        double s = sig_tab[k], e = eps_tab[k];
        double s5 = s * s * s * s * s, s6 = s5 * s, s11 = s6 * s5, s12 = s6 * s6;
        dsig_tab[k] = dA[k] * 48.0 * e * s11 + dB[k] * 24.0 * e * s5;
        deps_tab[k] = dA[k] * 4.0 * s12 + dB[k] * 4.0 * s6;
    }
    for (int t = 0; t < T; ++t) {
        double gs = 0.0, ge = 0.0;
        for (int b = 0; b < T; ++b) {
            int k = t * T + b;
            if (b == t) { gs += dsig_tab[k]; ge += deps_tab[k]; }
            else {
                gs += 0.5 * dsig_tab[k];
                /* d sqrt(eps_t eps_b)/d eps_t = eps_b / (2 sqrt(eps_t eps_b)) */
                if (eps[b] != 0.0f)
                    ge += deps_tab[k] * (double)eps[b] / (2.0 * sqrt((double)eps[t] * (double)eps[b]));
            }
        }
        dsig[t] = gs;
        deps[t] = (eps[t] == 0.0f) ? NAN : ge;
    }
}

/* ------------------------------------------------------------------ */
/* Binning reproduction: columns in x-y, z-sorted, padded to clusters.  */
/* ------------------------------------------------------------------ */

/* Column counts for one box: the largest n with n^3 * CLUSTER <= L^3 * rho,
 * so a column slab of one cluster is about cubic. */
static int col_count(double L, double rho)
{
    int n = 1;
    while (n < 4096 && (double)(n + 1) * (n + 1) * (n + 1) * ORC_CLUSTER <= L * L * L * rho) ++n;
    return n;
}

void orc_grid_dims(int64_t n, const float *box, int *nx, int *ny)
{
    double rho = (double)n / ((double)box[0] * (double)box[1] * (double)box[2]);
    *nx = col_count((double)box[0], rho);
    *ny = col_count((double)box[1], rho);
}

static const float *g_sort_z;
static int cmp_z_then_index(const void *pa, const void *pb)
{
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    float za = g_sort_z[3 * a + 2], zb = g_sort_z[3 * b + 2];
    if (za < zb) return -1;
    if (za > zb) return 1;
    return (a < b) ? -1 : (a > b);
}

/* Sorted slot order of one system (coordinates already wrapped).  perm has
 * room for n + (CLUSTER-1)*nx*ny slots; padding slots get -1.  col_start
 * [nx*ny+1] receives padded column offsets.  Returns the padded size.
 * This is a specification of the data layout (which slot each atom takes),
 * not a quantity the paper fixes: no result of the method depends on it, so
 * it has no pin of its own (parity unpinned as a layout); the tests compare
 * the GPU's sorted order with it slot by slot, and the pair set it induces
 * with brute-force enumeration. */
int64_t orc_binning(int64_t n, const float *pos, const float *box, int64_t *perm, int64_t *col_start)
{
    int nx, ny;
    orc_grid_dims(n, box, &nx, &ny);
    float ix = (float)((double)nx / (double)box[0]);
    float iy = (float)((double)ny / (double)box[1]);
    int64_t ncol = (int64_t)nx * ny;
    int64_t *cnt = (int64_t *)calloc((size_t)ncol, sizeof(int64_t));
    int64_t *col = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        float fx = pos[3 * i] * ix, fy = pos[3 * i + 1] * iy;
        int cx = (int)floorf(fx), cy = (int)floorf(fy);
        if (cx > nx - 1) cx = nx - 1;
        if (cx < 0) cx = 0;
        if (cy > ny - 1) cy = ny - 1;
        if (cy < 0) cy = 0;
        col[i] = (int64_t)cy * nx + cx;
        cnt[col[i]]++;
    }
    col_start[0] = 0;
    for (int64_t c = 0; c < ncol; ++c)
        col_start[c + 1] = col_start[c] + (cnt[c] + ORC_CLUSTER - 1) / ORC_CLUSTER * ORC_CLUSTER;
    int64_t npad = col_start[ncol];
    for (int64_t s = 0; s < npad; ++s) perm[s] = -1;
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncol);
    for (int64_t c = 0; c < ncol; ++c) fill[c] = col_start[c];
    for (int64_t i = 0; i < n; ++i) perm[fill[col[i]]++] = i; /* index order inside a column */
    g_sort_z = pos;
    for (int64_t c = 0; c < ncol; ++c)
        qsort(perm + col_start[c], (size_t)cnt[c], sizeof(int64_t), cmp_z_then_index);
    free(fill); free(col); free(cnt);
    return npad;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the OpenMP loops from now on (n >= 1); for timing only. */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
