// nb_host.cuh - host-side helpers shared by the context entry points and the
// allocation-free entry point: validation, column counts, type-pair tables,
// the erfcx fit and the pair / system constants.  None of them allocates.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>

#include "acenb.h"
#include "nb_internal.cuh"

namespace acenb {
namespace host {

constexpr double kDefaultKe = 332.0636;

// Number of x-y columns along one axis: the largest n with n^3 * 8 <= L^3 rho,
// so a one-cluster slab of a column is about cubic.  Evaluated in FP64 with a
// fixed operation order (the binning is part of the bit-exact cell contract).
inline int column_count(double L, double rho)
{
    int n = 1;
    while (n < 4096 && (double)(n + 1) * (n + 1) * (n + 1) * kCluster <= L * L * L * rho) ++n;
    return n;
}

// Weighted least squares min |W (A x - b)| by Householder QR, A m x n
// (row-major, n <= kErfcDeg + 1, m <= 96); A and b are overwritten.
inline void lsq_householder(int m, int n, double *A, double *b, double *x)
{
    for (int k = 0; k < n; ++k) {
        double nrm = 0.0;
        for (int i = k; i < m; ++i) nrm += A[i * n + k] * A[i * n + k];
        nrm = sqrt(nrm);
        const double alpha = A[k * n + k] > 0 ? -nrm : nrm;
        double v[96] = {0.0};
        for (int i = k; i < m; ++i) v[i] = A[i * n + k];
        v[k] -= alpha;
        double vn = 0.0;
        for (int i = k; i < m; ++i) vn += v[i] * v[i];
        if (vn == 0.0) continue;
        for (int j = k; j < n; ++j) {
            double s = 0.0;
            for (int i = k; i < m; ++i) s += v[i] * A[i * n + j];
            s = 2.0 * s / vn;
            for (int i = k; i < m; ++i) A[i * n + j] -= s * v[i];
        }
        double s = 0.0;
        for (int i = k; i < m; ++i) s += v[i] * b[i];
        s = 2.0 * s / vn;
        for (int i = k; i < m; ++i) b[i] -= s * v[i];
    }
    for (int k = n - 1; k >= 0; --k) {
        double s = b[k];
        for (int j = k + 1; j < n; ++j) s -= A[k * n + j] * x[j];
        x[k] = s / A[k * n + k];
    }
}

// Polynomial fit in relative error with the FP32 rounding of the
// coefficients taken into account: on m nodes with basis values
// T[i*n + k] = t_i^k and targets y_i, the constant coefficient is fitted
// (weights 1 / |y_i|), rounded to FP32 and fixed, the others refitted, and
// so on up to the highest.  A plain fit whose coefficients are rounded
// afterwards leaves a smooth error that changes sign across the interval (a
// bias of every summed pair energy that depends on the pair distance).
inline void fit_rounded_poly(int m, int n, const double *T, const double *y, float *coef)
{
    double fixed[16];
    for (int k = 0; k < n; ++k) {
        const int nf = n - k;  // free columns k..n-1
        double A[96 * 16], b[96], sol[16];
        for (int i = 0; i < m; ++i) {
            double r = y[i];
            for (int j = 0; j < k; ++j) r -= fixed[j] * T[i * n + j];
            const double w = 1.0 / fabs(y[i]);
            b[i] = w * r;
            for (int j = 0; j < nf; ++j) A[i * nf + j] = w * T[i * n + k + j];
        }
        lsq_householder(m, nf, A, b, sol);
        fixed[k] = (double)(float)sol[0];
    }
    for (int k = 0; k < n; ++k) coef[k] = (float)fixed[k];
}

// erfcx(x) = exp(x^2) erfc(x) as a degree-kErfcDeg polynomial in
// t = 1 / (1 + x/2) on x in [0, xmax] (fit_rounded_poly on 96
// Chebyshev-distributed nodes in t): within 2e-9 of erfcx at the working
// alpha rc = 2.88 (a plain fit with rounded coefficients: 7e-8, and a mean
// of -3.7e-8 over 1-2 A against +1.9e-8 over 6-9 A).  Returns the max
// relative error of exp(-x^2) P(t) against erfc(x) on a dense grid.
inline double fit_erfcx(double xmax, float *coef)
{
    constexpr int m = 96, n = kErfcDeg + 1;
    const double tmin = 1.0 / (1.0 + 0.5 * xmax);
    double T[m * n], y[m];
    for (int i = 0; i < m; ++i) {
        const double c = cos(M_PI * (i + 0.5) / m);
        const double t = 0.5 * (1.0 + tmin) + 0.5 * (1.0 - tmin) * c;
        const double x = 2.0 * (1.0 / t - 1.0);
        double p = 1.0;
        for (int k = 0; k < n; ++k) { T[i * n + k] = p; p *= t; }
        y[i] = erfc(x) * exp(x * x);
    }
    fit_rounded_poly(m, n, T, y, coef);
    double err = 0.0;
    for (int i = 0; i <= 4000; ++i) {
        const double x = xmax * i / 4000.0;
        const double t = 1.0 / (1.0 + 0.5 * x);
        double p = 0.0;
        for (int k = n - 1; k >= 0; --k) p = p * t + (double)coef[k];
        const double e = erfc(x);
        err = std::max(err, fabs(exp(-x * x) * p - e) / e);
    }
    return err;
}

// 2^f on f in [-1/2, 1/2] as a degree-kExp2Deg polynomial (fit_rounded_poly
// on 96 Chebyshev nodes): within 4e-9 relative, mean error 3e-10.  The pair
// kernels use it instead of ex2.approx, whose error has a mean of -5e-8 for
// arguments below -1 (about -1e-8 in [-1, 0)), measured on this GPU against
// FP64 -- a bias that would reach every Coulomb pair energy beyond 2.6 A.
// Returns the max relative error on a dense grid.
inline double fit_exp2(float *coef)
{
    constexpr int m = 96, n = kExp2Deg + 1;
    double T[m * n], y[m];
    for (int i = 0; i < m; ++i) {
        const double f = 0.5 * cos(M_PI * (i + 0.5) / m);
        double p = 1.0;
        for (int k = 0; k < n; ++k) { T[i * n + k] = p; p *= f; }
        y[i] = exp2(f);
    }
    fit_rounded_poly(m, n, T, y, coef);
    double err = 0.0;
    for (int i = 0; i <= 4000; ++i) {
        const double f = -0.5 + i / 4000.0;
        double p = 0.0;
        for (int k = n - 1; k >= 0; --k) p = p * f + (double)coef[k];
        err = std::max(err, fabs(p / exp2(f) - 1.0));
    }
    return err;
}

inline nb_status validate_one(const nb_params *p)
{
    if (!p) return NB_ERR_INVALID_ARG;
    if (p->n_atoms < 1 || p->flags != 0u) return NB_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (!(p->box[a] > 0.0f) || !isfinite(p->box[a])) return NB_ERR_INVALID_ARG;
    if (!(p->cutoff > 0.0f) || !isfinite(p->cutoff)) return NB_ERR_INVALID_ARG;
    if (!(p->switch_dist > 0.0f) || !isfinite(p->switch_dist)) return NB_ERR_INVALID_ARG;
    if (!(p->ewald_alpha >= 0.0f) || !isfinite(p->ewald_alpha)) return NB_ERR_INVALID_ARG;
    if (!(p->coulomb_k >= 0.0f) || !isfinite(p->coulomb_k)) return NB_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if ((double)p->box[a] * 0.5 - (double)p->cutoff < 1e-4 * (double)p->box[a]) return NB_ERR_BOX_TOO_SMALL;
    if (p->n_types < 1) return NB_ERR_INVALID_ARG;
    if (p->n_types > kMaxTypes) return NB_ERR_UNSUPPORTED;
    if (p->comb_rule == 0) {
        if (!p->sigma || !p->epsilon) return NB_ERR_INVALID_ARG;
        for (int t = 0; t < p->n_types; ++t)
            if (!(p->sigma[t] >= 0.0f) || !(p->epsilon[t] >= 0.0f) || !isfinite(p->sigma[t]) || !isfinite(p->epsilon[t]))
                return NB_ERR_INVALID_ARG;
    } else if (p->comb_rule == 1) {
        if (!p->sigma_tab || !p->eps_tab) return NB_ERR_INVALID_ARG;
        const int T = p->n_types;
        for (int a = 0; a < T; ++a)
            for (int b = 0; b < T; ++b) {
                float s = p->sigma_tab[a * T + b], e = p->eps_tab[a * T + b];
                if (!(s >= 0.0f) || !(e >= 0.0f) || !isfinite(s) || !isfinite(e)) return NB_ERR_INVALID_ARG;
                if (s != p->sigma_tab[b * T + a] || e != p->eps_tab[b * T + a]) return NB_ERR_INVALID_ARG;
            }
    } else {
        return NB_ERR_INVALID_ARG;
    }
    if (p->n_excl < 0 || p->n_14 < 0) return NB_ERR_INVALID_ARG;
    if ((p->n_excl > 0 && !p->excl) || (p->n_14 > 0 && !p->pairs14)) return NB_ERR_INVALID_ARG;
    for (int k = 0; k < p->n_excl; ++k) {
        int i = p->excl[2 * k], j = p->excl[2 * k + 1];
        if (i < 0 || j < 0 || i >= p->n_atoms || j >= p->n_atoms || i == j) return NB_ERR_INVALID_ARG;
    }
    for (int k = 0; k < p->n_14; ++k) {
        int i = p->pairs14[2 * k], j = p->pairs14[2 * k + 1];
        if (i < 0 || j < 0 || i >= p->n_atoms || j >= p->n_atoms || i == j) return NB_ERR_INVALID_ARG;
    }
    return NB_OK;
}

// (A, B) = (4 eps sig^12, 4 eps sig^6) per type pair, from per-type
// Lorentz-Berthelot parameters (comb_rule 0) or explicit pair tables.
// Type-pair tables: sigma_ab, eps_ab in FP64 and, per pair, (A, B, A - fl(A),
// B - fl(B)) with A = 4 eps sig^12, B = 4 eps sig^6 rounded to FP32 and
// their FP32 remainders (the energy adds them: a constant relative offset
// of up to 3e-8 per type pair would not cancel in a summed LJ energy).
inline void make_tables(int T, int comb_rule, const float *sigma, const float *eps, const float *sig_tab,
                        const float *eps_tab, double *sg_out, double *ep_out, float4 *lj, float4 *lj_d = nullptr)
{
    for (int a = 0; a < T; ++a)
        for (int b = 0; b < T; ++b) {
            double sg, ep;
            if (comb_rule == 0) {
                sg = 0.5 * ((double)sigma[a] + (double)sigma[b]);
                ep = sqrt((double)eps[a] * (double)eps[b]);
            } else {
                sg = sig_tab[a * T + b];
                ep = eps_tab[a * T + b];
            }
            sg_out[a * T + b] = sg;
            ep_out[a * T + b] = ep;
            double s6 = sg * sg * sg * sg * sg * sg;
            const double A = 4.0 * ep * s6 * s6, B = 4.0 * ep * s6;
            const float Af = (float)A, Bf = (float)B;
            lj[a * T + b] = make_float4(Af, Bf, (float)(A - (double)Af), (float)(B - (double)Bf));
            if (lj_d) {  // dA/dsig, dB/dsig, dA/deps, dB/deps
                const double s5 = sg * sg * sg * sg * sg, s11 = s6 * s5;
                lj_d[a * T + b] = make_float4((float)(48.0 * ep * s11), (float)(24.0 * ep * s5),
                                              (float)(4.0 * s6 * s6), (float)(4.0 * s6));
            }
        }
}

// Pair-model constants from the shared parameters of a system.
inline nb_status init_pair_params(const nb_params &P0, PairParams &pp)
{
    memset(&pp, 0, sizeof(pp));
    const float rc = P0.cutoff, rs = P0.switch_dist;
    pp.rc = rc;
    pp.rs = rs;
    pp.rc2 = rc * rc;
    pp.switched = rs < rc;
    if (pp.switched) {
        pp.rs2 = rs * rs;
        const double rc2 = (double)pp.rc2, rs2 = (double)pp.rs2;
        pp.sw_c0 = (float)(rc2 - 3.0 * rs2);
        pp.sw_inv = (float)(1.0 / ((rc2 - rs2) * (rc2 - rs2) * (rc2 - rs2)));
        pp.sw_a = (float)(1.0 / ((rc2 - rs2) * (rc2 - rs2)));
        pp.sw_b = (float)(-2.0 / ((rc2 - rs2) * (rc2 - rs2) * (rc2 - rs2)));
        pp.sw_c = (float)(12.0 / ((rc2 - rs2) * (rc2 - rs2) * (rc2 - rs2)));
    } else {
        pp.rs2 = pp.rc2;  // r2 > rs2 never holds inside the cutoff
        pp.sw_c0 = 0.0f;
        pp.sw_inv = 0.0f;
        pp.sw_a = pp.sw_b = pp.sw_c = 0.0f;
    }
    pp.ke = P0.coulomb_k > 0.0f ? P0.coulomb_k : (float)kDefaultKe;
    pp.alpha = P0.ewald_alpha;
    pp.ewald = P0.ewald_alpha > 0.0f;
    pp.alpha_half = 0.5f * P0.ewald_alpha;
    {
        const double c = -(double)P0.ewald_alpha * (double)P0.ewald_alpha * 1.4426950408889634;
        pp.neg_a2_log2e = (float)c;
        pp.neg_a2_log2e_lo = (float)(c - (double)pp.neg_a2_log2e);
    }
    pp.two_a_sqpi = (float)(2.0 * (double)P0.ewald_alpha / sqrt(M_PI));
    pp.s14_lj = P0.scale14_lj;
    pp.s14_c = P0.scale14_coul;
    pp.n_types = P0.n_types;
    pp.list_margin = 2e-3f;
    pp.rcm2 = (rc + pp.list_margin) * (rc + pp.list_margin);
    if (pp.ewald) {
        const double err = fit_erfcx((double)P0.ewald_alpha * (double)rc, pp.erfc_c);
        if (!(err < 2e-7)) return NB_ERR_UNSUPPORTED;
        if (!(fit_exp2(pp.exp2_c) < 1e-8)) return NB_ERR_UNSUPPORTED;
    }
    return NB_OK;
}

// Box, column grid and offsets of one system.
// Bins of the per-column z index: about 1 A high, at most max_nzb per column.
constexpr int kMaxZBins = 4096;

inline void init_sysdesc(const nb_params &p, SysDesc &S, int atom_begin, int col_begin, int zb_begin,
                         int max_nzb = kMaxZBins)
{
    memset(&S, 0, sizeof(S));
    const double rho = (double)p.n_atoms / ((double)p.box[0] * (double)p.box[1] * (double)p.box[2]);
    S.nx = column_count((double)p.box[0], rho);
    S.ny = column_count((double)p.box[1], rho);
    for (int a = 0; a < 3; ++a) {
        S.L[a] = p.box[a];
        S.half[a] = 0.5f * p.box[a];
    }
    S.inv_w[0] = (float)((double)S.nx / (double)p.box[0]);
    S.inv_w[1] = (float)((double)S.ny / (double)p.box[1]);
    S.w[0] = (float)((double)p.box[0] / S.nx);
    S.w[1] = (float)((double)p.box[1] / S.ny);
    S.atom_begin = atom_begin;
    S.n_atoms = p.n_atoms;
    S.col_begin = col_begin;
    int nzb = (int)ceil((double)p.box[2] / 1.0);
    S.nzb = nzb < 1 ? 1 : (nzb > max_nzb ? max_nzb : nzb);
    S.zb_begin = zb_begin;
    S.inv_dz = (float)((double)S.nzb / (double)p.box[2]);
    S.dz = (float)((double)p.box[2] / S.nzb);
}

// Entries of a system's z-bin index.
inline int64_t zbin_entries(const SysDesc &S) { return (int64_t)S.nx * S.ny * (S.nzb + 1); }

}  // namespace host
}  // namespace acenb
