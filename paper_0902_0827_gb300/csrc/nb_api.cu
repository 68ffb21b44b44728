// nb_api.cu - host side of the C ABI declared in include/acenb.h: parameter
// validation, type-pair tables, the erfcx fit, device allocation and the
// entry points.  Every compute step runs in the kernels of nb_build.cu,
// nb_force.cu and nb_adjoint.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <new>
#include <utility>
#include <vector>

#include "acenb.h"
#include "nb_internal.cuh"

using namespace acenb;

namespace {

constexpr double kDefaultKe = 332.0636;

nb_status cuda_status(cudaError_t e) { return e == cudaSuccess ? NB_OK : (e == cudaErrorMemoryAllocation ? NB_ERR_OOM : NB_ERR_CUDA); }

// Number of x-y columns along one axis: the largest n with n^3 * 8 <= L^3 rho,
// so a one-cluster slab of a column is about cubic.  Evaluated in FP64 with a
// fixed operation order (the binning is part of the bit-exact cell contract).
int column_count(double L, double rho)
{
    int n = 1;
    while (n < 4096 && (double)(n + 1) * (n + 1) * (n + 1) * kCluster <= L * L * L * rho) ++n;
    return n;
}

// Least-squares fit of erfcx(x) = exp(x^2) erfc(x) as a degree-kErfcDeg
// polynomial in t = 1 / (1 + x/2) on x in [0, xmax] (Householder QR on
// Chebyshev-distributed nodes).  Returns the max absolute error of
// exp(-x^2) P(t) against erfc(x) on a dense grid.
double fit_erfcx(double xmax, float *coef)
{
    const int m = 96, n = kErfcDeg + 1;
    const double tmin = 1.0 / (1.0 + 0.5 * xmax);
    std::vector<double> A(m * n), b(m);
    for (int i = 0; i < m; ++i) {
        double c = cos(M_PI * (i + 0.5) / m);
        double t = 0.5 * (1.0 + tmin) + 0.5 * (1.0 - tmin) * c;
        double x = 2.0 * (1.0 / t - 1.0);
        double p = 1.0;
        for (int k = 0; k < n; ++k) { A[i * n + k] = p; p *= t; }
        b[i] = erfc(x) * exp(x * x);
    }
    // Householder QR: A = Q R, solve R c = Q^T b
    for (int k = 0; k < n; ++k) {
        double nrm = 0.0;
        for (int i = k; i < m; ++i) nrm += A[i * n + k] * A[i * n + k];
        nrm = sqrt(nrm);
        double alpha = A[k * n + k] > 0 ? -nrm : nrm;
        std::vector<double> v(m, 0.0);
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
    double c[kErfcDeg + 1];
    for (int k = n - 1; k >= 0; --k) {
        double s = b[k];
        for (int j = k + 1; j < n; ++j) s -= A[k * n + j] * c[j];
        c[k] = s / A[k * n + k];
    }
    for (int k = 0; k < n; ++k) coef[k] = (float)c[k];
    double err = 0.0;
    for (int i = 0; i <= 4000; ++i) {
        double x = xmax * i / 4000.0;
        double t = 1.0 / (1.0 + 0.5 * x);
        double p = 0.0;
        for (int k = n - 1; k >= 0; --k) p = p * t + (double)coef[k];
        err = std::max(err, fabs(exp(-x * x) * p - erfc(x)));
    }
    return err;
}

template <class T>
cudaError_t dalloc(T **p, size_t count)
{
    if (count == 0) count = 1;
    return cudaMalloc((void **)p, count * sizeof(T));
}

void free_all(nb_ctx *c)
{
    auto &d = c->d;
    void *ptrs[] = {d.sys, d.atom_sys, d.atom_col, d.wpos, d.part_orig, d.col_sys, d.col_count, d.col_fill,
                    d.col_slot, d.stage, d.xyzq, d.tslot, d.perm, d.inv, d.ex_slot, d.bb,
                    d.clus_sys, d.list, d.list_n, d.sys_acc, d.tab_grad, d.counts, d.status, d.lj_tab,
                    d.dbg_n, d.dbg_ij, d.scratch_f, d.scratch_g};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    d = DevBuffers();
}

nb_status validate_one(const nb_params *p)
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

bool same_shared(const nb_params &a, const nb_params &b)
{
    if (a.cutoff != b.cutoff || a.switch_dist != b.switch_dist || a.ewald_alpha != b.ewald_alpha ||
        a.coulomb_k != b.coulomb_k || a.n_types != b.n_types || a.comb_rule != b.comb_rule ||
        a.scale14_lj != b.scale14_lj || a.scale14_coul != b.scale14_coul)
        return false;
    const int T = a.n_types;
    if (a.comb_rule == 0) {
        for (int t = 0; t < T; ++t)
            if (a.sigma[t] != b.sigma[t] || a.epsilon[t] != b.epsilon[t]) return false;
    } else {
        for (int k = 0; k < T * T; ++k)
            if (a.sigma_tab[k] != b.sigma_tab[k] || a.eps_tab[k] != b.eps_tab[k]) return false;
    }
    return true;
}

nb_status allocate(nb_ctx *c)
{
    auto &d = c->d;
    const int64_t N = c->n_atoms, C = c->n_cols, S = c->slot_cap, NC = c->clus_cap;
    const int T = c->pp.n_types;
    cudaError_t e = cudaSuccess;
#define ALLOC(ptr, n) \
    if (e == cudaSuccess) e = dalloc(&(ptr), (size_t)(n))
    ALLOC(d.sys, c->n_sys);
    ALLOC(d.atom_sys, N);
    ALLOC(d.atom_col, N);
    ALLOC(d.wpos, N);
    ALLOC(d.part_orig, N * c->K);
    ALLOC(d.col_sys, C);
    ALLOC(d.col_count, C);
    ALLOC(d.col_fill, C);
    ALLOC(d.col_slot, C + 1);
    ALLOC(d.stage, S);
    ALLOC(d.xyzq, S);
    ALLOC(d.tslot, S);
    ALLOC(d.perm, S);
    ALLOC(d.inv, N);
    ALLOC(d.ex_slot, S * c->K);
    ALLOC(d.bb, NC * 2);
    ALLOC(d.clus_sys, NC);
    ALLOC(d.list, NC * (int64_t)c->tune.list_capacity);
    ALLOC(d.list_n, NC);
    ALLOC(d.sys_acc, (int64_t)c->n_sys * kTaskVals);
    ALLOC(d.tab_grad, (int64_t)T * T * 2);
    ALLOC(d.counts, 4);
    ALLOC(d.status, 1);
    ALLOC(d.lj_tab, (int64_t)T * T);
    ALLOC(d.dbg_n, 2);
#undef ALLOC
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaMemset(d.tslot, 0, sizeof(int) * S);
    if (e == cudaSuccess) e = cudaMemset(d.status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(d.counts, 0, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMemset(d.list_n, 0, sizeof(int) * NC);
    return cuda_status(e);
}

// (A, B) = (4 eps sig^12, 4 eps sig^6) per type pair, from per-type
// Lorentz-Berthelot parameters (comb_rule 0) or explicit pair tables.
void make_tables(int T, int comb_rule, const float *sigma, const float *eps, const float *sig_tab,
                 const float *eps_tab, std::vector<double> &sg_out, std::vector<double> &ep_out,
                 std::vector<float2> &lj)
{
    sg_out.assign((size_t)T * T, 0.0);
    ep_out.assign((size_t)T * T, 0.0);
    lj.resize((size_t)T * T);
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
            lj[a * T + b] = make_float2((float)(4.0 * ep * s6 * s6), (float)(4.0 * ep * s6));
        }
}

}  // namespace

extern "C" {

const char *nb_status_string(nb_status s)
{
    switch (s) {
    case NB_OK: return "ok";
    case NB_ERR_INVALID_ARG: return "invalid argument";
    case NB_ERR_BOX_TOO_SMALL: return "box too small for the cutoff (need L/2 - rc >= 1e-4 L)";
    case NB_ERR_CUDA: return "CUDA runtime error";
    case NB_ERR_OOM: return "device out of memory";
    case NB_ERR_NOT_BUILT: return "no cell list built";
    case NB_ERR_OVERFLOW: return "fixed-point overflow";
    case NB_ERR_LIST_STALE: return "positions differ from the last build";
    case NB_ERR_TIMEOUT: return "device wait timed out";
    case NB_ERR_NONFINITE: return "non-finite coordinate";
    case NB_ERR_CAPACITY: return "cluster-pair list capacity exceeded";
    case NB_ERR_UNSUPPORTED: return "unsupported parameters";
    }
    return "unknown status";
}

nb_status nb_create_batch(int32_t n_sys, const nb_params *params, void *cuda_stream, nb_ctx **out)
{
    if (!out) return NB_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_sys < 1 || !params) return NB_ERR_INVALID_ARG;
    for (int s = 0; s < n_sys; ++s) {
        nb_status st = validate_one(&params[s]);
        if (st != NB_OK) return st;
        if (s > 0 && !same_shared(params[0], params[s])) return NB_ERR_INVALID_ARG;
    }
    int64_t N = 0;
    for (int s = 0; s < n_sys; ++s) N += params[s].n_atoms;
    if (N > (int64_t)1 << 28) return NB_ERR_UNSUPPORTED;

    nb_ctx *c = new (std::nothrow) nb_ctx();
    if (!c) return NB_ERR_OOM;
    c->n_sys = n_sys;
    c->n_atoms = N;
    c->stream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&c->device);
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (c->num_sms < 1) c->num_sms = 1;

    const nb_params &P0 = params[0];
    const int T = P0.n_types;
    // type-pair tables in FP64, then (A, B) in FP32
    std::vector<float2> lj;
    make_tables(T, P0.comb_rule, P0.sigma, P0.epsilon, P0.sigma_tab, P0.eps_tab, c->sig_tab, c->eps_tab, lj);
    c->comb_rule = P0.comb_rule;
    // pair constants
    PairParams &pp = c->pp;
    const float rc = P0.cutoff, rs = P0.switch_dist;
    pp.rc = rc;
    pp.rc2 = rc * rc;
    pp.switched = rs < rc;
    if (pp.switched) {
        pp.rs2 = rs * rs;
        double rc2 = (double)pp.rc2, rs2 = (double)pp.rs2;
        pp.sw_c0 = (float)(rc2 - 3.0 * rs2);
        pp.sw_inv = (float)(1.0 / ((rc2 - rs2) * (rc2 - rs2) * (rc2 - rs2)));
    } else {
        pp.rs2 = pp.rc2;  // r2 > rs2 never holds inside the cutoff
        pp.sw_c0 = 0.0f;
        pp.sw_inv = 0.0f;
    }
    pp.ke = P0.coulomb_k > 0.0f ? P0.coulomb_k : (float)kDefaultKe;
    pp.alpha = P0.ewald_alpha;
    pp.ewald = P0.ewald_alpha > 0.0f;
    pp.alpha_half = 0.5f * P0.ewald_alpha;
    pp.neg_a2_log2e = (float)(-(double)P0.ewald_alpha * (double)P0.ewald_alpha * 1.4426950408889634);
    pp.two_a_sqpi = (float)(2.0 * (double)P0.ewald_alpha / sqrt(M_PI));
    pp.s14_lj = P0.scale14_lj;
    pp.s14_c = P0.scale14_coul;
    pp.n_types = T;
    pp.list_margin = 2e-3f;
    pp.rcm2 = (rc + pp.list_margin) * (rc + pp.list_margin);
    if (pp.ewald) {
        double err = fit_erfcx((double)P0.ewald_alpha * (double)rc, pp.erfc_c);
        if (!(err < 2e-7)) {
            delete c;
            return NB_ERR_UNSUPPORTED;
        }
    }
    // systems, columns
    c->sys_h.resize(n_sys);
    int col = 0, atom = 0;
    std::vector<int> atom_sys(N), col_sys;
    for (int s = 0; s < n_sys; ++s) {
        const nb_params &p = params[s];
        SysDesc &S = c->sys_h[s];
        memset(&S, 0, sizeof(S));
        double rho = (double)p.n_atoms / ((double)p.box[0] * (double)p.box[1] * (double)p.box[2]);
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
        S.atom_begin = atom;
        S.n_atoms = p.n_atoms;
        S.col_begin = col;
        for (int a = 0; a < p.n_atoms; ++a) atom_sys[atom + a] = s;
        for (int k = 0; k < S.nx * S.ny; ++k) col_sys.push_back(s);
        atom += p.n_atoms;
        col += S.nx * S.ny;
    }
    c->n_cols = col;
    c->slot_cap = N + (int64_t)(kCluster - 1) * col;
    c->slot_cap = (c->slot_cap + kCluster - 1) / kCluster * kCluster;
    c->clus_cap = c->slot_cap / kCluster;
    // topology: per-atom partner lists (global indices), (orig << 1) | is14
    std::vector<std::vector<int>> part(N);
    for (int s = 0; s < n_sys; ++s) {
        const nb_params &p = params[s];
        const int base = c->sys_h[s].atom_begin;
        for (int k = 0; k < p.n_excl; ++k) {
            int i = base + p.excl[2 * k], j = base + p.excl[2 * k + 1];
            part[i].push_back(j << 1);
            part[j].push_back(i << 1);
        }
        for (int k = 0; k < p.n_14; ++k) {
            int i = base + p.pairs14[2 * k], j = base + p.pairs14[2 * k + 1];
            part[i].push_back((j << 1) | 1);
            part[j].push_back((i << 1) | 1);
        }
    }
    int K = 1;
    for (auto &v : part) {
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
        for (size_t k = 1; k < v.size(); ++k)
            if ((v[k] >> 1) == (v[k - 1] >> 1)) {  // same pair both excluded and 1-4
                delete c;
                return NB_ERR_INVALID_ARG;
            }
        K = std::max<int>(K, (int)v.size());
    }
    if (K > kMaxPartners) {
        delete c;
        return NB_ERR_UNSUPPORTED;
    }
    c->K = K;
    std::vector<int> part_flat((size_t)N * K, -1);
    for (int64_t a = 0; a < N; ++a)
        for (size_t k = 0; k < part[a].size(); ++k) part_flat[a * K + k] = part[a][k];
    // tuning defaults
    c->tune.blocks_per_sm = 3;
    c->tune.stage_capacity = 160;
    c->tune.list_capacity = 512;
    c->tune.reserved = 0;
    c->stage_cap = c->tune.stage_capacity;
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    c->smem_optin = smem_optin;

    nb_status st = allocate(c);
    if (st == NB_OK) {
        cudaError_t e = cudaMemcpy(c->d.sys, c->sys_h.data(), sizeof(SysDesc) * n_sys, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c->d.atom_sys, atom_sys.data(), sizeof(int) * N, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c->d.col_sys, col_sys.data(), sizeof(int) * col, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(c->d.part_orig, part_flat.data(), sizeof(int) * part_flat.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c->d.lj_tab, lj.data(), sizeof(float2) * lj.size(), cudaMemcpyHostToDevice);
        st = cuda_status(e);
    }
    if (st != NB_OK) {
        free_all(c);
        delete c;
        return st;
    }
    *out = c;
    return NB_OK;
}

nb_status nb_create(const nb_params *params, void *cuda_stream, nb_ctx **out)
{
    return nb_create_batch(1, params, cuda_stream, out);
}

nb_status nb_build_cells(nb_ctx *ctx, const float *d_pos)
{
    if (!ctx || !d_pos) return NB_ERR_INVALID_ARG;
    cudaError_t e = launch_build(ctx, d_pos);
    if (e != cudaSuccess) return NB_ERR_CUDA;
    ctx->built = true;
    return NB_OK;
}

nb_status nb_forces(nb_ctx *ctx, const float *d_pos, const float *d_q, const int32_t *d_type, float *d_F,
                    double *d_energy, double *d_virial)
{
    if (!ctx || !d_pos || !d_q || !d_type || !d_F) return NB_ERR_INVALID_ARG;
    if (!ctx->built) return NB_ERR_NOT_BUILT;
    cudaError_t e = launch_forces(ctx, d_pos, d_q, d_type, d_F, d_energy, d_virial, false);
    return e == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}

nb_status nb_backward(nb_ctx *ctx, const float *d_pos, const float *d_q, const int32_t *d_type,
                      const float *d_dLdF, const double *d_dLdE, float *d_dLdpos, float *d_dLdq,
                      double *d_dLdsig_tab, double *d_dLdeps_tab)
{
    if (!ctx || !d_pos || !d_q || !d_type || !d_dLdF) return NB_ERR_INVALID_ARG;
    if (!ctx->built) return NB_ERR_NOT_BUILT;
    cudaError_t e = launch_backward(ctx, d_pos, d_q, d_type, d_dLdF, d_dLdE, d_dLdpos, d_dLdq, d_dLdsig_tab,
                                    d_dLdeps_tab);
    return e == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}

nb_status nb_set_lj_params(nb_ctx *ctx, const float *h_sigma, const float *h_epsilon, const float *h_sigma_tab,
                           const float *h_eps_tab)
{
    if (!ctx) return NB_ERR_INVALID_ARG;
    const int T = ctx->pp.n_types;
    if (ctx->comb_rule == 0) {
        if (!h_sigma || !h_epsilon) return NB_ERR_INVALID_ARG;
        for (int t = 0; t < T; ++t)
            if (!(h_sigma[t] >= 0.0f) || !(h_epsilon[t] >= 0.0f) || !isfinite(h_sigma[t]) || !isfinite(h_epsilon[t]))
                return NB_ERR_INVALID_ARG;
    } else {
        if (!h_sigma_tab || !h_eps_tab) return NB_ERR_INVALID_ARG;
        for (int k = 0; k < T * T; ++k)
            if (!(h_sigma_tab[k] >= 0.0f) || !(h_eps_tab[k] >= 0.0f)) return NB_ERR_INVALID_ARG;
    }
    std::vector<float2> lj;
    make_tables(T, ctx->comb_rule, h_sigma, h_epsilon, h_sigma_tab, h_eps_tab, ctx->sig_tab, ctx->eps_tab, lj);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return NB_ERR_CUDA;
    if (cudaMemcpy(ctx->d.lj_tab, lj.data(), sizeof(float2) * lj.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return NB_ERR_CUDA;
    return NB_OK;
}

nb_status nb_get_status(nb_ctx *ctx)
{
    if (!ctx) return NB_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return NB_ERR_CUDA;
    int h = 0;
    if (cudaMemcpy(&h, ctx->d.status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return NB_ERR_CUDA;
    if (cudaMemset(ctx->d.status, 0, sizeof(int)) != cudaSuccess) return NB_ERR_CUDA;
    if (h & ST_NONFINITE) return NB_ERR_NONFINITE;
    if (h & ST_CAPACITY) return NB_ERR_CAPACITY;
    if (h & ST_STALE) return NB_ERR_LIST_STALE;
    if (h & ST_BADTYPE) return NB_ERR_INVALID_ARG;
    if (h & ST_OVERFLOW) return NB_ERR_OVERFLOW;
    if (h & ST_TIMEOUT) return NB_ERR_TIMEOUT;
    return NB_OK;
}

nb_status nb_set_stream(nb_ctx *ctx, void *cuda_stream)
{
    if (!ctx) return NB_ERR_INVALID_ARG;
    ctx->stream = (cudaStream_t)cuda_stream;
    return NB_OK;
}

nb_status nb_set_profiling(nb_ctx *ctx, int32_t on)
{
    if (!ctx) return NB_ERR_INVALID_ARG;
    if (on && ctx->prof_ev.empty()) {
        ctx->prof_ev.resize(2 * 4096);
        for (auto &e : ctx->prof_ev)
            if (cudaEventCreate(&e) != cudaSuccess) return NB_ERR_CUDA;
    }
    ctx->profiling = on != 0;
    ctx->prof_n = 0;
    return NB_OK;
}

nb_status nb_get_profile(nb_ctx *ctx, double *force_ms, int64_t *launches)
{
    if (!ctx) return NB_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return NB_ERR_CUDA;
    double tot = 0.0;
    for (int k = 0; k < ctx->prof_n; ++k) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, ctx->prof_ev[2 * k], ctx->prof_ev[2 * k + 1]) != cudaSuccess) return NB_ERR_CUDA;
        tot += ms;
    }
    if (force_ms) *force_ms = tot;
    if (launches) *launches = ctx->prof_n;
    ctx->prof_n = 0;
    return NB_OK;
}

void nb_destroy(nb_ctx *ctx)
{
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto &e : ctx->prof_ev) cudaEventDestroy(e);
    ctx->prof_ev.clear();
    free_all(ctx);
    delete ctx;
}

nb_status nb_set_tuning(nb_ctx *ctx, const nb_tuning *t)
{
    if (!ctx || !t) return NB_ERR_INVALID_ARG;
    if (t->blocks_per_sm < 1 || t->blocks_per_sm > 8 || t->reserved != 0) return NB_ERR_INVALID_ARG;
    if (t->stage_capacity < 16 || t->stage_capacity > 512 || t->stage_capacity % 4) return NB_ERR_INVALID_ARG;
    if (t->list_capacity < 64 || t->list_capacity > (1 << 16) || t->list_capacity % 4) return NB_ERR_INVALID_ARG;
    if (ctx->smem_optin > 0 && force_smem_for(ctx->pp.n_types, t->stage_capacity) > (size_t)ctx->smem_optin)
        return NB_ERR_UNSUPPORTED;
    if (t->list_capacity != ctx->tune.list_capacity) {
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return NB_ERR_CUDA;
        uint32_t *nl = nullptr;
        if (dalloc(&nl, (size_t)ctx->clus_cap * t->list_capacity) != cudaSuccess) return NB_ERR_OOM;
        cudaFree(ctx->d.list);
        ctx->d.list = nl;
        ctx->built = false;
    }
    ctx->tune = *t;
    ctx->stage_cap = t->stage_capacity;
    return NB_OK;
}

nb_status nb_get_tuning(nb_ctx *ctx, nb_tuning *t)
{
    if (!ctx || !t) return NB_ERR_INVALID_ARG;
    *t = ctx->tune;
    return NB_OK;
}

nb_status nb_get_sizes(nb_ctx *ctx, int64_t *n_atoms, int32_t *n_sys, int64_t *slot_capacity)
{
    if (!ctx) return NB_ERR_INVALID_ARG;
    if (n_atoms) *n_atoms = ctx->n_atoms;
    if (n_sys) *n_sys = ctx->n_sys;
    if (slot_capacity) *slot_capacity = ctx->slot_cap;
    return NB_OK;
}

nb_status nb_debug_cells(nb_ctx *ctx, int32_t *h_perm, int64_t *n_slots, int64_t *h_col_start, int64_t *n_columns)
{
    if (!ctx) return NB_ERR_INVALID_ARG;
    if (!ctx->built) return NB_ERR_NOT_BUILT;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return NB_ERR_CUDA;
    int counts[4];
    if (cudaMemcpy(counts, ctx->d.counts, sizeof(counts), cudaMemcpyDeviceToHost) != cudaSuccess) return NB_ERR_CUDA;
    if (n_slots) *n_slots = counts[0];
    if (n_columns) *n_columns = ctx->n_cols;
    if (h_perm && cudaMemcpy(h_perm, ctx->d.perm, sizeof(int) * counts[0], cudaMemcpyDeviceToHost) != cudaSuccess)
        return NB_ERR_CUDA;
    if (h_col_start) {
        std::vector<int> cs(ctx->n_cols + 1);
        if (cudaMemcpy(cs.data(), ctx->d.col_slot, sizeof(int) * cs.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
            return NB_ERR_CUDA;
        for (size_t k = 0; k < cs.size(); ++k) h_col_start[k] = cs[k];
    }
    return NB_OK;
}

nb_status nb_debug_pairs(nb_ctx *ctx, int32_t *h_ij, int64_t cap, int64_t *n, int64_t *n_ordered)
{
    if (!ctx || cap < 0) return NB_ERR_INVALID_ARG;
    if (!ctx->built) return NB_ERR_NOT_BUILT;
    auto &d = ctx->d;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return NB_ERR_CUDA;
    if (d.dbg_cap < cap || !d.dbg_ij) {
        if (d.dbg_ij) cudaFree(d.dbg_ij);
        d.dbg_ij = nullptr;
        if (dalloc(&d.dbg_ij, (size_t)std::max<int64_t>(cap, 1) * 2) != cudaSuccess) return NB_ERR_OOM;
        d.dbg_cap = cap;
    }
    if (!d.scratch_f && dalloc(&d.scratch_f, (size_t)ctx->n_atoms * 3) != cudaSuccess) return NB_ERR_OOM;
    if (cudaMemsetAsync(d.dbg_n, 0, 2 * sizeof(long long), ctx->stream) != cudaSuccess) return NB_ERR_CUDA;
    // positions/charges/types of the last build are already in sorted order
    cudaError_t e = launch_forces(ctx, nullptr, nullptr, nullptr, d.scratch_f, nullptr, nullptr, true);
    if (e != cudaSuccess) return NB_ERR_CUDA;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return NB_ERR_CUDA;
    long long hn[2];
    if (cudaMemcpy(hn, d.dbg_n, sizeof(hn), cudaMemcpyDeviceToHost) != cudaSuccess) return NB_ERR_CUDA;
    if (n_ordered) *n_ordered = hn[0];
    if (n) *n = hn[1];
    int64_t m = std::min<int64_t>(hn[1], cap);
    if (h_ij && m > 0 && cudaMemcpy(h_ij, d.dbg_ij, sizeof(int) * 2 * m, cudaMemcpyDeviceToHost) != cudaSuccess)
        return NB_ERR_CUDA;
    return NB_OK;
}

}  // extern "C"
