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
#include "nb_host.cuh"
#include "nb_internal.cuh"

using namespace acenb;
using namespace acenb::host;

namespace {

nb_status cuda_status(cudaError_t e) { return e == cudaSuccess ? NB_OK : (e == cudaErrorMemoryAllocation ? NB_ERR_OOM : NB_ERR_CUDA); }

template <class T>
cudaError_t dalloc(T **p, size_t count)
{
    if (count == 0) count = 1;
    return cudaMalloc((void **)p, count * sizeof(T));
}

void free_all(nb_ctx *c)
{
    auto &d = c->d;
    void *ptrs[] = {d.sys, d.atom_sys, d.atom_col, d.wpos, d.atom_t, d.part_orig, d.col_sys, d.col_count,
                    d.col_slot, d.stage, d.stage_fix, d.xyzq, d.tslot, d.perm, d.inv, d.bb,
                    d.clus_sys, d.sys_acc, d.facc, d.gacc, d.col_grp, d.grp, d.clus_grp, d.glist, d.glist_n, d.gmask,
                    d.zbin, d.tab_grad, d.counts, d.status, d.lj_tab,
                    d.dbg_n, d.dbg_ij, d.scratch_f, d.scratch_g, d.lj_d, d.gslot, d.eps_type, d.rtab};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    d = DevBuffers();
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
    ALLOC(d.atom_t, N);
    ALLOC(d.part_orig, N * c->K);
    ALLOC(d.col_sys, C);
    ALLOC(d.col_count, 2 * C + 1);
    ALLOC(d.col_slot, C + 1);
    ALLOC(d.stage, S);
    ALLOC(d.stage_fix, (int64_t)C * c->col_cap);
    ALLOC(d.xyzq, S);
    ALLOC(d.tslot, S);
    ALLOC(d.perm, S);
    ALLOC(d.inv, N);
    ALLOC(d.bb, NC * 2);
    ALLOC(d.clus_sys, NC);
    ALLOC(d.sys_acc, (int64_t)c->n_sys * kTaskVals);
    ALLOC(d.facc, S * 3);
    ALLOC(d.gacc, S * 4);
    ALLOC(d.col_grp, C + 1);
    ALLOC(d.grp, c->grp_cap);
    ALLOC(d.clus_grp, NC);
    ALLOC(d.glist, c->grp_cap * c->list_cap);
    ALLOC(d.glist_n, c->grp_cap * kListSegs);
    ALLOC(d.gmask, c->mask_cap * kMaxGroup);
    ALLOC(d.zbin, c->zb_total);
    ALLOC(d.tab_grad, (int64_t)T * T * 2);
    ALLOC(d.counts, 8);
    ALLOC(d.status, 1);
    ALLOC(d.lj_tab, (int64_t)T * T);
    ALLOC(d.lj_d, (int64_t)T * T);
    ALLOC(d.gslot, S);
    ALLOC(d.eps_type, T);
    ALLOC(d.dbg_n, 4);
#undef ALLOC
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaMemset(d.tslot, 0, sizeof(int) * S);
    if (e == cudaSuccess) e = cudaMemset(d.status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(d.counts, 0, sizeof(int) * 8);
    if (e == cudaSuccess) e = cudaMemset(d.col_count, 0, sizeof(int) * (2 * C + 1));  // kept zero between builds
    return cuda_status(e);
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
    case NB_ERR_TOO_LARGE: return "system exceeds the fixed scratch of nb_forces_noalloc";
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
    std::vector<float4> lj((size_t)T * T);
    std::vector<float4> ljd((size_t)T * T);
    c->sig_tab.assign((size_t)T * T, 0.0);
    c->eps_tab.assign((size_t)T * T, 0.0);
    make_tables(T, P0.comb_rule, P0.sigma, P0.epsilon, P0.sigma_tab, P0.eps_tab, c->sig_tab.data(),
                c->eps_tab.data(), lj.data(), ljd.data());
    c->comb_rule = P0.comb_rule;
    if (init_pair_params(P0, c->pp) != NB_OK) {
        delete c;
        return NB_ERR_UNSUPPORTED;
    }
    // systems, columns
    c->sys_h.resize(n_sys);
    int col = 0, atom = 0;
    int64_t zb = 0;
    std::vector<int> atom_sys(N), col_sys;
    double mean_col = 1.0;  // largest mean column population of the systems
    for (int s = 0; s < n_sys; ++s) {
        const nb_params &p = params[s];
        SysDesc &S = c->sys_h[s];
        if (zb > 0x7fffffff) {
            delete c;
            return NB_ERR_TOO_LARGE;
        }
        init_sysdesc(p, S, atom, col, (int)zb);
        zb += zbin_entries(S);
        for (int a = 0; a < p.n_atoms; ++a) atom_sys[atom + a] = s;
        for (int k = 0; k < S.nx * S.ny; ++k) col_sys.push_back(s);
        mean_col = std::max(mean_col, (double)p.n_atoms / (double)(S.nx * S.ny));
        atom += p.n_atoms;
        col += S.nx * S.ny;
    }
    c->n_cols = col;
    c->zb_total = zb;
    c->slot_cap = N + (int64_t)(kCluster - 1) * col;
    c->slot_cap = (c->slot_cap + kCluster - 1) / kCluster * kCluster;
    c->clus_cap = c->slot_cap / kCluster;
    c->grp_cap = group_capacity(c->clus_cap);
    c->mask_cap = mask_capacity(c->clus_cap);
    c->col_cap = column_capacity(mean_col);
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
    c->tune.stage_capacity = 96;
    c->tune.list_capacity = 512;
    c->tune.list_split = kDefaultListSplit;
    c->tune.group_clusters = kDefaultGroup;
    c->group = kDefaultGroup;
    c->stage_cap = c->tune.stage_capacity;
    c->list_cap = c->tune.list_capacity;
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
        if (e == cudaSuccess) e = cudaMemcpy(c->d.lj_tab, lj.data(), sizeof(float4) * lj.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c->d.lj_d, ljd.data(), sizeof(float4) * ljd.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && P0.comb_rule == 0)
            e = cudaMemcpy(c->d.eps_type, P0.epsilon, sizeof(float) * T, cudaMemcpyHostToDevice);
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

nb_status nb_forces_batch(nb_ctx *batch, const float *d_pos, const float *d_q, const int32_t *d_type, float *d_F,
                          double *d_energy, double *d_virial)
{
    return nb_forces(batch, d_pos, d_q, d_type, d_F, d_energy, d_virial);
}

nb_status nb_step(nb_ctx *ctx, const float *d_pos, const float *d_q, const int32_t *d_type, float *d_F,
                  double *d_energy, double *d_virial)
{
    if (!ctx || !d_pos || !d_q || !d_type || !d_F) return NB_ERR_INVALID_ARG;
    // the binning kernel and the column sort pack charges and types; PME (which needs only the
    // sorted atoms) is forked before the lists, beside the list and force kernels
    cudaError_t e = launch_build_cells(ctx, d_pos, d_q, d_type);
    const bool pme = ctx->pme != nullptr;
    if (e == cudaSuccess && pme) e = launch_pme_fork(ctx, d_pos, d_q);
    if (e == cudaSuccess) e = launch_build_lists(ctx);
    if (e != cudaSuccess) return NB_ERR_CUDA;
    ctx->built = true;
    e = launch_forces_packed(ctx, d_F, d_energy, d_virial, false, pme, pme, pme);
    return e == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}

nb_status nb_backward(nb_ctx *ctx, const float *d_pos, const float *d_q, const int32_t *d_type,
                      const float *d_dLdF, const double *d_dLdE, float *d_dLdpos, float *d_dLdq,
                      double *d_dLdsig_tab, double *d_dLdeps_tab)
{
    if (!ctx || !d_pos || !d_q || !d_type || !d_dLdF) return NB_ERR_INVALID_ARG;
    if (!ctx->built) return NB_ERR_NOT_BUILT;
    if (ctx->pme || ctx->tab_n > 0) return NB_ERR_UNSUPPORTED;
    cudaError_t e = launch_backward(ctx, d_pos, d_q, d_type, d_dLdF, d_dLdE, d_dLdpos, d_dLdq, d_dLdsig_tab,
                                    d_dLdeps_tab);
    return e == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}

// The six radial functions at r: E12 = S r^-12, E6 = S r^-6, Ec = erfc(alpha r)/r
// (1/r without Ewald) and F = -r dE/dr of each (FP64, host).
static void radial_functions(const PairParams &pp, double rc, double rs, double alpha, double r, double f[6])
{
    double S = 1.0, rS1 = 0.0;  // switch and r dS/dr
    if (pp.switched && r > rs) {
        const double rc2 = rc * rc, rs2 = rs * rs, r2 = r * r, D = (rc2 - rs2) * (rc2 - rs2) * (rc2 - rs2);
        S = (rc2 - r2) * (rc2 - r2) * (rc2 + 2.0 * r2 - 3.0 * rs2) / D;
        rS1 = 12.0 * r2 * (rc2 - r2) * (rs2 - r2) / D;
    }
    const double ir = 1.0 / r, ir6 = ir * ir * ir * ir * ir * ir, ir12 = ir6 * ir6;
    f[0] = S * ir12;
    f[1] = S * ir6;
    f[3] = 12.0 * S * ir12 - rS1 * ir12;
    f[4] = 6.0 * S * ir6 - rS1 * ir6;
    if (alpha > 0.0) {
        f[2] = std::erfc(alpha * r) * ir;
        f[5] = f[2] + 2.0 * alpha / std::sqrt(M_PI) * std::exp(-alpha * alpha * r * r);
    } else {
        f[2] = ir;
        f[5] = ir;
    }
}

nb_status nb_set_tables(nb_ctx *ctx, int32_t n_intervals)
{
    if (!ctx) return NB_ERR_INVALID_ARG;
    if (n_intervals != 0 && (n_intervals < 16 || n_intervals > 65536)) return NB_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return NB_ERR_CUDA;
    cudaFree(ctx->d.rtab);
    ctx->d.rtab = nullptr;
    ctx->tab_n = 0;
    ctx->pp.tab_n = 0;
    if (n_intervals == 0) return NB_OK;
    const int n = n_intervals;
    const double rc = (double)ctx->pp.rc, rs = (double)ctx->pp.rs, alpha = (double)ctx->pp.alpha;
    const double rfloor = 0.5;  // below it every point repeats the value at 0.5 A (never reached)
    std::vector<float4> h((size_t)3 * n);
    double f0[6], f1[6];
    for (int k = 0; k < n; ++k) {
        const double r0 = (double)k * rc / n, r1 = (double)(k + 1) * rc / n;
        radial_functions(ctx->pp, rc, rs, alpha, std::max(r0, rfloor), f0);
        radial_functions(ctx->pp, rc, rs, alpha, std::max(r1, rfloor), f1);
        float v[6], dv[6];
        for (int c = 0; c < 6; ++c) {
            v[c] = (float)f0[c];
            dv[c] = (float)(f1[c] - f0[c]);
        }
        h[3 * k] = make_float4(v[0], dv[0], v[1], dv[1]);
        h[3 * k + 1] = make_float4(v[2], dv[2], v[3], dv[3]);
        h[3 * k + 2] = make_float4(v[4], dv[4], v[5], dv[5]);
    }
    float4 *dt = nullptr;
    if (cudaMalloc(&dt, sizeof(float4) * h.size()) != cudaSuccess) return NB_ERR_OOM;
    if (cudaMemcpy(dt, h.data(), sizeof(float4) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(dt);
        return NB_ERR_CUDA;
    }
    ctx->d.rtab = dt;
    ctx->tab_n = n;
    ctx->pp.tab_n = n;
    ctx->pp.tab_inv_h = (float)((double)n / rc);
    return NB_OK;
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
    std::vector<float4> lj((size_t)T * T);
    std::vector<float4> ljd((size_t)T * T);
    make_tables(T, ctx->comb_rule, h_sigma, h_epsilon, h_sigma_tab, h_eps_tab, ctx->sig_tab.data(),
                ctx->eps_tab.data(), lj.data(), ljd.data());
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return NB_ERR_CUDA;
    if (cudaMemcpy(ctx->d.lj_tab, lj.data(), sizeof(float4) * lj.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return NB_ERR_CUDA;
    if (cudaMemcpy(ctx->d.lj_d, ljd.data(), sizeof(float4) * ljd.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return NB_ERR_CUDA;
    if (ctx->comb_rule == 0 &&
        cudaMemcpy(ctx->d.eps_type, h_epsilon, sizeof(float) * T, cudaMemcpyHostToDevice) != cudaSuccess)
        return NB_ERR_CUDA;
    return NB_OK;
}

nb_status nb_type_gradients(nb_ctx *ctx, const double *d_dLdsig_tab, const double *d_dLdeps_tab, double *d_dLdsigma,
                            double *d_dLdeps)
{
    if (!ctx || !d_dLdsig_tab || !d_dLdeps_tab || !d_dLdsigma || !d_dLdeps) return NB_ERR_INVALID_ARG;
    if (ctx->comb_rule != 0) return NB_ERR_UNSUPPORTED;
    return launch_type_grad(ctx, d_dLdsig_tab, d_dLdeps_tab, d_dLdsigma, d_dLdeps) == cudaSuccess ? NB_OK
                                                                                                  : NB_ERR_CUDA;
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
    pme_free(ctx);
    md_free(ctx);
    free_all(ctx);
    delete ctx;
}

nb_status nb_set_tuning(nb_ctx *ctx, const nb_tuning *t)
{
    if (!ctx || !t) return NB_ERR_INVALID_ARG;
    if (t->blocks_per_sm < 1 || t->blocks_per_sm > 8 || t->list_split < 0 || t->list_split > 8) return NB_ERR_INVALID_ARG;
    if (t->group_clusters != 0 && t->group_clusters != 1 && t->group_clusters != 4 && t->group_clusters != 8)
        return NB_ERR_INVALID_ARG;
    if (t->stage_capacity < 16 || t->stage_capacity > 512 || t->stage_capacity % 4) return NB_ERR_INVALID_ARG;
    if (t->list_capacity < 64 || t->list_capacity > 65536 || t->list_capacity % 4) return NB_ERR_INVALID_ARG;
    if (ctx->smem_optin > 0 && force_smem_for(ctx->pp.n_types, t->stage_capacity, ctx->K) > (size_t)ctx->smem_optin)
        return NB_ERR_UNSUPPORTED;
    if (t->list_capacity != ctx->list_cap) {
        // new list storage: the lists of the last build are gone
        uint2 *nl = nullptr;
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return NB_ERR_CUDA;
        if (dalloc(&nl, (size_t)ctx->grp_cap * t->list_capacity) != cudaSuccess) return NB_ERR_OOM;
        cudaFree(ctx->d.glist);
        ctx->d.glist = nl;
        ctx->list_cap = t->list_capacity;
        ctx->built = false;
    }
    const int gsize = t->group_clusters > 0 ? t->group_clusters : kDefaultGroup;
    if (gsize != ctx->group) {
        ctx->group = gsize;  // the lists are built for a group size: a new build is needed
        ctx->built = false;
    }
    ctx->tune = *t;
    ctx->tune.group_clusters = gsize;
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
    if (cudaMemsetAsync(d.dbg_n, 0, 4 * sizeof(long long), ctx->stream) != cudaSuccess) return NB_ERR_CUDA;
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

nb_status nb_debug_fill(nb_ctx *ctx, int64_t *tiles, int64_t *halves)
{
    if (!ctx || !tiles || !halves) return NB_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return NB_ERR_CUDA;
    long long hn[4];
    if (cudaMemcpy(hn, ctx->d.dbg_n, sizeof(hn), cudaMemcpyDeviceToHost) != cudaSuccess) return NB_ERR_CUDA;
    *tiles = hn[3];
    *halves = hn[2];
    return NB_OK;
}

nb_status nb_debug_pair_terms(nb_ctx *ctx, int64_t n, const float *d_xqi, const float *d_xqj, const int32_t *d_ti,
                              const int32_t *d_tj, float *d_out)
{
    if (!ctx || n < 0 || (n > 0 && (!d_xqi || !d_xqj || !d_ti || !d_tj || !d_out))) return NB_ERR_INVALID_ARG;
    if (n == 0) return NB_OK;
    const cudaError_t e = launch_debug_pair_terms(ctx, n, reinterpret_cast<const float4 *>(d_xqi),
                                                  reinterpret_cast<const float4 *>(d_xqj), d_ti, d_tj,
                                                  reinterpret_cast<float4 *>(d_out));
    return e == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}

}  // extern "C"
