// nb_adjoint.cu - adjoint of the non-bonded forces for force-field fitting:
// given G = dL/dF and gE = dL/dE (per system, LJ and Coulomb parts) it returns
// dL/dx (the Hessian-vector product -H G plus the energy term), dL/dq and the
// gradients with respect to the type-pair parameters sig_ab, eps_ab.  The
// pairs are found again from the last build's cluster-pair lists (the same
// tiles and membership test as the forward kernel); nothing per pair is
// stored between the forward and the adjoint.
#include <cuda_runtime.h>

#include "nb_internal.cuh"

namespace acenb {

// dL/dF of every sorted slot (zero for padding).
__global__ void k_gather_g(int slot_cap, const int *__restrict__ counts, const int *__restrict__ perm,
                           const float *__restrict__ G, float4 *__restrict__ gslot, long long *__restrict__ gacc)
{
    pdl_entry();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < slot_cap) {  // zero the adjoint's fixed-point sums
        gacc[4ll * s] = 0;
        gacc[4ll * s + 1] = 0;
        gacc[4ll * s + 2] = 0;
        gacc[4ll * s + 3] = 0;
    }
    if (s >= slot_cap || s >= counts[0]) return;
    const int a = perm[s];
    gslot[s] = a >= 0 ? make_float4(G[3 * (long long)a], G[3 * (long long)a + 1], G[3 * (long long)a + 2], 0.0f)
                      : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

// Symmetric type-pair gradients: each unique pair added its derivative to
// [t_i][t_j] for the order in which it was visited, so the value of the
// symmetric parameter is [a][b] + [b][a] (a != b) or [a][a].
__global__ void k_tab_finalize(int T, const long long *__restrict__ acc, double *__restrict__ dsig,
                               double *__restrict__ deps)
{
    pdl_entry();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= T * T) return;
    const int a = k / T, b = k % T;
    const double sc = 1.0 / 4294967296.0;  // 2^-32
    long long s = acc[2 * k], e = acc[2 * k + 1];
    if (a != b) {
        s += acc[2 * (b * T + a)];
        e += acc[2 * (b * T + a) + 1];
    }
    if (dsig) dsig[k] = (double)s * sc;
    if (deps) deps[k] = (double)e * sc;
}

// Lorentz-Berthelot chain from type-pair to per-type gradients (one thread
// per type; T <= 64).
__global__ void k_type_grad(int T, const float *__restrict__ eps, const double *__restrict__ gsig_tab,
                            const double *__restrict__ geps_tab, double *__restrict__ gsig, double *__restrict__ geps)
{
    pdl_entry();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    double gs = 0.0, ge = 0.0;
    for (int b = 0; b < T; ++b) {
        const int k = t * T + b;
        if (b == t) {
            gs += gsig_tab[k];
            ge += geps_tab[k];
        } else {
            gs += 0.5 * gsig_tab[k];
            if (eps[b] != 0.0f) ge += geps_tab[k] * (double)eps[b] / (2.0 * sqrt((double)eps[t] * (double)eps[b]));
        }
    }
    gsig[t] = gs;
    geps[t] = eps[t] == 0.0f ? __longlong_as_double(0x7ff8000000000000ll) : ge;
}

cudaError_t launch_type_grad(nb_ctx *ctx, const double *gsig_tab, const double *geps_tab, double *gsig, double *geps)
{
    const int T = ctx->pp.n_types;
    launch_pdl(k_type_grad, dim3(1), dim3(64), 0, ctx->stream, T, ctx->d.eps_type, gsig_tab, geps_tab, gsig, geps);
    return cudaGetLastError();
}

cudaError_t launch_backward(nb_ctx *ctx, const float *d_pos, const float *d_q, const int32_t *d_type,
                            const float *d_dLdF, const double *d_dLdE, float *d_dLdpos, float *d_dLdq, double *d_dsig,
                            double *d_deps)
{
    auto &d = ctx->d;
    const int tb = 256;
    const int S = (int)ctx->slot_cap;
    const int T = ctx->pp.n_types;
    cudaError_t e = launch_pack(ctx, d_pos, d_q, d_type, false);
    if (e != cudaSuccess) return e;
    launch_pdl(k_gather_g, dim3((S + tb - 1) / tb), dim3(tb), 0, ctx->stream, S, d.counts, d.perm, d_dLdF, d.gslot,
               d.gacc);
    e = cudaMemsetAsync(d.tab_grad, 0, sizeof(long long) * 2 * T * T, ctx->stream);
    if (e != cudaSuccess) return e;
    e = launch_adjoint_tile(ctx, d_dLdE, d_dLdpos, d_dLdq);
    if (e != cudaSuccess) return e;
    if (d_dsig || d_deps)
        e = launch_pdl(k_tab_finalize, dim3((T * T + tb - 1) / tb), dim3(tb), 0, ctx->stream, T, d.tab_grad, d_dsig,
                       d_deps);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace acenb
