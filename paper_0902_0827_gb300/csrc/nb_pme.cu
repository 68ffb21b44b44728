// nb_pme.cu - smooth particle-mesh Ewald: the long-range half of the
// electrostatics whose short-range erfc half the force kernel evaluates
// (section "Molecular dynamics on the GPU": PME on the GPU with the FFT
// library; section "Performance": a 64^3 grid with fourth-order
// interpolation).  Smooth PME after Essmann et al.:
//
//   1. spread: Q(k) = sum_i q_i M_n(u_i1 - k1) M_n(u_i2 - k2) M_n(u_i3 - k3),
//      u_ia = K_a x_ia / L_a, cardinal B-splines M_n, periodic in k;
//   2. forward real-to-complex FFT of Q;
//   3. solve: E = 1/2 sum_m G(m) |FQ(m)|^2 with G = ke B(m) C(m),
//      C(m) = exp(-pi^2 m^2 / alpha^2) / (pi V m^2), B(m) the B-spline
//      moduli; the virial from the per-vector energies; FQ <- G FQ;
//   4. inverse complex-to-real FFT: the convolved potential theta;
//   5. gather: F_i = -q_i sum_k grad_i[M M M](k) theta(k);
//
// plus the Ewald self term -ke alpha/sqrt(pi) sum q^2 and, per excluded
// pair, -ke q_i q_j erf(alpha r)/r ((1 - s14) times that per 1-4 pair), which
// remove from the reciprocal sum what the real-space kernel leaves out.
//
// Determinism: the charge grid is accumulated in 64-bit fixed point (scale
// 2^40), forces in 64-bit fixed point (2^32) like the short-range forces,
// energies and virial in the per-system fixed-point sums; the FFTs are the
// FFT library's (cuFFT) with fixed plans.  Reruns are bit-identical.
#include <cufft.h>
#include <math.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "nb_internal.cuh"

namespace acenb {

constexpr double kGridScale = 1099511627776.0;  // 2^40: fixed-point scale of the charge grid
constexpr int kPmeThreads = 128;

struct PmeGeom {
    int K1, K2, K3, nk3;  // grid and the last axis of the half spectrum (K3/2 + 1)
    double L[3];          // box edges
    double scale[3];      // K_a / L_a
    float fscale[3];      // K_a / L_a in FP32 (chain rule of the gather)
    float inv_L[3];       // 1 / L_a in FP32 (reciprocal vectors of the solve)
};

struct PmeState {
    int K[3] = {0, 0, 0};
    int order = 0;
    long long *qfix = nullptr;  // [K1*K2*K3] charge grid, fixed point 2^40
    float *grid = nullptr;      // [K1*K2*K3] charges in FP32, then the convolved potential
    float2 *fq = nullptr;       // [K1*K2*(K3/2+1)] half spectrum
    float *gfac = nullptr;      // [K1*K2*(K3/2+1)] ke B(m) C(m)
    long long *pacc = nullptr;  // [N*3] forces in the caller's order, fixed point 2^32
    long long *acc = nullptr;   // [kPmeAcc]
    cufftHandle fwd = 0, inv = 0;
    bool have_fwd = false, have_inv = false;
    PmeGeom g{};
};

// Weights M_N(f + j) and derivatives M_N'(f + j), j = 0..N-1, of one axis for
// the fractional offset f in [0, 1): the two-term recursion
// M_p(x) = (x M_{p-1}(x) + (p - x) M_{p-1}(x - 1)) / (p - 1) from M_2, and
// M_p'(x) = M_{p-1}(x) - M_{p-1}(x - 1).
template <int N>
__device__ __forceinline__ void bspline_weights(float f, float (&w)[N], float (&dw)[N])
{
    w[0] = f;
    w[1] = 1.0f - f;
#pragma unroll
    for (int k = 2; k < N; ++k) w[k] = 0.0f;
#pragma unroll
    for (int p = 3; p <= N; ++p) {
        if (p == N) {
            dw[0] = w[0];
#pragma unroll
            for (int k = 1; k < N - 1; ++k) dw[k] = w[k] - w[k - 1];
            dw[N - 1] = -w[N - 2];
        }
        const float inv = 1.0f / (float)(p - 1);
        w[p - 1] = (1.0f - f) * w[p - 2] * inv;
#pragma unroll
        for (int k = p - 2; k >= 1; --k) w[k] = ((f + (float)k) * w[k] + ((float)(p - k) - f) * w[k - 1]) * inv;
        w[0] = f * w[0] * inv;
    }
}

// Grid base index floor(u) in [0, K) and offset f = u - floor(u) of one
// coordinate, u = K x / L with x wrapped into [0, L) in FP64.  A coordinate
// that is not finite (or so large that the wrap loses it) gives index 0 and
// f = 0, and clears ok.
__device__ __forceinline__ int grid_coord(float xf, double L, double scale, int K, float &f, bool &ok)
{
    double x = (double)xf;
    x -= L * floor(x / L);
    const double u = x * scale;
    const double fl = floor(u);
    if (!(fl >= 0.0 && fl <= (double)K)) {
        ok = false;
        f = 0.0f;
        return 0;
    }
    int i0 = (int)fl;
    f = (float)(u - fl);
    if (i0 >= K) i0 -= K;
    return i0;
}

__device__ __forceinline__ int wrap_down(int i, int K) { return i < 0 ? i + K : i; }

// Step 1.  Block of kPmeThreads atoms: weights to shared memory, then the
// block's (atom, grid point) items with the z offset fastest, so a warp's
// atomics cover a few contiguous 32-byte segments.  Also zeroes the atoms'
// force sums and (block 0) the energy/virial sums of this evaluation.
template <int N>
__global__ void __launch_bounds__(kPmeThreads) k_pme_spread(int n, const float *__restrict__ pos,
                                                           const float *__restrict__ q, PmeGeom g,
                                                           long long *__restrict__ qfix, long long *__restrict__ pacc,
                                                           long long *__restrict__ acc, int *__restrict__ status)
{
    pdl_entry();
    __shared__ int s_i0[3][kPmeThreads];
    __shared__ float s_w[3][N][kPmeThreads];
    __shared__ float s_q[kPmeThreads];
    const int t = threadIdx.x;
    const int a = blockIdx.x * kPmeThreads + t;
    if (blockIdx.x == 0 && t < kPmeAcc) acc[t] = 0;
    float qa = 0.0f;
    if (a < n) {
        qa = q[a];
        const int Ks[3] = {g.K1, g.K2, g.K3};
        bool ok = true;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            float f, w[N], dw[N];
            s_i0[ax][t] = grid_coord(pos[3ll * a + ax], g.L[ax], g.scale[ax], Ks[ax], f, ok);
            bspline_weights<N>(f, w, dw);
#pragma unroll
            for (int j = 0; j < N; ++j) s_w[ax][j][t] = w[j];
        }
        if (!ok) {
            atomicOr(status, ST_NONFINITE);
            qa = 0.0f;
        }
        pacc[3ll * a] = 0;
        pacc[3ll * a + 1] = 0;
        pacc[3ll * a + 2] = 0;
    }
    s_q[t] = qa;
    __syncthreads();
    const int na = min(kPmeThreads, n - (int)blockIdx.x * kPmeThreads);
    constexpr int N3 = N * N * N;
    const long long K23 = (long long)g.K2 * g.K3;
    for (int it = t; it < na * N3; it += kPmeThreads) {
        const int al = it / N3, p = it - al * N3;
        const int jx = p / (N * N), jy = (p / N) % N, jz = p % N;
        const float v = s_q[al] * s_w[0][jx][al] * s_w[1][jy][al] * s_w[2][jz][al];
        if (v == 0.0f) continue;
        const long long idx = wrap_down(s_i0[0][al] - jx, g.K1) * K23 +
                              (long long)wrap_down(s_i0[1][al] - jy, g.K2) * g.K3 + wrap_down(s_i0[2][al] - jz, g.K3);
        atomicAdd((unsigned long long *)&qfix[idx], (unsigned long long)__float2ll_rn(v * (float)kGridScale));
    }
}

// Fixed-point charge grid to FP32 for the FFT; clears the fixed-point grid
// for the next evaluation.
__global__ void k_pme_unfix(long long total, long long *__restrict__ qfix, float *__restrict__ grid)
{
    pdl_entry();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long v = qfix[i];
        grid[i] = __ll2float_rn(v) * (float)(1.0 / kGridScale);
        qfix[i] = 0;
    }
}

__device__ __forceinline__ long long warp_sum_ll(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Step 3 over the half spectrum (k3 = 0..K3/2): vectors with 0 < k3 < K3/2
// stand for themselves and their conjugate partners (weight 2).  Each term's
// energy e = w G |FQ|^2 / 2 and virial e (delta_ab - 2 (1 + pi^2 m^2/alpha^2)
// m_a m_b / m^2) go to the fixed-point sums; FQ is scaled by G in place.
__global__ void __launch_bounds__(256) k_pme_solve(int total, PmeGeom g, float pi2_over_a2,
                                                   const float *__restrict__ gfac, float2 *__restrict__ fq,
                                                   long long *__restrict__ acc)
{
    pdl_entry();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float e = 0.0f, w[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    if (i < total) {
        const int k3 = i % g.nk3;
        const int r = i / g.nk3;
        const int k2 = r % g.K2, k1 = r / g.K2;
        const float G = gfac[i];
        float2 z = fq[i];
        if (G != 0.0f) {
            const float wt = (k3 == 0 || 2 * k3 == g.K3) ? 0.5f : 1.0f;
            e = wt * G * fmaf(z.x, z.x, z.y * z.y);
            const float mx = (float)(k1 <= g.K1 / 2 ? k1 : k1 - g.K1) * g.inv_L[0];
            const float my = (float)(k2 <= g.K2 / 2 ? k2 : k2 - g.K2) * g.inv_L[1];
            const float mz = (float)k3 * g.inv_L[2];
            const float m2 = fmaf(mz, mz, fmaf(my, my, mx * mx));
            const float c = 2.0f * fmaf(pi2_over_a2, m2, 1.0f) / m2;
            const float ec = e * c;
            w[0] = e - ec * mx * mx;
            w[1] = e - ec * my * my;
            w[2] = e - ec * mz * mz;
            w[3] = -ec * mx * my;
            w[4] = -ec * mx * mz;
            w[5] = -ec * my * mz;
        }
        z.x *= G;
        z.y *= G;
        fq[i] = z;
    }
    long long s = warp_sum_ll(__float2ll_rn(e * (float)kFixScale));
    long long sw[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) sw[k] = warp_sum_ll(__float2ll_rn(w[k] * (float)kVirScale));
    if ((threadIdx.x & 31) == 0) {
        if (s) atomicAdd((unsigned long long *)&acc[0], (unsigned long long)s);
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (sw[k]) atomicAdd((unsigned long long *)&acc[3 + k], (unsigned long long)sw[k]);
    }
}

// Step 5 (one thread per atom) and the self and pair corrections of the
// atom's topology partners j > i, in FP64 with the FP64 minimum image.
template <int N>
__global__ void __launch_bounds__(kPmeThreads) k_pme_gather(int n, const float *__restrict__ pos,
                                                           const float *__restrict__ q, PmeGeom g,
                                                           const float *__restrict__ theta, const int *__restrict__ part,
                                                           int K, double ke, double alpha, double s14c,
                                                           long long *__restrict__ pacc, long long *__restrict__ acc)
{
    pdl_entry();
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    double e_self = 0.0, e_pair = 0.0, wv[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (a < n) {
        const float qa = q[a];
        if (qa != 0.0f) {
            int i0[3];
            float w[3][N], dw[3][N];
            const int Ks[3] = {g.K1, g.K2, g.K3};
            bool ok = true;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                float f;
                i0[ax] = grid_coord(pos[3ll * a + ax], g.L[ax], g.scale[ax], Ks[ax], f, ok);
                bspline_weights<N>(f, w[ax], dw[ax]);
            }
            float fx = 0.0f, fy = 0.0f, fz = 0.0f;
            const long long K23 = (long long)g.K2 * g.K3;
#pragma unroll
            for (int jx = 0; jx < N; ++jx) {
                const long long rx = wrap_down(i0[0] - jx, g.K1) * K23;
#pragma unroll
                for (int jy = 0; jy < N; ++jy) {
                    const long long ry = rx + (long long)wrap_down(i0[1] - jy, g.K2) * g.K3;
                    float sz = 0.0f, sdz = 0.0f;
#pragma unroll
                    for (int jz = 0; jz < N; ++jz) {
                        const float th = __ldg(&theta[ry + wrap_down(i0[2] - jz, g.K3)]);
                        sz = fmaf(w[2][jz], th, sz);
                        sdz = fmaf(dw[2][jz], th, sdz);
                    }
                    fx = fmaf(dw[0][jx] * w[1][jy], sz, fx);
                    fy = fmaf(w[0][jx] * dw[1][jy], sz, fy);
                    fz = fmaf(w[0][jx] * w[1][jy], sdz, fz);
                }
            }
            const float c = -qa;
            const float sc = (float)kFixScale;
            atomicAdd((unsigned long long *)&pacc[3ll * a], (unsigned long long)__float2ll_rn(c * g.fscale[0] * fx * sc));
            atomicAdd((unsigned long long *)&pacc[3ll * a + 1],
                      (unsigned long long)__float2ll_rn(c * g.fscale[1] * fy * sc));
            atomicAdd((unsigned long long *)&pacc[3ll * a + 2],
                      (unsigned long long)__float2ll_rn(c * g.fscale[2] * fz * sc));
            e_self = -ke * alpha * 0.56418958354775628 * (double)qa * (double)qa;  // 1/sqrt(pi)
            const double xi = pos[3ll * a], yi = pos[3ll * a + 1], zi = pos[3ll * a + 2];
            for (int k = 0; k < K; ++k) {
                const int p = part[(long long)a * K + k];
                if (p < 0) break;
                const int j = p >> 1;
                if (j <= a) continue;
                const double wgt = (p & 1) ? 1.0 - s14c : 1.0;
                const double qq = wgt * ke * (double)qa * (double)q[j];
                if (qq == 0.0) continue;
                double d[3] = {xi - (double)pos[3ll * j], yi - (double)pos[3ll * j + 1], zi - (double)pos[3ll * j + 2]};
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) d[ax] -= g.L[ax] * rint(d[ax] / g.L[ax]);
                const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (r2 == 0.0) {  // the limit erf(alpha r)/r -> 2 alpha/sqrt(pi), no force
                    e_pair -= qq * 2.0 * alpha * 0.56418958354775628;
                    continue;
                }
                const double r = sqrt(r2);
                const double er = erf(alpha * r);
                e_pair -= qq * er / r;
                // U = -qq erf(a r)/r, force on i = -dU/dr d/r
                const double fs =
                    qq * (2.0 * alpha * 0.56418958354775628 * exp(-alpha * alpha * r2) * r - er) / (r2 * r);
                const double f[3] = {fs * d[0], fs * d[1], fs * d[2]};
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    const long long v = __double2ll_rn(f[ax] * kFixScale);
                    atomicAdd((unsigned long long *)&pacc[3ll * a + ax], (unsigned long long)v);
                    atomicAdd((unsigned long long *)&pacc[3ll * j + ax], (unsigned long long)(-v));
                }
                wv[0] += d[0] * f[0];
                wv[1] += d[1] * f[1];
                wv[2] += d[2] * f[2];
                wv[3] += d[0] * f[1];
                wv[4] += d[0] * f[2];
                wv[5] += d[1] * f[2];
            }
        }
    }
    const long long s1 = warp_sum_ll(__double2ll_rn(e_self * kFixScale));
    const long long s2 = warp_sum_ll(__double2ll_rn(e_pair * kFixScale));
    long long sw[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) sw[k] = warp_sum_ll(__double2ll_rn(wv[k] * kVirScale));
    if ((threadIdx.x & 31) == 0) {
        if (s1) atomicAdd((unsigned long long *)&acc[1], (unsigned long long)s1);
        if (s2) atomicAdd((unsigned long long *)&acc[2], (unsigned long long)s2);
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (sw[k]) atomicAdd((unsigned long long *)&acc[3 + k], (unsigned long long)sw[k]);
    }
}

// Fixed-point sums of the stand-alone evaluation to the caller's outputs.
__global__ void k_pme_finalize(int n, const long long *__restrict__ pacc, const long long *__restrict__ acc,
                               float *__restrict__ F, double *__restrict__ energy, double *__restrict__ virial)
{
    pdl_entry();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const float sc = 2.3283064365386963e-10f;  // 2^-32
    if (i < 3 * n) F[i] = __ll2float_rn(pacc[i]) * sc;
    if (blockIdx.x == 0 && threadIdx.x < kPmeAcc) {
        const int k = threadIdx.x;
        const double v = (double)acc[k] * (k < 3 ? 1.0 / kFixScale : 1.0 / kVirScale);
        if (k < 3) {
            if (energy) energy[k] = v;
        } else if (virial) {
            virial[k - 3] = v;
        }
    }
}

// ---------------------------------------------------------------- host side

// M_n(k), k = 0..n-1, at the integers.
static std::vector<double> bspline_at_integers(int n)
{
    std::vector<double> w(n, 0.0);
    w[0] = 0.0;  // M_2(0)
    w[1] = 1.0;  // M_2(1)
    for (int p = 3; p <= n; ++p) {
        std::vector<double> v(n, 0.0);
        for (int k = 0; k < p; ++k) {
            const double a = k < p - 1 ? w[k] : 0.0, b = k >= 1 ? w[k - 1] : 0.0;
            v[k] = ((double)k * a + (double)(p - k) * b) / (double)(p - 1);
        }
        w = v;
    }
    return w;
}

// |b(m)|^2 = 1 / |sum_{j=0}^{n-2} M_n(j+1) exp(2 pi i m j / K)|^2.
static std::vector<double> bspline_moduli(int K, int n)
{
    const std::vector<double> M = bspline_at_integers(n);
    std::vector<double> b(K);
    for (int m = 0; m < K; ++m) {
        std::complex<double> s(0.0, 0.0);
        for (int j = 0; j <= n - 2; ++j) s += M[j + 1] * std::polar(1.0, 2.0 * M_PI * (double)m * j / K);
        b[m] = 1.0 / std::norm(s);
    }
    return b;
}

void pme_free(nb_ctx *ctx)
{
    PmeState *p = ctx->pme;
    if (!p) return;
    if (p->have_fwd) cufftDestroy(p->fwd);
    if (p->have_inv) cufftDestroy(p->inv);
    void *ptrs[] = {p->qfix, p->grid, p->fq, p->gfac, p->pacc, p->acc};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    delete p;
    ctx->pme = nullptr;
}

const long long *pme_forces_acc(const nb_ctx *ctx) { return ctx->pme ? ctx->pme->pacc : nullptr; }
const long long *pme_sums_acc(const nb_ctx *ctx) { return ctx->pme ? ctx->pme->acc : nullptr; }

template <int N>
static cudaError_t launch_pme_t(nb_ctx *ctx, const float *d_pos, const float *d_q)
{
    PmeState &P = *ctx->pme;
    const PmeGeom &g = P.g;
    const int n = (int)ctx->n_atoms;
    const cudaStream_t st = ctx->stream;
    const int blocks = (n + kPmeThreads - 1) / kPmeThreads;
    cudaError_t e = launch_pdl(k_pme_spread<N>, dim3(blocks), dim3(kPmeThreads), 0, st, n, d_pos, d_q, g, P.qfix,
                               P.pacc, P.acc, ctx->d.status);
    if (e != cudaSuccess) return e;
    const long long total = (long long)g.K1 * g.K2 * g.K3;
    const int ub = (int)std::min<long long>((total + 255) / 256, 8ll * ctx->num_sms);
    e = launch_pdl(k_pme_unfix, dim3(ub), dim3(256), 0, st, total, P.qfix, P.grid);
    if (e != cudaSuccess) return e;
    if (cufftSetStream(P.fwd, st) != CUFFT_SUCCESS || cufftExecR2C(P.fwd, P.grid, (cufftComplex *)P.fq) != CUFFT_SUCCESS)
        return cudaErrorUnknown;
    const int half = g.K1 * g.K2 * g.nk3;
    const float a = ctx->pp.alpha;
    const float pi2_over_a2 = (float)(M_PI * M_PI / ((double)a * (double)a));
    e = launch_pdl(k_pme_solve, dim3((half + 255) / 256), dim3(256), 0, st, half, g, pi2_over_a2, P.gfac, P.fq, P.acc);
    if (e != cudaSuccess) return e;
    if (cufftSetStream(P.inv, st) != CUFFT_SUCCESS || cufftExecC2R(P.inv, (cufftComplex *)P.fq, P.grid) != CUFFT_SUCCESS)
        return cudaErrorUnknown;
    return launch_pdl(k_pme_gather<N>, dim3(blocks), dim3(kPmeThreads), 0, st, n, d_pos, d_q, g,
                      (const float *)P.grid, (const int *)ctx->d.part_orig, ctx->K, (double)ctx->pp.ke,
                      (double)ctx->pp.alpha, (double)ctx->pp.s14_c, P.pacc, P.acc);
}

cudaError_t launch_pme(nb_ctx *ctx, const float *d_pos, const float *d_q)
{
    switch (ctx->pme->order) {
    case 4: return launch_pme_t<4>(ctx, d_pos, d_q);
    case 6: return launch_pme_t<6>(ctx, d_pos, d_q);
    case 8: return launch_pme_t<8>(ctx, d_pos, d_q);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace acenb

using namespace acenb;

extern "C" nb_status nb_set_pme(nb_ctx *ctx, const nb_pme_params *p)
{
    if (!ctx) return NB_ERR_INVALID_ARG;
    if (!p) {
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return NB_ERR_CUDA;
        pme_free(ctx);
        return NB_OK;
    }
    if (p->flags != 0) return NB_ERR_INVALID_ARG;
    if (p->order != 4 && p->order != 6 && p->order != 8) return NB_ERR_UNSUPPORTED;
    for (int a = 0; a < 3; ++a)
        if (p->grid[a] < p->order || p->grid[a] > kPmeMaxGrid) return NB_ERR_INVALID_ARG;
    if (ctx->n_sys != 1 || !ctx->pp.ewald) return NB_ERR_UNSUPPORTED;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return NB_ERR_CUDA;
    pme_free(ctx);
    PmeState *P = new PmeState();
    ctx->pme = P;
    for (int a = 0; a < 3; ++a) P->K[a] = p->grid[a];
    P->order = p->order;
    const int K1 = P->K[0], K2 = P->K[1], K3 = P->K[2], nk3 = K3 / 2 + 1;
    const float *Lf = ctx->sys_h[0].L;
    PmeGeom &g = P->g;
    g.K1 = K1;
    g.K2 = K2;
    g.K3 = K3;
    g.nk3 = nk3;
    for (int a = 0; a < 3; ++a) {
        g.L[a] = (double)Lf[a];
        g.scale[a] = (double)P->K[a] / (double)Lf[a];
        g.fscale[a] = (float)g.scale[a];
        g.inv_L[a] = (float)(1.0 / (double)Lf[a]);
    }
    const size_t total = (size_t)K1 * K2 * K3, half = (size_t)K1 * K2 * nk3;
    cudaError_t e = cudaMalloc(&P->qfix, sizeof(long long) * total);
    if (e == cudaSuccess) e = cudaMalloc(&P->grid, sizeof(float) * total);
    if (e == cudaSuccess) e = cudaMalloc(&P->fq, sizeof(float2) * half);
    if (e == cudaSuccess) e = cudaMalloc(&P->gfac, sizeof(float) * half);
    if (e == cudaSuccess) e = cudaMalloc(&P->pacc, sizeof(long long) * 3 * std::max<int64_t>(ctx->n_atoms, 1));
    if (e == cudaSuccess) e = cudaMalloc(&P->acc, sizeof(long long) * kPmeAcc);
    if (e == cudaSuccess) e = cudaMemset(P->qfix, 0, sizeof(long long) * total);
    if (e != cudaSuccess) {
        pme_free(ctx);
        return e == cudaErrorMemoryAllocation ? NB_ERR_OOM : NB_ERR_CUDA;
    }
    // influence function G(m) = ke B(m) C(m) on the half spectrum, FP64 on the host
    const double alpha = (double)ctx->pp.alpha, ke = (double)ctx->pp.ke;
    const double V = g.L[0] * g.L[1] * g.L[2];
    const std::vector<double> b1 = bspline_moduli(K1, P->order), b2 = bspline_moduli(K2, P->order),
                              b3 = bspline_moduli(K3, P->order);
    std::vector<float> G(half);
    for (int k1 = 0; k1 < K1; ++k1)
        for (int k2 = 0; k2 < K2; ++k2)
            for (int k3 = 0; k3 < nk3; ++k3) {
                const double mx = (double)(k1 <= K1 / 2 ? k1 : k1 - K1) / g.L[0];
                const double my = (double)(k2 <= K2 / 2 ? k2 : k2 - K2) / g.L[1];
                const double mz = (double)k3 / g.L[2];
                const double m2 = mx * mx + my * my + mz * mz;
                const size_t i = ((size_t)k1 * K2 + k2) * nk3 + k3;
                G[i] = m2 == 0.0 ? 0.0f
                                 : (float)(ke * b1[k1] * b2[k2] * b3[k3] * exp(-M_PI * M_PI * m2 / (alpha * alpha)) /
                                           (M_PI * V * m2));
            }
    e = cudaMemcpy(P->gfac, G.data(), sizeof(float) * half, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        pme_free(ctx);
        return NB_ERR_CUDA;
    }
    if (cufftPlan3d(&P->fwd, K1, K2, K3, CUFFT_R2C) != CUFFT_SUCCESS) {
        pme_free(ctx);
        return NB_ERR_CUDA;
    }
    P->have_fwd = true;
    if (cufftPlan3d(&P->inv, K1, K2, K3, CUFFT_C2R) != CUFFT_SUCCESS) {
        pme_free(ctx);
        return NB_ERR_CUDA;
    }
    P->have_inv = true;
    return NB_OK;
}

extern "C" nb_status nb_pme_forces(nb_ctx *ctx, const float *d_pos, const float *d_q, float *d_F, double *d_energy,
                                   double *d_virial)
{
    if (!ctx || !d_pos || !d_q || !d_F) return NB_ERR_INVALID_ARG;
    if (!ctx->pme) return NB_ERR_NOT_BUILT;
    cudaError_t e = launch_pme(ctx, d_pos, d_q);
    if (e != cudaSuccess) return NB_ERR_CUDA;
    const int n = (int)ctx->n_atoms;
    e = launch_pdl(k_pme_finalize, dim3((3 * n + 255) / 256), dim3(256), 0, ctx->stream, n,
                   (const long long *)ctx->pme->pacc, (const long long *)ctx->pme->acc, d_F, d_energy, d_virial);
    return e == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}
