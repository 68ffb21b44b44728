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
// Determinism: the charge grid is accumulated in fixed point (scale 2^32)
// in shared memory, forces in 64-bit fixed point (2^32) like the short-range forces,
// energies and virial in the per-system fixed-point sums; the FFTs are the
// FFT library's (cuFFT) with fixed plans.  Reruns are bit-identical.
#include <cufft.h>
#include <math.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "nb_internal.cuh"

namespace acenb {

constexpr double kGridScale = 4294967296.0;     // 2^32: fixed-point scale of the charge grid
constexpr double kQ2Scale = 68719476736.0;      // 2^36: fixed-point scale of sum q^2
constexpr int kPmeThreads = 512;                // threads of a spread block
constexpr int kColBatch = 64;                   // cell-list columns staged per pass of the spread
constexpr int kTileElems = 512;                 // grid points of one spread tile (4 KB: two int32 words each)

struct PmeGeom {
    int K1, K2, K3, nk3;  // grid and the last axis of the half spectrum (K3/2 + 1)
    int Ty;               // grid rows (y) per spread tile
    float s_hi[3];        // K_a / L_a = s_hi + s_lo (FP32 pair)
    float s_lo[3];
    float h[3];           // L_a / K_a (grid spacing, FP32)
    float fscale[3];      // K_a / L_a in FP32 (chain rule of the gather)
    float inv_L[3];       // 1 / L_a in FP32 (reciprocal vectors of the solve)
};

constexpr int kSeriesTerms = 12;
constexpr int kErfxTerms = 26;  // erf(x)/x series terms for x^2 <= 4 (last term below 4e-13 of the sum)

struct PmeCorr {
    float ke, alpha, one_m_s14;  // Coulomb constant, Ewald alpha, 1 - s14_coul
    float two_a_sqpi;            // 2 alpha / sqrt(pi)
    float two_a3_sqpi;           // 2 alpha^3 / sqrt(pi)
    float L[3], half[3];         // box and half box (minimum image)
    // g(x) = erf(x) - 2 x exp(-x^2) / sqrt(pi) = 2 x^3 / sqrt(pi) sum_n c_n x^(2n),
    // c_n = (-1)^n 2 (n+1) / ((2n+3) (n+1)!), from the Maclaurin series of
    // erf and of x exp(-x^2); used for x < 1, where the direct difference
    // loses digits
    float series[kSeriesTerms];
    // erf(x)/x = sum_n e_n x^(2n), e_n = (2/sqrt(pi)) (-1)^n / (n! (2n+1)), as
    // (hi, lo) pairs, and alpha^2 as a pair: the pair energies in
    // double-FP32 arithmetic (x^2 = alpha^2 r^2 needs no square root)
    float2 erfx[kErfxTerms];
    float2 a2;
};

// Double-FP32 arithmetic (Dekker 1971; Knuth, TAOCP vol. 2): a value is
// hi + lo, about 48 significant bits.  two_sum and two_prod give the exact
// rounding error of a sum and (by FMA) of a product; the intrinsics keep the
// compiler from contracting or reordering them.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ DF df_fast_two_sum(float a, float b)  // |a| >= |b| or a = 0
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ DF df_add(DF a, DF b)
{
    const DF s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ DF df_mul(DF a, DF b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = __fmaf_rn(a.hi, b.hi, -p);
    return df_fast_two_sum(p, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e)));
}

__device__ __forceinline__ DF df_mul_f(DF a, float b)
{
    const float p = __fmul_rn(a.hi, b);
    return df_fast_two_sum(p, __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p)));
}

struct PmeState {
    int K[3] = {0, 0, 0};
    int order = 0;
    float *grid = nullptr;      // [K1*K2*K3] charges in FP32, then the convolved potential
    float2 *fq = nullptr;       // [K1*K2*(K3/2+1)] half spectrum
    float *gfac = nullptr;      // [K1*K2*(K3/2+1)] ke B(m) C(m)
    long long *pacc = nullptr;  // [slot_cap*3] forces in sorted-slot order, fixed point 2^32
    long long *acc = nullptr;   // [kPmeAcc]: E_recip (2^32), sum q^2 (2^36), E_excl (2^32), W[6] (2^20)
    double self_coef = 0.0;     // -ke alpha / sqrt(pi)
    cufftHandle fwd = 0, inv = 0;
    bool have_fwd = false, have_inv = false;
    // nb_forces runs the chain on `side`, forked from and joined back to the
    // context's stream, so it overlaps the short-range kernel
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaEvent_t lists = nullptr;  // the pair lists are built (the short-range helper may start)
    PmeGeom g{};
    PmeCorr c{};
};

// Weights M_N(f + j) and derivatives M_N'(f + j), j = 0..N-1, of one axis for
// the fractional offset f in [0, 1]: the two-term recursion
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

// Grid base index floor(u) in [0, K) and offset f = u - floor(u) of a
// coordinate x in [0, L), u = x K / L (any other input gives index 0 and
// f = 0, so no index leaves the grid).  K / L is carried as an FP32 pair
// (s_hi + s_lo) and the product's rounding error is recovered with an FMA,
// so f is accurate to FP32 rounding of f itself (about 6e-8 grid spacings)
// although u reaches K.
__device__ __forceinline__ int grid_coord(float x, float s_hi, float s_lo, int K, float &f)
{
    const float p = x * s_hi;
    const float c = fmaf(x, s_lo, fmaf(x, s_hi, -p));
    float fl = floorf(p);
    float fr = (p - fl) + c;  // p - floor(p) is exact
    if (fr < 0.0f) {
        fr += 1.0f;
        fl -= 1.0f;
    } else if (fr >= 1.0f) {
        fr -= 1.0f;
        fl += 1.0f;
    }
    int i0 = (int)fl;
    if (i0 >= K) i0 -= K;
    if (i0 < 0) i0 += K;
    if ((unsigned)i0 >= (unsigned)K || !(fr >= 0.0f && fr <= 1.0f)) {  // not a wrapped coordinate
        i0 = 0;
        fr = 0.0f;
    }
    f = fr;
    return i0;
}

__device__ __forceinline__ int wrap_down(int i, int K) { return i < 0 ? i + K : i; }
__device__ __forceinline__ int wrap_mod(int i, int K) { return ((i % K) + K) % K; }

__device__ __forceinline__ long long warp_sum_ll(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums v[0..n) over the block (integers: order independent) and adds the
// block totals to dst[idx[k]] with one atomic each.
template <int NV>
__device__ __forceinline__ void block_flush(long long (&v)[NV], long long *__restrict__ dst, const int (&idx)[NV])
{
    __shared__ long long red[32][NV];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const long long s = warp_sum_ll(v[k]);
        if (lane == 0) red[w][k] = s;
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            long long s = lane < nw ? red[lane][k] : 0;
            s = warp_sum_ll(s);
            if (lane == 0 && s) atomicAdd((unsigned long long *)&dst[idx[k]], (unsigned long long)s);
        }
    }
}

// Step 1.  One block per (x plane p, tile of Ty rows): every atom whose
// stencil reaches the tile (floor(u_x) in [p, p+N-1], floor(u_y) within
// N-1 rows of the tile, periodic) adds q M M M to the tile in shared memory;
// the atoms come from the cell-list columns that cover that x-y range, in
// their sorted order.  Each contribution is a 64-bit fixed-point value
// X = rint(v 2^32) split as X = hi 2^16 + lo with lo = X mod 2^16, and hi and
// lo are summed in separate 32-bit words with 32-bit shared-memory atomics
// (exact and order independent while fewer than 2^13 contributions of
// |v| < 4 reach one point of one tile).  The tile is written to the FFT input as FP32 with
// plain stores.
template <int N>
__global__ void __launch_bounds__(kPmeThreads) k_pme_spread(PmeGeom g, const SysDesc *__restrict__ sysd,
                                                           const int *__restrict__ col_slot,
                                                           const float4 *__restrict__ xyzq, const int *__restrict__ perm,
                                                           const float *__restrict__ q, float *__restrict__ grid,
                                                           long long *__restrict__ acc)
{
    pdl_entry();
    extern __shared__ int tile[];  // [2][Ty][K3]: hi words, then lo words
    __shared__ int s_beg[kColBatch], s_scan[kColBatch + 1];
    __shared__ int2 s_iyz[kPmeThreads];      // hits of one round: grid rows/columns,
    __shared__ float s_qx[kPmeThreads];      // q times the x weight of this plane,
    __shared__ float s_wy[N][kPmeThreads];   // y and z weights
    __shared__ float s_wz[N][kPmeThreads];
    __shared__ int s_nhit;
    const int p = blockIdx.x;
    const int y0 = blockIdx.y * g.Ty;
    const int ty = min(g.Ty, g.K2 - y0);
    const int tn = ty * g.K3;
    int *thi = tile, *tlo = tile + g.Ty * g.K3;
    const SysDesc S = sysd[0];
    for (int i = threadIdx.x; i < tn; i += blockDim.x) {
        thi[i] = 0;
        tlo[i] = 0;
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x < kPmeAcc) acc[threadIdx.x] = 0;
    if (threadIdx.x == 0) s_nhit = 0;
    // columns covering x in [p h, (p+N) h) and y in [y0 h, (y0+ty+N-1) h),
    // widened by 1e-3 A for atoms binned next to a column edge
    const float eps = 1e-3f;
    int cxa = (int)floorf(((float)p * g.h[0] - eps) * S.inv_w[0]);
    int cxb = (int)floorf(((float)(p + N) * g.h[0] + eps) * S.inv_w[0]);
    if (cxb - cxa + 1 >= S.nx) {
        cxa = 0;
        cxb = S.nx - 1;
    }
    int cya = (int)floorf(((float)y0 * g.h[1] - eps) * S.inv_w[1]);
    int cyb = (int)floorf(((float)(y0 + ty + N - 1) * g.h[1] + eps) * S.inv_w[1]);
    if (cyb - cya + 1 >= S.ny) {
        cya = 0;
        cyb = S.ny - 1;
    }
    const int ncx = cxb - cxa + 1, ncol = ncx * (cyb - cya + 1);
    for (int cb = 0; cb < ncol; cb += kColBatch) {
        const int nb = min(kColBatch, ncol - cb);
        __syncthreads();  // tile zeroed / previous batch consumed
        if (threadIdx.x < nb) {
            const int k = cb + threadIdx.x;
            const int cx = wrap_mod(cxa + k % ncx, S.nx), cy = wrap_mod(cya + k / ncx, S.ny);
            const int c = S.col_begin + cy * S.nx + cx;
            s_beg[threadIdx.x] = col_slot[c];
            s_scan[threadIdx.x + 1] = col_slot[c + 1] - col_slot[c];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_scan[0] = 0;
            for (int k = 1; k <= nb; ++k) s_scan[k] += s_scan[k - 1];
        }
        __syncthreads();
        const int total = s_scan[nb];
        // rounds of blockDim.x slots: test each slot's atom against the tile
        // (cheap), compact the hits with their weights, then spread the
        // hits' (y, z) stencil points over the whole block
        for (int base = 0; base < total; base += blockDim.x) {
            const int it = base + threadIdx.x;
            if (it < total) {
                int lo = 0, hi = nb - 1;  // column k with s_scan[k] <= it < s_scan[k+1]
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_scan[mid] <= it) lo = mid;
                    else hi = mid - 1;
                }
                const int slot = s_beg[lo] + it - s_scan[lo];
                const int a = perm[slot];
                if (a >= 0) {
                    const float4 x = xyzq[slot];
                    float fx, fy;
                    const int ix = grid_coord(x.x, g.s_hi[0], g.s_lo[0], g.K1, fx);
                    const int iy = grid_coord(x.y, g.s_hi[1], g.s_lo[1], g.K2, fy);
                    const int jx = wrap_down(ix - p, g.K1);
                    bool hit = jx < N;
                    if (hit) {
                        hit = false;
#pragma unroll
                        for (int jy = 0; jy < N; ++jy) {
                            const int r = wrap_down(iy - jy, g.K2) - y0;
                            hit |= r >= 0 && r < ty;
                        }
                    }
                    if (hit) {
                        float fz, wx[N], wy[N], wz[N], dw[N];
                        const int iz = grid_coord(x.z, g.s_hi[2], g.s_lo[2], g.K3, fz);
                        bspline_weights<N>(fx, wx, dw);
                        bspline_weights<N>(fy, wy, dw);
                        bspline_weights<N>(fz, wz, dw);
                        float wxj = 0.0f;
#pragma unroll
                        for (int j = 0; j < N; ++j)
                            if (j == jx) wxj = wx[j];
                        const int h = atomicAdd(&s_nhit, 1);
                        s_iyz[h] = make_int2(iy, iz);
                        s_qx[h] = q[a] * wxj;
#pragma unroll
                        for (int j = 0; j < N; ++j) {
                            s_wy[j][h] = wy[j];
                            s_wz[j][h] = wz[j];
                        }
                    }
                }
            }
            __syncthreads();
            const int nitem = s_nhit * (N * N);
            for (int k = threadIdx.x; k < nitem; k += blockDim.x) {
                const int h = k / (N * N), t = k - h * (N * N);
                const int jy = t / N, jz = t - jy * N;
                const int2 iyz = s_iyz[h];
                const int r = wrap_down(iyz.x - jy, g.K2) - y0;
                if (r < 0 || r >= ty) continue;
                const float v = s_qx[h] * s_wy[jy][h] * s_wz[jz][h];
                if (v == 0.0f) continue;
                const long long X = __float2ll_rn(v * (float)kGridScale);
                const int z = r * g.K3 + wrap_down(iyz.y - jz, g.K3);
                atomicAdd(&thi[z], (int)(X >> 16));
                atomicAdd(&tlo[z], (int)(X & 0xFFFF));
            }
            __syncthreads();  // the hits are consumed
            if (threadIdx.x == 0) s_nhit = 0;
            __syncthreads();  // the reset is seen before the next round's hits
        }
    }
    __syncthreads();
    float *out = grid + ((long long)p * g.K2 + y0) * g.K3;
    for (int i = threadIdx.x; i < tn; i += blockDim.x)
        out[i] = __ll2float_rn((long long)thi[i] * 65536ll + (long long)(unsigned)tlo[i]) *
                 (float)(1.0 / kGridScale);
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
    long long v[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int k3 = i % g.nk3;
        const int r = i / g.nk3;
        const int k2 = r % g.K2, k1 = r / g.K2;
        const float G = gfac[i];
        float2 z = fq[i];
        if (G != 0.0f) {
            const float wt = (k3 == 0 || 2 * k3 == g.K3) ? 0.5f : 1.0f;
            const float e = wt * G * fmaf(z.x, z.x, z.y * z.y);
            const float mx = (float)(k1 <= g.K1 / 2 ? k1 : k1 - g.K1) * g.inv_L[0];
            const float my = (float)(k2 <= g.K2 / 2 ? k2 : k2 - g.K2) * g.inv_L[1];
            const float mz = (float)k3 * g.inv_L[2];
            const float m2 = fmaf(mz, mz, fmaf(my, my, mx * mx));
            const float c = 2.0f * fmaf(pi2_over_a2, m2, 1.0f) / m2;
            const float ec = e * c;
            const float vs = (float)kVirScale;
            v[0] += __float2ll_rn(e * (float)kFixScale);
            v[1] += __float2ll_rn((e - ec * mx * mx) * vs);
            v[2] += __float2ll_rn((e - ec * my * my) * vs);
            v[3] += __float2ll_rn((e - ec * mz * mz) * vs);
            v[4] += __float2ll_rn(-ec * mx * my * vs);
            v[5] += __float2ll_rn(-ec * mx * mz * vs);
            v[6] += __float2ll_rn(-ec * my * mz * vs);
        }
        z.x *= G;
        z.y *= G;
        fq[i] = z;
    }
    const int idx[7] = {0, 3, 4, 5, 6, 7, 8};
    block_flush<7>(v, acc, idx);
}

// Step 5 and the corrections.  A group of G lanes per atom (sorted slot
// order, so the grid reads of neighbouring atoms overlap in cache): the
// lanes share the N x N (x, y) offsets of the atom's stencil, each summing
// the N grid points along z of its offsets; they also share the atom's
// exclusion / 1-4 partners j, whose correction force on the atom they add
// (every pair is evaluated from both sides, so no atomics are needed), and
// the pair's energy and virial are counted from the side with the smaller
// index.  FP32 pair arithmetic with the FP32 minimum image of the sorted
// (wrapped) coordinates.  The group's force goes to the slot's fixed-point
// sum with plain stores; the atom's q^2 to the self-energy sum.  The
// caller's coordinates are checked against those of the last build.
template <int N>
struct GatherLanes {
    static constexpr int G = N <= 4 ? 4 : 8;
};

template <int N>
__global__ void __launch_bounds__(256) k_pme_gather(PmeGeom g, PmeCorr cc, int slot_cap, const int *__restrict__ counts,
                                                   const int *__restrict__ perm, const int *__restrict__ inv,
                                                   const float4 *__restrict__ xyzq, const float *__restrict__ pos,
                                                   const float *__restrict__ q, const float *__restrict__ theta,
                                                   const int *__restrict__ part, int K, int sums, long long *__restrict__ pacc,
                                                   long long *__restrict__ acc, int *__restrict__ status)
{
    pdl_entry();
    constexpr int G = GatherLanes<N>::G;
    const int gl = threadIdx.x & (G - 1);
    const int nslots = min(slot_cap, counts[0]);
    const int groups = gridDim.x * (blockDim.x / G);
    long long v[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // sum q^2, E_excl, W[6]
    const int last = (nslots + groups - 1) / groups * groups;  // every group runs the same trip count
    for (int s = (blockIdx.x * blockDim.x + threadIdx.x) / G; s < last; s += groups) {
        const int a = s < nslots ? perm[s] : -1;
        float fx = 0.0f, fy = 0.0f, fz = 0.0f;
        if (a >= 0) {
            const float4 xa = xyzq[s];
            const float qa = q[a];
            if (gl == 0) {
                const float px = wrap_coord(pos[3ll * a], cc.L[0]), py = wrap_coord(pos[3ll * a + 1], cc.L[1]),
                            pz = wrap_coord(pos[3ll * a + 2], cc.L[2]);
                if (px != xa.x || py != xa.y || pz != xa.z) atomicOr(status, ST_STALE);
                // q^2 exactly: hi + lo from an FMA, each to fixed point
                const float q2 = qa * qa, q2l = fmaf(qa, qa, -q2);
                v[0] += __float2ll_rn(q2 * (float)kQ2Scale) + __float2ll_rn(q2l * (float)kQ2Scale);
            }
            if (qa != 0.0f) {
                float f, wx[N], dwx[N], wy[N], dwy[N], wz[N], dwz[N];
                const int ix = grid_coord(xa.x, g.s_hi[0], g.s_lo[0], g.K1, f);
                bspline_weights<N>(f, wx, dwx);
                const int iy = grid_coord(xa.y, g.s_hi[1], g.s_lo[1], g.K2, f);
                bspline_weights<N>(f, wy, dwy);
                const int iz = grid_coord(xa.z, g.s_hi[2], g.s_lo[2], g.K3, f);
                bspline_weights<N>(f, wz, dwz);
                float sx = 0.0f, sy = 0.0f, sz = 0.0f;
                for (int t = gl; t < N * N; t += G) {
                    const int jx = t / N, jy = t - jx * N;
                    float wxj = 0.0f, dwxj = 0.0f, wyj = 0.0f, dwyj = 0.0f;
#pragma unroll
                    for (int j = 0; j < N; ++j) {
                        if (j == jx) {
                            wxj = wx[j];
                            dwxj = dwx[j];
                        }
                        if (j == jy) {
                            wyj = wy[j];
                            dwyj = dwy[j];
                        }
                    }
                    const float *row = theta + ((long long)wrap_down(ix - jx, g.K1) * g.K2 + wrap_down(iy - jy, g.K2)) *
                                                   g.K3;
                    float th[N];
#pragma unroll
                    for (int jz = 0; jz < N; ++jz) th[jz] = __ldg(&row[wrap_down(iz - jz, g.K3)]);
                    float tz = 0.0f, tdz = 0.0f;
#pragma unroll
                    for (int jz = 0; jz < N; ++jz) {
                        tz = fmaf(wz[jz], th[jz], tz);
                        tdz = fmaf(dwz[jz], th[jz], tdz);
                    }
                    sx = fmaf(dwxj * wyj, tz, sx);
                    sy = fmaf(wxj * dwyj, tz, sy);
                    sz = fmaf(wxj * wyj, tdz, sz);
                }
                fx = -qa * g.fscale[0] * sx;
                fy = -qa * g.fscale[1] * sy;
                fz = -qa * g.fscale[2] * sz;
                for (int k = gl; k < K; k += G) {
                    const int pp = part[(long long)a * K + k];
                    if (pp < 0) continue;
                    const int j = pp >> 1;
                    const float wgt = (pp & 1) ? cc.one_m_s14 : 1.0f;
                    const float qq = wgt * cc.ke * qa * q[j];
                    if (qq == 0.0f) continue;
                    const float4 xj = xyzq[inv[j]];
                    float d[3] = {xa.x - xj.x, xa.y - xj.y, xa.z - xj.z};
                    float sh[3] = {0.0f, 0.0f, 0.0f};  // image shift of each axis: -1, 0, +1 box
#pragma unroll
                    for (int ax = 0; ax < 3; ++ax) {
                        if (d[ax] > cc.half[ax]) {
                            d[ax] -= cc.L[ax];
                            sh[ax] = -1.0f;
                        } else if (d[ax] < -cc.half[ax]) {
                            d[ax] += cc.L[ax];
                            sh[ax] = 1.0f;
                        }
                    }
                    const float r2 = fmaf(d[2], d[2], fmaf(d[1], d[1], d[0] * d[0]));
                    // U = -qq erf(a r)/r; force on the atom = -dU/dr d/r = -qq g(a r) / r^3 d
                    float fs;
                    const float x2 = cc.alpha * cc.alpha * r2;
                    if (x2 < 1.0f) {
                        float P = cc.series[kSeriesTerms - 1];
#pragma unroll
                        for (int t = kSeriesTerms - 2; t >= 0; --t) P = fmaf(P, x2, cc.series[t]);
                        fs = -qq * cc.two_a3_sqpi * P;
                    } else {
                        const float r = sqrtf(r2), ir = 1.0f / r;
                        const float er = erff(cc.alpha * r);
                        fs = qq * (cc.two_a_sqpi * expf(-x2) * r - er) * (ir * ir * ir);
                    }
                    const float f0 = fs * d[0], f1 = fs * d[1], f2 = fs * d[2];
                    fx += f0;
                    fy += f1;
                    fz += f2;
                    if (sums && j > a) {
                        // The pair's energy -qq erf(alpha r)/r = -qq alpha erf(x)/x,
                        // x^2 = alpha^2 r^2, in double-FP32 arithmetic from the exact
                        // displacement of the FP32 inputs: these corrections sum to
                        // about 80 times the total Coulomb energy (they cancel the
                        // self term), and the rigid waters repeat the same distances,
                        // so FP32 rounding would add up coherently (2.7e-8 of the
                        // sum, 2e-6 of the total on the solvated chain).  Partners
                        // beyond 2 / alpha (where the series needs more terms) take
                        // FP64, which is slow on this GPU but rare.
                        DF r2df = {0.0f, 0.0f};
                        double dd[3];
#pragma unroll
                        for (int ax = 0; ax < 3; ++ax) {
                            const float xi = ax == 0 ? xa.x : (ax == 1 ? xa.y : xa.z);
                            const float xo = ax == 0 ? xj.x : (ax == 1 ? xj.y : xj.z);
                            DF da = df_two_sum(xi, -xo);  // exact
                            if (sh[ax] != 0.0f) da = df_add(da, DF{sh[ax] * cc.L[ax], 0.0f});
                            r2df = df_add(r2df, df_mul(da, da));
                            dd[ax] = (double)da.hi + (double)da.lo;
                        }
                        const DF x2 = df_mul(DF{cc.a2.x, cc.a2.y}, r2df);
                        DF kq = df_mul_f(df_mul_f(df_mul_f(DF{cc.ke, 0.0f}, qa), q[j]), wgt);
                        kq = df_mul_f(kq, cc.alpha);
                        double ed;
                        if (x2.hi <= 4.0f) {
                            DF S = {cc.erfx[kErfxTerms - 1].x, cc.erfx[kErfxTerms - 1].y};
#pragma unroll 1
                            for (int t = kErfxTerms - 2; t >= 0; --t)
                                S = df_add(df_mul(S, x2), DF{cc.erfx[t].x, cc.erfx[t].y});
                            const DF e = df_mul(kq, S);
                            ed = -((double)e.hi + (double)e.lo);
                        } else {
                            const double rd = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
                            const double qqd = (double)wgt * (double)cc.ke * (double)qa * (double)q[j];
                            ed = -qqd * erf((double)cc.alpha * rd) / rd;
                        }
                        const float vs = (float)kVirScale;
                        v[1] += __double2ll_rn(ed * kFixScale);
                        v[2] += __float2ll_rn(d[0] * f0 * vs);
                        v[3] += __float2ll_rn(d[1] * f1 * vs);
                        v[4] += __float2ll_rn(d[2] * f2 * vs);
                        v[5] += __float2ll_rn(d[0] * f1 * vs);
                        v[6] += __float2ll_rn(d[0] * f2 * vs);
                        v[7] += __float2ll_rn(d[1] * f2 * vs);
                    }
                }
            }
        }
#pragma unroll
        for (int o = 1; o < G; o <<= 1) {
            fx += __shfl_xor_sync(0xffffffffu, fx, o);
            fy += __shfl_xor_sync(0xffffffffu, fy, o);
            fz += __shfl_xor_sync(0xffffffffu, fz, o);
        }
        if (gl == 0 && s < nslots) {
            const float sc = (float)kFixScale;
            pacc[3ll * s] = __float2ll_rn(fx * sc);
            pacc[3ll * s + 1] = __float2ll_rn(fy * sc);
            pacc[3ll * s + 2] = __float2ll_rn(fz * sc);
        }
    }
    const int idx[8] = {1, 2, 3, 4, 5, 6, 7, 8};
    block_flush<8>(v, acc, idx);
}

// Fixed-point sums of the stand-alone evaluation to the caller's outputs.
__global__ void k_pme_finalize(int slot_cap, const int *__restrict__ counts, const int *__restrict__ perm,
                               const long long *__restrict__ pacc, const long long *__restrict__ acc, double self_coef,
                               float *__restrict__ F, double *__restrict__ energy, double *__restrict__ virial)
{
    pdl_entry();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const float sc = 2.3283064365386963e-10f;  // 2^-32
    if (s < slot_cap && s < counts[0]) {
        const int a = perm[s];
        if (a >= 0) {
            F[3ll * a] = __ll2float_rn(pacc[3ll * s]) * sc;
            F[3ll * a + 1] = __ll2float_rn(pacc[3ll * s + 1]) * sc;
            F[3ll * a + 2] = __ll2float_rn(pacc[3ll * s + 2]) * sc;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x < kPmeAcc) {
        const int k = threadIdx.x;
        if (k < 3) {
            const double v = k == 1 ? self_coef * ((double)acc[1] / kQ2Scale) : (double)acc[k] / kFixScale;
            if (energy) energy[k] = v;
        } else if (virial) {
            virial[k - 3] = (double)acc[k] / kVirScale;
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
    if (p->side) {
        cudaStreamSynchronize(p->side);
        cudaStreamDestroy(p->side);
    }
    if (p->fork) cudaEventDestroy(p->fork);
    if (p->join) cudaEventDestroy(p->join);
    if (p->lists) cudaEventDestroy(p->lists);
    void *ptrs[] = {p->grid, p->fq, p->gfac, p->pacc, p->acc};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    delete p;
    ctx->pme = nullptr;
}

const long long *pme_forces_acc(const nb_ctx *ctx) { return ctx->pme ? ctx->pme->pacc : nullptr; }
const long long *pme_sums_acc(const nb_ctx *ctx) { return ctx->pme ? ctx->pme->acc : nullptr; }
double pme_self_coef(const nb_ctx *ctx) { return ctx->pme ? ctx->pme->self_coef : 0.0; }

template <int N>
static cudaError_t launch_pme_t(nb_ctx *ctx, cudaStream_t st, const float *d_pos, const float *d_q, bool sums)
{
    PmeState &P = *ctx->pme;
    const PmeGeom &g = P.g;
    auto &d = ctx->d;
    const dim3 sgrid(g.K1, (g.K2 + g.Ty - 1) / g.Ty);
    const size_t smem = 2 * sizeof(int) * g.Ty * g.K3;
    cudaError_t e = launch_pdl(k_pme_spread<N>, sgrid, dim3(kPmeThreads), smem, st, g, (const SysDesc *)d.sys,
                               (const int *)d.col_slot, (const float4 *)d.xyzq, (const int *)d.perm, d_q, P.grid, P.acc);
    if (e != cudaSuccess) return e;
    if (cufftSetStream(P.fwd, st) != CUFFT_SUCCESS || cufftExecR2C(P.fwd, P.grid, (cufftComplex *)P.fq) != CUFFT_SUCCESS)
        return cudaErrorUnknown;
    const int half = g.K1 * g.K2 * g.nk3;
    const float a = ctx->pp.alpha;
    const float pi2_over_a2 = (float)(M_PI * M_PI / ((double)a * (double)a));
    const int sb = std::max(1, std::min((half + 255) / 256, 2 * ctx->num_sms));
    e = launch_pdl(k_pme_solve, dim3(sb), dim3(256), 0, st, half, g, pi2_over_a2, (const float *)P.gfac, P.fq, P.acc);
    if (e != cudaSuccess) return e;
    if (cufftSetStream(P.inv, st) != CUFFT_SUCCESS || cufftExecC2R(P.inv, (cufftComplex *)P.fq, P.grid) != CUFFT_SUCCESS)
        return cudaErrorUnknown;
    constexpr int G = GatherLanes<N>::G;
    const int S = (int)ctx->slot_cap;
    const int gt = 256;
    const int gb = std::max(1, std::min((S * G + gt - 1) / gt, 16 * ctx->num_sms));
    return launch_pdl(k_pme_gather<N>, dim3(gb), dim3(gt), 0, st, g, P.c, S, (const int *)d.counts,
                      (const int *)d.perm, (const int *)d.inv, (const float4 *)d.xyzq, d_pos, d_q,
                      (const float *)P.grid, (const int *)d.part_orig, ctx->K, sums ? 1 : 0, P.pacc, P.acc, d.status);
}

static cudaError_t launch_pme_on(nb_ctx *ctx, cudaStream_t st, const float *d_pos, const float *d_q, bool sums)
{
    switch (ctx->pme->order) {
    case 4: return launch_pme_t<4>(ctx, st, d_pos, d_q, sums);
    case 6: return launch_pme_t<6>(ctx, st, d_pos, d_q, sums);
    case 8: return launch_pme_t<8>(ctx, st, d_pos, d_q, sums);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_pme(nb_ctx *ctx, const float *d_pos, const float *d_q)
{
    return launch_pme_on(ctx, ctx->stream, d_pos, d_q, true);
}

cudaError_t launch_pme_fork(nb_ctx *ctx, const float *d_pos, const float *d_q, bool sums,
                            cudaError_t (*side_first)(nb_ctx *, cudaStream_t, const float *))
{
    PmeState &P = *ctx->pme;
    cudaError_t e = cudaEventRecord(P.fork, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P.side, P.fork, 0);
    if (e == cudaSuccess && side_first) e = side_first(ctx, P.side, d_pos);
    if (e == cudaSuccess) e = launch_pme_on(ctx, P.side, d_pos, d_q, sums);
    if (e == cudaSuccess) e = cudaEventRecord(P.join, P.side);
    return e;
}

cudaStream_t pme_side_stream(const nb_ctx *ctx) { return ctx->pme->side; }

cudaError_t pme_side_after_lists(nb_ctx *ctx)
{
    PmeState &P = *ctx->pme;
    cudaError_t e = cudaEventRecord(P.lists, ctx->stream);
    return e == cudaSuccess ? cudaStreamWaitEvent(P.side, P.lists, 0) : e;
}

cudaError_t pme_side_rejoin(nb_ctx *ctx) { return cudaEventRecord(ctx->pme->join, ctx->pme->side); }

cudaError_t launch_pme_join(nb_ctx *ctx)
{
    return cudaStreamWaitEvent(ctx->stream, ctx->pme->join, 0);
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
    double Ld[3];
    PmeGeom &g = P->g;
    g.K1 = K1;
    g.K2 = K2;
    g.K3 = K3;
    g.nk3 = nk3;
    g.Ty = std::max(1, std::min(K2, kTileElems / K3));
    for (int a = 0; a < 3; ++a) {
        Ld[a] = (double)Lf[a];
        const double sc = (double)P->K[a] / Ld[a];
        g.s_hi[a] = (float)sc;
        g.s_lo[a] = (float)(sc - (double)g.s_hi[a]);
        g.h[a] = (float)(Ld[a] / (double)P->K[a]);
        g.fscale[a] = (float)sc;
        g.inv_L[a] = (float)(1.0 / Ld[a]);
    }
    const double alpha = (double)ctx->pp.alpha, ke = (double)ctx->pp.ke;
    PmeCorr &cc = P->c;
    cc.ke = ctx->pp.ke;
    cc.alpha = ctx->pp.alpha;
    cc.one_m_s14 = (float)(1.0 - (double)ctx->pp.s14_c);
    cc.two_a_sqpi = (float)(2.0 * alpha / sqrt(M_PI));
    cc.two_a3_sqpi = (float)(2.0 * alpha * alpha * alpha / sqrt(M_PI));
    {
        double fact = 1.0;  // (n+1)!
        for (int n = 0; n < kSeriesTerms; ++n) {
            fact *= (double)(n + 1);
            cc.series[n] = (float)((n % 2 ? -2.0 : 2.0) * (double)(n + 1) / ((double)(2 * n + 3) * fact));
        }
    }
    {
        double fact = 1.0;  // n!
        for (int n = 0; n < kErfxTerms; ++n) {
            if (n > 0) fact *= (double)n;
            const double c = (n % 2 ? -2.0 : 2.0) / (sqrt(M_PI) * fact * (double)(2 * n + 1));
            const float hi = (float)c;
            cc.erfx[n] = make_float2(hi, (float)(c - (double)hi));
        }
        const double a2 = (double)ctx->pp.alpha * (double)ctx->pp.alpha;  // exact: 24-bit alpha squared
        cc.a2 = make_float2((float)a2, (float)(a2 - (double)(float)a2));
    }
    for (int a = 0; a < 3; ++a) {
        cc.L[a] = Lf[a];
        cc.half[a] = ctx->sys_h[0].half[a];
    }
    P->self_coef = -ke * alpha / sqrt(M_PI);
    const size_t total = (size_t)K1 * K2 * K3, half = (size_t)K1 * K2 * nk3;
    cudaError_t e = cudaMalloc(&P->grid, sizeof(float) * total);
    if (e == cudaSuccess) e = cudaMalloc(&P->fq, sizeof(float2) * half);
    if (e == cudaSuccess) e = cudaMalloc(&P->gfac, sizeof(float) * half);
    if (e == cudaSuccess) e = cudaMalloc(&P->pacc, sizeof(long long) * 3 * std::max<int64_t>(ctx->slot_cap, 1));
    if (e == cudaSuccess) e = cudaMalloc(&P->acc, sizeof(long long) * kPmeAcc);
    if (e == cudaSuccess) e = cudaMemset(P->acc, 0, sizeof(long long) * kPmeAcc);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->lists, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        pme_free(ctx);
        return e == cudaErrorMemoryAllocation ? NB_ERR_OOM : NB_ERR_CUDA;
    }
    // influence function G(m) = ke B(m) C(m) on the half spectrum, FP64 on the host
    const double V = Ld[0] * Ld[1] * Ld[2];
    const std::vector<double> b1 = bspline_moduli(K1, P->order), b2 = bspline_moduli(K2, P->order),
                              b3 = bspline_moduli(K3, P->order);
    std::vector<float> G(half);
    for (int k1 = 0; k1 < K1; ++k1)
        for (int k2 = 0; k2 < K2; ++k2)
            for (int k3 = 0; k3 < nk3; ++k3) {
                const double mx = (double)(k1 <= K1 / 2 ? k1 : k1 - K1) / Ld[0];
                const double my = (double)(k2 <= K2 / 2 ? k2 : k2 - K2) / Ld[1];
                const double mz = (double)k3 / Ld[2];
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
    if (!ctx->pme || !ctx->built) return NB_ERR_NOT_BUILT;
    cudaError_t e = launch_pme(ctx, d_pos, d_q);
    if (e != cudaSuccess) return NB_ERR_CUDA;
    const int S = (int)ctx->slot_cap;
    e = launch_pdl(k_pme_finalize, dim3((S + 255) / 256), dim3(256), 0, ctx->stream, S, (const int *)ctx->d.counts,
                   (const int *)ctx->d.perm, (const long long *)ctx->pme->pacc, (const long long *)ctx->pme->acc,
                   ctx->pme->self_coef, d_F, d_energy, d_virial);
    return e == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}
