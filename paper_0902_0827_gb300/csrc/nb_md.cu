// nb_md.cu - the molecular-dynamics step around the non-bonded path
// (section "Molecular dynamics on the GPU": bonded force terms,
// velocity-Verlet integration, Langevin thermostat, M-SHAKE and RATTLE
// constraints; section "Performance": the DHFR step with PME).
//
// One step of length dt from (x, v, F(x)); one lane per unconstrained atom,
// three per rigid water (one per atom, the constraints solved on all three):
//   k_md_first   O: v <- c v + sigma xi (c = exp(-gamma dt/2),
//                sigma = sqrt((1 - c^2) kT / m)), B: v += dt/2 F/m,
//                A: x' = x + dt v; waters then M-SHAKE (Newton on the 3
//                distance equations with the reference bond vectors of x):
//                x'' = x' + disp and v += disp / dt
//   cell list, short-range forces (+ PME), k_md_bonded
//   k_md_second  reads the short-range (+ PME) forces from their
//                fixed-point sums (no unpack kernel), B: v += dt/2 F/m,
//                O: v <- c v + sigma xi'; waters then RATTLE
//                (r_k . (v_a - v_b) = 0); kinetic energy; the last block
//                writes the energies and advances the step counter
// xi: Philox4x32-10 (Salmon et al. 2011) on the counter (atom, step,
// stream, 0) and key (seed), 24-bit uniforms, Box-Muller.  Units kcal/mol,
// A, amu, ps: F/m in kcal/mol/A/amu times 418.4 is A/ps^2.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "nb_internal.cuh"

namespace acenb {

constexpr float kAccel = 418.4f;          // (A/ps)^2 per kcal/mol/amu
constexpr double kBoltzmann = 0.0019872041;  // kcal/mol/K
constexpr int kMdAcc = 8;                  // E_bond, E_angle, E_dihedral, E_kin (2^32), spare, ticket
constexpr int kMdTicket = 7;               // blocks of the second half-step done

struct MdState {
    int n = 0, nb = 0, na = 0, nd = 0, nw = 0;
    float dt = 0.0f, c = 1.0f;             // O-step factor exp(-gamma dt / 2)
    bool langevin = false;
    unsigned long long seed = 0;
    int shake_iter = 10;
    float shake_tol = 1e-6f;
    float d2[2] = {0.0f, 0.0f};            // (r_OH)^2, (r_HH)^2
    bool have_forces = false;
    // device
    float *mass = nullptr;                 // [N]
    float *sigv = nullptr;                 // [N] sqrt((1 - c^2) kT 418.4 / m)
    int *free_atoms = nullptr;             // [n_free] atoms in no water (one integration thread each)
    int n_free = 0;
    int2 *bonds = nullptr;                 // [nb]
    float2 *bond_p = nullptr;              // (k, r0)
    int4 *angles = nullptr;                // [na] (i, j, k, -)
    float2 *angle_p = nullptr;             // (k, theta0)
    int4 *dihedrals = nullptr;             // [nd]
    float4 *dihedral_p = nullptr;          // (k, n, delta, -)
    int4 *waters = nullptr;                // [nw] (O, H1, H2, -)
    float *Fnb = nullptr;                  // [N*3] short-range (+ PME) forces of the last evaluation
    float *Ftot = nullptr;                 // [N*3] total forces at the current positions
    long long *bacc = nullptr;             // [N*3] bonded forces, fixed point 2^32
    double *enb = nullptr;                 // [2] E_LJ, E_Coul of the last evaluation
    long long *acc = nullptr;              // [kMdAcc]
    unsigned long long *step = nullptr;    // [1] device step counter
    unsigned *amax = nullptr;              // [2] minimisation: largest |F_i| / m_i (float bits), two slots
    cudaStream_t bside = nullptr;          // the bonded terms' stream beside the short-range path (with PME)
    cudaEvent_t bfork = nullptr, bjoin = nullptr;
};

// ------------------------------------------------------------------ Philox

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Three standard normals for (atom, step, stream): 24-bit uniforms
// u = ((x >> 8) + 1/2) 2^-24 (exact in FP32), Box-Muller on (u0, u1), (u2, u3).
__device__ __forceinline__ float3 md_normals(unsigned atom, unsigned long long step, unsigned stream,
                                             unsigned long long seed)
{
    uint32_t c[4] = {atom, (uint32_t)step, stream, 0u};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    float u[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) u[k] = ((float)(c[k] >> 8) + 0.5f) * 5.9604644775390625e-8f;  // 2^-24
    const float r0 = sqrtf(-2.0f * logf(u[0])), r1 = sqrtf(-2.0f * logf(u[2]));
    float s0, c0, s1, c1;
    sincospif(2.0f * u[1], &s0, &c0);
    sincospif(2.0f * u[3], &s1, &c1);
    return make_float3(r0 * c0, r0 * s0, r1 * c1);
}

__device__ __forceinline__ float min_img(float d, float L, float h)
{
    return d > h ? d - L : (d < -h ? d + L : d);
}

__device__ __forceinline__ long long warp_sum64(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block sum of NV fixed-point values added to dst[idx[k]].
template <int NV>
__device__ __forceinline__ void md_flush(long long (&v)[NV], long long *__restrict__ dst, const int (&idx)[NV])
{
    __shared__ long long red[32][NV];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const long long s = warp_sum64(v[k]);
        if (lane == 0) red[w][k] = s;
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            long long s = lane < nw ? red[lane][k] : 0;
            s = warp_sum64(s);
            if (lane == 0 && s) atomicAdd((unsigned long long *)&dst[idx[k]], (unsigned long long)s);
        }
    }
}

__device__ __forceinline__ void add_force(long long *__restrict__ bacc, int a, float fx, float fy, float fz)
{
    const float sc = 4294967296.0f;
    atomicAdd((unsigned long long *)&bacc[3ll * a], (unsigned long long)__float2ll_rn(fx * sc));
    atomicAdd((unsigned long long *)&bacc[3ll * a + 1], (unsigned long long)__float2ll_rn(fy * sc));
    atomicAdd((unsigned long long *)&bacc[3ll * a + 2], (unsigned long long)__float2ll_rn(fz * sc));
}

struct Box3 {
    float L[3], h[3];
};

__device__ __forceinline__ float3 disp(const float *__restrict__ x, int from, int to, const Box3 &B)
{
    return make_float3(min_img(x[3ll * to] - x[3ll * from], B.L[0], B.h[0]),
                       min_img(x[3ll * to + 1] - x[3ll * from + 1], B.L[1], B.h[1]),
                       min_img(x[3ll * to + 2] - x[3ll * from + 2], B.L[2], B.h[2]));
}

__device__ __forceinline__ float dot3(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 cross3(float3 a, float3 b)
{
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 scale3(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float3 add3(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }

// Bonded terms, one thread per term (bonds, then angles, then dihedrals):
// U = k (r - r0)^2; U = k (theta - theta0)^2 with theta = atan2(|a x b|, a . b);
// U = k (1 + cos(n phi - delta)) with the IUPAC phi = atan2(|b2| b1 . n2, n1 . n2).
// Forces to the fixed-point sums (2^32), energies to acc[0..2].
__global__ void __launch_bounds__(256) k_md_bonded(int nb, int na, int nd, const int2 *__restrict__ bonds,
                                                   const float2 *__restrict__ bond_p, const int4 *__restrict__ angles,
                                                   const float2 *__restrict__ angle_p, const int4 *__restrict__ dih,
                                                   const float4 *__restrict__ dih_p, const float *__restrict__ x,
                                                   Box3 B, long long *__restrict__ bacc, long long *__restrict__ acc)
{
    pdl_entry();
    long long v[3] = {0, 0, 0};
    const float es = 4294967296.0f;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nb + na + nd; t += gridDim.x * blockDim.x) {
        if (t < nb) {
            const int2 ij = bonds[t];
            const float2 p = bond_p[t];
            const float3 d = disp(x, ij.x, ij.y, B);
            const float r = sqrtf(dot3(d, d));
            const float dr = r - p.y;
            v[0] += __float2ll_rn(p.x * dr * dr * es);
            const float f = 2.0f * p.x * dr / r;  // force on i along d
            add_force(bacc, ij.x, f * d.x, f * d.y, f * d.z);
            add_force(bacc, ij.y, -f * d.x, -f * d.y, -f * d.z);
        } else if (t < nb + na) {
            const int u = t - nb;
            const int4 q = angles[u];
            const float2 p = angle_p[u];
            const float3 a = disp(x, q.y, q.x, B), b = disp(x, q.y, q.z, B);
            const float la = sqrtf(dot3(a, a)), lb = sqrtf(dot3(b, b));
            const float s = sqrtf(dot3(cross3(a, b), cross3(a, b))), c = dot3(a, b);
            const float th = atan2f(s, c);
            const float dth = th - p.y;
            v[1] += __float2ll_rn(p.x * dth * dth * es);
            const float dU = 2.0f * p.x * dth;
            const float inv = 1.0f / (la * lb);
            const float cs = c * inv, sn = fmaxf(s * inv, 1e-6f);
            const float3 ah = scale3(1.0f / la, a), bh = scale3(1.0f / lb, b);
            // F_i = -dU dtheta/da, dtheta/da = (cos a^ - b^) / (|a| sin)
            const float3 fi = scale3(-dU / (la * sn), add3(scale3(cs, ah), scale3(-1.0f, bh)));
            const float3 fk = scale3(-dU / (lb * sn), add3(scale3(cs, bh), scale3(-1.0f, ah)));
            add_force(bacc, q.x, fi.x, fi.y, fi.z);
            add_force(bacc, q.z, fk.x, fk.y, fk.z);
            add_force(bacc, q.y, -fi.x - fk.x, -fi.y - fk.y, -fi.z - fk.z);
        } else {
            const int u = t - nb - na;
            const int4 q = dih[u];
            const float4 p = dih_p[u];
            const float3 b1 = disp(x, q.x, q.y, B), b2 = disp(x, q.y, q.z, B), b3 = disp(x, q.z, q.w, B);
            const float3 n1 = cross3(b1, b2), n2 = cross3(b2, b3);
            const float lb2 = sqrtf(dot3(b2, b2));
            const float phi = atan2f(lb2 * dot3(b1, n2), dot3(n1, n2));
            const float arg = p.y * phi - p.z;
            float sa, ca;
            sincosf(arg, &sa, &ca);
            v[2] += __float2ll_rn(p.x * (1.0f + ca) * es);
            const float dU = -p.x * p.y * sa;
            const float n1s = fmaxf(dot3(n1, n1), 1e-12f), n2s = fmaxf(dot3(n2, n2), 1e-12f);
            // dphi/dx: i -(|b2|/|n1|^2) n1, l (|b2|/|n2|^2) n2,
            // j -(1 + p1) g_i + p3 g_l, k -(1 + p3) g_l + p1 g_i
            const float3 gi = scale3(-lb2 / n1s, n1), gl = scale3(lb2 / n2s, n2);
            const float ib2 = 1.0f / (lb2 * lb2);
            const float p1 = dot3(b1, b2) * ib2, p3 = dot3(b3, b2) * ib2;
            const float3 gj = add3(scale3(-(1.0f + p1), gi), scale3(p3, gl));
            const float3 gk = add3(scale3(-(1.0f + p3), gl), scale3(p1, gi));
            add_force(bacc, q.x, -dU * gi.x, -dU * gi.y, -dU * gi.z);
            add_force(bacc, q.y, -dU * gj.x, -dU * gj.y, -dU * gj.z);
            add_force(bacc, q.z, -dU * gk.x, -dU * gk.y, -dU * gk.z);
            add_force(bacc, q.w, -dU * gl.x, -dU * gl.y, -dU * gl.z);
        }
    }
    const int idx[3] = {0, 1, 2};
    md_flush<3>(v, acc, idx);
}

// The short-range (+ PME) forces of atom a straight from the fixed-point
// sums in sorted order, converted as the unpack kernel converts them (the
// same bits): the MD step reads them here instead of running the unpack.
struct NbSums {
    const int *inv;           // atom -> sorted slot
    const long long *facc;    // [S*3] short-range sums (2^32)
    const long long *pme_f;   // [S*3] PME sums, or null
};

__device__ __forceinline__ float3 nb_force_of(const NbSums &N, int a)
{
    const float sc = 2.3283064365386963e-10f;  // 2^-32
    const long long s = N.inv[a];
    const long long p0 = N.pme_f ? N.pme_f[3 * s] : 0, p1 = N.pme_f ? N.pme_f[3 * s + 1] : 0,
                    p2 = N.pme_f ? N.pme_f[3 * s + 2] : 0;
    return make_float3(__ll2float_rn(N.facc[3 * s] + p0) * sc, __ll2float_rn(N.facc[3 * s + 1] + p1) * sc,
                       __ll2float_rn(N.facc[3 * s + 2] + p2) * sc);
}

// Total forces F = F_short + bonded (the fixed-point bonded sums are cleared).
__device__ __forceinline__ void collect_force(int a, const float *__restrict__ Fnb, long long *__restrict__ bacc,
                                              float *__restrict__ Ftot, float &fx, float &fy, float &fz)
{
    const float sc = 2.3283064365386963e-10f;  // 2^-32
    fx = Fnb[3ll * a] + __ll2float_rn(bacc[3ll * a]) * sc;
    fy = Fnb[3ll * a + 1] + __ll2float_rn(bacc[3ll * a + 1]) * sc;
    fz = Fnb[3ll * a + 2] + __ll2float_rn(bacc[3ll * a + 2]) * sc;
    bacc[3ll * a] = 0;
    bacc[3ll * a + 1] = 0;
    bacc[3ll * a + 2] = 0;
    Ftot[3ll * a] = fx;
    Ftot[3ll * a + 1] = fy;
    Ftot[3ll * a + 2] = fz;
}

__global__ void k_md_collect(int n, const float *__restrict__ Fnb, long long *__restrict__ bacc,
                             float *__restrict__ Ftot)
{
    pdl_entry();
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    float fx, fy, fz;
    collect_force(a, Fnb, bacc, Ftot, fx, fy, fz);
}

// O (stream 0), B, A of atom a: returns x' = x + dt v (v updated in place).
__device__ __forceinline__ float3 kick_drift(int a, float dt, float c, bool langevin, unsigned long long seed,
                                             unsigned long long step, const float *__restrict__ mass,
                                             const float *__restrict__ sigv, const float *__restrict__ Ftot,
                                             const float *__restrict__ x, float *__restrict__ v)
{
    // every load is issued first and the noise computed while they are in flight
    float vx = v[3ll * a], vy = v[3ll * a + 1], vz = v[3ll * a + 2];
    const float sa = langevin ? sigv[a] : 0.0f, ma = mass[a];
    const float f0 = Ftot[3ll * a], f1 = Ftot[3ll * a + 1], f2 = Ftot[3ll * a + 2];
    const float x0 = x[3ll * a], x1 = x[3ll * a + 1], x2 = x[3ll * a + 2];
    if (langevin) {
        const float3 xi = md_normals((unsigned)a, step, 0u, seed);
        vx = fmaf(c, vx, sa * xi.x);
        vy = fmaf(c, vy, sa * xi.y);
        vz = fmaf(c, vz, sa * xi.z);
    }
    const float h = 0.5f * dt * kAccel / ma;
    vx = fmaf(h, f0, vx);
    vy = fmaf(h, f1, vy);
    vz = fmaf(h, f2, vz);
    v[3ll * a] = vx;
    v[3ll * a + 1] = vy;
    v[3ll * a + 2] = vz;
    return make_float3(fmaf(dt, vx, x0), fmaf(dt, vy, x1), fmaf(dt, vz, x2));
}

// B and O (stream 1) of atom a with the new forces (v updated in place).
__device__ __forceinline__ float3 kick(int a, float dt, float c, bool langevin, unsigned long long seed,
                                       unsigned long long step, const float *__restrict__ mass,
                                       const float *__restrict__ sigv, const NbSums &Nb,
                                       long long *__restrict__ bacc, float *__restrict__ Ftot, float *__restrict__ v)
{
    const float sc = 2.3283064365386963e-10f;  // 2^-32
    // every load is issued first and the noise (integer and special-function
    // work that needs none of them) computed while they are in flight
    const float3 fn = nb_force_of(Nb, a);
    const long long b0 = bacc[3ll * a], b1 = bacc[3ll * a + 1], b2 = bacc[3ll * a + 2];
    const float ma = mass[a], sa = langevin ? sigv[a] : 0.0f;
    const float v0 = v[3ll * a], v1 = v[3ll * a + 1], v2 = v[3ll * a + 2];
    const float3 xi = langevin ? md_normals((unsigned)a, step, 1u, seed) : make_float3(0.0f, 0.0f, 0.0f);
    const float fx = fn.x + __ll2float_rn(b0) * sc;
    const float fy = fn.y + __ll2float_rn(b1) * sc;
    const float fz = fn.z + __ll2float_rn(b2) * sc;
    bacc[3ll * a] = 0;
    bacc[3ll * a + 1] = 0;
    bacc[3ll * a + 2] = 0;
    Ftot[3ll * a] = fx;
    Ftot[3ll * a + 1] = fy;
    Ftot[3ll * a + 2] = fz;
    const float h = 0.5f * dt * kAccel / ma;
    float vx = fmaf(h, fx, v0), vy = fmaf(h, fy, v1), vz = fmaf(h, fz, v2);
    if (langevin) {
        vx = fmaf(c, vx, sa * xi.x);
        vy = fmaf(c, vy, sa * xi.y);
        vz = fmaf(c, vz, sa * xi.z);
    }
    v[3ll * a] = vx;
    v[3ll * a + 1] = vy;
    v[3ll * a + 2] = vz;
    return make_float3(vx, vy, vz);
}

// Rigid water: constraint k joins (O, H1), (O, H2), (H1, H2).
// (written as functions so that unrolled loops resolve them at compile time)
__device__ __forceinline__ constexpr int con_a(int k) { return k == 2 ? 1 : 0; }
__device__ __forceinline__ constexpr int con_b(int k) { return k == 0 ? 1 : 2; }

// s(i, l): +1 if atom i (0 = O, 1 = H1, 2 = H2) is the first atom of
// constraint l, -1 if the second, else 0.
__device__ __forceinline__ float sgn(int i, int l) { return i == con_a(l) ? 1.0f : (i == con_b(l) ? -1.0f : 0.0f); }

// 3 x 3 solve by the adjugate (the constraint systems are well conditioned).
__device__ __forceinline__ void solve3(const float A[3][3], const float b[3], float x[3])
{
    const float c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
    const float c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
    const float c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
    const float det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
    const float id = 1.0f / det;
    const float i00 = c00 * id, i10 = c01 * id, i20 = c02 * id;
    const float i01 = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) * id;
    const float i11 = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) * id;
    const float i21 = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) * id;
    const float i02 = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) * id;
    const float i12 = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) * id;
    const float i22 = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) * id;
    x[0] = i00 * b[0] + i01 * b[1] + i02 * b[2];
    x[1] = i10 * b[0] + i11 * b[1] + i12 * b[2];
    x[2] = i20 * b[0] + i21 * b[1] + i22 * b[2];
}

struct MdStep {
    float dt, c;
    bool langevin;
    unsigned long long seed;
    float d2oh, d2hh, tol;
    int max_iter;
};

// M-SHAKE of one water (atoms at[], inverse masses im[]) from the reference
// positions x to the unconstrained new positions xn: the displacements dsp
// that restore |r_k''|^2 = d_k^2; false when max_iter iterations did not
// reach the tolerance.
// The reference bond vectors r_k = x_a - x_b of a water (minimum image).
__device__ __forceinline__ void water_bonds(const int (&at)[3], const float *__restrict__ x, const Box3 &B,
                                            float3 (&r)[3])
{
#pragma unroll
    for (int k = 0; k < 3; ++k) r[k] = disp(x, at[con_b(k)], at[con_a(k)], B);
}

__device__ __forceinline__ bool water_shake(const float3 (&r)[3], const float3 (&xn)[3], const float (&im)[3],
                                            const Box3 &B, const MdStep &P, float3 (&dsp)[3])
{
    float3 u[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float3 pa = xn[con_a(k)], pb = xn[con_b(k)];
        u[k] = make_float3(min_img(pa.x - pb.x, B.L[0], B.h[0]), min_img(pa.y - pb.y, B.L[1], B.h[1]),
                           min_img(pa.z - pb.z, B.L[2], B.h[2]));
    }
    const float d2[3] = {P.d2oh, P.d2oh, P.d2hh};
    float C[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l) C[k][l] = sgn(con_a(k), l) * im[con_a(k)] - sgn(con_b(k), l) * im[con_b(k)];
    float lam[3] = {0.0f, 0.0f, 0.0f};
    bool conv = false;
    for (int it = 0; it < P.max_iter; ++it) {
        float3 rr[3];
        float g[3];
        float worst = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            rr[k] = u[k];
#pragma unroll
            for (int l = 0; l < 3; ++l) rr[k] = add3(rr[k], scale3(lam[l] * C[k][l], r[l]));
            g[k] = dot3(rr[k], rr[k]) - d2[k];
            worst = fmaxf(worst, fabsf(g[k]) / d2[k]);
        }
        if (worst < P.tol) {
            conv = true;
            break;
        }
        float J[3][3], dl[3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int l = 0; l < 3; ++l) J[k][l] = 2.0f * C[k][l] * dot3(rr[k], r[l]);
        solve3(J, g, dl);
#pragma unroll
        for (int l = 0; l < 3; ++l) lam[l] -= dl[l];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        dsp[i] = make_float3(0.0f, 0.0f, 0.0f);
#pragma unroll
        for (int l = 0; l < 3; ++l) dsp[i] = add3(dsp[i], scale3(lam[l] * sgn(i, l) * im[i], r[l]));
    }
    return conv;
}

// Lanes of the two half-step kernels: the first ceil(n_free / 32) warps take
// one unconstrained atom per lane; every later warp takes kWatersPerWarp
// rigid waters, three lanes each (lane 3 j + i: atom i of water j; lanes 30
// and 31 idle), so that a water's three atoms are kicked on three lanes and
// the constraint solve, done redundantly on the three lanes with the same
// inputs, gives every lane the same result.
constexpr int kWatersPerWarp = 10;

struct MdLane {
    bool water_warp;  // the warp takes waters (warp-uniform)
    bool active;      // the lane holds an atom
    int item;         // free: index into free_atoms; water: water index
    int i;            // water: atom of the water (0 = O, 1, 2 = H)
};

__device__ __forceinline__ MdLane md_lane(int n_free, int nw)
{
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    const int free_warps = (n_free + 31) >> 5;
    MdLane L;
    L.water_warp = gw >= free_warps;
    if (!L.water_warp) {
        L.item = gw * 32 + lane;
        L.i = 0;
        L.active = L.item < n_free;
    } else {
        L.item = (gw - free_warps) * kWatersPerWarp + lane / 3;
        L.i = lane % 3;
        L.active = lane < 3 * kWatersPerWarp && L.item < nw;
    }
    return L;
}

inline int md_lane_blocks(int n_free, int nw)
{
    const int warps = (n_free + 31) / 32 + (nw + kWatersPerWarp - 1) / kWatersPerWarp;
    return std::max(1, (warps + 1) / 2);  // 64-thread blocks
}

// Value v of lane base + k of this warp, for k = 0, 1, 2 (the water's atoms).
__device__ __forceinline__ float3 water_lanes3(float3 v, int base, int k)
{
    return make_float3(__shfl_sync(0xffffffffu, v.x, base + k), __shfl_sync(0xffffffffu, v.y, base + k),
                       __shfl_sync(0xffffffffu, v.z, base + k));
}

// First half of a step.  An unconstrained atom: O, B, A.  A water: each of
// its three lanes kicks and drifts its atom, then M-SHAKE on the three
// lanes: lambda by Newton iterations on |r_k''|^2 = d_k^2,
// r_k'' = u_k + sum_l lambda_l C_kl r_l (u: new, r: reference vectors of x,
// C_kl = s(a_k, l)/m_{a_k} - s(b_k, l)/m_{b_k}), disp_i =
// sum_l lambda_l s(i, l) r_l / m_i, until every |g_k| / d_k^2 < tol or
// max_iter iterations; each lane moves its atom.  New positions wrapped into
// the box.  Block 0 clears the energy sums of this step.
__global__ void __launch_bounds__(64) k_md_first(int n_free, int nw, MdStep P,
                                                 const unsigned long long *__restrict__ step,
                                                 const int *__restrict__ free_atoms, const int4 *__restrict__ waters,
                                                 const float *__restrict__ mass, const float *__restrict__ sigv,
                                                 const float *__restrict__ Ftot, float *__restrict__ x,
                                                 float *__restrict__ v, Box3 B, long long *__restrict__ acc,
                                                 int *__restrict__ status)
{
    pdl_entry();
    if (blockIdx.x == 0 && threadIdx.x < kMdAcc) acc[threadIdx.x] = 0;
    const unsigned long long st = step[0];
    const MdLane L = md_lane(n_free, nw);
    if (!L.water_warp) {
        if (!L.active) return;
        const int a = free_atoms[L.item];
        const float3 p = kick_drift(a, P.dt, P.c, P.langevin, P.seed, st, mass, sigv, Ftot, x, v);
        x[3ll * a] = wrap_coord(p.x, B.L[0]);
        x[3ll * a + 1] = wrap_coord(p.y, B.L[1]);
        x[3ll * a + 2] = wrap_coord(p.z, B.L[2]);
        return;
    }
    // water warp: every lane stays to the end (shuffles, warp barrier)
    const int4 W = L.active ? waters[L.item] : make_int4(0, 0, 0, 0);
    const int at[3] = {W.x, W.y, W.z};
    const int a = L.i == 0 ? at[0] : (L.i == 1 ? at[1] : at[2]);
    float3 r[3];  // the reference bonds (loads issued before the kick)
    if (L.active) water_bonds(at, x, B, r);
    float3 mine = make_float3(0.0f, 0.0f, 0.0f);
    float im_mine = 1.0f;
    if (L.active) {
        mine = kick_drift(a, P.dt, P.c, P.langevin, P.seed, st, mass, sigv, Ftot, x, v);
        im_mine = 1.0f / mass[a];
    }
    const int base = (threadIdx.x & 31) - L.i;
    float3 xn[3];
    float im[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        xn[k] = water_lanes3(mine, base, k);
        im[k] = __shfl_sync(0xffffffffu, im_mine, base + k);
    }
    float3 dsp[3];
    if (L.active && !water_shake(r, xn, im, B, P, dsp) && L.i == 0) atomicOr(status, ST_TIMEOUT);
    __syncwarp();  // the three lanes read the reference positions x before any writes them
    if (!L.active) return;
    const float3 d = L.i == 0 ? dsp[0] : (L.i == 1 ? dsp[1] : dsp[2]);
    const float idt = 1.0f / P.dt;
    x[3ll * a] = wrap_coord(mine.x + d.x, B.L[0]);
    x[3ll * a + 1] = wrap_coord(mine.y + d.y, B.L[1]);
    x[3ll * a + 2] = wrap_coord(mine.z + d.z, B.L[2]);
    v[3ll * a] = fmaf(d.x, idt, v[3ll * a]);
    v[3ll * a + 1] = fmaf(d.y, idt, v[3ll * a + 1]);
    v[3ll * a + 2] = fmaf(d.z, idt, v[3ll * a + 2]);
}

// Second half of a step, same lanes: B and O with the new forces (the
// short-range and PME forces read from their fixed-point sums); a water's
// velocities then by RATTLE on its three lanes, mu from the 3 x 3 system
// sum_l mu_l C_kl (r_k . r_l) = -r_k . (v_a - v_b), v_i += sum_l mu_l s(i,l) r_l / m_i;
// kinetic energy (a water's on its first lane).  The last block to finish
// writes the energies (short-range + long-range from their sums, the
// fixed-point sums of acc) to energy, when given, and advances the device
// step counter.
__global__ void __launch_bounds__(64) k_md_second(int n_free, int nw, MdStep P,
                                                  unsigned long long *__restrict__ step,
                                                  const int *__restrict__ free_atoms, const int4 *__restrict__ waters,
                                                  const float *__restrict__ mass, const float *__restrict__ sigv,
                                                  NbSums Nb, long long *__restrict__ bacc,
                                                  float *__restrict__ Ftot, const float *__restrict__ x,
                                                  float *__restrict__ v, Box3 B, long long *__restrict__ acc,
                                                  const long long *__restrict__ sys_acc, const long long *__restrict__ pme_s,
                                                  double pme_self, double *__restrict__ energy)
{
    pdl_entry();
    const unsigned long long st = step[0];
    long long ke[1] = {0};
    const MdLane L = md_lane(n_free, nw);
    if (!L.water_warp) {
        if (L.active) {
            const int a = free_atoms[L.item];
            const float3 u = kick(a, P.dt, P.c, P.langevin, P.seed, st, mass, sigv, Nb, bacc, Ftot, v);
            ke[0] = __float2ll_rn(0.5f * mass[a] * fmaf(u.x, u.x, fmaf(u.y, u.y, u.z * u.z)) / kAccel *
                                  4294967296.0f);
        }
    } else {
        const int4 W = L.active ? waters[L.item] : make_int4(0, 0, 0, 0);
        const int at[3] = {W.x, W.y, W.z};
        const int a = L.i == 0 ? at[0] : (L.i == 1 ? at[1] : at[2]);
        float3 r[3];  // the bonds (loads issued before the kick)
        if (L.active) water_bonds(at, x, B, r);
        float3 mine = make_float3(0.0f, 0.0f, 0.0f);
        float m_mine = 1.0f;
        if (L.active) {
            mine = kick(a, P.dt, P.c, P.langevin, P.seed, st, mass, sigv, Nb, bacc, Ftot, v);
            m_mine = mass[a];
        }
        const int base = (threadIdx.x & 31) - L.i;
        float m[3], im[3], vv[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float3 u = water_lanes3(mine, base, k);
            vv[k][0] = u.x;
            vv[k][1] = u.y;
            vv[k][2] = u.z;
            m[k] = __shfl_sync(0xffffffffu, m_mine, base + k);
            im[k] = 1.0f / m[k];
        }
        if (L.active) {
            float A[3][3], b[3], mu[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int ka = con_a(k), kb = con_b(k);
                const float3 dv = make_float3(vv[ka][0] - vv[kb][0], vv[ka][1] - vv[kb][1], vv[ka][2] - vv[kb][2]);
                b[k] = -dot3(r[k], dv);
#pragma unroll
                for (int l = 0; l < 3; ++l)
                    A[k][l] = (sgn(ka, l) * im[ka] - sgn(kb, l) * im[kb]) * dot3(r[k], r[l]);
            }
            solve3(A, b, mu);
            float e = 0.0f, mx = 0.0f, my = 0.0f, mz = 0.0f;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                float3 dv = make_float3(0.0f, 0.0f, 0.0f);
#pragma unroll
                for (int l = 0; l < 3; ++l) dv = add3(dv, scale3(mu[l] * sgn(i, l) * im[i], r[l]));
                const float vx = vv[i][0] + dv.x, vy = vv[i][1] + dv.y, vz = vv[i][2] + dv.z;
                if (i == L.i) {
                    mx = vx;
                    my = vy;
                    mz = vz;
                }
                e = fmaf(0.5f * m[i], fmaf(vx, vx, fmaf(vy, vy, vz * vz)), e);
            }
            v[3ll * a] = mx;
            v[3ll * a + 1] = my;
            v[3ll * a + 2] = mz;
            if (L.i == 0) ke[0] = __float2ll_rn(e / kAccel * 4294967296.0f);
        }
    }
    const int idx[1] = {3};
    if (energy) md_flush<1>(ke, acc, idx);  // the kinetic energy only when reported
    else __syncthreads();                   // (its barrier: every thread has read step before the ticket)
    if (threadIdx.x == 0) {  // the thread that added this block's sum
        __threadfence();
        const unsigned long long done =
            atomicAdd((unsigned long long *)&acc[kMdTicket], 1ull);
        if (done == gridDim.x - 1ull) {  // every block has read step and added its sum
            __threadfence();
            const volatile long long *va = acc;
            if (energy) {  // the short-range (+ PME) energies as the unpack kernel converts them
                long long e_lj = sys_acc[0], e_c = sys_acc[1];
                if (pme_s) e_c += pme_s[0] + pme_s[2] + __double2ll_rn(pme_self * (double)pme_s[1] * (1.0 / 16.0));
                energy[0] = (double)e_lj * (1.0 / kFixScale);
                energy[1] = (double)e_c * (1.0 / kFixScale);
                for (int k = 0; k < 4; ++k) energy[2 + k] = (double)va[k] * (1.0 / 4294967296.0);
            }
            step[0] += 1ull;
        }
    }
}

__global__ void k_md_bonded_out(int n, const long long *__restrict__ bacc, const long long *__restrict__ acc,
                                float *__restrict__ F, double *__restrict__ energy)
{
    pdl_entry();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 3 * n) F[i] = __ll2float_rn(bacc[i]) * 2.3283064365386963e-10f;
    if (i < 3 && energy) energy[i] = (double)acc[i] * (1.0 / 4294967296.0);
}

// Energy minimisation by steepest descent in mass-weighted coordinates with
// a displacement cap and the rigid waters kept by M-SHAKE.  Part 1: total
// forces F = F_short (+ PME) + bonded (as k_md_collect) and the largest
// |F_i| / m_i over the atoms into *amax (the bits of a non-negative float,
// whose order an unsigned atomicMax keeps).
__global__ void __launch_bounds__(256) k_min_collect(int n, const float *__restrict__ Fnb, long long *__restrict__ bacc,
                                                     float *__restrict__ Ftot, const float *__restrict__ mass,
                                                     unsigned *__restrict__ amax)
{
    pdl_entry();
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    float g = 0.0f;
    if (a < n) {
        float fx, fy, fz;
        collect_force(a, Fnb, bacc, Ftot, fx, fy, fz);
        g = sqrtf(fmaf(fx, fx, fmaf(fy, fy, fz * fz))) / mass[a];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) g = fmaxf(g, __shfl_xor_sync(0xffffffffu, g, o));
    if ((threadIdx.x & 31) == 0) atomicMax(amax, __float_as_uint(g));
}

// Part 2, one thread per unconstrained atom or per water: x <- x + h F / m
// with h = dmax / max_i |F_i| / m_i (the atom with the largest mass-weighted
// force moves by dmax before the constraints), then M-SHAKE of every water
// from x; positions wrapped into the box.  Clears the other slot of amax for
// the next step.
__global__ void __launch_bounds__(64) k_min_move(int n_free, int nw, MdStep P, const int *__restrict__ free_atoms,
                                                 const int4 *__restrict__ waters, const float *__restrict__ mass,
                                                 const float *__restrict__ Ftot, float *__restrict__ x, Box3 B,
                                                 float dmax, const unsigned *__restrict__ amax_cur,
                                                 unsigned *__restrict__ amax_next, int *__restrict__ status)
{
    pdl_entry();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) *amax_next = 0u;
    const float gmax = __uint_as_float(*amax_cur);
    const float h = gmax > 0.0f ? dmax / gmax : 0.0f;
    if (t < n_free) {
        const int a = free_atoms[t];
        const float s = h / mass[a];
#pragma unroll
        for (int c = 0; c < 3; ++c) x[3ll * a + c] = wrap_coord(fmaf(s, Ftot[3ll * a + c], x[3ll * a + c]), B.L[c]);
        return;
    }
    const int w = t - n_free;
    if (w >= nw) return;
    const int4 W = waters[w];
    const int at[3] = {W.x, W.y, W.z};
    float3 xn[3];
    float im[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int a = at[i];
        im[i] = 1.0f / mass[a];
        const float s = h * im[i];
        xn[i] = make_float3(fmaf(s, Ftot[3ll * a], x[3ll * a]), fmaf(s, Ftot[3ll * a + 1], x[3ll * a + 1]),
                            fmaf(s, Ftot[3ll * a + 2], x[3ll * a + 2]));
    }
    float3 dsp[3];
    float3 r[3];
    water_bonds(at, x, B, r);
    if (!water_shake(r, xn, im, B, P, dsp)) atomicOr(status, ST_TIMEOUT);
    // the reference vectors above read x: write the new positions afterwards
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int a = at[i];
        x[3ll * a] = wrap_coord(xn[i].x + dsp[i].x, B.L[0]);
        x[3ll * a + 1] = wrap_coord(xn[i].y + dsp[i].y, B.L[1]);
        x[3ll * a + 2] = wrap_coord(xn[i].z + dsp[i].z, B.L[2]);
    }
}

// Energies at the positions of the last force evaluation: E_LJ, E_Coul,
// E_bond, E_angle, E_dihedral, and 0 kinetic energy.
__global__ void k_min_energy(const double *__restrict__ enb, const long long *__restrict__ acc,
                             double *__restrict__ energy)
{
    pdl_entry();
    const int i = threadIdx.x;
    if (i < 2) energy[i] = enb[i];
    else if (i < 5) energy[i] = (double)acc[i - 2] * (1.0 / 4294967296.0);
    else if (i == 5) energy[i] = 0.0;
}

// ---------------------------------------------------------------- host side

static Box3 box_of(const nb_ctx *ctx)
{
    Box3 B;
    for (int a = 0; a < 3; ++a) {
        B.L[a] = ctx->sys_h[0].L[a];
        B.h[a] = ctx->sys_h[0].half[a];
    }
    return B;
}

void md_free(nb_ctx *ctx)
{
    MdState *m = ctx->md;
    if (!m) return;
    void *p[] = {m->mass, m->sigv, m->free_atoms, m->bonds, m->bond_p, m->angles, m->angle_p, m->dihedrals,
                 m->dihedral_p, m->waters, m->Fnb, m->Ftot, m->bacc, m->enb, m->acc, m->step, m->amax};
    for (void *q : p)
        if (q) cudaFree(q);
    if (m->bside) {
        cudaStreamSynchronize(m->bside);
        cudaStreamDestroy(m->bside);
    }
    if (m->bfork) cudaEventDestroy(m->bfork);
    if (m->bjoin) cudaEventDestroy(m->bjoin);
    delete m;
    ctx->md = nullptr;
}

static cudaError_t launch_bonded(nb_ctx *ctx, cudaStream_t st, const float *d_pos)
{
    MdState &M = *ctx->md;
    const int terms = M.nb + M.na + M.nd;
    if (terms == 0) return cudaSuccess;
    const int blocks = std::max(1, std::min((terms + 255) / 256, 4 * ctx->num_sms));
    return launch_pdl(k_md_bonded, dim3(blocks), dim3(256), 0, st, M.nb, M.na, M.nd,
                      (const int2 *)M.bonds, (const float2 *)M.bond_p, (const int4 *)M.angles,
                      (const float2 *)M.angle_p, (const int4 *)M.dihedrals, (const float4 *)M.dihedral_p, d_pos,
                      box_of(ctx), M.bacc, M.acc);
}

// Forces at d_pos: cell list, short-range forces, PME (when enabled) and
// bonded terms.  The PME chain needs the sorted atoms but not the pair
// lists, so it is forked onto its side stream right after the column sort
// and the charge pack: it overlaps the list kernel and the short-range
// kernel, and behind it a helper launch of the short-range kernel takes
// units from the same counter; the bonded terms (positions only) run on a
// stream of their own, off both.  sums: the energies of this evaluation are
// reported (the PME pair-correction energies are summed only then).
static cudaError_t md_forces(nb_ctx *ctx, const float *d_pos, const float *d_q, const int32_t *d_type, bool sums,
                             bool unpack = true)
{
    MdState &M = *ctx->md;
    cudaError_t e = launch_build_cells(ctx, d_pos, d_q, d_type);  // q and types packed on the way
    const bool pme = ctx->pme != nullptr;
    const bool bside = pme && M.nb + M.na + M.nd > 0;
    if (e == cudaSuccess && bside) {
        e = cudaEventRecord(M.bfork, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(M.bside, M.bfork, 0);
        if (e == cudaSuccess) e = launch_bonded(ctx, M.bside, d_pos);
        if (e == cudaSuccess) e = cudaEventRecord(M.bjoin, M.bside);
    }
    if (e == cudaSuccess && pme) e = launch_pme_fork(ctx, d_pos, d_q, sums);
    if (e == cudaSuccess) e = launch_build_lists(ctx);
    if (e != cudaSuccess) return e;
    ctx->built = true;
    e = launch_forces_packed(ctx, unpack ? M.Fnb : nullptr, unpack ? M.enb : nullptr, nullptr, false, pme, pme, pme);
    if (e != cudaSuccess) return e;
    if (pme) return bside ? cudaStreamWaitEvent(ctx->stream, M.bjoin, 0) : cudaSuccess;
    return launch_bonded(ctx, ctx->stream, d_pos);
}

}  // namespace acenb

using namespace acenb;

template <class T>
static cudaError_t upload(T **dst, const T *src, size_t n)
{
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc(dst, sizeof(T) * n);
    if (e == cudaSuccess) e = cudaMemcpy(*dst, src, sizeof(T) * n, cudaMemcpyHostToDevice);
    return e;
}

extern "C" nb_status nb_md_init(nb_ctx *ctx, const nb_md_params *p)
{
    if (!ctx || !p) return NB_ERR_INVALID_ARG;
    if (ctx->n_sys != 1) return NB_ERR_UNSUPPORTED;
    const int N = (int)ctx->n_atoms;
    if (!p->mass || !(p->dt > 0.0f) || !(p->gamma >= 0.0f) || !(p->temperature >= 0.0f) || p->flags != 0 ||
        p->n_bonds < 0 || p->n_angles < 0 || p->n_dihedrals < 0 || p->n_waters < 0 || p->shake_max_iter < 1 ||
        !(p->shake_tolerance > 0.0f))
        return NB_ERR_INVALID_ARG;
    if ((p->n_bonds && (!p->bonds || !p->bond_k || !p->bond_r0)) ||
        (p->n_angles && (!p->angles || !p->angle_k || !p->angle_theta0)) ||
        (p->n_dihedrals && (!p->dihedrals || !p->dihedral_k || !p->dihedral_n || !p->dihedral_phase)) ||
        (p->n_waters && (!p->waters || !(p->water_roh > 0.0f) || !(p->water_rhh > 0.0f))))
        return NB_ERR_INVALID_ARG;
    auto in_range = [N](const int32_t *v, int64_t n) {
        for (int64_t i = 0; i < n; ++i)
            if (v[i] < 0 || v[i] >= N) return false;
        return true;
    };
    if (!in_range(p->bonds, 2ll * p->n_bonds) || !in_range(p->angles, 3ll * p->n_angles) ||
        !in_range(p->dihedrals, 4ll * p->n_dihedrals) || !in_range(p->waters, 3ll * p->n_waters))
        return NB_ERR_INVALID_ARG;
    for (int i = 0; i < N; ++i)
        if (!(p->mass[i] > 0.0f)) return NB_ERR_INVALID_ARG;
    std::vector<int> water_of(N, -1);
    for (int w = 0; w < p->n_waters; ++w)
        for (int k = 0; k < 3; ++k) {
            const int a = p->waters[3 * w + k];
            if (water_of[a] >= 0) return NB_ERR_INVALID_ARG;  // an atom in two waters
            water_of[a] = w;
        }
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return NB_ERR_CUDA;
    md_free(ctx);
    MdState *M = new MdState();
    ctx->md = M;
    if (cudaStreamCreateWithFlags(&M->bside, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&M->bfork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&M->bjoin, cudaEventDisableTiming) != cudaSuccess) {
        md_free(ctx);
        return NB_ERR_CUDA;
    }
    M->n = N;
    M->nb = p->n_bonds;
    M->na = p->n_angles;
    M->nd = p->n_dihedrals;
    M->nw = p->n_waters;
    M->dt = p->dt;
    M->langevin = p->gamma > 0.0f;
    const double c = std::exp(-(double)p->gamma * (double)p->dt / 2.0);
    M->c = (float)c;
    M->seed = p->seed;
    M->shake_iter = p->shake_max_iter;
    M->shake_tol = p->shake_tolerance;
    M->d2[0] = p->water_roh * p->water_roh;
    M->d2[1] = p->water_rhh * p->water_rhh;
    const double kT = kBoltzmann * (double)p->temperature;
    std::vector<float> sig(N);
    for (int i = 0; i < N; ++i) sig[i] = (float)std::sqrt((1.0 - c * c) * kT * (double)kAccel / (double)p->mass[i]);
    std::vector<int2> bonds(M->nb);
    std::vector<float2> bp(M->nb);
    for (int i = 0; i < M->nb; ++i) {
        bonds[i] = make_int2(p->bonds[2 * i], p->bonds[2 * i + 1]);
        bp[i] = make_float2(p->bond_k[i], p->bond_r0[i]);
    }
    std::vector<int4> ang(M->na);
    std::vector<float2> ap(M->na);
    for (int i = 0; i < M->na; ++i) {
        ang[i] = make_int4(p->angles[3 * i], p->angles[3 * i + 1], p->angles[3 * i + 2], 0);
        ap[i] = make_float2(p->angle_k[i], p->angle_theta0[i]);
    }
    std::vector<int4> dih(M->nd);
    std::vector<float4> dp(M->nd);
    for (int i = 0; i < M->nd; ++i) {
        dih[i] = make_int4(p->dihedrals[4 * i], p->dihedrals[4 * i + 1], p->dihedrals[4 * i + 2],
                           p->dihedrals[4 * i + 3]);
        dp[i] = make_float4(p->dihedral_k[i], (float)p->dihedral_n[i], p->dihedral_phase[i], 0.0f);
    }
    std::vector<int> free_atoms;
    for (int i = 0; i < N; ++i)
        if (water_of[i] < 0) free_atoms.push_back(i);
    M->n_free = (int)free_atoms.size();
    std::vector<int4> wat(M->nw);
    for (int i = 0; i < M->nw; ++i) wat[i] = make_int4(p->waters[3 * i], p->waters[3 * i + 1], p->waters[3 * i + 2], 0);
    cudaError_t e = upload(&M->mass, p->mass, N);
    if (e == cudaSuccess) e = upload(&M->sigv, sig.data(), N);
    if (e == cudaSuccess) e = upload(&M->free_atoms, free_atoms.data(), free_atoms.size());
    if (e == cudaSuccess) e = upload(&M->bonds, bonds.data(), bonds.size());
    if (e == cudaSuccess) e = upload(&M->bond_p, bp.data(), bp.size());
    if (e == cudaSuccess) e = upload(&M->angles, ang.data(), ang.size());
    if (e == cudaSuccess) e = upload(&M->angle_p, ap.data(), ap.size());
    if (e == cudaSuccess) e = upload(&M->dihedrals, dih.data(), dih.size());
    if (e == cudaSuccess) e = upload(&M->dihedral_p, dp.data(), dp.size());
    if (e == cudaSuccess) e = upload(&M->waters, wat.data(), wat.size());
    if (e == cudaSuccess) e = cudaMalloc(&M->Fnb, sizeof(float) * 3 * N);
    if (e == cudaSuccess) e = cudaMalloc(&M->Ftot, sizeof(float) * 3 * N);
    if (e == cudaSuccess) e = cudaMalloc(&M->bacc, sizeof(long long) * 3 * N);
    if (e == cudaSuccess) e = cudaMalloc(&M->enb, sizeof(double) * 2);
    if (e == cudaSuccess) e = cudaMalloc(&M->acc, sizeof(long long) * kMdAcc);
    if (e == cudaSuccess) e = cudaMalloc(&M->step, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&M->amax, 2 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(M->bacc, 0, sizeof(long long) * 3 * N);
    if (e == cudaSuccess) e = cudaMemset(M->acc, 0, sizeof(long long) * kMdAcc);
    if (e == cudaSuccess) e = cudaMemset(M->step, 0, sizeof(unsigned long long));
    if (e != cudaSuccess) {
        md_free(ctx);
        return e == cudaErrorMemoryAllocation ? NB_ERR_OOM : NB_ERR_CUDA;
    }
    return NB_OK;
}

extern "C" nb_status nb_bonded_forces(nb_ctx *ctx, const float *d_pos, float *d_F, double *d_energy)
{
    if (!ctx || !d_pos || !d_F) return NB_ERR_INVALID_ARG;
    if (!ctx->md) return NB_ERR_NOT_BUILT;
    MdState &M = *ctx->md;
    cudaError_t e = cudaMemsetAsync(M.bacc, 0, sizeof(long long) * 3 * M.n, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(M.acc, 0, sizeof(long long) * kMdAcc, ctx->stream);
    if (e == cudaSuccess) e = launch_bonded(ctx, ctx->stream, d_pos);
    if (e == cudaSuccess)
        e = launch_pdl(k_md_bonded_out, dim3((3 * M.n + 255) / 256), dim3(256), 0, ctx->stream, M.n,
                       (const long long *)M.bacc, (const long long *)M.acc, d_F, d_energy);
    if (e == cudaSuccess) e = cudaMemsetAsync(M.bacc, 0, sizeof(long long) * 3 * M.n, ctx->stream);
    return e == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}

extern "C" nb_status nb_md_step(nb_ctx *ctx, float *d_pos, float *d_vel, const float *d_q, const int32_t *d_type,
                                int32_t n_steps, double *d_energy)
{
    if (!ctx || !d_pos || !d_vel || !d_q || !d_type || n_steps < 0) return NB_ERR_INVALID_ARG;
    if (!ctx->md) return NB_ERR_NOT_BUILT;
    MdState &M = *ctx->md;
    const cudaStream_t st = ctx->stream;
    const Box3 B = box_of(ctx);
    const int N = M.n;
    const int ab = (N + 255) / 256;
    // one lane per unconstrained atom, three per rigid water, 64-thread
    // blocks (the integration is latency bound: spread it over the SMs)
    const int ib = md_lane_blocks(M.n_free, M.nw);
    MdStep P;
    P.dt = M.dt;
    P.c = M.c;
    P.langevin = M.langevin;
    P.seed = M.seed;
    P.d2oh = M.d2[0];
    P.d2hh = M.d2[1];
    P.tol = M.shake_tol;
    P.max_iter = M.shake_iter;
    cudaError_t e = cudaSuccess;
    if (!M.have_forces) {  // forces at the starting positions
        e = md_forces(ctx, d_pos, d_q, d_type, false);
        if (e == cudaSuccess)
            e = launch_pdl(k_md_collect, dim3(ab), dim3(256), 0, st, N, (const float *)M.Fnb, M.bacc, M.Ftot);
        if (e != cudaSuccess) return NB_ERR_CUDA;
        M.have_forces = true;
    }
    for (int s = 0; s < n_steps && e == cudaSuccess; ++s) {
        e = launch_pdl(k_md_first, dim3(ib), dim3(64), 0, st, M.n_free, M.nw, P,
                       (const unsigned long long *)M.step, (const int *)M.free_atoms, (const int4 *)M.waters,
                       (const float *)M.mass, (const float *)M.sigv, (const float *)M.Ftot, d_pos, d_vel, B, M.acc,
                       ctx->d.status);
        // the second half reads the short-range sums itself (no unpack kernel)
        if (e == cudaSuccess) e = md_forces(ctx, d_pos, d_q, d_type, d_energy && s == n_steps - 1, false);
        if (e == cudaSuccess)
            e = launch_pdl(k_md_second, dim3(ib), dim3(64), 0, st, M.n_free, M.nw, P,
                           M.step, (const int *)M.free_atoms, (const int4 *)M.waters,
                           (const float *)M.mass, (const float *)M.sigv,
                           NbSums{ctx->d.inv, ctx->d.facc, ctx->pme ? pme_forces_acc(ctx) : nullptr}, M.bacc,
                           M.Ftot, (const float *)d_pos, d_vel, B, M.acc, (const long long *)ctx->d.sys_acc,
                           ctx->pme ? pme_sums_acc(ctx) : nullptr, ctx->pme ? pme_self_coef(ctx) : 0.0,
                           s == n_steps - 1 ? d_energy : (double *)nullptr);
    }
    return e == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}

extern "C" nb_status nb_md_minimize(nb_ctx *ctx, float *d_pos, const float *d_q, const int32_t *d_type,
                                    int32_t n_steps, float max_disp, double *d_energy)
{
    if (!ctx || !d_pos || !d_q || !d_type || n_steps < 0 || !(max_disp > 0.0f) || !(max_disp < 1e30f))
        return NB_ERR_INVALID_ARG;
    if (!ctx->md) return NB_ERR_NOT_BUILT;
    MdState &M = *ctx->md;
    const cudaStream_t st = ctx->stream;
    const Box3 B = box_of(ctx);
    const int N = M.n;
    const int ab = (N + 255) / 256;
    const int ib = std::max(1, (M.n_free + M.nw + 63) / 64);
    MdStep P = {};
    P.d2oh = M.d2[0];
    P.d2hh = M.d2[1];
    P.tol = M.shake_tol;
    P.max_iter = M.shake_iter;
    cudaError_t e = cudaMemsetAsync(M.amax, 0, 2 * sizeof(unsigned), st);
    // n_steps moves, each from the forces at the current positions, and the
    // forces at the final positions (left for the next nb_md_step)
    for (int s = 0; s <= n_steps && e == cudaSuccess; ++s) {
        e = cudaMemsetAsync(M.acc, 0, sizeof(long long) * kMdAcc, st);
        if (e == cudaSuccess) e = md_forces(ctx, d_pos, d_q, d_type, d_energy && s == n_steps);
        if (e == cudaSuccess)
            e = launch_pdl(k_min_collect, dim3(ab), dim3(256), 0, st, N, (const float *)M.Fnb, M.bacc, M.Ftot,
                           (const float *)M.mass, M.amax + (s & 1));
        if (e == cudaSuccess && s < n_steps)
            e = launch_pdl(k_min_move, dim3(ib), dim3(64), 0, st, M.n_free, M.nw, P, (const int *)M.free_atoms,
                           (const int4 *)M.waters, (const float *)M.mass, (const float *)M.Ftot, d_pos, B, max_disp,
                           (const unsigned *)(M.amax + (s & 1)), M.amax + ((s + 1) & 1), ctx->d.status);
    }
    if (e == cudaSuccess && d_energy)
        e = launch_pdl(k_min_energy, dim3(1), dim3(32), 0, st, (const double *)M.enb, (const long long *)M.acc,
                       d_energy);
    if (e != cudaSuccess) return NB_ERR_CUDA;
    M.have_forces = true;  // Ftot holds the forces at the final positions
    return NB_OK;
}

extern "C" nb_status nb_md_set_step(nb_ctx *ctx, uint64_t step)
{
    if (!ctx || !ctx->md) return NB_ERR_INVALID_ARG;
    const unsigned long long s = step;
    return cudaMemcpyAsync(ctx->md->step, &s, sizeof(s), cudaMemcpyHostToDevice, ctx->stream) == cudaSuccess &&
                   cudaStreamSynchronize(ctx->stream) == cudaSuccess
               ? NB_OK
               : NB_ERR_CUDA;
}

// Test export of the noise generator: Philox4x32-10 of n counter blocks.
__global__ void k_debug_philox(long long n, const uint32_t *__restrict__ ctr, const uint32_t *__restrict__ key,
                               uint32_t *__restrict__ out)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    uint32_t c[4] = {ctr[4 * k], ctr[4 * k + 1], ctr[4 * k + 2], ctr[4 * k + 3]};
    philox4x32_10(c, key[2 * k], key[2 * k + 1]);
    for (int w = 0; w < 4; ++w) out[4 * k + w] = c[w];
}

extern "C" nb_status nb_debug_philox(int64_t n, const uint32_t *d_ctr, const uint32_t *d_key, uint32_t *d_out,
                                     void *cuda_stream)
{
    if (n < 0 || (n > 0 && (!d_ctr || !d_key || !d_out))) return NB_ERR_INVALID_ARG;
    if (n == 0) return NB_OK;
    const int tb = 128;
    k_debug_philox<<<(unsigned)((n + tb - 1) / tb), tb, 0, (cudaStream_t)cuda_stream>>>(n, d_ctr, d_key, d_out);
    return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}
