// nb_pair.cuh - FP32 pair arithmetic shared by the forward and adjoint
// kernels: LJ 12-6 with the CHARMM switch and real-space Ewald Coulomb
// (section "Molecular dynamics on the GPU": Lennard-Jones and electrostatic
// terms of every pair inside the cutoff; section "Performance": switched at
// 7.5 A; PME real space erfc(alpha r)/r).
#pragma once

#include "nb_internal.cuh"

namespace acenb {

// Single-instruction special-function approximations (MUFU), flushing
// subnormals: relative error about 2^-22 for rsqrt and rcp and 2^-22.5 for
// ex2, far below the 5e-6 force target, but not centred on zero (measured
// against FP64 on this GPU: mean -5e-9 for rsqrt, +0.6 to +6e-9 for rcp,
// -5e-8 for ex2 below -1).  Summed energies of many terms of both signs
// would inherit those biases, so the forward pair arithmetic refines rsqrt
// and rcp by one Newton step and replaces ex2 by a fitted polynomial; the
// adjoint (1e-4 tolerances) uses them as they are.  The membership predicate
// uses exactly rounded operations.
__device__ __forceinline__ float fast_rsqrt(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float fast_rcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float fast_exp2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// erfcx(x) = exp(x^2) erfc(x) as a polynomial in t = 1 / (1 + x/2), fitted on
// the host on [0, alpha rc]; erfc(x) = exp(-x^2) * P(t).
__device__ __forceinline__ float erfcx_poly(const PairParams &P, float t)
{
    float p = P.erfc_c[kErfcDeg];
#pragma unroll
    for (int k = kErfcDeg - 1; k >= 0; --k) p = fmaf(p, t, P.erfc_c[k]);
    return p;
}

// Minimum-image displacement d = x_j - x_i and its FP32 squared length, the
// membership quantity: r2 = fma(dz, dz, fma(dy, dy, dx * dx)).
__device__ __forceinline__ float disp_r2(float xj, float yj, float zj, float xi, float yi, float zi,
                                         float &dx, float &dy, float &dz)
{
    dx = __fsub_rn(xj, xi);
    dy = __fsub_rn(yj, yi);
    dz = __fsub_rn(zj, zi);
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// 1/r and r of a pair from r2.  rsqrt.approx is refined by one Newton step,
// rinv = y (1 + (1 - r2 y^2) / 2): the approximation's own error (about
// 2^-22, not centred on zero) would reach r^-12 twelvefold and bias every
// summed LJ energy; after the step the error is the FP32 rounding of the
// step itself.  r = r2 y is the unrefined product: it only enters the erfc
// polynomial's variable t, whose sensitivity to r is small.
__device__ __forceinline__ void pair_rinv(float r2, float &rinv, float &r)
{
    const float y = fast_rsqrt(r2);
    r = __fmul_rn(r2, y);
    const float res = __fmaf_rn(-r, y, 1.0f);
    rinv = __fmaf_rn(__fmul_rn(0.5f, y), res, y);
}

// 1/d by rcp.approx refined by one Newton step, y (1 + (1 - d y)): the
// approximation's mean error (+0.6 to +6e-9 over [1, 2.5], measured against
// FP64) would reach erfc through the polynomial variable t.
__device__ __forceinline__ float rcp_refined(float d)
{
    const float y = fast_rcp(d);
    return __fmaf_rn(y, __fmaf_rn(-d, y, 1.0f), y);
}

// exp(-alpha^2 r2) = 2^(r2 c), c = -alpha^2 log2(e) held as two FP32 words
// (hi + lo).  y = fl(r2 hi) is split exactly into n = rint(y) (the 1.5 2^23
// rounding trick) and y - n in [-1/2, 1/2]; the part of r2 c that y lost (the
// product's exact rounding error by FMA, plus r2 lo) is added to the
// fraction, 2^fraction comes from the fitted polynomial P.exp2_c (within
// 4e-9, no bias) and 2^n is added to its exponent field (y > -126 here:
// alpha r < 9.3).  Without the polynomial, ex2.approx's mean error (-5e-8
// below -1) and the rounding of y (up to 2^-21 at alpha r = 2.9) would reach
// every Coulomb pair energy as an error that depends on the distance.
__device__ __forceinline__ float exp_neg_a2r2(const PairParams &P, float r2)
{
    const float y = __fmul_rn(r2, P.neg_a2_log2e);
    const float dy = __fmaf_rn(r2, P.neg_a2_log2e_lo, __fmaf_rn(r2, P.neg_a2_log2e, -y));
    const float big = __fadd_rn(y, 12582912.0f);  // 1.5 2^23 + rint(y): the integer sits in the low bits
    const float n = __fsub_rn(big, 12582912.0f);
    const float f = __fadd_rn(__fsub_rn(y, n), dy);
    float p = P.exp2_c[kExp2Deg];
#pragma unroll
    for (int k = kExp2Deg - 1; k >= 0; --k) p = __fmaf_rn(p, f, P.exp2_c[k]);
    // (bits of big) << 23 = n 2^23 modulo 2^32: adds n to p's exponent
    return __int_as_float(__float_as_int(p) + (__float_as_int(big) << 23));
}

// Radial part of one pair at squared distance r2 (inside the cutoff), from
// r, rinv = 1/r (pair_rinv), r2inv = 1/r2 and the type pair's LJ
// coefficients lj = (A, B, 12 A, 6 B) and the FP32 remainders lo of A and B
// (the energy adds them; the force does not need them):
//   elj, ec : LJ (switched) and Coulomb energies (unweighted);
//   frlj, frc : -dU/dr * r of each part.
template <bool EWALD, bool SWITCH>
__device__ __forceinline__ void pair_radial(const PairParams &P, float r2, float r, float rinv, float r2inv,
                                            float4 lj, float2 lo, float qq, float &elj, float &frlj, float &ec,
                                            float &frc)
{
    const float ir6 = r2inv * r2inv * r2inv;
    // A r^-12 - B r^-6: the remainders' term (below half an ulp of the
    // result) enters the last FMA beside the exact product, before its one
    // rounding; added to an already rounded value it would vanish
    elj = fmaf(ir6, fmaf(lj.x, ir6, -lj.y), ir6 * fmaf(lo.x, ir6, -lo.y));
    frlj = ir6 * fmaf(lj.z, ir6, -lj.w);  // 12 A r^-12 - 6 B r^-6
    if (SWITCH) {
        // with t = rc2 - r2 and u = rs2 - r2, for r > rs:
        // S = t^2 (rc2 + 2 r2 - 3 rs2) / (rc2 - rs2)^3 = t^2 (sw_a + sw_b u),
        // r dS/dr = 12 r2 t u / (rc2 - rs2)^3 = sw_c r2 t u.
        const float t = P.rc2 - r2, u = P.rs2 - r2;
        const float S = (t * t) * fmaf(P.sw_b, u, P.sw_a);
        const float rdS = P.sw_c * r2 * t * u;
        const bool sw = r2 > P.rs2;
        frlj = sw ? fmaf(S, frlj, -elj * rdS) : frlj;
        elj = sw ? S * elj : elj;
    }
    if (EWALD) {
        const float t = rcp_refined(fmaf(P.alpha_half, r, 1.0f));
        const float ex = exp_neg_a2r2(P, r2);               // exp(-alpha^2 r^2)
        const float erfcr = ex * erfcx_poly(P, t) * rinv;  // erfc(alpha r) / r
        ec = qq * erfcr;
        // -d/dr [erfc(a r)/r] * r = erfc(a r)/r + (2a/sqrt(pi)) exp(-a^2 r^2)
        frc = qq * fmaf(P.two_a_sqpi, ex, erfcr);
    } else {
        ec = qq * rinv;
        frc = ec;
    }
}

// Radial part by linear interpolation of the tables (section "Molecular
// dynamics on the GPU": radial components of the van der Waals and
// electrostatic terms interpolated from lookup tables).  Interval k of
// [0, rc] (n intervals, r_k = k rc / n) holds three float4:
// (E12, dE12, E6, dE6), (Ec, dEc, F12, dF12), (F6, dF6, Fc, dFc) -- the
// values at r_k of E12 = S r^-12, E6 = S r^-6, Ec = erfc(alpha r)/r and of
// F = -r dE/dr for each, with the differences to r_{k+1}.  Same outputs as
// pair_radial.  The interpolation is FP32 (one FMA per function) on the
// caller's r = r2 rsqrt(r2).
__device__ __forceinline__ void pair_radial_tab(const PairParams &P, const float4 *__restrict__ tab, float r,
                                                float A, float B, float2 lo, float qq, float &elj, float &frlj,
                                                float &ec, float &frc)
{
    const float x = r * P.tab_inv_h;
    const int k = max(0, min((int)x, P.tab_n - 1));
    const float t = x - (float)k;
    const float4 a = __ldg(&tab[3 * k]), b = __ldg(&tab[3 * k + 1]), c = __ldg(&tab[3 * k + 2]);
    const float e12 = fmaf(t, a.y, a.x), e6 = fmaf(t, a.w, a.z);
    const float ecv = fmaf(t, b.y, b.x), f12 = fmaf(t, b.w, b.z);
    const float f6 = fmaf(t, c.y, c.x), fcv = fmaf(t, c.w, c.z);
    elj = fmaf(A, e12, fmaf(-B, e6, fmaf(lo.x, e12, -lo.y * e6)));
    frlj = fmaf(A, f12, -B * f6);
    ec = qq * ecv;
    frc = qq * fcv;
}

}  // namespace acenb
