// nb_force.cu - the non-bonded force kernels (section "Molecular dynamics on
// the GPU": the non-bonded kernel computes the full Lennard-Jones and
// electrostatic force on each particle).  The paper's kernel does not reuse
// the reciprocal force F_ji; here both kernels do (Newton's third law): every
// unique pair is evaluated once, from the cluster whose half list holds it,
// and its contribution goes to both atoms as 64-bit fixed point (2^32), so
// the sums stay exact and order independent.
//
// Forward (k_force): one warp per listed cluster pair as an 8 x 8 tile,
// forces on i kept in registers, forces on j summed over lanes (see the
// comment above k_force).
//
// Adjoint (k_adjoint): the same tiles, work units and staging, with the
// pair adjoint; the type-pair gradients go to a block table in shared
// memory.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <atomic>

#include "nb_pair.cuh"

namespace acenb {

constexpr unsigned kFull = 0xffffffffu;

struct ForceArgs {
    const SysDesc *sys;
    const int *counts;
    int *work;                // work-unit counter of the tile kernels (zeroed by k_pack)
    const float4 *xyzq;
    const int *tslot;
    const int *perm;
    const int *clus_sys;
    const uint32_t *list;     // [NC*cap] per cluster: its half list (Newton's third law)
    const int *list_n;        // [NC] lengths
    const int *pslot;         // [S*K] partner slots (slot << 1) | is14, -1 pad
    int cap;                  // entries per list
    int K;
    const float2 *lj_tab;
    const float4 *rtab;       // [n*3] tabulated radial functions, or null
    long long *facc;          // [S*3] fixed-point forces in sorted order (forward)
    long long *sys_acc;
    int *status;
    long long *dbg_n;
    int *dbg_ij;
    long long dbg_cap;
    PairParams P;
    // adjoint only
    const float4 *gslot;     // [S] dL/dF in sorted order (x, y, z, 0)
    const double *dLdE;      // [n_sys*2] dL/dE_LJ, dL/dE_C, or null
    const float4 *lj_d;      // [T*T] 48 eps sig^11, 24 eps sig^5, 4 sig^12, 4 sig^6
    long long *tab_acc;      // [T*T*2] fixed-point dL/dsig_ab, dL/deps_ab (each unique pair in one order)
    long long *gacc;         // [S*4] fixed-point dL/dx, dL/dq in sorted order (both atoms of each pair)
};

__device__ __forceinline__ long long to_fixed(float v, int *status)
{
    // |v| < 2^26 keeps a sum of 32 lanes inside int64 at scale 2^32
    if (!(fabsf(v) < 67108864.0f)) {
        atomicOr(status, ST_OVERFLOW);
        return 0;
    }
    return __float2ll_rn(v * 4294967296.0f);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Slot of atom k of staged entry e (swizzle by e, conflict-free lane access).
__device__ __forceinline__ int swz(int e, int k) { return e * kCluster + (k ^ (e & (kCluster - 1))); }

struct Acc {
    float fx, fy, fz, elj, ec;
};

struct AccAdj {
    float dx, dy, dz, dq;
};

constexpr double kTabScale = 4294967296.0;  // fixed-point scale of the parameter gradients (2^32)

__device__ __forceinline__ long long to_fixed_tab(float v, int *status)
{
    if (!(fabsf(v) < 1073741824.0f)) {  // 2^30 per contribution
        atomicOr(status, ST_OVERFLOW);
        return 0;
    }
    return __float2ll_rn(v * (float)kTabScale);
}

// Adjoint of one ordered pair (i, j) for L = sum G.F + gE_lj E_lj + gE_c E_C.
// With d = x_j - x_i, F_i = h d where h = U'(r)/r, and g = G_i - G_j:
//   dL/dx_i -= h g + (h'/r)(g.d) d + (gE-weighted h) d     (h' = dh/dr)
//   dL/dq_i += w_c ke q_j (phi'(r)/r (g.d) + gE_c phi(r))
//   dL/dsig_ab, dL/deps_ab (each unique pair is visited once)
// through dU/dA = w S r^-12, dU/dB = -w S r^-6 and the chain factors
// dA/dsig = 48 eps sig^11, dB/dsig = 24 eps sig^5, dA/deps = 4 sig^12,
// dB/deps = 4 sig^6 of the type pair.
struct AdjTables {
    const float2 *lj;           // (A, B) per type pair
    const float4 *ljd;          // derivative factors per type pair
    unsigned long long *tacc;   // block table of fixed-point parameter gradients
};

template <bool EWALD>
__device__ __forceinline__ void eval_pair_adj(const PairParams &P, const AdjTables &S, int ti_row, float qi_ke, float gix,
                                              float giy, float giz, float gE_lj, float gE_c, bool in, float dx,
                                              float dy, float dz, float r2, float qj, int tj, float4 gj, bool is14,
                                              int *status, AccAdj &acc, float &jx, float &jy, float &jz, float &jq,
                                              float &dsig, float &deps)
{
    if (!in) {  // masked lanes: keep every product finite (padding sits far away)
        dx = 0.0f;
        dy = 0.0f;
        dz = 0.0f;
    }
    const float rinv = fast_rsqrt(r2);
    const float r = r2 * rinv, ir2 = rinv * rinv;
    const float2 ab = S.lj[ti_row + tj];
    const float ir6 = ir2 * ir2 * ir2, ir12 = ir6 * ir6;
    // LJ V = A r^-12 - B r^-6 and its r-derivatives
    const float t12 = ab.x * ir12, t6 = ab.y * ir6;
    const float V = t12 - t6;
    const float V1 = (6.0f * t6 - 12.0f * t12) * rinv;
    const float V2 = (156.0f * t12 - 42.0f * t6) * ir2;
    // switch S(r), S', S'' (r > rs)
    float Sw = 1.0f, S1 = 0.0f, S2 = 0.0f;
    if (r2 > P.rs2) {
        const float t = P.rc2 - r2, u = P.rs2 - r2;
        Sw = t * t * fmaf(2.0f, r2, P.sw_c0) * P.sw_inv;
        S1 = 12.0f * r * t * u * P.sw_inv;
        S2 = 12.0f * (t * u - 2.0f * r2 * u - 2.0f * r2 * t) * P.sw_inv;
    }
    const float wlj = is14 ? P.s14_lj : 1.0f;
    const float wc = is14 ? P.s14_c : 1.0f;
    const float Ulj1 = wlj * fmaf(S1, V, Sw * V1);
    const float Ulj2 = wlj * (S2 * V + 2.0f * S1 * V1 + Sw * V2);
    // Coulomb phi = erfc(a r)/r and its r-derivatives (without q_i q_j)
    float phi, phi1, phi2;
    if (EWALD) {
        const float tt = fast_rcp(fmaf(P.alpha_half, r, 1.0f));
        const float ex = fast_exp2(r2 * P.neg_a2_log2e);
        const float erfcv = ex * erfcx_poly(P, tt);
        const float cg = P.two_a_sqpi * ex;
        phi = erfcv * rinv;
        phi1 = -(cg + phi) * rinv;
        phi2 = 2.0f * P.alpha * P.alpha * cg + 2.0f * (cg + phi) * ir2;
    } else {
        phi = rinv;
        phi1 = -ir2;
        phi2 = 2.0f * ir2 * rinv;
    }
    const float qq = qi_ke * qj;
    const float U1 = fmaf(wc * qq, phi1, Ulj1);
    const float U2 = fmaf(wc * qq, phi2, Ulj2);
    const float h = U1 * rinv;
    const float h1r = (U2 - U1 * rinv) * ir2;  // (dh/dr) / r
    const float gx = gix - gj.x, gy = giy - gj.y, gz = giz - gj.z;
    const float gd = fmaf(gx, dx, fmaf(gy, dy, gz * dz));
    const float hE = (gE_lj * Ulj1 + gE_c * wc * qq * phi1) * rinv;
    const float cd = fmaf(h1r, gd, hE);
    const float m = in ? 1.0f : 0.0f;
    // the pair seen from j: d -> -d and g -> -g, so dL/dx_j gets the opposite
    // of dL/dx_i's term and dL/dq_j the same bracket times q_j's partner q_i
    jx = m * fmaf(h, gx, cd * dx);
    jy = m * fmaf(h, gy, cd * dy);
    jz = m * fmaf(h, gz, cd * dz);
    acc.dx -= jx;
    acc.dy -= jy;
    acc.dz -= jz;
    const float xq = m * wc * fmaf(phi1 * rinv, gd, gE_c * phi);
    acc.dq += xq * P.ke * qj;
    jq = xq * qi_ke;
    // type-pair parameters
    const float uA = wlj * Sw * ir12, uB = -wlj * Sw * ir6;
    const float uA1 = wlj * fmaf(S1, ir12, -12.0f * Sw * ir12 * rinv);
    const float uB1 = -wlj * fmaf(S1, ir6, -6.0f * Sw * ir6 * rinv);
    const float gA = fmaf(uA1 * rinv, gd, gE_lj * uA), gB = fmaf(uB1 * rinv, gd, gE_lj * uB);
    const float4 c = S.ljd[ti_row + tj];
    dsig = in ? fmaf(gA, c.x, gB * c.y) : 0.0f;
    deps = in ? fmaf(gA, c.z, gB * c.w) : 0.0f;
}

// 64-bit integer add to shared memory by two native 32-bit atomics: the low
// word's carry (seen from the value the first atomic returns) goes into the
// high word, so the 64-bit sum is exact and order independent.  (A 64-bit
// shared-memory atomic add is a compare-and-swap loop here, and many lanes
// of a warp hit the same few type-pair slots: the loop's retries cost more
// than the whole pair adjoint.)
__device__ __forceinline__ void shared_add64(unsigned long long *p, unsigned long long v)
{
    unsigned int *w = reinterpret_cast<unsigned int *>(p);  // little endian: low word first
    const unsigned int lo = (unsigned int)v, hi = (unsigned int)(v >> 32);
    const unsigned int old = atomicAdd(w, lo);
    const unsigned int h = hi + ((unsigned int)(old + lo) < old ? 1u : 0u);
    if (h) atomicAdd(w + 1, h);
}

// Add a lane's type-pair derivatives (key = t_i T + t_j, -1 for a masked
// lane) to the block table.  (Summing equal keys over the warp first, by
// match/ballot rounds or by the warp's integer reduction on 21-bit parts, was
// slower than the atomics: 0.37 and 0.50 ms against 0.19 ms per adjoint
// step.)
__device__ __forceinline__ void add_type_grads(const AdjTables &S, int key, float dsig, float deps, int *status)
{
    if (key >= 0) {
        shared_add64(&S.tacc[2 * key], (unsigned long long)to_fixed_tab(dsig, status));
        shared_add64(&S.tacc[2 * key + 1], (unsigned long long)to_fixed_tab(deps, status));
    }
}

// One candidate pair of the forward kernel: d = x_j - x_i (exact-shift
// image), r2 its FP32 squared length; the arithmetic is done for every
// candidate and masked by `in`.  RAD: radial functions evaluated directly
// with plain Coulomb (0) or Ewald (1), or interpolated from the tables (2).
// W14: the pair may be a scaled 1-4 pair (is14), else both weights are 1
// (the same bits either way for an unscaled pair).  lj holds (A, B, 12 A,
// 6 B) per type pair.  The force on i is subtracted from acc and the force
// on j added to fj with explicit FMA, so that the bits do not depend on how
// the caller was inlined.
template <int RAD, bool W14>
__device__ __forceinline__ void eval_pair(const PairParams &P, const float4 *__restrict__ lj,
                                          const float4 *__restrict__ rtab, int ti_row, float qi, bool in, float dx,
                                          float dy, float dz, float r2, float qj, int tj, bool is14, Acc &acc,
                                          float &fjx, float &fjy, float &fjz)
{
    float rinv, r;
    pair_rinv(r2, rinv, r);
    const float r2inv = __fmul_rn(rinv, rinv);
    const float4 ab = lj[ti_row + tj];
    float elj, frlj, ec, frc;
    if constexpr (RAD == 2)
        pair_radial_tab(P, rtab, r, ab.x, ab.y, qi * qj, elj, frlj, ec, frc);
    else
        pair_radial<RAD == 1, true>(P, r2, r, rinv, r2inv, ab, qi * qj, elj, frlj, ec, frc);
    // F_i = U'(r) d / r = -fs d with fs = -U'(r) / r
    float fs, wel, wec;
    if (W14) {
        const float wlj = is14 ? P.s14_lj : 1.0f;
        const float wc = is14 ? P.s14_c : 1.0f;
        fs = __fmul_rn(__fmaf_rn(wlj, frlj, __fmul_rn(wc, frc)), r2inv);
        wel = __fmul_rn(wlj, elj);
        wec = __fmul_rn(wc, ec);
    } else {
        fs = __fmul_rn(__fadd_rn(frlj, frc), r2inv);
        wel = elj;
        wec = ec;
    }
    fs = in ? fs : 0.0f;
    acc.elj = __fadd_rn(acc.elj, in ? wel : 0.0f);
    acc.ec = __fadd_rn(acc.ec, in ? wec : 0.0f);
    acc.fx = __fmaf_rn(-fs, dx, acc.fx);
    acc.fy = __fmaf_rn(-fs, dy, acc.fy);
    acc.fz = __fmaf_rn(-fs, dz, acc.fz);
    fjx = __fmaf_rn(fs, dx, fjx);  // F_j = -F_i
    fjy = __fmaf_rn(fs, dy, fjy);
    fjz = __fmaf_rn(fs, dz, fjz);
}

// ---------------------------------------------------------------------------
// Forward kernel (k_force) on cluster-pair tiles.
//
// One warp evaluates one listed cluster pair (I, J) at a time as an 8 x 8
// tile: lane = jj + 8 ih holds j atom jj of J and the i atoms ih and ih + 4
// of I, so every lane computes two pairs and the tile needs no compaction:
// pairs beyond the cutoff (and excluded pairs, padding) are evaluated and
// masked.  The force on i stays in the lane's registers for the whole work
// unit; the force on j (two pairs per lane) is summed over the 4 lanes of
// that j atom with shuffles and added to the global 64-bit fixed-point sums,
// one atomic per atom and component, as is the force on i (summed over its 8
// lanes) when the unit is done.  The FP32 sums run in a fixed order and meet
// only in integer sums, so results are run-to-run bit-identical.  A
// cluster's half list is cut into `parts` work units, which the warps of a
// persistent grid claim from a counter (dynamic balance of the uneven list
// lengths), the next claim issued while the current unit runs.  Each batch
// of up to 32 entries has the listed clusters' atoms staged in the warp's
// shared memory (cp.async) and is then walked, plain entries first.
constexpr int kTileWarps = 8;            // warps per block of the tile kernel
#ifndef ACENB_TILE_MIN_BLOCKS
#define ACENB_TILE_MIN_BLOCKS 3          // resident blocks per SM the register budget is cut for
#endif
constexpr float kFarCoord = 3.0e18f;     // i-side padding: far from every atom and from the j-side padding

// One i atom of a lane: coordinates, ke q_i, type row.
struct TileI {
    float x, y, z, q;
    int trow;
    int orig;  // caller index (pair export)
};

__device__ __forceinline__ TileI load_tile_i(const ForceArgs &A, long long slot, int T, bool debug)
{
    float4 p = __ldg(A.xyzq + slot);
    if (!is_real_coord(p.x)) p.x = p.y = p.z = kFarCoord;
    TileI t;
    t.x = p.x;
    t.y = p.y;
    t.z = p.z;
    t.q = p.w * A.P.ke;
    t.trow = __ldg(A.tslot + slot) * T;
    t.orig = debug ? __ldg(A.perm + slot) : -1;
    return t;
}

// Fixed-point value (2^32) of an FP32 sum; a value too large for the sums
// (or not finite) adds zero and sets ovf.
__device__ __forceinline__ long long tile_fixed(float f, bool &ovf)
{
    const bool ok = fabsf(f) < 67108864.0f;
    ovf = ovf || !ok;
    return __float2ll_rn((ok ? f : 0.0f) * 4294967296.0f);
}

// Membership of one pair of a tile: the i atom at its image for the entry's
// shift code (IMG: x_i - L on axes with code 2; the j side was shifted by
// the caller), d = x_j - x_i and the FP32 predicate r2 < rc2 of the other
// kernels.
template <bool IMG>
__device__ __forceinline__ bool tile_member(const ForceArgs &A, const TileI &ti, uint32_t code, float4 pj, float Lx,
                                            float Ly, float Lz, float &dx, float &dy, float &dz, float &r2)
{
    float ax = ti.x, ay = ti.y, az = ti.z;
    if (IMG) {
        if ((code & 3u) == 2u) ax = __fsub_rn(ax, Lx);
        if (((code >> 2) & 3u) == 2u) ay = __fsub_rn(ay, Ly);
        if ((code >> 4) == 2u) az = __fsub_rn(az, Lz);
    }
    r2 = disp_r2(pj.x, pj.y, pj.z, ax, ay, az, dx, dy, dz);
    return r2 < A.P.rc2;
}

// Masked evaluation of one pair of a tile (see eval_pair); the force on j
// is added to fj.
template <int RAD, bool SPECIAL, bool DEBUG>
__device__ __forceinline__ void tile_eval(const ForceArgs &A, const float4 *__restrict__ lj, const TileI &ti, bool in,
                                          float dx, float dy, float dz, float r2, float4 pj, int tj, bool is14,
                                          int jorig, Acc &acc, float &fjx, float &fjy, float &fjz)
{
    if (DEBUG && in) {
        atomicAdd((unsigned long long *)&A.dbg_n[0], 1ull);
        const long long q = (long long)atomicAdd((unsigned long long *)&A.dbg_n[1], 1ull);
        if (q < A.dbg_cap) {
            A.dbg_ij[2 * q] = min(ti.orig, jorig);
            A.dbg_ij[2 * q + 1] = max(ti.orig, jorig);
        }
    }
    // only a special entry can hold r2 = 0 (an atom and itself, masked)
    eval_pair<RAD, SPECIAL>(A.P, lj, A.rtab, ti.trow, ti.q, in, dx, dy, dz, SPECIAL ? (in ? r2 : 1.0f) : r2, pj.w, tj,
                            is14, acc, fjx, fjy, fjz);
}

// One listed cluster J against the lane's two i atoms.  The tile's i atoms
// are z-sorted, so the lower half (atoms 0..3, pair A of every lane) and the
// upper half (4..7, pair B) are often not both within the cutoff of J: the
// membership of both pairs comes first, and the radial arithmetic of a half
// runs only when one of its 32 pairs is in range (warp vote).  SPECIAL
// entries are I's own cluster (pairs j > i only) and entries flagged as
// holding a topology partner (exclusions removed, 1-4 pairs scaled); IMG
// entries have a periodic shift code.  (Each kind has its own code: the
// plain kind, most entries, then carries no weights or image selects.)
template <int RAD, bool VIRIAL, bool DEBUG, bool SPECIAL, bool IMG>
__device__ __forceinline__ void tile_entry(const ForceArgs &A, const float4 *__restrict__ lj,
                                           const int *__restrict__ spart, int I, uint32_t ent, float4 pj, int tj,
                                           const TileI &ia, const TileI &ib, int jj, int ih, float Lx, float Ly,
                                           float Lz, Acc &acA, Acc &acB, float (&wimg)[6], bool &ovf)
{
    const int J = (int)(ent & kJMask);
    const uint32_t code = IMG ? (ent >> kShiftBit) & 0x3Fu : 0u;
    if (IMG) {  // j-side images (code 1): fl(x_j - L), as the other kernels stage them
        if ((code & 3u) == 1u) pj.x = __fsub_rn(pj.x, Lx);
        if (((code >> 2) & 3u) == 1u) pj.y = __fsub_rn(pj.y, Ly);
        if ((code >> 4) == 1u) pj.z = __fsub_rn(pj.z, Lz);
    }
    float dxA, dyA, dzA, r2A, dxB, dyB, dzB, r2B;
    bool inA = tile_member<IMG>(A, ia, code, pj, Lx, Ly, Lz, dxA, dyA, dzA, r2A);
    bool inB = tile_member<IMG>(A, ib, code, pj, Lx, Ly, Lz, dxB, dyB, dzB, r2B);
    bool s14A = false, s14B = false;
    if (SPECIAL) {
        if (J == I && code == 0u) {
            inA = inA && jj > ih;
            inB = inB && jj > ih + 4;
        }
        if (ent & kExclFlag) {
            const int jslot = J * kCluster + jj;
            for (int m = 0; m < A.K; ++m) {
                const int pa = spart[ih * A.K + m], pb = spart[(ih + 4) * A.K + m];
                if (pa >= 0 && (pa >> 1) == jslot) {
                    if (pa & 1) s14A = true;
                    else inA = false;
                }
                if (pb >= 0 && (pb >> 1) == jslot) {
                    if (pb & 1) s14B = true;
                    else inB = false;
                }
            }
        }
    }
    const bool anyA = __any_sync(kFull, inA), anyB = __any_sync(kFull, inB);
    if (!anyA && !anyB) return;
    const int jorig = DEBUG ? __ldg(A.perm + (long long)J * kCluster + jj) : -1;
    float fjx = 0.0f, fjy = 0.0f, fjz = 0.0f;
    if (anyA) tile_eval<RAD, SPECIAL, DEBUG>(A, lj, ia, inA, dxA, dyA, dzA, r2A, pj, tj, s14A, jorig, acA, fjx, fjy, fjz);
    if (anyB) tile_eval<RAD, SPECIAL, DEBUG>(A, lj, ib, inB, dxB, dyB, dzB, r2B, pj, tj, s14B, jorig, acB, fjx, fjy, fjz);
    // the force on j atom jj: sum over its 4 lanes, then lanes ih = 0, 1, 2
    // add the x, y, z components
#pragma unroll
    for (int o = 8; o < 32; o <<= 1) {
        fjx = __fadd_rn(fjx, __shfl_xor_sync(kFull, fjx, o));
        fjy = __fadd_rn(fjy, __shfl_xor_sync(kFull, fjy, o));
        fjz = __fadd_rn(fjz, __shfl_xor_sync(kFull, fjz, o));
    }
    const float fc = ih == 0 ? fjx : (ih == 1 ? fjy : fjz);
    const long long fv = tile_fixed(fc, ovf);  // every lane (lane ih = 3 holds z again): no branch
    if (ih < 3) atomicAdd((unsigned long long *)&A.facc[24ll * J + 3 * jj + ih], (unsigned long long)fv);
    if (VIRIAL && IMG && ih == 0) {
        // periodic-image part of the virial: s (x) f_j with the entry's
        // shift s of j (code 1: -L, code 2: +L per axis)
        const uint32_t cx = code & 3u, cy = (code >> 2) & 3u, cz = code >> 4;
        const float sx = cx == 1u ? -Lx : (cx == 2u ? Lx : 0.0f);
        const float sy = cy == 1u ? -Ly : (cy == 2u ? Ly : 0.0f);
        const float sz = cz == 1u ? -Lz : (cz == 2u ? Lz : 0.0f);
        wimg[0] = __fmaf_rn(sx, fjx, wimg[0]);
        wimg[1] = __fmaf_rn(sy, fjy, wimg[1]);
        wimg[2] = __fmaf_rn(sz, fjz, wimg[2]);
        wimg[3] = __fmaf_rn(sx, fjy, wimg[3]);
        wimg[4] = __fmaf_rn(sx, fjz, wimg[4]);
        wimg[5] = __fmaf_rn(sy, fjz, wimg[5]);
    }
}

// The image virial of a work unit (FP32 per lane) to the warp's fixed-point
// sums (2^20): lane k < 6 holds component k in wv.  Rounded per unit, so the
// sums do not depend on which warp took which unit.
__device__ __forceinline__ void tile_virial_unit(float (&wimg)[6], long long &wv, int lane)
{
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        long long x = __float2ll_rn(wimg[k] * (float)kVirScale);
        wimg[k] = 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
        if (lane == k) wv += x;
    }
}

// Warp sums of a system's energies (2^32) and image virial (2^20); clears
// the per-lane sums.
template <bool VIRIAL>
__device__ __forceinline__ void tile_warp_sums(long long (&e)[2], long long &wv, long long (&out)[kTaskVals])
{
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        long long x = e[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
        out[k] = x;
    }
    if (VIRIAL)
#pragma unroll
        for (int k = 0; k < 6; ++k) out[2 + k] = __shfl_sync(kFull, wv, k);
    e[0] = e[1] = 0;
    wv = 0;
}

template <int RAD, bool VIRIAL, bool DEBUG>
__global__ void __launch_bounds__(kTileWarps * 32, ACENB_TILE_MIN_BLOCKS) k_force(ForceArgs A, int parts)
{
    pdl_entry();
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_val[kTileWarps][kTaskVals];
    __shared__ int s_sys[kTileWarps];
    const int T = A.P.n_types;
    const int K = A.K;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, jj = lane & 7, ih = lane >> 3;
    float4 *lj = reinterpret_cast<float4 *>(smem);  // (A, B, 12 A, 6 B) per type pair
    size_t off = (size_t)T * T * 16;
    int *spart = reinterpret_cast<int *>(smem + off) + w * kCluster * K;
    off += align16((size_t)kTileWarps * kCluster * K * 4);
    float4 *sjp = reinterpret_cast<float4 *>(smem + off) + w * 32 * kCluster;  // staged j coordinates + charges
    off += (size_t)kTileWarps * 32 * kCluster * 16;
    int *sjt = reinterpret_cast<int *>(smem + off) + w * 32 * kCluster;  // staged j types
    for (int k = threadIdx.x; k < T * T; k += blockDim.x) {
        const float2 ab = A.lj_tab[k];
        lj[k] = make_float4(ab.x, ab.y, 12.0f * ab.x, 6.0f * ab.y);
    }
    __syncthreads();
    const int n_units = A.counts[1] * parts;
    int cur_sys = -1;
    float Lx = 0.0f, Ly = 0.0f, Lz = 0.0f;
    long long esum[2] = {0, 0};  // per lane: fixed-point energies of the current system
    float wimg[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};  // image virial of the current unit
    long long wv = 0;  // lane k < 6: fixed-point image virial component k of the current system
    bool ovf = false;  // a j-force sum out of the fixed-point range
    int u = 0;
    if (lane == 0) u = atomicAdd(A.work, 1);
    u = __shfl_sync(kFull, u, 0);
    while (u < n_units) {
        int u_next = 0;
        if (lane == 0) u_next = atomicAdd(A.work, 1);  // claimed now, used after this unit
        const int I = u / parts, part = u - I * parts;
        const int sys_id = __ldg(A.clus_sys + I);
        if (sys_id != cur_sys) {
            if (!DEBUG && cur_sys >= 0) {
                long long v[kTaskVals];
                tile_warp_sums<VIRIAL>(esum, wv, v);
                if (lane == 0)
                    for (int k = 0; k < (VIRIAL ? kTaskVals : 2); ++k)
                        if (v[k]) atomicAdd((unsigned long long *)&A.sys_acc[cur_sys * kTaskVals + k], (unsigned long long)v[k]);
            }
            cur_sys = sys_id;
            Lx = A.sys[sys_id].L[0];
            Ly = A.sys[sys_id].L[1];
            Lz = A.sys[sys_id].L[2];
        }
        const int nA = __ldg(A.list_n + I);
        const int per = (nA + parts - 1) / parts;
        const int e_begin = min(nA, part * per), e_end = min(nA, e_begin + per);
        if (e_begin < e_end) {
            const long long s0 = (long long)I * kCluster;
            const TileI ia = load_tile_i(A, s0 + ih, T, DEBUG);
            const TileI ib = load_tile_i(A, s0 + ih + 4, T, DEBUG);
            for (int t = lane; t < kCluster * K; t += 32) spart[t] = __ldg(A.pslot + s0 * K + t);
            __syncwarp();
            Acc acA = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, acB = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            const uint32_t *row = A.list + (long long)I * A.cap;
            uint32_t ents = lane < e_end - e_begin ? __ldg(row + e_begin + lane) : 0u;
            bool unit_img = false;  // the unit holds an image entry (warp uniform)
            for (int e0 = e_begin; e0 < e_end; e0 += 32) {
                const int ne = min(32, e_end - e0);
                const uint32_t cur_ents = ents;
                if (e0 + 32 < e_end)  // the next 32 entries, ahead of use
                    ents = lane < e_end - e0 - 32 ? __ldg(row + e0 + 32 + lane) : 0u;
                // stage the batch's j atoms: lane k copies the 8 coordinates
                // and types of entry k (atom a at swz(k, a): conflict-free
                // reads of one entry's 8 atoms)
                if (lane < ne) {
                    const long long jb = (long long)(cur_ents & kJMask) * kCluster;
#pragma unroll
                    for (int a = 0; a < kCluster; ++a) {
                        cp_async16(sjp + swz(lane, a), A.xyzq + jb + a);
                        cp_async4(sjt + swz(lane, a), A.tslot + jb + a);
                    }
                }
                cp_async_wait_all();
                __syncwarp();
                // the batch's plain entries first (no image code, no partner
                // flag, not I itself: one code path without a dispatch), then
                // the others
                const bool my_img = ((cur_ents >> kShiftBit) & 0x3Fu) != 0u;
                const bool my_spc = (cur_ents & kExclFlag) != 0u || ((int)(cur_ents & kJMask) == I && !my_img);
                const unsigned in_batch = lane < ne;
                unsigned plain = __ballot_sync(kFull, in_batch && !my_img && !my_spc);
                unsigned other = __ballot_sync(kFull, in_batch) & ~plain;
                unit_img = unit_img || __ballot_sync(kFull, in_batch && my_img) != 0u;
                while (plain) {
                    const int k = __ffs(plain) - 1;
                    plain &= plain - 1u;
                    const uint32_t ent = __shfl_sync(kFull, cur_ents, k);
                    tile_entry<RAD, VIRIAL, DEBUG, false, false>(A, lj, spart, I, ent, sjp[swz(k, jj)],
                                                                sjt[swz(k, jj)], ia, ib, jj, ih, Lx, Ly, Lz, acA, acB,
                                                                wimg, ovf);
                }
                while (other) {
                    const int k = __ffs(other) - 1;
                    other &= other - 1u;
                    const uint32_t ent = __shfl_sync(kFull, cur_ents, k);
                    const float4 pj = sjp[swz(k, jj)];
                    const int tj = sjt[swz(k, jj)];
                    const bool img = ((ent >> kShiftBit) & 0x3Fu) != 0u;
                    const bool special = (ent & kExclFlag) != 0u || ((int)(ent & kJMask) == I && !img);
                    if (img) {
                        if (special)
                            tile_entry<RAD, VIRIAL, DEBUG, true, true>(A, lj, spart, I, ent, pj, tj, ia, ib, jj, ih,
                                                                      Lx, Ly, Lz, acA, acB, wimg, ovf);
                        else
                            tile_entry<RAD, VIRIAL, DEBUG, false, true>(A, lj, spart, I, ent, pj, tj, ia, ib, jj, ih,
                                                                       Lx, Ly, Lz, acA, acB, wimg, ovf);
                    } else {
                        tile_entry<RAD, VIRIAL, DEBUG, true, false>(A, lj, spart, I, ent, pj, tj, ia, ib, jj, ih, Lx,
                                                                   Ly, Lz, acA, acB, wimg, ovf);
                    }
                }
                __syncwarp();  // the staging buffer is rewritten by the next batch
            }
            // force on the i atoms: the 8 lanes of each atom summed in FP32
            // (a fixed butterfly: every lane ends with the same bits), then
            // lanes jj < 3 add atom ih, jj = 3..5 atom ih + 4 in fixed point
            float v[6] = {acA.fx, acA.fy, acA.fz, acB.fx, acB.fy, acB.fz};
#pragma unroll
            for (int o = 1; o < 8; o <<= 1)
#pragma unroll
                for (int c = 0; c < 6; ++c) v[c] = __fadd_rn(v[c], __shfl_xor_sync(kFull, v[c], o));
            float mine = v[0];
#pragma unroll
            for (int c = 1; c < 6; ++c) mine = jj == c ? v[c] : mine;
            const long long fi = tile_fixed(mine, ovf);
            if (jj < 6 && fi != 0) {
                const long long slot = s0 + ih + (jj < 3 ? 0 : 4);
                atomicAdd((unsigned long long *)&A.facc[3 * slot + (jj < 3 ? jj : jj - 3)], (unsigned long long)fi);
            }
            esum[0] += tile_fixed(acA.elj, ovf) + tile_fixed(acB.elj, ovf);
            esum[1] += tile_fixed(acA.ec, ovf) + tile_fixed(acB.ec, ovf);
            if (VIRIAL && unit_img) tile_virial_unit(wimg, wv, lane);  // image entries only add to wimg
            if (__any_sync(kFull, ovf)) {
                if (lane == 0) atomicOr(A.status, ST_OVERFLOW);
                ovf = false;
            }
            __syncwarp();  // spart is rewritten by the next unit
        }
        u = __shfl_sync(kFull, u_next, 0);
    }
    if (DEBUG) return;
    // the block's sums: one atomic per value for the system most warps
    // ended in, direct atomics for any other
    long long v[kTaskVals];
    tile_warp_sums<VIRIAL>(esum, wv, v);
    if (lane == 0) {
        s_sys[w] = cur_sys;
        for (int k = 0; k < kTaskVals; ++k) s_val[w][k] = k < (VIRIAL ? kTaskVals : 2) ? v[k] : 0;
    }
    __syncthreads();
    if (threadIdx.x < (VIRIAL ? kTaskVals : 2)) {
        const int k = threadIdx.x;
        const int nw = blockDim.x >> 5;
        int base = -1;
        long long sum = 0;
        for (int q = 0; q < nw; ++q) {
            const int sq = s_sys[q];
            if (sq < 0) continue;
            if (base < 0) base = sq;
            if (sq == base) sum += s_val[q][k];
            else if (s_val[q][k]) atomicAdd((unsigned long long *)&A.sys_acc[sq * kTaskVals + k], (unsigned long long)s_val[q][k]);
        }
        if (base >= 0 && sum) atomicAdd((unsigned long long *)&A.sys_acc[base * kTaskVals + k], (unsigned long long)sum);
    }
}

// ---------------------------------------------------------------------------
// Adjoint kernel on cluster-pair tiles (k_adjoint): the forward
// kernel's tiles, half-tile votes, work units and staging, with the pair
// adjoint of eval_pair_adj.  The j-side terms of an entry (dL/dx_j, dL/dq_j)
// are summed over the 4 lanes of each j atom and lane ih adds component ih
// (x, y, z, q) to the fixed-point sums; the i-side terms stay in registers
// for the unit; the type-pair gradients go to a block table in shared
// memory (integer atomics) flushed at the end.
constexpr int kAdjWarps = 4;             // warps per block of the adjoint tile kernel

// One instance serves every kind of entry (special and image entries as
// uniform branches): the pair adjoint is long, and an instance per kind, as
// in the forward kernel, overflowed the instruction cache (0.188 against
// 0.168 ms per adjoint step).
template <int RAD>
__device__ __forceinline__ void tile_adj_entry(bool special, bool img, const ForceArgs &A, const AdjTables &tab,
                                               const int *__restrict__ spart, int I, uint32_t ent, float4 pj, int tj,
                                               float4 gj, const TileI &ia, const TileI &ib, float4 gia, float4 gib,
                                               float gE_lj, float gE_c, int jj, int ih, float Lx, float Ly, float Lz,
                                               AccAdj &acA, AccAdj &acB, bool &ovf)
{
    const int J = (int)(ent & kJMask);
    const uint32_t code = img ? (ent >> kShiftBit) & 0x3Fu : 0u;
    if (img) {
        if ((code & 3u) == 1u) pj.x = __fsub_rn(pj.x, Lx);
        if (((code >> 2) & 3u) == 1u) pj.y = __fsub_rn(pj.y, Ly);
        if ((code >> 4) == 1u) pj.z = __fsub_rn(pj.z, Lz);
    }
    float dxA, dyA, dzA, r2A, dxB, dyB, dzB, r2B;
    bool inA = img ? tile_member<true>(A, ia, code, pj, Lx, Ly, Lz, dxA, dyA, dzA, r2A)
                   : tile_member<false>(A, ia, code, pj, Lx, Ly, Lz, dxA, dyA, dzA, r2A);
    bool inB = img ? tile_member<true>(A, ib, code, pj, Lx, Ly, Lz, dxB, dyB, dzB, r2B)
                   : tile_member<false>(A, ib, code, pj, Lx, Ly, Lz, dxB, dyB, dzB, r2B);
    bool s14A = false, s14B = false;
    if (special) {
        if (J == I && code == 0u) {
            inA = inA && jj > ih;
            inB = inB && jj > ih + 4;
        }
        if (ent & kExclFlag) {
            const int jslot = J * kCluster + jj;
            for (int m = 0; m < A.K; ++m) {
                const int pa = spart[ih * A.K + m], pb = spart[(ih + 4) * A.K + m];
                if (pa >= 0 && (pa >> 1) == jslot) {
                    if (pa & 1) s14A = true;
                    else inA = false;
                }
                if (pb >= 0 && (pb >> 1) == jslot) {
                    if (pb & 1) s14B = true;
                    else inB = false;
                }
            }
        }
    }
    const bool anyA = __any_sync(kFull, inA), anyB = __any_sync(kFull, inB);
    if (!anyA && !anyB) return;
    float jx = 0.0f, jy = 0.0f, jz = 0.0f, jq = 0.0f;
    if (anyA) {
        float a, b, c, d, ds, de;
        eval_pair_adj<RAD == 1>(A.P, tab, ia.trow, ia.q, gia.x, gia.y, gia.z, gE_lj, gE_c, inA, dxA, dyA, dzA,
                                inA ? r2A : 1.0f, pj.w, tj, gj, s14A, A.status, acA, a, b, c, d, ds, de);
        add_type_grads(tab, inA ? ia.trow + tj : -1, ds, de, A.status);
        jx = a;
        jy = b;
        jz = c;
        jq = d;
    }
    if (anyB) {
        float a, b, c, d, ds, de;
        eval_pair_adj<RAD == 1>(A.P, tab, ib.trow, ib.q, gib.x, gib.y, gib.z, gE_lj, gE_c, inB, dxB, dyB, dzB,
                                inB ? r2B : 1.0f, pj.w, tj, gj, s14B, A.status, acB, a, b, c, d, ds, de);
        add_type_grads(tab, inB ? ib.trow + tj : -1, ds, de, A.status);
        jx = __fadd_rn(jx, a);
        jy = __fadd_rn(jy, b);
        jz = __fadd_rn(jz, c);
        jq = __fadd_rn(jq, d);
    }
#pragma unroll
    for (int o = 8; o < 32; o <<= 1) {
        jx = __fadd_rn(jx, __shfl_xor_sync(kFull, jx, o));
        jy = __fadd_rn(jy, __shfl_xor_sync(kFull, jy, o));
        jz = __fadd_rn(jz, __shfl_xor_sync(kFull, jz, o));
        jq = __fadd_rn(jq, __shfl_xor_sync(kFull, jq, o));
    }
    const float gc = ih == 0 ? jx : (ih == 1 ? jy : (ih == 2 ? jz : jq));
    atomicAdd((unsigned long long *)&A.gacc[32ll * J + 4 * jj + ih], (unsigned long long)tile_fixed(gc, ovf));
}

template <int RAD>
__global__ void __launch_bounds__(kAdjWarps * 32) k_adjoint(ForceArgs A, int parts)
{
    pdl_entry();
    extern __shared__ __align__(16) unsigned char smem[];
    const int T = A.P.n_types;
    const int K = A.K;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, jj = lane & 7, ih = lane >> 3;
    size_t off = 0;
    unsigned long long *tacc = reinterpret_cast<unsigned long long *>(smem + off);
    off += (size_t)T * T * 16;
    float4 *ljd = reinterpret_cast<float4 *>(smem + off);
    off += (size_t)T * T * 16;
    float2 *lj = reinterpret_cast<float2 *>(smem + off);
    off += align16((size_t)T * T * 8);
    int *spart = reinterpret_cast<int *>(smem + off) + w * kCluster * K;
    off += align16((size_t)kAdjWarps * kCluster * K * 4);
    float4 *sjp = reinterpret_cast<float4 *>(smem + off) + w * 32 * kCluster;  // staged j coordinates + charges
    off += (size_t)kAdjWarps * 32 * kCluster * 16;
    float4 *sjg = reinterpret_cast<float4 *>(smem + off) + w * 32 * kCluster;  // staged j dL/dF
    off += (size_t)kAdjWarps * 32 * kCluster * 16;
    int *sjt = reinterpret_cast<int *>(smem + off) + w * 32 * kCluster;  // staged j types
    for (int k = threadIdx.x; k < T * T; k += blockDim.x) {
        lj[k] = A.lj_tab[k];
        ljd[k] = A.lj_d[k];
        tacc[2 * k] = 0ull;
        tacc[2 * k + 1] = 0ull;
    }
    __syncthreads();
    const AdjTables tab{lj, ljd, tacc};
    const int n_units = A.counts[1] * parts;
    int cur_sys = -1;
    float Lx = 0.0f, Ly = 0.0f, Lz = 0.0f, gE_lj = 0.0f, gE_c = 0.0f;
    bool ovf = false;
    int u = 0;
    if (lane == 0) u = atomicAdd(A.work, 1);
    u = __shfl_sync(kFull, u, 0);
    while (u < n_units) {
        int u_next = 0;
        if (lane == 0) u_next = atomicAdd(A.work, 1);
        const int I = u / parts, part = u - I * parts;
        const int sys_id = __ldg(A.clus_sys + I);
        if (sys_id != cur_sys) {
            cur_sys = sys_id;
            Lx = A.sys[sys_id].L[0];
            Ly = A.sys[sys_id].L[1];
            Lz = A.sys[sys_id].L[2];
            gE_lj = A.dLdE ? (float)A.dLdE[2 * sys_id] : 0.0f;
            gE_c = A.dLdE ? (float)A.dLdE[2 * sys_id + 1] : 0.0f;
        }
        const int nA = __ldg(A.list_n + I);
        const int per = (nA + parts - 1) / parts;
        const int e_begin = min(nA, part * per), e_end = min(nA, e_begin + per);
        if (e_begin < e_end) {
            const long long s0 = (long long)I * kCluster;
            const TileI ia = load_tile_i(A, s0 + ih, T, false);
            const TileI ib = load_tile_i(A, s0 + ih + 4, T, false);
            const float4 gia = __ldg(A.gslot + s0 + ih), gib = __ldg(A.gslot + s0 + ih + 4);
            for (int t = lane; t < kCluster * K; t += 32) spart[t] = __ldg(A.pslot + s0 * K + t);
            __syncwarp();
            AccAdj acA = {0.0f, 0.0f, 0.0f, 0.0f}, acB = {0.0f, 0.0f, 0.0f, 0.0f};
            const uint32_t *row = A.list + (long long)I * A.cap;
            uint32_t ents = lane < e_end - e_begin ? __ldg(row + e_begin + lane) : 0u;
            for (int e0 = e_begin; e0 < e_end; e0 += 32) {
                const int ne = min(32, e_end - e0);
                const uint32_t cur_ents = ents;
                if (e0 + 32 < e_end) ents = lane < e_end - e0 - 32 ? __ldg(row + e0 + 32 + lane) : 0u;
                if (lane < ne) {
                    const long long jb = (long long)(cur_ents & kJMask) * kCluster;
#pragma unroll
                    for (int a = 0; a < kCluster; ++a) {
                        cp_async16(sjp + swz(lane, a), A.xyzq + jb + a);
                        cp_async16(sjg + swz(lane, a), A.gslot + jb + a);
                        cp_async4(sjt + swz(lane, a), A.tslot + jb + a);
                    }
                }
                cp_async_wait_all();
                __syncwarp();
                for (int k = 0; k < ne; ++k) {
                    const uint32_t ent = __shfl_sync(kFull, cur_ents, k);
                    const float4 pj = sjp[swz(k, jj)];
                    const float4 gj = sjg[swz(k, jj)];
                    const int tj = sjt[swz(k, jj)];
                    const bool img = ((ent >> kShiftBit) & 0x3Fu) != 0u;
                    const bool special = (ent & kExclFlag) != 0u || ((int)(ent & kJMask) == I && !img);
                    tile_adj_entry<RAD>(special, img, A, tab, spart, I, ent, pj, tj, gj, ia, ib, gia, gib, gE_lj, gE_c,
                                        jj, ih, Lx, Ly, Lz, acA, acB, ovf);
                }
                __syncwarp();  // the staging buffers are rewritten by the next batch
            }
            // i-side terms: the 8 lanes of each atom summed in FP32 (fixed
            // butterfly), then lane jj < 4 adds component jj of atom ih,
            // jj >= 4 component jj - 4 of atom ih + 4, in fixed point
            float v[8] = {acA.dx, acA.dy, acA.dz, acA.dq, acB.dx, acB.dy, acB.dz, acB.dq};
#pragma unroll
            for (int o = 1; o < 8; o <<= 1)
#pragma unroll
                for (int c = 0; c < 8; ++c) v[c] = __fadd_rn(v[c], __shfl_xor_sync(kFull, v[c], o));
            float vm = v[0];
#pragma unroll
            for (int c = 1; c < 8; ++c) vm = jj == c ? v[c] : vm;
            const long long mine = tile_fixed(vm, ovf);
            if (mine != 0) {
                const long long slot = s0 + ih + (jj < 4 ? 0 : 4);
                atomicAdd((unsigned long long *)&A.gacc[4 * slot + (jj & 3)], (unsigned long long)mine);
            }
            if (__any_sync(kFull, ovf)) {
                if (lane == 0) atomicOr(A.status, ST_OVERFLOW);
                ovf = false;
            }
            __syncwarp();  // spart is rewritten by the next unit
        }
        u = __shfl_sync(kFull, u_next, 0);
    }
    // block table of parameter gradients -> global (integer sums)
    __syncthreads();
    for (int k = threadIdx.x; k < 2 * T * T; k += blockDim.x)
        if (tacc[k]) atomicAdd((unsigned long long *)&A.tab_acc[k], tacc[k]);
}

// Gather charges and types into sorted order and check that the positions
// are those of the last build.
__global__ void k_pack(int slot_cap, const int *__restrict__ counts, const int *__restrict__ perm,
                       float4 *__restrict__ xyzq, int *__restrict__ tslot, const float *__restrict__ pos,
                       const float *__restrict__ q, const int *__restrict__ type, const SysDesc *__restrict__ sys,
                       const int *__restrict__ atom_sys, int T, int *__restrict__ status,
                       long long *__restrict__ facc, long long *__restrict__ sys_acc, int n_acc,
                       int *__restrict__ work)
{
    pdl_entry();
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (work && s == 0) *work = 0;  // the force kernel's work-unit counter
    // zero the force kernel's fixed-point sums (forward calls pass them)
    if (facc && s < slot_cap) {
        facc[3ll * s] = 0;
        facc[3ll * s + 1] = 0;
        facc[3ll * s + 2] = 0;
    }
    if (sys_acc && s < n_acc) sys_acc[s] = 0;
    if (s >= slot_cap || s >= counts[0]) return;
    int a = perm[s];
    if (a < 0) return;
    const SysDesc &S = sys[atom_sys[a]];
    float4 p = xyzq[s];
    float x = wrap_coord(pos[3 * (long long)a], S.L[0]);
    float y = wrap_coord(pos[3 * (long long)a + 1], S.L[1]);
    float z = wrap_coord(pos[3 * (long long)a + 2], S.L[2]);
    if (x != p.x || y != p.y || z != p.z) atomicOr(status, ST_STALE);
    int t = type[a];
    if (t < 0 || t >= T) {
        atomicOr(status, ST_BADTYPE);
        t = 0;
    }
    xyzq[s] = make_float4(p.x, p.y, p.z, q[a]);
    tslot[s] = t;
}

// Add a warp's per-lane fixed-point virial terms (lanes with sys < 0 hold
// none) to the per-system sums: one reduction and 6 atomics per distinct
// system among the lanes, into the block's shared sums when the system is
// the block's (blk_sys), else straight to global memory.
__device__ __forceinline__ void flush_virial_warp(long long *w, int sys, long long *sys_acc, int blk_sys,
                                                  unsigned long long *blk_w)
{
    unsigned rem = __ballot_sync(kFull, sys >= 0);
    while (rem) {
        const int leader = __ffs(rem) - 1;
        const int cs = __shfl_sync(kFull, sys, leader);
        const bool mine = sys == cs;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            long long x = mine ? w[k] : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
            if ((int)(threadIdx.x & 31) == leader) {
                if (cs == blk_sys) atomicAdd(&blk_w[k], (unsigned long long)x);
                else atomicAdd((unsigned long long *)&sys_acc[cs * kTaskVals + 2 + k], (unsigned long long)x);
            }
        }
        rem &= ~__ballot_sync(kFull, mine);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) w[k] = 0;
}

// Fixed-point forces (sorted order) to FP32 in the caller's order.  With
// VIRIAL, also the atom part of the virial: for central pair forces
// W_ab = sum_pairs d_a f_b (d = x_j' - x_i, f the force on j) equals
// sum_atoms x_a F_b over the wrapped coordinates x and total forces F, plus
// the periodic-image terms added by the force kernel.  Each atom's terms are
// rounded to the 2^20 fixed-point grid in FP64 and summed as integers per
// thread (grid-stride loop, slots in system order) and per warp.
template <bool VIRIAL>
__global__ void __launch_bounds__(256) k_unpack_forces(int slot_cap, int *__restrict__ counts,
                                                       const int *__restrict__ perm, const long long *__restrict__ facc,
                                                       float *__restrict__ F, const float4 *__restrict__ xyzq,
                                                       const int *__restrict__ clus_sys, long long *__restrict__ sys_acc,
                                                       int n_sys, double *__restrict__ energy, double *__restrict__ virial,
                                                       const long long *__restrict__ pme_f,
                                                       const long long *__restrict__ pme_s, double pme_self)
{
    pdl_entry();
    const int nslots = min(slot_cap, counts[0]);
    long long w[6] = {0, 0, 0, 0, 0, 0};
    int wsys = -1;
    __shared__ unsigned long long blk_w[6];
    __shared__ int blk_sys;
    if (VIRIAL) {
        if (threadIdx.x < 6) blk_w[threadIdx.x] = 0ull;
        if (threadIdx.x == 0) {
            const int s0 = blockIdx.x * blockDim.x;
            blk_sys = s0 < nslots ? clus_sys[s0 / kCluster] : -1;
        }
        __syncthreads();
    }
    for (int s0 = blockIdx.x * blockDim.x; s0 < nslots; s0 += gridDim.x * blockDim.x) {
        const int s = s0 + threadIdx.x;
        const int a = s < nslots ? perm[s] : -1;
        int sys = -1;
        long long c[6];
        if (a >= 0) {
            const long long v0 = facc[3ll * s], v1 = facc[3ll * s + 1], v2 = facc[3ll * s + 2];
            const float sc = 2.3283064365386963e-10f;  // 2^-32
            // PME forces (same slot order) join the sum before the one
            // rounding; the atom part of the virial is the short-range forces' alone
            const long long p0 = pme_f ? pme_f[3ll * s] : 0, p1 = pme_f ? pme_f[3ll * s + 1] : 0,
                            p2 = pme_f ? pme_f[3ll * s + 2] : 0;
            F[3ll * a] = __ll2float_rn(v0 + p0) * sc;
            F[3ll * a + 1] = __ll2float_rn(v1 + p1) * sc;
            F[3ll * a + 2] = __ll2float_rn(v2 + p2) * sc;
            if (VIRIAL) {
                const double r = kVirScale / kFixScale;
                const double fx = (double)v0 * r, fy = (double)v1 * r, fz = (double)v2 * r;
                const float4 x = xyzq[s];
                c[0] = __double2ll_rn(x.x * fx);
                c[1] = __double2ll_rn(x.y * fy);
                c[2] = __double2ll_rn(x.z * fz);
                c[3] = __double2ll_rn(x.x * fy);
                c[4] = __double2ll_rn(x.x * fz);
                c[5] = __double2ll_rn(x.y * fz);
                sys = clus_sys[s / kCluster];
            }
        }
        if (VIRIAL) {
            // slots come in system order: flush a lane's sums before it moves on
            if (__any_sync(kFull, sys >= 0 && wsys >= 0 && sys != wsys)) {
                flush_virial_warp(w, wsys, sys_acc, blk_sys, blk_w);
                wsys = -1;
            }
            if (sys >= 0) {
                wsys = sys;
#pragma unroll
                for (int k = 0; k < 6; ++k) w[k] += c[k];
            }
        }
    }
    if (VIRIAL) {
        flush_virial_warp(w, wsys, sys_acc, blk_sys, blk_w);
        __syncthreads();
        if (threadIdx.x < 6 && blk_sys >= 0 && blk_w[threadIdx.x])
            atomicAdd((unsigned long long *)&sys_acc[blk_sys * kTaskVals + 2 + threadIdx.x], blk_w[threadIdx.x]);
    }
    if (!energy && !virial) return;
    // the last block to finish converts the per-system sums (counts[2] is the
    // completion ticket: zero on entry, reset here)
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&counts[2], 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int i = threadIdx.x; i < n_sys * kTaskVals; i += blockDim.x) {
        const int sy = i / kTaskVals, k = i % kTaskVals;
        long long raw = __ldcg(&sys_acc[i]);
        if (pme_s) {  // single system: reciprocal + self + pair corrections join E_Coul and W
            if (k == 1)  // the self term from sum q^2 (scale 2^36) to the energy scale 2^32
                raw += __ldcg(&pme_s[0]) + __ldcg(&pme_s[2]) +
                       __double2ll_rn(pme_self * (double)__ldcg(&pme_s[1]) * (1.0 / 16.0));
            if (k >= 2) raw += __ldcg(&pme_s[1 + k]);
        }
        const double v = (double)raw * (k < 2 ? 1.0 / kFixScale : 1.0 / kVirScale);
        if (k < 2) {
            if (energy) energy[2 * sy + k] = v;
        } else if (virial) {
            virial[6 * sy + k - 2] = v;
        }
    }
    if (threadIdx.x == 0) counts[2] = 0;
}

// Adjoint sums (sorted order, fixed point) to FP32 dL/dx, dL/dq in the
// caller's order.
__global__ void k_unpack_adjoint(int slot_cap, const int *__restrict__ counts, const int *__restrict__ perm,
                                 const long long *__restrict__ gacc, float *__restrict__ dpos, float *__restrict__ dq)
{
    pdl_entry();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= slot_cap || s >= counts[0]) return;
    const int a = perm[s];
    if (a < 0) return;
    const float sc = 2.3283064365386963e-10f;  // 2^-32
    if (dpos) {
        dpos[3ll * a] = __ll2float_rn(gacc[4ll * s]) * sc;
        dpos[3ll * a + 1] = __ll2float_rn(gacc[4ll * s + 1]) * sc;
        dpos[3ll * a + 2] = __ll2float_rn(gacc[4ll * s + 2]) * sc;
    }
    if (dq) dq[a] = __ll2float_rn(gacc[4ll * s + 3]) * sc;
}

// Kernel function attributes belong to each device's context, so the
// shared-memory opt-in is made once per device (one bit per device in
// `done`; devices beyond 63 set it at every launch).  Concurrent first calls
// may both set it, which is harmless.
template <typename Kernel>
static void smem_optin_once(Kernel kernel, int device, int bytes, std::atomic<unsigned long long> &done)
{
    const unsigned long long bit = device >= 0 && device < 64 ? 1ull << device : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return;
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (bit) done.fetch_or(bit, std::memory_order_release);
}

size_t tile_smem_bytes(int T, int K)
{
    return (size_t)T * T * 16 + align16((size_t)kTileWarps * kCluster * K * 4) +
           (size_t)kTileWarps * 32 * kCluster * (16 + 4);
}

// beside_pme: the PME chain, forked before the list kernel, runs on its side
// stream during this kernel; the persistent grid then leaves one block slot
// per SM free, so that the PME kernels run alongside instead of after it.
template <int RAD, bool VIRIAL, bool DEBUG>
static void launch_force_t(nb_ctx *ctx, const ForceArgs &A, bool beside_pme)
{
    const size_t smem = tile_smem_bytes(A.P.n_types, A.K);
    static std::atomic<unsigned long long> optin{0};
    smem_optin_once(k_force<RAD, VIRIAL, DEBUG>, ctx->device, 200 * 1024, optin);
    // persistent grid: never more blocks than can be resident at once
    int resident = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_force<RAD, VIRIAL, DEBUG>, kTileWarps * 32, smem);
    const int per_sm = std::max(1, std::min(ctx->tune.blocks_per_sm, resident) - (beside_pme ? 1 : 0));
    const int parts = ctx->tune.list_split > 0 ? ctx->tune.list_split : kDefaultListSplit;
    launch_pdl(k_force<RAD, VIRIAL, DEBUG>, dim3(ctx->num_sms * per_sm), dim3(kTileWarps * 32), smem,
               ctx->stream, A, parts);
}

static ForceArgs make_args(nb_ctx *ctx)
{
    auto &d = ctx->d;
    ForceArgs A;
    memset(&A, 0, sizeof(A));
    A.sys = d.sys;
    A.counts = d.counts;
    A.work = d.counts + 3;
    A.xyzq = d.xyzq;
    A.tslot = d.tslot;
    A.perm = d.perm;
    A.clus_sys = d.clus_sys;
    A.list = d.list;
    A.list_n = d.list_n;
    A.pslot = d.pslot;
    A.cap = ctx->list_cap;
    A.K = ctx->K;
    A.lj_tab = d.lj_tab;
    A.rtab = d.rtab;
    A.sys_acc = d.sys_acc;
    A.status = d.status;
    A.dbg_n = d.dbg_n;
    A.dbg_ij = d.dbg_ij;
    A.dbg_cap = d.dbg_cap;
    A.P = ctx->pp;
    return A;
}

cudaError_t launch_pack(nb_ctx *ctx, const float *d_pos, const float *d_q, const int32_t *d_type, bool zero_sums)
{
    auto &d = ctx->d;
    const int tb = 256;
    const int S = (int)ctx->slot_cap;
    return launch_pdl(k_pack, dim3((S + tb - 1) / tb), dim3(tb), 0, ctx->stream, S, d.counts, d.perm, d.xyzq,
                      d.tslot, d_pos, d_q, d_type, d.sys, d.atom_sys, ctx->pp.n_types, d.status,
                      zero_sums ? d.facc : nullptr, zero_sums ? d.sys_acc : nullptr, kTaskVals * ctx->n_sys,
                      d.counts + 3);
}

cudaError_t launch_forces(nb_ctx *ctx, const float *d_pos, const float *d_q, const int32_t *d_type, float *d_F,
                          double *d_energy, double *d_virial, bool debug_pairs)
{
    auto &d = ctx->d;
    if (d_pos) {  // packs and zeroes the fixed-point sums
        cudaError_t e = launch_pack(ctx, d_pos, d_q, d_type, true);
        if (e != cudaSuccess) return e;
    } else {  // the debug pair export reuses the last packed values
        cudaMemsetAsync(d.sys_acc, 0, sizeof(long long) * kTaskVals * ctx->n_sys, ctx->stream);
        cudaMemsetAsync(d.facc, 0, sizeof(long long) * 3 * ctx->slot_cap, ctx->stream);
        cudaMemsetAsync(d.counts + 3, 0, sizeof(int), ctx->stream);
    }
    // smooth PME: forked onto its own stream so that it overlaps the
    // short-range kernel; joined back before the unpack reads its sums
    const bool pme = ctx->pme && d_pos && !debug_pairs;
    if (pme) {
        cudaError_t e = launch_pme_fork(ctx, d_pos, d_q);
        if (e != cudaSuccess) return e;
    }
    return launch_forces_packed(ctx, d_F, d_energy, d_virial, debug_pairs, pme, false);
}

cudaError_t launch_forces_packed(nb_ctx *ctx, float *d_F, double *d_energy, double *d_virial, bool debug_pairs,
                                 bool pme, bool beside_pme)
{
    auto &d = ctx->d;
    ForceArgs A = make_args(ctx);
    A.facc = d.facc;
    const bool ewald = ctx->pp.ewald != 0;
    const bool virial = d_virial != nullptr;
    const bool prof = ctx->profiling && ctx->prof_n < (int)ctx->prof_ev.size() / 2;
    if (prof) cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n], ctx->stream);
    if (debug_pairs) {  // the pair set does not depend on the radial functions
        if (ewald) launch_force_t<1, false, true>(ctx, A, beside_pme);
        else launch_force_t<0, false, true>(ctx, A, beside_pme);
    } else if (ctx->tab_n > 0) {
        if (virial) launch_force_t<2, true, false>(ctx, A, beside_pme);
        else launch_force_t<2, false, false>(ctx, A, beside_pme);
    } else if (ewald) {
        if (virial) launch_force_t<1, true, false>(ctx, A, beside_pme);
        else launch_force_t<1, false, false>(ctx, A, beside_pme);
    } else {
        if (virial) launch_force_t<0, true, false>(ctx, A, beside_pme);
        else launch_force_t<0, false, false>(ctx, A, beside_pme);
    }
    if (prof) {
        cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n + 1], ctx->stream);
        ctx->prof_n++;
    }
    if (pme) {
        cudaError_t e = launch_pme_join(ctx);
        if (e != cudaSuccess) return e;
    }
    {
        const int tb = 256;
        const int S = (int)ctx->slot_cap;
        const int blocks = std::max(1, std::min((S + tb - 1) / tb, 4 * ctx->num_sms));
        double *en = debug_pairs ? nullptr : d_energy;
        double *vi = debug_pairs ? nullptr : d_virial;
        const long long *pf = pme ? pme_forces_acc(ctx) : nullptr, *ps = pme ? pme_sums_acc(ctx) : nullptr;
        const double pself = pme ? pme_self_coef(ctx) : 0.0;
        if (virial)
            launch_pdl(k_unpack_forces<true>, dim3(blocks), dim3(tb), 0, ctx->stream, S, d.counts, d.perm, d.facc, d_F,
                       d.xyzq, d.clus_sys, d.sys_acc, ctx->n_sys, en, vi, pf, ps, pself);
        else
            launch_pdl(k_unpack_forces<false>, dim3(blocks), dim3(tb), 0, ctx->stream, S, d.counts, d.perm, d.facc,
                       d_F, d.xyzq, d.clus_sys, d.sys_acc, ctx->n_sys, en, vi, pf, ps, pself);
    }
    return cudaGetLastError();
}

size_t adjoint_smem_bytes(int T, int K)
{
    return (size_t)T * T * 32 + align16((size_t)T * T * 8) + align16((size_t)kAdjWarps * kCluster * K * 4) +
           (size_t)kAdjWarps * 32 * kCluster * (16 + 16 + 4);
}

template <int RAD>
static void launch_adjoint_t(nb_ctx *ctx, const ForceArgs &A)
{
    const size_t smem = adjoint_smem_bytes(A.P.n_types, A.K);
    static std::atomic<unsigned long long> optin{0};
    smem_optin_once(k_adjoint<RAD>, ctx->device, 220 * 1024, optin);
    int resident = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_adjoint<RAD>, kAdjWarps * 32, smem);
    const int parts = ctx->tune.list_split > 0 ? ctx->tune.list_split : kDefaultListSplit;
    launch_pdl(k_adjoint<RAD>, dim3(ctx->num_sms * std::max(1, resident)), dim3(kAdjWarps * 32), smem,
               ctx->stream, A, parts);
}

size_t force_smem_for(int T, int scap, int K)
{
    (void)scap;  // unused: the kernels stage per 32-entry batch
    return std::max(tile_smem_bytes(T, K), adjoint_smem_bytes(T, K));
}

cudaError_t launch_adjoint_tile(nb_ctx *ctx, const double *d_dLdE, float *d_dpos, float *d_dq)
{
    auto &d = ctx->d;
    ForceArgs A = make_args(ctx);
    A.gslot = d.gslot;
    A.dLdE = d_dLdE;
    A.lj_d = d.lj_d;
    A.tab_acc = d.tab_grad;
    A.gacc = d.gacc;
    if (ctx->pp.ewald) launch_adjoint_t<1>(ctx, A);
    else launch_adjoint_t<0>(ctx, A);
    const int tb = 256;
    const int S = (int)ctx->slot_cap;
    return launch_pdl(k_unpack_adjoint, dim3((S + tb - 1) / tb), dim3(tb), 0, ctx->stream, S, d.counts, d.perm,
                      d.gacc, d_dpos, d_dq);
}

// Test export of the pair arithmetic (nb_debug_pair_terms): pair k of the
// given lists evaluated by eval_pair exactly as the forward kernel does it
// (unit weights, d = x_j - x_i as given); out[2k] = (E_LJ, E_Coul, r2, 0),
// out[2k + 1] = the force on j.
template <int RAD>
__global__ void k_debug_pair_terms(PairParams P, const float2 *__restrict__ lj_tab, const float4 *__restrict__ rtab,
                                   long long n, const float4 *__restrict__ xi, const float4 *__restrict__ xj,
                                   const int *__restrict__ ti, const int *__restrict__ tj, float4 *__restrict__ out)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float4 a = xi[k], b = xj[k];
    const float2 ab = lj_tab[ti[k] * P.n_types + tj[k]];
    const float4 lj4 = make_float4(ab.x, ab.y, 12.0f * ab.x, 6.0f * ab.y);
    float dx, dy, dz;
    const float r2 = disp_r2(b.x, b.y, b.z, a.x, a.y, a.z, dx, dy, dz);
    Acc acc = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    float fjx = 0.0f, fjy = 0.0f, fjz = 0.0f;
    eval_pair<RAD, false>(P, &lj4, rtab, 0, a.w * P.ke, true, dx, dy, dz, r2, b.w, 0, false, acc, fjx, fjy, fjz);
    out[2 * k] = make_float4(acc.elj, acc.ec, r2, 0.0f);
    out[2 * k + 1] = make_float4(fjx, fjy, fjz, 0.0f);
}

cudaError_t launch_debug_pair_terms(nb_ctx *ctx, long long n, const float4 *xi, const float4 *xj, const int *ti,
                                    const int *tj, float4 *out)
{
    const int tb = 128;
    const unsigned g = (unsigned)((n + tb - 1) / tb);
    const PairParams &P = ctx->pp;
    if (ctx->tab_n > 0)
        k_debug_pair_terms<2><<<g, tb, 0, ctx->stream>>>(P, ctx->d.lj_tab, ctx->d.rtab, n, xi, xj, ti, tj, out);
    else if (P.ewald)
        k_debug_pair_terms<1><<<g, tb, 0, ctx->stream>>>(P, ctx->d.lj_tab, ctx->d.rtab, n, xi, xj, ti, tj, out);
    else
        k_debug_pair_terms<0><<<g, tb, 0, ctx->stream>>>(P, ctx->d.lj_tab, ctx->d.rtab, n, xi, xj, ti, tj, out);
    return cudaGetLastError();
}

}  // namespace acenb
