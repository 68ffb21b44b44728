// nb_force.cu - the non-bonded force kernels (section "Molecular dynamics on
// the GPU": the non-bonded kernel computes the full Lennard-Jones and
// electrostatic force on each particle).  The paper's kernel does not reuse
// the reciprocal force F_ji; here both kernels do (Newton's third law): every
// unique pair is evaluated once, from the i-group whose list holds it, and
// its contribution goes to both atoms as 64-bit fixed point (2^32), so the
// sums stay exact and order independent.
//
// Forward: k_force1 for i-groups of one cluster (one warp per listed
// cluster pair as an 8 x 8 tile, the i cluster and its forces in registers,
// forces on j summed over lanes; see the comment above k_force1), k_force<G>
// for groups of 4 or 8 clusters (the group's atoms and i-force partials in
// shared memory; see the comment above k_force).
//
// Adjoint: k_adjoint1 and k_adjoint<G>, the same tiles, work units and
// staging with the pair adjoint; the type-pair gradients go to a block table
// in shared memory.
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
    int *work;                // work-unit counter of the tile kernels (zeroed by k_pack or the column sort)
    const float4 *xyzq;
    const int *tslot;
    const int *perm;
    const int *clus_sys;
    const int2 *grp;          // [GC] i-groups: (first cluster, clusters)
    const uint2 *glist;       // [GC*cap] per group: its list, kListSegs segments of cap / kListSegs
    const int *glist_n;       // [GC*kListSegs] segment lengths
    const ulonglong2 *gmask;  // exclusion bitmask records of the flagged entries
    int cap;                  // entries per group list
    int K;
    const float4 *lj_tab;     // [T*T] (A, B, A - fl(A), B - fl(B))
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
// The LJ coefficients of the forward kernels in shared memory: lj (A, B,
// 12 A, 6 B) per type pair, followed by lo (the FP32 remainders of A, B).
template <int RAD, bool W14>
__device__ __forceinline__ float pair_fs(const PairParams &P, const float4 *__restrict__ lj,
                                         const float4 *__restrict__ rtab, int ti_row, float qi, bool in, float r2,
                                         float qj, int tj, bool is14, float &elj_acc, float &ec_acc)
{
    float rinv, r;
    pair_rinv(r2, rinv, r);
    const float r2inv = __fmul_rn(rinv, rinv);
    const float4 ab = lj[ti_row + tj];
    const float2 lo = reinterpret_cast<const float2 *>(lj + P.n_types * P.n_types)[ti_row + tj];
    float elj, frlj, ec, frc;
    if constexpr (RAD == 2)
        pair_radial_tab(P, rtab, r, ab.x, ab.y, lo, qi * qj, elj, frlj, ec, frc);
    else
        pair_radial<RAD == 1, true>(P, r2, r, rinv, r2inv, ab, lo, qi * qj, elj, frlj, ec, frc);
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
    elj_acc = __fadd_rn(elj_acc, in ? wel : 0.0f);
    ec_acc = __fadd_rn(ec_acc, in ? wec : 0.0f);
    return in ? fs : 0.0f;
}

// One pair: fs as above, the force on i subtracted from acc and the force on
// j added to fj with explicit FMA (bits independent of inlining).
template <int RAD, bool W14>
__device__ __forceinline__ void eval_pair(const PairParams &P, const float4 *__restrict__ lj,
                                          const float4 *__restrict__ rtab, int ti_row, float qi, bool in, float dx,
                                          float dy, float dz, float r2, float qj, int tj, bool is14, Acc &acc,
                                          float &fjx, float &fjy, float &fjz)
{
    const float fs = pair_fs<RAD, W14>(P, lj, rtab, ti_row, qi, in, r2, qj, tj, is14, acc.elj, acc.ec);
    acc.fx = __fmaf_rn(-fs, dx, acc.fx);
    acc.fy = __fmaf_rn(-fs, dy, acc.fy);
    acc.fz = __fmaf_rn(-fs, dz, acc.fz);
    fjx = __fmaf_rn(fs, dx, fjx);  // F_j = -F_i
    fjy = __fmaf_rn(fs, dy, fjy);
    fjz = __fmaf_rn(fs, dz, fjz);
}

// ---------------------------------------------------------------------------
// Pair export of the debug instantiation: every evaluated pair inside the
// cutoff and not excluded, as caller indices (i < j).
__device__ __forceinline__ void record_pair(const ForceArgs &A, int io, int jo)
{
    atomicAdd((unsigned long long *)&A.dbg_n[0], 1ull);
    const long long q = (long long)atomicAdd((unsigned long long *)&A.dbg_n[1], 1ull);
    if (q < A.dbg_cap) {
        A.dbg_ij[2 * q] = min(io, jo);
        A.dbg_ij[2 * q + 1] = max(io, jo);
    }
}

// Tile fill counters of the debug instantiation: tiles visited (dbg_n[3])
// and tile halves whose radial arithmetic runs (dbg_n[2]); with the pair
// count they give the fraction of evaluated lanes inside the cutoff.
__device__ __forceinline__ void count_tile(const ForceArgs &A, bool anyA, bool anyB)
{
    if ((threadIdx.x & 31) == 0) {
        atomicAdd((unsigned long long *)&A.dbg_n[3], 1ull);
        const unsigned long long h = (anyA ? 1ull : 0ull) + (anyB ? 1ull : 0ull);
        if (h) atomicAdd((unsigned long long *)&A.dbg_n[2], h);
    }
}

// Forward kernel (k_force) on i-group tiles.
//
// A work unit is one part of one segment of an i-group's list (the group:
// G consecutive clusters of a column, 8 G atoms).  A warp holds the group's
// atoms in its shared memory and walks the entries; an entry (J, image,
// cluster mask) stands for the tiles (group cluster c, J) of the clusters c
// in its mask.  Lane = ia + 8 jb computes, for every tile, the pairs of i
// atom ia of cluster c with j atoms jb and jb + 4 of J (an 8 x 8 tile, two
// pairs per lane, nothing compacted: pairs beyond the cutoff, excluded pairs
// and padding are evaluated and masked).  J's atoms are read once per entry
// and the force on them is summed over all tiles of the entry in registers,
// then over the 8 lanes of each j atom and added to the global 64-bit
// fixed-point sums (one atomic per atom and component), so the per-entry
// cost (staging, decode, j-force reduction and atomics) is shared by the
// entry's tiles.  The force on i accumulates per lane and cluster in shared
// memory and is summed and added when the unit is done.  J's z-sorted atoms
// form a lower half (jb) and an upper half (jb + 4), which are often not
// both within reach of cluster c: the membership of both pairs comes first
// and the radial arithmetic of a half runs only when one of its 32 pairs is
// in range (warp vote).  Flagged entries carry exclusion bitmasks per tile
// (excluded pairs dropped, 1-4 pairs scaled; the direct self tile's pairs
// j <= i excluded).  The FP32 sums run in a fixed order and meet only in
// integer sums, so results are run-to-run bit-identical.
constexpr int kTileWarps = 8;            // warps per block of the tile kernel
constexpr int kBatch = 16;               // entries staged per batch
#ifndef ACENB_TILE_MIN_BLOCKS
#define ACENB_TILE_MIN_BLOCKS 3          // resident blocks per SM the register budget is cut for
#endif
constexpr float kFarCoord = 3.0e18f;     // i-side padding: far from every atom and from the j-side padding

// Fixed-point value (2^32) of an FP32 sum; a value too large for the sums
// (or not finite) adds zero and sets ovf.
__device__ __forceinline__ long long tile_fixed(float f, bool &ovf)
{
    const bool ok = fabsf(f) < 67108864.0f;
    ovf = ovf || !ok;
    return __float2ll_rn((ok ? f : 0.0f) * 4294967296.0f);
}

// Claim of the next work unit (lane 0).  min_left > 0 (a helper launch):
// claim only while at least min_left units are unclaimed, else return
// n_units (the launch's own warps finish the rest sooner than a late
// helper unit would).
__device__ __forceinline__ int claim_unit(const ForceArgs &A, int n_units, int min_left)
{
    if (min_left > 0 && n_units - *(volatile const int *)A.work < min_left) return n_units;
    return atomicAdd(A.work, 1);
}

// Work unit u of the tile kernels: group, segment of its list, part of the
// segment, and the entry range [e_begin, e_end) of that part.
struct Unit {
    int g, e_begin, e_end;
    long long base;  // first entry of the segment in the group lists
};

__device__ __forceinline__ Unit unit_of(const ForceArgs &A, int u, int parts)
{
    Unit U;
    const int per_g = kListSegs * parts;
    U.g = u / per_g;
    const int r = u - U.g * per_g;
    const int seg = r / parts, part = r - seg * parts;
    const int n = __ldg(A.glist_n + (long long)U.g * kListSegs + seg);
    const int per = (n + parts - 1) / parts;
    U.e_begin = min(n, part * per);
    U.e_end = min(n, U.e_begin + per);
    U.base = (long long)U.g * A.cap + (long long)seg * (A.cap / kListSegs);
    return U;
}

// The exclusion and 1-4 bits of a lane's two pairs (i atom ia, j atoms jb
// and jb + 4) in a flagged tile.
__device__ __forceinline__ void tile_mask_bits(ulonglong2 m, int ia, int jb, bool &inA, bool &inB, bool &s14A,
                                               bool &s14B)
{
    const int bA = ia * kCluster + jb, bB = bA + 4;
    inA = inA && !((m.x >> bA) & 1ull);
    inB = inB && !((m.x >> bB) & 1ull);
    s14A = (m.y >> bA) & 1ull;
    s14B = (m.y >> bB) & 1ull;
}

// One tile (group cluster c, entry J) of a lane: i atom ia of cluster c at
// its image (IMG: x_i - L on axes with code 2), the pairs with the lane's
// j atoms pjA (jb) and pjB (jb + 4), already at their image (code 1 axes).
// SPECIAL: the entry carries exclusion bitmasks (gm).
template <int RAD, bool DEBUG, bool SPECIAL, bool IMG>
__device__ __forceinline__ void tile_pair2(const ForceArgs &A, const float4 *__restrict__ lj, float4 pi, int trow,
                                           int iorig, float4 pjA, float4 pjB, int tjA, int tjB, int jorigA,
                                           int jorigB, uint32_t code, float Lx, float Ly, float Lz, ulonglong2 gm,
                                           int ia, int jb, float4 &fi, float &elj, float &ec, float &fjAx,
                                           float &fjAy, float &fjAz, float &fjBx, float &fjBy, float &fjBz)
{
    if (IMG) {
        if ((code & 3u) == 2u) pi.x = __fsub_rn(pi.x, Lx);
        if (((code >> 2) & 3u) == 2u) pi.y = __fsub_rn(pi.y, Ly);
        if ((code >> 4) == 2u) pi.z = __fsub_rn(pi.z, Lz);
    }
    float dxA, dyA, dzA, dxB, dyB, dzB;
    const float r2A = disp_r2(pjA.x, pjA.y, pjA.z, pi.x, pi.y, pi.z, dxA, dyA, dzA);
    const float r2B = disp_r2(pjB.x, pjB.y, pjB.z, pi.x, pi.y, pi.z, dxB, dyB, dzB);
    bool inA = r2A < A.P.rc2, inB = r2B < A.P.rc2;
    bool s14A = false, s14B = false;
    if (SPECIAL) tile_mask_bits(gm, ia, jb, inA, inB, s14A, s14B);
    const bool anyA = __any_sync(kFull, inA), anyB = __any_sync(kFull, inB);
    if (DEBUG) count_tile(A, anyA, anyB);
    if (!anyA && !anyB) return;
    Acc acc = {fi.x, fi.y, fi.z, elj, ec};
    if (anyA) {
        if (DEBUG && inA) record_pair(A, iorig, jorigA);
        // only a special (flagged) tile can hold r2 = 0 (the self tile's diagonal, masked)
        eval_pair<RAD, SPECIAL>(A.P, lj, A.rtab, trow, pi.w, inA, dxA, dyA, dzA, SPECIAL ? (inA ? r2A : 1.0f) : r2A,
                                pjA.w, tjA, s14A, acc, fjAx, fjAy, fjAz);
    }
    if (anyB) {
        if (DEBUG && inB) record_pair(A, iorig, jorigB);
        eval_pair<RAD, SPECIAL>(A.P, lj, A.rtab, trow, pi.w, inB, dxB, dyB, dzB, SPECIAL ? (inB ? r2B : 1.0f) : r2B,
                                pjB.w, tjB, s14B, acc, fjBx, fjBy, fjBz);
    }
    fi = make_float4(acc.fx, acc.fy, acc.fz, 0.0f);
    elj = acc.elj;
    ec = acc.ec;
}

// One entry: J's atoms for the lane (jb, jb + 4) from the staged batch, the
// tiles of every group cluster in its mask, then the force on J's atoms.
template <int G, int RAD, bool VIRIAL, bool DEBUG, bool SPECIAL, bool IMG>
__device__ __forceinline__ void tile_entry(const ForceArgs &A, const float4 *__restrict__ lj,
                                           const float4 *__restrict__ s_ix, const int *__restrict__ s_it,
                                           const int *__restrict__ s_io, float4 *__restrict__ s_fi, uint2 ent,
                                           float4 pjA, float4 pjB, int tjA, int tjB, int ia, int jb, int lane, float Lx,
                                           float Ly, float Lz, float &elj, float &ec, float (&wimg)[6], bool &ovf)
{
    const int J = (int)(ent.x & kJMask);
    const uint32_t code = IMG ? (ent.x >> kShiftBit) & 0x3Fu : 0u;
    if (IMG) {  // j-side images (code 1): fl(x_j - L), as the other kernels stage them
        if ((code & 3u) == 1u) { pjA.x = __fsub_rn(pjA.x, Lx); pjB.x = __fsub_rn(pjB.x, Lx); }
        if (((code >> 2) & 3u) == 1u) { pjA.y = __fsub_rn(pjA.y, Ly); pjB.y = __fsub_rn(pjB.y, Ly); }
        if ((code >> 4) == 1u) { pjA.z = __fsub_rn(pjA.z, Lz); pjB.z = __fsub_rn(pjB.z, Lz); }
    }
    const int jorigA = DEBUG ? __ldg(A.perm + (long long)J * kCluster + jb) : -1;
    const int jorigB = DEBUG ? __ldg(A.perm + (long long)J * kCluster + jb + 4) : -1;
    const ulonglong2 *rec = SPECIAL ? A.gmask + (long long)(ent.y >> kMaskSlotBit) * G : nullptr;
    float fjAx = 0.0f, fjAy = 0.0f, fjAz = 0.0f, fjBx = 0.0f, fjBy = 0.0f, fjBz = 0.0f;
    for (unsigned cm = ent.y & 0xFFu; cm; cm &= cm - 1u) {
        const int c = __ffs(cm) - 1;
        const int ii = c * kCluster + ia;
        const ulonglong2 gm = SPECIAL ? rec[c] : make_ulonglong2(0ull, 0ull);
        float4 fi = s_fi[c * 32 + lane];
        tile_pair2<RAD, DEBUG, SPECIAL, IMG>(A, lj, s_ix[ii], s_it[ii], DEBUG ? s_io[ii] : -1, pjA, pjB, tjA, tjB,
                                             jorigA, jorigB, code, Lx, Ly, Lz, gm, ia, jb, fi, elj, ec, fjAx, fjAy,
                                             fjAz, fjBx, fjBy, fjBz);
        s_fi[c * 32 + lane] = fi;
    }
    // the force on J's atoms: sum over the 8 lanes of each (lanes ia), then
    // lanes ia = 0, 1, 2 add atom jb's x, y, z and ia = 3, 4, 5 atom jb + 4's
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        fjAx = __fadd_rn(fjAx, __shfl_xor_sync(kFull, fjAx, o));
        fjAy = __fadd_rn(fjAy, __shfl_xor_sync(kFull, fjAy, o));
        fjAz = __fadd_rn(fjAz, __shfl_xor_sync(kFull, fjAz, o));
        fjBx = __fadd_rn(fjBx, __shfl_xor_sync(kFull, fjBx, o));
        fjBy = __fadd_rn(fjBy, __shfl_xor_sync(kFull, fjBy, o));
        fjBz = __fadd_rn(fjBz, __shfl_xor_sync(kFull, fjBz, o));
    }
    const float fv = ia == 0 ? fjAx : ia == 1 ? fjAy : ia == 2 ? fjAz : ia == 3 ? fjBx : ia == 4 ? fjBy : fjBz;
    const long long fx = tile_fixed(fv, ovf);  // every lane (ia = 6, 7 hold z of B again): no branch
    if (ia < 6 && fx != 0) {
        const int j = ia < 3 ? jb : jb + 4;
        atomicAdd((unsigned long long *)&A.facc[24ll * J + 3 * j + (ia < 3 ? ia : ia - 3)], (unsigned long long)fx);
    }
    if (VIRIAL && IMG && ia == 0) {
        // periodic-image part of the virial: s (x) f_j with the entry's
        // shift s of j (code 1: -L, code 2: +L per axis)
        const uint32_t cx = code & 3u, cy = (code >> 2) & 3u, cz = code >> 4;
        const float sx = cx == 1u ? -Lx : (cx == 2u ? Lx : 0.0f);
        const float sy = cy == 1u ? -Ly : (cy == 2u ? Ly : 0.0f);
        const float sz = cz == 1u ? -Lz : (cz == 2u ? Lz : 0.0f);
        const float gx = __fadd_rn(fjAx, fjBx), gy = __fadd_rn(fjAy, fjBy), gz = __fadd_rn(fjAz, fjBz);
        wimg[0] = __fmaf_rn(sx, gx, wimg[0]);
        wimg[1] = __fmaf_rn(sy, gy, wimg[1]);
        wimg[2] = __fmaf_rn(sz, gz, wimg[2]);
        wimg[3] = __fmaf_rn(sx, gy, wimg[3]);
        wimg[4] = __fmaf_rn(sx, gz, wimg[4]);
        wimg[5] = __fmaf_rn(sy, gz, wimg[5]);
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

// Bytes of the forward kernels' LJ table: (A, B, 12 A, 6 B) and (A, B)
// remainders per type pair, rounded up to 16.
__host__ __device__ inline size_t lj_table_bytes(int T) { return align16((size_t)T * T * 24); }

// Shared memory of the forward kernel: the type-pair table (A, B, 12 A, 6 B)
// and per warp the unit's i atoms (coordinates + ke q, type row, caller
// index), the lanes' i-force partials per cluster, and one staged batch of
// entries' j atoms (coordinates + charge, type).
__host__ __device__ inline size_t tile_warp_bytes(int G)
{
    return (size_t)kCluster * G * (16 + 4 + 4) + (size_t)G * 32 * 16 + (size_t)kBatch * kCluster * (16 + 4);
}

template <int G, int RAD, bool VIRIAL, bool DEBUG>
__global__ void __launch_bounds__(kTileWarps * 32, ACENB_TILE_MIN_BLOCKS) k_force(ForceArgs A, int parts, int min_left)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_val[kTileWarps][kTaskVals];
    __shared__ int s_sys[kTileWarps];
    const int T = A.P.n_types;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, ia = lane & 7, jb = lane >> 3;
    float4 *lj = reinterpret_cast<float4 *>(smem);  // (A, B, 12 A, 6 B) per type pair
    unsigned char *wbase = smem + lj_table_bytes(T) + (size_t)w * tile_warp_bytes(G);
    float4 *s_ix = reinterpret_cast<float4 *>(wbase);                          // [8 G]
    float4 *s_fi = s_ix + kCluster * G;                                          // [G * 32]
    float4 *sjp = s_fi + G * 32;                                                 // [kBatch * 8]
    int *s_it = reinterpret_cast<int *>(sjp + kBatch * kCluster);                // [8 G]
    int *s_io = s_it + kCluster * G;                                             // [8 G]
    int *sjt = s_io + kCluster * G;                                              // [kBatch * 8]
    for (int k = threadIdx.x; k < T * T; k += blockDim.x) {
        const float4 ab = A.lj_tab[k];
        lj[k] = make_float4(ab.x, ab.y, 12.0f * ab.x, 6.0f * ab.y);
        reinterpret_cast<float2 *>(lj + T * T)[k] = make_float2(ab.z, ab.w);
    }
    pdl_entry();  // the type-pair tables do not depend on the preceding kernels
    __syncthreads();
    const int n_units = A.counts[4] * kListSegs * parts;
    int cur_sys = -1;
    float Lx = 0.0f, Ly = 0.0f, Lz = 0.0f;
    long long esum[2] = {0, 0};  // per lane: fixed-point energies of the current system
    float wimg[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};  // image virial of the current unit
    long long wv = 0;  // lane k < 6: fixed-point image virial component k of the current system
    bool ovf = false;  // a force sum out of the fixed-point range
    int u = 0;
    if (lane == 0) u = claim_unit(A, n_units, min_left);
    u = __shfl_sync(kFull, u, 0);
    while (u < n_units) {
        int u_next = 0;
        if (lane == 0) u_next = claim_unit(A, n_units, min_left);  // claimed now, used after this unit
        const Unit U = unit_of(A, u, parts);
        if (U.e_begin < U.e_end) {
            const int2 gr = __ldg(A.grp + U.g);
            const int c0 = gr.x, ncl = gr.y;
            const int sys_id = __ldg(A.clus_sys + c0);
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
            // the group's atoms (padding slots and absent clusters far away)
            for (int t = lane; t < kCluster * G; t += 32) {
                const long long slot = (long long)c0 * kCluster + t;
                float4 p = make_float4(kFarCoord, kFarCoord, kFarCoord, 0.0f);
                int tr = 0, orig = -1;
                if (t < kCluster * ncl) {
                    p = __ldg(A.xyzq + slot);
                    if (!is_real_coord(p.x)) p.x = p.y = p.z = kFarCoord;
                    p.w *= A.P.ke;
                    tr = __ldg(A.tslot + slot) * T;
                    orig = DEBUG ? __ldg(A.perm + slot) : -1;
                }
                s_ix[t] = p;
                s_it[t] = tr;
                s_io[t] = orig;
            }
#pragma unroll
            for (int c = 0; c < G; ++c) s_fi[c * 32 + lane] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            __syncwarp();
            float elj = 0.0f, ec = 0.0f;
            const uint2 *row = A.glist + U.base;
            bool unit_img = false;  // the unit holds an image entry (warp uniform)
            for (int e0 = U.e_begin; e0 < U.e_end; e0 += kBatch) {
                const int ne = min(kBatch, U.e_end - e0);
                const uint2 my = lane < ne ? __ldg(row + e0 + lane) : make_uint2(0u, 0u);
                // stage the batch's j atoms: lane k copies the 8 coordinates
                // and types of entry k (atom a at swz(k, a))
                if (lane < ne) {
                    const long long jbase = (long long)(my.x & kJMask) * kCluster;
#pragma unroll
                    for (int a = 0; a < kCluster; ++a) {
                        cp_async16(sjp + swz(lane, a), A.xyzq + jbase + a);
                        cp_async4(sjt + swz(lane, a), A.tslot + jbase + a);
                    }
                }
                cp_async_wait_all();
                __syncwarp();
                // the batch's plain entries first (no image code, no masks:
                // one code path without a dispatch), then the others
                const bool my_img = ((my.x >> kShiftBit) & 0x3Fu) != 0u;
                const bool my_spc = (my.x & kExclFlag) != 0u;
                const bool in_batch = lane < ne;
                unsigned plain = __ballot_sync(kFull, in_batch && !my_img && !my_spc);
                unsigned other = __ballot_sync(kFull, in_batch) & ~plain;
                unit_img = unit_img || __ballot_sync(kFull, in_batch && my_img) != 0u;
                while (plain) {
                    const int k = __ffs(plain) - 1;
                    plain &= plain - 1u;
                    const uint2 ent = make_uint2(__shfl_sync(kFull, my.x, k), __shfl_sync(kFull, my.y, k));
                    tile_entry<G, RAD, VIRIAL, DEBUG, false, false>(
                        A, lj, s_ix, s_it, s_io, s_fi, ent, sjp[swz(k, jb)], sjp[swz(k, jb + 4)], sjt[swz(k, jb)],
                        sjt[swz(k, jb + 4)], ia, jb, lane, Lx, Ly, Lz, elj, ec, wimg, ovf);
                }
                while (other) {
                    const int k = __ffs(other) - 1;
                    other &= other - 1u;
                    const uint2 ent = make_uint2(__shfl_sync(kFull, my.x, k), __shfl_sync(kFull, my.y, k));
                    const float4 pjA = sjp[swz(k, jb)], pjB = sjp[swz(k, jb + 4)];
                    const int tjA = sjt[swz(k, jb)], tjB = sjt[swz(k, jb + 4)];
                    const bool img = ((ent.x >> kShiftBit) & 0x3Fu) != 0u;
                    const bool special = (ent.x & kExclFlag) != 0u;
                    if (img) {
                        if (special)
                            tile_entry<G, RAD, VIRIAL, DEBUG, true, true>(A, lj, s_ix, s_it, s_io, s_fi, ent, pjA, pjB,
                                                                         tjA, tjB, ia, jb, lane, Lx, Ly, Lz, elj, ec,
                                                                         wimg, ovf);
                        else
                            tile_entry<G, RAD, VIRIAL, DEBUG, false, true>(A, lj, s_ix, s_it, s_io, s_fi, ent, pjA,
                                                                          pjB, tjA, tjB, ia, jb, lane, Lx, Ly, Lz, elj,
                                                                          ec, wimg, ovf);
                    } else {
                        tile_entry<G, RAD, VIRIAL, DEBUG, true, false>(A, lj, s_ix, s_it, s_io, s_fi, ent, pjA, pjB,
                                                                      tjA, tjB, ia, jb, lane, Lx, Ly, Lz, elj, ec, wimg,
                                                                      ovf);
                    }
                }
                __syncwarp();  // the staging buffer is rewritten by the next batch
            }
            // force on the group's atoms: each lane's partials summed over the
            // 4 lanes of the same atom (jb) in FP32 (a fixed butterfly: every
            // lane ends with the same bits), then lane jb adds clusters c with
            // c % 4 == jb in fixed point
#pragma unroll
            for (int c = 0; c < G; ++c) {
                float4 f = s_fi[c * 32 + lane];
#pragma unroll
                for (int o = 8; o < 32; o <<= 1) {
                    f.x = __fadd_rn(f.x, __shfl_xor_sync(kFull, f.x, o));
                    f.y = __fadd_rn(f.y, __shfl_xor_sync(kFull, f.y, o));
                    f.z = __fadd_rn(f.z, __shfl_xor_sync(kFull, f.z, o));
                }
                if ((c & 3) == jb && c < ncl) {
                    const long long slot = (long long)c0 * kCluster + c * kCluster + ia;
                    const long long fx = tile_fixed(f.x, ovf), fy = tile_fixed(f.y, ovf), fz = tile_fixed(f.z, ovf);
                    if (fx) atomicAdd((unsigned long long *)&A.facc[3 * slot], (unsigned long long)fx);
                    if (fy) atomicAdd((unsigned long long *)&A.facc[3 * slot + 1], (unsigned long long)fy);
                    if (fz) atomicAdd((unsigned long long *)&A.facc[3 * slot + 2], (unsigned long long)fz);
                }
            }
            esum[0] += tile_fixed(elj, ovf);
            esum[1] += tile_fixed(ec, ovf);
            if (VIRIAL && unit_img) tile_virial_unit(wimg, wv, lane);  // image entries only add to wimg
            if (__any_sync(kFull, ovf)) {
                if (lane == 0) atomicOr(A.status, ST_OVERFLOW);
                ovf = false;
            }
            __syncwarp();  // the i atoms and partials are rewritten by the next unit
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
// Forward kernel for i-groups of one cluster (k_force1): the lists are the
// same, each entry holds one tile (I, J).  Lane = jj + 8 ih holds j atom jj
// of J and the i atoms ih and ih + 4 of I in registers, so every lane
// computes two pairs of the 8 x 8 tile and the force on j is summed over only
// 4 lanes; the i atoms' z-sorted lower half (pair A) and upper half (pair B)
// are voted separately.  With one cluster per group the per-entry work is
// per tile, but the i side needs no shared memory and the j-force sum is
// short; which of this and the group kernel is faster depends on the system
// (the autotuner measures it).
constexpr int kBatch1 = 32;  // entries staged per batch (one per lane)

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

// Membership of one pair: the i atom at its image for the entry's shift code
// (IMG: x_i - L on axes with code 2; the j side was shifted by the caller),
// d = x_j - x_i and the FP32 predicate r2 < rc2.
template <bool IMG>
__device__ __forceinline__ bool tile1_member(const ForceArgs &A, const TileI &ti, uint32_t code, float4 pj, float Lx,
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

template <int RAD, bool VIRIAL, bool DEBUG, bool SPECIAL, bool IMG>
__device__ __forceinline__ void tile1_entry(const ForceArgs &A, const float4 *__restrict__ lj, uint2 ent, float4 pj,
                                            int tj, const TileI &ia, const TileI &ib, int jj, int ih, float Lx,
                                            float Ly, float Lz, Acc &acA, Acc &acB, float (&wimg)[6], bool &ovf)
{
    const int J = (int)(ent.x & kJMask);
    const uint32_t code = IMG ? (ent.x >> kShiftBit) & 0x3Fu : 0u;
    if (IMG) {  // j-side images (code 1): fl(x_j - L), as the other kernels stage them
        if ((code & 3u) == 1u) pj.x = __fsub_rn(pj.x, Lx);
        if (((code >> 2) & 3u) == 1u) pj.y = __fsub_rn(pj.y, Ly);
        if ((code >> 4) == 1u) pj.z = __fsub_rn(pj.z, Lz);
    }
    float dxA, dyA, dzA, r2A, dxB, dyB, dzB, r2B;
    bool inA = tile1_member<IMG>(A, ia, code, pj, Lx, Ly, Lz, dxA, dyA, dzA, r2A);
    bool inB = tile1_member<IMG>(A, ib, code, pj, Lx, Ly, Lz, dxB, dyB, dzB, r2B);
    bool s14A = false, s14B = false;
    if (SPECIAL) {  // exclusion bitmask of the tile: bit 8 i + j
        const ulonglong2 m = A.gmask[ent.y >> kMaskSlotBit];  // records of one cluster
        const int bA = ih * kCluster + jj, bB = bA + 4 * kCluster;
        inA = inA && !((m.x >> bA) & 1ull);
        inB = inB && !((m.x >> bB) & 1ull);
        s14A = (m.y >> bA) & 1ull;
        s14B = (m.y >> bB) & 1ull;
    }
    const bool anyA = __any_sync(kFull, inA), anyB = __any_sync(kFull, inB);
    if (DEBUG) count_tile(A, anyA, anyB);
    if (!anyA && !anyB) return;
    const int jorig = DEBUG ? __ldg(A.perm + (long long)J * kCluster + jj) : -1;
    float fjx = 0.0f, fjy = 0.0f, fjz = 0.0f;
    if (anyA) {
        if (DEBUG && inA) record_pair(A, ia.orig, jorig);
        // only a special (flagged) tile can hold r2 = 0 (the self tile's diagonal, masked)
        eval_pair<RAD, SPECIAL>(A.P, lj, A.rtab, ia.trow, ia.q, inA, dxA, dyA, dzA, SPECIAL ? (inA ? r2A : 1.0f) : r2A,
                                pj.w, tj, s14A, acA, fjx, fjy, fjz);
    }
    if (anyB) {
        if (DEBUG && inB) record_pair(A, ib.orig, jorig);
        eval_pair<RAD, SPECIAL>(A.P, lj, A.rtab, ib.trow, ib.q, inB, dxB, dyB, dzB, SPECIAL ? (inB ? r2B : 1.0f) : r2B,
                                pj.w, tj, s14B, acB, fjx, fjy, fjz);
    }
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

__host__ __device__ inline size_t tile1_warp_bytes() { return (size_t)kBatch1 * kCluster * (16 + 4); }

template <int RAD, bool VIRIAL, bool DEBUG>
__global__ void __launch_bounds__(kTileWarps * 32, ACENB_TILE_MIN_BLOCKS) k_force1(ForceArgs A, int parts, int min_left)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_val[kTileWarps][kTaskVals];
    __shared__ int s_sys[kTileWarps];
    const int T = A.P.n_types;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, jj = lane & 7, ih = lane >> 3;
    float4 *lj = reinterpret_cast<float4 *>(smem);  // (A, B, 12 A, 6 B) per type pair
    float4 *sjp = reinterpret_cast<float4 *>(smem + lj_table_bytes(T) + (size_t)w * tile1_warp_bytes());
    int *sjt = reinterpret_cast<int *>(sjp + kBatch1 * kCluster);
    for (int k = threadIdx.x; k < T * T; k += blockDim.x) {
        const float4 ab = A.lj_tab[k];
        lj[k] = make_float4(ab.x, ab.y, 12.0f * ab.x, 6.0f * ab.y);
        reinterpret_cast<float2 *>(lj + T * T)[k] = make_float2(ab.z, ab.w);
    }
    pdl_entry();  // the type-pair tables do not depend on the preceding kernels
    __syncthreads();
    const int n_units = A.counts[4] * kListSegs * parts;
    int cur_sys = -1;
    float Lx = 0.0f, Ly = 0.0f, Lz = 0.0f;
    long long esum[2] = {0, 0};
    float wimg[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    long long wv = 0;
    bool ovf = false;
    int u = 0;
    if (lane == 0) u = claim_unit(A, n_units, min_left);
    u = __shfl_sync(kFull, u, 0);
    while (u < n_units) {
        int u_next = 0;
        if (lane == 0) u_next = claim_unit(A, n_units, min_left);
        const Unit U = unit_of(A, u, parts);
        // what needs only the unit's group and segment is loaded before the
        // segment's length is known: one-cluster groups are numbered like
        // their clusters, and a segment holds at least its first batch
        const int I = U.g;
        const int sys_id = __ldg(A.clus_sys + I);
        const long long s0 = (long long)I * kCluster;
        const TileI ia = load_tile_i(A, s0 + ih, T, DEBUG);
        const TileI ib = load_tile_i(A, s0 + ih + 4, T, DEBUG);
        const uint2 *row = A.glist + U.base;
        const uint2 first = lane < A.cap / kListSegs ? __ldg(row + lane) : make_uint2(0u, 0u);
        if (U.e_begin < U.e_end) {
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
            Acc acA = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, acB = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            bool unit_img = false;
            for (int e0 = U.e_begin; e0 < U.e_end; e0 += kBatch1) {
                const int ne = min(kBatch1, U.e_end - e0);
                const uint2 my = lane < ne ? (e0 == 0 ? first : __ldg(row + e0 + lane)) : make_uint2(0u, 0u);
                if (lane < ne) {
                    const long long jbase = (long long)(my.x & kJMask) * kCluster;
#pragma unroll
                    for (int a = 0; a < kCluster; ++a) {
                        cp_async16(sjp + swz(lane, a), A.xyzq + jbase + a);
                        cp_async4(sjt + swz(lane, a), A.tslot + jbase + a);
                    }
                }
                cp_async_wait_all();
                __syncwarp();
                const bool my_img = ((my.x >> kShiftBit) & 0x3Fu) != 0u;
                const bool my_spc = (my.x & kExclFlag) != 0u;
                const bool in_batch = lane < ne;
                unsigned plain = __ballot_sync(kFull, in_batch && !my_img && !my_spc);
                unsigned other = __ballot_sync(kFull, in_batch) & ~plain;
                unit_img = unit_img || __ballot_sync(kFull, in_batch && my_img) != 0u;
                while (plain) {
                    const int k = __ffs(plain) - 1;
                    plain &= plain - 1u;
                    const uint2 ent = make_uint2(__shfl_sync(kFull, my.x, k), __shfl_sync(kFull, my.y, k));
                    tile1_entry<RAD, VIRIAL, DEBUG, false, false>(A, lj, ent, sjp[swz(k, jj)], sjt[swz(k, jj)], ia, ib,
                                                                  jj, ih, Lx, Ly, Lz, acA, acB, wimg, ovf);
                }
                while (other) {
                    const int k = __ffs(other) - 1;
                    other &= other - 1u;
                    const uint2 ent = make_uint2(__shfl_sync(kFull, my.x, k), __shfl_sync(kFull, my.y, k));
                    const float4 pj = sjp[swz(k, jj)];
                    const int tj = sjt[swz(k, jj)];
                    const bool img = ((ent.x >> kShiftBit) & 0x3Fu) != 0u;
                    const bool special = (ent.x & kExclFlag) != 0u;
                    if (img) {
                        if (special)
                            tile1_entry<RAD, VIRIAL, DEBUG, true, true>(A, lj, ent, pj, tj, ia, ib, jj, ih, Lx, Ly, Lz,
                                                                        acA, acB, wimg, ovf);
                        else
                            tile1_entry<RAD, VIRIAL, DEBUG, false, true>(A, lj, ent, pj, tj, ia, ib, jj, ih, Lx, Ly,
                                                                         Lz, acA, acB, wimg, ovf);
                    } else {
                        tile1_entry<RAD, VIRIAL, DEBUG, true, false>(A, lj, ent, pj, tj, ia, ib, jj, ih, Lx, Ly, Lz,
                                                                     acA, acB, wimg, ovf);
                    }
                }
                __syncwarp();  // the staging buffer is rewritten by the next batch
            }
            // force on the i atoms: the 8 lanes of each atom summed in FP32
            // (a fixed butterfly), then lanes jj < 3 add atom ih, jj = 3..5
            // atom ih + 4 in fixed point
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
            if (VIRIAL && unit_img) tile_virial_unit(wimg, wv, lane);
            if (__any_sync(kFull, ovf)) {
                if (lane == 0) atomicOr(A.status, ST_OVERFLOW);
                ovf = false;
            }
        }
        u = __shfl_sync(kFull, u_next, 0);
    }
    if (DEBUG) return;
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
// Adjoint kernel on i-group tiles (k_adjoint): the forward kernel's units,
// entries, tiles, half-tile votes and staging, with the pair adjoint of
// eval_pair_adj.  Per entry the j-side terms (dL/dx_j, dL/dq_j) of all its
// tiles are summed in registers, then over the 8 lanes of each j atom, and
// lane ia adds component ia % 4 of atom jb (ia < 4) or jb + 4 to the
// fixed-point sums; the i-side terms accumulate per lane and cluster in
// shared memory until the unit is done; the type-pair gradients go to a
// block table in shared memory (integer atomics) flushed at the end.  One
// inlined instance of the entry code serves every entry kind (the pair
// adjoint is long; an instance per kind overflowed the instruction cache).
constexpr int kAdjWarps = 4;             // warps per block of the adjoint tile kernel

__host__ __device__ inline size_t adj_warp_bytes(int G)
{
    return (size_t)kCluster * G * (16 + 16 + 4) + (size_t)G * 32 * 16 + (size_t)kBatch * kCluster * (16 + 16 + 4);
}

template <int G, int RAD>
__device__ __forceinline__ void adj_entry(const ForceArgs &A, const AdjTables &tab, const float4 *__restrict__ s_ix,
                                          const int *__restrict__ s_it, const float4 *__restrict__ s_ig,
                                          float4 *__restrict__ s_ai, uint2 ent, float4 pjA, float4 pjB, float4 gjA,
                                          float4 gjB, int tjA, int tjB, float gE_lj, float gE_c, int ia, int jb,
                                          int lane, float Lx, float Ly, float Lz, bool &ovf)
{
    const int J = (int)(ent.x & kJMask);
    const uint32_t code = (ent.x >> kShiftBit) & 0x3Fu;
    const bool img = code != 0u, special = (ent.x & kExclFlag) != 0u;
    if (img) {
        if ((code & 3u) == 1u) { pjA.x = __fsub_rn(pjA.x, Lx); pjB.x = __fsub_rn(pjB.x, Lx); }
        if (((code >> 2) & 3u) == 1u) { pjA.y = __fsub_rn(pjA.y, Ly); pjB.y = __fsub_rn(pjB.y, Ly); }
        if ((code >> 4) == 1u) { pjA.z = __fsub_rn(pjA.z, Lz); pjB.z = __fsub_rn(pjB.z, Lz); }
    }
    const ulonglong2 *rec = special ? A.gmask + (long long)(ent.y >> kMaskSlotBit) * G : nullptr;
    float jA[4] = {0.0f, 0.0f, 0.0f, 0.0f}, jB[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (unsigned cm = ent.y & 0xFFu; cm; cm &= cm - 1u) {
        const int c = __ffs(cm) - 1;
        const int ii = c * kCluster + ia;
        float4 pi = s_ix[ii];
        if (img) {
            if ((code & 3u) == 2u) pi.x = __fsub_rn(pi.x, Lx);
            if (((code >> 2) & 3u) == 2u) pi.y = __fsub_rn(pi.y, Ly);
            if ((code >> 4) == 2u) pi.z = __fsub_rn(pi.z, Lz);
        }
        float dxA, dyA, dzA, dxB, dyB, dzB;
        const float r2A = disp_r2(pjA.x, pjA.y, pjA.z, pi.x, pi.y, pi.z, dxA, dyA, dzA);
        const float r2B = disp_r2(pjB.x, pjB.y, pjB.z, pi.x, pi.y, pi.z, dxB, dyB, dzB);
        bool inA = r2A < A.P.rc2, inB = r2B < A.P.rc2;
        bool s14A = false, s14B = false;
        if (special) tile_mask_bits(rec[c], ia, jb, inA, inB, s14A, s14B);
        const bool anyA = __any_sync(kFull, inA), anyB = __any_sync(kFull, inB);
        if (!anyA && !anyB) continue;
        const int trow = s_it[ii];
        const float4 gi = s_ig[ii];
        float4 ai = s_ai[c * 32 + lane];
        AccAdj acc = {ai.x, ai.y, ai.z, ai.w};
        if (anyA) {
            float a, b, cc, d, ds, de;
            eval_pair_adj<RAD == 1>(A.P, tab, trow, pi.w, gi.x, gi.y, gi.z, gE_lj, gE_c, inA, dxA, dyA, dzA,
                                    inA ? r2A : 1.0f, pjA.w, tjA, gjA, s14A, A.status, acc, a, b, cc, d, ds, de);
            add_type_grads(tab, inA ? trow + tjA : -1, ds, de, A.status);
            jA[0] = __fadd_rn(jA[0], a);
            jA[1] = __fadd_rn(jA[1], b);
            jA[2] = __fadd_rn(jA[2], cc);
            jA[3] = __fadd_rn(jA[3], d);
        }
        if (anyB) {
            float a, b, cc, d, ds, de;
            eval_pair_adj<RAD == 1>(A.P, tab, trow, pi.w, gi.x, gi.y, gi.z, gE_lj, gE_c, inB, dxB, dyB, dzB,
                                    inB ? r2B : 1.0f, pjB.w, tjB, gjB, s14B, A.status, acc, a, b, cc, d, ds, de);
            add_type_grads(tab, inB ? trow + tjB : -1, ds, de, A.status);
            jB[0] = __fadd_rn(jB[0], a);
            jB[1] = __fadd_rn(jB[1], b);
            jB[2] = __fadd_rn(jB[2], cc);
            jB[3] = __fadd_rn(jB[3], d);
        }
        s_ai[c * 32 + lane] = make_float4(acc.dx, acc.dy, acc.dz, acc.dq);
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            jA[k] = __fadd_rn(jA[k], __shfl_xor_sync(kFull, jA[k], o));
            jB[k] = __fadd_rn(jB[k], __shfl_xor_sync(kFull, jB[k], o));
        }
    float gv = jA[0];
#pragma unroll
    for (int k = 1; k < 4; ++k) gv = ia == k ? jA[k] : gv;
#pragma unroll
    for (int k = 0; k < 4; ++k) gv = ia == 4 + k ? jB[k] : gv;
    const long long gx = tile_fixed(gv, ovf);
    if (gx != 0) {
        const int j = ia < 4 ? jb : jb + 4;
        atomicAdd((unsigned long long *)&A.gacc[32ll * J + 4 * j + (ia & 3)], (unsigned long long)gx);
    }
}

template <int G, int RAD>
__global__ void __launch_bounds__(kAdjWarps * 32) k_adjoint(ForceArgs A, int parts)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int T = A.P.n_types;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, ia = lane & 7, jb = lane >> 3;
    size_t off = 0;
    unsigned long long *tacc = reinterpret_cast<unsigned long long *>(smem + off);
    off += (size_t)T * T * 16;
    float4 *ljd = reinterpret_cast<float4 *>(smem + off);
    off += (size_t)T * T * 16;
    float2 *lj = reinterpret_cast<float2 *>(smem + off);
    off += align16((size_t)T * T * 8);
    unsigned char *wbase = smem + off + (size_t)w * adj_warp_bytes(G);
    float4 *s_ix = reinterpret_cast<float4 *>(wbase);    // [8 G] x, y, z, ke q
    float4 *s_ig = s_ix + kCluster * G;                    // [8 G] dL/dF of the i atoms
    float4 *s_ai = s_ig + kCluster * G;                    // [G * 32] i-side partials
    float4 *sjp = s_ai + G * 32;                           // [kBatch * 8]
    float4 *sjg = sjp + kBatch * kCluster;                 // [kBatch * 8]
    int *s_it = reinterpret_cast<int *>(sjg + kBatch * kCluster);  // [8 G]
    int *sjt = s_it + kCluster * G;                        // [kBatch * 8]
    for (int k = threadIdx.x; k < T * T; k += blockDim.x) {
        lj[k] = make_float2(A.lj_tab[k].x, A.lj_tab[k].y);
        ljd[k] = A.lj_d[k];
        tacc[2 * k] = 0ull;
        tacc[2 * k + 1] = 0ull;
    }
    pdl_entry();  // the type-pair tables do not depend on the preceding kernels
    __syncthreads();
    const AdjTables tab{lj, ljd, tacc};
    const int n_units = A.counts[4] * kListSegs * parts;
    int cur_sys = -1;
    float Lx = 0.0f, Ly = 0.0f, Lz = 0.0f, gE_lj = 0.0f, gE_c = 0.0f;
    bool ovf = false;
    int u = 0;
    if (lane == 0) u = atomicAdd(A.work, 1);
    u = __shfl_sync(kFull, u, 0);
    while (u < n_units) {
        int u_next = 0;
        if (lane == 0) u_next = atomicAdd(A.work, 1);
        const Unit U = unit_of(A, u, parts);
        if (U.e_begin < U.e_end) {
            const int2 gr = __ldg(A.grp + U.g);
            const int c0 = gr.x, ncl = gr.y;
            const int sys_id = __ldg(A.clus_sys + c0);
            if (sys_id != cur_sys) {
                cur_sys = sys_id;
                Lx = A.sys[sys_id].L[0];
                Ly = A.sys[sys_id].L[1];
                Lz = A.sys[sys_id].L[2];
                gE_lj = A.dLdE ? (float)A.dLdE[2 * sys_id] : 0.0f;
                gE_c = A.dLdE ? (float)A.dLdE[2 * sys_id + 1] : 0.0f;
            }
            for (int t = lane; t < kCluster * G; t += 32) {
                const long long slot = (long long)c0 * kCluster + t;
                float4 p = make_float4(kFarCoord, kFarCoord, kFarCoord, 0.0f);
                float4 gi = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                int tr = 0;
                if (t < kCluster * ncl) {
                    p = __ldg(A.xyzq + slot);
                    if (!is_real_coord(p.x)) p.x = p.y = p.z = kFarCoord;
                    p.w *= A.P.ke;
                    gi = __ldg(A.gslot + slot);
                    tr = __ldg(A.tslot + slot) * T;
                }
                s_ix[t] = p;
                s_ig[t] = gi;
                s_it[t] = tr;
            }
#pragma unroll
            for (int c = 0; c < G; ++c) s_ai[c * 32 + lane] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            __syncwarp();
            const uint2 *row = A.glist + U.base;
            for (int e0 = U.e_begin; e0 < U.e_end; e0 += kBatch) {
                const int ne = min(kBatch, U.e_end - e0);
                const uint2 my = lane < ne ? __ldg(row + e0 + lane) : make_uint2(0u, 0u);
                if (lane < ne) {
                    const long long jbase = (long long)(my.x & kJMask) * kCluster;
#pragma unroll
                    for (int a = 0; a < kCluster; ++a) {
                        cp_async16(sjp + swz(lane, a), A.xyzq + jbase + a);
                        cp_async16(sjg + swz(lane, a), A.gslot + jbase + a);
                        cp_async4(sjt + swz(lane, a), A.tslot + jbase + a);
                    }
                }
                cp_async_wait_all();
                __syncwarp();
                for (int k = 0; k < ne; ++k) {
                    const uint2 ent = make_uint2(__shfl_sync(kFull, my.x, k), __shfl_sync(kFull, my.y, k));
                    adj_entry<G, RAD>(A, tab, s_ix, s_it, s_ig, s_ai, ent, sjp[swz(k, jb)], sjp[swz(k, jb + 4)],
                                      sjg[swz(k, jb)], sjg[swz(k, jb + 4)], sjt[swz(k, jb)], sjt[swz(k, jb + 4)],
                                      gE_lj, gE_c, ia, jb, lane, Lx, Ly, Lz, ovf);
                }
                __syncwarp();  // the staging buffers are rewritten by the next batch
            }
            // i-side terms: the 4 lanes of each atom summed in FP32 (fixed
            // butterfly), then lane jb adds clusters c with c % 4 == jb
#pragma unroll
            for (int c = 0; c < G; ++c) {
                float4 a = s_ai[c * 32 + lane];
#pragma unroll
                for (int o = 8; o < 32; o <<= 1) {
                    a.x = __fadd_rn(a.x, __shfl_xor_sync(kFull, a.x, o));
                    a.y = __fadd_rn(a.y, __shfl_xor_sync(kFull, a.y, o));
                    a.z = __fadd_rn(a.z, __shfl_xor_sync(kFull, a.z, o));
                    a.w = __fadd_rn(a.w, __shfl_xor_sync(kFull, a.w, o));
                }
                if ((c & 3) == jb && c < ncl) {
                    const long long slot = (long long)c0 * kCluster + c * kCluster + ia;
                    const long long v0 = tile_fixed(a.x, ovf), v1 = tile_fixed(a.y, ovf), v2 = tile_fixed(a.z, ovf),
                                    v3 = tile_fixed(a.w, ovf);
                    if (v0) atomicAdd((unsigned long long *)&A.gacc[4 * slot], (unsigned long long)v0);
                    if (v1) atomicAdd((unsigned long long *)&A.gacc[4 * slot + 1], (unsigned long long)v1);
                    if (v2) atomicAdd((unsigned long long *)&A.gacc[4 * slot + 2], (unsigned long long)v2);
                    if (v3) atomicAdd((unsigned long long *)&A.gacc[4 * slot + 3], (unsigned long long)v3);
                }
            }
            if (__any_sync(kFull, ovf)) {
                if (lane == 0) atomicOr(A.status, ST_OVERFLOW);
                ovf = false;
            }
            __syncwarp();
        }
        u = __shfl_sync(kFull, u_next, 0);
    }
    // block table of parameter gradients -> global (integer sums)
    __syncthreads();
    for (int k = threadIdx.x; k < 2 * T * T; k += blockDim.x)
        if (tacc[k]) atomicAdd((unsigned long long *)&A.tab_acc[k], tacc[k]);
}

// Adjoint kernel for i-groups of one cluster (k_adjoint1): the structure of
// k_force1.  Lane = jj + 8 ih holds j atom jj of the entry's cluster J and i
// atoms ih and ih + 4 of the unit's cluster, whose positions, dL/dF and
// type rows stay in registers for the whole unit; the i-side terms (dL/dx_i,
// dL/dq_i) accumulate per lane in registers.  Per entry the j-side terms of
// the lane's two pairs share its j atom: they are summed over the 4 lanes of
// that atom (two shuffle levels) and lane ih adds component ih (x, y, z, q)
// to the fixed-point sums.  The type-pair gradients go to the block table
// as in k_adjoint.
struct TileIA {
    float x, y, z, qk;  // position, ke q
    float4 g;           // dL/dF of the atom
    int trow;           // type row (t T)
};

__device__ __forceinline__ TileIA load_tile_ia(const ForceArgs &A, long long slot, int T)
{
    TileIA t;
    const float4 p = __ldg(A.xyzq + slot);
    const bool real = is_real_coord(p.x);
    t.x = real ? p.x : kFarCoord;
    t.y = real ? p.y : kFarCoord;
    t.z = real ? p.z : kFarCoord;
    t.qk = p.w * A.P.ke;
    t.g = __ldg(A.gslot + slot);
    t.trow = __ldg(A.tslot + slot) * T;
    return t;
}

template <int RAD>
__device__ __forceinline__ void adj1_entry(const ForceArgs &A, const AdjTables &tab, uint2 ent, float4 pj, float4 gj,
                                           int tj, const TileIA &ia, const TileIA &ib, int jj, int ih, float Lx,
                                           float Ly, float Lz, float gE_lj, float gE_c, AccAdj &acA, AccAdj &acB,
                                           bool &ovf)
{
    const int J = (int)(ent.x & kJMask);
    const uint32_t code = (ent.x >> kShiftBit) & 0x3Fu;
    const bool img = code != 0u, special = (ent.x & kExclFlag) != 0u;
    float ax = ia.x, ay = ia.y, az = ia.z, bx = ib.x, by = ib.y, bz = ib.z;
    if (img) {  // j side: x_j - L on code-1 axes; i side: x_i - L on code-2 axes
        if ((code & 3u) == 1u) pj.x = __fsub_rn(pj.x, Lx);
        if (((code >> 2) & 3u) == 1u) pj.y = __fsub_rn(pj.y, Ly);
        if ((code >> 4) == 1u) pj.z = __fsub_rn(pj.z, Lz);
        if ((code & 3u) == 2u) { ax = __fsub_rn(ax, Lx); bx = __fsub_rn(bx, Lx); }
        if (((code >> 2) & 3u) == 2u) { ay = __fsub_rn(ay, Ly); by = __fsub_rn(by, Ly); }
        if ((code >> 4) == 2u) { az = __fsub_rn(az, Lz); bz = __fsub_rn(bz, Lz); }
    }
    float dxA, dyA, dzA, dxB, dyB, dzB;
    const float r2A = disp_r2(pj.x, pj.y, pj.z, ax, ay, az, dxA, dyA, dzA);
    const float r2B = disp_r2(pj.x, pj.y, pj.z, bx, by, bz, dxB, dyB, dzB);
    bool inA = r2A < A.P.rc2, inB = r2B < A.P.rc2;
    bool s14A = false, s14B = false;
    if (special) {  // exclusion bitmask of the tile: bit 8 i + j
        const ulonglong2 m = A.gmask[ent.y >> kMaskSlotBit];
        const int bA = ih * kCluster + jj, bB = bA + 4 * kCluster;
        inA = inA && !((m.x >> bA) & 1ull);
        inB = inB && !((m.x >> bB) & 1ull);
        s14A = (m.y >> bA) & 1ull;
        s14B = (m.y >> bB) & 1ull;
    }
    const bool anyA = __any_sync(kFull, inA), anyB = __any_sync(kFull, inB);
    if (!anyA && !anyB) return;
    float jt[4] = {0.0f, 0.0f, 0.0f, 0.0f};  // the j atom's terms (x, y, z, q)
    if (anyA) {
        float a, b, c, d, ds, de;
        eval_pair_adj<RAD == 1>(A.P, tab, ia.trow, ia.qk, ia.g.x, ia.g.y, ia.g.z, gE_lj, gE_c, inA, dxA, dyA, dzA,
                                inA ? r2A : 1.0f, pj.w, tj, gj, s14A, A.status, acA, a, b, c, d, ds, de);
        add_type_grads(tab, inA ? ia.trow + tj : -1, ds, de, A.status);
        jt[0] = a;
        jt[1] = b;
        jt[2] = c;
        jt[3] = d;
    }
    if (anyB) {
        float a, b, c, d, ds, de;
        eval_pair_adj<RAD == 1>(A.P, tab, ib.trow, ib.qk, ib.g.x, ib.g.y, ib.g.z, gE_lj, gE_c, inB, dxB, dyB, dzB,
                                inB ? r2B : 1.0f, pj.w, tj, gj, s14B, A.status, acB, a, b, c, d, ds, de);
        add_type_grads(tab, inB ? ib.trow + tj : -1, ds, de, A.status);
        jt[0] = __fadd_rn(jt[0], a);
        jt[1] = __fadd_rn(jt[1], b);
        jt[2] = __fadd_rn(jt[2], c);
        jt[3] = __fadd_rn(jt[3], d);
    }
#pragma unroll
    for (int o = 8; o < 32; o <<= 1)
#pragma unroll
        for (int k = 0; k < 4; ++k) jt[k] = __fadd_rn(jt[k], __shfl_xor_sync(kFull, jt[k], o));
    const float gv = ih == 0 ? jt[0] : (ih == 1 ? jt[1] : (ih == 2 ? jt[2] : jt[3]));
    const long long gx = tile_fixed(gv, ovf);
    if (gx != 0) atomicAdd((unsigned long long *)&A.gacc[32ll * J + 4 * jj + ih], (unsigned long long)gx);
}

constexpr int kBatchA = 16;  // entries staged per batch of the single-cluster adjoint (shared memory per block)

__host__ __device__ inline size_t adj1_warp_bytes() { return (size_t)kBatchA * kCluster * (16 + 16 + 4); }

size_t adjoint1_smem_bytes(int T)
{
    return (size_t)T * T * 32 + align16((size_t)T * T * 8) + (size_t)kAdjWarps * adj1_warp_bytes();
}

template <int RAD>
__global__ void __launch_bounds__(kAdjWarps * 32) k_adjoint1(ForceArgs A, int parts)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int T = A.P.n_types;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, jj = lane & 7, ih = lane >> 3;
    size_t off = 0;
    unsigned long long *tacc = reinterpret_cast<unsigned long long *>(smem + off);
    off += (size_t)T * T * 16;
    float4 *ljd = reinterpret_cast<float4 *>(smem + off);
    off += (size_t)T * T * 16;
    float2 *lj = reinterpret_cast<float2 *>(smem + off);
    off += align16((size_t)T * T * 8);
    float4 *sjp = reinterpret_cast<float4 *>(smem + off + (size_t)w * adj1_warp_bytes());  // [kBatchA * 8]
    float4 *sjg = sjp + kBatchA * kCluster;                                                // [kBatchA * 8]
    int *sjt = reinterpret_cast<int *>(sjg + kBatchA * kCluster);                          // [kBatchA * 8]
    for (int k = threadIdx.x; k < T * T; k += blockDim.x) {
        lj[k] = make_float2(A.lj_tab[k].x, A.lj_tab[k].y);
        ljd[k] = A.lj_d[k];
        tacc[2 * k] = 0ull;
        tacc[2 * k + 1] = 0ull;
    }
    pdl_entry();  // the type-pair tables do not depend on the preceding kernels
    __syncthreads();
    const AdjTables tab{lj, ljd, tacc};
    const int n_units = A.counts[4] * kListSegs * parts;
    int cur_sys = -1;
    float Lx = 0.0f, Ly = 0.0f, Lz = 0.0f, gE_lj = 0.0f, gE_c = 0.0f;
    bool ovf = false;
    int u = 0;
    if (lane == 0) u = atomicAdd(A.work, 1);
    u = __shfl_sync(kFull, u, 0);
    while (u < n_units) {
        int u_next = 0;
        if (lane == 0) u_next = atomicAdd(A.work, 1);
        const Unit U = unit_of(A, u, parts);
        // as in k_force1: what needs only the unit's group and segment is
        // loaded before the segment's length is known
        const int I = U.g;  // one-cluster groups are numbered like their clusters
        const int sys_id = __ldg(A.clus_sys + I);
        const long long s0 = (long long)I * kCluster;
        const TileIA ia = load_tile_ia(A, s0 + ih, T);
        const TileIA ib = load_tile_ia(A, s0 + ih + 4, T);
        const uint2 *row = A.glist + U.base;
        const uint2 first = lane < A.cap / kListSegs ? __ldg(row + lane) : make_uint2(0u, 0u);
        if (U.e_begin < U.e_end) {
            if (sys_id != cur_sys) {
                cur_sys = sys_id;
                Lx = A.sys[sys_id].L[0];
                Ly = A.sys[sys_id].L[1];
                Lz = A.sys[sys_id].L[2];
                gE_lj = A.dLdE ? (float)A.dLdE[2 * sys_id] : 0.0f;
                gE_c = A.dLdE ? (float)A.dLdE[2 * sys_id + 1] : 0.0f;
            }
            AccAdj acA = {0.0f, 0.0f, 0.0f, 0.0f}, acB = {0.0f, 0.0f, 0.0f, 0.0f};
            for (int e0 = U.e_begin; e0 < U.e_end; e0 += kBatchA) {
                const int ne = min(kBatchA, U.e_end - e0);
                const uint2 my = lane < ne ? (e0 == 0 ? first : __ldg(row + e0 + lane)) : make_uint2(0u, 0u);
                if (lane < ne) {
                    const long long jbase = (long long)(my.x & kJMask) * kCluster;
#pragma unroll
                    for (int a = 0; a < kCluster; ++a) {
                        cp_async16(sjp + swz(lane, a), A.xyzq + jbase + a);
                        cp_async16(sjg + swz(lane, a), A.gslot + jbase + a);
                        cp_async4(sjt + swz(lane, a), A.tslot + jbase + a);
                    }
                }
                cp_async_wait_all();
                __syncwarp();
                for (int k = 0; k < ne; ++k) {
                    const uint2 ent = make_uint2(__shfl_sync(kFull, my.x, k), __shfl_sync(kFull, my.y, k));
                    adj1_entry<RAD>(A, tab, ent, sjp[swz(k, jj)], sjg[swz(k, jj)], sjt[swz(k, jj)], ia, ib, jj, ih,
                                    Lx, Ly, Lz, gE_lj, gE_c, acA, acB, ovf);
                }
                __syncwarp();  // the staging buffers are rewritten by the next batch
            }
            // i-side terms: the 8 lanes of each atom summed in FP32 (a fixed
            // butterfly), then lanes jj < 4 add component jj of atom ih and
            // lanes jj >= 4 component jj - 4 of atom ih + 4
            float v[8] = {acA.dx, acA.dy, acA.dz, acA.dq, acB.dx, acB.dy, acB.dz, acB.dq};
#pragma unroll
            for (int o = 1; o < 8; o <<= 1)
#pragma unroll
                for (int c = 0; c < 8; ++c) v[c] = __fadd_rn(v[c], __shfl_xor_sync(kFull, v[c], o));
            float mine = v[0];
#pragma unroll
            for (int c = 1; c < 8; ++c) mine = jj == c ? v[c] : mine;
            const long long gi = tile_fixed(mine, ovf);
            if (gi != 0) {
                const long long slot = s0 + ih + (jj < 4 ? 0 : 4);
                atomicAdd((unsigned long long *)&A.gacc[4 * slot + (jj & 3)], (unsigned long long)gi);
            }
            if (__any_sync(kFull, ovf)) {
                if (lane == 0) atomicOr(A.status, ST_OVERFLOW);
                ovf = false;
            }
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

// Fixed-point forces (sorted order) to FP32 in the caller's order, one
// thread per atom in caller order (gathers from the sorted sums, and
// coalesced writes of F, which may be page-locked host memory).  With
// VIRIAL, also the atom part of the virial: for central pair forces
// W_ab = sum_pairs d_a f_b (d = x_j' - x_i, f the force on j) equals
// sum_atoms x_a F_b over the wrapped coordinates x and total forces F, plus
// the periodic-image terms added by the force kernel.  Each atom's terms are
// rounded to the 2^20 fixed-point grid in FP64 and summed as integers per
// thread (grid-stride loop, atoms in system order) and per warp.
template <bool VIRIAL>
__global__ void __launch_bounds__(256) k_unpack_forces(int n_atoms, int *__restrict__ counts,
                                                       const int *__restrict__ inv, const long long *__restrict__ facc,
                                                       float *__restrict__ F, const float4 *__restrict__ xyzq,
                                                       const int *__restrict__ atom_sys, long long *__restrict__ sys_acc,
                                                       int n_sys, double *__restrict__ energy, double *__restrict__ virial,
                                                       const long long *__restrict__ pme_f,
                                                       const long long *__restrict__ pme_s, double pme_self)
{
    pdl_entry();
    long long w[6] = {0, 0, 0, 0, 0, 0};
    int wsys = -1;
    __shared__ unsigned long long blk_w[6];
    __shared__ int blk_sys;
    if (VIRIAL) {
        if (threadIdx.x < 6) blk_w[threadIdx.x] = 0ull;
        if (threadIdx.x == 0) {
            const int a0 = blockIdx.x * blockDim.x;
            blk_sys = a0 < n_atoms ? atom_sys[a0] : -1;
        }
        __syncthreads();
    }
    for (int a0 = blockIdx.x * blockDim.x; a0 < n_atoms; a0 += gridDim.x * blockDim.x) {
        const int a = a0 + threadIdx.x;
        const int s = a < n_atoms ? inv[a] : -1;
        int sys = -1;
        long long c[6];
        if (s >= 0) {
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
                sys = atom_sys[a];
            }
        }
        if (VIRIAL) {
            // atoms come in system order: flush a lane's sums before it moves on
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

size_t tile_smem_bytes(int T, int G) { return lj_table_bytes(T) + (size_t)kTileWarps * tile_warp_bytes(G); }

// beside_pme: the PME chain, forked before the list kernel, runs on its side
// stream during this kernel; the persistent grid then leaves one block slot
// per SM free, so that the PME kernels run alongside instead of after it,
// and a second launch of the same kernel, one block per SM on the side
// stream behind the PME chain (and the lists), takes units from the same
// counter once the chain is done (helper).  Which block takes which unit
// does not change any result.
template <int G, int RAD, bool VIRIAL, bool DEBUG>
static void launch_force_g(nb_ctx *ctx, const ForceArgs &A, bool beside_pme, bool helper)
{
    const size_t smem = tile_smem_bytes(A.P.n_types, G);
    static std::atomic<unsigned long long> optin{0};
    smem_optin_once(k_force<G, RAD, VIRIAL, DEBUG>, ctx->device, 200 * 1024, optin);
    // persistent grid: never more blocks than can be resident at once
    int resident = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_force<G, RAD, VIRIAL, DEBUG>, kTileWarps * 32, smem);
    const int per_sm = helper ? 1 : std::max(1, std::min(ctx->tune.blocks_per_sm, resident) - (beside_pme ? 1 : 0));
    const int parts = ctx->tune.list_split > 0 ? ctx->tune.list_split : kDefaultListSplit;
    // a helper claims units while more are left than the main launch's warps hold
    const int min_left = helper ? ctx->num_sms * std::max(1, std::min(ctx->tune.blocks_per_sm, resident) - 1) * kTileWarps : 0;
    launch_pdl(k_force<G, RAD, VIRIAL, DEBUG>, dim3(ctx->num_sms * per_sm), dim3(kTileWarps * 32), smem,
               helper ? pme_side_stream(ctx) : ctx->stream, A, parts, min_left);
}

template <int RAD, bool VIRIAL, bool DEBUG>
static void launch_force_1(nb_ctx *ctx, const ForceArgs &A, bool beside_pme, bool helper)
{
    const size_t smem = lj_table_bytes(A.P.n_types) + (size_t)kTileWarps * tile1_warp_bytes();
    static std::atomic<unsigned long long> optin{0};
    smem_optin_once(k_force1<RAD, VIRIAL, DEBUG>, ctx->device, 200 * 1024, optin);
    int resident = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_force1<RAD, VIRIAL, DEBUG>, kTileWarps * 32, smem);
    const int per_sm = helper ? 1 : std::max(1, std::min(ctx->tune.blocks_per_sm, resident) - (beside_pme ? 1 : 0));
    const int parts = ctx->tune.list_split > 0 ? ctx->tune.list_split : kDefaultListSplit;
    const int min_left = helper ? ctx->num_sms * std::max(1, std::min(ctx->tune.blocks_per_sm, resident) - 1) * kTileWarps : 0;
    launch_pdl(k_force1<RAD, VIRIAL, DEBUG>, dim3(ctx->num_sms * per_sm), dim3(kTileWarps * 32), smem,
               helper ? pme_side_stream(ctx) : ctx->stream, A, parts, min_left);
}

template <int RAD, bool VIRIAL, bool DEBUG>
static void launch_force_t(nb_ctx *ctx, const ForceArgs &A, bool beside_pme, bool helper)
{
    helper = helper && beside_pme;
    // the lists are the last work on the context's stream here: the side
    // stream waits for them before the helper
    if (helper && pme_side_after_lists(ctx) != cudaSuccess) return;
    for (int h = 0; h < (helper ? 2 : 1); ++h) {  // h = 1: the helper behind the PME chain
        if (ctx->built_group == 1) launch_force_1<RAD, VIRIAL, DEBUG>(ctx, A, beside_pme, h == 1);
        else if (ctx->built_group == 4) launch_force_g<4, RAD, VIRIAL, DEBUG>(ctx, A, beside_pme, h == 1);
        else launch_force_g<8, RAD, VIRIAL, DEBUG>(ctx, A, beside_pme, h == 1);
        if (h == 1) pme_side_rejoin(ctx);
    }
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
    A.grp = d.grp;
    A.glist = d.glist;
    A.glist_n = d.glist_n;
    A.gmask = d.gmask;
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
                                 bool pme, bool beside_pme, bool helper)
{
    auto &d = ctx->d;
    ForceArgs A = make_args(ctx);
    A.facc = d.facc;
    const bool ewald = ctx->pp.ewald != 0;
    const bool virial = d_virial != nullptr;
    const bool prof = ctx->profiling && ctx->prof_n < (int)ctx->prof_ev.size() / 2;
    if (prof) cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n], ctx->stream);
    if (debug_pairs) {  // the pair set does not depend on the radial functions
        if (ewald) launch_force_t<1, false, true>(ctx, A, beside_pme, helper);
        else launch_force_t<0, false, true>(ctx, A, beside_pme, helper);
    } else if (ctx->tab_n > 0) {
        if (virial) launch_force_t<2, true, false>(ctx, A, beside_pme, helper);
        else launch_force_t<2, false, false>(ctx, A, beside_pme, helper);
    } else if (ewald) {
        if (virial) launch_force_t<1, true, false>(ctx, A, beside_pme, helper);
        else launch_force_t<1, false, false>(ctx, A, beside_pme, helper);
    } else {
        if (virial) launch_force_t<0, true, false>(ctx, A, beside_pme, helper);
        else launch_force_t<0, false, false>(ctx, A, beside_pme, helper);
    }
    if (prof) {
        cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n + 1], ctx->stream);
        ctx->prof_n++;
    }
    if (pme) {
        cudaError_t e = launch_pme_join(ctx);
        if (e != cudaSuccess) return e;
    }
    if (d_F) {  // else the caller's next kernel reads the fixed-point sums (the MD step)
        const int tb = 256;
        const int S = (int)ctx->n_atoms;
        const int blocks = std::max(1, std::min((S + tb - 1) / tb, 4 * ctx->num_sms));
        double *en = debug_pairs ? nullptr : d_energy;
        double *vi = debug_pairs ? nullptr : d_virial;
        const long long *pf = pme ? pme_forces_acc(ctx) : nullptr, *ps = pme ? pme_sums_acc(ctx) : nullptr;
        const double pself = pme ? pme_self_coef(ctx) : 0.0;
        if (virial)
            launch_pdl(k_unpack_forces<true>, dim3(blocks), dim3(tb), 0, ctx->stream, S, d.counts, d.inv, d.facc, d_F,
                       d.xyzq, d.atom_sys, d.sys_acc, ctx->n_sys, en, vi, pf, ps, pself);
        else
            launch_pdl(k_unpack_forces<false>, dim3(blocks), dim3(tb), 0, ctx->stream, S, d.counts, d.inv, d.facc,
                       d_F, d.xyzq, d.atom_sys, d.sys_acc, ctx->n_sys, en, vi, pf, ps, pself);
    }
    return cudaGetLastError();
}

size_t adjoint_smem_bytes(int T, int G)
{
    return (size_t)T * T * 32 + align16((size_t)T * T * 8) + (size_t)kAdjWarps * adj_warp_bytes(G);
}

template <int G, int RAD>
static void launch_adjoint_g(nb_ctx *ctx, const ForceArgs &A)
{
    const size_t smem = adjoint_smem_bytes(A.P.n_types, G);
    static std::atomic<unsigned long long> optin{0};
    smem_optin_once(k_adjoint<G, RAD>, ctx->device, 220 * 1024, optin);
    int resident = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_adjoint<G, RAD>, kAdjWarps * 32, smem);
    const int parts = ctx->tune.list_split > 0 ? ctx->tune.list_split : kDefaultListSplit;
    launch_pdl(k_adjoint<G, RAD>, dim3(ctx->num_sms * std::max(1, resident)), dim3(kAdjWarps * 32), smem,
               ctx->stream, A, parts);
}

template <int RAD>
static void launch_adjoint_1(nb_ctx *ctx, const ForceArgs &A)
{
    const size_t smem = adjoint1_smem_bytes(A.P.n_types);
    static std::atomic<unsigned long long> optin{0};
    smem_optin_once(k_adjoint1<RAD>, ctx->device, 220 * 1024, optin);
    int resident = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_adjoint1<RAD>, kAdjWarps * 32, smem);
    const int parts = ctx->tune.list_split > 0 ? ctx->tune.list_split : kDefaultListSplit;
    launch_pdl(k_adjoint1<RAD>, dim3(ctx->num_sms * std::max(1, resident)), dim3(kAdjWarps * 32), smem, ctx->stream,
               A, parts);
}

template <int RAD>
static void launch_adjoint_t(nb_ctx *ctx, const ForceArgs &A)
{
    if (ctx->built_group == 1) launch_adjoint_1<RAD>(ctx, A);
    else if (ctx->built_group == 4) launch_adjoint_g<4, RAD>(ctx, A);
    else launch_adjoint_g<8, RAD>(ctx, A);
}

size_t force_smem_for(int T, int scap, int K)
{
    (void)scap;  // unused: the kernels stage per batch of entries
    (void)K;     // the exclusion masks are built by the list kernel
    return std::max(tile_smem_bytes(T, kMaxGroup), adjoint_smem_bytes(T, kMaxGroup));
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
__global__ void k_debug_pair_terms(PairParams P, const float4 *__restrict__ lj_tab, const float4 *__restrict__ rtab,
                                   long long n, const float4 *__restrict__ xi, const float4 *__restrict__ xj,
                                   const int *__restrict__ ti, const int *__restrict__ tj, float4 *__restrict__ out)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float4 a = xi[k], b = xj[k];
    const float4 ab = lj_tab[ti[k] * P.n_types + tj[k]];
    float4 lj4[2];  // one type pair: (A, B, 12 A, 6 B), then the remainders at lj4 + n_types^2
    lj4[0] = make_float4(ab.x, ab.y, 12.0f * ab.x, 6.0f * ab.y);
    lj4[1] = make_float4(ab.z, ab.w, 0.0f, 0.0f);
    float dx, dy, dz;
    const float r2 = disp_r2(b.x, b.y, b.z, a.x, a.y, a.z, dx, dy, dz);
    Acc acc = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    float fjx = 0.0f, fjy = 0.0f, fjz = 0.0f;
    PairParams P1 = P;
    P1.n_types = 1;  // the one-pair table above
    eval_pair<RAD, false>(P1, lj4, rtab, 0, a.w * P.ke, true, dx, dy, dz, r2, b.w, 0, false, acc, fjx, fjy, fjz);
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
