// nb_force.cu - the non-bonded force kernel (section "Molecular dynamics on
// the GPU": the non-bonded kernel computes the full Lennard-Jones and
// electrostatic force on each particle; as in the paper, the reciprocal force
// F_ji is not reused, so every atom accumulates its own force and no
// scattered writes or atomics are needed).
//
// Work decomposition (GB300 design, not the paper's one-cell-per-block):
//   task  = (cluster I of 8 sorted atoms, i-group of MI consecutive atoms);
//   warp  = one task at a time, persistent grid of warps;
//   lanes = MI i-atoms x JS = 32/MI j-slots.
// For each task the warp streams I's cluster-pair list, tests every candidate
// j atom against the i-group's bounding box and compacts the survivors into a
// per-warp shared-memory queue (x, y, z, q and a type/exclusion word).  Full
// JS-wide steps of the queue are then evaluated pair by pair in FP32.  Queue
// entries needing an i-side periodic shift, an exclusion test or the i == j
// test (the paper's "inner" kernel) go to the top of the queue and use the
// general path; everything else (the "outer" kernel) uses the fast path.
#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "nb_pair.cuh"

namespace acenb {

constexpr int kQCap = 256;   // queue entries per warp
using FastT = std::integral_constant<bool, false>;  // outer (no exclusion test) path
using GenT = std::integral_constant<bool, true>;    // inner path
constexpr unsigned kFull = 0xffffffffu;

struct ForceArgs {
    const SysDesc *sys;
    const int *counts;
    const float4 *xyzq;
    const int *tslot;
    const int *perm;
    const int *clus_sys;
    const uint32_t *list;
    const int *list_n;
    int cap;
    const int *ex_slot;
    int K;
    const float2 *lj_tab;
    float *F;
    long long *task_part;
    int *status;
    long long *dbg_n;
    int *dbg_ij;
    long long dbg_cap;
    PairParams P;
};

struct Acc {
    float fx, fy, fz, elj, ec;
    float w[6];
};

template <bool EWALD, bool VIRIAL, bool DEBUG, bool GENERAL>
__device__ __forceinline__ void eval_entry(const ForceArgs &A, const float2 *__restrict__ lj, int ti_row,
                                           float xi, float yi, float zi, float xim, float yim, float zim,
                                           float qi, int il, int iorig, float4 pj, uint32_t w, int jorig,
                                           Acc &acc)
{
    float ax = xi, ay = yi, az = zi;
    if (GENERAL) {
        if (w & (1u << kQIShift)) ax = xim;
        if (w & (2u << kQIShift)) ay = yim;
        if (w & (4u << kQIShift)) az = zim;
    }
    float dx, dy, dz;
    const float r2 = disp_r2(pj.x, pj.y, pj.z, ax, ay, az, dx, dy, dz);
    bool in = r2 < A.P.rc2;
    float wlj = 1.0f, wc = 1.0f;
    if (GENERAL) {
        if ((w >> (kQExcl + il)) & 1u) in = false;
        if ((w >> (kQ14 + il)) & 1u) { wlj = A.P.s14_lj; wc = A.P.s14_c; }
    }
    const float rinv = rsqrtf(r2);
    const float2 ab = lj[ti_row + (int)(w & 0xFFu)];
    float elj, frlj, ec, frc;
    pair_radial<EWALD, true>(A.P, r2, rinv, ab.x, ab.y, qi * pj.w, elj, frlj, ec, frc);
    float fs = fmaf(wlj, frlj, wc * frc) * (rinv * rinv);
    fs = in ? fs : 0.0f;
    // F_i = U'(r) d / r = -fs d  with fs = -U'(r) / r
    acc.fx = fmaf(-fs, dx, acc.fx);
    acc.fy = fmaf(-fs, dy, acc.fy);
    acc.fz = fmaf(-fs, dz, acc.fz);
    acc.elj += in ? wlj * elj : 0.0f;
    acc.ec += in ? wc * ec : 0.0f;
    if (VIRIAL) {
        // W_ab += d_ij,a f_ij,b with d_ij = -d and f_ij = -fs d
        const float fdx = fs * dx, fdy = fs * dy, fdz = fs * dz;
        acc.w[0] = fmaf(fdx, dx, acc.w[0]);
        acc.w[1] = fmaf(fdy, dy, acc.w[1]);
        acc.w[2] = fmaf(fdz, dz, acc.w[2]);
        acc.w[3] = fmaf(fdx, dy, acc.w[3]);
        acc.w[4] = fmaf(fdx, dz, acc.w[4]);
        acc.w[5] = fmaf(fdy, dz, acc.w[5]);
    }
    if (DEBUG && in) {
        atomicAdd((unsigned long long *)&A.dbg_n[0], 1ull);
        if (iorig < jorig) {
            long long k = (long long)atomicAdd((unsigned long long *)&A.dbg_n[1], 1ull);
            if (k < A.dbg_cap) {
                A.dbg_ij[2 * k] = iorig;
                A.dbg_ij[2 * k + 1] = jorig;
            }
        }
    }
}

__device__ __forceinline__ long long to_fixed(float v, int *status)
{
    // |v| < 2^26 keeps the sum of 32 lanes inside int64 at scale 2^32
    if (!(fabsf(v) < 67108864.0f)) {
        atomicOr(status, ST_OVERFLOW);
        return 0;
    }
    return __float2ll_rn(v * 4294967296.0f);
}

template <int MI, bool EWALD, bool VIRIAL, bool DEBUG>
__global__ void __launch_bounds__(256) k_force(ForceArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int GPC = kCluster / MI;
    constexpr int JS = 32 / MI;
    const int T = A.P.n_types;
    const int nwarps = blockDim.x >> 5;
    const int wib = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;

    float2 *lj = reinterpret_cast<float2 *>(smem);
    const int tab_bytes = (T * T * 8 + 15) & ~15;
    float4 *qpos = reinterpret_cast<float4 *>(smem + tab_bytes) + wib * kQCap;
    uint32_t *qword = reinterpret_cast<uint32_t *>(smem + tab_bytes + nwarps * kQCap * 16) + wib * kQCap;
    int *qorig = DEBUG ? reinterpret_cast<int *>(smem + tab_bytes + nwarps * kQCap * 20) + wib * kQCap : nullptr;
    for (int k = threadIdx.x; k < T * T; k += blockDim.x) lj[k] = A.lj_tab[k];
    __syncthreads();

    const int il = lane % MI;
    const int js = lane / MI;
    const int n_tasks = A.counts[1] * GPC;
    const int npk = MI * A.K;
    const float4 padj = make_float4(-kFar, -kFar, -kFar, 0.0f);

    for (int t = blockIdx.x * nwarps + wib; t < n_tasks; t += gridDim.x * nwarps) {
        const int I = t / GPC;
        const int i0 = I * kCluster + (t - I * GPC) * MI;
        const float4 pi = A.xyzq[i0 + il];
        const int ti = A.tslot[i0 + il];
        const bool iv = pi.x == pi.x;
        const SysDesc &S = A.sys[A.clus_sys[I]];
        const float Lx = S.L[0], Ly = S.L[1], Lz = S.L[2];
        const float xi = iv ? pi.x : kFar, yi = iv ? pi.y : kFar, zi = iv ? pi.z : kFar;
        const float xim = __fsub_rn(xi, Lx), yim = __fsub_rn(yi, Ly), zim = __fsub_rn(zi, Lz);
        const float qi = iv ? pi.w * A.P.ke : 0.0f;
        const int ti_row = ti * T;
        const int iorig = DEBUG ? A.perm[i0 + il] : -1;
        // bounding box of the i-group (valid atoms only)
        float lox = iv ? pi.x : INFINITY, loy = iv ? pi.y : INFINITY, loz = iv ? pi.z : INFINITY;
        float hix = iv ? pi.x : -INFINITY, hiy = iv ? pi.y : -INFINITY, hiz = iv ? pi.z : -INFINITY;
#pragma unroll
        for (int o = 1; o < MI; o <<= 1) {
            lox = fminf(lox, __shfl_xor_sync(kFull, lox, o));
            loy = fminf(loy, __shfl_xor_sync(kFull, loy, o));
            loz = fminf(loz, __shfl_xor_sync(kFull, loz, o));
            hix = fmaxf(hix, __shfl_xor_sync(kFull, hix, o));
            hiy = fmaxf(hiy, __shfl_xor_sync(kFull, hiy, o));
            hiz = fmaxf(hiz, __shfl_xor_sync(kFull, hiz, o));
        }
        if (!__any_sync(kFull, iv)) {
            if (lane < kTaskVals) A.task_part[(long long)t * kTaskVals + lane] = 0;
            continue;
        }
        const int pe = lane < npk ? A.ex_slot[(long long)i0 * A.K + lane] : -1;

        Acc acc;
        acc.fx = acc.fy = acc.fz = acc.elj = acc.ec = 0.0f;
#pragma unroll
        for (int k = 0; k < 6; ++k) acc.w[k] = 0.0f;

        auto drain = [&](int beg, int end, auto general) {
            constexpr bool GEN = decltype(general)::value;
            for (int k = beg; k < end; k += JS) {
                const int e = k + js;
                const float4 pj = qpos[e];
                const uint32_t w = qword[e];
                const int jo = DEBUG ? qorig[e] : 0;
                eval_entry<EWALD, VIRIAL, DEBUG, GEN>(A, lj, ti_row, xi, yi, zi, xim, yim, zim, qi, il, iorig,
                                                      pj, w, jo, acc);
            }
        };

        int nA = 0, nB = 0;
        const int nE = A.list_n[I];
        const uint32_t *L0 = A.list + (long long)I * A.cap;
        for (int e0 = 0; e0 < nE; e0 += 4) {
            const int e = e0 + (lane >> 3);
            const bool ok = e < nE;
            const uint32_t ent = ok ? L0[e] : 0u;
            const int J = (int)(ent & kJMask);
            const int cx = (ent >> kShiftBit) & 3, cy = (ent >> (kShiftBit + 2)) & 3, cz = (ent >> (kShiftBit + 4)) & 3;
            const bool fl = (ent & kExclFlag) != 0u;
            const int j = J * kCluster + (lane & 7);
            float4 pj = ok ? A.xyzq[j] : padj;
            const int tj = ok ? A.tslot[j] : 0;
            const bool jv = ok && (pj.x == pj.x);
            if (cx == 1) pj.x = __fsub_rn(pj.x, Lx);
            if (cy == 1) pj.y = __fsub_rn(pj.y, Ly);
            if (cz == 1) pj.z = __fsub_rn(pj.z, Lz);
            const float bxl = cx == 2 ? lox - Lx : lox, bxh = cx == 2 ? hix - Lx : hix;
            const float byl = cy == 2 ? loy - Ly : loy, byh = cy == 2 ? hiy - Ly : hiy;
            const float bzl = cz == 2 ? loz - Lz : loz, bzh = cz == 2 ? hiz - Lz : hiz;
            const float gx = fmaxf(fmaxf(bxl - pj.x, pj.x - bxh), 0.0f);
            const float gy = fmaxf(fmaxf(byl - pj.y, pj.y - byh), 0.0f);
            const float gz = fmaxf(fmaxf(bzl - pj.z, pj.z - bzh), 0.0f);
            const bool keep = jv && (gx * gx + gy * gy + gz * gz < A.P.rcm2);
            const uint32_t ish = (uint32_t)(cx == 2) | ((uint32_t)(cy == 2) << 1) | ((uint32_t)(cz == 2) << 2);
            const bool self = (J == I) && (((ent >> kShiftBit) & 0x3Fu) == 0u);
            const bool clsB = keep && (ish != 0u || self || fl);
            uint32_t word = (uint32_t)tj | (ish << kQIShift);
            if (__any_sync(kFull, clsB && (self || fl))) {
                uint32_t bits = 0u;
                if (self) {
                    const int m = j - i0;
                    if (m >= 0 && m < MI) bits |= 1u << (kQExcl + m);
                }
                for (int m = 0; m < npk; ++m) {
                    const int pv = __shfl_sync(kFull, pe, m);
                    if (fl && pv >= 0 && (pv >> 1) == j)
                        bits |= 1u << (((pv & 1) ? kQ14 : kQExcl) + m / A.K);
                }
                word |= bits;
            }
            const bool toA = keep && !clsB;
            const unsigned bA = __ballot_sync(kFull, toA);
            const unsigned bB = __ballot_sync(kFull, clsB);
            if (toA) {
                const int p = nA + __popc(bA & lt);
                qpos[p] = pj;
                qword[p] = word;
                if (DEBUG) qorig[p] = A.perm[j];
            }
            if (clsB) {
                const int p = kQCap - 1 - (nB + __popc(bB & lt));
                qpos[p] = pj;
                qword[p] = word;
                if (DEBUG) qorig[p] = A.perm[j];
            }
            nA += __popc(bA);
            nB += __popc(bB);
            __syncwarp();
            if (nA + nB + 32 > kQCap) {
                // drain whole JS-wide steps from the inner end of each region;
                // the remainders stay where they are (bottom of A, top of B)
                const int remA = nA % JS;
                drain(remA, nA, FastT{});
                nA = remA;
                if (nA + nB + 32 > kQCap) {
                    const int remB = nB % JS;
                    drain(kQCap - nB, kQCap - remB, GenT{});
                    nB = remB;
                }
                __syncwarp();
            }
        }
        // final drains: whole steps first, then one padded step per region
        {
            const int remB = nB % JS;
            drain(kQCap - nB, kQCap - remB, GenT{});
            const int remA = nA % JS;
            drain(remA, nA, FastT{});
            __syncwarp();
            if (remA) {
                if (lane >= remA && lane < JS) { qpos[lane] = padj; qword[lane] = 0u; if (DEBUG) qorig[lane] = 0; }
                __syncwarp();
                drain(0, JS, FastT{});
            }
            if (remB) {
                const int p = kQCap - JS + lane;
                if (lane < JS - remB) { qpos[p] = padj; qword[p] = 0u; if (DEBUG) qorig[p] = 0; }
                __syncwarp();
                drain(kQCap - JS, kQCap, GenT{});
            }
            __syncwarp();
        }
        // forces: sum the JS lanes of each i atom in 64-bit fixed point
        long long vx = to_fixed(acc.fx, A.status), vy = to_fixed(acc.fy, A.status), vz = to_fixed(acc.fz, A.status);
#pragma unroll
        for (int o = MI; o < 32; o <<= 1) {
            vx += __shfl_xor_sync(kFull, vx, o);
            vy += __shfl_xor_sync(kFull, vy, o);
            vz += __shfl_xor_sync(kFull, vz, o);
        }
        if (js == 0 && iv) {
            const int a = A.perm[i0 + il];
            const float sc = 2.3283064365386963e-10f;  // 2^-32
            A.F[3 * (long long)a] = __ll2float_rn(vx) * sc;
            A.F[3 * (long long)a + 1] = __ll2float_rn(vy) * sc;
            A.F[3 * (long long)a + 2] = __ll2float_rn(vz) * sc;
        }
        // energies and virial of the task: FP32 butterfly (fixed order), then fixed point
        float v[kTaskVals] = {acc.elj, acc.ec, acc.w[0], acc.w[1], acc.w[2], acc.w[3], acc.w[4], acc.w[5]};
#pragma unroll
        for (int k = 0; k < (VIRIAL ? kTaskVals : 2); ++k) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(kFull, v[k], o);
        }
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < kTaskVals; ++k)
                A.task_part[(long long)t * kTaskVals + k] = (VIRIAL || k < 2) ? to_fixed(v[k], A.status) : 0ll;
        }
    }
}

// Gather charges and types into sorted order and check that the positions
// are those of the last build.
__global__ void k_pack(int slot_cap, const int *__restrict__ counts, const int *__restrict__ perm,
                       float4 *__restrict__ xyzq, int *__restrict__ tslot, const float *__restrict__ pos,
                       const float *__restrict__ q, const int *__restrict__ type, const SysDesc *__restrict__ sys,
                       const int *__restrict__ atom_sys, int T, int *__restrict__ status)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
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

// Per-system energy/virial: exact int64 sum of the task partials (order
// independent, hence deterministic), halved because every pair is visited
// from both of its atoms.
__global__ void k_reduce(const SysDesc *__restrict__ sys, int gpc, const long long *__restrict__ task_part,
                         double *__restrict__ energy, double *__restrict__ virial)
{
    __shared__ long long red[kTaskVals][256];
    const int s = blockIdx.x;
    const int t0 = sys[s].clus_begin * gpc, t1 = sys[s].clus_end * gpc;
    long long acc[kTaskVals] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x)
#pragma unroll
        for (int k = 0; k < kTaskVals; ++k) acc[k] += task_part[(long long)t * kTaskVals + k];
#pragma unroll
    for (int k = 0; k < kTaskVals; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
#pragma unroll
            for (int k = 0; k < kTaskVals; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < kTaskVals) {
        const double v = (double)red[threadIdx.x][0] * (0.5 / kFixScale);
        if (threadIdx.x < 2) {
            if (energy) energy[2 * s + threadIdx.x] = v;
        } else if (virial) {
            virial[6 * s + threadIdx.x - 2] = v;
        }
    }
}

template <int MI, bool EWALD, bool VIRIAL, bool DEBUG>
static void launch_force_t(nb_ctx *ctx, const ForceArgs &A)
{
    const int nw = ctx->tune.warps_per_block;
    const int tab_bytes = (A.P.n_types * A.P.n_types * 8 + 15) & ~15;
    const size_t smem = (size_t)tab_bytes + (size_t)nw * kQCap * (DEBUG ? 24 : 20);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_force<MI, EWALD, VIRIAL, DEBUG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
        attr_set = true;
    }
    const int grid = ctx->num_sms * ctx->tune.blocks_per_sm;
    k_force<MI, EWALD, VIRIAL, DEBUG><<<grid, nw * 32, smem, ctx->stream>>>(A);
}

template <int MI>
static void launch_force_mi(nb_ctx *ctx, const ForceArgs &A, bool ewald, bool virial, bool debug)
{
    if (debug) {
        if (ewald) launch_force_t<MI, true, false, true>(ctx, A);
        else launch_force_t<MI, false, false, true>(ctx, A);
        return;
    }
    if (ewald) {
        if (virial) launch_force_t<MI, true, true, false>(ctx, A);
        else launch_force_t<MI, true, false, false>(ctx, A);
    } else {
        if (virial) launch_force_t<MI, false, true, false>(ctx, A);
        else launch_force_t<MI, false, false, false>(ctx, A);
    }
}

cudaError_t launch_forces(nb_ctx *ctx, const float *d_pos, const float *d_q, const int32_t *d_type, float *d_F,
                          double *d_energy, double *d_virial, bool debug_pairs)
{
    auto &d = ctx->d;
    const int tb = 256;
    const int S = (int)ctx->slot_cap;
    if (d_pos)  // the debug pair export reuses the last packed values
        k_pack<<<(S + tb - 1) / tb, tb, 0, ctx->stream>>>(S, d.counts, d.perm, d.xyzq, d.tslot, d_pos, d_q, d_type,
                                                           d.sys, d.atom_sys, ctx->pp.n_types, d.status);
    ForceArgs A;
    A.sys = d.sys;
    A.counts = d.counts;
    A.xyzq = d.xyzq;
    A.tslot = d.tslot;
    A.perm = d.perm;
    A.clus_sys = d.clus_sys;
    A.list = d.list;
    A.list_n = d.list_n;
    A.cap = ctx->tune.list_capacity;
    A.ex_slot = d.ex_slot;
    A.K = ctx->K;
    A.lj_tab = d.lj_tab;
    A.F = d_F;
    A.task_part = d.task_part;
    A.status = d.status;
    A.dbg_n = d.dbg_n;
    A.dbg_ij = d.dbg_ij;
    A.dbg_cap = d.dbg_cap;
    A.P = ctx->pp;
    const bool ewald = ctx->pp.ewald != 0;
    const bool virial = d_virial != nullptr;
    const bool prof = ctx->profiling && ctx->prof_n < (int)ctx->prof_ev.size() / 2;
    if (prof) cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n], ctx->stream);
    switch (ctx->tune.i_group) {
    case 4: launch_force_mi<4>(ctx, A, ewald, virial, debug_pairs); break;
    default: launch_force_mi<2>(ctx, A, ewald, virial, debug_pairs); break;
    }
    if (prof) {
        cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n + 1], ctx->stream);
        ctx->prof_n++;
    }
    if (!debug_pairs && (d_energy || d_virial)) {
        const int gpc = kCluster / (ctx->tune.i_group == 4 ? 4 : 2);
        k_reduce<<<ctx->n_sys, 256, 0, ctx->stream>>>(d.sys, gpc, d.task_part, d_energy, d_virial);
    }
    return cudaGetLastError();
}

}  // namespace acenb
