// nb_build.cu - cell-list construction: wrap, column binning, per-column
// z-sort, cluster bounding boxes, sorted exclusion map and the cluster-pair
// list.  Section "Molecular dynamics on the GPU": particles are binned
// according to their coordinates, one particle per thread, with atomic
// operations for concurrent updates of the cell arrays.  Here the bins are
// x-y columns whose atoms are z-sorted and cut into 8-atom clusters, so the
// force kernel can prune whole clusters by bounding box.
#include <cuda_runtime.h>
#include <math.h>

#include "nb_internal.cuh"

namespace acenb {

__device__ __forceinline__ int column_of(float x, float inv_w, int n)
{
    int c = (int)floorf(__fmul_rn(x, inv_w));
    if (c > n - 1) c = n - 1;
    if (c < 0) c = 0;
    return c;
}

// A1: one atom per thread: wrap, column index, column histogram.
__global__ void k_bin(int n, const float *__restrict__ pos, const SysDesc *__restrict__ sys,
                      const int *__restrict__ atom_sys, float4 *__restrict__ wpos, int *__restrict__ atom_col,
                      int *__restrict__ col_count, int *__restrict__ status)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    const SysDesc &S = sys[atom_sys[a]];
    float x = pos[3 * a], y = pos[3 * a + 1], z = pos[3 * a + 2];
    if (!(isfinite(x) && isfinite(y) && isfinite(z))) {
        atomicOr(status, ST_NONFINITE);
        x = 0.0f; y = 0.0f; z = 0.0f;
    }
    x = wrap_coord(x, S.L[0]);
    y = wrap_coord(y, S.L[1]);
    z = wrap_coord(z, S.L[2]);
    int col = S.col_begin + column_of(y, S.inv_w[1], S.ny) * S.nx + column_of(x, S.inv_w[0], S.nx);
    atom_col[a] = col;
    wpos[a] = make_float4(x, y, z, 0.0f);
    atomicAdd(&col_count[col], 1);
}

// A2: exclusive scan of the padded column sizes (single block).  Also fills
// the scatter cursors, the totals and the per-system slot/cluster ranges.
__global__ void k_scan(int n_cols, int n_sys, const int *__restrict__ col_count, int *__restrict__ col_slot,
                       int *__restrict__ col_fill, SysDesc *__restrict__ sys, int *__restrict__ counts)
{
    __shared__ int warp_sum[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int base = 0; base < n_cols; base += blockDim.x) {
        int c = base + threadIdx.x;
        int v = c < n_cols ? (col_count[c] + kCluster - 1) / kCluster * kCluster : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int s = lane < nw ? warp_sum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            if (lane < nw) warp_sum[lane] = s;
        }
        __syncthreads();
        int excl = carry + (wid ? warp_sum[wid - 1] : 0) + x - v;
        if (c < n_cols) { col_slot[c] = excl; col_fill[c] = excl; }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        col_slot[n_cols] = carry;
        counts[0] = carry;
        counts[1] = carry / kCluster;
    }
    __syncthreads();
    for (int s = threadIdx.x; s < n_sys; s += blockDim.x) {
        int c0 = sys[s].col_begin, c1 = c0 + sys[s].nx * sys[s].ny;
        sys[s].slot_begin = col_slot[c0];
        sys[s].clus_begin = col_slot[c0] / kCluster;
        sys[s].clus_end = col_slot[c1] / kCluster;
    }
}

// A3a: place atoms into their column segment (order fixed by the sort below).
__global__ void k_scatter(int n, const int *__restrict__ atom_col, int *__restrict__ col_fill,
                          int *__restrict__ stage)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    int p = atomicAdd(&col_fill[atom_col[a]], 1);
    stage[p] = a;
}

constexpr int kSortSmem = 1024;  // atoms per column sorted from shared memory

// A3b: one block per column: rank sort by (z, atom index), write the sorted
// slot arrays and padding, then the cluster bounding boxes.
__global__ void k_colsort(const int *__restrict__ col_count, const int *__restrict__ col_slot,
                          const int *__restrict__ col_sys, const int *__restrict__ stage,
                          const float4 *__restrict__ wpos, float4 *__restrict__ xyzq, int *__restrict__ tslot,
                          int *__restrict__ perm, int *__restrict__ inv, float4 *__restrict__ bb,
                          int *__restrict__ clus_sys)
{
    __shared__ float sz[kSortSmem];
    __shared__ int sid[kSortSmem];
    __shared__ float4 sp[kSortSmem];
    const int c = blockIdx.x;
    const int n = col_count[c];
    const int base = col_slot[c];
    const int npad = (n + kCluster - 1) / kCluster * kCluster;
    const bool small = n <= kSortSmem;
    if (small) {
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            int a = stage[base + k];
            sid[k] = a;
            sz[k] = wpos[a].z;
        }
        __syncthreads();
    }
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        int a = small ? sid[k] : stage[base + k];
        float z = small ? sz[k] : wpos[a].z;
        int rank = 0;
        for (int m = 0; m < n; ++m) {
            int b = small ? sid[m] : stage[base + m];
            float zb = small ? sz[m] : wpos[b].z;
            rank += (zb < z) || (zb == z && b < a);
        }
        int slot = base + rank;
        float4 p = wpos[a];
        perm[slot] = a;
        inv[a] = slot;
        xyzq[slot] = make_float4(p.x, p.y, p.z, 0.0f);
        if (small) sp[rank] = p;
    }
    for (int k = n + threadIdx.x; k < npad; k += blockDim.x) {
        perm[base + k] = -1;
        tslot[base + k] = 0;
        xyzq[base + k] = make_float4(kPadCoord, kPadCoord, kPadCoord, 0.0f);
    }
    __syncthreads();
    // cluster bounding boxes over the real atoms of each 8-slot cluster
    const int nclus = npad / kCluster;
    for (int q = threadIdx.x; q < nclus; q += blockDim.x) {
        float lx = INFINITY, ly = INFINITY, lz = INFINITY, hx = -INFINITY, hy = -INFINITY, hz = -INFINITY;
        for (int k = q * kCluster; k < min(n, (q + 1) * kCluster); ++k) {
            float4 p = small ? sp[k] : xyzq[base + k];
            lx = fminf(lx, p.x); ly = fminf(ly, p.y); lz = fminf(lz, p.z);
            hx = fmaxf(hx, p.x); hy = fmaxf(hy, p.y); hz = fmaxf(hz, p.z);
        }
        int I = base / kCluster + q;
        bb[2 * I] = make_float4(lx, ly, lz, 0.0f);
        bb[2 * I + 1] = make_float4(hx, hy, hz, 0.0f);
        clus_sys[I] = col_sys[c];
    }
}

// A4a: exclusion/1-4 partners in sorted-slot space.
__global__ void k_exmap(int slot_cap, const int *__restrict__ counts, int K, const int *__restrict__ perm,
                        const int *__restrict__ part_orig, const int *__restrict__ inv, int *__restrict__ ex_slot)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= slot_cap || s >= counts[0]) return;
    int a = perm[s];
    for (int k = 0; k < K; ++k) {
        int v = -1;
        if (a >= 0) {
            int p = part_orig[(long long)a * K + k];
            if (p >= 0) v = (inv[p >> 1] << 1) | (p & 1);
        }
        ex_slot[(long long)s * K + k] = v;
    }
}

// A4b: cluster-pair list, one warp per cluster I.  Enumerates the columns
// within reach of I's bounding box (with periodic images), tests every
// cluster of those columns against I under each admissible z image, and
// appends (J, shift codes, exclusion flag) for bounding-box gaps below the
// cutoff (plus a rounding margin).
__global__ void k_list(const SysDesc *__restrict__ sys, const int *__restrict__ counts,
                       const float4 *__restrict__ bb,
                       const int *__restrict__ clus_sys, const int *__restrict__ col_slot,
                       const int *__restrict__ ex_slot, int K, float rcm, int cap,
                       uint32_t *__restrict__ list, int *__restrict__ list_n, int *__restrict__ status)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int n_clus = counts[1];
    const float rcm2 = rcm * rcm;
    const unsigned lt = (1u << lane) - 1u;
    for (int I = gw; I < n_clus; I += nw) {
        const SysDesc &S = sys[clus_sys[I]];
        const float4 lo = bb[2 * I], hi = bb[2 * I + 1];
        // distinct partner clusters of I (lanes 0..npc-1 of pcl)
        int pcl = -1, npc = 0;
        bool flag_all = false;
        const int np = kCluster * K;
        for (int b = 0; b < np; b += 32) {
            int v = -1;
            if (b + lane < np) {
                int e = ex_slot[(long long)I * kCluster * K + b + lane];
                if (e >= 0) v = (e >> 1) / kCluster;
            }
            unsigned peers = __match_any_sync(FULL, v);
            bool leader = (v >= 0) && ((__ffs(peers) - 1) == lane);
            // drop values already present
            for (int m = 0; m < npc; ++m) {
                int u = __shfl_sync(FULL, pcl, m);
                if (u == v) leader = false;
            }
            unsigned bal = __ballot_sync(FULL, leader);
            if (npc + __popc(bal) > 32) flag_all = true;
            // append the new leaders to the lane-distributed list pcl
            int p = npc;
            for (unsigned b2 = bal; b2; b2 &= b2 - 1u, ++p) {
                int vv = __shfl_sync(FULL, v, __ffs(b2) - 1);
                if (lane == p) pcl = vv;
            }
            npc = min(32, npc + __popc(bal));
        }
        int cnt = 0;
        const int cxa = max(-S.nx, (int)floorf((lo.x - rcm) * S.inv_w[0]));
        const int cxb = min(2 * S.nx - 1, (int)floorf((hi.x + rcm) * S.inv_w[0]));
        const int cya = max(-S.ny, (int)floorf((lo.y - rcm) * S.inv_w[1]));
        const int cyb = min(2 * S.ny - 1, (int)floorf((hi.y + rcm) * S.inv_w[1]));
        const bool zdn = (lo.z - rcm) < 0.0f;
        const bool zup = (hi.z + rcm) >= S.L[2];
        const int ncx = cxb - cxa + 1, ncand = ncx * (cyb - cya + 1);
        // lanes over candidate columns; clusters of a column in lock-step
        for (int c0 = 0; c0 < ncand; c0 += 32) {
            const int c = c0 + lane;
            const bool cv = c < ncand;
            const int cy = cya + (cv ? c / ncx : 0), cx = cxa + (cv ? c % ncx : 0);
            const int ccy = cy < 0 ? cy + S.ny : (cy >= S.ny ? cy - S.ny : cy);
            const int ccx = cx < 0 ? cx + S.nx : (cx >= S.nx ? cx - S.nx : cx);
            const int sy = cy < 0 ? 1 : (cy >= S.ny ? 2 : 0);
            const int sx = cx < 0 ? 1 : (cx >= S.nx ? 2 : 0);
            const float oy = sy == 1 ? -S.L[1] : (sy == 2 ? S.L[1] : 0.0f);
            const float ox = sx == 1 ? -S.L[0] : (sx == 2 ? S.L[0] : 0.0f);
            int jb = 0, nj = 0;
            if (cv) {
                const int col = S.col_begin + ccy * S.nx + ccx;
                jb = col_slot[col] / kCluster;
                nj = col_slot[col + 1] / kCluster - jb;
            }
            int maxj = nj;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) maxj = max(maxj, __shfl_xor_sync(FULL, maxj, o));
            const uint32_t code_xy = ((uint32_t)sx << kShiftBit) | ((uint32_t)sy << (kShiftBit + 2));
            for (int k0 = 0; k0 < maxj; k0 += 4) {
                float4 jl[4], jh[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const bool v = k0 + u < nj;
                    jl[u] = v ? bb[2 * (jb + k0 + u)] : make_float4(INFINITY, INFINITY, INFINITY, 0.0f);
                    jh[u] = v ? bb[2 * (jb + k0 + u) + 1] : make_float4(INFINITY, INFINITY, INFINITY, 0.0f);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (k0 + u >= maxj) break;
                    const int J = jb + k0 + u;
                    const bool v = k0 + u < nj;
                    const float gx = fmaxf(fmaxf((jl[u].x + ox) - hi.x, lo.x - (jh[u].x + ox)), 0.0f);
                    const float gy = fmaxf(fmaxf((jl[u].y + oy) - hi.y, lo.y - (jh[u].y + oy)), 0.0f);
                    const float gxy = gx * gx + gy * gy;
                    bool fl = flag_all;
                    for (int m = 0; m < npc; ++m) fl |= (__shfl_sync(FULL, pcl, m) == J);
#pragma unroll
                    for (int sz = 0; sz < 3; ++sz) {
                        const float oz = sz == 1 ? -S.L[2] : (sz == 2 ? S.L[2] : 0.0f);
                        const float gz = fmaxf(fmaxf((jl[u].z + oz) - hi.z, lo.z - (jh[u].z + oz)), 0.0f);
                        const bool zok = sz == 0 || (sz == 1 && zdn) || (sz == 2 && zup);
                        const bool keep = v && zok && (gxy + gz * gz < rcm2);
                        const unsigned bal = __ballot_sync(FULL, keep);
                        if (keep) {
                            const int p = cnt + __popc(bal & lt);
                            const uint32_t ent = (uint32_t)J | code_xy | ((uint32_t)sz << (kShiftBit + 4)) |
                                                 (fl ? kExclFlag : 0u);
                            if (p < cap) list[(long long)I * cap + p] = ent;
                        }
                        cnt += __popc(bal);
                    }
                }
            }
        }
        if (lane == 0) {
            list_n[I] = min(cnt, cap);
            if (cnt > cap) atomicOr(status, ST_CAPACITY);
        }
    }
}

cudaError_t launch_build(nb_ctx *ctx, const float *d_pos)
{
    auto &d = ctx->d;
    cudaStream_t st = ctx->stream;
    const int N = (int)ctx->n_atoms;
    cudaError_t e = cudaMemsetAsync(d.col_count, 0, sizeof(int) * ctx->n_cols, st);
    if (e != cudaSuccess) return e;
    const int tb = 256;
    k_bin<<<(N + tb - 1) / tb, tb, 0, st>>>(N, d_pos, d.sys, d.atom_sys, d.wpos, d.atom_col, d.col_count, d.status);
    k_scan<<<1, 1024, 0, st>>>(ctx->n_cols, ctx->n_sys, d.col_count, d.col_slot, d.col_fill, d.sys, d.counts);
    k_scatter<<<(N + tb - 1) / tb, tb, 0, st>>>(N, d.atom_col, d.col_fill, d.stage);
    k_colsort<<<ctx->n_cols, 128, 0, st>>>(d.col_count, d.col_slot, d.col_sys, d.stage, d.wpos, d.xyzq, d.tslot,
                                           d.perm, d.inv, d.bb, d.clus_sys);
    const int S = (int)ctx->slot_cap;
    k_exmap<<<(S + tb - 1) / tb, tb, 0, st>>>(S, d.counts, ctx->K, d.perm, d.part_orig, d.inv, d.ex_slot);
    const int lw = 8;  // warps per block in the list kernel
    int lblocks = (int)((ctx->clus_cap + lw - 1) / lw);
    int lmax = ctx->num_sms * 16;
    if (lblocks > lmax) lblocks = lmax;
    if (lblocks < 1) lblocks = 1;
    k_list<<<lblocks, lw * 32, 0, st>>>(d.sys, d.counts, d.bb, d.clus_sys, d.col_slot, d.ex_slot,
                                        ctx->K, ctx->pp.rc + ctx->pp.list_margin, ctx->tune.list_capacity,
                                        d.list, d.list_n, d.status);
    return cudaGetLastError();
}

}  // namespace acenb
