// nb_build.cu - cell-list construction: wrap, column binning, per-column
// z-sort, cluster bounding boxes and the cluster-pair lists.  Section
// "Molecular dynamics on the GPU": particles are binned according to their
// coordinates, one particle per thread, with atomic operations for concurrent
// updates of the cell arrays; the force kernel then visits the neighbour
// cells within the cutoff.  Here the bins are x-y columns whose atoms are
// z-sorted and cut into 8-atom clusters, and each cluster gets the list of
// clusters whose bounding boxes come within the cutoff, so the force kernel
// can stage exactly those.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "nb_internal.cuh"

namespace acenb {

__device__ __forceinline__ int column_of(float x, float inv_w, int n)
{
    int c = (int)floorf(__fmul_rn(x, inv_w));
    if (c > n - 1) c = n - 1;
    if (c < 0) c = 0;
    return c;
}

// Warp-aggregated counter update: lanes with the same key (-1 = none) take
// consecutive positions from one atomic per distinct key; returns the old
// counter value plus the lane's rank among its peers.
__device__ __forceinline__ int warp_aggregated_add(int *counter_base, int key)
{
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (key >= 0 && lane == leader) base = atomicAdd(&counter_base[key], __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    return base + __popc(peers & ((1u << lane) - 1u));
}

// Block-wide exclusive scan of the padded column sizes (one block).  Fills
// the column slot offsets, the scatter cursors, the totals and the
// per-system slot/cluster ranges.
__device__ void scan_columns(int n_cols, int n_sys, const int *__restrict__ col_count, int *__restrict__ col_slot,
                             int *__restrict__ col_fill, SysDesc *__restrict__ sys, int *__restrict__ counts)
{
    __shared__ int warp_sum[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int base = 0; base < n_cols; base += blockDim.x) {
        int c = base + threadIdx.x;
        int v = c < n_cols ? (__ldcg(&col_count[c]) + kCluster - 1) / kCluster * kCluster : 0;
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

// A1 + A2: one atom per thread: wrap, column index, column histogram
// (warp-aggregated atomics); the last block to finish scans the histogram.
// col_count[n_cols] is the completion ticket (zero on entry, reset on exit).
__global__ void k_bin(int n, const float *__restrict__ pos, SysDesc *__restrict__ sys,
                      const int *__restrict__ atom_sys, float4 *__restrict__ wpos, int *__restrict__ atom_col,
                      int *__restrict__ col_count, int n_cols, int n_sys, int *__restrict__ col_slot,
                      int *__restrict__ col_fill, int *__restrict__ counts, int *__restrict__ status)
{
    pdl_entry();
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    int col = -1;
    if (a < n) {
        const SysDesc &S = sys[atom_sys[a]];
        float x = pos[3ll * a], y = pos[3ll * a + 1], z = pos[3ll * a + 2];
        if (!(isfinite(x) && isfinite(y) && isfinite(z))) {
            atomicOr(status, ST_NONFINITE);
            x = 0.0f; y = 0.0f; z = 0.0f;
        }
        x = wrap_coord(x, S.L[0]);
        y = wrap_coord(y, S.L[1]);
        z = wrap_coord(z, S.L[2]);
        // a finite coordinate too large for the FP32 wrap (|x| beyond ~2^24 L)
        // is reported like a non-finite one: every later index stays in range
        if (!(x >= 0.0f && x < S.L[0] && y >= 0.0f && y < S.L[1] && z >= 0.0f && z < S.L[2])) {
            atomicOr(status, ST_NONFINITE);
            x = 0.0f; y = 0.0f; z = 0.0f;
        }
        col = S.col_begin + column_of(y, S.inv_w[1], S.ny) * S.nx + column_of(x, S.inv_w[0], S.nx);
        atom_col[a] = col;
        wpos[a] = make_float4(x, y, z, 0.0f);
    }
    warp_aggregated_add(col_count, col);
    // last block: the histogram is complete.  The barrier orders the block's
    // counter updates before thread 0's fence, which (cumulatively) orders
    // them before the ticket.
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&col_count[n_cols], 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    scan_columns(n_cols, n_sys, col_count, col_slot, col_fill, sys, counts);
    if (threadIdx.x == 0) col_count[n_cols] = 0;
}

// A3a: place atoms into their column segment (order fixed by the sort below).
__global__ void k_scatter(int n, const int *__restrict__ atom_col, int *__restrict__ col_fill,
                          int *__restrict__ stage)
{
    pdl_entry();
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int col = a < n ? atom_col[a] : -1;
    const int p = warp_aggregated_add(col_fill, col);
    if (a < n) stage[p] = a;
}

constexpr int kSortSmem = 1024;  // atoms per column sorted from shared memory
constexpr int kSortThreads = 128;
constexpr int kSortPer = kSortSmem / kSortThreads;  // atoms per thread (shared-memory path)

// Sort key of (z, atom index): z >= 0 after wrapping (+0.0f turns -0 into
// +0), so its IEEE bits order like the value; the index breaks ties.
__device__ __forceinline__ unsigned long long zkey(float z, int a)
{
    return ((unsigned long long)__float_as_uint(z + 0.0f) << 32) | (unsigned)a;
}

// rank[u] += number of the n shared keys smaller than key[u], u < U.
template <int U>
__device__ __forceinline__ void rank_keys(const unsigned long long *skey, int n, const unsigned long long *key,
                                          int *rank)
{
#pragma unroll 4
    for (int m = 0; m < n; ++m) {
        const unsigned long long km = skey[m];
#pragma unroll
        for (int u = 0; u < U; ++u) rank[u] += km < key[u];
    }
}

// A3b: one block per column: rank sort by (z, atom index), write the sorted
// slot arrays and padding, the cluster bounding boxes and the column's z-bin
// index (the clusters are z-sorted, so their z_lo and z_hi never decrease).
// Columns of up to kSortSmem atoms sort from shared memory: every thread
// holds up to kSortPer keys and counts, per broadcast key, how many are
// smaller.
__global__ void __launch_bounds__(kSortThreads) k_colsort(
    const int *__restrict__ col_count, const int *__restrict__ col_slot, const int *__restrict__ col_sys,
    const SysDesc *__restrict__ sys, const int *__restrict__ stage, const float4 *__restrict__ wpos,
    float4 *__restrict__ xyzq, int *__restrict__ tslot, int *__restrict__ perm, int *__restrict__ inv,
    float4 *__restrict__ bb, int *__restrict__ clus_sys, int2 *__restrict__ zbin)
{
    pdl_entry();
    __shared__ unsigned long long skey[kSortSmem];
    __shared__ float4 sp[kSortSmem];
    const int c = blockIdx.x;
    const int tid = threadIdx.x;
    const int n = col_count[c];
    const int base = col_slot[c];
    const int npad = (n + kCluster - 1) / kCluster * kCluster;
    const bool small = n <= kSortSmem;
    if (small) {
        const int nper = (n + kSortThreads - 1) / kSortThreads;
        unsigned long long key[kSortPer];
        float4 p[kSortPer];
        int rank[kSortPer];
#pragma unroll
        for (int u = 0; u < kSortPer; ++u) {
            const int k = tid + u * kSortThreads;
            key[u] = ~0ull;
            rank[u] = 0;
            if (k < n) {
                const int a = stage[base + k];
                p[u] = wpos[a];
                key[u] = zkey(p[u].z, a);
                skey[k] = key[u];
            }
        }
        __syncthreads();
        if (nper <= 1) rank_keys<1>(skey, n, key, rank);
        else if (nper <= 2) rank_keys<2>(skey, n, key, rank);
        else if (nper <= 4) rank_keys<4>(skey, n, key, rank);
        else rank_keys<kSortPer>(skey, n, key, rank);
#pragma unroll
        for (int u = 0; u < kSortPer; ++u) {
            const int k = tid + u * kSortThreads;
            if (k < n) {
                const int a = (int)(unsigned)(key[u] & 0xffffffffull);
                const int slot = base + rank[u];
                perm[slot] = a;
                inv[a] = slot;
                xyzq[slot] = make_float4(p[u].x, p[u].y, p[u].z, 0.0f);
                sp[rank[u]] = p[u];
            }
        }
    } else {
        for (int k = tid; k < n; k += blockDim.x) {
            const int a = stage[base + k];
            const float4 pa = wpos[a];
            const unsigned long long ka = zkey(pa.z, a);
            int rank = 0;
            for (int m = 0; m < n; ++m) {
                const int b = stage[base + m];
                rank += zkey(wpos[b].z, b) < ka;
            }
            const int slot = base + rank;
            perm[slot] = a;
            inv[a] = slot;
            xyzq[slot] = make_float4(pa.x, pa.y, pa.z, 0.0f);
        }
    }
    for (int k = n + tid; k < npad; k += blockDim.x) {
        perm[base + k] = -1;
        tslot[base + k] = 0;
        xyzq[base + k] = make_float4(kPadCoord, kPadCoord, kPadCoord, 0.0f);
    }
    __syncthreads();
    // cluster bounding boxes over the real atoms of each 8-slot cluster
    const int nclus = npad / kCluster;
    for (int q = tid; q < nclus; q += blockDim.x) {
        float lx = INFINITY, ly = INFINITY, lz = INFINITY, hx = -INFINITY, hy = -INFINITY, hz = -INFINITY;
        for (int k = q * kCluster; k < min(n, (q + 1) * kCluster); ++k) {
            const float4 p = small ? sp[k] : xyzq[base + k];
            lx = fminf(lx, p.x); ly = fminf(ly, p.y); lz = fminf(lz, p.z);
            hx = fmaxf(hx, p.x); hy = fmaxf(hy, p.y); hz = fmaxf(hz, p.z);
        }
        const int I = base / kCluster + q;
        bb[2 * I] = make_float4(lx, ly, lz, 0.0f);
        bb[2 * I + 1] = make_float4(hx, hy, hz, 0.0f);
        clus_sys[I] = col_sys[c];
    }
    __syncthreads();
    // z-bin index: for b = 0..nzb, (first cluster with z_hi >= b dz, first
    // cluster with z_lo > (b + 1) dz), by binary search over the column.  The
    // atoms are z-sorted: a cluster's z_lo is its first atom's z and its z_hi
    // its last real atom's z.
    const SysDesc &S = sys[col_sys[c]];
    const float4 *cb = bb + 2ll * (base / kCluster);
    int2 *zt = zbin + S.zb_begin + (long long)(c - S.col_begin) * (S.nzb + 1);
    for (int b = tid; b <= S.nzb; b += blockDim.x) {
        const float z0 = (float)b * S.dz, z1 = (float)(b + 1) * S.dz;
        int lo = 0, hi = nclus;  // first q with z_hi(q) >= z0
        while (lo < hi) {
            const int m = (lo + hi) >> 1;
            const float zh = small ? sp[min(n, (m + 1) * kCluster) - 1].z : cb[2 * m + 1].z;
            if (zh >= z0) hi = m;
            else lo = m + 1;
        }
        int lo2 = 0, hi2 = nclus;  // first q with z_lo(q) > z1
        while (lo2 < hi2) {
            const int m = (lo2 + hi2) >> 1;
            const float zl = small ? sp[m * kCluster].z : cb[2 * m].z;
            if (zl > z1) hi2 = m;
            else lo2 = m + 1;
        }
        zt[b] = make_int2(lo, lo2);
    }
}

// Opposite periodic image of a list entry's shift code: 1 <-> 2 on every axis.
__device__ __forceinline__ uint32_t opposite_code(uint32_t c) { return ((c & 0x15u) << 1) | ((c & 0x2Au) >> 1); }

// Half list for Newton's third law: of the two entries (I, J, c) and
// (J, I, opposite c) of one cluster pair exactly one is kept, chosen by a
// checkerboard on the indices so that every cluster keeps about half of its
// neighbours; of a cluster's own periodic images the smaller code of each
// opposite pair, and the direct self entry (whose pairs j > i the force kernel
// takes).
__device__ __forceinline__ bool keep_half(int I, int J, uint32_t code)
{
    if (J == I) return code == 0u || code < opposite_code(code);
    return ((I ^ J) & 1) ? (I < J) : (I > J);
}

// Candidate v of a column window (virtual index: image -L below 0, +L from
// nj): J when its bounding box comes within rc + margin of I's, else -1;
// code receives the entry's shift code.
__device__ __forceinline__ int window_candidate(const float4 *__restrict__ bb, float4 lo, float4 hi, int v, int jb,
                                                int nj, uint32_t code_xy, float ox, float oy, float Lz, float rcm2,
                                                uint32_t &code)
{
    const uint32_t zimg = v < 0 ? 1u : (v >= nj ? 2u : 0u);
    const int J = jb + v + (zimg == 1u ? nj : (zimg == 2u ? -nj : 0));
    const float oz = zimg == 1u ? -Lz : (zimg == 2u ? Lz : 0.0f);
    const float4 jl = bb[2 * J], jh = bb[2 * J + 1];
    const float gx = fmaxf(fmaxf((jl.x + ox) - hi.x, lo.x - (jh.x + ox)), 0.0f);
    const float gy = fmaxf(fmaxf((jl.y + oy) - hi.y, lo.y - (jh.y + oy)), 0.0f);
    const float gz = fmaxf(fmaxf((jl.z + oz) - hi.z, lo.z - (jh.z + oz)), 0.0f);
    code = code_xy | (zimg << 4);
    return gx * gx + gy * gy + gz * gz < rcm2 ? J : -1;
}

// Bit of a cluster index in the 64-bit partner-cluster filter (multiplicative
// hash of the index within the cluster's system, so that a system's lists
// and flags do not depend on the other systems of a batch).
__device__ __forceinline__ unsigned bloom_bit(int c) { return ((unsigned)c * 0x9E3779B1u) >> 26; }

constexpr int kListWarps = 8;   // warps (clusters in flight) per block of the list kernel
constexpr int kListGroup = 64;  // candidate columns compacted per pass
constexpr int kOwnCap = 512;    // flattened candidates whose owner lane is tabulated
constexpr int kPartnerRounds = (kCluster * kMaxPartners + 31) / 32;

// A4: cluster-pair lists, one warp per cluster I.  The columns within reach
// of I's bounding box (with periodic images) go to the lanes.  Clusters of a
// column are z-sorted, so the ones whose z-range (under the z images -L, 0,
// +L, concatenated as virtual indices -nj..2nj-1) comes within the cutoff of
// I form one window per column; the windows of all lanes are flattened and
// every candidate (J, image) is tested by bounding-box gap < rc + margin.
// Of the entries kept, those of I's half (Newton's third law: every cluster
// pair appears in the list of exactly one of its two clusters, see
// keep_half) are compacted in (column round, candidate round, lane) order,
// so the lists are deterministic.  Also writes the partner slots of I's atoms and flags the
// entries whose cluster may hold a topology partner of I (a Bloom filter of
// the partners' clusters: never a missed partner, rarely a spurious flag).
__global__ void __launch_bounds__(kListWarps * 32)
    k_list(const SysDesc *__restrict__ sys, const int *__restrict__ counts, const float4 *__restrict__ bb,
           const int *__restrict__ clus_sys, const int *__restrict__ col_slot, const int2 *__restrict__ zbin,
           const int *__restrict__ perm, const int *__restrict__ part_orig, const int *__restrict__ inv, int K,
           float rcm, int cap, uint32_t *__restrict__ list, int *__restrict__ list_n, int *__restrict__ pslot,
           int *__restrict__ status)
{
    pdl_entry();
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int n_clus = counts[1];
    const float rcm2 = rcm * rcm;
    __shared__ int s_col[kListWarps][kListGroup];  // compacted candidate columns per warp
    __shared__ unsigned char s_own[kListWarps][kOwnCap];  // owner lane of each flattened candidate
    const int wib = threadIdx.x >> 5;
    for (int I = gw; I < n_clus; I += nw) {
        const SysDesc &S = sys[clus_sys[I]];
        const float4 lo = bb[2 * I], hi = bb[2 * I + 1];
        // partner slots of I's atoms, and a 64-bit Bloom filter of the
        // clusters that hold them: an entry is flagged when its cluster's
        // bit is set (false positives only cost the force kernel a partner
        // check, a real partner is never missed)
        unsigned long long bloom = 0ull;
        const int np = kCluster * K;
        // the loads of all rounds first (three dependent levels, not three per round)
        int pv[kPartnerRounds];
#pragma unroll
        for (int r = 0; r < kPartnerRounds; ++r) {
            const int t = r * 32 + lane;
            pv[r] = t < np ? perm[I * kCluster + t / K] : -1;
        }
#pragma unroll
        for (int r = 0; r < kPartnerRounds; ++r) {
            const int t = r * 32 + lane;
            pv[r] = pv[r] >= 0 ? part_orig[(long long)pv[r] * K + t % K] : -1;
        }
#pragma unroll
        for (int r = 0; r < kPartnerRounds; ++r) {
            const int t = r * 32 + lane;
            pv[r] = pv[r] >= 0 ? (inv[pv[r] >> 1] << 1) | (pv[r] & 1) : -1;
            if (t < np) pslot[(long long)I * np + t] = pv[r];
        }
#pragma unroll
        for (int r = 0; r < kPartnerRounds; ++r)
            if (pv[r] >= 0) bloom |= 1ull << bloom_bit((pv[r] >> 1) / kCluster - S.clus_begin);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) bloom |= __shfl_xor_sync(FULL, bloom, o);
        const int cxa = max(-S.nx, (int)floorf((lo.x - rcm) * S.inv_w[0]));
        const int cxb = min(2 * S.nx - 1, (int)floorf((hi.x + rcm) * S.inv_w[0]));
        const int cya = max(-S.ny, (int)floorf((lo.y - rcm) * S.inv_w[1]));
        const int cyb = min(2 * S.ny - 1, (int)floorf((hi.y + rcm) * S.inv_w[1]));
        const float Lz = S.L[2];
        // conservative margin of the column-geometry test (binning rounds in FP32)
        const float cmarg = 1e-3f + 1e-6f * fmaxf(S.L[0], S.L[1]);
        const int ncx = cxb - cxa + 1, ncand = ncx * (cyb - cya + 1);
        int nA = 0;
        uint32_t *LA = list + (long long)I * cap;
        for (int g0 = 0; g0 < ncand; g0 += kListGroup) {
            // the candidate columns of this group whose geometry (a lower bound of
            // the xy gap) passes, compacted in order
            int npass = 0;
            for (int h = 0; h < kListGroup; h += 32) {
                const int c = g0 + h + lane;
                bool pass = false;
                if (c < ncand) {
                    const int cy = cya + c / ncx, cx = cxa + c % ncx;
                    const float gcx = fmaxf(fmaxf(cx * S.w[0] - hi.x, lo.x - (cx + 1) * S.w[0]) - cmarg, 0.0f);
                    const float gcy = fmaxf(fmaxf(cy * S.w[1] - hi.y, lo.y - (cy + 1) * S.w[1]) - cmarg, 0.0f);
                    pass = gcx * gcx + gcy * gcy < rcm2;
                }
                const unsigned b = __ballot_sync(FULL, pass);
                if (pass) s_col[wib][npass + __popc(b & lt)] = c;
                npass += __popc(b);
            }
            __syncwarp();
            for (int r0 = 0; r0 < npass; r0 += 32) {
                const int c = r0 + lane < npass ? s_col[wib][r0 + lane] : -1;
                int jb = 0, nj = 0, va = 0, cnt = 0;
                uint32_t code_xy = 0u;
                float ox = 0.0f, oy = 0.0f;
                if (c >= 0) {
                    const int cy = cya + c / ncx, cx = cxa + c % ncx;
                    const int ccy = cy < 0 ? cy + S.ny : (cy >= S.ny ? cy - S.ny : cy);
                    const int ccx = cx < 0 ? cx + S.nx : (cx >= S.nx ? cx - S.nx : cx);
                    const uint32_t sy = cy < 0 ? 1u : (cy >= S.ny ? 2u : 0u);
                    const uint32_t sx = cx < 0 ? 1u : (cx >= S.nx ? 2u : 0u);
                    ox = sx == 1u ? -S.L[0] : (sx == 2u ? S.L[0] : 0.0f);
                    oy = sy == 1u ? -S.L[1] : (sy == 2u ? S.L[1] : 0.0f);
                    code_xy = sx | (sy << 2);
                    const int col = S.col_begin + ccy * S.nx + ccx;
                    jb = col_slot[col] / kCluster;
                    nj = col_slot[col + 1] / kCluster - jb;
                    // z window over the virtual indices v (image -L: v - nj, 0: v, +L: v + nj)
                    // from the column's z-bin index, one bin wider on each side
                    // than the FP32 bin arithmetic needs
                    const int2 *zt = zbin + S.zb_begin + (long long)(col - S.col_begin) * (S.nzb + 1);
                    const float za = lo.z - rcm, zb = hi.z + rcm;
                    const int ba = (int)floorf((za < 0.0f ? za + Lz : za) * S.inv_dz) - 1;
                    const int bz = (int)floorf((zb >= Lz ? zb - Lz : zb) * S.inv_dz) + 1;
                    const int vlo = zt[min(max(ba, 0), S.nzb)].x - (za < 0.0f ? nj : 0);
                    const int vhi = zt[min(max(bz, 0), S.nzb)].y + (zb >= Lz ? nj : 0);  // one past
                    if (vhi > vlo) {
                        va = vlo;
                        cnt = vhi - vlo;
                    }
                }
                // flatten the windows of the 32 lanes
                int incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(FULL, incl, o);
                    if (lane >= o) incl += y;
                }
                const int off = incl - cnt, total = __shfl_sync(FULL, incl, 31);
                // owner lane of each flattened candidate, for the first kOwnCap
                for (int t = off; t < min(off + cnt, kOwnCap); ++t) s_own[wib][t] = (unsigned char)lane;
                __syncwarp();
                // two candidate rounds at a time: both rounds' box loads are in
                // flight together; entries are appended in round order
                for (int p0 = 0; p0 < total; p0 += 64) {
                    int J[2];
                    uint32_t code[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int p = p0 + 32 * h + lane;
                        // owner lane: the last lane whose window starts at or before p
                        int src = 0;
                        if (p0 + 32 * h + 31 < kOwnCap) {
                            src = p < total ? s_own[wib][p] : 0;
                        } else {
#pragma unroll
                            for (int step = 16; step >= 1; step >>= 1) {
                                const int o2 = __shfl_sync(FULL, off, src + step);
                                if (o2 <= p) src += step;
                            }
                        }
                        const int s_off = __shfl_sync(FULL, off, src), s_va = __shfl_sync(FULL, va, src);
                        const int s_jb = __shfl_sync(FULL, jb, src), s_nj = __shfl_sync(FULL, nj, src);
                        const uint32_t s_code = __shfl_sync(FULL, code_xy, src);
                        const float s_ox = __shfl_sync(FULL, ox, src), s_oy = __shfl_sync(FULL, oy, src);
                        J[h] = -1;
                        code[h] = 0u;
                        if (p < total)
                            J[h] = window_candidate(bb, lo, hi, s_va + (p - s_off), s_jb, s_nj, s_code, s_ox, s_oy, Lz,
                                                    rcm2, code[h]);
                    }
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const bool fl = J[h] >= 0 && ((bloom >> bloom_bit(J[h] - S.clus_begin)) & 1ull);
                        const uint32_t ent = (uint32_t)J[h] | (code[h] << kShiftBit) | (fl ? kExclFlag : 0u);
                        const bool hit = J[h] >= 0 && keep_half(I, J[h], code[h]);
                        const unsigned b = __ballot_sync(FULL, hit);
                        if (hit) {
                            const int q = nA + __popc(b & lt);
                            if (q < cap) LA[q] = ent;
                        }
                        nA += __popc(b);
                    }
                }
                __syncwarp();  // the owner table is rewritten by the next round
            }
            __syncwarp();
        }
        if (lane == 0) {
            list_n[I] = min(nA, cap);
            if (nA > cap) atomicOr(status, ST_CAPACITY);
        }
    }
}

cudaError_t launch_build_cells(nb_ctx *ctx, const float *d_pos)
{
    auto &d = ctx->d;
    cudaStream_t st = ctx->stream;
    const int N = (int)ctx->n_atoms;
    cudaError_t e = cudaMemsetAsync(d.col_count, 0, sizeof(int) * (ctx->n_cols + 1), st);
    if (e != cudaSuccess) return e;
    const int tb = 256;
    e = launch_pdl(k_bin, dim3((N + tb - 1) / tb), dim3(tb), 0, st, N, d_pos, d.sys, d.atom_sys, d.wpos, d.atom_col,
                   d.col_count, ctx->n_cols, ctx->n_sys, d.col_slot, d.col_fill, d.counts, d.status);
    if (e == cudaSuccess)
        e = launch_pdl(k_scatter, dim3((N + tb - 1) / tb), dim3(tb), 0, st, N, d.atom_col, d.col_fill, d.stage);
    if (e == cudaSuccess)
        e = launch_pdl(k_colsort, dim3(ctx->n_cols), dim3(kSortThreads), 0, st, d.col_count, d.col_slot, d.col_sys,
                       d.sys, d.stage, d.wpos, d.xyzq, d.tslot, d.perm, d.inv, d.bb, d.clus_sys, d.zbin);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_build_lists(nb_ctx *ctx)
{
    auto &d = ctx->d;
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaSuccess;
    const int lw = kListWarps;
    const int lblocks = (int)std::max<int64_t>(1, (ctx->clus_cap + lw - 1) / lw);
    if (e == cudaSuccess)
        e = launch_pdl(k_list, dim3(lblocks), dim3(lw * 32), 0, st, d.sys, d.counts, d.bb, d.clus_sys, d.col_slot,
                       d.zbin, d.perm, d.part_orig, d.inv, ctx->K, ctx->pp.rc + ctx->pp.list_margin, ctx->list_cap,
                       d.list, d.list_n, d.pslot, d.status);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_build(nb_ctx *ctx, const float *d_pos)
{
    const cudaError_t e = launch_build_cells(ctx, d_pos);
    return e != cudaSuccess ? e : launch_build_lists(ctx);
}

}  // namespace acenb
