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
// the column slot offsets, the totals and the per-system slot/cluster
// ranges; then the first i-group of every column (ceil(clusters / group)
// groups per column), copying each column's count behind the histogram for
// the column sort and zeroing the histogram for the next build.
__device__ void scan_columns(int n_cols, int n_sys, int *__restrict__ col_count, int *__restrict__ col_slot,
                             SysDesc *__restrict__ sys, int *__restrict__ counts, int group,
                             int *__restrict__ col_grp)
{
    __shared__ int warp_sum[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int pass = 0; pass < 2; ++pass) {
    for (int base = 0; base < n_cols; base += blockDim.x) {
        int c = base + threadIdx.x;
        const int cnt = c < n_cols ? __ldcg(&col_count[c]) : 0;
        const int ncl = (cnt + kCluster - 1) / kCluster;
        if (pass == 1 && c < n_cols) {  // the count for the column sort; the histogram is zero again
            col_count[n_cols + 1 + c] = cnt;
            col_count[c] = 0;
        }
        int v = pass == 0 ? ncl * kCluster : (ncl + group - 1) / group;
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
        if (c < n_cols) {
            if (pass == 0) {
                col_slot[c] = excl;
            } else {
                col_grp[c] = excl;
            }
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (pass == 0) {
            col_slot[n_cols] = carry;
            counts[0] = carry;
            counts[1] = carry / kCluster;
        } else {
            col_grp[n_cols] = carry;
            counts[4] = carry;  // groups
            counts[5] = 0;      // exclusion-mask pool records used by the list kernel
        }
        carry = 0;
    }
    __syncthreads();
    }
    for (int s = threadIdx.x; s < n_sys; s += blockDim.x) {
        int c0 = sys[s].col_begin, c1 = c0 + sys[s].nx * sys[s].ny;
        sys[s].slot_begin = col_slot[c0];
        sys[s].clus_begin = col_slot[c0] / kCluster;
        sys[s].clus_end = col_slot[c1] / kCluster;
    }
}

// The step's charges and types when they are in host memory, read by the
// binning kernel beside the positions (coalesced, in caller order, across
// the host link): the charge goes to the wrapped position's w, the
// range-checked type to atom_t, and the column sort carries both into sorted
// order.  q = null: positions only (w = 0); device-resident charges and
// types are gathered by the column sort instead (faster there).
struct AtomPack {
    const float *q;
    const int *type;
    int T;
    int *atom_t;  // [N] checked types in caller order
};

// A1 + A2 + A3a: one atom per thread: wrap, column index, column histogram
// (warp-aggregated atomics, whose returned counts are the atoms' places in
// their column): each atom goes to its place in its column's fixed-capacity
// staging row (stage_fix[col * col_cap + place]; a place at or beyond
// col_cap is left to the column sort's fallback).  The last block to finish
// scans the histogram.  col_count[n_cols] is the completion ticket (zero on
// entry, reset on exit).
__global__ void k_bin(int n, const float *__restrict__ pos, SysDesc *__restrict__ sys,
                      const int *__restrict__ atom_sys, float4 *__restrict__ wpos, int *__restrict__ atom_col,
                      int *__restrict__ col_count, int n_cols, int n_sys, int *__restrict__ col_slot,
                      int *__restrict__ stage_fix, int col_cap, int *__restrict__ counts, int *__restrict__ status,
                      int group, int *__restrict__ col_grp, AtomPack ap)
{
    pdl_entry();
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    int col = -1;
    if (a < n) {
        const SysDesc &S = sys[n_sys == 1 ? 0 : atom_sys[a]];  // one system: no dependent load
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
        float qa = 0.0f;
        if (ap.q) {  // charge and checked type, read beside the position
            qa = ap.q[a];
            int t = ap.type[a];
            if (t < 0 || t >= ap.T) {
                atomicOr(status, ST_BADTYPE);
                t = 0;
            }
            ap.atom_t[a] = t;
        }
        wpos[a] = make_float4(x, y, z, qa);
    }
    const int place = warp_aggregated_add(col_count, col);
    if (col >= 0 && place < col_cap) stage_fix[(long long)col * col_cap + place] = a;
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
    scan_columns(n_cols, n_sys, col_count, col_slot, sys, counts, group, col_grp);
    if (threadIdx.x == 0) col_count[n_cols] = 0;
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

// Sort the P (a power of two) shared keys ascending by a bitonic network:
// log2(P) (log2(P) + 1) / 2 compare-exchange stages of P / 2 pairs each.
__device__ void bitonic_sort(unsigned long long *skey, int P)
{
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < (P >> 1); i += blockDim.x) {
                const int l = 2 * i - (i & (j - 1)), r = l + j;  // the pair (l, l + j), l with bit j clear
                const unsigned long long a = skey[l], b = skey[r];
                if ((a > b) == ((l & k) == 0)) {
                    skey[l] = b;
                    skey[r] = a;
                }
            }
            __syncthreads();
        }
    }
}

constexpr int kRankSortMax = 256;  // columns up to this many atoms are rank-sorted (no barriers)

// Per-atom inputs of the force kernels packed by the column sort when the
// caller passes them with the positions (nb_step): charges into xyzq.w,
// checked types into tslot, and the force kernels' sums and work counter
// zeroed (k_pack's work, without its stale-position check: the positions
// were just binned).  q == nullptr: the column sort leaves that to k_pack.
struct ColPack {
    const float *q;      // kPackGather: charges and types in caller order, gathered here
    const int *type;
    int T;
    const int *atom_t;   // kPackAtomT: checked types from the binning kernel, charges in wpos.w
    long long *facc;     // [3 slots] fixed-point forces
    long long *sys_acc;  // [n_acc] per-system energy and virial sums
    int n_acc;
    int *work;           // the force kernels' work-unit counter
    int *status;
};

// What the column sort packs (a template parameter: no per-atom branches).
enum PackMode { kPackNone = 0, kPackGather = 1, kPackAtomT = 2 };

__device__ __forceinline__ int checked_type(const ColPack &pk, int t)
{
    if (t < 0 || t >= pk.T) {
        atomicOr(pk.status, ST_BADTYPE);
        t = 0;
    }
    return t;
}

// Charge (into p.w) and type of atom a for the sorted arrays, as loaded: a
// type from the caller's array is range-checked by sorted_type when it is
// written (so that no load is waited for before the sort).
template <int PACK>
__device__ __forceinline__ int pack_atom(const ColPack &pk, int a, float4 &p)
{
    if (PACK == kPackAtomT) return pk.atom_t[a];  // p.w holds the charge already
    if (PACK == kPackNone) return 0;
    p.w = pk.q[a];
    return pk.type[a];
}

template <int PACK>
__device__ __forceinline__ int sorted_type(const ColPack &pk, int t)
{
    return PACK == kPackAtomT ? t : checked_type(pk, t);
}

// A3b: one block per column: sort by (z, atom index), write the sorted slot
// arrays and padding, the cluster bounding boxes and the column's z-bin
// index (the clusters are z-sorted, so their z_lo and z_hi never decrease).
// Columns of up to kSortSmem atoms sort from shared memory: up to
// kRankSortMax atoms by rank (every thread holds up to kSortPer keys and
// counts, per broadcast key, how many are smaller: n^2 compares), longer
// ones by a bitonic network (n log^2 n).  The keys are unique, so both give
// the same order.  PACK selects how the step's charges and types are packed
// (a template parameter: no per-atom branches); the register budget of 6
// blocks per SM (80 registers) measured faster than the compiler's choice
// (94 for the gathering instance) in both the step and the MD step.
template <int PACK>
__global__ void __launch_bounds__(kSortThreads, 6) k_colsort(
    const int *__restrict__ col_count, const int *__restrict__ col_slot, const int *__restrict__ col_sys,
    const SysDesc *__restrict__ sys, const int *__restrict__ stage_fix, int col_cap, int *__restrict__ stage,
    const int *__restrict__ atom_col, const float4 *__restrict__ wpos,
    float4 *__restrict__ xyzq, int *__restrict__ tslot, int *__restrict__ perm, int *__restrict__ inv,
    float4 *__restrict__ bb, int *__restrict__ clus_sys, int2 *__restrict__ zbin, int group,
    const int *__restrict__ col_grp, int2 *__restrict__ grp, int *__restrict__ clus_grp, ColPack pk)
{
    pdl_entry();
    __shared__ unsigned long long skey[kSortSmem];
    __shared__ float4 sp[kSortSmem];
    const int c = blockIdx.x;
    const int tid = threadIdx.x;
    const int n = col_count[c];
    const int base = col_slot[c];
    const int npad = (n + kCluster - 1) / kCluster * kCluster;
    // the column's atoms: its staging row, or, when the column outgrew the
    // row's capacity (strongly uneven density), gathered here from the
    // system's atoms into the column's own slots (slow, rare)
    const int *src = stage_fix + (long long)c * col_cap;
    if (n > col_cap) {
        __shared__ int s_fill;
        if (tid == 0) s_fill = 0;
        __syncthreads();
        const SysDesc &S0 = sys[col_sys[c]];
        for (int a = S0.atom_begin + tid; a < S0.atom_begin + S0.n_atoms; a += blockDim.x)
            if (atom_col[a] == c) stage[base + atomicAdd(&s_fill, 1)] = a;
        __syncthreads();
        src = stage + base;
    }
    const bool small = n <= kSortSmem;
    if (small && n > kRankSortMax) {
        int P = 1;
        while (P < n) P <<= 1;
        for (int k = tid; k < P; k += blockDim.x) {
            unsigned long long key = ~0ull;  // padding sorts last
            if (k < n) {
                const int a = src[k];
                key = zkey(wpos[a].z, a);
            }
            skey[k] = key;
        }
        __syncthreads();
        bitonic_sort(skey, P);
        for (int k = tid; k < n; k += blockDim.x) {
            const int a = (int)(unsigned)(skey[k] & 0xffffffffull);
            float4 pa = wpos[a];
            const int slot = base + k;
            perm[slot] = a;
            inv[a] = slot;
            const int t = pack_atom<PACK>(pk, a, pa);
            xyzq[slot] = pa;  // w: the charge (0 without packing)
            if (PACK != kPackNone) tslot[slot] = sorted_type<PACK>(pk, t);
            sp[k] = pa;
        }
    } else if (small) {
        const int nper = (n + kSortThreads - 1) / kSortThreads;
        unsigned long long key[kSortPer];
        float4 p[kSortPer];  // w: the charge (0 without packing)
        int typ[kSortPer];
        int rank[kSortPer];
#pragma unroll
        for (int u = 0; u < kSortPer; ++u) {
            const int k = tid + u * kSortThreads;
            key[u] = ~0ull;
            rank[u] = 0;
            typ[u] = 0;
            if (k < n) {
                const int a = src[k];
                p[u] = wpos[a];
                typ[u] = pack_atom<PACK>(pk, a, p[u]);  // loaded now, written after the sort
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
                xyzq[slot] = p[u];
                if (PACK != kPackNone) tslot[slot] = sorted_type<PACK>(pk, typ[u]);
                sp[rank[u]] = p[u];
            }
        }
    } else {
        for (int k = tid; k < n; k += blockDim.x) {
            const int a = src[k];
            float4 pa = wpos[a];
            const unsigned long long ka = zkey(pa.z, a);
            int rank = 0;
            for (int m = 0; m < n; ++m) {
                const int b = src[m];
                rank += zkey(wpos[b].z, b) < ka;
            }
            const int slot = base + rank;
            perm[slot] = a;
            inv[a] = slot;
            const int t = pack_atom<PACK>(pk, a, pa);
            xyzq[slot] = pa;
            if (PACK != kPackNone) tslot[slot] = sorted_type<PACK>(pk, t);
        }
    }
    for (int k = n + tid; k < npad; k += blockDim.x) {
        perm[base + k] = -1;
        tslot[base + k] = 0;
        xyzq[base + k] = make_float4(kPadCoord, kPadCoord, kPadCoord, 0.0f);
    }
    if (PACK != kPackNone) {
        for (int k = tid; k < 3 * npad; k += blockDim.x) pk.facc[3ll * base + k] = 0;
        if (c == 0) {
            for (int k = tid; k < pk.n_acc; k += blockDim.x) pk.sys_acc[k] = 0;
            if (tid == 0) *pk.work = 0;
        }
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
        // i-groups: runs of `group` consecutive clusters of the column
        const int gi = col_grp[c] + q / group;
        clus_grp[I] = gi;
        if (q % group == 0) grp[gi] = make_int2(I, min(group, nclus - q));
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

// Newton's third law at group level.  Every pair of clusters (I, J) of two
// different i-groups is listed by exactly one of the two groups, chosen by a
// checkerboard on the group indices (so that every group lists about half of
// its neighbours): all tiles between two groups sit in one group's list.
// The parity and the order of two indices do not change when both are
// offset by the same amount, so a system's lists are the same in a batch as
// alone.
__device__ __forceinline__ bool keep_groups(int gA, int gB) { return ((gA ^ gB) & 1) ? (gA < gB) : (gA > gB); }

// Within one group, of the tiles (I, J, c) and (J, I, opposite c) the one
// with I < J; for I == J the direct tile (whose pairs j > i are taken) and
// of a cluster's own periodic images the smaller code of each opposite pair.
__device__ __forceinline__ bool keep_in_group(int I, int J, uint32_t code)
{
    if (I != J) return I < J;
    return code == 0u || code < opposite_code(code);
}

// Candidate v of a column window (virtual index: image -L below 0, +L from
// nj): J, its shift code and its bounding box at that image.
__device__ __forceinline__ int window_cluster(const float4 *__restrict__ bb, int v, int jb, int nj, uint32_t code_xy,
                                              float ox, float oy, float Lz, uint32_t &code, float4 &jl, float4 &jh)
{
    const uint32_t zimg = v < 0 ? 1u : (v >= nj ? 2u : 0u);
    const int J = jb + v + (zimg == 1u ? nj : (zimg == 2u ? -nj : 0));
    const float oz = zimg == 1u ? -Lz : (zimg == 2u ? Lz : 0.0f);
    jl = bb[2 * J];
    jh = bb[2 * J + 1];
    jl.x += ox; jh.x += ox;
    jl.y += oy; jh.y += oy;
    jl.z += oz; jh.z += oz;
    code = code_xy | (zimg << 4);
    return J;
}

// Squared gap between two boxes (0 when they overlap).
__device__ __forceinline__ float box_gap2(float4 al, float4 ah, float4 bl, float4 bh)
{
    const float gx = fmaxf(fmaxf(bl.x - ah.x, al.x - bh.x), 0.0f);
    const float gy = fmaxf(fmaxf(bl.y - ah.y, al.y - bh.y), 0.0f);
    const float gz = fmaxf(fmaxf(bl.z - ah.z, al.z - bh.z), 0.0f);
    return gx * gx + gy * gy + gz * gz;
}

// The block's set of clusters that hold a topology partner of a group atom:
// open addressing in shared memory, bounded probing; insert returns the
// key's slot (-1 when the table is full: the caller then flags every entry),
// find returns it or -1.
constexpr int kHashSlots = 256;
__device__ __forceinline__ unsigned hset_slot(int key) { return ((unsigned)key * 0x9E3779B1u) >> 24; }

__device__ __forceinline__ int hset_insert(int *h, int key)
{
    unsigned s = hset_slot(key);
    for (int probe = 0; probe < kHashSlots; ++probe) {
        const int old = atomicCAS(&h[s], -1, key);
        if (old == -1 || old == key) return (int)s;
        s = (s + 1) & (kHashSlots - 1);
    }
    return -1;
}

__device__ __forceinline__ int hset_find(const int *h, int key)
{
    unsigned s = hset_slot(key);
    for (int probe = 0; probe < kHashSlots; ++probe) {
        const int v = h[s];
        if (v == key) return (int)s;
        if (v == -1) return -1;
        s = (s + 1) & (kHashSlots - 1);
    }
    return -1;
}

constexpr int kOwnCap = 512;    // flattened candidates whose owner lane is tabulated

// Bits jj <= ia of an 8 x 8 tile (bit 8 ia + jj): the pairs of the direct
// self tile that are not evaluated (each unique pair once, j > i).
constexpr unsigned long long kSelfTriangle = 0xFF7F3F1F0F070301ull;

// Exclusion bitmasks of one flagged entry (section "Molecular dynamics on
// the GPU": bitmaps select the non-bonded terms to exclude or scale), by one
// lane into record rec: for every group cluster c in cm, bit 8 ia + jj of
// (excluded, scaled 1-4) for i atom ia of cluster c0 + c and j atom jj of J;
// the direct self tile (J = c0 + c, no shift) also excludes jj <= ia.  The
// partners of the group's atoms that lie in J are the chain of J's slot in
// the warp's partner-cluster table: s_pslot[t] is a partner slot
// ((slot << 1) | is14) and s_link[t] packs the next entry of the chain
// (kLinkEnd at its end) with the group atom the partner belongs to (<< 16).
constexpr int kLinkEnd = 0xFFFF;

__device__ void entry_masks(const int *__restrict__ s_pslot, const int *__restrict__ s_link, int head, int c0,
                            unsigned cm, int J, uint32_t code, ulonglong2 *__restrict__ rec)
{
    // per cluster of the mask: walk J's chain, keep that cluster's bits in
    // registers, one store (the chains are a few partners long)
    for (unsigned cc = cm; cc; cc &= cc - 1u) {
        const int c = __ffs(cc) - 1;
        unsigned long long ex = 0ull, s14 = 0ull;
        for (int t = head, guard = 0; t != kLinkEnd && guard < kCluster * kMaxGroup * kMaxPartners; ++guard) {
            const int lk = s_link[t];
            const int a = lk >> 16;
            if (a / kCluster == c) {
                const int v = s_pslot[t];
                const unsigned long long bit = 1ull << ((a % kCluster) * kCluster + ((v >> 1) & (kCluster - 1)));
                if (v & 1) s14 |= bit;
                else ex |= bit;
            }
            t = lk & kLinkEnd;
        }
        if (code == 0u && J == c0 + c) ex |= kSelfTriangle;
        rec[c] = make_ulonglong2(ex, s14);
    }
}

// q = a / b and r = a % b for 0 <= a < 2^20, b >= 1: a rounded FP32 quotient
// estimate (within 1/4 of the true one there) and one correction each way.
__device__ __forceinline__ int div_small(int a, int b, float inv_b, int &r)
{
    int q = __float2int_rz(((float)a + 0.5f) * inv_b);
    r = a - q * b;
    if (r < 0) {
        --q;
        r += b;
    } else if (r >= b) {
        ++q;
        r -= b;
    }
    return q;
}

// A4: i-group lists, one warp per group of up to 8 consecutive clusters of a
// column (clusters c0 .. c0 + n - 1), kGListWarps groups per block.  The
// columns within reach of the group's bounding box (with periodic images)
// are scanned in order.  Clusters of a column are
// z-sorted, so the ones whose z-range (under the z images -L, 0, +L,
// concatenated as virtual indices -nj..2nj-1) comes within the cutoff of the
// group form one window per column; the windows of 32 columns are flattened
// and every candidate (J, image) gets the mask of the group clusters whose
// boxes come within rc + margin of J's and whose tile the group keeps
// (keep_groups, keep_in_group); a non-empty mask makes an entry.  Two rounds
// of 32 candidates are in flight at a time (their box loads overlap).  The
// entries are dealt round-robin, in scan order, to the kListSegs segments of
// the group's list (entry r to segment r % kListSegs, position r / kListSegs),
// so the segments are equally long and the lists deterministic.
// Entries whose J holds a topology partner of a group atom (found in the
// warp's partner-cluster table), or that contain the direct self tile, are
// flagged and get a record of exclusion bitmasks (entry_masks): the group's
// own records first (kMaskRecsPerCluster per cluster, taken in scan order
// without atomics), then the shared pool.
struct GListArgs {
    const SysDesc *sys;
    const int *counts;
    int *pool_count;         // pool records used (counts[5], zeroed by the binning kernel)
    const float4 *bb;
    const int *clus_sys;
    const int *col_slot;
    const int2 *zbin;
    const int *perm;
    const int *part_orig;
    const int *inv;
    const int2 *grp;
    const int *clus_grp;
    uint2 *glist;
    int *glist_n;
    ulonglong2 *gmask;
    int *status;
    long long pool_base;     // first pool record (after every group's own records)
    long long mask_cap;
    int K;
    float rcm;
    int cap;                 // entries per group (all segments)
    int group;               // clusters per group of the lists being built (records hold `group` mask pairs)
};

constexpr int kGListWarps = 4;  // groups (warps) per block of the list kernel
#ifndef ACENB_GLIST_MIN_BLOCKS
#define ACENB_GLIST_MIN_BLOCKS 7  // resident blocks per SM the register budget allows (72 registers)
#endif
constexpr int kPartnerBatch = 4;  // rounds of partner loads in flight

__host__ __device__ inline size_t glist_warp_ints(int K, int group) { return 2 * (size_t)kCluster * group * K; }

__global__ void __launch_bounds__(kGListWarps * 32, ACENB_GLIST_MIN_BLOCKS) k_glist(GListArgs A)
{
    const unsigned FULL = 0xffffffffu;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x * kGListWarps + w;
    __shared__ int s_hash_all[kGListWarps][kHashSlots];
    __shared__ int s_head_all[kGListWarps][kHashSlots];
    for (int t = lane; t < kHashSlots; t += 32) {  // cleared before the wait: no input needed
        s_hash_all[w][t] = -1;
        s_head_all[w][t] = kLinkEnd;
    }
    pdl_entry();
    if (g >= A.counts[4]) return;  // the whole warp
    const unsigned lt = (1u << lane) - 1u;
    // one-cluster groups are numbered like their clusters (the scans of
    // cluster and group counts per column coincide): no load
    const int2 gr = A.group == 1 ? make_int2(g, 1) : A.grp[g];
    const int c0 = gr.x, n = gr.y, K = A.K;
    __shared__ float4 s_lo_all[kGListWarps][kMaxGroup], s_hi_all[kGListWarps][kMaxGroup];
    __shared__ int s_col_all[kGListWarps][32];
    __shared__ int4 s_ci_all[kGListWarps][32];    // per window: jb, nj, first virtual index - offset, code
    __shared__ float2 s_co_all[kGListWarps][32];  // per window: x, y image shift
    __shared__ unsigned char s_own_all[kGListWarps][kOwnCap];
    extern __shared__ int s_dyn[];
    float4 *s_lo = s_lo_all[w], *s_hi = s_hi_all[w];
    int *s_hash = s_hash_all[w], *s_head = s_head_all[w], *s_col = s_col_all[w];
    int4 *s_ci = s_ci_all[w];
    float2 *s_co = s_co_all[w];
    unsigned char *s_own = s_own_all[w];
    int *s_pslot = s_dyn + (size_t)w * glist_warp_ints(K, A.group);  // [8 n K] partner slots (slot << 1) | is14
    int *s_link = s_pslot + kCluster * A.group * K;                   // [8 n K] chains of the partner-cluster table
    if (lane < n) {
        s_lo[lane] = A.bb[2 * (c0 + lane)];
        s_hi[lane] = A.bb[2 * (c0 + lane) + 1];
    }
    __syncwarp();
    const int np = kCluster * n * K;
    const float inv_K = 1.0f / (float)K;
    bool full = false;
    // groups of one cluster (8 K <= 128 partner entries, one batch): every
    // lane keeps its entries (partner cluster << 7 | is14 << 6 | bit 8 a + jj)
    // for the warp-cooperative masks
    int pk[kPartnerBatch] = {-1, -1, -1, -1};  // the partner table overflowed: flag every entry
    for (int t0 = 0; t0 < np; t0 += kPartnerBatch * 32) {
        // the three dependent loads of kPartnerBatch rounds at a time
        int pv[kPartnerBatch];
#pragma unroll
        for (int r = 0; r < kPartnerBatch; ++r) {
            const int t = t0 + r * 32 + lane;
            int rr;
            pv[r] = t < np ? A.perm[c0 * kCluster + div_small(t, K, inv_K, rr)] : -1;
        }
#pragma unroll
        for (int r = 0; r < kPartnerBatch; ++r) {
            const int t = t0 + r * 32 + lane;
            int rr;
            const int a = div_small(t, K, inv_K, rr);
            pv[r] = pv[r] >= 0 ? A.part_orig[(long long)pv[r] * K + rr] : -1;
            (void)a;
        }
#pragma unroll
        for (int r = 0; r < kPartnerBatch; ++r) pv[r] = pv[r] >= 0 ? (A.inv[pv[r] >> 1] << 1) | (pv[r] & 1) : -1;
#pragma unroll
        for (int r = 0; r < kPartnerBatch; ++r) {
            const int t = t0 + r * 32 + lane;
            if (t >= np) continue;
            s_pslot[t] = pv[r];
            if (pv[r] >= 0) {
                const int hs = hset_insert(s_hash, (pv[r] >> 1) / kCluster);
                int rr;
                const int a = div_small(t, K, inv_K, rr);  // group atom of entry t
                if (hs < 0) full = true;
                else s_link[t] = (atomicExch(&s_head[hs], t) & kLinkEnd) | (a << 16);
                if (t0 == 0 && A.group == 1)
                    pk[r] = (((pv[r] >> 1) / kCluster) << 7) | ((pv[r] & 1) << 6) | (a * kCluster + ((pv[r] >> 1) & 7));
            }
        }
    }
    const bool all_flag = __any_sync(FULL, full);
    __syncwarp();
    const SysDesc &S = A.sys[A.clus_sys[c0]];
    float4 lo = s_lo[0], hi = s_hi[0];
    for (int c = 1; c < n; ++c) {
        const float4 a = s_lo[c], b = s_hi[c];
        lo.x = fminf(lo.x, a.x); lo.y = fminf(lo.y, a.y); lo.z = fminf(lo.z, a.z);
        hi.x = fmaxf(hi.x, b.x); hi.y = fmaxf(hi.y, b.y); hi.z = fmaxf(hi.z, b.z);
    }
    const float rcm = A.rcm, rcm2 = rcm * rcm;
    const int cxa = max(-S.nx, (int)floorf((lo.x - rcm) * S.inv_w[0]));
    const int cxb = min(2 * S.nx - 1, (int)floorf((hi.x + rcm) * S.inv_w[0]));
    const int cya = max(-S.ny, (int)floorf((lo.y - rcm) * S.inv_w[1]));
    const int cyb = min(2 * S.ny - 1, (int)floorf((hi.y + rcm) * S.inv_w[1]));
    const float Lz = S.L[2];
    // conservative margin of the column-geometry test (binning rounds in FP32)
    const float cmarg = 1e-3f + 1e-6f * fmaxf(S.L[0], S.L[1]);
    const int ncx = cxb - cxa + 1, ncand = ncx * (cyb - cya + 1);
    const int seg_cap = A.cap / kListSegs;
    uint2 *LA = A.glist + (long long)g * A.cap;
    int ntot = 0;  // entries so far (entry r goes to segment r % kListSegs)
    const long long loc_base = (long long)c0 * kMaskRecsPerCluster;  // the group's own mask records
    const int loc_cap = n * kMaskRecsPerCluster;
    int nloc = 0;
    const float inv_ncx = 1.0f / (float)ncx;
    for (int c_lo = 0; c_lo < ncand; c_lo += 32) {
        // the candidate columns of this round whose geometry (a lower bound
        // of the xy gap) passes, compacted in order
        const int cc = c_lo + lane;
        bool pass = false;
        int ccx = 0, ccy = 0;
        if (cc < ncand) {
            ccy = div_small(cc, ncx, inv_ncx, ccx);
            const int cy = cya + ccy, cx = cxa + ccx;
            const float gcx = fmaxf(fmaxf(cx * S.w[0] - hi.x, lo.x - (cx + 1) * S.w[0]) - cmarg, 0.0f);
            const float gcy = fmaxf(fmaxf(cy * S.w[1] - hi.y, lo.y - (cy + 1) * S.w[1]) - cmarg, 0.0f);
            pass = gcx * gcx + gcy * gcy < rcm2;
        }
        const unsigned b = __ballot_sync(FULL, pass);
        if (pass) s_col[__popc(b & lt)] = ccx | (ccy << 16);
        const int npass = __popc(b);
        __syncwarp();
        if (npass == 0) continue;
        const int c = lane < npass ? s_col[lane] : -1;
        int jb = 0, nj = 0, va = 0, cnt = 0;
        uint32_t code_xy = 0u;
        float ox = 0.0f, oy = 0.0f;
        if (c >= 0) {
            const int cy = cya + (c >> 16), cx = cxa + (c & 0xFFFF);
            const int ky = cy < 0 ? cy + S.ny : (cy >= S.ny ? cy - S.ny : cy);
            const int kx = cx < 0 ? cx + S.nx : (cx >= S.nx ? cx - S.nx : cx);
            const uint32_t sy = cy < 0 ? 1u : (cy >= S.ny ? 2u : 0u);
            const uint32_t sx = cx < 0 ? 1u : (cx >= S.nx ? 2u : 0u);
            ox = sx == 1u ? -S.L[0] : (sx == 2u ? S.L[0] : 0.0f);
            oy = sy == 1u ? -S.L[1] : (sy == 2u ? S.L[1] : 0.0f);
            code_xy = sx | (sy << 2);
            const int col = S.col_begin + ky * S.nx + kx;
            jb = A.col_slot[col] / kCluster;
            nj = A.col_slot[col + 1] / kCluster - jb;
            // z window over the virtual indices v (image -L: v - nj, 0: v, +L: v + nj)
            // from the column's z-bin index, one bin wider on each side
            // than the FP32 bin arithmetic needs
            const int2 *zt = A.zbin + S.zb_begin + (long long)(col - S.col_begin) * (S.nzb + 1);
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
        s_ci[lane] = make_int4(jb, nj, va - off, (int)code_xy);
        s_co[lane] = make_float2(ox, oy);
        for (int t = off; t < min(off + cnt, kOwnCap); ++t) s_own[t] = (unsigned char)lane;
        __syncwarp();
        for (int p0 = 0; p0 < total; p0 += 64) {
            // both rounds' candidates and box loads first
            int J[2];
            uint32_t code[2];
            float4 jl[2], jh[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int p = p0 + 32 * h + lane;
                // owner lane: the last lane whose window starts at or before p
                int src = 0;
                if (p0 + 32 * h + 31 < kOwnCap) {
                    src = p < total ? s_own[p] : 0;
                } else {
#pragma unroll
                    for (int step = 16; step >= 1; step >>= 1) {
                        const int o2 = __shfl_sync(FULL, off, src + step);
                        if (o2 <= p) src += step;
                    }
                }
                J[h] = -1;
                code[h] = 0u;
                jl[h] = jh[h] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (p < total) {
                    const int4 ci = s_ci[src];
                    const float2 co = s_co[src];
                    J[h] = window_cluster(A.bb, p + ci.z, ci.x, ci.y, (uint32_t)ci.w, co.x, co.y, Lz, code[h], jl[h],
                                          jh[h]);
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (p0 + 32 * h >= total) break;  // the whole warp
                unsigned cm = 0u;
                int hs = -1;
                bool flag = false;
                if (J[h] >= 0 && box_gap2(lo, hi, jl[h], jh[h]) < rcm2) {
                    const int gJ = A.group == 1 ? J[h] : A.clus_grp[J[h]];  // groups of one cluster: the same index
                    const bool other = gJ != g;
                    if (!other || keep_groups(g, gJ)) {
                        if (n == 1) {
                            cm = other || keep_in_group(c0, J[h], code[h]) ? 1u : 0u;
                        } else {
                            for (int q = 0; q < n; ++q)
                                if (box_gap2(s_lo[q], s_hi[q], jl[h], jh[h]) < rcm2 &&
                                    (other || keep_in_group(c0 + q, J[h], code[h])))
                                    cm |= 1u << q;
                        }
                    }
                    if (cm) {
                        const bool self = !other && code[h] == 0u && ((cm >> (J[h] - c0)) & 1u);
                        hs = hset_find(s_hash, J[h]);
                        flag = all_flag || self || hs >= 0;
                    }
                }
                const bool hit = cm != 0u;
                uint2 ent = make_uint2((uint32_t)J[h] | (code[h] << kShiftBit) | (flag ? kExclFlag : 0u), cm);
                // flagged entries: a mask record each, filled by its own lane
                const bool fl = hit && flag;
                const unsigned fb = __ballot_sync(FULL, fl);
                if (fb) {
                    long long slot = -1;
                    const int q = nloc + __popc(fb & lt);
                    if (fl && q < loc_cap) slot = loc_base + q;
                    nloc += __popc(fb);
                    const unsigned ob = __ballot_sync(FULL, fl && slot < 0);
                    if (ob) {  // the group's own records are used up: the pool
                        int pb = 0;
                        if (lane == 0) pb = atomicAdd(A.pool_count, __popc(ob));
                        pb = __shfl_sync(FULL, pb, 0);
                        if (fl && slot < 0) slot = A.pool_base + pb + __popc(ob & lt);
                    }
                    const bool ok = fl && slot < A.mask_cap;
                    if (A.group == 1) {
                        // warp-cooperative: for each flagged lane L, every lane
                        // tests its partner entries against L's cluster and the
                        // bits are OR-reduced over the warp
                        for (unsigned f = fb; f; f &= f - 1u) {
                            const int L = __ffs(f) - 1;
                            const int JL = __shfl_sync(FULL, J[h], L);
                            unsigned e0 = 0u, e1 = 0u, s0 = 0u, s1 = 0u;
#pragma unroll
                            for (int r = 0; r < kPartnerBatch; ++r) {
                                const int v = pk[r];
                                if (v >= 0 && (v >> 7) == JL) {
                                    const int bit = v & 63;
                                    const unsigned m = 1u << (bit & 31);
                                    if (v & 64) {
                                        if (bit < 32) s0 |= m;
                                        else s1 |= m;
                                    } else {
                                        if (bit < 32) e0 |= m;
                                        else e1 |= m;
                                    }
                                }
                            }
                            e0 = __reduce_or_sync(FULL, e0);
                            e1 = __reduce_or_sync(FULL, e1);
                            s0 = __reduce_or_sync(FULL, s0);
                            s1 = __reduce_or_sync(FULL, s1);
                            if (lane == L && ok) {
                                unsigned long long ex = ((unsigned long long)e1 << 32) | e0;
                                if (code[h] == 0u && J[h] == c0) ex |= kSelfTriangle;
                                A.gmask[slot] = make_ulonglong2(ex, ((unsigned long long)s1 << 32) | s0);
                            }
                        }
                    }
                    if (fl) {
                        if (ok) {
                            ulonglong2 *rec = A.gmask + slot * A.group;
                            if (A.group != 1)
                                entry_masks(s_pslot, s_link, hs >= 0 ? s_head[hs] : kLinkEnd, c0, cm, J[h], code[h],
                                            rec);
                            if (all_flag && A.group != 1) {  // the table overflowed: scan every partner
                                for (unsigned ccm = cm; ccm; ccm &= ccm - 1u) {
                                    const int q2 = __ffs(ccm) - 1;
                                    ulonglong2 r = rec[q2];
                                    for (int t = q2 * kCluster * K; t < (q2 + 1) * kCluster * K; ++t) {
                                        const int v = s_pslot[t];
                                        if (v < 0 || ((v >> 1) / kCluster) != J[h]) continue;
                                        const unsigned long long bit =
                                            1ull << (((t / K) % kCluster) * kCluster + ((v >> 1) & 7));
                                        if (v & 1) r.y |= bit;
                                        else r.x |= bit;
                                    }
                                    rec[q2] = r;
                                }
                            }
                            ent.y |= (uint32_t)slot << kMaskSlotBit;
                        } else {
                            atomicOr(A.status, ST_CAPACITY);
                            ent.x &= ~kExclFlag;
                        }
                    }
                }
                // entry r (in scan order) to segment r % kListSegs, position r / kListSegs
                const unsigned bh = __ballot_sync(FULL, hit);
                if (hit) {
                    const int r = ntot + __popc(bh & lt);
                    const int q = r / kListSegs;
                    if (q < seg_cap) LA[(long long)(r % kListSegs) * seg_cap + q] = ent;
                }
                ntot += __popc(bh);
            }
        }
        __syncwarp();  // the owner table and column lists are rewritten by the next round
    }
    if (lane < kListSegs) {
        const int m = (ntot + kListSegs - 1 - lane) / kListSegs;
        A.glist_n[(long long)g * kListSegs + lane] = min(m, seg_cap);
        if (m > seg_cap) atomicOr(A.status, ST_CAPACITY);
    }
}

// Whether the charges are in page-locked host memory (then the binning
// kernel reads charges and types beside the positions, coalesced, instead of
// the column sort gathering them across the host link).  The pointer is
// queried outside stream capture; during a capture the last answer stands
// (it only selects between two ways of reading that give the same result).
static bool inputs_in_host_memory(nb_ctx *ctx, const void *p)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess) {
        cudaGetLastError();
        return ctx->host_inputs;
    }
    if (cs != cudaStreamCaptureStatusNone) return ctx->host_inputs;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return ctx->host_inputs = false;
    }
    return ctx->host_inputs = at.type == cudaMemoryTypeHost;
}

cudaError_t launch_build_cells(nb_ctx *ctx, const float *d_pos, const float *d_q, const int32_t *d_type)
{
    auto &d = ctx->d;
    cudaStream_t st = ctx->stream;
    const int N = (int)ctx->n_atoms;
    const bool host_in = d_q && inputs_in_host_memory(ctx, d_q);
    // the column counts are zero here: zeroed at create and by the scan of
    // the previous build's binning kernel, which leaves a copy for the sort
    const int tb = 256;
    cudaError_t e = launch_pdl(k_bin, dim3((N + tb - 1) / tb), dim3(tb), 0, st, N, d_pos, d.sys, d.atom_sys, d.wpos, d.atom_col,
                   d.col_count, ctx->n_cols, ctx->n_sys, d.col_slot, d.stage_fix, ctx->col_cap, d.counts, d.status,
                   ctx->group, d.col_grp,
                   host_in ? AtomPack{d_q, d_type, ctx->pp.n_types, d.atom_t} : AtomPack{nullptr, nullptr, 0, nullptr});
    if (e == cudaSuccess)
        e = launch_pdl(!d_q ? k_colsort<kPackNone> : (host_in ? k_colsort<kPackAtomT> : k_colsort<kPackGather>),
                       dim3(ctx->n_cols), dim3(kSortThreads), 0, st, (const int *)d.col_count + ctx->n_cols + 1,
                       d.col_slot, d.col_sys, d.sys, (const int *)d.stage_fix, ctx->col_cap, d.stage,
                       (const int *)d.atom_col, d.wpos, d.xyzq, d.tslot, d.perm, d.inv, d.bb, d.clus_sys, d.zbin,
                       ctx->group, d.col_grp, d.grp, d.clus_grp,
                       ColPack{d_q, d_type, ctx->pp.n_types, d.atom_t, d.facc, d.sys_acc, kTaskVals * ctx->n_sys,
                               d.counts + 3, d.status});
    if (e != cudaSuccess) return e;
    ctx->built_group = ctx->group;
    return cudaGetLastError();
}

cudaError_t launch_build_lists(nb_ctx *ctx)
{
    auto &d = ctx->d;
    GListArgs A;
    A.sys = d.sys;
    A.counts = d.counts;
    A.pool_count = d.counts + 5;
    A.bb = d.bb;
    A.clus_sys = d.clus_sys;
    A.col_slot = d.col_slot;
    A.zbin = d.zbin;
    A.perm = d.perm;
    A.part_orig = d.part_orig;
    A.inv = d.inv;
    A.grp = d.grp;
    A.clus_grp = d.clus_grp;
    A.glist = d.glist;
    A.glist_n = d.glist_n;
    A.gmask = d.gmask;
    A.status = d.status;
    A.pool_base = mask_pool_base(ctx->clus_cap);
    A.mask_cap = ctx->mask_cap;
    A.K = ctx->K;
    A.rcm = ctx->pp.rc + ctx->pp.list_margin;
    A.cap = ctx->list_cap;
    A.group = ctx->built_group;
    const size_t smem = sizeof(int) * kGListWarps * glist_warp_ints(ctx->K, ctx->built_group);
    const int64_t blocks = std::max<int64_t>(1, (ctx->grp_cap + kGListWarps - 1) / kGListWarps);
    cudaError_t e = launch_pdl(k_glist, dim3((unsigned)blocks), dim3(kGListWarps * 32), smem, ctx->stream, A);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_build(nb_ctx *ctx, const float *d_pos)
{
    const cudaError_t e = launch_build_cells(ctx, d_pos);
    return e != cudaSuccess ? e : launch_build_lists(ctx);
}

}  // namespace acenb
