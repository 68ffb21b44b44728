// nb_build.cu - cell-list construction: wrap, column binning, per-column
// z-sort and cluster bounding boxes.  (Each cluster's pair list is built in
// shared memory by the force kernel itself.)  Section "Molecular dynamics on the GPU": particles are binned
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
    return cudaGetLastError();
}

}  // namespace acenb
