// nb_internal.cuh - internal types shared by the translation units of the
// GB300 non-bonded library (never installed; the public ABI is acenb.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>
#include <vector>

#include "acenb.h"

namespace acenb {

constexpr int kCluster = 8;          // atoms per cluster (column chunk)
constexpr int kMaxTypes = 64;        // type-pair table lives in shared memory
constexpr int kMaxPartners = 16;     // exclusion + 1-4 partners per atom
constexpr int kErfcDeg = 8;          // degree of the erfcx polynomial in t
constexpr int kExp2Deg = 6;          // degree of the 2^f polynomial on [-1/2, 1/2]
constexpr int kDefaultListSplit = 1; // tile kernels: work units per segment of a group list
constexpr int kMaxGroup = 8;         // clusters per i-group, largest (the masks hold 8 bits)
constexpr int kDefaultGroup = 1;     // clusters per i-group, default (the autotuner may choose 4 or 8)
constexpr int kMaskRecsPerCluster = 6; // exclusion-mask records allocated per cluster
constexpr int kListSegs = 4;         // segments of a group's list (one per list-kernel warp)
constexpr double kFixScale = 4294967296.0;   // 2^32: fixed-point scale
constexpr int kTaskVals = 8;         // per system: E_lj, E_c (scale 2^32), W[6] (scale 2^20)
constexpr double kVirScale = 1048576.0;      // 2^20: fixed-point scale of the virial sums
constexpr int kPmeAcc = 9;           // PME sums: E_recip, E_self, E_excl (2^32), W[6] (2^20)
constexpr int kPmeMaxGrid = 1024;    // largest PME grid edge
struct PmeState;                     // smooth PME state of a single-system context (nb_pme.cu)
struct MdState;                      // molecular-dynamics state of a single-system context (nb_md.cu)
// Padding slots of the sorted arrays sit at this finite, far-away coordinate:
// their squared distance to any atom (about 3e36) stays finite and is never
// inside a cutoff, so masked pair arithmetic needs no further guards.
constexpr float kPadCoord = -1.0e18f;
__host__ __device__ inline bool is_real_coord(float x) { return x > -1.0e17f; }

// Group list entry (uint2).  x: J (bits 0..24) | shift codes x,y,z (2 bits
// each, bits 25..30: 0 none, 1 = j-side shift x_j - L, 2 = i-side shift
// x_i - L) | mask flag (bit 31: the entry's tiles have exclusion masks).
// y: the group's clusters in reach of J (bits 0..7, bit c = cluster c of the
// group) | mask record (bits 8..31, when flagged).
constexpr uint32_t kJMask = 0x01FFFFFFu;
constexpr int kShiftBit = 25;
constexpr uint32_t kExclFlag = 0x80000000u;
constexpr int kMaskSlotBit = 8;

// Device status bits (first error wins when reported).
enum : int {
    ST_NONFINITE = 1 << 0,
    ST_CAPACITY = 1 << 1,
    ST_STALE = 1 << 2,
    ST_OVERFLOW = 1 << 3,
    ST_BADTYPE = 1 << 4,
    ST_TIMEOUT = 1 << 5,
};

// Per-system descriptor (device resident).  Fields marked [build] are
// written by the binning kernels at every build.
struct SysDesc {
    float L[3];          // box edges
    float half[3];       // 0.5 * L (FP32, exact)
    float inv_w[2];      // nx / Lx, ny / Ly rounded to FP32 (column scale)
    float w[2];          // Lx / nx, Ly / ny (FP32, for list bounds)
    int nx, ny;          // columns per axis
    int atom_begin;      // first atom in the concatenated input arrays
    int n_atoms;
    int col_begin;       // first global column
    int slot_begin;      // [build] first sorted slot
    int clus_begin;      // [build] first cluster
    int clus_end;        // [build] one past the last cluster
    // z-bin index of every column: bins of height dz = Lz / nzb; per column
    // nzb + 1 pairs (first cluster with z_hi >= b dz, first cluster with
    // z_lo > (b + 1) dz), at zb_begin + local column * (nzb + 1)
    int nzb;
    int zb_begin;
    float inv_dz;        // nzb / Lz (FP32)
    float dz;            // Lz / nzb (FP32)
};

// Pair-model constants passed by value to kernels.
struct PairParams {
    float rc2;           // rc * rc (FP32, the membership threshold)
    float rc, rs2;       // FP32 cutoff and switch distance squared
    float sw_c0;         // rc2 - 3 rs2
    float sw_inv;        // 1 / (rc2 - rs2)^3
    float sw_a, sw_b, sw_c;  // 1 / (rc2 - rs2)^2, -2 sw_inv, 12 sw_inv (forward kernel's form of the switch)
    float ke;            // Coulomb constant
    float alpha_half;    // alpha / 2: t = 1 / (1 + (alpha/2) r)
    float alpha;         // Ewald alpha
    float neg_a2_log2e;  // -alpha^2 log2(e): exp(-alpha^2 r^2) = 2^(r2 * this)
    float neg_a2_log2e_lo; // the FP32 remainder: -alpha^2 log2(e) = neg_a2_log2e + this (to ~2^-48)
    float two_a_sqpi;    // 2 alpha / sqrt(pi)
    float s14_lj, s14_c;
    float list_margin;   // additive margin on bounding-box distances (A)
    float rcm2;          // (rc + list_margin)^2, bounding-box pruning threshold
    int n_types;
    int switched;        // rs < rc
    int ewald;           // alpha > 0
    float erfc_c[kErfcDeg + 1]; // erfcx(x) ~ sum c_k t^k on [0, alpha rc]
    float exp2_c[kExp2Deg + 1]; // 2^f ~ sum c_k f^k on [-1/2, 1/2]
    float rs;            // FP32 switch distance
    float tab_inv_h;     // n / rc (FP32) of the radial-function tables
    int tab_n;           // intervals of the tables (0: direct evaluation)
};

struct DevBuffers {
    SysDesc *sys = nullptr;          // [n_sys]
    int *atom_sys = nullptr;         // [N]
    int *atom_col = nullptr;         // [N] global column of each atom
    float4 *wpos = nullptr;          // [N] wrapped coordinates (w: the charge when the step packs them)
    int *atom_t = nullptr;           // [N] range-checked types in caller order (nb_step and MD steps)
    int *part_orig = nullptr;        // [N*K] partner (orig << 1) | is14, -1 pad (static)
    int *col_sys = nullptr;          // [C] system of each column (static)
    int *col_count = nullptr;        // [2C+1] column histogram (zero between builds); [C] = completion ticket
                                     // of the binning kernel; [C+1+c] = column c's count for the column sort
    int *col_slot = nullptr;         // [C+1] padded slot offsets
    int *stage = nullptr;            // [S] unsorted atoms of a column whose staging row overflowed
    int *stage_fix = nullptr;        // [C * col_cap] unsorted atoms per column, fixed capacity
    float4 *xyzq = nullptr;          // [S] sorted x, y, z, q (kPadCoord for padding)
    int *tslot = nullptr;            // [S] sorted types
    int *perm = nullptr;             // [S] slot -> atom (-1 padding)
    int *inv = nullptr;              // [N] atom -> slot
    float4 *bb = nullptr;            // [NC*2] cluster bounding boxes (lo, hi interleaved)
    int *clus_sys = nullptr;         // [NC] system of each cluster
    long long *sys_acc = nullptr;    // [n_sys*kTaskVals] per-system fixed-point energies (2^32) and virial (2^20)
    long long *facc = nullptr;       // [S*3] fixed-point forces in sorted order (both atoms of each pair)
    long long *gacc = nullptr;       // [S*4] adjoint: fixed-point dL/dx, dL/dq in sorted order
    int *col_grp = nullptr;          // [C+1] first i-group of each column
    int2 *grp = nullptr;             // [GC] i-group: (first cluster, clusters)
    int *clus_grp = nullptr;         // [NC] i-group of each cluster
    uint2 *glist = nullptr;          // [GC*list_cap] per i-group: its list (Newton's third law at group level)
    int *glist_n = nullptr;          // [GC*kListSegs] lengths of the segments (list_cap / kListSegs entries each)
    ulonglong2 *gmask = nullptr;     // [MC*kMaxGroup] per flagged entry and group cluster: (excluded, 1-4) bits
    int2 *zbin = nullptr;            // [zb_total] z-bin index of the columns (see SysDesc)
    long long *tab_grad = nullptr;   // [T*T*2] adjoint dL/dsig_ab, dL/deps_ab (fixed point, one ordered half)
    int *counts = nullptr;           // [8]: n_slots, n_clusters, unpack ticket, work-unit counter,
                                     //      n_groups, mask records used, -, -
    int *status = nullptr;           // [1]
    float4 *lj_tab = nullptr;        // [T*T] (A, B, A - fl(A), B - fl(B)): FP32 and the FP32 remainders
    float4 *lj_d = nullptr;          // [T*T] 48 eps sig^11, 24 eps sig^5, 4 sig^12, 4 sig^6
    float4 *rtab = nullptr;          // [tab_n*3] tabulated radial functions (nb_set_tables)
    float4 *gslot = nullptr;         // [S] adjoint input dL/dF in sorted order
    float *eps_type = nullptr;       // [T] per-type epsilon (Lorentz-Berthelot chain)
    long long *dbg_n = nullptr;      // [4] debug counters: pair evaluations, pairs, evaluated tile halves, tiles
    int *dbg_ij = nullptr;           // [cap*2]
    int64_t dbg_cap = 0;
    float *scratch_f = nullptr;      // [N*3] debug force sink
    double *scratch_g = nullptr;     // [T*T*2] adjoint scratch
};

}  // namespace acenb

struct nb_ctx {
    int n_sys = 0;
    int64_t n_atoms = 0;
    int n_cols = 0;
    int64_t slot_cap = 0;
    int64_t clus_cap = 0;
    int K = 1;                     // partners per atom (>= 1)
    int comb_rule = 0;
    int stage_cap = 96;            // nb_tuning.stage_capacity (no effect on the kernels)
    int list_cap = 512;            // entries per group list
    int group = acenb::kDefaultGroup;  // clusters per i-group of the last/next build (4 or 8)
    int built_group = 0;           // the group size the current lists were built with
    int64_t grp_cap = 0;           // i-group slots (enough for groups of 4)
    int64_t mask_cap = 0;          // exclusion-mask records
    int col_cap = 0;               // atoms per column staging row (about twice the mean column)
    int tab_n = 0;                 // radial-function table intervals (0: direct evaluation)
    int64_t zb_total = 0;          // entries of the z-bin index
    int smem_optin = 0;            // device opt-in shared memory per block
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    bool built = false;
    bool host_inputs = false;      // the step's charges and types were in host memory at the last query
    acenb::PairParams pp{};
    nb_tuning tune{};
    std::vector<acenb::SysDesc> sys_h;
    std::vector<double> sig_tab, eps_tab;  // FP64 type-pair parameters
    acenb::DevBuffers d;
    acenb::PmeState *pme = nullptr;  // smooth PME, when enabled by nb_set_pme
    acenb::MdState *md = nullptr;    // molecular dynamics, after nb_md_init
    // profiling: event pairs around force-kernel launches
    bool profiling = false;
    std::vector<cudaEvent_t> prof_ev;
    int prof_n = 0;
};

namespace acenb {

// Wrap one FP32 coordinate into [0, L) with IEEE round-to-nearest operations
// in a fixed order: k = floor(x / L); x = fma(-k, L, x); then one conditional
// +L and one conditional -L.
__device__ __forceinline__ float wrap_coord(float x, float L)
{
    if (x >= 0.0f && x < L) return x;
    float k = floorf(__fdiv_rn(x, L));
    x = __fmaf_rn(-k, L, x);
    if (x < 0.0f) x = __fadd_rn(x, L);
    if (x >= L) x = __fsub_rn(x, L);
    return x;
}

// Programmatic dependent launch.  Every kernel of the library calls
// pdl_entry() before it reads or writes anything that another kernel writes
// (at its start, or after a prologue that only fills shared memory from
// tables set at creation): griddepcontrol.wait blocks until the preceding
// kernel in the stream has completed and its memory is visible (a no-op for
// a plain launch), then launch_dependents lets the next kernel's blocks be
// scheduled while this one runs, so consecutive launches do not leave the
// GPU idle.
__device__ __forceinline__ void pdl_entry()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launch with programmatic stream serialization (see pdl_entry).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// i-group slots for a context: every column's clusters form groups of
// `group` clusters, the last one partial, so at most NC / group + C; the
// capacity covers every supported group size (groups of one cluster: NC).
inline int64_t group_capacity(int64_t clus_cap) { return clus_cap + 1; }
// exclusion-mask records (one 16-byte mask pair per cluster of the group, so
// `group` of them per record): the self tiles (one per cluster) and the
// entries whose cluster holds a topology partner of a group atom (a few per
// cluster).  Group (c0, n) fills records c0 kMaskRecsPerCluster ..
// (c0 + n) kMaskRecsPerCluster - 1, the rest come from a shared pool behind
// them.
inline int64_t mask_pool_base(int64_t clus_cap) { return clus_cap * kMaskRecsPerCluster; }
inline int64_t mask_capacity(int64_t clus_cap) { return mask_pool_base(clus_cap) + clus_cap / 2 + 64; }
// atoms per column staging row for a mean column population: twice the mean
// and 32 more, in whole warps (rows that overflow are gathered by the column
// sort's slow fallback)
inline int column_capacity(double mean_atoms) { return ((int)(2.0 * mean_atoms) + 32 + 31) / 32 * 32; }

// Launchers implemented in the .cu files (all asynchronous on ctx->stream).
cudaError_t launch_build(nb_ctx *ctx, const float *d_pos);
// the two halves of launch_build: binning, column sort and cluster boxes;
// then the cluster-pair lists
cudaError_t launch_build_cells(nb_ctx *ctx, const float *d_pos, const float *d_q = nullptr,
                               const int32_t *d_type = nullptr);
cudaError_t launch_build_lists(nb_ctx *ctx);
cudaError_t launch_forces(nb_ctx *ctx, const float *d_pos, const float *d_q, const int32_t *d_type,
                          float *d_F, double *d_energy, double *d_virial, bool debug_pairs);
// launch_forces after its pack (and, when pme_forked, the PME fork): the
// short-range kernel, the PME join and the unpack; beside_pme: the PME chain
// was forked early enough to share the SMs with the short-range kernel;
// helper: a second launch of the short-range kernel behind the PME chain
// takes units from the same counter (worth it when the PME chain ends well
// before the short-range kernel)
cudaError_t launch_forces_packed(nb_ctx *ctx, float *d_F, double *d_energy, double *d_virial, bool debug_pairs,
                                 bool pme_forked, bool beside_pme, bool helper = false);
size_t force_smem_for(int T, int scap, int K);
cudaError_t launch_pack(nb_ctx *ctx, const float *d_pos, const float *d_q, const int32_t *d_type, bool zero_sums);
cudaError_t launch_type_grad(nb_ctx *ctx, const double *gsig_tab, const double *geps_tab, double *gsig, double *geps);
cudaError_t launch_adjoint_tile(nb_ctx *ctx, const double *d_dLdE, float *d_dpos, float *d_dq);
// Smooth PME (nb_pme.cu): the reciprocal-space chain into the context's PME
// force and energy sums; the sums' device arrays (NULL when PME is off).
cudaError_t launch_pme(nb_ctx *ctx, const float *d_pos, const float *d_q);
// the same chain forked onto the PME side stream, and the join back
// sums: also the pair-correction energy and virial (the forces always)
// side_first: launched on the side stream before the PME chain (work that
// is independent of the short-range path, e.g. the MD step's bonded terms).
// The PME side stream; after_lists makes it wait for the pair lists (an event
// on the context's stream), rejoin moves the join event to its current end.
cudaStream_t pme_side_stream(const nb_ctx *ctx);
cudaError_t pme_side_after_lists(nb_ctx *ctx);
cudaError_t pme_side_rejoin(nb_ctx *ctx);
cudaError_t launch_pme_fork(nb_ctx *ctx, const float *d_pos, const float *d_q, bool sums = true,
                            cudaError_t (*side_first)(nb_ctx *, cudaStream_t, const float *) = nullptr);
cudaError_t launch_pme_join(nb_ctx *ctx);
void pme_free(nb_ctx *ctx);
const long long *pme_forces_acc(const nb_ctx *ctx);
const long long *pme_sums_acc(const nb_ctx *ctx);
double pme_self_coef(const nb_ctx *ctx);  // -ke alpha / sqrt(pi), multiplies sum q^2
void md_free(nb_ctx *ctx);
// nb_debug_pair_terms: the forward kernel's pair arithmetic for given pairs
cudaError_t launch_debug_pair_terms(nb_ctx *ctx, long long n, const float4 *xi, const float4 *xj, const int *ti,
                                    const int *tj, float4 *out);
cudaError_t launch_backward(nb_ctx *ctx, const float *d_pos, const float *d_q, const int32_t *d_type,
                            const float *d_dLdF, const double *d_dLdE, float *d_dLdpos, float *d_dLdq,
                            double *d_dsig, double *d_deps);

}  // namespace acenb
