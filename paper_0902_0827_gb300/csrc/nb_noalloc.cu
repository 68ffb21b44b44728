// nb_noalloc.cu - force evaluation for callers that cannot allocate device
// memory.
//
// Some callers of this library may not call cudaMalloc: a host application
// whose memory is handed out by its own pool or arena (every device byte has
// to be accounted for there), a plug-in loaded into a process that forbids
// allocation after start-up, or code that must not trigger the implicit
// synchronisation an allocation can cause.  nb_forces_noalloc serves them: it
// runs the same binning and force kernels as nb_build_cells + nb_forces for
// one system of at most NB_NOALLOC_MAX_ATOMS atoms, with every scratch buffer
// carved from one file-scope device array (g_noalloc_scratch below, about
// 6.0 MiB).  That array exists on every GPU that loads this library, for as
// long as the library stays loaded.
//
// In host code the name g_noalloc_scratch only stands for the device symbol;
// it is not a device address.  The device address is looked up once per
// device with cudaGetSymbolAddress while that device is current, during the
// first call on the device (so that first call should come before any stream
// capture), and cached.  Host-side set-up uses fixed-size static buffers, so
// nothing is allocated on the host heap either.
//
// All calls share the one array and it keeps the previous call's contents:
// the entry point clears what must start at zero (status word, column counts,
// energy accumulators, the sorted type array) at every call.  Calls whose
// kernels overlap on the GPU (different streams, or several host threads at
// once) race on the array and on the host staging buffers; callers must
// serialise them.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>

#include "acenb.h"
#include "nb_host.cuh"
#include "nb_internal.cuh"

using namespace acenb;

namespace {

constexpr int kMaxAtoms = NB_NOALLOC_MAX_ATOMS;
constexpr int kMaxCols = NB_NOALLOC_MAX_COLUMNS;
constexpr int kListCap = 384;  // entries per i-group list
constexpr int kZbEntries = 65536;  // z-bin index entries (bins per column shrink to fit)
constexpr int kMaxDevices = 64;
constexpr long long kSlots = ((long long)kMaxAtoms + (kCluster - 1) * (long long)kMaxCols + kCluster - 1) /
                             kCluster * kCluster;
constexpr long long kClus = kSlots / kCluster;
constexpr long long kGrp = kClus + 1;                          // i-group slots (group_capacity)
constexpr long long kMaskRecs = kClus * kMaskRecsPerCluster + kClus / 2 + 64;  // exclusion-mask records (mask_capacity)

constexpr size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// Byte offsets of every scratch buffer inside the static array.
constexpr size_t oSys = 0;
constexpr size_t oAtomSys = oSys + a256(sizeof(SysDesc));
constexpr size_t oAtomCol = oAtomSys + a256(4ull * kMaxAtoms);
constexpr size_t oWpos = oAtomCol + a256(4ull * kMaxAtoms);
constexpr size_t oPart = oWpos + a256(16ull * kMaxAtoms);
constexpr size_t oColSys = oPart + a256(4ull * kMaxAtoms * kMaxPartners);
constexpr size_t oColCount = oColSys + a256(4ull * kMaxCols);
constexpr long long kStageFix = 4 * kSlots;  // column staging rows (col_cap per column, fitted to the system)
constexpr size_t oStageFix = oColCount + a256(4ull * (2 * kMaxCols + 1));
constexpr size_t oColSlot = oStageFix + a256(4ull * kStageFix);
constexpr size_t oStage = oColSlot + a256(4ull * (kMaxCols + 1));
constexpr size_t oXyzq = oStage + a256(4ull * kSlots);
constexpr size_t oTslot = oXyzq + a256(16ull * kSlots);
constexpr size_t oPerm = oTslot + a256(4ull * kSlots);
constexpr size_t oInv = oPerm + a256(4ull * kSlots);
constexpr size_t oBb = oInv + a256(4ull * kMaxAtoms);
constexpr size_t oClusSys = oBb + a256(32ull * kClus);
constexpr size_t oSysAcc = oClusSys + a256(4ull * kClus);
constexpr size_t oFacc = oSysAcc + a256(8ull * kTaskVals);
constexpr size_t oColGrp = oFacc + a256(24ull * kSlots);
constexpr size_t oGrp = oColGrp + a256(4ull * (kMaxCols + 1));
constexpr size_t oClusGrp = oGrp + a256(8ull * kGrp);
constexpr size_t oGlist = oClusGrp + a256(4ull * kClus);
constexpr size_t oGlistN = oGlist + a256(8ull * kGrp * kListCap);
constexpr size_t oGmask = oGlistN + a256(4ull * kGrp * kListSegs);
constexpr size_t oZbin = oGmask + a256(16ull * kMaskRecs * kDefaultGroup);  // records of one-cluster groups
constexpr size_t oCounts = oZbin + a256(8ull * kZbEntries);
constexpr size_t oStatus = oCounts + a256(32);
constexpr size_t oLj = oStatus + a256(16);
constexpr size_t oDbg = oLj + a256(16ull * kMaxTypes * kMaxTypes);
constexpr size_t kScratchBytes = oDbg + a256(16);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// host-side staging (fixed size, no heap)
SysDesc h_sys;
int h_part[kMaxAtoms * kMaxPartners];
int h_cnt[kMaxAtoms];
double h_sg[kMaxTypes * kMaxTypes], h_ep[kMaxTypes * kMaxTypes];
float4 h_lj[kMaxTypes * kMaxTypes];
unsigned char *g_dev_scratch[kMaxDevices];  // cached device address per device

template <class T>
T *at(unsigned char *base, size_t off)
{
    return reinterpret_cast<T *>(base + off);
}

nb_status add_partner(int i, int v)
{
    for (int k = 0; k < h_cnt[i]; ++k) {
        if (h_part[i * kMaxPartners + k] == v) return NB_OK;             // duplicate
        if ((h_part[i * kMaxPartners + k] >> 1) == (v >> 1)) return NB_ERR_INVALID_ARG;  // excluded and 1-4
    }
    if (h_cnt[i] >= kMaxPartners) return NB_ERR_UNSUPPORTED;
    h_part[i * kMaxPartners + h_cnt[i]++] = v;
    return NB_OK;
}

}  // namespace

extern "C" nb_status nb_forces_noalloc(const nb_params *params, const float *d_pos, const float *d_q,
                                       const int32_t *d_type, float *d_F, double *d_energy, double *d_virial,
                                       void *cuda_stream)
{
    if (!params || !d_pos || !d_q || !d_type || !d_F) return NB_ERR_INVALID_ARG;
    nb_status st = host::validate_one(params);
    if (st != NB_OK) return st;
    const nb_params &p = *params;
    if (p.n_atoms > kMaxAtoms) return NB_ERR_TOO_LARGE;
    SysDesc S;
    host::init_sysdesc(p, S, 0, 0, 0);
    const int C = S.nx * S.ny;
    if (C > kMaxCols) return NB_ERR_TOO_LARGE;
    host::init_sysdesc(p, S, 0, 0, 0, kZbEntries / C - 1);
    PairParams pp;
    if (host::init_pair_params(p, pp) != NB_OK) return NB_ERR_UNSUPPORTED;
    // topology: per-atom partners (orig << 1) | is14, padded with -1
    const int N = p.n_atoms;
    memset(h_cnt, 0, sizeof(int) * N);
    for (int k = 0; k < p.n_excl && st == NB_OK; ++k) {
        const int i = p.excl[2 * k], j = p.excl[2 * k + 1];
        st = add_partner(i, j << 1);
        if (st == NB_OK) st = add_partner(j, i << 1);
    }
    for (int k = 0; k < p.n_14 && st == NB_OK; ++k) {
        const int i = p.pairs14[2 * k], j = p.pairs14[2 * k + 1];
        st = add_partner(i, (j << 1) | 1);
        if (st == NB_OK) st = add_partner(j, (i << 1) | 1);
    }
    if (st != NB_OK) return st;
    int K = 1;
    for (int i = 0; i < N; ++i) K = h_cnt[i] > K ? h_cnt[i] : K;
    // repack to stride K
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < K; ++k) h_part[i * K + k] = k < h_cnt[i] ? h_part[i * kMaxPartners + k] : -1;
    const int T = p.n_types;
    host::make_tables(T, p.comb_rule, p.sigma, p.epsilon, p.sigma_tab, p.eps_tab, h_sg, h_ep, h_lj);
    h_sys = S;

    // the device address of the scratch array, looked up once per device
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NB_ERR_CUDA;
    if (!g_dev_scratch[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return NB_ERR_CUDA;
        g_dev_scratch[dev] = static_cast<unsigned char *>(ptr);
    }
    unsigned char *base = g_dev_scratch[dev];

    nb_ctx c;  // lives on the stack; its host vectors stay empty
    c.n_sys = 1;
    c.n_atoms = N;
    c.n_cols = C;
    c.slot_cap = ((long long)N + (long long)(kCluster - 1) * C + kCluster - 1) / kCluster * kCluster;
    c.clus_cap = c.slot_cap / kCluster;
    c.K = K;
    c.stream = (cudaStream_t)cuda_stream;
    c.device = dev;
    cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (c.num_sms < 1) c.num_sms = 1;
    c.built = true;
    c.pp = pp;
    c.tune.blocks_per_sm = 3;
    c.tune.stage_capacity = 96;
    c.tune.list_capacity = kListCap;
    c.tune.list_split = kDefaultListSplit;
    c.tune.group_clusters = kDefaultGroup;
    c.group = kDefaultGroup;
    c.grp_cap = kGrp;
    c.mask_cap = kMaskRecs;
    c.col_cap = std::max(1, std::min(column_capacity((double)N / (double)C), (int)(kStageFix / C)));
    c.stage_cap = 96;
    c.list_cap = kListCap;
    c.zb_total = host::zbin_entries(S);
    c.comb_rule = p.comb_rule;
    DevBuffers &d = c.d;
    d.sys = at<SysDesc>(base, oSys);
    d.atom_sys = at<int>(base, oAtomSys);
    d.atom_col = at<int>(base, oAtomCol);
    d.wpos = at<float4>(base, oWpos);
    d.part_orig = at<int>(base, oPart);
    d.col_sys = at<int>(base, oColSys);
    d.col_count = at<int>(base, oColCount);
    d.stage_fix = at<int>(base, oStageFix);
    d.col_slot = at<int>(base, oColSlot);
    d.stage = at<int>(base, oStage);
    d.xyzq = at<float4>(base, oXyzq);
    d.tslot = at<int>(base, oTslot);
    d.perm = at<int>(base, oPerm);
    d.inv = at<int>(base, oInv);
    d.bb = at<float4>(base, oBb);
    d.clus_sys = at<int>(base, oClusSys);
    d.sys_acc = at<long long>(base, oSysAcc);
    d.facc = at<long long>(base, oFacc);
    d.col_grp = at<int>(base, oColGrp);
    d.grp = at<int2>(base, oGrp);
    d.clus_grp = at<int>(base, oClusGrp);
    d.glist = at<uint2>(base, oGlist);
    d.glist_n = at<int>(base, oGlistN);
    d.gmask = at<ulonglong2>(base, oGmask);
    d.zbin = at<int2>(base, oZbin);
    d.counts = at<int>(base, oCounts);
    d.status = at<int>(base, oStatus);
    d.lj_tab = at<float4>(base, oLj);
    d.dbg_n = at<long long>(base, oDbg);

    // per-call inputs of the scratch; zero what the kernels expect zeroed
    cudaStream_t s = c.stream;
    cudaError_t e = cudaMemcpyAsync(d.sys, &h_sys, sizeof(SysDesc), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.atom_sys, 0, sizeof(int) * N, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.col_sys, 0, sizeof(int) * C, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.part_orig, h_part, sizeof(int) * N * K, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.lj_tab, h_lj, sizeof(float4) * T * T, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.status, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.col_count, 0, sizeof(int) * (C + 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.tslot, 0, sizeof(int) * c.slot_cap, s);
    if (e == cudaSuccess) e = launch_build(&c, d_pos);
    if (e == cudaSuccess) e = launch_forces(&c, d_pos, d_q, d_type, d_F, d_energy, d_virial, false);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, d.status, sizeof(int), cudaMemcpyDeviceToHost);
    c.d = DevBuffers();  // the scratch belongs to the static array, not to c
    if (e != cudaSuccess) return NB_ERR_CUDA;
    if (h & ST_NONFINITE) return NB_ERR_NONFINITE;
    if (h & ST_CAPACITY) return NB_ERR_CAPACITY;
    if (h & ST_BADTYPE) return NB_ERR_INVALID_ARG;
    if (h & ST_OVERFLOW) return NB_ERR_OVERFLOW;
    return NB_OK;
}
