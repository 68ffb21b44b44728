/*
 * acenb.h - C ABI of the GB300 short-range non-bonded library.
 *
 * The library evaluates the short-range non-bonded forces, energies and
 * virial of an all-atom system as described in Harvey, Giupponi & De
 * Fabritiis (2009), section "Molecular dynamics on the GPU": atoms are binned
 * into a cell list built from their coordinates ("one particle per thread"),
 * and the non-bonded kernel evaluates Lennard-Jones and electrostatic terms
 * for every pair within the cutoff R, excluding or scaling bonded pairs
 * ("exclusion bitmaps", inner/outer kernels).  It adds the adjoint used for
 * force-field fitting and a batched form for many independent boxes.
 *
 * Functional forms (the paper names them but prints no formula):
 *   U_LJ = w_lj * S(r) * (A_ab / r^12 - B_ab / r^6),
 *          A_ab = 4 eps_ab sig_ab^12, B_ab = 4 eps_ab sig_ab^6,
 *          Lorentz-Berthelot: sig_ab = (sig_a + sig_b) / 2, eps_ab = sqrt(eps_a eps_b)
 *          (CHARMM force field, section "Molecular dynamics on the GPU");
 *   S(r) = 1 for r <= rs, (rc^2 - r^2)^2 (rc^2 + 2 r^2 - 3 rs^2) / (rc^2 - rs^2)^3
 *          for rs < r < rc (CHARMM switch; "switched at 7.5 A", section
 *          "Performance");
 *   U_C  = w_c * ke * q_i q_j * erfc(alpha r) / r, truncated at rc (real-space
 *          Ewald part of PME, section "Molecular dynamics on the GPU");
 *   w    = 0 for excluded (1-2, 1-3) pairs, (s14_lj, s14_coul) for 1-4 pairs,
 *          1 otherwise.
 * A pair (i, j) is inside the cutoff iff r2 < rc*rc evaluated in FP32 with the
 * minimum-image displacement d = x_j - x_i taken per axis as
 *   s = x_j - x_i;  s > L/2: d = (x_j - L) - x_i;  s < -L/2: d = x_j - (x_i - L);
 *   else d = s;     r2 = fma(dz, dz, fma(dy, dy, dx * dx)).
 * Coordinates are first wrapped into [0, L) per axis with FP32 operations.
 * Pair arithmetic is FP32; per-lane partial sums are combined in 64-bit
 * fixed point (scale 2^32), so every result is bit-identical from run to run.
 *
 * Conventions
 *   - d_* arguments are device pointers owned by the caller; h_* are host
 *     pointers.  The context owns all scratch memory (allocated at create).
 *   - Calls are asynchronous on the context's CUDA stream and launch kernels
 *     only (no host synchronisation, no allocation), so they can be captured
 *     into a CUDA graph.  Host-detectable errors are returned immediately;
 *     device-detected errors are recorded in a device status word and
 *     reported (and cleared) by nb_get_status.
 *   - Arrays are row-major.  Positions, forces and gradients are [N, 3] FP32.
 *   - A batch holds n_sys independent systems; per-atom arrays are the
 *     systems' arrays concatenated in system order, energies are [n_sys, 2]
 *     (LJ, Coulomb) and virials [n_sys, 6] (xx, yy, zz, xy, xz, yz).
 *     W_ab = sum over pairs of d_ab,a * f_ab,b with d = x_i - x_j and f the
 *     force on i due to j (so dE/dlambda = -tr W under x -> lambda x).
 */
#ifndef ACENB_H
#define ACENB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ACENB_VERSION 2

typedef enum {
    NB_OK = 0,
    NB_ERR_INVALID_ARG = 1,   /* a host-checked argument is invalid */
    NB_ERR_BOX_TOO_SMALL = 2, /* L/2 - rc < 1e-4 L on some axis (minimum image ambiguous) */
    NB_ERR_CUDA = 3,          /* a CUDA runtime call failed */
    NB_ERR_OOM = 4,           /* device allocation failed at create */
    NB_ERR_NOT_BUILT = 5,     /* nb_forces/nb_backward before nb_build_cells */
    NB_ERR_OVERFLOW = 6,      /* a value left the 64-bit fixed-point range */
    NB_ERR_LIST_STALE = 7,    /* positions differ from those of the last build */
    NB_ERR_TIMEOUT = 8,       /* a bounded device-side wait gave up */
    NB_ERR_NONFINITE = 9,     /* a coordinate is NaN or infinite */
    NB_ERR_CAPACITY = 10,     /* a per-cluster neighbour list exceeded its capacity */
    NB_ERR_UNSUPPORTED = 11,  /* parameters outside the supported range */
    NB_ERR_TOO_LARGE = 12     /* system larger than nb_forces_noalloc's fixed scratch */
} nb_status;

typedef struct nb_ctx nb_ctx;

/* Parameters of one system.  Host arrays are copied by nb_create; the caller
 * may free them afterwards. */
typedef struct {
    int32_t n_atoms;        /* N >= 1 */
    float box[3];           /* orthorhombic edges L_x, L_y, L_z (A); L/2 - rc >= 1e-4 L */
    float cutoff;           /* rc (A), > 0 */
    float switch_dist;      /* rs (A); rs >= rc disables the switch */
    float ewald_alpha;      /* alpha (1/A); 0 gives plain truncated Coulomb */
    float coulomb_k;        /* ke (kcal A / (mol e^2)); 0 selects 332.0636 */
    int32_t n_types;        /* T, 1 <= T <= 64 */
    const float *sigma;     /* host [T] per-type sigma (A), comb_rule 0 */
    const float *epsilon;   /* host [T] per-type epsilon (kcal/mol), comb_rule 0 */
    int32_t comb_rule;      /* 0: Lorentz-Berthelot; 1: explicit pair tables */
    const float *sigma_tab; /* host [T*T] symmetric sig_ab, comb_rule 1 */
    const float *eps_tab;   /* host [T*T] symmetric eps_ab, comb_rule 1 */
    int32_t n_excl;         /* number of excluded pairs; every atom has at most 16 topology
                               partners (excluded + scaled 1-4), NB_ERR_UNSUPPORTED otherwise */
    const int32_t *excl;    /* host [n_excl*2] atom pairs (i, j), i != j, 0-based */
    int32_t n_14;           /* number of scaled 1-4 pairs */
    const int32_t *pairs14; /* host [n_14*2], disjoint from excl */
    float scale14_lj;       /* LJ scale of 1-4 pairs (e.g. 0.5) */
    float scale14_coul;     /* Coulomb scale of 1-4 pairs (e.g. 1/1.2) */
    uint32_t flags;         /* reserved, must be 0 */
} nb_params;

/* Tuning knobs (chosen by the autotuner; defaults are safe). */
typedef struct {
    int32_t blocks_per_sm;  /* blocks per SM of the forward kernel's persistent grid, 1..8 */
    int32_t stage_capacity; /* no effect (both kernels stage their lists in 32-entry batches);
                               validated as 16..512, multiple of 4 */
    int32_t list_capacity;  /* entries of an i-group's list (its share of the cluster pairs:
                               every pair of clusters is listed by one of its two groups),
                               64..65536, multiple of 4 */
    int32_t list_split;     /* tile kernels: work units (warps) per segment of a group's list
                               (4 segments per group), 1..8; 0 = default (1) */
    int32_t group_clusters; /* clusters per i-group, 1, 4 or 8: the tile shape of the forward
                               kernel (1: one 8 x 8 tile per list entry, the i atoms in
                               registers; 4 or 8: a warp works on 32 or 64 i atoms against one
                               listed 8-atom cluster at a time); 0 = default (1).  A change
                               takes effect at the next nb_build_cells. */
} nb_tuning;

/* nb_create - one system.  Copies params, validates them (box/cutoff ratio,
 * index ranges, disjoint topology), allocates all device scratch and binds
 * the context to `cuda_stream` (a cudaStream_t; NULL = legacy default).
 * Errors: NB_ERR_INVALID_ARG, NB_ERR_BOX_TOO_SMALL, NB_ERR_UNSUPPORTED,
 * NB_ERR_OOM, NB_ERR_CUDA.  *out is NULL on error. */
nb_status nb_create(const nb_params *params, void *cuda_stream, nb_ctx **out);

/* nb_create_batch - n_sys independent systems evaluated together in one
 * persistent launch.  params[s] gives system s; cutoff, switch_dist,
 * ewald_alpha, coulomb_k, types and 1-4 scales must be equal across systems
 * (NB_ERR_INVALID_ARG otherwise); n_atoms, box and topology may differ. */
nb_status nb_create_batch(int32_t n_sys, const nb_params *params, void *cuda_stream, nb_ctx **out);

/* nb_build_cells - wrap d_pos [N, 3] into the box, bin atoms into x-y
 * columns, z-sort each column, pad columns to whole 8-atom clusters, compute
 * cluster bounding boxes, map exclusions to the sorted order and build the
 * cluster-pair list (section "Molecular dynamics on the GPU", cell-list
 * construction).  Asynchronous.  Device errors: NB_ERR_NONFINITE,
 * NB_ERR_CAPACITY. */
nb_status nb_build_cells(nb_ctx *ctx, const float *d_pos);

/* nb_forces - forces, energies and virial for the positions of the last
 * build (section "Molecular dynamics on the GPU", non-bonded kernel).
 *   d_pos   [N, 3]  must hold the positions passed to nb_build_cells
 *                   (NB_ERR_LIST_STALE is recorded otherwise);
 *   d_q     [N]     charges (e);  d_type [N] LJ types in [0, T);
 *   d_F     [N, 3]  output forces (kcal/mol/A), overwritten;
 *   d_energy[n_sys*2] output (E_LJ, E_Coul) in kcal/mol, or NULL;
 *   d_virial[n_sys*6] output, or NULL.
 * Returns NB_ERR_NOT_BUILT without a preceding build. */
nb_status nb_forces(nb_ctx *ctx, const float *d_pos, const float *d_q, const int32_t *d_type,
                    float *d_F, double *d_energy, double *d_virial);

/* nb_forces_batch - nb_forces on a context made by nb_create_batch: the
 * systems' concatenated arrays (atom ranges in system order, offsets fixed at
 * create), energies [n_sys, 2] and virials [n_sys, 6]; all systems are
 * evaluated by one persistent launch of the force kernel.  The same call as
 * nb_forces (which also accepts batch contexts), under the batch name. */
nb_status nb_forces_batch(nb_ctx *batch, const float *d_pos, const float *d_q, const int32_t *d_type,
                          float *d_F, double *d_energy, double *d_virial);

/* nb_step - one evaluation from positions: nb_build_cells followed by
 * nb_forces on the same arrays (section "Molecular dynamics on the GPU":
 * the cell list is rebuilt and the forces evaluated every step), in fewer
 * kernels: the binning kernel reads the charges and types beside the
 * positions and the column sort carries them into sorted order, and with
 * PME the reciprocal chain starts before the pair lists.
 * Arguments, outputs and errors as for nb_forces; the context is built
 * afterwards, so nb_forces and nb_backward may follow on the same
 * positions.  Results are bit-identical to nb_build_cells + nb_forces.
 * Each array may also be page-locked host memory that the device addresses
 * at the same address (cudaHostAlloc under unified addressing): the kernels
 * then read the inputs and write the results across the host link, with
 * no separate copy, and the results are in host memory once the stream has
 * completed.  Other host memory must not be passed. */
nb_status nb_step(nb_ctx *ctx, const float *d_pos, const float *d_q, const int32_t *d_type, float *d_F,
                  double *d_energy, double *d_virial);

/* nb_backward - adjoint of L = sum_i G_i . F_i + sum_s gE_s . E_s, the pair
 * list recomputed from the last build (short-range terms, direct radial
 * functions; a context with smooth PME or tables enabled returns
 * NB_ERR_UNSUPPORTED).
 *   d_dLdF      [N, 3]      G;  d_dLdE [n_sys*2] gE (LJ, Coulomb) or NULL (= 0);
 *   d_dLdpos    [N, 3]      dL/dx = -H G - (gE weighted) F   (Hessian-vector product);
 *   d_dLdq      [N]         dL/dq;
 *   d_dLdsig_tab, d_dLdeps_tab [T*T] FP64 gradients with respect to the
 *               symmetric type-pair parameters sig_ab, eps_ab (each unordered
 *               pair's value stored at [a][b] and [b][a]).
 * Any output pointer may be NULL to skip it. */
nb_status nb_backward(nb_ctx *ctx, const float *d_pos, const float *d_q, const int32_t *d_type,
                      const float *d_dLdF, const double *d_dLdE,
                      float *d_dLdpos, float *d_dLdq, double *d_dLdsig_tab, double *d_dLdeps_tab);

/* nb_set_lj_params - replace the LJ type parameters between calls (e.g. after
 * a fitting step).  comb_rule 0: h_sigma, h_epsilon [T]; comb_rule 1:
 * h_sigma_tab, h_eps_tab [T*T] symmetric.  Synchronises the context's stream
 * and copies the new (A, B) table; not capturable in a CUDA graph.
 * Errors: NB_ERR_INVALID_ARG for missing or negative values. */
nb_status nb_set_lj_params(nb_ctx *ctx, const float *h_sigma, const float *h_epsilon,
                           const float *h_sigma_tab, const float *h_eps_tab);

/* nb_type_gradients - per-type gradients from the type-pair gradients of
 * nb_backward under the Lorentz-Berthelot rule (comb_rule 0):
 *   dL/dsig_t = sum_{b != t} dL/dsig_tb / 2 + dL/dsig_tt,
 *   dL/deps_t = sum_{b != t} dL/deps_tb * eps_b / (2 sqrt(eps_t eps_b)) + dL/deps_tt
 * (NaN for a type with eps_t = 0, where sqrt(eps_t eps_b) has no derivative).
 *   d_dLdsig_tab, d_dLdeps_tab [T*T] FP64 device inputs; d_dLdsigma, d_dLdeps
 *   [T] FP64 device outputs.  Asynchronous.  NB_ERR_UNSUPPORTED for comb_rule 1. */
nb_status nb_type_gradients(nb_ctx *ctx, const double *d_dLdsig_tab, const double *d_dLdeps_tab,
                            double *d_dLdsigma, double *d_dLdeps);

/* nb_get_status - synchronise the context's stream, return the first
 * recorded device error (or NB_OK) and clear it. */
nb_status nb_get_status(nb_ctx *ctx);

/* nb_set_stream - rebind the context to another stream. */
nb_status nb_set_stream(nb_ctx *ctx, void *cuda_stream);

/* nb_destroy - free every device and host resource of the context. */
void nb_destroy(nb_ctx *ctx);

/* nb_set_tuning / nb_get_tuning - read or change the launch configuration;
 * takes effect at the next launch.  A changed list_capacity reallocates the
 * pair lists (synchronises the stream; not allowed during stream capture) and
 * requires a new nb_build_cells.  Errors: NB_ERR_INVALID_ARG for values out of
 * range, NB_ERR_UNSUPPORTED when the shared-memory footprint of the force
 * kernel would exceed the device limit, NB_ERR_OOM. */
nb_status nb_set_tuning(nb_ctx *ctx, const nb_tuning *t);
nb_status nb_get_tuning(nb_ctx *ctx, nb_tuning *t);

/* Sizes of the context: total atoms, systems, sorted slots capacity. */
nb_status nb_get_sizes(nb_ctx *ctx, int64_t *n_atoms, int32_t *n_sys, int64_t *slot_capacity);

/* nb_debug_cells - synchronous copy of the last build's binning:
 * h_perm [slot_capacity] receives, per sorted slot, the original atom index
 * (batch-global) or -1 for padding; *n_slots the number of used slots;
 * h_col_start [n_columns+1] the padded slot offset of each column (columns of
 * system s follow those of s-1, column id = cy * nx + cx); *n_columns their
 * count.  Either array may be NULL. */
nb_status nb_debug_cells(nb_ctx *ctx, int32_t *h_perm, int64_t *n_slots,
                         int64_t *h_col_start, int64_t *n_columns);

/* nb_debug_pairs - run the pair filter of the force kernel for the last
 * build and copy out every evaluated pair inside the cutoff and not excluded,
 * as original atom indices (i < j), into h_ij [cap*2]; *n receives the total
 * count of such unique pairs (may exceed cap) and *n_ordered the number of
 * pair evaluations of the forward kernel (equal to n: it evaluates every
 * unique pair once and applies the force to both atoms).  Synchronous. */
nb_status nb_debug_pairs(nb_ctx *ctx, int32_t *h_ij, int64_t cap, int64_t *n, int64_t *n_ordered);

/* nb_debug_fill - tile fill of the last nb_debug_pairs run: *tiles receives
 * the number of 8 x 8 cluster-pair tiles the forward kernel visited and
 * *halves the number of 4 x 8 tile halves whose pair arithmetic ran (at
 * least one of their 32 pairs inside the cutoff and not excluded).  With the
 * pair count n of nb_debug_pairs, n / (64 tiles) is the tile fill and
 * n / (32 halves) the fraction of evaluated lanes doing useful work.
 * Measurement export without a counterpart in the paper.  Synchronous. */
nb_status nb_debug_fill(nb_ctx *ctx, int64_t *tiles, int64_t *halves);

/* nb_debug_pair_terms - the forward kernel's FP32 pair arithmetic (section
 * "Molecular dynamics on the GPU": the Lennard-Jones and electrostatic terms
 * of one pair; forms in the header comment above) for n given pairs, so that
 * its rounding can be measured pair by pair against an FP64 evaluation.
 * d_xqi, d_xqj [n,4]: (x, y, z, q) of atoms i and j, 16-byte aligned;
 * d = x_j - x_i is taken as given (no minimum image), and each pair must lie
 * inside the cutoff with d != 0.  d_ti, d_tj [n]: types (< n_types).
 * d_out [n,8]: (E_LJ switched, E_Coul, r2, 0, then the force on j (x, y, z),
 * 0) with unit weights (no exclusion or 1-4 scaling), through the radial
 * functions the context uses (direct or tabulated).  Asynchronous on the
 * context's stream; needs no build. */
nb_status nb_debug_pair_terms(nb_ctx *ctx, int64_t n, const float *d_xqi, const float *d_xqj,
                              const int32_t *d_ti, const int32_t *d_tj, float *d_out);

/* nb_debug_philox - Philox4x32-10 (Salmon, Moraes, Dror & Shaw 2011), the
 * counter-based generator of the MD step's Langevin noise (the paper's
 * thermostat draws Gaussian noise per atom and step), for n counter blocks:
 * d_ctr [n,4] counters, d_key [n,2] keys, d_out [n,4] the ten-round outputs.
 * A test export: it pins the device generator to published known-answer
 * vectors.  Asynchronous on cuda_stream; no context needed. */
nb_status nb_debug_philox(int64_t n, const uint32_t *d_ctr, const uint32_t *d_key, uint32_t *d_out,
                          void *cuda_stream);

/* nb_set_profiling - when on != 0, every later force-kernel launch is
 * bracketed by CUDA events on the context's stream (at most 4096 launches are
 * recorded; do not enable during stream capture).  nb_get_profile
 * synchronises, returns the summed duration in milliseconds and the number
 * of recorded launches of the force kernel, and clears the record. */
nb_status nb_set_profiling(nb_ctx *ctx, int32_t on);
nb_status nb_get_profile(nb_ctx *ctx, double *force_ms, int64_t *launches);

/* nb_forces_noalloc - forces, energies and virial of ONE system for callers
 * that cannot allocate device memory (for example a host application whose
 * device memory all comes from its own pool, or a plug-in that may not call
 * cudaMalloc after start-up).  The paper has no counterpart: this is an
 * interface convenience around the same binning and force kernels as
 * nb_build_cells + nb_forces.
 *   params   as for nb_create (one system);
 *   d_pos, d_q, d_type, d_F, d_energy [2], d_virial [6]: as for nb_forces
 *            (d_energy / d_virial may be NULL);
 *   cuda_stream: the stream the work runs on.
 * All scratch lives in one static device array of about 6.0 MiB that every
 * GPU loading this library holds until the library is unloaded; it bounds
 * the system to NB_NOALLOC_MAX_ATOMS atoms and NB_NOALLOC_MAX_COLUMNS x-y
 * columns (NB_ERR_TOO_LARGE otherwise).  The call allocates nothing (no
 * cudaMalloc, no cudaFree, no host heap).  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  The call
 * synchronises its stream and returns device-detected errors itself.  Every
 * call reuses the same array: calls that overlap on the GPU, or run from
 * several host threads at once, race and must be serialised by the caller. */
#define NB_NOALLOC_MAX_ATOMS 4096
#define NB_NOALLOC_MAX_COLUMNS 1024
nb_status nb_forces_noalloc(const nb_params *params, const float *d_pos, const float *d_q,
                            const int32_t *d_type, float *d_F, double *d_energy, double *d_virial,
                            void *cuda_stream);

/* nb_set_tables - evaluate the radial functions of the forward kernel by
 * linear interpolation of lookup tables instead of directly (section
 * "Molecular dynamics on the GPU": the texture units interpolate the radial
 * parts of the van der Waals and electrostatic terms from tables; its error
 * figure uses n = 4096 points).  n_intervals > 0 tabulates, on [0, rc] with
 * r_k = k rc / n, the six functions E12 = S r^-12, E6 = S r^-6,
 * Ec = erfc(alpha r)/r (1/r without Ewald) and F = -r dE/dr of each, as the
 * FP32 values at r_k (at max(r_k, 0.5 A)) and the FP32 differences to
 * r_{k+1}; a pair at distance r uses interval k = floor(r n / rc) (at most
 * n - 1) and f = T_k + t D_k with t = r n / rc - k, in FP32.  Then
 * U_LJ = w_lj (A E12 - B E6) and U_C = w_c ke q_i q_j Ec.  n_intervals = 0
 * restores direct evaluation.  The pair set is unchanged.  Allocates
 * 48 n bytes, synchronises the stream, not capturable; applies to nb_forces
 * (nb_backward returns NB_ERR_UNSUPPORTED while tables are on).
 * Errors: NB_ERR_INVALID_ARG (n_intervals not 0 and outside 16..65536),
 * NB_ERR_OOM, NB_ERR_CUDA. */
nb_status nb_set_tables(nb_ctx *ctx, int32_t n_intervals);

/* Smooth particle-mesh Ewald (section "Molecular dynamics on the GPU": the
 * long-range electrostatics by PME with the FFT library; section
 * "Performance": 64^3 grid, fourth-order interpolation), after Essmann et
 * al.: charges spread on a K1 x K2 x K3 grid with cardinal B-splines of
 * order n, E_recip = 1/2 sum_{m != 0} ke B(m) C(m) |FQ(m)|^2 with
 * C(m) = exp(-pi^2 m^2 / alpha^2) / (pi V m^2) and the B-spline moduli B(m),
 * forces by differentiating the B-splines, virial
 * W_ab = sum_m E(m) (delta_ab - 2 (1 + pi^2 m^2 / alpha^2) m_a m_b / m^2).
 * With it come the Ewald corrections that make real + reciprocal space the
 * Coulomb sum the topology asks for: the self energy
 * E_self = -ke alpha / sqrt(pi) sum_i q_i^2 and, per excluded pair,
 * -ke q_i q_j erf(alpha r) / r, per scaled 1-4 pair (1 - scale14_coul) times
 * that (FP32 pair arithmetic on the wrapped coordinates, minimum image).  Each
 * pair then contributes w_c ke q_i q_j / r in total: 0 when excluded,
 * scale14_coul when 1-4, 1 otherwise.
 * The charges are spread from the cell list of the last nb_build_cells (each
 * x plane of the grid by one block, from the columns its atoms can come
 * from), summed in fixed point (scale 2^32) in shared memory; forces,
 * energies and virial go to the library's fixed-point sums, so reruns are
 * bit-identical.  B-spline weights and pair terms are FP32; the FFTs are
 * cuFFT's (FP32). */
typedef struct {
    int32_t grid[3]; /* K1, K2, K3: grid points per box edge, order..1024 */
    int32_t order;   /* B-spline order n: 4, 6 or 8 */
    int32_t flags;   /* reserved, must be 0 */
} nb_pme_params;

/* nb_set_pme - enable smooth PME on a single-system context with Ewald
 * (ewald_alpha > 0), or disable it (p == NULL).  Allocates the grids and the
 * FFT plans and tabulates B(m) C(m) for the context's box; synchronises the
 * stream; not capturable.  Once enabled, nb_forces adds the reciprocal-space
 * forces and the corrections to d_F, E_recip + E_self + the pair corrections
 * to the Coulomb energy and their virial to d_virial.
 * Errors: NB_ERR_INVALID_ARG (grid out of range, flags != 0),
 * NB_ERR_UNSUPPORTED (batch context, alpha = 0, order not 4/6/8),
 * NB_ERR_OOM, NB_ERR_CUDA (also for an FFT plan failure). */
nb_status nb_set_pme(nb_ctx *ctx, const nb_pme_params *p);

/* nb_pme_forces - the long-range part alone, for the positions of the last
 * nb_build_cells (NB_ERR_LIST_STALE is recorded otherwise):
 *   d_pos [N, 3] coordinates, d_q [N] charges;
 *   d_F [N, 3] output: reciprocal-space forces plus the corrections' forces;
 *   d_energy [3] output (E_recip, E_self, E_excl) or NULL;
 *   d_virial [6] output (reciprocal + corrections) or NULL.
 * Asynchronous.  NB_ERR_NOT_BUILT when PME is not enabled or no build
 * preceded the call. */
nb_status nb_pme_forces(nb_ctx *ctx, const float *d_pos, const float *d_q, float *d_F, double *d_energy,
                        double *d_virial);

/* Molecular dynamics around the non-bonded path (section "Molecular dynamics
 * on the GPU": bonded terms, velocity-Verlet integration, Langevin
 * thermostat, M-SHAKE and RATTLE constraints; section "Performance": the
 * DHFR step).  Functional forms (the paper names the terms but prints no
 * formula):
 *   bond     U = k (r - r0)^2;
 *   angle    U = k (theta - theta0)^2, theta at the middle atom;
 *   dihedral U = k (1 + cos(n phi - delta)), IUPAC phi =
 *            atan2(|b2| b1 . (b2 x b3), (b1 x b2) . (b2 x b3)),
 *            b1 = x_j - x_i, b2 = x_k - x_j, b3 = x_l - x_k (minimum images);
 *   rigid 3-site waters (O, H1, H2): |O-H| = water_roh, |H-H| = water_rhh.
 * One step of length dt (ps), Langevin velocity Verlet with constraints:
 *   v <- c v + sqrt((1 - c^2) kT / m) xi, c = exp(-gamma dt / 2);
 *   v <- v + dt/2 F/m;  x' = x + dt v;  M-SHAKE on every water (Newton
 *   iterations on the three distance equations along the bond vectors of
 *   x, at most shake_max_iter, until every |r^2 - d^2| / d^2 <
 *   shake_tolerance; NB_ERR_TIMEOUT is recorded otherwise) with the velocity
 *   changed by the constraint displacement / dt;  F = forces(x'') (cell
 *   list + short-range + PME when enabled + bonded);  v <- v + dt/2 F/m;
 *   v <- c v + sqrt((1 - c^2) kT / m) xi';  RATTLE on every water.
 * xi: Philox4x32-10 on the counter (atom, step, stream 0 or 1, 0) with the
 * key (seed low, seed high), 24-bit uniforms, Box-Muller.  Units kcal/mol,
 * A, amu, ps (F/m times 418.4 is A/ps^2), K. */
typedef struct {
    const float *mass;           /* host [N] atomic masses (amu), > 0 */
    int32_t n_bonds;
    const int32_t *bonds;        /* host [n_bonds*2] */
    const float *bond_k;         /* [n_bonds] kcal/mol/A^2 */
    const float *bond_r0;        /* [n_bonds] A */
    int32_t n_angles;
    const int32_t *angles;       /* host [n_angles*3], middle atom at the vertex */
    const float *angle_k;        /* kcal/mol/rad^2 */
    const float *angle_theta0;   /* rad */
    int32_t n_dihedrals;
    const int32_t *dihedrals;    /* host [n_dihedrals*4] */
    const float *dihedral_k;     /* kcal/mol */
    const int32_t *dihedral_n;   /* multiplicity */
    const float *dihedral_phase; /* rad */
    int32_t n_waters;
    const int32_t *waters;       /* host [n_waters*3] (O, H1, H2), each atom in one water at most */
    float water_roh, water_rhh;  /* constraint lengths (A) */
    float dt;                    /* time step (ps), > 0 */
    float gamma;                 /* friction (1/ps); 0 = NVE velocity Verlet */
    float temperature;           /* K */
    uint64_t seed;               /* Philox key */
    int32_t shake_max_iter;      /* >= 1 */
    float shake_tolerance;       /* > 0, relative */
    uint32_t flags;              /* reserved, must be 0 */
} nb_md_params;

/* nb_md_init - attach an MD state to a single-system context (copies the
 * topology; synchronises the stream; not capturable).  The step counter of
 * the noise starts at 0.  Errors: NB_ERR_INVALID_ARG (indices out of range,
 * non-positive masses, an atom in two waters, ...), NB_ERR_UNSUPPORTED
 * (batch context), NB_ERR_OOM, NB_ERR_CUDA. */
nb_status nb_md_init(nb_ctx *ctx, const nb_md_params *p);

/* nb_md_step - advance d_pos [N,3] and d_vel [N,3] (FP32, A and A/ps,
 * updated in place; positions are kept wrapped into the box) by n_steps
 * steps with charges d_q and types d_type.  The first call after
 * nb_md_init evaluates the forces at the starting positions; later calls
 * reuse those of the previous step, so between calls the positions must
 * change only through nb_md_step.  d_energy [6] (E_LJ, E_Coul (with PME
 * when enabled), E_bond, E_angle, E_dihedral, E_kin; kcal/mol) receives
 * the energies after the last step, or NULL.  Asynchronous, capturable
 * (a device counter numbers the steps, so graph replays draw new noise).
 * NB_ERR_NOT_BUILT without nb_md_init. */
nb_status nb_md_step(nb_ctx *ctx, float *d_pos, float *d_vel, const float *d_q, const int32_t *d_type,
                     int32_t n_steps, double *d_energy);

/* nb_md_minimize - energy minimisation of d_pos [N,3] (FP32, A, updated in
 * place and kept wrapped) with charges d_q and types d_type before MD: n_steps
 * steps of steepest descent in mass-weighted coordinates,
 *   x_i <- x_i + h F_i / m_i,  h = max_disp / max_j (|F_j| / m_j),
 * with F the total forces of nb_md_step at x (cell list, short-range, PME
 * when enabled, bonded terms) and the rigid waters restored by M-SHAKE from
 * x after every move; the atom with the largest |F| / m moves by max_disp (A)
 * before the constraints.  The forces are evaluated once more at the final
 * positions and kept for the next nb_md_step; d_energy [6] receives the
 * energies there (E_LJ, E_Coul, E_bond, E_angle, E_dihedral, 0), or NULL.
 * Velocities are not touched.  Asynchronous, capturable.  The paper prints
 * no minimiser: this is the plain capped steepest descent that prepares a
 * synthetic start for the dynamics.  Errors: NB_ERR_INVALID_ARG (n_steps <
 * 0, max_disp not positive and finite), NB_ERR_NOT_BUILT without nb_md_init;
 * NB_ERR_TIMEOUT is recorded when M-SHAKE does not converge. */
nb_status nb_md_minimize(nb_ctx *ctx, float *d_pos, const float *d_q, const int32_t *d_type, int32_t n_steps,
                         float max_disp, double *d_energy);

/* nb_bonded_forces - the bonded terms alone at d_pos: d_F [N,3] forces,
 * d_energy [3] (bond, angle, dihedral) or NULL.  FP32 terms, forces summed
 * in 64-bit fixed point (2^32).  NB_ERR_NOT_BUILT without nb_md_init. */
nb_status nb_bonded_forces(nb_ctx *ctx, const float *d_pos, float *d_F, double *d_energy);

/* nb_md_set_step - set the device step counter (synchronises the stream). */
nb_status nb_md_set_step(nb_ctx *ctx, uint64_t step);

/* nb_fp32_peak_launch - measurement utility without a counterpart in the
 * paper: launches an FP32 FMA throughput kernel on the current device (every
 * SM busy with independent chains of dependent FMAs, iters iterations per
 * chain; iters a positive multiple of 16) on cuda_stream, and returns in
 * *flop the FLOP it performs (2 per FMA).  The caller times it with CUDA
 * events: FLOP / time is the measured FP32 peak that the force kernel's
 * roofline is reported against.  d_sink: one writable device float.
 * Asynchronous. */
nb_status nb_fp32_peak_launch(int64_t iters, void *cuda_stream, float *d_sink, double *flop);

/* nb_status_string - static description of a status code. */
const char *nb_status_string(nb_status s);

#ifdef __cplusplus
}
#endif

#endif /* ACENB_H */
