// Internal declarations shared by the translation units of libwick.
// Device code never crosses translation units (no relocatable device code):
// each kernel lives in one .cu file and is reached through a host launcher
// declared here.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/wick.h"

namespace wick {

constexpr int kMaxOps = 4;       // block types per layout
constexpr int kMaxX = 48;        // distinct diquark lists over all ops
constexpr int kMaxXTerms = 512;  // (row2, row3, weight) entries over all lists
constexpr int kMaxOsTerms = 256; // (row1, list) entries over all (op, spin)
constexpr int kMaxSpin = 4;
constexpr int kMaxA = 8;

// ---------------------------------------------------------------------------
// Block-build plan.  A nucleon table sum_e w_e S1(r1_e,c1) S1(r2_e,c2) S2(r3_e,c3)
// is regrouped as   P_{op,s}(c1,c2,c3) = sum_{(r1, l) in OS(op,s)} S1(r1,c1) X_l(c2,c3),
//                   X_l(c2,c3)         = sum_{(r2, r3, w) in list l} w S1(r2,c2) S2(r3,c3)
// where equal lists are shared between spins (for the nucleon operators of
// Eqs. 1000/1001 the list depends on the colour of slot 1 only).  Rows are
// stored compactly: row index r -> position in rows[flavour].
// ---------------------------------------------------------------------------
struct BlockPlan {
    int n_ops, n_spin, n_chi;
    int n_out;                 // n_ops * n_spin * n_chi^3
    int chi[12];
    int f1[kMaxOps];           // pair flavour of each op
    int n_rows[2];             // rows of S used per flavour
    int8_t rows[2][12];
    int n_x;                   // diquark lists
    int x_op[kMaxX];
    int x_off[kMaxX + 1];      // into xt_*
    int8_t xt_r2[kMaxXTerms];  // compact row of S_{f1(op)}
    int8_t xt_r3[kMaxXTerms];  // compact row of S_{f2(op)}
    float xt_w[kMaxXTerms];    // integer weights (exact in float)
    int pow2_w;                // every diquark weight is +-2^k (exact scaling of a float)
    int os_off[kMaxOps * kMaxSpin + 1];
    int8_t os_r1[kMaxOsTerms]; // compact row of S_{f1(op)}
    int16_t os_x[kMaxOsTerms];
};

int build_block_plan(const wick_nucleon_op *ops, const wick_block_layout *layout, BlockPlan *plan);

// launchers (blocks.cu): the block build of one configuration.  partials: block_partial_bytes;
// counters: block_counter_bytes (the tensor-core path; zero before its first use, cleared again by
// every launch; a region that holds nothing else)
int launch_block_build(const BlockPlan &plan, const void *Su, int dtype_u, const void *Sd, int dtype_d,
                       int V, int n_slices, int precision, int range_sites, int *counters, void *partials,
                       double2 *blocks, cudaStream_t stream);
size_t block_partial_bytes(const BlockPlan &plan, int V, int n_slices, int precision, int range_sites);
// three-point blocks: the derivative of the blocks in the direction of the sequential propagator Sg of
// flavour sub_flav (each quark line of that flavour replaced by Sg in turn), on the CUDA cores (FP64 or
// double-FP32); partials: block_3pt_partial_bytes
size_t block_3pt_partial_bytes(const BlockPlan &plan, int V, int n_slices);
int launch_block_build_3pt(const BlockPlan &plan, const void *Su, const void *Sd, const void *Sg, int dtype,
                           int sub_flav, int V, int n_slices, int precision, void *partials, double2 *dblocks,
                           cudaStream_t stream);
size_t block_counter_bytes(const BlockPlan &plan, int n_slices, int precision);
// tensor-core update stage (blocks_tc.cu): upper-spin plans, double-FP32-exact
// the 16-byte words of one site that wick_upload_rows gathers: flavour << 15 | word in the site
constexpr int kMaxUploadWords = 2 * 12 * 12;   // both flavours, all rows, complex128
struct UploadMap {
    int n;
    uint16_t word[kMaxUploadWords];
};
int launch_upload_rows(const UploadMap &map, const void *hu, const void *hd, const void *du, const void *dd,
                       size_t n_sites, int words_u, int words_d, cudaStream_t stream);
bool tc_applicable(const BlockPlan &plan);
// derivative blocks on the tensor cores: the rows of both flavours and of the sequential propagator fit
bool tc_applicable_3pt(const BlockPlan &plan, int sub);
int block_build_launches(const BlockPlan &plan, int precision);  // kernels one launch_block_build issues
// tensor-core block build (blocks_tc.cu): one launch for up to tc_max_configs() configurations; its
// scratch holds one counter per (configuration, slice, block type) -- zero before the first launch,
// cleared again by every launch -- and the FP64 partials of every site range
int tc_range_sites(int requested);               // the range size a request (0 = default) resolves to
// the same for a launch of n_cfg configurations of n_slices slices and V sites (n_pass: 3 for derivative
// blocks); callers that size scratch for one shape and launch smaller ones pass its result on
int tc_range_for(const BlockPlan &plan, int requested, int n_pass, int n_cfg, int n_slices, int V);
int tc_max_configs();
size_t tc_counter_bytes(const BlockPlan &plan, int n_slices, int n_cfg);
size_t tc_partial_bytes(const BlockPlan &plan, int V, int n_slices, int n_cfg, int range_sites, int n_pass = 1);
// Sg, sub >= 0: the derivative blocks in the direction of the sequential propagators Sg of flavour sub
// (three role passes; partials: tc_partial_bytes with n_pass = 3)
int launch_block_tc(const BlockPlan &plan, const void *const *Su, const void *const *Sd, int n_cfg, int dtype, int V,
                    int n_slices, int range_sites, int *counters, double2 *partials, double2 *blocks, int *status,
                    cudaStream_t stream, const void *const *Sg = nullptr, int sub = -1);

// ---------------------------------------------------------------------------
// Term reduction (dedup.cu)
// ---------------------------------------------------------------------------
struct EnumPlan {
    int A, nq, nu, nd;
    int n_sink, n_M;           // sink terms, antisymmetrised source multisets
    int64_t fu, fd;            // n_u!, n_d!
    int64_t n_raw;             // n_sink * n_M * n_u! * n_d!
    int ju[24], jd[24];        // source positions of u / d quarks
    int n_spin, n_chi, n_blk;
};

struct ReduceResult {
    int64_t U, n_zero, n_keys;
    uint16_t *d_ids;  // [U][A]
    int64_t *d_w;     // [U]
    int64_t *d_rep;   // [U]
};

// Antisymmetrised source (host-prepared): n_M multisets, each the sorted
// layout indices of its u quarks (Mu, n_M x nu) and d quarks (Md, n_M x nd),
// with the summed signed source weight CM.
// identity-testing keys (two values mod p, canonical sign eps; eps = 0 for a zero key) of given terms
// (device ids [U][A]) with the block values mod p of run_reduce for the same seed, trials and sites
int term_keys(const BlockPlan &bp, int n_blk, const uint16_t *ids, int64_t U, int A, uint64_t seed, int trials,
              int sites, uint64_t *keys, int8_t *eps, cudaStream_t stream);
int run_reduce(const EnumPlan &ep, const BlockPlan &bp, const wick_nucleus *nuc, const int8_t *Mu,
               const int8_t *Md, const int64_t *CM, const int8_t *sink_flav, const int8_t *sink_ord,
               const int8_t *sink_eta, uint64_t seed, int trials, int sites, ReduceResult *out,
               cudaStream_t stream);

// ---------------------------------------------------------------------------
// Contraction (contract.cu): one persistent launch over (configuration,
// slice, table, chunk of terms) work items
// ---------------------------------------------------------------------------
constexpr int kMaxTables = 8;
struct ContractTable {         // a reduced table as the contraction reads it
    const uint16_t *ids;       // [U][AP] block ids padded to AP = 4 (A <= 4) or 8
    const double *w;           // [U][n_el] weights as doubles (exact: |w| < 2^53)
    int64_t U;
    int A;
    double scale;
    const double *el_scale = nullptr;   // matrix tables: scale of each of the n_el elements (host)
    const float2 *wf = nullptr;         // [U][n_el] the weights as exact float pairs (hi, lo) (MIXED)
};
struct ContractTune {          // 0 = default
    int threads;               // per CTA: 32..512, multiple of 32 (default 256)
    int ctas_per_sm;           // resident CTAs per SM (default: as many as fit)
    int chunk_terms;           // terms per work item, about (default 4096)
};
struct ContractPlan {
    int kind;                  // 0 correlator, 1 three-point (derivative blocks), 4 / 9 / 16 matrix elements
    int threads, grid, stage;
    size_t smem;
    int n_chunks[kMaxTables], item_off[kMaxTables];
    int64_t chunk[kMaxTables];
    int items_per_cs;
    int64_t n_items;
    size_t counters;           // (configuration, table, slice) counters
    size_t counter_bytes;      // the item counters and the counters: zero before the first launch
    size_t partial_bytes;      // one complex128 per work item
    size_t convert_bytes;      // MIXED without staging: the blocks (and derivative blocks) as float pairs
};
int contract_plan(int n_blk, int n_cfg, int n_slices, const ContractTable *tabs, int n_tab, int precision,
                  const ContractTune &tune, int64_t max_items, ContractPlan *plan, int kind = 0);
// counters: plan.counter_bytes, zero before the first launch (cleared again by every launch; a region
// that holds nothing else); partials: plan.partial_bytes; convert: plan.convert_bytes (or null: the MIXED
// gathers then convert each block entry as they load it)
int launch_contract(const double2 *blocks, int n_blk, int n_cfg, int n_slices, const ContractTable *tabs, int n_tab,
                    int precision, const ContractPlan &plan, void *counters, double2 *partials, double2 *C_out,
                    cudaStream_t stream, const double2 *dblocks = nullptr, void *convert = nullptr);
int pad_table(const uint16_t *ids, const int64_t *w, int64_t U, int A, uint16_t *ids_pad, double *wd,
              cudaStream_t stream);
// wf[i] = the weight wd[i] as a pair of floats hi + lo (exact for |wd| < 2^48)
int split_weights(const double *wd, int64_t n, float2 *wf, cudaStream_t stream);
// per-term contribution magnitudes on n_slices slices of blocks (device, mag: U doubles)
int launch_magnitudes(const double2 *blocks, int n_blk, int n_slices, const ContractTable &tab, double *mag,
                      cudaStream_t stream);
// fixed scratch of wick_contract_noalloc (per device): the item counters and 65,536 counters, then
// 65,536 partials at a fixed offset
constexpr int64_t kNoAllocItems = 65536;
constexpr size_t kNoAllocCounterBytes = 256 + sizeof(int) * kNoAllocItems;
constexpr size_t kNoAllocBytes = kNoAllocCounterBytes + 16 * kNoAllocItems;
int noalloc_scratch(void **ptr, size_t *bytes);

// ---------------------------------------------------------------------------
// library workspace, tables and tuning (api.cu)
// ---------------------------------------------------------------------------
int terms_table(const wick_terms *t, ContractTable *tab, int *n_blk);
wick_tuning current_tuning();
ContractTune contract_tune(const wick_tuning &t);
// per-device cached scratch, zeroed when (re)allocated: 0 = block partials, 1 = contraction partials,
// 2 = determinant scratch, 3 = block-build counters, 4 = contraction counters (the counter slots hold
// nothing but counters, which every launch leaves at zero), 5 = blocks converted for the contraction
constexpr int kWsBlockPartials = 0, kWsContractPartials = 1, kWsDet = 2, kWsBlockCounters = 3,
              kWsContractCounters = 4, kWsContractConvert = 5, kWsSlots = 6;
void *workspace(int slot, size_t bytes, int *err);
// every device allocation of the library: cudaMalloc, or WICK_ENOMEM injected by wick_inject_alloc_failure
int dev_malloc(void **ptr, size_t bytes);
// bounded-wait self tests (dedup.cu: hash-slot wait; blocks_tc.cu: mbarrier wait); status: device word
int selftest_hash_wait(int limit, int *status, cudaStream_t stream);
int selftest_mbar_wait(int limit, int *status, cudaStream_t stream);
int *status_word(int *err);                     // per-device status word
int status_read_clear(cudaStream_t stream);

}  // namespace wick

#define WICK_CUDA_TRY(expr)                                  \
    do {                                                     \
        cudaError_t e__ = (expr);                            \
        if (e__ != cudaSuccess) {                            \
            (void)cudaGetLastError();                        \
            return e__ == cudaErrorMemoryAllocation ? WICK_ENOMEM : WICK_ECUDA; \
        }                                                    \
    } while (0)
