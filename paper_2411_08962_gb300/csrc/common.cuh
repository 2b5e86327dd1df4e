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

// launchers (blocks.cu)
int launch_block_build(const BlockPlan &plan, const void *Su, int dtype_u, const void *Sd, int dtype_d,
                       int V, int n_slices, int precision, double *partials, int n_splits, int chunk,
                       double2 *blocks, cudaStream_t stream);
size_t block_partials_bytes(const BlockPlan &plan, int V, int n_slices, int precision, int *n_splits,
                            int *chunk);
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
int block_build_launches(const BlockPlan &plan, int precision);  // kernels one launch_block_build issues
size_t tc_partials_bytes(const BlockPlan &plan, int V, int n_slices, int *n_splits, int *chunk);
int launch_block_tc(const BlockPlan &plan, const void *Su, const void *Sd, int dtype, int V, int n_slices,
                    double *partials, int n_splits, double2 *blocks, int *status, cudaStream_t stream);

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
int run_reduce(const EnumPlan &ep, const BlockPlan &bp, const wick_nucleus *nuc, const int8_t *Mu,
               const int8_t *Md, const int64_t *CM, const int8_t *sink_flav, const int8_t *sink_ord,
               const int8_t *sink_eta, uint64_t seed, int trials, int sites, ReduceResult *out,
               cudaStream_t stream);

// ---------------------------------------------------------------------------
// Contraction (contract.cu)
// ---------------------------------------------------------------------------
int launch_contract(const double2 *blocks, int n_slices, int n_blk, int A, int64_t U, const uint16_t *ids,
                    const int64_t *w, double scale, int precision, double2 *C_out, double *partials,
                    int n_chunks, cudaStream_t stream);
size_t contract_partials_bytes(int n_slices, int64_t U, int A, int n_blk, int *n_chunks);
// fixed scratch of wick_contract_noalloc (complex128 partials, per device)
constexpr size_t kNoAllocPartials = 65536;
int noalloc_partials(double2 **ptr, size_t *capacity);

// ---------------------------------------------------------------------------
// library workspace (api.cu)
// ---------------------------------------------------------------------------
// per-device cached scratch; slot 0 = block partials, slot 1 = contraction partials
void *workspace(int slot, size_t bytes, int *err);
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
