/*
 * wick.h -- C ABI of libwick, the GB300 (sm_103a) library for zero-momentum
 * nuclear two-point correlators with a plane-wave sink (the block algorithm
 * of arXiv:2411.08962).
 *
 * The hot path has three calls:
 *
 *   wick_build_blocks  baryon blocks from u/d propagators            (Eq. 2.4/2.5)
 *   wick_reduce_terms  randomised redundancy elimination of the Wick
 *                      terms by identity testing modulo 2^61 - 1    (Sec. III.B, App. C)
 *   wick_contract      signed gather-multiply-sum of the reduced
 *                      terms over the blocks, for every time slice   (Eq. 2.6, App. D)
 *
 * Conventions common to every call
 *   - Device buffers are allocated and owned by the caller (for example as
 *     torch tensors) and must stay alive until the stream work completes.
 *     Only wick_terms objects are owned by the library (wick_terms_free).
 *   - Every call is asynchronous on the given stream (NULL = legacy default
 *     stream) unless its comment says it synchronises.
 *   - Return value: WICK_OK (0) or a negative WICK_E* code; no exception or
 *     C++ type crosses the ABI.  wick_strerror() names a code.  Errors a
 *     kernel detects on the device (capacity, overflow, bounded waits that
 *     ran out) are recorded in a device status word and returned by the next
 *     call that synchronises (wick_reduce_terms, wick_status).
 *   - Combined colour-spin index: chi = 4 * colour + spin, colour in 0..2,
 *     spin in 0..3 (Dirac-Pauli basis; spins 0,1 are the upper components).
 *   - Complex numbers are stored as interleaved (re, im) pairs.
 */
#ifndef WICK_H
#define WICK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define WICK_OK 0
#define WICK_EINVAL (-1)    /* bad argument, shape or table */
#define WICK_ENOMEM (-2)    /* device or host allocation failed */
#define WICK_ECUDA (-3)     /* a CUDA runtime call or kernel launch failed */
#define WICK_ECAPACITY (-4) /* a library table (term hash table) is full */
#define WICK_EOVERFLOW (-5) /* an integer weight or count does not fit */
#define WICK_ETIMEOUT (-6)  /* a bounded device-side wait ran out */
#define WICK_EIO (-7)       /* term-table file missing, truncated or corrupt */
#define WICK_ESCRATCH (-8)  /* request larger than the fixed scratch of wick_contract_noalloc */

/* storage type of a propagator */
#define WICK_C128 0 /* complex double */
#define WICK_C64 1  /* complex float  */

/* arithmetic of a call */
#define WICK_FP64 0  /* FP64 products and sums */
#define WICK_MIXED 1 /* double-FP32 products on the float pipes, FP64 sums over site chunks and terms */
#define WICK_MIXED_SIMT 2 /* wick_build_blocks only: WICK_MIXED without the tensor-core update stage */

/* quark flavours */
#define WICK_U 0
#define WICK_D 1

typedef struct CUstream_st *wick_stream_t; /* a cudaStream_t */

/*
 * Quark propagator S_q(x, t; x0, 0) for every source, time slice and sink
 * site, S^{ab}_{alpha beta} with sink colour a / spin alpha first (the layout
 * the paper reads, App. A):
 *   data[src][t][x][a][alpha][b][beta], x = (z * L + y) * L + x_  (V = L^3),
 * complex, device memory, 16-byte aligned, caller-owned.
 */
typedef struct wick_prop {
    const void *data;
    int L, T, n_src;
    int dtype; /* WICK_C128 | WICK_C64 */
} wick_prop;

/*
 * Nucleon interpolating operator as an integer weight table (Eq. 2.7
 * restricted to three quarks; Eqs. 1000/1001 for p and n):
 *   N_s = sum_e w_e q1(chi_e1) q1(chi_e2) q2(chi_e3)      (over e with s_e = s)
 * entries[e] = (s, chi_e1, chi_e2, chi_e3), int8 x 4; w[e] int32.
 * Slots 1 and 2 carry the like-flavour pair flav_pair (WICK_U for the proton),
 * slot 3 the other flavour.  Host memory, read during the call only.
 */
typedef struct wick_nucleon_op {
    int n_entries;
    const int8_t *entries;
    const int32_t *w;
    int flav_pair;
} wick_nucleon_op;

/*
 * Which blocks exist and where they live.  Block entry (op, s, i1, i2, i3),
 * i = position of the source index chi' in chi[], has id
 *   id = (((op * n_spin + s) * n_chi + i1) * n_chi + i2) * n_chi + i3
 * and a block buffer holds, per (src, t), wick_block_count() complex128
 * values B[src][t][id].
 */
typedef struct wick_block_layout {
    int n_ops;      /* number of block types (nucleon operators) */
    int n_spin;     /* nucleon spin labels s = 0 .. n_spin-1 */
    int n_chi;      /* number of source indices kept, 1..12 */
    int8_t chi[12]; /* the kept source indices chi', strictly ascending */
} wick_block_layout;

/*
 * Nucleus operator at sink and source (Eq. 2.7, Sec. III.C):
 *   sink:   sum_i sink_w[i] prod_k N^{sink_type[i][k]}_{sink_spin[i][k]}
 *   source: sum_m src_w[m] prod_q qbar_{src_flav[q]}(src_chi[m][q]),
 *           q = 3k + slot lists the 3A source quarks nucleon by nucleon.
 * All arrays are host memory, row-major, read during the call only.
 * The correlator is scale * sum of the Wick terms (all weights integers).
 */
typedef struct wick_nucleus {
    int A;                    /* nucleons, 1..8 */
    int n_sink;
    const int8_t *sink_type;  /* n_sink x A, index into the op list */
    const int8_t *sink_spin;  /* n_sink x A */
    const int64_t *sink_w;    /* n_sink */
    int n_src;
    const int8_t *src_chi;    /* n_src x 3A, chi' in 0..11 (must be in layout.chi) */
    const int64_t *src_w;     /* n_src */
    const int8_t *src_flav;   /* 3A, WICK_U / WICK_D */
    double scale;
} wick_nucleus;

/* Reduced term table, library-owned (host and device copies). */
typedef struct wick_terms wick_terms;

/* Number of block entries per (src, t) of a layout; 0 if the layout is invalid. */
size_t wick_block_count(const wick_block_layout *layout);

/*
 * Baryon blocks, Eq. 2.4/2.5 generalised to any nucleon weight table and
 * projected to zero momentum (sum over sink sites x, plane-wave sink):
 *   B^op_s(c1,c2,c3)[src][t] = sum_x sum_e w_e [ S1(x)(chi_e1,c1) S1(x)(chi_e2,c2)
 *                                               - S1(x)(chi_e1,c2) S1(x)(chi_e2,c1) ] S2(x)(chi_e3,c3)
 * with S1 the propagator of the op's pair flavour and S2 the other one; the
 * bracket is the exchange of the two like-flavour source quarks (Eq. 2.4
 * writes the same exchange on the sink side).
 *   Su, Sd      propagators (same L, T, n_src; dtype may differ)
 *   ops         layout->n_ops nucleon operators
 *   precision   WICK_FP64: FP64 throughout.  WICK_MIXED: double-FP32 on the float
 *               pipes -- products of the float propagator entries formed exactly
 *               with FMA, sums as float pairs (about 44 significant bits) over a
 *               chunk of at most 256 sites -- and an FP64 sum of the chunks.
 *               C128 input is rounded to float first under WICK_MIXED.  For the
 *               upper- and full-spin tables with +-2^k weights the update sum
 *               over sites runs on the tensor cores (tcgen05, bf16) as an exact
 *               sliced product: U in 5 and the double-FP32 diquark values in 6
 *               fixed-point slices of 8 bits, slice pairs i + j <= 5, every
 *               128-site sum exact in FP32, rounds combined in double-FP32 (same
 *               accuracy class).  When the tables hold a proton-like and a
 *               neutron-like type whose diquark lists are each other's with the
 *               two rows exchanged (the nucleon operators of Eqs. 1000/1001), one
 *               CTA builds both types from one computation of the diquark values
 *               (wick_tuning.no_pair_kernel = 1 builds one type per CTA instead).
 *               WICK_MIXED_SIMT requests the CUDA-core double-FP32 kernel.
 *   blocks      device, caller-owned, complex128 [n_src][T][wick_block_count]
 * Uses a library-cached device workspace for the per-chunk FP64 partials
 * (allocated on first use and grown when needed: make the first call, with
 * the largest shape, before any stream capture).
 * Errors: WICK_EINVAL (shapes, tables, indices), WICK_ENOMEM, WICK_ECUDA.
 */
int wick_build_blocks(const wick_prop *Su, const wick_prop *Sd, const wick_nucleon_op *ops,
                      const wick_block_layout *layout, int precision, void *blocks,
                      wick_stream_t stream);

/*
 * Upload of the propagator rows a block build reads.  Eq. 2.4/2.5 take
 * S(x)(chi, c) only at the sink indices chi that the nucleon tables use (for
 * the upper-spin tables the six rows (a, alpha), alpha in {0, 1}: half of S),
 * so only those rows cross the host link.
 *   Su_host, Sd_host  page-locked host memory (cudaHostAlloc / cudaHostRegister),
 *                     the wick_prop layout; read after the call returns, so keep
 *                     them alive until `stream` reaches this point
 *   Su_dev, Sd_dev    device propagators of the same shape and dtype; the rows the
 *                     tables do not read are left as they are
 *   ops, layout       the tables of the wick_build_blocks call that follows
 *   mode              WICK_UPLOAD_KERNEL: a gather kernel reads the rows from the
 *                     device-mapped host buffers (16-byte words, one warp per site;
 *                     WICK_EINVAL when the host memory is not mapped);
 *                     WICK_UPLOAD_DMA: one pitched copy (cudaMemcpy2DAsync) per run of
 *                     consecutive rows and flavour, on the copy engines;
 *                     WICK_UPLOAD_AUTO: DMA (the kernel is faster on an idle GPU, 205
 *                     against 170 GB/s on a GB300's host link, but takes SM slots from a
 *                     block build that runs beside it)
 *   bytes             out, may be NULL: the bytes copied (both flavours)
 * Everything is enqueued on `stream`.
 * Errors: WICK_EINVAL (shapes or dtypes differ, invalid tables or mode, host memory
 * not page-locked, device pointer not 16-byte aligned), WICK_ECUDA.
 */
#define WICK_UPLOAD_AUTO 0
#define WICK_UPLOAD_DMA 1
#define WICK_UPLOAD_KERNEL 2
int wick_upload_rows(const wick_prop *Su_host, const wick_prop *Sd_host, const wick_prop *Su_dev,
                     const wick_prop *Sd_dev, const wick_nucleon_op *ops, const wick_block_layout *layout,
                     int mode, size_t *bytes, wick_stream_t stream);

/*
 * Randomised minimal-set search (Sec. III.B "Computation of non-redundant
 * minimal set", Theorem 1 and its error bound in App. C) for the block
 * form of the correlator (Eq. 2.6 generalised in App. D):
 *   source      first antisymmetrised (method B of Sec. III.C): a source tuple
 *               whose u (or d) indices repeat cancels in the permutation sum;
 *               every other tuple is a signed reordering of its sorted multiset
 *               pair M, so the source becomes the nonzero multisets (listed in
 *               lexicographic order) with C'(M) = sum C'_m sgn(sort_u) sgn(sort_d).
 *   raw terms   j = ((i_sink * n_M + M) * n_u! + rank(tau_u)) * n_d! + rank(tau_d):
 *               the sink quark of flavour-ordinal q takes entry tau(q) of M's
 *               sorted list; coefficient c_j = sink_w * C'(M) * sgn(tau_u) *
 *               sgn(tau_d) * eta (eta = parity of the identity flavour pairing,
 *               +1 when the source lists quarks in the sink's flavour order);
 *               monomial prod_k B^{type_k}_{s_k}(entries of the nucleon's three quarks);
 *               rank = lexicographic rank of the permutation.
 *   hashing     every monomial is evaluated at `trials` (1 or 2) random integer
 *               propagators on `sites` lattice sites, exactly modulo p = 2^61 - 1;
 *               the sign is canonicalised (first non-zero value <= (p-1)/2) and
 *               the value tuple is the key.  Keys equal to zero drop the term.
 *   merging     equal keys are merged: W = sum_j eps_j c_j.  Classes with W = 0
 *               are dropped.  Each kept term stores its smallest raw index j
 *               (its representative), that term's block ids and the weight
 *               W * eps_rep / 2^A (an integer: classes are unions of the 2^A
 *               like-pair exchange orbits).  Terms are ordered by representative,
 *               so the table depends only on the partition, not on the seed.
 * False-merge probability <= C(N_raw, 2) * (3A / p)^trials, N_raw the raw terms
 * above (reported by wick_terms_stats).  Synchronises `stream`; the table is library-owned.
 * Errors: WICK_EINVAL, WICK_ENOMEM, WICK_ECUDA, WICK_ECAPACITY (more distinct
 * keys than the hash table holds), WICK_EOVERFLOW (weights beyond int64 /
 * more than 2^62 raw terms), WICK_ETIMEOUT.
 */
int wick_reduce_terms(const wick_nucleus *nucleus, const wick_nucleon_op *ops,
                      const wick_block_layout *layout, uint64_t seed, int trials, int sites,
                      wick_terms **out, wick_stream_t stream);

/* Accessors of a reduced table. */
int64_t wick_terms_count(const wick_terms *terms);     /* U, or a negative error */
int wick_terms_nucleons(const wick_terms *terms);      /* A */
/* Block entries per (src, t) of the layout the table was reduced for
 * (wick_block_count of that layout), or a negative error. */
int64_t wick_terms_block_count(const wick_terms *terms);
/* Copy to host arrays: ids [U][A] uint16, w [U] int64, rep [U] int64 (any may be NULL; not for
 * correlation-matrix tables: wick_terms_copy_matrix). */
int wick_terms_copy(const wick_terms *terms, uint16_t *ids, int64_t *w, int64_t *rep);
/* stats[0] raw terms, [1] identically zero, [2] distinct keys, [3] kept terms;
 * *bound = the false-merge probability bound of App. C for this reduction. */
int wick_terms_stats(const wick_terms *terms, int64_t stats[4], double *bound);
/* Keep only the first n terms in a caller-given order of importance: the
 * table is replaced by the terms perm[0..n-1] (indices into the current
 * table), re-sorted by representative.  Used for top-fraction evaluation. */
int wick_terms_select(wick_terms *terms, const int64_t *perm, int64_t n);
/*
 * Top-fraction evaluation (Sec. V.C: the terms of a table are spread around zero, a small
 * fraction of them with large values carries the correlator, and the same terms dominate on every
 * gauge configuration).
 * wick_terms_magnitudes: each term's share of the correlator on the given blocks,
 *   mag[u] = sum_{slice < n_slices} | scale * w_u * prod_k B[slice][id_{u,k}] |
 * (FP64; blocks: device complex128 [n_slices][n_blk], for example a few time slices of a small
 * lattice; mag: host, U doubles, written).  Synchronises `stream`.  Errors: WICK_EINVAL,
 * WICK_ENOMEM, WICK_ECUDA.
 * wick_terms_top: keeps the ceil(fraction * U) terms of largest mag (ties: the earlier term in the
 * table first), 0 < fraction <= 1, through wick_terms_select.  Errors: WICK_EINVAL.
 */
int wick_terms_magnitudes(const void *blocks, int n_slices, const wick_terms *terms, double *mag,
                          wick_stream_t stream);
int wick_terms_top(wick_terms *terms, const double *mag, double fraction);
/* Binary term-table file (versioned header + arrays). */
int wick_terms_save(const wick_terms *terms, const char *path);
int wick_terms_load(const char *path, wick_terms **out);
void wick_terms_free(wick_terms *terms);

/*
 * Correlator from the reduced table, Eq. 2.6 / App. D in reduced form:
 *   C[src][t] = scale * sum_u w_u prod_k B[src][t][id_{u,k}]
 *   blocks     device complex128 [n_src][T][n_blk], from wick_build_blocks with
 *              the layout the table was reduced for (n_blk = wick_terms_block_count)
 *   precision  WICK_FP64: FP64 products and sums.  WICK_MIXED: block entries
 *              split into float pairs, products in double-FP32 on the float
 *              pipes, FP64 sum over terms.
 *   C_out      device complex128 [n_src][T], caller-owned, overwritten ([N * N][n_src][T] for a
 *              correlation-matrix table of wick_reduce_terms_matrix).
 * One persistent kernel launch: CTAs take (slice, chunk of terms) work items
 * from a device counter; each slice's blocks are staged in shared memory; the
 * chunk sums are added in chunk order by the last chunk of a slice to finish.
 * Deterministic (fixed reduction order, whatever CTA takes which item).
 * Uses a library-cached device workspace (allocated and zeroed on first use
 * and when it grows: make the first call, with the largest shape, before any
 * stream capture); calls that overlap on the GPU share it and must be ordered.
 * Errors: WICK_EINVAL, WICK_ENOMEM, WICK_ECUDA.
 */
int wick_contract(const void *blocks, int n_src, int T, const wick_terms *terms, int precision,
                  void *C_out, wick_stream_t stream);

/*
 * Launch tuning, process-wide: read by every later call when it plans its
 * launches (wick_build_blocks, wick_contract, wick_batch_create); a batch keeps
 * the tuning it was created with.  0 in a field means the default.  The
 * package's autotuner (paper_2411_08962_gb300.autotune) times candidates on a
 * workload and records its choice as JSON.
 *   range_sites            tensor-core block build: sites per CTA and per FP64 partial,
 *                          a multiple of 128 up to 4096 (default 1024 for the proton/neutron
 *                          pair kernel and the full-spin tables when a launch has at least 8
 *                          waves of such CTAs, else 512).  The range size sets the order of
 *                          the site sums: a batch reproduces its single calls bit for bit when
 *                          both take the same size -- always with a size set here; with the
 *                          default a large batch may take 1024 where a single call takes 512,
 *                          and the blocks then agree to rounding (about 1e-12)
 *   contract_threads       contraction CTA size, a multiple of 32 up to 512 (default 256)
 *   contract_ctas_per_sm   resident contraction CTAs per SM (default: as many as fit)
 *   contract_chunk_terms   terms per contraction work item, about (64 or more; default 4096);
 *                          the chunking depends on a table's size and this value only, so the
 *                          contraction of a batch adds in the same order as its single calls
 *   hash_log2_start        wick_reduce_terms / wick_reduce_terms_matrix: log2 of the first hash
 *                          table's slots, 4..28 (default: from the raw-term count).  A table that
 *                          fills to 3/4 is dropped and the enumeration rerun with twice the slots
 *   hash_log2_max          log2 of the largest table tried, 4..28 (default 28); past it the
 *                          reduction fails with WICK_ECAPACITY
 *   no_pair_kernel         1: build one block type per CTA even when a proton/neutron pair of
 *                          types could share its diquark values (0, the default: share them)
 * NULL restores the defaults.  Errors: WICK_EINVAL (a field out of range).
 */
typedef struct wick_tuning {
    int range_sites;
    int contract_threads;
    int contract_ctas_per_sm;
    int contract_chunk_terms;
    int hash_log2_start;
    int hash_log2_max;
    int no_pair_kernel;
} wick_tuning;
int wick_set_tuning(const wick_tuning *tuning);
int wick_get_tuning(wick_tuning *tuning);

/*
 * Failure detection, driven from the host (no GPU fault is ever provoked).
 *
 * wick_inject_alloc_failure: the k-th device allocation the library makes from
 * now on (workspace, tables, batch scratch, reduction buffers; k >= 1) reports
 * failure without calling cudaMalloc, so that the error path of every
 * allocation point can be exercised: the call in progress frees what it took,
 * returns WICK_ENOMEM and leaves every object it was given as it was.  k = 0
 * cancels.  Returns the allocations that were still to go before the injected
 * failure (0: none pending), or WICK_EINVAL for k < 0.  Process-wide.
 *
 * wick_selftest_wait: runs one of the library's bounded device waits on a flag
 * that nothing sets, with a limit of `limit` polls (1 .. 2^22), in a one-thread
 * kernel on `stream`: which = 0 the wait on a hash-table slot claimed by another
 * thread (the reduction's insert), 1 the wait on an mbarrier phase (the
 * tensor-core block build's wait for its MMAs).  The wait gives up, the kernel
 * records WICK_ETIMEOUT in its status word and returns, and the context stays
 * usable.  Synchronises `stream`.  Returns that status (WICK_ETIMEOUT when the
 * wait ran out as designed), or WICK_EINVAL / WICK_ECUDA / WICK_ENOMEM.
 */
int wick_inject_alloc_failure(int k);
int wick_selftest_wait(int which, int limit, wick_stream_t stream);

/*
 * wick_contract without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- for
 * example an application whose caching allocator has already reserved the
 * device memory it is allowed to use, or a runtime that forbids driver-level
 * allocations (and the implicit device synchronisation of cudaMalloc/cudaFree)
 * once its set-up phase is over.  wick_contract itself allocates its scratch
 * on first use; this variant calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *
 * Same arguments, result and errors as wick_contract.  Its scratch (the work
 * counters and the FP64 partial sums, one complex128 per work item) is a fixed
 * array of 1,310,976 bytes (65,536 counters and 65,536 partials) that every GPU
 * loading the library holds until the process exits.  A call takes at most
 * 65,536 slices (n_src * T); larger requests fail with WICK_ESCRATCH before
 * anything is enqueued.  When the usual chunking would need more than 65,536
 * work items, longer term chunks are used (the sum order then differs from
 * wick_contract's within rounding).  Each call clears the counters it starts
 * from (cudaMemsetAsync on `stream`, no allocation) before its launch.
 *   - Every call looks up the array's device address for the current device
 *     (cudaGetSymbolAddress).  Under lazy module loading the first call on a
 *     device may make the driver load the library's device code, which
 *     reserves the array and the kernels in device memory: make that first
 *     call in the caller's set-up phase, before any stream capture.
 *   - Every call shares the one array and it keeps the last call's contents;
 *     each call writes every partial it reads, so nothing needs clearing, but
 *     calls that overlap on the GPU (concurrent streams, other host threads)
 *     race on it: order them.
 * Errors: as wick_contract, plus WICK_ESCRATCH.
 */
int wick_contract_noalloc(const void *blocks, int n_src, int T, const wick_terms *terms, int precision,
                          void *C_out, wick_stream_t stream);

/*
 * Three-point functions with the plane-wave sink (Sec. IV.A "Three-point functions", Eq.
 * Proton3pt_seq, generalised to nuclei): the connected contribution of a current on `flavour`
 * (WICK_U or WICK_D), inserted through the sequential propagator Sig (device, the wick_prop layout,
 * same L, T, n_src and dtype as Su, Sd; obtained by inverting the Dirac operator on the current's
 * source, an input here), replaces one quark line of that flavour in every Wick term by Sig, summed
 * over the lines.  In block form that is the derivative of the correlator in the direction Sig:
 *   C3[src][t] = scale * sum_u w_u sum_k D[src][t][id_{u,k}] prod_{j != k} B[src][t][id_{u,j}]
 * with D the derivative blocks, a third block type beside B^p and B^n:
 * wick_build_blocks_3pt writes D (device complex128, the block layout of wick_build_blocks): every
 * block with each of its quark lines of `flavour` replaced by Sig in turn (Eq. 2.4 differentiated;
 * the exchange term included).  FP64 on the CUDA cores, or WICK_MIXED: for the tables the mixed
 * wick_build_blocks runs on the tensor cores (when the rows of Su, Sd and Sig fit the staging, as for
 * the upper-spin tables) the same exact sliced update in three role passes -- the U rows, the
 * pair-flavour diquark rows and the other diquark rows taken from Sig where their flavour is
 * `flavour` -- summed per block; otherwise double-FP32 on the CUDA cores.  Uses the library
 * workspace; asynchronous.
 * wick_contract_3pt evaluates C3 from B (wick_build_blocks) and D with the reduced table of the
 * two-point function; C_out device complex128 [n_src][T].  One persistent launch; deterministic.
 * Errors: WICK_EINVAL (shapes, dtypes, flavour, precision), WICK_ENOMEM, WICK_ECUDA.
 */
int wick_build_blocks_3pt(const wick_prop *Su, const wick_prop *Sd, const wick_prop *Sig, int flavour,
                          const wick_nucleon_op *ops, const wick_block_layout *layout, int precision,
                          void *dblocks, wick_stream_t stream);
int wick_contract_3pt(const void *blocks, const void *dblocks, int n_src, int T, const wick_terms *terms,
                      int precision, void *C_out, wick_stream_t stream);

/*
 * Correlation matrix with the plane-wave sink (Sec. "Application ... to the generalized eigenvalue
 * problem", Eqs. E1-E3): for N = n_nuc operators O_i with the same quark content (nuclei[i]; their
 * sink and source halves), element (i, j) = i * N + j is the correlator with the sink of O_i and the
 * source of O_j, scale sqrt(scale_i * scale_j).  Every element is reduced as wick_reduce_terms does;
 * the terms of all elements are then merged by their identity-testing keys (the same evaluation mod
 * 2^61 - 1 at the same random points), so a block product shared by several elements is one term
 * with a weight per element.  The result is a table with N * N weight columns
 * (wick_terms_elements): wick_contract evaluates each product once and writes C_out device
 * complex128 [N * N][n_src][T].  2 <= N <= 4, A <= 4.  Matrix tables are for wick_contract (and the
 * accessors below) only: wick_terms_copy, _select, _top, _magnitudes, _save, wick_contract_noalloc
 * and batches return WICK_EINVAL for them.  Synchronises `stream`.
 * Errors: as wick_reduce_terms, WICK_EINVAL for operators of different quark content.
 */
int wick_reduce_terms_matrix(const wick_nucleus *nuclei, int n_nuc, const wick_nucleon_op *ops,
                             const wick_block_layout *layout, uint64_t seed, int trials, int sites,
                             wick_terms **out, wick_stream_t stream);
/* Number of weight columns (matrix elements) of a table: 1, or N * N for a correlation matrix. */
int wick_terms_elements(const wick_terms *terms);
/* Copy ids [U][A] uint16, weights [U][n_el] int64 and the element scales [n_el] (any may be NULL). */
int wick_terms_copy_matrix(const wick_terms *terms, uint16_t *ids, int64_t *w, double *el_scale);

/*
 * Cluster sink (Sec. V.A: Li-7 as a He-4 cluster and a triton cluster, each
 * projected to zero momentum on its own): with no quark exchanged between
 * clusters the correlator is the product of the cluster correlators,
 *   out[i] = Ca[i] * Cb[i]   (device complex128, n entries, asynchronous).
 * Errors: WICK_EINVAL, WICK_ECUDA.
 */
int wick_cluster_product(const void *Ca, const void *Cb, int64_t n, void *out, wick_stream_t stream);

/*
 * Batched executor (the paper evaluates one configuration at a time; this
 * batches many configurations and nuclei into one CUDA graph).
 * wick_batch_create captures, for n_cfg configurations resident in device
 * memory, the block build of each configuration followed by wick_contract of
 * every table in `tables` (all reduced for `layout`, so the nuclei share the
 * blocks), and instantiates the graph.  The batch owns its scratch; the
 * caller's buffers must stay valid for the batch's lifetime:
 *   Su, Sd    n_cfg propagator pairs (same L, T, n_src, dtype)
 *   blocks    device complex128 [n_cfg][n_src][T][n_blk] (written per run)
 *   C_out     device complex128 [n_cfg][n_tables][n_src][T]
 * wick_batch_run launches the whole batch on `stream` (asynchronous).
 * Errors: WICK_EINVAL, WICK_ENOMEM, WICK_ECUDA.
 */
typedef struct wick_batch wick_batch;
int wick_batch_create(const wick_prop *Su, const wick_prop *Sd, int n_cfg, const wick_nucleon_op *ops,
                      const wick_block_layout *layout, const wick_terms *const *tables, int n_tables,
                      int precision, void *blocks, void *C_out, wick_batch **out);
int wick_batch_run(wick_batch *batch, wick_stream_t stream);
int wick_batch_launches(const wick_batch *batch);   /* kernels per run */
void wick_batch_free(wick_batch *batch);

/*
 * Synthetic propagator (input generation; no counterpart in the paper, which
 * reads HISQ/overlap propagators): i.i.d. complex Gaussians with variance 1/2
 * per component from counter-based SplitMix64 and Box-Muller, one stream per
 * (seed, flavour, src), written as data[t][x][a][alpha][b][beta] of one source
 * (out: device, T * L^3 * 144 complex of `dtype`).  The same definition as the
 * Python package's host generator (values may differ in the last bits: the
 * device uses CUDA's log and sincospi).  Asynchronous.  Errors: WICK_EINVAL,
 * WICK_ECUDA.
 */
int wick_synth_propagator(uint64_t seed, int flavour, int src, int L, int T, int dtype, void *out,
                          wick_stream_t stream);

/*
 * Point-sink correlators by the determinant algorithm (Sec. III.A, Eq. 2.9;
 * Sec. III.C, improved method B; App. A, Eqs. a1-a4).  With every quark of
 * the sink operator at the same site x,
 *   G(t) = scale * sum_x sum_{M, M'} C[M] C'[M'] det M^u(x; M_u, M'_u) det M^d(x; M_d, M'_d),
 *   M^f_ij = S_f(x, t)(chi_i, chi'_j)   (row: sink index, column: source index),
 * with C, C' antisymmetrised within each flavour (M, M' are flavour-ordered
 * index lists), evaluated as
 *   G(t) = scale * sum_x sum_{(k, l)} Theta(k, l) det M^u(x; zeta_u[k]) det M^d(x; zeta_d[l])
 * over the minimal sets of distinct determinants (Eq. a1).
 *
 * wick_quark_operator: an operator sum_terms w * u(chi_1)..u(chi_nu) d(chi_nu+1)..d(chi_n)
 *   n_u, n_d   quarks of each flavour (0..6 each, at least one quark)
 *   chi        n_terms x (n_u + n_d) indices 4*colour + spin (0..11), u quarks first
 *              (any regrouping of the fields into this order has its sign in w)
 *   w          integer weights, |w| < 2^31
 * Host memory, read during the call.
 */
typedef struct {
    int n_u, n_d;
    int n_terms;
    const int8_t *chi;
    const int64_t *w;
} wick_quark_operator;

/*
 * wick_det_reduce: antisymmetrises sink and source within each flavour,
 * forms the determinant pairs of every (M, M'), finds the distinct
 * determinants by evaluating each candidate mod p = 2^61 - 1 at `trials`
 * random integer matrices derived from `seed` (the randomised identity
 * testing of Sec. III.B / App. C: equal value vectors are one determinant,
 * up to a sign made canonical; all-zero vectors drop their terms), and
 * merges the integer weights into Theta.  Runs on the current device;
 * *out is library-owned (wick_det_free).  Synchronous.
 * Errors: WICK_EINVAL (sizes, indices, weights), WICK_ENOMEM, WICK_ECUDA,
 * WICK_EOVERFLOW (a Theta weight reaches 2^53).
 */
typedef struct wick_det_plan wick_det_plan;
int wick_det_reduce(const wick_quark_operator *sink, const wick_quark_operator *source, uint64_t seed, int trials,
                    wick_det_plan **out);
/*
 * wick_det_reduce_matrix: the N x N correlation matrix C_ij(t) = <O_i(t) Obar_j(0)>
 * of N operators with the same quark content (Sec. "Application ... to the
 * generalized eigenvalue problem", Eqs. E1-E3): one identity testing over the
 * index sets of all operators, so the determinants are shared by every
 * element, and one Theta per element (i, j), element index i * N + j.
 * N * N <= 16.  Errors as wick_det_reduce.
 */
int wick_det_reduce_matrix(const wick_quark_operator *ops, int n_ops, uint64_t seed, int trials, wick_det_plan **out);
/* out[7]: sink terms, source terms (antisymmetrised, summed over operators), |zeta_u|, |zeta_d|,
 * Theta non-zeros (all elements), n_u * 8 + n_d, number of matrix elements */
int wick_det_stats(const wick_det_plan *plan, int64_t *out);
/* off[n_el + 1]: element e owns Theta entries [off[e], off[e + 1]) in wick_det_copy's order */
int wick_det_element_offsets(const wick_det_plan *plan, int64_t *off);
/* Copies Theta (k, l, weight) and the minimal sets to host arrays sized from
 * wick_det_stats (any pointer may be NULL): zu rows/cols [|zeta_u|][n_u],
 * zd rows/cols [|zeta_d|][n_d]. */
int wick_det_copy(const wick_det_plan *plan, int32_t *k, int32_t *l, int64_t *w, int8_t *zu_rows, int8_t *zu_cols,
                  int8_t *zd_rows, int8_t *zd_cols);
/*
 * wick_det_contract: G[src][t] for propagators Su, Sd (device, caller-owned,
 * complex64 or complex128) into C_out (device complex128 [n_el][n_src][T],
 * n_el = 1 for wick_det_reduce, N * N for a correlation matrix).
 * Asynchronous on `stream`; scratch from the library's per-device workspace.
 * Per site the kernel builds the table of all 2 x 2 minors of S_u(x), S_d(x)
 * and, for a flavour with 5 or 6 quarks, of all 3 x 3 minors, and expands
 * every determinant of the minimal sets over them (Laplace expansion).
 *   precision  WICK_FP64: FP64 throughout.  WICK_MIXED: the minor tables, the
 *              determinants and the Theta sum in double-FP32 on the float
 *              pipes (about 44 significant bits per operation; complex128
 *              input split into float pairs), the per-chunk sums in FP64.
 * Errors: WICK_EINVAL, WICK_ENOMEM, WICK_ECUDA.
 */
int wick_det_contract(const wick_prop *Su, const wick_prop *Sd, const wick_det_plan *plan, double scale,
                      int precision, void *C_out, wick_stream_t stream);
/*
 * wick_det_contract_3pt: three-point function (Sec. "Three-point functions",
 * Eq. Proton3pt_seq, generalised to nuclei) with the current on `flavour`
 * (WICK_U or WICK_D) inserted through the sequential propagator Sig (device,
 * same L, T, n_src, dtype and layout as S; obtained by inverting the Dirac
 * operator on the current's source, an input here).  The connected
 * contribution replaces one quark line of that flavour in every Wick term by
 * Sig, summed over the lines: each determinant of that flavour becomes the
 * sum of the determinants with one row taken from Sig (the derivative of
 * Eq. 2.9 in the direction Sig).  Same plan, output layout and errors as
 * wick_det_contract; WICK_MIXED needs at most 3 quarks of `flavour` (the
 * cofactor form of the derivative), else WICK_EINVAL.
 */
int wick_det_contract_3pt(const wick_prop *Su, const wick_prop *Sd, const wick_prop *Sig, int flavour,
                          const wick_det_plan *plan, double scale, int precision, void *C_out, wick_stream_t stream);
void wick_det_free(wick_det_plan *plan);

/* Synchronises `stream` and returns (then clears) the device status word. */
int wick_status(wick_stream_t stream);

/* Human-readable name of an error code (static string). */
const char *wick_strerror(int code);

/* Library version, e.g. "0.1.0". */
const char *wick_version(void);

#ifdef __cplusplus
}
#endif
#endif /* WICK_H */
