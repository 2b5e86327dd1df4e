// Correlator from the reduced term table (Eq. 2.6 generalised in App. D):
//   C[cfg][table][slice] = scale * sum_u w_u prod_k B[cfg][slice][id_{u,k}]
//
// One persistent launch evaluates any number of configurations and reduced
// tables (nuclei) that share a block layout.  The work is cut into items
// (configuration, slice, table, chunk of terms), ordered so that the items of
// one (configuration, slice) are adjacent; the CTAs (a fixed number per SM)
// take items from a device counter in that order.  For an item a CTA stages
// the slice's blocks in shared memory -- once per slice, kept while the next
// item is on the same slice -- (complex128 for FP64, a double-FP32 pair per
// value for MIXED), then every thread walks the chunk's terms with stride
// blockDim: one 8- or 16-byte load of the padded block ids (4 or 8 uint16),
// the A gathered block entries multiplied, the product accumulated in FP64
// with the weight.  The CTA sums its threads with warp shuffles and a fixed
// order over warps, and writes the item's partial.  The last item of a
// (configuration, table, slice) to finish -- an atomic count, no waiting --
// adds the chunk partials in chunk order and writes C.  Every sum has a fixed
// order, so the result is bitwise reproducible whichever CTA takes which item.
// Counters reset themselves: the last item of a slice clears its count and the
// last CTA to leave clears the item counter, so the scratch is ready for the
// next launch without a memset.
//
// MIXED keeps every block entry as a double-FP32 pair and forms the products
// with error-free float operations (about 44 bits) on the float pipes.  Each
// thread sums its terms' weighted products in double-FP32 too (the integer
// weights as exact float pairs) and adds that partial into its FP64 sum every
// kMixedGroup terms (correlators, three-point functions and matrices of up
// to 4 elements), so the FP64 pipe -- a small fraction of the float rate on
// this GPU -- sees two conversions and two additions per component per group
// instead of per term.  Block layouts too large to stage are converted to
// float pairs once per launch (convert_kernel) instead of at every gather.
#include <algorithm>

#include "common.cuh"
#include "df32.cuh"

namespace wick {

namespace {

constexpr int kMaxThreads = 512;
constexpr int64_t kDefaultChunkTerms = 4096;   // terms per work item unless tuned
constexpr size_t kSmemStageLimit = 96 * 1024;   // stage a slice's blocks in shared memory up to this size
constexpr int kMixedGroup = 16;                 // MIXED: terms per double-FP32 partial of a thread

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// A double as a double-FP32 pair with integer operations only (the FP64 pipe is narrow on this GPU):
// hi = v with its mantissa truncated to 24 significant bits, lo = the next 23 bits of v's mantissa, so
// |v - hi - lo| < 2^-46 |v|.  Values below 2^-126 in magnitude become zero, values at or above 2^128
// (and infinities, NaNs) an infinity of their sign.
__device__ __forceinline__ df split_double_bits(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const int e = (int)((hw >> 20) & 0x7FF);          // biased double exponent
    const unsigned sign = hw & 0x80000000u;
    const int ef = e - 1023 + 127;                     // biased float exponent of hi
    if (ef <= 0) return {__uint_as_float(sign), __uint_as_float(sign)};
    if (ef >= 255) return {__uint_as_float(sign | 0x7F800000u), 0.f};
    const float h = __uint_as_float(sign | ((unsigned)ef << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
    // the next 23 mantissa bits r (bits 28..6 of the low word) weigh 2^(e - 1023 - 52 + 6) each:
    // r is exact in a float by the 2^23 magic constant, then scaled by a power of two (zero if it underflows)
    const unsigned r = (lw >> 6) & 0x7FFFFFu;
    const float rf = __fsub_rn(__uint_as_float(0x4B000000u | r), 8388608.f);
    const int es = e - 1023 - 46 + 127;
    const float l = __fmul_rn(rf, es > 0 ? __uint_as_float((unsigned)es << 23) : 0.f);
    return {h, sign ? -l : l};
}

__device__ __forceinline__ cdf to_cdf(double2 v) { return {split_double_bits(v.x), split_double_bits(v.y)}; }

template <bool MIXED>
struct Elem;
template <>
struct Elem<true> {
    using T = cdf;
    static __device__ __forceinline__ T from(double2 v) { return to_cdf(v); }
    static __device__ __forceinline__ T mul(const T &a, const T &b) { return cdf_mul(a, b); }
    static __device__ __forceinline__ T add(const T &a, const T &b) { return {df_add(a.x, b.x), df_add(a.y, b.y)}; }
    static __device__ __forceinline__ T one() { return {{1.f, 0.f}, {0.f, 0.f}}; }
    static __device__ __forceinline__ double re(const T &a) { return to_double(a.x); }
    static __device__ __forceinline__ double im(const T &a) { return to_double(a.y); }
};
template <>
struct Elem<false> {
    using T = double2;
    static __device__ __forceinline__ T from(double2 v) { return v; }
    static __device__ __forceinline__ T mul(const T &a, const T &b) { return cmul(a, b); }
    static __device__ __forceinline__ T add(const T &a, const T &b) { return make_double2(a.x + b.x, a.y + b.y); }
    static __device__ __forceinline__ T one() { return make_double2(1.0, 0.0); }
    static __device__ __forceinline__ double re(const T &a) { return a.x; }
    static __device__ __forceinline__ double im(const T &a) { return a.y; }
};

// What a launch evaluates per term: KIND 0 the product of the A blocks (a correlator); KIND 1 the
// sum over k of the product with block k taken from the derivative blocks D (a three-point
// function); KIND 4, 9, 16 the product once, added into that many matrix elements with weights of
// their own (a correlation matrix).
template <int KIND>
struct Kind {
    static constexpr bool DERIV = KIND == 1;
    static constexpr int NEL = KIND >= 4 ? KIND : 1;
};

struct TableWork {
    const uint16_t *ids;   // [U][AP]
    const double *w;       // [U][NEL]
    const float2 *wf;      // [U][NEL] the weights as exact float pairs
    int64_t U;
    int64_t chunk;         // terms per item
    int A, n_chunks;       // chunks per (configuration, slice)
    int item_off;          // first item of this table within a (configuration, slice)
    double scale;
};

struct ContractWork {
    TableWork tab[kMaxTables];
    int n_tab;
    const double2 *blocks;     // [n_cfg][n_slices][n_blk]
    const double2 *dblocks;    // derivative blocks (KIND 1), same layout
    const cdf *fblocks;        // MIXED without staging: blocks (and derivative blocks) converted to float
    const cdf *fdblocks;       //   pairs before the launch, or null (converted at each gather)
    int n_blk, n_cfg, n_slices;
    int items_per_cs;          // items of one (configuration, slice)
    int64_t n_items;
    double2 *C_out;            // [n_cfg][n_tab][NEL][n_slices]
    double2 *partials;         // [n_items][NEL]
    int *counters;             // [n_cfg][n_tab][n_slices]
    unsigned long long *queue; // [0] next item, [1] CTAs that have left
    double el_scale[16];       // matrix elements: scale of each element
};

__device__ __forceinline__ cdf ldcg_cdf(const cdf *p) {
    const float4 v = __ldcg(reinterpret_cast<const float4 *>(p));
    return {{v.x, v.y}, {v.z, v.w}};
}

// a block entry from shared memory (STAGE), from the pre-converted float pairs (PRE: MIXED without
// staging), or from the complex128 blocks.  The source is a compile-time choice: a run-time one becomes
// one load from a selected address with the conversion predicated, and predicated-off FP64 instructions
// still take the FP64 pipe's issue slots.
template <typename C, bool MIXED, bool STAGE, bool PRE>
__device__ __forceinline__ C load_block(const C *sB, const double2 *gB, const cdf *fB, int id) {
    if constexpr (STAGE) return sB[id];
    else if constexpr (PRE) return ldcg_cdf(fB + id);
    else return Elem<MIXED>::from(__ldcg(gB + id));
}

// this thread's share of terms [u0, u1) of one table, against one slice's blocks (and derivative blocks)
template <int A, bool MIXED, bool STAGE, int KIND, bool PRE>
__device__ __forceinline__ void eval_terms(const TableWork &tw, int64_t u0, int64_t u1,
                                           const typename Elem<MIXED>::T *sB, const typename Elem<MIXED>::T *sD,
                                           const double2 *gB, const double2 *gD, const cdf *fB, const cdf *fD,
                                           double *ax, double *ay) {
    using E = Elem<MIXED>;
    using C = typename E::T;
    using K = Kind<KIND>;
    constexpr int AP = A <= 4 ? 4 : 8;
    // MIXED: double-FP32 group partials (up to 4 matrix elements; more would not fit the registers, and
    // those sum each term in FP64)
    constexpr bool GROUP = MIXED && K::NEL <= 4;
    df gx[K::NEL], gy[K::NEL];
    int in_group = 0;
#pragma unroll
    for (int e = 0; e < K::NEL; ++e) gx[e] = gy[e] = df{0.f, 0.f};
    for (int64_t u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
        uint16_t id[AP];
        if constexpr (AP == 4) {
            const uint2 v = __ldg(reinterpret_cast<const uint2 *>(tw.ids) + u);
            id[0] = (uint16_t)(v.x & 0xFFFF); id[1] = (uint16_t)(v.x >> 16);
            id[2] = (uint16_t)(v.y & 0xFFFF); id[3] = (uint16_t)(v.y >> 16);
        } else {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(tw.ids) + u);
            const unsigned wd[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                id[2 * q] = (uint16_t)(wd[q] & 0xFFFF);
                id[2 * q + 1] = (uint16_t)(wd[q] >> 16);
            }
        }
        C p;
        if constexpr (K::DERIV) {
            // sum_k D_k prod_{j != k} B_j: prefix products forward, the suffix product backward
            C pre[A];
            pre[0] = E::one();
#pragma unroll
            for (int k = 1; k < A; ++k)
                pre[k] = E::mul(pre[k - 1], load_block<C, MIXED, STAGE, PRE>(sB, gB, fB, id[k - 1]));
            C suf = E::one();
            p = E::mul(pre[A - 1], load_block<C, MIXED, STAGE, PRE>(sD, gD, fD, id[A - 1]));
#pragma unroll
            for (int k = A - 2; k >= 0; --k) {
                suf = E::mul(suf, load_block<C, MIXED, STAGE, PRE>(sB, gB, fB, id[k + 1]));
                p = E::add(p, E::mul(E::mul(pre[k], load_block<C, MIXED, STAGE, PRE>(sD, gD, fD, id[k])), suf));
            }
        } else {
            p = load_block<C, MIXED, STAGE, PRE>(sB, gB, fB, id[0]);
#pragma unroll
            for (int k = 1; k < A; ++k) p = E::mul(p, load_block<C, MIXED, STAGE, PRE>(sB, gB, fB, id[k]));
        }
        if constexpr (GROUP) {
#pragma unroll
            for (int e = 0; e < K::NEL; ++e) {
                const float2 wv = __ldg(tw.wf + u * K::NEL + e);
                const df w{wv.x, wv.y};
                gx[e] = df_add(gx[e], df_mul(w, p.x));
                gy[e] = df_add(gy[e], df_mul(w, p.y));
            }
            if (++in_group == kMixedGroup) {
#pragma unroll
                for (int e = 0; e < K::NEL; ++e) {
                    ax[e] += to_double(gx[e]);
                    ay[e] += to_double(gy[e]);
                    gx[e] = gy[e] = df{0.f, 0.f};
                }
                in_group = 0;
            }
        } else {
            const double pr = E::re(p), pi = E::im(p);
#pragma unroll
            for (int e = 0; e < K::NEL; ++e) {
                const double wu = __ldg(tw.w + u * K::NEL + e);
                ax[e] = fma(wu, pr, ax[e]);
                ay[e] = fma(wu, pi, ay[e]);
            }
        }
    }
    if constexpr (GROUP) {
        if (in_group) {
#pragma unroll
            for (int e = 0; e < K::NEL; ++e) {
                ax[e] += to_double(gx[e]);
                ay[e] += to_double(gy[e]);
            }
        }
    }
}

template <bool MIXED, bool STAGE, int KIND, bool PRE>
__device__ __forceinline__ void eval_any(const TableWork &tw, int64_t u0, int64_t u1,
                                         const typename Elem<MIXED>::T *sB, const typename Elem<MIXED>::T *sD,
                                         const double2 *gB, const double2 *gD, const cdf *fB, const cdf *fD,
                                         double *ax, double *ay) {
    if constexpr (Kind<KIND>::NEL > 1) {   // correlation matrices: nuclei up to A = 4
        switch (tw.A) {
            case 1: eval_terms<1, MIXED, STAGE, KIND, PRE>(tw, u0, u1, sB, sD, gB, gD, fB, fD, ax, ay); break;
            case 2: eval_terms<2, MIXED, STAGE, KIND, PRE>(tw, u0, u1, sB, sD, gB, gD, fB, fD, ax, ay); break;
            case 3: eval_terms<3, MIXED, STAGE, KIND, PRE>(tw, u0, u1, sB, sD, gB, gD, fB, fD, ax, ay); break;
            default: eval_terms<4, MIXED, STAGE, KIND, PRE>(tw, u0, u1, sB, sD, gB, gD, fB, fD, ax, ay); break;
        }
    } else {
        switch (tw.A) {
            case 1: eval_terms<1, MIXED, STAGE, KIND, PRE>(tw, u0, u1, sB, sD, gB, gD, fB, fD, ax, ay); break;
            case 2: eval_terms<2, MIXED, STAGE, KIND, PRE>(tw, u0, u1, sB, sD, gB, gD, fB, fD, ax, ay); break;
            case 3: eval_terms<3, MIXED, STAGE, KIND, PRE>(tw, u0, u1, sB, sD, gB, gD, fB, fD, ax, ay); break;
            case 4: eval_terms<4, MIXED, STAGE, KIND, PRE>(tw, u0, u1, sB, sD, gB, gD, fB, fD, ax, ay); break;
            case 5: eval_terms<5, MIXED, STAGE, KIND, PRE>(tw, u0, u1, sB, sD, gB, gD, fB, fD, ax, ay); break;
            case 6: eval_terms<6, MIXED, STAGE, KIND, PRE>(tw, u0, u1, sB, sD, gB, gD, fB, fD, ax, ay); break;
            case 7: eval_terms<7, MIXED, STAGE, KIND, PRE>(tw, u0, u1, sB, sD, gB, gD, fB, fD, ax, ay); break;
            default: eval_terms<8, MIXED, STAGE, KIND, PRE>(tw, u0, u1, sB, sD, gB, gD, fB, fD, ax, ay); break;
        }
    }
}

// fixed-order sum over the CTA: a shuffle tree per warp, then warp 0 over the warps' sums
__device__ __forceinline__ double2 cta_sum(double ax, double ay, double2 *s_red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        ax += __shfl_down_sync(0xffffffffu, ax, off);
        ay += __shfl_down_sync(0xffffffffu, ay, off);
    }
    if (lane == 0) s_red[warp] = make_double2(ax, ay);
    __syncthreads();
    double2 r = make_double2(0.0, 0.0);
    if (warp == 0) {
        double bx = lane < nw ? s_red[lane].x : 0.0, by = lane < nw ? s_red[lane].y : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            bx += __shfl_down_sync(0xffffffffu, bx, off);
            by += __shfl_down_sync(0xffffffffu, by, off);
        }
        r = make_double2(bx, by);
    }
    __syncthreads();   // s_red free for the next sum
    return r;   // valid in thread 0
}

template <bool MIXED, bool STAGE, int KIND, bool PRE>
__global__ void __launch_bounds__(kMaxThreads)
contract_persistent_kernel(const __grid_constant__ ContractWork wk) {
    using E = Elem<MIXED>;
    using C = typename E::T;
    using K = Kind<KIND>;
    constexpr int NEL = K::NEL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sB = reinterpret_cast<C *>(smem_raw);
    C *sD = sB + (K::DERIV ? wk.n_blk : 0);
    __shared__ long long s_item;
    __shared__ int s_last;
    __shared__ double2 s_red[kMaxThreads / 32];
    long long staged = -1;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(wk.queue, 1ull);
        __syncthreads();
        const long long item = s_item;
        if (item >= wk.n_items) break;
        const long long cs = item / wk.items_per_cs;          // configuration * n_slices + slice
        const int r = (int)(item - cs * wk.items_per_cs);
        int tb = 0;
        while (tb + 1 < wk.n_tab && r >= wk.tab[tb + 1].item_off) ++tb;
        const TableWork &tw = wk.tab[tb];
        const int chunk = r - tw.item_off;
        const double2 *gB = wk.blocks + cs * wk.n_blk;
        const double2 *gD = K::DERIV ? wk.dblocks + cs * wk.n_blk : gB;
        const cdf *fB = wk.fblocks ? wk.fblocks + cs * wk.n_blk : nullptr;
        const cdf *fD = K::DERIV && wk.fdblocks ? wk.fdblocks + cs * wk.n_blk : fB;
        if constexpr (STAGE) {
            if (cs != staged) {   // every thread is past the previous item's gathers (barrier above)
                for (int i = threadIdx.x; i < wk.n_blk; i += blockDim.x) {
                    sB[i] = E::from(__ldcg(gB + i));
                    if constexpr (K::DERIV) sD[i] = E::from(__ldcg(gD + i));
                }
                __syncthreads();
                staged = cs;
            }
        }
        const int64_t u0 = (int64_t)chunk * tw.chunk;
        const int64_t u1 = min(tw.U, u0 + tw.chunk);
        double ax[NEL], ay[NEL];
#pragma unroll
        for (int e = 0; e < NEL; ++e) ax[e] = ay[e] = 0.0;
        eval_any<MIXED, STAGE, KIND, PRE>(tw, u0, u1, sB, sD, gB, gD, fB, fD, ax, ay);
        const int cfg = (int)(cs / wk.n_slices), slice = (int)(cs - (long long)cfg * wk.n_slices);
        int *cnt = wk.counters + ((size_t)cfg * wk.n_tab + tb) * wk.n_slices + slice;
#pragma unroll
        for (int e = 0; e < NEL; ++e) {
            const double2 tot = cta_sum(ax[e], ay[e], s_red);
            if (threadIdx.x == 0) wk.partials[item * NEL + e] = tot;
        }
        if (threadIdx.x == 0) {
            __threadfence();
            s_last = atomicAdd(cnt, 1) == tw.n_chunks - 1;
        }
        __syncthreads();
        if (s_last && threadIdx.x < NEL) {
            // every chunk of this (configuration, table, slice) has written its partials: sum them in chunk order
            const int e = threadIdx.x;
            __threadfence();
            const double2 *p = wk.partials + (item - chunk) * NEL + e;
            double x = 0.0, y = 0.0;
            for (int c = 0; c < tw.n_chunks; ++c) {
                const double2 v = __ldcg(p + (size_t)c * NEL);
                x += v.x;
                y += v.y;
            }
            const double sc = NEL > 1 ? wk.el_scale[e] : tw.scale;
            wk.C_out[(((size_t)cfg * wk.n_tab + tb) * NEL + e) * wk.n_slices + slice] = make_double2(sc * x, sc * y);
            if (e == 0) *cnt = 0;
        }
        // the next iteration's first barrier orders the reuse of s_item and s_last
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(wk.queue + 1, 1ull) == (unsigned long long)gridDim.x - 1) {
            wk.queue[0] = 0ull;   // every CTA has left: ready for the next launch
            wk.queue[1] = 0ull;
        }
    }
}

// the blocks as double-FP32 pairs (hi, lo of each component), once per launch
__global__ void convert_kernel(const double2 *__restrict__ b, int64_t n, cdf *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const cdf v = to_cdf(__ldcg(b + i));
        reinterpret_cast<float4 *>(out)[i] = make_float4(v.x.h, v.x.l, v.y.h, v.y.l);
    }
}

template <bool MIXED, bool STAGE, int KIND, bool PRE = false>
int launch_typed(const ContractWork &wk, int grid, int threads, size_t smem, cudaStream_t stream) {
    auto k = contract_persistent_kernel<MIXED, STAGE, KIND, PRE>;
    if (smem > 48 * 1024) WICK_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<grid, threads, smem, stream>>>(wk);
    WICK_CUDA_TRY(cudaGetLastError());
    return WICK_OK;
}

template <bool MIXED, bool STAGE, int KIND>
int max_ctas_per_sm(int threads, size_t smem) {
    int n = 0;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(contract_persistent_kernel<MIXED, STAGE, KIND, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return 1;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, contract_persistent_kernel<MIXED, STAGE, KIND, false>, threads,
                                                      smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return 1;
    }
    return n < 1 ? 1 : n;
}

template <int KIND>
int occupancy(bool mixed, bool stage, int threads, size_t smem) {
    return mixed ? (stage ? max_ctas_per_sm<true, true, KIND>(threads, smem) : max_ctas_per_sm<true, false, KIND>(threads, smem))
                 : (stage ? max_ctas_per_sm<false, true, KIND>(threads, smem) : max_ctas_per_sm<false, false, KIND>(threads, smem));
}

template <int KIND>
int launch_kind(const ContractWork &wk, bool mixed, bool stage, int grid, int threads, size_t smem, cudaStream_t stream) {
    if (mixed) return stage        ? launch_typed<true, true, KIND>(wk, grid, threads, smem, stream)
                      : wk.fblocks ? launch_typed<true, false, KIND, true>(wk, grid, threads, smem, stream)
                                   : launch_typed<true, false, KIND>(wk, grid, threads, smem, stream);
    return stage ? launch_typed<false, true, KIND>(wk, grid, threads, smem, stream)
                 : launch_typed<false, false, KIND>(wk, grid, threads, smem, stream);
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

// ---------------------------------------------------------------------------
// Planning: term chunks, grid, scratch.  The chunking of a table depends on
// its own size and the tuning only -- about chunk_terms terms per item, split
// evenly -- so a batch and the single calls of its configurations add the
// same partial sums in the same order (bitwise equal results).  A plan of
// more than max_items items takes longer chunks.
// ---------------------------------------------------------------------------
int contract_plan(int n_blk, int n_cfg, int n_slices, const ContractTable *tabs, int n_tab, int precision,
                  const ContractTune &tune, int64_t max_items, ContractPlan *plan, int kind) {
    if (n_tab < 1 || n_tab > kMaxTables || n_cfg < 1 || n_slices < 1 || n_blk < 1) return WICK_EINVAL;
    if (kind != 0 && kind != 1 && kind != 4 && kind != 9 && kind != 16) return WICK_EINVAL;
    ContractPlan &P = *plan;
    P = ContractPlan{};
    P.kind = kind;
    const int nel = kind >= 4 ? kind : 1;
    const bool mixed = precision == WICK_MIXED;
    P.threads = tune.threads > 0 ? tune.threads : 256;
    if (P.threads % 32 || P.threads < 32 || P.threads > kMaxThreads) return WICK_EINVAL;
    const size_t elem = 16 * (kind == 1 ? 2 : 1);   // complex128 or a double-FP32 complex pair (and D)
    P.stage = (size_t)n_blk * elem <= kSmemStageLimit;
    P.smem = P.stage ? (size_t)n_blk * elem : 0;
    int dev = 0, n_sm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int occ = kind == 0 ? occupancy<0>(mixed, P.stage, P.threads, P.smem)
                  : kind == 1 ? occupancy<1>(mixed, P.stage, P.threads, P.smem)
                  : kind == 4 ? occupancy<4>(mixed, P.stage, P.threads, P.smem)
                  : kind == 9 ? occupancy<9>(mixed, P.stage, P.threads, P.smem)
                              : occupancy<16>(mixed, P.stage, P.threads, P.smem);
    const int per_sm = tune.ctas_per_sm > 0 ? std::min(tune.ctas_per_sm, occ) : occ;
    const int64_t n_cs = (int64_t)n_cfg * n_slices;
    for (int k = 0; k < n_tab; ++k)
        if (tabs[k].U < 0 || tabs[k].A < 1 || tabs[k].A > (nel > 1 ? 4 : kMaxA)) return WICK_EINVAL;
    int64_t target = tune.chunk_terms > 0 ? tune.chunk_terms : kDefaultChunkTerms;
    for (;;) {
        int64_t ips = 0;
        for (int k = 0; k < n_tab; ++k) ips += std::max<int64_t>(1, (tabs[k].U + target - 1) / target);
        if (ips * n_cs * nel <= max_items) break;
        if (ips == n_tab) return WICK_ESCRATCH;   // one chunk per table and still too many items
        target *= 2;
    }
    int off = 0;
    for (int k = 0; k < n_tab; ++k) {
        const int nc = (int)std::max<int64_t>(1, (tabs[k].U + target - 1) / target);
        P.n_chunks[k] = nc;
        P.chunk[k] = std::max<int64_t>(1, (tabs[k].U + nc - 1) / nc);
        P.item_off[k] = off;
        off += nc;
    }
    P.items_per_cs = off;
    P.n_items = (int64_t)off * n_cs;
    const int64_t most = (int64_t)n_sm * per_sm;
    P.grid = (int)std::max<int64_t>(1, std::min<int64_t>(most, P.n_items));
    P.counters = (size_t)n_cfg * n_tab * n_slices;
    P.counter_bytes = 256 + align256(sizeof(int) * P.counters);
    P.partial_bytes = align256(sizeof(double2) * (size_t)P.n_items * nel);
    P.convert_bytes = mixed && !P.stage ? align256(16 * (size_t)n_cfg * n_slices * n_blk) * (kind == 1 ? 2 : 1) : 0;
    return WICK_OK;
}

int launch_contract(const double2 *blocks, int n_blk, int n_cfg, int n_slices, const ContractTable *tabs, int n_tab,
                    int precision, const ContractPlan &P, void *counters, double2 *partials, double2 *C_out,
                    cudaStream_t stream, const double2 *dblocks, void *convert) {
    if (!counters || !partials || (uintptr_t)counters % 256 || (uintptr_t)partials % 16) return WICK_EINVAL;
    if (P.kind == 1 && !dblocks) return WICK_EINVAL;
    ContractWork wk{};
    wk.n_tab = n_tab;
    for (int k = 0; k < n_tab; ++k) {
        if (precision == WICK_MIXED && tabs[k].U > 0 && !tabs[k].wf) return WICK_EINVAL;
        wk.tab[k] = {tabs[k].ids, tabs[k].w, tabs[k].wf, tabs[k].U, P.chunk[k], tabs[k].A, P.n_chunks[k],
                     P.item_off[k], tabs[k].scale};
        if (P.kind >= 4)
            for (int e = 0; e < P.kind; ++e) wk.el_scale[e] = tabs[k].el_scale ? tabs[k].el_scale[e] : tabs[k].scale;
    }
    wk.blocks = blocks;
    wk.dblocks = dblocks;
    wk.n_blk = n_blk;
    wk.n_cfg = n_cfg;
    wk.n_slices = n_slices;
    wk.items_per_cs = P.items_per_cs;
    wk.n_items = P.n_items;
    wk.C_out = C_out;
    unsigned char *base = static_cast<unsigned char *>(counters);
    wk.queue = reinterpret_cast<unsigned long long *>(base);
    wk.counters = reinterpret_cast<int *>(base + 256);
    wk.partials = partials;
    const bool mixed = precision == WICK_MIXED;
    if (mixed && !P.stage && convert && P.convert_bytes) {
        if ((uintptr_t)convert % 16) return WICK_EINVAL;
        const int64_t n = (int64_t)n_cfg * n_slices * n_blk;
        cdf *fb = static_cast<cdf *>(convert);
        const unsigned g = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
        convert_kernel<<<g, 256, 0, stream>>>(blocks, n, fb);
        WICK_CUDA_TRY(cudaGetLastError());
        wk.fblocks = fb;
        if (P.kind == 1) {
            cdf *fd = reinterpret_cast<cdf *>(static_cast<unsigned char *>(convert) + P.convert_bytes / 2);
            convert_kernel<<<g, 256, 0, stream>>>(dblocks, n, fd);
            WICK_CUDA_TRY(cudaGetLastError());
            wk.fdblocks = fd;
        }
    }
    switch (P.kind) {
        case 0: return launch_kind<0>(wk, mixed, P.stage, P.grid, P.threads, P.smem, stream);
        case 1: return launch_kind<1>(wk, mixed, P.stage, P.grid, P.threads, P.smem, stream);
        case 4: return launch_kind<4>(wk, mixed, P.stage, P.grid, P.threads, P.smem, stream);
        case 9: return launch_kind<9>(wk, mixed, P.stage, P.grid, P.threads, P.smem, stream);
        case 16: return launch_kind<16>(wk, mixed, P.stage, P.grid, P.threads, P.smem, stream);
        default: return WICK_EINVAL;
    }
}

// ---------------------------------------------------------------------------
// Fixed scratch of wick_contract_noalloc, in a file-scope device array instead
// of the library's cudaMalloc'd workspace: the item counters and one counter
// per slice (kNoAllocCounterBytes), then at that fixed offset the FP64 partial
// sums (one complex128 per work item).  Every device that loads the library
// holds these kNoAllocBytes until the process exits.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

int noalloc_scratch(void **ptr, size_t *bytes) {
    // In host code the array's name is only a host-side stand-in; its device
    // address comes from the runtime for the device that is current now.  It
    // is looked up on every call (no allocation, a table lookup once the
    // module is loaded), so a context that was reset or replaced never sees a
    // stale address.
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        (void)cudaGetLastError();
        return WICK_ECUDA;
    }
    *ptr = p;
    *bytes = kNoAllocBytes;
    return WICK_OK;
}

namespace {
__global__ void product_kernel(const double2 *__restrict__ a, const double2 *__restrict__ b, int64_t n,
                               double2 *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = cmul(a[i], b[i]);
}

// Contribution magnitudes (Sec. V.C): mag[u] = sum over slices of |scale w_u prod_k B[slice][id_{u,k}]|,
// FP64, one thread per term
__global__ void magnitude_kernel(const double2 *__restrict__ blocks, int n_blk, int n_slices,
                                 const uint16_t *__restrict__ ids, const double *__restrict__ w, int64_t U, int A,
                                 int AP, double scale, double *__restrict__ mag) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= U) return;
    double m = 0.0;
    for (int s = 0; s < n_slices; ++s) {
        const double2 *B = blocks + (size_t)s * n_blk;
        double2 p = B[ids[u * AP]];
        for (int k = 1; k < A; ++k) p = cmul(p, B[ids[u * AP + k]]);
        m += hypot(p.x, p.y);
    }
    mag[u] = m * fabs(w[u] * scale);
}

// contraction copies of a reduced table: ids padded to [U][AP], weights as doubles (exact below 2^53)
__global__ void pad_table_kernel(const uint16_t *__restrict__ ids, const int64_t *__restrict__ w, int64_t U, int A,
                                 int AP, uint16_t *__restrict__ ids_pad, double *__restrict__ wd) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= U) return;
    for (int k = 0; k < AP; ++k) ids_pad[u * AP + k] = k < A ? ids[u * A + k] : (uint16_t)0;
    if (w) wd[u] = (double)w[u];
}

// the weights as float pairs for the MIXED term sums: hi = wd rounded to float, lo = the rest
__global__ void split_weights_kernel(const double *__restrict__ wd, int64_t n, float2 *__restrict__ wf) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const df v = split_double(wd[i]);
    wf[i] = make_float2(v.h, v.l);
}
}  // namespace

int split_weights(const double *wd, int64_t n, float2 *wf, cudaStream_t stream) {
    if (n <= 0) return WICK_OK;
    split_weights_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(wd, n, wf);
    WICK_CUDA_TRY(cudaGetLastError());
    return WICK_OK;
}

int launch_magnitudes(const double2 *blocks, int n_blk, int n_slices, const ContractTable &tab, double *mag,
                      cudaStream_t stream) {
    if (tab.U <= 0) return WICK_OK;
    const int AP = tab.A <= 4 ? 4 : 8;
    magnitude_kernel<<<(unsigned)((tab.U + 255) / 256), 256, 0, stream>>>(blocks, n_blk, n_slices, tab.ids, tab.w,
                                                                          tab.U, tab.A, AP, tab.scale, mag);
    WICK_CUDA_TRY(cudaGetLastError());
    return WICK_OK;
}

int pad_table(const uint16_t *ids, const int64_t *w, int64_t U, int A, uint16_t *ids_pad, double *wd,
              cudaStream_t stream) {
    if (U <= 0) return WICK_OK;
    const int AP = A <= 4 ? 4 : 8;
    pad_table_kernel<<<(unsigned)((U + 255) / 256), 256, 0, stream>>>(ids, w, U, A, AP, ids_pad, wd);
    WICK_CUDA_TRY(cudaGetLastError());
    return WICK_OK;
}

}  // namespace wick

extern "C" int wick_cluster_product(const void *Ca, const void *Cb, int64_t n, void *out, wick_stream_t stream) {
    if (!Ca || !Cb || !out || n < 0) return WICK_EINVAL;
    if ((uintptr_t)Ca % 16 || (uintptr_t)Cb % 16 || (uintptr_t)out % 16) return WICK_EINVAL;
    if (n == 0) return WICK_OK;
    wick::product_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        (const double2 *)Ca, (const double2 *)Cb, n, (double2 *)out);
    WICK_CUDA_TRY(cudaGetLastError());
    return WICK_OK;
}
