// Baryon blocks (Eq. 2.4/2.5) projected to zero momentum.
//
// For every (src, t) slice and every block type / nucleon spin the kernel
// forms   P_{op,s}(c1,c2,c3) = sum_x sum_{(r1,l)} S1(x)(r1,c1) X_l(x)(c2,c3)
//         X_l(x)(c2,c3)      = sum_{(r2,r3,w) in l} w S1(x)(r2,c2) S2(x)(r3,c3)
// (the diquark lists X, then a rank-|OS|-per-site update of P), and the
// reduction kernel antisymmetrises  B(c1,c2,c3) = P(c1,c2,c3) - P(c2,c1,c3).
//
// Work split: grid = (slice, site chunk, output chunk).  Each CTA stages the
// rows of S its tables use for NS sites at a time in shared memory, computes
// the diquark lists of those sites, and every thread updates groups of three
// consecutive outputs (same op, spin and c1: one S1 load serves three
// products).  Accumulators live in registers for the whole chunk of at most
// 256 sites; chunk partials are written in FP64 and summed over chunks in a
// fixed order by the reduction kernel (deterministic).
//
// Arithmetic: WICK_FP64 -- double throughout.  WICK_MIXED -- double-FP32:
// products of the (float) propagator entries are formed exactly with FMA
// (TwoProd) and accumulated as float pairs with TwoSum (about 44 significant
// bits), on the FP32 pipes; chunk partials in FP64.  When every diquark weight
// is a signed power of two (all operators of Eqs. 1000/1001) the double-FP32
// steps run on the packed f32x2 instructions: each output keeps one packed
// accumulator with lanes (re, im) and one with lanes (im, re), so both halves
// of a complex product use the same operand pair.
#include <type_traits>

#include "common.cuh"
#include "df32.cuh"

namespace wick {

namespace {

#ifndef WICK_BLK_GROUPS
#define WICK_BLK_GROUPS 2
#endif
#ifndef WICK_BLK_MINB
#define WICK_BLK_MINB 2
#endif
#ifndef WICK_BLK_NS
#define WICK_BLK_NS 16
#endif
#ifndef WICK_BLK_SMEM_KB
#define WICK_BLK_SMEM_KB 72
#endif
constexpr int kThreads = 288;               // 9 warps: one output group per thread for the upper-spin tables
constexpr int kGroups = WICK_BLK_GROUPS;    // output groups per thread
constexpr int kMinBlocks = WICK_BLK_MINB;   // resident CTAs per SM the register budget aims at
constexpr int kMaxNs = WICK_BLK_NS;         // sites staged per tile, at most
constexpr int kSmemBudget = WICK_BLK_SMEM_KB * 1024;
constexpr int kChunk = 256;                 // sites per accumulation chunk

__device__ __forceinline__ float2 to_f2(float2 v) { return v; }
__device__ __forceinline__ float2 to_f2(double2 v) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }

__device__ __forceinline__ void cfma(double2 &acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}

// arithmetic modes of the block kernel
constexpr int kFP64 = 0, kDF32 = 1, kDF32X2 = 2;

template <int MODE> struct Types;
template <> struct Types<kDF32X2> { using S = float2; using X = pdf; };
template <> struct Types<kDF32> { using S = float2; using X = cdf; };
template <> struct Types<kFP64> { using S = double2; using X = double2; };

// accumulator of one output: packed mode keeps two (see above)
template <int MODE> struct Acc { typename Types<MODE>::X v; };
template <> struct Acc<kDF32X2> { pdf a, b; };

__device__ __forceinline__ void zero(cdf &a) { a.x = {0.f, 0.f}; a.y = {0.f, 0.f}; }
__device__ __forceinline__ void zero(double2 &a) { a = make_double2(0.0, 0.0); }
__device__ __forceinline__ void zero(pdf &a) { a.h = 0ull; a.l = 0ull; }
__device__ __forceinline__ void zero(Acc<kFP64> &a) { zero(a.v); }
__device__ __forceinline__ void zero(Acc<kDF32> &a) { zero(a.v); }
__device__ __forceinline__ void zero(Acc<kDF32X2> &a) { zero(a.a); zero(a.b); }
__device__ __forceinline__ double2 out_d2(const Acc<kFP64> &a) { return a.v; }
__device__ __forceinline__ double2 out_d2(const Acc<kDF32> &a) { return make_double2(to_double(a.v.x), to_double(a.v.y)); }
__device__ __forceinline__ double2 out_d2(const Acc<kDF32X2> &a) {
    float ah0, ah1, al0, al1, bh0, bh1, bl0, bl1;
    upk(a.a.h, ah0, ah1); upk(a.a.l, al0, al1);   // lanes (re, im)
    upk(a.b.h, bh0, bh1); upk(a.b.l, bl0, bl1);   // lanes (im, re)
    return make_double2(((double)ah0 + (double)bh1) + ((double)al0 + (double)bl1),
                        ((double)ah1 + (double)bh0) + ((double)al1 + (double)bl0));
}

// X(c2,c3) += w * a * b (a, b exact float complex), per mode
__device__ __forceinline__ void x_term(double2 &v, float w, double2 a, double2 b) {
    const double wd = (double)w;
    const double2 aw = make_double2(wd * a.x, wd * a.y);
    v.x = fma(aw.x, b.x, v.x); v.x = fma(-aw.y, b.y, v.x);
    v.y = fma(aw.x, b.y, v.y); v.y = fma(aw.y, b.x, v.y);
}
__device__ __forceinline__ void x_term(cdf &v, float w, float2 a, float2 b) { cacc_fma3(v, w, a, b); }

// P += a * X, per mode
__device__ __forceinline__ void p_term(Acc<kFP64> &acc, double2 a, const double2 &x) { cfma(acc.v, a, x); }
__device__ __forceinline__ void p_term(Acc<kDF32> &acc, float2 a, const cdf &x) { cacc_fma(acc.v, a, x); }

template <int MODE, typename ST>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
block_partial_kernel(const __grid_constant__ BlockPlan plan, const ST *__restrict__ Su, const ST *__restrict__ Sd,
                     const ST *__restrict__ Sg, int sub_flav, int sub_pass, int split0, int V, int n_slices, int chunk,
                     int ns_tile, double2 *__restrict__ partials) {
    constexpr bool DF = MODE != kFP64;
    using SC = typename Types<MODE>::S;
    using XC = typename Types<MODE>::X;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nc = plan.n_chi, nc2 = nc * nc, nc3 = nc2 * nc;
    const int nr0 = plan.n_rows[0], nr1 = plan.n_rows[1];
    // staged rows: flavour u, flavour d, then (a three-point build) the rows of the sequential
    // propagator Sg, which stands in for flavour sub_flav in one slot of every nucleon
    const int nrs = sub_flav >= 0 ? plan.n_rows[sub_flav] : 0;
    const int nr = nr0 + nr1 + nrs;
    SC *sS = reinterpret_cast<SC *>(smem_raw);
    XC *sX = reinterpret_cast<XC *>(smem_raw + sizeof(SC) * (size_t)ns_tile * nr * nc);
    // the staged section (first row) each slot of a type with pair flavour f1 reads: slot 1 (the U rows),
    // slot 2 (the first diquark factor), slot 3 (the second); pass 0 puts Sg into the first slot of flavour
    // sub_flav, pass 1 into the second (a type with one quark of that flavour then adds nothing)
    auto sec = [&](int f) { return f == 0 ? 0 : nr0; };
    auto slot_sec = [&](int f1, int slot) {
        const int f = slot == 3 ? 1 - f1 : f1;
        const bool sub = sub_flav == f && ((slot == 1 && sub_pass == 0) || (slot == 2 && sub_pass == 1) ||
                                           (slot == 3 && sub_pass == 0));
        return sub ? nr0 + nr1 : sec(f);
    };
    auto silent = [&](int f1) { return sub_flav == 1 - f1 && sub_pass == 1; };

    const int slice = blockIdx.x;
    const int x_begin = blockIdx.y * chunk;
    const int x_end = min(V, x_begin + chunk);
    const int gpr = (nc2 + 2) / 3;                       // output groups per (op, spin, c1) row
    const int n_groups = plan.n_ops * plan.n_spin * nc * gpr;

    int g_os[kGroups], g_i1[kGroups], g_i23[kGroups], g_cnt[kGroups], g_f[kGroups];
    Acc<MODE> acc[kGroups][3];
#pragma unroll
    for (int k = 0; k < kGroups; ++k) {
        const int g = blockIdx.z * (kThreads * kGroups) + threadIdx.x + k * kThreads;
        g_cnt[k] = 0;
        g_os[k] = 0; g_i1[k] = 0; g_i23[k] = 0; g_f[k] = 0;
        if (g < n_groups) {
            const int row = g / gpr, j = g - row * gpr;
            g_os[k] = row / nc;
            g_i1[k] = row - g_os[k] * nc;
            g_i23[k] = 3 * j;
            g_cnt[k] = min(3, nc2 - 3 * j);
            g_f[k] = plan.f1[g_os[k] / plan.n_spin];
            if (silent(g_f[k])) g_cnt[k] = -g_cnt[k];   // outputs written as zeros
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) zero(acc[k][q]);
    }

    // diquark lists needed by this CTA's outputs (lists are ordered by op)
    int l_lo = plan.n_x, l_hi = 0;
    {
        const int g0 = blockIdx.z * (kThreads * kGroups);
        const int g1 = min(n_groups, g0 + kThreads * kGroups) - 1;
        const int o_lo = (g0 / gpr) / nc / plan.n_spin, o_hi = (g1 / gpr) / nc / plan.n_spin;
        for (int l = 0; l < plan.n_x; ++l)
            if (plan.x_op[l] >= o_lo && plan.x_op[l] <= o_hi) {
                l_lo = min(l_lo, l);
                l_hi = max(l_hi, l + 1);
            }
    }
    const int n_xl = max(0, l_hi - l_lo);

    const ST *slice_u = Su + (size_t)slice * V * 144;
    const ST *slice_d = Sd + (size_t)slice * V * 144;
    const ST *slice_g = Sg ? Sg + (size_t)slice * V * 144 : slice_u;
    for (int xb = x_begin; xb < x_end; xb += ns_tile) {
        const int ns = min(ns_tile, x_end - xb);
        // stage the rows of S used by the tables: sS[site][row][i], flavour-0 rows first
        for (int e = threadIdx.x; e < ns * nr * nc; e += kThreads) {
            const int site = e / (nr * nc);
            const int rem = e - site * nr * nc;
            const int rc = rem / nc, ic = rem - rc * nc;
            const int f = rc < nr0 ? 0 : (rc < nr0 + nr1 ? 1 : 2);
            const int row = f == 0 ? plan.rows[0][rc] : (f == 1 ? plan.rows[1][rc - nr0] : plan.rows[sub_flav][rc - nr0 - nr1]);
            const size_t idx = (size_t)(xb + site) * 144 + row * 12 + plan.chi[ic];
            const ST v = f == 0 ? slice_u[idx] : (f == 1 ? slice_d[idx] : slice_g[idx]);
            if constexpr (DF) sS[e] = to_f2(v);
            else sS[e] = to_d2(v);
        }
        __syncthreads();
        // diquark lists X[site][l][i2 * nc + i3]
        for (int e2 = threadIdx.x; e2 < ns * n_xl * nc2; e2 += kThreads) {
            const int site = e2 / (n_xl * nc2);
            const int rem = e2 - site * n_xl * nc2;
            const int l = l_lo + rem / nc2, i23 = rem % nc2;
            const int e = (site * plan.n_x + l) * nc2 + i23;
            const int i2 = i23 / nc, i3 = i23 - i2 * nc;
            const int f1 = plan.f1[plan.x_op[l]];
            const SC *s1 = sS + (size_t)site * nr * nc + slot_sec(f1, 2) * nc;
            const SC *s2 = sS + (size_t)site * nr * nc + slot_sec(f1, 3) * nc;
            if constexpr (MODE == kDF32X2) {
                // lanes (re, im) += w a.x (b.x, b.y);  lanes (im, re) += w a.y (b.x, -b.y)
                pdf va, vb;
                zero(va);
                zero(vb);
                for (int t = plan.x_off[l]; t < plan.x_off[l + 1]; ++t) {
                    const float2 a = s1[plan.xt_r2[t] * nc + i2], b = s2[plan.xt_r3[t] * nc + i3];
                    const float w = plan.xt_w[t];
                    const float ax = w * a.x, ay = w * a.y;  // exact: w is +-2^k
                    const f2x B = pk(b.x, b.y);
                    pacc_exact(va, pk(ax, ax), pk(-ax, -ax), B);
                    pacc_exact(vb, pk(ay, -ay), pk(-ay, ay), B);
                }
                sX[e] = padd(va, pdf{swap2(vb.h), swap2(vb.l)});
            } else {
                XC v;
                zero(v);
                for (int t = plan.x_off[l]; t < plan.x_off[l + 1]; ++t)
                    x_term(v, plan.xt_w[t], s1[plan.xt_r2[t] * nc + i2], s2[plan.xt_r3[t] * nc + i3]);
                sX[e] = v;
            }
        }
        __syncthreads();
        // P update: three outputs per group share the S1 entry
#pragma unroll
        for (int k = 0; k < kGroups; ++k) {
            if (g_cnt[k] <= 0) continue;
            const int os = g_os[k];
            for (int site = 0; site < ns; ++site) {
                const SC *s1 = sS + (size_t)site * nr * nc + slot_sec(g_f[k], 1) * nc;
                const XC *xs = sX + (size_t)site * plan.n_x * nc2 + g_i23[k];
                for (int t = plan.os_off[os]; t < plan.os_off[os + 1]; ++t) {
                    const SC a = s1[plan.os_r1[t] * nc + g_i1[k]];
                    const XC *xl = xs + plan.os_x[t] * nc2;
                    if constexpr (MODE == kDF32X2) {
                        const f2x A1 = pk(a.x, a.x), nA1 = pk(-a.x, -a.x);
                        const f2x A2 = pk(a.y, -a.y), nA2 = pk(-a.y, a.y);
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            if (q < g_cnt[k]) {
                                const pdf x = xl[q];
                                pacc(acc[k][q].a, A1, nA1, x.h, x.l);  // (a.x X.re, a.x X.im)
                                pacc(acc[k][q].b, A2, nA2, x.h, x.l);  // (a.y X.re, -a.y X.im)
                            }
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 3; ++q)
                            if (q < g_cnt[k]) p_term(acc[k][q], a, xl[q]);
                    }
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < kGroups; ++k) {
        if (g_cnt[k] == 0) continue;
        const int cnt = g_cnt[k] < 0 ? -g_cnt[k] : g_cnt[k];
        const int out0 = (g_os[k] * nc + g_i1[k]) * nc2 + g_i23[k];
        double2 *dst = partials + ((size_t)(split0 + blockIdx.y) * n_slices + slice) * plan.n_out + out0;
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (q < cnt) dst[q] = out_d2(acc[k][q]);
    }
    (void)nc3;
}

// B = P(c1,c2,c3) - P(c2,c1,c3), each P the fixed-order sum over site chunks.
__global__ void block_reduce_kernel(const double2 *__restrict__ partials, int n_splits, int n_slices,
                                    int n_out, int nc, double2 *__restrict__ blocks) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)n_slices * n_out) return;
    const int slice = (int)(i / n_out), out = (int)(i % n_out);
    const int nc2 = nc * nc, nc3 = nc2 * nc;
    const int os = out / nc3, i1 = (out / nc2) % nc, i2 = (out / nc) % nc, i3 = out % nc;
    const int sw = os * nc3 + i2 * nc2 + i1 * nc + i3;
    double ax = 0, ay = 0, bx = 0, by = 0;
    for (int s = 0; s < n_splits; ++s) {
        const double2 a = partials[((size_t)s * n_slices + slice) * n_out + out];
        const double2 b = partials[((size_t)s * n_slices + slice) * n_out + sw];
        ax += a.x; ay += a.y; bx += b.x; by += b.y;
    }
    blocks[i] = make_double2(ax - bx, ay - by);
}

template <int MODE, typename ST>
int launch_typed(const BlockPlan &plan, const void *Su, const void *Sd, const void *Sg, int sub_flav, int V,
                 int n_slices, double2 *partials, int n_splits, int chunk, double2 *blocks, cudaStream_t stream) {
    using SC = typename Types<MODE>::S;
    using XC = typename Types<MODE>::X;
    const int nr = plan.n_rows[0] + plan.n_rows[1] + (sub_flav >= 0 ? plan.n_rows[sub_flav] : 0);
    const size_t per_site = sizeof(SC) * (size_t)nr * plan.n_chi + sizeof(XC) * (size_t)plan.n_x * plan.n_chi * plan.n_chi;
    int ns = (int)(kSmemBudget / per_site);
    ns = ns < 1 ? 1 : (ns > kMaxNs ? kMaxNs : ns);
    const size_t smem = per_site * ns;
    auto kern = block_partial_kernel<MODE, ST>;
    WICK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int gpr = (plan.n_chi * plan.n_chi + 2) / 3;
    const int n_groups = plan.n_ops * plan.n_spin * plan.n_chi * gpr;
    const int n_oc = (n_groups + kThreads * kGroups - 1) / (kThreads * kGroups);
    dim3 grid(n_slices, n_splits, n_oc);
    // a three-point build (sub_flav >= 0) runs two passes into two sets of splits, summed by the reduction
    const int passes = sub_flav >= 0 ? 2 : 1;
    for (int pass = 0; pass < passes; ++pass) {
        kern<<<grid, kThreads, smem, stream>>>(plan, (const ST *)Su, (const ST *)Sd, (const ST *)Sg, sub_flav, pass,
                                               pass * n_splits, V, n_slices, chunk, ns, partials);
        WICK_CUDA_TRY(cudaGetLastError());
    }
    const size_t n = (size_t)n_slices * plan.n_out;
    block_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(partials, passes * n_splits, n_slices,
                                                                         plan.n_out, plan.n_chi, blocks);
    WICK_CUDA_TRY(cudaGetLastError());
    return WICK_OK;
}

}  // namespace

size_t block_partial_bytes(const BlockPlan &plan, int V, int n_slices, int precision, int range_sites) {
    if (precision == WICK_MIXED && tc_applicable(plan)) return tc_partial_bytes(plan, V, n_slices, 1, range_sites);
    const int n_splits = (V + kChunk - 1) / kChunk;
    return sizeof(double2) * (size_t)n_splits * n_slices * plan.n_out;
}

size_t block_counter_bytes(const BlockPlan &plan, int n_slices, int precision) {
    return precision == WICK_MIXED && tc_applicable(plan) ? tc_counter_bytes(plan, n_slices, 1) : 0;
}

int block_build_launches(const BlockPlan &plan, int precision) {
    return precision == WICK_MIXED && tc_applicable(plan) ? 1 : 2;
}

int launch_block_build(const BlockPlan &plan, const void *Su, int dtype_u, const void *Sd, int dtype_d, int V,
                       int n_slices, int precision, int range_sites, int *counters, void *partials, double2 *blocks,
                       cudaStream_t stream) {
    if (dtype_u != dtype_d || !partials) return WICK_EINVAL;
    if (precision == WICK_MIXED && tc_applicable(plan)) {
        int err = WICK_OK;
        int *status = status_word(&err);
        if (err) return err;
        return launch_block_tc(plan, &Su, &Sd, 1, dtype_u, V, n_slices, range_sites, counters,
                               static_cast<double2 *>(partials), blocks, status, stream);
    }
    double2 *part = static_cast<double2 *>(partials);
    const int chunk = kChunk, n_splits = (V + kChunk - 1) / kChunk;
    if (precision == WICK_MIXED || precision == WICK_MIXED_SIMT) {
        if (plan.pow2_w) {
            if (dtype_u == WICK_C64)
                return launch_typed<kDF32X2, float2>(plan, Su, Sd, nullptr, -1, V, n_slices, part, n_splits, chunk, blocks, stream);
            return launch_typed<kDF32X2, double2>(plan, Su, Sd, nullptr, -1, V, n_slices, part, n_splits, chunk, blocks, stream);
        }
        if (dtype_u == WICK_C64)
            return launch_typed<kDF32, float2>(plan, Su, Sd, nullptr, -1, V, n_slices, part, n_splits, chunk, blocks, stream);
        return launch_typed<kDF32, double2>(plan, Su, Sd, nullptr, -1, V, n_slices, part, n_splits, chunk, blocks, stream);
    }
    if (dtype_u == WICK_C64)
        return launch_typed<kFP64, float2>(plan, Su, Sd, nullptr, -1, V, n_slices, part, n_splits, chunk, blocks, stream);
    return launch_typed<kFP64, double2>(plan, Su, Sd, nullptr, -1, V, n_slices, part, n_splits, chunk, blocks, stream);
}

size_t block_3pt_partial_bytes(const BlockPlan &plan, int V, int n_slices) {
    const int n_splits = (V + kChunk - 1) / kChunk;
    return 2 * sizeof(double2) * (size_t)n_splits * n_slices * plan.n_out;
}

int launch_block_build_3pt(const BlockPlan &plan, const void *Su, const void *Sd, const void *Sg, int dtype,
                           int sub_flav, int V, int n_slices, int precision, void *partials, double2 *dblocks,
                           cudaStream_t stream) {
    if (!partials || (sub_flav != WICK_U && sub_flav != WICK_D)) return WICK_EINVAL;
    double2 *part = static_cast<double2 *>(partials);
    const int chunk = kChunk, n_splits = (V + kChunk - 1) / kChunk;
    if (precision == WICK_MIXED || precision == WICK_MIXED_SIMT) {
        if (plan.pow2_w) {
            if (dtype == WICK_C64)
                return launch_typed<kDF32X2, float2>(plan, Su, Sd, Sg, sub_flav, V, n_slices, part, n_splits, chunk,
                                                     dblocks, stream);
            return launch_typed<kDF32X2, double2>(plan, Su, Sd, Sg, sub_flav, V, n_slices, part, n_splits, chunk,
                                                  dblocks, stream);
        }
        if (dtype == WICK_C64)
            return launch_typed<kDF32, float2>(plan, Su, Sd, Sg, sub_flav, V, n_slices, part, n_splits, chunk, dblocks,
                                               stream);
        return launch_typed<kDF32, double2>(plan, Su, Sd, Sg, sub_flav, V, n_slices, part, n_splits, chunk, dblocks,
                                            stream);
    }
    if (dtype == WICK_C64)
        return launch_typed<kFP64, float2>(plan, Su, Sd, Sg, sub_flav, V, n_slices, part, n_splits, chunk, dblocks,
                                           stream);
    return launch_typed<kFP64, double2>(plan, Su, Sd, Sg, sub_flav, V, n_slices, part, n_splits, chunk, dblocks,
                                        stream);
}

}  // namespace wick
