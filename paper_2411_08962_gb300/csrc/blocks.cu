// Baryon blocks (Eq. 2.4/2.5) projected to zero momentum.
//
// For every (src, t) slice and every block type / nucleon spin the kernel
// forms   P_{op,s}(c1,c2,c3) = sum_x sum_{(r1,l)} S1(x)(r1,c1) X_l(x)(c2,c3)
//         X_l(x)(c2,c3)      = sum_{(r2,r3,w) in l} w S1(x)(r2,c2) S2(x)(r3,c3)
// (the diquark X on CUDA cores, then the rank-3-per-site update of P), and
// the reduction kernel antisymmetrises  B(c1,c2,c3) = P(c1,c2,c3) - P(c2,c1,c3).
//
// Work split: grid = (slice, site chunk, output chunk).  Each CTA streams the
// rows of S it needs for a chunk of at most 256 sites through shared memory,
// NS sites at a time, and keeps its outputs in registers (OPT per thread).
// MIXED: products and the per-chunk sum in FP32; the per-chunk partials are
// written in FP64 and summed over chunks in a fixed order (deterministic).
// FP64: the same with double throughout.
#include "common.cuh"

namespace wick {

namespace {

template <typename T> struct Cx;
template <> struct Cx<float> { using type = float2; };
template <> struct Cx<double> { using type = double2; };

__device__ __forceinline__ float2 to_c(float2 v, float2*) { return v; }
__device__ __forceinline__ float2 to_c(double2 v, float2*) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ double2 to_c(float2 v, double2*) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 to_c(double2 v, double2*) { return v; }

template <typename C>
__device__ __forceinline__ C cfma(C acc, C a, C b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
    return acc;
}

constexpr int kThreads = 256;
constexpr int kOPT = 4;
constexpr int kChunk = 256;  // sites per FP32 partial sum

template <typename CT, typename ST>
__global__ void __launch_bounds__(kThreads)
block_partial_kernel(const __grid_constant__ BlockPlan plan, const ST *__restrict__ Su,
                     const ST *__restrict__ Sd, int V, int n_slices, int chunk, int ns_tile,
                     double2 *__restrict__ partials) {
    using C = typename Cx<CT>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sS = reinterpret_cast<C *>(smem_raw);
    const int nc = plan.n_chi, nc2 = nc * nc, nc3 = nc2 * nc;
    const int nr0 = plan.n_rows[0], nr1 = plan.n_rows[1], nr = nr0 + nr1;
    C *sX = sS + (size_t)ns_tile * nr * nc;

    const int slice = blockIdx.x;
    const int x_begin = blockIdx.y * chunk;
    const int x_end = min(V, x_begin + chunk);
    const int out0 = blockIdx.z * (kThreads * kOPT);

    int o_os[kOPT], o_i1[kOPT], o_i23[kOPT], o_f[kOPT];
    C acc[kOPT];
#pragma unroll
    for (int k = 0; k < kOPT; ++k) {
        const int out = out0 + threadIdx.x + k * kThreads;
        o_os[k] = -1;
        acc[k].x = 0; acc[k].y = 0;
        if (out < plan.n_out) {
            o_os[k] = out / nc3;
            o_i1[k] = (out / nc2) % nc;
            o_i23[k] = out % nc2;
            o_f[k] = plan.f1[o_os[k] / plan.n_spin];
        }
    }

    const ST *slice_u = Su + (size_t)slice * V * 144;
    const ST *slice_d = Sd + (size_t)slice * V * 144;
    for (int xb = x_begin; xb < x_end; xb += ns_tile) {
        const int ns = min(ns_tile, x_end - xb);
        // stage the rows of S used by the tables: sS[site][row][i] (flavour 0 rows first)
        for (int e = threadIdx.x; e < ns * nr * nc; e += kThreads) {
            const int site = e / (nr * nc);
            const int rem = e - site * nr * nc;
            const int rc = rem / nc, ic = rem - (rem / nc) * nc;
            const int f = rc < nr0 ? 0 : 1;
            const int row = f == 0 ? plan.rows[0][rc] : plan.rows[1][rc - nr0];
            const size_t idx = (size_t)(xb + site) * 144 + row * 12 + plan.chi[ic];
            sS[e] = to_c(f == 0 ? slice_u[idx] : slice_d[idx], (C *)nullptr);
        }
        __syncthreads();
        // diquark lists X[site][l][i2 * nc + i3]
        for (int e = threadIdx.x; e < ns * plan.n_x * nc2; e += kThreads) {
            const int site = e / (plan.n_x * nc2);
            const int rem = e - site * plan.n_x * nc2;
            const int l = rem / nc2, i23 = rem - l * nc2;
            const int i2 = i23 / nc, i3 = i23 - i2 * nc;
            const int f1 = plan.f1[plan.x_op[l]];
            const C *s1 = sS + (size_t)site * nr * nc + (f1 == 0 ? 0 : nr0 * nc);
            const C *s2 = sS + (size_t)site * nr * nc + (f1 == 0 ? nr0 * nc : 0);
            C v; v.x = 0; v.y = 0;
            for (int t = plan.x_off[l]; t < plan.x_off[l + 1]; ++t) {
                C a = s1[plan.xt_r2[t] * nc + i2];
                const CT w = (CT)plan.xt_w[t];
                a.x *= w; a.y *= w;
                v = cfma(v, a, s2[plan.xt_r3[t] * nc + i3]);
            }
            sX[e] = v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kOPT; ++k) {
            if (o_os[k] < 0) continue;
            const int os = o_os[k];
            for (int site = 0; site < ns; ++site) {
                const C *s1 = sS + (size_t)site * nr * nc + (o_f[k] == 0 ? 0 : nr0 * nc);
                const C *xs = sX + (size_t)site * plan.n_x * nc2;
                for (int t = plan.os_off[os]; t < plan.os_off[os + 1]; ++t)
                    acc[k] = cfma(acc[k], s1[plan.os_r1[t] * nc + o_i1[k]], xs[plan.os_x[t] * nc2 + o_i23[k]]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < kOPT; ++k) {
        const int out = out0 + threadIdx.x + k * kThreads;
        if (out < plan.n_out)
            partials[((size_t)blockIdx.y * n_slices + slice) * plan.n_out + out] =
                make_double2((double)acc[k].x, (double)acc[k].y);
    }
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

template <typename CT, typename ST>
int launch_typed(const BlockPlan &plan, const void *Su, const void *Sd, int V, int n_slices,
                 double2 *partials, int n_splits, int chunk, double2 *blocks, cudaStream_t stream) {
    using C = typename Cx<CT>::type;
    const int nr = plan.n_rows[0] + plan.n_rows[1];
    const size_t per_site = sizeof(C) * ((size_t)nr * plan.n_chi + (size_t)plan.n_x * plan.n_chi * plan.n_chi);
    int ns = (int)((96 * 1024) / per_site);
    ns = ns < 1 ? 1 : (ns > 16 ? 16 : ns);
    const size_t smem = per_site * ns;
    auto kern = block_partial_kernel<CT, ST>;
    WICK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int n_oc = (plan.n_out + kThreads * kOPT - 1) / (kThreads * kOPT);
    dim3 grid(n_slices, n_splits, n_oc);
    kern<<<grid, kThreads, smem, stream>>>(plan, (const ST *)Su, (const ST *)Sd, V, n_slices, chunk, ns,
                                           partials);
    WICK_CUDA_TRY(cudaGetLastError());
    const size_t n = (size_t)n_slices * plan.n_out;
    block_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(partials, n_splits, n_slices,
                                                                         plan.n_out, plan.n_chi, blocks);
    WICK_CUDA_TRY(cudaGetLastError());
    return WICK_OK;
}

}  // namespace

size_t block_partials_bytes(const BlockPlan &plan, int V, int n_slices, int precision, int *n_splits,
                            int *chunk) {
    (void)precision;
    *chunk = kChunk;
    *n_splits = (V + kChunk - 1) / kChunk;
    return sizeof(double2) * (size_t)(*n_splits) * n_slices * plan.n_out;
}

int launch_block_build(const BlockPlan &plan, const void *Su, int dtype_u, const void *Sd, int dtype_d,
                       int V, int n_slices, int precision, double *partials, int n_splits, int chunk,
                       double2 *blocks, cudaStream_t stream) {
    if (dtype_u != dtype_d) return WICK_EINVAL;
    double2 *part = reinterpret_cast<double2 *>(partials);
    if (precision == WICK_MIXED) {
        if (dtype_u == WICK_C64)
            return launch_typed<float, float2>(plan, Su, Sd, V, n_slices, part, n_splits, chunk, blocks, stream);
        return launch_typed<float, double2>(plan, Su, Sd, V, n_slices, part, n_splits, chunk, blocks, stream);
    }
    if (dtype_u == WICK_C64)
        return launch_typed<double, float2>(plan, Su, Sd, V, n_slices, part, n_splits, chunk, blocks, stream);
    return launch_typed<double, double2>(plan, Su, Sd, V, n_slices, part, n_splits, chunk, blocks, stream);
}

}  // namespace wick
