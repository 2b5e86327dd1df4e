// Correlator from the reduced term table (Eq. 2.6 generalised in App. D):
//   C[slice] = scale * sum_u w_u prod_k B[slice][id_{u,k}]
//
// grid = (slice, term chunk).  A CTA stages its slice's blocks in shared
// memory when they fit (complex128 for FP64, complex64 for MIXED), then each
// thread walks the chunk's terms with stride blockDim (coalesced reads of the
// uint16 ids and int64 weights), multiplies the A gathered block entries and
// accumulates in FP64.  MIXED keeps every block entry as a double-FP32 pair
// and forms the products with error-free float operations (about 44 bits),
// so the float pipes do the products and only the term sum is FP64.  The CTA reduces in a fixed tree; a second kernel sums
// the chunk partials in chunk order.  Both orders are fixed: the result is
// bitwise reproducible.
#include <type_traits>

#include "common.cuh"
#include "df32.cuh"

namespace wick {

namespace {

constexpr int kThreads = 256;
constexpr int kMinTermsPerChunk = 2048;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ cdf to_cdf(double2 v) { return {split_double(v.x), split_double(v.y)}; }

template <bool MIXED>
struct Elem;
template <>
struct Elem<true> {
    using T = cdf;
    static __device__ __forceinline__ T from(double2 v) { return to_cdf(v); }
    static __device__ __forceinline__ T mul(const T &a, const T &b) { return cdf_mul(a, b); }
    static __device__ __forceinline__ double re(const T &a) { return to_double(a.x); }
    static __device__ __forceinline__ double im(const T &a) { return to_double(a.y); }
};
template <>
struct Elem<false> {
    using T = double2;
    static __device__ __forceinline__ T from(double2 v) { return v; }
    static __device__ __forceinline__ T mul(const T &a, const T &b) { return cmul(a, b); }
    static __device__ __forceinline__ double re(const T &a) { return a.x; }
    static __device__ __forceinline__ double im(const T &a) { return a.y; }
};

template <int A, bool MIXED, bool SMEM>
__global__ void __launch_bounds__(kThreads)
contract_kernel(const double2 *__restrict__ blocks, int n_blk, int64_t U, const uint16_t *__restrict__ ids,
                const int64_t *__restrict__ w, int64_t chunk, int n_slices, double2 *__restrict__ partials) {
    using E = Elem<MIXED>;
    using C = typename E::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sB = reinterpret_cast<C *>(smem_raw);
    const int slice = blockIdx.x;
    const double2 *gB = blocks + (size_t)slice * n_blk;
    if constexpr (SMEM) {
        for (int i = threadIdx.x; i < n_blk; i += kThreads) sB[i] = E::from(gB[i]);
        __syncthreads();
    }
    const int64_t u0 = (int64_t)blockIdx.y * chunk;
    const int64_t u1 = min(U, u0 + chunk);
    double ax = 0.0, ay = 0.0;
    for (int64_t u = u0 + threadIdx.x; u < u1; u += kThreads) {
        const uint16_t *id = ids + u * A;
        C p;
        if constexpr (SMEM) p = sB[id[0]];
        else p = E::from(__ldg(gB + id[0]));
#pragma unroll
        for (int k = 1; k < A; ++k) {
            C b;
            if constexpr (SMEM) b = sB[id[k]];
            else b = E::from(__ldg(gB + id[k]));
            p = E::mul(p, b);
        }
        const double wu = (double)w[u];
        ax = fma(wu, E::re(p), ax);
        ay = fma(wu, E::im(p), ay);
    }
    __shared__ double rx[kThreads], ry[kThreads];
    rx[threadIdx.x] = ax;
    ry[threadIdx.x] = ay;
    __syncthreads();
    for (int off = kThreads / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            rx[threadIdx.x] += rx[threadIdx.x + off];
            ry[threadIdx.x] += ry[threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[(size_t)blockIdx.y * n_slices + slice] = make_double2(rx[0], ry[0]);
}

__global__ void contract_finish_kernel(const double2 *__restrict__ partials, int n_chunks, int n_slices,
                                       double scale, double2 *__restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_slices) return;
    double x = 0, y = 0;
    for (int c = 0; c < n_chunks; ++c) {
        const double2 v = partials[(size_t)c * n_slices + s];
        x += v.x;
        y += v.y;
    }
    out[s] = make_double2(scale * x, scale * y);
}

template <int A, bool MIXED>
int launch_a(const double2 *blocks, int n_slices, int n_blk, int64_t U, const uint16_t *ids, const int64_t *w,
             int64_t chunk, int n_chunks, double2 *partials, cudaStream_t stream) {
    const size_t smem = sizeof(typename Elem<MIXED>::T) * (size_t)n_blk;
    dim3 grid(n_slices, n_chunks);
    if (smem <= 200 * 1024) {
        auto k = contract_kernel<A, MIXED, true>;
        WICK_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k<<<grid, kThreads, smem, stream>>>(blocks, n_blk, U, ids, w, chunk, n_slices, partials);
    } else {
        contract_kernel<A, MIXED, false><<<grid, kThreads, 0, stream>>>(blocks, n_blk, U, ids, w, chunk, n_slices,
                                                                        partials);
    }
    WICK_CUDA_TRY(cudaGetLastError());
    return WICK_OK;
}

template <bool MIXED>
int launch_p(int A, const double2 *blocks, int n_slices, int n_blk, int64_t U, const uint16_t *ids,
             const int64_t *w, int64_t chunk, int n_chunks, double2 *partials, cudaStream_t stream) {
    switch (A) {
        case 1: return launch_a<1, MIXED>(blocks, n_slices, n_blk, U, ids, w, chunk, n_chunks, partials, stream);
        case 2: return launch_a<2, MIXED>(blocks, n_slices, n_blk, U, ids, w, chunk, n_chunks, partials, stream);
        case 3: return launch_a<3, MIXED>(blocks, n_slices, n_blk, U, ids, w, chunk, n_chunks, partials, stream);
        case 4: return launch_a<4, MIXED>(blocks, n_slices, n_blk, U, ids, w, chunk, n_chunks, partials, stream);
        case 5: return launch_a<5, MIXED>(blocks, n_slices, n_blk, U, ids, w, chunk, n_chunks, partials, stream);
        case 6: return launch_a<6, MIXED>(blocks, n_slices, n_blk, U, ids, w, chunk, n_chunks, partials, stream);
        case 7: return launch_a<7, MIXED>(blocks, n_slices, n_blk, U, ids, w, chunk, n_chunks, partials, stream);
        case 8: return launch_a<8, MIXED>(blocks, n_slices, n_blk, U, ids, w, chunk, n_chunks, partials, stream);
        default: return WICK_EINVAL;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Fixed scratch of wick_contract_noalloc: the FP64 partial sums, one complex128
// per (term chunk, slice), in a file-scope device array instead of the
// library's cudaMalloc'd workspace.  Every device that loads the library holds
// these kNoAllocPartials * 16 bytes (1 MiB) until the process exits.  Each call
// writes every partial it later reads, so nothing has to start at zero.
// ---------------------------------------------------------------------------
static __device__ __align__(256) double2 g_noalloc_partials[kNoAllocPartials];

int noalloc_partials(double2 **ptr, size_t *capacity) {
    // In host code the array's name is only a host-side stand-in; its device
    // address comes from the runtime for the device that is current now.  It
    // is looked up on every call (no allocation, a table lookup once the
    // module is loaded), so a context that was reset or replaced never sees a
    // stale address.
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess || !p) {
        (void)cudaGetLastError();
        return WICK_ECUDA;
    }
    *ptr = static_cast<double2 *>(p);
    *capacity = kNoAllocPartials;
    return WICK_OK;
}

size_t contract_partials_bytes(int n_slices, int64_t U, int A, int n_blk, int *n_chunks) {
    (void)A; (void)n_blk;
    int dev = 0, n_sm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    // enough CTAs for two waves, but never chunks of fewer than kMinTermsPerChunk terms
    int64_t want = (2 * (int64_t)n_sm + n_slices - 1) / n_slices;
    const int64_t most = (U + kMinTermsPerChunk - 1) / kMinTermsPerChunk;
    if (want > most) want = most;
    if (want < 1) want = 1;
    *n_chunks = (int)want;
    return sizeof(double2) * (size_t)want * n_slices;
}

int launch_contract(const double2 *blocks, int n_slices, int n_blk, int A, int64_t U, const uint16_t *ids,
                    const int64_t *w, double scale, int precision, double2 *C_out, double *partials_raw,
                    int n_chunks, cudaStream_t stream) {
    double2 *partials = reinterpret_cast<double2 *>(partials_raw);
    const int64_t chunk = (U + n_chunks - 1) / n_chunks;
    int e = precision == WICK_MIXED
                ? launch_p<true>(A, blocks, n_slices, n_blk, U, ids, w, chunk > 0 ? chunk : 1, n_chunks, partials, stream)
                : launch_p<false>(A, blocks, n_slices, n_blk, U, ids, w, chunk > 0 ? chunk : 1, n_chunks, partials, stream);
    if (e) return e;
    contract_finish_kernel<<<(n_slices + 127) / 128, 128, 0, stream>>>(partials, n_chunks, n_slices, scale, C_out);
    WICK_CUDA_TRY(cudaGetLastError());
    return WICK_OK;
}

namespace {
__global__ void product_kernel(const double2 *__restrict__ a, const double2 *__restrict__ b, int64_t n,
                               double2 *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = cmul(a[i], b[i]);
}
}  // namespace

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
