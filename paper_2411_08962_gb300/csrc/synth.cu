// Synthetic propagators generated on the device (input generation only; it
// holds none of the correlator arithmetic).  Same definition as the host
// generator of the Python package: counter-based SplitMix64 (Steele, Lea,
// Flood 2014), value i of the stream with key k = mix64(k + (i + 1) * gamma),
// and the Box-Muller transform with variance 1/2 per component:
//   u1 = ((r_{2n} >> 11) + 1) 2^-53,  u2 = (r_{2n+1} >> 11) 2^-53,
//   S_n = sqrt(-ln u1) (cos 2 pi u2 + i sin 2 pi u2)
// for entry n of the flat [t][x][a][alpha][b][beta] index of one
// (flavour, source) stream, key = mix64(mix64(seed + gamma (flavour + 1)) + gamma (src + 1)).
// The transcendental functions are CUDA's, so values can differ from the
// host generator's in the last bits.
#include "common.cuh"

namespace wick {
namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
inline uint64_t sm_mix_host(uint64_t z) { return sm_mix(z); }

template <typename C>
__global__ void synth_kernel(uint64_t key, uint64_t n, C *__restrict__ out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t r0 = sm_mix(key + (2 * i + 1) * kGamma);
        const uint64_t r1 = sm_mix(key + (2 * i + 2) * kGamma);
        const double u1 = ((double)(r0 >> 11) + 1.0) * (1.0 / 9007199254740992.0);
        const double u2 = (double)(r1 >> 11) * (1.0 / 9007199254740992.0);
        const double rad = sqrt(-log(u1));
        double s, c;
        sincospi(2.0 * u2, &s, &c);
        if constexpr (sizeof(C) == 8) out[i] = make_float2((float)(rad * c), (float)(rad * s));
        else out[i] = make_double2(rad * c, rad * s);
    }
}

}  // namespace
}  // namespace wick

extern "C" int wick_synth_propagator(uint64_t seed, int flavour, int src, int L, int T, int dtype, void *out,
                                     wick_stream_t stream) {
    using namespace wick;
    if (!out || L < 1 || T < 1 || src < 0 || (flavour != WICK_U && flavour != WICK_D)) return WICK_EINVAL;
    if (dtype != WICK_C64 && dtype != WICK_C128) return WICK_EINVAL;
    if ((uintptr_t)out % 16) return WICK_EINVAL;
    const uint64_t key = sm_mix_host(sm_mix_host(seed + kGamma * (uint64_t)(flavour + 1)) + kGamma * (uint64_t)(src + 1));
    const uint64_t n = (uint64_t)T * L * L * L * 144;
    int dev = 0, n_sm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const unsigned blocks = (unsigned)(n_sm * 8);
    if (dtype == WICK_C64) synth_kernel<float2><<<blocks, 256, 0, (cudaStream_t)stream>>>(key, n, (float2 *)out);
    else synth_kernel<double2><<<blocks, 256, 0, (cudaStream_t)stream>>>(key, n, (double2 *)out);
    WICK_CUDA_TRY(cudaGetLastError());
    return WICK_OK;
}
