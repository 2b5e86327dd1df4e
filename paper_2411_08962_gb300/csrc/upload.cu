// Upload of the propagator rows a block build reads: a gather from page-locked
// host memory (device-mapped) to a device propagator of the same layout.
#include "common.cuh"

namespace wick {

namespace {

// One warp per site: lane k copies the 16-byte words k, k + 32, ... of the site's row runs (three
// loads in flight per lane); the word list is loaded once per thread.  CTAs of 128 threads with at
// most 64 registers (8192 in all), so that one fits beside a block-build CTA on the same SM.
__global__ void __launch_bounds__(128, 8) upload_rows_kernel(const __grid_constant__ UploadMap map,
                                                             const uint4 *__restrict__ hu,
                                                             const uint4 *__restrict__ hd, uint4 *__restrict__ du,
                                                             uint4 *__restrict__ dd, size_t n_sites, int words_u,
                                                             int words_d) {
    constexpr int kPerLane = (kMaxUploadWords + 31) / 32;   // 9
    static_assert(kPerLane % 3 == 0, "groups of three");
    const int lane = threadIdx.x & 31;
    int wd[kPerLane];
#pragma unroll
    for (int i = 0; i < kPerLane; ++i) {
        const int k = lane + 32 * i;
        wd[i] = k < map.n ? map.word[k] : -1;
    }
    const size_t warp0 = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5;
    const size_t n_warps = ((size_t)gridDim.x * blockDim.x) >> 5;
    for (size_t site = warp0; site < n_sites; site += n_warps) {
        const uint4 *su = hu + site * words_u, *sd = hd + site * words_d;
        uint4 *tu = du + site * words_u, *td = dd + site * words_d;
#pragma unroll
        for (int i0 = 0; i0 < kPerLane; i0 += 3) {
            uint4 v[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const int w = wd[i0 + i];
                if (w >= 0) v[i] = (w >> 15) ? sd[w & 0x7FFF] : su[w & 0x7FFF];
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const int w = wd[i0 + i];
                if (w >= 0) {
                    if (w >> 15) td[w & 0x7FFF] = v[i];
                    else tu[w & 0x7FFF] = v[i];
                }
            }
        }
    }
}

}  // namespace

int launch_upload_rows(const UploadMap &map, const void *hu, const void *hd, const void *du, const void *dd,
                       size_t n_sites, int words_u, int words_d, cudaStream_t stream) {
    int dev = 0, n_sm = 0;
    WICK_CUDA_TRY(cudaGetDevice(&dev));
    WICK_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    const size_t warps = n_sites < (size_t)n_sm * 16 ? n_sites : (size_t)n_sm * 16;   // 4 CTAs per SM
    const unsigned blocks = (unsigned)((warps * 32 + 127) / 128);
    upload_rows_kernel<<<blocks, 128, 0, stream>>>(map, (const uint4 *)hu, (const uint4 *)hd,
                                                   (uint4 *)const_cast<void *>(du), (uint4 *)const_cast<void *>(dd),
                                                   n_sites, words_u, words_d);
    WICK_CUDA_TRY(cudaGetLastError());
    return WICK_OK;
}

}  // namespace wick
