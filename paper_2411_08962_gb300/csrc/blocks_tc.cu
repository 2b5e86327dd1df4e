// Baryon blocks (Eq. 2.4/2.5) with the update over sites on the tensor cores,
// exactly.
//
// For one block type o the update is a complex GEMM over sites and colour terms:
//   P_o[(s,c1)][c23] = sum_{x,a} U(x)[(a,s)][c1] * X_{o,a}(x)[c23]
// with U the pair-flavour propagator rows and X the diquark lists (blocks.cu).
// As a real GEMM -- rows (part, s, c1), K = (x, a, part) -- it runs on
// tcgen05.mma kind::f16 with bf16 operands and FP32 accumulators in TMEM.
//
// Exactness (an Ozaki-type error-free splitting).  Every U value is cut into
// 5 slices on a fixed-point grid 2^E (E bounds the |components| of its colour
// c1 over the CTA's sites), every X value -- a double-FP32 number -- into 6
// slices on a grid 2^F of its column (2^F >= sum|w| max|u| max|d|):
//     v = 2^E * sum_i q_i 2^(-7-8i),   |q_i| <= 128   (39 / 47 bits)
// A slice is an integer of at most 128 in magnitude, exact in bf16; a slice
// product is at most 2^14 in magnitude, and a sum of K <= 768 of them (128
// sites) below 2^24, so the FP32 accumulation in TMEM is exact for a whole
// round of 128 sites.  The pair (i, j) carries the weight 2^(E+F-14-8(i+j));
// pairs with i + j <= 5 are kept.  The grids bound the largest values of a
// 512-site range, so typical X values sit ~6 bits below 2^F: with 5 x 5 slices
// and i + j <= 4 the blocks came out ~1e-9 relative, with 5 x 6 and i + j <= 5
// ~5e-12 (the same class as the double-FP32 CUDA-core kernel).
// Each round's accumulators are scaled by that exact power of two and added in
// double-FP32 relative to 2^(E+F); the five U-slice rows of an output are
// combined at the end and converted to FP64.
//
// Layout.  The U slices are stacked along M (row i*R + r, R = 2 n_spin n_chi)
// and cut into M tiles of 128 rows; tile t meets only the X slices
// j <= 5 - (first slice in t), one MMA each (6 for the upper-spin tables,
// 6+5+4+2 for the full-spin ones).  A CTA owns (block type, column tile of the
// (c2, c3) columns, range of 512 sites, slice); the first two vary fastest in
// the grid so that the CTAs reading the same rows of S run together.  Per chunk
// of 16 sites (upper tables; 8 for the full-spin ones, for shared memory):
// the CTA builds the U and X slices of chunk c into one of two operand buffers
// from S staged two chunks ahead (three staging buffers, cp.async), meets at one
// barrier, and one thread of the least-loaded warp issues the chunk's MMAs and
// commits them to the buffer's mbarrier while the others go on to chunk c + 1.  The work of a chunk
// is a list of jobs -- one X value, or two U values -- ordered so that every
// warp does one kind.  Every wait on an mbarrier is bounded.
#include <cuda_bf16.h>

#include <cstring>

#include "common.cuh"
#include "df32.cuh"

namespace wick {

namespace {

constexpr int kThr = 512;                          // 16 warps
constexpr int kSlices = 5;                         // slices of U
constexpr int kSlicesX = 6;                        // slices of X
constexpr int kMaxPair = 5;                        // kept slice pairs: i + j <= kMaxPair
constexpr int kKa = 3;                             // colour-term slots per site
constexpr int kRoundSites = 128;                   // sites per exact TMEM accumulation
constexpr int kRangeSites = 512;                   // sites per CTA (one grid, one partial)
constexpr int kSpinLimit = 1 << 22;                // mbarrier polls before giving up
constexpr int kStage = 3;                          // staging buffers
constexpr int kMaxRows = 24;                       // staged S rows (both flavours)

// exponent bound of the largest colour-list weight sum, per block type
struct WeightExp {
    int e[kMaxOps];
};

// Compile-time shape of a table family: NC colours chi, NS spins, NT columns
// per MMA (multiple of 16), NMT M tiles, NX sites per operand chunk.
template <int NC_, int NS_, int NT_, int NMT_, int NX_> struct Shape {
    static constexpr int NC = NC_, NS = NS_, NT = NT_, NMT = NMT_, NX = NX_;
    static constexpr int KC = NX * kKa * 2;                 // K per chunk
    static constexpr int CHUNKS_PER_ROUND = kRoundSites / NX;
    static constexpr int NC2 = NC * NC;
    static constexpr int R = 2 * NS * NC;                   // real rows per U slice
    static constexpr int NCTA = NT >= NC2 ? NC2 : NT;       // (c2, c3) columns per CTA
    static constexpr int NCT = (NC2 + NT - 1) / NT;         // column tiles
    static constexpr int PER_TILE = 4 / NMT;                // warps of a lane quarter per M tile
    static constexpr int CW = NT / PER_TILE;                // readout columns per thread
    static constexpr int NXJOB = NX * kKa * NCTA;           // one X value each
    static constexpr int NUJOB = NX * kKa / 2 * NS * NC;    // two U values each
    static constexpr int jmax(int t) {
        return kSlicesX < kMaxPair + 1 - t * 128 / R ? kSlicesX : kMaxPair + 1 - t * 128 / R;
    }
    static constexpr int toff(int t, int j) {
        int c = 0;
        for (int u = 0; u < t; ++u) c += jmax(u) * NT;
        return c + j * NT;
    }
    static constexpr int TMEM_USED = toff(NMT - 1, 0) + jmax(NMT - 1) * NT;
    static constexpr int TMEM_COLS = TMEM_USED <= 32 ? 32 : TMEM_USED <= 64 ? 64 : TMEM_USED <= 128 ? 128
                                   : TMEM_USED <= 256 ? 256 : 512;
    static constexpr int A_BYTES = NMT * 128 * KC * 2;
    static constexpr int B_BYTES = kSlicesX * NT * KC * 2;
    static constexpr int S_BYTES = NX * kMaxRows * NC * 8;  // float2 staging
    static constexpr int SMEM = 2 * (A_BYTES + B_BYTES) + kStage * S_BYTES + 4 * (16 + 256) + 16 * kKa * 4 + 64 + 32;
    static_assert(NMT * 128 >= kSlices * R && (NMT - 1) * 128 < kSlices * R, "M tiles");
    static_assert(NC2 <= NT || NC2 % NT == 0, "column tiles");
    static_assert(TMEM_USED <= 512 && CW % 4 == 0 && CW <= 32, "TMEM / readout");
    static_assert(NXJOB % 32 == 0, "X jobs fill whole warps");
    static_assert((NXJOB + NUJOB) % 32 == 0, "U jobs fill whole warps");
    static_assert(R % 8 == 0, "U slices start on a core-matrix row group");
    static_assert(NCTA % 8 == 0 || NCTA % 8 == 4, "X job map");
    static_assert(kSlices * R * NT * 8 <= 2 * (A_BYTES + B_BYTES), "combine buffer");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};
using UpperShape = Shape<6, 2, 48, 1, 16>;   // nucleon upper spin components: 2 x 216 per type
using FullShape = Shape<12, 4, 16, 4, 8>;    // all four spins: 4 x 1728 per type

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// 2^k as a float, k in [-126, 127]
__device__ __forceinline__ float exp2i(int k) {
    k = k < -126 ? -126 : (k > 127 ? 127 : k);
    return __int_as_float((k + 127) << 23);
}

// 2^k as a double, k in [-1022, 1023]
__device__ __forceinline__ double exp2d(int k) {
    k = k < -1022 ? -1022 : (k > 1023 ? 1023 : k);
    return __longlong_as_double((long long)(k + 1023) << 52);
}


// smallest E >= -100 with m < 2^E (m >= 0); -100 stands for "zero"
__host__ __device__ __forceinline__ int exponent_bound(float m) {
    if (!(m > 0.f)) return -100;
    int e;
    frexpf(m, &e);
    return e < -100 ? -100 : e;
}

// K-major bf16 tile of 8x8 core matrices: element (row m, k) of a tile whose rows hold KC values
template <int KC> __device__ __forceinline__ int tile_off(int m, int k) {
    return ((m >> 3) * (KC / 8) + (k >> 3)) * 64 + (m & 7) * 8 + (k & 7);
}

// shared-memory matrix descriptor: no swizzle, core matrices 128 B apart along K, 8-row groups KC/8*128 B apart
template <int KC> __device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)((KC / 8 * 128) >> 4) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of the sm_100 family
    return d;
}


__device__ __forceinline__ float2 to_f2(float2 v) { return v; }
__device__ __forceinline__ float2 to_f2(double2 v) { return make_float2((float)v.x, (float)v.y); }

__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Poll the mbarrier for `parity` at most kSpinLimit times (this thread only).
__device__ __forceinline__ bool poll_parity(uint64_t *mbar, int parity) {
    uint32_t done = 0;
    for (int it = 0; it < kSpinLimit && !done; ++it)
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(parity)
            : "memory");
    return done != 0;
}

// Grids of one (slice, range of kRangeSites sites): for flavour f and colour
// column ic over the rows the tables use, E = bound of max(|re|, |im|) and
// G = bound of max(|re| + |im|).  bounds[(slice * n_ranges + range) * 48 + f * 24 + kind * 12 + ic].
template <typename ST>
__global__ void __launch_bounds__(256)
tc_bounds_kernel(const __grid_constant__ BlockPlan plan, const ST *__restrict__ Su, const ST *__restrict__ Sd,
                 int V, int n_ranges, int *__restrict__ bounds) {
    __shared__ unsigned smax[48];  // [f][kind][ic]
    const int tid = threadIdx.x;
    if (tid < 48) smax[tid] = 0u;
    __syncthreads();
    const int rng = blockIdx.x, slice = blockIdx.y;
    const int nc = plan.n_chi, nr0 = plan.n_rows[0], nr = nr0 + plan.n_rows[1];
    const int cols = nr * nc;
    const int parts = max(1, (int)blockDim.x / cols);
    const int x_begin = rng * kRangeSites, x_end = min(V, x_begin + kRangeSites);
    for (int e = tid; e < cols * parts; e += blockDim.x) {
        const int col = e % cols, part = e / cols;
        const int rc = col / nc, ic = col % nc;
        const int f = rc < nr0 ? 0 : 1;
        const int row = f == 0 ? plan.rows[0][rc] : plan.rows[1][rc - nr0];
        const ST *src = (f == 0 ? Su : Sd) + (size_t)slice * V * 144 + row * 12 + plan.chi[ic];
        float m1 = 0.f, m2 = 0.f;
#pragma unroll 8
        for (int x = x_begin + part; x < x_end; x += parts) {
            const float2 v = to_f2(src[(size_t)x * 144]);
            const float ax = fabsf(v.x), ay = fabsf(v.y);
            m1 = fmaxf(m1, fmaxf(ax, ay));
            m2 = fmaxf(m2, __fadd_ru(ax, ay));  // rounded up: still a bound of |re| + |im|
        }
        atomicMax(&smax[f * 24 + ic], __float_as_uint(m1));
        atomicMax(&smax[f * 24 + 12 + ic], __float_as_uint(m2));
    }
    __syncthreads();
    if (tid < 48) {
        const int ic = tid % 12;
        int *out = bounds + ((size_t)slice * n_ranges + rng) * 48;
        out[tid] = ic < nc ? exponent_bound(__uint_as_float(smax[tid])) : -100;
    }
}

// Packed slicing: lanes (re, im) of a complex value at once on the f32x2
// instructions.  Rounding to the nearest integer adds and subtracts 1.5 * 2^23
// (exact for |t| < 2^22); a slice, an integer of at most 128 in magnitude, is
// exact in bf16, whose bits are the upper half of the float's.
// U: v = 2^E sum_i q_i 2^(-7-8i); returns the re-row word (q_re, -q_im) and the
// im-row word (q_im, q_re) of every slice as bf16x2.
// sc = 2^(7-E), a power of two (clamped to the float range; zero rows stay zero)
__device__ __forceinline__ void slice_u2(float2 v, float sc, uint32_t *wre, uint32_t *wim) {
    const f2x magic = pk(12582912.f, 12582912.f), k256 = pk(256.f, 256.f);
    f2x r = mul2(pk(v.x, v.y), pk(sc, sc));  // exact: power-of-two scale
#pragma unroll
    for (int i = 0; i < kSlices; ++i) {
        const f2x q = sub2(add2(r, magic), magic);
        uint32_t lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "l"(q));
        wre[i] = __byte_perm(lo, hi, 0x7632) ^ 0x80000000u;  // (q_re, -q_im)
        wim[i] = __byte_perm(hi, lo, 0x7632);                // (q_im, q_re)
        r = mul2(sub2(r, q), k256);
    }
}

// X = (h + l) lane-wise: 2^F sum_j q_j 2^(-7-8j) + O(2^(F-48)); words (q_re, q_im) per slice;
// sc = 2^(7-F)
__device__ __forceinline__ void slice_x2(f2x h, f2x l, float sc, uint32_t *w) {
    const f2x magic = pk(12582912.f, 12582912.f), k256 = pk(256.f, 256.f), s2 = pk(sc, sc);
    f2x rh = mul2(h, s2), rl = mul2(l, s2);
#pragma unroll
    for (int j = 0; j < kSlicesX; ++j) {
        const f2x q = sub2(add2(rh, magic), magic);
        uint32_t lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "l"(q));
        w[j] = __byte_perm(lo, hi, 0x7632);
        // (rh - q) + rl exactly as a pair (TwoSum), then the next 8 bits up
        const f2x d = sub2(rh, q);
        const f2x t = add2(d, rl);
        const f2x bb = sub2(t, d);
        const f2x e = add2(sub2(d, sub2(t, bb)), sub2(rl, bb));
        rh = mul2(t, k256);
        rl = mul2(e, k256);
    }
}

constexpr int kListLen = 4;  // terms per diquark list the tensor-core path takes (exactly)

// double-FP32 list sum X_{o,a}[c23] of one staged site (lanes re, im).  term[t] = (row2 * NC,
// row3 * NC, weight bits): the list's terms, staged in shared memory; all loads first.
__device__ __forceinline__ pdf x_value(const int4 *term, const float2 *s1, const float2 *s2) {
    int4 tt[kListLen];
#pragma unroll
    for (int t = 0; t < kListLen; ++t) tt[t] = term[t];
    float2 u[kListLen], d[kListLen];
#pragma unroll
    for (int t = 0; t < kListLen; ++t) {
        u[t] = s1[tt[t].x];
        d[t] = s2[tt[t].y];
    }
    // one packed accumulator with lanes (re, im): w u d = (ax dx - ay dy, ax dy + ay dx) is the sum of
    // the lane products (ax, ax) (dx, dy) and (-ay, ay) (dy, dx), each exact as a TwoProd pair; the
    // first product starts the accumulator without a TwoSum
    pdf acc;
    {
        const float w = __int_as_float(tt[0].z);
        const float ax = w * u[0].x, ay = w * u[0].y;  // exact: w is +-2^k
        const f2x B1 = pk(d[0].x, d[0].y), B2 = pk(d[0].y, d[0].x);
        const f2x nA1 = pk(-ax, -ax);
        const f2x np = mul2(nA1, B1);                   // -RN(A1 B1)
        acc.h = sub2(0ull, np);
        acc.l = fma2(pk(ax, ax), B1, np);               // A1 B1 - RN(A1 B1)
        pacc_exact(acc, pk(-ay, ay), pk(ay, -ay), B2);
    }
#pragma unroll
    for (int t = 1; t < kListLen; ++t) {
        const float w = __int_as_float(tt[t].z);
        const float ax = w * u[t].x, ay = w * u[t].y;
        const f2x B1 = pk(d[t].x, d[t].y), B2 = pk(d[t].y, d[t].x);
        pacc_exact(acc, pk(ax, ax), pk(-ax, -ax), B1);
        pacc_exact(acc, pk(-ay, ay), pk(ay, -ay), B2);
    }
    return acc;
}

// X job jb -> (column n, combo gc = (site, a)).  A warp takes 8 columns x 4
// combos: its 32-bit stores then fall on 8 rows x 4 words of a core matrix,
// 32 different banks (the leftover 4 columns of a 36-column tile: 4 x 8, two
// ways).  Consecutive columns of one combo would meet only 8 banks.
template <typename SH> __device__ __forceinline__ void x_map(int jb, int &n, int &gc) {
    constexpr int NG = SH::NCTA / 8, GW = SH::NX * kKa / 4;
    const int w = jb >> 5, lane = jb & 31;
    if (w < NG * GW) {
        n = 8 * (w % NG) + (lane & 7);
        gc = 4 * (w / NG) + (lane >> 3);
    } else {
        n = 8 * NG + (lane & 3);
        gc = 8 * (w - NG * GW) + (lane >> 2);
    }
}

// X job jb: column n, combo gc = (site, a); 6 slices into B_j[n][(site, a, part)]
template <typename SH>
__device__ __forceinline__ void x_job(const int4 *sTerm, const float2 *S, int nr, int off1, int off2, int col0,
                                      int n_a, const int *sF, __nv_bfloat16 *B, int jb) {
    constexpr int NC = SH::NC, NT = SH::NT;
    int n, gc;
    x_map<SH>(jb, n, gc);
    const int site = gc / kKa, a = gc % kKa;
    uint32_t w[kSlicesX];
    if (a < n_a) {
        const int c23 = col0 + n;
        const pdf X = x_value(sTerm + a * kListLen, S + site * nr * NC + off1 + c23 / NC,
                              S + site * nr * NC + off2 + c23 % NC);
        slice_x2(X.h, X.l, exp2i(7 - sF[n]), w);
    } else {
#pragma unroll
        for (int j = 0; j < kSlicesX; ++j) w[j] = 0u;
    }
    __nv_bfloat16 *dst = B + tile_off<SH::KC>(n, gc * 2);
#pragma unroll
    for (int j = 0; j < kSlicesX; ++j) *reinterpret_cast<uint32_t *>(dst + j * NT * SH::KC) = w[j];
}

// two X jobs with independent chains (both jA, jB < NXJOB)
template <typename SH>
__device__ __forceinline__ void x_job2(const int4 *sTerm, const float2 *S, int nr, int off1, int off2, int col0,
                                       int n_a, const int *sF, __nv_bfloat16 *B, int jA, int jB) {
    constexpr int NC = SH::NC, NT = SH::NT;
    int nA, gA, nB, gB;
    x_map<SH>(jA, nA, gA);
    x_map<SH>(jB, nB, gB);
    const int aA = gA % kKa, aB = gB % kKa;
    const int cA = col0 + nA, cB = col0 + nB;
    const float2 *bA = S + (gA / kKa) * nr * NC, *bB = S + (gB / kKa) * nr * NC;
    pdf XA = x_value(sTerm + (aA < n_a ? aA : 0) * kListLen, bA + off1 + cA / NC, bA + off2 + cA % NC);
    pdf XB = x_value(sTerm + (aB < n_a ? aB : 0) * kListLen, bB + off1 + cB / NC, bB + off2 + cB % NC);
    if (aA >= n_a) XA.h = XA.l = 0ull;
    if (aB >= n_a) XB.h = XB.l = 0ull;
    uint32_t wA[kSlicesX], wB[kSlicesX];
    slice_x2(XA.h, XA.l, exp2i(7 - sF[nA]), wA);
    slice_x2(XB.h, XB.l, exp2i(7 - sF[nB]), wB);
    __nv_bfloat16 *dA = B + tile_off<SH::KC>(nA, gA * 2), *dB = B + tile_off<SH::KC>(nB, gB * 2);
#pragma unroll
    for (int j = 0; j < kSlicesX; ++j) {
        *reinterpret_cast<uint32_t *>(dA + j * NT * SH::KC) = wA[j];
        *reinterpret_cast<uint32_t *>(dB + j * NT * SH::KC) = wB[j];
    }
}

// U job ju: row (s, c1), combos 2 gp and 2 gp + 1; 5 slices into A[(i, part, s, c1)][(site, a, part')]
template <typename SH>
__device__ __forceinline__ void u_job(const int *sR1, const float2 *S, int nr, int n_a, const int *sEU,
                                      __nv_bfloat16 *A, int ju) {
    constexpr int NC = SH::NC, NS = SH::NS, R = SH::R;
    const int sc1 = ju % (NS * NC), gp = ju / (NS * NC);
    const int s = sc1 / NC, c1 = sc1 % NC;
    const float scu = exp2i(7 - sEU[c1]);
    uint32_t wre[2][kSlices], wim[2][kSlices];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int gc = 2 * gp + h, site = gc / kKa, a = gc % kKa;
        float2 u = make_float2(0.f, 0.f);
        if (a < n_a) u = S[site * nr * NC + sR1[s * kKa + a] + c1];
        slice_u2(u, scu, wre[h], wim[h]);
    }
    // re row: U_re X_re - U_im X_im ; im row: U_im X_re + U_re X_im
    __nv_bfloat16 *dre = A + tile_off<SH::KC>(s * NC + c1, gp * 4), *dim = A + tile_off<SH::KC>(NS * NC + s * NC + c1, gp * 4);
#pragma unroll
    for (int i = 0; i < kSlices; ++i) {
        *reinterpret_cast<uint2 *>(dre + tile_off<SH::KC>(i * R, 0)) = make_uint2(wre[0][i], wre[1][i]);
        *reinterpret_cast<uint2 *>(dim + tile_off<SH::KC>(i * R, 0)) = make_uint2(wim[0][i], wim[1][i]);
    }
}

template <typename ST, typename SH>
__global__ void __launch_bounds__(kThr, 1)
block_tc_kernel(const __grid_constant__ BlockPlan plan, const ST *__restrict__ Su, const ST *__restrict__ Sd,
                int V, int n_slices, int n_ranges, const int *__restrict__ bounds, const WeightExp ew,
                double2 *__restrict__ partials, int *status) {
    constexpr int NC = SH::NC, NS = SH::NS, NT = SH::NT, R = SH::R, NCTA = SH::NCTA;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // the CTAs of one (slice, range) are adjacent in the grid: they read the same rows of S (L2 reuse)
    const int o = blockIdx.x / SH::NCT, ct = blockIdx.x % SH::NCT;
    const int rng = blockIdx.y, slice = blockIdx.z;
    const int nr0 = plan.n_rows[0], nr = nr0 + plan.n_rows[1];
    const int f1 = plan.f1[o];
    const int col0 = ct * NT;
    const int t0 = plan.os_off[o * NS];
    const int n_a = plan.os_off[o * NS + 1] - t0;
    const int off1 = f1 == 0 ? 0 : nr0 * NC, off2 = f1 == 0 ? nr0 * NC : 0;  // flavour rows in a staged site

    __nv_bfloat16 *sA0 = reinterpret_cast<__nv_bfloat16 *>(smem);
    __nv_bfloat16 *sB0 = reinterpret_cast<__nv_bfloat16 *>(smem + 2 * SH::A_BYTES);
    float2 *sS0 = reinterpret_cast<float2 *>(smem + 2 * (SH::A_BYTES + SH::B_BYTES));
    int *sEU = reinterpret_cast<int *>(smem + 2 * (SH::A_BYTES + SH::B_BYTES) + kStage * SH::S_BYTES);
    int *sF = sEU + 16;                                       // [256] grid of X per column
    int4 *sTerm = reinterpret_cast<int4 *>(sF + 256);         // [kKa][kListLen] the op's diquark list terms
    int *sR1 = reinterpret_cast<int *>(sTerm + kKa * kListLen);   // [NS][kKa] staged offset of U's row
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sR1 + 16);      // [2]
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 2);

    // zero both operand buffers once: padding rows and unused colour terms stay zero
    {
        uint4 *z = reinterpret_cast<uint4 *>(smem);
        for (int e = tid; e < 2 * (SH::A_BYTES + SH::B_BYTES) / 16; e += kThr) z[e] = make_uint4(0u, 0u, 0u, 0u);
    }
    const int *bnd = bounds + ((size_t)slice * n_ranges + rng) * 48;
    if (tid < NC) sEU[tid] = bnd[f1 * 24 + tid];
    if (tid < NT) {
        const int c23 = col0 + tid;
        sF[tid] = tid < NCTA ? bnd[f1 * 24 + 12 + c23 / NC] + bnd[(1 - f1) * 24 + 12 + c23 % NC] + ew.e[o] : 0;
    }
    if (tid < kKa * kListLen) {
        const int a = tid / kListLen, t = tid % kListLen;
        int4 v = make_int4(0, 0, 0, 0);
        if (a < n_a) {
            const int q = plan.x_off[plan.os_x[t0 + a]] + t;
            v = make_int4(plan.xt_r2[q] * NC, plan.xt_r3[q] * NC, __float_as_int(plan.xt_w[q]), 0);
        }
        sTerm[tid] = v;
    }
    if (tid >= 32 && tid < 32 + NS * kKa) {
        const int s = (tid - 32) / kKa, a = (tid - 32) % kKa;
        sR1[s * kKa + a] = a < n_a ? off1 + plan.os_r1[plan.os_off[o * NS + s] + a] * NC : 0;
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(SH::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }

    const int x_begin = rng * kRangeSites, x_end = min(V, x_begin + kRangeSites);
    constexpr int NX = SH::NX, KC = SH::KC;
    const int n_chunks = (x_end - x_begin + NX - 1) / NX;
    const ST *su = Su + (size_t)slice * V * 144;
    const ST *sd = Sd + (size_t)slice * V * 144;
    // stage the rows of chunk c: sS[site][row][ic] as float2, flavour-0 rows first (zeros past the range)
    auto stage = [&](int c) {
        float2 *dst = sS0 + (c % kStage) * (SH::S_BYTES / 8);
        const int xb = x_begin + c * NX;
        for (int e = tid; e < NX * nr * NC; e += kThr) {
            const int site = e / (nr * NC);
            const int rem = e - site * nr * NC;
            const int rc = rem / NC, ic = rem - rc * NC;
            const int f = rc < nr0 ? 0 : 1;
            const int row = f == 0 ? plan.rows[0][rc] : plan.rows[1][rc - nr0];
            const ST *src = (f == 0 ? su : sd) + (size_t)(xb + site) * 144 + row * 12 + plan.chi[ic];
            if (xb + site >= x_end) dst[e] = make_float2(0.f, 0.f);
            else if constexpr (sizeof(ST) == 8) cp_async8(dst + e, src);
            else dst[e] = to_f2(*src);
        }
        cp_async_commit();
    };
    stage(0);
    cp_async_wait_all();
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tbase = *tslot;
    if (n_chunks > 1) stage(1);

    // readout ownership: lane quarter q of M tile t_own, column part cpart of the tile's columns
    const int q = warp & 3, g = warp >> 2;
    const int t_own = g / SH::PER_TILE, cpart = g % SH::PER_TILE;
    const int row = t_own * 128 + q * 32 + lane;        // stacked row of this thread
    const int my_i = row / R;
    const bool row_ok = row < kSlices * R;
    const int i_warp = (t_own * 128 + q * 32) / R;      // first slice among the warp's rows
    int jmax_own = 0;
#pragma unroll
    for (int t = 0; t < SH::NMT; ++t)
        if (t == t_own) jmax_own = SH::jmax(t);
    const int j_warp = min(kMaxPair - i_warp, jmax_own - 1);
    df acc[SH::CW];
#pragma unroll
    for (int n = 0; n < SH::CW; ++n) acc[n] = {0.f, 0.f};

    constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);
    int issued0 = 0, issued1 = 0, waited0 = 0, waited1 = 0, bad = 0;

    for (int c = 0; c < n_chunks; ++c) {
        const int buf = c & 1;
        __nv_bfloat16 *A = sA0 + buf * (SH::A_BYTES / 2);
        __nv_bfloat16 *B = sB0 + buf * (SH::B_BYTES / 2);
        const float2 *S = sS0 + (c % kStage) * (SH::S_BYTES / 8);
        // the MMAs of chunk c - 2 read this operand buffer
        if (buf == 0 && waited0 < issued0) {
            if (poll_parity(&mbar[0], waited0 & 1)) ++waited0;
            else bad = 1;
        } else if (buf == 1 && waited1 < issued1) {
            if (poll_parity(&mbar[1], waited1 & 1)) ++waited1;
            else bad = 1;
        }
        if (!bad) {
            // jobs j0 and j0 + kThr per round: two X values are built side by side (independent chains);
            // X jobs come first and fill whole warps, so every branch is warp-uniform
            constexpr int NJ = SH::NXJOB + SH::NUJOB;
            for (int j0 = tid; j0 < NJ; j0 += 2 * kThr) {
                const int jA = j0, jB = j0 + kThr;
                if (jB < SH::NXJOB) {
                    x_job2<SH>(sTerm, S, nr, off1, off2, col0, n_a, sF, B, jA, jB);
                } else {
                    if (jA < SH::NXJOB) x_job<SH>(sTerm, S, nr, off1, off2, col0, n_a, sF, B, jA);
                    else u_job<SH>(sR1, S, nr, n_a, sEU, A, jA - SH::NXJOB);
                    if (jB < NJ) u_job<SH>(sR1, S, nr, n_a, sEU, A, jB - SH::NXJOB);
                }
            }
        }
        // staged rows of chunk c + 1 complete (this thread's copies); operands of chunk c written
        cp_async_wait_all();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        if (__syncthreads_or(bad)) {
            bad = 1;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const bool fresh = c % SH::CHUNKS_PER_ROUND == 0;
        if (tid == kThr - 1) {  // the last warp has the fewest jobs
            const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
#pragma unroll
            for (int ks = 0; ks < KC / 16; ++ks)
#pragma unroll
                for (int t = 0; t < SH::NMT; ++t) {
                    const uint64_t da = smem_desc<KC>(a0 + (uint32_t)(t * 128 * KC * 2 + ks * 256));
#pragma unroll
                    for (int j = 0; j < SH::jmax(t); ++j) {
                        const uint64_t db = smem_desc<KC>(b0 + (uint32_t)(j * NT * KC * 2 + ks * 256));
                        const uint32_t acc_in = (fresh && ks == 0) ? 0u : 1u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
                                tbase + (uint32_t)SH::toff(t, j)),
                            "l"(da), "l"(db), "r"(idesc), "r"(acc_in));
                    }
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar[buf])));
        }
        if (buf) ++issued1;
        else ++issued0;
        // stage chunk c + 2 into the buffer chunk c - 1 was built from
        if (c + 2 < n_chunks) stage(c + 2);

        // end of a round: read the accumulators out of TMEM
        if (c % SH::CHUNKS_PER_ROUND == SH::CHUNKS_PER_ROUND - 1 || c == n_chunks - 1) {
            if (waited0 < issued0) {
                if (poll_parity(&mbar[0], waited0 & 1)) ++waited0;
                else bad = 1;
            }
            if (waited1 < issued1) {
                if (poll_parity(&mbar[1], waited1 & 1)) ++waited1;
                else bad = 1;
            }
            if (__syncthreads_or(bad)) {
                bad = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            for (int j = 0; j <= j_warp; ++j) {
                uint32_t r[SH::CW];
                int toffj = 0;
#pragma unroll
                for (int t = 0; t < SH::NMT; ++t)
                    if (t == t_own) toffj = SH::toff(t, 0) + j * NT;
                const uint32_t taddr = tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(toffj + cpart * SH::CW);
#pragma unroll
                for (int c4 = 0; c4 < SH::CW; c4 += 4)
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                                 : "=r"(r[c4]), "=r"(r[c4 + 1]), "=r"(r[c4 + 2]), "=r"(r[c4 + 3])
                                 : "r"(taddr + (uint32_t)c4));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                if (row_ok && my_i + j <= kMaxPair) {
                    const float scale = exp2i(-14 - 8 * (my_i + j));
#pragma unroll
                    for (int n = 0; n < SH::CW; ++n) acc_add(acc[n], df{__fmul_rn(__uint_as_float(r[n]), scale), 0.f});
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
        }
    }

    if (bad) {
        // a wait ran out; the MMAs may still run: wait (bounded) for their commits before TMEM is freed
        if (tid == 0) atomicCAS(status, 0, WICK_ETIMEOUT);
        if (waited0 < issued0) (void)poll_parity(&mbar[0], waited0 & 1);
        if (waited1 < issued1) (void)poll_parity(&mbar[1], waited1 & 1);
        cp_async_wait_all();
        asm volatile("tcgen05.fence::after_thread_sync;");
        __syncthreads();
        if (warp == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(SH::TMEM_COLS));
        return;
    }
    cp_async_wait_all();

    // combine the five U-slice rows of every output (double-FP32, relative to 2^(E+F)), then FP64
    float2 *comb = reinterpret_cast<float2 *>(smem);   // [kSlices * R][NT], reuses the operand buffers
    if (row_ok)
#pragma unroll
        for (int n = 0; n < SH::CW; ++n) comb[row * NT + cpart * SH::CW + n] = make_float2(acc[n].h, acc[n].l);
    __syncthreads();
    double *part = reinterpret_cast<double *>(partials + ((size_t)rng * n_slices + slice) * plan.n_out);
    for (int e = tid; e < R * NCTA; e += kThr) {
        const int rr = e / NCTA, n = e % NCTA;
        df s = {0.f, 0.f};
#pragma unroll
        for (int i = 0; i < kSlices; ++i) {
            const float2 v = comb[(i * R + rr) * NT + n];
            s = df_add(s, df{v.x, v.y});
        }
        const int pp = rr / (NS * NC), sc1 = rr % (NS * NC);   // part, (s, c1)
        const int s_ = sc1 / NC, c1 = sc1 % NC;
        const double v = ((double)s.h + (double)s.l) * exp2d(sEU[c1] + sF[n]);
        const size_t out = ((size_t)(o * NS + s_) * NC + c1) * SH::NC2 + col0 + n;
        part[2 * out + pp] = v;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(SH::TMEM_COLS));
}

// B = P(c1,c2,c3) - P(c2,c1,c3), summed over the site ranges in a fixed order
__global__ void tc_reduce_kernel(const double2 *__restrict__ partials, int n_splits, int n_slices, int n_out, int nc,
                                 double2 *__restrict__ blocks) {
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

// Which compiled shape a plan takes (0: none, 1: upper, 2: full): weights
// +-2^k, at most 3 colour lists per block type of exactly 4 terms each, the
// same lists for every spin, and at most 12 staged rows per flavour.
int tc_family(const BlockPlan &plan) {
    if (!plan.pow2_w || plan.n_ops < 1 || plan.n_rows[0] + plan.n_rows[1] > kMaxRows) return 0;
    const int ns = plan.n_spin;
    for (int o = 0; o < plan.n_ops; ++o) {
        const int b0 = plan.os_off[o * ns];
        const int n_a = plan.os_off[o * ns + 1] - b0;
        if (n_a < 1 || n_a > kKa) return 0;
        for (int a = 0; a < n_a; ++a) {
            const int l = plan.os_x[b0 + a];
            if (plan.x_off[l + 1] - plan.x_off[l] != kListLen) return 0;
        }
        for (int s = 0; s < ns; ++s) {
            const int t0 = plan.os_off[o * ns + s];
            if (plan.os_off[o * ns + s + 1] - t0 != n_a) return 0;
            for (int a = 0; a < n_a; ++a)
                if (plan.os_x[t0 + a] != plan.os_x[b0 + a]) return 0;
        }
    }
    if (plan.n_chi == UpperShape::NC && ns == UpperShape::NS) return 1;
    if (plan.n_chi == FullShape::NC && ns == FullShape::NS) return 2;
    return 0;
}

template <typename SH, typename ST>
int launch_shape(const BlockPlan &plan, const ST *Su, const ST *Sd, int V, int n_slices, int n_ranges,
                 const int *bounds, const WeightExp &ew, double2 *part, int *status, cudaStream_t stream) {
    auto k = block_tc_kernel<ST, SH>;
    WICK_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SH::SMEM));
    dim3 grid(plan.n_ops * SH::NCT, n_ranges, n_slices);
    k<<<grid, kThr, SH::SMEM, stream>>>(plan, Su, Sd, V, n_slices, n_ranges, bounds, ew, part, status);
    return WICK_OK;
}

}  // namespace

bool tc_applicable(const BlockPlan &plan) { return tc_family(plan) != 0; }

size_t tc_partials_bytes(const BlockPlan &plan, int V, int n_slices, int *n_splits, int *chunk) {
    const int n_ranges = (V + kRangeSites - 1) / kRangeSites;
    *n_splits = n_ranges;
    *chunk = kRangeSites;
    const size_t part = sizeof(double2) * (size_t)n_ranges * n_slices * plan.n_out;
    const size_t bnd = sizeof(int) * (size_t)n_ranges * n_slices * 48;
    return (part + 255) / 256 * 256 + bnd;
}

int launch_block_tc(const BlockPlan &plan, const void *Su, const void *Sd, int dtype, int V, int n_slices,
                    double *partials, int n_splits, double2 *blocks, int *status, cudaStream_t stream) {
    const int fam = tc_family(plan);
    if (!fam || n_splits != (V + kRangeSites - 1) / kRangeSites || n_splits > 65535 || n_slices > 65535)
        return WICK_EINVAL;
    const int n_ranges = n_splits;
    double2 *part = reinterpret_cast<double2 *>(partials);
    const size_t pbytes = (sizeof(double2) * (size_t)n_ranges * n_slices * plan.n_out + 255) / 256 * 256;
    int *bounds = reinterpret_cast<int *>(reinterpret_cast<unsigned char *>(partials) + pbytes);
    WeightExp ew = {};
    for (int o = 0; o < plan.n_ops; ++o) {
        const int b0 = plan.os_off[o * plan.n_spin];
        const int n_a = plan.os_off[o * plan.n_spin + 1] - b0;
        float wmax = 0.f;
        for (int a = 0; a < n_a; ++a) {
            const int l = plan.os_x[b0 + a];
            float w = 0.f;
            for (int qq = plan.x_off[l]; qq < plan.x_off[l + 1]; ++qq) w += fabsf(plan.xt_w[qq]);
            wmax = w > wmax ? w : wmax;
        }
        ew.e[o] = exponent_bound(wmax);
    }
    dim3 gb(n_ranges, n_slices);
    int err;
    if (dtype == WICK_C64) {
        const float2 *u = (const float2 *)Su, *d = (const float2 *)Sd;
        tc_bounds_kernel<float2><<<gb, 256, 0, stream>>>(plan, u, d, V, n_ranges, bounds);
        err = fam == 1 ? launch_shape<UpperShape>(plan, u, d, V, n_slices, n_ranges, bounds, ew, part, status, stream)
                       : launch_shape<FullShape>(plan, u, d, V, n_slices, n_ranges, bounds, ew, part, status, stream);
    } else {
        const double2 *u = (const double2 *)Su, *d = (const double2 *)Sd;
        tc_bounds_kernel<double2><<<gb, 256, 0, stream>>>(plan, u, d, V, n_ranges, bounds);
        err = fam == 1 ? launch_shape<UpperShape>(plan, u, d, V, n_slices, n_ranges, bounds, ew, part, status, stream)
                       : launch_shape<FullShape>(plan, u, d, V, n_slices, n_ranges, bounds, ew, part, status, stream);
    }
    if (err) return err;
    WICK_CUDA_TRY(cudaGetLastError());
    const size_t n = (size_t)n_slices * plan.n_out;
    tc_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(part, n_splits, n_slices, plan.n_out,
                                                                      plan.n_chi, blocks);
    WICK_CUDA_TRY(cudaGetLastError());
    return WICK_OK;
}

}  // namespace wick
