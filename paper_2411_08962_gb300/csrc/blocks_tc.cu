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
// c1 over the CTA's sites), every X value into 6 slices on a grid 2^F of its
// column (2^F >= sum|w| max|u| max|d|):
//     v = 2^(E-7) * sum_i q_i 2^(-8i),   |q_i| <= 128 (U) / 144 (X)   (39 / 47 bits)
// X is formed from the float propagator entries in a fixed-exponent float
// accumulator on the grid 2^(F-22) plus a float sum of the FMA-exact rounding
// remainders (facc below: four operations per product), accurate to about
// 2^-35 of 2^F.  Slice i is stored at its own weight, q_i 2^(-8i): at most 8
// significant bits, exact in bf16.  The products of the pair (i, j) are
// multiples of 2^(-8(i+j)) of magnitude below 2^(15-8(i+j)), and a sum of
// K <= 768 of them (128 sites) stays below 2^(24-8(i+j)), so the FP32
// accumulation in TMEM is exact for a whole round of 128 sites, and every
// accumulator is read with the one factor 2^(E+F-14).  Pairs with i + j <= 5
// are kept.  The grids bound the largest values of a 512-site range, so
// typical X values sit ~6 bits below 2^F; blocks come out ~1e-11 relative
// (the class of the double-FP32 CUDA-core kernel).
// Each round's accumulators are added in double-FP32 relative to 2^(E+F-14);
// the five U-slice rows of an output are combined at the end and converted to
// FP64.
//
// Layout.  The U slices are stacked along M (row i*R + r, R = 2 n_spin n_chi)
// and cut into M tiles of 128 rows; tile t meets only the X slices
// j <= 5 - (first slice in t), one MMA each (6 for the upper-spin tables,
// 6+5+4+2 for the full-spin ones).  A CTA owns (block type, column tile of the
// (c2, c3) columns, range of 512 sites, slice); the first two vary fastest in
// the grid so that the CTAs reading the same rows of S run together.  Per chunk
// of 16 sites (upper tables; 8 for the full-spin ones, for shared memory):
// the CTA builds the U and X slices of chunk c into one of two operand buffers
// from S staged two chunks ahead (two staging buffers, 4-byte cp.async into
// re / im planes with sites innermost), meets at one barrier, and one thread of
// the least-loaded warp issues the chunk's MMAs and commits them to the
// buffer's mbarrier while the others go on to chunk c + 1.  The work of a
// chunk is a list of jobs -- two X values (a site pair) of one column, or two
// U values of one row -- ordered so that every warp does one kind and one
// colour term.  Every wait on an mbarrier is bounded.
//
// One launch covers up to kMaxCfg configurations (grid.z = configuration x
// slice).  A CTA first scans its range of sites for the grid exponents (the
// largest |re|, |im| and |re| + |im| per flavour and source column), builds
// its FP64 partial sums, and arrives on a counter of its (configuration,
// slice, block type); the last CTA to arrive -- no CTA waits for another --
// adds the partials of every range in range order and writes the blocks,
// antisymmetrised in the like-flavour pair, B = P(c1,c2,c3) - P(c2,c1,c3),
// then clears the counter for the next launch.
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
// Level accumulators (full-spin family): the MMA of U slice i (rows i R .. i R + 127 of the stacked
// slices; rows past R are the next slice's, and their TMEM lanes are not read) with X slice j adds into
// an accumulator of its own for each pair of level i + j <= 2 -- (0,0), (0,1), (1,0), (0,2), (1,1),
// (2,0) -> 0..5 -- and into accumulator 3 + i + j for the levels 3, 4, 5.  Products of a level-k pair
// are multiples of 2^(-8k) below 2^(15-8k), so a one-pair accumulator stays exact for K <= 511 (85
// sites; a round is 64 sites); a level-k >= 3 sum of up to five pairs may round at 2^(-8k-6), below
// 2^-40 of a level-0 sum.
constexpr int kLevelAccs = 9;
constexpr int kLevelRoundSites = 64;
__host__ __device__ constexpr int level_acc(int i, int j) {
    return i + j >= 3 ? 3 + i + j : (i + j == 2 ? 3 + i : (i + j == 1 ? 1 + i : 0));
}
__host__ __device__ constexpr bool level_acc_exact(int a) { return a < 6; }
constexpr int kRangeSitesDefault = 512;            // sites per CTA (one grid, one partial) unless tuned
constexpr int kPairRangeSitesDefault = 1024;       // the same for block_pair_kernel and the full-spin shape
constexpr int kMaxCfg = 64;                        // configurations per launch
constexpr int kSpinLimit = 1 << 22;                // mbarrier polls before giving up
// staging buffers: chunk c + 2 is issued after the barrier that ends chunk c's jobs, into chunk c's buffer
constexpr int kStage = 2;
constexpr int kMaxRows = 24;                       // staged S rows (both flavours)
constexpr int kListLen = 4;                        // terms per diquark list the tensor-core path takes (exactly)

// exponent bound of the largest colour-list weight sum, per block type
struct WeightExp {
    int e[kMaxOps];
};

// the propagators of the configurations of one launch, and their sequential propagators (derivative
// blocks: the role passes below)
struct CfgPtrs {
    const void *su[kMaxCfg];
    const void *sd[kMaxCfg];
    const void *sg[kMaxCfg];
};

// Derivative blocks (three-point functions): a block is linear in each of its three propagator roles --
// the U rows (pair flavour f1), the diquark rows of the pair flavour and those of the other flavour -- so
// its derivative in the direction of a sequential propagator Sg of flavour `sub` is the sum over the
// roles of that flavour of the block with that role's rows taken from Sg.  Pass 0 substitutes the U
// rows, pass 1 the pair-flavour diquark rows, pass 2 the other diquark rows; a pass applies to a block
// type when its role has flavour sub.  Without Sg (sub < 0) there is one pass, without substitution.
__host__ __device__ __forceinline__ bool pass_applies(int pass, int sub, int f1) {
    return sub < 0 || (pass == 0 && f1 == sub) || (pass == 1 && f1 == sub) || (pass == 2 && 1 - f1 == sub);
}

// Compile-time shape of a table family: NC colours chi, NS spins, NT columns
// per MMA (multiple of 16), NMT M tiles, NX sites per operand chunk.
// LV_ = 1: one TMEM accumulator per slice level instead of per M tile and X slice (see LEVEL_ACCS).
template <int NC_, int NS_, int NT_, int NMT_, int NX_, int LV_ = 0> struct Shape {
    static constexpr int NC = NC_, NS = NS_, NT = NT_, NMT = NMT_, NX = NX_, LEVELS = LV_;
    static constexpr int KC = NX * kKa * 2;                 // K per chunk
    static constexpr int CHUNKS_PER_ROUND = (LEVELS ? kLevelRoundSites : kRoundSites) / NX;
    static constexpr int NC2 = NC * NC;
    static constexpr int R = 2 * NS * NC;                   // real rows per U slice
    static constexpr int NCTA = NT >= NC2 ? NC2 : NT;       // (c2, c3) columns per CTA
    static constexpr int NCT = (NC2 + NT - 1) / NT;         // column tiles
    static constexpr int PER_TILE = LEVELS ? 4 : 4 / NMT;   // warps of a lane quarter per M tile (LEVELS: one tile)
    static constexpr int CW = LEVELS ? NT / 4 : NT / PER_TILE;   // readout columns per thread
    static constexpr int NSP = NX / 2;                      // site pairs per chunk
    static constexpr int PS = kMaxRows * NC * NX;           // floats per staged plane (re or im)
    static constexpr int STAGERS = kMaxRows * NC * NX / 8;   // staging threads: one (row, colour), 8 sites each
    static constexpr int NXJOB = NCTA * kKa * NSP;          // two X values (a site pair) each
    static constexpr int NUJOB = NS * NC * kKa * NSP;       // two U values (a site pair) each
    // rotation of the thread -> job map in round r: the last round goes to the threads whose earlier
    // jobs were U jobs (the cheaper ones)
    static constexpr int rot(int r) {
        return (r + 1) * kThr < NXJOB + NUJOB ? 0 : NXJOB % kThr;
    }
    static constexpr int jmax(int t) {
        return kSlicesX < kMaxPair + 1 - t * 128 / R ? kSlicesX : kMaxPair + 1 - t * 128 / R;
    }
    static constexpr int toff(int t, int j) {
        int c = 0;
        for (int u = 0; u < t; ++u) c += jmax(u) * NT;
        return c + j * NT;
    }
    static constexpr int TMEM_USED = LEVELS ? kLevelAccs * NT : toff(NMT - 1, 0) + jmax(NMT - 1) * NT;
    static constexpr int TMEM_COLS = TMEM_USED <= 32 ? 32 : TMEM_USED <= 64 ? 64 : TMEM_USED <= 128 ? 128
                                   : TMEM_USED <= 256 ? 256 : 512;
    static constexpr int A_BYTES = NMT * 128 * KC * 2;
    static constexpr int B_BYTES = kSlicesX * NT * KC * 2;
    static constexpr int S_BYTES = 2 * PS * 4;              // two float planes
    static constexpr int SMEM = 2 * (A_BYTES + B_BYTES) + kStage * S_BYTES + 4 * (16 + 256) +
                                (16 + 8) * kKa * kListLen + 4 * 16 + 4 * kMaxRows * 12 + 32;
    static_assert(NMT * 128 >= kSlices * R && (NMT - 1) * 128 < kSlices * R, "M tiles");
    static_assert(!LEVELS || ((kSlices - 1) * R + 128 <= NMT * 128 && R <= 96 && R % 8 == 0), "level tiles");
    static_assert(NC2 <= NT || NC2 % NT == 0, "column tiles");
    static_assert(TMEM_USED <= 512 && CW % 4 == 0 && CW <= 32, "TMEM / readout");
    static_assert(NXJOB % 32 == 0 && NUJOB % 32 == 0, "jobs fill whole warps");
    static_assert(NX % 8 == 0, "site pairs in groups of 4 per warp");
    static_assert(STAGERS <= kThr, "staging threads");
    static_assert(R % 8 == 0, "U slices start on a core-matrix row group");
    static_assert(LEVELS || kSlices * R * NT * 8 <= 2 * (A_BYTES + B_BYTES), "combine buffer");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};
using UpperShape = Shape<6, 2, 48, 1, 16>;   // nucleon upper spin components: 2 x 216 per type
using FullShape = Shape<12, 4, 48, 4, 8, 1>; // all four spins: 4 x 1728 per type, level accumulators

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

// 4-byte copy; src_bytes 0 writes a zero
// L2 eviction policies: the grid-exponent scan marks the rows it reads evict-last, so that they are still
// in L2 when the CTA stages them; the pair kernel's staging (the rows' last reader) marks them evict-first
__device__ __forceinline__ uint64_t l2_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ float4 ldg4_hint(const void *p, uint64_t policy) {
    float4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p), "l"(policy));
    return v;
}
// 4-byte copy with an L2 policy; src_bytes 0 writes a zero
__device__ __forceinline__ void cp_async4_hint(void *dst, const void *src, int src_bytes, uint64_t policy) {
    asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 4, %2, %3;" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(src_bytes), "l"(policy)
                 : "memory");
}

__device__ __forceinline__ void cp_async4(void *dst, const void *src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Poll the mbarrier for `parity` at most `limit` times (this thread only).
__device__ __forceinline__ bool poll_parity(uint64_t *mbar, int parity, int limit = kSpinLimit) {
    uint32_t done = 0;
    for (int it = 0; it < limit && !done; ++it)
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(parity)
            : "memory");
    return done != 0;
}

// Packed slicing: lanes (re, im) of a complex value at once on the f32x2
// instructions.  A slice is kept at its own weight: slice i of r (|r| <= 128)
// is r rounded to the grid 2^(-8i), i.e. q_i 2^(-8i) with an integer
// |q_i| <= 128 -- at most 8 significant bits, exact in bf16, whose bits are
// the upper half of the float's.  Rounding to the grid 2^(-8i) adds and
// subtracts M_i = 1.5 * 2^(23-8i) (exact for |r| < 2^(22-8i)), and r minus
// its rounding is exact, so no rescaling between slices is needed.
__device__ __forceinline__ f2x round_grid(f2x r, int i) {
    const float m = 12582912.f * exp2i(-8 * i);   // 1.5 * 2^(23-8i); i is a compile-time constant
    const f2x M = pk(m, m);
    return sub2(add2(r, M), M);
}

// U: lanes = two sites, v = 2^(E-7) sum_i q_i 2^(-8i) + O(2^(E-40)); one bf16x2 word per slice.
// sc = 2^(7-E), a power of two (clamped to the float range; zero rows stay zero)
__device__ __forceinline__ void slice_u2(f2x v, float sc, uint32_t *w) {
    f2x r = mul2(v, pk(sc, sc));  // exact: power-of-two scale
#pragma unroll
    for (int i = 0; i < kSlices; ++i) {
        const f2x q = round_grid(r, i);
        uint32_t lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "l"(q));
        w[i] = __byte_perm(lo, hi, 0x7632);
        if (i + 1 < kSlices) r = sub2(r, q);
    }
}

// The diquark value X of a site pair is accumulated in units of 2^(F-7) (|X| <= 128 there: 2^F bounds
// sum |w| max|u| max|d| over the range) in a fixed-exponent float a = M + X, M = 384 = 1.5 * 2^8: every
// partial sum stays in [256, 512], so a is on the grid 2^-15 and each step rounds to that grid.  Per
// product A*B (A = w 2^(7-F) u, exact: w = +-2^k; B = d) the step is
//     n = fma(A, B, a),  nz = a - n (exact),  lo += fma(A, B, nz)
// where fma(A, B, nz) = A*B - (n - a), the rounding error of the step, is exact up to one rounding at
// 2^-40 (it is below 2^-16 and A*B has 48 bits above 2^-40 when |A*B| <= 128).  lo (below 2^-12 in
// magnitude: 16 products) is an ordinary float sum; its rounding errors stay below 2^-32 and are
// typically 2^-35.  Four f32x2 operations per product, against ten for a TwoProd-and-TwoSum chain.
constexpr float kFixedM = 384.f;

__device__ __forceinline__ void facc(f2x &a, f2x &lo, f2x A, f2x B) {
    const f2x n = fma2(A, B, a);
    const f2x nz = sub2(a, n);
    lo = add2(lo, fma2(A, B, nz));
    a = n;
}

// Slices of X = hi + lo (units 2^(F-7), lanes = two sites) at their own weight, one bf16x2 word each:
// hi = a - M is on the grid 2^-15 with |hi| <= 128, |lo| <= 2^-12.
//   q0 = hi rounded to an integer, q1 = the rest rounded to 2^-8 (both exact remainders);
//   q2 = the rest of hi (on 2^-15, |.| <= 2^-9) plus lo rounded to 2^-16: |q2| < 2^-8 on the grid 2^-16,
//        8 significant bits (|q2| 2^16 <= 144: products with a U slice stay below 2^15, so a 128-site
//        round of K = 768 products is still an exact float sum);
//   q3, q4, q5 = the rest of lo (|.| <= 2^-17) on the grids 2^-24, 2^-32, 2^-40.
// Representation error <= 2^-41 plus the rounding of lo.
__device__ __forceinline__ void slice_x2(f2x hi, f2x lo, uint32_t *w) {
    auto word = [](f2x q) {
        uint32_t l, h;
        asm("mov.b64 {%0, %1}, %2;" : "=r"(l), "=r"(h) : "l"(q));
        return __byte_perm(l, h, 0x7632);
    };
    f2x q = round_grid(hi, 0);
    w[0] = word(q);
    f2x r = sub2(hi, q);
    q = round_grid(r, 1);
    w[1] = word(q);
    r = sub2(r, q);
    const f2x l2 = round_grid(lo, 2);
    w[2] = word(add2(r, l2));
    r = sub2(lo, l2);
#pragma unroll
    for (int j = 3; j < kSlicesX; ++j) {
        q = round_grid(r, j);
        w[j] = word(q);
        if (j + 1 < kSlicesX) r = sub2(r, q);
    }
}

__device__ __forceinline__ f2x lds2(const float *p) { return *reinterpret_cast<const f2x *>(p); }

// The pair of sites (s, s + 1) of one column of the X_{o,a} list, lanes = sites, in units of 2^(F-7):
// re = sum_t w (ur dr - ui di), im = sum_t w (ur di + ui dr) as (a - M, lo) pairs (see facc).
// term[t] = (float offset of the u row, of the d row, w, w), wn[t] = (-w, -w); sc2 = (2^(7-F), 2^(7-F));
// the re / im planes are PS floats apart.  All loads first.
template <int PS>
__device__ __forceinline__ void x_pair(const int4 *term, const f2x *wn, f2x sc2, const float *bu, const float *bd,
                                       f2x &re_hi, f2x &re_lo, f2x &im_hi, f2x &im_lo) {
    f2x ur[kListLen], ui[kListLen], dr[kListLen], di[kListLen], ww[kListLen], nw[kListLen];
#pragma unroll
    for (int t = 0; t < kListLen; ++t) {
        const int4 tt = term[t];
        ur[t] = lds2(bu + tt.x);
        ui[t] = lds2(bu + tt.x + PS);
        dr[t] = lds2(bd + tt.y);
        di[t] = lds2(bd + tt.y + PS);
        asm("mov.b64 %0, {%1, %2};" : "=l"(ww[t]) : "r"(tt.z), "r"(tt.w));
        nw[t] = wn[t];
    }
    const f2x M = pk(kFixedM, kFixedM);
    f2x ra = M, ia = M, rl = 0ull, il = 0ull;
#pragma unroll
    for (int t = 0; t < kListLen; ++t) {
        const f2x w = mul2(ww[t], sc2), n = mul2(nw[t], sc2);   // +-w 2^(7-F): exact
        const f2x a = mul2(ur[t], w), b = mul2(ui[t], w), nb = mul2(ui[t], n);
        facc(ra, rl, a, dr[t]);
        facc(ra, rl, nb, di[t]);
        facc(ia, il, a, di[t]);
        facc(ia, il, b, dr[t]);
    }
    re_hi = sub2(ra, M);
    im_hi = sub2(ia, M);
    re_lo = rl;
    im_lo = il;
}

// Job jb over (row or column n < NN, colour term a < kKa, site pair sp < NSP) -> (n, a, sp).  A
// warp takes one a and 8 n x 4 site pairs: its 32-bit operand stores then fall on 8 rows x 4 words
// of a core matrix, 32 different banks; a leftover group of 4 n takes 4 n x 8 site pairs.
template <int NN, int NSP> __device__ __forceinline__ void job_map(int jb, int &n, int &a, int &sp) {
    constexpr int NG = NN / 8, FW = NG * (NSP / 4), GA = FW + (NN % 8 ? 1 : 0);
    static_assert(NN % 8 == 0 || (NN % 8 == 4 && NSP == 8), "job map");
    const int w = jb >> 5, lane = jb & 31;
    a = w / GA;
    const int wa = w - a * GA;
    if (wa < FW) {
        n = 8 * (wa % NG) + (lane >> 2);
        sp = 4 * (wa / NG) + (lane & 3);
    } else {
        n = 8 * NG + (lane >> 3);
        sp = lane & 7;
    }
}

// A thread's jobs are the same in every chunk; only the staging and operand buffers change.  Their
// offsets are decoded once: kind 1 = X job (column n, colour term a, sites 2 sp, 2 sp + 1), kind 2 =
// U job (row (s, c1), colour term a, sites 2 sp, 2 sp + 1), 0 = nothing (a colour term beyond the
// operator's, whose K rows stay zero).
struct Job {
    int kind, a;
    int s1, s2;      // X: staged offsets of the u-side and d-side columns; U: the U value, -
    int d1, d2;      // X: B offset of slice 0; U: A offsets of the re and im rows of slice 0
    float sc;        // 2^(7 - grid exponent)
};

template <typename SH>
__device__ __forceinline__ Job make_job(int jb, int col0, int n_a, const int *sF, const int *sR1, const int *sEU) {
    constexpr int NC = SH::NC, NS = SH::NS, NX = SH::NX, KC = SH::KC;
    Job j{0, 0, 0, 0, 0, 0, 0.f};
    if (jb < SH::NXJOB) {
        int n, a, sp;
        job_map<SH::NCTA, SH::NSP>(jb, n, a, sp);
        if (a >= n_a) return j;
        const int c23 = col0 + n;
        j = {1, a, (c23 / NC) * NX + 2 * sp, (c23 % NC) * NX + 2 * sp, tile_off<KC>(n, a * 2 * NX + 2 * sp), 0,
             exp2i(7 - sF[n])};
    } else if (jb < SH::NXJOB + SH::NUJOB) {
        int m, a, sp;
        job_map<NS * NC, SH::NSP>(jb - SH::NXJOB, m, a, sp);
        if (a >= n_a) return j;
        const int s = m / NC, c1 = m % NC;
        j = {2, a, sR1[s * kKa + a] + c1 * NX + 2 * sp, 0, tile_off<KC>(m, a * 2 * NX + 2 * sp),
             tile_off<KC>(NS * NC + m, a * 2 * NX + 2 * sp), exp2i(7 - sEU[c1])};
    }
    return j;
}

// X job: 6 slices of the site pair's re and im parts into B_j[n][k], k = (a, part, site)
template <typename SH>
__device__ __forceinline__ void x_job(const Job &j, const int4 *sTerm, const f2x *sTermN, const float *S,
                                      __nv_bfloat16 *B) {
    constexpr int NT = SH::NT, NX = SH::NX, KC = SH::KC;
    f2x rh, rl, ih, il;
    x_pair<SH::PS>(sTerm + j.a * kListLen, sTermN + j.a * kListLen, pk(j.sc, j.sc), S + j.s1, S + j.s2, rh, rl, ih,
                   il);
    uint32_t wr[kSlicesX], wi[kSlicesX];
    slice_x2(rh, rl, wr);
    slice_x2(ih, il, wi);
    __nv_bfloat16 *dst = B + j.d1;
#pragma unroll
    for (int i = 0; i < kSlicesX; ++i) {
        *reinterpret_cast<uint32_t *>(dst + i * NT * KC) = wr[i];
        *reinterpret_cast<uint32_t *>(dst + i * NT * KC + NX * 8) = wi[i];  // part 1: k + NX
    }
}

// U job: 5 slices into A[(i, part, s, c1)][k]: the re row takes (U_re, -U_im) against (X_re, X_im),
// the im row (U_im, U_re)
template <typename SH>
__device__ __forceinline__ void u_job(const Job &j, const float *S, __nv_bfloat16 *A) {
    constexpr int NX = SH::NX, R = SH::R, KC = SH::KC;
    const float *p = S + j.s1;
    uint32_t qr[kSlices], qi[kSlices];
    slice_u2(lds2(p), j.sc, qr);
    slice_u2(lds2(p + SH::PS), j.sc, qi);
    __nv_bfloat16 *dre = A + j.d1, *dim = A + j.d2;
#pragma unroll
    for (int i = 0; i < kSlices; ++i) {
        const int o = tile_off<KC>(i * R, 0);
        *reinterpret_cast<uint32_t *>(dre + o) = qr[i];
        *reinterpret_cast<uint32_t *>(dre + o + NX * 8) = qi[i] ^ 0x80008000u;
        *reinterpret_cast<uint32_t *>(dim + o) = qi[i];
        *reinterpret_cast<uint32_t *>(dim + o + NX * 8) = qr[i];
    }
}

// The grid exponents of one range of sites (this CTA's): for flavour f and source column ic over the
// rows the tables use, E = bound of max(|re|, |im|) and G = bound of max(|re| + |im|); out[f * 24 +
// kind * 12 + ic].  Every thread of the CTA takes part; ends with the CTA's barrier.
template <typename ST>
__device__ __forceinline__ void range_bounds(const BlockPlan &plan, const ST *su, const ST *sd, const ST *sg, int sub,
                                             int x_begin, int x_end, unsigned *smax, int *out) {
    const int tid = threadIdx.x;
    if (tid < 72) smax[tid] = 0u;
    __syncthreads();
    const int nc = plan.n_chi, nr0 = plan.n_rows[0], nr01 = nr0 + plan.n_rows[1];
    const int nr = nr01 + (sub >= 0 ? plan.n_rows[sub] : 0);   // row group 2: the rows of Sg
    // the kept columns in adjacent pairs (chi, chi + 1), as in the upper- and full-spin layouts: one
    // 16-byte load covers a pair of complex64 values (half the loads in flight per byte)
    bool pairs = sizeof(ST) == 8 && nc % 2 == 0;
    for (int i = 0; pairs && i < nc; i += 2) pairs = plan.chi[i] % 2 == 0 && plan.chi[i + 1] == plan.chi[i] + 1;
    const int per = pairs ? 2 : 1;                 // columns per load
    const int cols = nr * (nc / per);
    const int parts = max(1, (int)blockDim.x / cols);
    if (tid < cols * parts) {
        const int col = tid % cols, part = tid / cols;
        const int rc = col / (nc / per), ic = (col % (nc / per)) * per;
        const int f = rc < nr0 ? 0 : (rc < nr01 ? 1 : 2);
        const int row = f == 0 ? plan.rows[0][rc] : (f == 1 ? plan.rows[1][rc - nr0] : plan.rows[sub][rc - nr01]);
        const ST *src = (f == 0 ? su : (f == 1 ? sd : sg)) + row * 12 + plan.chi[ic];
        float a1 = 0.f, a2 = 0.f, b1 = 0.f, b2 = 0.f;   // columns ic and ic + 1
        if (pairs) {
            const uint64_t keep = l2_evict_last();
#pragma unroll 12
            for (int x = x_begin + part; x < x_end; x += parts) {
                const float4 v = ldg4_hint(src + (size_t)x * 144, keep);
                a1 = fmaxf(a1, fmaxf(fabsf(v.x), fabsf(v.y)));
                a2 = fmaxf(a2, __fadd_ru(fabsf(v.x), fabsf(v.y)));   // rounded up: a bound of |re| + |im|
                b1 = fmaxf(b1, fmaxf(fabsf(v.z), fabsf(v.w)));
                b2 = fmaxf(b2, __fadd_ru(fabsf(v.z), fabsf(v.w)));
            }
        } else {
#pragma unroll 8
            for (int x = x_begin + part; x < x_end; x += parts) {
                const float2 v = to_f2(src[(size_t)x * 144]);
                a1 = fmaxf(a1, fmaxf(fabsf(v.x), fabsf(v.y)));
                a2 = fmaxf(a2, __fadd_ru(fabsf(v.x), fabsf(v.y)));
            }
        }
        atomicMax(&smax[f * 24 + ic], __float_as_uint(a1));
        atomicMax(&smax[f * 24 + 12 + ic], __float_as_uint(a2));
        if (pairs) {
            atomicMax(&smax[f * 24 + ic + 1], __float_as_uint(b1));
            atomicMax(&smax[f * 24 + 12 + ic + 1], __float_as_uint(b2));
        }
    }
    __syncthreads();
    if (tid < 72) {
        const int ic = tid % 12;
        out[tid] = ic < nc ? exponent_bound(__uint_as_float(smax[tid])) : -100;
    }
    __syncthreads();
}

// The CTA's partials of (configuration x slice cs, block type o) are written; count it in.  The last
// of the n_ranges x NCT CTAs of (cs, o) sums the partials of every range in range order and writes
// B = P(c1,c2,c3) - P(c2,c1,c3) for the type's entries, then clears the counter.
template <typename SH>
__device__ __forceinline__ void arrive_and_reduce(const BlockPlan &plan, int cs, int o, int n_ranges, int n_pass,
                                                  int sub, const double2 *partials, int *counters, double2 *blocks,
                                                  int *s_last) {
    constexpr int NC = SH::NC, NS = SH::NS, NC2 = NC * NC, NC3 = NC2 * NC;
    const int tid = threadIdx.x;
    int *cnt = counters + (size_t)cs * plan.n_ops + o;
    __syncthreads();   // every partial of this CTA is written
    if (tid == 0) {
        __threadfence();
        *s_last = atomicAdd(cnt, 1) == n_pass * n_ranges * SH::NCT - 1;
    }
    __syncthreads();
    if (!*s_last) return;
    __threadfence();
    const size_t n_out = (size_t)plan.n_out;
    const double2 *P = partials + (size_t)cs * n_pass * n_ranges * n_out;   // [pass][range][entry]
    const int f1 = plan.f1[o];
    double2 *Bo = blocks + (size_t)cs * n_out;
    for (int e = tid; e < NS * NC3; e += blockDim.x) {
        const int out = o * NS * NC3 + e;
        const int os = out / NC3, i1 = (out / NC2) % NC, i2 = (out / NC) % NC, i3 = out % NC;
        const int sw = os * NC3 + i2 * NC2 + i1 * NC + i3;
        double ax = 0, ay = 0, bx = 0, by = 0;
        for (int p = 0; p < n_pass; ++p) {
            if (!pass_applies(p, sub, f1)) continue;   // its CTAs wrote nothing
            for (int r = 0; r < n_ranges; ++r) {
                const double2 a = __ldcg(P + ((size_t)p * n_ranges + r) * n_out + out);
                const double2 b = __ldcg(P + ((size_t)p * n_ranges + r) * n_out + sw);
                ax += a.x; ay += a.y; bx += b.x; by += b.y;
            }
        }
        Bo[out] = make_double2(ax - bx, ay - by);
    }
    if (tid == 0) *cnt = 0;
}

template <typename ST, typename SH>
__global__ void __launch_bounds__(kThr, 1)
block_tc_kernel(const __grid_constant__ BlockPlan plan, const __grid_constant__ CfgPtrs cfgp, int V, int n_slices,
                int n_ranges, int range_sites, const WeightExp ew, int sub, int n_pass,
                double2 *__restrict__ partials, int *__restrict__ counters, double2 *__restrict__ blocks,
                int *status) {
    constexpr int NC = SH::NC, NS = SH::NS, NT = SH::NT, R = SH::R, NCTA = SH::NCTA;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ unsigned s_max[72];
    __shared__ int s_bnd[72];
    __shared__ int s_last;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // the CTAs of one (slice, range) are adjacent in the grid: they read the same rows of S (L2 reuse)
    const int pass = blockIdx.x / (plan.n_ops * SH::NCT);
    const int ob = blockIdx.x - pass * plan.n_ops * SH::NCT;
    const int o = ob / SH::NCT, ct = ob % SH::NCT;
    const int rng = blockIdx.y, cs = blockIdx.z;             // cs = configuration * n_slices + slice
    const int cfg = cs / n_slices, slice = cs - cfg * n_slices;
    const int f1 = plan.f1[o];
    if (!pass_applies(pass, sub, f1)) {   // a role pass of the other flavour: nothing to add, count it in
        arrive_and_reduce<SH>(plan, cs, o, n_ranges, n_pass, sub, partials, counters, blocks, &s_last);
        return;
    }
    const ST *Su = static_cast<const ST *>(cfgp.su[cfg]);
    const ST *Sd = static_cast<const ST *>(cfgp.sd[cfg]);
    const ST *Sg = sub >= 0 ? static_cast<const ST *>(cfgp.sg[cfg]) : Su;
    // staged row groups: the u rows, the d rows, and (derivative blocks) the rows of Sg
    const int nr0 = plan.n_rows[0], nr01 = nr0 + plan.n_rows[1];
    const int nr = nr01 + (sub >= 0 ? plan.n_rows[sub] : 0);
    const int col0 = ct * NT;
    const int t0 = plan.os_off[o * NS];
    const int n_a = plan.os_off[o * NS + 1] - t0;
    constexpr int NX = SH::NX, KC = SH::KC, PS = SH::PS;
    // the first staged row and the bound group of each role: U rows and pair-flavour diquark rows from
    // flavour f1, the other diquark rows from flavour 1 - f1, or from Sg in the pass that substitutes them
    const bool subU = sub >= 0 && pass == 0, subX2 = sub >= 0 && pass == 1, subX3 = sub >= 0 && pass == 2;
    const int rc1 = f1 == 0 ? 0 : nr0, rc2 = f1 == 0 ? nr0 : 0;
    const int rcU = subU ? nr01 : rc1, rcX2 = subX2 ? nr01 : rc1, rcX3 = subX3 ? nr01 : rc2;
    const int gU = subU ? 2 : f1, gX2 = subX2 ? 2 : f1, gX3 = subX3 ? 2 : 1 - f1;

    __nv_bfloat16 *sA0 = reinterpret_cast<__nv_bfloat16 *>(smem);
    __nv_bfloat16 *sB0 = reinterpret_cast<__nv_bfloat16 *>(smem + 2 * SH::A_BYTES);
    float *sS0 = reinterpret_cast<float *>(smem + 2 * (SH::A_BYTES + SH::B_BYTES));
    int *sEU = reinterpret_cast<int *>(smem + 2 * (SH::A_BYTES + SH::B_BYTES) + kStage * SH::S_BYTES);
    int *sF = sEU + 16;                                       // [256] grid of X per column
    int4 *sTerm = reinterpret_cast<int4 *>(sF + 256);         // [kKa][kListLen] the op's diquark list terms
    f2x *sTermN = reinterpret_cast<f2x *>(sTerm + kKa * kListLen);  // [kKa][kListLen] (-w, -w)
    int *sR1 = reinterpret_cast<int *>(sTermN + kKa * kListLen);    // [NS][kKa] staged offset of U's row
    int *sSrc = sR1 + 16;                                     // [kMaxRows * NC] flavour << 16 | row * 12 + chi
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sSrc + kMaxRows * 12);   // [2]
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 2);

    // zero both operand buffers once: padding rows and unused colour terms stay zero
    {
        uint4 *z = reinterpret_cast<uint4 *>(smem);
        for (int e = tid; e < 2 * (SH::A_BYTES + SH::B_BYTES) / 16; e += kThr) z[e] = make_uint4(0u, 0u, 0u, 0u);
    }
    const int x_begin = rng * range_sites, x_end = min(V, x_begin + range_sites);
    const int n_chunks = (x_end - x_begin + NX - 1) / NX;
    const ST *su = Su + (size_t)slice * V * 144;
    const ST *sd = Sd + (size_t)slice * V * 144;
    const ST *sg = Sg + (size_t)slice * V * 144;
    range_bounds<ST>(plan, su, sd, sg, sub, x_begin, x_end, s_max, s_bnd);
    const int *bnd = s_bnd;
    if (tid < NC) sEU[tid] = bnd[gU * 24 + tid];
    if (tid < NT) {
        const int c23 = col0 + tid;
        sF[tid] = tid < NCTA ? bnd[gX2 * 24 + 12 + c23 / NC] + bnd[gX3 * 24 + 12 + c23 % NC] + ew.e[o] : 0;
    }
    if (tid < kKa * kListLen) {
        const int a = tid / kListLen, t = tid % kListLen;
        int4 v = make_int4(0, 0, 0, 0);
        float w = 0.f;
        if (a < n_a) {
            const int q = plan.x_off[plan.os_x[t0 + a]] + t;
            w = plan.xt_w[q];
            v = make_int4((rcX2 + plan.xt_r2[q]) * NC * NX, (rcX3 + plan.xt_r3[q]) * NC * NX, __float_as_int(w),
                          __float_as_int(w));
        }
        sTerm[tid] = v;
        sTermN[tid] = pk(-w, -w);
    }
    if (tid >= 32 && tid < 32 + NS * kKa) {
        const int s = (tid - 32) / kKa, a = (tid - 32) % kKa;
        sR1[s * kKa + a] = a < n_a ? (rcU + plan.os_r1[plan.os_off[o * NS + s] + a]) * NC * NX : 0;
    }
    for (int e = tid; e < nr * NC; e += kThr) {
        const int rc = e / NC, ic = e - rc * NC;
        const int f = rc < nr0 ? 0 : (rc < nr01 ? 1 : 2);
        const int row = f == 0 ? plan.rows[0][rc] : (f == 1 ? plan.rows[1][rc - nr0] : plan.rows[sub][rc - nr01]);
        sSrc[e] = f << 16 | (row * 12 + plan.chi[ic]);
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

    __syncthreads();   // sSrc
    // stage the rows of chunk c as two planes (re, im) of [row][ic][site], flavour-0 rows first, sites
    // innermost (zeros past the range).  The last STAGERS threads (the warps with the lightest jobs)
    // each copy one (row, colour) for 8 consecutive sites, from offsets computed once.
    const int st_t = tid - (kThr - SH::STAGERS);
    const int st_rcc = st_t >= 0 ? st_t / (NX / 8) : 0, st_part = st_t >= 0 ? st_t % (NX / 8) : 0;
    const bool stager = st_t >= 0 && st_rcc < nr * NC;
    const ST *st_src = su;
    if (stager) {
        const int src_off = sSrc[st_rcc];
        const int grp = src_off >> 16;
        st_src = (grp == 0 ? su : (grp == 1 ? sd : sg)) + (src_off & 0xFFFF);
    }
    auto stage = [&](int c) {
        if (stager) {
            float *dst = sS0 + (c % kStage) * (2 * PS) + st_rcc * NX + st_part * 8;
            const int xb = x_begin + c * NX + st_part * 8;
#pragma unroll
            for (int s8 = 0; s8 < 8; ++s8) {
                const bool in = xb + s8 < x_end;
                const ST *src = st_src + (size_t)(in ? xb + s8 : x_begin) * 144;
                if constexpr (sizeof(ST) == 8) {
                    cp_async4(dst + s8, reinterpret_cast<const float *>(src), in ? 4 : 0);
                    cp_async4(dst + s8 + PS, reinterpret_cast<const float *>(src) + 1, in ? 4 : 0);
                } else {
                    const float2 v = in ? to_f2(*src) : make_float2(0.f, 0.f);
                    dst[s8] = v.x;
                    dst[s8 + PS] = v.y;
                }
            }
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
    // (level accumulators: every warp of a lane quarter reads its own quarter of the NT columns)
    const int t_own = SH::LEVELS ? 0 : g / SH::PER_TILE, cpart = SH::LEVELS ? g : g % SH::PER_TILE;
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

    // one job per thread and round: X jobs first, then U jobs; both fill whole warps, so every branch
    // is warp-uniform.  The last round goes to the threads that took U jobs before.
    constexpr int NR = (SH::NXJOB + SH::NUJOB + kThr - 1) / kThr;
    Job job[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r)
        job[r] = make_job<SH>(r * kThr + (tid + kThr - SH::rot(r)) % kThr, col0, n_a, sF, sR1, sEU);

    constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);
    int issued0 = 0, issued1 = 0, waited0 = 0, waited1 = 0, bad = 0;

    for (int c = 0; c < n_chunks; ++c) {
        const int buf = c & 1;
        __nv_bfloat16 *A = sA0 + buf * (SH::A_BYTES / 2);
        __nv_bfloat16 *B = sB0 + buf * (SH::B_BYTES / 2);
        const float *S = sS0 + (c % kStage) * (2 * PS);
        // the MMAs of chunk c - 2 read this operand buffer
        if (buf == 0 && waited0 < issued0) {
            if (poll_parity(&mbar[0], waited0 & 1)) ++waited0;
            else bad = 1;
        } else if (buf == 1 && waited1 < issued1) {
            if (poll_parity(&mbar[1], waited1 & 1)) ++waited1;
            else bad = 1;
        }
        if (!bad) {
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                if (job[r].kind == 1) x_job<SH>(job[r], sTerm, sTermN, S, B);
                else if (job[r].kind == 2) u_job<SH>(job[r], S, A);
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
        if (SH::LEVELS && tid == kThr - 1) {
            const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
#pragma unroll
            for (int ks = 0; ks < KC / 16; ++ks)
#pragma unroll
                for (int i = 0; i < kSlices; ++i) {
                    const uint64_t da = smem_desc<KC>(a0 + (uint32_t)(i * R * KC * 2 + ks * 256));
#pragma unroll
                    for (int j = 0; j < kSlicesX && i + j <= kMaxPair; ++j) {
                        const uint64_t db = smem_desc<KC>(b0 + (uint32_t)(j * NT * KC * 2 + ks * 256));
                        const int ac = level_acc(i, j);
                        // the first MMA into an accumulator in a round starts it (merged levels: i = 0 comes first)
                        const uint32_t acc_in = (fresh && ks == 0 && (level_acc_exact(ac) || i == 0)) ? 0u : 1u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
                                tbase + (uint32_t)(ac * NT)),
                            "l"(da), "l"(db), "r"(idesc), "r"(acc_in));
                    }
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar[buf])));
        }
        if (!SH::LEVELS && tid == kThr - 1) {  // the last warp has the fewest jobs
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
        // stage chunk c + 2 into the buffer chunk c was built from (its jobs are done)
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
            if constexpr (SH::LEVELS) {
                if (q < 3) {   // lanes 96..127 hold rows of the next slice: not read
#pragma unroll
                    for (int ac = 0; ac < kLevelAccs; ++ac) {
                        uint32_t r[SH::CW];
                        const uint32_t taddr = tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(ac * NT + cpart * SH::CW);
#pragma unroll
                        for (int c4 = 0; c4 < SH::CW; c4 += 4)
                            asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                                         : "=r"(r[c4]), "=r"(r[c4 + 1]), "=r"(r[c4 + 2]), "=r"(r[c4 + 3])
                                         : "r"(taddr + (uint32_t)c4));
                        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                        for (int n = 0; n < SH::CW; ++n) {
                            // the one-pair accumulators join by TwoSum; the levels >= 3 join the low part
                            if (level_acc_exact(ac)) acc_add(acc[n], df{__uint_as_float(r[n]), 0.f});
                            else acc[n].l = __fadd_rn(acc[n].l, __uint_as_float(r[n]));
                        }
                    }
                }
            }
            for (int j = 0; !SH::LEVELS && j <= j_warp; ++j) {
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
#pragma unroll
                    for (int n = 0; n < SH::CW; ++n) acc_add(acc[n], df{__uint_as_float(r[n]), 0.f});
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
        }
    }

    if (bad) {
        // a wait ran out; the MMAs may still run: wait (bounded) for their commits before TMEM is freed.
        // The CTA still arrives below, so that the counts stay whole; the status word reports the error.
        if (tid == 0) atomicCAS(status, 0, WICK_ETIMEOUT);
        if (waited0 < issued0) (void)poll_parity(&mbar[0], waited0 & 1);
        if (waited1 < issued1) (void)poll_parity(&mbar[1], waited1 & 1);
        cp_async_wait_all();
        asm volatile("tcgen05.fence::after_thread_sync;");
        __syncthreads();
        if (warp == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(SH::TMEM_COLS));
        arrive_and_reduce<SH>(plan, cs, o, n_ranges, n_pass, sub, partials, counters, blocks, &s_last);
        return;
    }
    cp_async_wait_all();

    if constexpr (SH::LEVELS) {
        // every slice level is in this thread's accumulators: scale and write its row's partials
        if (q < 3) {
            double *part = reinterpret_cast<double *>(partials + (((size_t)cs * n_pass + pass) * n_ranges + rng) * plan.n_out);
            const int rr = q * 32 + lane;                          // < R
            const int pp = rr / (NS * NC), sc1 = rr % (NS * NC);   // part, (s, c1)
            const int s_ = sc1 / NC, c1 = sc1 % NC;
#pragma unroll
            for (int n0 = 0; n0 < SH::CW; ++n0) {
                const int n = cpart * SH::CW + n0;
                const double v = ((double)acc[n0].h + (double)acc[n0].l) * exp2d(sEU[c1] + sF[n] - 14);
                const size_t out = ((size_t)(o * NS + s_) * NC + c1) * SH::NC2 + col0 + n;
                part[2 * out + pp] = v;
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (warp == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(SH::TMEM_COLS));
        arrive_and_reduce<SH>(plan, cs, o, n_ranges, n_pass, sub, partials, counters, blocks, &s_last);
        return;
    }
    // combine the five U-slice rows of every output (double-FP32, relative to 2^(E+F)), then FP64
    float2 *comb = reinterpret_cast<float2 *>(smem);   // [kSlices * R][NT], reuses the operand buffers
    if (row_ok)
#pragma unroll
        for (int n = 0; n < SH::CW; ++n) comb[row * NT + cpart * SH::CW + n] = make_float2(acc[n].h, acc[n].l);
    __syncthreads();
    double *part = reinterpret_cast<double *>(partials + (((size_t)cs * n_pass + pass) * n_ranges + rng) * plan.n_out);
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
        const double v = ((double)s.h + (double)s.l) * exp2d(sEU[c1] + sF[n] - 14);
        const size_t out = ((size_t)(o * NS + s_) * NC + c1) * SH::NC2 + col0 + n;
        part[2 * out + pp] = v;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(SH::TMEM_COLS));
    arrive_and_reduce<SH>(plan, cs, o, n_ranges, n_pass, sub, partials, counters, blocks, &s_last);
}

// The wait for an MMA commit on an mbarrier that nothing arrives on: the poll gives up after `limit`
// tries and the status word gets WICK_ETIMEOUT, as in block_tc_kernel.
__global__ void mbar_wait_selftest_kernel(int limit, int *status) {
    __shared__ uint64_t mbar;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    if (!poll_parity(&mbar, 0, limit)) atomicCAS(status, 0, WICK_ETIMEOUT);
}

// ---------------------------------------------------------------------------
// Both block types of a proton/neutron pair in one CTA (upper-spin tables).
//
// Exchanging the two diquark rows of a list term flips the sign of the colour
// epsilon and of the antisymmetric spin matrix, so when the neutron's lists are
// the proton's with the two rows exchanged (checked on the host, pair_plan), the
// neutron's diquark values are the proton's with the columns transposed:
// X_n(c2, c3) = X_p(c3, c2).  The CTA computes X_p once for both types.
//
// The update runs with the roles of the operands turned around: A = the six X
// slices of the 36 (c2, c3) columns (row 40 j + n of two 128-row tiles; rows
// 36..39 of each slice are padding, so a slice's rows are 40 apart and its
// stores a constant stride apart), B = the five U slices of one type (row
// 24 i + 12 part + (s, c1), N = 128).  Every TMEM element then holds one slice
// pair (i, j): accumulator (type, tile) in 128 columns, four of them.  The neutron
// accumulators see A's columns transposed: lane (j, n) contributes to the neutron
// column n^T = (n mod 6) 6 + n / 6, whose grid is the proton column n's.
// Readout per 128-site round: each thread reads its lane's 120 columns, adds the
// five U slices with i + j <= 5 in double-FP32, and the six X slices of an output
// (six lanes, in different warps) are added into double-FP32 accumulators in
// shared memory, one slice j at a time.  Grids, slicing, exact rounds, staging,
// bounded waits and the range reduction are those of block_tc_kernel.
// ---------------------------------------------------------------------------
struct PairShape {
    static constexpr int NC = 6, NS = 2, NX = 8, NSP = NX / 2;
    static constexpr int KC = NX * kKa * 2;                  // K per chunk: 48
    static constexpr int NC2 = NC * NC;                      // 36 columns
    static constexpr int XSTRIDE = 40;                       // A rows per X slice
    static constexpr int R = 2 * NS * NC;                    // 24 U rows per slice
    static constexpr int CHUNKS_PER_ROUND = kRoundSites / NX;
    static constexpr int PS = kMaxRows * NC * NX;            // floats per staged plane
    static constexpr int STAGERS = kMaxRows * NC * NX / 8;   // one (row, colour), 8 sites each
    static constexpr int NXJOB = NC2 * kKa * NSP;            // 432: column, colour term, site pair
    static constexpr int NUJOB = 2 * NS * NC * kKa * NSP;    // 288: type, (s, c1), colour term, site pair
    static constexpr int A_BYTES = 256 * KC * 2;             // two M tiles of X slices
    static constexpr int B_BYTES = 2 * 128 * KC * 2;         // the U slices of both types
    static constexpr int S_BYTES = 2 * PS * 4;
    static constexpr int ACC_BYTES = 2 * 2 * NS * NC * NC2 * 8;   // [type][part][(s, c1)][column] df
    static constexpr int SMEM = 2 * (A_BYTES + B_BYTES) + kStage * S_BYTES + ACC_BYTES + 4 * (32 + 64) +
                                (16 + 8) * kKa * kListLen + 4 * 16 + 4 * kMaxRows * 12 + 64;
    static_assert(kSlicesX * XSTRIDE <= 256 && XSTRIDE % 8 == 0 && XSTRIDE >= NC2, "X rows");
    static_assert(kSlices * R <= 128 && R % 8 == 0, "U rows");
    static_assert(NXJOB + NUJOB <= 2 * kThr && STAGERS <= kThr, "jobs");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

template <typename ST>
__global__ void __launch_bounds__(kThr, 1)
block_pair_kernel(const __grid_constant__ BlockPlan plan, const __grid_constant__ CfgPtrs cfgp, int V, int n_slices,
                  int n_ranges, int range_sites, const WeightExp ew, int oP, int oN, double2 *__restrict__ partials,
                  int *__restrict__ counters, double2 *__restrict__ blocks, int *status) {
    using SH = PairShape;
    constexpr int NC = SH::NC, NS = SH::NS, NX = SH::NX, KC = SH::KC, PS = SH::PS, NC2 = SH::NC2, R = SH::R;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ unsigned s_max[72];
    __shared__ int s_bnd[72];
    __shared__ int s_last;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rng = blockIdx.y, cs = blockIdx.z;
    const int cfg = cs / n_slices, slice = cs - cfg * n_slices;
    const ST *Su = static_cast<const ST *>(cfgp.su[cfg]);
    const ST *Sd = static_cast<const ST *>(cfgp.sd[cfg]);
    const int nr0 = plan.n_rows[0], nr = nr0 + plan.n_rows[1];
    const int tP = plan.os_off[oP * NS];
    const int n_a = plan.os_off[oP * NS + 1] - tP;

    __nv_bfloat16 *sA0 = reinterpret_cast<__nv_bfloat16 *>(smem);
    __nv_bfloat16 *sB0 = reinterpret_cast<__nv_bfloat16 *>(smem + 2 * SH::A_BYTES);
    float *sS0 = reinterpret_cast<float *>(smem + 2 * (SH::A_BYTES + SH::B_BYTES));
    float2 *sAcc = reinterpret_cast<float2 *>(smem + 2 * (SH::A_BYTES + SH::B_BYTES) + kStage * SH::S_BYTES);
    int *sEU = reinterpret_cast<int *>(sAcc + 2 * 2 * NS * NC * NC2);   // [type][16] grid of U per colour
    int *sF = sEU + 32;                                       // [64] grid of X per proton column
    int4 *sTerm = reinterpret_cast<int4 *>(sF + 64);          // [kKa][kListLen] the proton's list terms
    f2x *sTermN = reinterpret_cast<f2x *>(sTerm + kKa * kListLen);
    int *sR1 = reinterpret_cast<int *>(sTermN + kKa * kListLen);    // [type][NS][kKa] staged offset of U's row
    int *sSrc = sR1 + 16;                                     // [kMaxRows * NC]
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sSrc + kMaxRows * 12);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 2);

    {   // zero the operand buffers (padding rows, unused colour terms) and the accumulators
        uint4 *z = reinterpret_cast<uint4 *>(smem);
        for (int e = tid; e < 2 * (SH::A_BYTES + SH::B_BYTES) / 16; e += kThr) z[e] = make_uint4(0u, 0u, 0u, 0u);
        for (int e = tid; e < 2 * 2 * NS * NC * NC2; e += kThr) sAcc[e] = make_float2(0.f, 0.f);
    }
    const int x_begin = rng * range_sites, x_end = min(V, x_begin + range_sites);
    const int n_chunks = (x_end - x_begin + NX - 1) / NX;
    const ST *su = Su + (size_t)slice * V * 144;
    const ST *sd = Sd + (size_t)slice * V * 144;
    range_bounds<ST>(plan, su, sd, su, -1, x_begin, x_end, s_max, s_bnd);
    const int *bnd = s_bnd;
    if (tid < 2 * NC) {   // type 0 = the proton (U rows from u), type 1 = the neutron (from d)
        const int ty = tid / NC, c1 = tid % NC;
        sEU[ty * 16 + c1] = bnd[ty * 24 + c1];
    }
    if (tid < NC2) sF[tid] = bnd[12 + tid / NC] + bnd[24 + 12 + tid % NC] + ew.e[oP];
    if (tid < kKa * kListLen) {
        const int a = tid / kListLen, t = tid % kListLen;
        int4 v = make_int4(0, 0, 0, 0);
        float w = 0.f;
        if (a < n_a) {
            const int q = plan.x_off[plan.os_x[tP + a]] + t;
            w = plan.xt_w[q];
            v = make_int4(plan.xt_r2[q] * NC * NX, (nr0 + plan.xt_r3[q]) * NC * NX, __float_as_int(w),
                          __float_as_int(w));
        }
        sTerm[tid] = v;
        sTermN[tid] = pk(-w, -w);
    }
    if (tid >= 32 && tid < 32 + 2 * NS * kKa) {
        const int e = tid - 32, ty = e / (NS * kKa), s = (e / kKa) % NS, a = e % kKa;
        const int o = ty ? oN : oP, rc = ty ? nr0 : 0;
        sR1[e] = a < n_a ? (rc + plan.os_r1[plan.os_off[o * NS + s] + a]) * NC * NX : 0;
    }
    for (int e = tid; e < nr * NC; e += kThr) {
        const int rc = e / NC, ic = e - rc * NC;
        const int f = rc < nr0 ? 0 : 1;
        const int row = f == 0 ? plan.rows[0][rc] : plan.rows[1][rc - nr0];
        sSrc[e] = f << 16 | (row * 12 + plan.chi[ic]);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();

    // staging: the last STAGERS threads, one (row, colour) for all 8 sites of a chunk
    const int st_t = tid - (kThr - SH::STAGERS);
    const int st_rcc = st_t >= 0 ? st_t : 0;
    const bool stager = st_t >= 0 && st_rcc < nr * NC;
    const ST *st_src = su;
    if (stager) {
        const int src_off = sSrc[st_rcc];
        st_src = ((src_off >> 16) ? sd : su) + (src_off & 0xFFFF);
    }
    const uint64_t drop = l2_evict_first();
    auto stage = [&](int c) {
        if (stager) {
            float *dst = sS0 + (c % kStage) * (2 * PS) + st_rcc * NX;
            const int xb = x_begin + c * NX;
#pragma unroll
            for (int s8 = 0; s8 < 8; ++s8) {
                const bool in = xb + s8 < x_end;
                const ST *src = st_src + (size_t)(in ? xb + s8 : x_begin) * 144;
                if constexpr (sizeof(ST) == 8) {
                    cp_async4_hint(dst + s8, reinterpret_cast<const float *>(src), in ? 4 : 0, drop);
                    cp_async4_hint(dst + s8 + PS, reinterpret_cast<const float *>(src) + 1, in ? 4 : 0, drop);
                } else {
                    const float2 v = in ? to_f2(*src) : make_float2(0.f, 0.f);
                    dst[s8] = v.x;
                    dst[s8 + PS] = v.y;
                }
            }
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

    // the thread's jobs.  Warps 0..13 take the X jobs (32 each, warp 13 half), the nine warp-loads of U
    // jobs go to warps 14, 15 and, as a second job, to warps 0, 1, 2, 3, 6, 7, 10, so that each of the
    // four warp schedulers (warp % 4) gets about the same work: 4, 4, 3 and 3 X warps, 1, 1, 4 and 3 U.
    int xk = -1, xs1 = 0, xs2 = 0, xd = 0;   // X job: colour term, u / d staged offsets, A offset of slice 0
    float xsc = 0.f;
    int uk[2] = {-1, -1}, us[2] = {0, 0}, ud1[2] = {0, 0}, ud2[2] = {0, 0};   // U jobs
    float usc[2] = {0.f, 0.f};
    {
        const int xw = warp < 14 ? warp : -1;
        int uw[2] = {warp >= 14 ? warp - 14 : -1, -1};
        switch (warp) {
            case 0: uw[1] = 2; break;
            case 1: uw[1] = 3; break;
            case 2: uw[1] = 4; break;
            case 3: uw[1] = 5; break;
            case 6: uw[1] = 6; break;
            case 7: uw[1] = 7; break;
            case 10: uw[1] = 8; break;
            default: break;
        }
        const int jb = xw * 32 + lane;
        if (xw >= 0 && jb < SH::NXJOB) {   // (a, column n, site pair): lanes take 8 columns x 4 site pairs
            const int a = jb / (NC2 * SH::NSP), rem = jb % (NC2 * SH::NSP), n = rem / SH::NSP, sp = rem % SH::NSP;
            if (a < n_a) {
                xk = a;
                xs1 = (n / NC) * NX + 2 * sp;
                xs2 = (n % NC) * NX + 2 * sp;
                xd = tile_off<KC>(n, a * 2 * NX + 2 * sp);
                xsc = exp2i(7 - sF[n]);
            }
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int u = uw[r] * 32 + lane;
            if (uw[r] < 0 || u >= SH::NUJOB) continue;
            // (type, a, (s, c1), site pair)
            const int ty = u / (kKa * NS * NC * SH::NSP), rem = u % (kKa * NS * NC * SH::NSP);
            const int a = rem / (NS * NC * SH::NSP), m = (rem / SH::NSP) % (NS * NC), sp = rem % SH::NSP;
            if (a < n_a) {
                const int s = m / NC, c1 = m % NC;
                uk[r] = ty;
                us[r] = sR1[(ty * NS + s) * kKa + a] + c1 * NX + 2 * sp;
                ud1[r] = ty * 128 * KC + tile_off<KC>(m, a * 2 * NX + 2 * sp);
                ud2[r] = ty * 128 * KC + tile_off<KC>(NS * NC + m, a * 2 * NX + 2 * sp);
                usc[r] = exp2i(7 - sEU[ty * 16 + c1]);
            }
        }
    }

    // readout ownership: accumulator (type, tile) = warp / 4, lane quarter = warp % 4
    const int q = warp & 3, g = warp >> 2, ty_own = g >> 1, tile_own = g & 1;
    const int xrow = tile_own * 128 + q * 32 + lane;            // A row of this thread's TMEM lane
    const int j_own = xrow / SH::XSTRIDE, n_own = xrow % SH::XSTRIDE;
    const bool row_ok = j_own < kSlicesX && n_own < NC2;
    const int n_out = ty_own ? (n_own % NC) * NC + n_own / NC : n_own;   // output column of this lane

    constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(128 >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);
    int issued0 = 0, issued1 = 0, waited0 = 0, waited1 = 0, bad = 0;
    for (int c = 0; c < n_chunks; ++c) {
        const int buf = c & 1;
        __nv_bfloat16 *A = sA0 + buf * (SH::A_BYTES / 2);
        __nv_bfloat16 *B = sB0 + buf * (SH::B_BYTES / 2);
        const float *S = sS0 + (c % kStage) * (2 * PS);
        if (buf == 0 && waited0 < issued0) {
            if (poll_parity(&mbar[0], waited0 & 1)) ++waited0;
            else bad = 1;
        } else if (buf == 1 && waited1 < issued1) {
            if (poll_parity(&mbar[1], waited1 & 1)) ++waited1;
            else bad = 1;
        }
        if (!bad) {
            if (xk >= 0) {   // X job: 6 slices of re and im into rows 40 j + n
                f2x rh, rl, ih, il;
                x_pair<PS>(sTerm + xk * kListLen, sTermN + xk * kListLen, pk(xsc, xsc), S + xs1, S + xs2, rh, rl, ih,
                           il);
                uint32_t wr[kSlicesX], wi[kSlicesX];
                slice_x2(rh, rl, wr);
                slice_x2(ih, il, wi);
                __nv_bfloat16 *dst = A + xd;
#pragma unroll
                for (int j = 0; j < kSlicesX; ++j) {
                    // row 40 j + n: 5 j row groups of 8 further on
                    *reinterpret_cast<uint32_t *>(dst + j * (SH::XSTRIDE / 8) * (KC / 8) * 64) = wr[j];
                    *reinterpret_cast<uint32_t *>(dst + j * (SH::XSTRIDE / 8) * (KC / 8) * 64 + NX * 8) = wi[j];
                }
            }
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                if (uk[r] < 0) continue;
                const float *p = S + us[r];
                uint32_t qr[kSlices], qi[kSlices];
                slice_u2(lds2(p), usc[r], qr);
                slice_u2(lds2(p + PS), usc[r], qi);
                __nv_bfloat16 *dre = B + ud1[r], *dim = B + ud2[r];
#pragma unroll
                for (int i = 0; i < kSlices; ++i) {
                    const int o = tile_off<KC>(i * R, 0);
                    *reinterpret_cast<uint32_t *>(dre + o) = qr[i];
                    *reinterpret_cast<uint32_t *>(dre + o + NX * 8) = qi[i] ^ 0x80008000u;
                    *reinterpret_cast<uint32_t *>(dim + o) = qi[i];
                    *reinterpret_cast<uint32_t *>(dim + o + NX * 8) = qr[i];
                }
            }
        }
        cp_async_wait_all();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        if (__syncthreads_or(bad)) {
            bad = 1;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const bool fresh = c % SH::CHUNKS_PER_ROUND == 0;
        if (tid == kThr - 1) {   // a thread of the last warp (one U job)
            const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
#pragma unroll
            for (int ks = 0; ks < KC / 16; ++ks)
#pragma unroll
                for (int ty = 0; ty < 2; ++ty)
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        const uint64_t da = smem_desc<KC>(a0 + (uint32_t)(t * 128 * KC * 2 + ks * 256));
                        const uint64_t db = smem_desc<KC>(b0 + (uint32_t)(ty * 128 * KC * 2 + ks * 256));
                        const uint32_t acc_in = (fresh && ks == 0) ? 0u : 1u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
                                tbase + (uint32_t)((ty * 2 + t) * 128)),
                            "l"(da), "l"(db), "r"(idesc), "r"(acc_in));
                    }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar[buf])));
        }
        if (buf) ++issued1;
        else ++issued0;
        if (c + 2 < n_chunks) stage(c + 2);

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
            // this lane's slice pairs: the five U slices with i + j <= 5, per (part, s, c1)
            df part[R];
#pragma unroll
            for (int e = 0; e < R; ++e) part[e] = {0.f, 0.f};
            const uint32_t taddr = tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)((ty_own * 2 + tile_own) * 128);
#pragma unroll
            for (int i = 0; i < kSlices; ++i) {
                uint32_t v[R];
#pragma unroll
                for (int c8 = 0; c8 < R; c8 += 8)
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                 : "=r"(v[c8]), "=r"(v[c8 + 1]), "=r"(v[c8 + 2]), "=r"(v[c8 + 3]), "=r"(v[c8 + 4]),
                                   "=r"(v[c8 + 5]), "=r"(v[c8 + 6]), "=r"(v[c8 + 7])
                                 : "r"(taddr + (uint32_t)(i * R + c8)));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                if (row_ok && i + j_own <= kMaxPair) {
#pragma unroll
                    for (int e = 0; e < R; ++e) acc_add(part[e], df{__uint_as_float(v[e]), 0.f});
                }
            }
            // the six X slices of an output column live in six lanes: add them one slice at a time
            for (int jj = 0; jj < kSlicesX; ++jj) {
                if (row_ok && j_own == jj) {
#pragma unroll
                    for (int e = 0; e < R; ++e) {   // e = part * 12 + (s, c1)
                        float2 *p = sAcc + ((ty_own * 2 + e / (NS * NC)) * (NS * NC) + e % (NS * NC)) * NC2 + n_out;
                        const df sum = df_add(df{p->x, p->y}, part[e]);
                        *p = make_float2(sum.h, sum.l);
                    }
                }
                __syncthreads();
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
        }
    }

    if (bad) {
        if (tid == 0) atomicCAS(status, 0, WICK_ETIMEOUT);
        if (waited0 < issued0) (void)poll_parity(&mbar[0], waited0 & 1);
        if (waited1 < issued1) (void)poll_parity(&mbar[1], waited1 & 1);
        cp_async_wait_all();
        asm volatile("tcgen05.fence::after_thread_sync;");
        __syncthreads();
        if (warp == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512));
        arrive_and_reduce<UpperShape>(plan, cs, oP, n_ranges, 1, -1, partials, counters, blocks, &s_last);
        arrive_and_reduce<UpperShape>(plan, cs, oN, n_ranges, 1, -1, partials, counters, blocks, &s_last);
        return;
    }
    cp_async_wait_all();
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512));
    // scale and write the partials of both types: output (type, s, c1, column) with the grids of its U colour
    // and of the X column it came from (the proton column, transposed for the neutron)
    double *part = reinterpret_cast<double *>(partials + ((size_t)cs * n_ranges + rng) * plan.n_out);
    for (int e = tid; e < 2 * 2 * NS * NC * NC2; e += kThr) {
        const int col = e % NC2, m = (e / NC2) % (NS * NC), pp = (e / (NC2 * NS * NC)) % 2, ty = e / (NC2 * NS * NC * 2);
        const int s_ = m / NC, c1 = m % NC;
        const int xcol = ty ? (col % NC) * NC + col / NC : col;
        const float2 v = sAcc[e];
        const double val = ((double)v.x + (double)v.y) * exp2d(sEU[ty * 16 + c1] + sF[xcol] - 14);
        const int o = ty ? oN : oP;
        const size_t out = ((size_t)(o * NS + s_) * NC + c1) * NC2 + col;
        part[2 * out + pp] = val;
    }
    arrive_and_reduce<UpperShape>(plan, cs, oP, n_ranges, 1, -1, partials, counters, blocks, &s_last);
    arrive_and_reduce<UpperShape>(plan, cs, oN, n_ranges, 1, -1, partials, counters, blocks, &s_last);
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
int launch_shape(const BlockPlan &plan, const CfgPtrs &cp, int n_cfg, int V, int n_slices, int n_ranges,
                 int range_sites, const WeightExp &ew, int sub, int n_pass, double2 *part, int *counters,
                 double2 *blocks, int *status, cudaStream_t stream) {
    auto k = block_tc_kernel<ST, SH>;
    WICK_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SH::SMEM));
    dim3 grid(n_pass * plan.n_ops * SH::NCT, n_ranges, n_cfg * n_slices);
    k<<<grid, kThr, SH::SMEM, stream>>>(plan, cp, V, n_slices, n_ranges, range_sites, ew, sub, n_pass, part, counters,
                                        blocks, status);
    WICK_CUDA_TRY(cudaGetLastError());
    return WICK_OK;
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// exponent bound of the largest colour-list weight sum of each block type
WeightExp weight_exponents(const BlockPlan &plan) {
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
    return ew;
}

// Upper-spin plans with a proton-like type (pair flavour u) and a neutron-like type (pair flavour d) whose
// diquark lists are the proton's with the two rows of every term exchanged (same rows staged for both
// flavours, same colour terms, same weight bound): block_pair_kernel builds both from one X.
bool pair_plan(const BlockPlan &plan, int *oP, int *oN) {
    if (current_tuning().no_pair_kernel) return false;
    if (tc_family(plan) != 1 || plan.n_ops != 2 || plan.f1[0] == plan.f1[1]) return false;
    *oP = plan.f1[0] == 0 ? 0 : 1;
    *oN = 1 - *oP;
    if (plan.n_rows[0] != plan.n_rows[1]) return false;
    for (int k = 0; k < plan.n_rows[0]; ++k)
        if (plan.rows[0][k] != plan.rows[1][k]) return false;
    const WeightExp ew = weight_exponents(plan);
    if (ew.e[0] != ew.e[1]) return false;
    const int ns = plan.n_spin;
    const int tP = plan.os_off[*oP * ns], tN = plan.os_off[*oN * ns];
    const int n_a = plan.os_off[*oP * ns + 1] - tP;
    if (plan.os_off[*oN * ns + 1] - tN != n_a) return false;
    for (int a = 0; a < n_a; ++a) {
        const int lp = plan.os_x[tP + a], ln = plan.os_x[tN + a];
        const int np = plan.x_off[lp + 1] - plan.x_off[lp];
        if (plan.x_off[ln + 1] - plan.x_off[ln] != np) return false;
        for (int i = 0; i < np; ++i) {   // every exchanged proton term is a neutron term
            const int qp = plan.x_off[lp] + i;
            bool found = false;
            for (int k = 0; k < np && !found; ++k) {
                const int qn = plan.x_off[ln] + k;
                found = plan.xt_r2[qn] == plan.xt_r3[qp] && plan.xt_r3[qn] == plan.xt_r2[qp] &&
                        plan.xt_w[qn] == plan.xt_w[qp];
            }
            if (!found) return false;
        }
    }
    return true;
}

template <typename ST>
int launch_pair(const BlockPlan &plan, const CfgPtrs &cp, int n_cfg, int V, int n_slices, int n_ranges,
                int range_sites, const WeightExp &ew, int oP, int oN, double2 *part, int *counters, double2 *blocks,
                int *status, cudaStream_t stream) {
    auto k = block_pair_kernel<ST>;
    WICK_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, PairShape::SMEM));
    dim3 grid(1, n_ranges, n_cfg * n_slices);
    k<<<grid, kThr, PairShape::SMEM, stream>>>(plan, cp, V, n_slices, n_ranges, range_sites, ew, oP, oN, part,
                                                counters, blocks, status);
    WICK_CUDA_TRY(cudaGetLastError());
    return WICK_OK;
}

}  // namespace

bool tc_applicable(const BlockPlan &plan) { return tc_family(plan) != 0; }

bool tc_applicable_3pt(const BlockPlan &plan, int sub) {
    return tc_family(plan) != 0 && (sub == 0 || sub == 1) &&
           plan.n_rows[0] + plan.n_rows[1] + plan.n_rows[sub] <= kMaxRows;
}

int selftest_mbar_wait(int limit, int *status, cudaStream_t stream) {
    mbar_wait_selftest_kernel<<<1, 1, 0, stream>>>(limit, status);
    WICK_CUDA_TRY(cudaGetLastError());
    WICK_CUDA_TRY(cudaStreamSynchronize(stream));
    return WICK_OK;
}

int tc_range_sites(int requested) {
    return requested >= kRoundSites && requested % kRoundSites == 0 && requested <= 4096 ? requested
                                                                                          : kRangeSitesDefault;
}

// The range size of a launch: the requested one, else 1024 sites for the pair kernel and the full-spin
// shape (the per-CTA scan and epilogue amortised over more sites: -4 to -5 % on one-source slabs) when
// that still gives at least 8 waves of CTAs, and 512 otherwise.
int tc_range_for(const BlockPlan &plan, int requested, int n_pass, int n_cfg, int n_slices, int V) {
    if (requested >= kRoundSites && requested % kRoundSites == 0 && requested <= 4096) return requested;
    int oP, oN;
    const bool pair = n_pass == 1 && pair_plan(plan, &oP, &oN);
    const bool full = tc_family(plan) == 2;
    if (!pair && !full) return kRangeSitesDefault;
    int dev = 0, n_sm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t per_range = pair ? 1 : (int64_t)plan.n_ops * FullShape::NCT * n_pass;
    const int64_t ctas = (int64_t)n_cfg * n_slices * per_range *
                         ((V + kPairRangeSitesDefault - 1) / kPairRangeSitesDefault);
    return ctas >= 8 * (int64_t)n_sm ? kPairRangeSitesDefault : kRangeSitesDefault;
}

int tc_max_configs() { return kMaxCfg; }

size_t tc_counter_bytes(const BlockPlan &plan, int n_slices, int n_cfg) {
    return align256(sizeof(int) * (size_t)n_cfg * n_slices * plan.n_ops);
}

size_t tc_partial_bytes(const BlockPlan &plan, int V, int n_slices, int n_cfg, int range_sites, int n_pass) {
    const int rs = tc_range_for(plan, range_sites, n_pass, n_cfg, n_slices, V);
    const size_t n_ranges = (size_t)(V + rs - 1) / rs;
    return sizeof(double2) * n_pass * n_ranges * n_cfg * n_slices * plan.n_out;
}

int launch_block_tc(const BlockPlan &plan, const void *const *Su, const void *const *Sd, int n_cfg, int dtype, int V,
                    int n_slices, int range_sites, int *counters, double2 *part, double2 *blocks, int *status,
                    cudaStream_t stream, const void *const *Sg, int sub) {
    const int fam = tc_family(plan);
    const int rs = tc_range_for(plan, range_sites, sub >= 0 ? 3 : 1, n_cfg, n_slices, V);
    const int n_ranges = (V + rs - 1) / rs;
    if (!fam || n_cfg < 1 || n_cfg > kMaxCfg || n_ranges > 65535 || (int64_t)n_cfg * n_slices > 65535)
        return WICK_EINVAL;
    if (!counters || !part) return WICK_EINVAL;
    if (sub >= 0 && (!Sg || !tc_applicable_3pt(plan, sub))) return WICK_EINVAL;
    const int n_pass = sub >= 0 ? 3 : 1;
    CfgPtrs cp{};
    for (int c = 0; c < n_cfg; ++c) {
        cp.su[c] = Su[c];
        cp.sd[c] = Sd[c];
        cp.sg[c] = sub >= 0 ? Sg[c] : nullptr;
        if (sub >= 0 && !Sg[c]) return WICK_EINVAL;
    }
    const WeightExp ew = weight_exponents(plan);
    int oP = 0, oN = 1;
    if (sub < 0 && pair_plan(plan, &oP, &oN))
        return dtype == WICK_C64 ? launch_pair<float2>(plan, cp, n_cfg, V, n_slices, n_ranges, rs, ew, oP, oN, part,
                                                       counters, blocks, status, stream)
                                 : launch_pair<double2>(plan, cp, n_cfg, V, n_slices, n_ranges, rs, ew, oP, oN, part,
                                                        counters, blocks, status, stream);
    if (dtype == WICK_C64)
        return fam == 1 ? launch_shape<UpperShape, float2>(plan, cp, n_cfg, V, n_slices, n_ranges, rs, ew, sub, n_pass,
                                                           part, counters, blocks, status, stream)
                        : launch_shape<FullShape, float2>(plan, cp, n_cfg, V, n_slices, n_ranges, rs, ew, sub, n_pass,
                                                          part, counters, blocks, status, stream);
    return fam == 1 ? launch_shape<UpperShape, double2>(plan, cp, n_cfg, V, n_slices, n_ranges, rs, ew, sub, n_pass,
                                                        part, counters, blocks, status, stream)
                    : launch_shape<FullShape, double2>(plan, cp, n_cfg, V, n_slices, n_ranges, rs, ew, sub, n_pass,
                                                       part, counters, blocks, status, stream);
}

}  // namespace wick
