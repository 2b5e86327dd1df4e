// Point-sink correlators by the determinant algorithm (Sec. III.A, Eq. 2.9;
// Sec. III.C, improved method B; App. A, Eqs. a1-a4).
//
// Reduction (host + device, once per operator pair):
//   1. antisymmetrise sink and source within each flavour: every index tuple
//      is sorted per flavour with the sign of the sorting, tuples with a
//      repeated index of one flavour vanish, equal tuples are merged (the
//      flavour-ordered lists M, M' of method A);
//   2. the candidate determinants are the pairs (sink index set, source index
//      set) of each flavour -- every distinct sink set meets every distinct
//      source set;
//   3. identity testing (Sec. III.B, App. C): each candidate is evaluated
//      mod p = 2^61 - 1 at `trials` random integer 12 x 12 matrices on the
//      device; equal value vectors (up to a canonical sign) are one
//      determinant of the minimal set zeta_f, all-zero vectors vanish;
//   4. Theta(k, l) = sum over (M, M') of C[M] C'[M'] times the signs of the
//      two determinants relative to their representatives (exact int64,
//      merged by sorting).
// Evaluation (device, FP64): a persistent grid walks (slice, chunk of sites);
// per site the CTA stages S_u(x), S_d(x) (12 x 12 complex each), computes
// every determinant of zeta_u and zeta_d into its scratch (one thread per
// determinant: explicit forms up to 3 x 3, LU with partial pivoting above),
// and sums Theta(k, l) U_k D_l; chunk partials are reduced in a fixed order.
#include <algorithm>
#include <cstring>
#include <map>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "df32.cuh"

#include <type_traits>

struct wick_det_plan {
    int n_u = 0, n_d = 0, device = 0;
    int64_t n_snk = 0, n_src = 0, n_zu = 0, n_zd = 0, n_theta = 0;
    int n_el = 1;                             // matrix elements (sink operator, source operator)
    int8_t *d_zu = nullptr, *d_zd = nullptr;  // [n][2][n_f]: rows (sink indices) then columns (source indices)
    int32_t *d_k = nullptr, *d_l = nullptr;
    double *d_w = nullptr;
    float2 *d_wf = nullptr;   // the same weights as float pairs (hi, lo), for the double-FP32 kernel
    int64_t *d_el_off = nullptr;              // Theta entries of element e: [el_off[e], el_off[e + 1])
    std::vector<int8_t> zu, zd;
    std::vector<int32_t> k, l;
    std::vector<int64_t> w, el_off;
};

namespace wick {

namespace {

// threads per CTA: 512 for the double-FP32 single-element kernel (its Theta gathers are latency-bound
// and it fits 128 registers), else 256
template <typename C, int MAXEL> __host__ __device__ constexpr int det_threads() {
    return std::is_same<C, cdf>::value && MAXEL == 1 ? 512 : 256;
}
constexpr int kDetChunk = 32;  // sites per work item at most (fewer when that leaves SMs idle)
constexpr int kMaxEl = 16;     // matrix elements (a 4 x 4 correlation matrix)
constexpr int kTheta = 8;      // Theta entries per thread in flight (double-FP32; FP64 is bound by its pipe)
constexpr uint64_t kP61 = (1ull << 61) - 1;

// ---------------------------------------------------------------------------
// mod-p determinants (identity testing)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t mulmod(uint64_t a, uint64_t b) {
    const uint64_t lo = a * b, hi = __umul64hi(a, b);
    uint64_t s = (lo & kP61) + ((lo >> 61) | (hi << 3));  // a, b < p: both parts < 2^61
    s = (s & kP61) + (s >> 61);
    return s >= kP61 ? s - kP61 : s;
}
__device__ __forceinline__ uint64_t submod(uint64_t a, uint64_t b) { return a >= b ? a - b : a + kP61 - b; }
__device__ uint64_t powmod(uint64_t a, uint64_t e) {
    uint64_t r = 1;
    while (e) {
        if (e & 1) r = mulmod(r, a);
        a = mulmod(a, a);
        e >>= 1;
    }
    return r;
}

// random 12 x 12 matrix entry e of (seed, trial, flavour), uniform in [0, p) up to a 2^-61 bias
__device__ __forceinline__ uint64_t rand_entry(uint64_t seed, int trial, int flavour, int e) {
    const uint64_t key = mix64(seed ^ (0xA5A5000000000000ull + 16ull * (uint64_t)trial + (uint64_t)flavour));
    return mix64(key + (uint64_t)(e + 1) * 0x9E3779B97F4A7C15ull) % kP61;
}

// det mod p of M[rows][cols] for every (sink set i, source set j): Gaussian elimination mod p
__global__ void det_modp_kernel(const int8_t *__restrict__ snk_sets, int n_snk_sets, const int8_t *__restrict__ src_sets,
                                int n_src_sets, int n, uint64_t seed, int trials, int flavour,
                                uint64_t *__restrict__ out) {
    __shared__ uint64_t M[144];
    const int64_t total = (int64_t)n_snk_sets * n_src_sets;
    for (int tr = 0; tr < trials; ++tr) {
        __syncthreads();
        for (int e = threadIdx.x; e < 144; e += blockDim.x) M[e] = rand_entry(seed, tr, flavour, e);
        __syncthreads();
        for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (int64_t)gridDim.x * blockDim.x) {
            const int8_t *r = snk_sets + (c / n_src_sets) * n, *q = src_sets + (c % n_src_sets) * n;
            uint64_t a[6][6];
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) a[i][j] = M[r[i] * 12 + q[j]];
            uint64_t det = 1;
            for (int col = 0; col < n && det; ++col) {
                int p = col;
                while (p < n && a[p][col] == 0) ++p;
                if (p == n) {
                    det = 0;
                    break;
                }
                if (p != col) {
                    for (int j = 0; j < n; ++j) {
                        const uint64_t t = a[p][j];
                        a[p][j] = a[col][j];
                        a[col][j] = t;
                    }
                    det = kP61 - det;
                }
                det = mulmod(det, a[col][col]);
                const uint64_t inv = powmod(a[col][col], kP61 - 2);
                for (int i = col + 1; i < n; ++i) {
                    const uint64_t f = mulmod(a[i][col], inv);
                    for (int j = col; j < n; ++j) a[i][j] = submod(a[i][j], mulmod(f, a[col][j]));
                }
            }
            out[c * trials + tr] = det % kP61;
        }
    }
}

// ---------------------------------------------------------------------------
// FP64 determinants of submatrices of a 12 x 12 complex matrix in shared memory
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
// the same on double-FP32 complex values (the WICK_MIXED evaluation)
__device__ __forceinline__ cdf cmul(const cdf &a, const cdf &b) { return cdf_mul(a, b); }
__device__ __forceinline__ cdf cadd(const cdf &a, const cdf &b) { return {df_add(a.x, b.x), df_add(a.y, b.y)}; }
__device__ __forceinline__ cdf csub(const cdf &a, const cdf &b) {
    return {df_add(a.x, df_neg(b.x)), df_add(a.y, df_neg(b.y))};
}
template <typename C> __device__ __forceinline__ C to_c(float2 v);
template <> __device__ __forceinline__ double2 to_c<double2>(float2 v) { return make_double2(v.x, v.y); }
template <> __device__ __forceinline__ cdf to_c<cdf>(float2 v) { return {{v.x, 0.f}, {v.y, 0.f}}; }
template <typename C> __device__ __forceinline__ C to_c(double2 v);
template <> __device__ __forceinline__ double2 to_c<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ cdf to_c<cdf>(double2 v) { return {split_double(v.x), split_double(v.y)}; }
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(const cdf &v) { return make_double2(to_double(v.x), to_double(v.y)); }
// acc += w p with an integer weight w
__device__ __forceinline__ void theta_acc(double2 &acc, double w, double2 p) {
    acc.x = fma(w, p.x, acc.x);
    acc.y = fma(w, p.y, acc.y);
}
__device__ __forceinline__ void theta_acc(cdf &acc, float2 w, const cdf &p) {
    const df wd = {w.x, w.y};
    acc.x = df_add(acc.x, df_mul(wd, p.x));
    acc.y = df_add(acc.y, df_mul(wd, p.y));
}

// determinant of the n x n matrix row[i][cols[j]] (rows given as pointers into 12 x 12 matrices, so
// that a row can come from another propagator)
template <int N>
__device__ __forceinline__ double2 det_lu(const double2 *const *row, const int8_t *cols) {
    double2 a[N][N];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) a[i][j] = row[i][cols[j]];
    double2 det = make_double2(1.0, 0.0);
#pragma unroll
    for (int c = 0; c < N; ++c) {
        // partial pivoting on |re| + |im|, rows swapped by selects (no dynamic register indexing)
        int p = c;
        double best = fabs(a[c][c].x) + fabs(a[c][c].y);
#pragma unroll
        for (int r = c + 1; r < N; ++r) {
            const double m = fabs(a[r][c].x) + fabs(a[r][c].y);
            if (m > best) {
                best = m;
                p = r;
            }
        }
        if (best == 0.0) return make_double2(0.0, 0.0);
        if (p != c) det = make_double2(-det.x, -det.y);
#pragma unroll
        for (int r = c + 1; r < N; ++r) {
            if (r == p) {
#pragma unroll
                for (int j = c; j < N; ++j) {
                    const double2 t = a[r][j];
                    a[r][j] = a[c][j];
                    a[c][j] = t;
                }
            }
        }
        det = cmul(det, a[c][c]);
        const double2 d = a[c][c];
        const double inv_n = 1.0 / (d.x * d.x + d.y * d.y);
        const double2 inv = make_double2(d.x * inv_n, -d.y * inv_n);
#pragma unroll
        for (int r = c + 1; r < N; ++r) {
            const double2 f = cmul(a[r][c], inv);
#pragma unroll
            for (int j = c + 1; j < N; ++j) a[r][j] = csub(a[r][j], cmul(f, a[c][j]));
        }
    }
    return det;
}

__device__ __forceinline__ double2 det_rows(const double2 *const *row, const int8_t *cols, int n) {
    switch (n) {
    case 1:
        return row[0][cols[0]];
    case 2:
        return csub(cmul(row[0][cols[0]], row[1][cols[1]]), cmul(row[0][cols[1]], row[1][cols[0]]));
    case 3: {
        const double2 *r0 = row[0], *r1 = row[1], *r2 = row[2];
        const int c0 = cols[0], c1 = cols[1], c2 = cols[2];
        const double2 m0 = csub(cmul(r1[c1], r2[c2]), cmul(r1[c2], r2[c1]));
        const double2 m1 = csub(cmul(r1[c0], r2[c2]), cmul(r1[c2], r2[c0]));
        const double2 m2 = csub(cmul(r1[c0], r2[c1]), cmul(r1[c1], r2[c0]));
        return cadd(csub(cmul(r0[c0], m0), cmul(r0[c1], m1)), cmul(r0[c2], m2));
    }
    case 4:
        return det_lu<4>(row, cols);
    case 5:
        return det_lu<5>(row, cols);
    case 6:
        return det_lu<6>(row, cols);
    default:
        return make_double2(1.0, 0.0);  // no quark of this flavour
    }
}

// rc: n row indices (sink) then n column indices (source) of S
__device__ __forceinline__ double2 det_small(const double2 *S, const int8_t *rc, int n) {
    const double2 *row[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) row[i] = S + (i < n ? rc[i] : 0) * 12;
    return det_rows(row, rc + n, n);
}

// the derivative of det S[rows][cols] in the direction Sig: the sum over the row taken from Sig
__device__ __forceinline__ double2 det_deriv(const double2 *S, const double2 *Sig, const int8_t *rc, int n) {
    double2 acc = make_double2(0.0, 0.0);
    for (int rep = 0; rep < n; ++rep) {
        const double2 *row[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) row[i] = (i == rep ? Sig : S) + (i < n ? rc[i] : 0) * 12;
        acc = cadd(acc, det_rows(row, rc + n, n));
    }
    return acc;
}

// ---------------------------------------------------------------------------
// determinants from a per-site table of all 2 x 2 minors of a 12 x 12 matrix:
// M2[pair(r0, r1)][pair(c0, c1)] = S[r0][c0] S[r1][c1] - S[r0][c1] S[r1][c0], pair(i < j) in 0..65
// ---------------------------------------------------------------------------
constexpr int kPairs = 66;
__host__ __device__ constexpr int pair_index(int i, int j) { return i * (23 - i) / 2 + (j - i - 1); }

template <typename C> __device__ __forceinline__ C m2(const C *M, int r0, int r1, int c0, int c1) {
    return M[pair_index(r0, r1) * kPairs + pair_index(c0, c1)];
}

// 4 x 4 by Laplace expansion along rows (r0, r1): sum over column pairs of the signed products of
// complementary 2 x 2 minors
template <typename C>
__device__ __forceinline__ C det4_m2(const C *M, int r0, int r1, int r2, int r3, const int *c) {
    C d = cmul(m2(M, r0, r1, c[0], c[1]), m2(M, r2, r3, c[2], c[3]));
    d = csub(d, cmul(m2(M, r0, r1, c[0], c[2]), m2(M, r2, r3, c[1], c[3])));
    d = cadd(d, cmul(m2(M, r0, r1, c[0], c[3]), m2(M, r2, r3, c[1], c[2])));
    d = cadd(d, cmul(m2(M, r0, r1, c[1], c[2]), m2(M, r2, r3, c[0], c[3])));
    d = csub(d, cmul(m2(M, r0, r1, c[1], c[3]), m2(M, r2, r3, c[0], c[2])));
    return cadd(d, cmul(m2(M, r0, r1, c[2], c[3]), m2(M, r2, r3, c[0], c[1])));
}

// det of S[rc[0..n)][rc[n..2n)] for n <= 5 from the minor table (n = 6 falls back to LU)
template <typename C> __device__ __forceinline__ C det_minors(const C *S, const C *M, const int8_t *rc, int n) {
    switch (n) {
    case 1:
        return S[rc[0] * 12 + rc[1]];
    case 2:
        return m2(M, rc[0], rc[1], rc[2], rc[3]);
    case 3: {
        const C *r0 = S + rc[0] * 12;
        const int a = rc[1], b = rc[2], c0 = rc[3], c1 = rc[4], c2 = rc[5];
        return cadd(csub(cmul(r0[c0], m2(M, a, b, c1, c2)), cmul(r0[c1], m2(M, a, b, c0, c2))),
                    cmul(r0[c2], m2(M, a, b, c0, c1)));
    }
    case 4: {
        const int c[4] = {rc[4], rc[5], rc[6], rc[7]};
        return det4_m2(M, rc[0], rc[1], rc[2], rc[3], c);
    }
    case 5: {
        // along the first row: sum_j (-1)^j S[r0][c_j] det4(rows r1..r4, columns without c_j)
        const C *r0 = S + rc[0] * 12;
        C d = C{};
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            int c[4], q = 0;
#pragma unroll
            for (int k = 0; k < 5; ++k)
                if (k != j) c[q++] = rc[5 + k];
            const C t = cmul(r0[rc[5 + j]], det4_m2(M, rc[1], rc[2], rc[3], rc[4], c));
            d = (j & 1) ? csub(d, t) : cadd(d, t);
        }
        return d;
    }
    default:
        if constexpr (std::is_same<C, double2>::value) return det_small(S, rc, n);
        else return C{};
    }
}

// ---------------------------------------------------------------------------
// 5 x 5 and 6 x 6 determinants from a per-site table of all 3 x 3 minors (in global scratch):
// M3[tri(r0, r1, r2)][tri(c0, c1, c2)], tri(i < j < k) = C(k, 3) + C(j, 2) + i in 0..219, built
// from the 2 x 2 minors by the first row.  5 x 5: Laplace expansion along the first two rows over
// the 10 column pairs; 6 x 6: along the first three rows over the 20 column triples.
// ---------------------------------------------------------------------------
constexpr int kTriples = 220;
__host__ __device__ constexpr int tri_index(int i, int j, int k) {
    return k * (k - 1) * (k - 2) / 6 + j * (j - 1) / 2 + i;
}

template <typename C>
__device__ __forceinline__ C m3(const C *__restrict__ T3, int r0, int r1, int r2, int c0, int c1, int c2) {
    return T3[tri_index(r0, r1, r2) * kTriples + tri_index(c0, c1, c2)];
}

template <typename C>
__device__ __forceinline__ C det_m3(const C *M, const C *__restrict__ T3, const int8_t *rc, int n) {
    const int8_t *r = rc, *c = rc + n;
    C d = C{};
    if (n == 5) {
#pragma unroll
        for (int a = 0; a < 5; ++a)
#pragma unroll
            for (int b = a + 1; b < 5; ++b) {
                int q[3], k = 0;
#pragma unroll
                for (int j = 0; j < 5; ++j)
                    if (j != a && j != b) q[k++] = c[j];
                const C t = cmul(m2(M, r[0], r[1], c[a], c[b]), m3(T3, r[2], r[3], r[4], q[0], q[1], q[2]));
                d = ((a + b) & 1) ? cadd(d, t) : csub(d, t);   // (-1)^(1 + a + b)
            }
    } else {   // n == 6
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int b = a + 1; b < 6; ++b)
#pragma unroll
                for (int e = b + 1; e < 6; ++e) {
                    int q[3], k = 0;
#pragma unroll
                    for (int j = 0; j < 6; ++j)
                        if (j != a && j != b && j != e) q[k++] = c[j];
                    const C t = cmul(m3(T3, r[0], r[1], r[2], c[a], c[b], c[e]),
                                           m3(T3, r[3], r[4], r[5], q[0], q[1], q[2]));
                    d = ((a + b + e) & 1) ? cadd(d, t) : csub(d, t);   // (-1)^(3 + a + b + e)
                }
    }
    return d;
}

// Derivative of det S[r][c] in the direction Sig (the three-point insertion) for n <= 3, by the
// cofactor expansion of each row-replaced determinant: sum_{i,j} (-1)^(i+j) Sig[r_i][c_j] times the
// minor of S without row r_i and column c_j (from the 2 x 2 minor table for n = 3).
template <typename C>
__device__ __forceinline__ C det_deriv_m2(const C *S, const C *Sig, const C *M, const int8_t *rc, int n) {
    const int8_t *r = rc, *c = rc + n;
    if (n == 1) return Sig[r[0] * 12 + c[0]];
    C d = C{};
    if (n == 2) {
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const C t = cmul(Sig[r[i] * 12 + c[j]], S[r[1 - i] * 12 + c[1 - j]]);
                d = ((i + j) & 1) ? csub(d, t) : cadd(d, t);
            }
        return d;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int ra = r[i == 0 ? 1 : 0], rb = r[i == 2 ? 1 : 2];
            const int ca = c[j == 0 ? 1 : 0], cb = c[j == 2 ? 1 : 2];
            const C t = cmul(Sig[r[i] * 12 + c[j]], m2(M, ra, rb, ca, cb));
            d = ((i + j) & 1) ? csub(d, t) : cadd(d, t);
        }
    return d;
}

struct DetArgs {
    int n_u, n_d, n_el;
    int seq_flavour;          // -1: two-point function; 0 / 1: current on u / d through Sig
    int m3_mask;              // bit f: flavour f (n_f = 5 or 6) takes the 3 x 3 minor table
    int64_t n_zu, n_zd;
    const int8_t *zu, *zd;
    const int32_t *k, *l;
    const double *w;
    const float2 *wf;
    const int64_t *el_off;
};

// C = double2: FP64 throughout; C = cdf: double-FP32 (the float pipes) for the minor tables,
// determinants and the Theta sum, FP64 for the per-chunk reduction.
template <typename ST, typename C, int MAXEL>
__global__ void __launch_bounds__(det_threads<C, MAXEL>())
det_eval_kernel(const DetArgs a, const ST *__restrict__ Su, const ST *__restrict__ Sd, const ST *__restrict__ Sig,
                int V, int n_slices, int n_chunks, int chunk_sites, double2 *__restrict__ scratch,
                double2 *__restrict__ partials) {
    static_assert(sizeof(C) == sizeof(double2), "one 16-byte complex value");
    constexpr int kDetThreads = det_threads<C, MAXEL>();
    __shared__ C sS[3][144];
    __shared__ double2 red[kDetThreads];
    extern __shared__ double2 sM_raw[];   // [2][kPairs * kPairs] 2 x 2 minor tables of S_u, S_d
    C *sM = reinterpret_cast<C *>(sM_raw);
    const int n_m3 = (a.m3_mask & 1) + (a.m3_mask >> 1 & 1);
    C *U = reinterpret_cast<C *>(scratch) + (size_t)blockIdx.x * (a.n_zu + a.n_zd + (size_t)n_m3 * kTriples * kTriples);
    C *D = U + a.n_zu;
    C *T3[2];   // this CTA's 3 x 3 minor tables
    T3[0] = D + a.n_zd;
    T3[1] = T3[0] + ((a.m3_mask & 1) ? kTriples * kTriples : 0);
    __shared__ int8_t sTri[kTriples][3];
    const int tid = threadIdx.x;
    if (a.m3_mask)
        for (int t = tid; t < kTriples; t += kDetThreads) {
            int k = 2;
            while (tri_index(0, 1, k + 1) <= t) ++k;   // C(k + 1, 3) <= t
            int j = 1;
            while (tri_index(0, j + 1, k) <= t) ++j;
            sTri[t][0] = (int8_t)(t - tri_index(0, j, k));
            sTri[t][1] = (int8_t)j;
            sTri[t][2] = (int8_t)k;
        }
    const int64_t items = (int64_t)n_slices * n_chunks;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int slice = (int)(it / n_chunks), chunk = (int)(it % n_chunks);
        const int x0 = chunk * chunk_sites, x1 = min(V, x0 + chunk_sites);
        C acc[MAXEL];
#pragma unroll
        for (int e = 0; e < MAXEL; ++e) acc[e] = C{};
        for (int x = x0; x < x1; ++x) {
            __syncthreads();  // the previous site's determinants are consumed
            const int n_mat = a.seq_flavour < 0 ? 2 : 3;
            for (int e = tid; e < 144 * n_mat; e += kDetThreads) {
                const ST *base = e < 144 ? Su : (e < 288 ? Sd : Sig);
                sS[e / 144][e % 144] = to_c<C>(base[((size_t)slice * V + x) * 144 + (e % 144)]);
            }
            __syncthreads();
            for (int e = tid; e < 2 * kPairs * kPairs; e += kDetThreads) {
                const int f = e / (kPairs * kPairs), rp = (e / kPairs) % kPairs, cp = e % kPairs;
                int r0 = 0, c0 = 0;
                while (pair_index(r0, 11) < rp) ++r0;      // first index of the pair
                while (pair_index(c0, 11) < cp) ++c0;
                const int r1 = rp - pair_index(r0, r0 + 1) + r0 + 1, c1 = cp - pair_index(c0, c0 + 1) + c0 + 1;
                const C *S = sS[f];
                sM[e] = csub(cmul(S[r0 * 12 + c0], S[r1 * 12 + c1]), cmul(S[r0 * 12 + c1], S[r1 * 12 + c0]));
            }
            __syncthreads();
            if (a.m3_mask) {
                for (int f = 0; f < 2; ++f) {
                    if (!(a.m3_mask >> f & 1)) continue;
                    const C *S = sS[f], *M = sM + f * kPairs * kPairs;
                    for (int e = tid; e < kTriples * kTriples; e += kDetThreads) {
                        const int rt = e / kTriples, ct = e - rt * kTriples;
                        const int r0 = sTri[rt][0], r1 = sTri[rt][1], r2 = sTri[rt][2];
                        const int c0 = sTri[ct][0], c1 = sTri[ct][1], c2 = sTri[ct][2];
                        const C *s0 = S + r0 * 12;
                        T3[f][e] = cadd(csub(cmul(s0[c0], m2(M, r1, r2, c1, c2)), cmul(s0[c1], m2(M, r1, r2, c0, c2))),
                                        cmul(s0[c2], m2(M, r1, r2, c0, c1)));
                    }
                }
                __syncthreads();
            }
            // the flavour carrying the current (three-point functions): cofactor expansion for n <= 3,
            // pivoted LU of the row-replaced matrices above (FP64 only)
            for (int f = 0; f < 2; ++f) {
                const int n = f == 0 ? a.n_u : a.n_d;
                const int64_t nz = f == 0 ? a.n_zu : a.n_zd;
                const int8_t *z = f == 0 ? a.zu : a.zd;
                C *out = f == 0 ? U : D;
                const C *M = sM + f * kPairs * kPairs;
                if (a.seq_flavour == f) {
                    for (int64_t q = tid; q < nz; q += kDetThreads) {
                        if (n <= 3) out[q] = det_deriv_m2(sS[f], sS[2], M, z + q * 2 * n, n);
                        else if constexpr (std::is_same<C, double2>::value)
                            out[q] = det_deriv(sS[f], sS[2], z + q * 2 * n, n);
                    }
                } else if (a.m3_mask >> f & 1) {
                    for (int64_t q = tid; q < nz; q += kDetThreads) out[q] = det_m3(M, T3[f], z + q * 2 * n, n);
                } else {
                    for (int64_t q = tid; q < nz; q += kDetThreads) out[q] = det_minors(sS[f], M, z + q * 2 * n, n);
                }
            }
            __syncthreads();
            // the determinants are shared by every matrix element (Eq. E3).  The gathers of U[k] and
            // D[l] come from L2: in double-FP32 each thread keeps kTheta of them in flight.
            constexpr int KT = std::is_same<C, cdf>::value ? kTheta : 1;
#pragma unroll
            for (int el = 0; el < MAXEL; ++el) {
                if (el >= a.n_el) break;
                const int64_t end = a.el_off[el + 1];
                for (int64_t e0 = a.el_off[el] + tid; e0 < end; e0 += KT * kDetThreads) {
                    using W = typename std::conditional<std::is_same<C, cdf>::value, float2, double>::type;
                    int kk[KT], ll[KT];
                    W ww[KT];
#pragma unroll
                    for (int u = 0; u < KT; ++u) {
                        const int64_t e = e0 + u * kDetThreads;
                        const bool ok = e < end;
                        kk[u] = ok ? a.k[e] : 0;
                        ll[u] = ok ? a.l[e] : 0;
                        if constexpr (std::is_same<C, cdf>::value) ww[u] = ok ? a.wf[e] : make_float2(0.f, 0.f);
                        else ww[u] = ok ? a.w[e] : 0.0;   // a zero weight adds nothing
                    }
                    C uu[KT], dd[KT];
#pragma unroll
                    for (int u = 0; u < KT; ++u) {
                        uu[u] = U[kk[u]];
                        dd[u] = D[ll[u]];
                    }
#pragma unroll
                    for (int u = 0; u < KT; ++u) theta_acc(acc[el], ww[u], cmul(uu[u], dd[u]));
                }
            }
        }
        // fixed-order block reduction of the chunk's sums (FP64)
#pragma unroll
        for (int el = 0; el < MAXEL; ++el) {
            if (el >= a.n_el) break;
            red[tid] = to_d2(acc[el]);
            __syncthreads();
            for (int s = kDetThreads / 2; s > 0; s >>= 1) {
                if (tid < s) red[tid] = cadd(red[tid], red[tid + s]);
                __syncthreads();
            }
            if (tid == 0) partials[((size_t)slice * n_chunks + chunk) * a.n_el + el] = red[0];
            __syncthreads();
        }
    }
}

// out[el][slice] = scale * sum over chunks (fixed order)
__global__ void det_finish_kernel(const double2 *__restrict__ partials, int n_slices, int n_chunks, int n_el,
                                  double scale, double2 *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_slices * n_el) return;
    const int el = i / n_slices, s = i % n_slices;
    double2 acc = make_double2(0.0, 0.0);
    for (int c = 0; c < n_chunks; ++c) acc = cadd(acc, partials[((size_t)s * n_chunks + c) * n_el + el]);
    out[i] = make_double2(scale * acc.x, scale * acc.y);
}

// ---------------------------------------------------------------------------
// host: antisymmetrisation and the minimal sets
// ---------------------------------------------------------------------------
using Key = std::vector<int8_t>;

struct Antisym {
    std::map<std::pair<Key, Key>, int64_t> terms;  // (sorted u set, sorted d set) -> weight
};

int antisymmetrise(const wick_quark_operator *op, Antisym &out) {
    if (!op || op->n_u < 0 || op->n_d < 0 || op->n_u > 6 || op->n_d > 6 || op->n_u + op->n_d < 1 ||
        op->n_terms < 0 || (op->n_terms > 0 && (!op->chi || !op->w)))
        return WICK_EINVAL;
    const int n = op->n_u + op->n_d;
    for (int t = 0; t < op->n_terms; ++t) {
        const int8_t *c = op->chi + (size_t)t * n;
        const int64_t w = op->w[t];
        if (w >= (1ll << 31) || w <= -(1ll << 31)) return WICK_EINVAL;
        Key u(c, c + op->n_u), d(c + op->n_u, c + n);
        int sign = 1;
        bool zero = false;
        for (Key *f : {&u, &d}) {
            for (int8_t v : *f)
                if (v < 0 || v > 11) return WICK_EINVAL;
            // insertion sort counting transpositions; a repeated index makes the term vanish
            for (size_t i = 1; i < f->size(); ++i)
                for (size_t j = i; j > 0 && (*f)[j - 1] >= (*f)[j]; --j) {
                    if ((*f)[j - 1] == (*f)[j]) zero = true;
                    std::swap((*f)[j - 1], (*f)[j]);
                    sign = -sign;
                }
        }
        if (zero || w == 0) continue;
        out.terms[{u, d}] += sign * w;
    }
    for (auto it = out.terms.begin(); it != out.terms.end();)
        it = it->second == 0 ? out.terms.erase(it) : std::next(it);
    return WICK_OK;
}

struct Classes {
    std::vector<int> cls;    // per candidate (sink set * n_src_sets + source set): class or -1
    std::vector<int> sign;   // relative to the class representative
    std::vector<int64_t> rep;  // candidate index of each class's representative
};

int classify(const std::vector<Key> &snk, const std::vector<Key> &src, int n, uint64_t seed, int trials, int flavour,
             Classes &out) {
    const int64_t total = (int64_t)snk.size() * (int64_t)src.size();
    out.cls.assign(total, -1);
    out.sign.assign(total, 0);
    if (total == 0) return WICK_OK;
    if (n == 0) {  // no quark of this flavour: one determinant, equal to 1
        for (int64_t c = 0; c < total; ++c) {
            out.cls[c] = 0;
            out.sign[c] = 1;
        }
        out.rep.push_back(0);
        return WICK_OK;
    }
    std::vector<int8_t> hs(snk.size() * n), hq(src.size() * n);
    for (size_t i = 0; i < snk.size(); ++i) std::copy(snk[i].begin(), snk[i].end(), hs.begin() + i * n);
    for (size_t i = 0; i < src.size(); ++i) std::copy(src[i].begin(), src[i].end(), hq.begin() + i * n);
    int8_t *ds = nullptr, *dq = nullptr;
    uint64_t *dv = nullptr;
    auto cleanup = [&]() {
        cudaFree(ds);
        cudaFree(dq);
        cudaFree(dv);
    };
    if (dev_malloc((void **)&ds, hs.size()) != WICK_OK || dev_malloc((void **)&dq, hq.size()) != WICK_OK ||
        dev_malloc((void **)&dv, sizeof(uint64_t) * total * trials) != WICK_OK) {
        cleanup();
        (void)cudaGetLastError();
        return WICK_ENOMEM;
    }
    std::vector<uint64_t> hv((size_t)total * trials);
    int err = WICK_OK;
    if (cudaMemcpy(ds, hs.data(), hs.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dq, hq.data(), hq.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        err = WICK_ECUDA;
    if (!err) {
        const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
        det_modp_kernel<<<blocks, 256>>>(ds, (int)snk.size(), dq, (int)src.size(), n, seed, trials, flavour, dv);
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(hv.data(), dv, sizeof(uint64_t) * hv.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
            err = WICK_ECUDA;
    }
    cleanup();
    if (err) return err;
    struct VecHash {
        size_t operator()(const std::vector<uint64_t> &v) const {
            uint64_t h = 0x9E3779B97F4A7C15ull;
            for (uint64_t x : v) h = mix64(h ^ x);
            return (size_t)h;
        }
    };
    std::unordered_map<std::vector<uint64_t>, int, VecHash> map;
    std::vector<int> rep_sign;
    std::vector<uint64_t> key(trials);
    for (int64_t c = 0; c < total; ++c) {
        bool nz = false;
        int s = 1;
        uint64_t first = 0;
        for (int t = 0; t < trials; ++t) {
            key[t] = hv[c * trials + t];
            if (!nz && key[t]) {
                nz = true;
                first = key[t];
            }
        }
        if (!nz) continue;  // identically zero determinant
        if (first > (kP61 - 1) / 2) {
            s = -1;
            for (auto &v : key) v = v ? kP61 - v : 0;
        }
        auto it = map.find(key);
        int cl;
        if (it == map.end()) {
            cl = (int)out.rep.size();
            map.emplace(key, cl);
            out.rep.push_back(c);
            rep_sign.push_back(s);
        } else {
            cl = it->second;
        }
        out.cls[c] = cl;
        out.sign[c] = s * rep_sign[cl];
    }
    return WICK_OK;
}

void free_plan(wick_det_plan *p) {
    if (!p) return;
    cudaFree(p->d_zu);
    cudaFree(p->d_zd);
    cudaFree(p->d_k);
    cudaFree(p->d_l);
    cudaFree(p->d_w);
    cudaFree(p->d_wf);
    cudaFree(p->d_el_off);
    delete p;
}

template <typename T> int upload(T **dst, const std::vector<T> &src) {
    const size_t bytes = sizeof(T) * std::max<size_t>(src.size(), 1);
    if (dev_malloc((void **)dst, bytes) != WICK_OK) {
        (void)cudaGetLastError();
        *dst = nullptr;
        return WICK_ENOMEM;
    }
    if (!src.empty() && cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return WICK_ECUDA;
    return WICK_OK;
}

}  // namespace

}  // namespace wick

using namespace wick;

extern "C" {

}  // extern "C"

namespace wick {
namespace {

// Minimal sets shared by the elements (i, j) of sinks x sources (Eq. E3) and one Theta per element.
int reduce_matrix(const wick_quark_operator *const *snk, int n_snk_ops, const wick_quark_operator *const *src,
                  int n_src_ops, uint64_t seed, int trials, wick_det_plan **out) {
    if (!out || n_snk_ops < 1 || n_src_ops < 1 || n_snk_ops * n_src_ops > kMaxEl || trials < 1 || trials > 8)
        return WICK_EINVAL;
    *out = nullptr;
    for (int i = 0; i < n_snk_ops; ++i)
        if (!snk[i]) return WICK_EINVAL;
    for (int j = 0; j < n_src_ops; ++j)
        if (!src[j]) return WICK_EINVAL;
    const int nu = snk[0]->n_u, nd = snk[0]->n_d;
    for (int i = 0; i < n_snk_ops; ++i)
        if (snk[i]->n_u != nu || snk[i]->n_d != nd) return WICK_EINVAL;
    for (int j = 0; j < n_src_ops; ++j)
        if (src[j]->n_u != nu || src[j]->n_d != nd) return WICK_EINVAL;
    std::vector<Antisym> As(n_snk_ops), Aq(n_src_ops);
    int err = WICK_OK;
    for (int i = 0; i < n_snk_ops && !err; ++i) err = antisymmetrise(snk[i], As[i]);
    for (int j = 0; j < n_src_ops && !err; ++j) err = antisymmetrise(src[j], Aq[j]);
    if (err) return err;
    // distinct index sets over all sink operators and over all source operators
    auto union_sets = [](const std::vector<Antisym> &ops, bool d_part, std::vector<Key> &sets,
                         std::vector<std::vector<int>> &ids) {
        std::map<Key, int> idx;
        for (auto &A : ops)
            for (auto &kv : A.terms) idx.emplace(d_part ? kv.first.second : kv.first.first, 0);
        int i = 0;
        for (auto &kv : idx) {
            kv.second = i++;
            sets.push_back(kv.first);
        }
        ids.resize(ops.size());
        for (size_t o = 0; o < ops.size(); ++o)
            for (auto &kv : ops[o].terms) ids[o].push_back(idx[d_part ? kv.first.second : kv.first.first]);
    };
    std::vector<Key> su, sd, qu, qd;
    std::vector<std::vector<int>> isu, isd, iqu, iqd;
    union_sets(As, false, su, isu);
    union_sets(As, true, sd, isd);
    union_sets(Aq, false, qu, iqu);
    union_sets(Aq, true, qd, iqd);
    if ((int64_t)su.size() * (int64_t)qu.size() > (1ll << 30) || (int64_t)sd.size() * (int64_t)qd.size() > (1ll << 30))
        return WICK_EINVAL;
    Classes cu, cd;
    err = classify(su, qu, nu, seed, trials, 0, cu);
    if (!err) err = classify(sd, qd, nd, seed, trials, 1, cd);
    if (err) return err;
    wick_det_plan *p = new (std::nothrow) wick_det_plan();
    if (!p) return WICK_ENOMEM;
    p->n_u = nu;
    p->n_d = nd;
    p->n_el = n_snk_ops * n_src_ops;
    cudaGetDevice(&p->device);
    for (auto &A : As) p->n_snk += (int64_t)A.terms.size();
    for (auto &A : Aq) p->n_src += (int64_t)A.terms.size();
    const int64_t n_cd = (int64_t)cd.rep.size();
    p->el_off.push_back(0);
    std::vector<std::pair<int64_t, int64_t>> acc;
    for (int i = 0; i < n_snk_ops; ++i)
        for (int j = 0; j < n_src_ops; ++j) {
            // Theta of element (i, j): every (M, M') -> (class_u, class_d), merged by sorting
            std::vector<int64_t> ws, wq;
            for (auto &kv : As[i].terms) ws.push_back(kv.second);
            for (auto &kv : Aq[j].terms) wq.push_back(kv.second);
            acc.clear();
            acc.reserve(ws.size() * wq.size());
            for (size_t a = 0; a < ws.size(); ++a)
                for (size_t b = 0; b < wq.size(); ++b) {
                    const int64_t ca = (int64_t)isu[i][a] * (int64_t)qu.size() + iqu[j][b];
                    const int64_t cb = (int64_t)isd[i][a] * (int64_t)qd.size() + iqd[j][b];
                    const int ku = cu.cls[ca], kd = cd.cls[cb];
                    if (ku < 0 || kd < 0) continue;
                    acc.push_back({(int64_t)ku * n_cd + kd, ws[a] * wq[b] * cu.sign[ca] * cd.sign[cb]});
                }
            std::sort(acc.begin(), acc.end(),
                      [](const std::pair<int64_t, int64_t> &x, const std::pair<int64_t, int64_t> &y) {
                          return x.first < y.first;
                      });
            for (size_t a = 0; a < acc.size();) {
                size_t b = a;
                int64_t sum = 0;
                for (; b < acc.size() && acc[b].first == acc[a].first; ++b) sum += acc[b].second;
                if (sum != 0) {
                    if (sum >= (1ll << 53) || sum <= -(1ll << 53)) {
                        free_plan(p);
                        return WICK_EOVERFLOW;
                    }
                    p->k.push_back((int32_t)(acc[a].first / n_cd));
                    p->l.push_back((int32_t)(acc[a].first % n_cd));
                    p->w.push_back(sum);
                }
                a = b;
            }
            p->el_off.push_back((int64_t)p->w.size());
        }
    // the minimal sets as (rows, columns) of each representative
    auto pack = [](const Classes &c, const std::vector<Key> &rs, const std::vector<Key> &cs, int n,
                   std::vector<int8_t> &dst) {
        for (int64_t r : c.rep) {
            const int64_t i = cs.empty() ? 0 : r / (int64_t)cs.size(), j = cs.empty() ? 0 : r % (int64_t)cs.size();
            for (int q = 0; q < n; ++q) dst.push_back(rs[i][q]);
            for (int q = 0; q < n; ++q) dst.push_back(cs[j][q]);
        }
    };
    pack(cu, su, qu, nu, p->zu);
    pack(cd, sd, qd, nd, p->zd);
    p->n_zu = (int64_t)cu.rep.size();
    p->n_zd = (int64_t)cd.rep.size();
    p->n_theta = (int64_t)p->w.size();
    std::vector<double> wd(p->w.begin(), p->w.end());
    std::vector<float2> wf(wd.size());
    for (size_t i = 0; i < wd.size(); ++i) {   // exact for |w| < 2^48
        const float h = (float)wd[i];
        wf[i] = make_float2(h, (float)(wd[i] - (double)h));
    }
    err = upload(&p->d_zu, p->zu);
    if (!err) err = upload(&p->d_zd, p->zd);
    if (!err) err = upload(&p->d_k, p->k);
    if (!err) err = upload(&p->d_l, p->l);
    if (!err) err = upload(&p->d_w, wd);
    if (!err) err = upload(&p->d_wf, wf);
    if (!err) err = upload(&p->d_el_off, p->el_off);
    if (err) {
        free_plan(p);
        return err;
    }
    *out = p;
    return WICK_OK;
}

}  // namespace
}  // namespace wick

extern "C" {

int wick_det_reduce(const wick_quark_operator *sink, const wick_quark_operator *source, uint64_t seed, int trials,
                    wick_det_plan **out) {
    if (!sink || !source) return WICK_EINVAL;
    return reduce_matrix(&sink, 1, &source, 1, seed, trials, out);
}

int wick_det_reduce_matrix(const wick_quark_operator *ops, int n_ops, uint64_t seed, int trials, wick_det_plan **out) {
    if (!ops || n_ops < 1 || n_ops * n_ops > kMaxEl) return WICK_EINVAL;
    std::vector<const wick_quark_operator *> v(n_ops);
    for (int i = 0; i < n_ops; ++i) v[i] = &ops[i];
    return reduce_matrix(v.data(), n_ops, v.data(), n_ops, seed, trials, out);
}

int wick_det_stats(const wick_det_plan *p, int64_t *out) {
    if (!p || !out) return WICK_EINVAL;
    out[0] = p->n_snk;
    out[1] = p->n_src;
    out[2] = p->n_zu;
    out[3] = p->n_zd;
    out[4] = p->n_theta;
    out[5] = p->n_u * 8 + p->n_d;
    out[6] = p->n_el;
    return WICK_OK;
}

int wick_det_element_offsets(const wick_det_plan *p, int64_t *off) {
    if (!p || !off) return WICK_EINVAL;
    std::copy(p->el_off.begin(), p->el_off.end(), off);
    return WICK_OK;
}

int wick_det_copy(const wick_det_plan *p, int32_t *k, int32_t *l, int64_t *w, int8_t *zu_rows, int8_t *zu_cols,
                  int8_t *zd_rows, int8_t *zd_cols) {
    if (!p) return WICK_EINVAL;
    if (k) std::copy(p->k.begin(), p->k.end(), k);
    if (l) std::copy(p->l.begin(), p->l.end(), l);
    if (w) std::copy(p->w.begin(), p->w.end(), w);
    for (int64_t i = 0; i < p->n_zu; ++i)
        for (int q = 0; q < p->n_u; ++q) {
            if (zu_rows) zu_rows[i * p->n_u + q] = p->zu[(i * 2) * p->n_u + q];
            if (zu_cols) zu_cols[i * p->n_u + q] = p->zu[(i * 2 + 1) * p->n_u + q];
        }
    for (int64_t i = 0; i < p->n_zd; ++i)
        for (int q = 0; q < p->n_d; ++q) {
            if (zd_rows) zd_rows[i * p->n_d + q] = p->zd[(i * 2) * p->n_d + q];
            if (zd_cols) zd_cols[i * p->n_d + q] = p->zd[(i * 2 + 1) * p->n_d + q];
        }
    return WICK_OK;
}

}  // extern "C"

namespace wick {
namespace {

bool props_match(const wick_prop *a, const wick_prop *b) {
    return a && b && a->data && b->data && a->L == b->L && a->T == b->T && a->n_src == b->n_src &&
           a->dtype == b->dtype;
}

int det_contract(const wick_prop *Su, const wick_prop *Sd, const wick_prop *Sig, int seq_flavour,
                 const wick_det_plan *plan, double scale, int precision, void *C_out, wick_stream_t stream) {
    if (!plan || !C_out || (precision != WICK_FP64 && precision != WICK_MIXED) || !props_match(Su, Sd))
        return WICK_EINVAL;
    // double-FP32 derivatives exist for the cofactor form only
    if (precision == WICK_MIXED && seq_flavour >= 0 && (seq_flavour == 0 ? plan->n_u : plan->n_d) > 3)
        return WICK_EINVAL;
    if (seq_flavour >= 0 && !props_match(Su, Sig)) return WICK_EINVAL;
    if (Su->L < 1 || Su->T < 1 || Su->n_src < 1 || (Su->dtype != WICK_C64 && Su->dtype != WICK_C128))
        return WICK_EINVAL;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != plan->device) return WICK_EINVAL;
    const int64_t V = (int64_t)Su->L * Su->L * Su->L, n_slices = (int64_t)Su->n_src * Su->T;
    if (V > (1 << 24) || n_slices > (1 << 24)) return WICK_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (plan->n_theta == 0) {
        WICK_CUDA_TRY(cudaMemsetAsync(C_out, 0, sizeof(double2) * n_slices * plan->n_el, st));
        return WICK_OK;
    }
    int n_sm = 0, occ = 0;
    WICK_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    const bool one = plan->n_el == 1;
    const bool c64 = Su->dtype == WICK_C64;
    const bool mixed = precision == WICK_MIXED;
    // the 2 x 2 minor tables always; flavours with 5 or 6 quarks also the 3 x 3 ones (except the one
    // carrying a three-point current)
    const int m3_mask = (plan->n_u >= 5 && seq_flavour != 0 ? 1 : 0) | (plan->n_d >= 5 && seq_flavour != 1 ? 2 : 0);
    const int n_m3 = (m3_mask & 1) + (m3_mask >> 1 & 1);
    const size_t dyn = sizeof(double2) * 2 * kPairs * kPairs;
    using KF = void (*)(const DetArgs, const float2 *, const float2 *, const float2 *, int, int, int, int,
                        double2 *, double2 *);
    using KD = void (*)(const DetArgs, const double2 *, const double2 *, const double2 *, int, int, int, int,
                        double2 *, double2 *);
    KF kf = mixed ? (one ? det_eval_kernel<float2, cdf, 1> : det_eval_kernel<float2, cdf, kMaxEl>)
                  : (one ? det_eval_kernel<float2, double2, 1> : det_eval_kernel<float2, double2, kMaxEl>);
    KD kd = mixed ? (one ? det_eval_kernel<double2, cdf, 1> : det_eval_kernel<double2, cdf, kMaxEl>)
                  : (one ? det_eval_kernel<double2, double2, 1> : det_eval_kernel<double2, double2, kMaxEl>);
    const void *kern = c64 ? (const void *)kf : (const void *)kd;
    WICK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    const int threads = mixed && one ? det_threads<cdf, 1>() : det_threads<double2, 1>();
    WICK_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, dyn));
    // sites per work item: 32, halved while that leaves fewer than two items per resident CTA
    const int64_t capacity = (int64_t)n_sm * std::max(occ, 1);
    int chunk_sites = kDetChunk;
    while (chunk_sites > 1 && n_slices * ((V + chunk_sites - 1) / chunk_sites) < 2 * capacity) chunk_sites /= 2;
    const int n_chunks = (int)((V + chunk_sites - 1) / chunk_sites);
    const int64_t items = n_slices * n_chunks;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)n_sm * std::max(occ, 1)));
    const size_t scratch_bytes =
        sizeof(double2) * (size_t)grid * (size_t)(plan->n_zu + plan->n_zd + (int64_t)n_m3 * kTriples * kTriples);
    const size_t part_bytes = sizeof(double2) * (size_t)items * plan->n_el;
    int err = WICK_OK;
    unsigned char *ws = (unsigned char *)workspace(2, scratch_bytes + part_bytes + 256, &err);
    if (err) return err;
    double2 *scratch = (double2 *)ws;
    double2 *partials = (double2 *)(ws + (scratch_bytes + 255) / 256 * 256);
    DetArgs a{plan->n_u, plan->n_d, plan->n_el, seq_flavour, m3_mask, plan->n_zu, plan->n_zd, plan->d_zu,
              plan->d_zd, plan->d_k, plan->d_l, plan->d_w, plan->d_wf, plan->d_el_off};
    const unsigned g = (unsigned)grid;
    const int iv = (int)V, is = (int)n_slices;
    if (c64) {
        const float2 *u = (const float2 *)Su->data, *d = (const float2 *)Sd->data;
        const float2 *q = seq_flavour >= 0 ? (const float2 *)Sig->data : u;
        kf<<<g, threads, dyn, st>>>(a, u, d, q, iv, is, n_chunks, chunk_sites, scratch, partials);
    } else {
        const double2 *u = (const double2 *)Su->data, *d = (const double2 *)Sd->data;
        const double2 *q = seq_flavour >= 0 ? (const double2 *)Sig->data : u;
        kd<<<g, threads, dyn, st>>>(a, u, d, q, iv, is, n_chunks, chunk_sites, scratch, partials);
    }
    WICK_CUDA_TRY(cudaGetLastError());
    const int64_t n_out = n_slices * plan->n_el;
    det_finish_kernel<<<(unsigned)((n_out + 127) / 128), 128, 0, st>>>(partials, (int)n_slices, n_chunks,
                                                                       plan->n_el, scale, (double2 *)C_out);
    WICK_CUDA_TRY(cudaGetLastError());
    return WICK_OK;
}

}  // namespace
}  // namespace wick

extern "C" {

int wick_det_contract(const wick_prop *Su, const wick_prop *Sd, const wick_det_plan *plan, double scale,
                      int precision, void *C_out, wick_stream_t stream) {
    return det_contract(Su, Sd, nullptr, -1, plan, scale, precision, C_out, stream);
}

int wick_det_contract_3pt(const wick_prop *Su, const wick_prop *Sd, const wick_prop *Sig, int flavour,
                          const wick_det_plan *plan, double scale, int precision, void *C_out, wick_stream_t stream) {
    if (flavour != WICK_U && flavour != WICK_D) return WICK_EINVAL;
    return det_contract(Su, Sd, Sig, flavour, plan, scale, precision, C_out, stream);
}

void wick_det_free(wick_det_plan *plan) { free_plan(plan); }

}  // extern "C"
