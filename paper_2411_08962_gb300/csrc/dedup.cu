// Randomised minimal-set search for the block correlator (Sec. III.B,
// Theorem 1 and "Implementation Procedures" of App. C).
//
// Pipeline (one stream, synchronised once at the end):
//   1. modp_blocks_kernel  block values R[trial][id] of the antisymmetric blocks
//                          (Eq. 2.4) at random integer propagators on `sites`
//                          sites, exactly modulo p = 2^61 - 1.
//   2. enum_hash_kernel    every raw Wick term j: decode (sink, source multiset,
//                          tau_u, tau_d), hash h_r = prod_k R[r][id_k] mod p, canonical
//                          sign, then one insertion per group of equal keys in a
//                          warp (match + reduce) into an open-addressing table
//                          holding (key, sum of eps*c, smallest j).
//   3. compact_kernel      classes with non-zero weight -> (rep, W) list.
//   4. radix sort          stable LSD sort of the list by representative j.
//   5. finalize_kernel     decode each representative: block ids, its sign
//                          eps_rep, weight W * eps_rep / 2^A.
// Every wait on another thread (a slot being claimed) is bounded; running out
// sets WICK_ETIMEOUT in the status word and drops the insertion.
#include <vector>

#include "common.cuh"

namespace wick {

namespace {

constexpr uint64_t P61 = (1ull << 61) - 1;
constexpr uint64_t EMPTY = ~0ull;
constexpr uint64_t BUSY = 1ull << 62;
constexpr int kSpinLimit = 1 << 20;

// x = a * b (a, b < 2^61) reduced with 2^61 == 1 (mod p)
__device__ __forceinline__ uint64_t mulmod(uint64_t a, uint64_t b) {
    const uint64_t lo = a * b, hi = __umul64hi(a, b);
    uint64_t s = (lo & P61) + ((hi << 3) | (lo >> 61));
    s = (s & P61) + (s >> 61);
    return s >= P61 ? s - P61 : s;
}
__device__ __forceinline__ uint64_t addmod(uint64_t a, uint64_t b) {
    const uint64_t s = a + b;
    return s >= P61 ? s - P61 : s;
}
__device__ __forceinline__ uint64_t submod(uint64_t a, uint64_t b) { return a >= b ? a - b : a + P61 - b; }
__device__ __forceinline__ uint64_t from_int(int64_t v) {
    if (v >= 0) return (uint64_t)v % P61;
    return submod(0, (uint64_t)(-v) % P61);
}

// SplitMix64 (Steele, Lea, Flood 2014): output function and counter use.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t rand_modp(uint64_t key, uint64_t i) {
    const uint64_t r = mix64(key + (i + 1) * 0x9E3779B97F4A7C15ull) >> 3;
    return r == P61 ? 0 : r;
}

// ---------------------------------------------------------------------------
// 1. block values mod p (antisymmetric in the like-flavour source pair)
// ---------------------------------------------------------------------------
__device__ uint64_t modp_P(const BlockPlan &plan, uint64_t key_u, uint64_t key_d, int sites, int os,
                           int c1, int c2, int c3) {
    const int op = os / plan.n_spin, f1 = plan.f1[op];
    const uint64_t k1 = f1 == 0 ? key_u : key_d, k2 = f1 == 0 ? key_d : key_u;
    uint64_t acc = 0;
    for (int v = 0; v < sites; ++v) {
        const uint64_t b1 = mix64(k1 + 0x51ull * (uint64_t)(v + 1)), b2 = mix64(k2 + 0x51ull * (uint64_t)(v + 1));
        for (int t = plan.os_off[os]; t < plan.os_off[os + 1]; ++t) {
            const int r1 = plan.rows[f1][plan.os_r1[t]];
            const int l = plan.os_x[t];
            uint64_t x = 0;
            for (int q = plan.x_off[l]; q < plan.x_off[l + 1]; ++q) {
                const int r2 = plan.rows[f1][plan.xt_r2[q]], r3 = plan.rows[1 - f1][plan.xt_r3[q]];
                uint64_t p = mulmod(rand_modp(b1, (uint64_t)(r2 * 12 + c2)), rand_modp(b2, (uint64_t)(r3 * 12 + c3)));
                p = mulmod(p, from_int((int64_t)plan.xt_w[q]));
                x = addmod(x, p);
            }
            acc = addmod(acc, mulmod(rand_modp(b1, (uint64_t)(r1 * 12 + c1)), x));
        }
    }
    return acc;
}

__global__ void modp_blocks_kernel(const __grid_constant__ BlockPlan plan, uint64_t seed, int trials, int sites,
                                   uint64_t *__restrict__ R, int n_blk) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= trials * n_blk) return;
    const int r = i / n_blk, id = i - r * n_blk;
    const int nc = plan.n_chi, nc3 = nc * nc * nc;
    const int os = id / nc3, i1 = (id / (nc * nc)) % nc, i2 = (id / nc) % nc, i3 = id % nc;
    const uint64_t key_u = mix64(seed ^ mix64(0xA5A5ull + 2 * (uint64_t)r));
    const uint64_t key_d = mix64(seed ^ mix64(0xA5A5ull + 2 * (uint64_t)r + 1));
    const int c1 = plan.chi[i1], c2 = plan.chi[i2], c3 = plan.chi[i3];
    R[i] = submod(modp_P(plan, key_u, key_d, sites, os, c1, c2, c3), modp_P(plan, key_u, key_d, sites, os, c2, c1, c3));
}

// ---------------------------------------------------------------------------
// raw-term decoding shared by the enumeration and the finalisation
// ---------------------------------------------------------------------------
struct TermTables {
    const int8_t *sink_type, *sink_spin;  // [n_sink][A]
    const int64_t *sink_w;                // [n_sink]
    const int8_t *sink_flav, *sink_ord;   // [n_sink][nq]
    const int8_t *sink_eta;               // [n_sink]
    const int8_t *Mu, *Md;                // [n_M][nu], [n_M][nd]: sorted layout positions
    const int64_t *CM;                    // [n_M] antisymmetrised source weight
    const uint8_t *pu, *pd;               // permutation tables [n!][n]
    const int8_t *su, *sd;                // their signs
    const uint64_t *R;                    // [trials][n_blk]
};

// Block ids of raw term (i, M, ru, rd) and its coefficient: the sink quark of
// flavour-ordinal q takes the tau(q)-th entry of the multiset's sorted list.
__device__ __forceinline__ int64_t term_ids(const EnumPlan &ep, const TermTables &tt, int i, int M, int64_t ru,
                                            int64_t rd, int *ids) {
    const uint8_t *pu = tt.pu + ru * ep.nu, *pd = tt.pd + rd * ep.nd;
    const int nc = ep.n_chi;
    for (int k = 0; k < ep.A; ++k) {
        int ix[3];
#pragma unroll
        for (int sl = 0; sl < 3; ++sl) {
            const int q = 3 * k + sl;
            const int f = tt.sink_flav[i * ep.nq + q], ord = tt.sink_ord[i * ep.nq + q];
            ix[sl] = f == 0 ? tt.Mu[M * ep.nu + pu[ord]] : tt.Md[M * ep.nd + pd[ord]];
        }
        const int o = tt.sink_type[i * ep.A + k], s = tt.sink_spin[i * ep.A + k];
        ids[k] = (((o * ep.n_spin + s) * nc + ix[0]) * nc + ix[1]) * nc + ix[2];
    }
    return tt.sink_w[i] * tt.CM[M] * tt.su[ru] * tt.sd[rd] * tt.sink_eta[i];
}

// Hash of a monomial; returns false for a zero key.  *eps = canonical sign.
__device__ __forceinline__ bool term_key(const EnumPlan &ep, const TermTables &tt, int trials, const int *ids,
                                         uint64_t *h0, uint64_t *h1, int *eps) {
    uint64_t h[2] = {1, 1};
    for (int r = 0; r < trials; ++r)
        for (int k = 0; k < ep.A; ++k) h[r] = mulmod(h[r], __ldg(tt.R + (size_t)r * ep.n_blk + ids[k]));
    if (trials == 1) h[1] = 0;
    const int first = h[0] != 0 ? 0 : (h[1] != 0 ? 1 : -1);
    if (first < 0) return false;
    *eps = 1;
    if (h[first] > (P61 - 1) / 2) {
        *eps = -1;
        h[0] = h[0] ? P61 - h[0] : 0;
        h[1] = h[1] ? P61 - h[1] : 0;
    }
    *h0 = h[0];
    *h1 = h[1];
    return true;
}

struct HashTable {
    uint64_t *k0, *k1;
    unsigned long long *W, *rep;
    uint64_t mask;
    unsigned long long *n_keys;  // keys inserted so far
    uint64_t max_keys;           // above this the table counts as full
};

__device__ __forceinline__ uint64_t load_volatile(const uint64_t *p) { return *(volatile const uint64_t *)p; }

// Find or claim the slot of (h0, h1); -1 on a full table or a wait that ran out.
__device__ int64_t table_slot(const HashTable &ht, uint64_t h0, uint64_t h1, int *status, int spin_limit = kSpinLimit) {
    uint64_t slot = mix64(h0 * 0x9E3779B97F4A7C15ull ^ h1) & ht.mask;
    for (uint64_t probe = 0; probe <= ht.mask; ++probe) {
        uint64_t k = load_volatile(ht.k0 + slot);
        if (k == EMPTY) {
            const unsigned long long prev =
                atomicCAS((unsigned long long *)(ht.k0 + slot), (unsigned long long)EMPTY, (unsigned long long)(h0 | BUSY));
            if (prev == EMPTY) {
                ht.k1[slot] = h1;
                __threadfence();
                atomicExch((unsigned long long *)(ht.k0 + slot), (unsigned long long)h0);
                const unsigned long long n = atomicAdd(ht.n_keys, 1ull);
                if (n + 1 > ht.max_keys) atomicCAS(status, 0, WICK_ECAPACITY);
                return (int64_t)slot;
            }
            k = prev;
        }
        int spins = 0;
        while (k & BUSY) {
            if (++spins > spin_limit) {
                atomicCAS(status, 0, WICK_ETIMEOUT);
                return -1;
            }
            k = load_volatile(ht.k0 + slot);
        }
        if (k == h0) {
            __threadfence();
            if (load_volatile(ht.k1 + slot) == h1) return (int64_t)slot;
        }
        slot = (slot + 1) & ht.mask;
    }
    atomicCAS(status, 0, WICK_ECAPACITY);
    return -1;
}

// ---------------------------------------------------------------------------
// 2. enumerate, hash and merge.  One warp task = one row (i, m, ru) and 32
// consecutive d-permutation ranks; lanes with equal keys are merged in the
// warp before touching the table.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
enum_hash_kernel(const __grid_constant__ EnumPlan ep, const TermTables tt, int trials, HashTable ht,
                 unsigned long long *n_zero, int *status, uint64_t n_tasks, uint32_t rd_tiles) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t task = warp0; task < n_tasks; task += n_warps) {
        int st = lane == 0 ? *(volatile int *)status : 0;
        if (__shfl_sync(0xffffffffu, st, 0) != 0) return;  // warp-uniform early exit
        const uint64_t row = task / rd_tiles;
        const int64_t rd = (int64_t)(task - row * rd_tiles) * 32 + lane;
        const int64_t ru = (int64_t)(row % (uint64_t)ep.fu);
        const uint64_t im = row / (uint64_t)ep.fu;
        const int m = (int)(im % (uint64_t)ep.n_M), i = (int)(im / (uint64_t)ep.n_M);
        const bool valid = rd < ep.fd;
        int ids[kMaxA];
        uint64_t h0 = 0, h1 = 0;
        int eps = 1;
        int64_t c = 0;
        bool nz = false;
        if (valid) {
            c = term_ids(ep, tt, i, m, ru, rd, ids);
            nz = term_key(ep, tt, trials, ids, &h0, &h1, &eps);
        }
        const unsigned zero_mask = __ballot_sync(0xffffffffu, valid && !nz);
        if (lane == 0 && zero_mask) atomicAdd(n_zero, (unsigned long long)__popc(zero_mask));
        const unsigned act = __ballot_sync(0xffffffffu, nz);
        if (!nz) continue;
        const unsigned grp = __match_any_sync(act, h0) & __match_any_sync(act, h1);
        const int contrib = (int)(eps * c);
        const int sum = (int)__reduce_add_sync(grp, (unsigned)contrib);
        if (lane == __ffs(grp) - 1) {  // the group leader holds the group's smallest j
            const int64_t slot = table_slot(ht, h0, h1, status);
            if (slot >= 0) {
                if (sum != 0) atomicAdd(ht.W + slot, (unsigned long long)(long long)sum);
                const uint64_t j = row * (uint64_t)ep.fd + (uint64_t)rd;
                atomicMin(ht.rep + slot, (unsigned long long)j);
            }
        }
    }
}

// The wait of table_slot on a slot that another thread has claimed (BUSY) but not yet published, on a
// one-slot table whose slot is claimed and never published: the wait gives up after spin_limit polls.
__global__ void hash_wait_selftest_kernel(HashTable ht, int spin_limit, int *status) {
    (void)table_slot(ht, 1ull, 2ull, status, spin_limit);
}

// ---------------------------------------------------------------------------
// 3. compaction of the kept classes
// ---------------------------------------------------------------------------
__global__ void compact_kernel(HashTable ht, unsigned long long *n_out, uint64_t *out_rep, int64_t *out_W,
                               unsigned long long *n_keys_seen) {
    const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s > ht.mask) return;
    if (ht.k0[s] == EMPTY) return;
    atomicAdd(n_keys_seen, 1ull);
    const long long W = (long long)ht.W[s];
    if (W == 0) return;
    const unsigned long long p = atomicAdd(n_out, 1ull);
    out_rep[p] = ht.rep[s];
    out_W[p] = W;
}

// ---------------------------------------------------------------------------
// 4. stable LSD radix sort of (key, value) pairs, 4-bit digits
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256, kSortItems = 8, kSortTile = kSortThreads * kSortItems;

__global__ void radix_hist_kernel(const uint64_t *__restrict__ keys, int64_t n, int shift,
                                  unsigned *__restrict__ hist, int n_tiles) {
    __shared__ unsigned h[16];
    if (threadIdx.x < 16) h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int q = threadIdx.x; q < kSortTile; q += kSortThreads) {
        const int64_t e = base + q;
        if (e < n) atomicAdd(&h[(keys[e] >> shift) & 15], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 16) hist[threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of hist[16 * n_tiles] (digit-major), one CTA
__global__ void radix_scan_kernel(unsigned *__restrict__ hist, int n) {
    __shared__ unsigned part[1024];
    const int per = (n + 1023) / 1024;
    const int b = threadIdx.x * per, e = min(n, b + per);
    unsigned s = 0;
    for (int i = b; i < e; ++i) s += hist[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const unsigned v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned run = threadIdx.x ? part[threadIdx.x - 1] : 0;
    for (int i = b; i < e; ++i) {
        const unsigned v = hist[i];
        hist[i] = run;
        run += v;
    }
}

__global__ void radix_scatter_kernel(const uint64_t *__restrict__ kin, const int64_t *__restrict__ vin,
                                     uint64_t *__restrict__ kout, int64_t *__restrict__ vout, int64_t n, int shift,
                                     const unsigned *__restrict__ offs, int n_tiles) {
    __shared__ unsigned cnt[16][kSortThreads + 1];
    const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)threadIdx.x * kSortItems;
    unsigned local[16];
#pragma unroll
    for (int d = 0; d < 16; ++d) local[d] = 0;
    for (int q = 0; q < kSortItems; ++q) {
        const int64_t e = base + q;
        if (e < n) local[(kin[e] >> shift) & 15]++;
    }
#pragma unroll
    for (int d = 0; d < 16; ++d) cnt[d][threadIdx.x] = local[d];
    __syncthreads();
    if (threadIdx.x < 16) {  // exclusive scan over threads, per digit (thread order = element order)
        unsigned run = 0;
        for (int t = 0; t < kSortThreads; ++t) {
            const unsigned v = cnt[threadIdx.x][t];
            cnt[threadIdx.x][t] = run;
            run += v;
        }
    }
    __syncthreads();
#pragma unroll
    for (int d = 0; d < 16; ++d) local[d] = offs[d * n_tiles + blockIdx.x] + cnt[d][threadIdx.x];
    for (int q = 0; q < kSortItems; ++q) {
        const int64_t e = base + q;
        if (e < n) {
            const int d = (int)((kin[e] >> shift) & 15);
            const unsigned p = local[d]++;
            kout[p] = kin[e];
            vout[p] = vin[e];
        }
    }
}

// ---------------------------------------------------------------------------
// 5. finalisation
// ---------------------------------------------------------------------------
__global__ void finalize_kernel(const __grid_constant__ EnumPlan ep, const TermTables tt, int trials,
                                const uint64_t *__restrict__ rep, const int64_t *__restrict__ W, int64_t U,
                                uint16_t *__restrict__ ids_out, int64_t *__restrict__ w_out,
                                int64_t *__restrict__ rep_out, int *status) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= U) return;
    const uint64_t j = rep[u];
    const uint64_t row = j / (uint64_t)ep.fd;
    const int64_t rd = (int64_t)(j - row * (uint64_t)ep.fd);
    const int64_t ru = (int64_t)(row % (uint64_t)ep.fu);
    const uint64_t im = row / (uint64_t)ep.fu;
    const int m = (int)(im % (uint64_t)ep.n_M), i = (int)(im / (uint64_t)ep.n_M);
    int ids[kMaxA];
    term_ids(ep, tt, i, m, ru, rd, ids);
    uint64_t h0, h1;
    int eps = 1;
    if (!term_key(ep, tt, trials, ids, &h0, &h1, &eps)) atomicCAS(status, 0, WICK_EOVERFLOW);
    const int64_t two_a = (int64_t)1 << ep.A;
    const int64_t w = W[u] * eps;
    if (w % two_a != 0) atomicCAS(status, 0, WICK_EOVERFLOW);
    w_out[u] = w / two_a;
    rep_out[u] = (int64_t)j;
    for (int k = 0; k < ep.A; ++k) ids_out[u * ep.A + k] = (uint16_t)ids[k];
}

template <typename T>
struct DevBuf {
    T *p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
    int alloc(size_t n) {
        if (dev_malloc((void **)&p, sizeof(T) * (n ? n : 1)) != WICK_OK) { (void)cudaGetLastError(); p = nullptr; return WICK_ENOMEM; }
        return WICK_OK;
    }
    int upload(const T *h, size_t n, cudaStream_t s) {
        int e = alloc(n);
        if (e) return e;
        return cudaMemcpyAsync(p, h, sizeof(T) * n, cudaMemcpyHostToDevice, s) == cudaSuccess ? WICK_OK : WICK_ECUDA;
    }
};

uint64_t next_pow2(uint64_t v) { uint64_t p = 1; while (p < v) p <<= 1; return p; }

}  // namespace

int run_reduce(const EnumPlan &ep, const BlockPlan &bp, const wick_nucleus *nuc, const int8_t *Mu,
               const int8_t *Md, const int64_t *CM, const int8_t *sink_flav, const int8_t *sink_ord,
               const int8_t *sink_eta, uint64_t seed, int trials, int sites, ReduceResult *out,
               cudaStream_t stream) {
    int err = WICK_OK;
    int *status = status_word(&err);
    if (err) return err;
    // permutation tables, lexicographic order, signs = parity of the Lehmer digit sum
    auto perm_table = [](int n, std::vector<uint8_t> &P, std::vector<int8_t> &S) {
        int64_t f = 1;
        for (int i = 2; i <= n; ++i) f *= i;
        P.assign((size_t)f * (n ? n : 1), 0);
        S.assign((size_t)f, 1);
        for (int64_t r = 0; r < f; ++r) {
            int used[32] = {0}, inv = 0;
            int64_t rr = r;
            for (int i = 0; i < n; ++i) {
                int64_t fi = 1;
                for (int q = 2; q <= n - 1 - i; ++q) fi *= q;
                const int d = (int)(rr / fi);
                rr %= fi;
                inv += d;
                for (int v = 0, c = -1; v < n; ++v)
                    if (!used[v] && ++c == d) { P[(size_t)r * n + i] = (uint8_t)v; used[v] = 1; break; }
            }
            S[(size_t)r] = (inv & 1) ? -1 : 1;
        }
    };
    std::vector<uint8_t> hpu, hpd;
    std::vector<int8_t> hsu, hsd;
    perm_table(ep.nu, hpu, hsu);
    perm_table(ep.nd, hpd, hsd);

    DevBuf<int8_t> d_type, d_spin, d_flav, d_ord, d_eta, d_mu, d_md, d_su, d_sd;
    DevBuf<int64_t> d_sw, d_cw;
    DevBuf<uint8_t> d_pu, d_pd;
    DevBuf<uint64_t> d_R;
    const size_t nsA = (size_t)ep.n_sink * ep.A, nsq = (size_t)ep.n_sink * ep.nq;
    if ((err = d_type.upload(nuc->sink_type, nsA, stream)) || (err = d_spin.upload(nuc->sink_spin, nsA, stream)) ||
        (err = d_sw.upload(nuc->sink_w, ep.n_sink, stream)) || (err = d_flav.upload(sink_flav, nsq, stream)) ||
        (err = d_ord.upload(sink_ord, nsq, stream)) || (err = d_eta.upload(sink_eta, ep.n_sink, stream)) ||
        (err = d_mu.upload(Mu, (size_t)ep.n_M * ep.nu, stream)) ||
        (err = d_md.upload(Md, (size_t)ep.n_M * ep.nd, stream)) ||
        (err = d_cw.upload(CM, ep.n_M, stream)) || (err = d_pu.upload(hpu.data(), hpu.size(), stream)) ||
        (err = d_pd.upload(hpd.data(), hpd.size(), stream)) || (err = d_su.upload(hsu.data(), hsu.size(), stream)) ||
        (err = d_sd.upload(hsd.data(), hsd.size(), stream)) || (err = d_R.alloc((size_t)2 * ep.n_blk)))
        return err;

    modp_blocks_kernel<<<(trials * ep.n_blk + 127) / 128, 128, 0, stream>>>(bp, seed, trials, sites, d_R.p, ep.n_blk);
    WICK_CUDA_TRY(cudaGetLastError());

    TermTables tt{d_type.p, d_spin.p, d_sw.p, d_flav.p, d_ord.p, d_eta.p, d_mu.p, d_md.p, d_cw.p,
                  d_pu.p, d_pd.p, d_su.p, d_sd.p, d_R.p};

    const uint32_t rd_tiles = (uint32_t)((ep.fd + 31) / 32);
    const uint64_t n_rows = (uint64_t)ep.n_sink * ep.n_M * (uint64_t)ep.fu;
    const uint64_t n_tasks = n_rows * rd_tiles;
    // table size: start from an estimate and double while it overflows
    const uint64_t upper = (uint64_t)(ep.n_raw >> ep.A) + 1024;
    const wick_tuning tune = current_tuning();
    uint64_t cap = next_pow2(upper < (1ull << 20) ? 2 * upper : (1ull << 21));
    const uint64_t cap_max = 1ull << (tune.hash_log2_max ? tune.hash_log2_max : 28);
    if (tune.hash_log2_start) cap = 1ull << tune.hash_log2_start;
    if (cap > cap_max) cap = cap_max;
    DevBuf<unsigned long long> d_cnt;  // [0] n_keys, [1] n_zero, [2] n_out, [3] n_keys_seen
    if ((err = d_cnt.alloc(4))) return err;
    for (;;) {
        DevBuf<uint64_t> k0, k1;
        DevBuf<unsigned long long> W, rep;
        if ((err = k0.alloc(cap)) || (err = k1.alloc(cap)) || (err = W.alloc(cap)) || (err = rep.alloc(cap)))
            return err;
        WICK_CUDA_TRY(cudaMemsetAsync(k0.p, 0xFF, sizeof(uint64_t) * cap, stream));
        WICK_CUDA_TRY(cudaMemsetAsync(W.p, 0, sizeof(uint64_t) * cap, stream));
        WICK_CUDA_TRY(cudaMemsetAsync(rep.p, 0xFF, sizeof(uint64_t) * cap, stream));
        WICK_CUDA_TRY(cudaMemsetAsync(d_cnt.p, 0, sizeof(unsigned long long) * 4, stream));
        WICK_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), stream));
        HashTable ht{k0.p, k1.p, W.p, rep.p, cap - 1, d_cnt.p, (cap / 4) * 3};
        int dev = 0, n_sm = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        uint64_t blocks = (n_tasks * 32 + 255) / 256;
        const uint64_t max_blocks = (uint64_t)n_sm * 8;
        if (blocks > max_blocks) blocks = max_blocks;
        if (blocks == 0) blocks = 1;  // no raw terms: the kernel exits at once
        enum_hash_kernel<<<(unsigned)blocks, 256, 0, stream>>>(ep, tt, trials, ht, d_cnt.p + 1, status, n_tasks,
                                                              rd_tiles);
        WICK_CUDA_TRY(cudaGetLastError());
        int h_status = 0;
        WICK_CUDA_TRY(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, stream));
        WICK_CUDA_TRY(cudaStreamSynchronize(stream));
        if (h_status == WICK_ECAPACITY && cap < cap_max) {
            cap <<= 1;
            continue;
        }
        if (h_status) return h_status;

        DevBuf<uint64_t> rk, rk2;
        DevBuf<int64_t> rv, rv2;
        if ((err = rk.alloc(cap)) || (err = rv.alloc(cap))) return err;
        compact_kernel<<<(unsigned)((cap + 255) / 256), 256, 0, stream>>>(ht, d_cnt.p + 2, rk.p, rv.p, d_cnt.p + 3);
        WICK_CUDA_TRY(cudaGetLastError());
        unsigned long long h_cnt[4];
        WICK_CUDA_TRY(cudaMemcpyAsync(h_cnt, d_cnt.p, sizeof(h_cnt), cudaMemcpyDeviceToHost, stream));
        WICK_CUDA_TRY(cudaStreamSynchronize(stream));
        const int64_t U = (int64_t)h_cnt[2];
        out->n_zero = (int64_t)h_cnt[1];
        out->n_keys = (int64_t)h_cnt[3];
        out->U = U;
        // sort by representative (bits of n_raw only)
        if (U > 1) {
            if ((err = rk2.alloc(U)) || (err = rv2.alloc(U))) return err;
            const int n_tiles = (int)((U + kSortTile - 1) / kSortTile);
            DevBuf<unsigned> hist;
            if ((err = hist.alloc((size_t)16 * n_tiles))) return err;
            int bits = 1;
            while (bits < 63 && (1ull << bits) < (uint64_t)ep.n_raw) ++bits;
            uint64_t *ka = rk.p, *kb = rk2.p;
            int64_t *va = rv.p, *vb = rv2.p;
            for (int shift = 0; shift < bits; shift += 4) {
                radix_hist_kernel<<<n_tiles, kSortThreads, 0, stream>>>(ka, U, shift, hist.p, n_tiles);
                radix_scan_kernel<<<1, 1024, 0, stream>>>(hist.p, 16 * n_tiles);
                radix_scatter_kernel<<<n_tiles, kSortThreads, 0, stream>>>(ka, va, kb, vb, U, shift, hist.p, n_tiles);
                WICK_CUDA_TRY(cudaGetLastError());
                std::swap(ka, kb);
                std::swap(va, vb);
            }
            if (ka != rk.p) {
                WICK_CUDA_TRY(cudaMemcpyAsync(rk.p, ka, sizeof(uint64_t) * U, cudaMemcpyDeviceToDevice, stream));
                WICK_CUDA_TRY(cudaMemcpyAsync(rv.p, va, sizeof(int64_t) * U, cudaMemcpyDeviceToDevice, stream));
            }
        }
        uint16_t *ids = nullptr;
        int64_t *w = nullptr, *reps = nullptr;
        if (dev_malloc((void **)&ids, sizeof(uint16_t) * (size_t)(U ? U : 1) * ep.A) != WICK_OK ||
            dev_malloc((void **)&w, sizeof(int64_t) * (size_t)(U ? U : 1)) != WICK_OK ||
            dev_malloc((void **)&reps, sizeof(int64_t) * (size_t)(U ? U : 1)) != WICK_OK) {
            (void)cudaGetLastError();
            cudaFree(ids); cudaFree(w); cudaFree(reps);
            return WICK_ENOMEM;
        }
        if (U > 0)
            finalize_kernel<<<(unsigned)((U + 255) / 256), 256, 0, stream>>>(ep, tt, trials, rk.p, rv.p, U, ids, w,
                                                                           reps, status);
        WICK_CUDA_TRY(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, stream));
        WICK_CUDA_TRY(cudaStreamSynchronize(stream));
        if (h_status) {
            cudaFree(ids); cudaFree(w); cudaFree(reps);
            return h_status;
        }
        out->d_ids = ids;
        out->d_w = w;
        out->d_rep = reps;
        return WICK_OK;
    }
    return WICK_ENOMEM;
}

namespace {
// keys of given reduced terms under the identity-testing evaluation of run_reduce (same R tables)
__global__ void key_kernel(const uint64_t *__restrict__ R, int n_blk, int trials, const uint16_t *__restrict__ ids,
                           int64_t U, int A, uint64_t *__restrict__ keys, int8_t *__restrict__ eps) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= U) return;
    EnumPlan ep;
    ep.A = A;
    ep.n_blk = n_blk;
    TermTables tt;
    tt.R = R;
    int id[kMaxA];
    for (int k = 0; k < A; ++k) id[k] = ids[u * A + k];
    uint64_t h0 = 0, h1 = 0;
    int e = 0;
    if (!term_key(ep, tt, trials, id, &h0, &h1, &e)) e = 0;
    keys[2 * u] = h0;
    keys[2 * u + 1] = h1;
    eps[u] = (int8_t)e;
}
}  // namespace

int term_keys(const BlockPlan &bp, int n_blk, const uint16_t *ids, int64_t U, int A, uint64_t seed, int trials,
              int sites, uint64_t *keys, int8_t *eps, cudaStream_t stream) {
    if (U <= 0) return WICK_OK;
    DevBuf<uint64_t> d_R, d_keys;
    DevBuf<int8_t> d_eps;
    int err;
    if ((err = d_R.alloc((size_t)trials * n_blk)) || (err = d_keys.alloc(2 * (size_t)U)) || (err = d_eps.alloc(U)))
        return err;
    modp_blocks_kernel<<<(trials * n_blk + 127) / 128, 128, 0, stream>>>(bp, seed, trials, sites, d_R.p, n_blk);
    key_kernel<<<(unsigned)((U + 255) / 256), 256, 0, stream>>>(d_R.p, n_blk, trials, ids, U, A, d_keys.p, d_eps.p);
    WICK_CUDA_TRY(cudaGetLastError());
    WICK_CUDA_TRY(cudaMemcpyAsync(keys, d_keys.p, sizeof(uint64_t) * 2 * (size_t)U, cudaMemcpyDeviceToHost, stream));
    WICK_CUDA_TRY(cudaMemcpyAsync(eps, d_eps.p, (size_t)U, cudaMemcpyDeviceToHost, stream));
    WICK_CUDA_TRY(cudaStreamSynchronize(stream));
    return WICK_OK;
}

int selftest_hash_wait(int limit, int *status, cudaStream_t stream) {
    DevBuf<uint64_t> k;   // k0[0] = the claimed slot, k1[0]
    DevBuf<unsigned long long> rest;
    int err = k.alloc(2);
    if (!err) err = rest.alloc(3);
    if (err) return err;
    const uint64_t claimed[2] = {1ull | BUSY, 0ull};
    WICK_CUDA_TRY(cudaMemcpyAsync(k.p, claimed, sizeof(claimed), cudaMemcpyHostToDevice, stream));
    WICK_CUDA_TRY(cudaMemsetAsync(rest.p, 0, 3 * sizeof(unsigned long long), stream));
    HashTable ht{k.p, k.p + 1, rest.p, rest.p + 1, 0, rest.p + 2, 1};
    hash_wait_selftest_kernel<<<1, 1, 0, stream>>>(ht, limit, status);
    WICK_CUDA_TRY(cudaGetLastError());
    WICK_CUDA_TRY(cudaStreamSynchronize(stream));
    return WICK_OK;
}

}  // namespace wick
