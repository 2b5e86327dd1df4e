// C ABI of libwick: argument validation, host-side plans, the library-owned
// term table and the per-device workspace.  All arithmetic of the path runs
// in the kernels of blocks.cu, dedup.cu and contract.cu.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <numeric>
#include <vector>

#include "common.cuh"

struct wick_terms {
    int A = 0;
    int64_t U = 0;
    int n_blk = 0, n_ops = 0, n_spin = 0, n_chi = 0;
    int8_t chi[12] = {0};
    double scale = 1.0;
    int64_t stats[4] = {0, 0, 0, 0};
    double bound = 0.0;
    std::vector<uint16_t> ids;  // host copies
    std::vector<int64_t> w, rep;
    uint16_t *d_ids = nullptr;  // device copies (on the device current at creation)
    int64_t *d_w = nullptr, *d_rep = nullptr;
    uint16_t *d_ids_pad = nullptr;  // the contraction's copies: ids padded to 4 or 8, weights as doubles
    double *d_wd = nullptr;
    int device = 0;
    // correlation-matrix tables (wick_reduce_terms_matrix): n_el weights per term, one scale per element
    int n_el = 1;
    std::vector<int64_t> wm;        // [U][n_el]
    std::vector<double> el_scale;   // [n_el]
};

namespace wick {

// ---------------------------------------------------------------------------
// per-device workspace and status word
// ---------------------------------------------------------------------------
namespace {
struct DevState {
    void *ws[kWsSlots] = {};   // see common.cuh (kWs*)
    size_t ws_bytes[kWsSlots] = {};
    int *status = nullptr;
};
std::mutex g_mu;
std::map<int, DevState> g_dev;
}  // namespace

namespace {
std::atomic<int> g_alloc_countdown{0};   // wick_inject_alloc_failure: allocations until the one that fails
}  // namespace

int dev_malloc(void **ptr, size_t bytes) {
    *ptr = nullptr;
    for (int n = g_alloc_countdown.load(); n > 0;)
        if (g_alloc_countdown.compare_exchange_weak(n, n - 1)) {
            if (n == 1) return WICK_ENOMEM;
            break;
        }
    if (cudaMalloc(ptr, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        *ptr = nullptr;
        return WICK_ENOMEM;
    }
    return WICK_OK;
}

void *workspace(int slot, size_t bytes, int *err) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { *err = WICK_ECUDA; return nullptr; }
    std::lock_guard<std::mutex> lk(g_mu);
    DevState &d = g_dev[dev];
    if (d.ws_bytes[slot] < bytes) {
        // cudaFree waits for the device, so work still using the old buffer finishes first
        if (d.ws[slot]) cudaFree(d.ws[slot]);
        d.ws[slot] = nullptr;
        d.ws_bytes[slot] = 0;
        size_t want = bytes + bytes / 4;
        if (dev_malloc((void **)&d.ws[slot], want) != WICK_OK) {
            (void)cudaGetLastError();
            *err = WICK_ENOMEM;
            return nullptr;
        }
        // zero once: the kernels' work counters start at zero and reset themselves after every launch
        if (cudaMemset(d.ws[slot], 0, want) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
            (void)cudaGetLastError();
            cudaFree(d.ws[slot]);
            d.ws[slot] = nullptr;
            *err = WICK_ECUDA;
            return nullptr;
        }
        d.ws_bytes[slot] = want;
    }
    *err = WICK_OK;
    return d.ws[slot];
}

int *status_word(int *err) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { *err = WICK_ECUDA; return nullptr; }
    std::lock_guard<std::mutex> lk(g_mu);
    DevState &d = g_dev[dev];
    if (!d.status) {
        if (dev_malloc((void **)&d.status, sizeof(int)) != WICK_OK || cudaMemset(d.status, 0, sizeof(int)) != cudaSuccess) {
            (void)cudaGetLastError();
            d.status = nullptr;
            *err = WICK_ENOMEM;
            return nullptr;
        }
    }
    *err = WICK_OK;
    return d.status;
}

int status_read_clear(cudaStream_t stream) {
    int err = WICK_OK;
    int *st = status_word(&err);
    if (err) return err;
    int h = 0;
    WICK_CUDA_TRY(cudaMemcpyAsync(&h, st, sizeof(int), cudaMemcpyDeviceToHost, stream));
    WICK_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(int), stream));
    WICK_CUDA_TRY(cudaStreamSynchronize(stream));
    return h;
}

// ---------------------------------------------------------------------------
// layouts and plans
// ---------------------------------------------------------------------------
int terms_table(const wick_terms *t, ContractTable *tab, int *n_blk) {
    if (!t) return WICK_EINVAL;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != t->device) return WICK_EINVAL;  // the device copies live on another GPU
    if (t->U > 0 && (!t->d_ids_pad || !t->d_wd)) return WICK_EINVAL;
    // the float-pair weights follow the doubles in the same allocation (make_contract_copies)
    const size_t nw = (size_t)(t->U ? t->U : 1) * t->n_el;
    *tab = {t->d_ids_pad, t->d_wd, t->U, t->A, t->scale, t->n_el > 1 ? t->el_scale.data() : nullptr,
            t->d_wd ? reinterpret_cast<const float2 *>(t->d_wd + nw) : nullptr};
    *n_blk = t->n_blk;
    return WICK_OK;
}

// ---------------------------------------------------------------------------
// process-wide tuning (set by wick_set_tuning, read when a call plans its launches)
// ---------------------------------------------------------------------------
namespace {
std::mutex g_tune_mu;
wick_tuning g_tuning = {0, 0, 0, 0, 0, 0, 0};
}  // namespace

wick_tuning current_tuning() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_tuning;
}

ContractTune contract_tune(const wick_tuning &t) { return {t.contract_threads, t.contract_ctas_per_sm, t.contract_chunk_terms}; }

static bool layout_ok(const wick_block_layout *l) {
    if (!l || l->n_ops < 1 || l->n_ops > kMaxOps || l->n_spin < 1 || l->n_spin > kMaxSpin || l->n_chi < 1 ||
        l->n_chi > 12)
        return false;
    for (int i = 0; i < l->n_chi; ++i) {
        if (l->chi[i] < 0 || l->chi[i] > 11) return false;
        if (i && l->chi[i] <= l->chi[i - 1]) return false;
    }
    return true;
}

int build_block_plan(const wick_nucleon_op *ops, const wick_block_layout *layout, BlockPlan *plan) {
    if (!ops || !layout_ok(layout)) return WICK_EINVAL;
    BlockPlan &P = *plan;
    memset(&P, 0, sizeof(P));
    P.n_ops = layout->n_ops;
    P.n_spin = layout->n_spin;
    P.n_chi = layout->n_chi;
    P.n_out = P.n_ops * P.n_spin * P.n_chi * P.n_chi * P.n_chi;
    for (int i = 0; i < P.n_chi; ++i) P.chi[i] = layout->chi[i];
    int row_pos[2][12];
    for (int f = 0; f < 2; ++f)
        for (int r = 0; r < 12; ++r) row_pos[f][r] = -1;
    // rows used per flavour
    for (int o = 0; o < P.n_ops; ++o) {
        const wick_nucleon_op &op = ops[o];
        if (op.flav_pair != WICK_U && op.flav_pair != WICK_D) return WICK_EINVAL;
        if (op.n_entries < 1 || !op.entries || !op.w) return WICK_EINVAL;
        P.f1[o] = op.flav_pair;
        for (int e = 0; e < op.n_entries; ++e) {
            const int8_t *en = op.entries + 4 * e;
            if (en[0] < 0 || en[0] >= P.n_spin) return WICK_EINVAL;
            for (int q = 1; q < 4; ++q)
                if (en[q] < 0 || en[q] > 11) return WICK_EINVAL;
            if (op.w[e] == 0 || op.w[e] > (1 << 20) || op.w[e] < -(1 << 20)) return WICK_EINVAL;
            const int f1 = op.flav_pair, f2 = 1 - f1;
            row_pos[f1][(int)en[1]] = row_pos[f1][(int)en[2]] = 0;
            row_pos[f2][(int)en[3]] = 0;
        }
    }
    for (int f = 0; f < 2; ++f)
        for (int r = 0; r < 12; ++r)
            if (row_pos[f][r] == 0) {
                row_pos[f][r] = P.n_rows[f];
                P.rows[f][P.n_rows[f]++] = (int8_t)r;
            }
    // diquark lists and (row1, list) terms
    int n_xt = 0, n_ost = 0;
    P.x_off[0] = 0;
    for (int o = 0; o < P.n_ops; ++o) {
        const wick_nucleon_op &op = ops[o];
        const int f1 = op.flav_pair, f2 = 1 - f1;
        std::vector<std::vector<std::pair<std::pair<int, int>, int>>> lists;  // per op, for reuse
        std::vector<int> list_index;
        for (int s = 0; s < P.n_spin; ++s) {
            const int os = o * P.n_spin + s;
            P.os_off[os] = n_ost;
            // group entries of spin s by row 1
            std::map<int, std::map<std::pair<int, int>, int>> by_r1;
            for (int e = 0; e < op.n_entries; ++e) {
                const int8_t *en = op.entries + 4 * e;
                if (en[0] != s) continue;
                by_r1[en[1]][{en[2], en[3]}] += op.w[e];
            }
            for (auto &kv : by_r1) {
                std::vector<std::pair<std::pair<int, int>, int>> L;
                for (auto &t : kv.second)
                    if (t.second != 0) L.push_back({t.first, t.second});
                if (L.empty()) continue;
                int li = -1;
                for (size_t q = 0; q < lists.size(); ++q)
                    if (lists[q] == L) li = list_index[q];
                if (li < 0) {
                    if (P.n_x >= kMaxX || n_xt + (int)L.size() > kMaxXTerms) return WICK_EINVAL;
                    li = P.n_x++;
                    P.x_op[li] = o;
                    for (auto &t : L) {
                        P.xt_r2[n_xt] = (int8_t)row_pos[f1][t.first.first];
                        P.xt_r3[n_xt] = (int8_t)row_pos[f2][t.first.second];
                        P.xt_w[n_xt] = (float)t.second;
                        ++n_xt;
                    }
                    P.x_off[li + 1] = n_xt;
                    lists.push_back(L);
                    list_index.push_back(li);
                }
                if (n_ost >= kMaxOsTerms) return WICK_EINVAL;
                P.os_r1[n_ost] = (int8_t)row_pos[f1][kv.first];
                P.os_x[n_ost] = (int16_t)li;
                ++n_ost;
            }
        }
    }
    P.os_off[P.n_ops * P.n_spin] = n_ost;
    P.pow2_w = 1;
    for (int q = 0; q < n_xt; ++q) {
        const int a = (int)fabsf(P.xt_w[q]);
        if (a == 0 || (a & (a - 1)) != 0) P.pow2_w = 0;
    }
    return WICK_OK;
}

static int prop_ok(const wick_prop *p) {
    if (!p || !p->data || p->L < 1 || p->T < 1 || p->n_src < 1) return 0;
    if (p->dtype != WICK_C128 && p->dtype != WICK_C64) return 0;
    if (((uintptr_t)p->data) % 16) return 0;
    return 1;
}

}  // namespace wick

using namespace wick;

// the contraction's copies of a table (padded ids; the weights as doubles, then as exact float pairs for
// the MIXED term sums), from its device ids and its weights
static int make_contract_copies(wick_terms *t) {
    cudaFree(t->d_ids_pad);
    cudaFree(t->d_wd);
    t->d_ids_pad = nullptr;
    t->d_wd = nullptr;
    const size_t U = (size_t)(t->U ? t->U : 1);
    const int AP = t->A <= 4 ? 4 : 8;
    if (dev_malloc((void **)&t->d_ids_pad, sizeof(uint16_t) * U * AP) != WICK_OK ||
        dev_malloc((void **)&t->d_wd, (sizeof(double) + sizeof(float2)) * U * t->n_el) != WICK_OK) {
        (void)cudaGetLastError();
        return WICK_ENOMEM;
    }
    const std::vector<int64_t> &w = t->n_el > 1 ? t->wm : t->w;
    for (int64_t v : w)
        if (v >= (1ll << 53) || v <= -(1ll << 53)) return WICK_EOVERFLOW;
    int err = pad_table(t->d_ids, t->n_el > 1 ? nullptr : t->d_w, t->U, t->A, t->d_ids_pad, t->d_wd, nullptr);
    if (err) return err;
    if (t->n_el > 1 && t->U > 0) {
        std::vector<double> wd(w.begin(), w.end());
        WICK_CUDA_TRY(cudaMemcpy(t->d_wd, wd.data(), sizeof(double) * wd.size(), cudaMemcpyHostToDevice));
    }
    err = split_weights(t->d_wd, t->U * t->n_el, reinterpret_cast<float2 *>(t->d_wd + U * t->n_el), nullptr);
    if (err) return err;
    WICK_CUDA_TRY(cudaDeviceSynchronize());
    return WICK_OK;
}

extern "C" {

size_t wick_block_count(const wick_block_layout *layout) {
    if (!layout_ok(layout)) return 0;
    return (size_t)layout->n_ops * layout->n_spin * layout->n_chi * layout->n_chi * layout->n_chi;
}

static int is_page_locked(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return a.type == cudaMemoryTypeHost;
}

int wick_upload_rows(const wick_prop *Su_host, const wick_prop *Sd_host, const wick_prop *Su_dev,
                     const wick_prop *Sd_dev, const wick_nucleon_op *ops, const wick_block_layout *layout,
                     int mode, size_t *bytes, wick_stream_t stream) {
    const wick_prop *h[2] = {Su_host, Sd_host}, *d[2] = {Su_dev, Sd_dev};
    if (mode != WICK_UPLOAD_AUTO && mode != WICK_UPLOAD_DMA && mode != WICK_UPLOAD_KERNEL) return WICK_EINVAL;
    for (int f = 0; f < 2; ++f) {
        if (!h[f] || !d[f] || !h[f]->data || !prop_ok(d[f])) return WICK_EINVAL;
        if (h[f]->L != d[f]->L || h[f]->T != d[f]->T || h[f]->n_src != d[f]->n_src || h[f]->dtype != d[f]->dtype ||
            (h[f]->dtype != WICK_C64 && h[f]->dtype != WICK_C128))
            return WICK_EINVAL;
        if (!is_page_locked(h[f]->data)) return WICK_EINVAL;
    }
    BlockPlan plan;
    int err = build_block_plan(ops, layout, &plan);
    if (err) return err;
    // the copy engines by default: the gather kernel moves the rows faster on an idle GPU but takes SM
    // slots from a block build that runs beside it
    const bool use_kernel = mode == WICK_UPLOAD_KERNEL;
    const void *hdev[2] = {nullptr, nullptr};   // the device addresses of the host buffers
    if (use_kernel)
        for (int f = 0; f < 2; ++f) {
            void *p = nullptr;
            if (cudaHostGetDevicePointer(&p, const_cast<void *>(h[f]->data), 0) != cudaSuccess) {
                (void)cudaGetLastError();
                return WICK_EINVAL;
            }
            if ((uintptr_t)p % 16) return WICK_EINVAL;
            hdev[f] = p;
        }
    size_t total = 0;
    UploadMap map;
    map.n = 0;
    for (int f = 0; f < 2; ++f) {
        const size_t el = h[f]->dtype == WICK_C64 ? 8 : 16;
        const size_t rows = (size_t)h[f]->n_src * h[f]->T * h[f]->L * h[f]->L * h[f]->L;   // sites x slices
        const size_t pitch = 144 * el;                                                     // one site
        // runs of consecutive rows (the plan lists them ascending): one pitched copy each
        for (int i = 0; i < plan.n_rows[f];) {
            int j = i + 1;
            while (j < plan.n_rows[f] && plan.rows[f][j] == plan.rows[f][j - 1] + 1) ++j;
            const size_t off = (size_t)plan.rows[f][i] * 12 * el, width = (size_t)(j - i) * 12 * el;
            if (use_kernel) {
                for (size_t wd = off / 16; wd < (off + width) / 16; ++wd) map.word[map.n++] = (uint16_t)(f << 15 | wd);
            } else {
                WICK_CUDA_TRY(cudaMemcpy2DAsync((char *)d[f]->data + off, pitch, (const char *)h[f]->data + off,
                                                pitch, width, rows, cudaMemcpyHostToDevice, (cudaStream_t)stream));
            }
            total += width * rows;
            i = j;
        }
    }
    if (use_kernel && map.n > 0) {
        const size_t n_sites = (size_t)h[0]->n_src * h[0]->T * h[0]->L * h[0]->L * h[0]->L;
        int err2 = launch_upload_rows(map, hdev[0], hdev[1], d[0]->data, d[1]->data, n_sites,
                                      h[0]->dtype == WICK_C64 ? 72 : 144, h[1]->dtype == WICK_C64 ? 72 : 144,
                                      (cudaStream_t)stream);
        if (err2) return err2;
    }
    if (bytes) *bytes = total;
    return WICK_OK;
}

int wick_build_blocks(const wick_prop *Su, const wick_prop *Sd, const wick_nucleon_op *ops,
                      const wick_block_layout *layout, int precision, void *blocks, wick_stream_t stream) {
    if (!prop_ok(Su) || !prop_ok(Sd) || !blocks) return WICK_EINVAL;
    if (Su->L != Sd->L || Su->T != Sd->T || Su->n_src != Sd->n_src || Su->dtype != Sd->dtype) return WICK_EINVAL;
    if (precision != WICK_FP64 && precision != WICK_MIXED && precision != WICK_MIXED_SIMT) return WICK_EINVAL;
    if ((uintptr_t)blocks % 16) return WICK_EINVAL;
    BlockPlan plan;
    int err = build_block_plan(ops, layout, &plan);
    if (err) return err;
    const int64_t V = (int64_t)Su->L * Su->L * Su->L;
    const int64_t n_slices = (int64_t)Su->n_src * Su->T;
    if (V > (1 << 24) || n_slices > 65535) return WICK_EINVAL;
    const int rs = current_tuning().range_sites;
    const size_t pbytes = block_partial_bytes(plan, (int)V, (int)n_slices, precision, rs);
    const size_t cbytes = block_counter_bytes(plan, (int)n_slices, precision);
    void *part = workspace(kWsBlockPartials, pbytes, &err);
    if (err) return err;
    void *cnt = cbytes ? workspace(kWsBlockCounters, cbytes, &err) : nullptr;
    if (err) return err;
    return launch_block_build(plan, Su->data, Su->dtype, Sd->data, Sd->dtype, (int)V, (int)n_slices, precision, rs,
                              (int *)cnt, part, (double2 *)blocks, (cudaStream_t)stream);
}

int wick_reduce_terms(const wick_nucleus *nuc, const wick_nucleon_op *ops, const wick_block_layout *layout,
                      uint64_t seed, int trials, int sites, wick_terms **out, wick_stream_t stream) {
    if (!out) return WICK_EINVAL;
    *out = nullptr;
    if (!nuc || trials < 1 || trials > 2 || sites < 1 || sites > 64) return WICK_EINVAL;
    BlockPlan bp;
    int err = build_block_plan(ops, layout, &bp);
    if (err) return err;
    const int A = nuc->A, nq = 3 * A;
    if (A < 1 || A > kMaxA || nuc->n_sink < 1 || nuc->n_src < 1 || !nuc->sink_type || !nuc->sink_spin ||
        !nuc->sink_w || !nuc->src_chi || !nuc->src_w || !nuc->src_flav)
        return WICK_EINVAL;
    EnumPlan ep;
    memset(&ep, 0, sizeof(ep));
    ep.A = A;
    ep.nq = nq;
    ep.n_sink = nuc->n_sink;
    ep.n_spin = layout->n_spin;
    ep.n_chi = layout->n_chi;
    ep.n_blk = (int)wick_block_count(layout);
    for (int q = 0; q < nq; ++q) {
        if (nuc->src_flav[q] == WICK_U) ep.ju[ep.nu++] = q;
        else if (nuc->src_flav[q] == WICK_D) ep.jd[ep.nd++] = q;
        else return WICK_EINVAL;
    }
    if (ep.nu > 12 || ep.nd > 12) return WICK_EINVAL;
    ep.fu = 1;
    for (int i = 2; i <= ep.nu; ++i) ep.fu *= i;
    ep.fd = 1;
    for (int i = 2; i <= ep.nd; ++i) ep.fd *= i;
    // source index positions in the layout
    int cidx[12];
    for (int c = 0; c < 12; ++c) cidx[c] = -1;
    for (int i = 0; i < layout->n_chi; ++i) cidx[(int)layout->chi[i]] = i;
    for (size_t e = 0; e < (size_t)nuc->n_src * nq; ++e) {
        const int c = nuc->src_chi[e];
        if (c < 0 || c > 11 || cidx[c] < 0) return WICK_EINVAL;
    }
    // Antisymmetrised source (method B of Sec. III.C): a source tuple whose u
    // (or d) indices repeat cancels in the sum over permutations; every other
    // tuple is a signed reordering of its sorted multiset pair, so the source
    // collapses onto the sorted multisets with summed signed weights.
    std::map<std::vector<int8_t>, int64_t> msets;
    auto sort_sign = [](int8_t *x, int n) {
        int sgn = 1;
        for (int a = 1; a < n; ++a)
            for (int b = a; b > 0 && x[b - 1] >= x[b]; --b) {
                if (x[b - 1] == x[b]) return 0;
                std::swap(x[b], x[b - 1]);
                sgn = -sgn;
            }
        for (int a = 1; a < n; ++a)
            if (x[a - 1] == x[a]) return 0;
        return sgn;
    };
    for (int m = 0; m < nuc->n_src; ++m) {
        std::vector<int8_t> key((size_t)(ep.nu + ep.nd));
        for (int k = 0; k < ep.nu; ++k) key[k] = (int8_t)cidx[(int)nuc->src_chi[(size_t)m * nq + ep.ju[k]]];
        for (int k = 0; k < ep.nd; ++k) key[ep.nu + k] = (int8_t)cidx[(int)nuc->src_chi[(size_t)m * nq + ep.jd[k]]];
        const int su = sort_sign(key.data(), ep.nu), sd = sort_sign(key.data() + ep.nu, ep.nd);
        if (!su || !sd) continue;
        msets[key] += nuc->src_w[m] * su * sd;
    }
    std::vector<int8_t> Mu, Md;
    std::vector<int64_t> CM;
    for (auto &kv : msets) {
        if (kv.second == 0) continue;
        Mu.insert(Mu.end(), kv.first.begin(), kv.first.begin() + ep.nu);
        Md.insert(Md.end(), kv.first.begin() + ep.nu, kv.first.end());
        CM.push_back(kv.second);
    }
    ep.n_M = (int)CM.size();
    if (Mu.empty()) Mu.push_back(0);
    if (Md.empty()) Md.push_back(0);
    // raw-term count, guarded against overflow
    long double nr = (long double)ep.n_sink * ep.n_M * (long double)ep.fu * (long double)ep.fd;
    if (nr > 4.0e18L) return WICK_EOVERFLOW;
    ep.n_raw = (int64_t)ep.n_sink * ep.n_M * ep.fu * ep.fd;
    // weights: the in-warp sum of 32 coefficients must fit in int32
    int64_t max_sw = 0, max_cw = 0;
    for (int i = 0; i < ep.n_sink; ++i) max_sw = std::max<int64_t>(max_sw, llabs(nuc->sink_w[i]));
    for (int64_t w : CM) max_cw = std::max<int64_t>(max_cw, llabs(w));
    if ((long double)max_sw * max_cw * 32.0L >= 2147483647.0L) return WICK_EOVERFLOW;
    // sink quark flavours, flavour ordinals and the identity-pairing parity
    std::vector<int8_t> sflav((size_t)ep.n_sink * nq), sord((size_t)ep.n_sink * nq), seta(ep.n_sink);
    for (int i = 0; i < ep.n_sink; ++i) {
        int mu = 0, md = 0;
        int pi[3 * kMaxA];
        for (int k = 0; k < A; ++k) {
            const int o = nuc->sink_type[i * A + k], s = nuc->sink_spin[i * A + k];
            if (o < 0 || o >= layout->n_ops || s < 0 || s >= layout->n_spin) return WICK_EINVAL;
            for (int sl = 0; sl < 3; ++sl) {
                const int f = sl < 2 ? ops[o].flav_pair : 1 - ops[o].flav_pair;
                const int q = 3 * k + sl;
                sflav[(size_t)i * nq + q] = (int8_t)f;
                const int ord = f == WICK_U ? mu++ : md++;
                sord[(size_t)i * nq + q] = (int8_t)ord;
                if (ord >= (f == WICK_U ? ep.nu : ep.nd)) return WICK_EINVAL;
                pi[q] = f == WICK_U ? ep.ju[ord] : ep.jd[ord];
            }
        }
        if (mu != ep.nu || md != ep.nd) return WICK_EINVAL;
        int inv = 0;
        for (int a = 0; a < nq; ++a)
            for (int b = a + 1; b < nq; ++b) inv += pi[a] > pi[b];
        seta[i] = (int8_t)((inv & 1) ? -1 : 1);
    }
    ReduceResult rr;
    memset(&rr, 0, sizeof(rr));
    err = run_reduce(ep, bp, nuc, Mu.data(), Md.data(), CM.data(), sflav.data(), sord.data(), seta.data(), seed,
                     trials, sites, &rr, (cudaStream_t)stream);
    if (err) return err;
    wick_terms *t = new (std::nothrow) wick_terms();
    if (!t) {
        cudaFree(rr.d_ids); cudaFree(rr.d_w); cudaFree(rr.d_rep);
        return WICK_ENOMEM;
    }
    cudaGetDevice(&t->device);
    t->A = A;
    t->U = rr.U;
    t->n_blk = ep.n_blk;
    t->n_ops = layout->n_ops;
    t->n_spin = layout->n_spin;
    t->n_chi = layout->n_chi;
    memcpy(t->chi, layout->chi, sizeof(t->chi));
    t->scale = nuc->scale;
    t->stats[0] = ep.n_raw;
    t->stats[1] = rr.n_zero;
    t->stats[2] = rr.n_keys;
    t->stats[3] = rr.U;
    const double pairs = 0.5 * (double)ep.n_raw * (double)ep.n_raw;
    t->bound = std::min(1.0, pairs * pow(3.0 * A / 2305843009213693951.0, trials));
    t->d_ids = rr.d_ids;
    t->d_w = rr.d_w;
    t->d_rep = rr.d_rep;
    t->ids.resize((size_t)rr.U * A);
    t->w.resize(rr.U);
    t->rep.resize(rr.U);
    if (rr.U > 0 &&
        (cudaMemcpy(t->ids.data(), rr.d_ids, sizeof(uint16_t) * t->ids.size(), cudaMemcpyDeviceToHost) != cudaSuccess ||
         cudaMemcpy(t->w.data(), rr.d_w, sizeof(int64_t) * rr.U, cudaMemcpyDeviceToHost) != cudaSuccess ||
         cudaMemcpy(t->rep.data(), rr.d_rep, sizeof(int64_t) * rr.U, cudaMemcpyDeviceToHost) != cudaSuccess)) {
        wick_terms_free(t);
        return WICK_ECUDA;
    }
    err = make_contract_copies(t);
    if (err) {
        wick_terms_free(t);
        return err;
    }
    *out = t;
    return WICK_OK;
}

int64_t wick_terms_count(const wick_terms *t) { return t ? t->U : WICK_EINVAL; }
int wick_terms_nucleons(const wick_terms *t) { return t ? t->A : WICK_EINVAL; }
int64_t wick_terms_block_count(const wick_terms *t) { return t ? (int64_t)t->n_blk : WICK_EINVAL; }

int wick_terms_copy(const wick_terms *t, uint16_t *ids, int64_t *w, int64_t *rep) {
    if (!t || t->n_el > 1) return WICK_EINVAL;
    if (ids && !t->ids.empty()) memcpy(ids, t->ids.data(), sizeof(uint16_t) * t->ids.size());
    if (w && !t->w.empty()) memcpy(w, t->w.data(), sizeof(int64_t) * t->w.size());
    if (rep && !t->rep.empty()) memcpy(rep, t->rep.data(), sizeof(int64_t) * t->rep.size());
    return WICK_OK;
}

int wick_terms_stats(const wick_terms *t, int64_t stats[4], double *bound) {
    if (!t) return WICK_EINVAL;
    if (stats) memcpy(stats, t->stats, sizeof(t->stats));
    if (bound) *bound = t->bound;
    return WICK_OK;
}

static int upload_terms(wick_terms *t) {
    cudaFree(t->d_ids); cudaFree(t->d_w); cudaFree(t->d_rep);
    t->d_ids = nullptr; t->d_w = nullptr; t->d_rep = nullptr;
    const size_t U = (size_t)(t->U ? t->U : 1);
    if (dev_malloc((void **)&t->d_ids, sizeof(uint16_t) * U * t->A) != WICK_OK ||
        dev_malloc((void **)&t->d_w, sizeof(int64_t) * U) != WICK_OK ||
        dev_malloc((void **)&t->d_rep, sizeof(int64_t) * U) != WICK_OK) {
        (void)cudaGetLastError();
        return WICK_ENOMEM;
    }
    if (t->U > 0 &&
        (cudaMemcpy(t->d_ids, t->ids.data(), sizeof(uint16_t) * t->ids.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(t->d_w, t->w.data(), sizeof(int64_t) * t->U, cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(t->d_rep, t->rep.data(), sizeof(int64_t) * t->U, cudaMemcpyHostToDevice) != cudaSuccess))
        return WICK_ECUDA;
    cudaGetDevice(&t->device);
    return make_contract_copies(t);
}

int wick_terms_select(wick_terms *t, const int64_t *perm, int64_t n) {
    if (!t || t->n_el > 1 || n < 0 || n > t->U || (n > 0 && !perm)) return WICK_EINVAL;
    std::vector<int64_t> keep(perm, perm + n);
    std::vector<char> seen((size_t)t->U, 0);
    for (int64_t v : keep) {
        if (v < 0 || v >= t->U || seen[(size_t)v]) return WICK_EINVAL;
        seen[(size_t)v] = 1;
    }
    std::sort(keep.begin(), keep.end());  // table order = order of representatives
    std::vector<uint16_t> ids((size_t)n * t->A);
    std::vector<int64_t> w(n), rep(n);
    for (int64_t q = 0; q < n; ++q) {
        const int64_t u = keep[q];
        memcpy(&ids[(size_t)q * t->A], &t->ids[(size_t)u * t->A], sizeof(uint16_t) * t->A);
        w[q] = t->w[u];
        rep[q] = t->rep[u];
    }
    t->ids.swap(ids);
    t->w.swap(w);
    t->rep.swap(rep);
    t->U = n;
    t->stats[3] = n;
    return upload_terms(t);
}

int wick_terms_magnitudes(const void *blocks, int n_slices, const wick_terms *t, double *mag, wick_stream_t stream) {
    if (!blocks || !t || !mag || n_slices < 1 || (uintptr_t)blocks % 16 || t->n_el > 1) return WICK_EINVAL;
    ContractTable tab;
    int n_blk = 0;
    int err = terms_table(t, &tab, &n_blk);
    if (err) return err;
    if (t->U == 0) return WICK_OK;
    double *d_mag = nullptr;
    if (dev_malloc((void **)&d_mag, sizeof(double) * (size_t)t->U) != WICK_OK) {
        (void)cudaGetLastError();
        return WICK_ENOMEM;
    }
    err = launch_magnitudes((const double2 *)blocks, n_blk, n_slices, tab, d_mag, (cudaStream_t)stream);
    if (!err && (cudaMemcpyAsync(mag, d_mag, sizeof(double) * (size_t)t->U, cudaMemcpyDeviceToHost,
                                 (cudaStream_t)stream) != cudaSuccess ||
                 cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)) {
        (void)cudaGetLastError();
        err = WICK_ECUDA;
    }
    cudaFree(d_mag);
    return err;
}

int wick_terms_top(wick_terms *t, const double *mag, double fraction) {
    if (!t || !mag || !(fraction > 0.0) || fraction > 1.0) return WICK_EINVAL;
    const int64_t U = t->U;
    int64_t n = (int64_t)ceil(fraction * (double)U - 1e-9);
    n = std::max<int64_t>(std::min<int64_t>(n, U), U > 0 ? 1 : 0);
    std::vector<int64_t> order((size_t)U);
    std::iota(order.begin(), order.end(), (int64_t)0);
    for (int64_t u = 0; u < U; ++u)
        if (!(mag[u] >= 0.0)) return WICK_EINVAL;   // negative or NaN
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return mag[a] > mag[b]; });
    return wick_terms_select(t, order.data(), n);
}

// file format: "WICKTBL1" | u32 version | header fields | arrays | u64 FNV-1a of the arrays
static uint64_t fnv1a(const void *p, size_t n, uint64_t h) {
    const unsigned char *c = (const unsigned char *)p;
    for (size_t i = 0; i < n; ++i) { h ^= c[i]; h *= 1099511628211ull; }
    return h;
}

int wick_terms_save(const wick_terms *t, const char *path) {
    if (!t || !path || t->n_el > 1) return WICK_EINVAL;
    FILE *f = fopen(path, "wb");
    if (!f) return WICK_EIO;
    const char magic[8] = {'W', 'I', 'C', 'K', 'T', 'B', 'L', '1'};
    const uint32_t version = 1;
    int32_t hdr[5] = {t->A, t->n_blk, t->n_ops, t->n_spin, t->n_chi};
    uint64_t h = 1469598103934665603ull;
    h = fnv1a(t->ids.data(), sizeof(uint16_t) * t->ids.size(), h);
    h = fnv1a(t->w.data(), sizeof(int64_t) * t->w.size(), h);
    h = fnv1a(t->rep.data(), sizeof(int64_t) * t->rep.size(), h);
    bool ok = fwrite(magic, 8, 1, f) == 1 && fwrite(&version, 4, 1, f) == 1 && fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
              fwrite(t->chi, 12, 1, f) == 1 && fwrite(&t->U, 8, 1, f) == 1 && fwrite(&t->scale, 8, 1, f) == 1 &&
              fwrite(t->stats, sizeof(t->stats), 1, f) == 1 && fwrite(&t->bound, 8, 1, f) == 1;
    if (ok && t->U > 0)
        ok = fwrite(t->ids.data(), sizeof(uint16_t), t->ids.size(), f) == t->ids.size() &&
             fwrite(t->w.data(), sizeof(int64_t), t->w.size(), f) == t->w.size() &&
             fwrite(t->rep.data(), sizeof(int64_t), t->rep.size(), f) == t->rep.size();
    ok = ok && fwrite(&h, 8, 1, f) == 1;
    ok = (fclose(f) == 0) && ok;
    return ok ? WICK_OK : WICK_EIO;
}

int wick_terms_load(const char *path, wick_terms **out) {
    if (!path || !out) return WICK_EINVAL;
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) return WICK_EIO;
    char magic[8];
    uint32_t version = 0;
    int32_t hdr[5];
    wick_terms *t = new (std::nothrow) wick_terms();
    if (!t) { fclose(f); return WICK_ENOMEM; }
    bool ok = fread(magic, 8, 1, f) == 1 && memcmp(magic, "WICKTBL1", 8) == 0 && fread(&version, 4, 1, f) == 1 &&
              version == 1 && fread(hdr, sizeof(hdr), 1, f) == 1 && fread(t->chi, 12, 1, f) == 1 &&
              fread(&t->U, 8, 1, f) == 1 && fread(&t->scale, 8, 1, f) == 1 &&
              fread(t->stats, sizeof(t->stats), 1, f) == 1 && fread(&t->bound, 8, 1, f) == 1;
    if (ok) {
        t->A = hdr[0]; t->n_blk = hdr[1]; t->n_ops = hdr[2]; t->n_spin = hdr[3]; t->n_chi = hdr[4];
        ok = t->A >= 1 && t->A <= kMaxA && t->U >= 0 && t->U < (1ll << 40) && t->n_blk > 0;
    }
    if (ok) {
        t->ids.resize((size_t)t->U * t->A);
        t->w.resize(t->U);
        t->rep.resize(t->U);
        if (t->U > 0)
            ok = fread(t->ids.data(), sizeof(uint16_t), t->ids.size(), f) == t->ids.size() &&
                 fread(t->w.data(), sizeof(int64_t), t->w.size(), f) == t->w.size() &&
                 fread(t->rep.data(), sizeof(int64_t), t->rep.size(), f) == t->rep.size();
    }
    uint64_t h_file = 0;
    ok = ok && fread(&h_file, 8, 1, f) == 1;
    fclose(f);
    if (ok) {
        uint64_t h = 1469598103934665603ull;
        h = fnv1a(t->ids.data(), sizeof(uint16_t) * t->ids.size(), h);
        h = fnv1a(t->w.data(), sizeof(int64_t) * t->w.size(), h);
        h = fnv1a(t->rep.data(), sizeof(int64_t) * t->rep.size(), h);
        ok = h == h_file;
        for (size_t i = 0; ok && i < t->ids.size(); ++i) ok = t->ids[i] < t->n_blk;
    }
    if (!ok) { delete t; return WICK_EIO; }
    int e = upload_terms(t);
    if (e) { wick_terms_free(t); return e; }
    *out = t;
    return WICK_OK;
}

void wick_terms_free(wick_terms *t) {
    if (!t) return;
    cudaFree(t->d_ids);
    cudaFree(t->d_w);
    cudaFree(t->d_rep);
    cudaFree(t->d_ids_pad);
    cudaFree(t->d_wd);
    delete t;
}

static int contract_args(const void *blocks, int n_src, int T, const wick_terms *t, int precision, void *C_out,
                         ContractTable *tab, int *n_blk) {
    if (!blocks || !t || !C_out || n_src < 1 || T < 1) return WICK_EINVAL;
    if (precision != WICK_FP64 && precision != WICK_MIXED) return WICK_EINVAL;
    if ((uintptr_t)blocks % 16 || (uintptr_t)C_out % 16) return WICK_EINVAL;
    if ((int64_t)n_src * T > 2147483647) return WICK_EINVAL;
    return terms_table(t, tab, n_blk);
}

int wick_contract(const void *blocks, int n_src, int T, const wick_terms *t, int precision, void *C_out,
                  wick_stream_t stream) {
    ContractTable tab;
    int n_blk = 0;
    int err = contract_args(blocks, n_src, T, t, precision, C_out, &tab, &n_blk);
    if (err) return err;
    const int n_slices = n_src * T;
    ContractPlan plan;
    err = contract_plan(n_blk, 1, n_slices, &tab, 1, precision, contract_tune(current_tuning()), INT64_MAX, &plan,
                        t->n_el > 1 ? t->n_el : 0);
    if (err) return err;
    void *part = workspace(kWsContractPartials, plan.partial_bytes, &err);
    if (err) return err;
    void *cnt = workspace(kWsContractCounters, plan.counter_bytes, &err);
    if (err) return err;
    void *conv = nullptr;
    if (plan.convert_bytes) {
        conv = workspace(kWsContractConvert, plan.convert_bytes, &err);
        if (err) return err;
    }
    return launch_contract((const double2 *)blocks, n_blk, 1, n_slices, &tab, 1, precision, plan, cnt,
                           (double2 *)part, (double2 *)C_out, (cudaStream_t)stream, nullptr, conv);
}

int wick_contract_noalloc(const void *blocks, int n_src, int T, const wick_terms *t, int precision, void *C_out,
                          wick_stream_t stream) {
    ContractTable tab;
    int n_blk = 0;
    int err = contract_args(blocks, n_src, T, t, precision, C_out, &tab, &n_blk);
    if (err) return err;
    const int64_t n_slices = (int64_t)n_src * T;
    if (t->n_el > 1) return WICK_EINVAL;
    if (n_slices > kNoAllocItems) return WICK_ESCRATCH;
    void *scratch = nullptr;
    size_t cap = 0;
    err = noalloc_scratch(&scratch, &cap);
    if (err) return err;
    ContractPlan plan;
    err = contract_plan(n_blk, 1, (int)n_slices, &tab, 1, precision, contract_tune(current_tuning()), kNoAllocItems,
                        &plan);
    if (err) return err;
    if (plan.counter_bytes > kNoAllocCounterBytes || plan.partial_bytes > cap - kNoAllocCounterBytes)
        return WICK_ESCRATCH;
    // the array keeps the last call's contents: clear the counters this launch starts from
    WICK_CUDA_TRY(cudaMemsetAsync(scratch, 0, plan.counter_bytes, (cudaStream_t)stream));
    double2 *partials = reinterpret_cast<double2 *>(static_cast<unsigned char *>(scratch) + kNoAllocCounterBytes);
    return launch_contract((const double2 *)blocks, n_blk, 1, (int)n_slices, &tab, 1, precision, plan, scratch,
                           partials, (double2 *)C_out, (cudaStream_t)stream);
}

int wick_terms_elements(const wick_terms *t) { return t ? t->n_el : WICK_EINVAL; }

int wick_terms_copy_matrix(const wick_terms *t, uint16_t *ids, int64_t *w, double *el_scale) {
    if (!t) return WICK_EINVAL;
    if (ids && !t->ids.empty()) memcpy(ids, t->ids.data(), sizeof(uint16_t) * t->ids.size());
    const std::vector<int64_t> &src = t->n_el > 1 ? t->wm : t->w;
    if (w && !src.empty()) memcpy(w, src.data(), sizeof(int64_t) * src.size());
    if (el_scale) {
        if (t->n_el > 1) memcpy(el_scale, t->el_scale.data(), sizeof(double) * t->n_el);
        else el_scale[0] = t->scale;
    }
    return WICK_OK;
}

int wick_reduce_terms_matrix(const wick_nucleus *nuclei, int n_nuc, const wick_nucleon_op *ops,
                             const wick_block_layout *layout, uint64_t seed, int trials, int sites, wick_terms **out,
                             wick_stream_t stream) {
    if (!out) return WICK_EINVAL;
    *out = nullptr;
    if (!nuclei || n_nuc < 2 || n_nuc > 4) return WICK_EINVAL;
    const int A = nuclei[0].A, nq = 3 * A;
    if (A < 1 || A > 4) return WICK_EINVAL;
    for (int i = 0; i < n_nuc; ++i) {
        if (nuclei[i].A != A || !nuclei[i].src_flav || !(nuclei[i].scale > 0.0)) return WICK_EINVAL;
        for (int q = 0; q < nq; ++q)
            if (nuclei[i].src_flav[q] != nuclei[0].src_flav[q]) return WICK_EINVAL;   // same quark content
    }
    BlockPlan bp;
    int err = build_block_plan(ops, layout, &bp);
    if (err) return err;
    const int n_blk = (int)wick_block_count(layout);
    const int n_el = n_nuc * n_nuc;
    wick_terms *t = new (std::nothrow) wick_terms();
    if (!t) return WICK_ENOMEM;
    t->A = A;
    t->n_blk = n_blk;
    t->n_ops = layout->n_ops;
    t->n_spin = layout->n_spin;
    t->n_chi = layout->n_chi;
    memcpy(t->chi, layout->chi, sizeof(t->chi));
    t->scale = 1.0;
    t->n_el = n_el;
    t->el_scale.resize(n_el);
    std::map<std::pair<uint64_t, uint64_t>, int64_t> index;   // key -> merged term
    std::vector<int8_t> eps_rep;
    double pairs = 0.0;
    for (int i = 0; i < n_nuc && !err; ++i)
        for (int j = 0; j < n_nuc && !err; ++j) {
            // element (i, j): the sink of operator i, the source of operator j (Eq. E1)
            wick_nucleus el = nuclei[i];
            el.n_src = nuclei[j].n_src;
            el.src_chi = nuclei[j].src_chi;
            el.src_w = nuclei[j].src_w;
            el.scale = sqrt(nuclei[i].scale * nuclei[j].scale);
            const int e = i * n_nuc + j;
            t->el_scale[e] = el.scale;
            wick_terms *te = nullptr;
            err = wick_reduce_terms(&el, ops, layout, seed, trials, sites, &te, stream);
            if (err) break;
            std::vector<uint64_t> keys(2 * (size_t)(te->U ? te->U : 1));
            std::vector<int8_t> eps((size_t)(te->U ? te->U : 1));
            err = term_keys(bp, n_blk, te->d_ids, te->U, A, seed, trials, sites, keys.data(), eps.data(),
                            (cudaStream_t)stream);
            for (int64_t u = 0; !err && u < te->U; ++u) {
                if (eps[u] == 0) { err = WICK_EINVAL; break; }   // a kept term has a non-zero key
                const auto key = std::make_pair(keys[2 * u], keys[2 * u + 1]);
                auto it = index.find(key);
                int64_t m;
                if (it == index.end()) {
                    m = t->U++;
                    index.emplace(key, m);
                    t->ids.insert(t->ids.end(), te->ids.begin() + u * A, te->ids.begin() + (u + 1) * A);
                    t->wm.resize((size_t)t->U * n_el, 0);
                    eps_rep.push_back(eps[u]);
                } else {
                    m = it->second;
                }
                // term value = eps_u * canonical value = eps_u * eps_rep * (product of the merged term's ids)
                t->wm[(size_t)m * n_el + e] += te->w[u] * eps[u] * eps_rep[m];
            }
            t->stats[0] += te->stats[0];
            t->stats[1] += te->stats[1];
            pairs += (double)te->stats[0];
            wick_terms_free(te);
        }
    if (err) {
        wick_terms_free(t);
        return err;
    }
    t->stats[2] = t->stats[3] = t->U;
    t->bound = std::min(1.0, 0.5 * pairs * pairs * pow(3.0 * A / 2305843009213693951.0, trials));
    t->w.assign(t->U, 0);
    t->rep.resize(t->U);
    std::iota(t->rep.begin(), t->rep.end(), (int64_t)0);
    cudaGetDevice(&t->device);
    const size_t U = (size_t)(t->U ? t->U : 1);
    if (dev_malloc((void **)&t->d_ids, sizeof(uint16_t) * U * A) != WICK_OK ||
        dev_malloc((void **)&t->d_w, sizeof(int64_t) * U) != WICK_OK || dev_malloc((void **)&t->d_rep, sizeof(int64_t) * U) != WICK_OK) {
        (void)cudaGetLastError();
        wick_terms_free(t);
        return WICK_ENOMEM;
    }
    if (t->U > 0 &&
        cudaMemcpy(t->d_ids, t->ids.data(), sizeof(uint16_t) * t->ids.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        (void)cudaGetLastError();
        wick_terms_free(t);
        return WICK_ECUDA;
    }
    err = make_contract_copies(t);
    if (err) {
        wick_terms_free(t);
        return err;
    }
    *out = t;
    return WICK_OK;
}

int wick_build_blocks_3pt(const wick_prop *Su, const wick_prop *Sd, const wick_prop *Sig, int flavour,
                          const wick_nucleon_op *ops, const wick_block_layout *layout, int precision, void *dblocks,
                          wick_stream_t stream) {
    if (!prop_ok(Su) || !prop_ok(Sd) || !prop_ok(Sig) || !dblocks || (uintptr_t)dblocks % 16) return WICK_EINVAL;
    if (Su->L != Sd->L || Su->T != Sd->T || Su->n_src != Sd->n_src || Su->dtype != Sd->dtype) return WICK_EINVAL;
    if (Sig->L != Su->L || Sig->T != Su->T || Sig->n_src != Su->n_src || Sig->dtype != Su->dtype) return WICK_EINVAL;
    if (flavour != WICK_U && flavour != WICK_D) return WICK_EINVAL;
    if (precision != WICK_FP64 && precision != WICK_MIXED) return WICK_EINVAL;
    BlockPlan plan;
    int err = build_block_plan(ops, layout, &plan);
    if (err) return err;
    const int64_t V = (int64_t)Su->L * Su->L * Su->L;
    const int64_t n_slices = (int64_t)Su->n_src * Su->T;
    if (V > (1 << 24) || n_slices > 65535) return WICK_EINVAL;
    if (precision == WICK_MIXED && tc_applicable_3pt(plan, flavour)) {
        // the tensor-core build with the role passes of the sequential propagator
        const int rs = current_tuning().range_sites;
        const size_t pbytes = tc_partial_bytes(plan, (int)V, (int)n_slices, 1, rs, 3);
        const size_t cbytes = tc_counter_bytes(plan, (int)n_slices, 1);
        void *part = workspace(kWsBlockPartials, pbytes, &err);
        if (err) return err;
        void *cnt = workspace(kWsBlockCounters, cbytes, &err);
        if (err) return err;
        int *status = status_word(&err);
        if (err) return err;
        return launch_block_tc(plan, &Su->data, &Sd->data, 1, Su->dtype, (int)V, (int)n_slices, rs, (int *)cnt,
                               (double2 *)part, (double2 *)dblocks, status, (cudaStream_t)stream, &Sig->data,
                               flavour);
    }
    const size_t bytes = block_3pt_partial_bytes(plan, (int)V, (int)n_slices);
    void *ws = workspace(kWsBlockPartials, bytes, &err);
    if (err) return err;
    return launch_block_build_3pt(plan, Su->data, Sd->data, Sig->data, Su->dtype, flavour, (int)V, (int)n_slices,
                                  precision, ws, (double2 *)dblocks, (cudaStream_t)stream);
}

int wick_contract_3pt(const void *blocks, const void *dblocks, int n_src, int T, const wick_terms *t, int precision,
                      void *C_out, wick_stream_t stream) {
    ContractTable tab;
    int n_blk = 0;
    int err = contract_args(blocks, n_src, T, t, precision, C_out, &tab, &n_blk);
    if (err) return err;
    if (!dblocks || (uintptr_t)dblocks % 16 || t->n_el > 1) return WICK_EINVAL;
    const int n_slices = n_src * T;
    ContractPlan plan;
    err = contract_plan(n_blk, 1, n_slices, &tab, 1, precision, contract_tune(current_tuning()), INT64_MAX, &plan, 1);
    if (err) return err;
    void *part = workspace(kWsContractPartials, plan.partial_bytes, &err);
    if (err) return err;
    void *cnt = workspace(kWsContractCounters, plan.counter_bytes, &err);
    if (err) return err;
    void *conv = nullptr;
    if (plan.convert_bytes) {
        conv = workspace(kWsContractConvert, plan.convert_bytes, &err);
        if (err) return err;
    }
    return launch_contract((const double2 *)blocks, n_blk, 1, n_slices, &tab, 1, precision, plan, cnt, (double2 *)part,
                           (double2 *)C_out, (cudaStream_t)stream, (const double2 *)dblocks, conv);
}

int wick_set_tuning(const wick_tuning *t) {
    wick_tuning v = {0, 0, 0, 0, 0, 0, 0};
    if (t) v = *t;
    if (v.no_pair_kernel != 0 && v.no_pair_kernel != 1) return WICK_EINVAL;
    if (v.hash_log2_start != 0 && (v.hash_log2_start < 4 || v.hash_log2_start > 28)) return WICK_EINVAL;
    if (v.hash_log2_max != 0 && (v.hash_log2_max < 4 || v.hash_log2_max > 28)) return WICK_EINVAL;
    if (v.range_sites < 0 || v.range_sites % 128 || v.range_sites > 4096) return WICK_EINVAL;
    if (v.contract_threads < 0 || v.contract_threads % 32 || v.contract_threads > 512) return WICK_EINVAL;
    if (v.contract_ctas_per_sm < 0 || v.contract_ctas_per_sm > 32) return WICK_EINVAL;
    if (v.contract_chunk_terms < 0 || (v.contract_chunk_terms > 0 && v.contract_chunk_terms < 64)) return WICK_EINVAL;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuning = v;
    return WICK_OK;
}

int wick_get_tuning(wick_tuning *t) {
    if (!t) return WICK_EINVAL;
    *t = current_tuning();
    return WICK_OK;
}

int wick_status(wick_stream_t stream) { return status_read_clear((cudaStream_t)stream); }

int wick_inject_alloc_failure(int k) {
    if (k < 0) return WICK_EINVAL;
    return g_alloc_countdown.exchange(k);
}

int wick_selftest_wait(int which, int limit, wick_stream_t stream) {
    if ((which != 0 && which != 1) || limit < 1 || limit > (1 << 22)) return WICK_EINVAL;
    const cudaStream_t s = (cudaStream_t)stream;
    int err = WICK_OK;
    int *status = status_word(&err);
    if (err) return err;
    err = status_read_clear(s);   // start from a clear word (an earlier error is dropped)
    (void)err;
    err = which == 0 ? selftest_hash_wait(limit, status, s) : selftest_mbar_wait(limit, status, s);
    if (err) return err;
    return status_read_clear(s);
}

const char *wick_strerror(int code) {
    switch (code) {
        case WICK_OK: return "ok";
        case WICK_EINVAL: return "invalid argument";
        case WICK_ENOMEM: return "out of memory";
        case WICK_ECUDA: return "CUDA error";
        case WICK_ECAPACITY: return "term table capacity exceeded";
        case WICK_EOVERFLOW: return "integer overflow";
        case WICK_ETIMEOUT: return "bounded device wait ran out";
        case WICK_EIO: return "term-table file missing, truncated or corrupt";
        case WICK_ESCRATCH: return "request exceeds the fixed scratch of wick_contract_noalloc";
        default: return "unknown error";
    }
}

const char *wick_version(void) { return "0.1.0"; }

}  // extern "C"
