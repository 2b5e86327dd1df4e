// Batched executor: many configurations x many nuclei in one CUDA graph of
// few launches.
//
// wick_batch_create records, for fixed device buffers, the block build of
// every configuration (Eq. 2.4/2.5) and the contraction of every reduced table
// against those blocks (Eq. 2.6 / App. D), captured on a private stream and
// instantiated once.  Nuclei built from the same nucleon operators share one
// block build per configuration.  With the tensor-core block build
// (WICK_MIXED) one launch covers up to 64 configurations (more launches only
// for larger batches or when their partial sums would pass kGroupBytes); one
// persistent launch then evaluates every (configuration, table, slice, chunk
// of terms) work item.  He-4-sized batches of up to 64 configurations are
// therefore two kernel launches.  The batch owns its scratch, zeroed at
// creation (the kernels' counters reset themselves after every launch), so
// the graph never depends on the library's shared workspace.  wick_batch_run
// launches the graph on a stream: one host call per batch.
#include <vector>

#include "common.cuh"

struct wick_batch {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    void *block_scratch = nullptr;
    void *contract_scratch = nullptr;
    int n_launches = 0;
};

namespace {
constexpr size_t kGroupBytes = size_t(4) << 30;   // partial sums of one block-build launch, at most
}

extern "C" int wick_batch_create(const wick_prop *Su, const wick_prop *Sd, int n_cfg, const wick_nucleon_op *ops,
                                 const wick_block_layout *layout, const wick_terms *const *tables, int n_tables,
                                 int precision, void *blocks, void *C_out, wick_batch **out) {
    using namespace wick;
    if (!out) return WICK_EINVAL;
    *out = nullptr;
    if (!Su || !Sd || n_cfg < 1 || !tables || n_tables < 1 || n_tables > kMaxTables || !blocks || !C_out)
        return WICK_EINVAL;
    if (precision != WICK_FP64 && precision != WICK_MIXED) return WICK_EINVAL;
    if ((uintptr_t)blocks % 16 || (uintptr_t)C_out % 16) return WICK_EINVAL;
    BlockPlan plan;
    int err = build_block_plan(ops, layout, &plan);
    if (err) return err;
    const int L = Su[0].L, T = Su[0].T, n_src = Su[0].n_src, dtype = Su[0].dtype;
    for (int c = 0; c < n_cfg; ++c) {
        const wick_prop *p[2] = {&Su[c], &Sd[c]};
        for (auto q : p)
            if (!q->data || q->L != L || q->T != T || q->n_src != n_src || q->dtype != dtype ||
                ((uintptr_t)q->data) % 16)
                return WICK_EINVAL;
    }
    const int64_t V = (int64_t)L * L * L, n_slices = (int64_t)n_src * T;
    if (V > (1 << 24) || n_slices > 65535 || L < 1 || T < 1 || n_src < 1) return WICK_EINVAL;
    std::vector<ContractTable> tabs(n_tables);
    for (int k = 0; k < n_tables; ++k) {
        int n_blk = 0;
        if (!tables[k]) return WICK_EINVAL;
        err = terms_table(tables[k], &tabs[k], &n_blk);
        if (err) return err;
        if (n_blk != plan.n_out) return WICK_EINVAL;  // reduced for another layout
        if (tabs[k].el_scale) return WICK_EINVAL;     // correlation-matrix tables: wick_contract only
    }
    const wick_tuning tune = current_tuning();
    int rs = tune.range_sites;
    const bool tc = precision == WICK_MIXED && tc_applicable(plan);
    int group = 1;
    size_t pbytes = block_partial_bytes(plan, (int)V, (int)n_slices, precision, rs), cbytes = 0;
    if (tc) {
        const size_t per_cfg = tc_partial_bytes(plan, (int)V, (int)n_slices, 1, rs);
        group = (int)std::max<size_t>(1, std::min<size_t>(kGroupBytes / per_cfg, (size_t)tc_max_configs()));
        group = std::min(group, n_cfg);
        while ((int64_t)group * n_slices > 65535) --group;
        // one range size for the scratch and every launch (a last, smaller group keeps it)
        rs = tc_range_for(plan, rs, 1, group, (int)n_slices, (int)V);
        pbytes = tc_partial_bytes(plan, (int)V, (int)n_slices, group, rs);
        cbytes = tc_counter_bytes(plan, (int)n_slices, group);
    }
    const size_t bbytes = cbytes + pbytes;   // counters first (256-byte multiple), then partials
    ContractPlan cplan;
    err = contract_plan(plan.n_out, n_cfg, (int)n_slices, tabs.data(), n_tables, precision, contract_tune(tune),
                        INT64_MAX, &cplan);
    if (err) return err;
    wick_batch *bt = new (std::nothrow) wick_batch();
    if (!bt) return WICK_ENOMEM;
    auto fail = [&](int e) {
        if (bt->exec) cudaGraphExecDestroy(bt->exec);
        if (bt->graph) cudaGraphDestroy(bt->graph);
        cudaFree(bt->block_scratch);
        cudaFree(bt->contract_scratch);
        delete bt;
        (void)cudaGetLastError();
        return e;
    };
    if (dev_malloc((void **)&bt->block_scratch, bbytes) != WICK_OK ||
        dev_malloc((void **)&bt->contract_scratch, cplan.counter_bytes + cplan.partial_bytes + cplan.convert_bytes) !=
            WICK_OK)
        return fail(WICK_ENOMEM);
    if (cudaMemset(bt->block_scratch, 0, bbytes) != cudaSuccess ||
        cudaMemset(bt->contract_scratch, 0, cplan.counter_bytes + cplan.partial_bytes + cplan.convert_bytes) !=
            cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess)
        return fail(WICK_ECUDA);
    unsigned char *bsc = static_cast<unsigned char *>(bt->block_scratch);
    unsigned char *csc = static_cast<unsigned char *>(bt->contract_scratch);
    int serr = WICK_OK;
    int *status = status_word(&serr);  // the device status word exists before capture (kernels report timeouts there)
    if (serr) return fail(serr);
    cudaStream_t cap;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return fail(WICK_ECUDA);
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        cudaStreamDestroy(cap);
        return fail(WICK_ECUDA);
    }
    const size_t blk_stride = (size_t)n_slices * plan.n_out;
    int launch_err = WICK_OK;
    if (tc) {
        std::vector<const void *> su(n_cfg), sd(n_cfg);
        for (int c = 0; c < n_cfg; ++c) {
            su[c] = Su[c].data;
            sd[c] = Sd[c].data;
        }
        for (int c0 = 0; c0 < n_cfg && !launch_err; c0 += group) {
            const int gn = std::min(group, n_cfg - c0);
            launch_err = launch_block_tc(plan, su.data() + c0, sd.data() + c0, gn, dtype, (int)V, (int)n_slices, rs,
                                         (int *)bsc, (double2 *)(bsc + cbytes),
                                         (double2 *)blocks + (size_t)c0 * blk_stride, status, cap);
            bt->n_launches += 1;
        }
    } else {
        for (int c = 0; c < n_cfg && !launch_err; ++c) {
            launch_err = launch_block_build(plan, Su[c].data, dtype, Sd[c].data, dtype, (int)V, (int)n_slices,
                                            precision, rs, nullptr, bsc, (double2 *)blocks + (size_t)c * blk_stride,
                                            cap);
            bt->n_launches += block_build_launches(plan, precision);
        }
    }
    if (!launch_err) {
        launch_err = launch_contract((const double2 *)blocks, plan.n_out, n_cfg, (int)n_slices, tabs.data(), n_tables,
                                     precision, cplan, csc, (double2 *)(csc + cplan.counter_bytes), (double2 *)C_out,
                                     cap, nullptr,
                                     cplan.convert_bytes ? csc + cplan.counter_bytes + cplan.partial_bytes : nullptr);
        bt->n_launches += cplan.convert_bytes ? 2 : 1;   // the block conversion, then the contraction
    }
    const cudaError_t ec = cudaStreamEndCapture(cap, &bt->graph);
    cudaStreamDestroy(cap);
    if (launch_err) return fail(launch_err);
    if (ec != cudaSuccess) return fail(WICK_ECUDA);
    if (cudaGraphInstantiate(&bt->exec, bt->graph, 0) != cudaSuccess) return fail(WICK_ECUDA);
    *out = bt;
    return WICK_OK;
}

extern "C" int wick_batch_run(wick_batch *b, wick_stream_t stream) {
    if (!b || !b->exec) return WICK_EINVAL;
    WICK_CUDA_TRY(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    return WICK_OK;
}

extern "C" int wick_batch_launches(const wick_batch *b) { return b ? b->n_launches : WICK_EINVAL; }

extern "C" void wick_batch_free(wick_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->block_scratch);
    cudaFree(b->contract_scratch);
    delete b;
}
