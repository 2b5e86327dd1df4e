// Batched executor: many configurations x many nuclei in one CUDA graph.
//
// wick_batch_create records, for fixed device buffers, the block build of
// every configuration (Eq. 2.4/2.5) followed by the contraction of every
// reduced table against those blocks (Eq. 2.6 / App. D), captured on a
// private stream and instantiated once.  Nuclei built from the same nucleon
// operators share one block build per configuration.  The batch owns its
// scratch (block partials, contraction partials), so the graph never depends
// on the library's shared workspace.  wick_batch_run launches the graph on a
// stream: one host call per batch, every kernel in stream order on the device.
#include <vector>

#include "common.cuh"

struct wick_batch {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    void *block_partials = nullptr;
    void *contract_partials = nullptr;
    int n_launches = 0;
};

namespace wick {
int terms_view(const wick_terms *t, int *A, int64_t *U, int *n_blk, const uint16_t **ids, const int64_t **w,
               double *scale);
}

extern "C" int wick_batch_create(const wick_prop *Su, const wick_prop *Sd, int n_cfg, const wick_nucleon_op *ops,
                                 const wick_block_layout *layout, const wick_terms *const *tables, int n_tables,
                                 int precision, void *blocks, void *C_out, wick_batch **out) {
    using namespace wick;
    if (!out) return WICK_EINVAL;
    *out = nullptr;
    if (!Su || !Sd || n_cfg < 1 || !tables || n_tables < 1 || !blocks || !C_out) return WICK_EINVAL;
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
    struct TV { int A, n_blk; int64_t U; const uint16_t *ids; const int64_t *w; double scale; };
    std::vector<TV> tv(n_tables);
    for (int k = 0; k < n_tables; ++k) {
        if (!tables[k]) return WICK_EINVAL;
        err = terms_view(tables[k], &tv[k].A, &tv[k].U, &tv[k].n_blk, &tv[k].ids, &tv[k].w, &tv[k].scale);
        if (err) return err;
        if (tv[k].n_blk != plan.n_out) return WICK_EINVAL;  // reduced for another layout
    }
    int n_splits = 0, chunk = 0;
    const size_t pbytes = block_partials_bytes(plan, (int)V, (int)n_slices, precision, &n_splits, &chunk);
    size_t cbytes = 16;
    std::vector<int> n_chunks(n_tables);
    for (int k = 0; k < n_tables; ++k) {
        const size_t b = contract_partials_bytes((int)n_slices, tv[k].U, tv[k].A, tv[k].n_blk, &n_chunks[k]);
        cbytes = b > cbytes ? b : cbytes;
    }
    wick_batch *bt = new (std::nothrow) wick_batch();
    if (!bt) return WICK_ENOMEM;
    auto fail = [&](int e) {
        if (bt->exec) cudaGraphExecDestroy(bt->exec);
        if (bt->graph) cudaGraphDestroy(bt->graph);
        cudaFree(bt->block_partials);
        cudaFree(bt->contract_partials);
        delete bt;
        (void)cudaGetLastError();
        return e;
    };
    if (cudaMalloc(&bt->block_partials, pbytes) != cudaSuccess ||
        cudaMalloc(&bt->contract_partials, cbytes) != cudaSuccess)
        return fail(WICK_ENOMEM);
    int serr = WICK_OK;
    (void)status_word(&serr);  // the device status word exists before capture (kernels report timeouts there)
    if (serr) return fail(serr);
    cudaStream_t cap;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return fail(WICK_ECUDA);
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        cudaStreamDestroy(cap);
        return fail(WICK_ECUDA);
    }
    const size_t blk_stride = (size_t)n_slices * plan.n_out;
    int launch_err = WICK_OK;
    for (int c = 0; c < n_cfg && !launch_err; ++c) {
        double2 *bc = (double2 *)blocks + (size_t)c * blk_stride;
        launch_err = launch_block_build(plan, Su[c].data, dtype, Sd[c].data, dtype, (int)V, (int)n_slices, precision,
                                        (double *)bt->block_partials, n_splits, chunk, bc, cap);
        bt->n_launches += block_build_launches(plan, precision);
        for (int k = 0; k < n_tables && !launch_err; ++k) {
            double2 *co = (double2 *)C_out + ((size_t)c * n_tables + k) * n_slices;
            launch_err = launch_contract(bc, (int)n_slices, tv[k].n_blk, tv[k].A, tv[k].U, tv[k].ids, tv[k].w,
                                         tv[k].scale, precision, co, (double *)bt->contract_partials, n_chunks[k], cap);
            bt->n_launches += 2;
        }
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
    cudaFree(b->block_partials);
    cudaFree(b->contract_partials);
    delete b;
}
