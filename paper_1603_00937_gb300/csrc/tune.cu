// Autotuner of the batched tensor-core squaring: every built launch configuration of a
// state's precision (K-chunk width x operand-ring depth x tile schedule) is timed on the caller's own
// problem, and the fastest is installed and cached in the context by state shape.
//
// All candidates replay one branch sequence (fixed by a first run with the caller's
// parameters), so each does the same squarings; times are CUDA-event means over `reps`
// runs after two untimed runs (the second captures the run's CUDA graphs).
#include <algorithm>
#include <cstring>

#include "gbe_internal.h"

namespace {

int timed_runs(gbe_ctx* ctx, const gbe_csr* H, const gbe_parts* parts, const gbe_sp2_params* prm, gbe_subs* X,
               int reps, float* ms) {
    // untimed: the first run of new inputs goes step by step, the second captures the graphs
    for (int i = 0; i < 2; ++i) GBE_TRY(gbe_sp2_run(ctx, H, parts, prm, X));
    GBE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GBE_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        gbe_set_error("cudaEventCreate failed");
        return GBE_ECUDA;
    }
    int r = GBE_OK;
    cudaEventRecord(e0, ctx->stream);
    for (int i = 0; i < reps && r == GBE_OK; ++i) r = gbe_sp2_run(ctx, H, parts, prm, X);
    cudaEventRecord(e1, ctx->stream);
    if (r == GBE_OK && cudaEventSynchronize(e1) != cudaSuccess) {
        gbe_set_error("autotune: timed runs failed: %s", cudaGetErrorString(cudaGetLastError()));
        r = GBE_ECUDA;
    }
    float t = 0.f;
    if (r == GBE_OK) cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != GBE_OK) return r;
    gbe_sp2_report rp;
    GBE_TRY(gbe_sp2_report_get(ctx, X, &rp));
    if (rp.status != GBE_OK) {
        gbe_set_error("autotune: the device recorded error %d", rp.status);
        return rp.status;
    }
    *ms = t / (float)reps;
    return GBE_OK;
}

}  // namespace

extern "C" int gbe_sp2_autotune(gbe_ctx* ctx, const gbe_csr* H, const gbe_parts* parts, const gbe_sp2_params* prm,
                                gbe_subs* X, int reps, gbe_tune_report* rep) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && H && parts && prm && X && rep, "NULL argument");
    GBE_CHECK_ARG(reps >= 1 && reps <= 1000, "reps must be in 1..1000");
    GBE_CHECK_ARG(H->on_device, "gbe_sp2_autotune needs a device CSR");
    GBE_CUDA_TRY(cudaSetDevice(ctx->device));
    memset(rep, 0, sizeof(*rep));

    // candidates: every ring depth the precision is built with x both schedules
    std::vector<gbe_tc_config> cand;
    if (X->prec == GBE_PREC_FP64) {
        cand.push_back(X->tc_cfg);
    } else {
        const std::vector<int64_t> key = gbe_subs_shape_key(ctx, X);
        for (const auto& kv : ctx->tune_cache)
            if (kv.first == key) {
                GBE_TRY(gbe_subs_apply_config(ctx, X, kv.second));
                rep->n = 1;
                rep->cand[0] = kv.second;
                rep->best = 0;
                rep->cached = 1;
                return GBE_OK;
            }
        for (int kc : {32, 16}) {
            int st[8];
            const int ns = gbe_tc_stage_options(X->prec, kc, st, 8);
            for (int i = 0; i < ns; ++i)
                for (int sched : {GBE_SCHED_ROUND_ROBIN, GBE_SCHED_BALANCED_RANGES})
                    if ((int)cand.size() < GBE_TUNE_MAX) cand.push_back(gbe_tc_config{st[i], sched, kc});
        }
    }

    // the branch sequence every candidate replays
    GBE_TRY(gbe_sp2_run(ctx, H, parts, prm, X));
    gbe_sp2_report base;
    GBE_TRY(gbe_sp2_report_get(ctx, X, &base));
    if (base.status != GBE_OK) {
        gbe_set_error("autotune: the first run recorded error %d", base.status);
        return base.status;
    }
    gbe_sp2_params p = *prm;
    p.branch_mode = GBE_BRANCH_REPLAY;
    p.seq_in = base.seq;
    p.seq_len = base.iters;
    p.fp64_tail = 0;
    p.n_max = std::max(p.n_max, base.iters);
    rep->iters = base.iters;

    int best = 0;
    for (size_t i = 0; i < cand.size(); ++i) {
        GBE_TRY(gbe_subs_apply_config(ctx, X, cand[i]));
        float ms = 0.f;
        GBE_TRY(timed_runs(ctx, H, parts, &p, X, reps, &ms));
        rep->cand[i] = cand[i];
        rep->ms[i] = ms;
        if (ms < rep->ms[best]) best = (int)i;
    }
    rep->n = (int)cand.size();
    rep->best = best;
    GBE_TRY(gbe_subs_apply_config(ctx, X, cand[best]));
    if (X->prec != GBE_PREC_FP64) {
        const std::vector<int64_t> key = gbe_subs_shape_key(ctx, X);
        bool stored = false;
        for (auto& kv : ctx->tune_cache)
            if (kv.first == key) { kv.second = cand[best]; stored = true; }
        if (!stored) ctx->tune_cache.emplace_back(key, cand[best]);
    }
    return GBE_OK;
}
