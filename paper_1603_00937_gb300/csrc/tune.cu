// Autotuner of the batched tensor-core squaring: every built launch configuration of a
// state's precision (K-chunk width x operand-ring depth x tile schedule) is timed on the caller's own
// problem, and the fastest is installed and cached in the context by state shape.
//
// All candidates replay one branch sequence (fixed by a first run with the caller's
// parameters), so each does the same squarings; times are CUDA-event means over `reps`
// runs after two untimed runs (the second captures the run's CUDA graphs).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>

#include "devmem.h"
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
    GBE_TRY(gbe_check_device_csr(ctx, H, "gbe_sp2_autotune H"));
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

// ----------------------------------------------------------------------------- partition size
namespace {

// Modelled squaring time of one SP2 step (microseconds on the whole GPU) for the subgraph
// sizes of a partition.
//  Tensor-core paths: every upper 128 x 128 tile costs max(E, C ceil(m_s / 32)) on one SM,
//  the epilogue (E: TMEM read-out, split and stores of the tile) overlapping the MMAs of
//  the next tile (C per 32-column K-chunk).  E = 7.5 us and C = 0.6 us (FP16X6; C halves with
//  BF16X3's 3 products) are fitted to GB300 launches of the 32^3 lattice with cores of 64
//  sites (5120 tiles of 15 chunks: 0.345 ms) and of 8 sites (12288 tiles of 6 chunks:
//  0.696 ms), both 152 SMs.
//  FP64 path: the FP64 pipe's flops, 2 * 64^2 * K per upper 64 x 64 tile with K in steps of
//  16, at 1.2 TFLOP/s.
double step_time_us(int prec, int sm_count, const std::vector<int64_t>& sub_ptr) {
    double t = 0.0;
    for (size_t s = 0; s + 1 < sub_ptr.size(); ++s) {
        const double m = (double)(sub_ptr[s + 1] - sub_ptr[s]);
        if (prec == GBE_PREC_FP64) {
            const double T = std::ceil(m / 64.0), k = 16.0 * std::ceil(m / 16.0);
            t += 2.0 * 64.0 * 64.0 * k * T * (T + 1.0) / 2.0 / 1.2e6;   // flops / (1.2e12 / 1e6)
        } else if (prec == GBE_PREC_FP64TC) {
            // 18 products per K-chunk (three times FP16X6's six) and an epilogue that does not
            // overlap the MMAs (the four accumulators fill the TMEM)
            const double T = std::ceil(m / 128.0), nk = std::ceil(m / 32.0);
            t += T * (T + 1.0) / 2.0 * (1.8 * nk + 10.0) / (double)sm_count;
        } else {
            const double T = std::ceil(m / 128.0), nk = std::ceil(m / 32.0);
            const double c = prec == GBE_PREC_FP16X6 ? 0.6 : 0.3;
            t += T * (T + 1.0) / 2.0 * std::max(7.5, c * nk) / (double)sm_count;
        }
    }
    return t;
}

}  // namespace

extern "C" int gbe_partition_autotune(gbe_ctx* ctx, const gbe_graph* S, const gbe_partition_params* params, int prec,
                                      const int32_t* candidates, int ncand, double* cost, int* best, gbe_parts** parts) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && S && params && candidates && cost && best && parts, "NULL argument");
    GBE_CHECK_ARG(ncand >= 1, "no candidates");
    GBE_CHECK_ARG(prec == GBE_PREC_FP64 || prec == GBE_PREC_FP16X6 || prec == GBE_PREC_BF16X3 || prec == GBE_PREC_FP64TC,
                  "unknown prec");
    GBE_CHECK_ARG(params->mode == GBE_PART_SPATIAL_CELLS || params->mode == GBE_PART_INDEX_BLOCKS, "partition mode");
    *parts = nullptr;
    *best = -1;
    gbe_parts* keep = nullptr;
    for (int i = 0; i < ncand; ++i) {
        gbe_partition_params p = *params;
        if (p.mode == GBE_PART_SPATIAL_CELLS)
            for (int d = 0; d < 3; ++d) p.ncell[d] = candidates[3 * i + d];
        else
            p.core_size = candidates[3 * i];
        gbe_parts* P = nullptr;
        const int r = gbe_partition(ctx, S, &p, &P);
        cost[i] = std::numeric_limits<double>::infinity();
        if (r == GBE_ECAPACITY) continue;   // infeasible candidate (a subgraph above max_sub)
        if (r != GBE_OK) {
            gbe_free_parts(keep);
            return r;
        }
        if (P->max_m > 8192) {   // beyond what the gather's hash table holds
            gbe_free_parts(P);
            continue;
        }
        cost[i] = step_time_us(prec, ctx->sm_count, P->h_sub_ptr);
        if (*best < 0 || cost[i] < cost[*best]) {
            gbe_free_parts(keep);
            keep = P;
            *best = i;
        } else {
            gbe_free_parts(P);
        }
    }
    if (!keep) {
        gbe_set_error("no candidate partition fits");
        return GBE_ECAPACITY;
    }
    *parts = keep;
    return GBE_OK;
}
