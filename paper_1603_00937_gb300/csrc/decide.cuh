// The SP2 step decision (global FP64 traces over core positions -> stop rule and branch of
// the next step).  Every path (a single rank's partials, a sharded run's exchanged sums)
// reduces in the same order with 256 threads, so all take the same decisions bit for bit.
#pragma once
#include <cmath>

#include "gbe_internal.h"

constexpr int kDecideThreads = 256;

struct DecideIn {
    const double* partials;
    int max_units;
    const int2* ranges;   // [P] work units of each subgraph for this kind
    int P;
    const double* sums;   // exchanged sums [2 P_global + 1], or NULL
    int64_t P_global;
    int kind;             // 0 after the gather, 1 after a tensor-core step, 2 after an FP64 step
};

// Trace sums of one subgraph over its work units, in unit order (the same arithmetic in a
// single-rank decision and in the per-subgraph sums a sharded run exchanges).
__device__ __forceinline__ void sub_trace(const double* __restrict__ partials, int max_units, int2 r, double& a,
                                          double& b) {
    double x = 0.0, y = 0.0;
    for (int u = r.x; u < r.x + r.y; ++u) {
        x += partials[u];
        y += partials[max_units + u];
    }
    a = x;
    b = y;
}

__device__ __forceinline__ double warp_sum_dd(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Thread t (of kDecideThreads) of the decision: its share of the two traces (subgraphs
// t, t + 256, ... in order), then the block sum through `bar` (a barrier over the 256
// threads), valid in thread 0.
template <class Bar>
__device__ void decide_traces(const DecideIn& in, int t, double* red, Bar bar, double& t1, double& t2) {
    double a = 0.0, b = 0.0;
    if (in.sums) {
        for (int64_t g = t; g < in.P_global; g += kDecideThreads) {
            a += in.sums[g];
            b += in.sums[in.P_global + g];
        }
    } else {
        for (int s = t; s < in.P; s += kDecideThreads) {
            double x, y;
            sub_trace(in.partials, in.max_units, in.ranges[s], x, y);
            a += x;
            b += y;
        }
    }
    a = warp_sum_dd(a);
    b = warp_sum_dd(b);
    const int w = t >> 5, l = t & 31;
    bar();
    if (l == 0) { red[w] = a; red[8 + w] = b; }
    bar();
    if (w == 0) {
        a = warp_sum_dd(l < kDecideThreads / 32 ? red[l] : 0.0);
        b = warp_sum_dd(l < kDecideThreads / 32 ? red[8 + l] : 0.0);
    }
    t1 = a;
    t2 = b;
}

// The decision from the two global traces, by one thread.
__device__ inline void decide_apply(Sp2Ctrl* C, const DecideIn& in, double t1, double t2) {
    const int kind = in.kind;
    C->pending = 0;
    if (kind != 0) {
        const int n_prev = C->iter;
        C->seq[n_prev] = (uint8_t)C->branch;
        C->iter = n_prev + 1;
        C->cur ^= 1;
        C->fmt = (kind == 2) ? 1 : 0;
        if (kind == 2) C->fp64_iters++;
    }
    const int n = C->iter;
    C->t1[n] = t1;
    C->t2[n] = t2;
    if (in.sums && in.sums[2 * in.P_global] != 0.0 && C->status == GBE_OK) C->status = GBE_EPEER;
    if (C->status != GBE_OK || !isfinite(t1) || !isfinite(t2)) {
        if (C->status == GBE_OK) C->status = GBE_ENUMERIC;
        C->stop = GBE_STOP_ERROR;
        return;
    }
    const double e = fabs(t1 - t2);
    const bool mixed = (C->prec == GBE_PREC_FP16X6 || C->prec == GBE_PREC_BF16X3);   // FP64TC is FP64-grade
    if (C->branch_mode == GBE_BRANCH_REPLAY) {
        if (n >= C->seq_len || n >= C->n_max) { C->stop = GBE_STOP_REPLAY; return; }
        C->branch = C->seq_in[n] ? 1 : 0;
        if (mixed && C->mode == 0 && n >= C->seq_len - C->fp64_tail) { C->mode = 1; C->switch_iter = n; }
        return;
    }
    const bool stalled = (n >= C->n_min && n >= 2 && e >= fabs(C->t1[n - 2] - C->t2[n - 2]));
    if (mixed && C->mode == 0 && C->fp64_tail > 0) {
        if (e <= C->tail_switch || e <= C->idem_tol || stalled) { C->mode = 1; C->switch_iter = n; }
    } else {
        const int since = (C->switch_iter >= 0) ? n - C->switch_iter : n;
        const bool tail_done = !mixed || C->fp64_tail == 0 || since >= C->fp64_tail;
        const bool stall_ok = (C->switch_iter < 0) || (since >= 2);
        if (e <= C->idem_tol && tail_done) { C->stop = GBE_STOP_TOL; return; }
        if (stalled && stall_ok && tail_done) { C->stop = GBE_STOP_STALL; return; }
    }
    if (n >= C->n_max) { C->stop = GBE_STOP_NMAX; return; }
    C->branch = (fabs(t2 - C->n_occ) < fabs(2.0 * t1 - t2 - C->n_occ)) ? 1 : 0;
}

// The last step of a loop body's decision in a graph-launched run: the loop node's condition
// (continue while the run has not stopped, and never beyond n_max + 8 iterations).
__device__ inline void decide_set_condition(Sp2Ctrl* C, cudaGraphConditionalHandle cond) {
    if (++C->loops > C->n_max + 8 && C->stop == 0) C->stop = GBE_STOP_NMAX;
    cudaGraphSetConditional(cond, C->stop == 0 ? 1u : 0u);
}
