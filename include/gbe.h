/*
 * gbe.h -- C ABI of libgbe: graph-partitioned SP2 density matrices on one GB300.
 *
 * The library computes the zero-temperature density matrix D = theta(mu I - H) of a
 * sparse Hamiltonian H with the graph-based method of Niklasson et al., "Graph-based
 * linear scaling electronic structure theory" (Sec. II.A): a data-dependency graph
 * S_tau (Eq. 2, Eq. 8) is cut into cores (communities, observation vi); every
 * core+halo subgraph s gives a small dense principal submatrix x[s] of
 * X_0 = (e_max I - H)/(e_max - e_min); one global SP2 recursive expansion
 * (X <- X^2 or 2X - X^2, the second-order recursion the paper uses) runs on all
 * submatrices at once; core columns are collected into D column by column (Eq. 6,
 * observation i).
 *
 * Conventions for every entry point
 *   - Return value: GBE_OK (0) or a negative GBE_E* code; gbe_strerror() names it.
 *     gbe_last_error_message() returns a thread-local detail string for the last error.
 *   - Work is ordered on the context's CUDA stream.  Entry points that return sizes or
 *     reports to the host synchronise that stream; the others only enqueue.
 *   - Pointers marked "device" must be device memory of the context's GPU; "host" means
 *     host memory; structs carrying an on_device flag accept either.
 *   - Inputs are borrowed for the duration of the call (and, for enqueue-only calls,
 *     until the stream reaches the enqueued work).  Opaque objects are owned by the
 *     library and released with the matching gbe_free_* call.  Output buffers in
 *     gbe_ell are owned by the caller.
 *   - There is no CPU fallback: without a usable sm_103 GPU, gbe_create returns
 *     GBE_ENODEV and every other call GBE_EINVAL on a NULL context.
 *   - Device-side waits are bounded; a wait that runs out reports GBE_ETIMEOUT and the
 *     context remains usable.
 *
 * Two tuners sit beside the method (neither is in the paper): gbe_sp2_autotune picks the
 * launch configuration of the batched squaring on the caller's problem (results are bit
 * for bit the same under every configuration), and gbe_partition_autotune picks the
 * partition size by a cost model of these kernels (a different partition changes D within
 * the truncation error of the graph, which Sec. II.B finds fairly insensitive to the
 * number of communities).
 */
#ifndef GBE_H
#define GBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GBE_OK          0
#define GBE_EINVAL     -1   /* bad argument, size or state                        */
#define GBE_ENOMEM     -2   /* device or host allocation failed                   */
#define GBE_ECUDA      -3   /* a CUDA runtime / driver call failed                */
#define GBE_ETIMEOUT   -4   /* a bounded device-side wait gave up                 */
#define GBE_ENOCONV    -5   /* SP2 reached n_max without meeting its stop rule    */
#define GBE_ENUMERIC   -6   /* NaN or Inf met in H or in an SP2 iterate           */
#define GBE_ECAPACITY  -7   /* a subgraph, ELL row or table exceeded its capacity */
#define GBE_ENODEV     -8   /* no usable sm_103 device                            */
#define GBE_EPEER      -9   /* another rank of a sharded run reported an error    */

typedef struct gbe_ctx gbe_ctx;
typedef struct gbe_graph gbe_graph;
typedef struct gbe_parts gbe_parts;
typedef struct gbe_subs gbe_subs;
typedef struct gbe_hamiltonian gbe_hamiltonian;

/* Sparse symmetric H in CSR: rows [0, n); column indices ascending within a row;
 * the diagonal entry of every row present.  rowptr[n+1] int64, col[nnz] int32,
 * val[nnz] float64.  on_device = 1: device pointers; 0: host pointers (copied in).
 * Arrays flagged on_device = 1 that are not device (or managed) memory of the context's
 * GPU are refused with GBE_EINVAL before any launch, here and in gbe_ell and gbe_sites. */
typedef struct {
    int64_t n, nnz;
    const int64_t* rowptr;
    const int32_t* col;
    const double* val;
    int on_device;
} gbe_csr;

/* Density matrix in ELLPACK, caller-owned: row i holds column i of D (the column
 * collection order of Eq. 6 / observation i).  col[n*width] int32, val[n*width]
 * float64, row-major; entries of a row are packed from the front, padding has
 * col = -1 and val = 0.  on_device selects device (1) or host (0) buffers. */
typedef struct {
    int64_t n, width;
    int32_t* col;
    double* val;
    int on_device;
} gbe_ell;

/* Sites of the tight-binding workload: pos[n][3] float64 inside [0, box), onsite[n]. */
typedef struct {
    int64_t n;
    const double* pos;
    const double* onsite;
    double box[3];
    int on_device;
} gbe_sites;

/* H_ij = hop * exp(-(r - a)/(decay)) for 0 < r < rcut (minimum image), H_ii = onsite. */
typedef struct {
    double a, rcut, decay, hop;
} gbe_tb_model;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`, ordering work on `cuda_stream`
 * (a cudaStream_t; NULL selects the legacy default stream).  Fails with GBE_ENODEV
 * when the device is absent or is not compute capability 10.3.  The context calls and
 * the error calls below are runtime with no counterpart in the paper. */
int gbe_create(gbe_ctx** ctx, int device, void* cuda_stream);
int gbe_destroy(gbe_ctx* ctx);
/* Change the stream later calls are ordered on (runtime; no counterpart in the paper).  Device memory of objects created
 * before the change stays ordered on the stream it was allocated on, and is released on
 * that stream when the object is freed: keep that stream alive until then. */
int gbe_set_stream(gbe_ctx* ctx, void* cuda_stream);
/* Profiling switch (runtime; no counterpart in the paper): when on, gbe_sp2_run records a CUDA event pair around every
 * squaring launch on the context stream and gbe_sp2_report_get sums the durations of
 * the launches that did work (ms_tc / n_tc, ms_fp64 / n_fp64). */
int gbe_set_profiling(gbe_ctx* ctx, int on);
/* Launch each SP2 run as two CUDA graphs (runtime; not in the paper; default on): the prologue (control block,
 * spectral bounds, gather, first decision) and a loop node whose body is one SP2 step,
 * repeated on the device while the run's own decision says continue, so exactly the steps
 * a run needs are executed and no host round trip is involved.  The graphs are captured on
 * the first run and relaunched while parameters and inputs (pointers, sizes) are unchanged.
 * Profiling (gbe_set_profiling) launches step by step instead, to time every squaring. */
int gbe_set_graph_launch(gbe_ctx* ctx, int on);
/* Number of SMs of the context's device (grids are sized from it; no counterpart in the paper).
 * gbe_strerror names a return code; gbe_last_error_message gives the calling thread's last
 * error detail (thread-local). */
int gbe_device_sm_count(const gbe_ctx* ctx);
const char* gbe_strerror(int code);
const char* gbe_last_error_message(void);

/* --------------------------------------------------------- Hamiltonian (a1) */

/* Build CSR H from sites with a cell list on the GPU (workload model; the paper's
 * SCC-DFTB H of Sec. II.B is not reproduced).  Output is library-owned device CSR;
 * gbe_hamiltonian_csr() gives a device view of it.  Synchronises (reads nnz). */
int gbe_build_hamiltonian(gbe_ctx* ctx, const gbe_sites* sites, const gbe_tb_model* model,
                          gbe_hamiltonian** H);
int gbe_hamiltonian_csr(const gbe_hamiltonian* H, gbe_csr* view);
int gbe_free_hamiltonian(gbe_hamiltonian* H);

/* ------------------------------------------------------------- graph (a2) */

enum {
    GBE_GRAPH_H2_THRESH    = 0, /* edge if |(H^2)_ij| >= thresh                        Eq. 2 */
    GBE_GRAPH_D_THRESH     = 1, /* edge if |D_ij| >= thresh or |D_ji| >= thresh        Eq. 2 on a prior D */
    GBE_GRAPH_EQ8_SYMBOLIC = 2, /* paths of length <= 2 in pattern(floor(D)_thresh) u pattern(H)  Eq. 8, eps = 0 */
    GBE_GRAPH_HK_PATTERN   = 3, /* paths of length <= k in pattern(H)                  */
    GBE_GRAPH_MLP          = 4  /* edges scored by a trained gbe_mlp, union pattern(H) */
};

typedef struct gbe_mlp gbe_mlp;

typedef struct {
    int mode;                 /* GBE_GRAPH_* */
    double thresh;            /* tau (or the H^2 threshold)                            */
    int k;                    /* path length for GBE_GRAPH_HK_PATTERN                   */
    const gbe_ell* D_prev;    /* prior density matrix (D_THRESH, EQ8_SYMBOLIC)          */
    const gbe_sites* sites;   /* MLP mode: candidate pairs r < rcand                    */
    const gbe_mlp* mlp;       /* MLP mode: trained classifier                           */
    double rcand;             /* MLP mode: candidate radius (units of length)           */
    double logit_cut;         /* MLP mode: keep edges with logit >= logit_cut           */
} gbe_graph_params;

/* Build S_tau on the GPU (Sec. II.A: Eq. 2 on H^2 or on a prior D, Eq. 8 in its symbolic
 * form, the pattern of H^k, or the learned proposal).  The graph is undirected, contains every diagonal entry, and
 * is held either explicitly (CSR) or as "base pattern A with path length k", meaning
 * S = pattern(A^k); partitioning expands core sets by k hops directly.  `H` is a
 * device or host CSR.  Synchronises. */
int gbe_build_graph(gbe_ctx* ctx, const gbe_csr* H, const gbe_graph_params* params, gbe_graph** S);
/* Materialise the explicit CSR of S_tau (Eq. 2; no-op for k = 1) and report its size. */
int gbe_graph_size(gbe_ctx* ctx, gbe_graph* S, int64_t* n, int64_t* nnz);
/* Copy the explicit CSR of S_tau (Eq. 2) to host arrays rowptr[n+1] (int64) and col[nnz] (int32). */
int gbe_graph_export(gbe_ctx* ctx, gbe_graph* S, int64_t* rowptr, int32_t* col);
int gbe_free_graph(gbe_graph* S);

/* --------------------------------------------------------- partition (a3) */

enum {
    GBE_PART_SPATIAL_CELLS = 0, /* cores = non-empty cells floor(x / box * ncell), ascending cell id */
    GBE_PART_INDEX_BLOCKS  = 1  /* cores = consecutive blocks of core_size vertices              */
};

typedef struct {
    int mode;
    int ncell[3];                /* SPATIAL_CELLS */
    const gbe_sites* sites;      /* SPATIAL_CELLS */
    int core_size;               /* INDEX_BLOCKS  */
    int max_sub;                 /* capacity of one core+halo subgraph (0: library default 4096) */
} gbe_partition_params;

/* Cut S into cores (communities, observation vi) and build each core+halo subgraph
 * (Sec. II.A, Fig. 1): local index list = core vertices ascending, then halo vertices
 * (neighbours of any core vertex, not in the core) ascending.  Synchronises (subgraph
 * sizes size every later buffer).  GBE_ECAPACITY when a subgraph exceeds max_sub. */
int gbe_partition(gbe_ctx* ctx, const gbe_graph* S, const gbe_partition_params* params,
                  gbe_parts** parts);
/* Cost-driven choice of the partition size (Sec. II.B: the error hardly depends on the number
 * of communities while the cost varies strongly with it, and an optimised partitioning
 * brings it down; Sec. III: adjust the partitioning to the computational platform).  Each
 * candidate replaces params->ncell (GBE_PART_SPATIAL_CELLS: candidates[3 i .. 3 i + 2]) or
 * params->core_size (GBE_PART_INDEX_BLOCKS: candidates[3 i]) and is partitioned with
 * gbe_partition; its cost is a model of the squaring time of one SP2 step on this
 * library's kernels for precision `prec`, in microseconds: GBE_PREC_FP16X6 / BF16X3 sum
 * over subgraphs of T_s (T_s + 1) / 2 upper tiles (T_s = ceil(m_s / 128)) times
 * max(7.5, c ceil(m_s / 32)) / (number of SMs), c = 0.6 (FP16X6) or 0.3 (BF16X3): a tile's
 * epilogue against its MMAs, fitted to GB300 runs; GBE_PREC_FP64 the FP64 flops
 * 2 x 64^2 x 16 ceil(m_s / 16) per upper 64 x 64 tile at 1.2 TFLOP/s.  A candidate whose
 * partition fails (a subgraph above max_sub or above the 8192 vertices the gather holds)
 * costs +inf; any other error of gbe_partition (an invalid candidate) is returned.
 * cost[ncand] receives the costs, *best the index of the cheapest and *parts its partition
 * (library-owned; NULL and GBE_ECAPACITY when every candidate failed).  Not in the paper as
 * an algorithm: the paper uses METIS with a chosen number of communities. */
int gbe_partition_autotune(gbe_ctx* ctx, const gbe_graph* S, const gbe_partition_params* params, int prec,
                           const int32_t* candidates, int ncand, double* cost, int* best, gbe_parts** parts);
/* Sizes of the core+halo subgraphs (Sec. II.A, Fig. 1): number P, total local indices, max size. */
int gbe_parts_info(const gbe_parts* parts, int64_t* P, int64_t* total, int64_t* max_m);
/* Copy the subgraphs (Sec. II.A, Fig. 1) to host: core_count[P] int32, sub_ptr[P+1] int64,
 * sub_idx[total] int32. */
int gbe_parts_export(gbe_ctx* ctx, const gbe_parts* parts, int32_t* core_count, int64_t* sub_ptr,
                     int32_t* sub_idx);
/* Build a partition from host arrays with the same meaning (core vertices first in
 * each list; any communities, obs. vi).  Validates ranges; does not check that the lists match any graph. */
int gbe_parts_import(gbe_ctx* ctx, int64_t n, int64_t P, const int32_t* core_count,
                     const int64_t* sub_ptr, const int32_t* sub_idx, gbe_parts** parts);
int gbe_free_parts(gbe_parts* parts);

/* ------------------------------------------- several GPUs: subgraphs sharded over ranks */

/* Assignment of the subgraphs of one partition to `world` ranks (host only, no GPU needed).
 * The subgraph expansions are independent (Sec. II.A, after Eq. 6; the paper spreads them
 * over 1, 16 and 32 GPUs, Sec. II.B), so each rank squares only its own subgraphs.  The
 * cost of subgraph s is m_s^3 (its dense squaring, the cost model of Sec. II.B) with
 * m_s = sub_ptr[s+1] - sub_ptr[s]; subgraphs are taken largest cost first (ties: lower
 * index first) and each goes to the rank with the smallest load so far (ties: lower rank)
 * -- greedy longest-processing-time, deterministic, the same on every rank.
 *   sub_ptr: host int64[P+1]; owner: host int32[P] receives the rank of each subgraph;
 *   load: host double[world] (nullable) receives the summed cost per rank.
 * GBE_EINVAL for P < 1, world < 1 or an empty subgraph. */
int gbe_shard_assign(int64_t P, const int64_t* sub_ptr, int world, int32_t* owner, double* load);

/* The shard of a partition that `rank` owns (the independent subgraph expansions of
 * Sec. II.A spread over GPUs as in Sec. II.B): its subgraphs (owner[s] == rank) in their
 * global order, as a partition of the same n vertices that remembers the global index of
 * each subgraph.  An SP2 run on a shard squares only these subgraphs; its traces are
 * combined with the other ranks' through gbe_sp2_params.exchange (global-trace mode) and
 * its assembly fills only the ELL rows of its own cores (the other rows are emptied).
 *   owner: host int32[P] (gbe_shard_assign or any other assignment); a rank that owns no
 *   subgraph gets GBE_EINVAL.  *local: library-owned, freed with gbe_free_parts; `parts`
 *   may be freed after the call. */
int gbe_parts_shard(gbe_ctx* ctx, const gbe_parts* parts, const int32_t* owner, int rank, gbe_parts** local);

/* Trace exchange of a sharded SP2 run.  Called by gbe_sp2_run on the calling thread, once
 * after the gather and once after every SP2 step in global-trace mode (never in replay
 * mode: a pre-determined sequence needs no exchange, Sec. II.C).  `buf` is device memory of
 * `count` doubles: this rank's per-subgraph trace sums at the global positions of its
 * subgraphs, zeros elsewhere, and an error flag in the last element.  The function must
 * replace buf by its element-wise sum over all ranks, ordered on `stream` (a cudaStream_t):
 * either by enqueuing an all-reduce on that stream (NCCL), or by synchronising the stream,
 * exchanging on the host and copying the sum back before it returns.  Every position has
 * one contributing rank, so the sum is exact whatever the reduction order, and every rank
 * takes the same branch decisions as a single-rank run of the whole partition.  Return 0
 * on success; anything else stops the run with GBE_EPEER. */
typedef int (*gbe_exchange_fn)(void* user, double* buf, int64_t count, void* stream);

/* ------------------------------------------------------ SP2 (a4 - a7) */

enum {
    GBE_PREC_FP64    = 0, /* every squaring in FP64 on the FP64 pipe                          */
    GBE_PREC_FP16X6  = 1, /* tensor cores: 3-level fp16 split, 6 products, FP32 accumulation,
                             exact accumulation of the fixed-point leading part               */
    GBE_PREC_BF16X3  = 2, /* tensor cores: per-element bf16 hi/lo split, 3 products            */
    GBE_PREC_FP64TC  = 3  /* tensor cores at FP64 grade: x held to 2^-50 as five fixed-point
                             fp16 slices (an Ozaki-type slicing; not in the paper), 18 fp16
                             products in four FP32 accumulators, the three leading ones exact */
};

enum {
    GBE_BRANCH_GLOBAL_TRACE = 0, /* branch from the global FP64 traces every iteration     */
    GBE_BRANCH_REPLAY       = 1  /* apply seq_in[0..seq_len) and stop after it; seq_len
                                    above n_max is rejected (GBE_EINVAL)                   */
};

enum {
    GBE_STOP_NONE = 0, GBE_STOP_TOL = 1, GBE_STOP_STALL = 2, GBE_STOP_NMAX = 3,
    GBE_STOP_REPLAY = 4, GBE_STOP_ERROR = 5
};

#define GBE_SEQ_MAX 256

typedef struct {
    double n_occ;          /* total occupation summed over all core positions (half filling: N/2) */
    double idem_tol;       /* stop when e_n = |Tr X_n - Tr X_n^2| <= idem_tol (core positions)      */
    int n_min;             /* stall rule active from this iteration on (e_n >= e_{n-2} stops)       */
    int n_max;             /* at most this many squarings (<= GBE_SEQ_MAX)                          */
    int prec;              /* GBE_PREC_*                                                            */
    int fp64_tail;         /* mixed precision: replay mode runs the last fp64_tail steps in FP64;
                              global mode switches to FP64 when e_n <= tail_switch or the mixed
                              iteration stalls, for at least fp64_tail further steps            */
    double tail_switch;    /* see fp64_tail (global mode)                                         */
    int branch_mode;       /* GBE_BRANCH_*                                                          */
    const uint8_t* seq_in; /* host; 1 = X^2, 0 = 2X - X^2 (replay mode)                             */
    int seq_len;
    int eps_given;         /* 1: use eps_min / eps_max below instead of Gershgorin bounds           */
    double eps_min, eps_max;
    double timeout_ms;     /* bound for device-side waits (0: library default, 2000 ms)             */
    /* sharded runs (parts from gbe_parts_shard): the trace exchange between ranks; NULL for a
       run on a whole partition.  A run with an exchange is launched step by step (never as a
       CUDA graph) and reads the stop flag back after every step, so that all ranks stop
       after the same step and make the same number of exchanges. */
    gbe_exchange_fn exchange;
    void* exchange_user;
} gbe_sp2_params;

typedef struct {
    int iters;             /* squarings performed                                      */
    int fp64_iters;        /* of which in FP64                                         */
    int stop_reason;       /* GBE_STOP_*                                               */
    int converged;         /* 1 when stopped by tolerance, stall or replay length      */
    int status;            /* GBE_OK or the error code the device recorded             */
    double eps_min, eps_max;
    double trace;          /* Tr over core positions of the final X                    */
    double idem_err;       /* e_n of the final X                                       */
    uint8_t seq[GBE_SEQ_MAX];
    double t1[GBE_SEQ_MAX + 1], t2[GBE_SEQ_MAX + 1];
    float ms_gather, ms_sp2;            /* CUDA-event times of the phases                */
    double mma_flops;      /* tensor-core flops issued (split products included)          */
    double alg_flops;      /* sum over iterations and subgraphs of 2 m_s^3                 */
    /* per-kernel CUDA-event times of the squaring launches that did work (filled only
       when profiling is on, see gbe_set_profiling) */
    float ms_tc, ms_fp64;
    int n_tc, n_fp64;
    double fp64_flops;     /* FP64 flops issued by the FP64 squarings                      */
} gbe_sp2_report;

/* Allocate the SP2 state for a partition and precision: the dense principal submatrices
 * x[s] of Eq. 6 (dense padded tiles in HBM,
 * ping-pong buffers, trace partials, device control block).  Reusable across calls.  A
 * mixed-precision state allocates its FP64 iterates only when a run first needs FP64 steps
 * (fp64_tail > 0); a state starts with the launch configuration the context's autotuner
 * cache holds for its shape, if any (gbe_sp2_autotune). */
int gbe_subs_create(gbe_ctx* ctx, const gbe_parts* parts, int prec, gbe_subs** X);
int gbe_free_subs(gbe_subs* X);

/* Enqueue one density-matrix build on the stream without synchronising: the recursive
 * expansion of Sec. II.A (SP2, X^2 or 2X - X^2) on every x[s] of Eq. 6.  With graph launch
 * on (gbe_set_graph_launch, the default) a state's second run with the same inputs and
 * parameters captures the run as two CUDA graphs and later such runs relaunch them; a first
 * run, or a run after a change, is launched kernel by kernel.  The build:
 * Gershgorin bounds of H (FP64, a4), gather + scale of every x[s] (a4), and the SP2
 * loop (a5 squarings, a6 global FP64 trace + branch, a7 branch apply in the squaring
 * epilogue), with convergence decided on the device.  `H` must be device CSR.
 * GBE_ECAPACITY (before any launch) when a subgraph has more than 8192 vertices: the
 * gather keeps an index hash table of the subgraph in one CTA's 227 KB of shared memory,
 * with the dense rows it stages beside it up to 2432 vertices and in global memory above
 * (the same bound applies to gbe_foe_run). */
int gbe_sp2_run(gbe_ctx* ctx, const gbe_csr* H, const gbe_parts* parts, const gbe_sp2_params* params,
                gbe_subs* X);
/* Synchronise and read the report of the last run on X (the traces and branch sequence of
 * the Sec. II.A recursion, timings, flops). */
int gbe_sp2_report_get(gbe_ctx* ctx, const gbe_subs* X, gbe_sp2_report* rep);

/* Replayed SP2 of a partition whose iterates need not fit the device together, and its D.
 * With a pre-determined branch sequence (Sec. II.C) no trace is shared between subgraphs,
 * and their expansions are independent (Sec. II.A, after Eq. 6), so they may run one batch
 * after another: the subgraphs are dealt to the fewest batches whose two ping-pong iterates
 * take at most budget_bytes each (gbe_shard_assign over the batches, largest m_s^3 first),
 * and each batch is created, runs gbe_sp2_run with `params` and writes the columns of its
 * own cores into D (Eq. 6) before it is freed.  D is as gbe_assemble_D fills it (device or
 * host ELL, width >= max m_s); *batches (nullable) receives the number of batches.  H must
 * be device CSR.  GBE_EINVAL unless params is in replay mode without an exchange;
 * GBE_ECAPACITY when one subgraph's iterates alone exceed the budget; the device status of
 * the first batch that recorded one (GBE_ENUMERIC for a non-finite H, GBE_ETIMEOUT), and
 * no further batch runs.  Synchronises. */
int gbe_sp2_replay_batched(gbe_ctx* ctx, const gbe_csr* H, const gbe_parts* parts, const gbe_sp2_params* params,
                           int64_t budget_bytes, double drop_tol, gbe_ell* D, int* batches);

/* gbe_sp2_run + gbe_sp2_report_get (Sec. II.A, Eq. 6).  *X NULL: allocate a new state; otherwise reuse it
 * (it must come from the same partition and precision).  H may be host CSR (copied in).
 * Returns GBE_ENOCONV when the run stopped at n_max, GBE_ENUMERIC / GBE_ETIMEOUT when
 * the device recorded one, GBE_OK otherwise. */
int gbe_sp2_submatrices(gbe_ctx* ctx, const gbe_csr* H, const gbe_parts* parts,
                        const gbe_sp2_params* params, gbe_subs** X, gbe_sp2_report* rep);

/* ------------------------------------------- launch configuration and autotuner */

/* Launch configuration of the tensor-core squaring that runs every submatrix of an SP2
 * step in one persistent launch (one CTA per SM):
 *   kchunk    columns of K one ring stage holds: 32 (or 0) or 16.  Half-width stages
 *             release their shared memory to the next copy twice as often, so the same
 *             bytes in flight cover more of the copy latency, at twice the barrier traffic
 *   stages    depth of the TMA operand ring (0: the default, 4 / 8 stages of 32 / 16
 *             columns for FP16X6 and 6 / 12 for BF16X3; FP16X6 is also built with 3 / 6,
 *             BF16X3 with 4, 7 / 14)
 *   schedule  how the upper-triangular 128 x 128 output tiles of all subgraphs (ordered
 *             subgraph by subgraph, largest first) are dealt to the CTAs:
 *             GBE_SCHED_ROUND_ROBIN    CTA b takes tiles b, b + grid, ... (the tiles of one
 *                                      subgraph run side by side on neighbouring CTAs)
 *             GBE_SCHED_BALANCED_RANGES CTA b takes one contiguous run of tiles, the runs
 *                                      cut so that every CTA gets about the same depth of
 *                                      K (sum over its tiles of ceil(m_s / 16))
 * The configuration changes no result: every tile is computed by the same instructions
 * in the same order whichever CTA runs it, and the trace partials are summed in tile
 * order.  It applies to GBE_PREC_FP16X6 / GBE_PREC_BF16X3 states (FP64 states ignore it).
 * This knob is not in the paper; the paper's GPU runs call a dense GEMM per submatrix. */
enum { GBE_SCHED_ROUND_ROBIN = 0, GBE_SCHED_BALANCED_RANGES = 1 };
typedef struct {
    int stages;
    int schedule;
    int kchunk;
} gbe_tc_config;

#define GBE_TUNE_MAX 16
typedef struct {
    int n;                            /* candidates timed                                    */
    gbe_tc_config cand[GBE_TUNE_MAX];
    float ms[GBE_TUNE_MAX];           /* mean CUDA-event time of one SP2 run (gather + loop) */
    int best;                         /* index of the configuration installed               */
    int iters;                        /* squarings per timed run (replayed sequence)         */
    int cached;                       /* 1: taken from the context's cache, nothing timed    */
} gbe_tune_report;

/* Read / install the configuration of a state (not in the paper).  Installing one rebuilds the tile schedule
 * on the device and drops the state's captured SP2 graphs (recaptured on the next run).
 * GBE_EINVAL for a depth the precision is not built with or an unknown schedule. */
int gbe_subs_get_config(const gbe_subs* X, gbe_tc_config* cfg);
int gbe_subs_set_config(gbe_ctx* ctx, gbe_subs* X, const gbe_tc_config* cfg);

/* Autotuner (not in the paper; the paper runs one dense GEMM per submatrix): time every built
 * configuration of X's precision on the caller's own problem and install the fastest.
 * One SP2 run with `params` (its branch decisions as given) fixes the branch sequence;
 * every candidate then replays that sequence without FP64 tail steps, twice untimed (the
 * second run captures its CUDA graphs) and `reps` times timed with CUDA events on the
 * context stream, so all candidates do the same work.  The choice is cached in the
 * context under the state's shape (precision, SM count, subgraph sizes): states created
 * later with the same shape start with it, and
 * a later autotune of such a state returns the cached choice without timing (rep->cached).
 * Afterwards X holds the last candidate's iterates: run gbe_sp2_run again for a result.
 * H must be device CSR.  Synchronises.  FP64 states: nothing to tune (one candidate). */
int gbe_sp2_autotune(gbe_ctx* ctx, const gbe_csr* H, const gbe_parts* parts, const gbe_sp2_params* params,
                     gbe_subs* X, int reps, gbe_tune_report* rep);

/* --------------------------------------------------------- assembly (a8) */

/* Collect the core columns of every final x[s] into ELL D (Eq. 6): row C_s[j] of the
 * ELL receives (sub_idx_s[k], x_s[k, j]) for k < m_s, in local order (core vertices,
 * then halo), skipping |value| < drop_tol when drop_tol > 0.  Query: with D->col NULL
 * the call only sets D->n and D->width (= max m_s) and returns.  GBE_ECAPACITY when
 * D->width < max m_s.  Device D: enqueue only; host D: synchronises and copies out. */
int gbe_assemble_D(gbe_ctx* ctx, const gbe_subs* X, const gbe_parts* parts, double drop_tol, gbe_ell* D);

/* Copy the final dense x_s (m_s x m_s, row-major, FP64) of subgraph s to host (the P(x[s])
 * of Eq. 6 before assembly). */
int gbe_subs_export(gbe_ctx* ctx, const gbe_subs* X, int64_t s, double* out);

/* ------------------------------------------------ finite temperature (Chebyshev expansion) */

/* D = [exp(beta (H - mu)) + 1]^-1 (Eq. 7) on every subgraph, assembled by Eq. 6: x_s =
 * (H_s - a I) / b with a, b the centre and half-width of the spectral bounds, and the
 * Chebyshev series of the Fermi function evaluated by Clenshaw's recurrence
 * b_k = c_k I + 2 x b_{k+1} - b_{k+2} (k = order..1), D_s = c_0 I + x b_1 - b_2
 * (order + 1 products of x with the current iterate).  The iterates are carried divided by
 * B >= max_k ||b_k|| (the scalar recurrence maximised over [-1, 1]) so that the tensor-core
 * split applies; gbe_assemble_D / gbe_subs_export multiply by B.
 *   beta, mu  inverse temperature (1/energy) and chemical potential (energy units of H)
 *   order     highest Chebyshev degree (1..100000)
 *   coeffs    NULL: the Fermi function's Chebyshev interpolant (gbe_fermi_coefficients); or
 *             order + 1 caller coefficients on [eps_min, eps_max]
 *   prec      GBE_PREC_FP64 or GBE_PREC_FP16X6 (must equal the state's)
 *   eps_given 0: Gershgorin bounds of H (computed on the device, read back once)
 * gbe_foe_run synchronises once (for the bounds when not given) and enqueues the rest. */
typedef struct {
    double beta, mu;
    int order;
    const double* coeffs;
    int prec;
    int eps_given;
    double eps_min, eps_max;
    double timeout_ms;
} gbe_foe_params;

typedef struct {
    int order, status;
    double scale;              /* B */
    double eps_min, eps_max;
    float ms_gather, ms_steps; /* gather (and clearing) / all order + 1 steps */
    double mma_flops, alg_flops;
} gbe_foe_report;

/* Chebyshev interpolant of the Fermi function of Eq. 7 on [eps_min, eps_max] at 2 (order + 1)
 * Chebyshev-Gauss nodes: c_n = (2 - delta_n0) / K sum_j f(a + b cos t_j) cos(n t_j).  Host only.
 * gbe_foe_run and gbe_foe_report_get run and report the Eq. 7 expansion described above. */
int gbe_fermi_coefficients(double beta, double mu, double eps_min, double eps_max, int order, double* coeffs);
int gbe_foe_run(gbe_ctx* ctx, const gbe_csr* H, const gbe_parts* parts, const gbe_foe_params* params, gbe_subs* X);
int gbe_foe_report_get(gbe_ctx* ctx, const gbe_subs* X, gbe_foe_report* rep);

/* ------------------------------------------------ pre-determined branch sequences */

/* Sec. II.C: in an MD run the SP2 sequence (shared by every subgraph) is fixed in advance
 * from a HOMO-LUMO gap estimated at the previous step, so that the expansions exchange no
 * traces.  Host-only functions (no context, no GPU).
 *
 * gbe_sp2_gap_estimate: HOMO/LUMO estimates (energy units of H) from a finished run's report
 * (its traces t1/t2, branch sequence and spectral bounds).  The last step k with idempotency
 * error t1[k]-t2[k] in [e_lo, e_hi] is modelled as two unconverged levels, the HOMO image
 * x_h and the LUMO image x_l (t1-t2 = x_h(1-x_h) + x_l(1-x_l), t1-n_occ = x_l-(1-x_h)), which
 * the inverse branch maps carry back to step 0.  Needs 0 < e_lo < e_hi < 0.5.  GBE_EINVAL when
 * no step lies in the window; GBE_ENUMERIC when the traces admit no such pair.  Reliable only
 * when the run reaches that two-level regime (dense or well-converged graph runs). */
int gbe_sp2_gap_estimate(const gbe_sp2_report* rep, double n_occ, double e_lo, double e_hi, double* homo,
                         double* lumo);

/* Sec. II.C: branch sequence (seq[i] = 1 for X^2, 0 for 2X-X^2; *len entries written) that drives every
 * eigenvalue <= homo within tol of 1 and every eigenvalue >= lumo within tol of 0 in the
 * scaled variable x = (eps_max - e)/(eps_max - eps_min): the branch rule applied to the
 * two-level matrix diag(x_homo, x_lumo) with one occupied level.  seq: caller-owned, n_max
 * (<= GBE_SEQ_MAX) bytes.  GBE_ENOCONV when n_max steps do not suffice. */
int gbe_sp2_sequence(double eps_min, double eps_max, double homo, double lumo, double tol, int n_max, uint8_t* seq,
                     int* len);

/* ------------------------------------------------ learned graph proposal (a9) */

/* A small classifier proposes the data-dependency graph when no prior density matrix
 * exists (not in the paper, whose graphs come from a prior D, Sec. II.A/II.C).
 * Candidate pairs are all i != j with minimum-image distance r_ij < rcand; each pair has
 * features f = [-log10(max(|H_ij|,1e-12))/12, -log10(max(|(H^2)_ij|,1e-12))/12,
 * r_ij/rcand, min(e_i,e_j), max(e_i,e_j)] (float32, symmetric in i and j; e = onsite).
 * Network: h1 = relu(W1 f + b1), h2 = relu(W2 h1 + b2), logit = w3.h2 + b3, width 64,
 * fp16-rounded weights and FP32 arithmetic.  Parameters (4609 float32): W1[64x5],
 * b1[64], W2[64x64] (row = output), b2[64], w3[64], b3.  Training minimises the mean
 * binary cross-entropy with logits (label 1 when |D_ij| >= tau) with Adam on the fp32
 * master copy; gradients are reduced in a fixed order (run-to-run identical). */
typedef struct gbe_pairs gbe_pairs;

/* Candidate pairs and features on the device (not in the paper; rows ordered by i, then j
 * ascending).  gbe_pairs_info gives their count.
 * sites and H may be host or device; H must be symmetric with sorted rows ((H^2)_ij is
 * accumulated in row i over k ascending, which equals the row-j sum bit for bit when H is
 * symmetric to the last bit, as gbe_build_hamiltonian's H is).  GBE_ECAPACITY above 1024
 * candidates per site; GBE_EINVAL unless box > 2 rcand.  Temporary device memory: a
 * staging slot of 512 candidates (2 KB) per site during the build.  Synchronises. */
int gbe_pairs_build(gbe_ctx* ctx, const gbe_sites* sites, const gbe_csr* H, double rcand, gbe_pairs** pairs);
int gbe_pairs_info(const gbe_pairs* pairs, int64_t* n, int64_t* npairs);
/* Host copies of the pairs (not in the paper): rowptr[n+1] (int64), j[npairs] (int32),
 * features[npairs*5] (float32); NULL skips. */
int gbe_pairs_export(gbe_ctx* ctx, const gbe_pairs* pairs, int64_t* rowptr, int32_t* j, float* features);
/* Library-owned device arrays of the pairs (not in the paper; valid until gbe_free_pairs);
 * NULL skips. */
int gbe_pairs_device(const gbe_pairs* pairs, const int64_t** rowptr, const int32_t** j, const float** features);
int gbe_free_pairs(gbe_pairs* pairs);

/* Network with zero parameters (not in the paper; hidden must be 64); set them with
 * gbe_mlp_set_params.  gbe_mlp_param_count gives their number (4609). */
int gbe_mlp_create(gbe_ctx* ctx, int hidden, gbe_mlp** mlp);
int gbe_mlp_param_count(const gbe_mlp* mlp);
/* host_params (not in the paper): gbe_mlp_param_count floats; setting also resets the Adam
 * moments and step count. */
int gbe_mlp_set_params(gbe_ctx* ctx, gbe_mlp* mlp, const float* host_params);
int gbe_mlp_get_params(gbe_ctx* ctx, const gbe_mlp* mlp, float* host_params);
/* Forward pass of the classifier (not in the paper); logits: device float[npairs].  Enqueue only. */
int gbe_mlp_forward(gbe_ctx* ctx, const gbe_mlp* mlp, const gbe_pairs* pairs, float* logits);
/* Mean BCE loss and its gradient at the current parameters (not in the paper); labels: device uint8[npairs]
 * (0/1).  loss (host, nullable) and grad_host (host float[param_count], nullable) are
 * written after a synchronisation.  The gradient stays on the device for the next
 * gbe_mlp_adam_step. */
int gbe_mlp_gradient(gbe_ctx* ctx, gbe_mlp* mlp, const gbe_pairs* pairs, const uint8_t* labels, double* loss,
                     float* grad_host);
/* One bias-corrected Adam step with the last gradient (not in the paper).  Enqueue only. */
int gbe_mlp_adam_step(gbe_ctx* ctx, gbe_mlp* mlp, float lr, float beta1, float beta2, float eps);
/* Training (not in the paper): epochs x (gradient + Adam(lr, 0.9, 0.999, 1e-8)) on the device; final_loss (host,
 * nullable) is the mean loss of the last epoch before its update.  Synchronises. */
int gbe_mlp_train(gbe_ctx* ctx, gbe_mlp* mlp, const gbe_pairs* pairs, const uint8_t* labels, int epochs, float lr,
                  double* final_loss);
/* Training labels of the candidate pairs from a density matrix (not in the paper; the
 * labels are the thresholded pattern floor(D)_tau whose graph Sec. II.A builds): labels[p]
 * = 1 when |D_ij| >= tau for pair p = (i, j), 0 otherwise, 0 also where D holds no entry
 * (i, j).  D: device ELL as gbe_assemble_D fills it (row j = column j of D, so D_ij is read
 * from row j), D->n = the pairs' n.  labels: device uint8[npairs].  GBE_EINVAL for a host
 * ELL, mismatched n or tau < 0.  Enqueue only. */
int gbe_mlp_labels(gbe_ctx* ctx, const gbe_pairs* pairs, const gbe_ell* D, double tau, uint8_t* labels);
int gbe_free_mlp(gbe_mlp* mlp);

/* ----------------------------------------------- allocation-free Gershgorin bounds */

/* Gershgorin bounds of a device CSR H, computed without allocating any device memory.
 * The paper has no counterpart; this is a library convenience for callers that must not
 * call cudaMalloc -- for example code whose device memory is entirely owned by another
 * allocator (a framework's memory pool with a fixed budget), or loops that cannot afford
 * the implicit device synchronisation an allocation can cause.
 *   bounds: caller-owned DEVICE memory for 2 doubles, receives {e_min, e_max} with
 *           e_min = min_i H_ii - sum_{j!=i}|H_ij| and e_max = max_i H_ii + sum_{j!=i}|H_ij|
 *           (the same values gbe_sp2_run uses); both NaN when H holds a NaN or Inf.
 *   H:      device CSR (on_device = 1); 1 <= n <= 4,194,304 rows, else GBE_EINVAL with a
 *           message naming the limit.
 * bounds, H->rowptr, H->col and H->val must be device memory of the context's GPU (or
 * managed memory); a host pointer is refused with GBE_EINVAL before anything is enqueued.
 * Scratch: a fixed file-scope device array of 16384 per-block partials (about 256 KB),
 * held by every GPU that loads the library until the process exits.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress, with the device
 * current), and the lookup is repeated when the device's current context has changed
 * since (after cudaDeviceReset); make the first call on a device, and the first call
 * after a reset, before any stream capture.  Every call shares the one
 * array and overwrites it, so calls that overlap on the GPU (different streams or
 * contexts on the same device) race and must be serialised by the caller.
 * Enqueues on the context stream and returns without synchronising. */
int gbe_gershgorin_noalloc(gbe_ctx* ctx, const gbe_csr* H, double* bounds);

#ifdef __cplusplus
}
#endif

#endif /* GBE_H */
