// Internal declarations shared by the libgbe translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/gbe.h"

// ----------------------------------------------------------------------------- errors
void gbe_set_error(const char* fmt, ...);

#define GBE_CUDA_TRY(expr)                                                               \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            gbe_set_error("%s:%d %s: %s", __FILE__, __LINE__, #expr, cudaGetErrorString(e_)); \
            return GBE_ECUDA;                                                            \
        }                                                                                \
    } while (0)

#define GBE_TRY(expr)                  \
    do {                               \
        int r_ = (expr);               \
        if (r_ != GBE_OK) return r_;   \
    } while (0)

#define GBE_CHECK_ARG(cond, msg)                          \
    do {                                                  \
        if (!(cond)) {                                    \
            gbe_set_error("invalid argument: %s", msg);   \
            return GBE_EINVAL;                            \
        }                                                 \
    } while (0)

// ----------------------------------------------------------------------------- objects
struct gbe_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    int smem_optin = 0;
    // small device scratch for counters and flags (4 KB), and its pinned host mirror
    void* d_scratch = nullptr;
    void* h_scratch = nullptr;
    int profile = 0;
    int graphs = 1;   // SP2 runs launched as CUDA graphs (when per-kernel profiling is off)
    // stream-ordered device memory pool of this context (freed blocks are kept for reuse)
    cudaMemPool_t pool = nullptr;
    // autotuned squaring configurations by state shape (precision, SM count, subgraph sizes)
    std::vector<std::pair<std::vector<int64_t>, gbe_tc_config>> tune_cache;
};

struct gbe_hamiltonian {
    int64_t n = 0, nnz = 0;
    int64_t* rowptr = nullptr;
    int32_t* col = nullptr;
    double* val = nullptr;
};

// Graph: explicit CSR of the base pattern A (undirected, diagonal present); the
// graph it stands for is pattern(A^hops).  `full_*` caches the explicit A^hops.
struct gbe_graph {
    int64_t n = 0, nnz = 0;
    int hops = 1;
    int64_t* rowptr = nullptr;
    int32_t* col = nullptr;
    int64_t full_nnz = -1;
    int64_t* full_rowptr = nullptr;
    int32_t* full_col = nullptr;
};

struct gbe_parts {
    int64_t n = 0;        // vertices
    int64_t P = 0;        // subgraphs
    int64_t total = 0;    // sum of m_s
    int64_t max_m = 0;
    int cores_cover = 0;  // every vertex is a core vertex of exactly one subgraph
    int32_t* d_core_count = nullptr;  // [P]
    int64_t* d_sub_ptr = nullptr;     // [P+1]
    int32_t* d_sub_idx = nullptr;     // [total]
    std::vector<int32_t> h_core_count;
    std::vector<int64_t> h_sub_ptr;
    // a shard of a larger partition (gbe_parts_shard): the whole partition has P_global
    // subgraphs, local subgraph s is global subgraph h_global_id[s], and d_local_of maps a
    // global index to the local one (-1: another rank's).  Not a shard: P_global = P and
    // the maps are the identity (h_global_id empty, d_local_of NULL).
    int64_t P_global = 0;
    std::vector<int64_t> h_global_id;
    int32_t* d_local_of = nullptr;   // [P_global]
};

// Device control block of one SP2 run (one per gbe_subs).
struct Sp2Ctrl {
    int iter;        // n of the current iterate X_n
    int stop;        // GBE_STOP_*
    int mode;        // 0 tensor-core squaring, 1 FP64 squaring
    int fmt;         // storage of X_n: 0 split planes, 1 FP64
    int cur;         // ping-pong side holding X_n
    int branch;      // 1: X_{n+1} = X_n^2, 0: 2 X_n - X_n^2 (valid while stop == 0)
    int status;      // GBE_OK or an error code recorded on the device
    int fp64_iters;
    int switch_iter; // first FP64 iteration in mixed runs (-1 before the switch)
    int pending;     // a squaring kernel ran since the last decision
    int loops;       // iterations of the graph's device-driven loop (guard)
    int foe;         // 1: a Chebyshev expansion (Eq. 7) instead of SP2
    double out_scale;  // factor applied by assembly / export (Chebyshev: the iterates' scale)
    uint8_t slot_ran[GBE_SEQ_MAX];  // per launch slot: bit 0 tensor-core kernel worked, bit 1 FP64 kernel
    int n_min, n_max, branch_mode, seq_len, fp64_tail, prec, eps_given;
    unsigned long long eps_min_key, eps_max_key;  // order-preserving keys for atomics
    double eps_min, eps_max;
    double n_occ, idem_tol, tail_switch;
    long long timeout_cycles;
    uint8_t seq_in[GBE_SEQ_MAX];
    uint8_t seq[GBE_SEQ_MAX];
    double t1[GBE_SEQ_MAX + 1];
    double t2[GBE_SEQ_MAX + 1];
};

// Work item of a squaring kernel: output tile (I, J), I <= J, of subgraph s.
struct TileItem {
    int s, I, J, pad;
};

struct SubsGeom {
    // per subgraph (device)
    const int64_t* off;    // element offset of x_s in a plane
    const int32_t* mpad;   // padded size (multiple of 128)
    const int32_t* m;      // m_s
    const int32_t* c;      // core count
};

struct gbe_subs {
    const gbe_parts* parts = nullptr;
    int prec = 0;
    int64_t P = 0;
    int64_t total_elems = 0;    // sum of mpad^2
    int max_mpad = 0;
    std::vector<int64_t> h_off;
    std::vector<int32_t> h_mpad, h_m, h_c;
    int64_t* d_off = nullptr;
    int32_t* d_mpad = nullptr;
    int32_t* d_m = nullptr;
    int32_t* d_c = nullptr;
    // storage
    // sides 0/1: ping-pong iterates; side 2: the fixed x of a Chebyshev expansion (allocated
    // by its first run)
    uint16_t* planes[3] = {nullptr, nullptr, nullptr};  // tensor-core path: gbe_subs_planes(prec) planes x total_elems
    double* f64[3] = {nullptr, nullptr, nullptr};       // FP64 iterates
    // the gather's dense-row staging in global memory, for subgraphs whose rows do not fit
    // shared memory: [P][8][max_mpad] uint2 (allocated by the first run that needs it)
    void* d_gather_rows = nullptr;
    // CTAs of the gather per subgraph (each takes every gather_split-th group of 8 rows and
    // writes one trace partial); 1 with global row staging
    int gather_split = 1;
    // work lists
    TileItem* d_items_tc = nullptr;  int n_items_tc = 0;   // 128x128 tiles
    TileItem* d_items_64 = nullptr;  int n_items_64 = 0;   // 64x64 tiles
    TileItem* d_items_tc_full = nullptr;  int n_items_tc_full = 0;   // all (I, J), for products x b
    TileItem* d_items_64_full = nullptr;  int n_items_64_full = 0;
    double* d_partials = nullptr;    int max_units = 0;    // [2][max_units] (t1, t2)
    // work units of each subgraph in the partials array, per decision kind (0: gather, one
    // unit per subgraph; 1: tensor-core tiles; 2: FP64 tiles): first unit and count
    int2* d_ranges[3] = {nullptr, nullptr, nullptr};
    // per-subgraph trace sums at global subgraph positions, exchanged between the ranks of
    // a sharded run: [0, P_global) t1, [P_global, 2 P_global) t2, [2 P_global] error flag
    double* d_sums = nullptr;
    int64_t P_global = 0;
    Sp2Ctrl* d_ctrl = nullptr;
    Sp2Ctrl* h_ctrl = nullptr;       // pinned
    // tensor maps for the split planes (opaque 128-byte CUtensorMap blobs)
    // TMA descriptors [side][view: K-chunk, transposed][box: A planes, B planes, diagonal B]
    alignas(64) unsigned char tmap[3][2][3][128];     // ring stages of 32 columns of K
    alignas(64) unsigned char tmap16[3][2][3][128];   // ring stages of 16 columns
    bool tmap_ok = false;
    // phase timing
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    std::vector<cudaEvent_t> ev_tc, ev_64;   // [2 * slot + {0,1}] when profiling
    int last_slots = 0;
    bool last_prof = false;
    // last Chebyshev expansion: order, scale of the iterates, run time (events ev[0..2])
    int foe_order = 0;
    double foe_scale = 0.0;
    // CUDA graphs of a run: [0] control init, bounds, gather, first decision; [1] a loop node
    // whose body is one SP2 step, repeated while the device's decision says continue.
    // Reused while a run's parameters and inputs match the key they were captured with.
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    std::vector<unsigned char> gkey;
    cudaStream_t cap_stream = nullptr;
    double alg_flops_per_iter = 0.0, mma_flops_per_iter = 0.0, fp64_flops_per_iter = 0.0;
    double mma_flops_full = 0.0, fp64_flops_full = 0.0;   // per product over all tiles
    // launch configuration of the tensor-core squaring (ring depth, work schedule); with the
    // balanced-range schedule CTA b takes items [d_cta_ptr[b], d_cta_ptr[b + 1])
    gbe_tc_config tc_cfg{0, GBE_SCHED_ROUND_ROBIN, 0};
    int32_t* d_cta_ptr = nullptr;
    int cta_grid = 0;
};

// ----------------------------------------------------------------------------- blocked layout
// A padded m x m submatrix (mpad a multiple of 128) is stored in row blocks of 128 rows;
// inside a row block, column groups of 8 follow each other, and a group holds its 128
// rows x 8 columns row by row:
//   element (r, c) -> off + (r / 128) * 128 * mpad + (c / 8) * 1024 + (r % 128) * 8 + c % 8.
// A 32-column K-chunk of a row block is one contiguous 8 KB run that is already the
// canonical K-major, unswizzled operand layout of the tensor cores (8-row x 16-byte core
// matrices: 128 B apart along rows, 2 KB apart along K), and a warp's 32 consecutive
// rows x 8 columns are 512 contiguous bytes.
__host__ __device__ inline int64_t blk_index(int64_t off, int mpad, int r, int c) {
    return off + (int64_t)(r >> 7) * 128 * mpad + ((int64_t)(c >> 3) << 10) + ((r & 127) << 3) + (c & 7);
}
// Split planes hold only upper-triangular 128 x 128 blocks (the iterates are symmetric):
// an element of a lower block is read from its mirror.
__host__ __device__ inline int64_t sym_index(int64_t off, int mpad, int r, int c) {
    return ((r >> 7) > (c >> 7)) ? blk_index(off, mpad, c, r) : blk_index(off, mpad, r, c);
}

// split planes of a tensor-core state (each plane total_elems fp16 / bf16 values)
inline int gbe_subs_planes(int prec) { return prec == GBE_PREC_FP64TC ? 10 : 4; }

// ----------------------------------------------------------------------------- launchers
int gbe_launch_gershgorin(gbe_ctx* ctx, const gbe_csr* H, gbe_subs* X);
int gbe_tc_make_tmaps(gbe_subs* X);
int gbe_tc_launch_square(gbe_ctx* ctx, gbe_subs* X, int slot);
int gbe_tc_launch_foe(gbe_ctx* ctx, gbe_subs* X, int a_side, int b_side, int c_side, float alpha, double gamma);
int gbe_tc_prepare(gbe_ctx* ctx);
// ring depths the SP2 squaring kernel of a precision and K-chunk width (0 = 32) is built
// with (returns their count)
int gbe_tc_stage_options(int prec, int kc, int* stages, int cap);
// install a launch configuration on a state (work schedule rebuilt, SP2 graphs dropped)
int gbe_subs_apply_config(gbe_ctx* ctx, gbe_subs* X, const gbe_tc_config& cfg);
// shape key of a state for the context's tuning cache
std::vector<int64_t> gbe_subs_shape_key(const gbe_ctx* ctx, const gbe_subs* X);

// helpers
// Device memory.  Inside an AllocScope (every entry point that takes a context opens one)
// gbe_alloc takes memory from the context's pool in the context's stream order; gbe_free
// returns it in the order of the stream it was allocated on (no device synchronisation).
// Outside a scope they fall back to cudaMalloc / cudaFree.
int gbe_alloc(void** p, size_t bytes);
void gbe_free(void* p);
struct AllocScope {
    explicit AllocScope(const gbe_ctx* ctx);
    ~AllocScope();
    AllocScope(const AllocScope&) = delete;
    AllocScope& operator=(const AllocScope&) = delete;
    cudaStream_t prev_stream;
    cudaMemPool_t prev_pool;
};
int gbe_sync(gbe_ctx* ctx);
