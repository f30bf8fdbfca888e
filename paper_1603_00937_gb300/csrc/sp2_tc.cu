// Tensor-core SP2 squaring on sm_103a: tcgen05.mma with TMEM accumulators, operand
// tiles staged by TMA (cp.async.bulk.tensor), branch X^2 / 2X - X^2 applied in the
// epilogue, next split written directly, FP64-grade core traces fused.
//
// One CTA per SM (persistent), 10 warps (14 for FP64TC):
//   warp 0  TMA producer      : K-chunks of 32 (16) for every split plane an MMA needs (one
//                               contiguous 8 KB (4 KB) box each, already in MMA operand order)
//   warp 1  MMA issuer        : 128xNx16 tcgen05.mma per product and k-step (N = 128, less in a
//                               subgraph's last column block) into the recipe's TMEM
//                               accumulators: two, double-buffered (4 x 128 cols), for the
//                               split formats; four, single-buffered, for FP64TC
//   warps 2.. epilogue        : TMEM -> registers, X_{n+1} = S or 2 X_n - S, split,
//                               store the tile, partial traces of core rows (counting the
//                               implied mirror of off-diagonal tiles); two warps per TMEM lane
//                               quarter, each taking half of the tile's columns (three for
//                               FP64TC, whose epilogue does not overlap the MMAs, each taking
//                               a third).  X_n values for the next chunk are fetched ahead.
// Only upper-triangular 128x128 blocks of each iterate are stored; a K-chunk that falls in
// a lower block is loaded from the mirror block as a transposed (MN-major) operand tile.
// Work items are upper-triangular output tiles (I <= J) of every subgraph.
//
// Every mbarrier wait is bounded by a clock budget; on expiry the CTA records
// GBE_ETIMEOUT in the control block, stops issuing, drains what it issued (again
// bounded) and frees its TMEM before returning.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "gbe_internal.h"
#include "split.cuh"

namespace {

// One operand slot holds a K-chunk of KC columns (32 or 16) of a 128-row block: KC/8 column
// groups of 128 rows x 16 bytes, contiguous in the blocked layout.
template <int KC>
constexpr int tile_bytes() { return 128 * KC * 2; }
constexpr int kTmemCols = 512;

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait; false when the budget ran out or another role aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long budget, volatile int* abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > budget) return false;
    }
}


// 3-D box (x, y, plane z): the planes of one operand side in a single copy.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// MMA and commit, executed by a whole warp with warp-uniform operands: one elected lane
// issues the instruction (tcgen05.mma is a single-thread instruction).
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p, e;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile(
        "{\n\t.reg .pred e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}\n" ::"r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Named barrier over the NT epilogue threads.
template <int NT>
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory"); }
// The same barrier, ORing a flag across the epilogue threads.
template <int NT>
__device__ __forceinline__ bool epi_bar_any(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(NT)
        : "memory");
    return r != 0;
}

// Shared-memory matrix descriptor: K-major operand without swizzling; core matrices of
// 8 rows x 16 bytes, 2048 bytes apart along K (leading byte offset) and 128 bytes apart
// along M/N (stride byte offset); descriptor version 1.
__device__ __forceinline__ uint64_t sdesc_kmajor(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)(2048 >> 4) << 16;
    d |= (uint64_t)(128 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// Same for an MN-major (transposed) operand tile [16 groups of 8 rows][KC k][8]: core
// matrices 128 bytes apart along K (leading byte offset), 16 KC bytes apart along M/N.
template <int KC>
__device__ __forceinline__ uint64_t sdesc_mnmajor(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)((16 * KC) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, A/B type (0 fp16, 1 bf16),
// K-major operands (bits 15/16 select MN-major per operand), N = n (a multiple of 16, at
// most 128 here), M = 128.
__host__ __device__ constexpr uint32_t idesc_f16(uint32_t ab_type, uint32_t n = 128) {
    return (1u << 4) | (ab_type << 7) | (ab_type << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

// Columns of output tile (I, J) that a squaring computes: in a subgraph's last column block
// only up to the first multiple of 16 at or past m (every iterate is zero beyond m, and those
// columns are never written: they keep the zeros the state starts with); all 128 for a
// Chebyshev step.
__device__ __forceinline__ int tile_cols(int m, int J, bool foe) {
    const int rest = m - 128 * J;
    return (foe || rest >= 128) ? 128 : ((rest + 15) >> 4) << 4;
}

// ------------------------------------------------------------------ recipes
// Operand slots of a stage: A slots first, then B slots, each side in storage-plane order
// so that one 3-D TMA box (planes as its third dimension) fills a side's slots.  A slot i
// holds plane i; B slot kA + j holds plane kBPlane0 + j.  On a diagonal tile B's planes
// below kA are A's (the same block), so B loads only its planes kDiagPlane.. (kDiag of
// them) into their own slots.  pa / pb / pacc: A slot, B slot and accumulator of product p.
// TMEM: kAcc accumulators of 128 columns per tile, kTmemBufCols columns per buffer, 512 /
// kTmemBufCols buffers (two: the epilogue of one tile overlaps the next tile's MMAs).
template <int PREC>
struct Recipe;

__host__ __device__ constexpr int nib(uint32_t v, int i) { return (int)((v >> (4 * i)) & 0xFu); }

template <>
struct Recipe<GBE_PREC_FP16X6> {
    // slots: A {s0, s1, s2}, B {s0, s1, s2, s1s}; products into acc0: s0 s0^T,
    // into acc1 (units 2^-11): s0 s1^T, s1 s0^T, s1 s1s^T, s0 s2^T, s2 s0^T
    static constexpr int kSlots = 7, kA = 3, kProducts = 6, kPlanes = 4, kStages = 4, kDiag = 1;
    static constexpr int kAcc = 2, kTmemBufCols = 256, kBPlane0 = 0, kDiagPlane = 3, kStages16 = 8;
    static constexpr int kEpiWarps = 8;
    static constexpr uint32_t kType = 0;  // fp16
    __host__ __device__ static constexpr int pa(int p) { return nib(0x201100u, p); }
    __host__ __device__ static constexpr int pb(int p) { return nib(0x356343u, p); }
    __host__ __device__ static constexpr int pacc(int p) { return nib(0x111110u, p); }
};

template <>
struct Recipe<GBE_PREC_BF16X3> {
    // slots: A {hi, lo}, B {hi, lo}; products hi hi^T + hi lo^T + lo hi^T into acc0
    static constexpr int kSlots = 4, kA = 2, kProducts = 3, kPlanes = 2, kStages = 6, kDiag = 0;
    static constexpr int kAcc = 1, kTmemBufCols = 256, kBPlane0 = 0, kDiagPlane = 2, kStages16 = 12;
    static constexpr int kEpiWarps = 8;
    static constexpr uint32_t kType = 1;  // bf16
    __host__ __device__ static constexpr int pa(int p) { return nib(0x100u, p); }
    __host__ __device__ static constexpr int pb(int p) { return nib(0x232u, p); }
    __host__ __device__ static constexpr int pacc(int p) { return 0; }
};

template <>
struct Recipe<GBE_PREC_FP64TC> {
    // planes 0 u', 1 t0, 2 t1, 3 t2, 4 t3, 5 u, 6 v, 7 t3', 8 t4', 9 t2' (split.cuh); A slots
    // 0-8 = planes 0-8, B slots 9-17 = planes 1-9 (B slot of plane q: 8 + q).  Four
    // accumulators fill the TMEM, so the epilogue does not overlap the next tile's MMAs;
    // only 16-column K-chunks fit (a stage of 18 slots is 72 KB).
    static constexpr int kSlots = 18, kA = 9, kProducts = 18, kPlanes = 10, kStages = 0, kDiag = 1;
    static constexpr int kAcc = 4, kTmemBufCols = 512, kBPlane0 = 1, kDiagPlane = 9, kStages16 = 3;
    static constexpr int kEpiWarps = 12;
    static constexpr uint32_t kType = 0;  // fp16
    //  ACC0: t0 t0 | ACC1: t0 t1, t1 t0, u' u | ACC2: t0 t2, t2 t0, u v, v u, v v |
    //  ACC3: t0 t3, t3 t0, t1 t2, t2 t1 (2^-30); t0 t4', t4' t0, t1 t3', t3' t1, t2 t2' (2^-40)
    __host__ __device__ static constexpr int pa(int p) {
        constexpr int t[18] = {1, 1, 2, 0, 1, 3, 5, 6, 6, 1, 4, 2, 3, 1, 8, 2, 7, 3};
        return t[p];
    }
    __host__ __device__ static constexpr int pb(int p) {
        constexpr int t[18] = {9, 10, 9, 13, 11, 9, 14, 13, 14, 12, 9, 11, 10, 16, 9, 15, 10, 17};
        return t[p];
    }
    __host__ __device__ static constexpr int pacc(int p) {
        constexpr int t[18] = {0, 1, 1, 1, 2, 2, 2, 2, 2, 3, 3, 3, 3, 3, 3, 3, 3, 3};
        return t[p];
    }
};

// Threads of a CTA: producer warp, MMA warp, the recipe's epilogue warps.
template <int PREC>
constexpr int threads_of() { return 64 + 32 * Recipe<PREC>::kEpiWarps; }

// A slot holding the same plane as B slot b on a diagonal tile, or -1 (loaded).
template <class R> __host__ __device__ constexpr int slot_alias(int b) {
    return (b >= R::kA && R::kBPlane0 + (b - R::kA) < R::kA) ? R::kBPlane0 + (b - R::kA) : -1;
}

// Default ring depth for a K-chunk width.
template <int PREC, int KC>
constexpr int default_stages() { return KC == 32 ? Recipe<PREC>::kStages : Recipe<PREC>::kStages16; }

// Bytes after the operand ring: 2 NS + 5 mbarriers, the TMEM address, abort flag and header
// words, then the per-tile trace reduction (two parities x 4 floats per epilogue warp).
constexpr size_t bar_area_bytes(int ns, int epi_warps) { return (size_t)(2 * ns + 8) * 8 + (size_t)32 * epi_warps; }

// Shared memory of a CTA with an NS-deep ring of KC-column chunks (NS = 0: the default).
template <int PREC, int NS = 0, int KC = 32>
constexpr size_t smem_bytes() {
    using R = Recipe<PREC>;
    constexpr int ns = NS ? NS : default_stages<PREC, KC>();
    return 1024 /*align slack*/ + (size_t)ns * R::kSlots * tile_bytes<KC>() + bar_area_bytes(ns, R::kEpiWarps);
}

// Optional wait-time counters (build with -DGBE_TC_STATS): cycles each role spends in
// barrier waits, summed over CTAs into a device array of 8 counters.
#ifdef GBE_TC_STATS
__device__ unsigned long long g_tc_stats[16];
#define TC_T0() const long long _t0 = clock64()
#define TC_ACC(i) (st_acc[i] += (unsigned long long)(clock64() - _t0))
#define TC_FLUSH()                                                       \
    for (int i_ = 0; i_ < 8; ++i_)                                       \
        if (st_acc[i_]) atomicAdd(&g_tc_stats[i_], st_acc[i_])
#else
#define TC_T0()
#define TC_ACC(i)
#define TC_FLUSH()
#endif

// 3-D tensor maps [side][view][box] (sides 0/1: ping-pong iterates, 2: the fixed x of a
// Chebyshev expansion): view 0 = K-chunk view of stored blocks, view 1 =
// transposed view (lower blocks); box 0 = A planes (depth kA), 1 = B planes (depth kSlots-kA),
// 2 = B planes of a diagonal tile (depth kDiag, from plane kA).
struct TcMaps {
    CUtensorMap m[3][2][3];
};

struct TcArgs {
    Sp2Ctrl* ctrl;
    SubsGeom g;
    const TileItem* items;
    int n_items;
    uint16_t* planes[3];
    int64_t ps;  // plane stride in elements
    // Chebyshev step (FOE kernels): out = alpha (x b) - c + gamma I with x on side a_side,
    // b on side b_side, c read from and the result written to side c_side; gamma is split
    // into its 2^-20-grid part (added to the exact leading term) and the remainder
    int a_side, b_side, c_side;
    float alpha, gamma_g, gamma_r;
    double* partials;
    int max_units;
    int slot;
    // work schedule: NULL = round-robin over items (CTA b takes b, b + grid, ...);
    // otherwise CTA b takes the contiguous range [cta_ptr[b], cta_ptr[b + 1])
    const int32_t* cta_ptr;
};

// FOE = false: one SP2 squaring X_{n+1} = X_n^2 or 2 X_n - X_n^2 (branch from the device).
// FOE = true: one step of a Chebyshev expansion, out = alpha x b - c + gamma I (arguments).
// NS_: depth of the operand ring (0: the default for KC); KC: columns of K per ring stage
// (32, or 16 for twice as many stages in the same shared memory).
template <int PREC, bool FOE, int NS_, int KC>
__global__ void __launch_bounds__(threads_of<PREC>(), 1)
    sp2_square_tc_kernel(const __grid_constant__ TcMaps maps, TcArgs args) {
    using R = Recipe<PREC>;
    constexpr int EW = R::kEpiWarps, ENT = 32 * EW;   // epilogue warps and threads
    static_assert(EW == 8 || EW == 12, "two or three epilogue warps per TMEM lane quarter");
    static_assert(R::kAcc * 128 <= R::kTmemBufCols && 512 % R::kTmemBufCols == 0, "accumulators must fit a TMEM buffer");
    constexpr int NS = NS_ ? NS_ : default_stages<PREC, KC>();
    constexpr int kTileBytes = tile_bytes<KC>();
    constexpr int kCPB = 128 / KC;            // K-chunks per 128-column block
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* tiles = smem;                                          // NS * kSlots * KC/4 KB
    uint64_t* bars = (uint64_t*)(tiles + (size_t)NS * R::kSlots * kTileBytes);
    uint64_t* full = bars;             // [NS]
    uint64_t* empty = bars + NS;       // [NS]
    uint64_t* tfull = bars + 2 * NS;   // [2]
    uint64_t* tempty = bars + 2 * NS + 2;  // [2]
    uint64_t* drain = bars + 2 * NS + 4;   // [1]
    uint32_t* tmem_holder = (uint32_t*)(bars + 2 * NS + 5);
    volatile int* abort_flag = (volatile int*)(tmem_holder + 1);
    int* hdr = (int*)(tmem_holder + 2);           // run, cur, branch
    double* red = (double*)(bars + 2 * NS + 8);   // 2 x 32 floats (by tile parity)

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Sp2Ctrl* ctrl = args.ctrl;
#ifdef GBE_TC_STATS
    const long long g_kernel_t0 = clock64();
    unsigned long long st_acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#endif
    if (threadIdx.x == 0) {
        hdr[0] = (ctrl->stop == 0 && ctrl->mode == 0);
        hdr[1] = ctrl->cur;
        hdr[2] = ctrl->branch;
        *abort_flag = 0;
        for (int i = 0; i < NS; ++i) { mbar_init(&full[i], 1); mbar_init(&empty[i], 1); }
        for (int i = 0; i < 2; ++i) { mbar_init(&tfull[i], 1); mbar_init(&tempty[i], ENT); }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (!hdr[0]) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctrl->pending = 1;
        if (args.slot >= 0) ctrl->slot_ran[args.slot] |= 1;   // launch slots (profiled runs) only
    }
    const int cur = hdr[1], branch = hdr[2];
    const long long budget = ctrl->timeout_cycles;
    // the drains after an abort wait for work already issued (copies, MMAs), which finishes
    // in microseconds: at least ~1 s of clock whatever the caller's budget, so that no copy
    // lands and no MMA writes TMEM after the CTA has released them
    const long long drain_budget = budget > 2000000000LL ? budget : 2000000000LL;
    // [view][box] maps of the A and B operand sides; planes the epilogue reads and writes
    const CUtensorMap(*tmA)[3] = maps.m[FOE ? args.a_side : cur];
    const CUtensorMap(*tmB)[3] = maps.m[FOE ? args.b_side : cur];
    // (selects, not an indexed parameter array, which would be copied to local memory)
    uint16_t* const pc = args.c_side == 0 ? args.planes[0] : (args.c_side == 1 ? args.planes[1] : args.planes[2]);
    const uint16_t* pin = FOE ? pc : (cur ? args.planes[1] : args.planes[0]);
    uint16_t* pout = FOE ? pc : (cur ? args.planes[0] : args.planes[1]);
    const bool use_c = FOE || !branch;   // the update reads the stored planes at its own tile
    const int64_t ps = args.ps;
    // the same item sequence for the producer, the MMA issuer and the epilogue
    int it_first = blockIdx.x, it_end = args.n_items, it_step = gridDim.x;
    if (args.cta_ptr) {
        it_first = args.cta_ptr[blockIdx.x];
        it_end = args.cta_ptr[blockIdx.x + 1];
        it_step = 1;
    }

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_holder;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t issued_mask = 0, issued_par = 0;   // per stage: armed, and the parity it was armed with
            bool ok = true;
            for (int it = it_first; it < it_end && ok; it += it_step) {
                const TileItem w = args.items[it];
                const int mpad = args.g.mpad[w.s], m = args.g.m[w.s];
                const int64_t off = args.g.off[w.s];
                const int nk = (m + KC - 1) / KC;
                // a diagonal tile of a squaring takes B's planes s0..s2 from A's slots
                const bool diag = (w.I == w.J) && !FOE;
                const int nload = R::kA + (diag ? R::kDiag : R::kSlots - R::kA);
                for (int kc = 0; kc < nk; ++kc) {
                    bool got;
                    {
                        TC_T0();
                        got = mbar_wait(&empty[stage], phase ^ 1, budget, abort_flag);
                        TC_ACC(0);
                    }
                    if (!got) { ok = false; break; }
                    mbar_arrive_expect_tx(&full[stage], (uint32_t)(nload * kTileBytes));
                    issued_mask |= 1u << stage;
                    issued_par = (issued_par & ~(1u << stage)) | (phase << stage);
                    unsigned char* st = tiles + (size_t)stage * R::kSlots * kTileBytes;
                    const int kb = kc / kCPB;
                    const int64_t g0 = off >> 10;
                    // side A (row block I), then side B (column block J): one box per side
#pragma unroll
                    for (int side = 0; side < 2; ++side) {
                        const int Rt = side == 0 ? w.I : w.J;
                        const int bx = side == 0 ? 0 : (diag ? 2 : 1);
                        if (side == 1 && diag && R::kDiag == 0) continue;
                        // B: planes kBPlane0.. into slots kA..; on a diagonal tile only planes
                        // kDiagPlane.. (the others are A's) into their own slots
                        const int slot0 = side == 0 ? 0 : (diag ? R::kA + R::kDiagPlane - R::kBPlane0 : R::kA);
                        const int z = side == 0 ? 0 : (diag ? R::kDiagPlane : R::kBPlane0);
                        unsigned char* dst = st + (size_t)slot0 * kTileBytes;
                        const CUtensorMap(*tm)[3] = side == 0 ? tmA : tmB;
                        // a Chebyshev step's b is not symmetric to the last bit: its block (kb, J)
                        // itself, as an MN-major tile, whatever kb and J are
                        if (Rt <= kb && !(FOE && side == 1)) {
                            // stored block (Rt, kb): KC/8 column groups of 1024 elements = KC/2
                            // view rows of 256
                            const int64_t y = (g0 + (int64_t)Rt * (mpad >> 3) + (KC / 8) * kc) << 2;
                            tma_load_3d(dst, &tm[0][bx], &full[stage], 0, (int)y, z);
                        } else {
                            // lower block: rows KC (kc mod kCPB).. of stored block (kb, Rt), its 16
                            // column groups -> [16 groups][KC rows][8], an MN-major operand tile
                            const int64_t y = g0 + (int64_t)kb * (mpad >> 3) + 16 * Rt;
                            tma_load_3d(dst, &tm[1][bx], &full[stage], 8 * KC * (kc % kCPB), (int)y, z);
                        }
                    }
                    if (++stage == NS) { stage = 0; phase ^= 1; }
                }
            }
            if (!ok) {
                *abort_flag = 1;
                atomicExch(&ctrl->status, GBE_ETIMEOUT);
                // drain copies this thread issued so no TMA write lands after exit
                for (int i = 0; i < NS; ++i)
                    if (issued_mask & (1u << i)) {
                        const long long t0 = clock64();
                        while (!mbar_try_wait(&full[i], (issued_par >> i) & 1u) && clock64() - t0 < drain_budget) {
                        }
                    }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        // The whole warp runs the loop (every operand is warp-uniform); one elected lane
        // issues each tcgen05 instruction and lane 0 waits on the barriers for the warp.
        int stage = 0;
        uint32_t phase = 0;
        int tb = 0;
        uint32_t tph = 0;
        bool ok = true;
        const uint32_t tiles_addr = smem_u32(tiles);
        auto wait_warp = [&](uint64_t* bar, uint32_t par) {
            int g = 1;
            if (lane == 0) g = mbar_wait(bar, par, budget, abort_flag) ? 1 : 0;
            return __shfl_sync(0xffffffffu, g, 0) != 0;
        };
        for (int it = it_first; it < it_end && ok; it += it_step) {
#ifdef GBE_TC_STATS
            const long long ts0 = clock64();
#endif
            const TileItem w = args.items[it];
            const int m = args.g.m[w.s];
            const int nk = (m + KC - 1) / KC;
            const bool diag = (w.I == w.J) && !FOE;
            const uint32_t idesc = idesc_f16(R::kType, (uint32_t)tile_cols(m, w.J, FOE));
#ifdef GBE_TC_STATS
            st_acc[6] += (unsigned long long)(clock64() - ts0);
#endif
            bool got;
            {
                TC_T0();
                got = wait_warp(&tempty[tb], tph ^ 1);
                TC_ACC(1);
            }
            if (!got) { ok = false; break; }
            tc_fence_after();
            const uint32_t dacc0 = tmem_base + (uint32_t)(tb * R::kTmemBufCols);
            for (int kc = 0; kc < nk; ++kc) {
                {
                    TC_T0();
                    got = wait_warp(&full[stage], phase);
                    TC_ACC(2);
                }
                if (!got) { ok = false; break; }
#ifdef GBE_TC_STATS
                const long long ti0 = clock64();
#endif
                tc_fence_after();
                const uint32_t sbase = tiles_addr + (uint32_t)(stage * R::kSlots * kTileBytes);
                const int kb = kc / kCPB;
                const bool tA = w.I > kb, tB = FOE || w.J > kb;   // operand loaded transposed (MN-major)
                const uint32_t idesc_t = idesc | ((uint32_t)tA << 15) | ((uint32_t)tB << 16);
                // k-steps of 16 holding columns below m (a squaring skips the last chunk's second
                // half when it is all padding; a Chebyshev step runs every k-step)
                const int ksn = FOE ? KC / 16 : min(KC / 16, (m - kc * KC + 15) >> 4);
#pragma unroll
                for (int ks = 0; ks < KC / 16; ++ks) {
                    if (ks >= ksn) break;
#pragma unroll
                    for (int p = 0; p < R::kProducts; ++p) {
                        const int a = R::pa(p), acc = R::pacc(p);
                        int b = R::pb(p);
                        if (diag && slot_alias<R>(b) >= 0) b = slot_alias<R>(b);   // never for FOE
                        const uint32_t aa = sbase + a * kTileBytes, ba = sbase + b * kTileBytes;
                        const uint64_t da = tA ? sdesc_mnmajor<KC>(aa + ks * 256) : sdesc_kmajor(aa + ks * 4096);
                        const uint64_t db = tB ? sdesc_mnmajor<KC>(ba + ks * 256) : sdesc_kmajor(ba + ks * 4096);
                        // the first product into each accumulator overwrites it
                        bool first = (kc == 0 && ks == 0);
                        if (first) {
                            for (int q = 0; q < p; ++q)
                                if (R::pacc(q) == acc) first = false;
                        }
                        umma_f16(dacc0 + acc * 128, da, db, idesc_t, first ? 0u : 1u);
                    }
                }
                umma_commit(&empty[stage]);
#ifdef GBE_TC_STATS
                st_acc[7] += (unsigned long long)(clock64() - ti0);
#endif
                if (++stage == NS) { stage = 0; phase ^= 1; }
            }
            if (!ok) break;
            umma_commit(&tfull[tb]);
            if (++tb == 512 / R::kTmemBufCols) { tb = 0; tph ^= 1; }
        }
        if (!ok && lane == 0) {
            *abort_flag = 1;
            atomicExch(&ctrl->status, GBE_ETIMEOUT);
        }
        // all issued MMAs complete before TMEM is released
        umma_commit(drain);
        if (lane == 0) {
            const long long t0 = clock64();
            while (!mbar_try_wait(drain, 0) && clock64() - t0 < drain_budget) {
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue (warps 2..9)
        const int q = warp & 3;                 // TMEM lane quarter this warp may access
        const int ew = warp - 2;                // 0..EW-1
        const int part = ew >> 2;               // this warp's share of the tile's columns
        // columns [cbeg, cend): halves (16-column chunks) for the split recipes; for FP64TC
        // thirds of its sixteen 8-column chunks (6, 5, 5)
        constexpr int kParts = EW / 4;
        const int cbeg = kParts == 2 ? 64 * part : 8 * (part == 0 ? 0 : 1 + 5 * part);
        const int cend = kParts == 2 ? cbeg + 64 : 8 * (6 + 5 * part);
        const int a = 32 * q + lane;
        const uint32_t lane_addr = tmem_base + ((uint32_t)(32 * q) << 16);
        constexpr int kXP = (R::kPlanes == 4) ? 3 : 2;   // planes of X_n the update reads
        int tb = 0;
        uint32_t tph = 0;
        int par = 0;
        for (int it = it_first; it < it_end; it += it_step) {
            const TileItem w = args.items[it];
            const int mpad = args.g.mpad[w.s], c = args.g.c[w.s];
            const int64_t off = args.g.off[w.s];
            const int row = 128 * w.I + a;
            const bool core_row = row < c;
            const bool offdiag = (w.I != w.J);
            const int ncol = tile_cols(args.g.m[w.s], w.J, FOE);   // columns the MMAs computed
            // this warp's 16-column chunks (FP64TC: 8-column chunks) inside them, 0..4 (0..8)
            const int nch = max(0, min((cend - cbeg) >> 4, (ncol - cbeg + 15) >> 4));
            const int nch8 = max(0, min((cend - cbeg) >> 3, (ncol - cbeg + 7) >> 3));
            // X_n of the first chunk, fetched before the accumulator is ready
            uint32_t xn[kXP][8];
            auto fetch_x = [&](int ch) {
                const int64_t e = blk_index(off, mpad, row, 128 * w.J + 16 * ch);
#pragma unroll
                for (int p = 0; p < kXP; ++p) {
                    const uint4 v0 = *reinterpret_cast<const uint4*>(pin + p * ps + e);
                    const uint4 v1 = *reinterpret_cast<const uint4*>(pin + p * ps + e + 1024);
                    xn[p][0] = v0.x; xn[p][1] = v0.y; xn[p][2] = v0.z; xn[p][3] = v0.w;
                    xn[p][4] = v1.x; xn[p][5] = v1.y; xn[p][6] = v1.z; xn[p][7] = v1.w;
                }
            };
            if (use_c && PREC != GBE_PREC_FP64TC && nch > 0) fetch_x(cbeg >> 4);
            // FP64TC: X_n's digits t0..t3 (planes 1-4) and t4' (plane 8) of an 8-column chunk,
            // the first chunk fetched before the accumulators are ready, later ones one ahead
            uint4 xv[5] = {};
            auto fetch_dig = [&](int cc) {
                const int64_t e = blk_index(off, mpad, row, 128 * w.J + cbeg + 8 * cc);
#pragma unroll
                for (int p = 0; p < 5; ++p) xv[p] = *reinterpret_cast<const uint4*>(pin + (p < 4 ? p + 1 : 8) * ps + e);
            };
            if (PREC == GBE_PREC_FP64TC && use_c && nch8 > 0) fetch_dig(0);
            bool ok;
            {
                TC_T0();
                ok = mbar_wait(&tfull[tb], tph, budget, abort_flag);
                if (lane == 0) TC_ACC(3);
            }
            // all epilogue warps leave together, so no named barrier is left waiting
            if (epi_bar_any<ENT>(!ok)) {
                *abort_flag = 1;
                atomicExch(&ctrl->status, GBE_ETIMEOUT);
                break;
            }
            tc_fence_after();
            float sh = 0.f, sl = 0.f, dP = 0.f, dQ = 0.f;
            if ((PREC == GBE_PREC_FP64TC ? nch8 : nch) == 0) {
                // no column of this warp's share was computed: nothing to read or write
                tc_fence_before();
                mbar_arrive(&tempty[tb]);
            }
            if constexpr (PREC == GBE_PREC_FP64TC) {
                // X^2 = ACC0 + 2^-10 ACC1 + 2^-20 ACC2 + 2^-30 ACC3 as an integer V in units of
                // 2^-50 (ACC0..2 hold exact multiples of 2^-20; ACC3 is rounded there), the branch
                // 2 X_n - X^2 in the same integers, then the digits of the next iterate
                for (int cc = 0; cc < nch8; ++cc) {
                    const int col0 = 128 * w.J + cbeg + 8 * cc;
                    const uint32_t ta = lane_addr + (uint32_t)(tb * R::kTmemBufCols + cbeg + 8 * cc);
                    uint32_t r0[8], r1[8], r2[8], r3[8];
                    tmem_ld8(ta, r0);
                    tmem_ld8(ta + 128, r1);
                    tmem_ld8(ta + 256, r2);
                    tmem_ld8(ta + 384, r3);
                    const int64_t e0 = blk_index(off, mpad, row, col0);
                    uint4 xw[5];
#pragma unroll
                    for (int p = 0; p < 5; ++p) xw[p] = xv[p];
                    if (use_c && cc + 1 < nch8) fetch_dig(cc + 1);
                    tmem_wait_ld();
                    if (cc == nch8 - 1) {
                        tc_fence_before();
                        mbar_arrive(&tempty[tb]);
                    }
                    uint32_t ow[GBE_F64TC_PLANES][4];
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        F64Digits d[2];
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const int j = 2 * jj + e;
                            const int n0 = __float2int_rn(__uint_as_float(r0[j]) * 1048576.0f);
                            const int n1 = __float2int_rn(__uint_as_float(r1[j]) * 1048576.0f);
                            const int n2 = __float2int_rn(__uint_as_float(r2[j]) * 1048576.0f);
                            const int n3 = __float2int_rn(__uint_as_float(r3[j]) * 1048576.0f);
                            long long V = ((long long)n0 << 30) + ((long long)n1 << 20) + ((long long)n2 << 10) + (long long)n3;
                            if (use_c) {
                                const int sh16 = 16 * e;
                                auto hw = [&](const uint4& u) {
                                    const uint32_t wd = jj == 0 ? u.x : (jj == 1 ? u.y : (jj == 2 ? u.z : u.w));
                                    return (uint16_t)(wd >> sh16);
                                };
                                const long long Vn = f64tc_from_planes(hw(xw[0]), hw(xw[1]), hw(xw[2]), hw(xw[3]), hw(xw[4]));
                                V = 2 * Vn - V;
                            }
                            d[e] = f64tc_digits(V);
                            float P, Q;
                            f64tc_pair(d[e], P, Q);
                            const int colg = col0 + j;
                            const float wgt = (float)((int)core_row + (int)(offdiag && colg < c));
                            if (wgt != 0.0f) df_add_sq(sh, sl, P, Q, wgt);
                            const bool dg = (colg == row);
                            dP = dg ? P : dP;
                            dQ = dg ? Q : dQ;
                        }
                        uint32_t w10[GBE_F64TC_PLANES];
                        f64tc_planes2(d[0], d[1], w10);
#pragma unroll
                        for (int p = 0; p < GBE_F64TC_PLANES; ++p) ow[p][jj] = w10[p];
                    }
#pragma unroll
                    for (int p = 0; p < GBE_F64TC_PLANES; ++p)
                        *reinterpret_cast<uint4*>(pout + p * ps + e0) = make_uint4(ow[p][0], ow[p][1], ow[p][2], ow[p][3]);
                }
            } else
            for (int cc = 0; cc < nch; ++cc) {
                const int ch = (cbeg >> 4) + cc;
                const int col0 = 128 * w.J + 16 * ch;
                uint32_t ra[16], rb[16];
                tmem_ld16(lane_addr + (uint32_t)(tb * R::kTmemBufCols + 16 * ch), ra);
                if (R::kPlanes == 4) tmem_ld16(lane_addr + (uint32_t)(tb * R::kTmemBufCols + 128 + 16 * ch), rb);
                uint32_t xw[kXP][8];
#pragma unroll
                for (int p = 0; p < kXP; ++p)
#pragma unroll
                    for (int k = 0; k < 8; ++k) xw[p][k] = xn[p][k];
                if (use_c && cc < nch - 1) fetch_x(ch + 1);
                tmem_wait_ld();
                if (cc == nch - 1) {
                    tc_fence_before();
                    mbar_arrive(&tempty[tb]);
                }
                uint32_t ow[R::kPlanes][8];
                if constexpr (PREC == GBE_PREC_FP16X6) {
                    // adjacent column pairs: packed half conversions, words written whole
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) {
                        float P[2], Q[2];
                        const float A0 = __uint_as_float(ra[2 * jj]), A1 = __uint_as_float(ra[2 * jj + 1]);
                        const float B0 = __uint_as_float(rb[2 * jj]), B1 = __uint_as_float(rb[2 * jj + 1]);
                        if (use_c) {
                            const float2 c0 = h2_val(xw[0][jj]), c1 = h2_val(xw[1][jj]), c2 = h2_val(xw[2][jj]);
                            if constexpr (FOE) {
                                // alpha x b - c + gamma I: every term but gamma_r is a multiple of
                                // 2^-20 (exact in FP32), gamma_r joins the small correction
                                const bool g0 = (col0 + 2 * jj == row), g1 = (col0 + 2 * jj + 1 == row);
                                P[0] = args.alpha * A0 - c0.x + (g0 ? args.gamma_g : 0.0f);
                                Q[0] = (args.alpha * B0 - (c1.x + c2.x)) * GBE_OZ_R_INV + (g0 ? args.gamma_r : 0.0f);
                                P[1] = args.alpha * A1 - c0.y + (g1 ? args.gamma_g : 0.0f);
                                Q[1] = (args.alpha * B1 - (c1.y + c2.y)) * GBE_OZ_R_INV + (g1 ? args.gamma_r : 0.0f);
                            } else {
                                P[0] = 2.0f * c0.x - A0;
                                Q[0] = (2.0f * (c1.x + c2.x) - B0) * GBE_OZ_R_INV;
                                P[1] = 2.0f * c0.y - A1;
                                Q[1] = (2.0f * (c1.y + c2.y) - B1) * GBE_OZ_R_INV;
                            }
                        } else {
                            P[0] = A0;
                            Q[0] = B0 * GBE_OZ_R_INV;
                            P[1] = A1;
                            Q[1] = B1 * GBE_OZ_R_INV;
                        }
                        const OzSplit2 o = oz_split_pq2(P[0], Q[0], P[1], Q[1]);
                        ow[0][jj] = o.s0;
                        ow[1][jj] = o.s1;
                        ow[2][jj] = o.s2;
                        ow[R::kPlanes - 1][jj] = o.s1s;
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const int colg = col0 + 2 * jj + e;
                            const float wgt = (float)((int)core_row + (int)(offdiag && colg < c));
                            if (wgt != 0.0f) df_add_sq(sh, sl, P[e], Q[e], wgt);
                            const bool dg = (colg == row);
                            dP = dg ? P[e] : dP;
                            dQ = dg ? Q[e] : dQ;
                        }
                    }
                } else {
#pragma unroll
                    for (int p = 0; p < R::kPlanes; ++p)
#pragma unroll
                        for (int k = 0; k < 8; ++k) ow[p][k] = 0u;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int sh16 = 16 * (j & 1);
#define XV(p) ((uint16_t)(xw[p][j >> 1] >> sh16))
                        const float A = __uint_as_float(ra[j]);
                        const float P = branch ? A : 2.0f * (b_val(XV(0)) + b_val(XV(1))) - A;
                        const float Q = 0.0f;
                        const __nv_bfloat16 hi = __float2bfloat16_rn(P);
                        ow[0][j >> 1] |= (uint32_t)b_bits(hi) << sh16;
                        ow[1][j >> 1] |= (uint32_t)b_bits(__float2bfloat16_rn(P - __bfloat162float(hi))) << sh16;
#undef XV
                        const int colg = col0 + j;
                        const float wgt = (float)((int)core_row + (int)(offdiag && colg < c));
                        if (wgt != 0.0f) df_add_sq(sh, sl, P, Q, wgt);
                        const bool dg = (colg == row);
                        dP = dg ? P : dP;
                        dQ = dg ? Q : dQ;
                    }
                }
                const int64_t e0 = blk_index(off, mpad, row, col0);
#pragma unroll
                for (int p = 0; p < R::kPlanes; ++p) {
                    *reinterpret_cast<uint4*>(pout + p * ps + e0) = make_uint4(ow[p][0], ow[p][1], ow[p][2], ow[p][3]);
                    *reinterpret_cast<uint4*>(pout + p * ps + e0 + 1024) = make_uint4(ow[p][4], ow[p][5], ow[p][6], ow[p][7]);
                }
            }
            // partial traces of this tile: FP32-pair (TwoSum) reduction in a fixed order over
            // the warp, FP64 only for the final per-tile sum (FP64 is a narrow pipe here)
            const bool has_diag = core_row && !offdiag && (row >> 7) == w.J && (row & 127) >= cbeg && (row & 127) < cend;
            float d1h = has_diag ? dP : 0.f, d1l = has_diag ? dQ : 0.f;
            for (int o = 16; o > 0; o >>= 1) {
                df_add(sh, sl, __shfl_xor_sync(0xffffffffu, sh, o), __shfl_xor_sync(0xffffffffu, sl, o));
                df_add(d1h, d1l, __shfl_xor_sync(0xffffffffu, d1h, o), __shfl_xor_sync(0xffffffffu, d1l, o));
            }
            float* rd = reinterpret_cast<float*>(red) + 4 * EW * par;
            if (lane == 0) { rd[4 * ew] = d1h; rd[4 * ew + 1] = d1l; rd[4 * ew + 2] = sh; rd[4 * ew + 3] = sl; }
            epi_bar<ENT>();
            if (ew == 0 && lane == 0) {
                double r1 = 0.0, r2 = 0.0;
                for (int k = 0; k < EW; ++k) {
                    r1 += (double)rd[4 * k] + (double)rd[4 * k + 1];
                    r2 += (double)rd[4 * k + 2] + (double)rd[4 * k + 3];
                }
                args.partials[it] = r1;
                args.partials[args.max_units + it] = r2;
            }
            par ^= 1;
#ifdef GBE_TC_STATS
            if (lane == 0) st_acc[4] += 1ull;
#endif
            if (++tb == 512 / R::kTmemBufCols) { tb = 0; tph ^= 1; }
        }
        tc_fence_before();
    }
#ifdef GBE_TC_STATS
    if (lane == 0) TC_FLUSH();
#endif
    __syncthreads();
#ifdef GBE_TC_STATS
    if (threadIdx.x == 0) atomicAdd(&g_tc_stats[5], (unsigned long long)(clock64() - g_kernel_t0));
#endif
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols) : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode_tiled = nullptr;

}  // namespace

#ifdef GBE_TC_STATS
extern "C" int gbe_tc_stats(unsigned long long* out, int reset) {
    cudaMemcpyFromSymbol(out, g_tc_stats, sizeof(g_tc_stats));
    if (reset) {
        unsigned long long z[16] = {0};
        cudaMemcpyToSymbol(g_tc_stats, z, sizeof(z));
    }
    return 0;
}
#endif

// Every launchable variant of the squaring kernel: precision, Chebyshev step or not, ring
// depth.  The autotuner chooses among the SP2 variants of a precision.
struct TcVariant {
    int prec;
    bool foe;
    int kc;       // K-chunk width of a ring stage
    int stages;
    const void* fn;
    size_t smem;
    int threads;
};
#define GBE_TC_VARIANT(P, F, N, K)                                                                          \
    TcVariant {                                                                                              \
        P, F, K, N ? N : default_stages<P, K>(), (const void*)sp2_square_tc_kernel<P, F, N, K>, smem_bytes<P, N, K>(), \
            threads_of<P>()                                                                                  \
    }
static const TcVariant kVariants[] = {
    GBE_TC_VARIANT(GBE_PREC_FP16X6, false, 0, 32), GBE_TC_VARIANT(GBE_PREC_FP16X6, false, 3, 32),
    GBE_TC_VARIANT(GBE_PREC_FP16X6, false, 0, 16), GBE_TC_VARIANT(GBE_PREC_FP16X6, false, 6, 16),
    GBE_TC_VARIANT(GBE_PREC_FP16X6, true, 0, 32),  GBE_TC_VARIANT(GBE_PREC_BF16X3, false, 0, 32),
    GBE_TC_VARIANT(GBE_PREC_BF16X3, false, 4, 32), GBE_TC_VARIANT(GBE_PREC_BF16X3, false, 7, 32),
    GBE_TC_VARIANT(GBE_PREC_BF16X3, false, 0, 16), GBE_TC_VARIANT(GBE_PREC_BF16X3, false, 14, 16),
    GBE_TC_VARIANT(GBE_PREC_FP64TC, false, 0, 16),
};
#undef GBE_TC_VARIANT

// stages = 0: the default depth for the chunk width; kc = 0: 32 columns
static int default_kchunk(int prec) { return prec == GBE_PREC_FP64TC ? 16 : 32; }

static const TcVariant* find_variant(int prec, bool foe, int stages, int kc) {
    if (kc == 0) kc = default_kchunk(prec);
    if (stages == 0) {
        if (prec == GBE_PREC_FP16X6) stages = kc == 32 ? default_stages<GBE_PREC_FP16X6, 32>() : default_stages<GBE_PREC_FP16X6, 16>();
        else if (prec == GBE_PREC_BF16X3) stages = kc == 32 ? default_stages<GBE_PREC_BF16X3, 32>() : default_stages<GBE_PREC_BF16X3, 16>();
        else stages = default_stages<GBE_PREC_FP64TC, 16>();
    }
    for (const TcVariant& v : kVariants)
        if (v.prec == prec && v.foe == foe && v.kc == kc && v.stages == stages) return &v;
    return nullptr;
}

int gbe_tc_prepare(gbe_ctx* ctx) {
    if (g_encode_tiled) return GBE_OK;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
        gbe_set_error("cuTensorMapEncodeTiled not available: %s", cudaGetErrorString(e));
        return GBE_ECUDA;
    }
    for (const TcVariant& v : kVariants) {
        if ((int)v.smem > ctx->smem_optin) {
            gbe_set_error("tensor-core kernel (%d stages) needs %zu bytes of shared memory, device allows %d", v.stages,
                          v.smem, ctx->smem_optin);
            return GBE_ENODEV;
        }
        e = cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
        if (e != cudaSuccess) {
            gbe_set_error("cudaFuncSetAttribute: %s", cudaGetErrorString(e));
            return GBE_ECUDA;
        }
    }
    g_encode_tiled = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return GBE_OK;
}

int gbe_tc_stage_options(int prec, int kc, int* stages, int cap) {
    if (kc == 0) kc = default_kchunk(prec);
    int n = 0;
    for (const TcVariant& v : kVariants)
        if (v.prec == prec && !v.foe && v.kc == kc && n < cap) stages[n++] = v.stages;
    return n;
}

int gbe_tc_make_tmaps(gbe_subs* X) {
    if (!g_encode_tiled) {
        gbe_set_error("tensor maps requested before gbe_tc_prepare");
        return GBE_ECUDA;
    }
    // plane buffers hold gbe_subs_planes(prec) planes of total_elems (4 for the two split
    // formats, 10 for FP64TC); boxes: A planes, B planes, a diagonal tile's own B planes
    const int nplanes = gbe_subs_planes(X->prec);
    const bool fp16 = X->prec != GBE_PREC_BF16X3;
    int depth[3] = {fp16 ? 3 : 2, fp16 ? 4 : 2, 1};
    if (X->prec == GBE_PREC_FP64TC) {
        depth[0] = Recipe<GBE_PREC_FP64TC>::kA;
        depth[1] = Recipe<GBE_PREC_FP64TC>::kSlots - Recipe<GBE_PREC_FP64TC>::kA;
        depth[2] = Recipe<GBE_PREC_FP64TC>::kDiag;
    }
    for (int w = 0; w < 2; ++w)   // ring stages of 32 (w = 0) or 16 (w = 1) columns of K
    for (int side = 0; side < 3; ++side)
        for (int view = 0; view < 2; ++view)
            for (int bx = 0; bx < 3; ++bx) {
                unsigned char* slot = w == 0 ? X->tmap[side][view][bx] : X->tmap16[side][view][bx];
                const cuuint32_t kc = w == 0 ? 32 : 16;
                CUtensorMap m;
                memset(&m, 0, sizeof(m));
                // view 0: rows of 256 elements (512 B); a KC-column K-chunk of a row block is one
                // contiguous run of KC/8 column groups = a 256 x KC/2 box per plane, copied unchanged.
                // view 1 (transposed): one 2 KB column group per row; an 8 KC x 16 box takes KC rows
                // of 16 consecutive column groups.  Planes are the third dimension.
                const cuuint64_t inner = view == 0 ? 256 : 1024;
                cuuint64_t dims[3] = {inner, (cuuint64_t)(X->total_elems / inner), (cuuint64_t)nplanes};
                cuuint64_t strides[2] = {inner * 2, (cuuint64_t)X->total_elems * 2};
                cuuint32_t box[3] = {view == 0 ? 256u : 8u * kc, view == 0 ? kc / 2u : 16u, (cuuint32_t)depth[bx]};
                cuuint32_t estr[3] = {1, 1, 1};
                // side 2 exists only once a Chebyshev expansion ran; FP64TC runs 16-column chunks only
                if (!X->planes[side] || (X->prec == GBE_PREC_FP64TC && w == 0)) {
                    memset(slot, 0, 128);
                    continue;
                }
                CUresult r = g_encode_tiled(&m, fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                                            X->planes[side], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                if (r != CUDA_SUCCESS) {
                    gbe_set_error("cuTensorMapEncodeTiled (view %d, box %d) failed (%d)", view, bx, (int)r);
                    return GBE_ECUDA;
                }
                static_assert(sizeof(CUtensorMap) == 128, "CUtensorMap size");
                memcpy(slot, &m, sizeof(m));
            }
    X->tmap_ok = true;
    return GBE_OK;
}

static TcArgs tc_args(gbe_subs* X, int slot) {
    TcArgs a;
    memset(&a, 0, sizeof(a));
    a.ctrl = X->d_ctrl;
    a.g = SubsGeom{X->d_off, X->d_mpad, X->d_m, X->d_c};
    a.items = X->d_items_tc;
    a.n_items = X->n_items_tc;
    for (int i = 0; i < 3; ++i) a.planes[i] = X->planes[i];
    a.ps = X->total_elems;
    a.partials = X->d_partials;
    a.max_units = X->max_units;
    a.slot = slot;
    return a;
}

int gbe_tc_launch_square(gbe_ctx* ctx, gbe_subs* X, int slot) {
    if (!X->tmap_ok) {
        gbe_set_error("tensor maps missing");
        return GBE_ECUDA;
    }
    const TcVariant* v = find_variant(X->prec, false, X->tc_cfg.stages, X->tc_cfg.kchunk);
    if (!v) {
        gbe_set_error("no tensor-core kernel with %d stages of %d columns for precision %d", X->tc_cfg.stages,
                      X->tc_cfg.kchunk, X->prec);
        return GBE_EINVAL;
    }
    TcArgs a = tc_args(X, slot);
    int grid = std::max(1, std::min(X->n_items_tc, ctx->sm_count));
    if (X->d_cta_ptr) {
        a.cta_ptr = X->d_cta_ptr;
        grid = X->cta_grid;
    }
    TcMaps maps;
    static_assert(sizeof(maps) == sizeof(X->tmap) && sizeof(maps) == sizeof(X->tmap16), "tensor map set size");
    memcpy(&maps, v->kc == 16 ? X->tmap16 : X->tmap, sizeof(maps));
    void* kargs[2] = {&maps, &a};
    GBE_CUDA_TRY(cudaLaunchKernel(v->fn, dim3(grid), dim3(v->threads), kargs, v->smem, ctx->stream));
    return GBE_OK;
}

int gbe_tc_launch_foe(gbe_ctx* ctx, gbe_subs* X, int a_side, int b_side, int c_side, float alpha, double gamma) {
    if (!X->tmap_ok || !X->planes[2] || X->prec != GBE_PREC_FP16X6) {
        gbe_set_error("Chebyshev tensor-core step needs FP16X6 planes on three sides");
        return GBE_ECUDA;
    }
    TcArgs a = tc_args(X, -1);
    a.items = X->d_items_tc_full;   // every tile: x b is computed as it is, not mirrored
    a.n_items = X->n_items_tc_full;
    a.a_side = a_side;
    a.b_side = b_side;
    a.c_side = c_side;
    a.alpha = alpha;
    const double gg = rint(gamma * 1048576.0) / 1048576.0;   // 2^-20 grid
    a.gamma_g = (float)gg;
    a.gamma_r = (float)(gamma - gg);
    TcMaps maps;
    memcpy(&maps, X->tmap, sizeof(maps));
    const int gridf = std::max(1, std::min(X->n_items_tc_full, ctx->sm_count));
    sp2_square_tc_kernel<GBE_PREC_FP16X6, true, 0, 32>
        <<<gridf, threads_of<GBE_PREC_FP16X6>(), smem_bytes<GBE_PREC_FP16X6, 0, 32>(), ctx->stream>>>(maps, a);
    GBE_CUDA_TRY(cudaGetLastError());
    return GBE_OK;
}
