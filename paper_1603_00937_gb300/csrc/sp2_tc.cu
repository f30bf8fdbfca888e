// Tensor-core SP2 squaring on sm_103a: tcgen05.mma with TMEM accumulators, operand
// tiles staged by TMA (cp.async.bulk.tensor), branch X^2 / 2X - X^2 applied in the
// epilogue, next split written directly, FP64-grade core traces fused.
//
// One CTA per SM (persistent), 6 warps:
//   warp 0  TMA producer      : K-chunks of 32 for every split plane an MMA needs
//   warp 1  MMA issuer        : 128x128x16 tcgen05.mma per product and k-step into
//                               two TMEM accumulators, double-buffered (4 x 128 cols)
//   warps 2-5 epilogue        : TMEM -> registers, X_{n+1} = S or 2 X_n - S, split,
//                               store tile and (off-diagonal tiles) its transpose,
//                               partial traces of core rows
// Work items are upper-triangular output tiles (I <= J) of every subgraph; the
// iterate is exactly symmetric because every off-diagonal tile is mirrored.
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

constexpr int kThreads = 192;
constexpr int kTileBytes = 128 * 32 * 2;   // 128 rows x 32 halfs (64-byte rows, 64B swizzle)
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

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
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
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
// Named barrier over the 128 epilogue threads that also ORs a flag across them.
__device__ __forceinline__ bool epi_bar_any(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}

// Shared-memory matrix descriptor: K-major operand, 64-byte swizzle, 8-row atoms of
// 512 bytes (stride byte offset 512), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, A/B type (0 fp16, 1 bf16),
// both K-major, N = 128, M = 128.
__host__ __device__ constexpr uint32_t idesc_f16(uint32_t ab_type) {
    return (1u << 4) | (ab_type << 7) | (ab_type << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
}

// ------------------------------------------------------------------ recipes
// Operand slots of a stage: A slots first, then B slots; `plane` is the storage plane,
// `alias` the A slot holding the same plane on diagonal tiles (-1: always loaded).
template <int PREC>
struct Recipe;

// Tables are packed 4-bit fields indexed by slot / product number.
template <>
struct Recipe<GBE_PREC_FP16X6> {
    // slots: A {s0, s1, s2}, B {s0, s1, s1s, s2}; products into acc0: s0 s0^T,
    // into acc1 (units 2^-11): s0 s1^T, s1 s0^T, s1 s1s^T, s0 s2^T, s2 s0^T
    static constexpr int kSlots = 7, kA = 3, kProducts = 6, kPlanes = 4, kStages = 3;
    static constexpr uint32_t kType = 0;  // fp16
    static constexpr uint32_t kPlane = 0x2310210u, kAlias1 = 0x3021000u;
    static constexpr uint32_t kPa = 0x201100u, kPb = 0x365343u, kPacc = 0x111110u;
};

template <>
struct Recipe<GBE_PREC_BF16X3> {
    // slots: A {hi, lo}, B {hi, lo}; products hi hi^T + hi lo^T + lo hi^T into acc0
    static constexpr int kSlots = 4, kA = 2, kProducts = 3, kPlanes = 2, kStages = 4;
    static constexpr uint32_t kType = 1;  // bf16
    static constexpr uint32_t kPlane = 0x1010u, kAlias1 = 0x2100u;
    static constexpr uint32_t kPa = 0x100u, kPb = 0x232u, kPacc = 0x0u;
};

__host__ __device__ constexpr int nib(uint32_t v, int i) { return (int)((v >> (4 * i)) & 0xFu); }
template <class R> __device__ __forceinline__ int slot_plane(int s) { return nib(R::kPlane, s); }
template <class R> __device__ __forceinline__ int slot_alias(int s) { return nib(R::kAlias1, s) - 1; }

template <int PREC>
constexpr size_t smem_bytes() {
    using R = Recipe<PREC>;
    return 1024 /*align slack*/ + (size_t)R::kStages * R::kSlots * kTileBytes + (size_t)R::kPlanes * 16 * 128 * 2 +
           256 /*barriers, flags, reduction*/;
}

struct TcArgs {
    Sp2Ctrl* ctrl;
    SubsGeom g;
    const TileItem* items;
    int n_items;
    uint16_t* planes[2];
    int64_t ps;  // plane stride in elements
    double* partials;
    int max_units;
    int slot;
};

// Double-float accumulation of w * (P + Q)^2 (FP64-grade traces from FP32 parts).
__device__ __forceinline__ void df_add_sq(float& sh, float& sl, float P, float Q, float w) {
    const float p2 = P * P;
    const float e2 = fmaf(P, P, -p2);
    const float th = w * p2;
    const float tl = w * (e2 + Q * (2.0f * P + Q));
    const float s = sh + th;
    const float bp = s - sh;
    const float err = (sh - (s - bp)) + (th - bp);
    sh = s;
    sl += err + tl;
}

template <int PREC>
__global__ void __launch_bounds__(kThreads, 1)
    sp2_square_tc_kernel(const __grid_constant__ CUtensorMap tmap0, const __grid_constant__ CUtensorMap tmap1,
                         TcArgs args) {
    using R = Recipe<PREC>;
    constexpr int NS = R::kStages;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* tiles = smem;                                          // NS * kSlots * 8 KB
    uint16_t* stg = (uint16_t*)(tiles + (size_t)NS * R::kSlots * kTileBytes);  // kPlanes x 16 x 128
    uint64_t* bars = (uint64_t*)((unsigned char*)stg + (size_t)R::kPlanes * 16 * 128 * 2);
    uint64_t* full = bars;             // [NS]
    uint64_t* empty = bars + NS;       // [NS]
    uint64_t* tfull = bars + 2 * NS;   // [2]
    uint64_t* tempty = bars + 2 * NS + 2;  // [2]
    uint64_t* drain = bars + 2 * NS + 4;   // [1]
    uint32_t* tmem_holder = (uint32_t*)(bars + 2 * NS + 5);
    volatile int* abort_flag = (volatile int*)(tmem_holder + 1);
    int* hdr = (int*)(tmem_holder + 2);           // run, cur, branch
    double* red = (double*)(bars + 2 * NS + 8);   // 8 doubles

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Sp2Ctrl* ctrl = args.ctrl;
    if (threadIdx.x == 0) {
        hdr[0] = (ctrl->stop == 0 && ctrl->mode == 0);
        hdr[1] = ctrl->cur;
        hdr[2] = ctrl->branch;
        *abort_flag = 0;
        for (int i = 0; i < NS; ++i) { mbar_init(&full[i], 1); mbar_init(&empty[i], 1); }
        for (int i = 0; i < 2; ++i) { mbar_init(&tfull[i], 1); mbar_init(&tempty[i], 128); }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (!hdr[0]) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) { ctrl->pending = 1; ctrl->slot_ran[args.slot] |= 1; }
    const int cur = hdr[1], branch = hdr[2];
    const long long budget = ctrl->timeout_cycles;
    const CUtensorMap* tmap = cur ? &tmap1 : &tmap0;
    const uint16_t* pin = args.planes[cur];
    uint16_t* pout = args.planes[cur ^ 1];
    const int64_t ps = args.ps;

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
            int issued_stage[NS], issued_parity[NS];
            for (int i = 0; i < NS; ++i) issued_stage[i] = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < args.n_items && ok; it += gridDim.x) {
                const TileItem w = args.items[it];
                const int mpad = args.g.mpad[w.s], m = args.g.m[w.s];
                const int64_t off = args.g.off[w.s];
                const int nk = (m + 31) >> 5;
                const bool diag = (w.I == w.J);
                int nload = 0;
                for (int sl = 0; sl < R::kSlots; ++sl) nload += !(diag && slot_alias<R>(sl) >= 0);
                for (int kc = 0; kc < nk; ++kc) {
                    if (!mbar_wait(&empty[stage], phase ^ 1, budget, abort_flag)) { ok = false; break; }
                    mbar_arrive_expect_tx(&full[stage], (uint32_t)(nload * kTileBytes));
                    issued_stage[stage] = 1;
                    issued_parity[stage] = phase;
                    unsigned char* st = tiles + (size_t)stage * R::kSlots * kTileBytes;
                    const int x = (kc & 1) * 32;
                    for (int sl = 0; sl < R::kSlots; ++sl) {
                        if (diag && slot_alias<R>(sl) >= 0) continue;
                        const int Rt = (sl < R::kA) ? w.I : w.J;
                        const int64_t y = (int64_t)slot_plane<R>(sl) * (ps >> 6) + (off >> 6) +
                                          ((int64_t)(Rt * (mpad >> 6) + (kc >> 1)) << 7);
                        tma_load_2d(st + (size_t)sl * kTileBytes, tmap, &full[stage], x, (int)y);
                    }
                    if (++stage == NS) { stage = 0; phase ^= 1; }
                }
            }
            if (!ok) {
                *abort_flag = 1;
                atomicExch(&ctrl->status, GBE_ETIMEOUT);
                // drain copies this thread issued so no TMA write lands after exit
                for (int i = 0; i < NS; ++i)
                    if (issued_stage[i]) {
                        const long long t0 = clock64();
                        while (!mbar_try_wait(&full[i], issued_parity[i]) && clock64() - t0 < budget) {
                        }
                    }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_f16(R::kType);
            int stage = 0;
            uint32_t phase = 0;
            int tb = 0;
            uint32_t tph = 0;
            bool ok = true;
            const uint32_t tiles_addr = smem_u32(tiles);
            for (int it = blockIdx.x; it < args.n_items && ok; it += gridDim.x) {
                const TileItem w = args.items[it];
                const int m = args.g.m[w.s];
                const int nk = (m + 31) >> 5;
                const bool diag = (w.I == w.J);
                if (!mbar_wait(&tempty[tb], tph ^ 1, budget, abort_flag)) { ok = false; break; }
                tc_fence_after();
                const uint32_t dacc0 = tmem_base + (uint32_t)(tb * 256);
                for (int kc = 0; kc < nk; ++kc) {
                    if (!mbar_wait(&full[stage], phase, budget, abort_flag)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sbase = tiles_addr + (uint32_t)(stage * R::kSlots * kTileBytes);
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
#pragma unroll
                        for (int p = 0; p < R::kProducts; ++p) {
                            const int a = nib(R::kPa, p), acc = nib(R::kPacc, p);
                            int b = nib(R::kPb, p);
                            if (diag && slot_alias<R>(b) >= 0) b = slot_alias<R>(b);
                            const uint64_t da = sdesc_sw64(sbase + a * kTileBytes + ks * 32);
                            const uint64_t db = sdesc_sw64(sbase + b * kTileBytes + ks * 32);
                            // the first product into each accumulator overwrites it
                            bool first = (kc == 0 && ks == 0);
                            if (first) {
                                for (int q = 0; q < p; ++q)
                                    if (nib(R::kPacc, q) == acc) first = false;
                            }
                            umma_f16(dacc0 + acc * 128, da, db, idesc, first ? 0u : 1u);
                        }
                    }
                    umma_commit(&empty[stage]);
                    if (++stage == NS) { stage = 0; phase ^= 1; }
                }
                if (!ok) break;
                umma_commit(&tfull[tb]);
                tb ^= 1;
                if (tb == 0) tph ^= 1;
            }
            if (!ok) {
                *abort_flag = 1;
                atomicExch(&ctrl->status, GBE_ETIMEOUT);
            }
            // all issued MMAs complete before TMEM is released
            umma_commit(drain);
            const long long t0 = clock64();
            while (!mbar_try_wait(drain, 0) && clock64() - t0 < budget) {
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue (warps 2..5)
        const int q = warp & 3;
        const int ew = warp - 2;
        const int a = 32 * q + lane;
        const uint32_t lane_addr = tmem_base + ((uint32_t)(32 * q) << 16);
        int tb = 0;
        uint32_t tph = 0;
        for (int it = blockIdx.x; it < args.n_items; it += gridDim.x) {
            const TileItem w = args.items[it];
            const int mpad = args.g.mpad[w.s], c = args.g.c[w.s];
            const int64_t off = args.g.off[w.s];
            const bool ok = mbar_wait(&tfull[tb], tph, budget, abort_flag);
            // all four epilogue warps leave together, so no named barrier is left waiting
            if (epi_bar_any(!ok)) {
                *abort_flag = 1;
                atomicExch(&ctrl->status, GBE_ETIMEOUT);
                break;
            }
            tc_fence_after();
            const int row = 128 * w.I + a;
            const bool core_row = row < c;
            float sh = 0.f, sl = 0.f;
            double t1 = 0.0;
            for (int ch = 0; ch < 8; ++ch) {
                const int col0 = 128 * w.J + 16 * ch;
                uint32_t ra[16], rb[16];
                tmem_ld16(lane_addr + (uint32_t)(tb * 256 + 16 * ch), ra);
                if (R::kPlanes == 4) tmem_ld16(lane_addr + (uint32_t)(tb * 256 + 128 + 16 * ch), rb);
                tmem_wait_ld();
                if (ch == 7) {
                    tc_fence_before();
                    mbar_arrive(&tempty[tb]);
                }
                const int64_t e0 = blk_index(off, mpad, row, col0);
                uint16_t xv[3][16];
                if (!branch) {
#pragma unroll
                    for (int p = 0; p < (R::kPlanes == 4 ? 3 : 2); ++p) {
                        const uint4* src = reinterpret_cast<const uint4*>(pin + p * ps + e0);
                        uint4 v0 = src[0], v1 = src[1];
                        memcpy(&xv[p][0], &v0, 16);
                        memcpy(&xv[p][8], &v1, 16);
                    }
                }
                uint16_t ov[R::kPlanes][16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float A = __uint_as_float(ra[j]);
                    float P, Q;
                    if constexpr (PREC == GBE_PREC_FP16X6) {
                        const float B = __uint_as_float(rb[j]);
                        if (branch) {
                            P = A;
                            Q = B * GBE_OZ_R_INV;
                        } else {
                            const float s0 = h_val(xv[0][j]), s1 = h_val(xv[1][j]), s2 = h_val(xv[2][j]);
                            P = 2.0f * s0 - A;
                            Q = (2.0f * (s1 + s2) - B) * GBE_OZ_R_INV;
                        }
                        const OzSplit o = oz_split_pq(P, Q);
                        ov[0][j] = o.s0;
                        ov[1][j] = o.s1;
                        ov[2][j] = o.s2;
                        ov[3][j] = o.s1s;
                    } else {
                        P = branch ? A : 2.0f * (b_val(xv[0][j]) + b_val(xv[1][j])) - A;
                        Q = 0.0f;
                        const __nv_bfloat16 hi = __float2bfloat16_rn(P);
                        ov[0][j] = b_bits(hi);
                        ov[1][j] = b_bits(__float2bfloat16_rn(P - __bfloat162float(hi)));
                    }
                    const int colg = col0 + j;
                    const float wgt = (float)((int)core_row + (int)((w.I != w.J) && colg < c));
                    if (wgt != 0.0f) df_add_sq(sh, sl, P, Q, wgt);
                    if (colg == row && core_row) t1 += (double)P + (double)Q;
                }
#pragma unroll
                for (int p = 0; p < R::kPlanes; ++p) {
                    uint4* dst = reinterpret_cast<uint4*>(pout + p * ps + e0);
                    uint4 v0, v1;
                    memcpy(&v0, &ov[p][0], 16);
                    memcpy(&v1, &ov[p][8], 16);
                    dst[0] = v0;
                    dst[1] = v1;
                }
                if (w.I != w.J) {
#pragma unroll
                    for (int p = 0; p < R::kPlanes; ++p)
#pragma unroll
                        for (int j = 0; j < 16; ++j) stg[(p * 16 + j) * 128 + a] = ov[p][j];
                    epi_bar();
                    // transposed rows: (plane, j) pairs split over the 4 epilogue warps
                    for (int pr = ew; pr < R::kPlanes * 16; pr += 4) {
                        const int p = pr >> 4, j = pr & 15;
                        const int trow = 128 * w.J + 16 * ch + j;
                        const uint2 v = *reinterpret_cast<const uint2*>(&stg[(p * 16 + j) * 128 + 4 * lane]);
                        *reinterpret_cast<uint2*>(pout + p * ps + blk_index(off, mpad, trow, 128 * w.I + 4 * lane)) = v;
                    }
                    epi_bar();
                }
            }
            // partial traces of this tile: fixed-order reduction over the 128 threads
            double t2 = (double)sh + (double)sl;
            for (int o = 16; o > 0; o >>= 1) {
                t1 += __shfl_xor_sync(0xffffffffu, t1, o);
                t2 += __shfl_xor_sync(0xffffffffu, t2, o);
            }
            if (lane == 0) { red[2 * ew] = t1; red[2 * ew + 1] = t2; }
            epi_bar();
            if (ew == 0 && lane == 0) {
                args.partials[it] = ((red[0] + red[2]) + red[4]) + red[6];
                args.partials[args.max_units + it] = ((red[1] + red[3]) + red[5]) + red[7];
            }
            epi_bar();
            tb ^= 1;
            if (tb == 0) tph ^= 1;
        }
        tc_fence_before();
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols) : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode_tiled = nullptr;

}  // namespace

int gbe_tc_prepare(gbe_ctx* ctx) {
    (void)ctx;
    if (g_encode_tiled) return GBE_OK;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
        gbe_set_error("cuTensorMapEncodeTiled not available: %s", cudaGetErrorString(e));
        return GBE_ECUDA;
    }
    g_encode_tiled = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    int prec_list[2] = {GBE_PREC_FP16X6, GBE_PREC_BF16X3};
    for (int p : prec_list) {
        const size_t bytes = p == GBE_PREC_FP16X6 ? smem_bytes<GBE_PREC_FP16X6>() : smem_bytes<GBE_PREC_BF16X3>();
        if ((int)bytes > ctx->smem_optin) {
            gbe_set_error("tensor-core kernel needs %zu bytes of shared memory, device allows %d", bytes, ctx->smem_optin);
            return GBE_ENODEV;
        }
    }
    e = cudaFuncSetAttribute(sp2_square_tc_kernel<GBE_PREC_FP16X6>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes<GBE_PREC_FP16X6>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sp2_square_tc_kernel<GBE_PREC_BF16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_bytes<GBE_PREC_BF16X3>());
    if (e != cudaSuccess) {
        gbe_set_error("cudaFuncSetAttribute: %s", cudaGetErrorString(e));
        return GBE_ECUDA;
    }
    return GBE_OK;
}

int gbe_tc_make_tmaps(gbe_subs* X) {
    if (!g_encode_tiled) {
        gbe_set_error("tensor maps requested before gbe_tc_prepare");
        return GBE_ECUDA;
    }
    const int nplanes = 4;
    for (int side = 0; side < 2; ++side) {
        CUtensorMap m;
        memset(&m, 0, sizeof(m));
        cuuint64_t dims[2] = {64, (cuuint64_t)(nplanes * X->total_elems / 64)};
        cuuint64_t strides[1] = {128};
        cuuint32_t box[2] = {32, 128};
        cuuint32_t estr[2] = {1, 1};
        CUresult r = g_encode_tiled(&m, X->prec == GBE_PREC_BF16X3 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                                    2, X->planes[side], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                    CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            gbe_set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
            return GBE_ECUDA;
        }
        static_assert(sizeof(CUtensorMap) == 128, "CUtensorMap size");
        memcpy(X->tmap[side], &m, sizeof(m));
    }
    X->tmap_ok = true;
    return GBE_OK;
}

int gbe_tc_launch_square(gbe_ctx* ctx, gbe_subs* X, int slot) {
    if (!X->tmap_ok) {
        gbe_set_error("tensor maps missing");
        return GBE_ECUDA;
    }
    TcArgs a;
    a.ctrl = X->d_ctrl;
    a.g = SubsGeom{X->d_off, X->d_mpad, X->d_m, X->d_c};
    a.items = X->d_items_tc;
    a.n_items = X->n_items_tc;
    a.planes[0] = X->planes[0];
    a.planes[1] = X->planes[1];
    a.ps = X->total_elems;
    a.partials = X->d_partials;
    a.max_units = X->max_units;
    a.slot = slot;
    CUtensorMap m0, m1;
    memcpy(&m0, X->tmap[0], sizeof(m0));
    memcpy(&m1, X->tmap[1], sizeof(m1));
    const int grid = std::max(1, std::min(X->n_items_tc, ctx->sm_count));
    if (X->prec == GBE_PREC_FP16X6)
        sp2_square_tc_kernel<GBE_PREC_FP16X6><<<grid, kThreads, smem_bytes<GBE_PREC_FP16X6>(), ctx->stream>>>(m0, m1, a);
    else
        sp2_square_tc_kernel<GBE_PREC_BF16X3><<<grid, kThreads, smem_bytes<GBE_PREC_BF16X3>(), ctx->stream>>>(m0, m1, a);
    GBE_CUDA_TRY(cudaGetLastError());
    return GBE_OK;
}
