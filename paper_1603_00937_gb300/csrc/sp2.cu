// SP2 on core+halo submatrices: state, Gershgorin bounds, gather, device-side branch
// decisions, the FP64 squaring, column assembly and export.
//
// One density-matrix build (Sec. II.A: Eq. 6 with the recursive zero-temperature
// expansion D = lim f_n(...f_0(H)), f_n(X) = X^2 or 2X - X^2):
//   gershgorin  -> e_min, e_max of the whole H                      (FP64)
//   gather      -> X_0[s] = (e_max I - x[s]) / (e_max - e_min)        per subgraph
//   decide      -> global FP64 traces over core positions, branch / stop
//   repeat: square (tensor-core or FP64 kernel; branch applied in its epilogue) -> decide
// The decision lives in a device control block, so the host enqueues a fixed number
// of slots and finished runs turn later slots into immediate exits.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "decide.cuh"
#include "devmem.h"
#include "gbe_internal.h"
#include "split.cuh"

// ----------------------------------------------------------------------------- helpers
__device__ __forceinline__ unsigned long long dkey(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_inv(unsigned long long k) {
    unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

static double dkey_inv_host(unsigned long long k) {
    const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    double d;
    memcpy(&d, &b, sizeof(d));
    return d;
}

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum in a fixed order (deterministic for a fixed blockDim).
template <int NT>
__device__ double block_sum_d(double v, double* sh) {
    v = warp_sum_d(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = (l < NT / 32) ? sh[l] : 0.0;
        r = warp_sum_d(r);
    }
    return r;  // valid in thread 0
}

// ----------------------------------------------------------------------------- Gershgorin
__global__ void __launch_bounds__(256) gershgorin_kernel(const int64_t* __restrict__ rowptr,
                                                         const int32_t* __restrict__ col,
                                                         const double* __restrict__ val, int64_t n,
                                                         Sp2Ctrl* ctrl) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double lo = INFINITY, hi = -INFINITY;
    bool bad = false;
    for (int64_t i = warp; i < n; i += nwarps) {
        double off = 0.0, d = 0.0;
        for (int64_t p = rowptr[i] + lane; p < rowptr[i + 1]; p += 32) {
            double v = val[p];
            if (!isfinite(v)) bad = true;
            if (col[p] == i) d = v; else off += fabs(v);
        }
        off = warp_sum_d(off);
        d = warp_sum_d(d);
        lo = fmin(lo, d - off);
        hi = fmax(hi, d + off);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    // the block's bounds first, then one atomic pair per block (per-warp atomics on the two
    // words serialise in L2)
    __shared__ double slo[8], shi[8];
    __shared__ int sbad;
    const int w = threadIdx.x >> 5;
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    const bool wbad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
        slo[w] = lo;
        shi[w] = hi;
        if (wbad) sbad = 1;
    }
    __syncthreads();
    if (w == 0) {
        lo = lane < (int)(blockDim.x >> 5) ? slo[lane] : INFINITY;
        hi = lane < (int)(blockDim.x >> 5) ? shi[lane] : -INFINITY;
        for (int o = 16; o > 0; o >>= 1) {
            lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0) {
            if (sbad) atomicExch(&ctrl->status, GBE_ENUMERIC);
            if (lo <= hi) {
                atomicMin(&ctrl->eps_min_key, dkey(lo));
                atomicMax(&ctrl->eps_max_key, dkey(hi));
            }
        }
    }
}

// ----------------------------------------------------------------------------- gather
// Local index of a global site: open-addressing hash table (key = global index, value =
// local index; at most half full, so every probe sequence ends at an empty slot).
__device__ __forceinline__ unsigned gidx_hash(int g, int hbits) { return ((unsigned)g * 2654435761u) >> (32 - hbits); }

__device__ __forceinline__ int hash_local(const int2* htab, int hbits, int g) {
    const unsigned mask = (1u << hbits) - 1u;
    for (unsigned h = gidx_hash(g, hbits);; h = (h + 1u) & mask) {
        const int2 e = htab[h];
        if (e.x == g) return e.y;
        if (e.x == -1) return -1;
    }
}

// G CTAs (8 warps each) per subgraph, CTA `part` taking the groups of 8 consecutive rows
// a0..a0+7 with a0 = 8 part, 8 (part + G), ..., one row per warp:
// lanes map the row's H entries to local columns (a shared-memory hash table of the
// subgraph's sites), split them and scatter them into the warp's dense row buffer (4 split
// planes packed in 8 bytes per column, or the FP64 value; in shared memory, or for
// subgraphs too large for it in this CTA's slice rows_g of a global buffer).  X_0 is symmetric, so the
// 8 rows are also columns a0..a0+7: for the split planes the whole CTA then writes that
// 8-column group of every stored (upper) block, each thread one row r of it (16 contiguous
// bytes per plane; a warp covers 512 contiguous bytes).  The FP64 iterate (stored in full)
// is written row by row.  Every element of the padded tile is written, zeros included, so
// the planes need no separate clear.  Each CTA builds its own copy of the hash table and
// writes the trace sums of its rows as one partial (work unit s G + part).
template <int prec>
__global__ void __launch_bounds__(256) gather_kernel(Sp2Ctrl* ctrl, const int64_t* __restrict__ rowptr,
                                                     const int32_t* __restrict__ col, const double* __restrict__ val,
                                                     const int64_t* __restrict__ sub_ptr,
                                                     const int32_t* __restrict__ sub_idx, SubsGeom g, int max_mpad,
                                                     uint16_t* planes, int64_t plane_stride, double* f,
                                                     double* partials, int max_units, int htab_off, int hbits,
                                                     uint2* rows_g, int G) {
    extern __shared__ unsigned char gsm[];
    __shared__ double red[16];
    const int s = blockIdx.x / G, part = blockIdx.x % G;
    const int m = g.m[s], c = g.c[s], mpad = g.mpad[s];
    const int64_t off = g.off[s];
    const int64_t base = sub_ptr[s];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // [8][max_mpad] dense rows, then the m_s local -> global list
    uint2* rows8 = rows_g ? rows_g + (size_t)blockIdx.x * 8 * max_mpad : reinterpret_cast<uint2*>(gsm);
    uint2* rowbuf = rows8 + (size_t)warp * max_mpad;
    int32_t* sidx = reinterpret_cast<int32_t*>(gsm + (rows_g ? (size_t)0 : (size_t)8 * max_mpad * 8));
    int2* htab = reinterpret_cast<int2*>(gsm + htab_off);
    for (int i = threadIdx.x; i < (1 << hbits); i += blockDim.x) htab[i] = make_int2(-1, 0);
    __syncthreads();
    for (int a = threadIdx.x; a < m; a += blockDim.x) {
        const int gi = sub_idx[base + a];
        sidx[a] = gi;
        // the sites of a subgraph are distinct, so an empty slot is always found
        for (unsigned h = gidx_hash(gi, hbits);; h = (h + 1u) & ((1u << hbits) - 1u)) {
            if (atomicCAS(&htab[h].x, -1, gi) == -1) {
                htab[h].y = a;
                break;
            }
        }
    }
    __syncthreads();
    double emin, emax;
    if (ctrl->eps_given) { emin = ctrl->eps_min; emax = ctrl->eps_max; }
    else { emin = dkey_inv(ctrl->eps_min_key); emax = dkey_inv(ctrl->eps_max_key); }
    const double range = emax - emin;
    // SP2: X_0 = (emax I - H) / (emax - emin); Chebyshev: x = (H - a I) / b with a, b the
    // centre and half-width of [emin, emax]; both as x = (shift I - H) * gsc
    const bool foe = ctrl->foe != 0;
    const double half = 0.5 * range, centre = 0.5 * (emax + emin);
    const double shift = foe ? centre : emax;
    const double gsc = foe ? -1.0 / half : 1.0 / range;
    float ih = 0.f, il = 0.f;              // gsc as an FP32 pair (split paths)
    f64_to_f32_pair(gsc, ih, il);
    double t1 = 0.0, t2 = 0.0;
    float t2h = 0.f, t2l = 0.f;             // double-float Tr X_0^2 (split paths)
    // A lane takes the entries p0, p0 + 32, p0 + 64 of a row together (their loads issued at
    // once), then the next 96, in that order (the order the traces add them).  The first 96
    // entries of the warp's next row are loaded one iteration ahead and its row range two
    // iterations ahead, so that their latency overlaps the current rows' write-out.
    auto row_range = [&](int ar, int64_t& r0, int64_t& r1) {
        if (ar < m) {
            const int64_t gi = sidx[ar];
            r0 = rowptr[gi];
            r1 = rowptr[gi + 1];
        } else {
            r0 = 0;
            r1 = 0;
        }
    };
    auto load3 = [&](int64_t p0, int64_t r1, int (&cj)[3], double (&hv)[3]) {
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            const int64_t p = p0 + 32 * u;
            cj[u] = p < r1 ? col[p] : -1;
            hv[u] = p < r1 ? val[p] : 0.0;
        }
    };
    int64_t r0c, r1c, r0n, r1n;
    int cjc[3];
    double hvc[3];
    const int step = 8 * G;   // this CTA's groups of 8 rows: 8 part, 8 (part + G), ...
    row_range(8 * part + warp, r0c, r1c);
    load3(r0c + lane, r1c, cjc, hvc);
    row_range(8 * part + step + warp, r0n, r1n);
    for (int a0 = 8 * part; a0 < mpad; a0 += step) {
        const int a = a0 + warp;
        for (int b = lane; b < mpad; b += 32) rowbuf[b] = make_uint2(0u, 0u);
        __syncwarp();
        {
            const int64_t r0 = r0c, r1 = r1c;   // empty for a >= m
            for (int64_t p0 = r0 + lane; p0 < r1; p0 += 96) {
                int cj[3];
                double hv[3];
                if (p0 == r0 + lane) {
#pragma unroll
                    for (int u = 0; u < 3; ++u) { cj[u] = cjc[u]; hv[u] = hvc[u]; }
                } else {
                    load3(p0, r1, cj, hv);
                }
#pragma unroll
                for (int u = 0; u < 3; ++u) {
                    if (cj[u] < 0) continue;
                    const int b = hash_local(htab, hbits, cj[u]);
                    if (b < 0) continue;
                    const double h = hv[u];
                    uint2 packed;
                    if constexpr (prec == GBE_PREC_FP64 || prec == GBE_PREC_FP64TC) {
                        // the exact quotients, as the FP64 oracle computes them
                        const double x = foe ? (h - (a == b ? centre : 0.0)) / half : ((a == b ? emax : 0.0) - h) / range;
                        if (a < c) {
                            t2 += x * x;
                            if (a == b) t1 += x;
                        }
                        if constexpr (prec == GBE_PREC_FP64) {
                            packed = make_uint2((uint32_t)__double2loint(x), (uint32_t)__double2hiint(x));
                        } else {
                            // FP64TC: x on the fixed-point grid 2^-50 (digits cut at write-out)
                            const long long V = __double2ll_rn(x * 1125899906842624.0);
                            packed = make_uint2((uint32_t)(unsigned long long)V, (uint32_t)((unsigned long long)V >> 32));
                        }
                    } else {
                        // split paths need x to ~2^-35: off-diagonal x = -h / range as an FP32 pair
                        // product (no FP64 arithmetic: this part's FP64 pipe is narrow); the diagonal
                        // (one entry per row) in FP64
                        float xh, xl;
                        if (a == b) {
                            const double x = (shift - h) * gsc;
                            f64_to_f32_pair(x, xh, xl);
                            if (a < c) t1 += x;
                        } else {
                            float hh, hl;
                            f64_to_f32_pair(h, hh, hl);
                            neg_mul_pair(hh, hl, ih, il, xh, xl);
                        }
                        if (a < c) df_add_sq(t2h, t2l, xh, xl, 1.0f);
                        if constexpr (prec == GBE_PREC_FP16X6) {
                            const OzSplit o = oz_split_pq(xh, xl);
                            packed = make_uint2((uint32_t)o.s0 | ((uint32_t)o.s1 << 16), (uint32_t)o.s2 | ((uint32_t)o.s1s << 16));
                        } else {
                            const __nv_bfloat16 hi = __float2bfloat16_rn(xh);
                            const uint16_t lo = b_bits(__float2bfloat16_rn((xh - __bfloat162float(hi)) + xl));
                            packed = make_uint2((uint32_t)b_bits(hi) | ((uint32_t)lo << 16), 0u);
                        }
                    }
                    rowbuf[b] = packed;
                }
            }
        }
        // the next row's first entries and the range of the row after it
        load3(r0n + lane, r1n, cjc, hvc);
        r0c = r0n;
        r1c = r1n;
        row_range(a + 2 * step, r0n, r1n);
        if constexpr (prec == GBE_PREC_FP64) {
            __syncwarp();
            // row a, all column groups: 64 contiguous bytes per lane and group
            for (int gi8 = lane; gi8 < (mpad >> 3); gi8 += 32) {
                const int c0 = gi8 << 3;
                uint4* d = reinterpret_cast<uint4*>(f + blk_index(off, mpad, a, c0));
                const uint4* rb4 = reinterpret_cast<const uint4*>(rowbuf + c0);
#pragma unroll
                for (int k = 0; k < 4; ++k) d[k] = rb4[k];
            }
            __syncwarp();
        } else {
            __syncthreads();
            // columns a0..a0+7 (= rows a0..a0+7 by symmetry) of blocks I = 0..J, J = a0 / 128
            const int rows = ((a0 >> 7) + 1) << 7;
            for (int r = threadIdx.x; r < rows; r += blockDim.x) {
                uint2 u[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) u[k] = rows8[(size_t)k * max_mpad + r];
                if constexpr (prec == GBE_PREC_FP64TC) {
                    // ten digit planes of the 8 values (split.cuh)
                    uint32_t w10[GBE_F64TC_PLANES][4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const long long V0 = (long long)(((unsigned long long)u[2 * k].y << 32) | u[2 * k].x);
                        const long long V1 = (long long)(((unsigned long long)u[2 * k + 1].y << 32) | u[2 * k + 1].x);
                        uint32_t t[GBE_F64TC_PLANES];
                        f64tc_planes2(f64tc_digits(V0), f64tc_digits(V1), t);
#pragma unroll
                        for (int q = 0; q < GBE_F64TC_PLANES; ++q) w10[q][k] = t[q];
                    }
                    const int64_t e = blk_index(off, mpad, r, a0);
#pragma unroll
                    for (int q = 0; q < GBE_F64TC_PLANES; ++q)
                        *reinterpret_cast<uint4*>(planes + e + q * plane_stride) = make_uint4(w10[q][0], w10[q][1], w10[q][2], w10[q][3]);
                } else {
                uint32_t w[4][4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    w[0][k] = (u[2 * k].x & 0xffffu) | (u[2 * k + 1].x << 16);
                    w[1][k] = (u[2 * k].x >> 16) | (u[2 * k + 1].x & 0xffff0000u);
                    w[2][k] = (u[2 * k].y & 0xffffu) | (u[2 * k + 1].y << 16);
                    w[3][k] = (u[2 * k].y >> 16) | (u[2 * k + 1].y & 0xffff0000u);
                }
                const int64_t e = blk_index(off, mpad, r, a0);
                const int np = (prec == GBE_PREC_FP16X6) ? 4 : 2;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (q < np) *reinterpret_cast<uint4*>(planes + e + q * plane_stride) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
                }
            }
            __syncthreads();
        }
    }
    if constexpr (prec != GBE_PREC_FP64 && prec != GBE_PREC_FP64TC) t2 = (double)t2h + (double)t2l;
    double s1 = block_sum_d<256>(t1, red);
    double s2 = block_sum_d<256>(t2, red + 8);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = s1;
        partials[max_units + blockIdx.x] = s2;
        if (blockIdx.x == 0) { ctrl->eps_min = emin; ctrl->eps_max = emax; }
    }
}

// ----------------------------------------------------------------------------- init
// Control-block initialisation from parameters passed by value (no host staging, so
// consecutive runs enqueue without synchronising).
struct Sp2Init {
    int mode, fmt, n_min, n_max, branch_mode, seq_len, fp64_tail, prec, eps_given, foe, cur;
    double eps_min, eps_max, n_occ, idem_tol, tail_switch, out_scale;
    long long timeout_cycles;
    uint8_t seq_in[GBE_SEQ_MAX];
};

__global__ void init_ctrl_kernel(Sp2Ctrl* C, Sp2Init in) {
    // zero the whole block, then set the run's parameters
    uint32_t* w = reinterpret_cast<uint32_t*>(C);
    for (int i = threadIdx.x; i < (int)(sizeof(Sp2Ctrl) / 4); i += blockDim.x) w[i] = 0u;
    __syncthreads();
    for (int i = threadIdx.x; i < GBE_SEQ_MAX; i += blockDim.x) C->seq_in[i] = in.seq_in[i];
    if (threadIdx.x == 0) {
        C->mode = in.mode; C->fmt = in.fmt; C->switch_iter = -1;
        C->n_min = in.n_min; C->n_max = in.n_max; C->branch_mode = in.branch_mode; C->seq_len = in.seq_len;
        C->fp64_tail = in.fp64_tail; C->prec = in.prec; C->eps_given = in.eps_given;
        C->eps_min = in.eps_min; C->eps_max = in.eps_max;
        C->eps_min_key = ~0ull; C->eps_max_key = 0ull;
        C->n_occ = in.n_occ; C->idem_tol = in.idem_tol; C->tail_switch = in.tail_switch;
        C->timeout_cycles = in.timeout_cycles;
        C->foe = in.foe;
        C->cur = in.cur;
        C->out_scale = in.out_scale;
    }
}

// ----------------------------------------------------------------------------- decide
// Per-subgraph trace sums of this rank at global subgraph positions (zeros at other ranks'
// positions) and its error flag: the buffer a sharded run's exchange sums over the ranks.
__global__ void __launch_bounds__(256) sub_sums_kernel(const Sp2Ctrl* ctrl, const double* __restrict__ partials,
                                                       int max_units, const int2* __restrict__ ranges,
                                                       const int32_t* __restrict__ local_of, int64_t P_global,
                                                       double* sums) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < P_global; g += (int64_t)gridDim.x * blockDim.x) {
        const int s = local_of ? local_of[g] : (int)g;
        double a = 0.0, b = 0.0;
        if (s >= 0) sub_trace(partials, max_units, ranges[s], a, b);
        sums[g] = a;
        sums[P_global + g] = b;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) sums[2 * P_global] = (ctrl->status != GBE_OK) ? 1.0 : 0.0;
}

// Global FP64 traces over core positions -> stop rule and branch of the next step
// (decide.cuh).  The traces are the per-subgraph sums added in global subgraph order, taken
// from this rank's partials (sums == NULL) or from the exchanged buffer of a sharded run.
// A kernel whose step did no work (the run had stopped, or the other precision's kernel
// ran) leaves the state alone.  In a graph-launched
// run the last decision of a loop iteration (set_cond) also sets the loop node's condition.
__global__ void __launch_bounds__(kDecideThreads) decide_kernel(Sp2Ctrl* ctrl, DecideIn in,
                                                                cudaGraphConditionalHandle cond, int set_cond) {
    __shared__ double red[16];
    __shared__ int run;
    if (threadIdx.x == 0) run = (in.kind == 0) ? 1 : ctrl->pending;
    __syncthreads();
    if (run) {
        double t1, t2;
        decide_traces(in, threadIdx.x, red, [] { __syncthreads(); }, t1, t2);
        if (threadIdx.x == 0) decide_apply(ctrl, in, t1, t2);
    }
    if (set_cond && threadIdx.x == 0) {
        __threadfence_block();
        decide_set_condition(ctrl, cond);
    }
}

// ----------------------------------------------------------------------------- FP64 squaring
// 64 x 64 output tiles (I <= J) of X_{n+1} = f(X_n) per subgraph, DFMA with register
// blocking; the branch is applied in the epilogue and the tile is mirrored to (J, I).
// FP32 -> FP64 widening with integer operations only (exact for zero and normal floats,
// which every split plane value and the partial sums below are).
__device__ __forceinline__ double f32_to_f64_int(float x) {
    const uint32_t u = __float_as_uint(x);
    const uint32_t e = (u >> 23) & 0xFFu;
    if (e == 0) return 0.0;
    const unsigned long long b = ((unsigned long long)(u >> 31) << 63) | ((unsigned long long)(e + 896u) << 52) |
                                 ((unsigned long long)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)b);
}

// The values of oz_value / bf_value with at most one FP64 addition (the narrow FP64 pipe is
// what bounds an element-wise pass over the planes): s1 + s2 is exact in FP32 (s2 is the
// fp16 rounding residual of s1, the two significands span at most 22 bits), and the sums
// are exact in FP64.
// FP16X6 without any FP64 instruction: s0 = k0 2^-10 and s1 + s2 = R 2^-24 exactly (fp16
// values on the split's grids), so x = (k0 2^25 + R) 2^-35 with an integer below 2^36 that
// is normalised into the FP64 bit pattern directly.
__device__ __forceinline__ double oz_value_fast(uint16_t s0, uint16_t s1, uint16_t s2) {
    const long long k0 = (long long)__float2int_rn(h_val(s0) * 1024.0f);
    const long long R = (long long)__float2int_rn((h_val(s1) + h_val(s2)) * 16777216.0f);
    const long long total = (k0 << 25) + R;
    if (total == 0) return 0.0;
    const unsigned long long sign = total < 0 ? 1ull : 0ull;
    const unsigned long long mag = (unsigned long long)(total < 0 ? -total : total);
    const int e = 63 - __clzll((long long)mag);   // top bit, below 36
    const unsigned long long mant = (mag << (52 - e)) & 0xFFFFFFFFFFFFFull;
    return __longlong_as_double((long long)((sign << 63) | ((unsigned long long)(e - 35 + 1023) << 52) | mant));
}

__device__ __forceinline__ double bf_value_fast(uint16_t hi, uint16_t lo) {
    return f32_to_f64_int(b_val(hi)) + f32_to_f64_int(b_val(lo));
}

__device__ __forceinline__ double load_x(int fmt, int prec, const uint16_t* pl, int64_t ps, const double* f,
                                         int64_t off, int mpad, int r, int c) {
    if (fmt == 1) return f[blk_index(off, mpad, r, c)];
    const int64_t e = sym_index(off, mpad, r, c);
    if (prec == GBE_PREC_FP16X6) return oz_value(pl[e], pl[e + ps], pl[e + 2 * ps]);
    if (prec == GBE_PREC_FP64TC)
        return (double)f64tc_from_planes(pl[e + ps], pl[e + 2 * ps], pl[e + 3 * ps], pl[e + 4 * ps], pl[e + 8 * ps]) *
               8.881784197001252e-16;   // 2^-50
    return bf_value(pl[e], pl[e + ps]);
}

__global__ void __launch_bounds__(256) square_fp64_kernel(Sp2Ctrl* ctrl, SubsGeom g,
                                                          const TileItem* __restrict__ items, int n_items,
                                                          uint16_t* planes0, uint16_t* planes1,
                                                          int64_t plane_stride, double* f0, double* f1,
                                                          double* partials, int max_units, int slot) {
    __shared__ double As[2][16][64];
    __shared__ double Bs[2][16][64];
    __shared__ double red[8];
    __shared__ int hdr[5];
    if (threadIdx.x == 0) {
        hdr[0] = (ctrl->stop == 0 && ctrl->mode == 1);
        hdr[1] = ctrl->cur;
        hdr[2] = ctrl->fmt;
        hdr[3] = ctrl->branch;
        hdr[4] = ctrl->prec;
    }
    __syncthreads();
    if (!hdr[0]) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctrl->pending = 1;
        if (slot >= 0) ctrl->slot_ran[slot] |= 2;   // launch slots (profiled runs) only
    }
    const int cur = hdr[1], fmt = hdr[2], branch = hdr[3], prec = hdr[4];
    const uint16_t* pin = cur ? planes1 : planes0;
    const double* fin = cur ? f1 : f0;
    double* fout = cur ? f0 : f1;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int lr = threadIdx.x >> 2, lk = (threadIdx.x & 3) * 4;

    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const TileItem w = items[it];
        const int mpad = g.mpad[w.s], m = g.m[w.s], c = g.c[w.s];
        const int64_t off = g.off[w.s];
        const int kend = (m + 15) & ~15;
        double acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
        const int ra = w.I * 64 + lr, rb = w.J * 64 + lr;
        double va[4], vb[4];
        auto fetch = [&](int k0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                va[q] = load_x(fmt, prec, pin, plane_stride, fin, off, mpad, ra, k0 + lk + q);
                vb[q] = load_x(fmt, prec, pin, plane_stride, fin, off, mpad, rb, k0 + lk + q);
            }
        };
        fetch(0);
        int buf = 0;
        for (int k0 = 0; k0 < kend; k0 += 16) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                As[buf][lk + q][lr] = va[q];
                Bs[buf][lk + q][lr] = vb[q];
            }
            __syncthreads();
            if (k0 + 16 < kend) fetch(k0 + 16);
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                double a[4], b[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j) b[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
            buf ^= 1;
        }
        double t1 = 0.0, t2 = 0.0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = w.I * 64 + ty + 16 * i;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int cc = w.J * 64 + tx + 16 * j;
                const int64_t e = blk_index(off, mpad, r, cc);
                double x = acc[i][j];
                if (!branch) x = 2.0 * load_x(fmt, prec, pin, plane_stride, fin, off, mpad, r, cc) - x;
                fout[e] = x;
                if (w.I != w.J) fout[blk_index(off, mpad, cc, r)] = x;
                const int wgt = (r < c) + ((w.I != w.J) && (cc < c));
                t2 += wgt * (x * x);
                if (r == cc && r < c) t1 += x;
            }
        }
        double s1 = block_sum_d<256>(t1, red);
        double s2 = block_sum_d<256>(t2, red);
        if (threadIdx.x == 0) {
            partials[it] = s1;
            partials[max_units + it] = s2;
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------- Chebyshev step (FP64)
// Every 64 x 64 output tile (I, J) of out = alpha x b - c + gamma I with x (side fx,
// symmetric) and b (side fb) multiplied as they are: x and b commute only up to rounding,
// and computing upper tiles and mirroring them would turn that rounding into a growing
// error of the recurrence.  c is read from and overwritten in fc (each tile only its own
// elements, so the update is in place).
__global__ void __launch_bounds__(256) cheb_fp64_kernel(SubsGeom g, const TileItem* __restrict__ items, int n_items,
                                                        const double* __restrict__ fx, const double* __restrict__ fb,
                                                        double* fc, double alpha, double gamma) {
    __shared__ double As[2][16][64];
    __shared__ double Bs[2][16][64];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int lr = threadIdx.x >> 2, lk = (threadIdx.x & 3) * 4;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const TileItem w = items[it];
        const int mpad = g.mpad[w.s], m = g.m[w.s];
        const int64_t off = g.off[w.s];
        const int kend = (m + 15) & ~15;
        double acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
        const int ra = w.I * 64 + lr, rb = w.J * 64 + lr;
        double va[4], vb[4];
        auto fetch = [&](int k0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                va[q] = fx[blk_index(off, mpad, ra, k0 + lk + q)];
                vb[q] = fb[blk_index(off, mpad, k0 + lk + q, rb)];   // b[k][column rb]
            }
        };
        fetch(0);
        int buf = 0;
        for (int k0 = 0; k0 < kend; k0 += 16) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                As[buf][lk + q][lr] = va[q];
                Bs[buf][lk + q][lr] = vb[q];
            }
            __syncthreads();
            if (k0 + 16 < kend) fetch(k0 + 16);
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                double a[4], b[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j) b[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
            buf ^= 1;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = w.I * 64 + ty + 16 * i;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int cc = w.J * 64 + tx + 16 * j;
                const int64_t e = blk_index(off, mpad, r, cc);
                fc[e] = alpha * acc[i][j] - fc[e] + (r == cc ? gamma : 0.0);
            }
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------- assembly
// One CTA per subgraph, one warp per core column j: ELL row idx_s[j] <- (idx_s[k], x_s[j,k]).
__global__ void __launch_bounds__(256) assemble_kernel(const Sp2Ctrl* ctrl, const int64_t* __restrict__ sub_ptr,
                                                       const int32_t* __restrict__ sub_idx, SubsGeom g,
                                                       const uint16_t* planes0, const uint16_t* planes1,
                                                       int64_t plane_stride, const double* f0, const double* f1,
                                                       int64_t width, int32_t* ell_col, double* ell_val,
                                                       double drop_tol, int jblocks) {
    // jblocks CTAs per subgraph, one core column (ELL row) per warp
    const int s = blockIdx.x / jblocks, j = (blockIdx.x % jblocks) * 8 + (threadIdx.x >> 5);
    const int m = g.m[s], c = g.c[s], mpad = g.mpad[s];
    const int64_t off = g.off[s], base = sub_ptr[s];
    const int cur = ctrl->cur, fmt = ctrl->fmt, prec = ctrl->prec;
    const double scale = ctrl->out_scale;
    const uint16_t* pl = cur ? planes1 : planes0;
    const double* f = cur ? f1 : f0;
    const int lane = threadIdx.x & 31;
    __shared__ double abuf[8][32 * 9];
    if (j < c && drop_tol <= 0.0) {
        // every entry kept, in local order: lane takes 8 consecutive k; in an upper block
        // they are one 16-byte run per plane (64 bytes of FP64)
        const int64_t row = sub_idx[base + j];
        int32_t* oc = ell_col + row * width;
        double* ov = ell_val + row * width;
        const int jb = j >> 7;
        const bool unit_scale = (scale == 1.0);
        for (int kb0 = 0; kb0 < m; kb0 += 256) {   // warp-uniform trip count
            const int k0 = kb0 + 8 * lane;
            double v[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            if (k0 >= m) {
                // past the row's end: nothing to load (k0 + 7 < mpad holds for k0 < m only)
            } else if ((k0 >> 7) >= jb) {
                const int64_t e = blk_index(off, mpad, j, k0);
                if (fmt == 1) {
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const double2 d2 = reinterpret_cast<const double2*>(f + e)[t];
                        v[2 * t] = d2.x;
                        v[2 * t + 1] = d2.y;
                    }
                } else if (prec == GBE_PREC_FP64TC) {
                    uint4 dg[5];
#pragma unroll
                    for (int p = 0; p < 5; ++p) dg[p] = *reinterpret_cast<const uint4*>(pl + (p < 4 ? p + 1 : 8) * plane_stride + e);
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const int sh = 16 * (t & 1);
                        auto hw = [&](const uint4& u) {
                            const int q = t >> 1;
                            return (uint16_t)((q == 0 ? u.x : (q == 1 ? u.y : (q == 2 ? u.z : u.w))) >> sh);
                        };
                        v[t] = (double)f64tc_from_planes(hw(dg[0]), hw(dg[1]), hw(dg[2]), hw(dg[3]), hw(dg[4])) *
                               8.881784197001252e-16;
                    }
                } else if (prec == GBE_PREC_FP16X6) {
                    const uint4 a = *reinterpret_cast<const uint4*>(pl + e);
                    const uint4 b = *reinterpret_cast<const uint4*>(pl + plane_stride + e);
                    const uint4 cc = *reinterpret_cast<const uint4*>(pl + 2 * plane_stride + e);
                    const uint32_t aw[4] = {a.x, a.y, a.z, a.w}, bw[4] = {b.x, b.y, b.z, b.w},
                                   cw[4] = {cc.x, cc.y, cc.z, cc.w};
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const int sh = 16 * (t & 1);
                        v[t] = oz_value_fast((uint16_t)(aw[t >> 1] >> sh), (uint16_t)(bw[t >> 1] >> sh),
                                             (uint16_t)(cw[t >> 1] >> sh));
                    }
                } else {
                    const uint4 a = *reinterpret_cast<const uint4*>(pl + e);
                    const uint4 b = *reinterpret_cast<const uint4*>(pl + plane_stride + e);
                    const uint32_t aw[4] = {a.x, a.y, a.z, a.w}, bw[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const int sh = 16 * (t & 1);
                        v[t] = bf_value_fast((uint16_t)(aw[t >> 1] >> sh), (uint16_t)(bw[t >> 1] >> sh));
                    }
                }
            } else {
#pragma unroll
                for (int t = 0; t < 8; ++t) v[t] = load_x(fmt, prec, pl, plane_stride, f, off, mpad, j, k0 + t);
            }
            // through shared memory (rows of 9 doubles: at most 2-way bank conflicts) so that
            // each store instruction writes 32 consecutive entries of the ELL row
            double* tb = abuf[threadIdx.x >> 5];
            __syncwarp();
#pragma unroll
            for (int t = 0; t < 8; ++t) tb[9 * lane + t] = v[t];
            __syncwarp();
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int pidx = lane + 32 * q, k = kb0 + pidx;
                if (k < m) {
                    const double x = tb[9 * (pidx >> 3) + (pidx & 7)];
                    oc[k] = sub_idx[base + k];
                    ov[k] = unit_scale ? x : x * scale;
                }
            }
        }
        for (int p = m + lane; p < width; p += 32) {
            oc[p] = -1;
            ov[p] = 0.0;
        }
    } else if (j < c) {
        const int64_t row = sub_idx[base + j];
        int32_t* oc = ell_col + row * width;
        double* ov = ell_val + row * width;
        int pos = 0;
        for (int k0 = 0; k0 < m; k0 += 32) {
            const int k = k0 + lane;
            double v = 0.0;
            int gk = -1;
            if (k < m) {
                v = load_x(fmt, prec, pl, plane_stride, f, off, mpad, j, k) * scale;
                gk = sub_idx[base + k];
            }
            const bool keep = (k < m) && !(drop_tol > 0.0 && fabs(v) < drop_tol);
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int p = pos + __popc(bal & ((1u << lane) - 1u));
                oc[p] = gk;
                ov[p] = v;
            }
            pos += __popc(bal);
        }
        for (int p = pos + lane; p < width; p += 32) {
            oc[p] = -1;
            ov[p] = 0.0;
        }
    }
}

__global__ void fill_ell_kernel(int64_t total, int32_t* col, double* val) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        col[i] = -1;
        val[i] = 0.0;
    }
}

__global__ void export_kernel(const Sp2Ctrl* ctrl, SubsGeom g, int s, const uint16_t* planes0,
                              const uint16_t* planes1, int64_t plane_stride, const double* f0, const double* f1,
                              double* out) {
    const int m = g.m[s], mpad = g.mpad[s];
    const int64_t off = g.off[s];
    const int cur = ctrl->cur, fmt = ctrl->fmt, prec = ctrl->prec;
    const uint16_t* pl = cur ? planes1 : planes0;
    const double* f = cur ? f1 : f0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)m * m; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / m), cc = (int)(i % m);
        out[i] = load_x(fmt, prec, pl, plane_stride, f, off, mpad, r, cc) * ctrl->out_scale;
    }
}

// ============================================================================= host side
static SubsGeom geom_of(const gbe_subs* X) { return SubsGeom{X->d_off, X->d_mpad, X->d_m, X->d_c}; }

extern "C" int gbe_parts_import(gbe_ctx* ctx, int64_t n, int64_t P, const int32_t* core_count,
                                const int64_t* sub_ptr, const int32_t* sub_idx, gbe_parts** out) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && out && core_count && sub_ptr && sub_idx, "NULL argument");
    GBE_CHECK_ARG(n > 0 && n < INT32_MAX && P > 0, "bad sizes");
    GBE_CHECK_ARG(sub_ptr[0] == 0, "sub_ptr[0] must be 0");
    int64_t max_m = 0;
    for (int64_t s = 0; s < P; ++s) {
        const int64_t m = sub_ptr[s + 1] - sub_ptr[s];
        GBE_CHECK_ARG(m > 0, "empty subgraph");
        GBE_CHECK_ARG(core_count[s] > 0 && core_count[s] <= m, "core count out of range");
        max_m = std::max(max_m, m);
    }
    const int64_t total = sub_ptr[P];
    for (int64_t i = 0; i < total; ++i) GBE_CHECK_ARG(sub_idx[i] >= 0 && sub_idx[i] < n, "sub_idx out of range");
    GBE_CUDA_TRY(cudaSetDevice(ctx->device));
    // do the cores partition the vertices (then every row of D is written by one subgraph)?
    int cover = 1;
    {
        std::vector<uint8_t> seen((size_t)n, 0);
        int64_t cores = 0;
        for (int64_t s = 0; s < P && cover; ++s)
            for (int64_t i = sub_ptr[s]; i < sub_ptr[s] + core_count[s]; ++i) {
                if (seen[sub_idx[i]]) { cover = 0; break; }
                seen[sub_idx[i]] = 1;
                ++cores;
            }
        if (cores != n) cover = 0;
    }
    gbe_parts* p = new gbe_parts();
    p->n = n; p->P = P; p->total = total; p->max_m = max_m;
    p->cores_cover = cover;
    p->h_core_count.assign(core_count, core_count + P);
    p->h_sub_ptr.assign(sub_ptr, sub_ptr + P + 1);
    int r = GBE_OK;
    if ((r = gbe_alloc((void**)&p->d_core_count, P * 4)) != GBE_OK ||
        (r = gbe_alloc((void**)&p->d_sub_ptr, (P + 1) * 8)) != GBE_OK ||
        (r = gbe_alloc((void**)&p->d_sub_idx, total * 4)) != GBE_OK) {
        gbe_free_parts(p);
        return r;
    }
    cudaMemcpyAsync(p->d_core_count, core_count, P * 4, cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(p->d_sub_ptr, sub_ptr, (P + 1) * 8, cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(p->d_sub_idx, sub_idx, total * 4, cudaMemcpyHostToDevice, ctx->stream);
    GBE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    *out = p;
    return GBE_OK;
}

extern "C" int gbe_parts_info(const gbe_parts* p, int64_t* P, int64_t* total, int64_t* max_m) {
    GBE_CHECK_ARG(p != nullptr, "parts is NULL");
    if (P) *P = p->P;
    if (total) *total = p->total;
    if (max_m) *max_m = p->max_m;
    return GBE_OK;
}

extern "C" int gbe_parts_export(gbe_ctx* ctx, const gbe_parts* p, int32_t* core_count, int64_t* sub_ptr,
                                int32_t* sub_idx) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && p, "NULL argument");
    if (core_count) memcpy(core_count, p->h_core_count.data(), p->P * 4);
    if (sub_ptr) memcpy(sub_ptr, p->h_sub_ptr.data(), (p->P + 1) * 8);
    if (sub_idx) {
        GBE_CUDA_TRY(cudaMemcpyAsync(sub_idx, p->d_sub_idx, p->total * 4, cudaMemcpyDeviceToHost, ctx->stream));
        GBE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    }
    return GBE_OK;
}

extern "C" int gbe_free_parts(gbe_parts* p) {
    if (!p) return GBE_OK;
    gbe_free(p->d_core_count);
    gbe_free(p->d_sub_ptr);
    gbe_free(p->d_sub_idx);
    gbe_free(p->d_local_of);
    delete p;
    return GBE_OK;
}

extern "C" int gbe_shard_assign(int64_t P, const int64_t* sub_ptr, int world, int32_t* owner, double* load) {
    GBE_CHECK_ARG(sub_ptr && owner && P >= 1 && world >= 1, "bad argument");
    std::vector<double> cost(P);
    for (int64_t s = 0; s < P; ++s) {
        const double m = (double)(sub_ptr[s + 1] - sub_ptr[s]);
        GBE_CHECK_ARG(m >= 1, "empty subgraph");
        cost[s] = m * m * m;
    }
    std::vector<int64_t> order(P);
    for (int64_t s = 0; s < P; ++s) order[s] = s;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return cost[a] > cost[b]; });
    std::vector<double> ld(world, 0.0);
    for (int64_t s : order) {
        int best = 0;
        for (int r = 1; r < world; ++r)
            if (ld[r] < ld[best]) best = r;
        owner[s] = best;
        ld[best] += cost[s];
    }
    if (load)
        for (int r = 0; r < world; ++r) load[r] = ld[r];
    return GBE_OK;
}

extern "C" int gbe_parts_shard(gbe_ctx* ctx, const gbe_parts* parts, const int32_t* owner, int rank, gbe_parts** local) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && parts && owner && local, "NULL argument");
    GBE_CHECK_ARG(parts->h_global_id.empty(), "a shard cannot be sharded again");
    const int64_t P = parts->P;
    std::vector<int32_t> idx(parts->total);
    GBE_CUDA_TRY(cudaSetDevice(ctx->device));
    GBE_CUDA_TRY(cudaMemcpyAsync(idx.data(), parts->d_sub_idx, parts->total * 4, cudaMemcpyDeviceToHost, ctx->stream));
    GBE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    std::vector<int32_t> cc;
    std::vector<int64_t> sp(1, 0), gid;
    std::vector<int32_t> si;
    std::vector<int32_t> local_of(P, -1);
    for (int64_t s = 0; s < P; ++s) {
        if (owner[s] != rank) continue;
        local_of[s] = (int32_t)gid.size();
        gid.push_back(s);
        cc.push_back(parts->h_core_count[s]);
        si.insert(si.end(), idx.begin() + parts->h_sub_ptr[s], idx.begin() + parts->h_sub_ptr[s + 1]);
        sp.push_back((int64_t)si.size());
    }
    GBE_CHECK_ARG(!gid.empty(), "this rank owns no subgraph");
    gbe_parts* p = nullptr;
    GBE_TRY(gbe_parts_import(ctx, parts->n, (int64_t)gid.size(), cc.data(), sp.data(), si.data(), &p));
    p->P_global = P;
    p->h_global_id = gid;
    int r = gbe_alloc((void**)&p->d_local_of, P * 4);
    if (r != GBE_OK) {
        gbe_free_parts(p);
        return r;
    }
    cudaError_t e = cudaMemcpyAsync(p->d_local_of, local_of.data(), P * 4, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        gbe_free_parts(p);
        gbe_set_error("gbe_parts_shard: %s", cudaGetErrorString(e));
        return GBE_ECUDA;
    }
    *local = p;
    return GBE_OK;
}

static void drop_graphs(gbe_subs* X);

extern "C" int gbe_free_subs(gbe_subs* X) {
    if (!X) return GBE_OK;
    gbe_free(X->d_off); gbe_free(X->d_mpad); gbe_free(X->d_m); gbe_free(X->d_c);
    for (int i = 0; i < 3; ++i) { gbe_free(X->planes[i]); gbe_free(X->f64[i]); }
    gbe_free(X->d_items_tc); gbe_free(X->d_items_64); gbe_free(X->d_partials); gbe_free(X->d_ctrl);
    gbe_free(X->d_items_tc_full); gbe_free(X->d_items_64_full);
    gbe_free(X->d_cta_ptr);
    for (int k = 0; k < 3; ++k) gbe_free(X->d_ranges[k]);
    gbe_free(X->d_sums);
    gbe_free(X->d_gather_rows);
    if (X->h_ctrl) cudaFreeHost(X->h_ctrl);
    for (int i = 0; i < 3; ++i) if (X->ev[i]) cudaEventDestroy(X->ev[i]);
    for (auto e : X->ev_tc) cudaEventDestroy(e);
    for (auto e : X->ev_64) cudaEventDestroy(e);
    drop_graphs(X);
    if (X->cap_stream) cudaStreamDestroy(X->cap_stream);
    delete X;
    return GBE_OK;
}

// FP64 iterates of both ping-pong sides, allocated (and cleared) on first use.
static int ensure_f64(gbe_subs* X, cudaStream_t st) {
    for (int i = 0; i < 2; ++i)
        if (!X->f64[i]) {
            GBE_TRY(gbe_alloc((void**)&X->f64[i], X->total_elems * 8));
            GBE_CUDA_TRY(cudaMemsetAsync(X->f64[i], 0, X->total_elems * 8, st));
        }
    return GBE_OK;
}

static void make_items(const std::vector<int32_t>& dim, const std::vector<int32_t>& cost, int tile,
                       std::vector<TileItem>& items, bool full = false) {
    items.clear();
    const int64_t P = (int64_t)dim.size();
    std::vector<int64_t> order(P);
    for (int64_t s = 0; s < P; ++s) order[s] = s;
    // longest K first, so a static round-robin over persistent CTAs stays balanced
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return cost[a] > cost[b]; });
    for (int64_t s : order) {
        const int T = (dim[s] + tile - 1) / tile;
        for (int I = 0; I < T; ++I)
            for (int J = full ? 0 : I; J < T; ++J) items.push_back(TileItem{(int)s, I, J, 0});
    }
}

// The number of items make_items builds for these arguments, and (rg non-NULL) each
// subgraph's contiguous range of them, without building the list.
static int64_t item_ranges(const std::vector<int32_t>& dim, const std::vector<int32_t>& cost, int tile, bool full,
                           std::vector<int2>* rg) {
    const int64_t P = (int64_t)dim.size();
    std::vector<int64_t> order(P);
    for (int64_t s = 0; s < P; ++s) order[s] = s;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return cost[a] > cost[b]; });
    int64_t n = 0;
    for (int64_t s : order) {
        const int64_t T = (dim[s] + tile - 1) / tile;
        const int64_t c = full ? T * T : T * (T + 1) / 2;
        if (rg) (*rg)[s] = make_int2((int)n, (int)c);
        n += c;
    }
    return n;
}

// A device tile list built on first use: the 64-row tiles of the FP64 squaring (full = false)
// or every 128- and 64-row tile of a Chebyshev expansion (full = true).  Enqueued on the
// context's stream, outside any capture.
static int ensure_items(gbe_ctx* ctx, gbe_subs* X, bool full) {
    std::vector<int32_t> m64(X->h_m.begin(), X->h_m.end());
    std::vector<TileItem> it;
    if (!full && !X->d_items_64) {
        make_items(m64, X->h_mpad, 64, it);
        GBE_TRY(gbe_alloc((void**)&X->d_items_64, std::max<size_t>(1, it.size()) * sizeof(TileItem)));
        if (!it.empty())
            GBE_CUDA_TRY(cudaMemcpyAsync(X->d_items_64, it.data(), it.size() * sizeof(TileItem), cudaMemcpyHostToDevice,
                                         ctx->stream));
    }
    if (full && !X->d_items_tc_full) {
        make_items(X->h_mpad, X->h_mpad, 128, it, true);
        GBE_TRY(gbe_alloc((void**)&X->d_items_tc_full, std::max<size_t>(1, it.size()) * sizeof(TileItem)));
        if (!it.empty())
            GBE_CUDA_TRY(cudaMemcpyAsync(X->d_items_tc_full, it.data(), it.size() * sizeof(TileItem),
                                         cudaMemcpyHostToDevice, ctx->stream));
    }
    if (full && !X->d_items_64_full) {
        make_items(m64, X->h_mpad, 64, it, true);
        GBE_TRY(gbe_alloc((void**)&X->d_items_64_full, std::max<size_t>(1, it.size()) * sizeof(TileItem)));
        if (!it.empty())
            GBE_CUDA_TRY(cudaMemcpyAsync(X->d_items_64_full, it.data(), it.size() * sizeof(TileItem),
                                         cudaMemcpyHostToDevice, ctx->stream));
    }
    return GBE_OK;
}

// Dynamic shared memory of the gather: 8 dense rows, the local->global list, and a hash
// table of >= 2 m slots (global -> local).  Subgraphs up to 2432 vertices keep the rows in
// the 227 KB of a GB300 CTA; larger ones stage them in global memory (L2) and keep the list
// and the hash table in shared memory, up to 8192 vertices.
struct GatherLayout {
    size_t smem;
    int htab_off, hbits;
    bool rows_global;
};
static GatherLayout gather_layout(const gbe_ctx* ctx, const gbe_subs* X) {
    GatherLayout L;
    const int64_t max_m = X->parts->max_m;
    L.hbits = 6;
    while ((1ll << L.hbits) < 2 * max_m) ++L.hbits;
    L.rows_global = false;
    L.htab_off = (int)((((size_t)8 * X->max_mpad * 8 + (size_t)max_m * 4) + 7) & ~(size_t)7);
    L.smem = (size_t)L.htab_off + ((size_t)8 << L.hbits);
    if ((int64_t)L.smem > (int64_t)ctx->smem_optin) {
        L.rows_global = true;
        L.htab_off = (int)(((size_t)max_m * 4 + 7) & ~(size_t)7);
        L.smem = (size_t)L.htab_off + ((size_t)8 << L.hbits);
    }
    return L;
}

// CTAs of the gather per subgraph: enough CTAs for about eight per SM, each keeping at
// least two groups of 8 rows of the smallest padded subgraph.
static int gather_split_of(const gbe_ctx* ctx, const gbe_subs* X, const GatherLayout& L) {
    if (L.rows_global || X->P <= 0) return 1;
    int min_mpad = X->max_mpad;
    for (int64_t s = 0; s < X->P; ++s) min_mpad = std::min(min_mpad, X->h_mpad[s]);
    const int64_t target = 8ll * ctx->sm_count;
    int G = (int)std::min<int64_t>(8, (target + X->P - 1) / X->P);
    G = std::min(G, std::max(1, min_mpad / 16));
    return std::max(1, G);
}

extern "C" int gbe_subs_create(gbe_ctx* ctx, const gbe_parts* parts, int prec, gbe_subs** out) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && parts && out, "NULL argument");
    GBE_CHECK_ARG(prec == GBE_PREC_FP64 || prec == GBE_PREC_FP16X6 || prec == GBE_PREC_BF16X3 || prec == GBE_PREC_FP64TC,
                  "unknown prec");
    GBE_CUDA_TRY(cudaSetDevice(ctx->device));
    gbe_subs* X = new gbe_subs();
    X->parts = parts;
    X->prec = prec;
    X->P = parts->P;
    X->h_off.resize(X->P); X->h_mpad.resize(X->P); X->h_m.resize(X->P); X->h_c.resize(X->P);
    int64_t total = 0;
    double alg = 0.0, mma = 0.0, f64 = 0.0, mma_full = 0.0, f64_full = 0.0;
    const int nprod = (prec == GBE_PREC_FP16X6) ? 6 : (prec == GBE_PREC_FP64TC ? 18 : 3);
    const int kcw = (prec == GBE_PREC_FP64TC) ? 16 : 32;   // K-chunk width of the tensor-core kernel
    for (int64_t s = 0; s < X->P; ++s) {
        const int m = (int)(parts->h_sub_ptr[s + 1] - parts->h_sub_ptr[s]);
        const int mpad = (m + 127) & ~127;
        X->h_m[s] = m; X->h_mpad[s] = mpad; X->h_c[s] = parts->h_core_count[s];
        X->h_off[s] = total;
        total += (int64_t)mpad * mpad;
        X->max_mpad = std::max(X->max_mpad, mpad);
        alg += 2.0 * (double)m * m * m;
        // executed MMA work: K in steps of 16 (a squaring skips an all-padding second half of
        // its last chunk), the last column block only up to the next multiple of 16 past m;
        // a Chebyshev step runs whole chunks and whole tiles
        const int T = mpad / 128, kk = (m + kcw - 1) / kcw * kcw, kt = (m + 15) & ~15;
        const int nlast = ((m - 128 * (T - 1) + 15) >> 4) << 4;
        mma += (double)nprod * 2.0 * 128.0 * kt * (128.0 * (T - 1) * T / 2 + (double)nlast * T);
        mma_full += (double)nprod * 2.0 * 128.0 * 128.0 * kk * (T * T);
        const int T64 = (m + 63) / 64, k16 = (m + 15) & ~15;
        f64 += 2.0 * 64.0 * 64.0 * k16 * (T64 * (T64 + 1) / 2);
        f64_full += 2.0 * 64.0 * 64.0 * k16 * (T64 * T64);
    }
    X->total_elems = total;
    X->alg_flops_per_iter = alg;
    X->mma_flops_per_iter = mma;
    X->fp64_flops_per_iter = f64;
    X->mma_flops_full = mma_full;
    X->fp64_flops_full = f64_full;
    // the 128-row tiles of the squaring now; the 64-row tiles of FP64 steps and the full tile
    // lists of a Chebyshev expansion are built on first use (ensure_items), only their
    // counts and ranges here.  Work units of each subgraph per decision kind: the tiles of a
    // subgraph are contiguous in its list.
    std::vector<TileItem> it_tc;
    std::vector<int32_t> m64(X->h_m.begin(), X->h_m.end());
    make_items(X->h_mpad, X->h_mpad, 128, it_tc);
    X->n_items_tc = (int)it_tc.size();
    std::vector<int2> rg[3];
    for (int k = 0; k < 3; ++k) rg[k].assign(X->P, make_int2(0, 0));
    X->n_items_64 = (int)item_ranges(m64, X->h_mpad, 64, false, &rg[2]);
    X->n_items_tc_full = (int)item_ranges(X->h_mpad, X->h_mpad, 128, true, nullptr);
    X->n_items_64_full = (int)item_ranges(m64, X->h_mpad, 64, true, nullptr);
    item_ranges(X->h_mpad, X->h_mpad, 128, false, &rg[1]);
    X->gather_split = gather_split_of(ctx, X, gather_layout(ctx, X));
    X->max_units = (int)std::max<int64_t>(X->P * X->gather_split, std::max(X->n_items_tc_full, X->n_items_64_full));
    for (int64_t q = 0; q < X->P; ++q) rg[0][q] = make_int2((int)q * X->gather_split, X->gather_split);
    X->P_global = parts->h_global_id.empty() ? X->P : parts->P_global;
    int r = GBE_OK;
#define ALLOC(ptr, bytes) \
    do { if (r == GBE_OK) r = gbe_alloc((void**)&(ptr), (bytes)); } while (0)
    ALLOC(X->d_off, X->P * 8);
    ALLOC(X->d_mpad, X->P * 4);
    ALLOC(X->d_m, X->P * 4);
    ALLOC(X->d_c, X->P * 4);
    ALLOC(X->d_items_tc, std::max<int64_t>(1, X->n_items_tc) * sizeof(TileItem));
    ALLOC(X->d_partials, 2 * (int64_t)X->max_units * 8);
    ALLOC(X->d_ctrl, sizeof(Sp2Ctrl));
    for (int k = 0; k < 3; ++k) ALLOC(X->d_ranges[k], X->P * sizeof(int2));
    ALLOC(X->d_sums, (2 * X->P_global + 1) * 8);
    // FP64 iterates exist from the start only in FP64 states; mixed states allocate them when
    // a run first needs FP64 steps (ensure_f64)
    for (int i = 0; i < 2; ++i) {
        if (prec == GBE_PREC_FP64) {
            ALLOC(X->f64[i], total * 8);
        } else {
            ALLOC(X->planes[i], (int64_t)gbe_subs_planes(prec) * total * 2);
        }
    }
    if (r == GBE_OK && prec != GBE_PREC_FP64 && !(X->planes[0] && X->planes[1])) r = GBE_ENOMEM;
#undef ALLOC
    if (r != GBE_OK) { gbe_free_subs(X); return r; }
    if (cudaMallocHost((void**)&X->h_ctrl, sizeof(Sp2Ctrl)) != cudaSuccess) {
        gbe_free_subs(X);
        gbe_set_error("cudaMallocHost(ctrl) failed");
        return GBE_ENOMEM;
    }
    for (int i = 0; i < 3; ++i) cudaEventCreate(&X->ev[i]);
    cudaStream_t st = ctx->stream;
    cudaMemcpyAsync(X->d_off, X->h_off.data(), X->P * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(X->d_mpad, X->h_mpad.data(), X->P * 4, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(X->d_m, X->h_m.data(), X->P * 4, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(X->d_c, X->h_c.data(), X->P * 4, cudaMemcpyHostToDevice, st);
    if (X->n_items_tc) cudaMemcpyAsync(X->d_items_tc, it_tc.data(), it_tc.size() * sizeof(TileItem), cudaMemcpyHostToDevice, st);
    for (int k = 0; k < 3; ++k) cudaMemcpyAsync(X->d_ranges[k], rg[k].data(), X->P * sizeof(int2), cudaMemcpyHostToDevice, st);
    // Side 1 starts at zero: a squaring leaves the columns of a subgraph's last block past the
    // next multiple of 16 above m unwritten, and they must read as zero.  Side 0 needs no
    // clear: every SP2 run starts with the gather, which writes every stored (upper) block of
    // side 0, padding included (the FP64 iterate in full); lower blocks are never read.  A
    // Chebyshev expansion clears its sides itself.
    if (X->f64[1]) cudaMemsetAsync(X->f64[1], 0, total * 8, st);
    if (X->planes[1]) cudaMemsetAsync(X->planes[1], 0, (size_t)gbe_subs_planes(prec) * total * 2, st);
    GBE_CUDA_TRY(cudaStreamSynchronize(st));
    if (prec != GBE_PREC_FP64) {
        r = gbe_tc_make_tmaps(X);
        if (r != GBE_OK) { gbe_free_subs(X); return r; }
        // a configuration the autotuner chose for a state of this shape
        const std::vector<int64_t> key = gbe_subs_shape_key(ctx, X);
        for (const auto& kv : ctx->tune_cache)
            if (kv.first == key) {
                r = gbe_subs_apply_config(ctx, X, kv.second);
                if (r != GBE_OK) { gbe_free_subs(X); return r; }
                break;
            }
    }
    *out = X;
    return GBE_OK;
}

std::vector<int64_t> gbe_subs_shape_key(const gbe_ctx* ctx, const gbe_subs* X) {
    // precision, SM count, number of subgraphs, then (padded size, count) per size bucket
    std::vector<int64_t> key = {X->prec, ctx->sm_count, X->P};
    std::vector<int32_t> mp(X->h_mpad);
    std::sort(mp.begin(), mp.end());
    for (size_t i = 0; i < mp.size();) {
        size_t j = i;
        while (j < mp.size() && mp[j] == mp[i]) ++j;
        key.push_back(mp[i]);
        key.push_back((int64_t)(j - i));
        i = j;
    }
    return key;
}

int gbe_subs_apply_config(gbe_ctx* ctx, gbe_subs* X, const gbe_tc_config& cfg) {
    GBE_CHECK_ARG(cfg.schedule == GBE_SCHED_ROUND_ROBIN || cfg.schedule == GBE_SCHED_BALANCED_RANGES, "schedule");
    GBE_CHECK_ARG(cfg.kchunk == 0 || cfg.kchunk == 16 || cfg.kchunk == 32, "kchunk must be 0, 16 or 32");
    GBE_CHECK_ARG(X->prec != GBE_PREC_FP64TC || cfg.kchunk != 32, "the FP64TC squaring runs 16-column K-chunks only");
    if (X->prec != GBE_PREC_FP64 && cfg.stages != 0) {
        int opt[8];
        const int n = gbe_tc_stage_options(X->prec, cfg.kchunk, opt, 8);
        bool found = false;
        for (int i = 0; i < n; ++i) found = found || opt[i] == cfg.stages;
        GBE_CHECK_ARG(found, "the squaring kernel of this precision is not built with that many stages");
    }
    drop_graphs(X);
    gbe_free(X->d_cta_ptr);
    X->d_cta_ptr = nullptr;
    X->cta_grid = 0;
    if (cfg.schedule == GBE_SCHED_BALANCED_RANGES && X->n_items_tc > 0) {
        // the items in launch order (as built by gbe_subs_create), cost = K-chunks of the tile
        std::vector<TileItem> items;
        make_items(X->h_mpad, X->h_mpad, 128, items);
        const int n = (int)items.size();
        const int grid = std::max(1, std::min(n, ctx->sm_count));
        std::vector<double> cost(n);
        double total = 0.0;
        for (int i = 0; i < n; ++i) {
            cost[i] = (double)((X->h_m[items[i].s] + 15) / 16);
            total += cost[i];
        }
        // contiguous runs of nearly equal cost, at least one item each
        std::vector<int32_t> ptr(grid + 1, 0);
        double acc = 0.0;
        int j = 0;
        for (int b = 0; b < grid - 1; ++b) {
            const double target = total * (double)(b + 1) / grid;
            const int lo = ptr[b] + 1, hi = n - (grid - 1 - b);
            while (j < lo) acc += cost[j++];
            while (j < hi && acc + 0.5 * cost[j] < target) acc += cost[j++];
            ptr[b + 1] = j;
        }
        ptr[grid] = n;
        GBE_TRY(gbe_alloc((void**)&X->d_cta_ptr, (grid + 1) * sizeof(int32_t)));
        GBE_CUDA_TRY(cudaMemcpyAsync(X->d_cta_ptr, ptr.data(), (grid + 1) * sizeof(int32_t), cudaMemcpyHostToDevice,
                                     ctx->stream));
        GBE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        X->cta_grid = grid;
    }
    X->tc_cfg = cfg;
    return GBE_OK;
}

extern "C" int gbe_subs_get_config(const gbe_subs* X, gbe_tc_config* cfg) {
    GBE_CHECK_ARG(X && cfg, "NULL argument");
    *cfg = X->tc_cfg;
    return GBE_OK;
}

extern "C" int gbe_subs_set_config(gbe_ctx* ctx, gbe_subs* X, const gbe_tc_config* cfg) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && X && cfg, "NULL argument");
    GBE_CUDA_TRY(cudaSetDevice(ctx->device));
    return gbe_subs_apply_config(ctx, X, *cfg);
}

int gbe_launch_gershgorin(gbe_ctx* ctx, const gbe_csr* H, gbe_subs* X) {
    const int blocks = std::max(1, std::min<int>((int)((H->n + 7) / 8), ctx->sm_count * 8));
    gershgorin_kernel<<<blocks, 256, 0, ctx->stream>>>(H->rowptr, H->col, H->val, H->n, X->d_ctrl);
    GBE_CUDA_TRY(cudaGetLastError());
    return GBE_OK;
}

typedef void (*GatherFn)(Sp2Ctrl*, const int64_t*, const int32_t*, const double*, const int64_t*, const int32_t*,
                         SubsGeom, int, uint16_t*, int64_t, double*, double*, int, int, int, uint2*, int);
static GatherFn gather_for(int prec) {
    switch (prec) {
        case GBE_PREC_FP64: return gather_kernel<GBE_PREC_FP64>;
        case GBE_PREC_FP16X6: return gather_kernel<GBE_PREC_FP16X6>;
        case GBE_PREC_FP64TC: return gather_kernel<GBE_PREC_FP64TC>;
        default: return gather_kernel<GBE_PREC_BF16X3>;
    }
}

// Checks that the gather fits and allocates its global row staging when it needs one (called
// before any launch or capture of a run).
static int prepare_gather(const gbe_ctx* ctx, gbe_subs* X) {
    const GatherLayout L = gather_layout(ctx, X);
    if ((int64_t)L.smem > (int64_t)ctx->smem_optin) {
        gbe_set_error("a subgraph of %lld vertices needs %zu bytes of gather shared memory, the device allows %d",
                      (long long)X->parts->max_m, L.smem, ctx->smem_optin);
        return GBE_ECAPACITY;
    }
    if (L.rows_global && !X->d_gather_rows)
        GBE_TRY(gbe_alloc(&X->d_gather_rows, (size_t)X->P * 8 * X->max_mpad * sizeof(uint2)));
    return GBE_OK;
}

static uint2* gather_rows_arg(const GatherLayout& L, const gbe_subs* X) {
    return L.rows_global ? static_cast<uint2*>(X->d_gather_rows) : nullptr;
}

// Decision after the gather (kind 0) or a squaring (1 tensor-core, 2 FP64).  With a trace
// exchange (sharded global-trace run) this rank's per-subgraph sums are written at their
// global positions, summed over the ranks by the caller's exchange, and decided from.
static DecideIn decide_in(const gbe_subs* X, int kind) {
    DecideIn in;
    in.partials = X->d_partials;
    in.max_units = X->max_units;
    in.ranges = X->d_ranges[kind];
    in.P = (int)X->P;
    in.sums = nullptr;
    in.P_global = X->P_global;
    in.kind = kind;
    return in;
}

static int enqueue_decide(gbe_ctx* ctx, gbe_subs* X, int kind, const gbe_sp2_params* xp, cudaGraphConditionalHandle cond,
                          bool set_cond) {
    cudaStream_t st = ctx->stream;
    DecideIn in = decide_in(X, kind);
    if (xp && xp->exchange) {
        const int blocks = (int)std::min<int64_t>(ctx->sm_count, (X->P_global + 255) / 256);
        sub_sums_kernel<<<std::max(1, blocks), 256, 0, st>>>(X->d_ctrl, X->d_partials, X->max_units, X->d_ranges[kind],
                                                              X->parts->d_local_of, X->P_global, X->d_sums);
        GBE_CUDA_TRY(cudaGetLastError());
        const int rc = xp->exchange(xp->exchange_user, X->d_sums, 2 * X->P_global + 1, (void*)st);
        if (rc != 0) {
            gbe_set_error("trace exchange returned %d", rc);
            return GBE_EPEER;
        }
        in.sums = X->d_sums;
    }
    decide_kernel<<<1, kDecideThreads, 0, st>>>(X->d_ctrl, in, cond, set_cond ? 1 : 0);
    GBE_CUDA_TRY(cudaGetLastError());
    return GBE_OK;
}

// Control init, spectral bounds, gather and the first decision of a run (on ctx->stream).
static int enqueue_prologue(gbe_ctx* ctx, const gbe_csr* H, const Sp2Init& in, gbe_subs* X,
                            const gbe_sp2_params* xp = nullptr) {
    cudaStream_t st = ctx->stream;
    init_ctrl_kernel<<<1, 256, 0, st>>>(X->d_ctrl, in);
    GBE_CUDA_TRY(cudaGetLastError());
    if (!in.eps_given) GBE_TRY(gbe_launch_gershgorin(ctx, H, X));
    const gbe_parts* parts = X->parts;
    const GatherLayout L = gather_layout(ctx, X);
    auto gk = gather_for(X->prec);
    gk<<<(unsigned)(X->P * X->gather_split), 256, L.smem, st>>>(
        X->d_ctrl, H->rowptr, H->col, H->val, parts->d_sub_ptr, parts->d_sub_idx, geom_of(X), X->max_mpad, X->planes[0],
        X->total_elems, X->f64[0], X->d_partials, X->max_units, L.htab_off, L.hbits, gather_rows_arg(L, X),
        X->gather_split);
    GBE_CUDA_TRY(cudaGetLastError());
    return enqueue_decide(ctx, X, 0, xp, 0, false);
}

// One SP2 step: the tensor-core squaring and/or the FP64 squaring, each followed by its
// decision (kernels whose turn it is not exit at once).  slot >= 0 records profiling
// events; in a graph body slot = -1 and the last decision sets the loop condition.
static int enqueue_step(gbe_ctx* ctx, gbe_subs* X, bool fp64_steps, int slot, cudaGraphConditionalHandle cond,
                        bool set_cond, const gbe_sp2_params* xp = nullptr) {
    cudaStream_t st = ctx->stream;
    const bool prof = slot >= 0 && ctx->profile != 0;
    const bool has_tc = X->prec != GBE_PREC_FP64;
    if (has_tc) {
        if (prof) cudaEventRecord(X->ev_tc[2 * slot], st);
        GBE_TRY(gbe_tc_launch_square(ctx, X, slot));
        if (prof) cudaEventRecord(X->ev_tc[2 * slot + 1], st);
        GBE_TRY(enqueue_decide(ctx, X, 1, xp, cond, set_cond && !fp64_steps));
    }
    if (fp64_steps) {
        const int grid64 = std::max(1, std::min(X->n_items_64, ctx->sm_count * 4));
        if (prof) cudaEventRecord(X->ev_64[2 * slot], st);
        square_fp64_kernel<<<grid64, 256, 0, st>>>(X->d_ctrl, geom_of(X), X->d_items_64, X->n_items_64, X->planes[0],
                                                   X->planes[1], X->total_elems, X->f64[0], X->f64[1], X->d_partials,
                                                   X->max_units, slot);
        if (prof) cudaEventRecord(X->ev_64[2 * slot + 1], st);
        GBE_CUDA_TRY(cudaGetLastError());
        GBE_TRY(enqueue_decide(ctx, X, 2, xp, cond, set_cond));
    }
    return GBE_OK;
}

static void drop_graphs(gbe_subs* X) {
    for (int i = 0; i < 2; ++i)
        if (X->gexec[i]) { cudaGraphExecDestroy(X->gexec[i]); X->gexec[i] = nullptr; }
    X->gkey.clear();
}

// Capture the two graphs of a run on the state's own capture stream (capture is not
// possible on the legacy default stream) and instantiate them.
static int build_graphs(gbe_ctx* ctx, const gbe_csr* H, const Sp2Init& in, gbe_subs* X, bool fp64_steps) {
    drop_graphs(X);
    if (!X->cap_stream) GBE_CUDA_TRY(cudaStreamCreateWithFlags(&X->cap_stream, cudaStreamNonBlocking));
    const cudaStream_t saved = ctx->stream;
    ctx->stream = X->cap_stream;
    int r = GBE_OK;
    cudaGraph_t g0 = nullptr, g1 = nullptr, tmp = nullptr;
    // graph 0: prologue
    cudaError_t e = cudaStreamBeginCapture(X->cap_stream, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        r = enqueue_prologue(ctx, H, in, X);
        e = cudaStreamEndCapture(X->cap_stream, &g0);
    }
    // graph 1: while (the last decision says continue) { one SP2 step }
    cudaGraphConditionalHandle cond = 0;
    if (e == cudaSuccess && r == GBE_OK) e = cudaGraphCreate(&g1, 0);
    if (e == cudaSuccess && r == GBE_OK) e = cudaGraphConditionalHandleCreate(&cond, g1, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np = {};
    if (e == cudaSuccess && r == GBE_OK) {
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = cond;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        e = cudaGraphAddNode(&node, g1, nullptr, nullptr, 0, &np);
    }
    if (e == cudaSuccess && r == GBE_OK) {
        e = cudaStreamBeginCaptureToGraph(X->cap_stream, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            r = enqueue_step(ctx, X, fp64_steps, -1, cond, true);
            e = cudaStreamEndCapture(X->cap_stream, &tmp);
        }
    }
    if (e == cudaSuccess && r == GBE_OK) e = cudaGraphInstantiate(&X->gexec[0], g0, 0);
    if (e == cudaSuccess && r == GBE_OK) e = cudaGraphInstantiate(&X->gexec[1], g1, 0);
    ctx->stream = saved;
    if (g0) cudaGraphDestroy(g0);
    if (g1) cudaGraphDestroy(g1);
    if (r == GBE_OK && e != cudaSuccess) {
        gbe_set_error("SP2 graph capture: %s", cudaGetErrorString(e));
        (void)cudaGetLastError();
        r = GBE_ECUDA;
    }
    if (r != GBE_OK) drop_graphs(X);
    return r;
}

extern "C" int gbe_sp2_run(gbe_ctx* ctx, const gbe_csr* H, const gbe_parts* parts, const gbe_sp2_params* prm,
                           gbe_subs* X) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && H && parts && prm && X, "NULL argument");
    GBE_CHECK_ARG(H->on_device, "gbe_sp2_run needs a device CSR (use gbe_sp2_submatrices for host H)");
    GBE_TRY(gbe_check_device_csr(ctx, H, "gbe_sp2_run H"));
    GBE_CHECK_ARG(X->parts == parts, "state was created for another partition");
    GBE_CHECK_ARG(H->n == parts->n, "H and partition sizes differ");
    GBE_CHECK_ARG(prm->prec == X->prec, "params.prec differs from the state's precision");
    GBE_CHECK_ARG(prm->n_max > 0 && prm->n_max <= GBE_SEQ_MAX, "n_max out of range");
    GBE_CHECK_ARG(prm->branch_mode == GBE_BRANCH_GLOBAL_TRACE || prm->branch_mode == GBE_BRANCH_REPLAY, "branch_mode");
    GBE_CHECK_ARG(prm->branch_mode != GBE_BRANCH_REPLAY || (prm->seq_in && prm->seq_len >= 0 && prm->seq_len <= GBE_SEQ_MAX),
                  "replay needs seq_in / seq_len <= GBE_SEQ_MAX");
    // a replayed sequence is applied whole: a longer one than n_max would be cut silently
    // (and its FP64 tail, placed at its end, never reached)
    GBE_CHECK_ARG(prm->branch_mode != GBE_BRANCH_REPLAY || prm->seq_len <= prm->n_max,
                  "replay sequence longer than n_max");
    if (parts->max_m > 8192) {
        gbe_set_error("a subgraph of %lld vertices exceeds the 8192 the gather holds", (long long)parts->max_m);
        return GBE_ECAPACITY;
    }
    GBE_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    Sp2Init in;
    memset(&in, 0, sizeof(in));
    in.mode = (prm->prec == GBE_PREC_FP64) ? 1 : 0;
    in.fmt = (prm->prec == GBE_PREC_FP64) ? 1 : 0;
    in.n_min = prm->n_min;
    in.n_max = prm->n_max;
    in.branch_mode = prm->branch_mode;
    in.seq_len = prm->branch_mode == GBE_BRANCH_REPLAY ? prm->seq_len : 0;
    in.fp64_tail = prm->prec == GBE_PREC_FP64TC ? 0 : prm->fp64_tail;   // FP64TC is FP64-grade throughout
    in.prec = prm->prec;
    in.eps_given = prm->eps_given;
    in.eps_min = prm->eps_min;
    in.eps_max = prm->eps_max;
    in.n_occ = prm->n_occ;
    in.idem_tol = prm->idem_tol;
    in.tail_switch = prm->tail_switch;
    const double tmo = prm->timeout_ms > 0 ? prm->timeout_ms : 2000.0;
    in.timeout_cycles = (long long)(tmo * 2.2e6);
    in.out_scale = 1.0;
    if (in.branch_mode == GBE_BRANCH_REPLAY && in.seq_len) memcpy(in.seq_in, prm->seq_in, in.seq_len);
    if (in.prec != GBE_PREC_FP64 && in.branch_mode == GBE_BRANCH_REPLAY && in.seq_len <= in.fp64_tail) in.mode = 1;
    const bool fp64_steps = X->prec == GBE_PREC_FP64 || in.fp64_tail > 0;
    GBE_TRY(prepare_gather(ctx, X));
    if (fp64_steps) {
        GBE_TRY(ensure_f64(X, st));
        GBE_TRY(ensure_items(ctx, X, false));
    }
    // kernel attributes are set outside any capture
    {
        const GatherLayout L = gather_layout(ctx, X);
        auto gk = gather_for(X->prec);
        GBE_CUDA_TRY(cudaFuncSetAttribute(gk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem));
    }
    const bool prof = ctx->profile != 0;
    // a sharded global-trace run exchanges traces through the caller after every decision
    const gbe_sp2_params* xp = (prm->exchange && in.branch_mode == GBE_BRANCH_GLOBAL_TRACE) ? prm : nullptr;
    GBE_CHECK_ARG(!prm->exchange || !X->parts->h_global_id.empty() || X->P_global == X->P,
                  "exchange given for a partition that is not a shard");
    if (ctx->graphs && !prof && !xp) {
        // graph launch: the loop runs exactly as many steps as the device decides
        std::vector<unsigned char> key(sizeof(in) + 5 * sizeof(int64_t) + 1);
        unsigned char* k = key.data();
        memcpy(k, &in, sizeof(in));
        const int64_t ptrs[5] = {(int64_t)(uintptr_t)H->rowptr, (int64_t)(uintptr_t)H->col, (int64_t)(uintptr_t)H->val,
                                 H->n, H->nnz};
        memcpy(k + sizeof(in), ptrs, sizeof(ptrs));
        k[sizeof(in) + sizeof(ptrs)] = fp64_steps ? 1 : 0;
        // The graphs are captured on the second run with the same inputs and parameters, and
        // relaunched while they stay the same: a run made once (such as a new state per MD
        // step) is launched step by step instead of paying for a capture.
        const bool have = X->gexec[0] && key == X->gkey;
        if (have || (!X->gexec[0] && key == X->gkey)) {
            if (!have) {
                GBE_TRY(build_graphs(ctx, H, in, X, fp64_steps));
                X->gkey = key;
            }
            cudaEventRecord(X->ev[0], st);
            GBE_CUDA_TRY(cudaGraphLaunch(X->gexec[0], st));
            cudaEventRecord(X->ev[1], st);
            GBE_CUDA_TRY(cudaGraphLaunch(X->gexec[1], st));
            cudaEventRecord(X->ev[2], st);
            X->last_slots = 0;
            X->last_prof = false;
            return GBE_OK;
        }
        drop_graphs(X);
        X->gkey = key;
    }
    cudaEventRecord(X->ev[0], st);
    GBE_TRY(enqueue_prologue(ctx, H, in, X, xp));
    cudaEventRecord(X->ev[1], st);
    if (prof && (int)X->ev_tc.size() < 2 * prm->n_max) {
        for (int i = (int)X->ev_tc.size(); i < 2 * prm->n_max; ++i) {
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            X->ev_tc.push_back(a);
            X->ev_64.push_back(b);
        }
    }
    // a replayed sequence takes exactly seq_len steps; otherwise n_max slots (the slots after
    // the device's stop decision exit at once)
    const int slots = in.branch_mode == GBE_BRANCH_REPLAY ? std::min(prm->n_max, in.seq_len) : prm->n_max;
    X->last_slots = slots;
    for (int slot = 0; slot < slots; ++slot) {
        GBE_TRY(enqueue_step(ctx, X, fp64_steps, slot, 0, false, xp));
        if (xp) {
            // every rank takes the same decisions, so all stop after the same step and make
            // the same number of exchanges
            GBE_CUDA_TRY(cudaMemcpyAsync(&X->h_ctrl->stop, &X->d_ctrl->stop, sizeof(int), cudaMemcpyDeviceToHost, st));
            GBE_CUDA_TRY(cudaStreamSynchronize(st));
            if (X->h_ctrl->stop != 0) {
                X->last_slots = slot + 1;
                break;
            }
        }
    }
    X->last_prof = prof;
    GBE_CUDA_TRY(cudaGetLastError());
    cudaEventRecord(X->ev[2], st);
    return GBE_OK;
}

extern "C" int gbe_sp2_report_get(gbe_ctx* ctx, const gbe_subs* X, gbe_sp2_report* rep) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && X && rep, "NULL argument");
    GBE_CUDA_TRY(cudaMemcpyAsync(X->h_ctrl, X->d_ctrl, sizeof(Sp2Ctrl), cudaMemcpyDeviceToHost, ctx->stream));
    GBE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    const Sp2Ctrl* C = X->h_ctrl;
    memset(rep, 0, sizeof(*rep));
    rep->iters = C->iter;
    rep->fp64_iters = C->fp64_iters;
    rep->stop_reason = C->stop;
    rep->converged = (C->stop == GBE_STOP_TOL || C->stop == GBE_STOP_STALL || C->stop == GBE_STOP_REPLAY);
    rep->status = C->status;
    rep->eps_min = C->eps_min;
    rep->eps_max = C->eps_max;
    rep->trace = C->t1[C->iter];
    rep->idem_err = fabs(C->t1[C->iter] - C->t2[C->iter]);
    memcpy(rep->seq, C->seq, GBE_SEQ_MAX);
    memcpy(rep->t1, C->t1, sizeof(rep->t1));
    memcpy(rep->t2, C->t2, sizeof(rep->t2));
    cudaEventElapsedTime(&rep->ms_gather, X->ev[0], X->ev[1]);
    cudaEventElapsedTime(&rep->ms_sp2, X->ev[1], X->ev[2]);
    const int mixed_iters = C->iter - C->fp64_iters;
    rep->mma_flops = X->mma_flops_per_iter * mixed_iters;
    rep->alg_flops = X->alg_flops_per_iter * C->iter;
    rep->fp64_flops = X->fp64_flops_per_iter * C->fp64_iters;
    if (X->last_prof) {
        for (int slot = 0; slot < X->last_slots; ++slot) {
            float ms = 0.f;
            if ((C->slot_ran[slot] & 1) && cudaEventElapsedTime(&ms, X->ev_tc[2 * slot], X->ev_tc[2 * slot + 1]) == cudaSuccess) {
                rep->ms_tc += ms;
                rep->n_tc += 1;
            }
            if ((C->slot_ran[slot] & 2) && cudaEventElapsedTime(&ms, X->ev_64[2 * slot], X->ev_64[2 * slot + 1]) == cudaSuccess) {
                rep->ms_fp64 += ms;
                rep->n_fp64 += 1;
            }
        }
    }
    return GBE_OK;
}

// Host CSR -> temporary device copy.
struct DevCsr {
    gbe_csr view{};
    void* buf = nullptr;
    ~DevCsr() { if (buf) gbe_free(buf); }
};

static int csr_to_device(gbe_ctx* ctx, const gbe_csr* H, DevCsr& d) {
    if (H->on_device) { d.view = *H; return GBE_OK; }
    const size_t b0 = (H->n + 1) * 8, b1 = ((H->nnz * 4 + 15) / 16) * 16, b2 = H->nnz * 8;
    GBE_TRY(gbe_alloc(&d.buf, b0 + b1 + b2));
    char* p = (char*)d.buf;
    GBE_CUDA_TRY(cudaMemcpyAsync(p, H->rowptr, b0, cudaMemcpyHostToDevice, ctx->stream));
    GBE_CUDA_TRY(cudaMemcpyAsync(p + b0, H->col, H->nnz * 4, cudaMemcpyHostToDevice, ctx->stream));
    GBE_CUDA_TRY(cudaMemcpyAsync(p + b0 + b1, H->val, b2, cudaMemcpyHostToDevice, ctx->stream));
    d.view = *H;
    d.view.rowptr = (const int64_t*)p;
    d.view.col = (const int32_t*)(p + b0);
    d.view.val = (const double*)(p + b0 + b1);
    d.view.on_device = 1;
    return GBE_OK;
}

extern "C" int gbe_sp2_submatrices(gbe_ctx* ctx, const gbe_csr* H, const gbe_parts* parts,
                                   const gbe_sp2_params* prm, gbe_subs** X, gbe_sp2_report* rep) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && H && parts && prm && X, "NULL argument");
    bool created = false;
    if (*X == nullptr) {
        GBE_TRY(gbe_subs_create(ctx, parts, prm->prec, X));
        created = true;
    }
    DevCsr d;
    int r = csr_to_device(ctx, H, d);
    if (r == GBE_OK) r = gbe_sp2_run(ctx, &d.view, parts, prm, *X);
    gbe_sp2_report tmp;
    gbe_sp2_report* R = rep ? rep : &tmp;
    if (r == GBE_OK) r = gbe_sp2_report_get(ctx, *X, R);
    if (r != GBE_OK) {
        if (created) { gbe_free_subs(*X); *X = nullptr; }
        return r;
    }
    if (R->status != GBE_OK) {
        gbe_set_error("device recorded status %d (%s)", R->status, gbe_strerror(R->status));
        return R->status;
    }
    if (R->stop_reason == GBE_STOP_NMAX) {
        gbe_set_error("SP2 stopped at n_max=%d with idempotency error %.3e", prm->n_max, R->idem_err);
        return GBE_ENOCONV;
    }
    return GBE_OK;
}

// Core columns of every subgraph of X into a device ELL (col, val of width `width`); rows
// outside X's cores are emptied first when `clear` is set.  Enqueue only.
static int assemble_device(gbe_ctx* ctx, const gbe_subs* X, const gbe_parts* parts, double drop_tol, int64_t width,
                           int32_t* col, double* val, bool clear) {
    cudaStream_t st = ctx->stream;
    const int64_t total = parts->n * width;
    // rows outside every core keep the empty entry (the assembly pads the rows it writes)
    if (clear && !parts->cores_cover) fill_ell_kernel<<<ctx->sm_count * 4, 256, 0, st>>>(total, col, val);
    int max_c = 1;
    for (int64_t q = 0; q < X->P; ++q) max_c = std::max(max_c, X->h_c[q]);
    const int jblocks = (max_c + 7) / 8;
    assemble_kernel<<<(unsigned)(X->P * jblocks), 256, 0, st>>>(X->d_ctrl, parts->d_sub_ptr, parts->d_sub_idx, geom_of(X),
                                                                 X->planes[0], X->planes[1], X->total_elems, X->f64[0],
                                                                 X->f64[1], width, col, val, drop_tol, jblocks);
    GBE_CUDA_TRY(cudaGetLastError());
    return GBE_OK;
}

// Device ELL buffers for D: D's own when on the device, else a staging pair (tmp).
static int ell_device_buffers(const gbe_ctx* ctx, const gbe_ell* D, void** tmp, int32_t** col, double** val) {
    const int64_t total = D->n * D->width;
    GBE_TRY(gbe_check_device_ell(ctx, D, "D"));
    *tmp = nullptr;
    *col = D->col;
    *val = D->val;
    if (!D->on_device) {
        const int64_t col_bytes = ((total * 4 + 15) / 16) * 16;
        GBE_TRY(gbe_alloc(tmp, col_bytes + total * 8));
        *col = (int32_t*)*tmp;
        *val = (double*)((char*)*tmp + col_bytes);
    }
    return GBE_OK;
}

// A host D from its device staging pair (the copy engines move it over the host link faster
// than the kernels' own stores to page-locked host memory), then the stream is synchronised.
static int ell_finish(gbe_ctx* ctx, const gbe_ell* D, const int32_t* col, const double* val) {
    cudaStream_t st = ctx->stream;
    const int64_t total = D->n * D->width;
    cudaError_t e = cudaSuccess;
    if (!D->on_device) {
        e = cudaMemcpyAsync(D->col, col, total * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(D->val, val, total * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) {
        gbe_set_error("assemble: %s", cudaGetErrorString(e));
        return GBE_ECUDA;
    }
    return GBE_OK;
}

extern "C" int gbe_assemble_D(gbe_ctx* ctx, const gbe_subs* X, const gbe_parts* parts, double drop_tol, gbe_ell* D) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && X && parts && D, "NULL argument");
    GBE_CHECK_ARG(X->parts == parts, "state was created for another partition");
    if (D->col == nullptr) {
        D->n = parts->n;
        D->width = parts->max_m;
        return GBE_OK;
    }
    GBE_CHECK_ARG(D->val != nullptr && D->n == parts->n, "D buffers / n");
    if (D->width < parts->max_m) {
        gbe_set_error("ELL width %lld < max subgraph size %lld", (long long)D->width, (long long)parts->max_m);
        return GBE_ECAPACITY;
    }
    GBE_CUDA_TRY(cudaSetDevice(ctx->device));
    void* tmp = nullptr;
    int32_t* col;
    double* val;
    GBE_TRY(ell_device_buffers(ctx, D, &tmp, &col, &val));
    int r = assemble_device(ctx, X, parts, drop_tol, D->width, col, val, true);
    if (r == GBE_OK) r = ell_finish(ctx, D, col, val);
    if (tmp) gbe_free(tmp);
    return r;
}

// Bytes of the two ping-pong iterates of a subgraph with padded size mpad.
static int64_t iterate_bytes(int prec, int64_t mpad, bool fp64_also) {
    const int64_t e = mpad * mpad;
    int64_t b = prec == GBE_PREC_FP64 ? 2 * 8 * e : 2 * (int64_t)gbe_subs_planes(prec) * 2 * e;
    if (fp64_also && prec != GBE_PREC_FP64) b += 2 * 8 * e;
    return b;
}

extern "C" int gbe_sp2_replay_batched(gbe_ctx* ctx, const gbe_csr* H, const gbe_parts* parts,
                                      const gbe_sp2_params* prm, int64_t budget_bytes, double drop_tol, gbe_ell* D,
                                      int* batches) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && H && parts && prm && D && D->col && D->val, "NULL argument");
    GBE_CHECK_ARG(prm->branch_mode == GBE_BRANCH_REPLAY && prm->seq_in && prm->seq_len > 0,
                  "a batched run replays a pre-determined sequence");
    GBE_CHECK_ARG(prm->exchange == nullptr, "a batched run exchanges no traces");
    GBE_CHECK_ARG(parts->h_global_id.empty(), "parts is a shard");
    GBE_CHECK_ARG(D->n == parts->n, "D rows");
    if (D->width < parts->max_m) {
        gbe_set_error("ELL width %lld < max subgraph size %lld", (long long)D->width, (long long)parts->max_m);
        return GBE_ECAPACITY;
    }
    const int64_t P = parts->P;
    const int prec = prm->prec;
    const bool tail = prm->fp64_tail > 0;
    std::vector<int64_t> bytes(P);
    int64_t total = 0, largest = 0;
    for (int64_t s = 0; s < P; ++s) {
        const int64_t m = parts->h_sub_ptr[s + 1] - parts->h_sub_ptr[s];
        bytes[s] = iterate_bytes(prec, (m + 127) / 128 * 128, tail);
        total += bytes[s];
        largest = std::max(largest, bytes[s]);
    }
    if (largest > budget_bytes) {
        gbe_set_error("a subgraph's iterates take %lld bytes, above the budget of %lld", (long long)largest,
                      (long long)budget_bytes);
        return GBE_ECAPACITY;
    }
    // the fewest batches, dealt by m_s^3, whose iterates each fit the budget
    std::vector<int32_t> owner(P);
    int B = (int)std::max<int64_t>(1, (total + budget_bytes - 1) / budget_bytes);
    for (;; ++B) {
        GBE_TRY(gbe_shard_assign(P, parts->h_sub_ptr.data(), B, owner.data(), nullptr));
        std::vector<int64_t> per(B, 0);
        for (int64_t s = 0; s < P; ++s) per[owner[s]] += bytes[s];
        if (*std::max_element(per.begin(), per.end()) <= budget_bytes) break;
        if (B >= P) break;   // one subgraph per batch fits (largest <= budget)
    }
    GBE_CUDA_TRY(cudaSetDevice(ctx->device));
    void* tmp = nullptr;
    int32_t* col;
    double* val;
    GBE_TRY(ell_device_buffers(ctx, D, &tmp, &col, &val));
    int r = GBE_OK;
    if (!parts->cores_cover) fill_ell_kernel<<<ctx->sm_count * 4, 256, 0, ctx->stream>>>(D->n * D->width, col, val);
    for (int b = 0; b < B && r == GBE_OK; ++b) {
        gbe_parts* local = nullptr;
        gbe_subs* X = nullptr;
        r = gbe_parts_shard(ctx, parts, owner.data(), b, &local);
        if (r == GBE_OK) r = gbe_subs_create(ctx, local, prec, &X);
        if (r == GBE_OK) r = gbe_sp2_run(ctx, H, local, prm, X);
        // each batch writes the rows of its own cores; no batch clears the others'
        if (r == GBE_OK) r = assemble_device(ctx, X, local, drop_tol, D->width, col, val, false);
        if (r == GBE_OK) {
            const cudaError_t e = cudaStreamSynchronize(ctx->stream);
            if (e != cudaSuccess) { gbe_set_error("batched replay: %s", cudaGetErrorString(e)); r = GBE_ECUDA; }
        }
        // the status the batch's kernels recorded (non-finite H, a wait that ran out)
        gbe_sp2_report R;
        if (r == GBE_OK) r = gbe_sp2_report_get(ctx, X, &R);
        if (r == GBE_OK && R.status != GBE_OK) {
            gbe_set_error("batch %d: device recorded status %d (%s)", b, R.status, gbe_strerror(R.status));
            r = R.status;
        }
        if (X) gbe_free_subs(X);
        if (local) gbe_free_parts(local);
    }
    if (r == GBE_OK) r = ell_finish(ctx, D, col, val);
    if (tmp) gbe_free(tmp);
    if (r == GBE_OK && batches) *batches = B;
    return r;
}

extern "C" int gbe_subs_export(gbe_ctx* ctx, const gbe_subs* X, int64_t s, double* out) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && X && out && s >= 0 && s < X->P, "bad argument");
    const int64_t m = X->h_m[s];
    void* tmp = nullptr;
    GBE_TRY(gbe_alloc(&tmp, m * m * 8));
    export_kernel<<<ctx->sm_count, 256, 0, ctx->stream>>>(X->d_ctrl, geom_of(X), (int)s, X->planes[0], X->planes[1],
                                                          X->total_elems, X->f64[0], X->f64[1], (double*)tmp);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, m * m * 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    gbe_free(tmp);
    if (e != cudaSuccess) {
        gbe_set_error("export: %s", cudaGetErrorString(e));
        return GBE_ECUDA;
    }
    return GBE_OK;
}

// ============================================================================= Chebyshev expansion
// Finite-temperature D = [exp(beta (H - mu)) + 1]^-1 (Eq. 7) per subgraph: x = (H_s - a I) / b
// on the Gershgorin interval, the Chebyshev series of the Fermi function evaluated by
// Clenshaw's recurrence b_k = c_k I + 2 x b_{k+1} - b_{k+2}, D_s = c_0 I + x b_1 - b_2, and
// the core columns assembled by Eq. 6.  The iterates are carried divided by B, a bound on
// max_k ||b_k|| (the scalar recurrence maximised over [-1, 1]), so that they have spectral
// norm <= 1 as the tensor-core split requires; assembly multiplies by B.

extern "C" int gbe_fermi_coefficients(double beta, double mu, double eps_min, double eps_max, int order, double* c) {
    GBE_CHECK_ARG(c && order >= 1 && eps_max > eps_min && beta > 0.0, "bad argument");
    const double a = 0.5 * (eps_max + eps_min), b = 0.5 * (eps_max - eps_min);
    const int K = 2 * (order + 1);
    const double pi = 3.14159265358979323846;
    std::vector<double> f(K), t(K);
    for (int j = 0; j < K; ++j) {
        t[j] = pi * (j + 0.5) / K;
        const double z = beta * (a + b * std::cos(t[j]) - mu);
        f[j] = 0.5 * (1.0 - std::tanh(0.5 * z));   // Fermi function without overflow
    }
    for (int n = 0; n <= order; ++n) {
        double s = 0.0;
        for (int j = 0; j < K; ++j) s += std::cos(n * t[j]) * f[j];
        c[n] = (n == 0 ? 1.0 : 2.0) * s / K;
    }
    return GBE_OK;
}

// max over k and x in [-1, 1] of |b_k(x)| for the scalar recurrence, on a fine grid
// (Chebyshev-Lobatto points, at least 4 per degree), with a 5% margin.
static double clenshaw_bound(const double* c, int order) {
    const int npts = std::max(4096, 4 * order);
    const double pi = 3.14159265358979323846;
    double mx = 0.0;
    for (int i = 0; i <= npts; ++i) {
        const double x = std::cos(pi * i / npts);
        double b1 = 0.0, b2 = 0.0;
        for (int k = order; k >= 1; --k) {
            const double b0 = c[k] + 2.0 * x * b1 - b2;
            b2 = b1;
            b1 = b0;
            mx = std::max(mx, std::fabs(b0));
        }
        mx = std::max(mx, std::fabs(c[0] + x * b1 - b2));
    }
    return 1.05 * std::max(mx, 1e-300);
}

extern "C" int gbe_foe_run(gbe_ctx* ctx, const gbe_csr* H, const gbe_parts* parts, const gbe_foe_params* prm,
                           gbe_subs* X) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && H && parts && prm && X, "NULL argument");
    GBE_CHECK_ARG(H->on_device, "gbe_foe_run needs a device CSR");
    GBE_TRY(gbe_check_device_csr(ctx, H, "gbe_foe_run H"));
    GBE_CHECK_ARG(X->parts == parts && H->n == parts->n, "state / partition / H mismatch");
    GBE_CHECK_ARG(X->prec == GBE_PREC_FP64 || X->prec == GBE_PREC_FP16X6, "Chebyshev expansion supports FP64 and FP16X6");
    GBE_CHECK_ARG(prm->order >= 1 && prm->order <= 100000, "order out of range");
    GBE_CHECK_ARG(prm->coeffs || prm->beta > 0.0, "beta must be positive (or coefficients given)");
    if (parts->max_m > 8192) {
        gbe_set_error("a subgraph of %lld vertices exceeds the 8192 the gather holds", (long long)parts->max_m);
        return GBE_ECAPACITY;
    }
    GBE_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const bool fp64 = X->prec == GBE_PREC_FP64;
    if (fp64) GBE_TRY(ensure_f64(X, st));
    GBE_TRY(ensure_items(ctx, X, true));
    // the fixed x lives on side 2
    if (fp64 && !X->f64[2]) GBE_TRY(gbe_alloc((void**)&X->f64[2], X->total_elems * 8));
    if (!fp64 && !X->planes[2]) {
        GBE_TRY(gbe_alloc((void**)&X->planes[2], 4 * X->total_elems * 2));
        GBE_TRY(gbe_tc_make_tmaps(X));
    }
    Sp2Init in;
    memset(&in, 0, sizeof(in));
    in.mode = fp64 ? 1 : 0;
    in.fmt = fp64 ? 1 : 0;
    in.prec = X->prec;
    in.n_max = 1;
    in.branch_mode = GBE_BRANCH_REPLAY;
    in.foe = 1;
    const double tmo = prm->timeout_ms > 0 ? prm->timeout_ms : 2000.0;
    in.timeout_cycles = (long long)(tmo * 2.2e6);
    // spectral bounds on the host (the coefficients depend on them)
    double emin = prm->eps_min, emax = prm->eps_max;
    if (!prm->eps_given) {
        in.out_scale = 1.0;
        init_ctrl_kernel<<<1, 256, 0, st>>>(X->d_ctrl, in);
        GBE_TRY(gbe_launch_gershgorin(ctx, H, X));
        GBE_CUDA_TRY(cudaMemcpyAsync(X->h_ctrl, X->d_ctrl, sizeof(Sp2Ctrl), cudaMemcpyDeviceToHost, st));
        GBE_CUDA_TRY(cudaStreamSynchronize(st));
        emin = dkey_inv_host(X->h_ctrl->eps_min_key);
        emax = dkey_inv_host(X->h_ctrl->eps_max_key);
    }
    GBE_CHECK_ARG(std::isfinite(emin) && std::isfinite(emax) && emax > emin, "spectral bounds");
    const int M = prm->order;
    std::vector<double> c(M + 1);
    if (prm->coeffs) std::copy(prm->coeffs, prm->coeffs + M + 1, c.begin());
    else GBE_TRY(gbe_fermi_coefficients(prm->beta, prm->mu, emin, emax, M, c.data()));
    const double B = clenshaw_bound(c.data(), M);
    // sides: b_{k+1} on p, b_{k+2} on q (overwritten by b_k), then swap
    int p = 0, q = 1;
    for (int k = M; k >= 1; --k) std::swap(p, q);
    in.cur = q;   // the final step writes side q
    in.eps_given = 1;
    in.eps_min = emin;
    in.eps_max = emax;
    in.out_scale = B;
    GBE_TRY(prepare_gather(ctx, X));
    const GatherLayout L = gather_layout(ctx, X);
    auto gk = fp64 ? gather_kernel<GBE_PREC_FP64> : gather_kernel<GBE_PREC_FP16X6>;
    GBE_CUDA_TRY(cudaFuncSetAttribute(gk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem));
    cudaEventRecord(X->ev[0], st);
    init_ctrl_kernel<<<1, 256, 0, st>>>(X->d_ctrl, in);
    gk<<<(unsigned)(X->P * X->gather_split), 256, L.smem, st>>>(
        X->d_ctrl, H->rowptr, H->col, H->val, parts->d_sub_ptr, parts->d_sub_idx, geom_of(X), X->max_mpad, X->planes[2],
        X->total_elems, X->f64[2], X->d_partials, X->max_units, L.htab_off, L.hbits, gather_rows_arg(L, X),
        X->gather_split);
    GBE_CUDA_TRY(cudaGetLastError());
    for (int s = 0; s < 2; ++s) {
        if (fp64) GBE_CUDA_TRY(cudaMemsetAsync(X->f64[s], 0, X->total_elems * 8, st));
        else GBE_CUDA_TRY(cudaMemsetAsync(X->planes[s], 0, 4 * X->total_elems * 2, st));
    }
    cudaEventRecord(X->ev[1], st);
    p = 0;
    q = 1;
    const int grid64 = std::max(1, std::min(X->n_items_64_full, ctx->sm_count * 4));
    for (int k = M; k >= 0; --k) {
        const double alpha = k > 0 ? 2.0 : 1.0;   // k = 0: the final combination c_0 I + x b_1 - b_2
        const double gamma = c[k] / B;
        if (fp64)
            cheb_fp64_kernel<<<grid64, 256, 0, st>>>(geom_of(X), X->d_items_64_full, X->n_items_64_full, X->f64[2], X->f64[p],
                                                     X->f64[q], alpha, gamma);
        else
            GBE_TRY(gbe_tc_launch_foe(ctx, X, 2, p, q, (float)alpha, gamma));
        GBE_CUDA_TRY(cudaGetLastError());
        if (k > 0) std::swap(p, q);
    }
    cudaEventRecord(X->ev[2], st);
    X->foe_order = M;
    X->foe_scale = B;
    X->last_slots = 0;
    X->last_prof = false;
    return GBE_OK;
}

extern "C" int gbe_foe_report_get(gbe_ctx* ctx, const gbe_subs* X, gbe_foe_report* rep) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && X && rep, "NULL argument");
    GBE_CUDA_TRY(cudaMemcpyAsync(X->h_ctrl, X->d_ctrl, sizeof(Sp2Ctrl), cudaMemcpyDeviceToHost, ctx->stream));
    GBE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    memset(rep, 0, sizeof(*rep));
    rep->order = X->foe_order;
    rep->scale = X->foe_scale;
    rep->status = X->h_ctrl->status;
    rep->eps_min = X->h_ctrl->eps_min;
    rep->eps_max = X->h_ctrl->eps_max;
    cudaEventElapsedTime(&rep->ms_gather, X->ev[0], X->ev[1]);
    cudaEventElapsedTime(&rep->ms_steps, X->ev[1], X->ev[2]);
    const double steps = X->foe_order + 1;
    rep->mma_flops = (X->prec == GBE_PREC_FP64 ? X->fp64_flops_full : X->mma_flops_full) * steps;
    rep->alg_flops = X->alg_flops_per_iter * steps;
    return GBE_OK;
}
