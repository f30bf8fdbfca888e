// Learned proposal of the data-dependency graph: candidate pairs, local features, a
// width-64 three-layer MLP (fp16-rounded weights, FP32 arithmetic), its training on the
// GPU (forward, binary cross-entropy, backward, Adam) and the GBE_GRAPH_MLP graph mode.
//
// Not in the paper (its graphs come from a prior density matrix, Sec. II.A/II.C); this is
// a way to obtain S_tau when no prior D exists.
//   candidates  i != j with minimum-image distance r_ij < rcand (cell list)
//   features    [-log10(max|H_ij|,1e-12)/12, -log10(max|(H^2)_ij|,1e-12)/12, r_ij/rcand,
//                min(e_i,e_j), max(e_i,e_j)]       (symmetric in i, j)
//   network     h1 = relu(W1 f + b1), h2 = relu(W2 h1 + b2), z = w3.h2 + b3
//   parameters  W1[64x5], b1[64], W2[64x64] (out x in), b2[64], w3[64], b3  (4609 floats)
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_fp16.h>

#include "devutil.cuh"
#include "gbe_internal.h"

using namespace gbe_dev;

namespace {

constexpr int kHid = 64;
constexpr int kNF = 5;
constexpr int kNParams = kHid * kNF + kHid + kHid * kHid + kHid + kHid + 1;   // 4609
constexpr int OW1 = 0, OB1 = OW1 + kHid * kNF, OW2 = OB1 + kHid, OB2 = OW2 + kHid * kHid, OW3 = OB2 + kHid,
              OB3 = OW3 + kHid;
constexpr int kPairCap = 1024;     // candidates per site a warp can hold
constexpr int kBatch = 128;        // pairs per training batch (one per thread)
constexpr int kLd = 68;            // padded row length of the batch activations (floats)

// ------------------------------------------------------------------ candidate pairs + features
constexpr int kPairStage = 512;    // staging slot per site of the single-pass pair search

// Features 0, 2, 3, 4 of the pair (i, j): -log10|H_ij| / 12 (H_ij by binary search in row i),
// r / rcand, min and max of the two onsite energies.  Feature 1, the (H^2)_ij feature, is
// written by h2_feature_kernel.
__device__ __forceinline__ void pair_features(const double* __restrict__ pos, const double* __restrict__ onsite,
                                              const CellGrid& g, int64_t i, double xi, double yi, double zi,
                                              double ei, int j, double rcand, const int64_t* __restrict__ hrp,
                                              const int32_t* __restrict__ hci, const double* __restrict__ hva,
                                              float* f) {
    const double r = sqrt(pair_dist2(pos, xi, yi, zi, j, g));
    double hij = 0.0;
    int64_t a = hrp[i], b = hrp[i + 1] - 1;
    while (a <= b) {
        const int64_t mid = (a + b) >> 1;
        const int v = hci[mid];
        if (v == j) { hij = hva[mid]; break; }
        if (v < j) a = mid + 1; else b = mid - 1;
    }
    const double ej = onsite[j];
    f[0] = -log10f(fmaxf((float)fabs(hij), 1e-12f)) / 12.0f;
    f[2] = (float)(r / rcand);
    f[3] = (float)fmin(ei, ej);
    f[4] = (float)fmax(ei, ej);
}

// One warp per site.  pass 2: count the site's candidates and write them sorted into its
// staging slot of kPairStage entries (pair_stage_kernel then writes the CSR and the
// features); a site with more sets overflow[1], and the host runs pass 1, which writes the
// sorted candidates and their features into the CSR directly.
__global__ void __launch_bounds__(256) pairs_kernel(const double* __restrict__ pos, const float4* __restrict__ pos4,
                                                    const double* __restrict__ onsite, int64_t n, CellGrid g, float lim2,
                                                    float lim2_in, const int64_t* __restrict__ cstart,
                                                    const int32_t* __restrict__ members, double rcand, int pass,
                                                    int32_t* cnt, const int64_t* __restrict__ rowptr, int32_t* pj,
                                                    float* feat, const int64_t* __restrict__ hrp,
                                                    const int32_t* __restrict__ hci, const double* __restrict__ hva,
                                                    int* overflow) {
    __shared__ int buf[8][kPairCap];
    __shared__ int bcount[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * 8 + w;
    if (i >= n) return;
    const double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
    const double rcand2 = rcand * rcand;
    const float4 pi = pos4[i];
    const float bx = (float)g.box[0], by = (float)g.box[1], bz = (float)g.box[2];
    const float ix = (float)g.inv[0], iy = (float)g.inv[1], iz = (float)g.inv[2];
    const int ci = cell_of(pos + 3 * i, g);
    const int cc[3] = {ci / (g.nc[1] * g.nc[2]), (ci / g.nc[2]) % g.nc[1], ci % g.nc[2]};
    if (lane == 0) bcount[w] = 0;
    __syncwarp();
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        if (g.nc[d] >= 3) { lo[d] = -1; hi[d] = 1; }
        else { lo[d] = -cc[d]; hi[d] = g.nc[d] - 1 - cc[d]; }
    }
    // the (at most 27) neighbour cells' member ranges, one per lane, and their exclusive prefix
    // sums: the candidates of all cells are one flat range across the lanes (the row is sorted
    // afterwards, so the order found is free)
    const int ncx = hi[0] - lo[0] + 1, ncy = hi[1] - lo[1] + 1, ncz = hi[2] - lo[2] + 1;
    const int ncell = ncx * ncy * ncz;
    int64_t c0 = 0;
    int clen = 0;
    if (lane < ncell) {
        const int dx = lo[0] + lane / (ncy * ncz), dy = lo[1] + (lane / ncz) % ncy, dz = lo[2] + lane % ncz;
        const int ax = (cc[0] + dx + g.nc[0]) % g.nc[0];
        const int ay = (cc[1] + dy + g.nc[1]) % g.nc[1];
        const int az = (cc[2] + dz + g.nc[2]) % g.nc[2];
        const int cell = (ax * g.nc[1] + ay) * g.nc[2] + az;
        c0 = cstart[cell];
        clen = (int)(cstart[cell + 1] - c0);
    }
    int incl = clen;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const int excl = incl - clen;
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    // (every lane runs every iteration: the shuffles need the whole warp)
    for (int t0 = 0; t0 < total; t0 += 32) {
        const int t = t0 + lane;
        // the candidate's cell: the last one whose range starts at or before t
        int c = 0;
        for (int step = 16; step > 0; step >>= 1) {
            const int e = __shfl_sync(0xffffffffu, excl, (c + step) & 31);
            if (c + step < ncell && e <= t) c += step;
        }
        const int64_t p = __shfl_sync(0xffffffffu, c0, c) + (t - __shfl_sync(0xffffffffu, excl, c));
        if (t < total) {
            const int j = members[p];
            if (j != i) {
                // FP32 separation: inside the inner bound kept, outside the outer one dropped,
                // between them r < rcand in FP64 (up to an ulp at the cutoff)
                const float r2f = dist2_f32(pi, pos4[j], bx, by, bz, ix, iy, iz);
                if (r2f < lim2_in || (r2f < lim2 && pair_dist2(pos, xi, yi, zi, j, g) < rcand2)) {
                    const int k = atomicAdd(&bcount[w], 1);
                    if (k < kPairCap) buf[w][k] = j;
                }
            }
        }
    }
    __syncwarp();
    const int m = bcount[w];
    if (m > kPairCap) {
        if (lane == 0) atomicExch(overflow, 1);
        return;
    }
    if (pass == 2) {
        if (lane == 0) cnt[i] = m;
        if (m > kPairStage) {
            if (lane == 0) atomicExch(overflow + 1, 1);
            return;
        }
    }
    // bitonic sort of the m candidates, padded to a power of two with INT_MAX
    int np2 = 1;
    while (np2 < m) np2 <<= 1;
    for (int t = m + lane; t < np2; t += 32) buf[w][t] = 0x7FFFFFFF;
    __syncwarp();
    for (int k = 2; k <= np2; k <<= 1)
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int t2 = lane; t2 < (np2 >> 1); t2 += 32) {
                const int lo = (t2 / jj) * 2 * jj + (t2 % jj), hi = lo + jj;
                const int x = buf[w][lo], y = buf[w][hi];
                if ((x > y) == ((lo & k) == 0)) { buf[w][lo] = y; buf[w][hi] = x; }
            }
            __syncwarp();
        }
    if (pass == 2) {
        for (int t = lane; t < m; t += 32) pj[i * kPairStage + t] = buf[w][t];   // pj = the staging slots
        return;
    }
    const int64_t base = rowptr[i];
    const double ei = onsite[i];
    for (int t = lane; t < m; t += 32) {
        const int j = buf[w][t];
        pair_features(pos, onsite, g, i, xi, yi, zi, ei, j, rcand, hrp, hci, hva, feat + (base + t) * kNF);
        pj[base + t] = j;
    }
}

// Staged candidates (kPairStage apart) -> CSR and features 0, 2, 3, 4, one warp per site.
__global__ void __launch_bounds__(256) pair_stage_kernel(const double* __restrict__ pos, const double* __restrict__ onsite,
                                                         int64_t n, CellGrid g, double rcand,
                                                         const int32_t* __restrict__ stage,
                                                         const int64_t* __restrict__ rowptr, int32_t* pj, float* feat,
                                                         const int64_t* __restrict__ hrp,
                                                         const int32_t* __restrict__ hci,
                                                         const double* __restrict__ hva) {
    const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
    const double ei = onsite[i];
    const int64_t base = rowptr[i], m = rowptr[i + 1] - base;
    for (int64_t t = lane; t < m; t += 32) {
        const int j = stage[i * kPairStage + t];
        pair_features(pos, onsite, g, i, xi, yi, zi, ei, j, rcand, hrp, hci, hva, feat + (base + t) * kNF);
        pj[base + t] = j;
    }
}

// The (H^2)_ij feature of every candidate pair.  One warp per site i keys a shared-memory hash
// table by the site's candidates j and accumulates (H^2)_ij = sum_k H_ik H_kj into it, taking
// k in ascending order (one row k at a time, its entries across the lanes; an entry l of row
// k that is not a candidate is skipped): every (H^2)_ij is then the same sequence of products
// and additions as the ordered merge of rows i and j (H is symmetric to the last bit), so the
// feature is symmetric in (i, j) bit for bit.  A site with more candidates than three
// quarters of the table is computed by that merge.
constexpr int kH2Bits = 9;
constexpr int kH2Slots = 1 << kH2Bits;              // hash slots per warp (~270 candidates within 4a)
constexpr int kH2MaxKeys = kH2Slots * 3 / 4;
constexpr int kH2Warps = 4;
constexpr size_t kH2Smem = (size_t)kH2Warps * kH2Slots * (4 + 8);

__device__ __forceinline__ unsigned h2_hash(int l) { return ((unsigned)l * 2654435761u) >> (32 - kH2Bits); }

__global__ void __launch_bounds__(32 * kH2Warps) h2_feature_kernel(int64_t n, const int64_t* __restrict__ hrp,
                                                                    const int32_t* __restrict__ hci,
                                                                    const double* __restrict__ hva,
                                                                    const int64_t* __restrict__ prp,
                                                                    const int32_t* __restrict__ pj, float* feat) {
    extern __shared__ unsigned char h2sm[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * kH2Warps + w;
    if (i >= n) return;
    int* keys = reinterpret_cast<int*>(h2sm) + w * kH2Slots;
    double* vals = reinterpret_cast<double*>(h2sm + (size_t)kH2Warps * kH2Slots * 4) + w * kH2Slots;
    for (int t = lane; t < kH2Slots; t += 32) {
        keys[t] = -1;
        vals[t] = 0.0;
    }
    __syncwarp();
    // the table is keyed by the site's candidates (distinct j, at most three quarters of the
    // slots, so every probe sequence ends at an empty slot); a product H_ik H_kl is added only
    // when l is one of them, the other entries of row i of H^2 are not features
    const int64_t c0 = prp[i], c1 = prp[i + 1];
    bool ok = (c1 - c0) <= kH2MaxKeys;
    if (ok) {
        for (int64_t t = c0 + lane; t < c1; t += 32) {
            const int j = pj[t];
            unsigned h = h2_hash(j);
            for (int probes = 0; probes < kH2Slots; ++probes) {
                const int old = atomicCAS(&keys[h], -1, j);
                if (old == -1 || old == j) break;
                h = (h + 1) & (kH2Slots - 1);
            }
        }
    }
    __syncwarp();
    // row i's entries 32 at a time, each lane holding one k with its H_ik and the range of row
    // k (loaded together), then taken in ascending order across the warp
    const int64_t p0 = hrp[i], p1 = ok ? hrp[i + 1] : p0;
    for (int64_t pb = p0; pb < p1; pb += 32) {
        const int64_t pl = pb + lane;
        double hl = 0.0;
        int64_t ql0 = 0, ql1 = 0;
        if (pl < p1) {
            const int kl = hci[pl];
            hl = hva[pl];
            ql0 = hrp[kl];
            ql1 = hrp[kl + 1];
        }
        const int nk = (p1 - pb) < 32 ? (int)(p1 - pb) : 32;
        for (int u = 0; u < nk; ++u) {
            const double hik = __shfl_sync(0xffffffffu, hl, u);
            const int64_t q0 = __shfl_sync(0xffffffffu, ql0, u), q1 = __shfl_sync(0xffffffffu, ql1, u);
            for (int64_t q = q0 + lane; q < q1; q += 32) {
                const int l = hci[q];
                unsigned h = h2_hash(l);
                int key = keys[h];
                for (int probes = 1; key != l && key != -1 && probes < kH2Slots; ++probes) {
                    h = (h + 1) & (kH2Slots - 1);
                    key = keys[h];
                }
                if (key == l) vals[h] = __dadd_rn(vals[h], __dmul_rn(hik, hva[q]));   // one lane per key
            }
            __syncwarp();
        }
    }
    ok = __all_sync(0xffffffffu, ok);
    for (int64_t t = prp[i] + lane; t < prp[i + 1]; t += 32) {
        const int j = pj[t];
        double h2 = 0.0;
        if (ok) {
            unsigned h = h2_hash(j);
            for (int probes = 0; probes < kH2Slots; ++probes) {
                const int key = keys[h];
                if (key == j) { h2 = vals[h]; break; }
                if (key == -1) break;
                h = (h + 1) & (kH2Slots - 1);
            }
        } else {
            h2 = row_dot(hrp, hci, hva, (int)i, j);
        }
        feat[t * kNF + 1] = -log10f(fmaxf((float)fabs(h2), 1e-12f)) / 12.0f;
    }
}

// ------------------------------------------------------------------ MLP
__device__ __forceinline__ uint32_t h2_bits_mlp(__half2 h) {
    uint32_t u;
    memcpy(&u, &h, 4);
    return u;
}

__global__ void round_params_kernel(const float* __restrict__ p, float* pw) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNParams; i += gridDim.x * blockDim.x)
        pw[i] = __half2float(__float2half_rn(p[i]));
}

// ------------------------------------------------------------------ forward on the tensor cores
// The 64 x 64 layer as mma.sync m16n8k16 (fp16 operands, FP32 accumulation): a warp takes 16
// pairs at a time (the M rows), the hidden units are K (4 k-steps of 16) and the outputs N
// (8 tiles of 8).  W2 is fp16-rounded already, so its fragments are exact; h1 is carried as
// hi = fp16(h1) plus lo = fp16(h1 - hi) (relative error 2^-22), two MMAs per fragment, so
// the layer keeps FP32-class accuracy.  Layer 1 (5 inputs) runs on the FP32 pipe straight
// into the A-fragment layout; layer 3 is a dot product finished across the 4 lanes of a
// fragment row.  (|h1| must stay below the fp16 range, 65504.)
__device__ __forceinline__ uint32_t pack_h2(float lo_elem, float hi_elem) {
    return h2_bits_mlp(__floats2half2_rn(lo_elem, hi_elem));
}

__device__ __forceinline__ void mma_16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(256) mlp_forward_tc_kernel(const float* __restrict__ feat, int64_t npairs,
                                                             const float* __restrict__ pw, float* logits) {
    __shared__ float W1s[kHid * kNF], B1s[kHid], B2s[kHid], W3s[kHid];
    for (int i = threadIdx.x; i < kHid * kNF; i += blockDim.x) W1s[i] = pw[OW1 + i];
    for (int i = threadIdx.x; i < kHid; i += blockDim.x) {
        B1s[i] = pw[OB1 + i];
        B2s[i] = pw[OB2 + i];
        W3s[i] = pw[OW3 + i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    // B fragments of W2^T (k = input unit, n = output unit): rows 2t, 2t+1 and 2t+8, 2t+9 of
    // each 16 x 8 block, column g
    uint32_t bf[4][8][2];
#pragma unroll
    for (int ks = 0; ks < 4; ++ks)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const float* r = pw + OW2 + (8 * nt + g) * kHid + 16 * ks + 2 * t;
            bf[ks][nt][0] = pack_h2(r[0], r[1]);
            bf[ks][nt][1] = pack_h2(r[8], r[9]);
        }
    const float b3 = pw[OB3];
    const int64_t ngroups = (npairs + 15) / 16;
    for (int64_t grp = (int64_t)blockIdx.x * 8 + warp; grp < ngroups; grp += (int64_t)gridDim.x * 8) {
        const int64_t p0 = grp * 16 + g, p1 = p0 + 8;   // the two fragment rows of this lane
        float f[2][kNF];
#pragma unroll
        for (int q = 0; q < kNF; ++q) {
            f[0][q] = p0 < npairs ? feat[p0 * kNF + q] : 0.0f;
            f[1][q] = p1 < npairs ? feat[p1 * kNF + q] : 0.0f;
        }
        float acc[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            acc[nt][0] = acc[nt][2] = B2s[8 * nt + 2 * t];
            acc[nt][1] = acc[nt][3] = B2s[8 * nt + 2 * t + 1];
        }
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            // h1 of units 16 ks + 2t + {0, 1, 8, 9} for both rows, split into fp16 hi + lo
            float hi[2][4], lo[2][4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int u = 16 * ks + 2 * t + (e & 1) + 8 * (e >> 1);
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    float a = B1s[u];
#pragma unroll
                    for (int q = 0; q < kNF; ++q) a = fmaf(W1s[u * kNF + q], f[r][q], a);
                    const float h = fmaxf(a, 0.0f);
                    hi[r][e] = __half2float(__float2half_rn(h));
                    lo[r][e] = h - hi[r][e];
                }
            }
            const uint32_t ah[4] = {pack_h2(hi[0][0], hi[0][1]), pack_h2(hi[1][0], hi[1][1]), pack_h2(hi[0][2], hi[0][3]),
                                    pack_h2(hi[1][2], hi[1][3])};
            const uint32_t al[4] = {pack_h2(lo[0][0], lo[0][1]), pack_h2(lo[1][0], lo[1][1]), pack_h2(lo[0][2], lo[0][3]),
                                    pack_h2(lo[1][2], lo[1][3])};
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                mma_16816(acc[nt], ah, bf[ks][nt][0], bf[ks][nt][1]);
                mma_16816(acc[nt], al, bf[ks][nt][0], bf[ks][nt][1]);
            }
        }
        float z0 = 0.0f, z1 = 0.0f;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const float w0 = W3s[8 * nt + 2 * t], w1 = W3s[8 * nt + 2 * t + 1];
            z0 = fmaf(w0, fmaxf(acc[nt][0], 0.0f), z0);
            z0 = fmaf(w1, fmaxf(acc[nt][1], 0.0f), z0);
            z1 = fmaf(w0, fmaxf(acc[nt][2], 0.0f), z1);
            z1 = fmaf(w1, fmaxf(acc[nt][3], 0.0f), z1);
        }
        z0 += __shfl_xor_sync(0xffffffffu, z0, 1);
        z1 += __shfl_xor_sync(0xffffffffu, z1, 1);
        z0 += __shfl_xor_sync(0xffffffffu, z0, 2);
        z1 += __shfl_xor_sync(0xffffffffu, z1, 2);
        if (t == 0) {
            if (p0 < npairs) logits[p0] = z0 + b3;
            if (p1 < npairs) logits[p1] = z1 + b3;
        }
    }
}

// Gradient on the tensor cores.  Per batch of 128 pairs (4 warps x 2 tiles of 16 rows):
//   forward   h1 (FP32 pipe, A-fragment layout, fp16 hi + lo), a2 = W2 h1 + b2 (mma), h2, z
//   backward  dz' = sigmoid(z) - y (the 1/n of the mean is applied at the end, so that the
//             small values stay in fp16's range), d2' = (h2 > 0) dz' w3,
//             d1' = (h1 > 0) (d2' W2) (mma: the layer-2 accumulator fragments are the A
//             fragments of this product), and per warp gW2 rows += d2'^T h1 over the batch
//             (mma with the batch as K, from the hi/lo halves staged in shared memory:
//             hi hi + hi lo + lo hi, relative error ~2^-21)
//   the small blocks (w3, b3, b2, W1, b1) are reduced over the batch by owner threads in a
//   fixed order, as on the FP32 pipe; gW2 stays in each warp's registers across batches.
struct GradSmem {
    float W[kNParams];
    float G[kNParams];
    uint32_t w2t[4][8][2][32];   // B fragments of W2^T (forward), per lane
    uint32_t w2n[4][8][2][32];   // B fragments of W2 (backward to h1), per lane
    __half H1h[kBatch][kHid + 8], H1l[kBatch][kHid + 8];   // h1 = hi + lo
    __half D2h[kBatch][kHid + 8], D2l[kBatch][kHid + 8];   // d2' = hi + lo
    float H2[kBatch][kLd];
    float D1[kBatch][kLd];      // dL/dh1 (with the 1/n)
    float F[kBatch][8];
    float dz[kBatch];           // dL/dz (with the 1/n)
};

__device__ __forceinline__ uint32_t ld_pair(const __half* p0, const __half* p1) {
    return (uint32_t)__half_as_ushort(*p0) | ((uint32_t)__half_as_ushort(*p1) << 16);
}

__global__ void __launch_bounds__(kBatch) mlp_grad_kernel(const float* __restrict__ feat,
                                                          const uint8_t* __restrict__ labels, int64_t npairs,
                                                          const float* __restrict__ pw, float inv_n, float* partials,
                                                          double* loss_part) {
    extern __shared__ unsigned char gsm_raw[];
    GradSmem& S = *reinterpret_cast<GradSmem*>(gsm_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    for (int i = tid; i < kNParams; i += kBatch) { S.W[i] = pw[i]; S.G[i] = 0.0f; }
    __syncthreads();
    // this lane's B fragments: W2^T (k = input unit, n = output) and W2 (k = output, n = input)
    for (int e = tid; e < 4 * 8 * 2 * 32; e += kBatch) {
        const int ln = e & 31, reg = (e >> 5) & 1, nt = (e >> 6) & 7, ks = e >> 9;
        const int gg = ln >> 2, tt = ln & 3;
        const int k0 = 16 * ks + 2 * tt + 8 * reg, n = 8 * nt + gg;
        S.w2t[ks][nt][reg][ln] = pack_h2(S.W[OW2 + n * kHid + k0], S.W[OW2 + n * kHid + k0 + 1]);
        S.w2n[ks][nt][reg][ln] = pack_h2(S.W[OW2 + k0 * kHid + n], S.W[OW2 + (k0 + 1) * kHid + n]);
    }
    __syncthreads();
    float gw2[8][4];   // gW2 rows 16 warp + {g, g + 8}, columns 8 nt + 2t + {0, 1}
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) gw2[nt][0] = gw2[nt][1] = gw2[nt][2] = gw2[nt][3] = 0.0f;
    double lsum = 0.0;
    for (int64_t b0 = (int64_t)blockIdx.x * kBatch; b0 < npairs; b0 += (int64_t)gridDim.x * kBatch) {
#pragma unroll 1
        for (int rt = 0; rt < 2; ++rt) {
            const int r0 = 32 * warp + 16 * rt + g, r1 = r0 + 8;     // rows of the batch
            const int64_t q0 = b0 + r0, q1 = b0 + r1;
            const bool v0 = q0 < npairs, v1 = q1 < npairs;
            float f[2][kNF];
#pragma unroll
            for (int q = 0; q < kNF; ++q) {
                f[0][q] = v0 ? feat[q0 * kNF + q] : 0.0f;
                f[1][q] = v1 ? feat[q1 * kNF + q] : 0.0f;
            }
            if (t == 0) {
#pragma unroll
                for (int q = 0; q < kNF; ++q) { S.F[r0][q] = f[0][q]; S.F[r1][q] = f[1][q]; }
            }
            // forward: h1 (hi/lo A fragments, also staged for gW2), a2 = W2 h1 + b2
            float acc[8][4];
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                acc[nt][0] = acc[nt][2] = S.W[OB2 + 8 * nt + 2 * t];
                acc[nt][1] = acc[nt][3] = S.W[OB2 + 8 * nt + 2 * t + 1];
            }
            uint32_t h1pos = 0;   // bit (4 ks + e) * 2 + row: h1 > 0
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                float hi[2][4], lo[2][4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int u = 16 * ks + 2 * t + (e & 1) + 8 * (e >> 1);
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        float a = S.W[OB1 + u];
#pragma unroll
                        for (int q = 0; q < kNF; ++q) a = fmaf(S.W[OW1 + u * kNF + q], f[r][q], a);
                        const float h = fmaxf(a, 0.0f);
                        if (h > 0.0f) h1pos |= 1u << ((4 * ks + e) * 2 + r);
                        hi[r][e] = __half2float(__float2half_rn(h));
                        lo[r][e] = h - hi[r][e];
                    }
                }
                const uint32_t ah[4] = {pack_h2(hi[0][0], hi[0][1]), pack_h2(hi[1][0], hi[1][1]),
                                        pack_h2(hi[0][2], hi[0][3]), pack_h2(hi[1][2], hi[1][3])};
                const uint32_t al[4] = {pack_h2(lo[0][0], lo[0][1]), pack_h2(lo[1][0], lo[1][1]),
                                        pack_h2(lo[0][2], lo[0][3]), pack_h2(lo[1][2], lo[1][3])};
                *reinterpret_cast<uint32_t*>(&S.H1h[r0][16 * ks + 2 * t]) = ah[0];
                *reinterpret_cast<uint32_t*>(&S.H1h[r1][16 * ks + 2 * t]) = ah[1];
                *reinterpret_cast<uint32_t*>(&S.H1h[r0][16 * ks + 2 * t + 8]) = ah[2];
                *reinterpret_cast<uint32_t*>(&S.H1h[r1][16 * ks + 2 * t + 8]) = ah[3];
                *reinterpret_cast<uint32_t*>(&S.H1l[r0][16 * ks + 2 * t]) = al[0];
                *reinterpret_cast<uint32_t*>(&S.H1l[r1][16 * ks + 2 * t]) = al[1];
                *reinterpret_cast<uint32_t*>(&S.H1l[r0][16 * ks + 2 * t + 8]) = al[2];
                *reinterpret_cast<uint32_t*>(&S.H1l[r1][16 * ks + 2 * t + 8]) = al[3];
#pragma unroll
                for (int nt = 0; nt < 8; ++nt) {
                    const uint32_t bb0 = S.w2t[ks][nt][0][lane], bb1 = S.w2t[ks][nt][1][lane];
                    mma_16816(acc[nt], ah, bb0, bb1);
                    mma_16816(acc[nt], al, bb0, bb1);
                }
            }
            // h2, z, loss, dz'
            float z0 = 0.0f, z1 = 0.0f;
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[nt][e] = fmaxf(acc[nt][e], 0.0f);
                const float w0 = S.W[OW3 + 8 * nt + 2 * t], w1 = S.W[OW3 + 8 * nt + 2 * t + 1];
                z0 = fmaf(w0, acc[nt][0], z0);
                z0 = fmaf(w1, acc[nt][1], z0);
                z1 = fmaf(w0, acc[nt][2], z1);
                z1 = fmaf(w1, acc[nt][3], z1);
                S.H2[r0][8 * nt + 2 * t] = acc[nt][0];
                S.H2[r0][8 * nt + 2 * t + 1] = acc[nt][1];
                S.H2[r1][8 * nt + 2 * t] = acc[nt][2];
                S.H2[r1][8 * nt + 2 * t + 1] = acc[nt][3];
            }
            z0 += __shfl_xor_sync(0xffffffffu, z0, 1);
            z1 += __shfl_xor_sync(0xffffffffu, z1, 1);
            z0 += __shfl_xor_sync(0xffffffffu, z0, 2);
            z1 += __shfl_xor_sync(0xffffffffu, z1, 2);
            z0 += S.W[OB3];
            z1 += S.W[OB3];
            const float y0 = v0 ? (float)labels[q0] : 0.0f, y1 = v1 ? (float)labels[q1] : 0.0f;
            const float d0 = v0 ? 1.0f / (1.0f + __expf(-z0)) - y0 : 0.0f;
            const float d1 = v1 ? 1.0f / (1.0f + __expf(-z1)) - y1 : 0.0f;
            if (t == 0) {
                if (v0) lsum += (double)(fmaxf(z0, 0.0f) - y0 * z0 + log1pf(__expf(-fabsf(z0))));
                if (v1) lsum += (double)(fmaxf(z1, 0.0f) - y1 * z1 + log1pf(__expf(-fabsf(z1))));
                S.dz[r0] = d0 * inv_n;
                S.dz[r1] = d1 * inv_n;
            }
            // d2' = (h2 > 0) dz' w3 as hi/lo A fragments of the product d2' W2 (the C fragment
            // tiles 2 ks and 2 ks + 1 are the k = 16 ks .. 16 ks + 15 columns), staged for gW2
            float acc1[8][4];
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) acc1[nt][0] = acc1[nt][1] = acc1[nt][2] = acc1[nt][3] = 0.0f;
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                float dv[2][2][2];   // [tile 2ks + j][row][col pair]
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int nt = 2 * ks + j;
                    const float w0 = S.W[OW3 + 8 * nt + 2 * t], w1 = S.W[OW3 + 8 * nt + 2 * t + 1];
                    dv[j][0][0] = acc[nt][0] > 0.0f ? d0 * w0 : 0.0f;
                    dv[j][0][1] = acc[nt][1] > 0.0f ? d0 * w1 : 0.0f;
                    dv[j][1][0] = acc[nt][2] > 0.0f ? d1 * w0 : 0.0f;
                    dv[j][1][1] = acc[nt][3] > 0.0f ? d1 * w1 : 0.0f;
                }
                float hh[2][2][2], ll[2][2][2];
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int r = 0; r < 2; ++r)
#pragma unroll
                        for (int c = 0; c < 2; ++c) {
                            hh[j][r][c] = __half2float(__float2half_rn(dv[j][r][c]));
                            ll[j][r][c] = dv[j][r][c] - hh[j][r][c];
                        }
                const uint32_t ah[4] = {pack_h2(hh[0][0][0], hh[0][0][1]), pack_h2(hh[0][1][0], hh[0][1][1]),
                                        pack_h2(hh[1][0][0], hh[1][0][1]), pack_h2(hh[1][1][0], hh[1][1][1])};
                const uint32_t al[4] = {pack_h2(ll[0][0][0], ll[0][0][1]), pack_h2(ll[0][1][0], ll[0][1][1]),
                                        pack_h2(ll[1][0][0], ll[1][0][1]), pack_h2(ll[1][1][0], ll[1][1][1])};
                *reinterpret_cast<uint32_t*>(&S.D2h[r0][16 * ks + 2 * t]) = ah[0];
                *reinterpret_cast<uint32_t*>(&S.D2h[r1][16 * ks + 2 * t]) = ah[1];
                *reinterpret_cast<uint32_t*>(&S.D2h[r0][16 * ks + 2 * t + 8]) = ah[2];
                *reinterpret_cast<uint32_t*>(&S.D2h[r1][16 * ks + 2 * t + 8]) = ah[3];
                *reinterpret_cast<uint32_t*>(&S.D2l[r0][16 * ks + 2 * t]) = al[0];
                *reinterpret_cast<uint32_t*>(&S.D2l[r1][16 * ks + 2 * t]) = al[1];
                *reinterpret_cast<uint32_t*>(&S.D2l[r0][16 * ks + 2 * t + 8]) = al[2];
                *reinterpret_cast<uint32_t*>(&S.D2l[r1][16 * ks + 2 * t + 8]) = al[3];
#pragma unroll
                for (int nt = 0; nt < 8; ++nt) {
                    const uint32_t bb0 = S.w2n[ks][nt][0][lane], bb1 = S.w2n[ks][nt][1][lane];
                    mma_16816(acc1[nt], ah, bb0, bb1);
                    mma_16816(acc1[nt], al, bb0, bb1);
                }
            }
            // d1 = (h1 > 0) d1' / n, columns 8 nt + 2t + {0, 1}: A-fragment unit 16 ks + 2t + e
            // of layer 1 is C tile nt = 2 ks + (e >> 1), column 2t + (e & 1)
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int e = (c & 1) + 2 * (nt & 1), ks = nt >> 1;
                    const bool p0 = (h1pos >> ((4 * ks + e) * 2)) & 1u, p1 = (h1pos >> ((4 * ks + e) * 2 + 1)) & 1u;
                    S.D1[r0][8 * nt + 2 * t + c] = p0 ? acc1[nt][c] * inv_n : 0.0f;
                    S.D1[r1][8 * nt + 2 * t + c] = p1 ? acc1[nt][2 + c] * inv_n : 0.0f;
                }
        }
        __syncthreads();
        // small blocks, each entry owned by one thread, batch order fixed
        if (tid < kHid) {
            float acc = 0.0f;
            for (int b = 0; b < kBatch; ++b) acc = fmaf(S.dz[b], S.H2[b][tid], acc);
            S.G[OW3 + tid] += acc;
            float gw[kNF] = {0.f, 0.f, 0.f, 0.f, 0.f};
            float gb = 0.0f;
            for (int b = 0; b < kBatch; ++b) {
                const float d = S.D1[b][tid];
                gb += d;
#pragma unroll
                for (int q = 0; q < kNF; ++q) gw[q] = fmaf(d, S.F[b][q], gw[q]);
            }
#pragma unroll
            for (int q = 0; q < kNF; ++q) S.G[OW1 + tid * kNF + q] += gw[q];
            S.G[OB1 + tid] += gb;
        } else {
            const int o = tid - kHid;
            float acc = 0.0f;
            for (int b = 0; b < kBatch; ++b) acc += __half2float(S.D2h[b][o]) + __half2float(S.D2l[b][o]);
            S.G[OB2 + o] += acc * inv_n;
            if (o == 0) {
                float a3 = 0.0f;
                for (int b = 0; b < kBatch; ++b) a3 += S.dz[b];
                S.G[OB3] += a3;
            }
        }
        // gW2 rows 16 warp .. 16 warp + 15: d2'^T h1 with the batch as K (hi hi + hi lo + lo hi)
#pragma unroll 1
        for (int kb = 0; kb < kBatch / 16; ++kb) {
            const int bA = 16 * kb + 2 * t, o0 = 16 * warp + g;
            uint32_t dh[4], dl[4];
            dh[0] = ld_pair(&S.D2h[bA][o0], &S.D2h[bA + 1][o0]);
            dh[1] = ld_pair(&S.D2h[bA][o0 + 8], &S.D2h[bA + 1][o0 + 8]);
            dh[2] = ld_pair(&S.D2h[bA + 8][o0], &S.D2h[bA + 9][o0]);
            dh[3] = ld_pair(&S.D2h[bA + 8][o0 + 8], &S.D2h[bA + 9][o0 + 8]);
            dl[0] = ld_pair(&S.D2l[bA][o0], &S.D2l[bA + 1][o0]);
            dl[1] = ld_pair(&S.D2l[bA][o0 + 8], &S.D2l[bA + 1][o0 + 8]);
            dl[2] = ld_pair(&S.D2l[bA + 8][o0], &S.D2l[bA + 9][o0]);
            dl[3] = ld_pair(&S.D2l[bA + 8][o0 + 8], &S.D2l[bA + 9][o0 + 8]);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const int i = 8 * nt + g;
                const uint32_t hh0 = ld_pair(&S.H1h[bA][i], &S.H1h[bA + 1][i]);
                const uint32_t hh1 = ld_pair(&S.H1h[bA + 8][i], &S.H1h[bA + 9][i]);
                const uint32_t hl0 = ld_pair(&S.H1l[bA][i], &S.H1l[bA + 1][i]);
                const uint32_t hl1 = ld_pair(&S.H1l[bA + 8][i], &S.H1l[bA + 9][i]);
                mma_16816(gw2[nt], dh, hh0, hh1);
                mma_16816(gw2[nt], dh, hl0, hl1);
                mma_16816(gw2[nt], dl, hh0, hh1);
            }
        }
        __syncthreads();
    }
    for (int i = tid; i < kNParams; i += kBatch)
        if (i < OW2 || i >= OB2) partials[(int64_t)blockIdx.x * kNParams + i] = S.G[i];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int o = 16 * warp + g, i = 8 * nt + 2 * t;
        float* dst = partials + (int64_t)blockIdx.x * kNParams + OW2;
        dst[o * kHid + i] = gw2[nt][0] * inv_n;
        dst[o * kHid + i + 1] = gw2[nt][1] * inv_n;
        dst[(o + 8) * kHid + i] = gw2[nt][2] * inv_n;
        dst[(o + 8) * kHid + i + 1] = gw2[nt][3] * inv_n;
    }
    // fixed-order loss reduction within the CTA
    __shared__ double lred[kBatch];
    lred[tid] = lsum;
    __syncthreads();
    if (tid == 0) {
        double sum = 0.0;
        for (int b = 0; b < kBatch; ++b) sum += lred[b];
        loss_part[blockIdx.x] = sum;
    }
}

__global__ void reduce_grad_kernel(const float* __restrict__ partials, int nblocks, float* g, const double* loss_part,
                                   double* loss_out, double inv_n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNParams; i += gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int b = 0; b < nblocks; ++b) s += partials[(int64_t)b * kNParams + i];
        g[i] = s;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += loss_part[b];
        *loss_out = s * inv_n;
    }
}

__global__ void adam_kernel(float* p, float* m, float* v, const float* __restrict__ g, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNParams; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// selected edges (logit >= cut): counts per site, then fill
__global__ void select_count_kernel(const int64_t* __restrict__ rowptr, const float* __restrict__ logits, int64_t n,
                                    float cut, int32_t* cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = 0;
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) c += logits[p] >= cut;
    cnt[i] = c;
}

__global__ void select_fill_kernel(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ pj,
                                   const float* __restrict__ logits, int64_t n, float cut, const int64_t* __restrict__ orp,
                                   int32_t* oci) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t o = orp[i];
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
        if (logits[p] >= cut) oci[o++] = pj[p];
}

size_t grad_smem() { return sizeof(GradSmem); }

}  // namespace

struct gbe_pairs {
    int64_t n = 0, npairs = 0;
    int64_t* rowptr = nullptr;
    int32_t* j = nullptr;
    float* feat = nullptr;
};

struct gbe_mlp {
    float* p = nullptr;        // fp32 master parameters
    float* pw = nullptr;       // fp16-rounded copy used by the forward pass
    float* m = nullptr;
    float* v = nullptr;
    float* g = nullptr;
    double* loss = nullptr;    // last mean loss (device)
    float* partials = nullptr; // [nblocks][kNParams]
    double* loss_part = nullptr;
    int nblocks = 0;
    int t = 0;                 // Adam steps taken
};

extern "C" int gbe_free_pairs(gbe_pairs* P) {
    if (!P) return GBE_OK;
    gbe_free(P->rowptr); gbe_free(P->j); gbe_free(P->feat);
    delete P;
    return GBE_OK;
}

extern "C" int gbe_pairs_build(gbe_ctx* ctx, const gbe_sites* st, const gbe_csr* Hin, double rcand, gbe_pairs** out) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && st && Hin && out, "NULL argument");
    GBE_CHECK_ARG(st->n > 0 && st->n == Hin->n && st->n < INT32_MAX, "sites / H sizes");
    GBE_CHECK_ARG(rcand > 0.0, "rcand");
    for (int d = 0; d < 3; ++d) GBE_CHECK_ARG(st->box[d] > 2.0 * rcand, "box must exceed 2 rcand (minimum image)");
    GBE_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    const int64_t n = st->n;
    DevBuf hpos, hons, hrp, hci, hva;
    const double *pos, *ons;
    GBE_TRY(to_device(ctx, st->pos, n * 24, st->on_device, hpos, (const void**)&pos));
    GBE_TRY(to_device(ctx, st->onsite, n * 8, st->on_device, hons, (const void**)&ons));
    const int64_t* rp;
    const int32_t* ci;
    const double* va;
    GBE_TRY(to_device(ctx, Hin->rowptr, (n + 1) * 8, Hin->on_device, hrp, (const void**)&rp));
    GBE_TRY(to_device(ctx, Hin->col, Hin->nnz * 4, Hin->on_device, hci, (const void**)&ci));
    GBE_TRY(to_device(ctx, Hin->val, Hin->nnz * 8, Hin->on_device, hva, (const void**)&va));
    CellGrid g;
    int64_t ncells = 1;
    for (int d = 0; d < 3; ++d) {
        g.nc[d] = std::max(1, (int)floor(st->box[d] / rcand));
        g.box[d] = st->box[d];
        g.inv[d] = 1.0 / st->box[d];
        ncells *= g.nc[d];
    }
    DevBuf cell, ccnt, cst, cur, mem, cnt, flag;
    GBE_TRY(gbe_alloc(&cell.p, n * 4));
    GBE_TRY(gbe_alloc(&ccnt.p, ncells * 4));
    GBE_TRY(gbe_alloc(&cst.p, (ncells + 1) * 8));
    GBE_TRY(gbe_alloc(&cur.p, ncells * 4));
    GBE_TRY(gbe_alloc(&mem.p, n * 4));
    GBE_TRY(gbe_alloc(&cnt.p, n * 4));
    GBE_TRY(gbe_alloc(&flag.p, 8));   // [0] a site above kPairCap, [1] a site above kPairStage
    cudaMemsetAsync(ccnt.p, 0, ncells * 4, s);
    cudaMemsetAsync(cur.p, 0, ncells * 4, s);
    cudaMemsetAsync(flag.p, 0, 8, s);
    const unsigned nb = (unsigned)((n + 255) / 256);
    cell_count_kernel<<<nb, 256, 0, s>>>(pos, n, g, cell.as<int32_t>(), ccnt.as<int32_t>());
    GBE_TRY(scan_exclusive(ctx, ccnt.as<int32_t>(), cst.as<int64_t>(), ncells, nullptr));
    cell_fill_kernel<<<nb, 256, 0, s>>>(cell.as<int32_t>(), n, cst.as<int64_t>(), cur.as<int32_t>(), mem.as<int32_t>());
    const unsigned rb = (unsigned)((n + 7) / 8);
    DevBuf p4;
    GBE_TRY(gbe_alloc(&p4.p, n * 16));
    pos_f32_kernel<<<nb, 256, 0, s>>>(pos, n, p4.as<float4>());
    const float lim2 = filter_lim2(rcand, st->box), lim2_in = filter_lim2_in(rcand, st->box);
    // one search: sorted candidates into staging slots (pass 2); a site with more candidates
    // than a slot sends the build through the counting and filling passes 0 and 1
    DevBuf stage;
    GBE_TRY(gbe_alloc(&stage.p, (size_t)n * kPairStage * 4));
    pairs_kernel<<<rb, 256, 0, s>>>(pos, p4.as<float4>(), ons, n, g, lim2, lim2_in, cst.as<int64_t>(), mem.as<int32_t>(), rcand, 2,
                                    cnt.as<int32_t>(),
                                    nullptr, stage.as<int32_t>(), nullptr, rp, ci, va, flag.as<int>());
    GBE_CUDA_TRY(cudaGetLastError());
    gbe_pairs* P = new gbe_pairs();
    P->n = n;
    int r = gbe_alloc((void**)&P->rowptr, (n + 1) * 8);
    int64_t np = 0;
    if (r == GBE_OK) r = scan_exclusive(ctx, cnt.as<int32_t>(), P->rowptr, n, &np);
    int ovf[2] = {0, 0};
    if (r == GBE_OK) {
        cudaError_t fe = cudaMemcpyAsync(ovf, flag.p, 8, cudaMemcpyDeviceToHost, s);
        if (fe == cudaSuccess) fe = cudaStreamSynchronize(s);
        if (fe != cudaSuccess) {
            gbe_set_error("pairs: reading the overflow flags: %s", cudaGetErrorString(fe));
            r = GBE_ECUDA;
        }
    }
    if (r == GBE_OK && ovf[0]) { gbe_set_error("a site has more than %d candidates within rcand", kPairCap); r = GBE_ECAPACITY; }
    if (r == GBE_OK) r = gbe_alloc((void**)&P->j, std::max<int64_t>(np, 1) * 4);
    if (r == GBE_OK) r = gbe_alloc((void**)&P->feat, std::max<int64_t>(np, 1) * kNF * 4);
    if (r != GBE_OK) { gbe_free_pairs(P); return r; }
    P->npairs = np;
    if (!ovf[1])
        pair_stage_kernel<<<rb, 256, 0, s>>>(pos, ons, n, g, rcand, stage.as<int32_t>(), P->rowptr, P->j, P->feat, rp, ci,
                                             va);
    else
        pairs_kernel<<<rb, 256, 0, s>>>(pos, p4.as<float4>(), ons, n, g, lim2, lim2_in, cst.as<int64_t>(), mem.as<int32_t>(),
                                        rcand, 1, cnt.as<int32_t>(), P->rowptr, P->j, P->feat, rp, ci, va, flag.as<int>());
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(h2_feature_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kH2Smem);
    if (e == cudaSuccess) {
        h2_feature_kernel<<<(unsigned)((n + kH2Warps - 1) / kH2Warps), 32 * kH2Warps, kH2Smem, s>>>(n, rp, ci, va, P->rowptr,
                                                                                                   P->j, P->feat);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        gbe_free_pairs(P);
        gbe_set_error("pairs: %s", cudaGetErrorString(e));
        return GBE_ECUDA;
    }
    *out = P;
    return GBE_OK;
}

extern "C" int gbe_pairs_info(const gbe_pairs* P, int64_t* n, int64_t* npairs) {
    GBE_CHECK_ARG(P != nullptr, "pairs is NULL");
    if (n) *n = P->n;
    if (npairs) *npairs = P->npairs;
    return GBE_OK;
}

extern "C" int gbe_pairs_export(gbe_ctx* ctx, const gbe_pairs* P, int64_t* rowptr, int32_t* j, float* features) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && P, "NULL argument");
    cudaStream_t s = ctx->stream;
    if (rowptr) GBE_CUDA_TRY(cudaMemcpyAsync(rowptr, P->rowptr, (P->n + 1) * 8, cudaMemcpyDeviceToHost, s));
    if (j && P->npairs) GBE_CUDA_TRY(cudaMemcpyAsync(j, P->j, P->npairs * 4, cudaMemcpyDeviceToHost, s));
    if (features && P->npairs) GBE_CUDA_TRY(cudaMemcpyAsync(features, P->feat, P->npairs * kNF * 4, cudaMemcpyDeviceToHost, s));
    GBE_CUDA_TRY(cudaStreamSynchronize(s));
    return GBE_OK;
}

extern "C" int gbe_pairs_device(const gbe_pairs* P, const int64_t** rowptr, const int32_t** j, const float** features) {
    GBE_CHECK_ARG(P, "NULL pairs");
    if (rowptr) *rowptr = P->rowptr;
    if (j) *j = P->j;
    if (features) *features = P->feat;
    return GBE_OK;
}

extern "C" int gbe_free_mlp(gbe_mlp* M) {
    if (!M) return GBE_OK;
    gbe_free(M->p); gbe_free(M->pw); gbe_free(M->m); gbe_free(M->v); gbe_free(M->g); gbe_free(M->loss);
    gbe_free(M->partials); gbe_free(M->loss_part);
    delete M;
    return GBE_OK;
}

extern "C" int gbe_mlp_create(gbe_ctx* ctx, int hidden, gbe_mlp** out) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && out, "NULL argument");
    GBE_CHECK_ARG(hidden == kHid, "only hidden width 64 is built");
    GBE_CUDA_TRY(cudaSetDevice(ctx->device));
    gbe_mlp* M = new gbe_mlp();
    M->nblocks = ctx->sm_count;
    int r = GBE_OK;
    if (r == GBE_OK) r = gbe_alloc((void**)&M->p, kNParams * 4);
    if (r == GBE_OK) r = gbe_alloc((void**)&M->pw, kNParams * 4);
    if (r == GBE_OK) r = gbe_alloc((void**)&M->m, kNParams * 4);
    if (r == GBE_OK) r = gbe_alloc((void**)&M->v, kNParams * 4);
    if (r == GBE_OK) r = gbe_alloc((void**)&M->g, kNParams * 4);
    if (r == GBE_OK) r = gbe_alloc((void**)&M->loss, 8);
    if (r == GBE_OK) r = gbe_alloc((void**)&M->partials, (size_t)M->nblocks * kNParams * 4);
    if (r == GBE_OK) r = gbe_alloc((void**)&M->loss_part, (size_t)M->nblocks * 8);
    if (r != GBE_OK) { gbe_free_mlp(M); return r; }
    cudaMemsetAsync(M->p, 0, kNParams * 4, ctx->stream);
    cudaMemsetAsync(M->m, 0, kNParams * 4, ctx->stream);
    cudaMemsetAsync(M->v, 0, kNParams * 4, ctx->stream);
    cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem());
    GBE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    *out = M;
    return GBE_OK;
}

extern "C" int gbe_mlp_param_count(const gbe_mlp* M) { return M ? kNParams : 0; }

extern "C" int gbe_mlp_set_params(gbe_ctx* ctx, gbe_mlp* M, const float* host_params) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && M && host_params, "NULL argument");
    GBE_CUDA_TRY(cudaMemcpyAsync(M->p, host_params, kNParams * 4, cudaMemcpyHostToDevice, ctx->stream));
    GBE_CUDA_TRY(cudaMemsetAsync(M->m, 0, kNParams * 4, ctx->stream));
    GBE_CUDA_TRY(cudaMemsetAsync(M->v, 0, kNParams * 4, ctx->stream));
    M->t = 0;
    GBE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return GBE_OK;
}

extern "C" int gbe_mlp_get_params(gbe_ctx* ctx, const gbe_mlp* M, float* host_params) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && M && host_params, "NULL argument");
    GBE_CUDA_TRY(cudaMemcpyAsync(host_params, M->p, kNParams * 4, cudaMemcpyDeviceToHost, ctx->stream));
    GBE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return GBE_OK;
}

static int mlp_forward_dev(gbe_ctx* ctx, const gbe_mlp* M, const gbe_pairs* P, float* logits) {
    round_params_kernel<<<8, 256, 0, ctx->stream>>>(M->p, M->pw);
    // 8 warps per CTA, 16 pairs per warp and iteration
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((P->npairs + 127) / 128, (int64_t)ctx->sm_count * 8));
    if (P->npairs) mlp_forward_tc_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(P->feat, P->npairs, M->pw, logits);
    GBE_CUDA_TRY(cudaGetLastError());
    return GBE_OK;
}

extern "C" int gbe_mlp_forward(gbe_ctx* ctx, const gbe_mlp* M, const gbe_pairs* P, float* logits) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && M && P && logits, "NULL argument");
    return mlp_forward_dev(ctx, M, P, logits);
}

static int mlp_grad_dev(gbe_ctx* ctx, gbe_mlp* M, const gbe_pairs* P, const uint8_t* labels) {
    GBE_CHECK_ARG(P->npairs > 0, "no pairs");
    round_params_kernel<<<8, 256, 0, ctx->stream>>>(M->p, M->pw);
    const int blocks = (int)std::min<int64_t>(M->nblocks, (P->npairs + kBatch - 1) / kBatch);
    mlp_grad_kernel<<<blocks, kBatch, grad_smem(), ctx->stream>>>(P->feat, labels, P->npairs, M->pw,
                                                                 (float)(1.0 / (double)P->npairs), M->partials,
                                                                 M->loss_part);
    reduce_grad_kernel<<<(kNParams + 255) / 256, 256, 0, ctx->stream>>>(M->partials, blocks, M->g, M->loss_part, M->loss,
                                                                         1.0 / (double)P->npairs);
    GBE_CUDA_TRY(cudaGetLastError());
    return GBE_OK;
}

extern "C" int gbe_mlp_gradient(gbe_ctx* ctx, gbe_mlp* M, const gbe_pairs* P, const uint8_t* labels, double* loss,
                                float* grad_host) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && M && P && labels, "NULL argument");
    GBE_TRY(gbe_check_device(ctx, labels, (size_t)P->npairs, "gbe_mlp_gradient labels"));
    GBE_TRY(mlp_grad_dev(ctx, M, P, labels));
    if (loss) GBE_CUDA_TRY(cudaMemcpyAsync(loss, M->loss, 8, cudaMemcpyDeviceToHost, ctx->stream));
    if (grad_host) GBE_CUDA_TRY(cudaMemcpyAsync(grad_host, M->g, kNParams * 4, cudaMemcpyDeviceToHost, ctx->stream));
    GBE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return GBE_OK;
}

extern "C" int gbe_mlp_adam_step(gbe_ctx* ctx, gbe_mlp* M, float lr, float beta1, float beta2, float eps) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && M, "NULL argument");
    M->t += 1;
    const float c1 = 1.0f - powf(beta1, (float)M->t), c2 = 1.0f - powf(beta2, (float)M->t);
    adam_kernel<<<(kNParams + 255) / 256, 256, 0, ctx->stream>>>(M->p, M->m, M->v, M->g, lr, beta1, beta2, eps, c1, c2);
    GBE_CUDA_TRY(cudaGetLastError());
    return GBE_OK;
}

extern "C" int gbe_mlp_train(gbe_ctx* ctx, gbe_mlp* M, const gbe_pairs* P, const uint8_t* labels, int epochs,
                             float lr, double* final_loss) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && M && P && labels && epochs > 0, "bad argument");
    GBE_TRY(gbe_check_device(ctx, labels, (size_t)P->npairs, "gbe_mlp_train labels"));
    for (int e = 0; e < epochs; ++e) {
        GBE_TRY(mlp_grad_dev(ctx, M, P, labels));
        GBE_TRY(gbe_mlp_adam_step(ctx, M, lr, 0.9f, 0.999f, 1e-8f));
    }
    if (final_loss) GBE_CUDA_TRY(cudaMemcpyAsync(final_loss, M->loss, 8, cudaMemcpyDeviceToHost, ctx->stream));
    GBE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return GBE_OK;
}

// Training labels from an assembled density matrix (the thresholded D patterns the network
// learns, Sec. II.A's floor(D)_tau): y_p = 1 when |D_ij| >= tau for pair p = (i, j), else 0
// (also when D has no entry (i, j)).  Row j of the ELL holds column j of D, so D_ij is the
// entry of row j whose column index is i.  One block per site i; each warp takes pairs of
// row i in turn, its lanes scanning row j 32 entries at a time up to the row's padding.
__global__ void pair_labels_kernel(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ pj,
                                   const int32_t* __restrict__ ecol, const double* __restrict__ eval, int64_t width,
                                   double tau, uint8_t* __restrict__ labels) {
    const int64_t i = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t p1 = rowptr[i + 1];
    for (int64_t p = rowptr[i] + warp; p < p1; p += blockDim.x >> 5) {
        const int64_t base = (int64_t)pj[p] * width;
        uint8_t y = 0;
        for (int64_t k0 = 0; k0 < width; k0 += 32) {
            const int64_t k = k0 + lane;
            const int32_t ck = k < width ? ecol[base + k] : -1;
            const unsigned hit = __ballot_sync(0xffffffffu, ck == (int32_t)i);
            if (hit) {
                const int src = __ffs(hit) - 1;
                const double v = __shfl_sync(0xffffffffu, lane == src ? eval[base + k] : 0.0, src);
                y = fabs(v) >= tau ? 1 : 0;
                break;
            }
            if (__ballot_sync(0xffffffffu, ck < 0)) break;   // padding: row j holds no more entries
        }
        if (lane == 0) labels[p] = y;
    }
}

extern "C" int gbe_mlp_labels(gbe_ctx* ctx, const gbe_pairs* P, const gbe_ell* D, double tau, uint8_t* labels) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && P && D && labels, "NULL argument");
    GBE_CHECK_ARG(D->on_device == 1 && D->col && D->val, "D must be a device ELL");
    GBE_CHECK_ARG(D->n == P->n && D->width >= 1, "D must have one row per site of the pairs");
    GBE_CHECK_ARG(tau >= 0.0, "tau must be >= 0");
    if (P->npairs == 0) return GBE_OK;
    GBE_TRY(gbe_check_device_ell(ctx, D, "gbe_mlp_labels D"));
    GBE_TRY(gbe_check_device(ctx, labels, (size_t)P->npairs, "gbe_mlp_labels labels"));
    pair_labels_kernel<<<(unsigned)P->n, 256, 0, ctx->stream>>>(P->rowptr, P->j, D->col, D->val, D->width, tau, labels);
    GBE_CUDA_TRY(cudaGetLastError());
    return GBE_OK;
}

// GBE_GRAPH_MLP: pairs within rcand scored by the network, kept when logit >= cut; the
// graph adds the pattern of H and the diagonal (union and symmetrisation in graph.cu).
int gbe_graph_mlp_select(gbe_ctx* ctx, const gbe_csr* H, const gbe_graph_params* p, int64_t** rp_out, int32_t** ci_out) {
    GBE_CHECK_ARG(p->sites && p->mlp && p->rcand > 0.0, "MLP graph needs sites, mlp and rcand");
    gbe_pairs* P = nullptr;
    GBE_TRY(gbe_pairs_build(ctx, p->sites, H, p->rcand, &P));
    const int64_t n = P->n;
    DevBuf logits, cnt;
    int r = gbe_alloc(&logits.p, std::max<int64_t>(P->npairs, 1) * 4);
    if (r == GBE_OK) r = gbe_alloc(&cnt.p, n * 4);
    if (r == GBE_OK) r = mlp_forward_dev(ctx, p->mlp, P, logits.as<float>());
    int64_t* rp = nullptr;
    int32_t* ci = nullptr;
    int64_t nsel = 0;
    if (r == GBE_OK) {
        select_count_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(P->rowptr, logits.as<float>(), n,
                                                                                 (float)p->logit_cut, cnt.as<int32_t>());
        r = gbe_alloc((void**)&rp, (n + 1) * 8);
    }
    if (r == GBE_OK) r = scan_exclusive(ctx, cnt.as<int32_t>(), rp, n, &nsel);
    if (r == GBE_OK) r = gbe_alloc((void**)&ci, std::max<int64_t>(nsel, 1) * 4);
    if (r == GBE_OK) {
        select_fill_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(P->rowptr, P->j, logits.as<float>(), n,
                                                                                (float)p->logit_cut, rp, ci);
        const cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) { gbe_set_error("mlp select: %s", cudaGetErrorString(e)); r = GBE_ECUDA; }
    }
    gbe_free_pairs(P);
    if (r != GBE_OK) { gbe_free(rp); gbe_free(ci); return r; }
    *rp_out = rp;
    *ci_out = ci;
    return GBE_OK;
}
