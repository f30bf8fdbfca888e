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
__global__ void __launch_bounds__(256) pairs_kernel(const double* __restrict__ pos, const float4* __restrict__ pos4,
                                                    const double* __restrict__ onsite, int64_t n, CellGrid g, float lim2,
                                                    const int64_t* __restrict__ cstart,
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
    for (int dx = lo[0]; dx <= hi[0]; ++dx)
        for (int dy = lo[1]; dy <= hi[1]; ++dy)
            for (int dz = lo[2]; dz <= hi[2]; ++dz) {
                const int ax = (cc[0] + dx + g.nc[0]) % g.nc[0];
                const int ay = (cc[1] + dy + g.nc[1]) % g.nc[1];
                const int az = (cc[2] + dz + g.nc[2]) % g.nc[2];
                const int cell = (ax * g.nc[1] + ay) * g.nc[2] + az;
                for (int64_t p = cstart[cell] + lane; p < cstart[cell + 1]; p += 32) {
                    const int j = members[p];
                    if (j == i) continue;
                    // FP32 pre-filter, then r < rcand in FP64 (up to an ulp at the cutoff)
                    if (near_f32(pi, pos4[j], bx, by, bz, ix, iy, iz, lim2) && pair_dist2(pos, xi, yi, zi, j, g) < rcand2) {
                        const int k = atomicAdd(&bcount[w], 1);
                        if (k < kPairCap) buf[w][k] = j;
                    }
                }
            }
    __syncwarp();
    const int m = bcount[w];
    if (m > kPairCap) {
        if (lane == 0) atomicExch(overflow, 1);
        return;
    }
    if (pass == 0) {
        if (lane == 0) cnt[i] = m;
        return;
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
    const int64_t base = rowptr[i];
    const double ei = onsite[i];
    for (int t = lane; t < m; t += 32) {
        const int j = buf[w][t];
        const double r = sqrt(pair_dist2(pos, xi, yi, zi, j, g));
        // H_ij by binary search in row i, (H^2)_ij by the ordered merge dot product
        double hij = 0.0;
        int64_t a = hrp[i], b = hrp[i + 1] - 1;
        while (a <= b) {
            const int64_t mid = (a + b) >> 1;
            const int v = hci[mid];
            if (v == j) { hij = hva[mid]; break; }
            if (v < j) a = mid + 1; else b = mid - 1;
        }
        const double ej = onsite[j];
        float* f = feat + (base + t) * kNF;
        f[0] = -log10f(fmaxf((float)fabs(hij), 1e-12f)) / 12.0f;
        // f[1], the (H^2)_ij feature, is written by h2_feature_kernel
        f[2] = (float)(r / rcand);
        f[3] = (float)fmin(ei, ej);
        f[4] = (float)fmax(ei, ej);
        pj[base + t] = j;
    }
}

// Row i of H^2 for every site i, then the (H^2)_ij feature of its candidate pairs.  One warp
// per site accumulates (H^2)_il = sum_k H_ik H_kl in a shared-memory hash table keyed by l,
// taking k in ascending order (one row k at a time, its entries across the lanes): every
// (H^2)_ij is then the same sequence of products and additions as the ordered merge of rows
// i and j (H is symmetric to the last bit), so the feature is symmetric in (i, j) bit for
// bit.  A row of H^2 with more entries than the table holds is computed by that merge.
constexpr int kH2Slots = 1024;   // hash slots per warp (a row of H^2 within 5a has ~520 entries)
constexpr int kH2Warps = 4;
constexpr size_t kH2Smem = (size_t)kH2Warps * kH2Slots * (4 + 8);

__device__ __forceinline__ unsigned h2_hash(int l) { return ((unsigned)l * 2654435761u) >> 22; }   // 10 bits

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
    bool ok = true;
    for (int64_t p = hrp[i]; p < hrp[i + 1]; ++p) {
        const int k = hci[p];
        const double hik = hva[p];
        for (int64_t q = hrp[k] + lane; q < hrp[k + 1]; q += 32) {
            const int l = hci[q];
            unsigned h = h2_hash(l);
            int probes = 0;
            while (true) {
                const int old = atomicCAS(&keys[h], -1, l);
                if (old == -1 || old == l) break;
                if (++probes == kH2Slots) break;
                h = (h + 1) & (kH2Slots - 1);
            }
            if (probes < kH2Slots) vals[h] = __dadd_rn(vals[h], __dmul_rn(hik, hva[q]));   // one lane per key
            else ok = false;
        }
        __syncwarp();
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
__global__ void round_params_kernel(const float* __restrict__ p, float* pw) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNParams; i += gridDim.x * blockDim.x)
        pw[i] = __half2float(__float2half_rn(p[i]));
}

__global__ void __launch_bounds__(256) mlp_forward_kernel(const float* __restrict__ feat, int64_t npairs,
                                                          const float* __restrict__ pw, float* logits) {
    __shared__ __align__(16) float W[kNParams];
    for (int i = threadIdx.x; i < kNParams; i += blockDim.x) W[i] = pw[i];
    __syncthreads();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < npairs; t += (int64_t)gridDim.x * blockDim.x) {
        // base pointer the compiler cannot treat as loop-invariant (t < 2^40), so that the
        // weight loads stay in the loop instead of being hoisted into hundreds of registers
        const float* Wt = W + (int)(t >> 40);
        float f[kNF], h1[kHid];
#pragma unroll
        for (int q = 0; q < kNF; ++q) f[q] = feat[t * kNF + q];
#pragma unroll
        for (int k = 0; k < kHid; ++k) {  // h1 stays in registers (64)
            float a = Wt[OB1 + k];
#pragma unroll
            for (int q = 0; q < kNF; ++q) a = fmaf(Wt[OW1 + k * kNF + q], f[q], a);
            h1[k] = fmaxf(a, 0.0f);
        }
        float z = Wt[OB3];
#pragma unroll 1
        for (int o = 0; o < kHid; ++o) {
            const float4* w4 = reinterpret_cast<const float4*>(Wt + OW2 + o * kHid);
            float a0 = Wt[OB2 + o], a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
            for (int k4 = 0; k4 < kHid / 4; ++k4) {
                const float4 wv = w4[k4];
                a0 = fmaf(wv.x, h1[4 * k4], a0);
                a1 = fmaf(wv.y, h1[4 * k4 + 1], a1);
                a2 = fmaf(wv.z, h1[4 * k4 + 2], a2);
                a3 = fmaf(wv.w, h1[4 * k4 + 3], a3);
            }
            z = fmaf(Wt[OW3 + o], fmaxf((a0 + a1) + (a2 + a3), 0.0f), z);
        }
        logits[t] = z;
    }
}

struct GradSmem {
    float W[kNParams];
    float G[kNParams];
    float H1[kBatch][kLd];
    float H2[kBatch][kLd];      // activations h2, then dL/dh2
    float D1[kBatch][kLd];      // dL/dh1
    float F[kBatch][8];
    float dz[kBatch];
};

// Forward + BCE + backward over batches of 128 pairs; each CTA accumulates the gradient of
// the mean loss in shared memory (every entry owned by one thread, no atomics) and writes
// it to its partial slot; loss terms likewise.
__global__ void __launch_bounds__(kBatch) mlp_grad_kernel(const float* __restrict__ feat,
                                                          const uint8_t* __restrict__ labels, int64_t npairs,
                                                          const float* __restrict__ pw, float inv_n, float* partials,
                                                          double* loss_part) {
    extern __shared__ unsigned char gsm_raw[];
    GradSmem& S = *reinterpret_cast<GradSmem*>(gsm_raw);
    const int t = threadIdx.x;
    for (int i = t; i < kNParams; i += kBatch) { S.W[i] = pw[i]; S.G[i] = 0.0f; }
    double lsum = 0.0;
    __syncthreads();
    for (int64_t b0 = (int64_t)blockIdx.x * kBatch; b0 < npairs; b0 += (int64_t)gridDim.x * kBatch) {
        const int64_t pidx = b0 + t;
        const bool valid = pidx < npairs;
        float f[kNF], h1[kHid];
#pragma unroll
        for (int q = 0; q < kNF; ++q) f[q] = valid ? feat[pidx * kNF + q] : 0.0f;
        const float y = valid ? (float)labels[pidx] : 0.0f;
        // forward, keeping h1 and h2 for the backward pass
#pragma unroll
        for (int k = 0; k < kHid; ++k) {
            float a = S.W[OB1 + k];
#pragma unroll
            for (int q = 0; q < kNF; ++q) a = fmaf(S.W[OW1 + k * kNF + q], f[q], a);
            h1[k] = fmaxf(a, 0.0f);
            S.H1[t][k] = h1[k];
        }
        float z = S.W[OB3];
        for (int o = 0; o < kHid; ++o) {
            float a = S.W[OB2 + o];
#pragma unroll
            for (int k = 0; k < kHid; ++k) a = fmaf(S.W[OW2 + o * kHid + k], h1[k], a);
            const float h2 = fmaxf(a, 0.0f);
            S.H2[t][o] = h2;
            z = fmaf(S.W[OW3 + o], h2, z);
        }
        const float sig = 1.0f / (1.0f + __expf(-z));
        const float dz = valid ? (sig - y) * inv_n : 0.0f;
        if (valid) lsum += (double)(fmaxf(z, 0.0f) - y * z + log1pf(__expf(-fabsf(z))));
#pragma unroll
        for (int q = 0; q < kNF; ++q) S.F[t][q] = f[q];
        S.dz[t] = dz;
        __syncthreads();
        // gradients of the output layer (thread o < 64 owns w3[o]; thread 64 owns b3)
        if (t < kHid) {
            float acc = 0.0f;
            for (int b = 0; b < kBatch; ++b) acc = fmaf(S.dz[b], S.H2[b][t], acc);
            S.G[OW3 + t] += acc;
        } else if (t == kHid) {
            float acc = 0.0f;
            for (int b = 0; b < kBatch; ++b) acc += S.dz[b];
            S.G[OB3] += acc;
        }
        __syncthreads();
        // backward through layer 2 for this thread's pair: dh2 (overwrites h2), dh1
        {
            float d1[kHid];
#pragma unroll
            for (int k = 0; k < kHid; ++k) d1[k] = 0.0f;
            for (int o = 0; o < kHid; ++o) {
                const float d2 = S.H2[t][o] > 0.0f ? dz * S.W[OW3 + o] : 0.0f;
                S.H2[t][o] = d2;
#pragma unroll
                for (int k = 0; k < kHid; ++k) d1[k] = fmaf(d2, S.W[OW2 + o * kHid + k], d1[k]);
            }
#pragma unroll
            for (int k = 0; k < kHid; ++k) S.D1[t][k] = S.H1[t][k] > 0.0f ? d1[k] : 0.0f;
        }
        __syncthreads();
        // weight gradients: thread owns a 4 (out) x 8 (in) block of W2, plus b2 for its
        // 4 outputs when it holds the first input block
        {
            const int o0 = (t >> 3) * 4, k0 = (t & 7) * 8;
            float acc[4][8];
            float accb[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[a][c] = 0.0f;
            for (int b = 0; b < kBatch; ++b) {
                float d[4], h[8];
#pragma unroll
                for (int a = 0; a < 4; ++a) d[a] = S.H2[b][o0 + a];
#pragma unroll
                for (int c = 0; c < 8; ++c) h[c] = S.H1[b][k0 + c];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    accb[a] += d[a];
#pragma unroll
                    for (int c = 0; c < 8; ++c) acc[a][c] = fmaf(d[a], h[c], acc[a][c]);
                }
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
#pragma unroll
                for (int c = 0; c < 8; ++c) S.G[OW2 + (o0 + a) * kHid + k0 + c] += acc[a][c];
                if (k0 == 0) S.G[OB2 + o0 + a] += accb[a];
            }
        }
        // layer-1 gradients: 64 x (5 + 1) entries, threads 0..63 own one hidden unit each
        if (t < kHid) {
            float gw[kNF] = {0.f, 0.f, 0.f, 0.f, 0.f};
            float gb = 0.0f;
            for (int b = 0; b < kBatch; ++b) {
                const float d = S.D1[b][t];
                gb += d;
#pragma unroll
                for (int q = 0; q < kNF; ++q) gw[q] = fmaf(d, S.F[b][q], gw[q]);
            }
#pragma unroll
            for (int q = 0; q < kNF; ++q) S.G[OW1 + t * kNF + q] += gw[q];
            S.G[OB1 + t] += gb;
        }
        __syncthreads();
    }
    for (int i = t; i < kNParams; i += kBatch) partials[(int64_t)blockIdx.x * kNParams + i] = S.G[i];
    // fixed-order loss reduction within the CTA
    __shared__ double lred[kBatch];
    lred[t] = lsum;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int b = 0; b < kBatch; ++b) s += lred[b];
        loss_part[blockIdx.x] = s;
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
    GBE_TRY(gbe_alloc(&flag.p, 4));
    cudaMemsetAsync(ccnt.p, 0, ncells * 4, s);
    cudaMemsetAsync(cur.p, 0, ncells * 4, s);
    cudaMemsetAsync(flag.p, 0, 4, s);
    const unsigned nb = (unsigned)((n + 255) / 256);
    cell_count_kernel<<<nb, 256, 0, s>>>(pos, n, g, cell.as<int32_t>(), ccnt.as<int32_t>());
    GBE_TRY(scan_exclusive(ctx, ccnt.as<int32_t>(), cst.as<int64_t>(), ncells, nullptr));
    cell_fill_kernel<<<nb, 256, 0, s>>>(cell.as<int32_t>(), n, cst.as<int64_t>(), cur.as<int32_t>(), mem.as<int32_t>());
    const unsigned rb = (unsigned)((n + 7) / 8);
    DevBuf p4;
    GBE_TRY(gbe_alloc(&p4.p, n * 16));
    pos_f32_kernel<<<nb, 256, 0, s>>>(pos, n, p4.as<float4>());
    const float lim2 = filter_lim2(rcand, st->box);
    pairs_kernel<<<rb, 256, 0, s>>>(pos, p4.as<float4>(), ons, n, g, lim2, cst.as<int64_t>(), mem.as<int32_t>(), rcand, 0,
                                    cnt.as<int32_t>(),
                                    nullptr, nullptr, nullptr, rp, ci, va, flag.as<int>());
    GBE_CUDA_TRY(cudaGetLastError());
    gbe_pairs* P = new gbe_pairs();
    P->n = n;
    int r = gbe_alloc((void**)&P->rowptr, (n + 1) * 8);
    int64_t np = 0;
    if (r == GBE_OK) r = scan_exclusive(ctx, cnt.as<int32_t>(), P->rowptr, n, &np);
    int ovf = 0;
    if (r == GBE_OK) r = read_flag(ctx, flag.as<int>(), &ovf);
    if (r == GBE_OK && ovf) { gbe_set_error("a site has more than %d candidates within rcand", kPairCap); r = GBE_ECAPACITY; }
    if (r == GBE_OK) r = gbe_alloc((void**)&P->j, std::max<int64_t>(np, 1) * 4);
    if (r == GBE_OK) r = gbe_alloc((void**)&P->feat, std::max<int64_t>(np, 1) * kNF * 4);
    if (r != GBE_OK) { gbe_free_pairs(P); return r; }
    P->npairs = np;
    pairs_kernel<<<rb, 256, 0, s>>>(pos, p4.as<float4>(), ons, n, g, lim2, cst.as<int64_t>(), mem.as<int32_t>(), rcand, 1,
                                    cnt.as<int32_t>(),
                                    P->rowptr, P->j, P->feat, rp, ci, va, flag.as<int>());
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
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((P->npairs + 255) / 256, (int64_t)ctx->sm_count * 8));
    if (P->npairs) mlp_forward_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(P->feat, P->npairs, M->pw, logits);
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
    for (int e = 0; e < epochs; ++e) {
        GBE_TRY(mlp_grad_dev(ctx, M, P, labels));
        GBE_TRY(gbe_mlp_adam_step(ctx, M, lr, 0.9f, 0.999f, 1e-8f));
    }
    if (final_loss) GBE_CUDA_TRY(cudaMemcpyAsync(final_loss, M->loss, 8, cudaMemcpyDeviceToHost, ctx->stream));
    GBE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
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
