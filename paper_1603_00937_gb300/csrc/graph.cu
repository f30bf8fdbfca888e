// Hamiltonian build (cell list), data-dependency graphs and core+halo partitions.
//
//  * gbe_build_hamiltonian: H_ij = hop exp(-(r - a)/decay) for 0 < r < rcut, minimum
//    image, H_ii = onsite; sites binned into cells of edge >= rcut, one warp per row.
//  * gbe_build_graph (Eq. 2, Eq. 8): a graph is a base pattern A (undirected, diagonal
//    present) and a path length k, S = pattern(A^k).  Row sets are built per row with a
//    shared-memory hash set, sorted, and written as CSR by a count / scan / fill pattern.
//    |(H^2)_ij| is a merge dot product of two sorted rows in ascending k (deterministic).
//  * gbe_partition (Sec. II.A, Fig. 1, observation vi): cores are non-empty spatial cells
//    (ascending cell id) or index blocks; each core set is expanded by k hops over A in a
//    shared-memory hash set, sorted, and emitted as core vertices then halo vertices.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "gbe_internal.h"
#include "devutil.cuh"

using namespace gbe_dev;

namespace {

constexpr int kHashCap = 8192;   // hash-set capacity of one row / core set (ints)
constexpr int kSetMax = 4096;    // largest set a CTA sorts and emits

// ------------------------------------------------------------------ shared-memory hash set
__device__ __forceinline__ unsigned hslot(int v) { return ((unsigned)v * 2654435761u) >> (32 - 13); }  // 8192 slots

// Insert v; returns false when the table is full.
__device__ __forceinline__ bool hset_insert(int* table, int* count, int v) {
    unsigned h = hslot(v);
    for (int probe = 0; probe < kHashCap; ++probe) {
        const int cur = table[h];
        if (cur == v) return true;
        if (cur == -1) {
            const int old = atomicCAS(&table[h], -1, v);
            if (old == -1) {
                atomicAdd(count, 1);
                return true;
            }
            if (old == v) return true;
        }
        h = (h + 1) & (kHashCap - 1);
    }
    return false;
}

// Ascending bitonic sort of n <= cap ints in shared memory (cap a power of two).
__device__ void bitonic_sort(int* a, int n, int cap) {
    for (int i = n + threadIdx.x; i < cap; i += blockDim.x) a[i] = INT32_MAX;
    __syncthreads();
    int size = 1;
    while (size < n) size <<= 1;
    for (int k = 2; k <= size; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < size; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = ((i & k) == 0);
                    const int x = a[i], y = a[l];
                    if ((x > y) == up) { a[i] = y; a[l] = x; }
                }
            }
            __syncthreads();
        }
    }
}

// Move the hash-set contents into list[0..count) (unordered).
__device__ int hset_compact(const int* table, int* list, int* cursor) {
    if (threadIdx.x == 0) *cursor = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < kHashCap; i += blockDim.x) {
        const int v = table[i];
        if (v != -1) list[atomicAdd(cursor, 1)] = v;
    }
    __syncthreads();
    return *cursor;
}

__device__ void hset_clear(int* table, int* count, int* flag) {
    for (int i = threadIdx.x; i < kHashCap; i += blockDim.x) table[i] = -1;
    if (threadIdx.x == 0) { *count = 0; *flag = 0; }
    __syncthreads();
}

// Expand the set in the table by `hops` steps over CSR A.  Returns false on overflow.
__device__ bool hset_expand(int* table, int* count, int* list, int* cursor, int* flag, const int64_t* __restrict__ rp,
                            const int32_t* __restrict__ ci, int hops) {
    if (threadIdx.x == 0) *flag = 0;
    for (int h = 0; h < hops; ++h) {
        const int n = hset_compact(table, list, cursor);
        if (n > kSetMax) { if (threadIdx.x == 0) *flag = 1; __syncthreads(); return false; }
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int t = warp; t < n; t += nw) {
            const int v = list[t];
            for (int64_t p = rp[v] + lane; p < rp[v + 1]; p += 32)
                if (!hset_insert(table, count, ci[p])) *flag = 1;
        }
        __syncthreads();
        if (*flag || *count > kSetMax) { if (threadIdx.x == 0) *flag = 1; __syncthreads(); return false; }
    }
    return true;
}

// ------------------------------------------------------------------ Hamiltonian
// Sort the members of each cell ascending (cells are small; one warp per cell).
__global__ void cell_sort_kernel(const int64_t* __restrict__ start, int ncells, int32_t* members) {
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= ncells) return;
    int32_t* a = members + start[wid];
    const int n = (int)(start[wid + 1] - start[wid]);
    // odd-even transposition sort, warp-cooperative
    for (int phase = 0; phase < n; ++phase) {
        for (int i = 2 * lane + (phase & 1); i + 1 < n; i += 64) {
            const int x = a[i], y = a[i + 1];
            if (x > y) { a[i] = y; a[i + 1] = x; }
        }
        __syncwarp();
    }
}

struct HModel {
    double a, rcut, inv_decay, hop, rcut2;
};

constexpr int kRowCap = 1024;
constexpr int kStageCap = 128;   // staging slot per row of the single-pass H build

// Staged rows (kStageCap apart) -> CSR.
__global__ void compact_rows_kernel(const int32_t* __restrict__ scol, const double* __restrict__ sval, int64_t n,
                                    const int64_t* __restrict__ rowptr, int32_t* col, double* val) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = t / kStageCap;
    const int k = (int)(t % kStageCap);
    if (i >= n) return;
    const int64_t b = rowptr[i];
    if (k < rowptr[i + 1] - b) {
        col[b + k] = scol[i * kStageCap + k];
        val[b + k] = sval[i * kStageCap + k];
    }
}

// One warp per row.  pass 0: count neighbours; pass 1: write sorted (col, val).
__global__ void __launch_bounds__(256) hbuild_kernel(const double* __restrict__ pos, const float4* __restrict__ pos4,
                                                     const double* __restrict__ onsite, int64_t n, CellGrid g,
                                                     float lim2, float lim2_in, const int64_t* __restrict__ cstart,
                                                     const int32_t* __restrict__ members, HModel mdl, int pass,
                                                     int32_t* cnt, const int64_t* __restrict__ rowptr, int32_t* col,
                                                     double* val, int* overflow) {
    __shared__ int buf[8][kRowCap];
    __shared__ int bcount[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * 8 + w;
    if (i >= n) return;
    const double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
    const float4 pi = pos4[i];
    const float bx = (float)g.box[0], by = (float)g.box[1], bz = (float)g.box[2];
    const float ix = (float)g.inv[0], iy = (float)g.inv[1], iz = (float)g.inv[2];
    const int ci = cell_of(pos + 3 * i, g);
    int cc[3] = {ci / (g.nc[1] * g.nc[2]), (ci / g.nc[2]) % g.nc[1], ci % g.nc[2]};
    if (lane == 0) bcount[w] = 0;
    __syncwarp();
    // neighbour cells: offsets -1..1, or every cell along an axis with fewer than 3 cells
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        if (g.nc[d] >= 3) { lo[d] = -1; hi[d] = 1; }
        else { lo[d] = -cc[d]; hi[d] = g.nc[d] - 1 - cc[d]; }
    }
    // The (at most 27) neighbour cells' member ranges, one per lane, and their exclusive prefix
    // sums: the candidates of all cells are then one flat range across the lanes, whose loads
    // do not wait on one another (the row is sorted afterwards, so the order found is free).
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
            // FP32 separation first: below the inner bound the pair is inside, above the outer one
            // outside; between them r^2 < rcut^2 decides in FP64 (which differs from r < rcut
            // only within an ulp of the cutoff)
            const float r2f = j == i ? 0.0f : dist2_f32(pi, pos4[j], bx, by, bz, ix, iy, iz);
            if (j == i || r2f < lim2_in || (r2f < lim2 && pair_dist2(pos, xi, yi, zi, j, g) < mdl.rcut2)) {
                const int k = atomicAdd(&bcount[w], 1);
                if (k < kRowCap) buf[w][k] = j;
            }
        }
    }
    __syncwarp();
    const int m = bcount[w];
    if (m > kRowCap) {
        if (lane == 0) atomicExch(overflow, 1);
        return;
    }
    if (pass == 0) {
        if (lane == 0) cnt[i] = m;
        return;
    }
    if (pass == 2) {
        // single-pass build: the sorted row goes to a staging slot of kStageCap entries (a
        // longer row sets the staging flag, overflow[1], and the host runs the fill pass instead)
        if (lane == 0) cnt[i] = m;
        if (m > kStageCap) {
            if (lane == 0) atomicExch(overflow + 1, 1);
            return;
        }
    }
    // sort the row's columns: bitonic within the warp, padded to a power of two with INT_MAX
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
    const int64_t base = pass == 2 ? i * kStageCap : rowptr[i];
    for (int t = lane; t < m; t += 32) {
        const int j = buf[w][t];
        double v;
        if (j == i) {
            v = onsite[i];
        } else {
            const double r = sqrt(pair_dist2(pos, xi, yi, zi, j, g));
            v = mdl.hop * exp(-(r - mdl.a) * mdl.inv_decay);
        }
        col[base + t] = j;
        val[base + t] = v;
    }
}

// ------------------------------------------------------------------ graph row sets
struct RowSetSmem {
    int table[kHashCap];
    int list[kHashCap];
    int count, cursor, flag;
};

// mode 0: |(H^2)_ij| >= thresh (numeric), hops over H = 1 then filter
// mode 1: union of sources given as CSR lists (A1 row i, A2 row i, A3 row i) + diagonal
// mode 2: pattern of A^hops (materialisation)
__global__ void __launch_bounds__(256) rowset_kernel(int mode, int64_t n, const int64_t* __restrict__ hrp,
                                                     const int32_t* __restrict__ hci, const double* __restrict__ hva,
                                                     double thresh, const int64_t* __restrict__ s1rp,
                                                     const int32_t* __restrict__ s1ci, const int64_t* __restrict__ s2rp,
                                                     const int32_t* __restrict__ s2ci, const int64_t* __restrict__ s3rp,
                                                     const int32_t* __restrict__ s3ci, int hops, int pass, int32_t* cnt,
                                                     const int64_t* __restrict__ outrp, int32_t* outci, int* overflow,
                                                     int stage_cap) {
    extern __shared__ unsigned char smraw[];
    RowSetSmem& S = *reinterpret_cast<RowSetSmem*>(smraw);
    for (int64_t row = blockIdx.x; row < n; row += gridDim.x) {
        const int i = (int)row;
        hset_clear(S.table, &S.count, &S.flag);
        if (threadIdx.x == 0) hset_insert(S.table, &S.count, i);
        __syncthreads();
        bool ok = true;
        if (mode == 0) {
            // candidates: union of H rows of H's neighbours of i
            for (int64_t p = hrp[i]; p < hrp[i + 1]; ++p) {
                const int k = hci[p];
                for (int64_t q = hrp[k] + threadIdx.x; q < hrp[k + 1]; q += blockDim.x)
                    if (!hset_insert(S.table, &S.count, hci[q])) S.flag = 1;
            }
            __syncthreads();
        } else if (mode == 1) {
            const int64_t* rps[3] = {s1rp, s2rp, s3rp};
            const int32_t* cis[3] = {s1ci, s2ci, s3ci};
            for (int s = 0; s < 3; ++s) {
                if (!rps[s]) continue;
                for (int64_t q = rps[s][i] + threadIdx.x; q < rps[s][i + 1]; q += blockDim.x)
                    hset_insert(S.table, &S.count, cis[s][q]);
            }
            __syncthreads();
        } else {
            ok = hset_expand(S.table, &S.count, S.list, &S.cursor, &S.flag, s1rp, s1ci, hops);
        }
        if (!ok || S.flag || S.count > kSetMax) {
            if (threadIdx.x == 0) atomicExch(overflow, 1);
            __syncthreads();
            continue;
        }
        int m = hset_compact(S.table, S.list, &S.cursor);
        bitonic_sort(S.list, m, kHashCap);
        if (mode == 0) {
            // keep |(H^2)_ij| >= thresh or j == i; compact in order
            if (threadIdx.x == 0) S.cursor = 0;
            __syncthreads();
            for (int t0 = 0; t0 < m; t0 += blockDim.x) {
                const int t = t0 + threadIdx.x;
                int keep = 0, j = 0;
                if (t < m) {
                    j = S.list[t];
                    keep = (j == i) || (fabs(row_dot(hrp, hci, hva, i, j)) >= thresh);
                }
                // ordered compaction within the block
                __shared__ int wsum[8];
                const unsigned bal = __ballot_sync(0xffffffffu, keep);
                const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
                if (lane == 0) wsum[w] = __popc(bal);
                __syncthreads();
                int before = 0;
                for (int q = 0; q < w; ++q) before += wsum[q];
                const int base = S.cursor;
                __syncthreads();
                if (keep) S.table[base + before + __popc(bal & ((1u << lane) - 1u))] = j;
                __syncthreads();
                if (threadIdx.x == 0) {
                    int tot = 0;
                    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += wsum[q];
                    S.cursor = base + tot;
                }
                __syncthreads();
            }
            m = S.cursor;
            for (int t = threadIdx.x; t < m; t += blockDim.x) S.list[t] = S.table[t];
            __syncthreads();
        }
        if (pass == 0) {
            if (threadIdx.x == 0) cnt[i] = m;
        } else if (pass == 2) {
            // single-pass build: the sorted row goes to a staging slot of stage_cap entries (a
            // longer row sets overflow[1], and the host runs the fill pass instead)
            if (threadIdx.x == 0) {
                cnt[i] = m;
                if (m > stage_cap) atomicExch(overflow + 1, 1);
            }
            if (m <= stage_cap) {
                const int64_t base = (int64_t)i * stage_cap;
                for (int t = threadIdx.x; t < m; t += blockDim.x) outci[base + t] = S.list[t];
            }
        } else {
            const int64_t base = outrp[i];
            for (int t = threadIdx.x; t < m; t += blockDim.x) outci[base + t] = S.list[t];
        }
        __syncthreads();
    }
}

// A warp per row, for rowset_kernel's modes 0 and 1 on rows that fit a warp's table.
// MODE 0, rows of |(H^2)_ij| >= thresh by accumulation instead of one merge per candidate:
// the warp sums (H^2)_il = sum_k H_ik H_kl into a shared-memory hash table keyed by l, taking k
// in ascending order (one row k at a time, its entries across the lanes: a row's columns are
// distinct, so each slot has one writer per k).  That is the same sequence of products and
// additions as row_dot's ordered merge of rows i and l, so the kept set is the same.
// MODE 1, the union of row i of up to three CSR lists and i itself.
// The kept columns (i itself always) are compacted in slot order, sorted in the warp, and
// written as rowset_kernel's passes 1 and 2 write them.  A row with more distinct columns than
// the table holds sets overflow[2] (the host then builds the graph with rowset_kernel).
constexpr int kH2RowSlots = 1024;
constexpr int kH2RowWarps = 4;
constexpr size_t kH2RowSmem = (size_t)kH2RowWarps * kH2RowSlots * (4 + 8);

__device__ __forceinline__ unsigned h2row_hash(int l) { return ((unsigned)l * 2654435761u) >> 22; }   // 10 bits

// Insert l into a warp's hash table; the slot, or -1 when the table is full.
__device__ __forceinline__ int h2row_insert(int* keys, int l) {
    unsigned h = h2row_hash(l);
    for (int probes = 0; probes < kH2RowSlots; ++probes) {
        const int old = atomicCAS(&keys[h], -1, l);
        if (old == -1 || old == l) return (int)h;
        h = (h + 1) & (kH2RowSlots - 1);
    }
    return -1;
}

template <int MODE>
__global__ void __launch_bounds__(32 * kH2RowWarps) warp_rowset_kernel(int64_t n, const int64_t* __restrict__ hrp,
                                                                       const int32_t* __restrict__ hci,
                                                                       const double* __restrict__ hva, double thresh,
                                                                       const int64_t* __restrict__ s1rp,
                                                                       const int32_t* __restrict__ s1ci,
                                                                       const int64_t* __restrict__ s2rp,
                                                                       const int32_t* __restrict__ s2ci,
                                                                       const int64_t* __restrict__ s3rp,
                                                                       const int32_t* __restrict__ s3ci, int pass,
                                                                       int32_t* cnt, const int64_t* __restrict__ outrp,
                                                                       int32_t* outci, int* overflow, int stage_cap) {
    extern __shared__ unsigned char h2rsm[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t row = (int64_t)blockIdx.x * kH2RowWarps + w;
    if (row >= n) return;   // whole warps only: nothing below synchronises the block
    const int i = (int)row;
    int* keys = reinterpret_cast<int*>(h2rsm) + w * kH2RowSlots;
    double* vals = reinterpret_cast<double*>(h2rsm + (size_t)kH2RowWarps * kH2RowSlots * 4) + w * kH2RowSlots;
    for (int t = lane; t < kH2RowSlots; t += 32) {
        keys[t] = -1;
        vals[t] = 0.0;
    }
    __syncwarp();
    bool ok = true;
    if constexpr (MODE == 0) {
        // row i's entries 32 at a time, each lane holding one k with its H_ik and the range of
        // row k (loaded together), then taken in ascending order across the warp
        const int64_t p0 = hrp[i], p1 = hrp[i + 1];
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
                    const int h = h2row_insert(keys, hci[q]);
                    if (h >= 0) vals[h] = __dadd_rn(vals[h], __dmul_rn(hik, hva[q]));
                    else ok = false;
                }
                __syncwarp();
            }
        }
    } else {
        if (lane == 0 && h2row_insert(keys, i) < 0) ok = false;
        const int64_t* rps[3] = {s1rp, s2rp, s3rp};
        const int32_t* cis[3] = {s1ci, s2ci, s3ci};
#pragma unroll
        for (int src = 0; src < 3; ++src) {
            if (!rps[src]) continue;
            for (int64_t q = rps[src][i] + lane; q < rps[src][i + 1]; q += 32)
                if (h2row_insert(keys, cis[src][q]) < 0) ok = false;
        }
        __syncwarp();
    }
    if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) atomicExch(overflow + 2, 1);
        return;
    }
    // kept columns to keys[0..m) in slot order (a chunk's slots are read before any is written)
    int m = 0;
    for (int t0 = 0; t0 < kH2RowSlots; t0 += 32) {
        const int key = keys[t0 + lane];
        const bool keep = key >= 0 && (MODE == 1 || key == i || fabs(vals[t0 + lane]) >= thresh);
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        __syncwarp();
        if (keep) keys[m + __popc(bal & ((1u << lane) - 1u))] = key;
        m += __popc(bal);
        __syncwarp();
    }
    // bitonic sort of keys[0..m) within the warp (padded to a power of two)
    int size = 1;
    while (size < m) size <<= 1;
    for (int t = m + lane; t < size; t += 32) keys[t] = INT32_MAX;
    __syncwarp();
    for (int kk = 2; kk <= size; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int t = lane; t < size; t += 32) {
                const int l = t ^ j;
                if (l > t) {
                    const bool up = ((t & kk) == 0);
                    const int x = keys[t], y = keys[l];
                    if ((x > y) == up) { keys[t] = y; keys[l] = x; }
                }
            }
            __syncwarp();
        }
    }
    if (pass == 0) {
        if (lane == 0) cnt[i] = m;
    } else if (pass == 2) {
        if (lane == 0) {
            cnt[i] = m;
            if (m > stage_cap) atomicExch(overflow + 1, 1);
        }
        if (m <= stage_cap) {
            const int64_t base = (int64_t)i * stage_cap;
            for (int t = lane; t < m; t += 32) outci[base + t] = keys[t];
        }
    } else {
        const int64_t base = outrp[i];
        for (int t = lane; t < m; t += 32) outci[base + t] = keys[t];
    }
}

// Staged rows (stage_cap apart) -> CSR column indices, one warp per row.
__global__ void compact_set_rows_kernel(const int32_t* __restrict__ stage, int64_t n, int stage_cap,
                                        const int64_t* __restrict__ rp, int32_t* ci) {
    const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (i >= n) return;
    const int64_t b = rp[i], m = rp[i + 1] - b;
    for (int64_t t = threadIdx.x & 31; t < m; t += 32) ci[b + t] = stage[i * stage_cap + t];
}

// ELL D -> pattern of kept entries (|D_ki| >= tau) as CSR by ELL row (row i lists k),
// and the transposed lists (row k lists i).  A warp per ELL row, 32 consecutive entries at
// a time (coalesced); an entry is kept when it lies before the row's first padding entry
// (col < 0) and |val| >= tau.  The order within a list is free (the union that consumes
// the lists sorts every row).
constexpr int kEllWarps = 8;

// The kept entries of ELL row i's chunk t0..t0+31: the lane's column (or -1) and whether the
// row ends in this chunk.
__device__ __forceinline__ int ell_kept(const int32_t* __restrict__ col, const double* __restrict__ val, int64_t i,
                                        int64_t W, int64_t t0, double tau, int lane, bool& last) {
    const int64_t t = t0 + lane;
    const int k = t < W ? col[i * W + t] : -1;
    const unsigned pad = __ballot_sync(0xffffffffu, k < 0);
    const int limit = pad ? __ffs(pad) - 1 : 32;
    last = pad != 0;
    return (lane < limit && fabs(val[i * W + t]) >= tau) ? k : -1;
}

__global__ void __launch_bounds__(32 * kEllWarps) ell_count_kernel(const int32_t* __restrict__ col,
                                                                   const double* __restrict__ val, int64_t n, int64_t W,
                                                                   double tau, int32_t* cnt_own, int32_t* cnt_tr) {
    const int64_t i = (int64_t)blockIdx.x * kEllWarps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;   // whole warps
    int own = 0;
    bool last = false;
    for (int64_t t0 = 0; t0 < W && !last; t0 += 32) {
        const int k = ell_kept(col, val, i, W, t0, tau, lane, last);
        own += __popc(__ballot_sync(0xffffffffu, k >= 0));
        if (k >= 0) atomicAdd(&cnt_tr[k], 1);
    }
    if (lane == 0) cnt_own[i] = own;
}

__global__ void __launch_bounds__(32 * kEllWarps) ell_fill_kernel(const int32_t* __restrict__ col,
                                                                  const double* __restrict__ val, int64_t n, int64_t W,
                                                                  double tau, const int64_t* __restrict__ rp_own,
                                                                  int32_t* ci_own, const int64_t* __restrict__ rp_tr,
                                                                  int32_t* cur_tr, int32_t* ci_tr) {
    const int64_t i = (int64_t)blockIdx.x * kEllWarps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    int64_t o = rp_own[i];
    bool last = false;
    for (int64_t t0 = 0; t0 < W && !last; t0 += 32) {
        const int k = ell_kept(col, val, i, W, t0, tau, lane, last);
        const unsigned keep = __ballot_sync(0xffffffffu, k >= 0);
        if (k >= 0) {
            ci_own[o + __popc(keep & ((1u << lane) - 1u))] = k;
            ci_tr[rp_tr[k] + atomicAdd(&cur_tr[k], 1)] = (int32_t)i;
        }
        o += __popc(keep);
    }
}

// ------------------------------------------------------------------ partition
// Core set of subgraph s: members[core_start[s] .. core_start[s+1]) (ascending).
// Writes m_s, c_s and the local index list (cores, then sorted halo) into a slot of
// capacity `cap` at s * cap.
__global__ void __launch_bounds__(256) halo_kernel(int64_t P, const int64_t* __restrict__ core_start,
                                                   const int32_t* __restrict__ members,
                                                   const int64_t* __restrict__ arp, const int32_t* __restrict__ aci,
                                                   int hops, int cap, int32_t* msize, int32_t* csize, int32_t* slots,
                                                   int* overflow) {
    extern __shared__ unsigned char smraw[];
    RowSetSmem& S = *reinterpret_cast<RowSetSmem*>(smraw);
    for (int64_t s = blockIdx.x; s < P; s += gridDim.x) {
        const int64_t c0 = core_start[s];
        const int c = (int)(core_start[s + 1] - c0);
        hset_clear(S.table, &S.count, &S.flag);
        for (int t = threadIdx.x; t < c; t += blockDim.x) hset_insert(S.table, &S.count, members[c0 + t]);
        __syncthreads();
        const bool ok = (c <= kSetMax) && hset_expand(S.table, &S.count, S.list, &S.cursor, &S.flag, arp, aci, hops);
        if (!ok || S.count > cap || S.count > kSetMax) {
            if (threadIdx.x == 0) { atomicExch(overflow, max(S.count, c)); msize[s] = 0; csize[s] = c; }
            __syncthreads();
            continue;
        }
        const int m = hset_compact(S.table, S.list, &S.cursor);
        bitonic_sort(S.list, m, kHashCap);
        int32_t* out = slots + s * (int64_t)cap;
        for (int t = threadIdx.x; t < c; t += blockDim.x) out[t] = members[c0 + t];
        // halo = sorted set minus the (sorted) core members, order kept: ordered compaction
        if (threadIdx.x == 0) S.cursor = 0;
        __syncthreads();
        for (int t0 = 0; t0 < m; t0 += blockDim.x) {
            const int t = t0 + threadIdx.x;
            int keep = 0, v = 0;
            if (t < m) {
                v = S.list[t];
                int lo = 0, hi = c - 1;
                keep = 1;
                while (lo <= hi) {
                    const int mid = (lo + hi) >> 1;
                    const int x = members[c0 + mid];
                    if (x == v) { keep = 0; break; }
                    if (x < v) lo = mid + 1; else hi = mid - 1;
                }
            }
            __shared__ int wsum[8];
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
            if (lane == 0) wsum[w] = __popc(bal);
            __syncthreads();
            int before = 0;
            for (int q = 0; q < w; ++q) before += wsum[q];
            const int base = S.cursor;
            __syncthreads();
            if (keep) out[c + base + before + __popc(bal & ((1u << lane) - 1u))] = v;
            __syncthreads();
            if (threadIdx.x == 0) {
                int tot = 0;
                for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += wsum[q];
                S.cursor = base + tot;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) { msize[s] = c + S.cursor; csize[s] = c; }
        __syncthreads();
    }
}

__global__ void compact_slots_kernel(int64_t P, const int32_t* __restrict__ slots, int cap,
                                     const int64_t* __restrict__ sub_ptr, int32_t* sub_idx) {
    for (int64_t s = blockIdx.x; s < P; s += gridDim.x) {
        const int64_t b = sub_ptr[s], m = sub_ptr[s + 1] - b;
        for (int64_t t = threadIdx.x; t < m; t += blockDim.x) sub_idx[b + t] = slots[s * (int64_t)cap + t];
    }
}

__global__ void iota_blocks_kernel(int64_t n, int32_t* members) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) members[i] = (int32_t)i;
}

// ------------------------------------------------------------------ host helpers
size_t rowset_smem() { return sizeof(RowSetSmem); }

// Build a CSR whose row i is produced by rowset_kernel (count, scan, fill).
int rowset_csr(gbe_ctx* ctx, int mode, int64_t n, const gbe_csr* H, double thresh, const int64_t* s1rp,
               const int32_t* s1ci, const int64_t* s2rp, const int32_t* s2ci, const int64_t* s3rp, const int32_t* s3ci,
               int hops, int64_t** rp_out, int32_t** ci_out, int64_t* nnz_out) {
    DevBuf cnt, flag, stage;
    GBE_TRY(gbe_alloc(&cnt.p, n * 4));
    // [0] a row above kSetMax, [1] a row above the staging slot, [2] a row of H^2 above the
    // warp table of warp_rowset_kernel
    GBE_TRY(gbe_alloc(&flag.p, 12));
    GBE_CUDA_TRY(cudaMemsetAsync(flag.p, 0, 12, ctx->stream));
    // one set construction per row into staging slots (at most 64 Mi entries in all), then a
    // compaction; a row longer than its slot falls back to a second construction pass
    const int stage_cap = (int)std::min<int64_t>(kSetMax, std::max<int64_t>(128, ((int64_t)64 << 20) / n));
    GBE_TRY(gbe_alloc(&stage.p, n * stage_cap * 4));
    const size_t sm = rowset_smem();
    cudaFuncSetAttribute(rowset_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const int grid = (int)std::min<int64_t>(n, (int64_t)ctx->sm_count * 3);
    const int64_t* hrp = H ? H->rowptr : nullptr;
    const int32_t* hci = H ? H->col : nullptr;
    const double* hva = H ? H->val : nullptr;
    // modes 0 and 1 a warp per row, unless a row overflows the warp's table
    bool h2acc = mode == 0 || mode == 1;
    auto launch = [&](int pass, const int64_t* outrp, int32_t* outci) {
        const unsigned wb = (unsigned)((n + kH2RowWarps - 1) / kH2RowWarps);
        if (h2acc && mode == 0)
            warp_rowset_kernel<0><<<wb, 32 * kH2RowWarps, kH2RowSmem, ctx->stream>>>(
                n, hrp, hci, hva, thresh, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, pass, cnt.as<int32_t>(),
                outrp, outci, flag.as<int>(), stage_cap);
        else if (h2acc)
            warp_rowset_kernel<1><<<wb, 32 * kH2RowWarps, kH2RowSmem, ctx->stream>>>(
                n, nullptr, nullptr, nullptr, 0.0, s1rp, s1ci, s2rp, s2ci, s3rp, s3ci, pass, cnt.as<int32_t>(), outrp,
                outci, flag.as<int>(), stage_cap);
        else
            rowset_kernel<<<grid, 256, sm, ctx->stream>>>(mode, n, hrp, hci, hva, thresh, s1rp, s1ci, s2rp, s2ci, s3rp,
                                                          s3ci, hops, pass, cnt.as<int32_t>(), outrp, outci,
                                                          flag.as<int>(), stage_cap);
    };
    if (h2acc) {
        GBE_CUDA_TRY(cudaFuncSetAttribute(warp_rowset_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kH2RowSmem));
        GBE_CUDA_TRY(cudaFuncSetAttribute(warp_rowset_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kH2RowSmem));
        launch(2, nullptr, stage.as<int32_t>());
        int ovf2 = 0;
        GBE_CUDA_TRY(cudaGetLastError());
        GBE_CUDA_TRY(cudaMemcpyAsync(&ovf2, flag.as<int>() + 2, 4, cudaMemcpyDeviceToHost, ctx->stream));
        GBE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        if (ovf2) {
            h2acc = false;
            GBE_CUDA_TRY(cudaMemsetAsync(flag.p, 0, 12, ctx->stream));
        }
    }
    if (!h2acc) launch(2, nullptr, stage.as<int32_t>());
    GBE_CUDA_TRY(cudaGetLastError());
    int64_t* rp = nullptr;
    GBE_TRY(gbe_alloc((void**)&rp, (n + 1) * 8));
    int64_t nnz = 0;
    int r = scan_exclusive(ctx, cnt.as<int32_t>(), rp, n, &nnz);
    int ovf[2] = {0, 0};
    if (r == GBE_OK) {
        cudaError_t fe = cudaMemcpyAsync(ovf, flag.p, 8, cudaMemcpyDeviceToHost, ctx->stream);
        if (fe == cudaSuccess) fe = cudaStreamSynchronize(ctx->stream);
        if (fe != cudaSuccess) {
            gbe_set_error("rowset: reading the overflow flags: %s", cudaGetErrorString(fe));
            r = GBE_ECUDA;
        }
    }
    if (r == GBE_OK && ovf[0]) {
        gbe_set_error("graph row exceeds %d entries", kSetMax);
        r = GBE_ECAPACITY;
    }
    int32_t* ci = nullptr;
    if (r == GBE_OK) r = gbe_alloc((void**)&ci, std::max<int64_t>(nnz, 1) * 4);
    if (r != GBE_OK) { gbe_free(rp); return r; }
    if (!ovf[1])
        compact_set_rows_kernel<<<(unsigned)((n + 7) / 8), 256, 0, ctx->stream>>>(stage.as<int32_t>(), n, stage_cap, rp,
                                                                                ci);
    else
        launch(1, rp, ci);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        gbe_free(rp); gbe_free(ci);
        gbe_set_error("rowset: %s", cudaGetErrorString(e));
        return GBE_ECUDA;
    }
    *rp_out = rp; *ci_out = ci; *nnz_out = nnz;
    return GBE_OK;
}

}  // namespace

// ============================================================================= Hamiltonian
extern "C" int gbe_build_hamiltonian(gbe_ctx* ctx, const gbe_sites* st, const gbe_tb_model* model, gbe_hamiltonian** out) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && st && model && out, "NULL argument");
    GBE_CHECK_ARG(st->n > 0 && st->n < INT32_MAX && st->pos && st->onsite, "sites");
    GBE_CHECK_ARG(model->rcut > 0 && model->decay > 0, "model");
    for (int d = 0; d < 3; ++d) GBE_CHECK_ARG(st->box[d] > 2.0 * model->rcut, "box must exceed 2 rcut (minimum image)");
    GBE_CUDA_TRY(cudaSetDevice(ctx->device));
    const int64_t n = st->n;
    cudaStream_t s = ctx->stream;
    DevBuf hpos, hons;
    const double *pos, *ons;
    GBE_TRY(to_device(ctx, st->pos, n * 24, st->on_device, hpos, (const void**)&pos));
    GBE_TRY(to_device(ctx, st->onsite, n * 8, st->on_device, hons, (const void**)&ons));
    CellGrid g;
    int64_t ncells = 1;
    for (int d = 0; d < 3; ++d) {
        g.nc[d] = std::max(1, (int)floor(st->box[d] / model->rcut));
        g.box[d] = st->box[d];
        g.inv[d] = 1.0 / st->box[d];
        ncells *= g.nc[d];
    }
    DevBuf cell, ccnt, cstart, cur, mem, cnt, flag;
    GBE_TRY(gbe_alloc(&cell.p, n * 4));
    GBE_TRY(gbe_alloc(&ccnt.p, ncells * 4));
    GBE_TRY(gbe_alloc(&cstart.p, (ncells + 1) * 8));
    GBE_TRY(gbe_alloc(&cur.p, ncells * 4));
    GBE_TRY(gbe_alloc(&mem.p, n * 4));
    GBE_TRY(gbe_alloc(&cnt.p, n * 4));
    GBE_TRY(gbe_alloc(&flag.p, 8));   // [0] a row above kRowCap, [1] a row above kStageCap
    GBE_CUDA_TRY(cudaMemsetAsync(ccnt.p, 0, ncells * 4, s));
    GBE_CUDA_TRY(cudaMemsetAsync(cur.p, 0, ncells * 4, s));
    GBE_CUDA_TRY(cudaMemsetAsync(flag.p, 0, 8, s));
    const unsigned nb = (unsigned)((n + 255) / 256);
    cell_count_kernel<<<nb, 256, 0, s>>>(pos, n, g, cell.as<int32_t>(), ccnt.as<int32_t>());
    GBE_TRY(scan_exclusive(ctx, ccnt.as<int32_t>(), cstart.as<int64_t>(), ncells, nullptr));
    cell_fill_kernel<<<nb, 256, 0, s>>>(cell.as<int32_t>(), n, cstart.as<int64_t>(), cur.as<int32_t>(), mem.as<int32_t>());
    HModel mdl{model->a, model->rcut, 1.0 / model->decay, model->hop, model->rcut * model->rcut};
    DevBuf p4;
    GBE_TRY(gbe_alloc(&p4.p, n * 16));
    pos_f32_kernel<<<nb, 256, 0, s>>>(pos, n, p4.as<float4>());
    const float lim2 = filter_lim2(model->rcut, st->box), lim2_in = filter_lim2_in(model->rcut, st->box);
    const unsigned rb = (unsigned)((n + 7) / 8);
    // one neighbour search: sorted rows into staging slots, then a compaction; a row longer
    // than a slot falls back to a second search that writes the CSR directly
    DevBuf scol, sval;
    GBE_TRY(gbe_alloc(&scol.p, n * kStageCap * 4));
    GBE_TRY(gbe_alloc(&sval.p, n * kStageCap * 8));
    hbuild_kernel<<<rb, 256, 0, s>>>(pos, p4.as<float4>(), ons, n, g, lim2, lim2_in, cstart.as<int64_t>(), mem.as<int32_t>(), mdl, 2,
                                     cnt.as<int32_t>(),
                                     nullptr, scol.as<int32_t>(), sval.as<double>(), flag.as<int>());
    GBE_CUDA_TRY(cudaGetLastError());
    gbe_hamiltonian* H = new gbe_hamiltonian();
    H->n = n;
    int r = gbe_alloc((void**)&H->rowptr, (n + 1) * 8);
    int64_t nnz = 0;
    if (r == GBE_OK) r = scan_exclusive(ctx, cnt.as<int32_t>(), H->rowptr, n, &nnz);
    int ovf[2] = {0, 0};
    if (r == GBE_OK) {
        cudaError_t fe = cudaMemcpyAsync(ovf, flag.p, 8, cudaMemcpyDeviceToHost, s);
        if (fe == cudaSuccess) fe = cudaStreamSynchronize(s);
        if (fe != cudaSuccess) {
            gbe_set_error("hbuild: reading the overflow flags: %s", cudaGetErrorString(fe));
            r = GBE_ECUDA;
        }
    }
    if (r == GBE_OK && ovf[0]) { gbe_set_error("a row of H has more than %d neighbours", kRowCap); r = GBE_ECAPACITY; }
    if (r == GBE_OK) r = gbe_alloc((void**)&H->col, nnz * 4);
    if (r == GBE_OK) r = gbe_alloc((void**)&H->val, nnz * 8);
    if (r != GBE_OK) { gbe_free_hamiltonian(H); return r; }
    H->nnz = nnz;
    if (!ovf[1])
        compact_rows_kernel<<<(unsigned)((n * kStageCap + 255) / 256), 256, 0, s>>>(
            scol.as<int32_t>(), sval.as<double>(), n, H->rowptr, H->col, H->val);
    else
        hbuild_kernel<<<rb, 256, 0, s>>>(pos, p4.as<float4>(), ons, n, g, lim2, lim2_in, cstart.as<int64_t>(), mem.as<int32_t>(), mdl,
                                         1, cnt.as<int32_t>(), H->rowptr, H->col, H->val, flag.as<int>());
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        gbe_free_hamiltonian(H);
        gbe_set_error("hbuild: %s", cudaGetErrorString(e));
        return GBE_ECUDA;
    }
    *out = H;
    return GBE_OK;
}

extern "C" int gbe_hamiltonian_csr(const gbe_hamiltonian* H, gbe_csr* v) {
    GBE_CHECK_ARG(H && v, "NULL argument");
    v->n = H->n; v->nnz = H->nnz; v->rowptr = H->rowptr; v->col = H->col; v->val = H->val; v->on_device = 1;
    return GBE_OK;
}

extern "C" int gbe_free_hamiltonian(gbe_hamiltonian* H) {
    if (!H) return GBE_OK;
    gbe_free(H->rowptr); gbe_free(H->col); gbe_free(H->val);
    delete H;
    return GBE_OK;
}

// ============================================================================= graph
extern "C" int gbe_free_graph(gbe_graph* S) {
    if (!S) return GBE_OK;
    gbe_free(S->rowptr); gbe_free(S->col);
    if (S->full_rowptr != S->rowptr) { gbe_free(S->full_rowptr); gbe_free(S->full_col); }
    delete S;
    return GBE_OK;
}

int gbe_graph_mlp_select(gbe_ctx* ctx, const gbe_csr* H, const gbe_graph_params* p, int64_t** rp, int32_t** ci);

extern "C" int gbe_build_graph(gbe_ctx* ctx, const gbe_csr* Hin, const gbe_graph_params* p, gbe_graph** out) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && Hin && p && out, "NULL argument");
    GBE_CHECK_ARG(Hin->n > 0 && Hin->n < INT32_MAX, "H size");
    GBE_CUDA_TRY(cudaSetDevice(ctx->device));
    const int64_t n = Hin->n;
    // H on the device
    DevBuf hrp, hci, hva;
    gbe_csr H = *Hin;
    GBE_TRY(gbe_check_device_csr(ctx, Hin, "gbe_build_graph H"));
    if (!Hin->on_device) {
        GBE_TRY(to_device(ctx, Hin->rowptr, (n + 1) * 8, 0, hrp, (const void**)&H.rowptr));
        GBE_TRY(to_device(ctx, Hin->col, Hin->nnz * 4, 0, hci, (const void**)&H.col));
        GBE_TRY(to_device(ctx, Hin->val, Hin->nnz * 8, 0, hva, (const void**)&H.val));
        H.on_device = 1;
    }
    gbe_graph* S = new gbe_graph();
    S->n = n;
    int r = GBE_OK;
    switch (p->mode) {
        case GBE_GRAPH_H2_THRESH:
            r = rowset_csr(ctx, 0, n, &H, p->thresh, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 1,
                           &S->rowptr, &S->col, &S->nnz);
            S->hops = 1;
            break;
        case GBE_GRAPH_HK_PATTERN:
            GBE_CHECK_ARG(p->k >= 1, "k >= 1");
            // base A = pattern(H) with the diagonal (union with itself adds the diagonal)
            r = rowset_csr(ctx, 1, n, nullptr, 0.0, H.rowptr, H.col, nullptr, nullptr, nullptr, nullptr, 1, &S->rowptr,
                           &S->col, &S->nnz);
            S->hops = p->k;
            break;
        case GBE_GRAPH_D_THRESH:
        case GBE_GRAPH_EQ8_SYMBOLIC: {
            const gbe_ell* D = p->D_prev;
            if (!D || !D->col || !D->val || D->n != n) { delete S; gbe_set_error("D_prev missing or wrong size"); return GBE_EINVAL; }
            DevBuf dcol, dval;
            const int32_t* ecol;
            const double* eval;
            r = to_device(ctx, D->col, D->n * D->width * 4, D->on_device, dcol, (const void**)&ecol);
            if (r == GBE_OK) r = to_device(ctx, D->val, D->n * D->width * 8, D->on_device, dval, (const void**)&eval);
            DevBuf co, ct, rpo, rpt, cio, cit, cur;
            if (r == GBE_OK) r = gbe_alloc(&co.p, n * 4);
            if (r == GBE_OK) r = gbe_alloc(&ct.p, n * 4);
            if (r == GBE_OK) r = gbe_alloc(&rpo.p, (n + 1) * 8);
            if (r == GBE_OK) r = gbe_alloc(&rpt.p, (n + 1) * 8);
            if (r == GBE_OK) r = gbe_alloc(&cur.p, n * 4);
            if (r != GBE_OK) break;
            cudaMemsetAsync(ct.p, 0, n * 4, ctx->stream);
            cudaMemsetAsync(cur.p, 0, n * 4, ctx->stream);
            const unsigned nb = (unsigned)((n + kEllWarps - 1) / kEllWarps);
            ell_count_kernel<<<nb, 32 * kEllWarps, 0, ctx->stream>>>(ecol, eval, n, D->width, p->thresh, co.as<int32_t>(),
                                                                     ct.as<int32_t>());
            int64_t no = 0, nt = 0;
            r = scan_exclusive(ctx, co.as<int32_t>(), rpo.as<int64_t>(), n, &no);
            if (r == GBE_OK) r = scan_exclusive(ctx, ct.as<int32_t>(), rpt.as<int64_t>(), n, &nt);
            if (r == GBE_OK) r = gbe_alloc(&cio.p, std::max<int64_t>(no, 1) * 4);
            if (r == GBE_OK) r = gbe_alloc(&cit.p, std::max<int64_t>(nt, 1) * 4);
            if (r != GBE_OK) break;
            ell_fill_kernel<<<nb, 32 * kEllWarps, 0, ctx->stream>>>(ecol, eval, n, D->width, p->thresh, rpo.as<int64_t>(),
                                                         cio.as<int32_t>(), rpt.as<int64_t>(), cur.as<int32_t>(), cit.as<int32_t>());
            const bool eq8 = (p->mode == GBE_GRAPH_EQ8_SYMBOLIC);
            r = rowset_csr(ctx, 1, n, nullptr, 0.0, rpo.as<int64_t>(), cio.as<int32_t>(), rpt.as<int64_t>(),
                           cit.as<int32_t>(), eq8 ? H.rowptr : nullptr, eq8 ? H.col : nullptr, 1, &S->rowptr, &S->col,
                           &S->nnz);
            S->hops = eq8 ? 2 : 1;
            break;
        }
        case GBE_GRAPH_MLP: {
            // pairs the network keeps (a symmetric set: features are symmetric in i, j),
            // united with the pattern of H and the diagonal
            int64_t* srp = nullptr;
            int32_t* sci = nullptr;
            r = gbe_graph_mlp_select(ctx, &H, p, &srp, &sci);
            if (r == GBE_OK)
                r = rowset_csr(ctx, 1, n, nullptr, 0.0, srp, sci, H.rowptr, H.col, nullptr, nullptr, 1, &S->rowptr,
                               &S->col, &S->nnz);
            gbe_free(srp);
            gbe_free(sci);
            S->hops = 1;
            break;
        }
        default:
            gbe_set_error("unknown graph mode %d", p->mode);
            r = GBE_EINVAL;
    }
    if (r != GBE_OK) { gbe_free_graph(S); return r; }
    if (S->hops == 1) { S->full_rowptr = S->rowptr; S->full_col = S->col; S->full_nnz = S->nnz; }
    *out = S;
    return GBE_OK;
}

extern "C" int gbe_graph_size(gbe_ctx* ctx, gbe_graph* S, int64_t* n, int64_t* nnz) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && S, "NULL argument");
    if (S->full_nnz < 0) {
        GBE_TRY(rowset_csr(ctx, 2, S->n, nullptr, 0.0, S->rowptr, S->col, nullptr, nullptr, nullptr, nullptr, S->hops,
                           &S->full_rowptr, &S->full_col, &S->full_nnz));
    }
    if (n) *n = S->n;
    if (nnz) *nnz = S->full_nnz;
    return GBE_OK;
}

extern "C" int gbe_graph_export(gbe_ctx* ctx, gbe_graph* S, int64_t* rowptr, int32_t* col) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && S && rowptr && col, "NULL argument");
    GBE_TRY(gbe_graph_size(ctx, S, nullptr, nullptr));
    GBE_CUDA_TRY(cudaMemcpyAsync(rowptr, S->full_rowptr, (S->n + 1) * 8, cudaMemcpyDeviceToHost, ctx->stream));
    if (S->full_nnz > 0)
        GBE_CUDA_TRY(cudaMemcpyAsync(col, S->full_col, S->full_nnz * 4, cudaMemcpyDeviceToHost, ctx->stream));
    GBE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return GBE_OK;
}

// ============================================================================= partition
extern "C" int gbe_partition(gbe_ctx* ctx, const gbe_graph* S, const gbe_partition_params* p, gbe_parts** out) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && S && p && out, "NULL argument");
    GBE_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const int64_t n = S->n;
    const int cap = p->max_sub > 0 ? std::min(p->max_sub, kSetMax) : kSetMax;
    DevBuf cstart, mem;
    int64_t P = 0;
    GBE_TRY(gbe_alloc(&mem.p, n * 4));
    if (p->mode == GBE_PART_SPATIAL_CELLS) {
        GBE_CHECK_ARG(p->sites && p->sites->n == n && p->sites->pos, "spatial cells need sites of the graph's size");
        GBE_CHECK_ARG(p->ncell[0] > 0 && p->ncell[1] > 0 && p->ncell[2] > 0, "ncell");
        DevBuf hpos;
        const double* pos;
        GBE_TRY(to_device(ctx, p->sites->pos, n * 24, p->sites->on_device, hpos, (const void**)&pos));
        CellGrid g;
        int64_t ncells = 1;
        for (int d = 0; d < 3; ++d) {
            g.nc[d] = p->ncell[d];
            g.box[d] = p->sites->box[d];
            g.inv[d] = 1.0 / p->sites->box[d];
            ncells *= g.nc[d];
        }
        GBE_CHECK_ARG(ncells < INT32_MAX, "too many cells");
        DevBuf cell, ccnt, cst, cur;
        GBE_TRY(gbe_alloc(&cell.p, n * 4));
        GBE_TRY(gbe_alloc(&ccnt.p, ncells * 4));
        GBE_TRY(gbe_alloc(&cst.p, (ncells + 1) * 8));
        GBE_TRY(gbe_alloc(&cur.p, ncells * 4));
        GBE_CUDA_TRY(cudaMemsetAsync(ccnt.p, 0, ncells * 4, st));
        GBE_CUDA_TRY(cudaMemsetAsync(cur.p, 0, ncells * 4, st));
        const unsigned nb = (unsigned)((n + 255) / 256);
        cell_count_kernel<<<nb, 256, 0, st>>>(pos, n, g, cell.as<int32_t>(), ccnt.as<int32_t>());
        GBE_TRY(scan_exclusive(ctx, ccnt.as<int32_t>(), cst.as<int64_t>(), ncells, nullptr));
        cell_fill_kernel<<<nb, 256, 0, st>>>(cell.as<int32_t>(), n, cst.as<int64_t>(), cur.as<int32_t>(), mem.as<int32_t>());
        cell_sort_kernel<<<(unsigned)((ncells * 32 + 255) / 256), 256, 0, st>>>(cst.as<int64_t>(), (int)ncells, mem.as<int32_t>());
        // non-empty cells, ascending id -> core_start
        std::vector<int64_t> hst(ncells + 1);
        GBE_CUDA_TRY(cudaMemcpyAsync(hst.data(), cst.p, (ncells + 1) * 8, cudaMemcpyDeviceToHost, st));
        GBE_CUDA_TRY(cudaStreamSynchronize(st));
        std::vector<int64_t> cs;
        cs.reserve(ncells + 1);
        for (int64_t c = 0; c < ncells; ++c)
            if (hst[c + 1] > hst[c]) cs.push_back(hst[c]);
        cs.push_back(hst[ncells]);
        P = (int64_t)cs.size() - 1;
        GBE_TRY(gbe_alloc(&cstart.p, (P + 1) * 8));
        GBE_CUDA_TRY(cudaMemcpyAsync(cstart.p, cs.data(), (P + 1) * 8, cudaMemcpyHostToDevice, st));
        GBE_CUDA_TRY(cudaStreamSynchronize(st));
    } else if (p->mode == GBE_PART_INDEX_BLOCKS) {
        GBE_CHECK_ARG(p->core_size > 0, "core_size");
        P = (n + p->core_size - 1) / p->core_size;
        std::vector<int64_t> cs(P + 1);
        for (int64_t s = 0; s <= P; ++s) cs[s] = std::min<int64_t>(s * p->core_size, n);
        GBE_TRY(gbe_alloc(&cstart.p, (P + 1) * 8));
        GBE_CUDA_TRY(cudaMemcpyAsync(cstart.p, cs.data(), (P + 1) * 8, cudaMemcpyHostToDevice, st));
        iota_blocks_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, mem.as<int32_t>());
        GBE_CUDA_TRY(cudaStreamSynchronize(st));
    } else {
        gbe_set_error("unknown partition mode %d", p->mode);
        return GBE_EINVAL;
    }
    DevBuf msz, csz, slots, flag;
    GBE_TRY(gbe_alloc(&msz.p, P * 4));
    GBE_TRY(gbe_alloc(&csz.p, P * 4));
    GBE_TRY(gbe_alloc(&slots.p, (size_t)P * cap * 4));
    GBE_TRY(gbe_alloc(&flag.p, 4));
    GBE_CUDA_TRY(cudaMemsetAsync(flag.p, 0, 4, st));
    const size_t sm = rowset_smem();
    cudaFuncSetAttribute(halo_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const int grid = (int)std::min<int64_t>(P, (int64_t)ctx->sm_count * 3);
    halo_kernel<<<grid, 256, sm, st>>>(P, cstart.as<int64_t>(), mem.as<int32_t>(), S->rowptr, S->col, S->hops, cap,
                                       msz.as<int32_t>(), csz.as<int32_t>(), slots.as<int32_t>(), flag.as<int>());
    GBE_CUDA_TRY(cudaGetLastError());
    int ovf = 0;
    GBE_TRY(read_flag(ctx, flag.as<int>(), &ovf));
    if (ovf) {
        gbe_set_error("a core+halo subgraph exceeds capacity %d (needs >= %d)", cap, ovf);
        return GBE_ECAPACITY;
    }
    gbe_parts* parts = new gbe_parts();
    parts->n = n;
    parts->P = P;
    parts->cores_cover = 1;   // cells and index blocks both partition the vertices
    parts->h_core_count.resize(P);
    std::vector<int32_t> hm(P);
    cudaMemcpyAsync(hm.data(), msz.p, P * 4, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(parts->h_core_count.data(), csz.p, P * 4, cudaMemcpyDeviceToHost, st);
    GBE_CUDA_TRY(cudaStreamSynchronize(st));
    parts->h_sub_ptr.resize(P + 1);
    parts->h_sub_ptr[0] = 0;
    for (int64_t s = 0; s < P; ++s) {
        parts->h_sub_ptr[s + 1] = parts->h_sub_ptr[s] + hm[s];
        parts->max_m = std::max<int64_t>(parts->max_m, hm[s]);
    }
    parts->total = parts->h_sub_ptr[P];
    int r = gbe_alloc((void**)&parts->d_core_count, P * 4);
    if (r == GBE_OK) r = gbe_alloc((void**)&parts->d_sub_ptr, (P + 1) * 8);
    if (r == GBE_OK) r = gbe_alloc((void**)&parts->d_sub_idx, parts->total * 4);
    if (r != GBE_OK) { gbe_free_parts(parts); return r; }
    cudaMemcpyAsync(parts->d_core_count, csz.p, P * 4, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(parts->d_sub_ptr, parts->h_sub_ptr.data(), (P + 1) * 8, cudaMemcpyHostToDevice, st);
    compact_slots_kernel<<<grid, 256, 0, st>>>(P, slots.as<int32_t>(), cap, parts->d_sub_ptr, parts->d_sub_idx);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        gbe_free_parts(parts);
        gbe_set_error("partition: %s", cudaGetErrorString(e));
        return GBE_ECUDA;
    }
    *out = parts;
    return GBE_OK;
}

