// Grid set-up kernels: per-cell records and the control cells of Sec. 2.2.5 (uniform axis-aligned
// bins over the grid's bounding box, each cell registered in every bin its padded box overlaps), and the finer
// bins of crowded control cells (the same registration one level down).
#include <float.h>

#include "ovs_internal.cuh"

namespace ovs {

namespace {

constexpr int kBuildThreads = 256;

// Per-block reduction of 9 doubles: 3 minima, 3 maxima, 3 sums (fixed order, deterministic).
__device__ void block_reduce9(double v[9], double* out) {
    __shared__ double sh[kBuildThreads / 32][9];
    unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            double o = __shfl_down_sync(0xffffffffu, v[q], off);
            v[q] = q < 3 ? fmin(v[q], o) : (q < 6 ? fmax(v[q], o) : v[q] + o);
        }
    }
    if (lane == 0)
        for (int q = 0; q < 9; ++q) sh[wid][q] = v[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 0; q < 9; ++q) {
            double acc = sh[0][q];
            for (int w = 1; w < kBuildThreads / 32; ++w)
                acc = q < 3 ? fmin(acc, sh[w][q]) : (q < 6 ? fmax(acc, sh[w][q]) : acc + sh[w][q]);
            out[q] = acc;
        }
    }
}

__device__ __forceinline__ void split_store(double v, float* hi, float* lo) {
    float h = (float)v;
    *hi = h;
    *lo = (float)(v - (double)h);
}

// Orientation of a cell from the Jacobian determinants of its trilinear map at its 8 corners (FP64): +1 all
// positive, -1 all negative, 0 mixed or zero (a folded or degenerate cell).
__device__ __forceinline__ int cell_orientation(const double X[8][3]) {
    int pos = 0, neg = 0;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        double e[3][3];
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const int b = a ^ (1 << m);
            const double s = (a >> m) & 1 ? -1.0 : 1.0;  // the edge leaving corner a toward +index m
#pragma unroll
            for (int c = 0; c < 3; ++c) e[m][c] = s * (X[b][c] - X[a][c]);
        }
        const double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                           e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                           e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
        pos += det > 0.0;
        neg += det < 0.0;
    }
    return pos == 8 ? 1 : (neg == 8 ? -1 : 0);
}

// orient: 3 counters (cells with all corner Jacobians positive, all negative, mixed or zero)
__global__ void __launch_bounds__(kBuildThreads) k_build_records(GridDev g, CellRec* rec, float* xff,
                                                                 double* partials, unsigned long long* orient) {
    // node coordinates as FP32 pairs, SoA [xh | xl | yh | yl | zh | zl]
    for (int64_t nd = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; nd < g.nnodes;
         nd += (int64_t)gridDim.x * blockDim.x) {
        split_store(g.x[nd], xff + nd, xff + g.nnodes + nd);
        split_store(g.y[nd], xff + 2 * g.nnodes + nd, xff + 3 * g.nnodes + nd);
        split_store(g.z[nd], xff + 4 * g.nnodes + nd, xff + 5 * g.nnodes + nd);
    }
    double v[9] = {DBL_MAX, DBL_MAX, DBL_MAX, -DBL_MAX, -DBL_MAX, -DBL_MAX, 0, 0, 0};
    for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < g.ncells;
         cell += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        cell_ijk(g, cell, i, j, k);
        double X[8][3];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            int64_t nd = corner_node(g, i, j, k, a);
            X[a][0] = g.x[nd];
            X[a][1] = g.y[nd];
            X[a][2] = g.z[nd];
        }
        CellRec r;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double e1 = X[1][c] - X[0][c], e2 = X[2][c] - X[0][c], e3 = X[3][c] - X[0][c], e4 = X[4][c] - X[0][c],
                   e5 = X[5][c] - X[0][c], e6 = X[6][c] - X[0][c], e7 = X[7][c] - X[0][c];
            split_store(X[0][c], &r.x0h[c], &r.x0l[c]);
            r.a[c] = (float)e1;
            r.a[3 + c] = (float)e2;
            r.a[6 + c] = (float)e4;
            r.a[9 + c] = (float)(e3 - e1 - e2);
            r.a[12 + c] = (float)(e6 - e2 - e4);
            r.a[15 + c] = (float)(e5 - e1 - e4);
            r.a[18 + c] = (float)(e7 - e3 - e5 - e6 + e1 + e2 + e4);
            double mn = X[0][c], mx = X[0][c];
#pragma unroll
            for (int a = 1; a < 8; ++a) {
                mn = fmin(mn, X[a][c]);
                mx = fmax(mx, X[a][c]);
            }
            v[c] = fmin(v[c], mn);
            v[3 + c] = fmax(v[3 + c], mx);
            v[6 + c] += mx - mn;
        }
#pragma unroll
        for (int q = 0; q < 5; ++q) r.pad[q] = 0.f;
        rec[cell] = r;
        const int o = cell_orientation(X);
        atomicAdd(orient + (o > 0 ? 0 : (o < 0 ? 1 : 2)), 1ull);
    }
    block_reduce9(v, partials + 9 * blockIdx.x);
}

__global__ void __launch_bounds__(kBuildThreads) k_reduce_partials(const double* partials, int nblocks, double* out9) {
    // one block: thread t folds partials t, t + 256, ... in order, then the block reduction (fixed order)
    double v[9] = {DBL_MAX, DBL_MAX, DBL_MAX, -DBL_MAX, -DBL_MAX, -DBL_MAX, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += kBuildThreads)
        for (int q = 0; q < 9; ++q) {
            double o = partials[9 * b + q];
            v[q] = q < 3 ? fmin(v[q], o) : (q < 6 ? fmax(v[q], o) : v[q] + o);
        }
    block_reduce9(v, out9);
}

__device__ __forceinline__ void cell_bin_range(const GridDev& g, const CellRec& r, int b0[3], int b1[3]) {
    double lo[3], hi[3];
    rec_box(r, lo, hi);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double t0 = (lo[c] - g.lo[c]) * g.inv_w[c], t1 = (hi[c] - g.lo[c]) * g.inv_w[c];
        b0[c] = (int)fmin(fmax(floor(t0), 0.0), (double)(g.nb[c] - 1));
        b1[c] = (int)fmin(fmax(floor(t1), 0.0), (double)(g.nb[c] - 1));
    }
}

__global__ void __launch_bounds__(kBuildThreads) k_bin_count(GridDev g, uint32_t* counts) {
    for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < g.ncells;
         cell += (int64_t)gridDim.x * blockDim.x) {
        CellRec r;
        load_rec(g.rec, cell, r);
        int b0[3], b1[3];
        cell_bin_range(g, r, b0, b1);
        for (int bz = b0[2]; bz <= b1[2]; ++bz)
            for (int by = b0[1]; by <= b1[1]; ++by)
                for (int bx = b0[0]; bx <= b1[0]; ++bx)
                    atomicAdd(counts + (bx + (int64_t)g.nb[0] * (by + (int64_t)g.nb[1] * bz)), 1u);
    }
}

__global__ void __launch_bounds__(kBuildThreads) k_bin_fill(GridDev g, const int32_t* start, uint32_t* cursor,
                                                            int32_t* cells, int32_t* rep) {
    for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < g.ncells;
         cell += (int64_t)gridDim.x * blockDim.x) {
        CellRec r;
        load_rec(g.rec, cell, r);
        int b0[3], b1[3];
        cell_bin_range(g, r, b0, b1);
        for (int bz = b0[2]; bz <= b1[2]; ++bz)
            for (int by = b0[1]; by <= b1[1]; ++by)
                for (int bx = b0[0]; bx <= b1[0]; ++bx) {
                    int64_t b = bx + (int64_t)g.nb[0] * (by + (int64_t)g.nb[1] * bz);
                    uint32_t pos = atomicAdd(cursor + b, 1u);
                    cells[start[b] + pos] = (int32_t)cell;
                    atomicMin(rep + b, (int32_t)cell);
                }
    }
}

// Crowded control cells: those listing more than thr cells.
__global__ void __launch_bounds__(kBuildThreads) k_crowd_mark(const int32_t* start, int64_t nbins, int32_t thr,
                                                              int32_t* crowd, uint32_t* n, int cap) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nbins; b += (int64_t)gridDim.x * blockDim.x)
        if (start[b + 1] - start[b] > thr) {
            const uint32_t k = atomicAdd(n, 1u);
            if (k < (uint32_t)cap) crowd[k] = (int32_t)b;
        }
}

// The finer bins of crowded control cell b that a cell's padded box overlaps, per axis [s0, s1].
__device__ __forceinline__ void cell_sub_range(const GridDev& g, const CellRec& r, int64_t b, int s0[3], int s1[3]) {
    double lo[3], hi[3];
    rec_box(r, lo, hi);
    const int bi[3] = {(int)(b % g.nb[0]), (int)((b / g.nb[0]) % g.nb[1]), (int)(b / ((int64_t)g.nb[0] * g.nb[1]))};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        s0[c] = sub_coord(g, c, lo[c], bi[c]);
        s1[c] = sub_coord(g, c, hi[c], bi[c]);
    }
}

// One block per crowded control cell; its threads take the cells of its list.  FILL = false: count the
// registrations per finer bin; true: write them at start (cursor counts them again from zero).
template <bool FILL>
__global__ void __launch_bounds__(kBuildThreads) k_sub_bins(GridDev g, uint32_t* counts, const int32_t* start,
                                                            int32_t* cells) {
    for (int k = blockIdx.x; k < g.ncrowd; k += gridDim.x) {
        const int64_t b = g.crowd[k];
        const int32_t r0 = g.bin_start[b], r1 = g.bin_start[b + 1];
        for (int32_t r = r0 + (int32_t)threadIdx.x; r < r1; r += kBuildThreads) {
            const int32_t cell = g.bin_cells[r];
            CellRec rec;
            load_rec(g.rec, cell, rec);
            int s0[3], s1[3];
            cell_sub_range(g, rec, b, s0, s1);
            for (int sz = s0[2]; sz <= s1[2]; ++sz)
                for (int sy = s0[1]; sy <= s1[1]; ++sy)
                    for (int sx = s0[0]; sx <= s1[0]; ++sx) {
                        const int64_t sb = (int64_t)k * kSub3 + sub_index(sx, sy, sz);
                        const uint32_t pos = atomicAdd(counts + sb, 1u);
                        if (FILL) cells[start[sb] + pos] = cell;
                    }
        }
    }
}

// ---- exclusive scan of uint32 counts into int32 offsets (n + 1 entries) ----
constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;
static_assert(kScanTile == kScanTileElems, "scan tile size");

__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
    __shared__ uint32_t sh[kScanThreads / 32];
    unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        uint32_t o = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += o;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = lane < kScanThreads / 32 ? sh[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            uint32_t o = __shfl_up_sync(0xffffffffu, s, off);
            if (lane >= off) s += o;
        }
        if (lane < kScanThreads / 32) sh[lane] = s;
    }
    __syncthreads();
    uint32_t base = wid ? sh[wid - 1] : 0;
    *total = sh[kScanThreads / 32 - 1];
    __syncthreads();
    return base + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const uint32_t* in, int32_t* out, int64_t n,
                                                             uint32_t* tile_sums) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    uint32_t v[kScanPer], s = 0;
#pragma unroll
    for (int q = 0; q < kScanPer; ++q) {
        v[q] = base + q < n ? in[base + q] : 0u;
        s += v[q];
    }
    uint32_t tot;
    uint32_t pre = block_exclusive_scan(s, &tot);
#pragma unroll
    for (int q = 0; q < kScanPer; ++q) {
        if (base + q < n) out[base + q] = (int32_t)pre;
        pre += v[q];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(uint32_t* sums, int64_t ntiles, int32_t* out_total) {
    // single block: each thread scans a contiguous chunk
    int64_t per = (ntiles + kScanThreads - 1) / kScanThreads;
    int64_t b0 = threadIdx.x * per, b1 = min(ntiles, b0 + per);
    uint32_t s = 0;
    for (int64_t b = b0; b < b1; ++b) s += sums[b];
    uint32_t tot;
    uint32_t pre = block_exclusive_scan(s, &tot);
    for (int64_t b = b0; b < b1; ++b) {
        uint32_t x = sums[b];
        sums[b] = pre;
        pre += x;
    }
    if (threadIdx.x == 0) *out_total = (int32_t)tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_add(int32_t* out, int64_t n, const uint32_t* tile_off) {
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    uint32_t add = tile_off[blockIdx.x];
    for (int q = threadIdx.x; q < kScanTile; q += kScanThreads)
        if (base + q < n) out[base + q] += (int32_t)add;
}

}  // namespace

cudaError_t launch_build_records(const GridDev& g, CellRec* rec, float* xff, double* partials, int nblocks,
                                 double* out9, unsigned long long* orient, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(orient, 0, 3 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_build_records<<<nblocks, kBuildThreads, 0, st>>>(g, rec, xff, partials, orient);
    k_reduce_partials<<<1, kBuildThreads, 0, st>>>(partials, nblocks, out9);
    return cudaGetLastError();
}

cudaError_t launch_bin_count(const GridDev& g, uint32_t* counts, cudaStream_t st) {
    int64_t nb = (g.ncells + kBuildThreads - 1) / kBuildThreads;
    int blocks = (int)(nb < 152 * 64 ? nb : 152 * 64);
    k_bin_count<<<blocks, kBuildThreads, 0, st>>>(g, counts);
    return cudaGetLastError();
}

size_t scan_scratch_elems(int64_t n) { return (size_t)((n + kScanTile - 1) / kScanTile) + 1; }

__global__ void k_mark_blocked(GridDev g, const uint8_t* __restrict__ iblank, CellRec* __restrict__ rec) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.ncells;
         c += (int64_t)gridDim.x * blockDim.x) {
        uint32_t blocked = 0u;
        if (iblank) {
            int i, j, k;
            cell_ijk(g, c, i, j, k);
#pragma unroll
            for (int a = 0; a < 8; ++a)
                if (!__ldg(iblank + corner_node(g, i, j, k, a))) blocked = 1u;
        }
        rec[c].pad[0] = __uint_as_float(blocked);
    }
}

cudaError_t launch_mark_blocked(const GridDev& g, const uint8_t* iblank, cudaStream_t st) {
    const int64_t blocks = std::min<int64_t>((g.ncells + 255) / 256, 152 * 32);
    k_mark_blocked<<<(unsigned)std::max<int64_t>(1, blocks), 256, 0, st>>>(g, iblank, (CellRec*)g.rec);
    return cudaGetLastError();
}

cudaError_t launch_scan(const uint32_t* counts, int32_t* start, int64_t n, uint32_t* block_sums, cudaStream_t st) {
    int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    k_scan_tiles<<<(unsigned)ntiles, kScanThreads, 0, st>>>(counts, start, n, block_sums);
    k_scan_sums<<<1, kScanThreads, 0, st>>>(block_sums, ntiles, start + n);
    k_scan_add<<<(unsigned)ntiles, kScanThreads, 0, st>>>(start, n, block_sums);
    return cudaGetLastError();
}

cudaError_t launch_crowd_mark(const GridDev& g, int64_t nbins, int32_t thr, int32_t* crowd, uint32_t* n, int cap,
                              cudaStream_t st) {
    const int64_t nb = (nbins + kBuildThreads - 1) / kBuildThreads;
    const int blocks = (int)(nb < 152 * 64 ? (nb > 0 ? nb : 1) : 152 * 64);
    k_crowd_mark<<<blocks, kBuildThreads, 0, st>>>(g.bin_start, nbins, thr, crowd, n, cap);
    return cudaGetLastError();
}

cudaError_t launch_sub_count(const GridDev& g, uint32_t* counts, cudaStream_t st) {
    if (g.ncrowd <= 0) return cudaSuccess;
    k_sub_bins<false><<<(unsigned)g.ncrowd, kBuildThreads, 0, st>>>(g, counts, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_sub_fill(const GridDev& g, const int32_t* start, uint32_t* cursor, int32_t* cells, cudaStream_t st) {
    if (g.ncrowd <= 0) return cudaSuccess;
    k_sub_bins<true><<<(unsigned)g.ncrowd, kBuildThreads, 0, st>>>(g, cursor, start, cells);
    return cudaGetLastError();
}

cudaError_t launch_bin_fill(const GridDev& g, const int32_t* start, uint32_t* cursor, int32_t* cells, int32_t* rep,
                            cudaStream_t st) {
    int64_t nb = (g.ncells + kBuildThreads - 1) / kBuildThreads;
    int blocks = (int)(nb < 152 * 64 ? nb : 152 * 64);
    k_bin_fill<<<blocks, kBuildThreads, 0, st>>>(g, start, cursor, cells, rep);
    return cudaGetLastError();
}

}  // namespace ovs
