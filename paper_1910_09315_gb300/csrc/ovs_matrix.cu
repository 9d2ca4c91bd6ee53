// The interpolation as a sparse matrix (Sec. 2.2.6: the boundary interpolation written as a matrix whose rows
// are the receiver points and whose columns are donor nodes, 8 trilinear weights per row), and the matrix-vector
// product that applies it, e.g. once per iteration of an implicit solve that keeps the donors fixed.
//
//   k_csr_count   1 / 0 per point: found in a donor grid or not (the scan turns it into row starts / 8)
//   k_csr_fill    a found point's 8 columns (global node id = the donor grid's node offset + node) and weights
//   k_spmv<T>     y = A x, a thread per row, the row's entries summed in column order
#include "ovs_internal.cuh"
#include "ovs_matrix.cuh"

namespace ovs {

namespace {

constexpr int kMatThreads = 256;

__global__ void __launch_bounds__(kMatThreads) k_csr_count(const uint8_t* __restrict__ status,
                                                           const int32_t* __restrict__ grid, int64_t n,
                                                           uint32_t* __restrict__ counts) {
    for (int64_t t = blockIdx.x * (int64_t)kMatThreads + threadIdx.x; t < n; t += (int64_t)gridDim.x * kMatThreads)
        counts[t] = ((__ldg(status + t) & OVS_STATUS_MASK) == OVS_STATUS_FOUND && __ldg(grid + t) >= 0) ? 1u : 0u;
}

// weights in the value type V from the stored local coordinates (the same products as the gather of k_interp)
template <typename V>
__global__ void __launch_bounds__(kMatThreads) k_csr_fill(const GridDev* __restrict__ G, int ngrids, NodeOffsets off,
                                                          const int32_t* __restrict__ grid,
                                                          const int32_t* __restrict__ cell, const void* __restrict__ xi,
                                                          int xi_f64, int64_t n, const int32_t* __restrict__ found_before,
                                                          int32_t* __restrict__ row_ptr, int64_t* __restrict__ col,
                                                          V* __restrict__ val, int32_t* __restrict__ err) {
    for (int64_t t = blockIdx.x * (int64_t)kMatThreads + threadIdx.x; t < n; t += (int64_t)gridDim.x * kMatThreads) {
        const int32_t k0 = __ldg(found_before + t), k1 = __ldg(found_before + t + 1);
        row_ptr[t] = 8 * k0;
        if (t == n - 1) row_ptr[n] = 8 * k1;
        if (k1 == k0) continue;  // not found: an empty row
        const int32_t gd = __ldg(grid + t), c = __ldg(cell + t);
        if (gd >= ngrids || c < 0 || c >= G[gd].ncells) {
            // a donor record this call cannot use: an empty 8-entry block (columns -1, weights 0)
            atomicOr(err, kErrBadCell);
            for (int a = 0; a < 8; ++a) {
                col[8 * (int64_t)k0 + a] = -1;
                val[8 * (int64_t)k0 + a] = (V)0;
            }
            continue;
        }
        V u, v, w;
        if (xi_f64) {
            const double* x = (const double*)xi;
            u = (V)__ldg(x + t);
            v = (V)__ldg(x + n + t);
            w = (V)__ldg(x + 2 * n + t);
        } else {
            const float* x = (const float*)xi;
            u = (V)__ldg(x + t);
            v = (V)__ldg(x + n + t);
            w = (V)__ldg(x + 2 * n + t);
        }
        const GridDev& g = G[gd];
        int i, j, k;
        cell_ijk(g, c, i, j, k);
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            col[8 * (int64_t)k0 + a] = off.off[gd] + corner_node(g, i, j, k, a);
            val[8 * (int64_t)k0 + a] = ((a & 1) ? u : (V)1 - u) * ((a & 2) ? v : (V)1 - v) * ((a & 4) ? w : (V)1 - w);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kMatThreads) k_spmv(int64_t nrows, const int32_t* __restrict__ row_ptr,
                                                      const int64_t* __restrict__ col, const T* __restrict__ val,
                                                      const T* __restrict__ x, T* __restrict__ y) {
    for (int64_t r = blockIdx.x * (int64_t)kMatThreads + threadIdx.x; r < nrows;
         r += (int64_t)gridDim.x * kMatThreads) {
        const int32_t e0 = __ldg(row_ptr + r), e1 = __ldg(row_ptr + r + 1);
        T s = (T)0;
        if (e1 - e0 == 8 && (e0 & 7) == 0) {
            // a full row (every row of ovs_interp_matrix): its 8 columns and values in 16-byte loads, then the 8
            // gathers together; summed in entry order as below
            const longlong2* cp = reinterpret_cast<const longlong2*>(col + e0);
            long long c[8];
            T v[8], xv[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const longlong2 cc = __ldg(cp + q);
                c[2 * q] = cc.x;
                c[2 * q + 1] = cc.y;
            }
#pragma unroll
            for (int a = 0; a < 8; ++a) v[a] = __ldg(val + e0 + a);
#pragma unroll
            for (int a = 0; a < 8; ++a) xv[a] = c[a] >= 0 ? __ldg(x + c[a]) : (T)0;
#pragma unroll
            for (int a = 0; a < 8; ++a)
                if (c[a] >= 0) s += v[a] * xv[a];
        } else {
            for (int32_t e = e0; e < e1; ++e) {
                const int64_t cidx = __ldg(col + e);
                if (cidx >= 0) s += __ldg(val + e) * __ldg(x + cidx);
            }
        }
        y[r] = s;
    }
}

unsigned grid_for(int64_t n, int nsm) {
    const int64_t want = (n + kMatThreads - 1) / kMatThreads;
    const int64_t cap = (int64_t)nsm * 16;
    return (unsigned)(want < 1 ? 1 : (want < cap ? want : cap));
}

}  // namespace

cudaError_t launch_interp_matrix(const GridDev* dgrids, int ngrids, const NodeOffsets& off, const uint8_t* status,
                                 const int32_t* grid, const int32_t* cell, const void* xi, int xi_f64, int64_t n,
                                 uint32_t* scratch, int32_t* row_ptr, int64_t* col, void* val, int val_f64,
                                 int32_t* err, int nsm, cudaStream_t st) {
    // scratch: n flags, then the n + 1 exclusive sums of the flags (int32), then the scan's tile sums
    uint32_t* flags = scratch;
    int32_t* found_before = (int32_t*)(scratch + n);
    uint32_t* tile_sums = (uint32_t*)(found_before + n + 1);
    const unsigned blocks = grid_for(n, nsm);
    k_csr_count<<<blocks, kMatThreads, 0, st>>>(status, grid, n, flags);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = launch_scan(flags, found_before, n, tile_sums, st)) != cudaSuccess) return e;
    if (val_f64)
        k_csr_fill<double><<<blocks, kMatThreads, 0, st>>>(dgrids, ngrids, off, grid, cell, xi, xi_f64, n, found_before,
                                                          row_ptr, col, (double*)val, err);
    else
        k_csr_fill<float><<<blocks, kMatThreads, 0, st>>>(dgrids, ngrids, off, grid, cell, xi, xi_f64, n, found_before,
                                                         row_ptr, col, (float*)val, err);
    return cudaGetLastError();
}

size_t interp_matrix_scratch_bytes(int64_t n) {
    const int64_t tiles = (n + kScanTileElems - 1) / kScanTileElems + 1;
    return sizeof(uint32_t) * (size_t)n + sizeof(int32_t) * (size_t)(n + 1) + sizeof(uint32_t) * (size_t)tiles;
}

cudaError_t launch_spmv(int64_t nrows, const int32_t* row_ptr, const int64_t* col, const void* val, const void* x,
                        void* y, int f64, int nsm, cudaStream_t st) {
    const unsigned blocks = grid_for(nrows, nsm);
    if (f64)
        k_spmv<double><<<blocks, kMatThreads, 0, st>>>(nrows, row_ptr, col, (const double*)val, (const double*)x,
                                                       (double*)y);
    else
        k_spmv<float><<<blocks, kMatThreads, 0, st>>>(nrows, row_ptr, col, (const float*)val, (const float*)x,
                                                      (float*)y);
    return cudaGetLastError();
}

}  // namespace ovs
