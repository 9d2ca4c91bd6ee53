// The interpolation matrix and its product (see ovs_matrix.cu).
#pragma once
#include "ovs_internal.cuh"

namespace ovs {

// column offset of each grid's nodes in the global node numbering: the sum of the node counts of the grids
// created before it
struct NodeOffsets {
    int64_t off[OVS_MAX_GRIDS];
};

// scratch bytes of launch_interp_matrix for n points
size_t interp_matrix_scratch_bytes(int64_t n);
cudaError_t launch_interp_matrix(const GridDev* dgrids, int ngrids, const NodeOffsets& off, const uint8_t* status,
                                 const int32_t* grid, const int32_t* cell, const void* xi, int xi_f64, int64_t n,
                                 uint32_t* scratch, int32_t* row_ptr, int64_t* col, void* val, int val_f64,
                                 int32_t* err, int nsm, cudaStream_t st);
cudaError_t launch_spmv(int64_t nrows, const int32_t* row_ptr, const int64_t* col, const void* val, const void* x,
                        void* y, int f64, int nsm, cudaStream_t st);

}  // namespace ovs
