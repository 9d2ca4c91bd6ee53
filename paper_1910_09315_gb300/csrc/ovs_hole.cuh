// Hole cutting against closed triangulated body surfaces (see ovs_hole.cu).
#pragma once
#include <algorithm>
#include <cmath>
#include <vector>

#include "ovs_internal.cuh"

namespace ovs {

// A surface in the device workspace: vertices (body frame of its grid, FP64, xyz per vertex), triangles (3 vertex
// ids each), and the bins of the projected y-z box (CSR: bin_start[nb0 * nb1 + 1], bin_tris).
struct SurfaceDev {
    const double* v;
    const int32_t* tri;
    const int32_t* bin_start;
    const int32_t* bin_tris;
    const float2* bin_uv;  // per registration: the triangle's three vertices in the projection plane, FP32
    int64_t nv, nt;
    int32_t ax[3];  // the ray's axis (the shortest of the surface's box, the first on a tie), then the plane's two
    float mag;      // the surface box's largest coordinate magnitude (scale of the FP32 screen's bound)
    int32_t nb[2];
    double lo[2], inv_w[2];
    double bmin[3], bmax[3];
};

// host: fills S's box and bins, the CSR in start / tris; returns the number of registrations
int64_t surface_bins(const double* v, int64_t nv, const int32_t* tri, int64_t nt, SurfaceDev& S,
                     std::vector<int32_t>& start, std::vector<int32_t>& tris, std::vector<float>* uv = nullptr);
cudaError_t launch_hole_cut(const SurfaceDev& S, const GridDev& target, const MotionDev& mt, const MotionDev& mb,
                            const int32_t* nodes, int64_t n, uint8_t* iblank, int32_t* err, int nsm, cudaStream_t st);

}  // namespace ovs
