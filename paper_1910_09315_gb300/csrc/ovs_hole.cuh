// Hole cutting against closed triangulated body surfaces (see ovs_hole.cu).
#pragma once
#include <algorithm>
#include <cmath>
#include <vector>

#include "ovs_internal.cuh"

namespace ovs {

// A surface in the device workspace: vertices (body frame of its grid, FP64, xyz per vertex), triangles (3 vertex
// ids each), and the bins of the projected box (CSR over registrations: bin_start[nb0 * nb1 + 1]).  A registration
// is 32 bytes, bin_rec[2 e] = (A.u, A.w, B.u, B.w) and bin_rec[2 e + 1] = (C.u, C.w, triangle id as int bits, 0):
// the triangle's vertices in the projection plane in FP32, then its id; tri_r[t] = (A.r, B.r, C.r, 0) in FP32.
constexpr double kBinMargin = 1e-5;  // a triangle's projected box is widened by kBinMargin * mag

struct SurfaceDev {
    const double* v;
    const int32_t* tri;
    const int32_t* bin_start;
    const float4* bin_rec;
    const float4* tri_r;
    int64_t nv, nt;
    int32_t ax[3];  // the ray's axis (the shortest of the surface's box, the first on a tie), then the plane's two
    float mag;      // the surface box's largest coordinate magnitude (scale of the FP32 screen's bound)
    int32_t nb[2];
    double lo[2], inv_w[2];     // bin of plane coordinate c along d: floor((c - lo[d]) * inv_w[d]), clamped
    float lo_f[2], inv_w_f[2];  // the same map in FP32 (the device's; triangles are registered with a margin)
    double bmin[3], bmax[3];
};

// host: fills S's box and bins, the CSR in start / tris; returns the number of registrations.  A triangle is
// registered in every bin that its projected box, widened by kBinMargin * mag, overlaps.
// With rec / tr given, also the registrations' 32-byte records (8 floats each) and the triangles' FP32 ray-axis
// coordinates (4 floats each) in the device layout.
int64_t surface_bins(const double* v, int64_t nv, const int32_t* tri, int64_t nt, SurfaceDev& S,
                     std::vector<int32_t>& start, std::vector<int32_t>& tris, std::vector<float>* rec = nullptr,
                     std::vector<float>* tr = nullptr);
// one surface's share of a hole-cutting launch: the surface, its body grid's motion, its candidate nodes (device,
// NULL: nodes 0 .. n-1 of the target grid)
struct HoleJob {
    const SurfaceDev* S;
    const MotionDev* mb;
    const int32_t* nodes;
    int64_t n;
};
// at most OVS_MAX_GRIDS jobs, all cutting the target grid (motion mt) in one launch
cudaError_t launch_hole_cut(const HoleJob* jobs, int njobs, const GridDev& target, const MotionDev& mt,
                            uint8_t* iblank, int32_t* err, int nsm, cudaStream_t st);

}  // namespace ovs
