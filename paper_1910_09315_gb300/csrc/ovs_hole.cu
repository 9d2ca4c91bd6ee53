// Hole cutting (Sec. 2.2.1): the nodes of a grid that lie inside a moving body's closed triangulated surface are
// blanked.  A point is inside iff a ray from it along the surface's shortest box axis r crosses the surface an odd
// number of times (with (u, w) the axes that follow r cyclically; below, x / y / z name r / u / w).  A triangle
// is crossed when the point's (y, z) lies in its projection on the y-z plane (edge functions in FP64, a point on
// a projected edge belonging to the one triangle whose counter-clockwise edge runs downward, or level toward -y)
// and the crossing lies strictly ahead in x.  Every FP64 operation is one rounding (no fused
// multiply-add: the _rn intrinsics), so the decision is reproducible.  The triangles are registered in a uniform
// grid of bins over the surface's projected box; a point tests only its bin's triangles.
#include "ovs_hole.cuh"

namespace ovs {

namespace {

__device__ __forceinline__ double edge2(double ay, double az, double by, double bz, double py, double pz) {
    return __dsub_rn(__dmul_rn(__dsub_rn(by, ay), __dsub_rn(pz, az)), __dmul_rn(__dsub_rn(bz, az), __dsub_rn(py, ay)));
}

__device__ __forceinline__ bool edge_owns(double ay, double az, double by, double bz) {
    return (bz < az) || (bz == az && by < ay);
}

__device__ __forceinline__ int ray_crosses(const double* A, const double* B, const double* C, double px, double py,
                                           double pz) {
    const double area = edge2(A[1], A[2], B[1], B[2], C[1], C[2]);
    if (area == 0.0) return 0;
    const double* a = A;
    const double* b = area > 0 ? B : C;
    const double* c = area > 0 ? C : B;
    const double w0 = edge2(b[1], b[2], c[1], c[2], py, pz);
    const double w1 = edge2(c[1], c[2], a[1], a[2], py, pz);
    const double w2 = edge2(a[1], a[2], b[1], b[2], py, pz);
    if (w0 < 0 || w1 < 0 || w2 < 0) return 0;
    if (w0 == 0 && !edge_owns(b[1], b[2], c[1], c[2])) return 0;
    if (w1 == 0 && !edge_owns(c[1], c[2], a[1], a[2])) return 0;
    if (w2 == 0 && !edge_owns(a[1], a[2], b[1], b[2])) return 0;
    const double s = __dadd_rn(__dadd_rn(w0, w1), w2);
    const double xs = __dadd_rn(__dadd_rn(__dmul_rn(w0, a[0]), __dmul_rn(w1, b[0])), __dmul_rn(w2, c[0]));
    return xs > __dmul_rn(px, s) ? 1 : 0;
}

// target-grid position -> body frame in FP32 (x_b = M x + t), and the surface box widened by the FP32 error bound
struct HoleF32 {
    float M[9], t[3], lo[3], hi[3];
    __device__ __forceinline__ float3 apply(float x, float y, float z) const {
        return make_float3(fmaf(M[0], x, fmaf(M[1], y, fmaf(M[2], z, t[0]))),
                           fmaf(M[3], x, fmaf(M[4], y, fmaf(M[5], z, t[1]))),
                           fmaf(M[6], x, fmaf(M[7], y, fmaf(M[8], z, t[2]))));
    }
};

// FP32 screen of one triangle (plane coordinates (y, z) of A, B, C and of the point): true when the FP64 test
// can only say "not crossed" -- the projected triangle's orientation is certain and the point lies outside one
// of its edges by more than the FP32 error bound.  With every coordinate of magnitude <= mag, the inputs' FP32
// rounding moves a difference by <= 1.2e-7 mag and the products round by <= 6e-8 of their size; the bound
// 1e-5 ((|dy| + mag)(|ez| + mag) + (|dz| + mag)(|ey| + mag)) exceeds both by a factor of about 80.
__device__ __forceinline__ bool surely_missed(const float* A, const float* B, const float* C, float qy, float qz,
                                              float mag) {
    const float ay = A[1], az = A[2], by = B[1], bz = B[2], cy = C[1], cz = C[2];
    auto e = [mag](float y0, float z0, float y1, float z1, float y2, float z2, float& err) {
        const float dy = y1 - y0, dz = z1 - z0, ey = y2 - y0, ez = z2 - z0;
        err = 1e-5f * ((fabsf(dy) + mag) * (fabsf(ez) + mag) + (fabsf(dz) + mag) * (fabsf(ey) + mag));
        return dy * ez - dz * ey;
    };
    float ea, e0, e1, e2;
    const float area = e(ay, az, by, bz, cy, cz, ea);
    if (!(fabsf(area) > ea)) return false;  // orientation unsure: decide in FP64
    const float s = area > 0 ? 1.f : -1.f;   // counter-clockwise order: the point inside has every s * w >= 0
    const float w0 = e(by, bz, cy, cz, qy, qz, e0), w1 = e(cy, cz, ay, az, qy, qz, e1), w2 = e(ay, az, by, bz, qy, qz, e2);
    return s * w0 < -e0 || s * w1 < -e1 || s * w2 < -e2;
}

__global__ void __launch_bounds__(256) k_hole_cut(SurfaceDev S, HoleF32 F, GridDev tg, MotionDev mt, MotionDev mb,
                                                  const int32_t* __restrict__ nodes, int64_t n,
                                                  uint8_t* __restrict__ iblank, int32_t* __restrict__ err) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t node = nodes ? (int64_t)__ldg(nodes + q) : q;
        if (node < 0 || node >= tg.nnodes) {
            atomicOr(err, kErrBadNode);
            continue;
        }
        {
            // FP32 pre-rejection from the grid's FP32 coordinates (FP64 is slow on this GPU): a point further than
            // 1e-4 (relative to its size and the box's) outside the surface's box in FP32 lies outside it in FP64
            const int64_t nn = tg.nnodes;
            const float3 pf = F.apply(__ldg(tg.xff + node), __ldg(tg.xff + 2 * nn + node), __ldg(tg.xff + 4 * nn + node));
            bool out = false;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float v = c == 0 ? pf.x : (c == 1 ? pf.y : pf.z);
                out = out || v < F.lo[c] || v > F.hi[c];
            }
            if (out) continue;
        }
        const double3 x = make_double3(__ldg(tg.x + node), __ldg(tg.y + node), __ldg(tg.z + node));
        const double3 p3 = to_body(mb, to_inertial(mt, x));
        if (!(p3.x >= S.bmin[0] && p3.x <= S.bmax[0] && p3.y >= S.bmin[1] && p3.y <= S.bmax[1] && p3.z >= S.bmin[2] &&
              p3.z <= S.bmax[2]))
            continue;  // outside the surface's box: outside the body
        const double pa[3] = {p3.x, p3.y, p3.z};
        const int ar = S.ax[0], au = S.ax[1], aw = S.ax[2];
        const double3 p = make_double3(pa[ar], pa[au], pa[aw]);  // (ray axis, plane axes)
        int by = (int)floor((p.y - S.lo[0]) * S.inv_w[0]);
        int bz = (int)floor((p.z - S.lo[1]) * S.inv_w[1]);
        by = min(max(by, 0), S.nb[0] - 1);
        bz = min(max(bz, 0), S.nb[1] - 1);
        const int64_t b = by + (int64_t)S.nb[0] * bz;
        int odd = 0;
        const float qy = (float)p.y, qz = (float)p.z;
        for (int32_t e = __ldg(S.bin_start + b); e < __ldg(S.bin_start + b + 1); ++e) {
            const float2 ua = __ldg(S.bin_uv + 3 * (int64_t)e), ub = __ldg(S.bin_uv + 3 * (int64_t)e + 1),
                         uc = __ldg(S.bin_uv + 3 * (int64_t)e + 2);
            const float A32[3] = {0.f, ua.x, ua.y}, B32[3] = {0.f, ub.x, ub.y}, C32[3] = {0.f, uc.x, uc.y};
            if (surely_missed(A32, B32, C32, qy, qz, S.mag)) continue;
            const int32_t t = __ldg(S.bin_tris + e);
            const int32_t i0 = __ldg(S.tri + 3 * t), i1 = __ldg(S.tri + 3 * t + 1), i2 = __ldg(S.tri + 3 * t + 2);
            const double A[3] = {__ldg(S.v + 3 * i0 + ar), __ldg(S.v + 3 * i0 + au), __ldg(S.v + 3 * i0 + aw)};
            const double B[3] = {__ldg(S.v + 3 * i1 + ar), __ldg(S.v + 3 * i1 + au), __ldg(S.v + 3 * i1 + aw)};
            const double C[3] = {__ldg(S.v + 3 * i2 + ar), __ldg(S.v + 3 * i2 + au), __ldg(S.v + 3 * i2 + aw)};
            odd ^= ray_crosses(A, B, C, p.x, p.y, p.z);
        }
        if (odd) iblank[node] = 0;
    }
}

}  // namespace

cudaError_t launch_hole_cut(const SurfaceDev& S, const GridDev& target, const MotionDev& mt, const MotionDev& mb,
                            const int32_t* nodes, int64_t n, uint8_t* iblank, int32_t* err, int nsm, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    // the FP32 map composed in FP64 on the host: M = R_b^T R_t, t = R_b^T (c_t - c_b); margin: 1e-4 of the
    // largest of the box's extent and the transformed magnitudes (far above the FP32 rounding of 3 products)
    HoleF32 F;
    double tmag = 0, ext = 0;
    for (int i = 0; i < 3; ++i) {
        double tv = 0;
        for (int k = 0; k < 3; ++k) {
            double m = 0;
            for (int j = 0; j < 3; ++j) m += (mb.identity ? (i == j) : mb.R[3 * j + i]) * (mt.identity ? (j == k) : mt.R[3 * j + k]);
            F.M[3 * i + k] = (float)m;
        }
        for (int j = 0; j < 3; ++j)
            tv += (mb.identity ? (i == j) : mb.R[3 * j + i]) * ((mt.identity ? 0.0 : mt.c[j]) - (mb.identity ? 0.0 : mb.c[j]));
        F.t[i] = (float)tv;
        tmag = std::max(tmag, std::fabs(tv));
        ext = std::max(ext, S.bmax[i] - S.bmin[i]);
    }
    double xmag = 0;
    for (int c = 0; c < 3; ++c) xmag = std::max(xmag, std::max(std::fabs(S.bmin[c]), std::fabs(S.bmax[c])));
    double gmag = 0;  // the target grid's coordinate magnitude (its padded box)
    for (int c = 0; c < 3; ++c) gmag = std::max(gmag, std::max(std::fabs(target.lo[c]), std::fabs(target.hi[c])));
    const double margin = 1e-4 * (ext + xmag + tmag + gmag);
    for (int c = 0; c < 3; ++c) {
        F.lo[c] = (float)(S.bmin[c] - margin);
        F.hi[c] = (float)(S.bmax[c] + margin);
    }
    const int64_t want = (n + 255) / 256;
    const unsigned blocks = (unsigned)std::min<int64_t>(want, (int64_t)nsm * 8);
    k_hole_cut<<<blocks, 256, 0, st>>>(S, F, target, mt, mb, nodes, n, iblank, err);
    return cudaGetLastError();
}

// Host: the bin grid of a surface (about one bin per triangle, shaped like the projected box), each triangle
// registered in every bin its projected box overlaps, with its plane coordinates in FP32 beside it (uv).  The device maps a point to its bin by the same IEEE operations (subtract, multiply, floor), and
// that map is monotone, so a point inside a triangle's box always falls in one of the triangle's bins.
int64_t surface_bins(const double* v, int64_t nv, const int32_t* tri, int64_t nt, SurfaceDev& S,
                     std::vector<int32_t>& start, std::vector<int32_t>& tris, std::vector<float>* uv) {
    for (int c = 0; c < 3; ++c) {
        S.bmin[c] = 1e300;
        S.bmax[c] = -1e300;
    }
    for (int64_t i = 0; i < nv; ++i)
        for (int c = 0; c < 3; ++c) {
            S.bmin[c] = std::min(S.bmin[c], v[3 * i + c]);
            S.bmax[c] = std::max(S.bmax[c], v[3 * i + c]);
        }
    int r = 0;
    for (int c = 1; c < 3; ++c)
        if (S.bmax[c] - S.bmin[c] < S.bmax[r] - S.bmin[r]) r = c;
    S.ax[0] = r;
    S.ax[1] = (r + 1) % 3;
    S.ax[2] = (r + 2) % 3;
    double mag = 0;
    for (int c = 0; c < 3; ++c) mag = std::max(mag, std::max(std::fabs(S.bmin[c]), std::fabs(S.bmax[c])));
    S.mag = (float)mag;
    // about one bin per triangle, shaped like the projected box
    const double e0 = std::max(S.bmax[S.ax[1]] - S.bmin[S.ax[1]], 1e-300),
                 e1 = std::max(S.bmax[S.ax[2]] - S.bmin[S.ax[2]], 1e-300);
    S.nb[0] = (int)std::max<double>(1.0, std::min<double>(4096.0, std::floor(std::sqrt((double)nt * e0 / e1))));
    S.nb[1] = (int)std::max<double>(1.0, std::min<double>(4096.0, std::floor((double)nt / S.nb[0])));
    for (int d = 0; d < 2; ++d) {
        S.lo[d] = S.bmin[S.ax[1 + d]];
        const double ext = S.bmax[S.ax[1 + d]] - S.bmin[S.ax[1 + d]];
        S.inv_w[d] = ext > 0 ? S.nb[d] / ext : 0.0;
    }
    const int nb0 = S.nb[0], nb1 = S.nb[1];
    auto bin_of = [&](int d, double x) {
        int b = (int)std::floor((x - S.lo[d]) * S.inv_w[d]);
        return std::min(std::max(b, 0), S.nb[d] - 1);
    };
    std::vector<int> lo0(nt), hi0(nt), lo1(nt), hi1(nt);
    std::vector<int64_t> count((size_t)nb0 * nb1 + 1, 0);
    for (int64_t t = 0; t < nt; ++t) {
        double mn[2] = {1e300, 1e300}, mx[2] = {-1e300, -1e300};
        for (int k = 0; k < 3; ++k)
            for (int d = 0; d < 2; ++d) {
                mn[d] = std::min(mn[d], v[3 * tri[3 * t + k] + S.ax[1 + d]]);
                mx[d] = std::max(mx[d], v[3 * tri[3 * t + k] + S.ax[1 + d]]);
            }
        lo0[t] = bin_of(0, mn[0]);
        hi0[t] = bin_of(0, mx[0]);
        lo1[t] = bin_of(1, mn[1]);
        hi1[t] = bin_of(1, mx[1]);
        for (int b1 = lo1[t]; b1 <= hi1[t]; ++b1)
            for (int b0 = lo0[t]; b0 <= hi0[t]; ++b0) ++count[b0 + (int64_t)nb0 * b1];
    }
    start.assign((size_t)nb0 * nb1 + 1, 0);
    int64_t acc = 0;
    for (int64_t b = 0; b < (int64_t)nb0 * nb1; ++b) {
        start[b] = (int32_t)acc;
        acc += count[b];
    }
    start[(size_t)nb0 * nb1] = (int32_t)acc;
    tris.assign((size_t)acc, 0);
    if (uv) uv->assign((size_t)acc * 6, 0.f);
    std::vector<int32_t> cursor(start.begin(), start.end() - 1);
    for (int64_t t = 0; t < nt; ++t)
        for (int b1 = lo1[t]; b1 <= hi1[t]; ++b1)
            for (int b0 = lo0[t]; b0 <= hi0[t]; ++b0) {
                const int32_t slot = cursor[b0 + (size_t)nb0 * b1]++;
                tris[slot] = (int32_t)t;
                if (uv)
                    for (int k = 0; k < 3; ++k) {
                        (*uv)[6 * (size_t)slot + 2 * k] = (float)v[3 * tri[3 * t + k] + S.ax[1]];
                        (*uv)[6 * (size_t)slot + 2 * k + 1] = (float)v[3 * tri[3 * t + k] + S.ax[2]];
                    }
            }
    return acc;
}

}  // namespace ovs
