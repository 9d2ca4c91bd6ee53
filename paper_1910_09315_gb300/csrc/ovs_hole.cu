// Hole cutting (Sec. 2.2.1): the nodes of a grid that lie inside a moving body's closed triangulated surface are
// blanked.  A point is inside iff a ray from it along the body frame's +x crosses the surface an odd number of
// times.  A triangle is crossed when the point's (y, z) lies in its projection on the y-z plane (edge functions
// in FP64, a point on a projected edge belonging to the one triangle whose counter-clockwise edge runs downward,
// or level toward -y) and the crossing lies strictly ahead in x.  Every FP64 operation is one rounding (no fused
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

__global__ void __launch_bounds__(256) k_hole_cut(SurfaceDev S, GridDev tg, MotionDev mt, MotionDev mb,
                                                  const int32_t* __restrict__ nodes, int64_t n,
                                                  uint8_t* __restrict__ iblank, int32_t* __restrict__ err) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t node = nodes ? (int64_t)__ldg(nodes + q) : q;
        if (node < 0 || node >= tg.nnodes) {
            atomicOr(err, kErrBadNode);
            continue;
        }
        const double3 x = make_double3(__ldg(tg.x + node), __ldg(tg.y + node), __ldg(tg.z + node));
        const double3 p = to_body(mb, to_inertial(mt, x));
        if (!(p.x >= S.bmin[0] && p.x <= S.bmax[0] && p.y >= S.bmin[1] && p.y <= S.bmax[1] && p.z >= S.bmin[2] &&
              p.z <= S.bmax[2]))
            continue;  // outside the surface's box: outside the body
        int by = (int)floor((p.y - S.lo[0]) * S.inv_w[0]);
        int bz = (int)floor((p.z - S.lo[1]) * S.inv_w[1]);
        by = min(max(by, 0), S.nb[0] - 1);
        bz = min(max(bz, 0), S.nb[1] - 1);
        const int64_t b = by + (int64_t)S.nb[0] * bz;
        int odd = 0;
        for (int32_t r = __ldg(S.bin_start + b); r < __ldg(S.bin_start + b + 1); ++r) {
            const int32_t t = __ldg(S.bin_tris + r);
            const int32_t i0 = __ldg(S.tri + 3 * t), i1 = __ldg(S.tri + 3 * t + 1), i2 = __ldg(S.tri + 3 * t + 2);
            const double A[3] = {__ldg(S.v + 3 * i0), __ldg(S.v + 3 * i0 + 1), __ldg(S.v + 3 * i0 + 2)};
            const double B[3] = {__ldg(S.v + 3 * i1), __ldg(S.v + 3 * i1 + 1), __ldg(S.v + 3 * i1 + 2)};
            const double C[3] = {__ldg(S.v + 3 * i2), __ldg(S.v + 3 * i2 + 1), __ldg(S.v + 3 * i2 + 2)};
            odd ^= ray_crosses(A, B, C, p.x, p.y, p.z);
        }
        if (odd) iblank[node] = 0;
    }
}

}  // namespace

cudaError_t launch_hole_cut(const SurfaceDev& S, const GridDev& target, const MotionDev& mt, const MotionDev& mb,
                            const int32_t* nodes, int64_t n, uint8_t* iblank, int32_t* err, int nsm, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t want = (n + 255) / 256;
    const unsigned blocks = (unsigned)std::min<int64_t>(want, (int64_t)nsm * 8);
    k_hole_cut<<<blocks, 256, 0, st>>>(S, target, mt, mb, nodes, n, iblank, err);
    return cudaGetLastError();
}

// Host: the bin grid of a surface (about 8 triangles a bin), each triangle registered in every bin its projected
// box overlaps, widened by one bin on each side (so that the device's bin of a point always lists every triangle
// whose projection can hold it).
int64_t surface_bins(const double* v, int64_t nv, const int32_t* tri, int64_t nt, SurfaceDev& S,
                     std::vector<int32_t>& start, std::vector<int32_t>& tris) {
    for (int c = 0; c < 3; ++c) {
        S.bmin[c] = 1e300;
        S.bmax[c] = -1e300;
    }
    for (int64_t i = 0; i < nv; ++i)
        for (int c = 0; c < 3; ++c) {
            S.bmin[c] = std::min(S.bmin[c], v[3 * i + c]);
            S.bmax[c] = std::max(S.bmax[c], v[3 * i + c]);
        }
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(1024, (int64_t)std::sqrt((double)nt / 8.0)));
    for (int d = 0; d < 2; ++d) {
        S.nb[d] = nb;
        S.lo[d] = S.bmin[1 + d];
        const double ext = S.bmax[1 + d] - S.bmin[1 + d];
        S.inv_w[d] = ext > 0 ? nb / ext : 0.0;
    }
    auto bin_of = [&](int d, double x) {
        int b = (int)std::floor((x - S.lo[d]) * S.inv_w[d]);
        return std::min(std::max(b, 0), S.nb[d] - 1);
    };
    std::vector<int> lo0(nt), hi0(nt), lo1(nt), hi1(nt);
    std::vector<int64_t> count((size_t)nb * nb + 1, 0);
    for (int64_t t = 0; t < nt; ++t) {
        double mn[2] = {1e300, 1e300}, mx[2] = {-1e300, -1e300};
        for (int k = 0; k < 3; ++k)
            for (int d = 0; d < 2; ++d) {
                mn[d] = std::min(mn[d], v[3 * tri[3 * t + k] + 1 + d]);
                mx[d] = std::max(mx[d], v[3 * tri[3 * t + k] + 1 + d]);
            }
        lo0[t] = std::max(0, bin_of(0, mn[0]) - 1);
        hi0[t] = std::min(nb - 1, bin_of(0, mx[0]) + 1);
        lo1[t] = std::max(0, bin_of(1, mn[1]) - 1);
        hi1[t] = std::min(nb - 1, bin_of(1, mx[1]) + 1);
        for (int b1 = lo1[t]; b1 <= hi1[t]; ++b1)
            for (int b0 = lo0[t]; b0 <= hi0[t]; ++b0) ++count[b0 + (int64_t)nb * b1];
    }
    start.assign((size_t)nb * nb + 1, 0);
    int64_t acc = 0;
    for (int64_t b = 0; b < (int64_t)nb * nb; ++b) {
        start[b] = (int32_t)acc;
        acc += count[b];
    }
    start[(size_t)nb * nb] = (int32_t)acc;
    tris.assign((size_t)acc, 0);
    std::vector<int32_t> cursor(start.begin(), start.end() - 1);
    for (int64_t t = 0; t < nt; ++t)
        for (int b1 = lo1[t]; b1 <= hi1[t]; ++b1)
            for (int b0 = lo0[t]; b0 <= hi0[t]; ++b0) tris[cursor[b0 + (size_t)nb * b1]++] = (int32_t)t;
    return acc;
}

}  // namespace ovs
