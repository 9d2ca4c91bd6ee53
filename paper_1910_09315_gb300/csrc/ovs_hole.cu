// Hole cutting (Sec. 2.2.1): the nodes of a grid that lie inside a moving body's closed triangulated surface are
// blanked.  A point is inside iff a ray from it along the surface's shortest box axis r crosses the surface an odd
// number of times (with (u, w) the axes that follow r cyclically; below, x / y / z name r / u / w).  A triangle
// is crossed when the point's (y, z) lies in its projection on the y-z plane (edge functions in FP64, a point on
// a projected edge belonging to the one triangle whose counter-clockwise edge runs downward, or level toward -y)
// and the crossing lies strictly ahead in x.  Every FP64 operation is one rounding (no fused
// multiply-add: the _rn intrinsics), so the decision is reproducible.  The triangles are registered in a uniform
// grid of bins over the surface's projected box; a point tests only its bin's triangles, each decided in FP32
// where an error bound (proven below) shows what the FP64 test would answer, and by the FP64 test otherwise.
#include "ovs_hole.cuh"

#include <cstring>

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

// target-grid position -> body frame, x_b = M x + t: in FP32 from the coordinates' high parts for a first
// rejection against the surface box widened by the FP32 error bound (lo, hi), and as FP32 pairs (X) for the rest
struct HoleXf {
    XfFF X;
    float M[9], t[3], lo[3], hi[3];
    float blo[3], bhi[3];  // the surface's box widened by kBinMargin * mag, in FP32 (the pair-precision test)
    __device__ __forceinline__ float3 apply(float x, float y, float z) const {
        return make_float3(fmaf(M[0], x, fmaf(M[1], y, fmaf(M[2], z, t[0]))),
                           fmaf(M[3], x, fmaf(M[4], y, fmaf(M[5], z, t[1]))),
                           fmaf(M[6], x, fmaf(M[7], y, fmaf(M[8], z, t[2]))));
    }
};

// The FP32 edge function dy ez - dz ey of (y0, z0) -> (y1, z1) at (y2, z2), and a bound on its distance from the
// exact value of the same function at the FP64 inputs (returned in err).  The FP32 inputs are the FP64 values
// rounded (each within u |c| <= u mag, u = 2^-24, every coordinate and the point being <= mag in size), so a
// computed difference d' of two of them is within D = 4 u mag of the exact difference d, a product d1' d2' within
// D (|d1| + |d2|) + D^2 + u |d1 d2|, and the edge function (with or without a fused multiply-add) within
// D (|dy| + |ez| + |dz| + |ey|) + 2 D^2 + 2 u (|dy ez| + |dz ey|); the FP64 test's own rounding adds a few 1e-16
// (|dy ez| + |dz ey|).  The bound 4e-6 (mag (|dy| + |dz| + |ey| + |ez|) + |dy ez| + |dz ey|) + 1e-12 mag^2
// exceeds all of it by a factor of at least 8.
__device__ __forceinline__ float edge_f32(float y0, float z0, float y1, float z1, float y2, float z2, float mag,
                                          float& err) {
    const float dy = y1 - y0, dz = z1 - z0, ey = y2 - y0, ez = z2 - z0;
    const float p0 = dy * ez, p1 = dz * ey;
    err = 4e-6f * (mag * (fabsf(dy) + fabsf(dz) + fabsf(ey) + fabsf(ez)) + fabsf(p0) + fabsf(p1)) + 1e-12f * mag * mag;
    return p0 - p1;
}

enum Screen { kMissed = 0, kCrossed = 1, kUnsure = 2 };

// FP32 decision of the FP64 test for one triangle (plane coordinates A, B, C; ray-axis coordinates r of A, B, C
// loaded on demand), or kUnsure.  With w0, w1, w2 the edge functions of B->C, C->A, A->B at the point q and s the
// sign of the projected area:
//  * area certain (|area| > its bound): the FP64 test has the same orientation; it misses if some s w_i is below
//    minus its bound, and if every s w_i is above its bound the point is strictly inside (no edge ownership), and
//    crossed iff s (w0 (A.r - q.r) + w1 (B.r - q.r) + w2 (C.r - q.r)) > 0 -- the FP64 comparison of the crossing
//    with the point along r, up to a positive factor -- when that sum exceeds its bound: each w_i is within e_i
//    / 8, each FP32 difference within 4 u mag, and the FP32 and FP64 sums' rounding within 3 u of the sum of the
//    terms' sizes, so e_i (|d_i| + 4e-6 mag) + 4e-6 |w_i| (mag + |d_i|) per term bounds the distance;
//  * area unsure: some w_i below minus its bound and some w_j above its bound means outside for either
//    orientation (and an FP64 area of 0 is never crossed).
__device__ __forceinline__ int screen(float4 g0, float4 g1, const float4* __restrict__ tri_r, float qy, float qz,
                                      float qr, float mag) {
    float ea, e0, e1, e2;
    const float area = edge_f32(g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, mag, ea);
    const float w0 = edge_f32(g0.z, g0.w, g1.x, g1.y, qy, qz, mag, e0);
    const float w1 = edge_f32(g1.x, g1.y, g0.x, g0.y, qy, qz, mag, e1);
    const float w2 = edge_f32(g0.x, g0.y, g0.z, g0.w, qy, qz, mag, e2);
    if (!(fabsf(area) > ea)) {
        const bool neg = w0 < -e0 || w1 < -e1 || w2 < -e2, pos = w0 > e0 || w1 > e1 || w2 > e2;
        return neg && pos ? kMissed : kUnsure;
    }
    const float s = area > 0 ? 1.f : -1.f;
    const float s0 = s * w0, s1 = s * w1, s2 = s * w2;
    if (s0 < -e0 || s1 < -e1 || s2 < -e2) return kMissed;
    if (!(s0 > e0 && s1 > e1 && s2 > e2)) return kUnsure;
    const float4 r = __ldg(tri_r + __float_as_int(g1.z));
    const float d0 = r.x - qr, d1 = r.y - qr, d2 = r.z - qr;
    const float D = s * (w0 * d0 + w1 * d1 + w2 * d2);
    const float eD = e0 * (fabsf(d0) + 4e-6f * mag) + e1 * (fabsf(d1) + 4e-6f * mag) + e2 * (fabsf(d2) + 4e-6f * mag) +
                     4e-6f * (fabsf(w0) * (mag + fabsf(d0)) + fabsf(w1) * (mag + fabsf(d1)) + fabsf(w2) * (mag + fabsf(d2)));
    if (D > eD) return kCrossed;
    if (D < -eD) return kMissed;
    return kUnsure;
}

// A point's bin in FP32.  The FP32 point is within u mag of the pair-precision one and the map's own rounding
// moves it by a few u mag more, far inside the margin (1e-5 mag) by which each triangle's projected box was
// widened when it was registered: every triangle whose box holds the point is in the point's bin.
__device__ __forceinline__ int64_t bin_of_point(const SurfaceDev& S, float qy, float qz) {
    int by = (int)floorf((qy - S.lo_f[0]) * S.inv_w_f[0]);
    int bz = (int)floorf((qz - S.lo_f[1]) * S.inv_w_f[1]);
    by = min(max(by, 0), S.nb[0] - 1);
    bz = min(max(bz, 0), S.nb[1] - 1);
    return by + (int64_t)S.nb[0] * bz;
}

// What the registration loop reads of a surface, held in registers for the loop (the surface itself sits in the
// kernel's parameters, picked by a runtime index).
struct SurfHot {
    const float4* __restrict__ rec;
    const float4* __restrict__ tri_r;
    const int32_t* __restrict__ tri;
    const double* __restrict__ v;
    float mag;
    int ar, au, aw;
};

// The candidate node in the body frame in FP64, by the frame maps' fixed order of operations (to_inertial of the
// target grid's motion, then to_body of the body's): the point every FP64 test decides on, computed on first use.
struct Exact64 {
    const GridDev* tg;
    const MotionDev* mt;
    const MotionDev* mb;
    int64_t node;
    int ar, au, aw;
    bool have;
    double p[3];
    __device__ __forceinline__ const double* get() {
        if (!have) {
            const double3 x = make_double3(__ldg(tg->x + node), __ldg(tg->y + node), __ldg(tg->z + node));
            const double3 b = to_body(*mb, to_inertial(*mt, x));
            const double q[3] = {b.x, b.y, b.z};
            p[0] = q[ar];
            p[1] = q[au];
            p[2] = q[aw];
            have = true;
        }
        return p;
    }
};

// The point (pr along the ray; pu, pw in the plane; FP32 pairs) against registration e: the FP32 decision (its
// bound covers the pairs' distance to the FP64 point, about 1e-14 relative), else the FP64 test at the FP64 point.
__device__ __forceinline__ int crosses(const SurfHot& H, int32_t e, ff pr, ff pu, ff pw, Exact64& x64) {
    const float4 g0 = __ldg(H.rec + 2 * (int64_t)e), g1 = __ldg(H.rec + 2 * (int64_t)e + 1);
    const int sc = screen(g0, g1, H.tri_r, pu.hi, pw.hi, pr.hi, H.mag);
    if (sc != kUnsure) return sc;
    const int32_t t = __float_as_int(g1.z);
    const int32_t i0 = __ldg(H.tri + 3 * t), i1 = __ldg(H.tri + 3 * t + 1), i2 = __ldg(H.tri + 3 * t + 2);
    const double A[3] = {__ldg(H.v + 3 * i0 + H.ar), __ldg(H.v + 3 * i0 + H.au), __ldg(H.v + 3 * i0 + H.aw)};
    const double B[3] = {__ldg(H.v + 3 * i1 + H.ar), __ldg(H.v + 3 * i1 + H.au), __ldg(H.v + 3 * i1 + H.aw)};
    const double C[3] = {__ldg(H.v + 3 * i2 + H.ar), __ldg(H.v + 3 * i2 + H.au), __ldg(H.v + 3 * i2 + H.aw)};
    const double* p = x64.get();
    return ray_crosses(A, B, C, p[0], p[1], p[2]);
}

constexpr int kHoleThreads = 256;
constexpr int kHeavyBin = 32;  // a point whose bin holds more registrations is tested by its whole warp

// Several surfaces cutting one target grid in one launch: surface s's candidates fill groups of 32 lanes
// group_begin[s] .. group_begin[s + 1] (its last group ragged), and the groups are dealt to the warps round-robin,
// so that every warp gets a share of every surface's (spatially clustered) heavy points.
struct HoleBatch {
    int32_t nsurf;
    int32_t pad;
    int64_t group_begin[OVS_MAX_GRIDS + 1];
    int64_t n[OVS_MAX_GRIDS];
    const int32_t* nodes[OVS_MAX_GRIDS];
    SurfaceDev S[OVS_MAX_GRIDS];
    HoleXf F[OVS_MAX_GRIDS];
    MotionDev mt;                 // the target grid's motion
    MotionDev mb[OVS_MAX_GRIDS];  // each surface's body motion
};
static_assert(sizeof(HoleBatch) + sizeof(GridDev) + 16 <= 32764, "kernel parameters exceed the 32764-byte limit");

// One lane per candidate node: the node's position in the body frame as FP32 pairs p (about 1e-14 relative),
// then its bin's registrations, each decided in FP32 and, where that is unsure, tested in FP64 at the point
// hi + lo of p.  The parity is that of every triangle the FP64 test crosses at that point: a triangle outside
// the bin has its box further than the margin from the point, and a point further than the margin outside the
// surface's box is outside the body.  FP64 (slow on this GPU) runs only in those unsure tests.  A point in a bin
// with more than kHeavyBin registrations (near a pole, where many triangles meet) is tested by all 32 lanes of its
// warp, a registration per lane, the parity a ballot's popcount: such bins would otherwise set the kernel's tail.
// Every lane of a warp works on the same group, so that all of them reach the ballots.
__global__ void __launch_bounds__(kHoleThreads) k_hole_cut(const __grid_constant__ HoleBatch P, GridDev tg,
                                                           uint8_t* __restrict__ iblank, int32_t* __restrict__ err) {
    const int lane = threadIdx.x & 31;
    const int64_t nn = tg.nnodes;
    const int64_t groups = P.group_begin[P.nsurf];
    const int64_t warps = (int64_t)gridDim.x * (kHoleThreads / 32);
    int si = 0;  // the surface of group gi (gi only grows: the search moves forward)
    for (int64_t gi = (blockIdx.x * (int64_t)kHoleThreads + threadIdx.x) >> 5; gi < groups; gi += warps) {
        while (si + 1 < P.nsurf && P.group_begin[si + 1] <= gi) ++si;  // warp-uniform
        const SurfaceDev& S = P.S[si];
        const HoleXf& F = P.F[si];
        const int ar = S.ax[0], au = S.ax[1], aw = S.ax[2];
        const int64_t q = (gi - P.group_begin[si]) * 32 + lane;
        const int32_t* __restrict__ nodes = P.nodes[si];
        int64_t node = -1;
        bool work = false;
        ff pr = {0.f, 0.f}, pu = {0.f, 0.f}, pw = {0.f, 0.f};
        int32_t e0 = 0, e1 = 0;
        if (q < P.n[si]) {
            node = nodes ? (int64_t)__ldg(nodes + q) : q;
            if (node < 0 || node >= nn) {
                atomicOr(err, kErrBadNode);
            } else {
                // first rejection from the coordinates' high parts alone (most candidates end here): further
                // than the FP32 error bound outside the surface's box
                const float xh = __ldg(tg.xff + node), yh = __ldg(tg.xff + 2 * nn + node),
                            zh = __ldg(tg.xff + 4 * nn + node);
                const float3 pf = F.apply(xh, yh, zh);
                work = !(pf.x < F.lo[0] || pf.x > F.hi[0] || pf.y < F.lo[1] || pf.y > F.hi[1] || pf.z < F.lo[2] ||
                         pf.z > F.hi[2]);
                if (work) {
                    const ff x[3] = {{xh, __ldg(tg.xff + nn + node)},
                                     {yh, __ldg(tg.xff + 3 * nn + node)},
                                     {zh, __ldg(tg.xff + 5 * nn + node)}};
                    ff pb[3];
                    xf_apply(F.X, x, pb);
#pragma unroll
                    for (int c = 0; c < 3; ++c) work = work && !(pb[c].hi < F.blo[c] || pb[c].hi > F.bhi[c]);
                    auto pick = [&pb](int c) { return c == 0 ? pb[0] : (c == 1 ? pb[1] : pb[2]); };  // registers
                    pr = pick(ar);
                    pu = pick(au);
                    pw = pick(aw);
                }
                if (work) {
                    const int64_t b = bin_of_point(S, pu.hi, pw.hi);
                    e0 = __ldg(S.bin_start + b);
                    e1 = __ldg(S.bin_start + b + 1);
                }
            }
        }
        const bool heavy = work && e1 - e0 > kHeavyBin;
        int odd = 0;
        if (!__any_sync(0xffffffffu, work)) continue;  // (warp-uniform)
        const SurfHot H = {S.bin_rec, S.tri_r, S.tri, S.v, S.mag, ar, au, aw};
        if (work && !heavy) {
            Exact64 x64 = {&tg, &P.mt, &P.mb[si], node, ar, au, aw, false, {0.0, 0.0, 0.0}};
#pragma unroll 4
            for (int32_t e = e0; e < e1; ++e) odd ^= crosses(H, e, pr, pu, pw, x64);
        }
        // the heavy points of this warp, one after another, each over all lanes
        for (unsigned hm = __ballot_sync(0xffffffffu, heavy); hm; hm &= hm - 1) {
            const int l = __ffs(hm) - 1;
            const int32_t h0 = __shfl_sync(0xffffffffu, e0, l), h1 = __shfl_sync(0xffffffffu, e1, l);
            const ff hr = {__shfl_sync(0xffffffffu, pr.hi, l), __shfl_sync(0xffffffffu, pr.lo, l)};
            const ff hu = {__shfl_sync(0xffffffffu, pu.hi, l), __shfl_sync(0xffffffffu, pu.lo, l)};
            const ff hw = {__shfl_sync(0xffffffffu, pw.hi, l), __shfl_sync(0xffffffffu, pw.lo, l)};
            Exact64 x64 = {&tg, &P.mt, &P.mb[si], (int64_t)__shfl_sync(0xffffffffu, (long long)node, l), ar, au, aw,
                           false, {0.0, 0.0, 0.0}};
            int par = 0;
            for (int32_t e = h0 + lane; e < h1; e += 32) par ^= crosses(H, e, hr, hu, hw, x64);
            const unsigned bits = __ballot_sync(0xffffffffu, par != 0);
            if (lane == l) odd = __popc(bits) & 1;
        }
        if (work && odd) iblank[node] = 0;
    }
}

}  // namespace

namespace {

// the body-frame map of one surface at the current motions: M = R_b^T R_t, t = R_b^T (c_t - c_b) composed in FP64;
// first-rejection box: the surface box widened by 1e-4 of the largest of its extent and the transformed
// magnitudes (far above the FP32 rounding of 3 products)
HoleXf hole_map(const SurfaceDev& S, const GridDev& target, const MotionDev& mt, const MotionDev& mb) {
    HoleXf F;
    memset(&F, 0, sizeof F);
    F.X.identity = mt.identity && mb.identity;
    double tmag = 0, ext = 0;
    auto split2 = [](double v, float& hi, float& lo) {
        hi = (float)v;
        lo = (float)(v - (double)hi);
    };
    for (int i = 0; i < 3; ++i) {
        double tv = 0;
        for (int k = 0; k < 3; ++k) {
            double m = 0;
            for (int j = 0; j < 3; ++j) m += (mb.identity ? (i == j) : mb.R[3 * j + i]) * (mt.identity ? (j == k) : mt.R[3 * j + k]);
            F.M[3 * i + k] = (float)m;
            split2(m, F.X.Mh[3 * i + k], F.X.Ml[3 * i + k]);
        }
        for (int j = 0; j < 3; ++j)
            tv += (mb.identity ? (i == j) : mb.R[3 * j + i]) * ((mt.identity ? 0.0 : mt.c[j]) - (mb.identity ? 0.0 : mb.c[j]));
        F.t[i] = (float)tv;
        split2(tv, F.X.th[i], F.X.tl[i]);
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
        F.blo[c] = (float)(S.bmin[c] - kBinMargin * S.mag);
        F.bhi[c] = (float)(S.bmax[c] + kBinMargin * S.mag);
    }
    return F;
}

}  // namespace

cudaError_t launch_hole_cut(const HoleJob* jobs, int njobs, const GridDev& target, const MotionDev& mt,
                            uint8_t* iblank, int32_t* err, int nsm, cudaStream_t st) {
    if (njobs > OVS_MAX_GRIDS) return cudaErrorInvalidValue;
    HoleBatch P;
    memset(&P, 0, sizeof P);
    int64_t g = 0;
    for (int j = 0; j < njobs; ++j) {
        if (jobs[j].n <= 0) continue;
        const int k = P.nsurf++;
        P.group_begin[k] = g;
        g += (jobs[j].n + 31) / 32;
        P.n[k] = jobs[j].n;
        P.nodes[k] = jobs[j].nodes;
        P.S[k] = *jobs[j].S;
        P.F[k] = hole_map(*jobs[j].S, target, mt, *jobs[j].mb);
        P.mb[k] = *jobs[j].mb;
    }
    P.group_begin[P.nsurf] = g;
    P.mt = mt;
    if (g == 0) return cudaSuccess;
    // one resident wave; the groups are dealt round-robin to its warps
    static int occ = 0;
    if (occ == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_hole_cut, kHoleThreads, 0);
        if (e != cudaSuccess || occ < 1) occ = 1;
    }
    const int64_t want = (g + kHoleThreads / 32 - 1) / (kHoleThreads / 32);
    const unsigned blocks = (unsigned)std::min<int64_t>(want, (int64_t)nsm * occ);
    k_hole_cut<<<blocks, kHoleThreads, 0, st>>>(P, target, iblank, err);
    return cudaGetLastError();
}

// Host: the bin grid of a surface (about one bin per triangle, shaped like the projected box), each triangle
// registered in every bin that its projected box, widened by the margin, overlaps, with its plane coordinates in
// FP32 and its id in the registration's record.
int64_t surface_bins(const double* v, int64_t nv, const int32_t* tri, int64_t nt, SurfaceDev& S,
                     std::vector<int32_t>& start, std::vector<int32_t>& tris, std::vector<float>* rec,
                     std::vector<float>* tr) {
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
        S.lo_f[d] = (float)S.lo[d];
        S.inv_w_f[d] = (float)S.inv_w[d];
    }
    const double reg_margin = kBinMargin * mag;
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
        lo0[t] = bin_of(0, mn[0] - reg_margin);
        hi0[t] = bin_of(0, mx[0] + reg_margin);
        lo1[t] = bin_of(1, mn[1] - reg_margin);
        hi1[t] = bin_of(1, mx[1] + reg_margin);
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
    if (rec) rec->assign((size_t)acc * 8, 0.f);
    if (tr) {
        tr->assign((size_t)nt * 4, 0.f);
        for (int64_t t = 0; t < nt; ++t)
            for (int k = 0; k < 3; ++k) (*tr)[4 * (size_t)t + k] = (float)v[3 * tri[3 * t + k] + S.ax[0]];
    }
    std::vector<int32_t> cursor(start.begin(), start.end() - 1);
    for (int64_t t = 0; t < nt; ++t)
        for (int b1 = lo1[t]; b1 <= hi1[t]; ++b1)
            for (int b0 = lo0[t]; b0 <= hi0[t]; ++b0) {
                const int32_t slot = cursor[b0 + (size_t)nb0 * b1]++;
                tris[slot] = (int32_t)t;
                if (rec) {
                    float* o = rec->data() + 8 * (size_t)slot;
                    for (int k = 0; k < 3; ++k) {
                        o[2 * k] = (float)v[3 * tri[3 * t + k] + S.ax[1]];
                        o[2 * k + 1] = (float)v[3 * tri[3 * t + k] + S.ax[2]];
                    }
                    const int32_t id = (int32_t)t;
                    std::memcpy(o + 6, &id, sizeof id);  // the triangle id, as its int bits
                }
            }
    return acc;
}

}  // namespace ovs
