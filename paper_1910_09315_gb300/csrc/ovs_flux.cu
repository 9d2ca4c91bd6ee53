// Contravariant fluxes at the receivers and the mass-conservation correction over closed interfaces.
//
//   Sec. 2.1 eq. "flux": U^r = u_q xi^r_q / J, the velocity dotted with the area vector of a face of constant xi^r.
//   On the structured grid a face is a quadrilateral of four nodes; its area vector is half the cross product of
//   its diagonals (the vector area of the bilinear face), the velocity on it the mean of its corners' values
//   (Sec. 2.3.1: the flux of each recipient face from the interpolated, frame-transformed velocities).
//   Sec. 2.4 "Mass conservation": the fluxes through a closed interface must sum to zero; the imbalance of the
//   reconstructed fluxes is subtracted from the faces in proportion to their areas.
//
//   k_face_flux     thread per face: four corner nodes (FP64 coordinates), area vector, mean corner velocity, U
//   k_flux_sum      block per closed surface: net outward flux and total area, summed in a fixed order (FP64)
//   k_flux_correct  thread per face: U -= sign * net * |S| / area
#include "ovs_flux.cuh"

namespace ovs {

namespace {

constexpr int kFluxThreads = 256;

// corners of face id = 3 * base node + d (order: base, +a, +a+b, +b with a = d+1, b = d+2 mod 3); false if the
// face leaves the grid or the id is out of range
__device__ __forceinline__ bool face_corners(const GridDev& g, int64_t face, int64_t c[4]) {
    if (face < 0 || face >= 3 * g.nnodes) return false;
    const int64_t node = face / 3;
    const int d = (int)(face - 3 * node);
    int q[3];
    q[0] = (int)(node % g.n[0]);
    q[1] = (int)((node / g.n[0]) % g.n[1]);
    q[2] = (int)(node / ((int64_t)g.n[0] * g.n[1]));
    const int a = d == 2 ? 0 : d + 1, b = d == 0 ? 2 : (d == 1 ? 0 : 1);
    const int da[4] = {0, 1, 1, 0}, db[4] = {0, 0, 1, 1};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int r[3] = {q[0], q[1], q[2]};
        r[a] += da[k];
        r[b] += db[k];
#pragma unroll
        for (int m = 0; m < 3; ++m)
            if (r[m] == g.n[m]) {
                if (!g.per[m]) return false;
                r[m] = 0;
            }
        c[k] = (int64_t)r[0] + (int64_t)g.n[0] * ((int64_t)r[1] + (int64_t)g.n[1] * r[2]);
    }
    return true;
}

__device__ __forceinline__ double3 area_vector(const GridDev& g, const int64_t c[4]) {
    const double d1x = __ldg(g.x + c[2]) - __ldg(g.x + c[0]), d1y = __ldg(g.y + c[2]) - __ldg(g.y + c[0]),
                 d1z = __ldg(g.z + c[2]) - __ldg(g.z + c[0]);
    const double d2x = __ldg(g.x + c[3]) - __ldg(g.x + c[1]), d2y = __ldg(g.y + c[3]) - __ldg(g.y + c[1]),
                 d2z = __ldg(g.z + c[3]) - __ldg(g.z + c[1]);
    return make_double3(0.5 * (d1y * d2z - d1z * d2y), 0.5 * (d1z * d2x - d1x * d2z), 0.5 * (d1x * d2y - d1y * d2x));
}

template <typename T>
__device__ __forceinline__ T vel_at(const FieldsDev& F, int comp, int64_t node) {
    return __ldg((const T*)F.f[comp] + node * F.stride);
}

template <typename T>
__global__ void __launch_bounds__(kFluxThreads) k_face_flux(const FluxParams P, const GridDev* __restrict__ G) {
    const GridDev& g = G[P.grid];
    T* flux = (T*)P.flux;
    for (int64_t f = blockIdx.x * (int64_t)kFluxThreads + threadIdx.x; f < P.nfaces;
         f += (int64_t)gridDim.x * kFluxThreads) {
        int64_t c[4];
        if (!face_corners(g, __ldg(P.faces + f), c)) {
            atomicOr(P.err, kErrBadCell);
            flux[f] = (T)0;
            continue;
        }
        const double3 S = area_vector(g, c);
        T u[3];
#pragma unroll
        for (int q = 0; q < 3; ++q)
            u[q] = (T)0.25 * (vel_at<T>(P.vel, q, c[0]) + vel_at<T>(P.vel, q, c[1]) + vel_at<T>(P.vel, q, c[2]) +
                              vel_at<T>(P.vel, q, c[3]));
        flux[f] = u[0] * (T)S.x + u[1] * (T)S.y + u[2] * (T)S.z;
    }
}

__device__ __forceinline__ double face_area(const GridDev& g, int64_t face) {
    int64_t c[4];
    if (!face_corners(g, face, c)) return 0.0;
    const double3 S = area_vector(g, c);
    return sqrt(S.x * S.x + S.y * S.y + S.z * S.z);
}

__device__ __forceinline__ double face_sign(const FluxParams& P, int64_t f) {
    return P.signs ? (double)__ldg(P.signs + f) : 1.0;
}

// one block per surface; fixed-order sums (thread-strided, then a fixed tree), so the result is reproducible
template <typename T>
__global__ void __launch_bounds__(kFluxThreads) k_flux_sum(const FluxParams P, const GridDev* __restrict__ G) {
    const GridDev& g = G[P.grid];
    const int s = blockIdx.x;
    const int64_t f0 = P.surf_start[s], f1 = P.surf_start[s + 1];
    const T* flux = (const T*)P.flux;
    double net = 0.0, area = 0.0;
    for (int64_t f = f0 + threadIdx.x; f < f1; f += kFluxThreads) {
        net += face_sign(P, f) * (double)flux[f];
        area += face_area(g, __ldg(P.faces + f));
    }
    __shared__ double sn[kFluxThreads], sa[kFluxThreads];
    sn[threadIdx.x] = net;
    sa[threadIdx.x] = area;
    __syncthreads();
    for (int h = kFluxThreads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            sn[threadIdx.x] += sn[threadIdx.x + h];
            sa[threadIdx.x] += sa[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        P.net[2 * s] = sn[0];
        P.net[2 * s + 1] = sa[0];
    }
}

template <typename T>
__global__ void __launch_bounds__(kFluxThreads) k_flux_correct(const FluxParams P, const GridDev* __restrict__ G) {
    const GridDev& g = G[P.grid];
    T* flux = (T*)P.flux;
    const int64_t end = P.surf_start[P.nsurf];
    for (int64_t f = P.surf_start[0] + blockIdx.x * (int64_t)kFluxThreads + threadIdx.x; f < end;
         f += (int64_t)gridDim.x * kFluxThreads) {
        int lo = 0, hi = P.nsurf - 1;  // the surface holding face f: the last one starting at or before it
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (P.surf_start[mid] <= f) lo = mid;
            else hi = mid - 1;
        }
        const double A = P.net[2 * lo + 1];
        if (!(A > 0.0)) continue;
        const double corr = face_sign(P, f) * P.net[2 * lo] * face_area(g, __ldg(P.faces + f)) / A;
        flux[f] = (T)((double)flux[f] - corr);
    }
}

template <typename T>
cudaError_t launch_t(const FluxParams& P, const GridDev* dgrids, int nsm, bool correct, cudaStream_t st) {
    const int64_t want = (P.nfaces + kFluxThreads - 1) / kFluxThreads;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)nsm * 8));
    if (P.nfaces > 0) k_face_flux<T><<<blocks, kFluxThreads, 0, st>>>(P, dgrids);
    if (P.nsurf > 0) {
        k_flux_sum<T><<<(unsigned)P.nsurf, kFluxThreads, 0, st>>>(P, dgrids);
        if (correct) k_flux_correct<T><<<blocks, kFluxThreads, 0, st>>>(P, dgrids);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_flux(const FluxParams& P, bool f64, const GridDev* dgrids, int nsm, bool correct, cudaStream_t st) {
    return f64 ? launch_t<double>(P, dgrids, nsm, correct, st) : launch_t<float>(P, dgrids, nsm, correct, st);
}

}  // namespace ovs
