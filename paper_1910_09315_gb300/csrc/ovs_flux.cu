// Contravariant fluxes at the receivers and the mass-conservation correction over closed interfaces.
//
//   Sec. 2.1 eq. "flux": U^r = u_q xi^r_q / J, the velocity dotted with the area vector of a face of constant xi^r.
//   On the structured grid a face is a quadrilateral of four nodes; its area vector is half the cross product of
//   its diagonals (the vector area of the bilinear face), the velocity on it the mean of its corners' values
//   (Sec. 2.3.1: the flux of each recipient face from the interpolated, frame-transformed velocities).
//   Sec. 2.4 "Mass conservation": the fluxes through a closed interface must sum to zero; the imbalance of the
//   reconstructed fluxes is subtracted from the faces in proportion to their areas.
//
//   k_flux_faces    a block per chunk of consecutive faces of one surface: each face's four corner nodes, area
//                   vector (FP32 from the corners' FP32 pairs for FP32 velocities, whose differences are exact to
//                   ~1e-14; FP64 coordinates for FP64 velocities), mean corner velocity and U; the chunk's net
//                   outward flux and area summed in a fixed order.  Further blocks take the faces outside every
//                   surface (U only).
//   k_flux_total    a block per surface: its chunks' sums added in a fixed order (the result depends only on the
//                   inputs, not on the timing of the blocks)
//   k_flux_correct  thread per surface face: U -= sign * net * |S| / area (|S| formed again as above)
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

// the same vector area in FP32 from the corners' FP32 pairs: each diagonal as (hi - hi) + (lo - lo)
__device__ __forceinline__ float3 area_vector32(const GridDev& g, const int64_t c[4]) {
    const int64_t nn = g.nnodes;
    float d1[3], d2[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float* h = g.xff + 2 * q * nn;
        const float* l = g.xff + (2 * q + 1) * nn;
        d1[q] = __fadd_rn(__fsub_rn(__ldg(h + c[2]), __ldg(h + c[0])), __fsub_rn(__ldg(l + c[2]), __ldg(l + c[0])));
        d2[q] = __fadd_rn(__fsub_rn(__ldg(h + c[3]), __ldg(h + c[1])), __fsub_rn(__ldg(l + c[3]), __ldg(l + c[1])));
    }
    return make_float3(0.5f * (d1[1] * d2[2] - d1[2] * d2[1]), 0.5f * (d1[2] * d2[0] - d1[0] * d2[2]),
                       0.5f * (d1[0] * d2[1] - d1[1] * d2[0]));
}

template <typename T>
__device__ __forceinline__ T vel_at(const FieldsDev& F, int comp, int64_t node) {
    return __ldg((const T*)F.f[comp] + node * F.stride);
}

// flux of face number f of the call (0 if its id leaves the grid: reported); |S| in *area
template <typename T>
__device__ __forceinline__ T one_face(const FluxParams& P, const GridDev& g, int64_t f, double* area) {
    int64_t c[4];
    if (!face_corners(g, __ldg(P.faces + f), c)) {
        atomicOr(P.err, kErrBadCell);
        *area = 0.0;
        return (T)0;
    }
    T S[3];
    if constexpr (sizeof(T) == 8) {
        const double3 s = area_vector(g, c);
        S[0] = s.x, S[1] = s.y, S[2] = s.z;
        *area = sqrt(s.x * s.x + s.y * s.y + s.z * s.z);
    } else {
        const float3 s = area_vector32(g, c);
        S[0] = s.x, S[1] = s.y, S[2] = s.z;
        *area = (double)sqrtf(s.x * s.x + s.y * s.y + s.z * s.z);
    }
    T u[3];
#pragma unroll
    for (int q = 0; q < 3; ++q)
        u[q] = (T)0.25 * (vel_at<T>(P.vel, q, c[0]) + vel_at<T>(P.vel, q, c[1]) + vel_at<T>(P.vel, q, c[2]) +
                          vel_at<T>(P.vel, q, c[3]));
    return u[0] * S[0] + u[1] * S[1] + u[2] * S[2];
}

__device__ __forceinline__ double face_sign(const FluxParams& P, int64_t f) {
    return P.signs ? (double)__ldg(P.signs + f) : 1.0;
}

// fixed-order sum of (a, b) over the block's threads (a tree over the thread index); the result in thread 0
__device__ __forceinline__ void block_sum2(double& a, double& b) {
    __shared__ double sa[kFluxThreads], sb[kFluxThreads];
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int h = kFluxThreads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            sa[threadIdx.x] += sa[threadIdx.x + h];
            sb[threadIdx.x] += sb[threadIdx.x + h];
        }
        __syncthreads();
    }
    a = sa[0];
    b = sb[0];
}

// the surface owning chunk (or face) x: the last s with start[s] <= x, for nondecreasing start[0..n]
template <typename I>
__device__ __forceinline__ int owner(const I* start, int n, int64_t x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// blocks [0, nchunk): surface chunks; blocks [nchunk, gridDim.x): the loose faces, grid-stride
template <typename T>
__global__ void __launch_bounds__(kFluxThreads) k_flux_faces(const FluxParams P, const GridDev* __restrict__ G) {
    const GridDev& g = G[P.grid];
    T* flux = (T*)P.flux;
    const int nchunk = P.nsurf > 0 ? P.chunk_start[P.nsurf] : 0;
    const int b = blockIdx.x;
    if (b < nchunk) {
        const int s = owner(P.chunk_start, P.nsurf, b);
        const int64_t f0 = P.surf_start[s] + (int64_t)(b - P.chunk_start[s]) * P.chunk;
        const int64_t f1 = min(f0 + P.chunk, P.surf_start[s + 1]);
        double net = 0.0, area = 0.0;
        for (int64_t f = f0 + threadIdx.x; f < f1; f += kFluxThreads) {
            double a;
            const T U = one_face<T>(P, g, f, &a);
            flux[f] = U;
            net += face_sign(P, f) * (double)U;
            area += a;
        }
        block_sum2(net, area);
        if (threadIdx.x == 0) {
            P.part[2 * b] = net;
            P.part[2 * b + 1] = area;
        }
        return;
    }
    // faces before the first surface and after the last one
    const int64_t lo = P.nsurf > 0 ? P.surf_start[0] : P.nfaces;
    const int64_t hi = P.nsurf > 0 ? P.surf_start[P.nsurf] : P.nfaces;
    const int64_t nloose = lo + (P.nfaces - hi);
    for (int64_t k = (int64_t)(b - nchunk) * kFluxThreads + threadIdx.x; k < nloose;
         k += (int64_t)(gridDim.x - nchunk) * kFluxThreads) {
        const int64_t f = k < lo ? k : hi + (k - lo);
        double a;
        flux[f] = one_face<T>(P, g, f, &a);
    }
}

// a block per surface: the sums of its chunks, thread-strided and then the fixed tree
__global__ void __launch_bounds__(kFluxThreads) k_flux_total(const FluxParams P) {
    const int s = blockIdx.x;
    double net = 0.0, area = 0.0;
    for (int q = P.chunk_start[s] + threadIdx.x; q < P.chunk_start[s + 1]; q += kFluxThreads) {
        net += P.part[2 * q];
        area += P.part[2 * q + 1];
    }
    block_sum2(net, area);
    if (threadIdx.x == 0) {
        P.net[2 * s] = net;
        P.net[2 * s + 1] = area;
    }
}

template <typename T>
__global__ void __launch_bounds__(kFluxThreads) k_flux_correct(const FluxParams P, const GridDev* __restrict__ G) {
    const GridDev& g = G[P.grid];
    T* flux = (T*)P.flux;
    const int64_t end = P.surf_start[P.nsurf];
    for (int64_t f = P.surf_start[0] + blockIdx.x * (int64_t)kFluxThreads + threadIdx.x; f < end;
         f += (int64_t)gridDim.x * kFluxThreads) {
        const int s = owner(P.surf_start, P.nsurf, f);
        const double A = P.net[2 * s + 1];
        if (!(A > 0.0)) continue;
        int64_t c[4];
        double a = 0.0;
        if (face_corners(g, __ldg(P.faces + f), c)) {
            if constexpr (sizeof(T) == 8) {
                const double3 v = area_vector(g, c);
                a = sqrt(v.x * v.x + v.y * v.y + v.z * v.z);
            } else {
                const float3 v = area_vector32(g, c);
                a = (double)sqrtf(v.x * v.x + v.y * v.y + v.z * v.z);
            }
        }
        const double corr = face_sign(P, f) * P.net[2 * s] * a / A;
        flux[f] = (T)((double)flux[f] - corr);
    }
}

template <typename T>
cudaError_t launch_t(const FluxParams& P, const GridDev* dgrids, int nsm, bool correct, cudaStream_t st) {
    const int nchunk = P.nsurf > 0 ? P.chunk_start[P.nsurf] : 0;
    const int64_t in_surf = P.nsurf > 0 ? P.surf_start[P.nsurf] - P.surf_start[0] : 0;
    const int64_t nloose = P.nfaces - in_surf;
    const int64_t lb = std::min<int64_t>((nloose + kFluxThreads - 1) / kFluxThreads, (int64_t)nsm * 8);
    const unsigned blocks = (unsigned)(nchunk + lb);
    if (blocks > 0) k_flux_faces<T><<<blocks, kFluxThreads, 0, st>>>(P, dgrids);
    if (P.nsurf > 0) {
        k_flux_total<<<(unsigned)P.nsurf, kFluxThreads, 0, st>>>(P);
        if (correct && in_surf > 0) {
            const unsigned cb = (unsigned)std::max<int64_t>(
                1, std::min<int64_t>((in_surf + kFluxThreads - 1) / kFluxThreads, (int64_t)nsm * 8));
            k_flux_correct<T><<<cb, kFluxThreads, 0, st>>>(P, dgrids);
        }
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_flux(const FluxParams& P, bool f64, const GridDev* dgrids, int nsm, bool correct, cudaStream_t st) {
    return f64 ? launch_t<double>(P, dgrids, nsm, correct, st) : launch_t<float>(P, dgrids, nsm, correct, st);
}

}  // namespace ovs
