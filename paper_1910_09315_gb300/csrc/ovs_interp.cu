// Boundary interpolation (Sec. 2.2.6) from donors found earlier: one thread per point, the trilinear gather of
// u, v, w, p from the caller's SoA node fields (FP32 or FP64) and the frame velocity transform (ovs_fields.cuh).
#include "ovs_fields.cuh"

namespace ovs {

namespace {

constexpr int kInterpThreads = 256;

// Interpolation of point t from its donor record.
template <typename T>
__device__ __forceinline__ void interp_one(const InterpParams& P, const GridDev* __restrict__ G, int64_t t,
                                           uint8_t st) {
    st &= OVS_STATUS_MASK;
    const int32_t gd = __ldg(P.in_grid + t);
    if (st != OVS_STATUS_FOUND || gd < 0) {
        zero_point<T>(P.out, t);
        return;
    }
    const int32_t cell = __ldg(P.in_cell + t);
    if (gd >= P.ngrids || cell < 0 || cell >= G[gd].ncells || !P.fields[gd].f[0] || !P.fields[gd].f[1] ||
        !P.fields[gd].f[2] || !P.fields[gd].f[3]) {
        // a donor record this call cannot use (not produced by ovs_assemble for these grids and fields)
        atomicOr(P.err, kErrBadCell);
        zero_point<T>(P.out, t);
        return;
    }
    T u, v, w;
    if (P.xi_f64) {
        const double* xi = (const double*)P.in_xi;
        u = (T)__ldg(xi + t);
        v = (T)__ldg(xi + P.total + t);
        w = (T)__ldg(xi + 2 * P.total + t);
    } else {
        const float* xi = (const float*)P.in_xi;
        u = (T)__ldg(xi + t);
        v = (T)__ldg(xi + P.total + t);
        w = (T)__ldg(xi + 2 * P.total + t);
    }
    const SetDev& s = P.s[find_set(P.s, P.nsets, t)];
    const int32_t node = __ldg(s.node_ids + (t - s.begin));
    const GridDev& gr = G[s.receiver];
    if (P.mode != OVS_VEL_NONE && P.mode != OVS_VEL_ABSOLUTE && (node < 0 || node >= gr.nnodes)) {
        atomicOr(P.err, kErrBadNode);
        zero_point<T>(P.out, t);
        return;
    }
    interp_point<T>(G[gd], gr, P.fields[gd], P.mode, P.mf[gd], P.mf[s.receiver], P.m[gd], P.m[s.receiver], node,
                    cell, u, v, w, P.out, t);
}

template <typename T>
__global__ void __launch_bounds__(kInterpThreads) k_interp(const __grid_constant__ InterpParams P,
                                                           const GridDev* __restrict__ G) {
    const int64_t t = blockIdx.x * (int64_t)kInterpThreads + threadIdx.x;
    if (t >= P.total) return;
    interp_one<T>(P, G, t, __ldg(P.in_status + t));
}

}  // namespace

cudaError_t launch_interp(const InterpParams& P, const GridDev* dgrids, cudaStream_t st, cudaEvent_t const* ev) {
    int64_t blocks = (P.total + kInterpThreads - 1) / kInterpThreads;
    if (ev && ev[0]) cudaEventRecord(ev[0], st);
    if (P.f64) k_interp<double><<<(unsigned)blocks, kInterpThreads, 0, st>>>(P, dgrids);
    else k_interp<float><<<(unsigned)blocks, kInterpThreads, 0, st>>>(P, dgrids);
    if (ev && ev[1]) cudaEventRecord(ev[1], st);
    return cudaGetLastError();
}

}  // namespace ovs
