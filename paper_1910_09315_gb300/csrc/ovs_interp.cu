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
    const int si = (int)(&s - P.s);
    interp_point<T>(G[gd], gr, P.fields[gd], P.mode, P.mf[gd], P.mf[s.receiver], P.m[gd], P.m[s.receiver], node,
                    cell, u, v, w, P.out, t, gd == s.donors[0] ? P.va + si : nullptr);
}

// Persistent grid (a multiple of the SM count), grid-stride over the call's points.
template <typename T>
__global__ void __launch_bounds__(kInterpThreads) k_interp(const InterpParams* __restrict__ Pp,
                                                           const GridDev* __restrict__ G) {
    const InterpParams& P = *Pp;
    const int64_t total = P.total;
    for (int64_t t = blockIdx.x * (int64_t)kInterpThreads + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * kInterpThreads)
        interp_one<T>(P, G, t, __ldg(P.in_status + t));
}

}  // namespace

int interp_default_blocks_per_sm(bool f64) {
    // blocks resident per SM at once, from the occupancy calculator (the same for every call on a device)
    static int per_sm[2] = {0, 0};
    int& bps = per_sm[f64 ? 1 : 0];
    if (bps <= 0) {
        int v = 0;
        cudaError_t e = f64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_interp<double>, kInterpThreads, 0)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_interp<float>, kInterpThreads, 0);
        if (e != cudaSuccess) return -(int)e;
        bps = v < 1 ? 1 : v;
    }
    return bps;
}

cudaError_t launch_interp(const InterpParams* dI, bool f64, const GridDev* dgrids, int nsm, int tuned_bps,
                          cudaStream_t st, cudaEvent_t const* ev) {
    int bps = tuned_bps;
    if (bps <= 0) {
        bps = interp_default_blocks_per_sm(f64);
        if (bps < 0) return (cudaError_t)(-bps);
    }
    const unsigned blocks = (unsigned)(nsm * bps);
    if (ev && ev[0]) cudaEventRecord(ev[0], st);
    if (f64) k_interp<double><<<blocks, kInterpThreads, 0, st>>>(dI, dgrids);
    else k_interp<float><<<blocks, kInterpThreads, 0, st>>>(dI, dgrids);
    if (ev && ev[1]) cudaEventRecord(ev[1], st);
    return cudaGetLastError();
}

}  // namespace ovs
