// Boundary interpolation (Sec. 2.2.6): q = sum_a N_a(xi) q_a over the donor's 8 nodes for u, v, w, p,
// then the frame velocity transform (Sec. 2.1 eq. "velocity": u_in = R u_rel + V + Omega x r, and
// Sec. 2.3.1 eq. "velocity_non": rotation only).  One thread per point; node fields are the caller's SoA
// arrays (FP32 or FP64), read with read-only loads.
#include "ovs_internal.cuh"

namespace ovs {

namespace {

constexpr int kInterpThreads = 256;

template <typename M, typename T>
__device__ __forceinline__ void rot(const M R[9], const T a[3], T out[3]) {
#pragma unroll
    for (int r = 0; r < 3; ++r) out[r] = (T)R[3 * r] * a[0] + (T)R[3 * r + 1] * a[1] + (T)R[3 * r + 2] * a[2];
}

template <typename M, typename T>
__device__ __forceinline__ void rotT(const M R[9], const T a[3], T out[3]) {
#pragma unroll
    for (int r = 0; r < 3; ++r) out[r] = (T)R[r] * a[0] + (T)R[3 + r] * a[1] + (T)R[6 + r] * a[2];
}

template <typename M, typename T>
__device__ __forceinline__ void cross_add(const M w[3], const T r[3], T acc[3], T sign) {
    acc[0] += sign * ((T)w[1] * r[2] - (T)w[2] * r[1]);
    acc[1] += sign * ((T)w[2] * r[0] - (T)w[0] * r[2]);
    acc[2] += sign * ((T)w[0] * r[1] - (T)w[1] * r[0]);
}

// FP32 velocity transform: positions from the receiver node's FP32 pair, motions from their FP32 copies.
// r_r = x_in - c_r = R_r x_r;  r_d = x_in - c_d = R_r x_r + (c_r - c_d)  (inertial components)
__device__ __forceinline__ void transform_f32(const InterpParams& P, const GridDev* __restrict__ G, const SetDev& s,
                                              int64_t t, int gd, float ud[3]) {
    const MotionF& md = P.mf[gd];
    const MotionF& mr = P.mf[s.receiver];
    float uin[3];
    if (P.mode == OVS_VEL_ABSOLUTE) {
        if (!md.identity) rot(md.R, ud, uin);
        else uin[0] = ud[0], uin[1] = ud[1], uin[2] = ud[2];
        if (!mr.identity) rotT(mr.R, uin, ud);
        else ud[0] = uin[0], ud[1] = uin[1], ud[2] = uin[2];
        return;
    }
    const int32_t node = __ldg(s.node_ids + (t - s.begin));
    const GridDev& gr = G[s.receiver];
    const int64_t nn = gr.nnodes;
    if (node < 0 || node >= nn) {
        atomicOr(P.err, kErrBadNode);
        ud[0] = ud[1] = ud[2] = 0.f;
        return;
    }
    float xh[3], xl[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        xh[c] = __ldg(gr.xff + 2 * c * nn + node);
        xl[c] = __ldg(gr.xff + (2 * c + 1) * nn + node);
    }
    float rr[3], rd[3];
    if (mr.identity) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            rd[c] = (xh[c] - md.ch[c]) + (xl[c] - md.cl[c]);
            rr[c] = 0.f;
        }
    } else {
        float xr[3] = {xh[0] + xl[0], xh[1] + xl[1], xh[2] + xl[2]};
        rot(mr.R, xr, rr);
#pragma unroll
        for (int c = 0; c < 3; ++c) rd[c] = rr[c] + ((mr.ch[c] - md.ch[c]) + (mr.cl[c] - md.cl[c]));
    }
    if (!md.identity) {
        rot(md.R, ud, uin);
#pragma unroll
        for (int c = 0; c < 3; ++c) uin[c] += md.V[c];
        cross_add(md.w, rd, uin, 1.f);
    } else {
        uin[0] = ud[0], uin[1] = ud[1], uin[2] = ud[2];
    }
    if (!mr.identity) {
#pragma unroll
        for (int c = 0; c < 3; ++c) uin[c] -= mr.V[c];
        cross_add(mr.w, rr, uin, -1.f);
        rotT(mr.R, uin, ud);
    } else {
        ud[0] = uin[0], ud[1] = uin[1], ud[2] = uin[2];
    }
}

// FP64 velocity transform (FP64 fields): positions from the receiver node's FP64 coordinates.
__device__ __forceinline__ void transform_f64(const InterpParams& P, const GridDev* __restrict__ G, const SetDev& s,
                                              int64_t t, int gd, double ud[3]) {
    const MotionDev& md = P.m[gd];
    const MotionDev& mr = P.m[s.receiver];
    double uin[3];
    if (P.mode == OVS_VEL_ABSOLUTE) {
        if (!md.identity) rot(md.R, ud, uin);
        else uin[0] = ud[0], uin[1] = ud[1], uin[2] = ud[2];
        if (!mr.identity) rotT(mr.R, uin, ud);
        else ud[0] = uin[0], ud[1] = uin[1], ud[2] = uin[2];
        return;
    }
    const int32_t node = __ldg(s.node_ids + (t - s.begin));
    const GridDev& gr = G[s.receiver];
    if (node < 0 || node >= gr.nnodes) {
        atomicOr(P.err, kErrBadNode);
        ud[0] = ud[1] = ud[2] = 0.0;
        return;
    }
    double xr[3] = {__ldg(gr.x + node), __ldg(gr.y + node), __ldg(gr.z + node)};
    double rr[3], rd[3];
    if (mr.identity) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            rd[c] = xr[c] - md.c[c];
            rr[c] = 0.0;
        }
    } else {
        rot(mr.R, xr, rr);
#pragma unroll
        for (int c = 0; c < 3; ++c) rd[c] = rr[c] + (mr.c[c] - md.c[c]);
    }
    if (!md.identity) {
        rot(md.R, ud, uin);
#pragma unroll
        for (int c = 0; c < 3; ++c) uin[c] += md.V[c];
        cross_add(md.w, rd, uin, 1.0);
    } else {
        uin[0] = ud[0], uin[1] = ud[1], uin[2] = ud[2];
    }
    if (!mr.identity) {
#pragma unroll
        for (int c = 0; c < 3; ++c) uin[c] -= mr.V[c];
        cross_add(mr.w, rr, uin, -1.0);
        rotT(mr.R, uin, ud);
    } else {
        ud[0] = uin[0], ud[1] = uin[1], ud[2] = uin[2];
    }
}

template <typename T>
__global__ void __launch_bounds__(kInterpThreads) k_interp(const __grid_constant__ InterpParams P,
                                                           const GridDev* __restrict__ G) {
    const int64_t t = blockIdx.x * (int64_t)kInterpThreads + threadIdx.x;
    if (t >= P.total) return;
    T* out[4] = {(T*)P.out[0], (T*)P.out[1], (T*)P.out[2], (T*)P.out[3]};
    const uint8_t st = __ldg(P.in_status + t) & OVS_STATUS_MASK;
    const int32_t gd = __ldg(P.in_grid + t);
    if (st != OVS_STATUS_FOUND || gd < 0) {
#pragma unroll
        for (int f = 0; f < 4; ++f) out[f][t] = (T)0;
        return;
    }
    const int32_t cell = __ldg(P.in_cell + t);
    if (gd >= P.ngrids || cell < 0 || cell >= G[gd].ncells || !P.fields[gd].f[0] || !P.fields[gd].f[1] ||
        !P.fields[gd].f[2] || !P.fields[gd].f[3]) {
        // a donor record this call cannot use (not produced by ovs_assemble for these grids and fields)
        atomicOr(P.err, kErrBadCell);
#pragma unroll
        for (int f = 0; f < 4; ++f) out[f][t] = (T)0;
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
    const GridDev& g = G[gd];
    int i, j, k;
    cell_ijk(g, cell, i, j, k);
    T q[4] = {0, 0, 0, 0};
    const T* f[4] = {(const T*)P.fields[gd].f[0], (const T*)P.fields[gd].f[1], (const T*)P.fields[gd].f[2],
                     (const T*)P.fields[gd].f[3]};
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        T wa = ((a & 1) ? u : (T)1 - u) * ((a & 2) ? v : (T)1 - v) * ((a & 4) ? w : (T)1 - w);
        int64_t nd = corner_node(g, i, j, k, a);
#pragma unroll
        for (int c = 0; c < 4; ++c) q[c] += wa * __ldg(f[c] + nd);
    }
    if (P.mode != OVS_VEL_NONE) {
        const int si = find_set(P.s, P.nsets, t);
        const SetDev& s = P.s[si];
        T ud[3] = {q[0], q[1], q[2]};
        if constexpr (sizeof(T) == 4) {
            transform_f32(P, G, s, t, gd, ud);
        } else {
            transform_f64(P, G, s, t, gd, ud);
        }
        q[0] = ud[0];
        q[1] = ud[1];
        q[2] = ud[2];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) out[c][t] = q[c];
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
