// Trilinear gather of node fields and the frame velocity transform, shared by the interpolation kernel and
// the fused assembly + interpolation kernels.
//   q = sum_a N_a(xi) q_a over the donor cell's 8 nodes (Sec. 2.2.6, factors (a-1) read as (1-a))
//   RELATIVE  u_in = R_d u_d + V_d + Omega_d x (x_in - c_d);  u_r = R_r^T (u_in - V_r - Omega_r x (x_in - c_r))
//             (Sec. 2.1 eq. "velocity": frame velocity = translation + Omega x position)
//   ABSOLUTE  u_r = R_r^T R_d u_d  (Sec. 2.3.1 eq. "velocity_non", Q = R^T)
// Pressure passes unchanged.
#pragma once
#include "ovs_internal.cuh"

namespace ovs {

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

// q[0..3] = trilinear interpolation of u, v, w, p at local coordinates (u, v, w) of `cell`
template <typename T>
__device__ __forceinline__ void gather8_ijk(const GridDev& g, const FieldsDev& F, int i, int j, int k, T u, T v, T w,
                                            T q[4]) {
    // corner a = node of (i + di, j + dj, k + dk): the cell's first node plus one offset per set bit (an index
    // that reaches n is on a periodic axis and wraps to 0)
    const int64_t n0 = g.n[0], n01 = (int64_t)g.n[0] * g.n[1];
    const int64_t base = (int64_t)i + n0 * ((int64_t)j + (int64_t)g.n[1] * k);
    const int64_t oi = i + 1 == g.n[0] ? -(int64_t)i : 1;
    const int64_t oj = j + 1 == g.n[1] ? -(int64_t)j * n0 : n0;
    const int64_t ok = k + 1 == g.n[2] ? -(int64_t)k * n01 : n01;
    auto corner = [&](int a) { return base + ((a & 1) ? oi : 0) + ((a & 2) ? oj : 0) + ((a & 4) ? ok : 0); };
    q[0] = q[1] = q[2] = q[3] = (T)0;
    if (F.rec4) {
        // one (u, v, w, p) record per corner: one 16-byte load (FP32) or two (FP64); the sums as below
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            T wa = ((a & 1) ? u : (T)1 - u) * ((a & 2) ? v : (T)1 - v) * ((a & 4) ? w : (T)1 - w);
            const int64_t nd = corner(a);
            T r[4];
            if constexpr (sizeof(T) == 4) {
                const float4 x = __ldg(reinterpret_cast<const float4*>(F.f[0]) + nd);
                r[0] = x.x, r[1] = x.y, r[2] = x.z, r[3] = x.w;
            } else {
                const double2 x0 = __ldg(reinterpret_cast<const double2*>(F.f[0]) + 2 * nd),
                              x1 = __ldg(reinterpret_cast<const double2*>(F.f[0]) + 2 * nd + 1);
                r[0] = x0.x, r[1] = x0.y, r[2] = x1.x, r[3] = x1.y;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) q[c] += wa * r[c];
        }
        return;
    }
    const T* f[4] = {(const T*)F.f[0], (const T*)F.f[1], (const T*)F.f[2], (const T*)F.f[3]};
    auto sum = [&](int64_t st) {
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            T wa = ((a & 1) ? u : (T)1 - u) * ((a & 2) ? v : (T)1 - v) * ((a & 4) ? w : (T)1 - w);
            const int64_t nd = corner(a) * st;
#pragma unroll
            for (int c = 0; c < 4; ++c) q[c] += wa * __ldg(f[c] + nd);
        }
    };
    if (F.stride == 1)
        sum(1);  // four contiguous arrays (the multiply folds away)
    else
        sum(F.stride);
}

template <typename T>
__device__ __forceinline__ void gather8(const GridDev& g, const FieldsDev& F, int64_t cell, T u, T v, T w, T q[4]) {
    int i, j, k;
    cell_ijk(g, cell, i, j, k);
    gather8_ijk<T>(g, F, i, j, k, u, v, w, q);
}

// FP32 velocity transform.  The receiver node's position is its FP32 pair (xh + xl) in the receiver frame;
// r_r = x_in - c_r = R_r x_r and r_d = x_in - c_d = R_r x_r + (c_r - c_d), in inertial components.
__device__ __forceinline__ void vel_transform_f32(int mode, const MotionF& md, const MotionF& mr, const float xh[3],
                                                  const float xl[3], float ud[3]) {
    float uin[3];
    if (mode == OVS_VEL_NONE) return;
    if (mode == OVS_VEL_ABSOLUTE) {
        if (!md.identity) rot(md.R, ud, uin);
        else uin[0] = ud[0], uin[1] = ud[1], uin[2] = ud[2];
        if (!mr.identity) rotT(mr.R, uin, ud);
        else ud[0] = uin[0], ud[1] = uin[1], ud[2] = uin[2];
        return;
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

// FP64 velocity transform (FP64 fields); xr is the receiver node's FP64 position in the receiver frame.
__device__ __forceinline__ void vel_transform_f64(int mode, const MotionDev& md, const MotionDev& mr, const double xr[3],
                                                  double ud[3]) {
    double uin[3];
    if (mode == OVS_VEL_NONE) return;
    if (mode == OVS_VEL_ABSOLUTE) {
        if (!md.identity) rot(md.R, ud, uin);
        else uin[0] = ud[0], uin[1] = ud[1], uin[2] = ud[2];
        if (!mr.identity) rotT(mr.R, uin, ud);
        else ud[0] = uin[0], ud[1] = uin[1], ud[2] = uin[2];
        return;
    }
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

// Interpolated and transformed (u, v, w, p) of one point at donor (gd, cell, xi), written to out[*][t].
// T = field type.  Receiver position: FP32 pair (T = float) or FP64 (T = double) of node `node`.  va: the set's
// affine velocity map when gd is the set's first donor and the fields are FP32 (else NULL: the two transforms).
// ijk (may be NULL): the cell's indices, when the caller has them; xr (may be NULL): the receiver node's position
// in its frame in FP32 (hi + lo of its pair), when the caller has it.
template <typename T>
__device__ __forceinline__ void interp_point(const GridDev& g, const GridDev& gr, const FieldsDev& F, int mode,
                                             const MotionF& mfd, const MotionF& mfr, const MotionDev& md,
                                             const MotionDev& mr, int32_t node, int64_t cell, T u, T v, T w,
                                             void* const out[4], int64_t t, const VelAffine* va = nullptr,
                                             const int* ijk = nullptr, const float* xr = nullptr) {
    T q[4];
    if (ijk) gather8_ijk<T>(g, F, ijk[0], ijk[1], ijk[2], u, v, w, q);
    else gather8<T>(g, F, cell, u, v, w, q);
    if constexpr (sizeof(T) == 4) {
        if (va) {
            const float ud[3] = {q[0], q[1], q[2]};
            float x[3] = {0.f, 0.f, 0.f};
            if (mode == OVS_VEL_RELATIVE) {
                const int64_t nn = gr.nnodes;
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    x[c] = xr ? xr[c] : __ldg(gr.xff + 2 * c * nn + node) + __ldg(gr.xff + (2 * c + 1) * nn + node);
            }
#pragma unroll
            for (int r = 0; r < 3; ++r)
                q[r] = fmaf(va->A[3 * r], ud[0], fmaf(va->A[3 * r + 1], ud[1], fmaf(va->A[3 * r + 2], ud[2],
                       fmaf(va->B[3 * r], x[0], fmaf(va->B[3 * r + 1], x[1], fmaf(va->B[3 * r + 2], x[2], va->b[r]))))));
#pragma unroll
            for (int c = 0; c < 4; ++c) ((T*)out[c])[t] = q[c];
            return;
        }
    }
    if (mode != OVS_VEL_NONE) {
        T ud[3] = {q[0], q[1], q[2]};
        if constexpr (sizeof(T) == 4) {
            const int64_t nn = gr.nnodes;
            float xh[3], xl[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                xh[c] = __ldg(gr.xff + 2 * c * nn + node);
                xl[c] = __ldg(gr.xff + (2 * c + 1) * nn + node);
            }
            vel_transform_f32(mode, mfd, mfr, xh, xl, ud);
        } else {
            double xr[3] = {__ldg(gr.x + node), __ldg(gr.y + node), __ldg(gr.z + node)};
            vel_transform_f64(mode, md, mr, xr, ud);
        }
        q[0] = ud[0];
        q[1] = ud[1];
        q[2] = ud[2];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) ((T*)out[c])[t] = q[c];
}

template <typename T>
__device__ __forceinline__ void zero_point(void* const out[4], int64_t t) {
#pragma unroll
    for (int c = 0; c < 4; ++c) ((T*)out[c])[t] = (T)0;
}

}  // namespace ovs
