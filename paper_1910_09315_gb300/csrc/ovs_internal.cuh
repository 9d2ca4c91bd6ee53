// Internal types and device helpers of libovs (sm_103a).
//
// Data layout in HBM
//   grid nodes   : caller's SoA FP64 x, y, z (i fastest), read only for exact FP64 decisions
//   cell records : 128 B per cell (one L2 line): corner 0 in FP64 and the 7 monomial coefficient
//                  vectors of the trilinear map relative to it in FP32, so one walk step is one
//                  line fetch and the FP32 Newton needs only 3 FP64 subtractions
//   bins         : control cells of Sec. 2.2.5, CSR (start[nbins+1], cells[]) + lowest registered
//                  cell per bin (cold-start cell)
//   hints        : per receiver node, uint32 (donor grid << 27 | cell) of the last donor found
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ovs.h"

namespace ovs {

constexpr float kNearFace = 1e-4f;   // FP32 xi within this of a face -> decide in FP64
constexpr float kAccept32 = 1e-4f;   // FP32 walk accepts a cell when xi is within this of [0,1]^3
constexpr double kWinLo = -1e-10;    // donor window (lowest-id rule)
constexpr double kWinHi = 1.0 + 1e-10;
constexpr double kNewtonTol64 = 1e-13;
constexpr int kNewtonMaxIt64 = 50;
constexpr int kNewtonMaxIt32 = 8;
constexpr float kNewtonTol32 = 2e-6f;
constexpr int kMaxJump = 4;
constexpr uint32_t kNoHint = 0xFFFFFFFFu;
constexpr int kCellBits = 27;

// One cell: x(xi) = x0 + a1 xi + a2 eta + a3 zeta + a4 xi eta + a5 eta zeta + a6 xi zeta + a7 xi eta zeta
struct __align__(16) CellRec {
    double x0[3];
    float a[21];  // a1.xyz, a2.xyz, ..., a7.xyz
    float pad[5];
};
static_assert(sizeof(CellRec) == 128, "cell record must be one 128-byte line");

struct GridDev {
    int32_t n[3];
    int32_t per[3];
    int32_t C[3];  // cells per axis
    int32_t role;
    int64_t ncells;
    int64_t nnodes;
    const double* x;
    const double* y;
    const double* z;
    const CellRec* rec;
    const int32_t* bin_start;  // nbins + 1
    const int32_t* bin_cells;
    const int32_t* bin_rep;    // lowest registered cell, -1 if empty
    uint32_t* hint;            // per node
    const void* mlp;           // guess network (device), or null
    double lo[3], hi[3];       // padded bounding box of the bins
    double inv_w[3];           // bins per unit length
    int32_t nb[3];
    int32_t mlp_hidden;
};

struct MotionDev {
    double R[9];  // body -> inertial, row-major
    double c[3];
    double V[3];
    double w[3];
    int32_t identity;
    int32_t pad;
};

struct SetDev {
    int32_t receiver;
    int32_t ndonor;
    int32_t donors[OVS_MAX_DONORS];
    const int32_t* node_ids;
    int64_t begin;
    int64_t n;
};

struct SlowEntry {
    int32_t t;      // point index
    int32_t di;     // position in the set's donor list to resume at
    int32_t cell;   // FP32 walk result, -1 if the walk got stuck
    float xi[3];
};

enum Counter { kCtrPoints = 0, kCtrWalk, kCtrRefined, kCtrFallback, kCtrGuess, kNumCounters };

struct AsmParams {
    int32_t nsets;
    int32_t xi_f64;
    int32_t max_walk;
    int32_t guess;
    int32_t stats;
    int32_t pad;
    int64_t total;
    int64_t queue_cap;
    int32_t* out_grid;
    int32_t* out_cell;
    void* out_xi;
    uint8_t* out_status;
    SlowEntry* queue;
    uint32_t* queue_count;
    unsigned long long* counters;
    int32_t* err;
    SetDev s[OVS_MAX_SETS];
    MotionDev m[OVS_MAX_GRIDS];
};

struct FieldsDev {
    const void* f[4];
};

struct InterpParams {
    int32_t nsets;
    int32_t xi_f64;
    int32_t mode;
    int32_t f64;
    int32_t ngrids;
    int32_t pad;
    int32_t* err;
    int64_t total;
    const int32_t* in_grid;
    const int32_t* in_cell;
    const void* in_xi;
    const uint8_t* in_status;
    void* out[4];
    SetDev s[OVS_MAX_SETS];
    MotionDev m[OVS_MAX_GRIDS];
    FieldsDev fields[OVS_MAX_GRIDS];
};

// error bits of the device status word
enum DevErr { kErrQueueOverflow = 1, kErrBadCell = 2, kErrBadNode = 4 };

// ------------------------------------------------------------------------------------------------
// small helpers
__device__ __forceinline__ int find_set(const SetDev* s, int nsets, int64_t t) {
    int lo = 0, hi = nsets - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (s[mid].begin <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ double3 to_inertial(const MotionDev& m, double3 x) {
    if (m.identity) return x;
    return make_double3(fma(m.R[0], x.x, fma(m.R[1], x.y, fma(m.R[2], x.z, m.c[0]))),
                        fma(m.R[3], x.x, fma(m.R[4], x.y, fma(m.R[5], x.z, m.c[1]))),
                        fma(m.R[6], x.x, fma(m.R[7], x.y, fma(m.R[8], x.z, m.c[2]))));
}

__device__ __forceinline__ double3 to_body(const MotionDev& m, double3 xin) {
    if (m.identity) return xin;
    double dx = xin.x - m.c[0], dy = xin.y - m.c[1], dz = xin.z - m.c[2];
    return make_double3(fma(m.R[0], dx, fma(m.R[3], dy, m.R[6] * dz)),
                        fma(m.R[1], dx, fma(m.R[4], dy, m.R[7] * dz)),
                        fma(m.R[2], dx, fma(m.R[5], dy, m.R[8] * dz)));
}

__device__ __forceinline__ bool finite3(double3 p) {
    return isfinite(p.x) && isfinite(p.y) && isfinite(p.z);
}

__device__ __forceinline__ void cell_ijk(const GridDev& g, int64_t cell, int& i, int& j, int& k) {
    int64_t cij = (int64_t)g.C[0] * g.C[1];
    k = (int)(cell / cij);
    int64_t r = cell - (int64_t)k * cij;
    j = (int)(r / g.C[0]);
    i = (int)(r - (int64_t)j * g.C[0]);
}

__device__ __forceinline__ int64_t cell_id(const GridDev& g, int i, int j, int k) {
    return (int64_t)i + (int64_t)g.C[0] * ((int64_t)j + (int64_t)g.C[1] * k);
}

// node id of corner (i+di, j+dj, k+dk) with periodic wrap
__device__ __forceinline__ int64_t corner_node(const GridDev& g, int i, int j, int k, int a) {
    int ii = i + (a & 1), jj = j + ((a >> 1) & 1), kk = k + ((a >> 2) & 1);
    if (ii == g.n[0]) ii = 0;
    if (jj == g.n[1]) jj = 0;
    if (kk == g.n[2]) kk = 0;
    return (int64_t)ii + (int64_t)g.n[0] * ((int64_t)jj + (int64_t)g.n[1] * kk);
}

// bin of a donor-frame point; -1 when outside the padded bounding box (no cell can contain it)
__device__ __forceinline__ int64_t point_bin(const GridDev& g, double3 p) {
    if (!(p.x >= g.lo[0] && p.x <= g.hi[0] && p.y >= g.lo[1] && p.y <= g.hi[1] && p.z >= g.lo[2] &&
          p.z <= g.hi[2]))
        return -1;
    int bx = min((int)((p.x - g.lo[0]) * g.inv_w[0]), g.nb[0] - 1);
    int by = min((int)((p.y - g.lo[1]) * g.inv_w[1]), g.nb[1] - 1);
    int bz = min((int)((p.z - g.lo[2]) * g.inv_w[2]), g.nb[2] - 1);
    return (int64_t)bx + (int64_t)g.nb[0] * ((int64_t)by + (int64_t)g.nb[1] * bz);
}

__device__ __forceinline__ void load_rec(const CellRec* rec, int64_t cell, CellRec& r) {
    const uint4* src = reinterpret_cast<const uint4*>(rec + cell);
    uint4 v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = __ldg(src + q);
    memcpy(&r, v, sizeof(CellRec));
}

// Padded bounding box of a cell from its record (sound for every point whose local coordinates lie in the
// donor window: the FP32 rounding of the coefficients and the 1e-10 window are both far below the pad).
__device__ __forceinline__ void rec_box(const CellRec& r, double lo[3], double hi[3]) {
    float mn[3], mx[3];
    double d2 = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float a1 = r.a[c], a2 = r.a[3 + c], a3 = r.a[6 + c], a4 = r.a[9 + c], a5 = r.a[12 + c],
              a6 = r.a[15 + c], a7 = r.a[18 + c];
        float e[8] = {0.f, a1, a2, a1 + a2 + a4, a3, a1 + a3 + a6, a2 + a3 + a5, a1 + a2 + a3 + a4 + a5 + a6 + a7};
        mn[c] = e[0];
        mx[c] = e[0];
#pragma unroll
        for (int q = 1; q < 8; ++q) {
            mn[c] = fminf(mn[c], e[q]);
            mx[c] = fmaxf(mx[c], e[q]);
        }
        double ext = (double)mx[c] - (double)mn[c];
        d2 += ext * ext;
    }
    double pad = 2e-6 * sqrt(d2) + 1e-300;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        lo[c] = r.x0[c] + (double)mn[c] - pad;
        hi[c] = r.x0[c] + (double)mx[c] + pad;
    }
}

// FP32 Newton on the monomial form.  Returns true if the last step was below tolerance.
__device__ __forceinline__ bool newton32(const CellRec& r, float dx, float dy, float dz, float& u, float& v,
                                         float& w) {
    const float* a = r.a;
    bool conv = false;
#pragma unroll 1
    for (int it = 0; it < kNewtonMaxIt32; ++it) {
        float uv = u * v, vw = v * w, uw = u * w, uvw = uv * w;
        float F[3], Ju[3], Jv[3], Jw[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float a1 = a[c], a2 = a[3 + c], a3 = a[6 + c], a4 = a[9 + c], a5 = a[12 + c], a6 = a[15 + c],
                  a7 = a[18 + c];
            float d = c == 0 ? dx : (c == 1 ? dy : dz);
            F[c] = fmaf(a1, u, fmaf(a2, v, fmaf(a3, w, fmaf(a4, uv, fmaf(a5, vw, fmaf(a6, uw, fmaf(a7, uvw, -d)))))));
            Ju[c] = fmaf(a4, v, fmaf(a6, w, fmaf(a7, vw, a1)));
            Jv[c] = fmaf(a4, u, fmaf(a5, w, fmaf(a7, uw, a2)));
            Jw[c] = fmaf(a5, v, fmaf(a6, u, fmaf(a7, uv, a3)));
        }
        // Cramer: columns Ju, Jv, Jw
        float cvw[3] = {Jv[1] * Jw[2] - Jv[2] * Jw[1], Jv[2] * Jw[0] - Jv[0] * Jw[2], Jv[0] * Jw[1] - Jv[1] * Jw[0]};
        float cwu[3] = {Jw[1] * Ju[2] - Jw[2] * Ju[1], Jw[2] * Ju[0] - Jw[0] * Ju[2], Jw[0] * Ju[1] - Jw[1] * Ju[0]};
        float cuv[3] = {Ju[1] * Jv[2] - Ju[2] * Jv[1], Ju[2] * Jv[0] - Ju[0] * Jv[2], Ju[0] * Jv[1] - Ju[1] * Jv[0]};
        float det = Ju[0] * cvw[0] + Ju[1] * cvw[1] + Ju[2] * cvw[2];
        float inv = -1.0f / det;
        float du = (F[0] * cvw[0] + F[1] * cvw[1] + F[2] * cvw[2]) * inv;
        float dv = (F[0] * cwu[0] + F[1] * cwu[1] + F[2] * cwu[2]) * inv;
        float dw = (F[0] * cuv[0] + F[1] * cuv[1] + F[2] * cuv[2]) * inv;
        u += du;
        v += dv;
        w += dw;
        float m = fmaxf(fabsf(du), fmaxf(fabsf(dv), fabsf(dw)));
        if (!(m < 1e30f)) return false;  // non-finite
        if (m < kNewtonTol32) {
            conv = true;
            break;
        }
    }
    return conv;
}

// FP64 Newton on the exact node coordinates (the donor rule's decision).  Starts at (u,v,w).
// Returns true iff converged (last step <= 1e-13 within 50 steps) and the result lies in the window.
__device__ __forceinline__ bool newton64_contains(const GridDev& g, int64_t cell, double3 p, double& u, double& v,
                                                  double& w) {
    int i, j, k;
    cell_ijk(g, cell, i, j, k);
    double X[8][3];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        int64_t nd = corner_node(g, i, j, k, a);
        X[a][0] = __ldg(g.x + nd);
        X[a][1] = __ldg(g.y + nd);
        X[a][2] = __ldg(g.z + nd);
    }
    double A[7][3], d[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double e1 = X[1][c] - X[0][c], e2 = X[2][c] - X[0][c], e3 = X[3][c] - X[0][c], e4 = X[4][c] - X[0][c],
               e5 = X[5][c] - X[0][c], e6 = X[6][c] - X[0][c], e7 = X[7][c] - X[0][c];
        A[0][c] = e1;
        A[1][c] = e2;
        A[2][c] = e4;
        A[3][c] = e3 - e1 - e2;
        A[4][c] = e6 - e2 - e4;
        A[5][c] = e5 - e1 - e4;
        A[6][c] = e7 - e3 - e5 - e6 + e1 + e2 + e4;
    }
    d[0] = p.x - X[0][0];
    d[1] = p.y - X[0][1];
    d[2] = p.z - X[0][2];
    bool conv = false;
#pragma unroll 1
    for (int it = 0; it < kNewtonMaxIt64; ++it) {
        double uv = u * v, vw = v * w, uw = u * w, uvw = uv * w;
        double F[3], Ju[3], Jv[3], Jw[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            F[c] = A[0][c] * u + A[1][c] * v + A[2][c] * w + A[3][c] * uv + A[4][c] * vw + A[5][c] * uw +
                   A[6][c] * uvw - d[c];
            Ju[c] = A[0][c] + A[3][c] * v + A[5][c] * w + A[6][c] * vw;
            Jv[c] = A[1][c] + A[3][c] * u + A[4][c] * w + A[6][c] * uw;
            Jw[c] = A[2][c] + A[4][c] * v + A[5][c] * u + A[6][c] * uv;
        }
        double cvw[3] = {Jv[1] * Jw[2] - Jv[2] * Jw[1], Jv[2] * Jw[0] - Jv[0] * Jw[2], Jv[0] * Jw[1] - Jv[1] * Jw[0]};
        double cwu[3] = {Jw[1] * Ju[2] - Jw[2] * Ju[1], Jw[2] * Ju[0] - Jw[0] * Ju[2], Jw[0] * Ju[1] - Jw[1] * Ju[0]};
        double cuv[3] = {Ju[1] * Jv[2] - Ju[2] * Jv[1], Ju[2] * Jv[0] - Ju[0] * Jv[2], Ju[0] * Jv[1] - Ju[1] * Jv[0]};
        double det = Ju[0] * cvw[0] + Ju[1] * cvw[1] + Ju[2] * cvw[2];
        if (!(fabs(det) > 0.0)) return false;
        double du = -(F[0] * cvw[0] + F[1] * cvw[1] + F[2] * cvw[2]) / det;
        double dv = -(F[0] * cwu[0] + F[1] * cwu[1] + F[2] * cwu[2]) / det;
        double dw = -(F[0] * cuv[0] + F[1] * cuv[1] + F[2] * cuv[2]) / det;
        u += du;
        v += dv;
        w += dw;
        if (!(isfinite(u) && isfinite(v) && isfinite(w))) return false;
        double m = fmax(fabs(du), fmax(fabs(dv), fabs(dw)));
        if (m <= kNewtonTol64) {
            conv = true;
            break;
        }
    }
    return conv && u >= kWinLo && u <= kWinHi && v >= kWinLo && v <= kWinHi && w >= kWinLo && w <= kWinHi;
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// host-side launchers (defined in the .cu files)
cudaError_t launch_build_records(const GridDev& g, CellRec* rec, double* partials, int nblocks, double* out9,
                                 cudaStream_t st);
cudaError_t launch_bin_count(const GridDev& g, uint32_t* counts, cudaStream_t st);
cudaError_t launch_scan(const uint32_t* counts, int32_t* start, int64_t n, uint32_t* block_sums, cudaStream_t st);
cudaError_t launch_bin_fill(const GridDev& g, const int32_t* start, uint32_t* cursor, int32_t* cells, int32_t* rep,
                            cudaStream_t st);
size_t scan_scratch_elems(int64_t n);
// ev: 3 optional events (before fast kernel, after it, after the slow kernel); 2 for interpolation
cudaError_t launch_assemble(const AsmParams& P, const GridDev* dgrids, cudaStream_t st, cudaEvent_t const* ev);
cudaError_t launch_interp(const InterpParams& P, const GridDev* dgrids, cudaStream_t st, cudaEvent_t const* ev);

}  // namespace ovs
