// Internal types and device helpers of libovs (sm_103a).
//
// Data layout in HBM
//   grid nodes   : caller's SoA FP64 x, y, z (i fastest), read only for exact FP64 decisions
//   cell records : 128 B per cell (one L2 line): corner 0 as an FP32 pair (hi + lo, ~48-bit) and the 7
//                  monomial coefficient vectors of the trilinear map relative to it in FP32, so one walk
//                  step is one line fetch and no FP64 instruction
//   node pairs   : per node, x, y, z as FP32 pairs (hi + lo), SoA [xh|xl|yh|yl|zh|zl]: the receiver points
//                  of the FP64-free fast path
//   bins         : control cells of Sec. 2.2.5, CSR (start[nbins+1], cells[]) + lowest registered
//                  cell per bin (cold-start cell)
//   hints        : per receiver node, uint32 (donor grid << 27 | cell) of the last donor found
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ovs.h"

namespace ovs {

constexpr float kAccept32 = 1e-4f;   // FP32 walk accepts a cell when xi is within this of [0,1]^3
constexpr double kWinLo = -1e-10;    // donor window (lowest-id rule)
constexpr double kWinHi = 1.0 + 1e-10;
constexpr double kNewtonTol64 = 1e-13;
constexpr int kNewtonMaxIt64 = 50;
constexpr int kNewtonMaxIt32 = 8;
// FP32 Newton stops once a step is below 1e-5: convergence is quadratic, so the local coordinates are then
// accurate to ~1e-10 plus FP32 rounding (~1e-7), and a tighter test would stall at the rounding floor of
// thin cells
constexpr float kNewtonTol32 = 1e-5f;
constexpr int kMaxJump = 4;           // cells per walk step along a non-periodic axis
constexpr int kMaxJumpPeriodic = 12;  // along a periodic (angular) axis, where the extrapolation stays good
constexpr int kHintWalk = 8;          // walk steps from a previous donor or a learned guess before restarting
constexpr uint32_t kNoHint = 0xFFFFFFFFu;
constexpr int kCellBits = 27;

// One cell: x(xi) = x0 + a1 xi + a2 eta + a3 zeta + a4 xi eta + a5 eta zeta + a6 xi zeta + a7 xi eta zeta
struct __align__(16) CellRec {
    float x0h[3];  // corner 0 = x0h + x0l (FP32 pair)
    float x0l[3];
    float a[21];   // a1.xyz, a2.xyz, ..., a7.xyz relative to corner 0
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
    const float* xff;          // node coordinates as FP32 pairs: 6 arrays of nnodes floats
    const void* mlp;           // guess network (device), or null
    double lo[3], hi[3];       // padded bounding box of the bins
    double inv_w[3];           // bins per unit length
    int32_t nb[3];
    int32_t mlp_hidden;
    int32_t blanked;  // 1 once ovs_set_iblank gave the grid a mask (cell records then carry blocked flags)
    int32_t overlap;  // 1: cells may overlap one another (folded cells found, or said by the caller): no point is
                      // final from the walk alone; each goes to the exhaustive lowest-id search of its control cell
    // crowded control cells (lists longer than a threshold), ascending bin id, each split into kSub^3 finer bins
    // whose lists the exhaustive search reads instead (every cell registered in each finer bin its padded box
    // overlaps, as in the first level)
    const int32_t* crowd;
    const int32_t* sub_start;  // ncrowd * kSub3 + 1
    const int32_t* sub_cells;
    int32_t ncrowd;
    int32_t pad2;
};

constexpr int kSub = 4;                 // finer bins per axis inside a crowded control cell
constexpr int kSub3 = kSub * kSub * kSub;
constexpr int32_t kCrowdedCount = 256;  // a control cell listing more cells than this is split (first try)
constexpr int kMaxCrowded = 4096;       // split control cells per grid at most

struct MotionDev {
    double R[9];  // body -> inertial, row-major
    double c[3];
    double V[3];
    double w[3];
    int32_t identity;
    int32_t pad;
};

// Receiver frame -> donor frame of a set's first donor, x_d = M x_r + t, as FP32 pairs (composed in FP64 on
// the host: M = R_d^T R_r, t = R_d^T (c_r - c_d)).
struct XfFF {
    float Mh[9], Ml[9];
    float th[3], tl[3];
    int32_t identity;
    int32_t pad;
};

// One grid's motion in FP32 for the FP32 velocity transform (c as an FP32 pair).
struct MotionF {
    float R[9];
    float ch[3], cl[3];
    float V[3];
    float w[3];
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

// A donor grid's fields: component c of node n at f[c] + n * stride; rec4: one 16-byte-aligned array of
// (u, v, w, p) records per node (stride 4, f[c] = f[0] + c), read as one record per corner.
struct FieldsDev {
    const void* f[4];
    int64_t stride;
    int32_t rec4;
    int32_t pad;
};

// the slow-path queue's counters (zeroed before each assembly call)
constexpr int kQueueCounters = 5;

struct SlowEntry {
    int32_t t;      // point index
    int32_t di;     // bits 0-7: position in the set's donor list to resume at; bits 8-13: near-face mask
                    // (bit 8+m: neighbour at -1 on axis m, bit 11+m: neighbour at +1 on axis m)
    int32_t cell;   // FP32 walk result, -1 if the walk got stuck
    float xi[3];
};

// Bound on the error of the FP32 local coordinates of a point in a cell: FP32 rounding of the offsets and
// coefficients (~6e-8 relative to the largest edge) amplified by the cell's aspect ratio and skew, with a
// safety factor of 64, plus 1e-5.  Below this distance from a face the FP32 decision is not trusted.
__device__ __forceinline__ float near_tau(const CellRec& r, float u, float v, float w) {
    const float* a = r.a;
    float Ju[3], Jv[3], Jw[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Ju[c] = a[c] + a[9 + c] * v + a[15 + c] * w + a[18 + c] * v * w;
        Jv[c] = a[3 + c] + a[9 + c] * u + a[12 + c] * w + a[18 + c] * u * w;
        Jw[c] = a[6 + c] + a[12 + c] * v + a[15 + c] * u + a[18 + c] * u * v;
    }
    float nu = sqrtf(Ju[0] * Ju[0] + Ju[1] * Ju[1] + Ju[2] * Ju[2]);
    float nv = sqrtf(Jv[0] * Jv[0] + Jv[1] * Jv[1] + Jv[2] * Jv[2]);
    float nw = sqrtf(Jw[0] * Jw[0] + Jw[1] * Jw[1] + Jw[2] * Jw[2]);
    float det = Ju[0] * (Jv[1] * Jw[2] - Jv[2] * Jw[1]) + Ju[1] * (Jv[2] * Jw[0] - Jv[0] * Jw[2]) +
                Ju[2] * (Jv[0] * Jw[1] - Jv[1] * Jw[0]);
    float mx = fmaxf(nu, fmaxf(nv, nw)), mn = fminf(nu, fminf(nv, nw));
    float t = 1e-5f + 4e-6f * mx * (nu * nv * nw) * __frcp_rn(mn * fabsf(det));
    return t < 0.25f ? t : 0.25f;  // also catches NaN (degenerate cell): everything counts as near
}

// near-face mask of FP32 local coordinates for threshold tau (see SlowEntry::di)
__device__ __forceinline__ int near_mask(float u, float v, float w, float tau) {
    int m = 0;
    if (u < tau) m |= 1;
    if (v < tau) m |= 2;
    if (w < tau) m |= 4;
    if (u > 1.f - tau) m |= 8;
    if (v > 1.f - tau) m |= 16;
    if (w > 1.f - tau) m |= 32;
    return m;
}

enum Counter {
    kCtrPoints = 0,
    kCtrWalk,
    kCtrRefined,
    kCtrFallback,
    kCtrGuess,
    kCtrNewton,    // FP32 Newton iterations of the walk
    kCtrWarpWalk,  // per warp and work item: the most walk steps of its lanes
    kCtrNear,      // points queued for the near-face decision
    kCtrStuck,     // points queued for the exhaustive search
    kNumCounters
};

// A donor grid's learned-guess network as a call sees it (hidden = 0: none): its padded bounding box and the input
// normalisation xn = (x - centre) * inv_half in FP32, and its region (packed fragments, ovs_guess.cuh).
struct GuessDev {
    float lo[3], hi[3];
    float centre[3], inv_half[3];
    int32_t hidden;
    int32_t pad;
    const void* region;
};

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
    uint32_t* queue_count;  // kQueueCounters: [0] near-face queue, [1] stuck queue (from k_assemble), [2] work
                            // counter of k_assemble, [3] work counter of k_slow, [4] near-face entries
                            // appended to the stuck ones (searched by k_slow_tail)
    unsigned long long* counters;
    int32_t* err;
    unsigned long long* guess_used;  // learned-guess statistics counter, or NULL
    int32_t guess_mlp;               // 1: points without a usable hint start where their first donor's network says
    int32_t guess_always;            // 1: every point of a set with a network gets a guess (hints ignored)
    SetDev s[OVS_MAX_SETS];
    XfFF xf[OVS_MAX_SETS];
    MotionDev m[OVS_MAX_GRIDS];
    GuessDev gn[OVS_MAX_GRIDS];
};

// The velocity transform of a set's points taken from its first donor grid, as one affine map of the donor
// velocity u_d and the receiver node's position x_r (receiver frame), composed in FP64 on the host:
//   RELATIVE  u_r = A u_d + B x_r + b,  A = R_r^T R_d,  B = R_r^T [Omega_d - Omega_r]x R_r,
//             b = R_r^T (V_d - V_r + Omega_d x (c_r - c_d))  (the two frame maps of Sec. 2.1 with x_in = R_r x_r + c_r)
//   ABSOLUTE  A = R_r^T R_d, B = 0, b = 0  (Sec. 2.3.1 eq. "velocity_non");  NONE  A = I, B = 0, b = 0
struct VelAffine {
    float A[9], B[9], b[3];
    int32_t pad;
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
    MotionF mf[OVS_MAX_GRIDS];
    FieldsDev fields[OVS_MAX_GRIDS];
    VelAffine va[OVS_MAX_SETS];  // per set, for its first donor grid (FP32 fields)
};

// Everything a step's kernels read, in one block of device memory written by one host-to-device copy per step
// (so that a captured step graph stays valid from one step to the next): the assembly's and the interpolation's
// parameters.
struct StepParams {
    AsmParams a;
    InterpParams i;
};

// error bits of the device status word
enum DevErr { kErrQueueOverflow = 1, kErrBadCell = 2, kErrBadNode = 4 };

// ------------------------------------------------------------------------------------------------
// FP32-pair ("double-float") arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2.  Error-free sum
// (Knuth, TAOCP vol. 2, Sec. 4.2.2, "TwoSum") and product (Dekker 1971, here with a fused multiply-add);
// written from those published definitions.  About 44-48 significant bits: enough to form point-minus-
// corner offsets of 1e-10 relative accuracy without FP64 instructions.
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // requires |a| >= |b| or a == 0
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    return fast_two_sum(p, e);
}

__device__ __forceinline__ bool ff_finite(ff a) { return fabsf(a.hi) <= 3.0e38f && fabsf(a.lo) <= 3.0e38f; }

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

// quotient: q1 = a.hi / b.hi, then one correction from the remainder a - q1 b (Dekker 1971)
__device__ __forceinline__ ff ff_div(ff a, ff b) {
    float q1 = __fdiv_rn(a.hi, b.hi);
    ff p = ff_mul(b, {q1, 0.f});
    ff r = ff_sub(a, p);
    float q2 = __fdiv_rn(r.hi, b.hi);
    return fast_two_sum(q1, q2);
}

__device__ __forceinline__ float ff_abs_f(ff a) { return fabsf(__fadd_rn(a.hi, a.lo)); }

// x_d = M x + t, all FP32 pairs
__device__ __forceinline__ void xf_apply(const XfFF& X, const ff x[3], ff xd[3]) {
    if (X.identity) {
        xd[0] = x[0];
        xd[1] = x[1];
        xd[2] = x[2];
        return;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        ff acc = {X.th[c], X.tl[c]};
#pragma unroll
        for (int k = 0; k < 3; ++k) acc = ff_add(acc, ff_mul({X.Mh[3 * c + k], X.Ml[3 * c + k]}, x[k]));
        xd[c] = acc;
    }
}

__device__ __forceinline__ ff split_double(double v) {
    float hi = (float)v;
    return {hi, (float)(v - (double)hi)};
}

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

// The frame maps in FP64 with a fixed order of operations, each product and sum rounded once (no fused
// multiply-add), so that the FP64 point a decision is taken on is defined bit for bit:
//   x_in_i = ((R_i0 x_0 + R_i1 x_1) + R_i2 x_2) + c_i              (Sec. 2.1: x_in = R x + c)
//   x_b_i  = (R_0i d_0 + R_1i d_1) + R_2i d_2,  d = x_in - c        (its inverse, R^T (x_in - c))
// An identity motion returns its input unchanged (which is also what these sums give).
__device__ __forceinline__ double3 to_inertial(const MotionDev& m, double3 x) {
    if (m.identity) return x;
    auto row = [&](int i, double c) {
        return __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(m.R[3 * i], x.x), __dmul_rn(m.R[3 * i + 1], x.y)),
                                   __dmul_rn(m.R[3 * i + 2], x.z)),
                         c);
    };
    return make_double3(row(0, m.c[0]), row(1, m.c[1]), row(2, m.c[2]));
}

__device__ __forceinline__ double3 to_body(const MotionDev& m, double3 xin) {
    if (m.identity) return xin;
    const double dx = __dsub_rn(xin.x, m.c[0]), dy = __dsub_rn(xin.y, m.c[1]), dz = __dsub_rn(xin.z, m.c[2]);
    auto col = [&](int i) {
        return __dadd_rn(__dadd_rn(__dmul_rn(m.R[i], dx), __dmul_rn(m.R[3 + i], dy)), __dmul_rn(m.R[6 + i], dz));
    };
    return make_double3(col(0), col(1), col(2));
}

__device__ __forceinline__ bool finite3(double3 p) {
    return isfinite(p.x) && isfinite(p.y) && isfinite(p.z);
}

// cell ids are < 2^27: 32-bit arithmetic
__device__ __forceinline__ void cell_ijk(const GridDev& g, int64_t cell, int& i, int& j, int& k) {
    uint32_t c = (uint32_t)cell, c0 = (uint32_t)g.C[0], c1 = (uint32_t)g.C[1];
    uint32_t q = c / c0;
    i = (int)(c - q * c0);
    k = (int)(q / c1);
    j = (int)(q - (uint32_t)k * c1);
}

__device__ __forceinline__ int64_t cell_id(const GridDev& g, int i, int j, int k) {
    return (int64_t)((uint32_t)i + (uint32_t)g.C[0] * ((uint32_t)j + (uint32_t)g.C[1] * (uint32_t)k));
}

// node id of corner (i+di, j+dj, k+dk) with periodic wrap
__device__ __forceinline__ int64_t corner_node(const GridDev& g, int i, int j, int k, int a) {
    int ii = i + (a & 1), jj = j + ((a >> 1) & 1), kk = k + ((a >> 2) & 1);
    if (ii == g.n[0]) ii = 0;
    if (jj == g.n[1]) jj = 0;
    if (kk == g.n[2]) kk = 0;
    return (int64_t)ii + (int64_t)g.n[0] * ((int64_t)jj + (int64_t)g.n[1] * kk);
}

// Index of finer bin (sx, sy, sz) in a crowded control cell, kSub per axis.
__device__ __forceinline__ int sub_index(int sx, int sy, int sz) { return sx + kSub * (sy + kSub * sz); }

// The finer bin along one axis of a coordinate x inside control cell bi (the control cells' own arithmetic,
// (x - lo) * inv_w, minus the cell's index, times kSub, floored and clamped): monotone in x, so a point inside a
// cell's padded box falls in one of the finer bins that box was registered in.
__device__ __forceinline__ int sub_coord(const GridDev& g, int c, double x, int bi) {
    const double t = ((x - g.lo[c]) * g.inv_w[c] - (double)bi) * (double)kSub;
    return (int)fmin(fmax(floor(t), 0.0), (double)(kSub - 1));
}

// The candidate list of the exhaustive search for a point in control cell b (which must be >= 0): the control
// cell's own list, or, in a crowded control cell, the list of the finer bin holding the point.
__device__ __forceinline__ void candidate_list(const GridDev& g, double3 p, int64_t b, const int32_t*& list,
                                               int32_t& r0, int32_t& r1) {
    list = g.bin_cells;
    r0 = __ldg(g.bin_start + b);
    r1 = __ldg(g.bin_start + b + 1);
    if (g.ncrowd <= 0 || r1 - r0 <= kCrowdedCount) return;
    int lo = 0, hi = g.ncrowd - 1;
    while (lo < hi) {  // the split control cells are sorted by id
        const int mid = (lo + hi) >> 1;
        if (__ldg(g.crowd + mid) < b) lo = mid + 1; else hi = mid;
    }
    if (__ldg(g.crowd + lo) != (int32_t)b) return;
    const int bx = (int)(b % g.nb[0]), by = (int)((b / g.nb[0]) % g.nb[1]), bz = (int)(b / ((int64_t)g.nb[0] * g.nb[1]));
    const int64_t sb = (int64_t)lo * kSub3 + sub_index(sub_coord(g, 0, p.x, bx), sub_coord(g, 1, p.y, by),
                                                       sub_coord(g, 2, p.z, bz));
    list = g.sub_cells;
    r0 = __ldg(g.sub_start + sb);
    r1 = __ldg(g.sub_start + sb + 1);
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

// A cell with a blanked corner node never donates (Sec. 2.4); the flag sits in the record's first pad word
// (nonzero bits: blocked), written by ovs_set_iblank and zero from the record build.
__device__ __forceinline__ bool rec_blocked(const CellRec& r) { return __float_as_uint(r.pad[0]) != 0u; }
__device__ __forceinline__ bool cell_blocked(const CellRec* rec, int64_t cell) {
    return __float_as_uint(__ldg(&rec[cell].pad[0])) != 0u;
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
        double x0 = (double)r.x0h[c] + (double)r.x0l[c];
        lo[c] = x0 + (double)mn[c] - pad;
        hi[c] = x0 + (double)mx[c] + pad;
    }
}

// FP32 Newton on the monomial form.  Returns true if the last step was below tolerance.
__device__ __forceinline__ bool newton32(const CellRec& r, float dx, float dy, float dz, float& u, float& v,
                                         float& w, int maxit = kNewtonMaxIt32, int* iters = nullptr) {
    const float* a = r.a;
    bool conv = false;
#pragma unroll 1
    for (int it = 0; it < maxit; ++it) {
        if (iters) ++*iters;
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
        float inv = -__frcp_rn(det);  // the correctly rounded reciprocal, as 1.0f / det
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
static __device__ __noinline__ bool newton64_contains(const GridDev& g, int64_t cell, double3 p, double& u, double& v,
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

// The donor predicate in FP32-pair arithmetic (~44 significant bits) on the node coordinates' FP32 pairs,
// started at (u,v,w): Newton's iteration for the trilinear map with the residual F(xi) = x(xi) - p formed in
// FP32 pairs (the map as the weights N_a(xi) of the corners' offsets X_a - X_0) and the step solved with the
// Jacobian in FP32 (iterative refinement: an FP32 Jacobian changes only how fast the steps shrink, by a factor of
// about 1e-7 times its condition number per step, not where they lead).  Converged when a step is <= 1e-12, or
// when the steps stop shrinking geometrically below 1e-9 (they have reached the pair arithmetic's rounding noise).
// Returns 1 (the cell holds the point), 0 (it does not) or -1 (undecided: not converged; the steps shrinking by
// less than a factor 0.9; the noise so large (> 1e-11) that the FP64 definition might itself not reach its 1e-13
// tolerance; or a local coordinate within the band of a window bound, where only the FP64 predicate may decide).
// Away from that band the FP64 definition gives the same answer, because both iterations approach the same root
// to within the band.
static __device__ __noinline__ int newton_ff(const GridDev& g, int64_t cell, const ff p[3], float u0, float v0, float w0,
                                             double& u, double& v, double& w) {
    int i, j, k;
    cell_ijk(g, cell, i, j, k);
    const int64_t nn = g.nnodes;
    ff X0[3], E[7][3], d[3];
    float A[7][3];  // FP32 monomial coefficients of the map (for the Jacobian)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int64_t n0 = corner_node(g, i, j, k, 0);
        X0[c] = {__ldg(g.xff + 2 * c * nn + n0), __ldg(g.xff + (2 * c + 1) * nn + n0)};
    }
#pragma unroll
    for (int a = 1; a < 8; ++a) {
        const int64_t nd = corner_node(g, i, j, k, a);
#pragma unroll
        for (int c = 0; c < 3; ++c)
            E[a - 1][c] = ff_sub({__ldg(g.xff + 2 * c * nn + nd), __ldg(g.xff + (2 * c + 1) * nn + nd)}, X0[c]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float e1 = E[0][c].hi, e2 = E[1][c].hi, e3 = E[2][c].hi, e4 = E[3][c].hi, e5 = E[4][c].hi,
                    e6 = E[5][c].hi, e7 = E[6][c].hi;
        A[0][c] = e1;
        A[1][c] = e2;
        A[2][c] = e4;
        A[3][c] = e3 - e1 - e2;
        A[4][c] = e6 - e2 - e4;
        A[5][c] = e5 - e1 - e4;
        A[6][c] = e7 - e3 - e5 - e6 + e1 + e2 + e4;
        d[c] = ff_sub(p[c], X0[c]);
    }
    ff U = {u0, 0.f}, V = {v0, 0.f}, W = {w0, 0.f};
    bool conv = false;
    float m_prev = 3.4e38f, m_noise = 0.f, rho = 0.f;
#pragma unroll 1
    for (int it = 0; it < kNewtonMaxIt64; ++it) {
        // residual: sum over corners a = 1..7 of N_a(xi) (X_a - X_0), minus (p - X_0), corner by corner
        const ff one = {1.f, 0.f};
        const ff mu = ff_sub(one, U), mv = ff_sub(one, V), mw = ff_sub(one, W);
        ff f0 = ff_neg(d[0]), f1 = ff_neg(d[1]), f2 = ff_neg(d[2]);
#pragma unroll 1
        for (int a = 1; a < 8; ++a) {
            const ff N = ff_mul(ff_mul((a & 1) ? U : mu, (a & 2) ? V : mv), (a & 4) ? W : mw);
            f0 = ff_add(f0, ff_mul(N, E[a - 1][0]));
            f1 = ff_add(f1, ff_mul(N, E[a - 1][1]));
            f2 = ff_add(f2, ff_mul(N, E[a - 1][2]));
        }
        const float F[3] = {__fadd_rn(f0.hi, f0.lo), __fadd_rn(f1.hi, f1.lo), __fadd_rn(f2.hi, f2.lo)};
        // step with the FP32 Jacobian at the FP32 iterate
        const float fu = U.hi, fv = V.hi, fw = W.hi;
        float Ju[3], Jv[3], Jw[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Ju[c] = fmaf(A[3][c], fv, fmaf(A[5][c], fw, fmaf(A[6][c], fv * fw, A[0][c])));
            Jv[c] = fmaf(A[3][c], fu, fmaf(A[4][c], fw, fmaf(A[6][c], fu * fw, A[1][c])));
            Jw[c] = fmaf(A[4][c], fv, fmaf(A[5][c], fu, fmaf(A[6][c], fu * fv, A[2][c])));
        }
        const float cvw[3] = {Jv[1] * Jw[2] - Jv[2] * Jw[1], Jv[2] * Jw[0] - Jv[0] * Jw[2], Jv[0] * Jw[1] - Jv[1] * Jw[0]};
        const float cwu[3] = {Jw[1] * Ju[2] - Jw[2] * Ju[1], Jw[2] * Ju[0] - Jw[0] * Ju[2], Jw[0] * Ju[1] - Jw[1] * Ju[0]};
        const float cuv[3] = {Ju[1] * Jv[2] - Ju[2] * Jv[1], Ju[2] * Jv[0] - Ju[0] * Jv[2], Ju[0] * Jv[1] - Ju[1] * Jv[0]};
        const float det = Ju[0] * cvw[0] + Ju[1] * cvw[1] + Ju[2] * cvw[2];
        if (!(fabsf(det) > 0.f)) return -1;
        const float inv = -__frcp_rn(det);
        const float du = (F[0] * cvw[0] + F[1] * cvw[1] + F[2] * cvw[2]) * inv;
        const float dv = (F[0] * cwu[0] + F[1] * cwu[1] + F[2] * cwu[2]) * inv;
        const float dw = (F[0] * cuv[0] + F[1] * cuv[1] + F[2] * cuv[2]) * inv;
        U = ff_add(U, {du, 0.f});
        V = ff_add(V, {dv, 0.f});
        W = ff_add(W, {dw, 0.f});
        const float m = fmaxf(fabsf(du), fmaxf(fabsf(dv), fabsf(dw)));
        if (!(m < 1e30f) || !ff_finite(U) || !ff_finite(V) || !ff_finite(W)) return 0;
        if (m <= 1e-12f) {
            conv = true;
            rho = m_prev < 3e38f ? m / m_prev : 0.f;
            break;
        }
        if (m < 1e-9f && m > 0.5f * m_prev) {  // no longer shrinking fast: at the rounding noise (or contracting slowly)
            conv = true;
            m_noise = m;
            rho = m / m_prev;
            break;
        }
        m_prev = m;
    }
    // a slow contraction (a nearly singular FP32 Jacobian) leaves the iterate up to m rho / (1 - rho) away
    if (!conv || m_noise > 1e-11f || rho >= 0.9f) return -1;
    // undecided band: 1e-12 plus the FP32-pair error of the point and corners (~4e-14 of the coordinates'
    // magnitude) measured in local-coordinate units of the cell's shortest edge; at least 8 times the distance the
    // remaining steps can still move the iterate when the iteration stopped at its rounding noise
    float pm = fmaxf(fabsf(p[0].hi), fmaxf(fabsf(p[1].hi), fabsf(p[2].hi))) +
               fmaxf(fabsf(X0[0].hi), fmaxf(fabsf(X0[1].hi), fabsf(X0[2].hi)));
    float hmin = 3.4e38f;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        float n2 = A[q][0] * A[q][0] + A[q][1] * A[q][1] + A[q][2] * A[q][2];
        hmin = fminf(hmin, sqrtf(n2));
    }
    const float band = fmaxf(1e-12f + 4e-14f * pm / hmin, 8.f * m_noise / (1.f - rho));
    ff q[3] = {U, V, W};
    bool in = true, amb = false;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float lo = __fadd_rn(q[c].hi, q[c].lo);                    // ~ xi (accurate near 0)
        ff one = ff_sub(q[c], {1.f, 0.f});
        float hi = __fadd_rn(one.hi, one.lo);                       // ~ xi - 1 (accurate near 1)
        float dlo = lo - (float)kWinLo, dhi = hi - (float)(kWinHi - 1.0);
        if (fabsf(dlo) <= band || fabsf(dhi) <= band) amb = true;
        if (dlo < 0.f || dhi > 0.f) in = false;
    }
    if (amb) return -1;
    u = (double)U.hi + (double)U.lo;
    v = (double)V.hi + (double)V.lo;
    w = (double)W.hi + (double)W.lo;
    return in ? 1 : 0;
}

// The donor predicate: FP32-pair Newton, and the FP64 definition (on the FP64 point p64) only where the
// FP32-pair iteration cannot decide.
template <class P64>
__device__ __forceinline__ bool contains_exact(const GridDev& g, int64_t cell, const ff p[3], const P64& p64, float u0,
                                               float v0, float w0, double& u, double& v, double& w) {
    int r = newton_ff(g, cell, p, u0, v0, w0, u, v, w);
    if (r >= 0) return r == 1;
    u = u0;
    v = v0;
    w = w0;
    return newton64_contains(g, cell, p64(), u, v, w);
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// host-side launchers (defined in the .cu files)
// orient: 3 device counters (cells right-handed, left-handed, folded or degenerate), zeroed here
cudaError_t launch_build_records(const GridDev& g, CellRec* rec, float* xff, double* partials, int nblocks,
                                 double* out9, unsigned long long* orient, cudaStream_t st);
cudaError_t launch_bin_count(const GridDev& g, uint32_t* counts, cudaStream_t st);
// exclusive scan of n counts into start[0..n] (start[n] = total); block_sums: one entry per tile of
// kScanTileElems counts
constexpr int kScanTileElems = 2048;
cudaError_t launch_scan(const uint32_t* counts, int32_t* start, int64_t n, uint32_t* block_sums, cudaStream_t st);
// marks each cell of g blocked (a corner with iblank 0) or not (iblank NULL: none blocked)
cudaError_t launch_mark_blocked(const GridDev& g, const uint8_t* iblank, cudaStream_t st);
// appends to crowd the control cells listing more than thr cells (n: their count, which may exceed cap)
cudaError_t launch_crowd_mark(const GridDev& g, int64_t nbins, int32_t thr, int32_t* crowd, uint32_t* n, int cap,
                              cudaStream_t st);
// per finer bin of the g.ncrowd crowded control cells (g.crowd), the number of cells registered (counts) / their
// lists (cells at start, cursor zeroed)
cudaError_t launch_sub_count(const GridDev& g, uint32_t* counts, cudaStream_t st);
cudaError_t launch_sub_fill(const GridDev& g, const int32_t* start, uint32_t* cursor, int32_t* cells, cudaStream_t st);
cudaError_t launch_bin_fill(const GridDev& g, const int32_t* start, uint32_t* cursor, int32_t* cells, int32_t* rep,
                            cudaStream_t st);
size_t scan_scratch_elems(int64_t n);
// ev: 3 optional events (before the fast kernel, after it, after the slow kernels); 2 for interpolation.
// interp: 0 assembly only; 1 / 2: the kernels also interpolate FP32 / FP64 fields (dS->i) for every point they
// decide.  asm_bps / slow_bps: blocks per SM of the persistent assembly grid and of each half of the slow-path
// grid (0: defaults)
cudaError_t launch_assemble(const StepParams* dS, int interp, bool mlp, uint32_t* queue_count, const GridDev* dgrids,
                            int nsm, int asm_bps, int slow_bps, cudaStream_t st, cudaEvent_t const* ev);
// blocks of k_interp resident per SM (occupancy calculator), or a negative CUDA error
int interp_default_blocks_per_sm(bool f64);
// bps: blocks per SM of the persistent grid (0: the occupancy calculator's figure)
cudaError_t launch_interp(const InterpParams* dI, bool f64, const GridDev* dgrids, int nsm, int bps, cudaStream_t st,
                          cudaEvent_t const* ev);

}  // namespace ovs
