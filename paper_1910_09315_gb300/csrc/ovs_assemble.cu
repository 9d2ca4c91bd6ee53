// Donor search (Sec. 2.2.5, Algorithm 3 "donor search", with Newton inversion of the trilinear map):
//
//   k_assemble       one thread per query point: frame map (FP64), localisation (hint | control cell),
//                    FP32 walk over 128-byte cell records with FP32 Newton; points that end strictly
//                    inside a cell (every local coordinate at least 1e-4 from a face) are final.
//                    Points near a face, points in FP64 precision mode and stuck walks are compacted
//                    (warp ballot + one atomic per warp) into the slow queue.
//   k_assemble_slow  one thread per queued point: FP64 Newton on the exact node coordinates over the
//                    cells sharing the near face/edge/corner, lowest linear id first; if none holds the
//                    point, the exhaustive search of the point's control cell of Sec. 2.2.5 (the paper's
//                    brute-force fallback) with the same FP64 predicate.  Then the later grids of the
//                    set's priority list (Sec. 2.4 item 1).
#include "ovs_internal.cuh"

namespace ovs {

namespace {

constexpr int kAsmThreads = 256;

enum WalkResult { kWalkFound = 0, kWalkStuck = 1 };

// FP32 walk from `cell`.  On kWalkFound, cell/u/v/w hold a cell whose FP32 local coordinates lie within
// kAccept32 of [0,1]^3.
__device__ __forceinline__ int walk32(const GridDev& g, double3 p, int64_t& cell, float& u, float& v, float& w,
                                      int max_walk, int& steps) {
    int i, j, k;
    cell_ijk(g, cell, i, j, k);
    u = v = w = 0.5f;
#pragma unroll 1
    for (int s = 0; s < max_walk; ++s) {
        ++steps;
        CellRec r;
        load_rec(g.rec, cell, r);
        float dx = (float)(p.x - r.x0[0]), dy = (float)(p.y - r.x0[1]), dz = (float)(p.z - r.x0[2]);
        bool conv = newton32(r, dx, dy, dz, u, v, w);
        if (!(fabsf(u) < 1e30f && fabsf(v) < 1e30f && fabsf(w) < 1e30f)) return kWalkStuck;
        bool in = u >= -kAccept32 && u <= 1.f + kAccept32 && v >= -kAccept32 && v <= 1.f + kAccept32 &&
                  w >= -kAccept32 && w <= 1.f + kAccept32;
        if (in && conv) return kWalkFound;
        // step toward the point by the sign (and size, up to kMaxJump) of the local coordinates: the
        // sign test of the paper's walk, applied to Newton's local coordinates
        float q[3] = {u, v, w};
        int cur[3] = {i, j, k};
        int nxt[3];
        bool moved = false;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            int jm = 0;
            if (q[m] < -kAccept32) jm = max(-kMaxJump, (int)floorf(fmaxf(q[m], -1e6f)));
            else if (q[m] > 1.f + kAccept32) jm = min(kMaxJump, (int)floorf(fminf(q[m], 1e6f)));
            int t = cur[m] + jm;
            if (g.per[m]) {
                t %= g.C[m];
                if (t < 0) t += g.C[m];
            } else {
                t = min(max(t, 0), g.C[m] - 1);
            }
            nxt[m] = t;
            int applied = t - cur[m];
            if (g.per[m] && applied != jm) applied = jm;  // wrapped: same local shift
            if (applied != 0) moved = true;
            q[m] = conv ? fminf(fmaxf(q[m] - (float)applied, -1.f), 2.f) : 0.5f;
        }
        if (!moved) return kWalkStuck;
        i = nxt[0];
        j = nxt[1];
        k = nxt[2];
        cell = cell_id(g, i, j, k);
        u = q[0];
        v = q[1];
        w = q[2];
    }
    return kWalkStuck;
}

__device__ __forceinline__ void write_donor(const AsmParams& P, int64_t t, int32_t gd, int64_t cell, double u,
                                            double v, double w, uint8_t status) {
    P.out_grid[t] = gd;
    P.out_cell[t] = (int32_t)cell;
    if (P.xi_f64) {
        double* xi = (double*)P.out_xi;
        xi[t] = u;
        xi[P.total + t] = v;
        xi[2 * P.total + t] = w;
    } else {
        float* xi = (float*)P.out_xi;
        xi[t] = (float)u;
        xi[P.total + t] = (float)v;
        xi[2 * P.total + t] = (float)w;
    }
    P.out_status[t] = status;
}

__device__ __forceinline__ void write_none(const AsmParams& P, int64_t t, uint8_t status) {
    P.out_grid[t] = -1;
    P.out_cell[t] = -1;
    if (P.xi_f64) {
        double* xi = (double*)P.out_xi;
        xi[t] = xi[P.total + t] = xi[2 * P.total + t] = __longlong_as_double(0x7ff8000000000000ll);
    } else {
        float* xi = (float*)P.out_xi;
        xi[t] = xi[P.total + t] = xi[2 * P.total + t] = __int_as_float(0x7fc00000);
    }
    P.out_status[t] = status;
}

__device__ __forceinline__ void warp_add(unsigned long long* ctr, unsigned v) {
    unsigned s = __reduce_add_sync(0xffffffffu, v);
    if (lane_id() == 0 && s) atomicAdd(ctr, (unsigned long long)s);
}

__global__ void __launch_bounds__(kAsmThreads) k_assemble(const __grid_constant__ AsmParams P,
                                                          const GridDev* __restrict__ G) {
    const int64_t t = blockIdx.x * (int64_t)kAsmThreads + threadIdx.x;
    const bool active = t < P.total;
    bool slow = false;
    SlowEntry e;
    int steps = 0;
    if (active) {
        const int si = find_set(P.s, P.nsets, t);
        const SetDev& s = P.s[si];
        const int32_t node = __ldg(s.node_ids + (t - s.begin));
        const GridDev& gr = G[s.receiver];
        const bool node_ok = node >= 0 && node < gr.nnodes;
        double3 xin = make_double3(0.0, 0.0, 0.0);
        if (node_ok) {
            double3 xr = make_double3(__ldg(gr.x + node), __ldg(gr.y + node), __ldg(gr.z + node));
            xin = to_inertial(P.m[s.receiver], xr);
        } else {
            atomicOr(P.err, kErrBadNode);
        }
        if (!node_ok || !finite3(xin)) {
            write_none(P, t, OVS_STATUS_BADINPUT);
        } else {
            bool done = false;
            for (int di = 0; di < s.ndonor && !done && !slow; ++di) {
                const int gd = s.donors[di];
                const GridDev& g = G[gd];
                double3 p = to_body(P.m[gd], xin);
                int64_t b = point_bin(g, p);
                if (b < 0) continue;
                int64_t cell = -1;
                if (P.guess == OVS_GUESS_HINT) {
                    uint32_t h = gr.hint[node];
                    if (h != kNoHint && (int)(h >> kCellBits) == gd) cell = h & ((1u << kCellBits) - 1);
                    if (cell >= g.ncells) cell = -1;
                }
                if (cell < 0) {
                    // lowest registered cell of the control cell; >= ncells marks an empty control cell, where
                    // no cell of this grid can hold the point
                    cell = __ldg(g.bin_rep + b);
                    if (cell < 0 || cell >= g.ncells) continue;
                }
                float u, v, w;
                int r = walk32(g, p, cell, u, v, w, P.max_walk, steps);
                e.t = (int32_t)t;
                e.di = di;
                if (r == kWalkFound) {
                    float mu = fminf(u, 1.f - u), mv = fminf(v, 1.f - v), mw = fminf(w, 1.f - w);
                    bool near = fminf(mu, fminf(mv, mw)) < kNearFace;
                    if (near || P.xi_f64) {
                        slow = true;
                        e.cell = (int32_t)cell;
                        e.xi[0] = u;
                        e.xi[1] = v;
                        e.xi[2] = w;
                    } else {
                        write_donor(P, t, gd, cell, u, v, w, OVS_STATUS_FOUND);
                        gr.hint[node] = ((uint32_t)gd << kCellBits) | (uint32_t)cell;
                        done = true;
                    }
                } else {
                    slow = true;
                    e.cell = -1;
                    e.xi[0] = e.xi[1] = e.xi[2] = 0.5f;
                }
            }
            if (!done && !slow) write_none(P, t, OVS_STATUS_ORPHAN);
        }
    }
    // warp-aggregated append to the slow queue
    unsigned mask = __ballot_sync(0xffffffffu, slow);
    if (mask) {
        unsigned lane = lane_id();
        int leader = __ffs(mask) - 1;
        uint32_t base = 0;
        if ((int)lane == leader) base = atomicAdd(P.queue_count, (uint32_t)__popc(mask));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (slow) {
            uint32_t idx = base + __popc(mask & ((1u << lane) - 1u));
            if (idx < P.queue_cap) P.queue[idx] = e;
            else atomicOr(P.err, kErrQueueOverflow);
        }
    }
    if (P.stats) {
        warp_add(P.counters + kCtrPoints, active ? 1u : 0u);
        warp_add(P.counters + kCtrWalk, (unsigned)steps);
    }
}

// Candidate cells sharing the near face / edge / corner of `cell` (FP32 local coordinates within kNearFace
// of a face), in ascending linear id.  Returns their count (<= 8) and the offsets to shift the FP32 guess.
__device__ int near_candidates(const GridDev& g, int64_t cell, const float xi32[3], int64_t ids[8], int off[8][3]) {
    int ijk[3];
    cell_ijk(g, cell, ijk[0], ijk[1], ijk[2]);
    int lo[3], hi[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        lo[m] = xi32[m] < kNearFace ? -1 : 0;
        hi[m] = xi32[m] > 1.f - kNearFace ? 1 : 0;
    }
    int nc = 0;
    for (int oz = lo[2]; oz <= hi[2]; ++oz)
        for (int oy = lo[1]; oy <= hi[1]; ++oy)
            for (int ox = lo[0]; ox <= hi[0]; ++ox) {
                int o[3] = {ox, oy, oz}, q[3];
                bool ok = true;
                for (int m = 0; m < 3; ++m) {
                    q[m] = ijk[m] + o[m];
                    if (g.per[m]) {
                        if (q[m] < 0) q[m] += g.C[m];
                        if (q[m] >= g.C[m]) q[m] -= g.C[m];
                    } else if (q[m] < 0 || q[m] >= g.C[m]) {
                        ok = false;
                    }
                }
                if (!ok) continue;
                int64_t id = cell_id(g, q[0], q[1], q[2]);
                int pos = nc++;
                while (pos > 0 && ids[pos - 1] > id) {
                    ids[pos] = ids[pos - 1];
                    off[pos][0] = off[pos - 1][0];
                    off[pos][1] = off[pos - 1][1];
                    off[pos][2] = off[pos - 1][2];
                    --pos;
                }
                ids[pos] = id;
                off[pos][0] = o[0];
                off[pos][1] = o[1];
                off[pos][2] = o[2];
            }
    return nc;
}

// Warp-cooperative lowest-id FP64 decision over the near candidates: lane q tests candidate q; the lowest
// lane (= lowest id) whose cell holds the point wins.  All 32 lanes must call this.
__device__ bool neighbourhood64_warp(const GridDev& g, double3 p, int64_t cell, const float xi32[3],
                                     int64_t& out_cell, double& u, double& v, double& w) {
    int64_t ids[8];
    int off[8][3];
    int nc = near_candidates(g, cell, xi32, ids, off);
    const int lane = (int)lane_id();
    bool hit = false;
    double a = 0, b = 0, c = 0;
    int64_t mine = -1;
    if (lane < nc) {
        // select this lane's candidate without dynamic register indexing
        int o0 = 0, o1 = 0, o2 = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (q == lane) {
                mine = ids[q];
                o0 = off[q][0];
                o1 = off[q][1];
                o2 = off[q][2];
            }
        a = (double)xi32[0] - o0;
        b = (double)xi32[1] - o1;
        c = (double)xi32[2] - o2;
        hit = newton64_contains(g, mine, p, a, b, c);
    }
    unsigned m = __ballot_sync(0xffffffffu, hit);
    if (!m) return false;
    int src = __ffs(m) - 1;
    out_cell = __shfl_sync(0xffffffffu, mine, src);
    u = __shfl_sync(0xffffffffu, a, src);
    v = __shfl_sync(0xffffffffu, b, src);
    w = __shfl_sync(0xffffffffu, c, src);
    return true;
}

// Warp-cooperative exhaustive search of the point's control cell (Sec. 2.2.5 brute-force fallback): lanes
// split the registered cells; a cell is rejected by its padded box (FP32, relative to its corner 0) or by a
// converged FP32 Newton that lands clearly outside; the rest get the FP64 predicate.  Lowest id wins.
__device__ bool exhaustive64_warp(const GridDev& g, double3 p, int64_t bin, int64_t& out_cell, double& u, double& v,
                                  double& w) {
    const int lane = (int)lane_id();
    uint32_t best = 0xFFFFFFFFu;
    double bu = 0, bv = 0, bw = 0;
    int32_t r0 = __ldg(g.bin_start + bin), r1 = __ldg(g.bin_start + bin + 1);
    for (int32_t r = r0 + lane; r < r1; r += 32) {
        uint32_t c = (uint32_t)__ldg(g.bin_cells + r);
        if (c >= best) continue;
        CellRec rec;
        load_rec(g.rec, c, rec);
        float dx = (float)(p.x - rec.x0[0]), dy = (float)(p.y - rec.x0[1]), dz = (float)(p.z - rec.x0[2]);
        float d[3] = {dx, dy, dz};
        bool inbox = true;
        float diag2 = 0.f;
        float mn[3], mx[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float a1 = rec.a[k], a2 = rec.a[3 + k], a3 = rec.a[6 + k], a4 = rec.a[9 + k], a5 = rec.a[12 + k],
                  a6 = rec.a[15 + k], a7 = rec.a[18 + k];
            float e[8] = {0.f, a1, a2, a1 + a2 + a4, a3, a1 + a3 + a6, a2 + a3 + a5,
                          a1 + a2 + a3 + a4 + a5 + a6 + a7};
            mn[k] = e[0];
            mx[k] = e[0];
#pragma unroll
            for (int q = 1; q < 8; ++q) {
                mn[k] = fminf(mn[k], e[q]);
                mx[k] = fmaxf(mx[k], e[q]);
            }
            diag2 += (mx[k] - mn[k]) * (mx[k] - mn[k]);
        }
        float pad = 4e-6f * sqrtf(diag2) + 1e-30f;
#pragma unroll
        for (int k = 0; k < 3; ++k) inbox = inbox && d[k] >= mn[k] - pad && d[k] <= mx[k] + pad;
        if (!inbox) continue;
        float fu = 0.5f, fv = 0.5f, fw = 0.5f;
        bool conv = newton32(rec, dx, dy, dz, fu, fv, fw);
        const float far = 0.05f;
        if (conv && (fu < -far || fu > 1.f + far || fv < -far || fv > 1.f + far || fw < -far || fw > 1.f + far))
            continue;
        double a = 0.5, b = 0.5, cc = 0.5;
        if (newton64_contains(g, c, p, a, b, cc)) {
            best = c;
            bu = a;
            bv = b;
            bw = cc;
        }
    }
    uint32_t wbest = __reduce_min_sync(0xffffffffu, best);
    if (wbest == 0xFFFFFFFFu) return false;
    unsigned m = __ballot_sync(0xffffffffu, best == wbest);
    int src = __ffs(m) - 1;
    out_cell = wbest;
    u = __shfl_sync(0xffffffffu, bu, src);
    v = __shfl_sync(0xffffffffu, bv, src);
    w = __shfl_sync(0xffffffffu, bw, src);
    return true;
}

constexpr int kSlowThreads = 256;

// One warp per queued point.
__global__ void __launch_bounds__(kSlowThreads) k_assemble_slow(const __grid_constant__ AsmParams P,
                                                                const GridDev* __restrict__ G) {
    uint32_t count = *P.queue_count;
    if (count > P.queue_cap) count = (uint32_t)P.queue_cap;
    const int lane = (int)lane_id();
    const uint32_t warp = (blockIdx.x * kSlowThreads + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * kSlowThreads) >> 5;
    unsigned refined = 0, fallback = 0;
    for (uint32_t q = warp; q < count; q += nwarps) {
        SlowEntry e = P.queue[q];
        const int64_t t = e.t;
        const int si = find_set(P.s, P.nsets, t);
        const SetDev& s = P.s[si];
        const int32_t node = __ldg(s.node_ids + (t - s.begin));
        const GridDev& gr = G[s.receiver];
        double3 xr = make_double3(gr.x[node], gr.y[node], gr.z[node]);
        double3 xin = to_inertial(P.m[s.receiver], xr);
        bool done = false;
        for (int di = e.di; di < s.ndonor && !done; ++di) {
            const int gd = s.donors[di];
            const GridDev& g = G[gd];
            double3 p = to_body(P.m[gd], xin);
            int64_t b = point_bin(g, p);
            if (b < 0) continue;
            int64_t cell = -1;
            double u = 0, v = 0, w = 0;
            uint8_t st = OVS_STATUS_FOUND | OVS_STATUS_REFINED;
            bool ok = false;
            if (di == e.di && e.cell >= 0) ok = neighbourhood64_warp(g, p, e.cell, e.xi, cell, u, v, w);
            if (!ok) {
                ok = exhaustive64_warp(g, p, b, cell, u, v, w);
                st |= OVS_STATUS_FALLBACK;
                ++fallback;
            }
            if (ok) {
                if (lane == 0) {
                    write_donor(P, t, gd, cell, u, v, w, st);
                    gr.hint[node] = ((uint32_t)gd << kCellBits) | (uint32_t)cell;
                }
                done = true;
                ++refined;
            }
        }
        if (!done && lane == 0) write_none(P, t, OVS_STATUS_ORPHAN | OVS_STATUS_FALLBACK);
    }
    if (P.stats && lane == 0) {
        if (refined) atomicAdd(P.counters + kCtrRefined, (unsigned long long)refined);
        if (fallback) atomicAdd(P.counters + kCtrFallback, (unsigned long long)fallback);
    }
}

}  // namespace

cudaError_t launch_assemble(const AsmParams& P, const GridDev* dgrids, cudaStream_t st, cudaEvent_t const* ev) {
    cudaError_t err = cudaMemsetAsync(P.queue_count, 0, sizeof(uint32_t), st);
    if (err != cudaSuccess) return err;
    int64_t blocks = (P.total + kAsmThreads - 1) / kAsmThreads;
    if (ev && ev[0]) cudaEventRecord(ev[0], st);
    k_assemble<<<(unsigned)blocks, kAsmThreads, 0, st>>>(P, dgrids);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    if (ev && ev[1]) cudaEventRecord(ev[1], st);
    k_assemble_slow<<<152 * 4, kSlowThreads, 0, st>>>(P, dgrids);
    if (ev && ev[2]) cudaEventRecord(ev[2], st);
    return cudaGetLastError();
}

}  // namespace ovs
