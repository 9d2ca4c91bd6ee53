// Donor search (Sec. 2.2.5, Algorithm 3 "donor search", with Newton inversion of the trilinear map):
//
//   k_assemble       one thread per query point, no FP64 instruction on its common path: frame map of the
//                    receiver node (FP32 pairs) into the first donor's frame, localisation (per-node hint |
//                    control cell), FP32 walk over 128-byte cell records with FP32 Newton.  Points that end
//                    strictly inside a cell (every local coordinate at least 1e-4 from a face) are final.
//                    Points near a face, points in FP64 precision mode and stuck walks are compacted (warp
//                    ballot + one atomic per warp) into the slow queue.
//   k_slow           then, in one persistent kernel whose blocks take units from a counter: the stuck entries,
//                    one block each (the exhaustive search of the point's control cell of Sec. 2.2.5, the paper's
//                    brute-force fallback: all threads filter the list, the exact test runs on every survivor at
//                    once; then the later grids of the set's priority list, Sec. 2.4 item 1), and the points near
//                    a face, one warp each (the donor predicate, FP32-pair Newton on the node coordinates and FP64
//                    where that cannot decide, over the cells sharing the near faces / edges / corner, one lane
//                    each, lowest linear id first; a point none of them holds joins the stuck entries).
//   k_slow_tail      the stuck entries k_slow appended, a block each (usually none).
//
// In a call that also interpolates (ovs_assemble_interpolate) the kernels go on, for every point whose donor
// they decide, to the trilinear interpolation of u, v, w, p and the frame velocity transform (Sec. 2.2.6,
// Sec. 2.1; ovs_fields.cuh) while donor, local coordinates and receiver node are at hand: one pass per point,
// no separate interpolation kernel re-reading the donor records.
#include "ovs_fields.cuh"
#include "ovs_mlp.cuh"

namespace ovs {

namespace {

constexpr int kAsmThreads = 256;
constexpr int kAsmMinBlocks = 2;  // 128 registers a thread: no spills (3 blocks spill about 0.6 KB a thread)

enum WalkResult { kWalkFound = 0, kWalkStuck = 1 };

// FP32 walk from `cell` toward the donor-frame point xd (FP32 pairs).  On kWalkFound, cell/u/v/w hold a cell
// whose FP32 local coordinates lie within kAccept32 of [0,1]^3.
__device__ __forceinline__ int walk32(const GridDev& g, const ff xd[3], int64_t& cell, float& u, float& v, float& w,
                                      float& tau, int max_walk, int& steps, int& iters, bool& blocked, int& i, int& j,
                                      int& k) {
    cell_ijk(g, cell, i, j, k);
    u = v = w = 0.5f;
#pragma unroll 1
    for (int s = 0; s < max_walk; ++s) {
        ++steps;
        CellRec r;
        load_rec(g.rec, cell, r);
        // point minus corner 0: the high parts cancel exactly near the cell, the low parts carry the rest
        float dx = __fadd_rn(__fsub_rn(xd[0].hi, r.x0h[0]), __fsub_rn(xd[0].lo, r.x0l[0]));
        float dy = __fadd_rn(__fsub_rn(xd[1].hi, r.x0h[1]), __fsub_rn(xd[1].lo, r.x0l[1]));
        float dz = __fadd_rn(__fsub_rn(xd[2].hi, r.x0h[2]), __fsub_rn(xd[2].lo, r.x0l[2]));
        bool conv = newton32(r, dx, dy, dz, u, v, w, kNewtonMaxIt32, &iters);
        if (!(fabsf(u) < 1e30f && fabsf(v) < 1e30f && fabsf(w) < 1e30f)) return kWalkStuck;
        bool in = u >= -kAccept32 && u <= 1.f + kAccept32 && v >= -kAccept32 && v <= 1.f + kAccept32 &&
                  w >= -kAccept32 && w <= 1.f + kAccept32;
        if (in && conv) {
            tau = near_tau(r, u, v, w);
            blocked = rec_blocked(r);
            return kWalkFound;
        }
        // step toward the point by the sign (and size, up to kMaxJump) of the local coordinates: the sign
        // test of the paper's walk, applied to Newton's local coordinates
        float q[3] = {u, v, w};
        int cur[3] = {i, j, k};
        int nxt[3];
        bool moved = false;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            int jm = 0;
            const int jmax = g.per[m] ? kMaxJumpPeriodic : kMaxJump;
            if (q[m] < -kAccept32) jm = max(-jmax, (int)floorf(fmaxf(q[m], -1e6f)));
            else if (q[m] > 1.f + kAccept32) jm = min(jmax, (int)floorf(fminf(q[m], 1e6f)));
            int t = cur[m] + jm;
            int applied;
            if (g.per[m]) {
                t %= g.C[m];
                if (t < 0) t += g.C[m];
                applied = jm;
            } else {
                t = min(max(t, 0), g.C[m] - 1);
                applied = t - cur[m];
            }
            nxt[m] = t;
            if (applied != 0) moved = true;
            q[m] = conv ? fminf(fmaxf(q[m] - (float)applied, -1.f), 2.f) : 0.5f;
        }
        if (!moved) {
            // converged and blocked by the grid's boundary: the point is outside (the exhaustive search decides);
            // not converged yet: keep iterating in this cell from where Newton got to
            if (conv) return kWalkStuck;
            continue;
        }
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

__device__ __forceinline__ void write_donor32(const AsmParams& P, int64_t t, int32_t gd, int64_t cell, float u,
                                              float v, float w, uint8_t status) {
    P.out_grid[t] = gd;
    P.out_cell[t] = (int32_t)cell;
    float* xi = (float*)P.out_xi;
    xi[t] = u;
    xi[P.total + t] = v;
    xi[2 * P.total + t] = w;
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

// Field type of a call: IM = 0 assembly only, 1 FP32 fields, 2 FP64 fields.
template <int IM>
struct FieldT {
    using T = float;
};
template <>
struct FieldT<2> {
    using T = double;
};

__device__ __forceinline__ void warp_add(unsigned long long* ctr, unsigned v) {
    unsigned s = __reduce_add_sync(0xffffffffu, v);
    if (lane_id() == 0 && s) atomicAdd(ctr, (unsigned long long)s);
}

// Per-warp shared staging of the learned guess: the network inputs of the warp's points that take a guess (one
// 16-byte row each) and the cells the network gives them.
struct GuessStage {
    float4 rows[32];
    uint32_t cell[32];
};

// The cell a network output points at: y = normalised curvilinear coordinates ((i + xi)/Ci, ...); the cell index
// floor(y C) per axis, wrapped on a periodic axis and clamped to the grid on the others.
__device__ __forceinline__ uint32_t guess_cell(const GridDev& g, const float y[3]) {
    int ijk[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float Cf = (float)g.C[c];
        float f = fminf(fmaxf(y[c] * Cf, -1e6f), 1e6f);
        if (g.per[c]) f -= Cf * floorf(f / Cf);
        ijk[c] = min(max((int)floorf(f), 0), g.C[c] - 1);
    }
    return (uint32_t)ijk[0] + (uint32_t)g.C[0] * ((uint32_t)ijk[1] + (uint32_t)g.C[1] * (uint32_t)ijk[2]);
}

template <int H>
__device__ __forceinline__ void guess_tiles(const GuessDev& gn, const GridDev& g, GuessStage& st, int nrow) {
    const MlpGlobal<H> W(gn.region);
    const int lane = (int)lane_id();
    for (int t0 = 0; t0 < nrow; t0 += 16) {
        float y[2][3];
        mlp_tile<H>(W, st.rows + t0, y);
        if ((lane & 3) == 0) {
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                const int row = t0 + (lane >> 2) + 8 * rr;
                if (row < nrow) st.cell[row] = guess_cell(g, y[rr]);
            }
        }
    }
}

// Learned initial guess for the lanes with `want` (warp-collective: every lane calls it).  The lanes are grouped by
// their donor grid's network (a warp's 32 points are consecutive in the call, so they usually share one set); each
// group's inputs go to the warp's shared rows, 16 to a tensor-core tile.  Returns the guessed cell, or -1.
__device__ __noinline__ int64_t learned_guess(const AsmParams& P, const GridDev* __restrict__ G, GuessStage& st,
                                                 bool want, int gd0, const float xn[3]) {
    const unsigned lane = lane_id();
    int64_t cell = -1;
    unsigned pending = __ballot_sync(0xffffffffu, want);
    while (pending) {
        const int gsel = __shfl_sync(0xffffffffu, gd0, __ffs(pending) - 1);
        const bool mine = want && gd0 == gsel;
        const unsigned grp = __ballot_sync(0xffffffffu, mine);
        pending &= ~grp;
        const int nrow = __popc(grp);
        const int row = __popc(grp & ((1u << lane) - 1u));
        __syncwarp();
        if (mine) st.rows[row] = make_float4(xn[0], xn[1], xn[2], 0.f);
        if ((int)lane >= nrow && (int)lane < ((nrow + 15) & ~15)) st.rows[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncwarp();
        const GuessDev& gn = P.gn[gsel];
        const GridDev& g = G[gsel];
        if (gn.hidden == 32) guess_tiles<32>(gn, g, st, nrow);
        else if (gn.hidden == 64) guess_tiles<64>(gn, g, st, nrow);
        else guess_tiles<128>(gn, g, st, nrow);
        __syncwarp();
        if (mine) cell = st.cell[row];
    }
    __syncwarp();
    return cell;
}

// One query point per thread (t may lie past the end: the lane then only takes part in the warp's collective
// steps).  All lanes of a warp call it together.
template <int IM, bool MLP>
__device__ __forceinline__ void assemble_point(const StepParams& S, const GridDev* __restrict__ G, GuessStage& gs,
                                               const int64_t t) {
    using T = typename FieldT<IM>::T;
    const AsmParams& P = S.a;
    const bool active = t < P.total;
    bool slow = false;
    SlowEntry e;
    int steps = 0, iters = 0;
    // the receiver node as FP32 pairs and its image in the first donor's frame
    int si = 0;
    int32_t node = -1;
    bool node_ok = false;
    ff xd[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    uint32_t h0 = kNoHint;  // the receiver node's donor at the previous call, loaded with its coordinates
    float xr32[3] = {0.f, 0.f, 0.f};  // the receiver node's position in its own frame, FP32
    // the set of point t: lane 0 searches the set table for the warp's first point, the other lanes step forward
    // from there (a work item of 32 consecutive points rarely crosses a set boundary)
    {
        const int64_t t0 = __shfl_sync(0xffffffffu, t, 0);
        int s0 = 0;
        if (lane_id() == 0) s0 = find_set(P.s, P.nsets, t0 < P.total ? t0 : P.total - 1);
        si = __shfl_sync(0xffffffffu, s0, 0);
        if (active)
            while (si + 1 < P.nsets && P.s[si + 1].begin <= t) ++si;
    }
    if (active) {
        const SetDev& s = P.s[si];
        node = __ldg(s.node_ids + (t - s.begin));
        const GridDev& gr = G[s.receiver];
        const int64_t nn = gr.nnodes;
        node_ok = node >= 0 && node < nn;
        if (!node_ok) atomicOr(P.err, kErrBadNode);
        ff x[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        if (node_ok) {
            const float* xf = gr.xff;
            // (xr32 below keeps the position in FP32 for the velocity transform of the interpolation)
#pragma unroll
            for (int c = 0; c < 3; ++c) x[c] = {__ldg(xf + 2 * c * nn + node), __ldg(xf + (2 * c + 1) * nn + node)};
            if (P.guess == OVS_GUESS_HINT) h0 = gr.hint[node];
        }
        xf_apply(P.xf[si], x, xd);
        xr32[0] = __fadd_rn(x[0].hi, x[0].lo);
        xr32[1] = __fadd_rn(x[1].hi, x[1].lo);
        xr32[2] = __fadd_rn(x[2].hi, x[2].lo);
    }
    const bool fast_ok = ff_finite(xd[0]) && ff_finite(xd[1]) && ff_finite(xd[2]);
    // learned guess (not in the paper): points whose first donor grid has a network and that have no usable hint
    // start where the network says.  Its input needs no more than FP32: the point in the donor frame, inside the
    // grid's padded box, normalised as in training.
    int64_t gcell = -1;
    if (MLP && P.guess_mlp) {  // uniform over the call
        bool want = false;
        int gd0 = -1;
        float xn[3] = {0.f, 0.f, 0.f};
        if (active && node_ok && fast_ok) {
            const SetDev& s = P.s[si];
            gd0 = s.donors[0];
            const GuessDev& gn = P.gn[gd0];
            if (gn.hidden) {
                bool valid = false;
                if (!P.guess_always)
                    valid = h0 != kNoHint && (int)(h0 >> kCellBits) == gd0 &&
                            (int64_t)(h0 & ((1u << kCellBits) - 1)) < G[gd0].ncells;
                if (!valid) {
                    bool inside = true;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float v = __fadd_rn(xd[c].hi, xd[c].lo);
                        inside = inside && v >= gn.lo[c] && v <= gn.hi[c];
                        xn[c] = (v - gn.centre[c]) * gn.inv_half[c];
                    }
                    want = inside;
                }
            }
        }
        // the network only for warps that have a point needing it (the call saves the warp's registers)
        if (__ballot_sync(0xffffffffu, want)) gcell = learned_guess(P, G, gs, want, gd0, xn);
        if (P.guess_used) warp_add(P.guess_used, gcell >= 0 ? 1u : 0u);
    }
    if (active) {
        const SetDev& s = P.s[si];
        const GridDev& gr = G[s.receiver];
        // FP64 route: later donors of the list, and points whose FP32-pair image is not finite
        bool have64 = false, bad = !node_ok;
        double3 xin = make_double3(0.0, 0.0, 0.0);
        bool done = false;
        for (int di = 0; di < s.ndonor && !done && !slow && !bad; ++di) {
            const int gd = s.donors[di];
            const GridDev& g = G[gd];
            if (di > 0 || !fast_ok) {
                if (!have64) {
                    double3 xr = make_double3(__ldg(gr.x + node), __ldg(gr.y + node), __ldg(gr.z + node));
                    xin = to_inertial(P.m[s.receiver], xr);
                    have64 = true;
                    if (!finite3(xin)) {
                        bad = true;
                        break;
                    }
                }
                double3 p = to_body(P.m[gd], xin);
                xd[0] = split_double(p.x);
                xd[1] = split_double(p.y);
                xd[2] = split_double(p.z);
                if (!(ff_finite(xd[0]) && ff_finite(xd[1]) && ff_finite(xd[2]))) {
                    if (finite3(p)) {  // finite in FP64 but beyond FP32 range: only the FP64 path can decide
                        slow = true;
                        e.t = (int32_t)t;
                        e.di = di;
                        e.cell = -1;
                        e.xi[0] = e.xi[1] = e.xi[2] = 0.5f;
                    }
                    continue;
                }
            }
            int64_t cell = di == 0 ? gcell : -1;
            if (cell < 0 && P.guess == OVS_GUESS_HINT) {
                if (h0 != kNoHint && (int)(h0 >> kCellBits) == gd) cell = h0 & ((1u << kCellBits) - 1);
                if (cell >= g.ncells) cell = -1;
            }
            const bool from_hint = cell >= 0;
            // cold start: the lowest registered cell of the point's control cell.  Outside the bins' box or in
            // an empty control cell (rep >= ncells), no cell of this grid can hold the point.
            auto control_cell = [&]() -> int64_t {
                double3 p = make_double3((double)xd[0].hi + (double)xd[0].lo, (double)xd[1].hi + (double)xd[1].lo,
                                         (double)xd[2].hi + (double)xd[2].lo);
                int64_t b = point_bin(g, p);
                if (b < 0) return -1;
                int64_t rep = __ldg(g.bin_rep + b);
                return (rep < 0 || rep >= g.ncells) ? -1 : rep;
            };
            if (cell < 0) {
                cell = control_cell();
                if (cell < 0) continue;
            }
            float u, v, w, tau = 0.25f;
            bool blocked = false;
            int ci, cj, ck;
            int r = walk32(g, xd, cell, u, v, w, tau, from_hint ? min(P.max_walk, kHintWalk) : P.max_walk, steps,
                           iters, blocked, ci, cj, ck);
            if (r != kWalkFound && from_hint) {
                // a walk from the previous donor or the learned guess that got stuck (on the grid's boundary, or
                // after kHintWalk steps) starts again from the control cell before the exhaustive search
                cell = control_cell();
                if (cell < 0) continue;
                r = walk32(g, xd, cell, u, v, w, tau, P.max_walk, steps, iters, blocked, ci, cj, ck);
            }
            e.t = (int32_t)t;
            e.di = di;
            if (r == kWalkFound && g.overlap) {
                // cells of this grid may overlap: a lower cell elsewhere may hold the point too, so the
                // exhaustive lowest-id search of the control cell decides
                slow = true;
                e.cell = -1;
                e.xi[0] = e.xi[1] = e.xi[2] = 0.5f;
            } else if (r == kWalkFound) {
                const int mask = near_mask(u, v, w, tau);
                // clear of every face: the only cell of this grid holding the point; blanked -> next donor grid
                if (mask == 0 && !P.xi_f64 && blocked) continue;
                if (mask == 0 && !P.xi_f64) {
                    write_donor32(P, t, gd, cell, u, v, w, OVS_STATUS_FOUND);
                    gr.hint[node] = ((uint32_t)gd << kCellBits) | (uint32_t)cell;
                    done = true;
                    if (IM) {
                        const InterpParams& I = S.i;
                        const int ijk[3] = {ci, cj, ck};
                        interp_point<T>(g, gr, I.fields[gd], I.mode, I.mf[gd], I.mf[s.receiver], I.m[gd],
                                        I.m[s.receiver], node, cell, (T)u, (T)v, (T)w, I.out, t,
                                        di == 0 ? I.va + si : nullptr, ijk, xr32);
                    }
                } else {
                    // near a face (FP64 decision among the neighbours), or FP64 precision (FP64 refinement)
                    slow = true;
                    e.di = di | (mask << 8);
                    e.cell = (int32_t)cell;
                    e.xi[0] = u;
                    e.xi[1] = v;
                    e.xi[2] = w;
                }
            } else {
                slow = true;
                e.cell = -1;
                e.xi[0] = e.xi[1] = e.xi[2] = 0.5f;
            }
        }
        if (bad) write_none(P, t, OVS_STATUS_BADINPUT);
        else if (!done && !slow) write_none(P, t, OVS_STATUS_ORPHAN);
        if (IM && (bad || (!done && !slow))) zero_point<T>(S.i.out, t);  // no donor: 0, as ovs_interpolate
    }
    // warp-aggregated append to the slow queues: points near a face (a candidate cell is known) from the front
    // of the buffer, stuck walks from the back.  Each point is queued at most once, so the two never meet.
    const bool near = slow && e.cell >= 0;
    const unsigned lane = lane_id();
#pragma unroll
    for (int qk = 0; qk < 2; ++qk) {
        const bool mine = qk == 0 ? near : (slow && !near);
        unsigned mask = __ballot_sync(0xffffffffu, mine);
        if (!mask) continue;
        int leader = __ffs(mask) - 1;
        uint32_t base = 0;
        if ((int)lane == leader) base = atomicAdd(P.queue_count + qk, (uint32_t)__popc(mask));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (mine) {
            uint32_t idx = base + __popc(mask & ((1u << lane) - 1u));
            if (idx < P.queue_cap) P.queue[qk == 0 ? idx : P.queue_cap - 1 - idx] = e;
            else atomicOr(P.err, kErrQueueOverflow);
        }
    }
    if (P.stats) {
        warp_add(P.counters + kCtrPoints, active ? 1u : 0u);
        warp_add(P.counters + kCtrWalk, (unsigned)steps);
        warp_add(P.counters + kCtrNewton, (unsigned)iters);
        warp_add(P.counters + kCtrNear, near ? 1u : 0u);
        warp_add(P.counters + kCtrStuck, slow && !near ? 1u : 0u);
        const unsigned mx = __reduce_max_sync(0xffffffffu, (unsigned)steps);
        if (lane == 0 && mx) atomicAdd(P.counters + kCtrWarpWalk, (unsigned long long)mx);
    }
}

// Persistent: a fixed grid (a multiple of the SM count, so that a captured step graph fits every call) whose
// warps take work items of 32 consecutive points of the call (all sets of all grids in one index space) from a
// counter, so that uneven walks balance across the GPU.
template <int IM, bool MLP>
__global__ void __launch_bounds__(kAsmThreads, kAsmMinBlocks) k_assemble(const StepParams* __restrict__ Sp,
                                                                         const GridDev* __restrict__ G) {
    const AsmParams& P = Sp->a;
    const int64_t total = P.total;
    const unsigned lane = lane_id();
    __shared__ GuessStage gstage[kAsmThreads / 32];
    GuessStage& gs = gstage[threadIdx.x >> 5];
    for (;;) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(P.queue_count + 2, 32u);
        base = __shfl_sync(0xffffffffu, base, 0);
        if ((int64_t)base >= total) break;
        assemble_point<IM, MLP>(*Sp, G, gs, (int64_t)base + lane);
    }
}

// ------------------------------------------------------------------------------------------------------
// slow path

// Candidate cells sharing the near faces / edges / corner of `cell` given by the near-face mask, in ascending
// linear id.  Returns their count (<= 8) and the offsets to shift the FP32 guess.
__device__ int near_candidates(const GridDev& g, int64_t cell, int mask, int64_t ids[8], int off[8][3]) {
    int ijk[3];
    cell_ijk(g, cell, ijk[0], ijk[1], ijk[2]);
    int lo[3], hi[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        lo[m] = (mask >> m) & 1 ? -1 : 0;
        hi[m] = (mask >> (3 + m)) & 1 ? 1 : 0;
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

// Warp-cooperative lowest-id decision over the near candidates (donor predicate of contains_exact): lane q
// tests candidate q; the lowest lane (= lowest id) whose cell holds the point wins.  All 32 lanes of the warp
// must call this.
template <class P64>
__device__ bool neighbourhood_warp(const GridDev& g, const ff pf[3], const P64& p64, int64_t cell, int mask,
                                   const float xi32[3], int64_t& out_cell, double& u, double& v, double& w) {
    int64_t ids[8];
    int off[8][3];
    int nc = near_candidates(g, cell, mask, ids, off);
    const int lane = (int)lane_id();
    bool hit = false;
    double a = 0, b = 0, c = 0;
    int64_t mine = -1;
    if (lane < nc) {
        int o0 = 0, o1 = 0, o2 = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (q == lane) {
                mine = ids[q];
                o0 = off[q][0];
                o1 = off[q][1];
                o2 = off[q][2];
            }
        hit = contains_exact(g, mine, pf, p64, xi32[0] - (float)o0, xi32[1] - (float)o1, xi32[2] - (float)o2, a, b,
                             c);
        if (hit && g.blanked && cell_blocked(g.rec, mine)) hit = false;  // a blanked cell never donates
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

// 512 threads (16 warps) at the 128 registers the slow-path code takes anyway: a stuck entry whose control cell
// lists thousands of cells filters them twice as fast as with 256 (the exhaustive search of the most crowded
// control cells is the slow kernel's longest chain), and 16 near-face entries run side by side per block
constexpr int kSlowThreads = 512;
constexpr int kSlowWarps = kSlowThreads / 32;

// Cheap rejections of one cell of an exhaustive search, all in FP32 from the point's FP32 pair (offsets to corner 0
// as in the walk): its padded box, the
// slabs along its three affine face normals (the cell, the convex hull of its corners, lies between the extreme
// corner projections), and the FP32 Newton iteration from the cell centre (up to 24 steps) ending more than
// 1e-3 outside [0,1]^3 (the same iteration in FP32 pairs or FP64 from the same start follows it to within
// rounding, ~1e-5 in local coordinates for the cells accepted here, so it cannot end in the donor window).
// On pass, xi holds the FP32 iterate, the start of the donor predicate.
__device__ __noinline__ bool exhaustive_filter(const GridDev& g, const ff pf[3], uint32_t c, float xi[3]) {
    CellRec rec;
    load_rec(g.rec, c, rec);
    float d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = __fadd_rn(__fsub_rn(pf[k].hi, rec.x0h[k]), __fsub_rn(pf[k].lo, rec.x0l[k]));
    const float* A = rec.a;
    float E[8][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float a1 = A[k], a2 = A[3 + k], a3 = A[6 + k], a4 = A[9 + k], a5 = A[12 + k], a6 = A[15 + k], a7 = A[18 + k];
        E[0][k] = 0.f;
        E[1][k] = a1;
        E[2][k] = a2;
        E[3][k] = a1 + a2 + a4;
        E[4][k] = a3;
        E[5][k] = a1 + a3 + a6;
        E[6][k] = a2 + a3 + a5;
        E[7][k] = a1 + a2 + a3 + a4 + a5 + a6 + a7;
    }
    float mn[3], mx[3], diag2 = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        mn[k] = mx[k] = 0.f;
#pragma unroll
        for (int a = 1; a < 8; ++a) {
            mn[k] = fminf(mn[k], E[a][k]);
            mx[k] = fmaxf(mx[k], E[a][k]);
        }
        diag2 += (mx[k] - mn[k]) * (mx[k] - mn[k]);
    }
    const float pad = 4e-6f * sqrtf(diag2) + 1e-30f;
#pragma unroll
    for (int k = 0; k < 3; ++k)
        if (!(d[k] >= mn[k] - pad && d[k] <= mx[k] + pad)) return false;
    const float* c1 = A;
    const float* c2 = A + 3;
    const float* c3 = A + 6;
    const float nrm[3][3] = {{c2[1] * c3[2] - c2[2] * c3[1], c2[2] * c3[0] - c2[0] * c3[2], c2[0] * c3[1] - c2[1] * c3[0]},
                             {c3[1] * c1[2] - c3[2] * c1[1], c3[2] * c1[0] - c3[0] * c1[2], c3[0] * c1[1] - c3[1] * c1[0]},
                             {c1[1] * c2[2] - c1[2] * c2[1], c1[2] * c2[0] - c1[0] * c2[2], c1[0] * c2[1] - c1[1] * c2[0]}};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        float lo = 0.f, hi = 0.f;
#pragma unroll
        for (int a = 1; a < 8; ++a) {
            float pr = nrm[q][0] * E[a][0] + nrm[q][1] * E[a][1] + nrm[q][2] * E[a][2];
            lo = fminf(lo, pr);
            hi = fmaxf(hi, pr);
        }
        float len = sqrtf(nrm[q][0] * nrm[q][0] + nrm[q][1] * nrm[q][1] + nrm[q][2] * nrm[q][2]);
        float pp = nrm[q][0] * d[0] + nrm[q][1] * d[1] + nrm[q][2] * d[2];
        float sp = pad * len + 1e-6f * (hi - lo) + 1e-30f;  // rounding of the FP32 projections
        if (!(pp >= lo - sp && pp <= hi + sp)) return false;
    }
    float fu = 0.5f, fv = 0.5f, fw = 0.5f;
    newton32(rec, d[0], d[1], d[2], fu, fv, fw, 24);
    const float far = 1e-3f;
    if (!(fu >= -far && fu <= 1.f + far && fv >= -far && fv <= 1.f + far && fw >= -far && fw <= 1.f + far))
        return false;
    xi[0] = fu;
    xi[1] = fv;
    xi[2] = fw;
    return !(g.blanked && rec_blocked(rec));  // a blanked cell never donates
}

// Warp-level exhaustive search of a control cell (lanes stride its list); lowest id wins.  All lanes call.
__device__ bool exhaustive_warp(const GridDev& g, double3 p, const ff pf[3], const int32_t* list, int32_t r0,
                                int32_t r1, int64_t& cell, double& u, double& v, double& w) {
    const int lane = (int)lane_id();
    uint32_t best = 0xFFFFFFFFu;
    double bu = 0, bv = 0, bw = 0;
    for (int32_t r = r0 + lane; r < r1; r += 32) {
        uint32_t c = (uint32_t)__ldg(list + r);
        if (c >= best) continue;
        float xi[3];
        if (!exhaustive_filter(g, pf, c, xi)) continue;
        double a, bb, cc;
        if (contains_exact(g, c, pf, [&]() { return p; }, xi[0], xi[1], xi[2], a, bb, cc)) {
            best = c;
            bu = a;
            bv = bb;
            bw = cc;
        }
    }
    uint32_t wbest = __reduce_min_sync(0xffffffffu, best);
    if (wbest == 0xFFFFFFFFu) return false;
    int src = __ffs(__ballot_sync(0xffffffffu, best == wbest)) - 1;
    cell = wbest;
    u = __shfl_sync(0xffffffffu, bu, src);
    v = __shfl_sync(0xffffffffu, bv, src);
    w = __shfl_sync(0xffffffffu, bw, src);
    return true;
}

// Everything a queued point needs: its set, receiver node, and the donor-frame point for one donor.
struct SlowPoint {
    int64_t t;
    int si;
    int32_t node;
    int di0, mask0;
};

__device__ __forceinline__ SlowPoint slow_point(const AsmParams& P, const SlowEntry& e) {
    SlowPoint sp;
    sp.t = e.t;
    sp.si = find_set(P.s, P.nsets, sp.t);
    sp.node = __ldg(P.s[sp.si].node_ids + (sp.t - P.s[sp.si].begin));
    sp.di0 = e.di & 0xFF;
    sp.mask0 = (e.di >> 8) & 0x3F;
    return sp;
}

// FP64 image of the receiver node in donor gd's frame (the donor rule's definition)
__device__ __forceinline__ double3 point64(const AsmParams& P, const GridDev* G, const SlowPoint& sp, int gd) {
    const SetDev& s = P.s[sp.si];
    const GridDev& gr = G[s.receiver];
    double3 xr = make_double3(gr.x[sp.node], gr.y[sp.node], gr.z[sp.node]);
    return to_body(P.m[gd], to_inertial(P.m[s.receiver], xr));
}

// The point as FP32 pairs in donor di's frame: the fast kernel's transform for the first donor, else from FP64
__device__ __forceinline__ bool point_ff(const AsmParams& P, const GridDev* G, const SlowPoint& sp, int di, ff pf[3]) {
    const SetDev& s = P.s[sp.si];
    if (di == 0) {
        const GridDev& gr = G[s.receiver];
        const int64_t nn = gr.nnodes;
        ff x[3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            x[c] = {__ldg(gr.xff + 2 * c * nn + sp.node), __ldg(gr.xff + (2 * c + 1) * nn + sp.node)};
        xf_apply(P.xf[sp.si], x, pf);
    } else {
        double3 pp = point64(P, G, sp, s.donors[di]);
        pf[0] = split_double(pp.x);
        pf[1] = split_double(pp.y);
        pf[2] = split_double(pp.z);
    }
    return ff_finite(pf[0]) && ff_finite(pf[1]) && ff_finite(pf[2]);
}

template <int IM>
__device__ __forceinline__ void finish(const StepParams& S, const GridDev* G, const SlowPoint& sp, int gd,
                                       int64_t cell, double u, double v, double w, uint8_t st) {
    const AsmParams& P = S.a;
    write_donor(P, sp.t, gd, cell, u, v, w, st);
    const int32_t r = P.s[sp.si].receiver;
    G[r].hint[sp.node] = ((uint32_t)gd << kCellBits) | (uint32_t)cell;
    if (IM) {
        // the local coordinates as stored in the donor record (FP32 or FP64)
        using T = typename FieldT<IM>::T;
        const T a = P.xi_f64 ? (T)u : (T)(float)u, b = P.xi_f64 ? (T)v : (T)(float)v,
                c = P.xi_f64 ? (T)w : (T)(float)w;
        const InterpParams& I = S.i;
        interp_point<T>(G[gd], G[r], I.fields[gd], I.mode, I.mf[gd], I.mf[r], I.m[gd], I.m[r], sp.node, cell, a, b, c,
                        I.out, sp.t, gd == P.s[sp.si].donors[0] ? I.va + sp.si : nullptr);
    }
}

template <int IM>
__device__ __forceinline__ void finish_none(const StepParams& S, int64_t t) {
    write_none(S.a, t, OVS_STATUS_ORPHAN | OVS_STATUS_FALLBACK);
    if (IM) zero_point<typename FieldT<IM>::T>(S.i.out, t);
}

// A slow-path queue entry (near-face entries from the front, stuck entries from the back), read once, through L2.
__device__ __forceinline__ SlowEntry load_entry(const SlowEntry* e) {
    const int* w = reinterpret_cast<const int*>(e);
    SlowEntry r;
    r.t = __ldcg(w);
    r.di = __ldcg(w + 1);
    r.cell = __ldcg(w + 2);
    r.xi[0] = __int_as_float(__ldcg(w + 3));
    r.xi[1] = __int_as_float(__ldcg(w + 4));
    r.xi[2] = __int_as_float(__ldcg(w + 5));
    return r;
}

// A point near a face, by one warp: one lane per candidate cell (the cells sharing the near faces / edges /
// corner, lowest id first).  A point none of them holds is appended to the stuck entries (lane 0), for the
// exhaustive search of its control cell (and the later grids of its list), which runs a block wide: a warp alone
// would walk a crowded control cell in a long chain of dependent loads.  Returns true if decided here.
template <int IM>
__device__ __forceinline__ bool near_entry(const StepParams& S, const GridDev* __restrict__ G, uint32_t q,
                                           uint32_t n_near, uint32_t n_stuck0) {
    const AsmParams& P = S.a;
    const int lane = (int)lane_id();
    const SlowEntry e = P.queue[q];
    const SlowPoint sp = slow_point(P, e);
    const int gd = P.s[sp.si].donors[sp.di0];
    const GridDev& g = G[gd];
    auto p64 = [&]() { return point64(P, G, sp, gd); };
    ff pf[3];
    const bool pf_ok = point_ff(P, G, sp, sp.di0, pf);
    int64_t cell = -1;
    double u = 0, v = 0, w = 0;
    bool ok = false;
    if (pf_ok) ok = neighbourhood_warp(g, pf, p64, e.cell, sp.mask0, e.xi, cell, u, v, w);
    if (ok) {
        if (lane == 0) finish<IM>(S, G, sp, gd, cell, u, v, w, OVS_STATUS_FOUND | OVS_STATUS_REFINED);
    } else if (lane == 0) {
        // behind the stuck entries of the assembly kernel, in the back of the queue (the near-face entries hold
        // the front)
        const uint32_t idx = n_stuck0 + atomicAdd(P.queue_count + 4, 1u);
        if ((int64_t)idx < P.queue_cap - (int64_t)n_near) {
            SlowEntry r = e;
            r.di = sp.di0;
            r.cell = -1;
            r.xi[0] = r.xi[1] = r.xi[2] = 0.5f;
            P.queue[P.queue_cap - 1 - idx] = r;
        } else {
            atomicOr(P.err, kErrQueueOverflow);
        }
    }
    return ok;
}

constexpr int kMaxCand = 128;

// Block-shared state of the exhaustive search of one stuck entry.
struct StuckShared {
    uint32_t cand[kMaxCand];
    float cxi[kMaxCand][3];
    int ncand;
    int found;
    long long fcell;
    double fuvw[3];
    double3 p64;  // the point in the donor's frame: FP64 (the decision's), and as FP32 pairs
    ff pf[3];
    long long bin;
    int32_t r0, r1;  // the candidate list: [r0, r1) of the control cell's list, or of its finer bin's (sub = 1)
    int32_t sub;
};

// A stuck walk (a point outside the grid, or where the walk gave up), stuck entry number q, by the whole block:
// all threads filter the control cell's list (box, slabs, FP32 Newton), then the donor predicate runs on every
// survivor at once; the later grids of the set's list follow if none holds the point.
template <int IM>
__device__ __forceinline__ void stuck_entry(const StepParams& S, const GridDev* __restrict__ G, uint32_t q,
                                            StuckShared& sh, unsigned& nref, unsigned& nfb) {
    const AsmParams& P = S.a;
    static_assert(kMaxCand <= kSlowThreads, "one thread per candidate");
    constexpr long long kNoCellLL = 0x7FFFFFFFFFFFFFFFll;
    const int lane = (int)lane_id();
    const int warp = threadIdx.x >> 5;
    const SlowEntry e = load_entry(P.queue + (P.queue_cap - 1 - q));
    const SlowPoint sp = slow_point(P, e);
    const SetDev& s = P.s[sp.si];
    bool done = false;
    for (int di = sp.di0; di < s.ndonor && !done; ++di) {
        const int gd = s.donors[di];
        const GridDev& g = G[gd];
        // the point and its control cell, by one thread (FP64 is slow here) for the whole block
        __syncthreads();
        if (threadIdx.x == 0) {
            const double3 p0 = point64(P, G, sp, gd);
            sh.bin = point_bin(g, p0);
            if (sh.bin >= 0) {
                const int32_t* list;
                candidate_list(g, p0, sh.bin, list, sh.r0, sh.r1);
                sh.sub = list != g.bin_cells;
            }
            ff pq[3];
            if (!point_ff(P, G, sp, di, pq)) {
                pq[0] = split_double(p0.x);
                pq[1] = split_double(p0.y);
                pq[2] = split_double(p0.z);
            }
            sh.p64 = p0;
            sh.pf[0] = pq[0];
            sh.pf[1] = pq[1];
            sh.pf[2] = pq[2];
        }
        __syncthreads();
        const double3 p = sh.p64;
        const int64_t b = sh.bin;
        if (b < 0) continue;  // outside the bins' box: no cell of this grid holds the point
        const ff pf[3] = {sh.pf[0], sh.pf[1], sh.pf[2]};
        if (threadIdx.x == 0) {
            sh.ncand = 0;
            sh.found = 0;
        }
        __syncthreads();
        const int32_t r0 = sh.r0, r1 = sh.r1;
        const int32_t* list = sh.sub ? g.sub_cells : g.bin_cells;
        for (int32_t r = r0 + (int32_t)threadIdx.x; r < r1; r += kSlowThreads) {
            uint32_t c = (uint32_t)__ldg(list + r);
            float xi[3];
            if (exhaustive_filter(g, pf, c, xi)) {
                int k = atomicAdd(&sh.ncand, 1);
                if (k < kMaxCand) {
                    sh.cand[k] = c;
                    sh.cxi[k][0] = xi[0];
                    sh.cxi[k][1] = xi[1];
                    sh.cxi[k][2] = xi[2];
                }
            }
        }
        __syncthreads();
        const int nc = sh.ncand;
        if (nc <= kMaxCand) {
            // the exact test on every survivor at once, a thread per candidate; the lowest containing id wins
            if (threadIdx.x == 0) sh.fcell = kNoCellLL;
            __syncthreads();
            double a = 0, bb = 0, cc = 0;
            bool hit = false;
            uint32_t c = 0xFFFFFFFFu;
            if ((int)threadIdx.x < nc) {
                c = sh.cand[threadIdx.x];
                hit = contains_exact(g, c, pf, [&]() { return p; }, sh.cxi[threadIdx.x][0], sh.cxi[threadIdx.x][1],
                                     sh.cxi[threadIdx.x][2], a, bb, cc);
                if (hit) atomicMin((unsigned long long*)&sh.fcell, (unsigned long long)c);
            }
            __syncthreads();
            if (hit && (long long)c == sh.fcell) {
                sh.found = 1;
                sh.fuvw[0] = a;
                sh.fuvw[1] = bb;
                sh.fuvw[2] = cc;
            }
        } else if (warp == 0) {
            // more survivors than the list holds: the warp-cooperative exhaustive search
            int64_t cell = -1;
            double u = 0, v = 0, w = 0;
            const bool ok = exhaustive_warp(g, p, pf, list, r0, r1, cell, u, v, w);
            if (ok && lane == 0) {
                sh.found = 1;
                sh.fcell = cell;
                sh.fuvw[0] = u;
                sh.fuvw[1] = v;
                sh.fuvw[2] = w;
            }
        }
        __syncthreads();
        ++nfb;
        if (sh.found) {
            if (threadIdx.x == 0)
                finish<IM>(S, G, sp, gd, sh.fcell, sh.fuvw[0], sh.fuvw[1], sh.fuvw[2],
                           OVS_STATUS_FOUND | OVS_STATUS_REFINED | OVS_STATUS_FALLBACK);
            done = true;
            ++nref;
        }
        __syncthreads();
    }
    if (!done && threadIdx.x == 0) finish_none<IM>(S, sp.t);
}

// The slow paths in one persistent kernel, so that the near-face decisions and the exhaustive searches run at
// the same time.  Blocks take units from a counter: first the stuck entries of the assembly kernel (a block
// each: they are the long ones), then groups of kSlowWarps near-face entries (a warp each).  A near-face point
// none of whose neighbouring cells holds it is appended behind the stuck entries, for k_slow_tail.
template <int IM>
__global__ void __launch_bounds__(kSlowThreads) k_slow(const StepParams* __restrict__ Sp,
                                                       const GridDev* __restrict__ G) {
    const StepParams& S = *Sp;
    const AsmParams& P = S.a;
    __shared__ StuckShared sh;
    __shared__ uint32_t s_unit;
    const uint32_t n_near = min(P.queue_count[0], (uint32_t)P.queue_cap);
    const uint32_t n_stuck0 = min(P.queue_count[1], (uint32_t)P.queue_cap);  // final: the assembly kernel has ended
    const uint32_t n_groups = (n_near + kSlowWarps - 1) / kSlowWarps;
    const uint32_t n_units = n_stuck0 + n_groups;
    unsigned nref_near = 0, nref = 0, nfb = 0;
    for (;;) {
        if (threadIdx.x == 0) s_unit = atomicAdd(P.queue_count + 3, 1u);
        __syncthreads();
        const uint32_t u = s_unit;
        __syncthreads();
        if (u >= n_units) break;
        if (u < n_stuck0) {
            stuck_entry<IM>(S, G, u, sh, nref, nfb);
            continue;
        }
        const uint32_t q = (u - n_stuck0) * kSlowWarps + (threadIdx.x >> 5);
        if (q < n_near && near_entry<IM>(S, G, q, n_near, n_stuck0)) ++nref_near;
    }
    if (P.stats) {
        if ((threadIdx.x & 31) == 0 && nref_near) atomicAdd(P.counters + kCtrRefined, (unsigned long long)nref_near);
        if (threadIdx.x == 0) {
            if (nref) atomicAdd(P.counters + kCtrRefined, (unsigned long long)nref);
            if (nfb) atomicAdd(P.counters + kCtrFallback, (unsigned long long)nfb);
        }
    }
}

// The near-face points k_slow appended to the stuck entries (none of their neighbouring cells holds them): the
// exhaustive search, a block each.  Usually there are none and the launch ends at once; with many (blanked donor
// cells, FP64 local coordinates) they are searched side by side rather than by one block.
template <int IM>
__global__ void __launch_bounds__(kSlowThreads) k_slow_tail(const StepParams* __restrict__ Sp,
                                                            const GridDev* __restrict__ G) {
    const StepParams& S = *Sp;
    const AsmParams& P = S.a;
    __shared__ StuckShared sh;
    const uint32_t n_near = min(P.queue_count[0], (uint32_t)P.queue_cap);
    const uint32_t n_stuck0 = min(P.queue_count[1], (uint32_t)P.queue_cap);
    const uint32_t n_app = min(P.queue_count[4], (uint32_t)P.queue_cap);
    unsigned nref = 0, nfb = 0;
    for (uint32_t k = blockIdx.x; k < n_app && n_stuck0 + k < (uint32_t)P.queue_cap - n_near; k += gridDim.x)
        stuck_entry<IM>(S, G, n_stuck0 + k, sh, nref, nfb);
    if (P.stats && threadIdx.x == 0) {
        if (nref) atomicAdd(P.counters + kCtrRefined, (unsigned long long)nref);
        if (nfb) atomicAdd(P.counters + kCtrFallback, (unsigned long long)nfb);
    }
}

}  // namespace

cudaError_t launch_assemble(const StepParams* dS, int interp, bool mlp, uint32_t* queue_count, const GridDev* dgrids,
                            int nsm, int asm_bps, int slow_bps, cudaStream_t st, cudaEvent_t const* ev) {
    const unsigned ab = (unsigned)(nsm * (asm_bps > 0 ? asm_bps : kAsmMinBlocks));
    const unsigned sb = (unsigned)(nsm * (slow_bps > 0 ? slow_bps : 1));
    // the queue counters and the work counters (near-face, stuck, assembly work, slow-path work, near-face entries
    // appended to the stuck ones)
    cudaError_t err = cudaMemsetAsync(queue_count, 0, kQueueCounters * sizeof(uint32_t), st);
    if (err != cudaSuccess) return err;
    if (ev && ev[0]) cudaEventRecord(ev[0], st);
    // the learned guess in its own instantiation: without it the kernel holds no call site whose saved
    // registers would weigh on the plain path
    if (mlp) {
        if (interp == 1) k_assemble<1, true><<<ab, kAsmThreads, 0, st>>>(dS, dgrids);
        else if (interp == 2) k_assemble<2, true><<<ab, kAsmThreads, 0, st>>>(dS, dgrids);
        else k_assemble<0, true><<<ab, kAsmThreads, 0, st>>>(dS, dgrids);
    } else {
        if (interp == 1) k_assemble<1, false><<<ab, kAsmThreads, 0, st>>>(dS, dgrids);
        else if (interp == 2) k_assemble<2, false><<<ab, kAsmThreads, 0, st>>>(dS, dgrids);
        else k_assemble<0, false><<<ab, kAsmThreads, 0, st>>>(dS, dgrids);
    }
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    if (ev && ev[1]) cudaEventRecord(ev[1], st);
    if (interp == 1) k_slow<1><<<sb, kSlowThreads, 0, st>>>(dS, dgrids);
    else if (interp == 2) k_slow<2><<<sb, kSlowThreads, 0, st>>>(dS, dgrids);
    else k_slow<0><<<sb, kSlowThreads, 0, st>>>(dS, dgrids);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    if (interp == 1) k_slow_tail<1><<<sb, kSlowThreads, 0, st>>>(dS, dgrids);
    else if (interp == 2) k_slow_tail<2><<<sb, kSlowThreads, 0, st>>>(dS, dgrids);
    else k_slow_tail<0><<<sb, kSlowThreads, 0, st>>>(dS, dgrids);
    if (ev && ev[2]) cudaEventRecord(ev[2], st);
    return cudaGetLastError();
}

}  // namespace ovs
