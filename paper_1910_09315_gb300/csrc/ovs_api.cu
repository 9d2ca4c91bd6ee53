// C ABI of libovs: argument checking, workspace carving, grid set-up and launches.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "ovs_flux.cuh"
#include "ovs_guess.cuh"
#include "ovs_hole.cuh"
#include "ovs_matrix.cuh"
#include "ovs_internal.cuh"

using namespace ovs;

namespace {

constexpr size_t kAlign = 256;
constexpr int kReduceBlocks = 1024;
constexpr double kRegsPerCell = 12.0;  // registration capacity of the control-cell lists

inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct GridHost {
    ovs_grid_desc desc;
    void* ws;
    size_t ws_bytes;
    int64_t nbins;
    int64_t nreg;
    int64_t nsubreg;  // registrations in the finer bins of crowded control cells
    int64_t orient[3];  // cells right-handed, left-handed, folded or degenerate (corner Jacobians at creation)
};

}  // namespace

struct ovs_ctx {
    int device = 0;
    int nsm = 1;  // streaming multiprocessors of the device (persistent grids)
    cudaStream_t stream = nullptr;
    std::string err;
    // context workspace
    void* ws = nullptr;
    size_t ws_bytes = 0;
    int64_t max_points = 0;
    GridDev* d_grids = nullptr;
    unsigned long long* d_counters = nullptr;
    int32_t* d_err = nullptr;
    uint32_t* d_qcount = nullptr;
    SlowEntry* d_queue = nullptr;
    double* d_flux_part = nullptr;  // chunk sums of ovs_interface_flux
    // grids
    int ngrids = 0;
    GridDev grids[OVS_MAX_GRIDS];
    GridHost gh[OVS_MAX_GRIDS];
    MotionDev motion[OVS_MAX_GRIDS];
    int hidden[OVS_MAX_GRIDS] = {};  // width of each grid's trained guess network, 0 if none
    ovs_options opts;
    cudaEvent_t trace[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool tracing = false;
    // step parameters: the device copy (context workspace) and two pinned staging buffers, each with the event
    // that marks the end of the last call that read it
    StepParams* d_step = nullptr;
    StepParams* h_step[2] = {nullptr, nullptr};
    cudaEvent_t step_done[2] = {nullptr, nullptr};
    bool step_used[2] = {false, false};
    int stage = 0;
    // CUDA graphs of the launch sequences, one pair (per staging buffer) for each kind of call
    cudaStream_t gstream = nullptr;  // capture stream
    struct GraphEntry {
        uint32_t kind;
        cudaGraphExec_t exec[2];
    };
    std::vector<GraphEntry> graphs;
    ovs_tuning tune = {0, 0, 0, 0};  // launch shapes (0: defaults)
    // body surfaces for hole cutting
    int nsurf = 0;
    SurfaceDev surf[OVS_MAX_GRIDS];
    int32_t surf_body[OVS_MAX_GRIDS];
};

namespace {

int fail(ovs_ctx* c, int code, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

int cuda_fail(ovs_ctx* c, cudaError_t e, const char* what) {
    return fail(c, OVS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define OVS_CUDA(c, call)                                   \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
    } while (0)

void identity_motion(MotionDev& m) {
    memset(&m, 0, sizeof m);
    m.R[0] = m.R[4] = m.R[8] = 1.0;
    m.identity = 1;
}

int64_t cells_axis(const ovs_grid_desc& d, int a) { return d.periodic[a] ? d.n[a] : d.n[a] - 1; }

struct GridLayout {
    size_t rec, bin_start, bin_count, bin_rep, bin_cells, hint, xff, mlp, partials, scan, out9, crowd, sub_start,
        sub_count, sub_cells, total;
    int64_t ncells, nnodes, nbins_max, reg_cap, sub_cap;
};

GridLayout grid_layout(const ovs_grid_desc& d) {
    GridLayout L;
    L.ncells = cells_axis(d, 0) * cells_axis(d, 1) * cells_axis(d, 2);
    L.nnodes = (int64_t)d.n[0] * d.n[1] * d.n[2];
    L.nbins_max = std::max<int64_t>(1, L.ncells);
    L.reg_cap = (int64_t)(kRegsPerCell * (double)L.ncells) + 64;
    size_t off = 0;
    L.rec = off;
    off = align_up(off + (size_t)L.ncells * sizeof(CellRec));
    L.bin_start = off;
    off = align_up(off + (size_t)(L.nbins_max + 1) * 4);
    L.bin_count = off;
    off = align_up(off + (size_t)L.nbins_max * 4);
    L.bin_rep = off;
    off = align_up(off + (size_t)L.nbins_max * 4);
    L.bin_cells = off;
    off = align_up(off + (size_t)L.reg_cap * 4);
    L.hint = off;
    off = align_up(off + (size_t)L.nnodes * 4);
    L.xff = off;
    off = align_up(off + (size_t)L.nnodes * 6 * sizeof(float));
    L.mlp = off;
    off = align_up(off + mlp_region_bytes());
    L.partials = off;
    off = align_up(off + (size_t)kReduceBlocks * 9 * sizeof(double));
    L.scan = off;
    off = align_up(off + scan_scratch_elems(std::max<int64_t>(L.nbins_max, (int64_t)kMaxCrowded * kSub3)) * 4);
    L.out9 = off;
    off = align_up(off + 9 * sizeof(double) + 3 * sizeof(unsigned long long));
    // the finer bins of crowded control cells: their ids (and a device counter), list starts, counts, lists
    L.sub_cap = std::min<int64_t>(2 * L.ncells + 4096, (int64_t)1 << 23);
    L.crowd = off;
    off = align_up(off + (size_t)kMaxCrowded * 4 + 16);
    L.sub_start = off;
    off = align_up(off + ((size_t)kMaxCrowded * kSub3 + 1) * 4);
    L.sub_count = off;
    off = align_up(off + (size_t)kMaxCrowded * kSub3 * 4);
    L.sub_cells = off;
    off = align_up(off + (size_t)L.sub_cap * 4);
    L.total = off;
    return L;
}

int check_desc(ovs_ctx* c, const ovs_grid_desc* d) {
    if (!d) return fail(c, OVS_ERR_ARG, "grid descriptor is NULL");
    for (int a = 0; a < 3; ++a) {
        if (d->n[a] < 2) return fail(c, OVS_ERR_ARG, "grid axis %d has %d nodes (need >= 2)", a, d->n[a]);
        if (d->periodic[a] != 0 && d->periodic[a] != 1)
            return fail(c, OVS_ERR_ARG, "periodic[%d] must be 0 or 1", a);
        if (d->periodic[a] && d->n[a] < 3) return fail(c, OVS_ERR_ARG, "periodic axis %d needs >= 3 nodes", a);
    }
    if (!d->x || !d->y || !d->z) return fail(c, OVS_ERR_ARG, "grid coordinate pointer is NULL");
    if (d->role != 0 && d->role != 1) return fail(c, OVS_ERR_ARG, "role must be 0 (background) or 1 (body)");
    int64_t ncells = cells_axis(*d, 0) * cells_axis(*d, 1) * cells_axis(*d, 2);
    if (ncells >= OVS_MAX_CELLS - 1)
        return fail(c, OVS_ERR_ARG, "grid has %lld cells; the limit is %lld", (long long)ncells,
                    (long long)(OVS_MAX_CELLS - 1));
    return OVS_OK;
}

int check_sets(ovs_ctx* c, const ovs_fringe_set* sets, int32_t nsets, int64_t* total) {
    if (nsets < 0 || nsets > OVS_MAX_SETS) return fail(c, OVS_ERR_ARG, "nsets = %d (0..%d)", nsets, OVS_MAX_SETS);
    if (nsets > 0 && !sets) return fail(c, OVS_ERR_ARG, "sets is NULL");
    int64_t tot = 0;
    for (int s = 0; s < nsets; ++s) {
        const ovs_fringe_set& f = sets[s];
        if (f.receiver < 0 || f.receiver >= c->ngrids)
            return fail(c, OVS_ERR_ARG, "set %d: receiver grid %d does not exist", s, f.receiver);
        if (f.n_donors < 1 || f.n_donors > OVS_MAX_DONORS)
            return fail(c, OVS_ERR_ARG, "set %d: n_donors = %d (1..%d)", s, f.n_donors, OVS_MAX_DONORS);
        for (int d = 0; d < f.n_donors; ++d)
            if (f.donors[d] < 0 || f.donors[d] >= c->ngrids)
                return fail(c, OVS_ERR_ARG, "set %d: donor grid %d does not exist", s, f.donors[d]);
        if (f.n < 0) return fail(c, OVS_ERR_ARG, "set %d: n = %lld", s, (long long)f.n);
        if (f.n > 0 && !f.node_ids) return fail(c, OVS_ERR_ARG, "set %d: node_ids is NULL", s);
        tot += f.n;
    }
    if (tot > c->max_points)
        return fail(c, OVS_ERR_WORKSPACE, "%lld points exceed the workspace's max_points %lld", (long long)tot,
                    (long long)c->max_points);
    if (tot >= ((int64_t)1 << 31) - 1) return fail(c, OVS_ERR_ARG, "more than 2^31 points in one call");
    *total = tot;
    return OVS_OK;
}

void fill_sets(const ovs_fringe_set* sets, int32_t nsets, SetDev* out) {
    int64_t begin = 0;
    for (int s = 0; s < nsets; ++s) {
        out[s].receiver = sets[s].receiver;
        out[s].ndonor = sets[s].n_donors;
        for (int d = 0; d < OVS_MAX_DONORS; ++d) out[s].donors[d] = d < sets[s].n_donors ? sets[s].donors[d] : -1;
        out[s].node_ids = sets[s].node_ids;
        out[s].begin = begin;
        out[s].n = sets[s].n;
        begin += sets[s].n;
    }
    // empty sets share the next set's begin; the point -> set lookup takes the last set with begin <= t
}

// FP32-pair split of an FP64 value: hi = nearest float, lo = nearest float to the remainder
void split(double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

// Per set: the receiver -> first-donor transform x_d = M x_r + t, composed in FP64 (M = R_d^T R_r,
// t = R_d^T (c_r - c_d)) and handed to the kernel as FP32 pairs.
void fill_xforms(const ovs_ctx* c, const ovs_fringe_set* sets, int32_t nsets, XfFF* out) {
    for (int s = 0; s < nsets; ++s) {
        const MotionDev& r = c->motion[sets[s].receiver];
        const MotionDev& d = c->motion[sets[s].donors[0]];
        XfFF& X = out[s];
        memset(&X, 0, sizeof X);
        X.identity = r.identity && d.identity;
        for (int i = 0; i < 3; ++i) {
            for (int k = 0; k < 3; ++k) {
                double m = 0;
                for (int j = 0; j < 3; ++j) m += d.R[3 * j + i] * r.R[3 * j + k];
                split(m, X.Mh[3 * i + k], X.Ml[3 * i + k]);
            }
            double tv = 0;
            for (int j = 0; j < 3; ++j) tv += d.R[3 * j + i] * (r.c[j] - d.c[j]);
            split(tv, X.th[i], X.tl[i]);
        }
    }
}

// Per set: the velocity transform from its first donor's frame to the receiver's as one affine map (FP64 here,
// FP32 on the device): u_r = A u_d + B x_r + b (see VelAffine).
void fill_vel_affine(const ovs_ctx* c, const ovs_fringe_set* sets, int32_t nsets, int mode, VelAffine* out) {
    for (int s = 0; s < nsets; ++s) {
        const MotionDev& r = c->motion[sets[s].receiver];
        const MotionDev& d = c->motion[sets[s].donors[0]];
        VelAffine& V = out[s];
        memset(&V, 0, sizeof V);
        double A[9], B[9] = {0}, b[3] = {0};
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) {
                double m = 0;
                for (int j = 0; j < 3; ++j) m += r.R[3 * j + i] * d.R[3 * j + k];  // (R_r^T R_d)_ik
                A[3 * i + k] = mode == OVS_VEL_NONE ? (i == k ? 1.0 : 0.0) : m;
            }
        if (mode == OVS_VEL_RELATIVE) {
            const double w[3] = {d.w[0] - r.w[0], d.w[1] - r.w[1], d.w[2] - r.w[2]};
            const double W[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};  // [w]x
            double WR[9];
            for (int i = 0; i < 3; ++i)
                for (int k = 0; k < 3; ++k) {
                    double m = 0;
                    for (int j = 0; j < 3; ++j) m += W[3 * i + j] * r.R[3 * j + k];
                    WR[3 * i + k] = m;
                }
            for (int i = 0; i < 3; ++i)
                for (int k = 0; k < 3; ++k) {
                    double m = 0;
                    for (int j = 0; j < 3; ++j) m += r.R[3 * j + i] * WR[3 * j + k];
                    B[3 * i + k] = m;
                }
            const double dc[3] = {r.c[0] - d.c[0], r.c[1] - d.c[1], r.c[2] - d.c[2]};
            const double e[3] = {d.V[0] - r.V[0] + d.w[1] * dc[2] - d.w[2] * dc[1],
                                 d.V[1] - r.V[1] + d.w[2] * dc[0] - d.w[0] * dc[2],
                                 d.V[2] - r.V[2] + d.w[0] * dc[1] - d.w[1] * dc[0]};
            for (int i = 0; i < 3; ++i) b[i] = r.R[i] * e[0] + r.R[3 + i] * e[1] + r.R[6 + i] * e[2];
        }
        for (int q = 0; q < 9; ++q) {
            V.A[q] = (float)A[q];
            V.B[q] = (float)B[q];
        }
        for (int q = 0; q < 3; ++q) V.b[q] = (float)b[q];
    }
}

// FP32 copies of the motions for the FP32 velocity transform
void fill_motion_f32(const ovs_ctx* c, MotionF* out) {
    for (int g = 0; g < OVS_MAX_GRIDS; ++g) {
        const MotionDev& m = c->motion[g];
        MotionF& f = out[g];
        memset(&f, 0, sizeof f);
        for (int q = 0; q < 9; ++q) f.R[q] = (float)m.R[q];
        for (int q = 0; q < 3; ++q) {
            split(m.c[q], f.ch[q], f.cl[q]);
            f.V[q] = (float)m.V[q];
            f.w[q] = (float)m.w[q];
        }
        f.identity = m.identity;
    }
}

}  // namespace

extern "C" {

// frees what a context owns on the host and the device (its streams, events, graphs, staging buffers)
static void release(ovs_ctx* c) {
    for (auto& g : c->graphs)
        for (auto& x : g.exec)
            if (x) cudaGraphExecDestroy(x);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    for (int b = 0; b < 2; ++b) {
        if (c->step_done[b]) cudaEventDestroy(c->step_done[b]);
        if (c->h_step[b]) cudaFreeHost(c->h_step[b]);
    }
    delete c;
}

int ovs_ctx_create(ovs_ctx** out, int device, void* cuda_stream) {
    if (!out) return OVS_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
        cudaGetLastError();
        return OVS_ERR_NO_DEVICE;
    }
    if (device < 0 || device >= ndev) return OVS_ERR_ARG;
    ovs_ctx* c = new (std::nothrow) ovs_ctx();
    if (!c) return OVS_ERR_ARG;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    for (int g = 0; g < OVS_MAX_GRIDS; ++g) identity_motion(c->motion[g]);
    c->opts.velocity_mode = OVS_VEL_RELATIVE;
    c->opts.guess = OVS_GUESS_HINT;
    c->opts.max_walk = 48;
    c->opts.collect_stats = 0;
    c->opts.launch = OVS_LAUNCH_GRAPH;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return OVS_ERR_NO_DEVICE;
    }
    if (cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->step_done[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->step_done[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaHostAlloc((void**)&c->h_step[0], sizeof(StepParams), cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void**)&c->h_step[1], sizeof(StepParams), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        release(c);
        return OVS_ERR_CUDA;
    }
    *out = c;
    return OVS_OK;
}

int ovs_ctx_destroy(ovs_ctx* c) {
    if (!c) return OVS_ERR_ARG;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    release(c);
    return OVS_OK;
}

const char* ovs_last_error(const ovs_ctx* c) {
    if (!c) return "null context";
    return c->err.c_str();
}

int ovs_set_stream(ovs_ctx* c, void* s) {
    if (!c) return OVS_ERR_ARG;
    c->stream = (cudaStream_t)s;
    return OVS_OK;
}

int ovs_workspace_size(const ovs_ctx* c, int64_t max_points, size_t* bytes) {
    if (!c || !bytes || max_points < 0) return OVS_ERR_ARG;
    size_t off = align_up(sizeof(GridDev) * OVS_MAX_GRIDS);
    off = align_up(off + sizeof(unsigned long long) * kNumCounters);
    off = align_up(off + (1 + kQueueCounters) * sizeof(int32_t));
    // the slow-path queue: two entries per point (a near-face point the neighbourhood test cannot place is queued
    // again for the exhaustive search)
    off = align_up(off + (size_t)std::max<int64_t>(1, 2 * max_points) * sizeof(SlowEntry));
    off = align_up(off + sizeof(StepParams));
    off = align_up(off + 2 * sizeof(double) * kFluxChunks);
    *bytes = off;
    return OVS_OK;
}

int ovs_workspace_attach(ovs_ctx* c, void* dptr, size_t bytes, int64_t max_points) {
    if (!c) return OVS_ERR_ARG;
    size_t need = 0;
    if (ovs_workspace_size(c, max_points, &need) != OVS_OK) return fail(c, OVS_ERR_ARG, "bad max_points");
    if (!dptr) return fail(c, OVS_ERR_ARG, "workspace pointer is NULL");
    if ((uintptr_t)dptr % kAlign) return fail(c, OVS_ERR_ARG, "workspace must be 256-byte aligned");
    if (bytes < need)
        return fail(c, OVS_ERR_WORKSPACE, "workspace has %zu bytes, needs %zu for %lld points", bytes, need,
                    (long long)max_points);
    OVS_CUDA(c, cudaSetDevice(c->device));
    char* base = (char*)dptr;
    size_t off = 0;
    c->d_grids = (GridDev*)(base + off);
    off = align_up(off + sizeof(GridDev) * OVS_MAX_GRIDS);
    c->d_counters = (unsigned long long*)(base + off);
    off = align_up(off + sizeof(unsigned long long) * kNumCounters);
    c->d_err = (int32_t*)(base + off);
    c->d_qcount = (uint32_t*)(base + off + sizeof(int32_t));  // the slow-path queue's counters
    off = align_up(off + (1 + kQueueCounters) * sizeof(int32_t));
    c->d_queue = (SlowEntry*)(base + off);
    off = align_up(off + (size_t)std::max<int64_t>(1, 2 * max_points) * sizeof(SlowEntry));
    c->d_step = (StepParams*)(base + off);
    off = align_up(off + sizeof(StepParams));
    c->d_flux_part = (double*)(base + off);
    off = align_up(off + 2 * sizeof(double) * kFluxChunks);
    c->ws = dptr;
    c->ws_bytes = bytes;
    c->max_points = max_points;
    OVS_CUDA(c, cudaMemsetAsync(dptr, 0, off, c->stream));
    if (c->ngrids)
        OVS_CUDA(c, cudaMemcpyAsync(c->d_grids, c->grids, sizeof(GridDev) * c->ngrids, cudaMemcpyHostToDevice,
                                    c->stream));
    OVS_CUDA(c, cudaStreamSynchronize(c->stream));
    return OVS_OK;
}

int ovs_grid_workspace_size(const ovs_grid_desc* d, size_t* bytes) {
    if (!bytes) return OVS_ERR_ARG;
    int rc = check_desc(nullptr, d);
    if (rc != OVS_OK) return rc;
    *bytes = grid_layout(*d).total;
    return OVS_OK;
}

int ovs_create_grid(ovs_ctx* c, const ovs_grid_desc* d, void* dws, size_t bytes, int32_t* grid_id) {
    if (!c) return OVS_ERR_ARG;
    int rc = check_desc(c, d);
    if (rc != OVS_OK) return rc;
    if (!grid_id) return fail(c, OVS_ERR_ARG, "grid_id is NULL");
    if (!c->ws) return fail(c, OVS_ERR_STATE, "attach the context workspace before creating grids");
    if (c->ngrids >= OVS_MAX_GRIDS) return fail(c, OVS_ERR_STATE, "at most %d grids", OVS_MAX_GRIDS);
    GridLayout L = grid_layout(*d);
    if (!dws) return fail(c, OVS_ERR_ARG, "grid workspace is NULL");
    if ((uintptr_t)dws % kAlign) return fail(c, OVS_ERR_ARG, "grid workspace must be 256-byte aligned");
    if (bytes < L.total) return fail(c, OVS_ERR_WORKSPACE, "grid workspace has %zu bytes, needs %zu", bytes, L.total);
    OVS_CUDA(c, cudaSetDevice(c->device));
    char* base = (char*)dws;
    GridDev g;
    memset(&g, 0, sizeof g);
    for (int a = 0; a < 3; ++a) {
        g.n[a] = d->n[a];
        g.per[a] = d->periodic[a];
        g.C[a] = (int32_t)cells_axis(*d, a);
    }
    g.role = d->role;
    g.ncells = L.ncells;
    g.nnodes = L.nnodes;
    g.x = d->x;
    g.y = d->y;
    g.z = d->z;
    g.rec = (const CellRec*)(base + L.rec);
    g.bin_start = (const int32_t*)(base + L.bin_start);
    g.bin_cells = (const int32_t*)(base + L.bin_cells);
    g.bin_rep = (const int32_t*)(base + L.bin_rep);
    g.hint = (uint32_t*)(base + L.hint);
    g.xff = (const float*)(base + L.xff);
    g.mlp = base + L.mlp;
    double* out9 = (double*)(base + L.out9);
    unsigned long long* orient = (unsigned long long*)(out9 + 9);
    int nblk = (int)std::min<int64_t>(kReduceBlocks, (L.ncells + 255) / 256);
    OVS_CUDA(c, launch_build_records(g, (CellRec*)(base + L.rec), (float*)(base + L.xff),
                                     (double*)(base + L.partials), nblk, out9, orient, c->stream));
    double h9[9];
    unsigned long long ho[3];
    OVS_CUDA(c, cudaMemcpyAsync(h9, out9, sizeof h9, cudaMemcpyDeviceToHost, c->stream));
    OVS_CUDA(c, cudaMemcpyAsync(ho, orient, sizeof ho, cudaMemcpyDeviceToHost, c->stream));
    OVS_CUDA(c, cudaStreamSynchronize(c->stream));
    // cells of both handednesses, or folded ones: the grid may overlap itself
    g.overlap = (ho[2] > 0 || (ho[0] > 0 && ho[1] > 0)) ? 1 : 0;
    double ext_max = 0;
    for (int a = 0; a < 3; ++a) {
        if (!isfinite(h9[a]) || !isfinite(h9[3 + a]))
            return fail(c, OVS_ERR_ARG, "grid coordinates are not finite");
        ext_max = std::max(ext_max, h9[3 + a] - h9[a]);
    }
    double pad = 4e-6 * ext_max + 1e-300;
    double ext[3], mean[3];
    for (int a = 0; a < 3; ++a) {
        g.lo[a] = h9[a] - pad;
        g.hi[a] = h9[3 + a] + pad;
        ext[a] = g.hi[a] - g.lo[a];
        mean[a] = std::max(h9[6 + a] / (double)L.ncells, 1e-12 * ext_max + 1e-300);
    }
    // bins about 0.6 mean cell extents wide, at most one bin per cell (retried coarser if that exceeds the bin or
    // registration capacity): fine enough that the control cells of crowded regions (an O-grid's polar axis, thin
    // near-wall cells) list few cells, which bounds the exhaustive search and makes cold starts close
    double scale = 0.6;
    int64_t nreg = 0;
    for (int attempt = 0; attempt < 8; ++attempt) {
        int64_t nb_tot = 1;
        for (int a = 0; a < 3; ++a) {
            double nb = ceil(ext[a] / (scale * mean[a]));
            g.nb[a] = (int32_t)std::min(4096.0, std::max(1.0, nb));
            nb_tot *= g.nb[a];
        }
        if (nb_tot > L.nbins_max) {
            scale *= 1.26;
            continue;
        }
        for (int a = 0; a < 3; ++a) g.inv_w[a] = (double)g.nb[a] / ext[a];
        uint32_t* counts = (uint32_t*)(base + L.bin_count);
        int32_t* start = (int32_t*)(base + L.bin_start);
        OVS_CUDA(c, cudaMemsetAsync(counts, 0, (size_t)nb_tot * 4, c->stream));
        OVS_CUDA(c, launch_bin_count(g, counts, c->stream));
        OVS_CUDA(c, launch_scan(counts, start, nb_tot, (uint32_t*)(base + L.scan), c->stream));
        int32_t tot = 0;
        OVS_CUDA(c, cudaMemcpyAsync(&tot, start + nb_tot, 4, cudaMemcpyDeviceToHost, c->stream));
        OVS_CUDA(c, cudaStreamSynchronize(c->stream));
        if (tot < 0 || (int64_t)tot > L.reg_cap) {
            scale *= 1.5;
            continue;
        }
        nreg = tot;
        OVS_CUDA(c, cudaMemsetAsync(counts, 0, (size_t)nb_tot * 4, c->stream));
        OVS_CUDA(c, cudaMemsetAsync(base + L.bin_rep, 0x7F, (size_t)nb_tot * 4, c->stream));
        OVS_CUDA(c, launch_bin_fill(g, start, counts, (int32_t*)(base + L.bin_cells), (int32_t*)(base + L.bin_rep),
                                    c->stream));
        // bins left at 0x7F7F7F7F (>= ncells) are empty; the lookup treats them so
        c->gh[c->ngrids].nbins = nb_tot;
        break;
    }
    if (nreg == 0 && L.ncells > 0) return fail(c, OVS_ERR_WORKSPACE, "control-cell lists exceed the workspace");
    // crowded control cells (thin or clustered cells crowding a bin, as at a fish's tail) get kSub^3 finer bins,
    // which the exhaustive search reads instead of the whole list; the threshold is raised until their number
    // and registrations fit the space set aside (none split is always a valid outcome)
    g.crowd = (const int32_t*)(base + L.crowd);
    g.sub_start = (const int32_t*)(base + L.sub_start);
    g.sub_cells = (const int32_t*)(base + L.sub_cells);
    g.ncrowd = 0;
    int64_t nsubreg = 0;
    if (nreg > 0) {
        int32_t* crowd = (int32_t*)(base + L.crowd);
        uint32_t* dn = (uint32_t*)(base + L.crowd + (size_t)kMaxCrowded * 4);
        uint32_t* counts = (uint32_t*)(base + L.sub_count);
        int32_t* sstart = (int32_t*)(base + L.sub_start);
        const int64_t nbins = (int64_t)g.nb[0] * g.nb[1] * g.nb[2];
        for (int32_t thr = kCrowdedCount; thr < (1 << 29); thr *= 2) {
            OVS_CUDA(c, cudaMemsetAsync(dn, 0, sizeof(uint32_t), c->stream));
            OVS_CUDA(c, launch_crowd_mark(g, nbins, thr, crowd, dn, kMaxCrowded, c->stream));
            uint32_t hn = 0;
            OVS_CUDA(c, cudaMemcpyAsync(&hn, dn, sizeof hn, cudaMemcpyDeviceToHost, c->stream));
            OVS_CUDA(c, cudaStreamSynchronize(c->stream));
            if (hn == 0) break;
            if (hn > (uint32_t)kMaxCrowded) continue;
            std::vector<int32_t> hc(hn);
            OVS_CUDA(c, cudaMemcpyAsync(hc.data(), crowd, hn * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
            OVS_CUDA(c, cudaStreamSynchronize(c->stream));
            std::sort(hc.begin(), hc.end());  // the search looks a control cell up by bisection
            OVS_CUDA(c, cudaMemcpyAsync(crowd, hc.data(), hn * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
            OVS_CUDA(c, cudaStreamSynchronize(c->stream));
            g.ncrowd = (int32_t)hn;
            const int64_t nsub = (int64_t)hn * kSub3;
            OVS_CUDA(c, cudaMemsetAsync(counts, 0, (size_t)nsub * 4, c->stream));
            OVS_CUDA(c, launch_sub_count(g, counts, c->stream));
            OVS_CUDA(c, launch_scan(counts, sstart, nsub, (uint32_t*)(base + L.scan), c->stream));
            int32_t tot = 0;
            OVS_CUDA(c, cudaMemcpyAsync(&tot, sstart + nsub, 4, cudaMemcpyDeviceToHost, c->stream));
            OVS_CUDA(c, cudaStreamSynchronize(c->stream));
            if (tot < 0 || (int64_t)tot > L.sub_cap) {
                g.ncrowd = 0;
                continue;
            }
            OVS_CUDA(c, cudaMemsetAsync(counts, 0, (size_t)nsub * 4, c->stream));
            OVS_CUDA(c, launch_sub_fill(g, sstart, counts, (int32_t*)(base + L.sub_cells), c->stream));
            nsubreg = tot;
            break;
        }
    }
    OVS_CUDA(c, cudaMemsetAsync(base + L.hint, 0xFF, (size_t)L.nnodes * 4, c->stream));
    OVS_CUDA(c, cudaMemsetAsync(base + L.mlp, 0, sizeof(MlpHeader), c->stream));  // no guess network yet
    int id = c->ngrids;
    c->grids[id] = g;
    c->gh[id].desc = *d;
    c->gh[id].ws = dws;
    c->gh[id].ws_bytes = bytes;
    c->gh[id].nreg = nreg;
    c->gh[id].nsubreg = nsubreg;
    for (int q = 0; q < 3; ++q) c->gh[id].orient[q] = (int64_t)ho[q];
    identity_motion(c->motion[id]);
    OVS_CUDA(c, cudaMemcpyAsync(c->d_grids + id, &c->grids[id], sizeof(GridDev), cudaMemcpyHostToDevice, c->stream));
    OVS_CUDA(c, cudaStreamSynchronize(c->stream));
    OVS_CUDA(c, cudaGetLastError());
    c->ngrids = id + 1;
    *grid_id = id;
    return OVS_OK;
}

int ovs_grid_check(const ovs_ctx* c, int32_t gid, int64_t cells[3], int32_t* overlap) {
    if (!c || gid < 0 || gid >= c->ngrids) return OVS_ERR_ARG;
    if (cells)
        for (int q = 0; q < 3; ++q) cells[q] = c->gh[gid].orient[q];
    if (overlap) *overlap = c->grids[gid].overlap;
    return OVS_OK;
}

int ovs_grid_bins(const ovs_ctx* c, int32_t gid, int64_t out[4]) {
    if (!c || !out || gid < 0 || gid >= c->ngrids) return OVS_ERR_ARG;
    out[0] = c->gh[gid].nbins;
    out[1] = c->gh[gid].nreg;
    out[2] = c->grids[gid].ncrowd;
    out[3] = c->gh[gid].nsubreg;
    return OVS_OK;
}

int ovs_set_grid_overlap(ovs_ctx* c, int32_t gid, int32_t overlap) {
    if (!c) return OVS_ERR_ARG;
    if (gid < 0 || gid >= c->ngrids) return fail(c, OVS_ERR_ARG, "grid %d does not exist", gid);
    if (overlap != 0 && overlap != 1) return fail(c, OVS_ERR_ARG, "overlap must be 0 or 1");
    const int64_t* o = c->gh[gid].orient;
    if (!overlap && (o[2] > 0 || (o[0] > 0 && o[1] > 0)))
        return fail(c, OVS_ERR_ARG, "grid %d has folded cells: its cells may overlap", gid);
    OVS_CUDA(c, cudaSetDevice(c->device));
    c->grids[gid].overlap = overlap;
    OVS_CUDA(c, cudaMemcpyAsync(c->d_grids + gid, &c->grids[gid], sizeof(GridDev), cudaMemcpyHostToDevice, c->stream));
    OVS_CUDA(c, cudaStreamSynchronize(c->stream));
    return OVS_OK;
}

int ovs_set_motion(ovs_ctx* c, int32_t gid, const double R[9], const double cc[3], const double V[3],
                   const double w[3]) {
    if (!c) return OVS_ERR_ARG;
    if (gid < 0 || gid >= c->ngrids) return fail(c, OVS_ERR_ARG, "grid %d does not exist", gid);
    if (!R || !cc || !V || !w) return fail(c, OVS_ERR_ARG, "motion array is NULL");
    for (int q = 0; q < 9; ++q)
        if (!isfinite(R[q])) return fail(c, OVS_ERR_ARG, "R is not finite");
    for (int q = 0; q < 3; ++q)
        if (!isfinite(cc[q]) || !isfinite(V[q]) || !isfinite(w[q])) return fail(c, OVS_ERR_ARG, "c/V/omega not finite");
    // orthogonality and orientation
    double err = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += R[3 * k + a] * R[3 * k + b];
            err = std::max(err, fabs(s - (a == b ? 1.0 : 0.0)));
        }
    double det = R[0] * (R[4] * R[8] - R[5] * R[7]) - R[1] * (R[3] * R[8] - R[5] * R[6]) +
                 R[2] * (R[3] * R[7] - R[4] * R[6]);
    if (err > 1e-12 || det < 0) return fail(c, OVS_ERR_ARG, "R is not a rotation (|R^T R - I| = %g, det %g)", err, det);
    MotionDev& m = c->motion[gid];
    memcpy(m.R, R, sizeof m.R);
    memcpy(m.c, cc, sizeof m.c);
    memcpy(m.V, V, sizeof m.V);
    memcpy(m.w, w, sizeof m.w);
    bool id = R[0] == 1 && R[4] == 1 && R[8] == 1 && R[1] == 0 && R[2] == 0 && R[3] == 0 && R[5] == 0 && R[6] == 0 &&
              R[7] == 0;
    for (int q = 0; q < 3; ++q) id = id && cc[q] == 0 && V[q] == 0 && w[q] == 0;
    m.identity = id ? 1 : 0;
    return OVS_OK;
}

namespace {
struct SurfaceLayout {
    size_t v, tri, start, rec, tr, total;
};
// sections of a surface workspace, each 256-byte aligned
SurfaceLayout surface_layout(int64_t nv, int64_t nt, int64_t nbins, int64_t nreg) {
    SurfaceLayout L;
    size_t off = 0;
    L.v = off;
    off = align_up(off + sizeof(double) * 3 * (size_t)nv);
    L.tri = off;
    off = align_up(off + sizeof(int32_t) * 3 * (size_t)nt);
    L.start = off;
    off = align_up(off + sizeof(int32_t) * (size_t)(nbins + 1));
    L.rec = off;
    off = align_up(off + sizeof(float) * 8 * (size_t)std::max<int64_t>(1, nreg));
    L.tr = off;
    off = align_up(off + sizeof(float) * 4 * (size_t)nt);
    L.total = off;
    return L;
}
bool surface_ok(int64_t nv, const double* v, int64_t nt, const int32_t* tri) {
    if (nv < 3 || nt < 1 || !v || !tri) return false;
    for (int64_t q = 0; q < 3 * nt; ++q)
        if (tri[q] < 0 || tri[q] >= nv) return false;
    for (int64_t q = 0; q < 3 * nv; ++q)
        if (!std::isfinite(v[q])) return false;
    return nt < ((int64_t)1 << 31) / 3;
}
}  // namespace

int ovs_surface_workspace_size(int64_t nv, const double* v, int64_t nt, const int32_t* tri, size_t* bytes) {
    if (!bytes || !surface_ok(nv, v, nt, tri)) return OVS_ERR_ARG;
    SurfaceDev S;
    std::vector<int32_t> start, tris;
    const int64_t nreg = surface_bins(v, nv, tri, nt, S, start, tris);
    *bytes = surface_layout(nv, nt, (int64_t)S.nb[0] * S.nb[1], nreg).total;
    return OVS_OK;
}

int ovs_create_surface(ovs_ctx* c, int32_t body_grid, int64_t nv, const double* v, int64_t nt, const int32_t* tri,
                       void* dws, size_t bytes, int32_t* surface_id) {
    if (!c) return OVS_ERR_ARG;
    if (body_grid < 0 || body_grid >= c->ngrids) return fail(c, OVS_ERR_ARG, "grid %d does not exist", body_grid);
    if (!surface_ok(nv, v, nt, tri)) return fail(c, OVS_ERR_ARG, "bad surface (empty, non-finite or vertex id out of range)");
    if (c->nsurf >= OVS_MAX_GRIDS) return fail(c, OVS_ERR_ARG, "more than %d surfaces", OVS_MAX_GRIDS);
    if (!dws || (uintptr_t)dws % kAlign) return fail(c, OVS_ERR_ARG, "surface workspace NULL or not 256-byte aligned");
    SurfaceDev S;
    std::vector<int32_t> start, tris;
    std::vector<float> rec, tr;
    const int64_t nreg = surface_bins(v, nv, tri, nt, S, start, tris, &rec, &tr);
    const SurfaceLayout L = surface_layout(nv, nt, (int64_t)S.nb[0] * S.nb[1], nreg);
    if (bytes < L.total)
        return fail(c, OVS_ERR_WORKSPACE, "surface workspace has %zu bytes, needs %zu", bytes, L.total);
    OVS_CUDA(c, cudaSetDevice(c->device));
    char* base = (char*)dws;
    OVS_CUDA(c, cudaMemcpyAsync(base + L.v, v, sizeof(double) * 3 * nv, cudaMemcpyHostToDevice, c->stream));
    OVS_CUDA(c, cudaMemcpyAsync(base + L.tri, tri, sizeof(int32_t) * 3 * nt, cudaMemcpyHostToDevice, c->stream));
    OVS_CUDA(c, cudaMemcpyAsync(base + L.start, start.data(), sizeof(int32_t) * start.size(), cudaMemcpyHostToDevice,
                                c->stream));
    if (!rec.empty())
        OVS_CUDA(c, cudaMemcpyAsync(base + L.rec, rec.data(), sizeof(float) * rec.size(), cudaMemcpyHostToDevice,
                                    c->stream));
    OVS_CUDA(c, cudaMemcpyAsync(base + L.tr, tr.data(), sizeof(float) * tr.size(), cudaMemcpyHostToDevice, c->stream));
    OVS_CUDA(c, cudaStreamSynchronize(c->stream));  // the host vectors go out of scope
    S.v = (const double*)(base + L.v);
    S.tri = (const int32_t*)(base + L.tri);
    S.bin_start = (const int32_t*)(base + L.start);
    S.bin_rec = (const float4*)(base + L.rec);
    S.tri_r = (const float4*)(base + L.tr);
    S.nv = nv;
    S.nt = nt;
    c->surf[c->nsurf] = S;
    c->surf_body[c->nsurf] = body_grid;
    if (surface_id) *surface_id = c->nsurf;
    ++c->nsurf;
    return OVS_OK;
}

int ovs_hole_cut_many(ovs_ctx* c, int32_t nsurf, const int32_t* surface_ids, int32_t target_grid, const int64_t* n,
                      const int32_t* const* nodes, uint8_t* iblank) {
    if (!c) return OVS_ERR_ARG;
    if (nsurf < 0 || nsurf > OVS_MAX_GRIDS) return fail(c, OVS_ERR_ARG, "nsurf = %d (0 .. %d)", nsurf, OVS_MAX_GRIDS);
    if (nsurf == 0) return OVS_OK;
    if (!surface_ids || !n) return fail(c, OVS_ERR_ARG, "surface_ids or n is NULL");
    if (target_grid < 0 || target_grid >= c->ngrids) return fail(c, OVS_ERR_ARG, "grid %d does not exist", target_grid);
    HoleJob jobs[OVS_MAX_GRIDS];
    int64_t total = 0;
    for (int32_t s = 0; s < nsurf; ++s) {
        const int32_t id = surface_ids[s];
        if (id < 0 || id >= c->nsurf) return fail(c, OVS_ERR_ARG, "surface %d does not exist", id);
        if (n[s] < 0) return fail(c, OVS_ERR_ARG, "n[%d] = %lld", s, (long long)n[s]);
        const int32_t* nd = nodes ? nodes[s] : nullptr;
        if (!nd && n[s] > c->grids[target_grid].nnodes)
            return fail(c, OVS_ERR_ARG, "n[%d] exceeds the grid's node count", s);
        jobs[s] = {&c->surf[id], &c->motion[c->surf_body[id]], nd, n[s]};
        total += n[s];
    }
    if (total == 0) return OVS_OK;
    if (!iblank) return fail(c, OVS_ERR_ARG, "iblank is NULL");
    OVS_CUDA(c, cudaSetDevice(c->device));
    cudaError_t e = launch_hole_cut(jobs, nsurf, c->grids[target_grid], c->motion[target_grid], iblank, c->d_err,
                                    c->nsm, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "hole_cut launch");
    return OVS_OK;
}

int ovs_hole_cut(ovs_ctx* c, int32_t surface_id, int32_t target_grid, int64_t n, const int32_t* nodes,
                 uint8_t* iblank) {
    const int32_t* nl[1] = {nodes};
    return ovs_hole_cut_many(c, 1, &surface_id, target_grid, &n, nl, iblank);
}

int ovs_set_iblank(ovs_ctx* c, int32_t grid_id, const uint8_t* iblank) {
    if (!c) return OVS_ERR_ARG;
    if (grid_id < 0 || grid_id >= c->ngrids) return fail(c, OVS_ERR_ARG, "grid %d does not exist", grid_id);
    OVS_CUDA(c, cudaSetDevice(c->device));
    cudaError_t e = launch_mark_blocked(c->grids[grid_id], iblank, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_iblank launch");
    c->grids[grid_id].blanked = iblank ? 1 : 0;
    OVS_CUDA(c, cudaMemcpyAsync(c->d_grids + grid_id, &c->grids[grid_id], sizeof(GridDev), cudaMemcpyHostToDevice,
                                c->stream));
    OVS_CUDA(c, cudaStreamSynchronize(c->stream));  // the host copy is the source of the transfer
    return OVS_OK;
}

int ovs_set_options(ovs_ctx* c, const ovs_options* o) {
    if (!c) return OVS_ERR_ARG;
    if (!o) return fail(c, OVS_ERR_ARG, "options is NULL");
    if (o->velocity_mode < OVS_VEL_RELATIVE || o->velocity_mode > OVS_VEL_NONE)
        return fail(c, OVS_ERR_ARG, "velocity_mode %d", o->velocity_mode);
    if (o->guess < OVS_GUESS_HINT || o->guess > OVS_GUESS_MLP_ONLY) return fail(c, OVS_ERR_ARG, "guess %d", o->guess);
    if (o->max_walk < 1 || o->max_walk > 1024) return fail(c, OVS_ERR_ARG, "max_walk %d (1..1024)", o->max_walk);
    if (o->launch != OVS_LAUNCH_DIRECT && o->launch != OVS_LAUNCH_GRAPH) return fail(c, OVS_ERR_ARG, "launch %d", o->launch);
    c->opts = *o;
    return OVS_OK;
}

int ovs_get_options(const ovs_ctx* c, ovs_options* o) {
    if (!c || !o) return OVS_ERR_ARG;
    *o = c->opts;
    return OVS_OK;
}

}  // extern "C"

namespace {

// fields checks shared by ovs_interpolate and ovs_assemble_interpolate
int check_fields(ovs_ctx* c, const ovs_fringe_set* sets, int32_t nsets, const ovs_fields* fields, int32_t nfields,
                 const ovs_fields_out* out) {
    if (!fields || nfields != c->ngrids) return fail(c, OVS_ERR_ARG, "fields must have one entry per grid (%d)", c->ngrids);
    if (!out) return fail(c, OVS_ERR_ARG, "fields output is NULL");
    if (out->dtype != OVS_F32 && out->dtype != OVS_F64) return fail(c, OVS_ERR_ARG, "output dtype");
    if (!out->u || !out->v || !out->w || !out->p) return fail(c, OVS_ERR_ARG, "output array is NULL");
    // every possible donor of these sets must carry fields of the output dtype
    for (int s = 0; s < nsets; ++s)
        for (int d = 0; d < sets[s].n_donors; ++d) {
            const ovs_fields& f = fields[sets[s].donors[d]];
            if (!f.u || !f.v || !f.w || !f.p)
                return fail(c, OVS_ERR_ARG, "donor grid %d has a NULL field", sets[s].donors[d]);
            if (f.dtype != out->dtype)
                return fail(c, OVS_ERR_ARG, "donor grid %d fields dtype %d != output dtype %d", sets[s].donors[d],
                            f.dtype, out->dtype);
            if (f.stride < 0) return fail(c, OVS_ERR_ARG, "donor grid %d fields stride %d", sets[s].donors[d], f.stride);
        }
    return OVS_OK;
}

void fill_interp(const ovs_ctx* c, const ovs_fringe_set* sets, int32_t nsets, const ovs_donors* in,
                 const ovs_fields* fields, const ovs_fields_out* out, int64_t total, InterpParams* P) {
    P->nsets = nsets;
    P->xi_f64 = in->xi_dtype == OVS_F64;
    P->mode = c->opts.velocity_mode;
    P->f64 = out->dtype == OVS_F64;
    P->ngrids = c->ngrids;
    P->err = c->d_err;
    P->total = total;
    P->in_grid = in->grid;
    P->in_cell = in->cell;
    P->in_xi = in->xi;
    P->in_status = in->status;
    P->out[0] = out->u;
    P->out[1] = out->v;
    P->out[2] = out->w;
    P->out[3] = out->p;
    fill_sets(sets, nsets, P->s);
    memcpy(P->m, c->motion, sizeof P->m);
    fill_motion_f32(c, P->mf);
    fill_vel_affine(c, sets, nsets, P->mode, P->va);
    for (int g = 0; g < c->ngrids; ++g) {
        FieldsDev& F = P->fields[g];
        F.f[0] = fields[g].u;
        F.f[1] = fields[g].v;
        F.f[2] = fields[g].w;
        F.f[3] = fields[g].p;
        F.stride = fields[g].stride > 1 ? fields[g].stride : 1;
        const size_t es = fields[g].dtype == OVS_F64 ? 8 : 4;
        const char* u = (const char*)fields[g].u;
        F.rec4 = F.stride == 4 && u && (uintptr_t)u % 16 == 0 && (const char*)fields[g].v == u + es &&
                 (const char*)fields[g].w == u + 2 * es && (const char*)fields[g].p == u + 3 * es;
        F.pad = 0;
    }
}

// Kinds of call (bit set): which kernels a call launches.
constexpr uint32_t kStepAssemble = 1, kStepInterp = 2, kStepInterpF64 = 4, kStepNoAlloc = 8, kStepMlp = 16;

// The learned guess of a call: with OVS_GUESS_MLP / OVS_GUESS_MLP_ONLY, every grid's network (width, box, input
// normalisation as in its header, region) for the assembly kernel, which evaluates it for the points that have no
// usable hint.  Returns whether any grid has one.
bool fill_guess(const ovs_ctx* c, AsmParams* P) {
    const bool mlp = c->opts.guess == OVS_GUESS_MLP || c->opts.guess == OVS_GUESS_MLP_ONLY;
    bool any = false;
    for (int g = 0; g < OVS_MAX_GRIDS; ++g) {
        GuessDev& d = P->gn[g];
        memset(&d, 0, sizeof d);
        if (!mlp || g >= c->ngrids || !c->hidden[g]) continue;
        const GridDev& gr = c->grids[g];
        for (int a = 0; a < 3; ++a) {
            d.lo[a] = (float)gr.lo[a];
            d.hi[a] = (float)gr.hi[a];
            d.centre[a] = (float)(0.5 * (gr.lo[a] + gr.hi[a]));
            d.inv_half[a] = (float)(2.0 / (gr.hi[a] - gr.lo[a]));
        }
        d.hidden = c->hidden[g];
        d.region = gr.mlp;
        any = true;
    }
    P->guess_mlp = any ? 1 : 0;
    P->guess_always = any && c->opts.guess == OVS_GUESS_MLP_ONLY;
    P->guess_used = any && c->opts.collect_stats ? c->d_counters + kCtrGuess : nullptr;
    return any;
}

// The staging buffer for the next call, once the call that last read it has finished.
cudaError_t acquire_stage(ovs_ctx* c, int* b) {
    const int k = c->stage;
    if (c->step_used[k]) {
        cudaError_t e = cudaEventSynchronize(c->step_done[k]);
        if (e != cudaSuccess) return e;
    }
    c->stage ^= 1;
    *b = k;
    return cudaSuccess;
}

// The launch sequence of one call on stream st: the parameter copy from staging buffer b, then the kernels.
cudaError_t enqueue_step(ovs_ctx* c, int b, uint32_t kind, uint32_t* qcount, cudaStream_t st, bool trace) {
    cudaError_t e = cudaMemcpyAsync(c->d_step, c->h_step[b], sizeof(StepParams), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    if (kind & kStepAssemble) {
        // with fields, the assembly kernels interpolate every point as they decide its donor (one pass)
        const int im = (kind & kStepInterp) ? ((kind & kStepInterpF64) ? 2 : 1) : 0;
        e = launch_assemble(c->d_step, im, (kind & kStepMlp) != 0, qcount, c->d_grids, c->nsm,
                            c->tune.assemble_blocks_per_sm, c->tune.slow_blocks_per_sm, st,
                            trace ? c->trace : nullptr);
        if (e != cudaSuccess || !im) return e;
        if (trace && c->trace[3]) cudaEventRecord(c->trace[3], st);
        if (trace && c->trace[4]) cudaEventRecord(c->trace[4], st);
        return cudaSuccess;
    }
    if (kind & kStepInterp)
        e = launch_interp(&c->d_step->i, (kind & kStepInterpF64) != 0, c->d_grids, c->nsm,
                          c->tune.interp_blocks_per_sm, st, trace ? c->trace + 3 : nullptr);
    return e;
}

// Run one call whose parameters sit in staging buffer b: as the CUDA graph of its kind (captured on the kind's
// first call, one instance per staging buffer) or as direct launches; the buffer stays busy until the call ends.
cudaError_t run_step(ovs_ctx* c, int b, uint32_t kind, uint32_t* qcount, bool allow_graph) {
    cudaError_t e = cudaSuccess;
    if (allow_graph && c->opts.launch == OVS_LAUNCH_GRAPH && !c->tracing) {
        ovs_ctx::GraphEntry* ge = nullptr;
        for (auto& g : c->graphs)
            if (g.kind == kind) ge = &g;
        if (!ge) {
            ovs_ctx::GraphEntry ng{kind, {nullptr, nullptr}};
            for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
                cudaGraph_t graph = nullptr;
                e = cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeRelaxed);
                if (e != cudaSuccess) break;
                const cudaError_t e1 = enqueue_step(c, k, kind, qcount, c->gstream, false);
                const cudaError_t e2 = cudaStreamEndCapture(c->gstream, &graph);
                e = e1 != cudaSuccess ? e1 : e2;
                if (e == cudaSuccess) e = cudaGraphInstantiate(&ng.exec[k], graph, 0);
                if (graph) cudaGraphDestroy(graph);
            }
            if (e != cudaSuccess) {
                for (auto& x : ng.exec)
                    if (x) cudaGraphExecDestroy(x);
                return e;
            }
            c->graphs.push_back(ng);
            ge = &c->graphs.back();
        }
        e = cudaGraphLaunch(ge->exec[b], c->stream);
    } else {
        e = enqueue_step(c, b, kind, qcount, c->stream, c->tracing);
    }
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(c->step_done[b], c->stream);
    c->step_used[b] = true;
    return e;
}

// Forget the captured graphs (after the launch shapes change); waits for the stream first.
void drop_graphs(ovs_ctx* c) {
    cudaStreamSynchronize(c->stream);
    for (auto& g : c->graphs)
        for (auto& x : g.exec)
            if (x) cudaGraphExecDestroy(x);
    c->graphs.clear();
}

int assemble_impl(ovs_ctx* c, const ovs_fringe_set* sets, int32_t nsets, const ovs_donors* out,
                  const ovs_fields* fields, int32_t nfields, const ovs_fields_out* fout) {
    if (!c) return OVS_ERR_ARG;
    if (!c->ws) return fail(c, OVS_ERR_STATE, "no workspace attached");
    int64_t total = 0;
    int rc = check_sets(c, sets, nsets, &total);
    if (rc != OVS_OK) return rc;
    if (!out) return fail(c, OVS_ERR_ARG, "donors output is NULL");
    if (out->n < total) return fail(c, OVS_ERR_ARG, "donors capacity %lld < %lld points", (long long)out->n, (long long)total);
    if (fout) {
        rc = check_fields(c, sets, nsets, fields, nfields, fout);
        if (rc != OVS_OK) return rc;
    }
    if (total == 0) return OVS_OK;
    if (!out->grid || !out->cell || !out->xi || !out->status) return fail(c, OVS_ERR_ARG, "donors array is NULL");
    if (out->xi_dtype != OVS_F32 && out->xi_dtype != OVS_F64) return fail(c, OVS_ERR_ARG, "xi_dtype");
    if (out->n != total)
        return fail(c, OVS_ERR_ARG, "donors.n (%lld) must equal the number of points (%lld): xi is SoA over n",
                    (long long)out->n, (long long)total);
    OVS_CUDA(c, cudaSetDevice(c->device));
    int b = 0;
    OVS_CUDA(c, acquire_stage(c, &b));
    StepParams& S = *c->h_step[b];
    AsmParams* P = &S.a;
    memset(P, 0, offsetof(AsmParams, s));
    P->nsets = nsets;
    P->xi_f64 = out->xi_dtype == OVS_F64;
    P->max_walk = c->opts.max_walk;
    // learned guess: the assembly kernel starts the points without a usable hint where the network says, the
    // others from their hints
    const bool mlp = c->opts.guess == OVS_GUESS_MLP || c->opts.guess == OVS_GUESS_MLP_ONLY;
    P->guess = mlp ? OVS_GUESS_HINT : c->opts.guess;
    P->stats = c->opts.collect_stats;
    P->total = total;
    P->queue_cap = 2 * c->max_points;
    P->out_grid = out->grid;
    P->out_cell = out->cell;
    P->out_xi = out->xi;
    P->out_status = out->status;
    P->queue = c->d_queue;
    P->queue_count = c->d_qcount;
    P->counters = c->d_counters;
    P->err = c->d_err;
    fill_sets(sets, nsets, P->s);
    fill_xforms(c, sets, nsets, P->xf);
    memcpy(P->m, c->motion, sizeof P->m);
    uint32_t kind = kStepAssemble | (fill_guess(c, P) ? kStepMlp : 0u);
    if (fout) {
        memset(&S.i, 0, offsetof(InterpParams, s));
        fill_interp(c, sets, nsets, out, fields, fout, total, &S.i);
        kind |= kStepInterp | (S.i.f64 ? kStepInterpF64 : 0);
    }
    cudaError_t e = run_step(c, b, kind, c->d_qcount, true);
    if (e != cudaSuccess) return cuda_fail(c, e, "assemble launch");
    return OVS_OK;
}

}  // namespace

extern "C" {

int ovs_assemble(ovs_ctx* c, const ovs_fringe_set* sets, int32_t nsets, const ovs_donors* out) {
    return assemble_impl(c, sets, nsets, out, nullptr, 0, nullptr);
}

int ovs_assemble_interpolate(ovs_ctx* c, const ovs_fringe_set* sets, int32_t nsets, const ovs_donors* out,
                             const ovs_fields* fields, int32_t nfields, const ovs_fields_out* fout) {
    if (c && !fout) return fail(c, OVS_ERR_ARG, "fields output is NULL");
    return assemble_impl(c, sets, nsets, out, fields, nfields, fout);
}

int ovs_interpolate(ovs_ctx* c, const ovs_fringe_set* sets, int32_t nsets, const ovs_donors* in,
                    const ovs_fields* fields, int32_t nfields, const ovs_fields_out* out) {
    if (!c) return OVS_ERR_ARG;
    if (!c->ws) return fail(c, OVS_ERR_STATE, "no workspace attached");
    int64_t total = 0;
    int rc = check_sets(c, sets, nsets, &total);
    if (rc != OVS_OK) return rc;
    if (!in || !out) return fail(c, OVS_ERR_ARG, "donors or output is NULL");
    if (in->n != total) return fail(c, OVS_ERR_ARG, "donors.n (%lld) != points (%lld)", (long long)in->n, (long long)total);
    if (total == 0) return OVS_OK;
    rc = check_fields(c, sets, nsets, fields, nfields, out);
    if (rc != OVS_OK) return rc;
    if (!in->grid || !in->cell || !in->xi || !in->status) return fail(c, OVS_ERR_ARG, "donors array is NULL");
    OVS_CUDA(c, cudaSetDevice(c->device));
    int b = 0;
    OVS_CUDA(c, acquire_stage(c, &b));
    InterpParams* P = &c->h_step[b]->i;
    memset(P, 0, offsetof(InterpParams, s));
    fill_interp(c, sets, nsets, in, fields, out, total, P);
    cudaError_t e = run_step(c, b, kStepInterp | (P->f64 ? kStepInterpF64 : 0), c->d_qcount, true);
    if (e != cudaSuccess) return cuda_fail(c, e, "interpolate launch");
    return OVS_OK;
}

int ovs_guess_param_count(int32_t hidden, int64_t* count) {
    if (!count || (hidden != 32 && hidden != 64 && hidden != 128)) return OVS_ERR_ARG;
    *count = mlp_param_count(hidden);
    return OVS_OK;
}

int ovs_train_workspace_size(const ovs_train_desc* d, size_t* bytes) {
    if (!d || !bytes || d->n_samples < 1) return OVS_ERR_ARG;
    *bytes = align_up((size_t)d->n_samples * 6 * sizeof(float));
    return OVS_OK;
}

}  // extern "C"

namespace {

int set_header(ovs_ctx* c, int gid, int H, int ready) {
    MlpHeader h;
    memset(&h, 0, sizeof h);
    h.hidden = H;
    h.ready = ready;
    const GridDev& g = c->grids[gid];
    for (int a = 0; a < 3; ++a) {
        h.centre[a] = (float)(0.5 * (g.lo[a] + g.hi[a]));
        h.inv_half[a] = (float)(2.0 / (g.hi[a] - g.lo[a]));
    }
    OVS_CUDA(c, cudaMemcpyAsync((void*)g.mlp, &h, sizeof h, cudaMemcpyHostToDevice, c->stream));
    OVS_CUDA(c, cudaStreamSynchronize(c->stream));
    return OVS_OK;
}

int check_grid(ovs_ctx* c, int32_t gid) {
    if (!c) return OVS_ERR_ARG;
    if (gid < 0 || gid >= c->ngrids) return fail(c, OVS_ERR_ARG, "grid %d does not exist", gid);
    return OVS_OK;
}

}  // namespace

extern "C" {

int ovs_train_guess(ovs_ctx* c, int32_t gid, const ovs_train_desc* d, float* final_loss) {
    int rc = check_grid(c, gid);
    if (rc != OVS_OK) return rc;
    if (!d) return fail(c, OVS_ERR_ARG, "training descriptor is NULL");
    const int H = d->hidden;
    if (H != 32 && H != 64 && H != 128) return fail(c, OVS_ERR_ARG, "hidden width %d (32, 64 or 128)", H);
    if (d->n_samples < 1 || !d->cells || !d->xi || !d->init_params) return fail(c, OVS_ERR_ARG, "samples or initial parameters");
    if (d->epochs < 1 || d->batch < 1 || !(d->lr > 0) || !(d->lr_final >= 0))
        return fail(c, OVS_ERR_ARG, "epochs, batch and lr must be positive (lr_final >= 0)");
    size_t need = 0;
    ovs_train_workspace_size(d, &need);
    if (!d->scratch || d->scratch_bytes < need)
        return fail(c, OVS_ERR_WORKSPACE, "training scratch has %zu bytes, needs %zu", d->scratch_bytes, need);
    OVS_CUDA(c, cudaSetDevice(c->device));
    char* region = (char*)c->grids[gid].mlp;
    const int np = mlp_param_count(H);
    float* params = (float*)(region + kMlpParamsOffset);
    float* m = (float*)(region + kMlpMOffset);
    float* v = (float*)(region + kMlpVOffset);
    float* grads = (float*)(region + kMlpGOffset);
    float* loss = (float*)(region + kMlpLossOffset);
    c->hidden[gid] = 0;
    if ((rc = set_header(c, gid, H, 0)) != OVS_OK) return rc;
    MlpHeader h;
    OVS_CUDA(c, cudaMemcpy(&h, region, sizeof h, cudaMemcpyDeviceToHost));
    OVS_CUDA(c, cudaMemcpyAsync(params, d->init_params, sizeof(float) * np, cudaMemcpyDeviceToDevice, c->stream));
    OVS_CUDA(c, cudaMemsetAsync(m, 0, sizeof(float) * np, c->stream));
    OVS_CUDA(c, cudaMemsetAsync(v, 0, sizeof(float) * np, c->stream));
    OVS_CUDA(c, cudaMemsetAsync(grads, 0, sizeof(float) * np, c->stream));
    const int64_t n = d->n_samples;
    float* X = (float*)d->scratch;
    float* T = X + 3 * n;
    OVS_CUDA(c, launch_train_samples(c->grids[gid], h, d->cells, d->xi, n, X, T, c->stream));
    int step = 0;
    int64_t nb = 0;
    const int64_t per_epoch = (n + d->batch - 1) / d->batch;
    const double total_steps = (double)per_epoch * d->epochs;
    for (int ep = 0; ep < d->epochs; ++ep) {
        OVS_CUDA(c, cudaMemsetAsync(loss, 0, sizeof(float), c->stream));
        nb = 0;
        for (int64_t off = 0; off < n; off += d->batch) {
            const int64_t B = std::min<int64_t>(d->batch, n - off);
            // cosine decay from lr to lr_final over all steps (constant when lr_final is 0)
            double lr = d->lr;
            if (d->lr_final > 0)
                lr = d->lr_final + 0.5 * (d->lr - d->lr_final) * (1.0 + cos(M_PI * step / std::max(1.0, total_steps - 1)));
            OVS_CUDA(c, launch_train_grad(H, params, X, T, n, off, B, grads, loss, 1.0f / (3.0f * (float)B), c->stream));
            OVS_CUDA(c, launch_adam(params, grads, m, v, np, (float)lr, ++step, c->stream));
            ++nb;
        }
    }
    float lsum = 0;
    OVS_CUDA(c, cudaMemcpyAsync(&lsum, loss, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    OVS_CUDA(c, launch_pack(params, H, region, c->stream));
    OVS_CUDA(c, cudaStreamSynchronize(c->stream));
    if ((rc = set_header(c, gid, H, 1)) != OVS_OK) return rc;
    c->hidden[gid] = H;
    if (final_loss) *final_loss = lsum / (float)nb;
    return OVS_OK;
}

int ovs_guess_set_params(ovs_ctx* c, int32_t gid, int32_t H, const float* dparams) {
    int rc = check_grid(c, gid);
    if (rc != OVS_OK) return rc;
    if (H != 32 && H != 64 && H != 128) return fail(c, OVS_ERR_ARG, "hidden width %d (32, 64 or 128)", H);
    if (!dparams) return fail(c, OVS_ERR_ARG, "parameters are NULL");
    OVS_CUDA(c, cudaSetDevice(c->device));
    char* region = (char*)c->grids[gid].mlp;
    float* params = (float*)(region + kMlpParamsOffset);
    c->hidden[gid] = 0;
    if ((rc = set_header(c, gid, H, 0)) != OVS_OK) return rc;
    OVS_CUDA(c, cudaMemcpyAsync(params, dparams, sizeof(float) * mlp_param_count(H), cudaMemcpyDeviceToDevice,
                                c->stream));
    OVS_CUDA(c, launch_pack(params, H, region, c->stream));
    if ((rc = set_header(c, gid, H, 1)) != OVS_OK) return rc;
    c->hidden[gid] = H;
    return OVS_OK;
}

int ovs_guess_get_params(ovs_ctx* c, int32_t gid, float* dparams, int32_t* hidden) {
    int rc = check_grid(c, gid);
    if (rc != OVS_OK) return rc;
    if (!hidden) return fail(c, OVS_ERR_ARG, "hidden is NULL");
    *hidden = c->hidden[gid];
    if (!c->hidden[gid]) return OVS_OK;
    if (!dparams) return fail(c, OVS_ERR_ARG, "parameters are NULL");
    OVS_CUDA(c, cudaSetDevice(c->device));
    const char* region = (const char*)c->grids[gid].mlp;
    OVS_CUDA(c, cudaMemcpyAsync(dparams, region + kMlpParamsOffset, sizeof(float) * mlp_param_count(c->hidden[gid]),
                                cudaMemcpyDeviceToDevice, c->stream));
    return OVS_OK;
}

int ovs_guess_eval(ovs_ctx* c, int32_t gid, int64_t n, const float* xn, float* out) {
    int rc = check_grid(c, gid);
    if (rc != OVS_OK) return rc;
    if (!c->hidden[gid]) return fail(c, OVS_ERR_STATE, "grid %d has no guess network", gid);
    if (n < 0 || (n > 0 && (!xn || !out))) return fail(c, OVS_ERR_ARG, "inputs or outputs");
    if (n == 0) return OVS_OK;
    OVS_CUDA(c, cudaSetDevice(c->device));
    OVS_CUDA(c, launch_guess_eval(c->hidden[gid], c->grids[gid].mlp, xn, n, out, c->stream));
    return OVS_OK;
}

int ovs_mlp_loss_grad(ovs_ctx* c, int32_t H, int64_t n, const float* xn, const float* target, const float* params,
                      float* grads, float* loss) {
    if (!c) return OVS_ERR_ARG;
    if (H != 32 && H != 64 && H != 128) return fail(c, OVS_ERR_ARG, "hidden width %d (32, 64 or 128)", H);
    if (n < 1 || !xn || !target || !params || !grads || !loss) return fail(c, OVS_ERR_ARG, "arguments");
    OVS_CUDA(c, cudaSetDevice(c->device));
    OVS_CUDA(c, cudaMemsetAsync(grads, 0, sizeof(float) * mlp_param_count(H), c->stream));
    OVS_CUDA(c, cudaMemsetAsync(loss, 0, sizeof(float), c->stream));
    OVS_CUDA(c, launch_train_grad(H, params, xn, target, n, 0, n, grads, loss, 1.0f / (3.0f * (float)n), c->stream));
    return OVS_OK;
}

int ovs_sync(ovs_ctx* c) {
    if (!c) return OVS_ERR_ARG;
    OVS_CUDA(c, cudaSetDevice(c->device));
    OVS_CUDA(c, cudaStreamSynchronize(c->stream));
    if (!c->ws) return OVS_OK;
    int32_t err = 0;
    OVS_CUDA(c, cudaMemcpy(&err, c->d_err, 4, cudaMemcpyDeviceToHost));
    if (err) {
        OVS_CUDA(c, cudaMemset(c->d_err, 0, 4));
        return fail(c, OVS_ERR_DEVICE, "device status word 0x%x%s%s%s", err,
                    (err & kErrQueueOverflow) ? " (slow-path queue overflow)" : "",
                    (err & kErrBadNode) ? " (node id out of range: points marked BADINPUT)" : "",
                    (err & kErrBadCell) ? " (donor record unusable: outputs zeroed)" : "");
    }
    return OVS_OK;
}

int ovs_get_stats(ovs_ctx* c, ovs_stats* out, int reset) {
    if (!c || !out) return OVS_ERR_ARG;
    if (!c->ws) return fail(c, OVS_ERR_STATE, "no workspace attached");
    OVS_CUDA(c, cudaSetDevice(c->device));
    unsigned long long h[kNumCounters];
    OVS_CUDA(c, cudaMemcpyAsync(h, c->d_counters, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    OVS_CUDA(c, cudaStreamSynchronize(c->stream));
    out->points = (int64_t)h[kCtrPoints];
    out->walk_steps = (int64_t)h[kCtrWalk];
    out->refined = (int64_t)h[kCtrRefined];
    out->fallback = (int64_t)h[kCtrFallback];
    out->guess_used = (int64_t)h[kCtrGuess];
    out->newton_iterations = (int64_t)h[kCtrNewton];
    out->warp_walk_steps = (int64_t)h[kCtrWarpWalk];
    out->near_face = (int64_t)h[kCtrNear];
    out->stuck = (int64_t)h[kCtrStuck];
    if (reset) OVS_CUDA(c, cudaMemsetAsync(c->d_counters, 0, sizeof h, c->stream));
    return OVS_OK;
}

int ovs_set_trace_events(ovs_ctx* c, void* const* ev, int32_t n) {
    if (!c) return OVS_ERR_ARG;
    if (n < 0 || n > 7) return fail(c, OVS_ERR_ARG, "n = %d (0..7)", n);
    for (int q = 0; q < 7; ++q) c->trace[q] = (ev && q < n) ? (cudaEvent_t)ev[q] : nullptr;
    c->tracing = ev && n > 0;
    return OVS_OK;
}

int ovs_reset_hints(ovs_ctx* c) {
    if (!c) return OVS_ERR_ARG;
    OVS_CUDA(c, cudaSetDevice(c->device));
    for (int g = 0; g < c->ngrids; ++g)
        OVS_CUDA(c, cudaMemsetAsync(c->grids[g].hint, 0xFF, (size_t)c->grids[g].nnodes * 4, c->stream));
    return OVS_OK;
}

int ovs_get_donors(ovs_ctx* c, int32_t grid_id, uint32_t* dst) {
    if (!c) return OVS_ERR_ARG;
    if (grid_id < 0 || grid_id >= c->ngrids) return fail(c, OVS_ERR_ARG, "grid %d does not exist", grid_id);
    if (!dst) return fail(c, OVS_ERR_ARG, "dst is NULL");
    OVS_CUDA(c, cudaSetDevice(c->device));
    OVS_CUDA(c, cudaMemcpyAsync(dst, c->grids[grid_id].hint, (size_t)c->grids[grid_id].nnodes * 4,
                                cudaMemcpyDeviceToDevice, c->stream));
    return OVS_OK;
}

int ovs_set_donors(ovs_ctx* c, int32_t grid_id, const uint32_t* src) {
    if (!c) return OVS_ERR_ARG;
    if (grid_id < 0 || grid_id >= c->ngrids) return fail(c, OVS_ERR_ARG, "grid %d does not exist", grid_id);
    if (!src) return fail(c, OVS_ERR_ARG, "src is NULL");
    OVS_CUDA(c, cudaSetDevice(c->device));
    OVS_CUDA(c, cudaMemcpyAsync(c->grids[grid_id].hint, src, (size_t)c->grids[grid_id].nnodes * 4,
                                cudaMemcpyDeviceToDevice, c->stream));
    return OVS_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------------
// the interpolation matrix
extern "C" {

int ovs_interp_matrix(ovs_ctx* c, const ovs_donors* in, int32_t* row_ptr, int64_t* col, void* val,
                      int32_t val_dtype) {
    if (!c) return OVS_ERR_ARG;
    if (!c->ws) return fail(c, OVS_ERR_STATE, "no workspace attached");
    if (!in || !row_ptr) return fail(c, OVS_ERR_ARG, "donors or row_ptr is NULL");
    if (val_dtype != OVS_F32 && val_dtype != OVS_F64) return fail(c, OVS_ERR_ARG, "val_dtype %d", val_dtype);
    if (in->n < 0) return fail(c, OVS_ERR_ARG, "donors.n = %lld", (long long)in->n);
    if (in->n > c->max_points)
        return fail(c, OVS_ERR_WORKSPACE, "%lld points exceed the workspace's max_points %lld", (long long)in->n,
                    (long long)c->max_points);
    if (8 * in->n >= ((int64_t)1 << 31)) return fail(c, OVS_ERR_ARG, "more than 2^31 matrix entries");
    OVS_CUDA(c, cudaSetDevice(c->device));
    if (in->n == 0) {
        OVS_CUDA(c, cudaMemsetAsync(row_ptr, 0, sizeof(int32_t), c->stream));
        return OVS_OK;
    }
    if (!in->grid || !in->cell || !in->xi || !in->status || !col || !val)
        return fail(c, OVS_ERR_ARG, "a donors array, col or val is NULL");
    if (in->xi_dtype != OVS_F32 && in->xi_dtype != OVS_F64) return fail(c, OVS_ERR_ARG, "xi_dtype");
    if (interp_matrix_scratch_bytes(in->n) > (size_t)std::max<int64_t>(1, c->max_points) * sizeof(SlowEntry))
        return fail(c, OVS_ERR_WORKSPACE, "workspace scratch too small");
    NodeOffsets off;
    int64_t o = 0;
    for (int g = 0; g < OVS_MAX_GRIDS; ++g) {
        off.off[g] = o;
        if (g < c->ngrids) o += c->grids[g].nnodes;
    }
    cudaError_t e = launch_interp_matrix(c->d_grids, c->ngrids, off, in->status, in->grid, in->cell, in->xi,
                                         in->xi_dtype == OVS_F64, in->n, (uint32_t*)c->d_queue, row_ptr, col, val,
                                         val_dtype == OVS_F64, c->d_err, c->nsm, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "interp_matrix launch");
    return OVS_OK;
}

int ovs_spmv(ovs_ctx* c, int64_t nrows, const int32_t* row_ptr, const int64_t* col, const void* val, const void* x,
             void* y, int32_t dtype) {
    if (!c) return OVS_ERR_ARG;
    if (nrows < 0) return fail(c, OVS_ERR_ARG, "nrows = %lld", (long long)nrows);
    if (dtype != OVS_F32 && dtype != OVS_F64) return fail(c, OVS_ERR_ARG, "dtype %d", dtype);
    if (nrows == 0) return OVS_OK;
    if (!row_ptr || !col || !val || !x || !y) return fail(c, OVS_ERR_ARG, "a matrix or vector pointer is NULL");
    OVS_CUDA(c, cudaSetDevice(c->device));
    cudaError_t e = launch_spmv(nrows, row_ptr, col, val, x, y, dtype == OVS_F64, c->nsm, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "spmv launch");
    return OVS_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------------
// launch shapes and the autotuner
extern "C" {

int ovs_set_tuning(ovs_ctx* c, const ovs_tuning* t) {
    if (!c) return OVS_ERR_ARG;
    ovs_tuning v = t ? *t : ovs_tuning{0, 0, 0, 0, 0};
    if (v.assemble_blocks_per_sm < 0 || v.assemble_blocks_per_sm > 12 || v.interp_blocks_per_sm < 0 ||
        v.interp_blocks_per_sm > 32 || v.slow_blocks_per_sm < 0 || v.slow_blocks_per_sm > 8 ||
        v.guess_blocks_per_sm < 0 || v.guess_blocks_per_sm > 32 ||
        (v.launch != 0 && v.launch != OVS_LAUNCH_GRAPH && v.launch != OVS_LAUNCH_DIRECT))
        return fail(c, OVS_ERR_ARG, "tuning out of range (%d, %d, %d, %d, launch %d)", v.assemble_blocks_per_sm,
                    v.interp_blocks_per_sm, v.slow_blocks_per_sm, v.guess_blocks_per_sm, v.launch);
    OVS_CUDA(c, cudaSetDevice(c->device));
    drop_graphs(c);
    if (v.launch) c->opts.launch = v.launch;
    v.launch = 0;
    c->tune = v;
    return OVS_OK;
}

int ovs_get_tuning(const ovs_ctx* c, ovs_tuning* t) {
    if (!c || !t) return OVS_ERR_ARG;
    *t = c->tune;
    t->launch = c->opts.launch;
    return OVS_OK;
}

int ovs_autotune(ovs_ctx* c, const ovs_fringe_set* sets, int32_t nsets, const ovs_donors* out,
                 const ovs_fields* fields, int32_t nfields, const ovs_fields_out* fout, int32_t reps,
                 ovs_tuning* best) {
    if (!c) return OVS_ERR_ARG;
    if (reps < 1 || reps > 1000) return fail(c, OVS_ERR_ARG, "reps = %d (1..1000)", reps);
    OVS_CUDA(c, cudaSetDevice(c->device));
    const int saved_launch = c->opts.launch;
    const ovs_tuning saved = c->tune;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(c, cudaGetLastError(), "autotune events");
    }
    // candidates run as direct launches (no capture per candidate)
    c->opts.launch = OVS_LAUNCH_DIRECT;
    auto trial = [&](const ovs_tuning& t, float* ms) -> int {
        c->tune = t;
        int rc = assemble_impl(c, sets, nsets, out, fields, nfields, fout);  // untimed
        if (rc != OVS_OK) return rc;
        if (cudaEventRecord(e0, c->stream) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "autotune");
        for (int r = 0; r < reps && rc == OVS_OK; ++r) rc = assemble_impl(c, sets, nsets, out, fields, nfields, fout);
        if (rc != OVS_OK) return rc;
        cudaError_t e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
        if (e != cudaSuccess) return cuda_fail(c, e, "autotune timing");
        *ms /= (float)reps;
        return OVS_OK;
    };
    const int occ = interp_default_blocks_per_sm(false);
    ovs_tuning cur = {3, occ > 0 ? occ : 4, 1, 0};
    float best_ms = 0.f;
    int rc = trial(cur, &best_ms);
    const int cand_asm[] = {1, 2, 3, 4, 6};
    const int cand_slow[] = {1, 2, 4, 8};
    auto sweep = [&](int32_t ovs_tuning::*knob, const int* vals, int nv) {
        for (int k = 0; k < nv && rc == OVS_OK; ++k) {
            if (vals[k] == cur.*knob) continue;
            ovs_tuning t = cur;
            t.*knob = vals[k];
            float ms = 0.f;
            rc = trial(t, &ms);
            if (rc == OVS_OK && ms < 0.99f * best_ms) {
                cur = t;
                best_ms = ms;
            }
        }
    };
    if (rc == OVS_OK) sweep(&ovs_tuning::assemble_blocks_per_sm, cand_asm, 5);
    if (rc == OVS_OK) sweep(&ovs_tuning::slow_blocks_per_sm, cand_slow, 4);
    // the launch mode for the chosen shapes: a CUDA graph per call (captured by the untimed call) or direct
    int launch = saved_launch;
    if (rc == OVS_OK) {
        float direct_ms = 0.f, graph_ms = 0.f;
        rc = trial(cur, &direct_ms);
        if (rc == OVS_OK) {
            drop_graphs(c);
            c->opts.launch = OVS_LAUNCH_GRAPH;
            rc = trial(cur, &graph_ms);
            c->opts.launch = OVS_LAUNCH_DIRECT;
        }
        if (rc == OVS_OK) launch = direct_ms < 0.99f * graph_ms ? OVS_LAUNCH_DIRECT : OVS_LAUNCH_GRAPH;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->opts.launch = saved_launch;
    if (rc != OVS_OK) {
        c->tune = saved;
        return rc;
    }
    drop_graphs(c);
    c->tune = cur;
    c->opts.launch = launch;
    if (best) {
        *best = cur;
        best->launch = launch;
    }
    return OVS_OK;
}

int ovs_interface_flux(ovs_ctx* c, int32_t gid, int64_t nfaces, const int64_t* faces, const int8_t* signs,
                       int32_t nsurf, const int64_t* surf_start, const ovs_fields* vel, void* flux, double* net,
                       int32_t correct) {
    if (!c) return OVS_ERR_ARG;
    if (!c->ws) return fail(c, OVS_ERR_STATE, "no workspace attached");
    if (gid < 0 || gid >= c->ngrids) return fail(c, OVS_ERR_ARG, "grid %d does not exist", gid);
    if (nfaces < 0 || (nfaces > 0 && (!faces || !flux))) return fail(c, OVS_ERR_ARG, "faces / flux");
    if (!vel || !vel->u || !vel->v || !vel->w) return fail(c, OVS_ERR_ARG, "velocity arrays");
    if (vel->dtype != OVS_F32 && vel->dtype != OVS_F64) return fail(c, OVS_ERR_ARG, "velocity dtype");
    if (vel->stride < 0) return fail(c, OVS_ERR_ARG, "velocity stride %d", vel->stride);
    if (nsurf < 0 || nsurf > kMaxFluxSurfaces) return fail(c, OVS_ERR_ARG, "nsurf = %d (0..%d)", nsurf, kMaxFluxSurfaces);
    if (nsurf > 0 && (!surf_start || !net)) return fail(c, OVS_ERR_ARG, "surf_start / net");
    if (correct && nsurf == 0) return fail(c, OVS_ERR_ARG, "a correction needs at least one closed surface");
    FluxParams P;
    memset(&P, 0, sizeof P);
    for (int s = 0; s < nsurf; ++s)
        if (surf_start[s] < 0 || surf_start[s + 1] < surf_start[s] || surf_start[s + 1] > nfaces)
            return fail(c, OVS_ERR_ARG, "surf_start must be nondecreasing within [0, nfaces]");
    for (int s = 0; nsurf > 0 && s <= nsurf; ++s) P.surf_start[s] = surf_start[s];
    // chunks of consecutive faces of one surface, each summed by one block: at least 1024 faces, and few enough
    // that every surface's chunks fit the kFluxChunks partial sums
    if (nsurf > 0) {
        const int64_t in_surf = surf_start[nsurf] - surf_start[0];
        int64_t L = std::max<int64_t>(1024, (in_surf + (kFluxChunks - nsurf) - 1) / (kFluxChunks - nsurf));
        L = (L + 255) / 256 * 256;
        if (L > INT32_MAX / 2) return fail(c, OVS_ERR_ARG, "%lld faces on the surfaces", (long long)in_surf);
        P.chunk = (int32_t)L;
        P.chunk_start[0] = 0;
        for (int s = 0; s < nsurf; ++s)
            P.chunk_start[s + 1] = P.chunk_start[s] + (int32_t)((surf_start[s + 1] - surf_start[s] + L - 1) / L);
    }
    P.part = c->d_flux_part;
    P.grid = gid;
    P.nsurf = nsurf;
    P.nfaces = nfaces;
    P.faces = faces;
    P.signs = signs;
    P.vel.f[0] = vel->u;
    P.vel.f[1] = vel->v;
    P.vel.f[2] = vel->w;
    P.vel.f[3] = vel->u;
    P.vel.stride = vel->stride > 1 ? vel->stride : 1;
    P.flux = flux;
    P.net = net;
    P.err = c->d_err;
    if (nfaces == 0 && nsurf == 0) return OVS_OK;
    OVS_CUDA(c, cudaSetDevice(c->device));
    OVS_CUDA(c, launch_flux(P, vel->dtype == OVS_F64, c->d_grids, c->nsm, correct != 0, c->stream));
    return OVS_OK;
}

int ovs_autotune_guess(ovs_ctx* c, const ovs_fringe_set* sets, int32_t nsets, const ovs_donors* out,
                       const ovs_fields* fields, int32_t nfields, const ovs_fields_out* fout, int32_t ncand,
                       const int32_t* hidden, const float* const* params, int32_t reps, float* ms, int32_t* best) {
    if (!c) return OVS_ERR_ARG;
    if (ncand < 1 || ncand > 16 || !hidden || !best) return fail(c, OVS_ERR_ARG, "ncand = %d (1..16), hidden, best", ncand);
    if (reps < 1 || reps > 1000) return fail(c, OVS_ERR_ARG, "reps = %d (1..1000)", reps);
    for (int k = 0; k < ncand; ++k) {
        if (hidden[k] != 0 && hidden[k] != 32 && hidden[k] != 64 && hidden[k] != 128)
            return fail(c, OVS_ERR_ARG, "candidate %d: hidden width %d (0, 32, 64 or 128)", k, hidden[k]);
        if (hidden[k] && !params) return fail(c, OVS_ERR_ARG, "candidate %d has a width but params is NULL", k);
    }
    if (c->opts.guess != OVS_GUESS_MLP && c->opts.guess != OVS_GUESS_MLP_ONLY)
        return fail(c, OVS_ERR_STATE, "set options.guess to OVS_GUESS_MLP (or MLP_ONLY) before tuning the guess");
    OVS_CUDA(c, cudaSetDevice(c->device));
    // candidate k's networks: params[k * ngrids + g] for grid g (NULL: grid g has none); width 0: no networks
    auto install = [&](int k) -> int {
        for (int g = 0; g < c->ngrids; ++g) {
            const float* p = hidden[k] ? params[(size_t)k * c->ngrids + g] : nullptr;
            if (p) {
                int rc = ovs_guess_set_params(c, g, hidden[k], p);
                if (rc != OVS_OK) return rc;
            } else {
                c->hidden[g] = 0;  // the assembly then starts this grid's points from hints and control cells
            }
        }
        return OVS_OK;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(c, cudaGetLastError(), "autotune events");
    }
    // one call timed alone (events around it on the context stream); cold = after the hints were reset
    auto timed_call = [&](bool cold, float* acc) -> int {
        if (cold) {
            int rc = ovs_reset_hints(c);
            if (rc != OVS_OK) return rc;
        }
        if (cudaEventRecord(e0, c->stream) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "autotune");
        int rc = assemble_impl(c, sets, nsets, out, fields, nfields, fout);
        if (rc != OVS_OK) return rc;
        cudaError_t e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e != cudaSuccess) return cuda_fail(c, e, "autotune timing");
        *acc += t;
        return OVS_OK;
    };
    int rc = OVS_OK, kbest = -1;
    float best_score = 0.f;
    for (int k = 0; k < ncand && rc == OVS_OK; ++k) {
        rc = install(k);
        float cold = 0.f, warm = 0.f, scratch = 0.f;
        if (rc == OVS_OK) rc = timed_call(true, &scratch);  // untimed: graph capture, caches
        for (int r = 0; r < reps && rc == OVS_OK; ++r) rc = timed_call(true, &cold);
        if (rc == OVS_OK) rc = timed_call(false, &scratch);  // hints now warm
        for (int r = 0; r < reps && rc == OVS_OK; ++r) rc = timed_call(false, &warm);
        if (rc != OVS_OK) break;
        cold /= (float)reps;
        warm /= (float)reps;
        if (ms) {
            ms[2 * k] = cold;
            ms[2 * k + 1] = warm;
        }
        // a time loop pays the cold call once and warm calls after it: both count
        const float score = cold + warm;
        if (kbest < 0 || score < best_score) {
            kbest = k;
            best_score = score;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == OVS_OK) rc = install(kbest);
    if (rc != OVS_OK) return rc;
    *best = kbest;
    return OVS_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------------
// ovs_assemble_noalloc: the slow-path queue of k_assemble in a fixed device array instead of the context
// workspace (see include/ovs.h for who needs this and its limits).
//
// Layout of the array: [queue counters, padded to 256 bytes][2 x OVS_NOALLOC_MAX_POINTS slow-path entries].
// In host code `ovs_noalloc_scratch` is only a host-side stand-in for the symbol; the device address comes
// from cudaGetSymbolAddress, looked up once per device with that device current.
namespace {
constexpr size_t kNoAllocHead = 256;
static_assert(kQueueCounters * sizeof(uint32_t) <= kNoAllocHead, "queue counters fit the head");
constexpr size_t kNoAllocBytes = kNoAllocHead + 2 * (size_t)OVS_NOALLOC_MAX_POINTS * sizeof(SlowEntry);
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};
}  // namespace

static __device__ __align__(256) unsigned char ovs_noalloc_scratch[kNoAllocBytes];

extern "C" int ovs_assemble_noalloc(ovs_ctx* c, const ovs_fringe_set* sets, int32_t nsets, const ovs_donors* out) {
    if (!c) return OVS_ERR_ARG;
    if (!c->ws) return fail(c, OVS_ERR_STATE, "no context workspace attached (it holds the grid table)");
    if (c->device < 0 || c->device >= kNoAllocMaxDevices) return fail(c, OVS_ERR_ARG, "device %d", c->device);
    // the same checks as ovs_assemble, with the fixed array's capacity as the point limit
    if (nsets < 0 || nsets > OVS_MAX_SETS) return fail(c, OVS_ERR_ARG, "nsets = %d (0..%d)", nsets, OVS_MAX_SETS);
    if (nsets > 0 && !sets) return fail(c, OVS_ERR_ARG, "sets is NULL");
    int64_t total = 0;
    for (int s = 0; s < nsets; ++s) {
        const ovs_fringe_set& f = sets[s];
        if (f.receiver < 0 || f.receiver >= c->ngrids)
            return fail(c, OVS_ERR_ARG, "set %d: receiver grid %d does not exist", s, f.receiver);
        if (f.n_donors < 1 || f.n_donors > OVS_MAX_DONORS)
            return fail(c, OVS_ERR_ARG, "set %d: n_donors = %d (1..%d)", s, f.n_donors, OVS_MAX_DONORS);
        for (int d = 0; d < f.n_donors; ++d)
            if (f.donors[d] < 0 || f.donors[d] >= c->ngrids)
                return fail(c, OVS_ERR_ARG, "set %d: donor grid %d does not exist", s, f.donors[d]);
        if (f.n < 0) return fail(c, OVS_ERR_ARG, "set %d: n = %lld", s, (long long)f.n);
        if (f.n > 0 && !f.node_ids) return fail(c, OVS_ERR_ARG, "set %d: node_ids is NULL", s);
        total += f.n;
    }
    if (total > OVS_NOALLOC_MAX_POINTS)
        return fail(c, OVS_ERR_WORKSPACE,
                    "ovs_assemble_noalloc: %lld points exceed its fixed capacity of %d points per call "
                    "(split the sets or use ovs_assemble with a larger workspace)",
                    (long long)total, OVS_NOALLOC_MAX_POINTS);
    if (!out) return fail(c, OVS_ERR_ARG, "donors output is NULL");
    if (out->n != total)
        return fail(c, OVS_ERR_ARG, "donors.n (%lld) must equal the number of points (%lld)", (long long)out->n,
                    (long long)total);
    if (total == 0) return OVS_OK;
    if (!out->grid || !out->cell || !out->xi || !out->status) return fail(c, OVS_ERR_ARG, "donors array is NULL");
    if (out->xi_dtype != OVS_F32 && out->xi_dtype != OVS_F64) return fail(c, OVS_ERR_ARG, "xi_dtype");
    OVS_CUDA(c, cudaSetDevice(c->device));
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[c->device]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, ovs_noalloc_scratch);
            if (e != cudaSuccess || !p) return cuda_fail(c, e, "cudaGetSymbolAddress(ovs_noalloc_scratch)");
            g_noalloc_ptr[c->device] = p;
        }
        base = g_noalloc_ptr[c->device];
    }
    // parameters in the context's pinned staging buffer (made with the context), launched directly (no graph is
    // captured on this path)
    int b = 0;
    OVS_CUDA(c, acquire_stage(c, &b));
    StepParams& S = *c->h_step[b];
    AsmParams& P = S.a;
    memset(&P, 0, offsetof(AsmParams, s));
    P.nsets = nsets;
    P.xi_f64 = out->xi_dtype == OVS_F64;
    P.max_walk = c->opts.max_walk;
    // the guess modes as in ovs_assemble (the learned guess runs inside the assembly kernel)
    const bool mlp = c->opts.guess == OVS_GUESS_MLP || c->opts.guess == OVS_GUESS_MLP_ONLY;
    P.guess = mlp ? OVS_GUESS_HINT : c->opts.guess;
    P.stats = c->opts.collect_stats;
    P.total = total;
    P.queue_cap = 2 * (int64_t)OVS_NOALLOC_MAX_POINTS;
    P.out_grid = out->grid;
    P.out_cell = out->cell;
    P.out_xi = out->xi;
    P.out_status = out->status;
    P.queue_count = (uint32_t*)base;  // the queue's counters, zeroed on the stream by launch_assemble first
    P.queue = (SlowEntry*)((char*)base + kNoAllocHead);
    P.counters = c->d_counters;
    P.err = c->d_err;
    fill_sets(sets, nsets, P.s);
    fill_xforms(c, sets, nsets, P.xf);
    memcpy(P.m, c->motion, sizeof P.m);
    const uint32_t mk = fill_guess(c, &P) ? kStepMlp : 0u;
    cudaError_t e = run_step(c, b, kStepAssemble | kStepNoAlloc | mk, (uint32_t*)base, false);
    if (e != cudaSuccess) return cuda_fail(c, e, "assemble (no-alloc) launch");
    return OVS_OK;
}
