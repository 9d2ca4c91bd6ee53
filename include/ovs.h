/*
 * ovs.h -- C ABI of libovs: per-time-step overset grid assembly (donor search)
 * and boundary interpolation on one GPU.
 *
 * The method is the moving-overset assembly of Hedayat & Borazjani,
 * "A parallel dynamic overset grid framework for immersed boundary methods"
 * (arXiv 1910.09315):
 *   - every moving grid carries a non-inertial frame: x_in = R x_body + c,
 *     frame velocity V + omega x (x_in - c)            (Sec. 2.1, eq. "velocity")
 *   - query (fringe) points of one grid get a donor hexahedron in another
 *     grid, localised by control cells and found by a walking search with a
 *     brute-force fallback                                (Sec. 2.2.5, Alg. 3)
 *   - values are interpolated trilinearly from the donor's 8 nodes
 *                                                        (Sec. 2.2.6)
 *   - velocities are carried between frames              (Sec. 2.3.1,
 *     eq. "velocity_non"), and a query point takes its donor from the first grid
 *     of a priority list that has one                    (Sec. 2.4 item 1).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - All pointers marked "device" are CUDA device pointers on the context's
 *    device; the library never allocates device memory: the caller provides
 *    workspaces (sizes from the *_workspace_size calls) and all inputs and
 *    outputs.  Host pointers are read during the call only.
 *  - Every call that launches work enqueues it on the context's stream and
 *    returns without waiting, except the set-up and control calls, which
 *    synchronise the stream: ovs_workspace_attach, ovs_create_grid (it sizes
 *    its control-cell bins), ovs_create_surface, ovs_set_iblank,
 *    ovs_set_tuning, ovs_autotune, ovs_train_guess, ovs_guess_set_params,
 *    ovs_sync, ovs_get_stats and ovs_ctx_destroy.  (A step call can also wait,
 *    on the host, for the call two calls earlier: see OVS_LAUNCH_*.)
 *  - Return value: OVS_OK (0) or a negative OVS_ERR_* code; ovs_last_error()
 *    gives a message.  No C++ exception crosses the ABI.  A context is used by
 *    one host thread at a time.
 *  - Node arrays are structure-of-arrays, i fastest: node = i + ni (j + nj k).
 *    Cell (i,j,k) has corners (i+di, j+dj, k+dk), corner a = di + 2 dj + 4 dk;
 *    on a periodic axis index n wraps to 0; cells per axis: n-1, or n if
 *    periodic; linear cell id = i + Ci (j + Cj k).
 *  - Donor rule: among all cells of a donor grid whose local coordinates of
 *    the point, from FP64 Newton inversion of the trilinear map, lie in
 *    [-1e-10, 1 + 1e-10]^3, the one with the lowest linear id.
 */
#ifndef OVS_H
#define OVS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define OVS_OK 0
#define OVS_ERR_ARG (-1)       /* invalid argument (null pointer, bad size, non-orthogonal R, ...) */
#define OVS_ERR_STATE (-2)     /* call out of order (no workspace attached, unknown grid, ...) */
#define OVS_ERR_WORKSPACE (-3) /* a workspace is too small for the request */
#define OVS_ERR_CUDA (-4)      /* a CUDA runtime call failed */
#define OVS_ERR_NO_DEVICE (-5) /* no usable CUDA device: there is no CPU fallback */
#define OVS_ERR_DEVICE (-6)    /* a kernel reported an error through the device status word */

/* ---- per-point status (ovs_donors.status) ---- */
#define OVS_STATUS_FOUND 0    /* donor found */
#define OVS_STATUS_ORPHAN 1   /* no grid of the priority list contains the point */
#define OVS_STATUS_BADINPUT 2 /* the point's coordinates are not finite */
#define OVS_STATUS_MASK 0x0F  /* the bits above are statistics, not results: */
#define OVS_STATUS_REFINED 0x20  /* decided by FP64 Newton (near a face, or FP64 precision mode) */
#define OVS_STATUS_FALLBACK 0x10 /* decided by the exhaustive control-cell search */

/* ---- dtypes ---- */
#define OVS_F32 0
#define OVS_F64 1

/* ---- limits ---- */
#define OVS_MAX_GRIDS 31
#define OVS_MAX_SETS 64
#define OVS_MAX_DONORS 8
#define OVS_MAX_CELLS ((int64_t)1 << 27) /* cells per grid: < 2^27 - 1 (donor hints pack the grid id) */

/* ---- options (ovs_set_options) ---- */
#define OVS_VEL_RELATIVE 0 /* u_in = R_d u_d + V_d + w_d x (x_in - c_d); u_r = R_r^T (u_in - V_r - w_r x (x_in - c_r)) */
#define OVS_VEL_ABSOLUTE 1 /* u_r = R_r^T R_d u_d (Sec. 2.3.1, eq. "velocity_non" with Q = R^T) */
#define OVS_VEL_NONE 2     /* no transform: u, v, w interpolated like p */

#define OVS_GUESS_HINT 0 /* start from the donor found for the same receiver node last call, else bins */
#define OVS_GUESS_BINS 1 /* always start from the control-cell bin of the point */
#define OVS_GUESS_MLP 2  /* body grids with a trained guess network: start there when no hint */
#define OVS_GUESS_MLP_ONLY 3 /* body grids with a trained guess network: always start there (hints ignored) */
/* How a call's kernels reach the GPU.  Every call first copies its parameters (sets, frame maps, motions,
 * output pointers: one block) from a double-buffered pinned staging area to the context workspace; the
 * kernels read them there, and their grids are persistent (a multiple of the SM count), so the launch
 * sequence of a call depends only on which kernels it needs.
 *   GRAPH:  that sequence is captured once per kind of call (assemble, assemble+interpolate in FP32 or FP64,
 *           the set of guess-network widths) as a CUDA graph, two instances (one per staging buffer), and every
 *           later call of the same kind is one cudaGraphLaunch on the context stream.
 *   DIRECT: the same copy and kernels launched one by one (always the case while trace events are set, and
 *           always for ovs_assemble_noalloc).
 * A call that reuses a staging buffer first waits (host) for the call that used it two calls earlier. */
#define OVS_LAUNCH_DIRECT 0
#define OVS_LAUNCH_GRAPH 1

typedef struct ovs_ctx ovs_ctx;

typedef struct {
    int32_t n[3];        /* node counts ni, nj, nk (>= 2 each) */
    int32_t periodic[3]; /* 1 if the axis wraps (its last node connects to its first) */
    const double* x;     /* device, n0*n1*n2 node coordinates in the grid's own frame (borrowed: must */
    const double* y;     /*   stay valid and unchanged until ovs_ctx_destroy) */
    const double* z;
    int32_t role;        /* 0 background (inertial frame), 1 body (moving frame) */
} ovs_grid_desc;

typedef struct {
    int32_t receiver;                     /* receiver grid id */
    int32_t n_donors;                     /* 1..OVS_MAX_DONORS */
    int32_t donors[OVS_MAX_DONORS];       /* donor grid ids, priority order (Sec. 2.4 item 1) */
    int64_t n;                            /* number of query points (0 allowed) */
    const int32_t* node_ids;              /* device, n receiver node ids */
} ovs_fringe_set;

typedef struct {
    int64_t n;       /* capacity in points: >= sum of the sets' n (points are laid out set after set) */
    int32_t* grid;   /* device [n]: donor grid id, -1 if none */
    int32_t* cell;   /* device [n]: donor linear cell id, -1 if none */
    void* xi;        /* device [3n] SoA: xi[0..n) eta[n..2n) zeta[2n..3n); float or double; NaN if none */
    int32_t xi_dtype;/* OVS_F32 (FP32 Newton, FP64 only near faces) or OVS_F64 (FP64 for every point) */
    uint8_t* status; /* device [n]: OVS_STATUS_* */
} ovs_donors;

typedef struct {
    const void* u;   /* device, one value per node of the grid; NULL for a grid never used as donor */
    const void* v;
    const void* w;
    const void* p;
    int32_t dtype;   /* OVS_F32 or OVS_F64 */
    int32_t stride;  /* elements from one node's value to the next node's, the same for u, v, w and p: 0 or 1 =
                        four contiguous arrays; 4 with v = u + 1, w = u + 2, p = u + 3 and u 16-byte aligned =
                        one array of (u, v, w, p) records per node (the layout of a 4-dof structured-grid vector),
                        read one record per corner; any other value >= 1: strided arrays.  Negative: OVS_ERR_ARG */
} ovs_fields;

typedef struct {
    void* u;         /* device [n] per point, in the receiver grid's frame */
    void* v;
    void* w;
    void* p;
    int32_t dtype;   /* must equal the donor fields' dtype */
} ovs_fields_out;

typedef struct {
    int32_t velocity_mode; /* OVS_VEL_* (default RELATIVE) */
    int32_t guess;         /* OVS_GUESS_* (default HINT) */
    int32_t max_walk;      /* walk steps before the exhaustive fallback (default 48, 1..1024) */
    int32_t collect_stats; /* 1: count walk steps / slow-path points (small atomic cost) */
    int32_t launch;        /* OVS_LAUNCH_* (default GRAPH) */
} ovs_options;

typedef struct {
    int64_t points;      /* points assembled since the last reset */
    int64_t walk_steps;  /* cells visited by the FP32 walk */
    int64_t refined;     /* points decided by FP64 Newton */
    int64_t fallback;    /* points decided by the exhaustive control-cell search */
    int64_t guess_used;  /* points started from a guess network */
    int64_t newton_iterations; /* FP32 Newton iterations of the walk */
    int64_t warp_walk_steps;   /* sum over the warps' 32-point work items of the most walk steps of one of them
                                  (walk_steps / (32 warp_walk_steps) = the share of lanes busy while a warp walks) */
    int64_t near_face;   /* points handed to the near-face decision among a cell's neighbours */
    int64_t stuck;       /* points handed to the exhaustive control-cell search (walk stuck or outside) */
} ovs_stats;

/* Create a context on CUDA device `device`, enqueuing on `cuda_stream` (a cudaStream_t; NULL = legacy
 * default stream).  Returns OVS_ERR_NO_DEVICE when no CUDA device is usable. */
int ovs_ctx_create(ovs_ctx** out, int device, void* cuda_stream);
/* Destroy a context (waits for its stream).  Borrowed memory is not freed. */
int ovs_ctx_destroy(ovs_ctx* ctx);
/* Message of the last error on this context (never NULL). */
const char* ovs_last_error(const ovs_ctx* ctx);
/* Change the stream later calls enqueue on. */
int ovs_set_stream(ovs_ctx* ctx, void* cuda_stream);

/* Bytes of the context workspace needed for calls of up to `max_points` query points (slow-path
 * queue of two entries per point, counters, status word, step parameters, and 64 KiB of partial sums for
 * ovs_interface_flux). */
int ovs_workspace_size(const ovs_ctx* ctx, int64_t max_points, size_t* bytes);
/* Attach a caller-owned device workspace (256-byte aligned) of at least ovs_workspace_size bytes. */
int ovs_workspace_attach(ovs_ctx* ctx, void* dptr, size_t bytes, int64_t max_points);

/* Bytes of the per-grid workspace for a grid of these dimensions: cell records (128 B per cell),
 * control-cell bins, the finer bins of crowded control cells (about 2 MiB plus up to 8 B per cell, at most
 * 32 MiB), the node coordinates as FP32 pairs and the per-node donor hints. */
int ovs_grid_workspace_size(const ovs_grid_desc* desc, size_t* bytes);
/* Register a structured curvilinear grid (Sec. 2.2: one block of the composite grid).  Builds, in the
 * caller's workspace, per-cell records and the control cells of Sec. 2.2.5 (uniform axis-aligned bins over
 * the grid's bounding box, each cell registered in every bin its bounding box overlaps).  Synchronises the
 * stream.  Grid ids are 0, 1, 2, ... in creation order.  Motion starts as the identity. */
int ovs_create_grid(ovs_ctx* ctx, const ovs_grid_desc* desc, void* dworkspace, size_t bytes, int32_t* grid_id);

/* Cells that overlap one another.  The fast path takes a point's donor from the walk as soon as the point lies
 * clear (by more than the FP32 error bound) of every face of a cell, and near a face it tests only the cells
 * sharing that face: this is the lowest-id rule only if no other cell of the grid holds the point, i.e. if the
 * grid's cells do not overlap.  ovs_create_grid classifies every cell by the Jacobian determinants of its
 * trilinear map at its 8 corners (FP64): all positive, all negative, or mixed / zero (folded or degenerate); a
 * grid with folded cells or with cells of both signs may overlap itself and is searched exhaustively: every
 * point the walk finds in it goes to the lowest-id search of its control cell (slower, same rule).
 * ovs_grid_check: the three counts (cells[3]: positive, negative, folded) and whether the grid is searched
 * exhaustively (*overlap; either pointer may be NULL).  ovs_set_grid_overlap: the caller's statement for grids
 * that overlap without folding (e.g. a periodic seam whose end cells overlap, a C-grid wake cut): 1 = search
 * exhaustively, 0 = the cells do not overlap (refused, OVS_ERR_ARG, for a grid with folded cells).
 * Synchronises the stream.  Errors: OVS_ERR_ARG (unknown grid, flag not 0 or 1). */
int ovs_grid_check(const ovs_ctx* ctx, int32_t grid_id, int64_t cells[3], int32_t* overlap);
int ovs_set_grid_overlap(ovs_ctx* ctx, int32_t grid_id, int32_t overlap);
/* The control cells of a grid (Sec. 2.2.5: the uniform axis-aligned bins that start the walk and bound the
 * exhaustive search; each cell is listed in every bin its padded box overlaps), as built by ovs_create_grid:
 * out[0] bins, out[1] registrations in their lists, out[2] crowded control cells (lists of more than 256 cells,
 * as around a thin or clustered region; the threshold doubles until at most 4096 of them, and their finer lists,
 * fit the grid workspace) that were split into 4 x 4 x 4 finer bins, out[3] registrations in those finer bins.  The exhaustive search of a point in a split control cell reads only its finer bin's list, which
 * holds every cell whose padded box reaches the point (the same rule one level down), so results do not depend
 * on the split.  Host only.  Errors: OVS_ERR_ARG (unknown grid, out NULL). */
int ovs_grid_bins(const ovs_ctx* ctx, int32_t grid_id, int64_t out[4]);

/* Set a grid's rigid frame (Sec. 2.1, Fig. "non-inertial"): R (row-major 3x3, body -> inertial, must be
 * orthogonal with det +1 to 1e-12), origin c, translational velocity V and angular velocity omega (inertial
 * components).  Host arrays; takes effect for later calls. */
int ovs_set_motion(ovs_ctx* ctx, int32_t grid_id, const double R[9], const double c[3], const double V[3],
                   const double omega[3]);

/* Hole cutting (Sec. 2.2.1): a closed triangulated body surface, fixed in the frame of body_grid (it moves with
 * that grid's motion), and the blanking of another grid's nodes inside it.
 * v: host FP64 [nv x 3] vertex coordinates (row-major, body frame); tri: host int32 [nt x 3] vertex ids; the
 * surface must be closed (every edge shared by two triangles) for "inside" to be meaningful.
 * ovs_surface_workspace_size: bytes of the device workspace the surface needs (its vertices, triangles and a
 * grid of bins over its projection along its shortest box axis). */
int ovs_surface_workspace_size(int64_t nv, const double* v, int64_t nt, const int32_t* tri, size_t* bytes);
/* Copies the surface into the caller's workspace dws (256-byte aligned, at least the size above; borrowed until
 * ovs_ctx_destroy) and returns its id (0, 1, ... in creation order, at most OVS_MAX_GRIDS).  Synchronises the
 * stream.  Errors: OVS_ERR_ARG (bad grid id, vertex id out of range, empty surface), OVS_ERR_WORKSPACE. */
int ovs_create_surface(ovs_ctx* ctx, int32_t body_grid, int64_t nv, const double* v, int64_t nt, const int32_t* tri,
                       void* dws, size_t bytes, int32_t* surface_id);
/* For each node in nodes (device int32 [n], ids of target_grid's nodes; NULL: nodes 0 .. n-1), sets
 * iblank[node] = 0 (device uint8 [target_grid's node count]) if the node lies inside the surface at the
 * frames' current motions; other entries are left as they are (start from all ones; several surfaces can cut
 * the same mask in turn).  Inside = an odd number of crossings of a ray along the surface's shortest box axis r
 * of the body frame (the first on a tie; u, w = the next axes cyclically): the point's (u, w) in a triangle's
 * projection, with a point on a projected edge owned by the one triangle whose counter-clockwise edge runs
 * toward -w (or level toward -u), and the crossing strictly ahead along r; FP64, one rounding per operation
 * (the node carried to the body frame in FP32 pairs, about 1e-14 relative; FP32 decides wherever its error
 * bound proves the FP64 answer).  Enqueued on the context stream; bad node ids are reported by ovs_sync.
 * Errors: OVS_ERR_ARG (unknown surface or grid, n < 0, n above the node count with nodes NULL, iblank NULL). */
int ovs_hole_cut(ovs_ctx* ctx, int32_t surface_id, int32_t target_grid, int64_t n, const int32_t* nodes,
                 uint8_t* iblank);
/* Several surfaces cutting one target grid in one launch, the same result as ovs_hole_cut for each in turn:
 * surface_ids, n: host arrays [nsurf] (0 <= nsurf <= OVS_MAX_GRIDS); nodes: host array [nsurf] of device int32
 * node-id arrays (an entry NULL, or nodes NULL: nodes 0 .. n[s]-1).  The candidates of all surfaces are spread
 * over the whole GPU together, which balances surfaces whose inside points cluster.  Errors as ovs_hole_cut. */
int ovs_hole_cut_many(ovs_ctx* ctx, int32_t nsurf, const int32_t* surface_ids, int32_t target_grid,
                      const int64_t* n, const int32_t* const* nodes, uint8_t* iblank);

/* Blanked nodes of a grid (Sec. 2.4: blanked donors are rejected).  iblank: device uint8 [its node count], 0 =
 * blanked (a hole point: never a donor node), nonzero = active; NULL: every node active (the state after
 * ovs_create_grid).  From then on a cell with a blanked corner node never donates: a point is given the
 * lowest-id cell holding it that has no blanked corner, else the next grid of its priority list, else it is
 * an orphan.  The mask is read on the context stream by this call (it marks the grid's cell records); a later
 * change to it needs another call.  Errors: OVS_ERR_ARG (unknown grid). */
int ovs_set_iblank(ovs_ctx* ctx, int32_t grid_id, const uint8_t* iblank);

int ovs_set_options(ovs_ctx* ctx, const ovs_options* opts);
int ovs_get_options(const ovs_ctx* ctx, ovs_options* opts);

/* Donor search for every query point of `sets` (Sec. 2.2.5): frame map receiver -> inertial -> donor
 * frame, localisation (hint / control cell / guess network), FP32 walk + Newton inversion of the trilinear
 * map, FP64 decision near cell faces and lowest-id rule, exhaustive control-cell fallback.  Writes the
 * donors of sets[0] first, then sets[1], ...  Updates the per-node hints of the receiver grids. */
int ovs_assemble(ovs_ctx* ctx, const ovs_fringe_set* sets, int32_t nsets, const ovs_donors* out);

/* ovs_assemble followed by ovs_interpolate for the same sets, fields and motions, in one call (one time step
 * of the method: donors, then the interpolated boundary values).  Writes the same donors and field values as
 * the two calls (`out` as in ovs_assemble, `fields`/`fout` as in ovs_interpolate), in one pass per point: the
 * assembly kernels interpolate each point from the local coordinates as stored in `out` as soon as its donor is
 * decided. */
int ovs_assemble_interpolate(ovs_ctx* ctx, const ovs_fringe_set* sets, int32_t nsets, const ovs_donors* out,
                             const ovs_fields* fields, int32_t nfields, const ovs_fields_out* fout);

/* Trilinear interpolation (Sec. 2.2.6) of u, v, w, p from the donors found by ovs_assemble for the same
 * sets, followed by the velocity transform of the options (Sec. 2.1 / Sec. 2.3.1), using the motions set
 * now.  `fields` is indexed by grid id (nfields = number of grids).  Points without a donor get 0. */
int ovs_interpolate(ovs_ctx* ctx, const ovs_fringe_set* sets, int32_t nsets, const ovs_donors* in,
                    const ovs_fields* fields, int32_t nfields, const ovs_fields_out* out);

/* ---- learned initial guess (not in the paper: the paper starts its walk from a control cell) ----
 * Each body grid can carry a small network 3 -> H -> H -> 3 (SiLU) that maps normalised body-frame coordinates
 * xn = (x - centre) * 2 / extent (centre and extent of the grid's bounding box) to normalised curvilinear
 * coordinates ((i + xi)/Ci, (j + eta)/Cj, (k + zeta)/Ck).  With options.guess = OVS_GUESS_MLP, points without a
 * usable hint start their walk at the cell the network points at (evaluated with FP16 operands on tensor cores,
 * FP32 accumulation); the exact in-cell test is unchanged, so donors do not depend on the network.
 * Parameters (FP32): W1 [H x 3] row-major, b1 [H], W2 [H x H] row-major (W2[out][in]), b2 [H], W3 [3 x H],
 * b3 [3]: H*H + 8*H + 3 values.  H is 32, 64 or 128. */
typedef struct {
    int32_t hidden;            /* H */
    int32_t epochs;            /* passes over the samples */
    int32_t batch;             /* samples per Adam step (beta 0.9 / 0.999, eps 1e-8) */
    float lr;                  /* Adam learning rate at the first step */
    float lr_final;            /* learning rate at the last step (cosine decay between them); 0: constant lr */
    int32_t pad;
    int64_t n_samples;
    const int32_t* cells;      /* device [n_samples]: cell of each sample (the caller draws them) */
    const float* xi;           /* device [3 n_samples] SoA: local coordinates in [0,1]^3 of each sample */
    const float* init_params;  /* device: initial parameters (the caller draws them) */
    void* scratch;             /* device scratch of ovs_train_workspace_size bytes (inputs and targets) */
    size_t scratch_bytes;
} ovs_train_desc;

int ovs_guess_param_count(int32_t hidden, int64_t* count);
int ovs_train_workspace_size(const ovs_train_desc* desc, size_t* bytes);
/* Train grid_id's network on samples of the grid itself: input = the trilinear map of (cell, xi), target = the
 * sample's normalised curvilinear coordinates; mean squared error, Adam.  Synchronises the stream; writes the
 * mean loss of the last epoch to *final_loss (may be NULL). */
int ovs_train_guess(ovs_ctx* ctx, int32_t grid_id, const ovs_train_desc* desc, float* final_loss);
/* Checkpoint / restore of a grid's network (device FP32 parameters in the layout above). */
int ovs_guess_get_params(ovs_ctx* ctx, int32_t grid_id, float* dparams, int32_t* hidden);
int ovs_guess_set_params(ovs_ctx* ctx, int32_t grid_id, int32_t hidden, const float* dparams);
/* Evaluate grid_id's network (the FP16 tensor-core path) on n normalised inputs xn (device, 3n SoA) -> out (3n). */
int ovs_guess_eval(ovs_ctx* ctx, int32_t grid_id, int64_t n, const float* xn, float* out);
/* Mean squared error and its gradient (FP32, the training kernel) for parameters `params` on n samples with
 * normalised inputs xn and targets (device, 3n SoA each): grads (device, param count) and *loss (device). */
int ovs_mlp_loss_grad(ovs_ctx* ctx, int32_t hidden, int64_t n, const float* xn, const float* target,
                      const float* params, float* grads, float* loss);

/* Wait for the stream; returns OVS_ERR_DEVICE (and clears it) if a kernel flagged an error. */
int ovs_sync(ovs_ctx* ctx);
/* Read (synchronously) and optionally reset the statistics counters. */
int ovs_get_stats(ovs_ctx* ctx, ovs_stats* out, int reset);

/* The interpolation as a sparse matrix (Sec. 2.2.6: the boundary interpolation assembled as a matrix whose rows
 * are the receiver points and whose columns are donor nodes, applied inside an implicit solve).  From the donors
 * `in` of a call (as ovs_assemble wrote them): one row per point; a point FOUND in a donor grid has 8 entries,
 * every other row none.  Entry a of a row (a = 0..7; bits 0 / 1 / 2 of a: the corner at +1 along i / j / k of
 * the donor cell): column = node_offset(donor grid) + that corner's node id, value = its trilinear weight from
 * the stored xi (the weights ovs_interpolate uses).  node_offset(g) = the sum of the node counts of grids
 * 0 .. g-1 in creation order, so the x of ovs_spmv holds every grid's node values back to back.
 * row_ptr: device int32 [in->n + 1] (row_ptr[in->n] = the number of entries); col: device int64 and val: device
 * FP32 or FP64 (val_dtype, OVS_F32 / OVS_F64), each with room for 8 * in->n entries.  Uses the context
 * workspace as scratch (in->n <= its max_points, else OVS_ERR_WORKSPACE).  Enqueued on the context stream; a
 * donor record that names no cell of its grid is reported by ovs_sync (its entries: columns -1, values 0). */
int ovs_interp_matrix(ovs_ctx* ctx, const ovs_donors* in, int32_t* row_ptr, int64_t* col, void* val,
                      int32_t val_dtype);
/* y = A x for a matrix of ovs_interp_matrix (nrows = its number of rows): y[r] = the sum of the row's entries'
 * val * x[col] in entry order (entries with column -1 skipped).  val, x and y share dtype (OVS_F32 / OVS_F64);
 * device pointers; x in the global node numbering above.  Enqueued on the context stream. */
int ovs_spmv(ovs_ctx* ctx, int64_t nrows, const int32_t* row_ptr, const int64_t* col, const void* val, const void* x,
             void* y, int32_t dtype);

/* Forget all per-node donor hints (next assemble starts cold). */
int ovs_reset_hints(ovs_ctx* ctx);

/* Checkpoint / resume of what a time loop carries from one step to the next (no counterpart in the paper):
 * the previous donor of every node of a receiver grid, which the next assembly starts its walk from.
 * dst / src: device uint32 [the grid's node count], one entry per node: (donor grid id << 27) | donor cell id,
 * or 0xFFFFFFFF for none.  Copied on the context stream (the caller synchronises before reading dst or
 * reusing src).  ovs_set_donors accepts any values: an entry that names no cell of its donor grid is ignored
 * (that node's search starts cold), so a checkpoint can never change a result, only how fast it is found.
 * With the guess networks (ovs_guess_get_params / ovs_guess_set_params) this is the whole state: a resumed
 * run gives the donors of an uninterrupted one, bit for bit.  Errors: OVS_ERR_ARG (unknown grid, NULL). */
int ovs_get_donors(ovs_ctx* ctx, int32_t grid_id, uint32_t* dst);
int ovs_set_donors(ovs_ctx* ctx, int32_t grid_id, const uint32_t* src);

/* Launch shapes of the persistent kernels: blocks per SM of each grid (a kernel's grid is this many blocks
 * times the SM count, whatever the call's size).  0 = the default: assembly 3 (its launch bound), interpolation
 * the occupancy calculator's figure, slow path 1. */
typedef struct {
    int32_t assemble_blocks_per_sm; /* k_assemble, 256 threads a block: 1..12 */
    int32_t interp_blocks_per_sm;   /* k_interp, 256 threads a block: 1..32 */
    int32_t slow_blocks_per_sm;     /* the slow-path kernels (near-face decisions and exhaustive searches side
                                       by side, then the searches the decisions hand on), 256 threads a block:
                                       1..8 */
    int32_t guess_blocks_per_sm;    /* 0..32, accepted and kept but without effect: the learned guess runs inside
                                       the assembly kernel, in its launch shape */
    int32_t launch;                 /* OVS_LAUNCH_GRAPH or OVS_LAUNCH_DIRECT (the option of ovs_set_options);
                                       0 in ovs_set_tuning: leave the launch mode as it is */
} ovs_tuning;

/* Set (NULL or all zero: defaults) / read the launch shapes.  Drops the context's captured graphs. */
int ovs_set_tuning(ovs_ctx* ctx, const ovs_tuning* t);
int ovs_get_tuning(const ovs_ctx* ctx, ovs_tuning* t);
/* Autotuner: times the call ovs_assemble_interpolate(sets, nsets, out, fields, nfields, fout) (fout may be NULL:
 * ovs_assemble) under candidate launch shapes, one knob at a time (each knob over a few values around its
 * default, the others held), `reps` timed calls per candidate after one untimed call, with CUDA events on the
 * context stream; keeps the fastest; then times the chosen shapes as one CUDA graph per call and as direct
 * launches and keeps the faster launch mode (it becomes the launch option); writes the result to *best (may
 * be NULL).  The calls run for real: their outputs and the donor hints are those of the last one.
 * Synchronises the stream. */
int ovs_autotune(ovs_ctx* ctx, const ovs_fringe_set* sets, int32_t nsets, const ovs_donors* out,
                 const ovs_fields* fields, int32_t nfields, const ovs_fields_out* fout, int32_t reps,
                 ovs_tuning* best);

/* Fluxes at the receivers and mass conservation over closed interfaces (Sec. 2.1 eq. "flux": the contravariant
 * flux U^r = u_q xi^r_q / J through a face of constant xi^r; Sec. 2.3.1: fluxes of the recipient faces from the
 * interpolated, frame-transformed velocities; Sec. 2.4 "Mass conservation": the fluxes through a closed interface
 * must sum to zero, so their imbalance is removed by a correction).
 *   Face id = 3 * (node id of its base corner) + d: the face of constant index along axis d spanned by the axes
 *   a = d+1 and b = d+2 (mod 3); corners base, base + e_a, base + e_a + e_b, base + e_b (wrapped on periodic
 *   axes).  Its area vector S = (corner 2 - corner 0) x (corner 3 - corner 1) / 2 (in the precision stated at the
 *   end; it points toward increasing index d on a right-handed grid); the velocity on it is the mean of its
 *   corners' values; its flux U = u . S, in the grid's own frame.
 * faces: device int64 [nfaces]; signs: device int8 [nfaces], +1 where S points out of the region a surface encloses,
 * -1 where it points in (NULL: all +1); vel: the grid's node velocities u, v, w (p unused; FP32 or FP64, stride as
 * in ovs_fields; for a receiver grid, its fringe nodes hold the interpolated values); flux: device [nfaces] of vel's
 * dtype, the faces' fluxes U (not multiplied by the sign).  Closed surfaces: surface s is faces surf_start[s] ..
 * surf_start[s+1]-1 (host int64 [nsurf + 1], nondecreasing, within [0, nfaces]; faces outside every surface only
 * get their flux), at most 64; net: device FP64 [2 nsurf]: the net outward flux sum(sign U) before any correction
 * and the total area sum |S|, summed in a fixed order that depends only on nfaces, nsurf and surf_start
 * (reproducible: blocks sum chunks of consecutive faces, then one block per surface sums its chunks).
 * correct = 1: each face of surface s then gets U - sign * net * |S| / area (the imbalance taken out in
 * proportion to face area), after which the surface's net flux is zero.  Enqueued on the context stream; a face id that leaves the grid is reported by ovs_sync (its
 * flux 0).  The face areas are formed in FP64 from the grid's coordinates for FP64 velocities and in FP32 from
 * their FP32 pairs for FP32 velocities.  Errors: OVS_ERR_ARG (unknown grid, NULL arrays, bad surf_start, correct
 * without surfaces). */
int ovs_interface_flux(ovs_ctx* ctx, int32_t grid_id, int64_t nfaces, const int64_t* faces, const int8_t* signs,
                       int32_t nsurf, const int64_t* surf_start, const ovs_fields* vel, void* flux, double* net,
                       int32_t correct);

/* Autotuner of the learned guess (its network width, or none): ncand candidates, candidate k = networks of width
 * hidden[k] (32, 64 or 128; 0 = no networks, the plain start from hints and control cells), with the device FP32
 * parameters (layout of ovs_guess_set_params) of grid g at params[k * ngrids + g] (NULL: grid g gets no network;
 * params may be NULL when every width is 0).  For each candidate it installs the networks and times `reps` calls
 * of ovs_assemble_interpolate(sets, ..., fout) (fout NULL: ovs_assemble) started cold (donor hints reset before
 * each) and `reps` started warm (after a call of the same sets), with CUDA events on the context stream, after one
 * untimed call of each kind.  The score of a candidate is its mean cold plus its mean warm call time (a time loop
 * pays both: the first step, and every step after it); the candidate with the lowest score stays installed and its
 * index is written to *best; ms (may be NULL): [ncand][2] mean cold and warm milliseconds per call.  Requires
 * options.guess = OVS_GUESS_MLP or OVS_GUESS_MLP_ONLY (else OVS_ERR_STATE).  The calls run for real (outputs and
 * hints are those of the last one).  Synchronises the stream. */
int ovs_autotune_guess(ovs_ctx* ctx, const ovs_fringe_set* sets, int32_t nsets, const ovs_donors* out,
                       const ovs_fields* fields, int32_t nfields, const ovs_fields_out* fout, int32_t ncand,
                       const int32_t* hidden, const float* const* params, int32_t reps, float* ms, int32_t* best);

/* Tracing: record caller-created CUDA events (cudaEvent_t, NULL to skip one) on the context's stream at
 * fixed points of later calls: ev[0] before the fast assembly kernel, ev[1] after it, ev[2] after the
 * slow-path kernels (end of ovs_assemble), ev[3] before the interpolation kernel, ev[4] after it; ev[5] and ev[6]
 * are not recorded (the learned guess runs inside the fast assembly kernel, between ev[0] and ev[1]).  In
 * ovs_assemble_interpolate the two assembly kernels interpolate each point as they decide its donor (there is
 * no interpolation kernel): ev[3] and ev[4] are then both recorded after the slow-path kernel.
 * n = 0 (or ev = NULL) switches tracing off.  The events must outlive their use. */
int ovs_set_trace_events(ovs_ctx* ctx, void* const* ev, int32_t n);

/* Assembly for callers that cannot allocate device memory when they call it.
 *
 * The paper has no counterpart: this is a property of the library, not of the method.  ovs_assemble needs
 * a context workspace sized for the largest call (ovs_workspace_size(max_points)), so a caller whose
 * point count grows must allocate a larger one.  Some callers cannot: solver plug-ins whose host
 * application owns all device memory and hands them none, and time loops that must not take the implicit
 * device synchronisation of cudaMalloc/cudaFree in the middle of a step.  This entry point computes what
 * ovs_assemble computes (the same donors, hints, statistics and guess modes) but keeps its only per-call
 * scratch (the slow-path queue of points decided near a face or by the exhaustive search) in a fixed array
 * inside the library instead of the context workspace.  It differs from ovs_assemble in how it launches:
 * always as direct kernel launches, never as a captured CUDA graph (the launch option is ignored).
 *
 *  - Limit: at most OVS_NOALLOC_MAX_POINTS points per call (sum over the sets); larger calls return
 *    OVS_ERR_WORKSPACE without launching anything.  The array is 48 MiB of device memory
 *    (two slow-path entries of 24 bytes per point: OVS_NOALLOC_MAX_POINTS x 48 bytes + 256), held by every
 *    GPU on which the library's kernels are loaded until the process exits.
 *  - Allocates nothing: no cudaMalloc/cudaFree and no allocating library routine, host or device.  It
 *    still needs a context with a workspace attached and grids created (set-up time objects): the grid
 *    table, the device status word and the statistics counters live there.
 *  - The first call on each device looks up the array's device address (cudaGetSymbolAddress) with that
 *    device current; make that first call before any stream capture begins.
 *  - Every call on a device shares the one array and resets its queue counter: calls whose kernels
 *    overlap on the GPU (other streams, other contexts, other threads) race and corrupt each other's
 *    results.  Order them on one stream or synchronise between them.
 *  - Errors and outputs as ovs_assemble. */
#define OVS_NOALLOC_MAX_POINTS (1 << 20)
int ovs_assemble_noalloc(ovs_ctx* ctx, const ovs_fringe_set* sets, int32_t nsets, const ovs_donors* out);

#ifdef __cplusplus
}
#endif
#endif /* OVS_H */
