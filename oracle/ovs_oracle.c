/*
 * ovs_oracle.c -- plain FP64 CPU oracle for overset donor search.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline
 * leg do.  It shares no code, header, table or constant generator with the
 * CUDA library.
 *
 * What it computes (a plain definition, written for a reader to check by eye):
 *
 *  * Cells (Sec. 2.2.5, Fig. "control-cell"): the donor grid's node-based
 *    hexahedra.  Cell (i,j,k) has the 8 corner nodes (i+di, j+dj, k+dk),
 *    di,dj,dk in {0,1}; corner a = di + 2 dj + 4 dk.  On a periodic axis the
 *    index n wraps to 0.  Cell counts per axis: n-1, or n if periodic.  The
 *    linear cell id is i + Ci (j + Cj k).
 *  * Trilinear map and weights (Sec. 2.2.6, eq. "trilinear interpolation",
 *    with the factors (a-1) read as (1-a)): N_a(xi) = prod over the three axes
 *    of (1-xi) when the corner's offset on that axis is 0, xi when it is 1.
 *  * In-cell predicate: Newton's method on F(xi) = sum_a N_a(xi) X_a - p,
 *    started at xi = (1/2,1/2,1/2), each step solving J delta = -F by Gaussian
 *    elimination with partial pivoting.  F and J are formed from corner
 *    offsets X_a - X_0 and p - X_0 (the same function, since sum_a N_a = 1,
 *    without the cancellation error of absolute coordinates).  Converged when
 *    max|delta| <= 1e-13, within 50 steps.  The cell contains p iff Newton
 *    converged and every component of xi lies in [-1e-10, 1 + 1e-10].
 *  * Control cells (Sec. 2.2.5): uniform axis-aligned bins over the grid's
 *    node bounding box.  A cell is registered in every bin that its corner
 *    bounding box, inflated by 1e-9 times the cell diagonal, overlaps (the
 *    trilinear image of the xi window lies inside that box).
 *  * Selection: among the cells registered in p's bin, visited in ascending
 *    linear id, the first that contains p (= the lowest id) is the donor.
 *    A brute-force variant visits every cell of the grid instead.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OG_WIN_LO (-1e-10)
#define OG_WIN_HI (1.0 + 1e-10)
#define OG_NEWTON_TOL 1e-13
#define OG_NEWTON_MAXIT 50
#define OG_INFLATE 1e-9

typedef struct {
    int32_t n[3];   /* node counts */
    int32_t per[3]; /* 1 if the axis is periodic */
    const double* x;
    const double* y;
    const double* z;
    const uint8_t* iblank; /* per node, 0 = blanked (a hole point, never a donor node); NULL: every node active */
} og_grid;

typedef struct {
    int32_t nb[3];   /* bins per axis */
    double lo[3];    /* bounding box low corner */
    double hi[3];    /* bounding box high corner */
    double w[3];     /* bin widths */
    int64_t* start;  /* nb0*nb1*nb2 + 1 offsets */
    int32_t* cells;  /* registered cell ids, ascending within a bin */
    int64_t nreg;
} og_bins;

static int64_t og_cells_axis(const og_grid* g, int d) { return g->per[d] ? g->n[d] : g->n[d] - 1; }

int64_t og_num_cells(const og_grid* g) { return og_cells_axis(g, 0) * og_cells_axis(g, 1) * og_cells_axis(g, 2); }

int og_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* threads of the calling thread's later parallel loops (n <= 0: one per processor); timing only */
void og_set_num_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
#else
    (void)n;
#endif
}

/* Node ids of the 8 corners of a cell, corner a = di + 2dj + 4dk. */
void og_cell_nodes(const og_grid* g, int64_t cell, int64_t nodes[8]) {
    int64_t ci = og_cells_axis(g, 0), cj = og_cells_axis(g, 1);
    int64_t i = cell % ci, j = (cell / ci) % cj, k = cell / (ci * cj);
    for (int a = 0; a < 8; ++a) {
        int64_t ii = i + (a & 1), jj = j + ((a >> 1) & 1), kk = k + ((a >> 2) & 1);
        if (ii == g->n[0]) ii = 0; /* only reachable on a periodic axis */
        if (jj == g->n[1]) jj = 0;
        if (kk == g->n[2]) kk = 0;
        nodes[a] = ii + (int64_t)g->n[0] * (jj + (int64_t)g->n[1] * kk);
    }
}

static void og_cell_corners(const og_grid* g, int64_t cell, double X[8][3]) {
    int64_t nodes[8];
    og_cell_nodes(g, cell, nodes);
    for (int a = 0; a < 8; ++a) {
        X[a][0] = g->x[nodes[a]];
        X[a][1] = g->y[nodes[a]];
        X[a][2] = g->z[nodes[a]];
    }
}

/* Trilinear shape functions N_a(xi). */
void og_shape(const double xi[3], double N[8]) {
    for (int a = 0; a < 8; ++a) {
        double f0 = (a & 1) ? xi[0] : 1.0 - xi[0];
        double f1 = (a & 2) ? xi[1] : 1.0 - xi[1];
        double f2 = (a & 4) ? xi[2] : 1.0 - xi[2];
        N[a] = f0 * f1 * f2;
    }
}

/* dN_a/dxi_m. */
static void og_shape_grad(const double xi[3], double dN[8][3]) {
    for (int a = 0; a < 8; ++a) {
        double f[3], df[3];
        for (int m = 0; m < 3; ++m) {
            int on = (a >> m) & 1;
            f[m] = on ? xi[m] : 1.0 - xi[m];
            df[m] = on ? 1.0 : -1.0;
        }
        dN[a][0] = df[0] * f[1] * f[2];
        dN[a][1] = f[0] * df[1] * f[2];
        dN[a][2] = f[0] * f[1] * df[2];
    }
}

/* Solve A x = b (3x3) by Gaussian elimination with partial pivoting. Returns 0 if singular. */
static int og_solve3(double A[3][3], double b[3], double x[3]) {
    for (int col = 0; col < 3; ++col) {
        int piv = col;
        for (int r = col + 1; r < 3; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (!(fabs(A[piv][col]) > 0.0)) return 0;
        if (piv != col) {
            for (int c = 0; c < 3; ++c) {
                double t = A[col][c];
                A[col][c] = A[piv][c];
                A[piv][c] = t;
            }
            double t = b[col];
            b[col] = b[piv];
            b[piv] = t;
        }
        for (int r = col + 1; r < 3; ++r) {
            double f = A[r][col] / A[col][col];
            for (int c = col; c < 3; ++c) A[r][c] -= f * A[col][c];
            b[r] -= f * b[col];
        }
    }
    for (int r = 2; r >= 0; --r) {
        double s = b[r];
        for (int c = r + 1; c < 3; ++c) s -= A[r][c] * x[c];
        x[r] = s / A[r][r];
    }
    return isfinite(x[0]) && isfinite(x[1]) && isfinite(x[2]);
}

/* Newton inversion of the trilinear map of one hexahedron.  Returns 1 if converged; xi holds the
 * last iterate either way; *iters the number of Newton steps taken. */
int og_newton(const double X[8][3], const double p[3], double xi[3], int* iters) {
    double E[8][3], b[3];
    for (int a = 0; a < 8; ++a)
        for (int c = 0; c < 3; ++c) E[a][c] = X[a][c] - X[0][c];
    for (int c = 0; c < 3; ++c) b[c] = p[c] - X[0][c];
    xi[0] = xi[1] = xi[2] = 0.5;
    for (int it = 0; it < OG_NEWTON_MAXIT; ++it) {
        double N[8], dN[8][3], F[3] = {0, 0, 0}, J[3][3] = {{0}}, negF[3], d[3];
        og_shape(xi, N);
        og_shape_grad(xi, dN);
        for (int a = 0; a < 8; ++a)
            for (int c = 0; c < 3; ++c) {
                F[c] += N[a] * E[a][c];
                for (int m = 0; m < 3; ++m) J[c][m] += dN[a][m] * E[a][c];
            }
        for (int c = 0; c < 3; ++c) negF[c] = -(F[c] - b[c]);
        if (!og_solve3(J, negF, d)) {
            if (iters) *iters = it + 1;
            return 0;
        }
        for (int m = 0; m < 3; ++m) xi[m] += d[m];
        double dmax = fmax(fabs(d[0]), fmax(fabs(d[1]), fabs(d[2])));
        if (!isfinite(xi[0]) || !isfinite(xi[1]) || !isfinite(xi[2])) {
            if (iters) *iters = it + 1;
            return 0;
        }
        if (dmax <= OG_NEWTON_TOL) {
            if (iters) *iters = it + 1;
            return 1;
        }
    }
    if (iters) *iters = OG_NEWTON_MAXIT;
    return 0;
}

static int og_in_window(const double xi[3]) {
    for (int m = 0; m < 3; ++m)
        if (!(xi[m] >= OG_WIN_LO && xi[m] <= OG_WIN_HI)) return 0;
    return 1;
}

/* The in-cell predicate for one cell. */
int og_cell_contains(const og_grid* g, int64_t cell, const double p[3], double xi[3]) {
    double X[8][3];
    og_cell_corners(g, cell, X);
    return og_newton(X, p, xi, NULL) && og_in_window(xi);
}

/* ---------------------------------------------------------------- bins */

static void og_cell_box(const og_grid* g, int64_t cell, double lo[3], double hi[3]) {
    double X[8][3];
    og_cell_corners(g, cell, X);
    for (int c = 0; c < 3; ++c) {
        lo[c] = hi[c] = X[0][c];
        for (int a = 1; a < 8; ++a) {
            lo[c] = fmin(lo[c], X[a][c]);
            hi[c] = fmax(hi[c], X[a][c]);
        }
    }
    double d2 = 0;
    for (int c = 0; c < 3; ++c) d2 += (hi[c] - lo[c]) * (hi[c] - lo[c]);
    double pad = OG_INFLATE * sqrt(d2);
    for (int c = 0; c < 3; ++c) {
        lo[c] -= pad;
        hi[c] += pad;
    }
}

static int32_t og_bin_index(const og_bins* b, int d, double v) {
    double t = (v - b->lo[d]) / b->w[d];
    if (t < 0) return 0;
    int64_t k = (int64_t)floor(t);
    if (k >= b->nb[d]) k = b->nb[d] - 1;
    return (int32_t)k;
}

og_bins* og_bins_build(const og_grid* g, int nbx, int nby, int nbz) {
    og_bins* b = (og_bins*)calloc(1, sizeof(og_bins));
    int64_t nn = (int64_t)g->n[0] * g->n[1] * g->n[2];
    const double* xs[3] = {g->x, g->y, g->z};
    int nbv[3] = {nbx, nby, nbz};
    double glo[3], ghi[3], ext = 0;
    for (int d = 0; d < 3; ++d) {
        glo[d] = ghi[d] = xs[d][0];
        for (int64_t q = 1; q < nn; ++q) {
            glo[d] = fmin(glo[d], xs[d][q]);
            ghi[d] = fmax(ghi[d], xs[d][q]);
        }
        ext = fmax(ext, ghi[d] - glo[d]);
    }
    /* the padded box contains every cell's inflated box (1e-9 x diagonal <= 1e-8 x extent) */
    double pad = 1e-8 * ext + 1e-300;
    for (int d = 0; d < 3; ++d) {
        b->lo[d] = glo[d] - pad;
        b->hi[d] = ghi[d] + pad;
        b->nb[d] = nbv[d] < 1 ? 1 : nbv[d];
        b->w[d] = (b->hi[d] - b->lo[d]) / b->nb[d];
    }
    int64_t nbins = (int64_t)b->nb[0] * b->nb[1] * b->nb[2];
    b->start = (int64_t*)calloc((size_t)nbins + 1, sizeof(int64_t));
    int64_t ncell = og_num_cells(g);
    /* pass 1: count registrations per bin */
    for (int64_t c = 0; c < ncell; ++c) {
        double lo[3], hi[3];
        og_cell_box(g, c, lo, hi);
        int32_t a0[3], a1[3];
        for (int d = 0; d < 3; ++d) {
            a0[d] = og_bin_index(b, d, lo[d]);
            a1[d] = og_bin_index(b, d, hi[d]);
        }
        for (int32_t kz = a0[2]; kz <= a1[2]; ++kz)
            for (int32_t ky = a0[1]; ky <= a1[1]; ++ky)
                for (int32_t kx = a0[0]; kx <= a1[0]; ++kx)
                    b->start[kx + (int64_t)b->nb[0] * (ky + (int64_t)b->nb[1] * kz) + 1] += 1;
    }
    for (int64_t q = 0; q < nbins; ++q) b->start[q + 1] += b->start[q];
    b->nreg = b->start[nbins];
    b->cells = (int32_t*)malloc((size_t)(b->nreg > 0 ? b->nreg : 1) * sizeof(int32_t));
    int64_t* fill = (int64_t*)malloc((size_t)nbins * sizeof(int64_t));
    memcpy(fill, b->start, (size_t)nbins * sizeof(int64_t));
    /* pass 2: fill in ascending cell order, so each bin's list is ascending */
    for (int64_t c = 0; c < ncell; ++c) {
        double lo[3], hi[3];
        og_cell_box(g, c, lo, hi);
        int32_t a0[3], a1[3];
        for (int d = 0; d < 3; ++d) {
            a0[d] = og_bin_index(b, d, lo[d]);
            a1[d] = og_bin_index(b, d, hi[d]);
        }
        for (int32_t kz = a0[2]; kz <= a1[2]; ++kz)
            for (int32_t ky = a0[1]; ky <= a1[1]; ++ky)
                for (int32_t kx = a0[0]; kx <= a1[0]; ++kx) {
                    int64_t q = kx + (int64_t)b->nb[0] * (ky + (int64_t)b->nb[1] * kz);
                    b->cells[fill[q]++] = (int32_t)c;
                }
    }
    free(fill);
    return b;
}

void og_bins_free(og_bins* b) {
    if (!b) return;
    free(b->start);
    free(b->cells);
    free(b);
}

int64_t og_bins_nreg(const og_bins* b) { return b->nreg; }

/* A cell may donate only if none of its corner nodes is blanked (Sec. 2.4: blanked donors are rejected). */
static int og_cell_usable(const og_grid* g, int64_t c) {
    if (!g->iblank) return 1;
    int64_t nd[8];
    og_cell_nodes(g, c, nd);
    for (int a = 0; a < 8; ++a)
        if (!g->iblank[nd[a]]) return 0;
    return 1;
}

/* Donor cell of p by the control-cell bins: lowest-id usable containing cell, or -1. */
int64_t og_find_donor(const og_grid* g, const og_bins* b, const double p[3], double xi[3]) {
    for (int d = 0; d < 3; ++d)
        if (!(p[d] >= b->lo[d] && p[d] <= b->hi[d])) return -1;
    int64_t q = og_bin_index(b, 0, p[0]) +
                (int64_t)b->nb[0] * (og_bin_index(b, 1, p[1]) + (int64_t)b->nb[1] * og_bin_index(b, 2, p[2]));
    for (int64_t r = b->start[q]; r < b->start[q + 1]; ++r) {
        if (og_cell_usable(g, b->cells[r]) && og_cell_contains(g, b->cells[r], p, xi)) return b->cells[r];
    }
    return -1;
}

/* Same selection without bins: every cell of the grid in ascending id. */
int64_t og_find_donor_brute(const og_grid* g, const double p[3], double xi[3]) {
    int64_t ncell = og_num_cells(g);
    for (int64_t c = 0; c < ncell; ++c)
        if (og_cell_usable(g, c) && og_cell_contains(g, c, p, xi)) return c;
    return -1;
}

/* Donor search for n points (donor-frame coordinates p, n x 3 row-major).  Outputs: cell id (or -1),
 * xi (n x 3), the 8 corner node ids (n x 8) and the 8 trilinear weights (n x 8) of each found donor.
 * Points with a non-finite coordinate are skipped (cell = -2).  brute != 0 ignores the bins. */
void og_search(const og_grid* g, const og_bins* b, int brute, int64_t n, const double* p, int64_t* cell,
               double* xi, int64_t* nodes, double* w) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < n; ++q) {
        const double* pq = p + 3 * q;
        double xq[3] = {NAN, NAN, NAN};
        int64_t c;
        if (!isfinite(pq[0]) || !isfinite(pq[1]) || !isfinite(pq[2]))
            c = -2;
        else
            c = brute ? og_find_donor_brute(g, pq, xq) : og_find_donor(g, b, pq, xq);
        cell[q] = c;
        if (c >= 0) {
            double N[8];
            int64_t nd[8];
            og_shape(xq, N);
            og_cell_nodes(g, c, nd);
            for (int a = 0; a < 8; ++a) {
                nodes[8 * q + a] = nd[a];
                w[8 * q + a] = N[a];
            }
            for (int m = 0; m < 3; ++m) xi[3 * q + m] = xq[m];
        } else {
            for (int a = 0; a < 8; ++a) {
                nodes[8 * q + a] = -1;
                w[8 * q + a] = 0.0;
            }
            for (int m = 0; m < 3; ++m) xi[3 * q + m] = NAN;
        }
    }
}

/* Newton on one explicit hexahedron (for tests): X is 8x3 row-major. */
int og_newton_hex(const double* X, const double* p, double* xi, int* iters) {
    double Xa[8][3];
    for (int a = 0; a < 8; ++a)
        for (int c = 0; c < 3; ++c) Xa[a][c] = X[3 * a + c];
    return og_newton(Xa, p, xi, iters);
}

/* ---------------------------------------------------------------------------------------------------------
 * Hole cutting (Sec. 2.2.1): a point is inside a closed triangulated body surface iff a ray from it crosses the
 * surface an odd number of times.  The ray runs along the surface's shortest bounding-box axis r (the first
 * such axis on a tie), with (u, w) the two axes that follow it cyclically; a triangle is crossed when the point's
 * (u, w) lies in the triangle's projection on the u-w plane and the crossing lies strictly ahead along r.  A
 * point on a projected edge belongs to the one triangle whose counter-clockwise edge runs toward -w (or, level,
 * toward -u), so a ray through a shared edge or vertex is counted once.  Every operation is one FP64 rounding
 * (no fused multiply-add), so the decision is reproducible.  (For a closed surface the parity does not depend
 * on the ray's direction away from those ties; the shortest axis keeps the projected triangles apart.)
 * ------------------------------------------------------------------------------------------------------- */
__attribute__((optimize("fp-contract=off"))) static double og_edge2(double ay, double az, double by, double bz,
                                                                   double py, double pz) {
    return (by - ay) * (pz - az) - (bz - az) * (py - ay);
}

static int og_edge_owns(double ay, double az, double by, double bz) { return (bz < az) || (bz == az && by < ay); }

/* ax = {r, u, w}: the ray's axis and the projection plane's two axes */
__attribute__((optimize("fp-contract=off"))) static int og_ray_crosses(const double* A, const double* B,
                                                                      const double* C, const double* p,
                                                                      const int ax[3]) {
    const int r = ax[0], u = ax[1], w = ax[2];
    const double area = og_edge2(A[u], A[w], B[u], B[w], C[u], C[w]);
    if (area == 0.0) return 0; /* edge-on: never crossed */
    const double* a = A;
    const double* b = area > 0 ? B : C; /* counter-clockwise order in the u-w plane */
    const double* c = area > 0 ? C : B;
    const double w0 = og_edge2(b[u], b[w], c[u], c[w], p[u], p[w]);
    const double w1 = og_edge2(c[u], c[w], a[u], a[w], p[u], p[w]);
    const double w2 = og_edge2(a[u], a[w], b[u], b[w], p[u], p[w]);
    if (w0 < 0 || w1 < 0 || w2 < 0) return 0;
    if (w0 == 0 && !og_edge_owns(b[u], b[w], c[u], c[w])) return 0;
    if (w1 == 0 && !og_edge_owns(c[u], c[w], a[u], a[w])) return 0;
    if (w2 == 0 && !og_edge_owns(a[u], a[w], b[u], b[w])) return 0;
    const double s = w0 + w1 + w2;
    const double xs = w0 * a[r] + w1 * b[r] + w2 * c[r]; /* s times the crossing's coordinate along r */
    return xs > p[r] * s;
}

/* inside[q] = 1 iff point q (n x 3, row-major) is inside the surface (nv vertices, nt triangles of vertex ids). */
void og_surface_inside(int64_t nv, const double* V, int64_t nt, const int32_t* T, int64_t n, const double* P,
                       uint8_t* inside) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < nv; ++i)
        for (int c = 0; c < 3; ++c) {
            if (V[3 * i + c] < lo[c]) lo[c] = V[3 * i + c];
            if (V[3 * i + c] > hi[c]) hi[c] = V[3 * i + c];
        }
    int r = 0;
    for (int c = 1; c < 3; ++c)
        if (hi[c] - lo[c] < hi[r] - lo[r]) r = c;
    const int ax[3] = {r, (r + 1) % 3, (r + 2) % 3};
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < n; ++q) {
        int odd = 0;
        for (int64_t t = 0; t < nt; ++t)
            odd ^= og_ray_crosses(V + 3 * T[3 * t], V + 3 * T[3 * t + 1], V + 3 * T[3 * t + 2], P + 3 * q, ax);
        inside[q] = (uint8_t)odd;
    }
}
