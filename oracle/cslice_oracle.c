/*
 * Plain FP64 CPU oracle for the convolution-surface lattice slicer
 * (arxiv 2101.05031). TEST INFRASTRUCTURE ONLY: the tests, the smoke check
 * and the CPU-baseline leg of the benchmark call this file; the product path
 * never does. It shares no code, header, table or constant with the CUDA
 * library: it is a single, self-contained C file written from the paper.
 *
 * Everything is single-threaded double precision. FP32 inputs (node
 * positions, radii) are widened to double exactly before any arithmetic.
 *
 * Readings of the paper that this file implements (where the paper is silent
 * or inconsistent):
 *   - Sign: the paper writes the solid as {F <= 0} (Eq. 1) but defines
 *     F = -C + sum(...) (Eq. 3, Eq. 6), which is largest on the skeleton.
 *     Reading: a point is inside iff Sigma(p) >= C, where Sigma is the
 *     weighted sum of Eq. 6 without the -C.
 *   - Jacobian: Eq. 7 integrates over the chord parameter s in [s1, s2];
 *     Eq. 6 integrates over arc length. Reading: arc length, i.e. Eq. 7 times
 *     the chord length l.
 *   - p1 -> p2 runs in the v_s -> v_e direction; a line that misses the
 *     sphere, an empty clip (s1 >= s2) or a zero-length edge contributes 0.
 *   - Weight (Sec. 3.2, "r_i" adjusts the radius): PHYSICAL mode maps the
 *     physical strut radius rho to w = C * 15 R^4 / (16 (R^2 - rho^2)^(5/2)),
 *     so that an isolated infinite strut has its iso-surface at distance rho
 *     (the infinite-line integral is 16 (R^2 - d^2)^(5/2) / (15 R^4)).
 *     RAW mode uses w = rho literally, as the paper's r_i.
 *   - Marching squares (Sec. 4, last paragraph; details are not given):
 *     linear interpolation of the crossing on each grid edge, the grid padded
 *     by one ring of outside samples so every contour closes, the asymptotic
 *     saddle rule on the mean of the four corners, loops oriented with the
 *     inside on the left, each loop started at its smallest grid-edge id and
 *     loops listed by that id.
 *   - Density (Eq. 9): deterministic m^3 stratified samples per cell and a
 *     sigmoid of (Sigma - C) / T instead of Monte-Carlo hits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MODE_PHYSICAL 0
#define ORC_MODE_RAW 1

/* ------------------------------------------------------------------------ */
/* Kernel, weight and segment integral (Sec. 3.2, Eq. 5-7)                   */
/* ------------------------------------------------------------------------ */

/* Eq. 5: quartic compactly supported kernel of the squared distance. */
double orc_kernel(double dist2, double R)
{
    if (dist2 >= R * R) return 0.0;
    double g = 1.0 - dist2 / (R * R);
    return g * g;
}

/* Per-edge weight r_i of Eq. 6 (see the reading above). */
double orc_weight(double rho, double R, double C, int mode)
{
    if (mode == ORC_MODE_RAW) return rho;
    double q = R * R - rho * rho;
    return C * 15.0 * pow(R, 4) / (16.0 * pow(q, 2.5));
}

/* d w / d rho of orc_weight. */
double orc_weight_drho(double rho, double R, double C, int mode)
{
    if (mode == ORC_MODE_RAW) return 1.0;
    double q = R * R - rho * rho;
    return orc_weight(rho, R, C, mode) * 5.0 * rho / q;
}

static double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/*
 * Eq. 7 with the arc-length Jacobian: the integral of f(p - x) over the edge
 * from vs to ve, x running along the edge by arc length.
 *   p1, p2: where the edge's line meets the sphere of radius R around p,
 *           ordered along vs -> ve;
 *   s1 = max(0, (vs - p1).(p2 - p1) / |p2 - p1|^2),
 *   s2 = min(1, (ve - p1).(p2 - p1) / |p2 - p1|^2),
 *   value = l * (3 l^4 s^5 - 15 a l^2 s^4 + 20 a^2 s^3) / (15 R^4) |_{s1}^{s2}
 *   with l = |p2 - p1| and a = (p - p1).(p2 - p1).
 */
double orc_segment_integral(const double p[3], const double vs[3], const double ve[3], double R)
{
    double d[3] = {ve[0] - vs[0], ve[1] - vs[1], ve[2] - vs[2]};
    double len2 = dot3(d, d);
    if (len2 == 0.0) return 0.0;
    double len = sqrt(len2);
    double u[3] = {d[0] / len, d[1] / len, d[2] / len};
    double q[3] = {p[0] - vs[0], p[1] - vs[1], p[2] - vs[2]};
    double t0 = dot3(q, u);
    double e[3] = {q[0] - t0 * u[0], q[1] - t0 * u[1], q[2] - t0 * u[2]};
    double dist2 = dot3(e, e);
    if (dist2 >= R * R) return 0.0;          /* the line misses the sphere */
    double hw = sqrt(R * R - dist2);
    double p1[3], p2[3], ch[3];
    for (int k = 0; k < 3; ++k) {
        p1[k] = vs[k] + (t0 - hw) * u[k];
        p2[k] = vs[k] + (t0 + hw) * u[k];
        ch[k] = p2[k] - p1[k];
    }
    double l2 = dot3(ch, ch);
    if (l2 == 0.0) return 0.0;               /* tangent line */
    double l = sqrt(l2);
    double a1[3] = {vs[0] - p1[0], vs[1] - p1[1], vs[2] - p1[2]};
    double a2[3] = {ve[0] - p1[0], ve[1] - p1[1], ve[2] - p1[2]};
    double s1 = dot3(a1, ch) / l2;
    double s2 = dot3(a2, ch) / l2;
    if (s1 < 0.0) s1 = 0.0;
    if (s2 > 1.0) s2 = 1.0;
    if (s1 >= s2) return 0.0;
    double pp[3] = {p[0] - p1[0], p[1] - p1[1], p[2] - p1[2]};
    double a = dot3(pp, ch);
    double l4 = l2 * l2;
    double F2 = 3.0 * l4 * pow(s2, 5) - 15.0 * a * l2 * pow(s2, 4) + 20.0 * a * a * pow(s2, 3);
    double F1 = 3.0 * l4 * pow(s1, 5) - 15.0 * a * l2 * pow(s1, 4) + 20.0 * a * a * pow(s1, 3);
    return l * (F2 - F1) / (15.0 * pow(R, 4));
}

/* ------------------------------------------------------------------------ */
/* Lattice helpers                                                          */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t n_edges;
    double* vs;      /* [n_edges][3], lower endpoint (v_s^z <= v_e^z, Eq. 8) */
    double* ve;      /* [n_edges][3] */
    double* w;       /* weight r_i of Eq. 6 */
    int64_t* order;  /* edge ids sorted by the lower endpoint's z (Sec. 4) */
} orc_edges;

static const double* g_sort_key;

static int cmp_lower_z(const void* A, const void* B)
{
    int64_t a = *(const int64_t*)A, b = *(const int64_t*)B;
    double za = g_sort_key[3 * a + 2], zb = g_sort_key[3 * b + 2];
    if (za < zb) return -1;
    if (za > zb) return 1;
    return (a < b) ? -1 : (a > b);
}

static int build_edges(const float* nodes, int64_t n_nodes, const int32_t* edges,
                       const float* radius, int64_t n_edges, double R, double C, int mode,
                       orc_edges* E)
{
    E->n_edges = n_edges;
    E->vs = (double*)malloc(sizeof(double) * 3 * (size_t)(n_edges ? n_edges : 1));
    E->ve = (double*)malloc(sizeof(double) * 3 * (size_t)(n_edges ? n_edges : 1));
    E->w = (double*)malloc(sizeof(double) * (size_t)(n_edges ? n_edges : 1));
    E->order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_edges ? n_edges : 1));
    if (!E->vs || !E->ve || !E->w || !E->order) return -2;
    for (int64_t j = 0; j < n_edges; ++j) {
        int32_t i0 = edges[2 * j], i1 = edges[2 * j + 1];
        if (i0 < 0 || i1 < 0 || i0 >= n_nodes || i1 >= n_nodes) return -1;
        const float* a = nodes + 3 * (int64_t)i0;
        const float* b = nodes + 3 * (int64_t)i1;
        /* v_s is the endpoint with the smaller z (Eq. 8). */
        int swap = ((double)b[2] < (double)a[2]);
        const float* lo = swap ? b : a;
        const float* hi = swap ? a : b;
        for (int k = 0; k < 3; ++k) {
            E->vs[3 * j + k] = (double)lo[k];
            E->ve[3 * j + k] = (double)hi[k];
        }
        E->w[j] = orc_weight((double)radius[j], R, C, mode);
        E->order[j] = j;
    }
    g_sort_key = E->vs;
    qsort(E->order, (size_t)n_edges, sizeof(int64_t), cmp_lower_z);
    return 0;
}

static void free_edges(orc_edges* E)
{
    free(E->vs);
    free(E->ve);
    free(E->w);
    free(E->order);
}

/* Active-edge list of Sec. 4 (Steps 1-6): edges whose swept sphere of radius
 * R meets the plane z = const (Eq. 8), maintained as the plane rises. */
typedef struct {
    int64_t* idx;
    int64_t n, cap;
    int64_t k;      /* next edge of the sorted list not yet examined */
} orc_active;

static void active_init(orc_active* A, int64_t cap)
{
    A->cap = cap > 16 ? cap : 16;
    A->idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)A->cap);
    A->n = 0;
    A->k = 0;
}

/* Step 2 and Step 3 for the plane at height z (z must not decrease). */
static void active_advance(orc_active* A, const orc_edges* E, double R, double z)
{
    /* Step 2: add edges until one whose swept solid is wholly above z. */
    while (A->k < E->n_edges) {
        int64_t j = E->order[A->k];
        if (E->vs[3 * j + 2] - R > z) break;
        if (A->n == A->cap) {
            A->cap *= 2;
            A->idx = (int64_t*)realloc(A->idx, sizeof(int64_t) * (size_t)A->cap);
        }
        A->idx[A->n++] = j;
        A->k++;
    }
    /* Step 3: drop edges whose swept solid is wholly below z. */
    int64_t m = 0;
    for (int64_t i = 0; i < A->n; ++i) {
        int64_t j = A->idx[i];
        if (E->ve[3 * j + 2] + R < z) continue;
        A->idx[m++] = j;
    }
    A->n = m;
}

/* Step 4 at one point: Sigma(p) = sum over active edges of r_i * integral. */
static double active_sigma(const orc_active* A, const orc_edges* E, double R, const double p[3])
{
    double s = 0.0;
    for (int64_t i = 0; i < A->n; ++i) {
        int64_t j = A->idx[i];
        s += E->w[j] * orc_segment_integral(p, E->vs + 3 * j, E->ve + 3 * j, R);
    }
    return s;
}

/* ------------------------------------------------------------------------ */
/* Slicing (Sec. 4, Steps 1-6)                                              */
/* ------------------------------------------------------------------------ */

/*
 * Sigma on the pixel centres (x0 + (i + 1/2) px, y0 + (j + 1/2) px, z_k),
 * z_k = z0 + k dz, k = 0 .. n_layers-1. out: [n_layers][ny][nx].
 * Returns 0, or -1 on a bad edge index, -2 on allocation failure.
 */
int orc_slice_sigma(const float* nodes, int64_t n_nodes, const int32_t* edges,
                    const float* radius, int64_t n_edges, double R, double C, int mode,
                    double z0, double dz, int32_t n_layers,
                    double x0, double y0, int32_t nx, int32_t ny, double px, double* out)
{
    orc_edges E;
    int rc = build_edges(nodes, n_nodes, edges, radius, n_edges, R, C, mode, &E);
    if (rc) { free_edges(&E); return rc; }
    orc_active A;
    active_init(&A, 1024);
    for (int32_t k = 0; k < n_layers; ++k) {            /* Steps 1, 5, 6 */
        double z = z0 + (double)k * dz;
        active_advance(&A, &E, R, z);                    /* Steps 2, 3 */
        for (int32_t j = 0; j < ny; ++j)                 /* Step 4 */
            for (int32_t i = 0; i < nx; ++i) {
                double p[3] = {x0 + ((double)i + 0.5) * px, y0 + ((double)j + 0.5) * px, z};
                out[((int64_t)k * ny + j) * nx + i] = active_sigma(&A, &E, R, p);
            }
    }
    free(A.idx);
    free_edges(&E);
    return 0;
}

static const double* g_pts;
static int cmp_pt_z(const void* A, const void* B)
{
    int64_t a = *(const int64_t*)A, b = *(const int64_t*)B;
    double za = g_pts[3 * a + 2], zb = g_pts[3 * b + 2];
    if (za < zb) return -1;
    if (za > zb) return 1;
    return (a < b) ? -1 : (a > b);
}

/* Sigma at arbitrary points: the same sweep, visiting the points in
 * ascending z. pts: [n][3]; out: [n]. */
int orc_sigma_points(const float* nodes, int64_t n_nodes, const int32_t* edges,
                     const float* radius, int64_t n_edges, double R, double C, int mode,
                     const double* pts, int64_t n, double* out)
{
    orc_edges E;
    int rc = build_edges(nodes, n_nodes, edges, radius, n_edges, R, C, mode, &E);
    if (rc) { free_edges(&E); return rc; }
    int64_t* ord = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    for (int64_t i = 0; i < n; ++i) ord[i] = i;
    g_pts = pts;
    qsort(ord, (size_t)n, sizeof(int64_t), cmp_pt_z);
    orc_active A;
    active_init(&A, 1024);
    for (int64_t t = 0; t < n; ++t) {
        int64_t i = ord[t];
        active_advance(&A, &E, R, pts[3 * i + 2]);
        out[i] = active_sigma(&A, &E, R, pts + 3 * i);
    }
    free(A.idx);
    free(ord);
    free_edges(&E);
    return 0;
}

/* Eq. 8 for one plane: writes the ids of the active edges (ascending id)
 * into out (capacity n_edges) and returns their count. */
int64_t orc_active_set(const float* nodes, int64_t n_nodes, const int32_t* edges,
                       const float* radius, int64_t n_edges, double R, double z, int64_t* out)
{
    int64_t n = 0;
    (void)radius;
    for (int64_t j = 0; j < n_edges; ++j) {
        int32_t i0 = edges[2 * j], i1 = edges[2 * j + 1];
        if (i0 < 0 || i1 < 0 || i0 >= n_nodes || i1 >= n_nodes) return -1;
        double za = nodes[3 * (int64_t)i0 + 2], zb = nodes[3 * (int64_t)i1 + 2];
        double lo = za < zb ? za : zb, hi = za < zb ? zb : za;
        if (lo - R <= z && hi + R >= z) out[n++] = j;
    }
    return n;
}

/* ------------------------------------------------------------------------ */
/* Marching squares and loop assembly (Sec. 4, last paragraph)              */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t n_loops;
    int64_t n_verts;
    int64_t* loop_off;   /* [n_loops + 1] */
    int64_t* edge_id;    /* [n_verts] grid-edge id of each vertex */
    double* xy;          /* [n_verts][2] in mm */
} orc_loops;

void orc_loops_free(orc_loops* L)
{
    if (!L) return;
    free(L->loop_off);
    free(L->edge_id);
    free(L->xy);
    free(L);
}

/*
 * Sample grid padded by one ring: padded index (I, J), I in [0, nx+1],
 * J in [0, ny+1]; sample (I, J) is pixel (I-1, J-1) when that exists, else an
 * outside sample of value 0. Grid edges: the horizontal edge from (I, J) to
 * (I+1, J) has id 2 (J (nx+2) + I); the vertical edge from (I, J) to (I, J+1)
 * has id 2 (J (nx+2) + I) + 1.
 */
typedef struct {
    const double* s;
    int32_t nx, ny;
    double x0, y0, px, C;
} ms_grid;

static double ms_val(const ms_grid* g, int64_t I, int64_t J)
{
    if (I < 1 || J < 1 || I > g->nx || J > g->ny) return 0.0;
    return g->s[(J - 1) * (int64_t)g->nx + (I - 1)];
}

static int ms_in(const ms_grid* g, int64_t I, int64_t J)
{
    if (I < 1 || J < 1 || I > g->nx || J > g->ny) return 0;   /* padding is outside */
    return ms_val(g, I, J) >= g->C;
}

static void ms_pos(const ms_grid* g, int64_t I, int64_t J, double* x, double* y)
{
    *x = g->x0 + ((double)(I - 1) + 0.5) * g->px;
    *y = g->y0 + ((double)(J - 1) + 0.5) * g->px;
}

/* Crossing point on the grid edge between samples A and B (one inside, one
 * outside): the zero of the linear interpolant of Sigma - C. */
static void ms_cross(const ms_grid* g, int64_t IA, int64_t JA, int64_t IB, int64_t JB, double xy[2])
{
    double sa = ms_val(g, IA, JA), sb = ms_val(g, IB, JB);
    double xa, ya, xb, yb;
    ms_pos(g, IA, JA, &xa, &ya);
    ms_pos(g, IB, JB, &xb, &yb);
    if (!ms_in(g, IA, JA)) {   /* make A the inside sample */
        double t;
        t = sa; sa = sb; sb = t;
        t = xa; xa = xb; xb = t;
        t = ya; ya = yb; yb = t;
    }
    double t = (sa - g->C) / (sa - sb);
    xy[0] = xa + t * (xb - xa);
    xy[1] = ya + t * (yb - ya);
}

orc_loops* orc_marching_squares(const double* sigma, int32_t nx, int32_t ny,
                                double x0, double y0, double px, double C)
{
    ms_grid g = {sigma, nx, ny, x0, y0, px, C};
    int64_t W = (int64_t)nx + 2, H = (int64_t)ny + 2;
    int64_t n_ids = 2 * W * H;
    int64_t* succ = (int64_t*)malloc(sizeof(int64_t) * (size_t)n_ids);
    unsigned char* has = (unsigned char*)calloc((size_t)n_ids, 1);
    if (!succ || !has) { free(succ); free(has); return NULL; }
    for (int64_t i = 0; i < n_ids; ++i) succ[i] = -1;

    /* Crossings on every grid edge. */
    for (int64_t J = 0; J < H; ++J)
        for (int64_t I = 0; I < W; ++I) {
            int64_t base = 2 * (J * W + I);
            if (I + 1 < W && ms_in(&g, I, J) != ms_in(&g, I + 1, J)) has[base] = 1;
            if (J + 1 < H && ms_in(&g, I, J) != ms_in(&g, I, J + 1)) has[base + 1] = 1;
        }

    /* One segment per crossing pair inside each cell. Corners counter-
     * clockwise: c0 (I,J), c1 (I+1,J), c2 (I+1,J+1), c3 (I,J+1); side k runs
     * from corner k to corner k+1: bottom, right, top, left. Walking the
     * sides counter-clockwise, a side that leaves an inside corner for an
     * outside one is where a contour (inside on its left) enters the cell,
     * and a side that goes from outside to inside is where it leaves. */
    for (int64_t J = 0; J + 1 < H; ++J)
        for (int64_t I = 0; I + 1 < W; ++I) {
            int64_t cI[4] = {I, I + 1, I + 1, I};
            int64_t cJ[4] = {J, J, J + 1, J + 1};
            int in[4];
            for (int k = 0; k < 4; ++k) in[k] = ms_in(&g, cI[k], cJ[k]);
            int64_t side[4] = {2 * (J * W + I), 2 * (J * W + I + 1) + 1,
                               2 * ((J + 1) * W + I), 2 * (J * W + I) + 1};
            int n_enter = 0;
            int enter[2], leave[2];
            int n_leave = 0;
            for (int k = 0; k < 4; ++k) {
                int a = in[k], b = in[(k + 1) & 3];
                if (a && !b) enter[n_enter++] = k;
                if (!a && b) leave[n_leave++] = k;
            }
            if (n_enter == 0) continue;
            if (n_enter == 1) {
                succ[side[enter[0]]] = side[leave[0]];
                continue;
            }
            /* Saddle: two inside corners on a diagonal. The mean of the four
             * corners decides whether the inside corners are joined through
             * the centre; if joined, each contour turns to the next side
             * counter-clockwise, else to the previous one. */
            double mean = 0.25 * (ms_val(&g, cI[0], cJ[0]) + ms_val(&g, cI[1], cJ[1]) +
                                  ms_val(&g, cI[2], cJ[2]) + ms_val(&g, cI[3], cJ[3]));
            int joined = mean >= C;
            for (int q = 0; q < 2; ++q) {
                int k = enter[q];
                int to = joined ? ((k + 1) & 3) : ((k + 3) & 3);
                succ[side[k]] = side[to];
            }
        }

    /* Follow successors; visiting ids in increasing order means each loop is
     * first met at its smallest edge id, so loops come out sorted by it. */
    int64_t n_cross = 0;
    for (int64_t i = 0; i < n_ids; ++i) n_cross += has[i];
    orc_loops* L = (orc_loops*)calloc(1, sizeof(orc_loops));
    L->loop_off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_cross + 1));
    L->edge_id = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_cross ? n_cross : 1));
    L->xy = (double*)malloc(sizeof(double) * 2 * (size_t)(n_cross ? n_cross : 1));
    unsigned char* seen = (unsigned char*)calloc((size_t)n_ids, 1);
    int64_t nv = 0, nl = 0;
    L->loop_off[0] = 0;
    for (int64_t i = 0; i < n_ids; ++i) {
        if (!has[i] || seen[i]) continue;
        int64_t e = i;
        while (!seen[e]) {
            seen[e] = 1;
            int64_t cell = e / 2;
            int64_t I = cell % W, J = cell / W;
            if ((e & 1) == 0) ms_cross(&g, I, J, I + 1, J, L->xy + 2 * nv);
            else ms_cross(&g, I, J, I, J + 1, L->xy + 2 * nv);
            L->edge_id[nv++] = e;
            e = succ[e];
            if (e < 0) { /* cannot happen for a closed padded grid */
                free(seen); free(succ); free(has); orc_loops_free(L); return NULL;
            }
        }
        L->loop_off[++nl] = nv;
    }
    L->n_loops = nl;
    L->n_verts = nv;
    free(seen);
    free(succ);
    free(has);
    return L;
}

/* ------------------------------------------------------------------------ */
/* Volume fraction of the smoothed solid per density cell (Eq. 9)           */
/* ------------------------------------------------------------------------ */

typedef struct {
    double ox, oy, oz, h;
    int32_t cx, cy, cz, m;
    double T;
} orc_cells;

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* Sample points of the listed cells: p = o + h (c + (k + 1/2) / m) per axis,
 * cell-major, sample index (kz m + ky) m + kx. */
static double* cell_samples(const orc_cells* c, const int64_t* cells, int64_t n_cells)
{
    int64_t m3 = (int64_t)c->m * c->m * c->m;
    double* P = (double*)malloc(sizeof(double) * 3 * (size_t)(n_cells * m3 > 0 ? n_cells * m3 : 1));
    for (int64_t q = 0; q < n_cells; ++q) {
        int64_t id = cells[q];
        int64_t ix = id % c->cx, iy = (id / c->cx) % c->cy, iz = id / ((int64_t)c->cx * c->cy);
        for (int64_t s = 0; s < m3; ++s) {
            int64_t kx = s % c->m, ky = (s / c->m) % c->m, kz = s / ((int64_t)c->m * c->m);
            double* p = P + 3 * (q * m3 + s);
            p[0] = c->ox + c->h * ((double)ix + ((double)kx + 0.5) / c->m);
            p[1] = c->oy + c->h * ((double)iy + ((double)ky + 0.5) / c->m);
            p[2] = c->oz + c->h * ((double)iz + ((double)kz + 0.5) / c->m);
        }
    }
    return P;
}

/* vf_c = (1/m^3) sum_k sigmoid((Sigma(p_ck) - C) / T) for each listed cell. */
int orc_volume_fraction(const float* nodes, int64_t n_nodes, const int32_t* edges,
                        const float* radius, int64_t n_edges, double R, double C, int mode,
                        double ox, double oy, double oz, double h, int32_t cx, int32_t cy,
                        int32_t cz, int32_t m, double T, const int64_t* cells, int64_t n_cells,
                        double* out_vf)
{
    orc_cells c = {ox, oy, oz, h, cx, cy, cz, m, T};
    int64_t m3 = (int64_t)m * m * m;
    double* P = cell_samples(&c, cells, n_cells);
    double* S = (double*)malloc(sizeof(double) * (size_t)(n_cells * m3 > 0 ? n_cells * m3 : 1));
    int rc = orc_sigma_points(nodes, n_nodes, edges, radius, n_edges, R, C, mode, P,
                              n_cells * m3, S);
    if (rc == 0)
        for (int64_t q = 0; q < n_cells; ++q) {
            double acc = 0.0;
            for (int64_t s = 0; s < m3; ++s) acc += sigmoid((S[q * m3 + s] - C) / T);
            out_vf[q] = acc / (double)m3;
        }
    free(P);
    free(S);
    return rc;
}

/*
 * Gradient of one edge's integral I = int_0^L f(|p - a - t u|^2) dt with
 * respect to its endpoints a, b (u = (b - a) / L). Differentiating under the
 * integral in the fixed-bounds form L int_0^1 f(|p - a - s (b - a)|^2) ds
 * (f is C^1 and vanishes with its derivative on the support sphere, so the
 * moving clip points add nothing). In the frame of the edge:
 * p - a = t0 u + e (e orthogonal to u), tau = t - t0, w^2 = R^2 - |e|^2,
 * f'(q) = -(2 / R^4) (w^2 - tau^2). With the moments over the clipped
 * interval [tau1, tau2]:
 *   M0 = int (w^2 - tau^2) dtau, M1 = int (w^2 - tau^2) tau dtau,
 *   M2 = int (w^2 - tau^2) tau^2 dtau,
 *   dI/da = -u I / L - (4/R^4) [u ((1 - t0/L) M1 - M2/L) - e ((1 - t0/L) M0 - M1/L)]
 *   dI/db = +u I / L - (4/R^4) [u ((t0/L) M1 + M2/L) - e ((t0/L) M0 + M1/L)].
 * Returns I; writes dI/da, dI/db.
 */
double orc_segment_integral_grad(const double p[3], const double a[3], const double b[3],
                                 double R, double dIda[3], double dIdb[3])
{
    for (int k = 0; k < 3; ++k) dIda[k] = dIdb[k] = 0.0;
    double d[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double L2 = dot3(d, d);
    if (L2 == 0.0) return 0.0;
    double L = sqrt(L2);
    double u[3] = {d[0] / L, d[1] / L, d[2] / L};
    double q[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
    double t0 = dot3(q, u);
    double e[3] = {q[0] - t0 * u[0], q[1] - t0 * u[1], q[2] - t0 * u[2]};
    double w2 = R * R - dot3(e, e);
    if (w2 <= 0.0) return 0.0;
    double w = sqrt(w2);
    double tau1 = -t0 > -w ? -t0 : -w;
    double tau2 = L - t0 < w ? L - t0 : w;
    if (tau1 >= tau2) return 0.0;
    double R4 = pow(R, 4);
#define ANTI_I(t) (w2 * w2 * (t) - (2.0 / 3.0) * w2 * pow((t), 3) + pow((t), 5) / 5.0)
#define ANTI_M0(t) (w2 * (t) - pow((t), 3) / 3.0)
#define ANTI_M1(t) (w2 * (t) * (t) / 2.0 - pow((t), 4) / 4.0)
#define ANTI_M2(t) (w2 * pow((t), 3) / 3.0 - pow((t), 5) / 5.0)
    double I = (ANTI_I(tau2) - ANTI_I(tau1)) / R4;
    double M0 = ANTI_M0(tau2) - ANTI_M0(tau1);
    double M1 = ANTI_M1(tau2) - ANTI_M1(tau1);
    double M2 = ANTI_M2(tau2) - ANTI_M2(tau1);
#undef ANTI_I
#undef ANTI_M0
#undef ANTI_M1
#undef ANTI_M2
    double ca_u = (1.0 - t0 / L) * M1 - M2 / L, ca_e = (1.0 - t0 / L) * M0 - M1 / L;
    double cb_u = (t0 / L) * M1 + M2 / L, cb_e = (t0 / L) * M0 + M1 / L;
    for (int k = 0; k < 3; ++k) {
        dIda[k] = -u[k] * I / L - (4.0 / R4) * (u[k] * ca_u - e[k] * ca_e);
        dIdb[k] = u[k] * I / L - (4.0 / R4) * (u[k] * cb_u - e[k] * cb_e);
    }
    return I;
}

/*
 * Gradient of the scalar loss L = sum over the listed cells of g_c vf_c with
 * respect to every radius and node position. grad_radius: [n_edges];
 * grad_nodes: [n_nodes][3]; both are overwritten.
 * dL/dSigma(p) = g_c / m^3 * s (1 - s) / T with s = sigmoid((Sigma - C) / T);
 * dSigma/drho_j = I_j(p) dw_j/drho_j; dSigma/da_j = w_j dI_j/da, likewise b.
 */
int orc_vf_backward(const float* nodes, int64_t n_nodes, const int32_t* edges,
                    const float* radius, int64_t n_edges, double R, double C, int mode,
                    double ox, double oy, double oz, double h, int32_t cx, int32_t cy,
                    int32_t cz, int32_t m, double T, const int64_t* cells, const double* g,
                    int64_t n_cells, double* grad_radius, double* grad_nodes)
{
    orc_cells c = {ox, oy, oz, h, cx, cy, cz, m, T};
    int64_t m3 = (int64_t)m * m * m;
    int64_t np = n_cells * m3;
    double* P = cell_samples(&c, cells, n_cells);
    orc_edges E;
    int rc = build_edges(nodes, n_nodes, edges, radius, n_edges, R, C, mode, &E);
    if (rc) { free(P); free_edges(&E); return rc; }
    memset(grad_radius, 0, sizeof(double) * (size_t)n_edges);
    memset(grad_nodes, 0, sizeof(double) * 3 * (size_t)n_nodes);
    /* Gradients with respect to the original endpoints (edges[2j], edges[2j+1]). */
    double* gw = (double*)calloc((size_t)(n_edges ? n_edges : 1), sizeof(double));
    double* ga = (double*)calloc(3 * (size_t)(n_edges ? n_edges : 1), sizeof(double));
    double* gb = (double*)calloc(3 * (size_t)(n_edges ? n_edges : 1), sizeof(double));
    int64_t* ord = (int64_t*)malloc(sizeof(int64_t) * (size_t)(np ? np : 1));
    for (int64_t i = 0; i < np; ++i) ord[i] = i;
    g_pts = P;
    qsort(ord, (size_t)np, sizeof(int64_t), cmp_pt_z);
    orc_active A;
    active_init(&A, 1024);
    for (int64_t t = 0; t < np; ++t) {
        int64_t i = ord[t];
        const double* p = P + 3 * i;
        double gc = g[i / m3];
        if (gc == 0.0) continue;
        active_advance(&A, &E, R, p[2]);
        double S = active_sigma(&A, &E, R, p);
        double s = sigmoid((S - C) / T);
        double alpha = gc / (double)m3 * s * (1.0 - s) / T;
        for (int64_t q = 0; q < A.n; ++q) {
            int64_t j = A.idx[q];
            double pa[3], pb[3], dIda[3], dIdb[3];
            int32_t i0 = edges[2 * j], i1 = edges[2 * j + 1];
            for (int k = 0; k < 3; ++k) {
                pa[k] = (double)nodes[3 * (int64_t)i0 + k];
                pb[k] = (double)nodes[3 * (int64_t)i1 + k];
            }
            double I = orc_segment_integral_grad(p, pa, pb, R, dIda, dIdb);
            if (I == 0.0) continue;
            gw[j] += alpha * I;
            for (int k = 0; k < 3; ++k) {
                ga[3 * j + k] += alpha * E.w[j] * dIda[k];
                gb[3 * j + k] += alpha * E.w[j] * dIdb[k];
            }
        }
    }
    for (int64_t j = 0; j < n_edges; ++j) {
        grad_radius[j] = gw[j] * orc_weight_drho((double)radius[j], R, C, mode);
        int32_t i0 = edges[2 * j], i1 = edges[2 * j + 1];
        for (int k = 0; k < 3; ++k) {
            grad_nodes[3 * (int64_t)i0 + k] += ga[3 * j + k];
            grad_nodes[3 * (int64_t)i1 + k] += gb[3 * j + k];
        }
    }
    free(A.idx);
    free(ord);
    free(gw);
    free(ga);
    free(gb);
    free(P);
    free_edges(&E);
    return 0;
}

/*
 * Central finite differences of L = sum_c g_c vf_c (listed cells), with step
 * hstep, for a list of parameters: kind 0 = radius of edge idx[q]; kind
 * 1..3 = coordinate (kind - 1) of node idx[q]. A perturbation changes only
 * the terms of the edges it touches, so each side of the difference is
 * evaluated as Sigma(p) minus the touched edges' old terms plus their new
 * terms, at every sample of every listed cell.
 */
int orc_vf_fd(const float* nodes, int64_t n_nodes, const int32_t* edges, const float* radius,
              int64_t n_edges, double R, double C, int mode, double ox, double oy, double oz,
              double h, int32_t cx, int32_t cy, int32_t cz, int32_t m, double T,
              const int64_t* cells, const double* g, int64_t n_cells, const int32_t* kind,
              const int64_t* idx, int64_t n_params, double hstep, double* out)
{
    orc_cells c = {ox, oy, oz, h, cx, cy, cz, m, T};
    int64_t m3 = (int64_t)m * m * m;
    int64_t np = n_cells * m3;
    double* P = cell_samples(&c, cells, n_cells);
    double* S = (double*)malloc(sizeof(double) * (size_t)(np ? np : 1));
    int rc = orc_sigma_points(nodes, n_nodes, edges, radius, n_edges, R, C, mode, P, np, S);
    if (rc) { free(P); free(S); return rc; }
    int64_t* touched = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_edges ? n_edges : 1));
    for (int64_t q = 0; q < n_params; ++q) {
        int64_t nt = 0;
        if (kind[q] == 0) touched[nt++] = idx[q];
        else
            for (int64_t j = 0; j < n_edges; ++j)
                if (edges[2 * j] == idx[q] || edges[2 * j + 1] == idx[q]) touched[nt++] = j;
        double Lpm[2] = {0.0, 0.0};
        for (int side = 0; side < 2; ++side) {
            double delta = side == 0 ? hstep : -hstep;
            double acc = 0.0;
            for (int64_t i = 0; i < np; ++i) {
                double gc = g[i / m3];
                if (gc == 0.0) continue;
                const double* p = P + 3 * i;
                double Snew = S[i];
                for (int64_t t = 0; t < nt; ++t) {
                    int64_t j = touched[t];
                    double a[3], b[3];
                    int32_t i0 = edges[2 * j], i1 = edges[2 * j + 1];
                    for (int k = 0; k < 3; ++k) {
                        a[k] = (double)nodes[3 * (int64_t)i0 + k];
                        b[k] = (double)nodes[3 * (int64_t)i1 + k];
                    }
                    double rho = (double)radius[j];
                    double w_old = orc_weight(rho, R, C, mode);
                    Snew -= w_old * orc_segment_integral(p, a, b, R);
                    if (kind[q] == 0) rho += delta;
                    else {
                        if (i0 == idx[q]) a[kind[q] - 1] += delta;
                        if (i1 == idx[q]) b[kind[q] - 1] += delta;
                    }
                    Snew += orc_weight(rho, R, C, mode) * orc_segment_integral(p, a, b, R);
                }
                acc += gc * sigmoid((Snew - C) / T);
            }
            Lpm[side] = acc / (double)m3;
        }
        out[q] = (Lpm[0] - Lpm[1]) / (2.0 * hstep);
    }
    free(touched);
    free(P);
    free(S);
    return 0;
}
