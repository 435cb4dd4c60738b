/*
 * FP64 CPU oracle for USPG/USCG algebraic reconstruction (arXiv 2208.12964).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU path computes.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant generator with the CUDA library: every grid
 * table, geometry formula and update rule is written out here again from the
 * paper.
 *
 * Contents (paper passages in brackets):
 *   - grid tables: ring areas and sector counts [Sec. II.A, Eq. 1], head
 *     recurrence [Sec. II.B, Eq. 2], slabs of the cylindrical grid [Sec. III.C]
 *   - direct tracing of one ray of one view: cylinder crossings [Sec. III.A,
 *     Eq. 3-4], axial planes, radial planes, sorting [Algorithm 1], midpoint
 *     cell assignment [Sec. III.B, Eq. 5-10], length weights
 *   - the view-0 store reused by rotation [Sec. III.B-C], as an in-oracle
 *     check that rotated rows equal directly traced rows
 *   - the first view's segment store of binary coefficients, re-binned to
 *     each view by adding its source angle [Sec. III.B-C, Algorithm 1]
 *   - scans: parallel-beam 2D, fan-beam 2D [Table 1], cone-beam 3D
 *   - MART, ray-sequential and per-view simultaneous, power rule or Eq. 18,
 *     Eq. 19 stopping [Sec. III.D, Eq. 17-19]
 *   - USPG -> Cartesian resampling [Sec. II.B]
 *
 * Readings of the paper taken here (each is listed with its reason in the
 * design notes of the repository):
 *   - sector rule: 6n (the workloads) or 4(2n-1) (Eq. 1) or a custom table
 *   - azimuth is atan2 mapped to [0, 2*pi), with a +1e-12 rad counter-clockwise
 *     nudge before the floor so that a point on a sector boundary belongs to
 *     the sector that starts there (Eq. 8-10)
 *   - Eq. 3 is read as d^2 = |S|^2 - t^2 |S-D'|^2, and the root of Eq. 4 is
 *     formed as (mr - d)(mr + d) to avoid cancellation near tangency
 *   - pieces shorter than 1e-9 of the cell size are dropped before merging
 *   - the closest-approach point of a ray inside the innermost ring is a
 *     crossing (all sectors of ring 0 meet at the axis); splitting a piece
 *     inside one sector changes no coefficient after merging
 *   - weights are piece lengths (LENGTH) or 1 per traversed cell (BINARY,
 *     Sec. III.B); a cell entered twice gets the sum of its pieces
 *
 * Parity status: every function below is pinned by tests against closed
 * forms, brute-force point sampling or values printed in the paper.  The
 * square-ring ordering of the bijective resample rests on a reading, because
 * the figure that fixes it (Fig. 3) is missing from the paper: it is pinned
 * against pixel orders listed by hand from that reading (counter-clockwise
 * from +x) and against azimuth monotonicity, not against the paper itself.
 * The per-view combination of several rays' corrections (geometric mean for
 * the power rule, arithmetic mean for Eq. 18) is likewise a reading: pinned
 * by closed forms of that reading.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_TWO_PI 6.283185307179586 /* 2*pi rounded to double */
#define OR_NUDGE 1e-12              /* counter-clockwise tie-break, radians */
#define OR_MIN_PIECE 1e-9           /* fraction of the cell size */

/* sector rules */
#define OR_SECT_6N 0
#define OR_SECT_4_2N1 1
#define OR_SECT_CUSTOM 2
/* geometries */
#define OR_PARALLEL_2D 0
#define OR_CONE_3D 1
#define OR_FAN_2D 2
/* weight modes */
#define OR_LENGTH 0
#define OR_BINARY 1
/* update rules */
#define OR_POWER 0
#define OR_LINEAR_EQ18 1

typedef struct {
    int32_t n_rings, n_slabs, sector_rule, geometry;
    double r, h, z_min;
    int32_t n_views, n_u, n_v, weight_mode;
    int64_t arc_num, arc_den;
    double du, dv, d_so, d_sd;
    const int32_t *custom_sectors;
    int32_t store_form; /* 0: rows traced per view; 1: view-0 segments re-binned per view (binary) */
} orc_problem;

typedef struct {
    orc_problem p;
    int32_t *ng;        /* sectors per ring, [n_rings] */
    int64_t *head;      /* first cell id of each ring within a slab */
    int64_t cells_slab; /* cells in one slab */
    int64_t n_cells;
    int32_t n_rays;
    double **bcos, **bsin; /* boundary directions of each ring */
    int32_t G;             /* gcd of the sector counts */
    int32_t threads;
} orc_ctx;

static int64_t gcd64(int64_t a, int64_t b)
{
    while (b) {
        int64_t t = a % b;
        a = b;
        b = t;
    }
    return a < 0 ? -a : a;
}

/* ---------------------------------------------------------------- grid --- */

/* Sector count of ring n (1-based).  Eq. 1 gives n_g = 4(2n-1) so that every
 * cell of the polar grid has area pi r^2; the workloads use 6n. */
static int32_t ring_sectors(const orc_problem *p, int32_t n)
{
    if (p->sector_rule == OR_SECT_6N) return 6 * n;
    if (p->sector_rule == OR_SECT_4_2N1) return 4 * (2 * n - 1);
    return p->custom_sectors[n - 1];
}

void orc_destroy(orc_ctx *c)
{
    if (!c) return;
    if (c->bcos) {
        for (int i = 0; i < c->p.n_rings; i++) free(c->bcos[i]);
        free(c->bcos);
    }
    if (c->bsin) {
        for (int i = 0; i < c->p.n_rings; i++) free(c->bsin[i]);
        free(c->bsin);
    }
    free(c->ng);
    free(c->head);
    free(c);
}

orc_ctx *orc_create(const orc_problem *p)
{
    if (p->n_rings < 1 || p->n_slabs < 1 || p->r <= 0.0) return NULL;
    if (p->geometry != OR_PARALLEL_2D && p->geometry != OR_CONE_3D && p->geometry != OR_FAN_2D) return NULL;
    if (p->geometry == OR_CONE_3D && p->h <= 0.0) return NULL;
    if (p->geometry == OR_FAN_2D && (p->n_v != 1 || !(p->d_so > 0.0) || !(p->d_sd > p->d_so))) return NULL;
    if (p->store_form != 0 && (p->store_form != 1 || p->weight_mode != OR_BINARY)) return NULL;
    if (p->n_views < 1 || p->n_u < 1 || p->n_v < 1 || p->arc_den < 1) return NULL;
    orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
    c->p = *p;
    c->threads = 1;
    int N = p->n_rings;
    c->ng = (int32_t *)malloc(sizeof(int32_t) * N);
    c->head = (int64_t *)malloc(sizeof(int64_t) * N);
    /* Eq. 2: H_1 = 0, H_{n+1} = H_n + n_g(n) */
    int64_t h = 0;
    int64_t g = 0;
    for (int n = 1; n <= N; n++) {
        int32_t s = ring_sectors(p, n);
        if (s < 1) {
            orc_destroy(c);
            return NULL;
        }
        c->ng[n - 1] = s;
        c->head[n - 1] = h;
        h += s;
        g = gcd64(g, s);
    }
    c->cells_slab = h;
    c->G = (int32_t)g;
    c->n_cells = h * (int64_t)(p->geometry == OR_CONE_3D ? p->n_slabs : 1);
    c->n_rays = p->n_u * (p->geometry == OR_CONE_3D ? p->n_v : 1);
    /* unit vectors of the radial boundaries: boundary j of ring i is the
     * half-line from the axis at angle 2*pi*j/n_g (numbering starts on +x and
     * runs counter-clockwise, Sec. II.B) */
    c->bcos = (double **)calloc(N, sizeof(double *));
    c->bsin = (double **)calloc(N, sizeof(double *));
    for (int i = 0; i < N; i++) {
        c->bcos[i] = (double *)malloc(sizeof(double) * c->ng[i]);
        c->bsin[i] = (double *)malloc(sizeof(double) * c->ng[i]);
        for (int j = 0; j < c->ng[i]; j++) {
            double a = OR_TWO_PI * (double)j / (double)c->ng[i];
            c->bcos[i][j] = cos(a);
            c->bsin[i][j] = sin(a);
        }
    }
    return c;
}

void orc_set_threads(orc_ctx *c, int32_t n) { c->threads = n < 1 ? 1 : n; }
int64_t orc_cells(const orc_ctx *c) { return c->n_cells; }
int64_t orc_cells_per_slab(const orc_ctx *c) { return c->cells_slab; }
int32_t orc_rays(const orc_ctx *c) { return c->n_rays; }
int32_t orc_gcd(const orc_ctx *c) { return c->G; }

int32_t orc_grid_tables(const orc_ctx *c, int32_t *ng, int64_t *head)
{
    for (int i = 0; i < c->p.n_rings; i++) {
        ng[i] = c->ng[i];
        head[i] = c->head[i];
    }
    return c->p.n_rings;
}

/* ------------------------------------------------------------ geometry --- */

/* View angle in radians.  Views are spread uniformly over the arc
 * arc_num/arc_den turns (Algorithm 1 steps the source by a constant angle);
 * view k sits at k*arc/p. */
static double view_angle(const orc_problem *p, int32_t k)
{
    double frac = (double)((int64_t)k * p->arc_num) / (double)(p->arc_den * (int64_t)p->n_views);
    return OR_TWO_PI * frac;
}

/* Endpoints S (start) and D (end) of ray `ray` of view `k`.
 * Parallel 2D: view 0 has detector axis e_u = (1,0) and rays along +y; bin b
 *   sits at u = (2b - (B-1)) * du/2, and the ray runs from u*e_u - 2R*e_r to
 *   u*e_u + 2R*e_r.
 * Cone 3D: the source is at (-d_so, 0, 0), the flat detector is centred at
 *   (d_sd - d_so, 0, 0) with e_u = (0,1,0), e_v = (0,0,1); pixel (a, c) with
 *   ray index c*n_u + a.
 * Fan 2D (Table 1, 2-D phantoms): the source is at (-d_so, 0), the line
 *   detector is centred at (d_sd - d_so, 0) with e_u = (0,1); bin a sits at
 *   u = (2a - (B-1)) * du/2 and its ray runs from the source to the bin.
 * All three rotate rigidly about z by the view angle (Sec. III.C; Table 1
 * places the source on -x and the detector on +x). */
static void ray_endpoints(const orc_ctx *c, int32_t k, int32_t ray, double S[3], double D[3])
{
    const orc_problem *p = &c->p;
    double th = view_angle(p, k);
    double ct = cos(th), st = sin(th);
    double R = (double)p->n_rings * p->r;
    if (p->geometry == OR_PARALLEL_2D) {
        double u = (double)(2 * ray - (p->n_u - 1)) * (0.5 * p->du);
        double eux = ct, euy = st, erx = -st, ery = ct;
        double L = 2.0 * R;
        S[0] = u * eux - L * erx;
        S[1] = u * euy - L * ery;
        S[2] = 0.0;
        D[0] = u * eux + L * erx;
        D[1] = u * euy + L * ery;
        D[2] = 0.0;
    } else if (p->geometry == OR_FAN_2D) {
        double u = (double)(2 * ray - (p->n_u - 1)) * (0.5 * p->du);
        double off = p->d_sd - p->d_so;
        S[0] = -p->d_so * ct;
        S[1] = -p->d_so * st;
        S[2] = 0.0;
        D[0] = off * ct + u * (-st);
        D[1] = off * st + u * ct;
        D[2] = 0.0;
    } else {
        int32_t a = ray % p->n_u, cc = ray / p->n_u;
        double u = (double)(2 * a - (p->n_u - 1)) * (0.5 * p->du);
        double v = (double)(2 * cc - (p->n_v - 1)) * (0.5 * p->dv);
        double off = p->d_sd - p->d_so;
        S[0] = -p->d_so * ct;
        S[1] = -p->d_so * st;
        S[2] = 0.0;
        D[0] = off * ct + u * (-st);
        D[1] = off * st + u * ct;
        D[2] = v;
    }
}

/* ------------------------------------------------------------- tracing --- */

typedef struct {
    int64_t cell;
    double w;
    double lam; /* entry parameter of the first piece, for a stable order */
} orc_piece;

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

static int cmp_piece(const void *a, const void *b)
{
    const orc_piece *x = (const orc_piece *)a, *y = (const orc_piece *)b;
    if (x->cell != y->cell) return (x->cell > y->cell) - (x->cell < y->cell);
    return (x->lam > y->lam) - (x->lam < y->lam);
}

typedef struct {
    double *lam;
    int64_t n, cap;
} dbuf;

static void dpush(dbuf *b, double v)
{
    if (b->n == b->cap) {
        b->cap = b->cap ? 2 * b->cap : 256;
        b->lam = (double *)realloc(b->lam, sizeof(double) * b->cap);
    }
    b->lam[b->n++] = v;
}

/* Direct trace of one ray of one view, written as the paper's steps:
 * all crossings with the cylinders (Eq. 3-4), the axial planes and the
 * radial planes are collected and sorted by distance to the source
 * (Algorithm 1), each piece between consecutive crossings is assigned to the
 * cell holding its midpoint (Eq. 5-10), and pieces in the same cell are
 * merged.  Output: `cells` ascending, unique; `w` = length (or 1 if binary).
 * Returns the entry count, or -(needed) if `cap` is too small. */
int32_t orc_trace(const orc_ctx *c, int32_t k, int32_t ray, int32_t cap, int64_t *cells, double *w)
{
    const orc_problem *p = &c->p;
    if (k < 0 || k >= p->n_views || ray < 0 || ray >= c->n_rays) return 0;
    const int N = p->n_rings;
    const double r = p->r;
    const double R = (double)N * r;
    const int is3d = p->geometry == OR_CONE_3D;
    double S[3], D[3];
    ray_endpoints(c, k, ray, S, D);
    double dx = D[0] - S[0], dy = D[1] - S[1], dz = D[2] - S[2];
    double L = sqrt(dx * dx + dy * dy + dz * dz);
    double unit = r;
    if (is3d && p->h < unit) unit = p->h;
    const double min_len = OR_MIN_PIECE * unit;

    /* Eq. 3: distance of the XY projection S D' from the axis */
    double ax = S[0], ay = S[1];
    double a = dx * dx + dy * dy; /* <S-D', S-D'> */
    if (a == 0.0) return 0;       /* ray parallel to the axis: not a scan ray */
    double t = -(ax * dx + ay * dy) / a;
    double d2 = (ax * ax + ay * ay) - t * t * a;
    if (d2 < 0.0) d2 = 0.0;
    double d = sqrt(d2);
    if (!(d < R)) return 0; /* misses (or grazes) the cylinder */

    /* Eq. 4: entry and exit of the outer cylinder */
    double kR = sqrt(((R - d) * (R + d)) / a);
    double lo = t - kR, hi = t + kR;
    if (lo < 0.0) lo = 0.0;
    if (hi > 1.0) hi = 1.0;
    /* clip to the slab stack [z_min, z_min + n_slabs*h] */
    if (is3d) {
        double z0 = p->z_min, z1 = p->z_min + (double)p->n_slabs * p->h;
        if (dz == 0.0) {
            if (!(S[2] > z0 && S[2] < z1)) return 0;
        } else {
            double l0 = (z0 - S[2]) / dz, l1 = (z1 - S[2]) / dz;
            if (l0 > l1) {
                double tmp = l0;
                l0 = l1;
                l1 = tmp;
            }
            if (l0 > lo) lo = l0;
            if (l1 < hi) hi = l1;
        }
    }
    if (!(hi > lo)) return 0;

    dbuf X = {0, 0, 0};
    dpush(&X, lo);
    dpush(&X, hi);
    /* cylinders of radius m*r, m = 1..N-1 (the outer one is the clip) */
    for (int m = 1; m < N; m++) {
        double rm = (double)m * r;
        if (!(rm > d)) continue;
        double km = sqrt(((rm - d) * (rm + d)) / a);
        double l1 = t - km, l2 = t + km;
        if (l1 > lo && l1 < hi) dpush(&X, l1);
        if (l2 > lo && l2 < hi) dpush(&X, l2);
    }
    /* axial planes z = z_min + s*h */
    if (is3d && dz != 0.0) {
        for (int s = 1; s < p->n_slabs; s++) {
            double zs = p->z_min + (double)s * p->h;
            double l = (zs - S[2]) / dz;
            if (l > lo && l < hi) dpush(&X, l);
        }
    }
    /* radial planes: boundary j of ring i is the segment from radius i*r to
     * (i+1)*r along direction (cos a_j, sin a_j).  Every boundary of every ring
     * the ray reaches is tested. */
    for (int i = 0; i < N; i++) {
        if (!((double)(i + 1) * r > d)) continue;
        double rin = (double)i * r, rout = (double)(i + 1) * r;
        for (int j = 0; j < c->ng[i]; j++) {
            double cj = c->bcos[i][j], sj = c->bsin[i][j];
            double den = dx * sj - dy * cj;
            if (den == 0.0) continue;
            double num = ax * sj - ay * cj;
            double l = -num / den;
            if (!(l > lo && l < hi)) continue;
            double px = ax + l * dx, py = ay + l * dy;
            double rho = px * cj + py * sj;
            if (rho >= rin && rho <= rout) dpush(&X, l);
        }
    }
    /* all sectors of ring 0 meet on the axis: the closest approach of a ray
     * passing through ring 0 is a crossing */
    if (d < r && t > lo && t < hi) dpush(&X, t);

    qsort(X.lam, X.n, sizeof(double), cmp_double);

    orc_piece *pc = (orc_piece *)malloc(sizeof(orc_piece) * (X.n + 1));
    int64_t np = 0;
    const int32_t NS = is3d ? p->n_slabs : 1;
    for (int64_t q = 0; q + 1 < X.n; q++) {
        double la = X.lam[q], lb = X.lam[q + 1];
        double len = (lb - la) * L;
        if (!(len >= min_len)) continue;
        /* Eq. 5: midpoint of the two crossings */
        double pax = S[0] + la * dx, pay = S[1] + la * dy, paz = S[2] + la * dz;
        double pbx = S[0] + lb * dx, pby = S[1] + lb * dy, pbz = S[2] + lb * dz;
        double mx = 0.5 * (pax + pbx), my = 0.5 * (pay + pby), mz = 0.5 * (paz + pbz);
        /* Eq. 7: ring from the midpoint radius (0-based) */
        double rho = sqrt(mx * mx + my * my);
        int64_t ring = (int64_t)floor(rho / r);
        if (ring < 0) ring = 0;
        if (ring > N - 1) ring = N - 1;
        /* Eq. 6: slab from the midpoint height */
        int64_t slab = 0;
        if (is3d) {
            slab = (int64_t)floor((mz - p->z_min) / p->h);
            if (slab < 0) slab = 0;
            if (slab > NS - 1) slab = NS - 1;
        }
        /* Eq. 8-10: azimuth -> sector -> cell id */
        int32_t ng = c->ng[ring];
        double phi = atan2(my, mx);
        if (phi < 0.0) phi += OR_TWO_PI;
        int64_t sec = (int64_t)floor(((phi + OR_NUDGE) * (double)ng) / OR_TWO_PI);
        if (sec >= ng) sec -= ng;
        if (sec < 0) sec = 0;
        pc[np].cell = slab * c->cells_slab + c->head[ring] + sec;
        pc[np].w = len;
        pc[np].lam = la;
        np++;
    }
    free(X.lam);
    qsort(pc, np, sizeof(orc_piece), cmp_piece);
    /* merge pieces of the same cell (a ray can enter a ring cell twice) */
    int64_t n = 0;
    for (int64_t q = 0; q < np; q++) {
        if (n > 0 && pc[q].cell == pc[n - 1].cell) {
            pc[n - 1].w += pc[q].w;
            continue;
        }
        pc[n++] = pc[q];
    }
    if (n > cap) {
        free(pc);
        return (int32_t)-n;
    }
    for (int64_t q = 0; q < n; q++) {
        cells[q] = pc[q].cell;
        w[q] = p->weight_mode == OR_BINARY ? 1.0 : pc[q].w;
    }
    free(pc);
    return (int32_t)n;
}

/* ------------------------------------------ view-0 segment store (binary) --- */

/* The paper's own store (Sec. III.B-C, Algorithm 1).  With binary
 * coefficients a line needs only its crossings with the cylinders (Eq. 3-4)
 * and the axial planes: between two consecutive crossings it stays in one
 * ring and one slice (Eq. 5-7 at the midpoint), and its cells there are the
 * sectors between the sectors of the segment's two end points (Eq. 8-16).
 * Only the segments of the first view are stored -- ring, slice and the
 * azimuths of the two end points -- and a view at source angle theta adds
 * theta to every stored azimuth.
 *
 * Azimuths are fixed-point turns, 2^64 to the turn, so that adding a view's
 * angle is exact modular arithmetic and the sector of azimuth F in a ring of
 * n_g sectors is floor(F n_g / 2^64).  Readings where the paper is silent:
 *   (1) a line whose closest approach to the axis lies inside ring 0 is cut
 *       there too (its azimuth turns by up to half a turn around it);
 *   (2) segments shorter than the piece threshold are dropped;
 *   (3) an end point on a sector boundary belongs to the sector the segment
 *       occupies next to it, and an end azimuth within 2^-40 turn of a
 *       boundary counts as on it, so that rounding noise in the azimuth of a
 *       crossing that lies on a boundary decides nothing; a segment of a line
 *       through the axis keeps one azimuth (taken at its midpoint) and the
 *       counter-clockwise nudge decides a boundary, as for pieces;
 *   (4) a cell that two segments share (the two halves of a ring around the
 *       line's dip, or the two sides of the ring-0 cut) is one active cell;
 *   (5) rounding cannot reverse a segment: an end azimuth that lies behind
 *       the start in the direction of turn is moved onto the start.
 * Pieces at a segment's end that are shorter than the threshold are dropped
 * by the direct trace but counted here: the two forms differ only where a
 * sector boundary passes within 1e-9 of a cell of a crossing. */

static uint64_t fixed_turns(double phi) /* phi in [0, 2 pi) */
{
    double t = phi / OR_TWO_PI;
    if (!(t >= 0.0) || t >= 1.0) t = 0.0;
    return (uint64_t)(t * 18446744073709551616.0);
}

static uint64_t azimuth_fixed(double x, double y)
{
    double phi = atan2(y, x);
    if (phi < 0.0) phi += OR_TWO_PI;
    return fixed_turns(phi);
}

/* Source angle of view k in fixed-point turns, floor(k arc 2^64 / p), exact. */
uint64_t orc_view_turns(const orc_ctx *c, int32_t k)
{
    const orc_problem *p = &c->p;
    int64_t den = p->arc_den * (int64_t)p->n_views;
    int64_t num = ((int64_t)k * p->arc_num) % den;
    return (uint64_t)((((unsigned __int128)num) << 64) / (unsigned __int128)den);
}

#define OR_SNAP_TURNS_LOG2 24 /* 2^24 fixed units = 2^-40 turn */

static int64_t sector_at(uint64_t F, int32_t ng) /* floor(F n_g / 2^64), lines through the axis */
{
    return (int64_t)(((unsigned __int128)F * (uint64_t)ng) >> 64);
}

/* Sector of an end azimuth F of a segment whose azimuth turns in direction
 * dir (+1 / -1); `start` tells which end.  The sector is floor(F n_g / 2^64)
 * unless F lies on (or within 2^-40 turn of) a boundary: then the one the
 * segment occupies next to that boundary. */
static int64_t end_sector(uint64_t F, int32_t ng, int dir, int start)
{
    unsigned __int128 prod = (unsigned __int128)F * (uint64_t)ng;
    int64_t j = (int64_t)(prod >> 64);
    uint64_t frac = (uint64_t)prod; /* position inside sector j, 2^-64 units */
    uint64_t tau = ((uint64_t)ng) << OR_SNAP_TURNS_LOG2;
    int below = frac < tau;         /* on boundary j */
    int above = frac > ~tau;        /* on boundary j+1 */
    int up = (dir > 0) == (start != 0); /* the segment lies above the boundary */
    if (below && !up) j -= 1;
    if (above && up) j += 1;
    j %= ng;
    return j < 0 ? j + ng : j;
}

/* First sector (*ja) and number of further sectors of a segment with end
 * azimuths A -> B turning in direction dir.  A segment narrower than twice
 * the boundary window has one cell, the sector of its start. */
static int64_t seg_span(uint64_t A, uint64_t B, int32_t ng, int dir, int64_t *ja_out)
{
    int64_t ja = end_sector(A, ng, dir, 1);
    if (ja_out) *ja_out = ja;
    uint64_t ext = dir > 0 ? B - A : A - B;
    if (ext < (2ull << OR_SNAP_TURNS_LOG2)) return 0;
    int64_t jb = end_sector(B, ng, dir, 0);
    int64_t span = dir > 0 ? jb - ja : ja - jb;
    return span < 0 ? span + ng : span;
}

/* Segments of ray `ray` of the first view, in path order: ring, slice, end
 * azimuths (fixed turns) and length; *dir = +1 / -1 when the azimuth grows /
 * falls along the line, 0 for a line through the axis.  Returns the count,
 * or -(needed) if `cap` is too small. */
int32_t orc_segments(const orc_ctx *c, int32_t ray, int32_t cap, int32_t *ring, int32_t *slab, uint64_t *fa,
                     uint64_t *fb, double *len, int32_t *dir)
{
    const orc_problem *p = &c->p;
    *dir = 0;
    if (ray < 0 || ray >= c->n_rays) return 0;
    const int N = p->n_rings;
    const double r = p->r;
    const double R = (double)N * r;
    const int is3d = p->geometry == OR_CONE_3D;
    double S[3], D[3];
    ray_endpoints(c, 0, ray, S, D);
    double dx = D[0] - S[0], dy = D[1] - S[1], dz = D[2] - S[2];
    double L = sqrt(dx * dx + dy * dy + dz * dz);
    double unit = r;
    if (is3d && p->h < unit) unit = p->h;
    const double min_len = OR_MIN_PIECE * unit;
    double ax = S[0], ay = S[1];
    double a = dx * dx + dy * dy;
    if (a == 0.0) return 0;
    double t = -(ax * dx + ay * dy) / a;
    double d2 = (ax * ax + ay * ay) - t * t * a;
    if (d2 < 0.0) d2 = 0.0;
    double d = sqrt(d2);
    if (!(d < R)) return 0;
    double kR = sqrt(((R - d) * (R + d)) / a);
    double lo = t - kR, hi = t + kR;
    if (lo < 0.0) lo = 0.0;
    if (hi > 1.0) hi = 1.0;
    if (is3d) {
        double z0 = p->z_min, z1 = p->z_min + (double)p->n_slabs * p->h;
        if (dz == 0.0) {
            if (!(S[2] > z0 && S[2] < z1)) return 0;
        } else {
            double l0 = (z0 - S[2]) / dz, l1 = (z1 - S[2]) / dz;
            if (l0 > l1) {
                double tmp = l0;
                l0 = l1;
                l1 = tmp;
            }
            if (l0 > lo) lo = l0;
            if (l1 < hi) hi = l1;
        }
    }
    if (!(hi > lo)) return 0;
    dbuf X = {0, 0, 0};
    dpush(&X, lo);
    dpush(&X, hi);
    for (int m = 1; m < N; m++) { /* cylinders, Eq. 4 */
        double rm = (double)m * r;
        if (!(rm > d)) continue;
        double km = sqrt(((rm - d) * (rm + d)) / a);
        double l1 = t - km, l2 = t + km;
        if (l1 > lo && l1 < hi) dpush(&X, l1);
        if (l2 > lo && l2 < hi) dpush(&X, l2);
    }
    if (is3d && dz != 0.0) { /* axial planes */
        for (int sl = 1; sl < p->n_slabs; sl++) {
            double zs = p->z_min + (double)sl * p->h;
            double l = (zs - S[2]) / dz;
            if (l > lo && l < hi) dpush(&X, l);
        }
    }
    if (d < r && t > lo && t < hi) dpush(&X, t); /* reading (1) */
    qsort(X.lam, X.n, sizeof(double), cmp_double);
    double sigma = ax * dy - ay * dx;
    *dir = sigma > 0.0 ? 1 : (sigma < 0.0 ? -1 : 0);
    int32_t n = 0;
    for (int64_t q = 0; q + 1 < X.n; q++) {
        double la = X.lam[q], lb = X.lam[q + 1];
        double ln = (lb - la) * L;
        if (!(ln >= min_len)) continue; /* reading (2) */
        double pax = S[0] + la * dx, pay = S[1] + la * dy, paz = S[2] + la * dz;
        double pbx = S[0] + lb * dx, pby = S[1] + lb * dy, pbz = S[2] + lb * dz;
        double mx = 0.5 * (pax + pbx), my = 0.5 * (pay + pby), mz = 0.5 * (paz + pbz);
        int64_t rg = (int64_t)floor(sqrt(mx * mx + my * my) / r); /* Eq. 7 */
        if (rg < 0) rg = 0;
        if (rg > N - 1) rg = N - 1;
        int64_t sb = 0;
        if (is3d) { /* Eq. 6 */
            sb = (int64_t)floor((mz - p->z_min) / p->h);
            if (sb < 0) sb = 0;
            if (sb > p->n_slabs - 1) sb = p->n_slabs - 1;
        }
        if (n < cap) {
            ring[n] = (int32_t)rg;
            slab[n] = (int32_t)sb;
            len[n] = ln;
            if (*dir == 0) { /* reading (3): one azimuth */
                fa[n] = fb[n] = azimuth_fixed(mx, my);
            } else {         /* Eq. 8 at both end points */
                fa[n] = azimuth_fixed(pax, pay);
                fb[n] = azimuth_fixed(pbx, pby);
                if ((int64_t)(fb[n] - fa[n]) * *dir < 0) fb[n] = fa[n]; /* reading (5) */
            }
        }
        n++;
    }
    free(X.lam);
    return n <= cap ? n : -n;
}

/* Cells of ray `ray` in view k from the first view's segments (the view loop
 * of Algorithm 1): ascending, unique, weight 1.  Returns the count, or
 * -(needed) if `cap` is too small. */
int32_t orc_rebin_row(const orc_ctx *c, int32_t k, int32_t ray, int32_t cap, int64_t *cells, double *w)
{
    const orc_problem *p = &c->p;
    if (k < 0 || k >= p->n_views) return 0;
    int32_t scap = 2 * p->n_rings + p->n_slabs + 8;
    int32_t *rg = (int32_t *)malloc(sizeof(int32_t) * scap), *sb = (int32_t *)malloc(sizeof(int32_t) * scap);
    uint64_t *fa = (uint64_t *)malloc(sizeof(uint64_t) * scap), *fb = (uint64_t *)malloc(sizeof(uint64_t) * scap);
    double *ln = (double *)malloc(sizeof(double) * scap);
    int32_t dir = 0;
    int32_t ns = orc_segments(c, ray, scap, rg, sb, fa, fb, ln, &dir);
    if (ns < 0) ns = 0; /* cannot happen: at most 2N + slabs + 2 segments */
    uint64_t T = orc_view_turns(c, k), nudge = fixed_turns(OR_NUDGE);
    int64_t total = 0;
    for (int32_t q = 0; q < ns; q++) { /* cells per segment */
        int32_t ng = c->ng[rg[q]];
        if (dir == 0) {
            total += 1;
        } else {
            total += seg_span(fa[q] + T, fb[q] + T, ng, dir, NULL) + 1;
        }
    }
    int64_t *all = (int64_t *)malloc(sizeof(int64_t) * (total ? total : 1));
    int64_t n = 0;
    for (int32_t q = 0; q < ns; q++) {
        int32_t ng = c->ng[rg[q]];
        int64_t base = (int64_t)sb[q] * c->cells_slab + c->head[rg[q]];
        if (dir == 0) {
            all[n++] = base + sector_at(fa[q] + T + nudge, ng);
            continue;
        }
        int64_t ja;
        int64_t span = seg_span(fa[q] + T, fb[q] + T, ng, dir, &ja);
        for (int64_t i = 0; i <= span; i++) {
            int64_t j = ja + dir * i;
            j %= ng;
            if (j < 0) j += ng;
            all[n++] = base + j;
        }
    }
    free(rg);
    free(sb);
    free(fa);
    free(fb);
    free(ln);
    qsort(all, n, sizeof(int64_t), cmp_i64);
    int64_t u = 0; /* reading (4) */
    for (int64_t q = 0; q < n; q++)
        if (u == 0 || all[q] != all[u - 1]) all[u++] = all[q];
    if (u > cap) {
        free(all);
        return (int32_t)-u;
    }
    for (int64_t q = 0; q < u; q++) {
        cells[q] = all[q];
        w[q] = 1.0;
    }
    free(all);
    return (int32_t)u;
}

/* --------------------------------------------- view classes and rotation --- */

/* Rotational reuse of stored rows (Sec. III.B-C, the view loop of Algorithm 1).
 * The grid maps onto itself under a rotation by 1/G turn, G = gcd of the
 * sector counts, which moves every ring by n_g/G sectors.  View k at
 * theta_k = k*arc/p turns is written theta_k = m_k/G + rho_k with
 * m_k = floor(theta_k*G); views with the same residual rho_k share the rows of
 * the first of them (their representative), rotated by (m_k - m_rep)/G turn.
 * Exact integer arithmetic: theta_k*G = k*arc_num*G / (arc_den*p). */
int32_t orc_view_classes(const orc_ctx *c, int32_t *rep_of_view, int32_t *shift_of_view)
{
    const orc_problem *p = &c->p;
    int64_t den = p->arc_den * (int64_t)p->n_views;
    int32_t n_reps = 0;
    for (int32_t k = 0; k < p->n_views; k++) {
        int64_t num = (int64_t)k * p->arc_num * (int64_t)c->G;
        int64_t m = num / den, key = num % den;
        int32_t rep = -1;
        for (int32_t q = 0; q < k; q++) {
            int64_t numq = (int64_t)q * p->arc_num * (int64_t)c->G;
            if (numq % den == key) {
                rep = q;
                break;
            }
        }
        if (rep < 0) {
            rep = k;
            n_reps++;
        }
        int64_t mrep = ((int64_t)rep * p->arc_num * (int64_t)c->G) / den;
        rep_of_view[k] = rep;
        shift_of_view[k] = (int32_t)(m - mrep);
    }
    return n_reps;
}

/* Row of view k rebuilt from its representative's directly traced row: the
 * slab and ring of every entry are kept and the sector moves by
 * shift*n_g/G (mod n_g).  Output sorted by cell id. */
int32_t orc_trace_rotated(const orc_ctx *c, int32_t k, int32_t ray, int32_t cap, int64_t *cells, double *w)
{
    const orc_problem *p = &c->p;
    if (k < 0 || k >= p->n_views) return 0;
    int32_t *rep = (int32_t *)malloc(sizeof(int32_t) * p->n_views);
    int32_t *sh = (int32_t *)malloc(sizeof(int32_t) * p->n_views);
    orc_view_classes(c, rep, sh);
    int32_t rk = rep[k], m = sh[k];
    free(rep);
    free(sh);
    int32_t n = orc_trace(c, rk, ray, cap, cells, w);
    if (n <= 0) return n;
    orc_piece *pc = (orc_piece *)malloc(sizeof(orc_piece) * n);
    for (int32_t q = 0; q < n; q++) {
        int64_t slab = cells[q] / c->cells_slab, rem = cells[q] % c->cells_slab;
        int32_t ring = 0;
        while (ring + 1 < p->n_rings && c->head[ring + 1] <= rem) ring++;
        int64_t sec = rem - c->head[ring];
        int64_t ng = c->ng[ring];
        int64_t shift = ((int64_t)m * ng) / c->G;
        sec = (sec + shift) % ng;
        pc[q].cell = slab * c->cells_slab + c->head[ring] + sec;
        pc[q].w = w[q];
        pc[q].lam = 0.0;
    }
    qsort(pc, n, sizeof(orc_piece), cmp_piece);
    for (int32_t q = 0; q < n; q++) {
        cells[q] = pc[q].cell;
        w[q] = pc[q].w;
    }
    free(pc);
    return n;
}

/* ------------------------------------------------------ system matrix --- */

/* All rows of one view, directly traced (the plain definition of the
 * coefficients alpha_{p,l,v} of Eq. 17). */
typedef struct {
    int64_t *ptr; /* [rays+1] */
    int64_t *cell;
    double *w;
} orc_rows;

static void rows_free(orc_rows *R)
{
    free(R->ptr);
    free(R->cell);
    free(R->w);
}

static int rows_build(const orc_ctx *c, int32_t k, orc_rows *R)
{
    int32_t nr = c->n_rays;
    int32_t *cnt = (int32_t *)calloc(nr, sizeof(int32_t));
    int64_t **cc = (int64_t **)calloc(nr, sizeof(int64_t *));
    double **ww = (double **)calloc(nr, sizeof(double *));
    int fail = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(c->threads)
#endif
    for (int32_t i = 0; i < nr; i++) {
        int32_t cap = 256;
        for (;;) {
            int64_t *cl = (int64_t *)malloc(sizeof(int64_t) * cap);
            double *wl = (double *)malloc(sizeof(double) * cap);
            int32_t n = c->p.store_form == 1 ? orc_rebin_row(c, k, i, cap, cl, wl) : orc_trace(c, k, i, cap, cl, wl);
            if (n >= 0) {
                cnt[i] = n;
                cc[i] = cl;
                ww[i] = wl;
                break;
            }
            free(cl);
            free(wl);
            cap = -n;
        }
    }
    R->ptr = (int64_t *)malloc(sizeof(int64_t) * (nr + 1));
    R->ptr[0] = 0;
    for (int32_t i = 0; i < nr; i++) R->ptr[i + 1] = R->ptr[i] + cnt[i];
    int64_t nnz = R->ptr[nr];
    R->cell = (int64_t *)malloc(sizeof(int64_t) * (nnz ? nnz : 1));
    R->w = (double *)malloc(sizeof(double) * (nnz ? nnz : 1));
    for (int32_t i = 0; i < nr; i++) {
        if (cnt[i]) {
            memcpy(R->cell + R->ptr[i], cc[i], sizeof(int64_t) * cnt[i]);
            memcpy(R->w + R->ptr[i], ww[i], sizeof(double) * cnt[i]);
        }
        free(cc[i]);
        free(ww[i]);
    }
    free(cc);
    free(ww);
    free(cnt);
    return fail;
}

/* Number of nonzeros of view k (directly traced). */
int64_t orc_view_nnz(const orc_ctx *c, int32_t k)
{
    orc_rows R;
    rows_build(c, k, &R);
    int64_t nnz = R.ptr[c->n_rays];
    rows_free(&R);
    return nnz;
}

/* Forward projection of one view: s_l = sum_v alpha_{k,l,v} f_v (Eq. 17). */
void orc_forward(const orc_ctx *c, int32_t k, const double *f, double *s)
{
    orc_rows R;
    rows_build(c, k, &R);
    for (int32_t i = 0; i < c->n_rays; i++) {
        double acc = 0.0;
        for (int64_t q = R.ptr[i]; q < R.ptr[i + 1]; q++) acc += R.w[q] * f[R.cell[q]];
        s[i] = acc;
    }
    rows_free(&R);
}

/* ---------------------------------------------------------------- MART --- */

/* Ray-sequential MART (Sec. III.D).  For each iteration, each view k in
 * order and each ray l in order: P_bar = sum_v alpha f_v (Eq. 17); rays with
 * no cells or P_bar <= 0 are skipped; otherwise every cell on the ray is
 * corrected by
 *   POWER:       f_v *= (P/P_bar)^(lambda * alpha_v / max_v alpha)
 *   LINEAR_EQ18: f_v *= 1 - lambda*(1 - P/P_bar)            (Eq. 18)
 * `proj` is [views][rays]; `f` (in/out) is [cells].  If `tol` > 0 the
 * iteration stops after the first sweep in which every correction satisfies
 * Eq. 19, |f_new - f_old| <= tol*|f_old|.  Returns the sweeps run. */
int32_t orc_mart_sequential(const orc_ctx *c, const float *proj, double *f, int32_t iters, double lambda,
                            int32_t rule, double tol)
{
    const orc_problem *p = &c->p;
    orc_rows *rows = (orc_rows *)malloc(sizeof(orc_rows) * p->n_views);
    for (int32_t k = 0; k < p->n_views; k++) rows_build(c, k, &rows[k]);
    int32_t it;
    for (it = 0; it < iters; it++) {
        int converged = 1;
        for (int32_t k = 0; k < p->n_views; k++) {
            const orc_rows *R = &rows[k];
            for (int32_t i = 0; i < c->n_rays; i++) {
                int64_t b = R->ptr[i], e = R->ptr[i + 1];
                if (b == e) continue;
                double s = 0.0, wmax = 0.0;
                for (int64_t q = b; q < e; q++) {
                    s += R->w[q] * f[R->cell[q]];
                    if (R->w[q] > wmax) wmax = R->w[q];
                }
                if (!(s > 0.0)) continue;
                double ratio = (double)proj[(int64_t)k * c->n_rays + i] / s;
                for (int64_t q = b; q < e; q++) {
                    double old = f[R->cell[q]];
                    double nw;
                    if (rule == OR_LINEAR_EQ18)
                        nw = old * (1.0 - lambda * (1.0 - ratio));
                    else
                        nw = old * pow(ratio, lambda * R->w[q] / wmax);
                    if (tol > 0.0 && fabs(nw - old) > tol * fabs(old)) converged = 0;
                    f[R->cell[q]] = nw;
                }
            }
        }
        if (tol > 0.0 && converged) {
            it++;
            break;
        }
    }
    for (int32_t k = 0; k < p->n_views; k++) rows_free(&rows[k]);
    free(rows);
    return it;
}

/* One per-view simultaneous MART step for view k (Sec. III.D): all ray sums
 * P_bar_l of the view are formed with the current image (Eq. 17), then every
 * cell v met by a ray with P_bar_l > 0 is corrected once, combining the
 * corrections the view's rays l would make one by one:
 *   POWER:       the weighted geometric mean of the ratios,
 *                f_v *= exp(lambda * sum_l alpha_lv ln(P_l/P_bar_l) / sum_l alpha_lv);
 *                a cell met by such a ray with P_l = 0 is set to 0 (the limit
 *                of the same product);
 *   LINEAR_EQ18: the weighted arithmetic mean of the factors of Eq. 18,
 *                f_v *= sum_l alpha_lv (1 - lambda (1 - P_l/P_bar_l)) / sum_l alpha_lv
 *                (lambda is the relaxation beta; P_l = 0 gives 1 - beta).
 * Cells met by no such ray keep their value.  Returns 1 if tol > 0 and some
 * correction breaks Eq. 19, |f_new - f_old| <= tol |f_old|; else 0. */
static int view_step(const orc_ctx *c, const orc_rows *R, int32_t k, const float *proj, double *f,
                     double lambda, int32_t rule, double tol, double *num, double *den, unsigned char *zero)
{
    int32_t nr = c->n_rays;
    memset(num, 0, sizeof(double) * c->n_cells);
    memset(den, 0, sizeof(double) * c->n_cells);
    memset(zero, 0, c->n_cells);
    double *s = (double *)malloc(sizeof(double) * nr);
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(c->threads)
#endif
    for (int32_t i = 0; i < nr; i++) {
        double acc = 0.0;
        for (int64_t q = R->ptr[i]; q < R->ptr[i + 1]; q++) acc += R->w[q] * f[R->cell[q]];
        s[i] = acc;
    }
    for (int32_t i = 0; i < nr; i++) {
        if (R->ptr[i] == R->ptr[i + 1] || !(s[i] > 0.0)) continue;
        double P = (double)proj[(int64_t)k * nr + i];
        if (rule == OR_LINEAR_EQ18) {
            double fac = 1.0 - lambda * (1.0 - P / s[i]);
            for (int64_t q = R->ptr[i]; q < R->ptr[i + 1]; q++) {
                num[R->cell[q]] += R->w[q] * fac;
                den[R->cell[q]] += R->w[q];
            }
            continue;
        }
        if (P == 0.0) {
            for (int64_t q = R->ptr[i]; q < R->ptr[i + 1]; q++) {
                zero[R->cell[q]] = 1;
                den[R->cell[q]] += R->w[q];
            }
            continue;
        }
        double lr = log(P / s[i]);
        for (int64_t q = R->ptr[i]; q < R->ptr[i + 1]; q++) {
            num[R->cell[q]] += R->w[q] * lr;
            den[R->cell[q]] += R->w[q];
        }
    }
    int moved = 0;
    for (int64_t v = 0; v < c->n_cells; v++) {
        if (!(den[v] > 0.0)) continue;
        double old = f[v], nw;
        if (rule == OR_LINEAR_EQ18)
            nw = old * (num[v] / den[v]);
        else if (zero[v])
            nw = 0.0;
        else
            nw = old * exp(lambda * num[v] / den[v]);
        if (tol > 0.0 && fabs(nw - old) > tol * fabs(old)) moved = 1;
        f[v] = nw;
    }
    free(s);
    return moved;
}

/* Per-view simultaneous MART: up to `iters` sweeps over the views in the
 * order `order` (NULL = 0..p-1), each view one step of view_step with the
 * update `rule`.  If tol > 0 the iteration stops after the first sweep in
 * which every correction satisfies Eq. 19.  Rows are traced once per view per
 * sweep.  Returns the sweeps run. */
int32_t orc_mart_per_view(const orc_ctx *c, const float *proj, double *f, int32_t iters, double lambda,
                          const int32_t *order, int32_t rule, double tol)
{
    const orc_problem *p = &c->p;
    double *num = (double *)malloc(sizeof(double) * c->n_cells);
    double *den = (double *)malloc(sizeof(double) * c->n_cells);
    unsigned char *zero = (unsigned char *)malloc(c->n_cells);
    int32_t it;
    for (it = 0; it < iters; it++) {
        int moved = 0;
        for (int32_t q = 0; q < p->n_views; q++) {
            int32_t k = order ? order[q] : q;
            orc_rows R;
            rows_build(c, k, &R);
            moved |= view_step(c, &R, k, proj, f, lambda, rule, tol, num, den, zero);
            rows_free(&R);
        }
        if (tol > 0.0 && !moved) {
            it++;
            break;
        }
    }
    free(num);
    free(den);
    free(zero);
    return it;
}

/* Same as orc_mart_per_view but over the views listed in `views` only, one
 * sweep; used to time a bounded sample of a large workload. */
int64_t orc_mart_views_sample(const orc_ctx *c, const float *proj, double *f, const int32_t *views, int32_t nv,
                              double lambda)
{
    double *num = (double *)malloc(sizeof(double) * c->n_cells);
    double *den = (double *)malloc(sizeof(double) * c->n_cells);
    unsigned char *zero = (unsigned char *)malloc(c->n_cells);
    int64_t nnz = 0;
    for (int32_t q = 0; q < nv; q++) {
        orc_rows R;
        rows_build(c, views[q], &R);
        nnz += R.ptr[c->n_rays];
        view_step(c, &R, views[q], proj, f, lambda, OR_POWER, 0.0, num, den, zero);
        rows_free(&R);
    }
    free(num);
    free(den);
    free(zero);
    return nnz;
}

/* ------------------------------------------------------------ resample --- */

/* Point sampling (Sec. II.B): each Cartesian pixel of an nx-by-ny image
 * covering [-R, R]^2 takes the value of the USPG cell holding its centre
 * (ring from the radius, sector from the azimuth with the same tie rule as
 * the tracing); pixels outside the disk are 0.  x grows with the column,
 * y with the row.  out is [slabs][ny][nx]. */
void orc_resample_point(const orc_ctx *c, const double *f, int32_t nx, int32_t ny, double *out)
{
    const orc_problem *p = &c->p;
    const int32_t NS = p->geometry == OR_CONE_3D ? p->n_slabs : 1;
    double R = (double)p->n_rings * p->r;
    for (int32_t s = 0; s < NS; s++)
        for (int32_t b = 0; b < ny; b++)
            for (int32_t a = 0; a < nx; a++) {
                double x = -R + ((double)a + 0.5) * (2.0 * R / (double)nx);
                double y = -R + ((double)b + 0.5) * (2.0 * R / (double)ny);
                double rho = sqrt(x * x + y * y);
                double v = 0.0;
                if (rho < R) {
                    int64_t ring = (int64_t)floor(rho / p->r);
                    if (ring > p->n_rings - 1) ring = p->n_rings - 1;
                    int32_t ng = c->ng[ring];
                    double phi = atan2(y, x);
                    if (phi < 0.0) phi += OR_TWO_PI;
                    int64_t sec = (int64_t)floor(((phi + OR_NUDGE) * (double)ng) / OR_TWO_PI);
                    if (sec >= ng) sec -= ng;
                    v = f[(int64_t)s * c->cells_slab + c->head[ring] + sec];
                }
                out[((int64_t)s * ny + b) * nx + a] = v;
            }
}

typedef struct {
    double ang;
    int64_t pix;
} orc_apix;

static int cmp_apix(const void *a, const void *b)
{
    const orc_apix *x = (const orc_apix *)a, *y = (const orc_apix *)b;
    return (x->ang > y->ang) - (x->ang < y->ang);
}

/* One-to-one map for 4(2n-1) grids (Sec. II.A-B): square ring C_n of a
 * 2N-by-2N Cartesian grid (pixels whose centre has Chebyshev radius n - 1/2
 * in pixel units) has 8n-4 pixels, as many as ring R_n has cells.  Reading
 * of the missing Fig. 3: both are numbered counter-clockwise from the +x
 * axis, so the j-th pixel of C_n in azimuth order takes cell H_n + j.
 * Returns -1 unless the grid uses the 4(2n-1) rule.  out is
 * [slabs][2N][2N]. */
int32_t orc_resample_bijection(const orc_ctx *c, const double *f, double *out)
{
    const orc_problem *p = &c->p;
    int32_t N = p->n_rings;
    for (int32_t n = 1; n <= N; n++)
        if (c->ng[n - 1] != 8 * n - 4) return -1;
    const int32_t NS = p->geometry == OR_CONE_3D ? p->n_slabs : 1;
    int32_t W = 2 * N;
    int64_t *cell_of_pix = (int64_t *)malloc(sizeof(int64_t) * W * W);
    orc_apix *buf = (orc_apix *)malloc(sizeof(orc_apix) * (8 * N));
    for (int32_t n = 1; n <= N; n++) {
        int32_t cnt = 0;
        for (int32_t b = 0; b < W; b++)
            for (int32_t a = 0; a < W; a++) {
                double x = (double)a - (double)N + 0.5, y = (double)b - (double)N + 0.5;
                double cheb = fabs(x) > fabs(y) ? fabs(x) : fabs(y);
                if (cheb != (double)n - 0.5) continue;
                double ang = atan2(y, x);
                if (ang < 0.0) ang += OR_TWO_PI;
                buf[cnt].ang = ang;
                buf[cnt].pix = (int64_t)b * W + a;
                cnt++;
            }
        qsort(buf, cnt, sizeof(orc_apix), cmp_apix);
        for (int32_t j = 0; j < cnt; j++) cell_of_pix[buf[j].pix] = c->head[n - 1] + j;
    }
    for (int32_t s = 0; s < NS; s++)
        for (int64_t q = 0; q < (int64_t)W * W; q++)
            out[(int64_t)s * W * W + q] = f[(int64_t)s * c->cells_slab + cell_of_pix[q]];
    free(buf);
    free(cell_of_pix);
    return 0;
}
