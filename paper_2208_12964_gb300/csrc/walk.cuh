// Ray walk of the FP64 coefficient generator (Sec. III.A-C), shared by the
// generator kernels.  Host+device so the same walk can be exercised on a CPU
// when diagnosing a kernel; the library itself runs it only on the GPU.
#pragma once

#include "internal.cuh"

#include <cstring>

#ifdef __CUDACC__
#define USPG_HD __host__ __device__
#else
#define USPG_HD
#endif

namespace uspg {

// a < b for finite FP64 values of which at least one is non-negative (the
// line parameters the walk compares: segment ends and accepted crossings lie
// in [0, 1], candidates may be negative, the sentinel is 2): the order of
// the IEEE bit patterns as signed integers, an integer compare instead of an
// FP64 one (GB300's FP64 pipe is the walk's bottleneck).
USPG_HD inline bool lt(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __double_as_longlong(a) < __double_as_longlong(b);
#else
    long long x, y;
    memcpy(&x, &a, sizeof x);
    memcpy(&y, &b, sizeof y);
    return x < y;
#endif
}

USPG_HD inline void flag(int *status, int bit)
{
#ifdef __CUDA_ARCH__
    atomicOr(status, bit);
#else
    *status |= bit;
#endif
}

USPG_HD inline void ray_endpoints(const Geometry &g, int k, int ray, double S[3], double D[3])
{
    double frac = (double)((long long)k * g.arc_num) / (double)(g.arc_den * (long long)g.n_views);
    double th = kTwoPi * frac;
    double ct = cos(th), st = sin(th);
    if (g.geometry == USPG_PARALLEL_2D) {
        double R = (double)g.n_rings * g.r;
        double u = (double)(2 * ray - (g.n_u - 1)) * (0.5 * g.du);
        double eux = ct, euy = st, erx = -st, ery = ct;
        double L = 2.0 * R;
        S[0] = u * eux - L * erx;
        S[1] = u * euy - L * ery;
        S[2] = 0.0;
        D[0] = u * eux + L * erx;
        D[1] = u * euy + L * ery;
        D[2] = 0.0;
    } else if (g.geometry == USPG_FAN_2D) {
        // fan (Table 1): source on -x, line detector on +x, bin along +y
        double u = (double)(2 * ray - (g.n_u - 1)) * (0.5 * g.du);
        double off = g.d_sd - g.d_so;
        S[0] = -g.d_so * ct;
        S[1] = -g.d_so * st;
        S[2] = 0.0;
        D[0] = off * ct + u * (-st);
        D[1] = off * st + u * ct;
        D[2] = 0.0;
    } else {
        int a = ray % g.n_u, c = ray / g.n_u;
        double u = (double)(2 * a - (g.n_u - 1)) * (0.5 * g.du);
        double v = (double)(2 * c - (g.n_v - 1)) * (0.5 * g.dv);
        double off = g.d_sd - g.d_so;
        S[0] = -g.d_so * ct;
        S[1] = -g.d_so * st;
        S[2] = 0.0;
        D[0] = off * ct + u * (-st);
        D[1] = off * st + u * ct;
        D[2] = v;
    }
}

// Per-ray tracing state shared by the segment walks.
struct Ray {
    double S[3], dx, dy, dz, L, a, t, d, lo, hi, min_len, sigma;
    // 1 / a and 1 / dz (0 when dz = 0): the circle roots and the axial-plane
    // parameters of the ray multiply by these instead of dividing per crossing
    double inv_a, inv_dz;
    // FP32 copies for the fast classification: closest approach point C of
    // the XY projection (z at the same parameter) and the direction
    float cx, cy, cz, fdx, fdy, fdz;
    float inv_r, inv_h, zmin, Rf, fS, fD;
    // error bounds of the FP32 estimates (set by ray_setup): midpoint x, y;
    // and the margins, in units of the floored quantity, inside which a ring
    // or slab index is left to the exact FP64 rule
    float exy, mr, mz;
};

// The FP32 estimate of a ring, slab or sector index is trusted only when
// its floor lies farther from an integer than twice the estimate's error
// bound (per ray, from the magnitudes of the FP32 operands; see ray_setup);
// otherwise the exact FP64 rule decides.  kMaxMargin caps the sector margin
// (a larger error sends the piece to the exact rule).
constexpr float kMaxMargin = 0.25f;
constexpr float kEps32 = 6.0e-8f;  // 2^-24, unit roundoff of FP32

// Repeated cells.  The walk emits pieces in ray order, so the pieces of one
// cell are adjacent -- except for a cell of ring j that the ray leaves
// inward and re-enters outward across the dip into the inner rings.  During
// the inbound half the sink records, per ring, the last cell it emitted in
// that ring (in_cell); during the outbound half a piece whose cell equals the
// record of its ring is merged into that entry.  Slivers next to a circle
// crossing that the midpoint rule puts in the neighbouring ring are
// adjacent (in ray order) to the piece they belong with.
struct CountSink {
    int n = 0;
    int tied = 0;  // some piece's decision lies in a tie band (classify_exact)
    uint32_t last = 0xffffffffu;
    bool outbound = false;
    uint32_t *in_cell = nullptr;
    double *root = nullptr;  // per-ring scratch: circle roots of the inbound half
    USPG_HD void emit(uint32_t cell, double)
    {
        if (n > 0 && cell == last) return;
        int j = cell_ring(cell);
        last = cell;
        if (outbound) {
            if (in_cell[j] == cell) return;
        } else {
            in_cell[j] = cell;
        }
        n++;
    }
};

struct FillSink {
    uint32_t *idx;
    double *w;
    int n = 0;
    int tied = 0;  // some piece's decision lies in a tie band (classify_exact)
    int cap = 0;
    uint32_t last = 0xffffffffu;
    int last_pos = -1;
    int overflow = 0;
    bool outbound = false;
    uint32_t *in_cell = nullptr;
    int *in_pos = nullptr;
    double *root = nullptr;
    USPG_HD void emit(uint32_t cell, double len)
    {
        if (last_pos >= 0 && cell == last) {
            w[last_pos] += len;
            return;
        }
        int j = cell_ring(cell);
        last = cell;
        if (outbound && in_cell[j] == cell) {
            last_pos = in_pos[j];
            w[last_pos] += len;
            return;
        }
        if (n >= cap) {
            overflow = 1;
            last_pos = -1;
            return;
        }
        idx[n] = cell;
        w[n] = len;
        last_pos = n;
        if (!outbound) {
            in_cell[j] = cell;
            in_pos[j] = n;
        }
        n++;
    }
};

// A piece whose sector decision lies this close (in sector widths) to a
// boundary, or whose midpoint lies this close (in ring widths) to the axis,
// where its azimuth is ill-conditioned, makes its row "tied": the mirror
// image of the row (transverse symmetry, generator.cu) is then traced
// directly instead of derived, because the tie rule (counter-clockwise
// nudge) does not commute with a reflection.  The bands are far wider than
// the nudge and than the FP64 rounding of the two geometries.
constexpr double kTieSector = 1e-7;
constexpr double kTieAxis = 1e-3;

// Exact classification of the piece [la, lb] (Eq. 5-10): FP64 midpoint of
// the two crossings, ring = floor(rho / r), slab = floor((z - z_min) / h),
// sector = floor((atan2 + nudge) n_g / 2 pi).  *tied (optional) is set when
// the decision lies within the tie bands above.
USPG_HD inline uint32_t classify_exact(const Geometry &g, const RingEntry *rt, const Ray &R, double la, double lb,
                                       int *tied = nullptr)
{
    double pax = R.S[0] + la * R.dx, pay = R.S[1] + la * R.dy, paz = R.S[2] + la * R.dz;
    double pbx = R.S[0] + lb * R.dx, pby = R.S[1] + lb * R.dy, pbz = R.S[2] + lb * R.dz;
    double mx = 0.5 * (pax + pbx), my = 0.5 * (pay + pby), mz = 0.5 * (paz + pbz);
    double rho = sqrt(mx * mx + my * my);
    long long ring = (long long)floor(rho / g.r);
    if (ring < 0) ring = 0;
    if (ring > g.n_rings - 1) ring = g.n_rings - 1;
    long long slab = 0;
    if (g.geometry == USPG_CONE_3D) {
        slab = (long long)floor((mz - g.z_min) / g.h);
        if (slab < 0) slab = 0;
        if (slab > g.n_slabs - 1) slab = g.n_slabs - 1;
    }
    int ng = rt[ring].ng;
    double phi = atan2(my, mx);
    if (phi < 0.0) phi += kTwoPi;
    double xs = ((phi + kNudge) * (double)ng) / kTwoPi;
    long long sec = (long long)floor(xs);
    if (tied) {
        double fr = xs - (double)sec;
        if (fr < kTieSector || fr > 1.0 - kTieSector || rho < kTieAxis * g.r) *tied = 1;
    }
    if (sec >= ng) sec -= ng;
    if (sec < 0) sec = 0;
    return pack_cell((int)slab, (int)ring, (int)sec);
}

// Same decision from an FP32 estimate of the midpoint; returns false when any
// of the three floors lies within twice its error bound of an integer (or the
// point is too close to the axis for its azimuth to be trusted), so that the
// caller takes the exact path.  Where it returns true it agrees with
// classify_exact.
USPG_HD inline bool classify_fast(const Geometry &g, const RingEntry *rt, const Ray &R, double la, double lb,
                                  uint32_t *out)
{
    float dl = (float)(0.5 * (la + lb) - R.t);
    float mx = R.cx + dl * R.fdx, my = R.cy + dl * R.fdy;
    float rho = sqrtf(mx * mx + my * my);
    float rr = rho * R.inv_r;
    float fr = floorf(rr);
    if (rr - fr < R.mr || rr - fr > 1.0f - R.mr) return false;
    int ring = (int)fr;
    if (ring > g.n_rings - 1) return false;
    int slab = 0;
    if (g.geometry == USPG_CONE_3D) {
        float zz = (R.cz + dl * R.fdz - R.zmin) * R.inv_h;
        float fz = floorf(zz);
        if (zz - fz < R.mz || zz - fz > 1.0f - R.mz) return false;
        slab = (int)fz;
        if (slab < 0 || slab > g.n_slabs - 1) return false;
    }
    int ng = rt[ring].ng;
    // azimuth error: the midpoint's position error over rho, plus atan2f's
    // and the scaling's roundoff, in sector units
    float scale = (float)ng * 0.15915494f;
    float mphi = 2.0f * ((1.5f * R.exy / rho + 4.0f * kEps32 * 6.2831853f) * scale + 4.0f * kEps32 * (float)ng);
    if (!(mphi < kMaxMargin)) return false;  // close to the axis
    float phi = atan2f(my, mx);
    if (phi < 0.0f) phi += 6.2831853f;
    float x = phi * scale;
    float fx = floorf(x);
    if (x - fx < mphi || x - fx > 1.0f - mphi) return false;
    int sec = (int)fx;
    if (sec >= ng) sec -= ng;
    if (sec < 0 || sec >= ng) return false;
    *out = pack_cell(slab, ring, sec);
    return true;
}

// Emit the piece [la, lb] unless it is a sliver.
template <class Sink>
USPG_HD inline void piece(const Geometry &g, const RingEntry *rt, const Ray &R, double la, double lb, Sink &sink)
{
    double len = (lb - la) * R.L;
    if (lt(len, R.min_len)) return;
    uint32_t cell;
    // the fast rule decides only at least ~3e-6 sector widths from a boundary
    // and away from the axis: only exact decisions can be tied
    if (!classify_fast(g, rt, R, la, lb, &cell)) cell = classify_exact(g, rt, R, la, lb, &sink.tied);
    sink.emit(cell, len);
}

// Axial-plane crossings of the whole ray, in ascending parameter order.  The
// candidates are the planes between the slabs of the ray's clipped ends, one
// extra on each side against the rounding of the floors; the ring segments
// come in ascending order and each takes the candidates strictly inside it,
// so every plane's parameter is formed once per ray.
struct ZStream {
    int s, s_end, step;  // candidate plane indices
    double next;         // parameter of the current candidate (2 when none is left)
    USPG_HD void init(const Geometry &g, const Ray &R, double sa, double sb)
    {
        next = 2.0;
        if (g.geometry != USPG_CONE_3D || R.dz == 0.0) {
            s = 0;
            s_end = 0;
            step = 1;
            return;
        }
        double za = R.S[2] + sa * R.dz, zb = R.S[2] + sb * R.dz;
        int ia = (int)floor((za - g.z_min) / g.h), ib = (int)floor((zb - g.z_min) / g.h);
        if (R.dz > 0.0) {
            s = ia;
            s_end = ib + 2;
            step = 1;
        } else {
            s = ia + 1;
            s_end = ib - 1;
            step = -1;
        }
        // candidates can only lie in [0, n_slabs]; keep the loop bounded
        int span = (s_end - s) * step;
        if (!(span >= 0 && span <= g.n_slabs + 3)) {
            s = 0;
            s_end = 0;
        }
    }
    // the next candidate plane (interior planes 1 .. n_slabs-1 only)
    USPG_HD void advance(const Geometry &g, const Ray &R)
    {
        next = 2.0;
        while (s != s_end) {
            int cs = s;
            s += step;
            if (cs < 1 || cs > g.n_slabs - 1) continue;
            double zs = g.z_min + (double)cs * g.h;
            next = (zs - R.S[2]) * R.inv_dz;
            return;
        }
    }
};

// Radial-plane crossings of ring i inside (sa, sb), ascending, for i >= 1:
// candidates are the boundaries between the azimuths of the segment ends
// (one extra on each side), each accepted by the exact test.
struct RStream {
    long long j, j_end;
    int dir, i, ng, head;
    double rin, rout, next;
    float da, db;
    USPG_HD void init(const Geometry &g, const RingEntry *rt, const Ray &R, int ring, double sa, double sb)
    {
        i = ring;
        ng = rt[ring].ng;
        head = rt[ring].head;
        rin = (double)ring * g.r;
        rout = (double)(ring + 1) * g.r;
        next = 2.0;
        da = (float)(sa - R.t);
        db = (float)(sb - R.t);
        float fa = atan2f(R.cy + da * R.fdy, R.cx + da * R.fdx), fb = atan2f(R.cy + db * R.fdy, R.cx + db * R.fdx);
        if (fa < 0.0f) fa += 6.2831853f;
        if (fb < 0.0f) fb += 6.2831853f;
        float scale = (float)ng * 0.15915494f;
        if (R.sigma > 0.0) {  // azimuth grows along the ray
            if (fb < fa) fb += 6.2831853f;
            j = (long long)floor(fa * scale);
            j_end = (long long)floor(fb * scale) + 2;
            dir = 1;
        } else if (R.sigma < 0.0) {
            if (fb > fa) fb -= 6.2831853f;
            j = (long long)floor(fa * scale) + 1;
            j_end = (long long)floor(fb * scale) - 1;
            dir = -1;
        } else {  // the ray meets the axis: the segment is radial
            j = (long long)floor(fa * scale) - 1;
            j_end = j + 3;
            dir = 1;
        }
        // at most one lap of candidates (plus the margins)
        long long span = (j_end - j) * dir;
        if (!(span >= 0 && span <= (long long)ng + 3)) {
            j = 0;
            j_end = ng;
            dir = 1;
        }
    }
    USPG_HD void advance(const Ray &R, const double2 *bdir, const float2 *bdirf, double sa, double sb)
    {
        next = 2.0;
        while (j != j_end) {
            long long jj = j % ng;
            if (jj < 0) jj += ng;
            j += dir;
            float2 ef = bdirf[head + jj];
            // FP32 pre-test in closest-approach coordinates (delta = lambda - t):
            // skip candidates whose crossing is clearly outside the segment or
            // off the ring's boundary segment before forming the FP64 root.
            // The error of dc is below 1e-6 (R + |dc| |d|) / |den| + 1e-6 |dc|
            // (FP32 inputs accurate to 2^-23); the tests use twice that.
            float denf = R.fdx * ef.y - R.fdy * ef.x;
            float dc = -(R.cx * ef.y - R.cy * ef.x) / denf;
            float tol = 2e-6f * ((R.Rf + fabsf(dc) * R.fD) / fabsf(denf) + fabsf(dc)) + 1e-6f;
            if (!(dc > da - tol && dc < db + tol)) continue;
            float rhof = (R.cx + dc * R.fdx) * ef.x + (R.cy + dc * R.fdy) * ef.y;
            float tolr = R.fD * tol + 2e-6f * R.Rf;
            if (!(rhof >= (float)rin - tolr && rhof <= (float)rout + tolr)) continue;
            double2 e = bdir[head + jj];
            double cj = e.x, sj = e.y;
            double den = R.dx * sj - R.dy * cj;
            if (den == 0.0) continue;
            double num = R.S[0] * sj - R.S[1] * cj;
            double l = -num / den;
            if (!(lt(sa, l) && lt(l, sb))) continue;
            bool inside = rhof >= (float)rin + tolr && rhof <= (float)rout - tolr;
            if (!inside) {  // near a vertex: the exact test decides
                double px = R.S[0] + l * R.dx, py = R.S[1] + l * R.dy;
                double rho = px * cj + py * sj;
                inside = rho >= rin && rho <= rout;
            }
            if (inside) {
                next = l;
                return;
            }
        }
    }
};

// Walk the ring-i segment [sa, sb] (already clipped) and emit its pieces.
template <class Sink>
USPG_HD void walk_segment(const Geometry &g, const RingEntry *rt, const double2 *bdir, const float2 *bdirf, const Ray &R, int ring,
                             double sa, double sb, ZStream &zs, Sink &sink, int *status)
{
    if (!(sb > sa)) return;
    while (!lt(sa, zs.next)) zs.advance(g, R);  // planes of earlier segments, or on their common end
    double prev = sa;
    if (ring == 0) {
        // all sectors of ring 0 meet on the axis: test every boundary and the
        // closest-approach point, then sort the few accepted crossings
        double xs[kMaxRing0Cross];
        int nx = 0;
        int ng = rt[0].ng;
        double rout = g.r;
        for (int jj = 0; jj < ng; jj++) {
            double2 e = bdir[jj];
            double den = R.dx * e.y - R.dy * e.x;
            if (den == 0.0) continue;
            double num = R.S[0] * e.y - R.S[1] * e.x;
            double l = -num / den;
            if (!(l > sa && l < sb)) continue;
            double px = R.S[0] + l * R.dx, py = R.S[1] + l * R.dy;
            double rho = px * e.x + py * e.y;
            if (rho >= 0.0 && rho <= rout) {
                if (nx < kMaxRing0Cross) xs[nx++] = l;
                else flag(status, kStatusRing0Overflow);
            }
        }
        if (R.d < g.r && R.t > sa && R.t < sb) {
            if (nx < kMaxRing0Cross) xs[nx++] = R.t;
            else flag(status, kStatusRing0Overflow);
        }
        for (int q = 1; q < nx; q++) {  // insertion sort
            double v = xs[q];
            int p = q - 1;
            while (p >= 0 && xs[p] > v) {
                xs[p + 1] = xs[p];
                p--;
            }
            xs[p + 1] = v;
        }
        int q = 0;
        for (;;) {
            double rn = q < nx ? xs[q] : 2.0;
            bool take_r = !lt(zs.next, rn);
            double nxt = take_r ? rn : zs.next;
            if (!lt(nxt, sb)) break;
            if (lt(prev, nxt)) {
                piece(g, rt, R, prev, nxt, sink);
                prev = nxt;
            }
            if (take_r) q++;
            else zs.advance(g, R);
        }
    } else {
        RStream rs;
        rs.init(g, rt, R, ring, sa, sb);
        rs.advance(R, bdir, bdirf, sa, sb);
        for (;;) {
            bool take_r = !lt(zs.next, rs.next);  // rs.next <= zs.next
            double nxt = take_r ? rs.next : zs.next;
            if (!lt(nxt, sb)) break;
            if (lt(prev, nxt)) {
                piece(g, rt, R, prev, nxt, sink);
                prev = nxt;
            }
            if (take_r) rs.advance(R, bdir, bdirf, sa, sb);
            else zs.advance(g, R);
        }
    }
    if (lt(prev, sb)) piece(g, rt, R, prev, sb, sink);
}

// half-chord parameter of the circle of radius m r: sqrt((m r)^2 - d^2) / |d|
// in units of the ray parameter, with the differences taken before the
// product (Eq. 4; the form that stays accurate near tangency)
USPG_HD inline double root_k(double m, double r, double d, double inv_a)
{
    double rm = m * r;
    return sqrt(((rm - d) * (rm + d)) * inv_a);
}

// Full walk of one ray: set-up per Eq. 3-4, then ring segments.
// Eq. 3-4 set-up of one ray: closest approach t, distance d, clip [lo, hi].
// Returns false if the ray misses the grid.  *m0 = smallest m >= 1 with
// m r > d (rings m0 .. N-1 are crossed twice, ring m0-1 is the deepest).
USPG_HD inline bool ray_setup(const Geometry &g, int view, int ray, Ray &R, double &kR, int &m0)
{
    double D[3];
    ray_endpoints(g, view, ray, R.S, D);
    R.dx = D[0] - R.S[0];
    R.dy = D[1] - R.S[1];
    R.dz = D[2] - R.S[2];
    R.L = sqrt(R.dx * R.dx + R.dy * R.dy + R.dz * R.dz);
    double unit = g.r;
    if (g.geometry == USPG_CONE_3D && g.h < unit) unit = g.h;
    R.min_len = kMinPiece * unit;
    double ax = R.S[0], ay = R.S[1];
    R.a = R.dx * R.dx + R.dy * R.dy;
    if (R.a == 0.0) return false;
    R.inv_a = 1.0 / R.a;
    R.inv_dz = R.dz != 0.0 ? 1.0 / R.dz : 0.0;
    R.t = -(ax * R.dx + ay * R.dy) / R.a;
    double d2 = (ax * ax + ay * ay) - R.t * R.t * R.a;
    if (d2 < 0.0) d2 = 0.0;
    R.d = sqrt(d2);
    const int N = g.n_rings;
    double Rc = (double)N * g.r;
    if (!(R.d < Rc)) return false;
    kR = root_k((double)N, g.r, R.d, R.inv_a);
    double lo = R.t - kR, hi = R.t + kR;
    if (lo < 0.0) lo = 0.0;
    if (hi > 1.0) hi = 1.0;
    if (g.geometry == USPG_CONE_3D) {
        double z0 = g.z_min, z1 = g.z_min + (double)g.n_slabs * g.h;
        if (R.dz == 0.0) {
            if (!(R.S[2] > z0 && R.S[2] < z1)) return false;
        } else {
            double l0 = (z0 - R.S[2]) / R.dz, l1 = (z1 - R.S[2]) / R.dz;
            if (l0 > l1) {
                double tmp = l0;
                l0 = l1;
                l1 = tmp;
            }
            if (l0 > lo) lo = l0;
            if (l1 < hi) hi = l1;
        }
    }
    if (!(hi > lo)) return false;
    R.lo = lo;
    R.hi = hi;
    R.sigma = ax * R.dy - ay * R.dx;
    R.cx = (float)(ax + R.t * R.dx);
    R.cy = (float)(ay + R.t * R.dy);
    R.cz = (float)(R.S[2] + R.t * R.dz);
    R.fdx = (float)R.dx;
    R.fdy = (float)R.dy;
    R.fdz = (float)R.dz;
    R.inv_r = (float)(1.0 / g.r);
    R.inv_h = (float)(1.0 / g.h);
    R.zmin = (float)g.z_min;
    R.Rf = (float)Rc;
    R.fS = (float)sqrt(ax * ax + ay * ay);
    R.fD = (float)sqrt(R.a);
    // FP32 midpoint m = c + dl d (|dl| <= 1): roundoff of c, dl, d, the
    // product and the sum is below eps (|c| + 3 |d| + |m|) per coordinate;
    // doubled for the two coordinates and the square root
    R.exy = 2.0f * kEps32 * (2.0f * R.Rf + 3.0f * R.fD);
    float err_r = (R.exy + 2.0f * kEps32 * R.Rf) * R.inv_r + 2.0f * kEps32 * (float)N;
    R.mr = fmaxf(2.0f * err_r, 1e-6f);
    R.mz = 1e-6f;
    if (g.geometry == USPG_CONE_3D) {
        float zext = (float)(fabs(g.z_min) + (double)g.n_slabs * g.h);
        float err_z = 2.0f * kEps32 * (fabsf(R.cz) + 3.0f * fabsf(R.fdz) + 2.0f * zext) * R.inv_h +
                      2.0f * kEps32 * (float)g.n_slabs;
        R.mz = fmaxf(2.0f * err_z, 1e-6f);
    }
    m0 = (int)floor(R.d / g.r) + 1;
    if (m0 < 1) m0 = 1;
    while (m0 > 1 && (double)(m0 - 1) * g.r > R.d) m0--;
    while (m0 <= N && !((double)m0 * g.r > R.d)) m0++;
    return true;
}

template <class Sink>
USPG_HD void walk_ray(const Geometry &g, const RingEntry *rt, const double2 *bdir, const float2 *bdirf, int view,
                      int ray, Sink &sink, int *status)
{
    Ray R;
    double kR;
    int m0;
    if (!ray_setup(g, view, ray, R, kR, m0)) return;
    const int N = g.n_rings;
    const double lo = R.lo, hi = R.hi;
    // Ray order: rings N-1 .. m0 inbound, the deepest ring m0-1, then rings
    // m0 .. N-1 outbound.
    for (int i = 0; i < N; i++) sink.in_cell[i] = 0xffffffffu;
    sink.outbound = false;
    ZStream zs;  // the segments below come in ascending parameter order
    zs.init(g, R, lo, hi);
    zs.advance(g, R);
    // each circle's root is formed once: the inbound half keeps it (in the
    // sink's per-ring scratch) for the outbound half.  One loop over the
    // segments, so the segment walk is compiled once (a smaller kernel).
    const int n_in = N - m0;
    double kout = kR;
    for (int k = 0; k <= 2 * n_in; k++) {
        int ring;
        double sa, sb;
        if (k < n_in) {  // inbound: ring N-1-k
            ring = N - 1 - k;
            double kin = root_k((double)ring, g.r, R.d, R.inv_a);
            sink.root[ring] = kin;
            sa = R.t - kout;
            sb = R.t - kin;
            kout = kin;
        } else if (k == n_in) {  // the deepest ring
            ring = m0 - 1;
            sa = R.t - kout;
            sb = R.t + kout;
        } else {  // outbound: ring m0 + (k - n_in - 1)
            ring = m0 + (k - n_in - 1);
            sink.outbound = true;
            double ki = sink.root[ring], ko = (ring == N - 1) ? kR : sink.root[ring + 1];
            sa = R.t + ki;
            sb = R.t + ko;
        }
        walk_segment(g, rt, bdir, bdirf, R, ring, sa > lo ? sa : lo, sb < hi ? sb : hi, zs, sink, status);
    }
}

// Upper bound on the pieces the FP64 walk can emit for one ray, from an FP32
// walk in closest-approach coordinates (delta = lambda - t) whose crossing
// tests are loosened by more than their rounding error, so that every
// crossing the FP64 walk accepts is counted (possibly twice near a segment
// end).  Pieces per segment <= crossings inside it + 1.
USPG_HD inline int size_segment(const Geometry &g, const RingEntry *rt, const float2 *bdirf, const Ray &R, int ring,
                                float da, float db, bool brute)
{
    if (!(db > da)) return 0;
    int n = 1;
    float rin = (float)((double)ring * g.r), rout = (float)((double)(ring + 1) * g.r);
    int ng = rt[ring].ng, head = rt[ring].head;
    long long j, j_end;
    if (brute) {
        j = 0;
        j_end = ng;
    } else if (R.sigma == 0.0) {
        // the ray meets the axis and the segment is radial: the FP64 walk
        // tests three boundaries around its azimuth (RStream::init), so it
        // accepts at most three radial crossings here
        n += 3;
        j = 0;
        j_end = 0;
    } else {
        float fa = atan2f(R.cy + da * R.fdy, R.cx + da * R.fdx), fb = atan2f(R.cy + db * R.fdy, R.cx + db * R.fdx);
        if (fa < 0.0f) fa += 6.2831853f;
        if (fb < 0.0f) fb += 6.2831853f;
        // the arc the segment sweeps, counter-clockwise from lo_a to hi_a
        float lo_a = R.sigma > 0.0 ? fa : fb, hi_a = R.sigma > 0.0 ? fb : fa;
        if (hi_a < lo_a) hi_a += 6.2831853f;
        float scale = (float)ng * 0.15915494f;
        j = (long long)floorf(lo_a * scale) - 1;
        j_end = (long long)floorf(hi_a * scale) + 2;
        if (j_end - j > ng + 3) {
            j = 0;
            j_end = ng;
        }
    }
    for (long long jj0 = j; jj0 < j_end; jj0++) {
        long long jj = jj0 % ng;
        if (jj < 0) jj += ng;
        float2 ef = bdirf[head + jj];
        float denf = R.fdx * ef.y - R.fdy * ef.x;
        float dc = -(R.cx * ef.y - R.cy * ef.x) / denf;
        float tol = 4e-6f * ((R.Rf + fabsf(dc) * R.fD) / fabsf(denf) + fabsf(dc)) + 2e-6f;
        if (!(dc > da - tol && dc < db + tol)) continue;
        float rhof = (R.cx + dc * R.fdx) * ef.x + (R.cy + dc * R.fdy) * ef.y;
        float tolr = R.fD * tol + 4e-6f * R.Rf;
        if (!(rhof >= rin - tolr && rhof <= rout + tolr)) continue;
        n++;
    }
    if (g.geometry == USPG_CONE_3D && R.fdz != 0.0f) {
        float za = R.cz + da * R.fdz, zb = R.cz + db * R.fdz;
        float z0 = fminf(za, zb), z1 = fmaxf(za, zb);
        float tolz = 4e-6f * (fabsf(R.cz) + fabsf(R.zmin) + fmaxf(fabsf(da), fabsf(db)) * fabsf(R.fdz)) + 1e-6f;
        int s0 = (int)ceilf((z0 - tolz - R.zmin) * R.inv_h - 1e-3f), s1 = (int)floorf((z1 + tolz - R.zmin) * R.inv_h + 1e-3f);
        if (s0 < 1) s0 = 1;
        if (s1 > g.n_slabs - 1) s1 = g.n_slabs - 1;
        if (s1 >= s0) n += s1 - s0 + 1;
    }
    if (ring == 0) n++;  // closest-approach split
    return n;
}

USPG_HD inline int size_ray(const Geometry &g, const RingEntry *rt, const float2 *bdirf, int view, int ray)
{
    Ray R;
    double kR;
    int m0;
    if (!ray_setup(g, view, ray, R, kR, m0)) return 0;
    const int N = g.n_rings;
    float dlo = (float)(R.lo - R.t), dhi = (float)(R.hi - R.t);
    float slack = 1e-6f * (fabsf(dlo) + fabsf(dhi)) + 1e-7f;
    // roots in FP32 from FP64 differences (rm - d) and (rm + d)
    auto kf = [&](int m) -> float {
        double rm = (double)m * g.r;
        return sqrtf((float)(rm - R.d) * (float)(rm + R.d) / (float)R.a);
    };
    int n = 0;
    float kout = (float)kR;
    for (int i = N - 1; i >= m0; i--) {
        float kin = kf(i);
        float a1 = -kout - slack, b1 = -kin + slack, a2 = kin - slack, b2 = kout + slack;
        n += size_segment(g, rt, bdirf, R, i, fmaxf(a1, dlo - slack), fminf(b1, dhi + slack), false);
        n += size_segment(g, rt, bdirf, R, i, fmaxf(a2, dlo - slack), fminf(b2, dhi + slack), false);
        kout = kin;
    }
    int i0 = m0 - 1;
    n += size_segment(g, rt, bdirf, R, i0, fmaxf(-kout - slack, dlo - slack), fminf(kout + slack, dhi + slack),
                      i0 == 0);
    return n + 2;
}

}  // namespace uspg
