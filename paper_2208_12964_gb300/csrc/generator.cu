// K1: FP64 coefficient generator (Sec. III.A-C, Algorithm 1).
//
// One thread traces one ray of one representative view.  The ray is cut at
// its crossings with the ring cylinders (Eq. 3-4, roots formed as
// (mr - d)(mr + d) so near-tangent rays keep their digits), the axial planes
// and the radial planes of the ring it is in; every piece between two
// consecutive crossings goes to the cell that holds its midpoint (Eq. 5-10)
// and pieces shorter than 1e-9 of a cell are dropped.  Unlike a global sort
// of all crossings, the walk visits the ray ring by ring (ring N-1 inbound,
// ring N-1 outbound, ring N-2 inbound, ...) and merges only the crossings of
// one ring segment, so each thread holds O(1) state.  A cell can be entered
// twice only across the dip into the inner rings, and the walk emits the
// last inbound and first outbound pieces of a ring back to back, so merging
// repeated cells needs only the previous entry.
//
// This file is compiled with -fmad=false: the crossings are formed with the
// same separately rounded operations as their definitions so the index lists
// do not depend on contraction.
//
// Passes: count -> scan -> fill (FP64 weights) -> convert to the stored dtype
// -> cell-major store (count per cell, slice widths, scan, scatter, per-cell
// sort by ray id so the layout is deterministic).
#include "internal.cuh"

#include <algorithm>

namespace uspg {

__device__ __forceinline__ void ray_endpoints(const Geometry &g, int k, int ray, double S[3], double D[3])
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
};

struct CountSink {
    int n = 0;
    uint32_t last = 0xffffffffu;
    __device__ void emit(uint32_t cell, double)
    {
        if (n > 0 && cell == last) return;
        last = cell;
        n++;
    }
};

struct FillSink {
    uint32_t *idx;
    double *w;
    int n = 0;
    int cap = 0;
    uint32_t last = 0xffffffffu;
    int overflow = 0;
    __device__ void emit(uint32_t cell, double len)
    {
        if (n > 0 && cell == last) {
            w[n - 1] += len;
            return;
        }
        if (n >= cap) {
            overflow = 1;
            return;
        }
        idx[n] = cell;
        w[n] = len;
        last = cell;
        n++;
    }
};

// Classify the piece [la, lb] by its midpoint (Eq. 5-10) and emit it.
template <class Sink>
__device__ __forceinline__ void piece(const Geometry &g, const RingEntry *rt, const Ray &R, double la, double lb,
                                      Sink &sink)
{
    double len = (lb - la) * R.L;
    if (!(len >= R.min_len)) return;
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
    long long sec = (long long)floor(((phi + kNudge) * (double)ng) / kTwoPi);
    if (sec >= ng) sec -= ng;
    if (sec < 0) sec = 0;
    sink.emit(pack_cell((int)slab, (int)ring, (int)sec), len);
}

// Axial-plane crossings inside (sa, sb), in ascending parameter order.
struct ZStream {
    int s, s_end, step;  // candidate plane indices
    double next;
    __device__ void init(const Geometry &g, const Ray &R, double sa, double sb)
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
    __device__ void advance(const Geometry &g, const Ray &R, double sa, double sb)
    {
        next = 2.0;
        while (s != s_end) {
            int cs = s;
            s += step;
            if (cs < 1 || cs > g.n_slabs - 1) continue;
            double zs = g.z_min + (double)cs * g.h;
            double l = (zs - R.S[2]) / R.dz;
            if (l > sa && l < sb) {
                next = l;
                return;
            }
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
    __device__ void init(const Geometry &g, const RingEntry *rt, const Ray &R, int ring, double sa, double sb)
    {
        i = ring;
        ng = rt[ring].ng;
        head = rt[ring].head;
        rin = (double)ring * g.r;
        rout = (double)(ring + 1) * g.r;
        next = 2.0;
        double xa = R.S[0] + sa * R.dx, ya = R.S[1] + sa * R.dy;
        double xb = R.S[0] + sb * R.dx, yb = R.S[1] + sb * R.dy;
        double fa = atan2(ya, xa), fb = atan2(yb, xb);
        if (fa < 0.0) fa += kTwoPi;
        if (fb < 0.0) fb += kTwoPi;
        double scale = (double)ng / kTwoPi;
        if (R.sigma > 0.0) {  // azimuth grows along the ray
            if (fb < fa) fb += kTwoPi;
            j = (long long)floor(fa * scale);
            j_end = (long long)floor(fb * scale) + 2;
            dir = 1;
        } else if (R.sigma < 0.0) {
            if (fb > fa) fb -= kTwoPi;
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
    __device__ void advance(const Ray &R, const double2 *bdir, double sa, double sb)
    {
        next = 2.0;
        while (j != j_end) {
            long long jj = j % ng;
            if (jj < 0) jj += ng;
            j += dir;
            double2 e = bdir[head + jj];
            double cj = e.x, sj = e.y;
            double den = R.dx * sj - R.dy * cj;
            if (den == 0.0) continue;
            double num = R.S[0] * sj - R.S[1] * cj;
            double l = -num / den;
            if (!(l > sa && l < sb)) continue;
            if (!(l > R.lo && l < R.hi)) continue;
            double px = R.S[0] + l * R.dx, py = R.S[1] + l * R.dy;
            double rho = px * cj + py * sj;
            if (rho >= rin && rho <= rout) {
                next = l;
                return;
            }
        }
    }
};

// Walk the ring-i segment [sa, sb] (already clipped) and emit its pieces.
template <class Sink>
__device__ void walk_segment(const Geometry &g, const RingEntry *rt, const double2 *bdir, const Ray &R, int ring,
                             double sa, double sb, Sink &sink, int *status)
{
    if (!(sb > sa)) return;
    ZStream zs;
    zs.init(g, R, sa, sb);
    zs.advance(g, R, sa, sb);
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
            if (!(l > R.lo && l < R.hi)) continue;
            double px = R.S[0] + l * R.dx, py = R.S[1] + l * R.dy;
            double rho = px * e.x + py * e.y;
            if (rho >= 0.0 && rho <= rout) {
                if (nx < kMaxRing0Cross) xs[nx++] = l;
                else atomicOr(status, kStatusRing0Overflow);
            }
        }
        if (R.d < g.r && R.t > sa && R.t < sb) {
            if (nx < kMaxRing0Cross) xs[nx++] = R.t;
            else atomicOr(status, kStatusRing0Overflow);
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
            double nxt = rn < zs.next ? rn : zs.next;
            if (!(nxt < sb)) break;
            if (nxt > prev) {
                piece(g, rt, R, prev, nxt, sink);
                prev = nxt;
            }
            if (rn <= zs.next) q++;
            else zs.advance(g, R, sa, sb);
        }
    } else {
        RStream rs;
        rs.init(g, rt, R, ring, sa, sb);
        rs.advance(R, bdir, sa, sb);
        for (;;) {
            double nxt = rs.next < zs.next ? rs.next : zs.next;
            if (!(nxt < sb)) break;
            if (nxt > prev) {
                piece(g, rt, R, prev, nxt, sink);
                prev = nxt;
            }
            if (rs.next <= zs.next) rs.advance(R, bdir, sa, sb);
            else zs.advance(g, R, sa, sb);
        }
    }
    if (sb > prev) piece(g, rt, R, prev, sb, sink);
}

__device__ __forceinline__ double root_k(double m, double r, double d, double a)
{
    double rm = m * r;
    return sqrt(((rm - d) * (rm + d)) / a);
}

// Full walk of one ray: set-up per Eq. 3-4, then ring segments.
template <class Sink>
__device__ void walk_ray(const Geometry &g, const RingEntry *rt, const double2 *bdir, int view, int ray, Sink &sink,
                         int *status)
{
    Ray R;
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
    if (R.a == 0.0) return;
    R.t = -(ax * R.dx + ay * R.dy) / R.a;
    double d2 = (ax * ax + ay * ay) - R.t * R.t * R.a;
    if (d2 < 0.0) d2 = 0.0;
    R.d = sqrt(d2);
    const int N = g.n_rings;
    double Rc = (double)N * g.r;
    if (!(R.d < Rc)) return;
    double kR = sqrt(((Rc - R.d) * (Rc + R.d)) / R.a);
    double lo = R.t - kR, hi = R.t + kR;
    if (lo < 0.0) lo = 0.0;
    if (hi > 1.0) hi = 1.0;
    if (g.geometry == USPG_CONE_3D) {
        double z0 = g.z_min, z1 = g.z_min + (double)g.n_slabs * g.h;
        if (R.dz == 0.0) {
            if (!(R.S[2] > z0 && R.S[2] < z1)) return;
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
    if (!(hi > lo)) return;
    R.lo = lo;
    R.hi = hi;
    R.sigma = ax * R.dy - ay * R.dx;
    // deepest ring: m0 = smallest m >= 1 with m r > d
    int m0 = (int)floor(R.d / g.r) + 1;
    if (m0 < 1) m0 = 1;
    while (m0 > 1 && (double)(m0 - 1) * g.r > R.d) m0--;
    while (m0 <= N && !((double)m0 * g.r > R.d)) m0++;
    // rings N-1 .. m0 are crossed twice
    double kout = kR;
    for (int i = N - 1; i >= m0; i--) {
        double kin = root_k((double)i, g.r, R.d, R.a);
        double a1 = R.t - kout, b1 = R.t - kin;
        double a2 = R.t + kin, b2 = R.t + kout;
        walk_segment(g, rt, bdir, R, i, a1 > lo ? a1 : lo, b1 < hi ? b1 : hi, sink, status);
        walk_segment(g, rt, bdir, R, i, a2 > lo ? a2 : lo, b2 < hi ? b2 : hi, sink, status);
        kout = kin;
    }
    int i0 = m0 - 1;
    double a0 = R.t - kout, b0 = R.t + kout;
    walk_segment(g, rt, bdir, R, i0, a0 > lo ? a0 : lo, b0 < hi ? b0 : hi, sink, status);
}

__global__ void k_boundaries(const RingEntry *rt, int n_rings, double2 *bdir)
{
    int i = blockIdx.x;
    if (i >= n_rings) return;
    int ng = rt[i].ng, h = rt[i].head;
    for (int j = threadIdx.x; j < ng; j += blockDim.x) {
        double a = kTwoPi * (double)j / (double)ng;
        bdir[h + j] = make_double2(cos(a), sin(a));
    }
}

__global__ void k_count(Geometry g, const RingEntry *rt, const double2 *bdir, const int *rep_view, int n_reps,
                        int *counts, int *status)
{
    long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long long)n_reps * g.n_rays) return;
    int rep = (int)(gid / g.n_rays), ray = (int)(gid % g.n_rays);
    CountSink sink;
    walk_ray(g, rt, bdir, rep_view[rep], ray, sink, status);
    counts[gid] = sink.n;
}

__global__ void k_fill(Geometry g, const RingEntry *rt, const double2 *bdir, const int *rep_view, int n_reps,
                       const int *counts, const long long *row_ptr, uint32_t *idx, double *w64, int *status)
{
    long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long long)n_reps * g.n_rays) return;
    int rep = (int)(gid / g.n_rays), ray = (int)(gid % g.n_rays);
    long long b = row_ptr[gid], e = row_ptr[gid + 1];
    FillSink sink;
    sink.idx = idx + b;
    sink.w = w64 + b;
    sink.cap = counts[gid];
    walk_ray(g, rt, bdir, rep_view[rep], ray, sink, status);
    if (sink.n != counts[gid] || sink.overflow) atomicOr(status, kStatusCountMismatch);
    for (long long q = b + sink.n; q < e; q++) {  // row padding: cell 0, weight 0
        idx[q] = 0;
        w64[q] = 0.0;
    }
}

// ---- prefix sums (exclusive, int64) -------------------------------------

template <typename T>
__global__ void k_scan_block(const T *in, long long n, int pad, long long *out, long long *block_sums)
{
    __shared__ long long sh[1024];
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long v = 0;
    if (i < n) {
        v = (long long)in[i];
        if (pad > 1) v = (v + pad - 1) / pad * pad;
    }
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < blockDim.x; off <<= 1) {
        long long x = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
        __syncthreads();
        sh[threadIdx.x] += x;
        __syncthreads();
    }
    if (i < n) out[i] = sh[threadIdx.x] - v;  // exclusive
    if (threadIdx.x == blockDim.x - 1) block_sums[blockIdx.x] = sh[threadIdx.x];
}

__global__ void k_scan_add(long long *out, long long n, const long long *block_off, long long *total,
                           const long long *block_sums, int nblocks)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += block_off[blockIdx.x];
    if (i == 0) *total = block_off[nblocks - 1] + block_sums[nblocks - 1];
}

// Exclusive scan of n values (rounded up to `pad`) into out[0..n], out[n] = total.
template <typename T>
static cudaError_t exclusive_scan(const T *in, long long n, int pad, long long *out, cudaStream_t s)
{
    const int B = 1024;
    long long nb = (n + B - 1) / B;
    if (nb == 0) return cudaMemsetAsync(out, 0, sizeof(long long), s);
    long long *sums = nullptr, *offs = nullptr;
    cudaError_t e = cudaMallocAsync(&sums, sizeof(long long) * nb, s);
    if (e) return e;
    e = cudaMallocAsync(&offs, sizeof(long long) * (nb + 1), s);
    if (e) return e;
    k_scan_block<T><<<(unsigned)nb, B, 0, s>>>(in, n, pad, out, sums);
    launch_counter()++;
    if (nb > 1) {
        e = exclusive_scan<long long>(sums, nb, 1, offs, s);
        if (e) return e;
    } else {
        cudaMemsetAsync(offs, 0, sizeof(long long), s);
    }
    k_scan_add<<<(unsigned)nb, B, 0, s>>>(out, n, offs, out + n, sums, (int)nb);
    launch_counter()++;
    cudaFreeAsync(sums, s);
    cudaFreeAsync(offs, s);
    return cudaGetLastError();
}

// ---- stored precision -----------------------------------------------------

template <typename WT>
__device__ __forceinline__ WT to_w(float x);
template <>
__device__ __forceinline__ float to_w<float>(float x) { return x; }
template <>
__device__ __forceinline__ __half to_w<__half>(float x)
{
    __half h = __float2half_rn(x);
    if (x > 0.0f && __half2float(h) == 0.0f) h = __ushort_as_half((unsigned short)1);  // keep w > 0
    return h;
}
template <>
__device__ __forceinline__ __nv_bfloat16 to_w<__nv_bfloat16>(float x)
{
    return __float2bfloat16_rn(x);
}
__device__ __forceinline__ float w_to_f(float x) { return x; }
__device__ __forceinline__ float w_to_f(__half x) { return __half2float(x); }
__device__ __forceinline__ float w_to_f(__nv_bfloat16 x) { return __bfloat162float(x); }

template <typename WT>
__global__ void k_convert(long long n_rows, const long long *row_ptr, const int *counts, const double *w64, int binary,
                         double inv_scale, WT *w, float *rowmax)
{
    long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n_rows) return;
    long long b = row_ptr[row], e = row_ptr[row + 1];
    long long n = counts[row];
    float mx = 0.0f;
    for (long long q = b; q < e; q++) {
        WT v;
        if (q - b < n) {
            double x = binary ? 1.0 : w64[q] * inv_scale;
            v = to_w<WT>((float)x);
        } else {
            v = to_w<WT>(0.0f);
        }
        w[q] = v;
        float fv = w_to_f(v);
        mx = fv > mx ? fv : mx;
    }
    rowmax[row] = mx;
}

// ---- cell-major store -------------------------------------------------------

__device__ __forceinline__ long long rep_cell_slice(const RingEntry *rt, int slices_per_slab, uint32_t pc, int *lane)
{
    int slab = cell_slab(pc), ring = cell_ring(pc), sec = cell_sector(pc);
    *lane = sec & (kSlice - 1);
    return (long long)slab * slices_per_slab + rt[ring].chunk0 + (sec >> 5);
}

__device__ __forceinline__ long long rep_cell_id(const RingEntry *rt, long long cps, uint32_t pc)
{
    return (long long)cell_slab(pc) * cps + rt[cell_ring(pc)].head + cell_sector(pc);
}

__global__ void k_cell_count(const long long *row_ptr, const int *counts, const uint32_t *idx, int n_rays,
                             const RingEntry *rt, long long cps, int *cell_cnt)
{
    long long ray = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= n_rays) return;
    long long b = row_ptr[ray];
    int n = counts[ray];
    for (int q = 0; q < n; q++) atomicAdd(&cell_cnt[rep_cell_id(rt, cps, idx[b + q])], 1);
}

// one warp per slice: width = max count over its 32 cells
__global__ void k_slice_width(const RingEntry *rt, int n_rings, int slices_per_slab, long long n_slices,
                              long long cps, const int *cell_cnt, int *width, uint32_t *meta)
{
    long long sl = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (sl >= n_slices) return;
    int slab = (int)(sl / slices_per_slab);
    int within = (int)(sl % slices_per_slab);
    // ring of this slice: largest ring with chunk0 <= within (binary search)
    int lo = 0, hi = n_rings - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (rt[mid].chunk0 <= within) lo = mid;
        else hi = mid - 1;
    }
    int ring = lo;
    int sec0 = (within - rt[ring].chunk0) * kSlice;
    int sec = sec0 + lane;
    int c = 0;
    if (sec < rt[ring].ng) c = cell_cnt[(long long)slab * cps + rt[ring].head + sec];
    for (int o = 16; o > 0; o >>= 1) c = max(c, __shfl_xor_sync(0xffffffffu, c, o));
    if (lane == 0) {
        width[sl] = c;
        meta[sl] = pack_cell(slab, ring, sec0);
    }
}

template <typename WT>
__global__ void k_cell_scatter(const long long *row_ptr, const int *counts, const uint32_t *idx, const WT *w,
                               int n_rays, const RingEntry *rt, long long cps, int slices_per_slab,
                               const long long *slice_off, int *cell_fill, uint32_t *sray, WT *sw)
{
    long long ray = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= n_rays) return;
    long long b = row_ptr[ray];
    int n = counts[ray];
    for (int q = 0; q < n; q++) {
        uint32_t pc = idx[b + q];
        int lane;
        long long sl = rep_cell_slice(rt, slices_per_slab, pc, &lane);
        int slot = atomicAdd(&cell_fill[rep_cell_id(rt, cps, pc)], 1);
        long long pos = slice_off[sl] + (long long)slot * kSlice + lane;
        sray[pos] = (uint32_t)ray;
        sw[pos] = w[b + q];
    }
}

// one thread per (slice, lane): sort the cell's entries by ray id, pad the rest
template <typename WT>
__global__ void k_cell_finish(long long n_slices, const long long *slice_off, const int *width, const uint32_t *meta,
                              const RingEntry *rt, long long cps, const int *cell_cnt, uint32_t *sray, WT *sw)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long sl = t >> 5;
    int lane = (int)(t & 31);
    if (sl >= n_slices) return;
    uint32_t m = meta[sl];
    int ring = cell_ring(m), sec = cell_sector(m) + lane;
    int n = 0;
    if (sec < rt[ring].ng) n = cell_cnt[(long long)cell_slab(m) * cps + rt[ring].head + sec];
    long long base = slice_off[sl] + lane;
    int W = width[sl];
    for (int q = 1; q < n; q++) {
        uint32_t rv = sray[base + (long long)q * kSlice];
        WT wv = sw[base + (long long)q * kSlice];
        int p = q - 1;
        while (p >= 0 && sray[base + (long long)p * kSlice] > rv) {
            sray[base + (long long)(p + 1) * kSlice] = sray[base + (long long)p * kSlice];
            sw[base + (long long)(p + 1) * kSlice] = sw[base + (long long)p * kSlice];
            p--;
        }
        sray[base + (long long)(p + 1) * kSlice] = rv;
        sw[base + (long long)(p + 1) * kSlice] = wv;
    }
    for (int q = n; q < W; q++) {
        sray[base + (long long)q * kSlice] = 0;
        sw[base + (long long)q * kSlice] = to_w<WT>(0.0f);
    }
}

__global__ void k_set_off(long long *dst, const long long *rel, long long n, long long base)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = base + rel[i] * kSlice;
}

static unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

template <typename WT>
static uspg_status build_typed(uspg_ctx *c, cudaStream_t s)
{
    Geometry g{};
    g.geometry = c->scan.geometry;
    g.n_rings = c->n_rings;
    g.n_slabs = c->n_slabs;
    g.n_u = c->scan.n_u;
    g.n_v = c->scan.n_v;
    g.n_rays = c->n_rays;
    g.n_views = c->scan.n_views;
    g.weight_mode = c->weight_mode;
    g.arc_num = c->scan.arc_num;
    g.arc_den = c->scan.arc_den;
    g.r = c->r;
    g.h = c->h;
    g.z_min = c->z_min;
    g.du = c->scan.du;
    g.dv = c->scan.dv;
    g.d_so = c->scan.src_to_axis;
    g.d_sd = c->scan.src_to_det;
    g.cells_per_slab = c->cells_per_slab;

    const int nreps = c->n_reps;
    const long long nrows = (long long)nreps * c->n_rays;
    const long long n_slices = c->slices_per_rep;
    if (!c->d_row_ptr) {  // geometry-sized buffers, allocated once
        USPG_CUDA(c, cudaMalloc(&c->d_rep_view, sizeof(int) * nreps));
        USPG_CUDA(c, cudaMemcpy(c->d_rep_view, c->rep_view.data(), sizeof(int) * nreps, cudaMemcpyHostToDevice));
        USPG_CUDA(c, cudaMalloc(&c->d_counts, sizeof(int) * (nrows + 1)));
        USPG_CUDA(c, cudaMalloc(&c->d_row_ptr, sizeof(long long) * (nrows + 1)));
        USPG_CUDA(c, cudaMalloc(&c->d_rowmax, sizeof(float) * (nrows + 1)));
        USPG_CUDA(c, cudaMalloc(&c->d_cell_cnt, sizeof(int) * c->n_cells));
        USPG_CUDA(c, cudaMalloc(&c->d_cell_fill, sizeof(int) * c->n_cells));
        USPG_CUDA(c, cudaMalloc(&c->d_rel, sizeof(long long) * (n_slices + 1)));
        USPG_CUDA(c, cudaMalloc(&c->d_slice_off, sizeof(long long) * n_slices * nreps));
        USPG_CUDA(c, cudaMalloc(&c->d_slice_meta, sizeof(uint32_t) * n_slices * nreps));
        USPG_CUDA(c, cudaMalloc(&c->d_slice_width, sizeof(int) * n_slices * nreps));
        c->store_moved = true;
    }
    int *d_rep_view = c->d_rep_view, *d_counts = c->d_counts;

    const int TB = 128;
    k_count<<<nblk(nrows, TB), TB, 0, s>>>(g, c->d_ring, c->d_bdir, d_rep_view, nreps, d_counts, c->d_status);
    launch_counter()++;
    USPG_CUDA(c, cudaGetLastError());
    USPG_CUDA(c, exclusive_scan<int>(d_counts, nrows, kRowPad, c->d_row_ptr, s));
    long long nnz_pad = 0;
    USPG_CUDA(c, cudaMemcpyAsync(&nnz_pad, c->d_row_ptr + nrows, sizeof(long long), cudaMemcpyDeviceToHost, s));
    USPG_CUDA(c, cudaStreamSynchronize(s));

    size_t need = (size_t)nnz_pad + kRowPad;
    if (need > c->cap_idx) {
        cudaFree(c->d_idx);
        cudaFree(c->d_w);
        cudaFree(c->d_w64);
        c->d_idx = nullptr;
        c->d_w = nullptr;
        c->d_w64 = nullptr;
        USPG_CUDA(c, cudaMalloc(&c->d_idx, sizeof(uint32_t) * need));
        USPG_CUDA(c, cudaMalloc(&c->d_w, sizeof(WT) * need));
        USPG_CUDA(c, cudaMalloc(&c->d_w64, sizeof(double) * need));
        c->cap_idx = need;
        c->store_moved = true;
    }
    double *d_w64 = c->d_w64;
    k_fill<<<nblk(nrows, TB), TB, 0, s>>>(g, c->d_ring, c->d_bdir, d_rep_view, nreps, d_counts, c->d_row_ptr,
                                          c->d_idx, d_w64, c->d_status);
    launch_counter()++;
    USPG_CUDA(c, cudaGetLastError());
    k_convert<WT><<<nblk(nrows, 256), 256, 0, s>>>(nrows, c->d_row_ptr, d_counts, d_w64,
                                                   c->weight_mode == USPG_BINARY, 1.0 / c->w_scale, (WT *)c->d_w,
                                                   c->d_rowmax);
    launch_counter()++;
    USPG_CUDA(c, cudaGetLastError());

    // statistics
    std::vector<int> h_counts(nrows);
    USPG_CUDA(c, cudaMemcpyAsync(h_counts.data(), d_counts, sizeof(int) * nrows, cudaMemcpyDeviceToHost, s));
    c->h_row_ptr.resize(nrows + 1);
    USPG_CUDA(c, cudaMemcpyAsync(c->h_row_ptr.data(), c->d_row_ptr, sizeof(long long) * (nrows + 1),
                                 cudaMemcpyDeviceToHost, s));
    USPG_CUDA(c, cudaStreamSynchronize(s));
    long long nnz = 0, maxrow = 0;
    std::vector<long long> rep_nnz(nreps, 0);
    for (long long q = 0; q < nrows; q++) {
        nnz += h_counts[q];
        rep_nnz[q / c->n_rays] += h_counts[q];
        maxrow = std::max<long long>(maxrow, h_counts[q]);
    }
    long long all = 0;
    for (int k = 0; k < c->scan.n_views; k++) all += rep_nnz[c->rep_of_view[k]];
    c->nnz_all_views = all;

    // cell-major store, one representative at a time
    int *d_cell_cnt = c->d_cell_cnt, *d_cell_fill = c->d_cell_fill;
    long long *d_rel = c->d_rel;
    // pass 1: slice widths and absolute offsets
    long long sell = 0;
    for (int rep = 0; rep < nreps; rep++) {
        const long long *rp = c->d_row_ptr + (long long)rep * c->n_rays;
        const int *cn = d_counts + (long long)rep * c->n_rays;
        USPG_CUDA(c, cudaMemsetAsync(d_cell_cnt, 0, sizeof(int) * c->n_cells, s));
        k_cell_count<<<nblk(c->n_rays, 128), 128, 0, s>>>(rp, cn, c->d_idx, c->n_rays, c->d_ring, c->cells_per_slab,
                                                          d_cell_cnt);
        launch_counter()++;
        int *wd = c->d_slice_width + rep * n_slices;
        uint32_t *md = c->d_slice_meta + rep * n_slices;
        k_slice_width<<<nblk(n_slices * 32, 256), 256, 0, s>>>(c->d_ring, c->n_rings, c->slices_per_slab, n_slices,
                                                               c->cells_per_slab, d_cell_cnt, wd, md);
        launch_counter()++;
        USPG_CUDA(c, exclusive_scan<int>(wd, n_slices, 1, d_rel, s));
        k_set_off<<<nblk(n_slices, 256), 256, 0, s>>>(c->d_slice_off + rep * n_slices, d_rel, n_slices, sell);
        launch_counter()++;
        long long tot = 0;
        USPG_CUDA(c, cudaMemcpyAsync(&tot, d_rel + n_slices, sizeof(long long), cudaMemcpyDeviceToHost, s));
        USPG_CUDA(c, cudaStreamSynchronize(s));
        sell += tot * kSlice;
    }
    if ((size_t)(sell + kSlice) > c->cap_sell) {
        cudaFree(c->d_sray);
        cudaFree(c->d_sw);
        c->d_sray = nullptr;
        c->d_sw = nullptr;
        USPG_CUDA(c, cudaMalloc(&c->d_sray, sizeof(uint32_t) * (sell + kSlice)));
        USPG_CUDA(c, cudaMalloc(&c->d_sw, sizeof(WT) * (sell + kSlice)));
        c->cap_sell = sell + kSlice;
        c->store_moved = true;
    }
    // pass 2: scatter each row entry to its cell's column, then sort and pad
    for (int rep = 0; rep < nreps; rep++) {
        const long long *rp = c->d_row_ptr + (long long)rep * c->n_rays;
        const int *cn = d_counts + (long long)rep * c->n_rays;
        const long long *so = c->d_slice_off + rep * n_slices;
        USPG_CUDA(c, cudaMemsetAsync(d_cell_cnt, 0, sizeof(int) * c->n_cells, s));
        USPG_CUDA(c, cudaMemsetAsync(d_cell_fill, 0, sizeof(int) * c->n_cells, s));
        k_cell_count<<<nblk(c->n_rays, 128), 128, 0, s>>>(rp, cn, c->d_idx, c->n_rays, c->d_ring, c->cells_per_slab,
                                                          d_cell_cnt);
        launch_counter()++;
        k_cell_scatter<WT><<<nblk(c->n_rays, 128), 128, 0, s>>>(rp, cn, c->d_idx, (const WT *)c->d_w, c->n_rays,
                                                                c->d_ring, c->cells_per_slab, c->slices_per_slab, so,
                                                                d_cell_fill, c->d_sray, (WT *)c->d_sw);
        launch_counter()++;
        k_cell_finish<WT><<<nblk(n_slices * 32, 256), 256, 0, s>>>(n_slices, so, c->d_slice_width + rep * n_slices,
                                                                   c->d_slice_meta + rep * n_slices, c->d_ring,
                                                                   c->cells_per_slab, d_cell_cnt, c->d_sray,
                                                                   (WT *)c->d_sw);
        launch_counter()++;
        USPG_CUDA(c, cudaGetLastError());
    }
    USPG_CUDA(c, cudaStreamSynchronize(s));
    c->gen.n_reps = nreps;
    c->gen.nnz = nnz;
    c->gen.nnz_pad = nnz_pad;
    c->gen.sell_entries = sell;
    c->gen.max_row = maxrow;
    return USPG_OK;
}

uspg_status build_store(uspg_ctx *c, cudaStream_t s)
{
    if (!c->d_bdir) {
        USPG_CUDA(c, cudaMalloc(&c->d_bdir, sizeof(double2) * c->cells_per_slab));
        k_boundaries<<<c->n_rings, 128, 0, s>>>(c->d_ring, c->n_rings, c->d_bdir);
        launch_counter()++;
        USPG_CUDA(c, cudaGetLastError());
    }
    if (c->dtype == USPG_F16) return build_typed<__half>(c, s);
    if (c->dtype == USPG_BF16) return build_typed<__nv_bfloat16>(c, s);
    return build_typed<float>(c, s);
}

}  // namespace uspg
