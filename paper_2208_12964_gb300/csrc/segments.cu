// The paper's coefficient store for binary weights (Sec. III.B-C, Algorithm 1)
// and the ray-sequential MART that reads it.
//
// With binary coefficients a line needs only its crossings with the ring
// cylinders (Eq. 3-4) and the axial planes: between two consecutive crossings
// it stays in one ring and one slab (Eq. 5-7 at the midpoint), and its cells
// there are the sectors between the sectors of the two end points (Eq. 8-16),
// taken in the direction the azimuth turns along the line.  Only the first
// view's segments are stored -- ring, slab and the azimuths of both ends -- and
// view k adds its source angle to every stored azimuth: one store serves every
// view, whatever its angle.
//
// Azimuths are fixed-point turns (2^64 to the turn), so adding a view's angle
// is exact modular arithmetic and the sector of azimuth F in a ring of n_g
// sectors is floor(F n_g / 2^64), one 64x64 multiply-high.  Readings where the
// paper is silent (the same in the FP64 oracle):
//  - a line whose closest approach to the axis lies inside ring 0 is also cut
//    there (its azimuth turns by up to half a turn around that point);
//  - segments shorter than 1e-9 of a cell are dropped;
//  - an end point on a sector boundary, or within 2^-40 turn of one, belongs
//    to the sector the segment occupies next to it, so the rounding of the
//    azimuth of a crossing that lies on a boundary decides nothing; a segment
//    of a line through the axis has one azimuth (its midpoint's) and the
//    counter-clockwise nudge decides a boundary;
//  - a cell met by two segments (the two halves of a ring around the line's
//    dip, or the two sides of the ring-0 cut) is one active cell: a segment
//    records how many segments back the previous one of its ring and slab is,
//    and drops its first sector when that is the other one's last;
//  - rounding cannot reverse a segment: an end azimuth behind the start in the
//    direction of turn is moved onto the start.
//
// This file is compiled with -fmad=false, like the generator: the crossings
// and end points are the same separately rounded FP64 operations as their
// definitions.
#include "internal.cuh"
#include "walk.cuh"

#include <algorithm>

namespace uspg {

constexpr int kSnapLog2 = 24;  // 2^24 fixed units = 2^-40 turn

__host__ __device__ inline uint64_t fixed_turns(double phi)  // phi in [0, 2 pi)
{
    double t = phi / kTwoPi;
    if (!(t >= 0.0) || t >= 1.0) t = 0.0;
    return (uint64_t)(t * 18446744073709551616.0);
}

__device__ inline uint64_t azimuth_fixed(double x, double y)
{
    double phi = atan2(y, x);
    if (phi < 0.0) phi += kTwoPi;
    return fixed_turns(phi);
}

// segment record: slab (10 b) | ring (10 b) | back (12 b): the previous
// segment of the same ring and slab is `back` segments earlier (0: none)
__host__ __device__ inline uint32_t seg_pack(int slab, int ring, int back)
{
    return (uint32_t(slab) << 22) | (uint32_t(ring) << 12) | uint32_t(back);
}
__host__ __device__ inline int seg_back(uint32_t x) { return int(x & 4095u); }

// Sector of an end azimuth F turning in direction dir; start tells which end
// of the segment F is.  floor(F n_g / 2^64) unless F lies within the window
// of a boundary: then the sector the segment occupies next to it.
__device__ inline int end_sector(uint64_t F, int ng, int dir, bool start)
{
    uint64_t g = (uint64_t)ng;
    long long j = (long long)__umul64hi(F, g);
    uint64_t frac = F * g;  // position inside sector j, 2^-64 units
    uint64_t tau = g << kSnapLog2;
    bool below = frac < tau, above = frac > ~tau;
    bool up = (dir > 0) == start;  // the segment lies above the boundary
    if (below && !up) j -= 1;
    if (above && up) j += 1;
    if (j < 0) j += ng;  // j is in [-1, ng]
    if (j >= ng) j -= ng;
    return (int)j;
}

// First sector and number of further sectors of a segment A -> B; a segment
// narrower than twice the window has one cell.
__device__ inline int seg_span(uint64_t A, uint64_t B, int ng, int dir, int *ja_out)
{
    int ja = end_sector(A, ng, dir, true);
    *ja_out = ja;
    uint64_t ext = dir > 0 ? B - A : A - B;
    if (ext < (2ull << kSnapLog2)) return 0;
    int jb = end_sector(B, ng, dir, false);
    int span = dir > 0 ? jb - ja : ja - jb;
    return span < 0 ? span + ng : span;
}

// Cells of segment q in a view at T fixed turns: base + (ja + dir i) mod ng
// for i = 0 .. n-1 (n = 0 when its only sector is the previous one's).
struct SegCells {
    long long base;
    int ja, n, ng;
};

__device__ inline int wrap(int j, int ng)  // j in (-ng, 2 ng)
{
    if (j < 0) j += ng;
    if (j >= ng) j -= ng;
    return j;
}

// Sectors of segment q before the shared-cell rule: first sector and count.
__device__ inline SegCells seg_range(const uint64_t *fa, const uint64_t *fb, uint32_t x, const RingEntry *rt,
                                     long long cps, long long q, uint64_t T, uint64_t nudge, int dir)
{
    int ring = cell_ring(x), ng = rt[ring].ng;
    SegCells sc;
    sc.ng = ng;
    sc.base = (long long)cell_slab(x) * cps + rt[ring].head;
    int span;
    if (dir == 0) {
        sc.ja = (int)__umul64hi(fa[q] + T + nudge, (uint64_t)ng);
        span = 0;
    } else {
        span = seg_span(fa[q] + T, fb[q] + T, ng, dir, &sc.ja);
    }
    sc.n = span + 1;
    return sc;
}

__device__ inline int seg_end(const SegCells &sc, int dir) { return wrap(sc.ja + dir * (sc.n - 1), sc.ng); }

// The shared-cell rule: the segment's first sector is dropped when it is the
// last sector of the previous segment of its ring and slab (prev_end).
__device__ inline void seg_dedup(SegCells &sc, int dir, int prev_end)
{
    if (prev_end == sc.ja) {
        sc.n -= 1;
        sc.ja = wrap(sc.ja + dir, sc.ng);
    }
}

__device__ inline SegCells seg_cells(const uint64_t *fa, const uint64_t *fb, const uint32_t *rs,
                                     const RingEntry *rt, long long cps, long long q, uint64_t T, uint64_t nudge,
                                     int dir)
{
    uint32_t x = rs[q];
    SegCells sc = seg_range(fa, fb, x, rt, cps, q, T, nudge, dir);
    int back = seg_back(x);
    if (back) seg_dedup(sc, dir, seg_end(seg_range(fa, fb, rs[q - back], rt, cps, q - back, T, nudge, dir), dir));
    return sc;
}

__device__ inline long long seg_cell(const SegCells &sc, int dir, int i)
{
    return sc.base + wrap(sc.ja + dir * i, sc.ng);
}

// ---- generator: the first view's segments ------------------------------------

// One thread per ray of the first view.  Crossings in path order: cylinders
// m = N-1 .. m0 inbound (lambda = t - k_m), the closest approach when it lies
// in ring 0, cylinders m0 .. N-1 outbound (t + k_m), merged with the axial
// planes; every pair of consecutive crossings inside the clipped chord is a
// segment.  Pass 0 counts, pass 1 writes at ptr[ray].
template <int MAXR>
__global__ void __launch_bounds__(128) k_seg_build(Geometry g, int pass, int *counts, const long long *ptr,
                                                   uint64_t *fa, uint64_t *fb, uint32_t *rs, signed char *sdir,
                                                   int *status)
{
    int ray = blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= g.n_rays) return;
    Ray R;
    double kR;
    int m0;
    int n = 0;
    if (!ray_setup(g, 0, ray, R, kR, m0)) {
        if (pass == 0) counts[ray] = 0;
        else sdir[ray] = 0;
        return;
    }
    const int N = g.n_rings;
    const int dir = R.sigma > 0.0 ? 1 : (R.sigma < 0.0 ? -1 : 0);
    const bool is3d = g.geometry == USPG_CONE_3D;
    long long out = pass ? ptr[ray] : 0, end = pass ? ptr[ray + 1] : 0;
    int last[MAXR];  // per ring: (index << 10) | slab of its latest segment, -1 for none
    if (pass)
        for (int i = 0; i < N; i++) last[i] = -1;
    ZStream zs;
    zs.init(g, R, R.lo, R.hi);
    zs.advance(g, R);
    // circle crossings in ascending order: phase 0 inbound m = N-1 .. m0,
    // phase 1 the closest approach (ring 0 only), phase 2 outbound m0 .. N-1
    int phase = 0, m = N - 1;
    auto next_circle = [&]() -> double {
        for (;;) {
            if (phase == 0) {
                if (m < m0) {
                    phase = 1;
                    continue;
                }
                double l = R.t - root_k((double)m, g.r, R.d, R.inv_a);
                m--;
                if (l > R.lo && l < R.hi) return l;
            } else if (phase == 1) {
                phase = 2;
                m = m0;
                if (R.d < g.r && R.t > R.lo && R.t < R.hi) return R.t;
            } else {
                if (m > N - 1) return 2.0;
                double l = R.t + root_k((double)m, g.r, R.d, R.inv_a);
                m++;
                if (l > R.lo && l < R.hi) return l;
            }
        }
    };
    double cnext = next_circle();
    while (zs.next <= R.lo) zs.advance(g, R);
    double prev = R.lo;
    for (;;) {
        double nxt = cnext < zs.next ? cnext : zs.next;
        if (!(nxt < R.hi)) nxt = R.hi;
        double la = prev, lb = nxt;
        if ((lb - la) * R.L >= R.min_len) {
            if (pass) {
                double pax = R.S[0] + la * R.dx, pay = R.S[1] + la * R.dy, paz = R.S[2] + la * R.dz;
                double pbx = R.S[0] + lb * R.dx, pby = R.S[1] + lb * R.dy, pbz = R.S[2] + lb * R.dz;
                double mx = 0.5 * (pax + pbx), my = 0.5 * (pay + pby), mz = 0.5 * (paz + pbz);
                long long ring = (long long)floor(sqrt(mx * mx + my * my) / g.r);  // Eq. 7
                if (ring < 0) ring = 0;
                if (ring > N - 1) ring = N - 1;
                long long slab = 0;
                if (is3d) {  // Eq. 6
                    slab = (long long)floor((mz - g.z_min) / g.h);
                    if (slab < 0) slab = 0;
                    if (slab > g.n_slabs - 1) slab = g.n_slabs - 1;
                }
                uint64_t a, b;
                if (dir == 0) {
                    a = b = azimuth_fixed(mx, my);
                } else {  // Eq. 8 at both ends
                    a = azimuth_fixed(pax, pay);
                    b = azimuth_fixed(pbx, pby);
                    if ((long long)(b - a) * dir < 0) b = a;
                }
                int back = 0;
                int rec = last[ring];
                if (rec >= 0 && (rec & 1023) == (int)slab) back = n - (rec >> 10);
                if (back > 4095) {  // cannot happen: a ray has at most 2N + slabs + 1 segments
                    flag(status, kStatusBounds);
                    back = 0;
                }
                last[ring] = (n << 10) | (int)slab;
                if (out + n < end) {  // the count pass sized the ray's range
                    fa[out + n] = a;
                    fb[out + n] = b;
                    rs[out + n] = seg_pack((int)slab, (int)ring, back);
                }
            }
            n++;
        }
        if (!(nxt < R.hi)) break;
        prev = nxt;
        if (cnext <= zs.next) cnext = next_circle();
        else zs.advance(g, R);
    }
    if (pass == 0) counts[ray] = n;
    else {
        sdir[ray] = (signed char)dir;
        if (ptr[ray] + n != ptr[ray + 1]) flag(status, kStatusCountMismatch);
    }
}

// Cells of every (view, ray): the size of the full matrix the store stands for.
__global__ void k_seg_count_cells(const long long *ptr, const uint64_t *fa, const uint64_t *fb, const uint32_t *rs,
                                  const signed char *sdir, const uint64_t *turns, const RingEntry *rt, int n_rays,
                                  int n_views, uint64_t nudge, unsigned long long *total, unsigned long long *longest)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long cnt = 0;
    if (i < (long long)n_rays * n_views) {
        int view = (int)(i / n_rays), ray = (int)(i % n_rays);
        int dir = sdir[ray];
        for (long long q = ptr[ray]; q < ptr[ray + 1]; q++) cnt += seg_cells(fa, fb, rs, rt, 0, q, turns[view], nudge, dir).n;
    }
    unsigned long long s = cnt, mx = cnt;
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(total, s);
        atomicMax(longest, mx);
    }
}

// One ray of one view, expanded (uspg_get_row).
__global__ void k_seg_row(const long long *ptr, const uint64_t *fa, const uint64_t *fb, const uint32_t *rs,
                          const signed char *sdir, uint64_t T, const RingEntry *rt, long long cps, int ray,
                          uint64_t nudge, long long *cells, int cap, int *count)
{
    int dir = sdir[ray];
    for (long long q = ptr[ray] + threadIdx.x; q < ptr[ray + 1]; q += blockDim.x) {
        SegCells sc = seg_cells(fa, fb, rs, rt, cps, q, T, nudge, dir);
        for (int i = 0; i < sc.n; i++) {
            int k = atomicAdd(count, 1);
            if (k < cap) cells[k] = seg_cell(sc, dir, i);
        }
    }
}

static unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

template <int MAXR>
static void seg_build_launch(unsigned grid, cudaStream_t s, const Geometry &g, int pass, uspg_ctx *c, int *counts)
{
    k_seg_build<MAXR><<<grid, 128, 0, s>>>(g, pass, counts, c->d_seg_ptr, c->d_seg_fa, c->d_seg_fb, c->d_seg_rs,
                                           c->d_seg_dir, c->d_status);
}

static void seg_build(unsigned grid, cudaStream_t s, const Geometry &g, int pass, uspg_ctx *c, int *counts)
{
    if (g.n_rings <= 64) seg_build_launch<64>(grid, s, g, pass, c, counts);
    else if (g.n_rings <= 128) seg_build_launch<128>(grid, s, g, pass, c, counts);
    else if (g.n_rings <= 256) seg_build_launch<256>(grid, s, g, pass, c, counts);
    else if (g.n_rings <= 512) seg_build_launch<512>(grid, s, g, pass, c, counts);
    else seg_build_launch<1024>(grid, s, g, pass, c, counts);
}

static uint64_t view_turns(const uspg_ctx *c, int k)  // floor(k arc 2^64 / p), exact
{
    long long den = c->scan.arc_den * (long long)c->scan.n_views;
    long long num = ((long long)k * c->scan.arc_num) % den;
    return (uint64_t)((((unsigned __int128)num) << 64) / (unsigned __int128)den);
}

void free_segments(uspg_ctx *c)
{
    cudaFree(c->d_seg_ptr);
    cudaFree(c->d_seg_fa);
    cudaFree(c->d_seg_fb);
    cudaFree(c->d_seg_rs);
    cudaFree(c->d_seg_dir);
    cudaFree(c->d_view_turns);
    c->d_seg_ptr = nullptr;
    c->d_seg_fa = c->d_seg_fb = nullptr;
    c->d_seg_rs = nullptr;
    c->d_seg_dir = nullptr;
    c->d_view_turns = nullptr;
}

uspg_status build_segments(uspg_ctx *c, cudaStream_t s)
{
    Geometry g = make_geometry(c);
    const int nr = c->n_rays, nv = c->scan.n_views;
    free_segments(c);
    c->store_moved = true;
    int *counts = nullptr;
    USPG_CUDA(c, cudaMalloc(&counts, sizeof(int) * (nr + 1)));
    USPG_CUDA(c, cudaMalloc(&c->d_seg_ptr, sizeof(long long) * (nr + 1)));
    USPG_CUDA(c, cudaMalloc(&c->d_seg_dir, sizeof(signed char) * nr));
    USPG_CUDA(c, cudaMalloc(&c->d_view_turns, sizeof(uint64_t) * nv));
    std::vector<uint64_t> turns(nv);
    for (int k = 0; k < nv; k++) turns[k] = view_turns(c, k);
    USPG_CUDA(c, cudaMemcpyAsync(c->d_view_turns, turns.data(), sizeof(uint64_t) * nv, cudaMemcpyHostToDevice, s));
    seg_build(nblk(nr, 128), s, g, 0, c, counts);
    launch_counter()++;
    USPG_CUDA(c, cudaGetLastError());
    USPG_CUDA(c, scan_counts(counts, nr, c->d_seg_ptr, s));
    long long total = 0;
    USPG_CUDA(c, cudaMemcpyAsync(&total, c->d_seg_ptr + nr, sizeof(long long), cudaMemcpyDeviceToHost, s));
    USPG_CUDA(c, cudaStreamSynchronize(s));
    size_t n = (size_t)std::max<long long>(total, 1);
    USPG_CUDA(c, cudaMalloc(&c->d_seg_fa, sizeof(uint64_t) * n));
    USPG_CUDA(c, cudaMalloc(&c->d_seg_fb, sizeof(uint64_t) * n));
    USPG_CUDA(c, cudaMalloc(&c->d_seg_rs, sizeof(uint32_t) * n));
    seg_build(nblk(nr, 128), s, g, 1, c, counts);
    launch_counter()++;
    USPG_CUDA(c, cudaGetLastError());
    // size of the full matrix the store stands for, and the longest row
    unsigned long long *acc = nullptr;
    USPG_CUDA(c, cudaMallocAsync(&acc, 2 * sizeof(unsigned long long), s));
    USPG_CUDA(c, cudaMemsetAsync(acc, 0, 2 * sizeof(unsigned long long), s));
    k_seg_count_cells<<<nblk((long long)nr * nv, 256), 256, 0, s>>>(c->d_seg_ptr, c->d_seg_fa, c->d_seg_fb,
                                                                    c->d_seg_rs, c->d_seg_dir, c->d_view_turns,
                                                                    c->d_ring, nr, nv, fixed_turns(kNudge), acc,
                                                                    acc + 1);
    launch_counter()++;
    USPG_CUDA(c, cudaGetLastError());
    unsigned long long h[2] = {0, 0};
    USPG_CUDA(c, cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
    USPG_CUDA(c, cudaFreeAsync(acc, s));
    std::vector<int> hc(nr);
    USPG_CUDA(c, cudaMemcpyAsync(hc.data(), counts, sizeof(int) * nr, cudaMemcpyDeviceToHost, s));
    USPG_CUDA(c, cudaStreamSynchronize(s));
    cudaFree(counts);
    c->n_segments = total;
    c->max_segments = hc.empty() ? 0 : *std::max_element(hc.begin(), hc.end());
    c->nnz_all_views = (long long)h[0];
    c->gen = GenOut{};
    c->gen.n_reps = 1;
    c->gen.nnz = total;
    c->gen.max_row = (long long)h[1];
    return USPG_OK;
}

uspg_status segment_row(uspg_ctx *c, int view, int ray, std::vector<long long> &cells)
{
    int cap = 4096, *d_cnt = nullptr;
    long long *d_cells = nullptr;
    for (int attempt = 0; attempt < 2; attempt++) {
        USPG_CUDA(c, cudaMalloc(&d_cells, sizeof(long long) * cap));
        USPG_CUDA(c, cudaMalloc(&d_cnt, sizeof(int)));
        USPG_CUDA(c, cudaMemset(d_cnt, 0, sizeof(int)));
        k_seg_row<<<1, 32>>>(c->d_seg_ptr, c->d_seg_fa, c->d_seg_fb, c->d_seg_rs, c->d_seg_dir, view_turns(c, view),
                             c->d_ring, c->cells_per_slab, ray, fixed_turns(kNudge), d_cells, cap, d_cnt);
        launch_counter()++;
        int n = 0;
        cudaError_t e = cudaMemcpy(&n, d_cnt, sizeof(int), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && n <= cap) {
            cells.resize(n);
            e = cudaMemcpy(cells.data(), d_cells, sizeof(long long) * n, cudaMemcpyDeviceToHost);
        }
        cudaFree(d_cells);
        cudaFree(d_cnt);
        USPG_CUDA(c, e);
        if (n <= cap) {
            std::sort(cells.begin(), cells.end());
            return USPG_OK;
        }
        cap = n;
    }
    return fail(c, USPG_EDEVICE, "segment row grew between expansions");
}

// ---- ray-sequential MART over the segment store ---------------------------------

// Image placement as in the representative-store kernel: all in shared
// memory, the outer rings in shared memory and the inner disk in global
// memory, or all in global memory.
enum { kSegGlobal = 0, kSegSmem = 1, kSegSplit = 2 };

// One warp walks iterations -> views -> rays in order (the paper's line
// order).  Per ray the lanes take its segments in turn (slot c of lane l is
// segment 32 c + l) and enumerate their sectors in the view (source angle
// added to the stored azimuths); each segment's last sector goes to shared
// memory so that the segment after it in the same ring and slab can apply the
// shared-cell rule, and the first kSegSlots sector ranges of every lane stay
// in registers for the update.  The lanes sum the image over the cells (Eq. 17
// with unit coefficients) and after the warp sum correct every cell by
// (P/Pbar)^lambda or 1 - lambda (1 - P/Pbar) (Eq. 18).
constexpr int kSegSlots = 8;  // segments per lane held in registers (rays of up to 256 segments)
constexpr int kSegUnroll = 4;  // cells of a segment read together (most segments have 1-3)

// Sum of the image over a segment's cells: kSegUnroll independent loads at a time.
template <class Img>
__device__ __forceinline__ float seg_sum(const SegCells &sc, int dir, const Img &F)
{
    float acc = 0.0f;
    for (int t0 = 0; t0 < sc.n; t0 += kSegUnroll) {
        float v[kSegUnroll];
#pragma unroll
        for (int u = 0; u < kSegUnroll; u++) v[u] = t0 + u < sc.n ? *F(seg_cell(sc, dir, t0 + u)) : 0.0f;
#pragma unroll
        for (int u = 0; u < kSegUnroll; u++) acc += v[u];
    }
    return acc;
}

template <int MODE>
__global__ void __launch_bounds__(32) k_seq_seg(const long long *__restrict__ ptr, const uint64_t *__restrict__ fa,
                                                const uint64_t *__restrict__ fb, const uint32_t *__restrict__ rs,
                                                const signed char *__restrict__ sdir,
                                                const uint64_t *__restrict__ turns, const RingEntry *__restrict__ rt,
                                                const float *__restrict__ proj, float *f_g, long long n_cells,
                                                long long cps, int n_views, int n_rays, int iters, float lambda,
                                                int rule, float tol, uint64_t nudge, long long n_sm, int *sweeps_out)
{
    extern __shared__ float4 smem4[];
    float *sm = (float *)smem4;
    const int lane = threadIdx.x;
    const long long lo = MODE == kSegSmem ? 0 : (MODE == kSegSplit ? n_cells - n_sm : n_cells);
    int *ends = (int *)(sm + (MODE == kSegGlobal ? 0 : ((n_cells - lo + 3) & ~3LL)));  // [segments of a ray]
    for (long long q = lo + lane; q < n_cells; q += 32) sm[q - lo] = f_g[q];
    __syncwarp();
    auto F = [&](long long cell) -> float * { return cell >= lo ? sm + (cell - lo) : f_g + cell; };
    int it = 0;
    for (; it < iters; it++) {
        int changed = 0;
        for (int k = 0; k < n_views; k++) {
            const uint64_t T = turns[k];
            const float *pk = proj + (long long)k * n_rays;
            long long nb = ptr[0], ne = ptr[1];
            int ndir = sdir[0];
            float np = pk[0];
            for (int ray = 0; ray < n_rays; ray++) {
                long long b = nb, e = ne;
                int dir = ndir;
                float p = np;
                if (ray + 1 < n_rays) {  // bounds, turn and projection of the next ray in flight
                    nb = e;
                    ne = ptr[ray + 2];
                    ndir = sdir[ray + 1];
                    np = pk[ray + 1];
                }
                if (e == b) continue;
                const int ns = (int)(e - b);
                SegCells reg[kSegSlots];
                int bk[kSegSlots];  // shared-cell links of the slots
                // sector ranges; each segment's last sector for the shared-cell rule
#pragma unroll
                for (int c = 0; c < kSegSlots; c++) {
                    int i = c * 32 + lane;
                    bk[c] = 0;
                    if (i < ns) {
                        long long q = b + i;
                        uint32_t x = rs[q];
                        bk[c] = seg_back(x);
                        reg[c] = seg_range(fa, fb, x, rt, cps, q, T, nudge, dir);
                        ends[i] = seg_end(reg[c], dir);
                    }
                }
                for (int i = kSegSlots * 32 + lane; i < ns; i += 32) {
                    long long q = b + i;
                    ends[i] = seg_end(seg_range(fa, fb, rs[q], rt, cps, q, T, nudge, dir), dir);
                }
                __syncwarp();
                float acc = 0.0f;
#pragma unroll
                for (int c = 0; c < kSegSlots; c++) {
                    int i = c * 32 + lane;
                    if (i < ns) {
                        if (bk[c]) seg_dedup(reg[c], dir, ends[i - bk[c]]);
                        acc += seg_sum(reg[c], dir, F);
                    }
                }
                for (int i = kSegSlots * 32 + lane; i < ns; i += 32) {
                    long long q = b + i;
                    uint32_t x = rs[q];
                    SegCells sc = seg_range(fa, fb, x, rt, cps, q, T, nudge, dir);
                    if (seg_back(x)) seg_dedup(sc, dir, ends[i - seg_back(x)]);
                    acc += seg_sum(sc, dir, F);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (acc > 0.0f && p >= 0.0f && p <= 3.402823466e38f) {  // a bad projection changes nothing
                    float ratio = p / acc;
                    float fac = rule == USPG_LINEAR_EQ18 ? 1.0f - lambda * (1.0f - ratio) : powf(ratio, lambda);
                    auto upd = [&](const SegCells &sc) {
                        for (int t0 = 0; t0 < sc.n; t0 += kSegUnroll) {
                            float *fp[kSegUnroll];
                            float old[kSegUnroll];
#pragma unroll
                            for (int u = 0; u < kSegUnroll; u++) {
                                fp[u] = F(seg_cell(sc, dir, t0 + u < sc.n ? t0 + u : t0));
                                old[u] = *fp[u];
                            }
#pragma unroll
                            for (int u = 0; u < kSegUnroll; u++) {
                                if (t0 + u < sc.n) {
                                    float nv = old[u] * fac;
                                    if (tol > 0.0f && fabsf(nv - old[u]) > tol * fabsf(old[u])) changed = 1;
                                    *fp[u] = nv;
                                }
                            }
                        }
                    };
#pragma unroll
                    for (int c = 0; c < kSegSlots; c++)
                        if (c * 32 + lane < ns) upd(reg[c]);
                    for (int i = kSegSlots * 32 + lane; i < ns; i += 32) {
                        long long q = b + i;
                        uint32_t x = rs[q];
                        SegCells sc = seg_range(fa, fb, x, rt, cps, q, T, nudge, dir);
                        if (seg_back(x)) seg_dedup(sc, dir, ends[i - seg_back(x)]);
                        upd(sc);
                    }
                }
                // the next ray may read a cell another lane has just written,
                // and rewrites the sector scratch
                if (MODE != kSegSmem) __threadfence_block();
                __syncwarp();
            }
        }
        if (tol > 0.0f && !__any_sync(0xffffffffu, changed)) {
            it++;
            break;
        }
    }
    __syncwarp();
    for (long long q = lo + lane; q < n_cells; q += 32) f_g[q] = sm[q - lo];
    if (lane == 0 && sweeps_out) *sweeps_out = it;
}

template <int MODE>
static cudaError_t seq_seg_launch(uspg_ctx *c, const uspg_mart_opts *o, long long n_sm, size_t smem, cudaStream_t s)
{
    auto k = k_seq_seg<MODE>;
    if (smem > 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<1, 32, smem, s>>>(c->d_seg_ptr, c->d_seg_fa, c->d_seg_fb, c->d_seg_rs, c->d_seg_dir, c->d_view_turns,
                          c->d_ring, c->d_proj, c->d_f, c->n_cells, c->cells_per_slab, c->scan.n_views, c->n_rays,
                          o->iterations, (float)o->lambda, o->update_rule, (float)o->stop_tol, fixed_turns(kNudge), n_sm,
                          c->d_sweeps);
    return cudaGetLastError();
}

uspg_status launch_sequential_segments(uspg_ctx *c, const uspg_mart_opts *o, cudaStream_t s)
{
    int dev = 0, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    size_t ends_bytes = sizeof(int) * ((c->max_segments + 3) & ~3);  // per-ray sector scratch
    size_t f_bytes = sizeof(float) * ((c->n_cells + 3) & ~3LL);
    long long n_sm = ((long long)max_smem - (long long)ends_bytes) / (long long)sizeof(float) & ~3LL;
    cudaError_t e;
    if (f_bytes + ends_bytes <= (size_t)max_smem)
        e = seq_seg_launch<kSegSmem>(c, o, c->n_cells, f_bytes + ends_bytes, s);
    else if (n_sm >= c->n_cells / 8)
        e = seq_seg_launch<kSegSplit>(c, o, n_sm, sizeof(float) * n_sm + ends_bytes, s);
    else
        e = seq_seg_launch<kSegGlobal>(c, o, 0, ends_bytes, s);
    launch_counter()++;
    USPG_CUDA(c, e);
    return USPG_OK;
}

}  // namespace uspg
