// K1: FP64 coefficient generator (Sec. III.A-C, Algorithm 1).
//
// One thread traces one ray of one representative view.  The ray is cut at
// its crossings with the ring cylinders (Eq. 3-4, roots formed as
// (mr - d)(mr + d) so near-tangent rays keep their digits), the axial planes
// and the radial planes of the ring it is in; every piece between two
// consecutive crossings goes to the cell that holds its midpoint (Eq. 5-10)
// and pieces shorter than 1e-9 of a cell are dropped.  Unlike a global sort
// of all crossings, the walk follows the ray in path order -- the inbound
// segments of rings N-1 .. m0, the deepest ring, then the outbound segments
// m0 .. N-1 -- and merges only the crossings of one ring segment at a time.
// A cell can be met twice only across the dip into the inner rings; a
// per-ring record of the cell and position of the ring's last inbound piece
// merges such repeats.
//
// This file is compiled with -fmad=false: the crossings are formed with the
// same separately rounded operations as their definitions so the index lists
// do not depend on contraction.
//
// Passes: size (FP32 bound) -> scan -> fill (FP64 walk, then the row in the
// stored dtype) -> cell-major store (count per cell, slice widths, scan,
// scatter, per-cell sort by ray key so the layout is deterministic, lanes
// ordered by count).  Centred cone scans trace and store only the lower
// detector rows (z-mirror); the cell-major store then holds the lower and
// middle slabs, each column serving a cell and its mirror.
#include "internal.cuh"
#include "walk.cuh"

#include <algorithm>
#include <map>

namespace uspg {

__global__ void k_boundaries(const RingEntry *rt, int n_rings, double2 *bdir, float2 *bdirf)
{
    int i = blockIdx.x;
    if (i >= n_rings) return;
    int ng = rt[i].ng, h = rt[i].head;
    for (int j = threadIdx.x; j < ng; j += blockDim.x) {
        double a = kTwoPi * (double)j / (double)ng;
        double c = cos(a), sn = sin(a);
        bdir[h + j] = make_double2(c, sn);
        bdirf[h + j] = make_float2((float)c, (float)sn);
    }
}

// ---- which rows are traced -------------------------------------------------
//
// Transverse symmetry (Sec. III.C: a quarter of the first view's lines
// suffice): the reflection y -> -y fixes the source axis and maps view theta
// onto view -theta, detector column a onto n_u-1-a (fan and cone; a parallel
// ray keeps its bin, reversed), and sector j of every ring onto sector
// -1-j (mod n_g).  Representatives pair up as (rho, 1/G - rho): the rows of
// one are the mirror images of the other's, rotated by whole 1/G turns.  A
// representative that is its own mirror (rho = 0 or 1/(2G); fan or cone)
// traces the columns 2a <= n_u-1 and mirrors the rest.  The walks run over a
// list of traced representatives; every other row is derived (k_derive).
struct TracePlan {
    const int *reps;  // [n] representatives whose rows are walked
    int n;
    const int *half;  // [n_reps] 1: walk only the columns 2a <= n_u-1
};

// mirror column of a stored ray: fan and cone flip the detector column
__host__ __device__ inline int mirror_column(const Geometry &g, int ray)
{
    if (g.geometry == USPG_PARALLEL_2D) return ray;
    int a = ray % g.n_u;
    return ray - a + (g.n_u - 1 - a);
}

__device__ __forceinline__ bool walked(const Geometry &g, const TracePlan &P, long long gid, int *rep, int *ray)
{
    if (gid >= (long long)P.n * g.n_rows) return false;
    const int nv = g.n_rows / g.n_u;  // stored detector rows
    if (g.geometry == USPG_CONE_3D && nv > 1) {
        // neighbouring threads trace one detector column of one
        // representative, row after row: rays with the same projection on
        // the transverse plane, so the same ring and sector crossings, and
        // only their axial-plane crossings differ -- the walks of a warp stay
        // in step
        long long t = gid / nv;
        int v = (int)(gid - t * nv);
        *rep = P.reps[t % P.n];
        int a = (int)(t / P.n);
        *ray = v * g.n_u + a;
    } else {
        // the same ray in different representative views: rotations about
        // the axis, so the same rings and nearly the same sector crossings
        *rep = P.reps[gid % P.n];
        *ray = (int)(gid / P.n);
    }
    return !(P.half[*rep] && 2 * (*ray % g.n_u) > g.n_u - 1);
}

// Upper bound on each walked row's length from the FP32 sizing walk.
__global__ void __launch_bounds__(128) k_size(Geometry g, const RingEntry *rt, const float2 *bdirf,
                                              const int *rep_view, TracePlan P, int *caps)
{
    int rep, ray;
    if (!walked(g, P, (long long)blockIdx.x * blockDim.x + threadIdx.x, &rep, &ray)) return;
    caps[(long long)rep * g.n_rows + ray] = size_ray(g, rt, bdirf, rep_view[rep], ray);
}

// Exact row lengths (the FP64 walk without storing); used only when a row
// outgrew its FP32 bound.
template <int MAXR>
__global__ void __launch_bounds__(128) k_count(Geometry g, const RingEntry *rt, const double2 *bdir,
                                               const float2 *bdirf, const int *rep_view, TracePlan P, int *counts,
                                               int *status)
{
    int rep, ray;
    if (!walked(g, P, (long long)blockIdx.x * blockDim.x + threadIdx.x, &rep, &ray)) return;
    uint32_t in_cell[MAXR];
    double root[MAXR];
    CountSink sink;
    sink.in_cell = in_cell;
    sink.root = root;
    walk_ray(g, rt, bdir, bdirf, rep_view[rep], ray, sink, status);
    counts[(long long)rep * g.n_rows + ray] = sink.n;
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

// A row in the stored precision (FP64 length / scale, or 1 when binary;
// padding slots 0); returns its largest stored weight.
template <typename WT>
__device__ float store_row(const double *w64, long long b, long long e, int n, int binary, double inv_scale, WT *w)
{
    float mx = 0.0f;
    for (long long q = b; q < e; q++) {
        WT v = q - b < n ? to_w<WT>((float)(binary ? 1.0 : w64[q] * inv_scale)) : to_w<WT>(0.0f);
        w[q] = v;
        float fv = w_to_f(v);
        mx = fv > mx ? fv : mx;
    }
    return mx;
}

// FP64 walk into the row's slots [row_ptr[i], row_ptr[i+1]); writes the
// entry count to counts[i], pads the rest of the row (cell 0, weight 0), and
// stores the row in the stored precision with its largest weight.  A row
// with more entries than slots raises kStatusCountMismatch.  The rows are
// the walked rows of plan P, or (list != NULL) the rows list[0 .. *n_list);
// tied (optional) receives each row's tie flag (classify_exact).
template <int MAXR>
__global__ void __launch_bounds__(128) k_fill(Geometry g, const RingEntry *rt, const double2 *bdir,
                                              const float2 *bdirf, const int *rep_view, TracePlan P,
                                              const long long *list, const int *n_list, int *counts,
                                              const long long *row_ptr, uint32_t *idx, double *w64, int *status,
                                              int dtype, double inv_scale, void *w, float *rowmax, int *tied)
{
    long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int rep, ray;
    if (list) {
        if (gid >= *n_list) return;
        rep = (int)(list[gid] / g.n_rows);
        ray = (int)(list[gid] % g.n_rows);
    } else if (!walked(g, P, gid, &rep, &ray)) {
        return;
    }
    long long row = (long long)rep * g.n_rows + ray;
    long long b = row_ptr[row], e = row_ptr[row + 1];
    uint32_t in_cell[MAXR];
    int in_pos[MAXR];
    double root[MAXR];
    FillSink sink;
    sink.root = root;
    sink.idx = idx + b;
    sink.w = w64 + b;
    sink.cap = (int)(e - b);
    sink.in_cell = in_cell;
    sink.in_pos = in_pos;
    walk_ray(g, rt, bdir, bdirf, rep_view[rep], ray, sink, status);
    if (sink.overflow) flag(status, kStatusCountMismatch);
    counts[row] = sink.n;
    if (tied) tied[row] = sink.tied;
    for (long long q = b + sink.n; q < e; q++) idx[q] = 0;  // padding (its stored weight is 0)
    int binary = g.weight_mode == USPG_BINARY;
    float mx;
    if (dtype == USPG_F16) mx = store_row(w64, b, e, sink.n, binary, inv_scale, (__half *)w);
    else if (dtype == USPG_BF16) mx = store_row(w64, b, e, sink.n, binary, inv_scale, (__nv_bfloat16 *)w);
    else mx = store_row(w64, b, e, sink.n, binary, inv_scale, (float *)w);
    rowmax[row] = mx;
}

// Source row of a derived row (rep, ray), or -1 for a walked row.
__device__ __forceinline__ long long derive_source(const Geometry &g, const int *rep_src, const int *half, int rep,
                                                   int ray)
{
    int src = rep_src[rep];
    if (src < 0 && !(half[rep] && 2 * (ray % g.n_u) > g.n_u - 1)) return -1;
    if (src < 0) src = rep;
    return (long long)src * g.n_rows + mirror_column(g, ray);
}

// Bounds of the derived rows: the source row's FP32 bound (a mirror image
// has the source's length), with a little slack for a row that is walked
// after all because its source is tied.
__global__ void k_derive_caps(Geometry g, int n_reps, const int *rep_src, const int *half, int *caps)
{
    long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= (long long)n_reps * g.n_rows) return;
    long long src = derive_source(g, rep_src, half, (int)(row / g.n_rows), (int)(row % g.n_rows));
    if (src >= 0) caps[row] = caps[src] + 4;
}

// One warp per derived row: the source row mirrored (sector j -> (shift -
// 1 - j) mod n_g with shift = M n_g / G, M = rep_shift[rep]; slab and ring
// and weights unchanged), or, when the source row is tied, the row is queued
// for the direct walk (retrace).
template <typename WT>
__global__ void k_derive(Geometry g, const RingEntry *rt, int n_reps, const int *rep_src, const int *half,
                         const int *rep_shift, const long long *row_ptr, int *counts, uint32_t *idx, WT *w,
                         float *rowmax, const int *tied, long long *retrace, int *n_retrace)
{
    long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (row >= (long long)n_reps * g.n_rows) return;
    int rep = (int)(row / g.n_rows);
    long long src = derive_source(g, rep_src, half, rep, (int)(row % g.n_rows));
    if (src < 0) return;
    if (tied[src]) {
        if (lane == 0) retrace[atomicAdd(n_retrace, 1)] = row;
        return;
    }
    int n = counts[src];
    long long sb = row_ptr[src], db = row_ptr[row], de = row_ptr[row + 1];
    int M = rep_shift[rep];
    for (long long q = lane; q < de - db; q += 32) {
        if (q < n) {
            uint32_t pc = idx[sb + q];
            int ring = cell_ring(pc), ng = rt[ring].ng;
            int sec = M * rt[ring].step - 1 - cell_sector(pc);
            sec = sec < 0 ? sec + ng : sec;
            idx[db + q] = pack_cell(cell_slab(pc), ring, sec);
            w[db + q] = w[sb + q];
        } else {
            idx[db + q] = 0;
            w[db + q] = to_w<WT>(0.0f);
        }
    }
    if (lane == 0) {
        counts[row] = n;
        rowmax[row] = rowmax[src];
    }
}

// A row walked after all (its source row was tied) is compared with the
// mirror image k_derive would have written, one warp per row.  Where its
// count and cells (in order) are the mirror image's, it takes the mirror
// image's stored weights and maximum too (they differ from its own at most
// in FP32 rounding), so that every row of the representative is an exact
// mirror image; where a cell differs (the tie went the other way), its
// representative's columns cannot be derived from the source's
// (differs[rep] = 1).
template <typename WT>
__global__ void k_retrace_check(Geometry g, const RingEntry *rt, const int *rep_src, const int *rep_shift,
                                const long long *list, const int *n_list, const long long *row_ptr,
                                const int *counts, const uint32_t *idx, WT *w, float *rowmax, int *differs)
{
    long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (i >= *n_list) return;
    long long row = list[i];
    int rep = (int)(row / g.n_rows);
    if (rep_src[rep] < 0) return;  // not a mirror-image representative
    long long src = (long long)rep_src[rep] * g.n_rows + mirror_column(g, (int)(row % g.n_rows));
    int n = counts[row];
    long long sb = row_ptr[src], db = row_ptr[row];
    bool diff = n != counts[src];
    if (!diff) {
        int M = rep_shift[rep];
        for (int q = lane; q < n && !diff; q += 32) {
            uint32_t pc = idx[sb + q];
            int ring = cell_ring(pc), ng = rt[ring].ng;
            int sec = M * rt[ring].step - 1 - cell_sector(pc);
            sec = sec < 0 ? sec + ng : sec;
            diff = idx[db + q] != pack_cell(cell_slab(pc), ring, sec);
        }
    }
    if (__any_sync(0xffffffffu, diff)) {
        if (lane == 0) differs[rep] = 1;
        return;
    }
    for (int q = lane; q < n; q += 32) w[db + q] = w[sb + q];
    if (lane == 0) rowmax[row] = rowmax[src];
}

// what k_fill writes besides the FP64 rows: stored weights and row maxima
struct FillOut {
    int dtype;
    double inv_scale;
    void *w;
    float *rowmax;
};

// what a walk reads besides the geometry: the rows to walk (a plan, or a
// list whose length is on the device) and where the tie flags go
struct WalkRows {
    TracePlan plan;
    const long long *list = nullptr;
    const int *n_list = nullptr;
    int *tied = nullptr;
};

template <int MAXR>
static void launch_walk(bool fill, unsigned grid, cudaStream_t s, const Geometry &g, const RingEntry *rt,
                        const double2 *bdir, const float2 *bdirf, const int *rep_view, const WalkRows &wr,
                        int *counts, const long long *row_ptr, uint32_t *idx, double *w64, int *status,
                        const FillOut &fo)
{
    if (fill)
        k_fill<MAXR><<<grid, 128, 0, s>>>(g, rt, bdir, bdirf, rep_view, wr.plan, wr.list, wr.n_list, counts, row_ptr,
                                          idx, w64, status, fo.dtype, fo.inv_scale, fo.w, fo.rowmax, wr.tied);
    else
        k_count<MAXR><<<grid, 128, 0, s>>>(g, rt, bdir, bdirf, rep_view, wr.plan, counts, status);
}

static void walk(bool fill, unsigned grid, cudaStream_t s, const Geometry &g, const RingEntry *rt,
                 const double2 *bdir, const float2 *bdirf, const int *rep_view, const WalkRows &wr, int *counts,
                 const long long *row_ptr, uint32_t *idx, double *w64, int *status, const FillOut &fo = FillOut{})
{
#define USPG_WALK(M) launch_walk<M>(fill, grid, s, g, rt, bdir, bdirf, rep_view, wr, counts, row_ptr, idx, w64, status, fo)
    if (g.n_rings <= 64) USPG_WALK(64);
    else if (g.n_rings <= 128) USPG_WALK(128);
    else if (g.n_rings <= 256) USPG_WALK(256);
    else if (g.n_rings <= 512) USPG_WALK(512);
    else USPG_WALK(1024);
#undef USPG_WALK
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

// Columns of the cell-major store fed by the stored entry (ray r, cell pc):
// up to two (column cell, key) pairs.  The key is the ray id; with the
// z-mirror only lower-half and middle slabs have columns, and bit 31 of the
// key marks an entry whose column cell sees the mirror ray (mirror_ray(r))
// while the column cell's own mirror sees r.  An entry in an upper slab
// feeds the column of its mirror cell; an entry in the middle slab (odd slab
// count) feeds its own column twice, as r and as its mirror; a row that is
// its own mirror (middle detector row) holds both halves itself, so its
// upper entries feed nothing and its middle ones feed once.
__device__ __forceinline__ int entry_columns(const Mirror &M, int r, uint32_t pc, uint32_t col[2], uint32_t key[2])
{
    col[0] = pc;
    key[0] = (uint32_t)r;
    if (!M.on) return 1;
    int side = 2 * cell_slab(pc) - (M.n_slabs - 1);  // < 0 lower, 0 middle, > 0 upper
    bool self = (M.n_v & 1) && ray_row(r, M.n_u) == (M.n_v - 1) / 2;
    if (side < 0) return 1;
    if (side > 0) {
        if (self) return 0;
        col[0] = flip_slab(pc, M.n_slabs);
        key[0] = (uint32_t)r | 0x80000000u;
        return 1;
    }
    if (self) return 1;
    col[1] = pc;
    key[1] = (uint32_t)r | 0x80000000u;
    return 2;
}

// weight of a stored entry as a float (the FP16/BF16 stores hold length / w_scale)
__device__ __forceinline__ float w_as_float(float x) { return x; }
__device__ __forceinline__ float w_as_float(__half x) { return __half2float(x); }
__device__ __forceinline__ float w_as_float(__nv_bfloat16 x) { return __bfloat162float(x); }

// Cell-major key of a column entry: the index of the ray-term pair the
// correction gathers -- the stored ray, plus n_rows when the column's cell
// sees the mirror ray (entry_columns' bit 31).
__device__ __forceinline__ uint32_t cm_key(uint32_t key, int n_rows)
{
    return (key & 0x7fffffffu) + ((key >> 31) ? (uint32_t)n_rows : 0u);
}

// one warp per row (coalesced entries).  Entries whose stored weight is 0
// (lengths below the smallest FP16 subnormal) add nothing to a correction
// and get no column.
template <typename WT>
__global__ void k_cell_count(const long long *row_ptr, const int *counts, const uint32_t *idx, const WT *w,
                             int n_rows, Mirror M, const RingEntry *rt, long long cps, int *cell_cnt)
{
    long long ray = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (ray >= n_rows) return;
    long long b = row_ptr[ray];
    int n = counts[ray];
    for (int q = lane; q < n; q += 32) {
        if (!(w_as_float(w[b + q]) > 0.0f)) continue;
        uint32_t col[2], key[2];
        int k = entry_columns(M, (int)ray, idx[b + q], col, key);
        for (int t = 0; t < k; t++) atomicAdd(&cell_cnt[rep_cell_id(rt, cps, col[t])], 1);
    }
}

// one warp per slice: width = max count over its 32 cells.  shift >= 0: the
// slices of a mirror-image representative, whose cell (slab, ring, j) has
// the count of the source's cell (slab, ring, (shift step - 1 - j) mod n_g)
// (the source's counts are in cell_cnt).
__global__ void k_slice_width(const RingEntry *rt, const int *slice_ring, int slices_per_slab, long long n_slices,
                              long long cps, const int *cell_cnt, int shift, int *width, uint32_t *meta, int *status)
{
    long long sl = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (sl >= n_slices) return;
    int slab = (int)(sl / slices_per_slab);
    int within = (int)(sl % slices_per_slab);
    int ring = slice_ring[within];
    RingEntry e = rt[ring];
    int sec0 = (within - e.chunk0) * kSlice;
    int sec = sec0 + lane;
    int c = 0;
    if (sec < e.ng) {
        int j = sec;
        if (shift >= 0) {
            j = shift * e.step - 1 - sec;
            j = j < 0 ? j + e.ng : j;
        }
        c = cell_cnt[(long long)slab * cps + e.head + j];
    }
    c = __reduce_max_sync(0xffffffffu, c);
    if (lane == 0) {
        width[sl] = c;
        meta[sl] = pack_cell(slab, ring, sec0);
        if (c > kMaxCellRays) atomicOr(status, kStatusCellRays);
    }
}

template <typename WT>
__global__ void k_cell_scatter(const long long *row_ptr, const int *counts, const uint32_t *idx, const WT *w,
                               int n_rows, Mirror M, const RingEntry *rt, long long cps, int slices_per_slab,
                               const long long *slice_off, int *cell_fill, uint32_t *sray, WT *sw)
{
    long long ray = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int wl = threadIdx.x & 31;
    if (ray >= n_rows) return;
    long long b = row_ptr[ray];
    int n = counts[ray];
    for (int q = wl; q < n; q += 32) {  // one warp per row
        if (!(w_as_float(w[b + q]) > 0.0f)) continue;  // as k_cell_count
        uint32_t col[2], key[2];
        int k = entry_columns(M, (int)ray, idx[b + q], col, key);
        for (int t = 0; t < k; t++) {
            int lane;
            long long sl = rep_cell_slice(rt, slices_per_slab, col[t], &lane);
            int slot = atomicAdd(&cell_fill[rep_cell_id(rt, cps, col[t])], 1);
            long long pos = slice_off[sl] + (long long)slot * kSlice + lane;
            sray[pos] = cm_key(key[t], n_rows);
            sw[pos] = w[b + q];
        }
    }
}

// heap step of the in-place column sort (the column's t-th entry is at
// base + 32 t)
template <typename WT>
__device__ void sift_down(uint32_t *ray, WT *w, long long base, int root, int n)
{
    for (;;) {
        int child = 2 * root + 1;
        if (child >= n) return;
        long long pc = base + (long long)child * kSlice;
        if (child + 1 < n && ray[pc + kSlice] > ray[pc]) {
            child++;
            pc += kSlice;
        }
        long long pr = base + (long long)root * kSlice;
        if (!(ray[pc] > ray[pr])) return;
        uint32_t tr = ray[pr];
        ray[pr] = ray[pc];
        ray[pc] = tr;
        WT tw = w[pr];
        w[pr] = w[pc];
        w[pc] = tw;
        root = child;
    }
}

// stats[rep] += entries of that representative's full rows (a stored row
// counts twice when its mirror row is not stored), stats[n_reps + rep] +=
// stored entries, stats[2 n_reps] = longest row
__global__ void k_row_stats(const int *counts, long long n_all, int n_rows, Mirror M, int n_reps, long long *stats)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int c = i < n_all ? counts[i] : 0;
    long long rep = i < n_all ? i / n_rows : -1;
    int ray = i < n_all ? (int)(i % n_rows) : 0;
    int mult = M.on && !((M.n_v & 1) && ray_row(ray, M.n_u) == (M.n_v - 1) / 2) ? 2 : 1;
    int mx = c;
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    unsigned long long *st = (unsigned long long *)stats;
    // warps whose rows all belong to one representative reduce first
    long long rep0 = __shfl_sync(0xffffffffu, rep, 0);
    bool uniform = __all_sync(0xffffffffu, rep == rep0) && rep0 >= 0;
    if (uniform) {
        int full = c * mult, sum = c;
        for (int o = 16; o > 0; o >>= 1) {
            full += __shfl_xor_sync(0xffffffffu, full, o);
            sum += __shfl_xor_sync(0xffffffffu, sum, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&st[rep0], (unsigned long long)full);
            atomicAdd(&st[n_reps + rep0], (unsigned long long)sum);
        }
    } else if (rep >= 0) {
        atomicAdd(&st[rep], (unsigned long long)c * mult);
        atomicAdd(&st[n_reps + rep], (unsigned long long)c);
    }
    if ((threadIdx.x & 31) == 0) atomicMax(&st[2 * n_reps], (unsigned long long)mx);
}

// Slot offsets of all slices: 32 x the scan of all representatives' widths
// (each representative's slices follow the earlier ones').
__global__ void k_set_off(long long *dst, const long long *rel, long long n)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = rel[i] * kSlice;
}

// ---- cell-major store with lanes ordered by ray count ----------------------------
//
// In each 32-cell slice the lanes are permuted so that ray counts fall from
// lane 0 to lane 31; row t of the slice then holds its present entries in a
// prefix of its 32 slots, and a kernel lane l reads entry t of its cell at
// slice_off + 32 t + l whenever t < count(l) -- addresses that depend on no
// loaded data, with the absent slots never fetched.  lane_desc[32 s + l] =
// (source lane << 11) | count.

// Sort and lane order in one pass: one warp per slice, each lane owning one
// cell whose column sits in arrival order at slice_off + 32 t + lane.  The
// lane's rank (counts falling from lane 0, ties by lane) and count go to
// lane_desc; the column, sorted by key (a total order: a ray meets a cell
// once per view, and a key of its mirror is offset by n_rows), goes to slots
// 32 t + rank of the lane-ordered store.  Columns of up to kOrderRegs entries
// are sorted in registers by odd-even transposition, with the network sized
// to the slice's longest column (slices are two or three entries wide at the
// median); longer ones in place first.
constexpr int kOrderRegs = 8;

template <typename WT>
__device__ __forceinline__ void cx(uint32_t &ra, WT &wa, uint32_t &rb, WT &wb)
{
    if (ra > rb) {
        uint32_t t = ra;
        ra = rb;
        rb = t;
        WT u = wa;
        wa = wb;
        wb = u;
    }
}

// column of cnt <= R entries (load(t, key, w) fetches entry t): sorted in
// registers, written to off + 32 t + rank
template <int R, typename WT, class Load>
__device__ __forceinline__ void order_in_regs(Load load, int cnt, uint32_t *dray, WT *dw, long long off, int rank)
{
    uint32_t r[R];
    WT w[R];
#pragma unroll
    for (int t = 0; t < R; t++) {
        r[t] = 0xffffffffu;  // absent entries sort last
        w[t] = to_w<WT>(0.0f);
        if (t < cnt) load(t, r[t], w[t]);
    }
#pragma unroll
    for (int pass = 0; pass < R; pass++) {
#pragma unroll
        for (int t = pass & 1; t + 1 < R; t += 2) cx(r[t], w[t], r[t + 1], w[t + 1]);
    }
#pragma unroll
    for (int t = 0; t < R; t++) {
        if (t < cnt) {
            dray[off + (long long)t * kSlice + rank] = r[t];
            dw[off + (long long)t * kSlice + rank] = w[t];
        }
    }
}

// a longer column, in arrival order at base + 32 t: sorted in place
// (insertion sort, or heapsort for a cell crossed by very many rays), then
// written to off + 32 t + rank
template <typename WT>
__device__ void order_in_place(uint32_t *sray, WT *sw, long long base, int cnt, uint32_t *dray, WT *dw, long long off,
                               int rank)
{
    if (cnt <= 32) {
        for (int q = 1; q < cnt; q++) {
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
    } else {
        for (int q = cnt / 2 - 1; q >= 0; q--) sift_down(sray, sw, base, q, cnt);
        for (int e = cnt - 1; e > 0; e--) {
            long long pe = base + (long long)e * kSlice;
            uint32_t tr = sray[base];
            sray[base] = sray[pe];
            sray[pe] = tr;
            WT tw = sw[base];
            sw[base] = sw[pe];
            sw[pe] = tw;
            sift_down(sray, sw, base, 0, e);
        }
    }
    for (int t = 0; t < cnt; t++) {
        dray[off + (long long)t * kSlice + rank] = sray[base + (long long)t * kSlice];
        dw[off + (long long)t * kSlice + rank] = sw[base + (long long)t * kSlice];
    }
}

// lane rank within a slice: counts falling from lane 0, ties by lane (one
// round per distinct count); *wmax receives the slice's longest column
__device__ __forceinline__ int lane_rank(int cnt, int lane, int *wmax)
{
    const unsigned lt_mask = (1u << lane) - 1u;
    unsigned left = 0xffffffffu;
    int rank = 0, above = 0;
    *wmax = -1;
    while (left) {
        int c = __reduce_max_sync(0xffffffffu, (left >> lane) & 1u ? cnt : -1);
        if (*wmax < 0) *wmax = c;
        unsigned eq = __ballot_sync(0xffffffffu, ((left >> lane) & 1u) && cnt == c);
        if ((eq >> lane) & 1u) rank = above + __popc(eq & lt_mask);
        above += __popc(eq);
        left &= ~eq;
    }
    return rank;
}

template <typename WT>
__global__ void k_cell_order(long long n_slices, const uint32_t *meta, const long long *slice_off,
                             const RingEntry *rt, long long cps, const int *cell_cnt, uint32_t *sray, WT *sw,
                             uint16_t *lane_desc, uint32_t *dray, WT *dw)
{
    long long sl = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (sl >= n_slices) return;
    uint32_t m = meta[sl];
    int ring = cell_ring(m), sec = cell_sector(m) + lane;
    int cnt = sec < rt[ring].ng ? cell_cnt[(long long)cell_slab(m) * cps + rt[ring].head + sec] : 0;
    int wmax;
    int rank = lane_rank(cnt, lane, &wmax);
    lane_desc[sl * 32 + rank] = (uint16_t)((lane << 11) | cnt);
    long long off = slice_off[sl], base = off + lane;
    auto load = [&](int t, uint32_t &r, WT &w) {
        r = sray[base + (long long)t * kSlice];
        w = sw[base + (long long)t * kSlice];
    };
    if (wmax <= 2) order_in_regs<2>(load, cnt, dray, dw, off, rank);
    else if (wmax <= 4) order_in_regs<4>(load, cnt, dray, dw, off, rank);
    else if (cnt <= kOrderRegs) order_in_regs<kOrderRegs>(load, cnt, dray, dw, off, rank);
    else order_in_place(sray, sw, base, cnt, dray, dw, off, rank);
}

// Columns of a representative whose rows are all mirror images of its
// source's (transverse symmetry; none of its rows was walked after all):
// cell (slab, ring, j) has the column of the source's cell (slab, ring,
// (M step - 1 - j) mod n_g) with each ray replaced by its mirror column
// (same n_rows offset for a mirror-ray key).  One warp per slice, read from
// the source's finished lane-ordered store (its lane_desc gives each source
// cell's lane rank and count) and written, sorted by the new keys, in this
// representative's lane order -- the same store the count, scatter and
// order passes would build from the derived rows.  Block size 256.
template <typename WT>
__global__ void __launch_bounds__(256) k_derive_columns(long long n_slices, int slices_per_slab, Geometry g,
                                                        const RingEntry *rt, int shift, const uint32_t *meta,
                                                        const long long *slice_off, const long long *src_off,
                                                        const uint16_t *src_desc, uint32_t *sray, WT *sw,
                                                        uint16_t *lane_desc, uint32_t *dray, WT *dw)
{
    __shared__ uint16_t inv[8][32];
    long long sl = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (sl >= n_slices) return;
    uint32_t m = meta[sl];
    int ring = cell_ring(m), sec = cell_sector(m) + lane;
    RingEntry e = rt[ring];
    bool valid = sec < e.ng;
    int ja = e.step * shift - 1 - sec;
    if (ja < 0) ja += e.ng;
    long long sla = (long long)cell_slab(m) * slices_per_slab + e.chunk0 + (ja >> 5);
    int la = ja & (kSlice - 1);
    // rank and count of each lane's source cell: one round per source slice
    // (at most three), inverting that slice's lane order in shared memory
    int rank_a = 0, cnt = 0;
    unsigned todo = __ballot_sync(0xffffffffu, valid);
    while (todo) {
        long long cur = __shfl_sync(0xffffffffu, sla, __ffs(todo) - 1);
        uint16_t d = src_desc[cur * 32 + lane];
        inv[wib][d >> 11] = (uint16_t)((lane << 11) | (d & 2047));
        __syncwarp();
        bool mine = valid && sla == cur;
        if (mine) {
            uint16_t v = inv[wib][la];
            rank_a = v >> 11;
            cnt = v & 2047;
        }
        __syncwarp();
        todo &= ~__ballot_sync(0xffffffffu, mine);
    }
    int wmax;
    int rank = lane_rank(cnt, lane, &wmax);
    lane_desc[sl * 32 + rank] = (uint16_t)((lane << 11) | cnt);
    long long off = slice_off[sl];
    long long abase = valid ? src_off[sla] + rank_a : 0;
    const uint32_t nr = (uint32_t)g.n_rows;
    auto load = [&](int t, uint32_t &r, WT &w) {
        uint32_t k = dray[abase + (long long)t * kSlice];
        uint32_t fl = k >= nr ? nr : 0u;
        r = (uint32_t)mirror_column(g, (int)(k - fl)) + fl;
        w = dw[abase + (long long)t * kSlice];
    };
    if (wmax <= 2) order_in_regs<2>(load, cnt, dray, dw, off, rank);
    else if (wmax <= 4) order_in_regs<4>(load, cnt, dray, dw, off, rank);
    else if (cnt <= kOrderRegs) order_in_regs<kOrderRegs>(load, cnt, dray, dw, off, rank);
    else {  // long column: mapped into this slice's arrival slots, then sorted in place
        long long base = off + lane;
        for (int t = 0; t < cnt; t++) {
            uint32_t r;
            WT w;
            load(t, r, w);
            sray[base + (long long)t * kSlice] = r;
            sw[base + (long long)t * kSlice] = w;
        }
        order_in_place(sray, sw, base, cnt, dray, dw, off, rank);
    }
}

// Correction descriptors of one representative's slices: {first slot
// relative to the representative's base, meta}, one 8-byte load per slice.
// All representatives in one launch: rep_first[r] is representative r's
// first slice in the scan of all widths (its slots start at 32 x that).
__global__ void k_slice_desc(uint2 *desc, const long long *slice_off, const uint32_t *meta,
                             const long long *rep_first, long long n_slices, long long n)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) desc[i] = make_uint2((uint32_t)(slice_off[i] - rep_first[i / n_slices] * kSlice), meta[i]);
}

// ray of every aligned group of kRowPad entries of the ray-major store (rows
// start and end on group boundaries, so a group never straddles two rays);
// one warp per row
__global__ void k_group_rays(const long long *row_ptr, long long n_all, int n_rows, uint32_t *grp_ray)
{
    long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= n_all) return;
    uint32_t ray = (uint32_t)(row % n_rows);
    long long g1 = row_ptr[row + 1] / kRowPad;
    for (long long g = row_ptr[row] / kRowPad + (threadIdx.x & 31); g < g1; g += 32) grp_ray[g] = ray;
}

// every stride-th prefix sum (the first entry or slice of each
// representative, and the end): one read-back
__global__ void k_rep_entry0(const long long *prefix, int n_reps, int stride, long long *out)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q <= n_reps) out[q] = prefix[(long long)q * stride];
}

static unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

Geometry make_geometry(const uspg_ctx *c)
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
    g.n_rows = c->mir.n_rows;
    return g;
}

cudaError_t scan_counts(const int *in, long long n, long long *out, cudaStream_t s)
{
    return exclusive_scan<int>(in, n, 1, out, s);
}

// Host side of the transverse symmetry: which representatives are walked,
// which are mirror images of which (and by how many 1/G turns the mirror
// image is rotated), which walk only half their columns.  View k sits at
// theta = (m + key / den) / G turns (m = floor(k arc G / den)); the mirror of
// residue key is residue (den - key) mod den.
struct SymPlan {
    std::vector<int> trace, half, src, shift;
    long long walked_rows = 0;
};

static SymPlan sym_plan(const uspg_ctx *c)
{
    const int nreps = c->n_reps;
    const long long den = c->scan.arc_den * (long long)c->scan.n_views;
    std::vector<long long> key(nreps), m(nreps);
    std::map<long long, int> rep_of_key;
    for (int r = 0; r < nreps; r++) {
        long long num = (long long)c->rep_view[r] * c->scan.arc_num * c->G;
        m[r] = num / den;
        key[r] = num % den;
        rep_of_key[key[r]] = r;
    }
    SymPlan P;
    P.half.assign(nreps, 0);
    P.src.assign(nreps, -1);
    P.shift.assign(nreps, 0);
    const bool columns_mirror = c->scan.geometry != USPG_PARALLEL_2D;  // a parallel ray is its own mirror
    for (int r = 0; r < nreps; r++) {
        if (P.src[r] >= 0) continue;  // a mirror image of an earlier representative
        auto it = rep_of_key.find((den - key[r]) % den);
        if (it != rep_of_key.end()) {
            int r2 = it->second;
            int M = (int)((m[r] + m[r2] + (key[r] != 0 ? 1 : 0)) % c->G);
            if (r2 == r && columns_mirror) {
                P.half[r] = 1;
                P.shift[r] = M;
            } else if (r2 > r) {
                P.src[r2] = r;
                P.shift[r2] = M;
            }
        }
        P.trace.push_back(r);
    }
    int n_u = c->scan.n_u, half_cols = 0;
    for (int a = 0; a < n_u; a++) half_cols += 2 * a <= n_u - 1;
    for (int r : P.trace) P.walked_rows += P.half[r] ? (long long)c->mir.n_rows / n_u * half_cols : c->mir.n_rows;
    return P;
}

template <typename WT>
static uspg_status build_typed(uspg_ctx *c, cudaStream_t s)
{
    Geometry g = make_geometry(c);
    const Mirror M = c->mir;
    const int n_rows = M.n_rows;

    const int nreps = c->n_reps;
    const long long nrows = (long long)nreps * n_rows;
    const long long n_slices = c->slices_per_rep;
    if (!c->d_row_ptr) {  // geometry-sized buffers, allocated once
        USPG_CUDA(c, cudaMalloc(&c->d_rep_view, sizeof(int) * nreps));
        USPG_CUDA(c, cudaMemcpy(c->d_rep_view, c->rep_view.data(), sizeof(int) * nreps, cudaMemcpyHostToDevice));
        USPG_CUDA(c, cudaMalloc(&c->d_counts, sizeof(int) * (nrows + 1)));
        USPG_CUDA(c, cudaMalloc(&c->d_row_ptr, sizeof(long long) * (nrows + 1)));
        USPG_CUDA(c, cudaMalloc(&c->d_rowmax, sizeof(float) * (nrows + 1)));
        USPG_CUDA(c, cudaMalloc(&c->d_cell_cnt, sizeof(int) * c->n_cells));
        USPG_CUDA(c, cudaMalloc(&c->d_cell_fill, sizeof(int) * c->n_cells));
        USPG_CUDA(c, cudaMalloc(&c->d_rel, sizeof(long long) * (n_slices * nreps + 1)));
        USPG_CUDA(c, cudaMalloc(&c->d_slice_off, sizeof(long long) * n_slices * nreps));
        USPG_CUDA(c, cudaMalloc(&c->d_slice_meta, sizeof(uint32_t) * n_slices * nreps));
        USPG_CUDA(c, cudaMalloc(&c->d_slice_desc, sizeof(uint2) * n_slices * nreps));
        USPG_CUDA(c, cudaMalloc(&c->d_slice_width, sizeof(int) * n_slices * nreps));
        USPG_CUDA(c, cudaMalloc(&c->d_stats, sizeof(long long) * (2 * nreps + 1)));
        // symmetry plan tables, tie flags, rows to walk after all
        USPG_CUDA(c, cudaMalloc(&c->d_plan, sizeof(int) * 6 * nreps));
        USPG_CUDA(c, cudaMalloc(&c->d_tied, sizeof(int) * (nrows + 1)));
        USPG_CUDA(c, cudaMalloc(&c->d_retrace, sizeof(long long) * (nrows + 1)));
        USPG_CUDA(c, cudaMallocHost(&c->h_gen_pin, sizeof(long long) * (4 * nreps + 8)));
        USPG_CUDA(c, cudaMalloc(&c->d_gen_small, sizeof(long long) * (nreps + 1)));
        c->store_moved = true;
    }
    // pinned read-back slots
    long long *pin_stats = c->h_gen_pin;                   // [2 reps + 1]
    long long *pin_entry0 = c->h_gen_pin + 2 * nreps + 1;  // [reps + 1]
    long long *pin_tot = c->h_gen_pin + 3 * nreps + 2;     // [reps + 1] first slice of each representative
    int *pin_flags = (int *)(c->h_gen_pin + 4 * nreps + 3);  // n_retrace, status, status
    int *d_rep_view = c->d_rep_view, *d_counts = c->d_counts;

    const int TB = 128;
    // with the z-mirror only the rows of rays 0 .. n_rows-1 (lower detector rows) are traced and stored
    // symmetry plan: d_plan = {walked reps, half, source, shift, all reps, zeros}
    SymPlan sp = sym_plan(c);
    {
        std::vector<int> tab(6 * nreps, 0);
        for (size_t q = 0; q < sp.trace.size(); q++) tab[q] = sp.trace[q];
        for (int r = 0; r < nreps; r++) {
            tab[nreps + r] = sp.half[r];
            tab[2 * nreps + r] = sp.src[r];
            tab[3 * nreps + r] = sp.shift[r];
            tab[4 * nreps + r] = r;
        }
        USPG_CUDA(c, cudaMemcpyAsync(c->d_plan, tab.data(), sizeof(int) * 6 * nreps, cudaMemcpyHostToDevice, s));
    }
    const int *d_trace = c->d_plan, *d_half = c->d_plan + nreps, *d_src = c->d_plan + 2 * nreps;
    const int *d_shift = c->d_plan + 3 * nreps, *d_all = c->d_plan + 4 * nreps, *d_zero = c->d_plan + 5 * nreps;
    // the symmetry pays only when the rows are more than the GPU walks at once:
    // a small store (a 2D scan) is walked whole in one wave, and deriving
    // would add a second, serial walk of its tied rows
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool sym = sp.walked_rows < nrows && c->symmetry != USPG_SYMMETRY_NEVER &&
                     (c->symmetry == USPG_SYMMETRY_ALWAYS || nrows >= 2LL * sms * 4 * TB);
    int *d_n_retrace = c->d_tied + nrows;  // counter after the flags
    // rows sized by the FP32 bound, filled by the FP64 walk; if any row
    // outgrows its bound the exact FP64 count sizes the rows instead (and
    // every row is walked)
    long long nnz_pad = 0;
    c->gen_walked_rows = nrows;
    // representatives whose rows are all mirror images of a source's: their
    // columns are derived from the source's columns (k_derive_columns)
    std::vector<char> cols_from_src(nreps, 0);
    std::vector<int> differs;
    for (int attempt = 0; attempt < 2; attempt++) {
        const bool use_sym = attempt == 0 && sym;
        WalkRows wr;
        wr.plan = use_sym ? TracePlan{d_trace, (int)sp.trace.size(), d_half} : TracePlan{d_all, nreps, d_zero};
        const unsigned grid = nblk((long long)wr.plan.n * n_rows, TB);
        if (attempt == 0) {
            k_size<<<grid, TB, 0, s>>>(g, c->d_ring, c->d_bdirf, d_rep_view, wr.plan, d_counts);
            if (use_sym) {
                launch_counter()++;
                k_derive_caps<<<nblk(nrows, 256), 256, 0, s>>>(g, nreps, d_src, d_half, d_counts);
            }
        } else {
            walk(false, grid, s, g, c->d_ring, c->d_bdir, c->d_bdirf, d_rep_view, wr, d_counts, nullptr, nullptr,
                 nullptr, c->d_status);
        }
        launch_counter()++;
        USPG_CUDA(c, cudaGetLastError());
        USPG_CUDA(c, exclusive_scan<int>(d_counts, nrows, kRowPad, c->d_row_ptr, s));
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
        FillOut fo{c->dtype, 1.0 / c->w_scale, c->d_w, c->d_rowmax};
        wr.tied = use_sym ? c->d_tied : nullptr;
        walk(true, grid, s, g, c->d_ring, c->d_bdir, c->d_bdirf, d_rep_view, wr, d_counts, c->d_row_ptr, c->d_idx,
             c->d_w64, c->d_status, fo);
        launch_counter()++;
        USPG_CUDA(c, cudaGetLastError());
        int n_retrace = 0;
        int st = 0;
        bool have_st = false;
        if (use_sym) {  // mirror images of the walked rows; tied ones are walked after all
            USPG_CUDA(c, cudaMemsetAsync(d_n_retrace, 0, sizeof(int), s));
            k_derive<WT><<<nblk(nrows * 32, 256), 256, 0, s>>>(g, c->d_ring, nreps, d_src, d_half, d_shift,
                                                               c->d_row_ptr, d_counts, c->d_idx, (WT *)c->d_w,
                                                               c->d_rowmax, c->d_tied, c->d_retrace,
                                                               d_n_retrace);
            launch_counter()++;
            USPG_CUDA(c, cudaGetLastError());
            USPG_CUDA(c, cudaMemcpyAsync(pin_flags, d_n_retrace, sizeof(int), cudaMemcpyDeviceToHost, s));
            USPG_CUDA(c, cudaMemcpyAsync(pin_flags + 1, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
            USPG_CUDA(c, cudaStreamSynchronize(s));
            n_retrace = pin_flags[0];
            st = pin_flags[1];
            have_st = n_retrace == 0;  // the status stands unless rows are walked again
            for (int r = 0; r < nreps; r++) cols_from_src[r] = sp.src[r] >= 0;
            if (n_retrace > 0) {
                WalkRows wl;
                wl.plan = wr.plan;
                wl.list = c->d_retrace;
                wl.n_list = d_n_retrace;
                walk(true, nblk(n_retrace, TB), s, g, c->d_ring, c->d_bdir, c->d_bdirf, d_rep_view, wl, d_counts,
                     c->d_row_ptr, c->d_idx, c->d_w64, c->d_status, fo);
                launch_counter()++;
                USPG_CUDA(c, cudaGetLastError());
                // representatives with a walked row that is not the mirror image build their own columns
                int *d_differs = (int *)c->d_stats;  // scratch until the statistics below
                USPG_CUDA(c, cudaMemsetAsync(d_differs, 0, sizeof(int) * nreps, s));
                k_retrace_check<WT><<<nblk((long long)n_retrace * 32, 256), 256, 0, s>>>(
                    g, c->d_ring, d_src, d_shift, c->d_retrace, d_n_retrace, c->d_row_ptr, d_counts, c->d_idx,
                    (WT *)c->d_w, c->d_rowmax, d_differs);
                launch_counter()++;
                USPG_CUDA(c, cudaGetLastError());
                differs.assign(nreps, 0);
                USPG_CUDA(c, cudaMemcpyAsync(differs.data(), d_differs, sizeof(int) * nreps, cudaMemcpyDeviceToHost, s));
            }
        }
        if (!have_st) {
            USPG_CUDA(c, cudaMemcpyAsync(pin_flags + 1, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
            USPG_CUDA(c, cudaStreamSynchronize(s));
            st = pin_flags[1];
        }
        for (int r = 0; r < nreps && r < (int)differs.size(); r++)
            if (differs[r]) cols_from_src[r] = 0;
        if (!(st & kStatusCountMismatch)) {
            c->gen_walked_rows = use_sym ? sp.walked_rows + n_retrace : nrows;
            break;
        }
        if (attempt == 1) return fail(c, USPG_EDEVICE, "generator rows changed between passes");
        std::fill(cols_from_src.begin(), cols_from_src.end(), 0);
        USPG_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), s));
        c->gen_fallbacks++;
    }

    // statistics on the device: per-representative nonzeros and longest row
    USPG_CUDA(c, cudaMemsetAsync(c->d_stats, 0, sizeof(long long) * (2 * nreps + 1), s));
    k_row_stats<<<nblk(nrows, 256), 256, 0, s>>>(d_counts, nrows, n_rows, M, nreps, c->d_stats);
    launch_counter()++;
    // statistics and entry offsets: read with the slice totals below
    USPG_CUDA(c, cudaMemcpyAsync(pin_stats, c->d_stats, sizeof(long long) * (2 * nreps + 1), cudaMemcpyDeviceToHost, s));
    k_rep_entry0<<<nblk(nreps + 1, 128), 128, 0, s>>>(c->d_row_ptr, nreps, n_rows, c->d_gen_small);
    launch_counter()++;
    USPG_CUDA(c, cudaMemcpyAsync(pin_entry0, c->d_gen_small, sizeof(long long) * (nreps + 1), cudaMemcpyDeviceToHost, s));
    c->h_row_ptr.clear();  // host copy made on demand by uspg_get_row

    // cell-major store, one representative at a time
    if (n_slices * kSlice >= (1LL << 31))
        return fail(c, USPG_EUNSUPPORTED, "a view's cell-major store has 2^26 slices or more");
    int *d_cell_cnt = c->d_cell_cnt, *d_cell_fill = c->d_cell_fill;
    long long *d_rel = c->d_rel;
    // pass 1: slice widths of every representative, then one scan over all
    // of them: every representative's slots follow the earlier ones'
    // mirror-image representative whose columns derive from rep's, or -1
    std::vector<int> partner(nreps, -1);
    for (int r = 0; r < nreps; r++)
        if (cols_from_src[r]) partner[sp.src[r]] = r;
    for (int rep = 0; rep < nreps; rep++) {
        const long long *rp = c->d_row_ptr + (long long)rep * n_rows;
        const int *cn = d_counts + (long long)rep * n_rows;
        int *wd = c->d_slice_width + rep * n_slices;
        if (!cols_from_src[rep]) {  // a mirror image's widths were set with its source's counts
            USPG_CUDA(c, cudaMemsetAsync(d_cell_cnt, 0, sizeof(int) * c->n_cells, s));
            k_cell_count<WT><<<nblk((long long)n_rows * 32, 256), 256, 0, s>>>(
                rp, cn, c->d_idx, (const WT *)c->d_w, n_rows, M, c->d_ring, c->cells_per_slab, d_cell_cnt);
            launch_counter()++;
            const int q = partner[rep];
            k_slice_width<<<nblk(n_slices * 32, 256), 256, 0, s>>>(
                c->d_ring, c->d_slice_ring, c->slices_per_slab, n_slices, c->cells_per_slab, d_cell_cnt, -1, wd,
                c->d_slice_meta + rep * n_slices, c->d_status);
            launch_counter()++;
            if (q >= 0) {
                k_slice_width<<<nblk(n_slices * 32, 256), 256, 0, s>>>(
                    c->d_ring, c->d_slice_ring, c->slices_per_slab, n_slices, c->cells_per_slab, d_cell_cnt,
                    sp.shift[q], c->d_slice_width + q * n_slices, c->d_slice_meta + q * n_slices, c->d_status);
                launch_counter()++;
            }
        }
    }
    const long long all_slices = (long long)nreps * n_slices;
    USPG_CUDA(c, exclusive_scan<int>(c->d_slice_width, all_slices, 1, d_rel, s));
    k_set_off<<<nblk(all_slices, 256), 256, 0, s>>>(c->d_slice_off, d_rel, all_slices);
    launch_counter()++;
    k_rep_entry0<<<nblk(nreps + 1, 128), 128, 0, s>>>(d_rel, nreps, (int)n_slices, c->d_gen_small);
    launch_counter()++;
    USPG_CUDA(c, cudaMemcpyAsync(pin_tot, c->d_gen_small, sizeof(long long) * (nreps + 1), cudaMemcpyDeviceToHost, s));
    USPG_CUDA(c, cudaMemcpyAsync(pin_flags + 2, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    USPG_CUDA(c, cudaStreamSynchronize(s));
    std::vector<long long> rep_tot(nreps);  // slices of each representative
    for (int r = 0; r < nreps; r++) rep_tot[r] = pin_tot[r + 1] - pin_tot[r];
    const long long *rep_nnz = pin_stats;
    const int st_cm = pin_flags[2];
    c->h_rep_entry0.assign(pin_entry0, pin_entry0 + nreps + 1);
    long long nnz = 0, nnz_full = 0, maxrow = rep_nnz[2 * nreps];
    for (int q = 0; q < nreps; q++) {
        nnz_full += rep_nnz[q];
        nnz += rep_nnz[nreps + q];
    }
    long long all = 0;
    for (int k = 0; k < c->scan.n_views; k++) all += rep_nnz[c->rep_of_view[k]];
    c->nnz_all_views = all;
    long long sell = 0;
    c->h_sell_base.assign(nreps + 1, 0);
    for (int rep = 0; rep < nreps; rep++) {
        c->h_sell_base[rep] = sell;
        if (rep_tot[rep] * kSlice >= (1LL << 32))
            return fail(c, USPG_EUNSUPPORTED, "a view's cell-major store exceeds 2^32 slots");
        sell += rep_tot[rep] * kSlice;
    }
    c->h_sell_base[nreps] = sell;
    if (st_cm & kStatusCellRays) {
        USPG_CUDA(c, cudaMemset(c->d_status, 0, sizeof(int)));
        return fail(c, USPG_EUNSUPPORTED, "a cell is crossed by more than 2047 rays of one view");
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
    if ((size_t)(sell + kSlice) > c->cap_cm) {  // lane-ordered copy of the padded layout
        cudaFree(c->d_cm_ray);
        cudaFree(c->d_cm_w);
        cudaFree(c->d_lane_desc);
        c->d_cm_ray = nullptr;
        c->d_cm_w = nullptr;
        c->d_lane_desc = nullptr;
        USPG_CUDA(c, cudaMalloc(&c->d_cm_ray, sizeof(uint32_t) * (sell + kSlice)));
        USPG_CUDA(c, cudaMalloc(&c->d_cm_w, sizeof(WT) * (sell + kSlice)));
        USPG_CUDA(c, cudaMemsetAsync(c->d_cm_ray, 0, sizeof(uint32_t) * (sell + kSlice), s));
        USPG_CUDA(c, cudaMemsetAsync(c->d_cm_w, 0, sizeof(WT) * (sell + kSlice), s));
        c->cap_cm = sell + kSlice;
        c->store_moved = true;
    }
    if (!c->d_lane_desc) {
        USPG_CUDA(c, cudaMalloc(&c->d_lane_desc, sizeof(uint16_t) * 32 * n_slices * nreps));
        c->store_moved = true;
    }
    // pass 2: scatter each row entry to its cell's column, then sort it into the
    // lane-ordered store
    // (a source's columns are finished before its mirror's: sources come first)
    k_slice_desc<<<nblk(all_slices, 256), 256, 0, s>>>(c->d_slice_desc, c->d_slice_off, c->d_slice_meta,
                                                        c->d_gen_small, n_slices, all_slices);
    launch_counter()++;
    c->gen_derived_reps = 0;
    for (int rep = 0; rep < nreps; rep++) {
        const long long *rp = c->d_row_ptr + (long long)rep * n_rows;
        const int *cn = d_counts + (long long)rep * n_rows;
        const long long *so = c->d_slice_off + rep * n_slices;
        if (cols_from_src[rep]) {
            const int src = sp.src[rep];
            k_derive_columns<WT><<<nblk(n_slices * 32, 256), 256, 0, s>>>(
                n_slices, c->slices_per_slab, g, c->d_ring, sp.shift[rep], c->d_slice_meta + rep * n_slices, so,
                c->d_slice_off + src * n_slices, c->d_lane_desc + 32 * src * n_slices, c->d_sray, (WT *)c->d_sw,
                c->d_lane_desc + 32 * rep * n_slices, c->d_cm_ray, (WT *)c->d_cm_w);
            launch_counter()++;
            USPG_CUDA(c, cudaGetLastError());
            c->gen_derived_reps++;
            continue;
        }
        USPG_CUDA(c, cudaMemsetAsync(d_cell_fill, 0, sizeof(int) * c->n_cells, s));
        k_cell_scatter<WT><<<nblk((long long)n_rows * 32, 256), 256, 0, s>>>(
            rp, cn, c->d_idx, (const WT *)c->d_w, n_rows, M, c->d_ring, c->cells_per_slab, c->slices_per_slab, so,
            d_cell_fill, c->d_sray, (WT *)c->d_sw);
        launch_counter()++;
        // the scatter's slot counters now hold every cell's count
        k_cell_order<WT><<<nblk(n_slices * 32, 256), 256, 0, s>>>(
            n_slices, c->d_slice_meta + rep * n_slices, so, c->d_ring, c->cells_per_slab, d_cell_fill, c->d_sray,
            (WT *)c->d_sw, c->d_lane_desc + 32 * rep * n_slices, c->d_cm_ray, (WT *)c->d_cm_w);
        launch_counter()++;
        USPG_CUDA(c, cudaGetLastError());
    }
    if (nnz_pad / kRowPad + 1 > c->cap_grp) {
        cudaFree(c->d_grp_ray);
        c->d_grp_ray = nullptr;
        USPG_CUDA(c, cudaMalloc(&c->d_grp_ray, sizeof(uint32_t) * (nnz_pad / kRowPad + 1)));
        c->cap_grp = nnz_pad / kRowPad + 1;
        c->store_moved = true;
    }
    k_group_rays<<<nblk(nrows * 32, 256), 256, 0, s>>>(c->d_row_ptr, nrows, n_rows, c->d_grp_ray);
    launch_counter()++;

    USPG_CUDA(c, cudaStreamSynchronize(s));

    c->gen.n_reps = nreps;
    c->gen.nnz = nnz;
    c->gen.nnz_reps_full = nnz_full;
    c->gen.nnz_pad = nnz_pad;
    c->gen.sell_entries = sell;
    c->gen.max_row = maxrow;
    return USPG_OK;
}

uspg_status build_store(uspg_ctx *c, cudaStream_t s)
{
    if (!c->d_bdir) {
        USPG_CUDA(c, cudaMalloc(&c->d_bdir, sizeof(double2) * c->cells_per_slab));
        USPG_CUDA(c, cudaMalloc(&c->d_bdirf, sizeof(float2) * c->cells_per_slab));
        k_boundaries<<<c->n_rings, 128, 0, s>>>(c->d_ring, c->n_rings, c->d_bdir, c->d_bdirf);
        launch_counter()++;
        USPG_CUDA(c, cudaGetLastError());
    }
    if (c->dtype == USPG_F16) return build_typed<__half>(c, s);
    if (c->dtype == USPG_BF16) return build_typed<__nv_bfloat16>(c, s);
    return build_typed<float>(c, s);
}

}  // namespace uspg
