// MART kernels (Sec. III.D, Eq. 17-19).
//
// Every view k reuses the rows stored for its representative: a stored entry
// (slab, ring, sector) of the representative becomes, in view k, cell
// slab*C + H_ring + (sector + q) mod n_g(ring) with q = (m_k mod G) * n_g/G,
// where m_k is the number of 1/G turns between the view and its
// representative (Sec. III.C: rotating the source about z moves only the
// angular position of a segment; slab and ring are unchanged).
//
// Per-view simultaneous schedule, two launches per view:
//   k_forward   one warp per ray streams the ray-major row with 16-byte
//               loads, gathers the rotated image values and reduces the ray
//               sum with warp shuffles (Eq. 17); it stores ln(P/Pbar) per ray
//               (-inf for P = 0, NaN for a ray that is skipped).
//   k_backward  one warp per 32-cell slice of the cell-major store: each lane
//               owns one cell, streams its rays and applies
//               f *= exp(lambda * sum w ln(P/Pbar) / sum w)   (0 if any P = 0).
//               No atomics: the store is transposed once at build time.
// Faithful ray-sequential schedule: k_sequential, one warp that keeps the
// image in shared memory (or global memory for large grids) and walks
// iterations -> views -> rays in order, prefetching the next row into
// registers while the current ray is reduced and corrected.
#include "internal.cuh"

#include <algorithm>
#include <cmath>
#include <mutex>

namespace uspg {

int64_t &launch_counter()
{
    static int64_t n = 0;
    return n;
}

StoreView store_view(const uspg_ctx *c, int rep)
{
    StoreView v;
    v.row_ptr = c->d_row_ptr + (long long)rep * c->n_rays;
    v.idx = c->d_idx;
    v.w = c->d_w;
    v.rowmax = c->d_rowmax + (long long)rep * c->n_rays;
    v.slice_off = c->d_slice_off + (long long)rep * c->slices_per_rep;
    v.slice_meta = c->d_slice_meta + (long long)rep * c->slices_per_rep;
    v.slice_width = c->d_slice_width + (long long)rep * c->slices_per_rep;
    v.sray = c->d_sray;
    v.sw = c->d_sw;
    return v;
}

// ---- weight loads ------------------------------------------------------------

__device__ __forceinline__ float4 load_w4(const float *w, long long q) { return *(const float4 *)(w + q); }
__device__ __forceinline__ float4 load_w4(const __half *w, long long q)
{
    uint2 u = *(const uint2 *)(w + q);
    float2 a = __half22float2(*(const __half2 *)&u.x), b = __half22float2(*(const __half2 *)&u.y);
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float4 load_w4(const __nv_bfloat16 *w, long long q)
{
    uint2 u = *(const uint2 *)(w + q);
    float2 a = __bfloat1622float2(*(const __nv_bfloat162 *)&u.x), b = __bfloat1622float2(*(const __nv_bfloat162 *)&u.y);
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float load_w1(const float *w, long long q) { return w[q]; }
__device__ __forceinline__ float load_w1(const __half *w, long long q) { return __half2float(w[q]); }
__device__ __forceinline__ float load_w1(const __nv_bfloat16 *w, long long q) { return __bfloat162float(w[q]); }

// rotated cell id of a stored entry; tab[ring] = {head, ng, q, 0}
__device__ __forceinline__ long long rot_cell(const int4 *tab, long long cps, uint32_t pc)
{
    int4 t = tab[cell_ring(pc)];
    int s = cell_sector(pc) + t.z;
    s = s >= t.y ? s - t.y : s;
    return (long long)cell_slab(pc) * cps + t.x + s;
}

__device__ __forceinline__ void fill_tab(int4 *tab, const RingEntry *rt, int n_rings, int mG, int tid, int nt)
{
    for (int i = tid; i < n_rings; i += nt) {
        RingEntry e = rt[i];
        tab[i] = make_int4(e.head, e.ng, mG * e.step, 0);
    }
}

// ---- per-view forward ----------------------------------------------------------

template <typename WT>
__global__ void __launch_bounds__(256) k_forward(const long long *__restrict__ row_ptr, const uint32_t *__restrict__ idx,
                                                 const WT *__restrict__ w, const float *__restrict__ f,
                                                 const RingEntry *__restrict__ rt, int n_rings, int mG, long long cps,
                                                 const float *__restrict__ proj, int n_rays, float w_scale,
                                                 float *__restrict__ out_s, float *__restrict__ out_res)
{
    extern __shared__ int4 tab[];
    fill_tab(tab, rt, n_rings, mG, threadIdx.x, blockDim.x);
    __syncthreads();
    int ray = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    int lane = threadIdx.x & 31;
    if (ray >= n_rays) return;
    long long b = row_ptr[ray], e = row_ptr[ray + 1];
    float acc = 0.0f;
    // two 128-entry chunks per pass: all stream loads are issued before the
    // eight dependent image gathers, so a typical row costs one round trip
    // for the row and one for the gathers
    for (long long q0 = b + 4 * lane; q0 < e; q0 += 256) {
        long long q1 = q0 + 128;
        bool two = q1 < e;
        uint4 i0 = __ldg((const uint4 *)(idx + q0));
        float4 w0 = load_w4(w, q0);
        uint4 i1 = make_uint4(0, 0, 0, 0);
        float4 w1 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (two) {
            i1 = __ldg((const uint4 *)(idx + q1));
            w1 = load_w4(w, q1);
        }
        float g0 = __ldg(f + rot_cell(tab, cps, i0.x)), g1 = __ldg(f + rot_cell(tab, cps, i0.y));
        float g2 = __ldg(f + rot_cell(tab, cps, i0.z)), g3 = __ldg(f + rot_cell(tab, cps, i0.w));
        float h0 = 0.f, h1 = 0.f, h2 = 0.f, h3 = 0.f;
        if (two) {
            h0 = __ldg(f + rot_cell(tab, cps, i1.x));
            h1 = __ldg(f + rot_cell(tab, cps, i1.y));
            h2 = __ldg(f + rot_cell(tab, cps, i1.z));
            h3 = __ldg(f + rot_cell(tab, cps, i1.w));
        }
        acc = fmaf(w0.x, g0, acc);
        acc = fmaf(w0.y, g1, acc);
        acc = fmaf(w0.z, g2, acc);
        acc = fmaf(w0.w, g3, acc);
        acc = fmaf(w1.x, h0, acc);
        acc = fmaf(w1.y, h1, acc);
        acc = fmaf(w1.z, h2, acc);
        acc = fmaf(w1.w, h3, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        float s = acc * w_scale;
        if (out_s) out_s[ray] = s;
        if (out_res) {
            float res;
            if (e == b || !(s > 0.0f)) {
                res = __int_as_float(0x7fc00000);  // skip this ray
            } else {
                float p = proj[ray];
                res = p > 0.0f ? logf(p / s) : -INFINITY;
            }
            out_res[ray] = res;
        }
    }
}

// ---- per-view correction (cell-major) -----------------------------------------

template <typename WT>
__global__ void __launch_bounds__(256) k_backward(const long long *__restrict__ slice_off,
                                                  const uint32_t *__restrict__ slice_meta,
                                                  const int *__restrict__ slice_width, const uint32_t *__restrict__ sray,
                                                  const WT *__restrict__ sw, const float *__restrict__ res,
                                                  float *__restrict__ f, const RingEntry *__restrict__ rt, int mG,
                                                  long long cps, long long n_slices, float lambda)
{
    long long sl = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (sl >= n_slices) return;
    uint32_t meta = slice_meta[sl];
    int width = slice_width[sl];
    long long off = slice_off[sl] + lane;
    int ring = cell_ring(meta);
    RingEntry re = rt[ring];
    int sec = cell_sector(meta) + lane;
    bool own = sec < re.ng;
    int s2 = sec + mG * re.step;
    s2 = s2 >= re.ng ? s2 - re.ng : s2;
    long long cell = (long long)cell_slab(meta) * cps + re.head + s2;
    float fv = own ? f[cell] : 0.0f;  // issued early, used at the end
    float num = 0.0f, den = 0.0f;
    bool zero = false;
    // four entries per pass: stream loads first, then the ray gathers
    for (int t = 0; t < width; t += 4) {
        uint32_t ry[4];
        float wv[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            long long pos = off + (long long)(t + u) * kSlice;
            bool in = t + u < width;
            ry[u] = in ? __ldg(sray + pos) : 0u;
            wv[u] = in ? load_w1(sw, pos) : 0.0f;
        }
        float r[4];
#pragma unroll
        for (int u = 0; u < 4; u++) r[u] = __ldg(res + ry[u]);
#pragma unroll
        for (int u = 0; u < 4; u++) {
            bool act = (wv[u] > 0.0f) && (r[u] == r[u]);
            bool zr = act && (r[u] == -INFINITY);
            den += act ? wv[u] : 0.0f;
            zero |= zr;
            num += (act && !zr) ? wv[u] * r[u] : 0.0f;
        }
    }
    if (own && den > 0.0f) f[cell] = zero ? 0.0f : fv * expf(lambda * (num / den));
}

// ---- per-view forward: entry-parallel ------------------------------------------
//
// Rows of the ray-major store start and end on multiples of kRowPad (= 8)
// entries, so every aligned group of 8 entries belongs to one ray (grp_ray).
// Each lane takes one group: two 16-byte index loads, the weights, eight
// independent image gathers; lanes holding the same ray (consecutive) are
// combined by a segmented shuffle reduction and the first lane of each ray
// segment adds the partial sum into sacc[ray].  The coefficient stream is
// read with evict-first loads (__ldcs) so the image stays in L2 across views.
// k_forward_finalize turns the sums into ln(P/Pbar) and clears sacc.

__device__ __forceinline__ void load_w8(const float *w, long long q, float o[8])
{
    float4 a = __ldcs((const float4 *)(w + q)), b = __ldcs((const float4 *)(w + q + 4));
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
}
__device__ __forceinline__ void load_w8(const __half *w, long long q, float o[8])
{
    uint4 u = __ldcs((const uint4 *)(w + q));
    const __half2 *h = (const __half2 *)&u;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        float2 v = __half22float2(h[i]);
        o[2 * i] = v.x;
        o[2 * i + 1] = v.y;
    }
}
__device__ __forceinline__ void load_w8(const __nv_bfloat16 *w, long long q, float o[8])
{
    uint4 u = __ldcs((const uint4 *)(w + q));
    const __nv_bfloat162 *h = (const __nv_bfloat162 *)&u;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        float2 v = __bfloat1622float2(h[i]);
        o[2 * i] = v.x;
        o[2 * i + 1] = v.y;
    }
}
__device__ __forceinline__ float load_cs(const float *w, long long q) { return __ldcs(w + q); }
__device__ __forceinline__ float load_cs(const __half *w, long long q)
{
    return __half2float(__ushort_as_half(__ldcs((const unsigned short *)(w + q))));
}
__device__ __forceinline__ float load_cs(const __nv_bfloat16 *w, long long q)
{
    return __bfloat162float(__ushort_as_bfloat16(__ldcs((const unsigned short *)(w + q))));
}

template <typename WT>
struct Group8 {
    uint32_t c[8];
    float w[8];
    uint32_t ray;
};

template <typename WT>
__device__ __forceinline__ void load_group(Group8<WT> &G, const uint32_t *idx, const WT *w, const uint32_t *grp_ray,
                                           long long g, bool valid)
{
    if (valid) {
        long long q = g * kRowPad;
        uint4 ia = __ldcs((const uint4 *)(idx + q)), ib = __ldcs((const uint4 *)(idx + q + 4));
        load_w8(w, q, G.w);
        G.ray = __ldcs(grp_ray + g);
        G.c[0] = ia.x; G.c[1] = ia.y; G.c[2] = ia.z; G.c[3] = ia.w;
        G.c[4] = ib.x; G.c[5] = ib.y; G.c[6] = ib.z; G.c[7] = ib.w;
    } else {
#pragma unroll
        for (int i = 0; i < 8; i++) {
            G.c[i] = 0;
            G.w[i] = 0.0f;
        }
        G.ray = 0xffffffffu;
    }
}

template <typename WT>
__global__ void __launch_bounds__(256) k_forward_flat(const uint32_t *__restrict__ idx, const WT *__restrict__ w,
                                                      const uint32_t *__restrict__ grp_ray, long long g0,
                                                      long long n_groups, const float *__restrict__ f,
                                                      const RingEntry *__restrict__ rt, int n_rings, int mG,
                                                      long long cps, float *__restrict__ sacc)
{
    extern __shared__ int4 tab[];
    fill_tab(tab, rt, n_rings, mG, threadIdx.x, blockDim.x);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long step = (((long long)gridDim.x * blockDim.x) >> 5) * 32;
    long long base = gw * 32;
    if (base >= n_groups) return;
    // two register buffers: the next chunk's stream loads are in flight while
    // the current chunk's gathers wait
    Group8<WT> cur, nxt;
    load_group(cur, idx, w, grp_ray, g0 + base + lane, base + lane < n_groups);
    for (; base < n_groups; base += step) {
        long long nb = base + step;
        load_group(nxt, idx, w, grp_ray, g0 + nb + lane, nb + lane < n_groups);
        float gv[8];
#pragma unroll
        for (int i = 0; i < 8; i++) gv[i] = cur.w[i] != 0.0f ? __ldg(f + rot_cell(tab, cps, cur.c[i])) : 0.0f;
        float acc = 0.0f;
#pragma unroll
        for (int i = 0; i < 8; i++) acc = fmaf(cur.w[i], gv[i], acc);
        uint32_t ray = cur.ray;
        // segmented sum over lanes of the same ray (they are consecutive)
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            float v2 = __shfl_down_sync(0xffffffffu, acc, o);
            uint32_t r2 = __shfl_down_sync(0xffffffffu, ray, o);
            if (lane + o < 32 && r2 == ray) acc += v2;
        }
        uint32_t rprev = __shfl_up_sync(0xffffffffu, ray, 1);
        if (ray != 0xffffffffu && (lane == 0 || rprev != ray)) atomicAdd(&sacc[ray], acc);
        cur = nxt;
    }
}

__global__ void k_forward_finalize(float *__restrict__ sacc, const float *__restrict__ proj, int n_rays, float w_scale,
                                   float *__restrict__ out_s, float *__restrict__ out_res)
{
    int ray = blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= n_rays) return;
    float sv = sacc[ray] * w_scale;
    sacc[ray] = 0.0f;
    if (out_s) out_s[ray] = sv;
    if (out_res) {
        float res;
        if (!(sv > 0.0f)) {
            res = __int_as_float(0x7fc00000);  // empty row or zero sum: skip this ray
        } else {
            float p = proj[ray];
            res = p > 0.0f ? logf(p / sv) : -INFINITY;
        }
        out_res[ray] = res;
    }
}

// ---- per-view correction: lane-ordered cell-major store --------------------------
//
// One warp takes SPW slices (32 cells each).  Lane l of a slice owns the cell
// of its source lane (lane_desc) and its count n; its t-th ray is at
// slice_off + 32 t + l for t < n.  All stream loads of the warp's slices are
// issued before the ray-value gathers, and the image value of each cell is
// fetched first so that its latency overlaps the stream.
struct SliceDesc {
    uint32_t d, m, off;
};

__device__ __forceinline__ void load_desc(SliceDesc &D, const long long *slice_off, long long base,
                                          const uint32_t *slice_meta, const uint16_t *lane_desc, long long sl,
                                          long long n_slices, int lane)
{
    if (sl < n_slices) {
        D.d = lane_desc[sl * 32 + lane];
        D.m = slice_meta[sl];
        D.off = (uint32_t)(slice_off[sl] - base);
    } else {
        D.d = 0;
        D.m = 0;
        D.off = 0;
    }
}

// rows 0..R-1 of one lane: loads first, then the ray-value gathers
template <typename WT, int R>
__device__ __forceinline__ void cm_rows(const uint32_t *cray, const WT *cw, const float *res, uint32_t off, int cnt,
                                        float &num, float &den, bool &zero)
{
    uint32_t ry[R];
    float wv[R], rv[R];
#pragma unroll
    for (int t = 0; t < R; t++) {
        bool in = t < cnt;
        uint32_t pos = off + (uint32_t)t * kSlice;
        ry[t] = in ? __ldcs(cray + pos) : 0u;
        wv[t] = in ? load_cs(cw, pos) : 0.0f;
    }
#pragma unroll
    for (int t = 0; t < R; t++) rv[t] = t < cnt ? __ldg(res + ry[t]) : 0.f;
#pragma unroll
    for (int t = 0; t < R; t++) {
        bool act = (wv[t] > 0.0f) && (rv[t] == rv[t]);
        bool zr = act && (rv[t] == -INFINITY);
        den += act ? wv[t] : 0.0f;
        zero |= zr;
        num += (act && !zr) ? wv[t] * rv[t] : 0.0f;
    }
}

// Persistent warps, one slice per step: the next slice's descriptor loads are
// issued before the current slice's gathers.  The slice's widest column is
// lane 0's (lanes are ordered by count), so the unrolled row loop is sized
// per slice (warp-uniform) to 2, 4 or 8 rows, with a loop beyond.
template <typename WT>
__global__ void __launch_bounds__(256) k_backward_sell(const long long *__restrict__ slice_off, long long base,
                                                       const uint32_t *__restrict__ slice_meta,
                                                       const uint16_t *__restrict__ lane_desc,
                                                       const uint32_t *__restrict__ cray, const WT *__restrict__ cw,
                                                       const float *__restrict__ res, float *__restrict__ f,
                                                       const RingEntry *__restrict__ rt, int mG, long long cps,
                                                       long long n_slices, float lambda)
{
    const int lane = threadIdx.x & 31;
    const long long wg = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long W = ((long long)gridDim.x * blockDim.x) >> 5;
    long long sl = wg;
    if (sl >= n_slices) return;
    const uint32_t *cr = cray + base;
    const WT *cwb = cw + base;
    SliceDesc cur, nxt;
    load_desc(cur, slice_off, base, slice_meta, lane_desc, sl, n_slices, lane);
    for (; sl < n_slices; sl += W) {
        int cnt = (int)(cur.d & 2047u);
        int width = __shfl_sync(0xffffffffu, cnt, 0);
        RingEntry re = rt[cell_ring(cur.m)];
        int sec = cell_sector(cur.m) + (int)(cur.d >> 11);
        int s2 = sec + mG * re.step;
        s2 = s2 >= re.ng ? s2 - re.ng : s2;
        long long cell = (long long)cell_slab(cur.m) * cps + re.head + s2;
        float fv = cnt > 0 ? f[cell] : 0.0f;
        uint32_t off = cur.off + lane;
        load_desc(nxt, slice_off, base, slice_meta, lane_desc, sl + W, n_slices, lane);
        float num = 0.f, den = 0.f;
        bool zero = false;
        if (width <= 2) {
            cm_rows<WT, 2>(cr, cwb, res, off, cnt, num, den, zero);
        } else if (width <= 4) {
            cm_rows<WT, 4>(cr, cwb, res, off, cnt, num, den, zero);
        } else {
            cm_rows<WT, 8>(cr, cwb, res, off, cnt, num, den, zero);
            for (int t = 8; t < cnt; t++) {  // long columns (cells close to the source)
                uint32_t pos = off + (uint32_t)t * kSlice;
                float wt = load_cs(cwb, pos);
                float r = __ldg(res + __ldcs(cr + pos));
                bool act = (wt > 0.0f) && (r == r);
                bool zr = act && (r == -INFINITY);
                den += act ? wt : 0.0f;
                zero |= zr;
                num += (act && !zr) ? wt * r : 0.0f;
            }
        }
        if (den > 0.0f) f[cell] = zero ? 0.0f : fv * expf(lambda * (num / den));
        cur = nxt;
    }
}

template <typename WT>
static uspg_status fwd_typed(uspg_ctx *c, int view, float *out_s, float *out_res, cudaStream_t s)
{
    int rep = c->rep_of_view[view];
    int mG = c->m_of_view[view] % c->G;
    const long long *rp = c->d_row_ptr + (long long)rep * c->n_rays;
    long long g0 = c->h_rep_entry0[rep] / kRowPad, ng = (c->h_rep_entry0[rep + 1] - c->h_rep_entry0[rep]) / kRowPad;
    (void)rp;
    const int TB = 256;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = c->fwd_blocks_per_sm > 0 ? c->fwd_blocks_per_sm : 8;
    long long want = (ng + TB - 1) / TB;  // one group per thread
    long long grid = std::min<long long>(want, (long long)sms * per_sm);
    if (grid < 1) grid = 1;
    size_t smem = sizeof(int4) * c->n_rings;
    k_forward_flat<WT><<<(unsigned)grid, TB, smem, s>>>(c->d_idx, (const WT *)c->d_w, c->d_grp_ray, g0, ng, c->d_f,
                                                        c->d_ring, c->n_rings, mG, c->cells_per_slab, c->d_sacc);
    launch_counter()++;
    USPG_CUDA(c, cudaGetLastError());
    k_forward_finalize<<<(unsigned)((c->n_rays + 255) / 256), 256, 0, s>>>(
        c->d_sacc, c->d_proj + (long long)view * c->n_rays, c->n_rays, (float)c->w_scale, out_s, out_res);
    launch_counter()++;
    USPG_CUDA(c, cudaGetLastError());
    return USPG_OK;
}

uspg_status launch_forward_view(uspg_ctx *c, int view, float *out_s, float *out_res, cudaStream_t s)
{
    if (c->dtype == USPG_F16) return fwd_typed<__half>(c, view, out_s, out_res, s);
    if (c->dtype == USPG_BF16) return fwd_typed<__nv_bfloat16>(c, view, out_s, out_res, s);
    return fwd_typed<float>(c, view, out_s, out_res, s);
}

template <typename WT>
static uspg_status bwd_typed(uspg_ctx *c, int view, float lambda, cudaStream_t s)
{
    int rep = c->rep_of_view[view];
    int mG = c->m_of_view[view] % c->G;
    const long long S = c->slices_per_rep;
    const int TB = 256;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = c->bwd_blocks_per_sm > 0 ? c->bwd_blocks_per_sm : 8;
    long long want = (S * 32 + TB - 1) / TB;
    long long grid = std::min<long long>(want, (long long)sms * per_sm);
    if (grid < 1) grid = 1;
    long long base = c->h_sell_base[rep];
    k_backward_sell<WT><<<(unsigned)grid, TB, 0, s>>>(c->d_slice_off + rep * S, base, c->d_slice_meta + rep * S,
                                                      c->d_lane_desc + 32 * rep * S, c->d_cm_ray, (const WT *)c->d_cm_w,
                                                      c->d_res, c->d_f, c->d_ring, mG, c->cells_per_slab, S, lambda);
    launch_counter()++;
    USPG_CUDA(c, cudaGetLastError());
    return USPG_OK;
}

uspg_status launch_backward_view(uspg_ctx *c, int view, float lambda, cudaStream_t s)
{
    if (c->dtype == USPG_F16) return bwd_typed<__half>(c, view, lambda, s);
    if (c->dtype == USPG_BF16) return bwd_typed<__nv_bfloat16>(c, view, lambda, s);
    return bwd_typed<float>(c, view, lambda, s);
}

// ---- faithful ray-sequential MART -----------------------------------------------

constexpr int kSeqChunks = 8;  // rows up to 256 entries live in registers

template <typename WT>
struct RowRegs {
    uint32_t ix[kSeqChunks];
    float w[kSeqChunks];
};

template <typename WT>
__device__ __forceinline__ void seq_load(RowRegs<WT> &R, const uint32_t *idx, const WT *w, long long b, long long e,
                                         int lane)
{
#pragma unroll
    for (int c = 0; c < kSeqChunks; c++) {
        long long q = b + c * 32 + lane;
        if (q < e) {
            R.ix[c] = __ldg(idx + q);
            R.w[c] = load_w1(w, q);
        } else {
            R.ix[c] = 0;
            R.w[c] = 0.0f;
        }
    }
}

// One warp.  f in shared memory when SMEM, else in global memory.
template <typename WT, bool SMEM>
__global__ void __launch_bounds__(32) k_sequential(const long long *__restrict__ row_ptr_all,
                                                   const uint32_t *__restrict__ idx, const WT *__restrict__ w,
                                                   const float *__restrict__ rowmax_all,
                                                   const int *__restrict__ view_rep, const int *__restrict__ view_mg,
                                                   int n_views, int n_rays, const float *__restrict__ proj,
                                                   float *f_g, long long n_cells, const RingEntry *__restrict__ rt,
                                                   int n_rings, long long cps, int iters, float lambda, int rule,
                                                   float tol, float w_scale, int *sweeps_out)
{
    extern __shared__ float4 smem4[];
    float *sm = (float *)smem4;
    const int lane = threadIdx.x;
    long long fcells = SMEM ? ((n_cells + 3) & ~3LL) : 0;
    float *fs = SMEM ? sm : f_g;
    int4 *tab = (int4 *)(sm + fcells);
    if (SMEM) {
        for (long long q = lane; q < n_cells; q += 32) fs[q] = f_g[q];
    }
    __syncwarp();
    int it = 0;
    for (; it < iters; it++) {
        int changed = 0;
        for (int k = 0; k < n_views; k++) {
            int rep = view_rep[k];
            fill_tab(tab, rt, n_rings, view_mg[k], lane, 32);
            __syncwarp();
            const long long *rp = row_ptr_all + (long long)rep * n_rays;
            const float *rmax = rowmax_all + (long long)rep * n_rays;
            const float *pk = proj + (long long)k * n_rays;
            RowRegs<WT> cur, nxt;
            long long cb = rp[0], ce = rp[1];
            seq_load(cur, idx, w, cb, ce, lane);
            for (int ray = 0; ray < n_rays; ray++) {
                long long nb = ce, ne = ce;
                if (ray + 1 < n_rays) {
                    ne = rp[ray + 2];
                    seq_load(nxt, idx, w, nb, ne, lane);
                }
                if (ce > cb) {
                    float acc = 0.0f;
                    long long cell[kSeqChunks];
#pragma unroll
                    for (int c = 0; c < kSeqChunks; c++) {
                        cell[c] = rot_cell(tab, cps, cur.ix[c]);
                        acc = fmaf(cur.w[c], fs[cell[c]], acc);
                    }
                    for (long long q = cb + kSeqChunks * 32 + lane; q < ce; q += 32)  // long rows
                        acc = fmaf(load_w1(w, q), fs[rot_cell(tab, cps, __ldg(idx + q))], acc);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                    float s = acc * w_scale;
                    if (s > 0.0f) {
                        float ratio = pk[ray] / s;
                        float l2 = log2f(ratio);
                        float ex = lambda / rmax[ray];
                        float lin = 1.0f - lambda * (1.0f - ratio);
#pragma unroll
                        for (int c = 0; c < kSeqChunks; c++) {
                            if (cur.w[c] > 0.0f) {
                                float old = fs[cell[c]];
                                float fac = rule == USPG_LINEAR_EQ18 ? lin : exp2f(ex * cur.w[c] * l2);
                                float nv = old * fac;
                                if (tol > 0.0f && fabsf(nv - old) > tol * fabsf(old)) changed = 1;
                                fs[cell[c]] = nv;
                            }
                        }
                        for (long long q = cb + kSeqChunks * 32 + lane; q < ce; q += 32) {
                            float wv = load_w1(w, q);
                            if (wv > 0.0f) {
                                long long cl = rot_cell(tab, cps, __ldg(idx + q));
                                float old = fs[cl];
                                float fac = rule == USPG_LINEAR_EQ18 ? lin : exp2f(ex * wv * l2);
                                float nv = old * fac;
                                if (tol > 0.0f && fabsf(nv - old) > tol * fabsf(old)) changed = 1;
                                fs[cl] = nv;
                            }
                        }
                    }
                    __syncwarp();
                    if (!SMEM) __threadfence_block();
                }
                cur = nxt;
                cb = nb;
                ce = ne;
            }
            __syncwarp();
        }
        if (tol > 0.0f) {
            if (!__any_sync(0xffffffffu, changed)) {
                it++;
                break;
            }
        }
    }
    if (SMEM) {
        __syncwarp();
        for (long long q = lane; q < n_cells; q += 32) f_g[q] = fs[q];
    }
    if (lane == 0 && sweeps_out) *sweeps_out = it;
}

template <typename WT>
static uspg_status seq_typed(uspg_ctx *c, const uspg_mart_opts *o, cudaStream_t s)
{
    int nv = c->scan.n_views;
    std::vector<int> vr(nv), vm(nv);
    for (int k = 0; k < nv; k++) {
        vr[k] = c->rep_of_view[k];
        vm[k] = c->m_of_view[k] % c->G;
    }
    int *d_v = nullptr;
    USPG_CUDA(c, cudaMallocAsync(&d_v, sizeof(int) * 2 * nv, s));
    USPG_CUDA(c, cudaMemcpyAsync(d_v, vr.data(), sizeof(int) * nv, cudaMemcpyHostToDevice, s));
    USPG_CUDA(c, cudaMemcpyAsync(d_v + nv, vm.data(), sizeof(int) * nv, cudaMemcpyHostToDevice, s));
    size_t tab_bytes = sizeof(int4) * c->n_rings;
    size_t f_bytes = sizeof(float) * ((c->n_cells + 3) & ~3LL);
    int dev = 0, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    bool use_smem = f_bytes + tab_bytes <= (size_t)max_smem;
    float tol = (float)o->stop_tol;
    if (use_smem) {
        size_t sm = f_bytes + tab_bytes;
        USPG_CUDA(c, cudaFuncSetAttribute(k_sequential<WT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_sequential<WT, true><<<1, 32, sm, s>>>(c->d_row_ptr, c->d_idx, (const WT *)c->d_w, c->d_rowmax, d_v, d_v + nv,
                                                 nv, c->n_rays, c->d_proj, c->d_f, c->n_cells, c->d_ring, c->n_rings,
                                                 c->cells_per_slab, o->iterations, (float)o->lambda, o->update_rule, tol,
                                                 (float)c->w_scale, c->d_sweeps);
    } else {
        k_sequential<WT, false><<<1, 32, tab_bytes, s>>>(c->d_row_ptr, c->d_idx, (const WT *)c->d_w, c->d_rowmax, d_v,
                                                         d_v + nv, nv, c->n_rays, c->d_proj, c->d_f, c->n_cells,
                                                         c->d_ring, c->n_rings, c->cells_per_slab, o->iterations,
                                                         (float)o->lambda, o->update_rule, tol, (float)c->w_scale,
                                                         c->d_sweeps);
    }
    launch_counter()++;
    USPG_CUDA(c, cudaGetLastError());
    USPG_CUDA(c, cudaFreeAsync(d_v, s));
    return USPG_OK;
}

uspg_status launch_sequential(uspg_ctx *c, const uspg_mart_opts *o, cudaStream_t s)
{
    if (c->dtype == USPG_F16) return seq_typed<__half>(c, o, s);
    if (c->dtype == USPG_BF16) return seq_typed<__nv_bfloat16>(c, o, s);
    return seq_typed<float>(c, o, s);
}

// ---- forward projection without device allocation ---------------------------------
//
// The ray-sum accumulator of uspg_forward_project_noalloc lives in this
// file-scope array instead of a context allocation.  Host code must not use
// the symbol as an address: it is resolved per device with
// cudaGetSymbolAddress and cached.
static __device__ __align__(256) float g_noalloc_acc[USPG_NOALLOC_MAX_RAYS];

__global__ void k_clear_acc(float *acc, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) acc[i] = 0.0f;
}

constexpr int kMaxDevices = 64;

// device address of g_noalloc_acc on the current device (looked up once)
static cudaError_t noalloc_acc(float **out)
{
    static std::mutex mu;
    static float *addr[kMaxDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_acc);
        if (e != cudaSuccess) return e;
        addr[dev] = (float *)p;
    }
    *out = addr[dev];
    return cudaSuccess;
}

template <typename WT>
static uspg_status fwd_noalloc_typed(uspg_ctx *c, int view, const float *f, float *out, float *acc, cudaStream_t s)
{
    int rep = c->rep_of_view[view];
    int mG = c->m_of_view[view] % c->G;
    long long g0 = c->h_rep_entry0[rep] / kRowPad, ng = (c->h_rep_entry0[rep + 1] - c->h_rep_entry0[rep]) / kRowPad;
    const int TB = 256;
    k_clear_acc<<<(unsigned)((c->n_rays + TB - 1) / TB), TB, 0, s>>>(acc, c->n_rays);
    launch_counter()++;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = c->fwd_blocks_per_sm > 0 ? c->fwd_blocks_per_sm : 8;
    long long grid = std::min<long long>((ng + TB - 1) / TB, (long long)sms * per_sm);
    if (grid < 1) grid = 1;
    k_forward_flat<WT><<<(unsigned)grid, TB, sizeof(int4) * c->n_rings, s>>>(
        c->d_idx, (const WT *)c->d_w, c->d_grp_ray, g0, ng, f, c->d_ring, c->n_rings, mG, c->cells_per_slab, acc);
    launch_counter()++;
    k_forward_finalize<<<(unsigned)((c->n_rays + TB - 1) / TB), TB, 0, s>>>(acc, c->d_proj, c->n_rays,
                                                                          (float)c->w_scale, out, nullptr);
    launch_counter()++;
    USPG_CUDA(c, cudaGetLastError());
    return USPG_OK;
}

}  // namespace uspg

extern "C" uspg_status uspg_forward_project_noalloc(const uspg_ctx *cc, int32_t view, const float *f, float *out,
                                                    uspg_stream stream)
{
    using namespace uspg;
    uspg_ctx *c = const_cast<uspg_ctx *>(cc);
    if (!c || !f || !out) return fail(c, USPG_EINVAL, "NULL argument");
    if (c->n_rays > USPG_NOALLOC_MAX_RAYS)
        return fail(c, USPG_EINVAL,
                    "uspg_forward_project_noalloc: " + std::to_string(c->n_rays) + " rays per view exceed the " +
                        std::to_string(USPG_NOALLOC_MAX_RAYS) + "-ray accumulator");
    if (view < 0 || view >= c->scan.n_views) return fail(c, USPG_EINVAL, "bad view");
    if (!c->built) return fail(c, USPG_ENOTREADY, "coefficients not built");
    float *acc = nullptr;
    USPG_CUDA(c, noalloc_acc(&acc));
    cudaStream_t s = (cudaStream_t)stream;
    if (c->dtype == USPG_F16) return fwd_noalloc_typed<__half>(c, view, f, out, acc, s);
    if (c->dtype == USPG_BF16) return fwd_noalloc_typed<__nv_bfloat16>(c, view, f, out, acc, s);
    return fwd_noalloc_typed<float>(c, view, f, out, acc, s);
}
