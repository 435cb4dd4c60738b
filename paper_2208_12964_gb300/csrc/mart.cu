// MART kernels (Sec. III.D, Eq. 17-19).
//
// Every view k reuses the rows stored for its representative: a stored entry
// (slab, ring, sector) of the representative becomes, in view k, cell
// slab*C + H_ring + (sector + q) mod n_g(ring) with q = (m_k mod G) * n_g/G,
// where m_k is the number of 1/G turns between the view and its
// representative (Sec. III.C: rotating the source about z moves only the
// angular position of a segment; slab and ring are unchanged).
//
// Per-view simultaneous schedule, three launches per view:
//   k_forward_flat      lanes stream 8-entry groups of the ray-major rows with
//                       16-byte loads, gather the rotated image values and
//                       combine each ray's partial sums with warp shuffles
//                       (Eq. 17);
//   k_forward_finalize  turns each ray sum into the ray's correction term
//                       {ln(P/Pbar) or P/Pbar, 1} ({0, 0} for a ray that is
//                       skipped) and clears the accumulator;
//   k_backward_sell     one warp per 32-cell slice of the cell-major store:
//                       each lane owns one cell, gathers its rays' terms and
//                       applies the rule's weighted mean, e.g.
//                       f *= exp(lambda * sum w ln(P/Pbar) / sum w) (0 if any P = 0).
//                       No atomics: the store is transposed once at build time.
// Faithful ray-sequential schedule: k_sequential, one warp that keeps the
// image in shared memory (or global memory for large grids) and walks
// iterations -> views -> rays in order, prefetching the next row into
// registers while the current ray is reduced and corrected.
#include "internal.cuh"
#include "device.cuh"

#include <algorithm>
#include <cmath>
#include <mutex>

namespace uspg {

std::atomic<int64_t> &launch_counter()
{
    static std::atomic<int64_t> n{0};
    return n;
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
// k_forward_finalize turns the sums into correction terms and clears sacc.

// PAIRS: the image is the context's mirrored pair layout; a mirrored store
// read with a caller's standard-layout image (no-alloc projection) uses
// MIR without PAIRS.
template <typename WT, bool MIR, bool PAIRS>
__global__ void __launch_bounds__(256) k_forward_flat(const uint32_t *__restrict__ idx, const WT *__restrict__ w,
                                                      const uint32_t *__restrict__ grp_ray, long long g0,
                                                      long long n_groups, const float *__restrict__ f,
                                                      const RingEntry *__restrict__ rt, int n_rings, int mG,
                                                      long long cps, float *__restrict__ sacc, Mirror M,
                                                      const int *__restrict__ done)
{
    extern __shared__ int4 tab[];
    fill_tab(tab, rt, n_rings, mG, threadIdx.x, blockDim.x);
    __syncthreads();
    if (done) {  // Eq. 19 stop: nothing to do once the iteration has converged
        grid_dep_wait();
        if (*done) return;
    }
    fwd_groups<WT, MIR, PAIRS>(idx, w, grp_ray, g0, n_groups, f, tab, cps, sacc,
                               ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                               ((long long)gridDim.x * blockDim.x) >> 5, threadIdx.x & 31, M);
}

__global__ void k_forward_finalize(float *__restrict__ sacc, const float *__restrict__ proj, int n_rays, float w_scale,
                                   int linear, float *__restrict__ out_s, float *__restrict__ out_res,
                                   const int *__restrict__ done)
{
    grid_dep_wait();
    if (done && *done) return;
    int ray = blockIdx.x * blockDim.x + threadIdx.x;
    if (ray < n_rays) finalize_ray(sacc, proj, ray, w_scale, linear, out_s, (float2 *)out_res);
}

// z-mirror store: one thread per stored ray finalizes it and its mirror
__global__ void k_forward_finalize_pairs(float *__restrict__ sacc, const float *__restrict__ proj, Mirror M,
                                         float w_scale, int linear, float *__restrict__ out_s,
                                         float *__restrict__ out_res, const int *__restrict__ done)
{
    grid_dep_wait();
    if (done && *done) return;
    int ray = blockIdx.x * blockDim.x + threadIdx.x;
    if (ray < M.n_rows) finalize_pair(sacc, proj, ray, M, w_scale, linear, out_s, (float4 *)out_res);
}

// Eq. 19 bookkeeping of a per-view run that may stop early (stop[0] = sweeps
// run, stop[1] = some correction of the current sweep moved a cell by more
// than the tolerance, stop[2] = converged): reset before the first sweep, and
// after each sweep count it and stop if no cell moved.
__global__ void k_stop_reset(int *stop)
{
    stop[0] = 0;
    stop[1] = 0;
    stop[2] = 0;
}

__global__ void k_sweep_end(int *stop)
{
    grid_dep_wait();
    if (stop[2]) return;
    stop[0]++;
    if (!stop[1]) stop[2] = 1;
    stop[1] = 0;
}

// ---- per-view correction: lane-ordered cell-major store --------------------------
//
// Lane l of a slice owns the cell of its source lane (lane_desc) and its
// count n; its t-th ray is at slice_off + 32 t + l for t < n.  Persistent
// warps, one slice per step: the next slice's descriptor loads are issued
// before the current slice's gathers, and the image value of each cell is
// fetched first so that its latency overlaps the stream.  The slice's widest
// column is lane 0's (lanes are ordered by count), so the unrolled row loop
// is sized per slice (warp-uniform) to 2, 4 or 8 rows, with a loop beyond.
template <typename WT, bool MIR>
__global__ void __launch_bounds__(256, MIR ? kBwdMinBlocksMirror : kBwdMinBlocks)
    k_backward_sell(const uint2 *__restrict__ sdesc, const uint16_t *__restrict__ lane_desc,
                    const uint32_t *__restrict__ cray, const WT *__restrict__ cw, const float *__restrict__ res,
                    float *__restrict__ f, const RingEntry *__restrict__ rt, int n_rings, int mG, long long cps,
                    int n_slices, UpdateRule U, Mirror M, const int *__restrict__ done)
{
    extern __shared__ int4 tab[];
    fill_tab(tab, rt, n_rings, mG, threadIdx.x, blockDim.x);
    __syncthreads();
    if (done) {
        grid_dep_wait();
        if (*done) return;
    }
    bwd_slices<WT, MIR>(sdesc, lane_desc, cray, cw, res, f, tab, (uint32_t)cps, n_slices, U,
                        (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), (int)((gridDim.x * blockDim.x) >> 5),
                        threadIdx.x & 31, M);
}

// Launch with programmatic stream serialization (see grid_dep_wait).
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                              Args... args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

static int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// forward ray sums of one view into acc (cleared on entry, cleared again by
// the finalize), then out_s = sums and out_res = the rays' correction terms
// (finalize_ray / finalize_pair)
// f_pairs: f is in the context's image layout (pairs when mirrored); false
// for a caller's standard-layout image
template <typename WT>
static uspg_status fwd_run(uspg_ctx *c, int view, const float *f, bool f_pairs, float *acc, float *out_s,
                           float *out_res, const float *proj, cudaStream_t s, int linear = 0,
                           const int *done = nullptr)
{
    int rep = c->rep_of_view[view];
    int mG = c->m_of_view[view] % c->G;
    long long g0 = c->h_rep_entry0[rep] / kRowPad, ng = (c->h_rep_entry0[rep + 1] - c->h_rep_entry0[rep]) / kRowPad;
    const int TB = 256;
    int per_sm = c->fwd_blocks_per_sm > 0 ? c->fwd_blocks_per_sm : 4;  // 4 x 256 threads at 64 registers fill an SM
    long long want = (ng + TB - 1) / TB;  // one group per thread
    long long grid = std::min<long long>(want, (long long)sm_count() * per_sm);
    if (grid < 1) grid = 1;
    size_t smem = sizeof(int4) * c->n_rings;
    const uint32_t *idx = c->d_idx, *grp = c->d_grp_ray;
    const WT *w = (const WT *)c->d_w;
    const RingEntry *rt = c->d_ring;
    long long cps = c->cells_per_slab;
    cudaError_t e;
    if (c->mir.on && f_pairs)
        e = launch_pdl(k_forward_flat<WT, true, true>, (unsigned)grid, TB, smem, s, idx, w, grp, g0, ng, f, rt,
                       c->n_rings, mG, cps, acc, c->mir, done);
    else if (c->mir.on)
        e = launch_pdl(k_forward_flat<WT, true, false>, (unsigned)grid, TB, smem, s, idx, w, grp, g0, ng, f, rt,
                       c->n_rings, mG, cps, acc, c->mir, done);
    else
        e = launch_pdl(k_forward_flat<WT, false, false>, (unsigned)grid, TB, smem, s, idx, w, grp, g0, ng, f, rt,
                       c->n_rings, mG, cps, acc, c->mir, done);
    launch_counter()++;
    USPG_CUDA(c, e);
    float ws = (float)c->w_scale;
    if (c->mir.on)
        e = launch_pdl(k_forward_finalize_pairs, (unsigned)((c->mir.n_rows + 255) / 256), 256, 0, s, acc, proj,
                       c->mir, ws, linear, out_s, out_res, done);
    else
        e = launch_pdl(k_forward_finalize, (unsigned)((c->n_rays + 255) / 256), 256, 0, s, acc, proj, c->n_rays, ws,
                       linear, out_s, out_res, done);
    launch_counter()++;
    USPG_CUDA(c, e);
    return USPG_OK;
}

uspg_status launch_forward_view(uspg_ctx *c, int view, float *out_s, float *out_res, cudaStream_t s, int linear,
                                const int *done)
{
    const float *proj = c->d_proj + (long long)view * c->n_rays;
    if (c->dtype == USPG_F16)
        return fwd_run<__half>(c, view, c->d_f, true, c->d_sacc, out_s, out_res, proj, s, linear, done);
    if (c->dtype == USPG_BF16)
        return fwd_run<__nv_bfloat16>(c, view, c->d_f, true, c->d_sacc, out_s, out_res, proj, s, linear, done);
    return fwd_run<float>(c, view, c->d_f, true, c->d_sacc, out_s, out_res, proj, s, linear, done);
}

template <typename WT>
static uspg_status bwd_typed(uspg_ctx *c, int view, const UpdateRule &U, const int *done, cudaStream_t s)
{
    int rep = c->rep_of_view[view];
    int mG = c->m_of_view[view] % c->G;
    const long long S = c->slices_per_rep;
    const int TB = 256;
    int per_sm = c->bwd_blocks_per_sm > 0 ? c->bwd_blocks_per_sm : (c->mir.on ? kBwdMinBlocksMirror : kBwdMinBlocks);
    long long want = (S * 32 + TB - 1) / TB;
    long long grid = std::min<long long>(want, (long long)sm_count() * per_sm);
    if (grid < 1) grid = 1;
    long long base = c->h_sell_base[rep];
    const uint2 *sd = c->d_slice_desc + rep * S;
    const uint16_t *ld = c->d_lane_desc + 32 * rep * S;
    const uint32_t *cr = (const uint32_t *)c->d_cm_ray + base;
    const WT *cw = (const WT *)c->d_cm_w + base;
    const float *res = c->d_res;
    size_t smem = sizeof(int4) * c->n_rings;
    cudaError_t e;
    if (c->mir.on)
        e = launch_pdl(k_backward_sell<WT, true>, (unsigned)grid, TB, smem, s, sd, ld, cr, cw, res, c->d_f,
                       (const RingEntry *)c->d_ring, c->n_rings, mG, c->cells_per_slab, (int)S, U, c->mir, done);
    else
        e = launch_pdl(k_backward_sell<WT, false>, (unsigned)grid, TB, smem, s, sd, ld, cr, cw, res, c->d_f,
                       (const RingEntry *)c->d_ring, c->n_rings, mG, c->cells_per_slab, (int)S, U, c->mir, done);
    launch_counter()++;
    USPG_CUDA(c, e);
    return USPG_OK;
}

uspg_status launch_backward_view(uspg_ctx *c, int view, const UpdateRule &U, const int *done, cudaStream_t s)
{
    if (c->dtype == USPG_F16) return bwd_typed<__half>(c, view, U, done, s);
    if (c->dtype == USPG_BF16) return bwd_typed<__nv_bfloat16>(c, view, U, done, s);
    return bwd_typed<float>(c, view, U, done, s);
}

uspg_status launch_stop_reset(uspg_ctx *c, cudaStream_t s)
{
    k_stop_reset<<<1, 1, 0, s>>>(c->d_sweeps);
    launch_counter()++;
    USPG_CUDA(c, cudaGetLastError());
    return USPG_OK;
}

uspg_status launch_sweep_end(uspg_ctx *c, cudaStream_t s)
{
    cudaError_t e = launch_pdl(k_sweep_end, 1, 1, 0, s, c->d_sweeps);
    launch_counter()++;
    USPG_CUDA(c, e);
    return USPG_OK;
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

// Where the sequential kernel keeps the image: in the shared memory of its
// block when it fits; otherwise its last n_sm cells (the outer rings, which
// every ray crosses) in shared memory and the inner disk in global memory,
// which only the rays passing near the axis reach; or, when little of it
// would fit, all of it in global memory.
enum { kSeqGlobal = 0, kSeqSmem = 1, kSeqSplit = 2 };

// One warp walks iterations -> views -> rays in order.  Per ray step the
// rows of the next ray, its projection value and row maximum are already in
// flight (issued one ray ahead), and the row bounds two rays ahead, so that
// the chain of a step is the image gathers, the warp sum and the update.
template <typename WT, int MODE>
__global__ void __launch_bounds__(32) k_sequential(const long long *__restrict__ row_ptr_all,
                                                   const uint32_t *__restrict__ idx, const WT *__restrict__ w,
                                                   const float *__restrict__ rowmax_all,
                                                   const int *__restrict__ view_rep, const int *__restrict__ view_mg,
                                                   int n_views, int n_rays, Mirror M, const float *__restrict__ proj,
                                                   float *f_g, long long n_cells, const RingEntry *__restrict__ rt,
                                                   int n_rings, long long cps, int iters, float lambda, int rule,
                                                   float tol, float w_scale, long long n_sm, int *sweeps_out)
{
    extern __shared__ float4 smem4[];
    float *sm = (float *)smem4;
    const int lane = threadIdx.x;
    long long fcells = MODE == kSeqSmem ? ((n_cells + 3) & ~3LL) : (MODE == kSeqSplit ? n_sm : 0);
    // cells [lo, n_cells) live in shared memory at sm[cell - lo]
    const long long lo = MODE == kSeqSmem ? 0 : (MODE == kSeqSplit ? n_cells - n_sm : n_cells);
    int4 *tab = (int4 *)(sm + fcells);
    for (long long q = lo + lane; q < n_cells; q += 32) sm[q - lo] = f_g[q];
    __syncwarp();
    auto F = [&](long long cell) -> float * {
        return MODE == kSeqSmem ? sm + cell : (MODE == kSeqSplit && cell >= lo ? sm + (cell - lo) : f_g + cell);
    };
    int it = 0;
    for (; it < iters; it++) {
        int changed = 0;
        for (int k = 0; k < n_views; k++) {
            int rep = view_rep[k];
            fill_tab(tab, rt, n_rings, view_mg[k], lane, 32);
            __syncwarp();
            const long long *rp = row_ptr_all + (long long)rep * M.n_rows;
            const float *rmax = rowmax_all + (long long)rep * M.n_rows;
            const float *pk = proj + (long long)k * n_rays;
            // rays of the upper detector rows of a mirrored store read their
            // mirror's row with the slab flipped
            auto row_of = [&](int r) { return M.on && r >= M.n_rows ? mirror_ray(r, M.n_u, M.n_v) : r; };
            auto cell_of = [&](uint32_t pc, bool flip) {
                return rot_cell(tab, cps, flip ? flip_slab(pc, M.n_slabs) : pc);
            };
            RowRegs<WT> cur, nxt;
            // ray 0: rows, projection and row maximum; ray 1: row bounds
            int crow = row_of(0);
            bool cflip = false;  // ray 0 is stored
            long long cb = rp[crow], ce = rp[crow + 1];
            float cp = pk[0], cmx = rmax[crow];
            seq_load(cur, idx, w, cb, ce, lane);
            int nrow = crow;
            bool nflip = false;
            long long nb = ce, ne = ce;
            if (n_rays > 1) {
                nrow = row_of(1);
                nflip = nrow != 1;
                nb = rp[nrow];
                ne = rp[nrow + 1];
            }
            for (int ray = 0; ray < n_rays; ray++) {
                float np = 0.0f, nmx = 1.0f;
                if (ray + 1 < n_rays) {  // rows and scalars of the next ray
                    seq_load(nxt, idx, w, nb, ne, lane);
                    np = pk[ray + 1];
                    nmx = rmax[nrow];
                }
                int n2row = nrow;
                bool n2flip = false;
                long long n2b = ne, n2e = ne;
                if (ray + 2 < n_rays) {  // row bounds two rays ahead
                    n2row = row_of(ray + 2);
                    n2flip = n2row != ray + 2;
                    n2b = rp[n2row];
                    n2e = rp[n2row + 1];
                }
                if (ce > cb) {
                    float acc = 0.0f;
                    long long cell[kSeqChunks];
                    float fv[kSeqChunks];  // each cell occurs once in a row: the update reuses these
#pragma unroll
                    for (int c = 0; c < kSeqChunks; c++) {
                        cell[c] = cell_of(cur.ix[c], cflip);
                        fv[c] = *F(cell[c]);
                        acc = fmaf(cur.w[c], fv[c], acc);
                    }
                    for (long long q = cb + kSeqChunks * 32 + lane; q < ce; q += 32)  // long rows
                        acc = fmaf(load_w1(w, q), *F(cell_of(__ldg(idx + q), cflip)), acc);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                    float s = acc * w_scale;
                    if (s > 0.0f && cp >= 0.0f && cp <= 3.402823466e38f) {  // a bad projection changes nothing
                        float ratio = cp / s;
                        float l2 = log2f(ratio);
                        float ex = lambda / cmx;
                        float lin = 1.0f - lambda * (1.0f - ratio);
#pragma unroll
                        for (int c = 0; c < kSeqChunks; c++) {
                            if (cur.w[c] > 0.0f) {
                                float old = fv[c];
                                float fac = rule == USPG_LINEAR_EQ18 ? lin : exp2f(ex * cur.w[c] * l2);
                                float nv = old * fac;
                                if (tol > 0.0f && fabsf(nv - old) > tol * fabsf(old)) changed = 1;
                                *F(cell[c]) = nv;
                            }
                        }
                        for (long long q = cb + kSeqChunks * 32 + lane; q < ce; q += 32) {
                            float wv = load_w1(w, q);
                            if (wv > 0.0f) {
                                float *fp = F(cell_of(__ldg(idx + q), cflip));
                                float old = *fp;
                                float fac = rule == USPG_LINEAR_EQ18 ? lin : exp2f(ex * wv * l2);
                                float nv = old * fac;
                                if (tol > 0.0f && fabsf(nv - old) > tol * fabsf(old)) changed = 1;
                                *fp = nv;
                            }
                        }
                    }
                    // the next ray may read a cell another lane has just written
                    if (MODE != kSeqSmem) __threadfence_block();
                    __syncwarp();
                }
                cur = nxt;
                cb = nb;
                ce = ne;
                crow = nrow;
                cflip = nflip;
                cp = np;
                cmx = nmx;
                nb = n2b;
                ne = n2e;
                nrow = n2row;
                nflip = n2flip;
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
    __syncwarp();
    for (long long q = lo + lane; q < n_cells; q += 32) f_g[q] = sm[q - lo];
    if (lane == 0 && sweeps_out) *sweeps_out = it;
}

template <typename WT, int MODE>
static cudaError_t seq_launch(uspg_ctx *c, const uspg_mart_opts *o, const int *d_v, float *img, long long n_sm,
                              size_t smem, cudaStream_t s)
{
    auto k = k_sequential<WT, MODE>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nv = c->scan.n_views;
    k<<<1, 32, smem, s>>>((const long long *)c->d_row_ptr, (const uint32_t *)c->d_idx, (const WT *)c->d_w,
                          (const float *)c->d_rowmax, d_v, d_v + nv, nv, (int)c->n_rays, c->mir,
                          (const float *)c->d_proj, img, (long long)c->n_cells, (const RingEntry *)c->d_ring,
                          c->n_rings, (long long)c->cells_per_slab, o->iterations, (float)o->lambda, o->update_rule,
                          (float)o->stop_tol, (float)c->w_scale, n_sm, c->d_sweeps);
    return cudaGetLastError();
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
    float *img = c->d_f;  // the sequential kernel works on the standard layout
    if (c->mir.on) {
        USPG_CUDA(c, cudaMallocAsync(&img, sizeof(float) * c->n_cells, s));
        USPG_CUDA(c, image_from_pairs(c, c->d_f, img, s));
    }
    size_t tab_bytes = sizeof(int4) * c->n_rings;
    size_t f_bytes = sizeof(float) * ((c->n_cells + 3) & ~3LL);
    int dev = 0, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // cells kept in shared memory by the split form: a multiple of 4, so the
    // ring table after them stays 16-byte aligned
    long long n_sm = ((long long)max_smem - (long long)tab_bytes) / (long long)sizeof(float) & ~3LL;
    cudaError_t e;
    if (f_bytes + tab_bytes <= (size_t)max_smem)
        e = seq_launch<WT, kSeqSmem>(c, o, d_v, img, 0, f_bytes + tab_bytes, s);
    else if (n_sm >= c->n_cells / 8)  // a useful share of the image fits
        e = seq_launch<WT, kSeqSplit>(c, o, d_v, img, n_sm, sizeof(float) * n_sm + tab_bytes, s);
    else
        e = seq_launch<WT, kSeqGlobal>(c, o, d_v, img, 0, tab_bytes, s);
    launch_counter()++;
    USPG_CUDA(c, e);
    USPG_CUDA(c, cudaGetLastError());
    USPG_CUDA(c, cudaFreeAsync(d_v, s));
    if (c->mir.on) {
        USPG_CUDA(c, image_to_pairs(c, img, c->d_f, s));
        USPG_CUDA(c, cudaFreeAsync(img, s));
    }
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
    const int TB = 256;
    k_clear_acc<<<(unsigned)((c->n_rays + TB - 1) / TB), TB, 0, s>>>(acc, c->n_rays);
    launch_counter()++;
    // sums only (no correction terms): the projections are not read
    return fwd_run<WT>(c, view, f, false, acc, out, nullptr, c->d_proj, s);
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
    if (c->store_form == USPG_STORE_SEGMENTS)
        return fail(c, USPG_EUNSUPPORTED, "the per-view kernels read the representative store");
    float *acc = nullptr;
    USPG_CUDA(c, noalloc_acc(&acc));
    cudaStream_t s = (cudaStream_t)stream;
    if (c->dtype == USPG_F16) return fwd_noalloc_typed<__half>(c, view, f, out, acc, s);
    if (c->dtype == USPG_BF16) return fwd_noalloc_typed<__nv_bfloat16>(c, view, f, out, acc, s);
    return fwd_noalloc_typed<float>(c, view, f, out, acc, s);
}
