// Batched per-view MART over many independent reconstructions (instances of
// uneven size: grids, view counts, detectors).  Instance i runs its own
// per-view schedule (Sec. III.D): view step t of instance i is view
// t mod p_i of sweep t div p_i, for t < iterations * p_i.  The instances
// advance together: global step t is three launches (forward sums, ray
// ratios, cell correction) whose 2D grid covers every instance still running
// (blockIdx.y = instance; each instance gets a number of blocks proportional
// to its work per view).  All global steps are captured in one CUDA graph,
// so a batch of small instances costs one graph launch instead of thousands
// of kernel launches.  The blocks-per-work ratio is tuned on creation.
#include "internal.cuh"
#include "device.cuh"

#include <algorithm>
#include <cstring>

namespace uspg {

struct BatchInst {
    const uint32_t *idx;
    const void *w;
    const uint32_t *grp_ray;
    const long long *rep_g0;  // [reps] first 8-entry group of each representative
    const long long *rep_ng;  // [reps] groups of each representative
    float *f;
    const RingEntry *rt;
    float *sacc;
    float *res;
    const float *proj;
    const uint2 *slice_desc;    // [reps * S] {first slot relative to the representative, meta}
    const uint16_t *lane_desc;
    const uint32_t *cray;
    const void *cw;
    const long long *rep_sell;  // [reps] first cell-major slot of each representative
    const int *view_rep;        // [views]
    const int *view_mg;         // [views]
    long long cps, S, steps;
    int n_rings, n_rays, n_views, fwd_blocks, bwd_blocks;
    float w_scale;
    Mirror mir;  // z-mirror store of the instance (mir.on == 0: every row stored)
};

template <typename WT>
__global__ void __launch_bounds__(256) k_batch_forward(const BatchInst *__restrict__ inst, long long step)
{
    extern __shared__ int4 tab[];
    const BatchInst &I = inst[blockIdx.y];
    if (step >= I.steps || (int)blockIdx.x >= I.fwd_blocks) return;  // block-uniform
    int view = (int)(step % I.n_views);
    int rep = I.view_rep[view];
    fill_tab(tab, I.rt, I.n_rings, I.view_mg[view], threadIdx.x, blockDim.x);
    __syncthreads();
    long long wg = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long W = ((long long)I.fwd_blocks * blockDim.x) >> 5;
    if (I.mir.on)  // block-uniform
        fwd_groups<WT, true>(I.idx, (const WT *)I.w, I.grp_ray, I.rep_g0[rep], I.rep_ng[rep], I.f, tab, I.cps, I.sacc,
                             wg, W, threadIdx.x & 31, I.mir);
    else
        fwd_groups<WT, false>(I.idx, (const WT *)I.w, I.grp_ray, I.rep_g0[rep], I.rep_ng[rep], I.f, tab, I.cps,
                              I.sacc, wg, W, threadIdx.x & 31, I.mir);
}

__global__ void k_batch_finalize(const BatchInst *__restrict__ inst, long long step)
{
    const BatchInst &I = inst[blockIdx.y];
    if (step >= I.steps) return;
    int ray = blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= I.mir.n_rows) return;  // the stored rays (all rays when not mirrored)
    int view = (int)(step % I.n_views);
    if (I.mir.on)
        finalize_pair(I.sacc, I.proj + (long long)view * I.n_rays, ray, I.mir, I.w_scale, 0, nullptr,
                      (float4 *)I.res);
    else
        finalize_ray(I.sacc, I.proj + (long long)view * I.n_rays, ray, I.w_scale, 0, nullptr, (float2 *)I.res);
}

template <typename WT>
__global__ void __launch_bounds__(256, kBwdMinBlocksMirror) k_batch_backward(const BatchInst *__restrict__ inst,
                                                                             long long step, float lambda)
{
    const BatchInst &I = inst[blockIdx.y];
    if (step >= I.steps || (int)blockIdx.x >= I.bwd_blocks) return;  // block-uniform
    extern __shared__ int4 tab[];
    const UpdateRule U{lambda, 0, 0.0f, nullptr};
    int view = (int)(step % I.n_views);
    int rep = I.view_rep[view];
    fill_tab(tab, I.rt, I.n_rings, I.view_mg[view], threadIdx.x, blockDim.x);
    __syncthreads();
    int wg = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    int W = (I.bwd_blocks * (int)blockDim.x) >> 5;
    long long base = I.rep_sell[rep];
    int S = (int)I.S;
    if (I.mir.on)  // block-uniform
        bwd_slices<WT, true>(I.slice_desc + rep * I.S, I.lane_desc + 32 * rep * I.S, I.cray + base,
                             (const WT *)I.cw + base, I.res, I.f, tab, (uint32_t)I.cps, S, U, wg, W, threadIdx.x & 31,
                             I.mir);
    else
        bwd_slices<WT, false>(I.slice_desc + rep * I.S, I.lane_desc + 32 * rep * I.S, I.cray + base,
                              (const WT *)I.cw + base, I.res, I.f, tab, (uint32_t)I.cps, S, U, wg, W,
                              threadIdx.x & 31, I.mir);
}

}  // namespace uspg

using namespace uspg;

struct uspg_batch {
    std::vector<uspg_ctx *> ctx;
    std::vector<BatchInst> host;
    BatchInst *d_inst = nullptr;
    void *d_tables = nullptr;  // per-instance rep/view tables
    int dtype = USPG_F32;
    double lambda = 0.1;
    long long max_steps = 0;
    int max_rings = 0, max_rays = 0;
    long long nnz_per_run = 0;  // ray-cell updates of one run
    std::vector<long long> groups_view, slices_view;  // per instance: mean groups / slices per view
    // launch shape: blocks per unit of work (8-entry group / slice), per
    // bucket of instances with the same ring count (tuned at creation)
    std::vector<int> bucket_of, bucket_rings;
    std::vector<double> fwd_ratio, bwd_ratio;
    float ms_default = 0.0f, ms_tuned = 0.0f;  // the tuning probe's time with the default and the chosen shapes
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t nodes = 0;
};

// per-instance block counts from the current ratios; returns the max of each
static void assign_blocks(uspg_batch *b, int &mf, int &mb)
{
    mf = mb = 1;
    for (size_t i = 0; i < b->host.size(); i++) {
        long long fb = (long long)(b->fwd_ratio[b->bucket_of[i]] * (double)b->groups_view[i]) + 1;
        long long bb = (long long)(b->bwd_ratio[b->bucket_of[i]] * (double)b->slices_view[i]) + 1;
        long long fmax = (b->groups_view[i] + 255) / 256 + 1, bmax = (b->slices_view[i] + 7) / 8 + 1;
        b->host[i].fwd_blocks = (int)std::min(fb, fmax);
        b->host[i].bwd_blocks = (int)std::min(bb, bmax);
        mf = std::max(mf, b->host[i].fwd_blocks);
        mb = std::max(mb, b->host[i].bwd_blocks);
    }
}

// block counts into the device instance table (synchronous)
static cudaError_t upload(uspg_batch *b, int &mf, int &mb)
{
    assign_blocks(b, mf, mb);
    return cudaMemcpy(b->d_inst, b->host.data(), sizeof(BatchInst) * b->host.size(), cudaMemcpyHostToDevice);
}

template <typename WT>
static cudaError_t enqueue_steps(uspg_batch *b, int mf, int mb, long long s0, long long s1, cudaStream_t s,
                                 int64_t *nodes)
{
    unsigned n = (unsigned)b->host.size();
    size_t smem = sizeof(int4) * b->max_rings;
    for (long long t = s0; t < s1; t++) {
        k_batch_forward<WT><<<dim3(mf, n), 256, smem, s>>>(b->d_inst, t);
        k_batch_finalize<<<dim3((b->max_rays + 255) / 256, n), 256, 0, s>>>(b->d_inst, t);
        k_batch_backward<WT><<<dim3(mb, n), 256, smem, s>>>(b->d_inst, t, (float)b->lambda);
        if (nodes) *nodes += 3;
    }
    return cudaGetLastError();
}

static cudaError_t enqueue(uspg_batch *b, int mf, int mb, long long s0, long long s1, cudaStream_t s, int64_t *nodes)
{
    if (b->dtype == USPG_F16) return enqueue_steps<__half>(b, mf, mb, s0, s1, s, nodes);
    if (b->dtype == USPG_BF16) return enqueue_steps<__nv_bfloat16>(b, mf, mb, s0, s1, s, nodes);
    return enqueue_steps<float>(b, mf, mb, s0, s1, s, nodes);
}

extern "C" {

void uspg_batch_destroy(uspg_batch *b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    cudaFree(b->d_inst);
    cudaFree(b->d_tables);
    delete b;
}

uspg_status uspg_batch_create(uspg_ctx *const *ctxs, int32_t n, const uspg_mart_opts *o, uspg_stream stream,
                              uspg_batch **out)
{
    if (!out || !ctxs || !o || n < 1) return fail(nullptr, USPG_EINVAL, "batch: NULL argument or n < 1");
    *out = nullptr;
    if (o->schedule != USPG_PER_VIEW || o->update_rule != USPG_POWER)
        return fail(nullptr, USPG_EUNSUPPORTED, "batch: per-view schedule with the power update only");
    if (o->iterations < 1 || !(o->lambda > 0.0 && o->lambda < 2.0))
        return fail(nullptr, USPG_EINVAL, "batch: iterations >= 1 and lambda in (0, 2)");
    uspg_batch *b = new uspg_batch();
    b->lambda = o->lambda;
    b->dtype = ctxs[0]->dtype;
    // per-instance tables: rep_g0, rep_ng, rep_sell (int64 [reps]) and view_rep, view_mg (int [views])
    std::vector<long long> off_tab(n);
    long long bytes = 0;
    for (int i = 0; i < n; i++) {
        uspg_ctx *c = ctxs[i];
        if (!c || !c->built || !c->have_proj) {
            uspg_batch_destroy(b);
            return fail(nullptr, USPG_ENOTREADY, "batch: every context needs coefficients and projections");
        }
        if (c->store_form == USPG_STORE_SEGMENTS) {
            uspg_batch_destroy(b);
            return fail(nullptr, USPG_EUNSUPPORTED, "batch: the per-view kernels read the representative store");
        }
        if (c->dtype != b->dtype) {
            uspg_batch_destroy(b);
            return fail(nullptr, USPG_EINVAL, "batch: all contexts must store coefficients in one dtype");
        }
        off_tab[i] = bytes;
        bytes += 8LL * 3 * c->n_reps + 4LL * 2 * c->scan.n_views;
        bytes = (bytes + 15) & ~15LL;
    }
    std::vector<unsigned char> tab(bytes);
    b->ctx.assign(ctxs, ctxs + n);
    b->host.resize(n);
    b->groups_view.resize(n);
    b->slices_view.resize(n);
    if (cudaMalloc(&b->d_tables, bytes + 16) != cudaSuccess || cudaMalloc(&b->d_inst, sizeof(BatchInst) * n) != cudaSuccess) {
        uspg_batch_destroy(b);
        return fail(nullptr, USPG_ENOMEM, "batch: device tables");
    }
    for (int i = 0; i < n; i++) {
        uspg_ctx *c = ctxs[i];
        int R = c->n_reps, V = c->scan.n_views;
        long long *g0 = (long long *)(tab.data() + off_tab[i]);
        long long *ng = g0 + R, *sb = ng + R;
        int *vr = (int *)(sb + R), *vm = vr + V;
        long long gsum = 0;
        for (int r = 0; r < R; r++) {
            g0[r] = c->h_rep_entry0[r] / kRowPad;
            ng[r] = (c->h_rep_entry0[r + 1] - c->h_rep_entry0[r]) / kRowPad;
            sb[r] = c->h_sell_base[r];
        }
        for (int k = 0; k < V; k++) {
            vr[k] = c->rep_of_view[k];
            vm[k] = c->m_of_view[k] % c->G;
            gsum += ng[vr[k]];
        }
        unsigned char *dt = (unsigned char *)b->d_tables + off_tab[i];
        BatchInst &I = b->host[i];
        I.idx = c->d_idx;
        I.w = c->d_w;
        I.grp_ray = c->d_grp_ray;
        I.rep_g0 = (const long long *)dt;
        I.rep_ng = I.rep_g0 + R;
        I.rep_sell = I.rep_ng + R;
        I.view_rep = (const int *)(I.rep_sell + R);
        I.view_mg = I.view_rep + V;
        I.f = c->d_f;
        I.rt = c->d_ring;
        I.sacc = c->d_sacc;
        I.res = c->d_res;
        I.proj = c->d_proj;
        I.slice_desc = c->d_slice_desc;
        I.lane_desc = c->d_lane_desc;
        I.cray = c->d_cm_ray;
        I.cw = c->d_cm_w;
        I.cps = c->cells_per_slab;
        I.S = c->slices_per_rep;
        I.steps = (long long)o->iterations * V;
        I.n_rings = c->n_rings;
        I.n_rays = c->n_rays;
        I.n_views = V;
        I.w_scale = (float)c->w_scale;
        I.mir = c->mir;
        b->groups_view[i] = std::max<long long>(1, gsum / V);
        b->slices_view[i] = std::max<long long>(1, I.S);
        b->max_steps = std::max(b->max_steps, I.steps);
        b->max_rings = std::max(b->max_rings, c->n_rings);
        b->max_rays = std::max(b->max_rays, c->n_rays);
        b->nnz_per_run += (long long)o->iterations * c->nnz_all_views;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(b->d_tables, tab.data(), bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) {
        uspg_batch_destroy(b);
        return fail(nullptr, USPG_ECUDA, "batch: table upload");
    }
    // tune the blocks-per-work ratios on the first steps; images are saved
    // and restored so the instances' state does not change
    std::vector<float *> saved(n, nullptr);
    for (int i = 0; i < n; i++) {
        if (cudaMallocAsync(&saved[i], sizeof(float) * image_floats(ctxs[i]), s) != cudaSuccess ||
            cudaMemcpyAsync(saved[i], ctxs[i]->d_f, sizeof(float) * image_floats(ctxs[i]), cudaMemcpyDeviceToDevice,
                            s) !=
                cudaSuccess) {
            uspg_batch_destroy(b);
            return fail(nullptr, USPG_ENOMEM, "batch: tuning scratch");
        }
    }
    // buckets: instances with the same ring count
    b->bucket_of.assign(n, 0);
    for (int i = 0; i < n; i++) {
        int rings = ctxs[i]->n_rings, q = 0;
        while (q < (int)b->bucket_rings.size() && b->bucket_rings[q] != rings) q++;
        if (q == (int)b->bucket_rings.size()) b->bucket_rings.push_back(rings);
        b->bucket_of[i] = q;
    }
    const int nb = (int)b->bucket_rings.size();
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const double fr[4] = {1.0 / 8192, 1.0 / 2048, 1.0 / 512, 1.0 / 128};  // blocks per 8-entry group
    const double br[4] = {1.0 / 2048, 1.0 / 512, 1.0 / 128, 1.0 / 32};    // blocks per slice
    long long probe = std::min<long long>(b->max_steps, 4);
    auto time_shape = [&]() -> float {  // one warm and one timed probe
        int mf, mb;
        cudaStreamSynchronize(s);
        if (upload(b, mf, mb) != cudaSuccess) return 1e30f;
        enqueue(b, mf, mb, 0, probe, s, nullptr);
        cudaEventRecord(e0, s);
        enqueue(b, mf, mb, 0, probe, s, nullptr);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) return 1e30f;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    // the default shape, then the best shape common to all buckets
    b->fwd_ratio.assign(nb, fr[1]);
    b->bwd_ratio.assign(nb, br[1]);
    b->ms_default = time_shape();
    float best = b->ms_default;
    double bf = fr[1], bbw = br[1];
    for (double a : fr)
        for (double c2 : br) {
            b->fwd_ratio.assign(nb, a);
            b->bwd_ratio.assign(nb, c2);
            float ms = time_shape();
            if (ms < best) {
                best = ms;
                bf = a;
                bbw = c2;
            }
        }
    b->fwd_ratio.assign(nb, bf);
    b->bwd_ratio.assign(nb, bbw);
    // then each bucket's own shape, the others fixed; a change must gain 1%
    if (nb > 1) {
        best = time_shape();
        for (int q = 0; q < nb; q++) {
            double qf = b->fwd_ratio[q], qb = b->bwd_ratio[q];
            for (double a : fr)
                for (double c2 : br) {
                    b->fwd_ratio[q] = a;
                    b->bwd_ratio[q] = c2;
                    float ms = time_shape();
                    if (ms < 0.99f * best) {
                        best = ms;
                        qf = a;
                        qb = c2;
                    }
                }
            b->fwd_ratio[q] = qf;
            b->bwd_ratio[q] = qb;
        }
    }
    b->ms_tuned = time_shape();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int i = 0; i < n; i++) {
        cudaMemcpyAsync(ctxs[i]->d_f, saved[i], sizeof(float) * image_floats(ctxs[i]), cudaMemcpyDeviceToDevice, s);
        cudaFreeAsync(saved[i], s);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        uspg_batch_destroy(b);
        return fail(nullptr, USPG_ECUDA, "batch: tuning failed");
    }
    // capture all global steps into one graph
    int mf = 1, mb = 1;
    if (upload(b, mf, mb) != cudaSuccess) {
        uspg_batch_destroy(b);
        return fail(nullptr, USPG_ECUDA, "batch: instance table upload");
    }
    cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        uspg_batch_destroy(b);
        return fail(nullptr, USPG_ECUDA, "batch: capture");
    }
    int64_t nodes = 0;
    cudaError_t ce = enqueue(b, mf, mb, 0, b->max_steps, b->cap, &nodes);
    cudaError_t ee = cudaStreamEndCapture(b->cap, &b->graph);
    if (ce || ee || cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) {
        uspg_batch_destroy(b);
        return fail(nullptr, USPG_ECUDA, "batch: graph capture or instantiation failed");
    }
    b->nodes = nodes;
    *out = b;
    return USPG_OK;
}

uspg_status uspg_batch_run(uspg_batch *b, uspg_stream stream)
{
    if (!b) return fail(nullptr, USPG_EINVAL, "NULL batch");
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(nullptr, USPG_ECUDA, std::string("batch launch: ") + cudaGetErrorString(e));
    launch_counter() += b->nodes;
    return USPG_OK;
}

uspg_status uspg_batch_tuning(const uspg_batch *b, int32_t cap, int32_t *rings, double *fwd_blocks_per_group,
                              double *bwd_blocks_per_slice, int32_t *n_buckets, float *ms_default, float *ms_tuned)
{
    if (!b || !n_buckets) return fail(nullptr, USPG_EINVAL, "NULL argument");
    int nb = (int)b->bucket_rings.size();
    *n_buckets = nb;
    if (ms_default) *ms_default = b->ms_default;
    if (ms_tuned) *ms_tuned = b->ms_tuned;
    if (nb > cap) return fail(nullptr, USPG_EINVAL, "batch tuning: more buckets than cap");
    for (int q = 0; q < nb; q++) {
        if (rings) rings[q] = b->bucket_rings[q];
        if (fwd_blocks_per_group) fwd_blocks_per_group[q] = b->fwd_ratio[q];
        if (bwd_blocks_per_slice) bwd_blocks_per_slice[q] = b->bwd_ratio[q];
    }
    return USPG_OK;
}

uspg_status uspg_batch_info(const uspg_batch *b, int64_t *updates_per_run, int64_t *kernel_nodes, int64_t *steps)
{
    if (!b) return fail(nullptr, USPG_EINVAL, "NULL batch");
    if (updates_per_run) *updates_per_run = b->nnz_per_run;
    if (kernel_nodes) *kernel_nodes = b->nodes;
    if (steps) *steps = b->max_steps;
    return USPG_OK;
}

}  // extern "C"
