// C-ABI host runtime of libuspg (include/uspg.h): context set-up, grid tables
// (Eq. 1-2), view classes (Sec. III.C), device buffers, data movement, the
// MART driver and its CUDA-graph cache.
#include "internal.cuh"
#include "device.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <sstream>
#include <vector>

namespace uspg {

static thread_local std::string g_create_err;

uspg_status fail(uspg_ctx *c, uspg_status st, const std::string &msg)
{
    if (c) c->err = msg;
    else g_create_err = msg;
    return st;
}

uspg_status cuda_fail(uspg_ctx *c, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? USPG_ENOMEM : USPG_ECUDA, m);
}

static long long gcd_ll(long long a, long long b)
{
    while (b) {
        long long t = a % b;
        a = b;
        b = t;
    }
    return a < 0 ? -a : a;
}

static void free_store(uspg_ctx *c)
{
    cudaFree(c->d_row_ptr);
    cudaFree(c->d_idx);
    cudaFree(c->d_w);
    cudaFree(c->d_rowmax);
    cudaFree(c->d_slice_off);
    cudaFree(c->d_slice_meta);
    cudaFree(c->d_slice_width);
    cudaFree(c->d_slice_desc);
    c->d_slice_desc = nullptr;
    cudaFree(c->d_sray);
    cudaFree(c->d_sw);
    cudaFree(c->d_counts);
    cudaFree(c->d_rep_view);
    cudaFree(c->d_cell_cnt);
    cudaFree(c->d_cell_fill);
    cudaFree(c->d_rel);
    cudaFree(c->d_stats);
    cudaFree(c->d_cm_ray);
    cudaFree(c->d_cm_w);
    cudaFree(c->d_lane_desc);
    c->d_cm_ray = nullptr;
    c->d_cm_w = nullptr;
    c->d_lane_desc = nullptr;
    c->cap_cm = 0;
    cudaFree(c->d_grp_ray);
    c->d_grp_ray = nullptr;
    c->cap_grp = 0;
    cudaFree(c->d_w64);
    cudaFreeHost(c->h_gen_pin);
    cudaFree(c->d_gen_small);
    c->h_gen_pin = nullptr;
    c->d_gen_small = nullptr;
    cudaFree(c->d_plan);
    cudaFree(c->d_tied);
    cudaFree(c->d_retrace);
    c->d_plan = c->d_tied = nullptr;
    c->d_retrace = nullptr;
    c->d_counts = c->d_rep_view = c->d_cell_cnt = c->d_cell_fill = nullptr;
    c->d_rel = nullptr;
    c->d_stats = nullptr;
    c->d_w64 = nullptr;
    c->cap_idx = c->cap_w = c->cap_w64 = c->cap_sell = 0;
    c->d_row_ptr = nullptr;
    c->d_idx = nullptr;
    c->d_w = nullptr;
    c->d_rowmax = nullptr;
    c->d_slice_off = nullptr;
    c->d_slice_meta = nullptr;
    c->d_slice_width = nullptr;
    c->d_sray = nullptr;
    c->d_sw = nullptr;
    c->built = false;
    for (auto &kv : c->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    c->graphs.clear();
}

// reconstruction state: image, projections, per-ray scratch, flags
static uspg_status alloc_state(uspg_ctx *c)
{
    if (c->d_f) return USPG_OK;
    USPG_CUDA(c, cudaMalloc(&c->d_f, sizeof(float) * image_floats(c)));
    USPG_CUDA(c, cudaMalloc(&c->d_proj, sizeof(float) * (long long)c->scan.n_views * c->n_rays));
    // per-ray correction terms {value, taken part}; mirrored stores keep
    // them as pairs of terms per stored ray, in both orders (finalize_pair)
    USPG_CUDA(c, cudaMalloc(&c->d_res, c->mir.on ? sizeof(float4) * 2 * c->mir.n_rows : sizeof(float2) * c->n_rays));
    USPG_CUDA(c, cudaMalloc(&c->d_sacc, sizeof(float) * c->n_rays));
    USPG_CUDA(c, cudaMemset(c->d_sacc, 0, sizeof(float) * c->n_rays));
    USPG_CUDA(c, cudaMalloc(&c->d_status, sizeof(int)));
    USPG_CUDA(c, cudaMemset(c->d_status, 0, sizeof(int)));
    USPG_CUDA(c, cudaMalloc(&c->d_sweeps, sizeof(int) * 4));
    USPG_CUDA(c, cudaMemset(c->d_sweeps, 0, sizeof(int) * 4));
    USPG_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    return USPG_OK;
}

static void free_state(uspg_ctx *c)
{
    for (auto &kv : c->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    c->graphs.clear();
    cudaFree(c->d_f);
    cudaFree(c->d_proj);
    cudaFree(c->d_proj_stage);
    cudaFree(c->d_first_bad);
    cudaFree(c->d_rs_std);
    cudaFree(c->d_rs_out);
    c->d_proj_stage = nullptr;
    c->d_first_bad = nullptr;
    c->d_rs_std = nullptr;
    c->d_rs_out = nullptr;
    c->cap_rs_out = 0;
    cudaFree(c->d_res);
    cudaFree(c->d_sacc);
    cudaFree(c->d_status);
    cudaFree(c->d_sweeps);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
}

// device buffers that do not depend on the store
static uspg_status ensure_state(uspg_ctx *c)
{
    if (c->d_ring) return alloc_state(c);
    std::vector<RingEntry> rt(c->n_rings);
    int chunk = 0;
    for (int i = 0; i < c->n_rings; i++) {
        rt[i].head = c->head[i];
        rt[i].ng = c->ng[i];
        rt[i].step = c->ng[i] / c->G;
        rt[i].chunk0 = chunk;
        chunk += (c->ng[i] + kSlice - 1) / kSlice;
    }
    c->slices_per_slab = chunk;
    // cell-major store: all slabs, or the lower half and the middle slab when mirrored
    int stored_slabs = c->scan.geometry == USPG_CONE_3D ? (c->mir.on ? (c->n_slabs + 1) / 2 : c->n_slabs) : 1;
    c->slices_per_rep = (long long)chunk * stored_slabs;
    std::vector<int> slice_ring(chunk);
    for (int i = 0; i < c->n_rings; i++)
        for (int q = rt[i].chunk0; q < rt[i].chunk0 + (c->ng[i] + kSlice - 1) / kSlice; q++) slice_ring[q] = i;
    USPG_CUDA(c, cudaMalloc(&c->d_ring, sizeof(RingEntry) * c->n_rings));
    USPG_CUDA(c, cudaMemcpy(c->d_ring, rt.data(), sizeof(RingEntry) * c->n_rings, cudaMemcpyHostToDevice));
    USPG_CUDA(c, cudaMalloc(&c->d_slice_ring, sizeof(int) * chunk));
    USPG_CUDA(c, cudaMemcpy(c->d_slice_ring, slice_ring.data(), sizeof(int) * chunk, cudaMemcpyHostToDevice));
    return alloc_state(c);
}

uspg_status ctx_share_store(const uspg_ctx *src, uspg_ctx **out)
{
    *out = nullptr;
    if (!src->built || src->store_src) return fail(nullptr, USPG_EINVAL, "share: source store not built or shared");
    uspg_ctx *c = new uspg_ctx(*src);  // host tables and store pointers
    c->store_src = src;
    c->graphs.clear();  // graphs capture the source's own image and scratch
    c->err.clear();
    c->have_proj = false;
    c->d_f = c->d_proj = c->d_res = c->d_sacc = nullptr;
    c->d_proj_stage = nullptr;
    c->d_first_bad = nullptr;
    c->d_rs_std = nullptr;
    c->d_rs_out = nullptr;
    c->cap_rs_out = 0;
    c->d_status = c->d_sweeps = nullptr;
    c->cap_stream = nullptr;
    c->d_counts = c->d_rep_view = c->d_cell_cnt = c->d_cell_fill = nullptr;  // generator scratch: never used
    c->d_rel = c->d_stats = nullptr;
    c->d_w64 = nullptr;
    c->h_gen_pin = nullptr;
    c->d_gen_small = nullptr;
    uspg_status st = alloc_state(c);
    if (st) {
        g_create_err = c->err;
        free_state(c);
        delete c;
        return st;
    }
    *out = c;
    return USPG_OK;
}

long long image_floats(const uspg_ctx *c)
{
    return c->mir.on ? 2 * image_pairs(c->cells_per_slab, c->n_slabs) : c->n_cells;
}

__global__ void k_to_pairs(const float *__restrict__ f, float2 *__restrict__ fp, long long n_pairs, long long cps,
                           int n_slabs)
{
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_pairs) return;
    long long s = k / cps, w = k - s * cps;
    fp[k] = make_float2(f[k], f[(n_slabs - 1 - s) * cps + w]);
}

__global__ void k_from_pairs(const float2 *__restrict__ fp, float *__restrict__ f, long long n_pairs, long long cps,
                             int n_slabs)
{
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_pairs) return;
    long long s = k / cps, w = k - s * cps;
    float2 v = fp[k];
    f[k] = v.x;
    if (2 * s != n_slabs - 1) f[(n_slabs - 1 - s) * cps + w] = v.y;  // the middle slab holds one cell
}

cudaError_t image_to_pairs(const uspg_ctx *c, const float *f, float *pairs, cudaStream_t s)
{
    long long n = image_pairs(c->cells_per_slab, c->n_slabs);
    k_to_pairs<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(f, (float2 *)pairs, n, c->cells_per_slab, c->n_slabs);
    launch_counter()++;
    return cudaGetLastError();
}

cudaError_t image_from_pairs(const uspg_ctx *c, const float *pairs, float *f, cudaStream_t s)
{
    long long n = image_pairs(c->cells_per_slab, c->n_slabs);
    k_from_pairs<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const float2 *)pairs, f, n, c->cells_per_slab,
                                                             c->n_slabs);
    launch_counter()++;
    return cudaGetLastError();
}

long long ctx_device_bytes(const uspg_ctx *c)
{
    int wb = c->dtype == USPG_F32 ? 4 : 2;
    long long rows = (long long)c->n_reps * c->mir.n_rows, slices = c->slices_per_rep * c->n_reps;
    long long b = 4LL * c->n_cells + 4LL * c->scan.n_views * c->n_rays + 16LL * c->n_rays;  // image, projections, scratch
    if (c->store_src) return b;
    b += (long long)sizeof(RingEntry) * c->n_rings + 24LL * c->cells_per_slab;  // ring table, boundaries
    if (c->d_seg_ptr) b += 20LL * c->n_segments + 9LL * (c->n_rays + 1) + 8LL * c->scan.n_views;
    if (c->d_row_ptr) {
        b += 8LL * (rows + 1) * 2 + 4LL * rows + 4LL * (rows + 1);                       // row pointers, counts, max
        b += (long long)c->cap_idx * (4 + wb + 8) + 4LL * c->cap_grp;                    // rows, FP64 weights, groups
        b += (long long)c->cap_sell * (4 + wb) + (long long)c->cap_cm * (4 + wb);        // padded and lane-ordered
        b += slices * (8 + 4 + 4 + 8 + 64) + 8LL * c->n_cells + 8LL * (c->slices_per_rep + 1);  // slices, cell scratch
    }
    return b;
}

}  // namespace uspg

using namespace uspg;

extern "C" {

int64_t uspg_kernel_launches(void) { return launch_counter(); }

const char *uspg_last_error(const uspg_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

uspg_status uspg_create(const uspg_grid_desc *grid, const uspg_scan_desc *scan, const uspg_coeff_opts *opts,
                        uspg_ctx **out)
{
    if (!out) return fail(nullptr, USPG_EINVAL, "out is NULL");
    *out = nullptr;
    if (!grid || !scan) return fail(nullptr, USPG_EINVAL, "grid and scan descriptions are required");
    const uspg_grid_desc &g = *grid;
    const uspg_scan_desc &s = *scan;
    if (g.n_rings < 1 || g.n_rings > kMaxRings) return fail(nullptr, USPG_EINVAL, "n_rings must be in [1, 1024]");
    if (!(g.ring_width > 0.0) || !std::isfinite(g.ring_width)) return fail(nullptr, USPG_EINVAL, "ring_width must be > 0");
    if (s.geometry != USPG_PARALLEL_2D && s.geometry != USPG_CONE_3D && s.geometry != USPG_FAN_2D)
        return fail(nullptr, USPG_EINVAL, "unknown scan geometry");
    int ns = s.geometry == USPG_CONE_3D ? g.n_slabs : 1;
    if (s.geometry != USPG_CONE_3D && g.n_slabs != 1)
        return fail(nullptr, USPG_EINVAL, "a 2D scan needs n_slabs = 1");
    if (ns < 1 || ns > kMaxSlabs) return fail(nullptr, USPG_EINVAL, "n_slabs must be in [1, 1024]");
    if (s.geometry == USPG_CONE_3D && !(g.slab_height > 0.0)) return fail(nullptr, USPG_EINVAL, "slab_height must be > 0");
    if (s.n_views < 1 || s.n_u < 1 || s.n_v < 1 || s.arc_den < 1 || s.arc_num < 0)
        return fail(nullptr, USPG_EINVAL, "n_views, n_u, n_v, arc_den must be >= 1 and arc_num >= 0");
    if (s.geometry != USPG_CONE_3D && s.n_v != 1) return fail(nullptr, USPG_EINVAL, "2D scans have n_v = 1");
    if (!(s.du > 0.0) || (s.geometry == USPG_CONE_3D && !(s.dv > 0.0)))
        return fail(nullptr, USPG_EINVAL, "detector pitch must be > 0");
    if ((long long)s.n_u * s.n_v >= (1LL << 31)) return fail(nullptr, USPG_EINVAL, "too many rays per view");
    double R = g.n_rings * g.ring_width;
    if (s.geometry != USPG_PARALLEL_2D) {
        if (!(s.src_to_axis > R) || !(s.src_to_det > s.src_to_axis) || !std::isfinite(s.src_to_det))
            return fail(nullptr, USPG_EINVAL, "cone and fan scans need src_to_det > src_to_axis > grid radius");
        // the detector must see the cylinder: its half-width at the axis must exceed 0
        double half_u = 0.5 * s.n_u * s.du * s.src_to_axis / s.src_to_det;
        if (!(half_u > 0.0)) return fail(nullptr, USPG_EINVAL, "detector misses the object");
    } else {
        double half = 0.5 * s.n_u * s.du;
        if (!(half > 0.0)) return fail(nullptr, USPG_EINVAL, "detector misses the object");
    }
    int wm = opts ? opts->weight_mode : USPG_LENGTH;
    int dt = opts ? opts->coeff_dtype : USPG_F32;
    int sf = opts ? opts->store_form : USPG_STORE_REPRESENTATIVES;
    if (wm != USPG_LENGTH && wm != USPG_BINARY) return fail(nullptr, USPG_EINVAL, "unknown weight_mode");
    if (dt != USPG_F32 && dt != USPG_F16 && dt != USPG_BF16) return fail(nullptr, USPG_EINVAL, "unknown coeff_dtype");
    if (sf != USPG_STORE_REPRESENTATIVES && sf != USPG_STORE_SEGMENTS)
        return fail(nullptr, USPG_EINVAL, "unknown store_form");
    if (sf == USPG_STORE_SEGMENTS && wm != USPG_BINARY)
        return fail(nullptr, USPG_EINVAL, "the segment store holds binary coefficients (weight_mode USPG_BINARY)");
    int sym = opts ? opts->symmetry : USPG_SYMMETRY_AUTO;
    if (sym != USPG_SYMMETRY_AUTO && sym != USPG_SYMMETRY_ALWAYS && sym != USPG_SYMMETRY_NEVER)
        return fail(nullptr, USPG_EINVAL, "unknown symmetry mode");

    uspg_ctx *c = new uspg_ctx();
    c->n_rings = g.n_rings;
    c->sector_rule = g.sector_rule;
    c->n_slabs = ns;
    c->r = g.ring_width;
    c->h = s.geometry == USPG_CONE_3D ? g.slab_height : 1.0;
    c->z_min = s.geometry == USPG_CONE_3D ? g.z_min : 0.0;
    c->scan = s;
    c->n_rays = s.n_u * (s.geometry == USPG_CONE_3D ? s.n_v : 1);
    // z-mirror (Sec. III.C symmetry): a cone scan whose source lies on the
    // mid-plane of a slab stack centred on z = 0 stores only detector rows
    // v < (n_v+1)/2; row n_v-1-v is the same row with slab s -> n_s-1-s
    c->mir.n_u = s.n_u;
    c->mir.n_v = s.geometry == USPG_CONE_3D ? s.n_v : 1;
    c->mir.n_slabs = ns;
    c->store_form = sf;
    c->mir.on = sf == USPG_STORE_REPRESENTATIVES && s.geometry == USPG_CONE_3D && s.n_v >= 2 &&
                c->z_min == -0.5 * (double)ns * c->h;
    c->mir.n_rows = c->mir.on ? (s.n_v + 1) / 2 * s.n_u : c->n_rays;
    c->weight_mode = wm;
    c->dtype = dt;
    c->symmetry = sym;
    double unit = c->r;
    if (s.geometry == USPG_CONE_3D && c->h < unit) unit = c->h;
    c->w_scale = dt == USPG_F32 ? 1.0 : unit;
    // Eq. 1 and Eq. 2: sector counts and heads
    c->ng.resize(g.n_rings);
    c->head.resize(g.n_rings);
    long long hsum = 0, G = 0;
    for (int n = 1; n <= g.n_rings; n++) {
        long long k;
        if (g.sector_rule == USPG_SECT_6N) k = 6LL * n;
        else if (g.sector_rule == USPG_SECT_4_2N1) k = 4LL * (2 * n - 1);
        else if (g.sector_rule == USPG_SECT_CUSTOM) {
            if (!g.sectors) {
                delete c;
                return fail(nullptr, USPG_EINVAL, "SECT_CUSTOM needs a sectors table");
            }
            k = g.sectors[n - 1];
        } else {
            delete c;
            return fail(nullptr, USPG_EINVAL, "unknown sector rule");
        }
        if (k < 1 || k > kMaxSectors) {
            delete c;
            return fail(nullptr, USPG_EINVAL, "sectors per ring must be in [1, 4096]");
        }
        c->ng[n - 1] = (int)k;
        c->head[n - 1] = (int)hsum;
        hsum += k;
        G = gcd_ll(G, k);
    }
    if (c->ng[0] > 2 * kMaxRing0Cross - 4) {
        delete c;
        return fail(nullptr, USPG_EUNSUPPORTED, "the innermost ring may have at most 60 sectors");
    }
    c->cells_per_slab = hsum;
    c->n_cells = hsum * ns;
    c->G = (int)G;
    if (c->n_cells >= (1LL << 31)) {
        delete c;
        return fail(nullptr, USPG_EINVAL, "grid has 2^31 cells or more");
    }
    // Sec. III.C: view k at theta_k = k*arc/p turns = m_k/G + rho_k; views with
    // equal residual rho_k share the stored rows of the first of them.
    int nv = s.n_views;
    long long den = s.arc_den * (long long)nv;
    c->rep_of_view.assign(nv, -1);
    c->m_of_view.assign(nv, 0);
    std::map<long long, int> first_of_key;
    for (int k = 0; k < nv; k++) {
        long long num = (long long)k * s.arc_num * G;
        long long m = num / den, key = num % den;
        auto it = first_of_key.find(key);
        if (it == first_of_key.end()) {
            first_of_key[key] = (int)c->rep_view.size();
            c->rep_of_view[k] = (int)c->rep_view.size();
            c->rep_view.push_back(k);
            c->m_of_view[k] = 0;
        } else {
            int rep = it->second;
            long long mrep = ((long long)c->rep_view[rep] * s.arc_num * G) / den;
            c->rep_of_view[k] = rep;
            c->m_of_view[k] = (int)(m - mrep);
        }
    }
    c->n_reps = (int)c->rep_view.size();
    *out = c;
    return USPG_OK;
}

void uspg_destroy(uspg_ctx *c)
{
    if (!c) return;
    cudaDeviceSynchronize();
    free_state(c);
    if (!c->store_src) {
        free_store(c);
        free_segments(c);
        cudaFree(c->d_ring);
        cudaFree(c->d_slice_ring);
        cudaFree(c->d_bdir);
        cudaFree(c->d_bdirf);
    }
    delete c;
}

uspg_status uspg_sync(uspg_ctx *c, uspg_stream stream)
{
    if (!c) return fail(nullptr, USPG_EINVAL, "NULL context");
    USPG_CUDA(c, cudaStreamSynchronize((cudaStream_t)stream));
    if (!c->d_status) return USPG_OK;
    int st = 0;
    USPG_CUDA(c, cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st) {
        USPG_CUDA(c, cudaMemset(c->d_status, 0, sizeof(int)));
        if (st & kStatusTimeout) return fail(c, USPG_ETIMEOUT, "a device-side wait gave up");
        std::ostringstream os;
        os << "device flag 0x" << std::hex << st << ": ";
        if (st & kStatusCountMismatch) os << "row count changed between generator passes; ";
        if (st & kStatusRing0Overflow) os << "too many crossings in the innermost ring; ";
        if (st & kStatusBounds) os << "index out of range; ";
        if (st & kStatusBadData) os << "device projections hold a value that is not finite and >= 0; ";
        return fail(c, USPG_EDEVICE, os.str());
    }
    return USPG_OK;
}

uspg_status uspg_build_coeffs(uspg_ctx *c, uspg_stream stream)
{
    if (!c) return fail(nullptr, USPG_EINVAL, "NULL context");
    if (c->store_src) return fail(c, USPG_EUNSUPPORTED, "this context reads another context's store");
    uspg_status st = ensure_state(c);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    c->built = false;
    c->store_moved = false;
    st = c->store_form == USPG_STORE_SEGMENTS ? build_segments(c, s) : build_store(c, s);
    if (st) return st;
    if (c->store_moved) {  // captured graphs point at the old buffers
        for (auto &kv : c->graphs) {
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
            if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
        }
        c->graphs.clear();
    }
    st = uspg_sync(c, stream);
    if (st) return st;
    c->built = true;
    return USPG_OK;
}

uspg_status uspg_coeff_stats(const uspg_ctx *c, uspg_stats *o)
{
    if (!c || !o) return fail(const_cast<uspg_ctx *>(c), USPG_EINVAL, "NULL argument");
    if (!c->built) return fail(const_cast<uspg_ctx *>(c), USPG_ENOTREADY, "coefficients not built");
    int wb = c->dtype == USPG_F32 ? 4 : 2;
    o->n_cells = c->n_cells;
    o->cells_per_slab = c->cells_per_slab;
    o->n_rays = c->n_rays;
    o->n_views = c->scan.n_views;
    if (c->store_form == USPG_STORE_SEGMENTS) {
        // one store for every view: 20 bytes a segment, row pointers, turn
        // directions and view angles; the full binary matrix would hold a
        // 4-byte cell id per nonzero and a row pointer per (view, ray)
        o->n_reps = 1;
        o->nnz_store = c->n_segments;
        o->nnz_all_views = c->nnz_all_views;
        o->store_bytes = c->n_segments * 20 + 8LL * (c->n_rays + 1) + c->n_rays + 8LL * c->scan.n_views;
        o->full_matrix_bytes = 4LL * c->nnz_all_views + 8LL * ((long long)c->scan.n_views * c->n_rays + 1);
        o->max_row = c->gen.max_row;
        o->gcd = c->G;
        o->mirrored = 0;
        o->slices = 0;
        o->walked_rows = c->n_rays;
        o->derived_reps = 0;
        return USPG_OK;
    }
    o->n_reps = c->n_reps;
    o->nnz_store = c->gen.nnz;
    o->nnz_all_views = c->nnz_all_views;
    long long rows = (long long)c->n_reps * c->mir.n_rows;
    long long slices = c->slices_per_rep * c->n_reps;
    o->store_bytes = c->gen.nnz_pad * (4 + wb) + (rows + 1) * 8 + rows * 4 + c->gen.sell_entries * (4 + wb) +
                     slices * (8 + 64);
    // the same layouts for every view, and without the z-mirror
    double per_view = c->n_reps ? (double)o->store_bytes / c->n_reps : 0.0;
    double unmirrored = c->gen.nnz ? (double)c->gen.nnz_reps_full / (double)c->gen.nnz : 1.0;
    o->full_matrix_bytes = (int64_t)(per_view * unmirrored * c->scan.n_views);
    o->max_row = c->gen.max_row;
    o->gcd = c->G;
    o->mirrored = c->mir.on;
    o->slices = c->slices_per_rep;
    o->walked_rows = c->gen_walked_rows;
    o->derived_reps = c->gen_derived_reps;
    return USPG_OK;
}

uspg_status uspg_get_row(const uspg_ctx *cc, int32_t view, int32_t ray, int32_t cap, int64_t *cells, double *w,
                         int32_t *n)
{
    uspg_ctx *c = const_cast<uspg_ctx *>(cc);
    if (!c || !n) return fail(c, USPG_EINVAL, "NULL argument");
    if (!c->built) return fail(c, USPG_ENOTREADY, "coefficients not built");
    if (view < 0 || view >= c->scan.n_views || ray < 0 || ray >= c->n_rays) return fail(c, USPG_EINVAL, "bad view/ray");
    if (c->store_form == USPG_STORE_SEGMENTS) {
        std::vector<long long> cl;
        uspg_status st = segment_row(c, view, ray, cl);
        if (st) return st;
        *n = (int32_t)cl.size();
        if ((long long)cl.size() > cap) return fail(c, USPG_EINVAL, "row longer than cap");
        if (!cells || !w) return cl.empty() ? USPG_OK : fail(c, USPG_EINVAL, "NULL cells or w");
        for (size_t q = 0; q < cl.size(); q++) {
            cells[q] = cl[q];
            w[q] = 1.0;
        }
        return USPG_OK;
    }
    int rep = c->rep_of_view[view];
    bool flip = c->mir.on && ray >= c->mir.n_rows;  // a mirrored row: stored as its mirror ray
    int stored = flip ? mirror_ray(ray, c->mir.n_u, c->mir.n_v) : ray;
    long long row = (long long)rep * c->mir.n_rows + stored;
    if (c->h_row_ptr.empty()) {
        long long nrows = (long long)c->n_reps * c->mir.n_rows;
        c->h_row_ptr.resize(nrows + 1);
        USPG_CUDA(c, cudaMemcpy(c->h_row_ptr.data(), c->d_row_ptr, sizeof(long long) * (nrows + 1),
                                cudaMemcpyDeviceToHost));
    }
    long long b = c->h_row_ptr[row], e = c->h_row_ptr[row + 1];
    std::vector<uint32_t> ix(e - b);
    int wb = c->dtype == USPG_F32 ? 4 : 2;
    std::vector<unsigned char> wr((e - b) * wb);
    if (e > b) {
        USPG_CUDA(c, cudaMemcpy(ix.data(), c->d_idx + b, sizeof(uint32_t) * (e - b), cudaMemcpyDeviceToHost));
        USPG_CUDA(c, cudaMemcpy(wr.data(), (char *)c->d_w + b * wb, wb * (e - b), cudaMemcpyDeviceToHost));
    }
    int mG = c->m_of_view[view] % c->G;
    int cnt = 0;
    for (long long q = 0; q < e - b; q++) {
        double wv;
        if (c->dtype == USPG_F32) {
            float f;
            std::memcpy(&f, &wr[q * 4], 4);
            wv = f;
        } else {
            uint16_t u;
            std::memcpy(&u, &wr[q * 2], 2);
            if (c->dtype == USPG_BF16) {
                uint32_t x = (uint32_t)u << 16;
                float f;
                std::memcpy(&f, &x, 4);
                wv = f;
            } else {
                __half_raw hr;
                hr.x = u;
                wv = (double)__half2float(__half(hr));
            }
        }
        if (!(wv > 0.0)) continue;  // row padding
        if (cnt < cap && cells && w) {
            uint32_t pc = flip ? flip_slab(ix[q], c->n_slabs) : ix[q];
            int ring = cell_ring(pc), ng = c->ng[ring];
            int sec = (cell_sector(pc) + mG * (ng / c->G)) % ng;
            cells[cnt] = (long long)cell_slab(pc) * c->cells_per_slab + c->head[ring] + sec;
            w[cnt] = wv * c->w_scale;
        }
        cnt++;
    }
    *n = cnt;
    if (cnt > cap) return fail(c, USPG_EINVAL, "row longer than cap");
    return USPG_OK;
}

// index of the first value that is not a finite number >= 0, or -1 (IEEE
// bit patterns: +0 .. the largest finite float, or -0)
static long long first_bad_value(const float *p, size_t n)
{
    const uint32_t *u = (const uint32_t *)p;
    const size_t chunk = 4096;
    for (size_t b = 0; b < n; b += chunk) {
        size_t e = std::min(n, b + chunk);
        uint32_t bad = 0;
        for (size_t i = b; i < e; i++) bad |= (uint32_t)(u[i] >= 0x7f800000u) & (uint32_t)(u[i] != 0x80000000u);
        if (bad)
            for (size_t i = b; i < e; i++)
                if (u[i] >= 0x7f800000u && u[i] != 0x80000000u) return (long long)i;
    }
    return -1;
}

// first index of a value that is not finite and >= 0 (the rule above), by
// atomicMin; *first starts at n
__global__ void k_first_bad(const float *__restrict__ v, long long n, unsigned long long *first)
{
    const long long n4 = n / 4;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        float4 x = ((const float4 *)v)[i];
        bool b0 = !(x.x >= 0.0f && x.x <= 3.402823466e38f), b1 = !(x.y >= 0.0f && x.y <= 3.402823466e38f);
        bool b2 = !(x.z >= 0.0f && x.z <= 3.402823466e38f), b3 = !(x.w >= 0.0f && x.w <= 3.402823466e38f);
        if (b0 | b1 | b2 | b3)
            atomicMin(first, (unsigned long long)(4 * i + (b0 ? 0 : b1 ? 1 : b2 ? 2 : 3)));
    }
    for (long long i = 4 * n4 + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        float x = v[i];
        if (!(x >= 0.0f && x <= 3.402823466e38f)) atomicMin(first, (unsigned long long)i);
    }
}

// device copy of projections that flags any value that is not finite and >= 0
__global__ void k_copy_checked(const float *__restrict__ src, float *__restrict__ dst, long long n, int *status)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    if (i < n) {
        float v = src[i];
        dst[i] = v;
        bad = !(v >= 0.0f && v <= 3.402823466e38f);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kStatusBadData);
}

uspg_status uspg_set_projections(uspg_ctx *c, const float *p, int32_t on_device, uspg_stream stream)
{
    if (!c || !p) return fail(c, USPG_EINVAL, "NULL argument");
    size_t n = (size_t)c->scan.n_views * c->n_rays;
    auto refuse = [&](long long bad) {
        std::ostringstream os;
        os << "projection " << bad << " (view " << bad / c->n_rays << ", ray " << bad % c->n_rays << ") is "
           << p[bad] << ": projections must be finite and >= 0";
        return fail(c, USPG_EINVAL, os.str());
    };
    // host data are checked before the context's projections change: a small
    // set on the host, a large one on the device in a staging buffer
    const bool staged = !on_device && n >= ((size_t)1 << 20);
    if (!on_device && !staged) {
        long long bad = first_bad_value(p, n);
        if (bad >= 0) return refuse(bad);
    }
    uspg_status st = ensure_state(c);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (on_device) {  // checked while copied; a bad value is reported by uspg_sync (EDEVICE)
        k_copy_checked<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, c->d_proj, (long long)n, c->d_status);
        launch_counter()++;
        USPG_CUDA(c, cudaGetLastError());
    } else if (staged) {
        if (!c->d_proj_stage) {
            USPG_CUDA(c, cudaMalloc(&c->d_proj_stage, sizeof(float) * n));
            USPG_CUDA(c, cudaMalloc(&c->d_first_bad, sizeof(unsigned long long)));
        }
        unsigned long long first = (unsigned long long)n;
        USPG_CUDA(c, cudaMemcpyAsync(c->d_first_bad, &first, sizeof(first), cudaMemcpyHostToDevice, s));
        USPG_CUDA(c, cudaMemcpyAsync(c->d_proj_stage, p, sizeof(float) * n, cudaMemcpyHostToDevice, s));
        k_first_bad<<<1216, 256, 0, s>>>(c->d_proj_stage, (long long)n, c->d_first_bad);  // 8 blocks per SM of 152
        launch_counter()++;
        USPG_CUDA(c, cudaGetLastError());
        USPG_CUDA(c, cudaMemcpyAsync(&first, c->d_first_bad, sizeof(first), cudaMemcpyDeviceToHost, s));
        USPG_CUDA(c, cudaStreamSynchronize(s));
        if (first < (unsigned long long)n) return refuse((long long)first);
        USPG_CUDA(c, cudaMemcpyAsync(c->d_proj, c->d_proj_stage, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
    } else {
        USPG_CUDA(c, cudaMemcpyAsync(c->d_proj, p, sizeof(float) * n, cudaMemcpyHostToDevice, s));
    }
    c->have_proj = true;
    return USPG_OK;
}

uspg_status uspg_set_image(uspg_ctx *c, const float *f, int32_t on_device, uspg_stream stream)
{
    if (!c || !f) return fail(c, USPG_EINVAL, "NULL argument");
    uspg_status st = ensure_state(c);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (!c->mir.on) {
        USPG_CUDA(c, cudaMemcpyAsync(c->d_f, f, sizeof(float) * c->n_cells,
                                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        return USPG_OK;
    }
    const float *src = f;  // mirrored: stage on the device, then pair up
    float *tmp = nullptr;
    if (!on_device) {
        USPG_CUDA(c, cudaMallocAsync(&tmp, sizeof(float) * c->n_cells, s));
        USPG_CUDA(c, cudaMemcpyAsync(tmp, f, sizeof(float) * c->n_cells, cudaMemcpyHostToDevice, s));
        src = tmp;
    }
    USPG_CUDA(c, image_to_pairs(c, src, c->d_f, s));
    if (tmp) USPG_CUDA(c, cudaFreeAsync(tmp, s));
    return USPG_OK;
}

__global__ void k_fill_value(float *f, long long n, float v)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) f[i] = v;
}

uspg_status uspg_fill_image(uspg_ctx *c, float value, uspg_stream stream)
{
    if (!c) return fail(c, USPG_EINVAL, "NULL context");
    uspg_status st = ensure_state(c);
    if (st) return st;
    long long n = image_floats(c);  // pairs hold the value twice
    k_fill_value<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(c->d_f, n, value);
    launch_counter()++;
    USPG_CUDA(c, cudaGetLastError());
    return USPG_OK;
}

uspg_status uspg_get_image(const uspg_ctx *cc, float *f, int32_t to_device, uspg_stream stream)
{
    uspg_ctx *c = const_cast<uspg_ctx *>(cc);
    if (!c || !f) return fail(c, USPG_EINVAL, "NULL argument");
    if (!c->d_f) return fail(c, USPG_ENOTREADY, "no image");
    cudaStream_t s = (cudaStream_t)stream;
    if (!c->mir.on) {
        USPG_CUDA(c, cudaMemcpyAsync(f, c->d_f, sizeof(float) * c->n_cells,
                                     to_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
        return USPG_OK;
    }
    if (to_device) {
        USPG_CUDA(c, image_from_pairs(c, c->d_f, f, s));
        return USPG_OK;
    }
    float *tmp = nullptr;
    USPG_CUDA(c, cudaMallocAsync(&tmp, sizeof(float) * c->n_cells, s));
    USPG_CUDA(c, image_from_pairs(c, c->d_f, tmp, s));
    USPG_CUDA(c, cudaMemcpyAsync(f, tmp, sizeof(float) * c->n_cells, cudaMemcpyDeviceToHost, s));
    USPG_CUDA(c, cudaFreeAsync(tmp, s));
    return USPG_OK;
}

// per-view simultaneous MART as one CUDA graph per option set
static uspg_status per_view(uspg_ctx *c, const uspg_mart_opts *o, cudaStream_t s)
{
    int nv = c->scan.n_views;
    std::vector<int> order(nv);
    if (o->view_order) {
        std::vector<char> seen(nv, 0);
        for (int q = 0; q < nv; q++) {
            int k = o->view_order[q];
            if (k < 0 || k >= nv || seen[k]) return fail(c, USPG_EINVAL, "view_order is not a permutation");
            seen[k] = 1;
            order[q] = k;
        }
    } else {
        std::iota(order.begin(), order.end(), 0);
    }
    long long steps = (long long)o->iterations * nv;
    if (o->view_steps > 0 && o->view_steps < steps) steps = o->view_steps;
    const int linear = o->update_rule == USPG_LINEAR_EQ18;
    const bool stop = o->stop_tol > 0.0;
    int *stop_flags = c->d_sweeps;  // [0] sweeps run, [1] a cell moved, [2] converged
    UpdateRule U{(float)o->lambda, linear, stop ? (float)o->stop_tol : 0.0f, stop_flags + 1};
    const int *done = stop ? stop_flags + 2 : nullptr;
    std::ostringstream key;
    key << steps << ':' << o->lambda << ':' << linear << ':' << o->stop_tol;
    for (int k : order) key << ',' << k;
    auto it = c->graphs.find(key.str());
    if (it == c->graphs.end()) {
        Graph g;
        cudaStream_t cs = c->cap_stream;
        int64_t before = launch_counter();
        USPG_CUDA(c, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        uspg_status st = stop ? launch_stop_reset(c, cs) : USPG_OK;
        for (long long q = 0; q < steps && !st; q++) {
            int k = order[q % nv];
            st = launch_forward_view(c, k, nullptr, c->d_res, cs, linear, done);
            if (!st) st = launch_backward_view(c, k, U, done, cs);
            if (!st && stop && q % nv == nv - 1) st = launch_sweep_end(c, cs);  // Eq. 19 after each sweep
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &graph);
        if (st) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        USPG_CUDA(c, e);
        g.graph = graph;
        g.nodes = launch_counter() - before;
        launch_counter() = before;  // captured, not launched
        USPG_CUDA(c, cudaGraphInstantiate(&g.exec, graph, 0));
        it = c->graphs.emplace(key.str(), g).first;
    }
    USPG_CUDA(c, cudaGraphLaunch(it->second.exec, s));
    launch_counter() += it->second.nodes;
    return USPG_OK;
}

uspg_status uspg_mart(uspg_ctx *c, const uspg_mart_opts *o, uspg_stream stream)
{
    if (!c || !o) return fail(c, USPG_EINVAL, "NULL argument");
    if (!c->built) return fail(c, USPG_ENOTREADY, "coefficients not built");
    if (!c->have_proj) return fail(c, USPG_ENOTREADY, "projections not set");
    if (o->iterations < 0 || o->view_steps < 0) return fail(c, USPG_EINVAL, "iterations and view_steps must be >= 0");
    if (!(o->lambda > 0.0) || !(o->lambda < 2.0)) return fail(c, USPG_EINVAL, "lambda must be in (0, 2)");
    cudaStream_t s = (cudaStream_t)stream;
    c->last_sweeps = o->iterations;
    if (o->iterations == 0) return USPG_OK;
    if (o->schedule == USPG_SEQUENTIAL) {
        if (o->update_rule != USPG_POWER && o->update_rule != USPG_LINEAR_EQ18)
            return fail(c, USPG_EINVAL, "unknown update rule");
        if (o->stop_tol < 0.0) return fail(c, USPG_EINVAL, "stop_tol must be >= 0");
        c->last_sweeps = -1;
        return c->store_form == USPG_STORE_SEGMENTS ? launch_sequential_segments(c, o, s) : launch_sequential(c, o, s);
    }
    if (o->schedule != USPG_PER_VIEW) return fail(c, USPG_EINVAL, "unknown schedule");
    if (c->store_form == USPG_STORE_SEGMENTS)
        return fail(c, USPG_EUNSUPPORTED, "the segment store serves the ray-sequential schedule");
    if (o->update_rule != USPG_POWER && o->update_rule != USPG_LINEAR_EQ18)
        return fail(c, USPG_EINVAL, "unknown update rule");
    if (o->stop_tol < 0.0) return fail(c, USPG_EINVAL, "stop_tol must be >= 0");
    if (o->stop_tol > 0.0 && o->view_steps > 0)
        return fail(c, USPG_EINVAL, "stop_tol (Eq. 19, checked after whole sweeps) excludes view_steps");
    if (o->stop_tol > 0.0) c->last_sweeps = -1;  // the sweeps run are read back from the device
    return per_view(c, o, s);
}

uspg_status uspg_mart_kernel_times(uspg_ctx *c, const uspg_mart_opts *o, float *ms_fwd, float *ms_bwd, int32_t cap,
                                   int32_t *n, uspg_stream stream)
{
    if (!c || !o || !ms_fwd || !ms_bwd || !n) return fail(c, USPG_EINVAL, "NULL argument");
    if (!c->built) return fail(c, USPG_ENOTREADY, "coefficients not built");
    if (!c->have_proj) return fail(c, USPG_ENOTREADY, "projections not set");
    if (o->schedule != USPG_PER_VIEW) return fail(c, USPG_EINVAL, "kernel timing covers the per-view schedule");
    if (c->store_form == USPG_STORE_SEGMENTS)
        return fail(c, USPG_EUNSUPPORTED, "the segment store serves the ray-sequential schedule");
    if (o->update_rule != USPG_POWER && o->update_rule != USPG_LINEAR_EQ18)
        return fail(c, USPG_EINVAL, "unknown update rule");
    const int linear = o->update_rule == USPG_LINEAR_EQ18;
    UpdateRule U{(float)o->lambda, linear, 0.0f, nullptr};
    int nv = c->scan.n_views;
    long long steps = (long long)o->iterations * nv;
    if (steps > cap) return fail(c, USPG_EINVAL, "cap < iterations * n_views");
    std::vector<int> order(nv);
    for (int q = 0; q < nv; q++) order[q] = o->view_order ? o->view_order[q] : q;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<cudaEvent_t> ev(2 * steps + 1);
    for (auto &e : ev) USPG_CUDA(c, cudaEventCreate(&e));
    USPG_CUDA(c, cudaEventRecord(ev[0], s));
    long long q = 0;
    uspg_status st = USPG_OK;
    for (int it = 0; it < o->iterations && !st; it++)
        for (int v = 0; v < nv && !st; v++, q++) {
            st = launch_forward_view(c, order[v], nullptr, c->d_res, s, linear);
            if (!st) st = (uspg_status)(cudaEventRecord(ev[2 * q + 1], s) ? USPG_ECUDA : USPG_OK);
            if (!st) st = launch_backward_view(c, order[v], U, nullptr, s);
            if (!st) st = (uspg_status)(cudaEventRecord(ev[2 * q + 2], s) ? USPG_ECUDA : USPG_OK);
        }
    cudaError_t e = cudaStreamSynchronize(s);
    for (long long i = 0; i < steps && !st && e == cudaSuccess; i++) {
        cudaEventElapsedTime(&ms_fwd[i], ev[2 * i], ev[2 * i + 1]);
        cudaEventElapsedTime(&ms_bwd[i], ev[2 * i + 1], ev[2 * i + 2]);
    }
    for (auto &x : ev) cudaEventDestroy(x);
    if (st) return st;
    USPG_CUDA(c, e);
    *n = (int32_t)steps;
    return USPG_OK;
}

uspg_status uspg_autotune(uspg_ctx *c, int32_t *choice, uspg_stream stream)
{
    if (!c) return fail(c, USPG_EINVAL, "NULL context");
    if (!c->built) return fail(c, USPG_ENOTREADY, "coefficients not built");
    if (c->store_form == USPG_STORE_SEGMENTS)
        return fail(c, USPG_EUNSUPPORTED, "the per-view kernels read the representative store");
    if (!c->have_proj) return fail(c, USPG_ENOTREADY, "projections not set");
    cudaStream_t s = (cudaStream_t)stream;
    float *saved = nullptr;
    USPG_CUDA(c, cudaMallocAsync(&saved, sizeof(float) * image_floats(c), s));
    USPG_CUDA(c, cudaMemcpyAsync(saved, c->d_f, sizeof(float) * image_floats(c), cudaMemcpyDeviceToDevice, s));
    cudaEvent_t e0, e1;
    USPG_CUDA(c, cudaEventCreate(&e0));
    USPG_CUDA(c, cudaEventCreate(&e1));
    // median-free best-of-4 (first run warms up) of one view's kernel
    auto time_it = [&](bool fwd) -> float {
        float best = 1e30f;
        for (int rep = 0; rep < 4; rep++) {
            cudaEventRecord(e0, s);
            uspg_status st = fwd ? launch_forward_view(c, 0, nullptr, c->d_res, s)
                                 : launch_backward_view(c, 0, UpdateRule{1e-3f, 0, 0.0f, nullptr}, nullptr, s);
            cudaEventRecord(e1, s);
            if (st != USPG_OK || cudaEventSynchronize(e1) != cudaSuccess) return 1e30f;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best) best = ms;
        }
        return best;
    };
    const int fwd_opts[4] = {2, 4, 6, 8};  // resident blocks per SM of the forward
    const int bwd_opts[4] = {2, 4, 6, 8};  // resident blocks per SM of the correction
    // a candidate replaces the kernels' default shape (0) only when it is at
    // least 5% faster, so timing noise (or a profiler's serialisation) leaves
    // the default in place
    const float kGain = 0.95f;
    c->fwd_blocks_per_sm = 0;
    float bf = time_it(true) * kGain;
    int fb = 0, bs = 0;
    for (int v : fwd_opts) {
        c->fwd_blocks_per_sm = v;
        float t = time_it(true);
        if (t < bf) {
            bf = t;
            fb = v;
        }
    }
    c->fwd_blocks_per_sm = fb;
    launch_forward_view(c, 0, nullptr, c->d_res, s);
    c->bwd_blocks_per_sm = 0;
    float bb = time_it(false) * kGain;
    for (int v : bwd_opts) {
        c->bwd_blocks_per_sm = v;
        float t = time_it(false);
        if (t < bb) {
            bb = t;
            bs = v;
        }
    }
    c->bwd_blocks_per_sm = bs;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    c->err.clear();
    USPG_CUDA(c, cudaMemcpyAsync(c->d_f, saved, sizeof(float) * image_floats(c), cudaMemcpyDeviceToDevice, s));
    USPG_CUDA(c, cudaFreeAsync(saved, s));
    USPG_CUDA(c, cudaStreamSynchronize(s));
    for (auto &kv : c->graphs) {  // captured launches carry the old configuration
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    c->graphs.clear();
    if (choice) {
        choice[0] = fb;
        choice[1] = bs;
    }
    return USPG_OK;
}

uspg_status uspg_mart_sweeps(uspg_ctx *c, int32_t *sweeps)
{
    if (!c || !sweeps) return fail(c, USPG_EINVAL, "NULL argument");
    if (c->last_sweeps >= 0) {
        *sweeps = c->last_sweeps;
        return USPG_OK;
    }
    int v = 0;
    USPG_CUDA(c, cudaMemcpy(&v, c->d_sweeps, sizeof(int), cudaMemcpyDeviceToHost));
    *sweeps = v;
    return USPG_OK;
}

uspg_status uspg_forward_project(uspg_ctx *c, int32_t view, float *out, uspg_stream stream)
{
    if (!c || !out) return fail(c, USPG_EINVAL, "NULL argument");
    if (!c->built) return fail(c, USPG_ENOTREADY, "coefficients not built");
    if (view < 0 || view >= c->scan.n_views) return fail(c, USPG_EINVAL, "bad view");
    if (c->store_form == USPG_STORE_SEGMENTS)
        return fail(c, USPG_EUNSUPPORTED, "the per-view kernels read the representative store");
    return launch_forward_view(c, view, out, nullptr, (cudaStream_t)stream);
}

uspg_status uspg_resample_cartesian(uspg_ctx *c, int32_t mode, int32_t nx, int32_t ny, float *out,
                                    int32_t out_on_device, uspg_stream stream)
{
    if (!c || !out) return fail(c, USPG_EINVAL, "NULL argument");
    uspg_status st = ensure_state(c);
    if (st) return st;
    int ns = c->scan.geometry == USPG_CONE_3D ? c->n_slabs : 1;
    if (mode == USPG_RESAMPLE_BIJECTION) {
        for (int n = 1; n <= c->n_rings; n++)
            if (c->ng[n - 1] != 8 * n - 4)
                return fail(c, USPG_EUNSUPPORTED, "the bijective resample needs 4(2n-1) sectors per ring");
        if (nx != 2 * c->n_rings || ny != 2 * c->n_rings)
            return fail(c, USPG_EINVAL, "the bijective resample writes a 2N x 2N image");
    } else if (mode != USPG_RESAMPLE_POINT) {
        return fail(c, USPG_EINVAL, "unknown resample mode");
    }
    if (nx < 1 || ny < 1) return fail(c, USPG_EINVAL, "nx, ny must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    size_t bytes = sizeof(float) * (size_t)nx * ny * ns;
    float *dst = out;
    if (!out_on_device) {  // the context's device image for host destinations, kept between calls
        if (bytes > c->cap_rs_out) {
            USPG_CUDA(c, cudaStreamSynchronize(s));
            cudaFree(c->d_rs_out);
            c->d_rs_out = nullptr;
            USPG_CUDA(c, cudaMalloc(&c->d_rs_out, bytes));
            c->cap_rs_out = bytes;
        }
        dst = c->d_rs_out;
    }
    st = launch_resample(c, mode, nx, ny, dst, s);
    if (st) return st;
    if (!out_on_device) {
        USPG_CUDA(c, cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, s));
        USPG_CUDA(c, cudaStreamSynchronize(s));
    }
    return USPG_OK;
}

}  // extern "C"
