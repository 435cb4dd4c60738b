// Internal definitions shared by the translation units of libuspg.
// Nothing here is part of the C ABI (see include/uspg.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <string>
#include <vector>
#include <map>
#include <atomic>

#include "../../include/uspg.h"

namespace uspg {

constexpr double kTwoPi = 6.283185307179586;  // 2*pi rounded to double
constexpr double kNudge = 1e-12;              // counter-clockwise tie-break (rad)
constexpr double kMinPiece = 1e-9;            // fraction of a cell dropped as a sliver
constexpr int kMaxRings = 1024;
constexpr int kMaxSlabs = 1024;
constexpr int kMaxSectors = 4096;
constexpr int kRowPad = 8;       // ray-major rows are padded to a multiple of this (16 B of FP16)
constexpr int kSlice = 32;       // cells per slice of the cell-major store
constexpr int kMaxRing0Cross = 32;
constexpr int kTileAlign = 8;  // tiles start on a multiple of this many entries

// device status bits (uspg_sync)
constexpr int kStatusCountMismatch = 1;
constexpr int kStatusRing0Overflow = 2;
constexpr int kStatusBounds = 4;
constexpr int kStatusTimeout = 8;
constexpr int kStatusCellRays = 16;
constexpr int kStatusBadData = 32;  // device projections with a value that is not finite and >= 0
constexpr int kMaxCellRays = 2047;  // rays of one view through one cell (11-bit lane count)

// Stored cell index of a representative row: slab (10 b) | ring (10 b) | sector (12 b).
__host__ __device__ inline uint32_t pack_cell(int slab, int ring, int sector)
{
    return (uint32_t(slab) << 22) | (uint32_t(ring) << 12) | uint32_t(sector);
}
__host__ __device__ inline int cell_slab(uint32_t x) { return int(x >> 22); }
__host__ __device__ inline int cell_ring(uint32_t x) { return int((x >> 12) & 1023u); }
__host__ __device__ inline int cell_sector(uint32_t x) { return int(x & 4095u); }

// z-mirror of a centred cone scan (source on the mid-plane z = 0 of a slab
// stack centred on it): detector rows v and n_v-1-v see mirror-image rays,
// whose pieces have the same lengths in slabs s and n_s-1-s.  Only the rows
// v < (n_v+1)/2 are stored (ray ids below n_rows); the rest are their mirrors.
struct Mirror {
    int on;                // 0: every row is stored
    int n_u, n_v, n_slabs;
    int n_rows;            // stored rays per view (= n_rays when off)
};

// A mirrored context keeps its image as pairs {f(slab s), f(slab n_s-1-s)}
// over the lower and middle slabs: pair k = s * cells_per_slab + c for
// s < (n_s+1)/2 (the middle slab of an odd stack holds its value twice), so
// one 8-byte access serves a cell and its mirror.
__host__ __device__ inline long long image_pairs(long long cells_per_slab, int n_slabs)
{
    return (long long)((n_slabs + 1) / 2) * cells_per_slab;
}

__host__ __device__ inline uint32_t flip_slab(uint32_t pc, int n_slabs)
{
    return (uint32_t(n_slabs - 1 - cell_slab(pc)) << 22) | (pc & 0x3fffffu);
}
// detector row of a ray (ray = row * n_u + column)
__host__ __device__ inline int ray_row(int ray, int n_u) { return ray / n_u; }
// mirror image of a ray: row v -> n_v-1-v, same column
__host__ __device__ inline int mirror_ray(int ray, int n_u, int n_v)
{
    return ray + (n_v - 1 - 2 * ray_row(ray, n_u)) * n_u;
}

// Per ring: first cell id in a slab (H_n of Eq. 2), sector count, and the
// sector shift produced by one 1/G-turn rotation (n_g / G).
struct RingEntry {
    int head;
    int ng;
    int step;
    int chunk0;  // first slice of this ring within a slab of the cell-major store
};

// Scan and grid geometry as the generator needs it (all by value).
struct Geometry {
    int geometry, n_rings, n_slabs, n_u, n_v, n_rays, n_views, weight_mode;
    int n_rows;  // traced rows per representative: rays 0 .. n_rows-1 (the lower detector rows when mirrored)
    long long arc_num, arc_den;
    double r, h, z_min, du, dv, d_so, d_sd;
    long long cells_per_slab;
};

// View of one representative's stored rows as a kernel sees it.
struct StoreView {
    const long long *row_ptr;  // [n_rays + 1], absolute entry offsets
    const uint32_t *idx;       // packed cells
    const void *w;             // weights, stored dtype
    const float *rowmax;       // [n_rays]
    const long long *slice_off;   // [slices_per_rep] absolute entry offsets
    const uint32_t *slice_meta;   // [slices_per_rep] pack_cell(slab, ring, sector0)
    const int *slice_width;       // [slices_per_rep]
    const uint32_t *sray;         // cell-major ray ids
    const void *sw;               // cell-major weights
};

std::atomic<int64_t> &launch_counter();  // kernels launched (host threads may launch concurrently)

// ---- generator (generator.cu) ----
struct GenOut {
    int n_reps;
    long long nnz;      // unpadded entries
    long long nnz_reps_full;  // entries of the representatives' full rows (mirrored rows counted)
    long long nnz_pad;  // padded ray-major entries
    long long sell_entries;
    long long max_row;
};

// ---- host runtime context ----
struct Graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t nodes = 0;
};

}  // namespace uspg

struct uspg_ctx {
    // grid
    int n_rings = 0, sector_rule = 0, n_slabs = 1, G = 1;
    double r = 0, h = 1, z_min = 0;
    std::vector<int> ng, head;
    long long cells_per_slab = 0, n_cells = 0;
    // scan
    uspg_scan_desc scan{};
    int n_rays = 0;
    uspg::Mirror mir{};  // z-mirror: stored rows per view mir.n_rows (all rays when mir.on == 0)
    // coefficient options
    int weight_mode = USPG_LENGTH, dtype = USPG_F32;
    int symmetry = USPG_SYMMETRY_AUTO;  // transverse mirror of representative rows (uspg_coeff_opts)
    double w_scale = 1.0;  // stored weight = length / w_scale
    // view classes
    int n_reps = 0;
    std::vector<int> rep_view;     // view index of each representative
    std::vector<int> rep_of_view;  // representative index of each view
    std::vector<int> m_of_view;    // rotation of each view from its representative, in 1/G turns
    // device tables
    uspg::RingEntry *d_ring = nullptr;
    int *d_slice_ring = nullptr;  // [slices_per_slab] ring of each slice of a slab (cell-major store)
    double2 *d_bdir = nullptr;  // boundary directions, indexed head + j
    float2 *d_bdirf = nullptr;  // the same in FP32 (pre-tests)
    int slices_per_slab = 0;
    long long slices_per_rep = 0;
    // store
    bool built = false;
    long long *d_row_ptr = nullptr;
    uint32_t *d_idx = nullptr;
    void *d_w = nullptr;
    float *d_rowmax = nullptr;
    long long *d_slice_off = nullptr;
    uint32_t *d_slice_meta = nullptr;
    uint2 *d_slice_desc = nullptr;  // [reps][slices] {first slot relative to the representative, meta}
    int *d_slice_width = nullptr;
    uint32_t *d_sray = nullptr;
    void *d_sw = nullptr;
    // cell-major store with the lanes of every slice ordered by ray count
    uint32_t *d_cm_ray = nullptr;    // [slots] ray ids
    void *d_cm_w = nullptr;          // [slots] weights, stored dtype
    uint16_t *d_lane_desc = nullptr; // [reps][slices][32] (source lane << 11) | count
    long long cap_cm = 0;
    uint32_t *d_grp_ray = nullptr;      // ray of each kRowPad-entry group of the ray-major store
    long long cap_grp = 0;
    float *d_sacc = nullptr;            // per-ray sum accumulator of the forward (kept zero between views)
    // launch shape of the per-view kernels (autotuned): resident blocks per SM
    int fwd_blocks_per_sm = 0, bwd_blocks_per_sm = 0;
    uspg::GenOut gen{};
    // generator scratch and capacities (buffers are reused across rebuilds so
    // that captured graphs stay valid; a reallocation clears the graph cache)
    int *d_counts = nullptr, *d_rep_view = nullptr, *d_cell_cnt = nullptr, *d_cell_fill = nullptr;
    long long *d_rel = nullptr, *d_stats = nullptr;
    double *d_w64 = nullptr;
    size_t cap_idx = 0, cap_w = 0, cap_w64 = 0, cap_sell = 0;
    bool store_moved = false;
    int gen_fallbacks = 0;  // builds whose FP32 row bound was exceeded
    long long gen_walked_rows = 0;  // rows the last build walked (the rest are mirror images)
    int gen_derived_reps = 0;        // representatives whose columns the last build derived
    int *d_plan = nullptr;          // transverse-symmetry tables (generator.cu)
    int *d_tied = nullptr;          // [rows + 1] tie flag of each walked row, then a counter
    long long *d_retrace = nullptr; // [rows] mirror rows walked after all
    long long nnz_all_views = 0;
    std::vector<long long> h_row_ptr;  // host copy for get_row
    std::vector<long long> h_rep_entry0;  // first ray-major entry of each representative (+ end)
    std::vector<long long> h_sell_base;   // first cell-major slot of each representative
    // pinned read-back area of the generator (statistics, entry offsets, slice
    // totals, flags): copies into it do not stall the host until it reads them
    long long *h_gen_pin = nullptr;
    long long *d_gen_small = nullptr;  // [reps + 1] gathered entry offsets
    // state
    float *d_f = nullptr;
    float *d_proj = nullptr;
    float *d_proj_stage = nullptr;         // large host projections land here to be checked (set_projections)
    float *d_rs_std = nullptr;             // resample: the image in the standard layout (mirrored contexts)
    float *d_rs_out = nullptr;             // resample: device image for a host destination
    size_t cap_rs_out = 0;
    unsigned long long *d_first_bad = nullptr;
    bool have_proj = false;
    float *d_res = nullptr;  // per-ray correction terms (float2 [n_rays], or float4 [2 n_rows] mirrored)
    int *d_status = nullptr;
    int *d_sweeps = nullptr;  // [4]: sweeps run, and the per-view Eq. 19 flags (moved, converged)
    cudaStream_t cap_stream = nullptr;
    std::map<std::string, uspg::Graph> graphs;
    int last_sweeps = 0;
    std::string err;
    // set on a context that reads another context's store and tables (which
    // must outlive it); its image, projections, scratch and graphs are its own
    const uspg_ctx *store_src = nullptr;
    // USPG_STORE_SEGMENTS: the first view's segments (binary model, Algorithm 1)
    int store_form = USPG_STORE_REPRESENTATIVES;
    long long *d_seg_ptr = nullptr;   // [n_rays + 1] first segment of each ray
    uint64_t *d_seg_fa = nullptr;     // [segments] azimuth where the segment starts (fixed turns)
    uint64_t *d_seg_fb = nullptr;     // [segments] azimuth where it ends
    uint32_t *d_seg_rs = nullptr;     // [segments] slab << 22 | ring << 12 | back (see segments.cu)
    signed char *d_seg_dir = nullptr; // [n_rays] direction the azimuth turns along the ray (+1, -1, 0)
    uint64_t *d_view_turns = nullptr; // [n_views] source angle of each view (fixed turns)
    long long n_segments = 0;
    int max_segments = 0;             // longest ray, in segments
};

namespace uspg {

// generator.cu
uspg_status build_store(uspg_ctx *c, cudaStream_t s);
Geometry make_geometry(const uspg_ctx *c);
// exclusive prefix sum of n counts into out[0..n] (out[n] = total)
cudaError_t scan_counts(const int *in, long long n, long long *out, cudaStream_t s);
// segments.cu: the first view's segment store of the binary model
uspg_status build_segments(uspg_ctx *c, cudaStream_t s);
uspg_status launch_sequential_segments(uspg_ctx *c, const uspg_mart_opts *o, cudaStream_t s);
uspg_status segment_row(uspg_ctx *c, int view, int ray, std::vector<long long> &cells);
void free_segments(uspg_ctx *c);
// mart.cu
struct UpdateRule;
// linear = 1: the ray terms carry P/Pbar (Eq. 18) instead of ln(P/Pbar); done
// (device, may be NULL): the per-view kernels do nothing once *done != 0
uspg_status launch_forward_view(uspg_ctx *c, int view, float *out_s, float *out_res, cudaStream_t s, int linear = 0,
                                const int *done = nullptr);
uspg_status launch_backward_view(uspg_ctx *c, int view, const UpdateRule &U, const int *done, cudaStream_t s);
// Eq. 19 bookkeeping of a per-view run on c->d_sweeps[0..2] (sweeps, moved, converged)
uspg_status launch_stop_reset(uspg_ctx *c, cudaStream_t s);
uspg_status launch_sweep_end(uspg_ctx *c, cudaStream_t s);
uspg_status launch_sequential(uspg_ctx *c, const uspg_mart_opts *o, cudaStream_t s);
// device bytes currently held by a context (its own buffers only)
long long ctx_device_bytes(const uspg_ctx *c);
// floats of the context's image buffer (pairs when mirrored)
long long image_floats(const uspg_ctx *c);
// image layout conversions (standard [cells] <-> mirrored pairs) on stream s
cudaError_t image_to_pairs(const uspg_ctx *c, const float *f, float *pairs, cudaStream_t s);
cudaError_t image_from_pairs(const uspg_ctx *c, const float *pairs, float *f, cudaStream_t s);
// a new context on src's grid, scan and built store, with its own image,
// projections and scratch: one more reconstruction of src's geometry without
// a second copy of the coefficients
uspg_status ctx_share_store(const uspg_ctx *src, uspg_ctx **out);
StoreView store_view(const uspg_ctx *c, int rep);
// resample.cu
uspg_status launch_resample(uspg_ctx *c, int mode, int nx, int ny, float *out, cudaStream_t s);

uspg_status fail(uspg_ctx *c, uspg_status st, const std::string &msg);
uspg_status cuda_fail(uspg_ctx *c, cudaError_t e, const char *what);

}  // namespace uspg

#define USPG_CUDA(ctx, call)                                           \
    do {                                                               \
        cudaError_t e__ = (call);                                      \
        if (e__ != cudaSuccess) return uspg::cuda_fail((ctx), e__, #call); \
    } while (0)
