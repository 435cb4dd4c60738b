/*
 * libuspg -- GB300 (sm_103a) MART reconstruction on Uniformly Sampled Polar /
 * Cylindrical Grids, after Chaudhary, Wahi and Munshi, "Uniformly Sampled
 * Polar and Cylindrical Grid Approach for 2D, 3D Image Reconstruction using
 * Algebraic Algorithm" (arXiv 2208.12964).
 *
 * The calls follow the paper's statement of the problem: a grid (rings,
 * per-ring sectors, axial slabs), a scan (parallel-beam 2D, fan-beam 2D or
 * cone-beam 3D,
 * view angles, detector), coefficients of the lines computed once for the
 * representative views and reused for every other view by rotation, measured
 * projections in, the field function out (Eq. 17-18), and a Cartesian
 * resample for display (Sec. II.B).
 *
 * Conventions shared by every call:
 *  - Every call returns a uspg_status; no exception crosses this boundary.
 *    uspg_last_error() gives a message for the last failing call on a
 *    context (or for a failed uspg_create, through a NULL context).
 *  - Pointers passed in are borrowed for the duration of the call only; a
 *    context owns every device and host buffer it allocates.
 *  - "device" pointers are CUDA global-memory addresses of the current
 *    device (for example a torch tensor's data_ptr()); "host" pointers are
 *    ordinary process memory.
 *  - A uspg_stream is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).  Device work is enqueued on it and the call returns
 *    without waiting unless it says otherwise; faults raised inside a kernel
 *    (a bounds flag, a wait that gave up) are reported by uspg_sync().
 *  - Layouts: cells of a slab are numbered ring by ring from the axis
 *    outward, each ring counter-clockwise from the +x axis starting at its
 *    head H_n (Eq. 2); cell id = slab * cells_per_slab + H_ring + sector.
 *    Images are float32 [slabs][cells_per_slab].  Projections are float32
 *    [views][rays]; 2D ray = detector bin, 3D ray = v_row * n_u + u_col.
 *  - Not thread-safe per context: one host thread (or external locking) per
 *    uspg_ctx.  Distinct contexts are independent.
 */
#ifndef USPG_H
#define USPG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    USPG_OK = 0,
    USPG_EINVAL = 1,       /* bad argument or geometry */
    USPG_ENOMEM = 2,       /* device or host allocation failed */
    USPG_ECUDA = 3,        /* a CUDA runtime call failed (message has the CUDA error) */
    USPG_ETIMEOUT = 4,     /* a device-side wait gave up (reported by uspg_sync) */
    USPG_EUNSUPPORTED = 5, /* valid request this build does not serve */
    USPG_EBUSY = 6,        /* server: no slot or memory for the job now */
    USPG_ENOTREADY = 7,    /* coefficients not built / result not finished */
    USPG_EDEVICE = 8       /* a kernel raised its bounds/consistency flag */
} uspg_status;

/* sector rules (Sec. II.A) */
enum { USPG_SECT_6N = 0, USPG_SECT_4_2N1 = 1, USPG_SECT_CUSTOM = 2 };
/* scan geometries (Sec. III, Table 1) */
enum { USPG_PARALLEL_2D = 0, USPG_CONE_3D = 1, USPG_FAN_2D = 2 };
/* coefficient models (Sec. III.B) */
enum { USPG_LENGTH = 0, USPG_BINARY = 1 };
/* coefficient stores (Sec. III.B-C):
 *  REPRESENTATIVES  rows of one representative view per class of views that
 *                   differ by a rotation of the grid (length or binary
 *                   weights; every schedule);
 *  SEGMENTS         the paper's store for binary weights (Algorithm 1): the
 *                   first view's segments between cylinder and axial-plane
 *                   crossings (ring, slab, azimuths of the two ends); every
 *                   view's cells are enumerated from them on the fly by adding
 *                   its source angle.  One store for all views, whatever their
 *                   angles; the ray-sequential schedule. */
enum { USPG_STORE_REPRESENTATIVES = 0, USPG_STORE_SEGMENTS = 1 };
/* transverse symmetry of the representative store (uspg_build_coeffs): derive
 * the rows that are mirror images of traced rows (ALWAYS), trace every row
 * (NEVER), or derive them when the store has more rows than the GPU traces
 * at once (AUTO, 0; a small 2D store is traced whole in one pass, which is
 * faster than tracing half and deriving the rest). */
enum { USPG_SYMMETRY_AUTO = 0, USPG_SYMMETRY_ALWAYS = 1, USPG_SYMMETRY_NEVER = 2 };
/* stored coefficient precision */
enum { USPG_F32 = 0, USPG_F16 = 1, USPG_BF16 = 2 };
/* MART schedules (Sec. III.D) */
enum { USPG_SEQUENTIAL = 0, USPG_PER_VIEW = 1 };
/* update rules (Sec. III.D).  Ray-sequential: POWER f *= (P/Pbar)^(lambda w/max w),
 * LINEAR_EQ18 f *= 1 - lambda (1 - P/Pbar) (Eq. 18).  Per-view, a cell met by
 * several rays of the view takes the weighted (by coefficient) geometric mean
 * of their ratios (POWER) or arithmetic mean of their Eq. 18 factors. */
enum { USPG_POWER = 0, USPG_LINEAR_EQ18 = 1 };
/* resample modes (Sec. II.B) */
enum { USPG_RESAMPLE_POINT = 0, USPG_RESAMPLE_BIJECTION = 1 };

typedef void *uspg_stream;
typedef struct uspg_ctx uspg_ctx;

/* Grid (Sec. II.A-B, Sec. III.C).  Ring n (1-based) spans radii
 * [(n-1) r, n r]; it has 6n sectors (SECT_6N), 4(2n-1) sectors (SECT_4_2N1,
 * Eq. 1) or sectors[n-1] (SECT_CUSTOM).  n_slabs = 1 with a parallel scan is
 * the 2D grid; a cone scan stacks n_slabs slabs of height slab_height from
 * z_min.  Limits: n_rings <= 1024, n_slabs <= 1024, sectors per ring <= 4096,
 * total cells < 2^31. */
typedef struct {
    int32_t n_rings;
    int32_t sector_rule;
    const int32_t *sectors; /* host, [n_rings], used only for SECT_CUSTOM */
    double ring_width;      /* r; the grid radius is n_rings * r */
    int32_t n_slabs;
    int32_t reserved;
    double slab_height;
    double z_min;
} uspg_grid_desc;

/* Scan (Sec. III.C, Table 1).  View k (0-based) is at k * arc / n_views turns,
 * arc = arc_num/arc_den turns (1/2 for a parallel half-turn, 1 for a cone full
 * turn).  Parallel 2D: n_u bins of width du centred on the axis, n_v = 1; the
 * rays of view 0 run along +y.  Cone 3D: source at (-src_to_axis, 0, 0), flat
 * detector of n_u x n_v pixels (pitch du, dv) centred at
 * (src_to_det - src_to_axis, 0, 0) with u along +y and v along +z; the set
 * rotates about z.  Fan 2D (Table 1, the paper's 2-D phantoms): n_slabs = 1,
 * n_v = 1, source at (-src_to_axis, 0), line detector of n_u bins of pitch du
 * centred at (src_to_det - src_to_axis, 0) along +y (bin a at
 * u = (2a - (n_u-1)) du/2); dv is ignored. */
typedef struct {
    int32_t geometry;
    int32_t n_views;
    int64_t arc_num, arc_den;
    int32_t n_u, n_v;
    double du, dv;
    double src_to_axis, src_to_det;
} uspg_scan_desc;

typedef struct {
    int32_t weight_mode; /* USPG_LENGTH | USPG_BINARY */
    int32_t coeff_dtype; /* USPG_F32 | USPG_F16 | USPG_BF16 */
    int32_t store_form;  /* USPG_STORE_REPRESENTATIVES | USPG_STORE_SEGMENTS (binary only) */
    int32_t symmetry;    /* USPG_SYMMETRY_AUTO | _ALWAYS | _NEVER (representative store) */
} uspg_coeff_opts;

typedef struct {
    int32_t iterations;
    int32_t schedule;    /* USPG_SEQUENTIAL | USPG_PER_VIEW */
    int32_t update_rule; /* USPG_POWER | USPG_LINEAR_EQ18 */
    int32_t view_steps;  /* PER_VIEW: stop after this many view steps (0 = all) */
    double lambda;             /* relaxation (beta of Eq. 18), in (0, 2) */
    double stop_tol;           /* Eq. 19 tolerance; 0 = run all iterations (PER_VIEW: not with view_steps) */
    const int32_t *view_order; /* host, [n_views] permutation for PER_VIEW; NULL = 0..n_views-1 */
} uspg_mart_opts;

typedef struct {
    int64_t n_cells, cells_per_slab, n_rays, n_views, n_reps;
    int64_t nnz_store;         /* nonzeros held for the representative views */
    int64_t nnz_all_views;     /* nonzeros of the full matrix over all views */
    int64_t store_bytes;       /* device bytes of the coefficient store (both layouts) */
    int64_t full_matrix_bytes; /* bytes the same layouts would need for every view */
    int64_t max_row;           /* longest row (entries) */
    int64_t gcd;               /* rotational symmetry order G of the grid */
    int64_t mirrored;          /* 1: z-mirror store (only the lower detector rows and slabs are held) */
    int64_t slices;            /* cell-major slices (32 cells) per representative */
    int64_t walked_rows;       /* representative rows the FP64 walk traced; the rest are mirror images
                                  (transverse symmetry, Sec. III.C) of traced rows */
    int64_t derived_reps;      /* representatives whose cell-major columns were derived from their
                                  mirror source's columns (all their rows mirror images) */
} uspg_stats;

/* --- context -------------------------------------------------------------- */

/* Validates the description, builds the grid tables (Eq. 1-2) and the view
 * classes (views that share stored rows, Sec. III.C), and allocates nothing
 * on the device yet.  *out receives a new context or NULL.  EINVAL on a
 * non-positive size, sectors < 1, limits exceeded, a cone or fan source not
 * outside the grid, a detector that misses it, or the segment store asked
 * for length weights. */
uspg_status uspg_create(const uspg_grid_desc *grid, const uspg_scan_desc *scan, const uspg_coeff_opts *opts,
                        uspg_ctx **out);
/* Frees the context and all its device memory (waits for its work first). */
void uspg_destroy(uspg_ctx *ctx);
/* Message for the last failing call on ctx (ctx may be NULL: last failed create). */
const char *uspg_last_error(const uspg_ctx *ctx);
/* Waits for the context's work on `stream` and reports device-side flags:
 * EDEVICE (bounds / store overflow) or ETIMEOUT (a bounded wait gave up). */
uspg_status uspg_sync(uspg_ctx *ctx, uspg_stream stream);

/* --- coefficients (Sec. III.A-C, Algorithm 1) -------------------------------- */

/* REPRESENTATIVES: traces the rays of the representative views in FP64
 * (cylinder roots of Eq. 3-4 formed as (mr-d)(mr+d), axial and radial plane
 * crossings, midpoint cell assignment of Eq. 5-10, pieces < 1e-9 of a cell
 * dropped, repeated cells merged) and stores the rows twice: ray-major for the
 * forward ray sums and cell-major for the correction.
 * Rows that are mirror images of others under the reflection about the
 * source axis (the paper's quarter symmetry of the first view's lines, Sec.
 * III.C: column u <-> -u, azimuth phi <-> -phi) are derived instead of traced;
 * a row with a piece whose cell decision lies within 1e-7 of a sector
 * boundary or 1e-3 ring widths of the axis is traced directly either way.
 * SEGMENTS: traces the first view's rays only, to their cylinder and
 * axial-plane crossings (no radial planes, Sec. III.B), and stores each
 * segment's ring, slab and end azimuths (64-bit fixed turns); an end azimuth
 * within 2^-40 turn of a sector boundary counts as on it.
 * Replaces any earlier store. */
uspg_status uspg_build_coeffs(uspg_ctx *ctx, uspg_stream stream);
uspg_status uspg_coeff_stats(const uspg_ctx *ctx, uspg_stats *out);
/* Host copy of row `ray` of view `view` as the MART kernels see it (stored
 * representative row, sectors rotated to the view; for the segment store the
 * sectors the view's segments cover, weight 1).  cells: host int64[cap],
 * w: host double[cap] (the stored precision widened), *n = entries; if the
 * row is longer than cap, *n = its length and nothing is copied (EINVAL).
 * Synchronous. */
uspg_status uspg_get_row(const uspg_ctx *ctx, int32_t view, int32_t ray, int32_t cap, int64_t *cells, double *w,
                         int32_t *n);

/* --- data in / out ------------------------------------------------------------ */

/* Projections P_{p,l} of Eq. 17, float32 [views][rays], copied into the
 * context.  Every value must be a finite number >= 0 (measured line
 * integrals; noisy data clamped at 0).  Host data are checked before the
 * context's projections change: EINVAL names the first bad value and leaves
 * them as they were.  A set of fewer than 2^20 values is checked on the host
 * and copied with cudaMemcpyAsync (the call may return before the copy ends
 * only for page-locked memory); a larger one is copied to a device staging
 * buffer, checked there (the call waits for the check) and then copied on.
 * Device data are checked while they are copied: a bad value raises the
 * context's device flag, which the next uspg_sync reports as EDEVICE.  A ray
 * whose value is bad is skipped by every schedule (it changes no cell). */
uspg_status uspg_set_projections(uspg_ctx *ctx, const float *p, int32_t on_device, uspg_stream stream);
/* Image f_v, float32 [cells]. */
uspg_status uspg_set_image(uspg_ctx *ctx, const float *f, int32_t on_device, uspg_stream stream);
/* Sets every cell of the image to `value` (the paper starts from an arbitrary
 * field; the workloads start from 1). */
uspg_status uspg_fill_image(uspg_ctx *ctx, float value, uspg_stream stream);
uspg_status uspg_get_image(const uspg_ctx *ctx, float *f, int32_t to_device, uspg_stream stream);

/* --- reconstruction (Sec. III.D, Eq. 17-19) ---------------------------------- */

/* Runs MART on the context's image with its projections.
 * SEQUENTIAL: views 0..p-1 in order, rays in order, each ray's cells corrected
 *   before the next ray (one persistent kernel).
 * PER_VIEW: for each view of view_order, all ray sums with the current image,
 *   then each cell corrected once from all of the view's rays that meet it:
 *   POWER, the weighted geometric mean of their ratios P/Pbar (P = 0 rays zero
 *   their cells); LINEAR_EQ18, the weighted arithmetic mean of their Eq. 18
 *   factors 1 - lambda (1 - P/Pbar).
 * With stop_tol > 0, stops after the first sweep in which every correction
 * satisfies Eq. 19, |f_new - f_old| <= stop_tol |f_old| (PER_VIEW: checked on
 * the device after each sweep, the remaining view steps do nothing; EINVAL
 * together with view_steps).  ENOTREADY without coefficients or projections.
 * A segment-store context serves SEQUENTIAL only (EUNSUPPORTED for PER_VIEW;
 * likewise uspg_forward_project, uspg_autotune, uspg_mart_kernel_times,
 * batches and server jobs, which read the representative store). */
uspg_status uspg_mart(uspg_ctx *ctx, const uspg_mart_opts *opts, uspg_stream stream);
/* Forward projection of one view with the current image (Eq. 17):
 * out = device float32 [rays]. */
uspg_status uspg_forward_project(uspg_ctx *ctx, int32_t view, float *out, uspg_stream stream);
/* Sweeps run by the last uspg_mart (with stop_tol > 0: may be fewer than
 * requested).  Synchronous. */
uspg_status uspg_mart_sweeps(uspg_ctx *ctx, int32_t *sweeps);

/* --- batched reconstructions ---------------------------------------------------- */

typedef struct uspg_batch uspg_batch;

/* Batched per-view MART (Sec. III.D) over n independent contexts of any sizes
 * (grids, view counts, detectors).  Every context needs built coefficients
 * and projections, and all must store coefficients in one dtype; each runs
 * opts->iterations sweeps of its own views from its current image, exactly as
 * uspg_mart with the same opts would (view order 0..p-1).  The contexts
 * advance together: global step t runs view step t of every context that has
 * one, as three launches covering all of them (each context gets blocks in
 * proportion to its work per view); all steps are captured in one CUDA graph.
 * Creation tunes the blocks-per-work ratios per ring-count bucket on the
 * first steps (images are saved and restored; uspg_batch_tuning) and
 * captures the graph.  The contexts must stay alive,
 * and must not rebuild their coefficients, until uspg_batch_destroy.
 * Synchronous.  opts->view_order, view_steps and stop_tol are ignored; the
 * batch applies the POWER rule (EUNSUPPORTED for another); errors are
 * reported through uspg_last_error(NULL). */
uspg_status uspg_batch_create(uspg_ctx *const *ctxs, int32_t n, const uspg_mart_opts *opts, uspg_stream stream,
                              uspg_batch **out);
/* One batched run (one graph launch) on `stream`. */
uspg_status uspg_batch_run(uspg_batch *batch, uspg_stream stream);
/* Ray-cell updates of one run, kernel nodes in the graph, global steps. */
uspg_status uspg_batch_info(const uspg_batch *batch, int64_t *updates_per_run, int64_t *kernel_nodes, int64_t *steps);
/* The launch shape uspg_batch_create chose.  Instances with the same ring
 * count form a bucket; each bucket's forward gets fwd_blocks_per_group
 * blocks per 8-entry group of a view's rows and its correction
 * bwd_blocks_per_slice blocks per 32-cell slice (capped at one group per
 * thread and one slice per warp).  The shape is chosen on the first global
 * steps: the best shape common to all buckets, then each bucket's own (kept
 * where it gains at least 1%).  ms_default / ms_tuned: the same probe steps
 * with the default shape and with the chosen one.  Arrays (optional) hold
 * cap entries; *n_buckets receives the bucket count (EINVAL if above cap,
 * with *n_buckets and the times set). */
uspg_status uspg_batch_tuning(const uspg_batch *batch, int32_t cap, int32_t *rings, double *fwd_blocks_per_group,
                              double *bwd_blocks_per_slice, int32_t *n_buckets, float *ms_default, float *ms_tuned);
void uspg_batch_destroy(uspg_batch *batch);

/* --- reconstruction server ------------------------------------------------------ */

/* A request loop that serves many reconstructions (Sec. III.D MART jobs of any
 * grid and scan) concurrently on one GPU.  One scheduler thread owns all
 * device work:
 *  - admission: a queued job starts when fewer than max_active jobs run and
 *    its device footprint fits device_budget (bytes) next to the running ones;
 *  - store sharing: the first job of a geometry (grid, scan, coefficient model
 *    and dtype) builds its coefficients; every later or concurrent job of that
 *    geometry reads the same store through a context of its own (image,
 *    projections, scratch), and finished jobs' contexts are pooled for reuse;
 *    a geometry with no running job is freed, least recently used first, when
 *    an admission needs its memory;
 *  - continuous batching: each running job has its own stream and advances by
 *    chunks of chunk_sweeps sweeps (PER_VIEW; one sweep = every view once, one
 *    CUDA-graph launch); every pass of the scheduler issues the next chunk of
 *    each job whose previous chunk has finished, so jobs overlap on the device
 *    and a new job starts without waiting for the running ones to end;
 *  - priority: a job's stream gets a CUDA stream priority from its size
 *    (iterations x rays x rings; smaller jobs higher), so short jobs are not
 *    queued behind a large job's kernels;
 *  - preparation: a second library thread builds the coefficients of a job
 *    whose geometry is not resident and uploads its projections, so neither
 *    stalls the running jobs.
 * Each job computes exactly what uspg_mart computes for it alone (the same
 * kernels on the same store, view order 0..p-1), up to the order of the
 * forward kernel's floating-point atomic additions.  Thread safe: submit,
 * poll and stats may be called from any host thread.  The server uses the
 * device current when it is created. */
typedef struct uspg_server uspg_server;

typedef struct {
    uspg_grid_desc grid;      /* grid.sectors (CUSTOM) is copied at submit */
    uspg_scan_desc scan;
    uspg_coeff_opts coeff;
    uspg_mart_opts mart;      /* view_order, view_steps and stop_tol are ignored for PER_VIEW */
    const float *projections; /* host float32 [views][rays]: copied at submit, or read in place
                                 with USPG_JOB_BORROW_PROJECTIONS */
    float f0;                 /* initial value of every cell */
    int32_t flags;            /* 0 or USPG_JOB_BORROW_PROJECTIONS */
} uspg_job;

/* The server reads the job's projections from the caller's buffer when it
 * prepares the job instead of copying them at submit; the caller keeps the
 * buffer alive and unchanged until uspg_server_poll has returned the job's
 * result.  Page-locked buffers upload fastest. */
#define USPG_JOB_BORROW_PROJECTIONS 1

typedef struct {
    uspg_status status;   /* the job's own outcome (ENOMEM: its store exceeds the budget) */
    int32_t reused_store; /* 1 if another job of the same geometry built the coefficients */
    int64_t n_cells;      /* floats written to image */
    int64_t updates;      /* ray-cell updates the job ran (iterations x nonzeros over all views) */
    double queue_s;       /* submit -> start */
    double run_s;         /* start -> image on host (includes any coefficient build) */
    double latency_s;     /* submit -> image on host */
    char message[200];    /* why a failed job failed (empty on success) */
} uspg_job_result;

typedef struct {
    int64_t submitted, completed, failed, queued, active;
    int64_t store_reuses;                   /* admissions that read a store another job built */
    int64_t device_bytes, peak_device_bytes; /* held by running and idle contexts */
    double p50_s, p99_s, mean_s;            /* latency (submit -> result) of completed jobs */
    double jobs_per_s, updates_per_s;       /* completed work / time since the first submit */
} uspg_server_report;

/* Starts the scheduler and preparer threads.  EINVAL for a zero budget,
 * max_active < 1 or chunk_sweeps < 1. */
uspg_status uspg_server_create(size_t device_budget, int32_t max_active, int32_t chunk_sweeps, uspg_server **out);
/* Copies the job (projections included) into the queue and returns its id.
 * EINVAL for a malformed job (NULL projections, iterations < 1, lambda
 * outside (0, 2), an unknown rule, bad sizes).
 * Geometry errors surface later as the job's status. */
uspg_status uspg_server_submit(uspg_server *server, const uspg_job *job, uint64_t *id);
/* ENOTREADY while job `id` is queued or running.  Once it has ended: fills
 * *result (optional), copies the image to host `image` (optional, float32
 * [n_cells]; nothing is copied for a failed job), forgets the job and
 * returns OK -- the job's own outcome is result->status.  EINVAL for an
 * unknown id. */
uspg_status uspg_server_poll(uspg_server *server, uint64_t id, float *image, uspg_job_result *result);
/* Blocks until every submitted job has ended, or ETIMEOUT after timeout_s. */
uspg_status uspg_server_drain(uspg_server *server, double timeout_s);
uspg_status uspg_server_stats(uspg_server *server, uspg_server_report *out);
/* Lets running jobs finish, drops queued ones, frees every context and the
 * jobs never polled, and joins the scheduler. */
void uspg_server_destroy(uspg_server *server);

/* --- display (Sec. II.B) ------------------------------------------------------- */

/* USPG -> Cartesian.  POINT: an nx x ny image over [-R, R]^2 per slab, each
 * pixel the cell holding its centre (0 outside the disk).  BIJECTION (grids
 * with 4(2n-1) sectors only, nx = ny = 2 n_rings): square ring n of the image
 * takes the cells of ring n in the same counter-clockwise order from +x.
 * out: float32 [slabs][ny][nx], device (out_on_device = 1) or host. */
uspg_status uspg_resample_cartesian(uspg_ctx *ctx, int32_t mode, int32_t nx, int32_t ny, float *out,
                                    int32_t out_on_device, uspg_stream stream);

/* --- projection without device allocation ------------------------------------------ */

/* Capacity, in rays, of the accumulator used by uspg_forward_project_noalloc. */
#define USPG_NOALLOC_MAX_RAYS (1 << 20)

/* Forward projection of one view, out = A_view f (the ray sums of view
 * `view` for the image f), for callers that must not allocate device memory while they run: processes
 * whose device memory is owned by a pooling allocator with a fixed budget
 * (an allocation outside the pool can fail or fragment memory the pool
 * expects to own), and latency-critical loops that forbid cudaMalloc after
 * start-up because it can synchronise the device and take milliseconds.  The
 * paper has no counterpart: this is an engineering entry point of the library.
 *
 * ctx: a context whose coefficients are built (read only).  view: 0-based.
 * f: device float32 [cells], the image to project (the context's own image is
 * not used).  out: device float32 [rays].  Work is enqueued on `stream`.
 *
 * The call allocates nothing: no cudaMalloc, cudaFree or allocating library
 * routine.  Its ray-sum accumulator is a file-scope __device__ array of
 * USPG_NOALLOC_MAX_RAYS floats (4 MiB) that every GPU which loads this
 * library holds until the process exits.  The first call on a device looks
 * up that array's address (cudaGetSymbolAddress, with the device current) and
 * keeps it; make that first call on each device before any stream capture.
 * All calls share the one array: each call clears the part it uses before
 * accumulating, and calls whose work overlaps on the GPU (on different
 * streams, or from different host threads) race on it and give wrong sums --
 * serialise them.  EINVAL if the view's rays exceed USPG_NOALLOC_MAX_RAYS or
 * a pointer is NULL; ENOTREADY without coefficients. */
uspg_status uspg_forward_project_noalloc(const uspg_ctx *ctx, int32_t view, const float *f, float *out,
                                         uspg_stream stream);

/* --- instrumentation ------------------------------------------------------------ */

/* Kernels launched by this library in this process (graph replays count each
 * kernel node). */
int64_t uspg_kernel_launches(void);
/* Picks the launch shape of the per-view kernels (resident blocks per SM of
 * the forward and of the correction kernel) by timing the candidates on view
 * 0 of this context's own store; the image is saved and restored, so the
 * reconstruction state does not change.  Needs coefficients and projections.
 * A candidate replaces a kernel's default shape only when it is at least 5%
 * faster.  choice (optional, host int32[2]) receives {forward blocks per SM,
 * correction blocks per SM}, 0 where the default was kept.  Synchronous. */
uspg_status uspg_autotune(uspg_ctx *ctx, int32_t *choice, uspg_stream stream);
/* Runs PER_VIEW MART exactly as uspg_mart does, but launches its kernels one
 * by one with a CUDA event between consecutive launches on `stream`, and
 * returns each launch's device time: ms_forward[i], ms_backward[i] for the
 * i-th view step (host float arrays of length cap >= iterations * n_views;
 * *n = steps written).  Synchronous.  For measurement only: the result
 * image equals uspg_mart's. */
uspg_status uspg_mart_kernel_times(uspg_ctx *ctx, const uspg_mart_opts *opts, float *ms_forward, float *ms_backward,
                                   int32_t cap, int32_t *n, uspg_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* USPG_H */
