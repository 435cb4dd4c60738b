// Reconstruction server: a request loop with continuous batching.
//
// Jobs (grid + scan + coefficient options + MART options + projections)
// arrive through uspg_server_submit from any host thread.  Two library
// threads do the device work:
//  - the scheduler admits queued jobs while a slot is free and the job's
//    device footprint fits the budget next to the resident ones, and advances
//    every running job by chunks of whole sweeps (per-view schedule; a sweep
//    is one graph launch of its view steps) on the job's own stream: each
//    pass issues the next chunk of each job whose previous chunk has
//    completed, so jobs that arrive while others run start at once and their
//    kernels overlap on the device (continuous batching);
//  - job streams get a priority by job size (smaller first), and the graphs
//    of a job run at its stream's priority, so short jobs are not stuck
//    behind the kernels of a large one;
//  - the preparer builds the coefficients of an admitted job whose geometry
//    has no resident store, uploads its projections and sets its initial
//    image, so that neither a build nor a large copy stalls the running jobs.
// Coefficients are kept per geometry: the first job of a geometry builds its
// store, and every later or concurrent job of that geometry reads the same
// store through a context of its own (image, projections, scratch, graphs).
// Finished jobs return their contexts to the geometry's pool, so a steady
// stream allocates nothing.  A geometry none of whose contexts is in use can
// be evicted, least recently used first, when an admission needs its memory.
// Per job the arithmetic is exactly the single-job path (the same kernels on
// the same store), so each result equals the job run alone up to the order of
// the forward kernel's atomic additions.
#include "internal.cuh"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <list>
#include <mutex>
#include <sstream>
#include <thread>

namespace {

using clk = std::chrono::steady_clock;

struct Job {
    uint64_t id = 0;
    uspg_grid_desc grid{};
    std::vector<int32_t> sectors;
    uspg_scan_desc scan{};
    uspg_coeff_opts copt{};
    uspg_mart_opts mopt{};
    std::vector<float> proj;   // owned copy of the projections
    const float *p = nullptr;  // projections read at preparation (proj or the caller's buffer)
    float f0 = 1.0f;
    std::string key;
    clk::time_point t_submit, t_start, t_done;
    uspg_ctx *ctx = nullptr;        // the job's context (set by the preparer for a new one)
    const uspg_ctx *src = nullptr;  // store to share when the preparer makes a new context
    bool builds = false;            // the job's context is a new store's owner and builds it
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    long long reserved = 0;  // bytes counted for the job while it is prepared
    long long steps_total = 0, steps_done = 0;  // sweeps (per-view) or 1 (sequential)
    int state = 0;  // 0 queued, 1 admitted, 2 ended
    uspg_status status = USPG_OK;
    int reused = 0;
    long long updates = 0, n_cells = 0;
    std::vector<float> image;
    std::string err;
};

// The coefficient store of one geometry and the contexts that read it.
struct Store {
    uspg_ctx *owner = nullptr;     // holds the store (and one reconstruction state)
    std::vector<uspg_ctx *> free;  // contexts of this geometry no job is using
    std::vector<uspg_ctx *> all;   // every context of this geometry, owner first
    int in_use = 0;                // contexts held by admitted jobs (or being made)
    int state = 0;                 // 0 building, 1 ready, 2 failed
    long long bytes = 0;           // device bytes of all its contexts, counted in `used`
    std::string err;               // why the build failed
    clk::time_point last;
};

std::string geometry_key(const Job &j)
{
    std::ostringstream k;
    k.precision(17);
    const uspg_grid_desc &g = j.grid;
    const uspg_scan_desc &s = j.scan;
    k << g.n_rings << ',' << g.sector_rule << ',' << g.ring_width << ',' << g.n_slabs << ',' << g.slab_height << ','
      << g.z_min << ';';
    for (int v : j.sectors) k << v << ',';
    k << ';' << s.geometry << ',' << s.n_views << ',' << s.arc_num << '/' << s.arc_den << ',' << s.n_u << ','
      << s.n_v << ',' << s.du << ',' << s.dv << ',' << s.src_to_axis << ',' << s.src_to_det << ';'
      << j.copt.weight_mode << ',' << j.copt.coeff_dtype;
    return k.str();
}

// Device bytes of a context before its first build, estimated from the
// number of stored rows and the entries of a row: a ray of a parallel scan
// meets about 2 cells per ring on average (more near the axis, fewer near the
// rim), a cone ray about 1.3 per ring plus the slabs it crosses; rows are
// padded to 8 entries, and each entry costs its index, weight and FP64
// weight in the ray-major store and its slot (with padding) in the two
// cell-major copies.  Replaced by the measured footprint once a context of
// the geometry has been built.
long long estimate_bytes(const uspg_ctx *c)
{
    int wb = c->dtype == USPG_F32 ? 4 : 2;
    bool cone = c->scan.geometry == USPG_CONE_3D;
    double per_ray = (cone ? 1.4 * c->n_rings + 0.25 * c->n_slabs : 2.1 * c->n_rings) + 8.0;
    double entries = (double)c->n_reps * c->n_rays * per_ray;
    double per_entry = (4 + wb + 8 + 0.5) + 2.0 * 1.3 * (4 + wb);
    double fixed = 12.0 * c->n_cells + 4.0 * c->scan.n_views * c->n_rays + 100.0 * c->cells_per_slab;
    return (long long)(entries * per_entry + fixed);
}

std::string over_budget(long long bytes)
{
    return "the job's device footprint (" + std::to_string(bytes) + " bytes) exceeds the server's budget";
}

}  // namespace

struct uspg_server {
    int device = 0;
    long long budget = 0, used = 0, peak = 0;  // used: all contexts + reservations (scheduler only)
    int max_active = 4, chunk = 8;
    std::mutex mu;
    std::condition_variable cv, cv_prep;
    // guarded by mu
    std::deque<Job *> queue;      // submitted, not admitted
    std::deque<Job *> prep_q;     // admitted, waiting for the preparer
    std::vector<Job *> prepared;  // prepared, waiting for the scheduler
    std::map<uint64_t, Job *> jobs;
    bool stop = false, stop_prep = false;
    uint64_t next_id = 1;
    long long submitted = 0, completed = 0, failed = 0, reuses = 0, updates = 0;
    long long used_seen = 0, peak_seen = 0;  // copies of used / peak for stats
    std::vector<double> latencies;
    bool started = false;
    clk::time_point t0;
    // scheduler thread only
    std::vector<Job *> active;
    int preparing = 0;
    std::map<std::string, Store> stores;
    std::map<std::string, long long> footprint;  // measured store bytes per geometry
    bool mem_wait = false;                       // the queue head waits for memory to be freed
    std::thread th, th_prep;

    void loop();
    void prep_loop();
    void finish(Job *j, uspg_status st, const std::string &why);
    int admit(Job *j);
    void activate(Job *j);
    void fail_job(Job *j, uspg_status st, const std::string &msg);
    bool make_room(long long need, const std::string &keep);
    void release(Store &st, const std::string &key);
};

void uspg_server::fail_job(Job *j, uspg_status st, const std::string &msg)
{
    std::lock_guard<std::mutex> lk(mu);
    j->err = msg;
    j->status = st;
    j->state = 2;
    j->t_done = clk::now();
    failed++;
    cv.notify_all();
}

// Frees a failed store once no job holds one of its contexts.
void uspg_server::release(Store &st, const std::string &key)
{
    if (st.state != 2 || st.in_use > 0) return;
    for (auto it = st.all.rbegin(); it != st.all.rend(); ++it) uspg_destroy(*it);  // owner last
    used -= st.bytes;
    stores.erase(key);
}

// Evicts idle geometries (least recently used first) until `need` more bytes
// fit; true if they fit.
bool uspg_server::make_room(long long need, const std::string &keep)
{
    while (used + need > budget) {
        auto victim = stores.end();
        for (auto it = stores.begin(); it != stores.end(); ++it) {
            if (it->first == keep || it->second.in_use > 0 || it->second.state != 1) continue;
            if (victim == stores.end() || it->second.last < victim->second.last) victim = it;
        }
        if (victim == stores.end()) return false;
        Store &st = victim->second;
        for (auto it = st.all.rbegin(); it != st.all.rend(); ++it) uspg_destroy(*it);
        used -= st.bytes;
        stores.erase(victim);
    }
    return true;
}

// Admission of the queue head: 1 = handed to the preparer, 0 = must wait for
// memory, -1 = failed (already reported).
int uspg_server::admit(Job *j)
{
    auto found = stores.find(j->key);
    if (found != stores.end() && found->second.state == 2) {
        fail_job(j, USPG_EDEVICE, "the coefficient build of this geometry failed: " + found->second.err);
        return -1;
    }
    if (found != stores.end() && !found->second.free.empty()) {  // an idle context of this geometry
        Store &st = found->second;
        j->ctx = st.free.back();
        st.free.pop_back();
        st.in_use++;
        j->reused = 1;
        reuses++;
    } else if (found != stores.end()) {  // a new context reading the resident (or building) store
        Store &st = found->second;
        const uspg_ctx *o = st.owner;
        long long need = 4LL * o->n_cells + 4LL * o->scan.n_views * o->n_rays + 12LL * o->n_rays;
        if (!make_room(need, j->key) && (!active.empty() || preparing > 0)) {
            mem_wait = true;
            return 0;
        }
        j->src = o;
        j->reserved = need;
        used += need;
        st.in_use++;
        j->reused = 1;  // built by the geometry's first job (possibly still building: the preparer waits)
        reuses++;
    } else {  // first job of this geometry: a new store
        uspg_grid_desc g = j->grid;
        if (!j->sectors.empty()) g.sectors = j->sectors.data();
        uspg_ctx *c = nullptr;
        uspg_status st = uspg_create(&g, &j->scan, &j->copt, &c);  // host only
        if (st) {
            fail_job(j, st, uspg_last_error(nullptr));
            return -1;
        }
        auto known = footprint.find(j->key);
        long long need = known != footprint.end() ? known->second : estimate_bytes(c);
        if (known != footprint.end() && need > budget) {  // measured before: it can never fit
            uspg_destroy(c);
            fail_job(j, USPG_ENOMEM, over_budget(need));
            return -1;
        }
        if (!make_room(need, j->key) && (!active.empty() || preparing > 0)) {
            uspg_destroy(c);
            mem_wait = true;  // retried when a resident job ends
            return 0;
        }
        Store &s = stores[j->key];
        s.owner = c;
        s.all.push_back(c);
        s.in_use = 1;
        s.last = clk::now();
        j->ctx = c;
        j->builds = true;
        j->reserved = need;
        used += need;
    }
    peak = std::max(peak, used);
    {
        std::lock_guard<std::mutex> lk(mu);
        j->state = 1;
        j->t_start = clk::now();
        prep_q.push_back(j);
    }
    preparing++;
    cv_prep.notify_one();
    return 1;
}

// Preparer thread: the store (first job of a geometry) or a context reading
// it, then projections and initial image.  Jobs are taken in admission order,
// so a store is built before any context that reads it is made.
void uspg_server::prep_loop()
{
    cudaSetDevice(device);
    for (;;) {
        Job *j = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_prep.wait(lk, [&] { return stop_prep || !prep_q.empty(); });
            if (prep_q.empty()) return;
            j = prep_q.front();
            prep_q.pop_front();
        }
        uspg_status st = USPG_OK;
        std::string msg;
        if (j->builds) {
            st = uspg_build_coeffs(j->ctx, j->stream);
            if (!st) st = uspg_sync(j->ctx, j->stream);
            if (st) msg = j->ctx->err;
        } else if (!j->ctx) {
            st = j->src->built ? uspg::ctx_share_store(j->src, &j->ctx) : USPG_EDEVICE;
            if (st) msg = j->src->built ? uspg_last_error(nullptr) : "the coefficient build of this geometry failed";
        }
        if (!st) st = uspg_set_projections(j->ctx, j->p, 0, j->stream);
        if (!st) st = uspg_fill_image(j->ctx, j->f0, j->stream);
        if (!st) st = uspg_sync(j->ctx, j->stream);
        if (st && msg.empty() && j->ctx) msg = j->ctx->err;
        std::lock_guard<std::mutex> lk(mu);
        j->status = st;
        j->err = msg;
        prepared.push_back(j);
        cv.notify_all();
    }
}

// A prepared job: settle its memory, then run it (or report its failure).
void uspg_server::activate(Job *j)
{
    preparing--;
    mem_wait = false;
    uspg_status st;
    std::string msg;
    {
        std::lock_guard<std::mutex> lk(mu);
        st = j->status;
        msg = j->err;
    }
    Store &s = stores[j->key];
    if (j->builds) {
        long long got = uspg::ctx_device_bytes(j->ctx);
        used += got - j->reserved;
        if (!st) footprint[j->key] = got;
        if (!st && got > budget) {  // the store alone exceeds the budget
            st = USPG_ENOMEM;
            msg = over_budget(got);
        }
        s.bytes += got;
        s.state = st ? 2 : 1;
        if (st) s.err = msg;
    } else if (j->src) {  // a new context: it joins the geometry's pool
        long long got = j->ctx ? uspg::ctx_device_bytes(j->ctx) : 0;
        used += got - j->reserved;
        s.bytes += got;
        if (j->ctx) s.all.push_back(j->ctx);
    }
    j->reserved = 0;
    peak = std::max(peak, used);
    if (st) {
        if (j->ctx && s.state != 2) s.free.push_back(j->ctx);
        j->ctx = nullptr;
        s.in_use--;
        release(s, j->key);
        fail_job(j, st, msg);
        return;
    }
    j->proj.clear();
    j->proj.shrink_to_fit();
    j->p = nullptr;
    j->n_cells = j->ctx->n_cells;
    j->steps_total = j->mopt.schedule == USPG_SEQUENTIAL ? 1 : j->mopt.iterations;
    j->updates = (long long)j->mopt.iterations * j->ctx->nnz_all_views;
    active.push_back(j);
}

// Image to host, context back to its geometry's pool.
void uspg_server::finish(Job *j, uspg_status st, const std::string &why)
{
    std::vector<float> img;
    std::string msg = why;
    if (!st) {
        img.resize(j->ctx->n_cells);
        st = uspg_get_image(j->ctx, img.data(), 0, j->stream);
        if (!st) st = uspg_sync(j->ctx, j->stream);
        if (st) msg = j->ctx->err;
    }
    Store &s = stores[j->key];
    s.free.push_back(j->ctx);
    s.in_use--;
    s.last = clk::now();
    j->ctx = nullptr;
    mem_wait = false;
    std::lock_guard<std::mutex> lk(mu);
    j->err = msg;
    if (st) img.clear();
    j->image.swap(img);
    j->status = st;
    j->state = 2;
    j->t_done = clk::now();
    if (st) {
        failed++;
    } else {
        completed++;
        updates += j->updates;
        latencies.push_back(std::chrono::duration<double>(j->t_done - j->t_submit).count());
    }
    cv.notify_all();
}

void uspg_server::loop()
{
    cudaSetDevice(device);
    for (;;) {
        // jobs the preparer has finished
        std::vector<Job *> ready;
        {
            std::lock_guard<std::mutex> lk(mu);
            ready.swap(prepared);
        }
        for (Job *j : ready) activate(j);
        bool progressed = !ready.empty();
        // advance or retire running jobs
        for (size_t q = 0; q < active.size();) {
            Job *j = active[q];
            if (cudaEventQuery(j->ev) == cudaErrorNotReady) {
                q++;
                continue;
            }
            uspg_status st = USPG_OK;
            if (j->steps_done < j->steps_total) {
                if (j->mopt.schedule == USPG_SEQUENTIAL) {
                    st = uspg_mart(j->ctx, &j->mopt, j->stream);
                    j->steps_done = 1;
                } else {  // a context caches the graph of a chunk, so a reused context reuses it too
                    uspg_mart_opts o = j->mopt;
                    o.iterations = (int)std::min<long long>(chunk, j->steps_total - j->steps_done);
                    st = uspg_mart(j->ctx, &o, j->stream);
                    j->steps_done += o.iterations;
                }
                if (!st && cudaEventRecord(j->ev, j->stream) != cudaSuccess) st = USPG_ECUDA;
                if (!st) {
                    progressed = true;
                    q++;
                    continue;
                }
            }
            finish(j, st, st ? j->ctx->err : std::string());
            active.erase(active.begin() + q);
            progressed = true;
        }
        // admit queued jobs while slots and memory allow
        while (!mem_wait && (int)active.size() + preparing < max_active) {
            Job *j = nullptr;
            {
                std::lock_guard<std::mutex> lk(mu);
                if (queue.empty()) break;
                j = queue.front();
            }
            if (admit(j) == 0) break;
            std::lock_guard<std::mutex> lk(mu);
            queue.pop_front();
            progressed = true;
        }
        std::unique_lock<std::mutex> lk(mu);
        used_seen = used;
        peak_seen = peak;
        if (stop && queue.empty() && active.empty() && preparing == 0) break;
        if (!progressed) cv.wait_for(lk, std::chrono::microseconds(50));
    }
}

extern "C" {

uspg_status uspg_server_create(size_t device_budget, int32_t max_active, int32_t chunk_sweeps, uspg_server **out)
{
    if (!out || device_budget == 0 || max_active < 1 || chunk_sweeps < 1)
        return uspg::fail(nullptr, USPG_EINVAL, "server: budget > 0, max_active >= 1, chunk_sweeps >= 1");
    uspg_server *s = new uspg_server();
    cudaGetDevice(&s->device);
    s->budget = (long long)device_budget;
    s->max_active = max_active;
    s->chunk = chunk_sweeps;
    s->th_prep = std::thread([s] { s->prep_loop(); });
    s->th = std::thread([s] { s->loop(); });
    *out = s;
    return USPG_OK;
}

uspg_status uspg_server_submit(uspg_server *s, const uspg_job *job, uint64_t *id)
{
    if (!s || !job || !id || !job->projections) return uspg::fail(nullptr, USPG_EINVAL, "server: NULL argument");
    const uspg_mart_opts &m = job->mart;
    if (m.iterations < 1 || !(m.lambda > 0.0 && m.lambda < 2.0))
        return uspg::fail(nullptr, USPG_EINVAL, "server: iterations >= 1 and lambda in (0, 2)");
    if (m.schedule != USPG_PER_VIEW && m.schedule != USPG_SEQUENTIAL)
        return uspg::fail(nullptr, USPG_EINVAL, "server: unknown schedule");
    if (m.update_rule != USPG_POWER && m.update_rule != USPG_LINEAR_EQ18)
        return uspg::fail(nullptr, USPG_EINVAL, "server: unknown update rule");
    if (job->coeff.store_form != USPG_STORE_REPRESENTATIVES)
        return uspg::fail(nullptr, USPG_EUNSUPPORTED, "server: jobs use the representative store");
    int ns = job->scan.geometry == USPG_CONE_3D ? job->scan.n_v : 1;
    long long n = (long long)job->scan.n_views * job->scan.n_u * ns;
    if (job->scan.n_views < 1 || job->scan.n_u < 1 || ns < 1 || n <= 0)
        return uspg::fail(nullptr, USPG_EINVAL, "server: bad scan size");
    if (job->grid.sector_rule == USPG_SECT_CUSTOM && (!job->grid.sectors || job->grid.n_rings < 1))
        return uspg::fail(nullptr, USPG_EINVAL, "server: custom sectors need a table");
    Job *j = new Job();
    j->grid = job->grid;
    if (job->grid.sector_rule == USPG_SECT_CUSTOM)
        j->sectors.assign(job->grid.sectors, job->grid.sectors + job->grid.n_rings);
    j->grid.sectors = nullptr;
    j->scan = job->scan;
    j->copt = job->coeff;
    j->mopt = job->mart;
    j->mopt.view_order = nullptr;
    j->mopt.view_steps = 0;
    if (j->mopt.schedule == USPG_PER_VIEW) j->mopt.stop_tol = 0.0;
    if (job->flags & ~USPG_JOB_BORROW_PROJECTIONS) {
        delete j;
        return uspg::fail(nullptr, USPG_EINVAL, "server: unknown job flags");
    }
    if (job->flags & USPG_JOB_BORROW_PROJECTIONS) {
        j->p = job->projections;
    } else {
        j->proj.assign(job->projections, job->projections + n);
        j->p = j->proj.data();
    }
    j->f0 = job->f0;
    j->key = geometry_key(*j);
    // smaller jobs get higher stream priority (graphs run at the priority of
    // the stream they are launched into), so that their kernels are scheduled
    // ahead of a large job's when SMs free up: work ~ sweeps x rays x rings
    int prio_low = 0, prio_high = 0;
    cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
    double work = (double)job->mart.iterations * (double)n * job->grid.n_rings;
    int prio = work < 2e9 ? prio_high : (work < 5e10 ? (prio_low + prio_high) / 2 : prio_low);
    if (cudaStreamCreateWithPriority(&j->stream, cudaStreamNonBlocking, prio) != cudaSuccess ||
        cudaEventCreateWithFlags(&j->ev, cudaEventDisableTiming) != cudaSuccess) {
        if (j->stream) cudaStreamDestroy(j->stream);
        delete j;
        return uspg::fail(nullptr, USPG_ECUDA, "server: stream or event creation failed");
    }
    j->t_submit = clk::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (!s->started) {
            s->started = true;
            s->t0 = j->t_submit;
        }
        j->id = s->next_id++;
        s->jobs[j->id] = j;
        s->queue.push_back(j);
        s->submitted++;
        *id = j->id;
    }
    s->cv.notify_all();
    return USPG_OK;
}

uspg_status uspg_server_poll(uspg_server *s, uint64_t id, float *image, uspg_job_result *r)
{
    if (!s) return uspg::fail(nullptr, USPG_EINVAL, "server: NULL");
    Job *j = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->jobs.find(id);
        if (it == s->jobs.end()) return uspg::fail(nullptr, USPG_EINVAL, "server: unknown job id");
        j = it->second;
        if (j->state != 2) return USPG_ENOTREADY;
        s->jobs.erase(it);
    }
    if (r) {
        std::memset(r, 0, sizeof(*r));
        r->status = j->status;
        r->reused_store = j->reused;
        r->n_cells = j->n_cells;
        r->updates = j->status ? 0 : j->updates;
        auto sec = [](clk::duration d) { return std::chrono::duration<double>(d).count(); };
        bool ran = j->t_start.time_since_epoch().count() != 0;
        r->queue_s = ran ? sec(j->t_start - j->t_submit) : sec(j->t_done - j->t_submit);
        r->run_s = ran ? sec(j->t_done - j->t_start) : 0.0;
        r->latency_s = sec(j->t_done - j->t_submit);
        std::snprintf(r->message, sizeof(r->message), "%s", j->err.c_str());
    }
    if (image && !j->image.empty()) std::memcpy(image, j->image.data(), sizeof(float) * j->image.size());
    cudaEventDestroy(j->ev);
    cudaStreamDestroy(j->stream);
    delete j;
    return USPG_OK;
}

uspg_status uspg_server_drain(uspg_server *s, double timeout_s)
{
    if (!s) return uspg::fail(nullptr, USPG_EINVAL, "server: NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto until = clk::now() + std::chrono::duration_cast<clk::duration>(std::chrono::duration<double>(timeout_s));
    while (s->completed + s->failed < s->submitted) {
        if (s->cv.wait_until(lk, until) == std::cv_status::timeout && s->completed + s->failed < s->submitted)
            return uspg::fail(nullptr, USPG_ETIMEOUT, "server: jobs still running at the drain timeout");
    }
    return USPG_OK;
}

uspg_status uspg_server_stats(uspg_server *s, uspg_server_report *o)
{
    if (!s || !o) return uspg::fail(nullptr, USPG_EINVAL, "server: NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(o, 0, sizeof(*o));
    o->submitted = s->submitted;
    o->completed = s->completed;
    o->failed = s->failed;
    o->queued = (int64_t)s->queue.size();
    o->active = s->submitted - s->completed - s->failed - o->queued;
    o->device_bytes = s->used_seen;
    o->peak_device_bytes = s->peak_seen;
    o->store_reuses = s->reuses;
    std::vector<double> l = s->latencies;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto pct = [&](double p) { return l[std::min(l.size() - 1, (size_t)(p * (l.size() - 1) + 0.5))]; };
        o->p50_s = pct(0.50);
        o->p99_s = pct(0.99);
        double sum = 0;
        for (double x : l) sum += x;
        o->mean_s = sum / l.size();
    }
    if (s->started) {
        double el = std::chrono::duration<double>(clk::now() - s->t0).count();
        if (el > 0) {
            o->jobs_per_s = s->completed / el;
            o->updates_per_s = s->updates / el;
        }
    }
    return USPG_OK;
}

void uspg_server_destroy(uspg_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (Job *j : s->queue) {  // never admitted
            j->state = 2;
            j->status = USPG_EBUSY;
        }
        s->queue.clear();
    }
    s->cv.notify_all();
    s->th.join();  // running and preparing jobs end first
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop_prep = true;
    }
    s->cv_prep.notify_all();
    s->th_prep.join();
    for (auto &kv : s->stores)  // owners last: the other contexts read their stores
        for (auto it = kv.second.all.rbegin(); it != kv.second.all.rend(); ++it) uspg_destroy(*it);
    for (auto &kv : s->jobs) {
        Job *j = kv.second;
        if (j->ev) cudaEventDestroy(j->ev);
        if (j->stream) cudaStreamDestroy(j->stream);
        delete j;
    }
    delete s;
}

}  // extern "C"
