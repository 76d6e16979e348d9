// Request server: continuous batching of HMult+relin, HRotate and Rescale
// requests on ciphertexts resident in device memory.
//
// The paper evaluates one operation at a time and batches limbs inside it
// (Sec. III-F1); a serving engine also receives operations one by one, at
// random times and at every level.  The server keeps the evaluation keys and
// the operand ciphertexts where the caller put them (device memory), queues
// incoming requests, and runs a dispatcher thread that
//   - admits queued requests in arrival order while their device memory (the
//     output ciphertext plus the key-switch scratch) fits in the server's
//     arena, whose size is the admission budget;
//   - as soon as one of its lanes (CUDA streams) is free, launches every
//     admitted request as one launch group: one launch per step of the key
//     switch for the whole group, through the same planner as the batched path,
//     so a request that arrives while other groups run on the GPU starts in
//     the next group on another stream and its work overlaps theirs;
//   - detects completion from a CUDA event per lane, frees the scratch and
//     queues a completion record (status, output, timestamps) for the caller.
// Outputs stay in the arena until the caller releases them.  Results are the
// same as those of the single-operation entry points: the planner builds the
// same kernels over the same inputs, and no request reads another's memory.
//
// A simulation mode replaces the GPU by a timer (a group "runs" for a time
// proportional to its limbs) so that admission, batching, cancellation,
// time-outs and injected faults can be exercised without a device.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fides_internal.cuh"
#include "launchplan.cuh"

namespace {

int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

constexpr size_t kGranule = 256;
constexpr size_t kNone = ~(size_t)0;

size_t round_up(size_t x) { return (x + kGranule - 1) / kGranule * kGranule; }

// First-fit allocator over the offsets [0, size) of the arena, with the free
// blocks kept by address and merged with their neighbours on release.
class Arena {
public:
    void init(size_t size)
    {
        size_ = size / kGranule * kGranule;
        free_.clear();
        if (size_) free_[0] = size_;
        used_ = peak_ = 0;
    }
    size_t alloc(size_t bytes)
    {
        bytes = round_up(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t off = it->first, rem = it->second - bytes;
            free_.erase(it);
            if (rem) free_[off + bytes] = rem;
            used_ += bytes;
            peak_ = std::max(peak_, used_);
            return off;
        }
        return kNone;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = round_up(bytes);
        used_ -= bytes;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
    size_t size() const { return size_; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

private:
    size_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

enum ReqState { R_PENDING, R_RUNNING, R_DONE, R_ABANDONED };

struct Req {
    uint64_t id;
    fides_request r;
    const fides_key *key;
    int nl, out_limbs;
    size_t out_bytes, scr_bytes;
    size_t out_off, scr_off;
    int64_t t_submit, t_admit, t_launch;
    double scale;
    ReqState state;
};

// The device side of a lane: what the dispatcher needs to start a launch
// group and to learn when it has finished.
struct Executor {
    virtual ~Executor() {}
    // Enqueues the group; returns its status (the group still counts as
    // running until query() reports it finished).
    virtual int start(int lane, std::vector<Req *> &group, int *kernels) = 0;
    // 1 finished, 0 running, < 0 a device error.
    virtual int query(int lane) = 0;
    // Device time of the lane's last group (ms), once finished.
    virtual double device_ms(int lane) = 0;
};

class CudaExecutor : public Executor {
public:
    CudaExecutor(const fides_ctx *c, unsigned char *arena, int lanes) : c_(c), arena_(arena), lanes_(lanes) {}

    int init(int max_batch)
    {
        // Table capacity: the largest single-op table image (any type, any
        // level) times the group size, plus alignment slack per launch.
        size_t per_op = 0;
        std::vector<u64> fake(1);
        const fides_key fake_key = {c_, fake.data(), 0};
        for (int type = FIDES_OP_HMULT; type <= FIDES_OP_RESCALE; ++type) {
            for (int nl = type == FIDES_OP_RESCALE ? 2 : 1; nl <= c_->L; ++nl) {
                fides_op o;
                memset(&o, 0, sizeof(o));
                o.type = type;
                o.a.data = o.b.data = o.out.data = fake.data();
                o.a.n_limbs = nl;
                o.key = &fake_key;
                u64 *s = fake.data();
                Plan P;
                plan_stage(c_, &o, 1, 0, &s, P);
                per_op = std::max(per_op, P.image.size());
            }
        }
        cap_ = per_op * (size_t)max_batch + 64 * 1024;
        st_.assign(lanes_, nullptr);
        ev0_.assign(lanes_, nullptr);
        ev1_.assign(lanes_, nullptr);
        dtab_.assign(lanes_, nullptr);
        htab_.assign(lanes_, nullptr);
        failed_record_.assign(lanes_, false);
        for (int i = 0; i < lanes_; ++i) {
            int rc = fides_check_cuda(cudaStreamCreateWithFlags(&st_[i], cudaStreamNonBlocking), "server: stream");
            if (!rc) rc = fides_check_cuda(cudaEventCreate(&ev0_[i]), "server: event");
            if (!rc) rc = fides_check_cuda(cudaEventCreate(&ev1_[i]), "server: event");
            if (!rc) rc = fides_check_cuda(cudaMalloc((void **)&dtab_[i], cap_), "server: tables");
            if (!rc) rc = fides_check_cuda(cudaMallocHost((void **)&htab_[i], cap_), "server: host tables");
            if (rc) return rc;
        }
        return FIDES_OK;
    }

    ~CudaExecutor() override
    {
        for (int i = 0; i < (int)st_.size(); ++i) {
            if (st_[i]) cudaStreamSynchronize(st_[i]);
            if (ev0_[i]) cudaEventDestroy(ev0_[i]);
            if (ev1_[i]) cudaEventDestroy(ev1_[i]);
            if (dtab_[i]) cudaFree(dtab_[i]);
            if (htab_[i]) cudaFreeHost(htab_[i]);
            if (st_[i]) cudaStreamDestroy(st_[i]);
        }
    }

    int start(int lane, std::vector<Req *> &group, int *kernels) override
    {
        const int n = (int)group.size();
        std::vector<fides_op> ops(n);
        std::vector<u64 *> scr(n);
        for (int i = 0; i < n; ++i) {
            const Req &q = *group[i];
            fides_op &o = ops[i];
            memset(&o, 0, sizeof(o));
            o.type = q.r.type;
            o.stage = 0;
            o.a = q.r.a;
            o.b = q.r.b;
            o.out.data = (u64 *)(arena_ + q.out_off);
            o.out.n_limbs = q.out_limbs;
            o.key = q.key;
            o.steps = q.r.steps;
            scr[i] = (u64 *)(arena_ + q.scr_off);
        }
        Plan P;
        plan_stage(c_, ops.data(), n, 0, scr.data(), P);
        for (int i = 0; i < n; ++i) group[i]->scale = ops[i].out.scale;
        *kernels = plan_kernel_count(c_, P.launches);
        cudaStream_t st = st_[lane];
        int rc = FIDES_OK;
        if (P.image.size() > cap_)
            rc = fides_set_error(FIDES_ERR_UNSUPPORTED, "server: launch tables exceed %zu bytes", cap_);
        if (!rc) {
            memcpy(htab_[lane], P.image.data(), P.image.size());
            rc = fides_check_cuda(cudaEventRecord(ev0_[lane], st), "server: event");
        }
        if (!rc)
            rc = fides_check_cuda(
                cudaMemcpyAsync(dtab_[lane], htab_[lane], P.image.size(), cudaMemcpyHostToDevice, st),
                "server: table upload");
        if (!rc) {
            plan_patch(P, dtab_[lane]);
            rc = plan_run(c_, P.launches, st);
        }
        // The end event follows whatever was enqueued, so the group's memory
        // is reused only after the stream has passed it, even after an error.
        failed_record_[lane] = cudaEventRecord(ev1_[lane], st) != cudaSuccess;
        if (failed_record_[lane]) cudaStreamSynchronize(st);
        return rc;
    }

    int query(int lane) override
    {
        if (failed_record_[lane]) return -1;
        cudaError_t e = cudaEventQuery(ev1_[lane]);
        if (e == cudaSuccess) return 1;
        if (e == cudaErrorNotReady) return 0;
        fides_check_cuda(e, "server: event query");
        return -1;
    }

    double device_ms(int lane) override
    {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev0_[lane], ev1_[lane]) != cudaSuccess) return 0.0;
        return ms;
    }

private:
    const fides_ctx *c_;
    unsigned char *arena_;
    int lanes_;
    size_t cap_ = 0;
    std::vector<bool> failed_record_;
    std::vector<cudaStream_t> st_;
    std::vector<cudaEvent_t> ev0_, ev1_;
    std::vector<unsigned char *> dtab_, htab_;
};

// Stands in for the GPU: a group finishes ns_per_limb x (its ciphertext
// limbs) after it starts.
class SimExecutor : public Executor {
public:
    SimExecutor(int lanes, int64_t ns_per_limb) : done_at_(lanes, 0), dur_(lanes, 0), ns_per_limb_(ns_per_limb) {}
    int start(int lane, std::vector<Req *> &group, int *kernels) override
    {
        int64_t limbs = 0;
        for (const Req *q : group) limbs += q->nl;
        dur_[lane] = ns_per_limb_ * limbs;
        done_at_[lane] = now_ns() + dur_[lane];
        *kernels = 0;
        return FIDES_OK;
    }
    int query(int lane) override { return now_ns() >= done_at_[lane] ? 1 : 0; }
    double device_ms(int lane) override { return dur_[lane] * 1e-6; }

private:
    std::vector<int64_t> done_at_, dur_;
    int64_t ns_per_limb_;
};

struct Lane {
    bool busy = false;
    std::vector<Req *> group;
    int status = FIDES_OK;     // status of the launch
    bool injected = false;     // launch failed by fault injection: nothing was enqueued
    bool timed_out = false;    // the watchdog has already reported the group
    int64_t t_launch = 0;
    int64_t hidden_until = 0;  // injected stall: completion not seen before this time
};

}  // namespace

struct fides_server {
    const fides_ctx *ctx = nullptr;
    fides_server_config cfg;
    int N = 0, L = 0, K = 0, alpha = 0;
    int device = 0;
    unsigned char *arena_base = nullptr;   // device memory (null in simulation)
    Executor *exec = nullptr;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> pending;
    std::deque<fides_completion> done;
    std::unordered_map<uint64_t, Req *> live;
    std::unordered_map<int64_t, const fides_key *> rot_keys;   // normalised steps -> key
    const fides_key *relin = nullptr;
    Arena arena;
    std::vector<Lane> lanes;
    bool stop = false, paused = false;
    uint64_t next_id = 1;
    uint64_t stalled_id = 0;
    int inject_launch_errors = 0;
    int64_t inject_stall_us = 0;
    fides_server_stats st;
    std::thread th;

    int64_t norm_steps(int64_t s) const
    {
        const int64_t half = N / 2;
        return ((s % half) + half) % half;
    }
};

namespace {

void complete(fides_server *s, Req *q, int status, const Lane *lane, int lane_id, int64_t t_done)
{
    fides_completion c;
    memset(&c, 0, sizeof(c));
    c.id = q->id;
    c.tag = q->r.tag;
    c.type = q->r.type;
    c.status = status;
    c.out.n_limbs = q->out_limbs;
    c.out.scale = q->scale;
    if (status == FIDES_OK && s->arena_base) c.out.data = (u64 *)(s->arena_base + q->out_off);
    c.t_submit_ns = q->t_submit;
    c.t_admit_ns = q->t_admit;
    c.t_launch_ns = q->t_launch;
    c.t_done_ns = t_done;
    c.group_ops = lane ? (int)lane->group.size() : 0;
    c.lane = lane_id;
    s->done.push_back(c);
    if (status == FIDES_OK) ++s->st.completed;
    else if (status == FIDES_ERR_CANCELLED) ++s->st.cancelled;
    else if (status == FIDES_ERR_TIMEOUT) ++s->st.timed_out;
    else ++s->st.failed;
}

// A lane's group has left the GPU: free its scratch, deliver completions (or
// free the outputs of failed requests) and free the lane.  Holds s->mu.
void retire(fides_server *s, int li, int dev_status, int64_t t)
{
    Lane &ln = s->lanes[li];
    const int status = ln.status ? ln.status : (dev_status < 0 ? FIDES_ERR_CUDA : FIDES_OK);
    s->st.device_ms += s->exec->device_ms(li);
    for (Req *q : ln.group) {
        s->arena.release(q->scr_off, q->scr_bytes);
        if (ln.timed_out || status != FIDES_OK) {
            s->arena.release(q->out_off, q->out_bytes);
            if (!ln.timed_out) complete(s, q, status, &ln, li, t);
            s->live.erase(q->id);
            delete q;
        } else {
            q->state = R_DONE;
            ++s->st.held;
            complete(s, q, FIDES_OK, &ln, li, t);
        }
    }
    s->st.in_flight -= ln.group.size();
    ln.group.clear();
    ln.busy = false;
    ln.status = FIDES_OK;
    ln.injected = ln.timed_out = false;
    s->cv_done.notify_all();
}

// Takes, in arrival order, the requests whose memory fits; stops at the first
// that does not (no overtaking, so a large request is not starved).  Holds s->mu.
void admit(fides_server *s, std::vector<Req *> &group, int64_t t)
{
    while (!s->pending.empty() && (int)group.size() < s->cfg.max_batch) {
        Req *q = s->pending.front();
        const size_t o = s->arena.alloc(q->out_bytes);
        const size_t sc = o == kNone ? kNone : s->arena.alloc(q->scr_bytes);
        if (sc == kNone) {
            if (o != kNone) s->arena.release(o, q->out_bytes);
            if (s->stalled_id != q->id) ++s->st.admission_stalls;   // count each waiting request once
            s->stalled_id = q->id;
            break;
        }
        s->pending.pop_front();
        q->out_off = o;
        q->scr_off = sc;
        q->t_admit = t;
        q->state = R_RUNNING;
        group.push_back(q);
    }
}

void dispatcher(fides_server *s)
{
    if (!s->cfg.simulate) cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // 1. finished groups, and the watchdog
        bool any_busy = false;
        for (int li = 0; li < (int)s->lanes.size(); ++li) {
            Lane &ln = s->lanes[li];
            if (!ln.busy) continue;
            const int64_t t = now_ns();
            int q = ln.injected ? 1 : s->exec->query(li);
            if (q == 1 && t < ln.hidden_until) q = 0;
            if (q != 0) {
                retire(s, li, q, t);
                continue;
            }
            any_busy = true;
            if (s->cfg.timeout_us > 0 && !ln.timed_out && t - ln.t_launch > s->cfg.timeout_us * 1000) {
                // Report the group now; its memory is freed once the device is done with it.
                ln.timed_out = true;
                for (Req *r : ln.group) {
                    r->state = R_ABANDONED;
                    complete(s, r, FIDES_ERR_TIMEOUT, &ln, li, t);
                }
                s->cv_done.notify_all();
            }
        }
        if (s->stop && !any_busy) break;

        // 2. launch admitted requests on free lanes
        bool launched = false;
        if (!s->paused && !s->stop) {
            for (int li = 0; li < (int)s->lanes.size() && !s->pending.empty(); ++li) {
                Lane &ln = s->lanes[li];
                if (ln.busy) continue;
                const int64_t t = now_ns();
                admit(s, ln.group, t);
                if (ln.group.empty()) break;
                ln.busy = true;
                ln.t_launch = t;
                ln.hidden_until = 0;
                s->st.in_flight += ln.group.size();
                for (Req *r : ln.group) r->t_launch = t;
                ++s->st.groups;
                s->st.grouped_ops += ln.group.size();
                s->st.max_group = std::max<uint64_t>(s->st.max_group, ln.group.size());
                if (s->inject_stall_us) {
                    ln.hidden_until = t + s->inject_stall_us * 1000;
                    s->inject_stall_us = 0;
                }
                if (s->inject_launch_errors > 0) {
                    --s->inject_launch_errors;
                    ln.injected = true;
                    ln.status = FIDES_ERR_CUDA;
                } else {
                    // Enqueue without the lock: submitters and pollers go on meanwhile.
                    int kernels = 0;
                    lk.unlock();
                    const int rc = s->exec->start(li, ln.group, &kernels);
                    lk.lock();
                    ln.status = rc;
                    s->st.kernel_launches += kernels;
                }
                int busy = 0;
                for (const Lane &x : s->lanes) busy += x.busy;
                s->st.max_lanes_busy = std::max(s->st.max_lanes_busy, busy);
                any_busy = true;
                launched = true;
            }
        }
        s->st.pending = s->pending.size();
        s->st.arena_used = s->arena.used();
        s->st.arena_peak = s->arena.peak();

        // 3. wait: poll the device while groups run, otherwise sleep until a
        //    submission, a release, a resume or the stop wakes us
        if (any_busy) {
            if (!launched) {
                lk.unlock();
                std::this_thread::yield();
                lk.lock();
            }
        } else if (!s->stop) {
            s->cv_work.wait(lk);
        }
    }
    // stop: whatever is still queued is cancelled
    while (!s->pending.empty()) {
        Req *q = s->pending.front();
        s->pending.pop_front();
        complete(s, q, FIDES_ERR_CANCELLED, nullptr, -1, now_ns());
        s->live.erase(q->id);
        delete q;
    }
    s->cv_done.notify_all();
}

int check_config(const fides_ctx *c, const fides_server_config *cfg)
{
    if (!cfg) return fides_set_error(FIDES_ERR_ARG, "fides_server_create: config is NULL");
    if (cfg->n_lanes < 1 || cfg->n_lanes > FIDES_SERVER_MAX_LANES)
        return fides_set_error(FIDES_ERR_ARG, "fides_server_create: n_lanes=%d outside [1, %d]", cfg->n_lanes,
                               FIDES_SERVER_MAX_LANES);
    if (cfg->max_batch < 1 || cfg->max_batch > FIDES_SERVER_MAX_BATCH)
        return fides_set_error(FIDES_ERR_ARG, "fides_server_create: max_batch=%d outside [1, %d]", cfg->max_batch,
                               FIDES_SERVER_MAX_BATCH);
    if (cfg->max_pending < 1) return fides_set_error(FIDES_ERR_ARG, "fides_server_create: max_pending < 1");
    if (cfg->timeout_us < 0) return fides_set_error(FIDES_ERR_ARG, "fides_server_create: timeout_us < 0");
    if (!cfg->simulate && !c) return fides_set_error(FIDES_ERR_ARG, "fides_server_create: ctx is NULL");
    if (cfg->simulate && !c) {
        if (cfg->logN < 2 || cfg->logN > 17 || cfg->L < 1 || cfg->K < 1 || cfg->dnum < 1 || cfg->dnum > cfg->L)
            return fides_set_error(FIDES_ERR_ARG, "fides_server_create: simulation needs logN, L, K, dnum");
        if (cfg->sim_ns_per_limb < 0) return fides_set_error(FIDES_ERR_ARG, "fides_server_create: sim_ns_per_limb < 0");
    }
    return FIDES_OK;
}

}  // namespace

extern "C" int fides_server_create(fides_ctx *c, const fides_server_config *cfg, fides_server **out)
{
    if (!out) return fides_set_error(FIDES_ERR_ARG, "fides_server_create: out is NULL");
    *out = nullptr;
    if (int rc = check_config(c, cfg)) return rc;
    fides_server *s = new fides_server();
    s->ctx = c;
    s->cfg = *cfg;
    memset(&s->st, 0, sizeof(s->st));
    if (c) {
        s->N = c->N; s->L = c->L; s->K = c->K; s->alpha = c->alpha; s->device = c->device;
    } else {
        s->N = 1 << cfg->logN; s->L = cfg->L; s->K = cfg->K; s->alpha = (cfg->L + cfg->dnum - 1) / cfg->dnum;
    }
    s->arena.init(cfg->arena_bytes);
    s->st.arena_bytes = s->arena.size();
    s->lanes.resize(cfg->n_lanes);
    int rc = FIDES_OK;
    if (cfg->simulate) {
        s->exec = new SimExecutor(cfg->n_lanes, cfg->sim_ns_per_limb);
    } else {
        rc = fides_check_cuda(cudaSetDevice(c->device), "fides_server_create: device");
        if (!rc && s->arena.size())
            rc = fides_check_cuda(cudaMalloc((void **)&s->arena_base, s->arena.size()), "fides_server_create: arena");
        if (!rc) {
            CudaExecutor *e = new CudaExecutor(c, s->arena_base, cfg->n_lanes);
            s->exec = e;
            rc = e->init(cfg->max_batch);
        }
    }
    if (rc) {
        delete s->exec;
        if (s->arena_base) cudaFree(s->arena_base);
        delete s;
        return rc;
    }
    s->th = std::thread(dispatcher, s);
    *out = s;
    return FIDES_OK;
}

extern "C" void fides_server_destroy(fides_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    s->th.join();
    delete s->exec;   // synchronises its streams
    for (auto &kv : s->live) delete kv.second;
    if (s->arena_base) cudaFree(s->arena_base);
    delete s;
}

extern "C" int fides_server_set_relin_key(fides_server *s, const fides_key *key)
{
    if (!s || !key) return fides_set_error(FIDES_ERR_ARG, "fides_server_set_relin_key: NULL argument");
    if (s->ctx)
        if (int rc = fides_check_key(s->ctx, key, FIDES_GALOIS_RELIN, "fides_server_set_relin_key")) return rc;
    std::lock_guard<std::mutex> lk(s->mu);
    s->relin = key;
    return FIDES_OK;
}

extern "C" int fides_server_add_rotation_key(fides_server *s, int64_t steps, const fides_key *key)
{
    if (!s || !key) return fides_set_error(FIDES_ERR_ARG, "fides_server_add_rotation_key: NULL argument");
    if (s->ctx)
        if (int rc = fides_check_key(s->ctx, key, fides_galois_elt(s->ctx, steps), "fides_server_add_rotation_key"))
            return rc;
    std::lock_guard<std::mutex> lk(s->mu);
    s->rot_keys[s->norm_steps(steps)] = key;
    return FIDES_OK;
}

extern "C" int fides_server_submit(fides_server *s, const fides_request *r, uint64_t *id_out)
{
    if (!s || !r) return fides_set_error(FIDES_ERR_ARG, "fides_server_submit: NULL argument");
    const int nl = r->a.n_limbs;
    std::unique_lock<std::mutex> lk(s->mu);
    auto reject = [&](int code, const char *why) {
        ++s->st.rejected;
        return fides_set_error(code, "fides_server_submit: %s", why);
    };
    if (s->stop) return reject(FIDES_ERR_ARG, "server is stopping");
    if (!r->a.data) return reject(FIDES_ERR_ARG, "a.data is NULL");
    const fides_key *key = nullptr;
    int out_limbs = nl;
    switch (r->type) {
    case FIDES_OP_HMULT:
        if (nl < 1 || nl > s->L) return reject(FIDES_ERR_ARG, "bad level");
        if (!r->b.data || r->b.n_limbs != nl) return reject(FIDES_ERR_ARG, "HMULT needs b at the level of a");
        if (!s->relin) return reject(FIDES_ERR_KEY, "no relinearisation key");
        key = s->relin;
        break;
    case FIDES_OP_ROTATE: {
        if (nl < 1 || nl > s->L) return reject(FIDES_ERR_ARG, "bad level");
        auto it = s->rot_keys.find(s->norm_steps(r->steps));
        if (it == s->rot_keys.end()) return reject(FIDES_ERR_KEY, "no rotation key for these steps");
        key = it->second;
        break;
    }
    case FIDES_OP_RESCALE:
        if (nl < 2 || nl > s->L) return reject(FIDES_ERR_ARG, "bad level for RESCALE");
        out_limbs = nl - 1;
        break;
    default:
        return reject(FIDES_ERR_ARG, "unknown request type");
    }
    const size_t limb = (size_t)s->N * sizeof(u64);
    const size_t out_bytes = 2 * (size_t)out_limbs * limb;
    const size_t scr_bytes = op_scratch_words(s->N, s->K, s->alpha, r->type, nl) * sizeof(u64);
    if (round_up(out_bytes) + round_up(scr_bytes) > s->arena.size())
        return reject(FIDES_ERR_NOMEM, "request larger than the arena");
    if ((int)s->pending.size() >= s->cfg.max_pending) return reject(FIDES_ERR_BUSY, "queue full");
    Req *q = new Req();
    memset(q, 0, sizeof(*q));
    q->id = s->next_id++;
    q->r = *r;
    q->key = key;
    q->nl = nl;
    q->out_limbs = out_limbs;
    q->out_bytes = out_bytes;
    q->scr_bytes = scr_bytes;
    q->t_submit = now_ns();
    q->state = R_PENDING;
    s->pending.push_back(q);
    s->live[q->id] = q;
    ++s->st.submitted;
    s->st.pending = s->pending.size();
    if (id_out) *id_out = q->id;
    lk.unlock();
    s->cv_work.notify_one();
    return FIDES_OK;
}

extern "C" int fides_server_poll(fides_server *s, fides_completion *out, int max, int64_t timeout_us, int *n_out)
{
    if (!s || !n_out || max < 0 || (max > 0 && !out)) return fides_set_error(FIDES_ERR_ARG, "fides_server_poll: bad arguments");
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && timeout_us != 0) {
        auto ready = [&] { return !s->done.empty(); };
        if (timeout_us < 0) s->cv_done.wait(lk, ready);
        else s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
    }
    int n = 0;
    while (n < max && !s->done.empty()) {
        out[n++] = s->done.front();
        s->done.pop_front();
    }
    *n_out = n;
    return FIDES_OK;
}

extern "C" int fides_server_release(fides_server *s, uint64_t id)
{
    if (!s) return fides_set_error(FIDES_ERR_ARG, "fides_server_release: NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->live.find(id);
    if (it == s->live.end() || it->second->state != R_DONE)
        return fides_set_error(FIDES_ERR_ARG, "fides_server_release: request %llu holds no output",
                               (unsigned long long)id);
    Req *q = it->second;
    s->arena.release(q->out_off, q->out_bytes);
    --s->st.held;
    s->live.erase(it);
    delete q;
    lk.unlock();
    s->cv_work.notify_one();
    return FIDES_OK;
}

extern "C" int fides_server_cancel(fides_server *s, uint64_t id)
{
    if (!s) return fides_set_error(FIDES_ERR_ARG, "fides_server_cancel: NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->live.find(id);
    if (it == s->live.end() || it->second->state != R_PENDING)
        return fides_set_error(FIDES_ERR_BUSY, "fides_server_cancel: request %llu is not queued", (unsigned long long)id);
    Req *q = it->second;
    s->pending.erase(std::find(s->pending.begin(), s->pending.end(), q));
    complete(s, q, FIDES_ERR_CANCELLED, nullptr, -1, now_ns());
    s->live.erase(it);
    delete q;
    s->st.pending = s->pending.size();
    lk.unlock();
    s->cv_done.notify_all();
    return FIDES_OK;
}

extern "C" int fides_server_pause(fides_server *s, int paused)
{
    if (!s) return fides_set_error(FIDES_ERR_ARG, "fides_server_pause: NULL server");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->paused = paused != 0;
    }
    s->cv_work.notify_one();
    return FIDES_OK;
}

extern "C" int fides_server_inject(fides_server *s, int fault, int64_t arg)
{
    if (!s || arg < 0) return fides_set_error(FIDES_ERR_ARG, "fides_server_inject: bad arguments");
    std::lock_guard<std::mutex> lk(s->mu);
    switch (fault) {
    case FIDES_FAULT_LAUNCH_ERROR: s->inject_launch_errors = (int)arg; return FIDES_OK;
    case FIDES_FAULT_STALL: s->inject_stall_us = arg; return FIDES_OK;
    default: return fides_set_error(FIDES_ERR_ARG, "fides_server_inject: unknown fault %d", fault);
    }
}

extern "C" int fides_server_stats_read(fides_server *s, fides_server_stats *out)
{
    if (!s || !out) return fides_set_error(FIDES_ERR_ARG, "fides_server_stats_read: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    s->st.pending = s->pending.size();
    s->st.arena_used = s->arena.used();
    s->st.arena_peak = s->arena.peak();
    *out = s->st;
    return FIDES_OK;
}

extern "C" int64_t fides_now_ns(void) { return now_ns(); }
