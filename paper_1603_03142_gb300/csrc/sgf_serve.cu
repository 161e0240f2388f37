// sgf_serve.cu -- the request loop of include/sgf.h (sgf_server_*).
//
// Continuous admission of force solves: requests wait in arrival order; every
// sgf_server_progress call first collects finished requests (a CUDA event per
// slot), then admits waiting requests while a slot is free and the memory they
// need fits the budget.  A slot = one CUDA stream + one plan (own workspace) +
// device copies of one request's sigma and forces; its request runs as
//   H2D sigma -> sgf_solve -> D2H Fx, Fy -> event
// on the slot's stream, so admitted requests overlap on the device.  Slots are
// kept after their request finishes and reused by the next request of the same
// shape; a new slot of a resident shape shares its spectra (sgf_plan_share_ex:
// FP32 and BF16X slots of one shape hold the same FP32 spectra).
// Memory pressure destroys the least recently used idle slots first.
//
// This file is a client of the plan API; it adds no kernels.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <vector>

#include "sgf_host.h"

using namespace sgf;

namespace {

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Pending {
    sgf_request r;
    std::string key;   // slot key: spectra key + precision
    std::string skey;  // spectra key
    size_t ws = 0, spectra = 0, build = 0, io = 0;  // bytes (sgf_plan_estimate; io = 3 L n^2 elements)
    size_t stream_budget = 0;  // SGF_SERVER_STREAM: the spectra budget of this shape's plans, else 0
    double t_submit = 0;
};

struct Slot {
    std::string key, skey;
    sgf_plan *plan = nullptr;
    void *d_io = nullptr;
    size_t ws = 0, io = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    bool built = false;  // the running request built this shape's spectra
    Pending req;
    double t_admit = 0, t_sim_done = 0;
    uint64_t last_use = 0;
};

struct Shape {
    size_t spectra = 0;
    int slots = 0;
};

// Spectra key of a request: FP32 and BF16X plans hold the same FP32 spectra.
std::string spectra_key(const sgf_request &r)
{
    std::string k;
    char buf[64];
    snprintf(buf, sizeof buf, "%d/%d/%s/%u", r.desc.n, r.desc.levels, r.precision == SGF_FP64 ? "f64" : "f32",
             r.plan_flags);
    k = buf;
    for (int l = 1; l < r.desc.levels; ++l) {
        snprintf(buf, sizeof buf, ":%d,%d", r.desc.off[l][0], r.desc.off[l][1]);
        k += buf;
    }
    return k;
}

}  // namespace

struct sgf_server {
    sgf_server_config cfg{};
    bool sim = false;
    int device = 0;
    std::chrono::steady_clock::time_point t0;
    std::deque<Pending> queue;
    std::vector<Slot *> slots;  // index = slot id; destroyed slots leave nullptr
    std::map<std::string, Shape> shapes;
    std::map<std::string, sgf_schedule> tuned;  // autotuned schedule per slot key
    std::deque<sgf_completion> out;
    size_t used = 0;
    uint64_t tick = 0;
    sgf_server_stats st{};

    double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
    int inflight() const
    {
        int n = 0;
        for (auto *s : slots)
            n += s && s->busy ? 1 : 0;
        return n;
    }
    void account(long long delta)
    {
        used = (size_t)((long long)used + delta);
        st.bytes_peak = std::max(st.bytes_peak, used);
    }
};

namespace {

struct DevGuard {
    int prev = -1;
    explicit DevGuard(const sgf_server *s)
    {
        if (s->sim)
            return;
        if (cudaGetDevice(&prev) == cudaSuccess && prev != s->device)
            cudaSetDevice(s->device);
        else
            prev = -1;
    }
    ~DevGuard()
    {
        if (prev >= 0)
            cudaSetDevice(prev);
    }
};

void slot_free(sgf_server *sv, Slot *s)
{
    if (!sv->sim) {
        if (s->stream)
            cudaStreamSynchronize(s->stream);
        if (s->plan)
            sgf_plan_destroy(s->plan);
        cudaFree(s->d_io);
        if (s->done)
            cudaEventDestroy(s->done);
        if (s->stream)
            cudaStreamDestroy(s->stream);
    }
    sv->account(-(long long)(s->ws + s->io));
    auto it = sv->shapes.find(s->skey);
    if (it != sv->shapes.end() && --it->second.slots == 0) {
        sv->account(-(long long)it->second.spectra);
        sv->shapes.erase(it);
    }
    delete s;
}

// Destroy the least recently used idle slot; false if every slot is busy.
bool evict_one(sgf_server *sv)
{
    int best = -1;
    for (int i = 0; i < (int)sv->slots.size(); ++i) {
        Slot *s = sv->slots[i];
        if (s && !s->busy && (best < 0 || s->last_use < sv->slots[best]->last_use))
            best = i;
    }
    if (best < 0)
        return false;
    slot_free(sv, sv->slots[best]);
    sv->slots[best] = nullptr;
    sv->st.slots_evicted++;
    return true;
}

void complete(sgf_server *sv, int idx, sgf_status status)
{
    Slot *s = sv->slots[idx];
    sgf_completion c{};
    c.id = s->req.r.id;
    c.status = status;
    c.slot = idx;
    c.built_shape = s->built ? 1 : 0;
    c.t_submit = s->req.t_submit;
    c.t_admit = s->t_admit;
    c.t_done = sv->now();
    sv->out.push_back(c);
    s->busy = false;
    s->built = false;
    sv->st.completed++;
}

// A new slot for the shape of p (plan, buffers, stream); bytes already checked.
sgf_status slot_create(sgf_server *sv, const Pending &p, Slot **out)
{
    Slot *s = new Slot();
    s->key = p.key;
    s->skey = p.skey;
    s->ws = p.ws;
    s->io = p.io;
    auto it = sv->shapes.find(p.skey);
    const bool resident = it != sv->shapes.end();
    sgf_status rc = SGF_OK;
    if (!sv->sim) {
        cudaError_t e;
        if ((e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)) != cudaSuccess)
            rc = cuda_fail(e, "cudaStreamCreate(slot)");
        if (rc == SGF_OK && resident) {
            const sgf_plan *tmpl = nullptr;
            for (auto *o : sv->slots)
                if (o && o->skey == p.skey) {
                    tmpl = o->plan;
                    break;
                }
            rc = tmpl ? sgf_plan_share_ex(tmpl, p.r.precision, &s->plan)
                      : fail(SGF_EINVAL, "resident shape without a slot");
        } else if (rc == SGF_OK) {
            rc = p.stream_budget ? sgf_plan_create(&p.r.desc, p.r.precision, p.stream_budget, &s->plan)
                                 : sgf_plan_create_ex(&p.r.desc, p.r.precision, p.r.plan_flags, &s->plan);
        }
        // the kernel schedule of this slot key: tuned once per server (on the slot's own
        // stream, while the other slots keep running), then reused
        if (rc == SGF_OK && !(sv->cfg.flags & SGF_SERVER_NO_AUTOTUNE)) {
            auto tt = sv->tuned.find(p.key);
            if (tt != sv->tuned.end()) {
                rc = sgf_plan_schedule_set(s->plan, &tt->second);
            } else {
                sgf_schedule sc{};
                rc = sgf_plan_autotune(s->plan, 2, s->stream, &sc, nullptr);
                if (rc == SGF_OK)
                    sv->tuned[p.key] = sc;
            }
        }
        if (rc == SGF_OK && (e = cudaMalloc(&s->d_io, p.io)) != cudaSuccess)
            rc = cuda_fail(e, "cudaMalloc(request buffers)");
        if (rc == SGF_OK && (e = cudaEventCreateWithFlags(&s->done, cudaEventDisableTiming)) != cudaSuccess)
            rc = cuda_fail(e, "cudaEventCreate(slot)");
        if (rc != SGF_OK) {
            std::string msg = sgf_last_error();
            if (s->plan)
                sgf_plan_destroy(s->plan);
            cudaFree(s->d_io);
            if (s->stream)
                cudaStreamDestroy(s->stream);
            delete s;
            fail(rc, "%s", msg.c_str());
            return rc;
        }
    }
    if (resident) {
        it->second.slots++;
    } else {
        Shape sh;
        sh.spectra = p.spectra;
        sh.slots = 1;
        sv->shapes[p.skey] = sh;
        sv->account((long long)p.spectra);
        sv->st.shapes_built++;
        s->built = true;
    }
    sv->account((long long)(p.ws + p.io));
    *out = s;
    return SGF_OK;
}

// Issue p's copies and solve on slot s.
sgf_status slot_launch(sgf_server *sv, Slot *s, const Pending &p)
{
    s->req = p;
    s->busy = true;
    s->t_admit = sv->now();
    s->last_use = ++sv->tick;
    const int L = p.r.desc.levels, n = p.r.desc.n;
    if (sv->sim) {
        const double bytes = (double)(p.ws + p.io + p.spectra);
        s->t_sim_done = s->t_admit + bytes / (sv->cfg.simulate_gbs * 1e9);
        return SGF_OK;
    }
    const size_t lvl = (size_t)n * n * (p.r.precision == SGF_FP64 ? 8 : 4);
    const size_t lal = align256(lvl);
    auto base = static_cast<unsigned char *>(s->d_io);
    const void *ds[SGF_MAX_LEVELS];
    void *dx[SGF_MAX_LEVELS], *dy[SGF_MAX_LEVELS];
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < L && e == cudaSuccess; ++l) {
        ds[l] = base + (size_t)l * lal;
        dx[l] = base + (size_t)(L + l) * lal;
        dy[l] = base + (size_t)(2 * L + l) * lal;
        e = cudaMemcpyAsync(const_cast<void *>(ds[l]), p.r.sigma[l], lvl, cudaMemcpyHostToDevice, s->stream);
    }
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync(request sigma)");
    sgf_status rc = sgf_solve(s->plan, ds, dx, dy, s->stream);
    if (rc != SGF_OK)
        return rc;
    for (int l = 0; l < L && e == cudaSuccess; ++l) {
        e = cudaMemcpyAsync(p.r.fx[l], dx[l], lvl, cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p.r.fy[l], dy[l], lvl, cudaMemcpyDeviceToHost, s->stream);
    }
    if (e == cudaSuccess)
        e = cudaEventRecord(s->done, s->stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "request copies");
    return SGF_OK;
}

}  // namespace

extern "C" {

sgf_status sgf_server_create(const sgf_server_config *config, sgf_server **out)
{
    if (!config || !out)
        return fail(SGF_EINVAL, "NULL argument");
    *out = nullptr;
    if (config->max_inflight < 1)
        return fail(SGF_EINVAL, "max_inflight = %d must be >= 1", config->max_inflight);
    if (config->flags & ~(SGF_SERVER_SIMULATE | SGF_SERVER_NO_AUTOTUNE | SGF_SERVER_STREAM))
        return fail(SGF_EINVAL, "unknown server flags 0x%x", config->flags);
    const bool sim = (config->flags & SGF_SERVER_SIMULATE) != 0;
    if (sim && !(config->simulate_gbs > 0.0))
        return fail(SGF_EINVAL, "SGF_SERVER_SIMULATE needs simulate_gbs > 0");
    if (sim && config->hbm_budget == 0)
        return fail(SGF_EINVAL, "SGF_SERVER_SIMULATE needs an explicit hbm_budget");
    sgf_server *sv = new sgf_server();
    sv->cfg = *config;
    sv->sim = sim;
    sv->t0 = std::chrono::steady_clock::now();
    if (!sim) {
        cudaError_t e = cudaGetDevice(&sv->device);
        size_t fr = 0, tot = 0;
        if (e == cudaSuccess && sv->cfg.hbm_budget == 0 && (e = cudaMemGetInfo(&fr, &tot)) == cudaSuccess)
            sv->cfg.hbm_budget = fr / 10 * 9;
        if (e != cudaSuccess) {
            delete sv;
            return cuda_fail(e, "server device");
        }
    }
    sv->st.hbm_budget = sv->cfg.hbm_budget;
    *out = sv;
    return SGF_OK;
}

double sgf_server_clock(const sgf_server *server) { return server ? server->now() : 0.0; }

sgf_status sgf_server_submit(sgf_server *sv, const sgf_request *r)
{
    if (!sv || !r)
        return fail(SGF_EINVAL, "NULL argument");
    Pending p;
    p.r = *r;
    sgf_status rc = sgf_plan_estimate(&r->desc, r->precision, r->plan_flags, &p.ws, &p.spectra, &p.build);
    if (rc != SGF_OK)
        return rc;
    if (r->plan_flags & SGF_PLAN_POTENTIAL)
        return fail(SGF_EUNSUPPORTED, "request %llu: the request loop solves forces, not SGF_PLAN_POTENTIAL",
                    (unsigned long long)r->id);
    const int L = r->desc.levels;
    for (int l = 0; l < L; ++l)
        if (!r->sigma[l] || !r->fx[l] || !r->fy[l])
            return fail(SGF_EINVAL, "request %llu: level %d has a NULL buffer", (unsigned long long)r->id, l);
    const size_t lvl = (size_t)r->desc.n * r->desc.n * (r->precision == SGF_FP64 ? 8 : 4);
    p.io = 3 * (size_t)L * align256(lvl);
    p.skey = spectra_key(*r);
    p.key = p.skey + "/p" + std::to_string((int)r->precision);
    if (sv->cfg.max_shape_bytes && p.spectra + p.build > sv->cfg.max_shape_bytes &&
        (sv->cfg.flags & SGF_SERVER_STREAM) && r->plan_flags == 0 && p.build < sv->cfg.max_shape_bytes) {
        // served by plans over a spectra budget: resident sets and a window within the budget,
        // the generator's workspace kept by every slot's plan
        const size_t esz = r->precision == SGF_FP64 ? 8 : 4;
        const size_t one_set = 6 * (size_t)(r->desc.n + 1) * 2 * r->desc.n * 2 * esz;
        const size_t budget = sv->cfg.max_shape_bytes - p.build;
        if (budget >= one_set) {
            p.stream_budget = budget;
            p.ws += p.build + budget;  // generator workspace and (at most) the window, per slot
            p.spectra = budget;        // the resident sets, at most the budget
        }
    }
    const size_t worst = p.ws + p.io + p.spectra + p.build;
    if (sv->cfg.max_shape_bytes && p.spectra + p.build > sv->cfg.max_shape_bytes) {
        sv->st.rejected++;
        return fail(SGF_ENOMEM, "request %llu: its shape needs %zu bytes of spectra and generator memory, above "
                    "max_shape_bytes %zu", (unsigned long long)r->id, p.spectra + p.build, sv->cfg.max_shape_bytes);
    }
    if (worst > sv->cfg.hbm_budget) {
        sv->st.rejected++;
        return fail(SGF_ENOMEM, "request %llu needs %zu bytes (spectra %zu, generator %zu), above the budget %zu",
                    (unsigned long long)r->id, worst, p.spectra, p.build, sv->cfg.hbm_budget);
    }
    p.t_submit = sv->now();
    sv->queue.push_back(p);
    sv->st.submitted++;
    return SGF_OK;
}

sgf_status sgf_server_progress(sgf_server *sv, sgf_completion *out, int32_t capacity, int32_t *count)
{
    if (!sv || !count || (capacity > 0 && !out) || capacity < 0)
        return fail(SGF_EINVAL, "bad arguments");
    *count = 0;
    DevGuard g(sv);
    // 1. collect finished requests
    for (int i = 0; i < (int)sv->slots.size(); ++i) {
        Slot *s = sv->slots[i];
        if (!s || !s->busy)
            continue;
        if (sv->sim) {
            if (sv->now() >= s->t_sim_done)
                complete(sv, i, SGF_OK);
            continue;
        }
        const cudaError_t e = cudaEventQuery(s->done);
        if (e == cudaErrorNotReady)
            continue;
        sgf_status rs = e == cudaSuccess ? sgf_plan_check(s->plan) : cuda_fail(e, "request on the device");
        complete(sv, i, rs);
    }
    // 2. admit in arrival order while a slot and memory allow
    sgf_status rc = SGF_OK;
    while (!sv->queue.empty() && sv->inflight() < sv->cfg.max_inflight) {
        const Pending &p = sv->queue.front();
        int idx = -1;
        for (int i = 0; i < (int)sv->slots.size(); ++i) {
            Slot *s = sv->slots[i];
            if (s && !s->busy && s->key == p.key && (idx < 0 || s->last_use > sv->slots[idx]->last_use))
                idx = i;
        }
        if (idx < 0) {
            const bool resident = sv->shapes.count(p.skey) != 0;
            const size_t need = p.ws + p.io + (resident ? 0 : p.spectra + p.build);
            while (sv->used + need > sv->cfg.hbm_budget && evict_one(sv)) {
            }
            if (sv->used + need > sv->cfg.hbm_budget)
                break;  // wait for running requests to finish
            Slot *s = nullptr;
            if ((rc = slot_create(sv, p, &s)) != SGF_OK)
                break;
            for (idx = 0; idx < (int)sv->slots.size() && sv->slots[idx]; ++idx) {
            }
            if (idx == (int)sv->slots.size())
                sv->slots.push_back(s);
            else
                sv->slots[idx] = s;
        }
        Slot *s = sv->slots[idx];
        Pending p2 = p;
        sv->queue.pop_front();
        sv->st.admitted++;
        const sgf_status ls = slot_launch(sv, s, p2);
        if (ls != SGF_OK) {
            if (!sv->sim && s->stream)
                cudaStreamSynchronize(s->stream);  // nothing of this request may still run
            complete(sv, idx, ls);
        }
        sv->st.inflight_peak = std::max(sv->st.inflight_peak, sv->inflight());
    }
    // 3. hand back completions, oldest first
    while (*count < capacity && !sv->out.empty()) {
        out[(*count)++] = sv->out.front();
        sv->out.pop_front();
    }
    return rc;
}

sgf_status sgf_server_stats_get(const sgf_server *sv, sgf_server_stats *st)
{
    if (!sv || !st)
        return fail(SGF_EINVAL, "NULL argument");
    *st = sv->st;
    st->queued = (int32_t)sv->queue.size();
    st->inflight = sv->inflight();
    int n = 0;
    for (auto *s : sv->slots)
        n += s ? 1 : 0;
    st->slots = n;
    st->shapes_resident = (int32_t)sv->shapes.size();
    st->bytes_used = sv->used;
    st->hbm_budget = sv->cfg.hbm_budget;
    return SGF_OK;
}

sgf_status sgf_server_destroy(sgf_server *sv)
{
    if (!sv)
        return SGF_OK;
    {
        DevGuard g(sv);
        for (auto *s : sv->slots)
            if (s)
                slot_free(sv, s);
    }
    delete sv;
    return SGF_OK;
}

}  // extern "C"
