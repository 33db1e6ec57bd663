// bn_server.cu — continuous-batching server for sampler-generation requests.
//
// A background thread owns every device object.  Requests are queued by bn_server_submit (any
// thread, non-blocking).  The loop, per chunk:
//   1. admits queued requests while a slot is free and the device-memory budget allows; each
//      admitted request gets a sampler initialised on a side stream (shifts, integrands,
//      permutation, counts), so admission overlaps the chunk already running on the GPU;
//   2. when the set of resident requests changed, rebuilds the fused batches over them: one for
//      the requests that run on the tensor-core schedule, one for the rest (one launch sequence
//      per batch for all its pairs, uneven tiles included).  Which batch a request joins is
//      the autotuner's choice for its signature (count width, N, T, radius, pair count and the
//      tile sides rounded up to powers of two), timed once on the first request of that
//      signature, on a scratch copy of its state, and cached for the server's lifetime;
//   3. runs up to sweeps_per_chunk passes for every resident request, each stopping at its own
//      remaining budget inside the launch;
//   4. retires the requests whose budget is spent (final Eq. 1, optimised shifts to host,
//      sampler freed) and records their submit / admit / done times.
// Requests are independent problems and every schedule gives identical results, so a request's
// outcome does not depend on what else is resident.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "bn_launch.h"
#include "bn_sampler.h"
#include "bn_trace.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Pending {
    int64_t id;
    bn_request req;
    double t_submit;
};

struct Resident {
    int64_t id;
    bn_request req;
    bn_sampler *s;
    int32_t left;
    double t_submit, t_admit;
    int64_t bytes;
    bool cancel;
    bool tensor;  // member of the tensor-core batch
};

// passes of each candidate schedule when a signature is tuned
constexpr int kTuneSweeps = 8;

int ceil_pow2(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

std::string signature(const bn_config &c)
{
    return std::to_string(c.n_points <= 64 ? 1 : 2) + "/" + std::to_string(c.n_points) + "/" +
           std::to_string(c.n_integrands) + "/" + std::to_string(c.radius) + "/" +
           std::to_string(c.n_pairs) + "/" + std::to_string(ceil_pow2(c.width)) + "x" +
           std::to_string(ceil_pow2(c.height));
}

}  // namespace

struct bn_server {
    bn_server_config cfg{};
    int device = 0;
    int64_t budget = 0;
    cudaStream_t run = nullptr, init = nullptr;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv, cv_done;
    bool stop = false;
    std::deque<Pending> pending;
    std::vector<Resident> active;
    std::vector<bn_result> done;
    std::map<int64_t, std::vector<float>> shifts;
    std::vector<int64_t> cancel_pending;
    int64_t next_id = 1;
    int64_t outstanding = 0;  // accepted by submit, result not yet posted
    int64_t mem_used = 0;
    bn_server_stats st{};
    Clock::time_point t0;
    bn_batch *batch[2] = {nullptr, nullptr};  // [0] other schedules, [1] tensor-core schedule
    std::map<std::string, bool> tuned;         // signature -> runs on the tensor-core schedule
    bool dirty = true;
    std::string thread_error;

    double now() const
    {
        return std::chrono::duration<double>(Clock::now() - t0).count();
    }
};

namespace {

void finish(bn_server *sv, const Resident &r, int status, const double *energy,
            std::vector<float> &&sh)
{
    bn_result res;
    memset(&res, 0, sizeof res);
    res.request_id = r.id;
    res.user_tag = r.req.user_tag;
    res.status = status;
    res.n_pairs = r.req.cfg.n_pairs;
    res.width = r.req.cfg.width;
    res.height = r.req.cfg.height;
    if (energy)
        for (int i = 0; i < r.req.cfg.n_pairs && i < 2; ++i) res.energy[i] = energy[i];
    res.t_submit = r.t_submit;
    res.t_admit = r.t_admit;
    res.t_done = sv->now();
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->done.push_back(res);
    --sv->outstanding;
    if (status == BN_OK) {
        sv->shifts[r.id] = std::move(sh);
        ++sv->st.completed;
    } else if (status == BN_ERR_BAD_STATE) {
        ++sv->st.cancelled;
    } else {
        ++sv->st.failed;
    }
    sv->cv_done.notify_all();
}

void loop(bn_server *sv)
{
    cudaSetDevice(sv->device);
    for (;;) {
        // ---- 1. admissions ------------------------------------------------------------------
        std::vector<Pending> admit;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv.wait(lk, [&] { return sv->stop || !sv->pending.empty() || !sv->active.empty(); });
            if (sv->stop) break;
            for (int64_t id : sv->cancel_pending)
                for (auto &r : sv->active)
                    if (r.id == id) r.cancel = true;
            sv->cancel_pending.clear();
            int64_t room = sv->budget - sv->mem_used;
            size_t slots = (size_t)sv->cfg.max_slots - sv->active.size();
            while (!sv->pending.empty() && admit.size() < slots) {
                const Pending &p = sv->pending.front();
                const int64_t bytes = bn::estimate_device_bytes(p.req.cfg);
                if (bytes > room) break;  // wait for memory to free up (oversize: rejected at submit)
                room -= bytes;
                admit.push_back(p);
                sv->pending.pop_front();
            }
            sv->st.pending = (int64_t)sv->pending.size();
        }
        for (const auto &p : admit) {
            bn::TraceRange trace_("bn.server.admit");
            Resident r{p.id, p.req, nullptr, p.req.n_sweeps, p.t_submit, 0.0,
                       bn::estimate_device_bytes(p.req.cfg), false, false};
            const int rc = bn_sampler_init(&p.req.cfg, sv->init, &r.s);
            r.t_admit = sv->now();
            if (rc != BN_OK) {
                finish(sv, r, rc, nullptr, {});
                continue;
            }
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->mem_used += r.bytes;
            sv->active.push_back(r);
            ++sv->st.admitted;
            sv->dirty = true;
        }
        // ---- retire cancelled ones ------------------------------------------------------------
        {
            std::vector<Resident> keep;
            for (auto &r : sv->active) {
                if (r.cancel) {
                    bn_sampler_destroy(r.s);
                    {
                        std::lock_guard<std::mutex> lk(sv->mu);
                        sv->mem_used -= r.bytes;
                    }
                    finish(sv, r, BN_ERR_BAD_STATE, nullptr, {});
                    sv->dirty = true;
                } else {
                    keep.push_back(r);
                }
            }
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->active.swap(keep);
            sv->st.active = (int64_t)sv->active.size();
            sv->st.memory_in_use = sv->mem_used;
        }
        if (sv->active.empty()) continue;
        // ---- 2. fused batches over the resident requests --------------------------------------
        if (sv->dirty) {
            bool ok = true;
            for (auto &r : sv->active) {
                if (!ok) break;
                const std::string key = signature(r.req.cfg);
                auto it = sv->tuned.find(key);
                bool tc = false;
                if (it != sv->tuned.end()) {
                    tc = it->second;
                } else {
                    tc = sv->cfg.tensor_policy == BN_SERVE_TENSOR_ALWAYS;
                    bool keep = true;
                    if (sv->cfg.tensor_policy == BN_SERVE_TENSOR_TUNED && bn::tensor_capable(r.s)) {
                        bn::TraceRange trace_("bn.server.tune");
                        bn_schedule best{};
                        // a trial that fails (no memory for its scratch copy, say) sends the
                        // request to the other batch and is not cached: a later request of the
                        // signature tries again
                        keep = bn::tune_schedule(r.s, kTuneSweeps, &best) == BN_OK;
                        if (!keep) cudaGetLastError();
                        tc = keep && best.kind == BN_SCHEDULE_TENSOR;
                        std::lock_guard<std::mutex> lk(sv->mu);
                        ++sv->st.tunes;
                    }
                    if (keep) sv->tuned.emplace(key, tc);
                }
                r.tensor = tc && bn::tensor_capable(r.s);
            }
            for (int g = 0; g < 2 && ok; ++g) {
                if (sv->batch[g]) bn_batch_destroy(sv->batch[g]);
                sv->batch[g] = nullptr;
                std::vector<bn_sampler *> members;
                for (auto &r : sv->active)
                    if (r.tensor == (g == 1)) members.push_back(r.s);
                if (members.empty()) continue;
                ok = bn::batch_create_as(members.data(), (int32_t)members.size(), sv->run,
                                         g ? BN_SCHEDULE_TENSOR : BN_SCHEDULE_AUTO,
                                         &sv->batch[g]) == BN_OK;
            }
            if (!ok) {
                std::lock_guard<std::mutex> lk(sv->mu);
                sv->thread_error = bn_last_error();
                break;
            }
            sv->dirty = false;
        }
        // ---- 3. one chunk of passes -------------------------------------------------------------
        std::vector<int32_t> n(sv->active.size());
        std::vector<int32_t> ng[2];
        int64_t props = 0;
        for (size_t i = 0; i < sv->active.size(); ++i) {
            n[i] = std::min(sv->active[i].left, sv->cfg.sweeps_per_chunk);
            ng[sv->active[i].tensor ? 1 : 0].push_back(n[i]);  // member order of the batches
            bn_info info;
            bn_get_info(sv->active[i].s, &info);
            props += (int64_t)n[i] * info.couples * sv->active[i].req.cfg.n_pairs;
        }
        bn::TraceRange trace_chunk("bn.server.chunk");
        bool run_ok = true;
        for (int g = 1; g >= 0 && run_ok; --g)
            if (!ng[g].empty())
                run_ok = bn_batch_optimize_each(sv->batch[g], ng[g].data(), nullptr) == BN_OK;
        if (!run_ok || cudaStreamSynchronize(sv->run) != cudaSuccess) {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->thread_error = bn_last_error();
            break;
        }
        // ---- 4. retire the finished -------------------------------------------------------------
        std::vector<Resident> keep;
        for (size_t i = 0; i < sv->active.size(); ++i) {
            Resident r = sv->active[i];
            r.left -= n[i];
            if (r.left > 0) {
                keep.push_back(r);
                continue;
            }
            double e[2] = {0.0, 0.0};
            const size_t nf = (size_t)r.req.cfg.n_pairs * r.req.cfg.width * r.req.cfg.height * 2;
            std::vector<float> sh(nf);
            int rc = bn_evaluate_energy(r.s, e);
            if (rc == BN_OK) rc = bn_fetch_shifts(r.s, sh.data(), nf, 0);
            bn_sampler_destroy(r.s);
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                sv->mem_used -= r.bytes;
            }
            finish(sv, r, rc, e, std::move(sh));
            sv->dirty = true;
        }
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->active.swap(keep);
        ++sv->st.chunks;
        if (!ng[1].empty()) ++sv->st.tensor_chunks;
        sv->st.proposals += props;
        sv->st.active = (int64_t)sv->active.size();
        sv->st.memory_in_use = sv->mem_used;
    }
    // shutdown: free whatever is still resident
    for (auto &b : sv->batch) {
        if (b) bn_batch_destroy(b);
        b = nullptr;
    }
    for (auto &r : sv->active) bn_sampler_destroy(r.s);
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->active.clear();
    sv->mem_used = 0;
    sv->cv_done.notify_all();
}

int sfail(int code, const std::string &msg)
{
    bn::set_last_error(msg.c_str());
    return code;
}

}  // namespace

extern "C" {

int bn_server_create(const bn_server_config *cfg, bn_server **out)
{
    if (!cfg || !out) return sfail(BN_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (cfg->max_slots < 1 || cfg->max_slots > 4096)
        return sfail(BN_ERR_INVALID_ARG, "max_slots must be in [1, 4096]");
    if (cfg->sweeps_per_chunk < 1 || cfg->sweeps_per_chunk > 500)
        return sfail(BN_ERR_INVALID_ARG, "sweeps_per_chunk must be in [1, 500]");
    if (cfg->memory_budget_bytes < 0) return sfail(BN_ERR_INVALID_ARG, "negative memory budget");
    if (cfg->tensor_policy < BN_SERVE_TENSOR_TUNED || cfg->tensor_policy > BN_SERVE_TENSOR_NEVER)
        return sfail(BN_ERR_INVALID_ARG, "tensor_policy must be a BN_SERVE_TENSOR_* value");
    auto *sv = new bn_server();
    sv->cfg = *cfg;
    sv->device = cfg->device;
    cudaError_t e = cudaSetDevice(sv->device);
    size_t free_b = 0, total_b = 0;
    if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->run, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->init, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        if (sv->run) cudaStreamDestroy(sv->run);
        if (sv->init) cudaStreamDestroy(sv->init);
        delete sv;
        return sfail(BN_ERR_CUDA, std::string("server set-up: ") + cudaGetErrorString(e));
    }
    sv->budget = cfg->memory_budget_bytes ? cfg->memory_budget_bytes : (int64_t)(0.8 * free_b);
    sv->st.memory_budget = sv->budget;
    sv->t0 = Clock::now();
    sv->th = std::thread(loop, sv);
    *out = sv;
    return BN_OK;
}

int bn_server_submit(bn_server *sv, const bn_request *req, int64_t *request_id)
{
    if (!sv || !req) return sfail(BN_ERR_INVALID_ARG, "null argument");
    if (req->n_sweeps < 1) return sfail(BN_ERR_INVALID_ARG, "n_sweeps must be >= 1");
    const int64_t bytes = bn::estimate_device_bytes(req->cfg);
    if (bytes < 0) return sfail(BN_ERR_INVALID_ARG, "invalid request configuration");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (!sv->thread_error.empty())
        return sfail(BN_ERR_BAD_STATE, "server stopped: " + sv->thread_error);
    ++sv->st.submitted;
    if (bytes > sv->budget) {
        ++sv->st.rejected;
        return sfail(BN_ERR_BUSY, "request needs " + std::to_string(bytes) +
                                      " device bytes, more than the server's budget");
    }
    Pending p{sv->next_id++, *req, sv->now()};
    p.req.cfg.schedule = BN_SCHEDULE_AUTO;  // the fused batch picks the schedule
    if (request_id) *request_id = p.id;
    sv->pending.push_back(p);
    ++sv->outstanding;
    sv->st.pending = (int64_t)sv->pending.size();
    sv->cv.notify_all();
    return BN_OK;
}

int bn_server_cancel(bn_server *sv, int64_t request_id)
{
    if (!sv) return sfail(BN_ERR_INVALID_ARG, "null server");
    std::unique_lock<std::mutex> lk(sv->mu);
    for (auto it = sv->pending.begin(); it != sv->pending.end(); ++it)
        if (it->id == request_id) {
            Resident r{it->id, it->req, nullptr, 0, it->t_submit, 0.0, 0, true};
            sv->pending.erase(it);
            lk.unlock();
            finish(sv, r, BN_ERR_BAD_STATE, nullptr, {});
            return BN_OK;
        }
    for (auto &r : sv->active)
        if (r.id == request_id) {
            sv->cancel_pending.push_back(request_id);
            sv->cv.notify_all();
            return BN_OK;
        }
    return sfail(BN_ERR_INVALID_ARG, "no such pending or resident request");
}

int bn_server_poll(bn_server *sv, bn_result *out, int32_t cap, int32_t *n_out)
{
    if (!sv || !n_out || (cap > 0 && !out)) return sfail(BN_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    const int32_t n = std::min<int32_t>(cap, (int32_t)sv->done.size());
    for (int32_t i = 0; i < n; ++i) out[i] = sv->done[i];
    sv->done.erase(sv->done.begin(), sv->done.begin() + n);
    *n_out = n;
    if (!sv->thread_error.empty())
        return sfail(BN_ERR_BAD_STATE, "server stopped: " + sv->thread_error);
    return BN_OK;
}

int bn_server_take_shifts(bn_server *sv, int64_t request_id, float *out, size_t n_floats)
{
    if (!sv || !out) return sfail(BN_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->shifts.find(request_id);
    if (it == sv->shifts.end()) return sfail(BN_ERR_INVALID_ARG, "no shifts held for this request");
    if (n_floats < it->second.size()) return sfail(BN_ERR_INVALID_ARG, "output buffer too small");
    memcpy(out, it->second.data(), sizeof(float) * it->second.size());
    sv->shifts.erase(it);
    return BN_OK;
}

int bn_server_get_stats(bn_server *sv, bn_server_stats *out)
{
    if (!sv || !out) return sfail(BN_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    *out = sv->st;
    out->pending = (int64_t)sv->pending.size();
    out->active = (int64_t)sv->active.size();
    out->memory_in_use = sv->mem_used;
    return BN_OK;
}

int bn_server_drain(bn_server *sv, double timeout_s)
{
    if (!sv) return sfail(BN_ERR_INVALID_ARG, "null server");
    std::unique_lock<std::mutex> lk(sv->mu);
    const bool ok = sv->cv_done.wait_for(
        lk, std::chrono::duration<double>(timeout_s),
        [&] { return sv->outstanding == 0 || !sv->thread_error.empty(); });
    if (!sv->thread_error.empty())
        return sfail(BN_ERR_BAD_STATE, "server stopped: " + sv->thread_error);
    if (!ok) return sfail(BN_ERR_BUSY, "requests still pending or resident at the timeout");
    return BN_OK;
}

void bn_server_destroy(bn_server *sv)
{
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->cv.notify_all();
    }
    if (sv->th.joinable()) sv->th.join();
    cudaSetDevice(sv->device);
    cudaStreamDestroy(sv->run);
    cudaStreamDestroy(sv->init);
    delete sv;
}

}  // extern "C"
