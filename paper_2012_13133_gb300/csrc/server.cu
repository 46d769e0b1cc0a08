// Continuous-batching request server over the Kryging C ABI.
//
// A server owns `nslots` worker threads, each with its own CUDA stream and
// kry_ctx, so the kernels of requests in different slots run concurrently on
// the device.  Submitted requests wait in one queue; a free slot admits the
// first queued request whose estimated device footprint fits in what the
// memory budget has left (later, smaller requests may pass a large one that
// does not fit yet).  Inputs arrive in host memory and are copied into the
// slot's device buffers; results are copied back into the caller's host
// buffers.  Each slot keeps its device buffers between requests (they grow to
// the largest request it served), so the budget counts each slot's peak.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "kry_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    uint64_t ticket = 0;
    kry_request req{};
    int64_t est_bytes = 0;
    Clock::time_point t_submit;
    Clock::time_point t_start;
    Clock::time_point t_done;
    kry_status status = KRY_OK;
    std::string err;
    bool done = false;
    int slot = -1;
};

struct Slot {
    int index = 0;
    cudaStream_t stream = nullptr;
    kry_ctx* ctx = nullptr;
    DevBuf mask, y, X, cells, Xc, mean;
    int64_t reserved = 0;   // bytes this slot holds against the budget
};

int pow2ge(int64_t x) {
    int M = 1;
    while (M < x) M *= 2;
    return M;
}

}  // namespace

struct kry_server {
    int device = 0;
    int64_t budget = 0;
    int64_t in_use = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Job>> queue;
    std::map<uint64_t, std::shared_ptr<Job>> jobs;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::vector<std::unique_ptr<Slot>> slots;
    std::vector<std::thread> threads;
    std::string err;
};

namespace {

// Device bytes a request needs in a slot (embedding, FFT intermediates, Krylov
// vectors, inputs and outputs), with 25% headroom.
int64_t estimate_bytes(const kry_request& r, int64_t p) {
    const int64_t N = (int64_t)r.n1 * r.n2;
    const int64_t M1 = pow2ge(2 * (int64_t)r.n1), M2 = pow2ge(2 * (int64_t)r.n2);
    const int64_t MM = M1 * M2;
    const int nc = r.ncov + 1 + ((r.ncov + 1) & 1);
    const int64_t vecs = (r.kind == KRY_REQ_LOGLIK) ? std::max(r.opts.nprobe, nc) : nc;
    // bytes per vector element: FP64 requests, and KRY_AUTO ones that will run in
    // FP64 for want of a nugget (a KRY_AUTO request promoted for its
    // conditioning, kappa > 4e6, needs up to twice the vector memory counted
    // here: the budget is meant to stay well below the device's memory)
    const int64_t es = (r.opts.prec == KRY_F64 || (r.opts.prec == KRY_AUTO && !(r.cov.tau2 > 0.0))) ? 8 : 4;
    int64_t b = 0;
    b += 36 * MM;                                  // eigenvalues (FP64 + FP32) and eigen scratch
    b += (int64_t)r.n1 * M2 * 2 * es * ((vecs + 1) / 2);   // Krylov slab
    b += (int64_t)r.n1 * M2 * 16 * ((nc + 1) / 2);    // FP64 slab (true residuals)
    b += 4 * vecs * p * es + 4 * nc * p * 8;       // Lanczos / CG vectors, FP64 residual work
    b += 3 * (int64_t)nc * p * 8 + (N + p) * 8;    // [y, X], solutions, kriging grid
    if (r.opts.precond) b += 16 * MM + (int64_t)nc * p * 4;   // preconditioner eigenvalues, z vectors
    if (r.kind == KRY_REQ_LOGLIK && r.opts.reorth)   // stored Lanczos basis
        b += (int64_t)r.opts.nprobe * r.opts.nsteps * p * (es == 4 ? 2 : 8) + 3 * vecs * p * es;   // FP16 store in FP32
    b += N + p * 8 * (1 + r.ncov) + (N - p) * 8 * (2 + r.ncov);   // inputs and outputs
    return b + b / 4 + (64 << 20);
}

void run_job(kry_server* s, Slot& sl, Job& j) {
    const kry_request& r = j.req;
    kry_ctx* ctx = sl.ctx;
    const int64_t N = (int64_t)r.n1 * r.n2;
    auto check = [&](kry_status st) {
        if (st != KRY_OK && st != KRY_ENOCONV) throw KryError{st, kry_last_error(ctx)};
        return st;
    };
    KRY_CUDA(cudaSetDevice(s->device));
    sl.mask.ensure(N);
    KRY_CUDA(cudaMemcpyAsync(sl.mask.p, r.mask, N, cudaMemcpyHostToDevice, sl.stream));
    kry_grid g{r.n1, r.n2, 1.0 / r.n1, 1.0 / r.n2};
    int64_t p = 0;
    check(kry_set_mask(ctx, &g, sl.mask.as<uint8_t>(), &p));
    sl.y.ensure(p * sizeof(double));
    sl.X.ensure((size_t)p * r.ncov * sizeof(double));
    KRY_CUDA(cudaMemcpyAsync(sl.y.p, r.y, p * sizeof(double), cudaMemcpyHostToDevice, sl.stream));
    KRY_CUDA(cudaMemcpyAsync(sl.X.p, r.X, (size_t)p * r.ncov * sizeof(double), cudaMemcpyHostToDevice, sl.stream));
    kry_status st = KRY_OK;
    if (r.kind == KRY_REQ_LOGLIK) {
        double ll = 0, ld = 0, se = 0;
        std::vector<double> beta(r.ncov);
        st = check(kry_profile_loglik(ctx, sl.y.as<double>(), sl.X.as<double>(), r.ncov, &r.cov, 1, &r.opts, &ll,
                                      beta.data(), &ld, &se));
        if (r.loglik) *r.loglik = ll;
        if (r.logdet) *r.logdet = ld;
        if (r.beta) memcpy(r.beta, beta.data(), r.ncov * sizeof(double));
    } else {
        const int64_t nt = N - p;
        KRY_REQUIRE(nt == 0 || (r.target_cells && r.target_X && r.mean), KRY_EINVAL,
                    "kriging request needs target_cells, target_X and mean");
        sl.cells.ensure(std::max<int64_t>(nt, 1) * sizeof(int64_t));
        sl.Xc.ensure(std::max<int64_t>(nt, 1) * r.ncov * sizeof(double));
        sl.mean.ensure(std::max<int64_t>(nt, 1) * sizeof(double));
        if (nt > 0) {
            KRY_CUDA(cudaMemcpyAsync(sl.cells.p, r.target_cells, nt * sizeof(int64_t), cudaMemcpyHostToDevice,
                                     sl.stream));
            KRY_CUDA(cudaMemcpyAsync(sl.Xc.p, r.target_X, (size_t)nt * r.ncov * sizeof(double),
                                     cudaMemcpyHostToDevice, sl.stream));
        }
        std::vector<double> beta(r.ncov);
        st = check(kry_krige(ctx, &r.cov, &r.opts, sl.y.as<double>(), sl.X.as<double>(), r.ncov,
                             nt > 0 ? sl.cells.as<int64_t>() : nullptr, nt > 0 ? sl.Xc.as<double>() : nullptr, nt,
                             nullptr, nullptr, 0, nt > 0 ? sl.mean.as<double>() : nullptr, nullptr, nullptr,
                             beta.data()));
        if (nt > 0)
            KRY_CUDA(cudaMemcpyAsync(r.mean, sl.mean.p, nt * sizeof(double), cudaMemcpyDeviceToHost, sl.stream));
        if (r.beta) memcpy(r.beta, beta.data(), r.ncov * sizeof(double));
    }
    KRY_CUDA(cudaStreamSynchronize(sl.stream));
    j.status = st;
}

void worker(kry_server* s, Slot* sl) {
    cudaSetDevice(s->device);
    for (;;) {
        std::shared_ptr<Job> job;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            for (;;) {
                if (s->stop) return;
                // admit the first queued request that fits in the budget
                for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
                    const int64_t extra = std::max<int64_t>(0, (*it)->est_bytes - sl->reserved);
                    if (s->in_use + extra <= s->budget) {
                        job = *it;
                        s->queue.erase(it);
                        s->in_use += extra;
                        sl->reserved += extra;
                        break;
                    }
                }
                if (job) break;
                if (!s->queue.empty() && sl->reserved > 0) {
                    // nothing fits: give this idle slot's cached buffers back to the budget
                    s->in_use -= sl->reserved;
                    sl->reserved = 0;
                    lk.unlock();
                    kry::ctx_trim(sl->ctx);
                    sl->mask.release();
                    sl->y.release();
                    sl->X.release();
                    sl->cells.release();
                    sl->Xc.release();
                    sl->mean.release();
                    lk.lock();
                    continue;
                }
                s->cv_work.wait(lk);
            }
        }
        job->t_start = Clock::now();
        job->slot = sl->index;
        try {
            run_job(s, *sl, *job);
        } catch (const KryError& e) {
            job->status = e.st;
            job->err = e.msg;
        } catch (const std::exception& e) {
            job->status = KRY_ECUDA;
            job->err = e.what();
        }
        job->t_done = Clock::now();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            job->done = true;
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
}

}  // namespace

extern "C" {

kry_status kry_server_create(kry_server** out, int device, int32_t nslots, int64_t mem_budget_bytes) {
    if (!out) return KRY_EINVAL;
    *out = nullptr;
    if (nslots < 1 || nslots > 64 || mem_budget_bytes <= 0) return KRY_EINVAL;
    kry_server* s = new kry_server();
    s->device = device;
    s->budget = mem_budget_bytes;
    for (int i = 0; i < nslots; ++i) {
        auto sl = std::make_unique<Slot>();
        sl->index = i;
        if (cudaSetDevice(device) != cudaSuccess ||
            cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess) {
            kry_server_destroy(s);
            return KRY_ECUDA;
        }
        for (DevBuf* b : {&sl->mask, &sl->y, &sl->X, &sl->cells, &sl->Xc, &sl->mean}) b->stream = sl->stream;
        kry_status st = kry_create(&sl->ctx, device, sl->stream);
        if (st != KRY_OK) {
            cudaStreamDestroy(sl->stream);
            kry_server_destroy(s);
            return st;
        }
        s->slots.push_back(std::move(sl));
    }
    for (auto& sl : s->slots) s->threads.emplace_back(worker, s, sl.get());
    *out = s;
    return KRY_OK;
}

kry_status kry_server_submit(kry_server* s, const kry_request* req, uint64_t* ticket) {
    if (!s || !req || !ticket) return KRY_EINVAL;
    const kry_request& r = *req;
    if (r.n1 < 4 || r.n2 < 4 || r.n1 > KRY_MAX_N || r.n2 > KRY_MAX_N || !r.mask || !r.y || !r.X || r.ncov < 1 ||
        r.ncov > KRY_MAX_COV || (r.kind != KRY_REQ_LOGLIK && r.kind != KRY_REQ_KRIGE))
        return KRY_EINVAL;
    if (r.kind == KRY_REQ_LOGLIK && !r.loglik) return KRY_EINVAL;
    int64_t p = 0;
    const int64_t N = (int64_t)r.n1 * r.n2;
    for (int64_t i = 0; i < N; ++i) p += r.mask[i] != 0;
    if (p < 1) return KRY_EINVAL;
    auto job = std::make_shared<Job>();
    job->req = r;
    job->est_bytes = estimate_bytes(r, p);
    if (job->est_bytes > s->budget) return KRY_ENOMEM;
    job->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        job->ticket = s->next_ticket++;
        s->queue.push_back(job);
        s->jobs[job->ticket] = job;
    }
    *ticket = job->ticket;
    s->cv_work.notify_all();
    return KRY_OK;
}

kry_status kry_server_wait(kry_server* s, uint64_t ticket, double timeout_s, kry_status* req_status,
                           double* latency_ms, int32_t* slot, char* err_buf, int32_t err_len) {
    if (!s) return KRY_EINVAL;
    std::shared_ptr<Job> job;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->jobs.find(ticket);
        if (it == s->jobs.end()) return KRY_EINVAL;
        job = it->second;
        const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                              std::chrono::duration<double>(std::max(0.0, timeout_s)));
        if (!s->cv_done.wait_until(lk, until, [&] { return job->done; })) return KRY_ETIMEOUT;
        s->jobs.erase(ticket);
    }
    if (req_status) *req_status = job->status;
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(job->t_done - job->t_submit).count();
    if (slot) *slot = job->slot;
    if (err_buf && err_len > 0) {
        const size_t n = std::min<size_t>(job->err.size(), (size_t)err_len - 1);
        memcpy(err_buf, job->err.data(), n);
        err_buf[n] = 0;
    }
    return KRY_OK;
}

int64_t kry_server_queued(kry_server* s) {
    if (!s) return -1;
    std::lock_guard<std::mutex> lk(s->mu);
    return (int64_t)s->queue.size();
}

void kry_server_destroy(kry_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->threads) t.join();
    for (auto& sl : s->slots) {
        cudaSetDevice(s->device);
        if (sl->ctx) kry_destroy(sl->ctx);
        sl->mask.release();
        sl->y.release();
        sl->X.release();
        sl->cells.release();
        sl->Xc.release();
        sl->mean.release();
        if (sl->stream) cudaStreamDestroy(sl->stream);
    }
    delete s;
}

}  // extern "C"
