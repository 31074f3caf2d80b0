// Host core of the serving loop: admission against a memory budget, continuous batching on
// several lanes, completion and latency bookkeeping.  It holds no CUDA code: a lane's batch is
// run by an Executor (dm_serve.cu implements one on CUDA streams), so this file also compiles
// alone with a host C++17 compiler.
//
// Requests arrive one set at a time (indices, weights, k, seed).  A request is admitted when the
// bytes of every admitted, unfinished request plus its own stay within the budget; otherwise the
// caller is told to retry (kEAGAIN).  Each lane has a worker thread that, whenever it is free,
// takes the oldest pending requests (up to the lane's byte capacity and a request cap), groups
// them by (k, seed) in order of first appearance, and hands the batch to the executor.  Several
// lanes keep several batches in flight, so a new batch starts as soon as a lane frees up instead
// of waiting for the batch before it (continuous batching).
#pragma once
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

namespace dm {
namespace serve {

using Clock = std::chrono::steady_clock;

// Status values, equal to the library's dm_status codes.
enum : int { kOK = 0, kEINVAL = 1, kENOMEM = 2, kECUDA = 3, kETIMEOUT = 4, kEAGAIN = 7 };

struct Request {
    int64_t ticket = 0;
    int32_t k = 0;
    uint64_t seed = 0;
    int64_t nnz = 0;
    const uint32_t *indices = nullptr;
    const float *weights = nullptr;
    std::unique_ptr<unsigned char[]> own;  // copy of indices and weights, for callers whose arrays may go away
    uint64_t *out = nullptr;               // caller's host buffer of k keys (null: not delivered)
    size_t bytes = 0;                      // admission bytes (request_bytes)
    Clock::time_point t_arrival;           // latency is measured from here
    Clock::time_point t_admit;             // batching window is measured from here
    Clock::time_point t_done;
    int status = kOK;
    bool done = false;
};

// Requests of one batch that share (k, seed), in arrival order.
struct Group {
    int32_t k = 0;
    uint64_t seed = 0;
    int64_t nnz = 0;
    std::vector<Request *> reqs;
};

// Device bytes a request occupies in a lane: CSR offsets, indices, weights, k output keys and
// per-set scratch, rounded up.  A batch also pays kGroupOverhead per group (alignment padding
// and per-call counters).
inline size_t request_bytes(int64_t nnz, int32_t k) { return 32 + 8 * (size_t)nnz + 8 * (size_t)k; }
constexpr size_t kGroupOverhead = 4096;

struct Executor {
    virtual ~Executor() = default;
    // Runs one batch on `lane` to completion (called only by that lane's worker): stages the
    // inputs, computes every request's k keys, writes them to req->out when it is not null and
    // sets req->status for requests that failed alone.  A non-zero return fails the whole batch.
    virtual int run(int lane, std::vector<Group> &groups) = 0;
};

struct Config {
    int lanes = 4;
    size_t budget = (size_t)8 << 30;       // admission budget (bytes of admitted requests)
    size_t lane_bytes = (size_t)64 << 20;  // capacity of one batch
    int max_batch = 4096;                  // requests per batch
    int64_t max_wait_us = 0;               // batching window (0: take what is pending)
    bool per_request = false;              // one request per batch (the plain per-request form)
};

struct Stats {
    int64_t submitted = 0, completed = 0, failed = 0, rejected = 0, batches = 0, groups = 0;
    double mean_batch = 0, p50_us = 0, p99_us = 0, max_us = 0;
    int64_t admitted_bytes = 0;
};

class Core {
  public:
    Core(const Config &cfg, Executor *exec) : cfg_(cfg), exec_(exec) {
        if (cfg_.lanes < 1) cfg_.lanes = 1;
        if (cfg_.max_batch < 1) cfg_.max_batch = 1;
        lat_.reserve(1024);
        for (int l = 0; l < cfg_.lanes; ++l) workers_.emplace_back([this, l] { worker(l); });
    }

    // Finishes every admitted request, then stops the lanes.
    ~Core() { stop(); }

    void stop() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            if (stopping_) return;
            stopping_ = true;
        }
        work_cv_.notify_all();
        for (auto &t : workers_) t.join();
        workers_.clear();
    }

    const Config &config() const { return cfg_; }

    // Admits a request (the caller keeps it alive until done).  tracked: the core owns it and
    // releases it when poll/wait report it done.  Returns kOK, kEAGAIN (budget full now),
    // kENOMEM (larger than a lane: never runnable) or kEINVAL (stopping).
    int submit(Request *r, std::unique_ptr<Request> tracked = nullptr) {
        r->bytes = request_bytes(r->nnz, r->k);
        if (r->bytes + kGroupOverhead > cfg_.lane_bytes || r->bytes > cfg_.budget) return kENOMEM;
        {
            std::lock_guard<std::mutex> lk(mu_);
            if (stopping_) return kEINVAL;
            if (admitted_ + r->bytes > cfg_.budget) {
                ++stats_.rejected;
                return kEAGAIN;
            }
            admitted_ += r->bytes;
            r->t_admit = Clock::now();
            r->done = false;
            r->ticket = ++next_ticket_;
            pending_.push_back(r);
            ++stats_.submitted;
            if (tracked) tickets_.emplace(r->ticket, std::move(tracked));
        }
        work_cv_.notify_one();
        return kOK;
    }

    // Waits until `bytes` more would be admitted (or the timeout passes).
    bool wait_capacity(size_t bytes, std::chrono::microseconds timeout) {
        std::unique_lock<std::mutex> lk(mu_);
        return done_cv_.wait_for(lk, timeout, [&] { return stopping_ || admitted_ + bytes <= cfg_.budget; });
    }

    // Blocks until r is done.
    void wait_done(Request *r) {
        std::unique_lock<std::mutex> lk(mu_);
        done_cv_.wait(lk, [&] { return r->done; });
    }

    // Tracked requests.  poll: kOK and *status (-1 while pending); kEINVAL for an unknown ticket.
    int poll(int64_t ticket, int *status) {
        std::lock_guard<std::mutex> lk(mu_);
        auto it = tickets_.find(ticket);
        if (it == tickets_.end()) return kEINVAL;
        if (!it->second->done) {
            *status = -1;
            return kOK;
        }
        *status = it->second->status;
        tickets_.erase(it);
        return kOK;
    }

    int wait(int64_t ticket, int64_t timeout_us, int *status) {
        std::unique_lock<std::mutex> lk(mu_);
        auto it = tickets_.find(ticket);
        if (it == tickets_.end()) return kEINVAL;
        Request *r = it->second.get();
        auto ready = [&] { return r->done; };
        if (timeout_us < 0) done_cv_.wait(lk, ready);
        else if (!done_cv_.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) return kETIMEOUT;
        *status = r->status;
        tickets_.erase(ticket);
        return kOK;
    }

    // Fails the next n batches before they reach the executor, as a launch failure would
    // (host-side fault injection for tests of the failure path).
    void fail_next_batches(int n) { fail_next_.store(n); }

    Stats stats() {
        std::lock_guard<std::mutex> lk(mu_);
        Stats s = stats_;
        s.admitted_bytes = (int64_t)admitted_;
        s.mean_batch = s.batches ? (double)batched_requests_ / (double)s.batches : 0.0;
        if (!lat_.empty()) {
            std::vector<int64_t> v(lat_);
            auto pct = [&](double q) {
                size_t i = (size_t)(q * (double)(v.size() - 1) + 0.5);
                std::nth_element(v.begin(), v.begin() + i, v.end());
                return (double)v[i] / 1000.0;
            };
            s.p50_us = pct(0.50);
            s.p99_us = pct(0.99);
            s.max_us = (double)*std::max_element(v.begin(), v.end()) / 1000.0;
        }
        return s;
    }

    void reset_stats() {
        std::lock_guard<std::mutex> lk(mu_);
        stats_ = Stats{};
        batched_requests_ = 0;
        lat_.clear();
        lat_next_ = 0;
    }

  private:
    static constexpr size_t kLatencyRing = (size_t)1 << 22;   // latencies kept for percentiles

    void worker(int lane) {
        std::vector<Request *> batch;
        std::vector<Group> groups;
        std::vector<std::pair<int32_t, uint64_t>> keys;
        for (;;) {
            batch.clear();
            {
                std::unique_lock<std::mutex> lk(mu_);
                for (;;) {
                    if (pending_.empty()) {
                        if (stopping_) return;
                        work_cv_.wait(lk);
                        continue;
                    }
                    // batching window: let a young, small queue grow a little
                    if (cfg_.max_wait_us > 0 && !stopping_ && !cfg_.per_request &&
                        (int64_t)pending_.size() < cfg_.max_batch) {
                        auto until = pending_.front()->t_admit + std::chrono::microseconds(cfg_.max_wait_us);
                        if (Clock::now() < until) {
                            work_cv_.wait_until(lk, until);
                            continue;
                        }
                    }
                    break;
                }
                size_t bytes = 0;
                keys.clear();
                while (!pending_.empty() && (int)batch.size() < cfg_.max_batch) {
                    Request *r = pending_.front();
                    bool new_group = true;
                    for (const auto &kk : keys)
                        if (kk.first == r->k && kk.second == r->seed) {
                            new_group = false;
                            break;
                        }
                    size_t add = r->bytes + (new_group ? kGroupOverhead : 0);
                    if (!batch.empty() && bytes + add > cfg_.lane_bytes) break;
                    bytes += add;
                    if (new_group) keys.emplace_back(r->k, r->seed);
                    batch.push_back(r);
                    pending_.pop_front();
                    if (cfg_.per_request) break;
                }
                // more work may remain for another lane
                if (!pending_.empty()) work_cv_.notify_one();
            }
            groups.clear();
            for (Request *r : batch) {
                Group *g = nullptr;
                for (auto &x : groups)
                    if (x.k == r->k && x.seed == r->seed) g = &x;
                if (!g) {
                    groups.emplace_back();
                    g = &groups.back();
                    g->k = r->k;
                    g->seed = r->seed;
                }
                g->reqs.push_back(r);
                g->nnz += r->nnz;
                r->status = kOK;
            }
            int rc;
            int f = fail_next_.load();
            if (f > 0 && fail_next_.compare_exchange_strong(f, f - 1)) rc = kECUDA;
            else rc = exec_->run(lane, groups);
            complete(batch, rc, (int64_t)groups.size());
        }
    }

    void complete(std::vector<Request *> &batch, int rc, int64_t ngroups) {
        const auto now = Clock::now();
        {
            std::lock_guard<std::mutex> lk(mu_);
            for (Request *r : batch) {
                if (rc) r->status = rc;
                r->t_done = now;
                admitted_ -= r->bytes;
                ++stats_.completed;
                if (r->status) ++stats_.failed;
                const int64_t ns = std::chrono::duration_cast<std::chrono::nanoseconds>(now - r->t_arrival).count();
                if (lat_.size() < kLatencyRing) lat_.push_back(ns);
                else lat_[lat_next_++ % kLatencyRing] = ns;
                r->done = true;
            }
            ++stats_.batches;
            stats_.groups += ngroups;
            batched_requests_ += (int64_t)batch.size();
        }
        done_cv_.notify_all();
    }

    Config cfg_;
    Executor *exec_;
    std::mutex mu_;
    std::condition_variable work_cv_, done_cv_;
    std::deque<Request *> pending_;
    std::unordered_map<int64_t, std::unique_ptr<Request>> tickets_;
    size_t admitted_ = 0;
    int64_t next_ticket_ = 0;
    bool stopping_ = false;
    std::atomic<int> fail_next_{0};
    Stats stats_;
    int64_t batched_requests_ = 0;
    std::vector<int64_t> lat_;
    size_t lat_next_ = 0;
    std::vector<std::thread> workers_;
};

// Plays a request trace in real time: request i is submitted at start + arrival_ns[i] (a
// request refused for lack of budget is resubmitted as capacity frees, its latency still counted
// from its scheduled arrival).  Returns after every request is done; latency_ns and status may be
// null.  reqs must already hold k, seed, nnz, indices, weights and out.
inline void replay(Core &core, std::vector<Request> &reqs, const int64_t *arrival_ns, int64_t *latency_ns,
                   int32_t *status) {
    const auto start = Clock::now() + std::chrono::milliseconds(2);
    for (size_t i = 0; i < reqs.size(); ++i) {
        Request &r = reqs[i];
        const auto target = start + std::chrono::nanoseconds(arrival_ns[i]);
        auto now = Clock::now();
        if (target - now > std::chrono::microseconds(300)) std::this_thread::sleep_until(target - std::chrono::microseconds(200));
        while (Clock::now() < target) std::this_thread::yield();
        r.t_arrival = target;
        int rc;
        while ((rc = core.submit(&r)) == kEAGAIN) core.wait_capacity(request_bytes(r.nnz, r.k), std::chrono::milliseconds(10));
        if (rc) {
            r.status = rc;
            r.t_done = Clock::now();
            r.done = true;
        }
    }
    for (size_t i = 0; i < reqs.size(); ++i) {
        core.wait_done(&reqs[i]);
        if (latency_ns)
            latency_ns[i] = std::chrono::duration_cast<std::chrono::nanoseconds>(reqs[i].t_done - reqs[i].t_arrival).count();
        if (status) status[i] = reqs[i].status;
    }
}

}  // namespace serve
}  // namespace dm
