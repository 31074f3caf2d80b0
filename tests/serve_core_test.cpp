// Host-only tests of the serving core (admission, continuous batching, completion, failure
// paths) with a fake executor standing in for the GPU.  Built and run by test_serve_core.py.
// The fake computes a placeholder key per slot (a mix of the request's inputs), not the method:
// what is checked here is that every request receives exactly its own result, whatever batch it
// lands in.
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <set>
#include <string>
#include <thread>

#include "serve_core.h"

using namespace dm::serve;

static int g_failed = 0;
#define CHECK(cond)                                                                   \
    do {                                                                              \
        if (!(cond)) {                                                                \
            std::printf("FAIL %s:%d: %s\n", __FILE__, __LINE__, #cond);              \
            ++g_failed;                                                               \
            return;                                                                   \
        }                                                                             \
    } while (0)

static uint64_t mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Placeholder result of a request: depends on every input, the seed, k and the slot.
static uint64_t fake_key(const uint32_t *idx, const float *w, int64_t nnz, int32_t k, uint64_t seed, int j) {
    uint64_t h = mix(seed ^ (uint64_t)k * 0x9E3779B97F4A7C15ull);
    for (int64_t i = 0; i < nnz; ++i) {
        uint32_t wb;
        std::memcpy(&wb, &w[i], 4);
        h = mix(h ^ idx[i] ^ ((uint64_t)wb << 32));
    }
    return mix(h + (uint64_t)j);
}

struct FakeExecutor : Executor {
    std::mutex mu;
    std::condition_variable cv;
    bool gated = false;                 // run() blocks while true
    std::atomic<int> running{0}, max_running{0}, batches{0};
    size_t lane_bytes = 0;
    int max_batch = 0;
    std::atomic<int> bad_batches{0};    // batches breaking a rule
    std::atomic<int> max_seen_batch{0};

    int run(int, std::vector<Group> &groups) override {
        int r = ++running;
        int m = max_running.load();
        while (r > m && !max_running.compare_exchange_weak(m, r)) {}
        {
            std::unique_lock<std::mutex> lk(mu);
            cv.wait(lk, [&] { return !gated; });
        }
        size_t bytes = 0, n = 0;
        int rc = kOK;
        std::set<std::pair<int32_t, uint64_t>> keys;
        for (auto &g : groups) {
            if (!keys.insert({g.k, g.seed}).second) ++bad_batches;        // a (k, seed) split in two groups
            bytes += kGroupOverhead;
            for (Request *q : g.reqs) {
                if (q->k != g.k || q->seed != g.seed) ++bad_batches;
                bytes += q->bytes;
                ++n;
                if (q->k == 13) rc = 9;                 // poison: fails its whole batch
                if (q->nnz == 0) {                      // fails alone
                    q->status = 5;
                    continue;
                }
                if (q->out)
                    for (int j = 0; j < q->k; ++j) q->out[j] = fake_key(q->indices, q->weights, q->nnz, q->k, q->seed, j);
            }
        }
        if (bytes > lane_bytes || (int)n > max_batch) ++bad_batches;
        int mb = max_seen_batch.load();
        while ((int)n > mb && !max_seen_batch.compare_exchange_weak(mb, (int)n)) {}
        ++batches;
        --running;
        return rc;
    }
    void set_gate(bool g) {
        {
            std::lock_guard<std::mutex> lk(mu);
            gated = g;
        }
        cv.notify_all();
    }
};

struct Owned {
    std::vector<uint32_t> idx;
    std::vector<float> w;
    std::vector<uint64_t> out;
    Request r;
};

static void make(Owned &o, uint64_t salt, int64_t nnz, int32_t k, uint64_t seed) {
    o.idx.resize((size_t)nnz);
    o.w.resize((size_t)nnz);
    for (int64_t i = 0; i < nnz; ++i) {
        o.idx[(size_t)i] = (uint32_t)(mix(salt * 131 + (uint64_t)i) & 0xFFFFFF);
        o.w[(size_t)i] = (float)((mix(salt * 977 + (uint64_t)i) >> 40) + 1) / 16777216.0f;
    }
    o.out.assign((size_t)k, 0);
    o.r.k = k;
    o.r.seed = seed;
    o.r.nnz = nnz;
    o.r.indices = o.idx.data();
    o.r.weights = o.w.data();
    o.r.out = o.out.data();
    o.r.t_arrival = Clock::now();
}

static bool result_ok(Owned &o) {
    for (int j = 0; j < o.r.k; ++j)
        if (o.out[(size_t)j] != fake_key(o.idx.data(), o.w.data(), o.r.nnz, o.r.k, o.r.seed, j)) return false;
    return true;
}

static void test_many_threads_mixed_k() {
    FakeExecutor ex;
    Config c;
    c.lanes = 3;
    c.lane_bytes = 1 << 20;
    c.max_batch = 64;
    ex.lane_bytes = c.lane_bytes;
    ex.max_batch = c.max_batch;
    std::vector<Owned> reqs(4000);
    {
        Core core(c, &ex);
        std::vector<std::thread> th;
        for (int t = 0; t < 4; ++t)
            th.emplace_back([&, t] {
                for (size_t i = (size_t)t; i < reqs.size(); i += 4) {
                    const int32_t ks[3] = {64, 256, 1024};
                    make(reqs[i], i, 1 + (int64_t)(mix(i) % 300), ks[i % 3], 1 + (i % 2));
                    int rc;
                    while ((rc = core.submit(&reqs[i].r)) == kEAGAIN) core.wait_capacity(reqs[i].r.bytes, std::chrono::milliseconds(5));
                    if (rc) std::abort();
                }
            });
        for (auto &x : th) x.join();
        for (auto &o : reqs) core.wait_done(&o.r);
        Stats s = core.stats();
        CHECK(s.completed == 4000 && s.failed == 0 && s.submitted == 4000);
        CHECK(s.batches == ex.batches.load());
        CHECK(s.admitted_bytes == 0);
        CHECK(s.p50_us >= 0 && s.p99_us >= s.p50_us && s.max_us >= s.p99_us);
    }
    for (auto &o : reqs) CHECK(o.r.done && o.r.status == 0 && result_ok(o));
    CHECK(ex.bad_batches.load() == 0);
    CHECK(ex.max_running.load() <= 3);
    std::printf("PASS many_threads_mixed_k (batches %d, largest %d)\n", ex.batches.load(), ex.max_seen_batch.load());
}

static void test_admission_budget() {
    FakeExecutor ex;
    ex.set_gate(true);
    Config c;
    c.lanes = 1;
    c.lane_bytes = 1 << 20;
    c.budget = 3 * request_bytes(10, 64) + 100;      // room for exactly three such requests
    ex.lane_bytes = c.lane_bytes;
    ex.max_batch = c.max_batch;
    std::vector<Owned> reqs(5);
    Core core(c, &ex);
    for (int i = 0; i < 5; ++i) make(reqs[(size_t)i], 100 + (uint64_t)i, 10, 64, 7);
    CHECK(core.submit(&reqs[0].r) == kOK);
    CHECK(core.submit(&reqs[1].r) == kOK);
    CHECK(core.submit(&reqs[2].r) == kOK);
    CHECK(core.submit(&reqs[3].r) == kEAGAIN);
    CHECK(core.stats().admitted_bytes == (int64_t)(3 * request_bytes(10, 64)));
    CHECK(core.stats().rejected == 1);
    CHECK(!core.wait_capacity(reqs[3].r.bytes, std::chrono::milliseconds(20)));   // still full
    ex.set_gate(false);
    CHECK(core.wait_capacity(reqs[3].r.bytes, std::chrono::seconds(5)));
    CHECK(core.submit(&reqs[3].r) == kOK);
    CHECK(core.submit(&reqs[4].r) == kOK);
    for (auto &o : reqs) core.wait_done(&o.r);
    for (auto &o : reqs) CHECK(o.r.status == 0 && result_ok(o));
    // a request larger than a lane can never run
    Owned big;
    make(big, 999, (int64_t)(c.lane_bytes / 8), 64, 1);
    CHECK(core.submit(&big.r) == kENOMEM);
    std::printf("PASS admission_budget\n");
}

static void test_failures() {
    FakeExecutor ex;
    Config c;
    c.lanes = 2;
    c.lane_bytes = 1 << 20;
    c.per_request = true;                           // one request per batch: failures are exact
    ex.lane_bytes = c.lane_bytes;
    ex.max_batch = c.max_batch;
    std::vector<Owned> reqs(40);
    {
        Core core(c, &ex);
        for (size_t i = 0; i < reqs.size(); ++i) {
            int32_t k = i == 7 ? 13 : 64;           // request 7 poisons its batch
            make(reqs[i], 500 + i, i == 11 ? 0 : 20, k, 3);   // request 11 fails alone
        }
        for (size_t i = 0; i < 20; ++i) CHECK(core.submit(&reqs[i].r) == kOK);
        for (size_t i = 0; i < 20; ++i) core.wait_done(&reqs[i].r);
        core.fail_next_batches(1);                  // injected launch failure
        CHECK(core.submit(&reqs[20].r) == kOK);
        core.wait_done(&reqs[20].r);
        for (size_t i = 21; i < reqs.size(); ++i) CHECK(core.submit(&reqs[i].r) == kOK);
        for (size_t i = 21; i < reqs.size(); ++i) core.wait_done(&reqs[i].r);
        Stats s = core.stats();
        CHECK(s.completed == 40 && s.failed == 3);
    }
    for (size_t i = 0; i < reqs.size(); ++i) {
        const int want = i == 7 ? 9 : (i == 11 ? 5 : (i == 20 ? kECUDA : 0));
        CHECK(reqs[i].r.status == want);
        if (want == 0) CHECK(result_ok(reqs[i]));
    }
    CHECK(ex.max_seen_batch.load() == 1);
    std::printf("PASS failures\n");
}

static void test_tickets_and_timeout() {
    FakeExecutor ex;
    ex.set_gate(true);
    Config c;
    c.lanes = 1;
    c.lane_bytes = 1 << 20;
    ex.lane_bytes = c.lane_bytes;
    ex.max_batch = c.max_batch;
    Core core(c, &ex);
    Owned o;
    make(o, 1234, 30, 256, 5);
    std::unique_ptr<Request> tr(new Request());
    tr->k = o.r.k;
    tr->seed = o.r.seed;
    tr->nnz = o.r.nnz;
    tr->indices = o.idx.data();
    tr->weights = o.w.data();
    tr->out = o.out.data();
    tr->t_arrival = Clock::now();
    Request *raw = tr.get();
    CHECK(core.submit(raw, std::move(tr)) == kOK);
    const int64_t ticket = raw->ticket;
    int st = 0;
    CHECK(core.poll(ticket, &st) == kOK && st == -1);
    CHECK(core.wait(ticket, 20000, &st) == kETIMEOUT);
    ex.set_gate(false);
    CHECK(core.wait(ticket, 5000000, &st) == kOK && st == 0);
    CHECK(result_ok(o));
    CHECK(core.poll(ticket, &st) == kEINVAL);       // released
    CHECK(core.poll(987654, &st) == kEINVAL);
    std::printf("PASS tickets_and_timeout\n");
}

static void test_stop_finishes_pending() {
    FakeExecutor ex;
    Config c;
    c.lanes = 2;
    c.lane_bytes = 1 << 18;
    c.max_batch = 8;
    ex.lane_bytes = c.lane_bytes;
    ex.max_batch = c.max_batch;
    std::vector<Owned> reqs(300);
    {
        Core core(c, &ex);
        for (size_t i = 0; i < reqs.size(); ++i) {
            make(reqs[i], 7000 + i, 50, 64, 1);
            CHECK(core.submit(&reqs[i].r) == kOK);
        }
    }   // destructor: every admitted request finishes first
    for (auto &o : reqs) CHECK(o.r.done && o.r.status == 0 && result_ok(o));
    CHECK(ex.bad_batches.load() == 0);
    std::printf("PASS stop_finishes_pending\n");
}

static void test_batching_window() {
    FakeExecutor ex;
    Config c;
    c.lanes = 1;
    c.lane_bytes = 1 << 20;
    c.max_wait_us = 200000;                        // 200 ms: the ten requests below share a batch
    ex.lane_bytes = c.lane_bytes;
    ex.max_batch = c.max_batch;
    std::vector<Owned> reqs(10);
    Core core(c, &ex);
    for (size_t i = 0; i < reqs.size(); ++i) {
        make(reqs[i], 800 + i, 5, 64, 1);
        CHECK(core.submit(&reqs[i].r) == kOK);
    }
    for (auto &o : reqs) core.wait_done(&o.r);
    CHECK(ex.batches.load() == 1);
    CHECK(core.stats().mean_batch == 10.0);
    std::printf("PASS batching_window\n");
}

static void test_replay() {
    FakeExecutor ex;
    Config c;
    c.lanes = 2;
    c.lane_bytes = 1 << 20;
    c.budget = 4 * request_bytes(40, 256);         // forces refusals and resubmission
    ex.lane_bytes = c.lane_bytes;
    ex.max_batch = c.max_batch;
    const size_t n = 500;
    std::vector<Owned> own(n);
    std::vector<Request> reqs(n);
    std::vector<int64_t> arr(n), lat(n);
    std::vector<int32_t> st(n);
    for (size_t i = 0; i < n; ++i) {
        make(own[i], 9000 + i, 1 + (int64_t)(i % 40), (int32_t)(64 << (i % 3)), 1);
        reqs[i].k = own[i].r.k;
        reqs[i].seed = own[i].r.seed;
        reqs[i].nnz = own[i].r.nnz;
        reqs[i].indices = own[i].idx.data();
        reqs[i].weights = own[i].w.data();
        reqs[i].out = own[i].out.data();
        arr[i] = (int64_t)i * 20000;               // 50,000 requests/s
    }
    const auto t0 = Clock::now();
    {
        Core core(c, &ex);
        replay(core, reqs, arr.data(), lat.data(), st.data());
        CHECK(core.stats().completed == (int64_t)n);
    }
    const double secs = std::chrono::duration<double>(Clock::now() - t0).count();
    CHECK(secs >= (double)arr[n - 1] * 1e-9);       // arrivals are honoured
    for (size_t i = 0; i < n; ++i) {
        CHECK(st[i] == 0 && lat[i] >= 0);
        CHECK(result_ok(own[i]));
    }
    std::printf("PASS replay\n");
}

int main() {
    test_many_threads_mixed_k();
    test_admission_budget();
    test_failures();
    test_tickets_and_timeout();
    test_stop_finishes_pending();
    test_batching_window();
    test_replay();
    if (g_failed) {
        std::printf("%d FAILED\n", g_failed);
        return 1;
    }
    std::printf("ALL PASS\n");
    return 0;
}
