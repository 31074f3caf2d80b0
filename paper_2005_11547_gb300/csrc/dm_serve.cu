// Serving loop of libdartminhash.so: dm_server_* (declared in include/dartminhash.h).
//
// The paper sketches one set at a time on a CPU; a GPU pays off when many small requests share
// launches.  Requests (one weighted set each, any k and seed) are admitted against a memory
// budget and batched continuously by serve_core.h; this file supplies the executor that runs a
// batch on one lane: a CUDA stream, a context of its own, one device buffer and one page-locked
// host buffer of the lane's capacity.  A batch is packed into the host buffer (CSR per (k, seed)
// group), copied to the device in one transfer, sketched with one dm_sketch-equivalent call per
// group, and its keys come back in one transfer.  Every request gets exactly the keys dm_sketch
// gives for its row alone: the kernels compute each set independently of its batch.
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "dm_internal.h"
#include "serve_core.h"

namespace {

using dm::serve::Group;
using dm::serve::Request;

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr int kGroupStreams = 4;  // groups of one batch run concurrently on these

struct Lane {
    dm_ctx *ctx[kGroupStreams] = {};   // one per group stream: each has its own side streams
    cudaStream_t st = nullptr;
    cudaStream_t gst[kGroupStreams] = {};
    cudaEvent_t ev_in = nullptr, ev_done[kGroupStreams] = {};
    unsigned char *d = nullptr;    // device buffer
    unsigned char *h = nullptr;    // page-locked host buffer, same size
};

struct GroupLayout {
    size_t ip, idx, w, out, scr;
};

class CudaExecutor : public dm::serve::Executor {
  public:
    int device = 0;
    size_t lane_bytes = 0;
    bool per_request = false;
    int large_nnz = 2048;
    int block_sets = 0;            // a group this small gives every set a block of 8 warps
    std::vector<Lane> lanes;
    std::atomic<int64_t> kernel_launches{0};

    int init(int dev, int n_lanes, size_t bytes) {
        device = dev;
        lane_bytes = bytes;
        lanes.resize((size_t)n_lanes);
        cudaError_t e = cudaSetDevice(dev);
        if (e != cudaSuccess) return DM_ECUDA;
        int sms = 0;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return DM_ECUDA;
        block_sets = 2 * sms;                       // two resident 8-warp blocks per SM
        for (auto &L : lanes) {
            for (int i = 0; i < kGroupStreams; ++i) {
                int rc = dm_create(&L.ctx[i], dev, 0);
                if (rc) return rc;
            }
            if ((e = cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&L.ev_in, cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaMalloc(&L.d, bytes)) != cudaSuccess || (e = cudaMallocHost(&L.h, bytes)) != cudaSuccess)
                return e == cudaErrorMemoryAllocation ? DM_ENOMEM : DM_ECUDA;
            for (int i = 0; i < kGroupStreams; ++i)
                if ((e = cudaStreamCreateWithFlags(&L.gst[i], cudaStreamNonBlocking)) != cudaSuccess ||
                    (e = cudaEventCreateWithFlags(&L.ev_done[i], cudaEventDisableTiming)) != cudaSuccess)
                    return DM_ECUDA;
        }
        return DM_OK;
    }

    ~CudaExecutor() override {
        cudaSetDevice(device);
        for (auto &L : lanes) {
            if (L.st) cudaStreamSynchronize(L.st);
            if (L.d) cudaFree(L.d);
            if (L.h) cudaFreeHost(L.h);
            for (int i = 0; i < kGroupStreams; ++i) {
                if (L.gst[i]) cudaStreamSynchronize(L.gst[i]);
                if (L.gst[i]) cudaStreamDestroy(L.gst[i]);
                if (L.ev_done[i]) cudaEventDestroy(L.ev_done[i]);
            }
            if (L.ev_in) cudaEventDestroy(L.ev_in);
            if (L.st) cudaStreamDestroy(L.st);
            for (int i = 0; i < kGroupStreams; ++i)
                if (L.ctx[i]) dm_destroy(L.ctx[i]);
        }
    }

    int run(int lane, std::vector<Group> &groups) override {
        Lane &L = lanes[(size_t)lane];
        cudaError_t e = cudaSetDevice(device);
        if (e != cudaSuccess) return DM_ECUDA;
        // layout: every group's inputs, then every group's outputs, then every group's scratch
        std::vector<GroupLayout> lay(groups.size());
        size_t off = 0;
        for (size_t g = 0; g < groups.size(); ++g) {
            const size_t n = groups[g].reqs.size(), z = (size_t)groups[g].nnz;
            lay[g].ip = off;
            off += al256(8 * (n + 1));
            lay[g].idx = off;
            off += al256(4 * z);
            lay[g].w = off;
            off += al256(4 * z);
        }
        const size_t in_end = off;
        for (size_t g = 0; g < groups.size(); ++g) {
            lay[g].out = off;
            off += al256(8 * groups[g].reqs.size() * (size_t)groups[g].k);
        }
        const size_t out_end = off;
        for (size_t g = 0; g < groups.size(); ++g) {
            lay[g].scr = off;
            off += dm::call_scratch_bytes((int64_t)groups[g].reqs.size());
        }
        if (off > lane_bytes) return DM_ENOMEM;     // admission arithmetic keeps this from happening
        // pack the CSR of each group into the host buffer
        for (size_t g = 0; g < groups.size(); ++g) {
            int64_t *ip = (int64_t *)(L.h + lay[g].ip);
            uint32_t *ix = (uint32_t *)(L.h + lay[g].idx);
            float *w = (float *)(L.h + lay[g].w);
            int64_t z = 0;
            ip[0] = 0;
            for (size_t i = 0; i < groups[g].reqs.size(); ++i) {
                const Request *r = groups[g].reqs[i];
                if (r->nnz) {
                    std::memcpy(ix + z, r->indices, (size_t)r->nnz * 4);
                    std::memcpy(w + z, r->weights, (size_t)r->nnz * 4);
                }
                z += r->nnz;
                ip[i + 1] = z;
            }
        }
        if ((e = cudaMemcpyAsync(L.d, L.h, in_end, cudaMemcpyHostToDevice, L.st)) != cudaSuccess) return DM_ECUDA;
        // the groups run concurrently, each on a stream of its own after the input copy
        const bool fork = !per_request && groups.size() > 1;
        if (fork && (e = cudaEventRecord(L.ev_in, L.st)) != cudaSuccess) return DM_ECUDA;
        for (size_t g = 0; g < groups.size(); ++g) {
            const size_t n = groups[g].reqs.size();
            int64_t max_nnz = 0;
            for (const Request *r : groups[g].reqs) max_nnz = r->nnz > max_nnz ? r->nnz : max_nnz;
            // plain per-request form; a small group gives each set a block of 8 warps (batched
            // form with every non-empty set in the large class); otherwise persistent warps, or
            // the batched form when a set is large enough for a block of its own
            int form = 2, large = -1;
            if (per_request) form = 1;
            else if ((int64_t)n <= block_sets) { form = 0; large = 1; }
            else if (large_nnz > 0 && max_nnz >= large_nnz) form = 0;
            cudaStream_t gs = fork ? L.gst[g % kGroupStreams] : L.st;
            dm_ctx *gctx = L.ctx[fork ? g % kGroupStreams : 0];
            if (fork && (e = cudaStreamWaitEvent(gs, L.ev_in, 0)) != cudaSuccess) return DM_ECUDA;
            int rc = dm::serve_sketch(gctx, (const int64_t *)(L.d + lay[g].ip), (const uint32_t *)(L.d + lay[g].idx),
                                      (const float *)(L.d + lay[g].w), (int64_t)n, groups[g].k, groups[g].seed,
                                      (uint64_t *)(L.d + lay[g].out), L.d + lay[g].scr, form, large, gs);
            if (rc) {
                cudaStreamSynchronize(L.st);
                for (int i = 0; i < kGroupStreams; ++i) cudaStreamSynchronize(L.gst[i]);
                return rc;
            }
            // kernels of the form: fast + general, plus classify, scan, scatter, large and the
            // general kernel's second launch over the fast kernel's deferrals (batched)
            kernel_launches += form == 0 ? 7 : 2;
        }
        if (fork)
            for (int i = 0; i < kGroupStreams && (size_t)i < groups.size(); ++i)
                if ((e = cudaEventRecord(L.ev_done[i], L.gst[i])) != cudaSuccess ||
                    (e = cudaStreamWaitEvent(L.st, L.ev_done[i], 0)) != cudaSuccess)
                    return DM_ECUDA;
        if (out_end > in_end &&
            (e = cudaMemcpyAsync(L.h + in_end, L.d + in_end, out_end - in_end, cudaMemcpyDeviceToHost, L.st)) !=
                cudaSuccess)
            return DM_ECUDA;
        const int nctx = fork ? (int)(groups.size() < (size_t)kGroupStreams ? groups.size() : kGroupStreams) : 1;
        for (int i = 0; i < nctx; ++i)
            if ((e = dm::status_to_host(L.ctx[i], L.st)) != cudaSuccess) return DM_ECUDA;
        if ((e = cudaStreamSynchronize(L.st)) != cudaSuccess) return DM_ECUDA;
        int status = 0;
        for (int i = 0; i < nctx; ++i) {
            const int s = dm::status_take(L.ctx[i], L.st);
            if (s == DM_ECUDA) return DM_ECUDA;
            if (!status) status = s;
        }
        // deliver; a kernel-recorded error (a weight or norm out of range) marks its rows all-ones,
        // which a set with a positive weight never gets otherwise: those requests carry the error
        for (size_t g = 0; g < groups.size(); ++g) {
            const size_t k = (size_t)groups[g].k;
            for (size_t i = 0; i < groups[g].reqs.size(); ++i) {
                Request *r = groups[g].reqs[i];
                const uint64_t *src = (const uint64_t *)(L.h + lay[g].out) + i * k;
                if (status) {
                    bool all_ones = true, positive = false;
                    for (size_t j = 0; j < k && all_ones; ++j) all_ones = src[j] == ~0ull;
                    for (int64_t j = 0; j < r->nnz && !positive; ++j) positive = r->weights[j] > 0.f;
                    if (all_ones && positive) r->status = status;
                }
                if (r->out) std::memcpy(r->out, src, k * 8);
            }
        }
        return DM_OK;
    }
};

// Checks one request on the host: k supported, weights finite and >= 0 (the domain of the
// method; the kernels would flag them too, but a serving caller wants the answer per request).
int check_request(const uint32_t *indices, const float *weights, int64_t nnz, int32_t k) {
    if (k < 1 || k > 8192 || dm_t_of_k(k) <= 0 || nnz < 0) return DM_EINVAL;
    if (nnz > 0 && (!indices || !weights)) return DM_EINVAL;
    for (int64_t j = 0; j < nnz; ++j)
        if (!(weights[j] >= 0.f) || std::isinf(weights[j])) return DM_EINVAL;
    return DM_OK;
}

}  // namespace

struct dm_server {
    CudaExecutor exec;
    dm::serve::Core *core = nullptr;
};

extern "C" {

int dm_server_create(dm_server **out, const dm_server_config *cfg) {
    if (!out || !cfg) return DM_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) return DM_ECUDA;
    if (cfg->device < 0 || cfg->device >= n || cfg->lanes < 0 || cfg->lanes > 64 || cfg->max_batch < 0 ||
        cfg->max_wait_us < 0 || cfg->large_nnz < 0)
        return DM_EINVAL;
    dm::serve::Config c;
    c.lanes = cfg->lanes ? cfg->lanes : 4;
    c.budget = cfg->mem_budget_bytes ? cfg->mem_budget_bytes : ((size_t)8 << 30);
    size_t lane = cfg->lane_bytes ? cfg->lane_bytes : ((size_t)64 << 20);
    if (lane > c.budget / (size_t)c.lanes) lane = c.budget / (size_t)c.lanes;    // lanes fit the budget
    lane &= ~(size_t)255;
    if (lane < ((size_t)1 << 16)) return DM_EINVAL;
    c.lane_bytes = lane;
    c.max_batch = cfg->max_batch ? cfg->max_batch : 4096;
    c.max_wait_us = cfg->max_wait_us;
    c.per_request = cfg->per_request != 0;
    dm_server *s = new (std::nothrow) dm_server();
    if (!s) return DM_ENOMEM;
    s->exec.per_request = c.per_request;
    s->exec.large_nnz = cfg->large_nnz ? cfg->large_nnz : 2048;
    int rc = s->exec.init(cfg->device, c.lanes, lane);
    if (rc) {
        delete s;
        return rc;
    }
    s->core = new dm::serve::Core(c, &s->exec);
    *out = s;
    return DM_OK;
}

int dm_server_destroy(dm_server *srv) {
    if (!srv) return DM_OK;
    delete srv->core;     // finishes every admitted request first
    delete srv;
    return DM_OK;
}

int dm_server_submit(dm_server *srv, const uint32_t *indices, const float *weights, int64_t nnz, int32_t k,
                     uint64_t seed, uint64_t *out, int64_t *ticket) {
    if (!srv || !ticket) return DM_EINVAL;
    int rc = check_request(indices, weights, nnz, k);
    if (rc) return rc;
    std::unique_ptr<Request> r(new (std::nothrow) Request());
    if (!r) return DM_ENOMEM;
    r->k = k;
    r->seed = seed;
    r->nnz = nnz;
    if (nnz > 0) {
        r->own.reset(new (std::nothrow) unsigned char[(size_t)nnz * 8]);
        if (!r->own) return DM_ENOMEM;
        std::memcpy(r->own.get(), indices, (size_t)nnz * 4);
        std::memcpy(r->own.get() + (size_t)nnz * 4, weights, (size_t)nnz * 4);
        r->indices = (const uint32_t *)r->own.get();
        r->weights = (const float *)(r->own.get() + (size_t)nnz * 4);
    }
    r->out = out;
    r->t_arrival = dm::serve::Clock::now();
    Request *raw = r.get();
    rc = srv->core->submit(raw, std::move(r));
    if (rc == DM_OK) *ticket = raw->ticket;
    return rc;
}

int dm_server_poll(dm_server *srv, int64_t ticket, int32_t *status) {
    if (!srv || !status) return DM_EINVAL;
    int s = 0;
    int rc = srv->core->poll(ticket, &s);
    *status = s;
    return rc;
}

int dm_server_wait(dm_server *srv, int64_t ticket, int64_t timeout_us, int32_t *status) {
    if (!srv || !status) return DM_EINVAL;
    int s = 0;
    int rc = srv->core->wait(ticket, timeout_us, &s);
    if (rc == DM_OK) *status = s;
    return rc;
}

int dm_server_replay(dm_server *srv, int64_t n, const int64_t *indptr, const uint32_t *indices,
                     const float *weights, const int32_t *k, const uint64_t *seed, const int64_t *arrival_ns,
                     uint64_t *out, int64_t *latency_ns, int32_t *status) {
    if (!srv || n < 0 || (n > 0 && (!indptr || !k || !seed || !arrival_ns))) return DM_EINVAL;
    if (n == 0) return DM_OK;
    if (indptr[0] != 0) return DM_EINVAL;
    for (int64_t i = 0; i < n; ++i)
        if (indptr[i + 1] < indptr[i] || arrival_ns[i] < 0 || (i > 0 && arrival_ns[i] < arrival_ns[i - 1]))
            return DM_EINVAL;
    // a request that fails the host checks is answered at once with its error
    std::vector<int64_t> valid;
    valid.reserve((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        const int64_t nnz = indptr[i + 1] - indptr[i];
        int rc = check_request(nnz ? indices + indptr[i] : nullptr, nnz ? weights + indptr[i] : nullptr, nnz, k[i]);
        if (rc) {
            if (latency_ns) latency_ns[i] = 0;
            if (status) status[i] = rc;
        } else {
            valid.push_back(i);
        }
    }
    std::vector<Request> reqs(valid.size());
    std::vector<int64_t> arr(valid.size()), lat(valid.size());
    std::vector<int32_t> st(valid.size());
    int64_t out_off = 0, next = 0;
    for (size_t j = 0; j < valid.size(); ++j) {
        const int64_t i = valid[j];
        for (; next < i; ++next) out_off += k[next] > 0 ? k[next] : 0;    // skipped (invalid) requests keep their place
        Request &r = reqs[j];
        r.k = k[i];
        r.seed = seed[i];
        r.nnz = indptr[i + 1] - indptr[i];
        r.indices = r.nnz ? indices + indptr[i] : nullptr;
        r.weights = r.nnz ? weights + indptr[i] : nullptr;
        r.out = out ? out + out_off : nullptr;
        out_off += k[i];
        next = i + 1;
        arr[j] = arrival_ns[i];
    }
    dm::serve::replay(*srv->core, reqs, arr.data(), lat.data(), st.data());
    for (size_t j = 0; j < valid.size(); ++j) {
        if (latency_ns) latency_ns[valid[j]] = lat[j];
        if (status) status[valid[j]] = st[j];
    }
    return DM_OK;
}

int dm_server_get_stats(dm_server *srv, dm_server_stats *out) {
    if (!srv || !out) return DM_EINVAL;
    dm::serve::Stats s = srv->core->stats();
    out->submitted = s.submitted;
    out->completed = s.completed;
    out->failed = s.failed;
    out->rejected = s.rejected;
    out->batches = s.batches;
    out->groups = s.groups;
    out->kernel_launches = srv->exec.kernel_launches.load();
    out->admitted_bytes = s.admitted_bytes;
    out->mean_batch = s.mean_batch;
    out->p50_us = s.p50_us;
    out->p99_us = s.p99_us;
    out->max_us = s.max_us;
    return DM_OK;
}

int dm_server_reset_stats(dm_server *srv) {
    if (!srv) return DM_EINVAL;
    srv->core->reset_stats();
    return DM_OK;
}

int dm_server_fail_batches(dm_server *srv, int32_t batches) {
    if (!srv || batches < 0) return DM_EINVAL;
    srv->core->fail_next_batches(batches);
    return DM_OK;
}

}  // extern "C"
