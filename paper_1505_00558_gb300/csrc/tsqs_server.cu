// tsqs_server.cu -- continuous batching of sort requests (the serving loop).
//
// A server owns n_streams lanes.  Each lane is a CUDA stream with its own sort context
// (scratch and graphs) and a staging buffer, both sized up front from the memory
// budget, so admission never allocates.  Requests wait in a FIFO queue; whenever a
// lane is idle, tsqs_server_progress forms the next batch from the queue:
//   - a request of >= kSoloKeys elements runs alone, sorted in place (no copies);
//   - smaller requests of the same key kind are packed: one kernel gathers them into
//     the lane's staging buffer back to back, one segmented sort sorts every request
//     as its own segment, one kernel scatters them back.
// Lanes run concurrently on the device, so requests that arrive while others are in
// flight are admitted as soon as a lane frees up and overlap with them.  Every request
// records when it was submitted, launched and seen complete.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tsqs.h"

namespace {

constexpr size_t kSoloKeys = 1u << 20;      // requests this large are sorted alone
constexpr size_t kWindow = 256;             // pending requests scanned to fill a batch

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct CopyDesc {
    void *req;                 // the request's device array
};

// Moves elements between the requests' arrays and the staging buffer.  Element e of
// the staging buffer belongs to request r with offs[r] <= e < offs[r+1].
template <class T>
__global__ void k_batch_copy(const CopyDesc *__restrict__ d, const uint64_t *__restrict__ offs,
                             uint32_t nreq, T *stage, int to_stage) {
    const uint64_t total = offs[nreq];
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < total;
         e += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = nreq;                     // largest r with offs[r] <= e
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) / 2;
            if (offs[mid] <= e) lo = mid; else hi = mid;
        }
        T *req = reinterpret_cast<T *>(d[lo].req);
        const uint64_t i = e - offs[lo];
        if (to_stage) stage[e] = req[i];
        else req[i] = stage[e];
    }
}

struct Req {
    void *d_base;
    size_t n, es;
    int kind;
    tsqs_result res;
};

struct Lane {
    cudaStream_t stream = nullptr;
    tsqs_ctx *ctx = nullptr;
    cudaEvent_t ev = nullptr;
    unsigned char *stage = nullptr;
    size_t stage_bytes = 0;
    uint64_t *d_offs = nullptr, *h_offs = nullptr;
    CopyDesc *d_desc = nullptr, *h_desc = nullptr;
    bool busy = false;
    std::vector<uint64_t> tickets;
};

}  // namespace

struct tsqs_server {
    size_t budget = 0;
    int max_batch = 0;
    std::vector<Lane> lanes;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Req> reqs;
    uint64_t next_ticket = 1;
    uint32_t next_batch = 1;
    size_t in_flight = 0;
    std::recursive_mutex mu;
};

namespace {

void destroy_lanes(tsqs_server *s) {
    for (Lane &L : s->lanes) {
        if (L.stream) cudaStreamSynchronize(L.stream);
        if (L.ctx) tsqs_ctx_destroy(L.ctx);
        if (L.ev) cudaEventDestroy(L.ev);
        if (L.stage) cudaFree(L.stage);
        if (L.d_offs) cudaFree(L.d_offs);
        if (L.d_desc) cudaFree(L.d_desc);
        if (L.h_offs) cudaFreeHost(L.h_offs);
        if (L.h_desc) cudaFreeHost(L.h_desc);
        if (L.stream) cudaStreamDestroy(L.stream);
    }
    s->lanes.clear();
}

// Launches one batch on lane L.  Called with the server lock held.
int launch_batch(tsqs_server *s, Lane &L, const std::vector<uint64_t> &batch) {
    const uint32_t id = s->next_batch++;
    const double t = now_s();
    Req &first = s->reqs[batch[0]];
    const size_t es = first.es;
    const int kind = first.kind;
    int rc = TSQS_OK;
    if (batch.size() == 1) {
        rc = tsqs_ctx_sort(L.ctx, first.d_base, first.n, es, kind, L.stream);
    } else {
        uint64_t acc = 0;
        for (size_t r = 0; r < batch.size(); r++) {
            const Req &q = s->reqs[batch[r]];
            L.h_offs[r] = acc;
            L.h_desc[r].req = q.d_base;
            acc += q.n;
        }
        L.h_offs[batch.size()] = acc;
        const uint32_t nreq = (uint32_t)batch.size();
        cudaMemcpyAsync(L.d_offs, L.h_offs, (nreq + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, L.stream);
        cudaMemcpyAsync(L.d_desc, L.h_desc, nreq * sizeof(CopyDesc), cudaMemcpyHostToDevice, L.stream);
        const unsigned grid = (unsigned)std::min<uint64_t>((acc + 255) / 256, 4096);
        if (es == 4) k_batch_copy<unsigned int><<<grid, 256, 0, L.stream>>>(L.d_desc, L.d_offs, nreq, (unsigned int *)L.stage, 1);
        else if (es == 8) k_batch_copy<unsigned long long><<<grid, 256, 0, L.stream>>>(L.d_desc, L.d_offs, nreq, (unsigned long long *)L.stage, 1);
        else k_batch_copy<uint4><<<grid, 256, 0, L.stream>>>(L.d_desc, L.d_offs, nreq, (uint4 *)L.stage, 1);
        rc = tsqs_ctx_sort_segmented(L.ctx, L.stage, acc, L.d_offs, nreq, es, kind, L.stream);
        if (es == 4) k_batch_copy<unsigned int><<<grid, 256, 0, L.stream>>>(L.d_desc, L.d_offs, nreq, (unsigned int *)L.stage, 0);
        else if (es == 8) k_batch_copy<unsigned long long><<<grid, 256, 0, L.stream>>>(L.d_desc, L.d_offs, nreq, (unsigned long long *)L.stage, 0);
        else k_batch_copy<uint4><<<grid, 256, 0, L.stream>>>(L.d_desc, L.d_offs, nreq, (uint4 *)L.stage, 0);
    }
    if (rc == TSQS_OK && cudaGetLastError() != cudaSuccess) rc = TSQS_ECUDA;
    if (rc == TSQS_OK && cudaEventRecord(L.ev, L.stream) != cudaSuccess) rc = TSQS_ECUDA;
    for (uint64_t tk : batch) {
        Req &q = s->reqs[tk];
        q.res.t_start = t;
        q.res.batch_id = id;
        q.res.batch_size = (uint32_t)batch.size();
        if (rc != TSQS_OK) { q.res.status = rc; q.res.done = 1; q.res.t_done = t; }
    }
    if (rc != TSQS_OK) return rc;
    L.busy = true;
    L.tickets = batch;
    return TSQS_OK;
}

}  // namespace

extern "C" {

tsqs_server *tsqs_server_create(size_t mem_budget_bytes, int n_streams, int max_batch) {
    if (n_streams < 1 || n_streams > 64 || mem_budget_bytes < (64u << 20)) return nullptr;
    tsqs_server *s = new (std::nothrow) tsqs_server();
    if (!s) return nullptr;
    s->budget = mem_budget_bytes;
    s->max_batch = max_batch > 0 ? max_batch : 256;
    // per lane: staging buffer + sort scratch for a batch of the same size (~1x) +
    // queues; 2.2x leaves headroom for the scratch's queues
    const size_t per_lane = mem_budget_bytes / (size_t)n_streams;
    const size_t stage = (size_t)((double)per_lane / 2.2) / 256 * 256;
    s->lanes.resize((size_t)n_streams);
    for (Lane &L : s->lanes) {
        bool ok = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming) == cudaSuccess &&
                  cudaMalloc(&L.stage, stage) == cudaSuccess &&
                  cudaMalloc((void **)&L.d_offs, ((size_t)s->max_batch + 1) * sizeof(uint64_t)) == cudaSuccess &&
                  cudaMalloc((void **)&L.d_desc, (size_t)s->max_batch * sizeof(CopyDesc)) == cudaSuccess &&
                  cudaHostAlloc((void **)&L.h_offs, ((size_t)s->max_batch + 1) * sizeof(uint64_t), 0) == cudaSuccess &&
                  cudaHostAlloc((void **)&L.h_desc, (size_t)s->max_batch * sizeof(CopyDesc), 0) == cudaSuccess;
        // lanes sort level by level: several lanes share the GPU, and the task-parallel
        // schedule's persistent kernel holds its SMs while its blocks wait for work, which
        // the other lanes' launches need (saturated throughput 20.0 against 15.3 Gkeys/s)
        tsqs_plan lp;
        tsqs_plan_default(TSQS_I32, 0, &lp);
        lp.schedule = 1;
        L.ctx = ok ? tsqs_ctx_create(&lp) : nullptr;
        // scratch for the largest batch of 4-byte keys this lane can hold
        if (!L.ctx || tsqs_ctx_reserve(L.ctx, stage / 4, (size_t)s->max_batch, 4) != TSQS_OK ||
            tsqs_ctx_reserve(L.ctx, stage / 16, (size_t)s->max_batch, 16) != TSQS_OK) {
            cudaGetLastError();
            destroy_lanes(s);
            delete s;
            return nullptr;
        }
        L.stage_bytes = stage;
    }
    return s;
}

int tsqs_server_submit(tsqs_server *s, void *d_base, size_t nmemb, size_t elem_size,
                       int key_kind, uint64_t *ticket) {
    if (!s || !ticket) return TSQS_EINVAL;
    const size_t es = key_kind >= TSQS_I32 && key_kind <= TSQS_F32 ? 4
                    : key_kind >= TSQS_I64 && key_kind <= TSQS_F64 ? 8
                    : key_kind == TSQS_U64_U64_REC ? 16 : 0;
    if (!es || es != elem_size || (nmemb && !d_base)) return TSQS_EINVAL;
    if ((uintptr_t)d_base % es) return TSQS_EINVAL;      // records need 16-byte alignment
    std::lock_guard<std::recursive_mutex> lk(s->mu);
    if (nmemb * es > s->lanes[0].stage_bytes) return TSQS_ENOMEM;   // can never fit a lane
    Req q{};
    q.d_base = d_base;
    q.n = nmemb;
    q.es = es;
    q.kind = key_kind;
    q.res.t_submit = now_s();
    const uint64_t tk = s->next_ticket++;
    if (nmemb <= 1) {                       // nothing to do
        q.res.done = 1;
        q.res.t_start = q.res.t_done = q.res.t_submit;
        s->reqs[tk] = q;
    } else {
        s->reqs[tk] = q;
        s->pending.push_back(tk);
    }
    *ticket = tk;
    return TSQS_OK;
}

int tsqs_server_progress(tsqs_server *s) {
    if (!s) return 0;
    std::lock_guard<std::recursive_mutex> lk(s->mu);
    // retire finished lanes
    for (Lane &L : s->lanes) {
        if (!L.busy) continue;
        const cudaError_t e = cudaEventQuery(L.ev);
        if (e == cudaErrorNotReady) continue;
        const double t = now_s();
        int st = e == cudaSuccess ? tsqs_ctx_device_status(L.ctx, L.stream) : TSQS_ECUDA;
        if (e != cudaSuccess) cudaGetLastError();
        for (uint64_t tk : L.tickets) {
            Req &q = s->reqs[tk];
            q.res.status = st;
            q.res.done = 1;
            q.res.t_done = t;
            s->in_flight -= q.n * q.es;
        }
        L.tickets.clear();
        L.busy = false;
    }
    // admit: fill every idle lane from the front of the queue
    for (Lane &L : s->lanes) {
        if (L.busy || s->pending.empty()) continue;
        std::vector<uint64_t> batch;
        const Req &head = s->reqs[s->pending.front()];
        size_t bytes = 0;
        if (head.n >= kSoloKeys) {
            batch.push_back(s->pending.front());
            bytes = head.n * head.es;
            s->pending.pop_front();
        } else {
            const int kind = head.kind;
            size_t scanned = 0;
            for (auto it = s->pending.begin(); it != s->pending.end() && scanned < kWindow;) {
                const Req &q = s->reqs[*it];
                scanned++;
                if (q.kind == kind && q.n < kSoloKeys && bytes + q.n * q.es <= L.stage_bytes &&
                    (int)batch.size() < s->max_batch) {
                    batch.push_back(*it);
                    bytes += q.n * q.es;
                    it = s->pending.erase(it);
                } else {
                    ++it;
                }
            }
        }
        if (batch.empty()) continue;
        s->in_flight += bytes;
        if (launch_batch(s, L, batch) != TSQS_OK) s->in_flight -= bytes;
    }
    size_t busy = 0;
    for (Lane &L : s->lanes) busy += L.tickets.size();
    return (int)(s->pending.size() + busy);
}

int tsqs_server_poll(tsqs_server *s, uint64_t ticket, tsqs_result *out) {
    if (!s || !out) return TSQS_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return TSQS_EINVAL;
    *out = it->second.res;
    return TSQS_OK;
}

int tsqs_server_drain(tsqs_server *s) {
    if (!s) return TSQS_EINVAL;
    for (;;) {
        if (tsqs_server_progress(s) == 0) return TSQS_OK;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

void tsqs_server_destroy(tsqs_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::recursive_mutex> lk(s->mu);
        destroy_lanes(s);
    }
    delete s;
}

}  // extern "C"
