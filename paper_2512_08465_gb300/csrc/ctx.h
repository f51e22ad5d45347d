// Context of libcs (host side): resident networks, workspaces, the request
// queue and the serving scheduler.  Shared by cs_api.cu (context, networks,
// direct evaluation, Risk Index) and serve.cu (requests, continuous batching,
// HBM admission).
#pragma once
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "cs_internal.h"
#include "symbolic.h"

namespace csi {

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    cudaError_t ensure(size_t nbytes) {
        if (nbytes <= bytes) return cudaSuccess;
        release();
        cudaError_t e = cudaMalloc(&p, nbytes);
        if (e == cudaSuccess) bytes = nbytes;
        return e;
    }
};

struct Network {
    int id = 0;
    int busy = 0;                     // calls reading its tables outside the context lock
    int opf_cap = 0, dyn_cap = 0;     // resident blocks per SM chosen by the autotuner (0 = default)
    int max_it = 50;                  // interior-point iteration cap of this network
    DevNet dev{};
    DevBuf blob;                      // all static device arrays
    Symbolic sym;
    int nlev = 0;
    std::vector<std::unique_ptr<DevBuf>> sev_n1, sev_pairs;   // per level
    // base-case results per level (host)
    std::vector<uint8_t> base_klass, base_severe;
    std::vector<int16_t> base_isl, base_iters;
    std::vector<double> base_cost, base_maxre, base_minz;
    size_t resident_bytes() const {
        size_t b = blob.bytes;
        for (auto& d : sev_n1) b += d->bytes;
        for (auto& d : sev_pairs) b += d->bytes;
        return b;
    }
};

// Device workspace of one evaluation in flight: per-CTA scratch, per-scenario
// intermediates of one chunk, work counters.  Evaluations that share a
// workspace are chained through `free` (each waits for the previous one,
// whatever its stream).
struct Workspace {
    DevBuf scratch, isl, opfx, opfst, counters, hbuf, abuf, a64, cand, hws;
    cudaEvent_t free = nullptr;
    bool used = false;
    size_t bytes() const {
        return scratch.bytes + isl.bytes + opfx.bytes + opfst.bytes + counters.bytes + hbuf.bytes + abuf.bytes +
               a64.bytes + cand.bytes + hws.bytes;
    }
    void release() {
        scratch.release(); isl.release(); opfx.release(); opfst.release(); counters.release();
        hbuf.release(); abuf.release(); a64.release(); cand.release(); hws.release();
    }
    ~Workspace() {
        if (free) cudaEventDestroy(free);
    }
};

// A request of the serving path: host copies of its element ids, its results
// once done.  state: 0 queued, 1 running (some of it handed to batches), 2 done,
// 3 failed (err).  A request is split over batches when it does not fit the one
// being formed, so a batch never waits for a whole large request.
struct ServeReq {
    uint64_t id = 0;
    int net_id = 0, level = 0;
    int64_t n = 0;
    int64_t next = 0;                 // scenarios handed to batches so far (in order)
    int64_t done_n = 0;               // scenarios whose records are back
    std::vector<int32_t> ei, ej;
    std::vector<char> out;            // records in result_layout order
    int state = 0;
    cs_status err = CS_OK;
};

// A slice of a request in a batch: records [roff, roff + cnt) of the request sit at
// [boff, boff + cnt) of the batch.
struct SliceRef {
    uint64_t rid;
    int64_t boff, roff, cnt;
};

// One batch slot of the scheduler: its own stream, workspace and staging.
struct Slot {
    Workspace ws;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    DevBuf d_in, d_out;
    void* h_in = nullptr;
    size_t h_in_bytes = 0;
    void* h_out = nullptr;
    size_t h_out_bytes = 0;
    bool busy = false;
    int64_t n = 0;
    std::vector<SliceRef> members;    // request slices in the batch
    size_t device_bytes() const { return ws.bytes() + d_in.bytes + d_out.bytes; }
    ~Slot() {
        if (h_in) cudaFreeHost(h_in);
        if (h_out) cudaFreeHost(h_out);
        if (done) cudaEventDestroy(done);
        if (stream) cudaStreamDestroy(stream);
    }
};

struct ServeStats {
    int64_t batches = 0, completed = 0, merged = 0, admission_waits = 0, nomem = 0;
    int64_t peak_reserved = 0;
};

}  // namespace csi

struct cs_ctx {
    std::mutex mu;
    cs_options opt{};
    int device = 0;
    int sms = 0;
    std::string err;
    std::map<int, std::unique_ptr<csi::Network>> nets;
    int next_net = 1;
    cudaStream_t req_stream = nullptr;            // library stream (risk index, base cases)
    csi::Workspace direct, direct2;               // workspaces of cs_evaluate_device (chunks alternate) and base cases
    cudaStream_t aux_stream = nullptr;            // second stream of cs_evaluate_device
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    csi::DevBuf err_word;                         // [0] device error bits, [1] FP64 re-run count
    csi::DevBuf hess_ws;                          // workspace of cs_hessenberg_tc
    int64_t launches = 0;
    // serving: request queue, batch slots, scheduler thread
    uint64_t next_req = 1;
    std::map<uint64_t, std::unique_ptr<csi::ServeReq>> sreqs;
    std::deque<uint64_t> queue;
    std::vector<std::unique_ptr<csi::Slot>> slots;
    std::thread sched;
    std::condition_variable cv_sched, cv_done;
    bool stop = false;
    csi::ServeStats stats;
    // optional per-kernel timing (cs_set_timing): events around each launch
    bool timing = false;
    std::vector<cudaEvent_t> ev;      // pairs (start, stop) per kernel launch, reused
    std::vector<int> ev_kind;         // 0 islands, 1 opf, 2 dyn (+record)
    size_t ev_used = 0;
    double kernel_ms[3] = {0.0, 0.0, 0.0};
    int64_t kernel_launches[3] = {0, 0, 0};
};

namespace csi {

cs_status fail(cs_ctx* c, cs_status st, const std::string& msg);
cs_status cuda_fail(cs_ctx* c, cudaError_t e, const char* where);

#define CS_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return csi::cuda_fail(ctx, e_, #call);   \
    } while (0)

// Chunk of scenarios per internal batch for a context and network (0 in the options:
// 8192, or what fits ~6 GB for mixed-form networks whose state matrices take the
// tensor-core path).
int64_t default_chunk(const cs_ctx* ctx, const Network& net);

// Device bytes a workspace needs to evaluate chunks of `chunk` scenarios of net.
size_t workspace_bytes(const cs_ctx* ctx, const Network& net, int64_t chunk);

// Device bytes currently held by the context (networks, workspaces, staging).
size_t reserved_bytes(const cs_ctx* ctx);

// Evaluate n scenarios of (net, level) from device ids into device records,
// asynchronously on s, with workspace ws, in chunks of at most `chunk`.
// Requires ctx->mu held.
cs_status evaluate_impl(cs_ctx* ctx, Workspace& ws, Network* net, int level, const int32_t* ei,
                        const int32_t* ej, int64_t n, const cs_result* out, cudaStream_t s, bool record,
                        int64_t chunk, const int32_t* ek = nullptr);

// Result records of n scenarios as one SoA block (doubles first; every per-scenario
// field, Vm / Va excluded): byte size and the pointers into a block at base.
size_t result_bytes(int64_t n);
void result_layout(char* base, int64_t n, cs_result* r);

// The records of r from scenario c0 on (optional arrays stay NULL; nb = buses per Vm / Va row).
cs_result result_at(const cs_result& r, int64_t c0, int nb);

// Serving scheduler (serve.cu): stop and join before the context goes away;
// true if a request in the queue or in flight refers to net_id.
void serve_shutdown(cs_ctx* ctx);
bool serve_uses_network(cs_ctx* ctx, int net_id);

}  // namespace csi
