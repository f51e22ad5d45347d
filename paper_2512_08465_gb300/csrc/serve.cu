// Serving path of libcs: requests with host buffers, continuous batching
// across requests and networks, admission by device-memory footprint.
//
// cs_submit_contingencies copies a request's element ids and queues it.  A
// scheduler thread per context keeps up to opt.serve_slots batches in flight,
// each on its own stream and workspace.  Whenever a slot is free it fills a
// batch of at most opt.batch_cap scenarios from the queue: the oldest request's
// next scenarios, then those of every later queued request for the same
// (network, level), in arrival order.  A request larger than what is left of
// the batch is split: its first scenarios go into this batch and the rest stay
// queued for the next free slot, so batches stay small enough to retire often
// and a request that arrives while others run gets a slot within about one
// batch time.  A request completes when its last slice is back.  Batches of
// different networks run side by side in different slots.  Before a batch starts, the device bytes it
// needs (workspace for its chunk size plus its id and record buffers) are
// checked against opt.hbm_budget together with everything the context
// already holds.  If they do not fit, the chunk is halved down to 64
// scenarios.  If it still does not fit, the batch waits for a running one to
// finish, or fails with CS_E_NOMEM when nothing else is running.  Finished
// batches are copied back through pinned staging and scattered into the
// requests, which cs_poll then hands to the caller.
#include <algorithm>
#include <chrono>
#include <cstring>

#include "ctx.h"

using namespace csi;

namespace {

constexpr int64_t kMinChunk = 64;

Slot* free_slot(cs_ctx* ctx) {
    for (auto& s : ctx->slots)
        if (!s->busy) return s.get();
    return nullptr;
}

bool any_busy(cs_ctx* ctx) {
    for (auto& s : ctx->slots)
        if (s->busy) return true;
    return false;
}

void fail_request(cs_ctx* ctx, uint64_t rid, cs_status st) {
    auto it = ctx->sreqs.find(rid);
    if (it == ctx->sreqs.end()) return;
    it->second->state = 3;
    it->second->err = st;
}

cudaError_t ensure_pinned(void** p, size_t* have, size_t want) {
    if (want <= *have) return cudaSuccess;
    if (*p) cudaFreeHost(*p);
    *p = nullptr;
    *have = 0;
    cudaError_t e = cudaMallocHost(p, want);
    if (e == cudaSuccess) *have = want;
    return e;
}

// Scatter a finished batch into its requests' slices.
void finish_batch(cs_ctx* ctx, Slot& sl, cudaError_t q) {
    cs_result b{};
    result_layout((char*)sl.h_out, sl.n, &b);
    for (const SliceRef& m : sl.members) {
        auto it = ctx->sreqs.find(m.rid);
        if (it == ctx->sreqs.end()) continue;                // failed and already polled
        ServeReq& r = *it->second;
        if (r.state == 3) continue;
        if (q != cudaSuccess) {
            r.state = 3;
            r.err = CS_E_CUDA;
            continue;
        }
        const int64_t o = m.boff, ro = m.roff, n = m.cnt;
        cs_result d{};
        result_layout(r.out.data(), r.n, &d);
        std::memcpy(d.cost + ro, b.cost + o, 8 * n);
        std::memcpy(d.max_re + ro, b.max_re + o, 8 * n);
        std::memcpy(d.min_zeta + ro, b.min_zeta + o, 8 * n);
        std::memcpy(d.n_islands + ro, b.n_islands + o, 2 * n);
        std::memcpy(d.opf_iters + ro, b.opf_iters + o, 2 * n);
        std::memcpy(d.klass + ro, b.klass + o, n);
        std::memcpy(d.severe + ro, b.severe + o, n);
        std::memcpy(d.v_margin + ro, b.v_margin + o, 8 * n);
        std::memcpy(d.max_loading + ro, b.max_loading + o, 8 * n);
        std::memcpy(d.shed_mw + ro, b.shed_mw + o, 8 * n);
        std::memcpy(d.main_klass + ro, b.main_klass + o, n);
        r.done_n += n;
        if (r.done_n == r.n) {
            r.state = 2;
            ctx->stats.completed += 1;
        }
    }
    if (q != cudaSuccess) ctx->err = std::string("serving batch: ") + cudaGetErrorString(q);
    sl.members.clear();
    sl.busy = false;
}

// Drop from the queue every request that failed or has been handed out in full.
void prune_queue(cs_ctx* ctx) {
    ctx->queue.erase(std::remove_if(ctx->queue.begin(), ctx->queue.end(),
                                    [&](uint64_t q) {
                                        auto it = ctx->sreqs.find(q);
                                        return it == ctx->sreqs.end() || it->second->state == 3 ||
                                               it->second->next >= it->second->n;
                                    }),
                     ctx->queue.end());
}

// Form and launch one batch on slot sl.  Returns false when the oldest
// request has to wait for memory (admission), true otherwise.
bool launch_batch(cs_ctx* ctx, Slot& sl) {
    const uint64_t rid0 = ctx->queue.front();
    ServeReq* r0 = ctx->sreqs[rid0].get();
    auto nit = ctx->nets.find(r0->net_id);
    if (nit == ctx->nets.end()) {                             // cannot happen: unload refuses busy networks
        fail_request(ctx, rid0, CS_E_UNKNOWN_ID);
        ctx->queue.pop_front();
        return true;
    }
    Network* net = nit->second.get();
    // members: the oldest request's next scenarios, then later ones of the same
    // (network, level), the last one possibly split
    const int64_t cap = ctx->opt.batch_cap;
    std::vector<SliceRef> take;
    int64_t total = 0;
    for (uint64_t rid : ctx->queue) {
        ServeReq* r = ctx->sreqs[rid].get();
        if (r->net_id != r0->net_id || r->level != r0->level || r->state == 3) continue;
        const int64_t cnt = std::min<int64_t>(r->n - r->next, cap - total);
        if (cnt <= 0) {
            if (total >= cap) break;
            continue;
        }
        take.push_back(SliceRef{rid, total, r->next, cnt});
        total += cnt;
        if (total >= cap) break;
    }
    auto fail_taken = [&](cs_status st) {
        for (const SliceRef& m : take) fail_request(ctx, m.rid, st);
        ctx->stats.nomem += (int64_t)take.size();
        prune_queue(ctx);
    };
    // admission: everything else the context holds + this slot's needs
    int64_t chunk = std::min<int64_t>(default_chunk(ctx, *net), std::max<int64_t>(total, 1));
    const size_t io = sizeof(int32_t) * 2 * total + result_bytes(total);
    if (ctx->opt.hbm_budget > 0) {
        const size_t others = reserved_bytes(ctx) - sl.device_bytes();
        const size_t budget = (size_t)ctx->opt.hbm_budget;
        while (chunk > kMinChunk && others + workspace_bytes(ctx, *net, chunk) + io > budget) chunk /= 2;
        if (others + workspace_bytes(ctx, *net, chunk) + io > budget) {
            if (any_busy(ctx)) {
                ctx->stats.admission_waits += 1;
                return false;
            }
            fail_taken(CS_E_NOMEM);
            ctx->err = "serving batch does not fit hbm_budget";
            return true;
        }
        // this slot's buffers are re-made to size when they exceed what fits
        if (others + sl.device_bytes() > budget) {
            sl.ws.release();
            sl.d_in.release();
            sl.d_out.release();
        }
    }
    // stage ids, launch, copy records back
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t x) { if (e == cudaSuccess) e = x; return e == cudaSuccess; };
    ok(ensure_pinned(&sl.h_in, &sl.h_in_bytes, sizeof(int32_t) * 2 * std::max<int64_t>(total, 1)));
    ok(ensure_pinned(&sl.h_out, &sl.h_out_bytes, result_bytes(std::max<int64_t>(total, 1))));
    ok(sl.d_in.ensure(sizeof(int32_t) * 2 * std::max<int64_t>(total, 1)));
    ok(sl.d_out.ensure(result_bytes(std::max<int64_t>(total, 1))));
    if (e != cudaSuccess) {
        fail_taken(CS_E_NOMEM);
        return true;
    } else {
        int32_t* hi = (int32_t*)sl.h_in;
        sl.members.clear();
        for (const SliceRef& m : take) {
            ServeReq* r = ctx->sreqs[m.rid].get();
            std::memcpy(hi + m.boff, r->ei.data() + m.roff, sizeof(int32_t) * m.cnt);
            std::memcpy(hi + total + m.boff, r->ej.data() + m.roff, sizeof(int32_t) * m.cnt);
            sl.members.push_back(m);
            if (r->out.empty()) r->out.resize(result_bytes(r->n));
            r->state = 1;
            r->next += m.cnt;
        }
        sl.n = total;
        cs_result dr{};
        result_layout((char*)sl.d_out.p, total, &dr);
        const int32_t* di = (const int32_t*)sl.d_in.p;
        ok(cudaMemcpyAsync(sl.d_in.p, sl.h_in, sizeof(int32_t) * 2 * total, cudaMemcpyHostToDevice, sl.stream));
        cs_status st = CS_OK;
        if (e == cudaSuccess) {
            ctx->launches = 0;
            st = evaluate_impl(ctx, sl.ws, net, r0->level, di, di + total, total, &dr, sl.stream, true, chunk);
        }
        if (e == cudaSuccess && st == CS_OK) {
            ok(cudaMemcpyAsync(sl.h_out, sl.d_out.p, result_bytes(total), cudaMemcpyDeviceToHost, sl.stream));
            ok(cudaEventRecord(sl.done, sl.stream));
        }
        if (e != cudaSuccess || st != CS_OK) {
            for (const SliceRef& m : take) fail_request(ctx, m.rid, st != CS_OK ? st : CS_E_CUDA);
            sl.members.clear();
        } else {
            sl.busy = true;
            ctx->stats.batches += 1;
            ctx->stats.merged += (int64_t)take.size() - 1;
        }
    }
    prune_queue(ctx);
    ctx->stats.peak_reserved = std::max<int64_t>(ctx->stats.peak_reserved, (int64_t)reserved_bytes(ctx));
    return true;
}

void scheduler(cs_ctx* ctx) {
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(ctx->mu);
    while (!ctx->stop) {
        bool progress = false;
        for (auto& sp : ctx->slots) {
            if (!sp->busy) continue;
            const cudaError_t q = cudaEventQuery(sp->done);
            if (q == cudaErrorNotReady) continue;
            finish_batch(ctx, *sp, q);
            progress = true;
        }
        while (!ctx->queue.empty()) {
            Slot* sl = free_slot(ctx);
            if (!sl || !launch_batch(ctx, *sl)) break;
            progress = true;
        }
        if (progress) ctx->cv_done.notify_all();
        if (ctx->stop) break;
        if (any_busy(ctx))
            ctx->cv_sched.wait_for(lk, std::chrono::microseconds(100));     // poll the batches in flight
        else if (!progress)
            ctx->cv_sched.wait(lk, [&] { return ctx->stop || !ctx->queue.empty(); });
    }
}

cs_status start_scheduler(cs_ctx* ctx) {
    if (ctx->sched.joinable()) return CS_OK;
    for (int k = 0; k < ctx->opt.serve_slots; ++k) {
        std::unique_ptr<Slot> sl(new Slot());
        CS_CUDA(cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking));
        CS_CUDA(cudaEventCreateWithFlags(&sl->done, cudaEventDisableTiming));
        ctx->slots.push_back(std::move(sl));
    }
    ctx->stop = false;
    ctx->sched = std::thread(scheduler, ctx);
    return CS_OK;
}

}  // namespace

namespace csi {

void serve_shutdown(cs_ctx* ctx) {
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->stop = true;
    }
    ctx->cv_sched.notify_all();
    if (ctx->sched.joinable()) ctx->sched.join();
}

bool serve_uses_network(cs_ctx* ctx, int net_id) {
    for (auto& kv : ctx->sreqs)
        if (kv.second->net_id == net_id && kv.second->state < 2) return true;
    return false;
}

}  // namespace csi

extern "C" {

cs_status cs_submit_contingencies(cs_ctx* ctx, int32_t net_id, int32_t level, const int32_t* ei, const int32_t* ej,
                                  int64_t n, uint64_t* request_id) {
    if (!ctx) return CS_E_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (!request_id || (n > 0 && (!ei || !ej))) return fail(ctx, CS_E_ARG, "NULL argument");
    auto it = ctx->nets.find(net_id);
    if (it == ctx->nets.end()) return fail(ctx, CS_E_UNKNOWN_ID, "unknown network");
    Network* net = it->second.get();
    if (level < 0 || level >= net->nlev) return fail(ctx, CS_E_ARG, "level out of range");
    if (n < 0 || n > (int64_t)1 << 31) return fail(ctx, CS_E_ARG, "n out of range");
    const int nE = net->dev.nE;
    for (int64_t q = 0; q < n; ++q) {
        const int a = ei[q], b = ej[q];
        if (a < -1 || a >= nE || b < -1 || b >= nE || (a < 0 && b >= 0))
            return fail(ctx, CS_E_ARG, "element id out of range at record " + std::to_string(q));
    }
    CS_CUDA(cudaSetDevice(ctx->device));
    if (start_scheduler(ctx) != CS_OK) return CS_E_CUDA;
    std::unique_ptr<ServeReq> r(new ServeReq());
    r->id = ctx->next_req++;
    r->net_id = net_id;
    r->level = level;
    r->n = n;
    r->ei.assign(ei, ei + n);
    r->ej.assign(ej, ej + n);
    *request_id = r->id;
    if (n == 0) {
        r->state = 2;
    } else {
        ctx->queue.push_back(r->id);
    }
    ctx->sreqs[r->id] = std::move(r);
    ctx->cv_sched.notify_all();
    return CS_OK;
}

cs_status cs_poll(cs_ctx* ctx, uint64_t request_id, int32_t timeout_us, const cs_result* out) {
    if (!ctx) return CS_E_ARG;
    std::unique_lock<std::mutex> lk(ctx->mu);
    auto it = ctx->sreqs.find(request_id);
    if (it == ctx->sreqs.end()) return fail(ctx, CS_E_UNKNOWN_ID, "unknown request");
    ServeReq* r = it->second.get();
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(std::max(0, timeout_us));
    while (r->state < 2) {
        if (ctx->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->state < 2) return CS_PENDING;
    }
    if (r->state == 3) {
        const cs_status st = r->err;
        ctx->sreqs.erase(it);
        return fail(ctx, st, "request failed");
    }
    const int64_t n = r->n;
    if (n > 0) {
        if (!out) return fail(ctx, CS_E_ARG, "NULL out");
        cs_result h{};
        result_layout(r->out.data(), n, &h);
        if (out->klass) std::memcpy(out->klass, h.klass, n);
        if (out->severe) std::memcpy(out->severe, h.severe, n);
        if (out->n_islands) std::memcpy(out->n_islands, h.n_islands, 2 * n);
        if (out->opf_iters) std::memcpy(out->opf_iters, h.opf_iters, 2 * n);
        if (out->cost) std::memcpy(out->cost, h.cost, 8 * n);
        if (out->max_re) std::memcpy(out->max_re, h.max_re, 8 * n);
        if (out->min_zeta) std::memcpy(out->min_zeta, h.min_zeta, 8 * n);
        if (out->v_margin) std::memcpy(out->v_margin, h.v_margin, 8 * n);
        if (out->max_loading) std::memcpy(out->max_loading, h.max_loading, 8 * n);
        if (out->shed_mw) std::memcpy(out->shed_mw, h.shed_mw, 8 * n);
        if (out->main_klass) std::memcpy(out->main_klass, h.main_klass, n);
    }
    ctx->sreqs.erase(it);
    return CS_OK;
}

cs_status cs_serving_stats(cs_ctx* ctx, int64_t* stats, int32_t n_stats) {
    if (!ctx || !stats || n_stats < 0) return CS_E_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    int64_t running = 0;
    for (auto& s : ctx->slots) running += s->busy ? 1 : 0;
    const int64_t v[9] = {ctx->stats.batches, ctx->stats.completed, ctx->stats.merged, ctx->stats.admission_waits,
                          ctx->stats.nomem, ctx->stats.peak_reserved, (int64_t)reserved_bytes(ctx),
                          (int64_t)ctx->queue.size(), running};
    for (int i = 0; i < n_stats && i < 9; ++i) stats[i] = v[i];
    return CS_OK;
}

}  // extern "C"
