// C ABI of libcs: context, network residency, evaluation, requests, Risk Index.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "ctx.h"

using namespace csi;

namespace csi {

cs_status fail(cs_ctx* c, cs_status st, const std::string& msg) {
    if (c) c->err = msg;
    return st;
}

cs_status cuda_fail(cs_ctx* c, cudaError_t e, const char* where) {
    return fail(c, CS_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

int64_t default_chunk(const cs_ctx* ctx, const Network& net) {
    if (ctx->opt.chunk > 0) return ctx->opt.chunk;
    // mixed form of a network whose state matrices go through the tensor-core reduction:
    // the chunk's padded matrices and reduction workspaces within about 6 GB
    if (ctx->opt.precision == CS_PREC_MIXED && !dyn_split_fits(net.dev, ctx->device)) {
        const size_t nmax = 5 * (size_t)net.dev.ng - 1;
        const size_t per = sizeof(float) * (dyn_abuf_stride(net.dev) + hess_tc_workspace_floats((int)nmax));
        return std::max<int64_t>(64, std::min<int64_t>(16384, (int64_t)(6e9 / (double)per)));
    }
    // Chunks alternate over two streams, so that one chunk's small-signal kernels run beside
    // the next one's OPF; a chunk must still give each of the OPF's resident CTAs (four per SM)
    // a dozen scenarios.  Measured on the 118-bus study (both levels, mixed form): 7,870 ms
    // with chunks of 4,096, 7,444 with 6,144, 7,400 with 8,192; on another box 7,540 with
    // 8,192, ~7,900 with 12,288 and with 16,384.
    return 8192;
}

namespace {
constexpr int kCounters = 6;      // work counters of one chunk: OPF, then five small-signal kernels
struct Grids {
    int g_opf, g_dyn;
    size_t per_opf, per_dyn;
};
constexpr int kDynCtasDefault = 2;
int cap_opf_of(const cs_ctx* ctx, const Network& net) {
    if (ctx->opt.ctas_per_sm > 0) return ctx->opt.ctas_per_sm;
    return net.opf_cap > 0 ? net.opf_cap : opf_ctas_per_sm();
}
int cap_dyn_of(const cs_ctx* ctx, const Network& net) {
    if (ctx->opt.ctas_per_sm > 0) return ctx->opt.ctas_per_sm;
    return net.dyn_cap > 0 ? net.dyn_cap : kDynCtasDefault;
}
Grids grids(const cs_ctx* ctx, const Network& net, int64_t cn) {
    // persistent kernels sized from occupancy, capped per SM (the network's tuned shape, if any)
    const DevNet& dn = net.dev;
    const int cap_opf = cap_opf_of(ctx, net);
    const int cap_dyn = cap_dyn_of(ctx, net);
    Grids g;
    g.g_opf = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)ctx->sms * cap_opf, cn));
    g.g_dyn = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)ctx->sms * cap_dyn, cn));
    g.per_opf = opf_scratch_doubles(dn);
    g.per_dyn = dyn_scratch_doubles(dn);
    return g;
}
bool split_path(const cs_ctx* ctx, const DevNet& dn) {
    return ctx->opt.precision == CS_PREC_MIXED && dyn_split_fits(dn, ctx->device);
}
bool large_path(const cs_ctx* ctx, const DevNet& dn) {
    return ctx->opt.precision == CS_PREC_MIXED && !dyn_split_fits(dn, ctx->device) && 5 * dn.ng - 1 >= 3;
}
}  // namespace

size_t workspace_bytes(const cs_ctx* ctx, const Network& net, int64_t chunk) {
    const DevNet& dn = net.dev;
    const int64_t cn = std::max<int64_t>(1, chunk);
    const Grids g = grids(ctx, net, cn);
    size_t b = std::max(g.per_opf * g.g_opf, g.per_dyn * g.g_dyn) * sizeof(double);
    b += sizeof(int) * cn + sizeof(double) * (2 * dn.nb + 2 * dn.ng) * cn + sizeof(int) * cn + sizeof(int) * kCounters;
    if (split_path(ctx, dn))
        b += (sizeof(float) * (dyn_hbuf_stride(dn) + dyn_abuf_stride(dn) + dyn_cand_stride()) +
              sizeof(double) * dyn_a64_stride(dn)) * cn;
    if (large_path(ctx, dn))
        b += sizeof(float) * (dyn_abuf_stride(dn) + hess_tc_workspace_floats(5 * dn.ng - 1)) * cn;
    return b;
}

size_t reserved_bytes(const cs_ctx* ctx) {
    size_t b = ctx->direct.bytes() + ctx->direct2.bytes() + ctx->err_word.bytes + ctx->hess_ws.bytes;
    for (auto& kv : ctx->nets) b += kv.second->resident_bytes();
    for (auto& sl : ctx->slots) b += sl->device_bytes();
    return b;
}

size_t result_bytes(int64_t n) { return (size_t)n * (8 * 6 + 2 + 2 + 1 + 1 + 1); }

cs_result result_at(const cs_result& r, int64_t c0, int nb) {
    cs_result o = r;
    o.klass = r.klass + c0;
    o.severe = r.severe + c0;
    o.n_islands = r.n_islands + c0;
    o.opf_iters = r.opf_iters + c0;
    o.cost = r.cost + c0;
    o.max_re = r.max_re + c0;
    o.min_zeta = r.min_zeta + c0;
    o.Vm = r.Vm ? r.Vm + c0 * nb : nullptr;
    o.Va = r.Va ? r.Va + c0 * nb : nullptr;
    o.v_margin = r.v_margin ? r.v_margin + c0 : nullptr;
    o.max_loading = r.max_loading ? r.max_loading + c0 : nullptr;
    o.shed_mw = r.shed_mw ? r.shed_mw + c0 : nullptr;
    o.main_klass = r.main_klass ? r.main_klass + c0 : nullptr;
    return o;
}

void result_layout(char* base, int64_t n, cs_result* r) {
    r->cost = (double*)base;                         // doubles first for alignment
    r->max_re = r->cost + n;
    r->min_zeta = r->max_re + n;
    r->v_margin = r->min_zeta + n;
    r->max_loading = r->v_margin + n;
    r->shed_mw = r->max_loading + n;
    r->n_islands = (int16_t*)(r->shed_mw + n);
    r->opf_iters = r->n_islands + n;
    r->klass = (uint8_t*)(r->opf_iters + n);
    r->severe = r->klass + n;
    r->main_klass = r->severe + n;
    r->Vm = nullptr;
    r->Va = nullptr;
}

}  // namespace csi

namespace {

// pack host vectors into one device blob
struct Packer {
    std::vector<char> host;
    size_t add(const void* src, size_t bytes) {
        size_t off = (host.size() + 255) & ~size_t(255);
        host.resize(off + std::max<size_t>(bytes, 1));
        if (bytes) std::memcpy(host.data() + off, src, bytes);
        return off;
    }
    template <class T>
    size_t add(const std::vector<T>& v) { return add(v.data(), v.size() * sizeof(T)); }
};

}  // namespace

cs_status csi::evaluate_impl(cs_ctx* ctx, Workspace& ws, Network* net, int level, const int32_t* ei,
                             const int32_t* ej, int64_t n, const cs_result* out, cudaStream_t s, bool record,
                             int64_t chunk, const int32_t* ek) {
    if (n <= 0) return CS_OK;
    const DevNet& dn = net->dev;
    const int nx = 2 * dn.nb + 2 * dn.ng;
    chunk = std::max<int64_t>(1, chunk);
    const int64_t cn = std::min<int64_t>(n, chunk);
    const Grids gr = grids(ctx, *net, cn);
    const int g_opf = gr.g_opf, g_dyn = gr.g_dyn;
    const size_t per_opf = gr.per_opf, per_dyn = gr.per_dyn;
    const size_t need = std::max(per_opf * g_opf, per_dyn * g_dyn) * sizeof(double);
    CS_CUDA(ws.scratch.ensure(need));
    CS_CUDA(ws.isl.ensure(sizeof(int) * cn));
    CS_CUDA(ws.opfx.ensure(sizeof(double) * nx * cn));
    CS_CUDA(ws.opfst.ensure(sizeof(int) * cn));
    CS_CUDA(ws.counters.ensure(sizeof(int) * kCounters));
    // balanced and packed Hessenberg matrices between the kernels of the FP32 screen
    const bool split = split_path(ctx, dn);
    if (split) {
        CS_CUDA(ws.hbuf.ensure(sizeof(float) * dyn_hbuf_stride(dn) * cn));
        CS_CUDA(ws.abuf.ensure(sizeof(float) * dyn_abuf_stride(dn) * cn));
        CS_CUDA(ws.a64.ensure(sizeof(double) * dyn_a64_stride(dn) * cn));
        CS_CUDA(ws.cand.ensure(sizeof(float) * dyn_cand_stride() * cn));
    }
    const bool large = large_path(ctx, dn);
    if (large) {
        CS_CUDA(ws.abuf.ensure(sizeof(float) * dyn_abuf_stride(dn) * cn));
        CS_CUDA(ws.hws.ensure(sizeof(float) * hess_tc_workspace_floats(5 * dn.ng - 1) * cn));
    }
    if (!ctx->err_word.p) {
        CS_CUDA(ctx->err_word.ensure(sizeof(int) * 2));
        CS_CUDA(cudaMemset(ctx->err_word.p, 0, sizeof(int) * 2));
    }
    int* counters = (int*)ws.counters.p;
    if (!ws.free) CS_CUDA(cudaEventCreateWithFlags(&ws.free, cudaEventDisableTiming));
    if (ws.used) CS_CUDA(cudaStreamWaitEvent(s, ws.free, 0));
    for (int64_t c0 = 0; c0 < n; c0 += chunk) {
        const int64_t m = std::min(chunk, n - c0);
        EvalArgs a{};
        a.ei = ei + c0;
        a.ej = ej + c0;
        a.ek = ek ? ek + c0 : nullptr;
        a.n = (int)m;
        a.level = level;
        a.out = result_at(*out, c0, dn.nb);
        a.main_island = ctx->opt.main_island != 0;
        a.sev_n1 = record ? (uint8_t*)net->sev_n1[level]->p : nullptr;
        a.sev_pairs = record ? (uint8_t*)net->sev_pairs[level]->p : nullptr;
        a.err = (int*)ctx->err_word.p;
        a.reruns = (int*)ctx->err_word.p + 1;
        OpfOut o{(double*)ws.opfx.p, (int*)ws.opfst.p};
        CS_CUDA(cudaMemsetAsync(counters, 0, sizeof(int) * kCounters, s));
        auto mark = [&](int kind) -> cudaError_t {     // start event of a timed launch
            if (!ctx->timing) return cudaSuccess;
            while (ctx->ev.size() < 2 * (ctx->ev_used + 1)) {
                cudaEvent_t e;
                cudaError_t r = cudaEventCreate(&e);
                if (r != cudaSuccess) return r;
                ctx->ev.push_back(e);
            }
            if ((int)ctx->ev_kind.size() <= (int)ctx->ev_used) ctx->ev_kind.resize(ctx->ev_used + 1);
            ctx->ev_kind[ctx->ev_used] = kind;
            return cudaEventRecord(ctx->ev[2 * ctx->ev_used], s);
        };
        auto done = [&]() -> cudaError_t {
            if (!ctx->timing) return cudaSuccess;
            cudaError_t r = cudaEventRecord(ctx->ev[2 * ctx->ev_used + 1], s);
            ctx->ev_used++;
            return r;
        };
        CS_CUDA(mark(0));
        CS_CUDA(launch_islands(dn, a, (int*)ws.isl.p, s));
        CS_CUDA(done());
        CS_CUDA(mark(1));
        CS_CUDA(launch_opf(dn, a, (const int*)ws.isl.p, o, ctx->opt.opf_tol, net->max_it,
                           (double*)ws.scratch.p, per_opf, std::min<int64_t>(g_opf, m), counters, s));
        CS_CUDA(done());
        CS_CUDA(mark(2));
        int nl = 0;
        CS_CUDA(launch_dyn(dn, a, o, ctx->opt.damping_min, ctx->opt.precision, (double*)ws.scratch.p, per_dyn,
                           std::min<int64_t>(g_dyn, m), (split || large) ? (float*)ws.abuf.p : nullptr,
                           split ? (float*)ws.hbuf.p : nullptr, split ? (double*)ws.a64.p : nullptr,
                           split ? (float*)ws.cand.p : nullptr, large ? (float*)ws.hws.p : nullptr, ctx->sms,
                           counters + 1, &nl, s));
        CS_CUDA(done());
        ctx->launches += 2 + nl;
    }
    CS_CUDA(cudaEventRecord(ws.free, s));
    ws.used = true;
    return CS_OK;
}

extern "C" {

void cs_default_options(cs_options* o) {
    if (!o) return;
    o->device = 0;
    o->damping_min = 0.05;
    o->opf_tol = 1e-8;
    o->opf_max_it = 50;
    o->require_secure_base = 0;
    o->ctas_per_sm = 0;
    o->chunk = 0;
    o->precision = CS_PREC_FP64;
    o->hbm_budget = 0;
    o->serve_slots = 3;
    o->batch_cap = 4096;
    o->main_island = 0;
    o->autotune = 0;
}

cs_status cs_create(const cs_options* opt, cs_ctx** out) {
    if (!out) return CS_E_ARG;
    *out = nullptr;
    std::unique_ptr<cs_ctx> c(new cs_ctx());
    if (opt) c->opt = *opt; else cs_default_options(&c->opt);
    if (c->opt.opf_max_it < 0 || c->opt.opf_max_it > 10000 || !(c->opt.opf_tol > 0.0)) return CS_E_ARG;
    if (c->opt.precision != CS_PREC_FP64 && c->opt.precision != CS_PREC_MIXED) return CS_E_ARG;
    if (c->opt.hbm_budget < 0 || c->opt.serve_slots < 1 || c->opt.serve_slots > 8 || c->opt.batch_cap < 1)
        return CS_E_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) return CS_E_CUDA;
    if (c->opt.device < 0 || c->opt.device >= ndev) return CS_E_ARG;
    c->device = c->opt.device;
    if (cudaSetDevice(c->device) != cudaSuccess) return CS_E_CUDA;
    if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) return CS_E_CUDA;
    if (cudaStreamCreateWithFlags(&c->req_stream, cudaStreamNonBlocking) != cudaSuccess) return CS_E_CUDA;
    if (cudaStreamCreateWithFlags(&c->aux_stream, cudaStreamNonBlocking) != cudaSuccess) return CS_E_CUDA;
    if (cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) != cudaSuccess) return CS_E_CUDA;
    if (cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming) != cudaSuccess) return CS_E_CUDA;
    *out = c.release();
    return CS_OK;
}

cs_status cs_destroy(cs_ctx* ctx) {
    if (!ctx) return CS_E_ARG;
    serve_shutdown(ctx);
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    ctx->sreqs.clear();
    ctx->slots.clear();
    ctx->nets.clear();
    for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
    if (ctx->req_stream) cudaStreamDestroy(ctx->req_stream);
    if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
    delete ctx;
    return CS_OK;
}

const char* cs_last_error(cs_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int64_t cs_last_launch_count(cs_ctx* ctx) { return ctx ? ctx->launches : 0; }

cs_status cs_eigen_reruns(cs_ctx* ctx, int64_t* count) {
    if (!ctx || !count) return CS_E_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    *count = 0;
    if (!ctx->err_word.p) return CS_OK;
    CS_CUDA(cudaDeviceSynchronize());
    int v = 0;
    CS_CUDA(cudaMemcpy(&v, (int*)ctx->err_word.p + 1, sizeof(int), cudaMemcpyDeviceToHost));
    *count = v;
    return CS_OK;
}

cs_status cs_set_timing(cs_ctx* ctx, int32_t enable) {
    if (!ctx) return CS_E_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    ctx->timing = enable != 0;
    ctx->ev_used = 0;
    for (int k = 0; k < 3; ++k) { ctx->kernel_ms[k] = 0.0; ctx->kernel_launches[k] = 0; }
    return CS_OK;
}

cs_status cs_kernel_times(cs_ctx* ctx, double* ms, int64_t* launches) {
    if (!ctx || !ms) return CS_E_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    for (size_t q = 0; q < ctx->ev_used; ++q) {
        CS_CUDA(cudaEventSynchronize(ctx->ev[2 * q + 1]));
        float t = 0.f;
        CS_CUDA(cudaEventElapsedTime(&t, ctx->ev[2 * q], ctx->ev[2 * q + 1]));
        ctx->kernel_ms[ctx->ev_kind[q]] += t;
        ctx->kernel_launches[ctx->ev_kind[q]] += 1;
    }
    ctx->ev_used = 0;
    for (int k = 0; k < 3; ++k) {
        ms[k] = ctx->kernel_ms[k];
        if (launches) launches[k] = ctx->kernel_launches[k];
    }
    return CS_OK;
}

}  // extern "C"

namespace {
// Host-side checks of a network descriptor (no device): sizes, indices, and every
// value the method needs finite and in range.  Returns an empty string when valid.
std::string check_desc(const cs_network_desc* d) {
    if (!d) return "NULL network descriptor";
    const int nb = d->n_bus, nbr = d->n_branch, ng = d->n_gen, nlev = d->n_levels;
    if (nb <= 0 || nbr < 0 || ng <= 0 || nlev <= 0 || d->ref_bus < 0 || d->ref_bus >= nb ||
        !(d->base_mva > 0) || !std::isfinite(d->base_mva) || !(d->f_hz > 0) || !std::isfinite(d->f_hz))
        return "invalid sizes, reference bus, base or frequency";
    const void* req[] = {d->Vmin, d->Vmax, d->Gs, d->Bs, d->Pd, d->Qd, d->f, d->t, d->r, d->x, d->b, d->rate,
                         d->tap, d->gbus, d->Pmin, d->Pmax, d->Qmin, d->Qmax, d->c2, d->c1, d->c0, d->H, d->D,
                         d->xd, d->xq, d->xdp, d->Td0p, d->Tq0p, d->KA, d->TA};
    for (const void* p : req)
        if (!p) return "NULL array in network descriptor";
    if ((long long)nbr + ng > 32767) return "too many outage elements";
    if (d->opf_max_it < 0 || d->opf_max_it > 10000) return "interior-point iteration cap outside 0..10000";
    auto fin = [](double v) { return std::isfinite(v); };
    for (int i = 0; i < nb; ++i) {
        if (!fin(d->Vmin[i]) || !fin(d->Vmax[i]) || !(d->Vmin[i] > 0) || !(d->Vmin[i] <= d->Vmax[i]))
            return "bus " + std::to_string(i) + ": voltage bounds not finite or not 0 < Vmin <= Vmax";
        if (!fin(d->Gs[i]) || !fin(d->Bs[i])) return "bus " + std::to_string(i) + ": shunt not finite";
    }
    for (long long q = 0; q < (long long)nlev * nb; ++q)
        if (!fin(d->Pd[q]) || !fin(d->Qd[q]))
            return "load level " + std::to_string(q / nb) + ", bus " + std::to_string(q % nb) + ": load not finite";
    for (int k = 0; k < nbr; ++k) {
        if (d->f[k] < 0 || d->f[k] >= nb || d->t[k] < 0 || d->t[k] >= nb || d->f[k] == d->t[k])
            return "branch " + std::to_string(k) + ": end out of range or self loop";
        if (!fin(d->r[k]) || !fin(d->x[k]) || !fin(d->b[k]) || !(std::fabs(d->r[k]) + std::fabs(d->x[k]) > 0))
            return "branch " + std::to_string(k) + ": impedance zero or not finite";
        if (!(d->rate[k] > 0) || !fin(d->rate[k]) || !(d->tap[k] > 0) || !fin(d->tap[k]))
            return "branch " + std::to_string(k) + ": rating or tap not positive and finite";
    }
    for (int k = 0; k < ng; ++k) {
        if (d->gbus[k] < 0 || d->gbus[k] >= nb) return "generator " + std::to_string(k) + ": bus out of range";
        const double v[] = {d->Pmin[k], d->Pmax[k], d->Qmin[k], d->Qmax[k], d->c2[k], d->c1[k], d->c0[k],
                            d->H[k], d->D[k], d->xd[k], d->xq[k], d->xdp[k], d->Td0p[k], d->Tq0p[k], d->KA[k],
                            d->TA[k]};
        for (double x : v)
            if (!fin(x)) return "generator " + std::to_string(k) + ": a value is not finite";
        if (!(d->Pmax[k] > 0) || !(d->Pmin[k] <= d->Pmax[k]) || !(d->Qmin[k] <= d->Qmax[k]) || d->c2[k] < 0)
            return "generator " + std::to_string(k) + ": limits or cost invalid";
        if (!(d->xdp[k] > 0) || !(d->xd[k] > 0) || !(d->xq[k] > 0) || !(d->H[k] > 0) || d->D[k] < 0 ||
            !(d->Td0p[k] > 0) || !(d->Tq0p[k] > 0) || !(d->TA[k] > 0) || !(d->KA[k] > 0))
            return "generator " + std::to_string(k) + ": machine data invalid";
    }
    return std::string();
}
// Launch-shape autotuner: resident OPF blocks per SM (1..the register limit) and
// resident small-signal blocks per SM (1, 2, 4), timed with the per-kernel events
// on a sample of the network's pairs (up to 3 blocks' worth per SM, spread evenly
// over the pair range, level 0, not recorded).  Shapes are tried in pairs (the two
// kernel groups are timed separately in each run); the fastest of each group is
// kept.  Results do not depend on the shape.
cs_status autotune_network(cs_ctx* ctx, Network* net) {
    const int64_t nE = net->dev.nE;
    const int64_t npairs = nE * (nE - 1) / 2;
    const int64_t ns = std::min<int64_t>(npairs, (int64_t)ctx->sms * 3);
    if (ns <= 0) return CS_OK;
    std::vector<int32_t> ids(2 * ns);
    for (int64_t q = 0, k = 0, i = 0; i < nE && q < ns; ++i)      // pair k = q * npairs / ns
        for (int64_t j = i + 1; j < nE && q < ns; ++j, ++k)
            if (k == q * npairs / ns) {
                ids[q] = (int32_t)i;
                ids[ns + q] = (int32_t)j;
                ++q;
            }
    DevBuf dids, dres;
    CS_CUDA(dids.ensure(sizeof(int32_t) * 2 * ns));
    CS_CUDA(cudaMemcpy(dids.p, ids.data(), sizeof(int32_t) * 2 * ns, cudaMemcpyHostToDevice));
    CS_CUDA(dres.ensure(result_bytes(ns)));
    cs_result r{};
    result_layout((char*)dres.p, ns, &r);
    const int opf_max = opf_ctas_per_sm();
    const int dyn_try[3] = {1, 2, 4};
    const int tries = std::max(opf_max, 3);
    double best_opf = 1e300, best_dyn = 1e300;
    int pick_opf = opf_max, pick_dyn = kDynCtasDefault;
    const bool was_timing = ctx->timing;
    for (int t = -1; t < tries; ++t) {                 // t = -1: warm-up with the defaults
        net->opf_cap = (t < 0) ? opf_max : 1 + (t % opf_max);
        net->dyn_cap = (t < 0) ? kDynCtasDefault : dyn_try[t % 3];
        ctx->timing = true;
        ctx->ev_used = 0;
        cs_status st = evaluate_impl(ctx, ctx->direct, net, 0, (const int32_t*)dids.p, (const int32_t*)dids.p + ns,
                                     ns, &r, ctx->req_stream, false, ns);
        ctx->timing = was_timing;
        if (st != CS_OK) return st;
        CS_CUDA(cudaStreamSynchronize(ctx->req_stream));
        double ms[3] = {0.0, 0.0, 0.0};
        for (size_t q = 0; q < ctx->ev_used; ++q) {
            float e = 0.f;
            CS_CUDA(cudaEventElapsedTime(&e, ctx->ev[2 * q], ctx->ev[2 * q + 1]));
            ms[ctx->ev_kind[q]] += e;
        }
        ctx->ev_used = 0;
        if (t < 0) continue;
        if (ms[1] < best_opf) { best_opf = ms[1]; pick_opf = net->opf_cap; }
        if (ms[2] < best_dyn) { best_dyn = ms[2]; pick_dyn = net->dyn_cap; }
    }
    net->opf_cap = pick_opf;
    net->dyn_cap = pick_dyn;
    return CS_OK;
}

}  // namespace

extern "C" {

cs_status cs_check_network(const cs_network_desc* d, char* msg, int32_t msg_len) {
    const std::string m = check_desc(d);
    if (msg && msg_len > 0) {
        const size_t n = std::min<size_t>(m.size(), (size_t)msg_len - 1);
        std::memcpy(msg, m.data(), n);
        msg[n] = '\0';
    }
    return m.empty() ? CS_OK : CS_E_ARG;
}

cs_status cs_load_network(cs_ctx* ctx, const cs_network_desc* d, int32_t* net_id) {
    if (!ctx) return CS_E_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (!d || !net_id) return fail(ctx, CS_E_ARG, "NULL argument");
    {
        const std::string m = check_desc(d);
        if (!m.empty()) return fail(ctx, CS_E_ARG, m);
    }
    const int nb = d->n_bus, nbr = d->n_branch, ng = d->n_gen, nlev = d->n_levels;
    CS_CUDA(cudaSetDevice(ctx->device));
    std::unique_ptr<Network> net(new Network());
    net->max_it = d->opf_max_it > 0 ? d->opf_max_it : ctx->opt.opf_max_it;
    std::vector<int> f(d->f, d->f + nbr), t(d->t, d->t + nbr);
    std::string msg = symbolic_analysis(nb, f, t, d->ref_bus, net->sym);
    if (!msg.empty()) return fail(ctx, CS_E_ARG, msg);
    const Symbolic& S = net->sym;
    const double B = d->base_mva;
    // per-unit conversion and branch two-port admittances
    std::vector<cplx> yff(nbr), yft(nbr), ytf(nbr), ytt(nbr);
    std::vector<double> smax2(nbr);
    for (int k = 0; k < nbr; ++k) {
        const double r = d->r[k], x = d->x[k], den = r * r + x * x;
        const cplx ys = cm(r / den, -x / den);
        const cplx yt = ys + cm(0.0, 0.5 * d->b[k]);
        const double tap = d->tap[k];
        ytt[k] = yt;
        yff[k] = (1.0 / (tap * tap)) * yt;
        yft[k] = (-1.0 / tap) * ys;
        ytf[k] = (-1.0 / tap) * ys;
        smax2[k] = (d->rate[k] / B) * (d->rate[k] / B);
    }
    std::vector<double> gsh(nb), bsh(nb), Pd((size_t)nlev * nb), Qd((size_t)nlev * nb);
    for (int i = 0; i < nb; ++i) {
        gsh[i] = d->Gs[i] / B;
        bsh[i] = d->Bs[i] / B;
    }
    for (size_t q = 0; q < (size_t)nlev * nb; ++q) {
        Pd[q] = d->Pd[q] / B;
        Qd[q] = d->Qd[q] / B;
    }
    std::vector<double> pmin(ng), pmax(ng), qmin(ng), qmax(ng), xd(ng), xq(ng), xp(ng), H2(ng), Dm(ng);
    for (int k = 0; k < ng; ++k) {
        pmin[k] = d->Pmin[k] / B;
        pmax[k] = d->Pmax[k] / B;
        qmin[k] = d->Qmin[k] / B;
        qmax[k] = d->Qmax[k] / B;
        const double zb = B / d->Pmax[k];       // machine base (MVA = Pmax) -> system base
        xd[k] = d->xd[k] * zb;
        xq[k] = d->xq[k] * zb;
        xp[k] = d->xdp[k] * zb;
        H2[k] = 2.0 * d->H[k] / zb;
        Dm[k] = d->D[k] / zb;
    }
    // incidence
    std::vector<int> bus_br_ptr(nb + 1, 0), bus_br(2 * nbr), bus_gen_ptr(nb + 1, 0), bus_gen(ng);
    for (int k = 0; k < nbr; ++k) { bus_br_ptr[f[k] + 1]++; bus_br_ptr[t[k] + 1]++; }
    for (int i = 0; i < nb; ++i) bus_br_ptr[i + 1] += bus_br_ptr[i];
    {
        std::vector<int> fill(bus_br_ptr.begin(), bus_br_ptr.end() - 1);
        for (int k = 0; k < nbr; ++k) {
            bus_br[fill[f[k]]++] = 2 * k;
            bus_br[fill[t[k]]++] = 2 * k + 1;
        }
    }
    for (int k = 0; k < ng; ++k) bus_gen_ptr[d->gbus[k] + 1]++;
    for (int i = 0; i < nb; ++i) bus_gen_ptr[i + 1] += bus_gen_ptr[i];
    {
        std::vector<int> fill(bus_gen_ptr.begin(), bus_gen_ptr.end() - 1);
        for (int k = 0; k < ng; ++k) bus_gen[fill[d->gbus[k]]++] = k;
    }
    auto vec = [](const double* p, int cnt) { return std::vector<double>(p, p + cnt); };
    Packer P;
    size_t o_f = P.add(f), o_t = P.add(t), o_yff = P.add(yff), o_yft = P.add(yft), o_ytf = P.add(ytf),
           o_ytt = P.add(ytt), o_smax2 = P.add(smax2);
    size_t o_vmin = P.add(vec(d->Vmin, nb)), o_vmax = P.add(vec(d->Vmax, nb)), o_gsh = P.add(gsh), o_bsh = P.add(bsh),
           o_Pd = P.add(Pd), o_Qd = P.add(Qd);
    std::vector<int> gbus(d->gbus, d->gbus + ng);
    size_t o_gbus = P.add(gbus), o_pmin = P.add(pmin), o_pmax = P.add(pmax), o_qmin = P.add(qmin),
           o_qmax = P.add(qmax), o_c2 = P.add(vec(d->c2, ng)), o_c1 = P.add(vec(d->c1, ng)), o_c0 = P.add(vec(d->c0, ng));
    size_t o_xd = P.add(xd), o_xq = P.add(xq), o_xp = P.add(xp), o_Td0 = P.add(vec(d->Td0p, ng)),
           o_Tq0 = P.add(vec(d->Tq0p, ng)), o_KA = P.add(vec(d->KA, ng)), o_TA = P.add(vec(d->TA, ng)),
           o_H2 = P.add(H2), o_Dm = P.add(Dm);
    size_t o_bbp = P.add(bus_br_ptr), o_bb = P.add(bus_br), o_bgp = P.add(bus_gen_ptr), o_bg = P.add(bus_gen);
    size_t o_perm = P.add(S.perm), o_iperm = P.add(S.iperm), o_Lcp = P.add(S.Lcolptr), o_Lr = P.add(S.Lrow),
           o_Lc = P.add(S.Lcol), o_Lrp = P.add(S.Lrowptr), o_Lrc = P.add(S.Lrowcol), o_Lrb = P.add(S.Lrowblk),
           o_lp = P.add(S.lev_ptr), o_lc = P.add(S.lev_col), o_tp = P.add(S.tgt_ptr), o_tg = P.add(S.tgt),
           o_up = P.add(S.upd_ptr), o_ua = P.add(S.upd_a), o_ub = P.add(S.upd_b), o_bbrp = P.add(S.blk_br_ptr),
           o_bbr = P.add(S.blk_br);
    if (ctx->opt.hbm_budget > 0) {                    // admission by device footprint
        const int64_t ne = (int64_t)nbr + ng;
        const size_t add = P.host.size() + (size_t)nlev * (size_t)(ne + ne * (ne - 1) / 2);
        if (reserved_bytes(ctx) + add > (size_t)ctx->opt.hbm_budget)
            return fail(ctx, CS_E_NOMEM, "network would exceed hbm_budget: " + std::to_string(reserved_bytes(ctx) + add) +
                                             " > " + std::to_string(ctx->opt.hbm_budget) + " bytes");
    }
    CS_CUDA(net->blob.ensure(P.host.size()));
    CS_CUDA(cudaMemcpy(net->blob.p, P.host.data(), P.host.size(), cudaMemcpyHostToDevice));
    char* base = (char*)net->blob.p;
    DevNet& dn = net->dev;
    dn.nb = nb; dn.nbr = nbr; dn.ng = ng; dn.nlev = nlev; dn.ref = d->ref_bus;
    dn.base = B; dn.ws = 2.0 * M_PI * d->f_hz; dn.nE = nbr + ng;
#define P_(T, o) ((const T*)(base + (o)))
    dn.f = P_(int, o_f); dn.t = P_(int, o_t);
    dn.yff = P_(cplx, o_yff); dn.yft = P_(cplx, o_yft); dn.ytf = P_(cplx, o_ytf); dn.ytt = P_(cplx, o_ytt);
    dn.smax2 = P_(double, o_smax2);
    dn.vmin = P_(double, o_vmin); dn.vmax = P_(double, o_vmax); dn.gsh = P_(double, o_gsh); dn.bsh = P_(double, o_bsh);
    dn.Pd = P_(double, o_Pd); dn.Qd = P_(double, o_Qd);
    dn.gbus = P_(int, o_gbus); dn.pmin = P_(double, o_pmin); dn.pmax = P_(double, o_pmax);
    dn.qmin = P_(double, o_qmin); dn.qmax = P_(double, o_qmax);
    dn.c2 = P_(double, o_c2); dn.c1 = P_(double, o_c1); dn.c0 = P_(double, o_c0);
    dn.xd = P_(double, o_xd); dn.xq = P_(double, o_xq); dn.xp = P_(double, o_xp); dn.Td0 = P_(double, o_Td0);
    dn.Tq0 = P_(double, o_Tq0); dn.KA = P_(double, o_KA); dn.TA = P_(double, o_TA); dn.H2 = P_(double, o_H2);
    dn.Dm = P_(double, o_Dm);
    dn.bus_br_ptr = P_(int, o_bbp); dn.bus_br = P_(int, o_bb); dn.bus_gen_ptr = P_(int, o_bgp); dn.bus_gen = P_(int, o_bg);
    dn.nL = (int)S.Lrow.size();
    dn.perm = P_(int, o_perm); dn.iperm = P_(int, o_iperm); dn.Lcolptr = P_(int, o_Lcp); dn.Lrow = P_(int, o_Lr);
    dn.Lcol = P_(int, o_Lc); dn.Lrowptr = P_(int, o_Lrp); dn.Lrowcol = P_(int, o_Lrc); dn.Lrowblk = P_(int, o_Lrb);
    dn.nlevels = S.nlevels; dn.lev_ptr = P_(int, o_lp); dn.lev_col = P_(int, o_lc); dn.tgt_ptr = P_(int, o_tp);
    dn.tgt = P_(int, o_tg); dn.upd_ptr = P_(int, o_up); dn.upd_a = P_(int, o_ua); dn.upd_b = P_(int, o_ub);
    dn.blk_br_ptr = P_(int, o_bbrp); dn.blk_br = P_(int, o_bbr);
#undef P_
    // severity tables, one per level, 255 = not evaluated
    const int64_t nE = nbr + ng;
    const int64_t npairs = nE * (nE - 1) / 2;
    net->nlev = nlev;
    for (int l = 0; l < nlev; ++l) {
        net->sev_n1.emplace_back(new DevBuf());
        net->sev_pairs.emplace_back(new DevBuf());
        CS_CUDA(net->sev_n1[l]->ensure(std::max<int64_t>(nE, 1)));
        CS_CUDA(net->sev_pairs[l]->ensure(std::max<int64_t>(npairs, 1)));
        CS_CUDA(cudaMemset(net->sev_n1[l]->p, 0xff, std::max<int64_t>(nE, 1)));
        CS_CUDA(cudaMemset(net->sev_pairs[l]->p, 0xff, std::max<int64_t>(npairs, 1)));
    }
    // base case of every level (Section II-A step 1)
    {
        DevBuf din, dout;
        CS_CUDA(din.ensure(2 * sizeof(int)));
        const int m1[2] = {-1, -1};
        CS_CUDA(cudaMemcpy(din.p, m1, sizeof(m1), cudaMemcpyHostToDevice));
        const size_t rec = 1 + 1 + 2 + 2 + 8 * 3;
        CS_CUDA(dout.ensure(64 + rec));
        char* ob = (char*)dout.p;
        cs_result r{};
        r.cost = (double*)(ob + 0);
        r.max_re = (double*)(ob + 8);
        r.min_zeta = (double*)(ob + 16);
        r.n_islands = (int16_t*)(ob + 24);
        r.opf_iters = (int16_t*)(ob + 26);
        r.klass = (uint8_t*)(ob + 28);
        r.severe = (uint8_t*)(ob + 29);
        for (int l = 0; l < nlev; ++l) {
            cs_status st = evaluate_impl(ctx, ctx->direct, net.get(), l, (const int*)din.p, (const int*)din.p + 1, 1,
                                         &r, 0, false, 1);
            if (st != CS_OK) return st;
            CS_CUDA(cudaDeviceSynchronize());
            char hb[32];
            CS_CUDA(cudaMemcpy(hb, ob, 30, cudaMemcpyDeviceToHost));
            double c, mr, mz;
            int16_t isl, it;
            std::memcpy(&c, hb, 8);
            std::memcpy(&mr, hb + 8, 8);
            std::memcpy(&mz, hb + 16, 8);
            std::memcpy(&isl, hb + 24, 2);
            std::memcpy(&it, hb + 26, 2);
            net->base_cost.push_back(c);
            net->base_maxre.push_back(mr);
            net->base_minz.push_back(mz);
            net->base_isl.push_back(isl);
            net->base_iters.push_back(it);
            net->base_klass.push_back((uint8_t)hb[28]);
            net->base_severe.push_back((uint8_t)hb[29]);
            if (ctx->opt.require_secure_base && hb[29])
                return fail(ctx, CS_E_BASE_INSECURE, "base case of level " + std::to_string(l) + " is not secure");
        }
    }
    if (ctx->opt.autotune && ctx->opt.ctas_per_sm == 0) {
        cs_status st = autotune_network(ctx, net.get());
        if (st != CS_OK) return st;
    }
    const int id = ctx->next_net++;
    net->id = id;
    ctx->nets[id] = std::move(net);
    *net_id = id;
    return CS_OK;
}

cs_status cs_unload_network(cs_ctx* ctx, int32_t net_id) {
    if (!ctx) return CS_E_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    auto it = ctx->nets.find(net_id);
    if (it == ctx->nets.end()) return fail(ctx, CS_E_UNKNOWN_ID, "unknown network");
    if (serve_uses_network(ctx, net_id)) return fail(ctx, CS_E_ARG, "network has queued or running requests");
    if (it->second->busy > 0) return fail(ctx, CS_E_ARG, "network is in use by a Risk Index call");
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    ctx->nets.erase(it);
    return CS_OK;
}

cs_status cs_network_stats(cs_ctx* ctx, int32_t net_id, int64_t* stats, int32_t n_stats) {
    if (!ctx) return CS_E_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    auto it = ctx->nets.find(net_id);
    if (it == ctx->nets.end()) return fail(ctx, CS_E_UNKNOWN_ID, "unknown network");
    if (!stats || n_stats < 0) return fail(ctx, CS_E_ARG, "NULL stats");
    const DevNet& d = it->second->dev;
    const Symbolic& S = it->second->sym;
    const int64_t v[12] = {d.nb, d.nbr, d.ng, d.nL, (int64_t)S.upd_a.size(), d.nlevels, 5LL * d.ng - 1,
                           (int64_t)it->second->nlev, cap_opf_of(ctx, *it->second), cap_dyn_of(ctx, *it->second),
                           (ctx->opt.ctas_per_sm == 0 && it->second->opf_cap > 0) ? 1 : 0, it->second->max_it};
    for (int i = 0; i < n_stats && i < 12; ++i) stats[i] = v[i];
    return CS_OK;
}

cs_status cs_symbolic_pattern(int32_t n_bus, int32_t n_branch, const int32_t* f, const int32_t* t,
                              int32_t ref_bus, int32_t* perm, int32_t* col_ptr, int32_t* row, int64_t cap,
                              int32_t* level, int64_t* stats) {
    if (n_bus <= 0 || n_branch < 0 || (n_branch > 0 && (!f || !t)) || ref_bus < -1 || ref_bus >= n_bus)
        return CS_E_ARG;
    std::vector<int> F(f, f + n_branch), T(t, t + n_branch);
    Symbolic S;
    if (!symbolic_analysis(n_bus, F, T, ref_bus, S).empty()) return CS_E_ARG;
    const int64_t nL = S.Lcolptr[n_bus];
    std::vector<int> height(n_bus, 0);
    for (int h = 0; h < S.nlevels; ++h)
        for (int w = S.lev_ptr[h]; w < S.lev_ptr[h + 1]; ++w) height[S.lev_col[w]] = h;
    if (stats) {
        stats[0] = nL;
        stats[1] = S.nlevels;
        stats[2] = S.block_updates;
        stats[3] = nL;
    }
    if (perm) std::copy(S.perm.begin(), S.perm.end(), perm);
    if (col_ptr) std::copy(S.Lcolptr.begin(), S.Lcolptr.end(), col_ptr);
    if (level) std::copy(height.begin(), height.end(), level);
    if (row) {
        if (cap < nL) return CS_E_ARG;
        std::copy(S.Lrow.begin(), S.Lrow.end(), row);
    }
    return CS_OK;
}

cs_status cs_base_result(cs_ctx* ctx, int32_t net_id, int32_t level, const cs_result* out) {
    if (!ctx) return CS_E_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    auto it = ctx->nets.find(net_id);
    if (it == ctx->nets.end()) return fail(ctx, CS_E_UNKNOWN_ID, "unknown network");
    Network* n = it->second.get();
    if (!out || level < 0 || level >= n->nlev) return fail(ctx, CS_E_ARG, "bad level or NULL out");
    if (out->klass) out->klass[0] = n->base_klass[level];
    if (out->severe) out->severe[0] = n->base_severe[level];
    if (out->n_islands) out->n_islands[0] = n->base_isl[level];
    if (out->opf_iters) out->opf_iters[0] = n->base_iters[level];
    if (out->cost) out->cost[0] = n->base_cost[level];
    if (out->max_re) out->max_re[0] = n->base_maxre[level];
    if (out->min_zeta) out->min_zeta[0] = n->base_minz[level];
    return CS_OK;
}

cs_status cs_evaluate_device(cs_ctx* ctx, int32_t net_id, int32_t level, const int32_t* ei, const int32_t* ej,
                             int64_t n, const cs_result* out, void* stream) {
    if (!ctx) return CS_E_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    auto it = ctx->nets.find(net_id);
    if (it == ctx->nets.end()) return fail(ctx, CS_E_UNKNOWN_ID, "unknown network");
    Network* net = it->second.get();
    if (level < 0 || level >= net->nlev) return fail(ctx, CS_E_ARG, "level out of range");
    if (n < 0 || n > (int64_t)1 << 31) return fail(ctx, CS_E_ARG, "n out of range");
    if (n == 0) return CS_OK;
    if (!ei || !ej || !out || !out->klass || !out->severe || !out->n_islands || !out->opf_iters || !out->cost ||
        !out->max_re || !out->min_zeta)
        return fail(ctx, CS_E_ARG, "NULL buffer");
    CS_CUDA(cudaSetDevice(ctx->device));
    const int64_t chunk = default_chunk(ctx, *net);
    if (ctx->opt.hbm_budget > 0) {
        const size_t want = workspace_bytes(ctx, *net, std::min<int64_t>(n, chunk)) * (n > chunk ? 2 : 1);
        const size_t have = ctx->direct.bytes() + ctx->direct2.bytes();
        if (want > have && reserved_bytes(ctx) - have + want > (size_t)ctx->opt.hbm_budget)
            return fail(ctx, CS_E_NOMEM, "workspace would exceed hbm_budget");
    }
    ctx->launches = 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (n <= chunk) return evaluate_impl(ctx, ctx->direct, net, level, ei, ej, n, out, s, true, chunk);
    // Several chunks: they alternate between two workspaces on the caller's stream and
    // a second stream, so that one chunk's kernels fill the SMs its predecessor's tail
    // leaves idle.  The second stream starts after the caller's prior work and the
    // caller's stream resumes after the last chunk of either.
    CS_CUDA(cudaEventRecord(ctx->fork_ev, s));
    CS_CUDA(cudaStreamWaitEvent(ctx->aux_stream, ctx->fork_ev, 0));
    int q = 0;
    for (int64_t c0 = 0; c0 < n; c0 += chunk, ++q) {
        const int64_t m = std::min(chunk, n - c0);
        const cs_result o = result_at(*out, c0, net->dev.nb);
        const bool second = (q & 1) != 0;
        cs_status st = evaluate_impl(ctx, second ? ctx->direct2 : ctx->direct, net, level, ei + c0, ej + c0, m, &o,
                                     second ? ctx->aux_stream : s, true, chunk);
        if (st != CS_OK) return st;
    }
    CS_CUDA(cudaEventRecord(ctx->join_ev, ctx->aux_stream));
    CS_CUDA(cudaStreamWaitEvent(s, ctx->join_ev, 0));
    return CS_OK;
}

cs_status cs_sync(cs_ctx* ctx, void* stream) {
    if (!ctx) return CS_E_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    CS_CUDA(cudaSetDevice(ctx->device));
    CS_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    if (ctx->err_word.p) {
        int e = 0;
        CS_CUDA(cudaMemcpy(&e, ctx->err_word.p, sizeof(int), cudaMemcpyDeviceToHost));
        if (e) {
            CS_CUDA(cudaMemset(ctx->err_word.p, 0, sizeof(int)));
            if (e & ERR_BAD_ELEMENT) return fail(ctx, CS_E_ARG, "element id out of range (record marked 255)");
            if (e & ERR_BAD_RATE)
                return fail(ctx, CS_E_ARG, "failure rate outside [2^-30, 2^10] in a batched Risk Index (entry NaN)");
            if (e & ERR_TIMEOUT) return fail(ctx, CS_E_TIMEOUT, "a bounded tensor-core wait gave up");
            return fail(ctx, CS_E_NUMERIC, "device error word " + std::to_string(e));
        }
    }
    return CS_OK;
}

// ------------------------------------------------------------ requests ----
// ---------------------------------------------------------- Risk Index ----
cs_status cs_risk_index(cs_ctx* ctx, int32_t net_id, int32_t level, const double* lambda, int32_t mode,
                        double* R_out, int64_t* n_missing) {
    if (!ctx) return CS_E_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    auto it = ctx->nets.find(net_id);
    if (it == ctx->nets.end()) return fail(ctx, CS_E_UNKNOWN_ID, "unknown network");
    Network* net = it->second.get();
    if (level < 0 || level >= net->nlev || !lambda || !R_out || (mode != CS_RISK_EQ3 && mode != CS_RISK_ORDERED))
        return fail(ctx, CS_E_ARG, "bad level, mode or NULL");
    const int nE = net->dev.nE;
    for (int i = 0; i < nE; ++i)
        if (!(lambda[i] >= std::ldexp(1.0, -30) && lambda[i] <= std::ldexp(1.0, 10)))
            return fail(ctx, CS_E_ARG, "lambda outside [2^-30, 2^10]");
    CS_CUDA(cudaSetDevice(ctx->device));
    DevBuf dl, dr, dm;
    CS_CUDA(dl.ensure(sizeof(double) * nE));
    CS_CUDA(dr.ensure(sizeof(double) * nE));
    CS_CUDA(dm.ensure(sizeof(int64_t)));
    cudaStream_t s = ctx->req_stream;
    CS_CUDA(cudaDeviceSynchronize());      // tables written by earlier evaluations on any stream
    CS_CUDA(cudaMemcpyAsync(dl.p, lambda, sizeof(double) * nE, cudaMemcpyHostToDevice, s));
    CS_CUDA(cudaMemsetAsync(dm.p, 0, sizeof(int64_t), s));
    CS_CUDA(launch_risk(nE, (const uint8_t*)net->sev_n1[level]->p, (const uint8_t*)net->sev_pairs[level]->p,
                        (const double*)dl.p, mode, (double*)dr.p, (int64_t*)dm.p, s));
    CS_CUDA(cudaMemcpyAsync(R_out, dr.p, sizeof(double) * nE, cudaMemcpyDeviceToHost, s));
    int64_t miss = 0;
    CS_CUDA(cudaMemcpyAsync(&miss, dm.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CS_CUDA(cudaStreamSynchronize(s));
    if (n_missing) *n_missing = miss;
    return CS_OK;
}

cs_status cs_evaluate_device_n3(cs_ctx* ctx, int32_t net_id, int32_t level, const int32_t* ei, const int32_t* ej,
                                const int32_t* ek, int64_t n, const cs_result* out, void* stream) {
    if (!ctx) return CS_E_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    auto it = ctx->nets.find(net_id);
    if (it == ctx->nets.end()) return fail(ctx, CS_E_UNKNOWN_ID, "unknown network");
    Network* net = it->second.get();
    if (level < 0 || level >= net->nlev) return fail(ctx, CS_E_ARG, "level out of range");
    if (n < 0 || n > (int64_t)1 << 31) return fail(ctx, CS_E_ARG, "n out of range");
    if (n == 0) return CS_OK;
    if (!ei || !ej || !ek || !out || !out->klass || !out->severe || !out->n_islands || !out->opf_iters ||
        !out->cost || !out->max_re || !out->min_zeta)
        return fail(ctx, CS_E_ARG, "NULL buffer");
    CS_CUDA(cudaSetDevice(ctx->device));
    ctx->launches = 0;
    return evaluate_impl(ctx, ctx->direct, net, level, ei, ej, n, out, (cudaStream_t)stream, true,
                         default_chunk(ctx, *net), ek);
}

cs_status cs_enumerate_triples_device(int32_t n_elem, int64_t first, int64_t count, int32_t* ei, int32_t* ej,
                                      int32_t* ek, void* stream) {
    const int64_t E = n_elem;
    const int64_t total = E < 3 ? 0 : E * (E - 1) * (E - 2) / 6;
    if (n_elem < 3 || n_elem > 32767 || first < 0 || count < 0 || first + count > total ||
        (count > 0 && (!ei || !ej || !ek)))
        return CS_E_ARG;
    cudaError_t e = launch_enumerate3(n_elem, first, count, ei, ej, ek, (cudaStream_t)stream);
    return e == cudaSuccess ? CS_OK : CS_E_CUDA;
}

cs_status cs_risk_index_pair_freq(cs_ctx* ctx, int32_t net_id, int32_t level, const double* lambda, const double* F,
                                  int32_t mode, double* R_out, int64_t* n_missing) {
    if (!ctx) return CS_E_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    auto it = ctx->nets.find(net_id);
    if (it == ctx->nets.end()) return fail(ctx, CS_E_UNKNOWN_ID, "unknown network");
    Network* net = it->second.get();
    if (level < 0 || level >= net->nlev || !lambda || !F || !R_out || (mode != CS_RISK_EQ3 && mode != CS_RISK_ORDERED))
        return fail(ctx, CS_E_ARG, "bad level, mode or NULL");
    const int nE = net->dev.nE;
    for (int i = 0; i < nE; ++i)
        if (!(lambda[i] >= std::ldexp(1.0, -30) && lambda[i] <= std::ldexp(1.0, 10)))
            return fail(ctx, CS_E_ARG, "lambda outside [2^-30, 2^10]");
    for (int64_t q = 0; q < (int64_t)nE * nE; ++q)
        if (!(F[q] == 0.0 || (F[q] >= std::ldexp(1.0, -60) && F[q] <= std::ldexp(1.0, 20))))
            return fail(ctx, CS_E_ARG, "pair frequency outside {0} U [2^-60, 2^20]");
    CS_CUDA(cudaSetDevice(ctx->device));
    DevBuf dl, dF, dr, dm;
    CS_CUDA(dl.ensure(sizeof(double) * nE));
    CS_CUDA(dF.ensure(sizeof(double) * (size_t)nE * nE));
    CS_CUDA(dr.ensure(sizeof(double) * nE));
    CS_CUDA(dm.ensure(sizeof(int64_t)));
    cudaStream_t s = ctx->req_stream;
    CS_CUDA(cudaDeviceSynchronize());      // tables written by earlier evaluations on any stream
    CS_CUDA(cudaMemcpyAsync(dl.p, lambda, sizeof(double) * nE, cudaMemcpyHostToDevice, s));
    CS_CUDA(cudaMemcpyAsync(dF.p, F, sizeof(double) * (size_t)nE * nE, cudaMemcpyHostToDevice, s));
    CS_CUDA(cudaMemsetAsync(dm.p, 0, sizeof(int64_t), s));
    CS_CUDA(launch_risk(nE, (const uint8_t*)net->sev_n1[level]->p, (const uint8_t*)net->sev_pairs[level]->p,
                        (const double*)dl.p, mode, (double*)dr.p, (int64_t*)dm.p, s, (const double*)dF.p));
    CS_CUDA(cudaMemcpyAsync(R_out, dr.p, sizeof(double) * nE, cudaMemcpyDeviceToHost, s));
    int64_t miss = 0;
    CS_CUDA(cudaMemcpyAsync(&miss, dm.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CS_CUDA(cudaStreamSynchronize(s));
    if (n_missing) *n_missing = miss;
    return CS_OK;
}

cs_status cs_risk_index_batch(cs_ctx* ctx, int32_t net_id, int32_t level, const double* lambda, int64_t n_samples,
                              int32_t mode, double* R, void* stream) {
    if (!ctx) return CS_E_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    auto it = ctx->nets.find(net_id);
    if (it == ctx->nets.end()) return fail(ctx, CS_E_UNKNOWN_ID, "unknown network");
    Network* net = it->second.get();
    if (level < 0 || level >= net->nlev || n_samples < 0 || (n_samples > 0 && (!lambda || !R)) ||
        (mode != CS_RISK_EQ3 && mode != CS_RISK_ORDERED))
        return fail(ctx, CS_E_ARG, "bad level, sample count, mode or NULL");
    if (n_samples == 0) return CS_OK;
    CS_CUDA(cudaSetDevice(ctx->device));
    if (!ctx->err_word.p) {
        CS_CUDA(ctx->err_word.ensure(sizeof(int) * 2));
        CS_CUDA(cudaMemset(ctx->err_word.p, 0, sizeof(int) * 2));
    }
    cudaStream_t s = (cudaStream_t)stream;
    // severity tables are written by evaluations on any stream of the context
    CS_CUDA(cudaDeviceSynchronize());
    CS_CUDA(launch_risk_batch(net->dev.nE, (const uint8_t*)net->sev_n1[level]->p,
                              (const uint8_t*)net->sev_pairs[level]->p, lambda, n_samples, mode, R,
                              (int*)ctx->err_word.p, 2, s));
    ctx->launches = 1;
    return CS_OK;
}

cs_status cs_risk_reduce_device(int32_t n_elem, const uint8_t* S1, const uint8_t* S2, const double* lambda,
                                int32_t mode, double* R, void* stream) {
    if (n_elem < 0 || (n_elem > 0 && (!S1 || !S2 || !lambda || !R)) || (mode != CS_RISK_EQ3 && mode != CS_RISK_ORDERED))
        return CS_E_ARG;
    cudaError_t e = launch_risk(n_elem, S1, S2, lambda, mode, R, nullptr, (cudaStream_t)stream);
    return e == cudaSuccess ? CS_OK : CS_E_CUDA;
}

cs_status cs_tc_gemm_update(cs_ctx* ctx, int32_t batch, int32_t M, int32_t N, int32_t K, const float* A,
                            int64_t lda, int64_t stride_a, const float* B, int64_t ldb, int64_t stride_b,
                            float* C, int64_t ldc, int64_t stride_c, float alpha, void* stream) {
    if (batch < 0 || M < 0 || N < 0 || K < 0 || lda < K || ldb < N || ldc < N || stride_a < 0 || stride_b < 0 ||
        stride_c < 0 || (batch > 0 && M > 0 && N > 0 && K > 0 && (!A || !B || !C)))
        return CS_E_ARG;
    int* err = nullptr;
    if (ctx) {
        std::lock_guard<std::mutex> lock(ctx->mu);
        if (cudaSetDevice(ctx->device) != cudaSuccess) return CS_E_CUDA;
        if (!ctx->err_word.p) {
            CS_CUDA(ctx->err_word.ensure(sizeof(int) * 2));
            CS_CUDA(cudaMemset(ctx->err_word.p, 0, sizeof(int) * 2));
        }
        err = (int*)ctx->err_word.p;
    }
    cudaError_t e = launch_tc_gemm(batch, M, N, K, A, lda, stride_a, B, ldb, stride_b, C, ldc, stride_c, alpha, err,
                                   (cudaStream_t)stream);
    return e == cudaSuccess ? CS_OK : CS_E_CUDA;
}

cs_status cs_hessenberg_tc(cs_ctx* ctx, int32_t batch, int32_t n, float* A, int64_t stride, void* stream) {
    if (!ctx) return CS_E_ARG;
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (batch < 0 || n < 0 || n > 32767 || stride < (int64_t)n * n || (batch > 0 && n > 0 && !A))
        return fail(ctx, CS_E_ARG, "bad batch, order, stride or NULL matrix");
    if (batch == 0 || n < 3) return CS_OK;
    CS_CUDA(cudaSetDevice(ctx->device));
    if (!ctx->err_word.p) {
        CS_CUDA(ctx->err_word.ensure(sizeof(int) * 2));
        CS_CUDA(cudaMemset(ctx->err_word.p, 0, sizeof(int) * 2));
    }
    CS_CUDA(ctx->hess_ws.ensure(sizeof(float) * hess_tc_workspace_floats(n) * (size_t)batch));
    CS_CUDA(launch_hess_tc(batch, n, A, stride, (float*)ctx->hess_ws.p, (int*)ctx->err_word.p, (cudaStream_t)stream));
    return CS_OK;
}

cs_status cs_enumerate_pairs_device(int32_t n_elem, int64_t first, int64_t count, int32_t* ei, int32_t* ej,
                                    void* stream) {
    const int64_t total = (int64_t)n_elem * (n_elem - 1) / 2;
    if (n_elem < 2 || first < 0 || count < 0 || first + count > total || (count > 0 && (!ei || !ej))) return CS_E_ARG;
    cudaError_t e = launch_enumerate(n_elem, first, count, ei, ej, (cudaStream_t)stream);
    return e == cudaSuccess ? CS_OK : CS_E_CUDA;
}


// ---------------------------------------------------------------------------
// Risk Index without any device allocation.
//
// Who needs it: a caller that must not call cudaMalloc/cudaFree between its
// own launches -- a serving loop whose other streams would stall behind the
// device-wide synchronisation cudaFree implies, or a process whose device
// memory is already reserved in full by another allocator (a caching
// allocator with a memory fraction), where a fresh cudaMalloc may fail.
// cs_risk_index allocates three small device buffers per call; this variant
// takes them from one file-scope device array instead.
//
// The array holds lambda[kStaticRiskMaxElem], R[kStaticRiskMaxElem] and the
// 64-bit missing-pair counter, which is cleared by cudaMemsetAsync before
// every launch (the other two are fully overwritten).  Its device address is
// looked up once per device, with that device current, on the first call for
// it; that first call should happen before any stream capture on the device.
// All calls in the process share the one array per device, so overlapping
// calls would race on it: a process-wide lock serialises them, and each returns
// only after its stream has drained.
//
// Ordering without a device-wide synchronisation: the library stream waits
// (on the device) for the completion events of every workspace of the context,
// i.e. for the evaluations issued before the call, whatever their streams.  The
// context lock is held only while that is enqueued; the copies and the wait
// for them run without it, so the serving scheduler keeps retiring and
// admitting batches meanwhile (the network is marked busy, so it cannot be
// unloaded under the call).
constexpr int kStaticRiskMaxElem = 4096;
constexpr int kStaticRiskDoubles = 2 * kStaticRiskMaxElem + 32;   // + counter, padded
static __device__ __align__(256) double g_static_risk[kStaticRiskDoubles];

namespace {
constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mu;
double* g_static_ptr[kStaticMaxDevices] = {};

cudaError_t static_risk_scratch(int device, double** p) {
    if (device < 0 || device >= kStaticMaxDevices) return cudaErrorInvalidDevice;
    if (!g_static_ptr[device]) {
        void* a = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&a, g_static_risk);
        if (e != cudaSuccess) return e;
        g_static_ptr[device] = (double*)a;
    }
    *p = g_static_ptr[device];
    return cudaSuccess;
}
}  // namespace

namespace {
// the library stream waits for every evaluation issued so far on the context's workspaces
cudaError_t wait_for_evaluations(cs_ctx* ctx, cudaStream_t s) {
    auto wait = [&](const Workspace& ws) -> cudaError_t {
        return (ws.used && ws.free) ? cudaStreamWaitEvent(s, ws.free, 0) : cudaSuccess;
    };
    cudaError_t e = wait(ctx->direct);
    if (e == cudaSuccess) e = wait(ctx->direct2);
    for (auto& sl : ctx->slots)
        if (e == cudaSuccess) e = wait(sl->ws);
    return e;
}
}  // namespace

cs_status cs_risk_index_static(cs_ctx* ctx, int32_t net_id, int32_t level, const double* lambda, int32_t mode,
                               double* R_out, int64_t* n_missing) {
    if (!ctx) return CS_E_ARG;
    std::lock_guard<std::mutex> glock(g_static_mu);
    Network* net = nullptr;
    const uint8_t *S1 = nullptr, *S2 = nullptr;
    double* base = nullptr;
    int nE = 0;
    cudaStream_t s = nullptr;
    {
        std::lock_guard<std::mutex> lock(ctx->mu);
        auto it = ctx->nets.find(net_id);
        if (it == ctx->nets.end()) return fail(ctx, CS_E_UNKNOWN_ID, "unknown network");
        net = it->second.get();
        if (level < 0 || level >= net->nlev || !lambda || !R_out || (mode != CS_RISK_EQ3 && mode != CS_RISK_ORDERED))
            return fail(ctx, CS_E_ARG, "bad level, mode or NULL");
        nE = net->dev.nE;
        if (nE > kStaticRiskMaxElem)
            return fail(ctx, CS_E_ARG, "cs_risk_index_static: " + std::to_string(nE) +
                                           " outage elements exceed its " + std::to_string(kStaticRiskMaxElem) +
                                           "-element static scratch; use cs_risk_index");
        for (int i = 0; i < nE; ++i)
            if (!(lambda[i] >= std::ldexp(1.0, -30) && lambda[i] <= std::ldexp(1.0, 10)))
                return fail(ctx, CS_E_ARG, "lambda outside [2^-30, 2^10]");
        CS_CUDA(cudaSetDevice(ctx->device));
        CS_CUDA(static_risk_scratch(ctx->device, &base));
        s = ctx->req_stream;
        CS_CUDA(wait_for_evaluations(ctx, s));     // tables written by earlier evaluations on any stream
        S1 = (const uint8_t*)net->sev_n1[level]->p;
        S2 = (const uint8_t*)net->sev_pairs[level]->p;
        net->busy++;
    }
    // copies, launch and wait without the context lock
    double* dl = base;
    double* dr = base + kStaticRiskMaxElem;
    int64_t* dm = (int64_t*)(base + 2 * kStaticRiskMaxElem);
    int64_t miss = 0;
    cudaError_t e = cudaSetDevice(ctx->device);
    const char* where = "cudaSetDevice";
    if (e == cudaSuccess) { e = cudaMemcpyAsync(dl, lambda, sizeof(double) * nE, cudaMemcpyHostToDevice, s); where = "copy of lambda"; }
    if (e == cudaSuccess) { e = cudaMemsetAsync(dm, 0, sizeof(int64_t), s); where = "clear of the missing-pair counter"; }
    if (e == cudaSuccess) { e = launch_risk(nE, S1, S2, dl, mode, dr, dm, s); where = "risk_kernel launch"; }
    if (e == cudaSuccess) { e = cudaMemcpyAsync(R_out, dr, sizeof(double) * nE, cudaMemcpyDeviceToHost, s); where = "copy of R"; }
    if (e == cudaSuccess) { e = cudaMemcpyAsync(&miss, dm, sizeof(int64_t), cudaMemcpyDeviceToHost, s); where = "copy of the count"; }
    if (e == cudaSuccess) { e = cudaStreamSynchronize(s); where = "cudaStreamSynchronize"; }
    std::lock_guard<std::mutex> lock(ctx->mu);
    net->busy--;
    if (e != cudaSuccess) return cuda_fail(ctx, e, where);
    if (n_missing) *n_missing = miss;
    return CS_OK;
}

}  // extern "C"
