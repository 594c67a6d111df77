// mk_server.cpp -- continuous-batching evaluation of many k-bit operator
// requests (Sec. 4.3-4.5 operators) from several clients.
//
// Every admitted request keeps its wire ciphertexts in one device pool (rows
// of k*n+1 words, a first-fit row allocator).  A wave is one batched
// bootstrap + key-switch launch over the ready gates of every running
// request: each request contributes the gates of its current netlist level
// (a level larger than the remaining wave capacity is split across waves);
// a request moves to its next level once all gates of the current one have
// run.  Requests are admitted at wave boundaries, in arrival order, as soon
// as the pool has room, so new work overlaps with requests already on the
// GPU.  Results do not depend on the mix: every gate reads only its own
// request's wires, and the arithmetic is exact (NTT forms).
#include <deque>

#include "mk_ctx.h"

namespace mk {
namespace {

struct ServerPlan {
    Netlist net;
    uint32_t pairs = 0, n_wires = 0;
    std::vector<GateDesc> desc;       // rows relative to the request's base row, levels concatenated
    std::vector<uint32_t> level_off;  // size levels + 1
    int32_t *d_outs = nullptr;        // outputs as 2*wire + negated
    ~ServerPlan() { cudaFree(d_outs); }
};

struct Request {
    uint64_t ticket;
    int op;
    uint32_t kbits, pairs;
    const uint32_t *d_a, *d_b;
    uint32_t *d_out, *d_out2;
    ServerPlan *plan = nullptr;
    uint64_t base = 0, rows = 0;  // pool rows [base, base + rows)
    uint32_t level = 0;           // index into plan->level_off
    uint32_t issued = 0;          // gates of the current level already run
    uint32_t in_wave = 0;         // gates of the current level in the wave being built
    int state = 0;                // 0 queued, 1 running, 2 done
};

}  // namespace
}  // namespace mk

struct mk_server {
    mk_ctx *ctx = nullptr;
    uint32_t wave_gates = 0;
    uint64_t pool_rows = 0;
    uint32_t *d_pool = nullptr, *d_ext = nullptr;
    GateDesc *d_desc = nullptr, *h_desc = nullptr;
    std::map<uint64_t, uint64_t> free_rows;  // start -> length
    std::map<std::tuple<int, uint32_t, uint32_t, int>, std::unique_ptr<ServerPlan>> plans;  // op, k, pairs, style
    std::deque<Request *> queued;
    std::vector<Request *> running;
    std::map<uint64_t, std::unique_ptr<Request>> all;
    uint64_t next_ticket = 1, waves = 0, gates = 0;
};

namespace mk {
namespace {

bool alloc_rows(mk_server *s, uint64_t n, uint64_t *base) {
    for (auto it = s->free_rows.begin(); it != s->free_rows.end(); ++it) {
        if (it->second < n) continue;
        *base = it->first;
        const uint64_t rest = it->second - n, start = it->first + n;
        s->free_rows.erase(it);
        if (rest) s->free_rows[start] = rest;
        return true;
    }
    return false;
}

void free_rows(mk_server *s, uint64_t base, uint64_t n) {
    auto it = s->free_rows.emplace(base, n).first;
    auto nx = std::next(it);
    if (nx != s->free_rows.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        s->free_rows.erase(nx);
    }
    if (it != s->free_rows.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            s->free_rows.erase(it);
        }
    }
}

int server_plan(mk_server *s, int op, uint32_t k, uint32_t pairs, ServerPlan **out) {
    mk_ctx *c = s->ctx;
    auto key = std::make_tuple(op, k, pairs, c->circuit_style);
    auto it = s->plans.find(key);
    if (it != s->plans.end()) {
        *out = it->second.get();
        return MK_OK;
    }
    auto plan = std::make_unique<ServerPlan>();
    if (!build_netlist(op, k, c->circuit_style, plan->net)) return fail(c, MK_EINVAL, "unsupported operator or kbits");
    const Netlist &net = plan->net;
    const std::vector<uint32_t> lev = netlist_levels(net);
    const uint32_t L = lev.empty() ? 0 : *std::max_element(lev.begin(), lev.end());
    const uint32_t base = 2 + net.ka + net.kb;
    plan->pairs = pairs;
    plan->n_wires = base + (uint32_t)net.gates.size();
    std::vector<std::vector<uint32_t>> by_level(L + 1);
    for (uint32_t g = 0; g < net.gates.size(); ++g) by_level[lev[g]].push_back(g);
    plan->level_off.push_back(0);
    for (uint32_t l = 1; l <= L; ++l) {
        for (uint32_t g : by_level[l]) {
            const mk_gate_rec &r = net.gates[g];
            const mk_lin lin = gate_lin(r);
            for (uint32_t p = 0; p < pairs; ++p)
                plan->desc.push_back(GateDesc{(uint32_t)r.a * pairs + p, (uint32_t)r.b * pairs + p, lin.cst, lin.s1,
                                              lin.s2, (base + g) * pairs + p});
        }
        plan->level_off.push_back((uint32_t)plan->desc.size());
    }
    std::vector<int32_t> outs;
    for (const Wire &w : net.outputs) outs.push_back(w.w * 2 + w.neg);
    MK_CUDA(c, cudaMalloc(&plan->d_outs, outs.size() * sizeof(int32_t)));
    MK_CUDA(c, cudaMemcpy(plan->d_outs, outs.data(), outs.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    *out = plan.get();
    s->plans[key] = std::move(plan);
    return MK_OK;
}

// Copy a request's operands into its rows (constants, then a and b bits).
cudaError_t admit_inputs(mk_server *s, Request *r) {
    mk_ctx *c = s->ctx;
    const uint32_t W = (uint32_t)c->W(), P = r->pairs;
    uint32_t *pool = s->d_pool + r->base * W;
    cudaError_t e = launch_circuit_consts(pool, P, W, c->stream);
    if (e == cudaSuccess) e = launch_circuit_inputs(pool, r->d_a, r->kbits, P, 2, W, c->stream);
    if (e == cudaSuccess) e = launch_circuit_inputs(pool, r->d_b, r->kbits, P, 2 + r->kbits, W, c->stream);
    return e;
}

cudaError_t finish_outputs(mk_server *s, Request *r) {
    mk_ctx *c = s->ctx;
    const uint32_t W = (uint32_t)c->W(), P = r->pairs;
    const uint32_t nout = (uint32_t)r->plan->net.outputs.size();
    const uint32_t *pool = s->d_pool + r->base * W;
    if (!r->d_out2) return launch_circuit_outputs(r->d_out, pool, r->plan->d_outs, nout, P, W, c->stream);
    cudaError_t e = launch_circuit_outputs(r->d_out, pool, r->plan->d_outs, nout / 2, P, W, c->stream);
    if (e == cudaSuccess)
        e = launch_circuit_outputs(r->d_out2, pool, r->plan->d_outs + nout / 2, nout - nout / 2, P, W, c->stream);
    return e;
}

}  // namespace
}  // namespace mk

extern "C" {

int mk_server_create(mk_ctx *c, uint32_t wave_gates, uint64_t pool_rows, mk_server **out) {
    if (!c || !out || wave_gates == 0 || pool_rows == 0) return MK_EINVAL;
    *out = nullptr;
    if (c->device < 0) return fail(c, MK_EDEVICE, "host-only context");
    int rc = ensure_device_keys(c);
    if (rc) return rc;
    auto s = std::make_unique<mk_server>();
    s->ctx = c;
    s->wave_gates = wave_gates;
    s->pool_rows = pool_rows;
    MK_CUDA(c, cudaSetDevice(c->device));
    MK_CUDA(c, cudaMalloc(&s->d_pool, pool_rows * c->W() * 4));
    MK_CUDA(c, cudaMalloc(&s->d_ext, (size_t)wave_gates * c->E() * 4));
    MK_CUDA(c, cudaMalloc(&s->d_desc, (size_t)wave_gates * sizeof(GateDesc)));
    MK_CUDA(c, cudaMallocHost(&s->h_desc, (size_t)wave_gates * sizeof(GateDesc)));
    s->free_rows[0] = pool_rows;
    *out = s.release();
    return MK_OK;
}

int mk_server_destroy(mk_server *s) {
    if (!s) return MK_EINVAL;
    mk_ctx *c = s->ctx;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    cudaFree(s->d_pool);
    cudaFree(s->d_ext);
    cudaFree(s->d_desc);
    cudaFreeHost(s->h_desc);
    delete s;
    return MK_OK;
}

int mk_server_submit(mk_server *s, int op, uint32_t kbits, const uint32_t *d_a, const uint32_t *d_b, uint32_t *d_out,
                     uint32_t *d_out2, uint32_t pairs, uint64_t *ticket) {
    if (!s || !ticket) return MK_EINVAL;
    mk_ctx *c = s->ctx;
    if (!d_a || !d_b || !d_out || pairs == 0) return fail(c, MK_EINVAL, "null pointer or no pairs");
    if ((op == MK_OP_DIV) != (d_out2 != nullptr)) return fail(c, MK_EINVAL, "the divider (only) needs d_out2");
    auto r = std::make_unique<Request>();
    r->ticket = s->next_ticket++;
    r->op = op;
    r->kbits = kbits;
    r->pairs = pairs;
    r->d_a = d_a;
    r->d_b = d_b;
    r->d_out = d_out;
    r->d_out2 = d_out2;
    int rc = server_plan(s, op, kbits, pairs, &r->plan);
    if (rc) return rc;
    r->rows = (uint64_t)r->plan->n_wires * pairs;
    if (r->rows > s->pool_rows) return fail(c, MK_EINVAL, "request larger than the server's pool");
    *ticket = r->ticket;
    s->queued.push_back(r.get());
    s->all[r->ticket] = std::move(r);
    return MK_OK;
}

int mk_server_step(mk_server *s, uint32_t *n_done) {
    if (!s) return MK_EINVAL;
    mk_ctx *c = s->ctx;
    if (n_done) *n_done = 0;
    MK_CUDA(c, cudaSetDevice(c->device));
    // 1. admission at the wave boundary, in arrival order, while rows are free
    while (!s->queued.empty()) {
        Request *r = s->queued.front();
        if (!alloc_rows(s, r->rows, &r->base)) break;
        s->queued.pop_front();
        const cudaError_t e = admit_inputs(s, r);
        if (e != cudaSuccess) return cuda_fail(c, e, "server admission");
        r->state = 1;
        r->level = 0;
        r->issued = 0;
        s->running.push_back(r);
    }
    // 2. the wave: ready gates of every running request, oldest first
    uint32_t n = 0;
    for (Request *r : s->running) {
        r->in_wave = 0;
        const uint32_t lo = r->plan->level_off[r->level] + r->issued, hi = r->plan->level_off[r->level + 1];
        const uint32_t take = std::min(hi - lo, s->wave_gates - n);
        const uint32_t base = (uint32_t)r->base;
        for (uint32_t g = 0; g < take; ++g) {
            GateDesc d = r->plan->desc[lo + g];
            d.ia += base;
            d.ib += base;
            d.out += base;
            s->h_desc[n + g] = d;
        }
        r->in_wave = take;
        n += take;
        if (n == s->wave_gates) break;
    }
    if (n > 0) {
        const LaunchShape S = c->shape();
        const DeviceKeys K = c->dkeys();
        cudaError_t e = cudaMemcpyAsync(s->d_desc, s->h_desc, (size_t)n * sizeof(GateDesc), cudaMemcpyHostToDevice,
                                        c->stream);
        if (e == cudaSuccess)
            e = timed(c, MK_KERNEL_BOOTSTRAP,
                      [&] { return launch_bootstrap_ntt(S, K, s->d_desc, s->d_pool, s->d_pool, s->d_ext, n, c->stream); });
        if (e == cudaSuccess)
            e = timed(c, MK_KERNEL_KEYSWITCH,
                      [&] { return launch_keyswitch(S, K, s->d_desc, s->d_ext, s->d_pool, n, c->stream); });
        if (e != cudaSuccess) return cuda_fail(c, e, "server wave");
        ++s->waves;
        s->gates += n;
    }
    // 3. progress; finished requests write their outputs and release their rows
    std::vector<Request *> still;
    uint32_t done = 0;
    for (Request *r : s->running) {
        r->issued += r->in_wave;
        r->in_wave = 0;
        while (r->level + 1 < r->plan->level_off.size() &&
               r->plan->level_off[r->level] + r->issued == r->plan->level_off[r->level + 1]) {
            ++r->level;
            r->issued = 0;
        }
        if (r->level + 1 >= r->plan->level_off.size()) {
            const cudaError_t e = finish_outputs(s, r);
            if (e != cudaSuccess) return cuda_fail(c, e, "server outputs");
            free_rows(s, r->base, r->rows);  // later work on the stream runs after the copy
            r->state = 2;
            ++done;
        } else {
            still.push_back(r);
        }
    }
    s->running.swap(still);
    MK_CUDA(c, cudaStreamSynchronize(c->stream));
    if (n_done) *n_done = done;
    return MK_OK;
}

int mk_server_poll(const mk_server *s, uint64_t ticket, int *state) {
    if (!s || !state) return MK_EINVAL;
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return MK_EINVAL;
    *state = it->second->state;
    return MK_OK;
}

int mk_server_stats(const mk_server *s, uint64_t *waves, uint64_t *gates, uint32_t *running, uint32_t *queued) {
    if (!s) return MK_EINVAL;
    if (waves) *waves = s->waves;
    if (gates) *gates = s->gates;
    if (running) *running = (uint32_t)s->running.size();
    if (queued) *queued = (uint32_t)s->queued.size();
    return MK_OK;
}

}  // extern "C"
