// Continuously batched serving of global-stage queries.
//
// Each request is one array (layout, dT, boundary conditions) against block
// models that are already resident. The server solves every running request
// together, as one batch, by FP64-residual iterative refinement: a step is
// one FP64 residual check for every running array followed by one inner
// solve of the correction (in the context's precision; FP64 when the context
// is FP64). Between steps the batch changes membership:
//   * arrays whose residual check stopped them (converged, or a limit) retire:
//     their per-element von Mises field is recovered into the request's own
//     device buffer, and their memory leaves the batch;
//   * queued requests are admitted in arrival order while the slot count and
//     the HBM budget allow (each request's device footprint is estimated from
//     its lattice and block counts);
//   * the packed batch is rebuilt for the new membership, carrying every
//     continuing array's FP64 iterate and refinement state.
// An array's arithmetic never depends on the other arrays of a batch (its work
// items, reductions and stopping tests are its own), so each result is the
// same alone and in the mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <unordered_map>

#include "solve.h"

namespace ms {
namespace {

enum { RQ_QUEUED = 0, RQ_RUNNING = 1, RQ_DONE = 2, RQ_FAILED = 3 };

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    int64_t id = 0;
    int state = RQ_QUEUED;
    int nx = 0, ny = 0;
    std::vector<uint8_t> site;
    std::vector<mstress_block> blocks;
    double dT = 0;
    int clamp_bottom = 1, clamp_top = 0;
    size_t need = 0;              // estimated device bytes while running
    double t_submit = 0, t_admit = 0, t_done = 0;
    ArrayResult res;
    DBuf vm;                      // von Mises per element, [block][n_el]
    size_t vm_bytes = 0;
    int fail_code = MSTRESS_OK;
};

}  // namespace
}  // namespace ms

struct mstress_server_s {
    mstress_ctx ctx = nullptr;
    int max_slots = 0;
    size_t budget = 0;
    int64_t next_id = 1;
    std::unordered_map<int64_t, std::unique_ptr<ms::Request>> reqs;
    std::deque<int64_t> queue;
    std::vector<int64_t> running;             // batch order
    std::deque<int64_t> finished;             // not yet polled
    std::unique_ptr<mstress_sol_s> batch;
    std::vector<int64_t> batch_ids;           // ids in the current batch, in array order
    size_t used = 0;                          // estimated bytes of running requests + held results
};

namespace ms {
namespace {

size_t estimate_bytes(const mstress_server_s* S, const Request& r) {
    mstress_block b = r.blocks[0];
    const int64_t n1 = b->n - 1;
    const int64_t lat = 3 * (r.nx * n1 + 1) * (r.ny * n1 + 1) * b->n;
    const int64_t nb = (int64_t)r.nx * r.ny;
    const int64_t ldY = round_up(b->m, 16);
    const bool mixed = S->ctx->opts.precision != MSTRESS_FP64;
    int64_t bytes = lat * (7 * 8 + (mixed ? 5 * 4 : 5 * 8));           // FP64 vectors + inner vectors
    bytes += nb * ldY * (8 + (mixed ? 4 : 0));                           // element products
    bytes += nb * (int64_t)b->n_el * (mixed ? 4 : 8) * 2;                // result + recovery staging
    bytes += nb * 64 + lat / 64 * 64;                                    // work lists, partials
    return (size_t)(bytes + bytes / 8 + (1 << 20));
}

// Rebuild the batch for the running requests, carrying the FP64 iterate and
// refinement state of arrays that were already in the previous batch.
void rebuild_batch(mstress_server_s* S) {
    mstress_ctx ctx = S->ctx;
    std::unique_ptr<mstress_sol_s> old = std::move(S->batch);
    std::vector<int64_t> old_ids = S->batch_ids;
    S->batch_ids = S->running;
    if (S->running.empty()) return;
    std::vector<mstress_layout> lays(S->running.size());
    std::vector<mstress_bc> bcs(S->running.size());
    std::vector<LayoutIn> in;
    for (size_t k = 0; k < S->running.size(); ++k) {
        Request& r = *S->reqs[S->running[k]];
        lays[k] = mstress_layout{r.nx, r.ny, r.site.data(), r.blocks.data(), (int)r.blocks.size()};
        bcs[k] = mstress_bc{r.clamp_bottom, r.clamp_top, nullptr, nullptr, 0};
        in.push_back(LayoutIn{&lays[k], r.dT, &bcs[k]});
    }
    std::unique_ptr<mstress_sol_s> s(new mstress_sol_s());
    s->ctx = ctx;
    s->precision = ctx->opts.precision;
    s->inner64 = s->precision == MSTRESS_FP64;
    validate_and_build(s.get(), in);
    s->results.assign(s->n_arrays, ArrayResult{});
    solve_prepare(s.get());
    refine_start(s.get());
    cudaStream_t st = ctx->stream;
    for (int a = 0; a < s->n_arrays; ++a) {
        Request& r = *S->reqs[S->running[a]];
        s->results[a] = r.res;   // inner iterations so far
        if (!old) continue;
        auto it = std::find(old_ids.begin(), old_ids.end(), r.id);
        if (it == old_ids.end()) continue;
        const int oa = (int)(it - old_ids.begin());
        s->results[a] = old->results[oa];   // inner iterations of the earlier steps
        const ArrayDev& A = s->arrays[a];
        const ArrayDev& OA = old->arrays[oa];
        MS_CUDA(cudaMemcpyAsync(s->v64.x.as<double>() + A.vec_off, old->v64.x.as<double>() + OA.vec_off,
                                A.n_dof * sizeof(double), cudaMemcpyDeviceToDevice, st));
        MS_CUDA(cudaMemcpyAsync(s->v64.state.as<PcgState>() + a, old->v64.state.as<PcgState>() + oa, sizeof(PcgState),
                                cudaMemcpyDeviceToDevice, st));
    }
    MS_CUDA(cudaStreamSynchronize(st));
    S->batch = std::move(s);
}

void admit(mstress_server_s* S, bool& changed) {
    while (!S->queue.empty() && (int)S->running.size() < S->max_slots) {
        Request& r = *S->reqs[S->queue.front()];
        if (r.need > S->budget) {   // can never fit
            r.state = RQ_FAILED;
            r.fail_code = MSTRESS_ENOMEM;
            r.t_done = now_s();
            S->finished.push_back(r.id);
            S->queue.pop_front();
            continue;
        }
        if (S->used + r.need > S->budget) break;   // wait for memory to free up
        S->queue.pop_front();
        r.state = RQ_RUNNING;
        r.t_admit = now_s();
        S->used += r.need;
        S->running.push_back(r.id);
        changed = true;
    }
}

// Recover the von Mises field of the listed arrays of the batch into their
// requests' buffers, and retire them.
void retire(mstress_server_s* S, const std::vector<int>& arrays, const std::vector<PcgState>& outer) {
    if (arrays.empty()) return;
    mstress_sol_s* s = S->batch.get();
    const bool fp64 = s->precision == MSTRESS_FP64;
    const size_t esz = fp64 ? sizeof(double) : sizeof(float);
    DBuf full;
    alloc_into(S->ctx, full, (size_t)s->n_blocks * s->n_el * esz, false);
    recover_arrays(s, MSTRESS_VM_ELEM, full.ptr, arrays);
    for (int a : arrays) {
        Request& r = *S->reqs[S->batch_ids[a]];
        const ArrayDev& A = s->arrays[a];
        r.vm_bytes = (size_t)A.nx * A.ny * s->n_el * esz;
        alloc_into(S->ctx, r.vm, r.vm_bytes, false);
        MS_CUDA(cudaMemcpyAsync(r.vm.ptr, static_cast<uint8_t*>(full.ptr) + (size_t)A.block_off * s->n_el * esz,
                                r.vm_bytes, cudaMemcpyDeviceToDevice, S->ctx->stream));
        r.res = s->results[a];
        r.res.outer = outer[a].iters;
        r.res.status = outer[a].status;
        r.res.rel_res = outer[a].bb > 0 ? std::sqrt(outer[a].rr / outer[a].bb) : 0.0;
        r.state = RQ_DONE;
        r.t_done = now_s();
        S->used = S->used - std::min(S->used, r.need) + r.vm_bytes;
        S->finished.push_back(r.id);
    }
    MS_CUDA(cudaStreamSynchronize(S->ctx->stream));
    std::vector<int64_t> keep;
    for (int64_t id : S->running)
        if (S->reqs[id]->state == RQ_RUNNING) keep.push_back(id);
    S->running = keep;
}

}  // namespace
}  // namespace ms

using namespace ms;

#define MS_SRV_BEGIN try {
#define MS_SRV_END(ctx)                          \
    }                                            \
    catch (const ms::Error& e) {                 \
        if (ctx) (ctx)->last_error = e.msg;      \
        return e.code;                           \
    }                                            \
    catch (const std::exception& e) {            \
        if (ctx) (ctx)->last_error = e.what();   \
        return MSTRESS_EINVAL;                   \
    }                                            \
    return MSTRESS_OK;

extern "C" {

int mstress_server_create(mstress_ctx ctx, int max_slots, size_t hbm_budget, mstress_server* out) {
    if (!ctx) return MSTRESS_EINVAL;
    if (!out || max_slots < 1) {
        ctx->last_error = "need out and max_slots >= 1";
        return MSTRESS_EINVAL;
    }
    mstress_server S = new mstress_server_s();
    S->ctx = ctx;
    S->max_slots = max_slots;
    S->budget = hbm_budget ? hbm_budget : (size_t)-1;
    *out = S;
    return MSTRESS_OK;
}

int mstress_server_submit(mstress_server S, const mstress_layout* L, double dT, const mstress_bc* bc, int64_t* id) {
    if (!S) return MSTRESS_EINVAL;
    mstress_ctx ctx = S->ctx;
    MS_SRV_BEGIN
    MS_REQUIRE(L && id, MSTRESS_EINVAL, "layout and id are required");
    MS_REQUIRE(L->nx >= 1 && L->ny >= 1 && L->site_type && L->blocks && L->n_blocks >= 1, MSTRESS_EINVAL,
               "bad layout");
    MS_REQUIRE(std::isfinite(dT), MSTRESS_EINVAL, "dT must be finite");
    MS_REQUIRE(!bc || bc->n_prescribed == 0, MSTRESS_EINVAL, "the server takes clamped faces only");
    MS_REQUIRE(!bc || bc->clamp_bottom || bc->clamp_top, MSTRESS_EINVAL, "no constrained DOF");
    std::unique_ptr<Request> r(new Request());
    r->id = S->next_id++;
    r->nx = L->nx;
    r->ny = L->ny;
    r->site.assign(L->site_type, L->site_type + (size_t)L->nx * L->ny);
    r->blocks.assign(L->blocks, L->blocks + L->n_blocks);
    for (auto b : r->blocks) MS_REQUIRE(b && b->ctx == ctx, MSTRESS_EINVAL, "block from another context");
    for (uint8_t t : r->site) MS_REQUIRE(t < L->n_blocks, MSTRESS_EINVAL, "site_type out of range");
    if (!S->running.empty()) {
        mstress_block b0 = S->reqs[S->running[0]]->blocks[0];
        MS_REQUIRE(r->blocks[0]->n == b0->n && r->blocks[0]->n_el == b0->n_el, MSTRESS_EINVAL,
                   "all requests of a server need the same basis order and block mesh size");
    }
    r->dT = dT;
    r->clamp_bottom = bc ? bc->clamp_bottom : 1;
    r->clamp_top = bc ? bc->clamp_top : 0;
    r->need = estimate_bytes(S, *r);
    r->t_submit = now_s();
    *id = r->id;
    S->queue.push_back(r->id);
    S->reqs[r->id] = std::move(r);
    MS_SRV_END(ctx)
}

int mstress_server_step(mstress_server S, int* n_queued, int* n_running, int* n_finished) {
    if (!S) return MSTRESS_EINVAL;
    mstress_ctx ctx = S->ctx;
    MS_SRV_BEGIN
    bool changed = false;
    admit(S, changed);
    if (changed || (S->batch && S->batch_ids != S->running)) rebuild_batch(S);
    int fin = 0;
    if (S->batch) {
        mstress_sol_s* s = S->batch.get();
        const bool any = refine_check(s);
        std::vector<PcgState> outer(s->n_arrays);
        MS_CUDA(cudaMemcpy(outer.data(), s->v64.state.ptr, outer.size() * sizeof(PcgState), cudaMemcpyDeviceToHost));
        std::vector<int> done;
        for (int a = 0; a < s->n_arrays; ++a)
            if (!outer[a].active) done.push_back(a);
        if (any) refine_inner(s);
        check_device_error(s);
        if (!done.empty()) {
            // results of the finished arrays are unchanged by the inner solve
            // (it skips arrays that stopped refining)
            retire(S, done, outer);
            fin = (int)done.size();
            bool ch2 = false;
            admit(S, ch2);
            rebuild_batch(S);
        }
    }
    if (n_queued) *n_queued = (int)S->queue.size();
    if (n_running) *n_running = (int)S->running.size();
    if (n_finished) *n_finished = fin;
    MS_SRV_END(ctx)
}

int mstress_server_poll(mstress_server S, int64_t* id) {
    if (!S || !id) return MSTRESS_EINVAL;
    if (S->finished.empty()) {
        *id = 0;
        return MSTRESS_OK;
    }
    *id = S->finished.front();
    S->finished.pop_front();
    return MSTRESS_OK;
}

int mstress_server_info(mstress_server S, int64_t id, int* state, int* iters, int* outer, double* rel_res,
                        double* latency_ms) {
    if (!S) return MSTRESS_EINVAL;
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return MSTRESS_EINVAL;
    const Request& r = *it->second;
    if (state) *state = r.state;
    if (iters) *iters = r.res.iters;
    if (outer) *outer = r.res.outer;
    if (rel_res) *rel_res = r.res.rel_res;
    if (latency_ms) *latency_ms = r.state >= RQ_DONE ? (r.t_done - r.t_submit) * 1e3 : -1.0;
    return r.state == RQ_FAILED ? r.fail_code : (r.state == RQ_DONE ? r.res.status : MSTRESS_OK);
}

int mstress_server_result(mstress_server S, int64_t id, void* dst, size_t dst_bytes, int dst_on_device) {
    if (!S) return MSTRESS_EINVAL;
    mstress_ctx ctx = S->ctx;
    MS_SRV_BEGIN
    auto it = S->reqs.find(id);
    MS_REQUIRE(it != S->reqs.end(), MSTRESS_EINVAL, "unknown request");
    Request& r = *it->second;
    MS_REQUIRE(r.state == RQ_DONE, MSTRESS_EINVAL, "request has no result");
    MS_REQUIRE(dst && dst_bytes >= r.vm_bytes, MSTRESS_EINVAL, "dst too small");
    MS_CUDA(cudaMemcpyAsync(dst, r.vm.ptr, r.vm_bytes,
                            dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    MS_CUDA(cudaStreamSynchronize(ctx->stream));
    MS_SRV_END(ctx)
}

int mstress_server_release(mstress_server S, int64_t id) {
    if (!S) return MSTRESS_EINVAL;
    auto it = S->reqs.find(id);
    if (it == S->reqs.end() || it->second->state < RQ_DONE) return MSTRESS_EINVAL;
    S->used -= std::min(S->used, it->second->vm_bytes);
    S->reqs.erase(it);
    return MSTRESS_OK;
}

void mstress_free_server(mstress_server S) {
    if (!S) return;
    cudaStreamSynchronize(S->ctx->stream);
    delete S;
}

}  // extern "C"
