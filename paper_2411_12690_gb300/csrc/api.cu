// C-ABI entry points for contexts and block models, device-memory budget,
// and the surface-node map shared by all kernels.
#include <atomic>
#include <cstdio>

#include "internal.h"

using namespace ms;

// ------------------------------------------------------------- memory
void mstress_ctx_s::budget_check(size_t bytes) const {
    if (opts.hbm_budget && in_use + bytes > opts.hbm_budget)
        throw Error{MSTRESS_ENOMEM, "HBM budget exceeded: holding " + std::to_string(in_use) +
                                        " B, asked " + std::to_string(bytes) + " B, budget " +
                                        std::to_string(opts.hbm_budget) + " B"};
}

namespace {
constexpr size_t kAllocGrain = 512;
constexpr size_t kCacheCap = size_t(8) << 30;   // freed bytes kept for reuse at most
}  // namespace

void* mstress_ctx_s::alloc(size_t bytes) {
    bytes = round_up(bytes == 0 ? 16 : bytes, kAllocGrain);
    budget_check(bytes);
    void* p = nullptr;
    size_t got = bytes;
    auto it = cache.lower_bound(bytes);
    if (it != cache.end() && it->first <= 2 * bytes) {
        // a block freed earlier on this context's stream: wait (normally a
        // no-op) until the work that used it is done, then reuse it
        if (cudaEventQuery(it->second.ev) != cudaSuccess) cudaEventSynchronize(it->second.ev);
        cudaEventDestroy(it->second.ev);
        p = it->second.p;
        got = it->first;
        cached -= got;
        cache.erase(it);
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            trim(0);
            e = cudaMalloc(&p, bytes);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw Error{MSTRESS_ENOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e)};
        }
    }
    allocs[p] = got;
    in_use += got;
    if (in_use > peak) peak = in_use;
    return p;
}

void mstress_ctx_s::release(void* p) {
    auto it = allocs.find(p);
    if (it == allocs.end()) return;
    const size_t bytes = it->second;
    in_use -= bytes;
    allocs.erase(it);
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ev, stream) != cudaSuccess) {
        cudaGetLastError();
        if (ev) cudaEventDestroy(ev);
        cudaFree(p);
        return;
    }
    cache.insert({bytes, Cached{p, ev}});
    cached += bytes;
    if (cached > kCacheCap) trim(kCacheCap / 2);
}

void mstress_ctx_s::trim(size_t keep) {
    while (cached > keep && !cache.empty()) {
        auto it = std::prev(cache.end());   // largest first
        cudaEventSynchronize(it->second.ev);
        cudaEventDestroy(it->second.ev);
        cudaFree(it->second.p);
        cached -= it->first;
        cache.erase(it);
    }
}

namespace ms {

static std::atomic<long long> g_launches{0};
thread_local bool g_capturing = false;
void note_launches(long long n) {
    if (!g_capturing) g_launches.fetch_add(n, std::memory_order_relaxed);
}

DBuf& DBuf::operator=(DBuf&& o) noexcept {
    if (this != &o) {
        reset();
        ctx = o.ctx;
        ptr = o.ptr;
        bytes = o.bytes;
        o.ctx = nullptr;
        o.ptr = nullptr;
        o.bytes = 0;
    }
    return *this;
}

void DBuf::reset() {
    if (ptr && ctx) ctx->release(ptr);
    ptr = nullptr;
    bytes = 0;
}

void alloc_into(mstress_ctx ctx, DBuf& b, size_t bytes, bool zero) {
    b.reset();
    b.ptr = ctx->alloc(bytes);
    b.ctx = ctx;
    b.bytes = bytes;
    if (zero) MS_CUDA(cudaMemsetAsync(b.ptr, 0, bytes, ctx->stream));
}

LocalMap make_local_map(int n) {
    LocalMap lm;
    std::memset(&lm, 0, sizeof(lm));
    MS_REQUIRE(n >= 2 && n <= kMaxN, MSTRESS_EINVAL, "basis order must be in [1, 7]");
    lm.n = n;
    int q = 0;
    for (int c = 0; c < n; ++c)
        for (int b = 0; b < n; ++b)
            for (int a = 0; a < n; ++a) {
                bool surf = a == 0 || a == n - 1 || b == 0 || b == n - 1 || c == 0 || c == n - 1;
                lm.surf_idx[(c * n + b) * n + a] = surf ? (int16_t)q : (int16_t)-1;
                if (surf) {
                    lm.qa[q] = (uint8_t)a;
                    lm.qb[q] = (uint8_t)b;
                    lm.qc[q] = (uint8_t)c;
                    ++q;
                }
            }
    lm.nsurf = q;
    lm.m = 3 * q;
    return lm;
}

}  // namespace ms

// ------------------------------------------------------------ helpers
#define MS_API_BEGIN try {
#define MS_API_END(ctx)                                        \
    }                                                          \
    catch (const ms::Error& e) {                               \
        if (ctx) (ctx)->last_error = e.msg;                    \
        return e.code;                                         \
    }                                                          \
    catch (const std::exception& e) {                          \
        if (ctx) (ctx)->last_error = e.what();                 \
        return MSTRESS_EINVAL;                                 \
    }                                                          \
    return MSTRESS_OK;

extern "C" {

int mstress_opts_default(mstress_opts* o) {
    if (!o) return MSTRESS_EINVAL;
    std::memset(o, 0, sizeof(*o));
    o->precision = MSTRESS_FP64;
    o->rtol = 1e-13;
    o->max_iter = 20000;
    o->inner_rtol = 0.0;   // per precision (see inner_tolerance)
    o->max_outer = 30;
    o->hbm_budget = 0;
    o->offline_max_iter = 20000;
    o->offline_rtol = 1e-13;
    return MSTRESS_OK;
}

static int check_opts(const mstress_opts* o, std::string& why) {
    if (o->precision < MSTRESS_FP64 || o->precision > MSTRESS_BF16X3) { why = "unknown precision mode"; return 0; }
    if (!(o->rtol > 0 && o->rtol < 1)) { why = "rtol must be in (0, 1)"; return 0; }
    if (o->max_iter < 1) { why = "max_iter must be >= 1"; return 0; }
    if (!(o->inner_rtol >= 0 && o->inner_rtol < 1)) { why = "inner_rtol must be in [0, 1)"; return 0; }
    if (o->max_outer < 1) { why = "max_outer must be >= 1"; return 0; }
    if (o->offline_max_iter < 1) { why = "offline_max_iter must be >= 1"; return 0; }
    if (!(o->offline_rtol > 0 && o->offline_rtol < 1)) { why = "offline_rtol must be in (0, 1)"; return 0; }
    return 1;
}

int mstress_create(mstress_ctx* out, void* cuda_stream, const mstress_opts* opts) {
    if (!out) return MSTRESS_EINVAL;
    *out = nullptr;
    mstress_ctx ctx = new mstress_ctx_s();
    MS_API_BEGIN
    if (opts) ctx->opts = *opts; else mstress_opts_default(&ctx->opts);
    std::string why;
    MS_REQUIRE(check_opts(&ctx->opts, why), MSTRESS_EINVAL, why);
    MS_CUDA(cudaGetDevice(&ctx->device));
    MS_CUDA(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device));
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    MS_CUDA(cudaHostAlloc((void**)&ctx->h_flag, 64, cudaHostAllocDefault));
    *out = ctx;
    }
    catch (const ms::Error& e) {
        int code = e.code;
        std::fprintf(stderr, "mstress_create: %s\n", e.msg.c_str());
        delete ctx;
        return code;
    }
    return MSTRESS_OK;
}

int mstress_set_opts(mstress_ctx ctx, const mstress_opts* opts) {
    if (!ctx || !opts) return MSTRESS_EINVAL;
    std::string why;
    if (!check_opts(opts, why)) { ctx->last_error = why; return MSTRESS_EINVAL; }
    ctx->opts = *opts;
    return MSTRESS_OK;
}

int mstress_get_opts(mstress_ctx ctx, mstress_opts* opts) {
    if (!ctx || !opts) return MSTRESS_EINVAL;
    *opts = ctx->opts;
    return MSTRESS_OK;
}

void mstress_free_ctx(mstress_ctx ctx) {
    if (!ctx) return;
    if (ctx->stream || true) cudaStreamSynchronize(ctx->stream);
    for (auto& kv : ctx->allocs) cudaFree(kv.first);
    ctx->allocs.clear();
    ctx->trim(0);
    if (ctx->h_flag) cudaFreeHost(ctx->h_flag);
    if (ctx->h_states) cudaFreeHost(ctx->h_states);
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    delete ctx;
}

int mstress_strip_partition(int ny, int order, int world, int rank, mstress_strip* out) {
    if (!out || ny < 1 || order < 1 || order > 7 || world < 1 || rank < 0 || rank >= world || world > ny)
        return MSTRESS_EINVAL;
    const int n1 = order;   // lattice rows per block row
    const int base = ny / world, extra = ny % world;
    const int j0 = rank * base + std::min(rank, extra);
    const int j1 = j0 + base + (rank < extra ? 1 : 0);
    const bool last = rank == world - 1;
    out->j0 = j0;
    out->j1 = j1;
    out->y_own0 = j0 * n1;
    out->y_own1 = last ? ny * n1 + 1 : j1 * n1;
    out->y_send = last ? -1 : j1 * n1;
    out->y_recv = rank == 0 ? -1 : j0 * n1;
    out->prev = rank == 0 ? -1 : rank - 1;
    out->next = last ? -1 : rank + 1;
    return MSTRESS_OK;
}

const char* mstress_last_error(mstress_ctx ctx) {
    if (!ctx) return "null context";
    return ctx->last_error.c_str();
}

int mstress_mem_info(mstress_ctx ctx, size_t* in_use, size_t* peak) {
    if (!ctx) return MSTRESS_EINVAL;
    if (in_use) *in_use = ctx->in_use;
    if (peak) *peak = ctx->peak;
    return MSTRESS_OK;
}

int mstress_launch_count(int64_t* n) {
    if (!n) return MSTRESS_EINVAL;
    *n = ms::g_launches.load();
    return MSTRESS_OK;
}

int mstress_sync(mstress_ctx ctx) {
    if (!ctx) return MSTRESS_EINVAL;
    MS_API_BEGIN
    MS_CUDA(cudaStreamSynchronize(ctx->stream));
    MS_API_END(ctx)
}

int mstress_build_block(mstress_ctx ctx, const mstress_block_mesh* mesh, const mstress_tsv_geom* tsv,
                        const mstress_material* mats, int n_mat, int order, mstress_block* out) {
    if (!ctx) return MSTRESS_EINVAL;
    if (!out) { ctx->last_error = "out is NULL"; return MSTRESS_EINVAL; }
    *out = nullptr;
    MS_API_BEGIN
    return ms::build_block(ctx, mesh, tsv, mats, n_mat, order, out);
    MS_API_END(ctx)
}

static void check_mesh(const mstress_block_mesh* mesh) {
    MS_REQUIRE(mesh, MSTRESS_EINVAL, "mesh is NULL");
    MS_REQUIRE(mesh->ex >= 1 && mesh->ey >= 1 && mesh->ez >= 1, MSTRESS_EINVAL, "mesh needs >= 1 element per axis");
    MS_REQUIRE((int64_t)mesh->ex * mesh->ey * mesh->ez <= (1 << 24), MSTRESS_EINVAL, "mesh too large");
    MS_REQUIRE(mesh->lx > 0 && mesh->ly > 0 && mesh->lz > 0, MSTRESS_EINVAL, "block lengths must be positive");
}

int mstress_block_import(mstress_ctx ctx, const mstress_block_mesh* mesh, int order, const double* K_r,
                         const double* b_r, const double* S, const double* F, mstress_block* out) {
    if (!ctx) return MSTRESS_EINVAL;
    if (!out) { ctx->last_error = "out is NULL"; return MSTRESS_EINVAL; }
    *out = nullptr;
    std::unique_ptr<mstress_block_s> blk(new mstress_block_s());
    MS_API_BEGIN
    check_mesh(mesh);
    MS_REQUIRE(K_r && b_r && S, MSTRESS_EINVAL, "K_r, b_r and S are required");
    LocalMap lm = make_local_map(order + 1);
    mstress_block_s& B = *blk;
    B.ctx = ctx;
    B.n = order + 1;
    B.m = lm.m;
    B.m1 = lm.m + 1;
    B.ld = (int)round_up(B.m1, 8);
    B.ex = mesh->ex; B.ey = mesh->ey; B.ez = mesh->ez;
    B.lx = mesh->lx; B.ly = mesh->ly; B.lz = mesh->lz;
    B.n_el = B.ex * B.ey * B.ez;
    B.n_nodes = (B.ex + 1) * (B.ey + 1) * (B.ez + 1);
    B.n_dof = 3 * B.n_nodes;
    const size_t m = B.m, m1 = B.m1, ld = B.ld;
    alloc_into(ctx, B.Kr, m * m * sizeof(double), false);
    alloc_into(ctx, B.br, m * sizeof(double), false);
    alloc_into(ctx, B.S, (size_t)48 * B.n_el * ld * sizeof(double));
    alloc_into(ctx, B.Smean, (size_t)6 * B.n_el * ld * sizeof(double));
    MS_CUDA(cudaMemcpyAsync(B.Kr.ptr, K_r, m * m * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    MS_CUDA(cudaMemcpyAsync(B.br.ptr, b_r, m * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    MS_CUDA(cudaMemcpy2DAsync(B.S.ptr, ld * sizeof(double), S, m1 * sizeof(double), m1 * sizeof(double),
                              (size_t)48 * B.n_el, cudaMemcpyHostToDevice, ctx->stream));
    if (F) {
        alloc_into(ctx, B.F, (size_t)B.n_dof * ld * sizeof(double));
        MS_CUDA(cudaMemcpy2DAsync(B.F.ptr, ld * sizeof(double), F, m1 * sizeof(double), m1 * sizeof(double),
                                  (size_t)B.n_dof, cudaMemcpyHostToDevice, ctx->stream));
        B.has_F = true;
    }
    block_compute_smean(&B);
    MS_CUDA(cudaStreamSynchronize(ctx->stream));
    *out = blk.release();
    MS_API_END(ctx)
}

int mstress_block_export(mstress_block blk, int what, double* dst, size_t count) {
    if (!blk) return MSTRESS_EINVAL;
    mstress_ctx ctx = blk->ctx;
    MS_API_BEGIN
    MS_REQUIRE(dst, MSTRESS_EINVAL, "dst is NULL");
    const size_t m = blk->m, m1 = blk->m1, ld = blk->ld;
    const void* src = nullptr;
    size_t rows = 0, cols = 0, spitch = 0;
    switch (what) {
        case MSTRESS_BLOCK_KR: src = blk->Kr.ptr; rows = m; cols = m; spitch = m; break;
        case MSTRESS_BLOCK_BR: src = blk->br.ptr; rows = 1; cols = m; spitch = m; break;
        case MSTRESS_BLOCK_S: src = blk->S.ptr; rows = (size_t)48 * blk->n_el; cols = m1; spitch = ld; break;
        case MSTRESS_BLOCK_SMEAN: src = blk->Smean.ptr; rows = (size_t)6 * blk->n_el; cols = m1; spitch = ld; break;
        case MSTRESS_BLOCK_SGRID:
            MS_REQUIRE(blk->n_grid > 0, MSTRESS_EINVAL, "no grid modes: call mstress_block_grid first");
            src = blk->Sgrid.ptr; rows = (size_t)6 * blk->n_grid; cols = m1; spitch = ld; break;
        case MSTRESS_BLOCK_F:
            MS_REQUIRE(blk->has_F, MSTRESS_EINVAL, "block holds no basis F");
            src = blk->F.ptr; rows = blk->n_dof; cols = m1; spitch = ld; break;
        default: throw Error{MSTRESS_EINVAL, "unknown block array"};
    }
    MS_REQUIRE(count >= rows * cols, MSTRESS_EINVAL, "dst too small");
    MS_CUDA(cudaMemcpy2DAsync(dst, cols * sizeof(double), src, spitch * sizeof(double), cols * sizeof(double),
                              rows, cudaMemcpyDeviceToHost, ctx->stream));
    MS_CUDA(cudaStreamSynchronize(ctx->stream));
    MS_API_END(ctx)
}

int mstress_block_grid(mstress_block blk, int side) {
    if (!blk) return MSTRESS_EINVAL;
    mstress_ctx ctx = blk->ctx;
    MS_API_BEGIN
    build_grid_modes(blk, side);
    MS_CUDA(cudaStreamSynchronize(ctx->stream));
    MS_API_END(ctx)
}

int mstress_block_info(mstress_block blk, int* m, int* n_el, int* n_dof, int* cg_iters) {
    if (!blk) return MSTRESS_EINVAL;
    if (m) *m = blk->m;
    if (n_el) *n_el = blk->n_el;
    if (n_dof) *n_dof = blk->n_dof;
    if (cg_iters) *cg_iters = blk->cg_iters;
    return MSTRESS_OK;
}

void mstress_free_block(mstress_block blk) {
    if (!blk) return;
    cudaStreamSynchronize(blk->ctx->stream);
    delete blk;
}

}  // extern "C"
