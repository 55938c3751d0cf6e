// Persistent cooperative Jacobi-PCG for the global stage (section 4.3, Eq. 20).
//
// One cooperative launch runs a whole PCG solve over every array of a batch.
// Each iteration has three phases separated by a grid barrier:
//   A  element products Y_e = A_element p_e (p = z + beta p formed in the
//      gather), on FP64 CUDA cores, reduced-precision CUDA cores or tcgen05;
//   B  interface sum q = sum_e G_e^T Y_e, p stored, <p,q> partials; the CTA that
//      completes an array's last work item folds that array's partials in a
//      fixed order and stores alpha = <r,z>/<p,q>;
//   C  x += alpha p, r -= alpha q, z = D^-1 r and the <r,z>, <r,r> partials,
//      folded the same way into beta, the stopping test and the iteration count.
// The folds are ordered by work-item index only, so an array's arithmetic is
// the same alone and inside any batch. The grid barrier and the tensor-core
// completion wait both spin with an iteration limit; on expiry the kernel
// records an error, releases its tensor memory and returns.
#include <algorithm>

#include "apply_items.cuh"
#include "pcg_items.cuh"

namespace ms {
namespace {

enum { AM_FP64 = 0, AM_TC = 1, AM_SIMT32 = 2 };
constexpr int kPT = 256;   // threads per CTA

struct PcgArgs {
    ApplyArgs ap;              // x = p, z = z, st, Y
    int apply_items, panels;   // work items of phase A; row panels per 32-block tile (CUDA-core apply)
    ai::TcShape sh;
    const VecWork* vwork;
    int n_vwork;
    const ArrayDev* arrays;
    int n_arrays;
    const LocalMap* lm;
    const double* dinv;
    void *x, *r, *z, *p, *q;
    PcgState* st;
    double *part_pq, *part_rz, *part_rr;
    int* tickets;              // 2 per array: phase B, phase C
    unsigned* bar;             // [0] arrivals, [1] generation
    int* n_active;             // arrays still iterating
    int* err;                  // 1: tensor-core wait expired, 2: grid barrier expired
    int* abort;
    int max_loops;
    unsigned long long* timers;   // optional: ns spent in phases A, B, C and the loop count
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// CTA 0 accumulates the wall time of a phase (from its start to the end of
// the grid barrier that closes it) into timers[phase].
__device__ __forceinline__ void phase_mark(const PcgArgs& a, int phase, unsigned long long& t_prev) {
    if (a.timers && blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned long long t = global_ns();
        a.timers[phase] += t - t_prev;
        t_prev = t;
    }
}

// Grid-wide barrier with a bounded wait. Returns false (in every thread of the
// CTA) when the grid is aborting or the wait expired.
__device__ __forceinline__ bool grid_sync(const PcgArgs& a, int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* gen = a.bar + 1;
        const unsigned g = *gen;            // read before arriving: cannot advance without us
        __threadfence();
        const unsigned arrived = atomicAdd(a.bar, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(a.bar, 0u);
            __threadfence();
            atomicAdd(a.bar + 1, 1u);
        } else {
            long long spins = 0;
            while (*gen == g) {
                if (*(volatile int*)a.abort) { ok = 0; break; }
                if (++spins > (1LL << 25)) {
                    atomicExch(a.err, 2);
                    atomicExch(a.abort, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        if (*(volatile int*)a.abort) ok = 0;
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

template <class V, int AM, int MODE, int RPT>
__global__ void __launch_bounds__(kPT) k_pcg(const __grid_constant__ PcgArgs a) {
    extern __shared__ uint8_t smraw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    __shared__ long long base[kTileTC];
    __shared__ int offs[3 * kMaxSurf];
    __shared__ double shr[kPT / 32], sh8[8];
    __shared__ int s_flag, s_ok;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x;
    constexpr int NS = MODE == MSTRESS_BF16X3 ? 2 : 1;
    ai::TcState ts;
    if (AM == AM_TC) {
        ts.sB = smem;
        ts.sA = smem + NS * a.sh.b_plane;
        for (uint32_t i = tid; i < NS * a.sh.a_plane / 16; i += kPT)
            reinterpret_cast<uint4*>(ts.sA)[i] = make_uint4(0, 0, 0, 0);
        if ((tid >> 5) == 0) tc::tmem_alloc(&tmem_base, (uint32_t)a.sh.tmem_cols);
        if (tid == 0) tc::mbar_init(&mbar, 1);
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        ts.tmem = tmem_base;
        ts.mbar = &mbar;
        ts.phase = 0;
        ts.cur_type = -1;
    }
    V* x = static_cast<V*>(a.x);
    V* r = static_cast<V*>(a.r);
    V* z = static_cast<V*>(a.z);
    V* p = static_cast<V*>(a.p);
    V* q = static_cast<V*>(a.q);
    unsigned long long t_prev = (a.timers && blockIdx.x == 0 && tid == 0) ? global_ns() : 0ull;
    for (int loop = 0; loop < a.max_loops; ++loop) {
        // ---- phase A: element products
        bool failed = false;
        for (int w = blockIdx.x; w < a.apply_items; w += gridDim.x) {
            if constexpr (AM == AM_TC) {
                const ApplyWork it = a.ap.work[w];
                if (!a.st[it.array].active) continue;
                if (!ai::apply_tc_item<MODE>(a.ap, a.sh, it, ts, base, offs)) {
                    failed = true;
                    break;
                }
            } else {
                const ApplyWork it = a.ap.work[w / a.panels];
                if (!a.st[it.array].active) continue;
                __syncthreads();
                if constexpr (AM == AM_FP64)
                    ai::apply64_item<RPT>(a.ap, it, w % a.panels, reinterpret_cast<double*>(smem),
                                          reinterpret_cast<double*>(smem) + (size_t)a.ap.m * kTile64, base, offs);
                else
                    ai::apply32_item<RPT, MODE>(a.ap, it, w % a.panels, reinterpret_cast<float*>(smem),
                                                reinterpret_cast<float*>(smem) + (size_t)NS * a.ap.m * kTile64, base,
                                                offs);
            }
        }
        if (failed && tid == 0) {
            atomicExch(a.err, 1);
            atomicExch(a.abort, 1);
        }
        if (!grid_sync(a, &s_ok)) break;
        phase_mark(a, 0, t_prev);
        // ---- phase B: interface sum, <p, q>, alpha
        for (int w = blockIdx.x; w < a.n_vwork; w += gridDim.x) {
            const VecWork it = a.vwork[w];
            const int k = it.array;
            if (!a.st[k].active) continue;
            const ArrayDev A = a.arrays[k];
            const double acc = pi::isum_item<V, V>(it, A, a.lm, a.dinv, a.ap.ldY, static_cast<const V*>(a.ap.Y), p, z,
                                                   q, a.st[k].beta);
            const double t = pi::block_sum(acc, shr);
            if (tid == 0) {
                a.part_pq[w] = t;
                __threadfence();
                s_flag = atomicAdd(&a.tickets[2 * k], 1) == A.n_vwork - 1;
            }
            __syncthreads();
            if (s_flag) {
                __threadfence();
                const double pq = pi::cta_fold8(a.part_pq + A.vwork_off, A.n_vwork, sh8);
                if (tid == 0) {
                    a.tickets[2 * k] = 0;
                    const double al = a.st[k].rz / pq;
                    if (!(pq > 0) || !isfinite(al)) {
                        a.st[k].alpha = 0.0;
                        a.st[k].active = 0;
                        a.st[k].status = MSTRESS_ENUMERIC;
                        atomicSub(a.n_active, 1);
                    } else {
                        a.st[k].alpha = al;
                    }
                }
            }
            __syncthreads();
        }
        if (!grid_sync(a, &s_ok)) break;
        phase_mark(a, 1, t_prev);
        // ---- phase C: vector update, <r,z>, <r,r>, beta, stopping test
        for (int w = blockIdx.x; w < a.n_vwork; w += gridDim.x) {
            const VecWork it = a.vwork[w];
            const int k = it.array;
            if (!a.st[k].active) continue;
            const ArrayDev A = a.arrays[k];
            double srz, srr;
            pi::vec1_item<V>(it, a.dinv, a.st[k].alpha, x, r, z, p, q, srz, srr);
            srz = pi::block_sum(srz, shr);
            srr = pi::block_sum(srr, shr);
            if (tid == 0) {
                a.part_rz[w] = srz;
                a.part_rr[w] = srr;
                __threadfence();
                s_flag = atomicAdd(&a.tickets[2 * k + 1], 1) == A.n_vwork - 1;
            }
            __syncthreads();
            if (s_flag) {
                __threadfence();
                const double rz = pi::cta_fold8(a.part_rz + A.vwork_off, A.n_vwork, sh8);
                const double rr = pi::cta_fold8(a.part_rr + A.vwork_off, A.n_vwork, sh8);
                if (tid == 0) {
                    a.tickets[2 * k + 1] = 0;
                    PcgState s = a.st[k];
                    s.iters += 1;
                    if (!isfinite(rz) || !isfinite(rr)) {
                        s.active = 0;
                        s.status = MSTRESS_ENUMERIC;
                    } else {
                        s.beta = rz / s.rz;
                        s.rz = rz;
                        s.rr = rr;
                        if (rr <= s.tol2) { s.active = 0; s.status = MSTRESS_OK; }
                        else if (s.iters >= s.max_iter) { s.active = 0; s.status = MSTRESS_ENOT_CONVERGED; }
                    }
                    a.st[k] = s;
                    if (!s.active) atomicSub(a.n_active, 1);
                }
            }
            __syncthreads();
        }
        if (!grid_sync(a, &s_ok)) break;
        phase_mark(a, 2, t_prev);
        if (a.timers && blockIdx.x == 0 && tid == 0) a.timers[3] += 1;
        if (*(volatile int*)a.n_active <= 0) break;
    }
    if (AM == AM_TC) {
        if (*(volatile int*)a.abort) tc::mbar_wait(&mbar, ts.phase ^ 1u, 1 << 20);   // bounded drain
        tc::fence_before();
        __syncthreads();
        if ((tid >> 5) == 0) tc::tmem_free(ts.tmem, (uint32_t)a.sh.tmem_cols);
    }
}

template <class KER>
bool launch_coop(KER kernel, mstress_sol_s* s, PcgArgs& a, size_t smem, int needed, int tmem_cols) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) { cudaGetLastError(); return false; }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kPT, smem);
    if (e != cudaSuccess || per_sm < 1) { cudaGetLastError(); return false; }
    if (tmem_cols > 0) per_sm = std::min(per_sm, 512 / tmem_cols);
    const int grid = std::max(1, std::min(needed, per_sm * s->ctx->num_sms));
    void* args[] = {&a};
    e = cudaLaunchCooperativeKernel((void*)kernel, grid, kPT, args, smem, s->ctx->stream);
    if (e != cudaSuccess) { cudaGetLastError(); return false; }
    note_launches(1);
    return true;
}

}  // namespace

// Run a whole PCG solve (already started: x, r, z, p and the per-array
// scalars set) as one cooperative launch. Returns false when the launch is not
// possible, so that the caller falls back to per-phase launches.
bool pcg_run_persistent(mstress_sol_s* s, PcgVectors& v, int prec, int max_iter, bool vec_fp32) {
    PcgArgs a;
    std::memset(&a, 0, sizeof(a));
    const bool tc = vec_fp32 && s->use_tc;
    a.ap = apply_args(s, v.p.ptr, v.z.ptr, v.state.as<PcgState>(), s->Y.ptr, tc);
    a.vwork = s->d_vwork.as<VecWork>();
    a.n_vwork = s->n_vwork;
    a.arrays = s->d_arrays.as<ArrayDev>();
    a.n_arrays = s->n_arrays;
    a.lm = s->d_lm.as<LocalMap>();
    a.dinv = s->dinv.as<double>();
    a.x = v.x.ptr;
    a.r = v.r.ptr;
    a.z = v.z.ptr;
    a.p = v.p.ptr;
    a.q = v.q.ptr;
    a.st = v.state.as<PcgState>();
    a.part_pq = s->part.as<double>();
    a.part_rz = a.part_pq + s->n_vwork;
    a.part_rr = a.part_rz + s->n_vwork;
    a.tickets = s->tickets.as<int>();
    int* flag = s->flag.as<int>();
    a.err = flag + 2;
    a.n_active = flag + 4;
    a.bar = reinterpret_cast<unsigned*>(flag + 5);
    a.abort = flag + 7;
    a.max_loops = max_iter + 1;
    a.timers = s->timers.as<unsigned long long>();
    MS_CUDA(cudaMemsetAsync(flag + 5, 0, 3 * sizeof(int), s->ctx->stream));
    MS_CUDA(cudaMemsetAsync(s->tickets.ptr, 0, s->tickets.bytes, s->ctx->stream));
    const int m = s->m;
    const int vneed = s->n_vwork;
    if (!vec_fp32) {
        if (m <= 80) {
            a.panels = (m + 15) / 16;
            a.apply_items = s->n_awork * a.panels;
            const size_t smem = (size_t)(m * kTile64 + 16 * m) * sizeof(double) + 1024;
            return launch_coop(k_pcg<double, AM_FP64, MSTRESS_FP64, 2>, s, a, smem, std::max(a.apply_items, vneed), 0);
        }
        a.panels = (m + 31) / 32;
        a.apply_items = s->n_awork * a.panels;
        const size_t smem = (size_t)(m * kTile64 + 32 * m) * sizeof(double) + 1024;
        return launch_coop(k_pcg<double, AM_FP64, MSTRESS_FP64, 4>, s, a, smem, std::max(a.apply_items, vneed), 0);
    }
    if (tc) {
        a.sh = tc_shape(m, prec);
        a.apply_items = s->n_awork_tc;
        a.panels = 1;
        const int need = std::max(a.apply_items, vneed);
        switch (prec) {
            case MSTRESS_TF32:
                return launch_coop(k_pcg<float, AM_TC, MSTRESS_TF32, 0>, s, a, a.sh.smem, need, a.sh.tmem_cols);
            case MSTRESS_BF16:
                return launch_coop(k_pcg<float, AM_TC, MSTRESS_BF16, 0>, s, a, a.sh.smem, need, a.sh.tmem_cols);
            default:
                return launch_coop(k_pcg<float, AM_TC, MSTRESS_BF16X3, 0>, s, a, a.sh.smem, need, a.sh.tmem_cols);
        }
    }
    const int ns = prec == MSTRESS_BF16X3 ? 2 : 1;
    const int rpt = m <= 80 ? 2 : 4;
    a.panels = (m + 8 * rpt - 1) / (8 * rpt);
    a.apply_items = s->n_awork * a.panels;
    const size_t smem = (size_t)ns * (m * kTile64 + 8 * rpt * m) * sizeof(float) + 1024;
    const int need = std::max(a.apply_items, vneed);
    if (rpt == 2) {
        if (prec == MSTRESS_TF32) return launch_coop(k_pcg<float, AM_SIMT32, MSTRESS_TF32, 2>, s, a, smem, need, 0);
        if (prec == MSTRESS_BF16) return launch_coop(k_pcg<float, AM_SIMT32, MSTRESS_BF16, 2>, s, a, smem, need, 0);
        return launch_coop(k_pcg<float, AM_SIMT32, MSTRESS_BF16X3, 2>, s, a, smem, need, 0);
    }
    if (prec == MSTRESS_TF32) return launch_coop(k_pcg<float, AM_SIMT32, MSTRESS_TF32, 4>, s, a, smem, need, 0);
    if (prec == MSTRESS_BF16) return launch_coop(k_pcg<float, AM_SIMT32, MSTRESS_BF16, 4>, s, a, smem, need, 0);
    return launch_coop(k_pcg<float, AM_SIMT32, MSTRESS_BF16X3, 4>, s, a, smem, need, 0);
}

}  // namespace ms
