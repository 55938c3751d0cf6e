// Persistent cooperative Jacobi-PCG for the global stage (section 4.3, Eq. 20).
//
// One cooperative launch runs a whole PCG solve over every array of a batch.
// With the resident tensor-core apply (small bases) an iteration has two
// phases separated by a grid barrier:
//   A  element products Y_e = A_element p_e (p = z + beta p formed in the
//      gather) and, in the epilogue, p_e^T Y_e summed per 8-block group;
//      alpha = <r,z> / sum_e p_e^T Y_e (= <p, A p>) is folded from the group
//      sums in a fixed order;
//   B  interface sum and vector update in one pass: p = z + beta p, q = sum_e
//      G_e^T Y_e (not stored), x += alpha p, r -= alpha q, z = D^-1 r and the
//      <r,z>, <r,r> partials, folded into beta, the stopping test and the
//      iteration count.
// p and z are kept as (p, z) pairs, so that the gather of phase A reads both
// with one load.
// Otherwise an iteration has three phases separated by a grid barrier:
//   A  element products Y_e = A_element p_e (p = z + beta p formed in the
//      gather), on FP64 CUDA cores, reduced-precision CUDA cores or tcgen05;
//   B  interface sum q = sum_e G_e^T Y_e, p stored, <p,q> partials; the CTA that
//      completes an array's last work item folds that array's partials in a
//      fixed order and stores alpha = <r,z>/<p,q>;
//   C  x += alpha p, r -= alpha q, z = D^-1 r and the <r,z>, <r,r> partials,
//      folded the same way into beta, the stopping test and the iteration count.
// The folds are ordered by work-item index only, so an array's arithmetic is
// the same alone and inside any batch. A CTA reports its finished work items
// of an array with one atomic per array per phase (not one per item), and
// reads an array's scalars once per phase. The grid barrier is one growing
// arrival counter and, like the tensor-core completion waits, spins with an
// iteration limit; on expiry the kernel records an error, releases its tensor
// memory and returns.
#include <algorithm>

#include "apply_items.cuh"
#include "pcg_items.cuh"

namespace ms {
namespace {

enum { AM_FP64 = 0, AM_TC = 1, AM_SIMT32 = 2, AM_TCS = 3 };

struct PcgArgs {
    ApplyArgs ap;              // x = p, z = z, st, Y
    int apply_items, panels;   // work items of phase A; row panels per 32-block tile (CUDA-core apply)
    ai::TcShape sh;
    ai::TcsShape shs;          // streamed tensor-core apply (large bases)
    const VecWork* vwork;
    int n_vwork;
    const ArrayDev* arrays;
    int n_arrays;
    const LocalMap* lm;
    const void* dinv;          // Jacobi inverse in the vector precision
    void *x, *r, *z, *p, *q;
    PcgState* st;
    double *part_pq, *part_rz, *part_rr;
    int* tickets;              // 2 per array: the alpha fold (phase B, or A when two-phase), the beta fold
    unsigned* bar;             // grid-barrier arrival counter (zero at launch)
    int* n_active;             // arrays still iterating
    int* err;                  // 1: tensor-core wait expired, 2: grid barrier expired
    int* abort;
    int max_loops;
    int resident;              // two-phase iteration, one array: vector slices may stay in shared memory
    long long wait_limit_ns;   // a grid-barrier wait gives up after this long
    int withhold_cta;          // this CTA skips its first barrier arrival (test hook), or -1
    unsigned long long* timers;   // optional: ns spent in phases A, B, C and the loop count (two-phase
                                  // iteration: A, B, and C = 0)
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// CTA 0 accumulates the wall time of a phase (from its start to the end of
// the grid barrier that closes it) in registers (acc[phase]); they are added
// to timers[] once, when the kernel ends, so that no global memory round trip
// joins the iteration's critical path.
__device__ __forceinline__ void phase_mark(const PcgArgs& a, int phase, unsigned long long& t_prev,
                                           unsigned long long (&acc)[4]) {
    if (a.timers && blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned long long t = global_ns();
        acc[phase] += t - t_prev;
        t_prev = t;
    }
}

// Grid barrier with a bounded wait, on kBarLanes arrival counters that only
// grow (128 bytes apart, so that the CTAs' atomics spread over several L2
// lines instead of queueing on one): CTA c adds 1 to counter c % kBarLanes in
// every barrier, and the k-th barrier of a launch is passed when counter j
// has reached k * n_j, n_j = the number of CTAs with c % kBarLanes == j
// (compared as signed differences, so the counters may wrap). Lane j of the
// CTA's first warp polls counter j. A wait longer than wait_limit_ns (device
// clock) gives up: it records the error, raises the abort flag that every
// other waiting CTA polls, and the kernel returns. *k_bar is the CTA's
// barrier count (shared). Returns false (in every thread of the CTA) when the
// grid is aborting or the wait expired.
constexpr int kBarLanes = 8;
constexpr int kBarStride = 32;   // unsigned words between counters (128 bytes)

__device__ __forceinline__ bool grid_sync(const PcgArgs& a, int* s_ok, unsigned* k_bar) {
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const unsigned kb = *k_bar + 1u;   // this barrier's ordinal
        const bool withhold = kb == 1u && (int)blockIdx.x == a.withhold_cta;
        const unsigned G = gridDim.x;
        __syncwarp();
        if (lane == 0) {
            *k_bar = kb;
            __threadfence();
            if (!withhold) atomicAdd(a.bar + (blockIdx.x % kBarLanes) * kBarStride, 1u);
        }
        __syncwarp();
        int ok = 1;
        if (lane < kBarLanes) {
            const unsigned nj = lane < (int)G ? (G - 1u - (unsigned)lane) / kBarLanes + 1u : 0u;
            const unsigned target = kb * nj;
            volatile unsigned* ctr = a.bar + lane * kBarStride;
            long long spins = 0;
            unsigned long long t0 = 0;
            while ((int)(*ctr - target) < 0) {
                if (spins == 0) t0 = global_ns();
                if ((++spins & 63) == 0) {
                    if (*(volatile int*)a.abort) { ok = 0; break; }
                    if ((long long)(global_ns() - t0) > a.wait_limit_ns) {
                        atomicExch(a.err, 2);
                        atomicExch(a.abort, 1);
                        ok = 0;
                        break;
                    }
                }
                __nanosleep(32);
            }
            __threadfence();   // acquire: this lane observed its counter's arrivals
        }
        ok = __all_sync(0xffffffffu, ok);
        if (lane == 0) {
            __threadfence();
            if (*(volatile int*)a.abort) ok = 0;
            *s_ok = ok;
        }
    }
    __syncthreads();
    return *s_ok != 0;
}

// Per-CTA bookkeeping of the work items of the array being processed.
struct ArrayCursor {
    int k, count;   // array, items done by this CTA in this phase run
};

// RES: compiled for one array on resident vector slices only (the host checks
// the conditions: one array, a.resident, n_vwork no larger than the grid), so
// that the batch paths do not count against this variant's registers.
template <class V, int AM, int MODE, int RPT, int NT, int MINB, bool RES = false>
__global__ void __launch_bounds__(NT, MINB) k_pcg(const __grid_constant__ PcgArgs a) {
    extern __shared__ uint8_t smraw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    __shared__ long long base[kTileTC], s_eidx[kTileTC];
    __shared__ __align__(16) int offs[3 * kMaxSurf];
    __shared__ double shr[2 * (NT / 32)], sh8[16];
    __shared__ int s_flag, s_ok, s_active;
    __shared__ unsigned s_kbar;   // grid barriers passed by this CTA
    __shared__ double s_scalar, s_scalar2;
    __shared__ ArrayDev s_A;
    // one array: every CTA keeps the scalars itself (see below)
    __shared__ double s_rz, s_beta, s_alpha, s_tol2;
    __shared__ int s_iters, s_max_iter;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ __align__(8) uint64_t bars[3 * 4 + 2];
    __shared__ int s_tcs_fail;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x;
    constexpr int NS = MODE == MSTRESS_BF16X3 ? 2 : 1;
    ai::TcState ts;
    ai::TcsState tss;
    if constexpr (AM == AM_TCS) {
        ai::tcs_init(tss, a.shs, smem, bars, &s_tcs_fail);
        if ((tid >> 5) == 0) tc::tmem_alloc(&tmem_base, (uint32_t)a.shs.tmem_cols);
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        tss.tmem = tmem_base;
    }
    constexpr bool FUSED = AM == AM_TC;   // two-phase iteration (see the top of this file)
    if constexpr (AM == AM_TC) {
        ts.sB = smem;
        ts.sA = smem + NS * a.sh.b_plane;
        ts.sP = reinterpret_cast<float*>(ts.sA + NS * a.sh.a_plane);
        ts.ldp = a.sh.ldp;
        ts.sDot = reinterpret_cast<double*>(ts.sP + (size_t)kTileTC * a.sh.ldp);
        for (uint32_t i = tid; i < NS * a.sh.a_plane / 16; i += NT)
            reinterpret_cast<uint4*>(ts.sA)[i] = make_uint4(0, 0, 0, 0);
        for (uint32_t i = tid; i < (uint32_t)kTileTC * a.sh.ldp; i += NT) ts.sP[i] = 0.f;
        if ((tid >> 5) == 0) tc::tmem_alloc_c<128>(&tmem_base);   // npad <= 128 on this path
        if (tid == 0) tc::mbar_init(&mbar, 1);
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        ts.tmem = tmem_base;
        ts.mbar = &mbar;
        ts.phase = 0;
        ts.cur_type = -1;
        ts.eidx = s_eidx;
        ts.cached_start = -1;
        ts.cached_array = -1;
        ts.A_pre = nullptr;
        ts.beta_pre = nullptr;
    }
    V* x = static_cast<V*>(a.x);
    V* r = static_cast<V*>(a.r);
    V* z = static_cast<V*>(a.z);
    V* p = static_cast<V*>(a.p);
    V* q = static_cast<V*>(a.q);

    // Switch the cursor to array k: report the items finished for the previous
    // array (one atomic; the last reporter folds), then read k's scalars.
    // phase 1: fold <p,q> into alpha; phase 2: fold <r,z>, <r,r> into beta;
    // phase 3 (two-phase iteration, apply): fold the group sums of p_e^T Y_e
    // into alpha (items counted in 8-block groups).
    auto switch_array = [&](ArrayCursor& cur, int k, int phase) {
        if (cur.k >= 0 && cur.count > 0) {
            const int kk = cur.k;
            if (tid == 0) {
                __threadfence();
                const int old = atomicAdd(&a.tickets[2 * kk + (phase == 2 ? 1 : 0)], cur.count);
                s_flag = old + cur.count == (phase == 3 ? s_A.n_grp : s_A.n_vwork);
            }
            __syncthreads();
            if (s_flag) {
                __threadfence();
                if (phase != 2) {
                    const double pq = phase == 3 ? pi::cta_fold8(a.ap.gpart + s_A.grp_off, s_A.n_grp, sh8)
                                                 : pi::cta_fold8(a.part_pq + s_A.vwork_off, s_A.n_vwork, sh8);
                    if (tid == 0) {
                        a.tickets[2 * kk] = 0;
                        const double al = __ldcg(&a.st[kk].rz) / pq;
                        if (!(pq > 0) || !isfinite(al)) {
                            a.st[kk].alpha = 0.0;
                            a.st[kk].active = 0;
                            a.st[kk].status = MSTRESS_ENUMERIC;
                            atomicSub(a.n_active, 1);
                        } else {
                            a.st[kk].alpha = al;
                        }
                    }
                } else {
                    double rz, rr;
                    pi::cta_fold8_2(a.part_rz + s_A.vwork_off, a.part_rr + s_A.vwork_off, s_A.n_vwork, sh8, rz, rr);
                    if (tid == 0) {
                        a.tickets[2 * kk + 1] = 0;
                        PcgState s;
                        s.rz = __ldcg(&a.st[kk].rz);
                        s.tol2 = __ldcg(&a.st[kk].tol2);
                        s.iters = __ldcg(&a.st[kk].iters) + 1;
                        s.max_iter = __ldcg(&a.st[kk].max_iter);
                        int active = 1, status = MSTRESS_OK;
                        double beta = 0;
                        if (!isfinite(rz) || !isfinite(rr)) {
                            active = 0;
                            status = MSTRESS_ENUMERIC;
                        } else {
                            beta = rz / s.rz;
                            if (rr <= s.tol2) active = 0;
                            else if (s.iters >= s.max_iter) { active = 0; status = MSTRESS_ENOT_CONVERGED; }
                        }
                        a.st[kk].beta = beta;
                        a.st[kk].rz = rz;
                        a.st[kk].rr = rr;
                        a.st[kk].iters = s.iters;
                        a.st[kk].status = status;
                        a.st[kk].active = active;
                        if (!active) atomicSub(a.n_active, 1);
                    }
                }
            }
            __syncthreads();
        }
        cur.k = k;
        cur.count = 0;
        if (k >= 0) {
            if (tid == 0) {
                s_A = a.arrays[k];
                s_active = __ldcg(&a.st[k].active);
                s_scalar = phase == 2 ? __ldcg(&a.st[k].alpha) : __ldcg(&a.st[k].beta);
                s_scalar2 = __ldcg(&a.st[k].beta);
            }
            __syncthreads();
        }
    };

    // One array (a single solve): after each reducing phase's grid barrier every
    // CTA folds all partial sums itself, in the same fixed order as the
    // ticket path, and keeps alpha, beta, rz and the stopping decision in
    // shared memory. The scalars are bitwise those of the ticket path (so a
    // solve alone and in a batch still agree) without the ticket atomic, the
    // fold by the last CTA and the broadcast through global memory on the
    // critical path. Every CTA stores the same beta for its own next gather;
    // CTA 0 writes the rest of the state for the host. (Not compiled for the
    // streamed tensor-core apply, whose registers are fully used and whose
    // workloads are batches.)
    const bool solo = RES || (AM != AM_TCS && a.n_arrays == 1);
    if constexpr (AM == AM_TC) {
        if (solo) {   // one array: its descriptor and beta come from this CTA's shared copies
            ts.A_pre = &s_A;
            ts.beta_pre = &s_beta;
        }
    }
    // Resident vector slice (two-phase iteration, one array, at most one vector
    // work item per CTA): the CTA's item never changes during the solve, so its
    // x, r, D^-1 and owner offsets live in shared memory (after the tensor-core
    // buffers) and only p and z go through global memory.
    const bool resident = RES || (FUSED && solo && a.resident && a.n_vwork <= (int)gridDim.x);
    V *sVd = nullptr, *sVx = nullptr, *sVr = nullptr;
    int* sOff = nullptr;
    long long v_start = 0;
    int v_count = 0;
    if constexpr (FUSED) {
        if (resident) {
            uint8_t* q0 = reinterpret_cast<uint8_t*>(ts.sDot + (size_t)(a.sh.npad / 16) * kTileTC);
            sVd = reinterpret_cast<V*>(q0);
            sVx = sVd + kVecChunkTC;
            sVr = sVx + kVecChunkTC;
            sOff = reinterpret_cast<int*>(sVr + kVecChunkTC);
            if ((int)blockIdx.x < a.n_vwork) {
                const VecWork it = a.vwork[blockIdx.x];
                v_start = it.start;
                v_count = (int)it.count;
                if (tid == 0) s_A = a.arrays[0];
                __syncthreads();
                pi::resident_setup<V>(s_A, a.lm, a.ap.ldY, v_start, v_count, static_cast<const V*>(a.dinv), x, r,
                                      sVd, sVx, sVr, sOff, kVecChunkTC);
            }
            __syncthreads();
        }
    }
    if (tid == 0) {
        s_kbar = 0;   // read first by thread 0 itself in the first barrier
        if (solo) {
            s_A = a.arrays[0];
            s_rz = __ldcg(&a.st[0].rz);
            s_beta = __ldcg(&a.st[0].beta);
            s_tol2 = __ldcg(&a.st[0].tol2);
            s_iters = __ldcg(&a.st[0].iters);
            s_max_iter = __ldcg(&a.st[0].max_iter);
            s_active = __ldcg(&a.st[0].active);
            s_scalar = s_beta;
        }
    }
    __syncthreads();
    // the CTA's first tile, read once (every iteration starts with it)
    const ApplyWork first_tile = (AM == AM_TC && (int)blockIdx.x < a.apply_items) ? a.ap.work[blockIdx.x] : ApplyWork{};
    // Folds overlapped with loads (the RES variant: one array, resident
    // slices): the loads that do not need a fold's result are issued right
    // after the barrier that precedes the fold, and the arithmetic that needs
    // it follows the fold -- the next gather's (p, z) loads before the beta
    // fold (ov_a: the CTA's only tile, gathered in one round), the element
    // products and pairs of the CTA's slice before the alpha fold (ov_b: one
    // round). The same operations in the same order as without the overlap.
    constexpr int kGU = 12;
    constexpr int kRU = pi::kResidentU;
    bool ov_a = false, ov_b = false;
    float2 gw[kGU];
    float rs[kRU];
    float2 rpz[kRU];
    if constexpr (AM == AM_TC && RES) {
        ov_a = a.ap.pz && (int)blockIdx.x < a.apply_items && a.apply_items <= (int)gridDim.x &&
               a.sh.kpad * first_tile.count <= kGU * NT;
        ov_b = (int)blockIdx.x < a.n_vwork && v_count <= kRU * NT;
        if (ov_a) {
            ai::apply_tc_setup<MODE>(a.ap, a.sh, first_tile, ts, base, offs);
            ai::gather_rows_pz_load<MODE, kGU>(a.ap.pz, a.ap.m, first_tile.count, base, offs,
                                              a.sh.kpad * a.sh.esz / 16, gw);
        }
    }
    unsigned long long t_prev = (a.timers && blockIdx.x == 0 && tid == 0) ? global_ns() : 0ull;
    unsigned long long t_acc[4] = {0, 0, 0, 0};
    for (int loop = 0; loop < a.max_loops; ++loop) {
        // ---- phase A: element products
        bool failed = false;
        ArrayCursor curA{solo ? 0 : -1, 0};   // two-phase iteration: groups done per array (alpha fold)
        if constexpr (AM == AM_TC) {
            if (ov_a && s_active) {   // the tile's loads are in gw: the direction update, then the products
                ai::gather_rows_pz_store<MODE, kGU>(gw, (float)s_beta, a.ap.m, first_tile.count,
                                                    a.sh.kpad * a.sh.esz / 16, ts.sA, a.sh.a_plane,
                                                    tc::sbo_bytes(a.sh.kpad, a.sh.esz), ts.sP, ts.ldp);
                failed = !ai::apply_tc_finish<MODE>(a.ap, a.sh, first_tile, ts);
            }
        }
        for (int w = blockIdx.x; w < a.apply_items && !ov_a; w += gridDim.x) {
            if constexpr (AM == AM_TC) {
                const ApplyWork it = w == (int)blockIdx.x ? first_tile : a.ap.work[w];
                if (!solo && it.array != curA.k) switch_array(curA, it.array, 3);
                if (!s_active) continue;
                if (!ai::apply_tc_item<MODE>(a.ap, a.sh, it, ts, base, offs)) {
                    failed = true;
                    break;
                }
                curA.count += (it.count + 7) >> 3;
            } else if constexpr (AM == AM_TCS) {
                break;   // the warp-specialised phase below takes all of the CTA's tiles
            } else {
                const ApplyWork it = a.ap.work[w / a.panels];
                if (!__ldcg(&a.st[it.array].active)) continue;
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
        if constexpr (AM == AM_TCS) failed = !ai::tcs_apply_phase<MODE, false>(a.ap, a.shs, tss, base, offs, blockIdx.x,
                                                                         gridDim.x);
        if constexpr (FUSED) {
            if (!solo && !failed) switch_array(curA, -1, 3);
        }
        if (failed && tid == 0) {
            atomicExch(a.err, 1);
            atomicExch(a.abort, 1);
        }
        if (!grid_sync(a, &s_ok, &s_kbar)) break;
        phase_mark(a, 0, t_prev, t_acc);
        if constexpr (FUSED) {
            if (ov_b && s_active)   // the slice's loads in flight during the alpha fold
                pi::resident_update_load<kRU>(v_start, v_count, tid, sOff, kVecChunkTC,
                                              static_cast<const float*>(a.ap.Y), a.ap.pz, rs, rpz);
            // ---- alpha from the group sums of p_e^T Y_e (one array: every CTA folds)
            if (solo && s_active) {
                const double pq = pi::cta_fold8(a.ap.gpart + s_A.grp_off, s_A.n_grp, sh8);
                if (tid == 0) {
                    const double al = s_rz / pq;
                    if (!(pq > 0) || !isfinite(al)) {
                        s_alpha = 0.0;
                        s_active = 0;
                        if (blockIdx.x == 0) {
                            a.st[0].alpha = 0.0;
                            a.st[0].active = 0;
                            a.st[0].status = MSTRESS_ENUMERIC;
                            atomicSub(a.n_active, 1);
                        }
                    } else {
                        s_alpha = al;
                        if (blockIdx.x == 0) a.st[0].alpha = al;
                    }
                    s_scalar = s_alpha;
                    s_scalar2 = s_beta;
                }
                __syncthreads();
            }
            // ---- phase B: interface sum + vector update, <r,z>, <r,r>
            ArrayCursor cur{solo ? 0 : -1, 0};
            if (resident) {
                if ((int)blockIdx.x < a.n_vwork && s_active) {
                    pi::DotAcc<float> srz, srr;
                    if (ov_b)
                        pi::resident_update_finish<kRU>(v_start, v_count, tid, sVd, sVx, sVr,
                                                        const_cast<float2*>(a.ap.pz), rs, rpz, (float)s_scalar2,
                                                        (float)s_scalar, srz, srr);
                    else
                        pi::resident_update_item_pz(v_start, v_count, sOff, kVecChunkTC, sVd, sVx, sVr,
                                                    static_cast<const float*>(a.ap.Y), const_cast<float2*>(a.ap.pz),
                                                    (float)s_scalar2, (float)s_scalar, srz, srr);
                    double rz, rr;
                    pi::block_sum2(srz, srr, shr, rz, rr);
                    if (tid == 0) {
                        a.part_rz[blockIdx.x] = rz;
                        a.part_rr[blockIdx.x] = rr;
                    }
                }
            } else
            for (int w = blockIdx.x; w < a.n_vwork; w += gridDim.x) {
                const VecWork it = a.vwork[w];
                if (it.array != cur.k) switch_array(cur, it.array, 2);
                if (!s_active) continue;
                pi::DotAcc<float> srz, srr;
                pi::isum_update_item_pz(it, s_A, a.lm, static_cast<const float*>(a.dinv), a.ap.ldY,
                                        static_cast<const float*>(a.ap.Y), const_cast<float2*>(a.ap.pz),
                                        reinterpret_cast<float*>(x), reinterpret_cast<float*>(r), (float)s_scalar2,
                                        (float)s_scalar, srz, srr);
                double rz, rr;
                pi::block_sum2(srz, srr, shr, rz, rr);
                if (tid == 0) {
                    a.part_rz[w] = rz;
                    a.part_rr[w] = rr;
                }
                cur.count += 1;
            }
            if (!solo) switch_array(cur, -1, 2);
        } else {
        // ---- phase B: interface sum, <p, q>, alpha
        {
            // one array: the cursor starts on it (s_A, s_active, s_scalar = beta preset)
            ArrayCursor cur{solo ? 0 : -1, 0};
            VecWork next = blockIdx.x < a.n_vwork ? a.vwork[blockIdx.x] : VecWork{};
            for (int w = blockIdx.x; w < a.n_vwork; w += gridDim.x) {
                const VecWork it = next;
                if (w + (int)gridDim.x < a.n_vwork) next = a.vwork[w + gridDim.x];   // overlaps this item
                if (it.array != cur.k) switch_array(cur, it.array, 1);
                if (!s_active) continue;
                const pi::DotAcc<V> acc = pi::isum_item<sizeof(V) == 8 ? 2 : (AM == AM_TC ? 5 : 4), V, V>(it, s_A, a.lm, static_cast<const V*>(a.dinv), a.ap.ldY,
                                                     static_cast<const V*>(a.ap.Y), p, z, q, (V)s_scalar);
                const double t = pi::block_sum(acc, shr);
                if (tid == 0) a.part_pq[w] = t;
                cur.count += 1;
            }
            if (!solo) switch_array(cur, -1, 1);
        }
        if (!grid_sync(a, &s_ok, &s_kbar)) break;
        phase_mark(a, 1, t_prev, t_acc);
        if (solo && s_active) {
            const double pq = pi::cta_fold8(a.part_pq + s_A.vwork_off, s_A.n_vwork, sh8);
            if (tid == 0) {
                const double al = s_rz / pq;
                if (!(pq > 0) || !isfinite(al)) {
                    s_alpha = 0.0;
                    s_active = 0;
                    if (blockIdx.x == 0) {
                        a.st[0].alpha = 0.0;
                        a.st[0].active = 0;
                        a.st[0].status = MSTRESS_ENUMERIC;
                        atomicSub(a.n_active, 1);
                    }
                } else {
                    s_alpha = al;
                    if (blockIdx.x == 0) a.st[0].alpha = al;
                }
                s_scalar = s_alpha;
            }
            __syncthreads();
        }
        // ---- phase C: vector update, <r,z>, <r,r>, beta, stopping test
        {
            ArrayCursor cur{solo ? 0 : -1, 0};   // one array: s_scalar = alpha preset
            VecWork next = blockIdx.x < a.n_vwork ? a.vwork[blockIdx.x] : VecWork{};
            for (int w = blockIdx.x; w < a.n_vwork; w += gridDim.x) {
                const VecWork it = next;
                if (w + (int)gridDim.x < a.n_vwork) next = a.vwork[w + gridDim.x];
                if (it.array != cur.k) switch_array(cur, it.array, 2);
                if (!s_active) continue;
                pi::DotAcc<V> srz, srr;
                pi::vec1_item<NT >= 512 ? 8 : 4, V>(it, static_cast<const V*>(a.dinv), (V)s_scalar, x, r, z, p, q, srz, srr);
                const double rz = pi::block_sum(srz, shr);
                const double rr = pi::block_sum(srr, shr);
                if (tid == 0) {
                    a.part_rz[w] = rz;
                    a.part_rr[w] = rr;
                }
                cur.count += 1;
            }
            if (!solo) switch_array(cur, -1, 2);
        }
        }   // three-phase iteration
        if (!grid_sync(a, &s_ok, &s_kbar)) break;
        phase_mark(a, FUSED ? 1 : 2, t_prev, t_acc);
        if constexpr (AM == AM_TC) {
            if (ov_a && s_active)   // the next phase A's loads in flight during the beta fold
                ai::gather_rows_pz_load<MODE, kGU>(a.ap.pz, a.ap.m, first_tile.count, base, offs,
                                                  a.sh.kpad * a.sh.esz / 16, gw);
        }
        if (solo && s_active) {
            double rz, rr;
            pi::cta_fold8_2(a.part_rz + s_A.vwork_off, a.part_rr + s_A.vwork_off, s_A.n_vwork, sh8, rz, rr);
            if (tid == 0) {
                const int iters = s_iters + 1;
                int active = 1, status = MSTRESS_OK;
                double beta = 0;
                if (!isfinite(rz) || !isfinite(rr)) {
                    active = 0;
                    status = MSTRESS_ENUMERIC;
                } else {
                    beta = rz / s_rz;
                    if (rr <= s_tol2) active = 0;
                    else if (iters >= s_max_iter) { active = 0; status = MSTRESS_ENOT_CONVERGED; }
                }
                s_rz = rz;
                s_beta = beta;
                s_scalar = beta;
                s_iters = iters;
                s_active = active;
                a.st[0].beta = beta;   // the same value from every CTA, read by its own next gather
                if (blockIdx.x == 0) {
                    a.st[0].rz = rz;
                    a.st[0].rr = rr;
                    a.st[0].iters = iters;
                    a.st[0].status = status;
                    a.st[0].active = active;
                    if (!active) atomicSub(a.n_active, 1);
                }
            }
            __syncthreads();
        }
        if (a.timers && blockIdx.x == 0 && tid == 0) t_acc[3] += 1;
        if (solo ? !s_active : *(volatile int*)a.n_active <= 0) break;
    }
    if (a.timers && blockIdx.x == 0 && tid == 0)
        for (int k = 0; k < 4; ++k) a.timers[k] += t_acc[k];
    if constexpr (FUSED) {
        if (resident && (int)blockIdx.x < a.n_vwork) {   // the slice's x and r back to global memory
            __syncthreads();
            for (int l = tid; l < v_count; l += NT) {
                x[v_start + l] = sVx[l];
                r[v_start + l] = sVr[l];
            }
        }
    }
    if constexpr (AM == AM_TC) {
        if (*(volatile int*)a.abort) tc::mbar_wait(&mbar, ts.phase ^ 1u, 1 << 20);   // bounded drain
        tc::fence_before();
        __syncthreads();
        if ((tid >> 5) == 0) tc::tmem_free_c<128>(ts.tmem);
    }
    if constexpr (AM == AM_TCS) {
        if (*(volatile int*)a.abort) ai::tcs_drain(tss, a.shs);
        tc::fence_before();
        __syncthreads();
        if ((tid >> 5) == 0) tc::tmem_free(tss.tmem, (uint32_t)a.shs.tmem_cols);
    }
}

template <int NT, class KER>
bool launch_coop(KER kernel, mstress_sol_s* s, PcgArgs& a, size_t smem, int needed, int tmem_cols) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) { cudaGetLastError(); return false; }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, NT, smem);
    if (e != cudaSuccess || per_sm < 1) { cudaGetLastError(); return false; }
    if (tmem_cols > 0) per_sm = std::min(per_sm, 512 / tmem_cols);
    per_sm = std::min(per_sm, 4);   // more CTAs only lengthen the barriers
    const int grid = std::max(1, std::min(needed, per_sm * s->ctx->num_sms));
    if (s->ctx->withhold_next) {   // test hook: the last CTA skips its first barrier arrival once
        a.withhold_cta = grid - 1;
        s->ctx->withhold_next = 0;
    }
    void* args[] = {&a};
    e = cudaLaunchCooperativeKernel((void*)kernel, grid, NT, args, smem, s->ctx->stream);
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
    a.ap = apply_args(s, v.p.ptr, v.z.ptr, v.state.as<PcgState>(), s->Y.ptr, tc);   // gathers p = z + beta p
    a.vwork = s->d_vwork.as<VecWork>();
    a.n_vwork = s->n_vwork;
    a.arrays = s->d_arrays.as<ArrayDev>();
    a.n_arrays = s->n_arrays;
    a.lm = s->d_lm.as<LocalMap>();
    a.dinv = vec_fp32 ? s->dinv32.ptr : s->dinv.ptr;
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
    a.abort = flag + 7;
    a.bar = s->barrier.as<unsigned>();
    a.max_loops = max_iter + 1;
    a.wait_limit_ns = s->ctx->wait_limit_ns;
    a.withhold_cta = -1;
    a.timers = s->timers.as<unsigned long long>();
    MS_CUDA(cudaMemsetAsync(flag + 7, 0, sizeof(int), s->ctx->stream));
    MS_CUDA(cudaMemsetAsync(s->barrier.ptr, 0, s->barrier.bytes, s->ctx->stream));
    MS_CUDA(cudaMemsetAsync(s->tickets.ptr, 0, s->tickets.bytes, s->ctx->stream));
    const int m = s->m;
    const int vneed = s->n_vwork;
    if (!vec_fp32) {
        if (apply_rpt(m, 8, 1) == 2) {
            a.panels = (m + 15) / 16;
            a.apply_items = s->n_awork * a.panels;
            const size_t smem = (size_t)(m * kTile64 + 16 * m) * sizeof(double) + 1024;
            return launch_coop<256>(k_pcg<double, AM_FP64, MSTRESS_FP64, 2, 256, 2>, s, a, smem,
                                    std::max(a.apply_items, vneed), 0);
        }
        a.panels = (m + 31) / 32;
        a.apply_items = s->n_awork * a.panels;
        const size_t smem = (size_t)(m * kTile64 + 32 * m) * sizeof(double) + 1024;
        return launch_coop<256>(k_pcg<double, AM_FP64, MSTRESS_FP64, 4, 256, 2>, s, a, smem,
                                std::max(a.apply_items, vneed), 0);
    }
    if (tc && tc_streamed(m)) {
        a.shs = tcs_shape(m, prec);
        a.shs.lg_tile = lg_ceil(s->tc_tile);
        a.apply_items = s->n_awork_tc;
        a.panels = 1;
        const int need = std::max(a.apply_items, vneed);
        const int tm = a.shs.tmem_cols;
        switch (prec) {
            case MSTRESS_TF32:
                return launch_coop<ai::kTcsThreads>(k_pcg<float, AM_TCS, MSTRESS_TF32, 0, ai::kTcsThreads, 1>, s, a, a.shs.smem, need, tm);
            case MSTRESS_BF16:
                return launch_coop<ai::kTcsThreads>(k_pcg<float, AM_TCS, MSTRESS_BF16, 0, ai::kTcsThreads, 1>, s, a, a.shs.smem, need, tm);
            default:
                return launch_coop<ai::kTcsThreads>(k_pcg<float, AM_TCS, MSTRESS_BF16X3, 0, ai::kTcsThreads, 1>, s, a, a.shs.smem, need, tm);
        }
    }
    if (tc) {
        a.sh = tc_shape(m, prec);
        a.sh.lg_tile = lg_ceil(s->tc_tile);
        if (a.sh.tmem_cols > 128) return false;   // the kernel allocates 128 tensor-memory columns
        a.apply_items = s->n_awork_tc;
        a.panels = 1;
        a.ap.gpart = s->gpart.as<double>();     // two-phase iteration: group sums of p_e^T Y_e
        a.ap.pz = s->pz.as<float2>();           // and the (p, z) pairs
        if (!a.ap.pz) return false;
        size_t smem = a.sh.smem + a.sh.dot_smem;
        // resident vector slices: one array whose element-product offsets fit in 32 bits
        const size_t vec_smem = (size_t)kVecChunkTC * (3 * sizeof(float) + 4 * sizeof(int));
        if (s->n_arrays == 1 && (int64_t)s->n_blocks * s->ldY < (1LL << 31) && smem + vec_smem <= 200 * 1024) {
            a.resident = 1;
            smem += vec_smem;
        }
        const int need = std::max(a.apply_items, vneed);
        // one array whose vector items fit one per SM: the variant compiled for it alone (every
        // cooperative grid has at least one CTA per SM, so each CTA keeps at most one item)
        if (a.resident && s->n_vwork <= s->ctx->num_sms) {
            switch (prec) {
                case MSTRESS_TF32:
                    return launch_coop<512>(k_pcg<float, AM_TC, MSTRESS_TF32, 0, 512, 1, true>, s, a, smem, need, 128);
                case MSTRESS_BF16:
                    return launch_coop<512>(k_pcg<float, AM_TC, MSTRESS_BF16, 0, 512, 1, true>, s, a, smem, need, 128);
                default:
                    return launch_coop<512>(k_pcg<float, AM_TC, MSTRESS_BF16X3, 0, 512, 1, true>, s, a, smem, need,
                                            128);
            }
        }
        switch (prec) {
            case MSTRESS_TF32:
                return launch_coop<512>(k_pcg<float, AM_TC, MSTRESS_TF32, 0, 512, 1>, s, a, smem, need, 128);
            case MSTRESS_BF16:
                return launch_coop<512>(k_pcg<float, AM_TC, MSTRESS_BF16, 0, 512, 1>, s, a, smem, need, 128);
            default:
                return launch_coop<512>(k_pcg<float, AM_TC, MSTRESS_BF16X3, 0, 512, 1>, s, a, smem, need, 128);
        }
    }
    const int ns = prec == MSTRESS_BF16X3 ? 2 : 1;
    const int rpt = apply_rpt(m, 4, ns);
    a.panels = (m + 8 * rpt - 1) / (8 * rpt);
    a.apply_items = s->n_awork * a.panels;
    const size_t smem = (size_t)ns * (m * kTile64 + 8 * rpt * m) * sizeof(float) + 1024;
    const int need = std::max(a.apply_items, vneed);
    if (rpt == 2) {
        if (prec == MSTRESS_TF32)
            return launch_coop<256>(k_pcg<float, AM_SIMT32, MSTRESS_TF32, 2, 256, 2>, s, a, smem, need, 0);
        if (prec == MSTRESS_BF16)
            return launch_coop<256>(k_pcg<float, AM_SIMT32, MSTRESS_BF16, 2, 256, 2>, s, a, smem, need, 0);
        return launch_coop<256>(k_pcg<float, AM_SIMT32, MSTRESS_BF16X3, 2, 256, 2>, s, a, smem, need, 0);
    }
    if (prec == MSTRESS_TF32)
        return launch_coop<256>(k_pcg<float, AM_SIMT32, MSTRESS_TF32, 4, 256, 2>, s, a, smem, need, 0);
    if (prec == MSTRESS_BF16)
        return launch_coop<256>(k_pcg<float, AM_SIMT32, MSTRESS_BF16, 4, 256, 2>, s, a, smem, need, 0);
    return launch_coop<256>(k_pcg<float, AM_SIMT32, MSTRESS_BF16X3, 4, 256, 2>, s, a, smem, need, 0);
}

}  // namespace ms
