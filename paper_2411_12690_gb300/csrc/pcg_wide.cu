// Per-phase PCG iteration for large batches on the streamed tensor-core apply
// (section 4.3, Eq. 20), captured in the solve's CUDA graph.
//
// The persistent cooperative solver holds one 512-thread CTA per SM for the
// whole solve, so its vector phases run at a quarter of the SM's warp slots;
// that is the right trade while an iteration is short (grid barriers instead
// of launches), but on a batch of several thousand blocks with a large basis
// the vector phases dominate and want the occupancy of kernels of their own.
// This path runs the same iteration as separate launches:
//   apply      the stand-alone streamed tensor-core apply (p = z + beta p
//              formed in the gather, the same operand bits and products);
//              p and z are kept as (p, z) pairs, so that it gathers both
//              with one 8-byte load (the interface sum writes the first half
//              of a pair, the update the second);
//   k_w_isum   interface sum q, p stored, <p,q> partial per vector item;
//   k_w_alpha  one CTA per array: alpha = <r,z> / <p,q> from the partials;
//   k_w_vec    x += alpha p, r -= alpha q, z = D^-1 r, <r,z>, <r,r> partials;
//   k_w_beta   one CTA per array: beta, stopping test, iteration count; the
//              last CTA sets the graph's loop condition.
// Every kernel calls the persistent solver's own per-item functions with the
// same 512 threads and the same fixed-order folds (cta_fold8, cta_fold8_2),
// so the scalars and vectors are bitwise those of the persistent solver: an
// array's result does not depend on which path its batch took.
#include <algorithm>

#include "pcg_items.cuh"

namespace ms {
namespace {

constexpr int kWT = 512;   // threads per CTA, as the persistent solver's streamed variant

struct WideArgs {
    const VecWork* vwork;
    int n_vwork;
    const ArrayDev* arrays;
    const LocalMap* lm;
    const float* dinv;
    int ldY;
    const float* Y;
    float *x, *r, *q;
    float2* pz;   // (p, z) pairs
    PcgState* st;
    double *part_pq, *part_rz, *part_rr;
    int* flag;   // [0] any active, [1] CTA ticket, [2] device error, [3] loop count, [5] arrays active
                 // this iteration
    int loop_cap;
    int use_cond;
    cudaGraphConditionalHandle cond;
};

// Per-CTA cursor over the arrays of its vector items: the array's descriptor,
// active flag and one scalar (beta or alpha), read once per array switch.
struct WideCursor {
    int k = -1;
};

__device__ __forceinline__ void wide_switch(const WideArgs& a, WideCursor& c, int k, bool want_alpha, ArrayDev& sA,
                                            int& s_active, double& s_scalar) {
    if (k == c.k) return;
    __syncthreads();   // the previous item's readers are done with the shared copies
    if (threadIdx.x == 0) {
        sA = a.arrays[k];
        s_active = a.st[k].active;
        s_scalar = want_alpha ? a.st[k].alpha : a.st[k].beta;
    }
    __syncthreads();
    c.k = k;
}

__global__ void __launch_bounds__(kWT, 2) k_w_isum(const __grid_constant__ WideArgs a) {
    __shared__ double shr[2 * (kWT / 32)];
    __shared__ ArrayDev sA;
    __shared__ int s_active;
    __shared__ double s_beta;
    WideCursor c;
    for (int w = blockIdx.x; w < a.n_vwork; w += gridDim.x) {
        const VecWork it = a.vwork[w];
        wide_switch(a, c, it.array, false, sA, s_active, s_beta);
        if (!s_active) continue;
        const pi::DotAcc<float> acc =
            pi::isum_item_pz<4, true>(it, sA, a.lm, a.dinv, a.ldY, a.Y, a.pz, a.q, (float)s_beta);
        const double t = pi::block_sum(acc, shr);
        if (threadIdx.x == 0) a.part_pq[w] = t;
    }
}

__global__ void __launch_bounds__(kWT) k_w_alpha(const __grid_constant__ WideArgs a) {
    __shared__ double sh8[8];
    const int k = blockIdx.x;
    if (!a.st[k].active) return;   // the same value in every thread
    const ArrayDev A = a.arrays[k];
    const double pq = pi::cta_fold8(a.part_pq + A.vwork_off, A.n_vwork, sh8);
    if (threadIdx.x == 0) {
        const double al = a.st[k].rz / pq;
        if (!(pq > 0) || !isfinite(al)) {
            a.st[k].alpha = 0.0;
            a.st[k].active = 0;
            a.st[k].status = MSTRESS_ENUMERIC;
        } else {
            a.st[k].alpha = al;
        }
    }
}

__global__ void __launch_bounds__(kWT, 2) k_w_vec(const __grid_constant__ WideArgs a) {
    __shared__ double shr[2 * (kWT / 32)];
    __shared__ ArrayDev sA;
    __shared__ int s_active;
    __shared__ double s_alpha;
    WideCursor c;
    for (int w = blockIdx.x; w < a.n_vwork; w += gridDim.x) {
        const VecWork it = a.vwork[w];
        wide_switch(a, c, it.array, true, sA, s_active, s_alpha);
        if (!s_active) continue;
        pi::DotAcc<float> srz, srr;
        // (4 DOFs per thread in flight: each thread still visits its DOFs, and adds
        // their products, in the persistent solver's order)
        pi::vec1_item_pz<4>(it, a.dinv, (float)s_alpha, a.x, a.r, a.pz, a.q, srz, srr);
        const double rz = pi::block_sum(srz, shr);
        const double rr = pi::block_sum(srr, shr);
        if (threadIdx.x == 0) {
            a.part_rz[w] = rz;
            a.part_rr[w] = rr;
        }
    }
}

__global__ void __launch_bounds__(kWT) k_w_beta(const __grid_constant__ WideArgs a) {
    __shared__ double sh16[16];
    __shared__ int s_last;
    const int k = blockIdx.x;
    if (a.st[k].active) {
        const ArrayDev A = a.arrays[k];
        double rz, rr;
        pi::cta_fold8_2(a.part_rz + A.vwork_off, a.part_rr + A.vwork_off, A.n_vwork, sh16, rz, rr);
        if (threadIdx.x == 0) {
            PcgState s = a.st[k];
            s.iters += 1;
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
            s.beta = beta;
            s.rz = rz;
            s.rr = rr;
            s.status = status;
            s.active = active;
            a.st[k] = s;
            if (active) atomicAdd(&a.flag[5], 1);
        }
    }
    // the last CTA: loop condition for the next iteration
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&a.flag[1], 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        int any = atomicExch(&a.flag[5], 0) > 0;
        a.flag[1] = 0;
        const int loops = a.flag[3] + 1;
        a.flag[3] = loops;
        if (loops >= a.loop_cap || a.flag[2] != 0) any = 0;   // the loop cap, or an apply's wait expired
        a.flag[0] = any;
        if (a.use_cond) cudaGraphSetConditional(a.cond, any ? 1u : 0u);
    }
}

}  // namespace

bool pcg_wide(const mstress_sol_s* s, int prec) {
    return prec != MSTRESS_FP64 && s->use_tc && tc_streamed(s->m) && s->n_blocks >= kWideBlocks;
}

void launch_apply_wide(mstress_sol_s* s, int prec, const PcgState* st) {
    MS_REQUIRE(s->pz.ptr, MSTRESS_EINVAL, "per-phase iteration without (p, z) pairs");
    ApplyArgs a = apply_args(s, s->v32.p.ptr, s->v32.z.ptr, st, s->Y.ptr, true);
    a.pz = s->pz.as<float2>();
    launch_apply_tc(s, prec, a);
}

void pcg_iteration_wide(mstress_sol_s* s, PcgVectors& v, int prec, int use_cond, cudaGraphConditionalHandle cond,
                        int loop_cap) {
    cudaStream_t stream = s->ctx->stream;
    PcgState* st = v.state.as<PcgState>();
    launch_apply_wide(s, prec, st);   // gathers p = z + beta p from the pairs
    WideArgs a;
    std::memset(&a, 0, sizeof(a));
    a.vwork = s->d_vwork.as<VecWork>();
    a.n_vwork = s->n_vwork;
    a.arrays = s->d_arrays.as<ArrayDev>();
    a.lm = s->d_lm.as<LocalMap>();
    a.dinv = s->dinv32.as<float>();
    a.ldY = s->ldY;
    a.Y = s->Y.as<float>();
    a.x = v.x.as<float>();
    a.r = v.r.as<float>();
    a.q = v.q.as<float>();
    a.pz = s->pz.as<float2>();
    a.st = st;
    a.part_pq = s->part.as<double>();
    a.part_rz = a.part_pq + s->n_vwork;
    a.part_rr = a.part_rz + s->n_vwork;
    a.flag = s->flag.as<int>();
    a.loop_cap = loop_cap;
    a.use_cond = use_cond;
    a.cond = cond;
    const int g = std::max(1, std::min(s->n_vwork, 4 * s->ctx->num_sms));
    k_w_isum<<<g, kWT, 0, stream>>>(a);
    MS_LAUNCH_CHECK();
    k_w_alpha<<<s->n_arrays, kWT, 0, stream>>>(a);
    MS_LAUNCH_CHECK();
    k_w_vec<<<g, kWT, 0, stream>>>(a);
    MS_LAUNCH_CHECK();
    k_w_beta<<<s->n_arrays, kWT, 0, stream>>>(a);
    MS_LAUNCH_CHECK();
}

}  // namespace ms
