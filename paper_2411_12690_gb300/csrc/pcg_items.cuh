// Device building blocks of the global-stage PCG shared by the stand-alone
// phase kernels (online.cu) and the persistent cooperative solver
// (pcg_persistent.cu): fixed-order reductions, the lattice/owner arithmetic of
// the implicit assembly, and the per-work-item bodies of the interface sum and
// the vector update.
#pragma once

#include "solve.h"

namespace ms {
namespace pi {

// Fixed-order sum of n values by one warp: lane-strided partial sums (four
// loads in flight, summed in index order), then a butterfly. Loads bypass L1
// because the values come from other CTAs.
__device__ __forceinline__ double warp_fold(const double* v, int n) {
    const int lane = threadIdx.x & 31;
    double s = 0;
    int i = lane;
    for (; i + 96 < n; i += 128) {
        const double a0 = __ldcg(v + i), a1 = __ldcg(v + i + 32), a2 = __ldcg(v + i + 64), a3 = __ldcg(v + i + 96);
        s += a0;
        s += a1;
        s += a2;
        s += a3;
    }
    for (; i < n; i += 32) s += __ldcg(v + i);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Fixed-order sum of n values by a whole CTA of nw warps: warp w folds the
// slice [w n / 8, (w+1) n / 8) for w < 8 (warps beyond 8 idle), thread 0 adds
// the 8 slice sums in order. The order depends only on n, never on which CTA
// or how many arrays. Result valid in thread 0. Needs all threads.
__device__ __forceinline__ double cta_fold8(const double* v, int n, double* sh8) {
    const int w = threadIdx.x >> 5;
    if (w < 8) {
        const int b = (int)((long long)n * w / 8), e = (int)((long long)n * (w + 1) / 8);
        const double s = warp_fold(v + b, e - b);
        if ((threadIdx.x & 31) == 0) sh8[w] = s;
    }
    __syncthreads();
    double t = 0;
    if (threadIdx.x == 0)
        for (int k = 0; k < 8; ++k) t += sh8[k];
    __syncthreads();
    return t;
}

// Block sum (blockDim.x threads, multiple of 32) in a fixed order; result valid in all threads.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[w] = v;
    __syncthreads();
    double t = 0;
    for (int k = 0; k < nw; ++k) t += sh[k];
    return t;
}

__device__ __forceinline__ void lattice_coords(const ArrayDev& A, long long g, int& comp, int& gx, int& gy, int& gz) {
    // an array's lattice holds fewer than 2^31 DOFs, so 32-bit division suffices
    const unsigned l = (unsigned)(g - A.vec_off);
    const unsigned node = l / 3u;
    comp = (int)(l - 3u * node);
    const unsigned X = (unsigned)A.X, t = node / X;
    gx = (int)(node - t * X);
    const unsigned Y = (unsigned)A.Y, zz = t / Y;
    gy = (int)(t - zz * Y);
    gz = (int)zz;
}

// Visit the blocks that own lattice point (gx, gy, gz) with the point's
// surface-node index there, rows ascending then columns ascending.
template <class Fn>
__device__ __forceinline__ void for_owners(const ArrayDev& A, const int16_t* __restrict__ surf, int n, int gx, int gy,
                                           int gz, Fn fn) {
    const int n1 = n - 1;
    int ih = gx / n1, il = (gx % n1 == 0) ? ih - 1 : ih;
    int jh = gy / n1, jl = (gy % n1 == 0) ? jh - 1 : jh;
    ih = min(ih, A.nx - 1);
    jh = min(jh, A.ny - 1);
    il = max(il, 0);
    jl = max(jl, 0);
    for (int j = jl; j <= jh; ++j)
        for (int i = il; i <= ih; ++i) {
            int a = gx - i * n1, b = gy - j * n1;
            int s = __ldg(surf + (gz * n + b) * n + a);
            if (s >= 0) fn(A.block_off + (long long)j * A.nx + i, s);
        }
}

// Interface sum of one vector work item: q_g = sum of Y_e over the owning
// blocks (fixed order), p updated to z + beta p when z is given; returns this
// thread's share of <p, q>.
template <class V, class YT>
__device__ __forceinline__ double isum_item(const VecWork& it, const ArrayDev& A, const LocalMap* lm, const double* dinv,
                                            int ldY, const YT* __restrict__ Y, V* __restrict__ p,
                                            const V* __restrict__ z, V* __restrict__ q, double beta) {
    double acc = 0;
    for (long long g = it.start + threadIdx.x; g < it.start + it.count; g += blockDim.x) {
        double s = 0;
        if (!dinv || dinv[g] != 0.0) {
            int comp, gx, gy, gz;
            lattice_coords(A, g, comp, gx, gy, gz);
            for_owners(A, lm->surf_idx, lm->n, gx, gy, gz,
                       [&](long long blk, int sidx) { s += (double)Y[blk * ldY + 3 * sidx + comp]; });
        }
        V pv = p[g];
        if (z) {
            pv = p_next(z[g], pv, beta);
            p[g] = pv;
        }
        q[g] = (V)s;
        acc += (double)pv * s;
    }
    return acc;
}

// Vector update of one work item: x += alpha p, r -= alpha q, z = D^-1 r;
// returns this thread's shares of <r, z> and <r, r>.
template <class V>
__device__ __forceinline__ void vec1_item(const VecWork& it, const double* dinv, double al, V* x, V* r, V* z,
                                          const V* p, const V* q, double& srz, double& srr) {
    srz = 0;
    srr = 0;
    for (long long g = it.start + threadIdx.x; g < it.start + it.count; g += blockDim.x) {
        double pv = (double)p[g], qv = (double)q[g];
        x[g] = (V)((double)x[g] + al * pv);
        V rv = (V)((double)r[g] - al * qv);
        V zv = (V)(dinv[g] * (double)rv);
        r[g] = rv;
        z[g] = zv;
        srz += (double)rv * (double)zv;
        srr += (double)rv * (double)rv;
    }
}

}  // namespace pi
}  // namespace ms
