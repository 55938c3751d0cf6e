// Device building blocks of the global-stage PCG shared by the stand-alone
// phase kernels (online.cu) and the persistent cooperative solver
// (pcg_persistent.cu): fixed-order reductions, the lattice/owner arithmetic of
// the implicit assembly, and the per-work-item bodies of the interface sum and
// the vector update.
#pragma once

#include "solve.h"

namespace ms {
namespace pi {

// Fixed-order sum of n values by one warp: lane-strided partial sums (each
// lane adds v[lane], v[lane + 32], ... in index order; up to eight loads are
// issued before they are added), then a butterfly. Loads bypass L1 because
// the values come from other CTAs.
__device__ __forceinline__ double warp_fold(const double* v, int n) {
    const int lane = threadIdx.x & 31;
    double s = 0;
    for (int i0 = lane; i0 < n; i0 += 256) {
        double a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = i0 + 32 * u < n ? __ldcg(v + i0 + 32 * u) : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (i0 + 32 * u < n) s += a[u];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Fixed-order sum of n values by a whole CTA of nw >= 8 warps: warp w folds the
// slice [w n / 8, (w+1) n / 8) for w < 8 (warps beyond 8 idle), then every
// thread adds the 8 slice sums in order. The order depends only on n, never
// on which CTA or how many arrays. Result valid in every thread. Needs all
// threads; sh8 must not be written again before every thread has returned
// (the callers pass a barrier first).
__device__ __forceinline__ double cta_fold8(const double* v, int n, double* sh8) {
    const int w = threadIdx.x >> 5;
    if (w < 8) {
        const int b = (int)((long long)n * w / 8), e = (int)((long long)n * (w + 1) / 8);
        const double s = warp_fold(v + b, e - b);
        if ((threadIdx.x & 31) == 0) sh8[w] = s;
    }
    __syncthreads();
    double t = 0;
    for (int k = 0; k < 8; ++k) t += sh8[k];
    return t;
}

// Two fixed-order sums at once (the <r,z> and <r,r> partials of one array):
// the same slices and order as cta_fold8 for each. Results valid in every
// thread; sh16 as sh8 above.
__device__ __forceinline__ void cta_fold8_2(const double* v1, const double* v2, int n, double* sh16, double& t1,
                                            double& t2) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w < 8) {
        // warp_fold of both slices with all their loads in flight together
        const int b = (int)((long long)n * w / 8), e = (int)((long long)n * (w + 1) / 8), cnt = e - b;
        double s1 = 0, s2 = 0;
        for (int i0 = lane; i0 < cnt; i0 += 256) {
            double a1[8], a2[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const bool in = i0 + 32 * u < cnt;
                a1[u] = in ? __ldcg(v1 + b + i0 + 32 * u) : 0.0;
                a2[u] = in ? __ldcg(v2 + b + i0 + 32 * u) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (i0 + 32 * u < cnt) {
                    s1 += a1[u];
                    s2 += a2[u];
                }
        }
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (lane == 0) {
            sh16[w] = s1;
            sh16[8 + w] = s2;
        }
    }
    __syncthreads();
    t1 = 0;
    t2 = 0;
    for (int k = 0; k < 8; ++k) {
        t1 += sh16[k];
        t2 += sh16[8 + k];
    }
}

using ms::DotAcc;   // dot-product accumulators (solve.h)

// Block sum of double-FP32 accumulators in a fixed order: butterfly of the
// pairs within each warp, the warp sums (hi + lo in FP64) added in FP64 by
// thread 0. Result valid in thread 0.
__device__ __forceinline__ double block_sum(DotAcc<float> v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) {
        const float ohi = __shfl_xor_sync(0xffffffffu, v.hi, o), olo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v.merge(ohi, olo);
    }
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[w] = (double)v.hi + (double)v.lo;
    __syncthreads();
    double t = 0;
    if (threadIdx.x == 0)
        for (int k = 0; k < nw; ++k) t += sh[k];
    return t;
}

// Two block sums at once (the <r,z> and <r,r> shares of a work item): each
// gives exactly block_sum's value, with one pair of barriers for both.
// sh holds 2 * (blockDim.x / 32) doubles. Results valid in thread 0.
__device__ __forceinline__ void block_sum2(DotAcc<float> a, DotAcc<float> b, double* sh, double& ta, double& tb) {
    for (int o = 16; o > 0; o >>= 1) {
        const float ahi = __shfl_xor_sync(0xffffffffu, a.hi, o), alo = __shfl_xor_sync(0xffffffffu, a.lo, o);
        const float bhi = __shfl_xor_sync(0xffffffffu, b.hi, o), blo = __shfl_xor_sync(0xffffffffu, b.lo, o);
        a.merge(ahi, alo);
        b.merge(bhi, blo);
    }
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        sh[w] = (double)a.hi + (double)a.lo;
        sh[nw + w] = (double)b.hi + (double)b.lo;
    }
    __syncthreads();
    ta = 0;
    tb = 0;
    if (threadIdx.x == 0)
        for (int k = 0; k < nw; ++k) {
            ta += sh[k];
            tb += sh[nw + k];
        }
}

__device__ __forceinline__ double block_sum(DotAcc<double> v, double* sh);

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

__device__ __forceinline__ double block_sum(DotAcc<double> v, double* sh) { return block_sum(v.s, sh); }

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
// blocks (fixed order), p updated to z + beta p when z is given (the apply
// gathered the same p_e with the same arithmetic); returns this thread's share
// of <p, q>. Arithmetic in the vector precision V (dinv, the constrained-row
// mask, in V as well).
// Each thread handles U DOFs at once and issues all their loads (mask,
// direction, up to four owner contributions) before combining, so a work item
// of U * blockDim.x DOFs costs one round trip to L2 instead of a chain of
// dependent ones. The owner candidates are visited rows ascending then columns
// ascending, as in for_owners; constrained rows are zeroed after the sum.
// NC: nothing writes Y during the kernel (a kernel of its own), so the
// owners' element products may come through L1 (ld.global.nc).
template <int U, class V, class YT, bool NC = false>
__device__ __forceinline__ DotAcc<V> isum_item(const VecWork& it, const ArrayDev& A, const LocalMap* lm, const V* dinv, int ldY,
                                       const YT* __restrict__ Y, V* __restrict__ p, const V* __restrict__ z,
                                       V* __restrict__ q, V beta) {
    const int n = lm->n, n1 = n - 1;
    const int16_t* __restrict__ surf = lm->surf_idx;
    const long long end = it.start + it.count;
    DotAcc<V> acc;
    for (long long g0 = it.start + threadIdx.x; g0 < end; g0 += (long long)blockDim.x * U) {
        V s[U], dv[U];
        V pv[U], zv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long g = g0 + (long long)u * blockDim.x;
            s[u] = 0;
            dv[u] = 0;
            pv[u] = V(0);
            zv[u] = V(0);
            if (g < end) {
                dv[u] = dinv ? dinv[g] : V(1);
                pv[u] = p[g];
                if (z) zv[u] = z[g];
                int comp, gx, gy, gz;
                lattice_coords(A, g, comp, gx, gy, gz);
                const int ih0 = gx / n1, jh0 = gy / n1;
                const int ih = min(ih0, A.nx - 1), jh = min(jh0, A.ny - 1);
                const int il = max((gx % n1 == 0) ? ih0 - 1 : ih0, 0), jl = max((gy % n1 == 0) ? jh0 - 1 : jh0, 0);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int j = (c >> 1) ? jh : jl, i = (c & 1) ? ih : il;
                    const bool use = ((c >> 1) == 0 || jh != jl) && ((c & 1) == 0 || ih != il);
                    if (use) {
                        const int sidx = __ldg(surf + (gz * n + (gy - j * n1)) * n + (gx - i * n1));
                        if (sidx >= 0) {
                            const YT* yp = Y + (A.block_off + (long long)j * A.nx + i) * ldY + 3 * sidx + comp;
                            s[u] += (V)(NC ? __ldg(yp) : __ldcg(yp));
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long g = g0 + (long long)u * blockDim.x;
            if (g < end) {
                const V sv = dv[u] != V(0) ? s[u] : V(0);
                V pn = pv[u];
                if (z) {
                    pn = p_next(zv[u], pv[u], beta);
                    p[g] = pn;
                }
                q[g] = sv;
                acc.add(pn, sv);
            }
        }
    }
    return acc;
}

// isum_item on (p, z) pairs (FP32, the per-phase iteration of large batches):
// the same arithmetic, p and z read from one pair and the new p written to its
// first half. NC: Y is read through L1 (nothing writes it during the kernel).
template <int U, bool NC>
__device__ __forceinline__ DotAcc<float> isum_item_pz(const VecWork& it, const ArrayDev& A, const LocalMap* lm,
                                                      const float* dinv, int ldY, const float* __restrict__ Y,
                                                      float2* __restrict__ pz, float* __restrict__ q, float beta) {
    const int n = lm->n, n1 = n - 1;
    const int16_t* __restrict__ surf = lm->surf_idx;
    const long long end = it.start + it.count;
    DotAcc<float> acc;
    for (long long g0 = it.start + threadIdx.x; g0 < end; g0 += (long long)blockDim.x * U) {
        float s[U], dv[U];
        float2 pzv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long g = g0 + (long long)u * blockDim.x;
            s[u] = 0.f;
            dv[u] = 0.f;
            pzv[u] = make_float2(0.f, 0.f);
            if (g < end) {
                dv[u] = dinv[g];
                pzv[u] = pz[g];
                int comp, gx, gy, gz;
                lattice_coords(A, g, comp, gx, gy, gz);
                const int ih0 = gx / n1, jh0 = gy / n1;
                const int ih = min(ih0, A.nx - 1), jh = min(jh0, A.ny - 1);
                const int il = max((gx % n1 == 0) ? ih0 - 1 : ih0, 0), jl = max((gy % n1 == 0) ? jh0 - 1 : jh0, 0);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int j = (c >> 1) ? jh : jl, i = (c & 1) ? ih : il;
                    const bool use = ((c >> 1) == 0 || jh != jl) && ((c & 1) == 0 || ih != il);
                    if (use) {
                        const int sidx = __ldg(surf + (gz * n + (gy - j * n1)) * n + (gx - i * n1));
                        if (sidx >= 0) {
                            const float* yp = Y + (A.block_off + (long long)j * A.nx + i) * ldY + 3 * sidx + comp;
                            s[u] += NC ? __ldg(yp) : __ldcg(yp);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long g = g0 + (long long)u * blockDim.x;
            if (g < end) {
                const float sv = dv[u] != 0.f ? s[u] : 0.f;
                const float pn = p_next(pzv[u].y, pzv[u].x, beta);
                reinterpret_cast<float*>(pz)[2 * g] = pn;
                q[g] = sv;
                acc.add(pn, sv);
            }
        }
    }
    return acc;
}

// vec1_item on (p, z) pairs: p read from the pair, the new z written to its
// second half; the same arithmetic and order.
template <int U>
__device__ __forceinline__ void vec1_item_pz(const VecWork& it, const float* dinv, float al, float* x, float* r,
                                             float2* pz, const float* q, DotAcc<float>& srz, DotAcc<float>& srr) {
    srz = DotAcc<float>();
    srr = DotAcc<float>();
    const long long end = it.start + it.count;
    for (long long g0 = it.start + threadIdx.x; g0 < end; g0 += (long long)blockDim.x * U) {
        float pv[U], qv[U], xv[U], rv0[U], dv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {   // all loads first
            const long long g = g0 + (long long)u * blockDim.x;
            if (g < end) {
                pv[u] = reinterpret_cast<const float*>(pz)[2 * g];
                qv[u] = q[g];
                xv[u] = x[g];
                rv0[u] = r[g];
                dv[u] = dinv[g];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long g = g0 + (long long)u * blockDim.x;
            if (g < end) {
                x[g] = fma(al, pv[u], xv[u]);
                const float rv = fma(-al, qv[u], rv0[u]);
                const float zv = dv[u] * rv;
                r[g] = rv;
                reinterpret_cast<float*>(pz)[2 * g + 1] = zv;
                srz.add(rv, zv);
                srr.add(rv, rv);
            }
        }
    }
}

// Resident vector slice: when a CTA keeps one vector work item for a whole
// solve, the item's x, r and D^-1 stay in shared memory (only this CTA reads
// or writes them) and the element-product offsets of each DOF's owners are
// computed once. resident_setup fills them; resident_update_item_pz (below)
// is then the same arithmetic as isum_update_item_pz (same owner order, same
// operations), with only the (p, z) pairs, which the apply of every CTA
// gathers, in global memory.
// soff[c * stride + l]: offset into Y of owner c of DOF start + l, or -1.
template <class V>
__device__ __forceinline__ void resident_setup(const ArrayDev& A, const LocalMap* lm, int ldY, long long start,
                                               int count, const V* dinv, const V* x, const V* r, V* sd, V* sx,
                                               V* sr, int* soff, int stride) {
    const int n = lm->n, n1 = n - 1;
    const int16_t* __restrict__ surf = lm->surf_idx;
    for (int l = threadIdx.x; l < count; l += blockDim.x) {
        const long long g = start + l;
        sd[l] = dinv[g];
        sx[l] = x[g];
        sr[l] = r[g];
        int comp, gx, gy, gz;
        lattice_coords(A, g, comp, gx, gy, gz);
        const int ih0 = gx / n1, jh0 = gy / n1;
        const int ih = min(ih0, A.nx - 1), jh = min(jh0, A.ny - 1);
        const int il = max((gx % n1 == 0) ? ih0 - 1 : ih0, 0), jl = max((gy % n1 == 0) ? jh0 - 1 : jh0, 0);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = (c >> 1) ? jh : jl, i = (c & 1) ? ih : il;
            const bool use = ((c >> 1) == 0 || jh != jl) && ((c & 1) == 0 || ih != il);
            int off = -1;
            if (use) {
                const int sidx = __ldg(surf + (gz * n + (gy - j * n1)) * n + (gx - i * n1));
                if (sidx >= 0) off = (int)((A.block_off + (long long)j * A.nx + i) * ldY + 3 * sidx + comp);
            }
            soff[c * stride + l] = off;
        }
    }
}

// Interface sum fused with the vector update (the second phase of the
// two-phase iteration, whose step length alpha = <r,z> / sum_e p_e^T Y_e was
// folded from the element products), on (p, z) pairs (float2 per DOF): per
// DOF, p = z + beta p (the same fused multiply-add as the apply's gather),
// q = sum of the owners' Y_e in fixed order (masked on constrained rows, never
// stored), x += alpha p, r -= alpha q, z = D^-1 r; the pair, x and r are
// stored and this thread's shares of <r,z> and <r,r> returned. U = 5 DOFs
// per thread with all their loads issued first. The resident variant reads x,
// r, D^-1 and the owner offsets from shared memory (resident_setup).
__device__ __forceinline__ void isum_update_item_pz(const VecWork& it, const ArrayDev& A, const LocalMap* lm,
                                                    const float* __restrict__ dinv, int ldY,
                                                    const float* __restrict__ Y, float2* __restrict__ pz,
                                                    float* __restrict__ x, float* __restrict__ r, float beta,
                                                    float al, DotAcc<float>& srz, DotAcc<float>& srr) {
    constexpr int U = 5;
    const int n = lm->n, n1 = n - 1;
    const int16_t* __restrict__ surf = lm->surf_idx;
    const long long end = it.start + it.count;
    srz = DotAcc<float>();
    srr = DotAcc<float>();
    for (long long g0 = it.start + threadIdx.x; g0 < end; g0 += (long long)blockDim.x * U) {
        float s[U], dv[U], xv[U], rv[U];
        float2 pzv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long g = g0 + (long long)u * blockDim.x;
            s[u] = 0.f;
            dv[u] = xv[u] = rv[u] = 0.f;
            pzv[u] = make_float2(0.f, 0.f);
            if (g < end) {
                dv[u] = dinv[g];
                pzv[u] = pz[g];
                xv[u] = x[g];
                rv[u] = r[g];
                int comp, gx, gy, gz;
                lattice_coords(A, g, comp, gx, gy, gz);
                const int ih0 = gx / n1, jh0 = gy / n1;
                const int ih = min(ih0, A.nx - 1), jh = min(jh0, A.ny - 1);
                const int il = max((gx % n1 == 0) ? ih0 - 1 : ih0, 0), jl = max((gy % n1 == 0) ? jh0 - 1 : jh0, 0);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int j = (c >> 1) ? jh : jl, i = (c & 1) ? ih : il;
                    const bool use = ((c >> 1) == 0 || jh != jl) && ((c & 1) == 0 || ih != il);
                    if (use) {
                        const int sidx = __ldg(surf + (gz * n + (gy - j * n1)) * n + (gx - i * n1));
                        if (sidx >= 0) s[u] += __ldcg(Y + (A.block_off + (long long)j * A.nx + i) * ldY + 3 * sidx + comp);
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long g = g0 + (long long)u * blockDim.x;
            if (g < end) {
                const float qv = dv[u] != 0.f ? s[u] : 0.f;
                const float pn = p_next(pzv[u].y, pzv[u].x, beta);
                const float rn = fmaf(-al, qv, rv[u]);
                const float zn = dv[u] * rn;
                pz[g] = make_float2(pn, zn);
                x[g] = fmaf(al, pn, xv[u]);
                r[g] = rn;
                srz.add(rn, zn);
                srr.add(rn, rn);
            }
        }
    }
}

// resident_update_item_pz in two halves: the loads of one round (U DOFs per
// thread: the pair and the owners' element products summed in fixed order),
// which need neither alpha nor beta, and the update itself. Between them the
// caller may fold alpha while the loads are in flight.
template <int U>
__device__ __forceinline__ void resident_update_load(long long start, int count, int l0,
                                                     const int* __restrict__ soff, int stride,
                                                     const float* __restrict__ Y, const float2* __restrict__ pz,
                                                     float (&s)[U], float2 (&pzv)[U]) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int l = l0 + u * (int)blockDim.x;
        s[u] = 0.f;
        pzv[u] = make_float2(0.f, 0.f);
        if (l < count) {
            pzv[u] = pz[start + l];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int off = soff[c * stride + l];
                if (off >= 0) s[u] += __ldcg(Y + off);
            }
        }
    }
}

template <int U>
__device__ __forceinline__ void resident_update_finish(long long start, int count, int l0, const float* sd, float* sx,
                                                       float* sr, float2* __restrict__ pz, const float (&s)[U],
                                                       const float2 (&pzv)[U], float beta, float al,
                                                       DotAcc<float>& srz, DotAcc<float>& srr) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int l = l0 + u * (int)blockDim.x;
        if (l < count) {
            const float dv = sd[l];
            const float qv = dv != 0.f ? s[u] : 0.f;
            const float pn = p_next(pzv[u].y, pzv[u].x, beta);
            const float rn = fmaf(-al, qv, sr[l]);
            const float zn = dv * rn;
            pz[start + l] = make_float2(pn, zn);
            sx[l] = fmaf(al, pn, sx[l]);
            sr[l] = rn;
            srz.add(rn, zn);
            srr.add(rn, rn);
        }
    }
}

constexpr int kResidentU = 5;   // DOFs per thread per round of the resident update

__device__ __forceinline__ void resident_update_item_pz(long long start, int count, const int* __restrict__ soff,
                                                        int stride, const float* sd, float* sx, float* sr,
                                                        const float* __restrict__ Y, float2* __restrict__ pz,
                                                        float beta, float al, DotAcc<float>& srz,
                                                        DotAcc<float>& srr) {
    constexpr int U = kResidentU;
    srz = DotAcc<float>();
    srr = DotAcc<float>();
    for (int l0 = threadIdx.x; l0 < count; l0 += (int)blockDim.x * U) {
        float s[U];
        float2 pzv[U];
        resident_update_load<U>(start, count, l0, soff, stride, Y, pz, s, pzv);
        resident_update_finish<U>(start, count, l0, sd, sx, sr, pz, s, pzv, beta, al, srz, srr);
    }
}

// Vector update of one work item: x += alpha p, r -= alpha q, z = D^-1 r in
// the vector precision V; returns this thread's shares of <r, z> and <r, r>
// (U DOFs per thread in flight).
template <int U, class V>
__device__ __forceinline__ void vec1_item(const VecWork& it, const V* dinv, V al, V* x, V* r, V* z, const V* p,
                                          const V* q, DotAcc<V>& srz, DotAcc<V>& srr) {
    srz = DotAcc<V>();
    srr = DotAcc<V>();
    const long long end = it.start + it.count;
    for (long long g0 = it.start + threadIdx.x; g0 < end; g0 += (long long)blockDim.x * U) {
        V pv[U], qv[U], xv[U], rv0[U], dv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {   // all loads first
            const long long g = g0 + (long long)u * blockDim.x;
            if (g < end) {
                pv[u] = p[g];
                qv[u] = q[g];
                xv[u] = x[g];
                rv0[u] = r[g];
                dv[u] = dinv[g];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long g = g0 + (long long)u * blockDim.x;
            if (g < end) {
                x[g] = fma(al, pv[u], xv[u]);
                const V rv = fma(-al, qv[u], rv0[u]);
                const V zv = dv[u] * rv;
                r[g] = rv;
                z[g] = zv;
                srz.add(rv, zv);
                srr.add(rv, rv);
            }
        }
    }
}

}  // namespace pi
}  // namespace ms
