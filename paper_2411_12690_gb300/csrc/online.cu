// Global stage of MORE-Stress (section 4.3, Eq. 20) on the GPU.
//
// The reduced global system A_global u = b_global is never assembled. Blocks
// act as abstract elements (section 4.3): block (i, j) of an nx*ny array owns
// the Lagrange-lattice points (i(n-1)+a, j(n-1)+b, c) of its surface nodes
// (a, b, c), so the element-to-global map is arithmetic. One Jacobi-PCG
// iteration is three launches:
//   1. apply:  gather p_e = G_e p for every block (with the pending update
//              p = z + beta p folded into the gather) and form the element
//              products Y_e = A_element[type e] p_e                    (Eq. 18)
//   2. isum:   q_g = sum of Y_e over the <= 4 blocks owning lattice DOF g, in
//              a fixed order (bitwise reproducible); stores the updated p and
//              the <p, q> partial sums
//   3. vec1:   alpha = <r,z>/<p,q>, x += alpha p, r -= alpha q, z = D^-1 r and
//              the <r,z>, <r,r> partials; the last CTA to finish folds them per
//              array (beta, stopping test, iteration count) and sets the
//              loop condition of the CUDA graph.
// Every phase is one launch over the work items of all arrays of a batch (a
// grid-stride persistent loop), each array with its own scalars. The loop runs
// as a CUDA-graph conditional WHILE node: one graph launch per solve, no host
// polling. Constrained DOFs (clamped faces, prescribed values) have D^-1 = 0,
// which keeps r, z, p zero there; prescribed values enter b by lifting (Eq. 13).
//
// Precision: FP64 vectors and FP64 operator in the plain mode; in the mixed
// modes an FP64 outer loop (residual b - A x with the FP64 operator)
// drives an inner PCG with FP32 vectors and a reduced-precision operator; the
// inner dot products are per-thread FP32 partial sums folded in FP64, and the
// step lengths are FP64.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <type_traits>

#include "apply_items.cuh"
#include "pcg_items.cuh"

namespace ms {
namespace {

constexpr int kThreads = 256;
using pi::block_sum;
using pi::for_owners;
using pi::lattice_coords;
using pi::warp_fold;

// ---------------------------------------------------------- a2: rhs, diag
struct RhsArgs {
    const VecWork* vwork;
    int n_vwork;
    const ArrayDev* arrays;
    const LocalMap* lm;
    const uint8_t* site;
    const uint8_t* fixed;   // optional per-DOF prescribed marker
    TypeTab tt;
    int m;
    double* b;
    double* dinv;
};

// b = dT sum_e G_e^T b_element[type e] (Eq. 19 assembled), D = sum_e G_e^T
// diag(A_element[type e]); constrained DOFs and lattice holes get b = 0, D^-1 = 0.
__global__ void __launch_bounds__(kThreads) k_rhs_diag(const __grid_constant__ RhsArgs a) {
    for (int w = blockIdx.x; w < a.n_vwork; w += gridDim.x) {
        const VecWork it = a.vwork[w];
        const ArrayDev A = a.arrays[it.array];
        for (long long g = it.start + threadIdx.x; g < it.start + it.count; g += kThreads) {
            int comp, gx, gy, gz;
            lattice_coords(A, g, comp, gx, gy, gz);
            double bs = 0, ds = 0;
            for_owners(A, a.lm->surf_idx, a.lm->n, gx, gy, gz, [&](long long blk, int s) {
                int t = a.site[blk];
                int k = 3 * s + comp;
                bs += a.tt.br[t][k];
                ds += a.tt.Kr[t][(size_t)k * a.m + k];
            });
            bool fixed = (A.clamp_bottom && gz == 0) || (A.clamp_top && gz == A.Z - 1) ||
                         (a.fixed && a.fixed[g]) || ds == 0.0;
            a.b[g] = fixed ? 0.0 : A.dT * bs;
            a.dinv[g] = fixed ? 0.0 : 1.0 / ds;
        }
    }
}

// ------------------------------------------------------ a3: operator apply
// Element products on CUDA cores; a work item is one panel of 8*RPT rows of
// A_element for a 32-block tile of one type and one array (apply_items.cuh),
// so the items spread evenly over the SMs. Shared: C [NS][m][32], K panel.
template <int RPT>
__global__ void __launch_bounds__(kThreads) k_apply64(const __grid_constant__ ApplyArgs a) {
    extern __shared__ double sm[];
    __shared__ long long base[kTile64];
    __shared__ int offs[3 * kMaxSurf];
    const int n_panels = (a.m + 8 * RPT - 1) / (8 * RPT);
    for (int w = blockIdx.x; w < a.n_work * n_panels; w += gridDim.x) {
        const ApplyWork it = a.work[w / n_panels];
        if (a.st && !a.st[it.array].active) continue;
        __syncthreads();
        ai::apply64_item<RPT>(a, it, w % n_panels, sm, sm + (size_t)a.m * kTile64, base, offs);
    }
}

// Reduced-precision element products on CUDA cores (FP32 vectors), used when
// the tensor-core tile does not cover the basis size.
template <int RPT, int MODE>
__global__ void __launch_bounds__(kThreads) k_apply32(const __grid_constant__ ApplyArgs a) {
    extern __shared__ float smf[];
    __shared__ long long base[kTile64];
    __shared__ int offs[3 * kMaxSurf];
    constexpr int NS = MODE == MSTRESS_BF16X3 ? 2 : 1;
    const int n_panels = (a.m + 8 * RPT - 1) / (8 * RPT);
    for (int w = blockIdx.x; w < a.n_work * n_panels; w += gridDim.x) {
        const ApplyWork it = a.work[w / n_panels];
        if (a.st && !a.st[it.array].active) continue;
        __syncthreads();
        ai::apply32_item<RPT, MODE>(a, it, w % n_panels, smf, smf + (size_t)NS * a.m * kTile64, base, offs);
    }
}

// ---------------------------------------------------- a3: interface sum
struct IsumArgs {
    const VecWork* vwork;
    int n_vwork;
    const ArrayDev* arrays;
    const LocalMap* lm;
    const PcgState* st;     // optional: skip stopped arrays, beta of the p update
    const void* dinv;       // optional, in the vector precision: zero the constrained rows
    int ldY;
    const void* Y;
    void* p;                // direction (updated in place when z is given)
    const void* z;          // optional: p = z + beta p before use
    void* q;
    double* part_pq;        // optional
};

// q_g = sum over owning blocks of Y_e[local DOF] (owner computes, fixed order).
template <class V, class YT>
__global__ void __launch_bounds__(kThreads) k_isum(const __grid_constant__ IsumArgs a) {
    __shared__ double sh[kThreads / 32];
    for (int w = blockIdx.x; w < a.n_vwork; w += gridDim.x) {
        const VecWork it = a.vwork[w];
        if (a.st && !a.st[it.array].active) continue;
        const ArrayDev A = a.arrays[it.array];
        const V beta = a.st ? (V)a.st[it.array].beta : V(0);
        const pi::DotAcc<V> acc = pi::isum_item<4, V, YT>(it, A, a.lm, static_cast<const V*>(a.dinv), a.ldY,
                                              static_cast<const YT*>(a.Y), static_cast<V*>(a.p),
                                              static_cast<const V*>(a.z), static_cast<V*>(a.q), beta);
        if (a.part_pq) {
            const double t = block_sum(acc, sh);
            if (threadIdx.x == 0) a.part_pq[w] = t;
        }
    }
}

// ------------------------------------------------------- a4: PCG vectors
struct VecArgs {
    const VecWork* vwork;
    int n_vwork;
    const ArrayDev* arrays;
    int n_arrays;
    PcgState* st;
    const double* dinv;
    const void* dinv_v;     // dinv in the vector precision
    void *x, *r, *z, *p, *q;
    void* pz;               // optional: (p, z) pairs of the two-phase tensor-core solver (FP32)
    const void* rhs;        // init / residual: right-hand side (FP64)
    double *part_pq, *part_rz, *part_rr;
    int* flag;              // [0] any active, [1] CTA ticket, [2] device error, [3] loop count
    int loop_cap;           // hard cap on loop iterations of the graph WHILE node
    int use_cond;
    cudaGraphConditionalHandle cond;
};

// x = 0, r = rhs on free DOFs, z = D^-1 r, p = 0 (so the first fused update
// gives p = z); partials <r,z>, <r,r>.
template <class V>
__global__ void __launch_bounds__(kThreads) k_pcg_init(const __grid_constant__ VecArgs a) {
    __shared__ double sh[kThreads / 32];
    V *x = (V*)a.x, *r = (V*)a.r, *z = (V*)a.z, *p = (V*)a.p;
    const double* rhs = (const double*)a.rhs;
    for (int w = blockIdx.x; w < a.n_vwork; w += gridDim.x) {
        const VecWork it = a.vwork[w];
        double srz = 0, srr = 0;
        for (long long g = it.start + threadIdx.x; g < it.start + it.count; g += kThreads) {
            double d = a.dinv[g];
            V rv = d != 0.0 ? (V)rhs[g] : (V)0;
            V zv = (V)(d * (double)rv);
            x[g] = (V)0;
            r[g] = rv;
            z[g] = zv;
            p[g] = (V)0;
            if (a.pz) static_cast<float2*>(a.pz)[g] = make_float2(0.f, (float)zv);
            srz += (double)rv * (double)zv;
            srr += (double)rv * (double)rv;
        }
        srz = block_sum(srz, sh);
        srr = block_sum(srr, sh);
        if (threadIdx.x == 0) { a.part_rz[w] = srz; a.part_rr[w] = srr; }
    }
}

// alpha, x += alpha p, r -= alpha q, z = D^-1 r, partials; then the last CTA
// folds the partials of every active array: beta = <r,z>_new / <r,z>_old,
// stopping test on <r,r>, iteration count, and the graph loop condition.
template <class V>
__global__ void __launch_bounds__(kThreads) k_vec1(const __grid_constant__ VecArgs a) {
    __shared__ double sh[kThreads / 32];
    __shared__ double s_alpha;
    __shared__ int s_last;
    V *x = (V*)a.x, *r = (V*)a.r, *z = (V*)a.z;
    const V *p = (const V*)a.p, *q = (const V*)a.q;
    for (int w = blockIdx.x; w < a.n_vwork; w += gridDim.x) {
        const VecWork it = a.vwork[w];
        const PcgState st = a.st[it.array];
        if (!st.active) continue;
        const ArrayDev A = a.arrays[it.array];
        __syncthreads();
        if (threadIdx.x < 32) {
            double pq = warp_fold(a.part_pq + A.vwork_off, A.n_vwork);
            double al = st.rz / pq;
            if (threadIdx.x == 0) s_alpha = (pq > 0 && isfinite(al)) ? al : 0.0;
        }
        __syncthreads();
        const V al = (V)s_alpha;
        pi::DotAcc<V> srz, srr;
        pi::vec1_item<4, V>(it, static_cast<const V*>(a.dinv_v), al, x, r, z, p, q, srz, srr);
        const double rz = block_sum(srz, sh);
        const double rr = block_sum(srr, sh);
        if (threadIdx.x == 0) { a.part_rz[w] = rz; a.part_rr[w] = rr; }
    }
    // ---- last CTA: per-array scalar phase
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&a.flag[1], 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int any = 0;
    for (int k = warp; k < a.n_arrays; k += kThreads / 32) {
        PcgState s = a.st[k];
        if (!s.active) continue;
        const ArrayDev A = a.arrays[k];
        double pq = warp_fold(a.part_pq + A.vwork_off, A.n_vwork);
        double rz = warp_fold(a.part_rz + A.vwork_off, A.n_vwork);
        double rr = warp_fold(a.part_rr + A.vwork_off, A.n_vwork);
        if (lane == 0) {
            s.iters += 1;
            if (!(pq > 0) || !isfinite(rz) || !isfinite(rr)) {
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
            any |= s.active;
        }
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        a.flag[1] = 0;
        int loops = a.flag[3] + 1;
        a.flag[3] = loops;
        if (loops >= a.loop_cap) any = 0;
        a.flag[0] = any;
        if (a.use_cond) cudaGraphSetConditional(a.cond, any ? 1u : 0u);
    }
}

// a5: r = b - q on free DOFs (FP64 residual of the outer refinement loop),
// and its partial <r, r>.
__global__ void __launch_bounds__(kThreads) k_residual(const __grid_constant__ VecArgs a) {
    __shared__ double sh[kThreads / 32];
    const double* b = (const double*)a.rhs;
    const double* q = (const double*)a.q;
    double* r = (double*)a.r;
    for (int w = blockIdx.x; w < a.n_vwork; w += gridDim.x) {
        const VecWork it = a.vwork[w];
        double srr = 0;
        for (long long g = it.start + threadIdx.x; g < it.start + it.count; g += kThreads) {
            double rv = a.dinv[g] != 0.0 ? b[g] - q[g] : 0.0;
            r[g] = rv;
            srr += rv * rv;
        }
        srr = block_sum(srr, sh);
        if (threadIdx.x == 0) a.part_rr[w] = srr;
    }
}

// x64 += d (the inner solution) for arrays still refining.
template <class D>
__global__ void __launch_bounds__(kThreads) k_correct(const VecWork* vwork, int n_vwork, const PcgState* outer,
                                                      double* x, const D* d) {
    for (int w = blockIdx.x; w < n_vwork; w += gridDim.x) {
        const VecWork it = vwork[w];
        if (!outer[it.array].active) continue;
        for (long long g = it.start + threadIdx.x; g < it.start + it.count; g += kThreads) x[g] += (double)d[g];
    }
}

__global__ void k_add_bc(long long n, double* x, const double* xbc) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) x[i] += xbc[i];
}

__global__ void k_narrow(long long n, const double* x, float* y) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = (float)x[i];
}

__global__ void k_widen(long long n, const float* x, double* y) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = (double)x[i];
}

__global__ void k_lift_rhs(long long n, double* b, const double* Axbc, const double* dinv) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n && dinv[i] != 0.0) b[i] -= Axbc[i];
}

// ----------------------------------------------------- a4: scalar phase
// mode 1: start of a PCG run (tolerance from rtol, beta = 0, gate: only arrays
// active in `gate` start); mode 2: outer refinement check (part_rr holds
// ||b - A x||^2 partials, st.bb = ||b||^2, iters counts refinement steps).
struct ScalarArgs {
    int n_arrays;
    const ArrayDev* arrays;
    PcgState* st;
    const double *part_rz, *part_rr;
    int* flag;
    int mode;
    double rtol;
    int max_iter;
    const PcgState* gate;
};

__global__ void __launch_bounds__(1024) k_scalars(const __grid_constant__ ScalarArgs a) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ int s_count;
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();
    int any = 0;
    for (int k = warp; k < a.n_arrays; k += 32) {
        const ArrayDev A = a.arrays[k];
        PcgState s = a.st[k];
        if (a.mode == 1) {
            double rz = warp_fold(a.part_rz + A.vwork_off, A.n_vwork);
            double rr = warp_fold(a.part_rr + A.vwork_off, A.n_vwork);
            if (lane == 0) {
                bool gate = a.gate ? a.gate[k].active != 0 : true;
                s.rz = rz;
                s.rr = rr;
                s.bb = rr;
                // the inner solve of a refinement step (gate = outer state) also
                // stops once its residual is below a tenth of the outer
                // tolerance: the last step needs only the reduction that is
                // left, and the outer FP64 residual decides convergence
                s.tol2 = a.rtol * a.rtol * rr;
                if (a.gate) s.tol2 = fmax(s.tol2, 0.01 * a.gate[k].tol2);
                s.beta = 0.0;
                s.iters = 0;
                s.max_iter = a.max_iter;
                s.status = isfinite(rr) ? MSTRESS_OK : MSTRESS_ENUMERIC;
                s.active = (gate && rr > 0 && isfinite(rr)) ? 1 : 0;
                a.st[k] = s;
            }
        } else {
            double rr = warp_fold(a.part_rr + A.vwork_off, A.n_vwork);
            if (lane == 0) {
                s.rr = rr;
                if (s.active) {
                    if (!isfinite(rr)) { s.active = 0; s.status = MSTRESS_ENUMERIC; }
                    else if (rr <= a.rtol * a.rtol * s.bb) { s.active = 0; s.status = MSTRESS_OK; }
                    else if (s.iters >= s.max_iter) { s.active = 0; s.status = MSTRESS_ENOT_CONVERGED; }
                    else s.iters += 1;
                }
                a.st[k] = s;
            }
        }
        if (lane == 0 && a.st[k].active) {
            any = 1;
            atomicAdd(&s_count, 1);
        }
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        a.flag[0] = any;
        a.flag[1] = 0;
        a.flag[3] = 0;
        a.flag[4] = s_count;   // arrays active (persistent solver)
    }
}

// ------------------------------------------------------------ launches
int grid_for(mstress_sol_s* s, int items, int per_sm) {
    return std::max(1, std::min(items, s->ctx->num_sms * per_sm));
}

constexpr int kMaxDynSmem = 200 * 1024;

// Raise the dynamic shared-memory limit of every apply kernel once per device
// (outside any stream capture).
void configure_apply_kernels(int device) {
    static bool done[64] = {};
    if (device < 0 || device >= 64 || done[device]) return;
    auto set = [](auto k) { MS_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem)); };
    set(k_apply64<2>);
    set(k_apply64<4>);
    set(k_apply32<2, MSTRESS_TF32>);
    set(k_apply32<2, MSTRESS_BF16>);
    set(k_apply32<2, MSTRESS_BF16X3>);
    set(k_apply32<4, MSTRESS_TF32>);
    set(k_apply32<4, MSTRESS_BF16>);
    set(k_apply32<4, MSTRESS_BF16X3>);
    configure_tc_kernels();
    done[device] = true;
}

template <class KER>
void launch_with_smem(KER kernel, mstress_sol_s* s, size_t smem, const ApplyArgs& a, int items_per_work = 1) {
    MS_REQUIRE(smem <= (size_t)kMaxDynSmem, MSTRESS_EINVAL, "apply tile does not fit in shared memory");
    const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(8, (200 * 1024) / (smem + 4096)));
    kernel<<<grid_for(s, a.n_work * items_per_work, per_sm), kThreads, smem, s->ctx->stream>>>(a);
    MS_LAUNCH_CHECK();
}

VecArgs vec_args(mstress_sol_s* s, PcgVectors& v) {
    VecArgs a;
    std::memset(&a, 0, sizeof(a));
    a.vwork = s->d_vwork.as<VecWork>();
    a.n_vwork = s->n_vwork;
    a.arrays = s->d_arrays.as<ArrayDev>();
    a.n_arrays = s->n_arrays;
    a.st = v.state.as<PcgState>();
    a.dinv = s->dinv.as<double>();
    a.dinv_v = &v == &s->v32 ? s->dinv32.ptr : s->dinv.ptr;
    a.x = v.x.ptr;
    a.r = v.r.ptr;
    a.z = v.z.ptr;
    a.p = v.p.ptr;
    a.q = v.q.ptr;
    a.pz = &v == &s->v32 ? s->pz.ptr : nullptr;
    a.part_pq = s->part.as<double>();
    a.part_rz = a.part_pq + s->n_vwork;
    a.part_rr = a.part_rz + s->n_vwork;
    a.flag = s->flag.as<int>();
    a.loop_cap = 1 << 30;
    return a;
}

ScalarArgs scalar_args(mstress_sol_s* s, PcgVectors& v, int mode, double rtol, int max_iter, const PcgState* gate) {
    ScalarArgs a;
    a.n_arrays = s->n_arrays;
    a.arrays = s->d_arrays.as<ArrayDev>();
    a.st = v.state.as<PcgState>();
    a.part_rz = s->part.as<double>() + s->n_vwork;
    a.part_rr = a.part_rz + s->n_vwork;
    a.flag = s->flag.as<int>();
    a.mode = mode;
    a.rtol = rtol;
    a.max_iter = max_iter;
    a.gate = gate;
    return a;
}

}  // namespace

ApplyArgs apply_args(mstress_sol_s* s, const void* x, const void* z, const PcgState* st, void* Y, bool tc) {
    ApplyArgs a;
    std::memset(&a, 0, sizeof(a));
    a.work = tc ? s->d_awork_tc.as<ApplyWork>() : s->d_awork.as<ApplyWork>();
    a.n_work = tc ? s->n_awork_tc : s->n_awork;
    a.blist = s->d_blist.as<int>();
    a.bref = s->d_bref.as<BlockRef>();
    a.arrays = s->d_arrays.as<ArrayDev>();
    a.lm = s->d_lm.as<LocalMap>();
    a.st = st;
    a.tt = s->tt;
    a.m = s->m;
    a.ldY = s->ldY;
    a.x = x;
    a.z = z;
    a.Y = Y;
    a.err = s->flag.as<int>() + 2;
    return a;
}

void launch_apply(mstress_sol_s* s, int prec, const void* x, const void* z, bool vec_fp32, const PcgState* st,
                  void* Y) {
    const int m = s->m;
    if (prec == MSTRESS_FP64) {
        MS_REQUIRE(!vec_fp32, MSTRESS_EINVAL, "FP64 apply needs FP64 vectors");
        ApplyArgs a = apply_args(s, x, z, st, Y, false);
        if (apply_rpt(m, 8, 1) == 2)
            launch_with_smem(k_apply64<2>, s, (size_t)(m * kTile64 + 16 * m) * sizeof(double), a, (m + 15) / 16);
        else
            launch_with_smem(k_apply64<4>, s, (size_t)(m * kTile64 + 32 * m) * sizeof(double), a, (m + 31) / 32);
        return;
    }
    MS_REQUIRE(vec_fp32, MSTRESS_EINVAL, "reduced-precision apply needs FP32 vectors");
    if (s->use_tc) {
        launch_apply_tc(s, prec, apply_args(s, x, z, st, Y, true));
        return;
    }
    ApplyArgs a = apply_args(s, x, z, st, Y, false);
    const int ns = prec == MSTRESS_BF16X3 ? 2 : 1;
    if (apply_rpt(m, 4, ns) == 2) {
        const size_t smem = (size_t)ns * (m * kTile64 + 16 * m) * sizeof(float);
        const int panels = (m + 15) / 16;
        if (prec == MSTRESS_TF32) launch_with_smem(k_apply32<2, MSTRESS_TF32>, s, smem, a, panels);
        else if (prec == MSTRESS_BF16) launch_with_smem(k_apply32<2, MSTRESS_BF16>, s, smem, a, panels);
        else launch_with_smem(k_apply32<2, MSTRESS_BF16X3>, s, smem, a, panels);
    } else {
        const size_t smem = (size_t)ns * (m * kTile64 + 32 * m) * sizeof(float);
        const int panels = (m + 31) / 32;
        if (prec == MSTRESS_TF32) launch_with_smem(k_apply32<4, MSTRESS_TF32>, s, smem, a, panels);
        else if (prec == MSTRESS_BF16) launch_with_smem(k_apply32<4, MSTRESS_BF16>, s, smem, a, panels);
        else launch_with_smem(k_apply32<4, MSTRESS_BF16X3>, s, smem, a, panels);
    }
}

void launch_isum(mstress_sol_s* s, const void* Y, bool y_fp32, void* p, const void* z, void* q, bool vec_fp32,
                 const void* dinv, const PcgState* st, double* part_pq) {
    IsumArgs a;
    a.vwork = s->d_vwork.as<VecWork>();
    a.n_vwork = s->n_vwork;
    a.arrays = s->d_arrays.as<ArrayDev>();
    a.lm = s->d_lm.as<LocalMap>();
    a.st = st;
    a.dinv = dinv;
    a.ldY = s->ldY;
    a.Y = Y;
    a.p = p;
    a.z = z;
    a.q = q;
    a.part_pq = part_pq;
    int g = grid_for(s, s->n_vwork, 8);
    cudaStream_t stream = s->ctx->stream;
    if (!vec_fp32 && !y_fp32) k_isum<double, double><<<g, kThreads, 0, stream>>>(a);
    else if (vec_fp32 && y_fp32) k_isum<float, float><<<g, kThreads, 0, stream>>>(a);
    else MS_REQUIRE(false, MSTRESS_EINVAL, "unsupported isum types");
    MS_LAUNCH_CHECK();
}

namespace {

// One PCG iteration over all arrays: apply, interface sum, vector update.
template <class V>
void pcg_iteration(mstress_sol_s* s, PcgVectors& v, int prec, int use_cond, cudaGraphConditionalHandle cond,
                   int loop_cap) {
    constexpr bool f32 = std::is_same<V, float>::value;
    cudaStream_t stream = s->ctx->stream;
    const PcgState* st = v.state.as<PcgState>();
    launch_apply(s, prec, v.p.ptr, v.z.ptr, f32, st, s->Y.ptr);   // gathers p = z + beta p
    launch_isum(s, s->Y.ptr, f32, v.p.ptr, v.z.ptr, v.q.ptr, f32, f32 ? s->dinv32.ptr : s->dinv.ptr, st,
                s->part.as<double>());
    VecArgs va = vec_args(s, v);
    va.use_cond = use_cond;
    va.cond = cond;
    va.loop_cap = loop_cap;
    k_vec1<V><<<grid_for(s, s->n_vwork, 8), kThreads, 0, stream>>>(va);
    MS_LAUNCH_CHECK();
}

// Start a PCG run on right-hand side rhs (FP64 device vector): x = 0, r = rhs
// on free DOFs, z = D^-1 r, p = 0, beta = 0; tolerance rtol relative to ||rhs||.
template <class V>
void pcg_start(mstress_sol_s* s, PcgVectors& v, const double* rhs, double rtol, int max_iter, const PcgState* gate) {
    cudaStream_t stream = s->ctx->stream;
    VecArgs va = vec_args(s, v);
    va.rhs = rhs;
    k_pcg_init<V><<<grid_for(s, s->n_vwork, 8), kThreads, 0, stream>>>(va);
    MS_LAUNCH_CHECK();
    ScalarArgs sa = scalar_args(s, v, 1, rtol, max_iter, gate);
    k_scalars<<<1, 1024, 0, stream>>>(sa);
    MS_LAUNCH_CHECK();
}

constexpr int kChunkIters = 16;

// Build the solve's graph: one conditional WHILE node whose body is one PCG
// iteration; the last CTA of the vector phase clears the condition when no
// array is still iterating (or the loop cap is reached).
template <class V>
bool build_while_graph(mstress_sol_s* s, PcgVectors& v, int prec, int gi, int max_iter) {
    cudaStream_t stream = s->ctx->stream;
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return false;
    cudaGraphConditionalHandle h;
    alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
    std::memset(cp_raw, 0, sizeof(cp_raw));
    cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
    cudaGraphNode_t node;
    bool ok = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) == cudaSuccess;
    }
    if (ok) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        ok = cudaStreamBeginCaptureToGraph(stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
             cudaSuccess;
        if (ok) {
            g_capturing = true;
            try {
                if constexpr (std::is_same<V, float>::value) {
                    if (pcg_wide(s, prec)) pcg_iteration_wide(s, v, prec, 1, h, max_iter + 2);
                    else pcg_iteration<V>(s, v, prec, 1, h, max_iter + 2);
                } else {
                    pcg_iteration<V>(s, v, prec, 1, h, max_iter + 2);
                }
            } catch (...) {
                ok = false;
            }
            g_capturing = false;
            cudaGraph_t out = nullptr;
            ok = (cudaStreamEndCapture(stream, &out) == cudaSuccess) && ok;
        }
    }
    if (ok) ok = cudaGraphInstantiate(&s->graph[gi], g, 0) == cudaSuccess;
    cudaGraphDestroy(g);
    cudaGetLastError();
    if (!ok) s->graph[gi] = nullptr;
    s->graph_iters[gi] = std::is_same<V, float>::value && pcg_wide(s, prec) ? 5 : 3;   // kernel nodes per loop iteration
    return ok;
}

// Iterate until every array has stopped.
template <class V>
void pcg_run(mstress_sol_s* s, PcgVectors& v, int prec, int max_iter) {
    constexpr int gi = std::is_same<V, float>::value ? 1 : 0;
    cudaStream_t stream = s->ctx->stream;
    int* flag = s->flag.as<int>();
    // preferred: one persistent cooperative launch for the whole run, except
    // for large batches on the streamed apply (per-phase launches, same bits)
    const bool wide = std::is_same<V, float>::value && pcg_wide(s, prec);
    // (no synchronisation: a wait that expired is reported by the next check of the
    // device error word, in the refinement check or at the end of the solve)
    if (!wide && pcg_run_persistent(s, v, prec, max_iter, std::is_same<V, float>::value)) return;
    if (stream != nullptr && !s->graph[gi] && !s->no_while[gi]) s->no_while[gi] = !build_while_graph<V>(s, v, prec, gi, max_iter);
    if (s->graph[gi]) {
        MS_CUDA(cudaGraphLaunch(s->graph[gi], stream));
        MS_CUDA(cudaMemcpyAsync(s->ctx->h_flag, flag, 4 * sizeof(int), cudaMemcpyDeviceToHost, stream));
        MS_CUDA(cudaStreamSynchronize(stream));
        note_launches((long long)s->ctx->h_flag[3] * s->graph_iters[gi]);
        return;
    }
    // no graph (legacy default stream, or conditional nodes unavailable):
    // launch chunks of iterations and poll the any-active flag between them
    for (int done_iters = 0; done_iters < max_iter + 2; done_iters += kChunkIters) {
        for (int k = 0; k < kChunkIters; ++k) {
            if constexpr (std::is_same<V, float>::value) {
                if (wide) {
                    pcg_iteration_wide(s, v, prec, 0, 0, max_iter + 2);
                    continue;
                }
            }
            pcg_iteration<V>(s, v, prec, 0, 0, max_iter + 2);
        }
        MS_CUDA(cudaMemcpyAsync(s->ctx->h_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, stream));
        MS_CUDA(cudaStreamSynchronize(stream));
        if (s->ctx->h_flag[0] == 0) break;
    }
}

// FP64 residual r = b - A x (a5) and the outer stopping test; returns whether
// any array still needs a refinement step. Y must be an FP64 element buffer.
bool outer_check(mstress_sol_s* s, void* Y64, int max_outer, bool x_zero) {
    cudaStream_t stream = s->ctx->stream;
    PcgVectors& v = s->v64;
    if (!x_zero) {
        launch_apply(s, MSTRESS_FP64, v.x.ptr, nullptr, false, nullptr, Y64);
        launch_isum(s, Y64, false, v.x.ptr, nullptr, v.q.ptr, false, s->dinv.as<double>(), nullptr, nullptr);
        VecArgs va = vec_args(s, v);
        va.rhs = s->b.ptr;
        k_residual<<<grid_for(s, s->n_vwork, 8), kThreads, 0, stream>>>(va);
        MS_LAUNCH_CHECK();
    }
    // x_zero: x = 0 since refine_start, whose start kernel left r = b on the free DOFs
    // and its <r, r> partials, in the same loop and order k_residual uses
    // (b - 0 = b): nothing to recompute
    ScalarArgs sa = scalar_args(s, v, 2, s->ctx->opts.rtol, max_outer, nullptr);
    k_scalars<<<1, 1024, 0, stream>>>(sa);
    MS_LAUNCH_CHECK();
    MS_CUDA(cudaMemcpyAsync(s->ctx->h_flag, s->flag.ptr, 4 * sizeof(int), cudaMemcpyDeviceToHost, stream));
    MS_CUDA(cudaStreamSynchronize(stream));
    flush_inner_iters(s);
    MS_REQUIRE(s->ctx->h_flag[2] == 0, MSTRESS_EDEVICE_TIMEOUT,
               "a tensor-core wait or a grid barrier timed out on the device");
    return s->ctx->h_flag[0] != 0;
}

}  // namespace

// -------------------------------------------------------- solve set-up
void validate_and_build(mstress_sol_s* s, const std::vector<LayoutIn>& in) {
    mstress_ctx ctx = s->ctx;
    for (auto& li : in) {
        const mstress_layout* L = li.L;
        MS_REQUIRE(L, MSTRESS_EINVAL, "layout is NULL");
        MS_REQUIRE(L->nx >= 1 && L->ny >= 1, MSTRESS_EINVAL, "array needs nx, ny >= 1");
        MS_REQUIRE((int64_t)L->nx * L->ny <= (1 << 26), MSTRESS_EINVAL, "array too large");
        MS_REQUIRE(L->site_type && L->blocks && L->n_blocks >= 1, MSTRESS_EINVAL, "layout needs site_type and blocks");
        MS_REQUIRE(std::isfinite(li.dT), MSTRESS_EINVAL, "dT must be finite");
        for (int k = 0; k < L->n_blocks; ++k) {
            mstress_block b = L->blocks[k];
            MS_REQUIRE(b && b->ctx == ctx, MSTRESS_EINVAL, "block is NULL or from another context");
            if (std::find(s->types.begin(), s->types.end(), b) == s->types.end()) s->types.push_back(b);
        }
        for (int k = 1; k < L->n_blocks; ++k) {
            mstress_block a = L->blocks[0], b = L->blocks[k];
            MS_REQUIRE(a->lx == b->lx && a->ly == b->ly && a->lz == b->lz, MSTRESS_EINVAL,
                       "blocks of one array must share their dimensions");
        }
        for (int64_t k = 0; k < (int64_t)L->nx * L->ny; ++k)
            MS_REQUIRE(L->site_type[k] < L->n_blocks, MSTRESS_EINVAL, "site_type out of range");
        const mstress_bc* bc = li.bc;
        if (bc) {
            MS_REQUIRE(bc->n_prescribed == 0 || (bc->prescribed_dof && bc->prescribed_val), MSTRESS_EINVAL,
                       "prescribed arrays are NULL");
            MS_REQUIRE(bc->clamp_bottom || bc->clamp_top || bc->n_prescribed > 0, MSTRESS_EINVAL,
                       "no constrained DOF: the reduced system is singular (rigid motions)");
        }
    }
    MS_REQUIRE((int)s->types.size() <= kMaxTypes, MSTRESS_EINVAL, "too many block models in one solve");
    s->n_types = (int)s->types.size();
    mstress_block t0 = s->types[0];
    for (auto b : s->types)
        MS_REQUIRE(b->n == t0->n && b->n_el == t0->n_el && b->n_dof == t0->n_dof, MSTRESS_EINVAL,
                   "all block models of a solve need the same basis order and mesh size");
    s->n = t0->n;
    s->m = t0->m;
    s->ldY = (int)round_up(s->m, 16);
    configure_apply_kernels(ctx->device);
    s->n_el = t0->n_el;
    s->n_dof_block = t0->n_dof;
    s->use_tc = s->precision != MSTRESS_FP64 && tc_supported(s->m);
    LocalMap lm = make_local_map(s->n);
    s->n_arrays = (int)in.size();
    const int n1 = s->n - 1;

    std::vector<BlockRef> bref;
    std::vector<VecWork> vwork;
    std::vector<ApplyWork> awork, awork_tc, awork_rec;
    std::vector<int> blist;
    std::vector<uint8_t> fixed;
    std::vector<double> xbc;
    bool any_presc = false;
    int64_t total_blocks = 0;
    for (auto& li : in) {
        if (li.bc && li.bc->n_prescribed) any_presc = true;
        total_blocks += (int64_t)li.L->nx * li.L->ny;
    }
    // tensor-core apply tiles: about one tile per SM (a multiple of 8 blocks,
    // at most 128); the autotuner may replace it (solve_prepare)
    s->tc_tile = (int)std::min<int64_t>(kTileTC, std::max<int64_t>(8, round_up((total_blocks + ctx->num_sms - 1) /
                                                                                   ctx->num_sms, 8)));
    int64_t vec_off = 0, block_off = 0;
    int n_groups = 0;
    for (int a = 0; a < s->n_arrays; ++a) {
        const mstress_layout* L = in[a].L;
        ArrayDev A{};
        A.nx = L->nx;
        A.ny = L->ny;
        A.X = L->nx * n1 + 1;
        A.Y = L->ny * n1 + 1;
        A.Z = s->n;
        A.clamp_bottom = in[a].bc ? in[a].bc->clamp_bottom : 1;
        A.clamp_top = in[a].bc ? in[a].bc->clamp_top : 0;
        A.vec_off = vec_off;
        A.n_dof = 3LL * A.X * A.Y * A.Z;
        A.block_off = block_off;
        A.dT = in[a].dT;
        A.vwork_off = (int)vwork.size();
        const int64_t chunk = s->precision == MSTRESS_FP64 || !s->use_tc ? kVecChunk64
                              : tc_streamed(s->m)                   ? kVecChunk32
                                                                    : kVecChunkTC;
        for (int64_t st = 0; st < A.n_dof; st += chunk)
            vwork.push_back(VecWork{a, 0, vec_off + st, std::min<int64_t>(chunk, A.n_dof - st)});
        A.n_vwork = (int)vwork.size() - A.vwork_off;
        std::vector<int> tmap(L->n_blocks);
        for (int k = 0; k < L->n_blocks; ++k)
            tmap[k] = (int)(std::find(s->types.begin(), s->types.end(), L->blocks[k]) - s->types.begin());
        std::vector<std::vector<int>> per_type(s->n_types);
        for (int j = 0; j < L->ny; ++j)
            for (int i = 0; i < L->nx; ++i) {
                int t = tmap[L->site_type[(int64_t)j * L->nx + i]];
                int64_t e = block_off + (int64_t)j * L->nx + i;
                bref.push_back(BlockRef{a, i, j, t});
                s->site.push_back((uint8_t)t);
                per_type[t].push_back((int)e);
            }
        // tiles of one type and one array over the same block list: 32 blocks
        // (CUDA-core kernels), tc_tile blocks (tensor-core apply) and 128
        // blocks (tensor-core recovery); every tile size is a multiple of 8,
        // so a tile starts on an 8-block group of its (array, type) run
        A.grp_off = n_groups;
        for (int t = 0; t < s->n_types; ++t) {
            auto& v = per_type[t];
            const int start = (int)blist.size();
            const int grp = n_groups;
            for (int e : v) blist.push_back(e);
            auto tiles = [&](std::vector<ApplyWork>& out, size_t tile) {
                for (size_t st = 0; st < v.size(); st += tile)
                    out.push_back(ApplyWork{t, a, start + (int)st, (int)std::min<size_t>(tile, v.size() - st),
                                            grp + (int)(st / 8)});
            };
            tiles(awork, kTile64);
            tiles(awork_tc, (size_t)s->tc_tile);
            tiles(awork_rec, kTileTC);
            if (!v.empty()) s->h_seg.push_back(ApplyWork{t, a, start, (int)v.size(), grp});
            n_groups += (int)((v.size() + 7) / 8);
        }
        A.n_grp = n_groups - A.grp_off;
        if (any_presc) {
            fixed.resize(vec_off + A.n_dof, 0);
            xbc.resize(vec_off + A.n_dof, 0.0);
            const mstress_bc* bc = in[a].bc;
            if (bc)
                for (size_t k = 0; k < bc->n_prescribed; ++k) {
                    int64_t d = bc->prescribed_dof[k];
                    MS_REQUIRE(d >= 0 && d < A.n_dof, MSTRESS_EINVAL, "prescribed DOF out of range");
                    MS_REQUIRE(std::isfinite(bc->prescribed_val[k]), MSTRESS_EINVAL, "prescribed value not finite");
                    fixed[vec_off + d] = 1;
                    xbc[vec_off + d] = bc->prescribed_val[k];
                }
        }
        s->arrays.push_back(A);
        vec_off += A.n_dof;
        block_off += (int64_t)L->nx * L->ny;
    }
    s->n_vec = vec_off;
    s->n_blocks = block_off;
    MS_REQUIRE(s->n_blocks < (1LL << 31), MSTRESS_EINVAL, "too many blocks");
    s->n_vwork = (int)vwork.size();
    s->n_grp = n_groups;
    s->n_awork = (int)awork.size();
    s->n_awork_tc = (int)awork_tc.size();
    s->n_awork_rec = (int)awork_rec.size();
    s->h_awork = awork;
    s->h_awork_rec = awork_rec;

    cudaStream_t st = ctx->stream;
    // the work lists go through one pinned staging buffer, so that their copies
    // are asynchronous (the stream's earlier work, which may still read the
    // staging buffer of a previous set-up, is waited for first)
    {
        const size_t need = sizeof(LocalMap) + s->arrays.size() * sizeof(ArrayDev) + bref.size() * sizeof(BlockRef) +
                            blist.size() * sizeof(int) +
                            (awork.size() + awork_tc.size() + awork_rec.size()) * sizeof(ApplyWork) +
                            vwork.size() * sizeof(VecWork) + s->site.size() + fixed.size() +
                            xbc.size() * sizeof(double) + 16 * 64;
        MS_CUDA(cudaStreamSynchronize(st));
        if (ctx->h_stage_bytes < need) {
            if (ctx->h_stage) MS_CUDA(cudaFreeHost(ctx->h_stage));
            ctx->h_stage = nullptr;
            ctx->h_stage_bytes = 0;
            MS_CUDA(cudaHostAlloc((void**)&ctx->h_stage, need, cudaHostAllocDefault));
            ctx->h_stage_bytes = need;
        }
    }
    size_t stage_off = 0;
    auto up = [&](DBuf& d, const void* src, size_t bytes) {
        alloc_into(ctx, d, bytes, false);
        if (bytes == 0) return;
        std::memcpy(ctx->h_stage + stage_off, src, bytes);
        MS_CUDA(cudaMemcpyAsync(d.ptr, ctx->h_stage + stage_off, bytes, cudaMemcpyHostToDevice, st));
        stage_off += (bytes + 63) / 64 * 64;
    };
    up(s->d_lm, &lm, sizeof(LocalMap));
    up(s->d_arrays, s->arrays.data(), s->arrays.size() * sizeof(ArrayDev));
    up(s->d_bref, bref.data(), bref.size() * sizeof(BlockRef));
    up(s->d_blist, blist.data(), blist.size() * sizeof(int));
    up(s->d_awork, awork.data(), awork.size() * sizeof(ApplyWork));
    up(s->d_awork_tc, awork_tc.data(), awork_tc.size() * sizeof(ApplyWork));
    up(s->d_awork_rec, awork_rec.data(), awork_rec.size() * sizeof(ApplyWork));
    up(s->d_vwork, vwork.data(), vwork.size() * sizeof(VecWork));
    up(s->d_site, s->site.data(), s->site.size());
    if (any_presc) {
        up(s->fixed, fixed.data(), fixed.size());
        up(s->xbc, xbc.data(), xbc.size() * sizeof(double));
    }
    for (int t = 0; t < s->n_types; ++t) {
        s->tt.Kr[t] = s->types[t]->Kr.as<double>();
        s->tt.br[t] = s->types[t]->br.as<double>();
    }
    const size_t nv = (size_t)s->n_vec;
    alloc_into(ctx, s->b, nv * sizeof(double), false);
    alloc_into(ctx, s->dinv, nv * sizeof(double), false);
    alloc_into(ctx, s->v64.x, nv * sizeof(double));
    alloc_into(ctx, s->v64.r, nv * sizeof(double), false);
    alloc_into(ctx, s->v64.z, nv * sizeof(double), false);
    alloc_into(ctx, s->v64.p, nv * sizeof(double), false);
    alloc_into(ctx, s->v64.q, nv * sizeof(double), false);
    alloc_into(ctx, s->v64.state, s->n_arrays * sizeof(PcgState));
    alloc_into(ctx, s->part, 3 * (size_t)s->n_vwork * sizeof(double));
    alloc_into(ctx, s->gpart, (size_t)std::max(1, s->n_grp) * sizeof(double));
    alloc_into(ctx, s->flag, 64);
    alloc_into(ctx, s->tickets, 2 * (size_t)s->n_arrays * sizeof(int));
    alloc_into(ctx, s->timers, 4 * sizeof(unsigned long long));
    alloc_into(ctx, s->barrier, 10 * 32 * sizeof(unsigned));
    const bool mixed = s->precision != MSTRESS_FP64;
    alloc_into(ctx, s->Y, (size_t)s->n_blocks * s->ldY * (mixed ? sizeof(float) : sizeof(double)), false);
    if (mixed) {
        for (int t = 0; t < s->n_types; ++t) {
            ensure_lowp(s->types[t], s->precision);
            s->tt.Klp[t] = s->use_tc ? s->types[t]->Kr_tc[s->precision].ptr : s->types[t]->Kr_lp[s->precision].ptr;
        }
        alloc_into(ctx, s->v32.x, nv * sizeof(float));
        alloc_into(ctx, s->v32.r, nv * sizeof(float), false);
        alloc_into(ctx, s->v32.z, nv * sizeof(float), false);
        alloc_into(ctx, s->v32.p, nv * sizeof(float), false);
        alloc_into(ctx, s->v32.q, nv * sizeof(float), false);
        alloc_into(ctx, s->v32.state, s->n_arrays * sizeof(PcgState));
        if (s->use_tc && (!tc_streamed(s->m) || pcg_wide(s, s->precision)))
            alloc_into(ctx, s->pz, nv * sizeof(float2), false);
    }
    if (s->inner64) {
        alloc_into(ctx, s->v64i.x, nv * sizeof(double));
        alloc_into(ctx, s->v64i.r, nv * sizeof(double), false);
        alloc_into(ctx, s->v64i.z, nv * sizeof(double), false);
        alloc_into(ctx, s->v64i.p, nv * sizeof(double), false);
        alloc_into(ctx, s->v64i.q, nv * sizeof(double), false);
        alloc_into(ctx, s->v64i.state, s->n_arrays * sizeof(PcgState));
    }
}

void check_device_error(mstress_sol_s* s) {
    MS_CUDA(cudaStreamSynchronize(s->ctx->stream));
    flush_inner_iters(s);
    int f[4];
    MS_CUDA(cudaMemcpy(f, s->flag.ptr, sizeof(f), cudaMemcpyDeviceToHost));
    MS_REQUIRE(f[2] == 0, MSTRESS_EDEVICE_TIMEOUT, "a tensor-core wait or a grid barrier timed out on the device");
}

// Rebuild the tensor-core tile list with tiles of `tile` blocks.
void set_tc_tiles(mstress_sol_s* s, int tile) {
    std::vector<ApplyWork> w;
    for (const ApplyWork& g : s->h_seg)
        for (int st = 0; st < g.count; st += tile)
            w.push_back(ApplyWork{g.type, g.array, g.start + st, std::min(tile, g.count - st), g.grp + st / 8});
    if (s->d_awork_tc.bytes < w.size() * sizeof(ApplyWork))
        alloc_into(s->ctx, s->d_awork_tc, w.size() * sizeof(ApplyWork), false);
    MS_CUDA(cudaMemcpyAsync(s->d_awork_tc.ptr, w.data(), w.size() * sizeof(ApplyWork), cudaMemcpyHostToDevice,
                            s->ctx->stream));
    s->n_awork_tc = (int)w.size();
    s->tc_tile = tile;
}

// Autotuner of the tensor-core tile (the MMA M extent actually filled, i.e.
// blocks per tile): for each candidate it runs a few iterations of the
// persistent solver on the solve's own right-hand side and reads the time of
// the element-product phase from the solver's device timers (or, when the
// solve will take the per-phase iteration, times the stand-alone apply kernel
// with CUDA events); the fastest is kept, and cached in the context per
// (basis size, precision, batch-size class) so later solves of that class
// skip the search. The trials leave nothing behind: every solve restarts its
// vectors and scalars.
void autotune_tc_tile(mstress_sol_s* s) {
    if (!s->use_tc || s->precision == MSTRESS_FP64 || s->h_seg.empty()) return;
    mstress_ctx ctx = s->ctx;
    if (s->n_blocks < 2LL * ctx->num_sms) return;   // at most a few blocks per SM: nothing to choose
    const int cls = 64 - __builtin_clzll((unsigned long long)s->n_blocks);
    const uint64_t key = ((uint64_t)s->m << 40) | ((uint64_t)s->precision << 32) | (uint64_t)cls;
    auto hit = ctx->tile_choice.find(key);
    s->tuned = true;
    if (hit != ctx->tile_choice.end()) {
        if (hit->second != s->tc_tile) set_tc_tiles(s, hit->second);
        return;
    }
    constexpr int kTrialIters = 6;
    const int h = s->tc_tile;
    std::vector<int> cand = {h, 32, 64, 128};
    for (int c : {(int)round_up(h / 2, 8), (int)round_up(h + h / 2, 8)}) cand.push_back(c);
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    cudaStream_t st = ctx->stream;
    int best = h;
    double best_ns = -1;
    if (pcg_wide(s, s->precision)) {   // the per-phase iteration's own apply kernel, timed alone
        pcg_start<float>(s, s->v32, s->b.as<double>(), 0.0, kTrialIters, nullptr);   // p = 0, z = D^-1 b
        cudaEvent_t e0, e1;
        MS_CUDA(cudaEventCreate(&e0));
        MS_CUDA(cudaEventCreate(&e1));
        for (int c : cand) {
            if (c < 8 || c > kTileTC) continue;
            set_tc_tiles(s, c);
            launch_apply_wide(s, s->precision, nullptr);   // warm-up
            MS_CUDA(cudaEventRecord(e0, st));
            for (int r = 0; r < 3; ++r) launch_apply_wide(s, s->precision, nullptr);
            MS_CUDA(cudaEventRecord(e1, st));
            MS_CUDA(cudaEventSynchronize(e1));
            float ms = 0;
            MS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (best_ns < 0 || ms < best_ns) {
                best_ns = ms;
                best = c;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        check_device_error(s);
        ctx->tile_choice[key] = best;
        if (best != s->tc_tile) set_tc_tiles(s, best);
        return;
    }
    for (int c : cand) {
        if (c < 8 || c > kTileTC) continue;
        set_tc_tiles(s, c);
        pcg_start<float>(s, s->v32, s->b.as<double>(), 0.0, kTrialIters, nullptr);
        MS_CUDA(cudaMemsetAsync(s->timers.ptr, 0, s->timers.bytes, st));
        if (!pcg_run_persistent(s, s->v32, s->precision, kTrialIters, true)) {
            best_ns = -1;   // no cooperative launch: keep the default tiles
            best = h;
            s->tuned = false;
            break;
        }
        unsigned long long t[4];
        MS_CUDA(cudaMemcpyAsync(t, s->timers.ptr, sizeof(t), cudaMemcpyDeviceToHost, st));
        MS_CUDA(cudaStreamSynchronize(st));
        const double ns = t[3] ? (double)t[0] / (double)t[3] : 0.0;
        if (best_ns < 0 || ns < best_ns) {
            best_ns = ns;
            best = c;
        }
    }
    check_device_error(s);
    MS_CUDA(cudaMemsetAsync(s->timers.ptr, 0, s->timers.bytes, st));
    ctx->tile_choice[key] = best;
    if (best != s->tc_tile) set_tc_tiles(s, best);
}

// a2: right-hand side and Jacobi diagonal, the FP64 element buffer of the
// mixed modes, and the lifting of prescribed values (Eq. 13).
void solve_prepare(mstress_sol_s* s) {
    mstress_ctx ctx = s->ctx;
    cudaStream_t stream = ctx->stream;
    RhsArgs ra;
    ra.vwork = s->d_vwork.as<VecWork>();
    ra.n_vwork = s->n_vwork;
    ra.arrays = s->d_arrays.as<ArrayDev>();
    ra.lm = s->d_lm.as<LocalMap>();
    ra.site = s->d_site.as<uint8_t>();
    ra.fixed = s->fixed.as<uint8_t>();
    ra.tt = s->tt;
    ra.m = s->m;
    ra.b = s->b.as<double>();
    ra.dinv = s->dinv.as<double>();
    k_rhs_diag<<<grid_for(s, s->n_vwork, 8), kThreads, 0, stream>>>(ra);
    MS_LAUNCH_CHECK();
    if (s->precision != MSTRESS_FP64) {
        alloc_into(ctx, s->dinv32, (size_t)s->n_vec * sizeof(float), false);
        k_narrow<<<(unsigned)((s->n_vec + 255) / 256), 256, 0, stream>>>(s->n_vec, s->dinv.as<double>(),
                                                                          s->dinv32.as<float>());
        MS_LAUNCH_CHECK();
        alloc_into(ctx, s->Y64own, (size_t)s->n_blocks * s->ldY * sizeof(double), false);
        s->Y64 = s->Y64own.ptr;
    } else {
        s->Y64 = s->Y.ptr;
    }
    if (s->xbc.ptr) {   // b -= A x_bc on the free DOFs
        launch_apply(s, MSTRESS_FP64, s->xbc.ptr, nullptr, false, nullptr, s->Y64);
        launch_isum(s, s->Y64, false, s->xbc.ptr, nullptr, s->v64.q.ptr, false, nullptr, nullptr, nullptr);
        k_lift_rhs<<<(unsigned)((s->n_vec + 255) / 256), 256, 0, stream>>>(s->n_vec, s->b.as<double>(),
                                                                            s->v64.q.as<double>(), s->dinv.as<double>());
        MS_LAUNCH_CHECK();
    }
    autotune_tc_tile(s);
}

// Outer (refinement) state from b: x = 0, ||b||, tolerance, step count 0.
void refine_start(mstress_sol_s* s) {
    const mstress_opts& o = s->ctx->opts;
    pcg_start<double>(s, s->v64, s->b.as<double>(), o.rtol, o.max_outer, nullptr);
}

// a5: FP64 residual and stopping test; true if any array takes another step.
bool refine_check(mstress_sol_s* s, bool x_zero) { return outer_check(s, s->Y64, s->ctx->opts.max_outer, x_zero); }

// Relative tolerance of an inner (reduced-precision) solve: the option, or,
// when it is 0, a per-precision value near the reduction one refinement step
// can deliver with that operator (measured on the 100x100 array: BF16X3 3e-4,
// TF32 1e-3 and BF16 3e-2 gave the shortest solves).
double inner_tolerance(const mstress_sol_s* s) {
    const double o = s->ctx->opts.inner_rtol;
    if (o > 0) return o;
    switch (s->precision) {
        case MSTRESS_TF32: return 1e-3;
        case MSTRESS_BF16: return 3e-2;
        default: return 3e-4;
    }
}

// One inner solve A d = r for every array still refining, in the inner
// precision (FP32 vectors with the reduced-precision operator, or FP64 for
// inner64), then x += d; inner iterations are added to the per-array counts.
void refine_inner(mstress_sol_s* s) {
    cudaStream_t stream = s->ctx->stream;
    const mstress_opts& o = s->ctx->opts;
    int used = 0;
    for (auto& r : s->results) used = std::max(used, r.iters);
    const int budget = std::max(1, o.max_iter - used);
    const PcgState* gate = s->v64.state.as<PcgState>();
    PcgVectors& vi = s->inner64 ? s->v64i : s->v32;
    if (s->inner64) {
        pcg_start<double>(s, vi, s->v64.r.as<double>(), inner_tolerance(s), budget, gate);
        pcg_run<double>(s, vi, MSTRESS_FP64, budget);
        k_correct<double><<<grid_for(s, s->n_vwork, 8), kThreads, 0, stream>>>(
            s->d_vwork.as<VecWork>(), s->n_vwork, gate, s->v64.x.as<double>(), vi.x.as<double>());
    } else {
        pcg_start<float>(s, vi, s->v64.r.as<double>(), inner_tolerance(s), budget, gate);
        pcg_run<float>(s, vi, s->precision, budget);
        k_correct<float><<<grid_for(s, s->n_vwork, 8), kThreads, 0, stream>>>(
            s->d_vwork.as<VecWork>(), s->n_vwork, gate, s->v64.x.as<double>(), vi.x.as<float>());
    }
    MS_LAUNCH_CHECK();
    // the iteration counts come back with the next synchronisation (flush_inner_iters)
    mstress_ctx ctx = s->ctx;
    const size_t bytes = (size_t)s->n_arrays * sizeof(PcgState);
    if (ctx->h_states_bytes < bytes) {
        if (ctx->h_states) MS_CUDA(cudaFreeHost(ctx->h_states));
        ctx->h_states = nullptr;
        ctx->h_states_bytes = 0;
        MS_CUDA(cudaHostAlloc(&ctx->h_states, bytes, cudaHostAllocDefault));
        ctx->h_states_bytes = bytes;
    }
    MS_CUDA(cudaMemcpyAsync(ctx->h_states, vi.state.ptr, bytes, cudaMemcpyDeviceToHost, stream));
    s->inner_pending = true;
}

void flush_inner_iters(mstress_sol_s* s) {
    if (!s->inner_pending) return;
    const PcgState* inner = static_cast<const PcgState*>(s->ctx->h_states);
    for (int a = 0; a < s->n_arrays; ++a) s->results[a].iters += inner[a].iters;
    s->inner_pending = false;
}

// True FP64 residual of the final iterate, per-array results, and the
// prescribed values added back to the solution. checked: the refinement loop
// ended with a check of the current iterate, whose FP64 residual ||b - A x||^2
// the outer state already holds (so it is not computed again).
void solve_finish(mstress_sol_s* s, bool refined, bool checked) {
    cudaStream_t stream = s->ctx->stream;
    check_device_error(s);
    std::vector<PcgState> before(s->n_arrays);
    MS_CUDA(cudaMemcpyAsync(before.data(), s->v64.state.ptr, before.size() * sizeof(PcgState), cudaMemcpyDeviceToHost,
                            stream));
    if (refined && checked) {
        MS_CUDA(cudaStreamSynchronize(stream));
        for (int a = 0; a < s->n_arrays; ++a) {
            ArrayResult& R = s->results[a];
            R.rel_res = before[a].bb > 0 ? std::sqrt(before[a].rr / before[a].bb) : 0.0;
            R.outer = before[a].iters;
            R.status = before[a].status;
            if (!std::isfinite(R.rel_res)) R.status = MSTRESS_ENUMERIC;
        }
        if (s->xbc.ptr) {
            k_add_bc<<<(unsigned)((s->n_vec + 255) / 256), 256, 0, stream>>>(s->n_vec, s->v64.x.as<double>(),
                                                                              s->xbc.as<double>());
            MS_LAUNCH_CHECK();
            MS_CUDA(cudaStreamSynchronize(stream));
        }
        return;
    }
    launch_apply(s, MSTRESS_FP64, s->v64.x.ptr, nullptr, false, nullptr, s->Y64);
    launch_isum(s, s->Y64, false, s->v64.x.ptr, nullptr, s->v64.q.ptr, false, s->dinv.as<double>(), nullptr, nullptr);
    VecArgs va = vec_args(s, s->v64);
    va.rhs = s->b.ptr;
    va.r = s->v64.z.ptr;   // residual into z (scratch) so r keeps the recursive residual
    k_residual<<<grid_for(s, s->n_vwork, 8), kThreads, 0, stream>>>(va);
    MS_LAUNCH_CHECK();
    std::vector<double> prr(s->n_vwork);
    MS_CUDA(cudaMemcpyAsync(prr.data(), va.part_rr, prr.size() * sizeof(double), cudaMemcpyDeviceToHost, stream));
    MS_CUDA(cudaStreamSynchronize(stream));
    for (int a = 0; a < s->n_arrays; ++a) {
        const ArrayDev& A = s->arrays[a];
        double rr = 0;
        for (int w = 0; w < A.n_vwork; ++w) rr += prr[A.vwork_off + w];
        ArrayResult& R = s->results[a];
        R.rel_res = before[a].bb > 0 ? std::sqrt(rr / before[a].bb) : 0.0;
        if (refined) R.outer = before[a].iters;
        else R.iters = before[a].iters;
        R.status = before[a].status;
        if (!std::isfinite(R.rel_res)) R.status = MSTRESS_ENUMERIC;
    }
    if (s->xbc.ptr) {
        k_add_bc<<<(unsigned)((s->n_vec + 255) / 256), 256, 0, stream>>>(s->n_vec, s->v64.x.as<double>(),
                                                                          s->xbc.as<double>());
        MS_LAUNCH_CHECK();
    }
    MS_CUDA(cudaStreamSynchronize(stream));
}

namespace {

void run_solve(mstress_sol_s* s) {
    const mstress_opts& o = s->ctx->opts;
    solve_prepare(s);
    if (s->precision == MSTRESS_FP64) {
        pcg_start<double>(s, s->v64, s->b.as<double>(), o.rtol, o.max_iter, nullptr);
        pcg_run<double>(s, s->v64, MSTRESS_FP64, o.max_iter);
        solve_finish(s, false, false);
        return;
    }
    refine_start(s);
    bool checked = false;
    for (int k = 0; k <= o.max_outer; ++k) {
        if (!refine_check(s, k == 0)) {
            checked = true;
            break;
        }
        refine_inner(s);
    }
    solve_finish(s, true, checked);
}

int solve_common(mstress_ctx ctx, const std::vector<LayoutIn>& in, mstress_sol* out) {
    std::unique_ptr<mstress_sol_s> s(new mstress_sol_s());
    s->ctx = ctx;
    s->precision = ctx->opts.precision;
    validate_and_build(s.get(), in);
    s->results.assign(s->n_arrays, ArrayResult{});
    run_solve(s.get());
    int status = MSTRESS_OK;
    for (auto& r : s->results)
        if (r.status != MSTRESS_OK) status = r.status;
    *out = s.release();
    if (status == MSTRESS_ENOT_CONVERGED) ctx->last_error = "PCG iteration limit reached";
    if (status == MSTRESS_ENUMERIC) ctx->last_error = "PCG breakdown (non-positive curvature or NaN)";
    return status;
}

}  // namespace
}  // namespace ms

mstress_sol_s::~mstress_sol_s() {
    for (auto& g : graph)
        if (g) cudaGraphExecDestroy(g);
}

using namespace ms;

#define MS_API_BEGIN try {
#define MS_API_END(ctx)                          \
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

int mstress_solve(mstress_ctx ctx, const mstress_layout* layout, double dT, const mstress_bc* bc, mstress_sol* out) {
    if (!ctx) return MSTRESS_EINVAL;
    if (!out) { ctx->last_error = "out is NULL"; return MSTRESS_EINVAL; }
    *out = nullptr;
    MS_API_BEGIN
    std::vector<LayoutIn> in{LayoutIn{layout, dT, bc}};
    return solve_common(ctx, in, out);
    MS_API_END(ctx)
}

int mstress_solve_batch(mstress_ctx ctx, const mstress_layout* layouts, const double* dT, const mstress_bc* bcs,
                        int n, mstress_sol* out) {
    if (!ctx) return MSTRESS_EINVAL;
    if (!out) { ctx->last_error = "out is NULL"; return MSTRESS_EINVAL; }
    *out = nullptr;
    MS_API_BEGIN
    MS_REQUIRE(layouts && dT && n >= 1, MSTRESS_EINVAL, "need n >= 1 layouts and dT values");
    std::vector<LayoutIn> in;
    for (int k = 0; k < n; ++k) in.push_back(LayoutIn{&layouts[k], dT[k], bcs ? &bcs[k] : nullptr});
    return solve_common(ctx, in, out);
    MS_API_END(ctx)
}

int mstress_sol_info(mstress_sol sol, int array, int* iters, int* outer, double* rel_res, int* status) {
    if (!sol || array < 0 || array >= sol->n_arrays) return MSTRESS_EINVAL;
    const ArrayResult& r = sol->results[array];
    if (iters) *iters = r.iters;
    if (outer) *outer = r.outer;
    if (rel_res) *rel_res = r.rel_res;
    if (status) *status = r.status;
    return MSTRESS_OK;
}

int mstress_set_wait_limit(mstress_ctx ctx, int64_t limit_ns, int withhold_next) {
    if (!ctx) return MSTRESS_EINVAL;
    if (limit_ns <= 0) {
        ctx->last_error = "the wait limit must be positive";
        return MSTRESS_EINVAL;
    }
    ctx->wait_limit_ns = limit_ns;
    ctx->withhold_next = withhold_next ? 1 : 0;
    return MSTRESS_OK;
}

int mstress_sol_tiling(mstress_sol sol, int* use_tc, int* tc_tile, int* tuned) {
    if (!sol) return MSTRESS_EINVAL;
    if (use_tc) *use_tc = sol->use_tc ? 1 : 0;
    if (tc_tile) *tc_tile = sol->use_tc ? sol->tc_tile : 0;
    if (tuned) *tuned = sol->tuned ? 1 : 0;
    return MSTRESS_OK;
}

int mstress_sol_count(mstress_sol sol, int* n_arrays, int64_t* n_blocks) {
    if (!sol) return MSTRESS_EINVAL;
    if (n_arrays) *n_arrays = sol->n_arrays;
    if (n_blocks) *n_blocks = sol->n_blocks;
    return MSTRESS_OK;
}

void mstress_free_sol(mstress_sol sol) {
    if (!sol) return;
    cudaStreamSynchronize(sol->ctx->stream);
    delete sol;
}

int mstress_apply(mstress_ctx ctx, const mstress_layout* layout, const double* x_dev, double* y_dev, int precision) {
    if (!ctx) return MSTRESS_EINVAL;
    MS_API_BEGIN
    MS_REQUIRE(x_dev && y_dev, MSTRESS_EINVAL, "x and y are required");
    MS_REQUIRE(precision >= MSTRESS_FP64 && precision <= MSTRESS_BF16X3, MSTRESS_EINVAL, "unknown precision");
    std::unique_ptr<mstress_sol_s> s(new mstress_sol_s());
    s->ctx = ctx;
    s->precision = precision;
    mstress_bc bc{1, 0, nullptr, nullptr, 0};
    std::vector<LayoutIn> in{LayoutIn{layout, 0.0, &bc}};
    validate_and_build(s.get(), in);
    cudaStream_t st = ctx->stream;
    if (precision == MSTRESS_FP64) {
        launch_apply(s.get(), MSTRESS_FP64, x_dev, nullptr, false, nullptr, s->Y.ptr);
        launch_isum(s.get(), s->Y.ptr, false, const_cast<double*>(x_dev), nullptr, y_dev, false, nullptr, nullptr,
                    nullptr);
    } else {   // x rounded to FP32, the inner solver's operator, y widened
        const unsigned g = (unsigned)((s->n_vec + 255) / 256);
        k_narrow<<<g, 256, 0, st>>>(s->n_vec, x_dev, s->v32.x.as<float>());
        MS_LAUNCH_CHECK();
        launch_apply(s.get(), precision, s->v32.x.ptr, nullptr, true, nullptr, s->Y.ptr);
        launch_isum(s.get(), s->Y.ptr, true, s->v32.x.ptr, nullptr, s->v32.q.ptr, true, nullptr, nullptr, nullptr);
        k_widen<<<g, 256, 0, st>>>(s->n_vec, s->v32.q.as<float>(), y_dev);
        MS_LAUNCH_CHECK();
    }
    MS_CUDA(cudaStreamSynchronize(st));
    MS_API_END(ctx)
}

int mstress_profile(mstress_ctx ctx, mstress_sol sol, int phase, int reps, double* avg_ms) {
    if (!ctx) return MSTRESS_EINVAL;
    MS_API_BEGIN
    MS_REQUIRE(sol && sol->ctx == ctx && avg_ms && reps >= 1, MSTRESS_EINVAL, "bad profile arguments");
    mstress_sol_s* s = sol;
    cudaStream_t st = ctx->stream;
    const bool mixed = s->precision != MSTRESS_FP64;
    DBuf y64, out;
    if (phase == 2 && mixed) alloc_into(ctx, y64, (size_t)s->n_blocks * s->ldY * sizeof(double), false);
    if (phase == 3) alloc_into(ctx, out, recover_bytes(s, MSTRESS_VM_ELEM), false);
    auto run = [&]() {
        switch (phase) {
            case 0:   // gathering p and z as an iteration does (p = z + beta p, beta = 0 here)
                if (mixed && pcg_wide(s, s->precision)) launch_apply_wide(s, s->precision, nullptr);
                else if (mixed) launch_apply(s, s->precision, s->v32.p.ptr, s->v32.z.ptr, true, nullptr, s->Y.ptr);
                else launch_apply(s, MSTRESS_FP64, s->v64.p.ptr, s->v64.z.ptr, false, nullptr, s->Y.ptr);
                break;
            case 1:
                if (mixed) launch_isum(s, s->Y.ptr, true, s->v32.p.ptr, nullptr, s->v32.q.ptr, true, s->dinv32.ptr,
                                       nullptr, s->part.as<double>());
                else launch_isum(s, s->Y.ptr, false, s->v64.p.ptr, nullptr, s->v64.q.ptr, false, s->dinv.as<double>(),
                                 nullptr, s->part.as<double>());
                break;
            case 2:
                launch_apply(s, MSTRESS_FP64, s->v64.x.ptr, nullptr, false, nullptr, mixed ? y64.ptr : s->Y.ptr);
                break;
            case 3:
                recover(s, MSTRESS_VM_ELEM, out.ptr, true);
                break;
            default: throw Error{MSTRESS_EINVAL, "unknown phase"};
        }
    };
    run();   // warm-up (and the one-time set-up of reduced-precision operands)
    MS_CUDA(cudaStreamSynchronize(st));
    cudaEvent_t e0, e1;
    MS_CUDA(cudaEventCreate(&e0));
    MS_CUDA(cudaEventCreate(&e1));
    MS_CUDA(cudaEventRecord(e0, st));
    for (int k = 0; k < reps; ++k) run();
    MS_CUDA(cudaEventRecord(e1, st));
    MS_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    MS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *avg_ms = ms / reps;
    check_device_error(s);
    MS_API_END(ctx)
}

int mstress_sol_phase_ms(mstress_sol sol, double* ms4) {
    if (!sol || !ms4) return MSTRESS_EINVAL;
    MS_API_BEGIN
    unsigned long long t[4] = {0, 0, 0, 0};
    MS_CUDA(cudaMemcpy(t, sol->timers.ptr, sizeof(t), cudaMemcpyDeviceToHost));
    for (int k = 0; k < 3; ++k) ms4[k] = t[k] * 1e-6;
    ms4[3] = (double)t[3];
    MS_API_END(sol->ctx)
}

int mstress_recover_size(mstress_sol sol, int what, size_t* bytes) {
    if (!sol || !bytes) return MSTRESS_EINVAL;
    MS_API_BEGIN
    *bytes = recover_bytes(sol, what);
    MS_API_END(sol->ctx)
}

int mstress_recover(mstress_ctx ctx, mstress_sol sol, int what, void* dst, size_t dst_bytes, int dst_on_device) {
    if (!ctx) return MSTRESS_EINVAL;
    MS_API_BEGIN
    MS_REQUIRE(sol && sol->ctx == ctx, MSTRESS_EINVAL, "solution is NULL or from another context");
    MS_REQUIRE(dst, MSTRESS_EINVAL, "dst is NULL");
    size_t need = recover_bytes(sol, what);
    MS_REQUIRE(dst_bytes >= need, MSTRESS_EINVAL, "dst too small: need " + std::to_string(need) + " B");
    recover(sol, what, dst, dst_on_device != 0);
    MS_API_END(ctx)
}

}  // extern "C"
