// Field recovery of MORE-Stress (section 4.3, last paragraph; Eq. 15 and
// Eq. 1): for every block e of type t, Sigma_e = M_t [c_e; dT], where c_e are
// the block's element DOFs gathered from the solved lattice vector and M_t is
// one of the block's mode matrices:
//   S     stress modes at the 8 Gauss points of every element (48 rows each),
//   Smean their Gauss mean (6 rows per element),
//   F     the local basis itself (fine nodal displacement, Eq. 15).
// The per-element von Mises output uses Smean: von Mises of the Gauss-mean
// stress, fused into the contraction's epilogue so no stress tensor is
// written. The mean over Gauss points is linear, so Smean [c; dT] is exactly
// the mean of the Gauss-point stresses S [c; dT].
#include <cmath>
#include <type_traits>

#include "solve.h"

namespace ms {
namespace {

constexpr int kRowTile = 192;   // 32 threads x 6 rows
constexpr int kKC = 32;         // reduction chunk

struct RecArgs {
    const ApplyWork* work;      // block tiles (one type, one array, <= 32 blocks)
    int n_work, n_rtiles;
    const int* blist;
    const BlockRef* bref;
    const ArrayDev* arrays;
    const LocalMap* lm;
    const void* rows[kMaxTypes];   // mode matrix per type, row stride ld (plane stride for X3)
    int m, m1, ld, n_rows, n_el;
    long long plane;               // element offset of the lo plane (BF16X3)
    const double* x;               // FP64 lattice solution
    void* out;
    long long out_ld;              // output elements per block
    int vm;                        // 1: von Mises epilogue (rows = 6 per element)
};

__device__ __forceinline__ float rnd_tf32(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}
__device__ __forceinline__ float rnd_bf16(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

template <class T>
__device__ __forceinline__ T von_mises(const T* s) {
    T a = s[0] - s[1], b = s[1] - s[2], c = s[2] - s[0];
    return sqrt(T(0.5) * (a * a + b * b + c * c) + T(3) * (s[3] * s[3] + s[4] * s[4] + s[5] * s[5]));
}

// MODE = MSTRESS_FP64: FP64 everywhere. Otherwise FP32 accumulation with
// operands in the mode's format: rows are pre-rounded (float storage), the
// gathered coefficients are rounded here; BF16X3 uses hi/lo planes and the
// three products hi*hi + hi*lo + lo*hi.
template <int MODE>
__global__ void __launch_bounds__(256) k_recover(const __grid_constant__ RecArgs a) {
    using T = typename std::conditional<MODE == MSTRESS_FP64, double, float>::type;
    constexpr int NS = MODE == MSTRESS_BF16X3 ? 2 : 1;
    extern __shared__ unsigned char smraw[];
    T* Cs = reinterpret_cast<T*>(smraw);                           // [NS][m1][32]
    T* Ms = Cs + (size_t)NS * a.m1 * kTile64;                       // [NS][kRowTile][kKC+1]
    __shared__ long long base[kTile64];
    __shared__ int offs[3 * kMaxSurf];
    const int tid = threadIdx.x;
    const int el = tid & 31, bg = tid >> 5;
    for (int w = blockIdx.x; w < a.n_work * a.n_rtiles; w += gridDim.x) {
        const ApplyWork it = a.work[w / a.n_rtiles];
        const int r0 = (w % a.n_rtiles) * kRowTile;
        const ArrayDev A = a.arrays[it.array];
        const int n1 = a.lm->n - 1;
        __syncthreads();
        for (int k = tid; k < a.m; k += 256) {
            int q = k / 3, c = k - 3 * q;
            offs[k] = ((a.lm->qc[q] * A.Y + a.lm->qb[q]) * A.X + a.lm->qa[q]) * 3 + c;
        }
        if (tid < kTile64 && tid < it.count) {
            BlockRef br = a.bref[a.blist[it.start + tid]];
            base[tid] = A.vec_off + 3LL * ((long long)br.j * n1 * A.X + (long long)br.i * n1);
        }
        __syncthreads();
        for (int idx = tid; idx < a.m1 * kTile64; idx += 256) {
            int k = idx >> 5, bt = idx & 31;
            double v = 0;
            if (bt < it.count) v = k < a.m ? a.x[base[bt] + offs[k]] : A.dT;
            if (MODE == MSTRESS_FP64) Cs[idx] = (T)v;
            else if (MODE == MSTRESS_TF32) Cs[idx] = rnd_tf32((float)v);
            else if (MODE == MSTRESS_BF16) Cs[idx] = rnd_bf16((float)v);
            else {
                float hi = rnd_bf16((float)v);
                Cs[idx] = hi;
                Cs[(size_t)a.m1 * kTile64 + idx] = rnd_bf16((float)(v - (double)hi));
            }
        }
        const T* __restrict__ M = static_cast<const T*>(a.rows[it.type]);
        T acc[6][4];
#pragma unroll
        for (int c = 0; c < 6; ++c)
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[c][u] = 0;
        for (int k0 = 0; k0 < a.m1; k0 += kKC) {
            __syncthreads();
            for (int s = 0; s < NS; ++s)
                for (int idx = tid; idx < kRowTile * kKC; idx += 256) {
                    int r = idx / kKC, kk = idx % kKC;
                    int row = r0 + r, k = k0 + kk;
                    T v = 0;
                    if (row < a.n_rows && k < a.m1) v = M[s * a.plane + (size_t)row * a.ld + k];
                    Ms[((size_t)s * kRowTile + r) * (kKC + 1) + kk] = v;
                }
            __syncthreads();
            const int kmax = min(kKC, a.m1 - k0);
            for (int kk = 0; kk < kmax; ++kk) {
                T sv[6], cv[4];
#pragma unroll
                for (int c = 0; c < 6; ++c) sv[c] = Ms[(6 * el + c) * (kKC + 1) + kk];
#pragma unroll
                for (int u = 0; u < 4; ++u) cv[u] = Cs[(k0 + kk) * kTile64 + bg * 4 + u];
#pragma unroll
                for (int c = 0; c < 6; ++c)
#pragma unroll
                    for (int u = 0; u < 4; ++u) acc[c][u] = fma(sv[c], cv[u], acc[c][u]);
                if (NS == 2) {
                    T sl[6], cl[4];
#pragma unroll
                    for (int c = 0; c < 6; ++c) sl[c] = Ms[((size_t)kRowTile + 6 * el + c) * (kKC + 1) + kk];
#pragma unroll
                    for (int u = 0; u < 4; ++u) cl[u] = Cs[(size_t)a.m1 * kTile64 + (k0 + kk) * kTile64 + bg * 4 + u];
#pragma unroll
                    for (int c = 0; c < 6; ++c)
#pragma unroll
                        for (int u = 0; u < 4; ++u) acc[c][u] = fma(sv[c], cl[u], fma(sl[c], cv[u], acc[c][u]));
                }
            }
        }
        // epilogue
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int bt = bg * 4 + u;
            if (bt >= it.count) continue;
            const long long e = a.blist[it.start + bt];
            if (a.vm) {
                const int elem = r0 / 6 + el;
                if (elem < a.n_el) {
                    T s6[6] = {acc[0][u], acc[1][u], acc[2][u], acc[3][u], acc[4][u], acc[5][u]};
                    static_cast<T*>(a.out)[e * a.out_ld + elem] = von_mises(s6);
                }
            } else {
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    const int row = r0 + 6 * el + c;
                    if (row < a.n_rows) static_cast<T*>(a.out)[e * a.out_ld + row] = acc[c][u];
                }
            }
        }
    }
}

// Element DOFs of every block, c_e = G_e x (FP64), [block][m].
__global__ void k_coeff(long long n_blocks, const BlockRef* bref, const ArrayDev* arrays, const LocalMap* lm, int m,
                        const double* x, double* out) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= n_blocks * m) return;
    long long e = t / m;
    int k = (int)(t - e * m);
    BlockRef br = bref[e];
    ArrayDev A = arrays[br.array];
    int n1 = lm->n - 1, q = k / 3, c = k - 3 * q;
    long long g = A.vec_off + 3LL * ((long long)(br.j * n1 + lm->qb[q] + (long long)lm->qc[q] * A.Y) * A.X +
                                     br.i * n1 + lm->qa[q]) + c;
    out[t] = x[g];
}

// Round FP64 rows to a tensor-core operand format, stored as float.
__global__ void k_round_rows(long long rows, int cols, int ld_src, int ld_dst, const double* src, float* dst,
                             long long plane, int mode) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= rows * ld_dst) return;
    long long r = t / ld_dst;
    int c = (int)(t - r * ld_dst);
    double v = c < cols ? src[r * ld_src + c] : 0.0;
    float f = (float)v;
    if (mode == MSTRESS_TF32) dst[t] = rnd_tf32(f);
    else if (mode == MSTRESS_BF16) dst[t] = rnd_bf16(f);
    else {
        float hi = rnd_bf16(f);
        dst[t] = hi;
        dst[plane + t] = rnd_bf16((float)(v - (double)hi));
    }
}

void round_rows(mstress_ctx ctx, DBuf& dst, const double* src, long long rows, int cols, int ld, int mode) {
    const int ns = mode == MSTRESS_BF16X3 ? 2 : 1;
    const long long plane = rows * ld;
    alloc_into(ctx, dst, (size_t)ns * plane * sizeof(float), false);
    long long n = rows * ld;
    k_round_rows<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(rows, cols, ld, ld, src, dst.as<float>(),
                                                                        plane, mode);
    MS_LAUNCH_CHECK();
}

}  // namespace

void ensure_lowp(mstress_block blk, int precision) {
    if (precision == MSTRESS_FP64) return;
    mstress_ctx ctx = blk->ctx;
    if (!blk->Kr_lp[precision].ptr) round_rows(ctx, blk->Kr_lp[precision], blk->Kr.as<double>(), blk->m, blk->m, blk->m, precision);
    if (tc_supported(blk->m)) build_tc_operator(blk, precision);
    if (!blk->Smean_lp[precision].ptr)
        round_rows(ctx, blk->Smean_lp[precision], blk->Smean.as<double>(), (long long)6 * blk->n_el, blk->m1, blk->ld,
                   precision);
}

static void ensure_grid_lowp(mstress_block blk, int precision) {
    if (!blk->Sgrid_lp[precision].ptr)
        round_rows(blk->ctx, blk->Sgrid_lp[precision], blk->Sgrid.as<double>(), (long long)6 * blk->n_grid, blk->m1,
                   blk->ld, precision);
}

// Grid points per block of a solution's gridded output (every block model of
// the solve must carry the same grid).
static int grid_points(const mstress_sol_s* s) {
    const int side = s->types[0]->grid_side;
    MS_REQUIRE(side > 0, MSTRESS_EINVAL, "no grid modes: call mstress_block_grid on the solution's block models");
    for (auto b : s->types)
        MS_REQUIRE(b->grid_side == side, MSTRESS_EINVAL, "the block models of a solve carry different grids");
    return side * side;
}

static void ensure_S_lowp(mstress_block blk, int precision) {
    if (!blk->S_lp[precision].ptr)
        round_rows(blk->ctx, blk->S_lp[precision], blk->S.as<double>(), (long long)48 * blk->n_el, blk->m1, blk->ld,
                   precision);
}

size_t recover_bytes(const mstress_sol_s* s, int what) {
    const size_t w = s->precision == MSTRESS_FP64 ? sizeof(double) : sizeof(float);
    switch (what) {
        case MSTRESS_COEFF: return (size_t)s->n_blocks * s->m * sizeof(double);
        case MSTRESS_VM_ELEM: return (size_t)s->n_blocks * s->n_el * w;
        case MSTRESS_SIGMA_GP: return (size_t)s->n_blocks * s->n_el * 48 * w;
        case MSTRESS_U_NODE: return (size_t)s->n_blocks * s->n_dof_block * sizeof(double);
        case MSTRESS_LATTICE: return (size_t)s->n_vec * sizeof(double);
        case MSTRESS_VM_GRID: return (size_t)s->n_blocks * grid_points(s) * w;
        default: throw Error{MSTRESS_EINVAL, "unknown recovery output"};
    }
}

void recover_arrays(mstress_sol_s* s, int what, void* dst_dev, const std::vector<int>& arrays) {
    std::vector<char> want(s->n_arrays, 0);
    for (int a : arrays) want[a] = 1;
    std::vector<ApplyWork> w, wr;
    for (auto& it : s->h_awork)
        if (want[it.array]) w.push_back(it);
    for (auto& it : s->h_awork_rec)
        if (want[it.array]) wr.push_back(it);
    if (w.empty()) return;
    DBuf dw, dwr;
    alloc_into(s->ctx, dw, w.size() * sizeof(ApplyWork), false);
    alloc_into(s->ctx, dwr, std::max<size_t>(1, wr.size()) * sizeof(ApplyWork), false);
    MS_CUDA(cudaMemcpyAsync(dw.ptr, w.data(), w.size() * sizeof(ApplyWork), cudaMemcpyHostToDevice, s->ctx->stream));
    if (!wr.empty())
        MS_CUDA(cudaMemcpyAsync(dwr.ptr, wr.data(), wr.size() * sizeof(ApplyWork), cudaMemcpyHostToDevice,
                                s->ctx->stream));
    // run the ordinary recovery over the filtered tile lists
    std::swap(s->d_awork, dw);
    std::swap(s->d_awork_rec, dwr);
    const int n0 = s->n_awork, n1 = s->n_awork_rec;
    s->n_awork = (int)w.size();
    s->n_awork_rec = (int)wr.size();
    try {
        recover(s, what, dst_dev, true);
    } catch (...) {
        std::swap(s->d_awork, dw);
        std::swap(s->d_awork_rec, dwr);
        s->n_awork = n0;
        s->n_awork_rec = n1;
        throw;
    }
    MS_CUDA(cudaStreamSynchronize(s->ctx->stream));
    std::swap(s->d_awork, dw);
    std::swap(s->d_awork_rec, dwr);
    s->n_awork = n0;
    s->n_awork_rec = n1;
}

void recover(mstress_sol_s* s, int what, void* dst, bool dst_dev) {
    mstress_ctx ctx = s->ctx;
    cudaStream_t st = ctx->stream;
    const size_t bytes = recover_bytes(s, what);
    DBuf tmp;
    void* out = dst;
    if (!dst_dev) {
        alloc_into(ctx, tmp, bytes, false);
        out = tmp.ptr;
    }
    if (what == MSTRESS_LATTICE) {
        MS_CUDA(cudaMemcpyAsync(out, s->v64.x.ptr, bytes, cudaMemcpyDeviceToDevice, st));
    } else if ((what == MSTRESS_VM_ELEM || what == MSTRESS_VM_GRID) && s->precision != MSTRESS_FP64 &&
               tc_recover_supported(s->types[0]->m1, s->precision)) {
        recover_vm_tc(s, static_cast<float*>(out), what == MSTRESS_VM_GRID);
    } else if (what == MSTRESS_COEFF) {
        long long n = s->n_blocks * s->m;
        k_coeff<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s->n_blocks, s->d_bref.as<BlockRef>(),
                                                              s->d_arrays.as<ArrayDev>(), s->d_lm.as<LocalMap>(), s->m,
                                                              s->v64.x.as<double>(), static_cast<double*>(out));
        MS_LAUNCH_CHECK();
    } else {
        int mode = s->precision;
        if (what == MSTRESS_U_NODE) mode = MSTRESS_FP64;
        RecArgs a;
        std::memset(&a, 0, sizeof(a));
        a.work = s->d_awork.as<ApplyWork>();
        a.n_work = s->n_awork;
        a.blist = s->d_blist.as<int>();
        a.bref = s->d_bref.as<BlockRef>();
        a.arrays = s->d_arrays.as<ArrayDev>();
        a.lm = s->d_lm.as<LocalMap>();
        a.m = s->m;
        mstress_block t0 = s->types[0];
        a.m1 = t0->m1;
        a.ld = t0->ld;
        const bool grid = what == MSTRESS_VM_GRID;
        a.n_el = grid ? grid_points(s) : s->n_el;
        a.x = s->v64.x.as<double>();
        a.out = out;
        a.vm = what == MSTRESS_VM_ELEM || grid;
        if (a.vm) a.n_rows = 6 * a.n_el;
        else if (what == MSTRESS_SIGMA_GP) a.n_rows = 48 * s->n_el;
        else a.n_rows = s->n_dof_block;
        a.out_ld = a.vm ? a.n_el : a.n_rows;
        a.plane = (long long)a.n_rows * a.ld;
        for (int t = 0; t < s->n_types; ++t) {
            mstress_block b = s->types[t];
            if (what == MSTRESS_U_NODE) {
                MS_REQUIRE(b->has_F, MSTRESS_EINVAL, "a block model holds no basis F (imported without it)");
                a.rows[t] = b->F.ptr;
            } else if (grid && mode == MSTRESS_FP64) {
                a.rows[t] = b->Sgrid.ptr;
            } else if (grid) {
                ensure_grid_lowp(b, mode);
                a.rows[t] = b->Sgrid_lp[mode].ptr;
            } else if (mode == MSTRESS_FP64) {
                a.rows[t] = what == MSTRESS_VM_ELEM ? b->Smean.ptr : b->S.ptr;
            } else if (what == MSTRESS_VM_ELEM) {
                ensure_lowp(b, mode);
                a.rows[t] = b->Smean_lp[mode].ptr;
            } else {
                ensure_S_lowp(b, mode);
                a.rows[t] = b->S_lp[mode].ptr;
            }
        }
        a.n_rtiles = (a.n_rows + kRowTile - 1) / kRowTile;
        const int ns = mode == MSTRESS_BF16X3 ? 2 : 1;
        const size_t esz = mode == MSTRESS_FP64 ? sizeof(double) : sizeof(float);
        const size_t smem = (size_t)ns * ((size_t)a.m1 * kTile64 + (size_t)kRowTile * (kKC + 1)) * esz;
        const long long items = (long long)a.n_work * a.n_rtiles;
        auto launch = [&](auto kern) {
            MS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            int per_sm = smem > 110 * 1024 ? 1 : (smem > 70 * 1024 ? 2 : 3);
            long long g = std::min<long long>(items, (long long)ctx->num_sms * per_sm);
            kern<<<(unsigned)std::max<long long>(1, g), 256, smem, st>>>(a);
            MS_LAUNCH_CHECK();
        };
        switch (mode) {
            case MSTRESS_FP64: launch(k_recover<MSTRESS_FP64>); break;
            case MSTRESS_TF32: launch(k_recover<MSTRESS_TF32>); break;
            case MSTRESS_BF16: launch(k_recover<MSTRESS_BF16>); break;
            default: launch(k_recover<MSTRESS_BF16X3>); break;
        }
    }
    if (!dst_dev) {   // host destination: copy back and wait; device destination stays asynchronous
        MS_CUDA(cudaMemcpyAsync(dst, out, bytes, cudaMemcpyDeviceToHost, st));
        MS_CUDA(cudaStreamSynchronize(st));
    }
}

}  // namespace ms
