// The resident solution of a (batched) global-stage solve and the device
// helpers shared by the solve, tensor-core and recovery units.
#pragma once

#include "internal.h"

namespace ms {

// Lattice DOFs per vector work item, matched to the solver CTA that runs the
// vector phases: 2048 for 256-thread CTAs (FP64: 2 rounds of 4 per thread),
// 2560 for the resident tensor-core solver (512 threads x 5: one round, and
// one item per SM at 100x100), 4096 for the streamed tensor-core solver (512
// threads x 8). The chunking is a function of the array, the precision and
// the basis size only, never of the batch.
constexpr int kVecChunk64 = 2048;
constexpr int kVecChunkTC = 2560;
constexpr int kVecChunk32 = 4096;
constexpr int kTile64 = 32;       // blocks per CUDA-core apply / recovery tile

// Rows per panel of the CUDA-core apply (8 x RPT): 32-row panels (RPT = 4)
// for mid-size bases, 16-row panels (RPT = 2) for small ones and for bases
// whose 32-row panel would not fit in shared memory next to the coefficient
// tile (bytes = (m x 32 + rows x m) x element size, at most 200 KB).
inline int apply_rpt(int m, int elem_bytes, int planes) {
    if (m <= 80) return 2;
    const long long need = (long long)planes * (m * 32LL + 32LL * m) * elem_bytes;
    return need <= 200 * 1024 - 1024 ? 4 : 2;
}
constexpr int kTileTC = 128;      // blocks per tensor-core apply tile (the MMA M dimension)

struct ArrayResult {
    int iters = 0, outer = 0, status = MSTRESS_OK;
    double rel_res = 0;
};

// Per-solve device vectors for one conjugate-gradient precision.
struct PcgVectors {
    DBuf x, r, z, p, q;   // packed lattice vectors of element type V
    DBuf state;           // PcgState per array
};

// Arguments of the element-product (operator apply) kernels.
struct ApplyArgs {
    const ApplyWork* work;
    int n_work;
    const int* blist;
    const BlockRef* bref;
    const ArrayDev* arrays;
    const LocalMap* lm;
    const PcgState* st;    // optional: skip stopped arrays; beta of the fused p update
    TypeTab tt;
    int m, ldY;
    const void* x;         // vector gathered (p, or x for a plain product)
    const void* z;         // optional: gather z + beta x instead of x
    void* Y;               // element products [block][ldY]
    int* err;              // device error word (bounded waits)
    double* gpart;         // optional: per 8-block group sums of p_e^T Y_e (tensor-core apply)
    const float2* pz;      // optional: gather p = z + beta p from (p, z) pairs instead of x and z
};

// The search-direction update p = z + beta p in the vector precision (one
// fused multiply-add), written once so that the gather of the apply and the
// interface sum compute identical bits.
template <class V>
__device__ __forceinline__ V p_next(V z, V p, V beta) {
    return fma(beta, p, z);
}

// Dot-product accumulators. FP64 vectors: a double. FP32 vectors: a
// double-FP32 pair (hi + lo) built from error-free transformations on the
// FP32 pipe (the exact product by fma, the exact sum by TwoSum), about 48
// significant bits, so the inner PCG's dot products keep FP64-level accuracy
// without the GPU's narrow FP64 pipe; the pairs are folded in FP64 across
// warps and work items.
template <class V>
struct DotAcc;

template <>
struct DotAcc<double> {
    double s = 0;
    __device__ __forceinline__ void add(double x, double y) { s = fma(x, y, s); }
};

template <>
struct DotAcc<float> {
    float hi = 0, lo = 0;
    // (the _rn intrinsics are never contracted into fused operations)
    __device__ __forceinline__ static void two_sum(float a, float b, float& sum, float& err) {
        sum = __fadd_rn(a, b);
        const float bb = __fsub_rn(sum, a);
        err = __fadd_rn(__fsub_rn(a, __fsub_rn(sum, bb)), __fsub_rn(b, bb));
    }
    __device__ __forceinline__ void add(float x, float y) {
        const float p = __fmul_rn(x, y), pe = fmaf(x, y, -p);   // x y = p + pe exactly
        float sum, err;
        two_sum(hi, p, sum, err);
        hi = sum;
        lo = __fadd_rn(lo, __fadd_rn(err, pe));
    }
    __device__ __forceinline__ void merge(float ohi, float olo) {
        float sum, err;
        two_sum(hi, ohi, sum, err);
        hi = sum;
        lo = __fadd_rn(lo, __fadd_rn(err, olo));
    }
};

// log2 of the smallest power of two >= v (v >= 1): rows spanned by a tile.
inline int lg_ceil(int v) { return v <= 1 ? 0 : 32 - __builtin_clz((unsigned)(v - 1)); }

// Per-tile gather set-up: lattice base index of each block of the tile and
// the per-array offset of each element DOF (Lagrange node (a, b, c) of the
// block sits on lattice point (i(n-1)+a, j(n-1)+b, c)).
// With eidx, the block index of each tile row is kept as well.
__device__ __forceinline__ void tile_setup(const ApplyArgs& a, const ApplyWork& it, const ArrayDev& A,
                                           long long* base, int* offs, int tile, long long* eidx = nullptr) {
    const int n1 = a.lm->n - 1;
    for (int k = threadIdx.x; k < a.m; k += blockDim.x) {
        int q = k / 3, c = k - 3 * q;
        offs[k] = ((a.lm->qc[q] * A.Y + a.lm->qb[q]) * A.X + a.lm->qa[q]) * 3 + c;
    }
    for (int t = threadIdx.x; t < tile; t += blockDim.x)
        if (t < it.count) {
            const int e = a.blist[it.start + t];
            BlockRef br = a.bref[e];
            base[t] = A.vec_off + 3LL * ((long long)br.j * n1 * A.X + (long long)br.i * n1);
            if (eidx) eidx[t] = e;
        }
}

}  // namespace ms

struct mstress_sol_s {
    mstress_ctx ctx = nullptr;
    int precision = MSTRESS_FP64;
    bool use_tc = false;                  // reduced-precision apply on tensor cores
    int n_arrays = 0, n_types = 0;
    int n = 0, m = 0, ldY = 0;
    int n_el = 0, n_dof_block = 0;
    int64_t n_blocks = 0, n_vec = 0;
    std::vector<ms::ArrayDev> arrays;
    std::vector<mstress_block> types;     // not owned
    std::vector<uint8_t> site;            // type per block (global block order)
    ms::DBuf d_lm, d_arrays, d_bref, d_blist, d_awork, d_awork_tc, d_awork_rec, d_vwork, d_site;
    int n_awork = 0, n_awork_tc = 0, n_awork_rec = 0, n_vwork = 0;
    std::vector<ms::ApplyWork> h_awork, h_awork_rec;   // host copies (filtered recovery)
    std::vector<ms::ApplyWork> h_seg;     // (type, array) runs of the block list (count = run length)
    bool tuned = false;                   // tc_tile picked (or recalled) by the tile autotuner
    int tc_tile = 128;                    // blocks per tensor-core apply tile (<= 128, a multiple of 8: about
                                          // one tile per SM when the batch is small; smaller tiles
                                          // spread a small array's gather over more SMs)
    ms::DBuf b, dinv, fixed;              // FP64 right-hand side, Jacobi inverse (0 on constrained DOFs)
    ms::DBuf dinv32;                      // Jacobi inverse in FP32 (inner PCG of the mixed modes)
    ms::DBuf xbc;                         // prescribed values (lifting), or empty
    ms::PcgVectors v64, v32;              // FP64 outer / plain vectors, FP32 inner vectors
    ms::PcgVectors v64i;                  // FP64 inner vectors (refinement with an FP64 inner solve)
    bool inner64 = false;                 // refinement steps solve the correction in FP64
    bool inner_pending = false;           // the last inner solve's states are on their way to
                                          // ctx->h_states (see flush_inner_iters)
    ms::DBuf Y64own;                      // FP64 element buffer of the mixed modes
    void* Y64 = nullptr;                  // FP64 element products (Y64own, or Y in FP64 mode)
    ms::DBuf Y;                           // element-by-element products [block][ldY]
    ms::DBuf pz;                          // (p, z) pairs of the two-phase tensor-core solver's inner
                                          // PCG (float2 per lattice DOF), or empty
    ms::DBuf part;                        // 3 * n_vwork partial sums
    ms::DBuf gpart;                       // n_grp partial sums of p_e^T Y_e per 8-block group
    int n_grp = 0;
    ms::DBuf cimg;                        // coefficient images of the tensor-core recovery (reused)
    ms::DBuf flag;                        // device ints: [0] any active, [1] CTA ticket, [2] error,
                                          // [3] loop count, [4] arrays active, [7] abort
    ms::DBuf tickets;                     // 2 ints per array (persistent solver folds)
    ms::DBuf timers;                      // 4 u64: ns in phases A, B, C of the persistent solver, loops
    ms::DBuf barrier;                     // grid-barrier words of the persistent solver
    ms::TypeTab tt{};
    std::vector<ms::ArrayResult> results;
    // CUDA graphs of the iteration loop (conditional WHILE node), by vector precision
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_iters[2] = {0, 0};          // kernel nodes per loop iteration
    bool no_while[2] = {false, false};    // conditional nodes unavailable: chunked launches
    ~mstress_sol_s();
};

namespace ms {

struct LayoutIn {
    const mstress_layout* L;
    double dT;
    const mstress_bc* bc;
};

// solve stages (online.cu): build the packed batch of arrays and its work
// lists; right-hand side, diagonal and lifting; the refinement loop pieces;
// final residuals and results
void validate_and_build(mstress_sol_s* s, const std::vector<LayoutIn>& in);
void solve_prepare(mstress_sol_s* s);
void refine_start(mstress_sol_s* s);
bool refine_check(mstress_sol_s* s, bool x_zero = false);   // x_zero: the first check after refine_start
void flush_inner_iters(mstress_sol_s* s);   // after a stream synchronisation: add the inner iterations
void refine_inner(mstress_sol_s* s);
void solve_finish(mstress_sol_s* s, bool refined, bool checked);
void check_device_error(mstress_sol_s* s);

// global-stage launches (online.cu)
ApplyArgs apply_args(mstress_sol_s* s, const void* x, const void* z, const PcgState* st, void* Y, bool tc);
void launch_apply(mstress_sol_s* s, int prec, const void* x, const void* z, bool vec_fp32, const PcgState* st,
                  void* Y);
void launch_isum(mstress_sol_s* s, const void* Y, bool y_fp32, void* p, const void* z, void* q, bool vec_fp32,
                 const void* dinv, const PcgState* st, double* part_pq);   // dinv in the vector precision

// persistent cooperative PCG (pcg_persistent.cu); false if it cannot be launched
bool pcg_run_persistent(mstress_sol_s* s, PcgVectors& v, int prec, int max_iter, bool vec_fp32);

// per-phase PCG iteration for large batches on the streamed tensor-core apply
// (pcg_wide.cu), bitwise equal to the persistent solver's iteration; taken
// from kWideBlocks blocks on (measured: below, the persistent solver's short
// iterations win; from about 3 000 blocks of the degree-4 basis on, the
// occupancy of separate kernels does)
constexpr int64_t kWideBlocks = 4096;
bool pcg_wide(const mstress_sol_s* s, int prec);
void launch_apply_wide(mstress_sol_s* s, int prec, const PcgState* st);   // its apply (st null: beta = 0)
void pcg_iteration_wide(mstress_sol_s* s, PcgVectors& v, int prec, int use_cond, cudaGraphConditionalHandle cond,
                        int loop_cap);

// tensor-core kernels (tc.cu)
bool tc_supported(int m);
bool tc_streamed(int m);   // operator streamed along K (large bases) instead of resident
void configure_tc_kernels();
void launch_apply_tc(mstress_sol_s* s, int prec, const ApplyArgs& a);
void build_tc_operator(mstress_block blk, int prec);   // K_r image for the tensor-core apply

// tensor-core von Mises recovery (tc_recover.cu)
bool tc_recover_supported(int m1, int prec);
// (grid: the cut-plane grid modes instead of the Gauss-mean stress modes)
void recover_vm_tc(mstress_sol_s* s, float* out, bool grid = false);

// recovery (recover.cu)
void recover(mstress_sol_s* s, int what, void* dst, bool dst_dev);
// recovery of the listed arrays only, into a device buffer laid out like the
// whole batch's output (other arrays' parts are left untouched)
void recover_arrays(mstress_sol_s* s, int what, void* dst_dev, const std::vector<int>& arrays);
size_t recover_bytes(const mstress_sol_s* s, int what);

}  // namespace ms
