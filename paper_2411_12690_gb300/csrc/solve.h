// The resident solution of a (batched) global-stage solve and the launch
// helpers the solve and recovery units share.
#pragma once

#include "internal.h"

namespace ms {

constexpr int kVecChunk = 2048;   // lattice DOFs per vector work item
constexpr int kTile64 = 32;       // blocks per FP64 apply / recovery tile

struct ArrayResult {
    int iters = 0, outer = 0, status = MSTRESS_OK;
    double rel_res = 0;
};

// Per-solve device scratch for one conjugate-gradient vector precision.
struct PcgVectors {
    DBuf x, r, z, p, q;   // packed lattice vectors of element type V
    DBuf state;           // PcgState per array
};

}  // namespace ms

struct mstress_sol_s {
    mstress_ctx ctx = nullptr;
    int precision = MSTRESS_FP64;
    int n_arrays = 0, n_types = 0;
    int n = 0, m = 0, ldY = 0;
    int n_el = 0, n_dof_block = 0;
    int64_t n_blocks = 0, n_vec = 0;
    std::vector<ms::ArrayDev> arrays;
    std::vector<mstress_block> types;     // not owned
    std::vector<uint8_t> site;            // type per block (global block order)
    ms::DBuf d_lm, d_arrays, d_bref, d_blist, d_awork, d_vwork, d_site;
    int n_awork = 0, n_vwork = 0;
    ms::DBuf b, dinv, fixed;              // FP64 right-hand side, Jacobi inverse (0 on constrained DOFs)
    ms::DBuf xbc;                         // prescribed values (lifting), or empty
    ms::PcgVectors v64, v32;              // FP64 outer / plain vectors, FP32 inner vectors
    ms::DBuf Y;                           // element-by-element products [block][ldY]
    ms::DBuf part;                        // 3 * n_vwork partial sums
    ms::DBuf flag;                        // device int: any array still iterating
    ms::TypeTab tt{};
    std::vector<ms::ArrayResult> results;
    // captured CUDA graphs of the iteration loop, by vector precision (0: FP64, 1: FP32)
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_iters[2] = {0, 0};
    ~mstress_sol_s();
};

namespace ms {

// global-stage kernels (online.cu)
void launch_apply(mstress_sol_s* s, int prec, const void* x, bool vec_fp32, const PcgState* st, void* Y);
void launch_isum(mstress_sol_s* s, const void* Y, bool y_fp32, const void* p, void* q, bool vec_fp32,
                 const double* dinv, const PcgState* st, double* part_pq);

// recovery (recover.cu)
void recover(mstress_sol_s* s, int what, void* dst, bool dst_dev);
size_t recover_bytes(const mstress_sol_s* s, int what);

}  // namespace ms
