// Element-product (operator apply) work-item bodies, shared by the stand-alone
// apply kernels and the persistent cooperative solver. A work item covers the
// blocks of one tile (one block type, one array):
//   apply64_item    FP64 on CUDA cores, one panel of 8*RPT rows of A_element
//                   for 32 blocks (blockDim.x == 256)
//   apply32_item    reduced precision on CUDA cores (fallback when the tensor
//                   core tile does not fit), 32 blocks (blockDim.x == 256)
//   apply_tc_item   tcgen05 tensor cores, up to 128 blocks (any multiple of 128 threads),
//                   operator resident in shared memory (small bases)
//   apply_tcs_item  tcgen05 tensor cores for large bases: the operator and the
//                   gathered coefficients are streamed through a ring of
//                   shared-memory stages along K
// Every item gathers its blocks' element DOFs straight from the lattice
// vector, optionally forming the search direction z + beta p on the fly.
#pragma once

#include "solve.h"
#include "tc.cuh"

namespace ms {
namespace ai {

__device__ __forceinline__ float round_tf32(float v) { return tc::to_tf32(v); }
__device__ __forceinline__ float round_bf16(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// Loads go through L2 (ld.global.cg): other CTAs of a persistent solve write
// these vectors between grid barriers.
template <class V>
__device__ __forceinline__ V gather(const V* x, const V* z, long long g, V beta) {
    return z ? p_next(__ldcg(z + g), __ldcg(x + g), beta) : __ldcg(x + g);
}

// The same through the read-only L1 path (ld.global.nc), for kernels during
// which nothing writes x or z (the stand-alone applies): neighbouring
// coefficients of one sector, read by separate loads, then hit L1.
template <class V>
__device__ __forceinline__ V gather_nc(const V* x, const V* z, long long g, V beta) {
    return z ? p_next(__ldg(z + g), __ldg(x + g), beta) : __ldg(x + g);
}

// (p, z) pairs through the read-only path: one 8-byte load per coefficient.
__device__ __forceinline__ float gather_pz_nc(const float2* pz, long long g, float beta) {
    const float2 v = __ldg(pz + g);
    return p_next(v.y, v.x, beta);
}

// Gather the element DOFs of a tile of (1 << tile_shift) blocks, index
// idx = k * tile + b, eight values per thread in flight at a time (the loads of
// a round are independent, so they overlap instead of queueing one L2 round
// trip behind another). store(idx, k, b, v) writes one value.
template <class V, class Store>
__device__ __forceinline__ void gather_tile(const V* __restrict__ x, const V* __restrict__ z, V beta, int m,
                                            int tile_shift, int count, const long long* base, const int* offs,
                                            Store store) {
    constexpr int GU = 8;
    const int total = m << tile_shift, mask = (1 << tile_shift) - 1;
    for (int idx0 = threadIdx.x; idx0 < total; idx0 += blockDim.x * GU) {
        V v[GU];
#pragma unroll
        for (int u = 0; u < GU; ++u) {
            const int idx = idx0 + u * blockDim.x;
            v[u] = V(0);
            if (idx < total) {
                const int k = idx >> tile_shift, b = idx & mask;
                if (b < count) v[u] = gather(x, z, base[b] + offs[k], beta);
            }
        }
#pragma unroll
        for (int u = 0; u < GU; ++u) {
            const int idx = idx0 + u * blockDim.x;
            if (idx < total) store(idx, idx >> tile_shift, idx & mask, v[u]);
        }
    }
}

// FP64 element products for one (32-block tile, row panel) item.
// Shared: Cs [m][32], Ks [8*RPT][m]. The caller synchronises before reuse.
template <int RPT>
__device__ __forceinline__ void apply64_item(const ApplyArgs& a, const ApplyWork& it, int panel, double* Cs,
                                             double* Ks, long long* base, int* offs) {
    const int m = a.m;
    const ArrayDev A = a.arrays[it.array];
    const double beta = a.st ? a.st[it.array].beta : 0.0;
    const double* __restrict__ x = static_cast<const double*>(a.x);
    const double* __restrict__ z = static_cast<const double*>(a.z);
    double* __restrict__ Y = static_cast<double*>(a.Y);
    tile_setup(a, it, A, base, offs, kTile64);
    __syncthreads();
    gather_tile(x, z, beta, m, 5, it.count, base, offs, [&](int idx, int, int, double v) { Cs[idx] = v; });
    const double* __restrict__ K = a.tt.Kr[it.type];
    const int r0 = panel * 8 * RPT;
    const int rows = min(8 * RPT, m - r0);
    for (int idx = threadIdx.x; idx < 8 * RPT * m; idx += blockDim.x)
        Ks[idx] = idx < rows * m ? K[(size_t)r0 * m + idx] : 0.0;
    __syncthreads();
    const int rg = threadIdx.x >> 5, bt = threadIdx.x & 31;
    double acc[RPT];
#pragma unroll
    for (int u = 0; u < RPT; ++u) acc[u] = 0;
    const double* kr = Ks + rg * RPT * m;
    for (int k = 0; k < m; ++k) {
        const double c = Cs[k * kTile64 + bt];
#pragma unroll
        for (int u = 0; u < RPT; ++u) acc[u] = fma(kr[u * m + k], c, acc[u]);
    }
    if (bt < it.count) {
        const long long e = a.blist[it.start + bt];
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
            const int r = r0 + rg * RPT + u;
            if (r < m) Y[e * a.ldY + r] = acc[u];
        }
    }
}

// Reduced-precision element products on CUDA cores for one (32-block tile,
// row panel) item. Klp holds K rounded to the operand format (as float;
// BF16X3: [K_hi; K_lo]); the gathered coefficients are rounded the same way
// and the products accumulate in FP32, as on the tensor cores.
template <int RPT, int MODE>
__device__ __forceinline__ void apply32_item(const ApplyArgs& a, const ApplyWork& it, int panel, float* Cs, float* Ks,
                                             long long* base, int* offs) {
    constexpr int NS = MODE == MSTRESS_BF16X3 ? 2 : 1;
    const int m = a.m;
    const ArrayDev A = a.arrays[it.array];
    const float beta = a.st ? (float)a.st[it.array].beta : 0.f;
    const float* __restrict__ x = static_cast<const float*>(a.x);
    const float* __restrict__ z = static_cast<const float*>(a.z);
    float* __restrict__ Y = static_cast<float*>(a.Y);
    tile_setup(a, it, A, base, offs, kTile64);
    __syncthreads();
    gather_tile(x, z, beta, m, 5, it.count, base, offs, [&](int idx, int, int, float v) {
        if (MODE == MSTRESS_TF32) Cs[idx] = round_tf32(v);
        else if (MODE == MSTRESS_BF16) Cs[idx] = round_bf16(v);
        else {
            const float hi = round_bf16(v);
            Cs[idx] = hi;
            Cs[(size_t)m * kTile64 + idx] = round_bf16(v - hi);
        }
    });
    const float* __restrict__ K = static_cast<const float*>(a.tt.Klp[it.type]);
    const int r0 = panel * 8 * RPT;
    const int rows = min(8 * RPT, m - r0);
    for (int s = 0; s < NS; ++s)
        for (int idx = threadIdx.x; idx < 8 * RPT * m; idx += blockDim.x)
            Ks[(size_t)s * 8 * RPT * m + idx] = idx < rows * m ? K[(size_t)s * m * m + (size_t)r0 * m + idx] : 0.0f;
    __syncthreads();
    const int rg = threadIdx.x >> 5, bt = threadIdx.x & 31;
    float acc[RPT];
#pragma unroll
    for (int u = 0; u < RPT; ++u) acc[u] = 0;
    const float* kr = Ks + rg * RPT * m;
    const float* krl = kr + (size_t)8 * RPT * m;
    for (int k = 0; k < m; ++k) {
        const float c = Cs[k * kTile64 + bt];
#pragma unroll
        for (int u = 0; u < RPT; ++u) acc[u] = fmaf(kr[u * m + k], c, acc[u]);
        if (NS == 2) {
            const float cl = Cs[(size_t)m * kTile64 + k * kTile64 + bt];
#pragma unroll
            for (int u = 0; u < RPT; ++u) acc[u] = fmaf(kr[u * m + k], cl, fmaf(krl[u * m + k], c, acc[u]));
        }
    }
    if (bt < it.count) {
        const long long e = a.blist[it.start + bt];
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
            const int r = r0 + rg * RPT + u;
            if (r < m) Y[e * a.ldY + r] = acc[u];
        }
    }
}

// ------------------------------------------------------- tensor cores
struct TcShape {
    int m, esz, kpad, npad, ksteps, tmem_cols, ns;
    int lg_tile;                 // log2 of the blocks per tile of the solve (rows gathered per tile)
    uint32_t a_plane, b_plane;   // bytes per operand plane (multiples of 1024)
    size_t smem;                 // dynamic shared memory of a CTA using this shape
    int ldp;                     // row stride (floats) of the FP32 copy of the gathered tile
    size_t dot_smem;             // extra shared memory for the epilogue dot products (FP32 tile + chunk sums)
};

}  // namespace ai

ai::TcShape tc_shape(int m, int prec);   // tensor-core apply tile geometry (tc.cu)

namespace ai {

__device__ __forceinline__ void put_operand(uint8_t* plane0, uint32_t plane_bytes, uint32_t off, float v, int mode) {
    if (mode == MSTRESS_TF32) {
        *reinterpret_cast<float*>(plane0 + off) = tc::to_tf32(v);
    } else {
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        *reinterpret_cast<__nv_bfloat16*>(plane0 + off) = hi;
        if (mode == MSTRESS_BF16X3)
            *reinterpret_cast<__nv_bfloat16*>(plane0 + plane_bytes + off) =
                __float2bfloat16_rn(v - __bfloat162float(hi));
    }
}

__device__ __forceinline__ void put_operand(uint8_t* plane0, uint32_t plane_bytes, uint32_t off, float v, int mode);

// Element idx of a gathered range of 16-byte K groups of a tile: consecutive
// indices take consecutive K values of one row, then the rows of the tile,
// then the K groups.
template <int MODE>
struct OperandMap {   // element idx of a gathered K-group range -> (row, column, shared-memory offset)
    static constexpr int ESZ = MODE == MSTRESS_TF32 ? 4 : 2;
    static constexpr int LGKE = MODE == MSTRESS_TF32 ? 2 : 3;   // log2 of values per K group
    static constexpr int KE = 1 << LGKE;
    __device__ __forceinline__ static int row(int idx, int lg_tile) { return (idx >> LGKE) & ((1 << lg_tile) - 1); }
    __device__ __forceinline__ static int col(int idx, int lg_tile, int kg0) {
        return ((kg0 + (idx >> (lg_tile + LGKE))) << LGKE) + (idx & (KE - 1));
    }
    __device__ __forceinline__ static uint32_t off(int idx, int lg_tile, uint32_t sbo) {
        const int b = row(idx, lg_tile);
        return (uint32_t)(b >> 3) * sbo + (uint32_t)(idx >> (lg_tile + LGKE)) * 128u + (uint32_t)(b & 7) * 16u +
               (uint32_t)(idx & (KE - 1)) * ESZ;
    }
};

// One round of the gather: the GU values idx0 + u * blockDim.x (u < GU) of a
// K-group range, loaded into registers (zero outside the tile's blocks and m).
template <int MODE, int GU>
__device__ __forceinline__ void operand_load(const float* __restrict__ x, const float* __restrict__ z, float beta,
                                             int m, int count, const long long* base, const int* offs, int lg_tile,
                                             int kg0, int total, int idx0, float (&v)[GU]) {
    using OM = OperandMap<MODE>;
#pragma unroll
    for (int u = 0; u < GU; ++u) {
        const int idx = idx0 + u * (int)blockDim.x;
        const int b = OM::row(idx, lg_tile), k = OM::col(idx, lg_tile, kg0);
        v[u] = 0.f;
        if (idx < total && b < count && k < m) v[u] = gather(x, z, base[b] + offs[k], beta);
    }
}

template <int MODE, int GU>
__device__ __forceinline__ void operand_store(int lg_tile, int total, int idx0, const float (&v)[GU], uint8_t* plane0,
                                              uint32_t plane_bytes, uint32_t sbo, float* sP = nullptr, int ldp = 0,
                                              int kg0 = 0) {
#pragma unroll
    for (int u = 0; u < GU; ++u) {
        const int idx = idx0 + u * (int)blockDim.x;
        if (idx < total) {
            put_operand(plane0, plane_bytes, OperandMap<MODE>::off(idx, lg_tile, sbo), v[u], MODE);
            if (sP) sP[OperandMap<MODE>::row(idx, lg_tile) * ldp + OperandMap<MODE>::col(idx, lg_tile, kg0)] = v[u];
        }
    }
}

// Gather K groups [kg0, kg0 + nkg) of a tile's coefficients into a K-major
// no-swizzle operand (K group = 16 bytes of K: 8 bf16 or 4 tf32 values; local
// group kgl of the destination at kgl * 128 bytes, row groups sbo apart). The
// thread mapping follows the core matrices: consecutive threads take
// consecutive K values of one row, then the next rows, so a warp's stores fill
// contiguous shared memory (no bank conflicts) and its loads run along a
// block's contiguous lattice DOFs. Rows [count, 1 << lg_tile) and columns
// >= m are written as zeros. Eight values per thread are in flight at a time.
// With sP, the gathered FP32 values are also kept at sP[row * ldp + column]
// (the element DOFs p_e for the dot products p_e^T Y_e of the epilogue).
template <int MODE>
__device__ __forceinline__ void gather_operand(const float* __restrict__ x, const float* __restrict__ z, float beta,
                                               int m, int count, const long long* base, const int* offs, int lg_tile,
                                               int kg0, int nkg, uint8_t* plane0, uint32_t plane_bytes, uint32_t sbo,
                                               float* sP = nullptr, int ldp = 0) {
    constexpr int GU = 8;
    const int total = nkg << (lg_tile + OperandMap<MODE>::LGKE);
    for (int idx0 = threadIdx.x; idx0 < total; idx0 += (int)blockDim.x * GU) {
        float v[GU];
        operand_load<MODE, GU>(x, z, beta, m, count, base, offs, lg_tile, kg0, total, idx0, v);
        operand_store<MODE, GU>(lg_tile, total, idx0, v, plane0, plane_bytes, sbo, sP, ldp, kg0);
    }
}

// Gather of a tile's coefficients into the K-major no-swizzle operand for
// its rows [0, count) only: element idx = (kg * count + row) * KE + e takes
// value e of 16-byte K group kg of block row `row` (consecutive threads fill
// one row's group, then the next rows, so a warp's stores cover contiguous
// shared memory). Rows beyond count keep what they held; the MMA rows they
// produce are never read back. GU values per thread are loaded before any is
// stored (one round of loads per GU * blockDim.x values). With sP, the FP32
// values are also kept at sP[row * ldp + k].
// (p, z) pairs: the direction update from one 8-byte load.
__device__ __forceinline__ float gather_pz(const float2* pz, long long g, float beta) {
    const float2 v = __ldcg(pz + g);
    return p_next(v.y, v.x, beta);
}

template <int MODE, int GU>
__device__ __forceinline__ void gather_rows(const float* __restrict__ x, const float* __restrict__ z, float beta,
                                            int m, int count, const long long* base, const int* offs, int nkg,
                                            uint8_t* plane0, uint32_t plane_bytes, uint32_t sbo, float* sP, int ldp,
                                            const float2* pz = nullptr) {
    using OM = OperandMap<MODE>;
    const int total = nkg * count * OM::KE;
    for (int idx0 = threadIdx.x; idx0 < total; idx0 += (int)blockDim.x * GU) {
        float v[GU];
#pragma unroll
        for (int u = 0; u < GU; ++u) {
            const int idx = idx0 + u * (int)blockDim.x;
            v[u] = 0.f;
            if (idx < total) {
                const int q = idx >> OM::LGKE, kg = q / count, row = q - kg * count;
                const int k = (kg << OM::LGKE) + (idx & (OM::KE - 1));
                if (k < m) v[u] = pz ? gather_pz(pz, base[row] + offs[k], beta) : gather(x, z, base[row] + offs[k], beta);
            }
        }
#pragma unroll
        for (int u = 0; u < GU; ++u) {
            const int idx = idx0 + u * (int)blockDim.x;
            if (idx < total) {
                const int e = idx & (OM::KE - 1), q = idx >> OM::LGKE, kg = q / count, row = q - kg * count;
                const uint32_t off = (uint32_t)(row >> 3) * sbo + (uint32_t)kg * 128u + (uint32_t)(row & 7) * 16u +
                                     (uint32_t)e * OM::ESZ;
                put_operand(plane0, plane_bytes, off, v[u], MODE);
                if (sP) sP[row * ldp + (kg << OM::LGKE) + e] = v[u];
            }
        }
    }
}

// gather_rows from (p, z) pairs in two halves, for a tile whose gather is a
// single round (kpad * count <= GU * blockDim.x): the loads, which need no
// beta, and then the direction update p = z + beta p with the same FMA and the
// same stores as gather_rows (so the operands are bitwise the same). Between
// the halves the caller may wait for beta while the loads are in flight.
template <int MODE, int GU>
__device__ __forceinline__ void gather_rows_pz_load(const float2* pz, int m, int count, const long long* base,
                                                    const int* offs, int nkg, float2 (&w)[GU]) {
    using OM = OperandMap<MODE>;
    const int total = nkg * count * OM::KE;
#pragma unroll
    for (int u = 0; u < GU; ++u) {
        const int idx = (int)threadIdx.x + u * (int)blockDim.x;
        w[u] = make_float2(0.f, 0.f);
        if (idx < total) {
            const int q = idx >> OM::LGKE, kg = q / count, row = q - kg * count;
            const int k = (kg << OM::LGKE) + (idx & (OM::KE - 1));
            if (k < m) w[u] = __ldcg(pz + base[row] + offs[k]);
        }
    }
}

template <int MODE, int GU>
__device__ __forceinline__ void gather_rows_pz_store(const float2 (&w)[GU], float beta, int m, int count, int nkg,
                                                     uint8_t* plane0, uint32_t plane_bytes, uint32_t sbo, float* sP,
                                                     int ldp) {
    using OM = OperandMap<MODE>;
    const int total = nkg * count * OM::KE;
#pragma unroll
    for (int u = 0; u < GU; ++u) {
        const int idx = (int)threadIdx.x + u * (int)blockDim.x;
        if (idx < total) {
            const int e = idx & (OM::KE - 1), q = idx >> OM::LGKE, kg = q / count, row = q - kg * count;
            const int k = (kg << OM::LGKE) + e;
            const float v = k < m ? p_next(w[u].y, w[u].x, beta) : 0.f;
            const uint32_t off = (uint32_t)(row >> 3) * sbo + (uint32_t)kg * 128u + (uint32_t)(row & 7) * 16u +
                                 (uint32_t)e * OM::ESZ;
            put_operand(plane0, plane_bytes, off, v, MODE);
            if (sP) sP[row * ldp + (kg << OM::LGKE) + e] = v;
        }
    }
}

// Per-CTA tensor-core state that persists across work items.
struct TcState {
    uint8_t* sA;        // gathered coefficients (NS planes)
    uint8_t* sB;        // operator image of the current type (NS planes)
    uint64_t* mbar;
    uint32_t tmem;
    uint32_t phase;
    int cur_type;
    float* sP;          // optional: FP32 gathered coefficients [128][ldp] (dot products p_e^T Y_e)
    double* sDot;       // [npad / 16][128] column-chunk partial dot products
    int ldp;
    long long* eidx;    // shared [kTileTC]: block index of each row of the current tile
    int cached_start;   // tile whose gather set-up (base, offs, eidx) is in shared memory, or -1
    int cached_array;
    const ArrayDev* A_pre;   // optional: the array and beta of every tile (one array, kept in
    const double* beta_pre;  // shared memory by the caller) instead of loading them per tile
};

// Tile set-up of the tensor-core apply: the operator image of the tile's type
// (when it changes) and the gather offsets (unless this tile's are cached);
// ends with a CTA barrier.
template <int MODE>
__device__ __forceinline__ void apply_tc_setup(const ApplyArgs& a, const TcShape& sh, const ApplyWork& it, TcState& ts,
                                               long long* base, int* offs) {
    constexpr int NS = MODE == MSTRESS_BF16X3 ? 2 : 1;
    const int tid = threadIdx.x;
    if (it.type != ts.cur_type) {
        const uint4* src = static_cast<const uint4*>(a.tt.Klp[it.type]);
        for (uint32_t i = tid; i < NS * sh.b_plane / 16; i += blockDim.x) reinterpret_cast<uint4*>(ts.sB)[i] = src[i];
        ts.cur_type = it.type;
    }
    if (it.start != ts.cached_start || it.array != ts.cached_array) {
        // the same tile again (a persistent CTA with one tile) keeps its set-up
        const ArrayDev A = ts.A_pre ? *ts.A_pre : a.arrays[it.array];
        tile_setup(a, it, A, base, offs, kTileTC, ts.eidx);
        ts.cached_start = it.start;
        ts.cached_array = it.array;
    }
    __syncthreads();
}

template <int MODE>
__device__ __forceinline__ bool apply_tc_finish(const ApplyArgs& a, const TcShape& sh, const ApplyWork& it,
                                                TcState& ts);

// D (128 x npad) = C (tile blocks x K) * K_r^T on the tensor cores for one
// tile; writes the element products Y of the tile's blocks. Returns false if
// the MMA completion wait timed out (the caller stops and reports it).
template <int MODE>
__device__ __forceinline__ bool apply_tc_item(const ApplyArgs& a, const TcShape& sh, const ApplyWork& it,
                                              TcState& ts, long long* base, int* offs) {
    const float* __restrict__ x = static_cast<const float*>(a.x);
    const float* __restrict__ z = static_cast<const float*>(a.z);
    float beta;
    if (ts.A_pre) {
        beta = ts.beta_pre ? (float)*ts.beta_pre : 0.f;
    } else {
        beta = a.st ? (float)a.st[it.array].beta : 0.f;
    }
    apply_tc_setup<MODE>(a, sh, it, ts, base, offs);
    const bool dots = a.gpart != nullptr && ts.sP != nullptr;
    gather_rows<MODE, 12>(x, z, beta, a.m, it.count, base, offs, sh.kpad * sh.esz / 16, ts.sA, sh.a_plane,
                          tc::sbo_bytes(sh.kpad, sh.esz), dots ? ts.sP : nullptr, ts.ldp, a.pz);
    return apply_tc_finish<MODE>(a, sh, it, ts);
}

// The rest of the tile once its operands are in shared memory: the MMAs, the
// element products Y and (two-phase iteration) the group sums of p_e^T Y_e.
template <int MODE>
__device__ __forceinline__ bool apply_tc_finish(const ApplyArgs& a, const TcShape& sh, const ApplyWork& it,
                                                TcState& ts) {
    constexpr bool TF32 = MODE == MSTRESS_TF32;
    constexpr int NS = MODE == MSTRESS_BF16X3 ? 2 : 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
    float* __restrict__ Y = static_cast<float*>(a.Y);
    const bool dots = a.gpart != nullptr && ts.sP != nullptr;
    tc::fence_smem_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid == 0) {
        const uint32_t idesc = tc::instr_desc(TF32, kTileTC, sh.npad);
        const uint32_t sbo = tc::sbo_bytes(sh.kpad, sh.esz);
        const uint32_t a0 = tc::smem_addr(ts.sA), b0 = tc::smem_addr(ts.sB);
        uint32_t acc = 0;
        for (int s = 0; s < sh.ksteps; ++s) {
            const uint32_t ko = (uint32_t)s * 2 * tc::kLBO;
            // products (A plane, B plane): (hi, hi) [, (lo, hi), (hi, lo)]
#pragma unroll
            for (int pr = 0; pr < (NS == 2 ? 3 : 1); ++pr) {
                const uint32_t pa = pr == 1 ? sh.a_plane : 0u, pb = pr == 2 ? sh.b_plane : 0u;
                tc::mma<TF32>(ts.tmem, tc::smem_desc(a0 + pa + ko, tc::kLBO, sbo),
                              tc::smem_desc(b0 + pb + ko, tc::kLBO, sbo), idesc, acc);
                acc = 1;
            }
        }
        tc::commit(ts.mbar);
    }
    const bool ok = tc::mbar_wait(ts.mbar, ts.phase, 1 << 24);
    ts.phase ^= 1u;
    tc::fence_after();
    if (__syncthreads_or(!ok)) return false;
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (one block each) and
    // column chunks 16 (w / 4), 16 (w / 4 + nw / 4), ...
    const int b = (warp & 3) * 32 + lane;
    const long long e = b < it.count ? ts.eidx[b] : 0;
    for (int c0 = 16 * (warp >> 2); c0 < sh.npad; c0 += 16 * (nw >> 2)) {
        float v[16];
        tc::tmem_ld16(ts.tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0, v);
        if (b < it.count && c0 < a.ldY) {
            float4* dst = reinterpret_cast<float4*>(Y + e * a.ldY + c0);
            dst[0] = make_float4(v[0], v[1], v[2], v[3]);
            dst[1] = make_float4(v[4], v[5], v[6], v[7]);
            dst[2] = make_float4(v[8], v[9], v[10], v[11]);
            dst[3] = make_float4(v[12], v[13], v[14], v[15]);
        }
        if (dots && b < it.count) {
            // this chunk's share of p_e^T Y_e, as a double-FP32 sum in column order
            DotAcc<float> acc;
            const float4* pp = reinterpret_cast<const float4*>(ts.sP + b * ts.ldp + c0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 p4 = pp[q];
                acc.add(p4.x, v[4 * q]);
                acc.add(p4.y, v[4 * q + 1]);
                acc.add(p4.z, v[4 * q + 2]);
                acc.add(p4.w, v[4 * q + 3]);
            }
            ts.sDot[(c0 >> 4) * kTileTC + b] = (double)acc.hi + (double)acc.lo;
        }
    }
    if (dots) {
        // one partial per 8-block group of the tile: each block's column
        // chunks summed in order (thread b of warps 0..3), then the group's
        // blocks in order by the first of its 8 lanes (independent of the
        // tile size)
        __syncthreads();
        if (tid < kTileTC) {
            const int nch = sh.npad >> 4;
            double sb = 0;
            if (tid < it.count)
                for (int c = 0; c < nch; ++c) sb += ts.sDot[c * kTileTC + tid];
            double sum = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const double v = __shfl_sync(0xffffffffu, sb, (lane & ~7) + j);
                if ((tid & ~7) + j < it.count) sum += v;
            }
            if ((lane & 7) == 0 && tid < it.count) a.gpart[it.grp + (tid >> 3)] = sum;
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    return true;
}

// ------------------------------------------- tensor cores, streamed along K
// Large bases (m > 80): K_r does not fit in shared memory next to the
// coefficient tile, so both operands move through `stages` ring slots of ck
// K-elements each (two MMA K steps). Slot c of the operator image is one
// contiguous block in global memory, fetched with a single bulk copy. N (= m
// padded to 16) is split into MMAs of at most 256 columns; the accumulator
// takes npad TMEM columns.
//
// The CTA is warp-specialised (kTcsThreads = 16 warps):
//   warp 0, lane 0   issues the operator copies and the MMAs;
//   warps 1..4       epilogue: TMEM lanes 32 (w % 4) .. +31 = the tile's
//                    blocks, all npad columns, written to Y;
//   warps 5..15      gather the coefficients of each K slot (352 threads).
// mbarriers per ring slot: fullA (the 352 gather threads arrive), fullB (the
// operator copy's bytes), empty (tcgen05.commit once the slot's MMAs are
// done); per CTA: accF (commit after a tile's last MMAs) and accE (the 128
// epilogue threads arrive when the accumulator has been read). Gather,
// operator copies, MMAs and the epilogue of consecutive slots and tiles
// overlap; every wait is bounded and a failure stops all roles.
struct TcsShape {
    int m, esz, ns, ck, nck, kpad, npad, n0, n1, tmem_cols, stages;
    int lg_tile;                 // log2 of the blocks per tile of the solve (rows gathered per tile)
    uint32_t a_plane, b_plane;   // bytes of one plane of a slot: A 128 x ck, B npad x ck
    uint32_t a_stage, b_stage;   // bytes of all planes of a slot
    size_t smem;
};

}  // namespace ai

ai::TcsShape tcs_shape(int m, int prec);   // streamed tensor-core apply geometry (tc.cu)

namespace ai {

constexpr int kTcsThreads = 512;       // 16 warps
constexpr int kTcsEpi0 = 32, kTcsEpi = 128;        // epilogue threads [32, 160)
constexpr int kTcsGather0 = 160, kTcsGather = 352; // gather threads [160, 512)
constexpr int kTcsQU = 3;              // gather units per thread per slot (352 x 3 >= 1024 units of 4 values)

struct TcsState {
    uint8_t* slots;        // stages x (A slot | B slot)
    uint64_t *fullA, *fullB, *empty, *accF, *accE;
    uint32_t tmem;
    uint32_t chunk;        // K slots used so far by this CTA (sets slot and parity)
    uint32_t tiles;        // tiles accumulated so far by this CTA (sets accumulator parity)
    int* fail;             // shared: a wait expired
};

__device__ __forceinline__ void named_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Named barrier that also ORs a predicate over the participating threads, so
// that they all take the same branch afterwards.
__device__ __forceinline__ bool named_sync_or(int id, int nthreads, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, %2, %3, p;\nselp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

// Per-tile gather set-up by the gather threads only (thread t of n).
__device__ __forceinline__ void tile_setup_part(const ApplyArgs& a, const ApplyWork& it, const ArrayDev& A,
                                                long long* base, int* offs, int t, int n) {
    const int n1 = a.lm->n - 1;
    for (int k = t; k < a.m; k += n) {
        const int q = k / 3, c = k - 3 * q;
        offs[k] = ((a.lm->qc[q] * A.Y + a.lm->qb[q]) * A.X + a.lm->qa[q]) * 3 + c;
    }
    for (int b = t; b < it.count; b += n) {
        const BlockRef br = a.bref[a.blist[it.start + b]];
        base[b] = A.vec_off + 3LL * ((long long)br.j * n1 * A.X + (long long)br.i * n1);
    }
}

// Gather of one K slot (4 groups of 16 bytes of K) of a tile in quads: a
// gather unit is 4 consecutive K values of one row, so each unit costs one
// base and one 16-byte offset lookup, eight global loads and one store per
// operand plane (8 bytes of bf16 or 16 bytes of tf32). Consecutive units run
// over the 8 rows of a core matrix, then its halves (bf16), then the K groups
// and the row groups, so a warp's stores cover whole core matrices.
template <int MODE>
struct QuadMap {
    static constexpr int LGHQ = MODE == MSTRESS_TF32 ? 0 : 1;   // log2 of quads per 16-byte K group
    static constexpr int UNITS = 128 * 4 << LGHQ;               // units of a 128-row slot
    __device__ __forceinline__ static int row(int ui) { return ((ui >> (5 + LGHQ)) << 3) + (ui & 7); }
    __device__ __forceinline__ static int kg(int ui) { return (ui >> (3 + LGHQ)) & 3; }
    __device__ __forceinline__ static int col(int ui) {   // first K value of the unit within the slot
        return (kg(ui) << (2 + LGHQ)) + (((ui >> 3) & ((1 << LGHQ) - 1)) << 2);
    }
    __device__ __forceinline__ static uint32_t off(int ui, uint32_t sbo) {
        return (uint32_t)(ui >> (5 + LGHQ)) * sbo + (uint32_t)kg(ui) * 128u + (uint32_t)(ui & 7) * 16u +
               (uint32_t)((ui >> 3) & ((1 << LGHQ) - 1)) * 8u;
    }
};

template <int MODE, int QU, bool NC>
__device__ __forceinline__ void quad_load(const float* __restrict__ x, const float* __restrict__ z, float beta, int m,
                                          int count, const long long* base, const int* offs, int k0, int u0, int nthr,
                                          float (&v)[QU][4], const float2* pz = nullptr) {
    using QM = QuadMap<MODE>;
#pragma unroll
    for (int q = 0; q < QU; ++q) {
        const int ui = u0 + q * nthr;
        const int b = QM::row(ui), k = k0 + QM::col(ui);
        const bool live = ui < QM::UNITS && b < count;
        long long bb = 0;
        int4 o = make_int4(0, 0, 0, 0);
        if (live) {
            bb = base[b];
            if (k + 3 < m) o = *reinterpret_cast<const int4*>(offs + k);
            else {
                o.x = k < m ? offs[k] : 0;
                o.y = k + 1 < m ? offs[k + 1] : 0;
                o.z = k + 2 < m ? offs[k + 2] : 0;
            }
        }
        if (NC && pz) {
            v[q][0] = live && k < m ? gather_pz_nc(pz, bb + o.x, beta) : 0.f;
            v[q][1] = live && k + 1 < m ? gather_pz_nc(pz, bb + o.y, beta) : 0.f;
            v[q][2] = live && k + 2 < m ? gather_pz_nc(pz, bb + o.z, beta) : 0.f;
            v[q][3] = live && k + 3 < m ? gather_pz_nc(pz, bb + o.w, beta) : 0.f;
        } else if constexpr (NC) {
            v[q][0] = live && k < m ? gather_nc(x, z, bb + o.x, beta) : 0.f;
            v[q][1] = live && k + 1 < m ? gather_nc(x, z, bb + o.y, beta) : 0.f;
            v[q][2] = live && k + 2 < m ? gather_nc(x, z, bb + o.z, beta) : 0.f;
            v[q][3] = live && k + 3 < m ? gather_nc(x, z, bb + o.w, beta) : 0.f;
        } else {
            v[q][0] = live && k < m ? gather(x, z, bb + o.x, beta) : 0.f;
            v[q][1] = live && k + 1 < m ? gather(x, z, bb + o.y, beta) : 0.f;
            v[q][2] = live && k + 2 < m ? gather(x, z, bb + o.z, beta) : 0.f;
            v[q][3] = live && k + 3 < m ? gather(x, z, bb + o.w, beta) : 0.f;
        }
    }
}

template <int MODE, int QU>
__device__ __forceinline__ void quad_store(int u0, int nthr, const float (&v)[QU][4], uint8_t* plane0,
                                           uint32_t plane_bytes, uint32_t sbo) {
    using QM = QuadMap<MODE>;
#pragma unroll
    for (int q = 0; q < QU; ++q) {
        const int ui = u0 + q * nthr;
        if (ui >= QM::UNITS) continue;
        uint8_t* dst = plane0 + QM::off(ui, sbo);
        if (MODE == MSTRESS_TF32) {
            *reinterpret_cast<float4*>(dst) =
                make_float4(tc::to_tf32(v[q][0]), tc::to_tf32(v[q][1]), tc::to_tf32(v[q][2]), tc::to_tf32(v[q][3]));
        } else {
            __nv_bfloat162 h0 = __floats2bfloat162_rn(v[q][0], v[q][1]), h1 = __floats2bfloat162_rn(v[q][2], v[q][3]);
            uint2 hw;
            hw.x = *reinterpret_cast<uint32_t*>(&h0);
            hw.y = *reinterpret_cast<uint32_t*>(&h1);
            *reinterpret_cast<uint2*>(dst) = hw;
            if (MODE == MSTRESS_BF16X3) {
                const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
                __nv_bfloat162 l0 = __floats2bfloat162_rn(v[q][0] - f0.x, v[q][1] - f0.y);
                __nv_bfloat162 l1 = __floats2bfloat162_rn(v[q][2] - f1.x, v[q][3] - f1.y);
                uint2 lw;
                lw.x = *reinterpret_cast<uint32_t*>(&l0);
                lw.y = *reinterpret_cast<uint32_t*>(&l1);
                *reinterpret_cast<uint2*>(dst + plane_bytes) = lw;
            }
        }
    }
}

// The tiles w0, w0 + wstride, ... (< a.n_work) of arrays still active: every
// thread of the CTA calls this; each takes its role. Returns false if a wait
// expired (ts.fail set). PREFETCH: the gather loads the next K slot's values
// while it stores the current one (two register sets); without it (a kernel
// with less register room) one set. NC: nothing writes x or z during the
// kernel, so the gather may read them through L1 (gather_nc).
template <int MODE, bool PREFETCH = true, bool NC = false>
__device__ bool tcs_apply_phase(const ApplyArgs& a, const TcsShape& sh, TcsState& ts, long long* base, int* offs,
                                int w0, int wstride) {
    constexpr bool TF32 = MODE == MSTRESS_TF32;
    constexpr int kTries = 1 << 24;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t S = (uint32_t)sh.stages;
    const uint32_t slot_bytes = sh.a_stage + sh.b_stage;
    const uint32_t sbo = tc::sbo_bytes(sh.ck, sh.esz);
    const float* __restrict__ x = static_cast<const float*>(a.x);
    const float* __restrict__ z = static_cast<const float*>(a.z);
    float* __restrict__ Y = static_cast<float*>(a.Y);
    uint32_t g = ts.chunk, tt = ts.tiles;
    int* fail = ts.fail;
    if (warp == 0) {
        // ---------------- operator copies and MMAs
        if (lane == 0) {
            const uint32_t id0 = tc::instr_desc(TF32, kTileTC, sh.n0);
            const uint32_t id1 = tc::instr_desc(TF32, kTileTC, sh.n1 > 0 ? sh.n1 : 16);
            const uint32_t b1 = (uint32_t)(sh.n0 >> 3) * sbo;   // row n0 of an operator slot
            for (int w = w0; w < a.n_work && !*(volatile int*)fail; w += wstride) {
                const ApplyWork it = a.work[w];
                if (a.st && !__ldcg(&a.st[it.array].active)) continue;
                const uint8_t* img = static_cast<const uint8_t*>(a.tt.Klp[it.type]);
                bool ok = true;
                // operator slots of the tile's first chunks (their previous MMAs must be done)
                for (uint32_t i = 0; i < S && (int)i < sh.nck && ok; ++i) {
                    const uint32_t gi = g + i, si = gi % S, ui = gi / S;
                    if (ui > 0) ok = tc::mbar_wait(&ts.empty[si], (ui - 1) & 1u, kTries);
                    if (ok) {
                        tc::mbar_expect_tx(&ts.fullB[si], sh.b_stage);
                        tc::bulk_g2s(ts.slots + si * slot_bytes + sh.a_stage, img + (size_t)i * sh.b_stage,
                                     sh.b_stage, &ts.fullB[si]);
                    }
                }
                // the accumulator is free once the previous tile's epilogue has read it
                if (ok && tt > 0) ok = tc::mbar_wait(ts.accE, (tt - 1) & 1u, kTries);
                for (int c = 0; c < sh.nck && ok; ++c, ++g) {
                    const uint32_t slot = g % S, use = g / S;
                    ok = tc::mbar_wait(&ts.fullA[slot], use & 1u, kTries) &&
                         tc::mbar_wait(&ts.fullB[slot], use & 1u, kTries);
                    tc::fence_after();
                    if (!ok) break;
                    const uint32_t a0 = tc::smem_addr(ts.slots + slot * slot_bytes);
                    const uint32_t bb0 = a0 + sh.a_stage;
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const uint32_t ko = (uint32_t)j * 2 * tc::kLBO;
                        // products (A plane, B plane): (hi, hi) [, (lo, hi), (hi, lo)]
#pragma unroll
                        for (int pr = 0; pr < (MODE == MSTRESS_BF16X3 ? 3 : 1); ++pr) {
                            const uint32_t pa = pr == 1 ? sh.a_plane : 0u, pb = pr == 2 ? sh.b_plane : 0u;
                            const uint32_t acc = (c > 0 || j > 0 || pr > 0) ? 1u : 0u;
                            const uint64_t da = tc::smem_desc(a0 + pa + ko, tc::kLBO, sbo);
                            tc::mma<TF32>(ts.tmem, da, tc::smem_desc(bb0 + pb + ko, tc::kLBO, sbo), id0, acc);
                            if (sh.n1 > 0)
                                tc::mma<TF32>(ts.tmem + (uint32_t)sh.n0, da,
                                              tc::smem_desc(bb0 + pb + b1 + ko, tc::kLBO, sbo), id1, acc);
                        }
                    }
                    tc::commit(&ts.empty[slot]);
                    if (c == sh.nck - 1) {
                        tc::commit(ts.accF);
                    } else if (c >= 1 && c - 1 + (int)S < sh.nck) {
                        // refill the previous chunk's operator slot once its MMAs are done
                        const uint32_t gp = g - 1, sp = gp % S;
                        ok = tc::mbar_wait(&ts.empty[sp], (gp / S) & 1u, kTries);
                        if (ok) {
                            tc::mbar_expect_tx(&ts.fullB[sp], sh.b_stage);
                            tc::bulk_g2s(ts.slots + sp * slot_bytes + sh.a_stage,
                                         img + (size_t)(c - 1 + S) * sh.b_stage, sh.b_stage, &ts.fullB[sp]);
                        }
                    }
                }
                if (!ok) {
                    *(volatile int*)fail = 1;
                    break;
                }
                ++tt;
            }
        }
    } else if (warp < 5) {
        // ---------------- epilogue: accumulator lanes -> element products Y
        const int b = ((warp & 3) << 5) + lane;
        for (int w = w0; w < a.n_work; w += wstride) {
            const ApplyWork it = a.work[w];
            if (a.st && !__ldcg(&a.st[it.array].active)) continue;
            bool ok = !*(volatile int*)fail && tc::mbar_wait(ts.accF, tt & 1u, kTries);
            ok = __all_sync(0xffffffffu, ok);   // tensor-memory loads are warp-collective: stop together
            tc::fence_after();
            if (!ok) {
                *(volatile int*)fail = 1;
                break;
            }
            const long long e = b < it.count ? a.blist[it.start + b] : -1;
            const uint32_t tl = ts.tmem + ((uint32_t)((warp & 3) << 5) << 16);
            for (int c0 = 0; c0 < sh.npad; c0 += 16) {
                float v[16];
                tc::tmem_ld16(tl + (uint32_t)c0, v);
                if (e >= 0) {
                    float4* dst = reinterpret_cast<float4*>(Y + e * a.ldY + c0);
                    dst[0] = make_float4(v[0], v[1], v[2], v[3]);
                    dst[1] = make_float4(v[4], v[5], v[6], v[7]);
                    dst[2] = make_float4(v[8], v[9], v[10], v[11]);
                    dst[3] = make_float4(v[12], v[13], v[14], v[15]);
                }
            }
            tc::fence_before();
            tc::mbar_arrive(ts.accE);
            ++tt;
        }
    } else {
        // ---------------- gather of the coefficient slots
        const int gt = tid - kTcsGather0;
        for (int w = w0; w < a.n_work; w += wstride) {
            const ApplyWork it = a.work[w];
            if (a.st && !__ldcg(&a.st[it.array].active)) continue;
            // the previous tile's gather is done with base / offs; every gather
            // thread takes the same decision to stop (a named barrier must not
            // be left with missing arrivals)
            if (named_sync_or(1, kTcsGather, *(volatile int*)fail != 0)) break;
            const ArrayDev A = a.arrays[it.array];
            const float beta = a.st ? (float)a.st[it.array].beta : 0.f;
            tile_setup_part(a, it, A, base, offs, gt, kTcsGather);
            named_sync(1, kTcsGather);
            float vc[kTcsQU][4], vn[kTcsQU][4];
            if (PREFETCH)
                quad_load<MODE, kTcsQU, NC>(x, z, beta, a.m, it.count, base, offs, 0, gt, kTcsGather, vc, a.pz);
            bool ok = true;
            for (int c = 0; c < sh.nck; ++c, ++g) {
                const uint32_t slot = g % S, use = g / S;
                if (!PREFETCH)   // loads issued before the wait for the slot, so they overlap it
                    quad_load<MODE, kTcsQU, NC>(x, z, beta, a.m, it.count, base, offs, c * sh.ck, gt, kTcsGather, vc,
                                                a.pz);
                if (use > 0) ok = tc::mbar_wait(&ts.empty[slot], (use - 1) & 1u, kTries);
                if (!ok) break;
                if (PREFETCH && c + 1 < sh.nck)   // next slot's values in flight while this one is stored
                    quad_load<MODE, kTcsQU, NC>(x, z, beta, a.m, it.count, base, offs, (c + 1) * sh.ck, gt, kTcsGather,
                                            vn, a.pz);
                quad_store<MODE, kTcsQU>(gt, kTcsGather, vc, ts.slots + slot * slot_bytes, sh.a_plane, sbo);
                tc::fence_smem_async();
                tc::mbar_arrive(&ts.fullA[slot]);
                if (PREFETCH) {
#pragma unroll
                    for (int q = 0; q < kTcsQU; ++q)
#pragma unroll
                        for (int j = 0; j < 4; ++j) vc[q][j] = vn[q][j];
                }
            }
            if (!ok) *(volatile int*)fail = 1;   // all gather threads stop at the next tile's barrier
        }
    }
    __syncthreads();
    // every role counted the same active tiles
    uint32_t n_tiles = 0;
    for (int w = w0; w < a.n_work; w += wstride)
        if (!a.st || __ldcg(&a.st[a.work[w].array].active)) ++n_tiles;
    ts.chunk += n_tiles * (uint32_t)sh.nck;
    ts.tiles += n_tiles;
    return *(volatile int*)fail == 0;
}

// Set up the barriers and zero the gathered-operand slots of a streamed
// tensor-core CTA (all threads call; the caller synchronises afterwards).
__device__ __forceinline__ void tcs_init(TcsState& ts, const TcsShape& sh, uint8_t* smem, uint64_t* bars, int* fail) {
    ts.slots = smem;
    ts.fullA = bars;
    ts.fullB = bars + sh.stages;
    ts.empty = bars + 2 * sh.stages;
    ts.accF = bars + 3 * sh.stages;
    ts.accE = ts.accF + 1;
    ts.chunk = 0;
    ts.tiles = 0;
    ts.fail = fail;
    if (threadIdx.x == 0) {
        for (int i = 0; i < sh.stages; ++i) {
            tc::mbar_init(&ts.fullA[i], kTcsGather);
            tc::mbar_init(&ts.fullB[i], 1);
            tc::mbar_init(&ts.empty[i], 1);
        }
        tc::mbar_init(ts.accF, 1);
        tc::mbar_init(ts.accE, kTcsEpi);
        *fail = 0;
    }
    // rows at or beyond the solve's tile size are never gathered: keep them zero
    for (int st = 0; st < sh.stages; ++st) {
        uint4* a0 = reinterpret_cast<uint4*>(smem + (size_t)st * (sh.a_stage + sh.b_stage));
        for (uint32_t i = threadIdx.x; i < sh.a_stage / 16; i += blockDim.x) a0[i] = make_uint4(0, 0, 0, 0);
    }
}

// Bounded drain before a streamed tensor-core CTA exits after a failed wait:
// let outstanding operator copies and MMAs finish so that neither writes
// shared or tensor memory after the CTA is gone.
__device__ __forceinline__ void tcs_drain(const TcsState& ts, const TcsShape& sh) {
    if (threadIdx.x != 0) return;
    for (int i = 0; i < sh.stages; ++i)
        for (uint32_t par = 0; par < 2; ++par) {
            tc::mbar_wait(&ts.fullB[i], par, 1 << 16);
            tc::mbar_wait(&ts.empty[i], par, 1 << 16);
        }
    tc::mbar_wait(ts.accF, 0, 1 << 16);
    tc::mbar_wait(ts.accF, 1, 1 << 16);
}

}  // namespace ai
}  // namespace ms
