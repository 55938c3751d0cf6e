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

template <class V>
__device__ __forceinline__ V gather(const V* x, const V* z, long long g, V beta) {
    return z ? p_next(z[g], x[g], beta) : x[g];
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

// Gather K groups [kg0, kg0 + nkg) of a tile's coefficients into a K-major
// no-swizzle operand (K group = 16 bytes of K: 8 bf16 or 4 tf32 values; local
// group kgl of the destination at kgl * 128 bytes, row groups sbo apart). The
// thread mapping follows the core matrices: consecutive threads take
// consecutive K values of one row, then the next rows, so a warp's stores fill
// contiguous shared memory (no bank conflicts) and its loads run along a
// block's contiguous lattice DOFs. Rows [count, 1 << lg_tile) and columns
// >= m are written as zeros. Eight values per thread are in flight at a time.
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
                                              uint32_t plane_bytes, uint32_t sbo) {
#pragma unroll
    for (int u = 0; u < GU; ++u) {
        const int idx = idx0 + u * (int)blockDim.x;
        if (idx < total) put_operand(plane0, plane_bytes, OperandMap<MODE>::off(idx, lg_tile, sbo), v[u], MODE);
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
template <int MODE>
__device__ __forceinline__ void gather_operand(const float* __restrict__ x, const float* __restrict__ z, float beta,
                                               int m, int count, const long long* base, const int* offs, int lg_tile,
                                               int kg0, int nkg, uint8_t* plane0, uint32_t plane_bytes, uint32_t sbo) {
    constexpr int GU = 8;
    const int total = nkg << (lg_tile + OperandMap<MODE>::LGKE);
    for (int idx0 = threadIdx.x; idx0 < total; idx0 += (int)blockDim.x * GU) {
        float v[GU];
        operand_load<MODE, GU>(x, z, beta, m, count, base, offs, lg_tile, kg0, total, idx0, v);
        operand_store<MODE, GU>(lg_tile, total, idx0, v, plane0, plane_bytes, sbo);
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
};

// D (128 x npad) = C (tile blocks x K) * K_r^T on the tensor cores for one
// tile; writes the element products Y of the tile's blocks. Returns false if
// the MMA completion wait timed out (the caller stops and reports it).
template <int MODE>
__device__ __forceinline__ bool apply_tc_item(const ApplyArgs& a, const TcShape& sh, const ApplyWork& it,
                                              TcState& ts, long long* base, int* offs) {
    constexpr bool TF32 = MODE == MSTRESS_TF32;
    constexpr int NS = MODE == MSTRESS_BF16X3 ? 2 : 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
    const int m = a.m;
    const ArrayDev A = a.arrays[it.array];
    const float beta = a.st ? (float)a.st[it.array].beta : 0.f;
    const float* __restrict__ x = static_cast<const float*>(a.x);
    const float* __restrict__ z = static_cast<const float*>(a.z);
    float* __restrict__ Y = static_cast<float*>(a.Y);
    if (it.type != ts.cur_type) {
        const uint4* src = static_cast<const uint4*>(a.tt.Klp[it.type]);
        for (uint32_t i = tid; i < NS * sh.b_plane / 16; i += blockDim.x) reinterpret_cast<uint4*>(ts.sB)[i] = src[i];
        ts.cur_type = it.type;
    }
    tile_setup(a, it, A, base, offs, kTileTC);
    __syncthreads();
    gather_operand<MODE>(x, z, beta, m, it.count, base, offs, sh.lg_tile, 0, sh.kpad * sh.esz / 16, ts.sA,
                         sh.a_plane, tc::sbo_bytes(sh.kpad, sh.esz));
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
    const long long e = b < it.count ? a.blist[it.start + b] : 0;
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
// contiguous block in global memory, fetched with a single bulk copy that runs
// while the CTA gathers the matching coefficient columns. An mbarrier per slot
// counts the copy's bytes (full); a tcgen05.commit per slot frees it once
// its MMAs are done (empty). N (= m padded to 16) is split into MMAs of at
// most 256 columns; the accumulator takes npad TMEM columns.
struct TcsShape {
    int m, esz, ns, ck, nck, kpad, npad, n0, n1, tmem_cols, stages;
    int lg_tile;                 // log2 of the blocks per tile of the solve (rows gathered per tile)
    uint32_t a_plane, b_plane;   // bytes of one plane of a slot: A 128 x ck, B npad x ck
    uint32_t a_stage, b_stage;   // bytes of all planes of a slot
    size_t smem;
};

struct TcsState {
    uint8_t* slots;        // stages x (A slot | B slot)
    uint64_t* full;        // [stages] operator copy landed
    uint64_t* empty;       // [stages] MMAs reading the slot are done
    uint32_t tmem;
    uint32_t chunk;        // slots used so far by this CTA (sets slot and parity)
};

}  // namespace ai

ai::TcsShape tcs_shape(int m, int prec);   // streamed tensor-core apply geometry (tc.cu)

namespace ai {

// D (128 x npad) = C (tile blocks x K) * K_r^T for one tile, K streamed.
// Returns false if a wait timed out (the caller stops and reports it).
template <int MODE>
__device__ __forceinline__ bool apply_tcs_item(const ApplyArgs& a, const TcsShape& sh, const ApplyWork& it,
                                               TcsState& ts, long long* base, int* offs) {
    constexpr bool TF32 = MODE == MSTRESS_TF32;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nt = blockDim.x, nw = nt >> 5;
    const int m = a.m;
    const ArrayDev A = a.arrays[it.array];
    const float beta = a.st ? (float)a.st[it.array].beta : 0.f;
    const float* __restrict__ x = static_cast<const float*>(a.x);
    const float* __restrict__ z = static_cast<const float*>(a.z);
    float* __restrict__ Y = static_cast<float*>(a.Y);
    const uint8_t* img = static_cast<const uint8_t*>(a.tt.Klp[it.type]);
    tile_setup(a, it, A, base, offs, kTileTC);
    __syncthreads();
    const uint32_t sbo = tc::sbo_bytes(sh.ck, sh.esz);
    const uint32_t slot_bytes = sh.a_stage + sh.b_stage;
    bool ok = true;
    uint32_t last = 0;
    // When a chunk is one round of loads (blockDim.x * 8 >= its values), the
    // values of chunk c + 1 are loaded into registers while chunk c is stored
    // and its MMAs are issued, so one load latency overlaps the next.
    constexpr int GU = 8;
    const int nkg = sh.ck * sh.esz / 16;
    const int total = nkg << (sh.lg_tile + OperandMap<MODE>::LGKE);
    const bool one_round = total <= nt * GU;
    float vcur[GU], vnext[GU];
    if (one_round) operand_load<MODE, GU>(x, z, beta, m, it.count, base, offs, sh.lg_tile, 0, total, tid, vcur);
    for (int c = 0; c < sh.nck; ++c) {
        const uint32_t g = ts.chunk++, slot = g % (uint32_t)sh.stages, use = g / (uint32_t)sh.stages;
        uint8_t* sA = ts.slots + slot * slot_bytes;
        uint8_t* sB = sA + sh.a_stage;
        last = g;
        if (use > 0 && ok) ok = tc::mbar_wait(&ts.empty[slot], (use - 1) & 1u, 1 << 24);
        if (__syncthreads_or(!ok)) return false;
        if (tid == 0) {
            tc::mbar_expect_tx(&ts.full[slot], sh.b_stage);
            tc::bulk_g2s(sB, img + (size_t)c * sh.b_stage, sh.b_stage, &ts.full[slot]);
        }
        if (one_round) {
            if (c + 1 < sh.nck)
                operand_load<MODE, GU>(x, z, beta, m, it.count, base, offs, sh.lg_tile, (c + 1) * nkg, total, tid,
                                       vnext);
            operand_store<MODE, GU>(sh.lg_tile, total, tid, vcur, sA, sh.a_plane, sbo);
#pragma unroll
            for (int u = 0; u < GU; ++u) vcur[u] = vnext[u];
        } else {
            gather_operand<MODE>(x, z, beta, m, it.count, base, offs, sh.lg_tile, c * nkg, nkg, sA, sh.a_plane, sbo);
        }
        tc::fence_smem_async();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (tid == 0) {
            ok = tc::mbar_wait(&ts.full[slot], use & 1u, 1 << 24);
            if (ok) {
                const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB);
                const uint32_t id0 = tc::instr_desc(TF32, kTileTC, sh.n0);
                const uint32_t id1 = tc::instr_desc(TF32, kTileTC, sh.n1 > 0 ? sh.n1 : 16);
                const uint32_t b1 = (uint32_t)(sh.n0 >> 3) * sbo;   // row n0 of the operator slot
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const uint32_t ko = (uint32_t)j * 2 * tc::kLBO;
                    // products (A plane, B plane): (hi, hi) [, (lo, hi), (hi, lo)]
#pragma unroll
                    for (int pr = 0; pr < (MODE == MSTRESS_BF16X3 ? 3 : 1); ++pr) {
                        const uint32_t pa = pr == 1 ? sh.a_plane : 0u, pb = pr == 2 ? sh.b_plane : 0u;
                        const uint32_t acc = (c > 0 || j > 0 || pr > 0) ? 1u : 0u;
                        const uint64_t da = tc::smem_desc(a0 + pa + ko, tc::kLBO, sbo);
                        tc::mma<TF32>(ts.tmem, da, tc::smem_desc(b0 + pb + ko, tc::kLBO, sbo), id0, acc);
                        if (sh.n1 > 0)
                            tc::mma<TF32>(ts.tmem + (uint32_t)sh.n0, da,
                                          tc::smem_desc(b0 + pb + b1 + ko, tc::kLBO, sbo), id1, acc);
                    }
                }
                tc::commit(&ts.empty[slot]);
            }
        }
    }
    if (__syncthreads_or(!ok)) return false;
    // all MMAs of the tile are done once the last slot's commit has arrived
    ok = tc::mbar_wait(&ts.empty[last % (uint32_t)sh.stages], (last / (uint32_t)sh.stages) & 1u, 1 << 24);
    tc::fence_after();
    if (__syncthreads_or(!ok)) return false;
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (one block each) and
    // column chunks 16 (w / 4), 16 (w / 4 + nw / 4), ...
    const int b = (warp & 3) * 32 + lane;
    const long long e = b < it.count ? a.blist[it.start + b] : 0;
    for (int c0 = 16 * (warp >> 2); c0 < sh.npad; c0 += 16 * (nw >> 2)) {
        float v[16];
        tc::tmem_ld16(ts.tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0, v);
        if (b < it.count) {
            float4* dst = reinterpret_cast<float4*>(Y + e * a.ldY + c0);
            dst[0] = make_float4(v[0], v[1], v[2], v[3]);
            dst[1] = make_float4(v[4], v[5], v[6], v[7]);
            dst[2] = make_float4(v[8], v[9], v[10], v[11]);
            dst[3] = make_float4(v[12], v[13], v[14], v[15]);
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    return true;
}

// Set up the slot barriers of a streamed tensor-core CTA (all threads call).
__device__ __forceinline__ void tcs_init(TcsState& ts, const TcsShape& sh, uint8_t* smem, uint64_t* bars) {
    ts.slots = smem;
    ts.full = bars;
    ts.empty = bars + sh.stages;
    ts.chunk = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < 2 * sh.stages; ++i) tc::mbar_init(&bars[i], 1);
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
    if (threadIdx.x != 0 || ts.chunk == 0) return;
    const uint32_t n = ts.chunk < (uint32_t)sh.stages ? ts.chunk : (uint32_t)sh.stages;
    for (uint32_t i = 0; i < n; ++i) {
        const uint32_t g = ts.chunk - 1 - i, slot = g % (uint32_t)sh.stages, use = g / (uint32_t)sh.stages;
        tc::mbar_wait(&ts.full[slot], use & 1u, 1 << 20);
        tc::mbar_wait(&ts.empty[slot], use & 1u, 1 << 20);
    }
}

}  // namespace ai
}  // namespace ms
