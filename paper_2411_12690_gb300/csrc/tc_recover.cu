// Per-element von Mises recovery on the tensor cores (tcgen05, sm_103a).
//
// For the blocks of one type, Sigma_mean = S_mean [c_e; dT] (Eq. 15 and Eq. 1,
// averaged over the 8 Gauss points of each element) is one dense contraction
//     D (blocks x rows) = C (blocks x K) * S_mean^T,   K = m + 1 (padded)
// where C holds the gathered element DOFs of 128 blocks plus the dT column and
// a 128-row tile of S_mean holds the 6 stress components of 21 elements
// (row 6 le + c; rows 126, 127 zero). The accumulator puts one block in each
// TMEM lane and an element's six components in six adjacent columns, so each
// thread of the epilogue forms the von Mises of its own block's elements with
// no data exchange; the results are staged in shared memory and written as
// runs of consecutive elements per block.
//
// A work item is one 128-block tile and a run of element tiles. Its coefficient
// tile stays in shared memory; the S_mean tiles stream through a ring of
// shared-memory stages by bulk copies (mbarriers count the bytes), and two
// TMEM accumulators let the MMAs of element tile t run while the epilogue of
// tile t - 1 reads the other accumulator. One thread issues copies and MMAs;
// all threads run the epilogue. Every wait has an iteration limit; on expiry
// the kernel records an error, drains what it issued and frees its TMEM.
//
// Operand images: the S_mean tile images are built once per block model; the
// coefficient images (one per 128-block tile) are built by a gather kernel at
// every recovery, in the same K-major core-matrix layout.
#include <algorithm>

#include "solve.h"
#include "tc.cuh"

namespace ms {
namespace {

constexpr int kRecThreads = 256;
constexpr int kElemPerTile = 21;   // 21 elements x 6 components = 126 of 128 rows
constexpr int kMaxStages = 3;

struct RecShape {
    int m1, esz, kpad, ksteps, ns, n_etiles, stages;
    uint32_t plane;                  // bytes of one 128 x kpad operand plane
    uint32_t set;                    // bytes of one operand tile (all planes)
    size_t smem;
};

RecShape rec_shape(int m1, int n_el, int prec) {
    RecShape s;
    s.m1 = m1;
    s.esz = prec == MSTRESS_TF32 ? 4 : 2;
    s.kpad = (int)round_up(m1, 32 / s.esz);
    s.ksteps = s.kpad * s.esz / 32;
    s.ns = prec == MSTRESS_BF16X3 ? 2 : 1;
    s.n_etiles = (n_el + kElemPerTile - 1) / kElemPerTile;
    s.plane = (uint32_t)round_up((int64_t)128 * s.kpad * s.esz, 1024);
    s.set = (uint32_t)s.ns * s.plane;
    const int64_t room = 200 * 1024 - 1024 - (int64_t)s.set;   // next to the resident coefficient tile
    s.stages = (int)std::max<int64_t>(0, std::min<int64_t>(kMaxStages, room / s.set));
    s.smem = (size_t)(1 + s.stages) * s.set + 1024;
    return s;
}

template <int MODE>
__device__ __forceinline__ void put(uint8_t* p0, uint32_t plane, uint32_t off, double v) {
    if (MODE == MSTRESS_TF32) {
        *reinterpret_cast<float*>(p0 + off) = tc::to_tf32((float)v);
    } else {
        const __nv_bfloat16 hi = __float2bfloat16_rn((float)v);
        *reinterpret_cast<__nv_bfloat16*>(p0 + off) = hi;
        if (MODE == MSTRESS_BF16X3)
            *reinterpret_cast<__nv_bfloat16*>(p0 + plane + off) =
                __float2bfloat16_rn((float)(v - (double)__bfloat162float(hi)));
    }
}

// S_mean tile images of one block model: tile t row r = 6 le + c holds
// S_mean[(21 t + le) * 6 + c][k] (zero beyond the last element, for rows
// 126, 127 and for k >= m+1).
template <int MODE>
__global__ void k_smean_image(const double* Smean, int ld, int m1, int n_el, RecShape sh, uint8_t* out) {
    const long long n = (long long)sh.n_etiles * 128 * sh.kpad;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int k = (int)(t % sh.kpad);
    const long long rt = t / sh.kpad;
    const int r = (int)(rt % 128);
    const int tile = (int)(rt / 128);
    const int le = r / 6, c = r % 6;
    const int el = tile * kElemPerTile + le;
    double v = 0.0;
    if (le < kElemPerTile && el < n_el && k < m1) v = Smean[((size_t)el * 6 + c) * ld + k];
    put<MODE>(out + (size_t)tile * sh.set, sh.plane, tc::operand_offset(r, k, sh.kpad, sh.esz), v);
}

// Coefficient images, one per 128-block tile: row b = block, column k < m is
// the element DOF c_e[k] gathered from the lattice solution, column m is dT.
// Consecutive threads take consecutive K values of one row (16-byte K groups,
// then rows, then groups), so the stores are contiguous and the loads run
// along a block's lattice DOFs.
template <int MODE>
__global__ void k_coeff_image(const __grid_constant__ ApplyArgs a, RecShape sh, uint8_t* out) {
    constexpr int ESZ = MODE == MSTRESS_TF32 ? 4 : 2;
    constexpr int LGKE = MODE == MSTRESS_TF32 ? 2 : 3;
    __shared__ long long base[kTileTC];
    __shared__ int offs[3 * kMaxSurf];
    const double* __restrict__ x = static_cast<const double*>(a.x);
    const uint32_t sbo = tc::sbo_bytes(sh.kpad, ESZ);
    const int total = sh.kpad * kTileTC;
    for (int w = blockIdx.x; w < a.n_work; w += gridDim.x) {
        const ApplyWork it = a.work[w];
        const ArrayDev A = a.arrays[it.array];
        __syncthreads();
        tile_setup(a, it, A, base, offs, kTileTC);
        __syncthreads();
        uint8_t* img = out + (size_t)w * sh.set;
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int kk = idx & ((1 << LGKE) - 1), b = (idx >> LGKE) & (kTileTC - 1), kg = idx >> (LGKE + 7);
            const int k = (kg << LGKE) + kk;
            double v = 0.0;
            if (b < it.count && k < a.m) v = x[base[b] + offs[k]];
            else if (b < it.count && k == a.m) v = A.dT;
            const uint32_t off = (uint32_t)(b >> 3) * sbo + (uint32_t)kg * 128u + (uint32_t)(b & 7) * 16u +
                                 (uint32_t)kk * ESZ;
            put<MODE>(img, sh.plane, off, v);
        }
    }
}

__device__ __forceinline__ float von_mises6(const float* s) {
    const float d0 = s[0] - s[1], d1 = s[1] - s[2], d2 = s[2] - s[0];
    return sqrtf(0.5f * (d0 * d0 + d1 * d1 + d2 * d2) + 3.0f * (s[3] * s[3] + s[4] * s[4] + s[5] * s[5]));
}

struct RecTcArgs {
    const ApplyWork* work;          // 128-block tiles (one type, one array)
    int n_work;
    const int* blist;
    const uint8_t* cimg;            // coefficient images, one per block tile
    const uint8_t* simg[kMaxTypes]; // S_mean tile images per type
    int n_el;
    float* out;                     // [block][n_el]
    int* err;
};

template <int MODE>
__global__ void __launch_bounds__(kRecThreads, 1) k_recover_tc(const __grid_constant__ RecTcArgs a,
                                                                const RecShape sh) {
    constexpr bool TF32 = MODE == MSTRESS_TF32;
    constexpr int NS = MODE == MSTRESS_BF16X3 ? 2 : 1;
    constexpr int kTries = 1 << 24;
    extern __shared__ uint8_t smraw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    uint8_t* sB = smem;              // coefficients of the item's block tile
    uint8_t* sA0 = smem + sh.set;    // S_mean tile stages
    __shared__ __align__(8) uint64_t bfull, afull[kMaxStages], aempty[kMaxStages], accfull[2], accempty[2];
    __shared__ uint32_t tmem_base;
    __shared__ long long eidx[kTileTC];
    __shared__ float ostage[kTileTC * kElemPerTile];   // von Mises of one element tile, [block][element]
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = sh.stages;
    if (warp == 0) tc::tmem_alloc(&tmem_base, 256);
    if (tid == 0) {
        tc::mbar_init(&bfull, 1);
        for (int i = 0; i < S; ++i) {
            tc::mbar_init(&afull[i], 1);
            tc::mbar_init(&aempty[i], 1);
        }
        for (int j = 0; j < 2; ++j) {
            tc::mbar_init(&accfull[j], 1);
            tc::mbar_init(&accempty[j], kRecThreads);
        }
        s_fail = 0;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = tc::instr_desc(TF32, 128, 128);
    const uint32_t sbo = tc::sbo_bytes(sh.kpad, sh.esz);
    // epilogue geometry: TMEM lane (= block of the tile) and which elements:
    // warps 0-3 elements 0..9 (columns 0..63), warps 4-7 elements 10..20 (columns 48..127)
    const int lg = warp & 3, half = warp >> 2;
    const int bl = 32 * lg + lane;
    uint32_t T = 0;                               // element tiles whose MMAs this CTA has issued
    uint32_t items = 0;                           // work items (coefficient tiles) finished
    bool ok = true;
    // this CTA's share of the (block tile, element tile) pairs, in block-tile
    // major order: a contiguous range, so every CTA gets the same number of
    // element tiles (+-1) and at most a few coefficient tiles
    const long long n_pairs = (long long)a.n_work * sh.n_etiles;
    const long long p_end = n_pairs * (blockIdx.x + 1) / gridDim.x;
    for (long long p = n_pairs * blockIdx.x / gridDim.x; p < p_end;) {
        const int tw = (int)(p / sh.n_etiles);
        const int e0 = (int)(p - (long long)tw * sh.n_etiles);
        const int nt = (int)min((long long)(sh.n_etiles - e0), p_end - p);
        p += nt;
        const ApplyWork it = a.work[tw];
        const uint8_t* simg = a.simg[it.type];
        __syncthreads();                          // the previous item's epilogue is done with eidx
        if (tid < kTileTC) eidx[tid] = tid < it.count ? (long long)a.blist[it.start + tid] : -1;
        if (tid == 0) {
            // every MMA of the previous item has completed (its last epilogue waited for it)
            tc::mbar_expect_tx(&bfull, sh.set);
            tc::bulk_g2s(sB, a.cimg + (size_t)tw * sh.set, sh.set, &bfull);
            for (int i = 0; i < min(S, nt); ++i) {
                const uint32_t g = T + i, s = g % S, use = g / S;
                if (use > 0 && !tc::mbar_wait(&aempty[s], (use - 1) & 1u, kTries)) s_fail = 1;
                tc::mbar_expect_tx(&afull[s], sh.set);
                tc::bulk_g2s(sA0 + (size_t)s * sh.set, simg + (size_t)(e0 + i) * sh.set, sh.set, &afull[s]);
            }
        }
        __syncthreads();
        for (int i = 0; i <= nt; ++i) {
            if (i < nt && tid == 0 && !s_fail) {   // MMAs of element tile e0 + i
                const uint32_t g = T + i, s = g % S, j = g & 1u;
                bool w_ok = true;
                if (i == 0) w_ok = tc::mbar_wait(&bfull, items & 1u, kTries);
                if (w_ok && g >= 2) w_ok = tc::mbar_wait(&accempty[j], ((g >> 1) - 1) & 1u, kTries);
                if (w_ok) w_ok = tc::mbar_wait(&afull[s], (g / S) & 1u, kTries);
                tc::fence_after();
                if (w_ok) {
                    const uint32_t a0 = tc::smem_addr(sA0 + (size_t)s * sh.set), b0 = tc::smem_addr(sB);
                    uint32_t acc = 0;
                    for (int ks = 0; ks < sh.ksteps; ++ks) {
                        const uint32_t ko = (uint32_t)ks * 2 * tc::kLBO;
#pragma unroll
                        for (int pr = 0; pr < (NS == 2 ? 3 : 1); ++pr) {
                            const uint32_t pa = pr == 1 ? sh.plane : 0u, pb = pr == 2 ? sh.plane : 0u;
                            // M = blocks (coefficients), N = S_mean rows
                            tc::mma<TF32>(tmem + 128u * j, tc::smem_desc(b0 + pb + ko, tc::kLBO, sbo),
                                          tc::smem_desc(a0 + pa + ko, tc::kLBO, sbo), idesc, acc);
                            acc = 1;
                        }
                    }
                    tc::commit(&accfull[j]);
                    tc::commit(&aempty[s]);
                    if (S >= 2 && i >= 1 && i - 1 + S < nt) {
                        // refill the stage of the previous tile (its MMAs have had a tile's time)
                        const uint32_t gp = g - 1, sp = gp % S;
                        w_ok = tc::mbar_wait(&aempty[sp], (gp / S) & 1u, kTries);
                        if (w_ok) {
                            tc::mbar_expect_tx(&afull[sp], sh.set);
                            tc::bulk_g2s(sA0 + (size_t)sp * sh.set, simg + (size_t)(e0 + i - 1 + S) * sh.set,
                                         sh.set, &afull[sp]);
                        }
                    } else if (S == 1 && i + 1 < nt) {
                        // a single stage: wait for this tile's MMAs, then fetch the next tile
                        w_ok = tc::mbar_wait(&aempty[0], g & 1u, kTries);
                        if (w_ok) {
                            tc::mbar_expect_tx(&afull[0], sh.set);
                            tc::bulk_g2s(sA0, simg + (size_t)(e0 + i + 1) * sh.set, sh.set, &afull[0]);
                        }
                    }
                }
                if (!w_ok) s_fail = 1;
            }
            if (i >= 1) {   // epilogue of element tile e0 + i - 1
                const uint32_t g = T + i - 1, j = g & 1u;
                const bool got = !s_fail && tc::mbar_wait(&accfull[j], (g >> 1) & 1u, kTries);
                tc::fence_after();
                if (got) {
                    const uint32_t tl = tmem + ((uint32_t)(32 * lg) << 16) + 128u * j;
                    float* orow = ostage + bl * kElemPerTile;
                    if (half == 0) {
                        float v[64];
#pragma unroll
                        for (int c = 0; c < 64; c += 16) tc::tmem_ld16(tl + (uint32_t)c, v + c);
#pragma unroll
                        for (int e = 0; e < 10; ++e) orow[e] = von_mises6(v + 6 * e);
                    } else {
                        float v[80];
#pragma unroll
                        for (int c = 0; c < 80; c += 16) tc::tmem_ld16(tl + 48u + (uint32_t)c, v + c);
#pragma unroll
                        for (int e = 10; e < kElemPerTile; ++e) orow[e] = von_mises6(v + 6 * e - 48);
                    }
                } else {
                    s_fail = 1;
                }
                tc::fence_before();
                tc::mbar_arrive(&accempty[j]);
                __syncthreads();
                // runs of up to 21 consecutive elements per block
                const int el0 = (e0 + i - 1) * kElemPerTile;
                const int ne = min(kElemPerTile, a.n_el - el0);
                for (int o = tid; o < it.count * kElemPerTile; o += kRecThreads) {
                    const int b = o / kElemPerTile, e = o - b * kElemPerTile;
                    if (e < ne) a.out[eidx[b] * a.n_el + el0 + e] = ostage[o];
                }
            }
            if (__syncthreads_or(s_fail)) {
                ok = false;
                break;
            }
        }
        if (!ok) break;
        T += nt;
        ++items;
    }
    if (!ok && tid == 0) {
        atomicExch(a.err, 1);
        // bounded drain: let issued copies and MMAs finish before the CTA leaves
        tc::mbar_wait(&bfull, (items & 1u), 1 << 20);
        for (int s = 0; s < S; ++s) {
            tc::mbar_wait(&afull[s], 0, 1 << 16);
            tc::mbar_wait(&afull[s], 1, 1 << 16);
        }
        for (int j = 0; j < 2; ++j) {
            tc::mbar_wait(&accfull[j], 0, 1 << 16);
            tc::mbar_wait(&accfull[j], 1, 1 << 16);
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, 256);
}

// ----------------------------------------------------------- streamed K
// Large bases (the coefficient tile does not fit in shared memory next to an
// S_mean stage): both operands stream along K in slots of kc values (two MMA K
// steps, 64 bytes of K per row). Both images are stored slot by slot (per
// tile, per slot, per plane a 128 x kc K-major no-swizzle block), so that one
// slot of each operand is one bulk copy. The CTA is split in two roles: warp 0
// (one thread) issues the copies and the MMAs, warps 1-8 run the epilogue.
// Barriers: full[s] (both copies' bytes), empty[s] (tcgen05.commit after the
// slot's MMAs), accfull[j] (commit after an element tile's last slot) and
// accempty[j] (the 256 epilogue threads arrive when the accumulator is read).
constexpr int kRecsThreads = 288;   // 1 + 8 warps
constexpr int kRecsEpi = 256;

struct RecsShape {
    int m1, esz, ns, kc, nks, kpad, n_etiles, stages;
    uint32_t plane;                  // bytes of one 128 x kc plane of a slot
    uint32_t slot;                   // ns * plane: one operand's bytes per slot
    size_t smem;
};

RecsShape recs_shape(int m1, int n_el, int prec) {
    RecsShape s;
    s.m1 = m1;
    s.esz = prec == MSTRESS_TF32 ? 4 : 2;
    s.ns = prec == MSTRESS_BF16X3 ? 2 : 1;
    s.kc = 64 / s.esz;
    s.nks = (m1 + s.kc - 1) / s.kc;
    s.kpad = s.nks * s.kc;
    s.n_etiles = (n_el + kElemPerTile - 1) / kElemPerTile;
    s.plane = (uint32_t)(128 * s.kc * s.esz);
    s.slot = (uint32_t)s.ns * s.plane;
    s.stages = (int)std::min<size_t>(4, (200 * 1024 - 1024) / (2 * (size_t)s.slot));
    s.smem = (size_t)s.stages * 2 * s.slot + 1024;
    return s;
}

// Byte offset of element (row, k) of tile t in a slot-by-slot image.
__device__ __forceinline__ size_t slot_offset(const RecsShape& sh, long long t, int row, int k) {
    const int ks = k / sh.kc, kk = k - ks * sh.kc;
    return ((size_t)t * sh.nks + ks) * sh.slot + tc::operand_offset(row, kk, sh.kc, sh.esz);
}

template <int MODE>
__global__ void k_smean_image_s(const double* Smean, int ld, int m1, int n_el, RecsShape sh, uint8_t* out) {
    const long long n = (long long)sh.n_etiles * 128 * sh.kpad;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int k = (int)(t % sh.kpad);
    const long long rt = t / sh.kpad;
    const int r = (int)(rt % 128);
    const long long tile = rt / 128;
    const int le = r / 6, c = r % 6;
    const long long el = tile * kElemPerTile + le;
    double v = 0.0;
    if (le < kElemPerTile && el < n_el && k < m1) v = Smean[((size_t)el * 6 + c) * ld + k];
    put<MODE>(out + slot_offset(sh, tile, r, k) - tc::operand_offset(r, k % sh.kc, sh.kc, sh.esz),
              sh.plane, tc::operand_offset(r, k % sh.kc, sh.kc, sh.esz), v);
}

template <int MODE>
__global__ void k_coeff_image_s(const __grid_constant__ ApplyArgs a, RecsShape sh, uint8_t* out) {
    __shared__ long long base[kTileTC];
    __shared__ int offs[3 * kMaxSurf];
    const double* __restrict__ x = static_cast<const double*>(a.x);
    const int total = sh.kpad * kTileTC;
    for (int w = blockIdx.x; w < a.n_work; w += gridDim.x) {
        const ApplyWork it = a.work[w];
        const ArrayDev A = a.arrays[it.array];
        __syncthreads();
        tile_setup(a, it, A, base, offs, kTileTC);
        __syncthreads();
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int b = idx / sh.kpad, k = idx - b * sh.kpad;   // consecutive threads: one row's K values
            double v = 0.0;
            if (b < it.count && k < a.m) v = x[base[b] + offs[k]];
            else if (b < it.count && k == a.m) v = A.dT;
            const uint32_t o = tc::operand_offset(b, k % sh.kc, sh.kc, sh.esz);
            put<MODE>(out + slot_offset(sh, w, b, k) - o, sh.plane, o, v);
        }
    }
}

__device__ __forceinline__ bool epi_sync_or(bool pred) {   // named barrier 1 over the epilogue warps
    uint32_t r;
    asm volatile(
        "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, 1, %2, p;\nselp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"((uint32_t)pred), "n"(kRecsEpi)
        : "memory");
    return r != 0;
}

template <int MODE>
__global__ void __launch_bounds__(kRecsThreads, 1) k_recover_tcs(const __grid_constant__ RecTcArgs a,
                                                                  const RecsShape sh) {
    constexpr bool TF32 = MODE == MSTRESS_TF32;
    constexpr int NS = MODE == MSTRESS_BF16X3 ? 2 : 1;
    constexpr int kTries = 1 << 24;
    extern __shared__ uint8_t smraw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[4], empty[4], accfull[2], accempty[2];
    __shared__ uint32_t tmem_base;
    __shared__ float ostage[kTileTC * kElemPerTile];
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t S = (uint32_t)sh.stages;
    if (warp == 0) tc::tmem_alloc_c<256>(&tmem_base);
    if (tid == 0) {
        for (uint32_t i = 0; i < S; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        for (int j = 0; j < 2; ++j) {
            tc::mbar_init(&accfull[j], 1);
            tc::mbar_init(&accempty[j], kRecsEpi);
        }
        s_fail = 0;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_base;
    // this CTA's contiguous range of (block tile, element tile) pairs, block-tile major
    const long long n_pairs = (long long)a.n_work * sh.n_etiles;
    const long long p0 = n_pairs * blockIdx.x / gridDim.x, p1 = n_pairs * (blockIdx.x + 1) / gridDim.x;
    const uint32_t n_tiles = (uint32_t)(p1 - p0), n_slots = n_tiles * (uint32_t)sh.nks;
    if (warp == 0) {
        if (lane == 0) {
            // the copies of global slot q: pair p0 + q / nks, K slot q % nks
            auto issue = [&](uint32_t q) {
                const long long pr = p0 + q / sh.nks;
                const int ks = (int)(q % sh.nks);
                const int bt = (int)(pr / sh.n_etiles), et = (int)(pr - (long long)bt * sh.n_etiles);
                const uint32_t s = q % S;
                uint8_t* dst = smem + (size_t)s * 2 * sh.slot;
                tc::mbar_expect_tx(&full[s], 2 * sh.slot);
                tc::bulk_g2s(dst, a.simg[a.work[bt].type] + ((size_t)et * sh.nks + ks) * sh.slot, sh.slot, &full[s]);
                tc::bulk_g2s(dst + sh.slot, a.cimg + ((size_t)bt * sh.nks + ks) * sh.slot, sh.slot, &full[s]);
            };
            const uint32_t idesc = tc::instr_desc(TF32, 128, 128);
            const uint32_t sbo = tc::sbo_bytes(sh.kc, sh.esz);
            bool ok = true;
            for (uint32_t q = 0; q < S && q < n_slots; ++q) issue(q);
            for (uint32_t g = 0; g < n_tiles && ok; ++g) {
                const uint32_t j = g & 1u;
                if (g >= 2) ok = tc::mbar_wait(&accempty[j], ((g >> 1) - 1) & 1u, kTries);
                for (int ks = 0; ks < sh.nks && ok; ++ks) {
                    const uint32_t q = g * (uint32_t)sh.nks + (uint32_t)ks, s = q % S;
                    ok = tc::mbar_wait(&full[s], (q / S) & 1u, kTries);
                    tc::fence_after();
                    if (!ok) break;
                    const uint32_t a0 = tc::smem_addr(smem + (size_t)s * 2 * sh.slot);   // S_mean slot
                    const uint32_t b0 = a0 + sh.slot;                                   // coefficient slot
#pragma unroll
                    for (int kj = 0; kj < 2; ++kj) {
                        const uint32_t ko = (uint32_t)kj * 2 * tc::kLBO;
#pragma unroll
                        for (int pr = 0; pr < (NS == 2 ? 3 : 1); ++pr) {
                            const uint32_t pa = pr == 1 ? sh.plane : 0u, pb = pr == 2 ? sh.plane : 0u;
                            const uint32_t acc = (ks > 0 || kj > 0 || pr > 0) ? 1u : 0u;
                            // M = blocks (coefficients), N = S_mean rows
                            tc::mma<TF32>(tmem + 128u * j, tc::smem_desc(b0 + pb + ko, tc::kLBO, sbo),
                                          tc::smem_desc(a0 + pa + ko, tc::kLBO, sbo), idesc, acc);
                        }
                    }
                    tc::commit(&empty[s]);
                    if (ks == sh.nks - 1) tc::commit(&accfull[j]);
                    // refill the previous slot's stage once its MMAs are done
                    if (q >= 1 && q - 1 + S < n_slots) {
                        const uint32_t sp = (q - 1) % S;
                        ok = tc::mbar_wait(&empty[sp], ((q - 1) / S) & 1u, kTries);
                        if (ok) issue(q - 1 + S);
                    }
                }
            }
            if (!ok) *(volatile int*)&s_fail = 1;
        }
    } else {
        // ---------------- epilogue: blocks on TMEM lanes, one element tile at a time
        const int et_id = tid - 32;                       // 0..255
        const int lg = warp & 3, half = (warp - 1) >> 2;  // warps 1-4: elements 0..9, warps 5-8: 10..20
        const int bl = 32 * lg + lane;
        for (uint32_t g = 0; g < n_tiles; ++g) {
            const uint32_t j = g & 1u;
            const long long pr = p0 + g;
            const int bt = (int)(pr / sh.n_etiles), et = (int)(pr - (long long)bt * sh.n_etiles);
            const bool got = !*(volatile int*)&s_fail && tc::mbar_wait(&accfull[j], (g >> 1) & 1u, kTries);
            tc::fence_after();
            if (got) {
                const uint32_t tl = tmem + ((uint32_t)(32 * lg) << 16) + 128u * j;
                float* orow = ostage + bl * kElemPerTile;
                if (half == 0) {
                    float v[64];
#pragma unroll
                    for (int c = 0; c < 64; c += 16) tc::tmem_ld16(tl + (uint32_t)c, v + c);
#pragma unroll
                    for (int e = 0; e < 10; ++e) orow[e] = von_mises6(v + 6 * e);
                } else {
                    float v[80];
#pragma unroll
                    for (int c = 0; c < 80; c += 16) tc::tmem_ld16(tl + 48u + (uint32_t)c, v + c);
#pragma unroll
                    for (int e = 10; e < kElemPerTile; ++e) orow[e] = von_mises6(v + 6 * e - 48);
                }
            } else {
                *(volatile int*)&s_fail = 1;
            }
            tc::fence_before();
            tc::mbar_arrive(&accempty[j]);
            if (epi_sync_or(!got)) break;
            const ApplyWork it = a.work[bt];
            const int el0 = et * kElemPerTile;
            const int ne = min(kElemPerTile, a.n_el - el0);
            for (int o = et_id; o < it.count * kElemPerTile; o += kRecsEpi) {
                const int b = o / kElemPerTile, e = o - b * kElemPerTile;
                if (e < ne) a.out[(long long)a.blist[it.start + b] * a.n_el + el0 + e] = ostage[o];
            }
            epi_sync_or(false);   // the stage is read before the next tile's epilogue writes it
        }
    }
    __syncthreads();
    if (tid == 0 && s_fail) {
        atomicExch(a.err, 1);
        for (uint32_t i = 0; i < S; ++i)   // bounded drain of copies and MMAs in flight
            for (uint32_t par = 0; par < 2; ++par) {
                tc::mbar_wait(&full[i], par, 1 << 16);
                tc::mbar_wait(&empty[i], par, 1 << 16);
            }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_free_c<256>(tmem);
}

void configure_tc_recover_kernels() {
    MS_CUDA(cudaFuncSetAttribute(k_recover_tcs<MSTRESS_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    MS_CUDA(cudaFuncSetAttribute(k_recover_tcs<MSTRESS_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    MS_CUDA(
        cudaFuncSetAttribute(k_recover_tcs<MSTRESS_BF16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    MS_CUDA(cudaFuncSetAttribute(k_recover_tc<MSTRESS_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    MS_CUDA(cudaFuncSetAttribute(k_recover_tc<MSTRESS_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    MS_CUDA(
        cudaFuncSetAttribute(k_recover_tc<MSTRESS_BF16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
}

}  // namespace

bool tc_recover_supported(int m1, int prec) {
    return prec != MSTRESS_FP64 && (rec_shape(m1, 1, prec).stages >= 1 || recs_shape(m1, 1, prec).stages >= 2);
}

void build_tc_smean(mstress_block blk, int prec) {
    if (blk->Smean_tc[prec].ptr) return;
    if (rec_shape(blk->m1, blk->n_el, prec).stages < 1) {   // streamed layout, slot by slot
        RecsShape sh = recs_shape(blk->m1, blk->n_el, prec);
        alloc_into(blk->ctx, blk->Smean_tc[prec], (size_t)sh.n_etiles * sh.nks * sh.slot, true);
        const long long n = (long long)sh.n_etiles * 128 * sh.kpad;
        const unsigned g = (unsigned)((n + 255) / 256);
        const double* Sm = blk->Smean.as<double>();
        uint8_t* out = blk->Smean_tc[prec].as<uint8_t>();
        cudaStream_t st = blk->ctx->stream;
        switch (prec) {
            case MSTRESS_TF32: k_smean_image_s<MSTRESS_TF32><<<g, 256, 0, st>>>(Sm, blk->ld, blk->m1, blk->n_el, sh, out); break;
            case MSTRESS_BF16: k_smean_image_s<MSTRESS_BF16><<<g, 256, 0, st>>>(Sm, blk->ld, blk->m1, blk->n_el, sh, out); break;
            default: k_smean_image_s<MSTRESS_BF16X3><<<g, 256, 0, st>>>(Sm, blk->ld, blk->m1, blk->n_el, sh, out); break;
        }
        MS_LAUNCH_CHECK();
        return;
    }
    RecShape sh = rec_shape(blk->m1, blk->n_el, prec);
    alloc_into(blk->ctx, blk->Smean_tc[prec], (size_t)sh.n_etiles * sh.set, true);
    const long long n = (long long)sh.n_etiles * 128 * sh.kpad;
    const unsigned g = (unsigned)((n + 255) / 256);
    const double* Sm = blk->Smean.as<double>();
    uint8_t* out = blk->Smean_tc[prec].as<uint8_t>();
    cudaStream_t st = blk->ctx->stream;
    switch (prec) {
        case MSTRESS_TF32: k_smean_image<MSTRESS_TF32><<<g, 256, 0, st>>>(Sm, blk->ld, blk->m1, blk->n_el, sh, out); break;
        case MSTRESS_BF16: k_smean_image<MSTRESS_BF16><<<g, 256, 0, st>>>(Sm, blk->ld, blk->m1, blk->n_el, sh, out); break;
        default: k_smean_image<MSTRESS_BF16X3><<<g, 256, 0, st>>>(Sm, blk->ld, blk->m1, blk->n_el, sh, out); break;
    }
    MS_LAUNCH_CHECK();
}

// Streamed variant of recover_vm_tc for large bases.
void recover_vm_tcs(mstress_sol_s* s, float* out) {
    mstress_ctx ctx = s->ctx;
    const int prec = s->precision;
    RecsShape sh = recs_shape(s->types[0]->m1, s->n_el, prec);
    MS_REQUIRE(sh.stages >= 2, MSTRESS_EINVAL, "basis too large for the streamed recovery");
    const size_t cbytes = (size_t)s->n_awork_rec * sh.nks * sh.slot;
    if (s->cimg.bytes < cbytes) alloc_into(ctx, s->cimg, cbytes, false);
    ApplyArgs aa = apply_args(s, s->v64.x.ptr, nullptr, nullptr, nullptr, true);
    aa.work = s->d_awork_rec.as<ApplyWork>();
    aa.n_work = s->n_awork_rec;
    const int gi = std::max(1, std::min(s->n_awork_rec, ctx->num_sms * 8));
    uint8_t* cimg = s->cimg.as<uint8_t>();
    switch (prec) {
        case MSTRESS_TF32: k_coeff_image_s<MSTRESS_TF32><<<gi, 256, 0, ctx->stream>>>(aa, sh, cimg); break;
        case MSTRESS_BF16: k_coeff_image_s<MSTRESS_BF16><<<gi, 256, 0, ctx->stream>>>(aa, sh, cimg); break;
        default: k_coeff_image_s<MSTRESS_BF16X3><<<gi, 256, 0, ctx->stream>>>(aa, sh, cimg); break;
    }
    MS_LAUNCH_CHECK();
    RecTcArgs ra;
    std::memset(&ra, 0, sizeof(ra));
    ra.work = s->d_awork_rec.as<ApplyWork>();
    ra.n_work = s->n_awork_rec;
    ra.blist = s->d_blist.as<int>();
    ra.cimg = cimg;
    for (int t = 0; t < s->n_types; ++t) {
        build_tc_smean(s->types[t], prec);
        ra.simg[t] = s->types[t]->Smean_tc[prec].as<uint8_t>();
    }
    ra.n_el = s->n_el;
    ra.out = out;
    ra.err = s->flag.as<int>() + 2;
    const long long pairs = (long long)s->n_awork_rec * sh.n_etiles;
    const int grid = (int)std::max(1LL, std::min(pairs, (long long)ctx->num_sms));
    switch (prec) {
        case MSTRESS_TF32: k_recover_tcs<MSTRESS_TF32><<<grid, kRecsThreads, sh.smem, ctx->stream>>>(ra, sh); break;
        case MSTRESS_BF16: k_recover_tcs<MSTRESS_BF16><<<grid, kRecsThreads, sh.smem, ctx->stream>>>(ra, sh); break;
        default: k_recover_tcs<MSTRESS_BF16X3><<<grid, kRecsThreads, sh.smem, ctx->stream>>>(ra, sh); break;
    }
    MS_LAUNCH_CHECK();
}

// Von Mises of every element of every block into out (FP32, [block][n_el]).
void recover_vm_tc(mstress_sol_s* s, float* out) {
    mstress_ctx ctx = s->ctx;
    const int prec = s->precision;
    mstress_block t0 = s->types[0];
    RecShape sh = rec_shape(t0->m1, s->n_el, prec);
    static bool configured = false;
    if (!configured) {
        configure_tc_recover_kernels();
        configured = true;
    }
    if (sh.stages < 1) {
        recover_vm_tcs(s, out);
        return;
    }
    const size_t cbytes = (size_t)s->n_awork_rec * sh.set;
    if (s->cimg.bytes < cbytes) alloc_into(ctx, s->cimg, cbytes, false);   // kept with the solution
    ApplyArgs aa = apply_args(s, s->v64.x.ptr, nullptr, nullptr, nullptr, true);
    aa.work = s->d_awork_rec.as<ApplyWork>();   // 128-block tiles
    aa.n_work = s->n_awork_rec;
    const int gi = std::max(1, std::min(s->n_awork_rec, ctx->num_sms * 8));
    uint8_t* cimg = s->cimg.as<uint8_t>();
    switch (prec) {
        case MSTRESS_TF32: k_coeff_image<MSTRESS_TF32><<<gi, 256, 0, ctx->stream>>>(aa, sh, cimg); break;
        case MSTRESS_BF16: k_coeff_image<MSTRESS_BF16><<<gi, 256, 0, ctx->stream>>>(aa, sh, cimg); break;
        default: k_coeff_image<MSTRESS_BF16X3><<<gi, 256, 0, ctx->stream>>>(aa, sh, cimg); break;
    }
    MS_LAUNCH_CHECK();
    RecTcArgs ra;
    std::memset(&ra, 0, sizeof(ra));
    ra.work = s->d_awork_rec.as<ApplyWork>();
    ra.n_work = s->n_awork_rec;
    ra.blist = s->d_blist.as<int>();
    ra.cimg = cimg;
    for (int t = 0; t < s->n_types; ++t) {
        build_tc_smean(s->types[t], prec);
        ra.simg[t] = s->types[t]->Smean_tc[prec].as<uint8_t>();
    }
    ra.n_el = s->n_el;
    ra.out = out;
    ra.err = s->flag.as<int>() + 2;
    const long long pairs = (long long)s->n_awork_rec * sh.n_etiles;
    const int grid = (int)std::max(1LL, std::min(pairs, (long long)ctx->num_sms));
    switch (prec) {
        case MSTRESS_TF32: k_recover_tc<MSTRESS_TF32><<<grid, kRecThreads, sh.smem, ctx->stream>>>(ra, sh); break;
        case MSTRESS_BF16: k_recover_tc<MSTRESS_BF16><<<grid, kRecThreads, sh.smem, ctx->stream>>>(ra, sh); break;
        default: k_recover_tc<MSTRESS_BF16X3><<<grid, kRecThreads, sh.smem, ctx->stream>>>(ra, sh); break;
    }
    MS_LAUNCH_CHECK();
}

}  // namespace ms
