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
__global__ void k_coeff_image(const __grid_constant__ ApplyArgs a, RecShape sh, int split, uint8_t* out) {
    constexpr int ESZ = MODE == MSTRESS_TF32 ? 4 : 2;
    constexpr int LGKE = MODE == MSTRESS_TF32 ? 2 : 3;
    constexpr int U = 4;   // loads in flight per thread
    __shared__ long long base[kTileTC];
    __shared__ int offs[3 * kMaxSurf];
    const double* __restrict__ x = static_cast<const double*>(a.x);
    const uint32_t sbo = tc::sbo_bytes(sh.kpad, ESZ);
    const int total = sh.kpad * kTileTC;
    // CTA c of a tile's split CTAs takes the index range [c total / split, (c+1) total / split)
    for (int wc = blockIdx.x; wc < a.n_work * split; wc += gridDim.x) {
        const int w = wc / split, c = wc - w * split;
        const ApplyWork it = a.work[w];
        const ArrayDev A = a.arrays[it.array];
        __syncthreads();
        tile_setup(a, it, A, base, offs, kTileTC);
        __syncthreads();
        uint8_t* img = out + (size_t)w * sh.set;
        const int i0 = (int)((long long)total * c / split), i1 = (int)((long long)total * (c + 1) / split);
        for (int i = i0 + threadIdx.x; i < i1; i += U * blockDim.x) {
            double v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int idx = i + u * blockDim.x;
                const int kk = idx & ((1 << LGKE) - 1), b = (idx >> LGKE) & (kTileTC - 1), kg = idx >> (LGKE + 7);
                const int k = (kg << LGKE) + kk;
                v[u] = 0.0;
                if (idx < i1 && b < it.count && k < a.m) v[u] = x[base[b] + offs[k]];
                else if (idx < i1 && b < it.count && k == a.m) v[u] = A.dT;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int idx = i + u * blockDim.x;
                if (idx >= i1) break;
                const int kk = idx & ((1 << LGKE) - 1), b = (idx >> LGKE) & (kTileTC - 1), kg = idx >> (LGKE + 7);
                const uint32_t off = (uint32_t)(b >> 3) * sbo + (uint32_t)kg * 128u + (uint32_t)(b & 7) * 16u +
                                     (uint32_t)kk * ESZ;
                put<MODE>(img, sh.plane, off, v[u]);
            }
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
    int n_seg;                      // streamed recovery: element-tile segments per block tile
    float* out;                     // [block][n_el]
    int* err;
};

// The CTA is split in two roles: warp 0 (one thread) issues the bulk copies
// and the MMAs, warps 1-16 run the epilogue. The epilogue warps synchronise
// among themselves only (named barrier 1), so the MMAs of the next element tile
// never wait for the output stores of the previous one.
constexpr int kRecsEpiWarps = 16;                 // four per TMEM lane group
constexpr int kRecsEpi = 32 * kRecsEpiWarps;      // epilogue threads
constexpr int kRecsThreads = 32 + kRecsEpi;       // + the copy / MMA warp

__device__ __forceinline__ bool epi_sync_or(bool pred) {   // named barrier 1 over the epilogue warps
    uint32_t r;
    asm volatile(
        "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, 1, %2, p;\nselp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"((uint32_t)pred), "n"(kRecsEpi)
        : "memory");
    return r != 0;
}

// Von Mises of one epilogue thread's elements of an accumulated element tile.
// Its block is TMEM lane 32 lg + lane (tl addresses the lane group and the
// accumulator); the four epilogue warps of a lane group split the 21 elements
// as 0-4, 5-9, 10-15, 16-20 (columns 0-29, 30-59, 60-95, 96-125, read in
// 16-column groups starting at C0). All TMEM reads are issued before one wait.
template <int C0, int N16, int E0, int E1>
__device__ __forceinline__ void epi_part(uint32_t tl, float* orow) {
    uint32_t r[N16][16];
#pragma unroll
    for (int c = 0; c < N16; ++c) tc::tmem_ld16_nw(tl + (uint32_t)(C0 + 16 * c), r[c]);
#pragma unroll
    for (int c = 0; c < N16; ++c) tc::tmem_wait16(r[c]);
    float v[16 * N16];
#pragma unroll
    for (int c = 0; c < 16 * N16; ++c) v[c] = __uint_as_float(r[c >> 4][c & 15]);
#pragma unroll
    for (int e = E0; e < E1; ++e) orow[e] = von_mises6(v + 6 * e - C0);
}

__device__ __forceinline__ void epi_vm(uint32_t tl, int part, float* orow) {
    switch (part) {
        case 0: epi_part<0, 2, 0, 5>(tl, orow); break;
        case 1: epi_part<16, 3, 5, 10>(tl, orow); break;
        case 2: epi_part<48, 3, 10, 16>(tl, orow); break;
        default: epi_part<96, 2, 16, kElemPerTile>(tl, orow); break;
    }
}

// Epilogue state across tiles: the block tile being written, its block count,
// and which of the two row-offset buffers holds its output rows.
struct EpiRows {
    int bt = -1, count = 0, buf = 1;
};

// Called by every epilogue thread (t = 0..kRecsEpi-1) before the tile's
// barrier: on a new block tile, fill the other row-offset buffer (the one
// used two block tiles ago; every thread passed a barrier since its last use).
__device__ __forceinline__ void epi_rows(const RecTcArgs& a, int bt, int t, long long (*rowoff)[kTileTC],
                                         EpiRows& er) {
    if (bt == er.bt) return;
    const ApplyWork it = a.work[bt];
    er.bt = bt;
    er.count = it.count;
    er.buf ^= 1;
    if (t < kTileTC) rowoff[er.buf][t] = t < it.count ? (long long)a.blist[it.start + t] * a.n_el : 0;
}

// Output of one element tile from its staging buffer, after the tile's
// barrier: runs of up to 21 consecutive elements per block, consecutive
// threads on consecutive elements; all staging reads before the stores.
__device__ __forceinline__ void epi_store(const RecTcArgs& a, const EpiRows& er, const long long* rowoff, int et,
                                          const float* os, int t) {
    constexpr int kIt = (kTileTC * kElemPerTile + kRecsEpi - 1) / kRecsEpi;
    const int el0 = et * kElemPerTile;
    const int ne = min(kElemPerTile, a.n_el - el0);
    const int n = er.count * kElemPerTile;
    float v[kIt];
    long long ad[kIt];
#pragma unroll
    for (int i = 0; i < kIt; ++i) {
        const int o = t + i * kRecsEpi;
        const int b = o / kElemPerTile, e = o - b * kElemPerTile;
        ad[i] = -1;
        if (o < n && e < ne) {
            v[i] = os[o];
            ad[i] = rowoff[b] + el0 + e;
        }
    }
#pragma unroll
    for (int i = 0; i < kIt; ++i)
        if (ad[i] >= 0) a.out[ad[i]] = v[i];
}

template <int MODE>
__global__ void __launch_bounds__(kRecsThreads, 1) k_recover_tc(const __grid_constant__ RecTcArgs a,
                                                                 const RecShape sh) {
    constexpr bool TF32 = MODE == MSTRESS_TF32;
    constexpr int NS = MODE == MSTRESS_BF16X3 ? 2 : 1;
    constexpr int kTries = 1 << 24;
    extern __shared__ uint8_t smraw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    uint8_t* sB = smem;              // coefficients of the current block tile
    uint8_t* sA0 = smem + sh.set;    // S_mean tile stages
    __shared__ __align__(8) uint64_t bfull, bempty, afull[kMaxStages], aempty[kMaxStages], accfull[2], accempty[2];
    __shared__ uint32_t tmem_base;
    __shared__ float ostage[2][kTileTC * kElemPerTile];   // von Mises of an element tile, [block][element]
    __shared__ long long rowoff[2][kTileTC];               // output row offsets of the block tile's blocks
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t S = (uint32_t)sh.stages;
    if (warp == 0) tc::tmem_alloc_c<256>(&tmem_base);
    if (tid == 0) {
        tc::mbar_init(&bfull, 1);
        tc::mbar_init(&bempty, 1);
        for (uint32_t i = 0; i < S; ++i) {
            tc::mbar_init(&afull[i], 1);
            tc::mbar_init(&aempty[i], 1);
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
    // this CTA's share of the (block tile, element tile) pairs, in block-tile
    // major order: a contiguous range, so every CTA gets the same number of
    // element tiles (+-1) and at most a few coefficient tiles
    const long long n_pairs = (long long)a.n_work * sh.n_etiles;
    const long long p0 = n_pairs * blockIdx.x / gridDim.x, p1 = n_pairs * (blockIdx.x + 1) / gridDim.x;
    const uint32_t n_tiles = (uint32_t)(p1 - p0);
    if (warp == 0) {
        if (lane == 0) {
            auto issue = [&](uint32_t g) {   // the S_mean tile of pair p0 + g into stage g % S
                const long long pr = p0 + g;
                const int bt = (int)(pr / sh.n_etiles), et = (int)(pr - (long long)bt * sh.n_etiles);
                const uint32_t st = g % S;
                tc::mbar_expect_tx(&afull[st], sh.set);
                tc::bulk_g2s(sA0 + (size_t)st * sh.set, a.simg[a.work[bt].type] + (size_t)et * sh.set, sh.set,
                             &afull[st]);
            };
            const uint32_t idesc = tc::instr_desc(TF32, 128, 128);
            const uint32_t sbo = tc::sbo_bytes(sh.kpad, sh.esz);
            bool ok = true;
            uint32_t items = 0;   // coefficient tiles loaded
            for (uint32_t g = 0; g < S && g < n_tiles; ++g) issue(g);
            int cur_bt = -1;
            for (uint32_t g = 0; g < n_tiles && ok; ++g) {
                const int bt = (int)((p0 + g) / sh.n_etiles);
                const uint32_t j = g & 1u, st = g % S;
                if (bt != cur_bt) {
                    // the previous block tile's MMAs have completed before its coefficients are replaced
                    if (items > 0) ok = tc::mbar_wait(&bempty, (items - 1) & 1u, kTries);
                    if (!ok) break;
                    tc::mbar_expect_tx(&bfull, sh.set);
                    tc::bulk_g2s(sB, a.cimg + (size_t)bt * sh.set, sh.set, &bfull);
                    ok = tc::mbar_wait(&bfull, items & 1u, kTries);
                    ++items;
                    cur_bt = bt;
                    if (!ok) break;
                }
                if (g >= 2) ok = tc::mbar_wait(&accempty[j], ((g >> 1) - 1) & 1u, kTries);
                if (ok) ok = tc::mbar_wait(&afull[st], (g / S) & 1u, kTries);
                tc::fence_after();
                if (!ok) break;
                const uint32_t a0 = tc::smem_addr(sA0 + (size_t)st * sh.set), b0 = tc::smem_addr(sB);
                for (int ks = 0; ks < sh.ksteps; ++ks) {
                    const uint32_t ko = (uint32_t)ks * 2 * tc::kLBO;
#pragma unroll
                    for (int pr = 0; pr < (NS == 2 ? 3 : 1); ++pr) {
                        const uint32_t pa = pr == 1 ? sh.plane : 0u, pb = pr == 2 ? sh.plane : 0u;
                        // M = blocks (coefficients), N = S_mean rows
                        tc::mma<TF32>(tmem + 128u * j, tc::smem_desc(b0 + pb + ko, tc::kLBO, sbo),
                                      tc::smem_desc(a0 + pa + ko, tc::kLBO, sbo), idesc,
                                      (ks > 0 || pr > 0) ? 1u : 0u);
                    }
                }
                tc::commit(&accfull[j]);
                tc::commit(&aempty[st]);
                if (g + 1 == n_tiles || (int)((p0 + g + 1) / sh.n_etiles) != bt) tc::commit(&bempty);
                if (S == 1) {
                    // a single stage: this tile's MMAs finish before the next tile is fetched
                    if (g + 1 < n_tiles) {
                        ok = tc::mbar_wait(&aempty[0], g & 1u, kTries);
                        if (ok) issue(g + 1);
                    }
                } else if (g >= 1 && g - 1 + S < n_tiles) {
                    // refill the previous tile's stage (its MMAs have had a tile's time)
                    const uint32_t sp = (g - 1) % S;
                    ok = tc::mbar_wait(&aempty[sp], ((g - 1) / S) & 1u, kTries);
                    if (ok) issue(g - 1 + S);
                }
            }
            if (!ok) *(volatile int*)&s_fail = 1;
        }
    } else {
        // ---------------- epilogue: blocks on TMEM lanes, one element tile at a time
        const int t = tid - 32;                            // 0..kRecsEpi-1
        const int lg = warp & 3, part = (warp - 1) >> 2;   // lane group, element part
        const int bl = 32 * lg + lane;
        EpiRows er;
        for (uint32_t g = 0; g < n_tiles; ++g) {
            const uint32_t j = g & 1u;
            const long long pr = p0 + g;
            const int bt = (int)(pr / sh.n_etiles), et = (int)(pr - (long long)bt * sh.n_etiles);
            epi_rows(a, bt, t, rowoff, er);
            bool got = !*(volatile int*)&s_fail && tc::mbar_wait(&accfull[j], (g >> 1) & 1u, kTries);
            got = __all_sync(0xffffffffu, got);   // the TMEM reads are warp-collective
            tc::fence_after();
            float* os = ostage[j];
            if (got) epi_vm(tmem + ((uint32_t)(32 * lg) << 16) + 128u * j, part, os + bl * kElemPerTile);
            else *(volatile int*)&s_fail = 1;
            tc::fence_before();
            tc::mbar_arrive(&accempty[j]);
            // one barrier per tile: the stages alternate, and a thread writes stage j
            // again only after every thread has passed the next tile's barrier
            if (epi_sync_or(!got)) break;
            epi_store(a, er, rowoff[er.buf], et, os, t);
        }
    }
    __syncthreads();
    if (tid == 0 && s_fail) {
        atomicExch(a.err, 1);
        // bounded drain: let issued copies and MMAs finish before the CTA leaves
        for (uint32_t par = 0; par < 2; ++par) {
            tc::mbar_wait(&bfull, par, 1 << 16);
            tc::mbar_wait(&bempty, par, 1 << 16);
            for (uint32_t i = 0; i < S; ++i) {
                tc::mbar_wait(&afull[i], par, 1 << 16);
                tc::mbar_wait(&aempty[i], par, 1 << 16);
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_free_c<256>(tmem);
}

// ----------------------------------------------------------- streamed K
// Large bases (the coefficient tile does not fit in shared memory next to an
// S_mean stage): both operands stream along K in slots of kc values (128 bytes
// of K per row, four MMA K steps). Both images are stored slot by slot (per
// tile, per slot, per plane a 128 x kc K-major block in the 128-byte swizzled
// layout, which the tensor cores read without shared-memory bank conflicts),
// so that one slot of each operand is one bulk copy. The CTA is split in two roles: warp 0
// (one thread) issues the copies and the MMAs, warps 1-16 run the epilogue.
// Barriers: full[s] (both copies' bytes), empty[s] (tcgen05.commit after the
// slot's MMAs), accfull[j] (commit after an element tile's last slot) and
// accempty[j] (the epilogue threads arrive when the accumulator is read).
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
    s.kc = 128 / s.esz;                      // one 128-byte swizzle row of K per slot
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
// Byte offset of slot ks of tile t in a slot-by-slot image, and of element
// (row, kk) within one plane of a slot (128-byte swizzled K-major).
__device__ __forceinline__ size_t slot_base(const RecsShape& sh, long long t, int ks) {
    return ((size_t)t * sh.nks + ks) * sh.slot;
}
__device__ __forceinline__ uint32_t in_slot(const RecsShape& sh, int row, int kk) {
    return tc::sw128_offset(row, kk * sh.esz);
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
    put<MODE>(out + slot_base(sh, tile, k / sh.kc), sh.plane, in_slot(sh, r, k % sh.kc), v);
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
        constexpr int U = 4;   // loads in flight per thread
        for (int i = threadIdx.x; i < total; i += U * blockDim.x) {
            double v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int idx = i + u * blockDim.x;
                const int b = idx / sh.kpad, k = idx - b * sh.kpad;   // consecutive threads: one row's K values
                v[u] = 0.0;
                if (idx < total && b < it.count && k < a.m) v[u] = x[base[b] + offs[k]];
                else if (idx < total && b < it.count && k == a.m) v[u] = A.dT;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int idx = i + u * blockDim.x;
                if (idx >= total) break;
                const int b = idx / sh.kpad, k = idx - b * sh.kpad;
                put<MODE>(out + slot_base(sh, w, k / sh.kc), sh.plane, in_slot(sh, b, k % sh.kc), v[u]);
            }
        }
    }
}

// Tile order of the streamed recovery. The units are (block tile, segment of
// the element tiles), u = bt * n_seg + seg; CTA c takes units c, c + G, c + 2G,
// ... (G CTAs) and sweeps each unit's element tiles in order. The CTAs of one
// round thus walk the same S_mean tiles at about the same time, so a tile
// comes from DRAM once per round and from L2 for the others, and each CTA's
// coefficient tile stays in L2 for a whole sweep. n_seg > 1 only when there are
// too few block tiles to keep every CTA busy.
struct UnitCursor {
    long long u;
    int bt, e, e1;
    __device__ __forceinline__ void begin(long long u_, int n_seg, int n_et) {
        u = u_;
        bt = (int)(u / n_seg);
        const int sg = (int)(u - (long long)bt * n_seg);
        e = (int)((long long)n_et * sg / n_seg);
        e1 = (int)((long long)n_et * (sg + 1) / n_seg);
    }
    __device__ __forceinline__ void next(int n_seg, int n_et) {
        if (++e >= e1) begin(u + gridDim.x, n_seg, n_et);
    }
};

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
    __shared__ float ostage[2][kTileTC * kElemPerTile];
    __shared__ long long rowoff[2][kTileTC];
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
    // this CTA's element tiles, unit by unit (UnitCursor)
    const int n_seg = a.n_seg;
    const long long n_units = (long long)a.n_work * n_seg;
    uint32_t n_tiles = 0;
    for (long long u = blockIdx.x; u < n_units; u += gridDim.x) {
        const int sg = (int)(u % n_seg);
        n_tiles += (uint32_t)((long long)sh.n_etiles * (sg + 1) / n_seg - (long long)sh.n_etiles * sg / n_seg);
    }
    const uint32_t n_slots = n_tiles * (uint32_t)sh.nks;
    if (warp == 0) {
        if (lane == 0) {
            // the copies of slot q = tile q / nks, K slot q % nks (issued in increasing q)
            UnitCursor ic;
            ic.begin(blockIdx.x, n_seg, sh.n_etiles);
            auto issue = [&](uint32_t q) {
                const int ks = (int)(q % sh.nks);
                if (ks == 0 && q > 0) ic.next(n_seg, sh.n_etiles);
                const int bt = ic.bt, et = ic.e;
                const uint32_t s = q % S;
                uint8_t* dst = smem + (size_t)s * 2 * sh.slot;
                tc::mbar_expect_tx(&full[s], 2 * sh.slot);
                tc::bulk_g2s(dst, a.simg[a.work[bt].type] + ((size_t)et * sh.nks + ks) * sh.slot, sh.slot, &full[s]);
                tc::bulk_g2s(dst + sh.slot, a.cimg + ((size_t)bt * sh.nks + ks) * sh.slot, sh.slot, &full[s]);
            };
            const uint32_t idesc = tc::instr_desc(TF32, 128, 128);

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
                    for (int kj = 0; kj < 4; ++kj) {   // four 32-byte K steps per 128-byte row
                        const uint32_t ko = (uint32_t)kj * 32u;
#pragma unroll
                        for (int pr = 0; pr < (NS == 2 ? 3 : 1); ++pr) {
                            const uint32_t pa = pr == 1 ? sh.plane : 0u, pb = pr == 2 ? sh.plane : 0u;
                            const uint32_t acc = (ks > 0 || kj > 0 || pr > 0) ? 1u : 0u;
                            // M = blocks (coefficients), N = S_mean rows
                            tc::mma<TF32>(tmem + 128u * j, tc::smem_desc_sw128(b0 + pb + ko),
                                          tc::smem_desc_sw128(a0 + pa + ko), idesc, acc);
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
        const int t = tid - 32;                            // 0..kRecsEpi-1
        const int lg = warp & 3, part = (warp - 1) >> 2;   // lane group, element part
        const int bl = 32 * lg + lane;
        UnitCursor ec;
        ec.begin(blockIdx.x, n_seg, sh.n_etiles);
        EpiRows er;
        for (uint32_t g = 0; g < n_tiles; ++g) {
            const uint32_t j = g & 1u;
            if (g > 0) ec.next(n_seg, sh.n_etiles);
            const int bt = ec.bt, et = ec.e;
            epi_rows(a, bt, t, rowoff, er);
            bool got = !*(volatile int*)&s_fail && tc::mbar_wait(&accfull[j], (g >> 1) & 1u, kTries);
            got = __all_sync(0xffffffffu, got);   // the TMEM reads are warp-collective
            tc::fence_after();
            float* os = ostage[j];
            if (got) epi_vm(tmem + ((uint32_t)(32 * lg) << 16) + 128u * j, part, os + bl * kElemPerTile);
            else *(volatile int*)&s_fail = 1;
            tc::fence_before();
            tc::mbar_arrive(&accempty[j]);
            // one barrier per tile (alternating stages, as in k_recover_tc)
            if (epi_sync_or(!got)) break;
            epi_store(a, er, rowoff[er.buf], et, os, t);
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

// Tensor-core image of a block's von Mises mode matrix: the Gauss-mean
// stress modes (per-element output) or, with grid, the cut-plane grid modes.
void build_tc_smean(mstress_block blk, int prec, bool grid) {
    ms::DBuf& img = grid ? blk->Sgrid_tc[prec] : blk->Smean_tc[prec];
    if (img.ptr) return;
    const int n_pts = grid ? blk->n_grid : blk->n_el;
    const double* Sm = grid ? blk->Sgrid.as<double>() : blk->Smean.as<double>();
    cudaStream_t st = blk->ctx->stream;
    if (rec_shape(blk->m1, n_pts, prec).stages < 1) {   // streamed layout, slot by slot
        RecsShape sh = recs_shape(blk->m1, n_pts, prec);
        alloc_into(blk->ctx, img, (size_t)sh.n_etiles * sh.nks * sh.slot, true);
        const long long n = (long long)sh.n_etiles * 128 * sh.kpad;
        const unsigned g = (unsigned)((n + 255) / 256);
        uint8_t* out = img.as<uint8_t>();
        switch (prec) {
            case MSTRESS_TF32: k_smean_image_s<MSTRESS_TF32><<<g, 256, 0, st>>>(Sm, blk->ld, blk->m1, n_pts, sh, out); break;
            case MSTRESS_BF16: k_smean_image_s<MSTRESS_BF16><<<g, 256, 0, st>>>(Sm, blk->ld, blk->m1, n_pts, sh, out); break;
            default: k_smean_image_s<MSTRESS_BF16X3><<<g, 256, 0, st>>>(Sm, blk->ld, blk->m1, n_pts, sh, out); break;
        }
        MS_LAUNCH_CHECK();
        return;
    }
    RecShape sh = rec_shape(blk->m1, n_pts, prec);
    alloc_into(blk->ctx, img, (size_t)sh.n_etiles * sh.set, true);
    const long long n = (long long)sh.n_etiles * 128 * sh.kpad;
    const unsigned g = (unsigned)((n + 255) / 256);
    uint8_t* out = img.as<uint8_t>();
    switch (prec) {
        case MSTRESS_TF32: k_smean_image<MSTRESS_TF32><<<g, 256, 0, st>>>(Sm, blk->ld, blk->m1, n_pts, sh, out); break;
        case MSTRESS_BF16: k_smean_image<MSTRESS_BF16><<<g, 256, 0, st>>>(Sm, blk->ld, blk->m1, n_pts, sh, out); break;
        default: k_smean_image<MSTRESS_BF16X3><<<g, 256, 0, st>>>(Sm, blk->ld, blk->m1, n_pts, sh, out); break;
    }
    MS_LAUNCH_CHECK();
}

// Streamed variant of recover_vm_tc for large bases.
void recover_vm_tcs(mstress_sol_s* s, float* out, bool grid) {
    mstress_ctx ctx = s->ctx;
    const int prec = s->precision;
    const int n_pts = grid ? s->types[0]->n_grid : s->n_el;
    RecsShape sh = recs_shape(s->types[0]->m1, n_pts, prec);
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
        build_tc_smean(s->types[t], prec, grid);
        ra.simg[t] = (grid ? s->types[t]->Sgrid_tc[prec] : s->types[t]->Smean_tc[prec]).as<uint8_t>();
    }
    ra.n_el = n_pts;
    ra.out = out;
    ra.err = s->flag.as<int>() + 2;
    const long long pairs = (long long)s->n_awork_rec * sh.n_etiles;
    const int ncta = (int)std::max(1LL, std::min(pairs, (long long)ctx->num_sms));
    // about eight units per CTA at least, so that the last round is nearly full
    ra.n_seg = (int)std::max(1LL, std::min((long long)sh.n_etiles,
                                           (8LL * ncta + s->n_awork_rec - 1) / std::max(1, s->n_awork_rec)));
    switch (prec) {
        case MSTRESS_TF32: k_recover_tcs<MSTRESS_TF32><<<ncta, kRecsThreads, sh.smem, ctx->stream>>>(ra, sh); break;
        case MSTRESS_BF16: k_recover_tcs<MSTRESS_BF16><<<ncta, kRecsThreads, sh.smem, ctx->stream>>>(ra, sh); break;
        default: k_recover_tcs<MSTRESS_BF16X3><<<ncta, kRecsThreads, sh.smem, ctx->stream>>>(ra, sh); break;
    }
    MS_LAUNCH_CHECK();
}

// Von Mises of every element of every block into out (FP32, [block][n_el]),
// or, with grid, of every cut-plane grid point ([block][n_grid]).
void recover_vm_tc(mstress_sol_s* s, float* out, bool grid) {
    mstress_ctx ctx = s->ctx;
    const int prec = s->precision;
    mstress_block t0 = s->types[0];
    const int n_pts = grid ? t0->n_grid : s->n_el;
    RecShape sh = rec_shape(t0->m1, n_pts, prec);
    static bool configured = false;
    if (!configured) {
        configure_tc_recover_kernels();
        configured = true;
    }
    if (sh.stages < 1) {
        recover_vm_tcs(s, out, grid);
        return;
    }
    const size_t cbytes = (size_t)s->n_awork_rec * sh.set;
    if (s->cimg.bytes < cbytes) alloc_into(ctx, s->cimg, cbytes, false);   // kept with the solution
    ApplyArgs aa = apply_args(s, s->v64.x.ptr, nullptr, nullptr, nullptr, true);
    aa.work = s->d_awork_rec.as<ApplyWork>();   // 128-block tiles
    aa.n_work = s->n_awork_rec;
    // a few CTAs per tile when there are few tiles, so that every SM gathers
    const int split = std::max(1, std::min(8, (4 * ctx->num_sms + s->n_awork_rec - 1) / std::max(1, s->n_awork_rec)));
    const int gi = std::max(1, std::min(s->n_awork_rec * split, ctx->num_sms * 8));
    uint8_t* cimg = s->cimg.as<uint8_t>();
    switch (prec) {
        case MSTRESS_TF32: k_coeff_image<MSTRESS_TF32><<<gi, 256, 0, ctx->stream>>>(aa, sh, split, cimg); break;
        case MSTRESS_BF16: k_coeff_image<MSTRESS_BF16><<<gi, 256, 0, ctx->stream>>>(aa, sh, split, cimg); break;
        default: k_coeff_image<MSTRESS_BF16X3><<<gi, 256, 0, ctx->stream>>>(aa, sh, split, cimg); break;
    }
    MS_LAUNCH_CHECK();
    RecTcArgs ra;
    std::memset(&ra, 0, sizeof(ra));
    ra.work = s->d_awork_rec.as<ApplyWork>();
    ra.n_work = s->n_awork_rec;
    ra.blist = s->d_blist.as<int>();
    ra.cimg = cimg;
    for (int t = 0; t < s->n_types; ++t) {
        build_tc_smean(s->types[t], prec, grid);
        ra.simg[t] = (grid ? s->types[t]->Sgrid_tc[prec] : s->types[t]->Smean_tc[prec]).as<uint8_t>();
    }
    ra.n_el = n_pts;
    ra.out = out;
    ra.err = s->flag.as<int>() + 2;
    const long long pairs = (long long)s->n_awork_rec * sh.n_etiles;
    const int ncta = (int)std::max(1LL, std::min(pairs, (long long)ctx->num_sms));
    switch (prec) {
        case MSTRESS_TF32: k_recover_tc<MSTRESS_TF32><<<ncta, kRecsThreads, sh.smem, ctx->stream>>>(ra, sh); break;
        case MSTRESS_BF16: k_recover_tc<MSTRESS_BF16><<<ncta, kRecsThreads, sh.smem, ctx->stream>>>(ra, sh); break;
        default: k_recover_tc<MSTRESS_BF16X3><<<ncta, kRecsThreads, sh.smem, ctx->stream>>>(ra, sh); break;
    }
    MS_LAUNCH_CHECK();
}

}  // namespace ms
