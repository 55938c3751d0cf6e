// Per-element von Mises recovery on the tensor cores (tcgen05, sm_103a).
//
// For the blocks of one type, Sigma_mean = S_mean [c_e; dT] (Eq. 15 and Eq. 1,
// averaged over the 8 Gauss points of each element) is one dense contraction
//     D (rows x blocks) = S_mean (rows x K) * C^T,   K = m + 1 (padded)
// where each 128-row tile of S_mean holds the 6 stress components of 21
// elements (row = 6 * element + component, rows 126-127 zero) and C holds the
// gathered element DOFs of 128 blocks plus the dT column. The MMA is issued by
// one thread from shared-memory operands (K-major, no swizzle), the FP32
// accumulator sits in tensor memory (128 lanes x 128 columns), and the
// epilogue stages 16 block columns at a time through shared memory so that one
// thread can take the von Mises of an element's 6 components.
//
// Operand images: the S_mean tile images are built once per block model; the
// coefficient images (one per 128-block tile) are built by a gather kernel at
// every recovery. Both are copied into shared memory with 16-byte loads.
#include "solve.h"
#include "tc.cuh"

namespace ms {
namespace {

constexpr int kRecThreads = 128;
constexpr int kElemPerTile = 21;     // 21 elements x 6 components = 126 rows of 128
constexpr int kTilesPerItem = 8;     // element tiles per work item (coefficients reused)

struct RecShape {
    int m1, esz, kpad, ksteps, ns, n_etiles;
    uint32_t plane;                  // bytes of one 128 x kpad operand plane
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
    s.smem = (size_t)2 * s.ns * s.plane + 128 * 17 * sizeof(float) + 1024;
    return s;
}

__device__ __forceinline__ void put(uint8_t* p0, uint32_t plane, uint32_t off, double v, int mode) {
    if (mode == MSTRESS_TF32) {
        *reinterpret_cast<float*>(p0 + off) = tc::to_tf32((float)v);
    } else {
        __nv_bfloat16 hi = __float2bfloat16_rn((float)v);
        *reinterpret_cast<__nv_bfloat16*>(p0 + off) = hi;
        if (mode == MSTRESS_BF16X3)
            *reinterpret_cast<__nv_bfloat16*>(p0 + plane + off) =
                __float2bfloat16_rn((float)(v - (double)__bfloat162float(hi)));
    }
}

// S_mean tile images of one block model: tile t, row r = 6 * le + c holds
// S_mean[(21 t + le) * 6 + c][k] (zero beyond the last element and for k >= m+1).
__global__ void k_smean_image(const double* Smean, int ld, int m1, int n_el, RecShape sh, int mode, uint8_t* out) {
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
    uint8_t* base = out + (size_t)tile * sh.ns * sh.plane;
    put(base, sh.plane, tc::operand_offset(r, k, sh.kpad, sh.esz), v, mode);
}

// Coefficient images, one per 128-block tile: row b = block, column k < m is
// the element DOF c_e[k] gathered from the lattice solution, column m is dT.
__global__ void k_coeff_image(const __grid_constant__ ApplyArgs a, RecShape sh, int mode, uint8_t* out) {
    __shared__ long long base[kTileTC];
    __shared__ int offs[3 * kMaxSurf];
    const double* __restrict__ x = static_cast<const double*>(a.x);
    for (int w = blockIdx.x; w < a.n_work; w += gridDim.x) {
        const ApplyWork it = a.work[w];
        const ArrayDev A = a.arrays[it.array];
        __syncthreads();
        tile_setup(a, it, A, base, offs, kTileTC);
        __syncthreads();
        uint8_t* img = out + (size_t)w * sh.ns * sh.plane;
        for (int idx = threadIdx.x; idx < sh.kpad * kTileTC; idx += blockDim.x) {
            const int k = idx >> 7, b = idx & (kTileTC - 1);
            double v = 0.0;
            if (b < it.count && k < a.m) v = x[base[b] + offs[k]];
            else if (b < it.count && k == a.m) v = A.dT;
            put(img, sh.plane, tc::operand_offset(b, k, sh.kpad, sh.esz), v, mode);
        }
    }
}

struct RecTcArgs {
    const ApplyWork* work;          // 128-block tiles (one type, one array)
    int n_work;
    const int* blist;
    const uint8_t* cimg;            // coefficient images, one per tile
    const uint8_t* simg[kMaxTypes]; // S_mean tile images per type
    int n_el;
    float* out;                     // [block][n_el]
    int* err;
};

template <int MODE>
__global__ void __launch_bounds__(kRecThreads) k_recover_tc(const __grid_constant__ RecTcArgs a, const RecShape sh) {
    constexpr bool TF32 = MODE == MSTRESS_TF32;
    constexpr int NS = MODE == MSTRESS_BF16X3 ? 2 : 1;
    extern __shared__ uint8_t smraw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;                          // NS planes: S_mean tile
    uint8_t* sB = smem + NS * sh.plane;          // NS planes: coefficients of 128 blocks
    float* stage = reinterpret_cast<float*>(smem + 2 * NS * sh.plane);   // [128 rows][17]
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ long long eidx[kTileTC];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(&tmem_base, 128);
    if (tid == 0) tc::mbar_init(&mbar, 1);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = tc::instr_desc(TF32, 128, 128);
    const uint32_t sbo = tc::sbo_bytes(sh.kpad, sh.esz);
    const int chunks = (sh.n_etiles + kTilesPerItem - 1) / kTilesPerItem;
    uint32_t phase = 0;
    bool failed = false;
    for (int w = blockIdx.x; w < a.n_work * chunks && !failed; w += gridDim.x) {
        const int tw = w / chunks, chunk = w % chunks;
        const ApplyWork it = a.work[tw];
        // coefficient image of this block tile
        const uint4* src = reinterpret_cast<const uint4*>(a.cimg + (size_t)tw * NS * sh.plane);
        for (uint32_t i = tid; i < NS * sh.plane / 16; i += kRecThreads) reinterpret_cast<uint4*>(sB)[i] = src[i];
        eidx[tid] = tid < it.count ? (long long)a.blist[it.start + tid] : -1;
        const int t_end = min(sh.n_etiles, (chunk + 1) * kTilesPerItem);
        for (int et = chunk * kTilesPerItem; et < t_end; ++et) {
            const uint4* sa = reinterpret_cast<const uint4*>(a.simg[it.type] + (size_t)et * NS * sh.plane);
            for (uint32_t i = tid; i < NS * sh.plane / 16; i += kRecThreads) reinterpret_cast<uint4*>(sA)[i] = sa[i];
            tc::fence_smem_async();
            tc::fence_before();
            __syncthreads();
            tc::fence_after();
            if (tid == 0) {
                const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB);
                uint32_t acc = 0;
                for (int s = 0; s < sh.ksteps; ++s) {
                    const uint32_t ko = (uint32_t)s * 2 * tc::kLBO;
#pragma unroll
                    for (int pr = 0; pr < (NS == 2 ? 3 : 1); ++pr) {
                        const uint32_t pa = pr == 1 ? sh.plane : 0u, pb = pr == 2 ? sh.plane : 0u;
                        tc::mma<TF32>(tmem, tc::smem_desc(a0 + pa + ko, tc::kLBO, sbo),
                                      tc::smem_desc(b0 + pb + ko, tc::kLBO, sbo), idesc, acc);
                        acc = 1;
                    }
                }
                tc::commit(&mbar);
            }
            const bool ok = tc::mbar_wait(&mbar, phase, 1 << 24);
            phase ^= 1u;
            tc::fence_after();
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            // epilogue: 16 block columns at a time through shared memory
            for (int c0 = 0; c0 < 128; c0 += 16) {
                float v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
                const int row = warp * 32 + lane;
#pragma unroll
                for (int j = 0; j < 16; ++j) stage[row * 17 + j] = v[j];
                __syncthreads();
                for (int o = tid; o < kElemPerTile * 16; o += kRecThreads) {
                    const int le = o % kElemPerTile, j = o / kElemPerTile;
                    const int el = et * kElemPerTile + le;
                    const long long e = eidx[c0 + j];
                    if (e >= 0 && el < a.n_el) {
                        const float* s6 = stage + (6 * le) * 17 + j;
                        float d0 = s6[0] - s6[17], d1 = s6[17] - s6[34], d2 = s6[34] - s6[0];
                        float vm = sqrtf(0.5f * (d0 * d0 + d1 * d1 + d2 * d2) +
                                         3.0f * (s6[51] * s6[51] + s6[68] * s6[68] + s6[85] * s6[85]));
                        a.out[e * a.n_el + el] = vm;
                    }
                }
                __syncthreads();
            }
            tc::fence_before();
            __syncthreads();
            tc::fence_after();
        }
    }
    if (failed) {
        if (tid == 0) atomicExch(a.err, 1);
        tc::mbar_wait(&mbar, phase ^ 1u, 1 << 20);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, 128);
}

}  // namespace

bool tc_recover_supported(int m1, int prec) {
    return prec != MSTRESS_FP64 && rec_shape(m1, 1, prec).smem <= 200 * 1024;
}

void configure_tc_recover_kernels() {
    MS_CUDA(cudaFuncSetAttribute(k_recover_tc<MSTRESS_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    MS_CUDA(cudaFuncSetAttribute(k_recover_tc<MSTRESS_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    MS_CUDA(
        cudaFuncSetAttribute(k_recover_tc<MSTRESS_BF16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
}

void build_tc_smean(mstress_block blk, int prec) {
    if (blk->Smean_tc[prec].ptr) return;
    RecShape sh = rec_shape(blk->m1, blk->n_el, prec);
    alloc_into(blk->ctx, blk->Smean_tc[prec], (size_t)sh.n_etiles * sh.ns * sh.plane, true);
    long long n = (long long)sh.n_etiles * 128 * sh.kpad;
    k_smean_image<<<(unsigned)((n + 255) / 256), 256, 0, blk->ctx->stream>>>(
        blk->Smean.as<double>(), blk->ld, blk->m1, blk->n_el, sh, prec, blk->Smean_tc[prec].as<uint8_t>());
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
    DBuf cimg;
    alloc_into(ctx, cimg, (size_t)s->n_awork_rec * sh.ns * sh.plane, true);
    ApplyArgs aa = apply_args(s, s->v64.x.ptr, nullptr, nullptr, nullptr, true);
    aa.work = s->d_awork_rec.as<ApplyWork>();   // 128-block tiles
    aa.n_work = s->n_awork_rec;
    k_coeff_image<<<std::max(1, std::min(s->n_awork_rec, ctx->num_sms * 8)), 256, 0, ctx->stream>>>(
        aa, sh, prec, cimg.as<uint8_t>());
    MS_LAUNCH_CHECK();
    RecTcArgs ra;
    std::memset(&ra, 0, sizeof(ra));
    ra.work = s->d_awork_rec.as<ApplyWork>();
    ra.n_work = s->n_awork_rec;
    ra.blist = s->d_blist.as<int>();
    ra.cimg = cimg.as<uint8_t>();
    for (int t = 0; t < s->n_types; ++t) {
        build_tc_smean(s->types[t], prec);
        ra.simg[t] = s->types[t]->Smean_tc[prec].as<uint8_t>();
    }
    ra.n_el = s->n_el;
    ra.out = out;
    ra.err = s->flag.as<int>() + 2;
    const int chunks = (sh.n_etiles + kTilesPerItem - 1) / kTilesPerItem;
    const int items = s->n_awork_rec * chunks;
    const int per_sm = sh.smem > 100 * 1024 ? 1 : 2;
    const int grid = std::max(1, std::min(items, ctx->num_sms * per_sm));
    switch (prec) {
        case MSTRESS_TF32: k_recover_tc<MSTRESS_TF32><<<grid, kRecThreads, sh.smem, ctx->stream>>>(ra, sh); break;
        case MSTRESS_BF16: k_recover_tc<MSTRESS_BF16><<<grid, kRecThreads, sh.smem, ctx->stream>>>(ra, sh); break;
        default: k_recover_tc<MSTRESS_BF16X3><<<grid, kRecThreads, sh.smem, ctx->stream>>>(ra, sh); break;
    }
    MS_LAUNCH_CHECK();
    // cimg is released when this returns; cudaFree waits for the kernels using it
}

}  // namespace ms
