// Reduced-precision operator apply of the global stage on the tensor cores
// (tcgen05, sm_103a): for a tile of 128 blocks of one type,
//     D (128 x N) = C (128 x K) * K_r^T,   D[b][n] = (A_element c_b)[n]   (Eq. 18)
// with C the gathered element DOFs of the tile's blocks (one row per block),
// K_r the block's reduced stiffness (symmetric), N = K = m padded. The MMA is
// issued by one thread, operands sit in shared memory in the K-major
// no-swizzle core-matrix layout, the FP32 accumulator lives in tensor memory
// and is read back with tcgen05.ld for the epilogue (the element products Y).
//   TF32    kind::tf32, one product
//   BF16    kind::f16 with bf16 operands, one product
//   BF16X3  operands split v = hi + lo (both bf16); hi*hi + lo*hi + hi*lo
// The operator image is built once per block model and copied into shared
// memory whenever a CTA moves to a tile of another type; the gather rounds
// the coefficients into the same format. CTAs are persistent over the tiles.
#include "solve.h"
#include "tc.cuh"

namespace ms {
namespace {

constexpr int kTcThreads = 128;

struct TcShape {
    int m, esz, kpad, npad, ksteps, tmem_cols, ns;
    uint32_t a_plane, b_plane;   // bytes per operand plane (multiples of 1024)
    size_t smem;
};

TcShape tc_shape(int m, int prec) {
    TcShape s;
    s.m = m;
    s.esz = prec == MSTRESS_TF32 ? 4 : 2;
    s.kpad = (int)round_up(m, 32 / s.esz);
    s.npad = (int)round_up(m, 16);
    s.ksteps = s.kpad * s.esz / 32;
    s.tmem_cols = 32;
    while (s.tmem_cols < s.npad) s.tmem_cols *= 2;
    s.ns = prec == MSTRESS_BF16X3 ? 2 : 1;
    s.a_plane = (uint32_t)round_up((int64_t)kTileTC * s.kpad * s.esz, 1024);
    s.b_plane = (uint32_t)round_up((int64_t)s.npad * s.kpad * s.esz, 1024);
    s.smem = (size_t)s.ns * (s.a_plane + s.b_plane) + 1024;   // + alignment slack
    return s;
}

__device__ __forceinline__ void put_operand(uint8_t* plane0, uint32_t plane_bytes, uint32_t off, float v, int mode) {
    if (mode == MSTRESS_TF32) {
        *reinterpret_cast<float*>(plane0 + off) = tc::to_tf32(v);
    } else {
        __nv_bfloat16 hi = __float2bfloat16_rn(v);
        *reinterpret_cast<__nv_bfloat16*>(plane0 + off) = hi;
        if (mode == MSTRESS_BF16X3)
            *reinterpret_cast<__nv_bfloat16*>(plane0 + plane_bytes + off) =
                __float2bfloat16_rn(v - __bfloat162float(hi));
    }
}

// Operator image: B[n][k] = K_r[n][k] (zero padded), rounded to the mode's format.
__global__ void k_build_image(const double* K, int m, int npad, int kpad, int esz, int mode, uint8_t* out,
                              uint32_t plane) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npad * kpad) return;
    int n = t / kpad, k = t % kpad;
    float v = (n < m && k < m) ? (float)K[(size_t)n * m + k] : 0.0f;
    uint32_t off = tc::operand_offset(n, k, kpad, esz);
    if (mode == MSTRESS_BF16X3) {   // lo part from the FP64 value
        double d = (n < m && k < m) ? K[(size_t)n * m + k] : 0.0;
        __nv_bfloat16 hi = __float2bfloat16_rn((float)d);
        *reinterpret_cast<__nv_bfloat16*>(out + off) = hi;
        *reinterpret_cast<__nv_bfloat16*>(out + plane + off) = __float2bfloat16_rn((float)(d - (double)__bfloat162float(hi)));
    } else {
        put_operand(out, plane, off, v, mode);
    }
}

template <int MODE>
__global__ void __launch_bounds__(kTcThreads) k_apply_tc(const __grid_constant__ ApplyArgs a, const TcShape sh) {
    constexpr bool TF32 = MODE == MSTRESS_TF32;
    constexpr int NS = MODE == MSTRESS_BF16X3 ? 2 : 1;
    extern __shared__ uint8_t smraw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    uint8_t* sB = smem;                              // NS planes of the operator image
    uint8_t* sA = smem + NS * sh.b_plane;            // NS planes of gathered coefficients
    __shared__ long long base[kTileTC];
    __shared__ int offs[3 * kMaxSurf];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = a.m;
    for (uint32_t i = tid; i < NS * sh.a_plane / 16; i += kTcThreads) reinterpret_cast<uint4*>(sA)[i] = make_uint4(0, 0, 0, 0);
    if (warp == 0) tc::tmem_alloc(&tmem_base, (uint32_t)sh.tmem_cols);
    if (tid == 0) tc::mbar_init(&mbar, 1);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = tc::instr_desc(TF32, kTileTC, sh.npad);
    const uint32_t sboA = tc::sbo_bytes(sh.kpad, sh.esz), sboB = sboA;
    const float* __restrict__ x = static_cast<const float*>(a.x);
    const float* __restrict__ z = static_cast<const float*>(a.z);
    float* __restrict__ Y = static_cast<float*>(a.Y);
    int cur_type = -1;
    uint32_t phase = 0;
    bool failed = false;
    for (int w = blockIdx.x; w < a.n_work; w += gridDim.x) {
        const ApplyWork it = a.work[w];
        if (a.st && !a.st[it.array].active) continue;
        const ArrayDev A = a.arrays[it.array];
        const double beta = a.st ? a.st[it.array].beta : 0.0;
        if (it.type != cur_type) {
            const uint4* src = static_cast<const uint4*>(a.tt.Klp[it.type]);
            for (uint32_t i = tid; i < NS * sh.b_plane / 16; i += kTcThreads) reinterpret_cast<uint4*>(sB)[i] = src[i];
            cur_type = it.type;
        }
        tile_setup(a, it, A, base, offs, kTileTC);
        __syncthreads();
        for (int idx = tid; idx < m * kTileTC; idx += kTcThreads) {
            const int k = idx >> 7, b = idx & (kTileTC - 1);
            float v = 0.0f;
            if (b < it.count) {
                long long g = base[b] + offs[k];
                v = z ? p_next(z[g], x[g], beta) : x[g];
            }
            put_operand(sA, sh.a_plane, tc::operand_offset(b, k, sh.kpad, sh.esz), v, MODE);
        }
        tc::fence_smem_async();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (tid == 0) {
            const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB);
            uint32_t acc = 0;
            for (int s = 0; s < sh.ksteps; ++s) {
                const uint32_t ko = (uint32_t)s * 2 * tc::kLBO;
                // products: (A plane, B plane) = (hi, hi) [, (lo, hi), (hi, lo)]
#pragma unroll
                for (int pr = 0; pr < (NS == 2 ? 3 : 1); ++pr) {
                    const uint32_t pa = pr == 1 ? sh.a_plane : 0u, pb = pr == 2 ? sh.b_plane : 0u;
                    const uint64_t da = tc::smem_desc(a0 + pa + ko, tc::kLBO, sboA);
                    const uint64_t db = tc::smem_desc(b0 + pb + ko, tc::kLBO, sboB);
                    tc::mma<TF32>(tmem, da, db, idesc, acc);
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
        const int b = warp * 32 + lane;
        const long long e = b < it.count ? a.blist[it.start + b] : 0;
        for (int c0 = 0; c0 < sh.npad; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
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
    }
    if (failed) {
        if (tid == 0) atomicExch(a.err, 1);
        tc::mbar_wait(&mbar, phase ^ 1u, 1 << 20);   // give in-flight MMAs a bounded chance to drain
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, (uint32_t)sh.tmem_cols);
}

}  // namespace

bool tc_supported(int m) {
    for (int prec : {MSTRESS_TF32, MSTRESS_BF16, MSTRESS_BF16X3}) {
        TcShape s = tc_shape(m, prec);
        if (s.npad > 256 || s.smem > 200 * 1024) return false;
    }
    return true;
}

void configure_tc_kernels() {
    MS_CUDA(cudaFuncSetAttribute(k_apply_tc<MSTRESS_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    MS_CUDA(cudaFuncSetAttribute(k_apply_tc<MSTRESS_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    MS_CUDA(cudaFuncSetAttribute(k_apply_tc<MSTRESS_BF16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
}

void build_tc_operator(mstress_block blk, int prec) {
    if (blk->Kr_tc[prec].ptr) return;
    TcShape s = tc_shape(blk->m, prec);
    alloc_into(blk->ctx, blk->Kr_tc[prec], (size_t)s.ns * s.b_plane, true);
    int n = s.npad * s.kpad;
    k_build_image<<<(n + 255) / 256, 256, 0, blk->ctx->stream>>>(blk->Kr.as<double>(), blk->m, s.npad, s.kpad, s.esz,
                                                                 prec, blk->Kr_tc[prec].as<uint8_t>(), s.b_plane);
    MS_LAUNCH_CHECK();
}

void launch_apply_tc(mstress_sol_s* s, int prec, const ApplyArgs& a) {
    TcShape sh = tc_shape(s->m, prec);
    MS_REQUIRE(sh.npad <= 256 && sh.smem <= 200 * 1024, MSTRESS_EINVAL, "basis too large for the tensor-core tile");
    const int per_sm = sh.smem > 100 * 1024 ? 1 : 2;   // TMEM: <= 2 x 256 columns per SM
    const int grid = std::max(1, std::min(a.n_work, s->ctx->num_sms * per_sm));
    cudaStream_t st = s->ctx->stream;
    switch (prec) {
        case MSTRESS_TF32: k_apply_tc<MSTRESS_TF32><<<grid, kTcThreads, sh.smem, st>>>(a, sh); break;
        case MSTRESS_BF16: k_apply_tc<MSTRESS_BF16><<<grid, kTcThreads, sh.smem, st>>>(a, sh); break;
        default: k_apply_tc<MSTRESS_BF16X3><<<grid, kTcThreads, sh.smem, st>>>(a, sh); break;
    }
    MS_LAUNCH_CHECK();
}

}  // namespace ms
