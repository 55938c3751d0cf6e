// Reduced-precision operator apply of the global stage on the tensor cores
// (tcgen05, sm_103a): for a tile of up to 128 blocks of one type,
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
// (The work-item body is shared with the persistent solver: apply_items.cuh.)
#include "apply_items.cuh"

namespace ms {

ai::TcShape tc_shape(int m, int prec) {
    ai::TcShape s;
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

namespace {

constexpr int kTcThreads = 128;

// Operator image: B[n][k] = K_r[n][k] (zero padded), rounded to the mode's
// format; BF16X3 takes the lo part from the FP64 value.
__global__ void k_build_image(const double* K, int m, int npad, int kpad, int esz, int mode, uint8_t* out,
                              uint32_t plane) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npad * kpad) return;
    int n = t / kpad, k = t % kpad;
    const double d = (n < m && k < m) ? K[(size_t)n * m + k] : 0.0;
    const uint32_t off = tc::operand_offset(n, k, kpad, esz);
    if (mode == MSTRESS_BF16X3) {
        const __nv_bfloat16 hi = __float2bfloat16_rn((float)d);
        *reinterpret_cast<__nv_bfloat16*>(out + off) = hi;
        *reinterpret_cast<__nv_bfloat16*>(out + plane + off) =
            __float2bfloat16_rn((float)(d - (double)__bfloat162float(hi)));
    } else {
        ai::put_operand(out, plane, off, (float)d, mode);
    }
}

template <int MODE>
__global__ void __launch_bounds__(kTcThreads) k_apply_tc(const __grid_constant__ ApplyArgs a, const ai::TcShape sh) {
    constexpr int NS = MODE == MSTRESS_BF16X3 ? 2 : 1;
    extern __shared__ uint8_t smraw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    __shared__ long long base[kTileTC];
    __shared__ int offs[3 * kMaxSurf];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x;
    ai::TcState ts;
    ts.sB = smem;
    ts.sA = smem + NS * sh.b_plane;
    for (uint32_t i = tid; i < NS * sh.a_plane / 16; i += kTcThreads)
        reinterpret_cast<uint4*>(ts.sA)[i] = make_uint4(0, 0, 0, 0);
    if ((tid >> 5) == 0) tc::tmem_alloc(&tmem_base, (uint32_t)sh.tmem_cols);
    if (tid == 0) tc::mbar_init(&mbar, 1);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    ts.tmem = tmem_base;
    ts.mbar = &mbar;
    ts.phase = 0;
    ts.cur_type = -1;
    bool failed = false;
    for (int w = blockIdx.x; w < a.n_work; w += gridDim.x) {
        const ApplyWork it = a.work[w];
        if (a.st && !a.st[it.array].active) continue;
        if (!ai::apply_tc_item<MODE>(a, sh, it, ts, base, offs)) {
            failed = true;
            break;
        }
    }
    if (failed) {
        if (tid == 0) atomicExch(a.err, 1);
        tc::mbar_wait(&mbar, ts.phase ^ 1u, 1 << 20);   // give in-flight MMAs a bounded chance to drain
    }
    tc::fence_before();
    __syncthreads();
    if ((tid >> 5) == 0) tc::tmem_free(ts.tmem, (uint32_t)sh.tmem_cols);
}

}  // namespace

bool tc_supported(int m) {
    for (int prec : {MSTRESS_TF32, MSTRESS_BF16, MSTRESS_BF16X3}) {
        ai::TcShape s = tc_shape(m, prec);
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
    ai::TcShape s = tc_shape(blk->m, prec);
    alloc_into(blk->ctx, blk->Kr_tc[prec], (size_t)s.ns * s.b_plane, true);
    int n = s.npad * s.kpad;
    k_build_image<<<(n + 255) / 256, 256, 0, blk->ctx->stream>>>(blk->Kr.as<double>(), blk->m, s.npad, s.kpad, s.esz,
                                                                 prec, blk->Kr_tc[prec].as<uint8_t>(), s.b_plane);
    MS_LAUNCH_CHECK();
}

void launch_apply_tc(mstress_sol_s* s, int prec, const ApplyArgs& a) {
    ai::TcShape sh = tc_shape(s->m, prec);
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
