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
// Bases too large for a resident operator (m > 80) stream the operator and
// the coefficients along K through a ring of shared-memory slots instead
// (bulk copies + mbarriers, apply_tcs_item); their image is stored slot by
// slot so that each slot is one contiguous copy.
// (The work-item bodies are shared with the persistent solver: apply_items.cuh.)
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
    s.lg_tile = 7;
    s.a_plane = (uint32_t)round_up((int64_t)kTileTC * s.kpad * s.esz, 1024);
    s.b_plane = (uint32_t)round_up((int64_t)s.npad * s.kpad * s.esz, 1024);
    s.smem = (size_t)s.ns * (s.a_plane + s.b_plane) + 1024;   // + alignment slack
    // row stride of the FP32 tile copy: >= both paddings, and 4 more floats
    // so that eight consecutive rows' 16-byte reads fall in distinct banks
    s.ldp = (int)round_up(std::max(s.kpad, s.npad), 4) + 4;
    s.dot_smem = (size_t)kTileTC * s.ldp * sizeof(float) + (size_t)(s.npad / 16) * kTileTC * sizeof(double);
    return s;
}

ai::TcsShape tcs_shape(int m, int prec) {
    ai::TcsShape s;
    s.m = m;
    s.esz = prec == MSTRESS_TF32 ? 4 : 2;
    s.ns = prec == MSTRESS_BF16X3 ? 2 : 1;
    s.ck = 64 / s.esz;                          // two MMA K steps per slot
    s.nck = (m + s.ck - 1) / s.ck;
    s.kpad = s.nck * s.ck;
    s.npad = (int)round_up(m, 16);
    s.n0 = std::min(256, s.npad);
    s.n1 = s.npad - s.n0;
    s.tmem_cols = 32;
    while (s.tmem_cols < s.npad) s.tmem_cols *= 2;
    s.lg_tile = 7;
    s.a_plane = (uint32_t)(kTileTC * s.ck * s.esz);
    s.b_plane = (uint32_t)(s.npad * s.ck * s.esz);
    s.a_stage = s.ns * s.a_plane;
    s.b_stage = s.ns * s.b_plane;
    // two CTAs per SM when the accumulator leaves room in TMEM for a second one
    const size_t limit = s.tmem_cols <= 256 ? 110 * 1024 : 200 * 1024;
    const size_t slot = (size_t)s.a_stage + s.b_stage;
    s.stages = (int)std::min<size_t>(4, (limit - 1024) / slot);
    s.smem = (size_t)s.stages * slot + 1024;
    return s;
}

bool tc_streamed(int m) {
    for (int prec : {MSTRESS_TF32, MSTRESS_BF16, MSTRESS_BF16X3}) {
        ai::TcShape s = tc_shape(m, prec);
        if (s.npad > 256 || s.smem > 200 * 1024) return true;
    }
    return false;
}

namespace {

constexpr int kTcThreads = 128;
using ai::kTcsThreads;

// Operator image: B[n][k] = K_r[n][k] (zero padded), rounded to the mode's
// format; BF16X3 takes the lo part from the FP64 value. Columns are stored in
// slots of ck K-elements (slot c at byte c * slot_bytes, planes plane bytes
// apart within it); the resident layout is the single slot ck = kpad.
__global__ void k_build_image(const double* K, int m, int npad, int kpad, int ck, size_t slot_bytes, int esz,
                              int mode, uint8_t* out, uint32_t plane) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npad * kpad) return;
    int n = t / kpad, k = t % kpad;
    const double d = (n < m && k < m) ? K[(size_t)n * m + k] : 0.0;
    const size_t off = (size_t)(k / ck) * slot_bytes + tc::operand_offset(n, k % ck, ck, esz);
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
    __shared__ __align__(16) int offs[3 * kMaxSurf];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x;
    ai::TcState ts;
    ts.sB = smem;
    ts.sA = smem + NS * sh.b_plane;
    ts.sP = nullptr;   // no epilogue dot products in the stand-alone apply
    ts.sDot = nullptr;
    ts.ldp = 0;
    __shared__ long long eidx[kTileTC];
    ts.eidx = eidx;
    ts.cached_start = -1;
    ts.cached_array = -1;
    ts.A_pre = nullptr;
    ts.beta_pre = nullptr;
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

// Streamed-operator variant (large bases): warp-specialised CTAs of
// kTcsThreads threads (apply_items.cuh).
template <int MODE>
__global__ void __launch_bounds__(kTcsThreads, 1) k_apply_tcs(const __grid_constant__ ApplyArgs a,
                                                              const ai::TcsShape sh) {
    extern __shared__ uint8_t smraw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    __shared__ long long base[kTileTC];
    __shared__ __align__(16) int offs[3 * kMaxSurf];
    __shared__ __align__(8) uint64_t bars[3 * 4 + 2];
    __shared__ uint32_t tmem_base;
    __shared__ int fail;
    const int tid = threadIdx.x;
    ai::TcsState ts;
    ai::tcs_init(ts, sh, smem, bars, &fail);
    if ((tid >> 5) == 0) tc::tmem_alloc(&tmem_base, (uint32_t)sh.tmem_cols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    ts.tmem = tmem_base;
    // stand-alone: x and z are not written during the kernel (read through L1)
    if (!ai::tcs_apply_phase<MODE, true, true>(a, sh, ts, base, offs, blockIdx.x, gridDim.x)) {
        if (tid == 0) atomicExch(a.err, 1);
        ai::tcs_drain(ts, sh);
    }
    tc::fence_before();
    __syncthreads();
    if ((tid >> 5) == 0) tc::tmem_free(ts.tmem, (uint32_t)sh.tmem_cols);
}

}  // namespace

bool tc_supported(int m) {
    if (!tc_streamed(m)) return true;
    for (int prec : {MSTRESS_TF32, MSTRESS_BF16, MSTRESS_BF16X3}) {
        ai::TcsShape s = tcs_shape(m, prec);
        if (s.npad > 512 || s.stages < 2 || s.stages > 4) return false;
    }
    return true;
}

void configure_tc_kernels() {
    MS_CUDA(cudaFuncSetAttribute(k_apply_tc<MSTRESS_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    MS_CUDA(cudaFuncSetAttribute(k_apply_tc<MSTRESS_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    MS_CUDA(cudaFuncSetAttribute(k_apply_tc<MSTRESS_BF16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    MS_CUDA(cudaFuncSetAttribute(k_apply_tcs<MSTRESS_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    MS_CUDA(cudaFuncSetAttribute(k_apply_tcs<MSTRESS_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    MS_CUDA(cudaFuncSetAttribute(k_apply_tcs<MSTRESS_BF16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
}

void build_tc_operator(mstress_block blk, int prec) {
    if (blk->Kr_tc[prec].ptr) return;
    int npad, kpad, ck, esz;
    size_t slot, bytes;
    uint32_t plane;
    if (tc_streamed(blk->m)) {
        ai::TcsShape s = tcs_shape(blk->m, prec);
        npad = s.npad, kpad = s.kpad, ck = s.ck, esz = s.esz, plane = s.b_plane, slot = s.b_stage;
        bytes = (size_t)s.nck * s.b_stage;
    } else {
        ai::TcShape s = tc_shape(blk->m, prec);
        npad = s.npad, kpad = s.kpad, ck = s.kpad, esz = s.esz, plane = s.b_plane, slot = 0;
        bytes = (size_t)s.ns * s.b_plane;
    }
    alloc_into(blk->ctx, blk->Kr_tc[prec], bytes, true);
    int n = npad * kpad;
    k_build_image<<<(n + 255) / 256, 256, 0, blk->ctx->stream>>>(blk->Kr.as<double>(), blk->m, npad, kpad, ck, slot,
                                                                 esz, prec, blk->Kr_tc[prec].as<uint8_t>(), plane);
    MS_LAUNCH_CHECK();
}

void launch_apply_tc(mstress_sol_s* s, int prec, const ApplyArgs& a) {
    cudaStream_t st = s->ctx->stream;
    if (tc_streamed(s->m)) {
        ai::TcsShape sh = tcs_shape(s->m, prec);
        sh.lg_tile = lg_ceil(s->tc_tile);
        MS_REQUIRE(sh.npad <= 512 && sh.stages >= 2, MSTRESS_EINVAL, "basis too large for the tensor-core tile");
        const int per_sm = sh.tmem_cols <= 256 ? 2 : 1;
        const int grid = std::max(1, std::min(a.n_work, s->ctx->num_sms * per_sm));
        switch (prec) {
            case MSTRESS_TF32: k_apply_tcs<MSTRESS_TF32><<<grid, kTcsThreads, sh.smem, st>>>(a, sh); break;
            case MSTRESS_BF16: k_apply_tcs<MSTRESS_BF16><<<grid, kTcsThreads, sh.smem, st>>>(a, sh); break;
            default: k_apply_tcs<MSTRESS_BF16X3><<<grid, kTcsThreads, sh.smem, st>>>(a, sh); break;
        }
        MS_LAUNCH_CHECK();
        return;
    }
    ai::TcShape sh = tc_shape(s->m, prec);
    sh.lg_tile = lg_ceil(s->tc_tile);
    MS_REQUIRE(sh.npad <= 256 && sh.smem <= 200 * 1024, MSTRESS_EINVAL, "basis too large for the tensor-core tile");
    const int per_sm = sh.smem > 100 * 1024 ? 1 : 2;   // TMEM: <= 2 x 256 columns per SM
    const int grid = std::max(1, std::min(a.n_work, s->ctx->num_sms * per_sm));
    switch (prec) {
        case MSTRESS_TF32: k_apply_tc<MSTRESS_TF32><<<grid, kTcThreads, sh.smem, st>>>(a, sh); break;
        case MSTRESS_BF16: k_apply_tc<MSTRESS_BF16><<<grid, kTcThreads, sh.smem, st>>>(a, sh); break;
        default: k_apply_tc<MSTRESS_BF16X3><<<grid, kTcThreads, sh.smem, st>>>(a, sh); break;
    }
    MS_LAUNCH_CHECK();
}

}  // namespace ms
