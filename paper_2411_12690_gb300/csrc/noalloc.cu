// Operator apply that allocates no memory: y = A_global x for one array whose
// sites all use the same block model, in FP64.
//
// Some callers cannot allocate device memory at the time they need the
// operator: code running inside a CUDA stream capture they do not control,
// real-time loops whose memory is fixed up front, or hosts whose allocator is
// owned by another runtime. mstress_apply (and every solve) allocates its work
// lists and the element-product buffer on each call; this entry point does
// not. Its only scratch is the element-product buffer, kept in a file-scope
// __device__ array of fixed size (kNoAllocScratchBytes) that every GPU which
// loads this library holds until the process exits. Work lists are replaced
// by arithmetic on the block index, and the surface-node table travels as a
// kernel parameter.
//
// Set-up: the device address of the scratch array is looked up with
// cudaGetSymbolAddress the first time the entry point runs on a device (with
// that device current) and cached; that first call must come before any
// stream capture and is refused (MSTRESS_EINVAL) on a capturing stream. The
// block's context device must be the current device. The block must outlive
// the work issued on cuda_stream: free it only after that work has finished. Every call shares the one array, which keeps the last call's
// contents; nothing in it needs to start at zero because each call writes
// every entry it reads. Calls whose work overlaps on the GPU (different
// streams, or different host threads on one stream without ordering) race on
// the array and must be serialised by the caller.
#include <mutex>

#include "pcg_items.cuh"

namespace ms {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;   // 32 MiB of element products
constexpr int kNaTile = 32;                                  // blocks per CTA tile
constexpr int kNaThreads = 256;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchBytes / sizeof(double)];

struct NaArgs {
    LocalMap lm;       // surface-node table (kernel parameter, no device copy)
    ArrayDev A;        // the array (vec_off 0, block_off 0)
    const double* K;   // A_element, m x m FP64
    int m, ldY;
    const double* x;
    double* y;
    double* Y;         // scratch: element products [block][ldY]
};

// Element products Y_e = A_element x[G_e] for 32 consecutive blocks per CTA.
__global__ void __launch_bounds__(kNaThreads) k_na_apply(const __grid_constant__ NaArgs a) {
    extern __shared__ double Cs[];   // [m][32]
    __shared__ long long base[kNaTile];
    __shared__ int offs[3 * kMaxSurf];
    const int m = a.m, n1 = a.lm.n - 1;
    const long long n_blocks = (long long)a.A.nx * a.A.ny;
    const long long e0 = (long long)blockIdx.x * kNaTile;
    const int count = (int)(n_blocks - e0 < kNaTile ? n_blocks - e0 : kNaTile);
    for (int k = threadIdx.x; k < m; k += kNaThreads) {
        const int q = k / 3, c = k - 3 * q;
        offs[k] = ((a.lm.qc[q] * a.A.Y + a.lm.qb[q]) * a.A.X + a.lm.qa[q]) * 3 + c;
    }
    if (threadIdx.x < count) {
        const long long e = e0 + threadIdx.x;
        const int i = (int)(e % a.A.nx), j = (int)(e / a.A.nx);
        base[threadIdx.x] = 3LL * ((long long)j * n1 * a.A.X + (long long)i * n1);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < m * kNaTile; idx += kNaThreads) {
        const int k = idx / kNaTile, bt = idx % kNaTile;
        Cs[idx] = bt < count ? a.x[base[bt] + offs[k]] : 0.0;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < m * count; o += kNaThreads) {
        const int r = o / count, bt = o % count;
        const double* kr = a.K + (size_t)r * m;
        double acc = 0;
        for (int k = 0; k < m; ++k) acc = fma(kr[k], Cs[k * kNaTile + bt], acc);
        a.Y[(e0 + bt) * a.ldY + r] = acc;
    }
}

// Interface sum y_g = sum of Y_e over the blocks owning lattice DOF g.
__global__ void __launch_bounds__(kNaThreads) k_na_isum(const __grid_constant__ NaArgs a) {
    const long long g = blockIdx.x * (long long)kNaThreads + threadIdx.x;
    if (g >= a.A.n_dof) return;
    int comp, gx, gy, gz;
    pi::lattice_coords(a.A, g, comp, gx, gy, gz);
    double s = 0;
    pi::for_owners(a.A, a.lm.surf_idx, a.lm.n, gx, gy, gz,
                   [&](long long blk, int sidx) { s += a.Y[blk * a.ldY + 3 * sidx + comp]; });
    a.y[g] = s;
}

std::mutex g_scratch_mutex;
void* g_scratch_ptr[64] = {};

// Device address of the scratch array on device dev (which must be current),
// looked up once per device (together with the apply kernel's shared-memory
// limit). The look-up is refused while `st` is being captured into a graph:
// the set-up calls would invalidate the caller's capture.
double* scratch_for_device(int dev, cudaStream_t st) {
    MS_REQUIRE(dev >= 0 && dev < 64, MSTRESS_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        MS_CUDA(cudaStreamIsCapturing(st, &cs));
        MS_REQUIRE(cs == cudaStreamCaptureStatusNone, MSTRESS_EINVAL,
                   "the first mstress_apply_noalloc call on a device sets up its scratch and must not be "
                   "captured: make one call before the capture begins");
        void* p = nullptr;
        MS_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        MS_CUDA(cudaFuncSetAttribute(k_na_apply, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(3 * kMaxSurf * kNaTile * sizeof(double))));
        g_scratch_ptr[dev] = p;
    }
    return static_cast<double*>(g_scratch_ptr[dev]);
}

}  // namespace
}  // namespace ms

using namespace ms;

extern "C" int mstress_apply_noalloc(mstress_block blk, int nx, int ny, const double* x_dev, double* y_dev,
                                     void* cuda_stream) {
    if (!blk) return MSTRESS_EINVAL;
    mstress_ctx ctx = blk->ctx;
    try {
        MS_REQUIRE(x_dev && y_dev, MSTRESS_EINVAL, "x and y are required");
        MS_REQUIRE(nx >= 1 && ny >= 1, MSTRESS_EINVAL, "array needs nx, ny >= 1");
        int dev = -1;
        MS_CUDA(cudaGetDevice(&dev));
        MS_REQUIRE(dev == ctx->device, MSTRESS_EINVAL,
                   "the block's device (" + std::to_string(ctx->device) + ") is not the current device (" +
                       std::to_string(dev) + ")");
        NaArgs a;
        std::memset(&a, 0, sizeof(a));
        a.lm = make_local_map(blk->n);
        a.m = blk->m;
        a.ldY = (int)round_up(blk->m, 16);
        const long long n_blocks = (long long)nx * ny;
        MS_REQUIRE(n_blocks * a.ldY * (long long)sizeof(double) <= (long long)kNoAllocScratchBytes, MSTRESS_EINVAL,
                   "array too large for the no-allocation scratch (" + std::to_string(kNoAllocScratchBytes) +
                       " bytes of element products: at most " +
                       std::to_string(kNoAllocScratchBytes / (a.ldY * sizeof(double))) + " blocks at m = " +
                       std::to_string(blk->m) + ")");
        const int n1 = blk->n - 1;
        a.A.nx = nx;
        a.A.ny = ny;
        a.A.X = nx * n1 + 1;
        a.A.Y = ny * n1 + 1;
        a.A.Z = blk->n;
        a.A.n_dof = 3LL * a.A.X * a.A.Y * a.A.Z;
        a.K = blk->Kr.as<double>();
        a.x = x_dev;
        a.y = y_dev;
        cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
        a.Y = scratch_for_device(dev, st);
        const size_t smem = (size_t)a.m * kNaTile * sizeof(double);
        k_na_apply<<<(unsigned)((n_blocks + kNaTile - 1) / kNaTile), kNaThreads, smem, st>>>(a);
        MS_LAUNCH_CHECK();
        k_na_isum<<<(unsigned)((a.A.n_dof + kNaThreads - 1) / kNaThreads), kNaThreads, 0, st>>>(a);
        MS_LAUNCH_CHECK();
    } catch (const ms::Error& e) {
        if (ctx) ctx->last_error = e.msg;
        return e.code;
    }
    return MSTRESS_OK;
}
