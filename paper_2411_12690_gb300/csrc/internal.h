// Internal declarations shared by the translation units of libmstress.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/mstress.h"

namespace ms {

// ----------------------------------------------------------------- errors
struct Error {
    int code;
    std::string msg;
};

#define MS_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            throw ::ms::Error{MSTRESS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
    } while (0)

#define MS_REQUIRE(cond, code, msg)                                   \
    do {                                                              \
        if (!(cond)) throw ::ms::Error{(code), std::string(msg)};     \
    } while (0)

#define MS_LAUNCH_CHECK()              \
    do {                               \
        MS_CUDA(cudaGetLastError());   \
        ::ms::note_launches(1);        \
    } while (0)

constexpr int kMaxN = 8;                          // Lagrange nodes per axis (order <= 7)
constexpr int kMaxSurf = kMaxN * kMaxN * kMaxN - (kMaxN - 2) * (kMaxN - 2) * (kMaxN - 2);
constexpr int kMaxTypes = 16;                     // block models in one solve
constexpr int kMaxMat = 16;                       // materials in one block mesh

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// Process-wide count of kernels this library launched (graph replays count
// their kernel nodes; launches recorded into a graph during capture do not).
extern thread_local bool g_capturing;
void note_launches(long long n);

// --------------------------------------------------------- device memory
// Device buffer owned by a context; freed (and un-budgeted) on destruction.
struct DBuf {
    mstress_ctx ctx = nullptr;
    void* ptr = nullptr;
    size_t bytes = 0;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept { *this = std::move(o); }
    DBuf& operator=(DBuf&& o) noexcept;
    ~DBuf() { reset(); }
    void reset();
    template <class T> T* as() const { return static_cast<T*>(ptr); }
};

// ------------------------------------------------------------- local map
// Surface Lagrange nodes of a block with n nodes per axis (Eqs. 8-9, 16):
// q-th node has local lattice offsets (qa, qb, qc); surf_idx maps
// (c*n + b)*n + a to q, or -1 for interior nodes.
struct LocalMap {
    int n, nsurf, m, pad;
    int16_t surf_idx[kMaxN * kMaxN * kMaxN];
    uint8_t qa[kMaxSurf], qb[kMaxSurf], qc[kMaxSurf];
};
LocalMap make_local_map(int n);

// ----------------------------------------------------- solve structures
struct ArrayDev {            // one array of a (batched) solve
    int nx, ny;              // sites
    int X, Y, Z;             // lattice points per axis
    int clamp_bottom, clamp_top;
    int n_presc;             // prescribed DOFs (lifting) in this array
    long long vec_off;       // first lattice DOF of this array in the packed vectors
    long long n_dof;         // X*Y*Z*3
    long long block_off;     // first block (site) of this array
    int vwork_off, n_vwork;  // lattice work items of this array
    int grp_off, n_grp;      // 8-block groups of this array (per-group partial sums of the apply)
    double dT;
};

struct BlockRef { int array, i, j, type; };            // one site of one array
// blist[start .. start+count); grp: first 8-block group of the tile (groups are
// 8 consecutive blist entries of one (array, type) run, numbered over the
// batch; tiles are multiples of 8 blocks and start on a group)
struct ApplyWork { int type, array, start, count, grp; };
struct VecWork { int array, pad; long long start, count; };  // packed lattice DOF range

struct PcgState {            // per-array conjugate-gradient scalars
    double rz, rr, bb, tol2;
    double beta;             // pending p = z + beta p of the next iteration
    double alpha;            // step length of the current iteration (persistent solver)
    int iters, active, status, max_iter;
};

struct TypeTab {             // block models of a solve, by type index
    const double* Kr[kMaxTypes];     // m*m FP64
    const double* br[kMaxTypes];     // m FP64
    const void* Klp[kMaxTypes];      // low-precision K_r copies (tensor-core layout)
    const double* rows[kMaxTypes];   // recovery mode matrix (S, Smean or F), ld = ld_rows
    const void* rows_lp[kMaxTypes];  // low-precision recovery modes
};

}  // namespace ms

// ------------------------------------------------------------ handles
struct mstress_ctx_s {
    int device = 0;
    int num_sms = 0;
    // bounded device waits of the persistent solver: a grid-barrier wait gives
    // up after wait_limit_ns; withhold_next: the next persistent launch's last
    // CTA skips its first barrier arrival once (test hook for the timeout path)
    long long wait_limit_ns = 2000000000LL;
    int withhold_next = 0;
    cudaStream_t stream = nullptr;
    mstress_opts opts{};
    size_t in_use = 0, peak = 0;
    std::map<void*, size_t> allocs;
    // tensor-core tile size chosen by the autotuner, per (basis size,
    // precision, batch-size class)
    std::map<uint64_t, int> tile_choice;
    // Freed blocks kept for reuse (size -> block, event recorded on the
    // context stream at release): repeated solves of the same shapes allocate
    // without cudaMalloc / cudaFree (which would synchronise the device).
    struct Cached {
        void* p;
        cudaEvent_t ev;
    };
    std::multimap<size_t, Cached> cache;
    size_t cached = 0;
    void trim(size_t keep);   // free cached blocks until at most keep bytes remain
    std::string last_error;
    // pinned host words for polling device flags
    int* h_flag = nullptr;
    // pinned host copy of the inner solves' per-array states (iteration counts),
    // read at the next stream synchronisation of the solve
    void* h_states = nullptr;
    size_t h_states_bytes = 0;
    // pinned host staging of a solve's work lists on their way to the device
    // (reused: a solve's set-up copies finish before the next set-up starts)
    uint8_t* h_stage = nullptr;
    size_t h_stage_bytes = 0;

    void* alloc(size_t bytes);
    void release(void* p);
    void budget_check(size_t bytes) const;
};

struct mstress_block_s {
    mstress_ctx ctx = nullptr;
    int n = 0, m = 0, m1 = 0, ld = 0;    // ld: leading dimension of S, Smean, F rows (>= m+1)
    int ex = 0, ey = 0, ez = 0;
    double lx = 0, ly = 0, lz = 0;
    int n_el = 0, n_nodes = 0, n_dof = 0;
    int cg_iters = 0;
    bool has_F = false;
    ms::DBuf Kr, br, S, Smean, F;
    // lazily created low-precision operand copies, by precision mode
    ms::DBuf Kr_lp[4], Smean_lp[4], S_lp[4];
    // tensor-core operand images (K-major, no-swizzle core-matrix layout), by precision mode
    ms::DBuf Kr_tc[4], Smean_tc[4];
    // fine-mesh materials (kept from the local stage; absent for imported blocks)
    bool has_mat = false;
    ms::DBuf mat_id;                       // n_el material indices
    double mat_lam[ms::kMaxMat] = {}, mat_mu[ms::kMaxMat] = {}, mat_tm[ms::kMaxMat] = {};
    // stress modes at the points of the half-height cut plane (gridded output)
    int grid_side = 0, n_grid = 0;         // side x side points, or none
    ms::DBuf Sgrid;                        // (6 n_grid) x ld FP64, row p*6+comp
    ms::DBuf Sgrid_lp[4], Sgrid_tc[4];     // low-precision copies / tensor-core images
};

namespace ms {

void alloc_into(mstress_ctx ctx, DBuf& b, size_t bytes, bool zero = true);

// offline (local stage) --------------------------------------------------
int build_block(mstress_ctx ctx, const mstress_block_mesh* mesh, const mstress_tsv_geom* tsv,
                const mstress_material* mats, int n_mat, int order, mstress_block* out);
void block_compute_smean(mstress_block blk);
void build_grid_modes(mstress_block blk, int side);   // Sgrid of the half-height plane

// low-precision operand preparation (tensor-core paths) --------------------
void ensure_lowp(mstress_block blk, int precision);

}  // namespace ms
