/*
 * mstress.h -- C ABI of libmstress, a GB300 (sm_103a) implementation of the
 * MORE-Stress method for thermal stress in TSV arrays (arXiv 2411.12690).
 *
 * The paper's method has two stages (section 4.1):
 *   - the one-shot LOCAL stage (section 4.2, Eqs. 8-16) reduces one unit block,
 *     meshed finely, to a dense element stiffness A_element = F^T A_local F
 *     (Eq. 18) and load b_element (Eq. 19) over the displacements of Lagrange
 *     nodes on the block surface; this is mstress_build_block();
 *   - the GLOBAL stage (section 4.3, Eq. 20) assembles blocks as abstract
 *     elements, solves the reduced system and recovers fine fields by the linear
 *     combination of Eq. 15 and the stress of Eq. 1; this is mstress_solve() and
 *     mstress_recover().
 * Sub-modeling (section 4.4) enters through prescribed boundary displacements
 * (mstress_bc) and "dummy" pure-silicon blocks (a second block model).
 *
 * Conventions
 *   Units: um and MPa (so u is in um, sigma in MPa, E in MPa, alpha in 1/K).
 *   Fine block mesh: structured ex*ey*ez Q1 hexahedra on [0,lx]x[0,ly]x[0,lz];
 *     node (ix,iy,iz) has id ix + (ex+1)*(iy + (ey+1)*iz), DOF 3*node + comp;
 *     element (kx,ky,kz) has id kx + ex*(ky + ey*kz).
 *   Element DOFs (the m reduced DOFs of a block): n = order+1 equally spaced
 *     Lagrange nodes per axis (Eqs. 8-9), surface nodes only, enumerated with
 *     the x index fastest, then y, then z; DOF 3*q + comp for surface node q.
 *     m = 3 (n^3 - (n-2)^3) (Eq. 16).
 *   Stress: Voigt order (xx, yy, zz, xy, yz, zx).
 *   Gauss points: 2x2x2, g = gx + 2 gy + 4 gz.
 *   Arrays: site (i, j), i = column (x), j = row (y), stored j*nx + i.
 *
 * Ownership: every handle is owned by the library and released only by its
 * mstress_free_* call; a handle must not outlive the context that made it.
 * Input arrays are owned by the caller and are copied before the call returns.
 * Output buffers are owned by the caller; their size is checked.
 *
 * Errors: every int-returning call returns MSTRESS_OK (0) or a negative
 * status; mstress_last_error() then holds a one-line description. A context is
 * not thread safe; calls on one context must be serialised by the caller.
 * Work is issued on the context's CUDA stream; calls that return host data
 * synchronise that stream.
 */
#ifndef MSTRESS_H
#define MSTRESS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define MSTRESS_OK               0
#define MSTRESS_EINVAL          -1   /* bad argument, layout or size            */
#define MSTRESS_ENOMEM          -2   /* device allocation refused (HBM budget)  */
#define MSTRESS_ENOT_CONVERGED  -3   /* iteration limit hit; result is returned */
#define MSTRESS_EDEVICE_TIMEOUT -4   /* a bounded device-side wait gave up      */
#define MSTRESS_ENUMERIC        -5   /* NaN/Inf or CG breakdown                 */
#define MSTRESS_ECUDA           -6   /* a CUDA runtime call failed              */

/* ------------------------------------------------------- precision modes
 * Arithmetic of the reduced operator apply (K_r times block coefficients) and
 * of the recovery contraction (S times [c; dT]).
 *   FP64    plain method: every product and sum in FP64.
 *   TF32    tensor cores (tcgen05, kind::tf32), FP32 accumulation; the solve
 *           is FP64-residual iterative refinement around an inner PCG whose
 *           vectors are FP32 and whose dot products and step lengths are FP64.
 *   BF16    as TF32 with bf16 operands (kind::f16).
 *   BF16X3  operands split into bf16 hi + lo parts, three tensor-core products
 *           (hi*hi + hi*lo + lo*hi) per contraction. */
#define MSTRESS_FP64    0
#define MSTRESS_TF32    1
#define MSTRESS_BF16    2
#define MSTRESS_BF16X3  3

/* ------------------------------------------------------------ handles */
typedef struct mstress_ctx_s*   mstress_ctx;    /* device, stream, HBM budget      */
typedef struct mstress_block_s* mstress_block;  /* resident reduced block model    */
typedef struct mstress_sol_s*   mstress_sol;    /* resident solution of 1..n arrays */

/* ------------------------------------------------------------ inputs */
typedef struct {
    double E;       /* Young modulus, MPa                  */
    double nu;      /* Poisson ratio                       */
    double alpha;   /* thermal expansion coefficient, 1/K  */
} mstress_material;

typedef struct {
    double lx, ly, lz;       /* block edge lengths, um                        */
    int ex, ey, ez;          /* elements per axis                             */
    const uint8_t* mat_id;   /* ex*ey*ez material indices (element order) or  */
                             /* NULL: voxelise the TSV geometry below         */
} mstress_block_mesh;

typedef struct {
    double r_cu;      /* Cu radius, um; <= 0 gives a pure-Si (dummy) block   */
    double t_liner;   /* SiO2 liner thickness, um                            */
} mstress_tsv_geom;   /* voxeliser: element takes the material at its centroid:
                         material 1 (Cu) if r <= r_cu, 2 (liner) if
                         r <= r_cu + t_liner, else 0 (Si); r from the block axis */

typedef struct {
    int nx, ny;                    /* sites per row (x) and rows (y)             */
    const uint8_t* site_type;      /* nx*ny entries, index into blocks[]         */
    const mstress_block* blocks;   /* block models; same basis order and size    */
    int n_blocks;
} mstress_layout;

typedef struct {
    int clamp_bottom;              /* 1: all DOFs on z = 0 fixed to zero          */
    int clamp_top;                 /* 1: all DOFs on z = lz fixed to zero         */
    /* Prescribed displacements (sub-modeling, section 4.4, imposed by lifting,
       Eq. 13): n_prescribed pairs of lattice DOF index and value. The lattice of
       an nx*ny array with n nodes per axis has X = nx(n-1)+1, Y = ny(n-1)+1,
       Z = n points; DOF index = 3*((z*Y + y)*X + x) + comp. NULL/0: none. */
    const int64_t* prescribed_dof;
    const double* prescribed_val;
    size_t n_prescribed;
} mstress_bc;

typedef struct {
    int precision;        /* MSTRESS_FP64 | _TF32 | _BF16 | _BF16X3           */
    double rtol;          /* stop when ||b - A x||_2 <= rtol ||b||_2 (FP64)   */
    int max_iter;         /* PCG iteration limit (inner iterations summed)     */
    double inner_rtol;    /* mixed modes: inner PCG relative tolerance (an inner
                             solve also stops below a tenth of the outer
                             tolerance); 0 = by precision: 3e-4 BF16X3, 1e-3
                             TF32, 3e-2 BF16                                */
    int max_outer;        /* mixed modes: refinement step limit                */
    size_t hbm_budget;    /* bytes this context may hold on the device; 0 = all */
    int offline_max_iter; /* local-stage CG iteration limit                    */
    double offline_rtol;  /* local-stage CG relative tolerance                 */
} mstress_opts;

/* Fill *o with defaults: FP64, rtol 1e-13, max_iter 20000, inner_rtol 0 (by precision),
   max_outer 30, hbm_budget 0, offline_max_iter 20000, offline_rtol 1e-13. */
int mstress_opts_default(mstress_opts* o);

/* ------------------------------------------------------------ context */
/* Create a context on the current CUDA device. cuda_stream is a cudaStream_t
   owned by the caller (NULL = the legacy default stream). */
int mstress_create(mstress_ctx* out, void* cuda_stream, const mstress_opts* opts);
int mstress_set_opts(mstress_ctx ctx, const mstress_opts* opts);
int mstress_get_opts(mstress_ctx ctx, mstress_opts* opts);
void mstress_free_ctx(mstress_ctx ctx);
const char* mstress_last_error(mstress_ctx ctx);
/* Bytes of device memory the context holds now, and the most it has held. */
int mstress_mem_info(mstress_ctx ctx, size_t* in_use, size_t* peak);
/* Wait for all work issued on the context's stream. */
int mstress_sync(mstress_ctx ctx);

/* ------------------------------------------------------- local stage
 * mstress_build_block: the one-shot local stage (section 4.2) on the GPU, FP64.
 * Assembles nothing: the fine operator is applied element by element (Q1 hex,
 * 2x2x2 Gauss, Eqs. 4-5). Solves the m+1 Dirichlet problems of Eqs. 13-15
 * (unit value at one Lagrange-node component, dT = 0; and zero boundary
 * values, dT = 1) together as one batched multi-right-hand-side PCG, then forms
 * A_element = F^T A F (Eq. 18), b_element = F^T b (Eq. 19, per unit dT), the
 * stress modes S (Eq. 1 at every Gauss point of every basis column; the last
 * column includes the thermal term) and their Gauss means.
 *   mesh:      geometry; mat_id NULL means voxelise with *tsv
 *   mats:      n_mat materials, indexed by mat_id values (voxeliser: 3: Si, Cu, SiO2)
 *   order:     face polynomial degree, n = order+1 nodes per axis, 1 <= order <= 7
 *   out:       new block handle (device resident)
 * Returns MSTRESS_ENOT_CONVERGED (and still the block) if the CG limit is hit. */
int mstress_build_block(mstress_ctx ctx, const mstress_block_mesh* mesh,
                        const mstress_tsv_geom* tsv, const mstress_material* mats,
                        int n_mat, int order, mstress_block* out);

/* Make a block from host arrays computed elsewhere (row-major FP64):
   K_r (m*m), b_r (m, per unit dT), S ((48*n_el)*(m+1), row (e*8+g)*6+comp),
   F (n_dof*(m+1), may be NULL: then U_NODE recovery is unavailable). */
int mstress_block_import(mstress_ctx ctx, const mstress_block_mesh* mesh, int order,
                         const double* K_r, const double* b_r, const double* S,
                         const double* F, mstress_block* out);

#define MSTRESS_BLOCK_KR     0   /* m*m          */
#define MSTRESS_BLOCK_BR     1   /* m            */
#define MSTRESS_BLOCK_S      2   /* 48*n_el*(m+1) */
#define MSTRESS_BLOCK_F      3   /* n_dof*(m+1)  */
#define MSTRESS_BLOCK_SMEAN  4   /* 6*n_el*(m+1): Gauss mean of S, row e*6+comp */
#define MSTRESS_BLOCK_SGRID  5   /* 6*side^2*(m+1): grid modes (mstress_block_grid), row p*6+comp */
/* Copy one block array to host memory (count = number of doubles in dst). */
int mstress_block_export(mstress_block blk, int what, double* dst, size_t count);
/* Gridded cut-plane output (the error measure of section 5.1 samples the von
   Mises stress on the plane through the half height of the blocks, on a
   100 x 100 grid per block). Builds the block's grid modes for side x side
   cell-centred points ((i + 1/2) lx/side, (j + 1/2) ly/side, lz/2), point
   p = i + side*j: the stress of Eq. 1 of every basis column of Eq. 15 at the
   point, evaluated in the fine element that holds it (trilinear shape
   functions at the point's local coordinates); a point on faces shared by
   elements takes the mean over those elements (the mean of the one-sided
   values of a stress that jumps there). Needs a block from
   mstress_build_block (materials and basis kept on the device); 1 <= side <=
   400; a later call with another side replaces the grid. Enables recovery
   output MSTRESS_VM_GRID for solutions whose blocks all have the same grid. */
int mstress_block_grid(mstress_block blk, int side);
/* m (element DOFs), n_el (fine elements), n_dof (fine DOFs), cg_iters (local stage). */
int mstress_block_info(mstress_block blk, int* m, int* n_el, int* n_dof, int* cg_iters);
/* Free a block model. Work the library issued on the context's stream is
   waited for; work that mstress_apply_noalloc issued on another stream with
   this block is not, so the caller must finish it first. */
void mstress_free_block(mstress_block blk);

/* ------------------------------------------------------- global stage
 * mstress_solve: assemble (implicitly) and solve Eq. 20 for one array by
 * Jacobi-preconditioned conjugate gradients, matrix free: each iteration
 * applies every block's A_element to its gathered element DOFs and sums the
 * element results into the shared lattice DOFs in a fixed order (bitwise
 * reproducible). The system is symmetric positive definite once a face is
 * clamped; the call fails with MSTRESS_EINVAL when no DOF is constrained. */
int mstress_solve(mstress_ctx ctx, const mstress_layout* layout, double dT,
                  const mstress_bc* bc, mstress_sol* out);

/* Solve n independent arrays in one batched solve: every PCG phase is one
   launch over all arrays, each array with its own scalars and stopping test.
   layouts[k], dT[k], bcs[k] (bcs may be NULL: bottom clamped). */
int mstress_solve_batch(mstress_ctx ctx, const mstress_layout* layouts, const double* dT,
                        const mstress_bc* bcs, int n, mstress_sol* out);

/* Recovery outputs (what). Arrays of a batch follow each other in order;
   within an array, blocks are in site order j*nx + i.
     COEFF     FP64  [block][m]        element DOFs c_e (reduced displacements)
     VM_ELEM   [block][n_el]           von Mises of the Gauss-mean stress per fine
               element; FP64 when the context precision is MSTRESS_FP64, FP32
               otherwise
     SIGMA_GP  [block][n_el*48]        Gauss-point stress S [c_e; dT] (Eq. 15 + Eq. 1);
               FP64 / FP32 as VM_ELEM
     U_NODE    FP64  [block][n_dof]    fine displacement F [c_e; dT] (Eq. 15)
     LATTICE   FP64  [X*Y*Z*3]         the global DOF vector u of Eq. 20 per array
     VM_GRID   [block][side^2]         von Mises on the half-height cut plane at the
               points of mstress_block_grid (section 5.1); FP64 / FP32 as VM_ELEM */
#define MSTRESS_COEFF    0
#define MSTRESS_VM_ELEM  1
#define MSTRESS_SIGMA_GP 2
#define MSTRESS_U_NODE   3
#define MSTRESS_LATTICE  4
#define MSTRESS_VM_GRID  5
/* Size in bytes that mstress_recover(what) writes for this solution. */
int mstress_recover_size(mstress_sol sol, int what, size_t* bytes);
/* Compute and write one recovery output into dst (device memory if
   dst_on_device, else host memory); dst_bytes must be at least the size. */
int mstress_recover(mstress_ctx ctx, mstress_sol sol, int what, void* dst,
                    size_t dst_bytes, int dst_on_device);

/* Per-array statistics: PCG iterations (inner iterations summed in the mixed
   modes), refinement steps, final relative FP64 residual ||b-Ax||/||b||,
   and status (MSTRESS_OK / _ENOT_CONVERGED / _ENUMERIC). */
int mstress_sol_info(mstress_sol sol, int array, int* iters, int* outer,
                     double* rel_res, int* status);
int mstress_sol_count(mstress_sol sol, int* n_arrays, int64_t* n_blocks);
/* How the solve's reduced-precision operator ran: *use_tc = 1 if on the
   tensor cores, *tc_tile = blocks per tensor-core tile (the M extent filled
   per MMA tile; 0 when the tensor cores are not used), *tuned = 1 if the tile
   autotuner picked it (solves of at least two blocks per SM; the choice is
   timed once per basis size, precision and batch-size class and then reused
   by the context). Any pointer may be NULL. */
int mstress_sol_tiling(mstress_sol sol, int* use_tc, int* tc_tile, int* tuned);
void mstress_free_sol(mstress_sol sol);

/* ------------------------------------------------------------ serving
 * Continuous batching of global-stage queries (not in the paper: a serving
 * layer over the global stage of section 4.3). A server owns a queue of
 * requests -- one array each (layout against resident block models, dT,
 * clamped faces) -- and solves every running request together as one batch by
 * FP64-residual iterative refinement (a step = one FP64 residual check for
 * every running array + one inner solve of the correction in the context's
 * precision). Between steps: arrays whose check stopped them retire (their
 * per-element von Mises field is recovered into the request), queued requests
 * are admitted in arrival order while at most max_slots run and the estimated
 * device footprint of running requests plus held results fits hbm_budget
 * (0 = unlimited), and the batch is rebuilt with every continuing array's
 * iterate. A request's arithmetic does not depend on the others, so its result
 * is the same alone and in the mix. Requests must share basis order and block
 * mesh size; prescribed displacements are not taken. Not thread safe. */
typedef struct mstress_server_s* mstress_server;
#define MSTRESS_RQ_QUEUED  0
#define MSTRESS_RQ_RUNNING 1
#define MSTRESS_RQ_DONE    2
#define MSTRESS_RQ_FAILED  3
int mstress_server_create(mstress_ctx ctx, int max_slots, size_t hbm_budget, mstress_server* out);
/* Queue a request; *id receives its handle. The layout is copied. */
int mstress_server_submit(mstress_server srv, const mstress_layout* layout, double dT, const mstress_bc* bc,
                          int64_t* id);
/* Admit, run one refinement step over the running batch, retire finished
   requests. Returns the queue length, running count and requests finished. */
int mstress_server_step(mstress_server srv, int* n_queued, int* n_running, int* n_finished);
/* Next finished (or failed) request not yet polled, 0 if none. */
int mstress_server_poll(mstress_server srv, int64_t* id);
/* State (MSTRESS_RQ_*), inner PCG iterations, refinement steps, final relative
   FP64 residual and latency from submit to retirement (ms, -1 while pending).
   Returns the request's status (MSTRESS_OK, _ENOT_CONVERGED, _ENUMERIC, or
   _ENOMEM if it can never fit the budget). */
int mstress_server_info(mstress_server srv, int64_t id, int* state, int* iters, int* outer, double* rel_res,
                        double* latency_ms);
/* Copy a finished request's von Mises field ([block][n_el], FP64 in FP64
   mode, else FP32) to dst (device if dst_on_device). */
int mstress_server_result(mstress_server srv, int64_t id, void* dst, size_t dst_bytes, int dst_on_device);
/* Forget a finished request and free its result. */
int mstress_server_release(mstress_server srv, int64_t id);
void mstress_free_server(mstress_server srv);

/* Bounded device waits. A grid-barrier wait of the persistent solver gives up
   after limit_ns nanoseconds of device time (default 2e9): the kernel records
   the failure, every CTA leaves, and the solve returns
   MSTRESS_EDEVICE_TIMEOUT; the context stays usable. withhold_next = 1 makes
   the next persistent solver launch on this context skip one CTA's first
   barrier arrival, once, so that the wait runs out: a test hook for the
   timeout path (no fault, no trap; every wait stays bounded). */
int mstress_set_wait_limit(mstress_ctx ctx, int64_t limit_ns, int withhold_next);

/* Row-strip partition of one array's global stage (section 4.3, Eq. 20) over
   `world` ranks: the plan of a solve split by block rows, in which each rank
   applies K_r to its own blocks, the lattice row on each strip boundary is
   summed across the two ranks whose blocks touch it, and the PCG scalars are
   summed over ranks. Host arithmetic only (no device call).
   For an array of ny block rows and basis order `order` (n = order + 1
   Lagrange nodes per axis, so block row j spans lattice rows j (n-1) ..
   (j+1)(n-1)), rank `rank` gets:
     j0, j1     its block rows [j0, j1): ny rows split as evenly as possible,
                lower ranks taking the extra rows;
     y_own0, y_own1  the lattice rows it owns, [y_own0, y_own1): from j0 (n-1)
                up to but excluding j1 (n-1), the last rank also the top row
                ny (n-1); every lattice row has exactly one owner;
     y_send     j1 (n-1), the row its blocks touch that rank + 1 owns: its
                partial interface sums there go to rank + 1, and rank + 1's
                values of the vector being applied there come back before each
                apply (-1 on the last rank);
     y_recv     j0 (n-1), the owned row for which it receives rank - 1's
                partial sums and to which it sends its values (-1 on rank 0);
     prev, next the neighbouring ranks (-1 where there is none).
   Returns MSTRESS_EINVAL for a NULL out, ny < 1, order outside [1, 7],
   world < 1, rank outside [0, world) or world > ny (every strip needs a block
   row). */
typedef struct {
    int j0, j1;
    int y_own0, y_own1;
    int y_send, y_recv;
    int prev, next;
} mstress_strip;

int mstress_strip_partition(int ny, int order, int world, int rank, mstress_strip* out);

/* Number of CUDA kernels this library has launched in this process (a graph
   replay counts its kernel nodes). For accounting in benchmarks. */
int mstress_launch_count(int64_t* n);

/* Time one kernel of a finished solve: reps launches between two CUDA events
   on the context stream, *avg_ms = mean duration of one launch. The kernel
   runs on the solution's own scratch vectors (the solution x is not touched).
     phase 0  operator apply (element products) in the solve's precision,
              gathering p and z as an iteration does (the kernel of the
              per-phase iteration of large batches; inside the persistent
              solver the same work is its phase A)
     phase 1  interface sum with the <p, q> partials
     phase 2  operator apply in FP64
     phase 3  von Mises recovery (contraction + epilogue) into scratch */
int mstress_profile(mstress_ctx ctx, mstress_sol sol, int phase, int reps, double* avg_ms);

/* Time spent inside the persistent solver's iterations of this solution,
   measured on the device at its grid barriers: ms4[0..2] = milliseconds in
   the element products, the interface sum and the vector update (summed over
   all iterations and refinement steps), ms4[3] = number of iterations. All
   zero when the solve ran the per-phase iteration (batches of at least 4096
   blocks on the streamed tensor-core apply). */
int mstress_sol_phase_ms(mstress_sol sol, double* ms4);

/* Apply the assembled reduced operator of a layout (one matrix-free K_r apply
   plus interface sum, the kernel pair of every PCG iteration):
   y = A_global x on the lattice vector (X*Y*Z*3 doubles, device pointers).
   precision MSTRESS_FP64: FP64 throughout. A reduced mode: x is rounded to
   FP32 and goes through the inner solver's operator (element products in the
   mode's operand format with FP32 accumulation, FP32 interface sum); y is the
   FP32 result widened. Constrained DOFs are not masked. For testing the
   operator in isolation. */
int mstress_apply(mstress_ctx ctx, const mstress_layout* layout, const double* x_dev,
                  double* y_dev, int precision);

/* Operator apply that allocates no memory (the paper has no counterpart; this
   is a service for callers that cannot allocate device memory when they need
   the operator: code inside a CUDA stream capture they do not own, loops whose
   memory is fixed up front, hosts whose allocator belongs to another runtime).
   Computes y = A_global x in FP64 for an nx*ny array whose sites all use the
   block model blk, with x and y device vectors on the lattice of that array
   (X*Y*Z*3 doubles, as in mstress_apply; constrained DOFs are not masked).
   Work is issued on cuda_stream (a cudaStream_t; NULL = legacy stream) and is
   not waited for. The only scratch, the element products, lives in a fixed
   32 MiB device array inside the library that every GPU loading the library
   holds until the process exits: nx*ny*round_up(m,16)*8 bytes must fit (e.g.
   at most 52428 blocks at m = 78, 13797 at m = 294), else MSTRESS_EINVAL.
   The first call on a device looks up that array's address; it must come
   before any stream capture, and on a stream that is being captured it is
   refused with MSTRESS_EINVAL. Later calls make no set-up call. The device
   of blk's context must be the current device (else MSTRESS_EINVAL). Every
   call shares the array and leaves its contents behind (nothing in it needs
   to start at zero); calls whose work may overlap on the GPU race on it and
   must be serialised by the caller. The call reads blk's K_r on cuda_stream
   without recording that use: the caller must let that work finish (e.g.
   cudaStreamSynchronize(cuda_stream)) before mstress_free_block(blk). */
int mstress_apply_noalloc(mstress_block blk, int nx, int ny, const double* x_dev, double* y_dev,
                          void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* MSTRESS_H */
