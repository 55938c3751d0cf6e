// One-shot local stage of MORE-Stress (section 4.2) on the GPU, all FP64.
//
// The unit block's fine operator is never assembled: every product A x is
// computed node by node from the 24x24 element matrices of the (at most
// kMaxMat) materials, which depend only on the material because the mesh is a
// structured box mesh. The m+1 Dirichlet problems of Eqs. 13-15 are solved
// together by one batched preconditioned conjugate-gradient run whose vectors
// hold all right-hand sides side by side ([node][component][column], column
// fastest, so a warp reads 32 right-hand sides of one DOF in one transaction).
// The preconditioner is the inverse of each node's 3x3 diagonal block.
#include <cmath>
#include <cstdio>

#include "internal.h"

namespace ms {
namespace {

constexpr int kRowNodes = 64;   // nodes per work chunk of the vector kernels
constexpr int kTY = 8;          // threads along nodes in a CTA (x: 32 columns)

// -------------------------------------------------------------- geometry
__global__ void k_voxelize(uint8_t* mat, int ex, int ey, int ez, double lx, double ly, double r_cu,
                           double t_liner) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ex * ey * ez) return;
    int kx = e % ex, ky = (e / ex) % ey;
    double cx = (kx + 0.5) * (lx / ex) - 0.5 * lx;
    double cy = (ky + 0.5) * (ly / ey) - 0.5 * ly;
    double r = sqrt(cx * cx + cy * cy);
    uint8_t id = 0;                               // Si
    if (r_cu > 0) {
        if (r <= r_cu + t_liner) id = 2;          // SiO2 liner
        if (r <= r_cu) id = 1;                    // Cu
    }
    mat[e] = id;
}

// B at the 8 Gauss points of a box element: Bg[g][row][3*l + c], Voigt rows
// (xx, yy, zz, xy, yz, zx), engineering shear; trilinear shape functions.
__global__ void k_bmat(double* Bg, double hx, double hy, double hz) {
    int t = threadIdx.x;   // 0..191: (g, l, c) -> one column of B at one Gauss point
    if (t >= 8 * 24) return;
    int g = t / 24, col = t % 24, l = col / 3, c = col % 3;
    const double gp = 1.0 / sqrt(3.0);
    double xi[3] = {(2 * (g & 1) - 1) * gp, (2 * ((g >> 1) & 1) - 1) * gp, (2 * ((g >> 2) & 1) - 1) * gp};
    double s[3] = {double(2 * (l & 1) - 1), double(2 * ((l >> 1) & 1) - 1), double(2 * ((l >> 2) & 1) - 1)};
    double h[3] = {hx, hy, hz};
    double f[3], grad[3];
    for (int d = 0; d < 3; ++d) f[d] = 0.5 * (1.0 + s[d] * xi[d]);
    for (int d = 0; d < 3; ++d) {
        double p = 0.5 * s[d] * (2.0 / h[d]);
        for (int e2 = 0; e2 < 3; ++e2)
            if (e2 != d) p *= f[e2];
        grad[d] = p;
    }
    double col6[6] = {0, 0, 0, 0, 0, 0};
    if (c == 0) { col6[0] = grad[0]; col6[3] = grad[1]; col6[5] = grad[2]; }
    if (c == 1) { col6[1] = grad[1]; col6[3] = grad[0]; col6[4] = grad[2]; }
    if (c == 2) { col6[2] = grad[2]; col6[4] = grad[1]; col6[5] = grad[0]; }
    for (int r = 0; r < 6; ++r) Bg[(g * 6 + r) * 24 + col] = col6[r];
}

struct MatTab {
    double lam[kMaxMat], mu[kMaxMat], tm[kMaxMat];   // Eq. 2 and alpha (3 lam + 2 mu)
};

// Ke[mat] = sum_g Bg^T D Bg detJ (Eq. 4), fe[mat] = sum_g Bg^T tm 1 detJ (Eq. 5).
__global__ void k_elem_mats(const double* Bg, MatTab mt, double detJ, double* Ke, double* fe) {
    int mat = blockIdx.x;
    double lam = mt.lam[mat], mu = mt.mu[mat], tm = mt.tm[mat];
    for (int t = threadIdx.x; t < 24 * 24; t += blockDim.x) {
        int i = t / 24, j = t % 24;
        double acc = 0;
        for (int g = 0; g < 8; ++g) {
            const double* B = Bg + g * 144;
            double bi[6], bj[6];
            for (int r = 0; r < 6; ++r) { bi[r] = B[r * 24 + i]; bj[r] = B[r * 24 + j]; }
            double tr = bj[0] + bj[1] + bj[2];
            // D bj: normal rows lam tr + 2 mu eps, shear rows mu gamma
            acc += bi[0] * (lam * tr + 2 * mu * bj[0]) + bi[1] * (lam * tr + 2 * mu * bj[1]) +
                   bi[2] * (lam * tr + 2 * mu * bj[2]) + mu * (bi[3] * bj[3] + bi[4] * bj[4] + bi[5] * bj[5]);
        }
        Ke[mat * 576 + t] = acc * detJ;
    }
    if (threadIdx.x < 24) {
        int i = threadIdx.x;
        double acc = 0;
        for (int g = 0; g < 8; ++g) {
            const double* B = Bg + g * 144;
            acc += tm * (B[0 * 24 + i] + B[1 * 24 + i] + B[2 * 24 + i]);
        }
        fe[mat * 24 + i] = acc * detJ;
    }
}

struct Mesh {
    int ex, ey, ez, NX, NY, NZ, n_nodes, n_mat;
};

__device__ __forceinline__ bool on_boundary(const Mesh& M, int vx, int vy, int vz) {
    return vx == 0 || vy == 0 || vz == 0 || vx == M.ex || vy == M.ey || vz == M.ez;
}

// Node-centric matrix-free product Y = A X over all columns (Eq. 6 operator):
// y_v = sum over elements e around v of sum over nodes w of e of Ke[mat e](v, w) x_w.
// interior_only: rows of boundary nodes are written as zero (the A_ff / A_f,bc rows).
// Optionally accumulates per-column partial dots <X, Y> for the CG step length.
// CTA: 32 columns x kTY threads, covering kRowNodes nodes of one column group.
__global__ void __launch_bounds__(256) k_local_apply(Mesh M, const uint8_t* __restrict__ mat,
                                                     const double* __restrict__ Ke_g, int NCP,
                                                     const double* __restrict__ X, double* __restrict__ Y,
                                                     int interior_only, double* partial_dot) {
    extern __shared__ double Ke[];   // n_mat * 576
    __shared__ double red[kTY][32];
    for (int t = threadIdx.y * 32 + threadIdx.x; t < M.n_mat * 576; t += 256) Ke[t] = Ke_g[t];
    __syncthreads();
    const int col = blockIdx.y * 32 + threadIdx.x;
    const int v0 = blockIdx.x * kRowNodes;
    double dot = 0;
    for (int v = v0 + threadIdx.y; v < min(v0 + kRowNodes, M.n_nodes); v += kTY) {
        int vx = v % M.NX, vy = (v / M.NX) % M.NY, vz = v / (M.NX * M.NY);
        double acc0 = 0, acc1 = 0, acc2 = 0;
        if (!(interior_only && on_boundary(M, vx, vy, vz))) {
            for (int dz = -1; dz <= 0; ++dz) {
                int kz = vz + dz;
                if (kz < 0 || kz >= M.ez) continue;
                for (int dy = -1; dy <= 0; ++dy) {
                    int ky = vy + dy;
                    if (ky < 0 || ky >= M.ey) continue;
                    for (int dx = -1; dx <= 0; ++dx) {
                        int kx = vx + dx;
                        if (kx < 0 || kx >= M.ex) continue;
                        int e = kx + M.ex * (ky + M.ey * kz);
                        int lv = (-dx) + 2 * (-dy) + 4 * (-dz);
                        const double* K = Ke + mat[e] * 576 + (3 * lv) * 24;
#pragma unroll
                        for (int lw = 0; lw < 8; ++lw) {
                            int w = (kx + (lw & 1)) + M.NX * ((ky + ((lw >> 1) & 1)) + M.NY * (kz + (lw >> 2)));
                            const double* xw = X + (size_t)w * 3 * NCP + col;
                            double x0 = xw[0], x1 = xw[NCP], x2 = xw[2 * NCP];
                            const double* k0 = K + 3 * lw;
                            acc0 += k0[0] * x0 + k0[1] * x1 + k0[2] * x2;
                            acc1 += k0[24] * x0 + k0[25] * x1 + k0[26] * x2;
                            acc2 += k0[48] * x0 + k0[49] * x1 + k0[50] * x2;
                        }
                    }
                }
            }
        }
        double* yv = Y + (size_t)v * 3 * NCP + col;
        yv[0] = acc0;
        yv[NCP] = acc1;
        yv[2 * NCP] = acc2;
        if (partial_dot) {
            const double* xv = X + (size_t)v * 3 * NCP + col;
            dot += xv[0] * acc0 + xv[NCP] * acc1 + xv[2 * NCP] * acc2;
        }
    }
    if (partial_dot) {
        red[threadIdx.y][threadIdx.x] = dot;
        __syncthreads();
        if (threadIdx.y == 0) {
            double s = 0;
            for (int t = 0; t < kTY; ++t) s += red[t][threadIdx.x];
            partial_dot[(size_t)blockIdx.x * NCP + col] = s;
        }
    }
}

// Thermal load per unit dT, node by node: b_v = sum over elements around v of fe[mat](v).
// Also the inverse of the node's 3x3 diagonal block (zero on boundary nodes).
__global__ void k_local_load_diag(Mesh M, const uint8_t* mat, const double* Ke, const double* fe,
                                  double* bfull, double* Minv) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= M.n_nodes) return;
    int vx = v % M.NX, vy = (v / M.NX) % M.NY, vz = v / (M.NX * M.NY);
    double b[3] = {0, 0, 0}, A[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int dz = -1; dz <= 0; ++dz)
        for (int dy = -1; dy <= 0; ++dy)
            for (int dx = -1; dx <= 0; ++dx) {
                int kx = vx + dx, ky = vy + dy, kz = vz + dz;
                if (kx < 0 || ky < 0 || kz < 0 || kx >= M.ex || ky >= M.ey || kz >= M.ez) continue;
                int e = kx + M.ex * (ky + M.ey * kz);
                int lv = (-dx) + 2 * (-dy) + 4 * (-dz);
                int mt = mat[e];
                for (int i = 0; i < 3; ++i) {
                    b[i] += fe[mt * 24 + 3 * lv + i];
                    for (int j = 0; j < 3; ++j) A[i * 3 + j] += Ke[mt * 576 + (3 * lv + i) * 24 + 3 * lv + j];
                }
            }
    for (int i = 0; i < 3; ++i) bfull[3 * v + i] = b[i];
    double inv[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (!on_boundary(M, vx, vy, vz)) {
        double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                     A[2] * (A[3] * A[7] - A[4] * A[6]);
        double id = 1.0 / det;
        inv[0] = (A[4] * A[8] - A[5] * A[7]) * id;
        inv[1] = (A[2] * A[7] - A[1] * A[8]) * id;
        inv[2] = (A[1] * A[5] - A[2] * A[4]) * id;
        inv[3] = (A[5] * A[6] - A[3] * A[8]) * id;
        inv[4] = (A[0] * A[8] - A[2] * A[6]) * id;
        inv[5] = (A[2] * A[3] - A[0] * A[5]) * id;
        inv[6] = (A[3] * A[7] - A[4] * A[6]) * id;
        inv[7] = (A[1] * A[6] - A[0] * A[7]) * id;
        inv[8] = (A[0] * A[4] - A[1] * A[3]) * id;
    }
    for (int i = 0; i < 9; ++i) Minv[9 * v + i] = inv[i];
}

// Lifted boundary data of Eq. 14: column 3q + c carries L_3D(r; q) (Eqs. 8-9)
// in component c on the boundary nodes; interior rows, the f_T column and
// padding columns are zero.
__global__ void k_lift(Mesh M, LocalMap lm, double lx, double ly, double lz, int NCP, double* U0) {
    int v = blockIdx.x;
    int col = threadIdx.x + blockIdx.y * blockDim.x;
    if (col >= NCP) return;
    int vx = v % M.NX, vy = (v / M.NX) % M.NY, vz = v / (M.NX * M.NY);
    double val = 0;
    int comp = col % 3;
    if (col < lm.m && on_boundary(M, vx, vy, vz)) {
        int q = col / 3, n = lm.n;
        double x[3] = {vx * (lx / M.ex), vy * (ly / M.ey), vz * (lz / M.ez)};
        double len[3] = {lx, ly, lz};
        int idx[3] = {lm.qa[q], lm.qb[q], lm.qc[q]};
        val = 1.0;
        for (int d = 0; d < 3; ++d) {
            double xi = len[d] * idx[d] / (n - 1);
            for (int j = 0; j < n; ++j) {
                if (j == idx[d]) continue;
                double xj = len[d] * j / (n - 1);
                val *= (x[d] - xj) / (xi - xj);
            }
        }
    }
    for (int c = 0; c < 3; ++c) U0[((size_t)v * 3 + c) * NCP + col] = (c == comp) ? val : 0.0;
}

// Right-hand sides: column i < m is -(A U0)_f (Eq. 14 with dT = 0), column m is
// b_f (dT = 1); boundary rows and padding columns are zero.
__global__ void k_rhs(Mesh M, int m, int NCP, const double* AU0, const double* bfull, double* R) {
    int v = blockIdx.x;
    int col = threadIdx.x + blockIdx.y * blockDim.x;
    if (col >= NCP) return;
    int vx = v % M.NX, vy = (v / M.NX) % M.NY, vz = v / (M.NX * M.NY);
    bool bnd = on_boundary(M, vx, vy, vz);
    for (int c = 0; c < 3; ++c) {
        size_t i = ((size_t)v * 3 + c) * NCP + col;
        double r = 0;
        if (!bnd) {
            if (col < m) r = -AU0[i];
            else if (col == m) r = bfull[3 * v + c];
        }
        R[i] = r;
    }
}

// ------------------------------------------------------ batched PCG vectors
struct ColState {
    double* rz;       // current <r, z> per column
    double* rr;       // current <r, r>
    double* tol2;     // rtol^2 <R, R>
    double* alpha;
    double* beta;
    int* active;
};

// z = Minv r (3x3 per node); optional x = 0, p = z; partial <r,z>, <r,r>.
__global__ void __launch_bounds__(256) k_cg_precond(Mesh M, int NCP, const double* Minv, const double* r,
                                                    double* z, double* p, double* x, double* prz, double* prr) {
    __shared__ double red[2][kTY][32];
    const int col = blockIdx.y * 32 + threadIdx.x;
    const int v0 = blockIdx.x * kRowNodes;
    double srz = 0, srr = 0;
    for (int v = v0 + threadIdx.y; v < min(v0 + kRowNodes, M.n_nodes); v += kTY) {
        const double* Mi = Minv + 9 * v;
        size_t b = (size_t)v * 3 * NCP + col;
        double r0 = r[b], r1 = r[b + NCP], r2 = r[b + 2 * NCP];
        double z0 = Mi[0] * r0 + Mi[1] * r1 + Mi[2] * r2;
        double z1 = Mi[3] * r0 + Mi[4] * r1 + Mi[5] * r2;
        double z2 = Mi[6] * r0 + Mi[7] * r1 + Mi[8] * r2;
        z[b] = z0; z[b + NCP] = z1; z[b + 2 * NCP] = z2;
        p[b] = z0; p[b + NCP] = z1; p[b + 2 * NCP] = z2;
        x[b] = 0; x[b + NCP] = 0; x[b + 2 * NCP] = 0;
        srz += r0 * z0 + r1 * z1 + r2 * z2;
        srr += r0 * r0 + r1 * r1 + r2 * r2;
    }
    red[0][threadIdx.y][threadIdx.x] = srz;
    red[1][threadIdx.y][threadIdx.x] = srr;
    __syncthreads();
    if (threadIdx.y == 0) {
        double a = 0, c = 0;
        for (int t = 0; t < kTY; ++t) { a += red[0][t][threadIdx.x]; c += red[1][t][threadIdx.x]; }
        prz[(size_t)blockIdx.x * NCP + col] = a;
        prr[(size_t)blockIdx.x * NCP + col] = c;
    }
}

// Sum per-column partials over the node chunks in a fixed order.
__device__ __forceinline__ double fold_col(const double* part, int n_chunks, int NCP, int col) {
    __shared__ double red[kTY][32];
    double s = 0;
    for (int c = threadIdx.y; c < n_chunks; c += kTY) s += part[(size_t)c * NCP + col];
    red[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    double t = 0;
    for (int k = 0; k < kTY; ++k) t += red[k][threadIdx.x];
    __syncthreads();
    return t;
}

__global__ void k_cg_init_scalars(int n_chunks, int NCP, int m1, const double* prz, const double* prr,
                                  double rtol, ColState cs) {
    const int col = blockIdx.x * 32 + threadIdx.x;
    double rz = fold_col(prz, n_chunks, NCP, col);
    double rr = fold_col(prr, n_chunks, NCP, col);
    if (threadIdx.y == 0) {
        cs.rz[col] = rz;
        cs.rr[col] = rr;
        cs.tol2[col] = rtol * rtol * rr;
        cs.active[col] = (col < m1 && rr > 0) ? 1 : 0;
    }
}

__global__ void k_cg_alpha(int n_chunks, int NCP, const double* ppq, ColState cs) {
    const int col = blockIdx.x * 32 + threadIdx.x;
    double pq = fold_col(ppq, n_chunks, NCP, col);
    if (threadIdx.y == 0) {
        double a = 0;
        if (cs.active[col] == 1) {
            a = cs.rz[col] / pq;
            if (!(pq > 0) || !isfinite(a)) { a = 0; cs.active[col] = -1; }   // breakdown
        }
        cs.alpha[col] = a;
    }
}

// x += alpha p, r -= alpha q, z = Minv r; partial <r,z>, <r,r>.
__global__ void __launch_bounds__(256) k_cg_update1(Mesh M, int NCP, const double* Minv, const double* alpha,
                                                    double* x, double* r, double* z, const double* p,
                                                    const double* q, double* prz, double* prr) {
    __shared__ double red[2][kTY][32];
    const int col = blockIdx.y * 32 + threadIdx.x;
    const int v0 = blockIdx.x * kRowNodes;
    const double a = alpha[col];
    double srz = 0, srr = 0;
    for (int v = v0 + threadIdx.y; v < min(v0 + kRowNodes, M.n_nodes); v += kTY) {
        size_t b = (size_t)v * 3 * NCP + col;
        double rv[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            size_t i = b + c * NCP;
            x[i] += a * p[i];
            rv[c] = r[i] - a * q[i];
            r[i] = rv[c];
        }
        const double* Mi = Minv + 9 * v;
        double z0 = Mi[0] * rv[0] + Mi[1] * rv[1] + Mi[2] * rv[2];
        double z1 = Mi[3] * rv[0] + Mi[4] * rv[1] + Mi[5] * rv[2];
        double z2 = Mi[6] * rv[0] + Mi[7] * rv[1] + Mi[8] * rv[2];
        z[b] = z0; z[b + NCP] = z1; z[b + 2 * NCP] = z2;
        srz += rv[0] * z0 + rv[1] * z1 + rv[2] * z2;
        srr += rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2];
    }
    red[0][threadIdx.y][threadIdx.x] = srz;
    red[1][threadIdx.y][threadIdx.x] = srr;
    __syncthreads();
    if (threadIdx.y == 0) {
        double s0 = 0, s1 = 0;
        for (int t = 0; t < kTY; ++t) { s0 += red[0][t][threadIdx.x]; s1 += red[1][t][threadIdx.x]; }
        prz[(size_t)blockIdx.x * NCP + col] = s0;
        prr[(size_t)blockIdx.x * NCP + col] = s1;
    }
}

// New <r,z>, <r,r> per column; beta; stopping test; any-active flag.
__global__ void k_cg_beta(int n_chunks, int NCP, const double* prz, const double* prr, ColState cs, int* any) {
    const int col = blockIdx.x * 32 + threadIdx.x;
    double rz = fold_col(prz, n_chunks, NCP, col);
    double rr = fold_col(prr, n_chunks, NCP, col);
    if (threadIdx.y == 0) {
        double b = 0;
        if (cs.active[col] == 1) {
            b = rz / cs.rz[col];
            cs.rz[col] = rz;
            cs.rr[col] = rr;
            if (!isfinite(rr) || !isfinite(b)) { cs.active[col] = -1; b = 0; }
            else if (rr <= cs.tol2[col]) cs.active[col] = 0;
            else atomicOr(any, 1);
        }
        cs.beta[col] = b;
    }
}

__global__ void __launch_bounds__(256) k_cg_update2(Mesh M, int NCP, const double* beta, const double* z, double* p) {
    const int col = blockIdx.y * 32 + threadIdx.x;
    const int v0 = blockIdx.x * kRowNodes;
    const double b = beta[col];
    for (int v = v0 + threadIdx.y; v < min(v0 + kRowNodes, M.n_nodes); v += kTY) {
        size_t i = (size_t)v * 3 * NCP + col;
        for (int c = 0; c < 3; ++c) p[i + c * NCP] = z[i + c * NCP] + b * p[i + c * NCP];
    }
}

__global__ void k_add(size_t n, double* a, const double* b) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) a[i] += b[i];
}

__global__ void k_set_col(int n_nodes, int NCP, int col, const double* bfull, double* Q) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 3 * n_nodes) Q[(size_t)i * NCP + col] = bfull[i];
}

// Partial G[i][j] = sum_rows F[row][i] * Q[row][j] over one row slab; i < mi, j < mj.
// CTA: 32x8 threads computing a 32x32 tile; grid (ceil(mj/32), ceil(mi/32), n_split).
__global__ void __launch_bounds__(256) k_atb(int rows, int NCP, int mi, int mj, int slab, const double* F,
                                             const double* Q, double* part) {
    __shared__ double Fs[32][33], Qs[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int j0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
    const int r_begin = blockIdx.z * slab, r_end = min(rows, r_begin + slab);
    double acc[4] = {0, 0, 0, 0};
    for (int r0 = r_begin; r0 < r_end; r0 += 32) {
        for (int k = ty; k < 32; k += 8) {
            int r = r0 + k;
            Fs[k][tx] = (r < r_end && i0 + tx < mi) ? F[(size_t)r * NCP + i0 + tx] : 0.0;
            Qs[k][tx] = (r < r_end && j0 + tx < mj) ? Q[(size_t)r * NCP + j0 + tx] : 0.0;
        }
        __syncthreads();
        for (int k = 0; k < 32; ++k) {
            double qv = Qs[k][tx];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] += Fs[k][ty * 4 + u] * qv;
        }
        __syncthreads();
    }
    const size_t ldp = (size_t)gridDim.x * 32;
    double* P = part + (size_t)blockIdx.z * gridDim.y * 32 * ldp;
    for (int u = 0; u < 4; ++u) P[(size_t)(i0 + ty * 4 + u) * ldp + j0 + tx] = acc[u];
}

// K_r = sym(G[:, :m]) (Eq. 18), b_r = G[:, m] (Eq. 19, per unit dT).
__global__ void k_atb_finish(int m, int n_split, size_t ldp, size_t plane, const double* part, double* Kr,
                             double* br) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * (m + 1)) return;
    int i = t / (m + 1), j = t % (m + 1);
    double s = 0, s2 = 0;
    for (int z = 0; z < n_split; ++z) {
        s += part[z * plane + (size_t)i * ldp + j];
        if (j < m) s2 += part[z * plane + (size_t)j * ldp + i];
    }
    if (j < m) Kr[i * m + j] = 0.5 * (s + s2);
    else br[i] = s;
}

// Stress modes at every Gauss point (Eq. 1 applied to each basis column of
// Eq. 15): S[(e*8+g)*6+c][col] = (D B_g F_e)[c] (minus alpha (3 lam + 2 mu) for
// the f_T column, which carries dT = 1), and their Gauss mean Smean[e*6+c][col].
__global__ void k_stress_modes(Mesh M, const uint8_t* mat, const double* Bg_g, MatTab mt, int m, int NCP, int ld,
                               const double* F, double* S, double* Smean) {
    __shared__ double Bg[8 * 144];
    for (int t = threadIdx.x; t < 8 * 144; t += blockDim.x) Bg[t] = Bg_g[t];
    __syncthreads();
    const int e = blockIdx.x;
    const int col = blockIdx.y * blockDim.x + threadIdx.x;
    if (col > m) return;
    int kx = e % M.ex, ky = (e / M.ex) % M.ey, kz = e / (M.ex * M.ey);
    double u[24];
    for (int l = 0; l < 8; ++l) {
        int w = (kx + (l & 1)) + M.NX * ((ky + ((l >> 1) & 1)) + M.NY * (kz + (l >> 2)));
        for (int c = 0; c < 3; ++c) u[3 * l + c] = F[((size_t)w * 3 + c) * NCP + col];
    }
    int k = mat[e];
    double lam = mt.lam[k], mu = mt.mu[k], th = (col == m) ? mt.tm[k] : 0.0;
    double mean[6] = {0, 0, 0, 0, 0, 0};
    for (int g = 0; g < 8; ++g) {
        double eps[6];
        for (int r = 0; r < 6; ++r) {
            double s = 0;
            for (int i = 0; i < 24; ++i) s += Bg[(g * 6 + r) * 24 + i] * u[i];
            eps[r] = s;
        }
        double tr = eps[0] + eps[1] + eps[2];
        double sig[6] = {lam * tr + 2 * mu * eps[0] - th, lam * tr + 2 * mu * eps[1] - th,
                         lam * tr + 2 * mu * eps[2] - th, mu * eps[3], mu * eps[4], mu * eps[5]};
        for (int r = 0; r < 6; ++r) {
            S[((size_t)(e * 8 + g) * 6 + r) * ld + col] = sig[r];
            mean[r] += sig[r];
        }
    }
    for (int r = 0; r < 6; ++r) Smean[((size_t)e * 6 + r) * ld + col] = mean[r] * 0.125;
}

// Elements of one axis holding coordinate x of [0, len] cut into ne equal
// elements: one element and its local coordinate in [-1, 1], or, on a face
// shared by two elements, both (at +1 and -1, weight 1/2 each), so that a
// stress that jumps across the face is read as the mean of its two one-sided
// values (the outer faces belong to their one element).
struct AxisPick {
    int n;
    int e[2];
    double xi[2];
    double w;
};

__device__ AxisPick axis_pick(double x, double len, int ne) {
    const double t = x / (len / ne);
    const double k = rint(t);
    AxisPick a;
    a.n = 0;
    if (fabs(t - k) <= 1e-9 * fmax(1.0, fabs(t))) {
        const int kk = (int)k;
        if (kk - 1 >= 0) { a.e[a.n] = kk - 1; a.xi[a.n] = 1.0; ++a.n; }
        if (kk <= ne - 1) { a.e[a.n] = kk; a.xi[a.n] = -1.0; ++a.n; }
        a.w = 1.0 / a.n;
    } else {
        int kk = (int)floor(t);
        kk = min(max(kk, 0), ne - 1);
        a.n = 1;
        a.e[0] = kk;
        a.xi[0] = 2.0 * (t - kk) - 1.0;
        a.w = 1.0;
    }
    return a;
}

// Stress modes at the points of the half-height cut plane (the gridded output
// of section 5.1): point p = i + side j at ((i + 1/2) lx / side, (j + 1/2) ly /
// side, lz / 2), basis column col: Sg[(p*6 + r)*ld + col] = (D B(xi) F_e)[r]
// of Eq. 1 in the element holding the point (minus alpha (3 lam + 2 mu) for
// the f_T column, which carries dT = 1), with B the strain of the trilinear
// shape functions at the point's local coordinates; on element faces the
// weighted mean over the elements meeting there (axis_pick per axis).
__global__ void k_grid_modes(Mesh M, const uint8_t* mat, MatTab mt, int m, int ld, const double* F, int side,
                             double lx, double ly, double lz, double* Sg) {
    const int p = blockIdx.x;
    const int col = blockIdx.y * blockDim.x + threadIdx.x;
    if (col > m) return;
    const int i = p % side, j = p / side;
    const AxisPick ax = axis_pick((i + 0.5) * lx / side, lx, M.ex);
    const AxisPick ay = axis_pick((j + 0.5) * ly / side, ly, M.ey);
    const AxisPick az = axis_pick(0.5 * lz, lz, M.ez);
    const double h[3] = {lx / M.ex, ly / M.ey, lz / M.ez};
    double sig[6] = {0, 0, 0, 0, 0, 0};
    for (int a = 0; a < ax.n; ++a)
        for (int b = 0; b < ay.n; ++b)
            for (int c = 0; c < az.n; ++c) {
                const int kx = ax.e[a], ky = ay.e[b], kz = az.e[c];
                const double xi[3] = {ax.xi[a], ay.xi[b], az.xi[c]};
                const double w = ax.w * ay.w * az.w;
                double eps[6] = {0, 0, 0, 0, 0, 0};
                for (int l = 0; l < 8; ++l) {
                    const double sgn[3] = {double(2 * (l & 1) - 1), double(2 * ((l >> 1) & 1) - 1),
                                           double(2 * ((l >> 2) & 1) - 1)};
                    double f[3], g[3];
                    for (int d = 0; d < 3; ++d) f[d] = 0.5 * (1.0 + sgn[d] * xi[d]);
                    for (int d = 0; d < 3; ++d) {
                        double q = 0.5 * sgn[d] * (2.0 / h[d]);
                        for (int d2 = 0; d2 < 3; ++d2)
                            if (d2 != d) q *= f[d2];
                        g[d] = q;
                    }
                    const int node = (kx + (l & 1)) + M.NX * ((ky + ((l >> 1) & 1)) + M.NY * (kz + (l >> 2)));
                    const double ux = F[((size_t)node * 3 + 0) * ld + col];
                    const double uy = F[((size_t)node * 3 + 1) * ld + col];
                    const double uz = F[((size_t)node * 3 + 2) * ld + col];
                    eps[0] += g[0] * ux;
                    eps[1] += g[1] * uy;
                    eps[2] += g[2] * uz;
                    eps[3] += g[1] * ux + g[0] * uy;
                    eps[4] += g[2] * uy + g[1] * uz;
                    eps[5] += g[2] * ux + g[0] * uz;
                }
                const int e = kx + M.ex * (ky + M.ey * kz);
                const int k = mat[e];
                const double lam = mt.lam[k], mu = mt.mu[k], th = (col == m) ? mt.tm[k] : 0.0;
                const double tr = eps[0] + eps[1] + eps[2];
                sig[0] += w * (lam * tr + 2 * mu * eps[0] - th);
                sig[1] += w * (lam * tr + 2 * mu * eps[1] - th);
                sig[2] += w * (lam * tr + 2 * mu * eps[2] - th);
                sig[3] += w * (mu * eps[3]);
                sig[4] += w * (mu * eps[4]);
                sig[5] += w * (mu * eps[5]);
            }
    for (int r = 0; r < 6; ++r) Sg[((size_t)p * 6 + r) * ld + col] = sig[r];
}

// Gauss mean of imported stress modes.
__global__ void k_smean(int n_el, int m1, int ld, const double* S, double* Smean) {
    size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t >= (size_t)n_el * 6 * m1) return;
    int col = t % m1;
    size_t er = t / m1;
    int e = er / 6, r = er % 6;
    double s = 0;
    for (int g = 0; g < 8; ++g) s += S[((size_t)(e * 8 + g) * 6 + r) * ld + col];
    Smean[er * ld + col] = s * 0.125;
}

}  // namespace

void build_grid_modes(mstress_block blk, int side) {
    MS_REQUIRE(side >= 1 && side <= 400, MSTRESS_EINVAL, "grid side must be in [1, 400]");
    MS_REQUIRE(blk->has_mat && blk->has_F, MSTRESS_EINVAL,
               "gridded output needs a block built by mstress_build_block (materials and basis on the device)");
    if (blk->grid_side == side) return;
    for (auto& d : blk->Sgrid_lp) d.reset();
    for (auto& d : blk->Sgrid_tc) d.reset();
    const int n_grid = side * side;
    alloc_into(blk->ctx, blk->Sgrid, (size_t)6 * n_grid * blk->ld * sizeof(double));
    MatTab mt;
    std::memset(&mt, 0, sizeof(mt));
    for (int k = 0; k < kMaxMat; ++k) {
        mt.lam[k] = blk->mat_lam[k];
        mt.mu[k] = blk->mat_mu[k];
        mt.tm[k] = blk->mat_tm[k];
    }
    Mesh M{blk->ex, blk->ey, blk->ez, blk->ex + 1, blk->ey + 1, blk->ez + 1, blk->n_nodes, 0};
    k_grid_modes<<<dim3(n_grid, (blk->m1 + 31) / 32), 32, 0, blk->ctx->stream>>>(
        M, blk->mat_id.as<uint8_t>(), mt, blk->m, blk->ld, blk->F.as<double>(), side, blk->lx, blk->ly, blk->lz,
        blk->Sgrid.as<double>());
    MS_LAUNCH_CHECK();
    blk->grid_side = side;
    blk->n_grid = n_grid;
}

void block_compute_smean(mstress_block blk) {
    size_t n = (size_t)blk->n_el * 6 * blk->m1;
    k_smean<<<(unsigned)((n + 255) / 256), 256, 0, blk->ctx->stream>>>(blk->n_el, blk->m1, blk->ld,
                                                                          blk->S.as<double>(), blk->Smean.as<double>());
    MS_LAUNCH_CHECK();
}

int build_block(mstress_ctx ctx, const mstress_block_mesh* mesh, const mstress_tsv_geom* tsv,
                const mstress_material* mats, int n_mat, int order, mstress_block* out) {
    MS_REQUIRE(mesh, MSTRESS_EINVAL, "mesh is NULL");
    MS_REQUIRE(mesh->ex >= 1 && mesh->ey >= 1 && mesh->ez >= 1, MSTRESS_EINVAL, "mesh needs >= 1 element per axis");
    MS_REQUIRE((int64_t)(mesh->ex + 1) * (mesh->ey + 1) * (mesh->ez + 1) <= (1 << 22), MSTRESS_EINVAL,
               "mesh too large");
    MS_REQUIRE(mesh->lx > 0 && mesh->ly > 0 && mesh->lz > 0, MSTRESS_EINVAL, "block lengths must be positive");
    MS_REQUIRE(mats && n_mat >= 1 && n_mat <= kMaxMat, MSTRESS_EINVAL, "need 1..16 materials");
    MS_REQUIRE(mesh->mat_id || tsv, MSTRESS_EINVAL, "need mat_id or a TSV geometry");
    MS_REQUIRE(order >= 1 && order <= kMaxN - 1, MSTRESS_EINVAL, "basis order must be in [1, 7]");
    MS_REQUIRE(order <= mesh->ex && order <= mesh->ey && order <= mesh->ez, MSTRESS_EINVAL,
               "basis order exceeds the elements per axis");
    for (int k = 0; k < n_mat; ++k)
        MS_REQUIRE(mats[k].E > 0 && mats[k].nu > -1 && mats[k].nu < 0.5, MSTRESS_EINVAL,
                   "material needs E > 0 and -1 < nu < 0.5");

    cudaStream_t st = ctx->stream;
    LocalMap lm = make_local_map(order + 1);
    std::unique_ptr<mstress_block_s> blk(new mstress_block_s());
    mstress_block_s& B = *blk;
    B.ctx = ctx;
    B.n = order + 1;
    B.m = lm.m;
    B.m1 = lm.m + 1;
    B.ld = (int)round_up(B.m1, 8);
    B.ex = mesh->ex; B.ey = mesh->ey; B.ez = mesh->ez;
    B.lx = mesh->lx; B.ly = mesh->ly; B.lz = mesh->lz;
    B.n_el = B.ex * B.ey * B.ez;
    B.n_nodes = (B.ex + 1) * (B.ey + 1) * (B.ez + 1);
    B.n_dof = 3 * B.n_nodes;
    const int m = B.m, m1 = B.m1, ld = B.ld;
    const int NCP = (int)round_up(m1, 32);
    Mesh M{B.ex, B.ey, B.ez, B.ex + 1, B.ey + 1, B.ez + 1, B.n_nodes, n_mat};

    DBuf d_mat, Bg, Ke, fe, bfull, Minv, U0, X, R, Z, P, Q, prz, prr, ppq, cols;
    alloc_into(ctx, d_mat, B.n_el);
    if (mesh->mat_id) {
        for (int e = 0; e < B.n_el; ++e)
            MS_REQUIRE(mesh->mat_id[e] < n_mat, MSTRESS_EINVAL, "mat_id out of range");
        MS_CUDA(cudaMemcpyAsync(d_mat.ptr, mesh->mat_id, B.n_el, cudaMemcpyHostToDevice, st));
    } else {
        MS_REQUIRE(n_mat >= 3, MSTRESS_EINVAL, "the TSV voxeliser needs materials 0 = Si, 1 = Cu, 2 = SiO2");
        MS_REQUIRE(tsv->r_cu <= 0 || tsv->t_liner >= 0, MSTRESS_EINVAL, "negative liner thickness");
        k_voxelize<<<(B.n_el + 255) / 256, 256, 0, st>>>(d_mat.as<uint8_t>(), B.ex, B.ey, B.ez, B.lx, B.ly,
                                                         tsv->r_cu, tsv->t_liner);
        MS_LAUNCH_CHECK();
    }
    MatTab mt;
    std::memset(&mt, 0, sizeof(mt));
    for (int k = 0; k < n_mat; ++k) {   // Eq. 2 (host side only packs the table the kernels use)
        double E = mats[k].E, nu = mats[k].nu;
        mt.lam[k] = E * nu / (1.0 + nu) / (1.0 - 2.0 * nu);
        mt.mu[k] = E / 2.0 / (1.0 + nu);
        mt.tm[k] = mats[k].alpha * (3.0 * mt.lam[k] + 2.0 * mt.mu[k]);
    }
    const double hx = B.lx / B.ex, hy = B.ly / B.ey, hz = B.lz / B.ez;
    alloc_into(ctx, Bg, 8 * 144 * sizeof(double));
    alloc_into(ctx, Ke, (size_t)n_mat * 576 * sizeof(double));
    alloc_into(ctx, fe, (size_t)n_mat * 24 * sizeof(double));
    k_bmat<<<1, 192, 0, st>>>(Bg.as<double>(), hx, hy, hz);
    MS_LAUNCH_CHECK();
    k_elem_mats<<<n_mat, 256, 0, st>>>(Bg.as<double>(), mt, hx * hy * hz / 8.0, Ke.as<double>(), fe.as<double>());
    MS_LAUNCH_CHECK();
    alloc_into(ctx, bfull, (size_t)B.n_dof * sizeof(double));
    alloc_into(ctx, Minv, (size_t)B.n_nodes * 9 * sizeof(double));
    k_local_load_diag<<<(B.n_nodes + 127) / 128, 128, 0, st>>>(M, d_mat.as<uint8_t>(), Ke.as<double>(),
                                                                fe.as<double>(), bfull.as<double>(), Minv.as<double>());
    MS_LAUNCH_CHECK();

    const size_t vbytes = (size_t)B.n_dof * NCP * sizeof(double);
    alloc_into(ctx, U0, vbytes, false);
    alloc_into(ctx, X, vbytes, false);
    alloc_into(ctx, R, vbytes, false);
    alloc_into(ctx, Z, vbytes, false);
    alloc_into(ctx, P, vbytes, false);
    alloc_into(ctx, Q, vbytes, false);
    const int n_chunks = (B.n_nodes + kRowNodes - 1) / kRowNodes;
    alloc_into(ctx, prz, (size_t)n_chunks * NCP * sizeof(double));
    alloc_into(ctx, prr, (size_t)n_chunks * NCP * sizeof(double));
    alloc_into(ctx, ppq, (size_t)n_chunks * NCP * sizeof(double));
    alloc_into(ctx, cols, (size_t)NCP * (5 * sizeof(double) + sizeof(int)) + 64);
    ColState cs;
    cs.rz = cols.as<double>();
    cs.rr = cs.rz + NCP;
    cs.tol2 = cs.rr + NCP;
    cs.alpha = cs.tol2 + NCP;
    cs.beta = cs.alpha + NCP;
    cs.active = reinterpret_cast<int*>(cs.beta + NCP);
    int* d_any = cs.active + NCP;

    dim3 gcol(NCP / 32, kTY);
    dim3 blk2(32, kTY);
    dim3 gvec(n_chunks, NCP / 32);
    dim3 gnode(B.n_nodes, (NCP + 31) / 32);
    const size_t ke_smem = (size_t)n_mat * 576 * sizeof(double);
    if (ke_smem > 48 * 1024)
        MS_CUDA(cudaFuncSetAttribute(k_local_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ke_smem));

    k_lift<<<gnode, 32, 0, st>>>(M, lm, B.lx, B.ly, B.lz, NCP, U0.as<double>());
    MS_LAUNCH_CHECK();
    k_local_apply<<<gvec, blk2, ke_smem, st>>>(M, d_mat.as<uint8_t>(), Ke.as<double>(), NCP, U0.as<double>(),
                                               Q.as<double>(), 1, nullptr);
    MS_LAUNCH_CHECK();
    k_rhs<<<gnode, 32, 0, st>>>(M, m, NCP, Q.as<double>(), bfull.as<double>(), R.as<double>());
    MS_LAUNCH_CHECK();
    k_cg_precond<<<gvec, blk2, 0, st>>>(M, NCP, Minv.as<double>(), R.as<double>(), Z.as<double>(), P.as<double>(),
                                        X.as<double>(), prz.as<double>(), prr.as<double>());
    MS_LAUNCH_CHECK();
    k_cg_init_scalars<<<NCP / 32, blk2, 0, st>>>(n_chunks, NCP, m1, prz.as<double>(), prr.as<double>(),
                                                 ctx->opts.offline_rtol, cs);
    MS_LAUNCH_CHECK();

    const int max_it = ctx->opts.offline_max_iter;
    const int chunk = 16;
    int it = 0;
    bool done = false;
    while (!done && it < max_it) {
        MS_CUDA(cudaMemsetAsync(d_any, 0, sizeof(int), st));
        int nk = std::min(chunk, max_it - it);
        for (int k = 0; k < nk; ++k) {
            k_local_apply<<<gvec, blk2, ke_smem, st>>>(M, d_mat.as<uint8_t>(), Ke.as<double>(), NCP,
                                                       P.as<double>(), Q.as<double>(), 1, ppq.as<double>());
            k_cg_alpha<<<NCP / 32, blk2, 0, st>>>(n_chunks, NCP, ppq.as<double>(), cs);
            k_cg_update1<<<gvec, blk2, 0, st>>>(M, NCP, Minv.as<double>(), cs.alpha, X.as<double>(), R.as<double>(),
                                                Z.as<double>(), P.as<double>(), Q.as<double>(), prz.as<double>(),
                                                prr.as<double>());
            k_cg_beta<<<NCP / 32, blk2, 0, st>>>(n_chunks, NCP, prz.as<double>(), prr.as<double>(), cs, d_any);
            k_cg_update2<<<gvec, blk2, 0, st>>>(M, NCP, cs.beta, Z.as<double>(), P.as<double>());
        }
        MS_LAUNCH_CHECK();
        it += nk;
        MS_CUDA(cudaMemcpyAsync(ctx->h_flag, d_any, sizeof(int), cudaMemcpyDeviceToHost, st));
        MS_CUDA(cudaStreamSynchronize(st));
        done = ctx->h_flag[0] == 0;
    }
    std::vector<int> act(NCP);
    MS_CUDA(cudaMemcpyAsync(act.data(), cs.active, NCP * sizeof(int), cudaMemcpyDeviceToHost, st));
    MS_CUDA(cudaStreamSynchronize(st));
    int status = MSTRESS_OK;
    for (int c = 0; c < m1; ++c) {
        if (act[c] < 0) status = MSTRESS_ENUMERIC;
        else if (act[c] > 0 && status == MSTRESS_OK) status = MSTRESS_ENOT_CONVERGED;
    }
    B.cg_iters = it;

    // F = lift + interior solution (Eq. 15 basis on the fine mesh)
    {
        size_t n = (size_t)B.n_dof * NCP;
        k_add<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, U0.as<double>(), X.as<double>());
        MS_LAUNCH_CHECK();
    }
    // Q = A F on every row, then column m := b_local, so F^T Q gives K_r and b_r together
    k_local_apply<<<gvec, blk2, ke_smem, st>>>(M, d_mat.as<uint8_t>(), Ke.as<double>(), NCP, U0.as<double>(),
                                               Q.as<double>(), 0, nullptr);
    MS_LAUNCH_CHECK();
    k_set_col<<<(B.n_dof + 255) / 256, 256, 0, st>>>(B.n_nodes, NCP, m, bfull.as<double>(), Q.as<double>());
    MS_LAUNCH_CHECK();
    {
        const int slab = 2048;
        const int n_split = (B.n_dof + slab - 1) / slab;
        dim3 g((m1 + 31) / 32, (m + 31) / 32, n_split);
        const size_t ldp = (size_t)g.x * 32, plane = (size_t)g.y * 32 * ldp;
        DBuf part;
        alloc_into(ctx, part, (size_t)n_split * plane * sizeof(double), false);
        k_atb<<<g, dim3(32, 8), 0, st>>>(B.n_dof, NCP, m, m1, slab, U0.as<double>(), Q.as<double>(),
                                         part.as<double>());
        MS_LAUNCH_CHECK();
        alloc_into(ctx, B.Kr, (size_t)m * m * sizeof(double), false);
        alloc_into(ctx, B.br, (size_t)m * sizeof(double), false);
        k_atb_finish<<<(m * m1 + 255) / 256, 256, 0, st>>>(m, n_split, ldp, plane, part.as<double>(),
                                                            B.Kr.as<double>(), B.br.as<double>());
        MS_LAUNCH_CHECK();
        MS_CUDA(cudaStreamSynchronize(st));
    }
    alloc_into(ctx, B.S, (size_t)48 * B.n_el * ld * sizeof(double));
    alloc_into(ctx, B.Smean, (size_t)6 * B.n_el * ld * sizeof(double));
    k_stress_modes<<<dim3(B.n_el, (m1 + 31) / 32), 32, 0, st>>>(M, d_mat.as<uint8_t>(), Bg.as<double>(), mt, m,
                                                                NCP, ld, U0.as<double>(), B.S.as<double>(),
                                                                B.Smean.as<double>());
    MS_LAUNCH_CHECK();
    alloc_into(ctx, B.F, (size_t)B.n_dof * ld * sizeof(double));
    MS_CUDA(cudaMemcpy2DAsync(B.F.ptr, ld * sizeof(double), U0.ptr, NCP * sizeof(double), m1 * sizeof(double),
                              B.n_dof, cudaMemcpyDeviceToDevice, st));
    B.has_F = true;
    B.mat_id = std::move(d_mat);   // kept for point evaluations (gridded output)
    for (int k = 0; k < kMaxMat; ++k) {
        B.mat_lam[k] = mt.lam[k];
        B.mat_mu[k] = mt.mu[k];
        B.mat_tm[k] = mt.tm[k];
    }
    B.has_mat = true;
    MS_CUDA(cudaStreamSynchronize(st));
    *out = blk.release();
    if (status != MSTRESS_OK)
        ctx->last_error = status == MSTRESS_ENUMERIC ? "local-stage CG breakdown" : "local-stage CG did not converge";
    return status;
}

}  // namespace ms
