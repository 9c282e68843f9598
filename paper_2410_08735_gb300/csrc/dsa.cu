// DSA preconditioner (paper appendix A, extended to the 2D X-Y geometry axis by axis), applied through
// one multigrid V-cycle per call.
//
// Operators on the DG space of an instance, per axis d (D_C: central flux, D_J: jump, exterior traces
// zero on the boundary), with D_j = sum_d Omega_d (D_C,d - sign(Omega_d)/2 D_J,d):
//   K = Sigma_a - sum_d kappa_d D_J,d - sum_d 3 mu2_d^2 D_C,d B_d^{-1} D_C,d
//   mu2_d = sum w Omega_d^2,  kappa_d = sum_{Omega_d>0} w Omega_d,  c_de = sum w Omega_d^2 |Omega_e|
//   B_d^{-1} = 1 / (3 mu2_d sigma_t)                                    partially consistent (default)
//   B_d^{-1} = cell-diagonal block of (3 mu2_d Sigma_t - 3/2 sum_e c_de D_J,e), inverted: a diagonal,
//              3 mu2_d sigma_t + 3/2 sum_e c_de (2 or 6)/h_e by the dof's degree along e
//                                                                      lumped fully consistent
// M_DSA^{-1} v = v + x,  x ~ K^{-1} Sigma_s v (the 0th-moment equation of the appendix).
//
// The approximate solve (the paper uses algebraic multigrid without fixing the cycle): one V-cycle.
//   DG level: x = omega Kcc^{-1} b (4x4 cell-block Jacobi), r = b - K x, coarse correction,
//             x += omega Kcc^{-1} (b - K x).
//   Level 1: continuous bilinear functions on the same mesh, embedded by P_c (vertex values -> Legendre
//            coefficients of the bilinear interpolant).  For a continuous u, D_C,d P_c u is cell-local
//            (interior central fluxes cancel the integration by parts; boundary faces keep half their
//            own trace) and D_J,d P_c u lives on boundary faces only, so the Galerkin operator P_c^T K P_c
//            is assembled from 4x4 element matrices E_T computed per cell.
//   Level l+1: the mesh coarsened by 2 per axis (while both counts are even and the mesh has more than
//            4 cells); bilinear interpolation nests the spaces, so the Galerkin element matrix of a coarse
//            cell is the sum over its 4 children of I^T E_child I.
//   Vertex levels: one damped point-Jacobi step before and after the coarse correction; the coarsest
//            level (<= kMaxCoarse vertices) is solved with its dense inverse, formed at set-up.
// FP32 throughout.  Set-up once per parameter set (k_dsa_setup_cells over every cell of every instance,
// k_dsa_setup_levels one block per instance), then k_dsa_vcycle once per preconditioner apply, one
// cluster of blocks per instance (hardware cluster barriers only: no spin-waits).
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "internal.h"

namespace rte {

namespace {

constexpr int kMaxLevels = 16;
constexpr int kMaxCoarse = 100;
constexpr int kThreads = 512;         // per block of the V-cycle cluster
constexpr int kCluster = 8;           // blocks per instance in the V-cycle
constexpr int kClusterVerts = 2048;   // vertex levels at least this large are split over the cluster
constexpr int kSetupThreads = 256;
constexpr float kSqrt3 = 1.7320508075688772f;

struct DsaInst {
  int nx, ny;                  // DG mesh (cells)
  int L;                       // vertex levels 1..L (L = coarsest)
  float hx, hy;
  long long o_sgs, o_sga, o_binv, o_kinv, o_b0, o_x0, o_t, o_r0;
  int ncx[kMaxLevels + 1], ncy[kMaxLevels + 1];
  long long o_E[kMaxLevels + 1], o_dinv[kMaxLevels + 1], o_u[kMaxLevels + 1], o_b[kMaxLevels + 1],
      o_r[kMaxLevels + 1];
  long long o_ainv;
};

struct DsaConst {
  float mu2[2], kappa[2], c[2][2];
  float omega, omega_v;
  int lumped;
};

// 1D axis factors of the orthonormal Legendre basis on a cell of width h: traces at the low and high
// ends and the volume term int p_1' p_0 = 2 sqrt(3) / h (the only nonzero entry).
struct Axis {
  float lo0, lo1, hi0, hi1, v10;
  __device__ explicit Axis(float h) {
    const float s = rsqrtf(h);
    lo0 = s;
    lo1 = -kSqrt3 * s;
    hi0 = s;
    hi1 = kSqrt3 * s;
    v10 = 2.f * kSqrt3 / h;
  }
};

// local dof of (degree a along axis d, transverse degree t)
__device__ __forceinline__ int dof_of(int d, int a, int t) { return d == 0 ? a + 2 * t : t + 2 * a; }

__device__ __forceinline__ void traces(const float* X, int d, float f0, float f1, float* T) {
#pragma unroll
  for (int t = 0; t < 2; ++t) T[t] = f0 * X[dof_of(d, 0, t)] + f1 * X[dof_of(d, 1, t)];
}

// (D_C,d X) on a cell from its own values and those of its low / high neighbours along d (absent
// neighbours: exterior trace zero).
__device__ void dc_cell(const float* Xc, const float* Xl, const float* Xh, bool has_l, bool has_h, int d,
                        const Axis& ax, float* out) {
  float Tl[2], Th[2], Nl[2] = {0.f, 0.f}, Nh[2] = {0.f, 0.f};
  traces(Xc, d, ax.lo0, ax.lo1, Tl);
  traces(Xc, d, ax.hi0, ax.hi1, Th);
  if (has_l) traces(Xl, d, ax.hi0, ax.hi1, Nl);
  if (has_h) traces(Xh, d, ax.lo0, ax.lo1, Nh);
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const float al = 0.5f * (Tl[t] + Nl[t]), ah = 0.5f * (Th[t] + Nh[t]);
    out[dof_of(d, 0, t)] = -ax.lo0 * al + ax.hi0 * ah;
    out[dof_of(d, 1, t)] = -ax.v10 * Xc[dof_of(d, 0, t)] - ax.lo1 * al + ax.hi1 * ah;
  }
}

// (D_J,d X) on a cell: -sum over its two faces of [X] [eta_k], [f] = f(high side) - f(low side).
__device__ void dj_cell(const float* Xc, const float* Xl, const float* Xh, bool has_l, bool has_h, int d,
                        const Axis& ax, float* out) {
  float Tl[2], Th[2], Nl[2] = {0.f, 0.f}, Nh[2] = {0.f, 0.f};
  traces(Xc, d, ax.lo0, ax.lo1, Tl);
  traces(Xc, d, ax.hi0, ax.hi1, Th);
  if (has_l) traces(Xl, d, ax.hi0, ax.hi1, Nl);
  if (has_h) traces(Xh, d, ax.lo0, ax.lo1, Nh);
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const float jl = Tl[t] - Nl[t], jh = Nh[t] - Th[t];
    out[dof_of(d, 0, t)] = -ax.lo0 * jl + ax.hi0 * jh;
    out[dof_of(d, 1, t)] = -ax.lo1 * jl + ax.hi1 * jh;
  }
}

// For a continuous function with DG coefficients X on a cell: D_C,d (cell-local; boundary faces keep
// half their own trace) and -D_J,d (boundary faces only).
__device__ void dc_cont(const float* X, bool has_l, bool has_h, int d, const Axis& ax, float* out) {
  float Tl[2], Th[2];
  traces(X, d, ax.lo0, ax.lo1, Tl);
  traces(X, d, ax.hi0, ax.hi1, Th);
  const float fl = has_l ? 1.f : 0.5f, fh = has_h ? 1.f : 0.5f;
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    out[dof_of(d, 0, t)] = -ax.lo0 * fl * Tl[t] + ax.hi0 * fh * Th[t];
    out[dof_of(d, 1, t)] = -ax.v10 * X[dof_of(d, 0, t)] - ax.lo1 * fl * Tl[t] + ax.hi1 * fh * Th[t];
  }
}
__device__ void mdj_cont(const float* X, bool has_l, bool has_h, int d, const Axis& ax, float* out) {
  float Tl[2], Th[2];
  traces(X, d, ax.lo0, ax.lo1, Tl);
  traces(X, d, ax.hi0, ax.hi1, Th);
  const float fl = has_l ? 0.f : 1.f, fh = has_h ? 0.f : 1.f;
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    out[dof_of(d, 0, t)] = ax.lo0 * fl * Tl[t] + ax.hi0 * fh * Th[t];
    out[dof_of(d, 1, t)] = ax.lo1 * fl * Tl[t] + ax.hi1 * fh * Th[t];
  }
}

__device__ __forceinline__ void load4(const float* p, float* x) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  x[0] = v.x;
  x[1] = v.y;
  x[2] = v.z;
  x[3] = v.w;
}
__device__ __forceinline__ void store4(float* p, const float* x) {
  *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
}

// P_c on one cell: Legendre coefficient k = a + 2b of the bilinear interpolant from corner q = vx + 2vy:
// F_x[a][vx] F_y[b][vy], F(h) = [[sqrt(h)/2, sqrt(h)/2], [-sqrt(h)/(2 sqrt 3), sqrt(h)/(2 sqrt 3)]].
__device__ __forceinline__ float pc_entry(int k, int q, float hx, float hy) {
  const int a = k & 1, b = k >> 1, vx = q & 1, vy = q >> 1;
  const float rx = sqrtf(hx), ry = sqrtf(hy);
  const float fx = a == 0 ? 0.5f * rx : (vx ? 1.f : -1.f) * rx / (2.f * kSqrt3);
  const float fy = b == 0 ? 0.5f * ry : (vy ? 1.f : -1.f) * ry / (2.f * kSqrt3);
  return fx * fy;
}

// neighbour bookkeeping of DG cell c = iy*nx + ix along axis d
struct Nb {
  bool l, h;
  int cl, ch;
};
__device__ __forceinline__ Nb nb_of(int ix, int iy, int nx, int ny, int d) {
  Nb n;
  if (d == 0) {
    n.l = ix > 0;
    n.h = ix < nx - 1;
    n.cl = iy * nx + max(ix - 1, 0);
    n.ch = iy * nx + min(ix + 1, nx - 1);
  } else {
    n.l = iy > 0;
    n.h = iy < ny - 1;
    n.cl = max(iy - 1, 0) * nx + ix;
    n.ch = min(iy + 1, ny - 1) * nx + ix;
  }
  return n;
}

// L2 loads of data written earlier in the same launch by other thread blocks of the cluster (the L1 of an
// SM is not coherent with the others)
__device__ __forceinline__ float ldg2(const float* p) { return __ldcg(p); }
__device__ __forceinline__ void load4cg(const float* p, float* x) {
  const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
  x[0] = v.x;
  x[1] = v.y;
  x[2] = v.z;
  x[3] = v.w;
}

template <bool CG>
__device__ __forceinline__ float ldv(const float* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

// y = A_l u at vertex (ix, iy) of a level with ncx x ncy cells and element matrices E [cells][4][4]
template <bool CG>
__device__ float vertex_apply(const float* E, const float* u, int ncx, int ncy, int ix, int iy) {
  const int nvx = ncx + 1;
  float y = 0.f;
#pragma unroll
  for (int sy = 0; sy < 2; ++sy) {
    const int cy = iy - 1 + sy;
    if (cy < 0 || cy >= ncy) continue;
#pragma unroll
    for (int sx = 0; sx < 2; ++sx) {
      const int cx = ix - 1 + sx;
      if (cx < 0 || cx >= ncx) continue;
      const int qv = (ix - cx) + 2 * (iy - cy);
      float e[4];
      load4(E + ((size_t)(cy * ncx + cx) * 16 + qv * 4), e);
      const int v0 = cy * nvx + cx;
      y += e[0] * ldv<CG>(u + v0) + e[1] * ldv<CG>(u + v0 + 1) + e[2] * ldv<CG>(u + v0 + nvx) +
           e[3] * ldv<CG>(u + v0 + nvx + 1);
    }
  }
  return y;
}

// B_d^{-1} of one cell (4 dofs) from its sigma_t
__device__ __forceinline__ void binv_of(float st, int d, const DsaConst& k, const float* hs, float* out) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float Bv = 3.f * k.mu2[d] * st;
    if (k.lumped)
#pragma unroll
      for (int e = 0; e < 2; ++e) Bv += 1.5f * k.c[d][e] * (((q >> e) & 1) ? 6.f : 2.f) / hs[e];
    out[q] = Bv > 0.f ? 1.f / Bv : 0.f;   // a void cell carries no diffusion
  }
}

// ----------------------------------------------------------------------------------------------- set-up
// Per cell, every instance at once (grid [cells / kSetupThreads, B]): cross sections, B_d^{-1}, the
// inverted 4x4 diagonal block of K and the level-1 element matrix.  Neighbours' B^{-1} are recomputed
// from their sigma_t, so cells are independent.
__global__ void __launch_bounds__(kSetupThreads) k_dsa_setup_cells(const DsaInst* dinfo, float* base,
                                                                   const double* sig_s, const double* sig_t, int R,
                                                                   int rx, int ry, DsaConst k) {
  const int b = blockIdx.y;
  const DsaInst& di = dinfo[b];
  const int nx = di.nx, ny = di.ny, nc = nx * ny;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const int cxr = nx / rx, cyr = ny / ry;
  const float hs[2] = {di.hx, di.hy};
  auto st_of = [&](int cell) {
    const int ix = cell % nx, iy = cell / nx;
    return (float)sig_t[(size_t)b * R + (iy / cyr) * rx + ix / cxr];
  };
  const int ix = c % nx, iy = c / nx;
  const int reg = (iy / cyr) * rx + ix / cxr;
  const float ss = (float)sig_s[(size_t)b * R + reg];
  const float st = (float)sig_t[(size_t)b * R + reg];
  const float sa = st - ss;
  base[di.o_sgs + c] = ss;
  base[di.o_sga + c] = sa;
  float bc[2][4];
  binv_of(st, 0, k, hs, bc[0]);
  binv_of(st, 1, k, hs, bc[1]);
  for (int d = 0; d < 2; ++d)
    for (int q = 0; q < 4; ++q) base[di.o_binv + (size_t)c * 8 + d * 4 + q] = bc[d][q];
  const Axis ax[2] = {Axis(di.hx), Axis(di.hy)};
  const float zero4[4] = {0.f, 0.f, 0.f, 0.f};
  // diagonal block of K, column by column: K e_col restricted to this cell
  float Kc[16];
  for (int col = 0; col < 4; ++col) {
    float e[4] = {0.f, 0.f, 0.f, 0.f};
    e[col] = 1.f;
    float out[4];
    for (int q = 0; q < 4; ++q) out[q] = sa * e[q];
    for (int d = 0; d < 2; ++d) {
      const Nb n = nb_of(ix, iy, nx, ny, d);
      float tmp[4];
      dj_cell(e, zero4, zero4, n.l, n.h, d, ax[d], tmp);
      for (int q = 0; q < 4; ++q) out[q] -= k.kappa[d] * tmp[q];
      // Y = B^{-1} D_C e on this cell and its neighbours (e lives on this cell only)
      float Yc[4], Yl[4] = {0.f, 0.f, 0.f, 0.f}, Yh[4] = {0.f, 0.f, 0.f, 0.f}, bn[4];
      dc_cell(e, zero4, zero4, n.l, n.h, d, ax[d], Yc);
      for (int q = 0; q < 4; ++q) Yc[q] *= bc[d][q];
      if (n.l) {
        dc_cell(zero4, zero4, e, true, true, d, ax[d], Yl);
        binv_of(st_of(n.cl), d, k, hs, bn);
        for (int q = 0; q < 4; ++q) Yl[q] *= bn[q];
      }
      if (n.h) {
        dc_cell(zero4, e, zero4, true, true, d, ax[d], Yh);
        binv_of(st_of(n.ch), d, k, hs, bn);
        for (int q = 0; q < 4; ++q) Yh[q] *= bn[q];
      }
      dc_cell(Yc, Yl, Yh, n.l, n.h, d, ax[d], tmp);
      const float f = 3.f * k.mu2[d] * k.mu2[d];
      for (int q = 0; q < 4; ++q) out[q] -= f * tmp[q];
    }
    for (int q = 0; q < 4; ++q) Kc[q * 4 + col] = out[q];
  }
  // Gauss-Jordan inverse in place (symmetric positive definite: no pivoting)
  for (int p = 0; p < 4; ++p) {
    const float piv = 1.f / Kc[p * 4 + p];
    Kc[p * 4 + p] = 1.f;
    for (int q = 0; q < 4; ++q) Kc[p * 4 + q] *= piv;
    for (int r = 0; r < 4; ++r) {
      if (r == p) continue;
      const float f = Kc[r * 4 + p];
      Kc[r * 4 + p] = 0.f;
      for (int q = 0; q < 4; ++q) Kc[r * 4 + q] -= f * Kc[p * 4 + q];
    }
  }
  for (int q = 0; q < 16; ++q) base[di.o_kinv + (size_t)c * 16 + q] = Kc[q];
  // element matrix: P^T (sigma_a + sum_e kappa_e J_e) P + sum_d 3 mu2_d^2 (G_d P)^T B_d^{-1} (G_d P)
  float Pq[4][4], M[4][4], G[2][4][4];
  for (int q = 0; q < 4; ++q) {
    for (int kk = 0; kk < 4; ++kk) Pq[q][kk] = pc_entry(kk, q, di.hx, di.hy);
    for (int kk = 0; kk < 4; ++kk) M[q][kk] = sa * Pq[q][kk];
    for (int d = 0; d < 2; ++d) {
      const Nb n = nb_of(ix, iy, nx, ny, d);
      float tmp[4];
      mdj_cont(Pq[q], n.l, n.h, d, ax[d], tmp);
      for (int kk = 0; kk < 4; ++kk) M[q][kk] += k.kappa[d] * tmp[kk];
      dc_cont(Pq[q], n.l, n.h, d, ax[d], G[d][q]);
    }
  }
  float* E1 = base + di.o_E[1];
  for (int q = 0; q < 4; ++q)
    for (int q2 = 0; q2 < 4; ++q2) {
      float s = 0.f;
      for (int kk = 0; kk < 4; ++kk) s += Pq[q][kk] * M[q2][kk];
      for (int d = 0; d < 2; ++d) {
        const float f = 3.f * k.mu2[d] * k.mu2[d];
        for (int kk = 0; kk < 4; ++kk) s += f * G[d][q][kk] * bc[d][kk] * G[d][q2][kk];
      }
      E1[(size_t)c * 16 + q * 4 + q2] = s;
    }
}

// Per instance (one block): coarse element matrices, inverse diagonals and the dense inverse of the
// coarsest level.
__global__ void __launch_bounds__(kSetupThreads) k_dsa_setup_levels(const DsaInst* dinfo, float* base) {
  __shared__ float A[kMaxCoarse * kMaxCoarse];
  const int b = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
  const DsaInst& di = dinfo[b];
  // coarse element matrices: sum over the 4 children of I^T E_child I
  for (int l = 2; l <= di.L; ++l) {
    const int ncx = di.ncx[l], ncy = di.ncy[l], fcx = di.ncx[l - 1];
    const float* Ef = base + di.o_E[l - 1];
    float* Ec = base + di.o_E[l];
    for (int cc = tid; cc < ncx * ncy; cc += nth) {
      const int CX = cc % ncx, CY = cc / ncx;
      float acc[16];
      for (int q = 0; q < 16; ++q) acc[q] = 0.f;
      for (int s = 0; s < 4; ++s) {
        const int sx = s & 1, sy = s >> 1;
        const float* e = Ef + (size_t)((2 * CY + sy) * fcx + 2 * CX + sx) * 16;
        // I[child corner][coarse corner] = w(Vx, (sx+vx)/2) w(Vy, (sy+vy)/2), w(0,t) = 1-t, w(1,t) = t
        float I[4][4];
        for (int qc = 0; qc < 4; ++qc) {
          const float tx = 0.5f * (sx + (qc & 1)), ty = 0.5f * (sy + (qc >> 1));
          for (int Q = 0; Q < 4; ++Q) I[qc][Q] = ((Q & 1) ? tx : 1.f - tx) * ((Q >> 1) ? ty : 1.f - ty);
        }
        float EI[4][4];
        for (int r = 0; r < 4; ++r)
          for (int Q = 0; Q < 4; ++Q) {
            float s2 = 0.f;
            for (int q = 0; q < 4; ++q) s2 += e[r * 4 + q] * I[q][Q];
            EI[r][Q] = s2;
          }
        for (int P = 0; P < 4; ++P)
          for (int Q = 0; Q < 4; ++Q) {
            float s2 = 0.f;
            for (int r = 0; r < 4; ++r) s2 += I[r][P] * EI[r][Q];
            acc[P * 4 + Q] += s2;
          }
      }
      for (int q = 0; q < 16; ++q) Ec[(size_t)cc * 16 + q] = acc[q];
    }
    __syncthreads();
  }
  // inverse diagonals of the vertex levels above the coarsest
  for (int l = 1; l < di.L; ++l) {
    const int ncx = di.ncx[l], ncy = di.ncy[l], nvx = ncx + 1, nv = nvx * (ncy + 1);
    const float* E = base + di.o_E[l];
    float* dinv = base + di.o_dinv[l];
    for (int v = tid; v < nv; v += nth) {
      const int ix = v % nvx, iy = v / nvx;
      float s = 0.f;
      for (int sy = 0; sy < 2; ++sy)
        for (int sx = 0; sx < 2; ++sx) {
          const int cx = ix - 1 + sx, cy = iy - 1 + sy;
          if (cx < 0 || cx >= ncx || cy < 0 || cy >= ncy) continue;
          const int qv = (ix - cx) + 2 * (iy - cy);
          s += E[(size_t)(cy * ncx + cx) * 16 + qv * 5];
        }
      dinv[v] = 1.f / s;
    }
  }
  // dense inverse of the coarsest level (Gauss-Jordan in shared memory, one row per thread)
  const int l = di.L, ncx = di.ncx[l], ncy = di.ncy[l], nvx = ncx + 1, n = nvx * (ncy + 1);
  const float* E = base + di.o_E[l];
  for (int idx = tid; idx < n * n; idx += nth) {
    const int i = idx / n, j = idx % n;
    const int ix = i % nvx, iy = i / nvx, jx = j % nvx, jy = j / nvx;
    float s = 0.f;
    if (abs(ix - jx) <= 1 && abs(iy - jy) <= 1)
      for (int cy = max(iy, jy) - 1; cy <= min(iy, jy); ++cy)
        for (int cx = max(ix, jx) - 1; cx <= min(ix, jx); ++cx) {
          if (cx < 0 || cx >= ncx || cy < 0 || cy >= ncy) continue;
          const int qi = (ix - cx) + 2 * (iy - cy), qj = (jx - cx) + 2 * (jy - cy);
          s += E[(size_t)(cy * ncx + cx) * 16 + qi * 4 + qj];
        }
    A[idx] = s;
  }
  for (int p = 0; p < n; ++p) {
    __syncthreads();
    const float piv = 1.f / A[p * n + p];
    const float fcol = tid < n ? A[tid * n + p] : 0.f;
    __syncthreads();
    if (tid < n) A[p * n + tid] = (tid == p ? 1.f : A[p * n + tid]) * piv;
    __syncthreads();
    if (tid < n && tid != p)
      for (int j = 0; j < n; ++j) A[tid * n + j] = (j == p ? 0.f : A[tid * n + j]) - fcol * A[p * n + j];
  }
  __syncthreads();
  float* ainv = base + di.o_ainv;
  for (int idx = tid; idx < n * n; idx += nth) ainv[idx] = A[idx];
}

// ---------------------------------------------------------------------------------------------- V-cycle
// One cluster of kCluster blocks per instance.  The DG stages and the vertex levels with at least
// kClusterVerts vertices are split over the cluster (barrier: cluster.sync, which orders the global
// writes; data written in this launch is read through L2); the smaller levels and the coarsest solve
// are done by block 0 alone.
namespace cg = cooperative_groups;

template <typename TV>
__global__ void __launch_bounds__(kThreads) k_dsa_vcycle(const InstInfo* inst, const DsaInst* dinfo, float* base,
                                                         DsaConst k, const TV* v, TV* z, const int* active,
                                                         const int* only) {
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int b = blockIdx.x / CS, tid = threadIdx.x, nth = blockDim.x;
  if (active && !active[b]) return;   // uniform over the cluster
  if (only && !only[b]) return;
  const int gt = rank * nth + tid, gn = CS * nth;
  __shared__ float Pc[16];
  const DsaInst& di = dinfo[b];
  const InstInfo in = inst[b];
  const int nx = di.nx, ny = di.ny, nc = nx * ny;
  const float* sgs = base + di.o_sgs;
  const float* sga = base + di.o_sga;
  const float* binv = base + di.o_binv;
  const float* kinv = base + di.o_kinv;
  float* b0 = base + di.o_b0;
  float* x0 = base + di.o_x0;
  float* t = base + di.o_t;
  float* r0 = base + di.o_r0;
  const TV* vb = v + in.off;
  TV* zb = z + in.off;
  const Axis ax[2] = {Axis(di.hx), Axis(di.hy)};
  const float om = k.omega, omv = k.omega_v;
  if (tid < 16) Pc[tid] = pc_entry(tid >> 2, tid & 3, di.hx, di.hy);   // [k][q]
  __syncthreads();
  // first vertex level handled by block 0 alone
  int lsplit = di.L;
  for (int l = 1; l < di.L; ++l)
    if ((di.ncx[l] + 1) * (di.ncy[l] + 1) < kClusterVerts) {
      lsplit = l;
      break;
    }

  // K x0 on cell c from x0 and t (= B^{-1} D_C x0 per axis)
  auto Kx = [&](int c, float* out) {
    const int ix = c % nx, iy = c / nx;
    float xc[4];
    load4cg(x0 + (size_t)c * 4, xc);
    for (int q = 0; q < 4; ++q) out[q] = sga[c] * xc[q];
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      const Nb n = nb_of(ix, iy, nx, ny, d);
      float xl[4], xh[4], tc[4], tl[4], th[4], tmp[4];
      load4cg(x0 + (size_t)n.cl * 4, xl);
      load4cg(x0 + (size_t)n.ch * 4, xh);
      dj_cell(xc, xl, xh, n.l, n.h, d, ax[d], tmp);
#pragma unroll
      for (int q = 0; q < 4; ++q) out[q] -= k.kappa[d] * tmp[q];
      const float* td = t + (size_t)d * nc * 4;
      load4cg(td + (size_t)c * 4, tc);
      load4cg(td + (size_t)n.cl * 4, tl);
      load4cg(td + (size_t)n.ch * 4, th);
      dc_cell(tc, tl, th, n.l, n.h, d, ax[d], tmp);
      const float f = 3.f * k.mu2[d] * k.mu2[d];
#pragma unroll
      for (int q = 0; q < 4; ++q) out[q] -= f * tmp[q];
    }
  };
  auto stage_t = [&]() {
    for (int c = gt; c < nc; c += gn) {
      const int ix = c % nx, iy = c / nx;
      float xc[4];
      load4cg(x0 + (size_t)c * 4, xc);
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        const Nb n = nb_of(ix, iy, nx, ny, d);
        float xl[4], xh[4], out[4], bi[4];
        load4cg(x0 + (size_t)n.cl * 4, xl);
        load4cg(x0 + (size_t)n.ch * 4, xh);
        dc_cell(xc, xl, xh, n.l, n.h, d, ax[d], out);
        load4(binv + (size_t)c * 8 + d * 4, bi);
#pragma unroll
        for (int q = 0; q < 4; ++q) out[q] *= bi[q];
        store4(t + ((size_t)d * nc + c) * 4, out);
      }
    }
  };
  // Vertex levels.  On entry to level l, b_l and the pre-smoothed u_l = omega D^{-1} b_l are stored
  // (written by the restriction into l).  descend: r_l = b_l - A u_l, then restriction into l+1 (with its
  // pre-smoothing).  ascend: u_l += P (u_{l+1} + omega D^{-1} r_{l+1}), the post-smoothing of level l+1
  // folded into the interpolation (none on the coarsest), then r_l = b_l - A u_l.  The post-smoothing
  // of level 1 is folded into the interpolation to the DG level.  CG: every load through L2 (stages split
  // over the cluster); otherwise block 0 alone, plain loads except those of b and u on the first level
  // of block 0, written by the cluster (ecg: through L2, since an L1 line may hold stale bytes).
  auto descend = [&](int l, int t0, int tn, auto sync, auto cgtag, bool ecg) {
    constexpr bool CG = decltype(cgtag)::value;
    const int ncx = di.ncx[l], ncy = di.ncy[l], nvx = ncx + 1, nv = nvx * (ncy + 1);
    const float* E = base + di.o_E[l];
    float* u = base + di.o_u[l];
    const float* bl = base + di.o_b[l];
    float* rl = base + di.o_r[l];
    if (CG || ecg)
      for (int vv = t0; vv < nv; vv += tn) rl[vv] = __ldcg(bl + vv) - vertex_apply<true>(E, u, ncx, ncy, vv % nvx, vv / nvx);
    else
      for (int vv = t0; vv < nv; vv += tn) rl[vv] = bl[vv] - vertex_apply<false>(E, u, ncx, ncy, vv % nvx, vv / nvx);
    sync();
    // full-weighting restriction (transpose of bilinear interpolation) and pre-smoothing of level l+1
    const int Cx = di.ncx[l + 1], Cy = di.ncy[l + 1], nCx = Cx + 1, nC = nCx * (Cy + 1);
    float* bc = base + di.o_b[l + 1];
    float* uc = base + di.o_u[l + 1];
    const float* dinvc = base + di.o_dinv[l + 1];
    const bool smooth_next = l + 1 < di.L;
    for (int V = t0; V < nC; V += tn) {
      const int I = V % nCx, J = V / nCx;
      float s = 0.f;
      for (int dj = -1; dj <= 1; ++dj) {
        const int fy = 2 * J + dj;
        if (fy < 0 || fy > ncy) continue;
        for (int dii = -1; dii <= 1; ++dii) {
          const int fx = 2 * I + dii;
          if (fx < 0 || fx > ncx) continue;
          s += (dii == 0 ? 1.f : 0.5f) * (dj == 0 ? 1.f : 0.5f) * ldv<CG>(rl + fy * nvx + fx);
        }
      }
      bc[V] = s;
      if (smooth_next) uc[V] = omv * dinvc[V] * s;
    }
    sync();
  };
  auto ascend = [&](int l, int t0, int tn, auto sync, auto cgtag, bool ecg) {
    constexpr bool CG = decltype(cgtag)::value;
    const int ncx = di.ncx[l], ncy = di.ncy[l], nvx = ncx + 1, nv = nvx * (ncy + 1);
    const int nCx = di.ncx[l + 1] + 1;
    const float* uc = base + di.o_u[l + 1];
    const float* rc = base + di.o_r[l + 1];
    const float* dinvc = base + di.o_dinv[l + 1];
    const float ws = l + 1 < di.L ? omv : 0.f;   // post-smoothing weight of level l+1
    const float* E = base + di.o_E[l];
    float* u = base + di.o_u[l];
    const float* bl = base + di.o_b[l];
    float* rl = base + di.o_r[l];
    auto ucf = [&](int V) { return ldv<CG>(uc + V) + (ws != 0.f ? ws * dinvc[V] * ldv<CG>(rc + V) : 0.f); };
    for (int vv = t0; vv < nv; vv += tn) {
      // bilinear interpolation: the coarse neighbours of an even index coincide
      const int ix = vv % nvx, iy = vv / nvx;
      const int x0i = ix >> 1, y0i = iy >> 1, x1i = (ix + 1) >> 1, y1i = (iy + 1) >> 1;
      const float uo = (CG || ecg) ? __ldcg(u + vv) : u[vv];
      u[vv] = uo + 0.25f * (ucf(y0i * nCx + x0i) + ucf(y0i * nCx + x1i) + ucf(y1i * nCx + x0i) + ucf(y1i * nCx + x1i));
    }
    sync();
    for (int vv = t0; vv < nv; vv += tn)
      rl[vv] = ((CG || ecg) ? __ldcg(bl + vv) : bl[vv]) - vertex_apply<CG>(E, u, ncx, ncy, vv % nvx, vv / nvx);
    sync();
  };
  auto csync = [&]() { cl.sync(); };
  auto bsync = [&]() { __syncthreads(); };
  using CgOn = std::integral_constant<bool, true>;
  using CgOff = std::integral_constant<bool, false>;

  // A: b0 = Sigma_s v, x0 = omega Kcc^{-1} b0
  for (int c = gt; c < nc; c += gn) {
    float bc[4], xc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) bc[q] = sgs[c] * (float)vb[(size_t)c * 4 + q];
    store4(b0 + (size_t)c * 4, bc);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      float kr[4];
      load4(kinv + (size_t)c * 16 + r * 4, kr);
      xc[r] = om * (kr[0] * bc[0] + kr[1] * bc[1] + kr[2] * bc[2] + kr[3] * bc[3]);
    }
    store4(x0 + (size_t)c * 4, xc);
  }
  cl.sync();
  stage_t();
  cl.sync();
  // C: r0 = b0 - K x0
  for (int c = gt; c < nc; c += gn) {
    float kx[4], bc[4];
    Kx(c, kx);
    load4cg(b0 + (size_t)c * 4, bc);
#pragma unroll
    for (int q = 0; q < 4; ++q) kx[q] = bc[q] - kx[q];
    store4(r0 + (size_t)c * 4, kx);
  }
  cl.sync();
  // D: restriction to level 1, b1_v = sum over the cells around v of (P_T^T r0_T)_v
  {
    const int nvx = nx + 1, nv = nvx * (ny + 1);
    float* b1 = base + di.o_b[1];
    for (int vv = gt; vv < nv; vv += gn) {
      const int ix = vv % nvx, iy = vv / nvx;
      float s = 0.f;
      for (int sy = 0; sy < 2; ++sy)
        for (int sx = 0; sx < 2; ++sx) {
          const int cx = ix - 1 + sx, cy = iy - 1 + sy;
          if (cx < 0 || cx >= nx || cy < 0 || cy >= ny) continue;
          const int qv = (ix - cx) + 2 * (iy - cy);
          float rc[4];
          load4cg(r0 + (size_t)(cy * nx + cx) * 4, rc);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) s += Pc[kk * 4 + qv] * rc[kk];
        }
      b1[vv] = s;
      if (di.L > 1) base[di.o_u[1] + vv] = omv * base[di.o_dinv[1] + vv] * s;
    }
  }
  cl.sync();
  for (int l = 1; l < lsplit; ++l) descend(l, gt, gn, csync, CgOn{}, true);
  if (rank == 0) {
    for (int l = lsplit; l < di.L; ++l) descend(l, tid, nth, bsync, CgOff{}, l == lsplit);
    // coarsest: dense inverse (b_L from the cluster when nothing was left to block 0)
    const int l = di.L, nvx = di.ncx[l] + 1, n = nvx * (di.ncy[l] + 1);
    const float* ainv = base + di.o_ainv;
    const float* bl = base + di.o_b[l];
    float* u = base + di.o_u[l];
    for (int i = tid; i < n; i += nth) {
      float s = 0.f;
      if (lsplit == di.L)
        for (int j = 0; j < n; ++j) s += ainv[(size_t)i * n + j] * __ldcg(bl + j);
      else
        for (int j = 0; j < n; ++j) s += ainv[(size_t)i * n + j] * bl[j];
      u[i] = s;
    }
    __syncthreads();
    for (int l2 = di.L - 1; l2 >= lsplit; --l2) ascend(l2, tid, nth, bsync, CgOff{}, l2 == lsplit);
  }
  cl.sync();
  for (int l = lsplit - 1; l >= 1; --l) ascend(l, gt, gn, csync, CgOn{}, true);
  // E: x0 += P_c (u1 + omega D^{-1} r1), the post-smoothing of level 1 folded in
  {
    const float* u1 = base + di.o_u[1];
    const float* r1 = base + di.o_r[1];
    const float* d1 = base + di.o_dinv[1];
    const float w1 = di.L > 1 ? omv : 0.f;
    const int nvx = nx + 1;
    auto uf = [&](int vv) { return ldg2(u1 + vv) + (w1 != 0.f ? w1 * d1[vv] * ldg2(r1 + vv) : 0.f); };
    for (int c = gt; c < nc; c += gn) {
      const int ix = c % nx, iy = c / nx;
      const int v0 = iy * nvx + ix;
      const float uq[4] = {uf(v0), uf(v0 + 1), uf(v0 + nvx), uf(v0 + nvx + 1)};
      float xc[4];
      load4cg(x0 + (size_t)c * 4, xc);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
#pragma unroll
        for (int q = 0; q < 4; ++q) xc[kk] += Pc[kk * 4 + q] * uq[q];
      store4(x0 + (size_t)c * 4, xc);
    }
  }
  cl.sync();
  stage_t();
  cl.sync();
  // G: z = v + x0 + omega Kcc^{-1} (b0 - K x0)
  for (int c = gt; c < nc; c += gn) {
    float kx[4], bc[4], xc[4];
    Kx(c, kx);
    load4cg(b0 + (size_t)c * 4, bc);
    load4cg(x0 + (size_t)c * 4, xc);
#pragma unroll
    for (int q = 0; q < 4; ++q) kx[q] = bc[q] - kx[q];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      float kr[4];
      load4(kinv + (size_t)c * 16 + r * 4, kr);
      const float x = xc[r] + om * (kr[0] * kx[0] + kr[1] * kx[1] + kr[2] * kx[2] + kr[3] * kx[3]);
      zb[(size_t)c * 4 + r] = vb[(size_t)c * 4 + r] + (TV)x;
    }
  }
}

// ------------------------------------------------------------------------------------------------ 1D slab
// In the slab the DSA systems are small and banded, so they are solved exactly.  Unknowns per cell c:
// x_c = (dphi_c0, dphi_c1, dJ_c0, dJ_c1); the two moment equations of appendix A,
//   (Sigma_a - kappa D_J) dphi + 3 mu2 D_C dJ = Sigma_s v,   mu2 D_C dphi + B dJ = 0,
// with B = 3 mu2 Sigma_t - 3/2 c D_J (fully consistent), its cell-diagonal blocks (lumped) or 3 mu2 Sigma_t
// (partially consistent), are block tridiagonal in the cells with 4x4 blocks (D_C and D_J couple a cell to its two
// neighbours only).  Eliminating dJ from the partially consistent form gives the appendix's
// K_PC = Sigma_a - kappa D_J - mu2 D_C Sigma_t^{-1} D_C exactly.  Block LU without inter-block pivoting (block
// Thomas), partial pivoting inside each 4x4 inversion, FP64, one thread per instance: the factors
// G_c^{-1} and M_c = L_c G_{c-1}^{-1} at set-up, forward and back substitution per apply.
//
// 2x2 blocks of D_C and D_J on a cell of width h (orthonormal Legendre, lo = (s, -sqrt3 s), hi = (s, sqrt3 s),
// s = 1/sqrt h; [f] = f(high side) - f(low side), {f} the mean; exterior traces zero):
//   diagonal:  D_C = -V - 1/2 lo lo^T + 1/2 hi hi^T,  V_10 = 2 sqrt3 / h;   D_J = -lo lo^T - hi hi^T
//   (c, c-1):  D_C = -1/2 lo hi^T,   D_J = lo hi^T
//   (c, c+1):  D_C =  1/2 hi lo^T,   D_J = hi lo^T                      (entry (k, l) = (test, trial))
__device__ void dsa1d_blocks(double h, double sa, double st, double mu2, double kap, double c11, int variant,
                             bool lower, bool upper, double* Dg, double* L, double* U) {
  const double s = 1.0 / sqrt(h), s3 = 1.7320508075688772;
  const double lo[2] = {s, -s3 * s}, hi[2] = {s, s3 * s};
  double dc[4], dj[4], lc[4], lj[4], uc[4], uj[4];
  for (int k = 0; k < 2; ++k)
    for (int l = 0; l < 2; ++l) {
      dc[k * 2 + l] = -0.5 * lo[k] * lo[l] + 0.5 * hi[k] * hi[l];
      dj[k * 2 + l] = -lo[k] * lo[l] - hi[k] * hi[l];
      lc[k * 2 + l] = -0.5 * lo[k] * hi[l];
      lj[k * 2 + l] = lo[k] * hi[l];
      uc[k * 2 + l] = 0.5 * hi[k] * lo[l];
      uj[k * 2 + l] = hi[k] * lo[l];
    }
  dc[2] -= 2.0 * s3 / h;   // -V: entry (1, 0)
  for (int e = 0; e < 16; ++e) { Dg[e] = 0.0; L[e] = 0.0; U[e] = 0.0; }
  // rows 0-1: dphi equation; rows 2-3: dJ equation; columns likewise
  for (int k = 0; k < 2; ++k)
    for (int l = 0; l < 2; ++l) {
      const int e = k * 2 + l;
      Dg[k * 4 + l] = (k == l ? sa : 0.0) - kap * dj[e];
      Dg[k * 4 + 2 + l] = 3.0 * mu2 * dc[e];
      Dg[(2 + k) * 4 + l] = mu2 * dc[e];
      Dg[(2 + k) * 4 + 2 + l] = (k == l ? 3.0 * mu2 * st : 0.0) - (variant == RTE_DSA_PARTIAL ? 0.0 : 1.5 * c11 * dj[e]);
      if (lower) {
        L[k * 4 + l] = -kap * lj[e];
        L[k * 4 + 2 + l] = 3.0 * mu2 * lc[e];
        L[(2 + k) * 4 + l] = mu2 * lc[e];
        L[(2 + k) * 4 + 2 + l] = variant == RTE_DSA_FULL ? -1.5 * c11 * lj[e] : 0.0;
      }
      if (upper) {
        U[k * 4 + l] = -kap * uj[e];
        U[k * 4 + 2 + l] = 3.0 * mu2 * uc[e];
        U[(2 + k) * 4 + l] = mu2 * uc[e];
        U[(2 + k) * 4 + 2 + l] = variant == RTE_DSA_FULL ? -1.5 * c11 * uj[e] : 0.0;
      }
    }
}

// inverse of a 4x4 matrix by Gauss-Jordan with partial pivoting (A destroyed); false if singular
__device__ bool inv4(double* A, double* X) {
  for (int e = 0; e < 16; ++e) X[e] = (e / 4 == e % 4) ? 1.0 : 0.0;
  for (int c = 0; c < 4; ++c) {
    int piv = c;
    for (int i = c + 1; i < 4; ++i)
      if (fabs(A[i * 4 + c]) > fabs(A[piv * 4 + c])) piv = i;
    if (A[piv * 4 + c] == 0.0) return false;
    if (piv != c)
      for (int j = 0; j < 4; ++j) {
        double t = A[c * 4 + j]; A[c * 4 + j] = A[piv * 4 + j]; A[piv * 4 + j] = t;
        t = X[c * 4 + j]; X[c * 4 + j] = X[piv * 4 + j]; X[piv * 4 + j] = t;
      }
    const double d = 1.0 / A[c * 4 + c];
    for (int j = 0; j < 4; ++j) { A[c * 4 + j] *= d; X[c * 4 + j] *= d; }
    for (int i = 0; i < 4; ++i) {
      if (i == c) continue;
      const double f = A[i * 4 + c];
      for (int j = 0; j < 4; ++j) { A[i * 4 + j] -= f * A[c * 4 + j]; X[i * 4 + j] -= f * X[c * 4 + j]; }
    }
  }
  return true;
}

__device__ void mm4(const double* A, const double* B, double* C) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double v = 0.0;
      for (int k = 0; k < 4; ++k) v += A[i * 4 + k] * B[k * 4 + j];
      C[i * 4 + j] = v;
    }
}

// set-up: one thread per instance; f = [cell][Ginv 16 | M 16 | U 16]
__global__ void k_dsa1d_setup(const InstInfo* inst, int B, const long long* o1d, const double* sig_s,
                              const double* sig_t, int R, int rx, double mu2, double kap, double c11, int variant,
                              double* f, int* bad) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const InstInfo in = inst[b];
  const int nx = in.nx, cx = nx / rx;
  double* fb = f + o1d[b] * 48;
  double Dg[16], L[16], U[16], G[16], T[16];
  for (int c = 0; c < nx; ++c) {
    const int reg = c / cx;
    const double st = sig_t[(size_t)b * R + reg], ss = sig_s[(size_t)b * R + reg];
    dsa1d_blocks(in.hx, st - ss, st, mu2, kap, c11, variant, c > 0, c < nx - 1, Dg, L, U);
    double* fc = fb + (size_t)c * 48;
    if (c > 0) {
      // M_c = L_c G_{c-1}^{-1};  G_c = Dg_c - M_c U_{c-1}
      const double* fp = fb + (size_t)(c - 1) * 48;
      mm4(L, fp, fc + 16);
      mm4(fc + 16, fp + 32, T);
      for (int e = 0; e < 16; ++e) G[e] = Dg[e] - T[e];
    } else {
      for (int e = 0; e < 16; ++e) { G[e] = Dg[e]; fc[16 + e] = 0.0; }
    }
    if (!inv4(G, fc)) { *bad = 1; return; }
    for (int e = 0; e < 16; ++e) fc[32 + e] = U[e];
  }
}

// z = v + dphi, dphi from the exact solve with right-hand side (Sigma_s v, 0); one thread per instance
template <typename TV>
__global__ void k_dsa1d_apply(const InstInfo* inst, int B, const long long* o1d, const double* sig_s, int R, int rx,
                              const double* f, double* y, const TV* v, TV* z, const int* active, const int* only) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  if ((active && !active[b]) || (only && !only[b])) return;
  const InstInfo in = inst[b];
  const int nx = in.nx, cx = nx / rx;
  const double* fb = f + o1d[b] * 48;
  double* yb = y + o1d[b] * 4;
  const TV* vb = v + in.off;
  TV* zb = z + in.off;
  double prev[4] = {0.0, 0.0, 0.0, 0.0};
  for (int c = 0; c < nx; ++c) {   // forward: y_c = b_c - M_c y_{c-1}
    const double ss = sig_s[(size_t)b * R + c / cx];
    double bc[4] = {ss * (double)vb[2 * c], ss * (double)vb[2 * c + 1], 0.0, 0.0};
    const double* M = fb + (size_t)c * 48 + 16;
    for (int i = 0; i < 4; ++i) {
      double t = bc[i];
      for (int k = 0; k < 4; ++k) t -= M[i * 4 + k] * prev[k];
      yb[c * 4 + i] = t;
    }
    for (int i = 0; i < 4; ++i) prev[i] = yb[c * 4 + i];
  }
  double next[4] = {0.0, 0.0, 0.0, 0.0};
  for (int c = nx - 1; c >= 0; --c) {   // back: x_c = G_c^{-1} (y_c - U_c x_{c+1})
    const double* Gi = fb + (size_t)c * 48;
    const double* U = fb + (size_t)c * 48 + 32;
    double r[4], x[4];
    for (int i = 0; i < 4; ++i) {
      double t = yb[c * 4 + i];
      for (int k = 0; k < 4; ++k) t -= U[i * 4 + k] * next[k];
      r[i] = t;
    }
    for (int i = 0; i < 4; ++i) {
      double t = 0.0;
      for (int k = 0; k < 4; ++k) t += Gi[i * 4 + k] * r[k];
      x[i] = t;
    }
    zb[2 * c] = (TV)((double)vb[2 * c] + x[0]);
    zb[2 * c + 1] = (TV)((double)vb[2 * c + 1] + x[1]);
    for (int i = 0; i < 4; ++i) next[i] = x[i];
  }
}

struct DsaWs {
  DevBuf<float> data;
  DevBuf<DsaInst> d_di;
  std::vector<DsaInst> di;
  int lumped = -1;
  int variant = -1;            // variant of the last set-up
  // 1D slab: exact block-tridiagonal factors, per instance and cell [Ginv 16 | M 16 | U 16] doubles, and the
  // forward-sweep vectors [4] per cell
  DevBuf<double> f1d, y1d;
  std::vector<long long> o1d;  // [B+1] cell offsets
  DevBuf<long long> d_o1d;
};

DsaWs* get_dsa_ws(rte_problem* p) {
  if (!p->dsa_ws) p->dsa_ws = std::make_shared<DsaWs>();
  return static_cast<DsaWs*>(p->dsa_ws.get());
}

long long align4(long long x) { return (x + 3) & ~3LL; }

// Layout of the workspace (float offsets, 16-byte aligned blocks); fails on meshes the V-cycle does not
// cover (1D, or a coarsest level above kMaxCoarse vertices, or more than kMaxLevels levels).
int dsa_layout(rte_problem* p, std::vector<DsaInst>& out, long long& total) {
  if (p->dim != 2) {
    set_error("DSA: the V-cycle covers 2D meshes only");
    return RTE_ERR_UNSUPPORTED;
  }
  out.assign(p->B, DsaInst{});
  long long o = 0;
  for (int b = 0; b < p->B; ++b) {
    DsaInst& d = out[b];
    d.nx = p->inst[b].nx;
    d.ny = p->inst[b].ny;
    d.hx = (float)p->inst[b].hx;
    d.hy = (float)p->inst[b].hy;
    const long long nc = (long long)d.nx * d.ny;
    d.o_sgs = o;
    o = align4(o + nc);
    d.o_sga = o;
    o = align4(o + nc);
    d.o_binv = o;
    o += 8 * nc;
    d.o_kinv = o;
    o += 16 * nc;
    d.o_b0 = o;
    o += 4 * nc;
    d.o_x0 = o;
    o += 4 * nc;
    d.o_t = o;
    o += 8 * nc;
    d.o_r0 = o;
    o += 4 * nc;
    int cx = d.nx, cy = d.ny, l = 1;
    while (true) {
      if (l > kMaxLevels) {
        set_error("DSA: too many multigrid levels");
        return RTE_ERR_UNSUPPORTED;
      }
      d.ncx[l] = cx;
      d.ncy[l] = cy;
      const long long nv = (long long)(cx + 1) * (cy + 1);
      d.o_E[l] = o;
      o += 16LL * cx * cy;
      d.o_dinv[l] = o;
      o = align4(o + nv);
      d.o_u[l] = o;
      o = align4(o + nv);
      d.o_b[l] = o;
      o = align4(o + nv);
      d.o_r[l] = o;
      o = align4(o + nv);
      if (cx % 2 == 0 && cy % 2 == 0 && cx * cy > 4) {
        cx /= 2;
        cy /= 2;
        ++l;
      } else {
        break;
      }
    }
    d.L = l;
    const long long nvL = (long long)(cx + 1) * (cy + 1);
    if (nvL > kMaxCoarse) {
      set_error("DSA: the coarsest multigrid level has more than 100 vertices (mesh counts need more "
                "factors of 2)");
      return RTE_ERR_UNSUPPORTED;
    }
    d.o_ainv = o;
    o = align4(o + nvL * nvL);
  }
  total = o;
  return RTE_OK;
}

DsaConst dsa_constants(rte_problem* p, int variant) {
  DsaConst k{};
  double mu2[2] = {0, 0}, kap[2] = {0, 0}, c[2][2] = {{0, 0}, {0, 0}};
  for (size_t j = 0; j < p->w.size(); ++j) {
    const double om[2] = {p->om_x[j], p->om_y[j]};
    for (int d = 0; d < 2; ++d) {
      mu2[d] += p->w[j] * om[d] * om[d];
      if (om[d] > 0) kap[d] += p->w[j] * om[d];
      for (int e = 0; e < 2; ++e) c[d][e] += p->w[j] * om[d] * om[d] * std::fabs(om[e]);
    }
  }
  for (int d = 0; d < 2; ++d) {
    k.mu2[d] = (float)mu2[d];
    k.kappa[d] = (float)kap[d];
    for (int e = 0; e < 2; ++e) k.c[d][e] = (float)c[d][e];
  }
  k.omega = 0.7f;
  k.omega_v = 0.7f;
  k.lumped = variant == RTE_DSA_LUMPED ? 1 : 0;
  return k;
}

}  // namespace

int dsa_check(rte_problem* p) {
  if (p->dim == 1) return RTE_OK;   // exact block-tridiagonal solve, any slab mesh
  std::vector<DsaInst> di;
  long long total = 0;
  return dsa_layout(p, di, total);
}

static int dsa1d_prepare(rte_problem* p, int variant, cudaStream_t st) {
  DsaWs* w = get_dsa_ws(p);
  if (w->o1d.empty()) {
    w->o1d.assign(p->B + 1, 0);
    for (int b = 0; b < p->B; ++b) w->o1d[b + 1] = w->o1d[b] + p->nx[b];
    RTE_TRY(w->f1d.alloc((size_t)w->o1d[p->B] * 48));
    RTE_TRY(w->y1d.alloc((size_t)w->o1d[p->B] * 4));
    RTE_TRY(w->d_o1d.alloc(p->B + 1));
    RTE_CHECK_CUDA(cudaMemcpy(w->d_o1d.p, w->o1d.data(), (p->B + 1) * sizeof(long long), cudaMemcpyHostToDevice));
  }
  // angular moments of the slab quadrature: mu2 = sum w mu^2, kappa = sum_{mu>0} w mu, c = sum w mu^2 |mu|
  double mu2 = 0.0, kap = 0.0, c11 = 0.0;
  for (size_t j = 0; j < p->w.size(); ++j) {
    const double mu = p->om_x[j];
    mu2 += p->w[j] * mu * mu;
    if (mu > 0) kap += p->w[j] * mu;
    c11 += p->w[j] * mu * mu * std::fabs(mu);
  }
  DevBuf<int> bad;
  RTE_TRY(bad.alloc(1));
  RTE_CHECK_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
  k_dsa1d_setup<<<(p->B + 63) / 64, 64, 0, st>>>(p->d_inst.p, p->B, w->d_o1d.p, p->d_sig_s.p, p->d_sig_t.p, p->R,
                                                 p->rx, mu2, kap, c11, variant, w->f1d.p, bad.p);
  count_launch();
  RTE_CHECK_CUDA(cudaGetLastError());
  int hbad = 0;
  RTE_CHECK_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  RTE_CHECK_CUDA(cudaStreamSynchronize(st));
  if (hbad) {
    set_error("DSA (1D): a block of the factorisation is singular (a region with sigma_t = 0?)");
    return RTE_ERR_NUMERIC;
  }
  w->variant = variant;
  w->lumped = variant == RTE_DSA_LUMPED ? 1 : 0;
  return RTE_OK;
}

int dsa_prepare(rte_problem* p, int variant, cudaStream_t st) {
  RTE_ARG(variant == RTE_DSA_PARTIAL || variant == RTE_DSA_LUMPED || variant == RTE_DSA_FULL, "unknown DSA variant");
  if (p->dim == 1) return dsa1d_prepare(p, variant, st);
  if (variant == RTE_DSA_FULL) {
    set_error("DSA: the fully consistent variant is solved exactly in the 1D slab only");
    return RTE_ERR_UNSUPPORTED;
  }
  DsaWs* w = get_dsa_ws(p);
  if (w->di.empty()) {
    long long total = 0;
    RTE_TRY(dsa_layout(p, w->di, total));
    RTE_TRY(w->data.alloc((size_t)total));
    RTE_TRY(w->d_di.alloc(w->di.size()));
    RTE_CHECK_CUDA(cudaMemcpy(w->d_di.p, w->di.data(), w->di.size() * sizeof(DsaInst), cudaMemcpyHostToDevice));
  }
  const DsaConst k = dsa_constants(p, variant);
  int max_nc = 0;
  for (const DsaInst& d : w->di) max_nc = std::max(max_nc, d.nx * d.ny);
  // cross-section profiles: the diffusion operator and its scattering source take the cell means (one "region"
  // per cell)
  k_dsa_setup_cells<<<dim3((max_nc + kSetupThreads - 1) / kSetupThreads, p->B), kSetupThreads, 0, st>>>(
      w->d_di.p, w->data.p, p->cellsig ? p->d_sigc_s.p : p->d_sig_s.p, p->cellsig ? p->d_sigc_t.p : p->d_sig_t.p,
      p->cellsig ? p->ncell : p->R, p->cellsig ? p->nx[0] : p->rx, p->cellsig ? p->ny[0] : p->ry, k);
  count_launch();
  k_dsa_setup_levels<<<p->B, kSetupThreads, 0, st>>>(w->d_di.p, w->data.p);
  count_launch();
  RTE_CHECK_CUDA(cudaGetLastError());
  w->lumped = k.lumped;
  w->variant = variant;
  return RTE_OK;
}

int dsa_launch(rte_problem* p, bool f64, const void* v, void* z, const int* active, const int* only,
               cudaStream_t st) {
  DsaWs* w = get_dsa_ws(p);
  if (p->dim == 1) {
    if (w->variant < 0 || w->o1d.empty()) {
      set_error("DSA: set-up missing");
      return RTE_ERR_INVALID_ARG;
    }
    const unsigned g = (unsigned)((p->B + 63) / 64);
    if (f64)
      k_dsa1d_apply<double><<<g, 64, 0, st>>>(p->d_inst.p, p->B, w->d_o1d.p, p->d_sig_s.p, p->R, p->rx, w->f1d.p,
                                              w->y1d.p, (const double*)v, (double*)z, active, only);
    else
      k_dsa1d_apply<float><<<g, 64, 0, st>>>(p->d_inst.p, p->B, w->d_o1d.p, p->d_sig_s.p, p->R, p->rx, w->f1d.p,
                                             w->y1d.p, (const float*)v, (float*)z, active, only);
    count_launch();
    RTE_CHECK_CUDA(cudaGetLastError());
    return RTE_OK;
  }
  if (w->di.empty() || w->lumped < 0) {
    set_error("DSA: set-up missing");
    return RTE_ERR_INVALID_ARG;
  }
  const DsaConst k = dsa_constants(p, w->lumped ? RTE_DSA_LUMPED : RTE_DSA_PARTIAL);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p->B * kCluster);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (f64)
    RTE_CHECK_CUDA(cudaLaunchKernelEx(&cfg, k_dsa_vcycle<double>, (const InstInfo*)p->d_inst.p,
                                      (const DsaInst*)w->d_di.p, w->data.p, k, (const double*)v, (double*)z, active,
                                      only));
  else
    RTE_CHECK_CUDA(cudaLaunchKernelEx(&cfg, k_dsa_vcycle<float>, (const InstInfo*)p->d_inst.p,
                                      (const DsaInst*)w->d_di.p, w->data.p, k, (const float*)v, (float*)z, active,
                                      only));
  count_launch();
  RTE_CHECK_CUDA(cudaGetLastError());
  return RTE_OK;
}

}  // namespace rte

using namespace rte;

extern "C" int rte_dsa_apply(rte_problem_t p, int variant, int dtype, const void* v, void* z, void* stream) {
  RTE_ARG(p && v && z, "null handle or pointer");
  RTE_ARG(dtype == RTE_F64 || dtype == RTE_F32, "unknown dtype");
  RTE_ARG(v != z, "v and z must not alias");
  cudaStream_t st = (cudaStream_t)stream;
  const bool keep = (variant & RTE_DSA_KEEP_SETUP) != 0;
  variant &= ~RTE_DSA_KEEP_SETUP;
  if (keep) {
    // reuse the set-up of an earlier call (it must exist and be of the same variant)
    DsaWs* w = get_dsa_ws(p);
    RTE_ARG(w->variant >= 0 && w->variant == variant,
            "RTE_DSA_KEEP_SETUP needs an earlier set-up of the same variant");
  } else {
    RTE_TRY(dsa_prepare(p, variant, st));
  }
  return dsa_launch(p, dtype == RTE_F64, v, z, nullptr, nullptr, st);
}
