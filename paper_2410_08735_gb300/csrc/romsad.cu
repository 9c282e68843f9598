// ROMSAD preconditioner (paper Sec. 4.1 and 4.3):
//   M_ROM^{-1} v = v + W (U_r^T A_mu U_r)^{-1} P^T Sigma_s v        (eq. rom-sa-preconditioner)
//   P = sum_j U_{r,j},  W = sum_j omega_j U_{r,j}                    (eq. rom-correction)
//   U^T A_mu U = A_D + sum_R (sigma_a,R + sigma_s,R) T_R - sum_R sigma_s,R S_R   (affine split, Sec. 4.1)
// with A_D = sum_j U_j^T D_j U_j, T_R = sum_j U_j^T chi_R U_j, S_R = P^T chi_R W.
//
// U is stored in direction blocks a (all N_Omega directions with multiplicity 1, or the unique
// in-plane directions with their multiplicity), so P = sum_a mult_a U_a and W = sum_a wA_a U_a.
// The affine operators are built column by column (the greedy adds columns one at a time).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "romsad.h"

namespace rte {

// P[:, k] = sum_a mult_a U_a[k], W[:, k] = sum_a wA_a U_a[k]
__global__ void k_pw_column(const double* U, int nA, int N, int k, int rmax, const double* mult, const double* wA,
                            double* P, double* W, float* P32, float* W32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double* Uk = U + (size_t)k * nA * N;
  double p = 0.0, w = 0.0;
  for (int a = 0; a < nA; ++a) {
    double v = Uk[(size_t)a * N + i];
    p += mult[a] * v;
    w += wA[a] * v;
  }
  P[(size_t)i * rmax + k] = p;
  W[(size_t)i * rmax + k] = w;
  P32[(size_t)i * rmax + k] = (float)p;
  W32[(size_t)i * rmax + k] = (float)w;
}

// For the new column k and every l <= k, partial sums over (block a, cells of region R):
//   out[.., 0] = sum mult_a U_a[k] . Y_a[l]     (A_D[k][l])
//   out[.., 1] = sum mult_a U_a[l] . Y_a[k]     (A_D[l][k])
//   out[.., 2] = sum mult_a U_a[k] . U_a[l] on R (T_R[k][l])
// grid: (l = 0..k, R, a-chunks); one partial triple per block, reduced on the host in fixed order.
__global__ void k_newcol_dots(const double* U, const double* Y, int nA, int N, int k, int nx, int ny, int nd, int rx,
                              int ry, const double* mult, int achunk, double* out) {
  const int l = blockIdx.x, R = blockIdx.y, ac = blockIdx.z;
  const int cx = nx / rx, cy = ny / ry;
  const int rxi = R % rx, ryi = R / rx;
  const int cells = cx * cy;
  const int a0 = ac * achunk, a1 = min(nA, a0 + achunk);
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  const double* Uk = U + (size_t)k * nA * N;
  const double* Ul = U + (size_t)l * nA * N;
  const double* Yk = Y + (size_t)k * nA * N;
  const double* Yl = Y + (size_t)l * nA * N;
  for (int a = a0; a < a1; ++a) {
    const double m = mult[a];
    double t0 = 0.0, t1 = 0.0, t2 = 0.0;
    for (int e = threadIdx.x; e < cells * nd; e += blockDim.x) {
      int cl = e / nd, kk = e % nd;
      int ix = rxi * cx + cl % cx, iy = ryi * cy + cl / cx;
      size_t i = (size_t)a * N + ((size_t)iy * nx + ix) * nd + kk;
      t0 += Uk[i] * Yl[i];
      t1 += Ul[i] * Yk[i];
      t2 += Uk[i] * Ul[i];
    }
    s0 += m * t0;
    s1 += m * t1;
    s2 += m * t2;
  }
  __shared__ double red[3][256];
  red[0][threadIdx.x] = s0;
  red[1][threadIdx.x] = s1;
  red[2][threadIdx.x] = s2;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    size_t o = (((size_t)l * gridDim.y + R) * gridDim.z + ac) * 3;
    out[o] = red[0][0];
    out[o + 1] = red[1][0];
    out[o + 2] = red[2][0];
  }
}

// S_R[k][l] = sum_{i in R} P[i][k] W[i][l] and S_R[l][k]; grid (l, R)
__global__ void k_newcol_S(const double* P, const double* W, int rmax, int k, int nx, int ny, int nd, int rx, int ry,
                           double* out) {
  const int l = blockIdx.x, R = blockIdx.y;
  const int cx = nx / rx, cy = ny / ry;
  const int rxi = R % rx, ryi = R / rx;
  double s0 = 0.0, s1 = 0.0;
  for (int e = threadIdx.x; e < cx * cy * nd; e += blockDim.x) {
    int cl = e / nd, kk = e % nd;
    int ix = rxi * cx + cl % cx, iy = ryi * cy + cl / cx;
    size_t i = ((size_t)iy * nx + ix) * nd + kk;
    s0 += P[i * rmax + k] * W[i * rmax + l];
    s1 += P[i * rmax + l] * W[i * rmax + k];
  }
  __shared__ double red[2][256];
  red[0][threadIdx.x] = s0;
  red[1][threadIdx.x] = s1;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[((size_t)l * gridDim.y + R) * 2] = red[0][0];
    out[((size_t)l * gridDim.y + R) * 2 + 1] = red[1][0];
  }
}

// Cross-section profiles: the same dots with the affine terms (profile blocks F, identity) in place of regions.
// grid (l = 0..k, term t = 0 (F) / 1 (I), a-chunks); term 0 gets t2 = sum_a mult_a sum_c U_a[k]_c^T F_c U_a[l]_c
// and no A_D part, term 1 all three sums over every dof.
__global__ void k_newcol_dots_cell(const double* U, const double* Y, int nA, int N, int k, const double* F,
                                   const double* mult, int achunk, double* out) {
  const int l = blockIdx.x, t = blockIdx.y, ac = blockIdx.z;
  const int a0 = ac * achunk, a1 = min(nA, a0 + achunk);
  const int ncell = N / 4;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  const double* Uk = U + (size_t)k * nA * N;
  const double* Ul = U + (size_t)l * nA * N;
  const double* Yk = Y + (size_t)k * nA * N;
  const double* Yl = Y + (size_t)l * nA * N;
  for (int a = a0; a < a1; ++a) {
    const double m = mult[a];
    double t0 = 0.0, t1 = 0.0, t2 = 0.0;
    if (t == 1) {
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const size_t g = (size_t)a * N + i;
        t0 += Uk[g] * Yl[g];
        t1 += Ul[g] * Yk[g];
        t2 += Uk[g] * Ul[g];
      }
    } else {
      for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
        const double* uk = Uk + (size_t)a * N + 4 * c;
        const double* ul = Ul + (size_t)a * N + 4 * c;
        const double* Fc = F + (size_t)c * 16;
        for (int r = 0; r < 4; ++r) t2 += uk[r] * (Fc[4 * r] * ul[0] + Fc[4 * r + 1] * ul[1] + Fc[4 * r + 2] * ul[2] +
                                                   Fc[4 * r + 3] * ul[3]);
      }
    }
    s0 += m * t0;
    s1 += m * t1;
    s2 += m * t2;
  }
  __shared__ double red[3][256];
  red[0][threadIdx.x] = s0;
  red[1][threadIdx.x] = s1;
  red[2][threadIdx.x] = s2;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const size_t o = (((size_t)l * gridDim.y + t) * gridDim.z + ac) * 3;
    out[o] = red[0][0];
    out[o + 1] = red[1][0];
    out[o + 2] = red[2][0];
  }
}

// S_t[k][l] = P[:, k]^T F_t W[:, l] and S_t[l][k] with F_0 = the profile blocks, F_1 = I; grid (l, t)
__global__ void k_newcol_S_cell(const double* P, const double* W, int rmax, int k, int N, const double* F,
                                double* out) {
  const int l = blockIdx.x, t = blockIdx.y;
  double s0 = 0.0, s1 = 0.0;
  for (int c = threadIdx.x; c < N / 4; c += blockDim.x) {
    double pk[4], pl[4], wk[4], wl[4];
    for (int r = 0; r < 4; ++r) {
      const size_t i = (size_t)(4 * c + r) * rmax;
      pk[r] = P[i + k];
      pl[r] = P[i + l];
      wk[r] = W[i + k];
      wl[r] = W[i + l];
    }
    for (int r = 0; r < 4; ++r) {
      double fwl = wl[r], fwk = wk[r];
      if (t == 0) {
        const double* Fr = F + (size_t)c * 16 + 4 * r;
        fwl = Fr[0] * wl[0] + Fr[1] * wl[1] + Fr[2] * wl[2] + Fr[3] * wl[3];
        fwk = Fr[0] * wk[0] + Fr[1] * wk[1] + Fr[2] * wk[2] + Fr[3] * wk[3];
      }
      s0 += pk[r] * fwl;
      s1 += pl[r] * fwk;
    }
  }
  __shared__ double red[2][256];
  red[0][threadIdx.x] = s0;
  red[1][threadIdx.x] = s1;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[((size_t)l * gridDim.y + t) * 2] = red[0][0];
    out[((size_t)l * gridDim.y + t) * 2 + 1] = red[1][0];
  }
}

static int grow_host(romsad* rom, int newr) {
  // host affine matrices are re-laid out for rank newr
  auto regrow = [&](std::vector<double>& M, int nmat) {
    std::vector<double> Nn((size_t)nmat * newr * newr, 0.0);
    for (int m = 0; m < nmat; ++m)
      for (int i = 0; i < rom->r; ++i)
        for (int j = 0; j < rom->r; ++j)
          Nn[((size_t)m * newr + i) * newr + j] = M[((size_t)m * rom->r + i) * rom->r + j];
    M.swap(Nn);
  };
  if (rom->A_D.empty()) rom->A_D.assign((size_t)rom->r * rom->r, 0.0);
  if (rom->T_R.empty()) rom->T_R.assign((size_t)rom->R * rom->r * rom->r, 0.0);
  if (rom->S_R.empty()) rom->S_R.assign((size_t)rom->R * rom->r * rom->r, 0.0);
  regrow(rom->A_D, 1);
  regrow(rom->T_R, rom->R);
  regrow(rom->S_R, rom->R);
  return RTE_OK;
}

// Add column k = rom->r (already written into U[k], and Y[k] = D U[k] computed by the caller):
// P, W columns and the affine operators' new row/column.
int rom_add_column(romsad* rom, DevBuf<double>& d_mult, DevBuf<double>& d_wA, cudaStream_t st) {
  const int k = rom->r, N = rom->N, nA = rom->nA, R = rom->R;
  k_pw_column<<<(N + 255) / 256, 256, 0, st>>>(rom->U.p, nA, N, k, rom->rmax, d_mult.p, d_wA.p, rom->P.p, rom->W.p,
                                               rom->P32.p, rom->W32.p);
  count_launch();
  RTE_CHECK_CUDA(cudaGetLastError());
  const int achunk = std::max(1, (nA + 7) / 8);
  const int nac = (nA + achunk - 1) / achunk;
  DevBuf<double> d_out;
  RTE_TRY(d_out.alloc((size_t)(k + 1) * R * nac * 3 + (size_t)(k + 1) * R * 2));
  dim3 g1(k + 1, R, nac);
  double* d_s = d_out.p + (size_t)(k + 1) * R * nac * 3;
  dim3 g2(k + 1, R);
  if (rom->sigma_modes) {
    if (!rom->F.p || R != 2) {
      set_error("ROM: cross-section profile blocks missing");
      return RTE_ERR_INVALID_ARG;
    }
    k_newcol_dots_cell<<<g1, 256, 0, st>>>(rom->U.p, rom->Y.p, nA, N, k, rom->F.p, d_mult.p, achunk, d_out.p);
    count_launch();
    k_newcol_S_cell<<<g2, 256, 0, st>>>(rom->P.p, rom->W.p, rom->rmax, k, N, rom->F.p, d_s);
    count_launch();
  } else {
    k_newcol_dots<<<g1, 256, 0, st>>>(rom->U.p, rom->Y.p, nA, N, k, rom->nx, rom->ny, rom->nd, rom->rx, rom->ry,
                                      d_mult.p, achunk, d_out.p);
    count_launch();
    k_newcol_S<<<g2, 256, 0, st>>>(rom->P.p, rom->W.p, rom->rmax, k, rom->nx, rom->ny, rom->nd, rom->rx, rom->ry, d_s);
    count_launch();
  }
  RTE_CHECK_CUDA(cudaGetLastError());
  RTE_CHECK_CUDA(cudaGetLastError());
  std::vector<double> h(d_out.n);
  RTE_CHECK_CUDA(cudaMemcpyAsync(h.data(), d_out.p, h.size() * 8, cudaMemcpyDeviceToHost, st));
  RTE_CHECK_CUDA(cudaStreamSynchronize(st));
  const int nr = k + 1;
  RTE_TRY(grow_host(rom, nr));
  rom->r = nr;
  for (int l = 0; l <= k; ++l) {
    double ad_kl = 0, ad_lk = 0;
    for (int Rr = 0; Rr < R; ++Rr) {
      double t = 0;
      for (int ac = 0; ac < nac; ++ac) {
        const double* q = &h[(((size_t)l * R + Rr) * nac + ac) * 3];
        ad_kl += q[0];
        ad_lk += q[1];
        t += q[2];
      }
      rom->T_R[((size_t)Rr * nr + k) * nr + l] = t;
      rom->T_R[((size_t)Rr * nr + l) * nr + k] = t;
      const double* sq = &h[(size_t)(k + 1) * R * nac * 3 + ((size_t)l * R + Rr) * 2];
      rom->S_R[((size_t)Rr * nr + k) * nr + l] = sq[0];
      rom->S_R[((size_t)Rr * nr + l) * nr + k] = sq[1];
    }
    rom->A_D[(size_t)k * nr + l] = ad_kl;
    rom->A_D[(size_t)l * nr + k] = ad_lk;
  }
  return rom_upload_affine(rom);
}

int rom_upload_affine(romsad* rom) {
  const int r = rom->r, R = rom->R;
  size_t rr = (size_t)r * r;
  RTE_TRY(rom->d_aff.ensure((size_t)(1 + 2 * R) * rr));
  std::vector<double> h((1 + 2 * R) * rr);
  std::memcpy(h.data(), rom->A_D.data(), rr * 8);
  std::memcpy(h.data() + rr, rom->T_R.data(), R * rr * 8);
  std::memcpy(h.data() + (1 + R) * rr, rom->S_R.data(), R * rr * 8);
  RTE_CHECK_CUDA(cudaMemcpy(rom->d_aff.p, h.data(), h.size() * 8, cudaMemcpyHostToDevice));
  return RTE_OK;
}

int rom_check_mesh(const romsad* rom, const rte_problem* p, int b) {
  RTE_ARG(rom->dim == p->dim && rom->nx == p->nx[b] && rom->ny == p->ny[b] && rom->ndir == p->ndir &&
              rom->nu == p->nu && rom->R == p->R && rom->rx == p->rx && rom->ry == p->ry,
          "ROM mesh/quadrature/regions do not match the instance");
  RTE_ARG(rom->sigma_modes == (p->cellsig ? 1 : 0), "ROM and instance differ in their cross-section form");
  for (int q = 0; q < 4; ++q) RTE_ARG(std::fabs(rom->box[q] - p->box[q]) < 1e-12, "ROM domain does not match");
  return RTE_OK;
}

// ---------------------------------------------------------------- online apply
// y[b][k] = sum_i P[i][k] sigma_s(i) v_b[i]; one block per listed instance, warp lanes over k.
template <typename TP>
__global__ void k_project(const TP* P, int rmax, int r, const InstInfo* inst, const int* list, const double* sig_s,
                          int R, int rx, int ry, int nd, const double* sblk, const double* v, double* y) {
  const int b = list[blockIdx.x];
  const InstInfo in = inst[b];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int cx = in.nx / rx, cy = in.ny / ry;
  double acc0 = 0.0, acc1 = 0.0;
  const double* vb = v + in.off;
  for (int i = warp; i < in.ndof; i += nw) {
    const int c = i / nd;
    const int ix = c % in.nx, iy = c / in.nx;
    double sv;
    if (sblk) {   // cross-section profiles: row (i mod 4) of the cell's Sigma_s block times the cell's values
      const double* S = sblk + ((size_t)(in.off / 4) + c) * 16 + (i & 3) * 4;
      const double* x = vb + 4 * c;
      sv = S[0] * x[0] + S[1] * x[1] + S[2] * x[2] + S[3] * x[3];
    } else {
      sv = sig_s[(size_t)b * R + (iy / cy) * rx + ix / cx] * vb[i];
    }
    if (lane < r) acc0 += (double)P[(size_t)i * rmax + lane] * sv;
    if (lane + 32 < r) acc1 += (double)P[(size_t)i * rmax + lane + 32] * sv;
  }
  __shared__ double red[32][64];
  red[warp][lane] = acc0;
  red[warp][lane + 32] = acc1;
  __syncthreads();
  if (warp == 0) {
    for (int q = 0; q < 2; ++q) {
      int k = lane + 32 * q;
      if (k < r) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += red[w][k];
        y[(size_t)blockIdx.x * 64 + k] = s;
      }
    }
  }
}

// Assemble U^T A_mu U for one listed instance, LU with partial pivoting, solve for c. One block per instance.
__global__ void k_small_solve(const double* aff, int r, int R, const double* sig_s, const double* sig_t,
                              const int* list, const double* y, double* c) {
  extern __shared__ double sm[];
  double* A = sm;           // r*r
  double* x = sm + r * r;   // r
  __shared__ int piv_s;
  const int b = list[blockIdx.x];
  const size_t rr = (size_t)r * r;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    double v = aff[e];
    for (int q = 0; q < R; ++q) {
      double ss = sig_s[(size_t)b * R + q], st = sig_t[(size_t)b * R + q];
      v += st * aff[(1 + q) * rr + e] - ss * aff[(1 + R + q) * rr + e];
    }
    A[e] = v;
  }
  for (int e = threadIdx.x; e < r; e += blockDim.x) x[e] = y[(size_t)blockIdx.x * 64 + e];
  __syncthreads();
  for (int col = 0; col < r; ++col) {
    if (threadIdx.x == 0) {
      int p = col;
      double best = fabs(A[col * r + col]);
      for (int i = col + 1; i < r; ++i)
        if (fabs(A[i * r + col]) > best) { best = fabs(A[i * r + col]); p = i; }
      piv_s = p;
    }
    __syncthreads();
    const int p = piv_s;
    if (p != col) {
      for (int j = threadIdx.x; j < r; j += blockDim.x) {
        double t = A[col * r + j]; A[col * r + j] = A[p * r + j]; A[p * r + j] = t;
      }
      if (threadIdx.x == 0) { double t = x[col]; x[col] = x[p]; x[p] = t; }
    }
    __syncthreads();
    const double d = A[col * r + col];
    for (int i = col + 1 + threadIdx.x; i < r; i += blockDim.x) {
      double f = A[i * r + col] / d;
      for (int j = col; j < r; ++j) A[i * r + j] -= f * A[col * r + j];
      x[i] -= f * x[col];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int i = r - 1; i >= 0; --i) {
      double s = x[i];
      for (int j = i + 1; j < r; ++j) s -= A[i * r + j] * x[j];
      x[i] = s / A[i * r + i];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < r; e += blockDim.x) c[(size_t)blockIdx.x * 64 + e] = x[e];
}

// z_b[i] = v_b[i] + sum_k W[i][k] c_b[k]; grid (chunks, listed instances)
template <typename TP>
__global__ void k_lift(const TP* W, int rmax, int r, const InstInfo* inst, const int* list, const double* v,
                       const double* c, double* z) {
  const int b = list[blockIdx.y];
  const InstInfo in = inst[b];
  __shared__ double cs[64];
  for (int k = threadIdx.x; k < r; k += blockDim.x) cs[k] = c[(size_t)blockIdx.y * 64 + k];
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < in.ndof; i += gridDim.x * blockDim.x) {
    const TP* w = W + (size_t)i * rmax;
    double s = 0.0;
    for (int k = 0; k < r; ++k) s += (double)w[k] * cs[k];
    z[in.off + i] = v[in.off + i] + s;
  }
}

// ------------------------------------------------- factor once, apply many times (online path)
// Inverse of U^T A_mu U (Gauss-Jordan with partial pivoting, FP64) for every listed instance, one block
// per instance; formed once per solve so that each ROMSAD apply needs one r x r matrix-vector product.
__global__ void k_rom_factor(const double* aff, int r, int R, const double* sig_s, const double* sig_t, const int* list,
                             double* inv, int* piv) {
  extern __shared__ double sm[];
  double* A = sm;            // r x r
  double* X = sm + r * r;    // r x r, becomes the inverse
  __shared__ int piv_s;
  const int b = list[blockIdx.x];
  const size_t rr = (size_t)r * r;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    double v = aff[e];
    for (int q = 0; q < R; ++q)
      v += sig_t[(size_t)b * R + q] * aff[(1 + q) * rr + e] - sig_s[(size_t)b * R + q] * aff[(1 + R + q) * rr + e];
    A[e] = v;
    X[e] = (e / r == e % r) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int col = 0; col < r; ++col) {
    if (threadIdx.x == 0) {
      int p = col;
      double best = fabs(A[col * r + col]);
      for (int i = col + 1; i < r; ++i)
        if (fabs(A[i * r + col]) > best) { best = fabs(A[i * r + col]); p = i; }
      piv_s = p;
      piv[(size_t)blockIdx.x * 64 + col] = p;
    }
    __syncthreads();
    const int p = piv_s;
    if (p != col)
      for (int j = threadIdx.x; j < r; j += blockDim.x) {
        double t = A[col * r + j]; A[col * r + j] = A[p * r + j]; A[p * r + j] = t;
        t = X[col * r + j]; X[col * r + j] = X[p * r + j]; X[p * r + j] = t;
      }
    __syncthreads();
    const double d = 1.0 / A[col * r + col];
    __syncthreads();
    for (int j = threadIdx.x; j < r; j += blockDim.x) { A[col * r + j] *= d; X[col * r + j] *= d; }
    __syncthreads();
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
      const int i = e / r, j = e % r;
      if (i == col) continue;
      const double f = A[i * r + col];
      if (j != col) A[i * r + j] -= f * A[col * r + j];
      X[i * r + j] -= f * X[col * r + j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < r; i += blockDim.x)
      if (i != col) A[i * r + col] = 0.0;
    __syncthreads();
  }
  double* out = inv + (size_t)blockIdx.x * 64 * 64;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) out[e] = X[e];
}

// Partial projections: part[(inst, chunk)][k] = sum over the chunk's dofs of P[i][k] sigma_s(i) v[i]
// (sigma_s per dof precomputed); grid (nchunk, ninst); 8 warps stride over the chunk, lanes over k.
template <typename TP>
__global__ void k_project_part(const TP* P, int rmax, int r, const InstInfo* inst, const int* list, const int* active,
                               const double* sig_dof, const double* sblk, const double* v, int chunk,
                               double* part) {
  const int b = list[blockIdx.y];
  if (active && !active[b]) return;
  const InstInfo in = inst[b];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int i0 = blockIdx.x * chunk, i1 = min(in.ndof, i0 + chunk);
  double acc0 = 0.0, acc1 = 0.0;
  const double* vb = v + in.off;
  const double* sb = sig_dof + in.off;
  for (int i = i0 + warp; i < i1; i += nw) {
    double sv;
    if (sblk) {   // cross-section profiles: row (i mod 4) of the cell's Sigma_s block times the cell's values
      const double* S = sblk + ((size_t)(in.off + i) >> 2) * 16 + (i & 3) * 4;
      const double* x = vb + (i & ~3);
      sv = S[0] * x[0] + S[1] * x[1] + S[2] * x[2] + S[3] * x[3];
    } else {
      sv = sb[i] * vb[i];
    }
    if (lane < r) acc0 += (double)P[(size_t)i * rmax + lane] * sv;
    if (lane + 32 < r) acc1 += (double)P[(size_t)i * rmax + lane + 32] * sv;
  }
  __shared__ double red[8][64];
  red[warp][lane] = acc0;
  red[warp][lane + 32] = acc1;
  __syncthreads();
  if (threadIdx.x < 64) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w][threadIdx.x];
    part[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 64 + threadIdx.x] = s;
  }
}

// c = (U^T A U)^{-1} y with y = sum of the partials (fixed chunk order); one block of 64 threads per instance.
__global__ void k_rom_inv_apply(const double* part, int nchunk, int r, const double* inv, const int* list,
                                const int* active, double* c) {
  const int b = list[blockIdx.x];
  if (active && !active[b]) return;
  __shared__ double y[64];
  const int t = threadIdx.x;
  if (t < r) {
    double s = 0.0;
    for (int ch = 0; ch < nchunk; ++ch) s += part[((size_t)blockIdx.x * nchunk + ch) * 64 + t];
    y[t] = s;
  }
  __syncthreads();
  if (t < r) {
    const double* row = inv + (size_t)blockIdx.x * 64 * 64 + (size_t)t * r;
    double s = 0.0;
    for (int k = 0; k < r; ++k) s += row[k] * y[k];
    c[(size_t)blockIdx.x * 64 + t] = s;
  }
}

// z_b = v_b + W c_b; grid (chunks, listed instances), skipping inactive instances
template <typename TP>
__global__ void k_lift_masked(const TP* W, int rmax, int r, const InstInfo* inst, const int* list, const int* active,
                              const double* v, const double* c, double* z) {
  const int b = list[blockIdx.y];
  if (active && !active[b]) return;
  const InstInfo in = inst[b];
  __shared__ double cs[64];
  for (int k = threadIdx.x; k < r; k += blockDim.x) cs[k] = c[(size_t)blockIdx.y * 64 + k];
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < in.ndof; i += gridDim.x * blockDim.x) {
    const TP* w = W + (size_t)i * rmax;
    double s = 0.0;
    for (int k = 0; k < r; ++k) s += (double)w[k] * cs[k];
    z[in.off + i] = v[in.off + i] + s;
  }
}

int RomPlan::build(romsad* rom_, rte_problem* p, const std::vector<int>& ids_, cudaStream_t st) {
  rom = rom_;
  ids = ids_;
  const int n = (int)ids.size();
  // ensure(): buffers are reused (same device pointers) when the plan is rebuilt for the same groups
  RTE_TRY(d_ids.ensure(n));
  RTE_CHECK_CUDA(cudaMemcpyAsync(d_ids.p, ids.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
  RTE_TRY(lu.ensure((size_t)n * 64 * 64));
  RTE_TRY(piv.ensure((size_t)n * 64));
  chunk = 256;
  nchunk = (rom->N + chunk - 1) / chunk;
  RTE_TRY(part.ensure((size_t)n * nchunk * 64));
  RTE_TRY(c.ensure((size_t)n * 64));
  size_t smem = (size_t)2 * rom->r * rom->r * 8;   // 64 KiB at the largest rank (64)
  // the attribute is per device: set on the current one at every plan build (once per solve, not on the hot path)
  if (smem > 48 * 1024)
    RTE_CHECK_CUDA(cudaFuncSetAttribute(k_rom_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_rom_factor<<<n, 256, smem, st>>>(rom->d_aff.p, rom->r, rom->R, p->d_sig_s.p, p->d_sig_t.p, d_ids.p, lu.p, piv.p);
  count_launch();
  RTE_CHECK_CUDA(cudaGetLastError());
  return RTE_OK;
}

int RomPlan::apply(rte_problem* p, const int* d_active, const double* v, double* z, bool f64, cudaStream_t st) {
  const int n = (int)ids.size();
  dim3 gp(nchunk, n);
  if (f64)
    k_project_part<double><<<gp, 256, 0, st>>>(rom->P.p, rom->rmax, rom->r, p->d_inst.p, d_ids.p, d_active,
                                               p->d_sig_dof.p, p->cellsig ? p->d_sblk64.p : nullptr, v, chunk,
                                               part.p);
  else
    k_project_part<float><<<gp, 256, 0, st>>>(rom->P32.p, rom->rmax, rom->r, p->d_inst.p, d_ids.p, d_active,
                                              p->d_sig_dof.p, p->cellsig ? p->d_sblk64.p : nullptr, v, chunk,
                                              part.p);
  count_launch();
  k_rom_inv_apply<<<n, 64, 0, st>>>(part.p, nchunk, rom->r, lu.p, d_ids.p, d_active, c.p);
  count_launch();
  dim3 gl((rom->N + 255) / 256, n);
  if (f64)
    k_lift_masked<double><<<gl, 256, 0, st>>>(rom->W.p, rom->rmax, rom->r, p->d_inst.p, d_ids.p, d_active, v, c.p, z);
  else
    k_lift_masked<float><<<gl, 256, 0, st>>>(rom->W32.p, rom->rmax, rom->r, p->d_inst.p, d_ids.p, d_active, v, c.p, z);
  count_launch();
  RTE_CHECK_CUDA(cudaGetLastError());
  return RTE_OK;
}

int rom_small_solve(romsad* rom, rte_problem* p, const int* d_list, int ninst, const double* y, double* c,
                    cudaStream_t st) {
  const int r = rom->r;
  size_t smem = ((size_t)r * r + r) * 8;
  k_small_solve<<<ninst, 128, smem, st>>>(rom->d_aff.p, r, rom->R, p->d_sig_s.p, p->d_sig_t.p, d_list, y, c);
  count_launch();
  RTE_CHECK_CUDA(cudaGetLastError());
  return RTE_OK;
}

int rom_lift_list(romsad* rom, rte_problem* p, const int* d_list, int ninst, const double* v, const double* c,
                  double* z, cudaStream_t st) {
  if (ninst == 0) return RTE_OK;
  dim3 grid((rom->N + 255) / 256, ninst);
  k_lift<double><<<grid, 256, 0, st>>>(rom->W.p, rom->rmax, rom->r, p->d_inst.p, d_list, v, c, z);
  count_launch();
  RTE_CHECK_CUDA(cudaGetLastError());
  return RTE_OK;
}

int rom_project_list(romsad* rom, rte_problem* p, const int* d_list, int ninst, const double* v, double* y,
                     cudaStream_t st) {
  if (ninst == 0) return RTE_OK;
  k_project<double><<<ninst, 256, 0, st>>>(rom->P.p, rom->rmax, rom->r, p->d_inst.p, d_list, p->d_sig_s.p, p->R, p->rx,
                                           p->ry, p->nd, p->cellsig ? p->d_sblk64.p : nullptr, v, y);
  count_launch();
  RTE_CHECK_CUDA(cudaGetLastError());
  return RTE_OK;
}


int rom_alloc_arrays(romsad* rom, int rmax, bool withU) {
  rom->rmax = rmax;
  RTE_TRY(rom->P.alloc((size_t)rom->N * rmax));
  RTE_TRY(rom->W.alloc((size_t)rom->N * rmax));
  RTE_TRY(rom->P32.alloc((size_t)rom->N * rmax));
  RTE_TRY(rom->W32.alloc((size_t)rom->N * rmax));
  RTE_CHECK_CUDA(cudaMemset(rom->P.p, 0, rom->P.n * 8));
  RTE_CHECK_CUDA(cudaMemset(rom->W.p, 0, rom->W.n * 8));
  RTE_CHECK_CUDA(cudaMemset(rom->P32.p, 0, rom->P32.n * 4));
  RTE_CHECK_CUDA(cudaMemset(rom->W32.p, 0, rom->W32.n * 4));
  if (withU) {
    RTE_TRY(rom->U.alloc((size_t)rmax * rom->nA * rom->N));
    RTE_TRY(rom->Y.alloc((size_t)rmax * rom->nA * rom->N));
  }
  return RTE_OK;
}

void rom_init_geometry(romsad* rom, const rte_problem* p, int b) {
  rom->dim = p->dim;
  rom->nx = p->nx[b];
  rom->ny = p->ny[b];
  rom->nd = p->nd;
  rom->ndir = p->ndir;
  rom->nu = p->nu;
  rom->R = p->R;
  rom->rx = p->rx;
  rom->ry = p->ry;
  std::memcpy(rom->box, p->box, sizeof(rom->box));
  rom->N = (int)(p->off[b + 1] - p->off[b]);
  rom->sigma_modes = p->cellsig ? 1 : 0;
  if (p->cellsig && rom->F.alloc((size_t)p->ncell * 16) == RTE_OK)
    cudaMemcpy(rom->F.p, p->d_F64.p, (size_t)p->ncell * 16 * 8, cudaMemcpyDeviceToDevice);
  rom->r = 0;
  rom->A_D.clear();
  rom->T_R.clear();
  rom->S_R.clear();
}

// Y[k] = D_u U_a[k] for every block a (sigma_t = 0): one forward launch per block.
int rom_compute_Y_column(romsad* rom, const rte_problem* p, int inst, int k, cudaStream_t st) {
  const InstInfo& in = p->inst[inst];
  for (int a = 0; a < rom->nA; ++a) {
    const UDir& u = p->udir[rom->uidx[a]];
    const double* x = rom->U.p + ((size_t)k * rom->nA + a) * rom->N;
    double* y = rom->Y.p + ((size_t)k * rom->nA + a) * rom->N;
    RTE_TRY(launch_forward_cols(p->dim, in.nx, in.ny, in.hx, in.hy, u, p->rx, p->ry, nullptr, x, 0, y, 0, 1, st));
  }
  return RTE_OK;
}

}  // namespace rte

using namespace rte;

extern "C" {

int romsad_create_from_basis(rte_problem_t tmpl, int instance, int r, const double* U_host, romsad_t* out) {
  RTE_ARG(tmpl && U_host && out, "null handle or pointer");
  RTE_ARG(instance >= 0 && instance < tmpl->B, "instance out of range");
  RTE_ARG(r >= 1 && r <= 64, "rank must be in [1, 64]");
  *out = nullptr;
  romsad* rom = new romsad();
  rom_init_geometry(rom, tmpl, instance);
  rom->nA = tmpl->ndir;
  rom->uidx = tmpl->uniq_of_dir;
  rom->dir_block.resize(tmpl->ndir);
  for (int j = 0; j < tmpl->ndir; ++j) rom->dir_block[j] = j;
  rom->mult.assign(tmpl->ndir, 1.0);
  rom->wA = tmpl->w;
  int s = rom_alloc_arrays(rom, r, true);
  DevBuf<double> d_mult, d_wA;
  if (s == RTE_OK) s = d_mult.alloc(rom->nA);
  if (s == RTE_OK) s = d_wA.alloc(rom->nA);
  if (s == RTE_OK) {
    cudaMemcpy(d_mult.p, rom->mult.data(), rom->nA * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(d_wA.p, rom->wA.data(), rom->nA * 8, cudaMemcpyHostToDevice);
    cudaError_t e = cudaMemcpy(rom->U.p, U_host, (size_t)r * rom->nA * rom->N * 8, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      set_error(std::string("romsad_create_from_basis: ") + cudaGetErrorString(e));
      s = RTE_ERR_CUDA;
    }
  }
  for (int k = 0; k < r && s == RTE_OK; ++k) {
    s = rom_compute_Y_column(rom, tmpl, instance, k, 0);
    if (s == RTE_OK) s = rom_add_column(rom, d_mult, d_wA, 0);
  }
  if (s != RTE_OK) {
    delete rom;
    return s;
  }
  *out = rom;
  return RTE_OK;
}

int romsad_rank(romsad_t rom, int* r) {
  RTE_ARG(rom && r, "null handle or pointer");
  *r = rom->r;
  return RTE_OK;
}

int romsad_get_basis(romsad_t rom, double* U_host) {
  RTE_ARG(rom && U_host, "null handle or pointer");
  RTE_ARG(rom->U.p != nullptr, "this ROM holds no basis (loaded from a checkpoint)");
  // expand stored blocks to all N_Omega directions
  std::vector<double> blk((size_t)rom->nA * rom->N);
  for (int k = 0; k < rom->r; ++k) {
    RTE_CHECK_CUDA(cudaMemcpy(blk.data(), rom->U.p + (size_t)k * rom->nA * rom->N, blk.size() * 8,
                              cudaMemcpyDeviceToHost));
    double* dst = U_host + (size_t)k * rom->ndir * rom->N;
    for (int j = 0; j < rom->ndir; ++j)
      std::memcpy(dst + (size_t)j * rom->N, blk.data() + (size_t)rom->dir_block[j] * rom->N, (size_t)rom->N * 8);
  }
  return RTE_OK;
}

int romsad_reduced_operator(romsad_t rom, const double* sigma_s, const double* sigma_a, double* A_host) {
  RTE_ARG(rom && sigma_s && sigma_a && A_host, "null handle or pointer");
  const int r = rom->r;
  for (int e = 0; e < r * r; ++e) {
    double v = rom->A_D[e];
    for (int q = 0; q < rom->R; ++q)
      v += (sigma_s[q] + sigma_a[q]) * rom->T_R[(size_t)q * r * r + e] - sigma_s[q] * rom->S_R[(size_t)q * r * r + e];
    A_host[e] = v;
  }
  return RTE_OK;
}

int romsad_galerkin_coefficients(romsad_t rom, rte_problem_t p, double* c_host) {
  RTE_ARG(rom && p && c_host, "null handle or pointer");
  RTE_ARG(rom->r >= 1, "empty ROM");
  for (int b = 0; b < p->B; ++b) RTE_TRY(rom_check_mesh(rom, p, b));
  // b~ (FP64 sweep), y = P^T Sigma_s b~, c = (U^T A_mu U)^{-1} y, every instance
  DevBuf<double> bt, ys, cs;
  DevBuf<int> d_all;
  RTE_TRY(bt.alloc((size_t)p->ntot));
  RTE_TRY(ys.alloc((size_t)p->B * 64));
  RTE_TRY(cs.alloc((size_t)p->B * 64));
  RTE_TRY(d_all.alloc(p->B));
  std::vector<int> all(p->B);
  for (int b = 0; b < p->B; ++b) all[b] = b;
  RTE_CHECK_CUDA(cudaMemcpy(d_all.p, all.data(), p->B * sizeof(int), cudaMemcpyHostToDevice));
  RTE_TRY(launch_T(p, MODE_RHS, true, nullptr, true, nullptr, bt.p, true, nullptr, 0));
  RTE_TRY(rom_project_list(rom, p, d_all.p, p->B, bt.p, ys.p, 0));
  RTE_TRY(rom_small_solve(rom, p, d_all.p, p->B, ys.p, cs.p, 0));
  std::vector<double> h((size_t)p->B * 64);
  RTE_CHECK_CUDA(cudaMemcpy(h.data(), cs.p, h.size() * 8, cudaMemcpyDeviceToHost));
  for (int b = 0; b < p->B; ++b)
    for (int k = 0; k < rom->r; ++k) c_host[(size_t)b * rom->r + k] = h[(size_t)b * 64 + k];
  return RTE_OK;
}

int romsad_apply(romsad_t rom, rte_problem_t p, int dtype, const void* v, void* z, void* stream) {
  RTE_ARG(rom && p && v && z, "null handle or pointer");
  RTE_ARG(dtype == RTE_F64 || dtype == RTE_F32, "dtype must be RTE_F64 or RTE_F32");
  for (int b = 0; b < p->B; ++b) RTE_TRY(rom_check_mesh(rom, p, b));
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int> ids(p->B);
  for (int b = 0; b < p->B; ++b) ids[b] = b;
  RomPlan plan;
  RTE_TRY(plan.build(rom, p, ids, st));
  if (dtype == RTE_F32) {
    if (p->cellsig) {
      set_error("romsad_apply: FP32 vectors run the tensor-core products, not available with cross-section profiles");
      return RTE_ERR_UNSUPPORTED;
    }
    RTE_TRY(rom_tc_plan_setup(plan, st));
    RTE_TRY(rom_tc_apply(plan, p, nullptr, (const float*)v, (float*)z, st));
  } else {
    RTE_TRY(plan.apply(p, nullptr, (const double*)v, (double*)z, true, st));
  }
  RTE_CHECK_CUDA(cudaStreamSynchronize(st));
  return RTE_OK;
}

int romsad_save(romsad_t rom, const char* path) {
  RTE_ARG(rom && path, "null handle or path");
  FILE* f = std::fopen(path, "wb");
  if (!f) {
    set_error(std::string("romsad_save: cannot open ") + path);
    return RTE_ERR_IO;
  }
  const char magic[8] = {'R', 'T', 'E', 'R', 'O', 'M', '1', 0};
  int hdr[12] = {rom->dim, rom->nx, rom->ny, rom->nd, rom->ndir, rom->nu, rom->R, rom->rx, rom->ry, rom->N, rom->r,
                 rom->sigma_modes};
  std::vector<double> P((size_t)rom->N * rom->r), W((size_t)rom->N * rom->r);
  for (int k = 0; k < rom->r; ++k) {
    std::vector<double> col(rom->N);
    RTE_CHECK_CUDA(cudaMemcpy2D(col.data(), 8, rom->P.p + k, rom->rmax * 8, 8, rom->N, cudaMemcpyDeviceToHost));
    for (int i = 0; i < rom->N; ++i) P[(size_t)i * rom->r + k] = col[i];
    RTE_CHECK_CUDA(cudaMemcpy2D(col.data(), 8, rom->W.p + k, rom->rmax * 8, 8, rom->N, cudaMemcpyDeviceToHost));
    for (int i = 0; i < rom->N; ++i) W[(size_t)i * rom->r + k] = col[i];
  }
  bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(int), 12, f) == 12 &&
            std::fwrite(rom->box, 8, 4, f) == 4 && std::fwrite(P.data(), 8, P.size(), f) == P.size() &&
            std::fwrite(W.data(), 8, W.size(), f) == W.size() &&
            std::fwrite(rom->A_D.data(), 8, rom->A_D.size(), f) == rom->A_D.size() &&
            std::fwrite(rom->T_R.data(), 8, rom->T_R.size(), f) == rom->T_R.size() &&
            std::fwrite(rom->S_R.data(), 8, rom->S_R.size(), f) == rom->S_R.size();
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) {
    set_error(std::string("romsad_save: write failed for ") + path);
    return RTE_ERR_IO;
  }
  return RTE_OK;
}

int romsad_load(const char* path, romsad_t* out) {
  RTE_ARG(path && out, "null path or handle");
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) {
    set_error(std::string("romsad_load: cannot open ") + path);
    return RTE_ERR_IO;
  }
  char magic[8];
  int hdr[12];
  romsad* rom = new romsad();
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "RTEROM1", 8) == 0 &&
            std::fread(hdr, sizeof(int), 12, f) == 12 && std::fread(rom->box, 8, 4, f) == 4;
  if (ok) {
    rom->dim = hdr[0]; rom->nx = hdr[1]; rom->ny = hdr[2]; rom->nd = hdr[3]; rom->ndir = hdr[4]; rom->nu = hdr[5];
    rom->R = hdr[6]; rom->rx = hdr[7]; rom->ry = hdr[8]; rom->N = hdr[9]; rom->r = hdr[10];
    rom->sigma_modes = hdr[11];
    ok = rom->r >= 1 && rom->r <= 64 && rom->N > 0 && rom->R >= 1 && rom->R <= 4096 &&
         (rom->sigma_modes == 0 || (rom->sigma_modes == 1 && rom->R == 2));
  }
  std::vector<double> P, W;
  if (ok) {
    size_t nr = (size_t)rom->N * rom->r, rr = (size_t)rom->r * rom->r;
    P.resize(nr);
    W.resize(nr);
    rom->A_D.resize(rr);
    rom->T_R.resize(rr * rom->R);
    rom->S_R.resize(rr * rom->R);
    ok = std::fread(P.data(), 8, nr, f) == nr && std::fread(W.data(), 8, nr, f) == nr &&
         std::fread(rom->A_D.data(), 8, rr, f) == rr && std::fread(rom->T_R.data(), 8, rr * rom->R, f) == rr * rom->R &&
         std::fread(rom->S_R.data(), 8, rr * rom->R, f) == rr * rom->R;
  }
  std::fclose(f);
  if (!ok) {
    delete rom;
    set_error(std::string("romsad_load: malformed checkpoint ") + path);
    return RTE_ERR_IO;
  }
  int s = rom_alloc_arrays(rom, rom->r, false);
  if (s == RTE_OK) {
    std::vector<float> P32(P.size()), W32(W.size());
    for (size_t i = 0; i < P.size(); ++i) { P32[i] = (float)P[i]; W32[i] = (float)W[i]; }
    cudaMemcpy(rom->P.p, P.data(), P.size() * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(rom->W.p, W.data(), W.size() * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(rom->P32.p, P32.data(), P32.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(rom->W32.p, W32.data(), W32.size() * 4, cudaMemcpyHostToDevice);
    s = rom_upload_affine(rom);
  }
  if (s != RTE_OK) {
    delete rom;
    return s;
  }
  *out = rom;
  return RTE_OK;
}

int romsad_destroy(romsad_t rom) {
  if (rom) {
    cudaDeviceSynchronize();
    delete rom;
  }
  return RTE_OK;
}

}  // extern "C"
