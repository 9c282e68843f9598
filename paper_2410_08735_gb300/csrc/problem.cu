// Problem setup (paper Sec. 2): quadrature, mesh/region maps, source moments and
// the per-(instance, direction, region) inverses of the cell blocks of D_j + Sigma_t.
//
// With the orthonormal tensor-Legendre basis eta_ab = p_a(x) q_b(y) on a uniform
// Cartesian cell, every cell block of the upwind DG operator (eq. DG, eq. upwind)
// is the Kronecker sum
//     L = alpha K (x) I + beta I (x) K + sigma_t I,  K = [[1, sqrt3], [-sqrt3, 3]],
// alpha = |Omega_x|/h_x, beta = |Omega_y|/h_y, written in the frame reflected so
// that both direction components are positive (odd modes change sign).  In 1D
// (P1, Sec. appendix A slab) L = alpha K + sigma_t I.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace rte {

// n-point Gauss-Legendre nodes (ascending) and weights by Newton's method on P_n.
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p0 = 1.0; p1 = z; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 1; k < n; ++k) {
      double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
      p0 = p1;
      p1 = p2;
    }
    if (n == 1) { p0 = 1.0; p1 = z; }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return x[a] < x[b]; });
  std::vector<double> xs(n), ws(n);
  for (int i = 0; i < n; ++i) { xs[i] = x[idx[i]]; ws[i] = w[idx[i]]; }
  x = xs;
  w = ws;
}

// Integrals of the two orthonormal Legendre modes of a cell [xl, xl+h] over [lo, hi] (inside the cell).
static void mode_integrals(double xl, double h, double lo, double hi, double* I) {
  double xc = xl + 0.5 * h;
  double a = 2.0 * (lo - xc) / h, b = 2.0 * (hi - xc) / h;
  I[0] = (hi - lo) / std::sqrt(h);
  I[1] = std::sqrt(3.0 / h) * (h / 4.0) * (b * b - a * a);
}

// Integrals of the two orthonormal Legendre modes of a cell [xl, xl+h] against exp(-a (x-xc)^2):
// with t = x - xc, int e = sqrt(pi/a)/2 (erf(sqrt(a) t1) - erf(sqrt(a) t0)) (through erfc on a one-signed
// interval, where the erf difference would cancel) and int t e = (exp(-a t0^2) - exp(-a t1^2)) / (2a);
// p_1 = sqrt(3/h) (2/h) (t + xc - x_mid).
static void gauss_mode_integrals(double xl, double h, double a, double xc, double* I) {
  const double t0 = xl - xc, t1 = xl + h - xc, sa = std::sqrt(a);
  double de;
  if (t0 >= 0.0) de = std::erfc(sa * t0) - std::erfc(sa * t1);
  else if (t1 <= 0.0) de = std::erfc(-sa * t1) - std::erfc(-sa * t0);
  else de = std::erf(sa * t1) - std::erf(sa * t0);
  const double ie = 0.5 * std::sqrt(M_PI / a) * de;
  const double ite = (std::exp(-a * t0 * t0) - std::exp(-a * t1 * t1)) / (2.0 * a);
  const double xm = xl + 0.5 * h;
  I[0] = ie / std::sqrt(h);
  I[1] = std::sqrt(3.0 / h) * (2.0 / h) * (ite + (xc - xm) * ie);
}

__global__ void k_linv(int B, int nu, int R, int dim, const InstInfo* inst, const UDir* ud,
                       const double* sig_t, double* out64, float* out32, float* outdf) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long total = (long long)B * nu * R;
  if (tid >= total) return;
  int r = (int)(tid % R);
  int u = (int)((tid / R) % nu);
  int b = (int)(tid / ((long long)R * nu));
  const double s3 = 1.7320508075688772;
  const double K[4] = {1.0, s3, -s3, 3.0};
  double sg = sig_t[(size_t)b * R + r];
  int nd = dim == 2 ? 4 : 2;
  double A[16], X[16];
  if (dim == 2) {
    double al = ud[u].ax / inst[b].hx, be = ud[u].ay / inst[b].hy;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        int a = i & 1, bb = i >> 1, c = j & 1, d = j >> 1;
        double v = 0.0;
        if (bb == d) v += al * K[a * 2 + c];
        if (a == c) v += be * K[bb * 2 + d];
        if (i == j) v += sg;
        A[i * 4 + j] = v;
      }
  } else {
    double al = ud[u].ax / inst[b].hx;
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) A[i * 2 + j] = al * K[i * 2 + j] + (i == j ? sg : 0.0);
  }
  // Gauss-Jordan with partial pivoting
  for (int i = 0; i < nd * nd; ++i) X[i] = (i / nd == i % nd) ? 1.0 : 0.0;
  for (int c = 0; c < nd; ++c) {
    int piv = c;
    double best = fabs(A[c * nd + c]);
    for (int i = c + 1; i < nd; ++i)
      if (fabs(A[i * nd + c]) > best) { best = fabs(A[i * nd + c]); piv = i; }
    if (piv != c)
      for (int j = 0; j < nd; ++j) {
        double t = A[c * nd + j]; A[c * nd + j] = A[piv * nd + j]; A[piv * nd + j] = t;
        t = X[c * nd + j]; X[c * nd + j] = X[piv * nd + j]; X[piv * nd + j] = t;
      }
    double inv = 1.0 / A[c * nd + c];
    for (int j = 0; j < nd; ++j) { A[c * nd + j] *= inv; X[c * nd + j] *= inv; }
    for (int i = 0; i < nd; ++i) {
      if (i == c) continue;
      double f = A[i * nd + c];
      for (int j = 0; j < nd; ++j) { A[i * nd + j] -= f * A[c * nd + j]; X[i * nd + j] -= f * X[c * nd + j]; }
    }
  }
  size_t base = (size_t)tid * nd * nd;
  for (int i = 0; i < nd * nd; ++i) {
    out64[base + i] = X[i];
    out32[base + i] = (float)X[i];
    // double-float pair: the FP32 rounding and the FP32 rounding of what it misses
    const float h = (float)X[i];
    outdf[2 * (base + i)] = h;
    outdf[2 * (base + i) + 1] = (float)(X[i] - (double)h);
  }
}

// Cell inverses with a full Sigma_t block per cell (cross-section profiles): thread (b, u, c) inverts
// alpha K (x) I + beta I (x) K + R_u T_c R_u, the cell block in the frame reflected so that Omega_x, Omega_y > 0
// (R_u flips the sign of the x-odd and y-odd Legendre modes: the reflection maps the block T_c to R_u T_c R_u).
__global__ void k_linv_cell(int B, int nu, int ncell, const InstInfo* inst, const UDir* ud, const double* tblk,
                            double* out64, float* out32) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long total = (long long)B * nu * ncell;
  if (tid >= total) return;
  const int c = (int)(tid % ncell);
  const int u = (int)((tid / ncell) % nu);
  const int b = (int)(tid / ((long long)ncell * nu));
  const double s3 = 1.7320508075688772;
  const double K[4] = {1.0, s3, -s3, 3.0};
  const double al = ud[u].ax / inst[b].hx, be = ud[u].ay / inst[b].hy;
  const double rs[4] = {1.0, (double)ud[u].sx, (double)ud[u].sy, (double)(ud[u].sx * ud[u].sy)};
  const double* T = tblk + ((size_t)b * ncell + c) * 16;
  double A[16], X[16];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      const int a = i & 1, bb = i >> 1, cc = j & 1, d = j >> 1;
      double v = rs[i] * rs[j] * T[i * 4 + j];
      if (bb == d) v += al * K[a * 2 + cc];
      if (a == cc) v += be * K[bb * 2 + d];
      A[i * 4 + j] = v;
      X[i * 4 + j] = i == j ? 1.0 : 0.0;
    }
  for (int col = 0; col < 4; ++col) {   // Gauss-Jordan with partial pivoting
    int piv = col;
    double best = fabs(A[col * 4 + col]);
    for (int i = col + 1; i < 4; ++i)
      if (fabs(A[i * 4 + col]) > best) { best = fabs(A[i * 4 + col]); piv = i; }
    if (piv != col)
      for (int j = 0; j < 4; ++j) {
        double t = A[col * 4 + j]; A[col * 4 + j] = A[piv * 4 + j]; A[piv * 4 + j] = t;
        t = X[col * 4 + j]; X[col * 4 + j] = X[piv * 4 + j]; X[piv * 4 + j] = t;
      }
    const double inv = 1.0 / A[col * 4 + col];
    for (int j = 0; j < 4; ++j) { A[col * 4 + j] *= inv; X[col * 4 + j] *= inv; }
    for (int i = 0; i < 4; ++i) {
      if (i == col) continue;
      const double fct = A[i * 4 + col];
      for (int j = 0; j < 4; ++j) { A[i * 4 + j] -= fct * A[col * 4 + j]; X[i * 4 + j] -= fct * X[col * 4 + j]; }
    }
  }
  const size_t o = (size_t)tid * 16;
  for (int i = 0; i < 16; ++i) {
    out64[o + i] = X[i];
    out32[o + i] = (float)X[i];
  }
}

// The variable-scattering profile of Sec. 5: r^4 (2 - r^2)^2 inside the unit disc, 1 outside.
static double varscat_profile(double x, double y) {
  const double r2 = x * x + y * y;
  return r2 <= 1.0 ? r2 * r2 * (2.0 - r2) * (2.0 - r2) : 1.0;
}

// Blocks F_c[k][l] = int_T f eta_k eta_l of the profile on the mesh of instance 0, by 16 x 16 Gauss-Legendre
// points per cell.  With eta_k = 2 / sqrt(hx hy) p_a(xi) p_b(zeta) (k = a + 2 b, p_0 = sqrt(1/2),
// p_1 = sqrt(3/2) xi) the Jacobian hx hy / 4 cancels the normalisation.
static void profile_blocks(const rte_problem* p, std::vector<double>& F) {
  std::vector<double> q, wq;
  gauss_legendre(16, q, wq);
  const InstInfo& in = p->inst[0];
  F.assign((size_t)p->ncell * 16, 0.0);
  const double s0 = std::sqrt(0.5), s1 = std::sqrt(1.5);
  for (int iy = 0; iy < in.ny; ++iy)
    for (int ix = 0; ix < in.nx; ++ix) {
      double* Fc = &F[((size_t)iy * in.nx + ix) * 16];
      for (int i = 0; i < 16; ++i)
        for (int j = 0; j < 16; ++j) {
          const double x = p->box[0] + (ix + 0.5 + 0.5 * q[i]) * in.hx;
          const double y = p->box[2] + (iy + 0.5 + 0.5 * q[j]) * in.hy;
          const double fw = varscat_profile(x, y) * wq[i] * wq[j];
          const double e[4] = {s0 * s0, s1 * q[i] * s0, s0 * s1 * q[j], s1 * q[i] * s1 * q[j]};
          for (int k = 0; k < 4; ++k)
            for (int l = 0; l < 4; ++l) Fc[k * 4 + l] += fw * e[k] * e[l];
        }
    }
}

// sigma_s of the cell of every dof (instance-major scalar-vector layout)
__global__ void k_sig_dof(const InstInfo* inst, int B, int R, int rx, int ry, int nd, const double* sig_s, double* out,
                          float* out32) {
  const int b = blockIdx.y;
  const InstInfo in = inst[b];
  const int cx = in.nx / rx, cy = in.ny / ry;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < in.ndof; i += gridDim.x * blockDim.x) {
    const int c = i / nd;
    const int ix = c % in.nx, iy = c / in.nx;
    const double v = sig_s[(size_t)b * R + (iy / cy) * rx + ix / cx];
    out[in.off + i] = v;
    out32[in.off + i] = (float)v;
  }
}

int quadrant_gcd(const rte_problem* p) {
  const int nq = p->dim == 2 ? 4 : 2;
  int g = 0;
  for (int q = 0; q < nq; ++q) {
    int a = p->quad_start[q + 1] - p->quad_start[q], b = g;
    while (b) { const int t = a % b; a = b; b = t; }
    g = a;
  }
  return g > 0 ? g : 1;
}

int upload_params(rte_problem* p) {
  std::vector<double> st(p->ss.size());
  std::vector<float> s32(p->ss.size()), sdf(2 * p->ss.size());
  for (size_t i = 0; i < st.size(); ++i) {
    st[i] = p->ss[i] + p->sa[i];
    s32[i] = (float)p->ss[i];
    sdf[2 * i] = s32[i];
    sdf[2 * i + 1] = (float)(p->ss[i] - (double)s32[i]);
  }
  RTE_CHECK_CUDA(cudaMemcpy(p->d_sig_s.p, p->ss.data(), st.size() * 8, cudaMemcpyHostToDevice));
  RTE_CHECK_CUDA(cudaMemcpy(p->d_sig_t.p, st.data(), st.size() * 8, cudaMemcpyHostToDevice));
  RTE_CHECK_CUDA(cudaMemcpy(p->d_sig_s32.p, s32.data(), s32.size() * 4, cudaMemcpyHostToDevice));
  RTE_CHECK_CUDA(cudaMemcpy(p->d_sig_s_df.p, sdf.data(), sdf.size() * 4, cudaMemcpyHostToDevice));
  long long total = (long long)p->B * p->nu * p->R;
  int threads = 128;
  k_linv<<<(unsigned)((total + threads - 1) / threads), threads>>>(p->B, p->nu, p->R, p->dim, p->d_inst.p,
                                                                  p->d_udir.p, p->d_sig_t.p, p->d_linv64.p,
                                                                  p->d_linv32.p, p->d_linv_df.p);
  count_launch();
  RTE_CHECK_CUDA(cudaGetLastError());
  {
    int maxn = 0;
    for (int b = 0; b < p->B; ++b) maxn = std::max(maxn, (int)(p->off[b + 1] - p->off[b]));
    dim3 g((maxn + 255) / 256, p->B);
    k_sig_dof<<<g, 256>>>(p->d_inst.p, p->B, p->R, p->rx, p->ry, p->nd, p->d_sig_s.p, p->d_sig_dof.p,
                            p->d_sig_dof32.p);
    count_launch();
    RTE_CHECK_CUDA(cudaGetLastError());
  }
  if (p->cellsig) {
    // Sigma_s = c_s0 F + c_s1 I, Sigma_t = c_t0 F + c_t1 I per cell (c_t = c_s + c_a), their cell means (the (0, 0)
    // entries: eta_0 is constant), then the cell inverses of every unique direction
    const size_t nb = (size_t)p->B * p->ncell;
    std::vector<double> S(nb * 16), T(nb * 16), ms(nb), mt(nb);
    std::vector<float> S32(nb * 16);
    for (int b = 0; b < p->B; ++b) {
      const double cs0 = p->ss[2 * b], cs1 = p->ss[2 * b + 1];
      const double ct0 = cs0 + p->sa[2 * b], ct1 = cs1 + p->sa[2 * b + 1];
      for (int c = 0; c < p->ncell; ++c) {
        const size_t o = ((size_t)b * p->ncell + c) * 16;
        for (int k = 0; k < 16; ++k) {
          const double f = p->F[(size_t)c * 16 + k], id = (k % 5 == 0) ? 1.0 : 0.0;
          S[o + k] = cs0 * f + cs1 * id;
          T[o + k] = ct0 * f + ct1 * id;
          S32[o + k] = (float)S[o + k];
        }
        ms[(size_t)b * p->ncell + c] = S[o];
        mt[(size_t)b * p->ncell + c] = T[o];
      }
    }
    RTE_CHECK_CUDA(cudaMemcpy(p->d_sblk64.p, S.data(), S.size() * 8, cudaMemcpyHostToDevice));
    RTE_CHECK_CUDA(cudaMemcpy(p->d_tblk64.p, T.data(), T.size() * 8, cudaMemcpyHostToDevice));
    RTE_CHECK_CUDA(cudaMemcpy(p->d_sblk32.p, S32.data(), S32.size() * 4, cudaMemcpyHostToDevice));
    RTE_CHECK_CUDA(cudaMemcpy(p->d_sigc_s.p, ms.data(), ms.size() * 8, cudaMemcpyHostToDevice));
    RTE_CHECK_CUDA(cudaMemcpy(p->d_sigc_t.p, mt.data(), mt.size() * 8, cudaMemcpyHostToDevice));
    const long long tot = (long long)p->B * p->nu * p->ncell;
    k_linv_cell<<<(unsigned)((tot + 127) / 128), 128>>>(p->B, p->nu, p->ncell, p->d_inst.p, p->d_udir.p,
                                                        p->d_tblk64.p, p->d_linvc64.p, p->d_linvc32.p);
    count_launch();
    RTE_CHECK_CUDA(cudaGetLastError());
  }
  RTE_CHECK_CUDA(cudaDeviceSynchronize());
  return RTE_OK;
}

static int create_impl(const rte_problem_desc* d, rte_problem* p) {
  RTE_ARG(d->dim == 1 || d->dim == 2, "dim must be 1 or 2");
  RTE_ARG(d->n_instances >= 1, "n_instances must be >= 1");
  RTE_ARG(d->nx != nullptr && (d->dim == 1 || d->ny != nullptr), "nx/ny arrays required");
  RTE_ARG(d->sigma_s != nullptr && d->sigma_a != nullptr, "sigma_s/sigma_a arrays required");
  RTE_ARG(d->n_polar >= 1 && d->n_polar <= 64, "n_polar must be in [1, 64]");
  RTE_ARG(d->rx >= 1 && (d->dim == 1 || d->ry >= 1), "region grid must be positive");
  RTE_ARG(d->box[1] > d->box[0] && (d->dim == 1 || d->box[3] > d->box[2]), "empty domain box");
  // N_theta = 2 mod 4 puts two Chebyshev azimuths at pi/2 and 3pi/2, where the computed cos is a rounding error
  // (+6e-17, -1.8e-16): those directions are swept in the quadrant of the computed signs, with an x-coupling of
  // that size, as any direction; the quadrants then hold unequal numbers of directions
  if (d->dim == 2) RTE_ARG(d->n_azim >= 4 && d->n_azim % 2 == 0 && d->n_azim <= 256,
                           "n_azim must be even and in [4, 256]");
  if (d->dim == 1) RTE_ARG(d->n_polar % 2 == 0, "1D n_polar must be even");
  p->dim = d->dim;
  p->B = d->n_instances;
  p->n_polar = d->n_polar;
  p->n_azim = d->dim == 2 ? d->n_azim : 0;
  p->nd = d->dim == 2 ? 4 : 2;
  p->rx = d->rx;
  p->ry = d->dim == 2 ? d->ry : 1;
  p->R = p->rx * p->ry;
  std::memcpy(p->box, d->box, sizeof(p->box));
  p->g = d->inflow_g;
  p->src_q = d->src_q;
  std::memcpy(p->src_box, d->src_box, sizeof(p->src_box));
  RTE_ARG(d->src_kind == RTE_SRC_BOX || d->src_kind == RTE_SRC_GAUSS, "unknown src_kind");
  if (d->src_kind == RTE_SRC_GAUSS) {
    RTE_ARG(d->dim == 2, "the Gaussian source is 2D");
    RTE_ARG(d->src_gauss[1] > 0.0 && std::isfinite(d->src_gauss[0]), "Gaussian source needs a > 0 and a finite A");
  }
  p->src_kind = d->src_kind;
  std::memcpy(p->src_gauss, d->src_gauss, sizeof(p->src_gauss));
  RTE_ARG(d->inflow_faces >= 0 && d->inflow_faces <= 15, "inflow_faces is a mask of 4 bits");
  RTE_ARG(d->dim == 2 || d->inflow_faces == 15 || (d->inflow_faces & 12) == 0,
          "a 1D slab has the faces x- and x+ only");
  p->inflow_mask = d->inflow_faces == 0 ? 15 : d->inflow_faces;
  RTE_ARG(d->sigma_modes == RTE_SIGMA_REGIONS || d->sigma_modes == RTE_SIGMA_VARSCAT, "unknown sigma_modes");
  p->cellsig = d->sigma_modes == RTE_SIGMA_VARSCAT;
  if (p->cellsig) {
    RTE_ARG(d->dim == 2 && d->rx * d->ry == 2, "RTE_SIGMA_VARSCAT is 2D with two coefficients (rx * ry = 2)");
    for (int b = 1; b < d->n_instances; ++b)
      RTE_ARG(d->nx[b] == d->nx[0] && d->ny[b] == d->ny[0], "RTE_SIGMA_VARSCAT needs every instance on one mesh");
  }
  p->nx.resize(p->B);
  p->ny.resize(p->B);
  p->off.assign(p->B + 1, 0);
  p->inst.resize(p->B);
  for (int b = 0; b < p->B; ++b) {
    p->nx[b] = d->nx[b];
    p->ny[b] = d->dim == 2 ? d->ny[b] : 1;
    RTE_ARG(p->nx[b] >= 1 && p->ny[b] >= 1 && p->nx[b] <= 8192 && p->ny[b] <= 8192, "mesh size out of range");
    RTE_ARG(p->nx[b] % p->rx == 0 && p->ny[b] % p->ry == 0, "region grid must divide every mesh");
    long long nb = (long long)p->nx[b] * p->ny[b] * p->nd;
    p->off[b + 1] = p->off[b] + nb;
    InstInfo& in = p->inst[b];
    in.nx = p->nx[b];
    in.ny = p->ny[b];
    in.off = p->off[b];
    in.ndof = (int)nb;
    in.hx = (d->box[1] - d->box[0]) / p->nx[b];
    in.hy = d->dim == 2 ? (d->box[3] - d->box[2]) / p->ny[b] : 1.0;
    in.g = d->inflow_g;
  }
  p->ntot = p->off[p->B];
  size_t nR = (size_t)p->B * p->R;
  p->ss.assign(d->sigma_s, d->sigma_s + nR);
  p->sa.assign(d->sigma_a, d->sigma_a + nR);
  for (size_t i = 0; i < nR; ++i)
    RTE_ARG(p->ss[i] >= 0.0 && p->sa[i] >= 0.0 && std::isfinite(p->ss[i]) && std::isfinite(p->sa[i]),
            "cross sections must be finite and non-negative");
  // quadrature (Sec. 2.1) and unique in-plane directions
  std::vector<double> zx, zw;
  gauss_legendre(d->n_polar, zx, zw);
  if (p->dim == 1) {
    p->ndir = d->n_polar;
    for (int j = 0; j < p->ndir; ++j) {
      p->om_x.push_back(zx[j]);
      p->om_y.push_back(0.0);
      p->om_z.push_back(0.0);
      p->w.push_back(zw[j] / 2.0);
    }
    // unique = all; quadrant 0: mu > 0 (ascending index), quadrant 1: mu < 0
    p->uniq_of_dir.assign(p->ndir, -1);
    p->quad_start.assign(3, 0);
    for (int q = 0; q < 2; ++q) {
      p->quad_start[q] = (int)p->udir.size();
      for (int j = 0; j < p->ndir; ++j) {
        bool pos = p->om_x[j] > 0;
        if ((q == 0) != pos) continue;
        UDir u{};
        u.ax = std::fabs(p->om_x[j]);
        u.ay = 0.0;
        u.w = p->w[j];
        u.sx = pos ? 1 : -1;
        u.sy = 1;
        u.quadrant = q;
        u.ndup = 1;
        u.dup[0] = j;
        p->uniq_of_dir[j] = (int)p->udir.size();
        p->udir.push_back(u);
      }
    }
    p->quad_start[2] = (int)p->udir.size();
  } else {
    int nt = d->n_azim, nz = d->n_polar;
    p->ndir = nt * nz;
    for (int j2 = 0; j2 < nz; ++j2)
      for (int j1 = 0; j1 < nt; ++j1) {
        double th = (2.0 * (j1 + 1) - 1.0) * M_PI / nt;
        double s = std::sqrt(1.0 - zx[j2] * zx[j2]);
        p->om_x.push_back(std::cos(th) * s);
        p->om_y.push_back(std::sin(th) * s);
        p->om_z.push_back(zx[j2]);
        p->w.push_back(zw[j2] / 2.0 / nt);
      }
    // +-Omega_z pairs (j2, nz-1-j2) share (Omega_x, Omega_y): merge them
    p->uniq_of_dir.assign(p->ndir, -1);
    std::vector<UDir> all;
    std::vector<std::vector<int>> members;
    for (int j2 = 0; j2 < (nz + 1) / 2; ++j2)
      for (int j1 = 0; j1 < nt; ++j1) {
        int ja = j2 * nt + j1, jb = (nz - 1 - j2) * nt + j1;
        UDir u{};
        u.ax = std::fabs(p->om_x[ja]);
        u.ay = std::fabs(p->om_y[ja]);
        u.sx = p->om_x[ja] > 0 ? 1 : -1;
        u.sy = p->om_y[ja] > 0 ? 1 : -1;
        u.quadrant = (u.sx < 0 ? 1 : 0) + (u.sy < 0 ? 2 : 0);
        u.ndup = (ja == jb) ? 1 : 2;
        u.dup[0] = ja;
        u.dup[1] = jb;
        u.w = p->w[ja] + (ja == jb ? 0.0 : p->w[jb]);
        all.push_back(u);
      }
    p->quad_start.assign(5, 0);
    for (int q = 0; q < 4; ++q) {
      p->quad_start[q] = (int)p->udir.size();
      for (auto& u : all)
        if (u.quadrant == q) {
          for (int k = 0; k < u.ndup; ++k) p->uniq_of_dir[u.dup[k]] = (int)p->udir.size();
          p->udir.push_back(u);
        }
    }
    p->quad_start[4] = (int)p->udir.size();
  }
  p->nu = (int)p->udir.size();
  // source moments G_k = int_T G eta_k (closed form, exact for the box source)
  std::vector<double> G(p->ntot, 0.0);
  if (p->src_kind == RTE_SRC_GAUSS) {
    for (int b = 0; b < p->B; ++b) {
      const InstInfo& in = p->inst[b];
      std::vector<double> Ix(2 * in.nx), Iy(2 * in.ny);
      for (int ix = 0; ix < in.nx; ++ix)
        gauss_mode_integrals(p->box[0] + ix * in.hx, in.hx, p->src_gauss[1], p->src_gauss[2], &Ix[2 * ix]);
      for (int iy = 0; iy < in.ny; ++iy)
        gauss_mode_integrals(p->box[2] + iy * in.hy, in.hy, p->src_gauss[1], p->src_gauss[3], &Iy[2 * iy]);
      for (int iy = 0; iy < in.ny; ++iy)
        for (int ix = 0; ix < in.nx; ++ix) {
          const long long c = (long long)iy * in.nx + ix;
          for (int k = 0; k < 4; ++k)
            G[in.off + 4 * c + k] = p->src_gauss[0] * Ix[2 * ix + (k & 1)] * Iy[2 * iy + (k >> 1)];
        }
    }
  }
  for (int b = 0; b < p->B && p->src_kind == RTE_SRC_BOX; ++b) {
    const InstInfo& in = p->inst[b];
    for (int iy = 0; iy < in.ny; ++iy)
      for (int ix = 0; ix < in.nx; ++ix) {
        double xl = p->box[0] + ix * in.hx;
        double lo = std::max(xl, p->src_box[0]), hi = std::min(xl + in.hx, p->src_box[1]);
        if (hi <= lo) continue;
        double Ix[2];
        mode_integrals(xl, in.hx, lo, hi, Ix);
        long long c = (long long)iy * in.nx + ix;
        if (p->dim == 1) {
          G[in.off + 2 * c] = p->src_q * Ix[0];
          G[in.off + 2 * c + 1] = p->src_q * Ix[1];
          continue;
        }
        double yl = p->box[2] + iy * in.hy;
        double ylo = std::max(yl, p->src_box[2]), yhi = std::min(yl + in.hy, p->src_box[3]);
        if (yhi <= ylo) continue;
        double Iy[2];
        mode_integrals(yl, in.hy, ylo, yhi, Iy);
        for (int k = 0; k < 4; ++k) G[in.off + 4 * c + k] = p->src_q * Ix[k & 1] * Iy[k >> 1];
      }
  }
  // device buffers
  RTE_TRY(p->d_inst.alloc(p->B));
  RTE_TRY(p->d_udir.alloc(p->nu));
  RTE_TRY(p->d_sig_s.alloc(nR));
  RTE_TRY(p->d_sig_t.alloc(nR));
  RTE_TRY(p->d_sig_s32.alloc(nR));
  RTE_TRY(p->d_sig_s_df.alloc(2 * nR));
  RTE_TRY(p->d_G.alloc(p->ntot));
  RTE_TRY(p->d_sig_dof.alloc(p->ntot));
  RTE_TRY(p->d_sig_dof32.alloc(p->ntot));
  size_t nl = (size_t)p->B * p->nu * p->R * p->nd * p->nd;
  RTE_TRY(p->d_linv64.alloc(nl));
  RTE_TRY(p->d_linv32.alloc(nl));
  RTE_TRY(p->d_linv_df.alloc(2 * nl));
  RTE_TRY(p->d_active.alloc(p->B));
  RTE_TRY(p->d_wq.alloc(p->ndir));
  if (p->cellsig) {
    p->ncell = p->nx[0] * p->ny[0];
    profile_blocks(p, p->F);
    const size_t nb = (size_t)p->B * p->ncell;
    RTE_TRY(p->d_F64.alloc((size_t)p->ncell * 16));
    RTE_TRY(p->d_sblk64.alloc(nb * 16));
    RTE_TRY(p->d_tblk64.alloc(nb * 16));
    RTE_TRY(p->d_sblk32.alloc(nb * 16));
    RTE_TRY(p->d_sigc_s.alloc(nb));
    RTE_TRY(p->d_sigc_t.alloc(nb));
    RTE_TRY(p->d_linvc64.alloc(nb * p->nu * 16));
    RTE_TRY(p->d_linvc32.alloc(nb * p->nu * 16));
    RTE_CHECK_CUDA(cudaMemcpy(p->d_F64.p, p->F.data(), p->F.size() * 8, cudaMemcpyHostToDevice));
  }
  RTE_CHECK_CUDA(cudaMemcpy(p->d_inst.p, p->inst.data(), p->B * sizeof(InstInfo), cudaMemcpyHostToDevice));
  RTE_CHECK_CUDA(cudaMemcpy(p->d_udir.p, p->udir.data(), p->nu * sizeof(UDir), cudaMemcpyHostToDevice));
  RTE_CHECK_CUDA(cudaMemcpy(p->d_G.p, G.data(), p->ntot * 8, cudaMemcpyHostToDevice));
  RTE_CHECK_CUDA(cudaMemcpy(p->d_wq.p, p->w.data(), p->ndir * 8, cudaMemcpyHostToDevice));
  std::vector<int> ones(p->B, 1);
  RTE_CHECK_CUDA(cudaMemcpy(p->d_active.p, ones.data(), p->B * sizeof(int), cudaMemcpyHostToDevice));
  return upload_params(p);
}

}  // namespace rte

extern "C" {

int rte_problem_create(const rte_problem_desc* desc, rte_problem_t* out) {
  RTE_ARG(desc != nullptr && out != nullptr, "null descriptor or output handle");
  *out = nullptr;
  rte_problem* p = new rte_problem();
  int s = rte::create_impl(desc, p);
  if (s != RTE_OK) {
    delete p;
    return s;
  }
  *out = p;
  return RTE_OK;
}

int rte_problem_destroy(rte_problem_t p) {
  if (p) {
    cudaDeviceSynchronize();
    delete p;
  }
  return RTE_OK;
}

int rte_problem_get_info(rte_problem_t p, rte_problem_info* info) {
  RTE_ARG(p != nullptr && info != nullptr, "null handle or info");
  info->dim = p->dim;
  info->n_instances = p->B;
  info->n_directions = p->ndir;
  info->n_unique_directions = p->nu;
  info->dofs_per_cell = p->nd;
  info->n_regions = p->R;
  info->n_dof_total = p->ntot;
  info->n_angular_total = (long long)p->ndir * p->ntot;
  return RTE_OK;
}

int rte_problem_offsets(rte_problem_t p, long long* offsets) {
  RTE_ARG(p != nullptr && offsets != nullptr, "null handle or offsets");
  for (int b = 0; b <= p->B; ++b) offsets[b] = p->off[b];
  return RTE_OK;
}

int rte_problem_set_params(rte_problem_t p, const double* sigma_s, const double* sigma_a) {
  RTE_ARG(p != nullptr && sigma_s != nullptr && sigma_a != nullptr, "null handle or parameter array");
  size_t nR = (size_t)p->B * p->R;
  for (size_t i = 0; i < nR; ++i)
    RTE_ARG(sigma_s[i] >= 0.0 && sigma_a[i] >= 0.0 && std::isfinite(sigma_s[i]) && std::isfinite(sigma_a[i]),
            "cross sections must be finite and non-negative");
  p->ss.assign(sigma_s, sigma_s + nR);
  p->sa.assign(sigma_a, sigma_a + nR);
  return rte::upload_params(p);
}

int rte_problem_set_inflow(rte_problem_t p, const double* g) {
  RTE_ARG(p != nullptr && g != nullptr, "null handle or inflow array");
  for (int b = 0; b < p->B; ++b) RTE_ARG(std::isfinite(g[b]), "inflow values must be finite");
  for (int b = 0; b < p->B; ++b) p->inst[b].g = g[b];
  RTE_CHECK_CUDA(cudaMemcpy(p->d_inst.p, p->inst.data(), p->B * sizeof(rte::InstInfo), cudaMemcpyHostToDevice));
  return RTE_OK;
}

}  // extern "C"
