/*
 * CPU oracle (test infrastructure only): the transport sweep of one discrete
 * ordinate and the forward upwind-DG operator, written plainly in FP64.
 *
 * Paper Sec. 3.1 (SI step, eq. SI-equation): for a fixed direction Omega_j the
 * upwind DG operator (D_j + Sigma_t) is block lower triangular once the cells
 * are ordered along the upwind direction, so one block Gauss-Seidel pass in
 * that order inverts it.  This file performs exactly that pass: cells are
 * visited row by row in the upwind y order and, inside a row, in the upwind x
 * order; each cell assembles its right-hand side from the already-known
 * upwind neighbours and solves its dense nd x nd block by Gaussian
 * elimination with partial pivoting.
 *
 * The per-direction local matrices come from the caller (assembled by Gauss
 * quadrature of the weak form, eq. DG):
 *   M[k*nd+l]          volume + outflow-face terms of one cell, without sigma_t
 *   C[f][k*nd+l]       coupling of the cell's test function k to the upwind
 *                      neighbour's basis function l across face f, i.e. the
 *                      integral of (Omega.n_f) eta_k eta_l^nbr over the face
 *   inflow[f]          1 if face f is an inflow face (Omega.n_f < 0)
 * Faces: 0 = x-low, 1 = x-high, 2 = y-low, 3 = y-high.  Cells are row-major
 * (c = iy*nx + ix), dofs c*nd + k.  Uniform Cartesian meshes only.
 */
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* Solve A x = b in place (A: n x n row-major, overwritten; b -> x). Returns 0, or 1 if singular. */
static int dense_solve(int n, double* A, double* b) {
  for (int col = 0; col < n; ++col) {
    int piv = col;
    double best = fabs(A[col * n + col]);
    for (int r = col + 1; r < n; ++r) {
      if (fabs(A[r * n + col]) > best) { best = fabs(A[r * n + col]); piv = r; }
    }
    if (best == 0.0) return 1;
    if (piv != col) {
      for (int k = 0; k < n; ++k) { double t = A[col * n + k]; A[col * n + k] = A[piv * n + k]; A[piv * n + k] = t; }
      double t = b[col]; b[col] = b[piv]; b[piv] = t;
    }
    for (int r = col + 1; r < n; ++r) {
      double f = A[r * n + col] / A[col * n + col];
      for (int k = col; k < n; ++k) A[r * n + k] -= f * A[col * n + k];
      b[r] -= f * b[col];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * b[k];
    b[r] = s / A[r * n + r];
  }
  return 0;
}

/* Index of the neighbour across face f, or -1 on the domain boundary. */
static int neighbour(int nx, int ny, int ix, int iy, int f) {
  switch (f) {
    case 0: return ix > 0 ? iy * nx + ix - 1 : -1;
    case 1: return ix < nx - 1 ? iy * nx + ix + 1 : -1;
    case 2: return iy > 0 ? (iy - 1) * nx + ix : -1;
    default: return iy < ny - 1 ? (iy + 1) * nx + ix : -1;
  }
}

/*
 * psi = (D_j + Sigma_t)^{-1} rhs for one direction.  rhs already contains the
 * source and any inflow-boundary terms (g_j^bc).  Returns 0, or 1 if a cell
 * block is singular.
 */
int oracle_sweep_dir(int nx, int ny, int nd, const double* M, const double* C, const int* inflow,
                     const double* sigt, const double* rhs, double* psi) {
  double A[64], b[8];
  if (nd > 8) return 2;
  int x_up = inflow[0] ? 1 : (inflow[1] ? -1 : 1);  /* +1: sweep x ascending */
  int y_up = inflow[2] ? 1 : (inflow[3] ? -1 : 1);
  for (int sy = 0; sy < ny; ++sy) {
    int iy = y_up > 0 ? sy : ny - 1 - sy;
    for (int sx = 0; sx < nx; ++sx) {
      int ix = x_up > 0 ? sx : nx - 1 - sx;
      int c = iy * nx + ix;
      for (int k = 0; k < nd; ++k) b[k] = rhs[c * nd + k];
      for (int f = 0; f < 4; ++f) {
        if (!inflow[f]) continue;
        int nb = neighbour(nx, ny, ix, iy, f);
        if (nb < 0) continue; /* inflow boundary: its data is already in rhs */
        const double* Cf = C + f * nd * nd;
        for (int k = 0; k < nd; ++k) {
          double s = 0.0;
          for (int l = 0; l < nd; ++l) s += Cf[k * nd + l] * psi[nb * nd + l];
          b[k] -= s;
        }
      }
      for (int k = 0; k < nd * nd; ++k) A[k] = M[k];
      for (int k = 0; k < nd; ++k) A[k * nd + k] += sigt[c];
      if (dense_solve(nd, A, b)) return 1;
      for (int k = 0; k < nd; ++k) psi[c * nd + k] = b[k];
    }
  }
  return 0;
}

/*
 * w = (D_j + Sigma_t) x for one direction (the forward operator; inflow-
 * boundary faces carry no term, matching the definition of D_j).
 */
int oracle_apply_dir(int nx, int ny, int nd, const double* M, const double* C, const int* inflow,
                     const double* sigt, const double* x, double* w) {
  for (int iy = 0; iy < ny; ++iy) {
    for (int ix = 0; ix < nx; ++ix) {
      int c = iy * nx + ix;
      for (int k = 0; k < nd; ++k) {
        double s = sigt[c] * x[c * nd + k];
        for (int l = 0; l < nd; ++l) s += M[k * nd + l] * x[c * nd + l];
        for (int f = 0; f < 4; ++f) {
          if (!inflow[f]) continue;
          int nb = neighbour(nx, ny, ix, iy, f);
          if (nb < 0) continue;
          const double* Cf = C + f * nd * nd;
          for (int l = 0; l < nd; ++l) s += Cf[k * nd + l] * x[nb * nd + l];
        }
        w[c * nd + k] = s;
      }
    }
  }
  return 0;
}

/*
 * The same two operators when Sigma_t is a full nd x nd block per cell (Sec. 2.3: (Sigma_t)_kl is the
 * integral of sigma_t eta_k eta_l over the cell, which is not diagonal when sigma_t varies inside it).
 * St holds the blocks row-major, cell after cell: St[(c*nd + k)*nd + l].
 */
int oracle_sweep_dir_blk(int nx, int ny, int nd, const double* M, const double* C, const int* inflow,
                         const double* St, const double* rhs, double* psi) {
  double A[64], b[8];
  if (nd > 8) return 2;
  int x_up = inflow[0] ? 1 : (inflow[1] ? -1 : 1);
  int y_up = inflow[2] ? 1 : (inflow[3] ? -1 : 1);
  for (int sy = 0; sy < ny; ++sy) {
    int iy = y_up > 0 ? sy : ny - 1 - sy;
    for (int sx = 0; sx < nx; ++sx) {
      int ix = x_up > 0 ? sx : nx - 1 - sx;
      int c = iy * nx + ix;
      for (int k = 0; k < nd; ++k) b[k] = rhs[c * nd + k];
      for (int f = 0; f < 4; ++f) {
        if (!inflow[f]) continue;
        int nb = neighbour(nx, ny, ix, iy, f);
        if (nb < 0) continue;
        const double* Cf = C + f * nd * nd;
        for (int k = 0; k < nd; ++k) {
          double s = 0.0;
          for (int l = 0; l < nd; ++l) s += Cf[k * nd + l] * psi[nb * nd + l];
          b[k] -= s;
        }
      }
      for (int k = 0; k < nd * nd; ++k) A[k] = M[k] + St[(size_t)c * nd * nd + k];
      if (dense_solve(nd, A, b)) return 1;
      for (int k = 0; k < nd; ++k) psi[c * nd + k] = b[k];
    }
  }
  return 0;
}

int oracle_apply_dir_blk(int nx, int ny, int nd, const double* M, const double* C, const int* inflow,
                         const double* St, const double* x, double* w) {
  for (int iy = 0; iy < ny; ++iy) {
    for (int ix = 0; ix < nx; ++ix) {
      int c = iy * nx + ix;
      for (int k = 0; k < nd; ++k) {
        double s = 0.0;
        for (int l = 0; l < nd; ++l) s += (M[k * nd + l] + St[((size_t)c * nd + k) * nd + l]) * x[c * nd + l];
        for (int f = 0; f < 4; ++f) {
          if (!inflow[f]) continue;
          int nb = neighbour(nx, ny, ix, iy, f);
          if (nb < 0) continue;
          const double* Cf = C + f * nd * nd;
          for (int l = 0; l < nd; ++l) s += Cf[k * nd + l] * x[nb * nd + l];
        }
        w[c * nd + k] = s;
      }
    }
  }
  return 0;
}
