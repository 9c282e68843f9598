// RBF-interpolated initial guess: the interpolation baseline of the paper's experiments (Sec. 5, the
// "Interp-IG" columns), which interpolates the high-fidelity scalar fluxes of sampled parameters.
//
// Features x = (log sigma_s[R], sigma_a[R]) standardised by the samples' mean and standard deviation (scale 1
// for a feature without spread); polyharmonic cubic kernel |x - x_k|^3 with a degree-1 polynomial term.  The
// interpolant of data F = [phi_1 .. phi_K]^T is s(x) = [g(x); p(x)]^T A^{-1} [F; 0] with A the symmetric
// saddle-point matrix [[Phi, P], [P^T, 0]], Phi_kl = |x_k - x_l|^3, P_k = (1, x_k), g_k(x) = |x - x_k|^3,
// p(x) = (1, x).  So s(x) = sum_k w_k(x) phi_k with the cardinal weights w(x) = (A^{-1} [g(x); p(x)])[0:K]:
// A^{-1} is formed once at create (host, FP64, Gauss-Jordan with partial pivoting), the weights per instance
// on the host (O(K^2)), and the N-long combination on the GPU.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

struct rte_rbf {
  int K = 0, R = 0, d = 0, dim = 2, nx = 0, ny = 0, nd = 4, rx = 1, ry = 1;
  double hx = 0, hy = 0;
  long long N = 0;
  std::vector<double> mean, scale, X;   // X [K][d] standardised
  std::vector<double> Ainv;             // [(K+d+1)^2]
  rte::DevBuf<double> sol;              // [K][N]
  rte::DevBuf<double> w;                // [B][K] of the last call
};

namespace rte {
namespace {

__global__ void k_rbf_combine(const double* sol, int K, long long N, const double* w, const InstInfo* inst,
                              double* phi0) {
  const int b = blockIdx.y;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double* wb = w + (size_t)b * K;
  double s = 0.0;
  for (int k = 0; k < K; ++k) s += wb[k] * sol[(size_t)k * N + i];
  phi0[inst[b].off + i] = s;
}

void feat(const double* ss, const double* sa, int R, double* x) {
  for (int q = 0; q < R; ++q) {
    x[q] = std::log(ss[q]);
    x[R + q] = sa[q];
  }
}

// in-place inverse of the n x n row-major matrix A; false if a pivot vanishes
bool invert(std::vector<double>& A, int n) {
  std::vector<double> I((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1.0;
  double amax = 0.0;
  for (double v : A) amax = std::max(amax, std::fabs(v));
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)piv * n + c])) piv = r;
    if (!(std::fabs(A[(size_t)piv * n + c]) > 1e-14 * amax)) return false;
    if (piv != c)
      for (int j = 0; j < n; ++j) {
        std::swap(A[(size_t)piv * n + j], A[(size_t)c * n + j]);
        std::swap(I[(size_t)piv * n + j], I[(size_t)c * n + j]);
      }
    const double inv = 1.0 / A[(size_t)c * n + c];
    for (int j = 0; j < n; ++j) {
      A[(size_t)c * n + j] *= inv;
      I[(size_t)c * n + j] *= inv;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = A[(size_t)r * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        A[(size_t)r * n + j] -= f * A[(size_t)c * n + j];
        I[(size_t)r * n + j] -= f * I[(size_t)c * n + j];
      }
    }
  }
  A.swap(I);
  return true;
}

}  // namespace
}  // namespace rte

using namespace rte;

extern "C" int rte_rbf_create(rte_problem_t tmpl, int K, const double* sigma_s, const double* sigma_a,
                              const void* solutions, rte_rbf_t* out) {
  RTE_ARG(tmpl && sigma_s && sigma_a && solutions && out, "null handle or pointer");
  *out = nullptr;
  const int R = tmpl->R, d = 2 * R;
  RTE_ARG(K >= d + 2, "rte_rbf_create needs at least 2R + 2 samples (the degree-1 polynomial term)");
  for (long long e = 0; e < (long long)K * R; ++e)
    RTE_ARG(sigma_s[e] > 0.0 && std::isfinite(sigma_a[e]), "sigma_s must be positive and sigma_a finite");
  rte_rbf* f = new rte_rbf();
  f->K = K;
  f->R = R;
  f->d = d;
  f->dim = tmpl->dim;
  f->nx = tmpl->inst[0].nx;
  f->ny = tmpl->inst[0].ny;
  f->nd = tmpl->nd;
  f->rx = tmpl->rx;
  f->ry = tmpl->ry;
  f->hx = tmpl->inst[0].hx;
  f->hy = tmpl->inst[0].hy;
  f->N = tmpl->off[1] - tmpl->off[0];
  // standardised features
  std::vector<double> X((size_t)K * d);
  for (int k = 0; k < K; ++k) feat(sigma_s + (size_t)k * R, sigma_a + (size_t)k * R, R, &X[(size_t)k * d]);
  f->mean.assign(d, 0.0);
  f->scale.assign(d, 1.0);
  for (int j = 0; j < d; ++j) {
    double m = 0.0, v = 0.0;
    for (int k = 0; k < K; ++k) m += X[(size_t)k * d + j];
    m /= K;
    for (int k = 0; k < K; ++k) v += (X[(size_t)k * d + j] - m) * (X[(size_t)k * d + j] - m);
    const double sd = std::sqrt(v / K);
    f->mean[j] = m;
    f->scale[j] = sd > 0.0 ? sd : 1.0;
    for (int k = 0; k < K; ++k) X[(size_t)k * d + j] = (X[(size_t)k * d + j] - m) / f->scale[j];
  }
  f->X = X;
  // augmented system and its inverse
  const int n = K + d + 1;
  std::vector<double> A((size_t)n * n, 0.0);
  for (int k = 0; k < K; ++k) {
    for (int l = 0; l < K; ++l) {
      double r2 = 0.0;
      for (int j = 0; j < d; ++j) {
        const double t = X[(size_t)k * d + j] - X[(size_t)l * d + j];
        r2 += t * t;
      }
      A[(size_t)k * n + l] = r2 * std::sqrt(r2);
    }
    A[(size_t)k * n + K] = A[(size_t)K * n + k] = 1.0;
    for (int j = 0; j < d; ++j) A[(size_t)k * n + K + 1 + j] = A[(size_t)(K + 1 + j) * n + k] = X[(size_t)k * d + j];
  }
  if (!invert(A, n)) {
    delete f;
    set_error("rte_rbf_create: the interpolation system is singular (repeated or affinely dependent samples)");
    return RTE_ERR_NUMERIC;
  }
  f->Ainv.swap(A);
  int s = f->sol.alloc((size_t)K * f->N);
  if (s == RTE_OK) {
    cudaError_t e = cudaMemcpy(f->sol.p, solutions, (size_t)K * f->N * sizeof(double), cudaMemcpyDefault);
    if (e != cudaSuccess) {
      set_error(std::string("rte_rbf_create: ") + cudaGetErrorString(e));
      s = RTE_ERR_CUDA;
    }
  }
  if (s != RTE_OK) {
    delete f;
    return s;
  }
  *out = f;
  return RTE_OK;
}

extern "C" int rte_rbf_initial_guess(rte_rbf_t f, rte_problem_t p, void* phi0, void* stream) {
  RTE_ARG(f && p && phi0, "null handle or pointer");
  RTE_ARG(p->R == f->R && p->rx == f->rx && p->ry == f->ry && p->dim == f->dim, "region grid differs");
  for (int b = 0; b < p->B; ++b) {
    const InstInfo& in = p->inst[b];
    RTE_ARG(in.nx == f->nx && in.ny == f->ny && std::fabs(in.hx - f->hx) <= 1e-12 * f->hx &&
                std::fabs(in.hy - f->hy) <= 1e-12 * f->hy,
            "every instance must use the mesh of the samples");
  }
  for (double v : p->ss) RTE_ARG(v > 0.0, "the RBF features take log sigma_s: sigma_s must be positive");
  cudaStream_t st = (cudaStream_t)stream;
  const int K = f->K, d = f->d, n = K + d + 1, B = p->B;
  std::vector<double> w((size_t)B * K), x(d), rhs(n);
  for (int b = 0; b < B; ++b) {
    feat(p->ss.data() + (size_t)b * f->R, p->sa.data() + (size_t)b * f->R, f->R, x.data());
    for (int j = 0; j < d; ++j) x[j] = (x[j] - f->mean[j]) / f->scale[j];
    for (int k = 0; k < K; ++k) {
      double r2 = 0.0;
      for (int j = 0; j < d; ++j) {
        const double t = x[j] - f->X[(size_t)k * d + j];
        r2 += t * t;
      }
      rhs[k] = r2 * std::sqrt(r2);
    }
    rhs[K] = 1.0;
    for (int j = 0; j < d; ++j) rhs[K + 1 + j] = x[j];
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int m = 0; m < n; ++m) s += f->Ainv[(size_t)k * n + m] * rhs[m];   // A^{-1} is symmetric
      w[(size_t)b * K + k] = s;
    }
  }
  RTE_TRY(f->w.ensure(w.size()));
  RTE_CHECK_CUDA(cudaMemcpyAsync(f->w.p, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  k_rbf_combine<<<dim3((unsigned)((f->N + 255) / 256), B), 256, 0, st>>>(f->sol.p, K, f->N, f->w.p, p->d_inst.p,
                                                                           (double*)phi0);
  count_launch();
  RTE_CHECK_CUDA(cudaGetLastError());
  RTE_CHECK_CUDA(cudaStreamSynchronize(st));   // w (host) must outlive the copy
  return RTE_OK;
}

extern "C" int rte_rbf_destroy(rte_rbf_t f) {
  delete f;
  return RTE_OK;
}
