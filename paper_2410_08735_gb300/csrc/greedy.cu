// Greedy ROM construction for the ROMSAD preconditioner (paper Sec. 4.4.2), on the GPU.
//
//   1  b~_mu for every training parameter (one batched sweep) and eta_mu^(0) = Sigma_s b~_mu.
//   2a high-fidelity FGMRES for the sampled mu_k, first cycle recorded; xi recurrence
//      xi^(1) = (phi - phi^(0)) / ||r^(0)||, xi^(l) = (z^(l-1) - sum_{i<l} H_{i,l-1} xi^(i)) / H_{l,l-1}
//      (eqs. correction-fgmres1/2).
//   2b angular corrections delta psi^(l)_j = (D_j + Sigma_t)^{-1} Sigma_s xi^(l) (eq. fgmres-psi-correction).
//   2c modified Gram-Schmidt with truncation (appendix B) into U_r, then P, W and the affine
//      reduced operators.
//   3  for every unsampled mu: c = (U^T A_mu U)^{-1} P^T eta^(0) (eq. greedy-rom) and the indicator
//      max_j ||(D_j + Sigma_t) U_j c - Sigma_s W c - eta^(0)|| (eq. rom-residual); sample the argmax.
//
// Readings where the paper is silent: the indicator is divided by ||eta^(0)||_2 before the eps_ROM
// test; the truncation test is relative to the snapshot norm; the high-fidelity solve is FGMRES-DSA as in
// the paper (partially consistent DSA through one V-cycle; opts->hf_dsa) or FGMRES with M = I;
// argmax ties go to the lowest index; mu_1 defaults to the training point nearest the centroid of
// (log sigma_s, sigma_a).  U is stored per unique in-plane direction (the +-Omega_z duplicates have
// identical angular fluxes) with the duplicate count as weight of the inner product.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "romsad.h"

namespace rte {

// Weighted dot of two stored-angular vectors: sum_a mult_a x_a . y_a; per-block partials.
__global__ void k_wdot(const double* x, const double* y, int nA, int N, const double* mult, double* part) {
  __shared__ double sh[256];
  double s = 0.0;
  const long long tot = (long long)nA * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x)
    s += mult[i / N] * x[i] * y[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_axpy(double* y, const double* x, double a, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}

__global__ void k_scal_copy(double* y, const double* x, double a, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

__global__ void k_to_f32(float* y, const double* x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

// base_mu[i] = sigma_s(i) (W c_mu)[i] + eta0_mu[i], eta0 = sigma_s b~; one instance per blockIdx.y
// With cross-section profiles (F: the profile blocks, sigma_s = c_0 F + c_1 I per cell) the cell's Sigma_s block
// multiplies the cell's four values of W c_mu + b~.
__global__ void k_base(const double* W, int rmax, int r, const double* c, const double* bt, const InstInfo* inst,
                       const double* sig_s, int R, int rx, int ry, int nd, const double* F, double* base) {
  const int b = blockIdx.y;
  const InstInfo in = inst[b];
  const int cx = in.nx / rx, cy = in.ny / ry;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < in.ndof; i += gridDim.x * blockDim.x) {
    const int cell = i / nd;
    if (F) {
      double x[4];
      for (int l = 0; l < 4; ++l) {
        const int il = 4 * cell + l;
        double s = 0.0;
        for (int k = 0; k < r; ++k) s += W[(size_t)il * rmax + k] * c[(size_t)b * 64 + k];
        x[l] = s + bt[in.off + il];
      }
      const double* Fr = F + (size_t)cell * 16 + (i & 3) * 4;
      base[in.off + i] = sig_s[(size_t)b * R] * (Fr[0] * x[0] + Fr[1] * x[1] + Fr[2] * x[2] + Fr[3] * x[3]) +
                         sig_s[(size_t)b * R + 1] * x[i & 3];
      continue;
    }
    const int ix = cell % in.nx, iy = cell / in.nx;
    const double sg = sig_s[(size_t)b * R + (iy / cy) * rx + ix / cx];
    double s = 0.0;
    for (int k = 0; k < r; ++k) s += W[(size_t)i * rmax + k] * c[(size_t)b * 64 + k];
    base[in.off + i] = sg * (s + bt[in.off + i]);
  }
}

// (F x)_i for the profile blocks F with the dofs of a cell on four consecutive lanes (i = chunk * 256 + thread, so
// i mod 4 = lane mod 4): gathers the cell's four x by shuffles; every lane of the warp calls it.  0 without F.
__device__ __forceinline__ double profile_times(const double* F, int i, double x, bool ok) {
  if (!F) return 0.0;
  const int g = (threadIdx.x & 31) & ~3;
  const double x0 = __shfl_sync(0xffffffffu, x, g), x1 = __shfl_sync(0xffffffffu, x, g + 1);
  const double x2 = __shfl_sync(0xffffffffu, x, g + 2), x3 = __shfl_sync(0xffffffffu, x, g + 3);
  if (!ok) return 0.0;
  const double* Fr = F + (size_t)(i >> 2) * 16 + (i & 3) * 4;
  return Fr[0] * x0 + Fr[1] * x1 + Fr[2] * x2 + Fr[3] * x3;
}

// Squared residual norms of eq. rom-residual, one partial per (mu, u, dof chunk):
//   e_i = sum_k (Y[k][u][i] + sigma_t(i) U[k][u][i]) c_mu[k] - base_mu[i]
// A block holds a chunk of 256 dofs of one direction u and a tile of MT parameters: each U/Y value
// is read once and used for all MT parameters (accumulators in registers).
template <typename T, int MT>
__global__ void k_indicator(const T* U, const T* Y, int nA, int N, int r, const double* c,
                            const double* base, const int* mus, int nmu, const double* sig_t, int R, int rx, int ry,
                            int nx, int ny, int nd, const double* F, double* part) {
  const int u = blockIdx.y;
  const int chunk = blockIdx.x;
  const int mt0 = blockIdx.z * MT;
  const int i = chunk * 256 + threadIdx.x;
  __shared__ T cs[64][MT];
  __shared__ double red[8][MT];
  for (int e = threadIdx.x; e < MT * 64; e += blockDim.x) {
    const int k = e / MT, m = e % MT;
    cs[k][m] = (T)((mt0 + m < nmu && k < r) ? c[(size_t)mus[mt0 + m] * 64 + k] : 0.0);
  }
  __syncthreads();
  T a[MT], b[MT];
#pragma unroll
  for (int m = 0; m < MT; ++m) { a[m] = (T)0; b[m] = (T)0; }
  int reg = 0;
  if (i < N) {
    for (int k = 0; k < r; ++k) {
      const T yk = Y[((size_t)k * nA + u) * N + i];
      const T uk = U[((size_t)k * nA + u) * N + i];
#pragma unroll
      for (int m = 0; m < MT; ++m) {
        a[m] += yk * cs[k][m];
        b[m] += uk * cs[k][m];
      }
    }
    const int cell = i / nd;
    const int ix = cell % nx, iy = cell / nx;
    reg = (iy / (ny / ry)) * rx + ix / (nx / rx);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int m = 0; m < MT; ++m) {
    double e2 = 0.0;
    const double fb = profile_times(F, i, (double)b[m], i < N);   // (F (U c))_i with profiles
    if (i < N && mt0 + m < nmu) {
      const int mu = mus[mt0 + m];
      const double st = F ? sig_t[(size_t)mu * R + 1] : sig_t[(size_t)mu * R + reg];
      double e = (double)a[m] + st * (double)b[m] - base[(size_t)mu * N + i];
      if (F) e += sig_t[(size_t)mu * R] * fb;
      e2 = e * e;
    }
    for (int o = 16; o > 0; o >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, o);
    if (lane == 0) red[warp][m] = e2;
  }
  __syncthreads();
  if (threadIdx.x < MT && mt0 + threadIdx.x < nmu) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w][threadIdx.x];
    part[(((size_t)mus[mt0 + threadIdx.x]) * nA + u) * gridDim.x + chunk] = s;   // indexed by training point
  }
}

// FP32 indicator for many parameters: a thread keeps the RMAX basis values U[k][u][i], Y[k][u][i] of its dof in
// registers and loops over all parameters in tiles of MT (coefficients of a tile staged in shared memory), so
// the basis is read from HBM once per greedy iteration.  Block (u, chunk): the blocks of one chunk follow one
// another in launch order, so the chunk of base_mu is read from HBM once and by the other directions' blocks
// from L2.  Same partial sums as k_indicator.
template <int RMAX, int MT>
__global__ void __launch_bounds__(256) k_indicator_reg(const float* U, const float* Y, int nA, int N, int r,
                                                       const double* c, const double* base, const int* mus, int nmu,
                                                       const double* sig_t, int R, int rx, int ry, int nx, int ny,
                                                       int nd, const double* F, int nchunk, double* part) {
  const int u = blockIdx.x;
  const int chunk = blockIdx.y;
  const int i = chunk * 256 + threadIdx.x;
  __shared__ __align__(16) float cs[MT][RMAX];
  __shared__ double red[8][MT];
  float uk[RMAX], yk[RMAX];
#pragma unroll
  for (int k = 0; k < RMAX; ++k) {
    uk[k] = 0.f;
    yk[k] = 0.f;
    if (k < r && i < N) {
      yk[k] = Y[((size_t)k * nA + u) * N + i];
      uk[k] = U[((size_t)k * nA + u) * N + i];
    }
  }
  int reg = 0;
  if (i < N) {
    const int cell = i / nd;
    const int ix = cell % nx, iy = cell / nx;
    reg = (iy / (ny / ry)) * rx + ix / (nx / rx);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int mt0 = 0; mt0 < nmu; mt0 += MT) {
    __syncthreads();   // the previous tile's coefficients and sums are consumed
    for (int e = threadIdx.x; e < MT * RMAX; e += blockDim.x) {
      const int m = e / RMAX, k = e % RMAX;
      cs[m][k] = (mt0 + m < nmu && k < r) ? (float)c[(size_t)mus[mt0 + m] * 64 + k] : 0.f;
    }
    __syncthreads();
    float a[MT], b[MT];
#pragma unroll
    for (int m = 0; m < MT; ++m) { a[m] = 0.f; b[m] = 0.f; }
#pragma unroll
    for (int k = 0; k < RMAX; k += 4) {
#pragma unroll
      for (int m = 0; m < MT; ++m) {
        const float4 cc = *reinterpret_cast<const float4*>(&cs[m][k]);
        a[m] += yk[k] * cc.x + yk[k + 1] * cc.y + yk[k + 2] * cc.z + yk[k + 3] * cc.w;
        b[m] += uk[k] * cc.x + uk[k + 1] * cc.y + uk[k + 2] * cc.z + uk[k + 3] * cc.w;
      }
    }
#pragma unroll
    for (int m = 0; m < MT; ++m) {
      double e2 = 0.0;
      const double fb = profile_times(F, i, (double)b[m], i < N);   // (F (U c))_i with profiles
      if (i < N && mt0 + m < nmu) {
        const int mu = mus[mt0 + m];
        const double st = F ? sig_t[(size_t)mu * R + 1] : sig_t[(size_t)mu * R + reg];
        double e = (double)a[m] + st * (double)b[m] - base[(size_t)mu * N + i];
        if (F) e += sig_t[(size_t)mu * R] * fb;
        e2 = e * e;
      }
      for (int o = 16; o > 0; o >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, o);
      if (lane == 0) red[warp][m] = e2;
    }
    __syncthreads();
    if (threadIdx.x < MT && mt0 + threadIdx.x < nmu) {
      double sum = 0.0;
      for (int w = 0; w < 8; ++w) sum += red[w][threadIdx.x];
      part[(((size_t)mus[mt0 + threadIdx.x]) * nA + u) * nchunk + chunk] = sum;
    }
  }
}

static int wdot(const double* x, const double* y, int nA, int N, const double* mult, DevBuf<double>& part,
                double* out, cudaStream_t st) {
  const int blocks = 256;
  RTE_TRY(part.ensure(blocks));
  k_wdot<<<blocks, 256, 0, st>>>(x, y, nA, N, mult, part.p);
  count_launch();
  RTE_CHECK_CUDA(cudaGetLastError());
  std::vector<double> h(blocks);
  RTE_CHECK_CUDA(cudaMemcpyAsync(h.data(), part.p, blocks * 8, cudaMemcpyDeviceToHost, st));
  RTE_CHECK_CUDA(cudaStreamSynchronize(st));
  double s = 0.0;
  for (double v : h) s += v;
  *out = s;
  return RTE_OK;
}

static int make_problem_like(const rte_problem* tmpl, int n, const double* ss, const double* sa, rte_problem_t* out) {
  std::vector<int> nx(n, tmpl->nx[0]), ny(n, tmpl->ny[0]);
  rte_problem_desc d{};
  d.dim = tmpl->dim;
  d.n_instances = n;
  d.nx = nx.data();
  d.ny = ny.data();
  std::memcpy(d.box, tmpl->box, sizeof(d.box));
  d.n_polar = tmpl->n_polar;
  d.n_azim = tmpl->n_azim;
  d.rx = tmpl->rx;
  d.ry = tmpl->ry;
  d.sigma_s = ss;
  d.sigma_a = sa;
  d.src_q = tmpl->src_q;
  std::memcpy(d.src_box, tmpl->src_box, sizeof(d.src_box));
  d.src_kind = tmpl->src_kind;
  std::memcpy(d.src_gauss, tmpl->src_gauss, sizeof(d.src_gauss));
  d.inflow_g = tmpl->inst[0].g;
  d.inflow_faces = tmpl->inflow_mask;
  d.sigma_modes = tmpl->cellsig ? RTE_SIGMA_VARSCAT : RTE_SIGMA_REGIONS;
  return rte_problem_create(&d, out);
}

struct ProblemGuard {
  rte_problem_t p = nullptr;
  ~ProblemGuard() {
    if (p) rte_problem_destroy(p);
  }
};

static int greedy_impl(rte_problem* tmpl, int n_train, const double* tss, const double* tsa,
                       const romsad_greedy_opts* o, romsad* rom, romsad_report* rep) {
  cudaStream_t st = 0;
  const int R = tmpl->R;
  const int window = o->window;
  // training problem (n_train instances on the template mesh) and the high-fidelity problem
  ProblemGuard tp, hp;
  RTE_TRY(make_problem_like(tmpl, n_train, tss, tsa, &tp.p));
  RTE_TRY(make_problem_like(tmpl, 1, tss, tsa, &hp.p));
  const int N = (int)(tp.p->off[1] - tp.p->off[0]);
  // Step 1: b~_mu for all training parameters (FP64 batched sweep)
  DevBuf<double> bt;
  RTE_TRY(bt.alloc((size_t)n_train * N));
  RTE_TRY(launch_T(tp.p, MODE_RHS, true, nullptr, true, nullptr, bt.p, true, nullptr, st));
  std::vector<double> eta_norm(n_train);
  {
    // ||eta0_mu|| = ||Sigma_s b~_mu||: base with c = 0 is exactly eta0
    DevBuf<double> zc, base;
    RTE_TRY(zc.alloc((size_t)n_train * 64));
    RTE_CHECK_CUDA(cudaMemsetAsync(zc.p, 0, zc.n * 8, st));
    RTE_TRY(base.alloc((size_t)n_train * N));
    dim3 g((N + 255) / 256, n_train);
    k_base<<<g, 256, 0, st>>>(rom->W.p, rom->rmax, 0, zc.p, bt.p, tp.p->d_inst.p, tp.p->d_sig_s.p, R, tp.p->rx,
                              tp.p->ry, tp.p->nd, tp.p->cellsig ? tp.p->d_F64.p : nullptr, base.p);
    count_launch();
    std::vector<double> h((size_t)n_train * N);
    RTE_CHECK_CUDA(cudaMemcpyAsync(h.data(), base.p, h.size() * 8, cudaMemcpyDeviceToHost, st));
    RTE_CHECK_CUDA(cudaStreamSynchronize(st));
    for (int m = 0; m < n_train; ++m) {
      double s = 0.0;
      for (int i = 0; i < N; ++i) s += h[(size_t)m * N + i] * h[(size_t)m * N + i];
      eta_norm[m] = std::sqrt(s);
    }
  }
  // mu_1
  int k_idx = o->mu1;
  if (k_idx < 0 || k_idx >= n_train) {
    std::vector<double> cen(2 * R, 0.0);
    for (int m = 0; m < n_train; ++m)
      for (int q = 0; q < R; ++q) {
        cen[q] += std::log(tss[(size_t)m * R + q]) / n_train;
        cen[R + q] += tsa[(size_t)m * R + q] / n_train;
      }
    double best = 1e300;
    k_idx = 0;
    for (int m = 0; m < n_train; ++m) {
      double d = 0.0;
      for (int q = 0; q < R; ++q) {
        const double a = std::log(tss[(size_t)m * R + q]) - cen[q], b = tsa[(size_t)m * R + q] - cen[R + q];
        d += a * a + b * b;
      }
      if (d < best) { best = d; k_idx = m; }
    }
  }
  std::vector<int> sampled{k_idx};
  std::vector<char> is_sampled(n_train, 0);
  is_sampled[k_idx] = 1;
  std::vector<double> max_ind;
  DevBuf<double> d_mult, d_wA, part, phi, xi, snap, work;
  RTE_TRY(d_mult.alloc(rom->nA));
  RTE_TRY(d_wA.alloc(rom->nA));
  RTE_CHECK_CUDA(cudaMemcpy(d_mult.p, rom->mult.data(), rom->nA * 8, cudaMemcpyHostToDevice));
  RTE_CHECK_CUDA(cudaMemcpy(d_wA.p, rom->wA.data(), rom->nA * 8, cudaMemcpyHostToDevice));
  RTE_TRY(phi.alloc(N));
  RTE_TRY(xi.alloc((size_t)std::max(1, window) * N));
  const long long nang = (long long)rom->nA * N;
  RTE_TRY(snap.alloc(nang));
  DevBuf<float> U32, Y32;   // FP32 copies of the basis for the FP32 indicator
  if (o->indicator_f32) {
    RTE_TRY(U32.alloc((size_t)rom->rmax * nang));
    RTE_TRY(Y32.alloc((size_t)rom->rmax * nang));
  }
  const unsigned vb = (unsigned)std::min<long long>(4096, (nang + 255) / 256);
  while (true) {
    // Step 2(a): high-fidelity solve for mu_k, first cycle recorded
    RTE_TRY(rte_problem_set_params(hp.p, tss + (size_t)k_idx * R, tsa + (size_t)k_idx * R));
    FirstCycle rec;
    rec.want = window;
    int its = 0, hst = 0;
    RTE_TRY(hf_solve(hp.p, o->hf_rtol, o->hf_restart, o->hf_max_iter, o->hf_dsa ? RTE_DSA_PARTIAL : -1, phi.p, &rec,
                     &its, &hst));
    if (hst != RTE_OK) {
      set_error("romsad_build_greedy: high-fidelity solve did not converge (raise hf_max_iter or hf_restart)");
      return RTE_ERR_NOT_CONVERGED;
    }
    // xi recurrence (eqs. correction-fgmres1/2), zero initial guess
    int nxi = 0;
    k_scal_copy<<<(N + 255) / 256, 256, 0, st>>>(xi.p, phi.p, 1.0 / rec.beta, N);
    count_launch();
    nxi = 1;
    for (int l = 2; l <= window; ++l) {
      // needs z^(l-1) and H_{l, l-1} from the first cycle
      const int col = l - 2;
      if (col >= rec.nz || col + 1 > rec.k) break;
      const double hll = rec.H[(size_t)col * (rec.m + 1) + (l - 1)];
      if (!(std::fabs(hll) > 0.0)) break;
      double* x = xi.p + (size_t)(l - 1) * N;
      k_scal_copy<<<(N + 255) / 256, 256, 0, st>>>(x, rec.Z.p + (size_t)col * N, 1.0, N);
      count_launch();
      for (int i = 1; i < l; ++i) {
        const double hi = rec.H[(size_t)col * (rec.m + 1) + (i - 1)];
        k_axpy<<<(N + 255) / 256, 256, 0, st>>>(x, xi.p + (size_t)(i - 1) * N, -hi, N);
        count_launch();
      }
      k_scal_copy<<<(N + 255) / 256, 256, 0, st>>>(x, x, 1.0 / hll, N);
      count_launch();
      ++nxi;
    }
    RTE_CHECK_CUDA(cudaGetLastError());
    // Steps 2(b), 2(c): snapshots, MGS with truncation, operators
    for (int l = 0; l < nxi && rom->r < o->max_rank; ++l) {
      RTE_TRY(launch_angular(hp.p, true, xi.p + (size_t)l * N, 0, snap.p, st, true, true));
      double n0 = 0.0;
      RTE_TRY(wdot(snap.p, snap.p, rom->nA, N, d_mult.p, part, &n0, st));
      n0 = std::sqrt(n0);
      for (int c = 0; c < rom->r; ++c) {
        double h = 0.0;
        const double* Uc = rom->U.p + (size_t)c * nang;
        RTE_TRY(wdot(Uc, snap.p, rom->nA, N, d_mult.p, part, &h, st));
        k_axpy<<<vb, 256, 0, st>>>(snap.p, Uc, -h, nang);
        count_launch();
      }
      double nu = 0.0;
      RTE_TRY(wdot(snap.p, snap.p, rom->nA, N, d_mult.p, part, &nu, st));
      nu = std::sqrt(nu);
      if (!(nu > o->eps_qr * n0)) continue;   // appendix B: not added
      k_scal_copy<<<vb, 256, 0, st>>>(rom->U.p + (size_t)rom->r * nang, snap.p, 1.0 / nu, nang);
      count_launch();
      RTE_TRY(rom_compute_Y_column(rom, hp.p, 0, rom->r, st));
      if (o->indicator_f32) {
        k_to_f32<<<vb, 256, 0, st>>>(U32.p + (size_t)rom->r * nang, rom->U.p + (size_t)rom->r * nang, nang);
        count_launch();
        k_to_f32<<<vb, 256, 0, st>>>(Y32.p + (size_t)rom->r * nang, rom->Y.p + (size_t)rom->r * nang, nang);
        count_launch();
      }
      RTE_TRY(rom_add_column(rom, d_mult, d_wA, st));
    }
    if ((int)sampled.size() >= o->max_greedy_iter || rom->r >= o->max_rank || (int)sampled.size() == n_train ||
        rom->r == 0)
      break;
    // Step 3: reduced solutions and indicators for the unsampled parameters
    std::vector<int> mus;
    for (int m = 0; m < n_train; ++m)
      if (!is_sampled[m]) mus.push_back(m);
    const int nmu = (int)mus.size();
    DevBuf<int> d_all, d_mus;
    DevBuf<double> ys, cs, base, ipart;
    RTE_TRY(d_all.alloc(n_train));
    RTE_TRY(d_mus.alloc(nmu));
    std::vector<int> all(n_train);
    for (int m = 0; m < n_train; ++m) all[m] = m;
    RTE_CHECK_CUDA(cudaMemcpy(d_all.p, all.data(), n_train * sizeof(int), cudaMemcpyHostToDevice));
    RTE_CHECK_CUDA(cudaMemcpy(d_mus.p, mus.data(), nmu * sizeof(int), cudaMemcpyHostToDevice));
    RTE_TRY(ys.alloc((size_t)n_train * 64));
    RTE_TRY(cs.alloc((size_t)n_train * 64));
    // y = P^T Sigma_s b~ = P^T eta0 for every training instance, then c = A_r(mu)^{-1} y
    RTE_TRY(rom_project_list(rom, tp.p, d_all.p, n_train, bt.p, ys.p, st));
    RTE_TRY(rom_small_solve(rom, tp.p, d_all.p, n_train, ys.p, cs.p, st));
    RTE_TRY(base.alloc((size_t)n_train * N));
    dim3 g((N + 255) / 256, n_train);
    k_base<<<g, 256, 0, st>>>(rom->W.p, rom->rmax, rom->r, cs.p, bt.p, tp.p->d_inst.p, tp.p->d_sig_s.p, R, tp.p->rx,
                              tp.p->ry, tp.p->nd, tp.p->cellsig ? tp.p->d_F64.p : nullptr, base.p);
    count_launch();
    const int nchunk = (N + 255) / 256;
    constexpr int MT = 8;
    RTE_TRY(ipart.alloc((size_t)n_train * rom->nA * nchunk));
    dim3 gi(nchunk, rom->nA, (nmu + MT - 1) / MT);
    const double* prof = tp.p->cellsig ? tp.p->d_F64.p : nullptr;
    if (o->indicator_f32) {
      // basis in registers, all parameters per block; RMAX the smallest of 8, 16, 32, 64 covering the rank
      dim3 gr(rom->nA, nchunk);
#define RTE_IND_REG(RM)                                                                                         \
  k_indicator_reg<RM, MT><<<gr, 256, 0, st>>>(U32.p, Y32.p, rom->nA, N, rom->r, cs.p, base.p, d_mus.p, nmu,      \
                                              tp.p->d_sig_t.p, R, tp.p->rx, tp.p->ry, tp.p->nx[0], tp.p->ny[0],  \
                                              tp.p->nd, prof, nchunk, ipart.p)
      if (rom->r <= 8) RTE_IND_REG(8);
      else if (rom->r <= 16) RTE_IND_REG(16);
      else if (rom->r <= 32) RTE_IND_REG(32);
      else RTE_IND_REG(64);
#undef RTE_IND_REG
    } else
      k_indicator<double, MT><<<gi, 256, 0, st>>>(rom->U.p, rom->Y.p, rom->nA, N, rom->r, cs.p, base.p, d_mus.p, nmu,
                                                  tp.p->d_sig_t.p, R, tp.p->rx, tp.p->ry, tp.p->nx[0], tp.p->ny[0],
                                                  tp.p->nd, prof, ipart.p);
    count_launch();
    RTE_CHECK_CUDA(cudaGetLastError());
    std::vector<double> hp_((size_t)n_train * rom->nA * nchunk);
    RTE_CHECK_CUDA(cudaMemcpy(hp_.data(), ipart.p, hp_.size() * 8, cudaMemcpyDeviceToHost));
    double best = -1.0;
    int best_i = -1;
    for (int m : mus) {
      double worst = 0.0;
      for (int u = 0; u < rom->nA; ++u) {
        double s = 0.0;
        for (int c = 0; c < nchunk; ++c) s += hp_[((size_t)m * rom->nA + u) * nchunk + c];
        worst = std::max(worst, std::sqrt(s));
      }
      const double ind = eta_norm[m] > 0 ? worst / eta_norm[m] : 0.0;
      if (ind > best) { best = ind; best_i = m; }
    }
    max_ind.push_back(best);
    if (best < o->eps_rom || best_i < 0) break;
    k_idx = best_i;
    sampled.push_back(k_idx);
    is_sampled[k_idx] = 1;
  }
  if (rep) {
    rep->n_sampled = (int)sampled.size();
    if (rep->sampled)
      for (size_t i = 0; i < sampled.size() && (int)i < o->max_greedy_iter; ++i) rep->sampled[i] = sampled[i];
    if (rep->max_indicator)
      for (int i = 0; i < (int)sampled.size() && i < o->max_greedy_iter; ++i)
        rep->max_indicator[i] = i < (int)max_ind.size() ? max_ind[i] : std::nan("");   // NaN: not evaluated
    rep->rank = rom->r;
    if (rep->labels && rom->r > 0) {
      // Galerkin coefficients of eq. greedy-rom on the final basis for every training parameter
      DevBuf<int> d_all;
      DevBuf<double> ys, cs;
      RTE_TRY(d_all.alloc(n_train));
      RTE_TRY(ys.alloc((size_t)n_train * 64));
      RTE_TRY(cs.alloc((size_t)n_train * 64));
      std::vector<int> all(n_train);
      for (int m = 0; m < n_train; ++m) all[m] = m;
      RTE_CHECK_CUDA(cudaMemcpy(d_all.p, all.data(), n_train * sizeof(int), cudaMemcpyHostToDevice));
      RTE_TRY(rom_project_list(rom, tp.p, d_all.p, n_train, bt.p, ys.p, st));
      RTE_TRY(rom_small_solve(rom, tp.p, d_all.p, n_train, ys.p, cs.p, st));
      std::vector<double> h((size_t)n_train * 64);
      RTE_CHECK_CUDA(cudaMemcpy(h.data(), cs.p, h.size() * 8, cudaMemcpyDeviceToHost));
      for (int m = 0; m < n_train; ++m)
        for (int k = 0; k < rom->r; ++k) rep->labels[(size_t)m * o->max_rank + k] = h[(size_t)m * 64 + k];
    }
  }
  return RTE_OK;
}

}  // namespace rte

using namespace rte;

extern "C" int romsad_build_greedy(rte_problem_t tmpl, int n_train, const double* train_sigma_s,
                                   const double* train_sigma_a, const romsad_greedy_opts* o, romsad_t* out,
                                   romsad_report* rep) {
  RTE_ARG(tmpl && train_sigma_s && train_sigma_a && o && out, "null handle or pointer");
  RTE_ARG(n_train >= 1, "n_train must be >= 1");
  RTE_ARG(o->window >= 1 && o->max_greedy_iter >= 1 && o->max_rank >= 1 && o->max_rank <= 64,
          "window >= 1, max_greedy_iter >= 1, 1 <= max_rank <= 64");
  RTE_ARG(o->hf_restart >= 1 && o->hf_restart <= 128 && o->hf_max_iter >= 1 && o->hf_rtol > 0,
          "high-fidelity solver options out of range");
  RTE_ARG(o->window <= o->hf_restart, "window must not exceed the high-fidelity restart length");
  *out = nullptr;
  romsad* rom = new romsad();
  rom_init_geometry(rom, tmpl, 0);
  rom->nA = tmpl->nu;
  rom->uidx.resize(tmpl->nu);
  rom->mult.resize(tmpl->nu);
  rom->wA.resize(tmpl->nu);
  rom->dir_block = tmpl->uniq_of_dir;
  for (int u = 0; u < tmpl->nu; ++u) {
    rom->uidx[u] = u;
    rom->mult[u] = tmpl->udir[u].ndup;
    rom->wA[u] = tmpl->udir[u].w;
  }
  int s = rom_alloc_arrays(rom, o->max_rank, true);
  if (s == RTE_OK) s = greedy_impl(tmpl, n_train, train_sigma_s, train_sigma_a, o, rom, rep);
  if (s == RTE_OK && rom->r == 0) {
    set_error("romsad_build_greedy: no snapshot was kept");
    s = RTE_ERR_NUMERIC;
  }
  if (s != RTE_OK) {
    delete rom;
    return s;
  }
  *out = rom;
  return RTE_OK;
}
