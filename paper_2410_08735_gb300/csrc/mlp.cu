// Learned warm start for FGMRES-ROMSAD: an MLP maps the material parameters mu = (sigma_s, sigma_a)
// of an instance to reduced-basis coefficients c (the Galerkin coefficients of eq. greedy-rom, which
// the greedy ROM construction produces for every training parameter).  Since delta phi = T Sigma_s xi
// = phi - b~ for the first FGMRES correction (eqs. density-relation, correction-fgmres1), W c
// approximates phi - b~ and phi0 = b~ + W c_hat(mu) is the warm start.
//
// Network: features x = standardised (log sigma_s, sigma_a); h1 = gelu(W1 x + b1),
// h2 = gelu(W2 h1 + b2), y = W3 h2 + b3, exact GELU t Phi(t) (Hendrycks and Gimpel 2016, erf form).
// Loss 0.5 ||y - c||^2 / r averaged over the batch; Adam (Kingma and Ba 2015).  Master weights are
// FP32; with bf16 = 1 every product uses the weights rounded to BF16, accumulating in FP32.
// The layers are small (<= 128 wide), so the kernels are plain CUDA-core loops: one thread per
// output element, batch-parallel.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "romsad.h"

struct rte_mlp {
  int din = 0, H = 0, dout = 0;
  int nparam = 0;
  rte::DevBuf<float> w, g, m, v;      // flat parameters: W1 [H][din], b1 [H], W2 [H][H], b2, W3 [dout][H], b3
  std::vector<float> mean, stdv;      // feature standardisation [din]
  int adam_t = 0;
  int off_W1 = 0, off_b1 = 0, off_W2 = 0, off_b2 = 0, off_W3 = 0, off_b3 = 0;
};

namespace rte {

__device__ __forceinline__ float wq(float x, int bf16) { return bf16 ? __bfloat162float(__float2bfloat16(x)) : x; }

__device__ __forceinline__ float gelu_f(float t) { return 0.5f * t * (1.0f + erff(t * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float t) {
  return 0.5f * (1.0f + erff(t * 0.70710678118654752f)) + t * expf(-0.5f * t * t) * 0.3989422804014327f;
}

// x[n][din] = (log sigma_s, sigma_a) standardised
__global__ void k_features(const double* mu, int n, int R, const float* mean, const float* stdv, float* x) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * 2 * R) return;
  const int i = t / (2 * R), f = t % (2 * R);
  const double v = mu[(size_t)i * 2 * R + f];
  const double raw = f < R ? log(v) : v;
  x[t] = (float)((raw - mean[f]) / stdv[f]);
}

// out[n][o] = act(sum_i W[o][i] in[n][i] + b[o]); pre[n][o] keeps the pre-activation
__global__ void k_dense_fwd(const float* in, int n, int ni, const float* W, const float* b, int no, int act, int bf16,
                            float* pre, float* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * no) return;
  const int s = t / no, o = t % no;
  float acc = b[o];
  const float* x = in + (size_t)s * ni;
  const float* w = W + (size_t)o * ni;
  for (int i = 0; i < ni; ++i) acc += wq(w[i], bf16) * x[i];
  if (pre) pre[t] = acc;
  out[t] = act ? gelu_f(acc) : acc;
}

// loss and dY = (y - c) / (n r)
__global__ void k_mse(const float* y, const double* c, int n, int r, float* dy, double* lpart) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * r; t += gridDim.x * blockDim.x) {
    const double d = (double)y[t] - c[t];
    dy[t] = (float)(d / ((double)n * r));
    s += d * d;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) lpart[blockIdx.x] = sh[0];
}

// dW[o][i] = sum_s dz[s][o] in[s][i], db[o] = sum_s dz[s][o]  (one thread per weight)
__global__ void k_dense_bwd_w(const float* dz, const float* in, int n, int ni, int no, float* dW, float* db) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < no * ni) {
    const int o = t / ni, i = t % ni;
    float acc = 0.0f;
    for (int s = 0; s < n; ++s) acc += dz[(size_t)s * no + o] * in[(size_t)s * ni + i];
    dW[t] = acc;
  }
  if (t < no) {
    float acc = 0.0f;
    for (int s = 0; s < n; ++s) acc += dz[(size_t)s * no + t];
    db[t] = acc;
  }
}

// din[s][i] = (sum_o W[o][i] dz[s][o]) * gelu'(pre_in[s][i])
__global__ void k_dense_bwd_x(const float* dz, const float* W, int n, int ni, int no, const float* pre_in, int bf16,
                              float* dx) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * ni) return;
  const int s = t / ni, i = t % ni;
  float acc = 0.0f;
  for (int o = 0; o < no; ++o) acc += wq(W[(size_t)o * ni + i], bf16) * dz[(size_t)s * no + o];
  dx[t] = acc * gelu_grad_f(pre_in[t]);
}

__global__ void k_adam(float* w, const float* g, float* m, float* v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float gt = g[t];
  const float mt = b1 * m[t] + (1.0f - b1) * gt;
  const float vt = b2 * v[t] + (1.0f - b2) * gt * gt;
  m[t] = mt;
  v[t] = vt;
  w[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
}

struct MlpScratch {
  DevBuf<double> mu, c, lpart;
  DevBuf<float> x, a1, h1, a2, h2, y, dy, d2, d1;
  int alloc(const rte_mlp* M, int n) {
    RTE_TRY(mu.ensure((size_t)n * M->din));
    RTE_TRY(c.ensure((size_t)n * M->dout));
    RTE_TRY(lpart.ensure(64));
    RTE_TRY(x.ensure((size_t)n * M->din));
    RTE_TRY(a1.ensure((size_t)n * M->H));
    RTE_TRY(h1.ensure((size_t)n * M->H));
    RTE_TRY(a2.ensure((size_t)n * M->H));
    RTE_TRY(h2.ensure((size_t)n * M->H));
    RTE_TRY(y.ensure((size_t)n * M->dout));
    RTE_TRY(dy.ensure((size_t)n * M->dout));
    RTE_TRY(d2.ensure((size_t)n * M->H));
    RTE_TRY(d1.ensure((size_t)n * M->H));
    return RTE_OK;
  }
};

static int blocks_for(long long n) { return (int)std::max<long long>(1, (n + 255) / 256); }

// forward pass on device features x (already standardised); fills S.y
static int mlp_forward_dev(rte_mlp* M, MlpScratch& S, int n, int bf16, cudaStream_t st) {
  const float* w = M->w.p;
  k_dense_fwd<<<blocks_for((long long)n * M->H), 256, 0, st>>>(S.x.p, n, M->din, w + M->off_W1, w + M->off_b1, M->H, 1,
                                                                bf16, S.a1.p, S.h1.p);
  count_launch();
  k_dense_fwd<<<blocks_for((long long)n * M->H), 256, 0, st>>>(S.h1.p, n, M->H, w + M->off_W2, w + M->off_b2, M->H, 1,
                                                                bf16, S.a2.p, S.h2.p);
  count_launch();
  k_dense_fwd<<<blocks_for((long long)n * M->dout), 256, 0, st>>>(S.h2.p, n, M->H, w + M->off_W3, w + M->off_b3,
                                                                   M->dout, 0, bf16, nullptr, S.y.p);
  count_launch();
  RTE_CHECK_CUDA(cudaGetLastError());
  return RTE_OK;
}

// loss and gradient (into M->g) for labels S.c; returns the loss on the host
static int mlp_loss_grad_dev(rte_mlp* M, MlpScratch& S, int n, int bf16, double* loss, cudaStream_t st) {
  RTE_TRY(mlp_forward_dev(M, S, n, bf16, st));
  k_mse<<<64, 256, 0, st>>>(S.y.p, S.c.p, n, M->dout, S.dy.p, S.lpart.p);
  count_launch();
  float* g = M->g.p;
  const float* w = M->w.p;
  k_dense_bwd_w<<<blocks_for((long long)M->dout * M->H), 256, 0, st>>>(S.dy.p, S.h2.p, n, M->H, M->dout,
                                                                        g + M->off_W3, g + M->off_b3);
  count_launch();
  k_dense_bwd_x<<<blocks_for((long long)n * M->H), 256, 0, st>>>(S.dy.p, w + M->off_W3, n, M->H, M->dout, S.a2.p,
                                                                  bf16, S.d2.p);
  count_launch();
  k_dense_bwd_w<<<blocks_for((long long)M->H * M->H), 256, 0, st>>>(S.d2.p, S.h1.p, n, M->H, M->H, g + M->off_W2,
                                                                     g + M->off_b2);
  count_launch();
  k_dense_bwd_x<<<blocks_for((long long)n * M->H), 256, 0, st>>>(S.d2.p, w + M->off_W2, n, M->H, M->H, S.a1.p, bf16,
                                                                  S.d1.p);
  count_launch();
  k_dense_bwd_w<<<blocks_for((long long)M->H * M->din), 256, 0, st>>>(S.d1.p, S.x.p, n, M->din, M->H, g + M->off_W1,
                                                                       g + M->off_b1);
  count_launch();
  RTE_CHECK_CUDA(cudaGetLastError());
  if (loss) {
    std::vector<double> h(64);
    RTE_CHECK_CUDA(cudaMemcpyAsync(h.data(), S.lpart.p, 64 * 8, cudaMemcpyDeviceToHost, st));
    RTE_CHECK_CUDA(cudaStreamSynchronize(st));
    double s = 0.0;
    for (double v : h) s += v;
    *loss = 0.5 * s / ((double)n * M->dout);
  }
  return RTE_OK;
}

static int upload_features(rte_mlp* M, MlpScratch& S, int n, const double* mu_host, cudaStream_t st) {
  RTE_CHECK_CUDA(cudaMemcpyAsync(S.mu.p, mu_host, (size_t)n * M->din * 8, cudaMemcpyHostToDevice, st));
  DevBuf<float> mean, stdv;
  RTE_TRY(mean.alloc(M->din));
  RTE_TRY(stdv.alloc(M->din));
  RTE_CHECK_CUDA(cudaMemcpyAsync(mean.p, M->mean.data(), M->din * 4, cudaMemcpyHostToDevice, st));
  RTE_CHECK_CUDA(cudaMemcpyAsync(stdv.p, M->stdv.data(), M->din * 4, cudaMemcpyHostToDevice, st));
  k_features<<<blocks_for((long long)n * M->din), 256, 0, st>>>(S.mu.p, n, M->din / 2, mean.p, stdv.p, S.x.p);
  count_launch();
  RTE_CHECK_CUDA(cudaGetLastError());
  RTE_CHECK_CUDA(cudaStreamSynchronize(st));
  return RTE_OK;
}

// c_hat for instances whose parameters are on the device ([B][R] sigma_s, sigma_a): used by the
// learned warm start inside fgmres_solve.  out: [B][64] doubles.
__global__ void k_pad_out(const float* y, int n, int r, double* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * 64) return;
  const int s = t / 64, k = t % 64;
  out[t] = k < r ? (double)y[(size_t)s * r + k] : 0.0;
}

int mlp_predict_instances(rte_mlp* M, rte_problem* p, const int* d_list, const std::vector<int>& list, double* c_out,
                          cudaStream_t st) {
  // every listed instance: mu from the device parameter arrays (sigma_t - sigma_s = sigma_a)
  const int n = (int)list.size();
  const int R = p->R;
  if (M->din != 2 * R) {
    set_error("learned warm start: MLP input width must be 2R");
    return RTE_ERR_INVALID_ARG;
  }
  MlpScratch S;
  RTE_TRY(S.alloc(M, n));
  std::vector<double> mu((size_t)n * 2 * R);
  for (int i = 0; i < n; ++i)
    for (int q = 0; q < R; ++q) {
      mu[(size_t)i * 2 * R + q] = p->ss[(size_t)list[i] * R + q];
      mu[(size_t)i * 2 * R + R + q] = p->sa[(size_t)list[i] * R + q];
    }
  RTE_TRY(upload_features(M, S, n, mu.data(), st));
  RTE_TRY(mlp_forward_dev(M, S, n, 1, st));
  k_pad_out<<<blocks_for((long long)n * 64), 256, 0, st>>>(S.y.p, n, M->dout, c_out);
  count_launch();
  RTE_CHECK_CUDA(cudaGetLastError());
  RTE_CHECK_CUDA(cudaStreamSynchronize(st));
  return RTE_OK;
}

}  // namespace rte

using namespace rte;

extern "C" {

int rte_mlp_create(int n_in, int hidden, int n_out, unsigned long long seed, rte_mlp_t* out) {
  RTE_ARG(out && n_in >= 1 && n_in <= 256 && hidden >= 1 && hidden <= 512 && n_out >= 1 && n_out <= 64,
          "MLP sizes out of range");
  *out = nullptr;
  rte_mlp* M = new rte_mlp();
  M->din = n_in;
  M->H = hidden;
  M->dout = n_out;
  M->off_W1 = 0;
  M->off_b1 = M->off_W1 + hidden * n_in;
  M->off_W2 = M->off_b1 + hidden;
  M->off_b2 = M->off_W2 + hidden * hidden;
  M->off_W3 = M->off_b2 + hidden;
  M->off_b3 = M->off_W3 + n_out * hidden;
  M->nparam = M->off_b3 + n_out;
  M->mean.assign(n_in, 0.0f);
  M->stdv.assign(n_in, 1.0f);
  int s = M->w.alloc(M->nparam);
  if (s == RTE_OK) s = M->g.alloc(M->nparam);
  if (s == RTE_OK) s = M->m.alloc(M->nparam);
  if (s == RTE_OK) s = M->v.alloc(M->nparam);
  if (s != RTE_OK) {
    delete M;
    return s;
  }
  // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases, from SplitMix64(seed)
  std::vector<float> h(M->nparam, 0.0f);
  unsigned long long x = seed;
  auto next = [&]() {
    x += 0x9E3779B97F4A7C15ULL;
    unsigned long long z = x;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  auto fill = [&](int off, int count, int fan_in) {
    const double a = 1.0 / std::sqrt((double)fan_in);
    for (int i = 0; i < count; ++i) h[off + i] = (float)((2.0 * next() - 1.0) * a);
  };
  fill(M->off_W1, hidden * n_in, n_in);
  fill(M->off_W2, hidden * hidden, hidden);
  fill(M->off_W3, n_out * hidden, hidden);
  cudaMemcpy(M->w.p, h.data(), h.size() * 4, cudaMemcpyHostToDevice);
  cudaMemset(M->m.p, 0, M->nparam * 4);
  cudaMemset(M->v.p, 0, M->nparam * 4);
  *out = M;
  return RTE_OK;
}

int rte_mlp_num_params(rte_mlp_t M, int* n) {
  RTE_ARG(M && n, "null handle or pointer");
  *n = M->nparam;
  return RTE_OK;
}

int rte_mlp_set_params(rte_mlp_t M, const float* flat, const float* mean, const float* stdv) {
  RTE_ARG(M && flat, "null handle or pointer");
  RTE_CHECK_CUDA(cudaMemcpy(M->w.p, flat, (size_t)M->nparam * 4, cudaMemcpyHostToDevice));
  if (mean) M->mean.assign(mean, mean + M->din);
  if (stdv) M->stdv.assign(stdv, stdv + M->din);
  return RTE_OK;
}

int rte_mlp_get_params(rte_mlp_t M, float* flat, float* mean, float* stdv) {
  RTE_ARG(M && flat, "null handle or pointer");
  RTE_CHECK_CUDA(cudaMemcpy(flat, M->w.p, (size_t)M->nparam * 4, cudaMemcpyDeviceToHost));
  if (mean) std::memcpy(mean, M->mean.data(), M->din * 4);
  if (stdv) std::memcpy(stdv, M->stdv.data(), M->din * 4);
  return RTE_OK;
}

int rte_mlp_loss_grad(rte_mlp_t M, int n, const double* mu, const double* c, int bf16, double* loss, float* grad) {
  RTE_ARG(M && mu && c && loss && n >= 1, "null handle or pointer");
  MlpScratch S;
  RTE_TRY(S.alloc(M, n));
  RTE_TRY(upload_features(M, S, n, mu, 0));
  RTE_CHECK_CUDA(cudaMemcpy(S.c.p, c, (size_t)n * M->dout * 8, cudaMemcpyHostToDevice));
  RTE_TRY(mlp_loss_grad_dev(M, S, n, bf16, loss, 0));
  if (grad) RTE_CHECK_CUDA(cudaMemcpy(grad, M->g.p, (size_t)M->nparam * 4, cudaMemcpyDeviceToHost));
  return RTE_OK;
}

int rte_mlp_train(rte_mlp_t M, int n, const double* mu, const double* c, const rte_mlp_train_opts* o,
                  double* final_loss) {
  RTE_ARG(M && mu && c && o && n >= 1, "null handle or pointer");
  RTE_ARG(o->epochs >= 1 && o->batch >= 1 && o->lr > 0.0, "training options out of range");
  // feature standardisation from the training set
  const int R = M->din / 2;
  for (int f = 0; f < M->din; ++f) {
    double s = 0.0, s2 = 0.0;
    for (int i = 0; i < n; ++i) {
      const double v = mu[(size_t)i * M->din + f];
      const double raw = f < R ? std::log(v) : v;
      s += raw;
      s2 += raw * raw;
    }
    const double mean = s / n, var = std::max(0.0, s2 / n - mean * mean);
    M->mean[f] = (float)mean;
    M->stdv[f] = (float)(var > 1e-24 ? std::sqrt(var) : 1.0);
  }
  const int bs = std::min(o->batch, n);
  MlpScratch S;
  RTE_TRY(S.alloc(M, bs));
  MlpScratch full;
  RTE_TRY(full.alloc(M, n));
  RTE_TRY(upload_features(M, full, n, mu, 0));
  RTE_CHECK_CUDA(cudaMemcpy(full.c.p, c, (size_t)n * M->dout * 8, cudaMemcpyHostToDevice));
  RTE_CHECK_CUDA(cudaMemset(M->m.p, 0, M->nparam * 4));
  RTE_CHECK_CUDA(cudaMemset(M->v.p, 0, M->nparam * 4));
  M->adam_t = 0;
  for (int ep = 0; ep < o->epochs; ++ep) {
    for (int s0 = 0; s0 + bs <= n; s0 += bs) {  // fixed order minibatches
      RTE_CHECK_CUDA(cudaMemcpyAsync(S.x.p, full.x.p + (size_t)s0 * M->din, (size_t)bs * M->din * 4,
                                     cudaMemcpyDeviceToDevice, 0));
      RTE_CHECK_CUDA(cudaMemcpyAsync(S.c.p, full.c.p + (size_t)s0 * M->dout, (size_t)bs * M->dout * 8,
                                     cudaMemcpyDeviceToDevice, 0));
      RTE_TRY(mlp_loss_grad_dev(M, S, bs, o->bf16, nullptr, 0));
      ++M->adam_t;
      const float c1 = 1.0f - (float)std::pow(o->beta1, M->adam_t), c2 = 1.0f - (float)std::pow(o->beta2, M->adam_t);
      k_adam<<<blocks_for(M->nparam), 256>>>(M->w.p, M->g.p, M->m.p, M->v.p, M->nparam, (float)o->lr, (float)o->beta1,
                                             (float)o->beta2, (float)o->eps, c1, c2);
      count_launch();
    }
  }
  RTE_CHECK_CUDA(cudaGetLastError());
  if (final_loss) RTE_TRY(mlp_loss_grad_dev(M, full, n, o->bf16, final_loss, 0));
  return RTE_OK;
}

int rte_mlp_infer(rte_mlp_t M, int n, const double* mu, double* c_out) {
  RTE_ARG(M && mu && c_out && n >= 1, "null handle or pointer");
  MlpScratch S;
  RTE_TRY(S.alloc(M, n));
  RTE_TRY(upload_features(M, S, n, mu, 0));
  RTE_TRY(mlp_forward_dev(M, S, n, 1, 0));
  std::vector<float> y((size_t)n * M->dout);
  RTE_CHECK_CUDA(cudaMemcpy(y.data(), S.y.p, y.size() * 4, cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < y.size(); ++i) c_out[i] = y[i];
  return RTE_OK;
}

int rte_mlp_destroy(rte_mlp_t M) {
  if (M) {
    cudaDeviceSynchronize();
    delete M;
  }
  return RTE_OK;
}

int romsad_attach_mlp(romsad_t rom, rte_mlp_t M) {
  RTE_ARG(rom, "null ROM handle");
  if (M) RTE_ARG(M->dout == rom->r && M->din == 2 * rom->R, "MLP output width must equal the ROM rank, input 2R");
  rom->mlp = M;
  return RTE_OK;
}

}  // extern "C"
