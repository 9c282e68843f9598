// Flexible GMRES (paper Sec. 4.2, Alg. 1) for A~ phi = b~, batched over parameter instances.
//
// All instances of a problem advance in lock step: one launch per step covers every instance that
// is still active in the current cycle.  Per iteration j (0-based):
//   z_j = M_j^{-1} v_j              ROMSAD (romsad.cu) for j < window, then the post-window operator
//   w   = A~ z_j                    sweep (sweep.cu, per-task partial fluxes), reduced into v_{j+1}
//   MGS: h_ij = w . v_i, w -= h_ij v_i (i = 0..j), h_{j+1,j} = ||w||, v_{j+1} = w / h  (inverse
//        compact-WY form)
//   Givens: rotate column j of H, new rotation, |g_{j+1}| = residual estimate
// At the end of a cycle y = R^{-1} g and phi += Z y.  In FP64 solves the Krylov vectors, MGS and Givens
// are FP64; the inner solves of the mixed modes run them in FP32 (RTE_MODE_MIXED) or in FP64 around
// FP32 sweeps (RTE_MODE_MIXED_F64KRYLOV).
//
// Readings where Alg. 1 is silent: stop when |g_{j+1}| / ||b~|| <= rtol; happy breakdown when
// h_{j+1,j} <= 1e-14 ||w|| (before orthogonalisation); restart: phi0 <- phi, r0 = b~ - A~ phi0
// (one sweep); after convergence the true residual is recomputed once (optional) and the solve
// restarts from it if it exceeds 2 rtol.  The window counts iterations from the start of the solve.
//
// Mixed modes: FP64 iterative refinement.  r_k = b~ - A~ phi_k in FP64 (FP64 sweep), inner FGMRES on
// A~ d = r_k to inner_rtol (FP32 sweeps and ROM products; Krylov vectors, MGS and Givens in FP32 or
// FP64 by mode), phi += d; an instance whose refinement stalls is finished by FP64 FGMRES.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <unordered_map>

#include <cooperative_groups.h>

#include "romsad.h"

namespace rte {

enum CycleFlag { RUN = 0, STOP_CONV = 1, STOP_BREAK = 2, STOP_RESTART = 3, STOP_NUMERIC = 4 };

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum (deterministic: fixed tree), result broadcast to all threads.
__device__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < nw ? sh[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) sh[32] = t;
  }
  __syncthreads();
  return sh[32];
}

// Norms accumulate in FP64 whatever the vector type (one launch per restart, not per iteration).
template <typename TV>
__global__ void k_norm(const TV* x, const InstInfo* inst, const int* active, double* out) {
  __shared__ double sh[33];
  const int b = blockIdx.x;
  if (active && !active[b]) return;
  const InstInfo in = inst[b];
  double s = 0.0;
  for (int i = threadIdx.x; i < in.ndof; i += blockDim.x) {
    double v = (double)x[in.off + i];
    s += v * v;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[b] = sqrt(s);
}

__global__ void k_linf(const double* x, const InstInfo* inst, double* out) {
  __shared__ double sh[33];
  const int b = blockIdx.x;
  const InstInfo in = inst[b];
  double s = 0.0;
  for (int i = threadIdx.x; i < in.ndof; i += blockDim.x) s = fmax(s, fabs(x[in.off + i]));
  for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, sh[w]);
    out[b] = m;
  }
}

// dst = src * (1/scale_b) on active instances; grid (chunks, B)
template <typename TV>
__global__ void k_scale(TV* dst, const TV* src, const double* scale, const InstInfo* inst, const int* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const InstInfo in = inst[b];
  const TV s = (TV)(1.0 / scale[b]);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < in.ndof; i += gridDim.x * blockDim.x)
    dst[in.off + i] = src[in.off + i] * s;
}

// dst = src (with conversion) on active instances
template <typename TD, typename TS>
__global__ void k_copy_active(TD* dst, const TS* src, const InstInfo* inst, const int* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const InstInfo in = inst[b];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < in.ndof; i += gridDim.x * blockDim.x)
    dst[in.off + i] = (TD)src[in.off + i];
}

// ------------------------------------------------------------------------------------------------
// Modified Gram-Schmidt in inverse compact-WY form.  The MGS recurrence h_i = v_i.w^(i-1),
// w^(i) = w^(i-1) - h_i v_i gives h_i = v_i.w - sum_{k<i} (v_i.v_k) h_k, i.e. (I + L) h = V^T w with L
// the strictly lower part of the Gram matrix V^T V, and w^(j) = w - V h.  The same coefficients are
// therefore obtained from one pass of dot products (V^T w, plus the new Gram row v_j . V) and one
// update pass instead of j+1 dependent reductions (Swirydowicz, Langou, Ananthan, Yang, Thomas,
// Numer. Linear Algebra Appl. 2020).  The triangular system is solved with T = (I + L)^{-1}, kept per
// instance and grown by one row per iteration: with l the new Gram row, T's new row is -l^T T and
// h = T a.  Both products are spread over the threads of a block, so no step of the iteration is a
// j-long serial chain of dependent arithmetic.  Rounding differs from the sequential loop; the
// projector is the MGS projector.
//
// Fused iteration kernels.  One Arnoldi iteration of one or many instances is three launches: the
// ROMSAD preconditioner (k_precond_coop), the sweep (sweep.cu, per-task partial fluxes), and the
// Arnoldi step (k_arnoldi_coop: reduction of the partials into w = A~ z, MGS, Givens,
// normalisation).  The two fused kernels are cooperative launches: phases over vector chunks ("items",
// 256 dofs of one instance) and phases over instances are separated by grid-wide barriers, so the
// per-instance reductions need no extra launches.  Partial sums are always combined in a fixed order.
//
// Both kernels are templated on the vector type TV.  FP64 solves run them in double; the inner solves
// of the mixed-precision refinement run them in float (Krylov basis, MGS, Givens, ROM products), which
// on this GPU's 1:64 FP64:FP32 throughput ratio removes FP64 arithmetic from the iteration.
struct RomInstDev {
  const double* P;
  const double* W;
  const float* P32;
  const float* W32;
  const double* inv;   // (U^T A_mu U)^{-1}, r x r row-major
  const float* inv32;  // the same, rounded to FP32
  const double* WT;    // W transposed, [r][N]
  const float* WT32;
  int r, rmax, has, N;
};

template <typename TV>
struct RomSel;
template <>
struct RomSel<double> {
  __device__ static const double* P(const RomInstDev& R) { return R.P; }
  __device__ static const double* W(const RomInstDev& R) { return R.W; }
  __device__ static const double* inv(const RomInstDev& R) { return R.inv; }
  __device__ static const double* WT(const RomInstDev& R) { return R.WT; }
};
template <>
struct RomSel<float> {
  __device__ static const float* P(const RomInstDev& R) { return R.P32; }
  __device__ static const float* W(const RomInstDev& R) { return R.W32; }
  __device__ static const float* inv(const RomInstDev& R) { return R.inv32; }
  __device__ static const float* WT(const RomInstDev& R) { return R.WT32; }
};

// four consecutive values from a 16-byte aligned address
__device__ __forceinline__ void load4(const float* p, float& a, float& b, float& c, float& d) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = v.x; b = v.y; c = v.z; d = v.w;
}
__device__ __forceinline__ void load4(const double* p, double& a, double& b, double& c, double& d) {
  const double2 v0 = reinterpret_cast<const double2*>(p)[0];
  const double2 v1 = reinterpret_cast<const double2*>(p)[1];
  a = v0.x; b = v0.y; c = v1.x; d = v1.y;
}

template <typename TV>
__device__ __forceinline__ TV warp_sum_t(TV v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// z = M_ROM^{-1} v = v + W (U^T A_mu U)^{-1} P^T Sigma_s v for instances with a ROM, z = v otherwise.
// slot (null: none): instances with slot[b] = 1 take the reduced coefficients from slot_c [B][64]
// instead of the reduced solve (the learned correction in the ROMSAD slot).
// Sigma_s w at global dof gdof of this lane: sigma_s per dof, or with cross-section profiles the cell's 4x4
// block times the cell's four values, gathered from the four consecutive lanes that hold them (a cell's dofs are
// 4 c .. 4 c + 3 and the lanes map to consecutive dofs from a multiple of 4).  Every lane of the warp calls it.
template <typename TV>
__device__ __forceinline__ TV sigma_s_times(const TV* sig_dof, const TV* sblk, long long gdof, TV wi, bool ok) {
  if (sblk) {
    const int g = (threadIdx.x & 31) & ~3;
    const TV x0 = __shfl_sync(0xffffffffu, wi, g), x1 = __shfl_sync(0xffffffffu, wi, g + 1);
    const TV x2 = __shfl_sync(0xffffffffu, wi, g + 2), x3 = __shfl_sync(0xffffffffu, wi, g + 3);
    if (!ok) return TV(0);
    const TV* S = sblk + (gdof >> 2) * 16 + (gdof & 3) * 4;
    return S[0] * x0 + S[1] * x1 + S[2] * x2 + S[3] * x3;
  }
  return ok ? sig_dof[gdof] * wi : TV(0);
}

template <typename TV>
__global__ void __launch_bounds__(256) k_precond_coop(int B, const int2* items, int nitems, const InstInfo* inst,
                                                      const int* active, const RomInstDev* ri, const TV* sig_dof,
                                                      const TV* sblk,
                                                      const TV* v, TV* z, TV* rpart, TV* rc, int nchunk,
                                                      const int* slot, const TV* slot_c) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  __shared__ TV red[8][64];
  __shared__ TV ys[64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // phase 1: copy (instances without a ROM) or projection partials P^T Sigma_s v over the chunk
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int b = items[it].x, ch = items[it].y;
    if (!active[b]) continue;
    const InstInfo in = inst[b];
    const int i0 = ch * 256, i1 = min(in.ndof, i0 + 256);
    const RomInstDev R = ri[b];
    if (!R.has) {
      const int i = i0 + threadIdx.x;
      if (i < i1) z[in.off + i] = v[in.off + i];
      continue;
    }
    // warp w owns rows i0 + 32 w .. +31: one coalesced load of Sigma_s v for its rows, then the 32
    // P rows (lane = rank index), all loads independent so that they are in flight together
    // (row and column indices are clamped into the array and the surplus terms multiplied by zero, so
    // that every load is unconditional)
    const TV* Pm = RomSel<TV>::P(R);
    const int ib = i0 + warp * 32;
    const int nrow = min(32, i1 - ib);
    TV acc0 = 0, acc1 = 0;
    if (nrow > 0) {
      const TV vl = lane < nrow ? v[in.off + ib + lane] : TV(0);
      const TV svl = sigma_s_times(sig_dof, sblk, in.off + ib + lane, vl, lane < nrow);
      const TV m0 = lane < R.r ? TV(1) : TV(0);
      const TV m1 = lane + 32 < R.r ? TV(1) : TV(0);
      const int c0 = min(lane, R.rmax - 1), c1 = min(lane + 32, R.rmax - 1);
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        const TV sv = __shfl_sync(0xffffffffu, svl, k);
        const TV* row = Pm + (size_t)(ib + min(k, nrow - 1)) * R.rmax;
        acc0 += row[c0] * (sv * m0);
      }
      if (R.r > 32) {
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          const TV sv = __shfl_sync(0xffffffffu, svl, k);
          const TV* row = Pm + (size_t)(ib + min(k, nrow - 1)) * R.rmax;
          acc1 += row[c1] * (sv * m1);
        }
      }
    }
    red[warp][lane] = acc0;
    red[warp][lane + 32] = acc1;
    __syncthreads();
    if (threadIdx.x < 64) {
      TV s = 0;
      for (int w = 0; w < 8; ++w) s += red[w][threadIdx.x];
      rpart[((size_t)b * nchunk + ch) * 64 + threadIdx.x] = s;
    }
    __syncthreads();
  }
  grid.sync();
  // phase 2: c = (U^T A_mu U)^{-1} (sum of the partials) per instance; warp w sums chunks w, w+8, ...
  for (int b = blockIdx.x; b < B; b += gridDim.x) {
    if (!active[b] || !ri[b].has) continue;
    if (slot && slot[b]) {
      if (threadIdx.x < 64) rc[(size_t)b * 64 + threadIdx.x] = slot_c[(size_t)b * 64 + threadIdx.x];
      continue;
    }
    const RomInstDev R = ri[b];
    const int nch = (inst[b].ndof + 255) / 256;
    for (int q = lane; q < 64; q += 32) {
      TV s = 0;
      if (q < R.r) {
#pragma unroll 8
        for (int c = warp; c < nch; c += 8) s += rpart[((size_t)b * nchunk + c) * 64 + q];
      }
      red[warp][q] = s;
    }
    __syncthreads();
    if (threadIdx.x < 64) {
      TV s = 0;
      for (int w = 0; w < 8; ++w) s += red[w][threadIdx.x];
      ys[threadIdx.x] = threadIdx.x < R.r ? s : TV(0);
    }
    __syncthreads();
    if (threadIdx.x < R.r) {
      const TV* row = RomSel<TV>::inv(R) + (size_t)threadIdx.x * R.r;
      TV s = 0;
#pragma unroll
      for (int q = 0; q < 32; ++q) s += row[min(q, R.r - 1)] * ys[q];
      if (R.r > 32) {
#pragma unroll
        for (int q = 32; q < 64; ++q) s += row[min(q, R.r - 1)] * ys[q];
      }
      rc[(size_t)b * 64 + threadIdx.x] = s;
    }
    __syncthreads();
  }
  grid.sync();
  // phase 3: z = v + W c
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int b = items[it].x, ch = items[it].y;
    if (!active[b] || !ri[b].has) continue;
    const InstInfo in = inst[b];
    const RomInstDev R = ri[b];
    __syncthreads();
    if (threadIdx.x < 64) ys[threadIdx.x] = threadIdx.x < R.r ? rc[(size_t)b * 64 + threadIdx.x] : TV(0);
    __syncthreads();
    const int i = ch * 256 + threadIdx.x;
    if (i >= in.ndof) continue;
    const TV* wt = RomSel<TV>::WT(R) + i;   // W^T: consecutive dofs per rank index (coalesced)
    TV s = 0;
#pragma unroll
    for (int q = 0; q < 32; ++q) s += wt[(size_t)min(q, R.r - 1) * R.N] * ys[q];
    if (R.r > 32) {
#pragma unroll
      for (int q = 32; q < 64; ++q) s += wt[(size_t)min(q, R.r - 1) * R.N] * ys[q];
    }
    z[in.off + i] = v[in.off + i] + s;
  }
}

// Arguments of one fused Arnoldi step (k_arnoldi_coop).
template <typename TP, typename TV>
struct ArnArgs {
  int B, nitems, ntask, j, m, nchunk, ldT, rom_next;
  long long ntot;
  const int2* items;
  const InstInfo* inst;
  int* active;          // device mask; cleared here for instances that stop
  int* active0;         // snapshot of active taken in phase B, read in phase C
  const TP* partial;    // per-task partial fluxes of the sweep of z_j
  const TV* z;          // z_j
  TV* V;                // Krylov basis; v_{j+1} is written here
  TV* znext;            // z_{j+1} = M_{j+1}^{-1} v_{j+1} (null: not needed)
  TV* part;             // [B][2m+3][nchunk] chunk partials of the dot products
  TV* npart;            // [B][nchunk] chunk partials of ||w||^2
  TV* Tm;               // [B][m+1][ldT] T = (I + L)^{-1}
  TV* rpart;            // [B][nchunk][64] chunk partials of P^T Sigma_s w
  const RomInstDev* ri;
  const TV* sig_dof;
  const TV* sblk;       // cross-section profiles: Sigma_s blocks [cells][16] (null: sigma_s per dof)
  double* H;            // [B][m][m+1] column j: rotated Hessenberg column
  double* Hraw;         // unrotated copy (first-cycle record) or null
  double* w0;           // [B] ||w|| before orthogonalisation
  double* cs;
  double* sn;
  double* g;
  double* est;
  const double* bnorm;
  const double* rtol;
  int* iters_left;
  int* flag;
  int* kcols;
};

// One Arnoldi iteration for every active instance, three phases over vector chunks ("items": 256
// dofs of one instance) separated by two grid-wide barriers:
//   A  w = z_j - sum_t partial_t (= A~ z_j) into V[j+1]; chunk partials of v_k . w (k <= j),
//      v_k . v_j (k < j) and w . w.
//   B  every block of an instance sums the partials of that instance itself (the same fixed order in
//      every block, so all blocks hold identical values) and forms h = T a: h_i = (T a)_i for i < j
//      from the stored rows of T, h_j = a_j - sum_{i<j} l_i h_i.  Then w -= V h on its chunk, the
//      chunk partial of ||w||^2 and, when the next iteration applies the ROM, of P^T Sigma_s w.  The
//      block of chunk 0 stores column j of H and the new row of T (-l^T T).
//   C  every block sums the ||w||^2 partials (h_{j+1,j}) and the projection partials, normalises its
//      chunk of v_{j+1} and writes z_{j+1} = v_{j+1} + W (U^T A_mu U)^{-1} P^T Sigma_s v_{j+1} (or
//      v_{j+1}); the block of chunk 0 applies the Givens rotations and sets the stopping flags.
// The per-instance reductions are repeated by each block of the instance instead of being done once
// behind an extra barrier: on a latency-bound problem a barrier costs more than the repeated sums.
template <typename TP, typename TV>
__global__ void __launch_bounds__(256) k_arnoldi_coop(ArnArgs<TP, TV> A) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = A.j, m = A.m, nslot = 2 * m + 3;
  const long long ntot = A.ntot;
  __shared__ TV sl[260];          // chunk dot products (phase A) / instance sums (phase B)
  __shared__ TV hsv[132];
  __shared__ __align__(16) TV wsh[256];
  __shared__ __align__(16) TV vjsh[256];
  __shared__ TV red[8][128];
  __shared__ TV ys[64];
  __shared__ TV css[128], sns[128];
  __shared__ TV hsc;
  auto used = [&](int t) { return t <= j || (t >= m + 1 && t < m + 1 + j) || t == 2 * m + 2; };
  // ---------------------------------------------------------------- phase A
  for (int it = blockIdx.x; it < A.nitems; it += gridDim.x) {
    const int b = A.items[it].x, ch = A.items[it].y;
    if (!A.active[b]) continue;
    const InstInfo in = A.inst[b];
    const int i0 = ch * 256;
    const int i = i0 + threadIdx.x;
    const bool ok = i < in.ndof;
    TV wi = 0;
    if (ok) {
      const TP* pp = A.partial + (size_t)A.ntask * in.off;
      TP s = 0;
#pragma unroll 32
      for (int t = 0; t < A.ntask; ++t) s += pp[(size_t)t * in.ndof + i];
      wi = A.z[in.off + i] - (TV)s;
      A.V[(size_t)(j + 1) * ntot + in.off + i] = wi;
    }
    wsh[threadIdx.x] = wi;
    vjsh[threadIdx.x] = ok ? A.V[(size_t)j * ntot + in.off + i] : TV(0);
    __syncthreads();
    const int nvalid = min(256, in.ndof - i0);
    // warp q owns k = q, q + 8, ...: its reductions are independent of the other warps'.  Vectors are
    // taken four at a time with the index clamped to j (the surplus results are not stored), so every
    // batch issues all of its loads before the first use and there is no remainder loop.
    for (int k0 = warp; k0 <= j; k0 += 32) {
      // lane l reads dofs 4l..4l+3 and 128+4l..128+4l+3 of the chunk as two 4-wide loads (chunk
      // offsets and instance sizes are multiples of 4); surplus lanes re-read valid dofs and meet zeros
      TV x[4][8];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const TV* vk = A.V + (size_t)min(k0 + 8 * u, j) * ntot + in.off + i0;
#pragma unroll
        for (int h = 0; h < 2; ++h)
          load4(vk + min(4 * lane + 128 * h, nvalid - 4), x[u][4 * h], x[u][4 * h + 1], x[u][4 * h + 2],
                x[u][4 * h + 3]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int kk = k0 + 8 * u;
        TV a = 0, gg = 0;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int ii = 4 * lane + 128 * (e >> 2) + (e & 3);
          a += x[u][e] * wsh[ii];
          gg += x[u][e] * vjsh[ii];
        }
        a = warp_sum_t(a);
        gg = warp_sum_t(gg);
        if (lane == 0 && kk <= j) {
          sl[kk] = a;
          if (kk < j) sl[m + 1 + kk] = gg;
        }
      }
    }
    if (warp == 7) {
      TV ww = 0;
#pragma unroll
      for (int e = 0; e < 8; ++e) ww += wsh[lane + 32 * e] * wsh[lane + 32 * e];
      ww = warp_sum_t(ww);
      if (lane == 0) sl[2 * m + 2] = ww;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nslot; t += blockDim.x)
      if (used(t)) A.part[((size_t)b * nslot + t) * A.nchunk + ch] = sl[t];
    __syncthreads();
  }
  grid.sync();
  // ---------------------------------------------------------------- phase B
  for (int it = blockIdx.x; it < A.nitems; it += gridDim.x) {
    const int b = A.items[it].x, ch = A.items[it].y;
    if (!A.active[b]) {
      if (ch == 0 && threadIdx.x == 0) A.active0[b] = 0;
      continue;
    }
    const InstInfo in = A.inst[b];
    const int nch = (in.ndof + 255) / 256;
    // instance sums of the chunk partials over the 2j+2 used slots (a_0..a_j, l_0..l_{j-1}, w.w):
    // warp w takes used slots w, w+8, ..., its lanes the chunks (coalesced; this path has at most 64
    // chunks per instance, two per lane), then a fixed shuffle tree.  Eight slots per batch, indices
    // clamped, all loads issued before the first use.
    const int nused = 2 * j + 2;
    auto slot_of = [&](int u) { return u <= j ? u : (u < 2 * j + 1 ? m + 1 + (u - j - 1) : 2 * m + 2); };
    for (int u0 = warp; u0 < nused; u0 += 64) {
      TV x0[8], x1[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const TV* pp = A.part + ((size_t)b * nslot + slot_of(min(u0 + 8 * q, nused - 1))) * A.nchunk;
        x0[q] = pp[min(lane, nch - 1)];
        x1[q] = pp[min(lane + 32, nch - 1)];
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        TV v = (lane < nch ? x0[q] : TV(0)) + (lane + 32 < nch ? x1[q] : TV(0));
        v = warp_sum_t(v);
        const int u = u0 + 8 * q;
        if (lane == 0 && u < nused) sl[slot_of(u)] = v;
      }
    }
    __syncthreads();
    // One pass over the stored triangle of T (rows r < j, columns k < r), 8 rows per warp and pass,
    // lanes over k.  Row sums give h_r = a_r + sum_k T[r][k] a_k; the block of chunk 0 also forms the
    // column sums sum_r l_r T[r][k] for the new row of T.  Row and column indices are clamped into the
    // array and the surplus terms selected away, so that every load of a pass is unconditional.
    const TV* Tb = A.Tm + (size_t)b * (m + 1) * A.ldT;
    const bool trow = ch == 0;
    TV cacc[4] = {0, 0, 0, 0};
    const int jm = max(j - 1, 0);
    for (int r0 = 0; r0 < j; r0 += 64) {
      TV tv[8][4];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const TV* row = Tb + (size_t)min(r0 + warp + 8 * q, jm) * A.ldT;
#pragma unroll
        for (int p = 0; p < 4; ++p) tv[q][p] = row[min(lane + 32 * p, A.ldT - 1)];
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int r = r0 + warp + 8 * q;
        const TV lr = sl[min(m + 1 + r, 2 * m + 1)];
        TV s = 0;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const int k = lane + 32 * p;
          const bool tri = r < j && k < r;
          s += tri ? tv[q][p] * sl[k] : TV(0);
          cacc[p] += tri ? lr * tv[q][p] : TV(0);
        }
        s = warp_sum_t(s);
        if (lane == 0 && r < j) hsv[r] = sl[r] + s;
      }
    }
    if (trow) {
#pragma unroll
      for (int p = 0; p < 4; ++p) red[warp][lane + 32 * p] = cacc[p];
    }
    __syncthreads();
    if (warp == 0) {
      // h_j = a_j - sum_{i<j} l_i h_i
      TV s = 0;
      for (int r = lane; r < j; r += 32) s += sl[m + 1 + r] * hsv[r];
      s = warp_sum_t(s);
      if (lane == 0) hsv[j] = sl[j] - s;
    }
    if (trow) {
      // new row of T: T[j][k] = -(l_k + sum_{r=k+1}^{j-1} l_r T[r][k]), k < j
      for (int k = threadIdx.x; k < j; k += blockDim.x) {
        TV s = sl[m + 1 + k];
        for (int w = 0; w < 8; ++w) s += red[w][k];
        A.Tm[(size_t)b * (m + 1) * A.ldT + (size_t)j * A.ldT + k] = -s;
      }
    }
    __syncthreads();
    if (trow) {
      double* h = A.H + ((size_t)b * m + j) * (m + 1);
      double* hr = A.Hraw ? A.Hraw + ((size_t)b * m + j) * (m + 1) : nullptr;
      for (int t = threadIdx.x; t <= j; t += blockDim.x) {
        h[t] = (double)hsv[t];
        if (hr) hr[t] = (double)hsv[t];
      }
      if (threadIdx.x == 0) {
        A.w0[b] = sqrt((double)sl[2 * m + 2]);
        A.active0[b] = 1;
      }
    }
    // w -= V h on this chunk, ||w||^2 partial
    const int i = ch * 256 + threadIdx.x;
    const bool ok = i < in.ndof;
    TV wi = 0;
    if (ok) {
      wi = A.V[(size_t)(j + 1) * ntot + in.off + i];
      // batches of U vectors, index clamped to j and the surplus terms selected away: no remainder loop
      constexpr int U = sizeof(TV) == 4 ? 32 : 8;
      for (int k0 = 0; k0 <= j; k0 += U) {
        TV x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) x[u] = A.V[(size_t)min(k0 + u, j) * ntot + in.off + i];
#pragma unroll
        for (int u = 0; u < U; ++u) wi -= (k0 + u <= j) ? hsv[min(k0 + u, j)] * x[u] : TV(0);
      }
      A.V[(size_t)(j + 1) * ntot + in.off + i] = wi;
    }
    TV s2 = warp_sum_t(wi * wi);
    __syncthreads();   // red is free again
    if (lane == 0) red[warp][0] = s2;
    __syncthreads();
    if (threadIdx.x == 0) {
      TV tot = 0;
      for (int w = 0; w < 8; ++w) tot += red[w][0];
      A.npart[(size_t)b * A.nchunk + ch] = tot;
    }
    // projection partials P^T Sigma_s w for the next preconditioner apply
    const RomInstDev R = A.ri[b];
    if (A.rom_next && A.znext && R.has) {
      wsh[threadIdx.x] = sigma_s_times(A.sig_dof, A.sblk, in.off + i, wi, ok);
      __syncthreads();
      const TV* Pm = RomSel<TV>::P(R);
      const int ib = warp * 32;                       // chunk-local first row of this warp
      const int nrow = min(32, in.ndof - ch * 256 - ib);
      TV acc0 = 0, acc1 = 0;
      if (nrow > 0) {
        const TV svl = wsh[ib + lane];
        const TV m0 = lane < R.r ? TV(1) : TV(0);
        const TV m1 = lane + 32 < R.r ? TV(1) : TV(0);
        const int c0 = min(lane, R.rmax - 1), c1 = min(lane + 32, R.rmax - 1);
        const size_t rb = (size_t)(ch * 256 + ib);
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          const TV sv = __shfl_sync(0xffffffffu, svl, k);
          acc0 += Pm[(rb + min(k, nrow - 1)) * R.rmax + c0] * (sv * m0);
        }
        if (R.r > 32) {
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            const TV sv = __shfl_sync(0xffffffffu, svl, k);
            acc1 += Pm[(rb + min(k, nrow - 1)) * R.rmax + c1] * (sv * m1);
          }
        }
      }
      __syncthreads();
      red[warp][lane] = acc0;
      red[warp][lane + 32] = acc1;
      __syncthreads();
      if (threadIdx.x < 64) {
        TV s = 0;
        for (int w = 0; w < 8; ++w) s += red[w][threadIdx.x];
        A.rpart[((size_t)b * A.nchunk + ch) * 64 + threadIdx.x] = s;
      }
    }
    __syncthreads();
  }
  grid.sync();
  // ---------------------------------------------------------------- phase C
  for (int it = blockIdx.x; it < A.nitems; it += gridDim.x) {
    const int b = A.items[it].x, ch = A.items[it].y;
    if (!A.active0[b]) continue;
    const InstInfo in = A.inst[b];
    const int nch = (in.ndof + 255) / 256;
    const RomInstDev R = A.ri[b];
    const bool lift = A.znext && A.rom_next && R.has;
    const int i = ch * 256 + threadIdx.x;
    const bool ok = i < in.ndof;
    const size_t o = (size_t)(j + 1) * ntot + in.off + min(i, in.ndof - 1);
    // loads that do not depend on this phase's sums are issued first: w, the W row and the inverse row
    // of this thread, w0, and the Givens inputs of the block of chunk 0
    const TV wv = A.V[o];
    const double w0b = A.w0[b];
    TV wr[32], ir[32];
    if (lift) {
      // W^T [r][N]: for each rank index the threads of a chunk read consecutive dofs
      const TV* wt = RomSel<TV>::WT(R) + min(i, in.ndof - 1);
#pragma unroll
      for (int q = 0; q < 32; ++q) wr[q] = wt[(size_t)min(q, R.r - 1) * R.N];
      const TV* row = RomSel<TV>::inv(R) + (size_t)min((int)threadIdx.x, R.r - 1) * R.r;
#pragma unroll
      for (int q = 0; q < 32; ++q) ir[q] = row[min(q, R.r - 1)];
    }
    if (ch == 0) {
      const double* h = A.H + ((size_t)b * m + j) * (m + 1);
      for (int t = threadIdx.x; t <= j; t += blockDim.x) hsv[t] = (TV)h[t];
      for (int t = threadIdx.x; t < j; t += blockDim.x) {
        css[t] = (TV)A.cs[(size_t)b * m + t];
        sns[t] = (TV)A.sn[(size_t)b * m + t];
      }
    }
    if (warp == 0) {
      TV acc = 0;
      for (int c = lane; c < nch; c += 32) acc += A.npart[(size_t)b * A.nchunk + c];
      acc = warp_sum_t(acc);
      if (lane == 0) hsc = sqrt(acc);
    }
    if (lift) {
      // warp w sums the projection partials of chunks w, w+8, ...
      for (int q = lane; q < 64; q += 32) {
        TV s = 0;
        if (q < R.r) {
#pragma unroll 8
          for (int c = warp; c < nch; c += 8) s += A.rpart[((size_t)b * A.nchunk + c) * 64 + q];
        }
        red[warp][q] = s;
      }
    }
    __syncthreads();
    const TV hn = hsc;
    const bool bk = !((double)hn > 1e-14 * w0b);
    const TV inv_h = bk ? TV(0) : TV(1) / hn;
    if (lift) {
      // c = (U^T A_mu U)^{-1} P^T Sigma_s w / h_{j+1,j}
      if (threadIdx.x < 64) {
        TV s = 0;
        for (int w = 0; w < 8; ++w) s += red[w][threadIdx.x];
        wsh[threadIdx.x] = threadIdx.x < R.r ? s * inv_h : TV(0);
      }
      __syncthreads();
      if (threadIdx.x < R.r) {
        TV s = 0;
#pragma unroll
        for (int q = 0; q < 32; ++q) s += ir[q] * wsh[q];
        if (R.r > 32) {
          const TV* row = RomSel<TV>::inv(R) + (size_t)threadIdx.x * R.r;
          for (int q = 32; q < R.r; ++q) s += row[q] * wsh[q];
        }
        ys[threadIdx.x] = s;
      } else if (threadIdx.x < 64) {
        ys[threadIdx.x] = TV(0);
      }
      __syncthreads();
    }
    // v_{j+1} = w / h_{j+1,j} and z_{j+1} on this chunk
    if (!bk && ok) {
      const TV v = wv * inv_h;
      A.V[o] = v;
      if (A.znext) {
        TV zv = v;
        if (lift) {
          TV s = 0;
#pragma unroll
          for (int q = 0; q < 32; ++q) s += wr[q] * ys[q];
          if (R.r > 32) {
            const TV* wt = RomSel<TV>::WT(R) + i;
            for (int q = 32; q < R.r; ++q) s += wt[(size_t)q * R.N] * ys[q];
          }
          zv += s;
        }
        A.znext[in.off + i] = zv;
      }
    }
    if (ch == 0) {
      // Givens rotations of column j: one thread, the running entry kept in a register; the rotated
      // entries are then stored by all threads (the FP64 conversions are slow one at a time)
      double* h = A.H + ((size_t)b * m + j) * (m + 1);
      if (threadIdx.x == 0) {
        TV cur = hsv[0];
#pragma unroll 4
        for (int t = 0; t < j; ++t) {
          const TV nx = hsv[t + 1], c = css[t], s = sns[t];
          hsv[t] = c * cur + s * nx;
          cur = c * nx - s * cur;
        }
        hsv[j] = cur;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < j; t += blockDim.x) h[t] = (double)hsv[t];
      if (threadIdx.x == 0) {
        // h_{j+1,j}, the new rotation, the residual estimate and the stopping flags
        double* gg = A.g + (size_t)b * (m + 1);
        if (A.Hraw) A.Hraw[((size_t)b * m + j) * (m + 1) + j + 1] = (double)hn;
        const TV cur = hsv[j];
        const TV den = hypot(cur, hn);
        TV cj = 1, sj = 0;
        if (den > TV(0)) {
          cj = cur / den;
          sj = hn / den;
        }
        A.cs[(size_t)b * m + j] = (double)cj;
        A.sn[(size_t)b * m + j] = (double)sj;
        h[j] = (double)den;
        h[j + 1] = 0.0;
        const TV gj = (TV)gg[j];
        gg[j + 1] = (double)(-sj * gj);
        gg[j] = (double)(cj * gj);
        const double e = fabs((double)(sj * gj));
        A.est[b] = e;
        A.kcols[b] = j + 1;
        int f = RUN;
        if (!isfinite(e) || !isfinite((double)den)) f = STOP_NUMERIC;
        else if (e <= A.rtol[0] * A.bnorm[b]) f = STOP_CONV;
        else if (bk) f = STOP_BREAK;
        else if (j + 1 == m || A.iters_left[b] <= 1) f = STOP_RESTART;
        A.flag[b] = f;
        A.iters_left[b] -= 1;
        if (f != RUN) A.active[b] = 0;
      }
    }
    __syncthreads();
  }
}

// Arnoldi step for large batches: the per-instance work (sums of the chunk partials, the T update and
// h = T a; norm, Givens and flags) runs once per instance, in phases of its own between grid-wide
// barriers (five phases, four barriers), and the preconditioner is a separate launch.  Compared with
// k_arnoldi_coop this adds barriers but does not repeat any reduction, which is the better trade
// once the chunks of the batch fill the GPU several times over.
template <typename TP, typename TV>
__global__ void __launch_bounds__(256) k_arnoldi_wide(
    int B, const int2* items, int nitems, const InstInfo* inst, int* active, const TP* partial, int ntask,
    const TV* z, TV* V, long long ntot, int j, int m, int nchunk, TV* part, TV* npart, TV* Tm, int ldT,
    double* H, double* Hraw, double* w0, double* cs, double* sn, double* g, int* brk, const double* bnorm,
    const double* rtol_p, int* iters_left, double* est, int* flag, int* kcols, double* hnorm, int* active0) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nslot = 2 * m + 3;
  __shared__ TV red[260];
  __shared__ TV as[130], ls[130], css[128], sns[128], hsv[130];
  // P0: w = z - sum_t partial_t (the A~ z of this iteration) into V[j+1], then the chunk's partial dots
  //     a_k = v_k . w (k <= j), g_k = v_k . v_j (k < j), w . w.  w and v_j are staged in shared memory
  //     and warp q owns k = q, q + 8, ...: its reductions are independent of the other warps'.
  __shared__ TV wsh[256], vjsh[256];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int b = items[it].x, ch = items[it].y;
    if (!active[b]) continue;
    const InstInfo in = inst[b];
    const int i0 = ch * 256;
    const int i = i0 + threadIdx.x;
    const bool ok = i < in.ndof;
    TV wi = 0;
    if (ok) {
      const TP* pp = partial + (size_t)ntask * in.off;
      TP s = 0;
#pragma unroll 8
      for (int t = 0; t < ntask; ++t) s += pp[(size_t)t * in.ndof + i];
      wi = z[in.off + i] - (TV)s;
      V[(size_t)(j + 1) * ntot + in.off + i] = wi;
    }
    wsh[threadIdx.x] = wi;
    vjsh[threadIdx.x] = ok ? V[(size_t)j * ntot + in.off + i] : TV(0);
    __syncthreads();
    const int nvalid = min(256, in.ndof - i0);
#pragma unroll 4
    for (int kk = warp; kk <= j; kk += 8) {
      const TV* vk = V + (size_t)kk * ntot + in.off + i0;
      TV a = 0, gg = 0;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int ii = lane + 32 * e;
        const TV x = vk[min(ii, nvalid - 1)];   // surplus lanes meet zeros in wsh / vjsh
        a += x * wsh[ii];
        gg += x * vjsh[ii];
      }
      a = warp_sum_t(a);
      gg = warp_sum_t(gg);
      if (lane == 0) {
        red[kk] = a;
        if (kk < j) red[m + 1 + kk] = gg;
      }
    }
    if (warp == 7) {
      TV ww = 0;
#pragma unroll
      for (int e = 0; e < 8; ++e) ww += wsh[lane + 32 * e] * wsh[lane + 32 * e];
      ww = warp_sum_t(ww);
      if (lane == 0) red[2 * m + 2] = ww;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nslot; t += blockDim.x) {
      const bool used = t <= j || (t >= m + 1 && t < m + 1 + j) || t == 2 * m + 2;
      if (used) part[((size_t)b * nslot + t) * nchunk + ch] = red[t];
    }
    __syncthreads();
  }
  grid.sync();
  // P1: per instance: sum the chunk partials, grow T = (I + L)^{-1} by the new row, h = T a
  for (int b = blockIdx.x; b < B; b += gridDim.x) {
    if (!active[b]) continue;
    const int nch = (inst[b].ndof + 255) / 256;
    for (int t = threadIdx.x; t < nslot; t += blockDim.x) {
      const bool used = t <= j || (t >= m + 1 && t < m + 1 + j) || t == 2 * m + 2;
      if (!used) continue;
      const TV* pp = part + ((size_t)b * nslot + t) * nchunk;
      TV acc = 0;
#pragma unroll 16
      for (int c = 0; c < nch; ++c) acc += pp[c];
      if (t <= j) as[t] = acc;
      else if (t < m + 1 + j) ls[t - m - 1] = acc;
      else w0[b] = sqrt((double)acc);
    }
    __syncthreads();
    TV* Tb = Tm + (size_t)b * (m + 1) * ldT;
    // row j of T: T[j][k] = -(l_k + sum_{i=k+1}^{j-1} l_i T[i][k]), k < j (T[i][i] = 1 implicit)
    for (int k = threadIdx.x; k < j; k += blockDim.x) {
      TV s = ls[k];
#pragma unroll 8
      for (int i = k + 1; i < j; ++i) s += ls[i] * Tb[(size_t)i * ldT + k];
      Tb[(size_t)j * ldT + k] = -s;
    }
    __syncthreads();
    double* h = H + ((size_t)b * m + j) * (m + 1);
    double* hr = Hraw ? Hraw + ((size_t)b * m + j) * (m + 1) : nullptr;
    for (int t = threadIdx.x; t <= j; t += blockDim.x) {
      const TV* row = Tb + (size_t)t * ldT;
      TV s = as[t];
#pragma unroll 8
      for (int k = 0; k < t; ++k) s += row[k] * as[k];
      h[t] = (double)s;
      if (hr) hr[t] = (double)s;
    }
    __syncthreads();
  }
  grid.sync();
  // P2: w -= sum_k h_k v_k over the chunk, partial ||w||^2
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int b = items[it].x, ch = items[it].y;
    if (!active[b]) continue;
    const InstInfo in = inst[b];
    const double* h = H + ((size_t)b * m + j) * (m + 1);
    for (int t = threadIdx.x; t <= j; t += blockDim.x) hsv[t] = (TV)h[t];
    __syncthreads();
    const int i = ch * 256 + threadIdx.x;
    TV s2 = 0;
    if (i < in.ndof) {
      TV wi = V[(size_t)(j + 1) * ntot + in.off + i];
#pragma unroll 16
      for (int kk = 0; kk <= j; ++kk) wi -= hsv[kk] * V[(size_t)kk * ntot + in.off + i];
      V[(size_t)(j + 1) * ntot + in.off + i] = wi;
      s2 = wi * wi;
    }
    s2 = warp_sum_t(s2);
    if (lane == 0) red[warp] = s2;
    __syncthreads();
    if (threadIdx.x == 0) {
      TV tot = 0;
      for (int w = 0; w < 8; ++w) tot += red[w];
      npart[(size_t)b * nchunk + ch] = tot;
    }
    __syncthreads();
  }
  grid.sync();
  // P3: per instance: h_{j+1,j} = ||w||, breakdown test, Givens rotation, stopping flags
  for (int b = blockIdx.x; b < B; b += gridDim.x) {
    if (!active[b]) {
      if (threadIdx.x == 0) active0[b] = 0;
      continue;
    }
    double* h = H + ((size_t)b * m + j) * (m + 1);
    double* c = cs + (size_t)b * m;
    double* s = sn + (size_t)b * m;
    double* gg = g + (size_t)b * (m + 1);
    for (int i = threadIdx.x; i <= j; i += blockDim.x) hsv[i] = (TV)h[i];
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
      css[i] = (TV)c[i];
      sns[i] = (TV)s[i];
    }
    if (warp == 0) {
      const int nch = (inst[b].ndof + 255) / 256;
      TV acc = 0;
      for (int cc = lane; cc < nch; cc += 32) acc += npart[(size_t)b * nchunk + cc];
      acc = warp_sum_t(acc);
      if (lane == 0) red[0] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const TV hn = sqrt(red[0]);
      hsv[j + 1] = hn;
      if (Hraw) Hraw[((size_t)b * m + j) * (m + 1) + j + 1] = (double)hn;
      hnorm[b] = (double)hn;
      const int bk = ((double)hn > 1e-14 * w0[b]) ? 0 : 1;
      brk[b] = bk;
      active0[b] = 1;
      for (int i = 0; i < j; ++i) {
        const TV t = css[i] * hsv[i] + sns[i] * hsv[i + 1];
        hsv[i + 1] = -sns[i] * hsv[i] + css[i] * hsv[i + 1];
        hsv[i] = t;
      }
      const TV den = hypot(hsv[j], hsv[j + 1]);
      TV cj = 1, sj = 0;
      if (den > TV(0)) {
        cj = hsv[j] / den;
        sj = hsv[j + 1] / den;
      }
      for (int i = 0; i < j; ++i) h[i] = (double)hsv[i];
      c[j] = (double)cj;
      s[j] = (double)sj;
      h[j] = (double)den;
      h[j + 1] = 0.0;
      const TV gj = (TV)gg[j];
      gg[j + 1] = (double)(-sj * gj);
      gg[j] = (double)(cj * gj);
      const double e = fabs((double)(sj * gj));
      est[b] = e;
      kcols[b] = j + 1;
      int f = RUN;
      if (!isfinite(e) || !isfinite((double)den)) f = STOP_NUMERIC;
      else if (e <= rtol_p[0] * bnorm[b]) f = STOP_CONV;
      else if (bk) f = STOP_BREAK;
      else if (j + 1 == m || iters_left[b] <= 1) f = STOP_RESTART;
      flag[b] = f;
      iters_left[b] -= 1;
      if (f != RUN) active[b] = 0;
    }
    __syncthreads();
  }
  grid.sync();
  // P4: v_{j+1} = w / h_{j+1,j}
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int b = items[it].x, ch = items[it].y;
    if (!active0[b] || brk[b]) continue;
    const InstInfo in = inst[b];
    const int i = ch * 256 + threadIdx.x;
    if (i < in.ndof) V[(size_t)(j + 1) * ntot + in.off + i] *= (TV)(1.0 / hnorm[b]);
  }
}


// y = R^{-1} g (R: rotated H, upper triangular k x k), one block per instance with k > 0:
// column-oriented back substitution, column i of R read by all threads (coalesced).  Arithmetic in TV.
template <typename TV>
__global__ void k_backsolve(const double* H, const double* g, int m, int B, const int* kcols, double* y) {
  const int b = blockIdx.x;
  const int k = kcols[b];
  if (k <= 0) return;
  __shared__ TV rhs[129];
  __shared__ TV yi;
  const double* Hb = H + (size_t)b * m * (m + 1);
  for (int i = threadIdx.x; i < k; i += blockDim.x) rhs[i] = (TV)g[(size_t)b * (m + 1) + i];
  __syncthreads();
  for (int i = k - 1; i >= 0; --i) {
    const double* col = Hb + (size_t)i * (m + 1);
    if (threadIdx.x == 0) {
      const TV d = (TV)col[i];
      yi = d != TV(0) ? rhs[i] / d : TV(0);
      y[(size_t)b * m + i] = (double)yi;
    }
    __syncthreads();
    const TV v = yi;
    for (int t = threadIdx.x; t < i; t += blockDim.x) rhs[t] -= (TV)col[t] * v;
    __syncthreads();
  }
}

// phi += sum_c y_c Z_c for instances with k > 0; grid (chunks, B)
template <typename TV>
__global__ void k_update(TV* phi, const TV* Z, long long ntot, int m, const InstInfo* inst, const int* kcols,
                         const double* y) {
  const int b = blockIdx.y;
  const int k = kcols[b];
  if (k <= 0) return;
  const InstInfo in = inst[b];
  __shared__ TV ys[128];
  for (int q = threadIdx.x; q < k; q += blockDim.x) ys[q] = (TV)y[(size_t)b * m + q];
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < in.ndof; i += gridDim.x * blockDim.x) {
    TV s = phi[in.off + i];
    for (int q = 0; q < k; ++q) s += ys[q] * Z[(size_t)q * ntot + in.off + i];
    phi[in.off + i] = s;
  }
}

// phi += d (FP64 phi), all instances in mask
template <typename TS>
__global__ void k_axpy_active(double* phi, const TS* d, const InstInfo* inst, const int* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const InstInfo in = inst[b];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < in.ndof; i += gridDim.x * blockDim.x)
    phi[in.off + i] += (double)d[in.off + i];
}

template <typename TV>
__global__ void k_zero_active(TV* x, const InstInfo* inst, const int* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const InstInfo in = inst[b];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < in.ndof; i += gridDim.x * blockDim.x) x[in.off + i] = TV(0);
}

// W^T [r][N] (FP64 and FP32) from W [N][rmax]
__global__ void k_w_transpose(const double* W, int N, int rmax, int r, double* WT, float* WT32) {
  const long long n = (long long)N * r;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(e / N), i = (int)(e % N);
    const double w = W[(size_t)i * rmax + q];
    WT[e] = w;
    WT32[e] = (float)w;
  }
}

// FP32 copy of the ROM inverse operators
__global__ void k_inv_to_f32(const double* a, float* b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// ----------------------------------------------------------------- host driver
struct Ws {
  int B = 0, m = 0;
  long long ntot = 0;
  bool withZ = false;
  DevBuf<double> V, Z, H, Hraw, cs, sn, g, y, bt, r, ro, d, phi_in;
  DevBuf<float> V32, Z32, r32, rin32, d32;     // FP32 Krylov basis of the mixed-precision inner solves
  // MGS scratch, typed double or float by the solve's vector type: T = (I + L)^{-1} [B][m+1][m+1],
  // chunk partials of the dot products [B][2m+3][nchunk] and of ||w||^2 [B][nchunk]
  DevBuf<double> Lt, part, npart, w0, hnorm;
  DevBuf<int> active0;
  int nchunk = 0;
  bool cwy_attr = false;
  // CUDA graphs of single iterations, keyed by (j, ROM on/off, precision, recording); they capture
  // device pointers, so they are dropped whenever a buffer they use is reallocated
  DevBuf<double> d_rtol;
  DevBuf<int> norom;            // [B] 1 for instances without a ROM
  double* h_rtol = nullptr;     // pinned
  cudaStream_t cap = nullptr;   // capture stream
  struct Graph {
    cudaGraphExec_t exec;
    int launches;
  };
  std::unordered_map<int, Graph> graphs;
  std::vector<RomPlan> plans;   // persistent across solves (same ROM groups -> same buffers)
  // fused iteration kernels: vector chunks (instance, 256-dof chunk), per-instance ROM data, and the
  // co-resident grid sizes of the cooperative launches
  DevBuf<int2> items;
  int nitems = 0;
  DevBuf<RomInstDev> rominst;
  DevBuf<double> rpart, rc;
  int grid_pre = 0, grid_post64 = 0, grid_post32 = 0, grid_wide64 = 0, grid_wide32 = 0;
  // latency-bound problems (all chunks resident at once, few chunks per instance) take the fused
  // two-barrier Arnoldi step; larger batches the multi-phase one (k_arnoldi_wide)
  bool fused = true;
  std::vector<romsad_t> plan_rom;
  std::vector<std::vector<int>> plan_ids;
  void drop_graphs() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second.exec);
    graphs.clear();
  }
  DevBuf<double> bnorm, beta, est, nrm;
  DevBuf<int> active, brk, flag, kcols, iters_left, list;
  DevBuf<double> rom_y, rom_c;
  // learned ROMSAD slot: per-instance flag and coefficients c_hat / beta (FP64 and FP32)
  DevBuf<int> slot;
  DevBuf<double> slot_c;
  DevBuf<float> slot_c32;
  int* hflag = nullptr;   // pinned host mirrors of flag and kcols
  int* hk = nullptr;
  ~Ws() {
    drop_graphs();
    if (cap) cudaStreamDestroy(cap);
    if (hflag) cudaFreeHost(hflag);
    if (hk) cudaFreeHost(hk);
    if (h_rtol) cudaFreeHost(h_rtol);
  }
  int alloc(rte_problem* p, int m_, bool withZ_) {
    if (B == p->B && m == m_ && ntot == p->ntot && (withZ == withZ_ || !withZ_)) return RTE_OK;
    drop_graphs();
    B = p->B;
    m = m_;
    ntot = p->ntot;
    withZ = withZ_ || withZ;
    RTE_TRY(V.alloc((size_t)(m + 1) * ntot));
    if (withZ) RTE_TRY(Z.alloc((size_t)m * ntot));
    RTE_TRY(V32.alloc((size_t)(m + 1) * ntot));
    if (withZ) RTE_TRY(Z32.alloc((size_t)m * ntot));
    RTE_TRY(r32.alloc(ntot));
    RTE_TRY(rin32.alloc(ntot));
    RTE_TRY(d32.alloc(ntot));
    RTE_TRY(H.alloc((size_t)B * m * (m + 1)));
    RTE_TRY(Hraw.alloc((size_t)B * m * (m + 1)));
    {
      int maxn = 0;
      for (int b = 0; b < p->B; ++b) maxn = std::max(maxn, (int)(p->off[b + 1] - p->off[b]));
      nchunk = (maxn + 255) / 256;
    }
    RTE_TRY(Lt.alloc((size_t)B * (m + 1) * (m + 1)));
    {
      std::vector<int2> it;
      for (int b = 0; b < p->B; ++b) {
        const int nb = (int)((p->off[b + 1] - p->off[b] + 255) / 256);
        for (int c = 0; c < nb; ++c) it.push_back(make_int2(b, c));
      }
      nitems = (int)it.size();
      RTE_TRY(items.alloc(it.size()));
      RTE_CHECK_CUDA(cudaMemcpy(items.p, it.data(), it.size() * sizeof(int2), cudaMemcpyHostToDevice));
      RTE_TRY(rominst.alloc(B));
      RTE_TRY(rpart.alloc((size_t)B * nchunk * 64));
      RTE_TRY(rc.alloc((size_t)B * 64));
      int dev = 0, nsm = 0, occ = 0;
      RTE_CHECK_CUDA(cudaGetDevice(&dev));
      RTE_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
      const int want = std::max(nitems, B);
      int o1 = 0, o2 = 0;
      RTE_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k_precond_coop<double>, 256, 0));
      RTE_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, k_precond_coop<float>, 256, 0));
      occ = std::min(o1, o2);
      grid_pre = std::min(want, std::max(1, occ) * nsm);
      // the FP64-vector grids serve both FP64 and FP32 sweeps (partials), so they take the smaller
      // co-resident count of the two instantiations
      RTE_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k_arnoldi_coop<double, double>, 256, 0));
      RTE_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, k_arnoldi_coop<float, double>, 256, 0));
      occ = std::min(o1, o2);
      grid_post64 = std::min(want, std::max(1, occ) * nsm);
      RTE_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_arnoldi_coop<float, float>, 256, 0));
      grid_post32 = std::min(want, std::max(1, occ) * nsm);
      fused = nitems <= std::min(grid_post32, grid_post64) && nchunk <= 64;
      RTE_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k_arnoldi_wide<double, double>, 256, 0));
      RTE_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, k_arnoldi_wide<float, double>, 256, 0));
      occ = std::min(o1, o2);
      grid_wide64 = std::min(want, std::max(1, occ) * nsm);
      RTE_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_arnoldi_wide<float, float>, 256, 0));
      grid_wide32 = std::min(want, std::max(1, occ) * nsm);
    }
    RTE_TRY(part.alloc((size_t)B * nchunk * (2 * m + 3)));
    RTE_TRY(npart.alloc((size_t)B * nchunk));
    RTE_TRY(w0.alloc(B));
    RTE_TRY(hnorm.alloc(B));
    RTE_TRY(active0.alloc(B));
    RTE_TRY(cs.alloc((size_t)B * m));
    RTE_TRY(sn.alloc((size_t)B * m));
    RTE_TRY(g.alloc((size_t)B * (m + 1)));
    RTE_TRY(y.alloc((size_t)B * m));
    RTE_TRY(bt.alloc(ntot));
    RTE_TRY(r.alloc(ntot));
    RTE_TRY(ro.alloc(ntot));
    RTE_TRY(d.alloc(ntot));
    RTE_TRY(bnorm.alloc(B));
    RTE_TRY(beta.alloc(B));
    RTE_TRY(est.alloc(B));
    RTE_TRY(nrm.alloc(B));
    RTE_TRY(active.alloc(B));
    RTE_TRY(brk.alloc(B));
    RTE_TRY(flag.alloc(B));
    RTE_TRY(kcols.alloc(B));
    RTE_TRY(iters_left.alloc(B));
    RTE_TRY(list.alloc(B));
    RTE_TRY(rom_y.alloc((size_t)B * 64));
    RTE_TRY(rom_c.alloc((size_t)B * 64));
    RTE_TRY(slot.alloc(B));
    RTE_TRY(slot_c.alloc((size_t)B * 64));
    RTE_TRY(slot_c32.alloc((size_t)B * 64));
    if (hflag) cudaFreeHost(hflag);
    if (hk) cudaFreeHost(hk);
    RTE_CHECK_CUDA(cudaMallocHost(&hflag, B * sizeof(int)));
    RTE_CHECK_CUDA(cudaMallocHost(&hk, B * sizeof(int)));
    RTE_TRY(d_rtol.alloc(1));
    RTE_TRY(norom.alloc(B));
    if (!h_rtol) RTE_CHECK_CUDA(cudaMallocHost(&h_rtol, sizeof(double)));
    if (!cap) RTE_CHECK_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    return RTE_OK;
  }
};

struct SolveCtx {
  rte_problem* p;
  const romsad_t* roms;  // [B] or null
  int m, window, post;
  cudaStream_t st;
  Ws* ws;
  FirstCycle* rec = nullptr;          // records the first cycle of instance 0 (greedy high-fidelity solve)
  std::vector<RomPlan>* plans = nullptr;  // one per ROM group (factored once per solve)
  std::vector<int> no_rom_mask;       // [B] 1 for instances without a ROM
  bool slot_pending = false;          // the next first-cycle preconditioner apply uses the learned slot
  bool any_rom = false;               // some instance has a ROM
  bool any_norom = false;             // some instance has none
  bool dsa = false;                   // DSA after the window (and throughout for instances without a ROM)
  bool rom_tc = false;                // FP32 runs: ROMSAD products on the tensor cores (romsad_tc.cu)
};


static dim3 vec_grid(rte_problem* p) {
  int maxn = 0;
  for (int b = 0; b < p->B; ++b) maxn = std::max(maxn, (int)(p->off[b + 1] - p->off[b]));
  return dim3((maxn + 255) / 256, p->B);
}

// Per-instance outcome of one inner (or FP64) FGMRES run.
struct RunStats {
  std::vector<int> iterations, sweeps, restarts, status;
  std::vector<double> est;
};

// Restarted FGMRES on A~ x = rhs for the instances with want[b] = 1.  x: initial guess (zero if
// zero_guess) and result.  TV: type of rhs, x, the Krylov vectors and the iteration arithmetic, and
// of the sweeps (double: FP64 solve; float: inner solve of the mixed-precision refinement).
// true_check: recompute the residual after convergence.  it_base: iterations already done per
// instance (window count).  max_it: per-instance iteration budget of this run.
template <typename TV, bool SW64>
static int run_fgmres_t(SolveCtx& C, const TV* rhs, TV* x, bool zero_guess, const std::vector<int>& want,
                        double rtol, const std::vector<int>& max_it, bool true_check, const std::vector<int>& it_base,
                        RunStats& rs) {
  constexpr bool f64 = std::is_same<TV, double>::value;   // Krylov vectors and iteration arithmetic
  constexpr bool sw64 = SW64;                             // sweep arithmetic
  using TP = typename std::conditional<SW64, double, float>::type;   // per-task partial fluxes
  static_assert(f64 || !sw64, "FP64 sweeps need FP64 vectors");
  rte_problem* p = C.p;
  Ws& W = *C.ws;
  if (C.rec && !(f64 && sw64)) {
    set_error("run_fgmres: the first-cycle record needs an FP64 solve");
    return RTE_ERR_UNSUPPORTED;
  }
  TV* Vb;
  TV* Zb;
  TV* rb;
  const TV* sig_dof;
  const TV* sblk = nullptr;   // cross-section profiles: Sigma_s blocks per cell
  if constexpr (f64) {
    Vb = W.V.p;
    Zb = W.Z.p;
    rb = W.r.p;
    sig_dof = p->d_sig_dof.p;
    if (p->cellsig) sblk = p->d_sblk64.p;
  } else {
    Vb = W.V32.p;
    Zb = W.Z32.p;
    rb = W.r32.p;
    sig_dof = p->d_sig_dof32.p;
    if (p->cellsig) sblk = p->d_sblk32.p;
  }
  const int B = p->B, m = C.m;
  const long long ntot = p->ntot;
  cudaStream_t st = C.st;
  const dim3 vg = vec_grid(p);
  rs.iterations.assign(B, 0);
  rs.sweeps.assign(B, 0);
  rs.restarts.assign(B, 0);
  rs.status.assign(B, RTE_OK);
  rs.est.assign(B, 0.0);
  std::vector<int> act(want), hflag(B), hk(B);
  std::vector<double> hb(B), hbn(B);
  // ||rhs||
  RTE_CHECK_CUDA(cudaMemcpyAsync(W.active.p, act.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
  k_norm<<<B, 512, 0, st>>>(rhs, p->d_inst.p, W.active.p, W.bnorm.p);
  count_launch();
  // r0
  if (zero_guess) {
    k_copy_active<<<vg, 256, 0, st>>>(rb, rhs, p->d_inst.p, W.active.p);
    count_launch();
    k_zero_active<<<vg, 256, 0, st>>>(x, p->d_inst.p, W.active.p);
    count_launch();
  } else {
    RTE_TRY(launch_T(p, MODE_RES, sw64, x, f64, rhs, rb, f64, W.active.p, st));
    for (int b = 0; b < B; ++b) rs.sweeps[b] += act[b];
  }
  RTE_CHECK_CUDA(cudaGetLastError());
  RTE_CHECK_CUDA(cudaMemcpyAsync(hbn.data(), W.bnorm.p, B * 8, cudaMemcpyDeviceToHost, st));
  RTE_CHECK_CUDA(cudaStreamSynchronize(st));
  for (int b = 0; b < B; ++b)
    if (act[b] && hbn[b] == 0.0) { act[b] = 0; rs.est[b] = 0.0; }
  TV* Zbase = W.withZ ? Zb : Vb;
  while (true) {
    // beta = ||r||
    RTE_CHECK_CUDA(cudaMemcpyAsync(W.active.p, act.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
    k_norm<<<B, 512, 0, st>>>(rb, p->d_inst.p, W.active.p, W.beta.p);
    count_launch();
    RTE_CHECK_CUDA(cudaMemcpyAsync(hb.data(), W.beta.p, B * 8, cudaMemcpyDeviceToHost, st));
    RTE_CHECK_CUDA(cudaStreamSynchronize(st));
    int nact = 0;
    for (int b = 0; b < B; ++b) {
      if (!act[b]) continue;
      if (!std::isfinite(hb[b])) { act[b] = 0; rs.status[b] = RTE_ERR_NUMERIC; continue; }
      rs.est[b] = hb[b] / hbn[b];
      if (hb[b] <= rtol * hbn[b]) { act[b] = 0; continue; }
      if (rs.iterations[b] >= max_it[b]) { act[b] = 0; rs.status[b] = RTE_ERR_NOT_CONVERGED; continue; }
      ++nact;
    }
    if (nact == 0) break;
    // v_0 = r / beta, g = beta e_1
    RTE_CHECK_CUDA(cudaMemcpyAsync(W.active.p, act.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
    k_scale<<<vg, 256, 0, st>>>(Vb, rb, W.beta.p, p->d_inst.p, W.active.p);
    count_launch();
    {
      std::vector<double> g0((size_t)B * (m + 1), 0.0);
      std::vector<int> left(B, 0);
      for (int b = 0; b < B; ++b) {
        g0[(size_t)b * (m + 1)] = hb[b];
        left[b] = max_it[b] - rs.iterations[b];
      }
      RTE_CHECK_CUDA(cudaMemcpyAsync(W.g.p, g0.data(), g0.size() * 8, cudaMemcpyHostToDevice, st));
      RTE_CHECK_CUDA(cudaMemcpyAsync(W.iters_left.p, left.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
      RTE_CHECK_CUDA(cudaMemsetAsync(W.kcols.p, 0, B * sizeof(int), st));
    }
    std::vector<int> incycle(act);
    std::vector<int> outcome(B, RUN);
    std::vector<int> its0(rs.iterations);   // iterations before this cycle
    int it_first = 0;
    for (int b = 0; b < B; ++b)
      if (act[b]) { it_first = it_base[b] + rs.iterations[b]; break; }
    // The device drops finished instances from the active mask itself (Arnoldi step, phase C), so the
    // host reads the flags only every kCheck iterations: instances that stopped in between are skipped
    // by every kernel until the host catches up.
    const int kCheck = 8;
    *W.h_rtol = rtol;
    RTE_CHECK_CUDA(cudaMemcpyAsync(W.d_rtol.p, W.h_rtol, sizeof(double), cudaMemcpyHostToDevice, st));
    // the learned ROMSAD slot replaces the reduced solve of the first preconditioner apply of the solve
    const bool slot_now = C.slot_pending && W.withZ;
    for (int j = 0; j < m; ++j) {
      const int jg = it_first + j + 1;   // lock-step instances share the global iteration index
      const bool use_rom = W.withZ && C.any_rom && (jg <= C.window || C.post == RTE_POST_ROM);
      const bool rom_next_full = W.withZ && C.any_rom && (jg + 1 <= C.window || C.post == RTE_POST_ROM);
      // tensor-core ROMSAD products: applied at the start of each window iteration by their own kernels
      // instead of inside the fused Arnoldi step
      const bool tc = C.rom_tc && !f64;
      const bool rom_next = rom_next_full && !tc;
      // DSA on z_j (cycle start or multi-phase step) and on z_{j+1} (after the fused step): for every
      // instance outside the ROM window, for instances without a ROM inside it
      const bool dsa_now = C.dsa && W.withZ && (!use_rom || C.any_norom);
      const bool dsa_next = C.dsa && W.withZ && W.fused && j + 1 < m && (!rom_next_full || C.any_norom);
      // One Arnoldi iteration: w = A~ z_j into V[j+1], MGS, Givens, and the next preconditioned vector
      // z_{j+1} (the first one of a cycle, z_0, by the preconditioner kernel).
      auto body = [&](cudaStream_t s) -> int {
        TV* vj = Vb + (size_t)j * ntot;
        TV* zj = Zbase + (size_t)j * ntot;
        const bool start_pre = W.withZ && (j == 0 || !W.fused);
        if (W.withZ && tc && use_rom) {
          if constexpr (!f64) {
            if (start_pre) {   // z = v everywhere, then the ROM instances' z from the tensor-core apply
              k_copy_active<<<vg, 256, 0, s>>>(zj, vj, p->d_inst.p, W.active.p);
              count_launch();
            }
            for (RomPlan& pl : *C.plans) RTE_TRY(rom_tc_apply(pl, p, W.active.p, vj, zj, s));
          }
          if (start_pre && dsa_now) RTE_TRY(dsa_launch(p, f64, vj, zj, W.active.p, W.norom.p, s));
        } else if (start_pre) {
          if (use_rom) {
            const int2* it_p = W.items.p;
            int nit = W.nitems, Bv = B, nch = W.nchunk;
            const InstInfo* inst_p = p->d_inst.p;
            const int* act_p = W.active.p;
            const RomInstDev* ri_p = W.rominst.p;
            const TV* sd_p = sig_dof;
            const TV* sb_p = sblk;
            const TV* v_p = vj;
            TV* rp_p = reinterpret_cast<TV*>(W.rpart.p);
            TV* rc_p = reinterpret_cast<TV*>(W.rc.p);
            const bool sl = slot_now && j == 0;
            const int* sl_p = sl ? W.slot.p : nullptr;
            const TV* slc_p = nullptr;
            if (sl) {
              if constexpr (f64) slc_p = W.slot_c.p;
              else slc_p = W.slot_c32.p;
            }
            void* args[] = {&Bv, &it_p, &nit, &inst_p, &act_p, &ri_p, &sd_p, &sb_p, &v_p, &zj, &rp_p, &rc_p, &nch, &sl_p,
                            &slc_p};
            RTE_CHECK_CUDA(cudaLaunchCooperativeKernel((const void*)k_precond_coop<TV>, dim3(W.grid_pre), dim3(256),
                                                       args, 0, s));
            count_launch();
          } else if (!dsa_now) {
            k_copy_active<<<vg, 256, 0, s>>>(zj, vj, p->d_inst.p, W.active.p);
            count_launch();
          }
          if (dsa_now) RTE_TRY(dsa_launch(p, f64, vj, zj, W.active.p, use_rom ? W.norom.p : nullptr, s));
        }
        RTE_TRY(launch_op_partials(p, sw64, zj, f64, W.active.p, s));
        if (!W.fused) {
          int Bv = B, nit = W.nitems, ntask = p->tasks_per_inst, jj = j, mm = m, nch = W.nchunk, ldT = m + 1;
          long long nt = ntot;
          const int2* it_p = W.items.p;
          const InstInfo* inst_p = p->d_inst.p;
          int* act_p = W.active.p;
          const TP* part_p = reinterpret_cast<const TP*>(p->d_partial.p);
          const TV* z_p = zj;
          TV* V_p = Vb;
          TV* dp_p = reinterpret_cast<TV*>(W.part.p);
          TV* np_p = reinterpret_cast<TV*>(W.npart.p);
          TV* Lt_p = reinterpret_cast<TV*>(W.Lt.p);
          double* H_p = W.H.p;
          double* Hr_p = C.rec ? W.Hraw.p : nullptr;
          double* w0_p = W.w0.p;
          double* cs_p = W.cs.p;
          double* sn_p = W.sn.p;
          double* g_p = W.g.p;
          int* brk_p = W.brk.p;
          const double* bn_p = W.bnorm.p;
          const double* rt_p = W.d_rtol.p;
          int* il_p = W.iters_left.p;
          double* est_p = W.est.p;
          int* fl_p = W.flag.p;
          int* kc_p = W.kcols.p;
          double* hn_p = W.hnorm.p;
          int* a0_p = W.active0.p;
          void* args[] = {&Bv, &it_p, &nit, &inst_p, &act_p, &part_p, &ntask, &z_p, &V_p, &nt, &jj, &mm, &nch,
                          &dp_p, &np_p, &Lt_p, &ldT, &H_p, &Hr_p, &w0_p, &cs_p, &sn_p, &g_p, &brk_p, &bn_p, &rt_p,
                          &il_p, &est_p, &fl_p, &kc_p, &hn_p, &a0_p};
          RTE_CHECK_CUDA(cudaLaunchCooperativeKernel((const void*)k_arnoldi_wide<TP, TV>,
                                                     dim3(f64 ? W.grid_wide64 : W.grid_wide32), dim3(256), args, 0,
                                                     s));
          count_launch();
        } else {
          ArnArgs<TP, TV> A;
          A.B = B;
          A.nitems = W.nitems;
          A.ntask = p->tasks_per_inst;
          A.j = j;
          A.m = m;
          A.nchunk = W.nchunk;
          A.ldT = m + 1;
          A.rom_next = rom_next ? 1 : 0;
          A.ntot = ntot;
          A.items = W.items.p;
          A.inst = p->d_inst.p;
          A.active = W.active.p;
          A.active0 = W.active0.p;
          A.partial = reinterpret_cast<const TP*>(p->d_partial.p);
          A.z = zj;
          A.V = Vb;
          A.znext = (W.withZ && j + 1 < m) ? Zbase + (size_t)(j + 1) * ntot : nullptr;
          A.part = reinterpret_cast<TV*>(W.part.p);
          A.npart = reinterpret_cast<TV*>(W.npart.p);
          A.Tm = reinterpret_cast<TV*>(W.Lt.p);
          A.rpart = reinterpret_cast<TV*>(W.rpart.p);
          A.ri = W.rominst.p;
          A.sig_dof = sig_dof;
          A.sblk = sblk;
          A.H = W.H.p;
          A.Hraw = C.rec ? W.Hraw.p : nullptr;
          A.w0 = W.w0.p;
          A.cs = W.cs.p;
          A.sn = W.sn.p;
          A.g = W.g.p;
          A.est = W.est.p;
          A.bnorm = W.bnorm.p;
          A.rtol = W.d_rtol.p;
          A.iters_left = W.iters_left.p;
          A.flag = W.flag.p;
          A.kcols = W.kcols.p;
          void* args[] = {&A};
          RTE_CHECK_CUDA(cudaLaunchCooperativeKernel((const void*)k_arnoldi_coop<TP, TV>,
                                                     dim3(f64 ? W.grid_post64 : W.grid_post32), dim3(256), args, 0,
                                                     s));
          count_launch();
          if (dsa_next)
            RTE_TRY(dsa_launch(p, f64, Vb + (size_t)(j + 1) * ntot, A.znext, W.active.p,
                               rom_next_full ? W.norom.p : nullptr, s));
        }
        RTE_CHECK_CUDA(cudaGetLastError());
        return RTE_OK;
      };
      const int key = j | (use_rom ? 1 << 8 : 0) | (f64 ? 1 << 9 : 0) | (C.rec ? 1 << 10 : 0) |
                      (rom_next ? 1 << 11 : 0) | (slot_now && j == 0 ? 1 << 12 : 0) | (sw64 ? 1 << 13 : 0) |
                      (dsa_now ? 1 << 14 : 0) | (dsa_next ? 1 << 15 : 0) | (tc ? 1 << 16 : 0);
      auto it = W.graphs.find(key);
      if (it == W.graphs.end()) {
        // capture this iteration once; later iterations with the same key replay it
        const long long n0 = launches_so_far();
        RTE_CHECK_CUDA(cudaStreamBeginCapture(W.cap, cudaStreamCaptureModeThreadLocal));
        const int rc = body(W.cap);
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(W.cap, &g);
        if (rc != RTE_OK) {
          if (g) cudaGraphDestroy(g);
          return rc;
        }
        RTE_CHECK_CUDA(ec);
        cudaGraphExec_t ex = nullptr;
        const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        RTE_CHECK_CUDA(ei);
        it = W.graphs.emplace(key, Ws::Graph{ex, (int)(launches_so_far() - n0)}).first;
        add_launches(-(long long)it->second.launches);   // counted when replayed
      }
      RTE_CHECK_CUDA(cudaGraphLaunch(it->second.exec, st));
      if (j == 0) C.slot_pending = false;
      add_launches(it->second.launches);
      if ((j + 1) % kCheck != 0 && j != m - 1) continue;
      RTE_CHECK_CUDA(cudaMemcpyAsync(W.hflag, W.flag.p, B * sizeof(int), cudaMemcpyDeviceToHost, st));
      RTE_CHECK_CUDA(cudaMemcpyAsync(W.hk, W.kcols.p, B * sizeof(int), cudaMemcpyDeviceToHost, st));
      RTE_CHECK_CUDA(cudaStreamSynchronize(st));
      int still = 0;
      for (int b = 0; b < B; ++b) {
        if (!act[b]) continue;
        rs.iterations[b] = its0[b] + W.hk[b];
        if (W.hflag[b] != RUN) {
          outcome[b] = W.hflag[b];
          act[b] = 0;
        } else {
          ++still;
        }
      }
      if (still == 0) break;
    }
    for (int b = 0; b < B; ++b)
      if (incycle[b]) rs.sweeps[b] += rs.iterations[b] - its0[b];   // one operator apply per iteration
    // first-cycle record for the xi recurrence: unrotated H, the Krylov basis (Z = V without a
    // preconditioner) and beta
    if (C.rec && !C.rec->done) {
      int k0 = 0;
      RTE_CHECK_CUDA(cudaMemcpyAsync(&k0, W.kcols.p, sizeof(int), cudaMemcpyDeviceToHost, st));
      RTE_CHECK_CUDA(cudaStreamSynchronize(st));
      C.rec->k = k0;
      C.rec->beta = hb[0];
      C.rec->m = m;
      C.rec->H.assign((size_t)m * (m + 1), 0.0);
      RTE_CHECK_CUDA(cudaMemcpyAsync(C.rec->H.data(), W.Hraw.p, C.rec->H.size() * 8, cudaMemcpyDeviceToHost, st));
      const int nv = std::min(k0, C.rec->want);
      RTE_TRY(C.rec->Z.ensure((size_t)std::max(1, nv) * ntot));
      if (nv > 0)
        RTE_CHECK_CUDA(cudaMemcpyAsync(C.rec->Z.p, Zbase, (size_t)nv * ntot * 8, cudaMemcpyDeviceToDevice, st));
      C.rec->nz = nv;
      C.rec->done = true;
    }
    // end of cycle: phi += Z y for the instances of this cycle
    k_backsolve<TV><<<B, 128, 0, st>>>(W.H.p, W.g.p, m, B, W.kcols.p, W.y.p);
    count_launch();
    k_update<<<vg, 256, 0, st>>>(x, Zbase, ntot, m, p->d_inst.p, W.kcols.p, W.y.p);
    count_launch();
    RTE_CHECK_CUDA(cudaGetLastError());
    std::vector<double> hest(B);
    RTE_CHECK_CUDA(cudaMemcpyAsync(hest.data(), W.est.p, B * 8, cudaMemcpyDeviceToHost, st));
    RTE_CHECK_CUDA(cudaStreamSynchronize(st));
    // decide per instance: finished, check residual, or restart
    std::vector<int> resid(B, 0);
    for (int b = 0; b < B; ++b) {
      if (!incycle[b]) continue;
      rs.est[b] = hest[b] / hbn[b];
      const int o = outcome[b];
      if (o == STOP_NUMERIC) { rs.status[b] = RTE_ERR_NUMERIC; continue; }
      if (o == STOP_CONV || o == STOP_BREAK) {
        if (true_check) resid[b] = 1;  // verified below (uncounted check sweep)
        continue;
      }
      // restart or iteration cap
      if (rs.iterations[b] >= max_it[b]) { rs.status[b] = RTE_ERR_NOT_CONVERGED; continue; }
      resid[b] = 2;
    }
    bool any = false;
    for (int b = 0; b < B; ++b) any = any || resid[b];
    if (!any) break;
    std::vector<int> mask(B);
    for (int b = 0; b < B; ++b) mask[b] = resid[b] ? 1 : 0;
    RTE_CHECK_CUDA(cudaMemcpyAsync(W.active.p, mask.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
    RTE_TRY(launch_T(p, MODE_RES, sw64, x, f64, rhs, rb, f64, W.active.p, st));
    for (int b = 0; b < B; ++b)
      if (resid[b] == 2) { rs.sweeps[b] += 1; rs.restarts[b] += 1; }
    for (int b = 0; b < B; ++b) act[b] = mask[b];
    // check-sweep instances: the loop head computes beta and stops them if within 2 rtol
    if (true_check) {
      k_norm<<<B, 512, 0, st>>>(rb, p->d_inst.p, W.active.p, W.nrm.p);
      count_launch();
      std::vector<double> hn(B);
      RTE_CHECK_CUDA(cudaMemcpyAsync(hn.data(), W.nrm.p, B * 8, cudaMemcpyDeviceToHost, st));
      RTE_CHECK_CUDA(cudaStreamSynchronize(st));
      for (int b = 0; b < B; ++b) {
        if (resid[b] != 1) continue;
        if (hn[b] <= 2.0 * rtol * hbn[b] || rs.iterations[b] >= max_it[b]) {
          act[b] = 0;
          if (!(hn[b] <= 2.0 * rtol * hbn[b])) rs.status[b] = RTE_ERR_NOT_CONVERGED;
        } else {
          rs.restarts[b] += 1;
        }
      }
    }
  }
  return RTE_OK;
}

// Precision of a run: everything FP64; everything FP32; or FP32 sweeps (and partial fluxes) with FP64
// Krylov vectors, MGS and Givens.  rhs and x are double unless the run is all FP32.
enum RunPrecision { RUN_F64 = 0, RUN_F32 = 1, RUN_F32_SWEEP_F64_KRYLOV = 2 };

static int run_fgmres(SolveCtx& C, const void* rhs, void* x, bool zero_guess, const std::vector<int>& want,
                      double rtol, const std::vector<int>& max_it, int prec, bool true_check,
                      const std::vector<int>& it_base, RunStats& rs) {
  if (prec == RUN_F64)
    return run_fgmres_t<double, true>(C, static_cast<const double*>(rhs), static_cast<double*>(x), zero_guess, want,
                                      rtol, max_it, true_check, it_base, rs);
  if (prec == RUN_F32_SWEEP_F64_KRYLOV)
    return run_fgmres_t<double, false>(C, static_cast<const double*>(rhs), static_cast<double*>(x), zero_guess, want,
                                       rtol, max_it, true_check, it_base, rs);
  return run_fgmres_t<float, false>(C, static_cast<const float*>(rhs), static_cast<float*>(x), zero_guess, want, rtol,
                                    max_it, true_check, it_base, rs);
}

static Ws* get_ws(rte_problem* p) {
  if (!p->krylov_ws) p->krylov_ws = std::shared_ptr<void>(new Ws(), [](void* q) { delete static_cast<Ws*>(q); });
  return static_cast<Ws*>(p->krylov_ws.get());
}

// High-fidelity FP64 FGMRES (zero initial guess) on a one-instance problem, recording the first cycle; used
// by the greedy ROM construction (step 2(a)).  dsa_variant < 0: M = I; otherwise FGMRES-DSA (the DSA
// preconditioner of that variant from the first iteration), the paper's high-fidelity solver.  The recorded
// Z holds the preconditioned vectors z = M^{-1} v the xi recurrence needs.  x: device output [N].
int hf_solve(rte_problem* p, double rtol, int restart, int max_iter, int dsa_variant, double* x, FirstCycle* rec,
             int* iterations, int* status) {
  Ws* ws = get_ws(p);
  const bool dsa = dsa_variant >= 0;
  if (dsa) RTE_TRY(dsa_check(p));
  RTE_TRY(ws->alloc(p, restart, dsa));
  RTE_TRY(prepare_sweeps(p));
  SolveCtx C{p, nullptr, restart, 0, dsa ? RTE_POST_DSA : RTE_POST_IDENTITY, 0, ws, rec};
  std::vector<RomPlan> none;
  C.plans = &none;
  if (dsa) {
    C.dsa = true;
    C.no_rom_mask.assign(p->B, 1);
    C.any_norom = true;
    RTE_CHECK_CUDA(cudaMemcpy(ws->norom.p, C.no_rom_mask.data(), p->B * sizeof(int), cudaMemcpyHostToDevice));
    RTE_TRY(dsa_prepare(p, dsa_variant, 0));
  }
  RTE_TRY(launch_T(p, MODE_RHS, true, nullptr, true, nullptr, ws->bt.p, true, nullptr, 0));
  std::vector<int> all(p->B, 1), zero(p->B, 0);
  RunStats rs;
  std::vector<int> cap(p->B, max_iter);
  RTE_TRY(run_fgmres(C, ws->bt.p, x, true, all, rtol, cap, RUN_F64, false, zero, rs));
  *iterations = rs.iterations[0];
  *status = rs.status[0];
  return RTE_OK;
}

}  // namespace rte

using namespace rte;

extern "C" int fgmres_solve(rte_problem_t p, const romsad_t* roms, const fgmres_opts* o, const void* phi0, void* phi,
                            fgmres_stats* stats, void* stream) {
  RTE_ARG(p && o && phi && stats, "null handle or pointer");
  RTE_ARG(o->restart >= 1 && o->restart <= 128, "restart must be in [1, 128]");
  RTE_ARG(o->rtol > 0.0 && o->max_iter >= 1, "rtol must be > 0 and max_iter >= 1");
  RTE_ARG(o->mode == RTE_MODE_FP64 || o->mode == RTE_MODE_MIXED || o->mode == RTE_MODE_MIXED_F64KRYLOV,
          "unknown mode");
  RTE_ARG(o->post_mode == RTE_POST_ROM || o->post_mode == RTE_POST_IDENTITY || o->post_mode == RTE_POST_DSA,
          "unknown post_mode");
  RTE_ARG(o->mode == RTE_MODE_FP64 || o->refine_residual == RTE_RESIDUAL_DF || o->refine_residual == RTE_RESIDUAL_FP64,
          "unknown refine_residual");
  RTE_ARG(o->rom_bf16 == 0 || o->rom_bf16 == 1, "rom_bf16 must be 0 or 1");
  if (p->cellsig && o->rom_bf16) {
    set_error("fgmres_solve: no tensor-core ROM products with cross-section profiles");
    return RTE_ERR_UNSUPPORTED;
  }
  const bool use_dsa = o->post_mode == RTE_POST_DSA;
  if (use_dsa) {
    RTE_ARG(o->dsa_variant == RTE_DSA_PARTIAL || o->dsa_variant == RTE_DSA_LUMPED || o->dsa_variant == RTE_DSA_FULL,
            "unknown dsa_variant");
    RTE_TRY(dsa_check(p));
  }
  if (roms)
    for (int b = 0; b < p->B; ++b)
      if (roms[b]) RTE_TRY(rom_check_mesh(roms[b], p, b));
  cudaStream_t st = (cudaStream_t)stream;
  bool any_rom = false;
  if (roms)
    for (int b = 0; b < p->B; ++b) any_rom = any_rom || roms[b] != nullptr;
  Ws* ws = get_ws(p);
  RTE_TRY(ws->alloc(p, o->restart, any_rom || use_dsa));
  // output location: device pointer, or host pointer (solve into a device buffer, copy back)
  cudaPointerAttributes attr;
  bool host_out = false;
  if (cudaPointerGetAttributes(&attr, phi) != cudaSuccess || attr.type == cudaMemoryTypeHost ||
      attr.type == cudaMemoryTypeUnregistered) {
    cudaGetLastError();
    host_out = true;
  }
  double* x;
  if (host_out) {
    RTE_TRY(ws->phi_in.ensure(p->ntot));
    x = ws->phi_in.p;
  } else {
    x = (double*)phi;
  }
  const int B = p->B;
  SolveCtx C{p, roms, o->restart, o->window, o->post_mode, st, ws};
  // ROM plans: group instances by ROM handle, assemble and factor U^T A_mu U once per solve
  // ROM plans: group instances by ROM handle and factor U^T A_mu U once per solve.  The plans live in
  // the workspace so that captured iteration graphs stay valid from one solve to the next.
  C.no_rom_mask.assign(B, 1);
  {
    std::vector<romsad_t> prom;
    std::vector<std::vector<int>> pids;
    if (roms) {
      std::vector<std::pair<romsad_t, int>> groups;
      for (int b = 0; b < B; ++b)
        if (roms[b]) { groups.push_back({roms[b], b}); C.no_rom_mask[b] = 0; }
      std::sort(groups.begin(), groups.end());
      size_t g0 = 0;
      while (g0 < groups.size()) {
        size_t g1 = g0;
        std::vector<int> ids;
        while (g1 < groups.size() && groups[g1].first == groups[g0].first) ids.push_back(groups[g1++].second);
        prom.push_back(groups[g0].first);
        pids.push_back(ids);
        g0 = g1;
      }
    }
    if (prom != ws->plan_rom || pids != ws->plan_ids) {
      ws->drop_graphs();
      ws->plans.clear();
      ws->plans.resize(prom.size());
      ws->plan_rom = prom;
      ws->plan_ids = pids;
    }
    for (size_t q = 0; q < prom.size(); ++q) {
      RomPlan& pl = ws->plans[q];
      RTE_TRY(pl.build(prom[q], p, pids[q], st));
      RTE_TRY(pl.inv32.ensure(pl.lu.n));
      k_inv_to_f32<<<64, 256, 0, st>>>(pl.lu.p, pl.inv32.p, (long long)pl.lu.n);
      count_launch();
      romsad* rm = prom[q];
      RTE_TRY(pl.WT.ensure((size_t)rm->N * std::max(1, rm->r)));
      RTE_TRY(pl.WT32.ensure((size_t)rm->N * std::max(1, rm->r)));
      k_w_transpose<<<152, 256, 0, st>>>(rm->W.p, rm->N, rm->rmax, rm->r, pl.WT.p, pl.WT32.p);
      count_launch();
      if (o->rom_bf16 && o->mode == RTE_MODE_MIXED) RTE_TRY(rom_tc_plan_setup(pl, st));
    }
    RTE_CHECK_CUDA(cudaMemcpyAsync(ws->norom.p, C.no_rom_mask.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
    C.any_rom = any_rom;
    for (int b = 0; b < B; ++b) C.any_norom = C.any_norom || C.no_rom_mask[b] != 0;
    C.dsa = use_dsa;
    C.rom_tc = o->rom_bf16 && o->mode == RTE_MODE_MIXED;
    if (use_dsa) RTE_TRY(dsa_prepare(p, o->dsa_variant, st));
    std::vector<RomInstDev> ri(B);
    for (int b = 0; b < B; ++b)
      ri[b] = RomInstDev{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0, 0, 0};
    for (size_t q = 0; q < prom.size(); ++q)
      for (size_t sl = 0; sl < pids[q].size(); ++sl) {
        romsad* rm = prom[q];
        ri[pids[q][sl]] = RomInstDev{rm->P.p,
                                     rm->W.p,
                                     rm->P32.p,
                                     rm->W32.p,
                                     ws->plans[q].lu.p + sl * 64 * 64,
                                     ws->plans[q].inv32.p + sl * 64 * 64,
                                     ws->plans[q].WT.p,
                                     ws->plans[q].WT32.p,
                                     rm->r,
                                     rm->rmax,
                                     1,
                                     rm->N};
      }
    RTE_CHECK_CUDA(cudaMemcpyAsync(ws->rominst.p, ri.data(), B * sizeof(RomInstDev), cudaMemcpyHostToDevice, st));
    RTE_CHECK_CUDA(cudaStreamSynchronize(st));
  }
  RTE_TRY(prepare_sweeps(p));
  C.plans = &ws->plans;
  std::vector<int> all(B, 1), zero(B, 0);
  // b~ (FP64 sweep, counted)
  RTE_TRY(launch_T(p, MODE_RHS, true, nullptr, true, nullptr, ws->bt.p, true, nullptr, st));
  bool warm = o->warm_start == 1 && phi0 != nullptr;
  if (warm) RTE_CHECK_CUDA(cudaMemcpyAsync(x, phi0, p->ntot * 8, cudaMemcpyDeviceToDevice, st));
  if (o->warm_start == 2 && roms) {
    // learned warm start: phi0 = b~ + W c_hat(mu) per ROM group with an MLP, zero elsewhere
    RTE_CHECK_CUDA(cudaMemsetAsync(x, 0, p->ntot * 8, st));
    std::vector<std::pair<romsad_t, int>> groups;
    for (int b = 0; b < p->B; ++b)
      if (roms[b] && roms[b]->mlp) groups.push_back({roms[b], b});
    std::sort(groups.begin(), groups.end());
    size_t g0 = 0;
    while (g0 < groups.size()) {
      size_t g1 = g0;
      std::vector<int> ids;
      while (g1 < groups.size() && groups[g1].first == groups[g0].first) ids.push_back(groups[g1++].second);
      RTE_CHECK_CUDA(cudaMemcpyAsync(ws->list.p, ids.data(), ids.size() * sizeof(int), cudaMemcpyHostToDevice, st));
      RTE_TRY(mlp_predict_instances(groups[g0].first->mlp, p, ws->list.p, ids, ws->rom_c.p, st));
      RTE_TRY(rom_lift_list(groups[g0].first, p, ws->list.p, (int)ids.size(), ws->bt.p, ws->rom_c.p, x, st));
      g0 = g1;
    }
    warm = !groups.empty();
  }
  std::vector<int> learned(B, 0);
  if (o->warm_start == 2 && warm) {
    // The plain ROMSAD start (zero) is the fallback for an instance whose learned start is not finite,
    // read from the norm of the start itself (no sweep).  (The residual norm is no test of a learned
    // start: it removes the slow, smooth error components that take FGMRES-ROMSAD many iterations while it
    // can raise the residual in fast ones.)
    std::vector<int> all1(B, 1);
    RTE_CHECK_CUDA(cudaMemcpyAsync(ws->active.p, all1.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
    k_norm<<<B, 512, 0, st>>>(x, p->d_inst.p, ws->active.p, ws->nrm.p);
    count_launch();
    std::vector<double> hx(B);
    RTE_CHECK_CUDA(cudaMemcpyAsync(hx.data(), ws->nrm.p, B * 8, cudaMemcpyDeviceToHost, st));
    RTE_CHECK_CUDA(cudaStreamSynchronize(st));
    std::vector<int> fallback(B, 0);
    bool anyf = false;
    for (int b = 0; b < B; ++b) {
      const bool has = roms[b] && roms[b]->mlp;
      learned[b] = has && std::isfinite(hx[b]);
      fallback[b] = !learned[b];
      anyf = anyf || fallback[b];
    }
    if (anyf) {
      const dim3 vg = vec_grid(p);
      RTE_CHECK_CUDA(cudaMemcpyAsync(ws->active.p, fallback.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
      k_zero_active<<<vg, 256, 0, st>>>(x, p->d_inst.p, ws->active.p);
      count_launch();
    }
  }
  // learned correction in the ROMSAD slot (zero start only): the first preconditioner apply takes the
  // coefficients c_hat(mu) / ||b~|| from each instance's ROM MLP instead of the reduced solve; instances
  // without an MLP, or whose prediction is not finite, keep the plain ROMSAD apply
  std::vector<int> slot_used(B, 0);
  if (o->learned_slot && roms && !warm) {
    std::vector<int> all1(B, 1);
    RTE_CHECK_CUDA(cudaMemcpyAsync(ws->active.p, all1.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
    k_norm<<<B, 512, 0, st>>>(ws->bt.p, p->d_inst.p, ws->active.p, ws->beta.p);
    count_launch();
    std::vector<double> hb(B), cs((size_t)B * 64, 0.0);
    RTE_CHECK_CUDA(cudaMemcpyAsync(hb.data(), ws->beta.p, B * 8, cudaMemcpyDeviceToHost, st));
    std::vector<std::pair<romsad_t, int>> groups;
    for (int b = 0; b < B; ++b)
      if (roms[b] && roms[b]->mlp) groups.push_back({roms[b], b});
    std::sort(groups.begin(), groups.end());
    size_t g0 = 0;
    while (g0 < groups.size()) {
      size_t g1 = g0;
      std::vector<int> ids;
      while (g1 < groups.size() && groups[g1].first == groups[g0].first) ids.push_back(groups[g1++].second);
      RTE_CHECK_CUDA(cudaMemcpyAsync(ws->list.p, ids.data(), ids.size() * sizeof(int), cudaMemcpyHostToDevice, st));
      RTE_TRY(mlp_predict_instances(groups[g0].first->mlp, p, ws->list.p, ids, ws->rom_c.p, st));
      std::vector<double> hc(ids.size() * 64);
      RTE_CHECK_CUDA(cudaMemcpyAsync(hc.data(), ws->rom_c.p, hc.size() * 8, cudaMemcpyDeviceToHost, st));
      RTE_CHECK_CUDA(cudaStreamSynchronize(st));
      for (size_t k = 0; k < ids.size(); ++k) {
        const int b = ids[k];
        const int r = roms[b]->r;
        bool ok = hb[b] > 0.0 && std::isfinite(hb[b]);
        for (int q = 0; q < r; ++q) ok = ok && std::isfinite(hc[k * 64 + q]);
        if (!ok) continue;
        slot_used[b] = 1;
        for (int q = 0; q < r; ++q) cs[(size_t)b * 64 + q] = hc[k * 64 + q] / hb[b];
      }
      g0 = g1;
    }
    std::vector<float> cs32(cs.begin(), cs.end());
    RTE_CHECK_CUDA(cudaMemcpyAsync(ws->slot.p, slot_used.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
    RTE_CHECK_CUDA(cudaMemcpyAsync(ws->slot_c.p, cs.data(), cs.size() * 8, cudaMemcpyHostToDevice, st));
    RTE_CHECK_CUDA(cudaMemcpyAsync(ws->slot_c32.p, cs32.data(), cs32.size() * 4, cudaMemcpyHostToDevice, st));
    RTE_CHECK_CUDA(cudaStreamSynchronize(st));
    for (int b = 0; b < B; ++b) C.slot_pending = C.slot_pending || slot_used[b];
  }
  std::vector<fgmres_stats> S(B);
  for (int b = 0; b < B; ++b) {
    std::memset(&S[b], 0, sizeof(fgmres_stats));
    S[b].sweeps = 1;
    S[b].sweeps_fp64 = 1;
    S[b].learned_start = learned[b];
    S[b].learned_slot = slot_used[b];
    S[b].true_rel_residual = NAN;
    S[b].true_linf_residual = NAN;
  }
  if (o->mode == RTE_MODE_FP64) {
    RunStats rs;
    std::vector<int> cap(B, o->max_iter);
    RTE_TRY(run_fgmres(C, ws->bt.p, x, !warm, all, o->rtol, cap, RUN_F64, o->true_residual_check != 0, zero, rs));
    for (int b = 0; b < B; ++b) {
      S[b].iterations = rs.iterations[b];
      S[b].sweeps += rs.sweeps[b];
      S[b].sweeps_fp64 += rs.sweeps[b];
      S[b].restarts = rs.restarts[b];
      S[b].est_rel_residual = rs.est[b];
      S[b].status = rs.status[b];
    }
  } else {
    // FP64 iterative refinement around the FP32-sweep inner FGMRES.  The outer residual has its own
    // buffer (ro): the inner solve keeps its working residual in r and recomputes it from its
    // right-hand side at every restart, so the two must not alias.
    //
    // Residual precision.  b~ is FP64.  A refinement residual b~ - A~ x only steers the next inner solve, so
    // it runs in double-float arithmetic (~1e-14 relative, on the FP32 pipe) unless the step is predicted to
    // converge; the residual that certifies convergence is always an FP64 sweep: an instance whose
    // double-float residual meets rtol is re-checked in FP64 before it stops (ro64 marks which residuals
    // are FP64).  refine_residual = RTE_RESIDUAL_FP64 makes every residual FP64.
    const bool res_df = o->refine_residual == RTE_RESIDUAL_DF && !p->cellsig;   // no double-float sweep with profiles
    const dim3 vg = vec_grid(p);
    double* ro = ws->ro.p;
    std::vector<int> act(B, 1), esc(B, 0), ro64(B, 1);
    auto residual = [&](const std::vector<int>& mask64, const std::vector<int>& maskdf) -> int {
      bool any64 = false, anydf = false;
      for (int b = 0; b < B; ++b) { any64 = any64 || mask64[b]; anydf = anydf || maskdf[b]; }
      if (any64) {
        RTE_CHECK_CUDA(cudaMemcpyAsync(ws->active.p, mask64.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
        RTE_TRY(launch_T(p, MODE_RES, true, x, true, ws->bt.p, ro, true, ws->active.p, st));
      }
      if (anydf) {
        RTE_CHECK_CUDA(cudaMemcpyAsync(ws->active.p, maskdf.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
        RTE_TRY(launch_T_df(p, MODE_RES, x, ws->bt.p, ro, ws->active.p, st));
      }
      for (int b = 0; b < B; ++b) {
        if (mask64[b]) { S[b].sweeps += 1; S[b].sweeps_fp64 += 1; ro64[b] = 1; }
        if (maskdf[b]) { S[b].sweeps += 1; S[b].sweeps_df += 1; ro64[b] = 0; }
      }
      return RTE_OK;
    };
    // A warm start (given or learned) is folded into the first inner solve: it solves A~ d = b~ from
    // d0 = phi0 in the inner precision (its starting residual is one FP32 sweep, counted by the inner run) and
    // replaces x, instead of a refinement residual of phi0 being computed first.  The outer residual then
    // starts at b~, as for a zero start.
    const bool fold_warm = warm;
    RTE_CHECK_CUDA(cudaMemcpyAsync(ro, ws->bt.p, p->ntot * 8, cudaMemcpyDeviceToDevice, st));
    if (!warm) RTE_CHECK_CUDA(cudaMemsetAsync(x, 0, p->ntot * 8, st));
    // An outer step is meant to cut the true residual by about inner_rtol.  An instance whose step
    // cut it by less than esc_ratio is one whose slowest modes the FP32 operator cannot resolve
    // (eigenvalues of A~ near the FP32 rounding of I - T Sigma_s); it leaves the refinement and is
    // finished by FP64 FGMRES from its current iterate.  Each inner solve is capped at inner_cap
    // iterations so that a stagnating instance is caught early.
    const double esc_ratio = std::max(0.25, std::sqrt(o->inner_rtol));
    const int inner_cap = std::max(4 * o->restart, 512);
    // a step predicted (inner solve's own residual reduction x current residual) to land below
    // kPredict * rtol takes its residual in FP64 directly, saving the double-float sweep of the check
    const double kPredict = 0.5;
    std::vector<double> hb(B), hr(B), hprev(B, 0.0);
    RTE_CHECK_CUDA(cudaMemcpyAsync(ws->active.p, act.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
    k_norm<<<B, 512, 0, st>>>(ws->bt.p, p->d_inst.p, ws->active.p, ws->nrm.p);
    count_launch();
    RTE_CHECK_CUDA(cudaMemcpyAsync(hb.data(), ws->nrm.p, B * 8, cudaMemcpyDeviceToHost, st));
    RTE_CHECK_CUDA(cudaStreamSynchronize(st));
    auto read_norms = [&]() -> int {
      RTE_CHECK_CUDA(cudaMemcpyAsync(ws->active.p, act.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
      k_norm<<<B, 512, 0, st>>>(ro, p->d_inst.p, ws->active.p, ws->nrm.p);
      count_launch();
      RTE_CHECK_CUDA(cudaMemcpyAsync(hr.data(), ws->nrm.p, B * 8, cudaMemcpyDeviceToHost, st));
      RTE_CHECK_CUDA(cudaStreamSynchronize(st));
      return RTE_OK;
    };
    for (int outer = 0; outer <= o->max_outer; ++outer) {
      RTE_TRY(read_norms());
      // certification: a double-float residual that meets rtol is recomputed in FP64
      {
        std::vector<int> cert(B, 0), none(B, 0);
        bool any = false;
        for (int b = 0; b < B; ++b) {
          if (!act[b] || ro64[b]) continue;
          const double rel = hb[b] > 0 ? hr[b] / hb[b] : 0.0;
          if (std::isfinite(rel) && rel <= o->rtol) { cert[b] = 1; any = true; }
        }
        if (any) {
          RTE_TRY(residual(cert, none));
          RTE_TRY(read_norms());
        }
      }
      int nact = 0;
      for (int b = 0; b < B; ++b) {
        if (!act[b]) continue;
        double rel = hb[b] > 0 ? hr[b] / hb[b] : 0.0;
        S[b].true_rel_residual = rel;
        S[b].est_rel_residual = rel;
        if (!std::isfinite(rel)) { act[b] = 0; S[b].status = RTE_ERR_NUMERIC; continue; }
        if (rel <= o->rtol) { act[b] = 0; continue; }
        if (S[b].iterations >= o->max_iter) {
          act[b] = 0;
          S[b].status = RTE_ERR_NOT_CONVERGED;
          continue;
        }
        if (outer == o->max_outer || (outer > 0 && hr[b] > esc_ratio * hprev[b])) {
          act[b] = 0;
          esc[b] = 1;
          continue;
        }
        hprev[b] = hr[b];
        ++nact;
      }
      if (nact == 0) break;
      // inner solve A~ d = ro, zero guess: entirely in FP32 (right-hand side rounded to FP32), or with FP32
      // sweeps and FP64 Krylov vectors, MGS and Givens (RTE_MODE_MIXED_F64KRYLOV)
      // the ROMSAD window counts the iterations of the whole solve: only the first inner solve opens with it
      std::vector<int> cap(B, 0), done(B, 0);
      for (int b = 0; b < B; ++b) {
        cap[b] = std::min(inner_cap, o->max_iter - S[b].iterations);
        done[b] = S[b].iterations;
      }
      RTE_CHECK_CUDA(cudaMemcpyAsync(ws->active.p, act.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
      RunStats rs;
      const bool from_x = fold_warm && outer == 0;   // first inner solve of a warm start: d0 = x, then x = d
      if (o->mode == RTE_MODE_MIXED_F64KRYLOV) {
        if (from_x) {
          k_copy_active<<<vg, 256, 0, st>>>(ws->d.p, x, p->d_inst.p, ws->active.p);
          count_launch();
        }
        RTE_TRY(run_fgmres(C, ro, ws->d.p, !from_x, act, o->inner_rtol, cap, RUN_F32_SWEEP_F64_KRYLOV, false, done,
                           rs));
        RTE_CHECK_CUDA(cudaMemcpyAsync(ws->active.p, act.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
        if (from_x) k_copy_active<<<vg, 256, 0, st>>>(x, ws->d.p, p->d_inst.p, ws->active.p);
        else k_axpy_active<<<vg, 256, 0, st>>>(x, ws->d.p, p->d_inst.p, ws->active.p);
      } else {
        k_copy_active<<<vg, 256, 0, st>>>(ws->rin32.p, ro, p->d_inst.p, ws->active.p);
        count_launch();
        if (from_x) {
          k_copy_active<<<vg, 256, 0, st>>>(ws->d32.p, x, p->d_inst.p, ws->active.p);
          count_launch();
        }
        RTE_TRY(run_fgmres(C, ws->rin32.p, ws->d32.p, !from_x, act, o->inner_rtol, cap, RUN_F32, false, done, rs));
        RTE_CHECK_CUDA(cudaMemcpyAsync(ws->active.p, act.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
        if (from_x) k_copy_active<<<vg, 256, 0, st>>>(x, ws->d32.p, p->d_inst.p, ws->active.p);
        else k_axpy_active<<<vg, 256, 0, st>>>(x, ws->d32.p, p->d_inst.p, ws->active.p);
      }
      count_launch();
      // ro = b~ - A~ x: FP64 where the step is predicted to converge, double-float elsewhere
      std::vector<int> m64(B, 0), mdf(B, 0);
      for (int b = 0; b < B; ++b) {
        if (!act[b]) continue;
        const double predicted = rs.est[b] * (hb[b] > 0 ? hr[b] / hb[b] : 0.0);
        if (!res_df || predicted <= kPredict * o->rtol) m64[b] = 1;
        else mdf[b] = 1;
      }
      RTE_TRY(residual(m64, mdf));
      for (int b = 0; b < B; ++b) {
        if (!act[b]) continue;
        S[b].iterations += rs.iterations[b];
        S[b].sweeps += rs.sweeps[b];
        S[b].restarts += rs.restarts[b];
        S[b].outer += 1;
        if (rs.status[b] == RTE_ERR_NUMERIC) { act[b] = 0; S[b].status = RTE_ERR_NUMERIC; }
      }
    }
    bool any_esc = false;
    for (int b = 0; b < B; ++b) any_esc = any_esc || esc[b];
    if (any_esc) {
      std::vector<int> cap(B, 0), done(B, 0);
      for (int b = 0; b < B; ++b) {
        cap[b] = std::max(1, o->max_iter - S[b].iterations);
        done[b] = S[b].iterations;
      }
      RunStats rs;
      RTE_TRY(run_fgmres(C, ws->bt.p, x, false, esc, o->rtol, cap, RUN_F64, o->true_residual_check != 0, done, rs));
      for (int b = 0; b < B; ++b) {
        if (!esc[b]) continue;
        S[b].iterations += rs.iterations[b];
        S[b].sweeps += rs.sweeps[b];
        S[b].sweeps_fp64 += rs.sweeps[b];
        S[b].restarts += rs.restarts[b];
        S[b].escalated = 1;
        S[b].status = rs.status[b];
      }
      // FP64 residual of the escalated instances for the report below (not a solver sweep)
      RTE_CHECK_CUDA(cudaMemcpyAsync(ws->active.p, esc.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
      RTE_TRY(launch_T(p, MODE_RES, true, x, true, ws->bt.p, ro, true, ws->active.p, st));
      for (int b = 0; b < B; ++b)
        if (esc[b]) ro64[b] = 1;
    }
    // instances that stopped on a double-float residual (not converged, or NaN): their reported residual is
    // recomputed in FP64 (not a solver sweep)
    {
      std::vector<int> redo(B, 0);
      bool any = false;
      for (int b = 0; b < B; ++b) { redo[b] = !ro64[b]; any = any || redo[b]; }
      if (any) {
        RTE_CHECK_CUDA(cudaMemcpyAsync(ws->active.p, redo.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
        RTE_TRY(launch_T(p, MODE_RES, true, x, true, ws->bt.p, ro, true, ws->active.p, st));
      }
    }
  }
  // FP64 true residual (l2, linf) for reporting; not counted as a solver sweep
  if (o->mode == RTE_MODE_FP64 && o->true_residual_check) {
    // the residual buffer already holds b~ - A~ phi for every instance that finished through the
    // check; recompute it for the others (not converged / numeric)
    std::vector<int> redo(B, 0);
    bool any = false;
    for (int b = 0; b < B; ++b) { redo[b] = S[b].status != RTE_OK; any = any || redo[b]; }
    if (any) {
      RTE_CHECK_CUDA(cudaMemcpyAsync(ws->active.p, redo.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
      RTE_TRY(launch_T(p, MODE_RES, true, x, true, ws->bt.p, ws->r.p, true, ws->active.p, st));
    }
  }
  if (o->mode != RTE_MODE_FP64 || o->true_residual_check) {
    const double* rfin = o->mode != RTE_MODE_FP64 ? ws->ro.p : ws->r.p;
    std::vector<int> all1(B, 1);
    RTE_CHECK_CUDA(cudaMemcpyAsync(ws->active.p, all1.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
    k_norm<<<B, 512, 0, st>>>(rfin, p->d_inst.p, ws->active.p, ws->nrm.p);
    count_launch();
    k_norm<<<B, 512, 0, st>>>(ws->bt.p, p->d_inst.p, ws->active.p, ws->beta.p);
    count_launch();
    k_linf<<<B, 512, 0, st>>>(rfin, p->d_inst.p, ws->est.p);
    count_launch();
    std::vector<double> hn(B), hb(B), hl(B);
    RTE_CHECK_CUDA(cudaMemcpyAsync(hn.data(), ws->nrm.p, B * 8, cudaMemcpyDeviceToHost, st));
    RTE_CHECK_CUDA(cudaMemcpyAsync(hb.data(), ws->beta.p, B * 8, cudaMemcpyDeviceToHost, st));
    RTE_CHECK_CUDA(cudaMemcpyAsync(hl.data(), ws->est.p, B * 8, cudaMemcpyDeviceToHost, st));
    RTE_CHECK_CUDA(cudaStreamSynchronize(st));
    for (int b = 0; b < B; ++b) {
      S[b].true_rel_residual = hb[b] > 0 ? hn[b] / hb[b] : 0.0;
      S[b].true_linf_residual = hl[b];
    }
  }
  if (host_out) {
    RTE_CHECK_CUDA(cudaMemcpyAsync(phi, x, p->ntot * 8, cudaMemcpyDeviceToHost, st));
    RTE_CHECK_CUDA(cudaStreamSynchronize(st));
  }
  int ret = RTE_OK;
  for (int b = 0; b < B; ++b) {
    stats[b] = S[b];
    if (S[b].status != RTE_OK && ret == RTE_OK) ret = S[b].status;
  }
  if (ret == RTE_ERR_NOT_CONVERGED) set_error("fgmres_solve: at least one instance missed its tolerance");
  if (ret == RTE_ERR_NUMERIC) set_error("fgmres_solve: NaN/Inf met");
  return ret;
}

// ----------------------------------------------------------------------------------------------- SI-SA
// Source iteration with synthetic acceleration as a preconditioned Richardson iteration (Sec. 3.2, eq.
// preconditioned-richardson): phi <- phi + M_l^{-1} r, r = b~ - A~ phi.  M_l = M_ROM for l <= window on
// instances with a ROM, then the post-window operator (DSA, ROMSAD kept, or none); instances without a ROM
// take the post-window operator from the first iteration when it is DSA, none otherwise.  FP64; every
// iteration ends with a host check of ||r|| / ||b~|| (an FP64 sweep costs far more than the round trip).
extern "C" int si_solve(rte_problem_t p, const romsad_t* roms, const fgmres_opts* o, const void* phi0, void* phi,
                        fgmres_stats* stats, void* stream) {
  RTE_ARG(p && o && phi && stats, "null handle or pointer");
  RTE_ARG(o->rtol > 0.0 && o->max_iter >= 1, "rtol must be > 0 and max_iter >= 1");
  RTE_ARG(o->post_mode == RTE_POST_ROM || o->post_mode == RTE_POST_IDENTITY || o->post_mode == RTE_POST_DSA,
          "unknown post_mode");
  if (o->mode != RTE_MODE_FP64) {
    set_error("si_solve: source iteration runs in FP64 only");
    return RTE_ERR_UNSUPPORTED;
  }
  const bool use_dsa = o->post_mode == RTE_POST_DSA;
  if (use_dsa) {
    RTE_ARG(o->dsa_variant == RTE_DSA_PARTIAL || o->dsa_variant == RTE_DSA_LUMPED || o->dsa_variant == RTE_DSA_FULL,
            "unknown dsa_variant");
    RTE_TRY(dsa_check(p));
  }
  const int B = p->B;
  if (roms)
    for (int b = 0; b < B; ++b)
      if (roms[b]) RTE_TRY(rom_check_mesh(roms[b], p, b));
  cudaStream_t st = (cudaStream_t)stream;
  Ws* ws = get_ws(p);
  RTE_TRY(ws->alloc(p, ws->m > 0 ? ws->m : 1, false));
  RTE_TRY(prepare_sweeps(p));
  cudaPointerAttributes attr;
  bool host_out = false;
  if (cudaPointerGetAttributes(&attr, phi) != cudaSuccess || attr.type == cudaMemoryTypeHost ||
      attr.type == cudaMemoryTypeUnregistered) {
    cudaGetLastError();
    host_out = true;
  }
  double* x;
  if (host_out) {
    RTE_TRY(ws->phi_in.ensure(p->ntot));
    x = ws->phi_in.p;
  } else {
    x = (double*)phi;
  }
  // ROM groups (one factorisation of U^T A_mu U per group)
  std::vector<int> norom(B, 1);
  std::vector<RomPlan> plans;
  bool any_rom = false, any_norom = false;
  if (roms) {
    std::vector<std::pair<romsad_t, int>> groups;
    for (int b = 0; b < B; ++b)
      if (roms[b]) {
        groups.push_back({roms[b], b});
        norom[b] = 0;
      }
    std::sort(groups.begin(), groups.end());
    size_t g0 = 0;
    while (g0 < groups.size()) {
      size_t g1 = g0;
      std::vector<int> ids;
      while (g1 < groups.size() && groups[g1].first == groups[g0].first) ids.push_back(groups[g1++].second);
      plans.emplace_back();
      RTE_TRY(plans.back().build(groups[g0].first, p, ids, st));
      g0 = g1;
    }
  }
  for (int b = 0; b < B; ++b) {
    any_rom = any_rom || !norom[b];
    any_norom = any_norom || norom[b];
  }
  RTE_CHECK_CUDA(cudaMemcpyAsync(ws->norom.p, norom.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
  if (use_dsa) RTE_TRY(dsa_prepare(p, o->dsa_variant, st));
  const dim3 vg = vec_grid(p);
  std::vector<fgmres_stats> S(B);
  for (int b = 0; b < B; ++b) {
    std::memset(&S[b], 0, sizeof(fgmres_stats));
    S[b].sweeps = 1;
    S[b].sweeps_fp64 = 1;
  }
  // b~ and its norm
  RTE_TRY(launch_T(p, MODE_RHS, true, nullptr, true, nullptr, ws->bt.p, true, nullptr, st));
  std::vector<int> act(B, 1), sub(B, 0);
  RTE_CHECK_CUDA(cudaMemcpyAsync(ws->active.p, act.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
  k_norm<<<B, 512, 0, st>>>(ws->bt.p, p->d_inst.p, ws->active.p, ws->bnorm.p);
  count_launch();
  if (phi0) {
    RTE_CHECK_CUDA(cudaMemcpyAsync(x, phi0, p->ntot * 8, cudaMemcpyDeviceToDevice, st));
  } else {
    RTE_CHECK_CUDA(cudaMemsetAsync(x, 0, p->ntot * 8, st));
  }
  std::vector<double> hb(B), hr(B);
  RTE_CHECK_CUDA(cudaMemcpyAsync(hb.data(), ws->bnorm.p, B * 8, cudaMemcpyDeviceToHost, st));
  for (int l = 0;; ++l) {
    // r = b~ - A~ x (r = b~ for a zero start)
    RTE_CHECK_CUDA(cudaMemcpyAsync(ws->active.p, act.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
    if (l == 0 && !phi0) {
      k_copy_active<<<vg, 256, 0, st>>>(ws->r.p, ws->bt.p, p->d_inst.p, ws->active.p);
      count_launch();
    } else {
      RTE_TRY(launch_T(p, MODE_RES, true, x, true, ws->bt.p, ws->r.p, true, ws->active.p, st));
      for (int b = 0; b < B; ++b)
        if (act[b]) {
          ++S[b].sweeps;
          ++S[b].sweeps_fp64;
        }
    }
    k_norm<<<B, 512, 0, st>>>(ws->r.p, p->d_inst.p, ws->active.p, ws->nrm.p);
    count_launch();
    k_linf<<<B, 512, 0, st>>>(ws->r.p, p->d_inst.p, ws->est.p);
    count_launch();
    std::vector<double> hl(B);
    RTE_CHECK_CUDA(cudaMemcpyAsync(hr.data(), ws->nrm.p, B * 8, cudaMemcpyDeviceToHost, st));
    RTE_CHECK_CUDA(cudaMemcpyAsync(hl.data(), ws->est.p, B * 8, cudaMemcpyDeviceToHost, st));
    RTE_CHECK_CUDA(cudaStreamSynchronize(st));
    int nact = 0;
    for (int b = 0; b < B; ++b) {
      if (!act[b]) continue;
      const double rel = hb[b] > 0 ? hr[b] / hb[b] : 0.0;
      S[b].true_rel_residual = S[b].est_rel_residual = rel;
      S[b].true_linf_residual = hl[b];
      if (!std::isfinite(rel)) {
        act[b] = 0;
        S[b].status = RTE_ERR_NUMERIC;
      } else if (rel <= o->rtol) {
        act[b] = 0;
      } else if (S[b].iterations >= o->max_iter) {
        act[b] = 0;
        S[b].status = RTE_ERR_NOT_CONVERGED;
      } else {
        ++nact;
      }
    }
    if (nact == 0) break;
    RTE_CHECK_CUDA(cudaMemcpyAsync(ws->active.p, act.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
    // z = M_l^{-1} r into d
    const bool rom_now = any_rom && (l + 1 <= o->window || o->post_mode == RTE_POST_ROM);
    if (rom_now) {
      for (RomPlan& pl : plans) RTE_TRY(pl.apply(p, ws->active.p, ws->r.p, ws->d.p, true, st));
      if (any_norom) {
        if (use_dsa) {
          RTE_TRY(dsa_launch(p, true, ws->r.p, ws->d.p, ws->active.p, ws->norom.p, st));
        } else {
          for (int b = 0; b < B; ++b) sub[b] = act[b] && norom[b];
          RTE_CHECK_CUDA(cudaMemcpyAsync(ws->list.p, sub.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
          k_copy_active<<<vg, 256, 0, st>>>(ws->d.p, ws->r.p, p->d_inst.p, ws->list.p);
          count_launch();
        }
      }
    } else if (use_dsa) {
      RTE_TRY(dsa_launch(p, true, ws->r.p, ws->d.p, ws->active.p, nullptr, st));
    } else {
      k_copy_active<<<vg, 256, 0, st>>>(ws->d.p, ws->r.p, p->d_inst.p, ws->active.p);
      count_launch();
    }
    k_axpy_active<<<vg, 256, 0, st>>>(x, ws->d.p, p->d_inst.p, ws->active.p);
    count_launch();
    RTE_CHECK_CUDA(cudaGetLastError());
    for (int b = 0; b < B; ++b)
      if (act[b]) ++S[b].iterations;
  }
  if (host_out) {
    RTE_CHECK_CUDA(cudaMemcpyAsync(phi, x, p->ntot * 8, cudaMemcpyDeviceToHost, st));
  }
  RTE_CHECK_CUDA(cudaStreamSynchronize(st));
  int ret = RTE_OK;
  for (int b = 0; b < B; ++b) {
    stats[b] = S[b];
    if (S[b].status != RTE_OK && ret == RTE_OK) ret = S[b].status;
  }
  if (ret == RTE_ERR_NOT_CONVERGED) set_error("si_solve: at least one instance missed its tolerance");
  if (ret == RTE_ERR_NUMERIC) set_error("si_solve: NaN/Inf met");
  return ret;
}
