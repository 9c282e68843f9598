// Transport sweep kernels (paper Sec. 3.1 eq. SI-equation and Sec. 3.2 eq. memory-efficient-SI /
// memory-efficient-rte):
//
//   psi_j = (D_j + Sigma_t)^{-1} s        one block Gauss-Seidel pass in upwind order per direction
//   T s   = sum_j omega_j psi_j            fused: psi is never stored
//   A~ z  = z - T (Sigma_s z)              fused Sigma_s scaling on load, subtraction in the reduce
//
// 2D work decomposition.  A task is (instance, quadrant, chunk of D unique directions); one warp
// runs one task.  Lane l owns mesh rows l, l+32, l+64, ... (rows counted in the upwind y order) and
// marches along its row in the upwind x order.  The 32 rows of a band form a diagonal wavefront:
// lane l handles column i of band k at step k*P + l + i (P = max(nx, 32)), so the y-inflow of a cell
// is the y-outflow its lower neighbour produced one step earlier, received with one warp shuffle;
// the x-inflow is the lane's own previous cell (registers).  Band k+1's first row takes its y-inflow
// from band k's last row through a per-column buffer in shared memory.  Each lane keeps D directions
// in flight per cell (independent dependency chains: instruction-level parallelism), shares the
// cell's source load between them, and accumulates omega_j psi_j in registers.  Every task writes one
// partial scalar flux; a second kernel sums the partials of an instance in a fixed order, so results
// are deterministic and independent of scheduling.
//
// Cell solve.  In the frame reflected so that Omega_x, Omega_y > 0 (odd Legendre modes change
// sign), the cell block is L = alpha K(x)I + beta I(x)K + sigma_t I with K = [[1, sqrt3], [-sqrt3, 3]];
// the right-hand side gets alpha phat_a tx_b + beta phat_b ty_a from the upwind traces, phat =
// (1, -sqrt3), tx_b = psi_0b + sqrt3 psi_1b (x-outflow trace), ty_a = psi_a0 + sqrt3 psi_a1; L^{-1}
// per (instance, direction, region) is precomputed (problem.cu) and staged in shared memory.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "dfloat.cuh"
#include "internal.h"

namespace rte {

struct SweepArgs {
  const InstInfo* inst;
  const UDir* udir;
  const SweepTask* tasks;
  int ntasks;
  const void* linv;     // compute type, [B][nu][R][nd*nd]
  const void* sig_s;    // compute type, [B][R]; null: no Sigma_s scaling of the input
  const void* src;      // input type, scalar vector
  int with_bc;
  int inflow_mask;      // faces carrying the inflow: 1 x-low, 2 x-high, 4 y-low, 8 y-high
  void* partial;        // compute type, [tasks_per_inst * off_b + t * N_b + i]
  int tasks_per_inst;
  void* psi;            // compute type, angular vector, or null
  int ndir, nu, R, rx, ry;
  const int* active;    // [B] or null
  int smem_per_warp;    // elements of the compute type
  int psi_unique;       // angular output: 0 = all N_Omega directions, 1 = one block per unique direction
};

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  __device__ static void load(const float* p, float& a, float& b, float& c, float& d) {
    float4 v = *reinterpret_cast<const float4*>(p);
    a = v.x; b = v.y; c = v.z; d = v.w;
  }
  __device__ static void store(float* p, float a, float b, float c, float d) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
  }
};
template <>
struct Vec4<double> {
  __device__ static void load(const double* p, double& a, double& b, double& c, double& d) {
    double2 v0 = reinterpret_cast<const double2*>(p)[0];
    double2 v1 = reinterpret_cast<const double2*>(p)[1];
    a = v0.x; b = v0.y; c = v1.x; d = v1.y;
  }
  __device__ static void store(double* p, double a, double b, double c, double d) {
    reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
    reinterpret_cast<double2*>(p)[1] = make_double2(c, d);
  }
};

template <>
struct Vec4<dfloat> {
  __device__ static void load(const dfloat* p, dfloat& a, dfloat& b, dfloat& c, dfloat& d) {
    const float4 v0 = reinterpret_cast<const float4*>(p)[0];
    const float4 v1 = reinterpret_cast<const float4*>(p)[1];
    a = dfloat(v0.x, v0.y); b = dfloat(v0.z, v0.w); c = dfloat(v1.x, v1.y); d = dfloat(v1.z, v1.w);
  }
  __device__ static void store(dfloat* p, dfloat a, dfloat b, dfloat c, dfloat d) {
    reinterpret_cast<float4*>(p)[0] = make_float4(a.hi, a.lo, b.hi, b.lo);
    reinterpret_cast<float4*>(p)[1] = make_float4(c.hi, c.lo, d.hi, d.lo);
  }
};

// value of the lane below (lane - 1) in the warp
template <typename T>
__device__ __forceinline__ T shfl_up1(T v) { return __shfl_up_sync(0xffffffffu, v, 1); }
template <>
__device__ __forceinline__ dfloat shfl_up1<dfloat>(dfloat v) {
  return dfloat(__shfl_up_sync(0xffffffffu, v.hi, 1), __shfl_up_sync(0xffffffffu, v.lo, 1));
}

// precision slot of a sweep arithmetic type (autotuner tables, partial-sum element size)
template <typename T>
constexpr int prec_of() { return std::is_same<T, float>::value ? PREC_F32 : (std::is_same<T, double>::value ? PREC_F64 : PREC_DF); }

// Angular output: lane (f's segment, cell e) stores one cell of the completed 8-cell segment of lane f,
// whose current column is colf at cell cf, from f's staging ring to every block of the task's
// directions (offsets ob0/ob1, or the direction table when a direction stands for more than two).
#define RTE_STORE_SEGMENT(f, cf, colf, e)                                                              \
  do {                                                                                                 \
    const int cs_ = (colf) & ~7;                                                                       \
    if ((e) <= (colf) - cs_) {                                                                         \
      const long long cellf_ = (cf) + (sx > 0 ? (cs_ + (e) - (colf)) : ((colf) - cs_ - (e)));          \
      const T* sr_ = ring - (size_t)(lane - (f)) * D * 32;                                             \
      _Pragma("unroll") for (int d = 0; d < D; ++d) {                                                  \
        T v0, v1, v2, v3;                                                                              \
        Vec4<T>::load(sr_ + d * 32 + (e) * 4, v0, v1, v2, v3);                                         \
        if (dup2) {                                                                                    \
          Vec4<T>::store(psi + ob0[d] + 4 * cellf_, v0, v1, v2, v3);                                   \
          if (ob1[d] >= 0) Vec4<T>::store(psi + ob1[d] + 4 * cellf_, v0, v1, v2, v3);                 \
        } else {                                                                                       \
          const UDir u_ = a.udir[tk.u0 + d];                                                           \
          for (int q = 0; q < u_.ndup; ++q)                                                            \
            Vec4<T>::store(psi + (size_t)u_.dup[q] * in.ndof + 4 * cellf_, v0, v1, v2, v3);           \
        }                                                                                              \
      }                                                                                                \
    }                                                                                                  \
  } while (0)

template <typename T, typename TI, int D, bool ANG, bool CELL = false>
__global__ void __launch_bounds__(128) k_sweep2d(SweepArgs a) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int tid = blockIdx.x * wpb + warp;
  if (tid >= a.ntasks) return;
  const SweepTask tk = a.tasks[tid];
  if (a.active && !a.active[tk.b]) return;
  const InstInfo in = a.inst[tk.b];
  const int nx = in.nx, ny = in.ny, R = a.R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tab = reinterpret_cast<T*>(smem_raw) + (size_t)warp * a.smem_per_warp;
  T* ybuf = tab + (CELL ? 0 : D * R * 16);
  T* sgs = ybuf + D * nx * 2;   // sigma_s per region
  // angular-output staging ring: per lane and direction the last 8 cells of its current row
  T* ring = ANG ? reinterpret_cast<T*>(smem_raw) + (size_t)wpb * a.smem_per_warp + ((size_t)warp * 32 + lane) * D * 32
                : nullptr;
  // cross-section profiles (CELL): cell inverses and Sigma_s blocks per cell, read from global memory; else the
  // per-region inverses and sigma_s staged in shared memory
  const long long ncell = (long long)nx * ny, cell0 = in.off / 4;
  const T* linvc = CELL ? reinterpret_cast<const T*>(a.linv) + ((size_t)cell0 * a.nu + (size_t)tk.u0 * ncell) * 16
                        : nullptr;
  const T* sblk = CELL && a.sig_s ? reinterpret_cast<const T*>(a.sig_s) + (size_t)cell0 * 16 : nullptr;
  if (!CELL) {
    const T* linv = reinterpret_cast<const T*>(a.linv) + ((size_t)tk.b * a.nu + tk.u0) * R * 16;
    for (int e = lane; e < D * R * 16; e += 32) tab[e] = linv[e];
    if (a.sig_s)
      for (int e = lane; e < R; e += 32) sgs[e] = reinterpret_cast<const T*>(a.sig_s)[(size_t)tk.b * R + e];
  }
  T al[D], be[D], wg[D];
  const int sx = a.udir[tk.u0].sx, sy = a.udir[tk.u0].sy;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const UDir u = a.udir[tk.u0 + d];
    al[d] = (T)(u.ax / in.hx);
    be[d] = (T)(u.ay / in.hy);
    wg[d] = (T)u.w;
  }
  // inflow traces of the constant g on the task's inflow faces (x face by the sign of Omega_x, y face by that of
  // Omega_y), zero on faces without inflow
  const double gtr = a.with_bc ? in.g * sqrt(in.hx * in.hy) : 0.0;
  const T bndx = (a.inflow_mask & (sx > 0 ? 1 : 2)) ? (T)gtr : (T)0;
  const T bndy = (a.inflow_mask & (sy > 0 ? 4 : 8)) ? (T)gtr : (T)0;
  const bool sig_s = a.sig_s != nullptr;
  const TI* src = reinterpret_cast<const TI*>(a.src) + in.off;
  T* part = reinterpret_cast<T*>(a.partial) + (size_t)a.tasks_per_inst * in.off + (size_t)tk.t * in.ndof;
  T* psi = ANG ? reinterpret_cast<T*>(a.psi) + (size_t)(a.psi_unique ? a.nu : a.ndir) * in.off : nullptr;
  // angular output: element offsets (within the instance) of the blocks each of the task's directions
  // is stored to (its unique block, or the one or two N_Omega blocks it stands for), read once here
  // instead of from the direction table at every flush
  int ob0[D], ob1[D];
  bool dup2 = true;   // every direction stands for at most two stored blocks
  if (ANG) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const UDir u = a.udir[tk.u0 + d];
      if (a.psi_unique) {
        ob0[d] = (tk.u0 + d) * in.ndof;
        ob1[d] = -1;
      } else {
        ob0[d] = u.dup[0] * in.ndof;
        ob1[d] = u.ndup > 1 ? u.dup[1] * in.ndof : -1;
        dup2 = dup2 && u.ndup <= 2;
      }
    }
  }
  // in a mesh whose width is a multiple of 8 the lanes that complete an 8-cell segment at step s are
  // exactly f = (s + 1) mod 8 + 8k, k = 0..3 (lane l works on column s - l modulo the band length)
  const bool regular = (in.nx & 7) == 0 && dup2;
  const T S3 = (T)1.7320508075688772;
  const int P = nx > 32 ? nx : 32;
  const int nbands = (ny + 31) >> 5;
  const int nsteps = (nbands - 1) * P + 31 + nx;
  const int cx = nx / a.rx, cy = ny / a.ry;
  T tx0[D], tx1[D], ty0[D], ty1[D];
#pragma unroll
  for (int d = 0; d < D; ++d) { tx0[d] = tx1[d] = ty0[d] = ty1[d] = (T)0; }
  // Cursor over this lane's cells: (band, col) advance by one column per step; the region index and
  // the cell offset are carried along so the step loop has no integer division.
  struct Cursor {
    int band, col, row, iy, ryb, xr, xrc;   // xr: region column, xrc: column inside it
    long long cell;
  };
  auto cur_init = [&](Cursor& c, int st) {
    const int rel = st - lane;
    c.band = rel >= 0 ? rel / P : 0;
    c.col = rel >= 0 ? rel - c.band * P : rel;   // negative before the lane starts
    c.row = c.band * 32 + lane;
    c.iy = sy > 0 ? c.row : ny - 1 - c.row;
    c.ryb = (c.row < ny ? c.iy / cy : 0) * a.rx;
    const int cc = c.col >= 0 ? c.col : 0;
    const int ix = sx > 0 ? cc : nx - 1 - cc;
    c.xr = ix / cx;
    c.xrc = ix - c.xr * cx;
    c.cell = (long long)c.iy * nx + ix;
  };
  auto cur_valid = [&](const Cursor& c) { return c.col >= 0 && c.col < nx && c.band < nbands && c.row < ny; };
  auto cur_next = [&](Cursor& c) {
    ++c.col;
    if (c.col == P) {      // next band: recompute (rare)
      const int band = c.band + 1;
      c.band = band;
      c.col = 0;
      c.row = band * 32 + lane;
      c.iy = sy > 0 ? c.row : ny - 1 - c.row;
      c.ryb = (c.row < ny ? c.iy / cy : 0) * a.rx;
      const int ix = sx > 0 ? 0 : nx - 1;
      c.xr = ix / cx;
      c.xrc = ix - c.xr * cx;
      c.cell = (long long)c.iy * nx + ix;
      return;
    }
    if (c.col <= 0) {      // the lane has not started yet (or starts now)
      if (c.col == 0) {
        const int ix = sx > 0 ? 0 : nx - 1;
        c.xr = ix / cx;
        c.xrc = ix - c.xr * cx;
        c.cell = (long long)c.iy * nx + ix;
      }
      return;
    }
    if (c.col >= nx) return;   // past the end of the row: idle until the next band
    if (sx > 0) {
      ++c.cell;
      if (++c.xrc == cx) { c.xrc = 0; ++c.xr; }
    } else {
      --c.cell;
      if (--c.xrc < 0) { c.xrc = cx - 1; --c.xr; }
    }
  };
  // Sources are read PF steps ahead into a register ring (their addresses do not depend on the
  // sweep), so the load latency overlaps PF wavefront steps instead of stalling each one.
  constexpr int PF = 4;
  TI q0[PF], q1[PF], q2[PF], q3[PF];
  int qreg[PF];
  Cursor cu, fu;   // cu: current step, fu: step s + PF (prefetch)
  cur_init(cu, 0);
  cur_init(fu, 0);
#pragma unroll
  for (int k = 0; k < PF; ++k) {
    if (cur_valid(fu)) Vec4<TI>::load(src + 4 * fu.cell, q0[k], q1[k], q2[k], q3[k]);
    qreg[k] = fu.ryb + fu.xr;
    cur_next(fu);
  }
  __syncwarp();
  for (int s0 = 0; s0 < nsteps; s0 += PF) {
#pragma unroll
  for (int kk = 0; kk < PF; ++kk) {
    const int s = s0 + kk;
    const bool act = s < nsteps && cur_valid(cu);
    const int col = cu.col, band = cu.band;
    const long long c = cu.cell;
    T s0v = (T)q0[kk], s1 = (T)q1[kk], s2 = (T)q2[kk], s3 = (T)q3[kk];
    const int reg = qreg[kk];
    if (cur_valid(fu)) Vec4<TI>::load(src + 4 * fu.cell, q0[kk], q1[kk], q2[kk], q3[kk]);
    qreg[kk] = fu.ryb + fu.xr;
    cur_next(fu);
    cur_next(cu);
    T yi0[D], yi1[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      yi0[d] = shfl_up1(ty0[d]);
      yi1[d] = shfl_up1(ty1[d]);
    }
    if (act) {
      if (lane == 0) {
        if (band == 0) {
#pragma unroll
          for (int d = 0; d < D; ++d) { yi0[d] = bndy; yi1[d] = (T)0; }
        } else {
#pragma unroll
          for (int d = 0; d < D; ++d) {
            yi0[d] = ybuf[(d * nx + col) * 2];
            yi1[d] = ybuf[(d * nx + col) * 2 + 1];
          }
        }
      }
      if (col == 0) {
#pragma unroll
        for (int d = 0; d < D; ++d) { tx0[d] = bndx; tx1[d] = (T)0; }
      }
      if (CELL && sig_s) {   // Sigma_s q with the cell's block (physical frame, before the reflection)
        T m[16];
        const T* S = sblk + (size_t)c * 16;
        Vec4<T>::load(S, m[0], m[1], m[2], m[3]);
        Vec4<T>::load(S + 4, m[4], m[5], m[6], m[7]);
        Vec4<T>::load(S + 8, m[8], m[9], m[10], m[11]);
        Vec4<T>::load(S + 12, m[12], m[13], m[14], m[15]);
        const T q0v = s0v, q1v = s1, q2v = s2, q3v = s3;
        s0v = m[0] * q0v + m[1] * q1v + m[2] * q2v + m[3] * q3v;
        s1 = m[4] * q0v + m[5] * q1v + m[6] * q2v + m[7] * q3v;
        s2 = m[8] * q0v + m[9] * q1v + m[10] * q2v + m[11] * q3v;
        s3 = m[12] * q0v + m[13] * q1v + m[14] * q2v + m[15] * q3v;
      } else if (sig_s) {
        const T sg = sgs[reg];
        s0v *= sg; s1 *= sg; s2 *= sg; s3 *= sg;
      }
      s1 = sx > 0 ? s1 : -s1;
      s2 = sy > 0 ? s2 : -s2;
      s3 = (sx * sy) > 0 ? s3 : -s3;
      T acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const T ax = al[d], by = be[d];
        const T r0 = s0v + ax * tx0[d] + by * yi0[d];
        const T r1 = s1 - S3 * ax * tx0[d] + by * yi1[d];
        const T r2 = s2 + ax * tx1[d] - S3 * by * yi0[d];
        const T r3 = s3 - S3 * (ax * tx1[d] + by * yi1[d]);
        const T* L = CELL ? linvc + ((size_t)d * ncell + c) * 16 : tab + (d * R + reg) * 16;
        T l[16];
        Vec4<T>::load(L, l[0], l[1], l[2], l[3]);
        Vec4<T>::load(L + 4, l[4], l[5], l[6], l[7]);
        Vec4<T>::load(L + 8, l[8], l[9], l[10], l[11]);
        Vec4<T>::load(L + 12, l[12], l[13], l[14], l[15]);
        const T p0 = l[0] * r0 + l[1] * r1 + l[2] * r2 + l[3] * r3;
        const T p1 = l[4] * r0 + l[5] * r1 + l[6] * r2 + l[7] * r3;
        const T p2 = l[8] * r0 + l[9] * r1 + l[10] * r2 + l[11] * r3;
        const T p3 = l[12] * r0 + l[13] * r1 + l[14] * r2 + l[15] * r3;
        tx0[d] = p0 + S3 * p1;
        tx1[d] = p2 + S3 * p3;
        ty0[d] = p0 + S3 * p2;
        ty1[d] = p1 + S3 * p3;
        acc0 += wg[d] * p0;
        acc1 += wg[d] * p1;
        acc2 += wg[d] * p2;
        acc3 += wg[d] * p3;
        if (lane == 31 && band + 1 < nbands) {
          ybuf[(d * nx + col) * 2] = ty0[d];
          ybuf[(d * nx + col) * 2 + 1] = ty1[d];
        }
        if (ANG) {
          const T q1 = sx > 0 ? p1 : -p1, q2 = sy > 0 ? p2 : -p2, q3 = (sx * sy) > 0 ? p3 : -p3;
          Vec4<T>::store(ring + d * 32 + (col & 7) * 4, p0, q1, q2, q3);
        }
      }
      acc1 = sx > 0 ? acc1 : -acc1;
      acc2 = sy > 0 ? acc2 : -acc2;
      acc3 = (sx * sy) > 0 ? acc3 : -acc3;
      Vec4<T>::store(part + 4 * c, acc0, acc1, acc2, acc3);
    }
    if (ANG) {
      // lanes that completed an aligned 8-cell row segment (or their row) hand it to the warp: lanes
      // 8k..8k+7 store the k-th completed segment, one cell each, i.e. whole 128-byte lines
      const bool flush = act && ((col & 7) == 7 || col == nx - 1);
      const long long myc = act ? c : 0;
      const int mycol = act ? col : 0;
      __syncwarp();
      const int k = lane >> 3, e = lane & 7;
      if (regular) {
        const int f = ((s + 1) & 7) + 8 * k;
        const bool ff = __shfl_sync(0xffffffffu, flush, f);
        const long long cf = __shfl_sync(0xffffffffu, myc, f);
        const int colf = __shfl_sync(0xffffffffu, mycol, f);
        if (ff) RTE_STORE_SEGMENT(f, cf, colf, e);
      } else {
        unsigned fm = __ballot_sync(0xffffffffu, flush);
        while (fm) {
          int fl[4], n = 0;
          while (fm && n < 4) {
            fl[n++] = __ffs(fm) - 1;
            fm &= fm - 1;
          }
          const int f = fl[k < n ? k : 0];
          const long long cf = __shfl_sync(0xffffffffu, myc, f);
          const int colf = __shfl_sync(0xffffffffu, mycol, f);
          if (k < n) RTE_STORE_SEGMENT(f, cf, colf, e);
        }
      }
    }
    __syncwarp();
  }
  }
}

// Band-parallel variant for meshes with ny <= 32 * 8: one CTA per task, warp w owns the 32-row band w
// (lane l owns row 32w + l).  Lane l of band w handles column col = s - (32 + SK) w - l at step s, so the
// y-inflow of a cell is the y-outflow of the lane below one step earlier (warp shuffle) and, for lane 0, the
// y-outflow that the last lane of the band below produced SK + 1 steps earlier (through shared memory).
// Bands are skewed by SK steps so that they need to meet at a CTA barrier only once every SK steps: a
// value read at step s of group m (steps m SK .. m SK + SK - 1) was written at step s - SK - 1, in an
// earlier group, before that group's barrier.  The critical path is the nx + ny - 1 diagonals plus the skew
// of the bands, and a lane's cell index moves by one per step, so the step loop has no division and the
// source prefetch is a plain +-PF offset.
template <typename T, typename TI, int D, bool ANG>
__global__ void __launch_bounds__(256) k_sweep2d_bands(SweepArgs a) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  const int tid = blockIdx.x;
  if (tid >= a.ntasks) return;
  const SweepTask tk = a.tasks[tid];
  if (a.active && !a.active[tk.b]) return;   // uniform for the CTA
  const InstInfo in = a.inst[tk.b];
  const int nx = in.nx, ny = in.ny, R = a.R;
  const int nb = (ny + 31) >> 5;             // bands of this instance (<= nwarps)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tab = reinterpret_cast<T*>(smem_raw);                 // [D][R][16]
  T* sgs = tab + D * R * 16;                                // [R] (4-aligned)
  T* ybuf = sgs + ((R + 3) & ~3);                           // [nwarps-1][D][nx][2]
  int* xreg = reinterpret_cast<int*>(ybuf + (((size_t)(nwarps > 1 ? nwarps - 1 : 1) * D * nx * 2 + 3) & ~(size_t)3));
  // angular output staging: per lane and direction the last 8 cells of its row (a ring), written out
  // as aligned 8-cell (128 B in FP32) row segments by the whole warp
  T* ring = reinterpret_cast<T*>(xreg + ((nx + 3) & ~3)) + ((size_t)warp * 32 + lane) * D * 32;
  const T* linv = reinterpret_cast<const T*>(a.linv) + ((size_t)tk.b * a.nu + tk.u0) * R * 16;
  for (int e = threadIdx.x; e < D * R * 16; e += blockDim.x) tab[e] = linv[e];
  if (a.sig_s)
    for (int e = threadIdx.x; e < R; e += blockDim.x) sgs[e] = reinterpret_cast<const T*>(a.sig_s)[(size_t)tk.b * R + e];
  const int cx = nx / a.rx, cy = ny / a.ry;
  for (int e = threadIdx.x; e < nx; e += blockDim.x) xreg[e] = e / cx;
  T al[D], be[D], wg[D], wg1[D], wg2[D], wg3[D];
  const int sx = a.udir[tk.u0].sx, sy = a.udir[tk.u0].sy;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const UDir u = a.udir[tk.u0 + d];
    al[d] = (T)(u.ax / in.hx);
    be[d] = (T)(u.ay / in.hy);
    wg[d] = (T)u.w;
    // quadrature weights with the reflection signs of the odd modes folded in
    wg1[d] = sx > 0 ? wg[d] : -wg[d];
    wg2[d] = sy > 0 ? wg[d] : -wg[d];
    wg3[d] = sx * sy > 0 ? wg[d] : -wg[d];
  }
  // inflow traces of the constant g on the task's inflow faces (x face by the sign of Omega_x, y face by that of
  // Omega_y), zero on faces without inflow
  const double gtr = a.with_bc ? in.g * sqrt(in.hx * in.hy) : 0.0;
  const T bndx = (a.inflow_mask & (sx > 0 ? 1 : 2)) ? (T)gtr : (T)0;
  const T bndy = (a.inflow_mask & (sy > 0 ? 4 : 8)) ? (T)gtr : (T)0;
  const bool sig_s = a.sig_s != nullptr;
  const TI* src = reinterpret_cast<const TI*>(a.src) + in.off;
  T* part = reinterpret_cast<T*>(a.partial) + (size_t)a.tasks_per_inst * in.off + (size_t)tk.t * in.ndof;
  T* psi = ANG ? reinterpret_cast<T*>(a.psi) + (size_t)(a.psi_unique ? a.nu : a.ndir) * in.off : nullptr;
  // angular output: element offsets (within the instance) of the blocks each of the task's directions
  // is stored to (its unique block, or the one or two N_Omega blocks it stands for), read once here
  // instead of from the direction table at every flush
  int ob0[D], ob1[D];
  bool dup2 = true;   // every direction stands for at most two stored blocks
  if (ANG) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const UDir u = a.udir[tk.u0 + d];
      if (a.psi_unique) {
        ob0[d] = (tk.u0 + d) * in.ndof;
        ob1[d] = -1;
      } else {
        ob0[d] = u.dup[0] * in.ndof;
        ob1[d] = u.ndup > 1 ? u.dup[1] * in.ndof : -1;
        dup2 = dup2 && u.ndup <= 2;
      }
    }
  }
  // in a mesh whose width is a multiple of 8 the lanes that complete an 8-cell segment at step s are
  // exactly f = (s + 1) mod 8 + 8k, k = 0..3 (lane l works on column s - l modulo the band length)
  const bool regular = (in.nx & 7) == 0 && dup2;
  const T S3 = (T)1.7320508075688772;
  const int band = warp;
  const int row = band * 32 + lane;
  const bool rowok = band < nb && row < ny;
  const int iy = sy > 0 ? row : ny - 1 - row;
  const long long rowbase = (long long)(rowok ? iy : 0) * nx;
  const int rowreg = rowok ? (iy / cy) * a.rx : 0;
  constexpr int SK = 8;                        // band skew = steps between CTA barriers (a multiple of 8)
  const int nsteps = (32 + SK) * (nb - 1) + 31 + nx;
  const int col0 = -((32 + SK) * band + lane);      // column at step 0
  auto cell_of = [&](int col) -> long long { return rowbase + (sx > 0 ? col : nx - 1 - col); };
  T tx0[D], tx1[D], ty0[D], ty1[D];
#pragma unroll
  for (int d = 0; d < D; ++d) { tx0[d] = tx1[d] = ty0[d] = ty1[d] = (T)0; }
  constexpr int PF = 8;
  static_assert(PF == SK, "the barrier closes each prefetch group of SK steps");
  TI q0[PF], q1[PF], q2[PF], q3[PF];
#pragma unroll
  for (int k = 0; k < PF; ++k) {
    const int c = col0 + k;
    if (rowok && c >= 0 && c < nx) Vec4<TI>::load(src + 4 * cell_of(c), q0[k], q1[k], q2[k], q3[k]);
  }
  __syncthreads();
  for (int s0 = 0; s0 < nsteps; s0 += PF) {
#pragma unroll
    for (int kk = 0; kk < PF; ++kk) {
      const int s = s0 + kk;
      const int col = col0 + s;
      const bool act = rowok && s < nsteps && col >= 0 && col < nx;
      T s0v = (T)q0[kk], s1 = (T)q1[kk], s2 = (T)q2[kk], s3 = (T)q3[kk];
      {
        const int cn = col + PF;
        if (rowok && cn >= 0 && cn < nx) Vec4<TI>::load(src + 4 * cell_of(cn), q0[kk], q1[kk], q2[kk], q3[kk]);
      }
      T yi0[D], yi1[D];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        yi0[d] = shfl_up1(ty0[d]);
        yi1[d] = shfl_up1(ty1[d]);
      }
      if (act) {
        if (lane == 0) {
          if (band == 0) {
#pragma unroll
            for (int d = 0; d < D; ++d) { yi0[d] = bndy; yi1[d] = (T)0; }
          } else {
            const T* yb = ybuf + (size_t)(band - 1) * D * nx * 2;
#pragma unroll
            for (int d = 0; d < D; ++d) {
              yi0[d] = yb[(d * nx + col) * 2];
              yi1[d] = yb[(d * nx + col) * 2 + 1];
            }
          }
        }
        if (col == 0) {
#pragma unroll
          for (int d = 0; d < D; ++d) { tx0[d] = bndx; tx1[d] = (T)0; }
        }
        const int ix = sx > 0 ? col : nx - 1 - col;
        const long long c = rowbase + ix;
        const int reg = rowreg + xreg[ix];
        if (sig_s) {
          const T sg = sgs[reg];
          s0v *= sg; s1 *= sg; s2 *= sg; s3 *= sg;
        }
        s1 = sx > 0 ? s1 : -s1;
        s2 = sy > 0 ? s2 : -s2;
        s3 = (sx * sy) > 0 ? s3 : -s3;
        T acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const T ax = al[d], by = be[d];
          const T r0 = s0v + ax * tx0[d] + by * yi0[d];
          const T r1 = s1 - S3 * ax * tx0[d] + by * yi1[d];
          const T r2 = s2 + ax * tx1[d] - S3 * by * yi0[d];
          const T r3 = s3 - S3 * (ax * tx1[d] + by * yi1[d]);
          const T* L = tab + (d * R + reg) * 16;
          T l[16];
          Vec4<T>::load(L, l[0], l[1], l[2], l[3]);
          Vec4<T>::load(L + 4, l[4], l[5], l[6], l[7]);
          Vec4<T>::load(L + 8, l[8], l[9], l[10], l[11]);
          Vec4<T>::load(L + 12, l[12], l[13], l[14], l[15]);
          const T p0 = l[0] * r0 + l[1] * r1 + l[2] * r2 + l[3] * r3;
          const T p1 = l[4] * r0 + l[5] * r1 + l[6] * r2 + l[7] * r3;
          const T p2 = l[8] * r0 + l[9] * r1 + l[10] * r2 + l[11] * r3;
          const T p3 = l[12] * r0 + l[13] * r1 + l[14] * r2 + l[15] * r3;
          tx0[d] = p0 + S3 * p1;
          tx1[d] = p2 + S3 * p3;
          ty0[d] = p0 + S3 * p2;
          ty1[d] = p1 + S3 * p3;
          acc0 += wg[d] * p0;
          acc1 += wg1[d] * p1;
          acc2 += wg2[d] * p2;
          acc3 += wg3[d] * p3;
          if (lane == 31 && band + 1 < nb) {
            T* yb = ybuf + (size_t)band * D * nx * 2;
            yb[(d * nx + col) * 2] = ty0[d];
            yb[(d * nx + col) * 2 + 1] = ty1[d];
          }
          if (ANG) {
            const T q1 = sx > 0 ? p1 : -p1, q2 = sy > 0 ? p2 : -p2, q3 = (sx * sy) > 0 ? p3 : -p3;
            Vec4<T>::store(ring + d * 32 + (col & 7) * 4, p0, q1, q2, q3);
          }
        }
        Vec4<T>::store(part + 4 * c, acc0, acc1, acc2, acc3);
      }
      if (ANG) {
        // lanes that completed an aligned 8-cell segment (or their row) hand it to the warp: lanes
        // 8k..8k+7 store the k-th completed segment, one cell each, so every store instruction writes
        // whole 128-byte lines
        const bool flush = act && ((col & 7) == 7 || col == nx - 1);
        __syncwarp();
        const int k = lane >> 3, e = lane & 7;
        // cell of the flushing lane f's current column (its row is band * 32 + f)
        auto cell_at = [&](int f, int colf) -> long long {
          const int rowf = band * 32 + f;
          const int iyf = sy > 0 ? rowf : ny - 1 - rowf;
          return (long long)iyf * nx + (sx > 0 ? colf : nx - 1 - colf);
        };
        if (regular) {
          const int f = ((s + 1) & 7) + 8 * k;
          const bool ff = __shfl_sync(0xffffffffu, flush, f);
          const int colf = s - (32 + SK) * band - f;
          if (ff) {
            const long long cf = cell_at(f, colf);
            RTE_STORE_SEGMENT(f, cf, colf, e);
          }
        } else {
          unsigned fm = __ballot_sync(0xffffffffu, flush);
          while (fm) {
            int fl[4], n = 0;
            while (fm && n < 4) {
              fl[n++] = __ffs(fm) - 1;
              fm &= fm - 1;
            }
            if (k < n) {
              const int f = fl[k];
              const int colf = s - (32 + SK) * band - f;
              const long long cf = cell_at(f, colf);
              RTE_STORE_SEGMENT(f, cf, colf, e);
            }
          }
        }
        __syncwarp();
      }
      // the bands meet once per group of SK steps (PF == SK: the last step of the prefetch group)
      if (nwarps > 1 && kk == PF - 1) __syncthreads();
      else __syncwarp();
    }
  }
}

// Pipelined band variant (operator apply only): a persistent CTA sweeps a run of tasks on meshes of one size
// back to back.  In the band kernel a band works only while the wavefront crosses its 32 rows, about half of the
// sweep on an 8-band mesh.  Here band w starts task k at step k P + (32 + SK) w, so a band that has finished its
// rows of task k goes straight on to task k + 1 while the bands above it still work on task k.  Run = (first
// task, tasks, period P); the CTA first drops the tasks of inactive instances.  Task k uses table buffer k & 1,
// loaded during the barrier group before band 0 starts it; the host picks P (a multiple of SK) with
// 2 P >= (32 + SK)(nb - 1) + nx + 40, so the buffer's previous task has left every band by then.  The y-outflow
// buffer between bands needs no second copy: band w writes column c of task k + 1 long after band w + 1 has read
// column c of task k.  A lane's shuffle partner (the lane below) is always on the same task and column.
template <typename T, typename TI, int D>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && D <= 4) ? 2 : 1) k_sweep2d_pipe(SweepArgs a, const int4* runs) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  const int4 run = runs[blockIdx.x];   // (first task, tasks, period, 0)
  const int t0 = run.x, P = run.z;
  constexpr int SK = 8, PF = 8;
  constexpr int KMAX = 64;
  __shared__ int klist[KMAX];          // the run's tasks whose instance is active
  __shared__ int kcount;
  if (threadIdx.x == 0) {
    int n = 0;
    for (int k = 0; k < run.y && k < KMAX; ++k) {
      const int b = a.tasks[t0 + k].b;
      if (!a.active || a.active[b]) klist[n++] = t0 + k;
    }
    kcount = n;
  }
  __syncthreads();
  const int K = kcount;
  if (K == 0) return;
  const InstInfo in0 = a.inst[a.tasks[klist[0]].b];
  const int nx = in0.nx, ny = in0.ny, R = a.R;
  const int nb = (ny + 31) >> 5;
  const int R4 = (R + 3) & ~3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tab = reinterpret_cast<T*>(smem_raw);                  // [2][D][R][16]
  T* sgs = tab + 2 * D * R * 16;                             // [2][R4]
  T* ybuf = sgs + 2 * R4;                                    // [nwarps-1][D][nx][2]
  int* xreg = reinterpret_cast<int*>(ybuf + (((size_t)(nwarps > 1 ? nwarps - 1 : 1) * D * nx * 2 + 3) & ~(size_t)3));
  const int cx = nx / a.rx, cy = ny / a.ry;
  for (int e = threadIdx.x; e < nx; e += blockDim.x) xreg[e] = e / cx;
  // per-task parameters, computed once per task by the loading threads (the FP64 divisions of the direction
  // coefficients must not run once per lane): coefficients, inflow traces, signs, partial-flux offset
  __shared__ T s_al[2][D], s_be[2][D], s_wg[2][D], s_bnd[2][2];
  __shared__ int s_sgn[2][2];
  __shared__ long long s_poff[2];
  auto load_table = [&](int k) {
    const SweepTask tk = a.tasks[klist[k]];
    const int bf = k & 1;
    const T* linv = reinterpret_cast<const T*>(a.linv) + ((size_t)tk.b * a.nu + tk.u0) * R * 16;
    T* dst = tab + (size_t)bf * D * R * 16;
    for (int e = threadIdx.x; e < D * R * 16; e += blockDim.x) dst[e] = linv[e];
    if (a.sig_s)
      for (int e = threadIdx.x; e < R; e += blockDim.x)
        sgs[bf * R4 + e] = reinterpret_cast<const T*>(a.sig_s)[(size_t)tk.b * R + e];
    if (threadIdx.x < D) {
      const InstInfo in = a.inst[tk.b];
      const UDir u = a.udir[tk.u0 + threadIdx.x];
      s_al[bf][threadIdx.x] = (T)(u.ax / in.hx);
      s_be[bf][threadIdx.x] = (T)(u.ay / in.hy);
      s_wg[bf][threadIdx.x] = (T)u.w;
    } else if (threadIdx.x == D) {
      const InstInfo in = a.inst[tk.b];
      const int tsx = a.udir[tk.u0].sx, tsy = a.udir[tk.u0].sy;
      const double gtr = a.with_bc ? in.g * sqrt(in.hx * in.hy) : 0.0;
      s_bnd[bf][0] = (a.inflow_mask & (tsx > 0 ? 1 : 2)) ? (T)gtr : (T)0;
      s_bnd[bf][1] = (a.inflow_mask & (tsy > 0 ? 4 : 8)) ? (T)gtr : (T)0;
      s_sgn[bf][0] = tsx;
      s_sgn[bf][1] = tsy;
      s_poff[bf] = (long long)a.tasks_per_inst * in.off + (long long)tk.t * in.ndof;
    }
  };
  load_table(0);
  __syncthreads();
  const bool sig_s = a.sig_s != nullptr;
  const T S3 = (T)1.7320508075688772;
  const int band = warp;
  const int row = band * 32 + lane;
  const bool rowok = band < nb && row < ny;
  const int nsteps = (K - 1) * P + (32 + SK) * (nb - 1) + 31 + nx;
  // state of the task the lane works on (k) and of the task its prefetch cursor is in (kp)
  int k = -1, col = -((32 + SK) * band + lane) - 1;   // advanced to step 0 below
  int kp = -1, colp = col + PF;
  T al[D], be[D], wg[D];
  T bndx = (T)0, bndy = (T)0;
  int sx = 1, sy = 1, rowreg = 0;
  long long rowbase = 0;
  T* part = nullptr;
  const TI* srcp = nullptr;   // prefetch task's source
  long long rowbase_p = 0;
  int sxp = 1;
#pragma unroll
  for (int d = 0; d < D; ++d) { al[d] = be[d] = wg[d] = (T)0; }
  auto enter_task = [&](int kk) {   // the lane's current task becomes kk (its parameters are in buffer kk & 1)
    const int bf = kk & 1;
    sx = s_sgn[bf][0];
    sy = s_sgn[bf][1];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      al[d] = s_al[bf][d];
      be[d] = s_be[bf][d];
      wg[d] = s_wg[bf][d];
    }
    bndx = s_bnd[bf][0];
    bndy = s_bnd[bf][1];
    const int iy = sy > 0 ? row : ny - 1 - row;
    rowbase = (long long)(rowok ? iy : 0) * nx;
    rowreg = rowok ? (iy / cy) * a.rx : 0;
    part = reinterpret_cast<T*>(a.partial) + s_poff[bf];
  };
  auto enter_prefetch = [&](int kk) {
    const SweepTask tk = a.tasks[klist[kk]];
    const InstInfo in = a.inst[tk.b];
    sxp = a.udir[tk.u0].sx;
    const int syp = a.udir[tk.u0].sy;
    const int iy = syp > 0 ? row : ny - 1 - row;
    rowbase_p = (long long)(rowok ? iy : 0) * nx;
    srcp = reinterpret_cast<const TI*>(a.src) + in.off;
  };
  // advance a (task, column) cursor by one step; returns true when it enters a new task
  auto step_cursor = [&](int& kk, int& cc) -> bool {
    ++cc;
    if (kk < 0) {
      if (cc == 0) { kk = 0; return true; }
      return false;
    }
    if (cc == P) {
      cc = 0;
      ++kk;
      return kk < K;
    }
    return false;
  };
  TI q0[PF], q1[PF], q2[PF], q3[PF];
  // fill the prefetch ring with the sources of steps 0 .. PF-1; the cursor then stands at step PF-1
  {
    int kq = -1, cq = col;   // the state before step 0
#pragma unroll
    for (int j = 0; j < PF; ++j) {
      if (step_cursor(kq, cq) && kq < K) enter_prefetch(kq);
      if (rowok && kq >= 0 && kq < K && cq < nx)
        Vec4<TI>::load(srcp + 4 * (rowbase_p + (sxp > 0 ? cq : nx - 1 - cq)), q0[j], q1[j], q2[j], q3[j]);
    }
    kp = kq;
    colp = cq;
  }
  T tx0[D], tx1[D], ty0[D], ty1[D];
#pragma unroll
  for (int d = 0; d < D; ++d) { tx0[d] = tx1[d] = ty0[d] = ty1[d] = (T)0; }
  for (int s0 = 0; s0 < nsteps; s0 += PF) {
    // the task that band 0 starts at the next group: its table goes into buffer (k & 1) now
    if ((s0 + PF) % P == 0) {
      const int kn = (s0 + PF) / P;
      if (kn < K) load_table(kn);
    }
#pragma unroll
    for (int kk = 0; kk < PF; ++kk) {
      const int s = s0 + kk;
      if (step_cursor(k, col) && k < K) enter_task(k);
      const bool act = rowok && s < nsteps && k >= 0 && k < K && col < nx;
      T s0v = (T)q0[kk], s1 = (T)q1[kk], s2 = (T)q2[kk], s3 = (T)q3[kk];
      if (step_cursor(kp, colp) && kp < K) enter_prefetch(kp);
      if (rowok && kp >= 0 && kp < K && colp < nx)
        Vec4<TI>::load(srcp + 4 * (rowbase_p + (sxp > 0 ? colp : nx - 1 - colp)), q0[kk], q1[kk], q2[kk], q3[kk]);
      T yi0[D], yi1[D];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        yi0[d] = shfl_up1(ty0[d]);
        yi1[d] = shfl_up1(ty1[d]);
      }
      if (act) {
        const int buf = k & 1;
        if (lane == 0) {
          if (band == 0) {
#pragma unroll
            for (int d = 0; d < D; ++d) { yi0[d] = bndy; yi1[d] = (T)0; }
          } else {
            const T* yb = ybuf + (size_t)(band - 1) * D * nx * 2;
#pragma unroll
            for (int d = 0; d < D; ++d) {
              yi0[d] = yb[(d * nx + col) * 2];
              yi1[d] = yb[(d * nx + col) * 2 + 1];
            }
          }
        }
        if (col == 0) {
#pragma unroll
          for (int d = 0; d < D; ++d) { tx0[d] = bndx; tx1[d] = (T)0; }
        }
        const int ix = sx > 0 ? col : nx - 1 - col;
        const long long c = rowbase + ix;
        const int reg = rowreg + xreg[ix];
        if (sig_s) {
          const T sg = sgs[buf * R4 + reg];
          s0v *= sg; s1 *= sg; s2 *= sg; s3 *= sg;
        }
        s1 = sx > 0 ? s1 : -s1;
        s2 = sy > 0 ? s2 : -s2;
        s3 = (sx * sy) > 0 ? s3 : -s3;
        T acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
        const T* tb = tab + (size_t)buf * D * R * 16;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const T ax = al[d], by = be[d];
          const T r0 = s0v + ax * tx0[d] + by * yi0[d];
          const T r1 = s1 - S3 * ax * tx0[d] + by * yi1[d];
          const T r2 = s2 + ax * tx1[d] - S3 * by * yi0[d];
          const T r3 = s3 - S3 * (ax * tx1[d] + by * yi1[d]);
          const T* L = tb + (d * R + reg) * 16;
          T l[16];
          Vec4<T>::load(L, l[0], l[1], l[2], l[3]);
          Vec4<T>::load(L + 4, l[4], l[5], l[6], l[7]);
          Vec4<T>::load(L + 8, l[8], l[9], l[10], l[11]);
          Vec4<T>::load(L + 12, l[12], l[13], l[14], l[15]);
          const T p0 = l[0] * r0 + l[1] * r1 + l[2] * r2 + l[3] * r3;
          const T p1 = l[4] * r0 + l[5] * r1 + l[6] * r2 + l[7] * r3;
          const T p2 = l[8] * r0 + l[9] * r1 + l[10] * r2 + l[11] * r3;
          const T p3 = l[12] * r0 + l[13] * r1 + l[14] * r2 + l[15] * r3;
          tx0[d] = p0 + S3 * p1;
          tx1[d] = p2 + S3 * p3;
          ty0[d] = p0 + S3 * p2;
          ty1[d] = p1 + S3 * p3;
          acc0 += wg[d] * p0;
          acc1 += wg[d] * p1;
          acc2 += wg[d] * p2;
          acc3 += wg[d] * p3;
          if (lane == 31 && band + 1 < nb) {
            T* yb = ybuf + (size_t)band * D * nx * 2;
            yb[(d * nx + col) * 2] = ty0[d];
            yb[(d * nx + col) * 2 + 1] = ty1[d];
          }
        }
        // odd modes back from the reflected frame (the task's directions share its quadrant)
        acc1 = sx > 0 ? acc1 : -acc1;
        acc2 = sy > 0 ? acc2 : -acc2;
        acc3 = (sx * sy) > 0 ? acc3 : -acc3;
        Vec4<T>::store(part + 4 * c, acc0, acc1, acc2, acc3);
      }
      if (nwarps > 1 && kk == PF - 1) __syncthreads();
      else __syncwarp();
    }
  }
}

// 1D slab (P1, 2 dofs per cell): one thread per (instance, direction) marches its chain.
template <typename T, typename TI, bool ANG>
__global__ void k_sweep1d(SweepArgs a) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= a.ntasks) return;
  const SweepTask tk = a.tasks[tid];
  if (a.active && !a.active[tk.b]) return;
  const InstInfo in = a.inst[tk.b];
  const UDir u = a.udir[tk.u0];
  const int nx = in.nx, R = a.R, cx = nx / a.rx;
  const T al = (T)(u.ax / in.hx), wg = (T)u.w;
  const T S3 = (T)1.7320508075688772;
  const T* linv = reinterpret_cast<const T*>(a.linv) + ((size_t)tk.b * a.nu + tk.u0) * R * 4;
  const T* sig_s = a.sig_s ? reinterpret_cast<const T*>(a.sig_s) + (size_t)tk.b * R : nullptr;
  const TI* src = reinterpret_cast<const TI*>(a.src) + in.off;
  T* part = reinterpret_cast<T*>(a.partial) + (size_t)a.tasks_per_inst * in.off + (size_t)tk.t * in.ndof;
  T* psi = ANG ? reinterpret_cast<T*>(a.psi) + (size_t)(a.psi_unique ? a.nu : a.ndir) * in.off +
                     (size_t)(a.psi_unique ? tk.u0 : u.dup[0]) * in.ndof
                : nullptr;
  T tx = a.with_bc && (a.inflow_mask & (u.sx > 0 ? 1 : 2)) ? (T)(in.g * sqrt(in.hx)) : (T)0;
  for (int col = 0; col < nx; ++col) {
    const int ix = u.sx > 0 ? col : nx - 1 - col;
    const int reg = ix / cx;
    T s0 = (T)src[2 * ix], s1 = (T)src[2 * ix + 1];
    if (sig_s) { s0 *= sig_s[reg]; s1 *= sig_s[reg]; }
    s1 = u.sx > 0 ? s1 : -s1;
    const T r0 = s0 + al * tx, r1 = s1 - S3 * al * tx;
    const T* L = linv + reg * 4;
    const T p0 = L[0] * r0 + L[1] * r1, p1 = L[2] * r0 + L[3] * r1;
    tx = p0 + S3 * p1;
    const T q1 = u.sx > 0 ? p1 : -p1;
    part[2 * ix] = wg * p0;
    part[2 * ix + 1] = wg * q1;
    if (ANG) { psi[2 * ix] = p0; psi[2 * ix + 1] = q1; }
  }
}

// out = sum_t partial[t]  (mode T),  z - sum (mode OP),  b - (z - sum) (mode RES); one instance per blockIdx.y.
template <typename TP, typename TZ, typename TO>
__global__ void k_reduce(const TP* partial, int ntask, const InstInfo* inst, int mode, const TZ* z, const TO* bvec,
                         TO* out, const int* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const InstInfo in = inst[b];
  const TP* pp = partial + (size_t)ntask * in.off;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < in.ndof; i += gridDim.x * blockDim.x) {
    TP s = 0;
    for (int t = 0; t < ntask; ++t) s += pp[(size_t)t * in.ndof + i];
    TO v = (TO)s;
    if (mode == MODE_OP) v = (TO)z[in.off + i] - v;
    if (mode == MODE_RES) v = bvec[in.off + i] - ((TO)z[in.off + i] - v);
    out[in.off + i] = v;
  }
}

// phi = sum_j omega_j psi_j from an angular vector (K3).
template <typename T>
__global__ void k_scalar_flux(const T* psi, const double* w, int ndir, const InstInfo* inst, T* phi) {
  const int b = blockIdx.y;
  const InstInfo in = inst[b];
  const T* pb = psi + (size_t)ndir * in.off;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < in.ndof; i += gridDim.x * blockDim.x) {
    T s = 0;
    for (int j = 0; j < ndir; ++j) s += (T)w[j] * pb[(size_t)j * in.ndof + i];
    phi[in.off + i] = s;
  }
}


// Forward operator y = (D_u + sigma_t) x for one unique direction u (no inflow-boundary term, as in
// the definition of D_j, Sec. 2.3): in the reflected frame y' = L0 x' - alpha phat_a tx_b(x'_up)
// - beta phat_b ty_a(x'_down) + sigma_t x', L0 = alpha K(x)I + beta I(x)K.  One thread per
// (cell, column); columns x[col*ldx + i], y[col*ldy + i].  sig_t: per-region array or null (= 0).
__global__ void k_forward(int dim, int nx, int ny, double hx, double hy, UDir u, int rx, int ry,
                          const double* sig_t, const double* x, long long ldx, double* y, long long ldy, int ncol) {
  const long long ncell = (long long)nx * ny;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= ncell * ncol) return;
  const int col = (int)(tid / ncell);
  const long long c = tid % ncell;
  const int ix = (int)(c % nx), iy = (int)(c / nx);
  const double S3 = 1.7320508075688772;
  const int reg = (iy / (ny / ry)) * rx + ix / (nx / rx);
  const double sg = sig_t ? sig_t[reg] : 0.0;
  const double* xc = x + col * ldx;
  double* yc = y + col * ldy;
  if (dim == 1) {
    const double al = u.ax / hx;
    const double f1 = u.sx > 0 ? 1.0 : -1.0;
    double x0 = xc[2 * c], x1 = f1 * xc[2 * c + 1];
    double y0 = al * (x0 + S3 * x1), y1 = al * (-S3 * x0 + 3.0 * x1);
    const int iup = ix - u.sx;
    if (iup >= 0 && iup < nx) {
      double t = xc[2 * iup] + S3 * f1 * xc[2 * iup + 1];
      y0 -= al * t;
      y1 += S3 * al * t;
    }
    yc[2 * c] = y0 + sg * xc[2 * c];
    yc[2 * c + 1] = f1 * y1 + sg * xc[2 * c + 1];
    return;
  }
  const double al = u.ax / hx, be = u.ay / hy;
  const double fx = u.sx > 0 ? 1.0 : -1.0, fy = u.sy > 0 ? 1.0 : -1.0;
  double v[4] = {xc[4 * c], fx * xc[4 * c + 1], fy * xc[4 * c + 2], fx * fy * xc[4 * c + 3]};
  const double K[4] = {1.0, S3, -S3, 3.0};
  double o[4];
  for (int k = 0; k < 4; ++k) {
    int a = k & 1, b = k >> 1;
    double s = 0.0;
    for (int cc = 0; cc < 2; ++cc) s += al * K[a * 2 + cc] * v[cc + 2 * b];
    for (int d = 0; d < 2; ++d) s += be * K[b * 2 + d] * v[a + 2 * d];
    o[k] = s;
  }
  const int ixu = ix - u.sx, iyu = iy - u.sy;
  if (ixu >= 0 && ixu < nx) {
    const double* n = xc + 4 * ((long long)iy * nx + ixu);
    double t0 = n[0] + S3 * fx * n[1], t1 = fy * n[2] + S3 * fx * fy * n[3];
    o[0] -= al * t0; o[1] += S3 * al * t0; o[2] -= al * t1; o[3] += S3 * al * t1;
  }
  if (iyu >= 0 && iyu < ny) {
    const double* n = xc + 4 * ((long long)iyu * nx + ix);
    double t0 = n[0] + S3 * fy * n[2], t1 = fx * n[1] + S3 * fx * fy * n[3];
    o[0] -= be * t0; o[2] += S3 * be * t0; o[1] -= be * t1; o[3] += S3 * be * t1;
  }
  yc[4 * c] = o[0] + sg * xc[4 * c];
  yc[4 * c + 1] = fx * o[1] + sg * xc[4 * c + 1];
  yc[4 * c + 2] = fy * o[2] + sg * xc[4 * c + 2];
  yc[4 * c + 3] = fx * fy * o[3] + sg * xc[4 * c + 3];
}

int launch_forward_cols(int dim, int nx, int ny, double hx, double hy, const UDir& u, int rx, int ry,
                        const double* sig_t_reg, const double* x, long long ldx, double* y, long long ldy, int ncol,
                        cudaStream_t st) {
  long long total = (long long)nx * ny * ncol;
  if (total == 0) return RTE_OK;
  k_forward<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(dim, nx, ny, hx, hy, u, rx, ry, sig_t_reg, x, ldx, y,
                                                             ldy, ncol);
  count_launch();
  RTE_CHECK_CUDA(cudaGetLastError());
  return RTE_OK;
}

// ----------------------------------------------------------------- host side
static int pick_D(const rte_problem* p, int prec, bool ang = false) {
  if (p->dim == 1) return 1;
  if (p->force_D > 0) return p->force_D;
  if (p->pin_D > 0 && (p->dim == 1 || quadrant_gcd(p) % p->pin_D == 0)) return p->pin_D;
  if (p->tuned_D[prec][ang ? 1 : 0] > 0) return p->tuned_D[prec][ang ? 1 : 0];
  const bool f64 = prec != PREC_F32;
  const int nq = quadrant_gcd(p);
  // Directions per warp: the largest D that still leaves at least 8 warps per SM (152 SMs) in
  // flight; with fewer tasks (a single small instance) parallelism wins and D = 1.  FP64 keeps D
  // small (registers; its pipe, not latency, bounds it).
  const int cands64[] = {4, 2, 1};
  const int cands32[] = {8, 4, 2, 1};
  const long long target = 152LL * 8;
  const int* c = f64 ? cands64 : cands32;
  const int nc = f64 ? 3 : 4;
  for (int k = 0; k < nc; ++k) {
    const int d = c[k];
    if (nq % d) continue;
    const long long ntasks = (long long)p->B * 4 * (nq / d);
    if (ntasks >= target) return d;
  }
  return 1;
}

static int ensure_tasks(rte_problem* p, int D) {
  if (D < 1 || D > 16) {
    set_error("sweep: directions per warp out of range");
    return RTE_ERR_UNSUPPORTED;
  }
  if (!p->d_tasks_by_D[D].p) {
    std::vector<SweepTask> tasks;
    int per_inst = 0;
    if (p->dim == 1) {
      per_inst = p->nu;
      for (int b = 0; b < p->B; ++b)
        for (int u = 0; u < p->nu; ++u) tasks.push_back(SweepTask{b, u, u, 0});
    } else {
      const int nquad = 4;
      for (int q = 0; q < nquad; ++q) per_inst += (p->quad_start[q + 1] - p->quad_start[q]) / D;
      for (int b = 0; b < p->B; ++b) {
        int t = 0;
        for (int q = 0; q < nquad; ++q)
          for (int u0 = p->quad_start[q]; u0 < p->quad_start[q + 1]; u0 += D) tasks.push_back(SweepTask{b, u0, t++, 0});
      }
      // longest tasks first (instances with the most cells): a static longest-processing-time order
      std::stable_sort(tasks.begin(), tasks.end(), [&](const SweepTask& x, const SweepTask& y) {
        return (long long)p->nx[x.b] * p->ny[x.b] > (long long)p->nx[y.b] * p->ny[y.b];
      });
    }
    RTE_TRY(p->d_tasks_by_D[D].alloc(tasks.size()));
    RTE_CHECK_CUDA(cudaMemcpy(p->d_tasks_by_D[D].p, tasks.data(), tasks.size() * sizeof(SweepTask),
                              cudaMemcpyHostToDevice));
    p->ntasks_by_D[D] = (int)tasks.size();
    p->per_inst_by_D[D] = per_inst;
  }
  p->tasks_D = D;
  p->ntasks = p->ntasks_by_D[D];
  p->tasks_per_inst = p->per_inst_by_D[D];
  return RTE_OK;
}

// Dynamic shared memory above the 48 KB default must be granted per kernel with cudaFuncSetAttribute, which
// acts on the current device only; granted[dev] remembers the size already granted on each device (zero-
// initialised statics), so a process that drives several GPUs grants it on each of them.
constexpr int kMaxDevices = 64;
template <typename K>
static int grant_smem(K kern, size_t smem, std::atomic<size_t>* granted) {
  if (smem <= 48 * 1024) return RTE_OK;
  int dev = 0;
  RTE_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("sweep: device ordinal beyond the supported range");
    return RTE_ERR_UNSUPPORTED;
  }
  if (smem > granted[dev].load(std::memory_order_acquire)) {
    RTE_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    granted[dev].store(smem, std::memory_order_release);
  }
  return RTE_OK;
}

// Runs of the pipelined band kernel for the task list of D directions per warp (the order of ensure_tasks):
// consecutive tasks on meshes of one size, at most K each, K chosen so that the runs fill about two CTAs per SM
// once.  Period P of a run: a multiple of 8 with P >= nx and 2 P >= 40 (nb - 1) + nx + 40 (the table buffer of
// task k - 2 is free when task k's table is loaded; see k_sweep2d_pipe).
static int ensure_runs(rte_problem* p, int D) {
  if (p->nruns_by_D[D] > 0) return RTE_OK;
  const int nt = p->ntasks_by_D[D];
  std::vector<SweepTask> tasks(nt);
  RTE_CHECK_CUDA(cudaMemcpy(tasks.data(), p->d_tasks_by_D[D].p, nt * sizeof(SweepTask), cudaMemcpyDeviceToHost));
  int dev = 0, sms = 0;
  RTE_CHECK_CUDA(cudaGetDevice(&dev));
  RTE_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int target = std::max(1, 2 * sms);
  const int K = p->pin_run > 0 ? p->pin_run : std::min(64, std::max(1, (nt + target - 1) / target));
  std::vector<int4> runs;
  for (int i = 0; i < nt;) {
    const int nx = p->nx[tasks[i].b], ny = p->ny[tasks[i].b];
    int j = i;
    while (j < nt && j - i < K && p->nx[tasks[j].b] == nx && p->ny[tasks[j].b] == ny) ++j;
    const int nb = (ny + 31) / 32;
    int P = std::max(std::max(nx, 24), (40 * (nb - 1) + nx + 40 + 1) / 2);
    P = (P + 7) & ~7;
    runs.push_back(make_int4(i, j - i, P, 0));
    i = j;
  }
  RTE_TRY(p->d_runs_by_D[D].alloc(runs.size()));
  RTE_CHECK_CUDA(cudaMemcpy(p->d_runs_by_D[D].p, runs.data(), runs.size() * sizeof(int4), cudaMemcpyHostToDevice));
  p->nruns_by_D[D] = (int)runs.size();
  return RTE_OK;
}

template <typename T, typename TI, bool ANG>
static int launch_sweep_t(rte_problem* p, int D, SweepArgs& a, cudaStream_t st) {
  if (p->dim == 1) {
    int threads = 128;
    k_sweep1d<T, TI, ANG><<<(a.ntasks + threads - 1) / threads, threads, 0, st>>>(a);
    count_launch();
    RTE_CHECK_CUDA(cudaGetLastError());
    return RTE_OK;
  }
  int maxnx = 0, maxny = 0;
  for (int b = 0; b < p->B; ++b) {
    maxnx = std::max(maxnx, p->nx[b]);
    maxny = std::max(maxny, p->ny[b]);
  }
  const int nbands = (maxny + 31) / 32;
  // The band kernel shortens the critical path (latency-bound launches, FP32); for FP64 launches with
  // enough tasks to fill the GPU the FP64 pipe is the limit and the warp-per-task kernel keeps more
  // warps per SM (no idle band warps on smaller meshes of a mixed batch).
  const bool throughput = a.ntasks >= 152 * 8;
  const bool fp64_throughput = sizeof(T) == 8 && throughput;   // FP64 or double-float
  // angular output with many tasks: independent warps (no per-step CTA barrier) hide the store latency
  const bool ang_throughput = ANG && throughput;
  const int tv = p->force_var >= 0 ? p->force_var
                                    : (p->pin_var >= 0 ? p->pin_var : p->tuned_var[prec_of<T>()][ANG ? 1 : 0]);
  if (p->cellsig) {
    // cross-section profiles: the warp-per-task kernel reads the cell inverses and Sigma_s blocks from global memory
    if constexpr (std::is_same<T, dfloat>::value) {
      set_error("sweep: no double-float sweep with cross-section profiles");
      return RTE_ERR_UNSUPPORTED;
    } else {
      a.smem_per_warp = ((D * maxnx * 2 + 1) + 3) & ~3;
      const size_t per_warp = (size_t)a.smem_per_warp * sizeof(T) + (ANG ? (size_t)32 * D * 32 * sizeof(T) : 0);
      int wpb = 4;
      while (wpb > 1 && per_warp * wpb > 96 * 1024) --wpb;
      const size_t smem = per_warp * wpb;
      if (smem > 227 * 1024) {
        set_error("sweep: shared memory too large for this mesh");
        return RTE_ERR_UNSUPPORTED;
      }
      const int blocks = (a.ntasks + wpb - 1) / wpb;
#define RTE_CELL_CASE(DD)                                                                                   \
  case DD: {                                                                                                \
    auto kern = k_sweep2d<T, TI, DD, ANG, true>;                                                            \
    static std::atomic<size_t> granted[kMaxDevices];                                                        \
    RTE_TRY(grant_smem(kern, smem, granted));                                                               \
    kern<<<blocks, wpb * 32, smem, st>>>(a);                                                                \
    count_launch();                                                                                         \
    break;                                                                                                  \
  }
      switch (D) {
        RTE_CELL_CASE(1)
        RTE_CELL_CASE(2)
        RTE_CELL_CASE(4)
        RTE_CELL_CASE(8)
        default:
          set_error("sweep: unsupported directions-per-warp");
          return RTE_ERR_UNSUPPORTED;
      }
#undef RTE_CELL_CASE
      RTE_CHECK_CUDA(cudaGetLastError());
      return RTE_OK;
    }
  }
  if constexpr (!ANG) {
    if (tv == 2 && nbands <= 8) {
      // pipelined band kernel: persistent CTAs over runs of tasks
      RTE_TRY(ensure_runs(p, D));
      const int W = nbands;
      size_t elems = (size_t)2 * D * p->R * 16 + 2 * (size_t)((p->R + 3) & ~3) +
                     (((size_t)(W > 1 ? W - 1 : 1) * D * maxnx * 2 + 3) & ~(size_t)3);
      size_t smem = elems * sizeof(T) + (size_t)((maxnx + 3) & ~3) * sizeof(int) + 16;
      if (smem > 227 * 1024) {
        set_error("sweep: shared-memory table too large for the pipelined kernel");
        return RTE_ERR_UNSUPPORTED;
      }
#define RTE_PIPE_CASE(DD)                                                                                   \
  case DD: {                                                                                                \
    auto kern = k_sweep2d_pipe<T, TI, DD>;                                                                  \
    static std::atomic<size_t> granted[kMaxDevices];                                                        \
    RTE_TRY(grant_smem(kern, smem, granted));                                                               \
    kern<<<p->nruns_by_D[D], W * 32, smem, st>>>(a, p->d_runs_by_D[D].p);                                   \
    count_launch();                                                                                         \
    break;                                                                                                  \
  }
      switch (D) {
        RTE_PIPE_CASE(1)
        RTE_PIPE_CASE(2)
        RTE_PIPE_CASE(4)
        RTE_PIPE_CASE(8)
        default:
          set_error("sweep: unsupported directions-per-warp");
          return RTE_ERR_UNSUPPORTED;
      }
#undef RTE_PIPE_CASE
      RTE_CHECK_CUDA(cudaGetLastError());
      return RTE_OK;
    }
  }
  const bool band = tv >= 0 ? ((tv == 0 || tv == 2) && nbands <= 8) : (nbands <= 8 && !fp64_throughput && !ang_throughput);
  if (band) {
    // band-parallel kernel: one CTA per task, one warp per 32-row band
    const int W = nbands;
    size_t elems = (size_t)D * p->R * 16 + ((p->R + 3) & ~3) + (((size_t)(W > 1 ? W - 1 : 1) * D * maxnx * 2 + 3) & ~(size_t)3);
    size_t smem = elems * sizeof(T) + (size_t)((maxnx + 3) & ~3) * sizeof(int) + 16;
    if (ANG) smem += (size_t)W * 32 * D * 32 * sizeof(T);   // output staging rings
    if (smem > 227 * 1024) {
      set_error("sweep: shared-memory table too large for this mesh/region count");
      return RTE_ERR_UNSUPPORTED;
    }
#define RTE_BAND_CASE(DD)                                                                                   \
  case DD: {                                                                                                \
    auto kern = k_sweep2d_bands<T, TI, DD, ANG>;                                                            \
    static std::atomic<size_t> granted[kMaxDevices];                                                        \
    RTE_TRY(grant_smem(kern, smem, granted));                                                               \
    kern<<<a.ntasks, W * 32, smem, st>>>(a);                                                                \
    count_launch();                                                                                         \
    break;                                                                                                  \
  }
    switch (D) {
      RTE_BAND_CASE(1)
      RTE_BAND_CASE(2)
      RTE_BAND_CASE(4)
      RTE_BAND_CASE(8)
      default:
        set_error("sweep: unsupported directions-per-warp");
        return RTE_ERR_UNSUPPORTED;
    }
#undef RTE_BAND_CASE
    RTE_CHECK_CUDA(cudaGetLastError());
    return RTE_OK;
  }
  a.smem_per_warp = D * p->R * 16 + D * maxnx * 2 + p->R;
  a.smem_per_warp = (a.smem_per_warp + 3) & ~3;
  size_t per_warp = (size_t)a.smem_per_warp * sizeof(T) + (ANG ? (size_t)32 * D * 32 * sizeof(T) : 0);
  int wpb = 4;
  while (wpb > 1 && per_warp * wpb > 96 * 1024) --wpb;
  size_t smem = per_warp * wpb;
  if (smem > 227 * 1024) {
    set_error("sweep: shared-memory table too large for this mesh/region count");
    return RTE_ERR_UNSUPPORTED;
  }
  int blocks = (a.ntasks + wpb - 1) / wpb;
#define RTE_SWEEP_CASE(DD)                                                                                  \
  case DD: {                                                                                                \
    auto kern = k_sweep2d<T, TI, DD, ANG>;                                                                  \
    static std::atomic<size_t> granted[kMaxDevices];                                                        \
    RTE_TRY(grant_smem(kern, smem, granted));                                                               \
    kern<<<blocks, wpb * 32, smem, st>>>(a);                                                                \
    count_launch();                                                                                         \
    break;                                                                                                  \
  }
  switch (D) {
    RTE_SWEEP_CASE(1)
    RTE_SWEEP_CASE(2)
    RTE_SWEEP_CASE(4)
    RTE_SWEEP_CASE(8)
    default:
      set_error("sweep: unsupported directions-per-warp");
      return RTE_ERR_UNSUPPORTED;
  }
#undef RTE_SWEEP_CASE
  RTE_CHECK_CUDA(cudaGetLastError());
  return RTE_OK;
}

// Sigma_s of the fused scaling: per region, or the cell blocks of cross-section profiles
static const void* sigma_s_arg(const rte_problem* p, bool f64) {
  if (p->cellsig) return f64 ? (const void*)p->d_sblk64.p : (const void*)p->d_sblk32.p;
  return f64 ? (const void*)p->d_sig_s.p : (const void*)p->d_sig_s32.p;
}

static void fill_args(rte_problem* p, SweepArgs& a, int prec) {
  std::memset(&a, 0, sizeof(a));
  a.inst = p->d_inst.p;
  a.udir = p->d_udir.p;
  a.tasks = p->d_tasks_by_D[p->tasks_D].p;
  a.ntasks = p->ntasks;
  if (p->cellsig)
    a.linv = prec == PREC_F64 ? (const void*)p->d_linvc64.p : (const void*)p->d_linvc32.p;
  else
    a.linv = prec == PREC_F64 ? (const void*)p->d_linv64.p
                              : (prec == PREC_DF ? (const void*)p->d_linv_df.p : (const void*)p->d_linv32.p);
  a.inflow_mask = p->inflow_mask;
  a.tasks_per_inst = p->tasks_per_inst;
  a.ndir = p->ndir;
  a.nu = p->nu;
  a.R = p->R;
  a.rx = p->rx;
  a.ry = p->ry;
}

static int ensure_partial(rte_problem* p, int prec) {
  size_t bytes = (size_t)p->tasks_per_inst * p->ntot * (prec == PREC_F32 ? 4 : 8);
  return p->d_partial.ensure(bytes);
}

// Sweep autotuner: times every valid (kernel variant, directions per warp) pair for one precision and
// output mode on this problem (two launches each after a warm-up, CUDA events on the stream) and keeps
// the fastest.  Candidates: D in {1, 2, 4, 8} dividing the directions of a quadrant (FP64 and
// double-float: D <= 4; angular output: D <= 4), variant band (ny <= 256) or warp-per-task.  The operator
// apply is timed with its partial-sum reduction, since D also sets the number of partials.
int autotune(rte_problem* p, int prec, bool ang, const void* src, void* psi, cudaStream_t st, bool scale_sigma_s,
             bool unique_layout) {
  const int fi = prec, ai = ang ? 1 : 0;
  const bool f64 = prec == PREC_F64;
  if (p->tuned_D[fi][ai] > 0 || p->dim == 1) return RTE_OK;
  const int nq = quadrant_gcd(p);
  int maxny = 0;
  for (int b = 0; b < p->B; ++b) maxny = std::max(maxny, p->ny[b]);
  RTE_TRY(p->d_tmp64.ensure((size_t)p->ntot));
  // partials for the largest candidate task count (D = 1)
  RTE_TRY(ensure_tasks(p, 1));
  RTE_TRY(ensure_partial(p, prec));
  const void* in = src;
  // the FP32 operator is timed with an FP32 input and output, as the inner solves launch it
  const bool in32 = prec == PREC_F32 && !ang && !src;
  if (in32) {
    RTE_TRY(p->d_tmp32.ensure((size_t)2 * p->ntot));
    RTE_CHECK_CUDA(cudaMemsetAsync(p->d_tmp32.p, 0, (size_t)2 * p->ntot * sizeof(float), st));
    in = p->d_tmp32.p;
  } else if (!in) {
    in = p->d_G.p;   // any input of the right size times the same
  }
  cudaEvent_t e0, e1;
  RTE_CHECK_CUDA(cudaEventCreate(&e0));
  RTE_CHECK_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int bestD = 0, bestV = -1;
  for (int var = 0; var < 3; ++var) {
    if (p->cellsig && var != 1) continue;   // cross-section profiles: the warp-per-task kernel only
    if ((var == 0 || var == 2) && (maxny + 31) / 32 > 8) continue;
    if (var == 2 && ang) continue;   // the pipelined kernel has no angular output
    for (int D : {1, 2, 4, 8}) {
      if (nq % D || (prec != PREC_F32 && D > 4) || (ang && D > 4)) continue;
      p->force_D = D;
      p->force_var = var;
      // one warm-up launch, then the best of five timed launches (robust to a slow outlier)
      int rc = RTE_OK;
      float cand = 1e30f;
      for (int rep = 0; rep < 6 && rc == RTE_OK; ++rep) {
        if (rep > 0) cudaEventRecord(e0, st);
        if (ang) rc = launch_angular(p, f64, in, 0, psi, st, scale_sigma_s, unique_layout);
        else if (in32) rc = launch_T(p, MODE_OP, false, in, false, nullptr, p->d_tmp32.p + p->ntot, false, nullptr, st);
        else if (prec == PREC_DF)
          rc = launch_T_df(p, MODE_OP, reinterpret_cast<const double*>(in), nullptr, p->d_tmp64.p, nullptr, st);
        else rc = launch_T(p, MODE_OP, f64, in, !f64 && src ? false : true, nullptr, p->d_tmp64.p, true, nullptr, st);
        if (rep > 0 && rc == RTE_OK) {
          float ms = 0.f;
          cudaEventRecord(e1, st);
          cudaEventSynchronize(e1);
          if (cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) cand = std::min(cand, ms);
        }
      }
      if (rc == RTE_OK && cand < best) {
        best = cand;
        bestD = D;
        bestV = var;
      }
      cudaGetLastError();
    }
  }
  p->force_D = 0;
  p->force_var = -1;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (bestD == 0) {
    set_error("sweep autotuner: no candidate ran");
    return RTE_ERR_CUDA;
  }
  p->tuned_D[fi][ai] = bestD;
  p->tuned_var[fi][ai] = bestV;
  p->tuned_ms[fi][ai] = best;
  return RTE_OK;
}

// Tune the three precisions of the operator apply (FP32, FP64, double-float), then build their task lists
// and size the partial-sum buffer (and the double-float input buffer) for the largest, so that later
// launches (including captured CUDA graphs) see stable device pointers.
int prepare_sweeps(rte_problem* p) {
  RTE_TRY(p->d_xdf.ensure((size_t)2 * p->ntot));
  RTE_TRY(autotune(p, PREC_F32, false, nullptr, nullptr, 0, false, false));
  RTE_TRY(autotune(p, PREC_F64, false, nullptr, nullptr, 0, false, false));
  if (!p->cellsig) RTE_TRY(autotune(p, PREC_DF, false, nullptr, nullptr, 0, false, false));
  size_t bytes = 0;
  for (int prec : {PREC_F32, PREC_F64, PREC_DF}) {
    if (p->cellsig && prec == PREC_DF) continue;
    RTE_TRY(ensure_tasks(p, pick_D(p, prec)));
    if (p->dim == 2) RTE_TRY(ensure_runs(p, pick_D(p, prec)));   // the pipelined kernel's runs, before any capture
    bytes = std::max(bytes, (size_t)p->tasks_per_inst * (size_t)p->ntot * (size_t)(prec == PREC_F32 ? 4 : 8));
  }
  return p->d_partial.ensure(bytes);
}

// x (FP64) -> double-float pairs, all instances
__global__ void k_split_df(const double* x, long long n, float2* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = x[i];
    const float h = (float)v;
    out[i] = make_float2(h, (float)(v - (double)h));
  }
}

int launch_T_df(rte_problem* p, int mode, const double* x, const double* bvec, double* out, const int* d_active,
                cudaStream_t st) {
  if (mode != MODE_OP && mode != MODE_RES) {
    set_error("launch_T_df: only the operator and the residual run in double-float");
    return RTE_ERR_UNSUPPORTED;
  }
  if (p->cellsig) {
    set_error("launch_T_df: no double-float sweep with cross-section profiles");
    return RTE_ERR_UNSUPPORTED;
  }
  RTE_TRY(p->d_xdf.ensure((size_t)2 * p->ntot));
  const int D = pick_D(p, PREC_DF);
  RTE_TRY(ensure_tasks(p, D));
  RTE_TRY(ensure_partial(p, PREC_DF));
  float2* xdf = reinterpret_cast<float2*>(p->d_xdf.p);
  k_split_df<<<(unsigned)std::min<long long>(4096, (p->ntot + 255) / 256), 256, 0, st>>>(x, p->ntot, xdf);
  count_launch();
  SweepArgs a;
  fill_args(p, a, PREC_DF);
  a.src = xdf;
  a.with_bc = 0;
  a.sig_s = p->d_sig_s_df.p;
  a.partial = p->d_partial.p;
  a.active = d_active;
  RTE_TRY((launch_sweep_t<dfloat, dfloat, false>(p, D, a, st)));
  int maxn = 0;
  for (int b = 0; b < p->B; ++b) maxn = std::max(maxn, (int)(p->off[b + 1] - p->off[b]));
  dim3 grid((maxn + 255) / 256, p->B);
  k_reduce<dfloat, double, double><<<grid, 256, 0, st>>>(reinterpret_cast<const dfloat*>(p->d_partial.p),
                                                         p->tasks_per_inst, p->d_inst.p, mode, x, bvec, out, d_active);
  count_launch();
  RTE_CHECK_CUDA(cudaGetLastError());
  return RTE_OK;
}

int launch_T(rte_problem* p, int mode, bool f64, const void* src, bool in_f64, const void* bvec, void* out,
             bool out_f64, const int* d_active, cudaStream_t st) {
  const int prec = f64 ? PREC_F64 : PREC_F32;
  int D = pick_D(p, prec);
  RTE_TRY(ensure_tasks(p, D));
  RTE_TRY(ensure_partial(p, prec));
  SweepArgs a;
  fill_args(p, a, prec);
  a.src = mode == MODE_RHS ? (const void*)p->d_G.p : src;
  bool src64 = mode == MODE_RHS ? true : in_f64;
  a.with_bc = mode == MODE_RHS ? 1 : 0;
  a.sig_s = (mode == MODE_OP || mode == MODE_RES) ? (sigma_s_arg(p, f64))
                                                   : nullptr;
  a.partial = p->d_partial.p;
  a.active = d_active;
  if (f64) {
    if (src64) RTE_TRY((launch_sweep_t<double, double, false>(p, D, a, st)));
    else RTE_TRY((launch_sweep_t<double, float, false>(p, D, a, st)));
  } else {
    if (src64) RTE_TRY((launch_sweep_t<float, double, false>(p, D, a, st)));
    else RTE_TRY((launch_sweep_t<float, float, false>(p, D, a, st)));
  }
  int maxn = 0;
  for (int b = 0; b < p->B; ++b) maxn = std::max(maxn, (int)(p->off[b + 1] - p->off[b]));
  dim3 grid((maxn + 255) / 256, p->B);
  int rmode = mode == MODE_RHS ? MODE_T : mode;
  if (rmode != MODE_T && !in_f64 && out_f64) {
    set_error("launch_T: FP32 operator input with FP64 output is not supported");
    return RTE_ERR_UNSUPPORTED;
  }
#define RTE_RED(TP, TZ, TO)                                                                                   \
  k_reduce<TP, TZ, TO><<<grid, 256, 0, st>>>(reinterpret_cast<const TP*>(p->d_partial.p), p->tasks_per_inst,    \
                                             p->d_inst.p, rmode, reinterpret_cast<const TZ*>(src),              \
                                             reinterpret_cast<const TO*>(bvec), reinterpret_cast<TO*>(out), d_active)
  if (f64) {
    if (out_f64) RTE_RED(double, double, double);
    else RTE_RED(double, float, float);
  } else {
    if (out_f64) RTE_RED(float, double, double);
    else RTE_RED(float, float, float);
  }
#undef RTE_RED
  count_launch();
  RTE_CHECK_CUDA(cudaGetLastError());
  return RTE_OK;
}

// Sweep part of A~ z only: fills the per-task partial scalar fluxes (Sigma_s scaling fused); the
// subtraction z - sum_t partial_t is left to the caller's kernel (the fused Arnoldi step).
int launch_op_partials(rte_problem* p, bool f64, const void* z, bool in_f64, const int* d_active, cudaStream_t st) {
  const int prec = f64 ? PREC_F64 : PREC_F32;
  int D = pick_D(p, prec);
  RTE_TRY(ensure_tasks(p, D));
  RTE_TRY(ensure_partial(p, prec));
  SweepArgs a;
  fill_args(p, a, prec);
  a.src = z;
  a.sig_s = sigma_s_arg(p, f64);
  a.partial = p->d_partial.p;
  a.active = d_active;
  if (f64) {
    if (in_f64) RTE_TRY((launch_sweep_t<double, double, false>(p, D, a, st)));
    else RTE_TRY((launch_sweep_t<double, float, false>(p, D, a, st)));
  } else {
    if (in_f64) RTE_TRY((launch_sweep_t<float, double, false>(p, D, a, st)));
    else RTE_TRY((launch_sweep_t<float, float, false>(p, D, a, st)));
  }
  return RTE_OK;
}

// A~ z (mode OP) with caller-provided task list and partial-sum storage: allocates nothing.  D must be
// a valid directions-per-warp value; tasks holds ntasks entries in the layout of ensure_tasks.
int launch_op_external(rte_problem* p, bool f64, const void* z, void* w, const SweepTask* tasks, int ntasks,
                       int tasks_per_inst, int D, void* partial, cudaStream_t st) {
  if (p->cellsig) {
    set_error("rte_apply_op_noalloc: not available with cross-section profiles");
    return RTE_ERR_UNSUPPORTED;
  }
  SweepArgs a;
  std::memset(&a, 0, sizeof(a));
  a.inst = p->d_inst.p;
  a.udir = p->d_udir.p;
  a.tasks = tasks;
  a.ntasks = ntasks;
  a.linv = f64 ? (const void*)p->d_linv64.p : (const void*)p->d_linv32.p;
  a.inflow_mask = p->inflow_mask;
  a.tasks_per_inst = tasks_per_inst;
  a.ndir = p->ndir;
  a.nu = p->nu;
  a.R = p->R;
  a.rx = p->rx;
  a.ry = p->ry;
  a.src = z;
  a.sig_s = sigma_s_arg(p, f64);
  a.partial = partial;
  if (f64) RTE_TRY((launch_sweep_t<double, double, false>(p, D, a, st)));
  else RTE_TRY((launch_sweep_t<float, float, false>(p, D, a, st)));
  int maxn = 0;
  for (int b = 0; b < p->B; ++b) maxn = std::max(maxn, (int)(p->off[b + 1] - p->off[b]));
  dim3 grid((maxn + 255) / 256, p->B);
  if (f64)
    k_reduce<double, double, double><<<grid, 256, 0, st>>>(reinterpret_cast<const double*>(partial), tasks_per_inst,
                                                          p->d_inst.p, MODE_OP, reinterpret_cast<const double*>(z),
                                                          nullptr, reinterpret_cast<double*>(w), nullptr);
  else
    k_reduce<float, float, float><<<grid, 256, 0, st>>>(reinterpret_cast<const float*>(partial), tasks_per_inst,
                                                       p->d_inst.p, MODE_OP, reinterpret_cast<const float*>(z),
                                                       nullptr, reinterpret_cast<float*>(w), nullptr);
  count_launch();
  RTE_CHECK_CUDA(cudaGetLastError());
  return RTE_OK;
}

int launch_angular(rte_problem* p, bool f64, const void* src, int with_bc, void* psi, cudaStream_t st,
                   bool scale_sigma_s, bool unique_layout) {
  const int prec = f64 ? PREC_F64 : PREC_F32;
  if (p->force_D == 0) RTE_TRY(autotune(p, prec, true, src, psi, st, scale_sigma_s, unique_layout));
  int D = pick_D(p, prec, true);
  RTE_TRY(ensure_tasks(p, D));
  RTE_TRY(ensure_partial(p, prec));
  SweepArgs a;
  fill_args(p, a, prec);
  a.src = src;
  a.with_bc = with_bc ? 1 : 0;
  a.partial = p->d_partial.p;
  a.psi = psi;
  a.psi_unique = unique_layout ? 1 : 0;
  if (scale_sigma_s) a.sig_s = sigma_s_arg(p, f64);
  if (f64) RTE_TRY((launch_sweep_t<double, double, true>(p, D, a, st)));
  else RTE_TRY((launch_sweep_t<float, float, true>(p, D, a, st)));
  return RTE_OK;
}

int launch_scalar_flux(rte_problem* p, bool f64, const void* psi, void* phi, cudaStream_t st) {
  DevBuf<double>* wdev = &p->d_wq;
  int maxn = 0;
  for (int b = 0; b < p->B; ++b) maxn = std::max(maxn, (int)(p->off[b + 1] - p->off[b]));
  dim3 grid((maxn + 255) / 256, p->B);
  if (f64)
    k_scalar_flux<double><<<grid, 256, 0, st>>>(reinterpret_cast<const double*>(psi), wdev->p, p->ndir, p->d_inst.p,
                                                 reinterpret_cast<double*>(phi));
  else
    k_scalar_flux<float><<<grid, 256, 0, st>>>(reinterpret_cast<const float*>(psi), wdev->p, p->ndir, p->d_inst.p,
                                                reinterpret_cast<float*>(phi));
  count_launch();
  RTE_CHECK_CUDA(cudaGetLastError());
  return RTE_OK;
}

}  // namespace rte

extern "C" {

static int check_dtype(int dtype) {
  RTE_ARG(dtype == RTE_F64 || dtype == RTE_F32, "dtype must be RTE_F64 or RTE_F32");
  return RTE_OK;
}

int rte_sweep(rte_problem_t p, int dtype, const void* src, int with_bc, void* psi, void* stream) {
  RTE_ARG(p && src && psi, "null handle or pointer");
  RTE_TRY(check_dtype(dtype));
  return rte::launch_angular(p, dtype == RTE_F64, src, with_bc, psi, (cudaStream_t)stream);
}

int rte_scalar_flux(rte_problem_t p, int dtype, const void* psi, void* phi, void* stream) {
  RTE_ARG(p && psi && phi, "null handle or pointer");
  RTE_TRY(check_dtype(dtype));
  return rte::launch_scalar_flux(p, dtype == RTE_F64, psi, phi, (cudaStream_t)stream);
}

int rte_apply_T(rte_problem_t p, int dtype, const void* s, void* phi, void* stream) {
  RTE_ARG(p && s && phi, "null handle or pointer");
  RTE_TRY(check_dtype(dtype));
  bool f = dtype == RTE_F64;
  return rte::launch_T(p, rte::MODE_T, f, s, f, nullptr, phi, f, nullptr, (cudaStream_t)stream);
}

int rte_apply_op(rte_problem_t p, int dtype, const void* z, void* w, void* stream) {
  RTE_ARG(p && z && w, "null handle or pointer");
  if (dtype == RTE_F64_DF)
    return rte::launch_T_df(p, rte::MODE_OP, reinterpret_cast<const double*>(z), nullptr, reinterpret_cast<double*>(w),
                            nullptr, (cudaStream_t)stream);
  RTE_TRY(check_dtype(dtype));
  bool f = dtype == RTE_F64;
  return rte::launch_T(p, rte::MODE_OP, f, z, f, nullptr, w, f, nullptr, (cudaStream_t)stream);
}

int rte_problem_set_sweep_variant(rte_problem_t p, int variant, int directions_per_warp, int tasks_per_run) {
  RTE_ARG(p, "null handle");
  RTE_ARG(tasks_per_run >= 0 && tasks_per_run <= 64, "tasks_per_run must be in [0, 64]");
  if (tasks_per_run != p->pin_run) {
    // runs are rebuilt with the new length
    p->pin_run = tasks_per_run;
    for (int d = 0; d < 17; ++d) p->nruns_by_D[d] = 0;
  }
  if (variant < 0) {
    p->pin_var = -1;
    p->pin_D = 0;
    return RTE_OK;
  }
  RTE_ARG(variant <= 2, "variant must be -1, 0 (band), 1 (warp per task) or 2 (pipelined band)");
  const int D = directions_per_warp;
  RTE_ARG(D == 1 || D == 2 || D == 4 || D == 8, "directions per warp must be 1, 2, 4 or 8");
  if (p->dim == 2) {
    RTE_ARG(rte::quadrant_gcd(p) % D == 0, "directions per warp must divide every quadrant's direction count");
    int maxny = 0;
    for (int b = 0; b < p->B; ++b) maxny = std::max(maxny, p->ny[b]);
    RTE_ARG(variant == 1 || (maxny + 31) / 32 <= 8, "the band variants cover meshes of at most 256 rows");
  }
  p->pin_var = variant;
  p->pin_D = D;
  return RTE_OK;
}

int rte_rhs(rte_problem_t p, int dtype, void* btilde, void* stream) {
  RTE_ARG(p && btilde, "null handle or pointer");
  RTE_TRY(check_dtype(dtype));
  bool f = dtype == RTE_F64;
  return rte::launch_T(p, rte::MODE_RHS, f, nullptr, true, nullptr, btilde, f, nullptr, (cudaStream_t)stream);
}

}  // extern "C"
