// Reduced-basis products of the ROMSAD apply on the tensor cores (paper Sec. 4.3, eq. rom-sa-preconditioner):
//
//   y_b = P^T (Sigma_s v_b)        for every instance b of a ROM group (all on the ROM's mesh)
//   c_b = (U^T A_mu_b U)^{-1} y_b  (the inverses formed once per solve, FP32 copy)
//   z_b = v_b + W c_b
//
// The instances of a group share P and W, so the projection and the lift are matrix products over the group:
// Y [inst x r] = (Sigma_s V)^T [inst x N] . P [N x r] and Z [N x inst] = V + W [N x r] . C [r x inst].  Both run
// on the tensor cores with mma.sync m16n8k16 (BF16 operands, FP32 accumulation): BF16 copies of P and W are
// made once per ROM, the vector operands are rounded to BF16 while they are staged in shared memory.  The
// projection reduces over the N dofs: one block per chunk of 128 dofs writes a partial [inst x r] and a second
// kernel sums the chunks in a fixed order (deterministic) before the reduced solve.
//
// Fragment layouts of mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 (PTX ISA): with g = lane / 4 and
// t = lane % 4, a thread holds A(g, 2t..2t+1), A(g+8, 2t..2t+1), A(g, 2t+8..2t+9), A(g+8, 2t+8..2t+9);
// B(2t..2t+1, g), B(2t+8..2t+9, g); and accumulates D(g, 2t..2t+1), D(g+8, 2t..2t+1).
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cstdint>

#include "romsad.h"

namespace rte {

namespace {

constexpr int kChunk = 128;     // dofs per projection block (8 k-steps)
constexpr int kMaxInst = 64;    // instances per block (4 m-tiles)
constexpr int kLiftRows = 128;  // dofs per lift block (8 m-tiles)

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  const uint32_t l = (uint32_t)__bfloat16_as_ushort(lo), h = (uint32_t)__bfloat16_as_ushort(hi);
  return l | (h << 16);
}

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void k_to_bf16(const float* x, long long n, __nv_bfloat16* y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

// Projection partials.  Block (chunk, instance group of up to 64): stage A = Sigma_s v (instances x 128 dofs)
// and B = P (128 dofs x rp) in shared memory as BF16, then 8 warps cover the (m-tile, n-tile) pairs, each
// accumulating over the 8 k-steps.  part[(chunk * ninst + i) * 64 + k].  rp: r rounded up to 8.
__global__ void __launch_bounds__(256) k_rom_project_tc(const __nv_bfloat16* P16, int rmax, int r, int rp,
                                                        const InstInfo* inst, const int* list, int ninst,
                                                        const int* active, const float* sig_dof, const float* v,
                                                        int N, float* part) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int ni = min(kMaxInst, ninst - blockIdx.y * kMaxInst);   // instances of this block
  const int mt = (ni + 15) / 16;                                  // m-tiles
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(smem);     // [mt*16][kChunk]
  __nv_bfloat16* Bs = As + (size_t)mt * 16 * kChunk;               // [kChunk][rp + 8] (padded row)
  const int ldb = rp + 8;
  const int n0 = blockIdx.x * kChunk;
  const int nk = min(kChunk, N - n0);
  // stage A: rows = instances (zero rows beyond ni, zero columns beyond the mesh, inactive instances zero); two
  // consecutive dofs per thread and load (instance offsets and N are even in 1D and 2D)
  for (int e = threadIdx.x; e < mt * 16 * (kChunk / 2); e += blockDim.x) {
    const int m = e / (kChunk / 2), k = 2 * (e % (kChunk / 2));
    float2 val = make_float2(0.f, 0.f);
    if (m < ni && k < nk) {
      const int b = list[blockIdx.y * kMaxInst + m];
      if (!active || active[b]) {
        const long long off = inst[b].off + n0 + k;
        const float2 sv = *reinterpret_cast<const float2*>(sig_dof + off);
        const float2 vv = *reinterpret_cast<const float2*>(v + off);
        val = make_float2(sv.x * vv.x, sv.y * vv.y);
      }
    }
    *reinterpret_cast<__nv_bfloat162*>(As + (size_t)m * kChunk + k) = __floats2bfloat162_rn(val.x, val.y);
  }
  // stage B: P rows n0..n0+nk, ranks < rp (zero beyond r and beyond the mesh)
  for (int e = threadIdx.x; e < kChunk * rp; e += blockDim.x) {
    const int k = e / rp, c = e % rp;
    Bs[k * ldb + c] = (k < nk && c < r) ? P16[(size_t)(n0 + k) * rmax + c] : __float2bfloat16_rn(0.f);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int ntile = rp / 8;
  for (int tile = warp; tile < mt * ntile; tile += 8) {
    const int mi = tile / ntile, nj = tile % ntile;
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    const __nv_bfloat16* Ar0 = As + (size_t)(mi * 16 + g) * kChunk;
    const __nv_bfloat16* Ar1 = Ar0 + 8 * kChunk;
#pragma unroll 4
    for (int ks = 0; ks < kChunk; ks += 16) {
      uint32_t a[4], b[2];
      a[0] = *reinterpret_cast<const uint32_t*>(Ar0 + ks + 2 * t);
      a[1] = *reinterpret_cast<const uint32_t*>(Ar1 + ks + 2 * t);
      a[2] = *reinterpret_cast<const uint32_t*>(Ar0 + ks + 2 * t + 8);
      a[3] = *reinterpret_cast<const uint32_t*>(Ar1 + ks + 2 * t + 8);
      const int col = nj * 8 + g;
      b[0] = pack_bf16(Bs[(ks + 2 * t) * ldb + col], Bs[(ks + 2 * t + 1) * ldb + col]);
      b[1] = pack_bf16(Bs[(ks + 2 * t + 8) * ldb + col], Bs[(ks + 2 * t + 9) * ldb + col]);
      mma_bf16(d, a, b);
    }
    // D(g, 2t..2t+1) and D(g+8, 2t..2t+1): instance rows, rank columns
    const int c0 = nj * 8 + 2 * t;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int m = mi * 16 + g + 8 * h;
      if (m < ni) {
        float* dst = part + ((size_t)blockIdx.x * ninst + blockIdx.y * kMaxInst + m) * 64;
        if (c0 < r) dst[c0] = d[2 * h];
        if (c0 + 1 < r) dst[c0 + 1] = d[2 * h + 1];
      }
    }
  }
}

// c_i = inv_i . (sum over chunks of the partials, fixed order), FP32; one block of 64 threads per instance.
__global__ void k_rom_solve_tc(const float* part, int nchunk, int ninst, int r, const float* inv, const int* list,
                               const int* active, float* c) {
  const int i = blockIdx.x;
  const int b = list[i];
  __shared__ float y[64];
  const int t = threadIdx.x;
  const bool on = !active || active[b];
  if (t < r) {
    float s = 0.f;
    if (on)
      for (int ch = 0; ch < nchunk; ++ch) s += part[((size_t)ch * ninst + i) * 64 + t];
    y[t] = s;
  }
  __syncthreads();
  if (t < 64) {
    float s = 0.f;
    if (t < r && on) {
      const float* row = inv + (size_t)i * 64 * 64 + (size_t)t * r;
      for (int k = 0; k < r; ++k) s += row[k] * y[k];
    }
    c[(size_t)i * 64 + t] = s;   // zero beyond r: the lift's padded ranks add nothing
  }
}

// Lift z = v + W c for up to 64 instances per block and 128 dofs: A = W (dofs x rank, BF16), B = C (rank x
// instances, BF16), D (dofs x instances) staged in shared memory and written instance by instance (coalesced).
__global__ void __launch_bounds__(256) k_rom_lift_tc(const __nv_bfloat16* W16, int rmax, int r, int kp,
                                                     const InstInfo* inst, const int* list, int ninst,
                                                     const int* active, const float* c, const float* v, float* z,
                                                     int N) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int ni = min(kMaxInst, ninst - blockIdx.y * kMaxInst);
  const int ntile = (ni + 7) / 8;                                 // n-tiles of instances
  const int lda = kp + 8;
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(smem);     // [kLiftRows][kp + 8]
  __nv_bfloat16* Bs = As + (size_t)kLiftRows * lda;                // [ntile*8][kp + 8]: Bs[n][k] = c_n[k]
  float* Ds = reinterpret_cast<float*>(Bs + (size_t)ntile * 8 * lda);   // [ntile*8][kLiftRows]
  const int n0 = blockIdx.x * kLiftRows;
  const int nr = min(kLiftRows, N - n0);
  for (int e = threadIdx.x; e < kLiftRows * kp; e += blockDim.x) {
    const int m = e / kp, k = e % kp;
    As[m * lda + k] = (m < nr && k < r) ? W16[(size_t)(n0 + m) * rmax + k] : __float2bfloat16_rn(0.f);
  }
  for (int e = threadIdx.x; e < ntile * 8 * kp; e += blockDim.x) {
    const int n = e / kp, k = e % kp;
    float val = 0.f;
    if (n < ni && k < r) val = c[(size_t)(blockIdx.y * kMaxInst + n) * 64 + k];
    Bs[n * lda + k] = __float2bfloat16_rn(val);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int mtile = kLiftRows / 16;
  for (int tile = warp; tile < mtile * ntile; tile += 8) {
    const int mi = tile / ntile, nj = tile % ntile;
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    const __nv_bfloat16* Ar0 = As + (size_t)(mi * 16 + g) * lda;
    const __nv_bfloat16* Ar1 = Ar0 + 8 * lda;
    const __nv_bfloat16* Bc = Bs + (size_t)(nj * 8 + g) * lda;
    for (int ks = 0; ks < kp; ks += 16) {
      uint32_t a[4], b[2];
      a[0] = *reinterpret_cast<const uint32_t*>(Ar0 + ks + 2 * t);
      a[1] = *reinterpret_cast<const uint32_t*>(Ar1 + ks + 2 * t);
      a[2] = *reinterpret_cast<const uint32_t*>(Ar0 + ks + 2 * t + 8);
      a[3] = *reinterpret_cast<const uint32_t*>(Ar1 + ks + 2 * t + 8);
      b[0] = *reinterpret_cast<const uint32_t*>(Bc + ks + 2 * t);
      b[1] = *reinterpret_cast<const uint32_t*>(Bc + ks + 2 * t + 8);
      mma_bf16(d, a, b);
    }
    const int nc = nj * 8 + 2 * t;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int m = mi * 16 + g + 8 * h;
      Ds[(size_t)nc * kLiftRows + m] = d[2 * h];
      Ds[(size_t)(nc + 1) * kLiftRows + m] = d[2 * h + 1];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ni * kLiftRows; e += blockDim.x) {
    const int n = e / kLiftRows, m = e % kLiftRows;
    if (m >= nr) continue;
    const int b = list[blockIdx.y * kMaxInst + n];
    if (active && !active[b]) continue;
    const long long o = inst[b].off + n0 + m;
    z[o] = v[o] + Ds[(size_t)n * kLiftRows + m];
  }
}

}  // namespace

int rom_tc_prepare(romsad* rom, cudaStream_t st) {
  // shared memory above 48 KB, granted per device (the attribute acts on the current device)
  constexpr int kMaxDev = 64;
  static std::atomic<int> granted[kMaxDev];
  int dev = 0;
  RTE_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDev) {
    set_error("romsad tensor-core path: device ordinal beyond the supported range");
    return RTE_ERR_UNSUPPORTED;
  }
  if (!granted[dev].load()) {
    RTE_CHECK_CUDA(cudaFuncSetAttribute(k_rom_project_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
    RTE_CHECK_CUDA(cudaFuncSetAttribute(k_rom_lift_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
    granted[dev].store(1);
  }
  if (rom->bf16_rank == rom->r && rom->P16.p) return RTE_OK;
  const size_t n = (size_t)rom->N * rom->rmax;
  RTE_TRY(rom->P16.ensure(n));
  RTE_TRY(rom->W16.ensure(n));
  const unsigned blocks = (unsigned)std::min<size_t>(4096, (n + 255) / 256);
  k_to_bf16<<<blocks, 256, 0, st>>>(rom->P32.p, (long long)n, reinterpret_cast<__nv_bfloat16*>(rom->P16.p));
  count_launch();
  k_to_bf16<<<blocks, 256, 0, st>>>(rom->W32.p, (long long)n, reinterpret_cast<__nv_bfloat16*>(rom->W16.p));
  count_launch();
  RTE_CHECK_CUDA(cudaGetLastError());
  rom->bf16_rank = rom->r;
  return RTE_OK;
}

__global__ void k_inv_f32(const double* a, float* b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

int rom_tc_plan_setup(RomPlan& pl, cudaStream_t st) {
  romsad* rom = pl.rom;
  const int n = (int)pl.ids.size();
  RTE_TRY(rom_tc_prepare(rom, st));
  const int nchunk = (rom->N + kChunk - 1) / kChunk;
  RTE_TRY(pl.part32.ensure((size_t)nchunk * std::max(1, n) * 64));
  RTE_TRY(pl.c32.ensure((size_t)std::max(1, n) * 64));
  RTE_TRY(pl.inv32.ensure(pl.lu.n));
  k_inv_f32<<<64, 256, 0, st>>>(pl.lu.p, pl.inv32.p, (long long)pl.lu.n);
  count_launch();
  RTE_CHECK_CUDA(cudaGetLastError());
  return RTE_OK;
}

int rom_tc_apply(RomPlan& pl, rte_problem* p, const int* d_active, const float* v, float* z, cudaStream_t st) {
  romsad* rom = pl.rom;
  const int n = (int)pl.ids.size();
  if (n == 0) return RTE_OK;
  if (rom->bf16_rank != rom->r || !rom->P16.p) {
    set_error("romsad tensor-core path: rom_tc_prepare was not called at this rank");
    return RTE_ERR_INVALID_ARG;
  }
  const int r = rom->r, rp = (r + 7) / 8 * 8, kp = (r + 15) / 16 * 16;
  const int N = rom->N;
  const int nchunk = (N + kChunk - 1) / kChunk;
  const int groups = (n + kMaxInst - 1) / kMaxInst;
  if (pl.part32.n < (size_t)nchunk * n * 64 || pl.c32.n < (size_t)n * 64 || pl.inv32.n < pl.lu.n) {
    set_error("romsad tensor-core path: rom_tc_plan_setup was not called for this plan");
    return RTE_ERR_INVALID_ARG;
  }
  const int mt = (std::min(n, kMaxInst) + 15) / 16;
  const size_t smem_p = (size_t)mt * 16 * kChunk * 2 + (size_t)kChunk * (rp + 8) * 2;
  const int ntile = (std::min(n, kMaxInst) + 7) / 8;
  const size_t smem_l = (size_t)kLiftRows * (kp + 8) * 2 + (size_t)ntile * 8 * (kp + 8) * 2 +
                        (size_t)ntile * 8 * kLiftRows * 4;
  k_rom_project_tc<<<dim3(nchunk, groups), 256, smem_p, st>>>(
      reinterpret_cast<const __nv_bfloat16*>(rom->P16.p), rom->rmax, r, rp, p->d_inst.p, pl.d_ids.p, n, d_active,
      p->d_sig_dof32.p, v, N, pl.part32.p);
  count_launch();
  k_rom_solve_tc<<<n, 64, 0, st>>>(pl.part32.p, nchunk, n, r, pl.inv32.p, pl.d_ids.p, d_active, pl.c32.p);
  count_launch();
  k_rom_lift_tc<<<dim3((N + kLiftRows - 1) / kLiftRows, groups), 256, smem_l, st>>>(
      reinterpret_cast<const __nv_bfloat16*>(rom->W16.p), rom->rmax, r, kp, p->d_inst.p, pl.d_ids.p, n, d_active,
      pl.c32.p, v, z, N);
  count_launch();
  RTE_CHECK_CUDA(cudaGetLastError());
  return RTE_OK;
}

}  // namespace rte
