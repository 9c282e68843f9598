// rte_apply_op_noalloc: the fused A~ z = z - T Sigma_s z of rte_apply_op for callers that must not
// allocate device memory.  Its scratch (the sweep task list and the per-task partial scalar fluxes)
// lives in one file-scope __device__ array instead of buffers obtained with cudaMalloc.
#include "internal.h"

namespace rte {

// Largest scratch the entry point accepts; every GPU that loads the library holds this array until
// the process exits.
constexpr size_t kNoAllocScratchBytes = 16u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Task list (instance-major, quadrant-major, chunks of D unique directions), built on the device.
__global__ void k_make_tasks(int B, int D, int q0, int q1, int q2, int q3, int q4, SweepTask* out) {
  const int qs[5] = {q0, q1, q2, q3, q4};
  int per_inst = 0;
  for (int q = 0; q < 4; ++q) per_inst += (qs[q + 1] - qs[q]) / D;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= B * per_inst) return;
  const int b = tid / per_inst, t = tid % per_inst;
  int rem = t, q = 0;
  while (rem >= (qs[q + 1] - qs[q]) / D) {
    rem -= (qs[q + 1] - qs[q]) / D;
    ++q;
  }
  out[tid] = SweepTask{b, qs[q] + rem * D, t, 0};
}

// Device address of g_noalloc_scratch on the current device.  It is looked up on every call (with the device
// current) rather than cached: cudaGetSymbolAddress allocates nothing once the library's module is loaded on
// the device, and a cached address would go stale if the caller reset the device or its primary context was
// released and re-created (the module, and the array with it, would then be loaded anew).
static int scratch_address(void** out) {
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess) {
    set_error(std::string("rte_apply_op_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    return RTE_ERR_CUDA;
  }
  *out = ptr;
  return RTE_OK;
}

// Scratch bytes (task list rounded to 256 bytes, then the partial fluxes) for D directions per warp.
static size_t scratch_bytes(const rte_problem* p, int D, bool f64, int* per_inst_out) {
  int per_inst = 0;
  if (p->dim == 1) {
    per_inst = p->nu;
  } else {
    for (int q = 0; q < 4; ++q) per_inst += (p->quad_start[q + 1] - p->quad_start[q]) / D;
  }
  *per_inst_out = per_inst;
  const size_t ntasks = (size_t)p->B * per_inst;
  return ((ntasks * sizeof(SweepTask) + 255) & ~(size_t)255) + (size_t)per_inst * p->ntot * (f64 ? 8 : 4);
}

}  // namespace rte

using namespace rte;

extern "C" int rte_apply_op_noalloc(rte_problem_t p, int dtype, const void* z, void* w, void* stream) {
  RTE_ARG(p && z && w, "null handle or pointer");
  RTE_ARG(dtype == RTE_F64 || dtype == RTE_F32, "dtype must be RTE_F64 or RTE_F32");
  if (p->cellsig) {
    set_error("rte_apply_op_noalloc: not available with cross-section profiles (RTE_SIGMA_VARSCAT)");
    return RTE_ERR_UNSUPPORTED;
  }
  const bool f64 = dtype == RTE_F64;
  // Directions per warp: the value the sweep autotuner picked for this precision (when rte_apply_op or a
  // solve has tuned it) if its scratch fits, else the smallest D whose scratch fits (the most warps in flight;
  // FP64 takes D <= 4 like the tuned launches).
  int D = 1;
  if (p->dim == 2) {
    const int nq = quadrant_gcd(p);
    const int tuned = p->tuned_D[f64 ? PREC_F64 : PREC_F32][0];
    int dummy = 0;
    D = 0;
    if (tuned > 0 && nq % tuned == 0 && scratch_bytes(p, tuned, f64, &dummy) <= kNoAllocScratchBytes) D = tuned;
    for (int d : {1, 2, 4, 8}) {
      if (D) break;
      if ((f64 && d > 4) || nq % d) continue;
      if (scratch_bytes(p, d, f64, &dummy) <= kNoAllocScratchBytes) D = d;
    }
    if (!D) D = f64 ? 4 : 8;   // nothing fits: reported below with the smallest requirement
    while (nq % D) D >>= 1;
  }
  int per_inst = 0;
  const size_t need = scratch_bytes(p, D, f64, &per_inst);
  if (need > kNoAllocScratchBytes) {
    set_error("rte_apply_op_noalloc: problem needs " + std::to_string(need) +
              " bytes of scratch, more than the fixed " + std::to_string(kNoAllocScratchBytes) +
              "; use rte_apply_op");
    return RTE_ERR_INVALID_ARG;
  }
  const size_t ntasks = (size_t)p->B * per_inst;
  const size_t task_bytes = (ntasks * sizeof(SweepTask) + 255) & ~(size_t)255;
  void* base = nullptr;
  RTE_TRY(scratch_address(&base));
  SweepTask* tasks = static_cast<SweepTask*>(base);
  void* partial = static_cast<unsigned char*>(base) + task_bytes;
  cudaStream_t st = (cudaStream_t)stream;
  if (p->dim == 1) {
    // one task per (instance, direction): same construction with D = 1 and two "quadrants"
    k_make_tasks<<<(unsigned)((ntasks + 255) / 256), 256, 0, st>>>(p->B, 1, p->quad_start[0], p->quad_start[1],
                                                                   p->quad_start[2], p->quad_start[2],
                                                                   p->quad_start[2], tasks);
  } else {
    k_make_tasks<<<(unsigned)((ntasks + 255) / 256), 256, 0, st>>>(p->B, D, p->quad_start[0], p->quad_start[1],
                                                                   p->quad_start[2], p->quad_start[3],
                                                                   p->quad_start[4], tasks);
  }
  count_launch();
  RTE_CHECK_CUDA(cudaGetLastError());
  return launch_op_external(p, f64, z, w, tasks, (int)ntasks, per_inst, D, partial, st);
}
