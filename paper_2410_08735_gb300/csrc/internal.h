// Internal declarations shared by the translation units of librte_gb300.
// Everything here is host C++ / CUDA for sm_103a; the public surface is include/rte.h.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "../../include/rte.h"

namespace rte {

// ----------------------------------------------------------------- errors
void set_error(const std::string& msg);
// number of kernels this library has launched (reported by rte_kernel_launches)
void count_launch();
void add_launches(long long n);
long long launches_so_far();
struct Status {
  int code = RTE_OK;
};
#define RTE_CHECK_CUDA(expr)                                                                 \
  do {                                                                                       \
    cudaError_t _e = (expr);                                                                 \
    if (_e != cudaSuccess) {                                                                 \
      ::rte::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));                  \
      return _e == cudaErrorMemoryAllocation ? RTE_ERR_OOM : RTE_ERR_CUDA;                   \
    }                                                                                        \
  } while (0)
#define RTE_TRY(expr)                \
  do {                               \
    int _s = (expr);                 \
    if (_s != RTE_OK) return _s;     \
  } while (0)
#define RTE_ARG(cond, msg)                                 \
  do {                                                     \
    if (!(cond)) {                                         \
      ::rte::set_error(std::string("invalid argument: ") + (msg)); \
      return RTE_ERR_INVALID_ARG;                          \
    }                                                      \
  } while (0)

// Device buffer owned by a handle.
template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  int alloc(size_t count) {
    release();
    if (count == 0) return RTE_OK;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
      return RTE_ERR_OOM;
    }
    n = count;
    return RTE_OK;
  }
  int ensure(size_t count) { return count <= n && p ? RTE_OK : alloc(count); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  ~DevBuf() { release(); }
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n) {
    o.p = nullptr;
    o.n = 0;
  }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p;
      n = o.n;
      o.p = nullptr;
      o.n = 0;
    }
    return *this;
  }
};

// Per-instance geometry as seen by the kernels.
struct InstInfo {
  int nx, ny;          // cells
  long long off;       // dof offset in a scalar vector
  int ndof;            // nx*ny*nd
  double hx, hy;       // cell sizes
  double g;            // isotropic inflow value on the inflow faces of the instance (eq. 1c)
};

// A unique in-plane direction (duplicates over +-Omega_z merged, weights summed).
struct UDir {
  double ax, ay;       // |Omega_x|, |Omega_y| (2D); |mu| in ax (1D)
  double w;            // merged weight
  int sx, sy;          // signs of Omega_x, Omega_y (+1/-1)
  int quadrant;        // 2D: 0 (+,+), 1 (-,+), 2 (+,-), 3 (-,-); 1D: 0 (mu>0), 1 (mu<0)
  int ndup;            // number of original directions mapped here
  int dup[4];          // their original indices (ndup <= 4)
};

// Sweep task: one warp sweeps D unique directions of one quadrant of one instance.
struct SweepTask {
  int b;       // instance
  int u0;      // first unique direction (directions u0..u0+D-1 share a quadrant)
  int t;       // task index within the instance (partial-sum slot)
  int pad;
};

// dsa.cu: DSA preconditioner through one multigrid V-cycle.  dsa_check: whether the meshes are covered;
// dsa_prepare: per-parameter set-up (cross sections, cell blocks, Galerkin hierarchy); dsa_launch:
// z = v + x (x ~ K^{-1} Sigma_s v) for instances with active[b] (and only[b], when given).
int dsa_check(rte_problem* p);
int dsa_prepare(rte_problem* p, int variant, cudaStream_t st);
int dsa_launch(rte_problem* p, bool f64, const void* v, void* z, const int* active, const int* only,
               cudaStream_t st);
}  // namespace rte

struct rte_problem {
  int dim = 2, B = 0, nd = 4, ndir = 0, nu = 0, R = 1, rx = 1, ry = 1;
  int n_polar = 0, n_azim = 0;       // quadrature orders as given at create
  std::vector<int> nx, ny;
  std::vector<long long> off;        // [B+1]
  long long ntot = 0;
  double box[4] = {0, 1, 0, 1};
  double g = 0.0, src_q = 0.0, src_box[4] = {0, 0, 0, 0};
  int inflow_mask = 15;              // domain faces with inflow g: 1 x-low, 2 x-high, 4 y-low, 8 y-high
  int src_kind = RTE_SRC_BOX;
  double src_gauss[4] = {0, 0, 0, 0};   // A, a, xc, yc
  std::vector<double> ss, sa;        // [B][R] host copies
  std::vector<double> om_x, om_y, om_z, w;  // [ndir] quadrature (paper order)
  std::vector<int> uniq_of_dir;      // [ndir]
  std::vector<rte::UDir> udir;       // [nu], grouped by quadrant, quadrant-major
  std::vector<int> quad_start;       // [nquad+1] first unique dir of each quadrant
  std::vector<rte::InstInfo> inst;   // [B]
  // device state
  rte::DevBuf<rte::InstInfo> d_inst;
  rte::DevBuf<rte::UDir> d_udir;
  rte::DevBuf<double> d_sig_s, d_sig_t;       // [B][R]
  rte::DevBuf<float> d_sig_s32;               // [B][R]
  rte::DevBuf<double> d_sig_dof;              // [ntot] sigma_s of every dof (ROM projections)
  rte::DevBuf<float> d_sig_dof32;             // the same in FP32
  rte::DevBuf<double> d_G;                    // [ntot] source moments
  rte::DevBuf<double> d_linv64;               // [B][nu][R][nd*nd]
  rte::DevBuf<float> d_linv32;
  rte::DevBuf<float> d_linv_df;               // the same as double-float pairs (hi, lo) [..][2]
  rte::DevBuf<float> d_sig_s_df;              // [B][R][2] sigma_s as double-float pairs
  rte::DevBuf<float> d_xdf;                   // [ntot][2] operator input split into double-float pairs
  // sweep scratch (grown on demand)
  rte::DevBuf<unsigned char> d_partial;       // partial scalar fluxes per task
  // task lists per directions-per-warp value D (index D), built once; stable device pointers
  rte::DevBuf<rte::SweepTask> d_tasks_by_D[17];
  int ntasks_by_D[17] = {0};
  // pipelined band kernel: runs of tasks per persistent CTA (first task, tasks, period, 0), per D
  rte::DevBuf<int4> d_runs_by_D[17];
  int nruns_by_D[17] = {0};
  size_t pipe_smem_elems_by_D[17] = {0};
  int per_inst_by_D[17] = {0};
  int tasks_D = -1;                           // D of the most recent launch
  // sweep autotuner (sweep.cu): tuned directions per warp and kernel variant per [precision][angular]
  // (precision: PREC_F32, PREC_F64, PREC_DF; 0 = not tuned); force_* steer launches while candidates are timed
  int tuned_D[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  int tuned_var[3][2] = {{-1, -1}, {-1, -1}, {-1, -1}};
  int force_D = 0, force_var = -1;
  int pin_D = 0, pin_var = -1;                // rte_problem_set_sweep_variant (a user's pin; overrides the tuning)
  int pin_run = 0;                            // tasks per run of the pipelined kernel (0: automatic)
  float tuned_ms[3][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  int ntasks = 0, tasks_per_inst = 0;
  rte::DevBuf<int> d_active;                  // [B] instance mask (1 = active), all 1 by default
  rte::DevBuf<double> d_tmp64;                // [ntot] temporaries
  rte::DevBuf<float> d_tmp32;                 // [2 ntot] FP32 input and output of the autotuner's timing
  rte::DevBuf<double> d_wq;                   // [ndir] quadrature weights (paper order)
  // cross-section profiles (RTE_SIGMA_VARSCAT): full 4x4 blocks per cell; every instance on the same mesh of ncell
  // cells, block (b, c) at [(b * ncell + c) * 16]
  bool cellsig = false;
  int ncell = 0;
  std::vector<double> F;                      // [ncell][16] blocks of the profile f (int_T f eta_k eta_l)
  rte::DevBuf<double> d_F64;                  // the same on the device
  rte::DevBuf<double> d_sblk64, d_tblk64;     // [B][ncell][16] Sigma_s and Sigma_t blocks
  rte::DevBuf<float> d_sblk32;                // Sigma_s blocks in FP32
  rte::DevBuf<double> d_sigc_s, d_sigc_t;     // [B][ncell] cell means (the DSA's cross sections)
  rte::DevBuf<double> d_linvc64;              // [B][nu][ncell][16] cell inverses (reflected frame of each direction)
  rte::DevBuf<float> d_linvc32;
  std::shared_ptr<void> krylov_ws;            // FGMRES workspace (krylov.cu), grown on demand
  std::shared_ptr<void> dsa_ws;               // DSA multigrid workspace (dsa.cu), sized once
};

namespace rte {
// problem.cu
int upload_params(rte_problem* p);
// greatest common divisor of the unique-direction counts of the quadrants (2D) or of the two half-ranges (1D):
// a directions-per-warp value must divide it
int quadrant_gcd(const rte_problem* p);
// sweep.cu: generic launcher.
//   src:  input vector (dtype in_f64 ? double : float)
//   mode: 0 phi = T s ; 1 w = z - T(Sigma_s z) ; 2 r = b - (z - T(Sigma_s z)) ; 3 b~ (src = G, bc)
//   compute_f64: arithmetic of the sweep; out_f64: type of out and b
enum SweepMode { MODE_T = 0, MODE_OP = 1, MODE_RES = 2, MODE_RHS = 3 };
// arithmetic of a sweep: FP32, FP64, or double-float (pairs of FP32, dfloat.cuh)
enum SweepPrec { PREC_F32 = 0, PREC_F64 = 1, PREC_DF = 2 };
int launch_T(rte_problem* p, int mode, bool compute_f64, const void* src, bool in_f64, const void* bvec,
             void* out, bool out_f64, const int* d_active, cudaStream_t st);
// A~ x (MODE_OP) or b - A~ x (MODE_RES) with FP64 vectors and double-float sweep arithmetic: x is split into
// double-float pairs, swept, and the partial fluxes are summed in double-float; the final z - T Sigma_s z and
// b - (.) are formed in FP64.
int launch_T_df(rte_problem* p, int mode, const double* x, const double* bvec, double* out, const int* d_active,
                cudaStream_t st);
// Angular-output sweep; scale_sigma_s multiplies the source by sigma_s, unique_layout writes one block
// per unique direction ([nu][N] per instance) instead of all N_Omega directions.
int launch_angular(rte_problem* p, bool f64, const void* src, int with_bc, void* psi, cudaStream_t st,
                   bool scale_sigma_s = false, bool unique_layout = false);
// task lists and partial buffer for both precisions (stable pointers for graph capture)
int prepare_sweeps(rte_problem* p);
// sweep part of A~ z (per-task partial fluxes in p->d_partial); z is double if in_f64, else float
int launch_op_partials(rte_problem* p, bool f64, const void* z, bool in_f64, const int* d_active, cudaStream_t st);
// A~ z with caller-provided task list and partial storage (no allocation)
int launch_op_external(rte_problem* p, bool f64, const void* z, void* w, const SweepTask* tasks, int ntasks,
                       int tasks_per_inst, int D, void* partial, cudaStream_t st);
int launch_scalar_flux(rte_problem* p, bool f64, const void* psi, void* phi, cudaStream_t st);
// forward operator y = (D_u + sigma_t) x (FP64) for ncol columns on one mesh; used offline
int launch_forward_cols(int dim, int nx, int ny, double hx, double hy, const UDir& u, int rx, int ry,
                        const double* sig_t_reg, const double* x, long long ldx, double* y, long long ldy, int ncol,
                        cudaStream_t st);
// dsa.cu: DSA preconditioner through one multigrid V-cycle.  dsa_check: whether the meshes are covered;
// dsa_prepare: per-parameter set-up (cross sections, cell blocks, Galerkin hierarchy); dsa_launch:
// z = v + x (x ~ K^{-1} Sigma_s v) for instances with active[b] (and only[b], when given).
int dsa_check(rte_problem* p);
int dsa_prepare(rte_problem* p, int variant, cudaStream_t st);
int dsa_launch(rte_problem* p, bool f64, const void* v, void* z, const int* active, const int* only,
               cudaStream_t st);
}  // namespace rte
