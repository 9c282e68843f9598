// ROMSAD data structures shared by romsad.cu, greedy.cu and krylov.cu.
#pragma once
#include <cstdint>

#include "internal.h"

struct rte_mlp;

struct romsad {
  // mesh the ROM belongs to (must match every instance it is applied to)
  int dim = 2, nx = 0, ny = 0, nd = 4, ndir = 0, nu = 0, R = 1, rx = 1, ry = 1;
  double box[4] = {0, 1, 0, 1};
  int N = 0;        // dofs of the mesh
  int r = 0;        // rank
  int rmax = 0;     // capacity of the device arrays (columns)
  // stored direction blocks of U: a = 0..nA-1 (all N_Omega directions, or the unique in-plane ones
  // with multiplicity); P = sum_a mult_a U_a, W = sum_a wA_a U_a
  int nA = 0;
  std::vector<int> uidx;       // [nA] unique direction of block a
  std::vector<double> mult;    // [nA]
  std::vector<double> wA;      // [nA]
  std::vector<int> dir_block;  // [ndir] stored block holding direction j
  // device arrays
  rte::DevBuf<double> P, W;    // [N][rmax] (dof-major, rank contiguous)
  rte::DevBuf<float> P32, W32;
  rte::DevBuf<double> U;       // [rmax][nA][N] (greedy / create_from_basis; may be empty after load)
  rte::DevBuf<double> Y;       // [rmax][nA][N]: D_u U_a (transport without collision), greedy only
  // affine reduced operators, host, row-major [r][r]
  std::vector<double> A_D;     // sum_a mult_a U_a^T D_u U_a
  std::vector<double> T_R;     // [R][r][r] sum_a mult_a U_a^T chi_R U_a
  std::vector<double> S_R;     // [R][r][r] P^T chi_R W
  rte::DevBuf<double> d_aff;   // [(1 + 2R)][r][r] device copy: A_D, T_R..., S_R...
  rte_mlp* mlp = nullptr;      // learned warm start (not owned)
  rte::DevBuf<uint16_t> P16, W16;   // BF16 copies of P32, W32 for the tensor-core products (romsad_tc.cu)
  // cross-section profiles (RTE_SIGMA_VARSCAT): the affine terms are the profile blocks F (term 0) and the identity
  // (term 1) instead of region indicators; F is kept (device) while columns are added
  int sigma_modes = 0;
  rte::DevBuf<double> F;            // [ncell][16]
  int bf16_rank = 0;                // rank the BF16 copies were made at (0: none)
};

namespace rte {
// First FGMRES cycle of a high-fidelity solve (instance 0), for the xi recurrence (Sec. 4.4.1).
struct FirstCycle {
  int want = 0;              // number of preconditioned vectors z to keep (the window)
  bool done = false;
  int k = 0, m = 0, nz = 0;  // columns in the first cycle, restart length, vectors kept
  double beta = 0.0;         // ||r^(0)||
  std::vector<double> H;     // unrotated Hessenberg, column-major [m][m+1]
  DevBuf<double> Z;          // [nz][N] z^(1..nz) (= v without a preconditioner)
};
int hf_solve(rte_problem* p, double rtol, int restart, int max_iter, int dsa_variant, double* x, FirstCycle* rec,
             int* iterations, int* status);
int rom_add_column(romsad* rom, DevBuf<double>& d_mult, DevBuf<double>& d_wA, cudaStream_t st);
int rom_compute_Y_column(romsad* rom, const rte_problem* p, int inst, int k, cudaStream_t st);
void rom_init_geometry(romsad* rom, const rte_problem* p, int b);
int rom_alloc_arrays(romsad* rom, int rmax, bool withU);
// y[b][k] = (P^T Sigma_s v_b)[k] for the listed instances (FP64), y laid out [ninst][64]
int rom_project_list(romsad* rom, rte_problem* p, const int* d_list, int ninst, const double* v, double* y,
                     cudaStream_t st);
// ROMSAD application plan for one ROM and the instances that use it, built once per solve: the
// reduced operators U^T A_mu U are assembled and LU-factored at build; apply() then costs one
// projection (multi-block partial sums), two triangular solves and one lift.
struct RomPlan {
  romsad* rom = nullptr;
  std::vector<int> ids;
  DevBuf<int> d_ids, piv;
  DevBuf<double> lu, part, c;
  DevBuf<float> inv32;   // FP32 copy of lu (the inverses), filled by the FGMRES driver
  DevBuf<double> WT;     // W transposed [r][N] (coalesced lift), filled by the FGMRES driver
  DevBuf<float> WT32;
  DevBuf<float> part32, c32;   // tensor-core path: projection partials [nchunk][n][64], coefficients [n][64]
  int chunk = 1024, nchunk = 0;
  int build(romsad* rom, rte_problem* p, const std::vector<int>& ids, cudaStream_t st);
  int apply(rte_problem* p, const int* d_active, const double* v, double* z, bool f64, cudaStream_t st);
};
// Assemble and LU-factor U^T A_mu U for the listed instances of p (device), then
// c = A_r^{-1} y per instance: y [ninst][r] in, c [ninst][r] out (FP64).
int rom_small_solve(romsad* rom, rte_problem* p, const int* d_list, int ninst, const double* y, double* c,
                    cudaStream_t st);
int rom_check_mesh(const romsad* rom, const rte_problem* p, int b);
// z_b = v_b + W c_b for the listed instances (c laid out [ninst][64])
int rom_lift_list(romsad* rom, rte_problem* p, const int* d_list, int ninst, const double* v, const double* c,
                  double* z, cudaStream_t st);
// c_hat of the listed instances from the MLP (host list, device list copy), out [ninst][64]
int mlp_predict_instances(rte_mlp* M, rte_problem* p, const int* d_list, const std::vector<int>& list, double* c_out,
                          cudaStream_t st);
int rom_upload_affine(romsad* rom);
// Tensor-core ROMSAD products (romsad_tc.cu).  rom_tc_prepare: BF16 copies of P and W at the current rank and
// the kernels' shared-memory limits on the current device; call it before any stream capture.  rom_tc_apply:
// z = v + W (U^T A_mu U)^{-1} P^T Sigma_s v for the plan's instances with FP32 vectors (pl.inv32 filled),
// projection and lift as BF16 mma.sync products with FP32 accumulation.
int rom_tc_prepare(romsad* rom, cudaStream_t st);
int rom_tc_apply(RomPlan& pl, rte_problem* p, const int* d_active, const float* v, float* z, cudaStream_t st);
// Before the first rom_tc_apply of a plan (and before any stream capture): rom_tc_prepare, the plan's partial
// and coefficient buffers, and the FP32 copy of its inverses (pl.inv32 from pl.lu).
int rom_tc_plan_setup(RomPlan& pl, cudaStream_t st);
int rom_build_operators_from_U(romsad* rom, rte_problem* tmpl, int inst, cudaStream_t st);
}  // namespace rte
