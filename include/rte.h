/*
 * rte.h -- C ABI of the GB300 (sm_103a) FGMRES-ROMSAD solver for the steady
 * one-group parametric radiative transfer equation (arXiv 2410.08735).
 *
 * Method (paper sections cited per call):
 *   Sec. 2    S_N discrete ordinates (Chebyshev-Legendre product rule in 2D,
 *             Gauss-Legendre in the 1D slab) and upwind DG with the orthonormal
 *             Q^1 basis (P^1 in 1D): (D_j + Sigma_t) psi_j = Sigma_s phi + G + g_j^bc.
 *   Sec. 3    memory-efficient form: A~ phi = (I - T Sigma_s) phi = b~,
 *             T = sum_j omega_j (D_j + Sigma_t)^{-1}, b~ = sum_j omega_j (D_j + Sigma_t)^{-1} G~_j.
 *   Sec. 4    ROMSAD preconditioner M_ROM^{-1} = I + W (U_r^T A U_r)^{-1} P^T Sigma_s,
 *             P = sum_j U_{r,j}, W = sum_j omega_j U_{r,j}; FGMRES (Alg. 1); greedy
 *             ROM construction (Sec. 4.4.2) with MGS truncation (appendix B).
 *
 * Conventions shared by every call:
 *   - Every call returns an int status (RTE_OK = 0 or one of RTE_ERR_*);
 *     rte_status_string() names it and rte_last_error() gives a thread-local
 *     detail message for the last failing call of the calling thread.
 *   - A problem holds B parameter instances, each on its own uniform Cartesian
 *     mesh.  A "scalar vector" concatenates the instances: instance b occupies
 *     [off_b, off_b + N_b) with N_b = nx_b*ny_b*nd (nd = 4 in 2D, 2 in 1D); the
 *     offsets are returned by rte_problem_offsets().  Inside an instance the
 *     layout is cell-major, cells row-major (c = iy*nx + ix), local dof
 *     k = a + 2b for the basis p_a(x) q_b(y) (orthonormal Legendre).
 *   - An "angular vector" (rte_sweep output) holds, per instance, N_Omega
 *     consecutive scalar vectors: instance b occupies [N_Omega*off_b, N_Omega*off_{b+1}),
 *     direction j at N_Omega*off_b + j*N_b, directions in the paper's index
 *     order j = (j2-1) N_theta + j1.
 *   - Data pointers are caller-owned.  Unless a call says otherwise they are
 *     DEVICE pointers (e.g. torch CUDA tensors, contiguous), of the type given
 *     by the dtype argument (RTE_F64: double, RTE_F32: float).  Host arrays
 *     in descriptors and parameter setters are copied before the call returns.
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls that return results to the host synchronise that stream.
 *   - Handles (rte_problem_t, romsad_t, rte_mlp_t) own their device memory;
 *     destroy them once no call on them is in flight.  A handle is not
 *     thread-safe: serialise calls on the same handle.
 */
#ifndef RTE_GB300_H
#define RTE_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define RTE_OK 0
#define RTE_ERR_INVALID_ARG 1   /* bad pointer, size, enum or mesh mismatch          */
#define RTE_ERR_CUDA 2          /* a CUDA runtime call failed (detail in last_error) */
#define RTE_ERR_OOM 3           /* device allocation failed                           */
#define RTE_ERR_NOT_CONVERGED 4 /* solver hit max_iter; outputs and stats written     */
#define RTE_ERR_NUMERIC 5       /* NaN/Inf met (e.g. in beta or a Hessenberg column)   */
#define RTE_ERR_TIMEOUT 6       /* a bounded device wait gave up                      */
#define RTE_ERR_UNSUPPORTED 7   /* valid request this build does not implement        */
#define RTE_ERR_IO 8            /* checkpoint file could not be read or written       */

/* arithmetic type of the vectors handed to a call */
#define RTE_F64 0
#define RTE_F32 1
#define RTE_F64_DF 2   /* FP64 vectors, sweep arithmetic in double-float (pairs of FP32 numbers, ~48
                          significant bits): accepted by rte_apply_op only (the refinement residual of the
                          mixed-precision solves, run on the FP32 pipe) */

const char* rte_status_string(int status);
const char* rte_last_error(void);
/* Library version; safe without a GPU. */
int rte_version(int* major, int* minor);
/* Number of CUDA kernels this library has launched in this process (monotonic counter). */
long long rte_kernel_launches(void);
/* Measured fused multiply-add throughput of the current device (no paper counterpart: the denominator of
 * the roofline fractions of the ALU-bound sweep kernels).  dtype RTE_F32 or RTE_F64; *tflops = the best
 * of three timed launches (after one warm-up) of a kernel whose threads run eight independent FMA chains
 * each, 2 flop per FMA, on a grid of 8 blocks of 256 threads per SM.  Synchronises the stream. */
int rte_fma_peak(int dtype, double* tflops, void* stream);

/* ----------------------------------------------------------------- problem */
typedef struct rte_problem_desc {
    int dim;               /* 1 (slab, Sec. appendix A geometry) or 2 (X-Y, Sec. 2)        */
    int n_instances;       /* B >= 1                                                        */
    const int* nx;         /* [B] cells in x, host                                          */
    const int* ny;         /* [B] cells in y, host (ignored in 1D)                          */
    double box[4];         /* domain x0, x1, y0, y1 (y ignored in 1D)                       */
    int n_polar;           /* 1D: Gauss-Legendre points in mu; 2D: GL points in Omega_z     */
    int n_azim;            /* 2D: Chebyshev azimuthal points N_theta (even); 1D: ignored    */
    int rx, ry;            /* region grid, R = rx*ry equal blocks (ry = 1 in 1D)            */
    const double* sigma_s; /* [B][R] host: scattering cross section per region (>= 0)       */
    const double* sigma_a; /* [B][R] host: absorption cross section per region (>= 0)       */
    double src_q;          /* isotropic source value inside src_box, 0 outside (eq. 1 G)    */
    double src_box[4];     /* xa, xb, ya, yb                                                */
    double inflow_g;       /* isotropic inflow value g on all inflow boundaries (eq. 1c)    */
    int src_kind;          /* RTE_SRC_BOX (src_q on src_box) or RTE_SRC_GAUSS (2D):
                              G = A exp(-a ((x-xc)^2 + (y-yc)^2)), src_gauss = (A, a, xc, yc),
                              projected in closed form (erf / exp differences per cell)      */
    double src_gauss[4];
    int inflow_faces;      /* faces carrying the inflow g: 0 = every boundary face, else a mask of
                              RTE_FACE_XLO | RTE_FACE_XHI | RTE_FACE_YLO | RTE_FACE_YHI (a 1D slab has
                              x- and x+ only); the other faces are vacuum (the paper's two-material
                              problem has inflow on the left face only, Sec. 5)              */
    int sigma_modes;       /* RTE_SIGMA_REGIONS: sigma_s, sigma_a constant on each region (diagonal
                              Sigma).  RTE_SIGMA_VARSCAT (2D, rx*ry = 2, every instance on the same
                              mesh): the two entries per instance are coefficients c_0, c_1 of
                              sigma(x, y) = c_0 f(x, y) + c_1 with f = r^4 (2 - r^2)^2 in the unit disc
                              and 1 outside, the variable-scattering problem of Sec. 5.  Sigma_s and
                              Sigma_t are then full 4x4 blocks per cell, (Sigma)_kl = int_T sigma eta_k
                              eta_l (Sec. 2.3), integrated with 16 x 16 Gauss-Legendre points per cell.
                              The DSA preconditioner takes the cell means of the cross sections.  Not
                              available in this mode: double-float sweeps (the mixed solves' refinement
                              residuals are FP64), the tensor-core ROM products, rte_apply_op_noalloc,
                              the band sweep kernels (the warp-per-task kernel runs)            */
} rte_problem_desc;
#define RTE_SIGMA_REGIONS 0
#define RTE_SIGMA_VARSCAT 1
#define RTE_FACE_XLO 1
#define RTE_FACE_XHI 2
#define RTE_FACE_YLO 4
#define RTE_FACE_YHI 8
#define RTE_SRC_BOX 0
#define RTE_SRC_GAUSS 1

typedef struct rte_problem* rte_problem_t;

typedef struct rte_problem_info {
    int dim, n_instances, n_directions, n_unique_directions, dofs_per_cell, n_regions;
    long long n_dof_total;     /* sum_b N_b                                       */
    long long n_angular_total; /* N_Omega * n_dof_total (rte_sweep output length) */
} rte_problem_info;

/* Build quadrature, geometry, region maps and the per-instance source on the device
 * (Sec. 2.1-2.3).  Returns RTE_ERR_INVALID_ARG for dim not in {1,2}, B < 1, a mesh
 * with fewer than 1 cell, a region grid that does not divide every mesh, an odd
 * n_azim, or negative cross sections.  With N_theta = 2 mod 4 two azimuths sit at pi/2 and
 * 3pi/2; their Omega_x is the FP64 cos of those angles (a rounding error of order 1e-16, not
 * exactly 0), and they are swept in the quadrant of its sign. */
int rte_problem_create(const rte_problem_desc* desc, rte_problem_t* out);
int rte_problem_destroy(rte_problem_t p);
int rte_problem_get_info(rte_problem_t p, rte_problem_info* info);
/* offsets: host array [B+1], off_0 = 0, off_B = n_dof_total. */
int rte_problem_offsets(rte_problem_t p, long long* offsets);
/* New material parameters mu = (sigma_s, sigma_a) per instance without rebuilding
 * (Sec. 4.1 parametric problem).  Host arrays [B][R], copied. */
int rte_problem_set_params(rte_problem_t p, const double* sigma_s, const double* sigma_a);
/* Per-instance inflow value g_b on the problem's inflow faces (host [B], copied), replacing the descriptor's
 * inflow_g: a parametric boundary condition (Sec. 5, two-material problem, b~ affine in the inflow). */
int rte_problem_set_inflow(rte_problem_t p, const double* g);

/* --------------------------------------------------------- transport (Sec. 3) */
/* Angular-output sweep (Sec. 3.1, eq. SI-equation): for every direction j,
 * psi_j = (D_j + Sigma_t)^{-1} (src + with_bc * g_j^bc).  src: scalar vector;
 * psi: angular vector (see conventions).  Directions with the same (Omega_x,
 * Omega_y) give identical psi_j and are computed once. */
int rte_sweep(rte_problem_t p, int dtype, const void* src, int with_bc, void* psi, void* stream);
/* phi = Q psi = sum_j omega_j psi_j (Sec. 2.3). psi: angular vector, phi: scalar vector. */
int rte_scalar_flux(rte_problem_t p, int dtype, const void* psi, void* phi, void* stream);
/* phi = T s = sum_j omega_j (D_j + Sigma_t)^{-1} s (eq. memory-efficient-SI), fused, psi never stored. */
int rte_apply_T(rte_problem_t p, int dtype, const void* s, void* phi, void* stream);
/* w = A~ z = z - T (Sigma_s z) (eq. memory-efficient-rte), fused.  dtype RTE_F64_DF: z and w are FP64, the
 * sweep and the sum of its partial fluxes run in double-float and z - (.) in FP64 (relative error ~1e-14). */
int rte_apply_op(rte_problem_t p, int dtype, const void* z, void* w, void* stream);
/* btilde = sum_j omega_j (D_j + Sigma_t)^{-1} (G + g_j^bc) (eq. memory-efficient-SI). */
int rte_rhs(rte_problem_t p, int dtype, void* btilde, void* stream);
/* Pin the sweep kernel of the operator applies and sweeps of p (no paper counterpart: a testing and tuning
 * aid): variant 0 = one CTA per task with one warp per 32-row band, 1 = one warp per task, 2 = persistent CTAs
 * that pipeline runs of tasks through the bands (operator applies only; angular output falls back to 0), with
 * directions_per_warp in {1, 2, 4, 8} dividing every quadrant's direction count; variant -1 returns to the
 * autotuner's choice.  tasks_per_run: tasks one CTA of the pipelined variant sweeps back to back (at most 64;
 * 0: chosen to fill about two CTAs per SM).  Band variants need meshes of at most 256 rows (RTE_ERR_INVALID_ARG
 * otherwise).  Call it before the first solve on p: the task lists and buffers of captured iteration graphs are
 * sized then. */
int rte_problem_set_sweep_variant(rte_problem_t p, int variant, int directions_per_warp, int tasks_per_run);
/* Allocation-free form of rte_apply_op (the paper has no counterpart; this is a deployment aid).
 * Computes the same w = z - T (Sigma_s z), but allocates no device memory: no cudaMalloc, cudaFree or
 * allocating library routine is called.  It is meant for callers that cannot allocate, for example a
 * host code whose own pool allocator owns all device memory, or a solver step issued where an implicit
 * device synchronisation of cudaMalloc is not acceptable.  Its scratch (sweep task list and per-task
 * partial scalar fluxes) lives in one fixed 16 MiB __device__ array that every GPU which loads the
 * library holds until the process exits; a problem needing more returns RTE_ERR_INVALID_ARG (use
 * rte_apply_op).  All calls share that array, so calls that overlap on the GPU (different streams,
 * threads or processes sharing the context) race: serialise them.  Nothing in the array needs to start
 * at zero: every call rewrites the parts it reads.  Every call looks up the array's device address
 * (cudaGetSymbolAddress) on the current device; the first call on a device may load the library's
 * module there, and the first launch of each kernel variant may load its code (device memory the driver
 * takes, not this entry point), so make a first call of the same shape before any stream capture or
 * allocation-free region.  Directions per warp: the value the
 * sweep autotuner chose for this precision (after rte_apply_op or a solve on the same problem) when its
 * scratch fits, else the smallest value whose scratch fits (FP64: at most 4).  The problem handle itself
 * must have been created beforehand (rte_problem_create allocates).  Results agree with rte_apply_op up to
 * the order of the partial sums. */
int rte_apply_op_noalloc(rte_problem_t p, int dtype, const void* z, void* w, void* stream);

/* ----------------------------------------------------------- ROMSAD (Sec. 4) */
typedef struct romsad* romsad_t;

/* ROM from an orthonormal basis U_r given on the HOST as [r][N_Omega][N_b] doubles
 * (1 <= r <= 64) for the mesh of instance `instance` of tmpl.  The library forms P, W and the
 * affine reduced operators A_D, T_R, S_R (Sec. 4.1):
 *   U^T A_mu U = A_D + sum_R (sigma_a,R + sigma_s,R) T_R - sum_R sigma_s,R S_R. */
int romsad_create_from_basis(rte_problem_t tmpl, int instance, int r, const double* U_host, romsad_t* out);

typedef struct romsad_greedy_opts {
    int window;           /* w: FGMRES iterations whose corrections enter the ROM (Sec. 4.3)  */
    int max_greedy_iter;  /* N_g-iter                                                         */
    int max_rank;         /* cap on r (at most 64)                                            */
    double eps_rom;       /* stop when max relative indicator R_mu/||eta_mu^(0)|| < eps_rom   */
    double eps_qr;        /* appendix B truncation, relative to the snapshot norm (1e-13)     */
    int mu1;              /* index of the first sample, or -1: nearest the centroid of
                             (log sigma_s, sigma_a) over the training set                    */
    double hf_rtol;       /* relative residual of the high-fidelity FGMRES of step 2(a)      */
    int hf_restart;       /* restart length of that solve                                    */
    int hf_max_iter;
    int indicator_f32;    /* 1: evaluate the eq. rom-residual indicator in FP32 (it only decides the
                             argmax sample); 0: FP64                                           */
    int hf_dsa;           /* 1: the high-fidelity solves of step 2(a) are FGMRES-DSA (partially consistent DSA
                             through one V-cycle from the first iteration, 2D), the paper's solver there;
                             the xi recurrence uses the recorded z = M^{-1} v.  0: FGMRES with M = I */
} romsad_greedy_opts;

typedef struct romsad_report {
    int n_sampled;
    int* sampled;          /* caller array [max_greedy_iter] or NULL: training indices in order */
    double* max_indicator; /* caller array [max_greedy_iter] or NULL: entry i = the largest error
                              indicator over the training set after sample i was added; NaN where
                              it was not evaluated (the iteration cap ended the greedy first)   */
    int rank;
    double* labels;        /* caller array [n_train][max_rank] or NULL: Galerkin coefficients
                              c_mu of eq. greedy-rom on the final basis (MLP labels)           */
} romsad_report;

/* Greedy ROM construction (Sec. 4.4.2) on the GPU for the mesh of instance 0 of
 * tmpl, over n_train parameter points (host arrays [n_train][R]).  tmpl's own
 * parameters are left unchanged. */
int romsad_build_greedy(rte_problem_t tmpl, int n_train, const double* train_sigma_s,
                        const double* train_sigma_a, const romsad_greedy_opts* opts,
                        romsad_t* out, romsad_report* report);
int romsad_rank(romsad_t rom, int* r);
/* Copy the basis to the host as [r][N_Omega][N] doubles. */
int romsad_get_basis(romsad_t rom, double* U_host);
/* Reduced operator U^T A_mu U (affine assembly) for per-region sigma (host [R]) -> host [r][r]. */
int romsad_reduced_operator(romsad_t rom, const double* sigma_s, const double* sigma_a, double* A_host);
/* Galerkin coefficients of eq. greedy-rom for every instance of p (all on the ROM's mesh) with its own mu:
 * c_mu = (U^T A_mu U)^{-1} P^T Sigma_s b~_mu (the first-correction coefficients, Sec. 4.4.1-4.4.2; the MLP's
 * labels).  c_host: host [B][r].  Synchronises the legacy stream. */
int romsad_galerkin_coefficients(romsad_t rom, rte_problem_t p, double* c_host);
/* z = M_ROM^{-1} v for every instance of p (all instances must use the ROM's mesh),
 * eq. rom-sa-preconditioner, with the instance's own sigma.  v, z: scalar vectors.
 * dtype RTE_F64: FP64 products on the CUDA cores.  dtype RTE_F32: FP32 vectors; the instances share P and W,
 * so the projection P^T Sigma_s V and the lift W C are matrix products over the instances, run on the tensor
 * cores (mma.sync m16n8k16, BF16 operands, FP32 accumulation, chunk sums in a fixed order), the reduced solve
 * with the FP32-rounded inverse of U^T A_mu U.  Synchronises the stream. */
int romsad_apply(romsad_t rom, rte_problem_t p, int dtype, const void* v, void* z, void* stream);
int romsad_save(romsad_t rom, const char* path);
int romsad_load(const char* path, romsad_t* out);
int romsad_destroy(romsad_t rom);

/* ------------------------------------------------------------ FGMRES (Alg. 1) */
#define RTE_POST_ROM 0       /* keep M_ROM after the window (a fixed linear operator) */
#define RTE_POST_IDENTITY 1  /* z = v after the window                                */
#define RTE_POST_DSA 2       /* the DSA preconditioner after the window, as in eq.
                                ROMSAD-preconditioner (rte_dsa_apply; 2D meshes); with
                                roms = NULL (or for instances without a ROM) DSA from the
                                first iteration: right-preconditioned GMRES-DSA         */
#define RTE_MODE_FP64 0      /* every sweep, MGS and least squares in FP64             */
#define RTE_MODE_MIXED 1     /* FP64 iterative refinement (FP64 b~, residuals and update)
                                around inner FGMRES solves that run entirely in FP32:
                                sweeps, ROM products, Krylov basis, MGS and Givens     */
#define RTE_MODE_MIXED_F64KRYLOV 2   /* the same refinement, inner solves with FP32 sweeps
                                        (and per-direction partial fluxes) but FP64 Krylov
                                        vectors, ROM products, MGS and Givens           */

/* ---------------------------------------------------------- DSA (appendix A) */
/* Diffusion synthetic acceleration consistent with the upwind DG discretisation, the paper's
 * preconditioner after the ROMSAD window (eq. ROMSAD-preconditioner, appendix A), extended to the
 * 2D X-Y geometry axis by axis.  Per axis d: central-flux and jump operators D_C,d and D_J,d (exterior
 * traces zero on the boundary), with D_j = sum_d Omega_d (D_C,d - sign(Omega_d)/2 D_J,d).  From the
 * 0th and first angular moments of the correction equation with a P1 angular shape, eliminating the
 * current dJ:
 *   K = Sigma_a - sum_d kappa_d D_J,d - sum_d 3 mu2_d^2 D_C,d B_d^{-1} D_C,d,
 *   mu2_d = sum w Omega_d^2, kappa_d = sum_{Omega_d>0} w Omega_d, c_de = sum w Omega_d^2 |Omega_e|;
 *   RTE_DSA_PARTIAL: B_d = 3 mu2_d Sigma_t (the partially consistent DSA of appendix A);
 *   RTE_DSA_LUMPED:  B_d = the cell-diagonal blocks of 3 mu2_d Sigma_t - 3/2 sum_e c_de D_J,e (the fully
 *                    consistent first-moment operator lumped to its diagonal blocks; fewer
 *                    iterations on optically thick problems, unstable in optically thin, strongly
 *                    scattering cells).
 * M_DSA^{-1} v = v + x with x = one multigrid V-cycle applied to K x = Sigma_s v (the paper solves
 * this system by algebraic multigrid): 4x4 cell-block Jacobi on the DG level, continuous bilinear
 * elements on the same mesh and on meshes coarsened by 2 (Galerkin operators), one damped Jacobi step
 * per vertex level, a dense solve on the coarsest.  Covers 2D meshes whose cell counts, halved while
 * both are even, end with at most 100 vertices (RTE_ERR_UNSUPPORTED otherwise).  Arithmetic in FP32 for both
 * dtypes.  In the 1D slab (appendix A's own geometry) the systems are solved exactly instead, in FP64: the two
 * moment equations in the unknowns (dphi, dJ) per cell form a block-tridiagonal system with 4x4 blocks, factored
 * once per parameter set (block LU) and solved per apply; there RTE_DSA_FULL gives the fully consistent DSA,
 * RTE_DSA_PARTIAL and RTE_DSA_LUMPED the B_d above (2D: RTE_DSA_FULL is RTE_ERR_UNSUPPORTED). */
#define RTE_DSA_PARTIAL 0
#define RTE_DSA_LUMPED 1
#define RTE_DSA_FULL 2      /* fully consistent (the coupled dphi, dJ system), 1D slab only */
/* z = M_DSA^{-1} v for every instance of p with its own sigma.  v, z: scalar vectors of dtype
 * (device, not aliased).  Each call redoes the per-parameter set-up (two extra kernels) unless the variant is
 * or-ed with RTE_DSA_KEEP_SETUP, which reuses the set-up of the last call (RTE_ERR_INVALID_ARG if there was
 * none, or it was of the other variant); the caller guarantees the parameters have not changed since. */
#define RTE_DSA_KEEP_SETUP 16
int rte_dsa_apply(rte_problem_t p, int variant, int dtype, const void* v, void* z, void* stream);

/* ---------------------------------------- RBF-interpolated initial guess (Sec. 5) */
/* The interpolation baseline of the paper's experiments: the high-fidelity scalar fluxes phi_k of K sampled
 * parameters mu_k are interpolated in parameter space and the interpolant at an instance's mu is used as
 * its initial guess (fgmres_solve with phi0).  The paper does not state the kernel; this build uses
 * features x = (log sigma_s[R], sigma_a[R]) standardised by the samples' mean and standard deviation and
 * the polyharmonic cubic kernel |x - x_k|^3 with a degree-1 polynomial term, so that
 * phi0(mu) = sum_k w_k(mu) phi_k with the cardinal weights w(mu) = (A^{-1} [g(x); 1; x])[0:K],
 * A = [[Phi, P], [P^T, 0]], Phi_kl = |x_k - x_l|^3, P_k = (1, x_k), g_k(x) = |x - x_k|^3. */
typedef struct rte_rbf* rte_rbf_t;
/* tmpl: the mesh and region grid of the samples (its instance 0).  sigma_s, sigma_a: host [K][R]
 * (sigma_s > 0); solutions: [K][N] FP64 scalar fluxes on that mesh, device or host, copied.  Needs
 * K >= 2R + 2; RTE_ERR_NUMERIC if the interpolation system is singular. */
int rte_rbf_create(rte_problem_t tmpl, int K, const double* sigma_s, const double* sigma_a, const void* solutions,
                   rte_rbf_t* out);
/* phi0 (device FP64 scalar vector of p) = the interpolant at every instance's parameters; every instance
 * must use the samples' mesh and region grid, and have sigma_s > 0.  Synchronises the stream. */
int rte_rbf_initial_guess(rte_rbf_t rbf, rte_problem_t p, void* phi0, void* stream);
int rte_rbf_destroy(rte_rbf_t rbf);

/* ------------------------------------------------- learned warm start (MLP) */
/* A small MLP maps mu = (sigma_s[R], sigma_a[R]) of an instance to the r reduced-basis
 * coefficients c of eq. greedy-rom (labels from romsad_build_greedy).  Since the first FGMRES
 * correction satisfies delta phi = T Sigma_s xi = phi - b~ (eqs. density-relation, correction-fgmres1),
 * phi0 = b~ + W c_hat(mu) is a warm start.  Features: standardised (log sigma_s, sigma_a); layers
 * 2R -> hidden -> hidden -> r with the exact (erf) GELU; FP32 master weights, products with BF16-
 * rounded weights when bf16 = 1, FP32 accumulation; loss 0.5 ||y - c||^2 / r averaged; Adam.
 * Parameters are one flat FP32 array: W1 [hidden][2R], b1, W2 [hidden][hidden], b2, W3 [r][hidden], b3. */
typedef struct rte_mlp* rte_mlp_t;
typedef struct rte_mlp_train_opts {
    int epochs;          /* passes over the training set                      */
    int batch;           /* minibatch size (fixed order, last partial dropped) */
    double lr, beta1, beta2, eps;   /* Adam                                  */
    int bf16;            /* 1: BF16-rounded weights in the products           */
} rte_mlp_train_opts;
/* Weights uniform in +-1/sqrt(fan_in) from SplitMix64(seed), biases 0, standardisation identity. */
int rte_mlp_create(int n_in, int hidden, int n_out, unsigned long long seed, rte_mlp_t* out);
int rte_mlp_num_params(rte_mlp_t mlp, int* n);
/* flat: host [n_params]; mean/stdv: host [n_in] feature standardisation (NULL keeps the current). */
int rte_mlp_set_params(rte_mlp_t mlp, const float* flat, const float* mean, const float* stdv);
int rte_mlp_get_params(rte_mlp_t mlp, float* flat, float* mean, float* stdv);
/* Loss and gradient on the GPU for n samples: mu host [n][n_in], c host [n][n_out] -> loss, grad host [n_params]. */
int rte_mlp_loss_grad(rte_mlp_t mlp, int n, const double* mu, const double* c, int bf16, double* loss, float* grad);
/* Sets the standardisation from the training set, then Adam for the given epochs; final_loss over all n. */
int rte_mlp_train(rte_mlp_t mlp, int n, const double* mu, const double* c, const rte_mlp_train_opts* opts,
                  double* final_loss);
/* c_out host [n][n_out] = network(mu host [n][n_in]) with BF16-rounded weights. */
int rte_mlp_infer(rte_mlp_t mlp, int n, const double* mu, double* c_out);
int rte_mlp_destroy(rte_mlp_t mlp);
/* The ROM uses the MLP for the learned warm start (fgmres_opts.warm_start = 2); NULL detaches.
 * The MLP must outlive the ROM's use of it. */
int romsad_attach_mlp(romsad_t rom, rte_mlp_t mlp);

typedef struct fgmres_opts {
    int restart;             /* m of Alg. 1 (Krylov vectors per cycle)                */
    double rtol;             /* FP64 mode: ||r||/||b~|| target; mixed: FP64 true residual target */
    int max_iter;            /* cap on Arnoldi iterations (summed over restarts / outer steps) */
    int window;              /* w of eq. ROMSAD-preconditioner                        */
    int post_mode;           /* RTE_POST_ROM, RTE_POST_IDENTITY or RTE_POST_DSA        */
    int mode;                /* RTE_MODE_FP64, RTE_MODE_MIXED or RTE_MODE_MIXED_F64KRYLOV */
    double inner_rtol;       /* mixed: relative target of each inner solve (1e-2 is a good
                                default: FP32 rounding of I - T Sigma_s limits the inner
                                solves of strongly scattering instances near 1e-3)     */
    int max_outer;           /* mixed: cap on refinement steps; an instance still above
                                rtol after it, or whose refinement step cut its FP64
                                residual by less than max(1/4, sqrt(inner_rtol)), is
                                finished by FP64 FGMRES from its current iterate       */
    int true_residual_check; /* FP64 mode: recompute b~ - A~ phi after convergence     */
    int warm_start;          /* 0: zero initial guess; 1: phi0; 2: learned phi0 = b~ + W c_hat(mu)
                                from each instance's ROM MLP (instances without one start at 0;
                                so does an instance whose learned start is not finite: plain
                                ROMSAD is the fallback) */
    int learned_slot;        /* 1: with a zero start, the first ROMSAD apply takes its reduced
                                coefficients from each instance's ROM MLP (c_hat(mu) / ||b~||)
                                instead of the reduced solve (instances without an MLP, or with a
                                non-finite prediction, keep the plain apply)               */
    int dsa_variant;         /* RTE_POST_DSA: RTE_DSA_PARTIAL or RTE_DSA_LUMPED            */
    int rom_bf16;            /* RTE_MODE_MIXED: 1 = the ROMSAD applies of the inner (FP32) solves take
                                their projection and lift on the tensor cores (BF16 operands, FP32
                                accumulation, as romsad_apply with RTE_F32); 0 = FP32 CUDA-core
                                products fused into the Arnoldi step                           */
    int refine_residual;     /* mixed: precision of the refinement residuals b~ - A~ phi that steer the
                                inner solves.  RTE_RESIDUAL_DF (0): double-float sweeps (~1e-14 relative,
                                on the FP32 pipe), except for a step predicted to converge; a residual that
                                meets rtol is always recomputed by an FP64 sweep before the instance stops,
                                so convergence is certified in FP64.  RTE_RESIDUAL_FP64 (1): every residual
                                an FP64 sweep.  b~ is FP64 in both.                              */
} fgmres_opts;
#define RTE_RESIDUAL_DF 0
#define RTE_RESIDUAL_FP64 1

typedef struct fgmres_stats {
    int status;              /* RTE_OK or RTE_ERR_NOT_CONVERGED / RTE_ERR_NUMERIC      */
    int iterations;          /* Arnoldi iterations (all cycles and outer steps)        */
    int sweeps;              /* operator applies counted as in Sec. 5 (1 + iterations
                                with a zero guess; +1 per restart / nonzero guess)   */
    int sweeps_fp64;         /* of which in FP64                                       */
    int sweeps_df;           /* of which in double-float (mixed refinement residuals)  */
    int restarts;
    int outer;               /* mixed: refinement steps                                */
    int escalated;           /* mixed: 1 if the instance was finished by FP64 FGMRES   */
    int learned_start;       /* 1 if the learned warm start was used (warm_start = 2); 0 if
                                the instance had no MLP or its learned start was not finite,
                                so it started from zero (plain ROMSAD) */
    int learned_slot;        /* 1 if the learned ROMSAD-slot correction was used            */
    double est_rel_residual; /* last Givens estimate |g_{j+1}| / ||b~||                */
    double true_rel_residual;/* ||b~ - A~ phi||_2 / ||b~||_2 in FP64 (NaN if not computed) */
    double true_linf_residual;
} fgmres_stats;

/* Solve A~_b phi_b = b~_b for every instance b (Alg. 1, restarted).  roms: NULL (no
 * preconditioner, M_j = I) or an array [B] of ROM handles (NULL entries allowed),
 * roms[b] built on instance b's mesh.  phi0: scalar vector (FP64, device) or NULL.
 * phi: scalar vector, FP64; may be a DEVICE or HOST pointer (detected): with a host
 * pointer the result is copied back and the stream synchronised.  stats: host [B].
 * Returns RTE_ERR_NOT_CONVERGED if any instance missed its target. */
int fgmres_solve(rte_problem_t p, const romsad_t* roms, const fgmres_opts* opts, const void* phi0,
                 void* phi, fgmres_stats* stats, void* stream);

/* Source iteration with synthetic acceleration, SI-ROMSAD (Sec. 3.1-3.2, eq. preconditioned-richardson):
 * phi <- phi + M_l^{-1} (b~ - A~ phi), with M_l = M_ROM for the first opts->window iterations on
 * instances with a ROM, then opts->post_mode (RTE_POST_DSA: SI-DSA; RTE_POST_ROM: the ROM throughout;
 * RTE_POST_IDENTITY: classical SI).  Instances without a ROM take DSA from the first iteration when
 * post_mode is RTE_POST_DSA, no correction otherwise.  Stops when ||b~ - A~ phi||_2 <= rtol ||b~||_2 or
 * after max_iter iterations.  Uses opts->rtol, max_iter, window, post_mode, dsa_variant; mode must be
 * RTE_MODE_FP64 (RTE_ERR_UNSUPPORTED otherwise); the other fields are ignored.  Arguments as for
 * fgmres_solve; stats: iterations, sweeps (b~ plus one per residual: a zero start takes r = b~), status,
 * true residuals of the returned phi. */
int si_solve(rte_problem_t p, const romsad_t* roms, const fgmres_opts* opts, const void* phi0, void* phi,
             fgmres_stats* stats, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RTE_GB300_H */
