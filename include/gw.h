/*
 * gw.h -- C ABI of the GB300 contour-deformation G0W0 library (libgw.so).
 *
 * Method: arXiv 2107.10423, "Scalable Molecular GW Calculations: Valence and
 * Core Spectra".  Closed-shell G0W0 in an orthonormal (Coulomb-metric)
 * auxiliary basis (Sec. 3.1): the input is the fitted three-index tensor
 * B_{P,pq} = (P|pq) restricted to the two slices the method touches:
 *
 *   B_ia : [n_aux][n_occ*n_virt], row-major, pair index ia = i*n_virt + a
 *          (i occupied, a virtual).  Builds Pi (Sec. 3.3, equation after
 *          "wauxbas").
 *   B_nm : [n_targets][n_bas][n_aux], row-major: the rows b_nm = (P|nm) of
 *          each target state n against every state m.  W_nm enters Sigma_nn
 *          (eqs. "inn" and "rnn").
 *
 * All energies are in Hartree.  KS energies eps[n_bas] are ascending, the
 * first n_occ occupied (closed shell, n_bas = n_occ + n_virt).
 *
 * Ownership: the caller owns every array it passes.  gw_plan_create copies
 * the inputs into device memory owned by the plan, unless
 * GW_BORROW_DEVICE_PTRS is given (then B_ia and B_nm must be device pointers
 * that stay valid until gw_plan_destroy).  Output arrays are host arrays
 * that the caller allocates.  Every call returns a gw_status; no call aborts
 * or throws.  A plan is used by one host thread at a time; work runs on the
 * stream given at creation (or a stream the plan creates).  Every call
 * synchronises that stream before returning.
 */
#ifndef GW_H
#define GW_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GW_OK = 0,
  GW_ERR_ARG = 1,              /* bad argument (sizes, NULL pointers, unsorted energies) */
  GW_ERR_OOM = 2,              /* device allocation failed */
  GW_ERR_CUDA = 3,             /* a CUDA call or kernel failed; see gw_last_error */
  GW_ERR_NOT_CONVERGED = 4,    /* a solver stopped at its iteration cap (results still written) */
  GW_ERR_TIMEOUT = 5,          /* a bounded device wait ran out */
  GW_ERR_UNIMPLEMENTED = 6,
  GW_ERR_NUMERIC = 7           /* a factorisation met a non-positive pivot, or NaN input */
} gw_status;

typedef enum {
  GW_PREC_FP64 = 0,            /* every step in FP64 */
  GW_PREC_MIXED = 1            /* Pi and the W table on tcgen05 tensor cores with BF16 hi+lo split
                                  products (FP32 accumulate); MINRES operator in FP32, Lanczos
                                  recurrences, quadrature and QP search in FP64 */
} gw_precision;

typedef enum {
  GW_QP_LINEARISED = 0,        /* one Newton step from eps_n (Sec. 3.4) */
  GW_QP_STEPTREE = 1,          /* iterative solver with the step-selection tree (Sec. 3.4, Fig. "steptree") */
  GW_QP_GRAPHICAL = 2          /* graphical solution (Sec. 3.4): f(w) = e_n + Sigma_x - V_xc + Re Sigma_c(w) - w on
                                  qp_window_points evenly spaced points of [e - qp_window, e + qp_window] around the
                                  starting point e (all points of all targets in one batched evaluation); the sign
                                  change with f decreasing closest to e, by linear interpolation, refined by the
                                  step tree; a state whose window holds no such change is not converged */
} gw_qp_mode;

/* Flags for gw_plan_create. */
#define GW_INPUT_ON_DEVICE     1u   /* B_ia and B_nm are device pointers (copied device-to-device) */
#define GW_BORROW_DEVICE_PTRS  2u   /* B_ia and B_nm are device pointers used in place (not copied) */

typedef struct {
  int n_occ, n_virt, n_aux;    /* sizes; n_bas = n_occ + n_virt */
  int n_freq;                  /* imaginary grid points (modified Gauss-Legendre, Sec. 3.3) */
  double x0;                   /* grid scale: xi = x0 (1+t)/(1-t) */
  double eta;                  /* real-axis broadening in Pi(x) (Ha) */
  int precision;               /* gw_precision */
  int minres_maxit;            /* MINRES iteration cap (paper default 25) */
  double minres_tol;           /* MINRES stop: ||r|| <= tol ||rhs|| (paper 5e-5) */
  double minres_fallback_tol;  /* dense solve if ||r||/||rhs|| > this after maxit (paper 1e-4) */
  int qp_maxit;                /* QP iterations (step tree) */
  double qp_tol;               /* QP convergence |f| < qp_tol (Ha) */
  int static_subtraction;      /* 1: I term with the W(0) sgn(a)/2 rewrite (exact); 0: literal quadrature */
  int max_rhs_batch;           /* residue right-hand sides per batched MINRES launch (0 = automatic) */
  int workspace_mb;            /* cap per large workspace class (frequency matrices, split operands,
                                  fallback matrices), MiB; 0 = 8192 */
  double refine_tol;           /* mixed: a dense-fallback solve whose first refinement correction (residual from the
                                  three-part tensor-core operator), relative to the solution in the 2-norm, exceeds
                                  refine_tol takes one more step with the residual from the FP64 operator
                                  (near-resonant, ill-conditioned residues); 0 = every solve, < 0 = none;
                                  default 1e-6 */
  int op_parts;                /* mixed: BF16 parts per operand of the MINRES operator: 2 (hi, lo: three products,
                                  about 2^-16 relative; default) or 3 (hi, mid, lo: six products, about
                                  FP32-accurate) */
  int deriv_fp64;              /* mixed: residue derivative pass y^T Pi'(x) y all in FP64 (1), or (0, default) FP32
                                  products with an FP64 reduction and FP64 terms for the pairs within 0.1 Ha of
                                  resonance (x = +-D_ia) */
  int refine_df;               /* mixed: the FP64-accurate refinement residual in double-float arithmetic (FP32
                                  pairs, 48-bit, on the FP32 pipes: 1, default) or in FP64 (0) */
  int tc_max_ctas;             /* mixed: cap on the persistent grid of the Pi kernel (CTAs, one per SM at most);
                                  0 = every SM.  A smaller grid leaves SMs to work that runs beside it */
  double qp_window;            /* graphical mode: half width of the search window (Ha), default 0.5 */
  int qp_window_points;        /* graphical mode: points per window (>= 2), default 64 */
  double qp_cluster_gap;       /* cluster layer (Sec. 3.4; step tree and graphical modes): targets whose KS energies are
                                  within this distance (Ha) of a neighbour in energy form a cluster; the member with the
                                  lowest KS energy is solved first and the others start from their KS energy shifted
                                  by its QP correction.  0 = off (default) */
  int pi_ksplit;               /* mixed: K ranges per (tile, frequency) of the Pi kernel: 0 = autotuned per
                                  problem shape (n_aux, n_occ n_virt, batch; every feasible split timed once per
                                  process, the fastest kept; only shapes whose tiles do not fill the GPU split),
                                  or 1, 2, 4, 8 forced.  Default 0 */
} gw_config;

typedef struct gw_plan* gw_plan_t;

/* Fill *cfg with defaults: n_freq 128, x0 0.5, eta 1e-3, FP64, MINRES 25 / 5e-5 / 1e-4,
 * qp_maxit 50, qp_tol 1e-8, static_subtraction 1, refine_tol 1e-6, op_parts 2, deriv_fp64 0, refine_df 1,
 * qp_window 0.5, qp_window_points 64, qp_cluster_gap 0, tc_max_ctas 0, pi_ksplit 0.
 * Sizes are set to 0. */
void gw_config_default(gw_config* cfg);

/* Create a plan (Algorithm 1, Init).
 *   eps      [n_bas] host, ascending.
 *   B_ia     [n_aux][n_occ*n_virt]; B_nm [n_targets][n_bas][n_aux] (host unless flags say device).
 *   targets  [n_targets] host, state indices in [0, n_bas).
 *   vxc      [n_targets] host or NULL.  NULL means V_xc := Sigma_x, so e_QP = e + Re Sigma_c(e_QP).
 *   xi, wt   [n_freq] host imaginary grid and weights, or NULL for the built-in grid.
 *   stream   cudaStream_t to run on, or NULL for a plan-owned stream.
 * Computes Sigma_x_nn = -sum_i sum_P B_P,ni^2 (Algorithm 1, Init).
 * On failure *out is NULL and gw_last_error(NULL) describes the error. */
gw_status gw_plan_create(const gw_config* cfg, const double* eps, const double* B_ia, const double* B_nm,
                         const int* targets, int n_targets, const double* vxc, const double* xi,
                         const double* wt, unsigned flags, void* stream, gw_plan_t* out);

/* Create a plan for an open-shell (spin-unrestricted) system.  Both spins share the orbital basis
 * (n_bas = cfg->n_occ + cfg->n_virt) and the auxiliary basis; cfg->n_occ is the alpha occupation, n_occ_b the
 * beta one (cfg->n_virt = n_bas - n_occ_alpha).
 *   eps_a, eps_b  [n_bas] host, ascending per spin.
 *   B_ia_a        [n_aux][n_occ_a * (n_bas - n_occ_a)], B_ia_b [n_aux][n_occ_b * (n_bas - n_occ_b)]: the
 *                 occupied-virtual blocks of each spin (pair index i * n_virt + a within the spin).
 *   B_nm          [n_targets][n_bas][n_aux]: each target's rows b_nm in its own spin.
 *   targets, spins [n_targets] host: state index and spin (0 alpha, 1 beta) of every target.
 *   vxc, xi, wt, flags, stream, out as in gw_plan_create (GW_BORROW_DEVICE_PTRS is not accepted: the plan keeps its
 *   own copy of the two B_ia blocks side by side).
 * The polarizability sums the spin channels, Pi = sum_sigma sum_{ia in sigma} B B [1/(z - D + i eta) +
 * 1/(-z - D + i eta)] (Sec. 3.3; the closed shell is the case of two equal channels); Sigma_c, Sigma_x and the QP
 * equation of a target use the energies and occupations of its spin.  Every other call is as for gw_plan_create. */
gw_status gw_plan_create_uks(const gw_config* cfg, const double* eps_a, const double* eps_b, int n_occ_b,
                             const double* B_ia_a, const double* B_ia_b, const double* B_nm, const int* targets,
                             const int* spins, int n_targets, const double* vxc, const double* xi, const double* wt,
                             unsigned flags, void* stream, gw_plan_t* out);

/* Polarizability on the imaginary axis (Sec. 3.3, equation after "wauxbas", eta = 0):
 *   Pi_PQ(i xi) = -4 sum_ia B_P,ia B_Q,ia D_ia / (D_ia^2 + xi^2),  D_ia = e_a - e_i.
 * With xi != NULL: builds Pi for the n_xi given frequencies and, if pi_out != NULL, writes
 * them to pi_out [n_xi][n_aux][n_aux] (host, full symmetric).
 * With xi == NULL: runs the imaginary-axis stage of Algorithm 1 on the plan's grid: Pi(i xi_g)
 * for every grid point and xi = 0, the factorisation of eps(i xi) = 1 - Pi (SPD), and the
 * table W^c_nm(i xi_g) = b_nm^T [eps^-1 - 1] b_nm for every target n and state m (kept on the
 * device for gw_sigma_cd / gw_qp_solve); pi_out must then be NULL. */
gw_status gw_polarizability(gw_plan_t plan, const double* xi, int n_xi, double* pi_out);

/* Correlation self-energy by contour deformation (eqs. "R", "I", "inn", "rnn"):
 *   Re Sigma^c_nn(omega_n) = R_nn(omega_n) - I_nn(omega_n)
 * for every target n at its own frequency omega[n_targets] (host), with the omega-derivative.
 * Builds the imaginary-axis table first if gw_polarizability(plan, NULL, ...) has not run.
 * Residues by batched MINRES (with dense fallback).  sigma_x may be NULL.
 * Returns GW_ERR_NOT_CONVERGED if a residue solve stayed above minres_fallback_tol even after the
 * dense fallback (values are still written). */
gw_status gw_sigma_cd(gw_plan_t plan, const double* omega, double* sigma_c, double* dsigma_c,
                      double* sigma_x);

/* Sigma_c and its omega-derivative by spectral decomposition (Sec. 2.2 and 3.2, the Casida route the paper uses
 * for small systems): the Hermitian Casida problem D^1/2 (D + 4 B_ia^T B_ia) D^1/2 T = T Omega^2 over the pairs
 * (both spin channels for an open-shell plan) is diagonalised once per plan in FP64 (cyclic Jacobi, to 1e-13
 * relative off-diagonal norm), then
 *   Sigma_c(omega) = sum_m sum_s w_nms^2 / (omega - e_m +/- Omega_s -/+ i eta)  (upper signs for occupied m),
 *   w_nms = b_nm . V_s / sqrt(2 Omega_s),  V = 2 B_ia D^1/2 T.
 * target_idx[p] (or NULL: point p is target p, n_points = n_targets) and omega[p] (host); sigma_c, dsigma_c host
 * [n_points] (real parts), either may be NULL.  O(N_ov^3) work and 2 N_ov^2 doubles: GW_ERR_ARG above
 * N_ov = 16384; GW_ERR_NOT_CONVERGED if 40 Jacobi sweeps do not converge.  The Casida solution is kept until W's
 * energies change (evGW). */
gw_status gw_sigma_sd(gw_plan_t plan, int n_points, const int* target_idx, const double* omega, double* sigma_c,
                      double* dsigma_c);

/* Sigma_c and its omega-derivative at n_points arbitrary (target, frequency) pairs, all in one batched evaluation
 * (the same I term, residue list and batched MINRES as gw_sigma_cd; the graphical solution of Sec. 3.4 samples its
 * windows this way).  target_idx[p] in [0, n_targets), omega[p] in Ha (host, [n_points]); sigma_c, dsigma_c host
 * [n_points], either may be NULL.  GW_ERR_ARG for a bad index or a non-finite frequency. */
gw_status gw_sigma_points(gw_plan_t plan, int n_points, const int* target_idx, const double* omega, double* sigma_c,
                          double* dsigma_c);

/* Residue terms (eq. "rnn") for an explicit list of n_rhs right-hand sides:
 *   W_nm(x) = b_nm^T [(1 - Pi(x))^-1 - 1] b_nm,  Pi(x) = 2 sum_ia B B [1/(x-D+i eta) + 1/(-x-D+i eta)]
 * solved matrix-free by MINRES on the real symmetric 2 n_aux embedding of the complex-symmetric
 * system, for target_idx[k] (index into the plan's targets), state m[k] and real frequency x[k].
 * Outputs (host, [n_rhs]): w_re, w_im, dw_re = Re dW/dx, iters, resnorm (relative), used_fallback.
 * Any output pointer may be NULL. */
gw_status gw_residues_minres(gw_plan_t plan, int n_rhs, const int* target_idx, const int* m, const double* x,
                             double* w_re, double* w_im, double* dw_re, int* iters, double* resnorm,
                             int* used_fallback);

/* Quasiparticle energies (Sec. 3.4, eq. "qpeqn"): e_QP = e_n + Sigma_x - V_xc + Re Sigma^c(e_QP).
 * Outputs (host, [n_targets]): e_qp, z_factor = 1/(1 - dSigma^c/domega) at the solution, and
 * state_status (0 converged, 1 not converged, 2 converged but a residue used the dense fallback).
 * Returns GW_ERR_NOT_CONVERGED if any state did not converge. */
gw_status gw_qp_solve(gw_plan_t plan, gw_qp_mode mode, double* e_qp, double* z_factor, int* state_status);

/* Eigenvalue self-consistency (Algorithm 1, the outer loop over iter; Sec. 1: evGW0 updates the quasiparticle
 * energies in G, evGW in G and W).  Cycle 1 is G0W0 (gw_qp_solve).  After each cycle the energies are updated:
 * every target takes its QP energy; every other occupied state moves by the QP correction of the highest occupied
 * target and every other virtual state by that of the lowest virtual target (no move where a class has no target).
 * The next cycle evaluates Sigma_c with those energies as the poles of G (the I and R terms) and, if update_w != 0,
 * as the pair energies D_ia = e_a - e_i of Pi (a new imaginary-axis table and new residue operators); the QP
 * equation keeps the KS energy, e_QP = e_n + Sigma_x - V_xc + Re Sigma_c(e_QP), and each cycle's search starts from
 * the previous cycle's QP energy (mode as in gw_qp_solve; linearised = one Newton step per cycle).
 * Stops when no target moves by more than tol (Ha) between cycles, or after max_iter cycles.
 * Outputs (host, [n_targets]): e_qp, z_factor, state_status of the last cycle; *iterations = cycles run.
 * Returns GW_ERR_NOT_CONVERGED if the cycles did not converge (outputs still written).  On return the plan is
 * back to G0W0 (G and W from the KS energies).  Any output pointer may be NULL. */
gw_status gw_evgw(gw_plan_t plan, int update_w, gw_qp_mode mode, int max_iter, double tol, double* e_qp,
                  double* z_factor, int* state_status, int* iterations);

/* Sharding one job across ranks (one process and one GPU per rank; Algorithm 1's imaginary-grid loop and
 * per-state residue loop partitioned as independent work):
 *   * the imaginary-axis stage computes only this rank's block of the n_freq + 1 frequency positions
 *     (gw_shard_columns; position 0 is xi = 0, position p > 0 is grid point p - 1), zeroes the other columns of
 *     its W table and sums the tables of all ranks with allreduce_sum (every column comes from one rank);
 *   * each Sigma evaluation solves only the residue right-hand sides j of its list with j % world == rank and
 *     sums the per-target R and dR/domega (2 n_targets doubles) with allreduce_sum; the I term, the QP search and
 *     every other step run on every rank with the same summed values, so all ranks return the same results.
 * allreduce_sum(buf, n, ctx) must replace the host array buf[n] by its element-wise sum over the ranks (for
 * example through MPI or torch.distributed) and return 0 on success; it is called at the same points, with the
 * same n, on every rank.  world = 1 turns sharding off.  The table is rebuilt on the next call that needs it. */
typedef int (*gw_allreduce_fn)(double* buf, long long n, void* ctx);
gw_status gw_set_shard(gw_plan_t plan, int rank, int world, gw_allreduce_fn allreduce_sum, void* ctx);
/* The block [*p0, *p1) of frequency positions rank `rank` of `world` computes (host only): contiguous,
 * floor((n_freq + 1) r / world) to floor((n_freq + 1)(r + 1) / world). */
gw_status gw_shard_columns(int n_freq, int rank, int world, int* p0, int* p1);

/* Copy the imaginary-axis table to the host: out [n_targets][n_bas][n_freq + 1] with
 * out[t][m][g] = W^c_nm(i xi_g) for the grid points g < n_freq and out[t][m][n_freq] = W^c_nm(0)
 * (Algorithm 1, imaginary-grid loop).  Builds the table first if needed. */
gw_status gw_w_table(gw_plan_t plan, double* out);

/* Timing and counters accumulated since plan creation (host, milliseconds / counts).  ms_kernel and
 * flops_kernel are per kernel class, timed with CUDA events on the plan's stream:
 *   0 Pi on tensor cores (tcgen05, weights applied in the kernel)   1 Pi (SIMT)
 *   2 W-table factorisation (Cholesky of 1 - Pi, or the tensor-core Newton-Schulz inverse in mixed mode)
 *   3 W-table reduction (triangular solves, or the tensor-core GEMM into W)
 *   4 MINRES iterations (the operator GEMMs and, since the iterations run as one CUDA graph per batch, the
 *     recurrence steps; flops count the operator of the iterations that ran) and the derivative pass
 *   5 MINRES recurrences outside the graph (initialisation)  6 dense Pi(x) of fallback solves
 *   7 batched complex LU + solve                          8 residual operators of the mixed-precision refinement
 *                                                           (three-part tensor-core, and FP64 where selected)
 * flops_kernel counts algorithmic floating-point operations (a multiply-add is 2). */
#define GW_N_KERNEL_CLASSES 9
typedef struct {
  double ms_screening;         /* Pi + factorisation + W table (last build) */
  double ms_pi;                /* Pi build alone (last build) */
  double ms_sigma_imag;        /* I-term quadrature */
  double ms_residues;          /* batched MINRES + fallback */
  double ms_qp;                /* last gw_qp_solve */
  long long n_rhs_solved;      /* residue right-hand sides solved */
  long long n_minres_iters;    /* sum over right-hand sides */
  long long n_fallback;        /* dense fallback solves */
  long long n_sigma_evals;     /* Sigma(omega) evaluations (per target) */
  long long n_kernel_launches; /* kernels this plan launched */
  double ms_kernel[GW_N_KERNEL_CLASSES];
  double flops_kernel[GW_N_KERNEL_CLASSES];
  long long launches_kernel[GW_N_KERNEL_CLASSES];
  long long n_refine_fp64;     /* dense-fallback solves that took the FP64-operator refinement step */
  long long bytes_device;      /* device bytes the plan holds now (inputs it copied, their mixed-precision copies,
                                  the W table and every work-space buffer) */
  long long bytes_device_peak; /* largest bytes_device since plan creation */
  long long n_graph_launches;  /* CUDA graph launches (one per MINRES batch: all of its iterations) */
  int pi_ksplit_last;          /* K split of the last Pi-kernel launch (autotuned or forced) */
} gw_stats;
gw_status gw_get_stats(gw_plan_t plan, gw_stats* out);

/* Upper bound on the device bytes a plan with this configuration can hold (host only, no GPU needed), for
 * admission by HBM footprint: the inputs it copies (none of B_ia and B_nm with GW_BORROW_DEVICE_PTRS), their
 * mixed-precision copies, the W table, and every work-space class at the size cfg->workspace_mb caps it to (a class
 * whose single item is larger than the cap is counted at that item's size).  Work space that grows with a call's
 * own arguments is not included: gw_polarizability with explicit frequencies (n_xi matrices) and the right-hand-side
 * lists of gw_residues_minres beyond n_targets * n_bas entries.  *bytes receives the bound.  Returns GW_ERR_ARG for
 * NULL pointers or non-positive sizes. */
gw_status gw_plan_footprint(const gw_config* cfg, int n_targets, unsigned flags, unsigned long long* bytes);

/* The built-in imaginary-frequency grid (host only, no GPU needed): modified Gauss-Legendre
 * (Sec. 3.3, text after eq. "inn"): Legendre nodes t_k on [-1, 1] mapped by
 * xi_k = x0 (1 + t_k)/(1 - t_k), weights w_k = 2 x0 w_GL,k/(1 - t_k)^2, ascending.
 * xi, wt: [n] host arrays owned by the caller.  Returns GW_ERR_ARG for n <= 0, x0 <= 0 or NULL. */
gw_status gw_grid(int n, double x0, double* xi, double* wt);

/* W table from caller-supplied Cholesky factors, for callers that cannot allocate device memory.
 * The paper has no counterpart: this is the library's imaginary-axis triangular-solve step exposed as a
 * stand-alone call that allocates nothing (no cudaMalloc, cudaFree or allocating library routine).
 * Callers that cannot allocate include a serving process that hands all GPU memory to its own pool at
 * start-up, a host application whose allocator forbids cudaMalloc after initialisation, and latency-
 * critical paths where an allocation may synchronise the device.
 *   L   device, [n_mats][n_aux][n_aux] row-major lower Cholesky factors of eps(i xi_g) = 1 - Pi(i xi_g)
 *       (entries above the diagonal are not read).
 *   Bn  device, [n_rows][n_aux]: the vectors b_r (for example the B_nm rows of every target n and state m).
 *   W   device, written at W[r * w_ld + g] = b_r^T (eps_g^-1 - 1) b_r for r < n_rows, g < n_mats.
 *   stream: cudaStream_t (NULL = default stream).  The call is asynchronous on that stream.
 * Work space is a fixed 32 MiB device array inside the library; every GPU that loads the library holds it
 * until the process exits.  Limits: n_aux <= 65536 and n_mats <= 4096; larger sizes return GW_ERR_ARG
 * before any device work.  Fewer CTAs run when n_aux is large (the array holds one slice per CTA).
 * The first call on each device looks up the array's device address with cudaGetSymbolAddress and fills a
 * small index table with a synchronous copy; make that first call before any stream capture.
 * Every call on a device shares the same array.  Each call writes its slices before reading them, so nothing
 * has to start at zero, but two calls that overlap on the same GPU (for example on two streams) race. */
gw_status gw_w_table_noalloc(const double* L, int n_aux, int n_mats, const double* Bn, int n_rows, double* W,
                             int w_ld, void* stream);

/* Release every device buffer the plan owns.  NULL is ignored. */
void gw_plan_destroy(gw_plan_t plan);

/* Last error message of this plan (or of the last failed gw_plan_create when plan is NULL). */
const char* gw_last_error(gw_plan_t plan);

#ifdef __cplusplus
}
#endif
#endif /* GW_H */
