// Internal declarations of libgw: kernel launchers shared between translation units.
// Not part of the public ABI (include/gw.h).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>

namespace gw {

// ---------------------------------------------------------------- dense kernels (kernels_dense.cu)
// Every kernel below takes the pair energies D_k (k < n_ov, the columns of B) as an array Dk.
// Pi_PQ(i xi_g) = -4 sum_k B[P][k] B[Q][k] D_k/(D_k^2 + xi_g^2)  (Sec. 3.3, eta = 0), for n_xi points.
// mode 0 writes Pi, mode 1 writes eps = 1 - Pi.  out: [n_xi][n_aux][n_aux] full symmetric.
template <typename T>
void launch_pi_syrk(const T* B, const double* Dk, long n_ov, int n_aux, const double* xi, int n_xi, T* out, int mode,
                    cudaStream_t s);

// Dense complex real-axis matrix A = 1 - Pi(x) as two real [n_aux][n_aux] halves (dense fallback).
void launch_pi_complex_dense(const double* B, const double* Dk, long n_ov, int n_aux, double x, double eta, double* Ar,
                             double* Ai, cudaStream_t s);

// In-place lower Cholesky of `batch` SPD matrices A[b] = base + b*stride (row-major n x n).
// info[b] = 0 on success, j+1 if pivot j was not positive.
template <typename T>
void launch_cholesky(T* base, int n, long stride, int batch, int* info, cudaStream_t s);

// W table from Cholesky factors: for matrices g in [0, n_g): y = L_g^-1 b_r for rows r of Bn [R][n],
// W[r*w_ld + g_out[g]] = |y|^2 - |b|^2 = b^T(eps^-1 - 1)b.  scratch: [n_cta][n][64] elements of T.
template <typename T>
cudaError_t launch_trsm_w(const T* Lbase, long Lstride, int n, int n_g, const int* g_out, const T* Bn, int R,
                          double* W, int w_ld, T* scratch, int n_cta, cudaStream_t s);
template <typename T>
size_t trsm_w_scratch_elems(int n, int n_cta);
int trsm_w_default_ctas();

// Matrix-free operator of the residue systems (MINRES), for a batch of nr right-hand sides.
// V: [2nr][n_aux] pairs (u, v) encoding z = u - i v.
// gemm1: mode 0: U[2j..2j+1][k] = c_k(x_j) * t_k, t = B^T z, with c_k(x) = 2[1/(x-D_k+i eta) + 1/(-x-D_k+i eta)];
//   mode 2: dw[j] += sum_k Re(c'_k(x_j) t_k^2) in FP64, c' the x-derivative (dw zeroed by the caller, U unused), skipping the pairs
//   with |x_j - D_k| < cut or |-x_j - D_k| < cut (added by launch_deriv_resonant).
// gemm2: S[r][P] = sum_k U[r][k] B[P][k]; mode 0 writes S (= [Re; Im] of Pi z),
//   mode 1 writes the real embedding [u - S_re; -v - S_im] of (1 - Pi) z.
template <typename T>
void launch_op_gemm1(const T* V, const T* B, const double* Dk, long n_ov, int n_aux, const double* x, double eta,
                     int nr, T* U, int mode, cudaStream_t s, double* dw = nullptr,
                     double cut = 0.0, long ldb = 0,    // ldb: row length of B (0 = n_ov)
                     const int* run_if = nullptr);      // device flag: the launch does nothing if *run_if == 0
// Double-float (FP32 pair, 48-bit) versions of op_gemm1 mode 0 and op_gemm2 mode 1 for the refinement residual:
// V, U, out FP64; B as its split Bh + Bl (launch_df_split of the FP64 B_ia): Bh [n_aux][ldh] is the FP32 rounding
// of B (the plan's FP32 copy), Bl [n_aux][n_ov] the rounding of the remainder.  launch_df_split writes h only if it
// is not NULL.
void launch_df_split(const double* x, long n, float* h, float* l, cudaStream_t s);
void launch_op_gemm1_df(const double* V, const float* Bh, const float* Bl, long ldh, const double* Dk, long n_ov,
                        int n_aux, const double* x, double eta, int nr, double* U, cudaStream_t s);
void launch_op_gemm2_df(const double* U, const float* Bh, const float* Bl, long ldh, int n_aux, int n_ov, int nr,
                        const double* V, double* out, cudaStream_t s);
// The pairs that mode 2 skips, in FP64: dw[j] += Re(c'_k(x_j) t_k^2) with t from the FP64 rows of V64 and the FP64
// B_ia [n_aux][n_ov]; Dsort ascending pair energies with their pair indices kidx.
void launch_deriv_resonant(const double* V64, const double* B, long n_ov, int n_aux, const double* Dsort,
                           const int* kidx, const double* xs, int nr, double eta, double cut, double* dw,
                           cudaStream_t s);
template <typename T>
void launch_op_gemm2(const T* U, const T* B, int n_aux, int n_ov, int nr, const T* V, T* out, int mode,
                     cudaStream_t s, const int* run_if = nullptr);

// ---------------------------------------------------------------- CD kernels (kernels_cd.cu)
// Sigma_x of each target; occ_t (device [n_t], or NULL for n_occ everywhere): occupied states of its spin.
void launch_sigma_x(const double* B_nm, int n_t, int n_bas, int n_aux, int n_occ, double* sx, cudaStream_t s,
                    const int* occ_t = nullptr);

// I term (eq. "inn") with optional static subtraction, per target t at omega[t].
// n_t evaluation points; point t reads the W rows of target tmap[t] (t itself when tmap is NULL) and the G energies
// eps + spin[target] * n_bas (eps [n_spin][n_bas]; spin NULL: one set).
void launch_sigma_imag(const double* W, int n_t, int n_bas, int n_g, const double* eps, const double* xi,
                       const double* wt, const double* omega, int static_sub, double* I, double* dI,
                       const unsigned char* active, cudaStream_t s, const int* tmap = nullptr,
                       const int* spin = nullptr);

struct MinresState {
  double beta, c2, s2, c1, s1, phibar, beta1, pad;
  int iters, done, pad0, pad1;
};

// Gather b_j = B_nm[t_j][m_j] into V as (u, v) = (b, 0); T is the operator precision.
template <typename T>
void launch_gather_rhs(const double* B_nm, int n_bas, int n_aux, const int* rhs_t, const int* rhs_m, int nr, T* V,
                       cudaStream_t s);
// From S = [Re; Im](Pi b): initialise MINRES (v_1 = rhs/|rhs|) and write v_1 into V.
template <typename T>
void launch_minres_init(const T* S, int nr, int n_aux, double* vprev, double* v, double* d1, double* d2, double* x,
                        MinresState* st, T* V, cudaStream_t s);
// One MINRES step given P = E v (embedding matvec output).  Writes the next Lanczos vector into V.
template <typename T>
void launch_minres_step(const T* P, int nr, int n_aux, double tol, double* vprev, double* v, double* d1, double* d2,
                        double* x, MinresState* st, T* V, int* n_active, cudaStream_t s);
// After MINRES: W = b^T delta; y = b + delta written into V as (u, v) = (y_r, -y_i) for the derivative pass
// (and into V64 in FP64 when given).
template <typename T>
void launch_minres_finish(const double* B_nm, int n_bas, int n_aux, const int* rhs_t, const int* rhs_m, int nr,
                          const double* x, const MinresState* st, double* w_re, double* w_im, int* iters,
                          double* resnorm, T* V, cudaStream_t s, double* V64 = nullptr);

// Batched complex LU with partial pivoting (kernels_lu.cu): matrices b at Ar + b*stride, Ai + b*stride.
template <typename T>
void launch_zlu(T* Ar, T* Ai, long stride, int n, int batch, int* piv, int* info, cudaStream_t s);
// Spectral-decomposition route (kernels_sd.cu): the Casida matrix M = D^1/2 (D + 4 B^T B) D^1/2 [Np][Np] (Np = N
// rounded up to even, identity padding) and T = I; one cyclic Jacobi sweep of M (rotations accumulated in T, cs [Np]
// work space); off[0] / off[1] = squared off-diagonal / diagonal Frobenius norms; Omega [N], V = 2 B D^1/2 T
// [n_aux][N] and the pole weights w2[r][s] = (Bn_r . V_s)^2 / (2 Omega_s) for the R rows of Bn; Sigma_c and its
// derivative at evaluation points (target tmap[p] at omega[p]) from those weights.
cudaError_t sd_casida_matrix(const double* B, const double* Dk, int n_aux, int N, int Np, double* M, double* T,
                             cudaStream_t s);
cudaError_t sd_jacobi_sweep(double* M, double* T, int Np, double* cs, cudaStream_t s);
cudaError_t sd_offdiag(const double* M, int Np, double* off, cudaStream_t s);
cudaError_t sd_weights(const double* B, const double* Dk, const double* M, const double* T, const double* Bn,
                       int n_aux, int N, int Np, int R, double* Om, double* V, double* w2, cudaStream_t s);
cudaError_t sd_sigma(const double* w2, const double* Om, int N, int n_bas, const double* eps, const int* tmap,
                     const int* spin, const int* occ_t, int n_occ, const double* omega, int npts, double eta,
                     double* S, double* dS, cudaStream_t s);
// Blocked FP32 LU of `batch` complex matrices (planes A and A + plane, matrix stride `stride`) with the trailing
// updates on the tensor cores; same factors and pivot convention as launch_zlu.  work: work_elems BF16, at least
// zlu_tc_work_elems(n, 1) (one matrix's split panel operands); the updates run in sub-batches that fit it.
size_t zlu_tc_work_elems(int n, int batch);
cudaError_t launch_zlu_tc(float* A, long stride, long plane, int n, int batch, int* piv, int* info,
                          __nv_bfloat16* work, size_t work_elems, int* err, cudaStream_t s);
template <typename T>
void launch_zlu_solve(const T* Ar, const T* Ai, long stride, int n, int batch, const int* piv, T* yr, T* yi,
                      long ystride, cudaStream_t s);
// Fallback bookkeeping: for k < nf with slot index idx[k] (into the MINRES batch), set y planes = (b, 0) before
// the solve (stage 0), or after it write W = b^T y - b^T b, resnorm 0 and the (u, v) = (y_r, -y_i) rows of V.
template <typename T>
void launch_fallback_rhs(const double* B_nm, int n_bas, int n_aux, const int* rt, const int* rm, const int* idx,
                         int nf, T* y, cudaStream_t s);
template <typename T>
void launch_fallback_finish(const double* B_nm, int n_bas, int n_aux, const int* rt, const int* rm, const int* idx,
                            int nf, const T* y, double* w_re, double* w_im, double* resnorm, T* V, cudaStream_t s);

// Iterative refinement of fallback solves (k < nf; y32 planes [nf][2][n], y64 the same in FP64):
//   stage 0: y64 = y32;            V32 rows (2k, 2k+1) = (Re y, -Im y)
//   stage 1: y32 = [b; 0] - S      (residual, next right-hand side; S = S32 rows (2k, 2k+1), or, if S64 is given,
//                                   S64 rows (2q, 2q+1) with q = pos[k] (q = k without pos; q < 0: y32 = 0))
//   stage 2: y64 += y32;           V32 rows = (Re y, -Im y); rho[k] = |y32| / |y64| if rho is given
void launch_refine(int stage, const double* B_nm, int n_bas, int n_aux, const int* rt, const int* rm, const int* idx,
                   int nf, float* y32, double* y64, float* V32, const float* S32, cudaStream_t s,
                   const double* S64 = nullptr, const int* pos = nullptr, double* rho = nullptr);
// V64 rows (2q, 2q+1) = (Re y, -Im y) of the FP64 solution sel[q] (q without sel) of y64 [.][2][n], q < m.
void launch_refine_v64(int m, int n_aux, const int* sel, const double* y64, double* V64, cudaStream_t s);
// W = b^T y - b^T b from FP64 solutions; V (operator precision) rows of slot idx[k] = (Re y, -Im y); resnorm 0.
template <typename T>
void launch_fallback_finish64(const double* B_nm, int n_bas, int n_aux, const int* rt, const int* rm, const int* idx,
                              int nf, const double* y64, double* w_re, double* w_im, double* resnorm, T* V,
                              cudaStream_t s, double* V64 = nullptr);

// R term reduction per target over its right-hand sides [start[t], start[t+1]).
// W[r][g] += W[r][n_g] for g < n_cols (table [R][n_g + 1]): columns held as differences from the static one.
void launch_w_add_static(double* W, long R, int n_g, int n_cols, cudaStream_t s);
// W[r][c] = 0 outside the processing positions [p0, p1) (position 0 = column n_g, position p > 0 = column p - 1).
void launch_w_keep_positions(double* W, long R, int n_g, int p0, int p1, cudaStream_t s);
void launch_residue_reduce(const int* start, int n_t, const double* coef, const double* w_re, const double* dw_re,
                           double* R, double* dR, cudaStream_t s);

struct QPState {
  double omega, f_prev, omega_prev, Z;
  double a, fa, b, fb, x, fx;
  double sigma, dsigma;
  int br_kind, has_prev, iter, status;   // status: 0 running, 1 converged, 2 not converged
};
void launch_qp_init(QPState* st, const double* omega0, int n, cudaStream_t s);   // omega0: starting points
// sigma = R - I, dsigma = dR - dI for active states, then one step-tree step.
void launch_qp_step(QPState* st, const double* R, const double* dR, const double* I, const double* dI,
                    const double* e_n, const double* shift, double tol, int maxit, int n, int linearised,
                    cudaStream_t s);

}  // namespace gw
