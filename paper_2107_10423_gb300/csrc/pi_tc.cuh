// tcgen05 batched GEMM with BF16 hi+lo split operands (tc_gemm.cu).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <vector>

namespace gw {
enum { TC_EPI_STORE = 0, TC_EPI_CPAIR = 1, TC_EPI_EMBED = 2, TC_EPI_AXPBY = 3, TC_EPI_WRED = 4, TC_EPI_SUB2 = 5 };

// Epilogue of the tensor-core GEMM (passed by value to the kernel).
struct TcEpi {
  int kind;
  // TC_EPI_STORE: out_b[m][n] (row length ldo) = v, delta_mn - v or -v (mode for even / odd batch entries)
  int mode_even, mode_odd;
  float* out;
  long out_bstride;
  int ldo;
  // TC_EPI_CPAIR: complex pair scaling of the residue operator into split BF16 rows (row length ldh)
  const double* Dk;    // [N] pair energies D_k
  const double* x;     // [M/2] residue frequencies
  float eta;
  __nv_bfloat16* ohi;
  __nv_bfloat16* olo;
  int ldh;
  __nv_bfloat16* olo2;   // third split part (TC_EPI_AXPBY, TC_EPI_CPAIR), or NULL
  // TC_EPI_EMBED: out[m][n] = (m even ? vin : -vin)[m][n] - v  (row lengths ldo, ldv)
  const float* vin;
  int ldv;
  // TC_EPI_AXPBY: y = alpha * xin_b[m][n] + gamma * v + beta * delta_mn, written to out (FP32, if not NULL) and
  // split into ohi/olo (if not NULL); batch strides out_bstride, x_bstride, oh_bstride (elements)
  const float* xin;
  long x_bstride;
  float alpha, gamma, beta;
  long oh_bstride;
  // TC_EPI_WRED: W[n * wld + gidx[b]] += sum_m bvec[n][m] * v[m][n]  (bvec FP32, row length ldb)
  double* W;
  int wld;
  const int* gidx;
  const float* bvec;
  int ldb;
  // TC_EPI_SUB2: out_b[r][c] -= v[r][c] for rows r < half and out_b[plane + (r - half) * ldo + c] -= v[r][c] for
  // the rows below (the two planes of a complex matrix updated by one stacked real product), batch stride
  // out_bstride, row length ldo
  long plane;
  int half;
  long limit;                 // TC_EPI_SUB2: elements writable from out (an index beyond it is recorded, code 66)
  // if not NULL: the whole launch does nothing when *run_if == 0 (device flag, read once at kernel start)
  const int* run_if;
};

// Row length (elements) of the split operand arrays for contraction length K (multiple of 8: 16-byte rows).
int tc_ld(int K);
// Row length (elements) of FP32 arrays read by TMA with contraction length K (multiple of 4: 16-byte rows).
int pf_ldw(int K);
// Weight table w [nb][pf_ldw(K)] (device, FP32, zero padded): w[b][k] = weight(kinds[b], D_k, params[b]) evaluated
// in FP64 from the pair energies Dk [K].  kinds (device [nb]): 0 Pi(i xi): -4D/(D^2 + xi^2) (param xi); 1 Re c(x),
// 2 Im c(x), c = 2[1/(x - D + i eta) + 1/(-x - D + i eta)] (param x); 3 unit; 4 Pi(i xi) - Pi(0):
// 4 xi^2/(D (D^2 + xi^2)).
cudaError_t tc_pair_weights(const double* Dk, int K, const int* kinds, const double* params, double eta, int nb,
                            float* w, cudaStream_t s);
// out_b = f(B diag(w_b) B^T) for b < nb on the tensor cores with the weight applied in the kernel (pi_fused.cu):
// B as its BF16 hi/lo split Bhi/Blo in the K-panel layout of tc_pi_panel_split ([P][n][256],
// P = tc_pi_panel_cols(K) / 256), w from tc_pair_weights, tiles (device) the table of tc_pi_fused_tile_order(n);
// out [nb][n][ldo] FP32 at batch stride out_bstride, full symmetric (lower tiles computed and mirrored);
// mode_even / mode_odd for even / odd b: 0 v, 1 delta - v, 2 -v.  max_ctas > 0 caps the persistent grid.
// ksplit > 0 asks for that many K ranges per (tile, entry), lowered by halving to the largest feasible split (every
// range at least 4 K blocks of 32, partials within part_bytes); ksplit = 0 autotunes it per shape (n, K, nb, max_ctas):
// every feasible split (partials [ksplit][nb][n][n] FP32 fit in part_bytes of `part`) is timed once and the
// fastest kept for the process.  *chosen (if not NULL) receives the split used.
cudaError_t tc_pi_fused(int n, int K, const float* w, int nb, const uint32_t* tiles,
                        const __nv_bfloat16* Bhi,
                        const __nv_bfloat16* Blo, int mode_even, int mode_odd, float* out, long out_bstride, int ldo,
                        int* err, cudaStream_t s, int max_ctas = 0, int ksplit = 1, float* part = nullptr,
                        size_t part_bytes = 0, int* chosen = nullptr);
// Work items of one unsplit tc_pi_fused launch (lower 128 x 256 tiles x entries); fewer than about two per SM
// leave the persistent grid partly idle, which is when a K split pays.
long tc_pi_fused_items(int n, int nb);
// Columns of the K-panel layout (K rounded up to the 256-column panel width) and the conversion to it: the BF16
// hi/lo split hp/lp[p][r][c] of B[r][256 p + c] (zero beyond K), from B FP32 [n][ldb] (n <= 65535).
long tc_pi_panel_cols(int K);
cudaError_t tc_pi_panel_split(const float* B, long ldb, int n, int K, __nv_bfloat16* hp, __nv_bfloat16* lp,
                              cudaStream_t s);
// The order in which tc_pi_fused visits its lower 128 x 256 tiles (bm | bn2 << 16, one entry per tile); the caller
// uploads it and passes it as `tiles`.
void tc_pi_fused_tile_order(int n, std::vector<uint32_t>& tiles);
// The split the autotuner chose for a shape with the given largest feasible split, or 0 if it has not seen it.
int tc_pi_fused_ksplit(int n, int K, int nb, int max_ctas, int max_split);
// out_b = f(A_b Bm^T) for b < batch, out [batch][M][N] FP32; lower != 0 computes lower tiles and mirrors.
// mode_even / mode_odd for even / odd b: 0 v, 1 delta - v, 2 -v.  *err (device) receives a nonzero code if a
// bounded wait inside the kernel ran out.
cudaError_t tc_gemm(const __nv_bfloat16* Ahi, const __nv_bfloat16* Alo, int batch, const __nv_bfloat16* Bhi,
                    const __nv_bfloat16* Blo, int M, int N, int K, int lower, int mode_even, int mode_odd, float* out,
                    int* err, cudaStream_t s);
// Split operand: parts p[0..nsplit) of [batch][rows][tc_ld(K)] BF16 (hi, lo[, lo2]).
struct TcOperand {
  const __nv_bfloat16* p[3];
};
// General form: B may also be batched (b_batched != 0: Bm_b has the same batch count as A); nsplit 2 uses three
// products (BF16x3), nsplit 3 the six products with part indices i + j <= 2 (about FP32-accurate).
cudaError_t tc_gemm_ex(const TcOperand& A, int batch, const TcOperand& B, int b_batched, int nsplit, int M, int N,
                       int K, int lower, const TcEpi& ep, int* err, cudaStream_t s);
// rows x cols FP32 (row length lds) split into BF16 hi/lo rows of tc_ld(cols) elements (zero padded).
cudaError_t tc_split_rows(const float* src, int rows, int cols, int lds, __nv_bfloat16* hi, __nv_bfloat16* lo,
                          cudaStream_t s, __nv_bfloat16* lo2 = nullptr);
// Spectrum estimates of SPD matrices A_b (n x n FP32, batch stride n*n), by `iters` power steps each (device
// outputs [batch]): hi_b, the Rayleigh quotient of A_b (an estimate of lambda_max from below), and lo_b = the
// Rayleigh quotient of s_b I - A_b with s_b = pad * hi_b (so s_b - lo_b estimates lambda_min from above).
// shift [batch], v and y [batch][n] are device work space.
cudaError_t tc_spectrum_bounds(const float* A, int n, int batch, int iters, float pad, float* hi, float* lo,
                               float* shift, float* v, float* y, cudaStream_t s);
// X_b = 2 a_b I - a_b^2 A_b (first Newton-Schulz iterate) with a_b = ab[b] (device), FP32 out [b][n][n] and split
// rows [b][n][tc_ld(n)].
cudaError_t tc_ns_init(const float* A, int n, int batch, const float* ab, float* X, __nv_bfloat16* hi,
                       __nv_bfloat16* lo, cudaStream_t s, __nv_bfloat16* lo2 = nullptr);
// Y_b = (X_b + X_b^T)/2 for n x n FP32 matrices (out of place), with its split parts (rows of tc_ld(n)).
cudaError_t tc_sym_split(const float* X, int n, int batch, float* Y, __nv_bfloat16* hi, __nv_bfloat16* lo,
                         __nv_bfloat16* lo2, cudaStream_t s);
// out[k][m] = B[m][k] split into BF16 hi/lo with rows of tc_ld(M) elements (B FP32 [M][ldb], ldb 0 = K).
cudaError_t tc_transpose_split(const float* B, int M, int K, __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t s,
                               __nv_bfloat16* lo2 = nullptr, long ldb = 0);
}  // namespace gw
