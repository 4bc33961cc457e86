// tcgen05 batched GEMM with BF16 hi+lo split operands (tc_gemm.cu).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>

namespace gw {
// Row length (elements) of the split operand arrays for contraction length K (multiple of 8: 16-byte rows).
int tc_ld(int K);
// A_b[m][k] = B[m][k] * w(kinds[b], D_k, params[b]) split into BF16 hi/lo, [batch][M][tc_ld(K)].
// kinds: 0 Pi(i xi) weight -4D/(D^2+xi^2) (param xi); 1 Re c(x); 2 Im c(x) (param x, broadening eta);
// 3 unit weight.  kinds/params are device arrays of length batch.  B is FP32 [M][K].  The weights are evaluated
// once per (entry, k) in FP64 into wtab [batch][K] (device scratch), then applied in FP32 while splitting.
cudaError_t tc_scale_split(const float* B, const double* eps, int n_occ, int n_virt, int M, int K, const int* kinds,
                           const double* params, double eta, int batch, float* wtab, __nv_bfloat16* hi,
                           __nv_bfloat16* lo, cudaStream_t s);
// out_b = f(A_b Bm^T) for b < batch, out [batch][M][N] FP32; lower != 0 computes lower tiles and mirrors.
// mode_even / mode_odd for even / odd b: 0 v, 1 delta - v, 2 -v.  *err (device) receives a nonzero code if a
// bounded wait inside the kernel ran out.
cudaError_t tc_gemm(const __nv_bfloat16* Ahi, const __nv_bfloat16* Alo, int batch, const __nv_bfloat16* Bhi,
                    const __nv_bfloat16* Blo, int M, int N, int K, int lower, int mode_even, int mode_odd, float* out,
                    int* err, cudaStream_t s);
}  // namespace gw
