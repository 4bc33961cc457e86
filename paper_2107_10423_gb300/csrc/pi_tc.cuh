// Tensor-core (tcgen05) build of Pi(i xi) with BF16 hi+lo split operands and FP32 accumulation.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include "gw.h"

namespace gw {
// Pi_g = -4 sum_k B[P][k] B[Q][k] D_k/(D_k^2 + xi_g^2) for n_xi frequencies, out [n_xi][n][n] FP32
// (mode 0: Pi, mode 1: 1 - Pi).  B is FP32 [n][n_ov].  Workspace grows through (*ws, *ws_bytes).
// *used is false when the shapes are not supported by the tensor-core kernel (caller falls back).
gw_status pi_tc_build(const float* B, const double* eps, int n_occ, int n_virt, int n, const double* xi, int n_xi,
                      float* out, int mode, void** ws, size_t* ws_bytes, cudaStream_t s, bool* used);
}  // namespace gw
