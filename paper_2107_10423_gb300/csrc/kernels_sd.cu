// Spectral-decomposition route (Sec. 2.2 and 3.2): the Casida problem in its Hermitian form
//   M T = T Omega^2,   M = D^1/2 (D + 4K) D^1/2,   K = B_ia^T B_ia   (N_ov x N_ov, symmetric positive definite),
// diagonalised by a parallel cyclic Jacobi method in FP64, then the pole weights
//   w2[t][m][s] = (b_tm . V_s)^2 / (2 Omega_s),   V = 2 B_ia D^1/2 T,
// so that Sigma^c_nn(omega) = sum_m sum_s w2 / (omega - e_m + Omega_s - i eta)  (m occupied)
//                           + sum_m sum_s w2 / (omega - e_m - Omega_s + i eta)  (m virtual).
// Jacobi rounds use the round-robin pairing of the indices: every round rotates N/2 disjoint pairs (p, q), each
// by the angle that zeroes M_pq, applied to rows (M <- J^T M), columns (M <- M J) and the eigenvectors (T <- T J).
#include "gw_internal.cuh"

#include <cmath>

namespace gw {
namespace {

constexpr int ST = 16;     // SIMT tile edge of the small GEMMs

// Round-robin pairing of 2h players (index 2h - 1 is fixed): pair k of round r.
__device__ __forceinline__ void rr_pair(int r, int k, int h, int& p, int& q) {
  const int m = 2 * h - 1;
  if (k == 0) {
    p = m;
    q = r % m;
  } else {
    p = (r + k) % m;
    q = (r - k + m) % m;
  }
  if (p > q) { const int t = p; p = q; q = t; }
}

// M = D^1/2 (D + 4 B^T B) D^1/2, padded to Np (extra indices: identity, never coupled).
__global__ void casida_matrix_kernel(const double* __restrict__ B, const double* __restrict__ Dk, int n_aux, int N,
                                     int Np, double* __restrict__ M) {
  __shared__ double As[ST][ST + 1], Bs[ST][ST + 1];
  const int i = blockIdx.y * ST + threadIdx.y, j = blockIdx.x * ST + threadIdx.x;
  double acc = 0.0;
  for (int p0 = 0; p0 < n_aux; p0 += ST) {
    const int pa = p0 + threadIdx.x, pb = p0 + threadIdx.y;
    As[threadIdx.y][threadIdx.x] = (i < N && pa < n_aux) ? B[(long)pa * N + i] : 0.0;
    Bs[threadIdx.y][threadIdx.x] = (j < N && pb < n_aux) ? B[(long)pb * N + j] : 0.0;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < ST; ++u) acc += As[threadIdx.y][u] * Bs[u][threadIdx.x];
    __syncthreads();
  }
  if (i < Np && j < Np) {
    double v;
    if (i < N && j < N) v = sqrt(Dk[i]) * (4.0 * acc + (i == j ? Dk[i] : 0.0)) * sqrt(Dk[j]);
    else v = (i == j) ? 1.0 : 0.0;
    M[(long)i * Np + j] = v;
  }
}

__global__ void identity_kernel(double* __restrict__ T, int Np) {
  const long n = (long)Np * Np;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    T[e] = (e / Np == e % Np) ? 1.0 : 0.0;
}

// Rotation of every pair of round r: (c, s) zeroing M_pq, stored per pair.
__global__ void jacobi_angles_kernel(const double* __restrict__ M, int Np, int r, double* __restrict__ cs) {
  const int h = Np / 2;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= h) return;
  int p, q;
  rr_pair(r, k, h, p, q);
  const double apq = M[(long)p * Np + q], app = M[(long)p * Np + p], aqq = M[(long)q * Np + q];
  double c = 1.0, s = 0.0;
  if (apq != 0.0 && fabs(apq) > 1e-300) {
    const double tau = (aqq - app) / (2.0 * apq);
    const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
    c = 1.0 / sqrt(1.0 + t * t);
    s = t * c;
  }
  cs[2 * k] = c;
  cs[2 * k + 1] = s;
}

// Rows p, q of M for every pair: (M_p, M_q) <- (c M_p - s M_q, s M_p + c M_q).
__global__ void jacobi_rows_kernel(double* __restrict__ M, int Np, int r, const double* __restrict__ cs) {
  const int h = Np / 2, k = blockIdx.y;
  int p, q;
  rr_pair(r, k, h, p, q);
  const double c = cs[2 * k], s = cs[2 * k + 1];
  if (s == 0.0) return;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < Np; j += gridDim.x * blockDim.x) {
    const double a = M[(long)p * Np + j], b = M[(long)q * Np + j];
    M[(long)p * Np + j] = c * a - s * b;
    M[(long)q * Np + j] = s * a + c * b;
  }
}

// Columns p, q of X (M, or the eigenvectors T): (X_.p, X_.q) <- (c X_.p - s X_.q, s X_.p + c X_.q).
__global__ void jacobi_cols_kernel(double* __restrict__ X, int Np, int r, const double* __restrict__ cs) {
  const int h = Np / 2, k = blockIdx.y;
  int p, q;
  rr_pair(r, k, h, p, q);
  const double c = cs[2 * k], s = cs[2 * k + 1];
  if (s == 0.0) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Np; i += gridDim.x * blockDim.x) {
    const double a = X[(long)i * Np + p], b = X[(long)i * Np + q];
    X[(long)i * Np + p] = c * a - s * b;
    X[(long)i * Np + q] = s * a + c * b;
  }
}

// off[0] += sum of squares of the off-diagonal elements, off[1] += of the diagonal ones.
__global__ void offdiag_kernel(const double* __restrict__ M, int Np, double* __restrict__ off) {
  __shared__ double red[2][32];
  double o = 0.0, d = 0.0;
  const long n = (long)Np * Np;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const double v = M[e];
    if (e / Np == e % Np) d += v * v; else o += v * v;
  }
  for (int w = 16; w > 0; w >>= 1) {
    o += __shfl_xor_sync(0xffffffffu, o, w);
    d += __shfl_xor_sync(0xffffffffu, d, w);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = o;
    red[1][threadIdx.x >> 5] = d;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double so = 0.0, sd = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { so += red[0][w]; sd += red[1][w]; }
    atomicAdd(off, so);
    atomicAdd(off + 1, sd);
  }
}

// V[P][s] = 2 sum_k B[P][k] sqrt(D_k) T[k][s]  (the eigenvectors in the auxiliary basis), s < N.
__global__ void casida_v_kernel(const double* __restrict__ B, const double* __restrict__ Dk,
                                const double* __restrict__ T, int n_aux, int N, int Np, double* __restrict__ V) {
  __shared__ double As[ST][ST + 1], Bs[ST][ST + 1];
  const int P = blockIdx.y * ST + threadIdx.y, sc = blockIdx.x * ST + threadIdx.x;
  double acc = 0.0;
  for (int k0 = 0; k0 < N; k0 += ST) {
    const int ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
    As[threadIdx.y][threadIdx.x] = (P < n_aux && ka < N) ? B[(long)P * N + ka] * sqrt(Dk[ka]) : 0.0;
    Bs[threadIdx.y][threadIdx.x] = (sc < N && kb < N) ? T[(long)kb * Np + sc] : 0.0;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < ST; ++u) acc += As[threadIdx.y][u] * Bs[u][threadIdx.x];
    __syncthreads();
  }
  if (P < n_aux && sc < N) V[(long)P * N + sc] = 2.0 * acc;
}

// w2[r][s] = (b_r . V_s)^2 / (2 Omega_s) for the rows r of Bn [R][n_aux].
__global__ void casida_w2_kernel(const double* __restrict__ Bn, const double* __restrict__ V,
                                 const double* __restrict__ Om, int n_aux, int R, int N, double* __restrict__ w2) {
  __shared__ double As[ST][ST + 1], Bs[ST][ST + 1];
  const int r = blockIdx.y * ST + threadIdx.y, sc = blockIdx.x * ST + threadIdx.x;
  double acc = 0.0;
  for (int p0 = 0; p0 < n_aux; p0 += ST) {
    const int pa = p0 + threadIdx.x, pb = p0 + threadIdx.y;
    As[threadIdx.y][threadIdx.x] = (r < R && pa < n_aux) ? Bn[(long)r * n_aux + pa] : 0.0;
    Bs[threadIdx.y][threadIdx.x] = (sc < N && pb < n_aux) ? V[(long)pb * N + sc] : 0.0;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < ST; ++u) acc += As[threadIdx.y][u] * Bs[u][threadIdx.x];
    __syncthreads();
  }
  if (r < R && sc < N) w2[(long)r * N + sc] = acc * acc / (2.0 * Om[sc]);
}

__global__ void casida_omega_kernel(const double* __restrict__ M, int Np, int N, double* __restrict__ Om) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < N) Om[s] = sqrt(fmax(M[(long)s * Np + s], 0.0));
}

// Sigma at evaluation points p: target tmap[p] (its G energies eps + spin offset, occupations occ) at omega[p].
__global__ void sigma_sd_kernel(const double* __restrict__ w2, const double* __restrict__ Om, int N, int n_bas,
                                const double* __restrict__ eps, const int* __restrict__ tmap,
                                const int* __restrict__ spin, const int* __restrict__ occ_t, int n_occ,
                                const double* __restrict__ omega, double eta, double* __restrict__ S,
                                double* __restrict__ dS) {
  __shared__ double red[2][32];
  const int p = blockIdx.x;
  const int t = tmap ? tmap[p] : p;
  const double* e = eps + (spin ? (long)spin[t] * n_bas : 0);
  const int occ = occ_t ? occ_t[t] : n_occ;
  const double w = omega[p];
  double s = 0.0, d = 0.0;
  const long n = (long)n_bas * N;
  for (long idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int m = (int)(idx / N), k = (int)(idx - (long)m * N);
    const double wt = w2[((long)t * n_bas + m) * N + k];
    // occupied m: 1/(w - e_m + Omega - i eta); virtual m: 1/(w - e_m - Omega + i eta)
    const double a = m < occ ? w - e[m] + Om[k] : w - e[m] - Om[k];
    const double den = a * a + eta * eta;
    s += wt * a / den;
    d -= wt * (a * a - eta * eta) / (den * den);
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    d += __shfl_xor_sync(0xffffffffu, d, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s;
    red[1][threadIdx.x >> 5] = d;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ts = 0.0, td = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { ts += red[0][i]; td += red[1][i]; }
    S[p] = ts;
    dS[p] = td;
  }
}

}  // namespace

cudaError_t sd_casida_matrix(const double* B, const double* Dk, int n_aux, int N, int Np, double* M, double* T,
                             cudaStream_t s) {
  dim3 g((Np + ST - 1) / ST, (Np + ST - 1) / ST);
  casida_matrix_kernel<<<g, dim3(ST, ST), 0, s>>>(B, Dk, n_aux, N, Np, M);
  identity_kernel<<<1024, 256, 0, s>>>(T, Np);
  return cudaGetLastError();
}

cudaError_t sd_jacobi_sweep(double* M, double* T, int Np, double* cs, cudaStream_t s) {
  const int h = Np / 2;
  const dim3 gr((Np + 255) / 256 < 8 ? (Np + 255) / 256 : 8, h);
  for (int r = 0; r < Np - 1; ++r) {
    jacobi_angles_kernel<<<(h + 127) / 128, 128, 0, s>>>(M, Np, r, cs);
    jacobi_rows_kernel<<<gr, 256, 0, s>>>(M, Np, r, cs);
    jacobi_cols_kernel<<<gr, 256, 0, s>>>(M, Np, r, cs);
    jacobi_cols_kernel<<<gr, 256, 0, s>>>(T, Np, r, cs);
  }
  return cudaGetLastError();
}

cudaError_t sd_offdiag(const double* M, int Np, double* off, cudaStream_t s) {
  cudaMemsetAsync(off, 0, 2 * sizeof(double), s);
  offdiag_kernel<<<256, 256, 0, s>>>(M, Np, off);
  return cudaGetLastError();
}

cudaError_t sd_weights(const double* B, const double* Dk, const double* M, const double* T, const double* Bn,
                       int n_aux, int N, int Np, int R, double* Om, double* V, double* w2, cudaStream_t s) {
  casida_omega_kernel<<<(N + 255) / 256, 256, 0, s>>>(M, Np, N, Om);
  casida_v_kernel<<<dim3((N + ST - 1) / ST, (n_aux + ST - 1) / ST), dim3(ST, ST), 0, s>>>(B, Dk, T, n_aux, N, Np, V);
  casida_w2_kernel<<<dim3((N + ST - 1) / ST, (R + ST - 1) / ST), dim3(ST, ST), 0, s>>>(Bn, V, Om, n_aux, R, N, w2);
  return cudaGetLastError();
}

cudaError_t sd_sigma(const double* w2, const double* Om, int N, int n_bas, const double* eps, const int* tmap,
                     const int* spin, const int* occ_t, int n_occ, const double* omega, int npts, double eta,
                     double* S, double* dS, cudaStream_t s) {
  if (npts > 0)
    sigma_sd_kernel<<<npts, 256, 0, s>>>(w2, Om, N, n_bas, eps, tmap, spin, occ_t, n_occ, omega, eta, S, dS);
  return cudaGetLastError();
}

}  // namespace gw
