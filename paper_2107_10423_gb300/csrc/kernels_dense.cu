// Dense kernels of the CD-G0W0 path (SIMT, templated on the arithmetic type):
//  * Pi(i xi) symmetric rank-N_ov update (Sec. 3.3, equation after "wauxbas"), lower tiles + mirror;
//  * batched in-place Cholesky of eps(i xi) = 1 - Pi (SPD, Sec. 3.3 text after "inn");
//  * triangular solves that turn the factors into the table W^c_nm(i xi) (Algorithm 1, imaginary-grid loop);
//  * the two skinny GEMMs of the matrix-free residue operator 1 - Pi(x) (Sec. 3.3, MINRES paragraph).
#include "gw_internal.cuh"
#include "gw.h"

#include <cstdio>
#include <mutex>

namespace gw {

namespace {

constexpr int TM = 64;     // tile rows
constexpr int TN = 64;     // tile cols
constexpr int TK = 16;     // k step
constexpr int NT = 256;    // threads per CTA (16 x 16, 4 x 4 outputs each)

// ------------------------------------------------------------------ Pi(i xi) SYRK
// grid.x: lower-triangular tile index (bi >= bj), grid.y: frequency index.
template <typename T>
__global__ void __launch_bounds__(NT) pi_syrk_kernel(const T* __restrict__ B, const double* __restrict__ Dk,
                                                     long n_ov, int n_aux,
                                                     const double* __restrict__ xi, T* __restrict__ out, int mode) {
  __shared__ T As[TK][TM + 4];
  __shared__ T Bs[TK][TN + 4];
  // decode lower tile (bi, bj) from linear index t = bi*(bi+1)/2 + bj
  int t = blockIdx.x;
  int bi = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
  while (bi * (bi + 1) / 2 > t) --bi;
  int bj = t - bi * (bi + 1) / 2;
  const int g = blockIdx.y;
  const double x2 = xi[g] * xi[g];
  const int p0 = bi * TM, q0 = bj * TN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  const int lr = tid >> 2, lk = (tid & 3) * 4;
  for (long k0 = 0; k0 < n_ov; k0 += TK) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      long k = k0 + lk + u;
      T wa = T(0), va = T(0), vb = T(0);
      if (k < n_ov) {
        const double D = Dk[k];
        wa = (T)(-4.0 * D / (D * D + x2));
        if (p0 + lr < n_aux) va = B[(long)(p0 + lr) * n_ov + k];
        if (q0 + lr < n_aux) vb = B[(long)(q0 + lr) * n_ov + k];
      }
      As[lk + u][lr] = va * wa;
      Bs[lk + u][lr] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  T* o = out + (long)g * n_aux * n_aux;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int p = p0 + ty + 16 * i;
    if (p >= n_aux) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int q = q0 + tx + 16 * j;
      if (q >= n_aux || q > p) continue;
      T v = acc[i][j];
      if (mode == 1) v = (p == q ? T(1) : T(0)) - v;
      o[(long)p * n_aux + q] = v;
      o[(long)q * n_aux + p] = v;
    }
  }
}

// Complex real-axis Pi(x) as A = 1 - Pi, two real halves (dense fallback only).
__global__ void __launch_bounds__(NT) pi_complex_kernel(const double* __restrict__ B, const double* __restrict__ Dk,
                                                        long n_ov, int n_aux, double x, double eta,
                                                        double* __restrict__ Ar, double* __restrict__ Ai) {
  __shared__ double Asr[TK][TM + 4];
  __shared__ double Asi[TK][TM + 4];
  __shared__ double Bs[TK][TN + 4];
  const int p0 = blockIdx.y * TM, q0 = blockIdx.x * TN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double accr[4][4], acci[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) accr[i][j] = acci[i][j] = 0.0;
  const int lr = tid >> 2, lk = (tid & 3) * 4;
  const double e2 = eta * eta;
  for (long k0 = 0; k0 < n_ov; k0 += TK) {
    for (int u = 0; u < 4; ++u) {
      long k = k0 + lk + u;
      double cr = 0, ci = 0, va = 0, vb = 0;
      if (k < n_ov) {
        const double D = Dk[k];
        double a1 = x - D, a2 = -x - D;
        double d1 = a1 * a1 + e2, d2 = a2 * a2 + e2;
        cr = 2.0 * (a1 / d1 + a2 / d2);
        ci = 2.0 * (-eta / d1 - eta / d2);
        if (p0 + lr < n_aux) va = B[(long)(p0 + lr) * n_ov + k];
        if (q0 + lr < n_aux) vb = B[(long)(q0 + lr) * n_ov + k];
      }
      Asr[lk + u][lr] = va * cr;
      Asi[lk + u][lr] = va * ci;
      Bs[lk + u][lr] = vb;
    }
    __syncthreads();
    for (int kk = 0; kk < TK; ++kk) {
      double ar[4], ai[4], b[4];
      for (int i = 0; i < 4; ++i) { ar[i] = Asr[kk][ty + 16 * i]; ai[i] = Asi[kk][ty + 16 * i]; }
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
          accr[i][j] = fma(ar[i], b[j], accr[i][j]);
          acci[i][j] = fma(ai[i], b[j], acci[i][j]);
        }
    }
    __syncthreads();
  }
  for (int i = 0; i < 4; ++i) {
    int p = p0 + ty + 16 * i;
    if (p >= n_aux) continue;
    for (int j = 0; j < 4; ++j) {
      int q = q0 + tx + 16 * j;
      if (q >= n_aux) continue;
      Ar[(long)p * n_aux + q] = (p == q ? 1.0 : 0.0) - accr[i][j];
      Ai[(long)p * n_aux + q] = -acci[i][j];
    }
  }
}

// ------------------------------------------------------------------ batched Cholesky, one CTA per matrix
constexpr int CH_NB = 32;
constexpr int CH_THREADS = 512;

template <typename T>
__global__ void __launch_bounds__(CH_THREADS) cholesky_kernel(T* base, int n, long stride, int* info) {
  __shared__ T Ld[CH_NB][CH_NB + 1];
  __shared__ T Pi_[64][CH_NB + 1];
  __shared__ T Pj_[64][CH_NB + 1];
  __shared__ int bad;
  T* A = base + (long)blockIdx.x * stride;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int j0 = 0; j0 < n; j0 += CH_NB) {
    const int nb = min(CH_NB, n - j0);
    // (1) diagonal block
    for (int idx = tid; idx < nb * nb; idx += CH_THREADS) {
      int r = idx / nb, c = idx % nb;
      Ld[r][c] = A[(long)(j0 + r) * n + j0 + c];
    }
    __syncthreads();
    for (int c = 0; c < nb; ++c) {
      if (tid == 0) {
        T d = Ld[c][c];
        if (!(d > T(0))) { bad = j0 + c + 1; d = T(1); }
        Ld[c][c] = sqrt(d);
      }
      __syncthreads();
      for (int r = c + 1 + tid; r < nb; r += CH_THREADS) Ld[r][c] /= Ld[c][c];
      __syncthreads();
      for (int idx = tid; idx < (nb - c - 1) * (nb - c - 1); idx += CH_THREADS) {
        int r = c + 1 + idx / (nb - c - 1), s = c + 1 + idx % (nb - c - 1);
        if (s <= r) Ld[r][s] -= Ld[r][c] * Ld[s][c];
      }
      __syncthreads();
    }
    for (int idx = tid; idx < nb * nb; idx += CH_THREADS) {
      int r = idx / nb, c = idx % nb;
      if (c <= r) A[(long)(j0 + r) * n + j0 + c] = Ld[r][c];
    }
    // (2) panel rows below: x L^T = a
    for (int i = j0 + nb + tid; i < n; i += CH_THREADS) {
      T xr[CH_NB];
      for (int c = 0; c < nb; ++c) {
        T v = A[(long)i * n + j0 + c];
        for (int s = 0; s < c; ++s) v -= xr[s] * Ld[c][s];
        xr[c] = v / Ld[c][c];
      }
      for (int c = 0; c < nb; ++c) A[(long)i * n + j0 + c] = xr[c];
    }
    __threadfence_block();
    __syncthreads();
    // (3) trailing lower update A[i][j] -= sum_c P[i][c] P[j][c], i >= j >= j0+nb
    const int t0 = j0 + nb;
    const int nt = (n - t0 + 63) / 64;
    for (int ti = 0; ti < nt; ++ti) {
      for (int tj = 0; tj <= ti; ++tj) {
        const int r0 = t0 + ti * 64, c0 = t0 + tj * 64;
        for (int idx = tid; idx < 64 * CH_NB; idx += CH_THREADS) {
          int r = idx / CH_NB, c = idx % CH_NB;
          Pi_[r][c] = (r0 + r < n && c < nb) ? A[(long)(r0 + r) * n + j0 + c] : T(0);
          Pj_[r][c] = (c0 + r < n && c < nb) ? A[(long)(c0 + r) * n + j0 + c] : T(0);
        }
        __syncthreads();
        const int r = tid >> 3;             // 0..63
        const int cb = tid & 7;             // cols cb + 8*jj
        T acc[8];
        for (int jj = 0; jj < 8; ++jj) acc[jj] = T(0);
        for (int c = 0; c < nb; ++c) {
          T a = Pi_[r][c];
          for (int jj = 0; jj < 8; ++jj) acc[jj] = fma(a, Pj_[cb + 8 * jj][c], acc[jj]);
        }
        const int gi = r0 + r;
        if (gi < n) {
          for (int jj = 0; jj < 8; ++jj) {
            int gj = c0 + cb + 8 * jj;
            if (gj < n && gj <= gi) A[(long)gi * n + gj] -= acc[jj];
          }
        }
        __syncthreads();
      }
    }
    __threadfence_block();
    __syncthreads();
  }
  if (tid == 0) info[blockIdx.x] = bad;
}

// ------------------------------------------------------------------ TRSM -> W table
// Work item = (matrix g, tile of 64 right-hand sides).  Y for the tile lives in this CTA's scratch slice.
template <typename T>
__global__ void __launch_bounds__(NT) trsm_w_kernel(const T* __restrict__ Lbase, long Lstride, int n, int n_g,
                                                    const int* __restrict__ g_out, const T* __restrict__ Bn, int R,
                                                    double* __restrict__ W, int w_ld, T* __restrict__ scratch) {
  extern __shared__ unsigned char smem_raw[];
  T* As = reinterpret_cast<T*>(smem_raw);             // [TK][TM+4]
  T* Bs = As + TK * (TM + 4);                          // [TK][TN+4]
  T* Ts = Bs + TK * (TN + 4);                          // [64][65]
  T* Ls = Ts + 64 * 65;                                // [64][65]
  double* red = reinterpret_cast<double*>(Ls + 64 * 65);  // [2][16][64]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int n_ct = (R + 63) / 64;
  const int nJ = (n + 63) / 64;
  // per-CTA slice of [nJ*64][64]: the last row block is written in full (zeros past n)
  T* Y = scratch + (long)blockIdx.x * nJ * 64 * 64;
  const long n_items = (long)n_g * n_ct;
  for (long item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int g = (int)(item / n_ct);
    const int r0 = (int)(item % n_ct) * 64;
    const T* L = Lbase + (long)g * Lstride;
    double ws[4] = {0, 0, 0, 0}, bs[4] = {0, 0, 0, 0};
    for (int J = 0; J < nJ; ++J) {
      const int P0 = J * 64;
      const int nr = min(64, n - P0);
      T acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          int P = P0 + ty + 16 * i, c = r0 + tx + 16 * j;
          T v = (P < n && c < R) ? Bn[(long)c * n + P] : T(0);
          acc[i][j] = v;
          bs[j] += (double)v * (double)v;
        }
      for (int K = 0; K < J; ++K) {
        for (int kk0 = 0; kk0 < 64; kk0 += TK) {
          {
            // As[kk][r] = L[P0+r][K*64+kk0+kk]; Bs[kk][c] = Y[(K*64+kk0+kk)*64 + c]
            int r = tid >> 2, k4 = (tid & 3) * 4;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              int kk = k4 + u;
              int col = K * 64 + kk0 + kk;
              As[kk * (TM + 4) + r] = (P0 + r < n) ? L[(long)(P0 + r) * n + col] : T(0);
            }
            int kr = tid >> 4, c4 = (tid & 15) * 4;
#pragma unroll
            for (int u = 0; u < 4; ++u) Bs[kr * (TN + 4) + c4 + u] = Y[(long)(K * 64 + kk0 + kr) * 64 + c4 + u];
          }
          __syncthreads();
#pragma unroll
          for (int kk = 0; kk < TK; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk * (TM + 4) + ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk * (TN + 4) + tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int j = 0; j < 4; ++j) acc[i][j] = fma(-a[i], b[j], acc[i][j]);
          }
          __syncthreads();
        }
      }
      // stage the right-hand side block and the diagonal factor block
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) Ts[(ty + 16 * i) * 65 + tx + 16 * j] = acc[i][j];
      for (int idx = tid; idx < 64 * 64; idx += NT) {
        int r = idx >> 6, c = idx & 63;
        Ls[r * 65 + c] = (r < nr && c <= r) ? L[(long)(P0 + r) * n + P0 + c] : (r == c ? T(1) : T(0));
      }
      __syncthreads();
      if (tid < 64) {
        const int c = tid;
        for (int p = 0; p < nr; ++p) {
          T v = Ts[p * 65 + c];
          for (int q = 0; q < p; ++q) v = fma(-Ls[p * 65 + q], Ts[q * 65 + c], v);
          Ts[p * 65 + c] = v / Ls[p * 65 + p];
        }
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          int p = ty + 16 * i, c = tx + 16 * j;
          T v = (p < nr) ? Ts[p * 65 + c] : T(0);
          Y[(long)(P0 + p) * 64 + c] = v;   // rows beyond n are never read
          ws[j] += (double)v * (double)v;
        }
      __threadfence_block();
      __syncthreads();
    }
    // reduce per column over ty
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      red[(0 * 16 + ty) * 64 + tx + 16 * j] = ws[j];
      red[(1 * 16 + ty) * 64 + tx + 16 * j] = bs[j];
    }
    __syncthreads();
    if (tid < 64) {
      double w = 0, b = 0;
      for (int y = 0; y < 16; ++y) { w += red[(0 * 16 + y) * 64 + tid]; b += red[(1 * 16 + y) * 64 + tid]; }
      int r = r0 + tid;
      if (r < R) W[(long)r * w_ld + g_out[g]] = w - b;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ residue operator GEMMs
// gemm1: rows r in [0, 2nr), cols k in [0, n_ov): acc = sum_P V[r][P] B[P][k]  (B is N-contiguous here)
template <typename T>
__global__ void __launch_bounds__(NT) op_gemm1_kernel(const T* __restrict__ V, const T* __restrict__ B,
                                                      const double* __restrict__ Dk, long n_ov,
                                                      int n_aux, const double* __restrict__ xs, double eta, int nr,
                                                      T* __restrict__ U, int mode, double* __restrict__ dw,
                                                      double cut, long ldb, const int* __restrict__ run_if) {
  if (run_if && *run_if == 0) return;
  __shared__ T As[TK][TM + 4];
  __shared__ T Bs[TK][TN + 4];
  const int M = 2 * nr;
  const int m0 = blockIdx.y * TM;
  const long k0c = (long)blockIdx.x * TN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int p0 = 0; p0 < n_aux; p0 += TK) {
    {
      int r = tid >> 2, k4 = (tid & 3) * 4;       // A: V rows, K (=P) contiguous
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        int P = p0 + k4 + u;
        As[k4 + u][r] = (m0 + r < M && P < n_aux) ? V[(long)(m0 + r) * n_aux + P] : T(0);
      }
      int kr = tid >> 4, c4 = (tid & 15) * 4;     // B: rows P, cols k contiguous
      int P = p0 + kr;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        long k = k0c + c4 + u;
        Bs[kr][c4 + u] = (P < n_aux && k < n_ov) ? B[(long)P * ldb + k] : T(0);
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][2 * ty + (i & 1) + 32 * (i >> 1)];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  const double e2 = eta * eta;
  if (mode == 2) {
    // derivative pass fused with its reduction: dw[j] += sum_k Re(c'_k(x_j) t_k^2) in FP64 (no U round trip),
    // c' = 2[-(a1 - i eta)^2/d1^2 + (a2 - i eta)^2/d2^2]
#pragma unroll
    for (int ip = 0; ip < 2; ++ip) {
      const int r = m0 + 2 * ty + 32 * ip;
      double sum = 0.0;
      if (r < M) {
        const double x = xs[r >> 1];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const long k = k0c + tx + 16 * j;
          if (k >= n_ov) continue;
          const double tr = (double)acc[2 * ip][j], ti = -(double)acc[2 * ip + 1][j];
          const double D = Dk[k];
          const double a1 = x - D, a2 = -x - D;
          if (fabs(a1) < cut || fabs(a2) < cut) continue;   // near resonance: FP64 pass (deriv_resonant)
          const double d1 = a1 * a1 + e2, d2 = a2 * a2 + e2;
          const double q1r = (a1 * a1 - e2) / (d1 * d1), q1i = -2.0 * a1 * eta / (d1 * d1);
          const double q2r = (a2 * a2 - e2) / (d2 * d2), q2i = -2.0 * a2 * eta / (d2 * d2);
          const double cr = 2.0 * (-q1r + q2r), ci = 2.0 * (-q1i + q2i);
          sum += cr * (tr * tr - ti * ti) - ci * (2.0 * tr * ti);
        }
      }
      // the 16 lanes tx of one ty hold the same row: reduce within each half warp
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if (tx == 0 && r < M) atomicAdd(dw + (r >> 1), sum);
    }
    return;
  }
#pragma unroll
  for (int ip = 0; ip < 2; ++ip) {
    int r = m0 + 2 * ty + 32 * ip;           // even row of the pair
    if (r >= M) continue;
    int jr = r >> 1;
    double x = xs[jr];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      long k = k0c + tx + 16 * j;
      if (k >= n_ov) continue;
      double tr = (double)acc[2 * ip][j], ti = -(double)acc[2 * ip + 1][j];
      const double D = Dk[k];
      double a1 = x - D, a2 = -x - D;
      double d1 = a1 * a1 + e2, d2 = a2 * a2 + e2;
      const double cr = 2.0 * (a1 / d1 + a2 / d2);
      const double ci = -2.0 * eta * (1.0 / d1 + 1.0 / d2);
      const double outr = cr * tr - ci * ti;
      const double outi = cr * ti + ci * tr;
      U[(long)r * n_ov + k] = (T)outr;
      U[(long)(r + 1) * n_ov + k] = (T)outi;
    }
  }
}

// First index q of the ascending array with a[q] >= v.
__device__ __forceinline__ long lower_index(const double* a, long n, double v) {
  long lo = 0, hi = n;
  while (lo < hi) {
    const long mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// FP64 part of the fused derivative pass: the pairs k near resonance with x_j (|x_j - D_k| < cut or
// |-x_j - D_k| < cut, the same test in the same arithmetic as the FP32 pass, which skips them).  One CTA per right-hand
// side; candidate windows come from the ascending pair energies Dsort (pair index kidx), widened by cut on each side
// and then filtered by the exact test, so every pair is counted once.  One warp per pair:
// t_k = sum_P B[P][k] (u_P - i v_P) from the FP64 rows (u, v) = V64 rows (2j, 2j+1); dw[j] += Re(c'_k(x_j) t_k^2).
__global__ void __launch_bounds__(256) deriv_resonant_kernel(const double* __restrict__ V64,
                                                             const double* __restrict__ B, long n_ov, int n_aux,
                                                             const double* __restrict__ Dsort,
                                                             const int* __restrict__ kidx,
                                                             const double* __restrict__ xs, double eta, double cut,
                                                             double* __restrict__ dw) {
  __shared__ long rng[4];
  __shared__ double red[8];
  const int j = blockIdx.x;
  const double x = xs[j], e2 = eta * eta;
  if (threadIdx.x == 0) {
    long l1 = lower_index(Dsort, n_ov, x - 2.0 * cut), h1 = lower_index(Dsort, n_ov, x + 2.0 * cut);
    long l2 = lower_index(Dsort, n_ov, -x - 2.0 * cut), h2 = lower_index(Dsort, n_ov, -x + 2.0 * cut);
    if (l2 < h1 && l1 < h2) {   // overlapping windows: one merged window
      l1 = l1 < l2 ? l1 : l2;
      h1 = h1 > h2 ? h1 : h2;
      l2 = h2 = 0;
    }
    rng[0] = l1; rng[1] = h1; rng[2] = l2; rng[3] = h2;
  }
  __syncthreads();
  const double* u = V64 + (long)(2 * j) * n_aux;
  const double* v = u + n_aux;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double sum = 0.0;
  for (int w = 0; w < 2; ++w) {
    for (long q = rng[2 * w] + warp; q < rng[2 * w + 1]; q += nw) {
      const double D = Dsort[q];
      const double a1 = x - D, a2 = -x - D;
      if (!(fabs(a1) < cut || fabs(a2) < cut)) continue;   // warp-uniform
      const long k = kidx[q];
      double tr = 0.0, tv = 0.0;
      for (int P = lane; P < n_aux; P += 32) {
        const double b = B[(long)P * n_ov + k];
        tr += b * u[P];
        tv += b * v[P];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        tr += __shfl_xor_sync(0xffffffffu, tr, o);
        tv += __shfl_xor_sync(0xffffffffu, tv, o);
      }
      const double ti = -tv;
      const double d1 = a1 * a1 + e2, d2 = a2 * a2 + e2;
      const double q1r = (a1 * a1 - e2) / (d1 * d1), q1i = -2.0 * a1 * eta / (d1 * d1);
      const double q2r = (a2 * a2 - e2) / (d2 * d2), q2i = -2.0 * a2 * eta / (d2 * d2);
      const double cr = 2.0 * (-q1r + q2r), ci = 2.0 * (-q1i + q2i);
      if (lane == 0) sum += cr * (tr * tr - ti * ti) - ci * (2.0 * tr * ti);
    }
  }
  if (lane == 0) red[warp] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w];
    atomicAdd(dw + j, t);
  }
}

// gemm2: rows r in [0, 2nr), cols P in [0, n_aux): acc = sum_k U[r][k] B[P][k]  (both K-contiguous)
template <typename T>
__global__ void __launch_bounds__(NT) op_gemm2_kernel(const T* __restrict__ U, const T* __restrict__ B, int n_aux,
                                                      long n_ov, int nr, const T* __restrict__ V,
                                                      T* __restrict__ out, int mode, const int* __restrict__ run_if) {
  if (run_if && *run_if == 0) return;
  __shared__ T As[TK][TM + 4];
  __shared__ T Bs[TK][TN + 4];
  const int M = 2 * nr;
  const int m0 = blockIdx.y * TM;
  const int q0 = blockIdx.x * TN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  const int lr = tid >> 2, lk = (tid & 3) * 4;
  for (long k0 = 0; k0 < n_ov; k0 += TK) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      long k = k0 + lk + u;
      As[lk + u][lr] = (m0 + lr < M && k < n_ov) ? U[(long)(m0 + lr) * n_ov + k] : T(0);
      Bs[lk + u][lr] = (q0 + lr < n_aux && k < n_ov) ? B[(long)(q0 + lr) * n_ov + k] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][2 * ty + (i & 1) + 32 * (i >> 1)];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int r = m0 + 2 * ty + (i & 1) + 32 * (i >> 1);
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int P = q0 + tx + 16 * j;
      if (P >= n_aux) continue;
      T v = acc[i][j];
      if (mode == 1) {
        T vin = V[(long)r * n_aux + P];
        v = ((r & 1) ? -vin : vin) - v;
      }
      out[(long)r * n_aux + P] = v;
    }
  }
}

// ------------------------------------------------------------------ double-float GEMMs (refinement residual)
// A double x is carried as the FP32 pair (h, l), h = fl(x), l = fl(x - h): 48 significant bits.  A multiply-add
// s += a b takes the product exactly to FP32 pair precision (h*h by an FMA error term, plus the two cross terms)
// and adds it with Knuth's TwoSum; the low word collects every rounding error and is folded in once at the end.
// The _rn intrinsics keep the compiler from contracting the error-free steps into FMAs.
__device__ __forceinline__ void df_split(double x, float& h, float& l) {
  h = __double2float_rn(x);
  l = __double2float_rn(x - (double)h);
}

__device__ __forceinline__ void df_mac(float ah, float al, float bh, float bl, float& sh, float& sl) {
  const float ph = __fmul_rn(ah, bh);
  float pe = __fmaf_rn(ah, bh, -ph);
  pe = __fmaf_rn(ah, bl, pe);
  pe = __fmaf_rn(al, bh, pe);
  const float t = __fadd_rn(sh, ph);
  const float v = __fsub_rn(t, sh);
  const float e = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, v)), __fsub_rn(ph, v));
  sl = __fadd_rn(sl, __fadd_rn(e, pe));
  sh = t;
}

// df gemm1: U[r][k] for rows r of V [2nr][n_aux] (FP64) against B = Bh + Bl [n_aux][n_ov], then the complex
// weights c_k(x_j) of the pair (2j, 2j+1) as in op_gemm1 mode 0; U in FP64.
__global__ void __launch_bounds__(NT) op_gemm1_df_kernel(const double* __restrict__ V, const float* __restrict__ Bh,
                                                         const float* __restrict__ Bl, long ldh,
                                                         const double* __restrict__ Dk,
                                                         long n_ov, int n_aux,
                                                         const double* __restrict__ xs, double eta, int nr,
                                                         double* __restrict__ U) {
  __shared__ float Ah_s[TK][TM + 4], Al_s[TK][TM + 4];
  __shared__ float Bh_s[TK][TN + 4], Bl_s[TK][TN + 4];
  const int M = 2 * nr;
  const int m0 = blockIdx.y * TM;
  const long k0c = (long)blockIdx.x * TN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float ah_[4][4], al_[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) ah_[i][j] = al_[i][j] = 0.f;
  for (int p0 = 0; p0 < n_aux; p0 += TK) {
    {
      const int r = tid >> 2, k4 = (tid & 3) * 4;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int P = p0 + k4 + u;
        float h = 0.f, l = 0.f;
        if (m0 + r < M && P < n_aux) df_split(V[(long)(m0 + r) * n_aux + P], h, l);
        Ah_s[k4 + u][r] = h;
        Al_s[k4 + u][r] = l;
      }
      const int kr = tid >> 4, c4 = (tid & 15) * 4;
      const int P = p0 + kr;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long k = k0c + c4 + u;
        const bool in = P < n_aux && k < n_ov;
        Bh_s[kr][c4 + u] = in ? Bh[(long)P * ldh + k] : 0.f;
        Bl_s[kr][c4 + u] = in ? Bl[(long)P * n_ov + k] : 0.f;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < TK; ++kk) {
      float a_h[4], a_l[4], b_h[4], b_l[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int c = 2 * ty + (i & 1) + 32 * (i >> 1);
        a_h[i] = Ah_s[kk][c];
        a_l[i] = Al_s[kk][c];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        b_h[j] = Bh_s[kk][tx + 16 * j];
        b_l[j] = Bl_s[kk][tx + 16 * j];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) df_mac(a_h[i], a_l[i], b_h[j], b_l[j], ah_[i][j], al_[i][j]);
    }
    __syncthreads();
  }
  const double e2 = eta * eta;
#pragma unroll
  for (int ip = 0; ip < 2; ++ip) {
    const int r = m0 + 2 * ty + 32 * ip;
    if (r >= M) continue;
    const double x = xs[r >> 1];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long k = k0c + tx + 16 * j;
      if (k >= n_ov) continue;
      const double tr = (double)ah_[2 * ip][j] + (double)al_[2 * ip][j];
      const double ti = -((double)ah_[2 * ip + 1][j] + (double)al_[2 * ip + 1][j]);
      const double D = Dk[k];
      const double a1 = x - D, a2 = -x - D;
      const double d1 = a1 * a1 + e2, d2 = a2 * a2 + e2;
      const double cr = 2.0 * (a1 / d1 + a2 / d2);
      const double ci = -2.0 * eta * (1.0 / d1 + 1.0 / d2);
      U[(long)r * n_ov + k] = cr * tr - ci * ti;
      U[(long)(r + 1) * n_ov + k] = cr * ti + ci * tr;
    }
  }
}

// df gemm2: acc[r][P] = sum_k U[r][k] B[P][k]; out = the real embedding [u - acc_re; -v - acc_im] (op_gemm2 mode 1).
__global__ void __launch_bounds__(NT) op_gemm2_df_kernel(const double* __restrict__ U, const float* __restrict__ Bh,
                                                         const float* __restrict__ Bl, long ldh, int n_aux, long n_ov,
                                                         int nr,
                                                         const double* __restrict__ V, double* __restrict__ out) {
  __shared__ float Ah_s[TK][TM + 4], Al_s[TK][TM + 4];
  __shared__ float Bh_s[TK][TN + 4], Bl_s[TK][TN + 4];
  const int M = 2 * nr;
  const int m0 = blockIdx.y * TM;
  const int q0 = blockIdx.x * TN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float ah_[4][4], al_[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) ah_[i][j] = al_[i][j] = 0.f;
  const int lr = tid >> 2, lk = (tid & 3) * 4;
  for (long k0 = 0; k0 < n_ov; k0 += TK) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long k = k0 + lk + u;
      float h = 0.f, l = 0.f;
      if (m0 + lr < M && k < n_ov) df_split(U[(long)(m0 + lr) * n_ov + k], h, l);
      Ah_s[lk + u][lr] = h;
      Al_s[lk + u][lr] = l;
      const bool in = q0 + lr < n_aux && k < n_ov;
      Bh_s[lk + u][lr] = in ? Bh[(long)(q0 + lr) * ldh + k] : 0.f;
      Bl_s[lk + u][lr] = in ? Bl[(long)(q0 + lr) * n_ov + k] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < TK; ++kk) {
      float a_h[4], a_l[4], b_h[4], b_l[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int c = 2 * ty + (i & 1) + 32 * (i >> 1);
        a_h[i] = Ah_s[kk][c];
        a_l[i] = Al_s[kk][c];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        b_h[j] = Bh_s[kk][tx + 16 * j];
        b_l[j] = Bl_s[kk][tx + 16 * j];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) df_mac(a_h[i], a_l[i], b_h[j], b_l[j], ah_[i][j], al_[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = m0 + 2 * ty + (i & 1) + 32 * (i >> 1);
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int P = q0 + tx + 16 * j;
      if (P >= n_aux) continue;
      const double v = (double)ah_[i][j] + (double)al_[i][j];
      const double vin = V[(long)r * n_aux + P];
      out[(long)r * n_aux + P] = ((r & 1) ? -vin : vin) - v;
    }
  }
}

__global__ void df_split_kernel(const double* __restrict__ x, long n, float* __restrict__ h, float* __restrict__ l) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    float hh, ll;
    df_split(x[i], hh, ll);
    if (h) h[i] = hh;
    l[i] = ll;
  }
}

}  // namespace

void launch_df_split(const double* x, long n, float* h, float* l, cudaStream_t s) {
  if (n > 0) df_split_kernel<<<1216, 256, 0, s>>>(x, n, h, l);
}

void launch_op_gemm1_df(const double* V, const float* Bh, const float* Bl, long ldh, const double* Dk, long n_ov,
                        int n_aux, const double* x, double eta, int nr, double* U, cudaStream_t s) {
  const dim3 grid((unsigned)((n_ov + TN - 1) / TN), (2 * nr + TM - 1) / TM);
  if (nr > 0) op_gemm1_df_kernel<<<grid, NT, 0, s>>>(V, Bh, Bl, ldh, Dk, n_ov, n_aux, x, eta, nr, U);
}

void launch_op_gemm2_df(const double* U, const float* Bh, const float* Bl, long ldh, int n_aux, int n_ov, int nr,
                        const double* V, double* out, cudaStream_t s) {
  const dim3 grid((n_aux + TN - 1) / TN, (2 * nr + TM - 1) / TM);
  if (nr > 0) op_gemm2_df_kernel<<<grid, NT, 0, s>>>(U, Bh, Bl, ldh, n_aux, (long)n_ov, nr, V, out);
}

void launch_deriv_resonant(const double* V64, const double* B, long n_ov, int n_aux, const double* Dsort,
                           const int* kidx, const double* xs, int nr, double eta, double cut, double* dw,
                           cudaStream_t s) {
  if (nr > 0) deriv_resonant_kernel<<<nr, 256, 0, s>>>(V64, B, n_ov, n_aux, Dsort, kidx, xs, eta, cut, dw);
}

// ------------------------------------------------------------------ launchers
template <typename T>
void launch_pi_syrk(const T* B, const double* Dk, long n_ov, int n_aux, const double* xi, int n_xi, T* out, int mode,
                    cudaStream_t s) {
  int nb = (n_aux + TM - 1) / TM;
  dim3 grid(nb * (nb + 1) / 2, n_xi);
  pi_syrk_kernel<T><<<grid, NT, 0, s>>>(B, Dk, n_ov, n_aux, xi, out, mode);
}

void launch_pi_complex_dense(const double* B, const double* Dk, long n_ov, int n_aux, double x, double eta, double* Ar,
                             double* Ai, cudaStream_t s) {
  int nb = (n_aux + TM - 1) / TM;
  dim3 grid(nb, nb);
  pi_complex_kernel<<<grid, NT, 0, s>>>(B, Dk, n_ov, n_aux, x, eta, Ar, Ai);
}

template <typename T>
void launch_cholesky(T* base, int n, long stride, int batch, int* info, cudaStream_t s) {
  cholesky_kernel<T><<<batch, CH_THREADS, 0, s>>>(base, n, stride, info);
}

int trsm_w_default_ctas() {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return 2 * (nsm > 0 ? nsm : 148);
}

template <typename T>
size_t trsm_w_scratch_elems(int n, int n_cta) {
  return (size_t)n_cta * (size_t)(((n + 63) / 64) * 64) * 64;
}

template <typename T>
cudaError_t launch_trsm_w(const T* Lbase, long Lstride, int n, int n_g, const int* g_out, const T* Bn, int R,
                          double* W, int w_ld, T* scratch, int n_cta, cudaStream_t s) {
  size_t smem = sizeof(T) * (2 * TK * (TM + 4) + 2 * 64 * 65) + sizeof(double) * 2 * 16 * 64;
  cudaError_t e = cudaFuncSetAttribute(trsm_w_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  long items = (long)n_g * ((R + 63) / 64);
  int grid = (int)(items < n_cta ? items : n_cta);
  if (grid <= 0) return cudaSuccess;
  // cudaLaunchKernel returns this launch's own status (an earlier error pending on the thread is left alone)
  void* args[] = {(void*)&Lbase, (void*)&Lstride, (void*)&n, (void*)&n_g, (void*)&g_out, (void*)&Bn,
                  (void*)&R, (void*)&W, (void*)&w_ld, (void*)&scratch};
  return cudaLaunchKernel((const void*)trsm_w_kernel<T>, dim3(grid), dim3(NT), args, smem, s);
}

template <typename T>
void launch_op_gemm1(const T* V, const T* B, const double* Dk, long n_ov, int n_aux, const double* x, double eta,
                     int nr, T* U, int mode, cudaStream_t s, double* dw, double cut, long ldb, const int* run_if) {
  dim3 grid((unsigned)((n_ov + TN - 1) / TN), (2 * nr + TM - 1) / TM);
  op_gemm1_kernel<T><<<grid, NT, 0, s>>>(V, B, Dk, n_ov, n_aux, x, eta, nr, U, mode, dw, cut,
                                         ldb > 0 ? ldb : n_ov, run_if);
}

template <typename T>
void launch_op_gemm2(const T* U, const T* B, int n_aux, int n_ov, int nr, const T* V, T* out, int mode,
                     cudaStream_t s, const int* run_if) {
  dim3 grid((n_aux + TN - 1) / TN, (2 * nr + TM - 1) / TM);
  op_gemm2_kernel<T><<<grid, NT, 0, s>>>(U, B, n_aux, (long)n_ov, nr, V, out, mode, run_if);
}

#define GW_INST(T)                                                                                              \
  template void launch_pi_syrk<T>(const T*, const double*, long, int, const double*, int, T*, int,             \
                                  cudaStream_t);                                                                \
  template void launch_cholesky<T>(T*, int, long, int, int*, cudaStream_t);                                     \
  template size_t trsm_w_scratch_elems<T>(int, int);                                                            \
  template cudaError_t launch_trsm_w<T>(const T*, long, int, int, const int*, const T*, int, double*, int, T*,   \
                                        int, cudaStream_t);                                                     \
  template void launch_op_gemm1<T>(const T*, const T*, const double*, long, int, const double*, double, int,    \
                                   T*, int, cudaStream_t, double*, double, long, const int*);                   \
  template void launch_op_gemm2<T>(const T*, const T*, int, int, int, const T*, T*, int, cudaStream_t,          \
                                   const int*);
GW_INST(double)
GW_INST(float)
#undef GW_INST

}  // namespace gw

// =====================================================================================================
// W table from caller-supplied Cholesky factors without any device allocation.
//
// Some callers cannot allocate device memory when they call into this library: a serving process that
// reserves all GPU memory for its own pool at start-up, a host application whose allocator forbids
// cudaMalloc after initialisation, or code on a latency-critical path where an allocation (which may
// synchronise the device) is not acceptable.  gw_w_table_noalloc gives them the W-table triangular solves
// with the per-CTA work space taken from the fixed array below instead of cudaMalloc.
// =====================================================================================================
#define GW_NOALLOC_SCRATCH_BYTES (32u << 20)   // 32 MiB, held by every GPU that loads the library
#define GW_NOALLOC_MAX_MATS 4096

static __device__ __align__(256) unsigned char g_noalloc_scratch[GW_NOALLOC_SCRATCH_BYTES];
static __device__ __align__(256) int g_noalloc_index[GW_NOALLOC_MAX_MATS];

namespace {
struct NoallocDevice {
  void* scratch = nullptr;
  int* index = nullptr;
  bool ready = false;
};
std::mutex g_noalloc_mu;
NoallocDevice g_noalloc_dev[128];
int g_noalloc_host_index[GW_NOALLOC_MAX_MATS];
}  // namespace

extern "C" gw_status gw_w_table_noalloc(const double* L, int n_aux, int n_mats, const double* Bn, int n_rows,
                                        double* W, int w_ld, void* stream) {
  if (!L || !Bn || !W || n_aux <= 0 || n_mats <= 0 || n_rows <= 0 || w_ld < n_mats) return GW_ERR_ARG;
  if (n_mats > GW_NOALLOC_MAX_MATS) return GW_ERR_ARG;
  const size_t slice = (size_t)((n_aux + 63) / 64) * 64 * 64 * sizeof(double);
  if (slice > GW_NOALLOC_SCRATCH_BYTES) return GW_ERR_ARG;   // n_aux beyond 65536
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return GW_ERR_CUDA;
  NoallocDevice& d = g_noalloc_dev[dev];
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!d.ready) {
      // once per device, with that device current: device addresses of the fixed arrays and the
      // frequency index table 0, 1, 2, ... (a synchronous copy, before any stream capture)
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return GW_ERR_CUDA;
      d.scratch = p;
      if (cudaGetSymbolAddress(&p, g_noalloc_index) != cudaSuccess) return GW_ERR_CUDA;
      d.index = static_cast<int*>(p);
      for (int i = 0; i < GW_NOALLOC_MAX_MATS; ++i) g_noalloc_host_index[i] = i;
      if (cudaMemcpyToSymbol(g_noalloc_index, g_noalloc_host_index, sizeof(g_noalloc_host_index)) != cudaSuccess)
        return GW_ERR_CUDA;
      d.ready = true;
    }
  }
  int n_cta = (int)(GW_NOALLOC_SCRATCH_BYTES / slice);
  const int full = gw::trsm_w_default_ctas();
  n_cta = n_cta < full ? n_cta : full;
  // the status is this launch's own (cudaFuncSetAttribute, then cudaLaunchKernel): an error that other work left
  // pending on the thread is neither reported here nor cleared
  const cudaError_t e = gw::launch_trsm_w<double>(L, (long)n_aux * n_aux, n_aux, n_mats, d.index, Bn, n_rows, W,
                                                  w_ld, static_cast<double*>(d.scratch), n_cta,
                                                  static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? GW_OK : GW_ERR_CUDA;
}
