// Batched dense solves of the residue systems (1 - Pi(x)) y = b for right-hand sides whose MINRES run
// stayed above the fallback threshold (Sec. 3.3: "the dielectric matrix is actually built" and factorised;
// the paper uses Bunch-Kaufman, this library a complex LU with partial pivoting, which gives the same solution).
// One CTA per matrix; the complex matrix is stored as two real planes (Ar, Ai), row-major n x n.
#include "gw_internal.cuh"
#include "pi_tc.cuh"

#include <algorithm>

namespace gw {
namespace {

constexpr int LU_NB = 32;        // panel width
constexpr int LU_T = 512;        // threads per CTA
constexpr int TTM = 64;          // trailing-update tile rows (16 thread rows x 4)
constexpr int TTN = 128;         // trailing-update tile columns (32 thread columns x 4)

template <typename T>
struct cplx {
  T r, i;
};

template <typename T>
__device__ __forceinline__ cplx<T> cdiv(cplx<T> a, cplx<T> b) {
  const T d = b.r * b.r + b.i * b.i;
  return {(a.r * b.r + a.i * b.i) / d, (a.i * b.r - a.r * b.i) / d};
}

// Block-wide argmax of |a|^2 over rows [r0, n) of column c; ties to the lower row.
template <typename T>
__device__ int pivot_row(const T* Ar, const T* Ai, int n, int c, int r0, double* sv, int* si) {
  double best = -1.0;
  int bidx = r0;
  for (int i = r0 + threadIdx.x; i < n; i += blockDim.x) {
    const double m = (double)Ar[(long)i * n + c] * Ar[(long)i * n + c] + (double)Ai[(long)i * n + c] * Ai[(long)i * n + c];
    if (m > best) { best = m; bidx = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
    if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) { sv[threadIdx.x >> 5] = best; si[threadIdx.x >> 5] = bidx; }
  __syncthreads();
  double bb = -1.0;
  int ii = r0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
    if (sv[w] > bb || (sv[w] == bb && si[w] < ii)) { bb = sv[w]; ii = si[w]; }
  return bb > 0.0 ? ii : -1;
}

// Columns [kbeg, kend) of the factorisation (kbeg a multiple of LU_NB): panels of LU_NB columns, each followed by
// its U12 solve and trailing update restricted to the columns below kend (kbeg = 0, kend = n: the whole LU).
// Rows are swapped in full (all n columns), so the factors and the not yet updated columns stay consistent.
// info[b]: the first zero pivot (column + 1), reset by the launch with kbeg = 0.
template <typename T>
__global__ void __launch_bounds__(LU_T) zlu_kernel(T* Ar_base, T* Ai_base, long stride, int n, int* piv_base,
                                                   int* info, int kbeg, int kend) {
  extern __shared__ __align__(16) unsigned char sm[];
  T* Lr = reinterpret_cast<T*>(sm);               // [TTM][LU_NB+1]
  T* Li = Lr + TTM * (LU_NB + 1);
  T* Ur = Li + TTM * (LU_NB + 1);                 // [LU_NB][TTN+1]
  T* Ui = Ur + LU_NB * (TTN + 1);
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ T L11r[LU_NB * (LU_NB + 1)], L11i[LU_NB * (LU_NB + 1)];   // strictly lower part of the panel's top block
  __shared__ T ucol_r[LU_NB], ucol_i[LU_NB];
  T* Ar = Ar_base + (long)blockIdx.x * stride;
  T* Ai = Ai_base + (long)blockIdx.x * stride;
  int* piv = piv_base + (long)blockIdx.x * n;
  int bad = 0;
  for (int k0 = kbeg; k0 < kend; k0 += LU_NB) {
    const int nb = min(LU_NB, kend - k0), k1 = k0 + nb;
    // ---- panel factorisation (columns k0..k1-1), left-looking with partial pivoting; rows swapped in full.
    // Column c is brought up to date only when it becomes the pivot column: its U part (rows k0..c-1) by a
    // triangular solve with L11 (kept in shared memory), its rows below by one matrix-vector pass (thread per
    // row, contiguous reads), so every panel element is written once.
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int c = k0; c < k1; ++c) {
      const int cc = c - k0;
      if (wid == 0) {
        // U part of column c: u_r = a_rc - sum_{q<r} L11[r][q] u_q, r = k0..c-1 (lane r holds u_r)
        T vr = lane < cc ? Ar[(long)(k0 + lane) * n + c] : T(0);
        T vi = lane < cc ? Ai[(long)(k0 + lane) * n + c] : T(0);
        for (int r = 1; r < cc; ++r) {
          T ar = T(0), ai = T(0);
          if (lane < r) {
            const T lr = L11r[r * (LU_NB + 1) + lane], li = L11i[r * (LU_NB + 1) + lane];
            ar = lr * vr - li * vi;
            ai = lr * vi + li * vr;
          }
          for (int o = 16; o > 0; o >>= 1) {
            ar += __shfl_xor_sync(0xffffffffu, ar, o);
            ai += __shfl_xor_sync(0xffffffffu, ai, o);
          }
          if (lane == r) { vr -= ar; vi -= ai; }
        }
        if (lane < cc) {
          ucol_r[lane] = vr;
          ucol_i[lane] = vi;
          Ar[(long)(k0 + lane) * n + c] = vr;
          Ai[(long)(k0 + lane) * n + c] = vi;
        }
      }
      __syncthreads();
      // rows c..n-1: a_ic -= sum_{q<c} L_iq u_q
      if (cc > 0) {
        for (int i = c + threadIdx.x; i < n; i += blockDim.x) {
          const T* lr = Ar + (long)i * n + k0;
          const T* li = Ai + (long)i * n + k0;
          T sr = T(0), si2 = T(0);
          for (int q = 0; q < cc; ++q) {
            sr += lr[q] * ucol_r[q] - li[q] * ucol_i[q];
            si2 += lr[q] * ucol_i[q] + li[q] * ucol_r[q];
          }
          Ar[(long)i * n + c] -= sr;
          Ai[(long)i * n + c] -= si2;
        }
      }
      __threadfence_block();
      __syncthreads();
      int p = pivot_row(Ar, Ai, n, c, c, sv, si);
      if (p < 0) { bad = c + 1; p = c; }
      if (threadIdx.x == 0) piv[c] = p;
      if (p != c) {
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
          T t = Ar[(long)c * n + j]; Ar[(long)c * n + j] = Ar[(long)p * n + j]; Ar[(long)p * n + j] = t;
          t = Ai[(long)c * n + j]; Ai[(long)c * n + j] = Ai[(long)p * n + j]; Ai[(long)p * n + j] = t;
        }
      }
      __threadfence_block();
      __syncthreads();
      // L11 row cc (multipliers of columns k0..c-1 of the new pivot row)
      if (threadIdx.x < cc) {
        L11r[cc * (LU_NB + 1) + threadIdx.x] = Ar[(long)c * n + k0 + threadIdx.x];
        L11i[cc * (LU_NB + 1) + threadIdx.x] = Ai[(long)c * n + k0 + threadIdx.x];
      }
      const cplx<T> d = {Ar[(long)c * n + c], Ai[(long)c * n + c]};
      const bool dz = (d.r == T(0) && d.i == T(0));
      for (int i = c + 1 + threadIdx.x; i < n; i += blockDim.x) {
        cplx<T> l = {Ar[(long)i * n + c], Ai[(long)i * n + c]};
        l = dz ? cplx<T>{T(0), T(0)} : cdiv(l, d);
        Ar[(long)i * n + c] = l.r;
        Ai[(long)i * n + c] = l.i;
      }
      __threadfence_block();
      __syncthreads();
    }
    if (k1 >= kend) break;
    // ---- U12 = L11^-1 A12 (unit lower), one column per thread, L11 from shared memory
    for (int j = k1 + threadIdx.x; j < kend; j += blockDim.x) {
      T* cr = Ar + (long)k0 * n + j;      // column j of the panel rows; solved entries are read back from cache
      T* ci = Ai + (long)k0 * n + j;
      for (int r = 1; r < nb; ++r) {
        T sr = cr[(long)r * n], sI = ci[(long)r * n];
        for (int q = 0; q < r; ++q) {
          const T lr = L11r[r * (LU_NB + 1) + q], li = L11i[r * (LU_NB + 1) + q];
          const T ur = cr[(long)q * n], ui = ci[(long)q * n];
          sr -= lr * ur - li * ui;
          sI -= lr * ui + li * ur;
        }
        cr[(long)r * n] = sr;
        ci[(long)r * n] = sI;
      }
    }
    __threadfence_block();
    __syncthreads();
    // ---- trailing update A22 -= L21 U12 in TTM x TTN tiles, 4 x 4 complex outputs per thread
    const int ntm = (n - k1 + TTM - 1) / TTM, ntn = (kend - k1 + TTN - 1) / TTN;
    const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
    for (int t = 0; t < ntm * ntn; ++t) {
      const int r0 = k1 + (t / ntn) * TTM, c0 = k1 + (t % ntn) * TTN;
      for (int idx = threadIdx.x; idx < TTM * LU_NB; idx += blockDim.x) {
        const int rr = idx / LU_NB, q = idx % LU_NB;
        const bool okr = (r0 + rr < n) && (q < nb);
        Lr[rr * (LU_NB + 1) + q] = okr ? Ar[(long)(r0 + rr) * n + k0 + q] : T(0);
        Li[rr * (LU_NB + 1) + q] = okr ? Ai[(long)(r0 + rr) * n + k0 + q] : T(0);
      }
      for (int idx = threadIdx.x; idx < LU_NB * TTN; idx += blockDim.x) {
        const int q = idx / TTN, cc = idx % TTN;
        const bool okc = (c0 + cc < kend) && (q < nb);
        Ur[q * (TTN + 1) + cc] = okc ? Ar[(long)(k0 + q) * n + c0 + cc] : T(0);
        Ui[q * (TTN + 1) + cc] = okc ? Ai[(long)(k0 + q) * n + c0 + cc] : T(0);
      }
      __syncthreads();
      // this thread's 4 x 4 outputs are loaded before the K loop so that their latency overlaps the FMAs
      T accr[4][4], acci[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int gi = r0 + ty + 16 * i;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int gj = c0 + tx + 32 * j;
          const bool in = gi < n && gj < kend;
          accr[i][j] = in ? Ar[(long)gi * n + gj] : T(0);
          acci[i][j] = in ? Ai[(long)gi * n + gj] : T(0);
        }
      }
      for (int q = 0; q < nb; ++q) {
        T lr[4], li[4], ur[4], ui[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          lr[i] = Lr[(ty + 16 * i) * (LU_NB + 1) + q];
          li[i] = Li[(ty + 16 * i) * (LU_NB + 1) + q];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          ur[j] = Ur[q * (TTN + 1) + tx + 32 * j];
          ui[j] = Ui[q * (TTN + 1) + tx + 32 * j];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            accr[i][j] = fma(-lr[i], ur[j], accr[i][j]);
            accr[i][j] = fma(li[i], ui[j], accr[i][j]);
            acci[i][j] = fma(-lr[i], ui[j], acci[i][j]);
            acci[i][j] = fma(-li[i], ur[j], acci[i][j]);
          }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int gi = r0 + ty + 16 * i;
        if (gi >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int gj = c0 + tx + 32 * j;
          if (gj < kend) {
            Ar[(long)gi * n + gj] = accr[i][j];
            Ai[(long)gi * n + gj] = acci[i][j];
          }
        }
      }
      __syncthreads();
    }
    __threadfence_block();
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (kbeg == 0) info[blockIdx.x] = bad;
    else if (bad && info[blockIdx.x] == 0) info[blockIdx.x] = bad;
  }
}

// Solve A y = rhs with the LU factors and pivots of zlu_kernel; rhs/y complex in two planes of length n
// (yr, yi), overwritten in place.  Forward and back substitution in blocks of 32 rows: the contribution
// of finished blocks is a parallel mat-vec, the 32 x 32 triangle is solved by one warp.
template <typename T>
__global__ void __launch_bounds__(LU_T) zlu_solve_kernel(const T* Ar_base, const T* Ai_base, long stride, int n,
                                                         const int* piv_base, T* yr_base, T* yi_base, long ystride) {
  __shared__ T pr[LU_T], pi_[LU_T];
  __shared__ T br[32], bi[32];
  const T* Ar = Ar_base + (long)blockIdx.x * stride;
  const T* Ai = Ai_base + (long)blockIdx.x * stride;
  const int* piv = piv_base + (long)blockIdx.x * n;
  T* yr = yr_base + (long)blockIdx.x * ystride;
  T* yi = yi_base + (long)blockIdx.x * ystride;
  if (threadIdx.x == 0) {
    for (int c = 0; c < n; ++c) {
      const int p = piv[c];
      if (p != c) {
        T t = yr[c]; yr[c] = yr[p]; yr[p] = t;
        t = yi[c]; yi[c] = yi[p]; yi[p] = t;
      }
    }
  }
  __threadfence_block();
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // forward: L (unit lower)
  for (int k0 = 0; k0 < n; k0 += 32) {
    const int nb = min(32, n - k0);
    // rows k0..k0+nb-1 minus L[row, 0:k0] y[0:k0]; 16 threads per row
    const int row = k0 + (threadIdx.x >> 4), part = threadIdx.x & 15;
    T sr = T(0), si = T(0);
    if ((threadIdx.x >> 4) < nb)
      for (int q = part; q < k0; q += 16) {
        const T lr = Ar[(long)row * n + q], li = Ai[(long)row * n + q];
        sr += lr * yr[q] - li * yi[q];
        si += lr * yi[q] + li * yr[q];
      }
    for (int o = 8; o > 0; o >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if (part == 0 && (threadIdx.x >> 4) < nb) { br[threadIdx.x >> 4] = yr[row] - sr; bi[threadIdx.x >> 4] = yi[row] - si; }
    __syncthreads();
    if (wid == 0) {
      T vr = lane < nb ? br[lane] : T(0), vi = lane < nb ? bi[lane] : T(0);
      for (int r = 1; r < nb; ++r) {
        // y_r -= sum_{q<r} L[k0+r][k0+q] y_q ; lane r accumulates, y_q broadcast by shuffles
        T ar = T(0), ai = T(0);
        if (lane < r) {
          const T lr = Ar[(long)(k0 + r) * n + k0 + lane], li = Ai[(long)(k0 + r) * n + k0 + lane];
          ar = lr * vr - li * vi;
          ai = lr * vi + li * vr;
        }
        for (int o = 16; o > 0; o >>= 1) {
          ar += __shfl_xor_sync(0xffffffffu, ar, o);
          ai += __shfl_xor_sync(0xffffffffu, ai, o);
        }
        if (lane == r) { vr -= ar; vi -= ai; }
      }
      if (lane < nb) { yr[k0 + lane] = vr; yi[k0 + lane] = vi; }
    }
    __threadfence_block();
    __syncthreads();
  }
  // backward: U (upper, with diagonal)
  const int nblk = (n + 31) / 32;
  for (int bk = nblk - 1; bk >= 0; --bk) {
    const int k0 = bk * 32, nb = min(32, n - k0), k1 = k0 + nb;
    const int row = k0 + (threadIdx.x >> 4), part = threadIdx.x & 15;
    T sr = T(0), si = T(0);
    if ((threadIdx.x >> 4) < nb)
      for (int q = k1 + part; q < n; q += 16) {
        const T ur = Ar[(long)row * n + q], ui = Ai[(long)row * n + q];
        sr += ur * yr[q] - ui * yi[q];
        si += ur * yi[q] + ui * yr[q];
      }
    for (int o = 8; o > 0; o >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if (part == 0 && (threadIdx.x >> 4) < nb) { br[threadIdx.x >> 4] = yr[row] - sr; bi[threadIdx.x >> 4] = yi[row] - si; }
    __syncthreads();
    if (wid == 0) {
      T vr = lane < nb ? br[lane] : T(0), vi = lane < nb ? bi[lane] : T(0);
      for (int r = nb - 1; r >= 0; --r) {
        // y_r = (b_r - sum_{q>r} U[k0+r][k0+q] y_q) / U[k0+r][k0+r]
        T ar = T(0), ai = T(0);
        if (lane > r && lane < nb) {
          const T ur = Ar[(long)(k0 + r) * n + k0 + lane], ui = Ai[(long)(k0 + r) * n + k0 + lane];
          ar = ur * vr - ui * vi;
          ai = ur * vi + ui * vr;
        }
        for (int o = 16; o > 0; o >>= 1) {
          ar += __shfl_xor_sync(0xffffffffu, ar, o);
          ai += __shfl_xor_sync(0xffffffffu, ai, o);
        }
        if (lane == r) {
          const cplx<T> num = {vr - ar, vi - ai};
          const cplx<T> dd = {Ar[(long)(k0 + r) * n + k0 + r], Ai[(long)(k0 + r) * n + k0 + r]};
          const cplx<T> q = (dd.r == T(0) && dd.i == T(0)) ? cplx<T>{T(0), T(0)} : cdiv(num, dd);
          vr = q.r;
          vi = q.i;
        }
        // broadcast of the solved y_r happens through the next iterations' shuffles (lane r holds it)
      }
      if (lane < nb) { yr[k0 + lane] = vr; yi[k0 + lane] = vi; }
    }
    __threadfence_block();
    __syncthreads();
  }
  (void)pr;
  (void)pi_;
}

// ---------------------------------------------------------------------------------------------------------------
// Blocked LU with the trailing update on the tensor cores (FP32 factors).  Per panel of TC_PW columns [k0, kend):
//   1. zlu_kernel factors the panel (rows k0..n-1, partial pivoting, rows swapped in full);
//   2. zlu_trsm_kernel: U12 = L11^-1 A12 for the columns right of the panel;
//   3. the complex update A22 -= L21 U12 as one real product with K = 2 TC_PW:
//        [Re; Im] A22 -= [[Re L, -Im L]; [Im L, Re L]] [Re U12; Im U12],
//      L21 and U12 split into three BF16 parts (six products, about FP32-accurate) by lu_split_l/u_kernel and
//      multiplied by tc_gemm_ex, whose epilogue subtracts the stacked result from the two planes.
constexpr int TC_PW = 64;
constexpr int TC_LDK = 2 * TC_PW;           // row length of the split operands (a multiple of 8)

// One thread per column j >= kend: rows k0..kend-1 of column j solved with the unit lower L11 (shared memory);
// the column itself is held in shared memory (thread-private slots, conflict-free).
// lim: elements addressable from Ar_base (the Ai plane and every matrix of the batch lie inside it); an index at
// or beyond it is recorded in *err (code 61) and skipped.
__global__ void __launch_bounds__(128) zlu_trsm_kernel(float* Ar_base, float* Ai_base, long stride, int n, int k0,
                                                       int kend, long lim, int* err) {
  extern __shared__ float trsm_sm[];
  float* Lr = trsm_sm;                        // [TC_PW][TC_PW + 1]
  float* Li = Lr + TC_PW * (TC_PW + 1);
  float* Ur = Li + TC_PW * (TC_PW + 1);       // [TC_PW][128]
  float* Ui = Ur + TC_PW * 128;
  float* Ar = Ar_base + (long)blockIdx.y * stride;
  float* Ai = Ai_base + (long)blockIdx.y * stride;
  const int pw = kend - k0;
  const long ai_off = Ai_base - Ar_base;
  if ((long)blockIdx.y * stride + ai_off + (long)n * n > lim || pw > TC_PW || pw < 1) {
    if (threadIdx.x == 0) atomicCAS(err, 0, 61);
    return;
  }
  for (int idx = threadIdx.x; idx < pw * pw; idx += blockDim.x) {
    const int r = idx / pw, q = idx % pw;
    Lr[r * (TC_PW + 1) + q] = Ar[(long)(k0 + r) * n + k0 + q];
    Li[r * (TC_PW + 1) + q] = Ai[(long)(k0 + r) * n + k0 + q];
  }
  const int t = threadIdx.x;
  const int j = kend + blockIdx.x * 128 + t;
  if (j < n)
    for (int r = 0; r < pw; ++r) {
      Ur[r * 128 + t] = Ar[(long)(k0 + r) * n + j];
      Ui[r * 128 + t] = Ai[(long)(k0 + r) * n + j];
    }
  __syncthreads();
  if (j >= n) return;
  for (int r = 1; r < pw; ++r) {
    float sr = Ur[r * 128 + t], si = Ui[r * 128 + t];
    for (int q = 0; q < r; ++q) {
      const float lr = Lr[r * (TC_PW + 1) + q], li = Li[r * (TC_PW + 1) + q];
      const float ur = Ur[q * 128 + t], ui = Ui[q * 128 + t];
      sr -= lr * ur - li * ui;
      si -= lr * ui + li * ur;
    }
    Ur[r * 128 + t] = sr;
    Ui[r * 128 + t] = si;
  }
  for (int r = 1; r < pw; ++r) {
    Ar[(long)(k0 + r) * n + j] = Ur[r * 128 + t];
    Ai[(long)(k0 + r) * n + j] = Ui[r * 128 + t];
  }
}

__device__ __forceinline__ void split3(float v, __nv_bfloat16* p0, __nv_bfloat16* p1, __nv_bfloat16* p2, long o) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  const float r = v - __bfloat162float(h);
  const __nv_bfloat16 l = __float2bfloat16_rn(r);
  p0[o] = h;
  p1[o] = l;
  p2[o] = __float2bfloat16_rn(r - __bfloat162float(l));
}

// Rows of the stacked left operand for the m = n - kend rows below the panel: row r = [Re L_r, -Im L_r],
// row m + r = [Im L_r, Re L_r] (L_r = row kend + r, panel columns k0..k0+TC_PW-1); out [batch][2m][TC_LDK].
// lim as in zlu_trsm_kernel; wlim: elements of each operand part (codes 62, 63).
__global__ void lu_split_l_kernel(const float* Ar_base, const float* Ai_base, long stride, int n, int k0, int kend,
                                  __nv_bfloat16* p0, __nv_bfloat16* p1, __nv_bfloat16* p2, long lim, long wlim,
                                  int* err) {
  const int m = n - kend;
  const int r = 2 * blockIdx.x + (threadIdx.x >> 7), q = threadIdx.x & 127;
  if (r >= m) return;
  const float* Ar = Ar_base + (long)blockIdx.y * stride;
  const float* Ai = Ai_base + (long)blockIdx.y * stride;
  const long src = (long)(kend + r) * n + k0 + (q & (TC_PW - 1));
  if ((long)blockIdx.y * stride + (Ai_base - Ar_base) + src >= lim) { atomicCAS(err, 0, 62); return; }
  const float lr = Ar[src], li = Ai[src];
  const long ob = (long)blockIdx.y * 2 * m * TC_LDK;
  if (ob + (long)(m + r) * TC_LDK + q >= wlim) { atomicCAS(err, 0, 63); return; }
  split3(q < TC_PW ? lr : -li, p0, p1, p2, ob + (long)r * TC_LDK + q);
  split3(q < TC_PW ? li : lr, p0, p1, p2, ob + (long)(m + r) * TC_LDK + q);
}

// Rows of the right operand: row c = [Re U12[:, c], Im U12[:, c]] for the columns kend + c (a transpose through
// shared memory); out [batch][m][TC_LDK].
// lim, wlim as in lu_split_l_kernel (codes 64, 65).
__global__ void lu_split_u_kernel(const float* Ar_base, const float* Ai_base, long stride, int n, int k0, int kend,
                                  __nv_bfloat16* p0, __nv_bfloat16* p1, __nv_bfloat16* p2, long lim, long wlim,
                                  int* err) {
  __shared__ float tile[TC_LDK][33];
  const int m = n - kend, c0 = blockIdx.x * 32;
  const float* Ar = Ar_base + (long)blockIdx.y * stride;
  const float* Ai = Ai_base + (long)blockIdx.y * stride;
  const long ai_off = Ai_base - Ar_base;
  for (int q = threadIdx.y; q < TC_LDK; q += blockDim.y) {
    const float* pl = q < TC_PW ? Ar : Ai;
    const int c = c0 + threadIdx.x;
    const long src = (long)(k0 + (q & (TC_PW - 1))) * n + kend + c;
    const bool in = (long)blockIdx.y * stride + (q < TC_PW ? 0 : ai_off) + src < lim;
    if (c < m && !in) atomicCAS(err, 0, 64);
    tile[q][threadIdx.x] = (c < m && in) ? pl[src] : 0.f;
  }
  __syncthreads();
  const long ob = (long)blockIdx.y * m * TC_LDK;
  for (int cc = threadIdx.y; cc < 32; cc += blockDim.y) {
    if (c0 + cc >= m) break;
    for (int q = threadIdx.x; q < TC_LDK; q += 32) {
      const long o = ob + (long)(c0 + cc) * TC_LDK + q;
      if (o >= wlim) { atomicCAS(err, 0, 65); continue; }
      split3(tile[q][cc], p0, p1, p2, o);
    }
  }
}

}  // namespace

size_t zlu_tc_work_elems(int n, int batch) {
  const long m = n > TC_PW ? n - TC_PW : 0;
  // three split parts, each holding the left [batch][2m] and the right [batch][m] rows of TC_LDK elements
  return (size_t)3 * batch * 3 * m * TC_LDK;
}

cudaError_t launch_zlu_tc(float* A, long stride, long plane, int n, int batch, int* piv, int* info,
                          __nv_bfloat16* work, size_t work_elems, int* err, cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  const size_t smem = sizeof(float) * (2 * TTM * (LU_NB + 1) + 2 * LU_NB * (TTN + 1));
  cudaError_t e = cudaFuncSetAttribute(zlu_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int trsm_smem = (int)sizeof(float) * (2 * TC_PW * (TC_PW + 1) + 2 * TC_PW * 128);
  e = cudaFuncSetAttribute(zlu_trsm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, trsm_smem);
  if (e != cudaSuccess) return e;
  if (plane + (long)n * n > stride) return cudaErrorInvalidValue;
  const long lim = (long)batch * stride;        // elements of the batch's matrices from A
  // the split operands of one panel update are held for sub-batches of bs matrices
  const size_t per = zlu_tc_work_elems(n, 1);
  if (n > TC_PW && work_elems < per) return cudaErrorInvalidValue;
  const int bs = n > TC_PW ? (int)std::min<size_t>((size_t)batch, work_elems / per) : batch;
  const size_t part = per / 3 * bs;
  __nv_bfloat16* lp[3] = {work, work + part, work + 2 * part};
  for (int k0 = 0; k0 < n; k0 += TC_PW) {
    const int kend = min(k0 + TC_PW, n);
    zlu_kernel<float><<<batch, LU_T, smem, s>>>(A, A + plane, stride, n, piv, info, k0, kend);
    if (kend >= n) break;
    const int m = n - kend;
    zlu_trsm_kernel<<<dim3((m + 127) / 128, batch), 128, trsm_smem, s>>>(A, A + plane, stride, n, k0, kend, lim,
                                                                        err);
    for (int b0 = 0; b0 < batch; b0 += bs) {
      const int nb = std::min(bs, batch - b0);
      float* Ab = A + (long)b0 * stride;
      const long limb = lim - (long)b0 * stride;
      // the left operand [nb][2m] rows, then the right operand [nb][m] rows, in each part's slot
      const long lsz = (long)nb * 2 * m * TC_LDK;
      __nv_bfloat16* ub[3] = {lp[0] + lsz, lp[1] + lsz, lp[2] + lsz};
      lu_split_l_kernel<<<dim3((m + 1) / 2, nb), 256, 0, s>>>(Ab, Ab + plane, stride, n, k0, kend, lp[0], lp[1],
                                                               lp[2], limb, lsz, err);
      lu_split_u_kernel<<<dim3((m + 31) / 32, nb), dim3(32, 8), 0, s>>>(Ab, Ab + plane, stride, n, k0, kend, ub[0],
                                                                        ub[1], ub[2], limb, (long)part - lsz, err);
      TcEpi ep{};
      ep.kind = TC_EPI_SUB2;
      ep.out = Ab + (long)kend * n + kend;
      ep.out_bstride = stride;
      ep.ldo = n;
      ep.plane = plane;
      ep.half = m;
      ep.limit = limb - ((long)kend * n + kend);
      const TcOperand ao{{lp[0], lp[1], lp[2]}}, bo{{ub[0], ub[1], ub[2]}};
      e = tc_gemm_ex(ao, nb, bo, 1, 3, 2 * m, m, TC_LDK, 0, ep, err, s);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaGetLastError();
}

template <typename T>
void launch_zlu(T* Ar, T* Ai, long stride, int n, int batch, int* piv, int* info, cudaStream_t s) {
  const size_t smem = sizeof(T) * (2 * TTM * (LU_NB + 1) + 2 * LU_NB * (TTN + 1));
  cudaFuncSetAttribute(zlu_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (batch > 0) zlu_kernel<T><<<batch, LU_T, smem, s>>>(Ar, Ai, stride, n, piv, info, 0, n);
}

template <typename T>
void launch_zlu_solve(const T* Ar, const T* Ai, long stride, int n, int batch, const int* piv, T* yr, T* yi,
                      long ystride, cudaStream_t s) {
  if (batch > 0) zlu_solve_kernel<T><<<batch, LU_T, 0, s>>>(Ar, Ai, stride, n, piv, yr, yi, ystride);
}

template void launch_zlu<float>(float*, float*, long, int, int, int*, int*, cudaStream_t);
template void launch_zlu<double>(double*, double*, long, int, int, int*, int*, cudaStream_t);
template void launch_zlu_solve<float>(const float*, const float*, long, int, int, const int*, float*, float*, long,
                                      cudaStream_t);
template void launch_zlu_solve<double>(const double*, const double*, long, int, int, const int*, double*, double*,
                                       long, cudaStream_t);

}  // namespace gw
