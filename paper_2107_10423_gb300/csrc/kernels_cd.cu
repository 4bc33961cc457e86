// Contour-deformation kernels: exchange self-energy, the imaginary-axis quadrature (eq. "inn"),
// batched MINRES recurrences for the residue systems (eq. "rnn", Sec. 3.3), fallback bookkeeping,
// and the step-tree QP search (Sec. 3.4, Fig. "steptree").  All arithmetic here is FP64.
#include "gw_internal.cuh"

#include <cmath>

namespace gw {

namespace {

constexpr int RT = 256;   // threads for per-vector kernels

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; every thread receives the total.  `buf` holds >= 32 doubles.
__device__ double block_sum(double v, double* buf) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) buf[wid] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < nw; ++w) t += buf[w];
  return t;
}

// Sigma_x_nn = -sum_{m < n_occ} sum_P B_nm[t][m][P]^2  (Algorithm 1, Init)
__global__ void sigma_x_kernel(const double* __restrict__ B_nm, int n_bas, int n_aux, int n_occ,
                               double* __restrict__ sx, const int* __restrict__ occ_t) {
  __shared__ double buf[32];
  if (occ_t) n_occ = occ_t[blockIdx.x];
  const double* b = B_nm + (long)blockIdx.x * n_bas * n_aux;
  double acc = 0.0;
  for (long i = threadIdx.x; i < (long)n_occ * n_aux; i += blockDim.x) acc += b[i] * b[i];
  acc = block_sum(acc, buf);
  if (threadIdx.x == 0) sx[blockIdx.x] = -acc;
}

// I_nn(omega) = sum_m [(1/pi) sum_g w_g (W_g - W_0) a/(a^2 + xi_g^2) + W_0 sgn(a)/2], a = omega - e_m,
// and dI/domega = (1/pi) sum_m sum_g w_g (W_g - W_0)(xi_g^2 - a^2)/(a^2 + xi_g^2)^2.
// W layout: [t][m][g], g in [0, n_g) the grid, g = n_g the static point xi = 0.
__global__ void sigma_imag_kernel(const double* __restrict__ W, int n_bas, int n_g, const double* __restrict__ eps,
                                  const double* __restrict__ xi, const double* __restrict__ wt,
                                  const double* __restrict__ omega, int static_sub, double* __restrict__ I,
                                  double* __restrict__ dI, const unsigned char* __restrict__ active,
                                  const int* __restrict__ tmap, const int* __restrict__ spin) {
  __shared__ double buf[32];
  const int t = blockIdx.x;                 // evaluation point; its target's W rows are tw's
  if (active && !active[t]) return;
  const int tw = tmap ? tmap[t] : t;
  eps += spin ? (long)spin[tw] * n_bas : 0;   // the target's own spin (G energies [n_spin][n_bas])
  const double w0 = omega[t];
  const int ld = n_g + 1;
  double si = 0.0, sd = 0.0, sj = 0.0;
  // one warp per state m, lanes over grid points
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int m = wid; m < n_bas; m += nw) {
    const double a = w0 - eps[m];
    const double* Wm = W + ((long)tw * n_bas + m) * ld;
    const double Ws = static_sub ? Wm[n_g] : 0.0;
    double pi_acc = 0.0, pd_acc = 0.0;
    for (int g = lane; g < n_g; g += 32) {
      double x2 = xi[g] * xi[g];
      double den = a * a + x2;
      double dW = Wm[g] - Ws;
      pi_acc += wt[g] * dW * a / den;
      pd_acc += wt[g] * dW * (x2 - a * a) / (den * den);
    }
    si += pi_acc;
    sd += pd_acc;
    if (lane == 0 && static_sub) sj += Ws * (a > 0.0 ? 0.5 : (a < 0.0 ? -0.5 : 0.0));
  }
  si = block_sum(si, buf);
  sd = block_sum(sd, buf);
  sj = block_sum(sj, buf);
  if (threadIdx.x == 0) {
    I[t] = si / M_PI + sj;
    dI[t] = sd / M_PI;
  }
}

template <typename T>
__global__ void gather_rhs_kernel(const double* __restrict__ B_nm, int n_bas, int n_aux, const int* __restrict__ rt,
                                  const int* __restrict__ rm, T* __restrict__ V) {
  const int j = blockIdx.x;
  const double* b = B_nm + ((long)rt[j] * n_bas + rm[j]) * n_aux;
  T* u = V + (long)(2 * j) * n_aux;
  for (int i = threadIdx.x; i < n_aux; i += blockDim.x) {
    u[i] = (T)b[i];
    u[n_aux + i] = T(0);
  }
}

template <typename T>
__global__ void minres_init_kernel(const T* __restrict__ S, int n_aux, double* vprev, double* v, double* d1,
                                   double* d2, double* x, MinresState* st, T* V) {
  __shared__ double buf[32];
  const int j = blockIdx.x;
  const long n2 = 2L * n_aux, off = (long)j * n2;
  double acc = 0.0;
  for (long i = threadIdx.x; i < n2; i += blockDim.x) {
    double r = (double)S[off + i];
    acc += r * r;
  }
  const double beta1 = sqrt(block_sum(acc, buf));
  const double inv = beta1 > 0.0 ? 1.0 / beta1 : 0.0;
  for (long i = threadIdx.x; i < n2; i += blockDim.x) {
    double vi = (double)S[off + i] * inv;
    v[off + i] = vi;
    vprev[off + i] = 0.0;
    d1[off + i] = 0.0;
    d2[off + i] = 0.0;
    x[off + i] = 0.0;
    V[off + i] = (T)vi;
  }
  if (threadIdx.x == 0) {
    MinresState s;
    s.beta = 0.0; s.c2 = 1.0; s.s2 = 0.0; s.c1 = 1.0; s.s1 = 0.0;
    s.phibar = beta1; s.beta1 = beta1; s.pad = 0.0;
    s.iters = 0; s.done = beta1 > 0.0 ? 0 : 1; s.pad0 = s.pad1 = 0;
    st[j] = s;
  }
}

// One Paige-Saunders MINRES step for right-hand side j (CTA j).  P = E v_k from the operator GEMMs.
template <typename T>
__global__ void minres_step_kernel(const T* __restrict__ P, int n_aux, double tol, double* vprev, double* v,
                                   double* d1, double* d2, double* x, MinresState* st, T* V, int* n_active) {
  __shared__ double buf[32];
  const int j = blockIdx.x;
  MinresState s = st[j];
  if (s.done) return;
  const long n2 = 2L * n_aux, off = (long)j * n2;
  // alpha = v . (P - beta vprev)
  double acc = 0.0;
  for (long i = threadIdx.x; i < n2; i += blockDim.x)
    acc += v[off + i] * ((double)P[off + i] - s.beta * vprev[off + i]);
  const double alpha = block_sum(acc, buf);
  acc = 0.0;
  for (long i = threadIdx.x; i < n2; i += blockDim.x) {
    double p = (double)P[off + i] - s.beta * vprev[off + i] - alpha * v[off + i];
    acc += p * p;
  }
  const double beta_next = sqrt(block_sum(acc, buf));
  // QR of the tridiagonal by Givens rotations
  const double eps_k = s.s2 * s.beta;
  const double dbar = s.c2 * s.beta;
  const double delta = s.c1 * dbar + s.s1 * alpha;
  const double gbar = -s.s1 * dbar + s.c1 * alpha;
  const double gamma = hypot(gbar, beta_next);
  bool breakdown = !(gamma > 0.0);
  const double c = breakdown ? 1.0 : gbar / gamma;
  const double sn = breakdown ? 0.0 : beta_next / gamma;
  const double tau = c * s.phibar;
  const double phibar = -sn * s.phibar;
  const double ginv = breakdown ? 0.0 : 1.0 / gamma;
  const bool done = breakdown || fabs(phibar) <= tol * s.beta1 || beta_next == 0.0;
  const double binv = done ? 0.0 : 1.0 / beta_next;
  for (long i = threadIdx.x; i < n2; i += blockDim.x) {
    const double vi = v[off + i];
    const double d = (vi - delta * d1[off + i] - eps_k * d2[off + i]) * ginv;
    x[off + i] += tau * d;
    d2[off + i] = d1[off + i];
    d1[off + i] = d;
    if (!done) {
      const double p = (double)P[off + i] - s.beta * vprev[off + i] - alpha * vi;
      const double vn = p * binv;
      vprev[off + i] = vi;
      v[off + i] = vn;
      V[off + i] = (T)vn;
    }
  }
  if (threadIdx.x == 0) {
    s.beta = beta_next;
    s.c2 = s.c1; s.s2 = s.s1; s.c1 = c; s.s1 = sn;
    s.phibar = phibar;
    s.iters += 1;
    s.done = done ? 1 : 0;
    st[j] = s;
    if (!done) atomicAdd(n_active, 1);
  }
}

template <typename T>
__global__ void minres_finish_kernel(const double* __restrict__ B_nm, int n_bas, int n_aux,
                                     const int* __restrict__ rt, const int* __restrict__ rm,
                                     const double* __restrict__ x, const MinresState* __restrict__ st,
                                     double* w_re, double* w_im, int* iters, double* resnorm, T* V,
                                     double* V64) {
  __shared__ double buf[32];
  const int j = blockIdx.x;
  const double* b = B_nm + ((long)rt[j] * n_bas + rm[j]) * n_aux;
  const long off = (long)j * 2 * n_aux;
  double ar = 0.0, ai = 0.0;
  for (int i = threadIdx.x; i < n_aux; i += blockDim.x) {
    const double x1 = x[off + i], x2 = x[off + n_aux + i];
    ar += b[i] * x1;
    ai += b[i] * x2;
    V[off + i] = (T)(b[i] + x1);     // u = Re y = b + x1
    V[off + n_aux + i] = (T)x2;      // v = -Im y = x2   (delta = x1 - i x2)
    if (V64) {
      V64[off + i] = b[i] + x1;
      V64[off + n_aux + i] = x2;
    }
  }
  ar = block_sum(ar, buf);
  ai = block_sum(ai, buf);
  if (threadIdx.x == 0) {
    w_re[j] = ar;
    w_im[j] = -ai;
    MinresState s = st[j];
    iters[j] = s.iters;
    resnorm[j] = s.beta1 > 0.0 ? fabs(s.phibar) / s.beta1 : 0.0;
  }
}

template <typename T>
__global__ void fallback_rhs_kernel(const double* __restrict__ B_nm, int n_bas, int n_aux, const int* __restrict__ rt,
                                    const int* __restrict__ rm, const int* __restrict__ idx, T* __restrict__ y) {
  const int k = blockIdx.x, j = idx[k];
  const double* b = B_nm + ((long)rt[j] * n_bas + rm[j]) * n_aux;
  T* yr = y + (long)k * 2 * n_aux;
  for (int i = threadIdx.x; i < n_aux; i += blockDim.x) {
    yr[i] = (T)b[i];
    yr[n_aux + i] = T(0);
  }
}

template <typename T>
__global__ void fallback_finish_kernel(const double* __restrict__ B_nm, int n_bas, int n_aux,
                                       const int* __restrict__ rt, const int* __restrict__ rm,
                                       const int* __restrict__ idx, const T* __restrict__ y, double* w_re,
                                       double* w_im, double* resnorm, T* V) {
  __shared__ double buf[32];
  const int k = blockIdx.x, j = idx[k];
  const double* b = B_nm + ((long)rt[j] * n_bas + rm[j]) * n_aux;
  const T* yr = y + (long)k * 2 * n_aux;
  const T* yi = yr + n_aux;
  double ar = 0.0, ai = 0.0;
  for (int i = threadIdx.x; i < n_aux; i += blockDim.x) {
    ar += b[i] * ((double)yr[i] - b[i]);
    ai += b[i] * (double)yi[i];
    V[(long)(2 * j) * n_aux + i] = yr[i];
    V[(long)(2 * j + 1) * n_aux + i] = -yi[i];
  }
  ar = block_sum(ar, buf);
  ai = block_sum(ai, buf);
  if (threadIdx.x == 0) {
    w_re[j] = ar;
    w_im[j] = ai;
    resnorm[j] = 0.0;
  }
}

__global__ void refine_kernel(int stage, const double* __restrict__ B_nm, int n_bas, int n_aux,
                              const int* __restrict__ rt, const int* __restrict__ rm, const int* __restrict__ idx,
                              float* y32, double* y64, float* V32, const float* __restrict__ S32,
                              const double* __restrict__ S64, const int* __restrict__ pos, double* rho) {
  __shared__ double buf[32];
  const int k = blockIdx.x;
  float* yr32 = y32 + (long)k * 2 * n_aux;
  double* yr64 = y64 + (long)k * 2 * n_aux;
  float* u = V32 + (long)(2 * k) * n_aux;
  if (stage == 1) {
    const int j = idx[k];
    const double* b = B_nm + ((long)rt[j] * n_bas + rm[j]) * n_aux;
    if (S64) {
      const int q = pos ? pos[k] : k;
      if (q < 0) {   // solve not selected: zero right-hand side, zero correction
        for (int i = threadIdx.x; i < 2 * n_aux; i += blockDim.x) yr32[i] = 0.0f;
        return;
      }
      const double* S = S64 + (long)(2 * q) * n_aux;
      for (int i = threadIdx.x; i < n_aux; i += blockDim.x) {
        yr32[i] = (float)(b[i] - S[i]);
        yr32[n_aux + i] = (float)(-S[n_aux + i]);
      }
    } else {
      const float* S = S32 + (long)(2 * k) * n_aux;
      for (int i = threadIdx.x; i < n_aux; i += blockDim.x) {
        yr32[i] = (float)(b[i] - (double)S[i]);
        yr32[n_aux + i] = (float)(-(double)S[n_aux + i]);
      }
    }
    return;
  }
  double cn = 0.0, yn = 0.0;
  for (int i = threadIdx.x; i < n_aux; i += blockDim.x) {
    double re, im;
    if (stage == 0) {
      re = yr32[i];
      im = yr32[n_aux + i];
    } else {
      const double cr = yr32[i], ci = yr32[n_aux + i];
      re = yr64[i] + cr;
      im = yr64[n_aux + i] + ci;
      cn += cr * cr + ci * ci;
    }
    yn += re * re + im * im;
    yr64[i] = re;
    yr64[n_aux + i] = im;
    u[i] = (float)re;
    u[n_aux + i] = (float)(-im);
  }
  if (rho) {
    cn = block_sum(cn, buf);
    yn = block_sum(yn, buf);
    if (threadIdx.x == 0) rho[k] = yn > 0.0 ? sqrt(cn / yn) : 0.0;
  }
}

template <typename T>
__global__ void fallback_finish64_kernel(const double* __restrict__ B_nm, int n_bas, int n_aux,
                                         const int* __restrict__ rt, const int* __restrict__ rm,
                                         const int* __restrict__ idx, const double* __restrict__ y64, double* w_re,
                                         double* w_im, double* resnorm, T* V, double* V64) {
  __shared__ double buf[32];
  const int k = blockIdx.x, j = idx[k];
  const double* b = B_nm + ((long)rt[j] * n_bas + rm[j]) * n_aux;
  const double* yr = y64 + (long)k * 2 * n_aux;
  const double* yi = yr + n_aux;
  double ar = 0.0, ai = 0.0;
  for (int i = threadIdx.x; i < n_aux; i += blockDim.x) {
    ar += b[i] * (yr[i] - b[i]);
    ai += b[i] * yi[i];
    V[(long)(2 * j) * n_aux + i] = (T)yr[i];
    V[(long)(2 * j + 1) * n_aux + i] = (T)(-yi[i]);
    if (V64) {
      V64[(long)(2 * j) * n_aux + i] = yr[i];
      V64[(long)(2 * j + 1) * n_aux + i] = -yi[i];
    }
  }
  ar = block_sum(ar, buf);
  ai = block_sum(ai, buf);
  if (threadIdx.x == 0) {
    w_re[j] = ar;
    w_im[j] = ai;
    resnorm[j] = 0.0;
  }
}

__global__ void refine_v64_kernel(int n_aux, const int* __restrict__ sel, const double* __restrict__ y64,
                                  double* __restrict__ V64) {
  const int q = blockIdx.x;
  const double* y = y64 + (long)(sel ? sel[q] : q) * 2 * n_aux;
  double* u = V64 + (long)(2 * q) * n_aux;
  for (int i = threadIdx.x; i < n_aux; i += blockDim.x) {
    u[i] = y[i];
    u[n_aux + i] = -y[n_aux + i];
  }
}

__global__ void w_add_static_kernel(double* W, long R, int n_g, int n_cols) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= R * n_cols) return;
  const long r = i / n_cols;
  const int g = (int)(i - r * n_cols);
  W[r * (n_g + 1) + g] += W[r * (n_g + 1) + n_g];
}

__global__ void residue_reduce_kernel(const int* __restrict__ start, int n_t, const double* __restrict__ coef,
                                      const double* __restrict__ w_re, const double* __restrict__ dw_re,
                                      double* R, double* dR) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_t) return;
  double r = 0.0, d = 0.0;
  for (int j = start[t]; j < start[t + 1]; ++j) {
    r += coef[j] * w_re[j];
    d -= coef[j] * dw_re[j];     // d/domega W(e_m - omega) = -W'(x)
  }
  R[t] = r;
  dR[t] = d;
}

// ------------------------------------------------------------------ QP step tree
__device__ __forceinline__ double sgn(double v) { return v > 0.0 ? 1.0 : (v < 0.0 ? -1.0 : 0.0); }

constexpr double kGold = 0.38196601125010515;   // (3 - sqrt 5)/2

// bracket kinds: 0 none, 1 sign change, 2 same sign (golden-section minimisation of |f| around x)
__device__ void update_bracket(QPState& s, double w1, double f1) {
  if (s.br_kind != 0 && s.a < w1 && w1 < s.b) {
    if (s.br_kind == 1) {
      if (sgn(f1) == sgn(s.fa)) { s.a = w1; s.fa = f1; }
      else { s.b = w1; s.fb = f1; }
      return;
    }
    if (sgn(f1) != sgn(s.fx)) {
      s.br_kind = 1;
      if (w1 < s.x) { s.a = w1; s.fa = f1; s.b = s.x; s.fb = s.fx; }
      else { s.a = s.x; s.fa = s.fx; s.b = w1; s.fb = f1; }
      return;
    }
    if (fabs(f1) < fabs(s.fx)) {
      if (w1 > s.x) { s.a = s.x; s.fa = s.fx; } else { s.b = s.x; s.fb = s.fx; }
      s.x = w1; s.fx = f1;
    } else {
      if (w1 > s.x) { s.b = w1; s.fb = f1; } else { s.a = w1; s.fa = f1; }
    }
    return;
  }
  if (!s.has_prev) return;
  const double w0 = s.omega_prev, f0 = s.f_prev;
  if (sgn(f1) != sgn(f0)) {
    s.br_kind = 1;
    if (w0 < w1) { s.a = w0; s.fa = f0; s.b = w1; s.fb = f1; }
    else { s.a = w1; s.fa = f1; s.b = w0; s.fb = f0; }
    return;
  }
  if (s.br_kind == 0 && fabs(f1) > fabs(f0)) {
    s.br_kind = 2;
    if (w0 < w1) { s.a = w0; s.fa = f0; s.b = w1; s.fb = f1; }
    else { s.a = w1; s.fa = f1; s.b = w0; s.fb = f0; }
    s.x = w0; s.fx = f0;
  }
}

__device__ double golden_point(const QPState& s) {
  if (s.br_kind == 1) return fabs(s.fa) <= fabs(s.fb) ? s.a + kGold * (s.b - s.a) : s.b - kGold * (s.b - s.a);
  return (s.b - s.x) >= (s.x - s.a) ? s.x + kGold * (s.b - s.x) : s.x - kGold * (s.x - s.a);
}

__global__ void qp_init_kernel(QPState* st, const double* omega0, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  QPState s;
  s.omega = omega0[t]; s.f_prev = 0.0; s.omega_prev = 0.0; s.Z = 1.0;
  s.a = s.fa = s.b = s.fb = s.x = s.fx = 0.0;
  s.sigma = s.dsigma = 0.0;
  s.br_kind = 0; s.has_prev = 0; s.iter = 0; s.status = 0;
  st[t] = s;
}

__global__ void qp_step_kernel(QPState* st, const double* __restrict__ R, const double* __restrict__ dR,
                               const double* __restrict__ I, const double* __restrict__ dI,
                               const double* __restrict__ e_n, const double* __restrict__ shift, double tol, int maxit,
                               int n, int linearised) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  QPState s = st[t];
  if (s.status != 0) return;
  const double sig = R[t] - I[t], dsig = dR[t] - dI[t];
  s.sigma = sig;
  s.dsigma = dsig;
  const double Z = 1.0 / (1.0 - dsig);
  s.Z = Z;
  if (linearised) {
    // one Newton step of f(w) = e + shift + Sigma_c(w) - w from the starting point w0:
    // e_QP = w0 + Z f(w0), Z = 1/(1 - Sigma_c'(w0)); from w0 = e this is e + Z (shift + Sigma_c(e))
    const double w0 = s.omega;
    s.omega = w0 == e_n[t] ? e_n[t] + Z * (shift[t] + sig) : w0 + Z * (e_n[t] + shift[t] + sig - w0);
    s.status = 1;
    s.iter = 1;
    st[t] = s;
    return;
  }
  const double w = s.omega;
  const double f = e_n[t] + shift[t] + sig - w;
  if (fabs(f) < tol) {
    s.status = 1;
    s.iter += 1;
    st[t] = s;
    return;
  }
  if (s.iter + 1 >= maxit) {
    s.status = 2;
    s.iter += 1;
    st[t] = s;
    return;
  }
  update_bracket(s, w, f);
  double nw;
  if (s.iter == 0) {
    nw = w + fmin(1.0, 0.1 / fabs(f)) * f;       // scaled residual, step capped at 0.1 Ha
  } else if (Z >= 0.3) {
    nw = w + Z * f;                              // Newton
  } else if (s.br_kind != 0) {
    nw = golden_point(s);                        // golden section inside the bracket
  } else if (Z >= 0.1) {
    nw = w + 0.7 * Z * f;                        // scaled Newton
  } else {
    nw = w + fmin(1.0, 0.1 / fabs(f)) * f;       // scaled residual
  }
  s.omega_prev = w;
  s.f_prev = f;
  s.has_prev = 1;
  s.omega = nw;
  s.iter += 1;
  st[t] = s;
}

}  // namespace

void launch_sigma_x(const double* B_nm, int n_t, int n_bas, int n_aux, int n_occ, double* sx, cudaStream_t s,
                    const int* occ_t) {
  if (n_t > 0) sigma_x_kernel<<<n_t, RT, 0, s>>>(B_nm, n_bas, n_aux, n_occ, sx, occ_t);
}

void launch_sigma_imag(const double* W, int n_t, int n_bas, int n_g, const double* eps, const double* xi,
                       const double* wt, const double* omega, int static_sub, double* I, double* dI,
                       const unsigned char* active, cudaStream_t s, const int* tmap, const int* spin) {
  if (n_t > 0)
    sigma_imag_kernel<<<n_t, RT, 0, s>>>(W, n_bas, n_g, eps, xi, wt, omega, static_sub, I, dI, active, tmap, spin);
}

template <typename T>
void launch_gather_rhs(const double* B_nm, int n_bas, int n_aux, const int* rhs_t, const int* rhs_m, int nr, T* V,
                       cudaStream_t s) {
  if (nr > 0) gather_rhs_kernel<T><<<nr, RT, 0, s>>>(B_nm, n_bas, n_aux, rhs_t, rhs_m, V);
}

template <typename T>
void launch_minres_init(const T* S, int nr, int n_aux, double* vprev, double* v, double* d1, double* d2, double* x,
                        MinresState* st, T* V, cudaStream_t s) {
  if (nr > 0) minres_init_kernel<T><<<nr, RT, 0, s>>>(S, n_aux, vprev, v, d1, d2, x, st, V);
}

template <typename T>
void launch_minres_step(const T* P, int nr, int n_aux, double tol, double* vprev, double* v, double* d1, double* d2,
                        double* x, MinresState* st, T* V, int* n_active, cudaStream_t s) {
  if (nr > 0) minres_step_kernel<T><<<nr, RT, 0, s>>>(P, n_aux, tol, vprev, v, d1, d2, x, st, V, n_active);
}

template <typename T>
void launch_minres_finish(const double* B_nm, int n_bas, int n_aux, const int* rhs_t, const int* rhs_m, int nr,
                          const double* x, const MinresState* st, double* w_re, double* w_im, int* iters,
                          double* resnorm, T* V, cudaStream_t s, double* V64) {
  if (nr > 0)
    minres_finish_kernel<T><<<nr, RT, 0, s>>>(B_nm, n_bas, n_aux, rhs_t, rhs_m, x, st, w_re, w_im, iters, resnorm, V,
                                              V64);
}

template <typename T>
void launch_fallback_rhs(const double* B_nm, int n_bas, int n_aux, const int* rt, const int* rm, const int* idx,
                         int nf, T* y, cudaStream_t s) {
  if (nf > 0) fallback_rhs_kernel<T><<<nf, RT, 0, s>>>(B_nm, n_bas, n_aux, rt, rm, idx, y);
}

template <typename T>
void launch_fallback_finish(const double* B_nm, int n_bas, int n_aux, const int* rt, const int* rm, const int* idx,
                            int nf, const T* y, double* w_re, double* w_im, double* resnorm, T* V, cudaStream_t s) {
  if (nf > 0)
    fallback_finish_kernel<T><<<nf, RT, 0, s>>>(B_nm, n_bas, n_aux, rt, rm, idx, y, w_re, w_im, resnorm, V);
}

void launch_refine(int stage, const double* B_nm, int n_bas, int n_aux, const int* rt, const int* rm, const int* idx,
                   int nf, float* y32, double* y64, float* V32, const float* S32, cudaStream_t s,
                   const double* S64, const int* pos, double* rho) {
  if (nf > 0)
    refine_kernel<<<nf, RT, 0, s>>>(stage, B_nm, n_bas, n_aux, rt, rm, idx, y32, y64, V32, S32, S64, pos, rho);
}

template <typename T>
void launch_fallback_finish64(const double* B_nm, int n_bas, int n_aux, const int* rt, const int* rm, const int* idx,
                              int nf, const double* y64, double* w_re, double* w_im, double* resnorm, T* V,
                              cudaStream_t s, double* V64) {
  if (nf > 0)
    fallback_finish64_kernel<T><<<nf, RT, 0, s>>>(B_nm, n_bas, n_aux, rt, rm, idx, y64, w_re, w_im, resnorm, V,
                                                  V64);
}
template void launch_fallback_finish64<float>(const double*, int, int, const int*, const int*, const int*, int,
                                              const double*, double*, double*, double*, float*, cudaStream_t,
                                              double*);

void launch_refine_v64(int m, int n_aux, const int* sel, const double* y64, double* V64, cudaStream_t s) {
  if (m > 0) refine_v64_kernel<<<m, RT, 0, s>>>(n_aux, sel, y64, V64);
}

void launch_w_add_static(double* W, long R, int n_g, int n_cols, cudaStream_t s) {
  const long nt = R * n_cols;
  if (nt > 0) w_add_static_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(W, R, n_g, n_cols);
}

void launch_residue_reduce(const int* start, int n_t, const double* coef, const double* w_re, const double* dw_re,
                           double* R, double* dR, cudaStream_t s) {
  if (n_t > 0) residue_reduce_kernel<<<(n_t + 127) / 128, 128, 0, s>>>(start, n_t, coef, w_re, dw_re, R, dR);
}

// W[r][c] = 0 for every column c outside the positions [p0, p1) (position 0 is column n_g, the static point;
// position p > 0 is grid column p - 1).
__global__ void w_keep_positions_kernel(double* __restrict__ W, long R, int n_g, int p0, int p1) {
  const long N = R * (n_g + 1);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i % (n_g + 1));
    const int pos = c == n_g ? 0 : c + 1;
    if (pos < p0 || pos >= p1) W[i] = 0.0;
  }
}

void launch_w_keep_positions(double* W, long R, int n_g, int p0, int p1, cudaStream_t s) {
  w_keep_positions_kernel<<<1024, 256, 0, s>>>(W, R, n_g, p0, p1);
}

void launch_qp_init(QPState* st, const double* e_n, int n, cudaStream_t s) {
  if (n > 0) qp_init_kernel<<<(n + 127) / 128, 128, 0, s>>>(st, e_n, n);
}

void launch_qp_step(QPState* st, const double* R, const double* dR, const double* I, const double* dI,
                    const double* e_n, const double* shift, double tol, int maxit, int n, int linearised,
                    cudaStream_t s) {
  if (n > 0) qp_step_kernel<<<(n + 127) / 128, 128, 0, s>>>(st, R, dR, I, dI, e_n, shift, tol, maxit, n, linearised);
}

#define GW_INST(T)                                                                                                \
  template void launch_gather_rhs<T>(const double*, int, int, const int*, const int*, int, T*, cudaStream_t);     \
  template void launch_minres_init<T>(const T*, int, int, double*, double*, double*, double*, double*,            \
                                      MinresState*, T*, cudaStream_t);                                            \
  template void launch_minres_step<T>(const T*, int, int, double, double*, double*, double*, double*, double*,    \
                                      MinresState*, T*, int*, cudaStream_t);                                      \
  template void launch_minres_finish<T>(const double*, int, int, const int*, const int*, int, const double*,      \
                                        const MinresState*, double*, double*, int*, double*, T*, cudaStream_t,    \
                                        double*);                                                                 \
  template void launch_fallback_rhs<T>(const double*, int, int, const int*, const int*, const int*, int, T*,       \
                                       cudaStream_t);                                                            \
  template void launch_fallback_finish<T>(const double*, int, int, const int*, const int*, const int*, int,       \
                                          const T*, double*, double*, double*, T*, cudaStream_t);
GW_INST(double)
GW_INST(float)
#undef GW_INST

}  // namespace gw
