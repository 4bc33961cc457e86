// C ABI of libgw (include/gw.h): plan lifetime, device memory, and the host-side orchestration of
// Algorithm 1 (imaginary-axis screening, then the per-state QP loop with batched residue solves).
#include "gw.h"
#include "gw_internal.cuh"
#include "pi_tc.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using gw::MinresState;
using gw::QPState;

namespace {

thread_local std::string g_create_error;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct gw_plan {
  gw_config cfg{};
  int n_bas = 0, n_ov = 0, n_t = 0, n_g = 0;
  unsigned flags = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<double> h_eps, h_xi, h_wt, h_shift, h_sx, h_en;
  // open shell: n_spin = 2, per-spin KS energies and occupations, each target's spin; closed shell: n_spin = 1
  int n_spin = 1;
  int occ_s[2] = {0, 0};
  std::vector<double> h_eps_s[2];
  std::vector<int> h_spin;
  int* d_spin = nullptr;        // [n_targets] (open shell only)
  int* d_occ_t = nullptr;       // [n_targets] occupied states of each target's spin (open shell only)
  std::vector<double> h_eps_g[2];   // poles of G per spin (the KS energies, or the updated ones inside gw_evgw)
  double* d_eps_g = nullptr;        // [n_spin][n_bas]
  std::vector<int> h_targets;
  double* d_eps = nullptr;     // energies of W: the pair energies D_ia of Pi
  double* d_B_ia = nullptr;
  double* d_B_nm = nullptr;
  bool own_B = true;
  double* d_xi = nullptr;     // [n_g + 1], last entry 0 (static point)
  double* d_wt = nullptr;     // [n_g]
  double* d_sx = nullptr;
  double* d_shift = nullptr;
  double* d_en = nullptr;
  double* d_W = nullptr;      // [n_t][n_bas][n_g + 1]
  float* d_B_ia_f = nullptr;  // mixed: FP32 copy of B_ia, rows of ld_f elements (16-byte rows for TMA)
  long ld_f = 0;
  float* d_B_nm_f = nullptr;  // mixed: FP32 copy of B_nm
  __nv_bfloat16* d_Bhi = nullptr;   // mixed: BF16 hi/lo split of B_ia, [n_aux][tc_ld(n_ov)]
  __nv_bfloat16* d_Blo = nullptr;
  __nv_bfloat16* d_BThi = nullptr;  // mixed: BF16 hi/lo split of B_ia^T, [n_ov][tc_ld(n_aux)]
  __nv_bfloat16* d_BTlo = nullptr;
  __nv_bfloat16* d_Blo2 = nullptr;  // mixed: third split parts of B_ia and B_ia^T (refinement operator)
  __nv_bfloat16* d_Bp_hi = nullptr; // mixed: BF16 hi/lo split of B_ia in the K-panel layout of the Pi kernel,
                                    // [P][n_aux][256]
  __nv_bfloat16* d_Bp_lo = nullptr;
  __nv_bfloat16* d_BTlo2 = nullptr;
  double* d_D = nullptr;            // pair energies D_ia [n_ov]
  double* d_Dsort = nullptr;        // mixed: D_ia ascending, with the pair index of each entry in d_Dkidx
  int* d_Dkidx = nullptr;
  double D_min = 0.0;               // smallest pair energy
  __nv_bfloat16* d_Bnhi = nullptr;  // mixed: BF16 hi/lo split of the B_nm rows, [n_t*n_bas][tc_ld(n_aux)]
  __nv_bfloat16* d_Bnlo = nullptr;
  __nv_bfloat16* d_Bnlo2 = nullptr;
  bool screening_done = false;
  // spectral-decomposition route (gw_sigma_sd): Casida matrix and eigenvectors, pole weights; valid while sd_done
  DevBuf sd_M, sd_T, sd_cs, sd_off, sd_Om, sd_V, sd_w2, sd_tmap, sd_om, sd_S, sd_dS;
  bool sd_done = false;
  int sd_sweeps = 0;
  // sharding across ranks (gw_set_shard): frequency positions [sh_p0, sh_p1) of the imaginary-axis stage and the
  // residue right-hand sides j with j % sh_world == sh_rank; sums across ranks through sh_reduce
  int sh_rank = 0, sh_world = 1;
  gw_allreduce_fn sh_reduce = nullptr;
  void* sh_ctx = nullptr;
  std::vector<double> sh_buf;
  int ns_iters_last = 0;
  int ns_kmax = 0;
  int ns_ndiff = 0;           // lowest grid points whose W column is built in the difference form
  std::vector<DevBuf*> bufs;
  int tc_tiles_n = 0;          // N_aux the tile-order table of the Pi kernel was built for
  DevBuf ws_mat, ws_info, ws_scratch, ws_gout, ws_xi, tc_part, tc_kind, tc_par, tc_err, tc_w, tc_tiles, ns_E, ns_X, ns_X2, ns_Xa, ns_Xb, ns_T, ns_lam,
      ns_E0, ns_vec;
  DevBuf mr_V, mr_U, mr_S, mr_vprev, mr_v, mr_d1, mr_d2, mr_x, mr_st, mr_rt, mr_rm, mr_xf, mr_wre, mr_wim,
      mr_dwre, mr_it, mr_res, mr_cnt, mr_Vhi, mr_Vlo, mr_Uhi, mr_Ulo, mr_Vlo2, mr_Ulo2, mr_V64;
  DevBuf sg_I, sg_dI, sg_R, sg_dR, sg_om, sg_start, sg_coef, sg_act, sg_tmap, qp_st, qp_om0;
  DevBuf fb_A, fb_y, fb_piv, fb_info, fb_idx, fb_y64, fb_V32, fb_S32, fb_Vp, fb_Up, fb_x, fb_V64, fb_U64, fb_S64, fb_sel,
      fb_pos, fb_rho, fb_xs, fb_Bl, fb_lu;
  int* h_cnt = nullptr;       // pinned
  std::string err;
  gw_stats stats{};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;
  // per-kernel-class timing: events recorded around launches, resolved after each call's final sync
  std::vector<cudaEvent_t> tpool;
  size_t tused = 0;
  struct Mark { int cls; size_t a, b; double flops; };
  std::vector<Mark> marks;

  gw_plan() {
    DevBuf* all[] = {&ws_mat, &ws_info, &ws_scratch, &ws_gout, &ws_xi, &tc_part, &tc_kind, &tc_par, &tc_err, &tc_w, &tc_tiles, &ns_E, &ns_X, &ns_X2, &ns_Xa, &ns_Xb, &ns_T, &ns_lam, &ns_E0, &ns_vec, &mr_V, &mr_U, &mr_S, &mr_vprev,
                     &mr_v, &mr_d1, &mr_d2, &mr_x, &mr_st, &mr_rt, &mr_rm, &mr_xf, &mr_wre, &mr_wim,
                     &mr_dwre, &mr_it, &mr_res, &mr_cnt, &mr_Vhi, &mr_Vlo, &mr_Uhi, &mr_Ulo, &mr_Vlo2, &mr_Ulo2, &mr_V64, &sg_I, &sg_dI, &sg_R, &sg_dR, &sg_om, &sg_start,
                     &sg_coef, &sg_act, &sg_tmap, &qp_st, &qp_om0, &fb_A, &fb_y, &fb_piv, &fb_info, &fb_idx, &fb_y64, &fb_V32, &fb_S32, &fb_Vp, &fb_Up, &fb_x, &fb_V64, &fb_U64, &fb_S64, &fb_sel, &fb_pos, &fb_rho, &fb_xs, &fb_Bl, &fb_lu, &sd_M, &sd_T, &sd_cs, &sd_off, &sd_Om, &sd_V, &sd_w2, &sd_tmap, &sd_om, &sd_S, &sd_dS};
    bufs.assign(all, all + sizeof(all) / sizeof(all[0]));
  }
};

namespace {

gw_status fail(gw_plan* p, gw_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (p) p->err = buf; else g_create_error = buf;
  return st;
}

#define CK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) {                                                                       \
      if (e_ == cudaErrorMemoryAllocation) { cudaGetLastError(); return fail(P, GW_ERR_OOM, "%s: %s", #call, cudaGetErrorString(e_)); } \
      return fail(P, GW_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));                        \
    }                                                                                              \
  } while (0)

#define LAUNCH(expr)                                                                               \
  do {                                                                                             \
    expr;                                                                                          \
    P->stats.n_kernel_launches++;                                                                  \
    cudaError_t e_ = cudaGetLastError();                                                           \
    if (e_ != cudaSuccess) return fail(P, GW_ERR_CUDA, "launch %s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

#define TRY(call)                                                                                  \
  do {                                                                                             \
    gw_status s_ = (call);                                                                         \
    if (s_ != GW_OK) return s_;                                                                    \
  } while (0)

void count_bytes(gw_plan* P, long long delta) {
  P->stats.bytes_device += delta;
  P->stats.bytes_device_peak = std::max(P->stats.bytes_device_peak, P->stats.bytes_device);
}

// Device allocation counted in gw_stats.bytes_device.
template <typename T>
gw_status dmalloc(gw_plan* P, T** p, size_t bytes) {
  CK(cudaMalloc(reinterpret_cast<void**>(p), bytes));
  count_bytes(P, (long long)bytes);
  return GW_OK;
}

gw_status ensure(gw_plan* P, DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return GW_OK;
  if (b.p) {
    CK(cudaStreamSynchronize(P->stream));
    cudaFree(b.p);
    count_bytes(P, -(long long)b.bytes);
    b.p = nullptr;
    b.bytes = 0;
  }
  if (bytes == 0) bytes = 16;
  CK(cudaMalloc(&b.p, bytes));
  count_bytes(P, (long long)bytes);
  b.bytes = bytes;
  return GW_OK;
}

template <typename T>
T* as(DevBuf& b) { return reinterpret_cast<T*>(b.p); }

size_t ws_bytes(const gw_plan* P) {
  return (size_t)(P->cfg.workspace_mb > 0 ? P->cfg.workspace_mb : 8192) << 20;
}

size_t tick(gw_plan* P) {
  if (P->tused == P->tpool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return (size_t)-1;
    P->tpool.push_back(e);
  }
  cudaEventRecord(P->tpool[P->tused], P->stream);
  return P->tused++;
}

void mark(gw_plan* P, int cls, size_t a, double flops) {
  size_t b = tick(P);
  if (a != (size_t)-1 && b != (size_t)-1) P->marks.push_back({cls, a, b, flops});
  P->stats.launches_kernel[cls]++;
}

// Accumulate the recorded intervals (the stream must be synchronised).
void resolve_marks(gw_plan* P) {
  for (const auto& m : P->marks) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, P->tpool[m.a], P->tpool[m.b]) == cudaSuccess) {
      P->stats.ms_kernel[m.cls] += ms;
      P->stats.flops_kernel[m.cls] += m.flops;
    }
  }
  P->marks.clear();
  P->tused = 0;
  cudaGetLastError();
}

double now_ms(gw_plan* P, cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  return (double)ms;
}

// Tensor-core weighted SYRK for `nb` batch entries: out_b = f(B diag(w_b) B^T) with (kind, param) per entry,
// the weights applied inside the kernel (tc_pi_fused).  reset_err = false keeps a bounded-wait code that earlier
// launches of the caller left in tc_err, so that the check at the end reports it.
gw_status tc_weighted_syrk(gw_plan* P, const int* kinds, const double* params, int nb, int mode_even, int mode_odd,
                           float* out, int cls, bool reset_err = true) {
  const int n = P->cfg.n_aux, K = P->n_ov;
  TRY(ensure(P, P->tc_kind, sizeof(int) * nb));
  TRY(ensure(P, P->tc_par, sizeof(double) * nb));
  TRY(ensure(P, P->tc_err, sizeof(int)));
  TRY(ensure(P, P->tc_w, sizeof(float) * (size_t)nb * gw::pf_ldw(K)));
  if (P->tc_tiles_n != n) {                  // tile order of the Pi kernel, uploaded once per plan
    std::vector<uint32_t> order;
    gw::tc_pi_fused_tile_order(n, order);
    TRY(ensure(P, P->tc_tiles, sizeof(uint32_t) * order.size()));
    CK(cudaMemcpy(P->tc_tiles.p, order.data(), sizeof(uint32_t) * order.size(), cudaMemcpyHostToDevice));
    P->tc_tiles_n = n;
  }
  CK(cudaMemcpyAsync(P->tc_kind.p, kinds, sizeof(int) * nb, cudaMemcpyHostToDevice, P->stream));
  CK(cudaMemcpyAsync(P->tc_par.p, params, sizeof(double) * nb, cudaMemcpyHostToDevice, P->stream));
  if (reset_err) CK(cudaMemsetAsync(P->tc_err.p, 0, sizeof(int), P->stream));
  const size_t t0 = tick(P);
  CK(gw::tc_pair_weights(P->d_D, K, as<int>(P->tc_kind), as<double>(P->tc_par),
                         P->cfg.eta, nb, as<float>(P->tc_w), P->stream));
  // split-K partials (only small problems, whose tiles x entry pairs do not fill the GPU, consider a split)
  float* part = nullptr;
  size_t part_bytes = 0;
  if (P->cfg.pi_ksplit != 1 && gw::tc_pi_fused_items(n, nb) < 2L * 152) {
    part_bytes = std::min(ws_bytes(P), (size_t)(P->cfg.pi_ksplit > 0 ? P->cfg.pi_ksplit : 8) * nb * n * n * 4);
    TRY(ensure(P, P->tc_part, part_bytes));
    part = as<float>(P->tc_part);
  }
  int chosen = 1;
  CK(gw::tc_pi_fused(n, K, as<float>(P->tc_w), nb, as<uint32_t>(P->tc_tiles), P->d_Bp_hi, P->d_Bp_lo, mode_even, mode_odd,
                     out, (long)n * n, n, as<int>(P->tc_err), P->stream, P->cfg.tc_max_ctas, P->cfg.pi_ksplit, part,
                     part_bytes, &chosen));
  P->stats.pi_ksplit_last = chosen;
  mark(P, cls, t0, (double)nb * n * n * K);     // symmetric rank-K update: n^2 K flops per entry
  P->stats.n_kernel_launches += 2;
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, P->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
  CK(cudaStreamSynchronize(P->stream));
  if (herr != 0) return fail(P, GW_ERR_TIMEOUT, "tensor-core GEMM: bounded wait ran out (code %d)", herr);
  return GW_OK;
}

// W table on the tensor cores (mixed precision) for nc frequency matrices eps_b = 1 - Pi_b held FP32 in ws_mat:
// Newton-Schulz X <- 2X - (X eps) X from the closed-form first iterate 2a I - a^2 eps (a = 2/(1 + lambda_max)),
// converging quadratically because the spectrum of eps lies in [1, lambda_max]; the last iterate is written as
// eps^-1 - 1, and W[r][g] = b_r^T (eps_g^-1 - 1) b_r is reduced straight out of one more GEMM.
gw_status ns_w_table(gw_plan* P, int g0, int nc) {
  const int n = P->cfg.n_aux, ldn = gw::tc_ld(n);
  const int R = P->n_t * P->n_bas, n_g1 = P->n_g + 1;
  const size_t mat = (size_t)n * n, smat = (size_t)n * ldn, sz = smat * nc;
  // three split parts per operand: the cheap iterations use two, the last iteration and the W reduction three
  TRY(ensure(P, P->ns_E, 3 * sizeof(__nv_bfloat16) * sz));
  TRY(ensure(P, P->ns_Xa, 3 * sizeof(__nv_bfloat16) * sz));
  TRY(ensure(P, P->ns_Xb, 3 * sizeof(__nv_bfloat16) * sz));
  TRY(ensure(P, P->ns_T, 3 * sizeof(__nv_bfloat16) * sz));
  TRY(ensure(P, P->ns_X, sizeof(float) * mat * nc));
  TRY(ensure(P, P->ns_X2, sizeof(float) * mat * nc));
  TRY(ensure(P, P->ns_lam, sizeof(float) * 4 * nc));         // per matrix: lambda estimates, shift, a_b
  TRY(ensure(P, P->ns_vec, sizeof(float) * 2 * (size_t)nc * n));
  TRY(ensure(P, P->tc_err, sizeof(int)));
  CK(cudaMemsetAsync(P->tc_err.p, 0, sizeof(int), P->stream));
  const float* eps = reinterpret_cast<const float*>(P->ws_mat.p);
  auto parts = [&](DevBuf& b) {
    __nv_bfloat16* p0 = as<__nv_bfloat16>(b);
    return gw::TcOperand{{p0, p0 + sz, p0 + 2 * sz}};
  };
  const gw::TcOperand E = parts(P->ns_E), T = parts(P->ns_T);
  const gw::TcOperand Xs[2] = {parts(P->ns_Xa), parts(P->ns_Xb)};
  float* X = as<float>(P->ns_X);
  const size_t t0 = tick(P);
  // Spectrum of each eps_b = 1 - Pi(i xi_b) in [L_b, H_b]: H_b = 1.25 x the power-iteration estimate of
  // lambda_max (power iteration approaches it from below), L_b = max(1, 0.75 x the estimate of lambda_min from the
  // shifted iteration, which approaches it from above); eps >= 1 because -Pi is positive semidefinite.  With
  // a_b = 2/(L_b + H_b) the first iterate X = 2 a I - a^2 eps leaves I - X eps = (I - a eps)^2, every eigenvalue in
  // [0, rho_b^2], rho_b = (H_b - L_b)/(H_b + L_b), and each Newton-Schulz step squares it.  An eigenvalue outside
  // the estimates still converges (0 < a lambda < 2 for lambda < L_b + H_b), only more slowly.
  // One iteration count for every frequency: the first chunk (xi = 0 and the lowest grid points, the widest
  // spectra) fixes it; a later chunk that needs more takes more.
  float* f_hi = as<float>(P->ns_lam);
  float* f_lo = f_hi + nc;
  float* f_ab = f_hi + 3 * nc;
  CK(gw::tc_spectrum_bounds(eps, n, nc, 20, 1.25f, f_hi, f_lo, f_hi + 2 * nc, as<float>(P->ns_vec),
                            as<float>(P->ns_vec) + (size_t)nc * n, P->stream));
  P->stats.n_kernel_launches += 2 + 2 * 2 * 20 + 1;
  std::vector<float> hl(2 * nc);
  CK(cudaMemcpyAsync(hl.data(), f_hi, sizeof(float) * 2 * nc, cudaMemcpyDeviceToHost, P->stream));
  CK(cudaStreamSynchronize(P->stream));
  std::vector<float> ab(nc);
  double rho = 0.0;
  for (int b = 0; b < nc; ++b) {
    const double H = 1.25 * std::max(1.0f, hl[b]);
    const double L = std::max(1.0, 0.75 * (H - hl[nc + b]));
    ab[b] = (float)(2.0 / (L + H));
    rho = std::max(rho, (H - L) / (H + L));
  }
  CK(cudaMemcpyAsync(f_ab, ab.data(), sizeof(float) * nc, cudaMemcpyHostToDevice, P->stream));
  // two-part iterations until rho^(2^k) <= e^-11.5 (about 1e-5), then one three-part iteration (quadratic: to
  // the FP32 floor)
  int k = 2;
  if (rho > 0.0) k = std::max(2, (int)std::ceil(std::log2(11.5 / -std::log(rho))) + 1);
  k = std::min(k, 24);
  if (g0 == 0 || P->ns_kmax == 0) P->ns_kmax = k;
  const int kmax = std::max(k, P->ns_kmax);
  CK(gw::tc_split_rows(eps, nc * n, n, n, const_cast<__nv_bfloat16*>(E.p[0]), const_cast<__nv_bfloat16*>(E.p[1]),
                       P->stream, const_cast<__nv_bfloat16*>(E.p[2])));
  CK(gw::tc_ns_init(eps, n, nc, f_ab, X, const_cast<__nv_bfloat16*>(Xs[0].p[0]),
                    const_cast<__nv_bfloat16*>(Xs[0].p[1]), P->stream, const_cast<__nv_bfloat16*>(Xs[0].p[2])));
  int cur = 0;
  float* Xf[2] = {X, as<float>(P->ns_X2)};
  int xf = 0;
  for (int k = 1; k < kmax; ++k) {
    const bool last = (k == kmax - 1);
    const int ns = last ? 3 : 2;
    if (last) {
      // the products below take X as its own transpose: make the iterate exactly symmetric before the
      // high-precision step, so that its error F maps to -F eps F (quadratic) for any F
      CK(gw::tc_sym_split(Xf[xf], n, nc, Xf[1 - xf], const_cast<__nv_bfloat16*>(Xs[cur].p[0]),
                          const_cast<__nv_bfloat16*>(Xs[cur].p[1]), const_cast<__nv_bfloat16*>(Xs[cur].p[2]),
                          P->stream));
      xf = 1 - xf;
    }
    gw::TcEpi et{};
    et.kind = gw::TC_EPI_AXPBY;
    et.gamma = 1.f;
    et.ldo = n;
    et.ohi = const_cast<__nv_bfloat16*>(T.p[0]);
    et.olo = const_cast<__nv_bfloat16*>(T.p[1]);
    et.olo2 = const_cast<__nv_bfloat16*>(T.p[2]);
    et.ldh = ldn;
    et.oh_bstride = (long)smat;
    // S = X eps   (eps is symmetric, so it is its own K-major B operand)
    CK(gw::tc_gemm_ex(Xs[cur], nc, E, 1, ns, n, n, n, 0, et, as<int>(P->tc_err), P->stream));
    gw::TcEpi ex{};
    ex.kind = gw::TC_EPI_AXPBY;
    ex.xin = Xf[xf];
    ex.x_bstride = (long)mat;
    ex.alpha = 2.f;
    ex.gamma = -1.f;
    ex.beta = last ? -1.f : 0.f;
    ex.out = Xf[xf];
    ex.out_bstride = (long)mat;
    ex.ldo = n;
    ex.ohi = const_cast<__nv_bfloat16*>(Xs[1 - cur].p[0]);
    ex.olo = const_cast<__nv_bfloat16*>(Xs[1 - cur].p[1]);
    ex.olo2 = const_cast<__nv_bfloat16*>(Xs[1 - cur].p[2]);
    ex.ldh = ldn;
    ex.oh_bstride = (long)smat;
    // X <- 2X - S X = 2X - X eps X  (X symmetric: X is its own transpose as the B operand); the last iterate is
    // written as X - I
    CK(gw::tc_gemm_ex(T, nc, Xs[cur], 1, ns, n, n, n, 0, ex, as<int>(P->tc_err), P->stream));
    cur = 1 - cur;
    P->stats.n_kernel_launches += 2;
  }
  mark(P, 2, t0, 2.0 * 2.0 * (double)(kmax - 1) * nc * (double)n * n * n);
  // W table, reduced in the epilogue of one more GEMM into the table zeroed before the chunks:
  //   static point and grid points g >= ns_ndiff:  W[r][g] = b_r^T (eps_g^-1 - 1) b_r
  //   grid points g < ns_ndiff (xi_g well below every D_ia):
  //     W[r][g] - W[r][n_g] = b_r^T eps_g^-1 M_g eps_0^-1 b_r,  M_g = Pi(i xi_g) - Pi(0)
  //                         = 4 xi_g^2 sum_ia B_ia B_ia^T / (D_ia (D_ia^2 + xi_g^2))   (eps_g = eps_0 - M_g).
  // The I term's omega-derivative weighs W_g - W_0 of the diagonal state by w_g/xi_g^2 at the first nodes; there
  // the difference is O(xi^2) and, formed from two separately computed columns, it would carry their rounding
  // error; in this form its error is relative to itself.  W[r][n_g] is added to those columns after the chunks.
  const gw::TcOperand Bn{{P->d_Bnhi, P->d_Bnlo, P->d_Bnlo2}};
  auto wred = [&](const gw::TcOperand& A, int nb, int pos) {
    gw::TcEpi ew{};
    ew.kind = gw::TC_EPI_WRED;
    ew.W = P->d_W;
    ew.wld = n_g1;
    ew.gidx = as<int>(P->ws_gout) + pos;
    ew.bvec = P->d_B_nm_f;
    ew.ldb = n;
    return gw::tc_gemm_ex(A, nb, Bn, 0, 3, n, R, n, 0, ew, as<int>(P->tc_err), P->stream);
  };
  auto shift = [&](const gw::TcOperand& op, int b) {
    return gw::TcOperand{{op.p[0] + b * smat, op.p[1] + b * smat, op.p[2] + b * smat}};
  };
  int b0 = 0;
  if (g0 == 0) {
    if (P->ns_ndiff > 0) {   // keep eps_0^-1 - 1 (split) for the difference columns of later chunks
      TRY(ensure(P, P->ns_E0, 3 * sizeof(__nv_bfloat16) * smat));
      __nv_bfloat16* e0 = as<__nv_bfloat16>(P->ns_E0);
      for (int i = 0; i < 3; ++i)
        CK(cudaMemcpyAsync(e0 + i * smat, Xs[cur].p[i], sizeof(__nv_bfloat16) * smat, cudaMemcpyDeviceToDevice,
                           P->stream));
    }
    b0 = 1;
  }
  // positions [b0, b1) of this chunk are difference columns (position p > 0 holds grid point p - 1)
  const int b1 = std::max(b0, std::min(nc, P->ns_ndiff + 1 - g0));
  const size_t t1 = tick(P);
  if (b0 > 0) CK(wred(Xs[cur], 1, g0));
  if (nc > b1) CK(wred(shift(Xs[cur], b1), nc - b1, g0 + b1));
  mark(P, 3, t1, 2.0 * (b0 + nc - b1) * (double)n * n * R);
  const int nb = b1 - b0;
  if (nb > 0) {
    __nv_bfloat16* e0 = as<__nv_bfloat16>(P->ns_E0);
    const gw::TcOperand E0{{e0, e0 + smat, e0 + 2 * smat}};
    std::vector<int> kinds(nb, 4);
    std::vector<double> xis(nb);
    for (int b = 0; b < nb; ++b) xis[b] = P->h_xi[g0 + b0 + b - 1];
    // M_b in FP32 (ws_mat: eps is no longer needed) and split (ns_E)
    float* Mf = as<float>(P->ws_mat);
    TRY(tc_weighted_syrk(P, kinds.data(), xis.data(), nb, 0, 0, Mf, 0, /*reset_err=*/false));
    const size_t t2 = tick(P);
    CK(gw::tc_split_rows(Mf, nb * n, n, n, const_cast<__nv_bfloat16*>(E.p[0]), const_cast<__nv_bfloat16*>(E.p[1]),
                         P->stream, const_cast<__nv_bfloat16*>(E.p[2])));
    // C_b = M_b eps_0^-1 = M_b E_0 + M_b   (E_0 = eps_0^-1 - 1 is symmetric: its own K-major operand)
    float* C = Xf[1 - xf];
    gw::TcEpi e1{};
    e1.kind = gw::TC_EPI_AXPBY;
    e1.gamma = 1.f;
    e1.alpha = 1.f;
    e1.xin = Mf;
    e1.x_bstride = (long)mat;
    e1.out = C;
    e1.out_bstride = (long)mat;
    e1.ldo = n;
    CK(gw::tc_gemm_ex(E, nb, E0, 0, 3, n, n, n, 0, e1, as<int>(P->tc_err), P->stream));
    // C_b^T = eps_0^-1 M_b, split, as the K-major operand of the next product
    for (int b = 0; b < nb; ++b)
      CK(gw::tc_transpose_split(C + b * mat, n, n, const_cast<__nv_bfloat16*>(T.p[0]) + b * smat,
                                const_cast<__nv_bfloat16*>(T.p[1]) + b * smat, P->stream,
                                const_cast<__nv_bfloat16*>(T.p[2]) + b * smat));
    // K_b = eps_b^-1 M_b eps_0^-1 = E_b C_b + C_b, written split for the reduction
    gw::TcEpi e2{};
    e2.kind = gw::TC_EPI_AXPBY;
    e2.gamma = 1.f;
    e2.alpha = 1.f;
    e2.xin = C;
    e2.x_bstride = (long)mat;
    e2.ldo = n;
    e2.ohi = const_cast<__nv_bfloat16*>(Xs[1 - cur].p[0]);
    e2.olo = const_cast<__nv_bfloat16*>(Xs[1 - cur].p[1]);
    e2.olo2 = const_cast<__nv_bfloat16*>(Xs[1 - cur].p[2]);
    e2.ldh = ldn;
    e2.oh_bstride = (long)smat;
    CK(gw::tc_gemm_ex(shift(Xs[cur], b0), nb, T, 1, 3, n, n, n, 0, e2, as<int>(P->tc_err), P->stream));
    mark(P, 2, t2, 2.0 * 2.0 * nb * (double)n * n * n);
    const size_t t3 = tick(P);
    CK(wred(Xs[1 - cur], nb, g0 + b0));
    mark(P, 3, t3, 2.0 * nb * (double)n * n * R);
    P->stats.n_kernel_launches += 4 + nb;
  }
  P->stats.n_kernel_launches += 5;
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, P->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
  CK(cudaStreamSynchronize(P->stream));
  if (herr != 0) return fail(P, GW_ERR_TIMEOUT, "tensor-core W table: bounded wait ran out (code %d)", herr);
  P->ns_iters_last = kmax;
  return GW_OK;
}

// ---------------------------------------------------------------- imaginary-axis screening
template <typename T>
gw_status screening_T(gw_plan* P, const T* B, const T* Bn) {
  const int n = P->cfg.n_aux;
  const int n_g1 = P->n_g + 1;
  const int R = P->n_t * P->n_bas;
  const bool use_tc = (P->cfg.precision == GW_PREC_MIXED);
  // frequency matrices held at once: <= 8 GiB (and the split-operand budget on the tensor-core path)
  const size_t per = (size_t)n * n * sizeof(T);
  int chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)n_g1, ws_bytes(P) / per));
  if (use_tc) {
    const size_t per_ns = (size_t)n * gw::tc_ld(n) * 24 + (size_t)n * n * 8;   // split E, Xa, Xb, T; FP32 X, eps
    chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)chunk, ws_bytes(P) / per_ns));
  }
  TRY(ensure(P, P->ws_mat, per * chunk));
  TRY(ensure(P, P->ws_info, sizeof(int) * chunk));
  TRY(ensure(P, P->ws_gout, sizeof(int) * n_g1));
  const int n_cta = gw::trsm_w_default_ctas();
  TRY(ensure(P, P->ws_scratch, sizeof(T) * gw::trsm_w_scratch_elems<T>(n, n_cta)));
  // processing order: the static point xi = 0 first, then the grid ascending; gout maps position -> W column
  std::vector<int> gout(n_g1);
  gout[0] = P->n_g;
  for (int g = 0; g < P->n_g; ++g) gout[g + 1] = g;
  CK(cudaMemcpyAsync(P->ws_gout.p, gout.data(), sizeof(int) * n_g1, cudaMemcpyHostToDevice, P->stream));
  std::vector<double> xi_all(n_g1);
  for (int i = 0; i < n_g1; ++i) xi_all[i] = gout[i] < P->n_g ? P->h_xi[gout[i]] : 0.0;
  TRY(ensure(P, P->ws_xi, sizeof(double) * n_g1));
  CK(cudaMemcpyAsync(P->ws_xi.p, xi_all.data(), sizeof(double) * n_g1, cudaMemcpyHostToDevice, P->stream));
  P->ns_kmax = 0;
  // difference-form columns: grid points with xi_g below a tenth of the smallest pair energy (there
  // |Pi(i xi_g) - Pi(0)| <= 1% of |Pi(0)|)
  P->ns_ndiff = 0;
  if (use_tc)
    while (P->ns_ndiff < P->n_g && P->h_xi[P->ns_ndiff] < 0.1 * P->D_min) ++P->ns_ndiff;
  // positions this rank computes: its block [p0, p1), from position 0 when the block holds difference-form
  // columns (they need eps(0)^-1); columns outside the block are zeroed before the sum across ranks
  int p0 = 0, p1 = n_g1;
  if (P->sh_world > 1) gw_shard_columns(P->n_g, P->sh_rank, P->sh_world, &p0, &p1);
  const int p_begin = (use_tc && p0 > 0 && p0 <= P->ns_ndiff) ? 0 : p0;
  if (use_tc || P->sh_world > 1)
    CK(cudaMemsetAsync(P->d_W, 0, sizeof(double) * (size_t)R * n_g1, P->stream));   // W is accumulated / summed
  std::vector<int> info(chunk);
  double ms_pi = 0.0;
  for (int g0 = p_begin; g0 < p1; g0 += chunk) {
    const int nc = std::min(chunk, p1 - g0);
    CK(cudaEventRecord(P->ev0, P->stream));
    if (use_tc) {
      std::vector<int> kinds(nc, 0);
      TRY(tc_weighted_syrk(P, kinds.data(), xi_all.data() + g0, nc, 1, 1, reinterpret_cast<float*>(P->ws_mat.p), 0));
    } else {
      const size_t t0 = tick(P);
      LAUNCH(gw::launch_pi_syrk<T>(B, P->d_D, P->n_ov, n, as<double>(P->ws_xi) + g0, nc,
                                   as<T>(P->ws_mat), 1, P->stream));
      mark(P, 1, t0, (double)nc * n * n * P->n_ov);
    }
    CK(cudaEventRecord(P->ev1, P->stream));
    if (use_tc) {
      CK(cudaStreamSynchronize(P->stream));
      ms_pi += now_ms(P, P->ev0, P->ev1);
      TRY(ns_w_table(P, g0, nc));
      continue;
    }
    size_t t1 = tick(P);
    LAUNCH(gw::launch_cholesky<T>(as<T>(P->ws_mat), n, (long)n * n, nc, as<int>(P->ws_info), P->stream));
    mark(P, 2, t1, (double)nc * n * n * (double)n / 3.0);
    t1 = tick(P);
    LAUNCH(gw::launch_trsm_w<T>(as<T>(P->ws_mat), (long)n * n, n, nc, as<int>(P->ws_gout) + g0, Bn, R, P->d_W,
                                n_g1, as<T>(P->ws_scratch), n_cta, P->stream));
    mark(P, 3, t1, (double)nc * (double)n * n * R);
    CK(cudaMemcpyAsync(info.data(), P->ws_info.p, sizeof(int) * nc, cudaMemcpyDeviceToHost, P->stream));
    CK(cudaStreamSynchronize(P->stream));
    ms_pi += now_ms(P, P->ev0, P->ev1);
    for (int i = 0; i < nc; ++i)
      if (info[i] != 0)
        return fail(P, GW_ERR_NUMERIC, "Cholesky of eps(i xi) failed at frequency %d, pivot %d", g0 + i, info[i]);
  }
  if (use_tc && P->ns_ndiff > 0) LAUNCH(gw::launch_w_add_static(P->d_W, R, P->n_g, P->ns_ndiff, P->stream));
  P->stats.ms_pi = ms_pi;
  if (P->sh_world > 1) {
    // keep the owned columns (positions [p0, p1): position 0 is column n_g, position p > 0 is column p - 1), then
    // sum the tables of all ranks: every column comes from exactly one rank
    LAUNCH(gw::launch_w_keep_positions(P->d_W, R, P->n_g, p0, p1, P->stream));
    const size_t cnt = (size_t)R * n_g1;
    P->sh_buf.resize(cnt);
    CK(cudaMemcpyAsync(P->sh_buf.data(), P->d_W, sizeof(double) * cnt, cudaMemcpyDeviceToHost, P->stream));
    CK(cudaStreamSynchronize(P->stream));
    if (P->sh_reduce(P->sh_buf.data(), (long long)cnt, P->sh_ctx) != 0)
      return fail(P, GW_ERR_CUDA, "shard all-reduce of the W table failed");
    CK(cudaMemcpyAsync(P->d_W, P->sh_buf.data(), sizeof(double) * cnt, cudaMemcpyHostToDevice, P->stream));
    CK(cudaStreamSynchronize(P->stream));
  }
  return GW_OK;
}

gw_status ensure_screening(gw_plan* P) {
  if (P->screening_done) return GW_OK;
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  CK(cudaEventRecord(a, P->stream));
  gw_status st;
  if (P->cfg.precision == GW_PREC_MIXED)
    st = screening_T<float>(P, P->d_B_ia_f, P->d_B_nm_f);
  else
    st = screening_T<double>(P, P->d_B_ia, P->d_B_nm);
  if (st != GW_OK) { cudaEventDestroy(a); cudaEventDestroy(b); return st; }
  CK(cudaEventRecord(b, P->stream));
  CK(cudaEventSynchronize(b));
  P->stats.ms_screening = now_ms(P, a, b);
  resolve_marks(P);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  P->screening_done = true;
  return GW_OK;
}

gw_status tc_operator3(gw_plan* P, int nf, const double* xf, const float* V32, float* S32);
gw_status ensure_third_parts(gw_plan* P);

// Half-width (Ha) of the window around each resonance x = +-D_ia whose derivative terms are computed in FP64.
constexpr double kResonantCut = 0.1;

// BF16 elements of the blocked LU's split panel operands for a fallback batch of fb matrices: the whole batch, or
// as many matrices as fit in 1 GiB (at least one); the panel updates then run in sub-batches.
size_t lu_work_elems(int n, long fb) {
  const size_t one = gw::zlu_tc_work_elems(n, 1);
  const size_t cap = std::max(one, ((size_t)1 << 29) / std::max<size_t>(one, 1) * one);
  return std::min(one * (size_t)std::max(1L, fb), cap);
}

// Dense solves for the MINRES batch slots in `need` (Sec. 3.3: build the dielectric matrix and factorise).
// A_j = 1 - Pi(x_j) is built on the tensor cores (mixed) or by the FP64 SIMT kernel, then factorised by the
// batched complex LU; W and the derivative-pass vectors are written into the slot.
template <typename T>
gw_status dense_fallback(gw_plan* P, const std::vector<int>& need, const int* rt, const int* rm, const double* xf,
                         double* w_re, double* w_im, double* resnorm) {
  const int n = P->cfg.n_aux;
  const size_t mat = (size_t)n * n;
  const int nneed = (int)need.size();
  // batch of dense matrices: A planes <= 8 GiB (one LU launch fills the GPU); the tensor-core build runs in
  // sub-batches sized by the split-operand budget
  int fb = (int)std::max<size_t>(1, ws_bytes(P) / (2 * mat * sizeof(T)));
  fb = std::min(fb, nneed);
  const int sub = fb;
  TRY(ensure(P, P->fb_A, sizeof(T) * 2 * mat * fb));
  TRY(ensure(P, P->fb_y, sizeof(T) * 2 * (size_t)n * fb));
  TRY(ensure(P, P->fb_piv, sizeof(int) * (size_t)n * fb));
  TRY(ensure(P, P->fb_info, sizeof(int) * fb));
  TRY(ensure(P, P->fb_idx, sizeof(int) * nneed));
  if (sizeof(T) == 4) {
    TRY(ensure(P, P->fb_y64, sizeof(double) * 2 * (size_t)n * fb));
    TRY(ensure(P, P->fb_V32, sizeof(float) * 2 * (size_t)n * fb));
    TRY(ensure(P, P->fb_S32, sizeof(float) * 2 * (size_t)n * fb));
    TRY(ensure(P, P->fb_Vp, 3 * sizeof(__nv_bfloat16) * 2 * (size_t)gw::tc_ld(n) * fb));
    TRY(ensure(P, P->fb_Up, 3 * sizeof(__nv_bfloat16) * 2 * (size_t)gw::tc_ld(P->n_ov) * fb));
    TRY(ensure(P, P->tc_err, sizeof(int)));
    TRY(ensure(P, P->fb_x, sizeof(double) * fb));
    TRY(ensure(P, P->fb_xs, sizeof(double) * fb));
    TRY(ensure(P, P->fb_rho, sizeof(double) * fb));
    TRY(ensure(P, P->fb_sel, sizeof(int) * fb));
    TRY(ensure(P, P->fb_pos, sizeof(int) * fb));
    TRY(ensure(P, P->fb_lu, sizeof(__nv_bfloat16) * lu_work_elems(n, fb)));
  }
  CK(cudaMemcpyAsync(P->fb_idx.p, need.data(), sizeof(int) * nneed, cudaMemcpyHostToDevice, P->stream));
  std::vector<double> hx(nneed);
  {
    int mx = 0;
    for (int j : need) mx = std::max(mx, j);
    std::vector<double> xs(mx + 1);
    CK(cudaMemcpyAsync(xs.data(), xf, sizeof(double) * (mx + 1), cudaMemcpyDeviceToHost, P->stream));
    CK(cudaStreamSynchronize(P->stream));
    for (int k = 0; k < nneed; ++k) hx[k] = xs[need[k]];
  }
  std::vector<int> info(fb);
  for (int k0 = 0; k0 < nneed; k0 += fb) {
    const int nf = std::min(fb, nneed - k0);
    T* A = as<T>(P->fb_A);
    if (sizeof(T) == 4) {
      for (int s0 = 0; s0 < nf; s0 += sub) {
        const int ns = std::min(sub, nf - s0);
        std::vector<int> kinds(2 * ns);
        std::vector<double> par(2 * ns);
        for (int k = 0; k < ns; ++k) {
          kinds[2 * k] = 1;
          kinds[2 * k + 1] = 2;
          par[2 * k] = par[2 * k + 1] = hx[k0 + s0 + k];
        }
        TRY(tc_weighted_syrk(P, kinds.data(), par.data(), 2 * ns, 1, 2,
                             reinterpret_cast<float*>(A) + 2 * mat * (size_t)s0, 6));
      }
    } else {
      const size_t t0 = tick(P);
      for (int k = 0; k < nf; ++k)
        LAUNCH(gw::launch_pi_complex_dense(P->d_B_ia, P->d_D, P->n_ov, n, hx[k0 + k],
                                           P->cfg.eta, reinterpret_cast<double*>(A) + 2 * mat * k,
                                           reinterpret_cast<double*>(A) + 2 * mat * k + mat, P->stream));
      mark(P, 6, t0, 4.0 * nf * (double)mat * P->n_ov);
    }
    LAUNCH(gw::launch_fallback_rhs<T>(P->d_B_nm, P->n_bas, n, rt, rm, as<int>(P->fb_idx) + k0, nf, as<T>(P->fb_y),
                                      P->stream));
    const size_t tl = tick(P);
    if (sizeof(T) == 4) {
      // FP32 factors, trailing updates on the tensor cores (about FP32-accurate six-product split); a bounded
      // wait that runs out in its GEMMs is reported by the refinement operator's check below
      CK(cudaMemsetAsync(P->tc_err.p, 0, sizeof(int), P->stream));
      CK(gw::launch_zlu_tc(reinterpret_cast<float*>(A), (long)(2 * mat), (long)mat, n, nf, as<int>(P->fb_piv),
                           as<int>(P->fb_info), as<__nv_bfloat16>(P->fb_lu), P->fb_lu.bytes / sizeof(__nv_bfloat16),
                           as<int>(P->tc_err), P->stream));
      P->stats.n_kernel_launches += 5 * ((n + 63) / 64);
    } else {
      LAUNCH(gw::launch_zlu<T>(A, A + mat, (long)(2 * mat), n, nf, as<int>(P->fb_piv), as<int>(P->fb_info),
                               P->stream));
    }
    LAUNCH(gw::launch_zlu_solve<T>(A, A + mat, (long)(2 * mat), n, nf, as<int>(P->fb_piv), as<T>(P->fb_y),
                                   as<T>(P->fb_y) + n, 2L * n, P->stream));
    mark(P, 7, tl, nf * (8.0 / 3.0 * (double)n * n * n + 8.0 * (double)n * n));
    if (sizeof(T) == 4) {
      // iterative refinement with the FP32 factors (matrix-free residuals), solution accumulated in FP64
      float* y32 = reinterpret_cast<float*>(P->fb_y.p);
      const int* idx = as<int>(P->fb_idx) + k0;
      std::vector<double> xk(hx.begin() + k0, hx.begin() + k0 + nf);
      CK(cudaMemcpyAsync(P->fb_x.p, xk.data(), sizeof(double) * nf, cudaMemcpyHostToDevice, P->stream));
      LAUNCH(gw::launch_refine(0, P->d_B_nm, P->n_bas, n, rt, rm, idx, nf, y32, as<double>(P->fb_y64),
                               as<float>(P->fb_V32), nullptr, P->stream));
      // step 1: residual from the three-part tensor-core operator (about FP32-accurate), FP32 LU correction
      {
        const size_t tr = tick(P);
        TRY(tc_operator3(P, nf, as<double>(P->fb_x), as<float>(P->fb_V32), as<float>(P->fb_S32)));
        mark(P, 8, tr, 2.0 * 2.0 * (2.0 * nf) * n * (double)P->n_ov);
        LAUNCH(gw::launch_refine(1, P->d_B_nm, P->n_bas, n, rt, rm, idx, nf, y32, as<double>(P->fb_y64),
                                 as<float>(P->fb_V32), as<float>(P->fb_S32), P->stream));
        LAUNCH(gw::launch_zlu_solve<T>(A, A + mat, (long)(2 * mat), n, nf, as<int>(P->fb_piv), as<T>(P->fb_y),
                                       as<T>(P->fb_y) + n, 2L * n, P->stream));
        LAUNCH(gw::launch_refine(2, P->d_B_nm, P->n_bas, n, rt, rm, idx, nf, y32, as<double>(P->fb_y64),
                                 as<float>(P->fb_V32), nullptr, P->stream, nullptr, nullptr,
                                 P->cfg.refine_tol > 0.0 ? as<double>(P->fb_rho) : nullptr));
      }
      // step 2, for the solves the first correction shows to be ill-conditioned (|dy|/|y| > refine_tol: a
      // near-resonant x_j, where the operator's FP32-level error limits step 1): residual from the FP64 operator
      if (P->cfg.refine_tol >= 0.0) {
        std::vector<int> sel, pos(nf, -1);
        std::vector<double> xs;
        if (P->cfg.refine_tol > 0.0) {
          std::vector<double> rho(nf);
          CK(cudaMemcpyAsync(rho.data(), P->fb_rho.p, sizeof(double) * nf, cudaMemcpyDeviceToHost, P->stream));
          CK(cudaStreamSynchronize(P->stream));
          for (int k = 0; k < nf; ++k)
            if (!(rho[k] <= P->cfg.refine_tol)) sel.push_back(k);   // NaN selects too
        } else {
          for (int k = 0; k < nf; ++k) sel.push_back(k);
        }
        const int m = (int)sel.size();
        if (m > 0) {
          for (int q = 0; q < m; ++q) {
            pos[sel[q]] = q;
            xs.push_back(hx[k0 + sel[q]]);
          }
          TRY(ensure(P, P->fb_V64, sizeof(double) * 2 * (size_t)n * m));
          TRY(ensure(P, P->fb_S64, sizeof(double) * 2 * (size_t)n * m));
          TRY(ensure(P, P->fb_U64, sizeof(double) * 2 * (size_t)P->n_ov * m));
          CK(cudaMemcpyAsync(P->fb_sel.p, sel.data(), sizeof(int) * m, cudaMemcpyHostToDevice, P->stream));
          CK(cudaMemcpyAsync(P->fb_pos.p, pos.data(), sizeof(int) * nf, cudaMemcpyHostToDevice, P->stream));
          CK(cudaMemcpyAsync(P->fb_xs.p, xs.data(), sizeof(double) * m, cudaMemcpyHostToDevice, P->stream));
          const size_t tr = tick(P);
          LAUNCH(gw::launch_refine_v64(m, n, as<int>(P->fb_sel), as<double>(P->fb_y64), as<double>(P->fb_V64),
                                       P->stream));
          if (P->cfg.refine_df) {
            // double-float (FP32 pair) residual: 48-bit products and sums on the FP32 pipes
            // the hi part of the split is the FP32 copy of B_ia already held by the plan; only the lo part is made
            if (!P->fb_Bl.p) {
              const size_t nb = (size_t)n * P->n_ov;
              TRY(ensure(P, P->fb_Bl, sizeof(float) * nb));
              LAUNCH(gw::launch_df_split(P->d_B_ia, (long)nb, nullptr, as<float>(P->fb_Bl), P->stream));
            }
            LAUNCH(gw::launch_op_gemm1_df(as<double>(P->fb_V64), P->d_B_ia_f, as<float>(P->fb_Bl), P->ld_f, P->d_D,
                                          P->n_ov, n, as<double>(P->fb_xs), P->cfg.eta, m, as<double>(P->fb_U64),
                                          P->stream));
            LAUNCH(gw::launch_op_gemm2_df(as<double>(P->fb_U64), P->d_B_ia_f, as<float>(P->fb_Bl), P->ld_f, n,
                                          P->n_ov, m, as<double>(P->fb_V64), as<double>(P->fb_S64), P->stream));
          } else {
            LAUNCH(gw::launch_op_gemm1<double>(as<double>(P->fb_V64), P->d_B_ia, P->d_D, P->n_ov, n, as<double>(P->fb_xs), P->cfg.eta, m,
                                               as<double>(P->fb_U64), 0, P->stream));
            LAUNCH(gw::launch_op_gemm2<double>(as<double>(P->fb_U64), P->d_B_ia, n, P->n_ov, m,
                                               as<double>(P->fb_V64), as<double>(P->fb_S64), 1, P->stream));
          }
          mark(P, 8, tr, 2.0 * 2.0 * (2.0 * m) * n * (double)P->n_ov);
          LAUNCH(gw::launch_refine(1, P->d_B_nm, P->n_bas, n, rt, rm, idx, nf, y32, as<double>(P->fb_y64),
                                   as<float>(P->fb_V32), nullptr, P->stream, as<double>(P->fb_S64),
                                   as<int>(P->fb_pos)));
          LAUNCH(gw::launch_zlu_solve<T>(A, A + mat, (long)(2 * mat), n, nf, as<int>(P->fb_piv), as<T>(P->fb_y),
                                         as<T>(P->fb_y) + n, 2L * n, P->stream));
          LAUNCH(gw::launch_refine(2, P->d_B_nm, P->n_bas, n, rt, rm, idx, nf, y32, as<double>(P->fb_y64),
                                   as<float>(P->fb_V32), nullptr, P->stream));
          P->stats.n_refine_fp64 += m;
        }
      }
      LAUNCH(gw::launch_fallback_finish64<T>(P->d_B_nm, P->n_bas, n, rt, rm, idx, nf, as<double>(P->fb_y64), w_re,
                                             w_im, resnorm, as<T>(P->mr_V), P->stream, as<double>(P->mr_V64)));
    } else {
      LAUNCH(gw::launch_fallback_finish<T>(P->d_B_nm, P->n_bas, n, rt, rm, as<int>(P->fb_idx) + k0, nf,
                                           as<T>(P->fb_y), w_re, w_im, resnorm, as<T>(P->mr_V), P->stream));
    }
    CK(cudaMemcpyAsync(info.data(), P->fb_info.p, sizeof(int) * nf, cudaMemcpyDeviceToHost, P->stream));
    CK(cudaStreamSynchronize(P->stream));
    for (int k = 0; k < nf; ++k)
      if (info[k] != 0) return fail(P, GW_ERR_NUMERIC, "dense residue solve: zero pivot at column %d", info[k]);
    P->stats.n_fallback += nf;
  }
  return GW_OK;
}

// Residue operator on the tensor cores (mixed precision), for nr right-hand sides held in V32 [2nr][n]:
// GEMM1 t = B^T z with the complex weights c_ia(x_j) fused into its epilogue (written as split BF16),
// GEMM2 B w with either the plain store (mode 0: [Re; Im] of Pi z) or the 2n embedding of (1 - Pi) z (mode 1).
gw_status tc_operator(gw_plan* P, int nr, const double* xf, const float* V32, float* S32, int mode,
                      const int* run_if = nullptr) {
  const int n = P->cfg.n_aux, n_ov = P->n_ov;
  const int ldov = gw::tc_ld(n_ov);
  const bool three = P->cfg.op_parts >= 3;
  if (three) TRY(ensure_third_parts(P));
  __nv_bfloat16* vlo2 = three ? as<__nv_bfloat16>(P->mr_Vlo2) : nullptr;
  __nv_bfloat16* ulo2 = three ? as<__nv_bfloat16>(P->mr_Ulo2) : nullptr;
  CK(gw::tc_split_rows(V32, 2 * nr, n, n, as<__nv_bfloat16>(P->mr_Vhi), as<__nv_bfloat16>(P->mr_Vlo), P->stream,
                       vlo2));
  gw::TcEpi e1{};
  e1.kind = gw::TC_EPI_CPAIR;
  e1.Dk = P->d_D;
  e1.x = xf;
  e1.eta = (float)P->cfg.eta;
  e1.ohi = as<__nv_bfloat16>(P->mr_Uhi);
  e1.olo = as<__nv_bfloat16>(P->mr_Ulo);
  e1.olo2 = ulo2;
  e1.ldh = ldov;
  e1.run_if = run_if;
  const gw::TcOperand Vop{{as<__nv_bfloat16>(P->mr_Vhi), as<__nv_bfloat16>(P->mr_Vlo), vlo2}};
  const gw::TcOperand BT{{P->d_BThi, P->d_BTlo, three ? P->d_BTlo2 : nullptr}};
  const int ns = three ? 3 : 2;
  CK(gw::tc_gemm_ex(Vop, 1, BT, 0, ns, 2 * nr, n_ov, n, 0, e1, as<int>(P->tc_err), P->stream));
  gw::TcEpi e2{};
  e2.kind = mode == 0 ? gw::TC_EPI_STORE : gw::TC_EPI_EMBED;
  e2.out = S32;
  e2.ldo = n;
  e2.vin = V32;
  e2.ldv = n;
  e2.run_if = run_if;
  const gw::TcOperand Uop{{as<__nv_bfloat16>(P->mr_Uhi), as<__nv_bfloat16>(P->mr_Ulo), ulo2}};
  const gw::TcOperand Bop{{P->d_Bhi, P->d_Blo, three ? P->d_Blo2 : nullptr}};
  CK(gw::tc_gemm_ex(Uop, 1, Bop, 0, ns, 2 * nr, n, n_ov, 0, e2, as<int>(P->tc_err), P->stream));
  P->stats.n_kernel_launches += 3;
  return GW_OK;
}

// Three-part (about FP32-accurate) residue operator for the refinement of dense fallback solves: the embedding
// output S32 = [Re; Im]((1 - Pi(x)) z) for nf right-hand sides z held as (u, v) rows in V32.
gw_status tc_operator3(gw_plan* P, int nf, const double* xf, const float* V32, float* S32) {
  TRY(ensure_third_parts(P));
  const int n = P->cfg.n_aux, n_ov = P->n_ov;
  const size_t sv = 2 * (size_t)nf * gw::tc_ld(n), su = 2 * (size_t)nf * gw::tc_ld(n_ov);
  __nv_bfloat16* vp = as<__nv_bfloat16>(P->fb_Vp);
  __nv_bfloat16* up = as<__nv_bfloat16>(P->fb_Up);
  // tc_err is not reset here: the caller clears it before the blocked LU, whose bounded waits this check covers too
  CK(gw::tc_split_rows(V32, 2 * nf, n, n, vp, vp + sv, P->stream, vp + 2 * sv));
  gw::TcEpi e1{};
  e1.kind = gw::TC_EPI_CPAIR;
  e1.Dk = P->d_D;
  e1.x = xf;
  e1.eta = (float)P->cfg.eta;
  e1.ohi = up;
  e1.olo = up + su;
  e1.olo2 = up + 2 * su;
  e1.ldh = gw::tc_ld(n_ov);
  const gw::TcOperand Vop{{vp, vp + sv, vp + 2 * sv}};
  const gw::TcOperand BT{{P->d_BThi, P->d_BTlo, P->d_BTlo2}};
  CK(gw::tc_gemm_ex(Vop, 1, BT, 0, 3, 2 * nf, n_ov, n, 0, e1, as<int>(P->tc_err), P->stream));
  gw::TcEpi e2{};
  e2.kind = gw::TC_EPI_EMBED;
  e2.out = S32;
  e2.ldo = n;
  e2.vin = V32;
  e2.ldv = n;
  const gw::TcOperand Uop{{up, up + su, up + 2 * su}};
  const gw::TcOperand Bop{{P->d_Bhi, P->d_Blo, P->d_Blo2}};
  CK(gw::tc_gemm_ex(Uop, 1, Bop, 0, 3, 2 * nf, n, n_ov, 0, e2, as<int>(P->tc_err), P->stream));
  P->stats.n_kernel_launches += 3;
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, P->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
  CK(cudaStreamSynchronize(P->stream));
  if (herr != 0) return fail(P, GW_ERR_TIMEOUT, "tensor-core refinement operator: bounded wait ran out (code %d)", herr);
  return GW_OK;
}

// ---------------------------------------------------------------- batched residue solves
// Device arrays in: rt, rm (target index, state), xf (frequency); out: w_re, w_im, dw_re, iters, resnorm.
template <typename T>
gw_status residues_T(gw_plan* P, int nr_total, const int* d_rt, const int* d_rm, const double* d_xf, double* w_re,
                     double* w_im, double* dw_re, int* iters, double* resnorm, int* h_fallback) {
  const T* B = (sizeof(T) == 8) ? reinterpret_cast<const T*>(P->d_B_ia) : reinterpret_cast<const T*>(P->d_B_ia_f);
  const int n = P->cfg.n_aux, n_ov = P->n_ov;
  int batch = P->cfg.max_rhs_batch;
  if (batch <= 0) {
    // keep the U buffer (2 batch x n_ov) within ~4 GiB
    size_t cap = (ws_bytes(P) / 2) / ((size_t)2 * n_ov * sizeof(T));
    batch = (int)std::max<size_t>(1, std::min<size_t>(cap, 2048));
  }
  batch = std::min(batch, std::max(1, nr_total));
  TRY(ensure(P, P->mr_V, sizeof(T) * 2 * (size_t)batch * n));
  TRY(ensure(P, P->mr_S, sizeof(T) * 2 * (size_t)batch * n));
  TRY(ensure(P, P->mr_U, sizeof(T) * 2 * (size_t)batch * n_ov));
  const bool d64 = (sizeof(T) == 4) && P->cfg.deriv_fp64;
  if (sizeof(T) == 4) TRY(ensure(P, P->mr_V64, sizeof(double) * 2 * (size_t)batch * n));
  double* V64 = (sizeof(T) == 4) ? as<double>(P->mr_V64) : nullptr;
  for (DevBuf* b : {&P->mr_vprev, &P->mr_v, &P->mr_d1, &P->mr_d2, &P->mr_x})
    TRY(ensure(P, *b, sizeof(double) * 2 * (size_t)batch * n));
  TRY(ensure(P, P->mr_st, sizeof(MinresState) * batch));
  TRY(ensure(P, P->mr_cnt, sizeof(int)));
  const bool tcop = (sizeof(T) == 4) && P->d_BThi != nullptr;
  if (tcop) {
    TRY(ensure(P, P->mr_Vhi, sizeof(__nv_bfloat16) * 2 * (size_t)batch * gw::tc_ld(n)));
    TRY(ensure(P, P->mr_Vlo, sizeof(__nv_bfloat16) * 2 * (size_t)batch * gw::tc_ld(n)));
    TRY(ensure(P, P->mr_Uhi, sizeof(__nv_bfloat16) * 2 * (size_t)batch * gw::tc_ld(n_ov)));
    TRY(ensure(P, P->mr_Ulo, sizeof(__nv_bfloat16) * 2 * (size_t)batch * gw::tc_ld(n_ov)));
    if (P->cfg.op_parts >= 3) {
      TRY(ensure(P, P->mr_Vlo2, sizeof(__nv_bfloat16) * 2 * (size_t)batch * gw::tc_ld(n)));
      TRY(ensure(P, P->mr_Ulo2, sizeof(__nv_bfloat16) * 2 * (size_t)batch * gw::tc_ld(n_ov)));
    }
    TRY(ensure(P, P->tc_err, sizeof(int)));
    CK(cudaMemsetAsync(P->tc_err.p, 0, sizeof(int), P->stream));
  }
  const double eta = P->cfg.eta;
  std::vector<double> h_res;
  for (int j0 = 0; j0 < nr_total; j0 += batch) {
    const int nr = std::min(batch, nr_total - j0);
    const int* rt = d_rt + j0;
    const int* rm = d_rm + j0;
    const double* xf = d_xf + j0;
    LAUNCH(gw::launch_gather_rhs<T>(P->d_B_nm, P->n_bas, n, rt, rm, nr, as<T>(P->mr_V), P->stream));
    // rhs = Pi(x) b
    if (tcop) {
      TRY(tc_operator(P, nr, xf, reinterpret_cast<const float*>(P->mr_V.p), reinterpret_cast<float*>(P->mr_S.p), 0));
    } else {
      LAUNCH(gw::launch_op_gemm1<T>(as<T>(P->mr_V), B, P->d_D, P->n_ov, n, xf, eta, nr,
                                    as<T>(P->mr_U), 0, P->stream));
      LAUNCH(gw::launch_op_gemm2<T>(as<T>(P->mr_U), B, n, n_ov, nr, as<T>(P->mr_V), as<T>(P->mr_S), 0, P->stream));
    }
    LAUNCH(gw::launch_minres_init<T>(as<T>(P->mr_S), nr, n, as<double>(P->mr_vprev), as<double>(P->mr_v),
                                     as<double>(P->mr_d1), as<double>(P->mr_d2), as<double>(P->mr_x),
                                     as<MinresState>(P->mr_st), as<T>(P->mr_V), P->stream));
    const double op_flops = 2.0 * 2.0 * (2.0 * nr) * n * (double)n_ov;   // two GEMMs, 2nr columns each
    // The minres_maxit iterations (operator, then one MINRES step of every right-hand side) are captured as one
    // CUDA graph and launched without host synchronisation.  mr_cnt holds the number of right-hand sides still
    // active after the last step; once it is 0 the operator launches of the remaining iterations return at once
    // and the step kernel leaves every converged right-hand side frozen.
    int* cnt = as<int>(P->mr_cnt);
    CK(cudaMemcpyAsync(cnt, &nr, sizeof(int), cudaMemcpyHostToDevice, P->stream));
    if (P->cfg.minres_maxit > 0) {
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      CK(cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal));
      gw_status cap = GW_OK;
      for (int it = 0; it < P->cfg.minres_maxit && cap == GW_OK; ++it) {
        if (tcop) {
          cap = tc_operator(P, nr, xf, reinterpret_cast<const float*>(P->mr_V.p),
                            reinterpret_cast<float*>(P->mr_S.p), 1, cnt);
        } else {
          gw::launch_op_gemm1<T>(as<T>(P->mr_V), B, P->d_D, P->n_ov, n, xf, eta, nr,
                                 as<T>(P->mr_U), 0, P->stream, nullptr, 0.0, 0, cnt);
          gw::launch_op_gemm2<T>(as<T>(P->mr_U), B, n, n_ov, nr, as<T>(P->mr_V), as<T>(P->mr_S), 1, P->stream,
                                 cnt);
          P->stats.n_kernel_launches += 2;
        }
        if (cudaMemsetAsync(cnt, 0, sizeof(int), P->stream) != cudaSuccess) cap = GW_ERR_CUDA;
        gw::launch_minres_step<T>(as<T>(P->mr_S), nr, n, P->cfg.minres_tol, as<double>(P->mr_vprev),
                                  as<double>(P->mr_v), as<double>(P->mr_d1), as<double>(P->mr_d2),
                                  as<double>(P->mr_x), as<MinresState>(P->mr_st), as<T>(P->mr_V), cnt, P->stream);
        P->stats.n_kernel_launches++;
      }
      const cudaError_t ec = cudaStreamEndCapture(P->stream, &graph);
      if (cap != GW_OK) {
        if (graph) cudaGraphDestroy(graph);
        return cap == GW_ERR_CUDA ? fail(P, GW_ERR_CUDA, "MINRES graph capture failed") : cap;
      }
      CK(ec);
      const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      CK(ei);
      const size_t tg = tick(P);
      const cudaError_t el = cudaGraphLaunch(exec, P->stream);
      const size_t tg1 = tick(P);
      if (el != cudaSuccess) {
        cudaGraphExecDestroy(exec);
        CK(el);
      }
      CK(cudaStreamSynchronize(P->stream));
      cudaGraphExecDestroy(exec);
      P->stats.n_graph_launches++;
      // operator iterations that ran: the largest MINRES iteration count of the batch (states of converged
      // right-hand sides are frozen)
      std::vector<MinresState> hst(nr);
      CK(cudaMemcpy(hst.data(), P->mr_st.p, sizeof(MinresState) * nr, cudaMemcpyDeviceToHost));
      int ran = 0;
      for (const auto& x : hst) ran = std::max(ran, x.iters);
      if (tg != (size_t)-1 && tg1 != (size_t)-1) P->marks.push_back({4, tg, tg1, op_flops * ran});
      P->stats.launches_kernel[4] += ran;
    }
    if (tcop) {
      int herr = 0;
      CK(cudaMemcpyAsync(&herr, P->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
      CK(cudaStreamSynchronize(P->stream));
      if (herr != 0) return fail(P, GW_ERR_TIMEOUT, "tensor-core operator GEMM: bounded wait ran out (code %d)", herr);
    }
    LAUNCH(gw::launch_minres_finish<T>(P->d_B_nm, P->n_bas, n, rt, rm, nr, as<double>(P->mr_x),
                                       as<MinresState>(P->mr_st), w_re + j0, w_im + j0, iters + j0, resnorm + j0,
                                       as<T>(P->mr_V), P->stream, V64));
    // dense fallback for right-hand sides above the fallback threshold (Sec. 3.3, MINRES defaults paragraph)
    h_res.resize(nr);
    CK(cudaMemcpyAsync(h_res.data(), resnorm + j0, sizeof(double) * nr, cudaMemcpyDeviceToHost, P->stream));
    CK(cudaStreamSynchronize(P->stream));
    std::vector<int> need;
    for (int j = 0; j < nr; ++j) {
      bool bad = !(h_res[j] <= P->cfg.minres_fallback_tol);
      if (h_fallback) h_fallback[j0 + j] = bad ? 1 : 0;
      if (bad) need.push_back(j);
    }
    if (!need.empty()) TRY(dense_fallback<T>(P, need, rt, rm, xf, w_re + j0, w_im + j0, resnorm + j0));
    // dW/dx = y^T Pi'(x) y, reduced in FP64 inside the GEMM.  Mixed: the FP32 pass leaves out the pairs within
    // kResonantCut of resonance, where c'(x) reaches 2/eta^2 and FP32 rounding of t = B^T y would dominate dW;
    // those are added in FP64.
    CK(cudaMemsetAsync(dw_re + j0, 0, sizeof(double) * nr, P->stream));
    const size_t td = tick(P);
    if (d64) {
      LAUNCH(gw::launch_op_gemm1<double>(V64, P->d_B_ia, P->d_D, P->n_ov, n, xf, eta, nr,
                                         nullptr, 2, P->stream, dw_re + j0));
    } else if (sizeof(T) == 4) {
      LAUNCH(gw::launch_op_gemm1<T>(as<T>(P->mr_V), B, P->d_D, P->n_ov, n, xf, eta, nr,
                                    nullptr, 2, P->stream, dw_re + j0, kResonantCut, P->ld_f));
      LAUNCH(gw::launch_deriv_resonant(V64, P->d_B_ia, n_ov, n, P->d_Dsort, P->d_Dkidx, xf, nr, eta, kResonantCut,
                                       dw_re + j0, P->stream));
    } else {
      LAUNCH(gw::launch_op_gemm1<T>(as<T>(P->mr_V), B, P->d_D, P->n_ov, n, xf, eta, nr,
                                    nullptr, 2, P->stream, dw_re + j0));
    }
    mark(P, 4, td, 2.0 * (2.0 * nr) * n * (double)n_ov);
  }
  return GW_OK;
}

gw_status residues(gw_plan* P, int nr, const int* d_rt, const int* d_rm, const double* d_xf, double* w_re,
                   double* w_im, double* dw_re, int* iters, double* resnorm, int* h_fallback) {
  if (nr <= 0) return GW_OK;
  CK(cudaEventRecord(P->ev2, P->stream));
  gw_status st = (P->cfg.precision == GW_PREC_MIXED)
                     ? residues_T<float>(P, nr, d_rt, d_rm, d_xf, w_re, w_im, dw_re, iters, resnorm, h_fallback)
                     : residues_T<double>(P, nr, d_rt, d_rm, d_xf, w_re, w_im, dw_re, iters, resnorm, h_fallback);
  if (st != GW_OK) return st;
  CK(cudaEventRecord(P->ev1, P->stream));
  CK(cudaEventSynchronize(P->ev1));
  P->stats.ms_residues += now_ms(P, P->ev2, P->ev1);
  resolve_marks(P);
  P->stats.n_rhs_solved += nr;
  std::vector<int> it(nr);
  CK(cudaMemcpy(it.data(), iters, sizeof(int) * nr, cudaMemcpyDeviceToHost));
  for (int v : it) P->stats.n_minres_iters += v;
  return GW_OK;
}

// Residues of eq. "rnn" at omega_t for the active targets: (t, m, x = e_m - omega_t, coef = sign * theta).
// Evaluation points p (target tmap[p], or p without a map) at omega[p]; start[p] .. start[p + 1] are point p's
// entries.
void build_residue_list(gw_plan* P, const std::vector<double>& omega, const std::vector<unsigned char>& active,
                        std::vector<int>& rt, std::vector<int>& rm, std::vector<double>& xf,
                        std::vector<double>& coef, std::vector<int>& start, const std::vector<int>* tmap = nullptr) {
  rt.clear(); rm.clear(); xf.clear(); coef.clear();
  const int np = (int)omega.size();
  start.assign(np + 1, 0);
  for (int pt = 0; pt < np; ++pt) {
    start[pt] = (int)rt.size();
    if (!active[pt]) continue;
    const int t = tmap ? (*tmap)[pt] : pt;
    const int sp = P->h_spin[t];
    const double w = omega[pt];
    for (int m = 0; m < P->n_bas; ++m) {
      const double e = P->h_eps_g[sp][m];
      double th;
      double sg;
      if (m < P->occ_s[sp]) {
        th = (e > w) ? 1.0 : (e == w ? 0.5 : 0.0);
        sg = -1.0;
      } else {
        th = (w > e) ? 1.0 : (w == e ? 0.5 : 0.0);
        sg = 1.0;
      }
      if (th == 0.0) continue;
      rt.push_back(t);
      rm.push_back(m);
      xf.push_back(e - w);
      coef.push_back(sg * th);
    }
  }
  start[np] = (int)rt.size();
}

// Sigma_c = R - I (and derivative) at evaluation points p: target tmap[p] (p itself without a map) at omega[p],
// for the active points, into sg_R/sg_dR/sg_I/sg_dI [n points].  Every point's residues share one batched solve.
gw_status sigma_eval(gw_plan* P, const std::vector<double>& omega, const std::vector<unsigned char>& active,
                     int* n_fallback_out, const std::vector<int>* tmap = nullptr) {
  const int n_t = (int)omega.size();
  TRY(ensure(P, P->sg_I, sizeof(double) * n_t));
  TRY(ensure(P, P->sg_dI, sizeof(double) * n_t));
  TRY(ensure(P, P->sg_R, sizeof(double) * n_t));
  TRY(ensure(P, P->sg_dR, sizeof(double) * n_t));
  TRY(ensure(P, P->sg_om, sizeof(double) * n_t));
  TRY(ensure(P, P->sg_act, n_t));
  TRY(ensure(P, P->sg_start, sizeof(int) * (n_t + 1)));
  CK(cudaMemcpyAsync(P->sg_om.p, omega.data(), sizeof(double) * n_t, cudaMemcpyHostToDevice, P->stream));
  CK(cudaMemcpyAsync(P->sg_act.p, active.data(), n_t, cudaMemcpyHostToDevice, P->stream));
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  CK(cudaEventRecord(a, P->stream));
  const int* d_tmap = nullptr;
  if (tmap) {
    TRY(ensure(P, P->sg_tmap, sizeof(int) * n_t));
    CK(cudaMemcpyAsync(P->sg_tmap.p, tmap->data(), sizeof(int) * n_t, cudaMemcpyHostToDevice, P->stream));
    d_tmap = as<int>(P->sg_tmap);
  }
  LAUNCH(gw::launch_sigma_imag(P->d_W, n_t, P->n_bas, P->n_g, P->d_eps_g, P->d_xi, P->d_wt, as<double>(P->sg_om),
                               P->cfg.static_subtraction, as<double>(P->sg_I), as<double>(P->sg_dI),
                               as<unsigned char>(P->sg_act), P->stream, d_tmap, P->d_spin));
  CK(cudaEventRecord(b, P->stream));
  std::vector<int> rt, rm, start;
  std::vector<double> xf, coef;
  build_residue_list(P, omega, active, rt, rm, xf, coef, start, tmap);
  if (P->sh_world > 1) {
    // this rank's right-hand sides: entry j of the full list with j % world == rank (the per-target sums of R
    // and dR are then added across ranks)
    std::vector<int> rt2, rm2, start2(n_t + 1, 0);
    std::vector<double> xf2, coef2;
    for (int t = 0; t < n_t; ++t) {
      start2[t] = (int)rt2.size();
      for (int j = start[t]; j < start[t + 1]; ++j)
        if (j % P->sh_world == P->sh_rank) {
          rt2.push_back(rt[j]);
          rm2.push_back(rm[j]);
          xf2.push_back(xf[j]);
          coef2.push_back(coef[j]);
        }
    }
    start2[n_t] = (int)rt2.size();
    rt.swap(rt2); rm.swap(rm2); xf.swap(xf2); coef.swap(coef2); start.swap(start2);
  }
  const int nr = (int)rt.size();
  TRY(ensure(P, P->mr_rt, sizeof(int) * std::max(1, nr)));
  TRY(ensure(P, P->mr_rm, sizeof(int) * std::max(1, nr)));
  TRY(ensure(P, P->mr_xf, sizeof(double) * std::max(1, nr)));
  TRY(ensure(P, P->sg_coef, sizeof(double) * std::max(1, nr)));
  TRY(ensure(P, P->mr_wre, sizeof(double) * std::max(1, nr)));
  TRY(ensure(P, P->mr_wim, sizeof(double) * std::max(1, nr)));
  TRY(ensure(P, P->mr_dwre, sizeof(double) * std::max(1, nr)));
  TRY(ensure(P, P->mr_it, sizeof(int) * std::max(1, nr)));
  TRY(ensure(P, P->mr_res, sizeof(double) * std::max(1, nr)));
  if (nr > 0) {
    CK(cudaMemcpyAsync(P->mr_rt.p, rt.data(), sizeof(int) * nr, cudaMemcpyHostToDevice, P->stream));
    CK(cudaMemcpyAsync(P->mr_rm.p, rm.data(), sizeof(int) * nr, cudaMemcpyHostToDevice, P->stream));
    CK(cudaMemcpyAsync(P->mr_xf.p, xf.data(), sizeof(double) * nr, cudaMemcpyHostToDevice, P->stream));
    CK(cudaMemcpyAsync(P->sg_coef.p, coef.data(), sizeof(double) * nr, cudaMemcpyHostToDevice, P->stream));
  }
  CK(cudaMemcpyAsync(P->sg_start.p, start.data(), sizeof(int) * (n_t + 1), cudaMemcpyHostToDevice, P->stream));
  std::vector<int> fb(std::max(1, nr), 0);
  TRY(residues(P, nr, as<int>(P->mr_rt), as<int>(P->mr_rm), as<double>(P->mr_xf), as<double>(P->mr_wre),
               as<double>(P->mr_wim), as<double>(P->mr_dwre), as<int>(P->mr_it), as<double>(P->mr_res), fb.data()));
  LAUNCH(gw::launch_residue_reduce(as<int>(P->sg_start), n_t, as<double>(P->sg_coef), as<double>(P->mr_wre),
                                   as<double>(P->mr_dwre), as<double>(P->sg_R), as<double>(P->sg_dR), P->stream));
  if (P->sh_world > 1) {
    // R and dR of every target summed over the ranks' residue subsets (the I term is computed on every rank)
    P->sh_buf.resize(2 * (size_t)n_t);
    CK(cudaMemcpyAsync(P->sh_buf.data(), P->sg_R.p, sizeof(double) * n_t, cudaMemcpyDeviceToHost, P->stream));
    CK(cudaMemcpyAsync(P->sh_buf.data() + n_t, P->sg_dR.p, sizeof(double) * n_t, cudaMemcpyDeviceToHost,
                       P->stream));
    CK(cudaStreamSynchronize(P->stream));
    if (P->sh_reduce(P->sh_buf.data(), 2LL * n_t, P->sh_ctx) != 0)
      return fail(P, GW_ERR_CUDA, "shard all-reduce of the residue terms failed");
    CK(cudaMemcpyAsync(P->sg_R.p, P->sh_buf.data(), sizeof(double) * n_t, cudaMemcpyHostToDevice, P->stream));
    CK(cudaMemcpyAsync(P->sg_dR.p, P->sh_buf.data() + n_t, sizeof(double) * n_t, cudaMemcpyHostToDevice,
                       P->stream));
  }
  CK(cudaStreamSynchronize(P->stream));
  P->stats.ms_sigma_imag += now_ms(P, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  int nf = 0;
  for (int j = 0; j < nr; ++j) nf += fb[j];
  if (n_fallback_out) *n_fallback_out = nf;
  for (int t = 0; t < n_t; ++t) P->stats.n_sigma_evals += active[t] ? 1 : 0;
  return GW_OK;
}

// Pair-energy table D [n_ov] (the columns of B_ia) on the device; in mixed precision also its ascending order with
// the pair index of each entry (for the resonance windows of the derivative pass) and its minimum.
gw_status set_pair_table(gw_plan* P, const std::vector<double>& D) {
  CK(cudaMemcpyAsync(P->d_D, D.data(), sizeof(double) * P->n_ov, cudaMemcpyHostToDevice, P->stream));
  double dmin = D.empty() ? 0.0 : D[0];
  for (double v : D) dmin = std::min(dmin, v);
  P->D_min = dmin;
  if (P->d_Dsort) {
    std::vector<int> order((size_t)P->n_ov);
    for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return D[a] < D[b]; });
    std::vector<double> Ds(order.size());
    for (size_t k = 0; k < order.size(); ++k) Ds[k] = D[order[k]];
    CK(cudaMemcpyAsync(P->d_Dsort, Ds.data(), sizeof(double) * P->n_ov, cudaMemcpyHostToDevice, P->stream));
    CK(cudaMemcpyAsync(P->d_Dkidx, order.data(), sizeof(int) * P->n_ov, cudaMemcpyHostToDevice, P->stream));
    CK(cudaStreamSynchronize(P->stream));
  }
  CK(cudaStreamSynchronize(P->stream));
  return GW_OK;
}

// W's energies: d_eps, the pair energies D_ia = e_a - e_i (ia = i n_virt + a) and, in mixed precision, their
// ascending order and the smallest one.
gw_status set_pair_energies(gw_plan* P, const double* eps, const double* eps_b = nullptr) {
  CK(cudaMemcpyAsync(P->d_eps, eps, sizeof(double) * P->n_bas, cudaMemcpyHostToDevice, P->stream));
  std::vector<double> D;
  D.reserve((size_t)P->n_ov);
  for (int sp = 0; sp < P->n_spin; ++sp) {      // spin blocks side by side: the columns of the (open-shell) B_ia
    const double* e = sp == 0 ? eps : eps_b;
    const int n_occ = P->occ_s[sp], n_virt = P->n_bas - n_occ;
    for (int i = 0; i < n_occ; ++i)
      for (int a = 0; a < n_virt; ++a) D.push_back(e[n_occ + a] - e[i]);
  }
  P->sd_done = false;             // the Casida poles follow W's energies
  return set_pair_table(P, D);
}

// G's energies (host copy for the residue list, device copy for the I term).
gw_status set_g_energies(gw_plan* P, int spin, const double* eps) {
  P->h_eps_g[spin].assign(eps, eps + P->n_bas);
  CK(cudaMemcpyAsync(P->d_eps_g + (size_t)spin * P->n_bas, eps, sizeof(double) * P->n_bas, cudaMemcpyHostToDevice,
                     P->stream));
  CK(cudaStreamSynchronize(P->stream));
  return GW_OK;
}

__global__ void convert_f64_f32_kernel(const double* __restrict__ a, float* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

__global__ void scale_kernel(double* __restrict__ a, size_t n, double f) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) a[i] *= f;
}

// rows x cols FP64 (contiguous) to FP32 rows of ldb elements, zero padded.
__global__ void convert_rows_kernel(const double* __restrict__ a, int rows, int cols, float* __restrict__ b,
                                    long ldb) {
  for (int r = blockIdx.y; r < rows; r += gridDim.y)
    for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < ldb; c += (long)gridDim.x * blockDim.x)
      b[(long)r * ldb + c] = c < cols ? (float)a[(long)r * cols + c] : 0.f;
}

// Third BF16 parts of B_ia and B_ia^T, made when a three-part operator first needs them (the hi and lo parts are
// rewritten with the same values).
gw_status ensure_third_parts(gw_plan* P) {
  if (P->d_Blo2) return GW_OK;
  const int n = P->cfg.n_aux;
  TRY(dmalloc(P, &P->d_Blo2, sizeof(__nv_bfloat16) * (size_t)n * gw::tc_ld(P->n_ov)));
  TRY(dmalloc(P, &P->d_BTlo2, sizeof(__nv_bfloat16) * (size_t)P->n_ov * gw::tc_ld(n)));
  CK(gw::tc_split_rows(P->d_B_ia_f, n, P->n_ov, (int)P->ld_f, P->d_Bhi, P->d_Blo, P->stream, P->d_Blo2));
  CK(gw::tc_transpose_split(P->d_B_ia_f, n, P->n_ov, P->d_BThi, P->d_BTlo, P->stream, P->d_BTlo2, P->ld_f));
  P->stats.n_kernel_launches += 2;
  return GW_OK;
}

}  // namespace

// ==================================================================== C ABI
extern "C" {

void gw_config_default(gw_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->n_freq = 128;
  c->x0 = 0.5;
  c->eta = 1e-3;
  c->precision = GW_PREC_FP64;
  c->minres_maxit = 25;
  c->minres_tol = 5e-5;
  c->minres_fallback_tol = 1e-4;
  c->qp_maxit = 50;
  c->qp_tol = 1e-8;
  c->static_subtraction = 1;
  c->max_rhs_batch = 0;
  c->refine_tol = 1e-6;
  c->op_parts = 2;
  c->refine_df = 1;
  c->qp_window = 0.5;
  c->qp_window_points = 64;
}

static void free_plan(gw_plan* P) {
  if (!P) return;
  if (P->stream) cudaStreamSynchronize(P->stream);
  for (DevBuf* b : P->bufs)
    if (b->p) cudaFree(b->p);
  double* owned[] = {P->d_eps, P->d_eps_g, P->d_xi, P->d_wt, P->d_sx, P->d_shift, P->d_en, P->d_W};
  if (P->d_spin) cudaFree(P->d_spin);
  if (P->d_occ_t) cudaFree(P->d_occ_t);
  for (double* p : owned)
    if (p) cudaFree(p);
  if (P->own_B) {
    if (P->d_B_ia) cudaFree(P->d_B_ia);
    if (P->d_B_nm) cudaFree(P->d_B_nm);
  }
  if (P->d_B_ia_f) cudaFree(P->d_B_ia_f);
  if (P->d_B_nm_f) cudaFree(P->d_B_nm_f);
  if (P->d_Bhi) cudaFree(P->d_Bhi);
  if (P->d_Blo) cudaFree(P->d_Blo);
  if (P->d_BThi) cudaFree(P->d_BThi);
  if (P->d_BTlo) cudaFree(P->d_BTlo);
  if (P->d_Blo2) cudaFree(P->d_Blo2);
  if (P->d_Bp_hi) cudaFree(P->d_Bp_hi);
  if (P->d_Bp_lo) cudaFree(P->d_Bp_lo);
  if (P->d_BTlo2) cudaFree(P->d_BTlo2);
  if (P->d_D) cudaFree(P->d_D);
  if (P->d_Dsort) cudaFree(P->d_Dsort);
  if (P->d_Dkidx) cudaFree(P->d_Dkidx);
  if (P->d_Bnhi) cudaFree(P->d_Bnhi);
  if (P->d_Bnlo) cudaFree(P->d_Bnlo);
  if (P->d_Bnlo2) cudaFree(P->d_Bnlo2);
  if (P->h_cnt) cudaFreeHost(P->h_cnt);
  if (P->ev0) cudaEventDestroy(P->ev0);
  if (P->ev1) cudaEventDestroy(P->ev1);
  if (P->ev2) cudaEventDestroy(P->ev2);
  for (cudaEvent_t e : P->tpool) cudaEventDestroy(e);
  if (P->own_stream && P->stream) cudaStreamDestroy(P->stream);
  delete P;
}

// Open-shell inputs of gw_plan_create_uks: the beta channel (its energies, occupations and B_ia block) and the
// spin of every target; the alpha channel comes through the closed-shell arguments.
struct UksInput {
  const double* eps_b;
  int n_occ_b;
  const double* B_ia_b;
  const int* spins;
};

static gw_status plan_create_impl(gw_plan* P, const gw_config* cfg, const double* eps, const double* B_ia,
                                  const double* B_nm, const int* targets, int n_targets, const double* vxc,
                                  const double* xi, const double* wt, unsigned flags, void* stream,
                                  const UksInput* uks = nullptr) {
  P->cfg = *cfg;
  P->flags = flags;
  P->n_bas = cfg->n_occ + cfg->n_virt;
  P->n_spin = uks ? 2 : 1;
  P->occ_s[0] = cfg->n_occ;
  P->occ_s[1] = uks ? uks->n_occ_b : cfg->n_occ;
  const long n_ov_a = (long)cfg->n_occ * cfg->n_virt;
  const long n_ov_b = uks ? (long)uks->n_occ_b * (P->n_bas - uks->n_occ_b) : 0;
  P->n_ov = (int)(n_ov_a + n_ov_b);
  P->n_t = n_targets;
  P->n_g = cfg->n_freq;
  if (stream) {
    P->stream = (cudaStream_t)stream;
  } else {
    CK(cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking));
    P->own_stream = true;
  }
  CK(cudaEventCreate(&P->ev0));
  CK(cudaEventCreate(&P->ev1));
  CK(cudaEventCreate(&P->ev2));
  CK(cudaMallocHost(&P->h_cnt, sizeof(int)));
  const int n = cfg->n_aux;
  P->h_eps.assign(eps, eps + P->n_bas);
  P->h_eps_s[0] = P->h_eps;
  P->h_eps_s[1] = uks ? std::vector<double>(uks->eps_b, uks->eps_b + P->n_bas) : P->h_eps;
  P->h_eps_g[0] = P->h_eps_s[0];
  P->h_eps_g[1] = P->h_eps_s[1];
  P->h_targets.assign(targets, targets + n_targets);
  P->h_spin.assign(n_targets, 0);
  if (uks)
    for (int t = 0; t < n_targets; ++t) P->h_spin[t] = uks->spins[t];
  // grid
  P->h_xi.resize(P->n_g);
  P->h_wt.resize(P->n_g);
  if (xi && wt) {
    for (int g = 0; g < P->n_g; ++g) { P->h_xi[g] = xi[g]; P->h_wt[g] = wt[g]; }
  } else {
    gw_grid(P->n_g, cfg->x0, P->h_xi.data(), P->h_wt.data());
  }
  std::vector<double> xi_all(P->h_xi);
  xi_all.push_back(0.0);
  TRY(dmalloc(P, &P->d_eps, sizeof(double) * P->n_bas));
  TRY(dmalloc(P, &P->d_eps_g, sizeof(double) * P->n_spin * P->n_bas));
  TRY(dmalloc(P, &P->d_xi, sizeof(double) * (P->n_g + 1)));
  TRY(dmalloc(P, &P->d_wt, sizeof(double) * std::max(1, P->n_g)));
  TRY(dmalloc(P, &P->d_sx, sizeof(double) * std::max(1, n_targets)));
  TRY(dmalloc(P, &P->d_shift, sizeof(double) * std::max(1, n_targets)));
  TRY(dmalloc(P, &P->d_en, sizeof(double) * std::max(1, n_targets)));
  TRY(dmalloc(P, &P->d_W, sizeof(double) * (size_t)n_targets * P->n_bas * (P->n_g + 1)));
  TRY(dmalloc(P, &P->d_D, sizeof(double) * (size_t)P->n_ov));
  for (int sp = 0; sp < P->n_spin; ++sp) TRY(set_g_energies(P, sp, P->h_eps_s[sp].data()));
  CK(cudaMemcpyAsync(P->d_xi, xi_all.data(), sizeof(double) * (P->n_g + 1), cudaMemcpyHostToDevice, P->stream));
  CK(cudaMemcpyAsync(P->d_wt, P->h_wt.data(), sizeof(double) * P->n_g, cudaMemcpyHostToDevice, P->stream));
  if (uks) {
    std::vector<int> occ_t(n_targets);
    for (int t = 0; t < n_targets; ++t) occ_t[t] = P->occ_s[P->h_spin[t]];
    TRY(dmalloc(P, &P->d_spin, sizeof(int) * n_targets));
    TRY(dmalloc(P, &P->d_occ_t, sizeof(int) * n_targets));
    CK(cudaMemcpyAsync(P->d_spin, P->h_spin.data(), sizeof(int) * n_targets, cudaMemcpyHostToDevice, P->stream));
    CK(cudaMemcpyAsync(P->d_occ_t, occ_t.data(), sizeof(int) * n_targets, cudaMemcpyHostToDevice, P->stream));
    CK(cudaStreamSynchronize(P->stream));
  }
  const size_t nB = (size_t)n * P->n_ov, nBn = (size_t)n_targets * P->n_bas * n;
  cudaMemcpyKind kind = (flags & GW_INPUT_ON_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (uks) {
    // the two spin channels side by side along the pair axis, each scaled by 1/sqrt(2): the closed-shell formulas
    // (factor 2 for the two spins) then give sum over sigma with factor 1 per channel (Sec. 3.3, Pi with Sigma_s)
    P->own_B = true;
    TRY(dmalloc(P, &P->d_B_ia, sizeof(double) * nB));
    TRY(dmalloc(P, &P->d_B_nm, sizeof(double) * nBn));
    CK(cudaMemcpy2DAsync(P->d_B_ia, sizeof(double) * P->n_ov, B_ia, sizeof(double) * n_ov_a, sizeof(double) * n_ov_a,
                         n, kind, P->stream));
    if (n_ov_b > 0)
      CK(cudaMemcpy2DAsync(P->d_B_ia + n_ov_a, sizeof(double) * P->n_ov, uks->B_ia_b, sizeof(double) * n_ov_b,
                           sizeof(double) * n_ov_b, n, kind, P->stream));
    LAUNCH((scale_kernel<<<1024, 256, 0, P->stream>>>(P->d_B_ia, nB, 0.70710678118654752440)));
    CK(cudaMemcpyAsync(P->d_B_nm, B_nm, sizeof(double) * nBn, kind, P->stream));
  } else if (flags & GW_BORROW_DEVICE_PTRS) {
    P->own_B = false;
    P->d_B_ia = const_cast<double*>(B_ia);
    P->d_B_nm = const_cast<double*>(B_nm);
  } else {
    P->own_B = true;
    TRY(dmalloc(P, &P->d_B_ia, sizeof(double) * nB));
    TRY(dmalloc(P, &P->d_B_nm, sizeof(double) * nBn));
    CK(cudaMemcpyAsync(P->d_B_ia, B_ia, sizeof(double) * nB, kind, P->stream));
    CK(cudaMemcpyAsync(P->d_B_nm, B_nm, sizeof(double) * nBn, kind, P->stream));
  }
  if (cfg->precision == GW_PREC_MIXED) {
    // FP32 B_ia with rows padded to 16 bytes (the fused Pi kernel reads it by TMA)
    P->ld_f = gw::pf_ldw(P->n_ov);
    TRY(dmalloc(P, &P->d_B_ia_f, sizeof(float) * (size_t)n * P->ld_f));
    TRY(dmalloc(P, &P->d_B_nm_f, sizeof(float) * nBn));
    LAUNCH((convert_rows_kernel<<<dim3(64, std::min(n, 65535)), 256, 0, P->stream>>>(P->d_B_ia, n, P->n_ov,
                                                                                   P->d_B_ia_f, P->ld_f)));
    LAUNCH((convert_f64_f32_kernel<<<1024, 256, 0, P->stream>>>(P->d_B_nm, P->d_B_nm_f, nBn)));
    const size_t nsplit = (size_t)n * gw::tc_ld(P->n_ov);
    TRY(dmalloc(P, &P->d_Bhi, sizeof(__nv_bfloat16) * nsplit));
    TRY(dmalloc(P, &P->d_Blo, sizeof(__nv_bfloat16) * nsplit));
    CK(gw::tc_split_rows(P->d_B_ia_f, n, P->n_ov, (int)P->ld_f, P->d_Bhi, P->d_Blo, P->stream));
    const size_t npanel = (size_t)n * gw::tc_pi_panel_cols(P->n_ov);
    TRY(dmalloc(P, &P->d_Bp_hi, sizeof(__nv_bfloat16) * npanel));
    TRY(dmalloc(P, &P->d_Bp_lo, sizeof(__nv_bfloat16) * npanel));
    CK(gw::tc_pi_panel_split(P->d_B_ia_f, P->ld_f, n, P->n_ov, P->d_Bp_hi, P->d_Bp_lo, P->stream));
    const size_t nsplitN = (size_t)n_targets * P->n_bas * gw::tc_ld(n);
    TRY(dmalloc(P, &P->d_Bnhi, sizeof(__nv_bfloat16) * nsplitN));
    TRY(dmalloc(P, &P->d_Bnlo, sizeof(__nv_bfloat16) * nsplitN));
    TRY(dmalloc(P, &P->d_Bnlo2, sizeof(__nv_bfloat16) * nsplitN));
    CK(gw::tc_split_rows(P->d_B_nm_f, n_targets * P->n_bas, n, n, P->d_Bnhi, P->d_Bnlo, P->stream, P->d_Bnlo2));
    const size_t nsplitT = (size_t)P->n_ov * gw::tc_ld(n);
    TRY(dmalloc(P, &P->d_BThi, sizeof(__nv_bfloat16) * nsplitT));
    TRY(dmalloc(P, &P->d_BTlo, sizeof(__nv_bfloat16) * nsplitT));
    CK(gw::tc_transpose_split(P->d_B_ia_f, n, P->n_ov, P->d_BThi, P->d_BTlo, P->stream, nullptr, P->ld_f));
    TRY(dmalloc(P, &P->d_Dsort, sizeof(double) * P->n_ov));
    TRY(dmalloc(P, &P->d_Dkidx, sizeof(int) * P->n_ov));
    CK(cudaStreamSynchronize(P->stream));
  }
  TRY(set_pair_energies(P, P->h_eps_s[0].data(), P->h_eps_s[1].data()));
  LAUNCH(gw::launch_sigma_x(P->d_B_nm, n_targets, P->n_bas, n, cfg->n_occ, P->d_sx, P->stream, P->d_occ_t));
  P->h_sx.resize(n_targets);
  CK(cudaMemcpyAsync(P->h_sx.data(), P->d_sx, sizeof(double) * n_targets, cudaMemcpyDeviceToHost, P->stream));
  CK(cudaStreamSynchronize(P->stream));
  P->h_shift.resize(n_targets);
  P->h_en.resize(n_targets);
  for (int t = 0; t < n_targets; ++t) {
    P->h_shift[t] = vxc ? P->h_sx[t] - vxc[t] : 0.0;
    P->h_en[t] = P->h_eps_s[P->h_spin[t]][targets[t]];
  }
  CK(cudaMemcpyAsync(P->d_shift, P->h_shift.data(), sizeof(double) * n_targets, cudaMemcpyHostToDevice, P->stream));
  CK(cudaMemcpyAsync(P->d_en, P->h_en.data(), sizeof(double) * n_targets, cudaMemcpyHostToDevice, P->stream));
  CK(cudaStreamSynchronize(P->stream));
  return GW_OK;
}

gw_status gw_plan_create(const gw_config* cfg, const double* eps, const double* B_ia, const double* B_nm,
                         const int* targets, int n_targets, const double* vxc, const double* xi, const double* wt,
                         unsigned flags, void* stream, gw_plan_t* out) {
  gw_plan* P = nullptr;
  if (!out) return fail(nullptr, GW_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!cfg || !eps || !B_ia || !B_nm || !targets) return fail(nullptr, GW_ERR_ARG, "NULL input pointer");
  if (cfg->n_occ <= 0 || cfg->n_virt <= 0 || cfg->n_aux <= 0 || n_targets <= 0 || cfg->n_freq <= 0)
    return fail(nullptr, GW_ERR_ARG, "sizes must be positive (n_occ %d n_virt %d n_aux %d n_targets %d n_freq %d)",
                cfg->n_occ, cfg->n_virt, cfg->n_aux, n_targets, cfg->n_freq);
  if ((long)cfg->n_occ * cfg->n_virt > 2147483647L) return fail(nullptr, GW_ERR_ARG, "n_occ*n_virt too large");
  if (cfg->precision != GW_PREC_FP64 && cfg->precision != GW_PREC_MIXED)
    return fail(nullptr, GW_ERR_ARG, "unknown precision %d", cfg->precision);
  if ((xi == nullptr) != (wt == nullptr)) return fail(nullptr, GW_ERR_ARG, "xi and wt must both be given or both NULL");
  if (!(cfg->x0 > 0.0) && !xi) return fail(nullptr, GW_ERR_ARG, "x0 must be positive");
  if (!(cfg->eta >= 0.0)) return fail(nullptr, GW_ERR_ARG, "eta must be >= 0");
  if (cfg->minres_maxit < 0 || cfg->qp_maxit <= 0) return fail(nullptr, GW_ERR_ARG, "bad iteration caps");
  if (cfg->tc_max_ctas < 0) return fail(nullptr, GW_ERR_ARG, "tc_max_ctas must be >= 0");
  if (!(cfg->qp_window > 0.0) || cfg->qp_window_points < 2 || !(cfg->qp_cluster_gap >= 0.0))
    return fail(nullptr, GW_ERR_ARG, "bad graphical window (%g Ha, %d points) or cluster gap %g", cfg->qp_window,
                cfg->qp_window_points, cfg->qp_cluster_gap);
  if (cfg->pi_ksplit != 0 && cfg->pi_ksplit != 1 && cfg->pi_ksplit != 2 && cfg->pi_ksplit != 4 && cfg->pi_ksplit != 8)
    return fail(nullptr, GW_ERR_ARG, "pi_ksplit must be 0 (autotune), 1, 2, 4 or 8 (got %d)", cfg->pi_ksplit);
  if (cfg->op_parts != 2 && cfg->op_parts != 3)
    return fail(nullptr, GW_ERR_ARG, "op_parts must be 2 or 3 (got %d)", cfg->op_parts);
  const int n_bas = cfg->n_occ + cfg->n_virt;
  for (int i = 0; i < n_bas; ++i) {
    if (!std::isfinite(eps[i])) return fail(nullptr, GW_ERR_ARG, "eps[%d] is not finite", i);
    if (i > 0 && eps[i] < eps[i - 1]) return fail(nullptr, GW_ERR_ARG, "eps must be ascending (index %d)", i);
  }
  if (eps[cfg->n_occ] <= eps[cfg->n_occ - 1]) return fail(nullptr, GW_ERR_ARG, "no gap between HOMO and LUMO");
  for (int t = 0; t < n_targets; ++t)
    if (targets[t] < 0 || targets[t] >= n_bas) return fail(nullptr, GW_ERR_ARG, "target %d out of range", targets[t]);
  if ((flags & GW_BORROW_DEVICE_PTRS) && cfg->precision == GW_PREC_MIXED) {
    // the FP32 copies are made from the borrowed FP64 arrays; fine
  }
  P = new (std::nothrow) gw_plan();
  if (!P) return fail(nullptr, GW_ERR_OOM, "host allocation failed");
  gw_status st = plan_create_impl(P, cfg, eps, B_ia, B_nm, targets, n_targets, vxc, xi, wt, flags, stream);
  if (st != GW_OK) {
    g_create_error = P->err;
    free_plan(P);
    return st;
  }
  *out = P;
  return GW_OK;
}

gw_status gw_plan_create_uks(const gw_config* cfg, const double* eps_a, const double* eps_b, int n_occ_b,
                             const double* B_ia_a, const double* B_ia_b, const double* B_nm, const int* targets,
                             const int* spins, int n_targets, const double* vxc, const double* xi, const double* wt,
                             unsigned flags, void* stream, gw_plan_t* out) {
  if (!out) return fail(nullptr, GW_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!cfg || !eps_a || !eps_b || !B_ia_a || !B_nm || !targets || !spins)
    return fail(nullptr, GW_ERR_ARG, "NULL input pointer");
  if (flags & GW_BORROW_DEVICE_PTRS) return fail(nullptr, GW_ERR_ARG, "open shell: B cannot be borrowed");
  const int n_bas = cfg->n_occ + cfg->n_virt;
  if (cfg->n_occ <= 0 || cfg->n_virt <= 0 || n_occ_b < 0 || n_occ_b >= n_bas || cfg->n_aux <= 0 || n_targets <= 0 ||
      cfg->n_freq <= 0)
    return fail(nullptr, GW_ERR_ARG, "bad sizes (n_occ %d/%d n_bas %d n_aux %d n_targets %d)", cfg->n_occ, n_occ_b,
                n_bas, cfg->n_aux, n_targets);
  if (n_occ_b > 0 && !B_ia_b) return fail(nullptr, GW_ERR_ARG, "B_ia_b is NULL");
  if ((long)cfg->n_occ * cfg->n_virt + (long)n_occ_b * (n_bas - n_occ_b) > 2147483647L)
    return fail(nullptr, GW_ERR_ARG, "too many pairs");
  if (cfg->precision != GW_PREC_FP64 && cfg->precision != GW_PREC_MIXED)
    return fail(nullptr, GW_ERR_ARG, "unknown precision %d", cfg->precision);
  if ((xi == nullptr) != (wt == nullptr)) return fail(nullptr, GW_ERR_ARG, "xi and wt must both be given or both NULL");
  if (!(cfg->x0 > 0.0) && !xi) return fail(nullptr, GW_ERR_ARG, "x0 must be positive");
  if (!(cfg->eta >= 0.0) || cfg->minres_maxit < 0 || cfg->qp_maxit <= 0 || (cfg->op_parts != 2 && cfg->op_parts != 3))
    return fail(nullptr, GW_ERR_ARG, "bad solver settings");
  const double* e2[2] = {eps_a, eps_b};
  const int occ[2] = {cfg->n_occ, n_occ_b};
  for (int sp = 0; sp < 2; ++sp) {
    for (int i = 0; i < n_bas; ++i) {
      if (!std::isfinite(e2[sp][i])) return fail(nullptr, GW_ERR_ARG, "spin %d: eps[%d] is not finite", sp, i);
      if (i > 0 && e2[sp][i] < e2[sp][i - 1]) return fail(nullptr, GW_ERR_ARG, "spin %d: eps not ascending", sp);
    }
    if (occ[sp] > 0 && e2[sp][occ[sp]] <= e2[sp][occ[sp] - 1])
      return fail(nullptr, GW_ERR_ARG, "spin %d: no gap between HOMO and LUMO", sp);
  }
  for (int t = 0; t < n_targets; ++t) {
    if (targets[t] < 0 || targets[t] >= n_bas) return fail(nullptr, GW_ERR_ARG, "target %d out of range", targets[t]);
    if (spins[t] != 0 && spins[t] != 1) return fail(nullptr, GW_ERR_ARG, "spin of target %d must be 0 or 1", t);
  }
  gw_plan* P = new (std::nothrow) gw_plan();
  if (!P) return fail(nullptr, GW_ERR_OOM, "host allocation failed");
  const UksInput uks{eps_b, n_occ_b, B_ia_b, spins};
  gw_status st = plan_create_impl(P, cfg, eps_a, B_ia_a, B_nm, targets, n_targets, vxc, xi, wt, flags, stream, &uks);
  if (st != GW_OK) {
    g_create_error = P->err;
    free_plan(P);
    return st;
  }
  *out = P;
  return GW_OK;
}

gw_status gw_polarizability(gw_plan_t P, const double* xi, int n_xi, double* pi_out) {
  if (!P) return GW_ERR_ARG;
  if (!xi) {
    if (pi_out) return fail(P, GW_ERR_ARG, "pi_out must be NULL when building the plan grid");
    P->screening_done = false;    // explicit request: rebuild the table
    return ensure_screening(P);
  }
  if (n_xi <= 0) return fail(P, GW_ERR_ARG, "n_xi must be positive");
  const int n = P->cfg.n_aux;
  DevBuf& dxi = P->ws_xi;
  gw_status st = ensure(P, dxi, sizeof(double) * n_xi);
  if (st != GW_OK) return st;
  CK(cudaMemcpyAsync(dxi.p, xi, sizeof(double) * n_xi, cudaMemcpyHostToDevice, P->stream));
  CK(cudaEventRecord(P->ev0, P->stream));
  if (P->cfg.precision == GW_PREC_MIXED) {
    TRY(ensure(P, P->ws_mat, sizeof(float) * (size_t)n * n * n_xi));
    std::vector<int> kinds(n_xi, 0);
    TRY(tc_weighted_syrk(P, kinds.data(), xi, n_xi, 0, 0, as<float>(P->ws_mat), 0));
    CK(cudaEventRecord(P->ev1, P->stream));
    if (pi_out) {
      std::vector<float> h((size_t)n * n * n_xi);
      CK(cudaMemcpyAsync(h.data(), P->ws_mat.p, sizeof(float) * h.size(), cudaMemcpyDeviceToHost, P->stream));
      CK(cudaStreamSynchronize(P->stream));
      for (size_t i = 0; i < h.size(); ++i) pi_out[i] = h[i];
    }
  } else {
    TRY(ensure(P, P->ws_mat, sizeof(double) * (size_t)n * n * n_xi));
    LAUNCH(gw::launch_pi_syrk<double>(P->d_B_ia, P->d_D, P->n_ov, n, as<double>(dxi), n_xi,
                                      as<double>(P->ws_mat), 0, P->stream));
    CK(cudaEventRecord(P->ev1, P->stream));
    if (pi_out)
      CK(cudaMemcpyAsync(pi_out, P->ws_mat.p, sizeof(double) * (size_t)n * n * n_xi, cudaMemcpyDeviceToHost,
                         P->stream));
  }
  CK(cudaStreamSynchronize(P->stream));
  P->stats.ms_pi = now_ms(P, P->ev0, P->ev1);
  resolve_marks(P);
  return GW_OK;
}

gw_status gw_sigma_cd(gw_plan_t P, const double* omega, double* sigma_c, double* dsigma_c, double* sigma_x) {
  if (!P || !omega) return P ? fail(P, GW_ERR_ARG, "omega is NULL") : GW_ERR_ARG;
  TRY(ensure_screening(P));
  const int n_t = P->n_t;
  std::vector<double> om(omega, omega + n_t);
  std::vector<unsigned char> act(n_t, 1);
  int nf = 0;
  TRY(sigma_eval(P, om, act, &nf));
  std::vector<double> R(n_t), dR(n_t), I(n_t), dI(n_t);
  CK(cudaMemcpy(R.data(), P->sg_R.p, sizeof(double) * n_t, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(dR.data(), P->sg_dR.p, sizeof(double) * n_t, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(I.data(), P->sg_I.p, sizeof(double) * n_t, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(dI.data(), P->sg_dI.p, sizeof(double) * n_t, cudaMemcpyDeviceToHost));
  for (int t = 0; t < n_t; ++t) {
    if (sigma_c) sigma_c[t] = R[t] - I[t];
    if (dsigma_c) dsigma_c[t] = dR[t] - dI[t];
    if (sigma_x) sigma_x[t] = P->h_sx[t];
  }
  return GW_OK;
}

// Spectral decomposition (Sec. 2.2, 3.2): the Hermitian Casida matrix M = D^1/2 (D + 4K) D^1/2 (K = B^T B over the
// pairs of every spin channel side by side; an open-shell plan stores each channel scaled by 1/sqrt 2, which turns
// the factor 4 into the 2 of each spin block) diagonalised by cyclic Jacobi sweeps in FP64 until the off-diagonal
// Frobenius norm is below 1e-13 of the diagonal one, then Omega_s and the pole weights of every (target, state).
constexpr long kSdMaxPairs = 16384;       // O(N_ov^3) work and 2 N_ov^2 doubles of storage
gw_status ensure_sd(gw_plan* P) {
  if (P->sd_done) return GW_OK;
  const long N = P->n_ov;
  if (N > kSdMaxPairs)
    return fail(P, GW_ERR_ARG, "spectral decomposition needs N_ov <= %ld (got %ld): O(N_ov^3)", kSdMaxPairs, N);
  const int n = P->cfg.n_aux, Np = (int)(N + (N & 1));
  TRY(ensure(P, P->sd_M, sizeof(double) * (size_t)Np * Np));
  TRY(ensure(P, P->sd_T, sizeof(double) * (size_t)Np * Np));
  TRY(ensure(P, P->sd_cs, sizeof(double) * (size_t)Np));
  TRY(ensure(P, P->sd_off, sizeof(double) * 2));
  TRY(ensure(P, P->sd_Om, sizeof(double) * (size_t)N));
  TRY(ensure(P, P->sd_V, sizeof(double) * (size_t)n * N));
  const int R = P->n_t * P->n_bas;
  TRY(ensure(P, P->sd_w2, sizeof(double) * (size_t)R * N));
  LAUNCH(CK(gw::sd_casida_matrix(P->d_B_ia, P->d_D, n, (int)N, Np, as<double>(P->sd_M), as<double>(P->sd_T),
                                 P->stream)));
  double off[2] = {1.0, 1.0};
  int sweeps = 0;
  for (; sweeps < 40; ++sweeps) {
    CK(gw::sd_offdiag(as<double>(P->sd_M), Np, as<double>(P->sd_off), P->stream));
    CK(cudaMemcpyAsync(off, P->sd_off.p, sizeof(off), cudaMemcpyDeviceToHost, P->stream));
    CK(cudaStreamSynchronize(P->stream));
    if (!(off[0] > 1e-26 * off[1])) break;
    CK(gw::sd_jacobi_sweep(as<double>(P->sd_M), as<double>(P->sd_T), Np, as<double>(P->sd_cs), P->stream));
    P->stats.n_kernel_launches += 4 * (Np - 1) + 1;
  }
  if (!(off[0] <= 1e-26 * off[1]))
    return fail(P, GW_ERR_NOT_CONVERGED, "Jacobi sweeps of the Casida matrix did not converge (off/diag %g)",
                std::sqrt(off[0] / off[1]));
  LAUNCH(CK(gw::sd_weights(P->d_B_ia, P->d_D, as<double>(P->sd_M), as<double>(P->sd_T), P->d_B_nm, n, (int)N, Np, R,
                           as<double>(P->sd_Om), as<double>(P->sd_V), as<double>(P->sd_w2), P->stream)));
  CK(cudaStreamSynchronize(P->stream));
  P->sd_sweeps = sweeps;
  P->sd_done = true;
  return GW_OK;
}

gw_status gw_sigma_sd(gw_plan_t P, int n_points, const int* target_idx, const double* omega, double* sigma_c,
                      double* dsigma_c) {
  if (!P) return GW_ERR_ARG;
  if (n_points < 0 || (n_points > 0 && !omega)) return fail(P, GW_ERR_ARG, "bad point list");
  if (n_points == 0) return GW_OK;
  std::vector<int> tmap(n_points);
  for (int p = 0; p < n_points; ++p) {
    tmap[p] = target_idx ? target_idx[p] : p;
    if (tmap[p] < 0 || tmap[p] >= P->n_t) return fail(P, GW_ERR_ARG, "target_idx[%d] out of range", p);
    if (!std::isfinite(omega[p])) return fail(P, GW_ERR_ARG, "omega[%d] not finite", p);
  }
  if (!target_idx && n_points != P->n_t) return fail(P, GW_ERR_ARG, "without target_idx, n_points = n_targets");
  TRY(ensure_sd(P));
  TRY(ensure(P, P->sd_tmap, sizeof(int) * n_points));
  TRY(ensure(P, P->sd_om, sizeof(double) * n_points));
  TRY(ensure(P, P->sd_S, sizeof(double) * n_points));
  TRY(ensure(P, P->sd_dS, sizeof(double) * n_points));
  CK(cudaMemcpyAsync(P->sd_tmap.p, tmap.data(), sizeof(int) * n_points, cudaMemcpyHostToDevice, P->stream));
  CK(cudaMemcpyAsync(P->sd_om.p, omega, sizeof(double) * n_points, cudaMemcpyHostToDevice, P->stream));
  LAUNCH(CK(gw::sd_sigma(as<double>(P->sd_w2), as<double>(P->sd_Om), (int)P->n_ov, P->n_bas, P->d_eps_g,
                         as<int>(P->sd_tmap), P->d_spin, P->d_occ_t, P->cfg.n_occ, as<double>(P->sd_om), n_points,
                         P->cfg.eta, as<double>(P->sd_S), as<double>(P->sd_dS), P->stream)));
  std::vector<double> S(n_points), dS(n_points);
  CK(cudaMemcpyAsync(S.data(), P->sd_S.p, sizeof(double) * n_points, cudaMemcpyDeviceToHost, P->stream));
  CK(cudaMemcpyAsync(dS.data(), P->sd_dS.p, sizeof(double) * n_points, cudaMemcpyDeviceToHost, P->stream));
  CK(cudaStreamSynchronize(P->stream));
  for (int p = 0; p < n_points; ++p) {
    if (sigma_c) sigma_c[p] = S[p];
    if (dsigma_c) dsigma_c[p] = dS[p];
  }
  return GW_OK;
}

gw_status gw_sigma_points(gw_plan_t P, int n_points, const int* target_idx, const double* omega, double* sigma_c,
                          double* dsigma_c) {
  if (!P) return GW_ERR_ARG;
  if (n_points < 0 || (n_points > 0 && (!target_idx || !omega))) return fail(P, GW_ERR_ARG, "bad point list");
  if (n_points == 0) return GW_OK;
  for (int p = 0; p < n_points; ++p) {
    if (target_idx[p] < 0 || target_idx[p] >= P->n_t) return fail(P, GW_ERR_ARG, "target_idx[%d] out of range", p);
    if (!std::isfinite(omega[p])) return fail(P, GW_ERR_ARG, "omega[%d] not finite", p);
  }
  TRY(ensure_screening(P));
  std::vector<double> om(omega, omega + n_points);
  std::vector<int> tmap(target_idx, target_idx + n_points);
  std::vector<unsigned char> act(n_points, 1);
  int nf = 0;
  TRY(sigma_eval(P, om, act, &nf, &tmap));
  std::vector<double> R(n_points), dR(n_points), I(n_points), dI(n_points);
  CK(cudaMemcpy(R.data(), P->sg_R.p, sizeof(double) * n_points, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(dR.data(), P->sg_dR.p, sizeof(double) * n_points, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(I.data(), P->sg_I.p, sizeof(double) * n_points, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(dI.data(), P->sg_dI.p, sizeof(double) * n_points, cudaMemcpyDeviceToHost));
  for (int p = 0; p < n_points; ++p) {
    if (sigma_c) sigma_c[p] = R[p] - I[p];
    if (dsigma_c) dsigma_c[p] = dR[p] - dI[p];
  }
  return GW_OK;
}

gw_status gw_residues_minres(gw_plan_t P, int n_rhs, const int* target_idx, const int* m, const double* x,
                             double* w_re, double* w_im, double* dw_re, int* iters, double* resnorm,
                             int* used_fallback) {
  if (!P) return GW_ERR_ARG;
  if (n_rhs < 0 || (n_rhs > 0 && (!target_idx || !m || !x))) return fail(P, GW_ERR_ARG, "bad right-hand side list");
  if (n_rhs == 0) return GW_OK;
  for (int j = 0; j < n_rhs; ++j) {
    if (target_idx[j] < 0 || target_idx[j] >= P->n_t) return fail(P, GW_ERR_ARG, "target_idx[%d] out of range", j);
    if (m[j] < 0 || m[j] >= P->n_bas) return fail(P, GW_ERR_ARG, "m[%d] out of range", j);
    if (!std::isfinite(x[j])) return fail(P, GW_ERR_ARG, "x[%d] not finite", j);
  }
  TRY(ensure(P, P->mr_rt, sizeof(int) * n_rhs));
  TRY(ensure(P, P->mr_rm, sizeof(int) * n_rhs));
  TRY(ensure(P, P->mr_xf, sizeof(double) * n_rhs));
  TRY(ensure(P, P->mr_wre, sizeof(double) * n_rhs));
  TRY(ensure(P, P->mr_wim, sizeof(double) * n_rhs));
  TRY(ensure(P, P->mr_dwre, sizeof(double) * n_rhs));
  TRY(ensure(P, P->mr_it, sizeof(int) * n_rhs));
  TRY(ensure(P, P->mr_res, sizeof(double) * n_rhs));
  CK(cudaMemcpyAsync(P->mr_rt.p, target_idx, sizeof(int) * n_rhs, cudaMemcpyHostToDevice, P->stream));
  CK(cudaMemcpyAsync(P->mr_rm.p, m, sizeof(int) * n_rhs, cudaMemcpyHostToDevice, P->stream));
  CK(cudaMemcpyAsync(P->mr_xf.p, x, sizeof(double) * n_rhs, cudaMemcpyHostToDevice, P->stream));
  std::vector<int> fb(n_rhs, 0);
  TRY(residues(P, n_rhs, as<int>(P->mr_rt), as<int>(P->mr_rm), as<double>(P->mr_xf), as<double>(P->mr_wre),
               as<double>(P->mr_wim), as<double>(P->mr_dwre), as<int>(P->mr_it), as<double>(P->mr_res), fb.data()));
  if (w_re) CK(cudaMemcpy(w_re, P->mr_wre.p, sizeof(double) * n_rhs, cudaMemcpyDeviceToHost));
  if (w_im) CK(cudaMemcpy(w_im, P->mr_wim.p, sizeof(double) * n_rhs, cudaMemcpyDeviceToHost));
  if (dw_re) CK(cudaMemcpy(dw_re, P->mr_dwre.p, sizeof(double) * n_rhs, cudaMemcpyDeviceToHost));
  if (iters) CK(cudaMemcpy(iters, P->mr_it.p, sizeof(int) * n_rhs, cudaMemcpyDeviceToHost));
  if (resnorm) CK(cudaMemcpy(resnorm, P->mr_res.p, sizeof(double) * n_rhs, cudaMemcpyDeviceToHost));
  if (used_fallback) std::memcpy(used_fallback, fb.data(), sizeof(int) * n_rhs);
  return GW_OK;
}

}  // extern "C"

namespace {

// QP loop (Sec. 3.4) for the targets with run[t] != 0, started at om0[t]: every running state's Sigma(omega) per
// evaluation (one batched residue solve for all of them), then one step of the linearised update or of the step
// tree.  Final states go to hs (states not run keep status 1 and om0); any_fb[t] is set when an evaluation of a
// running state used the dense fallback.
gw_status qp_loop(gw_plan* P, int lin, const std::vector<double>& om0, const std::vector<unsigned char>& run,
                  std::vector<QPState>& hs, std::vector<int>& any_fb) {
  const int n_t = P->n_t;
  TRY(ensure(P, P->qp_st, sizeof(QPState) * n_t));
  hs.assign(n_t, QPState{});
  for (int t = 0; t < n_t; ++t) {
    hs[t].omega = om0[t];
    hs[t].Z = 1.0;
    hs[t].status = run[t] ? 0 : 1;
  }
  CK(cudaMemcpyAsync(P->qp_st.p, hs.data(), sizeof(QPState) * n_t, cudaMemcpyHostToDevice, P->stream));
  std::vector<double> om(n_t);
  std::vector<unsigned char> act(n_t);
  const int maxit = lin ? 1 : P->cfg.qp_maxit;
  for (int it = 0; it < maxit; ++it) {
    CK(cudaMemcpyAsync(hs.data(), P->qp_st.p, sizeof(QPState) * n_t, cudaMemcpyDeviceToHost, P->stream));
    CK(cudaStreamSynchronize(P->stream));
    int n_act = 0;
    for (int t = 0; t < n_t; ++t) {
      om[t] = hs[t].omega;
      act[t] = hs[t].status == 0 ? 1 : 0;
      n_act += act[t];
    }
    if (n_act == 0) break;
    int nf = 0;
    TRY(sigma_eval(P, om, act, &nf));
    if (nf > 0)
      for (int t = 0; t < n_t; ++t)
        if (act[t]) any_fb[t] = 1;   // conservative: flag the active states of an evaluation that fell back
    LAUNCH(gw::launch_qp_step(as<QPState>(P->qp_st), as<double>(P->sg_R), as<double>(P->sg_dR),
                              as<double>(P->sg_I), as<double>(P->sg_dI), P->d_en, P->d_shift, P->cfg.qp_tol,
                              P->cfg.qp_maxit, n_t, lin, P->stream));
  }
  CK(cudaMemcpyAsync(hs.data(), P->qp_st.p, sizeof(QPState) * n_t, cudaMemcpyDeviceToHost, P->stream));
  CK(cudaStreamSynchronize(P->stream));
  for (int t = 0; t < n_t; ++t)
    if (!run[t]) hs[t].omega = om0[t];
  return GW_OK;
}

// Graphical search (Sec. 3.4): f(w) = e_n + shift + Sigma_c(w) - w on qp_window_points evenly spaced points of
// [c_t - qp_window, c_t + qp_window] for every target with run[t], all points of all targets in one batched
// evaluation.  root[t] = the sign change of f with f decreasing (a root of the QP equation, not a pole of Sigma)
// closest to c_t, by linear interpolation; found[t] = 0 if the window holds none.
gw_status graphical_scan(gw_plan* P, const std::vector<double>& c, const std::vector<unsigned char>& run,
                         std::vector<double>& root, std::vector<unsigned char>& found, std::vector<int>& any_fb) {
  const int n_t = P->n_t, np = std::max(2, P->cfg.qp_window_points);
  const double hw = P->cfg.qp_window;
  std::vector<int> tmap;
  std::vector<double> om;
  for (int t = 0; t < n_t; ++t)
    if (run[t])
      for (int j = 0; j < np; ++j) {
        tmap.push_back(t);
        om.push_back(c[t] + hw * (-1.0 + 2.0 * j / (np - 1)));
      }
  root = c;
  found.assign(n_t, 0);
  if (om.empty()) return GW_OK;
  std::vector<unsigned char> act(om.size(), 1);
  int nf = 0;
  TRY(sigma_eval(P, om, act, &nf, &tmap));
  std::vector<double> R(om.size()), I(om.size());
  CK(cudaMemcpyAsync(R.data(), P->sg_R.p, sizeof(double) * om.size(), cudaMemcpyDeviceToHost, P->stream));
  CK(cudaMemcpyAsync(I.data(), P->sg_I.p, sizeof(double) * om.size(), cudaMemcpyDeviceToHost, P->stream));
  CK(cudaStreamSynchronize(P->stream));
  for (size_t k = 0; k < om.size(); ++k) {
    const int t = tmap[k];
    if (nf > 0) any_fb[t] = 1;
    if (k + 1 >= om.size() || tmap[k + 1] != t) continue;
    const double f0 = P->h_en[t] + P->h_shift[t] + R[k] - I[k] - om[k];
    const double f1 = P->h_en[t] + P->h_shift[t] + R[k + 1] - I[k + 1] - om[k + 1];
    if ((f0 > 0.0 && f1 <= 0.0) || (f0 == 0.0 && f1 < 0.0)) {
      const double r = om[k] + (om[k + 1] - om[k]) * f0 / (f0 - f1);
      if (!found[t] || std::fabs(r - c[t]) < std::fabs(root[t] - c[t])) root[t] = r;
      found[t] = 1;
    }
  }
  return GW_OK;
}

// QP energies of the targets with run[t] from the starting points / window centres start[t]: linearised, step
// tree, or graphical search followed by the step tree from the root it found.
gw_status qp_solve_set(gw_plan* P, gw_qp_mode mode, const std::vector<double>& start,
                       const std::vector<unsigned char>& run, std::vector<QPState>& hs, std::vector<int>& any_fb,
                       std::vector<unsigned char>& no_root) {
  const int n_t = P->n_t;
  no_root.assign(n_t, 0);
  if (mode != GW_QP_GRAPHICAL) return qp_loop(P, mode == GW_QP_LINEARISED, start, run, hs, any_fb);
  std::vector<double> root;
  std::vector<unsigned char> found;
  TRY(graphical_scan(P, start, run, root, found, any_fb));
  std::vector<unsigned char> run2(n_t, 0);
  for (int t = 0; t < n_t; ++t) {
    run2[t] = run[t] && found[t];
    no_root[t] = run[t] && !found[t];
  }
  return qp_loop(P, 0, root, run2, hs, any_fb);
}

// QP equation of every target (Sec. 3.4), with the cluster layer when qp_cluster_gap > 0 (not in the linearised
// mode): targets whose KS energies are within qp_cluster_gap of a neighbour in energy form a cluster; the first
// member of each cluster (lowest KS energy) is solved first, then every other member starts from its KS energy
// shifted by that member's QP correction (the step tree's start, or the centre of the graphical window).
// omega0 (host [n_targets]) replaces the KS energies as starting points, or NULL.
gw_status qp_solve_impl(gw_plan* P, gw_qp_mode mode, const double* omega0, double* e_qp, double* z_factor,
                        int* state_status) {
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  CK(cudaEventRecord(a, P->stream));
  TRY(ensure_screening(P));
  const int n_t = P->n_t;
  std::vector<double> start(n_t);
  for (int t = 0; t < n_t; ++t) start[t] = omega0 ? omega0[t] : P->h_en[t];
  std::vector<QPState> hs;
  std::vector<int> any_fb(n_t, 0);
  std::vector<unsigned char> no_root;
  const bool cluster = P->cfg.qp_cluster_gap > 0.0 && mode != GW_QP_LINEARISED;
  if (!cluster) {
    std::vector<unsigned char> run(n_t, 1);
    TRY(qp_solve_set(P, mode, start, run, hs, any_fb, no_root));
  } else {
    std::vector<int> order(n_t);
    for (int t = 0; t < n_t; ++t) order[t] = t;
    std::sort(order.begin(), order.end(), [&](int x, int y) { return P->h_en[x] < P->h_en[y]; });
    std::vector<int> rep(n_t);
    std::vector<unsigned char> first(n_t, 0), rest(n_t, 0);
    for (int k = 0; k < n_t; ++k) {
      const int t = order[k];
      if (k == 0 || P->h_en[t] - P->h_en[order[k - 1]] > P->cfg.qp_cluster_gap) {
        rep[t] = t;
        first[t] = 1;
      } else {
        rep[t] = rep[order[k - 1]];
        rest[t] = 1;
      }
    }
    std::vector<QPState> h1;
    std::vector<unsigned char> nr1;
    TRY(qp_solve_set(P, mode, start, first, h1, any_fb, nr1));
    std::vector<double> start2(start);
    for (int t = 0; t < n_t; ++t)
      if (rest[t] && h1[rep[t]].status == 1 && !nr1[rep[t]])
        start2[t] = start[t] + (h1[rep[t]].omega - P->h_en[rep[t]]);
    TRY(qp_solve_set(P, mode, start2, rest, hs, any_fb, no_root));
    for (int t = 0; t < n_t; ++t)
      if (first[t]) {
        hs[t] = h1[t];
        no_root[t] = nr1[t];
      }
  }
  CK(cudaEventRecord(b, P->stream));
  CK(cudaStreamSynchronize(P->stream));
  P->stats.ms_qp = now_ms(P, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  bool all_ok = true;
  for (int t = 0; t < n_t; ++t) {
    const bool conv = hs[t].status == 1 && !no_root[t];
    if (e_qp) e_qp[t] = hs[t].omega;
    if (z_factor) z_factor[t] = no_root[t] ? NAN : hs[t].Z;
    if (!conv) all_ok = false;
    if (state_status) state_status[t] = conv ? (any_fb[t] ? 2 : 0) : 1;
  }
  return all_ok ? GW_OK : GW_ERR_NOT_CONVERGED;
}

// Energies of the next eigenvalue cycle, per spin: targets take their QP energies, every other occupied state moves
// by the correction of the highest occupied target of its spin, every other virtual state by that of the lowest
// virtual target of its spin.
std::vector<double> scissor(const gw_plan* P, int spin, const std::vector<double>& e_qp) {
  const int n_occ = P->occ_s[spin];
  const std::vector<double>& ks = P->h_eps_s[spin];
  std::vector<double> out(ks);
  double e_o = -INFINITY, d_o = 0.0, e_v = INFINITY, d_v = 0.0;
  for (int t = 0; t < P->n_t; ++t) {
    if (P->h_spin[t] != spin) continue;
    const int n = P->h_targets[t];
    const double e = ks[n], d = e_qp[t] - e;
    if (n < n_occ && (e > e_o || (e == e_o && d > d_o))) { e_o = e; d_o = d; }
    if (n >= n_occ && (e < e_v || (e == e_v && d < d_v))) { e_v = e; d_v = d; }
  }
  for (int m = 0; m < P->n_bas; ++m) out[m] += m < n_occ ? d_o : d_v;
  for (int t = 0; t < P->n_t; ++t)
    if (P->h_spin[t] == spin) out[P->h_targets[t]] = e_qp[t];
  return out;
}

}  // namespace

extern "C" {

gw_status gw_qp_solve(gw_plan_t P, gw_qp_mode mode, double* e_qp, double* z_factor, int* state_status) {
  if (!P) return GW_ERR_ARG;
  if (mode != GW_QP_LINEARISED && mode != GW_QP_STEPTREE && mode != GW_QP_GRAPHICAL)
    return fail(P, GW_ERR_ARG, "unknown QP mode %d", (int)mode);
  return qp_solve_impl(P, mode, nullptr, e_qp, z_factor, state_status);
}

gw_status gw_evgw(gw_plan_t P, int update_w, gw_qp_mode mode, int max_iter, double tol, double* e_qp,
                  double* z_factor, int* state_status, int* iterations) {
  if (!P) return GW_ERR_ARG;
  if (mode != GW_QP_LINEARISED && mode != GW_QP_STEPTREE && mode != GW_QP_GRAPHICAL)
    return fail(P, GW_ERR_ARG, "unknown QP mode %d", (int)mode);
  if (max_iter <= 0 || !(tol > 0.0)) return fail(P, GW_ERR_ARG, "max_iter must be positive and tol > 0");
  const int n_t = P->n_t;
  std::vector<double> prev(n_t), cur(n_t), z(n_t);
  std::vector<int> st(n_t);
  for (int t = 0; t < n_t; ++t) prev[t] = P->h_en[t];
  std::vector<double> eps_cur[2] = {P->h_eps_s[0], P->h_eps_s[1]};
  gw_status last = GW_OK;
  bool conv = false;
  int it = 0;
  for (it = 1; it <= max_iter; ++it) {
    for (int sp = 0; sp < P->n_spin; ++sp) TRY(set_g_energies(P, sp, eps_cur[sp].data()));
    if (update_w && it > 1) {            // evGW: W from the current energies (cycle 1 is G0W0)
      TRY(set_pair_energies(P, eps_cur[0].data(), eps_cur[1].data()));
      P->screening_done = false;
    }
    last = qp_solve_impl(P, mode, prev.data(), cur.data(), z.data(), st.data());
    if (last != GW_OK && last != GW_ERR_NOT_CONVERGED) break;
    double delta = 0.0;
    for (int t = 0; t < n_t; ++t) delta = std::max(delta, std::fabs(cur[t] - prev[t]));
    prev = cur;
    for (int sp = 0; sp < P->n_spin; ++sp) eps_cur[sp] = scissor(P, sp, cur);
    if (delta < tol) { conv = true; break; }
  }
  // the plan goes back to G0W0: G and W from the KS energies (W is rebuilt on the next call that needs it)
  gw_status rs = GW_OK;
  for (int sp = 0; sp < P->n_spin && rs == GW_OK; ++sp) rs = set_g_energies(P, sp, P->h_eps_s[sp].data());
  if (rs == GW_OK && update_w) {
    rs = set_pair_energies(P, P->h_eps_s[0].data(), P->h_eps_s[1].data());
    P->screening_done = false;
  }
  if (last != GW_OK && last != GW_ERR_NOT_CONVERGED) return last;
  if (rs != GW_OK) return rs;
  for (int t = 0; t < n_t; ++t) {
    if (e_qp) e_qp[t] = cur[t];
    if (z_factor) z_factor[t] = z[t];
    if (state_status) state_status[t] = st[t];
  }
  if (iterations) *iterations = std::min(it, max_iter);
  if (!conv) return fail(P, GW_ERR_NOT_CONVERGED, "eigenvalue cycles did not converge to %g Ha in %d", tol, max_iter);
  return last;
}

gw_status gw_shard_columns(int n_freq, int rank, int world, int* p0, int* p1) {
  if (n_freq <= 0 || world <= 0 || rank < 0 || rank >= world || !p0 || !p1) return GW_ERR_ARG;
  const long n = (long)n_freq + 1;
  *p0 = (int)(n * rank / world);
  *p1 = (int)(n * (rank + 1) / world);
  return GW_OK;
}

gw_status gw_set_shard(gw_plan_t P, int rank, int world, gw_allreduce_fn allreduce_sum, void* ctx) {
  if (!P) return GW_ERR_ARG;
  if (world < 1 || rank < 0 || rank >= world || (world > 1 && !allreduce_sum))
    return fail(P, GW_ERR_ARG, "bad shard (rank %d of %d)", rank, world);
  P->sh_rank = rank;
  P->sh_world = world;
  P->sh_reduce = world > 1 ? allreduce_sum : nullptr;
  P->sh_ctx = ctx;
  P->screening_done = false;
  return GW_OK;
}

gw_status gw_plan_footprint(const gw_config* c, int n_t, unsigned flags, unsigned long long* bytes) {
  if (!c || !bytes || c->n_occ <= 0 || c->n_virt <= 0 || c->n_aux <= 0 || c->n_freq <= 0 || n_t <= 0)
    return GW_ERR_ARG;
  // Mirrors the allocations of plan_create_impl and of every ensure() class below, each at its cap.
  typedef unsigned long long u64;
  const bool mixed = c->precision == GW_PREC_MIXED;
  const u64 n = c->n_aux, n_ov = (u64)c->n_occ * c->n_virt, n_bas = (u64)c->n_occ + c->n_virt;
  const u64 n_g1 = (u64)c->n_freq + 1, ts = mixed ? 4 : 8;
  const u64 ws = (u64)(c->workspace_mb > 0 ? c->workspace_mb : 8192) << 20;
  const u64 ldo = (u64)gw::tc_ld((int)std::min<u64>(n_ov, 2147483647ull)), ldn = (u64)gw::tc_ld(c->n_aux);
  const u64 rows = (u64)n_t * n_bas, nBn = rows * n;
  auto capped = [ws](u64 item, u64 want) { return std::max(item, std::min(ws / std::max<u64>(item, 1) * item, want)); };
  u64 b = 8 * (n_bas + 2 * n_g1 + 3 * (u64)n_t) + 8 * rows * n_g1;         // energies, grid, shifts, W table
  if (!(flags & GW_BORROW_DEVICE_PTRS)) b += 8 * (n * n_ov + nBn);           // B_ia, B_nm
  const u64 ldf = (u64)gw::pf_ldw((int)std::min<u64>(n_ov, 2147483647ull));
  if (mixed) {
    b += 4 * (n * ldf + nBn);                                                // FP32 copies
    b += 6 * (n * ldo + rows * ldn + n_ov * ldn);                             // three BF16 parts of B, B_nm, B^T
    b += 12 * n_ov;                                                          // sorted D and its pair index
    b += 4 * n * (u64)gw::tc_pi_panel_cols((int)std::min<u64>(n_ov, 2147483647ull));   // K-panel hi/lo of B
  }
  b += 8 * n_ov;                                                             // pair energies D_ia
  // imaginary-axis stage: frequency matrices, info/index lists
  b += capped(n * n * ts, n * n * ts * n_g1) + 24 * n_g1;
  if (mixed) {
    // weight table of one Pi launch: a screening chunk or two entries per fallback matrix
    const u64 nb = std::max<u64>(n_g1, 2 * std::max<u64>(1, ws / (2 * n * n * ts)));
    b += 4 * nb * ldf + 16 * nb;
    b += std::min(ws, 8 * nb * n * n * 4);                                     // split-K partials (small problems)
    const u64 per_ns = n * ldn * 24 + n * n * 8;                             // Newton-Schulz split/FP32 iterates
    b += capped(per_ns, per_ns * n_g1) + 6 * n * ldn + 4 * n_g1;             // + the split eps(0)^-1 - 1
    b += 8 * n * n_g1 + 16 * n_g1;                                           // spectrum-estimate vectors
  } else {
    b += 8 * (u64)gw::trsm_w_scratch_elems<double>(c->n_aux, gw::trsm_w_default_ctas());
  }
  // residue batch (at most one right-hand side per target and state at a time)
  u64 batch = c->max_rhs_batch > 0 ? (u64)c->max_rhs_batch
                                   : std::max<u64>(1, std::min<u64>((ws / 2) / (2 * n_ov * ts), 2048));
  batch = std::min(batch, std::max<u64>(1, rows));
  b += batch * (4 * n * ts + 2 * n_ov * ts + 10 * n * 8 + 64);               // V, S, U, Lanczos vectors, state
  if (mixed) {
    b += batch * (16 * n + 8 * ldn + 8 * ldo);                               // FP64 solutions, split V and U
    if (c->op_parts >= 3) b += batch * (4 * ldn + 4 * ldo);
  }
  b += 48 * std::max<u64>(1, rows) + 8 * 6 * (u64)n_t + 64;                  // residue lists, Sigma scratch
  // dense fallback batch
  const u64 mat2 = 2 * n * n * ts;
  const u64 fb = std::max<u64>(1, ws / mat2);
  b += capped(mat2, mat2 * fb) + fb * (2 * n * ts + 8 * n + 8);
  if (mixed) {
    b += fb * (16 * n + 16 * n + 12 * ldn + 12 * ldo + 40);                  // FP64 solutions, V/S, split parts
    b += fb * (32 * n + 16 * n_ov) + 4 * n * n_ov;                           // FP64-residual vectors, df lo part of B
    b += 2 * (u64)lu_work_elems(c->n_aux, (long)std::min<u64>(fb, 1u << 30));            // blocked-LU split operands
  }
  *bytes = b;
  return GW_OK;
}

gw_status gw_grid(int N, double x0, double* xi, double* wt) {
  if (N <= 0 || !(x0 > 0.0) || !xi || !wt) return GW_ERR_ARG;
  // P_N(t) and P_N'(t) by the three-term recurrence
  auto legendre = [N](double t, double* dp) {
    double p0 = 1.0, p1 = t;
    for (int l = 2; l <= N; ++l) {
      double p2 = ((2.0 * l - 1.0) * t * p1 - (l - 1.0) * p0) / l;
      p0 = p1;
      p1 = p2;
    }
    *dp = N * (t * p1 - p0) / (t * t - 1.0);
    return p1;
  };
  for (int k = 0; k < N; ++k) {
    double t = -std::cos(M_PI * (k + 0.75) / (N + 0.5));   // Newton from the asymptotic node estimate
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p = legendre(t, &dp);
      double dt = p / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    legendre(t, &dp);
    double wgl = 2.0 / ((1.0 - t * t) * dp * dp);
    xi[k] = x0 * (1.0 + t) / (1.0 - t);
    wt[k] = 2.0 * x0 * wgl / ((1.0 - t) * (1.0 - t));
  }
  return GW_OK;
}

gw_status gw_w_table(gw_plan_t P, double* out) {
  if (!P || !out) return P ? fail(P, GW_ERR_ARG, "out is NULL") : GW_ERR_ARG;
  TRY(ensure_screening(P));
  CK(cudaMemcpy(out, P->d_W, sizeof(double) * (size_t)P->n_t * P->n_bas * (P->n_g + 1), cudaMemcpyDeviceToHost));
  return GW_OK;
}

gw_status gw_get_stats(gw_plan_t P, gw_stats* out) {
  if (!P || !out) return GW_ERR_ARG;
  *out = P->stats;
  return GW_OK;
}

void gw_plan_destroy(gw_plan_t P) { free_plan(P); }

const char* gw_last_error(gw_plan_t P) {
  if (!P) return g_create_error.c_str();
  return P->err.c_str();
}

}  // extern "C"
