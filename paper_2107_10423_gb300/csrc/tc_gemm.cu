// tcgen05 (5th-generation tensor core) batched GEMM with BF16 hi+lo split operands, used for every
// dense contraction of the mixed-precision path:
//   out_b[m][n] = f( sum_k A_b[m][k] * Bm[n][k] ),   A_b = Ahi_b + Alo_b,  Bm = Bhi + Blo  (BF16)
// computed as Ahi*Bhi + Ahi*Blo + Alo*Bhi with FP32 accumulation in tensor memory (TMEM).
//  * Pi(i xi_b) (Sec. 3.3): A_b = B_ia o w_b with w_b,ia = -4 D_ia/(D_ia^2 + xi_b^2), Bm = B_ia, lower tiles.
//  * dense real-axis Pi(x_j) for the residue fallback: A = B_ia o Re c(x_j) and B_ia o Im c(x_j).
// Operands are staged by TMA (cp.async.bulk.tensor, 128-byte swizzle) into a 3-stage shared-memory
// ring; one elected thread issues tcgen05.mma; the accumulator is read back with tcgen05.ld.
// Every mbarrier wait is bounded: on timeout the kernel records an error code and unwinds.
#include "pi_tc.cuh"
#include "gw_internal.cuh"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstdio>

namespace gw {
namespace {

constexpr int BM = 128, BN = 128, BK = 64, THREADS = 192;
constexpr int EPI_U = 8;         // epilogue elements per thread whose global reads are in flight together
constexpr int TILE_BYTES = BM * BK * 2;               // one 128 x 64 BF16 tile = 16 KiB

// NSP split parts per operand: 2 (hi, lo: products hh, hl, lh) or 3 (hi, mid, lo: the six products with
// part indices i + j <= 2, about FP32-accurate).  A stage holds NSP A tiles and NSP B tiles.
template <int NSP>
struct TcCfg {
  static constexpr int CHUNK = NSP == 2 ? 4 : 1;     // k-blocks per TMEM chunk before the drain
  static constexpr int STAGES = NSP == 2 ? 3 : 2;
  static constexpr int STAGE_BYTES = 2 * NSP * TILE_BYTES;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
};
// Two chunk buffers x two accumulators (hi*hi alone; every cross product together) x 128 columns.  Keeping the
// dominant hi*hi product apart leaves its accumulator one accumulate per k-step; the cross terms are 2^8
// smaller, so their accumulator's rounding is negligible.
constexpr uint32_t TMEM_COLS = 512;
constexpr long long WAIT_LIMIT = 1ll << 26;           // bounded spin on every mbarrier

// tcgen05 instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, N = BN, M = BM.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait; returns false (and records `code`) if the phase did not complete in time.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code) {
  for (long long i = 0; i < WAIT_LIMIT; ++i)
    if (mbar_try(bar, parity)) return true;
  atomicCAS(err, 0, code);
  return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major tile with 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                  // leading byte offset (unused with 128-byte swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset
  d |= (uint64_t)1 << 46;                  // descriptor version
  d |= (uint64_t)2 << 61;                  // SWIZZLE_128B
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(IDESC), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Epilogues.  The tile is staged in shared memory as stg[BM][BN + 1] (row = output row), so any thread can combine
// elements of different rows (the complex pairs of the residue operator are adjacent rows).
__device__ __forceinline__ void split_store(float v, __nv_bfloat16* hi, __nv_bfloat16* lo, long o,
                                            __nv_bfloat16* lo2 = nullptr) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  hi[o] = h;
  const float r = v - __bfloat162float(h);
  const __nv_bfloat16 m = __float2bfloat16_rn(r);
  lo[o] = m;
  if (lo2) lo2[o] = __float2bfloat16_rn(r - __bfloat162float(m));
}

__device__ void epilogue(const TcEpi& ep, const float* stg, int m0, int n0, int M, int N, int b, int lower,
                         int* err) {
  if (ep.kind == TC_EPI_STORE) {
    const int mode = (b & 1) ? ep.mode_odd : ep.mode_even;
    float* o = ep.out + (long)b * ep.out_bstride;
    for (int idx = threadIdx.x; idx < BM * BN; idx += THREADS) {
      const int rr = idx / BN, cc = idx % BN;
      const int m = m0 + rr, n = n0 + cc;
      if (m >= M || n >= N) continue;
      if (lower && n > m) continue;
      float v = stg[rr * (BN + 1) + cc];
      v = mode == 0 ? v : (mode == 1 ? ((m == n ? 1.f : 0.f) - v) : -v);
      o[(long)m * ep.ldo + n] = v;
    }
    if (lower) {
      for (int idx = threadIdx.x; idx < BM * BN; idx += THREADS) {
        const int cc = idx / BM, rr = idx % BM;
        const int m = m0 + rr, n = n0 + cc;
        if (m >= M || n >= N || n >= m) continue;
        const float v = stg[rr * (BN + 1) + cc];
        o[(long)n * ep.ldo + m] = mode == 0 ? v : -v;
      }
    }
  } else if (ep.kind == TC_EPI_CPAIR) {
    // rows (2j, 2j+1) hold B^T u and B^T v of z_j = u - i v; column k is the pair ia.
    // w = c_k(x_j) (t_r + i t_i) with t = B^T z, c_k(x) = 2[1/(x - D_k + i eta) + 1/(-x - D_k + i eta)];
    // Re w and Im w go to rows 2j, 2j+1 of the split operand of the second GEMM.
    const float e2 = ep.eta * ep.eta;
    for (int idx = threadIdx.x; idx < (BM / 2) * BN; idx += THREADS) {
      const int pr = idx / BN, cc = idx % BN;
      const int m = m0 + 2 * pr, n = n0 + cc;
      if (m >= M || n >= N) continue;
      const double x = ep.x[m >> 1], D = ep.Dk[n];
      const float a1 = (float)(x - D), a2 = (float)(-x - D);
      const float d1 = a1 * a1 + e2, d2 = a2 * a2 + e2;
      const float cr = 2.f * (a1 / d1 + a2 / d2);
      const float ci = -2.f * ep.eta * (1.f / d1 + 1.f / d2);
      const float tr = stg[(2 * pr) * (BN + 1) + cc], ti = -stg[(2 * pr + 1) * (BN + 1) + cc];
      split_store(cr * tr - ci * ti, ep.ohi, ep.olo, (long)m * ep.ldh + n, ep.olo2);
      split_store(cr * ti + ci * tr, ep.ohi, ep.olo, (long)(m + 1) * ep.ldh + n, ep.olo2);
    }
  } else if (ep.kind == TC_EPI_AXPBY) {
    // EPI_U elements per thread and pass: their global reads are issued together before any store
    for (int base = threadIdx.x; base < BM * BN; base += THREADS * EPI_U) {
      float xv[EPI_U];
#pragma unroll
      for (int u = 0; u < EPI_U; ++u) {
        const int idx = base + u * THREADS, rr = idx / BN, cc = idx % BN, m = m0 + rr, n = n0 + cc;
        xv[u] = (ep.xin && idx < BM * BN && m < M && n < N)
                    ? ep.xin[(long)b * ep.x_bstride + (long)m * ep.ldo + n] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < EPI_U; ++u) {
        const int idx = base + u * THREADS, rr = idx / BN, cc = idx % BN, m = m0 + rr, n = n0 + cc;
        if (idx >= BM * BN || m >= M || n >= N) continue;
        const float y = ep.gamma * stg[rr * (BN + 1) + cc] + (m == n ? ep.beta : 0.f) + ep.alpha * xv[u];
        if (ep.out) ep.out[(long)b * ep.out_bstride + (long)m * ep.ldo + n] = y;
        if (ep.ohi) split_store(y, ep.ohi, ep.olo, (long)b * ep.oh_bstride + (long)m * ep.ldh + n, ep.olo2);
      }
    }
  } else if (ep.kind == TC_EPI_WRED) {
    // column n of the tile: sum over the tile's rows m of bvec[n][m] * v[m][n], added into W
    if (threadIdx.x < BN) {
      const int cc = threadIdx.x, n = n0 + cc;
      if (n < N) {
        const float* bv = ep.bvec + (long)n * ep.ldb;
        double acc = 0.0;
        for (int rr = 0; rr < BM && m0 + rr < M; ++rr) acc += (double)bv[m0 + rr] * stg[rr * (BN + 1) + cc];
        atomicAdd(ep.W + (long)n * ep.wld + ep.gidx[b], acc);
      }
    }
  } else if (ep.kind == TC_EPI_SUB2) {
    float* o = ep.out + (long)b * ep.out_bstride;
    for (int base = threadIdx.x; base < BM * BN; base += THREADS * EPI_U) {
      long off[EPI_U];
      float cv[EPI_U];
#pragma unroll
      for (int u = 0; u < EPI_U; ++u) {
        const int idx = base + u * THREADS, rr = idx / BN, cc = idx % BN, m = m0 + rr, n = n0 + cc;
        off[u] = -1;
        if (idx < BM * BN && m < M && n < N) {
          const long o1 = m < ep.half ? (long)m * ep.ldo + n : ep.plane + (long)(m - ep.half) * ep.ldo + n;
          if ((long)b * ep.out_bstride + o1 >= ep.limit || o1 < 0) atomicCAS(err, 0, 66);
          else off[u] = o1;
        }
        cv[u] = off[u] >= 0 ? o[off[u]] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < EPI_U; ++u) {
        const int idx = base + u * THREADS, rr = idx / BN, cc = idx % BN;
        if (off[u] >= 0) o[off[u]] = cv[u] - stg[rr * (BN + 1) + cc];
      }
    }
  } else if (ep.kind == TC_EPI_EMBED) {
    // real 2n embedding of (1 - Pi) z: rows 2j: u - (B w)_r, rows 2j+1: -v - (B w)_i
    for (int base = threadIdx.x; base < BM * BN; base += THREADS * EPI_U) {
      float vv[EPI_U];
#pragma unroll
      for (int u = 0; u < EPI_U; ++u) {
        const int idx = base + u * THREADS, rr = idx / BN, cc = idx % BN, m = m0 + rr, n = n0 + cc;
        vv[u] = (idx < BM * BN && m < M && n < N) ? ep.vin[(long)m * ep.ldv + n] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < EPI_U; ++u) {
        const int idx = base + u * THREADS, rr = idx / BN, cc = idx % BN, m = m0 + rr, n = n0 + cc;
        if (idx >= BM * BN || m >= M || n >= N) continue;
        ep.out[(long)m * ep.ldo + n] = ((m & 1) ? -vv[u] : vv[u]) - stg[rr * (BN + 1) + cc];
      }
    }
  }
}

// grid.x: output tile (lower-triangular enumeration when `lower`), grid.y: batch entry.
// Warp roles: warps 0-3 drain the accumulator (TMEM lane quarter = warp), warp 4 issues TMA, warp 5 issues MMA.
// The contraction is cut into chunks of CHUNK k-blocks; each chunk accumulates in one of two TMEM buffers and
// is then added into FP32 registers by the drain warps (round to nearest), so no partial sum runs through more
// than 4 * CHUNK tensor-core accumulates of the dominant hi*hi product (the tensor-core accumulator loses about
// one ulp per accumulate, which over long K leaves a systematic relative error).
// mode_even / mode_odd select the epilogue for even / odd batch entries:
//   0: v    1: delta_mn - v    2: -v
struct TcMaps {
  CUtensorMap a[3], b[3];
};

template <int NSP>
__global__ void __launch_bounds__(THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ TcMaps maps, int M, int N, int K, int lower, int b_batched, const TcEpi ep,
                   int* __restrict__ err) {
  constexpr int STAGES = TcCfg<NSP>::STAGES;
  constexpr int STAGE_BYTES = TcCfg<NSP>::STAGE_BYTES;
  constexpr int CHUNK = TcCfg<NSP>::CHUNK;
  if (ep.run_if && *ep.run_if == 0) return;     // uniform over the grid: nothing is allocated yet
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* smem = smem_raw + (base - raw);
  // barriers: full[S], empty[S], acc_full[2], acc_empty[2]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 4);
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int bm, bn;
  if (lower) {
    int t = blockIdx.x;
    bm = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((bm + 1) * (bm + 2) / 2 <= t) ++bm;
    while (bm * (bm + 1) / 2 > t) --bm;
    bn = t - bm * (bm + 1) / 2;
  } else {
    const int nbn = (N + BN - 1) / BN;
    bm = blockIdx.x / nbn;
    bn = blockIdx.x % nbn;
  }
  const int m0 = bm * BM, n0 = bn * BN, b = blockIdx.y;
  const int nk = (K + BK - 1) / BK;
  const int nchunks = (nk + CHUNK - 1) / CHUNK;

  uint32_t full[STAGES], empty[STAGES];
  for (int s = 0; s < STAGES; ++s) {
    full[s] = smem_u32(&bars[s]);
    empty[s] = smem_u32(&bars[STAGES + s]);
  }
  const uint32_t acc_full[2] = {smem_u32(&bars[2 * STAGES]), smem_u32(&bars[2 * STAGES + 1])};
  const uint32_t acc_empty[2] = {smem_u32(&bars[2 * STAGES + 2]), smem_u32(&bars[2 * STAGES + 3])};

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full[s], 1);
      mbar_init(empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(acc_full[i], 1);
      mbar_init(acc_empty[i], 4);      // one arrival per drain warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  float acc[BN];                    // drain warps: FP32 sum of the chunk partials for row (warp*32 + lane)
  bool ok = true;
  int issued = 0;
  if (warp == 4) {
    if (lane == 0) {
      // ---------------- TMA producer
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % STAGES, u = kb / STAGES;
        if (u > 0 && !mbar_wait(empty[s], (u - 1) & 1, err, 1)) { s_abort = 1; break; }
        if (*(volatile int*)&s_abort) break;
        const uint32_t st = base + s * STAGE_BYTES;
        mbar_expect_tx(full[s], STAGE_BYTES);
#pragma unroll
        for (int i = 0; i < NSP; ++i) tma_load_3d(st + i * TILE_BYTES, &maps.a[i], kb * BK, m0, b, full[s]);
#pragma unroll
        for (int j = 0; j < NSP; ++j)
          tma_load_3d(st + (NSP + j) * TILE_BYTES, &maps.b[j], kb * BK, n0, b_batched ? b : 0, full[s]);
        issued = kb + 1;
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {
      // ---------------- MMA issuer
      for (int kb = 0; kb < nk && !*(volatile int*)&s_abort; ++kb) {
        const int s = kb % STAGES, u = kb / STAGES;
        const int c = kb / CHUNK, buf = c & 1, first = (kb % CHUNK) == 0;
        if (first && c >= 2 && !mbar_wait(acc_empty[buf], ((c >> 1) - 1) & 1, err, 5)) { s_abort = 1; break; }
        if (!mbar_wait(full[s], u & 1, err, 2)) { s_abort = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t st = base + s * STAGE_BYTES;
        const uint32_t dbig = tmem + (uint32_t)(buf * 2 * BN), dsmall = dbig + BN;
#pragma unroll
        for (int k = 0; k < BK / 16; ++k) {
          const uint32_t off = k * 32;
#pragma unroll
          for (int i = 0; i < NSP; ++i)
#pragma unroll
            for (int j = 0; j + i < NSP; ++j) {
              const uint64_t ad = sdesc(st + i * TILE_BYTES + off), bd = sdesc(st + (NSP + j) * TILE_BYTES + off);
              const bool is_big = (i == 0 && j == 0);
              const bool first_in_acc = first && k == 0 && (is_big || (i == 0 && j == 1));
              mma_bf16(is_big ? dbig : dsmall, ad, bd, first_in_acc ? 0u : 1u);
            }
        }
        mma_commit(empty[s]);
        if ((kb % CHUNK) == CHUNK - 1 || kb == nk - 1) mma_commit(acc_full[buf]);
      }
    }
  } else {
    // ---------------- drain warps 0-3
#pragma unroll
    for (int j = 0; j < BN; ++j) acc[j] = 0.f;
    for (int c = 0; c < nchunks; ++c) {
      const int buf = c & 1;
      ok = mbar_wait(acc_full[buf], (c >> 1) & 1, err, 3);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int q = 0; q < BN / 32; ++q) {
        uint32_t v[32], w[32];
        const uint32_t col = (uint32_t)(buf * 2 * BN + q * 32);
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + col, v);
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + col + BN, w);
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[q * 32 + j] += __uint_as_float(v[j]) + __uint_as_float(w[j]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acc_empty[buf]) : "memory");
    }
  }
  __syncwarp();
  const bool all_ok = __syncthreads_and(ok && !s_abort) != 0;
  // drain copies still in flight if the pipeline was aborted
  if (!all_ok && warp == 4 && lane == 0)
    for (int kb = 0; kb < issued; ++kb) mbar_wait(full[kb % STAGES], (kb / STAGES) & 1, err, 4);
  __syncthreads();
  float* stg = reinterpret_cast<float*>(smem);     // [BM][BN + 1], reuses the operand ring
  if (all_ok && warp < 4) {
    const int r = warp * 32 + lane;
#pragma unroll
    for (int j = 0; j < BN; ++j) stg[r * (BN + 1) + j] = acc[j];
  }
  __syncthreads();
  if (all_ok) epilogue(ep, stg, m0, n0, M, N, b, lower, err);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

typedef CUresult (*PFN_encodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

PFN_encodeTiled get_encode() {
  static PFN_encodeTiled fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_encodeTiled>(p);
  }
  return fn;
}

bool make_map(CUtensorMap* map, const void* ptr, int rows, int K, int ld, int batch) {
  PFN_encodeTiled enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)ld * 2 * rows};
  cuuint32_t box[3] = {BK, BM, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, batch > 0 ? 3 : 2, const_cast<void*>(ptr), dims, strides,
                   box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

int tc_ld(int K) { return (K + 7) / 8 * 8; }

cudaError_t tc_gemm_ex(const TcOperand& A, int batch, const TcOperand& B, int b_batched, int nsplit, int M, int N,
                       int K, int lower, const TcEpi& ep, int* err, cudaStream_t s) {
  const int ld = tc_ld(K);
  TcMaps maps;
  const int bb = b_batched ? batch : 1;
  if (nsplit != 2 && nsplit != 3) return cudaErrorInvalidValue;
  for (int i = 0; i < nsplit; ++i)
    if (!A.p[i] || !B.p[i] || !make_map(&maps.a[i], A.p[i], M, K, ld, batch) ||
        !make_map(&maps.b[i], B.p[i], N, K, ld, bb))
      return cudaErrorInvalidValue;
  const int nbm = (M + BM - 1) / BM, nbn = (N + BN - 1) / BN;
  const int tiles = lower ? nbm * (nbm + 1) / 2 : nbm * nbn;
  dim3 grid(tiles, batch);
  if (nsplit == 2) {
    static bool attr = false;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           TcCfg<2>::SMEM_BYTES);
      if (e != cudaSuccess) return e;
      attr = true;
    }
    tc_gemm_kernel<2><<<grid, THREADS, TcCfg<2>::SMEM_BYTES, s>>>(maps, M, N, K, lower, b_batched, ep, err);
  } else {
    static bool attr = false;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           TcCfg<3>::SMEM_BYTES);
      if (e != cudaSuccess) return e;
      attr = true;
    }
    tc_gemm_kernel<3><<<grid, THREADS, TcCfg<3>::SMEM_BYTES, s>>>(maps, M, N, K, lower, b_batched, ep, err);
  }
  return cudaGetLastError();
}

cudaError_t tc_gemm(const __nv_bfloat16* Ahi, const __nv_bfloat16* Alo, int batch, const __nv_bfloat16* Bhi,
                    const __nv_bfloat16* Blo, int M, int N, int K, int lower, int mode_even, int mode_odd, float* out,
                    int* err, cudaStream_t s) {
  TcEpi ep{};
  ep.kind = TC_EPI_STORE;
  ep.mode_even = mode_even;
  ep.mode_odd = mode_odd;
  ep.out = out;
  ep.out_bstride = (long)M * N;
  ep.ldo = N;
  const TcOperand a{{Ahi, Alo, nullptr}}, bo{{Bhi, Blo, nullptr}};
  return tc_gemm_ex(a, batch, bo, 0, 2, M, N, K, lower, ep, err, s);
}

// B^T split: out[k][m] = B[m][k] as BF16 hi/lo, rows of length tc_ld(M).  32 x 32 tiles through shared memory.
__global__ void transpose_split_kernel(const float* __restrict__ B, int M, int K, long ldb, int ld,
                                       __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                                       __nv_bfloat16* __restrict__ lo2) {
  __shared__ float t[32][33];
  const int k0 = blockIdx.x * 32, m0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int m = m0 + r, k = k0 + threadIdx.x;
    t[r][threadIdx.x] = (m < M && k < K) ? B[(long)m * ldb + k] : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r, m = m0 + threadIdx.x;
    if (k < K && m < ld) split_store(m < M ? t[threadIdx.x][r] : 0.f, hi, lo, (long)k * ld + m, lo2);
  }
}

__global__ void split_rows_kernel(const float* __restrict__ src, int cols, int lds, __nv_bfloat16* __restrict__ hi,
                                  __nv_bfloat16* __restrict__ lo, __nv_bfloat16* __restrict__ lo2, int ldh) {
  const long r = blockIdx.y + (long)blockIdx.z * gridDim.y;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ldh; c += gridDim.x * blockDim.x)
    split_store(c < cols ? src[r * lds + c] : 0.f, hi, lo, r * ldh + c, lo2);
}

cudaError_t tc_split_rows(const float* src, int rows, int cols, int lds, __nv_bfloat16* hi, __nv_bfloat16* lo,
                          cudaStream_t s, __nv_bfloat16* lo2) {
  const int ldh = tc_ld(cols);
  if (rows <= 0) return cudaSuccess;
  int gy = rows, gz = 1;
  while (gy > 65535) { gz *= 2; gy = (rows + gz - 1) / gz; }
  if ((long)gy * gz != rows) {
    // rows not a multiple of the z split: run the tail separately
    const int main = (rows / gz) * gz;
    if (main > 0) split_rows_kernel<<<dim3((ldh + 255) / 256, main / gz, gz), 256, 0, s>>>(src, cols, lds, hi, lo, lo2, ldh);
    const int tail = rows - main;
    split_rows_kernel<<<dim3((ldh + 255) / 256, tail, 1), 256, 0, s>>>(src + (long)main * lds, cols, lds,
                                                                     hi + (long)main * ldh, lo + (long)main * ldh,
                                                                     lo2 ? lo2 + (long)main * ldh : nullptr, ldh);
    return cudaGetLastError();
  }
  split_rows_kernel<<<dim3((ldh + 255) / 256, gy, gz), 256, 0, s>>>(src, cols, lds, hi, lo, lo2, ldh);
  return cudaGetLastError();
}

// Power iterations for the spectrum of SPD matrices A_b (n x n FP32, batch stride n*n), many CTAs per matrix:
//   gemv:      y_b = A_b v_b (mode 0)  or  y_b = s_b v_b - A_b v_b (mode 1), one warp per row;
//   normalise: q_b = v_b . y_b (the Rayleigh quotient of the unit vector v_b), v_b = y_b / |y_b|.
__global__ void spec_gemv_kernel(const float* __restrict__ A, int n, const float* __restrict__ v,
                                 const float* __restrict__ shift, int mode, float* __restrict__ y) {
  const int b = blockIdx.y, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + wid;
  if (r >= n) return;
  const float* Ar = A + ((long)b * n + r) * n;
  const float* vb = v + (long)b * n;
  float a = 0.f;
  for (int c = lane; c < n; c += 32) a += Ar[c] * vb[c];
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (lane == 0) y[(long)b * n + r] = mode ? shift[b] * vb[r] - a : a;
}

__global__ void spec_normalise_kernel(int n, float* __restrict__ v, const float* __restrict__ y,
                                      float* __restrict__ q) {
  __shared__ float red[2][32];
  const int b = blockIdx.x;
  float* vb = v + (long)b * n;
  const float* yb = y + (long)b * n;
  float yy = 0.f, vy = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    yy += yb[i] * yb[i];
    vy += vb[i] * yb[i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    yy += __shfl_xor_sync(0xffffffffu, yy, o);
    vy += __shfl_xor_sync(0xffffffffu, vy, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = yy;
    red[1][threadIdx.x >> 5] = vy;
  }
  __syncthreads();
  float tyy = 0.f, tvy = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    tyy += red[0][w];
    tvy += red[1][w];
  }
  __syncthreads();
  const float inv = tyy > 0.f ? rsqrtf(tyy) : 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) vb[i] = yb[i] * inv;
  if (threadIdx.x == 0) q[b] = tvy;
}

__global__ void spec_start_kernel(int n, int batch, float* __restrict__ v) {
  const long N = (long)n * batch;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x)
    v[i] = rsqrtf((float)n) * (1.f + 0.25f * (float)((i % n) & 1));   // not orthogonal to any eigenvector
}

__global__ void spec_shift_kernel(int batch, const float* __restrict__ hi, float pad, float* __restrict__ s) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < batch) s[b] = pad * hi[b];
}

cudaError_t tc_spectrum_bounds(const float* A, int n, int batch, int iters, float pad, float* hi, float* lo,
                               float* shift, float* v, float* y, cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  const dim3 gg((n + 7) / 8, batch);
  for (int phase = 0; phase < 2; ++phase) {
    spec_start_kernel<<<256, 256, 0, s>>>(n, batch, v);
    if (phase == 1) spec_shift_kernel<<<(batch + 255) / 256, 256, 0, s>>>(batch, hi, pad, shift);
    for (int it = 0; it < iters; ++it) {
      spec_gemv_kernel<<<gg, 256, 0, s>>>(A, n, v, shift, phase, y);
      spec_normalise_kernel<<<batch, 1024, 0, s>>>(n, v, y, phase == 0 ? hi : lo);
    }
  }
  return cudaGetLastError();
}

__global__ void ns_init_kernel(const float* __restrict__ A, int n, const float* __restrict__ ab, float* __restrict__ X,
                               __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                               __nv_bfloat16* __restrict__ lo2, int ldh) {
  const int r = blockIdx.y, b = blockIdx.z;
  const float a = ab[b];
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ldh; c += gridDim.x * blockDim.x) {
    float y = 0.f;
    if (c < n) {
      y = -a * a * A[((long)b * n + r) * n + c] + (r == c ? 2.f * a : 0.f);
      X[((long)b * n + r) * n + c] = y;
    }
    split_store(y, hi, lo, ((long)b * n + r) * ldh + c, lo2);
  }
}

cudaError_t tc_ns_init(const float* A, int n, int batch, const float* ab, float* X, __nv_bfloat16* hi,
                       __nv_bfloat16* lo, cudaStream_t s, __nv_bfloat16* lo2) {
  const int ldh = tc_ld(n);
  dim3 grid((ldh + 255) / 256, n, batch);
  if (batch > 0) ns_init_kernel<<<grid, 256, 0, s>>>(A, n, ab, X, hi, lo, lo2, ldh);
  return cudaGetLastError();
}

// Y_b = (X_b + X_b^T)/2 (FP32, out of place) and its split parts; one thread per element.
__global__ void sym_split_kernel(const float* __restrict__ X, int n, float* __restrict__ Y, __nv_bfloat16* __restrict__ hi,
                                 __nv_bfloat16* __restrict__ lo, __nv_bfloat16* __restrict__ lo2, int ldh) {
  const int r = blockIdx.y, b = blockIdx.z;
  const float* Xb = X + (long)b * n * n;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ldh; c += gridDim.x * blockDim.x) {
    float v = 0.f;
    if (c < n) {
      v = 0.5f * (Xb[(long)r * n + c] + Xb[(long)c * n + r]);
      Y[((long)b * n + r) * n + c] = v;
    }
    split_store(v, hi, lo, ((long)b * n + r) * ldh + c, lo2);
  }
}

cudaError_t tc_sym_split(const float* X, int n, int batch, float* Y, __nv_bfloat16* hi, __nv_bfloat16* lo,
                         __nv_bfloat16* lo2, cudaStream_t s) {
  const int ldh = tc_ld(n);
  dim3 grid((ldh + 255) / 256, n, batch);
  if (batch > 0) sym_split_kernel<<<grid, 256, 0, s>>>(X, n, Y, hi, lo, lo2, ldh);
  return cudaGetLastError();
}

cudaError_t tc_transpose_split(const float* B, int M, int K, __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t s,
                               __nv_bfloat16* lo2, long ldb) {
  const int ld = tc_ld(M);
  dim3 grid((K + 31) / 32, (ld + 31) / 32);
  transpose_split_kernel<<<grid, dim3(32, 8), 0, s>>>(B, M, K, ldb > 0 ? ldb : K, ld, hi, lo, lo2);
  return cudaGetLastError();
}

}  // namespace gw
