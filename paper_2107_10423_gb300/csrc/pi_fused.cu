// Weighted symmetric rank-K products on the tcgen05 tensor cores with the weight applied inside the kernel:
//
//   out_b = f( B diag(w_b) B^T ),   B = B_ia [n][K] (FP32), w_b = row b of a weight table [nb][ldw] (FP32),
//
// for every batch entry b, lower-triangular 128 x 128 tiles mirrored into the upper triangle.  This is
//   * Pi(i xi) on the imaginary grid (Sec. 3.3, equation after "wauxbas"): w = -4 D_ia/(D_ia^2 + xi^2);
//   * the dense real-axis Pi(x) of the residue fallback (same section, Pi(z) with +i eta in both pole terms):
//     w = Re c(x) and Im c(x), c = 2[1/(x - D + i eta) + 1/(-x - D + i eta)], as the two entries of one pair;
//   * the difference-form products Pi(i xi) - Pi(0): w = 4 xi^2/(D (D^2 + xi^2)).
//
// Design (one CTA per SM, persistent over work items = (lower tile, pair of batch entries)):
//   * TMA streams, per 32-wide k-block, the FP32 rows of the weighted side (128 x 32) with the two weight rows
//     (2 x 32) into a 4-stage A ring that the transform releases, and the BF16 hi/lo tiles of the unweighted side
//     (2 x 128 x 32) into a 3-stage S ring whose stages also hold the transformed tiles: one barrier tells the
//     tensor core that a stage's B tiles have landed and its transformed tiles are written, and one commit frees
//     both, so the issuing thread does one wait and one commit per k-block.
//   * Two transform warpgroups (two threads per row) multiply the FP32 rows by the weights of both entries and
//     splits the products into BF16 hi/lo tiles (64-byte swizzle, the tensor core's K-major layout) in a
//     3-stage ring.  The weight never round-trips through HBM and the source tile serves both entries, which
//     halves the L2 bytes per tensor-core flop against one entry per pass.
//   * One thread issues tcgen05.mma (M128 N128 K16, BF16 in, FP32 accumulate in TMEM): hi*hi + hi*lo + lo*hi.
//   * Every CHUNK = 4 k-blocks an entry's TMEM partial is added (round to nearest) into its FP32 sum, also kept
//     in TMEM, by the drain warpgroup, so no partial runs through more than 24 tensor-core accumulates.  The two
//     entries' chunks are staggered by one k-block: while one entry's partial drains, the tensor core works on the
//     other entry.
//   * TMEM: partials of entries 0/1 in columns [0, 256), FP32 sums in [256, 512).
// Every mbarrier wait is bounded; on timeout the kernel records a code in *err, stops every role, waits for its
// copies and tensor-core work in flight, frees TMEM and returns.
#include "pi_tc.cuh"
#include "tc_ptx.cuh"

#include <cuda.h>
#include <cuda_bf16.h>
#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

namespace gw {
namespace {
using namespace ptx;

constexpr int BM = 128, BK = 32;
constexpr int A_STAGES = 4, S_STAGES = 3;
constexpr int A_BYTES = BM * BK * 4;            // FP32 rows of the weighted side: 16 KiB
constexpr int W_OFF = A_BYTES;                  // the two weight rows [2][BK] FP32 follow the FP32 tile
constexpr int AS_BYTES = A_BYTES + 1024;        // 17 KiB per A stage (keeps every stage 1 KiB aligned)
constexpr int H_BYTES = BM * BK * 2;            // one BF16 tile (128 rows x 64 bytes): 8 KiB
// S stage: the BF16 hi/lo tiles of the unweighted side (TMA), then the transformed tiles [entry][hi, lo]
constexpr int ST_OFF = 2 * H_BYTES;
constexpr int SS_BYTES = 6 * H_BYTES;           // 48 KiB
constexpr int A_TX = A_BYTES + 2 * BK * 4;
constexpr int B_TX = 2 * H_BYTES;
// mbarrier indices: A ring full/empty, S ring full/empty, accumulators, final
constexpr int BAR_AF = 0, BAR_AE = BAR_AF + A_STAGES, BAR_SF = BAR_AE + A_STAGES, BAR_SE = BAR_SF + S_STAGES,
              BAR_ACCF = BAR_SE + S_STAGES, BAR_ACCE = BAR_ACCF + 2, BAR_FIN = BAR_ACCE + 2, N_BARS = BAR_FIN + 1;
static_assert(N_BARS * 8 + 4 <= 256, "barrier area");
constexpr int SMEM_BYTES = A_STAGES * AS_BYTES + S_STAGES * SS_BYTES + 256 + 1024;
static_assert(SMEM_BYTES <= 232448, "shared memory per block");
constexpr int THREADS = 448;                    // warps 0-3 drain + epilogue, 4-11 transform, 12 TMA, 13 MMA
constexpr int TR_WARPS = 8;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t SBO64 = 8 * 64;              // 8-row groups of 64-byte rows
constexpr uint32_t SWZ64 = 4;                   // descriptor swizzle mode: 64-byte
// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, N = 128, M = 128
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(128 >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

struct PfMaps {
  CUtensorMap a, bh, bl, w;
};

// Chunk bookkeeping of entry f at k-block kb (nk k-blocks per item), CHUNK k-blocks per chunk.  Entry 0's chunks
// start at multiples of CHUNK, entry 1's half a chunk later (its first chunk is CHUNK/2 long); both end at the last
// k-block.  The staggering means that the two entries never drain at the same k-block.
constexpr int CHUNK = 4;
__device__ __forceinline__ bool chunk_first(int f, int kb) {
  return f == 0 ? (kb % CHUNK == 0) : (kb == 0 || kb % CHUNK == CHUNK / 2);
}
__device__ __forceinline__ bool chunk_last(int f, int kb, int nk) {
  return kb == nk - 1 || (f == 0 ? (kb % CHUNK == CHUNK - 1) : (kb % CHUNK == CHUNK / 2 - 1));
}
// The first chunk of the item ends at k-block kb (no running sum to add yet).
__device__ __forceinline__ bool chunk_first_of_item(int f, int kb) { return kb < (f == 0 ? CHUNK : CHUNK / 2); }
// Issue order within k-block kb: the entry that does not start a chunk first (the other one may still be
// draining its previous partial).
__device__ __forceinline__ int entry_at(int kb, int o) { return (kb % CHUNK == 0 && kb > 0) ? 1 - o : o; }

// Work item -> (lower tile (bm, bn), entry pair, K split ks).
__device__ __forceinline__ void decode_item(long item, int n_tiles, int ksplit, int& bm, int& bn, int& pair,
                                            int& ks) {
  ks = (int)(item % ksplit);
  item /= ksplit;
  pair = (int)(item / n_tiles);
  const int t = (int)(item % n_tiles);
  int m = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((m + 1) * (m + 2) / 2 <= t) ++m;
  while (m * (m + 1) / 2 > t) --m;
  bm = m;
  bn = t - m * (m + 1) / 2;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// With ksplit > 1 the k-blocks of every (tile, pair) are cut into ksplit contiguous ranges, each a work item of its
// own, which writes its raw partial product (lower and mirrored) to part [ksplit][nb][n][n]; pf_reduce_kernel
// then adds the partials in a fixed order (deterministic) and applies the output mode.
__global__ void __launch_bounds__(THREADS, 1)
    pi_fused_kernel(const __grid_constant__ PfMaps maps, int n, int K, int nb, int mode_even, int mode_odd,
                    float* __restrict__ out, long out_bstride, int ldo, int ksplit, float* __restrict__ part,
                    long out_limit, long part_limit, int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* smem = smem_raw + (base - raw);
  constexpr int S_OFF = A_STAGES * AS_BYTES, BAR_OFF = S_OFF + S_STAGES * SS_BYTES;
  const uint32_t s0 = base + S_OFF;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + BAR_OFF);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + N_BARS);
  const uint32_t bar0 = base + BAR_OFF;
  // barrier i at bar0 + 8 i (addresses computed, not held in an indexed array)
  auto bar = [bar0](int i) { return bar0 + 8u * (uint32_t)i; };
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nbt = (n + BM - 1) / BM;
  const int n_tiles = nbt * (nbt + 1) / 2;
  const int n_pairs = (nb + 1) / 2;
  const long items = (long)n_tiles * n_pairs * ksplit;
  const int nk = (K + BK - 1) / BK;

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < A_STAGES; ++s) {
      mbar_init(bar(BAR_AF + s), 1);
      mbar_init(bar(BAR_AE + s), TR_WARPS);    // one arrival per transform warp
    }
    for (int s = 0; s < S_STAGES; ++s) {
      mbar_init(bar(BAR_SF + s), TR_WARPS + 1);   // the producer's expect_tx arrival + one per transform warp
      mbar_init(bar(BAR_SE + s), 1);              // the MMA thread's commit
    }
    for (int f = 0; f < 2; ++f) {
      mbar_init(bar(BAR_ACCF + f), 1);
      mbar_init(bar(BAR_ACCE + f), 4);         // one arrival per drain warp
    }
    mbar_init(bar(BAR_FIN), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_async_smem();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 12) {
    if (lane == 0) {
      // ------------------------------------------------------------ TMA producer
      // A ring (FP32 rows + weights): released by the transform warps; B ring (BF16 hi/lo of the unweighted
      // side): released by the tensor core.  The A ring therefore refills as soon as a k-block is transformed.
      // ring positions kept as stage indices and phase bits (no divisions in the loop)
      long issued_a = 0, issued_s = 0;
      uint32_t sa = 0, pa = 0, ss = 0, ps = 0;
      bool a_wrapped = false, s_wrapped = false;
      bool ok = true;
      for (long it = blockIdx.x; it < items && ok; it += gridDim.x) {
        int bm, bn, pair, ks;
        decode_item(it, n_tiles, ksplit, bm, bn, pair, ks);
        const int kb0 = (int)((long)nk * ks / ksplit), nki = (int)((long)nk * (ks + 1) / ksplit) - kb0;
        for (int kb = 0; kb < nki; ++kb) {
          const int kx = (kb0 + kb) * BK;
          if (a_wrapped && !mbar_wait(bar(BAR_AE + sa), pa ^ 1u, err, 11)) { ok = false; break; }
          if (*(volatile int*)&s_abort) { ok = false; break; }
          const uint32_t as = base + sa * AS_BYTES;
          mbar_expect_tx(bar(BAR_AF + sa), A_TX);
          tma_load_2d(as, &maps.a, kx, bm * BM, bar(BAR_AF + sa));
          tma_load_2d(as + W_OFF, &maps.w, kx, 2 * pair, bar(BAR_AF + sa));
          ++issued_a;
          if (++sa == A_STAGES) { sa = 0; pa ^= 1u; a_wrapped = true; }
          if (s_wrapped && !mbar_wait(bar(BAR_SE + ss), ps ^ 1u, err, 13)) { ok = false; break; }
          if (*(volatile int*)&s_abort) { ok = false; break; }
          const uint32_t st = s0 + ss * SS_BYTES;
          mbar_expect_tx(bar(BAR_SF + ss), B_TX);
          tma_load_2d(st, &maps.bh, kx, bn * BM, bar(BAR_SF + ss));
          tma_load_2d(st + H_BYTES, &maps.bl, kx, bn * BM, bar(BAR_SF + ss));
          ++issued_s;
          if (++ss == S_STAGES) { ss = 0; ps ^= 1u; s_wrapped = true; }
        }
      }
      if (!ok) {
        s_abort = 1;
        // wait for the copies that may still be in flight (the latest phase of each stage; an S stage's phase
        // also needs the transform's arrivals, so that wait may run out after the copy itself has landed)
        for (long q = issued_a > A_STAGES ? issued_a - A_STAGES : 0; q < issued_a; ++q)
          mbar_wait(bar(BAR_AF + (int)(q % A_STAGES)), (uint32_t)((q / A_STAGES) & 1), err, 12);
        for (long q = issued_s > S_STAGES ? issued_s - S_STAGES : 0; q < issued_s; ++q)
          mbar_wait(bar(BAR_SF + (int)(q % S_STAGES)), (uint32_t)((q / S_STAGES) & 1), err, 14);
      }
    }
  } else if (warp == 13) {
    if (lane == 0) {
      // ------------------------------------------------------------ MMA issuer
      // The issuing thread's work between MMAs limits the tensor core's throughput as soon as it exceeds one MMA's
      // 64 cycles, so the loop keeps it minimal: ring positions as stage indices and phase bits, and shared-memory
      // descriptors formed once and advanced by adding the byte offset >> 4 to their start-address field.
      uint32_t ss = 0, ps = 0;
      uint32_t cf0 = 0, cf1 = 0;           // chunks started per entry
      const uint64_t dS = sdesc(s0, SBO64, SWZ64);
      bool ok = true;
      for (long it = blockIdx.x; it < items && ok; it += gridDim.x) {
        int bm, bn, pair, ks;
        decode_item(it, n_tiles, ksplit, bm, bn, pair, ks);
        const int nf = min(2, nb - 2 * pair);
        const int nki = (int)((long)nk * (ks + 1) / ksplit) - (int)((long)nk * ks / ksplit);
        for (int kb = 0; kb < nki && ok; ++kb) {
          // one wait: the stage's B tiles have landed and every transform warp has written its tiles
          if (*(volatile int*)&s_abort || !mbar_wait(bar(BAR_SF + ss), ps, err, 21)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t bh = dS + (uint64_t)((ss * SS_BYTES) >> 4), bl = bh + (uint64_t)(H_BYTES >> 4);
          const uint64_t td = bh + (uint64_t)(ST_OFF >> 4);
#pragma unroll
          for (int o = 0; o < 2; ++o) {
            const int f = entry_at(kb, o);
            if (f >= nf) continue;
            const bool first = chunk_first(f, kb);
            if (first) {
              const uint32_t cf = f ? cf1 : cf0;
              if (cf > 0 && !mbar_wait(bar(BAR_ACCE + f), (cf - 1) & 1u, err, 23)) { ok = false; break; }
              if (f) ++cf1; else ++cf0;
              tc_fence_after();
            }
            const uint32_t d = tmem + (uint32_t)(f * 128);
            const uint64_t ah = td + (uint64_t)((2 * f * H_BYTES) >> 4), al = ah + (uint64_t)(H_BYTES >> 4);
#pragma unroll
            for (int k = 0; k < BK / 16; ++k) {        // K16 step k: 32 bytes further along each 64-byte row
              const uint64_t o2 = (uint64_t)(2 * k);
              mma_bf16(d, ah + o2, bh + o2, IDESC, (first && k == 0) ? 0u : 1u);
              mma_bf16(d, ah + o2, bl + o2, IDESC, 1u);
              mma_bf16(d, al + o2, bh + o2, IDESC, 1u);
            }
            if (chunk_last(f, kb, nki)) mma_commit(bar(BAR_ACCF + f));
          }
          if (!ok) break;
          mma_commit(bar(BAR_SE + ss));        // frees the stage's B tiles and transformed tiles together
          if (++ss == S_STAGES) { ss = 0; ps ^= 1u; }
        }
      }
      if (!ok) s_abort = 1;
      // every tensor-core operation issued above has completed once the final barrier flips
      mma_commit(bar(BAR_FIN));
      mbar_wait(bar(BAR_FIN), 0, err, 24);
    }
  } else if (warp >= 4) {
    // -------------------------------------------------------------- transform: two threads per row of the tile,
    // each over 16 of the k-block's 32 columns
    const int t = threadIdx.x - 128;
    const int r = t & (BM - 1), h = t >> 7;
    uint32_t sa = 0, pa = 0, ss = 0, ps = 0;
    bool s_wrapped = false;
    bool ok = true;
    for (long it = blockIdx.x; it < items && ok; it += gridDim.x) {
      int bm, bn, pair, ks;
      decode_item(it, n_tiles, ksplit, bm, bn, pair, ks);
      const int nf = min(2, nb - 2 * pair);
      const int nki = (int)((long)nk * (ks + 1) / ksplit) - (int)((long)nk * ks / ksplit);
      for (int kb = 0; kb < nki; ++kb) {
        bool w_ok = !*(volatile int*)&s_abort && mbar_wait(bar(BAR_AF + sa), pa, err, 31);
        if (w_ok && s_wrapped) w_ok = mbar_wait(bar(BAR_SE + ss), ps ^ 1u, err, 32);
        if (!__all_sync(0xffffffffu, w_ok)) { ok = false; break; }
        const uint8_t* sp = smem + sa * AS_BYTES;
        const float* wrow = reinterpret_cast<const float*>(sp + W_OFF);
        constexpr int HK = BK / 2;
        float a[HK];
#pragma unroll
        for (int c = 0; c < HK / 4; ++c) {   // 128-byte swizzle: 16-byte chunk cc of row r sits at cc ^ (r & 7)
          const int cc = h * (HK / 4) + c;
          const float4 v = *reinterpret_cast<const float4*>(sp + r * 128 + ((cc ^ (r & 7)) << 4));
          a[4 * c] = v.x;
          a[4 * c + 1] = v.y;
          a[4 * c + 2] = v.z;
          a[4 * c + 3] = v.w;
        }
        uint8_t* tp = smem + S_OFF + ss * SS_BYTES + ST_OFF;
        for (int f = 0; f < nf; ++f) {
          float wv[HK];                        // the entry's weights for these columns (broadcast reads)
#pragma unroll
          for (int c = 0; c < HK / 4; ++c) {
            const float4 q = *reinterpret_cast<const float4*>(wrow + f * BK + h * HK + 4 * c);
            wv[4 * c] = q.x;
            wv[4 * c + 1] = q.y;
            wv[4 * c + 2] = q.z;
            wv[4 * c + 3] = q.w;
          }
#pragma unroll
          for (int jj = 0; jj < HK / 8; ++jj) {  // 64-byte swizzle: 16-byte chunk j of row r sits at j ^ ((r >> 1) & 3)
            const int j = h * (HK / 8) + jj;
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int k = 8 * jj + 2 * e;
              const float v0 = a[k] * wv[k], v1 = a[k + 1] * wv[k + 1];
              hi[e] = pack_bf16(v0, v1);
              const __nv_bfloat162 hh = *reinterpret_cast<const __nv_bfloat162*>(&hi[e]);
              lo[e] = pack_bf16(v0 - __low2float(hh), v1 - __high2float(hh));
            }
            const int off = r * 64 + ((j ^ ((r >> 1) & 3)) << 4);
            *reinterpret_cast<uint4*>(tp + (2 * f) * H_BYTES + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4*>(tp + (2 * f + 1) * H_BYTES + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
          }
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(bar(BAR_SF + ss));
          mbar_arrive(bar(BAR_AE + sa));
        }
        if (++sa == A_STAGES) { sa = 0; pa ^= 1u; }
        if (++ss == S_STAGES) { ss = 0; ps ^= 1u; s_wrapped = true; }
      }
    }
    if (!ok) s_abort = 1;
  } else {
    // -------------------------------------------------------------- drain + epilogue (TMEM lane quarter = warp)
    const int q = warp;
    long gd0 = 0, gd1 = 0;                // drains done per entry
    bool ok = true;
    for (long it = blockIdx.x; it < items && ok; it += gridDim.x) {
      int bm, bn, pair, ks;
      decode_item(it, n_tiles, ksplit, bm, bn, pair, ks);
      const int nf = min(2, nb - 2 * pair);
      const int nki = (int)((long)nk * (ks + 1) / ksplit) - (int)((long)nk * ks / ksplit);
      const int m0 = bm * BM, n0 = bn * BM;
      const int row = m0 + q * 32 + lane;
      for (int kb = 0; kb < nki && ok; ++kb) {
        for (int o = 0; o < 2; ++o) {
          const int f = entry_at(kb, o);
          if (f >= nf || !chunk_last(f, kb, nki)) continue;
          const bool first_of_item = chunk_first_of_item(f, kb);
          const bool final = kb == nki - 1;
          bool w_ok = !*(volatile int*)&s_abort && mbar_wait(bar(BAR_ACCF + f), (uint32_t)((f ? gd1 : gd0) & 1), err, 41);
          if (!__all_sync(0xffffffffu, w_ok)) { ok = false; break; }
          tc_fence_after();
          const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
          const int b = 2 * pair + f;
          // split K: the raw partial goes to its slot of `part` (mode 0, row length n); the reduction applies
          // the mode
          const bool raw = ksplit > 1;
          const int mode = raw ? 0 : ((b & 1) ? mode_odd : mode_even);
          const long ob0 = raw ? ((long)ks * nb + b) * n * n : (long)b * out_bstride;
          float* ob = (raw ? part : out) + ob0;
          const int ld = raw ? n : ldo;
          const long lim = (raw ? part_limit : out_limit) - ob0;   // elements writable from ob
#pragma unroll 1
          for (int c = 0; c < 4; ++c) {
            uint32_t v[32], w[32];
            tmem_ld32(lane_addr + (uint32_t)(f * 128 + c * 32), v);
            if (!first_of_item) tmem_ld32(lane_addr + (uint32_t)(256 + f * 128 + c * 32), w);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const float x = __uint_as_float(v[j]) + (first_of_item ? 0.f : __uint_as_float(w[j]));
              v[j] = __float_as_uint(x);
            }
            if (!final) {
              tmem_st32(lane_addr + (uint32_t)(256 + f * 128 + c * 32), v);
              continue;
            }
            // epilogue: lower element (row, col <= row) in place, mirrored element (col, row) for col < row
            const int c0 = n0 + c * 32;
            if (row < n) {
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                const int col = c0 + j;
                if (col > row || col >= n) continue;
                const float x = __uint_as_float(v[j]);
                const long o = (long)row * ld + col;
                if (o >= lim) { atomicCAS(err, 0, 51); continue; }    // outside the caller's buffer: record, skip
                ob[o] = mode == 0 ? x : (mode == 1 ? ((col == row ? 1.f : 0.f) - x) : -x);
              }
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int col = c0 + j;
              if (row < n && col < row && col < n) {
                const float x = __uint_as_float(v[j]);
                const long o = (long)col * ld + row;
                if (o >= lim) { atomicCAS(err, 0, 52); continue; }
                ob[o] = mode == 0 ? x : -x;
              }
            }
          }
          if (!final) tmem_wait_st();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(bar(BAR_ACCE + f));
          if (f) ++gd1; else ++gd0;
        }
      }
    }
    if (!ok) s_abort = 1;
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// out_b[i][j] = mode(sum_s part[s][b][i][j]) in the fixed order s = 0, 1, ... (split-K reduction).
__global__ void pf_reduce_kernel(const float* __restrict__ part, int ksplit, int nb, int n, int mode_even,
                                 int mode_odd, float* __restrict__ out, long out_bstride, int ldo, long out_limit,
                                 long part_limit, int* __restrict__ err) {
  const long nn = (long)n * n, N = nn * nb;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < N; idx += (long)gridDim.x * blockDim.x) {
    const int b = (int)(idx / nn);
    const long e = idx - (long)b * nn;
    const int i = (int)(e / n), j = (int)(e - (long)i * n);
    if (((long)(ksplit - 1) * nb + b) * nn + e >= part_limit) { atomicCAS(err, 0, 53); continue; }
    float v = 0.f;
    for (int s = 0; s < ksplit; ++s) v += part[((long)s * nb + b) * nn + e];
    const int mode = (b & 1) ? mode_odd : mode_even;
    const long o = (long)b * out_bstride + (long)i * ldo + j;
    if (o >= out_limit) { atomicCAS(err, 0, 54); continue; }
    out[o] = mode == 0 ? v : (mode == 1 ? ((i == j ? 1.f : 0.f) - v) : -v);
  }
}

// w[b][k] for k < K, in FP64 rounded to FP32 (one evaluation per entry and pair).  Kinds: 0 Pi(i xi):
// -4D/(D^2 + xi^2); 1 Re c(x); 2 Im c(x) (broadening eta); 3 unit weight; 4 Pi(i xi) - Pi(0): 4 xi^2/(D (D^2+xi^2)).
__device__ __forceinline__ double pair_weight(int kind, double D, double p, double eta) {
  if (kind == 0) return -4.0 * D / (D * D + p * p);
  if (kind == 3) return 1.0;
  if (kind == 4) return 4.0 * p * p / (D * (D * D + p * p));
  const double a1 = p - D, a2 = -p - D, e2 = eta * eta;
  const double d1 = a1 * a1 + e2, d2 = a2 * a2 + e2;
  if (kind == 1) return 2.0 * (a1 / d1 + a2 / d2);
  return -2.0 * eta * (1.0 / d1 + 1.0 / d2);
}

__global__ void pf_weight_kernel(const double* __restrict__ Dk, int K, const int* __restrict__ kinds,
                                 const double* __restrict__ params, double eta, float* __restrict__ w, int ldw) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
  if (k >= ldw) return;
  w[(long)b * ldw + k] = k < K ? (float)pair_weight(kinds[b], Dk[k], params[b], eta) : 0.f;
}

typedef CUresult (*PFN_encodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

PFN_encodeTiled encoder() {
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

bool map2d(CUtensorMap* map, CUtensorMapDataType dt, int esize, const void* ptr, int cols, int rows, long ld,
           int box_cols, int box_rows, CUtensorMapSwizzle swz) {
  PFN_encodeTiled enc = encoder();
  if (!enc || (reinterpret_cast<uintptr_t>(ptr) & 15) || ((ld * esize) & 15)) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * esize)};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return enc(map, dt, 2, const_cast<void*>(ptr), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
      n = 148;
  }
  return n;
}

}  // namespace

int pf_ldw(int K) { return (K + 3) / 4 * 4; }

cudaError_t tc_pair_weights(const double* Dk, int K, const int* kinds, const double* params, double eta, int nb,
                            float* w, cudaStream_t s) {
  const int ldw = pf_ldw(K);
  if (nb <= 0) return cudaSuccess;
  pf_weight_kernel<<<dim3((ldw + 255) / 256, nb), 256, 0, s>>>(Dk, K, kinds, params, eta, w, ldw);
  return cudaGetLastError();
}

namespace {

cudaError_t pf_launch(const PfMaps& maps, int n, int K, int nb, int mode_even, int mode_odd, float* out,
                      long out_bstride, int ldo, int ksplit, float* part, size_t part_bytes, int* err, cudaStream_t s,
                      int max_ctas) {
  const int nbt = (n + BM - 1) / BM;
  const long items = (long)nbt * (nbt + 1) / 2 * ((nb + 1) / 2) * ksplit;
  int grid = sm_count();
  if (max_ctas > 0 && max_ctas < grid) grid = max_ctas;
  if (items < grid) grid = (int)items;
  // elements the kernels may write: the nb output matrices, and the capacity of the partials buffer
  const long out_limit = (long)(nb - 1) * out_bstride + (long)n * ldo;
  const long part_limit = part ? (long)(part_bytes / sizeof(float)) : 0;
  if (ksplit > 1 && (long)ksplit * nb * n * n > part_limit) return cudaErrorInvalidValue;
  pi_fused_kernel<<<grid, THREADS, SMEM_BYTES, s>>>(maps, n, K, nb, mode_even, mode_odd, out, out_bstride, ldo,
                                                     ksplit, part, out_limit, part_limit, err);
  if (ksplit > 1) {
    const long N = (long)n * n * nb;
    pf_reduce_kernel<<<(int)std::min<long>((N + 255) / 256, 4096), 256, 0, s>>>(
        part, ksplit, nb, n, mode_even, mode_odd, out, out_bstride, ldo, out_limit, part_limit, err);
  }
  return cudaGetLastError();
}

// Split-K choices measured per problem shape (n, K, nb, grid cap) and largest split the caller's partials buffer
// allows (a choice made with a larger buffer is never reused with a smaller one), kept for the process.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, int> g_tune;

}  // namespace

int tc_pi_fused_ksplit(int n, int K, int nb, int max_ctas, int max_split) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(std::make_tuple(n, K, nb, max_ctas, max_split));
  return it == g_tune.end() ? 0 : it->second;
}

cudaError_t tc_pi_fused(const float* B, long ldb, int n, int K, const float* w, int nb, const __nv_bfloat16* Bhi,
                        const __nv_bfloat16* Blo, int mode_even, int mode_odd, float* out, long out_bstride, int ldo,
                        int* err, cudaStream_t s, int max_ctas, int ksplit, float* part, size_t part_bytes,
                        int* chosen) {
  if (nb <= 0 || n <= 0 || K <= 0) return cudaSuccess;
  PfMaps maps;
  const int ldh = tc_ld(K), ldw = pf_ldw(K);
  if (!map2d(&maps.a, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, B, K, n, ldb, BK, BM, CU_TENSOR_MAP_SWIZZLE_128B) ||
      !map2d(&maps.bh, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Bhi, K, n, ldh, BK, BM, CU_TENSOR_MAP_SWIZZLE_64B) ||
      !map2d(&maps.bl, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Blo, K, n, ldh, BK, BM, CU_TENSOR_MAP_SWIZZLE_64B) ||
      !map2d(&maps.w, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, w, K, nb, ldw, BK, 2, CU_TENSOR_MAP_SWIZZLE_NONE))
    return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(pi_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int nk = (K + BK - 1) / BK;
  const size_t per_split = (size_t)nb * n * n * sizeof(float);
  auto feasible = [&](int ks) {
    return ks == 1 || (part && (size_t)ks * per_split <= part_bytes && nk / ks >= 4);
  };
  if (ksplit > 0) {                        // forced: the largest feasible split not above the request
    while (ksplit > 1 && !feasible(ksplit)) ksplit /= 2;
    if (chosen) *chosen = ksplit;
    return pf_launch(maps, n, K, nb, mode_even, mode_odd, out, out_bstride, ldo, ksplit, part, part_bytes, err, s,
                     max_ctas);
  }
  // Autotuning over the K split: the persistent grid only fills the GPU when (tiles x entry pairs) reaches the SM
  // count, so small problems (few 128-row tiles) split K; each feasible split is timed once per shape (the
  // result of every trial is the same product) and the fastest is kept.
  const int nbt = (n + BM - 1) / BM;
  const long items1 = (long)nbt * (nbt + 1) / 2 * ((nb + 1) / 2);
  std::vector<int> cand{1};
  for (int ks : {2, 4, 8})
    if (items1 * (ks / 2) < 2L * sm_count() && feasible(ks)) cand.push_back(ks);
  const int max_split = cand.back();
  int best = tc_pi_fused_ksplit(n, K, nb, max_ctas, max_split);
  if (best == 0) {
    if (cand.size() == 1) {
      best = 1;
    } else {
      cudaEvent_t e0, e1;
      if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return cudaErrorUnknown;
      float best_ms = 1e30f;
      for (int ks : cand) {
        float ms = 0.f;
        for (int rep = 0; rep < 2; ++rep) {          // the first launch of a configuration warms it up
          cudaEventRecord(e0, s);
          cudaError_t e = pf_launch(maps, n, K, nb, mode_even, mode_odd, out, out_bstride, ldo, ks, part, part_bytes,
                                    err, s, max_ctas);
          cudaEventRecord(e1, s);
          if (e != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); return e; }
          if (cudaEventSynchronize(e1) != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); return cudaErrorUnknown; }
          cudaEventElapsedTime(&ms, e0, e1);
        }
        if (ms < best_ms) { best_ms = ms; best = ks; }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[std::make_tuple(n, K, nb, max_ctas, max_split)] = best;
  }
  if (chosen) *chosen = best;
  return pf_launch(maps, n, K, nb, mode_even, mode_odd, out, out_bstride, ldo, best, part, part_bytes, err, s,
                   max_ctas);
}

}  // namespace gw
