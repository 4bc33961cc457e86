/*
 * Seeded synthetic inputs for the CD-G0W0 path: the fitted three-index
 * tensor B_{P,pq} of water-cluster-shaped systems.
 *
 * This file holds no arithmetic of the GW method.  It draws one normal
 * variate per element from a counter-based generator, so any slice of the
 * symmetric tensor (the occupied-virtual block B_ia or the target rows
 * B_nm) can be produced without forming the full N_aux x N_bas^2 tensor,
 * and the two slices agree wherever they overlap (B_{P,na} = B_{P,an}).
 *
 * Generator: Philox4x32 with 10 rounds, as published by Salmon, Moraes,
 * Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11).
 * Counter = (P, min(p,q), max(p,q), 0), key = (seed low 32 bits, seed high
 * 32 bits xor stream).  Words 0,1 give a 53-bit uniform u1 in (0,1), words
 * 2,3 give u2; the normal variate is the first Box-Muller output
 * sqrt(-2 ln u1) cos(2 pi u2), scaled by sigma.
 */
#include <math.h>
#include <stdint.h>

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u
#define SYNTH_STREAM_B 0x42504951u

void synth_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += PHILOX_W0; k1 += PHILOX_W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static inline double unit53(uint32_t a, uint32_t b) {
  uint64_t u = (((uint64_t)a << 32) | (uint64_t)b) >> 11;      /* [0, 2^53) */
  return ((double)u + 0.5) * (1.0 / 9007199254740992.0);        /* (0, 1) */
}

static inline double normal_at(uint64_t seed, uint32_t P, uint32_t p, uint32_t q) {
  uint32_t lo = p < q ? p : q, hi = p < q ? q : p;
  uint32_t ctr[4] = {P, lo, hi, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ SYNTH_STREAM_B};
  uint32_t w[4];
  synth_philox4x32_10(ctr, key, w);
  double u1 = unit53(w[0], w[1]), u2 = unit53(w[2], w[3]);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* Rows P0 .. P0 + n_rows - 1 of B_ia: out[P - P0][i*n_virt + a] = sigma * N(seed; P, i, n_occ + a). */
void synth_b_ia_rows(uint64_t seed, double sigma, int P0, int n_rows, int n_occ, int n_virt, double* out) {
  long n_ov = (long)n_occ * n_virt;
#pragma omp parallel for schedule(static)
  for (long r = 0; r < n_rows; ++r)
    for (int i = 0; i < n_occ; ++i)
      for (int a = 0; a < n_virt; ++a)
        out[r * n_ov + (long)i * n_virt + a] =
            sigma * normal_at(seed, (uint32_t)(P0 + r), (uint32_t)i, (uint32_t)(n_occ + a));
}

/* B_ia[P][i*n_virt + a] = sigma * N(seed; P, i, n_occ + a). */
void synth_b_ia(uint64_t seed, double sigma, int n_aux, int n_occ, int n_virt, double* out) {
  synth_b_ia_rows(seed, sigma, 0, n_aux, n_occ, n_virt, out);
}

/* B_nm[t][m][P] = sigma * N(seed; P, targets[t], m) for m in [0, n_bas). */
void synth_b_nm(uint64_t seed, double sigma, int n_aux, int n_bas, const int* targets, int n_t,
                double* out) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int t = 0; t < n_t; ++t)
    for (int m = 0; m < n_bas; ++m)
      for (int P = 0; P < n_aux; ++P)
        out[((long)t * n_bas + m) * n_aux + P] =
            sigma * normal_at(seed, (uint32_t)P, (uint32_t)targets[t], (uint32_t)m);
}
