/*
 * philox.c -- CPU ORACLE (test infrastructure only): counter-based shot
 * sampling from the DEM.
 *
 * Philox4x32-10 is written from its published definition (Salmon, Moraes,
 * Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten
 * rounds of two 32x32->64 multiplications by 0xD2511F53 and 0xCD9E8D57 with
 * the Weyl key schedule 0x9E3779B9, 0xBB67AE85.
 *
 * Shot s fires DEM column c iff u < round(p_c 2^32), u = word (c mod 4) of
 * Philox(counter = (c / 4, s_lo, s_hi, 0), key = (seed_lo, seed_hi)).  The
 * shot's detector and observable bits are the XOR of the fired columns
 * (s = H_circ e, l = L e; Sec. III).  Columns without detectors (undetectable
 * logical faults) are sampled too.
 */
#include "qdo.h"
#include <math.h>
#include <string.h>

const int* qdo__col_ptr(const qdo_dem* d);
const int* qdo__col_dets(const qdo_dem* d);
const uint32_t* qdo__col_obs(const qdo_dem* d);
const double* qdo__col_p(const qdo_dem* d);
int qdo__ncols(const qdo_dem* d);
int qdo__ndet(const qdo_dem* d);

void qdo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Firing threshold of a column: round(p 2^32), saturated. */
static uint32_t threshold(double p) {
  double t = floor(p * 4294967296.0 + 0.5);
  if (t >= 4294967295.0) return 0xFFFFFFFFu;
  if (t <= 0.0) return 0u;
  return (uint32_t)t;
}

int qdo_sample(const qdo_dem* d, uint64_t seed, uint64_t shot_offset, int64_t n_shots,
               uint32_t* det_bits, uint32_t* obs_bits) {
  int nc = qdo__ncols(d), ndet = qdo__ndet(d);
  int dw = (ndet + 31) / 32;
  const int* cp = qdo__col_ptr(d);
  const int* cd = qdo__col_dets(d);
  const uint32_t* co = qdo__col_obs(d);
  const double* pr = qdo__col_p(d);
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int64_t s = 0; s < n_shots; ++s) {
    uint64_t shot = shot_offset + (uint64_t)s;
    uint32_t* db = det_bits + s * dw;
    memset(db, 0, sizeof(uint32_t) * dw);
    uint32_t ob = 0;
    uint32_t u[4];
    for (int c = 0; c < nc; ++c) {
      if ((c & 3) == 0) {
        uint32_t ctr[4] = {(uint32_t)(c >> 2), (uint32_t)shot, (uint32_t)(shot >> 32), 0u};
        qdo_philox4x32_10(ctr, key, u);
      }
      if (u[c & 3] < threshold(pr[c])) {
        for (int e = cp[c]; e < cp[c + 1]; ++e) db[cd[e] >> 5] ^= 1u << (cd[e] & 31);
        ob ^= co[c];
      }
    }
    obs_bits[s] = ob;
  }
  return 0;
}
