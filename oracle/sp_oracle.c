/*
 * sp_oracle.c -- plain, slow, single-threaded CPU oracle of the SLGA super
 * point detection scheme (Xu, Ding, Hu, "Most memory efficient distributed
 * super points detection on core networks", arXiv 1901.07306).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no header, helper, table or
 * constant generator with the CUDA library: every definition below is
 * restated from the paper on its own.
 *
 * Each function follows the paper's statement step by step:
 *   - Eq. 1 (Sec. 3.1)                 or_tau
 *   - Sec. 3.1 (H1, H2), Sec. 3.3 (H3), Sec. 3.3 (LH_i): or_hash_params, or_mas
 *   - Eq. 2 (Sec. 3.2)                 or_idx
 *   - Eq. 3 (Sec. 3.2)                 or_detect (LP reconstruction)
 *   - Sec. 3.2 constraints 1 and 2     or_check_params
 *   - Sec. 3.1 + Sec. 3.2 + Sec. 3.3   or_update  (per-pair scan)
 *   - Sec. 4.2                         or_merge   (global SEAV/LDCA)
 *   - Sec. 3.2 (HSE, CIdx, CIS, SEU) + Sec. 3.3 (ULDC, Eq. 4): or_detect
 *   - Eq. 4 turned into an integer test on z0: or_z_theta
 *
 * Readings of points where the paper is silent or garbled (they are listed
 * again in the design notes):
 *   - lsb(x) is the index of the lowest set bit of x; lsb(0) = 32.
 *   - the sample test is lsb(H1(oip)) >= tau (Sec. 3.1 writes both "bigger
 *     than" and ">="; we take ">=").
 *   - tau = ceil(log2(theta / 8)), clamped at 0, computed in integers as the
 *     smallest t >= 0 with 8 * 2^t >= theta.
 *   - hash family: Dietzfelbinger's multiply-add-shift,
 *       MAS_{a,b}(x) = floor(((a * x + b) mod 2^64) / 2^32),
 *     a, b drawn from SplitMix64 started at the seed, in the order
 *     H1, H3, LH_0 .. LH_{LR-1}.  H2 = top 3 bits of H1's output.
 *     H3 = top log2(k) bits of MAS_3(oip); LH_i = top log2(LC) bits of
 *     MAS_{LH_i}(hip).
 *   - the overlap constraint (Sec. 3.2, constraint 2) is read as "row i and
 *     row (i+1) mod SR share at least one LP bit", cyclically mod (32 - r).
 *   - a candidate index tuple whose rows disagree on an LP bit they both
 *     cover corresponds to no LP and is dropped.
 *   - "more than theta" at the SEU test is read as weight >= 3, and the
 *     super point test as Est >= theta (Def. 2).
 *   - merging LDCs of one host is bitwise AND (Sec. 3.3); merging sketches
 *     of different watch points is bitwise OR (Sec. 4.2).
 *   - output sorted by ascending IP; est = -k ln(z0 / k); z0 = 0 is flagged
 *     saturated with est = k ln k.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* Parameters, laid out for ctypes.  Independent of the CUDA library's own. */
typedef struct {
  uint32_t r;          /* SEAV: number of RP bits; 2^r SEAs                 */
  uint32_t sr;         /* rows per SEA                                       */
  uint32_t isb[8];     /* index starting bit per row (Def. 3)               */
  uint32_t ibn[8];     /* index bits number per row (Def. 4)                */
  uint32_t k_log2;     /* LDC length k = 2^k_log2 bits                       */
  uint32_t lr;         /* LDCA rows                                          */
  uint32_t lc_log2;    /* LDCA columns LC = 2^lc_log2                        */
  uint32_t theta;      /* super point threshold fixing tau                   */
  uint64_t seed;       /* hash seed                                          */
} or_params;

typedef struct {
  uint32_t ip;
  uint32_t z0;
  double est;
  uint32_t flags;      /* bit 0: saturated LDC union (z0 == 0) */
  uint32_t pad;
} or_candidate;

#define OR_FLAG_SATURATED 1u

/* ---- Eq. 1 ------------------------------------------------------------ */
uint32_t or_tau(uint32_t theta) {
  uint32_t t = 0;
  /* smallest t with 8 * 2^t >= theta; 8 * 2^29 = 2^32 exceeds every theta */
  while (t < 29 && ((uint64_t)8 << t) < (uint64_t)theta) t++;
  return t;
}

/* ---- lsb: index of the least significant set bit, 32 for zero -------- */
uint32_t or_lsb(uint32_t x) {
  uint32_t i;
  if (x == 0) return 32;
  for (i = 0; i < 32; i++)
    if ((x >> i) & 1u) return i;
  return 32;
}

uint32_t or_popcount(uint64_t x) {
  uint32_t c = 0;
  while (x) { c += (uint32_t)(x & 1u); x >>= 1; }
  return c;
}

/* ---- SplitMix64 (Steele, Lea, Flood 2014) ----------------------------- */
uint64_t or_splitmix64(uint64_t *state) {
  uint64_t z;
  *state = *state + 0x9E3779B97F4A7C15ull;
  z = *state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* ---- multiply-add-shift hash (Dietzfelbinger 1996) --------------------- */
uint32_t or_mas(uint64_t a, uint64_t b, uint32_t x) {
  uint64_t v = a * (uint64_t)x + b;   /* arithmetic mod 2^64 */
  return (uint32_t)(v >> 32);
}

/* Draws the (a, b) pairs: index 0 = H1, 1 = H3, 2 + i = LH_i. */
void or_hash_params(uint64_t seed, uint32_t lr, uint64_t *a, uint64_t *b) {
  uint64_t s = seed;
  uint32_t i;
  for (i = 0; i < 2 + lr; i++) {
    a[i] = or_splitmix64(&s);
    b[i] = or_splitmix64(&s);
  }
}

/* top `bits` bits of a 32-bit value (bits = 0 gives 0) */
static uint32_t or_top_bits(uint32_t v, uint32_t bits) {
  if (bits == 0) return 0;
  return v >> (32 - bits);
}

uint32_t or_h1(const uint64_t *a, const uint64_t *b, uint32_t oip) { return or_mas(a[0], b[0], oip); }
uint32_t or_h2(uint32_t h1) { return h1 >> 29; }  /* g = 8 */
uint32_t or_h3(const uint64_t *a, const uint64_t *b, uint32_t k_log2, uint32_t oip) {
  return or_top_bits(or_mas(a[1], b[1], oip), k_log2);
}
uint32_t or_lh(const uint64_t *a, const uint64_t *b, uint32_t lc_log2, uint32_t i, uint32_t hip) {
  return or_top_bits(or_mas(a[2 + i], b[2 + i], hip), lc_log2);
}

/* ---- Sec. 3.2: RP / LP -------------------------------------------------- */
uint32_t or_rp(uint32_t r, uint32_t ip) {
  uint32_t rp = 0, j;
  for (j = 0; j < r; j++) rp |= ((ip >> j) & 1u) << j;
  return rp;
}
uint32_t or_lp(uint32_t r, uint32_t ip) {
  uint32_t lp = 0, j;
  for (j = r; j < 32; j++) lp |= ((ip >> j) & 1u) << (j - r);
  return lp;
}

/* ---- Eq. 2: Idx(i, LP)[j] = LP[(ISB[i] + j) mod (32 - r)] --------------- */
uint32_t or_idx(const or_params *p, uint32_t i, uint32_t lp) {
  uint32_t L = 32 - p->r, idx = 0, j;
  for (j = 0; j < p->ibn[i]; j++) {
    uint32_t bitpos = (p->isb[i] + j) % L;
    idx |= ((lp >> bitpos) & 1u) << j;
  }
  return idx;
}

/* ---- sizes ---------------------------------------------------------------- */
uint64_t or_row_se_count(const or_params *p, uint32_t i) { return (uint64_t)1 << p->ibn[i]; }  /* SC(i) */
uint64_t or_sea_bytes(const or_params *p) {
  uint64_t s = 0; uint32_t i;
  for (i = 0; i < p->sr; i++) s += or_row_se_count(p, i);
  return s;
}
uint64_t or_seav_bytes(const or_params *p) { return ((uint64_t)1 << p->r) * or_sea_bytes(p); }
uint64_t or_ldca_words(const or_params *p) {
  return (uint64_t)p->lr * ((uint64_t)1 << p->lc_log2) * (((uint64_t)1 << p->k_log2) / 32);
}
static uint64_t or_row_offset(const or_params *p, uint32_t i) {
  uint64_t s = 0; uint32_t q;
  for (q = 0; q < i; q++) s += or_row_se_count(p, q);
  return s;
}

/* ---- Sec. 3.2 constraints; returns 0 if valid, else a reason code ------ */
int or_check_params(const or_params *p) {
  uint32_t L, i, j;
  if (p->r > 24) return 1;
  L = 32 - p->r;
  if (p->sr < 1 || p->sr > 8) return 2;
  for (i = 0; i < p->sr; i++) {
    if (p->ibn[i] < 1 || p->ibn[i] > 12 || p->ibn[i] > L) return 3;
    if (p->isb[i] >= L) return 4;
  }
  /* constraint 1: every LP bit lies in at least one index */
  for (j = 0; j < L; j++) {
    int covered = 0;
    for (i = 0; i < p->sr && !covered; i++) {
      uint32_t q;
      for (q = 0; q < p->ibn[i]; q++)
        if ((p->isb[i] + q) % L == j) { covered = 1; break; }
    }
    if (!covered) return 5;
  }
  /* constraint 2 (reading): row i and row (i+1) mod SR share an LP bit */
  if (p->sr > 1) {
    for (i = 0; i < p->sr; i++) {
      uint32_t n = (i + 1) % p->sr, q, w, shared = 0;
      for (q = 0; q < p->ibn[i] && !shared; q++)
        for (w = 0; w < p->ibn[n]; w++)
          if ((p->isb[i] + q) % L == (p->isb[n] + w) % L) { shared = 1; break; }
      if (!shared) return 6;
    }
  }
  if (p->k_log2 < 5 || p->k_log2 > 16) return 7;
  if (p->lr < 1 || p->lr > 8) return 8;
  if (p->lc_log2 > 24) return 9;
  if (p->theta == 0) return 10;
  return 0;
}

/* ---- per-pair scan: Sec. 3.1 (SE), Sec. 3.2 (SEAV), Sec. 3.3 (LDCA) ----- */
void or_update(const or_params *p, uint8_t *seav, uint32_t *ldca,
               const uint32_t *pairs, uint64_t n_pairs) {
  uint64_t a[10], b[10], n;
  uint32_t tau = or_tau(p->theta);
  uint64_t sea_bytes = or_sea_bytes(p);
  uint64_t lc = (uint64_t)1 << p->lc_log2;
  uint64_t ldc_words = ((uint64_t)1 << p->k_log2) / 32;
  or_hash_params(p->seed, p->lr, a, b);
  for (n = 0; n < n_pairs; n++) {
    uint32_t hip = pairs[2 * n], oip = pairs[2 * n + 1];
    uint32_t h1 = or_h1(a, b, oip);
    uint32_t i, h3;
    /* short estimator: sample by lsb(H1(oip)) >= tau, set bit H2(oip) */
    if (or_lsb(h1) >= tau) {
      uint32_t rp = or_rp(p->r, hip), lp = or_lp(p->r, hip);
      uint8_t bit = (uint8_t)(1u << or_h2(h1));
      for (i = 0; i < p->sr; i++) {
        uint64_t off = (uint64_t)rp * sea_bytes + or_row_offset(p, i) + or_idx(p, i, lp);
        seav[off] |= bit;
      }
    }
    /* long estimator: bit H3(oip) in LDC LH_i(hip) of every row */
    h3 = or_h3(a, b, p->k_log2, oip);
    for (i = 0; i < p->lr; i++) {
      uint64_t col = or_lh(a, b, p->lc_log2, i, hip);
      uint64_t word = ((uint64_t)i * lc + col) * ldc_words + h3 / 32;
      ldca[word] |= 1u << (h3 % 32);
    }
  }
}

/* ---- Sec. 4.2: global sketch from the watch points' sketches ----------- */
void or_merge(uint8_t *dst, const uint8_t *src, uint64_t n_bytes) {
  uint64_t i;
  for (i = 0; i < n_bytes; i++) dst[i] |= src[i];
}

/* ---- Eq. 4 as an integer test -----------------------------------------
 * est(z) = -k ln(z / k).  Z_theta = max { z in [0, k] : est(z) >= theta }.
 * est is decreasing in z, and est(0) = +inf, so Z_theta always exists. */
double or_est(uint32_t k_log2, uint32_t z0) {
  double k = (double)((uint64_t)1 << k_log2);
  return -k * log((double)z0 / k);
}
uint32_t or_z_theta(uint32_t k_log2, uint32_t theta) {
  uint32_t k = 1u << k_log2, z;
  for (z = k; z > 0; z--)
    if (or_est(k_log2, z) >= (double)theta) return z;
  return 0;
}

/* ---- restore: Sec. 3.2 (HSE, CIdx, CIS, SEU, Eq. 3) + Sec. 3.3 ---------- */
static int or_cmp_cand(const void *x, const void *y) {
  const or_candidate *u = (const or_candidate *)x, *v = (const or_candidate *)y;
  return (u->ip > v->ip) - (u->ip < v->ip);
}

/* Returns 0, or -1 if more than `cap` super points were found (out then holds
 * the first `cap` in ascending IP order and *n_total the full count). */
int or_detect(const or_params *p, const uint8_t *seav, const uint32_t *ldca,
              uint32_t threshold, or_candidate *out, uint64_t cap, uint64_t *n_total) {
  uint64_t a[10], b[10];
  uint32_t L = 32 - p->r, k = 1u << p->k_log2;
  uint64_t sea_bytes = or_sea_bytes(p);
  uint64_t lc = (uint64_t)1 << p->lc_log2, ldc_words = (uint64_t)k / 32;
  uint32_t zt = or_z_theta(p->k_log2, threshold);
  uint64_t rp, n_found = 0, n_alloc = 1024;
  or_candidate *found = (or_candidate *)malloc(n_alloc * sizeof(or_candidate));
  uint32_t *hse[8];
  uint32_t nhse[8], i;
  or_hash_params(p->seed, p->lr, a, b);
  for (i = 0; i < p->sr; i++) hse[i] = (uint32_t *)malloc(sizeof(uint32_t) * or_row_se_count(p, i));

  for (rp = 0; rp < ((uint64_t)1 << p->r); rp++) {
    const uint8_t *sea = seav + rp * sea_bytes;
    int any_empty = 0;
    uint32_t pos[8];
    /* HSE(i): the SEs of row i whose weight is at least 3 */
    for (i = 0; i < p->sr; i++) {
      const uint8_t *row = sea + or_row_offset(p, i);
      uint32_t c;
      nhse[i] = 0;
      for (c = 0; c < or_row_se_count(p, i); c++)
        if (or_popcount(row[c]) >= 3) hse[i][nhse[i]++] = c;
      if (nhse[i] == 0) any_empty = 1;
    }
    if (any_empty) continue;
    /* CIS: every CIdx = <c[0], ..., c[SR-1]> with c[i] in HSE(i) */
    for (i = 0; i < p->sr; i++) pos[i] = 0;
    for (;;) {
      uint8_t assigned[32], value[32];
      int consistent = 1;
      uint32_t lp = 0, j;
      uint8_t seu = 0xFF;
      memset(assigned, 0, sizeof(assigned));
      memset(value, 0, sizeof(value));
      /* Eq. 3: LP[(ISB(i) + j) mod L] = Idx(i)[j]; rows must agree */
      for (i = 0; i < p->sr && consistent; i++) {
        uint32_t c = hse[i][pos[i]];
        for (j = 0; j < p->ibn[i]; j++) {
          uint32_t bp = (p->isb[i] + j) % L;
          uint8_t v = (uint8_t)((c >> j) & 1u);
          if (assigned[bp] && value[bp] != v) { consistent = 0; break; }
          assigned[bp] = 1;
          value[bp] = v;
        }
      }
      if (consistent) {
        /* SEU: bitwise AND of the chosen SEs; keep when its weight >= 3 */
        for (i = 0; i < p->sr; i++) seu &= sea[or_row_offset(p, i) + hse[i][pos[i]]];
        if (or_popcount(seu) >= 3) {
          uint32_t ip, zeros = 0, w;
          for (j = 0; j < L; j++) lp |= (uint32_t)value[j] << j;
          ip = (uint32_t)(((uint64_t)lp << p->r) | rp);
          /* ULDC = AND of the host's LDC in every LDCA row; z0 = its zeros */
          for (w = 0; w < ldc_words; w++) {
            uint32_t u = 0xFFFFFFFFu;
            for (i = 0; i < p->lr; i++) {
              uint64_t col = or_lh(a, b, p->lc_log2, i, ip);
              u &= ldca[((uint64_t)i * lc + col) * ldc_words + w];
            }
            zeros += 32 - or_popcount(u);
          }
          if (zeros <= zt) {
            or_candidate cand;
            cand.ip = ip;
            cand.z0 = zeros;
            cand.flags = zeros == 0 ? OR_FLAG_SATURATED : 0;
            cand.est = zeros == 0 ? (double)k * log((double)k) : or_est(p->k_log2, zeros);
            cand.pad = 0;
            if (n_found == n_alloc) {
              n_alloc *= 2;
              found = (or_candidate *)realloc(found, n_alloc * sizeof(or_candidate));
            }
            found[n_found++] = cand;
          }
        }
      }
      /* next tuple of the cartesian product (odometer, row SR-1 fastest) */
      i = p->sr;
      while (i > 0) {
        i--;
        if (++pos[i] < nhse[i]) break;
        pos[i] = 0;
        if (i == 0) { i = (uint32_t)-1; break; }
      }
      if (i == (uint32_t)-1) break;
    }
  }
  qsort(found, n_found, sizeof(or_candidate), or_cmp_cand);
  *n_total = n_found;
  if (out) memcpy(out, found, (n_found < cap ? n_found : cap) * sizeof(or_candidate));
  for (i = 0; i < p->sr; i++) free(hse[i]);
  free(found);
  return n_found > cap ? -1 : 0;
}

/* ---- Lemma 1 and Theorem 1 (Sec. 3.4): sizing the LDCA ----------------
 * Psu: probability that a bit of a host's LDC union is 1 when N distinct
 * pairs are spread over LC columns in each of LR rows.  LR*: the row count
 * minimising Psu for a fixed number V = LR * LC of LDCs (continuous). */
double or_psu(double n_pairs, uint32_t k_log2, double lr, double lc) {
  double k = (double)((uint64_t)1 << k_log2);
  double keep0 = pow(1.0 - 1.0 / k, n_pairs / lc);   /* a bit stays 0 in one LDC */
  return pow(1.0 - keep0, lr);
}

double or_lr_star(double n_pairs, uint32_t k_log2, double v_ldcs) {
  double k = (double)((uint64_t)1 << k_log2);
  return -v_ldcs * log(2.0) / (n_pairs * log(1.0 - 1.0 / k));
}
