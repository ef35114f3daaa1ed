/* Seeded synthetic workload generators; see gen.h for the recipes.
 * Compile with -ffp-contract=off so that no multiply-add is fused and the
 * floating-point results agree bit for bit on x86_64 and aarch64. */
#include "gen.h"

#include <stdlib.h>
#include <string.h>

/* ---- random stream ----------------------------------------------------- */

/* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): used only to expand a 64-bit seed into the
 * xoshiro state. */
static uint64_t splitmix_next(uint64_t *state) {
  uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

typedef struct {
  uint64_t s[4];
} rng_t;

static uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

/* xoshiro256** (Blackman & Vigna, "Scrambled linear pseudorandom number
 * generators", ACM TOMS 2021). */
static uint64_t rng_next(rng_t *r) {
  uint64_t out = rotl64(r->s[1] * 5u, 7) * 9u;
  uint64_t t = r->s[1] << 17;
  r->s[2] ^= r->s[0];
  r->s[3] ^= r->s[1];
  r->s[1] ^= r->s[2];
  r->s[0] ^= r->s[3];
  r->s[2] ^= t;
  r->s[3] = rotl64(r->s[3], 45);
  return out;
}

static void rng_seed(rng_t *r, uint64_t seed) {
  uint64_t sm = seed;
  for (int k = 0; k < 4; ++k) r->s[k] = splitmix_next(&sm);
}

/* Uniform double in [0, 1) with 53 random bits. */
static double rng_unit(rng_t *r) {
  return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0);
}

/* Uniform integer in [0, bound) by rejection (no modulo bias). */
static uint64_t rng_below(rng_t *r, uint64_t bound) {
  if (bound <= 1) return 0;
  uint64_t limit = UINT64_MAX - (UINT64_MAX % bound);
  uint64_t x;
  do {
    x = rng_next(r);
  } while (x >= limit);
  return x % bound;
}

/* ---- deterministic elementary functions -------------------------------- */

static const double LN2 = 0.69314718055994530942;

/* ln(x) for x > 0: x = m * 2^e with m in [sqrt(1/2), sqrt(2)), then
 * ln(m) = 2 atanh((m-1)/(m+1)) by its power series. */
double gen_log(double x) {
  if (!(x > 0.0)) return -1.0e300;
  int e = 0;
  double m = x;
  while (m >= 1.4142135623730951) {
    m *= 0.5;
    ++e;
  }
  while (m < 0.70710678118654752) {
    m *= 2.0;
    --e;
  }
  double s = (m - 1.0) / (m + 1.0);
  double s2 = s * s;
  double term = s;
  double sum = 0.0;
  for (int k = 1; k < 60; k += 2) {
    sum += term / (double)k;
    term *= s2;
  }
  return 2.0 * sum + (double)e * LN2;
}

/* exp(x): x = k ln2 + r with |r| <= ln2/2, exp(r) by its Taylor series,
 * then scaled by 2^k through repeated doubling/halving. */
double gen_exp(double x) {
  if (x > 700.0) x = 700.0;
  if (x < -700.0) x = -700.0;
  double kd = x / LN2;
  long k = (long)(kd >= 0 ? kd + 0.5 : kd - 0.5);
  double r = x - (double)k * LN2;
  double term = 1.0, sum = 1.0;
  for (int j = 1; j < 30; ++j) {
    term = term * r / (double)j;
    sum += term;
  }
  while (k > 0) {
    sum *= 2.0;
    --k;
  }
  while (k < 0) {
    sum *= 0.5;
    ++k;
  }
  return sum;
}

/* ---- recipe helpers ---------------------------------------------------- */

static const uint8_t DNA[4] = {'A', 'C', 'G', 'T'};

/* Cumulative Zipf(s = 1.1) weights over ranks 1..255. */
static void zipf_cdf(double cdf[256]) {
  double acc = 0.0;
  cdf[0] = 0.0;
  for (int k = 1; k <= 255; ++k) {
    acc += gen_exp(-1.1 * gen_log((double)k));
    cdf[k] = acc;
  }
}

/* Draw a Zipf rank in 1..255 (= the byte value). */
static uint8_t zipf_draw(rng_t *r, const double cdf[256]) {
  double u = rng_unit(r) * cdf[255];
  int lo = 1, hi = 255; /* smallest k with cdf[k] > u */
  while (lo < hi) {
    int mid = (lo + hi) / 2;
    if (cdf[mid] > u)
      hi = mid;
    else
      lo = mid + 1;
  }
  return (uint8_t)lo;
}

/* ---- recipes ------------------------------------------------------------ */

void gen_dna_uniform(uint64_t seed, uint64_t n, uint8_t *out) {
  rng_t r;
  rng_seed(&r, seed);
  uint64_t i = 0;
  while (i < n) {
    uint64_t x = rng_next(&r);
    for (int k = 0; k < 32 && i < n; ++k, ++i) {
      out[i] = DNA[x >> 62];
      x <<= 2;
    }
  }
}

void gen_bytes_uniform(uint64_t seed, uint64_t n, uint8_t *out) {
  rng_t r;
  rng_seed(&r, seed);
  uint64_t i = 0;
  while (i < n) {
    uint64_t x = rng_next(&r);
    for (int k = 0; k < 8 && i < n; ++k, ++i) {
      out[i] = (uint8_t)(x >> 56);
      x <<= 8;
    }
  }
}

void gen_zipf_iid(uint64_t seed, uint64_t n, uint8_t *out) {
  double cdf[256];
  zipf_cdf(cdf);
  rng_t r;
  rng_seed(&r, seed);
  for (uint64_t i = 0; i < n; ++i) out[i] = zipf_draw(&r, cdf);
}

void gen_zipf_repeats(uint64_t seed, uint64_t n, uint8_t *out) {
  if (n == 0) return;
  double cdf[256];
  zipf_cdf(cdf);
  rng_t r;
  rng_seed(&r, seed);
  uint64_t copies = n < 256 ? 1 : 256;
  uint64_t base = (n + copies - 1) / copies;
  uint8_t *b = (uint8_t *)malloc(base);
  uint8_t *hit = (uint8_t *)malloc(base);
  for (uint64_t i = 0; i < base; ++i) b[i] = zipf_draw(&r, cdf);
  /* round(0.001 * base) substitutions per copy */
  uint64_t subs = (base + 500) / 1000;
  for (uint64_t c = 0; c < copies; ++c) {
    uint64_t start = c * base;
    if (start >= n) break;
    uint64_t len = (n - start < base) ? n - start : base;
    memcpy(out + start, b, len);
    memset(hit, 0, base);
    for (uint64_t s = 0; s < subs && s < base; ++s) {
      uint64_t p;
      do {
        p = rng_below(&r, base);
      } while (hit[p]);
      hit[p] = 1;
      uint8_t v;
      do {
        v = zipf_draw(&r, cdf);
      } while (v == b[p]);
      if (p < len) out[start + p] = v;
    }
  }
  free(b);
  free(hit);
}

void gen_markov_dna(uint64_t seed, uint64_t n, uint8_t *out, uint8_t *scratch) {
  if (n == 0) return;
  rng_t r;
  rng_seed(&r, seed);
  /* 64 context rows, each a Dirichlet(1,1,1,1) draw = normalised Exp(1). */
  double cum[64][4];
  for (int c = 0; c < 64; ++c) {
    double w[4], tot = 0.0;
    for (int k = 0; k < 4; ++k) {
      w[k] = -gen_log(1.0 - rng_unit(&r));
      tot += w[k];
    }
    double acc = 0.0;
    for (int k = 0; k < 4; ++k) {
      acc += w[k] / tot;
      cum[c][k] = acc;
    }
    cum[c][3] = 2.0; /* guard against rounding: the last symbol absorbs it */
  }
  unsigned ctx = 0;
  for (uint64_t i = 0; i < n; ++i) {
    unsigned sym;
    if (i < 3) {
      sym = (unsigned)rng_below(&r, 4);
    } else {
      double u = rng_unit(&r);
      sym = 0;
      while (u >= cum[ctx][sym]) ++sym;
    }
    out[i] = DNA[sym];
    ctx = ((ctx << 2) | sym) & 63u;
  }
  /* Copied segments, read from the pre-copy snapshot. */
  memcpy(scratch, out, n);
  uint64_t need = (n * 5 + 99) / 100, covered = 0;
  uint64_t lo = 1024, hi = 102400;
  if (hi > n / 4) hi = n / 4;
  if (lo > hi) lo = hi;
  if (hi == 0) return;
  while (covered < need) {
    uint64_t len = lo + rng_below(&r, hi - lo + 1);
    uint64_t src = rng_below(&r, n - len + 1);
    uint64_t dst = rng_below(&r, n - len + 1);
    memcpy(out + dst, scratch + src, len);
    covered += len;
  }
}

void gen_batch_lengths(uint64_t seed, uint32_t count, uint64_t lo, uint64_t hi,
                       uint64_t *lengths) {
  rng_t r;
  rng_seed(&r, seed);
  double a = gen_log((double)lo), b = gen_log((double)hi);
  for (uint32_t k = 0; k < count; ++k) {
    double v = gen_exp(a + (b - a) * rng_unit(&r));
    uint64_t len = (uint64_t)(v + 0.5);
    if (len < lo) len = lo;
    if (len > hi) len = hi;
    lengths[k] = len;
  }
}

void gen_request_stream(uint64_t seed, uint32_t count, double lambda,
                        uint64_t lo, uint64_t hi, double *arrival_s,
                        uint64_t *sizes, uint8_t *kinds) {
  rng_t r;
  rng_seed(&r, seed);
  double a = gen_log((double)lo), b = gen_log((double)hi);
  double t = 0.0;
  for (uint32_t k = 0; k < count; ++k) {
    t += -gen_log(1.0 - rng_unit(&r)) / lambda;
    arrival_s[k] = t;
    double v = gen_exp(a + (b - a) * rng_unit(&r));
    uint64_t len = (uint64_t)(v + 0.5);
    if (len < lo) len = lo;
    if (len > hi) len = hi;
    sizes[k] = len;
    kinds[k] = (uint8_t)(rng_next(&r) >> 63);
  }
}
