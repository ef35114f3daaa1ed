/* CPU oracle for suffix-array construction — TEST INFRASTRUCTURE ONLY.
 * See oracle.h for the contract, the citations and who may call this.
 *
 * ORACLE_MUTANT (compile-time, default 0) plants one known mistake per value
 * so that the pin tests can show each plausible mistake is caught; the
 * product never builds a mutant. */
#define _GNU_SOURCE
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

/* ---- the order on suffixes (Section 2 and the $ of Section 2.1) --------- */

/* Compare T[a, a+la) with T[b, b+lb) where la, lb are the lengths that are
 * looked at; the end of the text ($) is below every character, so when one
 * is a proper prefix of the other the shorter one is smaller. */
static int cmp_prefix(const uint8_t *T, int64_t a, int64_t la, int64_t b, int64_t lb) {
  int64_t l = la < lb ? la : lb;
  int c = memcmp(T + a, T + b, (size_t)l);
  if (c != 0) return c < 0 ? -1 : 1;
#if ORACLE_MUTANT == 5
  return (la > lb) ? -1 : (la < lb); /* mutant: $ above every character */
#elif ORACLE_MUTANT == 7
  return 0; /* mutant: prefixes compare equal */
#else
  return (la < lb) ? -1 : (la > lb);
#endif
}

static int cmp_suffix(const uint8_t *T, int64_t n, int64_t a, int64_t b) {
  return cmp_prefix(T, a, n - a, b, n - b);
}

typedef struct {
  const uint8_t *T;
  int64_t n;
  int64_t h; /* number of leading characters compared */
} sort_ctx;

static int qs_suffix(const void *x, const void *y, void *c) {
  const sort_ctx *s = (const sort_ctx *)c;
  int64_t a = *(const uint32_t *)x, b = *(const uint32_t *)y;
  return cmp_suffix(s->T, s->n, a, b);
}

void oracle_naive_sa(const uint8_t *T, int64_t n, uint32_t *sa) {
  for (int64_t i = 0; i < n; ++i) sa[i] = (uint32_t)i;
  sort_ctx c = {T, n, n};
  if (n > 1) qsort_r(sa, (size_t)n, sizeof(uint32_t), qs_suffix, &c);
}

/* ---- prefix doubling with discarding (Section 2.1) ---------------------- */

/* The first h characters of suffix a, compared as in the initial triples of
 * Algorithm 1 (there h = 2: (T[i], T[i+1]) with T[n] = $). */
static int qs_prefix_h(const void *x, const void *y, void *c) {
  const sort_ctx *s = (const sort_ctx *)c;
  int64_t a = *(const uint32_t *)x, b = *(const uint32_t *)y;
  int64_t la = s->n - a, lb = s->n - b;
  if (la > s->h) la = s->h;
  if (lb > s->h) lb = s->h;
  return cmp_prefix(s->T, a, la, b, lb);
}

/* The partner names r[0..a-2] of one suffix (the names of i + h, i + 2h,
 * ..., each shifted by one, 0 past the end) and its position, for one
 * suffix inside a group being refined. */
#define ORACLE_MAX_A 4
typedef struct {
  uint64_t r[ORACLE_MAX_A - 1];
  uint32_t pos;
} name_tuple;

/* Lexicographic order of the partner tuples (the group shares the first
 * name, so only the partners are compared). Unused entries are 0. */
static int qs_tuple(const void *x, const void *y) {
  const name_tuple *a = (const name_tuple *)x, *b = (const name_tuple *)y;
  for (int k = 0; k < ORACLE_MAX_A - 1; ++k)
    if (a->r[k] != b->r[k]) return a->r[k] < b->r[k] ? -1 : 1;
  return 0;
}

int64_t oracle_pd_sa(const uint8_t *T, int64_t n, int64_t h0, uint32_t *sa,
                     uint32_t *isa_out, uint32_t *trace, int64_t trace_cap) {
  return oracle_pq_sa(T, n, h0, 2, sa, isa_out, trace, trace_cap);
}

int64_t oracle_pq_sa(const uint8_t *T, int64_t n, int64_t h0, int64_t a, uint32_t *sa,
                     uint32_t *isa_out, uint32_t *trace, int64_t trace_cap) {
  if (n <= 0) return 0;
  if (h0 < 1) h0 = 1;
  if (a < 2 || a > ORACLE_MAX_A) return -1;
  uint32_t *isa = isa_out ? isa_out : (uint32_t *)malloc((size_t)n * sizeof(uint32_t));

  /* Initial names (Algorithm 1, first lines; Algorithm 5, first four lines):
   * sort the positions by their first h0 characters, then CmpName marks
   * every item whose prefix differs from its predecessor with its position
   * j (0 otherwise) and PrefixSum(max) turns the marks into names: the head
   * rank, i.e. the sorted position of the first member of the group. */
  for (int64_t i = 0; i < n; ++i) sa[i] = (uint32_t)i;
  sort_ctx c = {T, n, h0};
  qsort_r(sa, (size_t)n, sizeof(uint32_t), qs_prefix_h, &c);
  {
    uint32_t run_max = 0; /* PrefixSum with max */
    for (int64_t j = 0; j < n; ++j) {
      uint32_t mark = 0; /* CmpName */
      if (j > 0 && qs_prefix_h(&sa[j - 1], &sa[j], &c) != 0) mark = (uint32_t)j;
      if (mark > run_max) run_max = mark;
      isa[sa[j]] = run_max;
    }
  }
  if (trace && trace_cap > 0) memcpy(trace, isa, (size_t)n * sizeof(uint32_t));

  name_tuple *tup = (name_tuple *)malloc((size_t)n * sizeof(name_tuple));
  uint32_t *fresh = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  int64_t rounds = 0;
  int64_t h = h0; /* characters resolved by the current names */
#if ORACLE_MUTANT == 6
  int64_t lg = 0;
  while ((1LL << lg) < n) ++lg;
  /* mutant: the literal bound of Algorithm 1, whose first of its
   * ceil(log2 n) - 1 iterations forms the initial names */
  int64_t max_rounds = lg - 2;
#else
  int64_t max_rounds = 64;     /* never reached for n <= 2^31 */
#endif
  for (;;) {
    if (rounds >= max_rounds) break;
    /* Unique (Algorithm 6): a group is a maximal run of equal names in the
     * current order; a run of length 1 is unique and is discarded for good
     * (its name is already its rank). Every other run is refined below. */
    int any = 0;
    int64_t gs = 0;
    while (gs < n) {
      int64_t ge = gs + 1;
      while (ge < n && isa[sa[ge]] == isa[sa[gs]]) ++ge;
      if (ge - gs > 1) {
        any = 1;
        /* Partner names through the ISA (Algorithm 4): the name of suffix
         * i + k*h for k = 1 .. a-1 (a = 2: the pair of Algorithm 4; a = 4:
         * the rank quadruple of prefix quadrupling) if it exists, shifted
         * by one so that the sentinel 0 sorts below every real name. */
        for (int64_t j = gs; j < ge; ++j) {
          uint32_t i = sa[j];
          memset(&tup[j], 0, sizeof(name_tuple));
          for (int64_t k = 1; k < a; ++k) {
#if ORACLE_MUTANT == 1
            int64_t at = i + k * h;
            uint64_t r = (at < n) ? (uint64_t)isa[at] : 0; /* literal sentinel */
#elif ORACLE_MUTANT == 2
            int64_t off = h / 2 > 0 ? h / 2 : 1; /* the prose's i + 2^(k-1) */
            int64_t at = i + k * off;
            uint64_t r = (at < n) ? (uint64_t)isa[at] + 1 : 0;
#elif ORACLE_MUTANT == 5
            int64_t at = i + k * h;
            uint64_t r = (at < n) ? (uint64_t)isa[at] : (uint64_t)n + 1;
#elif ORACLE_MUTANT == 11
            int64_t at = i + (k == 3 ? 2 : k) * h; /* mutant: last partner repeated */
            uint64_t r = (at < n) ? (uint64_t)isa[at] + 1 : 0;
#else
            int64_t at = i + k * h;
            uint64_t r = (at < n) ? (uint64_t)isa[at] + 1 : 0;
#endif
            tup[j].r[k - 1] = r;
          }
          tup[j].pos = i;
        }
        /* Sort the group by its partner tuples (the group shares r). */
        qsort(tup + gs, (size_t)(ge - gs), sizeof(name_tuple), qs_tuple);
        /* NameDiscarding (Algorithm 6, corrected): all members share the
         * old name r = group head; a new subgroup starts where the partner
         * tuple changes; new name = r + (subgroup start - group start). */
        uint32_t r = isa[tup[gs].pos];
        int64_t sub = gs;
        for (int64_t j = gs; j < ge; ++j) {
          if (j > gs && qs_tuple(&tup[j], &tup[j - 1]) != 0) sub = j;
          sa[j] = tup[j].pos;
#if ORACLE_MUTANT == 4
          fresh[j] = r + (uint32_t)(sub - gs) + (sub > gs ? 1u : 0u);
#else
          fresh[j] = r + (uint32_t)(sub - gs);
#endif
        }
#if ORACLE_MUTANT == 3
        /* mutant: names rewritten before the other groups read them */
        for (int64_t j = gs; j < ge; ++j) isa[sa[j]] = fresh[j];
#endif
      }
      gs = ge;
    }
    if (!any) break; /* all names distinct (Algorithm 5, I.Size() = 0) */
    ++rounds;
    /* Only now, with every partner name of this round read, rewrite the
     * names of the refined groups. The pre-round names are still in isa[],
     * so the refined groups are again the runs of equal names. */
    {
      int64_t j = 0;
      while (j < n) {
        int64_t e = j + 1;
        uint32_t old = isa[sa[j]];
        while (e < n && isa[sa[e]] == old) ++e;
#if ORACLE_MUTANT != 3
        if (e - j > 1)
          for (int64_t k = j; k < e; ++k) isa[sa[k]] = fresh[k];
#endif
        j = e;
      }
    }
#if ORACLE_MUTANT == 12
    h *= 2; /* mutant: resolved length doubled whatever a is */
#else
    h *= a; /* the names now resolve a*h characters */
#endif
    if (trace && rounds < trace_cap)
      memcpy(trace + rounds * n, isa, (size_t)n * sizeof(uint32_t));
  }
  free(tup);
  free(fresh);
  if (!isa_out) free(isa);
  return rounds;
}

/* ---- DC7 recursion text (Section 2.2) ---------------------------------- */

#if ORACLE_MUTANT == 13
#define DC7_WIN 6 /* mutant: one character short of the window */
#else
#define DC7_WIN 7
#endif

typedef struct {
  int16_t c[7]; /* the window, -1 past the end of the text */
  int64_t slot; /* index in the recursion text */
} dc7_win;

static int qs_dc7(const void *x, const void *y) {
  const dc7_win *a = (const dc7_win *)x, *b = (const dc7_win *)y;
  for (int k = 0; k < DC7_WIN; ++k)
    if (a->c[k] != b->c[k]) return a->c[k] < b->c[k] ? -1 : 1;
  return 0;
}

int64_t oracle_dc7_names(const uint8_t *T, int64_t n, uint32_t *out) {
  static const int D7[3] = {0, 1, 3};
  if (n < 0) return 0;
  dc7_win *w = (dc7_win *)malloc((size_t)(3 * (n / 7 + 1) + 1) * sizeof(dc7_win));
  int64_t m = 0;
  for (int d = 0; d < 3; ++d)
    for (int64_t i = D7[d]; i <= n; i += 7) {
      for (int k = 0; k < 7; ++k) w[m].c[k] = i + k < n ? (int16_t)T[i + k] : (int16_t)-1;
      w[m].slot = m;
      ++m;
    }
  /* Sort the windows (a library sort), then name them in sorted order: a
   * new name wherever the window differs from its predecessor. */
  qsort(w, (size_t)m, sizeof(dc7_win), qs_dc7);
  uint32_t name = 0;
  for (int64_t k = 0; k < m; ++k) {
    if (k == 0 || qs_dc7(&w[k], &w[k - 1]) != 0) ++name;
    out[w[k].slot] = name;
  }
  free(w);
  return m;
}

/* ---- checkers ----------------------------------------------------------- */

int oracle_check_sa(const uint8_t *T, int64_t n, const uint32_t *sa, int64_t *bad) {
  if (n <= 0) return 0;
  int64_t *rank = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) rank[i] = -1;
  for (int64_t j = 0; j < n; ++j) {
    if ((int64_t)sa[j] >= n || rank[sa[j]] != -1) {
      if (bad) *bad = j;
      free(rank);
      return 1;
    }
    rank[sa[j]] = j;
  }
  for (int64_t j = 0; j + 1 < n; ++j) {
    int64_t a = sa[j], b = sa[j + 1];
    if (T[a] != T[b]) {
      if (T[a] > T[b]) {
        if (bad) *bad = j;
        free(rank);
        return 2;
      }
      continue;
    }
#if ORACLE_MUTANT == 8
    int64_t ra = (a + 1 < n) ? rank[a + 1] : n; /* mutant: empty suffix largest */
    int64_t rb = (b + 1 < n) ? rank[b + 1] : n;
#else
    int64_t ra = (a + 1 < n) ? rank[a + 1] : -1; /* the empty suffix is smallest */
    int64_t rb = (b + 1 < n) ? rank[b + 1] : -1;
#endif
    if (!(ra < rb)) {
      if (bad) *bad = j;
      free(rank);
      return 2;
    }
  }
  free(rank);
  return 0;
}

int oracle_check_permutation(const uint32_t *sa, int64_t n, int64_t *bad) {
  if (n <= 0) return 0;
  uint64_t *seen = (uint64_t *)calloc((size_t)(n + 63) / 64, sizeof(uint64_t));
  for (int64_t j = 0; j < n; ++j) {
    const uint64_t v = sa[j];
    if ((int64_t)v >= n || (seen[v >> 6] >> (v & 63)) & 1u) {
      if (bad) *bad = j;
      free(seen);
      return 1;
    }
    seen[v >> 6] |= 1ull << (v & 63);
  }
  free(seen);
  return 0;
}

int64_t oracle_check_adjacent(const uint8_t *T, int64_t n, const uint32_t *sa,
                              const int64_t *idx, int64_t count) {
  int64_t bad = 0;
  for (int64_t k = 0; k < count; ++k) {
    int64_t j = idx[k];
#if ORACLE_MUTANT == 15
    if (j <= 0 || j + 1 >= n) continue; /* mutant: the first pair never checked */
#else
    if (j < 0 || j + 1 >= n) continue; /* no pair (j, j+1) inside SA */
#endif
    if (sa[j] >= n || sa[j + 1] >= n) {
      ++bad;
      continue;
    }
#if ORACLE_MUTANT == 14
    const int c = cmp_suffix(T, n, sa[j + 1], sa[j]); /* mutant: operands swapped */
#else
    const int c = cmp_suffix(T, n, sa[j], sa[j + 1]);
#endif
#if ORACLE_MUTANT == 16
    if (c > 0) ++bad; /* mutant: equal suffixes (a repeated entry) pass */
#else
    if (c >= 0) ++bad; /* SA[j]'s suffix must be strictly smaller */
#endif
  }
  return bad;
}

int64_t oracle_suffix_rank(const uint8_t *T, int64_t n, int64_t i) {
  int64_t r = 0;
  for (int64_t j = 0; j < n; ++j)
    if (j != i && cmp_suffix(T, n, j, i) < 0) ++r;
  return r;
}

/* ---- Burrows-Wheeler transform (a consumer of SA, Section 3) ------------ */

void oracle_bwt(const uint8_t *T, int64_t n, const uint32_t *sa, uint8_t *bwt,
                int64_t *primary) {
  /* row 0: the suffix $ (empty), preceded by T[n-1] */
  bwt[0] = n > 0 ? T[n - 1] : 0;
  *primary = n > 0 ? -1 : 0;
  for (int64_t j = 0; j < n; ++j) {
    if (sa[j] == 0) {
      bwt[j + 1] = 0;
      *primary = j + 1;
    } else {
      bwt[j + 1] = T[sa[j] - 1];
    }
  }
}

int oracle_bwt_invert(const uint8_t *bwt, int64_t n, int64_t primary, uint8_t *out) {
  if (n <= 0) return 0;
  int64_t count[256] = {0};
  int64_t *occ = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
  for (int64_t r = 0; r <= n; ++r) {
    if (r == primary) {
      occ[r] = 0;
      continue;
    }
    occ[r] = count[bwt[r]]++;
  }
  /* C[c] = rows whose suffix starts below c: the $ row plus smaller chars */
  int64_t C[256];
#if ORACLE_MUTANT == 9
  int64_t acc = 0; /* mutant: forgets the $ row */
#else
  int64_t acc = 1;
#endif
  for (int c = 0; c < 256; ++c) {
    C[c] = acc;
    acc += count[c];
  }
  int64_t r = 0; /* the row of the empty suffix */
  for (int64_t k = n - 1; k >= 0; --k) {
    if (r == primary || r < 0 || r > n) {
      free(occ);
      return 1;
    }
    uint8_t ch = bwt[r];
    out[k] = ch;
    r = C[ch] + occ[r];
  }
  free(occ);
  return 0;
}

/* ---- LCP array (a consumer of SA, Section 3), by its definition -------- */

int64_t oracle_lcp_pair(const uint8_t *T, int64_t n, int64_t a, int64_t b) {
  int64_t l = 0;
#if ORACLE_MUTANT == 10
  /* mutant: stops one character before the end of text */
  while (a + l < n - 1 && b + l < n - 1 && T[a + l] == T[b + l]) ++l;
#else
  while (a + l < n && b + l < n && T[a + l] == T[b + l]) ++l;
#endif
  return l;
}

void oracle_lcp(const uint8_t *T, int64_t n, const uint32_t *sa, uint32_t *lcp) {
  if (n <= 0) return;
  lcp[0] = 0;
  for (int64_t j = 1; j < n; ++j) lcp[j] = (uint32_t)oracle_lcp_pair(T, n, sa[j - 1], sa[j]);
}
