/* CPU oracle for suffix-array construction — TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline and
 * reference legs may load or call this code. The CUDA library never does:
 * the two share no code, headers or helpers.
 *
 * Plain, sequential, obviously-correct C. Every function cites the passage
 * of Bingmann, Gog & Kurpicz, "Scalable Construction of Text Indexes"
 * (arXiv 1610.03007) that it follows. All arithmetic is integer.
 *
 * Pins (tests/test_oracle.py): the worked examples Ex 1, Ex 2 and Ex 3,
 * closed forms (a^n, (ab)^m, all-distinct), brute force over every binary
 * string up to length 14 against Python's own bytes ordering, the
 * invariants (permutation, ISA[SA[j]] = j, BWT inversion reproduces T),
 * the LCP array's textbook and closed-form values and brute force against
 * Python's own prefix comparison, the per-round names of the a-fold
 * variant against head ranks of a^k-length prefixes computed by brute
 * force, and planted-mutant builds of this file, each of which must fail a
 * pin.
 */
#ifndef GBSA_ORACLE_H
#define GBSA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Definition of the suffix array (Section 2): SA is the permutation of
 * [0,n) with T[SA[i],n) <=lex T[SA[j],n) for i <= j; bytes compare as
 * unsigned and a proper prefix is smaller (T[n] = $ is below every
 * character, Section 2.1). Written out as a comparison sort of all suffixes.
 * O(n log n) comparisons of O(LCP) each: small or low-repeat inputs only. */
void oracle_naive_sa(const uint8_t *T, int64_t n, uint32_t *sa);

/* Prefix doubling with discarding in inverse-suffix-array form
 * (Section 2.1: Algorithm 1 for the loop, Algorithm 2 CmpName plus the max
 * PrefixSum for head-rank names, Algorithm 4 for fetching the partner name
 * through the ISA, Algorithms 5/6 for discarding unique names and for the
 * NameDiscarding renaming rule).
 *
 * h0 = number of characters in the initial names (the paper uses 2: the
 *      pairs (T[i], T[i+1]) of Algorithm 1).
 * sa, isa: outputs of n entries each (isa may be NULL).
 * trace: if not NULL, the name of every position after the initial naming
 *      and after each refinement round is written to trace[k*n .. k*n+n)
 *      for k < trace_cap.
 * Returns the number of refinement rounds after the initial naming.
 *
 * Readings taken where the paper is silent, garbled or inconsistent:
 *  - the partner name is ISA[i+h]+1 and the sentinel past the end is 0
 *    (the literal sentinel 0 collides with the real name 0);
 *  - the loop runs until every name is unique (the bound ceil(log2 n)-1 of
 *    Algorithm 1 is one round short);
 *  - the partner offset is the current resolved length h (i + 2^k in the
 *    paper's indexing);
 *  - NameDiscarding: a new group iff the old names differ, a new subgroup iff
 *    the old names agree and the partner names differ; the new name is
 *    r + (subgroup start - group start);
 *  - all partner names of a round are read before any name of that round
 *    is rewritten. */
int64_t oracle_pd_sa(const uint8_t *T, int64_t n, int64_t h0, uint32_t *sa,
                     uint32_t *isa, uint32_t *trace, int64_t trace_cap);

/* Prefix doubling generalised to a-fold growth (Section 2.1, Prefix
 * Quadrupling): a round sorts each group by the tuple of the names of
 * i + h, i + 2h, ..., i + (a-1)h (each + 1, 0 past the end), in place of
 * the single partner name, so the resolved length grows from h to a*h; the
 * comparison (lexicographic on the tuple) and NameDiscarding (a new
 * subgroup where the tuple changes) are adapted accordingly, everything
 * else is oracle_pd_sa, which is this function with a = 2. a in [2, 4];
 * returns -1 for any other a, else the number of refinement rounds. */
int64_t oracle_pq_sa(const uint8_t *T, int64_t n, int64_t h0, int64_t a, uint32_t *sa,
                     uint32_t *isa, uint32_t *trace, int64_t trace_cap);

/* The recursion text of DC7's first level (Section 2.2, Algorithms 8-9):
 * the sample positions of the difference cover D7 = {0, 1, 3} modulo 7,
 * taken class by class (all i = 0 mod 7, then 1, then 3, each in text
 * order, each class running up to and including the first position whose
 * 7-character window reaches the end of the text: i <= n), each replaced
 * by its lexicographic name: 1 + the number of distinct 7-character
 * windows smaller than its own (characters past the end compare as the
 * end of text, below every byte). Writes m names to out (capacity
 * 3 * (n / 7 + 1)) and returns m. */
int64_t oracle_dc7_names(const uint8_t *T, int64_t n, uint32_t *out);

/* Checker of Burkhardt & Kaerkkaeinen (CPM 2003) for the definition above:
 * SA is a permutation of [0,n) and, for every adjacent pair a = SA[j],
 * b = SA[j+1], (T[a], rank(a+1)) < (T[b], rank(b+1)) with rank(n) = -1.
 * Returns 0 if SA is the suffix array of T; 1 if SA is not a permutation;
 * 2 if an adjacent pair is out of order. *bad (if not NULL) receives the
 * offending index. Linear time; any n. */
int oracle_check_sa(const uint8_t *T, int64_t n, const uint32_t *sa, int64_t *bad);

/* SA is a permutation of [0, n): every entry below n and none repeated
 * (a bitmap of n bits). Returns 0 if so, else 1 + the first bad index in
 * *bad. Linear time, n / 8 bytes of memory. */
int oracle_check_permutation(const uint32_t *sa, int64_t n, int64_t *bad);

/* Direct lexicographic check of sampled adjacent pairs (Section 2: SA lists
 * the suffixes in increasing lexicographic order, all distinct):
 * T[SA[j],n) < T[SA[j+1],n), strictly, for each j in idx[0..count).
 * Returns the number of sampled j that violate it; an entry SA[j] or
 * SA[j+1] >= n counts as a violation, a j with no pair (j < 0 or
 * j + 1 >= n) is skipped, and a j listed twice counts twice. */
int64_t oracle_check_adjacent(const uint8_t *T, int64_t n, const uint32_t *sa,
                              const int64_t *idx, int64_t count);

/* Rank of one suffix by counting (Section 2: ISA[i] = lexicographic rank):
 * the number of suffixes smaller than T[i,n). O(n * LCP). */
int64_t oracle_suffix_rank(const uint8_t *T, int64_t n, int64_t i);

/* Burrows-Wheeler transform of T$ from SA (n+1 rows; row 0 is the suffix $).
 * bwt[r] = the character preceding the r-th smallest suffix; the row whose
 * suffix is T itself holds $ (stored as 0) and its index goes to *primary. */
void oracle_bwt(const uint8_t *T, int64_t n, const uint32_t *sa, uint8_t *bwt,
                int64_t *primary);

/* Inverts oracle_bwt by LF-mapping; writes n bytes to out. Returns 0. */
int oracle_bwt_invert(const uint8_t *bwt, int64_t n, int64_t primary, uint8_t *out);

/* Longest common prefix of the suffixes T[a,n) and T[b,n): the number of
 * leading characters they share, compared one by one (Section 2's suffix
 * order; the LCP array of Section 3's future work is built from it). */
int64_t oracle_lcp_pair(const uint8_t *T, int64_t n, int64_t a, int64_t b);

/* LCP array by its definition: lcp[0] = 0 and, for j >= 1, lcp[j] =
 * oracle_lcp_pair(sa[j-1], sa[j]) for the suffix array sa of T.
 * O(n * average LCP). */
void oracle_lcp(const uint8_t *T, int64_t n, const uint32_t *sa, uint32_t *lcp);

#ifdef __cplusplus
}
#endif
#endif
