/* Seeded synthetic workload generators for suffix-array construction.
 *
 * This module holds no suffix-sorting arithmetic. It only produces input
 * texts, so both the CPU oracle (oracle/) and the CUDA path draw identical
 * inputs from it without sharing any code with each other.
 *
 * Every generator is deterministic and bit-reproducible across x86_64 and
 * aarch64: the random stream is xoshiro256** (Blackman & Vigna, 2018) seeded
 * through SplitMix64 (Steele, Lea & Flood, 2014), and the only floating-point
 * work uses +, -, *, / with contraction disabled plus the series-based
 * gen_log / gen_exp below (no libm), so both machines round identically.
 *
 * The workloads follow the five benchmark recipes of the project:
 *   1  i.i.d. uniform over the bytes 'A','C','G','T'
 *   2  a base of n/256 symbols drawn Zipf(s=1.1) over the byte values 1..255
 *      (Zipf rank k -> byte value k), tiled 256 times, each copy with
 *      round(0.001 * base) distinct positions substituted by a different Zipf
 *      draw (long repeats force many doubling rounds)
 *   3  order-3 Markov chain over 'A','C','G','T' with a seeded random
 *      transition table (each of the 64 context rows ~ Dirichlet(1,1,1,1)),
 *      plus copied segments of length U[1024, 102400] (clamped to n/4) taken
 *      from the pre-copy text until 5% of n is covered
 *   4  a batch of texts with log-uniform lengths in [lo, hi], i.i.d. uniform
 *      'ACGT'
 *   5  a Poisson request stream: exponential inter-arrival times, log-uniform
 *      sizes, a fair coin choosing recipe-1 DNA or i.i.d. Zipf(1.1) bytes.
 */
#ifndef GBSA_GEN_H
#define GBSA_GEN_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Recipe 1: n bytes, uniform over "ACGT". */
void gen_dna_uniform(uint64_t seed, uint64_t n, uint8_t *out);

/* Recipe 2: repeated Zipf(1.1) base with 0.1% substitutions per copy.
 * copies = 256 (or fewer when n < 256); base = ceil(n / copies). */
void gen_zipf_repeats(uint64_t seed, uint64_t n, uint8_t *out);

/* Recipe 3: order-3 Markov DNA plus 5% copied segments.
 * scratch must hold n bytes (the pre-copy snapshot). */
void gen_markov_dna(uint64_t seed, uint64_t n, uint8_t *out, uint8_t *scratch);

/* i.i.d. Zipf(1.1) bytes over 1..255 (the byte half of recipe 5). */
void gen_zipf_iid(uint64_t seed, uint64_t n, uint8_t *out);

/* Recipe 4 lengths: count lengths, log-uniform in [lo, hi], rounded. */
void gen_batch_lengths(uint64_t seed, uint32_t count, uint64_t lo, uint64_t hi,
                       uint64_t *lengths);

/* Recipe 5 arrivals: count requests at rate lambda (req/s). Writes arrival
 * times in seconds, sizes (log-uniform in [lo, hi]) and kinds (0 = DNA
 * uniform, 1 = Zipf bytes). */
void gen_request_stream(uint64_t seed, uint32_t count, double lambda,
                        uint64_t lo, uint64_t hi, double *arrival_s,
                        uint64_t *sizes, uint8_t *kinds);

/* Bytes uniform over the whole range 0..255 (edge-case tests). */
void gen_bytes_uniform(uint64_t seed, uint64_t n, uint8_t *out);

/* Deterministic natural log and exp (series-based, no libm). */
double gen_log(double x);
double gen_exp(double x);

#ifdef __cplusplus
}
#endif
#endif
