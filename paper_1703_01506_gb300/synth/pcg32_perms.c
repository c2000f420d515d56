/*
 * Seeded relabelling lists: PCG32 (O'Neill 2014, "PCG: A Family of Simple
 * Fast Space-Efficient Statistically Good Algorithms for Random Number
 * Generation", the XSH-RR output on a 64-bit LCG) driving Fisher-Yates
 * shuffles. Input generation only: it holds none of the method's
 * arithmetic and serves both the CUDA path and the oracle.
 */
#include <stdint.h>

typedef struct {
  uint64_t state;
  uint64_t inc;
} pcg32_t;

static uint32_t pcg32_next(pcg32_t* g) {
  uint64_t old = g->state;
  g->state = old * 6364136223846793005ULL + g->inc;
  uint32_t xorshifted = (uint32_t)(((old >> 18u) ^ old) >> 27u);
  uint32_t rot = (uint32_t)(old >> 59u);
  return (xorshifted >> rot) | (xorshifted << ((-rot) & 31u));
}

static void pcg32_seed(pcg32_t* g, uint64_t initstate, uint64_t initseq) {
  g->state = 0u;
  g->inc = (initseq << 1u) | 1u;
  pcg32_next(g);
  g->state += initstate;
  pcg32_next(g);
}

/* Unbiased draw in [0, bound) by rejecting the low 2^32 mod bound values. */
static uint32_t pcg32_bounded(pcg32_t* g, uint32_t bound) {
  uint32_t threshold = (uint32_t)(-bound) % bound;
  for (;;) {
    uint32_t r = pcg32_next(g);
    if (r >= threshold) return r % bound;
  }
}

/* First `count` raw outputs (for checking against published values). */
void pcg32_raw(uint64_t initstate, uint64_t initseq, int64_t count, uint32_t* out) {
  pcg32_t g;
  pcg32_seed(&g, initstate, initseq);
  for (int64_t k = 0; k < count; ++k) out[k] = pcg32_next(&g);
}

/*
 * P rows, each a uniformly random permutation of 0..n-1: every row starts
 * from the identity and is shuffled by Fisher-Yates from the top index
 * down (i = n-1 .. 1, j = bounded(i+1), swap). One generator stream for
 * all rows, in row order.
 */
void pcg32_fisher_yates(uint64_t initstate, uint64_t initseq, int32_t n, int64_t P,
                        int32_t* out) {
  pcg32_t g;
  pcg32_seed(&g, initstate, initseq);
  for (int64_t p = 0; p < P; ++p) {
    int32_t* row = out + p * (int64_t)n;
    for (int32_t s = 0; s < n; ++s) row[s] = s;
    for (int32_t i = n - 1; i >= 1; --i) {
      uint32_t j = pcg32_bounded(&g, (uint32_t)i + 1u);
      int32_t tmp = row[i];
      row[i] = row[j];
      row[j] = tmp;
    }
  }
}
