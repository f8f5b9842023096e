/*
 * pss_zipf.h — seeded synthetic input generator (host and device).
 *
 * This is the single module that both the CUDA path and the CPU oracle use:
 * it only manufactures input streams and holds none of the Space Saving
 * arithmetic.  The paper evaluates on synthetic streams "derived from a
 * zipfian distribution" with skew 1.1 and 1.8 (Section 4.1); its datasets are
 * not published, so seeded stand-ins are generated here.
 *
 * Definition of the stream (fixed, documented, identical on host and device):
 *
 *   item(seed, stream, i) = rank_to_item( Zipf_{s,U}(seed, stream, i), log2U )
 *
 *   - Zipf_{s,U}: P(rank = r) proportional to r^-s for r in [1, U], drawn by
 *     rejection-inversion (W. Hormann and G. Derflinger, "Rejection-inversion
 *     to generate variates from monotone discrete distributions", ACM TOMACS
 *     6(3), 1996), with its quick-acceptance bound.  Attempt a of item i
 *     consumes one uniform from the counter-based generator below.
 *   - Uniforms: Philox4x32-10 (J. Salmon, M. Moraes, R. Dror, D. Shaw,
 *     "Parallel random numbers: as easy as 1, 2, 3", SC 2011), key =
 *     (seed low word, seed high word), counter = (i low word, i high word,
 *     stream, attempt / 2); attempt a uses output words 2(a%2), 2(a%2)+1,
 *     turned into (j + 0.5) * 2^-52 with j a 52-bit integer, so u is in (0,1).
 *   - rank_to_item: a fixed bijection of r-1 on [0, 2^log2U) (two rounds of
 *     odd-multiply and xor-shift modulo 2^log2U) so that frequent items are
 *     scattered over the universe instead of being 0, 1, 2, ...
 *
 * Bit-exact reproducibility: all floating point is IEEE double with
 * operations +, -, *, / and explicit fused multiply-add (each correctly
 * rounded), and nothing else is contracted: device code goes through the
 * __d*_rn / __fma_rn intrinsics, host code uses C's fma and must be compiled
 * with -ffp-contract=off.  log and exp are this file's own (range reduction
 * plus series from the mathematics), so that no platform libm enters the
 * result; the sampler uses table-driven versions whose tables the accurate
 * ones build (pssg_tables, identical on both sides).
 */
#ifndef PSS_ZIPF_H_
#define PSS_ZIPF_H_

#include <math.h>
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define PSSG_FN static __host__ __device__ __forceinline__
#else
#define PSSG_FN static inline
#if defined(__GNUC__) && !defined(__clang__)
#pragma GCC optimize("fp-contract=off")
#endif
#endif

#if defined(__CUDA_ARCH__)
#define PSSG_FMA(a, b, c) __fma_rn((a), (b), (c))
#define PSSG_MUL(a, b) __dmul_rn((a), (b))
#define PSSG_ADD(a, b) __dadd_rn((a), (b))
#define PSSG_SUB(a, b) __dsub_rn((a), (b))
#define PSSG_DIV(a, b) __ddiv_rn((a), (b))
#else
#define PSSG_FMA(a, b, c) fma((a), (b), (c))
#define PSSG_MUL(a, b) ((a) * (b))
#define PSSG_ADD(a, b) ((a) + (b))
#define PSSG_SUB(a, b) ((a) - (b))
#define PSSG_DIV(a, b) ((a) / (b))
#endif

/* ---------------------------------------------------------------- Philox */

/* Philox4x32 with 10 rounds; c is the counter (in) and the output (out). */
PSSG_FN void pssg_philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u; /* Weyl key schedule: golden ratio */
      k1 += 0xBB67AE85u; /* and sqrt(3) - 1 */
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
  }
}

/* Uniform in (0,1) from two 32-bit words: (j + 0.5) / 2^52, j has 52 bits. */
PSSG_FN double pssg_u01(uint32_t w0, uint32_t w1) {
  uint64_t j = ((uint64_t)(w0 >> 6) << 26) | (uint64_t)(w1 >> 6);
  return PSSG_MUL(PSSG_ADD((double)j, 0.5), 0x1p-52);
}

/* ------------------------------------------------- own elementary functions */

PSSG_FN uint64_t pssg_bits(double x) { uint64_t b; memcpy(&b, &x, 8); return b; }
PSSG_FN double pssg_from_bits(uint64_t b) { double x; memcpy(&x, &b, 8); return x; }

/* floor for |v| < 2^62 */
PSSG_FN double pssg_floor(double v) {
  int64_t i = (int64_t)v; /* truncation toward zero: exact */
  if ((double)i > v) i -= 1;
  return (double)i;
}

/* 2^e for -1022 <= e <= 1023, exact. */
PSSG_FN double pssg_pow2(int e) { return pssg_from_bits((uint64_t)(e + 1023) << 52); }

/* ln 2 split so that n * PSSG_LN2_HI is exact for |n| < 2^21. */
#define PSSG_LN2_HI 0x1.62e42fee00000p-1
#define PSSG_LN2_LO 0x1.a39ef35793c76p-33
#define PSSG_INV_LN2 0x1.71547652b82fep+0
#define PSSG_SQRT2 0x1.6a09e667f3bcdp+0

/* Natural log for positive normal x: x = 2^e f with f in (sqrt(1/2), sqrt 2],
 * log f = 2 atanh(z), z = (f-1)/(f+1), |z| < 0.172, atanh series to z^21
 * (the next term is below 1e-18 relative). */
PSSG_FN double pssg_log(double x) {
  uint64_t b = pssg_bits(x);
  int e = (int)((b >> 52) & 0x7FF) - 1023;
  double f = pssg_from_bits((b & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull);
  if (f > PSSG_SQRT2) { f = PSSG_MUL(f, 0.5); e += 1; }
  double z = PSSG_DIV(PSSG_SUB(f, 1.0), PSSG_ADD(f, 1.0));
  double z2 = PSSG_MUL(z, z);
  double q = 1.0 / 21.0;
  q = PSSG_FMA(q, z2, 1.0 / 19.0);
  q = PSSG_FMA(q, z2, 1.0 / 17.0);
  q = PSSG_FMA(q, z2, 1.0 / 15.0);
  q = PSSG_FMA(q, z2, 1.0 / 13.0);
  q = PSSG_FMA(q, z2, 1.0 / 11.0);
  q = PSSG_FMA(q, z2, 1.0 / 9.0);
  q = PSSG_FMA(q, z2, 1.0 / 7.0);
  q = PSSG_FMA(q, z2, 1.0 / 5.0);
  q = PSSG_FMA(q, z2, 1.0 / 3.0);
  q = PSSG_FMA(q, z2, 1.0);
  double lf = PSSG_MUL(PSSG_MUL(2.0, z), q);
  double de = (double)e;
  return PSSG_FMA(de, PSSG_LN2_HI, PSSG_ADD(PSSG_MUL(de, PSSG_LN2_LO), lf));
}

/* exp(x) for |x| < 700: x = n ln2 + r, |r| <= ln2/2, Taylor series of e^r to
 * r^14/14! (truncation below 4e-18 relative), then scale by 2^n. */
PSSG_FN double pssg_exp(double x) {
  double nd = pssg_floor(PSSG_FMA(x, PSSG_INV_LN2, 0.5));
  double r = PSSG_SUB(PSSG_SUB(x, PSSG_MUL(nd, PSSG_LN2_HI)), PSSG_MUL(nd, PSSG_LN2_LO));
  double p = 1.0 / 87178291200.0; /* 1/14! */
  p = PSSG_FMA(p, r, 1.0 / 6227020800.0);
  p = PSSG_FMA(p, r, 1.0 / 479001600.0);
  p = PSSG_FMA(p, r, 1.0 / 39916800.0);
  p = PSSG_FMA(p, r, 1.0 / 3628800.0);
  p = PSSG_FMA(p, r, 1.0 / 362880.0);
  p = PSSG_FMA(p, r, 1.0 / 40320.0);
  p = PSSG_FMA(p, r, 1.0 / 5040.0);
  p = PSSG_FMA(p, r, 1.0 / 720.0);
  p = PSSG_FMA(p, r, 1.0 / 120.0);
  p = PSSG_FMA(p, r, 1.0 / 24.0);
  p = PSSG_FMA(p, r, 1.0 / 6.0);
  p = PSSG_FMA(p, r, 0.5);
  p = PSSG_FMA(p, r, 1.0);
  p = PSSG_FMA(p, r, 1.0);
  return PSSG_MUL(p, pssg_pow2((int)nd));
}

/* ------------------------------------------- table-driven log and exp
 *
 * The sampler's log and exp: the same mathematics with a finer range
 * reduction, so that short polynomials and no division suffice.
 *   log x: x = 2^e f, f in [1, 2); c_j = 1 + (j + 1/2)/128 for the top seven
 *     bits j of f; log x = e log 2 + log c_j + log(1 + d), d = f/c_j - 1 =
 *     fma(f, 1/c_j, -1), |d| <= 2^-8, series of log(1 + d) to d^7 (the next
 *     term is below 2^-59 relative).
 *   exp x: x = m L + r with L = log 2 / 64 and |r| <= L/2; exp x = 2^(m div 64)
 *     exp((m mod 64) L) e^r, series of e^r - 1 to r^6 (next term < 2e-20).
 * The tables hold 1/c_j (a correctly rounded quotient), log c_j and
 * exp(j L), each computed by this file's own pssg_log / pssg_exp above, so
 * host and device build identical tables. */

#define PSSG_LOG_TAB 128
#define PSSG_EXP_TAB 64
#define PSSG_L_HI 0x1.62e42fee00000p-7  /* PSSG_LN2_HI / 64 */
#define PSSG_L_LO 0x1.a39ef35793c76p-39 /* PSSG_LN2_LO / 64 */
#define PSSG_INV_L 0x1.71547652b82fep+6 /* 64 / ln 2 */

typedef struct {
  double rc[PSSG_LOG_TAB]; /* 1 / c_j */
  double lc[PSSG_LOG_TAB]; /* log c_j */
  double t2[PSSG_EXP_TAB]; /* exp(j L) */
} pssg_tables;

/* Entry i of every table that has one (i < PSSG_LOG_TAB covers all). */
PSSG_FN void pssg_tables_entry(pssg_tables* tb, int i) {
  if (i < PSSG_LOG_TAB) {
    double c = PSSG_ADD(1.0, PSSG_MUL(PSSG_ADD((double)i, 0.5), 0x1p-7)); /* exact */
    tb->rc[i] = PSSG_DIV(1.0, c);
    tb->lc[i] = pssg_log(c);
  }
  if (i < PSSG_EXP_TAB) {
    double di = (double)i;
    tb->t2[i] = pssg_exp(PSSG_ADD(PSSG_MUL(di, PSSG_L_HI), PSSG_MUL(di, PSSG_L_LO)));
  }
}

PSSG_FN void pssg_tables_init(pssg_tables* tb) {
  for (int i = 0; i < PSSG_LOG_TAB; ++i) pssg_tables_entry(tb, i);
}

/* log of a positive normal x; with cu != 0, log(x) + cu where cu is a
 * correction far below ulp(x) (used by log1p). */
PSSG_FN double pssg_log_tc(const pssg_tables* tb, double x, double c) {
  uint64_t b = pssg_bits(x);
  int e = (int)((b >> 52) & 0x7FF) - 1023;
  uint64_t mant = b & 0x000FFFFFFFFFFFFFull;
  int j = (int)(mant >> 45);
  double f = pssg_from_bits(mant | 0x3FF0000000000000ull);
  double d = PSSG_FMA(f, tb->rc[j], -1.0);
  /* log(1 + d) = d + d^2 (-1/2 + d/3 - d^2/4 + d^3/5 - d^4/6 + d^5/7) */
  double q = 1.0 / 7.0;
  q = PSSG_FMA(q, d, -1.0 / 6.0);
  q = PSSG_FMA(q, d, 1.0 / 5.0);
  q = PSSG_FMA(q, d, -1.0 / 4.0);
  q = PSSG_FMA(q, d, 1.0 / 3.0);
  q = PSSG_FMA(q, d, -0.5);
  double l1 = PSSG_FMA(PSSG_MUL(d, d), q, d);
  /* c / x with 1/x ~ rc_j 2^-e (c is tiny: the approximation is ample) */
  l1 = PSSG_FMA(c, PSSG_MUL(tb->rc[j], pssg_pow2(-e)), l1);
  double de = (double)e;
  return PSSG_ADD(PSSG_FMA(de, PSSG_LN2_HI, tb->lc[j]), PSSG_FMA(de, PSSG_LN2_LO, l1));
}

PSSG_FN double pssg_log_t(const pssg_tables* tb, double x) { return pssg_log_tc(tb, x, 0.0); }

/* exp(x) for |x| < 700 */
PSSG_FN double pssg_exp_t(const pssg_tables* tb, double x) {
  double md = pssg_floor(PSSG_FMA(x, PSSG_INV_L, 0.5));
  double r = PSSG_SUB(PSSG_SUB(x, PSSG_MUL(md, PSSG_L_HI)), PSSG_MUL(md, PSSG_L_LO));
  int64_t m = (int64_t)md;
  int j = (int)(m & 63);
  int n = (int)((m - j) / 64);
  double p = 1.0 / 720.0;
  p = PSSG_FMA(p, r, 1.0 / 120.0);
  p = PSSG_FMA(p, r, 1.0 / 24.0);
  p = PSSG_FMA(p, r, 1.0 / 6.0);
  p = PSSG_FMA(p, r, 0.5);
  double em1 = PSSG_FMA(PSSG_MUL(r, r), p, r);
  double t = tb->t2[j];
  return PSSG_MUL(PSSG_FMA(t, em1, t), pssg_pow2(n));
}

/* log(1 + t) / t for |t| < 2^-6 (value 1 at t = 0), series to t^9/10 (next
 * term < 2^-57) */
PSSG_FN double pssg_log1p_over_small(double t) {
  double p = -1.0 / 10.0;
  p = PSSG_FMA(p, t, 1.0 / 9.0);
  p = PSSG_FMA(p, t, -1.0 / 8.0);
  p = PSSG_FMA(p, t, 1.0 / 7.0);
  p = PSSG_FMA(p, t, -1.0 / 6.0);
  p = PSSG_FMA(p, t, 1.0 / 5.0);
  p = PSSG_FMA(p, t, -1.0 / 4.0);
  p = PSSG_FMA(p, t, 1.0 / 3.0);
  p = PSSG_FMA(p, t, -1.0 / 2.0);
  return PSSG_FMA(p, t, 1.0);
}

/* (e^w - 1) / w for |w| < 2^-5 (value 1 at w = 0), series to w^9/10! (next
 * term < 2^-60) */
PSSG_FN double pssg_expm1_over_small(double w) {
  double p = 1.0 / 39916800.0;
  p = PSSG_FMA(p, w, 1.0 / 3628800.0);
  p = PSSG_FMA(p, w, 1.0 / 362880.0);
  p = PSSG_FMA(p, w, 1.0 / 40320.0);
  p = PSSG_FMA(p, w, 1.0 / 5040.0);
  p = PSSG_FMA(p, w, 1.0 / 720.0);
  p = PSSG_FMA(p, w, 1.0 / 120.0);
  p = PSSG_FMA(p, w, 1.0 / 24.0);
  p = PSSG_FMA(p, w, 1.0 / 6.0);
  p = PSSG_FMA(p, w, 0.5);
  return PSSG_FMA(p, w, 1.0);
}

/* ------------------------------------------------ Zipf by rejection-inversion */

typedef struct {
  double s;        /* exponent, s > 0 */
  double one_m_s;  /* 1 - s */
  double inv_1ms;  /* 1 / (1 - s), 0 when s = 1 */
  double h_x1;     /* H(3/2) - h(1): left end of the sampled interval */
  double h_n;      /* H(N + 1/2): right end */
  double squeeze;  /* k - x <= squeeze accepts without evaluating H and h */
  uint64_t n;      /* number of ranks N = U */
} pssg_zipf;

/* H(x) = integral of t^-s from 1 to x = (x^(1-s) - 1) / (1 - s) (log x at s = 1) */
PSSG_FN double pssg_zipf_H(const pssg_zipf* z, const pssg_tables* tb, double x) {
  double lx = pssg_log_t(tb, x);
  double w = PSSG_MUL(z->one_m_s, lx);
  if (w > -0x1p-5 && w < 0x1p-5) return PSSG_MUL(lx, pssg_expm1_over_small(w));
  return PSSG_MUL(PSSG_SUB(pssg_exp_t(tb, w), 1.0), z->inv_1ms);
}

/* H^-1(y) = exp(log(1 + (1-s) y) / (1 - s)) (exp y at s = 1) */
PSSG_FN double pssg_zipf_Hinv(const pssg_zipf* z, const pssg_tables* tb, double y) {
  double t = PSSG_MUL(z->one_m_s, y);
  if (t > -0x1p-6 && t < 0x1p-6) return pssg_exp_t(tb, PSSG_MUL(y, pssg_log1p_over_small(t)));
  double u = PSSG_ADD(1.0, t);
  double c = PSSG_SUB(t, PSSG_SUB(u, 1.0)); /* the rounding error of u */
  return pssg_exp_t(tb, PSSG_MUL(pssg_log_tc(tb, u, c), z->inv_1ms));
}

/* h(x) = x^-s */
PSSG_FN double pssg_zipf_h(const pssg_zipf* z, const pssg_tables* tb, double x) {
  return pssg_exp_t(tb, PSSG_MUL(-z->s, pssg_log_t(tb, x)));
}

PSSG_FN void pssg_zipf_init(pssg_zipf* z, const pssg_tables* tb, double s, uint64_t n) {
  z->s = s;
  z->one_m_s = PSSG_SUB(1.0, s);
  z->inv_1ms = z->one_m_s == 0.0 ? 0.0 : PSSG_DIV(1.0, z->one_m_s);
  z->n = n;
  z->h_x1 = PSSG_SUB(pssg_zipf_H(z, tb, 1.5), 1.0);
  z->h_n = pssg_zipf_H(z, tb, PSSG_ADD((double)n, 0.5));
  /* the quick acceptance bound of rejection-inversion: 2 - H^-1(H(5/2) - h(2)) */
  z->squeeze = PSSG_SUB(2.0, pssg_zipf_Hinv(z, tb, PSSG_SUB(pssg_zipf_H(z, tb, 2.5),
                                                           pssg_zipf_h(z, tb, 2.0))));
}

/* One attempt with uniform u: 0 if rejected, else the rank in [1, N].  The
 * sampled variable is y uniform on (H(N + 1/2), H(3/2) - h(1)]; x = H^-1(y),
 * k = the integer nearest x.  The accepted part of the cell of rank k is
 * [H(k+1/2) - h(k), H(k+1/2)], of length h(k), so P(k) is proportional to k^-s. */
PSSG_FN uint64_t pssg_zipf_try(const pssg_zipf* z, const pssg_tables* tb, double u) {
  double y = PSSG_ADD(z->h_n, PSSG_MUL(u, PSSG_SUB(z->h_x1, z->h_n)));
  double x = pssg_zipf_Hinv(z, tb, y);
  double kd = pssg_floor(PSSG_ADD(x, 0.5));
  if (kd < 1.0) kd = 1.0;
  if (kd > (double)z->n) kd = (double)z->n;
  uint64_t k = (uint64_t)kd;
  double kk = (double)k;
  if (PSSG_SUB(kk, x) <= z->squeeze) return k;
  if (y >= PSSG_SUB(pssg_zipf_H(z, tb, PSSG_ADD(kk, 0.5)), pssg_zipf_h(z, tb, kk))) return k;
  return 0;
}

#define PSSG_MAX_ATTEMPTS 64

/* Rank of item index i of stream `stream` under `seed`.  After
 * PSSG_MAX_ATTEMPTS rejections (probability far below 1e-40) rank 1 is
 * returned, identically on both sides. */
PSSG_FN uint64_t pssg_zipf_rank(const pssg_zipf* z, const pssg_tables* tb, uint64_t seed,
                                uint32_t stream, uint64_t i) {
  for (uint32_t a = 0; a < PSSG_MAX_ATTEMPTS; a += 2) {
    uint32_t c[4] = {(uint32_t)i, (uint32_t)(i >> 32), stream, a >> 1};
    pssg_philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    uint64_t k = pssg_zipf_try(z, tb, pssg_u01(c[0], c[1]));
    if (k) return k;
    k = pssg_zipf_try(z, tb, pssg_u01(c[2], c[3]));
    if (k) return k;
  }
  return 1;
}

/* Bijection of [0, 2^b) (1 <= b <= 64) applied to r - 1. */
PSSG_FN uint64_t pssg_rank_to_item(uint64_t r, int b) {
  uint64_t mask = (b >= 64) ? ~0ull : ((1ull << b) - 1ull);
  int sh = (b + 1) / 2;
  uint64_t x = (r - 1ull) & mask;
  x = (x * 0x9E3779B97F4A7C15ull) & mask;
  x ^= x >> sh;
  x = (x * 0xBF58476D1CE4E5B9ull) & mask;
  x ^= x >> sh;
  return x;
}

/* Item i of the stream (seed, stream, s, U = 2^log2u). */
PSSG_FN uint64_t pssg_zipf_item(const pssg_zipf* z, const pssg_tables* tb, int log2u,
                                uint64_t seed, uint32_t stream, uint64_t i) {
  return pssg_rank_to_item(pssg_zipf_rank(z, tb, seed, stream, i), log2u);
}

#endif /* PSS_ZIPF_H_ */
