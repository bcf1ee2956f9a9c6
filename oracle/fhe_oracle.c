/*
 * CPU oracle for RNS-CKKS hybrid key switching -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the plain, slow, obviously-correct reference against which the
 * CUDA library is checked residue by residue.  Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or constant with the CUDA library: every constant (roots of unity,
 * inverses, base-conversion tables) is recomputed here from its definition.
 *
 * Arithmetic style: every product of two residues is formed as a 64-bit
 * integer and reduced with `%`; sums of products use unsigned __int128 and a
 * single `%`.  No Montgomery, Shoup or Barrett forms, no lazy ranges.
 *
 * Polynomial layout: limb-major, `[limb][N]` uint32, every residue in [0, q).
 * A "prime list" is the ciphertext primes q_0..q_{L-1} followed by the special
 * primes p_0..p_{K-1}; extended-basis polynomials use the same order
 * (q-limbs 0..level-1, then the K p-limbs).
 *
 * Paper sections followed (Theodosian, arXiv 2512.18345):
 *   - Section II-A: a polynomial is an L x N matrix of word-sized residues,
 *     row i reduced modulo its own prime.
 *   - Section II-B: NTT / INTT butterflies BFly_NTT(x,y,w) = (x+wy, x-wy) and
 *     BFly_INTT(x,y,w) = (x+y, w(x-y)); BConv = Red(T . a) with
 *     T[i][j] = (Qstar/Q_j) mod P_i and one final reduction (Section III-C).
 *   - Section IV, Fig. "keysw": key switching in three stages (ModUp =
 *     INTT + BConv + NTT; inner product with the key; ModDown =
 *     INTT + BConv + NTT + combine).
 * The key-switching mathematics the paper leaves to its citations (hybrid key
 * switching with dnum digits, rotation by the Galois map X -> X^(5^r), floor
 * rescale) is restated here in its textbook RNS form.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

/* ---------------------------------------------------------------- scalars */

static uint32_t mulmod(uint32_t a, uint32_t b, uint32_t q) { return (uint32_t)(((uint64_t)a * b) % q); }
static uint32_t addmod(uint32_t a, uint32_t b, uint32_t q) { return (uint32_t)(((uint64_t)a + b) % q); }
static uint32_t submod(uint32_t a, uint32_t b, uint32_t q) { return (uint32_t)(((uint64_t)a + q - b) % q); }

uint32_t orc_powmod(uint32_t a, uint64_t e, uint32_t q) {
  uint64_t r = 1 % q, b = a % q;
  while (e) {
    if (e & 1) r = (r * b) % q;
    b = (b * b) % q;
    e >>= 1;
  }
  return (uint32_t)r;
}

/* inverse by Fermat (q prime) */
uint32_t orc_invmod(uint32_t a, uint32_t q) { return orc_powmod(a, (uint64_t)q - 2, q); }

/* psi: a primitive 2N-th root of unity mod q, psi = g^((q-1)/2N) for the
 * smallest integer g >= 2 whose power has psi^N = -1 (mod q). */
uint32_t orc_psi(uint32_t q, uint32_t N) {
  for (uint32_t g = 2; g < q; g++) {
    uint32_t psi = orc_powmod(g, ((uint64_t)q - 1) / (2ull * N), q);
    if (orc_powmod(psi, N, q) == q - 1) return psi;
  }
  return 0;
}

static uint32_t bitrev(uint32_t x, int bits) {
  uint32_t r = 0;
  for (int i = 0; i < bits; i++) r |= ((x >> i) & 1u) << (bits - 1 - i);
  return r;
}

static int log2u(uint32_t n) {
  int l = 0;
  while ((1u << l) < n) l++;
  return l;
}

/* table[k] = root^brv(k) for k < N (powers by repeated multiplication) */
static uint32_t *psi_powers_bitrev(uint32_t root, uint32_t N, int logn, uint32_t q) {
  uint32_t *pow_nat = (uint32_t *)malloc(sizeof(uint32_t) * N);
  uint32_t *pw = (uint32_t *)malloc(sizeof(uint32_t) * N);
  pow_nat[0] = 1 % q;
  for (uint32_t k = 1; k < N; k++) pow_nat[k] = mulmod(pow_nat[k - 1], root, q);
  for (uint32_t k = 0; k < N; k++) pw[k] = pow_nat[bitrev(k, logn)];
  free(pow_nat);
  return pw;
}

/* ---------------------------------------------------------------- NTT */

/*
 * Forward negacyclic NTT of one limb, in place, natural order in, bit-reversed
 * order out:  out[i] = sum_n a[n] * psi^((2 brv(i) + 1) n)  (mod q).
 * Textbook iterative Cooley-Tukey with the psi powers merged into the
 * butterflies (Section II-B, BFly_NTT), stage m uses psi^brv(m + i).
 */
void orc_ntt(uint32_t *a, uint32_t N, uint32_t q) {
  int logn = log2u(N);
  uint32_t *pw = psi_powers_bitrev(orc_psi(q, N), N, logn, q);
  uint32_t t = N;
  for (uint32_t m = 1; m < N; m <<= 1) {
    t >>= 1;
    for (uint32_t i = 0; i < m; i++) {
      uint32_t w = pw[m + i];
      for (uint32_t j = 2 * i * t; j < 2 * i * t + t; j++) {
        uint32_t x = a[j], y = mulmod(w, a[j + t], q);
        a[j] = addmod(x, y, q);
        a[j + t] = submod(x, y, q);
      }
    }
  }
  free(pw);
}

/*
 * Inverse of orc_ntt: bit-reversed order in, natural order out.  Gentleman-
 * Sande butterflies (Section II-B, BFly_INTT) with psi^-brv(m + i), then a
 * final scaling by N^-1.
 */
void orc_intt(uint32_t *a, uint32_t N, uint32_t q) {
  int logn = log2u(N);
  uint32_t *pw = psi_powers_bitrev(orc_invmod(orc_psi(q, N), q), N, logn, q);
  uint32_t t = 1;
  for (uint32_t m = N >> 1; m >= 1; m >>= 1) {
    for (uint32_t i = 0; i < m; i++) {
      uint32_t w = pw[m + i];
      for (uint32_t j = 2 * i * t; j < 2 * i * t + t; j++) {
        uint32_t x = a[j], y = a[j + t];
        a[j] = addmod(x, y, q);
        a[j + t] = mulmod(w, submod(x, y, q), q);
      }
    }
    t <<= 1;
  }
  uint32_t n_inv = orc_invmod(N % q, q);
  for (uint32_t j = 0; j < N; j++) a[j] = mulmod(a[j], n_inv, q);
  free(pw);
}

/* limb-wise transforms of an [nlimbs][N] array, limb i modulo primes[i] */
void orc_ntt_limbs(uint32_t *a, int nlimbs, const uint32_t *primes, uint32_t N) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < nlimbs; i++) orc_ntt(a + (size_t)i * N, N, primes[i]);
}

void orc_intt_limbs(uint32_t *a, int nlimbs, const uint32_t *primes, uint32_t N) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < nlimbs; i++) orc_intt(a + (size_t)i * N, N, primes[i]);
}

/* ---------------------------------------------------------------- BConv */

/*
 * Fast base conversion (Section II-B "BConv", Section III-C table formula):
 *   y_j   = x_j * [(Qstar/q_j)^-1]_{q_j}  mod q_j
 *   out_i = Red( sum_j y_j * T[i][j] ),  T[i][j] = (Qstar/q_j) mod p_i,
 * with Qstar the product of the n_in input primes.  The exact integer sum is
 * formed in 128 bits and reduced once.  Inputs and outputs are in coefficient
 * form.  The result equals (x + e Qstar) mod p_i for some integer e in [0, n_in).
 */
void orc_bconv(const uint32_t *in, int n_in, const uint32_t *q_in, uint32_t *out, int n_out,
               const uint32_t *p_out, uint32_t N) {
  uint32_t *qhat_inv = (uint32_t *)malloc(sizeof(uint32_t) * n_in);
  uint32_t *T = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n_in * n_out);
  for (int j = 0; j < n_in; j++) {
    uint32_t prod = 1 % q_in[j];
    for (int k = 0; k < n_in; k++)
      if (k != j) prod = mulmod(prod, q_in[k] % q_in[j], q_in[j]);
    qhat_inv[j] = orc_invmod(prod, q_in[j]);
  }
  for (int i = 0; i < n_out; i++)
    for (int j = 0; j < n_in; j++) {
      uint32_t prod = 1 % p_out[i];
      for (int k = 0; k < n_in; k++)
        if (k != j) prod = mulmod(prod, q_in[k] % p_out[i], p_out[i]);
      T[(size_t)i * n_in + j] = prod;
    }
  uint32_t *y = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n_in * N);
  for (int j = 0; j < n_in; j++)
    for (uint32_t n = 0; n < N; n++) y[(size_t)j * N + n] = mulmod(in[(size_t)j * N + n], qhat_inv[j], q_in[j]);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n_out; i++)
    for (uint32_t n = 0; n < N; n++) {
      u128 acc = 0;
      for (int j = 0; j < n_in; j++) acc += (u128)y[(size_t)j * N + n] * T[(size_t)i * n_in + j];
      out[(size_t)i * N + n] = (uint32_t)(acc % p_out[i]);
    }
  free(y);
  free(T);
  free(qhat_inv);
}

/* ---------------------------------------------------------------- automorphism */

/*
 * Galois automorphism sigma_k : a(X) -> a(X^k), k odd, on one limb.
 * Coefficient form (the definition): X^n -> X^(nk mod 2N), with X^N = -1.
 */
void orc_automorph_coef(const uint32_t *in, uint32_t *out, uint32_t N, uint32_t k, uint32_t q) {
  for (uint32_t n = 0; n < N; n++) {
    uint64_t e = ((uint64_t)n * k) % (2ull * N);
    if (e < N)
      out[e] = in[n];
    else
      out[e - N] = in[n] ? q - in[n] : 0;
  }
}

/*
 * The same map on a limb in NTT (evaluation) form.  Slot i holds the value at
 * psi^(2 brv(i) + 1); sigma_k(a) evaluated there is a evaluated at
 * psi^((2 brv(i) + 1) k), so out[i] = in[j] with 2 brv(j) + 1 = (2 brv(i) + 1) k
 * mod 2N.  A pure permutation, no sign.
 */
void orc_automorph_ntt(const uint32_t *in, uint32_t *out, uint32_t N, uint32_t k) {
  int logn = log2u(N);
  for (uint32_t i = 0; i < N; i++) {
    uint64_t e = ((2ull * bitrev(i, logn) + 1) * k) % (2ull * N);
    uint32_t j = bitrev((uint32_t)((e - 1) / 2), logn);
    out[i] = in[j];
  }
}

/* k = 5^r mod 2N (r may be negative) */
uint32_t orc_galois_elt(int32_t r, uint32_t N) {
  uint64_t two_n = 2ull * N;
  /* the group <5> mod 2N has order N/2 */
  int64_t rr = r % (int64_t)(N / 2);
  if (rr < 0) rr += N / 2;
  uint64_t k = 1;
  for (int64_t i = 0; i < rr; i++) k = (k * 5) % two_n;
  return (uint32_t)k;
}

/* ---------------------------------------------------------------- key switching */

typedef struct {
  uint32_t N;
  int L;       /* number of ciphertext primes (maximum level) */
  int K;       /* number of special primes */
  int dnum;    /* number of digits */
  const uint32_t *primes; /* L + K primes: q_0..q_{L-1}, p_0..p_{K-1} */
} orc_params;

static int ceil_div(int a, int b) { return (a + b - 1) / b; }

int orc_alpha(const orc_params *P) { return ceil_div(P->L, P->dnum); }
int orc_beta(const orc_params *P, int level) { return ceil_div(level, orc_alpha(P)); }

/* prime of extended-basis limb t at `level`: q_t for t < level, else p_{t-level} */
static uint32_t ext_prime(const orc_params *P, int level, int t) {
  return t < level ? P->primes[t] : P->primes[P->L + (t - level)];
}

/* row of the key array that holds extended limb t at `level` */
static int key_row(const orc_params *P, int level, int t) { return t < level ? t : P->L + (t - level); }

/*
 * ModUp of digit j (stage 1 of key switching, Fig. "keysw"): d is in NTT form
 * over q_0..q_{level-1}.  Digit j is the limbs [j*alpha, min((j+1)*alpha, level)).
 * Output `ext` is [level + K][N] in NTT form: the digit's own limbs are copied
 * from d; every other limb is NTT(BConv(INTT(d restricted to digit j))).
 */
int orc_modup(const orc_params *P, const uint32_t *d, int level, int j, uint32_t *ext) {
  const uint32_t N = P->N;
  int alpha = orc_alpha(P);
  int lo = j * alpha, hi = (j + 1) * alpha < level ? (j + 1) * alpha : level;
  if (lo >= hi) return -1;
  int n_in = hi - lo, n_ext = level + P->K, n_out = n_ext - n_in;
  uint32_t *coef = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n_in * N);
  memcpy(coef, d + (size_t)lo * N, sizeof(uint32_t) * (size_t)n_in * N);
  orc_intt_limbs(coef, n_in, P->primes + lo, N);
  uint32_t *p_out = (uint32_t *)malloc(sizeof(uint32_t) * n_out);
  int *t_out = (int *)malloc(sizeof(int) * n_out);
  int c = 0;
  for (int t = 0; t < n_ext; t++)
    if (t < lo || t >= hi) {
      p_out[c] = ext_prime(P, level, t);
      t_out[c] = t;
      c++;
    }
  uint32_t *conv = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n_out * N);
  orc_bconv(coef, n_in, P->primes + lo, conv, n_out, p_out, N);
  orc_ntt_limbs(conv, n_out, p_out, N);
  for (int t = lo; t < hi; t++) memcpy(ext + (size_t)t * N, d + (size_t)t * N, sizeof(uint32_t) * N);
  for (int i = 0; i < n_out; i++) memcpy(ext + (size_t)t_out[i] * N, conv + (size_t)i * N, sizeof(uint32_t) * N);
  free(conv);
  free(t_out);
  free(p_out);
  free(coef);
  return 0;
}

/*
 * Stage 2: inner product with the key, u_c[t] = sum_j ext_j[t] * key[j][c][row(t)]
 * over the beta digits, for c = 0 (the "b" half) and c = 1 (the "a" half).
 * `key` is [dnum][2][L + K][N] in NTT form.  ext is [beta][level + K][N];
 * u is [2][level + K][N].
 */
void orc_inner_product(const orc_params *P, const uint32_t *ext, int level, const uint32_t *key, uint32_t *u) {
  const uint32_t N = P->N;
  int beta = orc_beta(P, level), n_ext = level + P->K, rows = P->L + P->K;
  for (int c = 0; c < 2; c++)
#pragma omp parallel for schedule(static)
    for (int t = 0; t < n_ext; t++) {
      uint32_t q = ext_prime(P, level, t);
      int r = key_row(P, level, t);
      for (uint32_t n = 0; n < N; n++) {
        u128 acc = 0;
        for (int j = 0; j < beta; j++)
          acc += (u128)ext[((size_t)j * n_ext + t) * N + n] * key[(((size_t)j * 2 + c) * rows + r) * N + n];
        u[((size_t)c * n_ext + t) * N + n] = (uint32_t)(acc % q);
      }
    }
}

/*
 * Stage 3: ModDown of one extended polynomial u ([level + K][N], NTT form)
 * to out ([level][N], NTT form), floor type:
 *   r = BConv_{P -> Q_level}(INTT(u restricted to the p-limbs)),
 *   out_i = (u_i - NTT(r)_i) * P^-1 mod q_i.
 */
void orc_moddown(const orc_params *P, const uint32_t *u, int level, uint32_t *out) {
  const uint32_t N = P->N;
  int K = P->K;
  const uint32_t *pp = P->primes + P->L;
  uint32_t *coef = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)K * N);
  memcpy(coef, u + (size_t)level * N, sizeof(uint32_t) * (size_t)K * N);
  orc_intt_limbs(coef, K, pp, N);
  uint32_t *r = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)level * N);
  orc_bconv(coef, K, pp, r, level, P->primes, N);
  orc_ntt_limbs(r, level, P->primes, N);
  for (int i = 0; i < level; i++) {
    uint32_t q = P->primes[i];
    uint32_t p_mod = 1 % q;
    for (int k = 0; k < K; k++) p_mod = mulmod(p_mod, pp[k] % q, q);
    uint32_t p_inv = orc_invmod(p_mod, q);
    for (uint32_t n = 0; n < N; n++)
      out[(size_t)i * N + n] = mulmod(submod(u[(size_t)i * N + n], r[(size_t)i * N + n], q), p_inv, q);
  }
  free(r);
  free(coef);
}

/*
 * Hybrid key switching of d ([level][N], NTT form) with `key`
 * ([dnum][2][L+K][N], NTT form): out = (out_0, out_1), [2][level][N].
 * out_0 + out_1 * s ~= d * s' when key encrypts s' under s.
 */
int orc_keyswitch(const orc_params *P, const uint32_t *d, int level, const uint32_t *key, uint32_t *out) {
  const uint32_t N = P->N;
  if (level < 1 || level > P->L) return -1;
  int beta = orc_beta(P, level), n_ext = level + P->K;
  uint32_t *ext = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)beta * n_ext * N);
  for (int j = 0; j < beta; j++) orc_modup(P, d, level, j, ext + (size_t)j * n_ext * N);
  uint32_t *u = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)2 * n_ext * N);
  orc_inner_product(P, ext, level, key, u);
  for (int c = 0; c < 2; c++) orc_moddown(P, u + (size_t)c * n_ext * N, level, out + (size_t)c * level * N);
  free(u);
  free(ext);
  return 0;
}

/* element-wise helpers on [n][N] arrays with limb i modulo primes[i] */
void orc_add(const uint32_t *a, const uint32_t *b, uint32_t *out, int nlimbs, const uint32_t *primes, uint32_t N) {
  for (int i = 0; i < nlimbs; i++)
    for (uint32_t n = 0; n < N; n++)
      out[(size_t)i * N + n] = addmod(a[(size_t)i * N + n], b[(size_t)i * N + n], primes[i]);
}

void orc_mul(const uint32_t *a, const uint32_t *b, uint32_t *out, int nlimbs, const uint32_t *primes, uint32_t N) {
  for (int i = 0; i < nlimbs; i++)
    for (uint32_t n = 0; n < N; n++)
      out[(size_t)i * N + n] = mulmod(a[(size_t)i * N + n], b[(size_t)i * N + n], primes[i]);
}

/*
 * HRotate: ct = (c0, c1) at `level`, NTT form, [2][level][N].  With
 * k = 5^rot mod 2N: c0' = sigma_k(c0), c1' = sigma_k(c1) (applied in NTT form
 * before ModUp), (k0, k1) = KS(c1'), out = (c0' + k0, k1).  `key` switches
 * from sigma_k(s) to s.
 */
int orc_rotate(const orc_params *P, const uint32_t *ct, int level, int32_t rot, const uint32_t *key, uint32_t *out) {
  const uint32_t N = P->N;
  uint32_t k = orc_galois_elt(rot, N);
  size_t poly = (size_t)level * N;
  uint32_t *rc = (uint32_t *)malloc(sizeof(uint32_t) * 2 * poly);
  for (int c = 0; c < 2; c++)
    for (int i = 0; i < level; i++) orc_automorph_ntt(ct + c * poly + (size_t)i * N, rc + c * poly + (size_t)i * N, N, k);
  uint32_t *ks = (uint32_t *)malloc(sizeof(uint32_t) * 2 * poly);
  int rc_ = orc_keyswitch(P, rc + poly, level, key, ks);
  if (rc_ == 0) {
    orc_add(rc, ks, out, level, P->primes, N);
    memcpy(out + poly, ks + poly, sizeof(uint32_t) * poly);
  }
  free(ks);
  free(rc);
  return rc_;
}

/*
 * Hoisted rotations of one ciphertext by rots[0..n): ModUp(c1) once, then for
 * each rotation sigma_k is applied to every extended digit (NTT-form
 * permutation), followed by the inner product with that rotation's key, ModDown,
 * and the addition of sigma_k(c0).  keys[i] is that rotation's key; outs is
 * [n][2][level][N].  A rotation by an index whose Galois element is 1 is the
 * identity (no key used).
 */
int orc_rotate_hoisted(const orc_params *P, const uint32_t *ct, int level, const int32_t *rots, int n,
                       const uint32_t *const *keys, uint32_t *outs) {
  const uint32_t N = P->N;
  int beta = orc_beta(P, level), n_ext = level + P->K;
  size_t poly = (size_t)level * N, ext_sz = (size_t)n_ext * N;
  uint32_t *ext = (uint32_t *)malloc(sizeof(uint32_t) * beta * ext_sz);
  for (int j = 0; j < beta; j++) orc_modup(P, ct + poly, level, j, ext + j * ext_sz);
  uint32_t *rext = (uint32_t *)malloc(sizeof(uint32_t) * beta * ext_sz);
  uint32_t *u = (uint32_t *)malloc(sizeof(uint32_t) * 2 * ext_sz);
  uint32_t *tmp = (uint32_t *)malloc(sizeof(uint32_t) * 2 * poly);
  for (int r = 0; r < n; r++) {
    uint32_t k = orc_galois_elt(rots[r], N);
    uint32_t *o = outs + (size_t)r * 2 * poly;
    if (k == 1) {
      memcpy(o, ct, sizeof(uint32_t) * 2 * poly);
      continue;
    }
    for (int j = 0; j < beta; j++)
      for (int t = 0; t < n_ext; t++) orc_automorph_ntt(ext + j * ext_sz + (size_t)t * N, rext + j * ext_sz + (size_t)t * N, N, k);
    orc_inner_product(P, rext, level, keys[r], u);
    for (int c = 0; c < 2; c++) orc_moddown(P, u + c * ext_sz, level, tmp + c * poly);
    for (int i = 0; i < level; i++) orc_automorph_ntt(ct + (size_t)i * N, o + (size_t)i * N, N, k);
    orc_add(o, tmp, o, level, P->primes, N);
    memcpy(o + poly, tmp + poly, sizeof(uint32_t) * poly);
  }
  free(tmp);
  free(u);
  free(rext);
  free(ext);
  return 0;
}

/*
 * HMult with relinearisation: a = (a0, a1), b = (b0, b1), NTT form.
 * d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1; (k0, k1) = KS(d2) with the
 * relinearisation key (s^2 -> s); out = (d0 + k0, d1 + k1).
 */
int orc_hmult(const orc_params *P, const uint32_t *a, const uint32_t *b, int level, const uint32_t *key, uint32_t *out) {
  const uint32_t N = P->N;
  size_t poly = (size_t)level * N;
  uint32_t *d = (uint32_t *)malloc(sizeof(uint32_t) * 3 * poly);
  uint32_t *t = (uint32_t *)malloc(sizeof(uint32_t) * poly);
  orc_mul(a, b, d, level, P->primes, N);
  orc_mul(a, b + poly, d + poly, level, P->primes, N);
  orc_mul(a + poly, b, t, level, P->primes, N);
  orc_add(d + poly, t, d + poly, level, P->primes, N);
  orc_mul(a + poly, b + poly, d + 2 * poly, level, P->primes, N);
  uint32_t *ks = (uint32_t *)malloc(sizeof(uint32_t) * 2 * poly);
  int rc = orc_keyswitch(P, d + 2 * poly, level, key, ks);
  if (rc == 0) {
    orc_add(d, ks, out, level, P->primes, N);
    orc_add(d + poly, ks + poly, out + poly, level, P->primes, N);
  }
  free(ks);
  free(t);
  free(d);
  return rc;
}

/*
 * Floor rescale of ct ([2][level][N], NTT form) to level-1:
 *   v = INTT_{q_last}(c_last) (coefficients in [0, q_last)),
 *   out_i = (c_i - NTT_{q_i}(v mod q_i)) * q_last^-1 mod q_i,  i < level-1.
 */
int orc_rescale(const orc_params *P, const uint32_t *ct, int level, uint32_t *out) {
  const uint32_t N = P->N;
  if (level < 2) return -1;
  uint32_t ql = P->primes[level - 1];
  uint32_t *v = (uint32_t *)malloc(sizeof(uint32_t) * N);
  uint32_t *w = (uint32_t *)malloc(sizeof(uint32_t) * N);
  for (int c = 0; c < 2; c++) {
    memcpy(v, ct + ((size_t)c * level + level - 1) * N, sizeof(uint32_t) * N);
    orc_intt(v, N, ql);
    for (int i = 0; i < level - 1; i++) {
      uint32_t q = P->primes[i];
      uint32_t inv = orc_invmod(ql % q, q);
      for (uint32_t n = 0; n < N; n++) w[n] = v[n] % q;
      orc_ntt(w, N, q);
      for (uint32_t n = 0; n < N; n++)
        out[((size_t)c * (level - 1) + i) * N + n] = mulmod(submod(ct[((size_t)c * level + i) * N + n], w[n], q), inv, q);
    }
  }
  free(w);
  free(v);
  return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
