/*
 * CPU oracle for the RNS-CKKS arithmetic behind encrypted CNN inference
 * (Jain et al., "Efficient CNN Building Blocks for Encrypted Data",
 * arXiv 2102.00319).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
 * GPU library is checked against.  Only the test-suite, the smoke check and
 * the benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or constant generator with the GPU library; it is written from the
 * definitions of the scheme, not from the GPU kernels.
 *
 * Everything here works on polynomials in COEFFICIENT form: a residue
 * polynomial ("limb") is N uint64 words, each in [0, q).  The product in
 * Z_q[X]/(X^N + 1) is, by definition, the schoolbook negacyclic convolution
 *     c_k = sum_{i+j=k} a_i b_j  -  sum_{i+j=k+N} a_i b_j     (mod q),
 * which is what or_poly_mul computes in mode 0.  Mode 1 computes the same
 * values through a textbook recursive number-theoretic transform (twist by
 * psi, cyclic DFT over omega = psi^2, pointwise product, inverse DFT,
 * untwist); the test-suite pins mode 1 to mode 0 and to big-integer brute
 * force.  Mode 1 exists only so that the large parity cases finish.
 *
 * Modular products use unsigned __int128 and the C '%' operator: slow and
 * obviously correct.  OpenMP runs independent limbs in parallel; it changes
 * no arithmetic.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;
typedef int64_t i64;
typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ */
/* Scalar modular arithmetic                                          */
/* ------------------------------------------------------------------ */

static u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static u64 addmod(u64 a, u64 b, u64 q) { u64 s = a + b; return s >= q ? s - q : s; }
static u64 submod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

u64 or_powmod(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

/* Inverse modulo a prime (Fermat). */
u64 or_invmod(u64 a, u64 q) { return or_powmod(a, q - 2, q); }

/* Signed integer -> residue in [0, q). */
static u64 signed_to_res(i64 v, u64 q) {
    if (v >= 0) return (u64)v % q;
    u64 m = (u64)(-(v + 1)) % q;  /* -(v) - 1 without overflow */
    return q - 1 - m;
}

/* ------------------------------------------------------------------ */
/* Primes: q = 1 (mod 2N), largest first below 2^bits                 */
/* ------------------------------------------------------------------ */

/* Deterministic Miller-Rabin: the first 12 primes as bases are enough for
 * every n < 3.3e24, so for every 64-bit n. */
int or_is_prime(u64 n) {
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; ++i) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    u64 d = n - 1;
    int r = 0;
    while ((d & 1) == 0) { d >>= 1; ++r; }
    for (int i = 0; i < 12; ++i) {
        u64 x = or_powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int composite = 1;
        for (int k = 1; k < r; ++k) {
            x = mulmod(x, x, n);
            if (x == n - 1) { composite = 0; break; }
        }
        if (composite) return 0;
    }
    return 1;
}

/* Prime chain.  For each requested bit size b (in order: q_0, q_1..q_L,
 * then the special primes p_0..), take the largest prime below 2^b that is
 * 1 mod 2N and not already taken.  Returns 0 on success, -1 if a size runs
 * out of candidates. */
int or_gen_primes(int log_n, const int *bits, int n, u64 *out) {
    u64 two_n = (u64)2 << log_n;
    for (int i = 0; i < n; ++i) {
        int b = bits[i];
        if (b < log_n + 2 || b > 62) return -1;
        u64 top = (u64)1 << b;
        u64 c = top - two_n + 1; /* largest value < 2^b that is 1 mod 2N */
        int found = 0;
        while (c > (top >> 1)) {
            int used = 0;
            for (int k = 0; k < i; ++k) if (out[k] == c) used = 1;
            if (!used && or_is_prime(c)) { out[i] = c; found = 1; break; }
            c -= two_n;
        }
        if (!found) return -1;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11)                  */
/* ------------------------------------------------------------------ */

static void mulhilo64(u64 a, u64 b, u64 *hi, u64 *lo) {
    u128 p = (u128)a * b;
    *hi = (u64)(p >> 64);
    *lo = (u64)p;
}

/* Ten rounds of the Philox-4x64 bijection; the key is bumped by the Weyl
 * constants between rounds. */
void or_philox4x64_10(const u64 ctr_in[4], const u64 key_in[2], u64 out[4]) {
    const u64 M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const u64 W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    u64 c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    u64 k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        u64 hi0, lo0, hi1, lo1;
        mulhilo64(M0, c0, &hi0, &lo0);
        mulhilo64(M1, c2, &hi1, &lo1);
        u64 n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Word i of the stream (seed, tag, lane): block i/4 of counter
 * (i/4, lane, 0, 0) under key (seed, tag), word i%4. */
static u64 stream_word(u64 seed, u64 tag, u64 lane, u64 i) {
    u64 ctr[4] = {i >> 2, lane, 0, 0}, key[2] = {seed, tag}, o[4];
    or_philox4x64_10(ctr, key, o);
    return o[i & 3];
}

/* Uniform ternary secret / encryption randomness: coefficient i is
 * (word_i mod 3) - 1, word_i from stream (seed, tag, lane 0). */
void or_sample_ternary(u64 seed, u64 tag, int n, i64 *out) {
    for (int i = 0; i < n; ++i) out[i] = (i64)(stream_word(seed, tag, 0, (u64)i) % 3) - 1;
}

/* Discrete Gaussian by cumulative-distribution table.  cdt[k] =
 * floor(2^63 * Pr[|X| <= k]) for k = 0..ncdt-1 (ncdt = tail cut).  From
 * word_i: bit 0 is the sign, the top 63 bits r give |X| = #{k : r >= cdt[k]}. */
void or_sample_gauss(u64 seed, u64 tag, int n, const u64 *cdt, int ncdt, i64 *out) {
    for (int i = 0; i < n; ++i) {
        u64 w = stream_word(seed, tag, 0, (u64)i);
        u64 r = w >> 1;
        i64 mag = 0;
        for (int k = 0; k < ncdt; ++k) if (r >= cdt[k]) ++mag;
        out[i] = (w & 1) ? -mag : mag;
    }
}

/* Uniform residue mod q for the limb with chain index `lane`: coefficient i
 * is (w_{2i+1} * 2^64 + w_{2i}) mod q, words from stream (seed, tag, lane). */
void or_sample_uniform(u64 seed, u64 tag, u64 lane, u64 q, int n, u64 *out) {
    for (int i = 0; i < n; ++i) {
        u64 lo = stream_word(seed, tag, lane, 2 * (u64)i);
        u64 hi = stream_word(seed, tag, lane, 2 * (u64)i + 1);
        out[i] = (u64)((((u128)hi << 64) | lo) % q);
    }
}

/* Signed integer polynomial -> residues modulo each of nl primes. */
void or_reduce_signed(const i64 *v, int n, const u64 *primes, int nl, u64 *out) {
    for (int l = 0; l < nl; ++l)
        for (int i = 0; i < n; ++i) out[(size_t)l * n + i] = signed_to_res(v[i], primes[l]);
}

/* ------------------------------------------------------------------ */
/* Negacyclic products                                                */
/* ------------------------------------------------------------------ */

/* 0 = schoolbook, 1 = textbook NTT, -1 = schoolbook for N <= 256 (the
 * definition itself) and the pinned NTT mode above. */
static int g_mode = -1;

void or_set_mode(int mode) { g_mode = mode; }
int or_get_mode(void) { return g_mode; }

static int use_schoolbook(int n) { return g_mode == 0 || (g_mode < 0 && n <= 256); }

/* Definition: c = a * b in Z_q[X]/(X^N + 1). */
static void negacyclic_schoolbook(const u64 *a, const u64 *b, u64 *c, int n, u64 q) {
    for (int k = 0; k < n; ++k) {
        u64 pos = 0, neg = 0;
        for (int i = 0; i <= k; ++i) pos = addmod(pos, mulmod(a[i], b[k - i], q), q);
        for (int i = k + 1; i < n; ++i) neg = addmod(neg, mulmod(a[i], b[n + k - i], q), q);
        c[k] = submod(pos, neg, q);
    }
}

/* A primitive 2N-th root of unity mod q: psi with psi^N = -1. */
static u64 find_psi(int n, u64 q) {
    for (u64 x = 2; x < q; ++x) {
        u64 psi = or_powmod(x, (q - 1) / (2 * (u64)n), q);
        if (or_powmod(psi, (u64)n, q) == q - 1) return psi;
    }
    return 0;
}

/* Recursive radix-2 decimation-in-time cyclic DFT of length n with root w:
 * A_k = sum_i a_i w^{ik}.  `scratch` holds n words. */
static void dft_rec(u64 *a, u64 *scratch, int n, u64 w, u64 q) {
    if (n == 1) return;
    int h = n / 2;
    u64 *ev = scratch, *od = scratch + h;
    for (int i = 0; i < h; ++i) { ev[i] = a[2 * i]; od[i] = a[2 * i + 1]; }
    u64 w2 = mulmod(w, w, q);
    dft_rec(ev, a, h, w2, q);
    dft_rec(od, a + h, h, w2, q);
    u64 wk = 1;
    for (int k = 0; k < h; ++k) {
        u64 t = mulmod(wk, od[k], q);
        a[k] = addmod(ev[k], t, q);
        a[k + h] = submod(ev[k], t, q);
        wk = mulmod(wk, w, q);
    }
}

/* The same product through the negative wrapped convolution:
 * a'_i = a_i psi^i, b'_i = b_i psi^i, c' = IDFT(DFT(a') . DFT(b')),
 * c_i = c'_i psi^{-i}. */
static void negacyclic_ntt(const u64 *a, const u64 *b, u64 *c, int n, u64 q) {
    u64 psi = find_psi(n, q);
    u64 psi_inv = or_invmod(psi, q);
    u64 omega = mulmod(psi, psi, q), omega_inv = or_invmod(omega, q);
    u64 n_inv = or_invmod((u64)n % q, q);
    u64 *A = malloc(sizeof(u64) * n), *B = malloc(sizeof(u64) * n), *S = malloc(sizeof(u64) * n);
    u64 pw = 1;
    for (int i = 0; i < n; ++i) {
        A[i] = mulmod(a[i], pw, q);
        B[i] = mulmod(b[i], pw, q);
        pw = mulmod(pw, psi, q);
    }
    dft_rec(A, S, n, omega, q);
    dft_rec(B, S, n, omega, q);
    for (int i = 0; i < n; ++i) A[i] = mulmod(A[i], B[i], q);
    dft_rec(A, S, n, omega_inv, q);
    pw = n_inv;
    for (int i = 0; i < n; ++i) {
        c[i] = mulmod(A[i], pw, q);
        pw = mulmod(pw, psi_inv, q);
    }
    free(A); free(B); free(S);
}

/* c = a * b, limb by limb, for nl limbs with primes[l]; a, b, c are
 * [nl][n] arrays.  c may alias neither a nor b. */
void or_poly_mul(const u64 *a, const u64 *b, u64 *c, const u64 *primes, int nl, int n) {
#pragma omp parallel for schedule(dynamic)
    for (int l = 0; l < nl; ++l) {
        const u64 *al = a + (size_t)l * n, *bl = b + (size_t)l * n;
        u64 *cl = c + (size_t)l * n;
        if (use_schoolbook(n)) negacyclic_schoolbook(al, bl, cl, n, primes[l]);
        else negacyclic_ntt(al, bl, cl, n, primes[l]);
    }
}

/* Batched products: for each job k, c_k = a_k * b_k, each an [nl][n] array
 * (pointers given per job).  Jobs x limbs run in parallel. */
void or_poly_mul_many(const u64 *const *a, const u64 *const *b, u64 *const *c, int njobs,
                      const u64 *primes, int nl, int n) {
#pragma omp parallel for schedule(dynamic) collapse(2)
    for (int k = 0; k < njobs; ++k)
        for (int l = 0; l < nl; ++l) {
            const u64 *al = a[k] + (size_t)l * n, *bl = b[k] + (size_t)l * n;
            u64 *cl = c[k] + (size_t)l * n;
            if (use_schoolbook(n)) negacyclic_schoolbook(al, bl, cl, n, primes[l]);
            else negacyclic_ntt(al, bl, cl, n, primes[l]);
        }
}

/* ------------------------------------------------------------------ */
/* Elementwise residue arithmetic                                      */
/* ------------------------------------------------------------------ */

void or_poly_add(const u64 *a, const u64 *b, u64 *c, const u64 *primes, int nl, int n) {
    for (int l = 0; l < nl; ++l)
        for (int i = 0; i < n; ++i) {
            size_t x = (size_t)l * n + i;
            c[x] = addmod(a[x], b[x], primes[l]);
        }
}

void or_poly_sub(const u64 *a, const u64 *b, u64 *c, const u64 *primes, int nl, int n) {
    for (int l = 0; l < nl; ++l)
        for (int i = 0; i < n; ++i) {
            size_t x = (size_t)l * n + i;
            c[x] = submod(a[x], b[x], primes[l]);
        }
}

void or_poly_neg(const u64 *a, u64 *c, const u64 *primes, int nl, int n) {
    for (int l = 0; l < nl; ++l)
        for (int i = 0; i < n; ++i) {
            size_t x = (size_t)l * n + i;
            c[x] = submod(0, a[x], primes[l]);
        }
}

/* c_l = a_l * s_l (mod primes[l]) with one scalar per limb. */
void or_poly_scalar_mul(const u64 *a, const u64 *s, u64 *c, const u64 *primes, int nl, int n) {
    for (int l = 0; l < nl; ++l)
        for (int i = 0; i < n; ++i) {
            size_t x = (size_t)l * n + i;
            c[x] = mulmod(a[x], s[l] % primes[l], primes[l]);
        }
}

/* c_l = a_l + s_l * [i == 0]: adds a constant polynomial (one residue per
 * limb) to the constant coefficient only. */
void or_poly_add_const(const u64 *a, const u64 *s, u64 *c, const u64 *primes, int nl, int n) {
    memcpy(c, a, sizeof(u64) * (size_t)nl * n);
    for (int l = 0; l < nl; ++l) c[(size_t)l * n] = addmod(a[(size_t)l * n], s[l] % primes[l], primes[l]);
}

/* ------------------------------------------------------------------ */
/* Galois automorphism kappa_g : a(X) -> a(X^g), g odd                 */
/* ------------------------------------------------------------------ */

/* X^i -> X^{i g mod 2N}; X^N = -1 folds indices >= N with a sign flip. */
void or_automorph(const u64 *a, u64 *c, const u64 *primes, int nl, int n, u64 g) {
    u64 two_n = 2 * (u64)n;
    for (int l = 0; l < nl; ++l) {
        u64 q = primes[l];
        const u64 *al = a + (size_t)l * n;
        u64 *cl = c + (size_t)l * n;
        for (int i = 0; i < n; ++i) {
            u64 e = ((u64)i * g) % two_n;
            if (e < (u64)n) cl[e] = al[i];
            else cl[e - n] = submod(0, al[i], q);
        }
    }
}

/* ------------------------------------------------------------------ */
/* Fast basis conversion (Cheon, Han, Kim, Kim, Song, SAC 2018)        */
/* ------------------------------------------------------------------ */

/* x has ns limbs over the source primes src[0..ns) (product D).  For each
 * destination prime t = dst[k]:
 *   y mod t  with  y = sum_i [x_i * (D/src_i)^{-1}]_{src_i} * (D/src_i),
 * the integer y taken without any reduction modulo D.  Each term is formed
 * exactly as the definition reads: the bracket is a residue in [0, src_i),
 * and (D/src_i) mod t is the product of the other source primes mod t. */
void or_fast_bconv(const u64 *x, const u64 *src, int ns, u64 *y, const u64 *dst, int nd, int n) {
    u64 *hat_inv = malloc(sizeof(u64) * ns);
    for (int i = 0; i < ns; ++i) {
        u64 prod = 1;
        for (int k = 0; k < ns; ++k) if (k != i) prod = mulmod(prod, src[k] % src[i], src[i]);
        hat_inv[i] = or_invmod(prod, src[i]);
    }
#pragma omp parallel for
    for (int d = 0; d < nd; ++d) {
        u64 t = dst[d];
        u64 *hat_mod_t = malloc(sizeof(u64) * ns);
        for (int i = 0; i < ns; ++i) {
            u64 prod = 1 % t;
            for (int k = 0; k < ns; ++k) if (k != i) prod = mulmod(prod, src[k] % t, t);
            hat_mod_t[i] = prod;
        }
        for (int c = 0; c < n; ++c) {
            u64 acc = 0;
            for (int i = 0; i < ns; ++i) {
                u64 v = mulmod(x[(size_t)i * n + c], hat_inv[i], src[i]);
                acc = addmod(acc, mulmod(v % t, hat_mod_t[i], t), t);
            }
            y[(size_t)d * n + c] = acc;
        }
        free(hat_mod_t);
    }
    free(hat_inv);
}

/* ------------------------------------------------------------------ */
/* Rescale by the last prime                                           */
/* ------------------------------------------------------------------ */

/* c has nl = l+1 limbs over primes[0..l]; out gets l limbs:
 *   out_i = (c_i - [c_l]) * q_l^{-1} mod q_i,
 * with [c_l] the centred representative of c_l in (-q_l/2, q_l/2). */
void or_rescale(const u64 *c, u64 *out, const u64 *primes, int nl, int n) {
    int l = nl - 1;
    u64 ql = primes[l];
    const u64 *last = c + (size_t)l * n;
    for (int i = 0; i < l; ++i) {
        u64 qi = primes[i];
        u64 inv = or_invmod(ql % qi, qi);
        for (int k = 0; k < n; ++k) {
            u64 r = last[k];
            i64 centred = r > (ql - 1) / 2 ? -(i64)(ql - r) : (i64)r;
            u64 rm = signed_to_res(centred, qi);
            out[(size_t)i * n + k] = mulmod(submod(c[(size_t)i * n + k], rm, qi), inv, qi);
        }
    }
}
