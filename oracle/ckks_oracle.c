/*
 * ckks_oracle.c -- plain, slow CPU reference for the ciphertext-branch
 * evaluation of bi-CryptoNets (levelled RNS-CKKS, one image per slot).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or table with the CUDA path.
 *
 * Every residue is held in a uint64_t and every modular product is the exact
 * 64-bit product reduced with the C `%` operator, so each step is the textbook
 * definition written out.  Citations are to the paper "Bi-CryptoNets:
 * Leveraging Different-Level Privacy for Encrypted Inference" (arXiv
 * 2402.01296).  The paper fixes the operations (App. A: Add, Mult, Rot with
 * D(Add(c,u)) = D(c)+u and D(Mult(c1,c2)) = D(c1)*D(c2)), the ring
 * R = Z_Q[x]/(x^N+1) (Sec. 2, App. A) and N = 2^14 for its own runs
 * (Sec. 5); it is silent on every cryptographic constant, so the readings
 * below (prime choice, sampling, key-switching variant) are this project's
 * and each is stated where it is used.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif


#define OC_MAXP 40

typedef struct {
    int log_n, N;
    int L;     /* data primes in the chain (q_0 > q_1 > ... > q_{L-1}) */
    int K;     /* special primes p_0..p_{K-1}, stored at q[L..L+K-1] */
    int alpha; /* primes per key-switching digit */
    uint64_t q[OC_MAXP];
    uint64_t psi[OC_MAXP];      /* primitive 2N-th root of unity mod q */
    uint64_t n_inv[OC_MAXP];    /* N^{-1} mod q */
    uint64_t *psi_pow[OC_MAXP]; /* psi^j, j < N */
    uint64_t *psi_ipow[OC_MAXP];/* psi^{-j}, j < N */
    uint64_t *w_pow[OC_MAXP];   /* omega^j with omega = psi^2, j < N/2 */
    uint64_t *w_ipow[OC_MAXP];  /* omega^{-j}, j < N/2 */
} oc_ctx;

/* ------------------------------------------------------------------ */
/* modular arithmetic (definitions)                                     */
/* ------------------------------------------------------------------ */
/* every residue in this file is below 2^31, so a*b < 2^62 is exact in 64 bits;
 * the precondition a, b < 2^32 is all that is needed */
static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q) { return (a * b) % q; }
static uint64_t addmod(uint64_t a, uint64_t b, uint64_t q) { return (a + b) % q; }
static uint64_t submod(uint64_t a, uint64_t b, uint64_t q) { return (a + q - b) % q; }
static uint64_t powmod(uint64_t a, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}
/* q prime: Fermat's little theorem */
static uint64_t invmod(uint64_t a, uint64_t q) { return powmod(a, q - 2, q); }
/* reduce a signed integer into [0, q) */
static uint64_t smod(int64_t v, uint64_t q) {
    int64_t r = v % (int64_t)q;
    if (r < 0) r += (int64_t)q;
    return (uint64_t)r;
}
/* centred representative of x in [0,q): x if x <= (q-1)/2 else x - q (q odd) */
static int64_t centred(uint64_t x, uint64_t q) { return x <= (q - 1) / 2 ? (int64_t)x : (int64_t)x - (int64_t)q; }

static int is_prime(uint64_t n) {
    if (n < 2) return 0;
    for (uint64_t d = 2; d * d <= n; d++)
        if (n % d == 0) return 0;
    return 1;
}

/* ------------------------------------------------------------------ */
/* parameters                                                           */
/* ------------------------------------------------------------------ */
/* Reading (the paper gives no primes): data primes are the L largest primes
 * q < 2^30 with q = 1 (mod 2N), in descending order; special primes are the
 * K largest primes p < 2^31 with p = 1 (mod 2N).  q = 1 (mod 2N) is what makes
 * a primitive 2N-th root of unity exist, i.e. what makes the negacyclic NTT
 * of R_q = Z_q[x]/(x^N+1) possible. */
static int find_primes(uint64_t bound, uint64_t m2n, int count, uint64_t *out) {
    uint64_t c = ((bound - 1) / m2n) * m2n + 1; /* largest value < bound that is 1 mod 2N */
    if (c >= bound) c -= m2n;
    int got = 0;
    while (got < count && c > m2n) {
        if (is_prime(c)) out[got++] = c;
        c -= m2n;
    }
    return got == count ? 0 : -1;
}

/* smallest primitive 2N-th root of unity: psi with psi^N = -1 (mod q) */
static uint64_t find_psi(uint64_t q, int N) {
    uint64_t two_n = 2 * (uint64_t)N, psi0 = 0;
    for (uint64_t g = 2; g < q; g++) {
        uint64_t cand = powmod(g, (q - 1) / two_n, q);
        if (powmod(cand, (uint64_t)N, q) == q - 1) { psi0 = cand; break; }
    }
    if (!psi0) return 0;
    /* all primitive 2N-th roots are psi0^(odd); take the smallest value */
    uint64_t best = psi0, sq = mulmod(psi0, psi0, q), cur = psi0;
    for (int i = 0; i < N; i++) {
        if (cur < best) best = cur;
        cur = mulmod(cur, sq, q);
    }
    return best;
}

oc_ctx *oc_create(int log_n, int L, int K, int alpha) {
    if (log_n < 1 || log_n > 17 || L < 1 || K < 0 || L + K > OC_MAXP || alpha < 1) return NULL;
    oc_ctx *c = (oc_ctx *)calloc(1, sizeof(oc_ctx));
    c->log_n = log_n;
    c->N = 1 << log_n;
    c->L = L;
    c->K = K;
    c->alpha = alpha;
    uint64_t m2n = 2 * (uint64_t)c->N;
    if (find_primes(1ull << 30, m2n, L, c->q) || (K && find_primes(1ull << 31, m2n, K, c->q + L))) {
        free(c);
        return NULL;
    }
    for (int t = 0; t < L + K; t++) {
        uint64_t q = c->q[t];
        int N = c->N;
        c->psi[t] = find_psi(q, N);
        c->n_inv[t] = invmod((uint64_t)N, q);
        c->psi_pow[t] = (uint64_t *)malloc(sizeof(uint64_t) * N);
        c->psi_ipow[t] = (uint64_t *)malloc(sizeof(uint64_t) * N);
        c->w_pow[t] = (uint64_t *)malloc(sizeof(uint64_t) * (N / 2 + 1));
        c->w_ipow[t] = (uint64_t *)malloc(sizeof(uint64_t) * (N / 2 + 1));
        uint64_t psi = c->psi[t], ipsi = invmod(psi, q);
        uint64_t w = mulmod(psi, psi, q), iw = mulmod(ipsi, ipsi, q);
        uint64_t a = 1, b = 1;
        for (int j = 0; j < N; j++) {
            c->psi_pow[t][j] = a;
            c->psi_ipow[t][j] = b;
            a = mulmod(a, psi, q);
            b = mulmod(b, ipsi, q);
        }
        a = 1; b = 1;
        for (int j = 0; j <= N / 2; j++) {
            c->w_pow[t][j] = a;
            c->w_ipow[t][j] = b;
            a = mulmod(a, w, q);
            b = mulmod(b, iw, q);
        }
    }
    return c;
}

void oc_destroy(oc_ctx *c) {
    if (!c) return;
    for (int t = 0; t < c->L + c->K; t++) {
        free(c->psi_pow[t]); free(c->psi_ipow[t]); free(c->w_pow[t]); free(c->w_ipow[t]);
    }
    free(c);
}

int oc_n(const oc_ctx *c) { return c->N; }
void oc_primes(const oc_ctx *c, uint64_t *out) { for (int t = 0; t < c->L + c->K; t++) out[t] = c->q[t]; }
uint64_t oc_psi(const oc_ctx *c, int t) { return c->psi[t]; }
int oc_dnum(const oc_ctx *c, int level) { return (level + c->alpha - 1) / c->alpha; }

void oc_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n);
#else
    (void)n;
#endif
}
int oc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* negacyclic NTT (textbook)                                            */
/* ------------------------------------------------------------------ */
/* Forward transform of a in R_q = Z_q[x]/(x^N+1):
 *     A_k = sum_j a_j psi^{(2k+1) j}   (k = 0..N-1, natural order),
 * i.e. evaluation of a at the N roots of x^N + 1.  Computed as the twist
 * a_j -> a_j psi^j followed by a cyclic DFT with omega = psi^2, the DFT done by
 * the iterative radix-2 Cooley-Tukey algorithm on bit-reversed input. */
static void bitrev_permute(uint64_t *a, int N) {
    for (int i = 1, j = 0; i < N; i++) {
        int bit = N >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { uint64_t t = a[i]; a[i] = a[j]; a[j] = t; }
    }
}

static void cyclic_dft(uint64_t *a, int N, uint64_t q, const uint64_t *wtab /* w^j, j <= N/2 */) {
    bitrev_permute(a, N);
    for (int len = 2; len <= N; len <<= 1) {
        int half = len / 2, step = N / len;
        for (int i = 0; i < N; i += len)
            for (int j = 0; j < half; j++) {
                uint64_t u = a[i + j];
                uint64_t v = mulmod(a[i + j + half], wtab[j * step], q);
                a[i + j] = addmod(u, v, q);
                a[i + j + half] = submod(u, v, q);
            }
    }
}

static void ntt_fwd(const oc_ctx *c, int t, uint64_t *a) {
    uint64_t q = c->q[t];
    for (int j = 0; j < c->N; j++) a[j] = mulmod(a[j], c->psi_pow[t][j], q);
    cyclic_dft(a, c->N, q, c->w_pow[t]);
}

static void ntt_inv(const oc_ctx *c, int t, uint64_t *a) {
    uint64_t q = c->q[t];
    cyclic_dft(a, c->N, q, c->w_ipow[t]);
    for (int j = 0; j < c->N; j++) a[j] = mulmod(mulmod(a[j], c->n_inv[t], q), c->psi_ipow[t][j], q);
}

/* exported for the pins: in place on N u32 residues of prime index t */
void oc_ntt_fwd(const oc_ctx *c, int t, uint32_t *a32) {
    uint64_t *a = (uint64_t *)malloc(sizeof(uint64_t) * c->N);
    for (int j = 0; j < c->N; j++) a[j] = a32[j];
    ntt_fwd(c, t, a);
    for (int j = 0; j < c->N; j++) a32[j] = (uint32_t)a[j];
    free(a);
}
void oc_ntt_inv(const oc_ctx *c, int t, uint32_t *a32) {
    uint64_t *a = (uint64_t *)malloc(sizeof(uint64_t) * c->N);
    for (int j = 0; j < c->N; j++) a[j] = a32[j];
    ntt_inv(c, t, a);
    for (int j = 0; j < c->N; j++) a32[j] = (uint32_t)a[j];
    free(a);
}

/* out = a * b in R_{q_t} (negacyclic product via the NTT) */
static void poly_mul(const oc_ctx *c, int t, const uint64_t *a, const uint64_t *b, uint64_t *out) {
    int N = c->N;
    uint64_t q = c->q[t];
    uint64_t *A = (uint64_t *)malloc(sizeof(uint64_t) * N), *B = (uint64_t *)malloc(sizeof(uint64_t) * N);
    memcpy(A, a, sizeof(uint64_t) * N);
    memcpy(B, b, sizeof(uint64_t) * N);
    ntt_fwd(c, t, A);
    ntt_fwd(c, t, B);
    for (int j = 0; j < N; j++) out[j] = mulmod(A[j], B[j], q);
    ntt_inv(c, t, out);
    free(A);
    free(B);
}
void oc_poly_mul(const oc_ctx *c, int t, const uint32_t *a32, const uint32_t *b32, uint32_t *o32) {
    int N = c->N;
    uint64_t *a = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N), *b = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N),
             *o = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    for (int j = 0; j < N; j++) { a[j] = a32[j]; b[j] = b32[j]; }
    poly_mul(c, t, a, b, o);
    for (int j = 0; j < N; j++) o32[j] = (uint32_t)o[j];
    free(a); free(b); free(o);
}

/* ------------------------------------------------------------------ */
/* seeded sampling                                                      */
/* ------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15, output = mix64(state)
 * with the published finaliser constants.  Each object draws from its own
 * stream; the stream (seed, tag, index) starts at
 * state = mix64(seed + GAMMA * ((tag << 40) + index + 1)). */
#define OC_GAMMA 0x9E3779B97F4A7C15ull
static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
typedef struct { uint64_t s; } oc_rng;
static void rng_init(oc_rng *r, uint64_t seed, uint64_t tag, uint64_t idx) {
    r->s = mix64(seed + OC_GAMMA * ((tag << 40) + idx + 1));
}
static uint64_t rng_next(oc_rng *r) { r->s += OC_GAMMA; return mix64(r->s); }
/* k-th output of the plain SplitMix64 generator started from `state` */
uint64_t oc_splitmix_raw(uint64_t state, uint64_t k) {
    oc_rng r = {state};
    uint64_t v = 0;
    for (uint64_t i = 0; i <= k; i++) v = rng_next(&r);
    return v;
}
uint64_t oc_rng_first(uint64_t seed, uint64_t tag, uint64_t idx, uint64_t k) {
    /* k-th output of stream (seed, tag, idx); exported for the pins */
    oc_rng r;
    rng_init(&r, seed, tag, idx);
    uint64_t v = 0;
    for (uint64_t i = 0; i <= k; i++) v = rng_next(&r);
    return v;
}

enum { TAG_SK = 1, TAG_EVK_A = 2, TAG_EVK_E = 3, TAG_ENC_A = 4, TAG_ENC_E = 5, TAG_GK_A = 6, TAG_GK_E = 7 };

/* ternary secret coefficient: (r mod 3) - 1 */
static int ternary(uint64_t r) { return (int)(r % 3) - 1; }
/* centred binomial, eta = 21: popcount of 21 bits minus popcount of the next 21 */
static int cbd21(uint64_t r) {
    uint64_t m = (1ull << 21) - 1;
    return __builtin_popcountll(r & m) - __builtin_popcountll((r >> 21) & m);
}
/* uniform residue mod q: low 32 bits, rejected above floor(2^32/q)*q */
static uint64_t uniform_mod(oc_rng *r, uint64_t q) {
    uint64_t bound = ((1ull << 32) / q) * q;
    for (;;) {
        uint64_t w = rng_next(r) & 0xFFFFFFFFull;
        if (w < bound) return w % q;
    }
}

/* ------------------------------------------------------------------ */
/* keys, encryption, decryption                                         */
/* ------------------------------------------------------------------ */
/* digit j of the key-switching decomposition at a level with `level` live
 * data primes covers q_{j*alpha} .. q_{min((j+1)*alpha, level) - 1}. */
static int digit_lo(const oc_ctx *c, int j) { return j * c->alpha; }
static int digit_hi(const oc_ctx *c, int j, int level) {
    int h = (j + 1) * c->alpha;
    return h < level ? h : level;
}

/* Secret key s (ternary) and the relinearisation key (hybrid key switching).
 * For digit j: evk_j = (b_j, a_j) over all L+K primes with
 *     b_j = -a_j s + e_j + P * g_j * s^2,
 * where P = prod p_m and g_j = 1 (mod q_i) for q_i in digit j, 0 (mod every
 * other prime).  Layout: evk[j][0 = b | 1 = a][L+K][N], coefficient form. */
int oc_keygen(const oc_ctx *c, uint64_t seed, int8_t *sk, uint32_t *evk) {
    int N = c->N, L = c->L, K = c->K, nb = L + K, dnum = oc_dnum(c, L);
    oc_rng r;
    rng_init(&r, seed, TAG_SK, 0);
    for (int j = 0; j < N; j++) sk[j] = (int8_t)ternary(rng_next(&r));
    uint64_t *s = (uint64_t *)malloc(8 * N), *s2 = (uint64_t *)malloc(8 * N), *as = (uint64_t *)malloc(8 * N);
    uint64_t *a = (uint64_t *)malloc(8 * N);
    int64_t *e = (int64_t *)malloc(8 * N);
    for (int dj = 0; dj < dnum; dj++) {
        oc_rng re;
        rng_init(&re, seed, TAG_EVK_E, (uint64_t)dj);
        for (int k = 0; k < N; k++) e[k] = cbd21(rng_next(&re));
        for (int t = 0; t < nb; t++) {
            uint64_t q = c->q[t];
            oc_rng ra;
            rng_init(&ra, seed, TAG_EVK_A, (uint64_t)dj * 256 + (uint64_t)t);
            for (int k = 0; k < N; k++) a[k] = uniform_mod(&ra, q);
            for (int k = 0; k < N; k++) s[k] = smod(sk[k], q);
            poly_mul(c, t, a, s, as);
            poly_mul(c, t, s, s, s2);
            uint64_t Pm = 1 % q;
            for (int m = 0; m < K; m++) Pm = mulmod(Pm, c->q[L + m] % q, q);
            int in_digit = (t < L) && t >= digit_lo(c, dj) && t < digit_hi(c, dj, L);
            uint32_t *bo = evk + ((size_t)(dj * 2 + 0) * nb + t) * N;
            uint32_t *ao = evk + ((size_t)(dj * 2 + 1) * nb + t) * N;
            for (int k = 0; k < N; k++) {
                uint64_t b = submod(smod(e[k], q), as[k], q);
                if (in_digit) b = addmod(b, mulmod(Pm, s2[k], q), q);
                bo[k] = (uint32_t)b;
                ao[k] = (uint32_t)a[k];
            }
        }
    }
    free(s); free(s2); free(as); free(a); free(e);
    return 0;
}

/* Symmetric encryption of encoded plaintexts (the client holds the key,
 * Sec. 2 threat model): ct = (-a s + e + m, a), a uniform per limb, e CBD.
 * pt: [n_ct][level][N] residues; ct out: [n_ct][2][level][N]. */
int oc_encrypt(const oc_ctx *c, const int8_t *sk, const uint32_t *pt, int n_ct, int level, uint64_t seed,
               uint32_t *ct) {
    int N = c->N;
    if (level < 1 || level > c->L) return -1;
#pragma omp parallel for schedule(dynamic)
    for (int ci = 0; ci < n_ct; ci++) {
        uint64_t *s = (uint64_t *)malloc(8 * N), *a = (uint64_t *)malloc(8 * N), *as = (uint64_t *)malloc(8 * N);
        int64_t *e = (int64_t *)malloc(8 * N);
        oc_rng re;
        rng_init(&re, seed, TAG_ENC_E, (uint64_t)ci);
        for (int k = 0; k < N; k++) e[k] = cbd21(rng_next(&re));
        for (int i = 0; i < level; i++) {
            uint64_t q = c->q[i];
            oc_rng ra;
            rng_init(&ra, seed, TAG_ENC_A, (uint64_t)ci * 256 + (uint64_t)i);
            for (int k = 0; k < N; k++) a[k] = uniform_mod(&ra, q);
            for (int k = 0; k < N; k++) s[k] = smod(sk[k], q);
            poly_mul(c, i, a, s, as);
            const uint32_t *m = pt + ((size_t)ci * level + i) * N;
            uint32_t *c0 = ct + (((size_t)ci * 2 + 0) * level + i) * N;
            uint32_t *c1 = ct + (((size_t)ci * 2 + 1) * level + i) * N;
            for (int k = 0; k < N; k++) {
                c0[k] = (uint32_t)addmod(submod(smod(e[k], q), as[k], q), m[k] % q, q);
                c1[k] = (uint32_t)a[k];
            }
        }
        free(s); free(a); free(as); free(e);
    }
    return 0;
}

/* Decryption to residues: m = sum_p c_p s^p (mod q_i), p < n_poly (2, or 3
 * for the output of a tensor square).  ct: [n_ct][n_poly][level][N]. */
int oc_decrypt(const oc_ctx *c, const int8_t *sk, const uint32_t *ct, int n_ct, int n_poly, int level,
               uint32_t *m_out) {
    int N = c->N;
#pragma omp parallel for schedule(dynamic)
    for (int ci = 0; ci < n_ct; ci++) {
        uint64_t *s = (uint64_t *)malloc(8 * N), *sp = (uint64_t *)malloc(8 * N), *cp = (uint64_t *)malloc(8 * N);
        uint64_t *tmp = (uint64_t *)malloc(8 * N), *acc = (uint64_t *)malloc(8 * N);
        for (int i = 0; i < level; i++) {
            uint64_t q = c->q[i];
            for (int k = 0; k < N; k++) { s[k] = smod(sk[k], q); sp[k] = (k == 0); acc[k] = 0; }
            for (int p = 0; p < n_poly; p++) {
                const uint32_t *src = ct + (((size_t)ci * n_poly + p) * level + i) * N;
                for (int k = 0; k < N; k++) cp[k] = src[k];
                poly_mul(c, i, cp, sp, tmp);
                for (int k = 0; k < N; k++) acc[k] = addmod(acc[k], tmp[k], q);
                poly_mul(c, i, sp, s, tmp);
                memcpy(sp, tmp, 8 * N);
            }
            uint32_t *dst = m_out + ((size_t)ci * level + i) * N;
            for (int k = 0; k < N; k++) dst[k] = (uint32_t)acc[k];
        }
        free(s); free(sp); free(cp); free(tmp); free(acc);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* homomorphic operations of the ciphertext branch                     */
/* ------------------------------------------------------------------ */
/* Conv / dense layer as Mult(c, u) with integer weights followed by Add of
 * ciphertexts (App. A), plus the unidirectional connection
 * x_{c,l} + z_{p,l} of Sec. 3.2 as Add(c, u) with an encoded plaintext:
 *     out[o] = sum_t w[o][t] * in[idx[o][t]]  (+ (pt[o], 0)).
 * idx[o][t] < 0 marks a zero-padding tap.  Exact integer arithmetic.
 * in: [n_in][2][level][N], pt: [n_out][level][N] or NULL,
 * out: [n_out][2][level][N].  Coefficient form (the map is linear, so the
 * domain does not matter). */
int oc_mac(const oc_ctx *c, int level, int n_in, int n_out, int K, const int32_t *idx, const int8_t *w,
           const uint32_t *in, const uint32_t *pt, uint32_t *out) {
    int N = c->N;
    for (size_t i = 0; i < (size_t)n_out * K; i++)
        if (idx[i] >= n_in) return -1;
#pragma omp parallel for schedule(dynamic)
    for (int o = 0; o < n_out; o++) {
        for (int p = 0; p < 2; p++)
            for (int i = 0; i < level; i++) {
                uint64_t q = c->q[i];
                for (int k = 0; k < N; k++) {
                    int64_t acc = 0;
                    for (int t = 0; t < K; t++) {
                        int32_t src = idx[(size_t)o * K + t];
                        if (src < 0) continue;
                        acc += (int64_t)w[(size_t)o * K + t] * (int64_t)in[(((size_t)src * 2 + p) * level + i) * N + k];
                    }
                    uint64_t r = smod(acc, q);
                    if (pt && p == 0) r = addmod(r, pt[((size_t)o * level + i) * N + k] % q, q);
                    out[(((size_t)o * 2 + p) * level + i) * N + k] = (uint32_t)r;
                }
            }
    }
    return 0;
}

/* Mult(c, c) before relinearisation: (c0 + c1 s)^2 = d0 + d1 s + d2 s^2 with
 * d0 = c0^2, d1 = 2 c0 c1, d2 = c1^2 in R_{q_i}.  Coefficient form in and
 * out: ct [2][level][N] -> d [3][level][N]. */
static void square_one(const oc_ctx *c, int level, const uint32_t *ct, uint64_t *d) {
    int N = c->N;
    uint64_t *a = (uint64_t *)malloc(8 * (size_t)N), *b = (uint64_t *)malloc(8 * (size_t)N);
    for (int i = 0; i < level; i++) {
        uint64_t q = c->q[i];
        for (int k = 0; k < N; k++) { a[k] = ct[(size_t)i * N + k]; b[k] = ct[((size_t)level + i) * N + k]; }
        ntt_fwd(c, i, a);
        ntt_fwd(c, i, b);
        uint64_t *d0 = d + (size_t)(0 * level + i) * N, *d1 = d + (size_t)(1 * level + i) * N,
                 *d2 = d + (size_t)(2 * level + i) * N;
        for (int k = 0; k < N; k++) {
            d0[k] = mulmod(a[k], a[k], q);
            d1[k] = mulmod(2, mulmod(a[k], b[k], q), q);
            d2[k] = mulmod(b[k], b[k], q);
        }
        ntt_inv(c, i, d0);
        ntt_inv(c, i, d1);
        ntt_inv(c, i, d2);
    }
    free(a);
    free(b);
}

/* The evaluation key in the NTT domain of each prime, for the level in use:
 * rows [dnum][2][level + K][N], limb t < level is q_t, limb level + m is p_m. */
static uint64_t *evk_to_ntt(const oc_ctx *c, int level, const uint32_t *evk) {
    int N = c->N, L = c->L, K = c->K, nb_key = L + K, nb = level + K, dnum = oc_dnum(c, level);
    uint64_t *out = (uint64_t *)malloc(8 * (size_t)dnum * 2 * nb * N);
#pragma omp parallel for collapse(2) schedule(dynamic)
    for (int j = 0; j < dnum; j++)
        for (int t = 0; t < nb; t++) {
            int pt = t < level ? t : L + (t - level);
            for (int b = 0; b < 2; b++) {
                const uint32_t *row = evk + ((size_t)(j * 2 + b) * nb_key + pt) * N;
                uint64_t *dst = out + ((size_t)(j * 2 + b) * nb + t) * N;
                for (int k = 0; k < N; k++) dst[k] = row[k];
                ntt_fwd(c, pt, dst);
            }
        }
    return out;
}

/* Key switching of one polynomial x (the s^2 component) at `level`:
 * returns (k0, k1) with k0 + k1 s ~= x s^2 (hybrid key switching; the
 * digit size alpha is the number of primes per digit).
 *   1. ModUp: for each digit j with primes D_j, y_i = [x_i * Dhat_i^{-1}]_{q_i}
 *      (centred) for q_i in D_j, Dhat_i = prod_{D_j} / q_i; for every other
 *      prime t of Q_level u P the fast basis conversion sum_i y_i * Dhat_i
 *      (mod t); on the digit's own primes the residue is x_i itself.
 *   2. inner product with evk_j over all primes of Q_level u P (NTT domain).
 *   3. ModDown: k_b(q_i) = (acc_b(q_i) - conv_{P->q_i}(acc_b)) * P^{-1}, with
 *      conv_{P->q}(v) = sum_m [v_m * Phat_m^{-1}]_{p_m} (centred) * Phat_m.
 * x: [level][N] coefficient form; evk_ntt from evk_to_ntt; out: [2][level][N]
 * coefficient form. */
static void keyswitch_one(const oc_ctx *c, int level, const uint64_t *evk_ntt, const uint64_t *x, uint64_t *out) {
    int N = c->N, L = c->L, K = c->K, nb = level + K;
    int *prime_of = (int *)malloc(sizeof(int) * nb);
    for (int t = 0; t < nb; t++) prime_of[t] = t < level ? t : L + (t - level);
    uint64_t *acc = (uint64_t *)calloc((size_t)2 * nb * N, 8);
    uint64_t *ext = (uint64_t *)malloc(8 * (size_t)N);
    int dnum = oc_dnum(c, level);
    for (int j = 0; j < dnum; j++) {
        int lo = digit_lo(c, j), hi = digit_hi(c, j, level);
        for (int t = 0; t < nb; t++) {
            uint64_t qt = c->q[prime_of[t]];
            if (t >= lo && t < hi) {
                for (int k = 0; k < N; k++) ext[k] = x[(size_t)t * N + k];
            } else {
                for (int k = 0; k < N; k++) ext[k] = 0;
                for (int i = lo; i < hi; i++) {
                    uint64_t qi = c->q[i], dhat_qi = 1, dhat_qt = 1;
                    for (int i2 = lo; i2 < hi; i2++)
                        if (i2 != i) {
                            dhat_qi = mulmod(dhat_qi, c->q[i2] % qi, qi);
                            dhat_qt = mulmod(dhat_qt, c->q[i2] % qt, qt);
                        }
                    uint64_t dhat_inv = invmod(dhat_qi, qi);
                    for (int k = 0; k < N; k++) {
                        int64_t y = centred(mulmod(x[(size_t)i * N + k], dhat_inv, qi), qi);
                        ext[k] = addmod(ext[k], mulmod(smod(y, qt), dhat_qt, qt), qt);
                    }
                }
            }
            ntt_fwd(c, prime_of[t], ext);
            for (int b = 0; b < 2; b++) {
                const uint64_t *key = evk_ntt + ((size_t)(j * 2 + b) * nb + t) * N;
                uint64_t *dst = acc + ((size_t)b * nb + t) * N;
                for (int k = 0; k < N; k++) dst[k] = addmod(dst[k], mulmod(ext[k], key[k], qt), qt);
            }
        }
    }
    for (int b = 0; b < 2; b++)
        for (int t = 0; t < nb; t++) ntt_inv(c, prime_of[t], acc + ((size_t)b * nb + t) * N);
    /* ModDown */
    for (int i = 0; i < level; i++) {
        uint64_t qi = c->q[i], P_qi = 1;
        for (int m = 0; m < K; m++) P_qi = mulmod(P_qi, c->q[L + m] % qi, qi);
        uint64_t Pinv = invmod(P_qi, qi);
        for (int b = 0; b < 2; b++) {
            uint64_t *res = out + ((size_t)b * level + i) * N;
            for (int k = 0; k < N; k++) res[k] = 0; /* conv_{P->q_i}(acc_b) */
            for (int m = 0; m < K; m++) {
                uint64_t pm = c->q[L + m], phat_pm = 1, phat_qi = 1;
                for (int m2 = 0; m2 < K; m2++)
                    if (m2 != m) {
                        phat_pm = mulmod(phat_pm, c->q[L + m2] % pm, pm);
                        phat_qi = mulmod(phat_qi, c->q[L + m2] % qi, qi);
                    }
                uint64_t phat_inv = invmod(phat_pm, pm);
                const uint64_t *v = acc + ((size_t)b * nb + level + m) * N;
                for (int k = 0; k < N; k++) {
                    int64_t y = centred(mulmod(v[k], phat_inv, pm), pm);
                    res[k] = addmod(res[k], mulmod(smod(y, qi), phat_qi, qi), qi);
                }
            }
            const uint64_t *a = acc + ((size_t)b * nb + i) * N;
            for (int k = 0; k < N; k++) res[k] = mulmod(submod(a[k], res[k], qi), Pinv, qi);
        }
    }
    free(prime_of); free(acc); free(ext);
}

/* Rescale (drop the last live prime q_top = q_{level-1}):
 * c_i <- (c_i - [c_top]_{q_top, centred}) * q_top^{-1} (mod q_i), i < level-1.
 * in [2][level][N] -> out [2][level-1][N], coefficient form. */
static void rescale_one(const oc_ctx *c, int level, const uint64_t *in, uint32_t *out) {
    int N = c->N, top = level - 1;
    uint64_t qt = c->q[top];
    for (int b = 0; b < 2; b++)
        for (int i = 0; i < top; i++) {
            uint64_t qi = c->q[i], inv = invmod(qt % qi, qi);
            for (int k = 0; k < N; k++) {
                int64_t v = centred(in[((size_t)b * level + top) * N + k], qt);
                uint64_t r = submod(in[((size_t)b * level + i) * N + k], smod(v, qi), qi);
                out[((size_t)b * top + i) * N + k] = (uint32_t)mulmod(r, inv, qi);
            }
        }
}

/* exported single-step operations (for op-level tests) */
int oc_square(const oc_ctx *c, int level, const uint32_t *ct, int n_ct, uint32_t *d_out) {
    int N = c->N;
    if (level < 1 || level > c->L) return -1;
#pragma omp parallel for schedule(dynamic)
    for (int ci = 0; ci < n_ct; ci++) {
        uint64_t *d = (uint64_t *)malloc(8 * (size_t)3 * level * N);
        square_one(c, level, ct + (size_t)ci * 2 * level * N, d);
        for (size_t k = 0; k < (size_t)3 * level * N; k++) d_out[(size_t)ci * 3 * level * N + k] = (uint32_t)d[k];
        free(d);
    }
    return 0;
}

/* key switching alone: x [n_ct][level][N] -> (k0, k1) [n_ct][2][level][N] */
int oc_keyswitch(const oc_ctx *c, int level, const uint32_t *evk, const uint32_t *x, int n_ct, uint32_t *out) {
    int N = c->N;
    if (level < 1 || level > c->L || c->K < 1) return -1;
    uint64_t *evk_ntt = evk_to_ntt(c, level, evk);
#pragma omp parallel for schedule(dynamic)
    for (int ci = 0; ci < n_ct; ci++) {
        size_t ln = (size_t)level * N;
        uint64_t *xx = (uint64_t *)malloc(8 * ln), *ks = (uint64_t *)malloc(8 * 2 * ln);
        for (size_t k = 0; k < ln; k++) xx[k] = x[(size_t)ci * ln + k];
        keyswitch_one(c, level, evk_ntt, xx, ks);
        for (size_t k = 0; k < 2 * ln; k++) out[(size_t)ci * 2 * ln + k] = (uint32_t)ks[k];
        free(xx); free(ks);
    }
    free(evk_ntt);
    return 0;
}

/* relinearise (d0, d1, d2) -> (d0 + k0, d1 + k1) with (k0, k1) = KeySwitch(d2);
 * d: [n_ct][3][level][N] -> [n_ct][2][level][N] */
int oc_relin(const oc_ctx *c, int level, const uint32_t *evk, const uint32_t *d, int n_ct, uint32_t *ct_out) {
    int N = c->N;
    if (level < 1 || level > c->L || c->K < 1) return -1;
    uint64_t *evk_ntt = evk_to_ntt(c, level, evk);
#pragma omp parallel for schedule(dynamic)
    for (int ci = 0; ci < n_ct; ci++) {
        size_t ln = (size_t)level * N;
        const uint32_t *dd = d + (size_t)ci * 3 * ln;
        uint64_t *x = (uint64_t *)malloc(8 * ln), *ks = (uint64_t *)malloc(8 * 2 * ln);
        for (size_t k = 0; k < ln; k++) x[k] = dd[2 * ln + k];
        keyswitch_one(c, level, evk_ntt, x, ks);
        for (int b = 0; b < 2; b++)
            for (int i = 0; i < level; i++)
                for (int k = 0; k < N; k++) {
                    size_t o = ((size_t)b * level + i) * N + k;
                    ct_out[(size_t)ci * 2 * ln + o] = (uint32_t)addmod(dd[o], ks[o], c->q[i]);
                }
        free(x); free(ks);
    }
    free(evk_ntt);
    return 0;
}

int oc_rescale(const oc_ctx *c, int level, const uint32_t *ct, int n_ct, uint32_t *out) {
    int N = c->N;
    if (level < 2 || level > c->L) return -1;
#pragma omp parallel for schedule(dynamic)
    for (int ci = 0; ci < n_ct; ci++) {
        uint64_t *in = (uint64_t *)malloc(8 * (size_t)2 * level * N);
        for (size_t k = 0; k < (size_t)2 * level * N; k++) in[k] = ct[(size_t)ci * 2 * level * N + k];
        rescale_one(c, level, in, out + (size_t)ci * 2 * (level - 1) * N);
        free(in);
    }
    return 0;
}

/* Square activation of the ciphertext branch (App. B replaces ReLU by the
 * square in the ciphertext branch): tensor square, relinearisation, then
 * rescale -- two separate roundings, in that order.
 * in [n_ct][2][level][N] -> out [n_ct][2][level-1][N]. */
int oc_square_relin_rescale(const oc_ctx *c, int level, const uint32_t *evk, const uint32_t *in, int n_ct,
                            uint32_t *out) {
    int N = c->N;
    if (level < 2 || level > c->L || c->K < 1) return -1;
    uint64_t *evk_ntt = evk_to_ntt(c, level, evk);
#pragma omp parallel for schedule(dynamic)
    for (int ci = 0; ci < n_ct; ci++) {
        size_t ln = (size_t)level * N;
        uint64_t *d = (uint64_t *)malloc(8 * 3 * ln), *ks = (uint64_t *)malloc(8 * 2 * ln);
        square_one(c, level, in + (size_t)ci * 2 * ln, d);
        keyswitch_one(c, level, evk_ntt, d + 2 * ln, ks);
        for (int b = 0; b < 2; b++)
            for (int i = 0; i < level; i++)
                for (int k = 0; k < N; k++) {
                    size_t o = ((size_t)b * level + i) * N + k;
                    ks[o] = addmod(d[o], ks[o], c->q[i]);
                }
        rescale_one(c, level, ks, out + (size_t)ci * 2 * (level - 1) * N);
        free(d); free(ks);
    }
    free(evk_ntt);
    return 0;
}

/* ------------------------------------------------------------------ */
/* rotations (App. A: Rot(c, k) rotates the slots of D(c) by k positions;  */
/* App. D builds convolutions and dense layers from them)                  */
/* ------------------------------------------------------------------ */
/* The automorphism sigma_g: a(X) -> a(X^g) of Z_q[X]/(X^N + 1), g odd.
 * Coefficient i moves to position i*g mod 2N and changes sign when that
 * position is N or more (X^N = -1).  With slot k at the root zeta^{5^k}
 * (the encoding of App. A as read here), sigma_g with g = 5^r mod 2N moves the
 * value of slot k + r into slot k: a rotation by r slots. */
static void automorph(int N, uint64_t g, const uint64_t *a, uint64_t *out, uint64_t q) {
    uint64_t two_n = 2 * (uint64_t)N;
    for (int i = 0; i < N; i++) {
        uint64_t j = ((uint64_t)i * g) % two_n;
        if (j < (uint64_t)N)
            out[j] = a[i];
        else
            out[j - N] = (q - a[i]) % q;
    }
}

/* in [n_poly][level][N] -> out [n_poly][level][N], limb i mod q_i */
int oc_automorphism(const oc_ctx *c, int level, uint64_t g, const uint32_t *in, int n_poly, uint32_t *out) {
    int N = c->N;
    if (level < 1 || level > c->L + c->K || (g & 1) == 0 || g >= 2 * (uint64_t)N) return -1;
#pragma omp parallel for schedule(dynamic)
    for (int p = 0; p < n_poly; p++) {
        uint64_t *a = (uint64_t *)malloc(8 * N), *b = (uint64_t *)malloc(8 * N);
        for (int i = 0; i < level; i++) {
            const uint32_t *src = in + ((size_t)p * level + i) * N;
            for (int k = 0; k < N; k++) a[k] = src[k];
            automorph(N, g, a, b, c->q[i]);
            for (int k = 0; k < N; k++) out[((size_t)p * level + i) * N + k] = (uint32_t)b[k];
        }
        free(a); free(b);
    }
    return 0;
}

/* Galois key of sigma_g: key switching from sigma_g(s) to s in the same hybrid
 * form as the relinearisation key, with s^2 replaced by sigma_g(s):
 *     gk_j = (-a_j s + e_j + P g_j sigma_g(s), a_j)   over Q_L u P.
 * Streams: a_j per limb (TAG_GK_A, (g << 20) + j*256 + limb), e_j
 * (TAG_GK_E, (g << 20) + j).  Layout [dnum][2][L+K][N] like the relinearisation key. */
int oc_galois_keygen(const oc_ctx *c, const int8_t *sk, uint64_t g, uint64_t seed, uint32_t *gk) {
    int N = c->N, L = c->L, K = c->K, nb = L + K, dnum = oc_dnum(c, L);
    if ((g & 1) == 0 || g >= 2 * (uint64_t)N) return -1;
    uint64_t *s = (uint64_t *)malloc(8 * N), *sg = (uint64_t *)malloc(8 * N), *as = (uint64_t *)malloc(8 * N);
    uint64_t *a = (uint64_t *)malloc(8 * N);
    int64_t *e = (int64_t *)malloc(8 * N);
    for (int dj = 0; dj < dnum; dj++) {
        oc_rng re;
        rng_init(&re, seed, TAG_GK_E, (g << 20) + (uint64_t)dj);
        for (int k = 0; k < N; k++) e[k] = cbd21(rng_next(&re));
        for (int t = 0; t < nb; t++) {
            uint64_t q = c->q[t];
            oc_rng ra;
            rng_init(&ra, seed, TAG_GK_A, (g << 20) + (uint64_t)dj * 256 + (uint64_t)t);
            for (int k = 0; k < N; k++) a[k] = uniform_mod(&ra, q);
            for (int k = 0; k < N; k++) s[k] = smod(sk[k], q);
            poly_mul(c, t, a, s, as);
            automorph(N, g, s, sg, q);
            uint64_t Pm = 1 % q;
            for (int m = 0; m < K; m++) Pm = mulmod(Pm, c->q[L + m] % q, q);
            int in_digit = (t < L) && t >= digit_lo(c, dj) && t < digit_hi(c, dj, L);
            uint32_t *bo = gk + ((size_t)(dj * 2 + 0) * nb + t) * N;
            uint32_t *ao = gk + ((size_t)(dj * 2 + 1) * nb + t) * N;
            for (int k = 0; k < N; k++) {
                uint64_t b = submod(smod(e[k], q), as[k], q);
                if (in_digit) b = addmod(b, mulmod(Pm, sg[k], q), q);
                bo[k] = (uint32_t)b;
                ao[k] = (uint32_t)a[k];
            }
        }
    }
    free(s); free(sg); free(as); free(a); free(e);
    return 0;
}

/* Rotation by the automorphism sigma_g: (c0, c1) -> (sigma_g(c0) + k0, k1) with
 * (k0, k1) = KeySwitch_gk(sigma_g(c1)), so that k0 + k1 s ~= sigma_g(c1) sigma_g(s)
 * and the result decrypts under s to sigma_g(m).  No rescale (no level used).
 * ct [n_ct][2][level][N] -> out [n_ct][2][level][N]. */
int oc_rotate(const oc_ctx *c, int level, const uint32_t *gk, uint64_t g, const uint32_t *ct, int n_ct,
              uint32_t *out) {
    int N = c->N;
    if (level < 1 || level > c->L || c->K < 1 || (g & 1) == 0 || g >= 2 * (uint64_t)N) return -1;
    uint64_t *gk_ntt = evk_to_ntt(c, level, gk);
#pragma omp parallel for schedule(dynamic)
    for (int ci = 0; ci < n_ct; ci++) {
        size_t ln = (size_t)level * N;
        uint64_t *a = (uint64_t *)malloc(8 * N), *r0 = (uint64_t *)malloc(8 * ln), *r1 = (uint64_t *)malloc(8 * ln);
        uint64_t *ks = (uint64_t *)malloc(8 * 2 * ln);
        const uint32_t *cc = ct + (size_t)ci * 2 * ln;
        for (int i = 0; i < level; i++) {
            for (int k = 0; k < N; k++) a[k] = cc[(size_t)i * N + k];
            automorph(N, g, a, r0 + (size_t)i * N, c->q[i]);
            for (int k = 0; k < N; k++) a[k] = cc[ln + (size_t)i * N + k];
            automorph(N, g, a, r1 + (size_t)i * N, c->q[i]);
        }
        keyswitch_one(c, level, gk_ntt, r1, ks);
        uint32_t *o = out + (size_t)ci * 2 * ln;
        for (int i = 0; i < level; i++)
            for (int k = 0; k < N; k++) {
                size_t x = (size_t)i * N + k;
                o[x] = (uint32_t)addmod(r0[x], ks[x], c->q[i]);
                o[ln + x] = (uint32_t)ks[ln + x];
            }
        free(a); free(r0); free(r1); free(ks);
    }
    free(gk_ntt);
    return 0;
}

/* Ciphertext-plaintext product (App. A Mult(c, u) with an encoded u, e.g. the
 * masks of App. D): (c0 u, c1 u) in R_{Q_level}, negacyclic products per prime;
 * ct [n_ct][2][level][N], pt [level][N] -> out [n_ct][2][level][N].  The
 * caller rescales afterwards (the mask carries a scale). */
int oc_mul_plain(const oc_ctx *c, int level, const uint32_t *ct, int n_ct, const uint32_t *pt, uint32_t *out) {
    int N = c->N;
    if (level < 1 || level > c->L) return -1;
#pragma omp parallel for schedule(dynamic)
    for (int ci = 0; ci < n_ct; ci++) {
        uint64_t *a = (uint64_t *)malloc(8 * N), *u = (uint64_t *)malloc(8 * N), *o = (uint64_t *)malloc(8 * N);
        for (int b = 0; b < 2; b++)
            for (int i = 0; i < level; i++) {
                const uint32_t *src = ct + (((size_t)ci * 2 + b) * level + i) * N;
                for (int k = 0; k < N; k++) {
                    a[k] = src[k];
                    u[k] = pt[(size_t)i * N + k];
                }
                poly_mul(c, i, a, u, o);
                for (int k = 0; k < N; k++) out[(((size_t)ci * 2 + b) * level + i) * N + k] = (uint32_t)o[k];
            }
        free(a); free(u); free(o);
    }
    return 0;
}
