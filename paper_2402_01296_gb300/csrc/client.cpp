// Client-side calls (host C++): keygen, weight quantisation, CKKS encode,
// symmetric encryption, decryption + decode.  The client holds the secret
// key (Sec. 2 threat model of the paper); none of this runs on the server's
// evaluation path.
#include <algorithm>
#include <cmath>
#include <complex>
#include <functional>
#include <thread>

#include "bcn_internal.h"

namespace bcn {
namespace {

// ---------------------------------------------------------------- threads
void parallel_for(int n, const std::function<void(int)> &fn) {
    int hw = (int)std::thread::hardware_concurrency();
    int nt = std::max(1, std::min(n, hw > 0 ? hw : 1));
    if (nt <= 1) {
        for (int i = 0; i < n; i++) fn(i);
        return;
    }
    std::vector<std::thread> th;
    for (int t = 0; t < nt; t++)
        th.emplace_back([&, t] {
            for (int i = t; i < n; i += nt) fn(i);
        });
    for (auto &x : th) x.join();
}

// ------------------------------------------------------ 32-bit modular math
inline uint32_t shoup(uint32_t a, uint32_t w, uint32_t wp, uint32_t q) {
    uint32_t hi = (uint32_t)(((uint64_t)a * wp) >> 32);
    uint32_t r = a * w - hi * q;
    return r >= q ? r - q : r;
}
inline uint32_t addq(uint32_t a, uint32_t b, uint32_t q) { uint32_t s = a + b; return s >= q ? s - q : s; }
inline uint32_t subq(uint32_t a, uint32_t b, uint32_t q) { return a >= b ? a - b : a + q - b; }
inline uint32_t mulq(uint32_t a, uint32_t b, uint32_t q) { return (uint32_t)((uint64_t)a * b % q); }
inline uint32_t from_signed(int64_t v, uint32_t q) {
    int64_t r = v % (int64_t)q;
    return (uint32_t)(r < 0 ? r + q : r);
}

// The integer a finite double x >= 2^52 in magnitude stands for (it has no
// fractional part), mod q: x = mant * 2^e with an integer mant < 2^53.
inline uint32_t big_mod(double x, uint32_t q) {
    int e2 = 0;
    const double f = std::frexp(std::fabs(x), &e2);  // |x| = f 2^e2, f in [0.5, 1)
    const uint64_t mant = (uint64_t)std::ldexp(f, 53);
    uint64_t r = mant % q, p2 = 2 % q;
    for (int e = e2 - 53; e > 0; e >>= 1) {  // r * 2^(e2 - 53) mod q
        if (e & 1) r = (uint64_t)(((unsigned __int128)r * p2) % q);
        p2 = (uint64_t)(((unsigned __int128)p2 * p2) % q);
    }
    return x < 0 && r ? (uint32_t)(q - r) : (uint32_t)r;
}

// negacyclic NTT, bit-reversed output (Cooley-Tukey) / input (Gentleman-Sande)
void ntt_fwd(const bcn_ctx *c, int t, uint32_t *a) {
    const uint32_t q = (uint32_t)c->primes[t];
    const uint32_t *w = c->h_tw_fwd[t].data();
    const int N = c->N;
    for (int m = 1, len = N >> 1; m < N; m <<= 1, len >>= 1)
        for (int i = 0; i < m; i++) {
            uint32_t W = w[2 * (m + i)], Wp = w[2 * (m + i) + 1];
            uint32_t *x = a + 2 * i * len, *y = x + len;
            for (int j = 0; j < len; j++) {
                uint32_t u = x[j], v = shoup(y[j], W, Wp, q);
                x[j] = addq(u, v, q);
                y[j] = subq(u, v, q);
            }
        }
}
void ntt_inv(const bcn_ctx *c, int t, uint32_t *a) {
    const uint32_t q = (uint32_t)c->primes[t];
    const uint32_t *w = c->h_tw_inv[t].data();
    const int N = c->N;
    for (int m = N >> 1, len = 1; m >= 1; m >>= 1, len <<= 1)
        for (int i = 0; i < m; i++) {
            uint32_t W = w[2 * (m + i)], Wp = w[2 * (m + i) + 1];
            uint32_t *x = a + 2 * i * len, *y = x + len;
            for (int j = 0; j < len; j++) {
                uint32_t u = x[j], v = y[j];
                x[j] = addq(u, v, q);
                y[j] = shoup(subq(u, v, q), W, Wp, q);
            }
        }
    const PrimeConst &pc = c->h_pc[t];
    for (int j = 0; j < N; j++) a[j] = shoup(a[j], pc.ninv, pc.ninv_shoup, q);
}

// ----------------------------------------------------------------- sampling
// SplitMix64 (Steele, Lea, Flood 2014) with per-object streams.
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
struct Stream {
    uint64_t s;
    Stream(uint64_t seed, uint64_t tag, uint64_t idx) : s(mix64(seed + kGamma * ((tag << 40) + idx + 1))) {}
    uint64_t next() { s += kGamma; return mix64(s); }
    uint32_t uniform(uint32_t q) {
        uint64_t bound = ((1ull << 32) / q) * q;
        for (;;) {
            uint64_t w = next() & 0xFFFFFFFFull;
            if (w < bound) return (uint32_t)(w % q);
        }
    }
    int cbd21() {
        uint64_t r = next(), m = (1ull << 21) - 1;
        return __builtin_popcountll(r & m) - __builtin_popcountll((r >> 21) & m);
    }
};
enum : uint64_t { kTagSk = 1, kTagEvkA = 2, kTagEvkE = 3, kTagEncA = 4, kTagEncE = 5, kTagGkA = 6, kTagGkE = 7 };

// --------------------------------------------------------------------- FFT
// Unnormalised DFT with positive exponent: F_j = sum_u Y_u exp(2 pi i j u / n).
struct Fft {
    int n, logn;
    std::vector<std::complex<double>> root;  // exp(2 pi i k / n), k < n
    std::vector<uint32_t> rev;
    explicit Fft(int n_) : n(n_), logn(0), root(n_), rev(n_) {
        while ((1 << logn) < n) logn++;
        for (int k = 0; k < n; k++) {
            double a = 2.0 * M_PI * (double)k / (double)n;
            root[k] = {std::cos(a), std::sin(a)};
        }
        for (int k = 0; k < n; k++) {
            uint32_t r = 0, x = (uint32_t)k;
            for (int b = 0; b < logn; b++) { r = (r << 1) | (x & 1); x >>= 1; }
            rev[k] = r;
        }
    }
    void run(std::complex<double> *a) const {
        for (int k = 0; k < n; k++)
            if ((int)rev[k] > k) std::swap(a[k], a[rev[k]]);
        for (int len = 2; len <= n; len <<= 1) {
            int half = len >> 1, step = n / len;
            for (int i = 0; i < n; i += len)
                for (int j = 0; j < half; j++) {
                    std::complex<double> u = a[i + j], v = a[i + j + half] * root[(size_t)j * step];
                    a[i + j] = u + v;
                    a[i + j + half] = u - v;
                }
        }
    }
};

// slot k sits at the odd exponent e_k = 5^k mod 2N; its conjugate at 2N - e_k
std::vector<uint32_t> slot_exponents(int N) {
    std::vector<uint32_t> e(N / 2);
    uint64_t v = 1;
    for (int k = 0; k < N / 2; k++) { e[k] = (uint32_t)v; v = v * 5 % (2 * (uint64_t)N); }
    return e;
}

}  // namespace
}  // namespace bcn

using namespace bcn;

extern "C" {

bcn_status bcn_keygen(const bcn_ctx *c, uint64_t seed, int8_t *sk, uint32_t *evk) {
    if (!c || !sk || !evk) return fail(BCN_E_INVAL, "bcn_keygen: null argument");
    const int N = c->N, L = c->L, K = c->K, P = L + K, A = c->alpha;
    Stream rs(seed, kTagSk, 0);
    for (int j = 0; j < N; j++) sk[j] = (int8_t)((int)(rs.next() % 3) - 1);
    // s and s^2 in the NTT domain of every prime
    std::vector<std::vector<uint32_t>> S(P, std::vector<uint32_t>(N)), S2(P, std::vector<uint32_t>(N));
    parallel_for(P, [&](int t) {
        uint32_t q = (uint32_t)c->primes[t];
        for (int j = 0; j < N; j++) S[t][j] = from_signed(sk[j], q);
        ntt_fwd(c, t, S[t].data());
        for (int j = 0; j < N; j++) S2[t][j] = mulq(S[t][j], S[t][j], q);
        ntt_inv(c, t, S2[t].data());  // s^2, coefficient form
    });
    std::vector<uint32_t> Pmod(P);
    for (int t = 0; t < P; t++) {
        uint64_t q = c->primes[t], v = 1 % q;
        for (int m = 0; m < K; m++) v = mulmod64(v, c->primes[L + m] % q, q);
        Pmod[t] = (uint32_t)v;
    }
    parallel_for(c->dnum * P, [&](int job) {
        int j = job / P, t = job % P;
        uint32_t q = (uint32_t)c->primes[t];
        Stream re(seed, kTagEvkE, (uint64_t)j);
        Stream ra(seed, kTagEvkA, (uint64_t)j * 256 + (uint64_t)t);
        uint32_t *b = evk + ((size_t)(j * 2 + 0) * P + t) * N;
        uint32_t *a = evk + ((size_t)(j * 2 + 1) * P + t) * N;
        std::vector<uint32_t> as(N);
        for (int k = 0; k < N; k++) a[k] = ra.uniform(q);
        std::copy(a, a + N, as.begin());
        ntt_fwd(c, t, as.data());
        for (int k = 0; k < N; k++) as[k] = mulq(as[k], S[t][k], q);
        ntt_inv(c, t, as.data());
        bool in_digit = t < L && t >= j * A && t < std::min((j + 1) * A, L);
        for (int k = 0; k < N; k++) {
            uint32_t v = subq(from_signed(re.cbd21(), q), as[k], q);
            if (in_digit) v = addq(v, mulq(Pmod[t], S2[t][k], q), q);
            b[k] = v;
        }
    });
    return BCN_OK;
}

uint32_t bcn_galois_elt(const bcn_ctx *c, int steps) {
    if (!c) return 0;
    const uint64_t two_n = 2 * (uint64_t)c->N, half = (uint64_t)c->N / 2;
    const uint64_t e = (uint64_t)(((long long)steps % (long long)half + (long long)half) % (long long)half);
    uint64_t g = 1, b = 5;
    for (uint64_t k = e; k; k >>= 1) {
        if (k & 1) g = g * b % two_n;
        b = b * b % two_n;
    }
    return (uint32_t)g;
}

bcn_status bcn_galois_keygen(const bcn_ctx *c, const int8_t *sk, int steps, uint64_t seed, uint32_t *gk) {
    if (!c || !sk || !gk) return fail(BCN_E_INVAL, "bcn_galois_keygen: null argument");
    const int N = c->N, L = c->L, K = c->K, P = L + K, A = c->alpha;
    const uint64_t g = bcn_galois_elt(c, steps), two_n = 2 * (uint64_t)N;
    // s in the NTT domain and sigma_g(s) in coefficient form, every prime
    std::vector<std::vector<uint32_t>> S(P, std::vector<uint32_t>(N)), SG(P, std::vector<uint32_t>(N));
    parallel_for(P, [&](int t) {
        uint32_t q = (uint32_t)c->primes[t];
        for (int i = 0; i < N; i++) {
            const uint32_t v = from_signed(sk[i], q);
            const uint64_t j = (uint64_t)i * g % two_n;  // X^i -> X^{i g}, X^N = -1
            if (j < (uint64_t)N)
                SG[t][j] = v;
            else
                SG[t][j - N] = v ? q - v : 0;
            S[t][i] = v;
        }
        ntt_fwd(c, t, S[t].data());
    });
    std::vector<uint32_t> Pmod(P);
    for (int t = 0; t < P; t++) {
        uint64_t q = c->primes[t], v = 1 % q;
        for (int m = 0; m < K; m++) v = mulmod64(v, c->primes[L + m] % q, q);
        Pmod[t] = (uint32_t)v;
    }
    parallel_for(c->dnum * P, [&](int job) {
        int j = job / P, t = job % P;
        uint32_t q = (uint32_t)c->primes[t];
        Stream re(seed, kTagGkE, (g << 20) + (uint64_t)j);
        Stream ra(seed, kTagGkA, (g << 20) + (uint64_t)j * 256 + (uint64_t)t);
        uint32_t *b = gk + ((size_t)(j * 2 + 0) * P + t) * N;
        uint32_t *a = gk + ((size_t)(j * 2 + 1) * P + t) * N;
        std::vector<uint32_t> as(N);
        for (int k = 0; k < N; k++) a[k] = ra.uniform(q);
        std::copy(a, a + N, as.begin());
        ntt_fwd(c, t, as.data());
        for (int k = 0; k < N; k++) as[k] = mulq(as[k], S[t][k], q);
        ntt_inv(c, t, as.data());
        bool in_digit = t < L && t >= j * A && t < std::min((j + 1) * A, L);
        for (int k = 0; k < N; k++) {
            uint32_t v = subq(from_signed(re.cbd21(), q), as[k], q);
            if (in_digit) v = addq(v, mulq(Pmod[t], SG[t][k], q), q);
            b[k] = v;
        }
    });
    return BCN_OK;
}

bcn_status bcn_quantize(const float *w, size_t n, int8_t *w_int, double *s_w) {
    if ((!w || !w_int) && n) return fail(BCN_E_INVAL, "bcn_quantize: null argument");
    if (!s_w) return fail(BCN_E_INVAL, "bcn_quantize: null s_w");
    double mx = 0.0;
    for (size_t i = 0; i < n; i++) mx = std::max(mx, std::fabs((double)w[i]));
    if (mx == 0.0) {
        for (size_t i = 0; i < n; i++) w_int[i] = 0;
        *s_w = 1.0;
        return BCN_OK;
    }
    double s = mx / 127.0;
    for (size_t i = 0; i < n; i++) {
        long long r = std::llround((double)w[i] / s);
        if (r > 127 || r < -127) return fail(BCN_E_INVAL, "bcn_quantize: value outside [-127, 127]");
        w_int[i] = (int8_t)r;
    }
    *s_w = s;
    return BCN_OK;
}

// the encoder: residues of `level` primes (pts), or the integer coefficients
// themselves (coeffs, when every |m_j| < 2^63)
static bcn_status encode_impl(const bcn_ctx *c, const double *values, int n_vec, int B, int level, double scale,
                              uint32_t *pts, int64_t *coeffs) {
    if (!c || (!values && n_vec) || (!pts && !coeffs && n_vec)) return fail(BCN_E_INVAL, "bcn_encode: null argument");
    const int N = c->N;
    if (B < 0 || B > N / 2 || level < 1 || level > c->L || n_vec < 0)
        return fail(BCN_E_INVAL, "bcn_encode: bad batch or level");
    Fft fft(N);
    std::vector<uint32_t> e = slot_exponents(N);
    std::vector<std::complex<double>> twist(N);  // omega^j = exp(i pi j / N)
    for (int j = 0; j < N; j++) twist[j] = {std::cos(M_PI * j / N), std::sin(M_PI * j / N)};
    std::vector<int> bad(n_vec, 0);
    parallel_for(n_vec, [&](int v) {
        // Y_u = Z_{2u+1}: slot k at exponents e_k and 2N - e_k
        std::vector<std::complex<double>> y(N, 0.0);
        const double *z = values + (size_t)v * B;
        for (int k = 0; k < B; k++) {
            y[(e[k] - 1) / 2] += z[k];
            y[(2 * N - e[k] - 1) / 2] += z[k];
        }
        fft.run(y.data());
        if (coeffs != nullptr) {
            int64_t *co = coeffs + (size_t)v * N;
            for (int j = 0; j < N; j++) {
                double x = (twist[j] * y[j]).real() * (scale / N);
                if (!std::isfinite(x) || std::fabs(x) >= 9223372036854775808.0) { bad[v] = 2; return; }  // 2^63
                // below 2^52: round half away from zero; above, already an integer
                co[j] = std::fabs(x) < 4503599627370496.0 ? (int64_t)std::llround(x) : (int64_t)x;
            }
            return;
        }
        uint32_t *out = pts + (size_t)v * level * N;
        for (int j = 0; j < N; j++) {
            double x = (twist[j] * y[j]).real() * (scale / N);
            if (!std::isfinite(x)) { bad[v] = 1; return; }
            if (std::fabs(x) < 4503599627370496.0) {  // 2^52: round half away from zero
                long long m = std::llround(x);
                for (int i = 0; i < level; i++) out[(size_t)i * N + j] = from_signed(m, (uint32_t)c->primes[i]);
            } else {  // already an integer
                for (int i = 0; i < level; i++) out[(size_t)i * N + j] = big_mod(x, (uint32_t)c->primes[i]);
            }
        }
    });
    for (int v = 0; v < n_vec; v++)
        if (bad[v]) return fail(BCN_E_SCALE, bad[v] == 2 ? "bcn_encode_i64: a coefficient is not below 2^63"
                                                         : "bcn_encode: a coefficient is not finite");
    return BCN_OK;
}

bcn_status bcn_encode(const bcn_ctx *c, const double *values, int n_vec, int B, int level, double scale,
                      uint32_t *pts) {
    return encode_impl(c, values, n_vec, B, level, scale, pts, nullptr);
}

bcn_status bcn_encode_i64(const bcn_ctx *c, const double *values, int n_vec, int B, double scale, int64_t *coeffs) {
    return encode_impl(c, values, n_vec, B, 1, scale, nullptr, coeffs);
}

// secret-key encryption; with c0_only the output is [n_ct][level][N] (c0 alone,
// c1 being the uniform stream the seed defines)
static bcn_status encrypt_impl(const bcn_ctx *c, const int8_t *sk, const uint32_t *pts, int n_ct, int level,
                               uint64_t seed, uint32_t *cts, bool c0_only) {
    if (!c || !sk || ((!pts || !cts) && n_ct)) return fail(BCN_E_INVAL, "bcn_encrypt: null argument");
    if (level < 1 || level > c->L || n_ct < 0) return fail(BCN_E_INVAL, "bcn_encrypt: bad level or count");
    const int N = c->N;
    std::vector<std::vector<uint32_t>> S(level, std::vector<uint32_t>(N));
    for (int i = 0; i < level; i++) {
        uint32_t q = (uint32_t)c->primes[i];
        for (int j = 0; j < N; j++) S[i][j] = from_signed(sk[j], q);
        ntt_fwd(c, i, S[i].data());
    }
    parallel_for(n_ct, [&](int ci) {
        std::vector<int> e(N);
        Stream re(seed, kTagEncE, (uint64_t)ci);
        for (int k = 0; k < N; k++) e[k] = re.cbd21();
        std::vector<uint32_t> as(N);
        for (int i = 0; i < level; i++) {
            uint32_t q = (uint32_t)c->primes[i];
            Stream ra(seed, kTagEncA, (uint64_t)ci * 256 + (uint64_t)i);
            uint32_t *c0 = c0_only ? cts + ((size_t)ci * level + i) * N : cts + (((size_t)ci * 2 + 0) * level + i) * N;
            uint32_t *c1 = c0_only ? as.data() : cts + (((size_t)ci * 2 + 1) * level + i) * N;
            for (int k = 0; k < N; k++) c1[k] = ra.uniform(q);
            if (!c0_only) std::copy(c1, c1 + N, as.begin());
            ntt_fwd(c, i, as.data());
            for (int k = 0; k < N; k++) as[k] = mulq(as[k], S[i][k], q);
            ntt_inv(c, i, as.data());
            const uint32_t *m = pts + ((size_t)ci * level + i) * N;
            for (int k = 0; k < N; k++) c0[k] = addq(subq(from_signed(e[k], q), as[k], q), m[k] % q, q);
        }
    });
    return BCN_OK;
}

bcn_status bcn_encrypt(const bcn_ctx *c, const int8_t *sk, const uint32_t *pts, int n_ct, int level,
                       uint64_t seed, uint32_t *cts) {
    return encrypt_impl(c, sk, pts, n_ct, level, seed, cts, false);
}

bcn_status bcn_encrypt_seeded(const bcn_ctx *c, const int8_t *sk, const uint32_t *pts, int n_ct, int level,
                              uint64_t seed, uint32_t *c0) {
    return encrypt_impl(c, sk, pts, n_ct, level, seed, c0, true);
}

static bcn_status encrypt_segment_impl(const bcn_ctx *c, const int8_t *sk, const uint8_t *images, int B, int H,
                                       int W, int C, const int seg[4], double scale, uint64_t seed, uint32_t *cts,
                                       bool c0_only);

bcn_status bcn_encrypt_segment(const bcn_ctx *c, const int8_t *sk, const uint8_t *images, int B, int H, int W,
                               int C, const int seg[4], double scale, uint64_t seed, uint32_t *cts) {
    return encrypt_segment_impl(c, sk, images, B, H, W, C, seg, scale, seed, cts, false);
}

bcn_status bcn_encrypt_segment_seeded(const bcn_ctx *c, const int8_t *sk, const uint8_t *images, int B, int H,
                                      int W, int C, const int seg[4], double scale, uint64_t seed, uint32_t *c0) {
    return encrypt_segment_impl(c, sk, images, B, H, W, C, seg, scale, seed, c0, true);
}

static bcn_status encrypt_segment_impl(const bcn_ctx *c, const int8_t *sk, const uint8_t *images, int B, int H,
                                       int W, int C, const int seg[4], double scale, uint64_t seed, uint32_t *cts,
                                       bool c0_only) {
    if (!c || !sk || !images || !seg || !cts) return fail(BCN_E_INVAL, "bcn_encrypt_segment: null argument");
    int y0 = seg[0], x0 = seg[1], h = seg[2], w = seg[3];
    if (B < 1 || B > c->N / 2 || y0 < 0 || x0 < 0 || h < 1 || w < 1 || y0 + h > H || x0 + w > W || C < 1)
        return fail(BCN_E_INVAL, "bcn_encrypt_segment: segment outside the image or bad batch");
    int n_ct = C * h * w;
    std::vector<double> vals((size_t)n_ct * B);
    for (int ch = 0; ch < C; ch++)
        for (int y = 0; y < h; y++)
            for (int x = 0; x < w; x++) {
                size_t ct = ((size_t)ch * h + y) * w + x;
                for (int b = 0; b < B; b++)
                    vals[ct * B + b] = images[(((size_t)b * H + y0 + y) * W + x0 + x) * C + ch] / 255.0;
            }
    std::vector<uint32_t> pts((size_t)n_ct * c->L * c->N);
    bcn_status st = bcn_encode(c, vals.data(), n_ct, B, c->L, scale, pts.data());
    if (st != BCN_OK) return st;
    return encrypt_impl(c, sk, pts.data(), n_ct, c->L, seed, cts, c0_only);
}

bcn_status bcn_decrypt_decode(const bcn_ctx *c, const int8_t *sk, const uint32_t *cts, int n_ct, int level,
                              double scale, int B, double *out) {
    if (!c || !sk || ((!cts || !out) && n_ct)) return fail(BCN_E_INVAL, "bcn_decrypt_decode: null argument");
    const int N = c->N;
    if (level < 1 || level > c->L || B < 0 || B > N / 2 || n_ct < 0)
        return fail(BCN_E_INVAL, "bcn_decrypt_decode: bad level or batch");
    std::vector<std::vector<uint32_t>> S(level, std::vector<uint32_t>(N));
    for (int i = 0; i < level; i++) {
        uint32_t q = (uint32_t)c->primes[i];
        for (int j = 0; j < N; j++) S[i][j] = from_signed(sk[j], q);
        ntt_fwd(c, i, S[i].data());
    }
    // balanced-digit Garner: x = v_0 + v_1 M_1 + ... , M_i = q_0...q_{i-1}, |v_i| <= (q_i-1)/2
    std::vector<std::vector<uint32_t>> Mmod(level, std::vector<uint32_t>(level));  // M_j mod q_i
    std::vector<uint32_t> Minv(level);                                             // M_i^{-1} mod q_i
    for (int i = 0; i < level; i++) {
        uint64_t qi = c->primes[i];
        for (int j = 0; j <= i; j++) {
            uint64_t v = 1 % qi;
            for (int k = 0; k < j; k++) v = mulmod64(v, c->primes[k] % qi, qi);
            Mmod[i][j] = (uint32_t)v;
        }
        Minv[i] = (uint32_t)invmod64(Mmod[i][i], qi);
    }
    Fft fft(N);
    std::vector<uint32_t> e = slot_exponents(N);
    std::vector<double> cs(N), sn(N);  // omega^k = exp(i pi k / N)
    for (int k = 0; k < N; k++) { cs[k] = std::cos(M_PI * k / N); sn[k] = std::sin(M_PI * k / N); }
    parallel_for(n_ct, [&](int ci) {
        std::vector<uint32_t> m((size_t)level * N), t(N);
        for (int i = 0; i < level; i++) {
            uint32_t q = (uint32_t)c->primes[i];
            const uint32_t *c0 = cts + (((size_t)ci * 2 + 0) * level + i) * N;
            const uint32_t *c1 = cts + (((size_t)ci * 2 + 1) * level + i) * N;
            std::copy(c1, c1 + N, t.begin());
            ntt_fwd(c, i, t.data());
            for (int k = 0; k < N; k++) t[k] = mulq(t[k], S[i][k], q);
            ntt_inv(c, i, t.data());
            for (int k = 0; k < N; k++) m[(size_t)i * N + k] = addq(c0[k] % q, t[k], q);
        }
        std::vector<std::complex<double>> y(N);
        std::vector<int64_t> v(level);
        for (int k = 0; k < N; k++) {
            for (int i = 0; i < level; i++) {
                uint32_t qi = (uint32_t)c->primes[i];
                uint32_t s = 0;  // x_{<i} mod q_i
                for (int j = 0; j < i; j++) s = addq(s, mulq(from_signed(v[j], qi), Mmod[i][j], qi), qi);
                uint32_t d = mulq(subq(m[(size_t)i * N + k], s, qi), Minv[i], qi);
                v[i] = d <= (qi - 1) / 2 ? (int64_t)d : (int64_t)d - (int64_t)qi;
            }
            double x = 0.0;
            for (int i = level - 1; i >= 0; i--) x = x * (double)c->primes[i] + (double)v[i];
            y[k] = {x * cs[k], x * sn[k]};  // m_k * omega^k
        }
        fft.run(y.data());  // X_{2u+1} = sum_k m_k omega^{k (2u+1)}
        for (int b = 0; b < B; b++) out[(size_t)ci * B + b] = y[(e[b] - 1) / 2].real() / scale;
    });
    return BCN_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- messages
// Serialised ciphertexts, plaintexts and keys (the client -> server messages
// of Sec. 2): a 64-byte little-endian header, then the payload words.
namespace {
constexpr uint32_t kMagic = 0x314E4342u;  // "BCN1" read as a little-endian word
constexpr size_t kHeader = 64;

void put32(uint8_t *p, uint32_t v) {
    for (int b = 0; b < 4; b++) p[b] = (uint8_t)(v >> (8 * b));
}
uint32_t get32(const uint8_t *p) {
    uint32_t v = 0;
    for (int b = 0; b < 4; b++) v |= (uint32_t)p[b] << (8 * b);
    return v;
}

// FNV-1a, 32 bits (Fowler, Noll, Vo): offset basis 2166136261, prime 16777619
uint32_t fnv1a(const uint8_t *p, size_t n) {
    uint32_t h = 2166136261u;
    for (size_t i = 0; i < n; i++) h = (h ^ p[i]) * 16777619u;
    return h;
}

// payload words and the prime index of word w (limb-major within each poly)
bool message_shape(const bcn_ctx *c, int kind, int level, int count, size_t *words, int *limbs) {
    if (kind == BCN_MSG_CIPHERTEXTS || kind == BCN_MSG_PLAINTEXTS) {
        if (level < 1 || level > c->L || count < 0) return false;
        *limbs = level;
        *words = (size_t)count * (kind == BCN_MSG_CIPHERTEXTS ? 2 : 1) * level * c->N;
        return true;
    }
    if (kind == BCN_MSG_RELIN_KEY || kind == BCN_MSG_GALOIS_KEY) {
        if (level != 0 || count != 1) return false;
        *limbs = c->L + c->K;
        *words = bcn_evk_words(c);
        return true;
    }
    return false;
}
}  // namespace

extern "C" size_t bcn_message_bytes(const bcn_ctx *c, int kind, int level, int count) {
    size_t words = 0;
    int limbs = 0;
    if (!c || !message_shape(c, kind, level, count, &words, &limbs)) return 0;
    return kHeader + 4 * words;
}

extern "C" bcn_status bcn_serialize(const bcn_ctx *c, int kind, int level, int count, uint32_t galois,
                                    const uint32_t *words, uint8_t *out, size_t out_bytes) {
    if (!c || !out) return fail(BCN_E_INVAL, "bcn_serialize: null argument");
    size_t n = 0;
    int limbs = 0;
    if (!message_shape(c, kind, level, count, &n, &limbs)) return fail(BCN_E_INVAL, "bcn_serialize: bad kind, level or count");
    if ((kind == BCN_MSG_GALOIS_KEY) != (galois != 0)) return fail(BCN_E_INVAL, "bcn_serialize: a Galois element belongs to Galois keys only");
    if (out_bytes < kHeader + 4 * n) return fail(BCN_E_BUDGET, "bcn_serialize: output buffer too small");
    if (n && !words) return fail(BCN_E_INVAL, "bcn_serialize: null payload");
    std::fill(out, out + kHeader, (uint8_t)0);
    put32(out + 0, kMagic);
    put32(out + 4, (uint32_t)kind);
    put32(out + 8, c->params.log_n);
    put32(out + 12, c->params.n_data);
    put32(out + 16, c->params.n_special);
    put32(out + 20, c->params.alpha);
    put32(out + 24, (uint32_t)level);
    put32(out + 28, (uint32_t)count);
    put32(out + 32, galois);
    put32(out + 36, (uint32_t)(n & 0xFFFFFFFFu));
    put32(out + 40, (uint32_t)((uint64_t)n >> 32));
    for (size_t w = 0; w < n; w++) put32(out + kHeader + 4 * w, words[w]);
    put32(out + 44, fnv1a(out + kHeader, 4 * n));
    return BCN_OK;
}

extern "C" bcn_status bcn_deserialize_header(const bcn_ctx *c, const uint8_t *in, size_t in_bytes, int *kind,
                                             int *level, int *count, uint32_t *galois) {
    if (!c || !in || !kind || !level || !count || !galois) return fail(BCN_E_INVAL, "bcn_deserialize_header: null argument");
    if (in_bytes < kHeader || get32(in) != kMagic) return fail(BCN_E_INVAL, "bcn_deserialize_header: not a message");
    for (size_t b = 48; b < kHeader; b++)
        if (in[b]) return fail(BCN_E_INVAL, "bcn_deserialize_header: reserved bytes are not zero");
    if (get32(in + 8) != c->params.log_n || get32(in + 12) != c->params.n_data ||
        get32(in + 16) != c->params.n_special || get32(in + 20) != c->params.alpha)
        return fail(BCN_E_INVAL, "bcn_deserialize_header: the message belongs to other parameters");
    const int k = (int)get32(in + 4), lv = (int)get32(in + 24), ct = (int)get32(in + 28);
    const uint32_t g = get32(in + 32);
    size_t n = 0;
    int limbs = 0;
    if (!message_shape(c, k, lv, ct, &n, &limbs)) return fail(BCN_E_INVAL, "bcn_deserialize_header: bad kind, level or count");
    if ((k == BCN_MSG_GALOIS_KEY) != (g != 0) || (g != 0 && (g % 2 == 0 || g >= 2 * (uint32_t)c->N)))
        return fail(BCN_E_INVAL, "bcn_deserialize_header: bad Galois element");
    const uint64_t nw = (uint64_t)get32(in + 36) | ((uint64_t)get32(in + 40) << 32);
    if (nw != n) return fail(BCN_E_INVAL, "bcn_deserialize_header: payload size does not match the shape");
    if (in_bytes < kHeader + 4 * n) return fail(BCN_E_INVAL, "bcn_deserialize_header: truncated payload");
    *kind = k;
    *level = lv;
    *count = ct;
    *galois = g;
    return BCN_OK;
}

extern "C" bcn_status bcn_deserialize(const bcn_ctx *c, const uint8_t *in, size_t in_bytes, uint32_t *words,
                                      size_t out_words) {
    int kind = 0, level = 0, count = 0;
    uint32_t g = 0;
    const bcn_status st = bcn_deserialize_header(c, in, in_bytes, &kind, &level, &count, &g);
    if (st != BCN_OK) return st;
    size_t n = 0;
    int limbs = 0;
    message_shape(c, kind, level, count, &n, &limbs);
    if (out_words < n || (n && !words)) return fail(BCN_E_BUDGET, "bcn_deserialize: output buffer too small");
    if (fnv1a(in + kHeader, 4 * n) != get32(in + 44)) return fail(BCN_E_INVAL, "bcn_deserialize: checksum mismatch");
    const size_t N = (size_t)c->N;
    for (size_t w = 0; w < n; w++) {
        const uint32_t v = get32(in + kHeader + 4 * w);
        const size_t limb = (w / N) % (size_t)limbs;
        if (v >= c->primes[limb]) return fail(BCN_E_INVAL, "bcn_deserialize: a residue is not below its prime");
        words[w] = v;
    }
    return BCN_OK;
}
