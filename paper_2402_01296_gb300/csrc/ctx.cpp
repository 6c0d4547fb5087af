// Context: prime chain, per-prime constants, NTT twiddles and the
// basis-conversion tables of hybrid key switching (host side).
#include <algorithm>
#include <cmath>
#include <new>

#include "bcn_internal.h"

namespace bcn {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }
bcn_status fail(bcn_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

uint64_t powmod64(uint64_t a, uint64_t e, uint64_t m) {
    uint64_t r = 1 % m;
    a %= m;
    while (e) {
        if (e & 1) r = mulmod64(r, a, m);
        a = mulmod64(a, a, m);
        e >>= 1;
    }
    return r;
}

// Deterministic Miller-Rabin for n < 3.4e14 (bases 2..17).
static bool is_prime_mr(uint64_t n) {
    if (n < 2) return false;
    static const uint64_t bases[] = {2, 3, 5, 7, 11, 13, 17};
    for (uint64_t b : bases)
        if (n % b == 0) return n == b;
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (uint64_t b : bases) {
        uint64_t x = powmod64(b, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s && comp; r++) {
            x = mulmod64(x, x, n);
            if (x == n - 1) comp = false;
        }
        if (comp) return false;
    }
    return true;
}

// The `count` largest primes below `bound` that are 1 mod 2N, descending.
static bool largest_ntt_primes(uint64_t bound, uint64_t two_n, int count, std::vector<uint64_t> &out) {
    uint64_t c = (bound - 1) / two_n * two_n + 1;
    if (c >= bound) c -= two_n;
    int got = 0;
    for (; got < count && c > two_n; c -= two_n)
        if (is_prime_mr(c)) { out.push_back(c); got++; }
    return got == count;
}

// a primitive 2N-th root of unity: g^((q-1)/2N) for the first g that gives psi^N = -1
static uint64_t primitive_2n_root(uint64_t q, uint64_t N) {
    for (uint64_t g = 2; g < q; g++) {
        uint64_t psi = powmod64(g, (q - 1) / (2 * N), q);
        if (powmod64(psi, N, q) == q - 1) return psi;
    }
    return 0;
}

static uint32_t bitrev(uint32_t x, int bits) {
    uint32_t r = 0;
    for (int i = 0; i < bits; i++) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

// Basis-conversion constants of hybrid key switching and rescale (see the
// layout comment on KsTables).
void build_ks_tables(bcn_ctx *c) {
    KsTables &t = c->ks;
    t.L = c->L; t.K = c->K; t.alpha = c->alpha; t.P = c->L + c->K;
    t.dnum_max = (c->L + c->alpha - 1) / c->alpha;
    const int L = c->L, K = c->K, A = c->alpha, P = t.P, D = t.dnum_max;
    size_t n_levels = (size_t)L + 1;
    size_t sz_dhat_inv = n_levels * D * A * 2, sz_dhat = n_levels * D * A * P * 2, sz_dprod = n_levels * D * P;
    size_t sz_phat_inv = (size_t)K * 2, sz_phat = (size_t)K * L * 2, sz_pmod = L, sz_pinv = (size_t)L * 2;
    size_t sz_qtop = (size_t)L * L * 2;
    auto up4 = [](size_t x) { return (x + 3) & ~(size_t)3; };  // keep every section 16-byte aligned
    t.off_dhat_inv = 0;
    t.off_dhat = up4(t.off_dhat_inv + sz_dhat_inv);
    t.off_dprod = up4(t.off_dhat + sz_dhat);
    t.off_phat_inv = up4(t.off_dprod + sz_dprod);
    t.off_phat = up4(t.off_phat_inv + sz_phat_inv);
    t.off_pmod = up4(t.off_phat + sz_phat);
    t.off_pinv = up4(t.off_pmod + sz_pmod);
    t.off_qtop_inv = up4(t.off_pinv + sz_pinv);
    size_t total = up4(t.off_qtop_inv + sz_qtop);
    t.host.assign(total, 0);
    uint32_t *h = t.host.data();
    auto put2 = [&](size_t off_words, size_t elem, uint64_t v, uint64_t q) {
        h[off_words + 2 * elem] = (uint32_t)v;
        h[off_words + 2 * elem + 1] = shoup_companion((uint32_t)v, (uint32_t)q);
    };
    const std::vector<uint64_t> &pr = c->primes;
    for (int n = 1; n <= L; n++) {
        int dnum = (n + A - 1) / A;
        for (int j = 0; j < dnum; j++) {
            int lo = j * A, hi = std::min((j + 1) * A, n);
            for (int p = 0; p < P; p++) {
                uint64_t dp = 1 % pr[p];
                for (int i = lo; i < hi; i++) dp = mulmod64(dp, pr[i] % pr[p], pr[p]);
                h[t.off_dprod + t.i_dprod(n, j, p)] = (uint32_t)dp;
            }
            for (int u = 0; u < hi - lo; u++) {
                int i = lo + u;
                uint64_t qi = pr[i], dh = 1;
                for (int i2 = lo; i2 < hi; i2++)
                    if (i2 != i) dh = mulmod64(dh, pr[i2] % qi, qi);
                put2(t.off_dhat_inv, t.i_dhat_inv(n, j, u), invmod64(dh, qi), qi);
                for (int p = 0; p < P; p++) {
                    uint64_t v = 1 % pr[p];
                    for (int i2 = lo; i2 < hi; i2++)
                        if (i2 != i) v = mulmod64(v, pr[i2] % pr[p], pr[p]);
                    put2(t.off_dhat, t.i_dhat(n, j, u, p), v, pr[p]);
                }
            }
        }
    }
    for (int m = 0; m < K; m++) {
        uint64_t pm = pr[L + m], ph = 1;
        for (int m2 = 0; m2 < K; m2++)
            if (m2 != m) ph = mulmod64(ph, pr[L + m2] % pm, pm);
        put2(t.off_phat_inv, m, invmod64(ph, pm), pm);
        for (int i = 0; i < L; i++) {
            uint64_t qi = pr[i], v = 1;
            for (int m2 = 0; m2 < K; m2++)
                if (m2 != m) v = mulmod64(v, pr[L + m2] % qi, qi);
            put2(t.off_phat, (size_t)m * L + i, v, qi);
        }
    }
    for (int i = 0; i < L; i++) {
        uint64_t qi = pr[i], pm = 1;
        for (int m = 0; m < K; m++) pm = mulmod64(pm, pr[L + m] % qi, qi);
        h[t.off_pmod + i] = (uint32_t)pm;
        put2(t.off_pinv, i, invmod64(pm, qi), qi);
    }
    for (int top = 1; top < L; top++)
        for (int i = 0; i < top; i++)
            put2(t.off_qtop_inv, (size_t)top * L + i, invmod64(pr[top] % pr[i], pr[i]), pr[i]);
}

}  // namespace bcn

using namespace bcn;

extern "C" {

const char *bcn_last_error(void) { return g_last_error.c_str(); }

bcn_status bcn_ctx_create(const bcn_params *p, int device, bcn_ctx **out) {
    if (!p || !out) return fail(BCN_E_INVAL, "bcn_ctx_create: null argument");
    *out = nullptr;
    if (p->log_n < 4 || p->log_n > (uint32_t)kMaxLogN) return fail(BCN_E_INVAL, "log_n must be in [4, 14]");
    if (p->n_data < 1 || p->n_data > 24) return fail(BCN_E_INVAL, "n_data must be in [1, 24]");
    if (p->n_special < 1 || p->n_special > 4) return fail(BCN_E_INVAL, "n_special must be in [1, 4]");
    if (p->alpha < 1 || p->alpha > p->n_special)
        return fail(BCN_E_INVAL, "alpha must be in [1, n_special] (digit product must not exceed P)");
    bcn_ctx *c = new (std::nothrow) bcn_ctx();
    if (!c) return fail(BCN_E_NOMEM, "bcn_ctx_create: out of host memory");
    c->params = *p;
    c->logN = (int)p->log_n;
    c->N = 1 << c->logN;
    c->L = (int)p->n_data;
    c->K = (int)p->n_special;
    c->alpha = (int)p->alpha;
    c->dnum = (c->L + c->alpha - 1) / c->alpha;
    c->device = -1;
    uint64_t two_n = 2 * (uint64_t)c->N;
    if (!largest_ntt_primes(1ull << 30, two_n, c->L, c->primes) ||
        !largest_ntt_primes(1ull << 31, two_n, c->K, c->primes)) {
        delete c;
        return fail(BCN_E_INVAL, "not enough NTT-friendly primes for this N");
    }
    // the device reduces MAC sums with a quotient estimate that wants the data
    // primes above 2^29 (they are the largest below 2^30 that are 1 mod 2N)
    for (int t = 0; t < c->L; t++) {
        if (c->primes[t] <= (1ull << 29)) {
            delete c;
            return fail(BCN_E_INVAL, "data primes must lie between 2^29 and 2^30");
        }
    }
    const int P = c->L + c->K, N = c->N;
    c->h_tw_fwd.resize(P);
    c->h_tw_inv.resize(P);
    c->h_pc.resize(P);
    for (int t = 0; t < P; t++) {
        uint64_t q = c->primes[t];
        uint64_t psi = primitive_2n_root(q, (uint64_t)N);
        uint64_t ipsi = invmod64(psi, q);
        std::vector<uint64_t> pw(N), ipw(N);
        uint64_t a = 1, b = 1;
        for (int k = 0; k < N; k++) { pw[k] = a; ipw[k] = b; a = mulmod64(a, psi, q); b = mulmod64(b, ipsi, q); }
        c->h_tw_fwd[t].resize(2 * (size_t)N);
        c->h_tw_inv[t].resize(2 * (size_t)N);
        for (int k = 0; k < N; k++) {
            uint32_t r = bitrev((uint32_t)k, c->logN);
            c->h_tw_fwd[t][2 * k] = (uint32_t)pw[r];
            c->h_tw_fwd[t][2 * k + 1] = shoup_companion((uint32_t)pw[r], (uint32_t)q);
            c->h_tw_inv[t][2 * k] = (uint32_t)ipw[r];
            c->h_tw_inv[t][2 * k + 1] = shoup_companion((uint32_t)ipw[r], (uint32_t)q);
        }
        PrimeConst &pc = c->h_pc[t];
        pc.q = (uint32_t)q;
        uint32_t inv = 1;  // q^{-1} mod 2^32 by Newton iteration
        for (int i = 0; i < 5; i++) inv *= 2u - (uint32_t)q * inv;
        pc.qneg_inv = (uint32_t)(0u - inv);
        pc.r_mod = (uint32_t)((1ull << 32) % q);
        pc.r_shoup = shoup_companion(pc.r_mod, pc.q);
        pc.ninv = (uint32_t)invmod64((uint64_t)N, q);
        pc.ninv_shoup = shoup_companion(pc.ninv, pc.q);
        pc.half = (uint32_t)((q - 1) / 2);
        pc.rn = (uint32_t)mulmod64(pc.r_mod, pc.ninv, q);
        pc.rn_shoup = shoup_companion(pc.rn, pc.q);
        pc.one = 1;
        pc.nmod = (uint32_t)((uint64_t)N % q);
        pc.nmod_shoup = shoup_companion(pc.nmod, pc.q);
        pc.barrett = (uint64_t)(((unsigned __int128)1 << 64) / q);
        pc.mac_offset = ((1ull << 58) / q + 1) * q;
    }
    build_ks_tables(c);
    if (device >= 0) {
        c->device = device;
        bcn_status st = device_ctx_init(c);
        if (st != BCN_OK) {
            std::string keep = g_last_error;
            device_ctx_free(c);
            delete c;
            return fail(st, keep);
        }
    }
    *out = c;
    return BCN_OK;
}

bcn_status bcn_ctx_destroy(bcn_ctx *c) {
    if (!c) return BCN_OK;
    if (c->device >= 0) device_ctx_free(c);
    delete c;
    return BCN_OK;
}

bcn_status bcn_ctx_get_info(const bcn_ctx *c, bcn_ctx_info *o) {
    if (!c || !o) return fail(BCN_E_INVAL, "bcn_ctx_get_info: null argument");
    o->N = (uint32_t)c->N; o->L = (uint32_t)c->L; o->K = (uint32_t)c->K;
    o->alpha = (uint32_t)c->alpha; o->dnum = (uint32_t)c->dnum; o->device = c->device;
    return BCN_OK;
}

bcn_status bcn_ctx_primes(const bcn_ctx *c, uint64_t *out) {
    if (!c || !out) return fail(BCN_E_INVAL, "bcn_ctx_primes: null argument");
    for (size_t i = 0; i < c->primes.size(); i++) out[i] = c->primes[i];
    return BCN_OK;
}

size_t bcn_evk_words(const bcn_ctx *c) {
    if (!c) return 0;
    return (size_t)c->dnum * 2 * (c->L + c->K) * c->N;
}

}  // extern "C"
