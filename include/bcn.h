/*
 * bcn.h -- C ABI of the GB300 ciphertext-branch engine for bi-CryptoNets
 * ("Bi-CryptoNets: Leveraging Different-Level Privacy for Encrypted
 * Inference", arXiv 2402.01296).
 *
 * The paper splits an image into a sensitive segment, encrypted with CKKS and
 * evaluated by a ciphertext branch, and an insensitive segment, perturbed and
 * evaluated in plaintext by a plaintext branch whose features enter the
 * ciphertext branch through unidirectional additions (Sec. 3, Sec. 3.2).  The
 * client holds the secret key and the server evaluates without it (Sec. 2,
 * threat model).  This library implements, in that order of the problem:
 *   keygen / encrypt of the sensitive segment       (client, host C++)
 *   plaintext-branch forward on the perturbed image (device, CUDA fp32)
 *   encode of its features                          (client, host C++, fp64)
 *   ciphertext-branch evaluation                    (server, device, CUDA)
 *   decrypt / decode                                (client, host C++)
 * The scheme is levelled RNS-CKKS with one image per slot (batch packing,
 * App. D); every step of the evaluation is exact modular integer arithmetic
 * in hand-written sm_103a kernels.
 *
 * Conventions
 *   - Every call returns a bcn_status; BCN_OK is 0, errors are negative.
 *     bcn_last_error() gives a thread-local message for the last failure.
 *     No exception and no device trap crosses this boundary.
 *   - Ring degree N = 2^log_n.  Data primes q_0 > q_1 > ... > q_{L-1} are the
 *     L largest primes below 2^30 with q = 1 (mod 2N); special primes
 *     p_0..p_{K-1} are the K largest primes below 2^31 with p = 1 (mod 2N).
 *     A ciphertext "at level l" lives modulo q_0 ... q_{l-1}.
 *   - Interchange layout (host and device): uint32 residues, canonical in
 *     [0, q), coefficient form, limbs in chain order:
 *         ciphertexts  [n_ct][2][level][N]   (c0, c1)
 *         plaintexts   [n_pt][level][N]
 *         secret key   [N] int8 in {-1, 0, 1}
 *         evk          [dnum][2][L+K][N]     (b, a) per digit, limbs q_0..q_{L-1}
 *                                            then p_0..p_{K-1}; dnum = ceil(L/alpha)
 *   - Buffers are owned by the caller.  The library owns only the opaque
 *     bcn_ctx / bcn_model / bcn_plain_model objects (and the small device
 *     tables inside them).  Device calls are asynchronous on the given CUDA
 *     stream (NULL = legacy default stream); host calls are synchronous.
 *   - A ctx created with device < 0 is host-only: client calls work, device
 *     calls return BCN_E_INVAL.
 */
#ifndef BCN_H
#define BCN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BCN_OK = 0,
    BCN_E_INVAL = -1,   /* bad argument, shape or layout */
    BCN_E_NOMEM = -2,   /* host or device allocation failed */
    BCN_E_CUDA = -3,    /* a CUDA runtime call failed */
    BCN_E_LEVEL = -4,   /* not enough levels left for the requested operation */
    BCN_E_SCALE = -5,   /* an encoded coefficient does not fit in 63 bits */
    BCN_E_TIMEOUT = -6, /* a bounded device-side wait gave up */
    BCN_E_BUDGET = -7   /* the caller's workspace is too small */
} bcn_status;

typedef struct bcn_ctx bcn_ctx;
typedef struct bcn_model bcn_model;
typedef struct bcn_plain_model bcn_plain_model;

typedef struct {
    uint32_t log_n;        /* N = 2^log_n, 4 <= log_n <= 14 */
    uint32_t n_data;       /* L data primes (between 2^29 and 2^30), 1 <= L <= 24 */
    uint32_t n_special;    /* K special primes (< 2^31), 1 <= K <= 4 */
    uint32_t alpha;        /* primes per key-switching digit, 1 <= alpha <= K */
} bcn_params;

typedef struct {
    uint32_t N, L, K, alpha, dnum; /* dnum = ceil(L / alpha) */
    int device;                    /* CUDA ordinal, or -1 for a host-only ctx */
} bcn_ctx_info;

/* Message of the last failure on this thread ("" if none). */
const char *bcn_last_error(void);

/* ---------------------------------------------------------------- context */
/* Builds the prime chain (the largest primes below 2^30, then below 2^31,
 * that are 1 mod 2N) and the NTT / basis-conversion tables; with device >= 0
 * also uploads the device tables to that GPU.  BCN_E_INVAL if the parameters
 * are out of range or the chain cannot be built (a data prime not above 2^29). */
bcn_status bcn_ctx_create(const bcn_params *params, int device, bcn_ctx **out);
bcn_status bcn_ctx_destroy(bcn_ctx *ctx);
bcn_status bcn_ctx_get_info(const bcn_ctx *ctx, bcn_ctx_info *out);
/* primes_out: L + K values, data primes then special primes. */
bcn_status bcn_ctx_primes(const bcn_ctx *ctx, uint64_t *primes_out);
/* number of uint32 words of an evaluation key: dnum * 2 * (L + K) * N */
size_t bcn_evk_words(const bcn_ctx *ctx);

/* Reads and clears the context's device status word (synchronous): 0 when no
 * kernel gave up a bounded wait since the last call; otherwise a bit set by
 * the kernel that gave up (1: the tensor-core MAC's wait for its MMAs), whose
 * outputs are then unspecified (bits 2 and 4: see the debug checks; bit 8: see
 * the seeded ciphertexts). */
bcn_status bcn_device_status(const bcn_ctx *ctx, uint32_t *status);
/* Debug checks (no compute-sanitizer here; the checks take its place for the
 * inputs): with them on -- bcn_ctx_set_debug(ctx, 1), or every context of a
 * library built with -DBCN_DEBUG -- bcn_eval, bcn_eval_stacked, bcn_op_mac,
 * bcn_op_square_relin_rescale, bcn_op_rotate, bcn_op_rotate_many and the
 * diagonal-method layers first run device-side checks on their inputs: every
 * residue of the input ciphertexts and feature plaintexts below its prime, and
 * (bcn_eval) every MAC tap index inside [-1, n_in) and output index inside
 * [0, n_out).  A failed check sets a bit of the status word (2: a residue not
 * below its prime; 4: an index out of range) instead of trapping; the host
 * waits for the checks, clears those bits and returns BCN_E_INVAL without
 * launching the operation.  The checks read every input once more and
 * synchronise the stream, and they are skipped on a stream being captured
 * into a graph.  Off by default. */
/* Block shape of the NTT-based kernels (the square activation's, the key
 * switch's, ModDown's, the transforms'): 0 the default, 1 an alternative, for
 * N = 4096 (16 residues per thread; alternative 8), 8192 (16; alternative 32)
 * and 16384 (32; alternative 16); smaller rings have one shape.  Every later
 * call on the context uses the selected shape; results are identical (the
 * element order of the NTT domain does not depend on the shape), only the
 * speed differs -- the autotuner measures both.  Not to be changed while work
 * on the context is in flight.  bcn_ctx_get_ntt_shape: the selection and its
 * residues per thread (-1 below N = 4096). */
bcn_status bcn_ctx_set_ntt_shape(bcn_ctx *ctx, int shape);
bcn_status bcn_ctx_get_ntt_shape(const bcn_ctx *ctx, int *shape, int *residues_per_thread);
bcn_status bcn_ctx_set_debug(bcn_ctx *ctx, int on);
bcn_status bcn_ctx_get_debug(const bcn_ctx *ctx, int *on);

/* ------------------------------------------------------------ client side */
/* Secret key (uniform ternary) and relinearisation key for hybrid key
 * switching (digit j covers q_{j*alpha} .. q_{j*alpha+alpha-1}):
 *     evk_j = (-a_j s + e_j + P g_j s^2, a_j),  P = prod p_m,
 *     g_j = 1 mod the primes of digit j, 0 mod every other prime,
 * a_j uniform, e_j centred binomial (eta 21).  Randomness: SplitMix64; the
 * stream (seed, tag, index) starts from state mix64(seed + G*((tag << 40) +
 * index + 1)), G = 0x9E3779B97F4A7C15, and each draw is state += G,
 * mix64(state).  Tags: 1 secret key (index 0; s = (r mod 3) - 1), 2 evk a_j
 * (index j*256 + limb; low 32 bits rejected above floor(2^32/q)*q, then
 * mod q), 3 evk e_j (index j; popcount of 21 bits minus popcount of the next
 * 21), 4 encryption a (index ct*256 + limb), 5 encryption e (index ct).
 * The key is what lets the server compute Mult(c1, c2) of App. A without the
 * secret.  sk_out: [N] int8; evk_out: bcn_evk_words() uint32, host memory. */
bcn_status bcn_keygen(const bcn_ctx *ctx, uint64_t seed, int8_t *sk_out, uint32_t *evk_out);

/* Per-tensor symmetric int8 quantisation of float weights:
 * s_w = max|w| / 127, w_int = round(w / s_w) (ties away from zero), computed
 * in fp64.  The ciphertext branch multiplies by integers (Mult(c, u) with an
 * integer u costs no level).  Host memory. */
bcn_status bcn_quantize(const float *w, size_t n, int8_t *w_int_out, double *s_w_out);

/* CKKS encode (App. A: N/2 slots per plaintext) of real vectors:
 * values [n_vec][B] (B <= N/2; slots B..N/2-1 are zero) at `scale` ->
 * pts_out [n_vec][level][N]: m_j = round(scale * (2/N) sum_k z_k cos(pi j 5^k / N)),
 * computed with an FFT in fp64; beyond 2^52 in magnitude m_j is the integer
 * value of the fp64 product itself (which has no fractional part), reduced mod
 * each prime.  BCN_E_SCALE if a product is not finite. Host memory. */
bcn_status bcn_encode(const bcn_ctx *ctx, const double *values, int n_vec, int B, int level, double scale,
                      uint32_t *pts_out);
/* The same encoding as integer coefficients, coeffs_out [n_vec][N] int64 (the
 * m_j whose residues bcn_encode writes), for uploads that let the device reduce
 * them (bcn_expand_i64, bcn_eval_host_compact_async): 8 bytes a coefficient
 * whatever the level.  BCN_E_SCALE if a coefficient is not below 2^63 in
 * magnitude (use bcn_encode there).  Host. */
bcn_status bcn_encode_i64(const bcn_ctx *ctx, const double *values, int n_vec, int B, double scale,
                          int64_t *coeffs_out);
/* coeffs_dev [n][N] int64 -> pts_dev [n][level][N], m_j mod q_i (device,
 * asynchronous on `cuda_stream`; the buffers must not overlap). */
bcn_status bcn_expand_i64(const bcn_ctx *ctx, const int64_t *coeffs_dev, int n, int level, uint32_t *pts_dev,
                          void *cuda_stream);

/* Symmetric encryption (the client holds the key, Sec. 2):
 * ct = (-a s + e + m, a) with a uniform per limb and e centred binomial, drawn
 * from SplitMix64 streams of `seed` indexed by the ciphertext's position in
 * this call.  pts [n_ct][level][N] -> cts_out [n_ct][2][level][N].  Host. */
bcn_status bcn_encrypt(const bcn_ctx *ctx, const int8_t *sk, const uint32_t *pts, int n_ct, int level,
                       uint64_t seed, uint32_t *cts_out);

/* Encrypt the sensitive segment (Sec. 3): images [B][H][W][C] uint8; seg =
 * {y0, x0, h, w}.  Ciphertext (c, y, x) (row-major) holds pixel
 * (y0+y, x0+x, c) / 255 of every image, image b in slot b, encoded at `scale`
 * at the top level L and encrypted as bcn_encrypt does.
 * cts_out: [C*h*w][2][L][N], host memory. */
bcn_status bcn_encrypt_segment(const bcn_ctx *ctx, const int8_t *sk, const uint8_t *images, int B, int H, int W,
                               int C, const int seg[4], double scale, uint64_t seed, uint32_t *cts_out);

/* Seeded ciphertexts (Sec. 2: the client uploads every encrypted segment; c1 = a
 * is uniform noise drawn from the seed, so c0 and the seed carry the whole
 * ciphertext in half the bytes).  bcn_encrypt_seeded / bcn_encrypt_segment_seeded
 * write c0 alone, [n_ct][level][N] (host), identical to the c0 of bcn_encrypt /
 * bcn_encrypt_segment with the same arguments.  bcn_expand_seeded (device):
 * c0_dev [n_ct][level][N] -> cts_dev [n_ct][2][level][N], c1 of ciphertext k
 * drawn from the stream of `seed` with index (ct_base + k) * 256 + limb exactly
 * as bcn_encrypt draws it (SplitMix64, rejection below floor(2^32/q) q); the
 * buffers must not overlap.  Asynchronous on `cuda_stream`; a limb that would
 * need more than N + 16384 draws (never seen: about one draw in 30000 is
 * rejected) sets bit 8 of the status word. */
bcn_status bcn_encrypt_seeded(const bcn_ctx *ctx, const int8_t *sk, const uint32_t *pts, int n_ct, int level,
                              uint64_t seed, uint32_t *c0_out);
bcn_status bcn_encrypt_segment_seeded(const bcn_ctx *ctx, const int8_t *sk, const uint8_t *images, int B, int H,
                                      int W, int C, const int seg[4], double scale, uint64_t seed, uint32_t *c0_out);
bcn_status bcn_expand_seeded(const bcn_ctx *ctx, const uint32_t *c0_dev, int n_ct, int level, uint64_t seed,
                             int ct_base, uint32_t *cts_dev, void *cuda_stream);

/* The client's last step (Sec. 2 threat model: only the client can decrypt
 * the inference result; App. A: the decryption function D, and the N/2 slots
 * that carry one value each): decrypt m = c0 + c1 s (mod q_i), recombine the
 * residues into the centred integer (balanced-digit Garner CRT, exact), decode
 * the first B slots and divide by `scale`.  cts [n_ct][2][level][N] -> out
 * [n_ct][B], host memory; BCN_E_INVAL on a null buffer, a level outside
 * 1..L or B outside 0..N/2. */
bcn_status bcn_decrypt_decode(const bcn_ctx *ctx, const int8_t *sk, const uint32_t *cts, int n_ct, int level,
                              double scale, int B, double *out);

/* Messages (Sec. 2: the client sends its encrypted segments, plaintexts and
 * evaluation keys to the server and receives the output ciphertexts).  A
 * message is a 64-byte header followed by the payload words; every field and
 * word is little-endian:
 *   bytes  0..3   magic "BCN1"
 *          4..7   kind (bcn_message_kind)
 *          8..23  log_n, n_data, n_special, alpha of the context (uint32 each)
 *         24..27  level (ciphertexts, plaintexts; 0 for keys)
 *         28..31  count (ciphertexts or plaintexts; 1 for a key)
 *         32..35  Galois element g (Galois keys; 0 otherwise)
 *         36..43  payload words (uint64)
 *         44..47  FNV-1a (32-bit) checksum of the payload bytes
 *         48..63  zero
 * Payload: ciphertexts [count][2][level][N], plaintexts [count][level][N]
 * (coefficient form), keys [dnum][2][L+K][N] in the raw form bcn_keygen and
 * bcn_galois_keygen write (the server prepares them with bcn_evk_prepare);
 * every residue below its prime.  bcn_message_bytes: the message size (0 for a
 * bad shape).  bcn_serialize writes header and payload to `out`.
 * bcn_deserialize_header checks the magic, the kind, the reserved bytes, the
 * context's parameters, the payload size against the shape and the buffer,
 * and reports kind, level, count and g; bcn_deserialize also verifies the
 * checksum and that every residue is below its prime, then copies the words.
 * BCN_E_INVAL on any mismatch, BCN_E_BUDGET if an output buffer is too small.
 * Host memory. */
typedef enum { BCN_MSG_CIPHERTEXTS = 1, BCN_MSG_RELIN_KEY = 2, BCN_MSG_GALOIS_KEY = 3, BCN_MSG_PLAINTEXTS = 4 } bcn_message_kind;
size_t bcn_message_bytes(const bcn_ctx *ctx, int kind, int level, int count);
bcn_status bcn_serialize(const bcn_ctx *ctx, int kind, int level, int count, uint32_t galois, const uint32_t *words,
                         uint8_t *out, size_t out_bytes);
bcn_status bcn_deserialize_header(const bcn_ctx *ctx, const uint8_t *in, size_t in_bytes, int *kind, int *level,
                                  int *count, uint32_t *galois);
bcn_status bcn_deserialize(const bcn_ctx *ctx, const uint8_t *in, size_t in_bytes, uint32_t *words_out,
                           size_t out_words);

/* ------------------------------------------------ plaintext branch (fp32) */
/* The plaintext branch (Sec. 3.1) runs on the whole image with the sensitive
 * segment set to zero and the insensitive segment perturbed by additive
 * noise; its taps give the unidirectional-connection features of Sec. 3.2:
 * Resize = centre crop (offset floor((h_p - h_c)/2)), CRot = a ch_c x ch_p
 * channel mix, or a fully connected map of the flattened (c, y, x) map. */
typedef enum {
    BCN_PLAIN_CONV = 0,     /* 2-D cross-correlation, weights [cout][cin][k][k], optional ReLU */
    BCN_PLAIN_AVGPOOL2 = 1, /* 2x2 average pool, stride 2 */
    BCN_PLAIN_TAP_CROP_CROT = 2, /* tap: centre crop to hc x wc, CRot weights [ch_c][ch_p] */
    BCN_PLAIN_TAP_FC = 3,   /* tap: fully connected, weights [n_out][C*H*W], then [n_out] bias if bias != 0 */
    /* tap: the plaintext neurons of the two-layer feature integration (Sec. 3.3)
     * and their contribution to the ciphertext neurons of the second layer:
     *     h = sigma(W'_1 x_p + b'_1),  feature = W_2 h + b_2,
     * x_p the flattened (c, y, x) map, sigma the square activation; weights
     * W'_1 [n_hidden][C*H*W], b'_1 [n_hidden], W_2 [n_out][n_hidden], b_2 [n_out]
     * back to back */
    BCN_PLAIN_TAP_INTEGRATE = 4
} bcn_plain_op;

typedef struct {
    int op;               /* bcn_plain_op */
    int cin, cout, k, stride, pad, relu; /* BCN_PLAIN_CONV */
    int hc, wc, ch_c;     /* BCN_PLAIN_TAP_CROP_CROT */
    int n_out;            /* BCN_PLAIN_TAP_FC, BCN_PLAIN_TAP_INTEGRATE */
    int n_hidden;         /* BCN_PLAIN_TAP_INTEGRATE */
    int bias;             /* BCN_PLAIN_TAP_FC: the weights are followed by a bias */
    const float *weights; /* host fp32, layout above (NULL for AVGPOOL2) */
} bcn_plain_stage;

bcn_status bcn_plain_model_create(bcn_ctx *ctx, const bcn_plain_stage *stages, int n_stages, int H, int W, int C,
                                  const int seg[4], bcn_plain_model **out);
bcn_status bcn_plain_model_destroy(bcn_plain_model *m);
/* total number of features over all taps (the rows of feats_dev) */
bcn_status bcn_plain_feature_count(const bcn_plain_model *m, int *n_feat);
bcn_status bcn_plain_workspace_bytes(const bcn_plain_model *m, int B, size_t *bytes);
/* images_dev [B][H][W][C] uint8, noise_dev [B][H][W][C] fp32 (the perturbation
 * drawn by the client), feats_dev [n_feat][B] fp32: taps in order, each tap's
 * features flattened (c, y, x).  Device memory; asynchronous on `stream`. */
bcn_status bcn_plain_branch_forward(const bcn_plain_model *m, const uint8_t *images_dev, const float *noise_dev,
                                    int B, float *feats_dev, void *workspace_dev, size_t workspace_bytes,
                                    void *cuda_stream);

/* -------------------------------------------------- ciphertext branch (server) */
typedef enum { BCN_LAYER_CONV = 0, BCN_LAYER_DENSE = 1 } bcn_layer_type;

/* One linear layer of the ciphertext branch: conv (weights [cout][cin][k][k],
 * input map cin x h x w, stride, zero padding `pad`) or dense (weights
 * [n_out][n_in]); int8 weights w_int with scale s_w.  Inputs and outputs are
 * flattened in (channel, row, column) order.  add != 0: a plaintext-branch
 * feature is added to every output (the unidirectional connection
 * x_{c,l} + z_{p,l}, Sec. 3.2).  square != 0: square activation (App. B),
 * i.e. tensor square, relinearisation and rescale (one level). */
typedef struct {
    int type;
    int cin, h, w, cout, k, stride, pad; /* conv */
    int n_in, n_out;                     /* dense */
    int add, square;
    const int8_t *w_int; /* host */
    double s_w;
} bcn_layer;

typedef struct {
    int n_layers;
    int n_in;         /* input ciphertexts of layer 0 (all requests of a stacked model) */
    int n_out;        /* output ciphertexts of the last layer (all requests of a stacked model) */
    int out_level;    /* level of the output ciphertexts */
    int n_add;        /* layers with add != 0 */
    int stack;        /* requests evaluated side by side (1 unless bcn_model_create_stacked) */
} bcn_model_info;

bcn_status bcn_model_create(bcn_ctx *ctx, const bcn_layer *layers, int n_layers, bcn_model **out);
/* The same network for `requests` (1..16) slot batches side by side, so that
 * one launch of every kernel serves all of them: request r's input
 * ciphertexts, feature plaintexts and outputs are the r-th block of each
 * buffer of bcn_eval ([requests * n][...] in place of [n][...]); every layer's
 * output groups are replicated with the inputs and outputs offset accordingly.
 * Each request may come from a different client: bcn_eval_stacked takes one
 * evaluation key per request, and the key switch of a ciphertext uses its
 * request's key.  Results equal `requests` separate evaluations bit for bit. */
bcn_status bcn_model_create_stacked(bcn_ctx *ctx, const bcn_layer *layers, int n_layers, int requests,
                                    bcn_model **out);
bcn_status bcn_model_destroy(bcn_model *m);
/* Ciphertexts per key-switching chunk of the square layers (0: automatic, a
 * chunk's intermediates bounded by 1 GiB).  Changes bcn_eval_workspace_bytes;
 * results do not depend on it. */
bcn_status bcn_model_set_chunk(bcn_model *m, int chunk);
/* MAC implementation: 0 (default) runs the layer groups with at most 512 taps
 * and at least 32 outputs (or at least 10 outputs and 64 taps) on the tensor
 * cores (the residues split into byte planes, fp16 operands, exact fp32 sums),
 * the rest on the CUDA cores with 64-bit multiply-adds; 1 runs every MAC on the
 * CUDA cores that way; 2 runs every MAC on the CUDA cores with dp4a on byte
 * planes (int8 weights against uint8 bytes, exact 32-bit sums; 64-bit
 * multiply-adds past 32768 taps), measured slower.  Results are identical in
 * every case. */
bcn_status bcn_model_set_mac_impl(bcn_model *m, int impl);
/* Streams of one evaluation: 1 (default) runs each square layer's chunk in two
 * halves side by side (the second on an internal stream forked from and joined
 * back to the caller's) and transforms the feature plaintexts that join
 * NTT-domain ciphertexts on another internal stream while earlier layers run;
 * 0 runs every kernel in order on the caller's stream (the plain per-request
 * path: one kernel at a time).  Results are identical either way. */
bcn_status bcn_model_set_overlap(bcn_model *m, int on);
bcn_status bcn_model_get_info(const bcn_model *m, bcn_model_info *out);
/* per layer: live level at its input and its output count (arrays of n_layers) */
bcn_status bcn_model_layers(const bcn_model *m, int *level_out, int *n_out_out);
/* Scale bookkeeping (host fp64): the weights divide the scale by s_w, a square
 * squares it, a rescale divides it by the dropped prime.  add_scales_out
 * [n_add]: the scale each added feature must be encoded at; out_scale: the
 * scale of the outputs, for bcn_decrypt_decode. */
bcn_status bcn_model_scales(const bcn_model *m, double input_scale, double *add_scales_out, double *out_scale);

/* Convert a boundary-layout evaluation key (coefficient form, device memory)
 * into the evaluator's form (NTT domain, Montgomery representation; the limbs
 * on special prime p_m also times Phat_m^{-1} = (P / p_m)^{-1} mod p_m, the
 * first factor of every ModDown conversion, applied here once) in
 * evk_eval_dev (same size; may equal evk_dev for in-place).  Relinearisation
 * and Galois keys alike. */
bcn_status bcn_evk_prepare(const bcn_ctx *ctx, const uint32_t *evk_dev, uint32_t *evk_eval_dev, void *cuda_stream);

bcn_status bcn_eval_workspace_bytes(const bcn_model *m, size_t *bytes);

/* Ciphertext-branch evaluation (the hot path; Sec. 3.2: the ciphertext
 * branch with its unidirectional connections x_{c,l} + CRot(Resize(x_{p,l})),
 * built from the CKKS operations of App. A -- Mult(c, u) with the integer
 * weights, Add(c1, c2) for the sums, Add(c, u) for the features, Mult(c1, c2)
 * for the square activation of App. B): for each layer the integer
 * weight multiply-accumulate, the optional feature add, the optional
 * square + relinearise + rescale.  cts_dev [n_in][2][L][N];
 * pts_dev[a] [n_out of the a-th add layer][its level][N] encoded at the scale
 * bcn_model_scales gives; out_dev [n_out][2][out_level][N].  All device
 * memory in the interchange layout (coefficient form; between square layers
 * the evaluation keeps ciphertexts in the NTT domain and transforms a copy of
 * the features that join them, in the workspace); evk_eval_dev from
 * bcn_evk_prepare; workspace of at least bcn_eval_workspace_bytes.
 * Asynchronous on `cuda_stream` (it may also use the model's internal streams,
 * forked from and joined back to `cuda_stream`).  Errors: BCN_E_BUDGET if the
 * workspace is smaller than bcn_eval_workspace_bytes, BCN_E_INVAL on a null or
 * unaligned (16-byte) buffer or a missing feature plaintext, BCN_E_CUDA if a
 * launch fails; nothing is written to out_dev before the first launch. */
bcn_status bcn_eval(const bcn_model *m, const uint32_t *evk_eval_dev, const uint32_t *cts_dev,
                    const uint32_t *const *pts_dev, uint32_t *out_dev, void *workspace_dev, size_t workspace_bytes,
                    void *cuda_stream);

/* Evaluation of a stacked model (bcn_model_create_stacked) with one prepared
 * evaluation key per request: evk_evals, a host array of n_keys device
 * pointers, n_keys equal to the model's request count; the other arguments as
 * for bcn_eval (bcn_eval on a stacked model uses its one key for every
 * request).  BCN_E_INVAL if n_keys differs or a key is null or unaligned. */
bcn_status bcn_eval_stacked(const bcn_model *m, const uint32_t *const *evk_evals, int n_keys, const uint32_t *cts_dev,
                            const uint32_t *const *pts_dev, uint32_t *out_dev, void *workspace_dev,
                            size_t workspace_bytes, void *cuda_stream);

/* Same evaluation with host inputs and outputs: copies cts_host and pts_host
 * to device staging buffers carved from the workspace (size:
 * bcn_eval_host_workspace_bytes), evaluates, copies the result to out_host
 * and synchronises the stream.  Page-locked host buffers give full-rate copies. */
bcn_status bcn_eval_host_workspace_bytes(const bcn_model *m, size_t *bytes);
bcn_status bcn_eval_host(const bcn_model *m, const uint32_t *evk_eval_dev, const uint32_t *cts_host,
                         const uint32_t *const *pts_host, uint32_t *out_host, void *workspace_dev,
                         size_t workspace_bytes, void *cuda_stream);
/* The same without the final synchronisation: the kernels and the result read
 * are queued on `cuda_stream` and out_host holds the result once that stream
 * has passed this call (synchronise it or record an event).  The host-to-device
 * copies run on the library's own streams and wait only for the previous
 * host-buffer evaluation that used the same workspace (the first time, for the
 * work queued on `cuda_stream`), so with two workspaces on one stream the next
 * evaluation's inputs copy while this one computes.  The host buffers must
 * stay valid and unchanged until the result is read, and earlier work must not
 * write the host input buffers. */
bcn_status bcn_eval_host_async(const bcn_model *m, const uint32_t *evk_eval_dev, const uint32_t *cts_host,
                               const uint32_t *const *pts_host, uint32_t *out_host, void *workspace_dev,
                               size_t workspace_bytes, void *cuda_stream);
/* bcn_eval_host_async from seeded ciphertexts: c0_host [n_in][L][N] (from
 * bcn_encrypt_segment_seeded with `seed`) is copied into the staging area's
 * first halves and c1 drawn there on the device, so half the ciphertext bytes
 * cross to the device.  Results equal bcn_eval_host_async's on the full
 * ciphertexts.  Single-request models only (a stacked model's requests have
 * seeds of their own): BCN_E_INVAL otherwise. */
bcn_status bcn_eval_host_seeded_async(const bcn_model *m, const uint32_t *evk_eval_dev, const uint32_t *c0_host,
                                      uint64_t seed, const uint32_t *const *pts_host, uint32_t *out_host,
                                      void *workspace_dev, size_t workspace_bytes, void *cuda_stream);
/* The same with the feature plaintexts as their integer coefficients
 * (bcn_encode_i64): feats_host[a] [n_out][N] int64 for the a-th layer with a
 * feature, 8 bytes a coefficient instead of 4 per prime; the device reduces
 * them mod each prime into the staging area (through the workspace's first
 * ciphertext buffer, so the evaluation's first layer waits for all of them).
 * Results equal bcn_eval_host_seeded_async's with the residues bcn_encode
 * gives.  BCN_E_BUDGET if the integer features exceed that buffer (the largest
 * layer output of the model). */
bcn_status bcn_eval_host_compact_async(const bcn_model *m, const uint32_t *evk_eval_dev, const uint32_t *c0_host,
                                       uint64_t seed, const int64_t *const *feats_host, uint32_t *out_host,
                                       void *workspace_dev, size_t workspace_bytes, void *cuda_stream);

/* ------------------------------------------------ batched evaluation (device) */
/* Many evaluations of different models (ring degrees, segment sizes) replayed
 * as one CUDA graph: items are spread over `lanes` streams by the longest-
 * processing-time rule on bcn_model_cost, each lane evaluates its items in
 * turn on its own workspace slice, the lanes run concurrently.  This is the
 * batched form of the ciphertext-branch evaluation (one launch for all items);
 * every item's output equals that of bcn_eval on the same inputs.  All
 * pointers are device memory on one device except `pts`, a host array of
 * device pointers (copied at creation). */
typedef struct bcn_batch bcn_batch;
typedef struct {
    const bcn_model *model;
    const uint32_t *evk_eval;     /* from bcn_evk_prepare on the model's ctx */
    const uint32_t *cts;          /* [n_in][2][L][N] */
    const uint32_t *const *pts;   /* one per add layer, as for bcn_eval */
    uint32_t *out;                /* [n_out][2][out_level][N] */
} bcn_batch_item;

/* workspace bytes the batch needs with this many lanes (sum over lanes of the
 * largest bcn_eval_workspace_bytes among the lane's items) */
bcn_status bcn_batch_plan(const bcn_batch_item *items, int n_items, int lanes, size_t *workspace_bytes);
/* Capture the launch sequence into a graph (the items' device must be
 * current; the workspace and every item buffer are baked into the graph). */
bcn_status bcn_batch_create(const bcn_batch_item *items, int n_items, int lanes, void *workspace_dev,
                            size_t workspace_bytes, bcn_batch **out);
/* one graph launch on `cuda_stream` (asynchronous) */
bcn_status bcn_batch_launch(bcn_batch *b, void *cuda_stream);
/* lane of every item, [n_items] */
bcn_status bcn_batch_lanes(const bcn_batch *b, int *lane_of_item);
bcn_status bcn_batch_destroy(bcn_batch *b);
/* the analytic cost the lane assignment uses: MAC products plus about four
 * products per NTT butterfly of the square layers */
bcn_status bcn_model_cost(const bcn_model *m, double *cost);

/* ------------------------------------------------- kernel timing (device) */
/* Classes of the kernels bcn_eval launches. */
typedef enum {
    BCN_KERNEL_MAC = 0,             /* integer-weight multiply-accumulate + feature add */
    BCN_KERNEL_SQUARE = 1,          /* NTT of (c0, c1), tensor square, inverse NTT of the three products */
    BCN_KERNEL_KEYSWITCH = 2,       /* ModUp + NTT + inner product with the evaluation key + inverse NTT */
    BCN_KERNEL_MODDOWN_RESCALE = 3, /* ModDown by P, add, rescale */
    BCN_KERNEL_COUNT = 4
} bcn_kernel_class;

/* With timing enabled, bcn_eval records a CUDA event pair around every kernel
 * it launches (on the evaluation's stream) and the algorithmic bytes that
 * launch must move (each input and output limb once).  Enabling resets the
 * totals.  bcn_profile_read waits for the recorded events and returns, for
 * one class, the summed device time in ms, the launch count and the bytes. */
bcn_status bcn_profile_enable(bcn_model *m, int enable);
bcn_status bcn_profile_read(bcn_model *m, int kernel_class, double *total_ms, long long *launches, double *bytes);

/* ------------------------------------------- single operations (device) */
/* Each runs the evaluator's kernels for one step, on device buffers in the
 * interchange layout, for op-level checks and benchmarks. */

/* In-place negacyclic NTT of n_poly polynomials at `level` ([n_poly][level][N]):
 * forward gives the evaluator's internal (bit-reversed) order, inverse undoes it. */
bcn_status bcn_op_ntt(const bcn_ctx *ctx, uint32_t *data_dev, int n_poly, int level, int inverse, void *cuda_stream);
/* out[o] = sum_t w[o][t] * in[idx[o][t]] (+ (pt[o], 0)); idx < 0 = zero tap.
 * idx_dev [n_out][K] int32, w_dev [n_out][K] int8, pt_dev may be NULL. */
bcn_status bcn_op_mac(const bcn_ctx *ctx, int level, int n_in, int n_out, int K, const int32_t *idx_dev,
                      const int8_t *w_dev, const uint32_t *in_dev, const uint32_t *pt_dev, uint32_t *out_dev,
                      void *cuda_stream);
/* workspace for bcn_op_square_relin_rescale on n_ct ciphertexts at level */
bcn_status bcn_op_workspace_bytes(const bcn_ctx *ctx, int level, int n_ct, size_t *bytes);
/* tensor square: [n_ct][2][level][N] -> [n_ct][3][level][N] (coefficient form) */
bcn_status bcn_op_tensor_square(const bcn_ctx *ctx, int level, const uint32_t *in_dev, int n_ct, uint32_t *out_dev,
                                void *workspace_dev, size_t workspace_bytes, void *cuda_stream);
/* square activation: tensor square, relinearise, rescale:
 * [n_ct][2][level][N] -> [n_ct][2][level-1][N] */
bcn_status bcn_op_square_relin_rescale(const bcn_ctx *ctx, int level, const uint32_t *evk_eval_dev,
                                       const uint32_t *in_dev, int n_ct, uint32_t *out_dev, void *workspace_dev,
                                       size_t workspace_bytes, void *cuda_stream);
/* The square activation above without any allocation.  The paper has no
 * counterpart: this is a service for callers that may not allocate device
 * memory themselves (a serving process whose device memory is budgeted by an
 * admission controller, code under a framework allocator that forbids
 * allocations behind its back; cudaMalloc/cudaFree would also synchronise the
 * device mid-request).  The caller passes only inputs and outputs; the key-
 * switching intermediates live in one file-scope device array of 32 MiB that
 * every GPU loading the library holds until exit.  Ciphertexts are processed in
 * chunks that fit it; BCN_E_BUDGET if a single ciphertext at `level` does not.
 * The first call on a device looks the array's device address up (once per
 * device, with that device current); make that first call before any stream
 * capture.  The address is kept for the life of the process: a device reset
 * (cudaDeviceReset, or a reset of the primary context) unloads the module and
 * leaves it stale, so do not call this entry point after one.  Every call shares the array, so calls that overlap on the GPU (other
 * streams, other threads) race; nothing in it has to start at zero (each word is
 * written before it is read within a call).  Same layouts, results and errors
 * as bcn_op_square_relin_rescale; allocates nothing (no cudaMalloc/cudaFree, no
 * allocating library routine). */
bcn_status bcn_op_square_relin_rescale_noalloc(const bcn_ctx *ctx, int level, const uint32_t *evk_eval_dev,
                                               const uint32_t *in_dev, int n_ct, uint32_t *out_dev,
                                               void *cuda_stream);
/* rescale alone: [n_ct][2][level][N] -> [n_ct][2][level-1][N] */
/* Rotation of the slots (App. A: D(Rot(c, k)) is D(c) rotated by k slots; App.
 * D builds its packed convolutions and dense layers from rotations).  With slot k
 * at the root zeta^{5^k}, a rotation by r slots (slot k + r moves to slot k,
 * cyclically over the N/2 slots) is the automorphism sigma_g: a(X) -> a(X^g),
 * g = 5^r mod 2N, followed by key switching from sigma_g(s) back to s:
 *     Rot(c0, c1) = (sigma_g(c0) + k0, k1),  (k0, k1) = KeySwitch_gk(sigma_g(c1)).
 * bcn_galois_elt: g for `steps` (taken mod N/2).  bcn_galois_keygen (client,
 * host): gk_j = (-a_j s + e_j + P g_j sigma_g(s), a_j) in the layout of the
 * relinearisation key (bcn_evk_words words; streams: tag 6 a (index
 * (g << 20) + j*256 + limb), tag 7 e (index (g << 20) + j)); make it device-ready
 * with bcn_evk_prepare.  bcn_op_rotate: n_ct ciphertexts in/out
 * [n_ct][2][level][N] (device, coefficient form; no level is used), workspace
 * bcn_op_workspace_bytes(level, n_ct); in and out must not overlap. */
uint32_t bcn_galois_elt(const bcn_ctx *ctx, int steps);
bcn_status bcn_galois_keygen(const bcn_ctx *ctx, const int8_t *sk, int steps, uint64_t seed, uint32_t *gk_out);
bcn_status bcn_op_rotate(const bcn_ctx *ctx, int level, const uint32_t *gk_eval_dev, int steps, const uint32_t *in_dev,
                         int n_ct, uint32_t *out_dev, void *workspace_dev, size_t workspace_bytes, void *cuda_stream);
/* Many rotations of each ciphertext with one shared ModUp (App. D builds its
 * packed convolutions and dense layers from many rotations of the same
 * ciphertext).  The automorphism commutes with ModUp (it permutes and negates
 * coefficients; the centred lift is odd and the basis conversion linear), so
 * the digit decomposition of c1, in the NTT domain, is computed once per
 * ciphertext and each rotation only permutes it, multiplies by its Galois key,
 * transforms back and runs ModDown: results equal bcn_op_rotate's, bit for bit.
 * steps[n_rot] (any sign, taken mod N/2; 0 copies the input), gk_evals[n_rot]
 * a host array of device pointers to prepared Galois keys (bcn_evk_prepare of
 * bcn_galois_keygen; ignored for steps = 0 mod N/2).  in [n_ct][2][level][N],
 * out [n_ct][n_rot][2][level][N], device, coefficient form; workspace of
 * bcn_op_rotate_many_workspace_bytes(level, n_ct).  BCN_E_INVAL on a bad
 * level, a missing key, unaligned or overlapping buffers; BCN_E_BUDGET if the
 * workspace is too small. */
bcn_status bcn_op_rotate_many_workspace_bytes(const bcn_ctx *ctx, int level, int n_ct, size_t *bytes);
bcn_status bcn_op_rotate_many(const bcn_ctx *ctx, int level, const uint32_t *const *gk_evals, const int *steps,
                              int n_rot, const uint32_t *in_dev, int n_ct, uint32_t *out_dev, void *workspace_dev,
                              size_t workspace_bytes, void *cuda_stream);
/* Homomorphic fully connected layer by the diagonal method (App. D): y = W x
 * for every image block of the slots, computed as
 *     Rescale_{q_{level-1}}( sum_r u_r * Rot(x, r) )
 * over the rotations r = i - j that W needs, u_r the r-th diagonal of W laid
 * out in the slots (u_r[b B + j] = W[j][j + r]) and encoded at the scale
 * q_{level-1}, so that the rescale keeps the ciphertext's scale.  The rotations
 * share one ModUp (bcn_op_rotate_many); each rotated copy is transformed, the
 * products are summed in the NTT domain and transformed back once.
 * steps[n_rot], gk_evals[n_rot] as for bcn_op_rotate_many; diag_ntt
 * [n_rot][level][N] the encoded diagonals of the same order in the NTT domain
 * (bcn_op_ntt forward of the coefficient-form encodings); in [n_ct][2][level][N]
 * -> out [n_ct][2][level-1][N], coefficient form, device; workspace of
 * bcn_op_fc_diag_workspace_bytes(level, n_rot).  level >= 2. */
bcn_status bcn_op_fc_diag_workspace_bytes(const bcn_ctx *ctx, int level, int n_rot, size_t *bytes);
bcn_status bcn_op_fc_diag(const bcn_ctx *ctx, int level, const uint32_t *const *gk_evals, const int *steps, int n_rot,
                          const uint32_t *diag_ntt_dev, const uint32_t *in_dev, int n_ct, uint32_t *out_dev,
                          void *workspace_dev, size_t workspace_bytes, void *cuda_stream);
/* The dense layer of App. D over c input ciphertexts per group (BHW packing
 * holds one channel per ciphertext, so a dense layer after a convolution reads
 * c of them), with the layer's plaintext feature added (Sec. 3.2's
 * unidirectional add, App. A Add(c, u)):
 *     y = Rescale_{q_{level-1}}( sum_k sum_r u_{k,r} * Rot(x_k, r) ) + f.
 * The inputs' slots may sit anywhere in each image block (a strided
 * convolution leaves its outputs at every s-th position): u_{k,r} carries
 * W[j][p] in output j's slot for every input position p of channel k at slot
 * distance r from it, which also drops the slots a strided convolution does
 * not keep.  Every input ciphertext's rotations share one ModUp; all products
 * are summed in the NTT domain, transformed back and rescaled once.
 * steps[n_rot], gk_evals[n_rot] as for bcn_op_rotate_many (the same rotations
 * for every input); diag_ntt [n_in][n_rot][level][N] (NTT domain, encoded at
 * scale q_{level-1}); in [n_groups][n_in][2][level][N] -> out
 * [n_groups][2][level-1][N], coefficient form, device; pt NULL or
 * [n_groups][level-1][N] (coefficient form) added to each output's first
 * polynomial.  Workspace bcn_op_fc_diag_workspace_bytes(level, n_rot).
 * BCN_E_INVAL on a bad level or count, an unaligned buffer or in/out overlap;
 * BCN_E_BUDGET if the workspace is too small. */
bcn_status bcn_op_fc_diag_sum(const bcn_ctx *ctx, int level, const uint32_t *const *gk_evals, const int *steps,
                              int n_rot, const uint32_t *diag_ntt_dev, const uint32_t *in_dev, int n_in, int n_groups,
                              const uint32_t *pt_dev, uint32_t *out_dev, void *workspace_dev, size_t workspace_bytes,
                              void *cuda_stream);
/* Ciphertext-plaintext product then rescale (App. A Mult(c, u) with an encoded
 * u -- the masks of App. D's packed layers): (c0 u, c1 u) in R_{Q_level}, then
 * the rescale by q_{level-1}.  Encode u at scale q_{level-1} to keep the
 * ciphertext's scale.  in [n_ct][2][level][N], pt [level][N] (coefficient form),
 * out [n_ct][2][level-1][N], device; workspace bcn_op_workspace_bytes(level,
 * n_ct).  level >= 2. */
bcn_status bcn_op_mul_plain_rescale(const bcn_ctx *ctx, int level, const uint32_t *in_dev, int n_ct,
                                    const uint32_t *pt_dev, uint32_t *out_dev, void *workspace_dev,
                                    size_t workspace_bytes, void *cuda_stream);
bcn_status bcn_op_rescale(const bcn_ctx *ctx, int level, const uint32_t *in_dev, int n_ct, uint32_t *out_dev,
                          void *cuda_stream);

/* ------------------------------------------- measurement (device) */
/* Integer-issue microbenchmark: the ceiling the NTT-based kernels' arithmetic
 * is reported against (the paper has no counterpart; it measures nothing on a
 * GPU).  One launch on the current device and `cuda_stream` (asynchronous):
 * every thread of a full-occupancy grid of 256-thread blocks runs `iters`
 * rounds of one sequence on 16 register-resident words.  kind:
 *   0  32-bit multiply-add, low half (16 a round)
 *   1  32-bit multiply-add, high half with an addend (16 a round)
 *   2  modular addition: add, then min(y, y - q) (16 a round)
 *   3  lazy forward NTT butterflies of the evaluator's NTT core (32 a round)
 *   4  lazy inverse NTT butterflies of the evaluator's NTT core (32 a round)
 *   5  lazy Montgomery multiply-add of the key switch's running sums (16 a round)
 *   6  Shoup multiply-add by a constant, as in the basis conversions (16 a round)
 *   7  signed 32 x 32 -> 64-bit multiply-add, the CUDA-core MAC's step (16 a round)
 *   8  4-way int8 x uint8 dot product with 32-bit accumulation, dp4a (16 a round)
 * units_out: the operations the launch performs (instructions for kinds 0-1 and
 * 7-8, modular additions, butterflies or multiply-adds for 2-6), to divide by the
 * launch's time.  sink_dev: device memory of at least bcn_int_peak_grid's
 * block count in uint32 words (written only if a result equals an improbable
 * value; it keeps the work from being optimised away).  BCN_E_INVAL for a kind
 * outside 0..8, iters < 1 or a null pointer; BCN_E_BUDGET if the sink is too
 * small. */
bcn_status bcn_int_peak_grid(int kind, int *blocks);
bcn_status bcn_int_peak_launch(int kind, int iters, uint32_t *sink_dev, size_t sink_words, void *cuda_stream,
                               double *units_out);

#ifdef __cplusplus
}
#endif
#endif /* BCN_H */
