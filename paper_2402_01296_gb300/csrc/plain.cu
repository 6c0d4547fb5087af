// Plaintext branch (fp32, device) with its unidirectional-connection taps.
//
// The plaintext branch runs on the whole image: the sensitive segment is set
// to zero and the insensitive segment carries the client's perturbation
// (Sec. 3.1 of the paper).  Each tap resizes a feature map to the ciphertext
// branch's size by a centre crop and mixes channels with CRot,
// z^i = sum_j W^{i,j} y^j (Sec. 3.2), applies a fully connected map (with an
// optional bias), or computes the plaintext half of the two-layer feature
// integration (Sec. 3.3): W_2 sigma(W'_1 x_p + b'_1) + b_2.
// Feature rows are written as [n_feat][B] so each row is one slot vector.
#include <algorithm>
#include <cuda_runtime.h>

#include "device_api.h"

struct bcn_plain_model {
    bcn_ctx *ctx;
    int H, W, C, seg[4];
    struct Stage {
        bcn_plain_stage s;
        int cin, hin, win, cout, hout, wout;  // map shape before / after
        float *d_w = nullptr;
        int feat_row = 0, n_feat = 0;  // taps
    };
    std::vector<Stage> stages;
    size_t max_act = 0;  // floats per image of the largest activation
    int n_feat = 0;
};

namespace bcn {

__global__ void k_perturb(const uint8_t *__restrict__ img, const float *__restrict__ noise, float *__restrict__ x,
                          int B, int H, int W, int C, int y0, int x0, int h, int w) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)B * C * H * W;
    if (i >= total) return;
    const int xx = (int)(i % W), yy = (int)(i / W % H), c = (int)(i / ((size_t)W * H) % C);
    const size_t b = i / ((size_t)W * H * C);
    const size_t src = ((b * H + yy) * W + xx) * C + c;
    const bool inside = yy >= y0 && yy < y0 + h && xx >= x0 && xx < x0 + w;
    x[i] = inside ? 0.0f : (float)img[src] / 255.0f + noise[src];
}

__global__ void k_conv(const float *__restrict__ in, const float *__restrict__ wt, float *__restrict__ out, int B,
                       int cin, int H, int W, int cout, int k, int stride, int pad, int Ho, int Wo, int relu) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)B * cout * Ho * Wo;
    if (i >= total) return;
    const int ox = (int)(i % Wo), oy = (int)(i / Wo % Ho), co = (int)(i / ((size_t)Wo * Ho) % cout);
    const size_t b = i / ((size_t)Wo * Ho * cout);
    float acc = 0.0f;
    for (int ci = 0; ci < cin; ci++)
        for (int ky = 0; ky < k; ky++) {
            const int iy = oy * stride - pad + ky;
            if (iy < 0 || iy >= H) continue;
            for (int kx = 0; kx < k; kx++) {
                const int ix = ox * stride - pad + kx;
                if (ix < 0 || ix >= W) continue;
                acc = fmaf(__ldg(wt + (((size_t)co * cin + ci) * k + ky) * k + kx),
                           in[((b * cin + ci) * H + iy) * W + ix], acc);
            }
        }
    out[i] = relu ? fmaxf(acc, 0.0f) : acc;
}

__global__ void k_avgpool2(const float *__restrict__ in, float *__restrict__ out, int B, int C, int H, int W) {
    const int Ho = H / 2, Wo = W / 2;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)B * C * Ho * Wo;
    if (i >= total) return;
    const int ox = (int)(i % Wo), oy = (int)(i / Wo % Ho);
    const size_t bc = i / ((size_t)Wo * Ho);
    const float *p = in + (bc * H + 2 * oy) * W + 2 * ox;
    out[i] = 0.25f * (p[0] + p[1] + p[W] + p[W + 1]);
}

// feats[row0 + (i*hc + y)*wc + x][b] = sum_j W[i][j] * act[b][j][oy + y][ox + x]
__global__ void k_crop_crot(const float *__restrict__ act, const float *__restrict__ wt, float *__restrict__ feats,
                            int B, int C, int H, int W, int hc, int wc, int ch_c, int row0) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)ch_c * hc * wc * B;
    if (i >= total) return;
    const int b = (int)(i % B);
    const size_t f = i / B;
    const int x = (int)(f % wc), y = (int)(f / wc % hc), ch = (int)(f / ((size_t)wc * hc));
    const int oy = (H - hc) / 2, ox = (W - wc) / 2;
    float acc = 0.0f;
    for (int j = 0; j < C; j++)
        acc = fmaf(__ldg(wt + (size_t)ch * C + j), act[(((size_t)b * C + j) * H + oy + y) * W + ox + x], acc);
    feats[((size_t)row0 + f) * B + b] = acc;
}

// feats[row0 + o][b] = sum_k W[o][k] * act[b][k] (+ bias[o])
__global__ void k_fc(const float *__restrict__ act, const float *__restrict__ wt, const float *__restrict__ bias,
                     float *__restrict__ feats, int B, int K, int n_out, int row0) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)n_out * B) return;
    const int b = (int)(i % B), o = (int)(i / B);
    float acc = bias != nullptr ? __ldg(bias + o) : 0.0f;
    for (int k = 0; k < K; k++) acc = fmaf(__ldg(wt + (size_t)o * K + k), act[(size_t)b * K + k], acc);
    feats[((size_t)row0 + o) * B + b] = acc;
}

// hidden[b][j] = (sum_k W[j][k] * act[b][k] + bias[j])^2: the plaintext neurons
// of the first integration layer, square activation
__global__ void k_fc_square(const float *__restrict__ act, const float *__restrict__ wt,
                            const float *__restrict__ bias, float *__restrict__ hidden, int B, int K, int n_hidden) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)n_hidden * B) return;
    const int j = (int)(i % n_hidden);
    const size_t b = i / n_hidden;
    float acc = __ldg(bias + j);
    for (int k = 0; k < K; k++) acc = fmaf(__ldg(wt + (size_t)j * K + k), act[b * K + k], acc);
    hidden[b * n_hidden + j] = acc * acc;
}

static unsigned blocks_for(size_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace bcn

using namespace bcn;

extern "C" {

bcn_status bcn_plain_model_create(bcn_ctx *c, const bcn_plain_stage *st, int n, int H, int W, int C,
                                  const int seg[4], bcn_plain_model **out) {
    if (!c || !st || !seg || !out || n < 1 || H < 1 || W < 1 || C < 1)
        return fail(BCN_E_INVAL, "bcn_plain_model_create: bad argument");
    if (c->device < 0) return fail(BCN_E_INVAL, "bcn_plain_model_create: host-only ctx");
    *out = nullptr;
    if (seg[0] < 0 || seg[1] < 0 || seg[2] < 0 || seg[3] < 0 || seg[0] + seg[2] > H || seg[1] + seg[3] > W)
        return fail(BCN_E_INVAL, "bcn_plain_model_create: segment outside the image");
    bcn_plain_model *m = new bcn_plain_model();
    m->ctx = c;
    m->H = H; m->W = W; m->C = C;
    std::copy(seg, seg + 4, m->seg);
    int ch = C, h = H, w = W;
    m->max_act = (size_t)C * H * W;
    auto bad = [&](const std::string &msg) {
        bcn_plain_model_destroy(m);
        return fail(BCN_E_INVAL, msg);
    };
    for (int i = 0; i < n; i++) {
        bcn_plain_model::Stage s;
        s.s = st[i];
        s.cin = ch; s.hin = h; s.win = w;
        size_t nw = 0;
        switch (st[i].op) {
        case BCN_PLAIN_CONV: {
            const bcn_plain_stage &x = st[i];
            if (x.cin != ch || x.cout < 1 || x.k < 1 || x.stride < 1 || x.pad < 0 || h + 2 * x.pad < x.k ||
                w + 2 * x.pad < x.k)
                return bad("plain conv stage " + std::to_string(i) + ": bad geometry");
            h = (h + 2 * x.pad - x.k) / x.stride + 1;
            w = (w + 2 * x.pad - x.k) / x.stride + 1;
            ch = x.cout;
            nw = (size_t)x.cout * x.cin * x.k * x.k;
            break;
        }
        case BCN_PLAIN_AVGPOOL2:
            if (h < 2 || w < 2) return bad("avgpool on a map smaller than 2x2");
            h /= 2; w /= 2;
            break;
        case BCN_PLAIN_TAP_CROP_CROT:
            if (st[i].hc < 1 || st[i].wc < 1 || st[i].hc > h || st[i].wc > w || st[i].ch_c < 1)
                return bad("crop/CRot tap " + std::to_string(i) + ": bad size");
            s.feat_row = m->n_feat;
            s.n_feat = st[i].ch_c * st[i].hc * st[i].wc;
            m->n_feat += s.n_feat;
            nw = (size_t)st[i].ch_c * ch;
            break;
        case BCN_PLAIN_TAP_FC:
            if (st[i].n_out < 1) return bad("fc tap: bad size");
            s.feat_row = m->n_feat;
            s.n_feat = st[i].n_out;
            m->n_feat += s.n_feat;
            nw = (size_t)st[i].n_out * ch * h * w + (st[i].bias ? (size_t)st[i].n_out : 0);
            break;
        case BCN_PLAIN_TAP_INTEGRATE:
            if (st[i].n_out < 1 || st[i].n_hidden < 1) return bad("integration tap: bad size");
            s.feat_row = m->n_feat;
            s.n_feat = st[i].n_out;
            m->n_feat += s.n_feat;
            nw = (size_t)st[i].n_hidden * ch * h * w + st[i].n_hidden + (size_t)st[i].n_out * st[i].n_hidden +
                 st[i].n_out;
            m->max_act = std::max(m->max_act, (size_t)st[i].n_hidden);  // the hidden layer's scratch
            break;
        default:
            return bad("unknown plain stage op");
        }
        s.cout = ch; s.hout = h; s.wout = w;
        m->max_act = std::max(m->max_act, (size_t)ch * h * w);
        if (nw) {
            if (!st[i].weights) return bad("plain stage " + std::to_string(i) + ": null weights");
            if (cudaMalloc(&s.d_w, nw * 4) != cudaSuccess) {
                m->stages.push_back(s);
                bcn_plain_model_destroy(m);
                return fail(BCN_E_NOMEM, "plain weights allocation failed");
            }
            m->stages.push_back(s);
            if (cudaMemcpy(s.d_w, st[i].weights, nw * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
                bcn_plain_model_destroy(m);
                return fail(BCN_E_CUDA, "plain weights upload failed");
            }
        } else {
            m->stages.push_back(s);
        }
    }
    *out = m;
    return BCN_OK;
}

bcn_status bcn_plain_model_destroy(bcn_plain_model *m) {
    if (!m) return BCN_OK;
    for (auto &s : m->stages) cudaFree(s.d_w);
    delete m;
    return BCN_OK;
}

bcn_status bcn_plain_feature_count(const bcn_plain_model *m, int *n) {
    if (!m || !n) return fail(BCN_E_INVAL, "bcn_plain_feature_count: null argument");
    *n = m->n_feat;
    return BCN_OK;
}

bcn_status bcn_plain_workspace_bytes(const bcn_plain_model *m, int B, size_t *bytes) {
    if (!m || !bytes || B < 1) return fail(BCN_E_INVAL, "bcn_plain_workspace_bytes: bad argument");
    *bytes = 2 * (((size_t)B * m->max_act * 4 + 255) / 256 * 256);
    return BCN_OK;
}

bcn_status bcn_plain_branch_forward(const bcn_plain_model *m, const uint8_t *img, const float *noise, int B,
                                    float *feats, void *ws, size_t ws_bytes, void *stream) {
    if (!m || !img || !noise || !feats || B < 1) return fail(BCN_E_INVAL, "bcn_plain_branch_forward: bad argument");
    size_t need = 0;
    bcn_plain_workspace_bytes(m, B, &need);
    if (!ws || ws_bytes < need) return fail(BCN_E_BUDGET, "bcn_plain_branch_forward: workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    float *buf[2] = {reinterpret_cast<float *>(ws), reinterpret_cast<float *>((char *)ws + need / 2)};
    int cur = 0;
    size_t tot = (size_t)B * m->C * m->H * m->W;
    k_perturb<<<blocks_for(tot), 256, 0, st>>>(img, noise, buf[0], B, m->H, m->W, m->C, m->seg[0], m->seg[1],
                                              m->seg[2], m->seg[3]);
    if (check_launch("k_perturb") != BCN_OK) return BCN_E_CUDA;
    for (const auto &s : m->stages) {
        const bcn_plain_stage &x = s.s;
        switch (x.op) {
        case BCN_PLAIN_CONV: {
            size_t n = (size_t)B * s.cout * s.hout * s.wout;
            k_conv<<<blocks_for(n), 256, 0, st>>>(buf[cur], s.d_w, buf[1 - cur], B, s.cin, s.hin, s.win, s.cout, x.k,
                                                  x.stride, x.pad, s.hout, s.wout, x.relu);
            cur = 1 - cur;
            break;
        }
        case BCN_PLAIN_AVGPOOL2: {
            size_t n = (size_t)B * s.cout * s.hout * s.wout;
            k_avgpool2<<<blocks_for(n), 256, 0, st>>>(buf[cur], buf[1 - cur], B, s.cin, s.hin, s.win);
            cur = 1 - cur;
            break;
        }
        case BCN_PLAIN_TAP_CROP_CROT: {
            size_t n = (size_t)s.n_feat * B;
            k_crop_crot<<<blocks_for(n), 256, 0, st>>>(buf[cur], s.d_w, feats, B, s.cin, s.hin, s.win, x.hc, x.wc,
                                                       x.ch_c, s.feat_row);
            break;
        }
        case BCN_PLAIN_TAP_FC: {
            const int K = s.cin * s.hin * s.win;
            size_t n = (size_t)s.n_feat * B;
            k_fc<<<blocks_for(n), 256, 0, st>>>(buf[cur], s.d_w, x.bias ? s.d_w + (size_t)x.n_out * K : nullptr,
                                                feats, B, K, x.n_out, s.feat_row);
            break;
        }
        case BCN_PLAIN_TAP_INTEGRATE: {
            const int K = s.cin * s.hin * s.win, nh = x.n_hidden;
            const float *w1 = s.d_w, *b1 = w1 + (size_t)nh * K, *w2 = b1 + nh, *b2 = w2 + (size_t)x.n_out * nh;
            float *hidden = buf[1 - cur];  // scratch; the trunk stays in buf[cur]
            k_fc_square<<<blocks_for((size_t)nh * B), 256, 0, st>>>(buf[cur], w1, b1, hidden, B, K, nh);
            if (check_launch("k_fc_square") != BCN_OK) return BCN_E_CUDA;
            k_fc<<<blocks_for((size_t)s.n_feat * B), 256, 0, st>>>(hidden, w2, b2, feats, B, nh, x.n_out,
                                                                    s.feat_row);
            break;
        }
        }
        if (check_launch("plain branch stage") != BCN_OK) return BCN_E_CUDA;
    }
    return BCN_OK;
}

}  // extern "C"
