// mlp_api.cu -- C ABI of the crater-surrogate MLP: parameters, forward pass, gradient and
// Adam training step on one caller-owned device buffer, plus the bare BF16 GEMM.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <new>
#include <string>
#include <vector>

#include "../../include/salec_mlp.h"
#include "mlp_internal.cuh"
#include "salec_trace.h"

using namespace salec::mlp;

namespace {

constexpr int kLayers = 5;
constexpr int kDims[kLayers + 1] = {SALEC_MLP_IN, 256, 256, 256, 256, SALEC_MLP_OUT};
constexpr int kHid = 256;
// BF16 row stride of the inputs and of W_1: 5 columns padded to 8 (16-byte rows, which the
// TMA-fed GEMM needs); the padding stays zero
constexpr int kInLd = 8;

// BF16 row stride of W_l
int w_ld(int l) { return l == 0 ? kInLd : kDims[l]; }
// BF16 row stride of W_l^T (n_in rows of n_out values, padded to 16-byte rows); layer 0
// needs none (no activation gradient below the first layer)
int wt_ld(int l) { return (kDims[l + 1] + 7) / 8 * 8; }
// rows of the transposed activation buffers: the layer's units, one row of ones (the bias
// gradients are the weight gradients of that row), padded
constexpr int kHidT = kHid + 16;
constexpr int kInT = 16;
long ld_t(int bmax) { return ((long)bmax + 7) / 8 * 8; }

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

long n_params()
{
    long n = 0;
    for (int l = 0; l < kLayers; ++l) n += (long)kDims[l + 1] * kDims[l] + kDims[l + 1];
    return n;
}

long n_weights_bf16()
{
    long n = 0;
    for (int l = 0; l < kLayers; ++l) n += (long)kDims[l + 1] * w_ld(l);
    return n;
}

long n_weights_bf16_t()
{
    long n = 0;
    for (int l = 1; l < kLayers; ++l) n += (long)kDims[l] * wt_ld(l);
    return n;
}

// The backward pass reads its operands K-major (K = the batch for the weight gradients, K =
// a layer's outputs for the activation gradients), so the TMA-fed GEMM serves it too: the
// forward epilogues also write the activations transposed (HT, XT), the backward epilogues
// the gradients transposed (GT), and the BF16 weights are kept transposed as well (wbfT).
struct Layout {
    size_t theta, m1, m2, grad, wmap, wbf, wmapT, wbfT, X, XT, Z[4], H[4], HT[4], Y, G[2], GT[2], part, loss, err,
        ts, total;
    Layout(int bmax)
    {
        const long P = n_params(), W = n_weights_bf16(), WT = n_weights_bf16_t(), ldT = ld_t(bmax);
        size_t o = 0;
        auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes); return r; };
        theta = take(P * 4); m1 = take(P * 4); m2 = take(P * 4); grad = take(P * 4);
        wmap = take(P * 4);
        wbf = take(W * 2);
        wmapT = take(P * 4);
        wbfT = take(WT * 2);
        X = take((size_t)bmax * kInLd * 2);
        XT = take((size_t)kInT * ldT * 2);
        for (int l = 0; l < 4; ++l) Z[l] = take((size_t)bmax * kHid * 4);
        for (int l = 0; l < 4; ++l) H[l] = take((size_t)bmax * kHid * 2);
        for (int l = 0; l < 4; ++l) HT[l] = take((size_t)kHidT * ldT * 2);
        Y = take((size_t)bmax * SALEC_MLP_OUT * 4);
        for (int l = 0; l < 2; ++l) G[l] = take((size_t)bmax * kHid * 2);
        for (int l = 0; l < 2; ++l) GT[l] = take((size_t)kHid * ldT * 2);
        part = take((size_t)kMaxSplit * kHid * (kHid + 1) * 4);   // split-K partials of a weight gradient
        loss = take(8);
        err = take(4);
        ts = take(sizeof(TrainState));
        total = o;
    }
};

}  // namespace

struct salec_mlp {
    int bmax = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    float *theta = nullptr, *m1 = nullptr, *m2 = nullptr, *grad = nullptr;
    int* wmap = nullptr;
    __nv_bfloat16* wbf = nullptr;
    int* wmapT = nullptr;
    __nv_bfloat16* wbfT = nullptr;
    __nv_bfloat16* X = nullptr;
    __nv_bfloat16* XT = nullptr;
    float* Z[4] = {};
    __nv_bfloat16* H[4] = {};
    __nv_bfloat16* HT[4] = {};
    float* Y = nullptr;
    __nv_bfloat16* G[2] = {};
    __nv_bfloat16* GT[2] = {};
    long ldT = 0;                         // row stride of the transposed buffers (batch_max, padded)
    float* part = nullptr;
    double* loss = nullptr;
    int* errflag = nullptr;
    TrainState* ts = nullptr;
    long steps = 0;                       // Adam steps taken
    // salec_mlp_train: a CUDA graph of kTrainChunk steps, for the arguments it was captured with
    cudaGraphExec_t tgraph = nullptr;
    const float* tg_t = nullptr;
    const float* tg_lr = nullptr;
    int tg_batch = 0;
    float tg_beta1 = 0.0f, tg_beta2 = 0.0f, tg_eps = 0.0f;
    bool tg_ok = true;                    // false after a capture failed: plain launches
    ~salec_mlp()
    {
        if (tgraph) cudaGraphExecDestroy(tgraph);
    }
    long woff[kLayers], boff[kLayers];    // offsets of W_l and b_l in theta
    long wbf_off[kLayers];                // offset of W_l in the BF16 weight block
    long wbfT_off[kLayers];               // offset of W_l^T in the transposed block (l >= 1)
};

namespace {

salec_status fail(salec_mlp* n, salec_status st, const std::string& msg)
{
    if (n) n->err = msg;
    return st;
}

salec_status cuda_fail(salec_mlp* n, cudaError_t e, const char* where)
{
    return fail(n, SALEC_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define MLP_CUDA(n, call, where)                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail((n), e_, (where)); \
    } while (0)

GemmArgs gemm0(int M, int N, int K, int* err)
{
    GemmArgs g = {};
    g.M = M; g.N = N; g.K = K;
    g.err = err;
    return g;
}

// Forward layer l on X (already BF16): Z_l, H_l (and H_l^T) for the hidden layers; the
// output layer with the plain store into y, or (with the targets t) the fused loss gradient.
// The pre-activations and the transposed copies are kept only for a backward pass.
GemmArgs fwd_gemm(salec_mlp* n, int l, int B, float* y, long ldy, const float* t, bool with_loss)
{
    const bool keep_z = with_loss;
    const int ni = kDims[l], no = kDims[l + 1];
    GemmArgs g = gemm0(B, no, ni, n->errflag);
    g.A = l == 0 ? n->X : n->H[l - 1]; g.a_sm = l == 0 ? kInLd : kHid; g.a_sk = 1;
    g.B = n->wbf + n->wbf_off[l]; g.b_sn = w_ld(l); g.b_sk = 1;
    g.bias = n->theta + n->boff[l];
    if (l + 1 < kLayers) {
        g.epi = kEpiBiasGelu;
        g.C = keep_z ? n->Z[l] : nullptr; g.ldc = kHid;
        g.Hout = n->H[l]; g.ldh = kHid;
        if (keep_z) { g.HoutT = n->HT[l]; g.ldhT = n->ldT; }
    } else if (with_loss) {
        g.epi = kEpiOutLoss;
        g.C = y; g.ldc = ldy;
        g.Tin = t; g.ldt = SALEC_MLP_OUT;
        g.Hout = n->G[0]; g.ldh = kHid;
        g.HoutT = n->GT[0]; g.ldhT = n->ldT;
        g.grad_scale = 2.0f / ((float)B * (float)SALEC_MLP_OUT);
        g.loss = n->loss;
    } else {
        g.epi = kEpiStore;
        g.C = y; g.ldc = ldy;
    }
    return g;
}

// Backward, layer l, from G[cur] = dL/dZ_l (BF16, GT[cur] its transpose).
// dW_l[o][i] = sum_b G[b][o] Hprev[b][i] and db_l[o] = sum_b G[b][o], as one product of
// G^T (no x B) with [Hprev | 1]^T ((ni + 1) x B): the row of ones after the transposed
// activations gives the bias gradient in the last column.
GemmArgs dw_gemm(salec_mlp* n, int l, int B, int cur, float* grad)
{
    const int ni = kDims[l], no = kDims[l + 1];
    GemmArgs g = gemm0(no, ni + 1, B, n->errflag);
    g.A = n->GT[cur]; g.a_sm = n->ldT; g.a_sk = 1;
    g.B = l > 0 ? n->HT[l - 1] : n->XT; g.b_sn = n->ldT; g.b_sk = 1;
    g.epi = kEpiStore;
    g.C = grad + n->woff[l]; g.ldc = ni;
    g.Cb = grad + n->boff[l];
    g.part = n->part;
    return g;
}

// dL/dZ_{l-1}[b][i] = (sum_o G[b][o] W_l[o][i]) gelu'(Z_{l-1}[b][i]) into G[cur ^ 1] and its
// transpose, W_l^T K-major (l >= 1).
GemmArgs dh_gemm(salec_mlp* n, int l, int B, int cur)
{
    const int ni = kDims[l], no = kDims[l + 1];
    GemmArgs g = gemm0(B, ni, no, n->errflag);
    g.A = n->G[cur]; g.a_sm = kHid; g.a_sk = 1;
    g.B = n->wbfT + n->wbfT_off[l]; g.b_sn = wt_ld(l); g.b_sk = 1;
    g.epi = kEpiGeluBwd;
    g.Zin = n->Z[l - 1]; g.ldz = kHid;
    g.Hout = n->G[cur ^ 1]; g.ldh = kHid;
    g.HoutT = n->GT[cur ^ 1]; g.ldhT = n->ldT;
    return g;
}

salec_status forward_impl(salec_mlp* n, int B, float* y, long ldy, const float* t, bool with_loss)
{
    for (int l = 0; l < kLayers; ++l)
        MLP_CUDA(n, launch_gemm(fwd_gemm(n, l, B, y, ldy, t, with_loss), n->stream), "mlp forward gemm");
    return SALEC_OK;
}

// backward pass from G[0] = dL/dY: weight and bias gradients into grad.  Every operand is
// read K-major, so every GEMM is TMA-fed.
salec_status backward_impl(salec_mlp* n, int B, float* grad)
{
    int cur = 0;
    for (int l = kLayers - 1; l >= 0; --l) {
        MLP_CUDA(n, launch_gemm(dw_gemm(n, l, B, cur, grad), n->stream), "mlp weight-gradient gemm");
        if (l == 0) break;
        MLP_CUDA(n, launch_gemm(dh_gemm(n, l, B, cur), n->stream), "mlp activation-gradient gemm");
        cur ^= 1;
    }
    return SALEC_OK;
}

salec_status check_batch(salec_mlp* n, int B)
{
    if (!n) return SALEC_EINVAL;
    if (B < 1 || B > n->bmax) return fail(n, SALEC_EINVAL, "batch outside 1..batch_max");
    return SALEC_OK;
}

constexpr int kTrainChunk = 25;

// One step of a multi-step call: its learning rate and bias corrections from the device
// state, then the gradient and the Adam update (the inputs are already in X).
salec_status train_one(salec_mlp* n, int B, const float* t_dev, const float* lr_dev, float beta1, float beta2,
                       float eps)
{
    MLP_CUDA(n, launch_train_begin(n->ts, lr_dev, beta1, beta2, n->loss, n->stream), "mlp train step");
    salec_status st = forward_impl(n, B, n->Y, SALEC_MLP_OUT, t_dev, true);
    if (st != SALEC_OK) return st;
    st = backward_impl(n, B, n->grad);
    if (st != SALEC_OK) return st;
    AdamArgs a;
    a.lr = 0.0f; a.c1 = 0.0f; a.c2 = 0.0f;
    a.beta1 = beta1; a.beta2 = beta2; a.eps = eps; a.ts = n->ts;
    MLP_CUDA(n, launch_adam(n->theta, n->m1, n->m2, n->grad, n_params(), a, n->wmap, n->wbf, n->stream, n->wmapT, n->wbfT), "mlp adam");
    return SALEC_OK;
}

// Capture kTrainChunk steps on a private stream (the graph can then be launched into any
// stream); false, with no error left pending, when capture is not possible.
bool capture_train(salec_mlp* n, int B, const float* t_dev, const float* lr_dev, float beta1, float beta2, float eps)
{
    if (n->tgraph) {
        cudaGraphExecDestroy(n->tgraph);
        n->tgraph = nullptr;
    }
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    cudaStream_t keep = n->stream;
    n->stream = cs;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    salec_status st = SALEC_OK;
    for (int k = 0; k < kTrainChunk && e == cudaSuccess && st == SALEC_OK; ++k)
        st = train_one(n, B, t_dev, lr_dev, beta1, beta2, eps);
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    n->stream = keep;
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess && st == SALEC_OK) e = cudaGraphInstantiate(&n->tgraph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess || st != SALEC_OK) {
        (void)cudaGetLastError();
        n->tgraph = nullptr;
        return false;
    }
    n->tg_t = t_dev; n->tg_lr = lr_dev; n->tg_batch = B;
    n->tg_beta1 = beta1; n->tg_beta2 = beta2; n->tg_eps = eps;
    return true;
}

}  // namespace

// Ensemble members trained together (salec_mlp_train_group): the member contexts and the
// CUDA graph of kTrainChunk steps captured for the arguments of the last call.
struct salec_mlp_group {
    std::vector<salec_mlp*> nets;
    cudaStream_t stream = nullptr;
    std::string err;
    cudaGraphExec_t tgraph = nullptr;
    const float* tg_t = nullptr;
    const float* tg_lr = nullptr;
    int tg_batch = 0;
    float tg_beta1 = 0.0f, tg_beta2 = 0.0f, tg_eps = 0.0f;
    bool tg_ok = true;
    ~salec_mlp_group()
    {
        if (tgraph) cudaGraphExecDestroy(tgraph);
    }
};

namespace {

salec_status gfail(salec_mlp_group* g, salec_status st, const std::string& msg)
{
    if (g) g->err = msg;
    return st;
}

#define GROUP_CUDA(g, call, where)                                                                                \
    do {                                                                                                          \
        cudaError_t e_ = (call);                                                                                  \
        if (e_ != cudaSuccess) return gfail((g), SALEC_ECUDA, std::string(where) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// One training step of every member: the step's start, the forward pass, the backward pass
// and Adam, each GEMM one launch for all members (the inputs are already in each X, X^T).
salec_status group_train_one(salec_mlp_group* G, cudaStream_t s, int B, const float* t_dev, const float* lr_dev,
                             float beta1, float beta2, float eps)
{
    const int n = (int)G->nets.size();
    GemmArgs args[kMaxGroup];
    BeginGroup bg;
    for (int k = 0; k < n; ++k) { bg.ts[k] = G->nets[k]->ts; bg.loss[k] = G->nets[k]->loss; }
    GROUP_CUDA(G, launch_train_begin_group(bg, n, lr_dev, beta1, beta2, s), "group train step");
    for (int l = 0; l < kLayers; ++l) {
        for (int k = 0; k < n; ++k) args[k] = fwd_gemm(G->nets[k], l, B, G->nets[k]->Y, SALEC_MLP_OUT, t_dev, true);
        GROUP_CUDA(G, launch_gemm_group(args, n, s), "group forward gemm");
    }
    int cur = 0;
    for (int l = kLayers - 1; l >= 0; --l) {
        for (int k = 0; k < n; ++k) args[k] = dw_gemm(G->nets[k], l, B, cur, G->nets[k]->grad);
        GROUP_CUDA(G, launch_gemm_group(args, n, s), "group weight-gradient gemm");
        if (l == 0) break;
        for (int k = 0; k < n; ++k) args[k] = dh_gemm(G->nets[k], l, B, cur);
        GROUP_CUDA(G, launch_gemm_group(args, n, s), "group activation-gradient gemm");
        cur ^= 1;
    }
    AdamGroup ag;
    for (int k = 0; k < n; ++k) {
        salec_mlp* m = G->nets[k];
        ag.theta[k] = m->theta; ag.m1[k] = m->m1; ag.m2[k] = m->m2; ag.grad[k] = m->grad;
        ag.wbf[k] = m->wbf; ag.wbfT[k] = m->wbfT; ag.ts[k] = m->ts;
    }
    GROUP_CUDA(G, launch_adam_group(ag, n, n_params(), beta1, beta2, eps, G->nets[0]->wmap, G->nets[0]->wmapT, s),
               "group adam");
    return SALEC_OK;
}

// Capture kTrainChunk group steps on a private stream; false, with no error left pending,
// when capture is not possible.
bool capture_group(salec_mlp_group* G, int B, const float* t_dev, const float* lr_dev, float beta1, float beta2, float eps)
{
    if (G->tgraph) {
        cudaGraphExecDestroy(G->tgraph);
        G->tgraph = nullptr;
    }
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    cudaGraph_t gr = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    salec_status st = SALEC_OK;
    for (int k = 0; k < kTrainChunk && e == cudaSuccess && st == SALEC_OK; ++k)
        st = group_train_one(G, cs, B, t_dev, lr_dev, beta1, beta2, eps);
    const cudaError_t e2 = cudaStreamEndCapture(cs, &gr);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess && st == SALEC_OK) e = cudaGraphInstantiate(&G->tgraph, gr, 0);
    if (gr) cudaGraphDestroy(gr);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess || st != SALEC_OK) {
        (void)cudaGetLastError();
        G->tgraph = nullptr;
        return false;
    }
    G->tg_t = t_dev; G->tg_lr = lr_dev; G->tg_batch = B;
    G->tg_beta1 = beta1; G->tg_beta2 = beta2; G->tg_eps = eps;
    return true;
}

}  // namespace

extern "C" {

int salec_mlp_n_params(void) { return (int)n_params(); }

salec_status salec_mlp_bytes(int batch_max, size_t* bytes)
{
    if (!bytes || batch_max < 1) return SALEC_EINVAL;
    *bytes = Layout(batch_max).total;
    return SALEC_OK;
}

salec_status salec_mlp_create(int batch_max, void* dev_buf, size_t bytes, void* stream, salec_mlp** out)
{
    if (!out || !dev_buf || batch_max < 1) return SALEC_EINVAL;
    *out = nullptr;
    Layout L(batch_max);
    if (bytes < L.total) return SALEC_ENOMEM;
    if (reinterpret_cast<uintptr_t>(dev_buf) & 255) return SALEC_EINVAL;
    salec_mlp* n = new (std::nothrow) salec_mlp();
    if (!n) return SALEC_ENOMEM;
    unsigned char* b = static_cast<unsigned char*>(dev_buf);
    n->bmax = batch_max;
    n->stream = static_cast<cudaStream_t>(stream);
    n->theta = reinterpret_cast<float*>(b + L.theta);
    n->m1 = reinterpret_cast<float*>(b + L.m1);
    n->m2 = reinterpret_cast<float*>(b + L.m2);
    n->grad = reinterpret_cast<float*>(b + L.grad);
    n->wmap = reinterpret_cast<int*>(b + L.wmap);
    n->wbf = reinterpret_cast<__nv_bfloat16*>(b + L.wbf);
    n->wmapT = reinterpret_cast<int*>(b + L.wmapT);
    n->wbfT = reinterpret_cast<__nv_bfloat16*>(b + L.wbfT);
    n->X = reinterpret_cast<__nv_bfloat16*>(b + L.X);
    n->XT = reinterpret_cast<__nv_bfloat16*>(b + L.XT);
    n->ldT = ld_t(batch_max);
    for (int l = 0; l < 4; ++l) {
        n->Z[l] = reinterpret_cast<float*>(b + L.Z[l]);
        n->H[l] = reinterpret_cast<__nv_bfloat16*>(b + L.H[l]);
        n->HT[l] = reinterpret_cast<__nv_bfloat16*>(b + L.HT[l]);
    }
    n->Y = reinterpret_cast<float*>(b + L.Y);
    for (int l = 0; l < 2; ++l) {
        n->G[l] = reinterpret_cast<__nv_bfloat16*>(b + L.G[l]);
        n->GT[l] = reinterpret_cast<__nv_bfloat16*>(b + L.GT[l]);
    }
    n->part = reinterpret_cast<float*>(b + L.part);
    n->loss = reinterpret_cast<double*>(b + L.loss);
    n->errflag = reinterpret_cast<int*>(b + L.err);
    n->ts = reinterpret_cast<TrainState*>(b + L.ts);
    // parameter offsets and the weight -> BF16 block map
    const long P = n_params();
    std::vector<int> wmap(P, -1), wmapT(P, -1);
    long o = 0, w = 0, wt = 0;
    for (int l = 0; l < kLayers; ++l) {
        const int ni = kDims[l], no = kDims[l + 1], ld = w_ld(l);
        n->woff[l] = o;
        n->wbf_off[l] = w;
        n->wbfT_off[l] = l > 0 ? wt : -1;
        for (int r = 0; r < no; ++r)
            for (int c = 0; c < ni; ++c) {
                wmap[o + (long)r * ni + c] = (int)(w + (long)r * ld + c);
                if (l > 0) wmapT[o + (long)r * ni + c] = (int)(wt + (long)c * wt_ld(l) + r);
            }
        o += (long)no * ni;
        w += (long)no * ld;
        if (l > 0) wt += (long)ni * wt_ld(l);
        n->boff[l] = o;
        o += no;
    }
    // the rows of ones under the transposed activations (BF16 1.0 = 0x3f80): columns past
    // the batch lie outside the tensor map and read as zero
    std::vector<uint16_t> ones((size_t)n->ldT, 0x3f80u);
    cudaError_t e = cudaMemsetAsync(dev_buf, 0, L.total, n->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(n->wmap, wmap.data(), P * sizeof(int), cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(n->wmapT, wmapT.data(), P * sizeof(int), cudaMemcpyHostToDevice, n->stream);
    for (int l = 0; l < 4 && e == cudaSuccess; ++l)
        e = cudaMemcpyAsync(n->HT[l] + (long)kHid * n->ldT, ones.data(), ones.size() * 2, cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(n->XT + (long)SALEC_MLP_IN * n->ldT, ones.data(), ones.size() * 2, cudaMemcpyHostToDevice,
                            n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    if (e != cudaSuccess) {
        delete n;
        return SALEC_ECUDA;
    }
    *out = n;
    return SALEC_OK;
}

salec_status salec_mlp_set_params(salec_mlp* n, const float* theta_host)
{
    if (!n || !theta_host) return SALEC_EINVAL;
    const long P = n_params();
    MLP_CUDA(n, cudaMemcpyAsync(n->theta, theta_host, P * 4, cudaMemcpyHostToDevice, n->stream), "set_params copy");
    MLP_CUDA(n, cudaMemsetAsync(n->m1, 0, P * 4, n->stream), "set_params reset");
    MLP_CUDA(n, cudaMemsetAsync(n->m2, 0, P * 4, n->stream), "set_params reset");
    MLP_CUDA(n, launch_refresh_bf16(n->theta, P, n->wmap, n->wbf, n->stream, n->wmapT, n->wbfT), "set_params bf16 copy");
    MLP_CUDA(n, cudaStreamSynchronize(n->stream), "set_params sync");
    n->steps = 0;
    return SALEC_OK;
}

salec_status salec_mlp_get_params(salec_mlp* n, float* theta_host)
{
    if (!n || !theta_host) return SALEC_EINVAL;
    MLP_CUDA(n, cudaMemcpyAsync(theta_host, n->theta, n_params() * 4, cudaMemcpyDeviceToHost, n->stream), "get_params");
    MLP_CUDA(n, cudaStreamSynchronize(n->stream), "get_params sync");
    return salec_mlp_check(n);
}

salec_status salec_mlp_forward(salec_mlp* n, const float* x_dev, int batch, float* y_dev)
{
    salec::HostRange range("salec_mlp_forward");
    salec_status st = check_batch(n, batch);
    if (st != SALEC_OK) return st;
    if (!x_dev || !y_dev) return fail(n, SALEC_EINVAL, "null pointer");
    MLP_CUDA(n, launch_inputs_bf16(x_dev, batch, SALEC_MLP_IN, kInLd, n->X, n->stream), "mlp input");
    // all five layers in one kernel, activations on chip; the layer-by-layer GEMMs when
    // the weights cannot be addressed by TMA
    FusedLaunch f;
    f.B = batch; f.X = n->X; f.ld_x = kInLd; f.Y = y_dev; f.err = n->errflag;
    for (int l = 0; l < kLayers; ++l) { f.W[l] = n->wbf + n->wbf_off[l]; f.bias[l] = n->theta + n->boff[l]; }
    const cudaError_t e = launch_mlp_forward_fused(f, n->stream);
    if (e == cudaSuccess) return SALEC_OK;
    if (e != cudaErrorNotSupported) return cuda_fail(n, e, "mlp fused forward");
    return forward_impl(n, batch, y_dev, SALEC_MLP_OUT, nullptr, false);
}

salec_status salec_mlp_gradient(salec_mlp* n, const float* x_dev, const float* t_dev, int batch, float* grad_dev,
                                double* loss_host)
{
    salec::HostRange range("salec_mlp_gradient");
    salec_status st = check_batch(n, batch);
    if (st != SALEC_OK) return st;
    if (!x_dev || !t_dev) return fail(n, SALEC_EINVAL, "null pointer");
    float* grad = grad_dev ? grad_dev : n->grad;
    MLP_CUDA(n, cudaMemsetAsync(n->loss, 0, 8, n->stream), "mlp loss reset");
    MLP_CUDA(n, launch_inputs_bf16(x_dev, batch, SALEC_MLP_IN, kInLd, n->X, n->stream, n->XT, n->ldT), "mlp input");
    st = forward_impl(n, batch, n->Y, SALEC_MLP_OUT, t_dev, true);
    if (st != SALEC_OK) return st;
    st = backward_impl(n, batch, grad);
    if (st != SALEC_OK) return st;
    if (loss_host) {
        double s = 0.0;
        MLP_CUDA(n, cudaMemcpyAsync(&s, n->loss, 8, cudaMemcpyDeviceToHost, n->stream), "mlp loss read");
        MLP_CUDA(n, cudaStreamSynchronize(n->stream), "mlp loss sync");
        *loss_host = s / ((double)batch * SALEC_MLP_OUT);
        return salec_mlp_check(n);
    }
    return SALEC_OK;
}

salec_status salec_mlp_train_step(salec_mlp* n, const float* x_dev, const float* t_dev, int batch, float lr,
                                  float beta1, float beta2, float eps, double* sse_dev)
{
    salec::HostRange range("salec_mlp_train_step");
    salec_status st = check_batch(n, batch);
    if (st != SALEC_OK) return st;
    if (!x_dev || !t_dev) return fail(n, SALEC_EINVAL, "null pointer");
    if (!(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return fail(n, SALEC_EINVAL, "bad Adam hyper-parameters");
    MLP_CUDA(n, cudaMemsetAsync(n->loss, 0, 8, n->stream), "mlp loss reset");
    MLP_CUDA(n, launch_inputs_bf16(x_dev, batch, SALEC_MLP_IN, kInLd, n->X, n->stream, n->XT, n->ldT), "mlp input");
    st = forward_impl(n, batch, n->Y, SALEC_MLP_OUT, t_dev, true);
    if (st != SALEC_OK) return st;
    st = backward_impl(n, batch, n->grad);
    if (st != SALEC_OK) return st;
    n->steps += 1;
    AdamArgs a;
    a.lr = lr; a.beta1 = beta1; a.beta2 = beta2; a.eps = eps; a.ts = nullptr;
    a.c1 = (float)(1.0 / (1.0 - std::pow((double)beta1, (double)n->steps)));
    a.c2 = (float)(1.0 / (1.0 - std::pow((double)beta2, (double)n->steps)));
    MLP_CUDA(n, launch_adam(n->theta, n->m1, n->m2, n->grad, n_params(), a, n->wmap, n->wbf, n->stream, n->wmapT, n->wbfT), "mlp adam");
    if (sse_dev) MLP_CUDA(n, cudaMemcpyAsync(sse_dev, n->loss, 8, cudaMemcpyDeviceToDevice, n->stream), "mlp loss copy");
    return SALEC_OK;
}

salec_status salec_mlp_train(salec_mlp* n, const float* x_dev, const float* t_dev, int batch, int steps,
                             const float* lr_dev, float beta1, float beta2, float eps, double* sse_dev)
{
    salec::HostRange range("salec_mlp_train");
    salec_status st = check_batch(n, batch);
    if (st != SALEC_OK) return st;
    if (steps < 0) return fail(n, SALEC_EINVAL, "negative step count");
    if (steps == 0) return SALEC_OK;
    if (!x_dev || !t_dev || !lr_dev) return fail(n, SALEC_EINVAL, "null pointer");
    if (!(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return fail(n, SALEC_EINVAL, "bad Adam hyper-parameters");
    if (n->steps + (long)steps > 0x7fffffffL) return fail(n, SALEC_EINVAL, "step count overflow");
    MLP_CUDA(n, launch_inputs_bf16(x_dev, batch, SALEC_MLP_IN, kInLd, n->X, n->stream, n->XT, n->ldT), "mlp input");
    MLP_CUDA(n, launch_train_reset(n->ts, (int)n->steps, n->stream), "mlp train reset");
    // the first step with plain launches (it also sets the kernels' attributes), then whole
    // chunks as graph replays, then the rest
    st = train_one(n, batch, t_dev, lr_dev, beta1, beta2, eps);
    if (st != SALEC_OK) return st;
    int done = 1;
    const int chunks = (steps - 1) / kTrainChunk;
    if (chunks > 0 && n->tg_ok) {
        const bool same = n->tgraph && n->tg_t == t_dev && n->tg_lr == lr_dev && n->tg_batch == batch &&
                          n->tg_beta1 == beta1 && n->tg_beta2 == beta2 && n->tg_eps == eps;
        if (!same && !capture_train(n, batch, t_dev, lr_dev, beta1, beta2, eps)) n->tg_ok = false;
        if (n->tgraph && n->tg_ok) {
            for (int c = 0; c < chunks; ++c) MLP_CUDA(n, cudaGraphLaunch(n->tgraph, n->stream), "mlp train graph");
            done += chunks * kTrainChunk;
        }
    }
    for (; done < steps; ++done) {
        st = train_one(n, batch, t_dev, lr_dev, beta1, beta2, eps);
        if (st != SALEC_OK) return st;
    }
    n->steps += steps;
    if (sse_dev) MLP_CUDA(n, cudaMemcpyAsync(sse_dev, n->loss, 8, cudaMemcpyDeviceToDevice, n->stream), "mlp loss copy");
    return SALEC_OK;
}

salec_status salec_mlp_check(salec_mlp* n)
{
    if (!n) return SALEC_EINVAL;
    int f = 0;
    MLP_CUDA(n, cudaMemcpyAsync(&f, n->errflag, 4, cudaMemcpyDeviceToHost, n->stream), "mlp flag read");
    MLP_CUDA(n, cudaStreamSynchronize(n->stream), "mlp flag sync");
    if (f) return fail(n, SALEC_ECUDA, "a tensor-core wait ran out of time");
    return SALEC_OK;
}

salec_status salec_gemm_bf16(int M, int N, int K, const void* A, long a_sm, long a_sk, const void* B, long b_sn,
                             long b_sk, float* C, long ldc, void* stream)
{
    if (M < 0 || N < 0 || K < 0) return SALEC_EINVAL;
    if (M > 0 && N > 0 && (!C || (K > 0 && (!A || !B)))) return SALEC_EINVAL;   // K = 0: C = 0, A and B unused
    GemmArgs g = gemm0(M, N, K, nullptr);
    g.A = static_cast<const __nv_bfloat16*>(A); g.a_sm = a_sm; g.a_sk = a_sk;
    g.B = static_cast<const __nv_bfloat16*>(B); g.b_sn = b_sn; g.b_sk = b_sk;
    g.epi = kEpiStore;
    g.C = C; g.ldc = ldc;
    if (launch_gemm(g, static_cast<cudaStream_t>(stream)) != cudaSuccess) return SALEC_ECUDA;
    return SALEC_OK;
}

salec_status salec_mlp_group_create(salec_mlp* const* nets, int n, void* stream, salec_mlp_group** out)
{
    if (!out || !nets || n < 1 || n > kMaxGroup) return SALEC_EINVAL;
    *out = nullptr;
    for (int k = 0; k < n; ++k) {
        if (!nets[k]) return SALEC_EINVAL;
        for (int j = 0; j < k; ++j)
            if (nets[j] == nets[k]) return SALEC_EINVAL;
    }
    salec_mlp_group* g = new (std::nothrow) salec_mlp_group();
    if (!g) return SALEC_ENOMEM;
    g->nets.assign(nets, nets + n);
    g->stream = static_cast<cudaStream_t>(stream);
    *out = g;
    return SALEC_OK;
}

salec_status salec_mlp_train_group(salec_mlp_group* G, const float* x_dev, const float* t_dev, int batch, int steps,
                                   const float* lr_dev, float beta1, float beta2, float eps)
{
    salec::HostRange range("salec_mlp_train_group");
    if (!G) return SALEC_EINVAL;
    if (steps < 0) return gfail(G, SALEC_EINVAL, "negative step count");
    if (steps == 0) return SALEC_OK;
    if (!x_dev || !t_dev || !lr_dev) return gfail(G, SALEC_EINVAL, "null pointer");
    if (!(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return gfail(G, SALEC_EINVAL, "bad Adam hyper-parameters");
    for (salec_mlp* m : G->nets) {
        if (batch < 1 || batch > m->bmax) return gfail(G, SALEC_EINVAL, "batch outside 1..batch_max of a member");
        if (m->steps + (long)steps > 0x7fffffffL) return gfail(G, SALEC_EINVAL, "step count overflow");
    }
    cudaStream_t s = G->stream;
    for (salec_mlp* m : G->nets) {
        GROUP_CUDA(G, launch_inputs_bf16(x_dev, batch, SALEC_MLP_IN, kInLd, m->X, s, m->XT, m->ldT), "group input");
        GROUP_CUDA(G, launch_train_reset(m->ts, (int)m->steps, s), "group train reset");
    }
    // the first step with plain launches (it also sets the kernels' attributes), then whole
    // chunks as graph replays, then the rest
    salec_status st = group_train_one(G, s, batch, t_dev, lr_dev, beta1, beta2, eps);
    if (st != SALEC_OK) return st;
    int done = 1;
    const int chunks = (steps - 1) / kTrainChunk;
    if (chunks > 0 && G->tg_ok) {
        const bool same = G->tgraph && G->tg_t == t_dev && G->tg_lr == lr_dev && G->tg_batch == batch &&
                          G->tg_beta1 == beta1 && G->tg_beta2 == beta2 && G->tg_eps == eps;
        if (!same && !capture_group(G, batch, t_dev, lr_dev, beta1, beta2, eps)) G->tg_ok = false;
        if (G->tgraph && G->tg_ok) {
            for (int c = 0; c < chunks; ++c) GROUP_CUDA(G, cudaGraphLaunch(G->tgraph, s), "group train graph");
            done += chunks * kTrainChunk;
        }
    }
    for (; done < steps; ++done) {
        st = group_train_one(G, s, batch, t_dev, lr_dev, beta1, beta2, eps);
        if (st != SALEC_OK) return st;
    }
    for (salec_mlp* m : G->nets) m->steps += steps;
    return SALEC_OK;
}

const char* salec_mlp_group_last_error(const salec_mlp_group* g) { return g ? g->err.c_str() : "null group"; }

void salec_mlp_group_destroy(salec_mlp_group* g) { delete g; }

const char* salec_mlp_last_error(const salec_mlp* n) { return n ? n->err.c_str() : ""; }

void salec_mlp_destroy(salec_mlp* n) { delete n; }

}  // extern "C"
