// mlp_internal.cuh -- argument blocks and launchers of the surrogate-MLP kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>

namespace salec {
namespace mlp {

// fused epilogues of the GEMM
enum Epi {
    kEpiStore = 0,      // C = acc (+ bias[n] if bias)                               FP32
    kEpiBiasGelu = 1,   // C = Z = acc + bias[n] (FP32; skipped when C is null), Hout = gelu(Z) (BF16)
    kEpiGeluBwd = 2,    // Hout = acc * gelu'(Zin) (BF16): dL/dZ of a hidden layer
    kEpiOutLoss = 3,    // C = Y = acc + bias[n]; Hout = grad_scale (Y - Tin) (BF16); loss += sum (Y - Tin)^2
};

struct GemmArgs {
    int M, N, K;
    const __nv_bfloat16* A;
    long a_sm, a_sk;
    const __nv_bfloat16* B;
    long b_sn, b_sk;
    int epi;
    float* C;                 // FP32 output, row stride ldc
    long ldc;
    const float* bias;        // [N] or null
    __nv_bfloat16* Hout;      // BF16 output, row stride ldh
    long ldh;
    __nv_bfloat16* HoutT;     // the same BF16 output transposed (HoutT[n * ldhT + m]), or null
    long ldhT;
    const float* Zin;         // saved pre-activations, row stride ldz
    long ldz;
    const float* Tin;         // targets, row stride ldt
    long ldt;
    float grad_scale;         // 2 / (B n_out)
    double* loss;             // sum of squared errors (atomic), or null
    int* err;                 // error flag, or null
    float* part;              // kEpiStore without bias: workspace for split-K partials
                              // (kMaxSplit x M x N floats), or null for no split
    float* Cb;                // with part: column N - 1 of C goes to Cb[m] instead (a bias
                              // gradient summed against a row of ones), C keeps columns < N - 1
    int nt, tmem_cols;        // set by the launcher
    int kchunk;               // set by the launcher: K per split (0: no split)
    int stages;               // set by the launcher: shared-memory stages of the TMA-fed kernel
};

constexpr int kMaxSplit = 16;
constexpr int kMaxGroup = 8;      // ensemble members one group launch takes

constexpr int SALEC_MLP_OUT_N = 66;

// the fused inference pass: inputs, weights (BF16, W_1 rows padded like X), biases, outputs
struct FusedLaunch {
    int B;
    const __nv_bfloat16* X;
    int ld_x;
    const __nv_bfloat16* W[5];
    const float* bias[5];
    float* Y;
    int* err;
};

// Device state of a multi-step training call: k = steps of the call begun so far, t0 = Adam
// steps before the call; the step's learning rate and bias corrections, formed once per step.
struct TrainState {
    int k, t0;
    float lr, c1, c2;
};

struct AdamArgs {
    float lr, beta1, beta2, eps, c1, c2;   // c1 = 1 / (1 - beta1^t), c2 = 1 / (1 - beta2^t)
    const TrainState* ts;                  // not null: lr, c1, c2 from here instead
};

cudaError_t launch_gemm(const GemmArgs& g, cudaStream_t s);
cudaError_t launch_mlp_forward_fused(const FusedLaunch& f, cudaStream_t s);
cudaError_t launch_inputs_bf16(const float* x, int rows, int cols, int ld, __nv_bfloat16* y, cudaStream_t s,
                               __nv_bfloat16* yT = nullptr, long ldT = 0);
// wmapT / wbfT (optional): a second BF16 copy of every weight at wmapT[i] (the transposed
// weights of the backward pass)
cudaError_t launch_adam(float* theta, float* m1, float* m2, const float* grad, long n, const AdamArgs& a,
                        const int* wmap, __nv_bfloat16* wbf, cudaStream_t s, const int* wmapT = nullptr,
                        __nv_bfloat16* wbfT = nullptr);
// one thread: ts->k = 0, ts->t0 = t0
cudaError_t launch_train_reset(TrainState* ts, int t0, cudaStream_t s);
// one thread, first kernel of a step: k += 1, lr = lr_dev[k - 1], the bias corrections of
// Adam step t0 + k, loss = 0
cudaError_t launch_train_begin(TrainState* ts, const float* lr_dev, float beta1, float beta2, double* loss,
                               cudaStream_t s);
cudaError_t launch_refresh_bf16(const float* theta, long n, const int* wmap, __nv_bfloat16* wbf, cudaStream_t s,
                                const int* wmapT = nullptr, __nv_bfloat16* wbfT = nullptr);
size_t gemm_smem_bytes(int nt);

// An ensemble's members advanced together: each GEMM of a step is one launch for every
// member (n <= kMaxGroup, the same shapes, each member's own buffers), with the same plan
// and arithmetic per member as launch_gemm; likewise the Adam update and the step's start.
cudaError_t launch_gemm_group(const GemmArgs* g, int n, cudaStream_t s);
struct AdamGroup {
    float* theta[kMaxGroup];
    float* m1[kMaxGroup];
    float* m2[kMaxGroup];
    const float* grad[kMaxGroup];
    __nv_bfloat16* wbf[kMaxGroup];
    __nv_bfloat16* wbfT[kMaxGroup];
    const TrainState* ts[kMaxGroup];
};
cudaError_t launch_adam_group(const AdamGroup& a, int n, long np, float beta1, float beta2, float eps, const int* wmap,
                              const int* wmapT, cudaStream_t s);
struct BeginGroup {
    TrainState* ts[kMaxGroup];
    double* loss[kMaxGroup];
};
cudaError_t launch_train_begin_group(const BeginGroup& b, int n, const float* lr_dev, float beta1, float beta2,
                                     cudaStream_t s);

}  // namespace mlp
}  // namespace salec
