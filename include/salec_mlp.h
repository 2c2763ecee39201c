/* salec_mlp.h -- C ABI of the crater-surrogate MLP.
 *
 * The paper has no learned component.  This network maps five impact parameters to the
 * crater outputs that the solver of salec.h produces (the crater profile the paper follows
 * in its verification runs, Sect. "Verification of the PML method", Fig. 3): a 64-point
 * radial depth profile, the transient crater depth and the crater diameter.
 *
 * Network: 5 inputs -> 4 hidden layers of 256 units with GELU in its erf form
 * (gelu(z) = z Phi(z), Hendrycks & Gimpel 2016) -> 66 linear outputs; loss = mean squared
 * error over all outputs of the batch; optimiser = Adam (Kingma & Ba 2015, Algorithm 1).
 *
 * Precision: FP32 master parameters; BF16 copies of the weights, BF16 inputs, hidden
 * activations and back-propagated gradients as tensor-core operands; FP32 accumulation in
 * tensor memory; FP32 biases, pre-activations and outputs; FP64 loss sum.
 *
 * Parameter vector: 215 874 floats, layer by layer W_l (n_out x n_in, row-major) then b_l.
 *
 * Memory: one caller-owned device buffer of salec_mlp_bytes(batch_max) bytes (256-byte
 * aligned) holds parameters, Adam moments, gradient and activations; the library
 * allocates no device memory.  All work goes on the stream given at creation and is
 * asynchronous unless stated.  Pointers named *_dev are device pointers, *_host host
 * pointers.  Errors: SALEC_EINVAL (bad argument), SALEC_ENOMEM (buffer too small),
 * SALEC_ECUDA (CUDA error, or a tensor-core wait that ran out of time, reported by
 * salec_mlp_check); salec_mlp_last_error() gives the message. */
#ifndef SALEC_MLP_H
#define SALEC_MLP_H

#include <stddef.h>

#include "salec.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SALEC_MLP_IN 5
#define SALEC_MLP_OUT 66

typedef struct salec_mlp salec_mlp;

int salec_mlp_n_params(void);
salec_status salec_mlp_bytes(int batch_max, size_t* bytes);
salec_status salec_mlp_create(int batch_max, void* dev_buf, size_t bytes, void* stream, salec_mlp** out);

/* Copies 215 874 FP32 parameters from the host, refreshes the BF16 weight copies and
 * resets the Adam moments and step count (synchronous). */
salec_status salec_mlp_set_params(salec_mlp* mlp, const float* theta_host);
/* Copies the FP32 parameters to the host (synchronous; also runs salec_mlp_check). */
salec_status salec_mlp_get_params(salec_mlp* mlp, float* theta_host);

/* y_dev[b][o] = network(x_dev[b][:]) for b < batch <= batch_max; x_dev is batch x 5 FP32,
 * y_dev batch x 66 FP32, both row-major device arrays.  One persistent kernel runs all
 * five layers on 128-sample tiles, two per SM at a time (one on the tensor cores while the
 * other's epilogue runs), with the activations kept on chip. */
salec_status salec_mlp_forward(salec_mlp* mlp, const float* x_dev, int batch, float* y_dev);

/* Forward and backward pass against targets t_dev (batch x 66 FP32): the gradient of the
 * loss goes to grad_dev (215 874 FP32, device; NULL: the internal gradient buffer).  If
 * loss_host is not NULL the call synchronises and stores the loss there. */
salec_status salec_mlp_gradient(salec_mlp* mlp, const float* x_dev, const float* t_dev, int batch, float* grad_dev,
                                double* loss_host);

/* One training step: gradient as above, then one Adam update of the FP32 parameters
 * (bias-corrected moments, step count kept by the context) and a refresh of the BF16 weight
 * copies.  If sse_dev is not NULL the step's sum of squared errors (FP64) is copied there
 * (device).  Asynchronous. */
salec_status salec_mlp_train_step(salec_mlp* mlp, const float* x_dev, const float* t_dev, int batch, float lr,
                                  float beta1, float beta2, float eps, double* sse_dev);

/* `steps` training steps as above, step k (0-based) with learning rate lr_dev[k] (`steps`
 * FP32 values on the device, read as each step begins), in one call: the inputs are
 * converted once, and after the first step whole chunks of 25 steps go out as CUDA-graph
 * replays into the context's stream (the graph is captured again when t_dev, lr_dev, batch
 * or a hyper-parameter changes).  The Adam step count continues from the context's; the
 * arithmetic of every step is that of salec_mlp_train_step, with the bias corrections
 * formed on the device.  Contexts on different streams train concurrently.  If sse_dev is
 * not NULL the last step's sum of squared errors is copied there.  SALEC_EINVAL for a
 * negative step count, a null pointer or a bad hyper-parameter.  Asynchronous. */
salec_status salec_mlp_train(salec_mlp* mlp, const float* x_dev, const float* t_dev, int batch, int steps,
                             const float* lr_dev, float beta1, float beta2, float eps, double* sse_dev);

/* Ensemble training: n (1..8) distinct networks trained together on the same inputs,
 * targets and learning-rate table, each step's GEMMs, Adam update and bookkeeping issued
 * as ONE launch for all members (a member index per CTA), each member with the same plan
 * and arithmetic as salec_mlp_train gives it alone, so the results are those of n separate
 * salec_mlp_train calls.  The group holds pointers to the member contexts (which must
 * outlive it) and works on `stream` (the members' own streams are not used by group
 * calls).  salec_mlp_train_group: `steps` steps, step k with learning rate lr_dev[k]; the
 * first step with plain launches, then chunks of 25 steps as CUDA-graph replays (captured
 * again when t_dev, lr_dev, batch or a hyper-parameter changes); every member's Adam step
 * count advances by `steps`.  SALEC_EINVAL for n outside 1..8, a repeated or null member,
 * a batch above a member's batch_max, a negative step count, a null pointer or a bad
 * hyper-parameter.  Asynchronous; salec_mlp_check on each member reports a tensor-core
 * wait that ran out. */
typedef struct salec_mlp_group salec_mlp_group;
salec_status salec_mlp_group_create(salec_mlp* const* nets, int n, void* stream, salec_mlp_group** out);
salec_status salec_mlp_train_group(salec_mlp_group* group, const float* x_dev, const float* t_dev, int batch,
                                   int steps, const float* lr_dev, float beta1, float beta2, float eps);
const char* salec_mlp_group_last_error(const salec_mlp_group* group);
void salec_mlp_group_destroy(salec_mlp_group* group);

/* Synchronises and reports whether a tensor-core wait ran out of time since creation. */
salec_status salec_mlp_check(salec_mlp* mlp);

/* C[m * ldc + n] = sum_k A[m * a_sm + k * a_sk] B[n * b_sn + k * b_sk] for m < M, n < N:
 * the tensor-core GEMM under the network, BF16 operands (device, any element strides), FP32
 * accumulation and output (device).  Asynchronous on `stream`. */
salec_status salec_gemm_bf16(int M, int N, int K, const void* A, long a_sm, long a_sk, const void* B, long b_sn,
                             long b_sk, float* C, long ldc, void* stream);

const char* salec_mlp_last_error(const salec_mlp* mlp);
void salec_mlp_destroy(salec_mlp* mlp);

#ifdef __cplusplus
}
#endif

#endif
