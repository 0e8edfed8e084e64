/*
 * sgnet.h -- C ABI of the learned warm start for the SG solver (include/sg.h).
 *
 * No counterpart in the paper: the paper's method starts GMRES from zero.  This network maps the
 * features z = (sigma, ell, sqrt(lambda_1..M)) of an SG system (Sec. 2.1, Eq. aKL) to a guess of
 * its chaos-coefficient field X (N x P, the layout of include/sg.h, flattened to D = N*P), which
 * sg_gmres_solve then takes as its initial iterate.  The final FP64 residual still decides
 * convergence, so a poor guess costs iterations, never accuracy.
 *
 * Model: z_hat = (z - mu) / sd,  h1 = tanh(W1 z_hat + b1),  h2 = tanh(W2 h1 + b2),
 * y = W3 h2 + b3; loss = sum (y - t)^2 / (B D).  Parameters are FP32 (the master copy of Adam);
 * with ``bf16`` = 1 the output layer, which holds almost all parameters, computes from a BF16
 * copy of W3 with FP32 accumulation, on the tensor cores (tcgen05 MMAs, h2 rounded to BF16) when
 * h2 <= 64.  Flat parameter order: W1 (h1 x in, row-major), b1, W2
 * (h2 x h1), b2, W3 (out x h2), b3.
 *
 * All array arguments are device pointers owned by the caller unless stated; calls are
 * asynchronous on ``stream`` unless they return a value to the host.  Errors as in sg.h
 * (SG_ERR_*, message from sg_last_error()).
 */
#ifndef SG_GB300_NET_H
#define SG_GB300_NET_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sgnet sgnet;

/* Create a network with in_dim <= 16, h1, h2 <= 128, out_dim >= 1, batches up to max_batch
 * (<= 1024).  Weights: Glorot-uniform from splitmix64(seed), biases 0, mu = 0, sd = 1. */
int sgnet_create(int in_dim, int h1, int h2, int out_dim, int max_batch, int bf16,
                 unsigned long long seed, sgnet** out);

/* From n training pairs (Z: n x in, T: n x out, FP32, device): mu, sd := per-feature mean and
 * standard deviation of Z (sd floored at 1e-6), b3 := per-output mean of T. */
int sgnet_set_stats(sgnet* net, const float* Z, const float* T, int n, void* stream);

/* Output basis from the training targets (call after sgnet_set_stats with the same T): the
 * first min(n, h2) centred targets T_r - b3 are orthonormalised (classical Gram-Schmidt applied
 * twice, FP64 sums), each basis vector q_j is scaled by s_j = max_r |q_j . (T_r - b3)| / 0.9, and
 * W3 := [s_j q_j] with the remaining columns 0; Adam then leaves W3 and b3 fixed.  Every
 * prediction lies in the span of training solutions around their mean, so its error is a smooth
 * combination of solutions rather than unstructured noise, which K would amplify in the initial
 * residual.  Synchronous. */
int sgnet_set_basis(sgnet* net, const float* T, int n, void* stream);

/* Forward pass for B <= max_batch inputs; Y: B x out FP32 (device). */
int sgnet_forward(sgnet* net, const float* Z, int B, float* Y, void* stream);

/* Forward pass written as FP64 (the SG solver's initial guess layout); X: B x out FP64. */
int sgnet_predict(sgnet* net, const float* Z, int B, double* X, void* stream);

/* Loss of the batch (Z, T) and its gradient, kept inside the network (see sgnet_get).
 * If ``loss`` (host) is not NULL the call synchronises the stream and stores the loss; it returns
 * SG_ERR_CUDA if a tensor-core kernel's bounded wait for its MMAs timed out.  With ``bf16`` = 1
 * and the output layer fixed by sgnet_set_basis, the output layer and the back-propagation into
 * the hidden layer run on the tensor cores (BF16 operands, FP32 accumulation; dY rounded to
 * BF16), and the gradient's W3 and b3 parts are not formed (Adam leaves them fixed). */
int sgnet_loss_grad(sgnet* net, const float* Z, const float* T, int B, float* loss, void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with the stored gradient. */
int sgnet_adam_step(sgnet* net, float lr, void* stream);

/* sgnet_loss_grad followed by sgnet_adam_step. */
int sgnet_train_step(sgnet* net, const float* Z, const float* T, int B, float lr, float* loss,
                     void* stream);

/* Number of parameters (the flat order above). */
long long sgnet_num_params(const sgnet* net);

/* Copy to host: what = 0 parameters, 1 gradient (count = sgnet_num_params), 2 mu then sd
 * (2 * in_dim).  Synchronous. */
int sgnet_get(const sgnet* net, int what, float* host, size_t count);

/* Overwrite the parameters (what = 0) or mu and sd (what = 2) from host memory. */
int sgnet_set(sgnet* net, int what, const float* host, size_t count);

void sgnet_free(sgnet* net);

#ifdef __cplusplus
}
#endif

#endif /* SG_GB300_NET_H */
