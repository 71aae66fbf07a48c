/*
 * npf_mlp.h -- C ABI of the learned surrogate of the NPF library: an ensemble of small
 * multilayer perceptrons that maps an operating-point parameter vector to the dominant NPF
 * magnitudes, trained and evaluated by hand-written BF16 tensor-core kernels (BF16 operands, FP32
 * accumulation). The paper has no learned part: its participation factors (Section II, Eq. 4-7,
 * Algorithm 2) are what the network is trained on, and the plain contraction (npf.h) remains the
 * reference and the fallback whenever the ensemble members disagree.
 *
 * Network of one member, layers l = 0 .. L-1 with widths w_0 (inputs) .. w_L (outputs):
 *     z_l = W_l h_l + b_l,   h_{l+1} = relu(z_l) for l < L-1,   y = z_{L-1}.
 * Loss of one member over a set of R rows: (1 / (R w_L)) sum_{r,o} (y_ro - t_ro)^2 (mean squared
 * error). Training: Adam (beta1 0.9, beta2 0.999, epsilon 1e-8, constant learning rate) on
 * minibatches drawn without replacement from a per-epoch permutation (one per member).
 *
 * Arithmetic: W_l, b_l, the inputs, the hidden activations and the back-propagated errors are
 * rounded to BF16 (round to nearest even) where they enter a product; products accumulate in
 * FP32; master weights, Adam moments, outputs, losses and gradients are FP32.
 *
 * Conventions
 *   - Weights (host or device, FP32): for member e = 0..E-1, layer l = 0..L-1 in order, the
 *     matrix [w_{l+1}][w_l + 1] row-major whose last column is the bias b_l. Members follow one
 *     another. npf_mlp_param_count() gives the floats per member.
 *   - Row-major float arrays; pointers may be host or device memory (classified with
 *     cudaPointerGetAttributes); the caller owns them; inputs are copied before use.
 *   - Return NPF_OK (0) or an error code of npf.h; the message is in npf_last_error().
 *   - Work runs on the stream given at creation; every call returns after it has finished.
 *   - Limits: 1 <= E <= 16, 2 <= L <= 8, w_0 <= 15, other widths 8 .. 1024 and hidden widths
 *     multiples of 16 (checked; NPF_ERR_ARG otherwise).
 */
#ifndef NPF_MLP_H_
#define NPF_MLP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct npf_mlp npf_mlp;

/* An ensemble of E members with L layers and widths[0..L]; weights as above (copied). stream is
 * a cudaStream_t (NULL = legacy default). NULL on error. */
npf_mlp* npf_mlp_create(int ensemble, int layers, const int* widths, const float* weights,
                        void* stream);

/* Floats per member in the weight layout above. */
int64_t npf_mlp_param_count(const npf_mlp* m);

/* Current FP32 master weights of every member into weights (layout above). */
int npf_mlp_get_weights(const npf_mlp* m, float* weights);

/* Outputs of every member for `rows` inputs X[rows][w_0]: Y[e][rows][w_L]. */
int npf_mlp_forward(npf_mlp* m, int rows, const float* X, float* Y);

/* Loss and its gradient for every member on the rows X[rows][w_0], targets T[rows][w_L]:
 * grads[e] in the weight layout (bias gradients in the bias column), loss[e]. rows <= 65536. */
int npf_mlp_loss_grad(npf_mlp* m, int rows, const float* X, const float* T, float* grads,
                      float* loss);

/* Train every member for `epochs` passes over X[rows][w_0], T[rows][w_L] with minibatches of
 * `batch` rows (the last partial batch of an epoch is dropped), learning rate lr. The per-epoch
 * permutations are drawn from splitmix64 seeded with seed + 7919 e for member e (Fisher-Yates).
 * epoch_loss[epochs] (may be NULL) receives the mean minibatch loss over members per epoch. */
int npf_mlp_train(npf_mlp* m, int rows, const float* X, const float* T, int epochs, int batch,
                  double lr, uint64_t seed, float* epoch_loss);

/* Gated ensemble prediction. The members' outputs are read as standardised logarithms,
 * v_e = exp(mu[o] + sigma[o] y_e), and for every row the ensemble mean mean[r][o] = mean_e v_e
 * and the largest relative spread spread[r] = max_o std_e(v_e) / mean_e(v_e) (population
 * standard deviation) are returned; fallback[r] = 1 when spread[r] > spread_limit (the row must
 * be recomputed by the plain method), else 0. mu, sigma: [w_L]. */
int npf_mlp_predict(npf_mlp* m, int rows, const float* X, const float* mu, const float* sigma,
                    double spread_limit, float* mean, float* spread, int* fallback);

void npf_mlp_destroy(npf_mlp* m);

#ifdef __cplusplus
}
#endif

#endif /* NPF_MLP_H_ */
