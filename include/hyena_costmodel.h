/* Learned cost model: a small perceptron on the GPU that predicts kernel
 * latencies of encrypted-convolution configurations (ring degree, limbs,
 * packing, tile shape, MAC schedule).  It has no counterpart in the paper,
 * which fixes its parameters by the noise analysis of Sec. 3.2.1; the model
 * ranks the configurations that analysis allows by predicted time, and
 * exhaustive timing (he_conv_time in hyena.h) is its fallback and its yardstick.
 *
 * Network: F features -> 64 -> 64 -> 1, ReLU after the two hidden layers,
 * fp32.  Features and target are standardised with the mean and standard
 * deviation of the training set (he_mlp_fit_scaling), and training minimises
 * the mean squared error of the standardised target with Adam (Kingma and
 * Ba, 2015; beta1 0.9, beta2 0.999, eps 1e-8) on mini-batches drawn with
 * replacement by a counter-based generator (SplitMix64 of seed and step),
 * so a run is deterministic for a seed.
 *
 * All arrays named d_* are device memory owned by the caller; X is row-major
 * [n][F] fp32, y is [n] fp32.  Calls return HE_OK or an HE_* error code with
 * the message in he_last_error(); they run on `stream` (NULL = default) and,
 * except he_mlp_predict, synchronise it. */
#ifndef HYENA_COSTMODEL_H
#define HYENA_COSTMODEL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct he_mlp he_mlp;

/* New network on the current device: He-uniform weights from `seed`, zero
 * biases, identity scaling.  1 <= n_features <= 64, else HE_EINVAL. */
int he_mlp_create(uint32_t n_features, uint64_t seed, he_mlp** out);
/* Number of floats of he_mlp_get_params: the weights in the order
 * W1[64][F], b1[64], W2[64][64], b2[64], w3[64], b3, then the scaling
 * mean[F], mean_y, std[F], std_y. */
int he_mlp_param_count(const he_mlp* m, uint32_t* count);
int he_mlp_get_params(const he_mlp* m, float* h_params);
/* Also resets the optimiser state.  Standard deviations must be positive. */
int he_mlp_set_params(he_mlp* m, const float* h_params);
/* Sets the scaling from the columns of X and from y (n >= 2). */
int he_mlp_fit_scaling(he_mlp* m, const float* d_X, const float* d_y, uint32_t n, void* stream);
/* One Adam step on a mini-batch of `batch` rows drawn from the n rows with
 * learning rate lr; *loss (may be NULL) = the batch's mean squared error of
 * the standardised target before the step. */
int he_mlp_step(he_mlp* m, const float* d_X, const float* d_y, uint32_t n, uint32_t batch, float lr, uint64_t seed,
                void* stream, float* loss);
/* he_mlp_fit_scaling, then `steps` Adam steps with the step size decayed from
 * lr to lr/10 along a half cosine; *final_loss (may be NULL) = the last
 * batch's loss. */
int he_mlp_train(he_mlp* m, const float* d_X, const float* d_y, uint32_t n, uint32_t steps, uint32_t batch, float lr,
                 uint64_t seed, void* stream, float* final_loss);
/* d_y[i] = prediction for row i, in the target's units.  Asynchronous. */
int he_mlp_predict(const he_mlp* m, const float* d_X, uint32_t n, float* d_y, void* stream);
void he_mlp_destroy(he_mlp* m);

#ifdef __cplusplus
}
#endif
#endif
