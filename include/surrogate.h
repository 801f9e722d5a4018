/* C ABI of the learned surrogate used to screen variational parameters before the MPDO re-scores
 * them.  The paper has no surrogate: this is the screening model the noisy-circuit workload is
 * paired with (an MLP from QAOA angles plus channel descriptors to predicted <H_MaxCut>/|E| and GHZ
 * fidelity), trained on data the MPDO itself produces.
 *
 * Model: in_dim -> hidden (x n_hidden, GELU(z) = z (1 + erf(z / sqrt 2)) / 2) -> out_dim (linear).
 * Parameters are held as FP32 masters with a BF16 copy; forward and backward products take BF16
 * weights and activations and accumulate in FP32 (the forward products of layers 32..256 wide on the
 * tensor cores, tcgen05 BF16 -> FP32; the rest on CUDA cores).  Loss: mean squared error over
 * batch x out_dim.
 * Optimiser: AdamW with decoupled weight decay on the weight matrices only (not on the biases).
 * Parameter vector order: for each layer l, W_l (out x in, row-major) then b_l.
 * All *_dev pointers are device FP32 arrays, row-major batch x dim; work is enqueued on the
 * handle's stream; host outputs synchronise.  Every call returns a surr_status. */
#ifndef SURROGATE_H
#define SURROGATE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct surr_ctx* surr_t;
typedef enum { SURR_OK = 0, SURR_EINVAL = 1, SURR_ENOMEM = 2, SURR_ECUDA = 7 } surr_status;

/* Initial weights: uniform(-a, a), a = sqrt(6 / fan_in) (halved for the output layer), from a
 * splitmix64 stream seeded with `seed`; biases 0.  max_batch bounds every later batch. */
surr_status surr_create(int in_dim, int hidden, int n_hidden, int out_dim, int max_batch, unsigned long long seed,
                        void* stream, surr_t* out);
surr_status surr_free(surr_t s);
long long surr_num_params(surr_t s);
surr_status surr_get_params(surr_t s, float* host);
surr_status surr_set_params(surr_t s, const float* host);
/* Y_dev (batch x out_dim) = model(X_dev (batch x in_dim)). */
surr_status surr_forward(surr_t s, const float* X_dev, int batch, float* Y_dev);
/* Gradients of the MSE against targets T_dev into the handle (read with surr_get_grads);
 * loss_host (nullable) receives the loss. */
surr_status surr_gradients(surr_t s, const float* X_dev, const float* T_dev, int batch, double* loss_host);
surr_status surr_get_grads(surr_t s, float* host);
/* One AdamW step with the stored gradients (bias-corrected moments, step counter in the handle). */
surr_status surr_adamw(surr_t s, float lr, float beta1, float beta2, float eps, float weight_decay);
/* surr_gradients + surr_adamw(lr, 0.9, 0.999, 1e-8, weight_decay). */
surr_status surr_train_step(surr_t s, const float* X_dev, const float* T_dev, int batch, float lr,
                            float weight_decay, double* loss_host);
/* Wait for the handle's stream.  SURR_ECUDA also when a tensor-core launch gave up waiting for its
 * matrix-multiply units (bounded wait; its output was left unwritten). */
surr_status surr_sync(surr_t s);

#ifdef __cplusplus
}
#endif
#endif
