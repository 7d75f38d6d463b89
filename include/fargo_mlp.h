/* C ABI of the surrogate network of the batched disk sweep: a multilayer
 * perceptron with ReLU hidden layers and a linear output, trained on the
 * GPU with a mean-squared-error loss and Adam (Kingma & Ba 2015).  The
 * paper has no counterpart; the network maps disk parameters and an
 * initial radial profile to the azimuthally averaged surface density the
 * solver reaches after a fixed number of orbits, and the solver stays the
 * fallback and the judge of its error.
 *
 * Arithmetic: weights, the network input, hidden activations and the
 * back-propagated gradients that feed the products are bfloat16 (round to
 * nearest even); every product runs on the fifth-generation tensor cores
 * (tcgen05, accumulator in tensor memory) and accumulates in FP32;
 * biases, pre-activations, the output, the loss, the gradients and the
 * Adam state (master weights, first and second moments) are FP32.
 *
 * Parameter vector layout (FP32, n = fargo_mlp_num_params): for each layer
 * l = 0 .. L-1 the weights W_l, dims[l+1] rows of dims[l] values (row-major),
 * then the biases b_l (dims[l+1] values).  Gradients use the same layout.
 *
 * Buffers: x, t and y are device pointers to FP32 row-major
 * [batch][dims[0]] / [batch][dims[L]] arrays on the network's device.  All
 * calls queue work on the network's stream and return without host
 * synchronisation unless stated.  Errors: FARGO_ERR_BADARG (NULL, sizes),
 * FARGO_ERR_SIZE (batch above max_batch or a wrong element count),
 * FARGO_ERR_OOM, FARGO_ERR_CUDA (codes of fargo.h). */
#ifndef FARGO_MLP_H
#define FARGO_MLP_H
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fargo_mlp fargo_mlp;

/* dims[0..nlayers]: layer widths (input, hidden..., output), each 1..4096,
 * nlayers in 1..16.  max_batch: the largest batch of any later call.
 * stream: cudaStream_t (NULL = a stream the network creates and owns).
 * Parameters start at zero; Adam's step counter at zero. */
int fargo_mlp_create(fargo_mlp **out, const int *dims, int nlayers, int max_batch, void *stream);
void fargo_mlp_destroy(fargo_mlp *net);
size_t fargo_mlp_num_params(const fargo_mlp *net);

/* Copy the FP32 parameter vector in (host, n values; also rounds the
 * bfloat16 weight copies and clears the Adam moments and step counter) or
 * out.  Synchronise. */
int fargo_mlp_set_params(fargo_mlp *net, const float *host, size_t n);
int fargo_mlp_get_params(fargo_mlp *net, float *host, size_t n);
/* FP32 gradients of the last fargo_mlp_backward (host, n values). Synchronises. */
int fargo_mlp_get_grads(fargo_mlp *net, float *host, size_t n);

/* Input map applied before the first layer: x' = (x - shift) * scale per
 * input feature (host arrays of dims[0] values; default 0 and 1).
 * Synchronises. */
int fargo_mlp_set_input_map(fargo_mlp *net, const float *shift, const float *scale);

/* Output map applied after the last layer: y = z * scale + shift per output
 * (host arrays of dims[L] values; default 0 and 1).  The loss compares y
 * with the targets, so its gradient with respect to z carries the scale.
 * Synchronises. */
int fargo_mlp_set_output_map(fargo_mlp *net, const float *shift, const float *scale);

/* Adam hyper-parameters read by every later fargo_mlp_adam (default
 * lr 1e-3, b1 0.9, b2 0.999, eps 1e-8).  Synchronises. */
int fargo_mlp_set_optimizer(fargo_mlp *net, float lr, float b1, float b2, float eps);

/* Inference: y = f(x) for `batch` samples. */
int fargo_mlp_forward(fargo_mlp *net, const float *x, int batch, float *y);

/* Forward pass, mean-squared-error loss against targets t, and the
 * gradient of that loss (the mean over batch * dims[L] squared errors)
 * into the network's gradient vector.  loss (device pointer to one float,
 * may be NULL) receives the loss. */
int fargo_mlp_backward(fargo_mlp *net, const float *x, const float *t, int batch, float *loss);

/* One Adam step with the current gradients: the step counter advances,
 * the FP32 master weights update and the bfloat16 copies are re-rounded. */
int fargo_mlp_adam(fargo_mlp *net);

/* fargo_mlp_backward then fargo_mlp_adam, replayed from a CUDA graph that is
 * captured on the first call with a given (x, t, batch, loss). */
int fargo_mlp_train_step(fargo_mlp *net, const float *x, const float *t, int batch, float *loss);

/* Synchronise and report a product that gave up waiting for its tensor-core
 * work (FARGO_ERR_BARRIER_TIMEOUT), else OK.  The flag stays set. */
int fargo_mlp_status(fargo_mlp *net);

/* Deep-ensemble statistics of k outputs stacked as ys[k][batch][n] (device):
 * mean[batch][n] and, per sample, the relative spread
 * |sample standard deviation over members|_2 / |mean|_2 (spread[batch]).
 * k >= 2.  Queued on `stream` (NULL = legacy default stream). */
int fargo_mlp_ensemble(const float *ys, int k, int batch, int n, float *mean, float *spread, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FARGO_MLP_H */
