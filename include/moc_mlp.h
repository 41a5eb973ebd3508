/*
 * moc_mlp.h -- C ABI of the learned warm start of the GB300 MOC library: a small multilayer
 * perceptron trained on the library's own converged solutions, mapping per-region features
 * (the region's cross sections, geometry descriptors and the instance's cross-section
 * perturbation) to the region's log scalar flux per group and an estimate of k.
 *
 * The paper has no counterpart: it is an added pattern on top of the paper's power iteration
 * (the fine-mesh MOC solve of Alg. 1), whose converged plain solve remains the reference for the
 * result; the cold start (flat flux, k = 1) stays the fallback.
 *
 * Network: n_layers = 4 linear layers, n_in -> width -> width -> width -> n_out, SiLU after the
 * first three. Weights are used in bf16 with FP32 accumulation; FP32 master weights are updated by
 * Adam. Inputs and targets are standardised with per-column mean/std set by the caller.
 *
 * Conventions: as in moc_gb300.h (status codes, caller-owned host arrays copied during the call).
 * The *_dev arguments are device pointers on the network's device, owned by the caller and
 * valid until the work enqueued on `stream` (a cudaStream_t, NULL = legacy default) completes.
 */
#ifndef MOC_MLP_H
#define MOC_MLP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct moc_mlp moc_mlp;

/* Create a network on `device` with random (seeded) Glorot-uniform weights and zero biases.
 * 1 <= n_in, n_out <= 1024; width in {32, 64, 128, 256, 512}. Errors: MOC_ERR_ARG, MOC_ERR_CUDA. */
int moc_mlp_create(moc_mlp **out, int device, int n_in, int width, int n_out, uint64_t seed);
void moc_mlp_destroy(moc_mlp *net);
const char *moc_mlp_last_error(const moc_mlp *net);

/* Number of parameters and the layer sizes (dims[5] = n_in, width, width, width, n_out). */
int moc_mlp_dims(const moc_mlp *net, int *dims, int64_t *n_params);

/* FP32 master weights in one flat host array: for each layer l, W_l [dims[l+1]][dims[l]] then
 * b_l [dims[l+1]]. set_params also refreshes the bf16 copies and resets the Adam moments. */
int moc_mlp_get_params(moc_mlp *net, float *params);
int moc_mlp_set_params(moc_mlp *net, const float *params);

/* Standardisation: x_norm = (x - in_mean)/in_std, y = y_norm * out_std + out_mean. */
int moc_mlp_set_normalization(moc_mlp *net, const float *in_mean, const float *in_std,
                              const float *out_mean, const float *out_std);

/* y_dev [n][n_out] = network(x_dev [n][n_in]) in de-standardised units. Asynchronous. */
int moc_mlp_forward(moc_mlp *net, const float *x_dev, float *y_dev, int64_t n, void *stream);

/* One Adam step on the mean squared error of the standardised outputs over a batch x_dev
 * [n][n_in], y_dev [n][n_out] (targets in de-standardised units). loss_out (may be NULL) gets the
 * batch loss before the update (synchronises when not NULL). */
int moc_mlp_train_step(moc_mlp *net, const float *x_dev, const float *y_dev, int64_t n, float lr,
                       float *loss_out, void *stream);

/* Gradients of the batch loss with respect to every parameter (flat layout of get_params) and the
 * loss, without updating anything: for checking the backward pass. Synchronous. */
int moc_mlp_gradients(moc_mlp *net, const float *x_dev, const float *y_dev, int64_t n, float *grad_out,
                      float *loss_out, void *stream);

/* Forward pass that allocates nothing, for callers that must not call cudaMalloc: code that runs
 * while a stream is being captured into a CUDA graph (an allocation there breaks the capture),
 * solvers that hand all device memory to their own pool up front and treat a driver allocation in
 * the solve loop as an error, and latency-bound loops where an allocation's implicit device
 * synchronisation is not acceptable. The paper has no counterpart.
 *
 * Same contract and result as moc_mlp_forward, except that the activations live in one fixed
 * workspace of MOC_MLP_NOALLOC_FLOATS floats (8 MiB) that the library declares as a static
 * device array: every GPU that loads the library holds it until the process exits. A call needs
 * n * (dims[0] + 2 dims[1] + 2 dims[2] + 2 dims[3] + dims[4]) floats of it and returns MOC_ERR_ARG
 * (touching nothing) when n is larger; split bigger batches. All calls on a device share the one
 * array and it keeps the last call's contents, so calls whose GPU work overlaps (other streams,
 * other threads) race and must be serialised by the caller. The first call on a device looks up
 * the array's device address (no allocation) and should come before any stream capture. */
#define MOC_MLP_NOALLOC_FLOATS (2u * 1024u * 1024u)
int moc_mlp_forward_noalloc(moc_mlp *net, const float *x_dev, float *y_dev, int64_t n, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MOC_MLP_H */
