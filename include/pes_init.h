/*
 * pes_init.h — C ABI of the learned initialiser of the iterated smoother.
 *
 * The paper starts its iteration (Sec. 3) from a nominal trajectory that it
 * leaves open; the plain choice, every state at its prior mean (x_init = NULL
 * in pes_ieks_run), stays the fallback. This library adds a small network
 * that maps the measurements of each trajectory to an initial nominal
 * x_init [5][N] for pes_ieks_run, trained on trajectories that the FP64
 * smoother itself has converged, so that fewer iterations are needed. The
 * paper has no counterpart; the smoother's results at convergence do not
 * depend on it.
 *
 * The network, for one trajectory with states k = 0..T (measurements at
 * k >= 1, the layout of pes.h):
 *   features  phi_k = (sin y_k^1, cos y_k^1, sin y_k^2, cos y_k^2, 1, 0, 0...)
 *             for k >= 1, (0, 0, 0, 0, 0, 1, 0...) at k = 0 (64 channels);
 *   4 conv    h_l[k] = relu(b_l + sum_{j<5} W_l[:, :, j] h_{l-1}[k + j - 2]),
 *   layers    64 -> 64 channels, zero outside 0..T;
 *   MLP head  z_k = relu(W5 h_4[k] + b5), o_k = W6 z_k + b6 (64 -> 64 -> 5);
 *   output    x_init[c][k] = mu_c + sigma_c * o_k[c].
 * Weights, features and hidden activations are bfloat16, accumulation is FP32
 * on the tensor cores (tcgen05); o is FP32. Parameters live on the device as
 * an FP32 master vector of PES_INIT_NPARAMS floats, packed in this order:
 * for l = 1..4, W_l [64][64][5] (output channel, input channel, tap), b_l [64];
 * W5 [64][64], b5 [64]; W6 [5][64], b6 [5].
 *
 * Training minimises the mean of (o_k[c] - (x*_k[c] - mu_c) / sigma_c)^2 over
 * the states and components of a minibatch, x* the converged smoother means,
 * with Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).
 *
 * Conventions: trajectories, offsets (DEVICE memory), y [2][N] and the
 * component-major layout are those of pes.h. PES_FP32 takes float arrays,
 * PES_FP64 double arrays (y, x_target, x_init); parameters are always float.
 * Every call enqueues on `stream` (cudaStream_t as void*); a call that returns
 * a host value (loss) synchronises the stream first. Arguments are checked
 * before anything is launched (PES_ERR_INVALID_ARG). Calls on one net must
 * not overlap in time (they share its workspace).
 */
#ifndef PES_INIT_H
#define PES_INIT_H

#include <stdint.h>

#include "pes.h"

#ifdef __cplusplus
extern "C" {
#endif

#define PES_INIT_NPARAMS 86661

typedef struct pes_init_net pes_init_net;

/* Create a net with workspace for up to max_states states in up to max_batch
 * trajectories per call (about 1.3 KB per state for training). Parameters
 * start at zero, mu = 0 and sigma = 1; set them with pes_init_set_params. */
pes_status pes_init_create(pes_init_net** out, int64_t max_states, int32_t max_batch);
pes_status pes_init_destroy(pes_init_net* net);
const char* pes_init_last_error(const pes_init_net* net);

/* Copy parameters in (HOST float [PES_INIT_NPARAMS]) and set the output
 * normalisation mu, sigma (HOST double [5], sigma > 0); resets Adam's moments
 * and step count. Synchronous. */
pes_status pes_init_set_params(pes_init_net* net, const float* params, const double* mu, const double* sigma);

/* Copy the current FP32 master parameters out (HOST float [PES_INIT_NPARAMS]).
 * Synchronous. */
pes_status pes_init_get_params(pes_init_net* net, float* params);

/* The training state, for checkpointing a run and resuming it: the FP32 master
 * parameters (HOST float [PES_INIT_NPARAMS]), the output normalisation mu,
 * sigma (HOST double [5]), Adam's first and second moments (HOST float
 * [PES_INIT_NPARAMS] each) and its step count. pes_init_get_state copies them
 * out (any pointer may be NULL to skip that part); pes_init_set_state copies
 * them in (all required; sigma > 0, moments finite, v >= 0, adam_t >= 0) and
 * republishes the layers' bfloat16 weights, so that the next
 * pes_init_train_step continues the saved run exactly. Both synchronise the
 * device. */
pes_status pes_init_get_state(pes_init_net* net, float* params, double* mu, double* sigma, float* adam_m,
                              float* adam_v, int64_t* adam_t);
pes_status pes_init_set_state(pes_init_net* net, const float* params, const double* mu, const double* sigma,
                              const float* adam_m, const float* adam_v, int64_t adam_t);

/* Inference: x_init [5][N] (component-major, float or double per `prec`) for
 * the B trajectories in y / offsets. */
pes_status pes_init_forward(pes_init_net* net, pes_precision prec, const void* y, const int64_t* offsets, int32_t B,
                            int64_t N, void* x_init, void* stream);

/* Loss of the minibatch against x_target [5][N] and its gradient, written to
 * grad (DEVICE float [PES_INIT_NPARAMS], packed like the parameters); *loss
 * (HOST) receives the loss when not NULL (the call then synchronises). The
 * parameters do not change. */
pes_status pes_init_loss_grad(pes_init_net* net, pes_precision prec, const void* y, const int64_t* offsets,
                              int32_t B, int64_t N, const void* x_target, float* grad, double* loss, void* stream);

/* One training step: the gradient of pes_init_loss_grad, then one Adam update
 * of the parameters with learning rate lr. *loss as above. */
pes_status pes_init_train_step(pes_init_net* net, pes_precision prec, const void* y, const int64_t* offsets,
                               int32_t B, int64_t N, const void* x_target, float lr, double* loss, void* stream);

#ifdef __cplusplus
}
#endif

#endif
