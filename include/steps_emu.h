/*
 * steps_emu.h -- C ABI of the correlation-function emulator.
 *
 * The simulations are run for the statistics of the density field (Sec. 1;
 * opening of Sec. 3).  The emulator is a small network that maps the
 * cosmological parameters and a separation to the central sphere's
 * correlation function, trained on the exact pair counts of batched runs
 * (steps_paircount), so that a parameter fit can query it instead of running
 * a simulation.  The paper trains no network: architecture and optimiser are
 * this library's, stated here.
 *
 * Network: 5 inputs -> 256 -> 256 -> 256 -> 1 output, SiLU (z * sigmoid(z))
 * after each hidden layer, linear output.  Loss: mean over the batch of
 * (y - t)^2.  Optimiser: Adam with bias correction, beta1 0.9, beta2 0.999,
 * eps 1e-8, the learning rate given per step.
 *
 * Arithmetic: every matrix-product operand is bfloat16, rounded to nearest
 * even -- the inputs, the weights, each hidden activation after the SiLU and
 * each back-propagated dL/dz -- and the products are summed in FP32 on the
 * tensor cores.  Biases, bias gradients (sums of the unrounded FP32 dL/dz),
 * the FP32 master weights and the Adam moments are never rounded to bfloat16.
 *
 * Parameters are exchanged packed in FP32, in this order:
 *   W1[256][5], b1[256], W2[256][256], b2[256], W3[256][256], b3[256],
 *   W4[1][256], b4[1]                       (STEPS_EMU_NPARAMS values)
 * where layer l computes z = a W^T + b.
 *
 * Every call returns a status (steps.h) and never aborts; pointers marked
 * "host or device" are classified by the library.  The context owns its
 * device memory until steps_emu_free and uses the stream given at creation.
 */
#ifndef STEPS_EMU_H
#define STEPS_EMU_H

#include <stdint.h>

#include "steps.h"

#ifdef __cplusplus
extern "C" {
#endif

#define STEPS_EMU_IN 5
#define STEPS_EMU_WIDTH 256
#define STEPS_EMU_NPARAMS 133377

typedef struct steps_emu steps_emu;

/*
 * Create an emulator with initial parameters params [STEPS_EMU_NPARAMS]
 * (host).  batch = rows per training step, a multiple of 64 in [64, 4096].
 * EINVAL on a bad batch or a non-finite parameter.
 */
steps_status steps_emu_create(steps_emu **out, const float *params, int batch, void *cuda_stream);

/*
 * Copy the training set: x [n][5] features, t [n] targets (host or device,
 * FP32).  Replaces any earlier set.  EINVAL on n < 1 or non-finite values.
 */
steps_status steps_emu_set_data(steps_emu *e, int64_t n, const float *x, const float *t);

/*
 * nsteps Adam steps.  Step s trains on the rows rows[s][0 .. batch) of the
 * training set (host, each in [0, n), else EINVAL) with learning rate lr[s]
 * (host).  loss_out [nsteps] (host, may be NULL) receives each step's loss
 * before its update.  One step is captured once as a CUDA graph and replayed.
 */
steps_status steps_emu_train(steps_emu *e, int nsteps, const int32_t *rows, const float *lr,
                             float *loss_out);

/*
 * Network outputs y [n] for inputs x [n][5] (host or device), in chunks of the
 * batch size.  n = 0 is a no-op.
 */
steps_status steps_emu_predict(steps_emu *e, int64_t n, const float *x, float *y);

/*
 * Loss and gradients, packed like the parameters, of one batch x [batch][5],
 * t [batch] (host) at the current parameters, without an update.
 */
steps_status steps_emu_gradients(steps_emu *e, const float *x, const float *t, float *grads,
                                 float *loss);

/*
 * Current FP32 master parameters and Adam moments, packed (host; any pointer
 * may be NULL), and the number of Adam steps taken.
 */
steps_status steps_emu_get_params(steps_emu *e, float *params, float *adam_m, float *adam_v,
                                  int64_t *adam_steps);

void steps_emu_free(steps_emu *e);

#ifdef __cplusplus
}
#endif

#endif /* STEPS_EMU_H */
