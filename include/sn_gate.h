/*
 * sn_gate.h -- learned boundary gate of libsn.so: trainer entry points.
 *
 * The paper's method is purely geometric (Sec. I-C notes that it is
 * differentiable apart from the adaptive support); this small network is an
 * addition that decides, per pixel, whether the full 9x9 window may be used
 * instead of the star-fill support.  q(p) estimates the probability that the
 * 5x5 patch centred at p is one valid surface:
 *   features f(p) (8 channels): log2(D(p + e_u)) - log2(D(p)) and
 *     log2(D(p + e_v)) - log2(D(p)) (0 where either pixel is invalid), the
 *     validity of p, five zeros;
 *   h1 = relu(conv3x3 8 -> 16), z = relu(conv3x3 16 -> 16),
 *   q = sigmoid(z . W3 + b3);
 *   gate(p) = min over the 5x5 neighbourhood of q >= tau, and the 9x9 window
 *   of p entirely valid.
 * Parameters (flat FP32 vector, sn_gate_param_count() floats, in this order):
 * W1 [16][9][8], b1 [16], W2 [16][9][16], b2 [16], W3 [16], b3 [1]; conv
 * taps t = (o_v + 1) * 3 + (o_u + 1).  Contractions run on tensor cores in
 * BF16 with FP32 accumulation; master weights and Adam state are FP32.
 *
 * Training samples are 6x6 patches of integer disparity codes
 * (int32 [B][36], row-major, centre at [2][2], 0 = invalid) with labels in
 * {0, 1} (float [B]); all pointers below are device pointers unless stated.
 */
#ifndef SN_GATE_H
#define SN_GATE_H

#include "sn.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sn_gate_trainer sn_gate_trainer;

/* Number of floats of the parameter vector. */
int sn_gate_param_count(void);

/* Allocates a trainer for batches of at most max_batch samples, starting
 * from theta0 (HOST, sn_gate_param_count floats). */
sn_status sn_gate_trainer_create(int max_batch, const float *theta0, sn_gate_trainer **out);
sn_status sn_gate_trainer_destroy(sn_gate_trainer *t);

/* Forward pass (q [B], may be NULL) and, when y is not NULL, the mean binary
 * cross-entropy (loss, 1 float) and its gradient (grad, sn_gate_param_count
 * floats) at the current weights.  Asynchronous on `stream`. */
sn_status sn_gate_trainer_grad(sn_gate_trainer *t, const int32_t *patches, const float *y, int B, float *grad,
                               float *q, float *loss, sn_stream stream);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on the batch; loss (device,
 * may be NULL) receives the batch loss before the step. */
sn_status sn_gate_trainer_step(sn_gate_trainer *t, const int32_t *patches, const float *y, int B, float lr,
                               float *loss, sn_stream stream);

/* Checkpoint: copies master weights, Adam moments (HOST arrays, may be NULL)
 * and the step count out; resume puts them back.  Synchronous. */
sn_status sn_gate_trainer_state(sn_gate_trainer *t, float *theta, float *m, float *v, long long *step);
sn_status sn_gate_trainer_resume(sn_gate_trainer *t, const float *theta, const float *m, const float *v,
                                 long long step);

/* Waits for `stream`, then reads and clears the trainer's device error word:
 * SN_ETIMEOUT if a bounded wait of a tensor-core GEMM gave up since the last
 * check (the gradients and steps of those calls are undefined), else SN_OK. */
sn_status sn_gate_trainer_check_device(sn_gate_trainer *t, sn_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* SN_GATE_H */
