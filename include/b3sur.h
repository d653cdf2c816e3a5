/*
 * b3sur.h -- C ABI of the learned fitness surrogate (BF16 MLP on tensor cores).
 *
 * What it computes.  In the paper's setting (Sec. 1: memetic and Lamarckian
 * evolution of robot morphologies and controllers, where every evaluation is
 * a physics simulation and, per Sec. 3, over 80 % of the run time is
 * simulation) a small network pre-screens offspring so that only the most
 * promising are simulated.  The network maps a 128-d genotype encoding to a
 * predicted fitness:
 *     y = W3 relu(W2 relu(W1 x + b1) + b2) + b3,   128 -> 256 -> 256 -> 1,
 * with BF16 weights and activations and FP32 accumulation (tensor cores).
 * Training minimises the mean squared error on standardised targets with
 * Adam (Kingma & Ba 2015) on FP32 master weights; the BF16 weights are
 * refreshed from the master copy after every update.
 *
 * Genotype encoding (128 floats per robot): for brick slots i = 0..19 (brick
 * i is body i + 1): present, parent / 20, face / 5, rotation / 3, CPG weight;
 * then the coupling weights of bricks 2..20 (slots 100..118); zeros after.
 *
 * Ownership: the context owns all device memory; host arrays belong to the
 * caller and are only read or written during the call.  Every call returns a
 * sur_status; sur_last_error() explains the last failure.  One context per
 * host thread.  Work runs on the context's stream; the calls below
 * synchronise before returning.
 */
#ifndef B3SUR_H
#define B3SUR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sur_ctx sur_ctx_t;

#define SUR_IN_DIM 128
#define SUR_HIDDEN 256
#define SUR_MAX_BATCH 65536
#define SUR_MAX_TOPK 8192

typedef enum { SUR_OK = 0, SUR_EINVAL = -1, SUR_ECUDA = -2, SUR_ENOMEM = -3 } sur_status;

typedef struct {
    uint64_t seed;       /* weight initialisation and shuffling             */
    float lr;            /* Adam step size                                  */
    float beta1, beta2;  /* Adam moment decay rates                         */
    float eps;           /* Adam denominator offset                         */
    int32_t device;      /* CUDA device ordinal                             */
    uint64_t stream;     /* cudaStream_t or 0 (the context creates one)     */
} sur_config;

/* Number of parameters: 256*128 + 256 + 256*256 + 256 + 256 + 1 (W1, b1, W2,
 * b2, W3, b3 in that order, row-major, as in sur_get_params). */
#define SUR_NPARAMS (SUR_HIDDEN * SUR_IN_DIM + SUR_HIDDEN + SUR_HIDDEN * SUR_HIDDEN + SUR_HIDDEN + SUR_HIDDEN + 1)

/* Create a context; weights He-uniform from cfg->seed, biases zero. */
int sur_create(const sur_config* cfg, sur_ctx_t** out);
int sur_destroy(sur_ctx_t* ctx);

/* Encode n robots on the GPU into X_out (n x 128 floats, host): the bricks'
 * zero-pose geometry and controller weights.  Per robot, arrays of 32 body
 * slots (body 0 = the core, parent[b] < b): parent, hinge axis index in the
 * body frame (0..2), joint frame R_fix (9 floats, row-major) and p_fix (3,
 * metres) in the parent frame, box centre in the body frame (3, metres), CPG
 * weight and coupling weight (to the parent's hinge); n_bodies in 1..21.
 * Joint frames are taken on the integer millimetre lattice the robots are
 * built on: R_fix rounded to its integer entries (a signed permutation),
 * offsets and centres rounded to whole millimetres.  Zero-pose kinematics
 * then place every brick exactly; the bricks are ordered by box centre in
 * the core frame (z, then x, then y) and brick i fills columns 6i .. 6i+5
 * with (x, y, z) / 256 mm, its hinge axis code (1, 2, 3: along the core's
 * x, y, z) / 3, its CPG weight, and its coupling weight (0 when its parent
 * is the core); columns 120..127 and unused slots are zero.  A paper-silent
 * reading: the paper defines no encoding.  Returns SUR_EINVAL on NULL
 * arrays, n < 1, n_bodies outside 1..21, a parent not before its child or
 * an axis outside 0..2. */
int sur_encode(sur_ctx_t* ctx, const int8_t* parent, const int8_t* axis, const float* R_fix, const float* p_fix,
               const float* box_center, const float* w_int, const float* w_cpl, const int32_t* n_bodies, int32_t n,
               float* X_out);

/* Train `epochs` passes over (X, y) (n x 128, n) in shuffled mini-batches of
 * `batch` (1..SUR_MAX_BATCH).  Targets are standardised with their mean and
 * standard deviation over this call's data, which sur_predict undoes.
 * *loss_out (may be NULL) gets the mean standardised loss of the last epoch. */
int sur_train(sur_ctx_t* ctx, const float* X, const float* y, int32_t n, int32_t epochs, int32_t batch,
              float* loss_out);

/* Predicted fitness of n robots (X: n x 128) into y_out (n). */
int sur_predict(sur_ctx_t* ctx, const float* X, int32_t n, float* y_out);

/* Indices of the k largest of n scores (1 <= k <= SUR_MAX_TOPK, k <= n),
 * ties to the lower index, ordered by descending score. */
int sur_topk(sur_ctx_t* ctx, const float* scores, int32_t n, int32_t k, int32_t* idx_out);

/* Gradients of the mean squared error on the raw targets y (no
 * standardisation) for one batch of n (<= SUR_MAX_BATCH) at the current
 * weights, packed like the parameters (SUR_NPARAMS floats); *loss_out gets
 * the loss.  No update is made. */
int sur_gradients(sur_ctx_t* ctx, const float* X, const float* y, int32_t n, float* grads, float* loss_out);

/* One Adam update on one batch (raw targets, as sur_gradients). */
int sur_train_step(sur_ctx_t* ctx, const float* X, const float* y, int32_t n, float* loss_out);

/* FP32 master parameters (SUR_NPARAMS floats, W1 b1 W2 b2 W3 b3), read and
 * replaced (replacing also resets the Adam moments and step count and the
 * target standardisation to mean 0, scale 1). */
int sur_get_params(sur_ctx_t* ctx, float* params);
int sur_set_params(sur_ctx_t* ctx, const float* params);

const char* sur_last_error(const sur_ctx_t* ctx);

#ifdef __cplusplus
}
#endif
#endif
