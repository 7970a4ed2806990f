/*
 * gbs_surrogate.h -- C ABI of the learned surrogate of the binned
 * total-count distribution (companion of gbs.h; same status codes and
 * conventions: every call returns a status, gbs_last_error() holds the
 * message, host buffers belong to the caller).
 *
 * The paper has no surrogate.  It computes P(m) -- the binned total-count
 * distribution of Eq. total_counts for squeezed inputs through T = t U
 * ("Applications to GBS") -- by the matrix-P ensemble; this library's
 * surrogate is a small multilayer perceptron that maps a network's
 * parameters to that distribution, trained on distributions the ensemble
 * itself produced, with the ensemble kept as its fallback and as the judge
 * of its error.
 *
 * Representation (shared by the feature, encode and decode calls):
 *   features u (10 doubles per network): ln N, ln M, mean r, std r
 *     (population), min r, max r, t, log2 K1, ln mu, ln s, where mu and s
 *     are the closed-form mean and standard deviation of the total count for
 *     T = t U (from the uniform-loss determinant generating function):
 *       mu  = t^2 sum_j sinh^2 r_j,
 *       s^2 = sum_j [t^2 sinh^2 r_j + t^4 sinh^2 r_j cosh 2 r_j];
 *     the feature record of a network holds 14 doubles: u[0..9], mu, s and
 *     its count window m_off, K1 (counts m_off .. m_off + K1 - 1).
 *   output o (512 floats per network): channel p = 0 (even counts) and
 *     p = 1 (odd counts), 256 values each, on the grid
 *     x_i = -8 + 16 (i + 1/2) / 256 of the standardised count x = (m - mu)/s:
 *       o[p*256 + i] = 100 (f_p(x_i) - phi(x_i)/2),
 *     f_p the density per unit x of the counts of parity p, phi the standard
 *     normal density.  Interpolation is Catmull-Rom cubic in both directions.
 *
 * MLP: layers l = 1..L, y_l = W_l h_{l-1} + b_l, h_l = silu(y_l) (l < L),
 * output y_L; loss (1/(B O)) sum (y_L - target)^2; Adam (Kingma & Ba 2015)
 * with beta1 = 0.9, beta2 = 0.999, eps = 1e-8.  Weights are kept as FP32
 * master copies; every product uses their BF16 rounding (nearest-even) on
 * the tcgen05 tensor cores with FP32 accumulation.  Activations and
 * gradients enter the products as two BF16 planes (hi + lo, ~16 significant
 * bits); biases stay FP32.
 */
#ifndef GBS_SURROGATE_H
#define GBS_SURROGATE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gbs_mlp *gbs_mlp_t;

#define GBS_SUR_FEATURES 10  /* features per network */
#define GBS_SUR_RECORD 14    /* doubles per feature record: u[10], mu, s, m_off, K1 */
#define GBS_SUR_GRID 256     /* grid points per parity channel */
#define GBS_SUR_OUT 512      /* outputs per network */

/*
 * gbs_mlp_create -- an MLP in_dim -> width -> ... -> width -> out_dim with
 * `layers` weight layers (layers >= 2), for batches of up to max_batch rows.
 *   in_dim    1..32;  width, out_dim: multiples of 256, <= 4096.
 *   max_batch 1..65536.
 *   stream    cudaStream_t (as void*) for all work of this object; NULL makes
 *             the object create (and own) a non-blocking stream.
 * Parameters start at zero (set them with gbs_mlp_set_params).  The device
 * memory is owned by the object until gbs_mlp_free.
 * Errors: EINVAL, ENOMEM, ECUDA, ENOTSUP (device without tcgen05).
 */
int gbs_mlp_create(int in_dim, int width, int out_dim, int layers, int max_batch, void *stream,
                   gbs_mlp_t *out);

/* Number of parameters in the packed layout of gbs_mlp_set_params. */
int gbs_mlp_param_count(gbs_mlp_t mlp, int64_t *count);

/*
 * gbs_mlp_set_params / gbs_mlp_get_params -- host FP32 parameters packed as
 * [W_1 (width x in_dim, row-major) | b_1 (width) | W_2 (width x width) | b_2 |
 *  ... | W_L (out_dim x width) | b_L (out_dim)].  Setting also clears the
 * Adam moments and step counter and refreshes the BF16 weight copies.
 * Both synchronise the object's stream.  Errors: EINVAL (non-finite value),
 * ECUDA.
 */
int gbs_mlp_set_params(gbs_mlp_t mlp, const float *params);
int gbs_mlp_get_params(gbs_mlp_t mlp, float *params);

/* Adam first and second moments (host, packed layout; either may be NULL)
 * and the number of Adam steps taken.  Synchronises. */
int gbs_mlp_get_adam_state(gbs_mlp_t mlp, float *m, float *v, int64_t *step);

/*
 * gbs_mlp_forward -- Y = MLP(X) for `batch` rows.
 *   X_dev  device, [batch][in_dim] FP32;  Y_dev device, [batch][out_dim] FP32.
 * Asynchronous on the object's stream.  Errors: EINVAL (batch out of range).
 */
int gbs_mlp_forward(gbs_mlp_t mlp, const float *X_dev, int batch, float *Y_dev);

/*
 * gbs_mlp_gradients -- loss and its gradient for one batch, no update.
 *   T_dev  device, [batch][out_dim] FP32 targets.
 *   loss   host, receives the mean squared error (may be NULL).
 *   grad   host, packed layout (may be NULL).
 * Synchronises.  Errors: EINVAL, ECUDA, ETIMEOUT.
 */
int gbs_mlp_gradients(gbs_mlp_t mlp, const float *X_dev, const float *T_dev, int batch,
                      double *loss, float *grad);

/*
 * gbs_mlp_train -- `steps` full-batch Adam steps on (X_dev, T_dev):
 * forward, loss, backward and update per step, captured once as a CUDA
 * graph and replayed.  lr: host, `steps` learning rates (step i uses lr[i]).
 * loss_hist: host, receives the loss before each step (may be NULL).
 * Synchronises.  Errors: EINVAL, ECUDA, ETIMEOUT.
 */
int gbs_mlp_train(gbs_mlp_t mlp, const float *X_dev, const float *T_dev, int batch, int steps,
                  const float *lr, float *loss_hist);

void gbs_mlp_free(gbs_mlp_t mlp);

/*
 * gbs_surrogate_features -- feature records of `count` networks.
 *   N, M, K1   host, count ints each (N >= 1, K1 a power of two <= 2^24).
 *   m_off      host, count window starts (>= 0).
 *   t          host, count amplitude transmissions in (0, 1].
 *   r, r_off   host: the squeezing parameters of network i are
 *              r[r_off[i] .. r_off[i+1]-1] (r_off has count+1 entries,
 *              r_off[i+1] - r_off[i] = N[i]); each r_j finite and > 0.
 *   feat_dev   device, [count][14] doubles (the feature records).
 * Uploads r on the stream, then computes on the GPU.  Synchronises the
 * stream before returning (the upload buffer is released).
 * Errors: EINVAL, ENOMEM, ECUDA.
 */
int gbs_surrogate_features(int count, const int *N, const int *M, const double *t, const int *K1,
                           const int64_t *m_off, const double *r, const int64_t *r_off, void *stream,
                           double *feat_dev);

/*
 * gbs_surrogate_feature_stats -- per feature, over `count` records:
 * stats_dev[0][f] = mean, [1][f] = standard deviation (population),
 * [2][f] = min, [3][f] = max (device, 4 x 10 doubles).  Asynchronous.
 */
int gbs_surrogate_feature_stats(int count, const double *feat_dev, void *stream,
                                double *stats_dev);

/*
 * gbs_surrogate_standardize -- network inputs X = (u - mean) / std (FP32,
 * [count][10]; a feature with std <= 1e-12 maps to 0) from the statistics
 * of gbs_surrogate_feature_stats (device, 4 x 10 doubles); in_domain_dev
 * (device, count ints, may be NULL) receives 1 where every feature lies in
 * [min - 0.02 (max - min), max + 0.02 (max - min)], else 0.  Asynchronous.
 */
int gbs_surrogate_standardize(int count, const double *feat_dev, const double *stats_dev,
                              void *stream, float *X_dev, int *in_domain_dev);

/*
 * gbs_surrogate_encode -- targets o (see the header comment) of `count`
 * distributions.  P_dev: device, network i's P(m) on the window of its
 * feature record at P_dev + i * ldP (ldP >= every K1).  Y_dev: device,
 * [count][512] FP32.  Asynchronous.  Errors: EINVAL.
 */
int gbs_surrogate_encode(int count, const double *feat_dev, const double *P_dev, int64_t ldP,
                         void *stream, float *Y_dev);

/*
 * gbs_surrogate_decode -- distributions from outputs: network i's P(m) on
 * the window of its feature record, renormalised to sum 1, into
 * P_dev + i * ldP (device, ldP >= every K1).  Y_dev: device, [count][512].
 * Asynchronous.  Errors: EINVAL.
 */
int gbs_surrogate_decode(int count, const double *feat_dev, const float *Y_dev, void *stream,
                         double *P_dev, int64_t ldP);

#ifdef __cplusplus
}
#endif

#endif /* GBS_SURROGATE_H */
