/* Learned initial-pose proposal for AS-ICP: C-ABI of the network's CUDA kernels.
 *
 * The paper samples initial particles from a Fibonacci sphere, shows in its
 * ablation (Section VII, Fig. 3) that a mixture of Gaussians placed with prior
 * knowledge of the object reaches the same success rate with fewer particles,
 * and names learned initial poses as future work (Conclusions).  This library
 * provides that proposal: a PointNet-style encoder of the object cloud (shared
 * per-point MLP 3 -> 64 -> 128 -> 256, max-pool over points, MLP 256 -> 256 ->
 * P x 16 x 10) whose outputs parameterise, per preshape, a mixture of 16 SE(3)
 * densities (weights, translation means and isotropic spreads relative to the
 * cloud's centroid, Watson rotation densities: mean axis and concentration).
 * Weights and stored activations are bfloat16, products are accumulated in
 * float32; master weights, gradients and the Adam state are float32.
 *
 * Parameter layout (flat float32): W1 [64][3], b1 [64], W2 [128][64], b2 [128],
 * W3 [256][128], b3 [256], W4 [256][256], b4 [256], W5 [P*160][256], b5 [P*160].
 * Raw outputs per preshape p, component c (o[p][c][0..9]): logit, translation
 * mean / 0.1 m (3), log spread (sigma = 0.1 m exp(clip(o4, -4, 1))), rotation
 * (4, normalised), log concentration (kappa = 4 exp(clip(o9, -2, 3))).  Loss
 * of one object: mean over preshapes and target poses of -log p(target).
 *
 * Pointers may be host or device memory (copied with cudaMemcpyDefault) unless
 * stated otherwise; every call runs on the handle's stream and returns when its
 * outputs are complete.  Errors: INVALID_ARG (NULL handle or argument, sizes out
 * of range), CUDA (a failed CUDA call), OOM. */
#ifndef ASICP_PROPOSAL_H
#define ASICP_PROPOSAL_H

#include <stddef.h>

#include "asicp.h"

#ifdef __cplusplus
extern "C" {
#endif

#define ASICP_PROP_COMPONENTS 16
#define ASICP_PROP_RAW 10             /* raw outputs per component */
#define ASICP_PROP_MAX_TARGETS 128    /* target poses per preshape and object */

typedef struct asicp_prop asicp_prop;

/* Number of float32 parameters for P preshapes. */
size_t asicp_prop_num_params(int P);

/* A network for P preshapes (1..16) taking clouds of exactly n_points points
 * (16..65536), batches of up to max_batch objects (1..256).  Parameters start at
 * zero: set them with asicp_prop_set_params. */
asicp_status asicp_prop_create(int P, int n_points, int max_batch, void *cuda_stream, asicp_prop **out);
asicp_status asicp_prop_destroy(asicp_prop *prop);

/* Replace the float32 master parameters (flat layout above) and reset the Adam
 * state; read them back. */
asicp_status asicp_prop_set_params(asicp_prop *prop, const float *params);
asicp_status asicp_prop_get_params(asicp_prop *prop, float *params);

/* Raw mixture outputs out [B][P][16][10] and centroids [B][3] (may be NULL) of B
 * object clouds clouds [B][n_points][3]. */
asicp_status asicp_prop_forward(asicp_prop *prop, const float *clouds, int B, float *out, float *centroids);

/* Mean loss over the B objects of clouds [B][n_points][3] with target poses
 * targets [B][P][T][7] ((t, q) in the object frame, T <= ASICP_PROP_MAX_TARGETS),
 * and its gradient with respect to the parameters, kept for asicp_prop_adam_step.
 * *loss (host) receives the loss; grad (flat, may be NULL) a copy of the gradient. */
asicp_status asicp_prop_loss_grad(asicp_prop *prop, const float *clouds, const float *targets, int B, int T,
                                  float *loss, float *grad);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr on the
 * gradient of the last asicp_prop_loss_grad; the bfloat16 weights follow. */
asicp_status asicp_prop_adam_step(asicp_prop *prop, float lr);

/* Initial poses theta [B][P][K][7] sampled from the mixtures out [B][P][16][10]
 * around centroids [B][3] (both from asicp_prop_forward), with caller-drawn
 * random numbers draws [B][P][K][8] = (u uniform in [0, 1) choosing the component
 * by cumulative weight, then 7 standard normals): t = centroid + mu_c + sigma_c
 * (n1, n2, n3), q = normalise(nu_c + (n4..n7) / sqrt(2 kappa_c)).  theta may feed
 * asicp_run. */
asicp_status asicp_prop_sample(asicp_prop *prop, const float *out, const float *centroids, int B, int K,
                               const float *draws, float *theta);

#ifdef __cplusplus
}
#endif
#endif
