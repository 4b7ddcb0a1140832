/* Learned warm start for the constrained DTT solver: a small 3-D convolutional
 * encoder-decoder that maps a cell's phase map, boundary/constraint masks and load to a
 * first guess of u~, trained on fields the solver produces.
 *
 * The paper only names this as a prospect (reducing iteration counts through better
 * initialisation, Section 5.4 and the conclusion); the network is this library's own.
 * Its forward and backward passes run in hand-written BF16 implicit-GEMM convolution
 * kernels with FP32 accumulation; master weights and the Adam optimiser are FP32.
 *
 * Network (node grid of the cell, channels last, 3x3x3 convolutions with zero padding,
 * bias; c1/c2/c3 channels at full, 1/2 and 1/4 resolution; "pool" = mean over 2x2x2 blocks,
 * partial at odd edges; "up" = nearest-neighbour back to the finer size):
 *   e1 = relu(conv(relu(conv(x))))             16 -> c1 -> c1
 *   e2 = relu(conv(relu(conv(pool(e1)))))      c1 -> c2 -> c2
 *   e3 = relu(conv(relu(conv(pool(e2)))))      c2 -> c3 -> c3
 *   d2 = relu(conv(relu(conv(up(e3))) + e2))   c3 -> c2, c2 -> c2
 *   d1 = relu(conv(relu(conv(up(d2))) + e1))   c2 -> c1, c1 -> c1
 *   y  = conv(d1)                               c1 -> 16, channels 0..2 used
 * Input features per node (16 channels, 13 used): mean normalised stiffness E/E_max of the
 * adjacent voxels; for each component, 1 where the DOF is fixed (Dirichlet face, a
 * constraint row, or the contact surface of an indenter); eps* (6 entries) times 1000; the node coordinates divided by the cell
 * edge.  Output: u~ / (n_max * 1e-3), n_max the largest voxel count of the cell's axes.
 * Parameters are packed layer by layer as W[27][cout][cin] (tap = 9 (dz+1) + 3 (dy+1) +
 * (dx+1)) followed by b[cout], in the layer order above; c1, c2, c3 are multiples of 16
 * in [16, 64].
 *
 * All calls return dtt_status (dtt.h); messages via dtt_last_error().  A dtt_net is used
 * on its own stream; calls on one net are not thread-safe. */
#ifndef DTT_NET_H
#define DTT_NET_H

#include <stdint.h>

#include "dtt.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dtt_net dtt_net;

/* Creates a network with He-normal weights drawn from `seed` and zero biases. */
dtt_status dtt_net_create(dtt_net** out, int32_t c1, int32_t c2, int32_t c3, uint64_t seed, void* cuda_stream);
void dtt_net_destroy(dtt_net* net);
int64_t dtt_net_num_params(const dtt_net* net);
/* FP32 master parameters in the packed order (host arrays of dtt_net_num_params floats). */
dtt_status dtt_net_get_params(const dtt_net* net, float* params);
dtt_status dtt_net_set_params(dtt_net* net, const float* params);

/* Loss and gradients of one input (tracing and parity aid).  x: host float array
 * [nz][ny][nx][16]; target: host [nz][ny][nx][3]; with d = y - target on the three output
 * channels and s the largest of nx, ny, nz,
 *   loss = mean over nodes and channels of  d^2 + w s^2 sum_axis (d(next node) - d)^2
 * (forward differences between neighbouring nodes inside the grid: the scaled difference
 * is a strain-like error, which is what the solver's first residual sees; w is set by
 * dtt_net_set_loss, default 0); grad (host, num_params floats) receives dloss/dparam. */
dtt_status dtt_net_loss_grad(dtt_net* net, int32_t nx, int32_t ny, int32_t nz, const float* x, const float* target,
                             double* loss, float* grad);

/* Weight w of the difference term of the training loss (>= 0; 0 = plain mean squares). */
dtt_status dtt_net_set_loss(dtt_net* net, float grad_weight);

/* Network output y[:, :, :, 0:3] for a host input x (as above) into host out [nz][ny][nx][3]. */
dtt_status dtt_net_forward(dtt_net* net, int32_t nx, int32_t ny, int32_t nz, const float* x, float* out);

/* Input features of a configured grid (material, constraints and load set), host float
 * [nz][ny][nx][16] in node order (feature layout above). */
dtt_status dtt_net_features(dtt_net* net, dtt_grid* grid, float* x);

/* One Adam step (lr, beta1 0.9, beta2 0.999, eps 1e-8) on one grid: features, forward,
 * loss against u_target (host, 3 x n_nodes float64 in the grid's node order, the solver's
 * converged u~), backward, update.  *loss receives the loss before the update. */
dtt_status dtt_net_train_step(dtt_net* net, dtt_grid* grid, const double* u_target, float lr, double* loss);

/* The first half of dtt_net_train_step for data-parallel training: features, forward, loss
 * and backward of one grid, dloss/dparam into grad (device, num_params floats,
 * caller-owned), the loss into *loss; the parameters and the Adam state are unchanged.
 * dtt_net_apply_grad (below) takes the step.  DTT_ERR_ARG for a grad pointer that is not
 * device memory of the current device. */
dtt_status dtt_net_grad_step(dtt_net* net, dtt_grid* grid, const double* u_target, float* grad, double* loss);

/* Writes the network's guess of u~ into the grid (as dtt_set_initial), for a solve with
 * init = DTT_INIT_GUESS. */
dtt_status dtt_net_predict(dtt_net* net, dtt_grid* grid);

/* ---- Increment mode: the warm start of one load increment of a sphere indentation ----
 *
 * Algorithm 2 solves the contact problem increment by increment, each from the previous
 * increment's field; its start sets the contact zone C = {g < 0} at the starting field
 * (Section 5.1.3).  The paper names a better initialisation as a prospect (Section 5.4,
 * conclusion).  In this mode the network maps the cell (stiffness, fixed-DOF masks, node
 * coordinates: channels 0-3 and 10-12 as above) and the load of the increment to a guess
 * of its displacement and of its contact pressure:
 *   channels 4-6: the secant prediction of the increment divided by dd = d_k - d_(k-1):
 *                 (u~_(k-1) - u~_(k-2)) s / dd with s = (d_k^1.5 - d_(k-1)^1.5) /
 *                 (d_(k-1)^1.5 - d_(k-2)^1.5) (the Hertz force grows like d^1.5);
 *   channel 7:    1 on the contact-surface nodes;
 *   channel 8:    on those nodes, the gap of the secant-predicted position to the moved
 *                 sphere (Section 5.1.1) divided by dd, clipped to [-8, 8];
 *   channel 9:    on those nodes, the previous increment's contact pressure -f_n divided
 *                 by its largest value f_max;
 *   channels 13-15: 0.
 * Outputs: channels 0-2 the correction c to the secant prediction, the guess being
 * u~_k = u~_(k-1) + dd (secant / dd + w c), w = 1 inside the window and falling linearly
 * to 0 over its last 8 nodes before each face that lies inside the grid; channel 3 the
 * contact pressure over f_max.  The
 * guess's initial contact zone is the previous increment's ({f_n < 0}, which only grows
 * under monotone loading) together with the nodes whose predicted pressure exceeds the
 * threshold (default 0.05).
 * Training loss: mean over nodes and channels 0-2 of (y - t)^2 plus w times the mean over
 * the surface nodes of (y_3 - t_3)^2 (w default 1), t the solver's converged increment
 * (correction form, clipped to [-8, 8]) and pressure (clipped to [0, 4]).
 *
 * Arguments common to the calls below: grid = a configured grid with an indenter, its u~
 * the converged field of increment k-1 and its sphere moved to increment k's centre;
 * u_prev2 = u~ of increment k-2 (device, 3 x n_nodes float64; NULL = zero); fn_prev = the
 * normal reactions of increment k-1 on its contact set and zero at the other surface nodes
 * (device, n_surface float64, the order of dtt_get_contact, whose fn holds the free nodes'
 * residual off the set; NULL: the grid's own reactions and contact set of its last solve,
 * read on the device); depth = {d_(k-2), d_(k-1), d_k} with 0 <= d_(k-2) < d_(k-1) <
 * d_k (d_(k-2) = 0 with u_prev2 = NULL for the second increment).  DTT_ERR_STATE without
 * an indenter, DTT_ERR_ARG on bad depths. */

/* Loss weight w of the pressure term (>= 0), the pressure threshold of the initial contact
 * zone, and the network's window: window_depth node layers from the contact face inward
 * and window_lateral nodes across it, centred under the sphere (0: the whole grid).  The
 * network sees, and corrects, only the window; outside it the guess is the secant
 * prediction and no surface node starts in contact.  Defaults: 1, 0.05, 0, 0. */
dtt_status dtt_net_set_increment(dtt_net* net, float pressure_weight, float active_threshold, int32_t window_lateral,
                                 int32_t window_depth);

/* Input features of increment k inside the window into host x [wz][wy][wx][16] (window
 * extents; may be NULL: computed only). */
dtt_status dtt_net_increment_features(dtt_net* net, dtt_grid* grid, const double* u_prev2, const double* fn_prev,
                                      const double depth[3], float* x);

/* One Adam step on increment k: u_target = its converged u~ (device, 3 x n_nodes float64),
 * fn_target = its normal reactions on its contact set, zero elsewhere (device, n_surface
 * float64).  *loss before the update. */
dtt_status dtt_net_train_increment(dtt_net* net, dtt_grid* grid, const double* u_prev2, const double* fn_prev,
                                   const double depth[3], const double* u_target, const double* fn_target, float lr,
                                   double* loss);

/* Data-parallel training: dtt_net_train_increment split at the optimiser, so that ranks
 * that each hold their own increments can sum their gradients (one all-reduce of
 * dtt_net_num_params floats per step) before every rank takes the same Adam step.
 *
 * dtt_net_grad_increment: the features, forward pass, loss and backward pass of increment k
 * (arguments as dtt_net_train_increment); grad (device, num_params floats, caller-owned)
 * receives dloss/dparam, *loss the loss; the parameters and the Adam state are unchanged.
 *
 * dtt_net_apply_grad: one Adam step (as dtt_net_train_step's) with the gradient scale x grad
 * (grad: device, num_params floats, complete when the call is made: the library reads it on
 * the net's stream; scale: finite, > 0, e.g. 1 / the number of gradients summed into grad).
 * grad_increment followed by apply_grad(scale 1) on its output is train_increment (the
 * weight gradients are summed with float atomics, so any two evaluations of one gradient
 * agree to the order of those sums, about 1e-7 relative).  Both calls synchronise the net's
 * stream before returning; DTT_ERR_ARG for a host pointer, memory of another device than
 * the current one, lr <= 0 or a bad scale. */
dtt_status dtt_net_grad_increment(dtt_net* net, dtt_grid* grid, const double* u_prev2, const double* fn_prev,
                                  const double depth[3], const double* u_target, const double* fn_target, float* grad,
                                  double* loss);
dtt_status dtt_net_apply_grad(dtt_net* net, const float* grad, float scale, float lr);

/* Writes the guess of increment k into the grid: u~ and the initial contact zone, the
 * current u~ (increment k-1's) kept as the fallback start.  The next solve with init =
 * DTT_INIT_GUESS evaluates the Eq. 5 residual at the guess (its zone) and at the previous
 * increment's field (zone {g < 0}) and starts from the lower. */
dtt_status dtt_net_predict_increment(dtt_net* net, dtt_grid* grid, const double* u_prev2, const double* fn_prev,
                                     const double depth[3]);

/* Tracing aid for per-layer parity: runs dtt_net_loss_grad's forward and backward passes on
 * host x [nz][ny][nx][16] and target [nz][ny][nx][3] and returns, for `layer` (0 .. 10 in the
 * order of the network listing above), its input activation act_in (host float [V][cin], the
 * BF16 values the layer read), the gradient of the loss with respect to its output taken
 * through its ReLU, as the weight-gradient kernel consumed it (host float [V][cout], BF16
 * values; the last layer has no ReLU), its parameter gradients grad_w ([27][cout][cin]) and
 * grad_b ([cout]), and the gradient with respect to its input grad_in ([V][cin], FP32; zero
 * for layer 0, whose input gradient is not formed); V = the node count of the layer's level
 * (full, half or quarter resolution, halves rounded up).  Any output pointer may be NULL.
 * DTT_ERR_ARG for a layer outside 0 .. 10. */
dtt_status dtt_net_layer_trace(dtt_net* net, int32_t nx, int32_t ny, int32_t nz, const float* x, const float* target,
                               int32_t layer, float* act_in, float* dz, float* grad_w, float* grad_b, float* grad_in);

/* Loss and gradients of the increment loss for host inputs (parity aid): x [nz][ny][nx][16],
 * target [nz][ny][nx][4], pmask [nz][ny][nx] (1 on surface nodes), grad (host, num_params). */
dtt_status dtt_net_loss_grad_increment(dtt_net* net, int32_t nx, int32_t ny, int32_t nz, const float* x,
                                       const float* target, const float* pmask, double* loss, float* grad);

#ifdef __cplusplus
}
#endif

#endif /* DTT_NET_H */
