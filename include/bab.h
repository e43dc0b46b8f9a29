/*
 * bab.h -- C ABI of libbab, a GB300 (sm_103a) library for the data-parallel
 * bounding hot path of BaB-ND: branch-and-bound planning over a learned
 * residual ReLU-MLP dynamics model (arXiv 2412.09584).
 *
 * The planning problem (Section 3, "Formulation", Eq. trajop) is
 *
 *     min_u f(u),  f(u) = sum_{t=1..H} ||x_t - g||^2 + rho sum_{t=0..H-1} ||u_t||^2,
 *     x_{t+1} = x_t + N([x_t; u_t]),  x_0 known,  u in C = [lo, hi] subset R^d, d = kH,
 *
 * where N is an L-layer ReLU MLP (ReLU after layers 1..L-1) with input size
 * s + k (state first) and output size s.  A "box" (subdomain C_i, Section 3
 * overview) is a pair of rows lo[d], hi[d]; actions are flattened t-major,
 * u[t*k + j].  Branch-and-bound (Algorithm 2) repeatedly searches boxes for
 * good plans (upper bounds), bounds them from below, prunes boxes whose lower
 * bound exceeds the incumbent, and bisects the survivors.
 *
 * Conventions shared by every call:
 *   - Return value: BAB_OK (0) or a negative BAB_ERR_* code; bab_last_error()
 *     describes the last failure of a context.  No exception crosses the ABI.
 *   - Array arguments are DEVICE pointers owned by the caller, contiguous and
 *     row-major, unless the comment says "host".  They must stay valid until
 *     the work queued on `stream` has finished.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All device work is queued on it asynchronously; a call returns
 *     before the work finishes.  A context must not be used from two host
 *     threads at once.
 *   - Row counts: `n` (host) is the number of boxes.  Where `d_n` is non-NULL
 *     it points to a device int holding the live count (<= n), read by the
 *     kernels, so that a call can be captured in a CUDA graph while the count
 *     changes between replays; `n` then only sizes the launch.
 *   - Scratch: the context owns its scratch device memory and grows it with
 *     cudaMalloc on demand.  Make the first call with the largest sizes before
 *     capturing a graph.
 *   - Network layout (same as the oracle's): params packs, for l = 1..L,
 *     W_l row-major [dims[l]][dims[l-1]] followed by b_l [dims[l]].
 *   - Hidden-neuron arrays (pre-activation bounds, alpha, Adam moments) are
 *     [n][H][sumh] with sumh = dims[1] + ... + dims[L-1]; per time step the
 *     hidden layers are concatenated in order.
 */
#ifndef BAB_H
#define BAB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BAB_OK 0
#define BAB_ERR_INVALID_ARG (-1)
#define BAB_ERR_SHAPE (-2)
#define BAB_ERR_CUDA (-3)
#define BAB_ERR_OOM (-4)
#define BAB_ERR_TIMEOUT (-5)
#define BAB_ERR_NUMERIC (-6)
#define BAB_ERR_UNSUPPORTED (-7)

/* Arithmetic of the dense products. */
#define BAB_PREC_FP32 0    /* FP32 on CUDA cores (round-to-nearest FMA chains) */
#define BAB_PREC_BF16X3 1  /* tcgen05 tensor cores, 3-term BF16 split operands, FP32 accumulate */
#define BAB_PREC_BF16 2    /* tcgen05 tensor cores, BF16 operands, FP32 accumulate (rollouts only) */
#define BAB_PREC_TF32X3 3  /* tcgen05 tensor cores, 3-term TF32 split operands, FP32 accumulate (CROWN, alpha, intervals) */

/* Split rules of bab_prune_branch. */
#define BAB_SPLIT_WIDEST 0 /* bisect the widest coordinate (Section 3.1), lowest index on ties */

/* Pick-out rules for the part of the quota not taken by smallest upper bound (Section 3.1). */
#define BAB_PICK_LB 0      /* smallest (lb, id): deterministic */
#define BAB_PICK_SOFTMAX 1 /* the softmax sampling of Eq. lf_pick (counter-based, reproducible) */

/* state cost of the objective (bab_set_cost) */
#define BAB_COST_SQUARED 0           /* ||x_t - g||^2 (default) */
#define BAB_COST_PUSHING_OBSTACLES 1 /* Appendix D.4, Eq. pushing_cost */

/* Limits of this build. */
#define BAB_MAX_LAYERS 8
#define BAB_MAX_WIDTH 256

typedef struct bab_ctx bab_ctx;

/* Library version, major * 10000 + minor * 100 + patch. */
int bab_version(void);

/*
 * Load the dynamics network f_dyn (Section 3, Formulation; Appendix B.1,
 * "Definition": z_l = W_l a_{l-1} + b_l, a_l = ReLU(z_l) for l < L) and create a
 * context on the current CUDA device.
 *   out        receives the new context (host pointer to a host pointer).
 *   n_layers   L, 1 <= L <= BAB_MAX_LAYERS.
 *   dims       host int[L+1]; dims[0] = state_dim + action_dim, dims[L] =
 *              state_dim, every width <= BAB_MAX_WIDTH.
 *   params     HOST float array packed as described above; copied, so the
 *              caller may free it on return.
 *   flags      reserved, pass 0.
 * Errors: BAB_ERR_INVALID_ARG (null pointer, flags), BAB_ERR_SHAPE (dims),
 * BAB_ERR_NUMERIC (a non-finite parameter), BAB_ERR_OOM, BAB_ERR_CUDA.
 */
int bab_load_dynamics(bab_ctx **out, int n_layers, const int *dims, const float *params, int state_dim,
                      int action_dim, unsigned flags);

/* Free a context and its device memory (synchronises the device first). */
int bab_destroy(bab_ctx *ctx);

/* Message of the last failure of ctx (empty string if none); valid until the next call on ctx. */
const char *bab_last_error(const bab_ctx *ctx);

/*
 * Sampled search (Section 3.3, batch_search, with uniform sampling): for each
 * box i < n draw `samples` action sequences u^m uniformly in the box, roll the
 * dynamics out for H steps and keep the best objective:
 *     ub[i] = min_m f(u^m),  best_u[i] = argmin (lowest m on ties).
 * Sample m, coordinate j of box i is u = lo + (hi - lo) * r, formed in FP32
 * without fused multiply-add, with r the top 24 bits of a SplitMix64 chain
 * over (seed, id[i], m, j) divided by 2^24:
 *     h = sm64(seed ^ sm64(id)),  h = sm64(h ^ (m << 32 | j)),  r = (h >> 40) / 2^24,
 * where sm64 is the SplitMix64 output function (Steele, Lea and Flood, 2014).
 *   x0, goal   device float[s]; horizon H >= 1; rho >= 0.
 *   lo, hi     device float[n][d], d = k * H; id device uint64[n] (distinct).
 *   samples    M >= 1.  precision: BAB_PREC_FP32, BAB_PREC_BF16X3 or BAB_PREC_BF16.
 *   ub         device float[n]; best_u device float[n][d] (nullable).
 *   inc_val, inc_u (both nullable, device double[1], float[d]): the incumbent
 *              of Algorithm 2 (its incumbent update).  If given, the box with the
 *              smallest ub (lowest index on ties) has its best_u re-evaluated
 *              in FP64 on the GPU, and if that value is below *inc_val the
 *              pair (*inc_val, inc_u) is replaced by it.  Requires best_u.
 * Errors: BAB_ERR_INVALID_ARG, BAB_ERR_SHAPE (H, n, samples, d), BAB_ERR_UNSUPPORTED
 * (precision not built for this network), BAB_ERR_CUDA.
 */
int bab_rollout(bab_ctx *ctx, const float *x0, const float *goal, int horizon, float rho, const float *lo,
                const float *hi, const uint64_t *id, int n, const int *d_n, int samples, uint64_t seed,
                int precision, float *ub, float *best_u, double *inc_val, float *inc_u, void *stream);

/*
 * The paper's own bounding (Section 3.2; Appendix B.2, Algorithm 3).
 *
 * bab_rollout_search_bounds: bab_rollout in FP32 (the same samples, ub,
 * best_u, incumbent) that also records, per box, the minimum and maximum over
 * its samples of every hidden pre-activation (pre_lo/pre_hi, device
 * float[n][H][sumh]) and of every state (x_lo/x_hi, device float[n][H+1][s];
 * x_0 exact): the search-integrated intermediate bounds.  They may
 * underestimate the true ranges.
 *
 * bab_bound_crown_given: the CROWN bound (FP32, adaptive slopes) with the
 * caller's intermediate bounds in place of bab_bound_ibp's, and propagation
 * early-stop at step t_stop (0 <= t_stop <= H; the early-stop set is the
 * state x_{t_stop}): the cost terms after t_stop are carried back to
 * x_{t_stop} and concretized on its interval, those at steps 1 .. t_stop are
 * bounded on their intervals, rho ||u||^2 on the box.  t_stop = 0 propagates
 * to the input.  With search-integrated bounds the result is the paper's
 * estimate of the lower bound, not a sound bound, and no rounding margin is
 * subtracted.  lb device float[n].
 * Errors: BAB_ERR_INVALID_ARG (t_stop out of range, null arrays), BAB_ERR_SHAPE, BAB_ERR_CUDA.
 */
int bab_rollout_search_bounds(bab_ctx *ctx, const float *x0, const float *goal, int horizon, float rho,
                              const float *lo, const float *hi, const uint64_t *id, int n, const int *d_n,
                              int samples, uint64_t seed, float *ub, float *best_u, double *inc_val, float *inc_u,
                              float *pre_lo, float *pre_hi, float *x_lo, float *x_hi, void *stream);
int bab_bound_crown_given(bab_ctx *ctx, const float *x0, const float *goal, int horizon, float rho, const float *lo,
                          const float *hi, int n, const int *d_n, const float *pre_lo, const float *pre_hi,
                          const float *x_lo, const float *x_hi, int t_stop, float *lb, void *stream);

/*
 * The incumbent step of Algorithm 2 on its own (bab_rollout does it when given
 * inc_val): the box with the smallest ub (lowest index on ties) has its plan
 * best_u re-evaluated in FP64; if that value is below *inc_val it becomes the
 * incumbent (inc_val, inc_u).  A separate call lets the FP64 re-score run on
 * another stream, concurrently with the bounds of the same boxes.
 *   ub device float[n], best_u device float[n][k H] (from bab_rollout).
 *   inc_val device double[1], inc_u device float[k H]: read and updated.
 * Errors: BAB_ERR_INVALID_ARG, BAB_ERR_SHAPE, BAB_ERR_CUDA.
 */
int bab_update_incumbent(bab_ctx *ctx, const float *x0, const float *goal, int horizon, float rho, const float *ub,
                         const float *best_u, int n, const int *d_n, double *inc_val, float *inc_u, void *stream);

/*
 * Interval bound propagation through the unrolled dynamics: the intermediate
 * (pre-activation) bounds that Lemma 1 (Appendix B.1) needs, in outward-rounded
 * FP32 so that they contain the exact interval bounds.  Per layer the input
 * interval [a_lo, a_hi] maps to [z_lo, z_hi] with z_lo = W+ a_lo + W- a_hi + b
 * (rounded down) and z_hi = W+ a_hi + W- a_lo + b (rounded up); ReLU clamps
 * both ends; x_{t+1} lies in [x_t] + [z_L].
 *   lb_ibp     device float[n] (nullable): interval lower bound of f.
 *   pre_lo, pre_hi  device float[n][H][sumh] (nullable, both or neither).
 *   x_lo, x_hi device float[n][H+1][s] (nullable, both or neither).
 * Errors: BAB_ERR_INVALID_ARG, BAB_ERR_SHAPE, BAB_ERR_CUDA.
 */
int bab_bound_ibp(bab_ctx *ctx, const float *x0, const float *goal, int horizon, float rho, const float *lo,
                  const float *hi, int n, const int *d_n, float *lb_ibp, float *pre_lo, float *pre_hi, float *x_lo,
                  float *x_hi, void *stream);

/*
 * Sound CROWN lower bound of f over each box (Appendix B.1: Lemma 1, Theorem
 * 1, Theorem 2 in box form), with interval intermediate bounds.  Each square
 * ||x_t - g||^2 is bounded below by its tangent at the midpoint of its
 * interval, the resulting linear function of the states is propagated
 * backward through the unrolled network (lower ReLU bound where the
 * coefficient is >= 0, upper where < 0), and the final function of u,
 * lin_const + mu . u + rho ||u||^2, is minimised exactly over the box.
 * lb[i] is that minimum MINUS margin[i], an a-posteriori bound on the FP32
 * rounding error of the whole computation, so lb[i] <= the exact CROWN bound
 * <= min_box f.
 *   alpha      device float[n][H][sumh] (nullable): lower slopes of unstable
 *              ReLUs, each in [0, 1]; NULL selects the adaptive slope
 *              (1 if u >= -l, else 0).
 *   precision  BAB_PREC_FP32, BAB_PREC_BF16X3 or BAB_PREC_TF32X3.  The split
 *              precisions evaluate every backward product A' W_l as
 *              A'h Wh + A'h Wl + A'l Wh on the tensor cores (BF16 halves: about
 *              2^-16 representation error per operand; TF32 halves: about
 *              2^-22, at twice the operand bytes and twice the instructions),
 *              and charge gamma_K sum |A'| |W| max|a| to the margin.
 *              BAB_PREC_TF32X3 takes the squared-distance cost and networks
 *              whose widths are all at most 256 (else BAB_ERR_UNSUPPORTED).
 *   lb         device float[n]; margin device float[n] (nullable).
 *   lin_coef   device float[n][d] (nullable): mu; lin_const device float[n]
 *              (nullable): the constant (before the margin).
 * Errors: BAB_ERR_INVALID_ARG, BAB_ERR_SHAPE, BAB_ERR_UNSUPPORTED, BAB_ERR_OOM, BAB_ERR_CUDA.
 */
int bab_bound_crown(bab_ctx *ctx, const float *x0, const float *goal, int horizon, float rho, const float *lo,
                    const float *hi, int n, const int *d_n, const float *alpha, int precision, float *lb,
                    float *margin, float *lin_coef, float *lin_const, void *stream);

/*
 * One step of alpha-CROWN: the free lower slopes alpha of Lemma 1 are raised
 * by projected Adam ascent on the sum of the boxes' bounds.  The step
 *   1. computes the bound at alpha (as bab_bound_crown, margin subtracted)
 *      and its gradient dLB/dalpha_j = A_j z~_j(u*) for unstable neurons whose
 *      lower bound is selected (A_j >= 0 the coefficient of the ReLU output, z~
 *      the pre-activation of the relaxed network at the concretizing point
 *      u*), 0 elsewhere;
 *   2. lb_best[i] = max(lb_best[i], lb[i]) (every alpha gives a valid bound);
 *   3. Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected with `step`,
 *      counting from 1) ascent on alpha with learning rate lr, then clamps
 *      alpha to [0, 1].
 *   alpha, adam_m, adam_v  device float[n][H][sumh], updated in place
 *              (m, v start at 0; alpha typically at the adaptive slopes).
 *   precision  BAB_PREC_FP32, BAB_PREC_BF16X3 or BAB_PREC_TF32X3 (the CROWN
 *              products, as bab_bound_crown).
 *   lb         device float[n] (nullable): bound at the incoming alpha.
 *   lb_best    device float[n] (nullable): running maximum, updated.
 *   grad_alpha device float[n][H][sumh] (nullable): the gradient.
 * Errors: as bab_bound_crown.
 */
int bab_alpha_step(bab_ctx *ctx, const float *x0, const float *goal, int horizon, float rho, const float *lo,
                   const float *hi, int n, const int *d_n, float *alpha, float *adam_m, float *adam_v, int step,
                   float lr, int precision, float *lb, float *lb_best, float *grad_alpha, void *stream);

/*
 * The bound at alpha and its gradient with respect to alpha, without an
 * optimiser step: step 1 of bab_alpha_step alone (Lemma 1's free lower slope;
 * dLB/dalpha_j = A_j z~_j(u*) for unstable neurons with the lower bound
 * selected, 0 elsewhere).  For use under an autodiff framework.
 *   alpha      device float[n][H][sumh] (read only).
 *   lb         device float[n]: the bound at alpha (margin subtracted).
 *   grad_alpha device float[n][H][sumh]: d lb[i] / d alpha[i].
 * Errors: as bab_bound_crown.
 */
int bab_alpha_grad(bab_ctx *ctx, const float *x0, const float *goal, int horizon, float rho, const float *lo,
                   const float *hi, int n, const int *d_n, const float *alpha, int precision, float *lb,
                   float *grad_alpha, void *stream);

/*
 * The bound and its gradient with respect to the box faces, FP32: d lb[i] /
 * d lo[i][j] and d lb[i] / d hi[i][j] with the slopes alpha held fixed (alpha
 * nullable: adaptive), almost everywhere (the bound is piecewise smooth in the
 * box).  The relaxation choices of Lemma 1 held fixed, the bound is the
 * minimum over the box of the relaxed network's objective (Theorems 1-2), so
 * it moves with each parameter of that objective as the objective's partial
 * derivative at the concretizing point: the upper chords of unstable neurons
 * and the tangent points of the cost (functions of the interval bounds, which
 * are functions of the box), and the box faces themselves where u* sits on
 * them.  No counterpart in the paper, which differentiates neither.
 *   alpha      device float[n][H][sumh] (nullable).
 *   lb         device float[n]: the bound (margin subtracted), as bab_bound_crown.
 *   grad_lo, grad_hi  device float[n][k H].
 * Errors: as bab_bound_crown.
 */
int bab_box_grad(bab_ctx *ctx, const float *x0, const float *goal, int horizon, float rho, const float *lo,
                 const float *hi, int n, const int *d_n, const float *alpha, float *lb, float *grad_lo,
                 float *grad_hi, void *stream);

/*
 * alpha-CROWN in one call: `steps` rounds of bab_alpha_step from the adaptive
 * slopes, with the interval bounds (which do not depend on alpha) computed
 * once, and the Adam moments in context scratch.  lb_best[i] receives the
 * best bound of box i over all steps (each a valid bound, margin subtracted).
 *   steps      number of Adam steps (>= 1); lr their learning rate.
 *   precision  BAB_PREC_FP32, BAB_PREC_BF16X3 or BAB_PREC_TF32X3.
 *   alpha      device float[n][H][sumh] (nullable): receives the final slopes.
 *   lb_best    device float[n].
 * All work is queued on `stream` without host synchronisation.  In FP32 the
 * whole loop runs as one launch after the interval bounds
 * (BAB_KERNEL_ALPHA_FUSED) with the same arithmetic, step for step, as the
 * separate bound, adjoint and Adam launches.
 * Errors: as bab_bound_crown.
 */
int bab_alpha_optimize(bab_ctx *ctx, const float *x0, const float *goal, int horizon, float rho, const float *lo,
                       const float *hi, int n, const int *d_n, int steps, float lr, int precision, float *alpha,
                       float *lb_best, void *stream);

/*
 * The adaptive lower slopes of every hidden neuron (1 where u >= -l, else 0,
 * with the interval bounds of bab_bound_ibp), to start alpha optimisation.
 *   alpha      device float[n][H][sumh], written.
 */
int bab_alpha_init(bab_ctx *ctx, const float *x0, const float *goal, int horizon, float rho, const float *lo,
                   const float *hi, int n, const int *d_n, float *alpha, void *stream);

/*
 * Prune, pick out and split one pool of n boxes (Algorithm 2: Pruner, then
 * batch_pick_out and batch_split of Section 3.1).
 *   1. Prune: box i is dropped iff (double)lb[i] > *inc_val (strict; a NaN
 *      bound is kept and latches BAB_ERR_NUMERIC in the device status read by
 *      bab_status, without stopping the call).  keep[i] = 1 if kept.
 *   2. Pick out up to n_pick survivors: all of them if there are at most
 *      n_pick; otherwise the ceil(eta * n_pick) smallest by (ub, id), then the
 *      rest of the quota by smallest (lb, id) among the others.
 *   3. Split each picked box on its widest coordinate (lowest index on ties)
 *      at mid = 0.5f * (lo + hi) in FP32: child 2p is the lower half, child
 *      2p + 1 the upper half, ids 2 id and 2 id + 1 (deeper than 62 splits,
 *      id >= 2^62: 2^62 + (splitmix64(2 id + c) >> 2), c = 0, 1), lb and ub
 *      inherited.
 * Output rows: the 2P children (picked boxes in pool order) followed by the R
 * unpicked survivors in pool order.  d_counts (device int[3]) receives
 * {2P, R, 2P + R}: pass d_counts (children) or d_counts + 2 (whole pool) as
 * the `d_n` of the next calls to chain an iteration without a host sync.
 * Everything is integer or exact FP32 work: results are bit-identical run to
 * run.
 *   d          box dimension; lo, hi device float[n][d]; lb, ub float[n]; id uint64[n] (distinct).
 *   inc_val    device double[1].
 *   n_pick >= 0, 0 <= eta <= 1, split_rule BAB_SPLIT_WIDEST.
 *   cap_out    rows available in the outputs; must be >= n + n_pick.
 *   out_*      device arrays of cap_out rows; keep device uint8[n].
 * Errors: BAB_ERR_INVALID_ARG, BAB_ERR_SHAPE (cap_out too small), BAB_ERR_CUDA.
 * Every picked box can be split, whatever its id: past 2^62 the children's
 * ids continue as the hash given above, so no depth limit is latched.
 */
int bab_prune_branch(bab_ctx *ctx, int d, const float *lo, const float *hi, const float *lb, const float *ub,
                     const uint64_t *id, int n, const int *d_n, const double *inc_val, int n_pick, float eta,
                     int split_rule, int cap_out, float *out_lo, float *out_hi, float *out_lb, float *out_ub,
                     uint64_t *out_id, uint8_t *keep, int *d_counts, void *stream);

/*
 * The paper's branching heuristics (Section 3.1).
 *
 * bab_prune_branch_heuristic: bab_prune_branch where the part of the pick-out
 * quota not taken by smallest ub is drawn by the softmax of Eq. lf_pick over
 * the min-max scaled lower bounds of the remaining survivors, with
 * temperature T (pick_rule BAB_PICK_SOFTMAX; BAB_PICK_LB keeps the smallest
 * (lb, id)): the n_pick - ceil(eta n_pick) candidates with the smallest race
 * keys s / T + log(-log U), U from SplitMix64 of (pick_seed, id), a draw
 * without replacement with those probabilities, reproducible bit for bit
 * (the logarithm is computed from basic FP32 operations).  NaN bounds come
 * last.  split_dim (device int[n], nullable) gives the dimension to split for
 * each pool row (out of range: widest); out_split_dim (device int[cap_out],
 * nullable) carries it along: unpicked rows keep theirs, children get -1
 * (their own split dimensions come from their search).  row_u (device
 * float[n][d], nullable) is a vector per pool row, such as the best input its
 * search found; out_row_u (float[cap_out][d], given with row_u) receives it:
 * unpicked rows keep theirs and both children inherit the parent's (the warm
 * start of their cross-entropy search, Section 3.3).  The rest is
 * bab_prune_branch.
 * Errors: as bab_prune_branch, BAB_ERR_INVALID_ARG for an unknown rule or
 * temperature <= 0.
 *
 * bab_split_dims: for each box, among its top_k samples (smallest (cost, m)
 * of costs, device float[n][samples], the objective per sample as the search
 * computed it), counts n_lo / n_up of the coordinates below / above the
 * midpoint of each dimension (samples re-drawn from the counter-based
 * sampler with `seed`), and writes to split_dim (device int[n]) the dimension
 * of largest (hi - lo) |n_lo - n_up| (lowest index on ties; the widest when
 * none is imbalanced).  1 <= top_k <= min(64, samples).
 *
 * bab_rollout_split: bab_rollout that also keeps every sample's objective
 * (costs, nullable: context scratch) and then runs bab_split_dims with
 * top_k = ceil(top_pct / 100 * samples) (clamped to [1, 64]).
 */
int bab_prune_branch_heuristic(bab_ctx *ctx, int d, const float *lo, const float *hi, const float *lb,
                               const float *ub, const uint64_t *id, int n, const int *d_n, const double *inc_val,
                               int n_pick, float eta, int pick_rule, float temperature, uint64_t pick_seed,
                               const int *split_dim, int cap_out, float *out_lo, float *out_hi, float *out_lb,
                               float *out_ub, uint64_t *out_id, int *out_split_dim, const float *row_u,
                               float *out_row_u, uint8_t *keep, int *d_counts, void *stream);
int bab_split_dims(bab_ctx *ctx, int d, const float *lo, const float *hi, const uint64_t *id, int n, const int *d_n,
                   uint64_t seed, const float *costs, int samples, int top_k, int *split_dim, void *stream);
int bab_rollout_split(bab_ctx *ctx, const float *x0, const float *goal, int horizon, float rho, const float *lo,
                      const float *hi, const uint64_t *id, int n, const int *d_n, int samples, uint64_t seed,
                      int precision, float top_pct, float *ub, float *best_u, double *inc_val, float *inc_u,
                      float *costs, int *split_dim, void *stream);

/*
 * ---------------------------------------------------------------------------
 * The state cost c(x_t), t = 1..H, of the objective f(u) = sum_t c(x_t) +
 * rho sum_t ||u_t||^2 (Section 3, Eq. trajop).  BAB_COST_SQUARED (default):
 * ||x_t - g||^2.  BAB_COST_PUSHING_OBSTACLES (Appendix D.4, Eq. pushing_cost):
 * w_t ||x_t - g|| + lambda sum_o [ReLU(s_o - ||p_t - p_o||) + sum_i ReLU(s_o -
 * ||x_t^(i) - p_o||)], the state being s / 2 planar keypoints x_t^(i) =
 * (x_{t,2i}, x_{t,2i+1}) and the action the planar pusher motion (k = 2), with
 * p_t = p0 + u_0 + ... + u_{t-1}.  Arguments (host): w [H] (w[t - 1] = w_t,
 * finite, >= 0; calls with a longer horizon are refused), lambda >= 0,
 * obstacles [n_obs][3] (x, y, size), n_obs <= 8, p0 [2].  The context keeps a
 * device copy; kind BAB_COST_SQUARED clears it.
 *
 * Paths that support the obstacle cost: bab_rollout (FP32; BF16X3 and BF16
 * for s <= 8, BF16 with each box's pick re-scored in FP32 under this cost),
 * bab_rollout_cem (FP32), bab_update_incumbent, bab_bound_ibp (FP32
 * intervals, whatever bab_set_interval_precision selects), bab_bound_crown
 * (FP32, adaptive or given slopes; BF16X3 when the backward image fits in
 * shared memory), bab_alpha_init and the alpha calls (bab_alpha_grad,
 * bab_alpha_step, bab_alpha_optimize, in the same precisions); the other
 * paths (TF32X3, the tensor-core cross-entropy search, early stop, batched
 * problems, the box gradient, the autotuner) return BAB_ERR_UNSUPPORTED.
 * Sound as for the squared cost: interval minima per term rounded down; in
 * CROWN the norm by its tangent plane at the box centre (w ||y|| >= w ghat . y,
 * |ghat| <= 1), each penalty by an affine function below the concave
 * s_o - distance at the box's vertices (or 0), with the same margin.
 * Errors: BAB_ERR_INVALID_ARG, BAB_ERR_UNSUPPORTED (s odd or k != 2), BAB_ERR_CUDA.
 */
int bab_set_cost(bab_ctx *ctx, int kind, int H, const float *w, float lambda, int n_obs, const float *obstacles,
                 const float *p0);

/*
 * ---------------------------------------------------------------------------
 * Cross-entropy search (Section 3.3: batch_search with CEM, warm-started from
 * the parent's best input).  Per box [lo, hi] the search distribution is a
 * diagonal normal (mu, sigma): mu starts at warm_u clipped to the box (device
 * float[n][d], nullable: the box centre), sigma at (hi - lo) / 2.  Each of
 * `iters` iterations draws `samples` inputs u = clip(mu + sigma z, lo, hi)
 * (z: the Irwin-Hall sum of four counter-based uniforms, centred and scaled
 * to unit variance; sample 0 of iteration 0 is mu itself), evaluates them,
 * ranks them by (objective, sample index) and refits mu and sigma to the
 * `elites` best: mu = their mean, sigma = their standard deviation plus
 * `jitter`, each sum in rank order.
 *
 * Results: ub[i] the best objective over all iterations (ties keep the earlier
 * iteration) and best_u [n][d] its input (both required); the incumbent
 * (inc_val, inc_u, nullable together) is updated as in bab_rollout.
 * precision BAB_PREC_FP32 (the objective with every dot product a fused
 * multiply-add chain in input order, the step cost summed state terms then
 * action terms: decisions reproducible by any implementation of that
 * definition) or BAB_PREC_BF16X3 (tensor cores); BAB_PREC_BF16 is
 * BAB_ERR_UNSUPPORTED.  1 <= samples <= BAB_CEM_MAX_SAMPLES,
 * 1 <= elites <= samples, iters >= 1, jitter finite and >= 0, warm_u finite.
 * The context keeps mu, sigma and the objectives of one iteration in its
 * scratch (grown on first use, so not inside a graph capture the first time).
 */
#define BAB_CEM_MAX_SAMPLES 4096
int bab_rollout_cem(bab_ctx *ctx, const float *x0, const float *goal, int horizon, float rho, const float *lo,
                    const float *hi, const uint64_t *id, int n, const int *d_n, int samples, int iters, int elites,
                    float jitter, uint64_t seed, int precision, const float *warm_u, float *ub, float *best_u,
                    double *inc_val, float *inc_u, void *stream);

/*
 * ---------------------------------------------------------------------------
 * The paper's synthetic objective (Section 4, synthetic example):
 * f(u) = sum_i 5 u_i^2 + cos(50 u_i) over boxes of [-1, 1]^d, searched and
 * bounded for the same prune / pick-out / bisect calls.  It needs no network:
 * bab_context_create makes a context without one (for these calls and
 * bab_prune_branch*; the network calls then return BAB_ERR_INVALID_ARG).
 *
 * bab_synth_search: per box (lo, hi, id: device [n][d], [n]) `samples` FP32
 * evaluations of f, uniform (iters = 0; the counter sampler of bab_rollout) or
 * by the cross-entropy search of bab_rollout_cem (iters >= 1 iterations of
 * `samples` each, elites, jitter, warm_u nullable); ub[n] the best value and
 * best_u [n][d] its input (required); inc_val / inc_u (nullable together) the
 * incumbent, the best row re-evaluated in FP64.
 *
 * bab_synth_bound: lb[n], a sound lower bound of f over each box: the sum
 * over coordinates of the exact minima of 5 u^2 and of cos(50 u) over the
 * coordinate's interval (no linear relaxation of a separable objective does
 * better), rounded outward (directed rounding; the cosine's 2-ulp error
 * covered by 2^-21 per coordinate).
 * Errors: BAB_ERR_INVALID_ARG, BAB_ERR_SHAPE, BAB_ERR_CUDA, BAB_ERR_OOM.
 */
int bab_context_create(bab_ctx **out);
int bab_synth_search(bab_ctx *ctx, int d, const float *lo, const float *hi, const uint64_t *id, int n, const int *d_n,
                     int samples, uint64_t seed, int iters, int elites, float jitter, const float *warm_u, float *ub,
                     float *best_u, double *inc_val, float *inc_u, void *stream);
int bab_synth_bound(bab_ctx *ctx, int d, const float *lo, const float *hi, int n, const int *d_n, float *lb,
                    void *stream);

/*
 * Synchronise `stream` and return the sticky device-side status of ctx (0 or
 * a BAB_ERR_* code recorded by a kernel), then clear it.
 */
int bab_status(bab_ctx *ctx, void *stream);

/*
 * ---------------------------------------------------------------------------
 * Batched problems: P independent planning problems that share one network
 * architecture (each with its own weights, x_0, goal, horizon and rho) are
 * searched, bounded and branched together, one launch per kernel for all of
 * them.  The paper plans one problem at a time; this is the same method
 * (Algorithm 2 per problem) run over many problems at once.
 *
 * Layout: problem p's arrays are x0[p][s], goal[p][s], horizon[p] (device
 * int, 1 <= horizon[p] <= max_horizon), rho[p] (device float, nullable: 0).
 * Box row i belongs to problem prob[i] (device int[n]; nullable when P = 1)
 * and stores its k * horizon[prob[i]] action coordinates first in a row of
 * d_stride >= k * max_horizon floats; the remaining coordinates are carried
 * along unchanged (set them to 0).  Problem indices and horizons outside
 * their ranges are clamped so that every access stays in bounds.
 * ---------------------------------------------------------------------------
 */

/* As bab_load_dynamics for n_problems parameter vectors stored back to back
 * in params (host, n_problems x the packed size of one network).  The
 * single-problem entry points use problem 0. */
int bab_load_dynamics_batch(bab_ctx **out, int n_problems, int n_layers, const int *dims, const float *params,
                            int state_dim, int action_dim, unsigned flags);

/*
 * bab_rollout for every row of every problem: per row `samples` uniform
 * samples (the same counter RNG as bab_rollout, over the row's own k * H_p
 * coordinates), ub[i], best_u[i] (coordinates beyond k * H_p are 0), and per
 * problem the incumbent inc_val[p] (device double[P]) / inc_u[p] (device
 * float[P][d_stride]) re-scored in FP64 from the best row of that problem.
 * precision as bab_rollout; on tensor cores each sample tile streams its own
 * problem's weights (samples >= 128 when there are several problems), and in
 * BF16 every row's best sample is re-scored in FP32.
 * Errors: BAB_ERR_INVALID_ARG, BAB_ERR_SHAPE, BAB_ERR_UNSUPPORTED, BAB_ERR_CUDA, BAB_ERR_OOM.
 */
int bab_rollout_batch(bab_ctx *ctx, const float *x0, const float *goal, const int *horizon, const float *rho,
                      int max_horizon, int d_stride, const float *lo, const float *hi, const uint64_t *id,
                      const int *prob, int n, const int *d_n, int samples, uint64_t seed, int precision, float *ub,
                      float *best_u, double *inc_val, float *inc_u, void *stream);

/*
 * Sound lower bounds of every row (FP32, outward-rounded, margin
 * subtracted): interval bounds, then CROWN with the adaptive slopes
 * (alpha_steps = 0) or alpha-CROWN with alpha_steps projected Adam steps of
 * learning rate lr keeping the best bound (as bab_alpha_optimize), one warp
 * per row.  lb device float[n]; lb_ibp device float[n] (nullable): the
 * interval bound of the cost.  Bit-identical, row by row, to bab_bound_ibp /
 * bab_bound_crown / bab_alpha_optimize in FP32 on the row's own problem.
 * Errors: as bab_bound_crown.
 */
int bab_bound_batch(bab_ctx *ctx, const float *x0, const float *goal, const int *horizon, const float *rho,
                    int max_horizon, int d_stride, const float *lo, const float *hi, const int *prob, int n,
                    const int *d_n, int alpha_steps, float lr, float *lb, float *lb_ibp, void *stream);

/*
 * bab_prune_branch applied to each problem's rows separately (its incumbent
 * inc_val[p], its pick quota n_pick[p] (device int[P]), the common eta; the
 * split uses only the problem's k * H_p coordinates), in one launch.  Output
 * rows: the children of problem 0, of problem 1, ..., then the unpicked
 * survivors of problem 0, of problem 1, ..., each in pool order; out_prob
 * (device int[cap_out], nullable) receives each output row's problem.
 * d_counts as bab_prune_branch (totals); d_pcounts (device int[P][2],
 * nullable) receives each problem's picked and unpicked survivor counts.
 * max_pick_total >= sum_p n_pick[p] and cap_out >= n + max_pick_total are
 * required; rows that would land beyond cap_out are dropped and latch
 * BAB_ERR_SHAPE in the device status.
 */
int bab_prune_branch_batch(bab_ctx *ctx, int d_stride, const int *horizon, int max_horizon, const float *lo,
                           const float *hi, const float *lb, const float *ub, const uint64_t *id, const int *prob,
                           int n, const int *d_n, const double *inc_val, const int *n_pick, int max_pick_total,
                           float eta, int split_rule, int cap_out, float *out_lo, float *out_hi, float *out_lb,
                           float *out_ub, uint64_t *out_id, int *out_prob, uint8_t *keep, int *d_counts,
                           int *d_pcounts, void *stream);

/*
 * Launch variants (tile shapes) and their autotuner.  The paper has no
 * counterpart: these choose between equivalent launch configurations only;
 * no variant changes a result beyond floating-point summation order (the
 * FP32 rollout variants, and the fused alpha loop against the separate
 * launches, give bit-identical results: each output is summed in the same
 * order whatever the tile).
 *   BAB_KERNEL_ROLLOUT_FP32  0: 64 samples x 256 threads, one CTA per SM;
 *                            1: 64 x 256 with <= 128 registers; 2: 32 x 128.
 *   BAB_KERNEL_ALPHA_FUSED   -2: separate bound / adjoint / Adam launches;
 *                            0, 1, 2: one launch, 2, 4 or 8 boxes per CTA with
 *                            all per-box state in shared memory (small
 *                            networks and horizons only: BAB_ERR_UNSUPPORTED
 *                            otherwise); 3 (and -1): one launch, one warp per
 *                            box, per-box state in global memory (squared-
 *                            distance cost only: with the obstacle cost -1
 *                            takes the separate launches and 3 is refused).
 *   BAB_KERNEL_ROLLOUT_TC    1 or 2 sample tiles per CTA; BF16 rollouts with
 *                            the image in shared memory, uniform samples and
 *                            the squared-distance cost run the fused-step
 *                            kernel (the output layer of step t and layer 1 of
 *                            step t + 1 as one product); 3 or 4: 1 or 2 tiles
 *                            per CTA, layer by layer in every case.
 *   BAB_KERNEL_CROWN_TC      3 or 4: feature-major products (the layer's
 *                            features on the MMA's 128 rows, 32 boxes on its
 *                            columns) with 8 or 16 epilogue warps; with
 *                            widths between 129 and 256 (either value) two
 *                            128-row feature blocks, 16 boxes a tile and the
 *                            image streamed through shared memory; squared-
 *                            distance cost and widths <= 256 only, 0 otherwise
 *                            (4 is the default where it applies);
 *                            0: box-major, one tile of up to 32 boxes per CTA,
 *                            each epilogue thread staging its next layer's
 *                            interval bounds in shared memory while the tensor
 *                            core runs (the default otherwise, where it fits;
 *                            1 where not); 1 or 2: tiles of up to 128 boxes
 *                            per CTA, the bounds read where needed.  Variants
 *                            0, 1, 2 give bit-identical results, and so do 3
 *                            and 4; the feature-major kernels sum each box's
 *                            constant in another order (within rounding).
 * -1 selects the built-in heuristic everywhere.  bab_set_variant returns
 * BAB_ERR_INVALID_ARG for an unknown kernel or variant; a variant whose tile
 * does not fit the network makes the later call fail with BAB_ERR_CUDA.
 */
/*
 * BF16 rollouts (BAB_PREC_BF16): after the tensor-core pass, ub[i] is the BF16
 * objective of box i's best sample.  With k = 0 (the default) every box's best
 * sample is then re-scored in FP32, so every ub is an FP32 objective value;
 * with k > 0 only the k boxes with the smallest BF16 ub (ties by id) are, the
 * others keep the BF16 value (about 1e-2 relative).  The incumbent is always
 * re-scored in FP64 from the box of smallest ub, so inc_val stays exact.
 * Errors: BAB_ERR_INVALID_ARG for k < 0.
 */
int bab_set_rescore_topk(bab_ctx *ctx, int k);

/*
 * Limit the context's scratch device memory to `bytes` (0: no limit, the
 * default).  The working set of a bound call grows with n x H x (hidden
 * width): interval bounds, the rounding-error helpers and, for the alpha
 * adjoint, the pre-relaxation coefficients and the concretizing point of every
 * box (about 1.3 MB a box for MLP 36-256x4-32 at H = 40).  Under a limit,
 * bab_bound_crown, bab_box_grad and bab_alpha_optimize bound the boxes in
 * consecutive chunks whose working set fits, recomputing each chunk's interval
 * bounds instead of holding them for all n; every box is bounded on its own,
 * so the results are bit-identical to one pass.  With d_n the device count is
 * read relative to each chunk's first row.  A scratch larger than the new
 * limit is freed at once (the call synchronises the device then).  No
 * counterpart in the paper (a memory policy of this library).
 * Errors: BAB_ERR_INVALID_ARG (null context); a later call whose single box
 * needs more than the limit returns BAB_ERR_OOM.
 */
int bab_set_scratch_limit(bab_ctx *ctx, size_t bytes);

/*
 * Arithmetic of the interval bounds (IBP, the intermediate bounds that Lemma 1
 * of Appendix B.1 relaxes) of every later bound call on this context.
 * BAB_PREC_FP32 (the default): FP32 sums with directed rounding, each input's
 * endpoint picked by the weight's sign.  BAB_PREC_BF16X3: on the tensor cores,
 * each layer's input in centre-radius form, W c and |W| r as 3-term BF16 split
 * products and |W| (|c| + r) as one BF16 product, the intervals widened by
 * gamma_split(K) |W| (|c| + r) (about 5e-5 of it): sound, and containing the
 * exact interval bounds, but wider than the FP32 ones by that margin per layer.
 * BAB_PREC_TF32X3: the same products from TF32 halves (16 boxes a tile), the
 * widening gamma_tf32(K) |W| (|c| + r) = (3.1 * 2^-22 + K 2^-23 / (1 - K 2^-23))
 * |W| (|c| + r), K the layer's inputs rounded up to 8: about a quarter of the
 * BF16 split's at K = 128, the accumulation term then dominating.
 * The weights are streamed through shared memory, so the network need not fit
 * there.  Squared-distance cost only (other costs keep the FP32 intervals).
 * No counterpart in the paper beyond Lemma 1's input.
 * Errors: BAB_ERR_INVALID_ARG (unknown precision), BAB_ERR_UNSUPPORTED
 * (BF16X3 or TF32X3 with a batch of several problems, or a width above 256).
 */
int bab_set_interval_precision(bab_ctx *ctx, int precision);

#define BAB_KERNEL_ROLLOUT_FP32 0
#define BAB_KERNEL_ALPHA_FUSED 1
#define BAB_KERNEL_ROLLOUT_TC 2
#define BAB_KERNEL_CROWN_TC 3
int bab_set_variant(bab_ctx *ctx, int kernel, int variant);
int bab_get_variant(bab_ctx *ctx, int kernel, int *variant);

/*
 * Times every variant of every kernel above on this problem (n boxes given as
 * for bab_rollout, `samples` rollouts each, alpha_steps Adam steps when > 0;
 * 3 timed runs after a warm-up, CUDA events on `stream`) and keeps the
 * fastest in ctx for later calls.  Synchronises the stream, allocates and
 * frees temporary device buffers, and must not be called while the stream is
 * being captured (BAB_ERR_INVALID_ARG).  Results of the timed calls are
 * discarded; the context's incumbent arguments are not touched.
 */
int bab_autotune(bab_ctx *ctx, const float *x0, const float *goal, int horizon, float rho, const float *lo,
                 const float *hi, const uint64_t *id, int n, int samples, int alpha_steps, void *stream);

/*
 * The FP32 FMA rate of the current GPU in TFLOP/s (2 FLOP per FMA), measured
 * with CUDA events on `stream`: independent FMA chains in every thread of two
 * 1024-thread CTAs per SM, best of three timed runs after a warm-up.  No
 * counterpart in the paper: it is the roof of the kernels that run on CUDA
 * cores (FP32 rollouts, interval bounds, FP32 CROWN), as the measured copy
 * bandwidth and BF16 GEMM rate are the roofs of the others.  Synchronises
 * `stream`.
 *   tflops         host double: scalar FMA rate (fma.rn.f32).
 *   tflops_paired  host double (nullable): rate of paired FMAs (fma.rn.f32x2).
 * Errors: BAB_ERR_INVALID_ARG (tflops NULL), BAB_ERR_CUDA.
 */
int bab_probe_fp32_peak(double *tflops, double *tflops_paired, void *stream);

/* Size of the fixed device working area of bab_bound_crown_static. */
#define BAB_STATIC_SCRATCH_BYTES (16u << 20)

/*
 * bab_bound_crown without any device allocation.  The paper has no
 * counterpart: this is a deployment variant of the CROWN bound above.
 *
 * It is for callers that may not call cudaMalloc (or cudaFree, which also
 * synchronises the device) when they need a bound: for example a plugin
 * whose enqueue step runs inside a host framework that owns all device
 * memory, or a real-time planning loop that must not allocate once it runs.
 * It takes no context (creating one allocates).  The network comes as a
 * DEVICE pointer in the layout of bab_load_dynamics, and all working memory
 * (padded weight images, interval bounds, rounding-error helpers) lives in
 * one fixed array of BAB_STATIC_SCRATCH_BYTES inside the library.  A GPU
 * holds the array from this entry point's first call on it until the
 * process exits.
 *   n_layers, dims (HOST int[L+1]), state_dim, action_dim: as bab_load_dynamics.
 *   params     DEVICE float array, packed W_1, b_1, ..., W_L, b_L (caller-owned).
 *   x0, goal, horizon, rho, lo, hi, n: as bab_bound_crown (adaptive slopes,
 *              FP32 arithmetic; d_n is not supported).
 *   lb, margin device float[n] (margin nullable): as bab_bound_crown.
 * The call needs 4 * (2 * image + n * H * (3 * sumh + s) + 2 * n * (H + 1) * s)
 * bytes (image = the padded network, about the parameter count); if that
 * exceeds BAB_STATIC_SCRATCH_BYTES it returns BAB_ERR_SHAPE before any
 * device work (sizes that large are refused before any product of them is
 * formed).  The first call on a device (with that device current) looks up
 * the array's device address and loads the entry point's kernels; under
 * CUDA's lazy module loading that first call may itself allocate device
 * memory.  So make one warm-up call per device first, with n = 0 (it does
 * only this set-up and returns BAB_OK), before the section that must not
 * allocate and before any stream capture.  All calls share the one array, so calls whose GPU work overlaps
 * (on different streams or host threads) race: order them on one stream.
 * Errors: BAB_ERR_INVALID_ARG, BAB_ERR_SHAPE, BAB_ERR_UNSUPPORTED (device
 * index >= 64), BAB_ERR_CUDA.  There is no context, so no bab_last_error.
 */
int bab_bound_crown_static(int n_layers, const int *dims, const float *params, int state_dim, int action_dim,
                           const float *x0, const float *goal, int horizon, float rho, const float *lo,
                           const float *hi, int n, float *lb, float *margin, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BAB_H */
