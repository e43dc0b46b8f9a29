/*
 * bab_oracle.c -- plain, slow FP64 CPU oracle for the bounding hot path of
 * BaB-ND (branch-and-bound planning over neural dynamics, arXiv 2412.09584).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker, not the product: only
 * the test suite, the package's smoke() check and the CPU-baseline and
 * reference legs of the benchmark may load it.  It shares no code, header, table or helper with the
 * CUDA library (paper_2412_09584_gb300/csrc), and the CUDA library never calls it.
 *
 * Everything is written as straight loops in double precision, in the order
 * the paper states the method, so that each function can be checked against
 * the paper by eye:
 *
 *   oracle_objective      Section 3 "Formulation", Eq. (trajop): the H-step
 *                         unrolled dynamics x_{t+1} = x_t + f(x_t, u_t) and the
 *                         summed cost, flattened to f(u) with d = kH.
 *   oracle_rollout        Section 3.3 (batch_search) with uniform sampling: the
 *                         best sampled objective of each box, an upper bound.
 *   oracle_ibp            interval bound propagation of the pre-activation
 *                         bounds (the intermediate bounds Lemma 1 needs).
 *   oracle_crown          Appendix B.1: Lemma 1 (ReLU relaxation), Theorem 1
 *                         (backward propagation of a linear lower bound) and
 *                         Theorem 2 (concretization) in box form.
 *   oracle_alpha_grad     d(lower bound)/d(alpha) for the free lower slopes of
 *                         Lemma 1, by a forward pass of the relaxed network.
 *   oracle_search_bounds  search-integrated (empirical) intermediate bounds,
 *                         Section 3.2 approach 2.
 *   oracle_crown_given    CROWN with given intermediate bounds and propagation
 *                         early-stop, Section 3.2 approach 1 / Algorithm 3.
 *   oracle_crown_margin   the CROWN bound with the outward rounding margin of
 *                         an FP32 or split-BF16 evaluation (the paper is silent
 *                         on floating point: a reading, see margin_gamma).
 *   oracle_box_grad       d(lower bound)/d(box faces), through the relaxation
 *                         choices and the interval bounds.
 *   oracle_adam_ascent    projected Adam ascent on alpha.
 *   oracle_prune_branch   Section 3 overview (prune when lower > incumbent),
 *                         Section 3.1 batch_pick_out and batch_split (bisection
 *                         of the widest dimension); oracle_prune_branch_heuristic
 *                         with the softmax pick-out (oracle_pick_key) and given
 *                         split dimensions (oracle_split_dims: the sample-
 *                         imbalance score).
 *   oracle_synth_*        Section 4, synthetic example: f(u) = sum 5 u_i^2 +
 *                         cos(50 u_i); its sampled search and the exact per-
 *                         term interval bound.
 *   oracle_cem            Section 3.3 batch_search with the cross-entropy
 *                         method, warm-started from the parent's best input;
 *                         it ranks samples by oracle_objective_f32 (the
 *                         objective in FP32, the precision the search decides
 *                         in), which is pinned to the FP64 objective.
 *
 * Layout conventions (these are the public conventions of the library too):
 *   network: L linear layers, dims[0] = s + k, dims[L] = s; params holds, for
 *            l = 1..L in order, W_l as a row-major dims[l] x dims[l-1] matrix
 *            followed by b_l (dims[l]).  ReLU follows layers 1..L-1.
 *   actions: u is t-major, u[t*k + j], t = 0..H-1 (Section 3, flattening).
 *   hidden : per time step the hidden pre-activations of layers 1..L-1 are
 *            concatenated (sumh values); per-box arrays are [H][sumh].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_LAYERS 16
#define ORC_MAX_WIDTH 1024

typedef struct {
    int L;
    int dims[ORC_MAX_LAYERS + 1];
    const double *W[ORC_MAX_LAYERS + 1];
    const double *b[ORC_MAX_LAYERS + 1];
    int hoff[ORC_MAX_LAYERS + 1]; /* offset of hidden layer l in the [sumh] vector */
    int sumh;
    int s, k;
} onet;

/* Returns 0 on success, -1 if the shapes are outside the oracle's limits. */
static int onet_init(onet *N, int L, const int *dims, const double *params, int s, int k)
{
    if (L < 1 || L > ORC_MAX_LAYERS || dims[0] != s + k || dims[L] != s) return -1;
    N->L = L;
    N->s = s;
    N->k = k;
    size_t off = 0;
    int h = 0;
    for (int l = 0; l <= L; ++l) {
        if (dims[l] < 1 || dims[l] > ORC_MAX_WIDTH) return -1;
        N->dims[l] = dims[l];
    }
    for (int l = 1; l <= L; ++l) {
        N->W[l] = params + off;
        off += (size_t)dims[l] * dims[l - 1];
        N->b[l] = params + off;
        off += dims[l];
        N->hoff[l] = h;
        if (l < L) h += dims[l];
    }
    N->sumh = h;
    return 0;
}

int oracle_param_count(int L, const int *dims)
{
    int n = 0;
    for (int l = 1; l <= L; ++l) n += dims[l] * dims[l - 1] + dims[l];
    return n;
}

int oracle_sumh(int L, const int *dims)
{
    int h = 0;
    for (int l = 1; l < L; ++l) h += dims[l];
    return h;
}

/* ------------------------------------------------------------------------ */
/* Task costs (Appendix D.4)                                                  */
/* ------------------------------------------------------------------------ */

/*
 * The state cost c(x_t) of Eq. (trajop), t = 1..H.  Kind 0 (default):
 * ||x_t - g||^2.  Kind 1, the pushing-with-obstacles cost of Appendix D.4
 * (Eq. pushing_cost): w_t ||x_t - g|| + lambda sum_o [ReLU(s_o - ||p_t - p_o||)
 * + sum_i ReLU(s_o - ||x_t^(i) - p_o||)], where the state holds s / 2 planar
 * keypoints x_t^(i) = (x_{t,2i}, x_{t,2i+1}), the action is the planar pusher
 * motion (k = 2) and p_t = p_0 + u_0 + ... + u_{t-1} is the pusher position
 * after t moves.  Both kinds add rho ||u_t||^2.  oracle_set_cost selects it
 * for every function of this file.
 */
#define ORC_MAX_OBS 8
#define ORC_MAX_H 4096

typedef struct {
    int kind;
    int H;
    double w[ORC_MAX_H + 1]; /* w[t], t = 1..H */
    double lambda;
    int n_obs;
    double ox[ORC_MAX_OBS], oy[ORC_MAX_OBS], os[ORC_MAX_OBS];
    double p0[2];
} ocost_t;

static ocost_t g_cost;

/* kind 0: squared distance; kind 1: w [H] (w_1..w_H), lambda, obstacles [n_obs][3] (x, y, size), p0 [2]. */
int oracle_set_cost(int kind, int H, const double *w, double lambda, int n_obs, const double *obs, const double *p0)
{
    memset(&g_cost, 0, sizeof(g_cost));
    if (kind == 0) return 0;
    if (kind != 1 || H < 1 || H > ORC_MAX_H || n_obs < 0 || n_obs > ORC_MAX_OBS) return -1;
    g_cost.kind = 1;
    g_cost.H = H;
    for (int t = 1; t <= H; ++t) g_cost.w[t] = w[t - 1];
    g_cost.lambda = lambda;
    g_cost.n_obs = n_obs;
    for (int o = 0; o < n_obs; ++o) {
        g_cost.ox[o] = obs[3 * o];
        g_cost.oy[o] = obs[3 * o + 1];
        g_cost.os[o] = obs[3 * o + 2];
    }
    g_cost.p0[0] = p0[0];
    g_cost.p0[1] = p0[1];
    return 0;
}

static double sq_min(double lo, double hi);
static double relu_d(double v) { return v > 0.0 ? v : 0.0; }

/* the state cost at step t (1..H) of state x with pusher position p */
static double state_cost(int t, int s, const double *x, const double *goal, const double *p)
{
    double c = 0.0;
    if (g_cost.kind == 0) {
        for (int i = 0; i < s; ++i) c += (x[i] - goal[i]) * (x[i] - goal[i]);
        return c;
    }
    double ss = 0.0;
    for (int i = 0; i < s; ++i) ss += (x[i] - goal[i]) * (x[i] - goal[i]);
    c = g_cost.w[t] * sqrt(ss);
    for (int o = 0; o < g_cost.n_obs; ++o) {
        c += g_cost.lambda * relu_d(g_cost.os[o] - hypot(p[0] - g_cost.ox[o], p[1] - g_cost.oy[o]));
        for (int i = 0; 2 * i + 1 < s; ++i)
            c += g_cost.lambda * relu_d(g_cost.os[o] - hypot(x[2 * i] - g_cost.ox[o], x[2 * i + 1] - g_cost.oy[o]));
    }
    return c;
}

/* the largest distance from (px, py) to the box [l0, u0] x [l1, u1] (at a vertex) */
static double max_dist(double l0, double u0, double l1, double u1, double px, double py)
{
    double a = fmax(fabs(l0 - px), fabs(u0 - px)), b = fmax(fabs(l1 - py), fabs(u1 - py));
    return hypot(a, b);
}

/* min over the box x in [xl, xu], p in [pl, pu] of the state cost at step t (each term on its own) */
static double state_cost_min(int t, int s, const double *xl, const double *xu, const double *goal, const double *pl,
                             const double *pu)
{
    double c = 0.0;
    if (g_cost.kind == 0) {
        for (int i = 0; i < s; ++i) c += sq_min(xl[i] - goal[i], xu[i] - goal[i]);
        return c;
    }
    double ss = 0.0; /* squared distance from g to the box */
    for (int i = 0; i < s; ++i) {
        double e = goal[i] < xl[i] ? xl[i] - goal[i] : (goal[i] > xu[i] ? goal[i] - xu[i] : 0.0);
        ss += e * e;
    }
    c = g_cost.w[t] * sqrt(ss);
    for (int o = 0; o < g_cost.n_obs; ++o) {
        c += g_cost.lambda * relu_d(g_cost.os[o] - max_dist(pl[0], pu[0], pl[1], pu[1], g_cost.ox[o], g_cost.oy[o]));
        for (int i = 0; 2 * i + 1 < s; ++i)
            c += g_cost.lambda *
                 relu_d(g_cost.os[o] - max_dist(xl[2 * i], xu[2 * i], xl[2 * i + 1], xu[2 * i + 1], g_cost.ox[o], g_cost.oy[o]));
    }
    return c;
}

/*
 * A linear lower bound a . q + b of ReLU(size - ||q - c||) over the box
 * [l0, u0] x [l1, u1]: h(q) = size - ||q - c|| is concave, so any affine
 * function below h at the four vertices is below h on the box; a is the
 * gradient of h at the box centre (0 if the centre is c) and b the largest
 * offset that keeps a . v + b <= h(v) at every vertex.  ReLU(h) >= h >= a . q + b
 * and ReLU(h) >= 0: the affine bound is used where it is positive at the box
 * centre (returns 1), else the bound 0 (returns 0, a = b = 0).
 */
int oracle_relu_dist_lower(double l0, double u0, double l1, double u1, double cx, double cy, double size,
                           double *a0, double *a1, double *b);
static int relu_dist_lower(double l0, double u0, double l1, double u1, double cx, double cy, double size, double *a0,
                           double *a1, double *b)
{
    return oracle_relu_dist_lower(l0, u0, l1, u1, cx, cy, size, a0, a1, b);
}
int oracle_relu_dist_lower(double l0, double u0, double l1, double u1, double cx, double cy, double size,
                           double *a0, double *a1, double *b)
{
    double mx = 0.5 * (l0 + u0), my = 0.5 * (l1 + u1);
    double dx = mx - cx, dy = my - cy, nd = hypot(dx, dy);
    double g0 = nd > 0.0 ? -dx / nd : 0.0, g1 = nd > 0.0 ? -dy / nd : 0.0;
    double vx[4] = {l0, u0, l0, u0}, vy[4] = {l1, l1, u1, u1};
    double bb = INFINITY;
    for (int v = 0; v < 4; ++v) {
        double off = size - hypot(vx[v] - cx, vy[v] - cy) - (g0 * vx[v] + g1 * vy[v]);
        if (off < bb) bb = off;
    }
    if (g0 * mx + g1 * my + bb > 0.0) {
        *a0 = g0;
        *a1 = g1;
        *b = bb;
        return 1;
    }
    *a0 = *a1 = *b = 0.0;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Objective (Section 3, Eq. trajop)                                          */
/* ------------------------------------------------------------------------ */

/*
 * One step of the residual dynamics x_{t+1} = x_t + N([x_t; u_t]) with N the
 * ReLU MLP.  pre (nullable) receives the hidden pre-activations (sumh values).
 */
static void step_forward(const onet *N, const double *x, const double *u, double *xnext, double *pre)
{
    double a[ORC_MAX_WIDTH], z[ORC_MAX_WIDTH];
    for (int i = 0; i < N->s; ++i) a[i] = x[i];
    for (int j = 0; j < N->k; ++j) a[N->s + j] = u[j];
    for (int l = 1; l <= N->L; ++l) {
        int no = N->dims[l], ni = N->dims[l - 1];
        for (int r = 0; r < no; ++r) {
            double acc = N->b[l][r];
            for (int c = 0; c < ni; ++c) acc += N->W[l][(size_t)r * ni + c] * a[c];
            z[r] = acc;
        }
        if (l < N->L) {
            for (int r = 0; r < no; ++r) {
                if (pre) pre[N->hoff[l] + r] = z[r];
                a[r] = z[r] > 0.0 ? z[r] : 0.0;
            }
        }
    }
    for (int i = 0; i < N->s; ++i) xnext[i] = x[i] + z[i];
}

/*
 * f(u) = sum_{t=1..H} c(x_t) + rho * sum_{t=0..H-1} ||u_t||^2, c the state
 * cost (||x_t - goal||^2 unless oracle_set_cost chose another).
 * traj (nullable) receives x_0..x_H ([H+1][s]); pre (nullable) the hidden
 * pre-activations of every step ([H][sumh]).
 */
double oracle_objective(int L, const int *dims, const double *params, int s, int k, int H, double rho,
                        const double *x0, const double *goal, const double *u, double *traj, double *pre)
{
    onet N;
    if (onet_init(&N, L, dims, params, s, k)) return NAN;
    double x[ORC_MAX_WIDTH], xn[ORC_MAX_WIDTH];
    for (int i = 0; i < s; ++i) x[i] = x0[i];
    if (traj) memcpy(traj, x0, sizeof(double) * s);
    double f = 0.0;
    double p[2] = {g_cost.p0[0], g_cost.p0[1]};
    for (int t = 0; t < H; ++t) {
        const double *ut = u + (size_t)t * k;
        step_forward(&N, x, ut, xn, pre ? pre + (size_t)t * N.sumh : NULL);
        for (int j = 0; j < k; ++j) f += rho * ut[j] * ut[j];
        if (g_cost.kind == 1) {
            p[0] += ut[0];
            p[1] += ut[1];
        }
        f += state_cost(t + 1, s, xn, goal, p);
        for (int i = 0; i < s; ++i) x[i] = xn[i];
        if (traj) memcpy(traj + (size_t)(t + 1) * s, x, sizeof(double) * s);
    }
    return f;
}

/* ------------------------------------------------------------------------ */
/* Sampled search (Section 3.3) with a counter-based generator               */
/* ------------------------------------------------------------------------ */

/*
 * SplitMix64 output function (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014): add the golden-ratio
 * increment, then two xor-shift-multiply rounds and a final xor-shift.
 */
uint64_t oracle_splitmix64(uint64_t state)
{
    uint64_t z = state + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/*
 * The uniform draw of sample m, coordinate j, of the box with identifier id:
 * chained SplitMix64 over (seed, id, m, j), top 24 bits as r in [0, 1), and
 * the sample u = lo + (hi - lo) * r formed in FP32 with one rounding per
 * operation (no fused multiply-add), so that every implementation that follows
 * this definition draws bit-identical samples.
 */
float oracle_sample(uint64_t seed, uint64_t id, uint32_t m, uint32_t j, float lo, float hi)
{
    uint64_t h = oracle_splitmix64(seed ^ oracle_splitmix64(id));
    h = oracle_splitmix64(h ^ ((uint64_t)m << 32 | (uint64_t)j));
    float r = (float)(h >> 40) * (1.0f / 16777216.0f);
    volatile float w = hi - lo;
    volatile float step = w * r;
    volatile float u = lo + step;
    return u;
}

/*
 * For each box i: draw M samples, evaluate f in FP64, and return the minimum
 * (ub[i]) with its argmin sample (best_u, [n][d]) and index (best_m).  Ties
 * go to the lowest m.
 */
int oracle_rollout(int L, const int *dims, const double *params, int s, int k, int H, double rho,
                   const double *x0, const double *goal, int n, const float *lo, const float *hi,
                   const uint64_t *id, int M, uint64_t seed, double *ub, float *best_u, int *best_m)
{
    onet N;
    if (onet_init(&N, L, dims, params, s, k)) return -1;
    int d = k * H;
    double *u = (double *)malloc(sizeof(double) * d);
    float *uf = (float *)malloc(sizeof(float) * d);
    for (int i = 0; i < n; ++i) {
        double best = INFINITY;
        int bm = -1;
        for (int m = 0; m < M; ++m) {
            for (int j = 0; j < d; ++j) {
                uf[j] = oracle_sample(seed, id[i], (uint32_t)m, (uint32_t)j, lo[(size_t)i * d + j],
                                      hi[(size_t)i * d + j]);
                u[j] = uf[j];
            }
            double f = oracle_objective(L, dims, params, s, k, H, rho, x0, goal, u, NULL, NULL);
            if (f < best || bm < 0) {
                best = f;
                bm = m;
                if (best_u) memcpy(best_u + (size_t)i * d, uf, sizeof(float) * d);
            }
        }
        ub[i] = best;
        if (best_m) best_m[i] = bm;
    }
    free(u);
    free(uf);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Interval bound propagation (intermediate bounds)                          */
/* ------------------------------------------------------------------------ */

/* min over s in [lo, hi] of s^2 */
static double sq_min(double lo, double hi)
{
    if (lo <= 0.0 && hi >= 0.0) return 0.0;
    return lo > 0.0 ? lo * lo : hi * hi;
}

/*
 * Interval bounds of one box through the unrolled dynamics.  Each layer maps
 * an input interval, in centre/radius form (c, r), to c' = W c + b and
 * r' = |W| r; the ReLU clamps both ends at zero; the next state interval is
 * the sum of the current state interval and the network output interval.
 * x_0 is known exactly.  Outputs per box: pre_lo/pre_hi [H][sumh], x_lo/x_hi
 * [H+1][s] (all nullable), and the interval lower bound of the objective.
 */
static double ibp_box(const onet *N, int H, double rho, const double *x0, const double *goal, const double *lo,
                      const double *hi, double *pre_lo, double *pre_hi, double *x_lo, double *x_hi)
{
    int s = N->s, k = N->k;
    double xl[ORC_MAX_WIDTH], xu[ORC_MAX_WIDTH];
    double c[ORC_MAX_WIDTH], r[ORC_MAX_WIDTH], cn[ORC_MAX_WIDTH], rn[ORC_MAX_WIDTH];
    double zl[ORC_MAX_WIDTH], zu[ORC_MAX_WIDTH];
    for (int i = 0; i < s; ++i) xl[i] = xu[i] = x0[i];
    if (x_lo) for (int i = 0; i < s; ++i) x_lo[i] = x_hi[i] = x0[i];
    double lb = 0.0;
    double pl[2] = {g_cost.p0[0], g_cost.p0[1]}, pu[2] = {g_cost.p0[0], g_cost.p0[1]}; /* pusher position box */
    for (int t = 0; t < H; ++t) {
        if (g_cost.kind == 1) {
            for (int j = 0; j < 2; ++j) {
                pl[j] += lo[t * k + j];
                pu[j] += hi[t * k + j];
            }
        }
        for (int i = 0; i < s; ++i) {
            c[i] = 0.5 * (xl[i] + xu[i]);
            r[i] = 0.5 * (xu[i] - xl[i]);
        }
        for (int j = 0; j < k; ++j) {
            double a = lo[t * k + j], bb = hi[t * k + j];
            c[s + j] = 0.5 * (a + bb);
            r[s + j] = 0.5 * (bb - a);
            lb += rho * sq_min(a, bb);
        }
        for (int l = 1; l <= N->L; ++l) {
            int no = N->dims[l], ni = N->dims[l - 1];
            for (int q = 0; q < no; ++q) {
                double cc = N->b[l][q], rr = 0.0;
                for (int p = 0; p < ni; ++p) {
                    double w = N->W[l][(size_t)q * ni + p];
                    cc += w * c[p];
                    rr += fabs(w) * r[p];
                }
                cn[q] = cc;
                rn[q] = rr;
                zl[q] = cc - rr;
                zu[q] = cc + rr;
            }
            if (l < N->L) {
                for (int q = 0; q < no; ++q) {
                    if (pre_lo) {
                        pre_lo[(size_t)t * N->sumh + N->hoff[l] + q] = zl[q];
                        pre_hi[(size_t)t * N->sumh + N->hoff[l] + q] = zu[q];
                    }
                    double al = zl[q] > 0.0 ? zl[q] : 0.0;
                    double au = zu[q] > 0.0 ? zu[q] : 0.0;
                    c[q] = 0.5 * (al + au);
                    r[q] = 0.5 * (au - al);
                }
            }
        }
        (void)cn;
        (void)rn;
        for (int i = 0; i < s; ++i) {
            xl[i] += zl[i];
            xu[i] += zu[i];
        }
        lb += state_cost_min(t + 1, s, xl, xu, goal, pl, pu);
        if (x_lo) {
            for (int i = 0; i < s; ++i) {
                x_lo[(size_t)(t + 1) * s + i] = xl[i];
                x_hi[(size_t)(t + 1) * s + i] = xu[i];
            }
        }
    }
    return lb;
}

int oracle_ibp(int L, const int *dims, const double *params, int s, int k, int H, double rho, const double *x0,
               const double *goal, int n, const double *lo, const double *hi, double *pre_lo, double *pre_hi,
               double *x_lo, double *x_hi, double *lb_ibp)
{
    onet N;
    if (onet_init(&N, L, dims, params, s, k)) return -1;
    int d = k * H;
    for (int i = 0; i < n; ++i) {
        double v = ibp_box(&N, H, rho, x0, goal, lo + (size_t)i * d, hi + (size_t)i * d,
                           pre_lo ? pre_lo + (size_t)i * H * N.sumh : NULL,
                           pre_hi ? pre_hi + (size_t)i * H * N.sumh : NULL,
                           x_lo ? x_lo + (size_t)i * (H + 1) * s : NULL,
                           x_hi ? x_hi + (size_t)i * (H + 1) * s : NULL);
        if (lb_ibp) lb_ibp[i] = v;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Relaxations                                                               */
/* ------------------------------------------------------------------------ */

/*
 * Tangent lower bound of s^2 at m: s^2 >= 2 m s - m^2 (exact at s = m).
 * Chord upper bound of s^2 on [L, U]: s^2 <= (L + U) s - L U (exact at L, U).
 */
double oracle_sq_tangent(double m, double s) { return 2.0 * m * s - m * m; }
double oracle_sq_chord(double L, double U, double s) { return (L + U) * s - L * U; }

/*
 * Lemma 1 for one neuron with pre-activation bounds [l, u]: the slope D and
 * intercept c of the lower (which = 0) or upper (which = 1) linear bound of
 * ReLU.  Active iff l >= 0, inactive iff u <= 0, otherwise unstable; the lower
 * bound of an unstable neuron is alpha * z (intercept 0) and the upper bound
 * is the chord u (z - l) / (u - l).
 */
void oracle_relu_relax(double l, double u, double alpha, int which, double *D, double *c)
{
    if (l >= 0.0) {
        *D = 1.0;
        *c = 0.0;
    } else if (u <= 0.0) {
        *D = 0.0;
        *c = 0.0;
    } else if (which == 0) {
        *D = alpha;
        *c = 0.0;
    } else {
        *D = u / (u - l);
        *c = -u * l / (u - l);
    }
}

/* The adaptive lower slope of an unstable neuron: 1 if u >= -l, else 0. */
static double adaptive_alpha(double l, double u) { return u >= -l ? 1.0 : 0.0; }

/* min over u in [lo, hi] of mu u + rho u^2, with its minimiser. */
static double quad_min(double mu, double rho, double lo, double hi, double *arg)
{
    double u;
    if (rho > 0.0) {
        u = -mu / (2.0 * rho);
        if (u < lo) u = lo;
        if (u > hi) u = hi;
    } else {
        u = mu >= 0.0 ? lo : hi;
    }
    *arg = u;
    return mu * u + rho * u * u;
}

/* ------------------------------------------------------------------------ */
/* CROWN backward bound (Appendix B.1, Lemma 1 / Theorem 1 / Theorem 2)      */
/* ------------------------------------------------------------------------ */

typedef struct {
    double lb;          /* concretized lower bound */
    double lin_const;   /* f(u) >= lin_const + mu . u + rho ||u||^2 on the box */
    double scale;       /* sum of |each term added into the bound|: the magnitude rounding errors scale with */
    double margin;      /* the outward rounding margin of an FP32 / split-BF16 evaluation (see margin_gamma) */
} crown_out;

/*
 * Outward rounding margin (the paper is silent on floating point; the bound
 * stays sound if every coefficient error is charged against the largest
 * magnitude its variable can take on the box).  A product of a coefficient
 * row A' (K = d_l entries) with W_l evaluated in floating point has, in each
 * output j, an error of at most gamma * sum_k |A'_k| |W_kj| (Higham,
 * "Accuracy and Stability of Numerical Algorithms", 2nd ed., Section 3.1);
 * charged against max |a_j| over the interval of the layer's input a, the
 * bound moves by at most gamma * sum_k |A'_k| S_k with
 * S_k = sum_j |W_kj| max|a_j|.  gamma per arithmetic (prec):
 *   0: FP32 products over K = d_l rounded up to a multiple of 4 terms,
 *      gamma_K = K u / (1 - K u), u = 2^-24;
 *   1: 3-term BF16 split (a_hi b_hi + a_hi b_lo + a_lo b_hi) with FP32
 *      accumulation over K = d_l rounded up to a multiple of 16 terms:
 *      3.1 * 2^-16 for the BF16 halves of both operands and the dropped
 *      lo * lo term, plus gamma_K with unit 2^-23 (an accumulator that may
 *      truncate).
 *   2: 3-term TF32 split, the same with halves of 11 significant bits
 *      (each operand's residual and the dropped lo * lo term at most about
 *      2^-22 of |a| |b|) over K = d_l rounded up to a multiple of 8 terms:
 *      3.1 * 2^-22 plus gamma_K with unit 2^-23.
 * Each other rounded coefficient operation costs at most 2^-23 (twice the
 * unit roundoff) of its magnitude times the largest magnitude of its
 * variable: the relaxation product A D of a neuron whose slope is neither 0
 * nor 1 (variable z in [l, u]), the state update lam + A_x + a_t (variable
 * x_t), and, for rho > 0, the choice of a face when the unconstrained
 * minimiser u_c of mu u + rho u^2 lies outside the box: rho (2^-23 u_c)^2.
 */
static double margin_gamma(int prec, int d)
{
    if (prec == 1) {
        double K = (double)((d + 15) / 16 * 16), u = ldexp(1.0, -23);
        return 3.1 * ldexp(1.0, -16) + K * u / (1.0 - K * u);
    }
    if (prec == 2) {
        double K = (double)((d + 7) / 8 * 8), u = ldexp(1.0, -23);
        return 3.1 * ldexp(1.0, -22) + K * u / (1.0 - K * u);
    }
    double K = (double)((d + 3) / 4 * 4), u = ldexp(1.0, -24);
    return K * u / (1.0 - K * u);
}

/* S_q = sum_p |W_l[q][p]| max|a_p| over the interval of layer l's input at step t (layer 1: [x_t; u_t]). */
static void margin_rowsums(const onet *N, int l, int t, const double *lo, const double *hi, const double *pre_hi,
                           const double *x_lo, const double *x_hi, double *S)
{
    int s = N->s, k = N->k, no = N->dims[l], ni = N->dims[l - 1];
    double amax[ORC_MAX_WIDTH];
    for (int p = 0; p < ni; ++p) {
        if (l == 1) {
            if (p < s) amax[p] = fmax(fabs(x_lo[(size_t)t * s + p]), fabs(x_hi[(size_t)t * s + p]));
            else amax[p] = fmax(fabs(lo[t * k + p - s]), fabs(hi[t * k + p - s]));
        } else {
            double u = pre_hi[(size_t)t * N->sumh + N->hoff[l - 1] + p];
            amax[p] = u > 0.0 ? u : 0.0;  /* ReLU output in [max(l, 0), max(u, 0)] */
        }
    }
    for (int q = 0; q < no; ++q) {
        double acc = 0.0;
        for (int p = 0; p < ni; ++p) acc += fabs(N->W[l][(size_t)q * ni + p]) * amax[p];
        S[q] = acc;
    }
}

/*
 * The bound of one box.  The cost term ||x_t - g||^2 (t >= 1) is bounded below
 * by its tangent at the midpoint m of the interval of s = x_{t,i} - g_i, which
 * turns the objective into a linear function of x_1..x_H plus the exact
 * rho ||u||^2.  The coefficient lam of x_{t+1} is then carried backward through
 * step t: lam . x_{t+1} = lam . x_t + lam . N([x_t; u_t]), and lam . N is
 * bounded below by Theorem 1 (last layer: A = lam; then, per hidden layer
 * from the top: relax each ReLU by Lemma 1, choosing the lower bound where the
 * coefficient is >= 0 and the upper bound where it is < 0, then multiply by
 * W_l), which leaves coefficients on x_t and u_t.  x_0 is a constant.
 * Theorem 2 in box form concretizes the remaining function of u.
 *
 * alpha (nullable, [H][sumh]) gives the lower slopes; NULL means adaptive.
 * Outputs (all nullable): mu [d] (coefficients of u), ustar [d] (concretizing
 * point), A_pre [H][sumh] (the coefficient of each ReLU output before its
 * relaxation), and tangent coefficients atan [H+1][s] (row 0 unused).
 */
static crown_out crown_box(const onet *N, int H, double rho, const double *x0, const double *goal,
                           const double *lo, const double *hi, const double *pre_lo, const double *pre_hi,
                           const double *x_lo, const double *x_hi, const double *alpha, double *mu,
                           double *ustar, double *A_pre, double *atan, int t_stop, int prec)
{
    int s = N->s, k = N->k, L = N->L, sumh = N->sumh;
    double lam[ORC_MAX_WIDTH], A[ORC_MAX_WIDTH], An[ORC_MAX_WIDTH], S[ORC_MAX_WIDTH];
    double cst = 0.0, cabs = 0.0, marg = 0.0;
    const double two_u = ldexp(1.0, -23);
    double *mu_loc = (double *)calloc((size_t)k * H, sizeof(double));

    /* linear lower bounds a_t . x_t + const of the state cost at the steps the backward pass carries
       (t > t_stop); the terms at or before the early-stop step are bounded on their intervals.  Squared
       distance: the tangent of s^2 at the midpoint m of the interval of s = x_{t,i} - g_i, a = 2 m, constant
       -2 m g - m^2.  Pushing with obstacles: w ||x - g|| >= w ghat . (x - g) with ghat = m / ||m|| (Cauchy-
       Schwarz; 0 if m = 0), and each obstacle term by relu_dist_lower on its box; the pusher terms are linear in
       p_t = p_0 + u_0 + ... + u_{t-1} and so add coefficients bp_t to every earlier action. */
    double *a = (double *)calloc((size_t)(H + 1) * s, sizeof(double));
    double *mu_extra = (double *)calloc((size_t)k * H, sizeof(double));
    double pl[2] = {g_cost.p0[0], g_cost.p0[1]}, pu[2] = {g_cost.p0[0], g_cost.p0[1]};
    for (int t = 1; t <= H; ++t) {
        const double *xl_t = x_lo + (size_t)t * s, *xu_t = x_hi + (size_t)t * s;
        if (g_cost.kind == 1) {
            for (int j = 0; j < 2; ++j) {
                pl[j] += lo[(t - 1) * k + j];
                pu[j] += hi[(t - 1) * k + j];
            }
        }
        if (t <= t_stop) {
            double v = state_cost_min(t, s, xl_t, xu_t, goal, pl, pu);
            cst += v;
            cabs += fabs(v);
            continue;
        }
        if (g_cost.kind == 0) {
            for (int i = 0; i < s; ++i) {
                double Ls = xl_t[i] - goal[i], Us = xu_t[i] - goal[i];
                double m = 0.5 * (Ls + Us);
                a[(size_t)t * s + i] = 2.0 * m;
                cst += -2.0 * m * goal[i] - m * m;
                cabs += fabs(2.0 * m * goal[i]) + m * m;
            }
            continue;
        }
        double m[ORC_MAX_WIDTH], nm = 0.0;
        for (int i = 0; i < s; ++i) {
            m[i] = 0.5 * (xl_t[i] + xu_t[i]) - goal[i];
            nm += m[i] * m[i];
        }
        nm = sqrt(nm);
        if (nm > 0.0) {
            for (int i = 0; i < s; ++i) {
                double gi = g_cost.w[t] * m[i] / nm;
                a[(size_t)t * s + i] += gi;
                cst -= gi * goal[i];
                cabs += fabs(gi * goal[i]);
            }
        }
        for (int o = 0; o < g_cost.n_obs; ++o) {
            double a0, a1, b, lam_ = g_cost.lambda;
            if (relu_dist_lower(pl[0], pu[0], pl[1], pu[1], g_cost.ox[o], g_cost.oy[o], g_cost.os[o], &a0, &a1, &b)) {
                /* lam (a . p_t + b) = lam (a . p_0 + b) + lam a . (u_0 + ... + u_{t-1}) */
                for (int tau = 0; tau < t; ++tau) {
                    mu_extra[tau * k] += lam_ * a0;
                    mu_extra[tau * k + 1] += lam_ * a1;
                }
                cst += lam_ * (a0 * g_cost.p0[0] + a1 * g_cost.p0[1] + b);
                cabs += fabs(lam_ * (a0 * g_cost.p0[0] + a1 * g_cost.p0[1] + b));
            }
            for (int i = 0; 2 * i + 1 < s; ++i) {
                if (relu_dist_lower(xl_t[2 * i], xu_t[2 * i], xl_t[2 * i + 1], xu_t[2 * i + 1], g_cost.ox[o],
                                    g_cost.oy[o], g_cost.os[o], &a0, &a1, &b)) {
                    a[(size_t)t * s + 2 * i] += lam_ * a0;
                    a[(size_t)t * s + 2 * i + 1] += lam_ * a1;
                    cst += lam_ * b;
                    cabs += fabs(lam_ * b);
                }
            }
        }
    }
    for (int i = 0; i < s; ++i) lam[i] = a[(size_t)H * s + i];

    for (int t = H - 1; t >= t_stop; --t) {
        /* last linear layer: A = lam on z_L */
        int nL = N->dims[L], nLm = N->dims[L - 1];
        for (int q = 0; q < nL; ++q) A[q] = lam[q];
        for (int q = 0; q < nL; ++q) {
            cst += A[q] * N->b[L][q];
            cabs += fabs(A[q] * N->b[L][q]);
        }
        margin_rowsums(N, L, t, lo, hi, pre_hi, x_lo, x_hi, S);
        for (int q = 0; q < nL; ++q) marg += margin_gamma(prec, nL) * fabs(A[q]) * S[q];
        for (int p = 0; p < nLm; ++p) {
            double acc = 0.0;
            for (int q = 0; q < nL; ++q) acc += A[q] * N->W[L][(size_t)q * nLm + p];
            An[p] = acc;
        }
        for (int p = 0; p < nLm; ++p) A[p] = An[p];
        /* hidden layers l = L-1 .. 1 */
        for (int l = L - 1; l >= 1; --l) {
            int no = N->dims[l], ni = N->dims[l - 1];
            for (int q = 0; q < no; ++q) {
                size_t idx = (size_t)t * sumh + N->hoff[l] + q;
                double zl = pre_lo[idx], zu = pre_hi[idx];
                double al = alpha ? alpha[idx] : adaptive_alpha(zl, zu);
                double D, c;
                if (A_pre) A_pre[idx] = A[q];
                oracle_relu_relax(zl, zu, al, A[q] >= 0.0 ? 0 : 1, &D, &c);
                cst += A[q] * c;
                cabs += fabs(A[q] * c);
                A[q] *= D;
                if (D != 0.0 && D != 1.0) marg += two_u * fabs(A[q]) * fmax(-zl, zu);
            }
            for (int q = 0; q < no; ++q) {
                cst += A[q] * N->b[l][q];
                cabs += fabs(A[q] * N->b[l][q]);
            }
            margin_rowsums(N, l, t, lo, hi, pre_hi, x_lo, x_hi, S);
            for (int q = 0; q < no; ++q) marg += margin_gamma(prec, no) * fabs(A[q]) * S[q];
            for (int p = 0; p < ni; ++p) {
                double acc = 0.0;
                for (int q = 0; q < no; ++q) acc += A[q] * N->W[l][(size_t)q * ni + p];
                An[p] = acc;
            }
            for (int p = 0; p < ni; ++p) A[p] = An[p];
        }
        /* A is now on [x_t; u_t] */
        for (int j = 0; j < k; ++j) mu_loc[t * k + j] = A[s + j];
        for (int i = 0; i < s; ++i) {
            double at = t >= 1 ? a[(size_t)t * s + i] : 0.0;
            double B = t >= 1 ? fmax(fabs(x_lo[(size_t)t * s + i]), fabs(x_hi[(size_t)t * s + i])) : fabs(x0[i]);
            marg += two_u * (fabs(lam[i]) + fabs(A[i]) + fabs(at)) * B;
            lam[i] = lam[i] + A[i] + at;
        }
    }
    if (t_stop == 0) {
        for (int i = 0; i < s; ++i) {
            cst += lam[i] * x0[i];
            cabs += fabs(lam[i] * x0[i]);
        }
    } else {
        /* early stop: concretize the coefficient of x_{t_stop} on that state's interval (Theorem 2, box form) */
        for (int i = 0; i < s; ++i) {
            double a_ = lam[i] * x_lo[(size_t)t_stop * s + i], b_ = lam[i] * x_hi[(size_t)t_stop * s + i];
            double v = a_ < b_ ? a_ : b_;
            cst += v;
            cabs += fabs(v);
        }
    }

    for (int j = 0; j < k * H; ++j) mu_loc[j] += mu_extra[j];
    double lb = cst;
    for (int j = 0; j < k * H; ++j) {
        double arg;
        double v = quad_min(mu_loc[j], rho, lo[j], hi[j], &arg);
        lb += v;
        cabs += fabs(v);
        if (rho > 0.0) {
            double uc = -mu_loc[j] / (2.0 * rho);
            if (uc < lo[j] || uc > hi[j]) marg += rho * (two_u * uc) * (two_u * uc);
        }
        if (ustar) ustar[j] = arg;
        if (mu) mu[j] = mu_loc[j];
    }
    if (atan) memcpy(atan, a, sizeof(double) * (size_t)(H + 1) * s);
    free(a);
    free(mu_extra);
    free(mu_loc);
    /* the obstacle cost's margin (pusher coefficients) is not stated here */
    crown_out o = {lb, cst, cabs, g_cost.kind == 0 ? marg : NAN};
    return o;
}

/*
 * CROWN lower bound of each box, with IBP intermediate bounds.  Outputs (all
 * but lb nullable): lb [n], lin_coef [n][d] and lin_const [n] such that
 * f(u) >= lin_const + lin_coef . u + rho ||u||^2 on the box, ustar [n][d],
 * A_pre [n][H][sumh], and scale [n]: the sum of the absolute values of every
 * term added into the bound (tangent constants, A.b, A.c, lam.x0 and the
 * concretized terms), the magnitude that rounding errors of any evaluation
 * order scale with; tests use it as the tolerance scale.
 */
int oracle_crown(int L, const int *dims, const double *params, int s, int k, int H, double rho, const double *x0,
                 const double *goal, int n, const double *lo, const double *hi, const double *alpha, double *lb,
                 double *lin_coef, double *lin_const, double *ustar, double *A_pre, double *scale)
{
    onet N;
    if (onet_init(&N, L, dims, params, s, k)) return -1;
    int d = k * H;
    size_t nh = (size_t)H * N.sumh, nx = (size_t)(H + 1) * s;
    double *pl = (double *)malloc(sizeof(double) * (nh ? nh : 1));
    double *pu = (double *)malloc(sizeof(double) * (nh ? nh : 1));
    double *xl = (double *)malloc(sizeof(double) * nx);
    double *xu = (double *)malloc(sizeof(double) * nx);
    for (int i = 0; i < n; ++i) {
        const double *bl = lo + (size_t)i * d, *bh = hi + (size_t)i * d;
        ibp_box(&N, H, rho, x0, goal, bl, bh, pl, pu, xl, xu);
        crown_out o = crown_box(&N, H, rho, x0, goal, bl, bh, pl, pu, xl, xu, alpha ? alpha + (size_t)i * nh : NULL,
                                lin_coef ? lin_coef + (size_t)i * d : NULL, ustar ? ustar + (size_t)i * d : NULL,
                                A_pre ? A_pre + (size_t)i * nh : NULL, NULL, 0, 0);
        lb[i] = o.lb;
        if (lin_const) lin_const[i] = o.lin_const;
        if (scale) scale[i] = o.scale;
    }
    free(pl);
    free(pu);
    free(xl);
    free(xu);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The paper's own bounding (Section 3.2, Appendix B.2)                      */
/* ------------------------------------------------------------------------ */

/*
 * Search-integrated bounds: per box, the minimum and maximum over the search's
 * samples (the same counter-based samples as oracle_rollout) of every hidden
 * pre-activation (pre_lo/pre_hi [n][H][sumh]) and of every state x_t
 * (x_lo/x_hi [n][H+1][s], x_0 exact).  Underestimates of the true ranges.
 */
int oracle_search_bounds(int L, const int *dims, const double *params, int s, int k, int H, double rho,
                         const double *x0, const double *goal, int n, const float *lo, const float *hi,
                         const uint64_t *id, int M, uint64_t seed, double *pre_lo, double *pre_hi, double *x_lo,
                         double *x_hi)
{
    onet N;
    if (onet_init(&N, L, dims, params, s, k)) return -1;
    int d = k * H, sumh = N.sumh;
    size_t nh = (size_t)H * sumh, nx = (size_t)(H + 1) * s;
    double *u = (double *)malloc(sizeof(double) * d);
    double *traj = (double *)malloc(sizeof(double) * nx);
    double *pre = (double *)malloc(sizeof(double) * (nh ? nh : 1));
    for (int i = 0; i < n; ++i) {
        double *pl = pre_lo + (size_t)i * nh, *pu = pre_hi + (size_t)i * nh;
        double *xl = x_lo + (size_t)i * nx, *xu = x_hi + (size_t)i * nx;
        for (size_t q = 0; q < nh; ++q) {
            pl[q] = INFINITY;
            pu[q] = -INFINITY;
        }
        for (size_t q = 0; q < nx; ++q) {
            xl[q] = INFINITY;
            xu[q] = -INFINITY;
        }
        for (int m = 0; m < M; ++m) {
            for (int j = 0; j < d; ++j)
                u[j] = oracle_sample(seed, id[i], (uint32_t)m, (uint32_t)j, lo[(size_t)i * d + j], hi[(size_t)i * d + j]);
            oracle_objective(L, dims, params, s, k, H, rho, x0, goal, u, traj, pre);
            for (size_t q = 0; q < nh; ++q) {
                if (pre[q] < pl[q]) pl[q] = pre[q];
                if (pre[q] > pu[q]) pu[q] = pre[q];
            }
            for (size_t q = 0; q < nx; ++q) {
                if (traj[q] < xl[q]) xl[q] = traj[q];
                if (traj[q] > xu[q]) xu[q] = traj[q];
            }
        }
    }
    free(u);
    free(traj);
    free(pre);
    return 0;
}

/*
 * CROWN with given intermediate bounds and propagation early-stop
 * (Algorithm 3 with the early-stop set S = {x_{t_stop}}): the cost terms after
 * step t_stop are tangent-linearised and carried backward through steps
 * H-1 .. t_stop, where the propagation stops and the remaining coefficient of
 * x_{t_stop} is concretized on that state's interval (Theorem 2, box form);
 * the cost terms at steps 1 .. t_stop are bounded on their intervals.  With
 * t_stop = 0 and the interval bounds of oracle_ibp this is oracle_crown; with
 * search-integrated bounds it is the paper's estimate, not a sound bound.
 * Adaptive lower slopes; outputs lb [n].
 */
int oracle_crown_given(int L, const int *dims, const double *params, int s, int k, int H, double rho,
                       const double *x0, const double *goal, int n, const double *lo, const double *hi,
                       const double *pre_lo, const double *pre_hi, const double *x_lo, const double *x_hi,
                       int t_stop, double *lb)
{
    onet N;
    if (onet_init(&N, L, dims, params, s, k)) return -1;
    if (t_stop < 0 || t_stop > H) return -1;
    int d = k * H;
    size_t nh = (size_t)H * N.sumh, nx = (size_t)(H + 1) * s;
    for (int i = 0; i < n; ++i) {
        crown_out o = crown_box(&N, H, rho, x0, goal, lo + (size_t)i * d, hi + (size_t)i * d, pre_lo + (size_t)i * nh,
                                pre_hi + (size_t)i * nh, x_lo + (size_t)i * nx, x_hi + (size_t)i * nx, NULL, NULL,
                                NULL, NULL, NULL, t_stop, 0);
        lb[i] = o.lb;
    }
    return 0;
}

/*
 * CROWN bound with its outward rounding margin (margin_gamma) for the
 * arithmetic `prec` (0: FP32 products, 1: 3-term BF16 split, 2: 3-term TF32 split), with given
 * intermediate bounds (pre_lo/pre_hi [n][H][sumh], x_lo/x_hi [n][H+1][s]) or,
 * when pre_lo is NULL, the interval bounds of oracle_ibp; alpha [n][H][sumh]
 * nullable (adaptive slopes).  Outputs per box: lb (exact FP64, no margin
 * subtracted), margin, scale (all but lb nullable).  The margin is stated for
 * the squared-distance cost (NaN otherwise).
 */
int oracle_crown_margin(int L, const int *dims, const double *params, int s, int k, int H, double rho,
                        const double *x0, const double *goal, int n, const double *lo, const double *hi,
                        const double *pre_lo, const double *pre_hi, const double *x_lo, const double *x_hi,
                        const double *alpha, int prec, double *lb, double *margin, double *scale)
{
    onet N;
    if (onet_init(&N, L, dims, params, s, k)) return -1;
    if (prec < 0 || prec > 2) return -1;
    int d = k * H;
    size_t nh = (size_t)H * N.sumh, nx = (size_t)(H + 1) * s;
    double *pl = (double *)malloc(sizeof(double) * (nh ? nh : 1));
    double *pu = (double *)malloc(sizeof(double) * (nh ? nh : 1));
    double *xl = (double *)malloc(sizeof(double) * nx);
    double *xu = (double *)malloc(sizeof(double) * nx);
    for (int i = 0; i < n; ++i) {
        const double *bl = lo + (size_t)i * d, *bh = hi + (size_t)i * d;
        const double *a_pl = pl, *a_pu = pu, *a_xl = xl, *a_xu = xu;
        if (pre_lo) {
            a_pl = pre_lo + (size_t)i * nh;
            a_pu = pre_hi + (size_t)i * nh;
            a_xl = x_lo + (size_t)i * nx;
            a_xu = x_hi + (size_t)i * nx;
        } else {
            ibp_box(&N, H, rho, x0, goal, bl, bh, pl, pu, xl, xu);
        }
        crown_out o = crown_box(&N, H, rho, x0, goal, bl, bh, a_pl, a_pu, a_xl, a_xu,
                                alpha ? alpha + (size_t)i * nh : NULL, NULL, NULL, NULL, NULL, 0, prec);
        lb[i] = o.lb;
        if (margin) margin[i] = o.margin;
        if (scale) scale[i] = o.scale;
    }
    free(pl);
    free(pu);
    free(xl);
    free(xu);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Gradient of the bound with respect to alpha                               */
/* ------------------------------------------------------------------------ */

/*
 * The backward pass of crown_box is a back-substitution through the "relaxed
 * network": every ReLU replaced by the linear bound Lemma 1 selected for it.
 * Its final linear function of u therefore equals the relaxed network's
 * objective (tangent-linearised cost plus rho ||u||^2), and the bound is that
 * objective at the concretizing point u*.  With the selections fixed, the
 * bound depends on a lower slope alpha_j only through the term
 * A_j * alpha_j * z_j, where A_j >= 0 is the coefficient of the ReLU output and
 * z_j the neuron's pre-activation in the relaxed network at u*.  Hence
 *   dLB/dalpha_j = A_j * z~_j(u*)   (unstable neurons whose lower bound was
 *                                    selected), 0 otherwise.
 * The argument holds for any cost relaxation that is linear in the states and
 * actions, the pushing-with-obstacles one included (its tangent plane and
 * penalty pieces do not depend on alpha).  relaxed_obj (nullable) receives the
 * relaxed network's objective at u*, which must equal lb; it is written out
 * for the squared-distance cost only (NaN for the obstacle cost).
 */
int oracle_alpha_grad(int L, const int *dims, const double *params, int s, int k, int H, double rho,
                      const double *x0, const double *goal, int n, const double *lo, const double *hi,
                      const double *alpha, double *lb, double *grad_alpha, double *relaxed_obj)
{
    onet N;
    if (onet_init(&N, L, dims, params, s, k)) return -1;
    int d = k * H, sumh = N.sumh;
    size_t nh = (size_t)H * sumh, nx = (size_t)(H + 1) * s;
    double *pl = (double *)malloc(sizeof(double) * (nh ? nh : 1));
    double *pu = (double *)malloc(sizeof(double) * (nh ? nh : 1));
    double *Ap = (double *)malloc(sizeof(double) * (nh ? nh : 1));
    double *xl = (double *)malloc(sizeof(double) * nx);
    double *xu = (double *)malloc(sizeof(double) * nx);
    double *at = (double *)malloc(sizeof(double) * nx);
    double *us = (double *)malloc(sizeof(double) * d);
    for (int i = 0; i < n; ++i) {
        const double *bl = lo + (size_t)i * d, *bh = hi + (size_t)i * d;
        const double *al = alpha ? alpha + (size_t)i * nh : NULL;
        double *g = grad_alpha + (size_t)i * nh;
        ibp_box(&N, H, rho, x0, goal, bl, bh, pl, pu, xl, xu);
        crown_out o = crown_box(&N, H, rho, x0, goal, bl, bh, pl, pu, xl, xu, al, NULL, us, Ap, at, 0, 0);
        lb[i] = o.lb;

        /* forward pass of the relaxed network from x_0 and u* */
        double x[ORC_MAX_WIDTH], a[ORC_MAX_WIDTH], z[ORC_MAX_WIDTH];
        double obj = 0.0;
        for (int q = 0; q < s; ++q) x[q] = x0[q];
        for (int t = 0; t < H; ++t) {
            for (int q = 0; q < s; ++q) a[q] = x[q];
            for (int j = 0; j < k; ++j) {
                a[s + j] = us[t * k + j];
                obj += rho * us[t * k + j] * us[t * k + j];
            }
            for (int l = 1; l <= L; ++l) {
                int no = N.dims[l], ni = N.dims[l - 1];
                for (int r = 0; r < no; ++r) {
                    double acc = N.b[l][r];
                    for (int c = 0; c < ni; ++c) acc += N.W[l][(size_t)r * ni + c] * a[c];
                    z[r] = acc;
                }
                if (l < L) {
                    for (int r = 0; r < no; ++r) {
                        size_t idx = (size_t)t * sumh + N.hoff[l] + r;
                        double zl = pl[idx], zu = pu[idx];
                        double alj = al ? al[idx] : adaptive_alpha(zl, zu);
                        int lower = Ap[idx] >= 0.0;
                        double D, c;
                        oracle_relu_relax(zl, zu, alj, lower ? 0 : 1, &D, &c);
                        g[idx] = (zl < 0.0 && zu > 0.0 && lower) ? Ap[idx] * z[r] : 0.0;
                        a[r] = D * z[r] + c;
                    }
                }
            }
            for (int q = 0; q < s; ++q) {
                x[q] += z[q];
                double m = 0.5 * at[(size_t)(t + 1) * s + q];
                obj += 2.0 * m * (x[q] - goal[q]) - m * m;
            }
        }
        if (relaxed_obj) relaxed_obj[i] = g_cost.kind == 0 ? obj : NAN;
    }
    free(pl);
    free(pu);
    free(Ap);
    free(xl);
    free(xu);
    free(at);
    free(us);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Gradient of the bound with respect to the box                             */
/* ------------------------------------------------------------------------ */

/*
 * With the relaxation choices fixed (which neurons are stable, which linear
 * bound each unstable one uses), the bound is the relaxed network's objective
 * at the concretizing point u*, min over the box of a function of u whose
 * parameters are: the box itself, the upper chords D z + c of unstable neurons
 * whose coefficient A < 0 (D = u/(u - l), c = -u l/(u - l) with [l, u] the
 * neuron's interval bounds), and the tangent points m = (L + U)/2 of the cost
 * terms (L, U the interval of x_{t,i} - g_i).  At a minimiser the derivative
 * of the minimum with respect to a parameter is the partial derivative of the
 * objective there, so (a.e., with z~, x~ the relaxed network's values at u*):
 *   chord neuron:  dLB/dD = A z~,  dLB/dc = A, hence
 *                  dLB/du = A l (l - z~)/(u - l)^2,  dLB/dl = A u (z~ - u)/(u - l)^2;
 *   tangent:       dLB/dm = 2 (x~ - g - m), and dm/dL = dm/dU = 1/2;
 *   box face:      dLB/dlo_j = mu_j + 2 rho lo_j when u*_j sits on lo_j (for
 *                  rho > 0: -mu_j/(2 rho) <= lo_j; for rho = 0: mu_j >= 0), and
 *                  the same at hi_j; 0 in the interior.
 * The interval bounds are themselves piecewise-linear functions of the box
 * (ibp_box: z_lo = W+ a_lo + W- a_hi + b, z_hi = W+ a_hi + W- a_lo + b, the
 * ReLU passing a derivative only where its end is positive, x_{t+1} = x_t +
 * z_L), so their sensitivities are carried back to the box by the transposed
 * steps.  Outputs: lb [n] and grad_lo, grad_hi [n][d].  The gradient is the
 * derivative of the bound with alpha held fixed (alpha nullable: adaptive,
 * piecewise constant in the bounds).
 */
int oracle_box_grad(int L, const int *dims, const double *params, int s, int k, int H, double rho,
                    const double *x0, const double *goal, int n, const double *lo, const double *hi,
                    const double *alpha, double *lb, double *grad_lo, double *grad_hi)
{
    onet N;
    if (onet_init(&N, L, dims, params, s, k)) return -1;
    int d = k * H, sumh = N.sumh;
    size_t nh = (size_t)H * sumh, nx = (size_t)(H + 1) * s;
    double *pl = (double *)malloc(sizeof(double) * (nh ? nh : 1));
    double *pu = (double *)malloc(sizeof(double) * (nh ? nh : 1));
    double *Ap = (double *)malloc(sizeof(double) * (nh ? nh : 1));
    double *zt = (double *)malloc(sizeof(double) * (nh ? nh : 1));   /* relaxed pre-activations at u* */
    double *gl = (double *)malloc(sizeof(double) * (nh ? nh : 1));   /* dLB / d pre_lo */
    double *gu = (double *)malloc(sizeof(double) * (nh ? nh : 1));   /* dLB / d pre_hi */
    double *xl = (double *)malloc(sizeof(double) * nx);
    double *xu = (double *)malloc(sizeof(double) * nx);
    double *gx = (double *)calloc(nx, sizeof(double));                 /* dLB / d x_lo = dLB / d x_hi (tangents) */
    double *at = (double *)malloc(sizeof(double) * nx);
    double *us = (double *)malloc(sizeof(double) * d);
    double *mu = (double *)malloc(sizeof(double) * d);
    for (int i = 0; i < n; ++i) {
        const double *bl = lo + (size_t)i * d, *bh = hi + (size_t)i * d;
        const double *al = alpha ? alpha + (size_t)i * nh : NULL;
        double *glo = grad_lo + (size_t)i * d, *ghi = grad_hi + (size_t)i * d;
        ibp_box(&N, H, rho, x0, goal, bl, bh, pl, pu, xl, xu);
        crown_out o = crown_box(&N, H, rho, x0, goal, bl, bh, pl, pu, xl, xu, al, mu, us, Ap, at, 0, 0);
        lb[i] = o.lb;

        /* relaxed network from x_0 and u*: z~ and the state x~_t, and the sensitivities */
        double x[ORC_MAX_WIDTH], a[ORC_MAX_WIDTH], z[ORC_MAX_WIDTH];
        memset(gx, 0, sizeof(double) * nx);
        for (int q = 0; q < s; ++q) x[q] = x0[q];
        for (int t = 0; t < H; ++t) {
            for (int q = 0; q < s; ++q) a[q] = x[q];
            for (int j = 0; j < k; ++j) a[s + j] = us[t * k + j];
            for (int l = 1; l <= L; ++l) {
                int no = N.dims[l], ni = N.dims[l - 1];
                for (int r = 0; r < no; ++r) {
                    double acc = N.b[l][r];
                    for (int c = 0; c < ni; ++c) acc += N.W[l][(size_t)r * ni + c] * a[c];
                    z[r] = acc;
                }
                if (l < L) {
                    for (int r = 0; r < no; ++r) {
                        size_t idx = (size_t)t * sumh + N.hoff[l] + r;
                        double zl = pl[idx], zu = pu[idx];
                        double alj = al ? al[idx] : adaptive_alpha(zl, zu);
                        int lower = Ap[idx] >= 0.0;
                        double D, c;
                        oracle_relu_relax(zl, zu, alj, lower ? 0 : 1, &D, &c);
                        zt[idx] = z[r];
                        gl[idx] = gu[idx] = 0.0;
                        if (zl < 0.0 && zu > 0.0 && !lower) {
                            double w2 = (zu - zl) * (zu - zl);
                            gu[idx] = Ap[idx] * zl * (zl - z[r]) / w2;
                            gl[idx] = Ap[idx] * zu * (z[r] - zu) / w2;
                        }
                        a[r] = D * z[r] + c;
                    }
                }
            }
            for (int q = 0; q < s; ++q) {
                x[q] += z[q];
                double m = 0.5 * at[(size_t)(t + 1) * s + q];
                gx[(size_t)(t + 1) * s + q] = (x[q] - goal[q]) - m;
            }
        }

        /* the interval bounds' sensitivities carried back to the box */
        double Gxl[ORC_MAX_WIDTH], Gxh[ORC_MAX_WIDTH], Gal[ORC_MAX_WIDTH], Gah[ORC_MAX_WIDTH];
        double Gzl[ORC_MAX_WIDTH], Gzh[ORC_MAX_WIDTH];
        for (int q = 0; q < s; ++q) Gxl[q] = Gxh[q] = gx[(size_t)H * s + q];
        for (int j = 0; j < d; ++j) glo[j] = ghi[j] = 0.0;
        for (int t = H - 1; t >= 0; --t) {
            /* x_{t+1} = x_t + z_L */
            for (int q = 0; q < s; ++q) {
                Gzl[q] = Gxl[q];
                Gzh[q] = Gxh[q];
            }
            for (int l = L; l >= 1; --l) {
                int no = N.dims[l], ni = N.dims[l - 1];
                if (l < L) {
                    /* a_l = max(z_l, 0) at each end, plus the bounds' own sensitivities */
                    for (int r = 0; r < no; ++r) {
                        size_t idx = (size_t)t * sumh + N.hoff[l] + r;
                        Gzl[r] = (pl[idx] > 0.0 ? Gal[r] : 0.0) + gl[idx];
                        Gzh[r] = (pu[idx] > 0.0 ? Gah[r] : 0.0) + gu[idx];
                    }
                }
                for (int c = 0; c < ni; ++c) {
                    double sl = 0.0, sh = 0.0;
                    for (int r = 0; r < no; ++r) {
                        double w = N.W[l][(size_t)r * ni + c];
                        if (w >= 0.0) {
                            sl += w * Gzl[r];
                            sh += w * Gzh[r];
                        } else {
                            sl += w * Gzh[r];
                            sh += w * Gzl[r];
                        }
                    }
                    Gal[c] = sl;
                    Gah[c] = sh;
                }
            }
            /* a_0 = [x_t; u_t]: the box coordinates of step t, and x_t (residual path, tangent at t) */
            for (int j = 0; j < k; ++j) {
                glo[t * k + j] += Gal[s + j];
                ghi[t * k + j] += Gah[s + j];
            }
            for (int q = 0; q < s; ++q) {
                double tg = t >= 1 ? gx[(size_t)t * s + q] : 0.0;
                Gxl[q] = Gxl[q] + Gal[q] + tg;
                Gxh[q] = Gxh[q] + Gah[q] + tg;
            }
        }
        /* the concretization's direct dependence on the faces */
        for (int j = 0; j < d; ++j) {
            int at_lo, at_hi;
            if (rho > 0.0) {
                double uc = -mu[j] / (2.0 * rho);
                at_lo = uc <= bl[j];
                at_hi = !at_lo && uc >= bh[j];
            } else {
                at_lo = mu[j] >= 0.0;
                at_hi = !at_lo;
            }
            if (at_lo) glo[j] += mu[j] + 2.0 * rho * bl[j];
            if (at_hi) ghi[j] += mu[j] + 2.0 * rho * bh[j];
        }
    }
    free(pl);
    free(pu);
    free(Ap);
    free(zt);
    free(gl);
    free(gu);
    free(xl);
    free(xu);
    free(gx);
    free(at);
    free(us);
    free(mu);
    return 0;
}

/*
 * One projected Adam ascent step (Kingma and Ba, 2015, Algorithm 1, with the
 * update sign flipped to ascend), then clamp to [clamp_lo, clamp_hi].  step
 * counts from 1.
 */
void oracle_adam_ascent(int count, double *param, double *m, double *v, const double *grad, int step, double lr,
                        double beta1, double beta2, double eps, double clamp_lo, double clamp_hi)
{
    double bc1 = 1.0 - pow(beta1, step), bc2 = 1.0 - pow(beta2, step);
    for (int i = 0; i < count; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * grad[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];
        double mh = m[i] / bc1, vh = v[i] / bc2;
        double p = param[i] + lr * mh / (sqrt(vh) + eps);
        if (p < clamp_lo) p = clamp_lo;
        if (p > clamp_hi) p = clamp_hi;
        param[i] = p;
    }
}

/* ------------------------------------------------------------------------ */
/* Prune, pick out, split (Section 3 overview, Section 3.1, Algorithm 2)     */
/* ------------------------------------------------------------------------ */

typedef struct {
    float key;
    uint64_t id;
    int row;
} okey;

static int okey_cmp(const void *pa, const void *pb)
{
    const okey *a = (const okey *)pa, *b = (const okey *)pb;
    /* NaN keys order last */
    int an = isnan(a->key), bn = isnan(b->key);
    if (an != bn) return an - bn;
    if (!an && a->key < b->key) return -1;
    if (!an && a->key > b->key) return 1;
    if (a->id < b->id) return -1;
    if (a->id > b->id) return 1;
    return 0;
}

/*
 * One prune-and-branch pass over a pool of n boxes.
 *  1. Prune (Section 3 overview, Algorithm 2): drop box i iff
 *     (double) lb[i] > inc_val; a NaN bound is kept.  keep[i] in {0,1}.
 *  2. Pick out up to n_pick survivors (Section 3.1): if there are at most
 *     n_pick survivors all are picked; otherwise the ceil(eta * n_pick) with
 *     smallest (ub, id) are picked first, and the rest of the quota is filled
 *     by smallest (lb, id) among the others.
 *  3. Split each picked box (Section 3.1) on its widest dimension, lowest
 *     index on ties, at mid = 0.5f * (lo + hi) in FP32: child 2p is the lower
 *     half, child 2p + 1 the upper half; ids 2 id and 2 id + 1; both inherit
 *     the parent's lb and ub.
 * Output rows: the 2 P children (picked boxes in pool order), then the R
 * unpicked survivors in pool order.  Returns 0.
 *
 * Child identifiers (oracle_child_id): 2 id + c (c = 0 lower, 1 upper half)
 * while id < 2^62, i.e. the binary path from the root box (id 1) through 62
 * splits; deeper, the path continues as a hash, 2^62 + (splitmix(2 id + c)
 * >> 2) (taken mod 2^64), so that the search can go arbitrarily deep; two
 * boxes then share an identifier (and so their samples) with probability
 * about 2^-62.
 */
uint64_t oracle_child_id(uint64_t id, int c)
{
    if (id < (1ULL << 62)) return 2 * id + (uint64_t)c;
    return (1ULL << 62) | (oracle_splitmix64(2 * id + (uint64_t)c) >> 2);
}

/*
 * Natural logarithm of a positive normal FP32 number with basic operations
 * only, each rounded once: x = 2^e m with m in [sqrt(1/2), sqrt(2)), then
 * log x = e ln 2 + 2 atanh(z), z = (m - 1)/(m + 1), |z| < 0.172, from the
 * atanh series z + z^3/3 + ... + z^13/13 (truncation below 2^-30 relative).
 * Any IEEE implementation of the same steps returns the same bits, which
 * keeps the softmax pick-out below reproducible across implementations.
 */
float oracle_log_det(float x)
{
    uint32_t b;
    memcpy(&b, &x, 4);
    int e = (int)((b >> 23) & 0xFF) - 127;
    uint32_t mb = (b & 0x007FFFFFu) | 0x3F800000u;
    volatile float m;
    float mm;
    memcpy(&mm, &mb, 4);
    m = mm;
    if (m > 1.41421356f) {
        m = m * 0.5f;
        e += 1;
    }
    volatile float num = m - 1.0f, den = m + 1.0f;
    volatile float z = num / den;
    volatile float z2 = z * z;
    volatile float pp = 0.0769230769f;           /* 1/13 */
    pp = pp * z2;
    pp = pp + 0.0909090909f;                     /* 1/11 */
    pp = pp * z2;
    pp = pp + 0.111111111f;                      /* 1/9 */
    pp = pp * z2;
    pp = pp + 0.142857143f;                      /* 1/7 */
    pp = pp * z2;
    pp = pp + 0.2f;                              /* 1/5 */
    pp = pp * z2;
    pp = pp + 0.333333333f;                      /* 1/3 */
    pp = pp * z2;
    pp = pp + 1.0f;
    volatile float t = z * pp;
    t = t + t;
    volatile float ef = (float)e;
    volatile float el = ef * 0.693147181f;       /* e ln 2 */
    volatile float r = el + t;
    return r;
}

/*
 * Key of the softmax pick-out (Section 3.1, Eq. lf_pick) as an exponential
 * race: candidate i wins with probability exp(-s_i / T) / sum_j exp(-s_j / T)
 * when the smallest key s_i / T + log(E_i) wins, E_i = -log(U_i) ~ Exp(1); the
 * k smallest keys are a draw of k candidates without replacement (Efraimidis
 * and Spirakis, 2006).  s = (lb - lb_min) / (lb_max - lb_min) over the
 * candidates (0 if they are all equal); U_i in (0, 1) from SplitMix64 of
 * (seed, id).  All in FP32, one rounding per operation.
 */
float oracle_pick_key(float lb, float lb_min, float lb_max, float temperature, uint64_t seed, uint64_t id)
{
    volatile float span = lb_max - lb_min;
    volatile float sc = 0.0f;
    if (span > 0.0f) {
        volatile float dlt = lb - lb_min;
        sc = dlt / span;
    }
    uint64_t h = oracle_splitmix64(seed ^ oracle_splitmix64(id));
    volatile float uu = ((float)(h >> 41) + 0.5f) * (1.0f / 8388608.0f);  /* (k + 1/2) 2^-23, exact, in (0, 1) */
    volatile float le = oracle_log_det(uu);
    volatile float E = -le;
    volatile float lg = oracle_log_det(E);
    volatile float q = sc / temperature;
    volatile float key = q + lg;
    return key;
}

/* One prune-and-branch pass; pick_rule 0: the rest of the quota by smallest (lb, id); 1: by the softmax race
   (keys of oracle_pick_key).  split_dim (nullable): the dimension to split of each pool row; NULL: widest. */
static int prune_branch_impl(int n, int d, const float *lo, const float *hi, const float *lb, const float *ub,
                             const uint64_t *id, double inc_val, int n_pick, double eta, int pick_rule,
                             float temperature, uint64_t pick_seed, const int *split_dim, float *out_lo,
                             float *out_hi, float *out_lb, float *out_ub, uint64_t *out_id, uint8_t *keep,
                             int *n_children, int *n_rest);

int oracle_prune_branch(int n, int d, const float *lo, const float *hi, const float *lb, const float *ub,
                        const uint64_t *id, double inc_val, int n_pick, double eta, float *out_lo, float *out_hi,
                        float *out_lb, float *out_ub, uint64_t *out_id, uint8_t *keep, int *n_children, int *n_rest)
{
    return prune_branch_impl(n, d, lo, hi, lb, ub, id, inc_val, n_pick, eta, 0, 1.0f, 0, NULL, out_lo, out_hi,
                             out_lb, out_ub, out_id, keep, n_children, n_rest);
}

int oracle_prune_branch_heuristic(int n, int d, const float *lo, const float *hi, const float *lb, const float *ub,
                                  const uint64_t *id, double inc_val, int n_pick, double eta, int pick_rule,
                                  float temperature, uint64_t pick_seed, const int *split_dim, float *out_lo,
                                  float *out_hi, float *out_lb, float *out_ub, uint64_t *out_id, uint8_t *keep,
                                  int *n_children, int *n_rest)
{
    return prune_branch_impl(n, d, lo, hi, lb, ub, id, inc_val, n_pick, eta, pick_rule, temperature, pick_seed,
                             split_dim, out_lo, out_hi, out_lb, out_ub, out_id, keep, n_children, n_rest);
}

static int prune_branch_impl(int n, int d, const float *lo, const float *hi, const float *lb, const float *ub,
                             const uint64_t *id, double inc_val, int n_pick, double eta, int pick_rule,
                             float temperature, uint64_t pick_seed, const int *split_dim, float *out_lo,
                             float *out_hi, float *out_lb, float *out_ub, uint64_t *out_id, uint8_t *keep,
                             int *n_children, int *n_rest)
{
    int *surv = (int *)malloc(sizeof(int) * (n ? n : 1));
    uint8_t *picked = (uint8_t *)calloc(n ? n : 1, 1);
    int ns = 0;
    for (int i = 0; i < n; ++i) {
        int kp = !((double)lb[i] > inc_val);
        keep[i] = (uint8_t)kp;
        if (kp) surv[ns++] = i;
    }
    if (ns <= n_pick) {
        for (int q = 0; q < ns; ++q) picked[surv[q]] = 1;
    } else {
        int n1 = (int)ceil(eta * n_pick);
        if (n1 > n_pick) n1 = n_pick;
        okey *ks = (okey *)malloc(sizeof(okey) * ns);
        for (int q = 0; q < ns; ++q) {
            ks[q].key = ub[surv[q]];
            ks[q].id = id[surv[q]];
            ks[q].row = surv[q];
        }
        qsort(ks, ns, sizeof(okey), okey_cmp);
        for (int q = 0; q < n1; ++q) picked[ks[q].row] = 1;
        float lmin = INFINITY, lmax = -INFINITY;
        if (pick_rule == 1)
            for (int q = 0; q < ns; ++q) {
                float v = lb[surv[q]];
                if (picked[surv[q]] || isnan(v)) continue;
                if (v < lmin) lmin = v;
                if (v > lmax) lmax = v;
            }
        int m = 0;
        for (int q = 0; q < ns; ++q) {
            if (picked[surv[q]]) continue;
            float v = lb[surv[q]];
            ks[m].key = (pick_rule == 1 && !isnan(v)) ? oracle_pick_key(v, lmin, lmax, temperature, pick_seed, id[surv[q]])
                                                      : v;
            ks[m].id = id[surv[q]];
            ks[m].row = surv[q];
            ++m;
        }
        qsort(ks, m, sizeof(okey), okey_cmp);
        for (int q = 0; q < n_pick - n1 && q < m; ++q) picked[ks[q].row] = 1;
        free(ks);
    }
    int P = 0;
    for (int q = 0; q < ns; ++q) {
        int i = surv[q];
        if (!picked[i]) continue;
        const float *pl = lo + (size_t)i * d, *ph = hi + (size_t)i * d;
        int js = 0;
        if (split_dim && split_dim[i] >= 0 && split_dim[i] < d) {
            js = split_dim[i];
        } else {
            float wbest = ph[0] - pl[0];
            for (int j = 1; j < d; ++j) {
                float w = ph[j] - pl[j];
                if (w > wbest) {
                    wbest = w;
                    js = j;
                }
            }
        }
        volatile float sum = pl[js] + ph[js];
        volatile float mid = 0.5f * sum;
        for (int c = 0; c < 2; ++c) {
            size_t o = (size_t)(2 * P + c);
            memcpy(out_lo + o * d, pl, sizeof(float) * d);
            memcpy(out_hi + o * d, ph, sizeof(float) * d);
            if (c == 0) out_hi[o * d + js] = mid;
            else out_lo[o * d + js] = mid;
            out_id[o] = oracle_child_id(id[i], c);
            out_lb[o] = lb[i];
            out_ub[o] = ub[i];
        }
        ++P;
    }
    int R = 0;
    for (int q = 0; q < ns; ++q) {
        int i = surv[q];
        if (picked[i]) continue;
        size_t o = (size_t)(2 * P + R);
        memcpy(out_lo + o * d, lo + (size_t)i * d, sizeof(float) * d);
        memcpy(out_hi + o * d, hi + (size_t)i * d, sizeof(float) * d);
        out_id[o] = id[i];
        out_lb[o] = lb[i];
        out_ub[o] = ub[i];
        ++R;
    }
    *n_children = 2 * P;
    *n_rest = R;
    free(surv);
    free(picked);
    return 0;
}

/*
 * The splitting heuristic of Section 3.1: for each box, the top_k samples of
 * smallest cost (ties by sample index; costs [n][M] as the search computed
 * them, FP32), their coordinates re-drawn from the counter-based sampler, and
 * per dimension j the counts n_lo (u_j <= mid_j) and n_up (u_j >= mid_j) with
 * mid_j = 0.5f (lo_j + hi_j); the score (hi_j - lo_j) |n_lo - n_up| in FP32,
 * the largest score (lowest j on ties) is the dimension to split.  When every
 * score is 0 (no imbalance) the widest dimension is used.
 */
typedef struct {
    float c;
    int m;
} ocost;

static int ocost_cmp(const void *pa, const void *pb)
{
    const ocost *a = (const ocost *)pa, *b = (const ocost *)pb;
    int an = isnan(a->c), bn = isnan(b->c);
    if (an != bn) return an - bn;
    if (!an && a->c < b->c) return -1;
    if (!an && a->c > b->c) return 1;
    return a->m - b->m;
}

int oracle_split_dims(int n, int d, const float *lo, const float *hi, const uint64_t *id, uint64_t seed,
                      const float *costs, int M, int top_k, int *split_dim)
{
    if (top_k < 1 || top_k > M) return -1;
    ocost *cs = (ocost *)malloc(sizeof(ocost) * M);
    for (int i = 0; i < n; ++i) {
        const float *bl = lo + (size_t)i * d, *bh = hi + (size_t)i * d;
        for (int m = 0; m < M; ++m) {
            cs[m].c = costs[(size_t)i * M + m];
            cs[m].m = m;
        }
        qsort(cs, M, sizeof(ocost), ocost_cmp);
        int jb = -1;
        float sb = 0.0f;
        for (int j = 0; j < d; ++j) {
            volatile float sum = bl[j] + bh[j];
            volatile float mid = 0.5f * sum;
            int nlo = 0, nup = 0;
            for (int q = 0; q < top_k; ++q) {
                float u = oracle_sample(seed, id[i], (uint32_t)cs[q].m, (uint32_t)j, bl[j], bh[j]);
                if (u <= mid) ++nlo;
                if (u >= mid) ++nup;
            }
            volatile float w = bh[j] - bl[j];
            volatile float sc = w * (float)abs(nlo - nup);
            if (sc > sb) {
                sb = sc;
                jb = j;
            }
        }
        if (jb < 0) {
            jb = 0;
            float wb = bh[0] - bl[0];
            for (int j = 1; j < d; ++j) {
                float w = bh[j] - bl[j];
                if (w > wb) {
                    wb = w;
                    jb = j;
                }
            }
        }
        split_dim[i] = jb;
    }
    free(cs);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Cross-entropy search (Section 3.3, batch_search with CEM)                 */
/* ------------------------------------------------------------------------ */

/*
 * The objective of Eq. (trajop) in FP32 with one rounding per operation, the
 * precision in which the search ranks its samples: each neuron's pre-
 * activation starts from its bias and adds the products w_c z_c in input order
 * c = 0, 1, ... by fused multiply-adds; ReLU; x_{t+1} = x_t + N([x_t; u_t]); the
 * step cost starts from 0, adds (x_{t+1,i} - g_i)^2 for i = 0..s-1 and then
 * (rho u_{t,j}) u_{t,j} for j = 0..k-1 by fused multiply-adds, and is added to
 * the running total.  For the pushing-with-obstacles cost the state part of
 * the step cost is w_t sqrt(sum_i (x_{t+1,i} - g_i)^2) (the squares summed by
 * fused multiply-adds, then one rounded product), followed, per obstacle o in
 * order, by lambda ReLU(s_o - d) for the pusher and then for each keypoint in
 * order (d = sqrt(dx dx + dy dy), dy dy rounded first; each added by a fused
 * multiply-add), the pusher position advancing by one rounded addition per
 * coordinate and step; the action terms follow as above.
 */
float oracle_objective_f32(int L, const int *dims, const double *params, int s, int k, int H, float rho,
                           const float *x0, const float *goal, const float *u)
{
    onet N;
    if (onet_init(&N, L, dims, params, s, k)) return NAN;
    float a[ORC_MAX_WIDTH], b[ORC_MAX_WIDTH], x[ORC_MAX_WIDTH];
    for (int i = 0; i < s; ++i) x[i] = x0[i];
    float pf[2] = {(float)g_cost.p0[0], (float)g_cost.p0[1]};
    float total = 0.0f;
    for (int t = 0; t < H; ++t) {
        for (int i = 0; i < s; ++i) a[i] = x[i];
        for (int j = 0; j < k; ++j) a[s + j] = u[t * k + j];
        float *in = a, *out = b;
        for (int l = 1; l <= L; ++l) {
            for (int q = 0; q < dims[l]; ++q) {
                float acc = (float)N.b[l][q];
                for (int c = 0; c < dims[l - 1]; ++c) acc = fmaf((float)N.W[l][(size_t)q * dims[l - 1] + c], in[c], acc);
                out[q] = (l < L) ? (acc > 0.0f ? acc : 0.0f) : acc;
            }
            float *tmp = in;
            in = out;
            out = tmp;
        }
        float c = 0.0f;
        if (g_cost.kind == 0) {
            for (int i = 0; i < s; ++i) {
                volatile float xn = x[i] + in[i];
                x[i] = xn;
                volatile float e = xn - goal[i];
                c = fmaf(e, e, c);
            }
        } else {
            for (int j = 0; j < 2; ++j) {
                volatile float pj = pf[j] + u[t * k + j];
                pf[j] = pj;
            }
            float ss = 0.0f;
            for (int i = 0; i < s; ++i) {
                volatile float xn = x[i] + in[i];
                x[i] = xn;
                volatile float e = xn - goal[i];
                ss = fmaf(e, e, ss);
            }
            volatile float wn = (float)g_cost.w[t + 1] * sqrtf(ss);
            c = wn;
            const float lamf = (float)g_cost.lambda;
            for (int o = 0; o < g_cost.n_obs; ++o) {
                const float ox = (float)g_cost.ox[o], oy = (float)g_cost.oy[o], osz = (float)g_cost.os[o];
                for (int q = -1; 2 * q + 1 < s; ++q) {
                    volatile float dx = (q < 0 ? pf[0] : x[2 * q]) - ox;
                    volatile float dy = (q < 0 ? pf[1] : x[2 * q + 1]) - oy;
                    volatile float dy2 = dy * dy;
                    float dd = fmaf(dx, dx, dy2);
                    volatile float r = osz - sqrtf(dd);
                    c = fmaf(lamf, r > 0.0f ? r : 0.0f, c);
                }
            }
        }
        for (int j = 0; j < k; ++j) {
            volatile float ru = rho * u[t * k + j];
            c = fmaf(ru, u[t * k + j], c);
        }
        volatile float tot = total + c;
        total = tot;
    }
    return total;
}

/*
 * The normal draw of the cross-entropy search for (box id, iteration it,
 * sample m, coordinate j): the Irwin-Hall sum of four uniforms,
 * z = (r_0 + r_1 + r_2 + r_3 - 2) sqrt(3), which has mean 0, variance 1 and
 * support |z| <= 2 sqrt(3).  r_c is the top 24 bits of a SplitMix64 chain:
 * box key b = splitmix(seed ^ splitmix(id)) as for the uniform draw, then
 * splitmix(b + C) with C = 0x632BE59BD9B4E019 (a stream of its own), then the
 * iteration, then (m << 32 | 4 j + c).  FP32, left to right, one rounding per
 * operation.  Sample 0 of iteration 0 is the mean itself (z = 0).
 */
float oracle_cem_normal(uint64_t seed, uint64_t id, uint32_t it, uint32_t m, uint32_t j)
{
    if (it == 0 && m == 0) return 0.0f;
    uint64_t h = oracle_splitmix64(seed ^ oracle_splitmix64(id));
    h = oracle_splitmix64(h + 0x632BE59BD9B4E019ULL);
    h = oracle_splitmix64(h ^ (uint64_t)it);
    volatile float acc = 0.0f;
    for (uint32_t c = 0; c < 4; ++c) {
        uint64_t hc = oracle_splitmix64(h ^ ((uint64_t)m << 32 | (uint64_t)(4u * j + c)));
        float r = (float)(hc >> 40) * (1.0f / 16777216.0f);
        acc = acc + r;
    }
    volatile float ctr = acc - 2.0f;
    volatile float z = ctr * 1.7320508f;
    return z;
}

/* The sample: mu + sigma z clipped to [lo, hi], in FP32. */
float oracle_cem_sample(uint64_t seed, uint64_t id, uint32_t it, uint32_t m, uint32_t j, float mu, float sigma,
                        float lo, float hi)
{
    float z = oracle_cem_normal(seed, id, it, m, j);
    volatile float sz = sigma * z;
    volatile float v = mu + sz;
    float u = v;
    if (u < lo) u = lo;
    if (u > hi) u = hi;
    return u;
}

typedef struct {
    float f;
    int m;
} ocem;

/* rank by objective (NaN last), then by sample index */
static int ocem_cmp(const void *pa, const void *pb)
{
    const ocem *a = (const ocem *)pa, *b = (const ocem *)pb;
    const int na = isnan(a->f), nb = isnan(b->f);
    if (na != nb) return na - nb;
    if (!na && a->f < b->f) return -1;
    if (!na && a->f > b->f) return 1;
    return a->m - b->m;
}

/*
 * Cross-entropy search of each box [lo, hi] (Section 3.3: batch_search with
 * CEM, warm-started from the parent's best input).  The search distribution is
 * a diagonal normal, started at mu = warm_u clipped to the box (warm_u NULL:
 * the box centre) and sigma = (hi - lo) / 2.  Each of `iters` iterations draws
 * M samples (oracle_cem_sample), ranks them by the FP32 objective, and refits
 * mu and sigma to the E best (the elites, in rank order): mu_j = (sum_e u_ej)
 * / E, sigma_j = sqrt((sum_e (u_ej - mu_j)^2) / E) + jitter, each sum in rank
 * order (the squares by fused multiply-adds).  The result is the best sample
 * over all iterations (ties: the earlier iteration, then the lower sample
 * index): ub[i] (its FP32 objective) and best_u [n][d].  mu_trace (nullable,
 * [n][iters][d]) receives mu after each refit.
 */
int oracle_cem(int L, const int *dims, const double *params, int s, int k, int H, float rho, const float *x0,
               const float *goal, int n, const float *lo, const float *hi, const uint64_t *id, const float *warm_u,
               int M, int iters, int E, float jitter, uint64_t seed, float *ub, float *best_u, float *mu_trace)
{
    if (M < 1 || iters < 1 || E < 1 || E > M) return -1;
    const int d = k * H;
    float *mu = (float *)malloc(sizeof(float) * d), *sg = (float *)malloc(sizeof(float) * d);
    float *u = (float *)malloc(sizeof(float) * d);
    float *nmu = (float *)malloc(sizeof(float) * d), *nsg = (float *)malloc(sizeof(float) * d);
    ocem *rk = (ocem *)malloc(sizeof(ocem) * M);
    for (int i = 0; i < n; ++i) {
        const float *bl = lo + (size_t)i * d, *bh = hi + (size_t)i * d;
        for (int j = 0; j < d; ++j) {
            if (warm_u) {
                float w = warm_u[(size_t)i * d + j];
                mu[j] = w < bl[j] ? bl[j] : (w > bh[j] ? bh[j] : w);
            } else {
                volatile float sum = bl[j] + bh[j];
                mu[j] = 0.5f * sum;
            }
            volatile float wd = bh[j] - bl[j];
            sg[j] = 0.5f * wd;
        }
        float best = NAN;
        int have = 0;
        for (int it = 0; it < iters; ++it) {
            for (int m = 0; m < M; ++m) {
                for (int j = 0; j < d; ++j)
                    u[j] = oracle_cem_sample(seed, id[i], (uint32_t)it, (uint32_t)m, (uint32_t)j, mu[j], sg[j], bl[j], bh[j]);
                rk[m].f = oracle_objective_f32(L, dims, params, s, k, H, rho, x0, goal, u);
                rk[m].m = m;
            }
            qsort(rk, M, sizeof(ocem), ocem_cmp);
            /* the iteration's best against the best so far (strictly better wins: earlier iterations keep ties) */
            if (!have || (!isnan(rk[0].f) && (isnan(best) || rk[0].f < best))) {
                best = rk[0].f;
                have = 1;
                for (int j = 0; j < d; ++j)
                    best_u[(size_t)i * d + j] = oracle_cem_sample(seed, id[i], (uint32_t)it, (uint32_t)rk[0].m,
                                                                  (uint32_t)j, mu[j], sg[j], bl[j], bh[j]);
            }
            /* refit to the elites (every coordinate from the current mu and sigma) */
            for (int j = 0; j < d; ++j) {
                float sum = 0.0f;
                for (int e = 0; e < E; ++e) {
                    float v = oracle_cem_sample(seed, id[i], (uint32_t)it, (uint32_t)rk[e].m, (uint32_t)j, mu[j], sg[j],
                                                bl[j], bh[j]);
                    volatile float t = sum + v;
                    sum = t;
                }
                volatile float mean = sum / (float)E;
                float acc = 0.0f;
                for (int e = 0; e < E; ++e) {
                    float v = oracle_cem_sample(seed, id[i], (uint32_t)it, (uint32_t)rk[e].m, (uint32_t)j, mu[j], sg[j],
                                                bl[j], bh[j]);
                    volatile float dv = v - mean;
                    acc = fmaf(dv, dv, acc);
                }
                volatile float var = acc / (float)E;
                volatile float sd = sqrtf(var);
                volatile float sj = sd + jitter;
                nmu[j] = mean;
                nsg[j] = sj;
            }
            memcpy(mu, nmu, sizeof(float) * d);
            memcpy(sg, nsg, sizeof(float) * d);
            if (mu_trace) memcpy(mu_trace + ((size_t)i * iters + it) * d, mu, sizeof(float) * d);
        }
        ub[i] = best;
    }
    free(mu);
    free(sg);
    free(u);
    free(nmu);
    free(nsg);
    free(rk);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Synthetic objective (Section 4, synthetic example)                         */
/* ------------------------------------------------------------------------ */

/* f(u) = sum_i 5 u_i^2 + cos(50 u_i), u in [-1, 1]^d. */
double oracle_synth_f(int d, const double *u)
{
    double f = 0.0;
    for (int i = 0; i < d; ++i) f += 5.0 * u[i] * u[i] + cos(50.0 * u[i]);
    return f;
}

#define ORC_PI 3.14159265358979323846

/* min of cos over [a, b], a <= b: -1 if an odd multiple of pi lies in [a, b], else the smaller end value. */
double oracle_cos_min(double a, double b)
{
    const double k = ceil((a / ORC_PI - 1.0) / 2.0); /* smallest k with (2k + 1) pi >= a */
    if ((2.0 * k + 1.0) * ORC_PI <= b) return -1.0;
    double ca = cos(a), cb = cos(b);
    return ca < cb ? ca : cb;
}

/*
 * Lower bound of f over each box: the sum over coordinates of the separate
 * minima of 5 u^2 over [lo, hi] and of cos(50 u) over [50 lo, 50 hi].  Each
 * term's minimum is exact; a separable objective's bound cannot be tighter than
 * the sum of its terms' minima under any linear relaxation of the terms.
 */
int oracle_synth_bound(int n, int d, const float *lo, const float *hi, double *lb)
{
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < d; ++j) {
            double l = lo[(size_t)i * d + j], h = hi[(size_t)i * d + j];
            s += 5.0 * sq_min(l, h) + oracle_cos_min(50.0 * l, 50.0 * h);
        }
        lb[i] = s;
    }
    return 0;
}

/* The search of each box: M uniform samples (oracle_sample), f in FP64, the minimum and its sample (ties: lowest
   sample index). */
int oracle_synth_search(int n, int d, const float *lo, const float *hi, const uint64_t *id, int M, uint64_t seed,
                        double *ub, float *best_u)
{
    double *u = (double *)malloc(sizeof(double) * d);
    float *uf = (float *)malloc(sizeof(float) * d);
    for (int i = 0; i < n; ++i) {
        double best = INFINITY;
        for (int m = 0; m < M; ++m) {
            for (int j = 0; j < d; ++j) {
                uf[j] = oracle_sample(seed, id[i], (uint32_t)m, (uint32_t)j, lo[(size_t)i * d + j], hi[(size_t)i * d + j]);
                u[j] = uf[j];
            }
            double f = oracle_synth_f(d, u);
            if (f < best || m == 0) {
                best = f;
                memcpy(best_u + (size_t)i * d, uf, sizeof(float) * d);
            }
        }
        ub[i] = best;
    }
    free(u);
    free(uf);
    return 0;
}
