// kernels.cuh -- argument blocks, the shared register-blocked dense product,
// and the host launchers of the libbab kernels.
#pragma once

#include "bab_internal.cuh"
#include "cost.cuh"

namespace bab {

// Many independent problems of one architecture in one launch.  Problem p has its own weights (images at
// p * img_floats / raw at p * raw_floats), x0 and goal (at p * s), horizon and rho; row i of the box arrays
// belongs to problem prob[i], uses the first k * H_p of its `d` (row stride) coordinates, and owns Hmax
// steps of every per-step array.  P = 1 with prob = H = rho = null is the single-problem case.
struct BatchDesc {
    const int *prob;   // [n] (nullable: every row is problem 0)
    const int *H;      // [P] (nullable: the call's horizon)
    const float *rho;  // [P] (nullable: the call's rho)
    int P;
    int Hmax;
};

// Out-of-range problem indices and horizons are clamped (to [0, P) and [0, Hmax]) so that every access
// stays inside the caller's arrays.
__device__ __forceinline__ int row_problem(const BatchDesc &b, int row)
{
    if (!b.prob) return 0;
    const int p = b.prob[row];
    return p < 0 ? 0 : (p >= b.P ? b.P - 1 : p);
}
__device__ __forceinline__ int problem_H(const BatchDesc &b, int p, int H)
{
    if (!b.H) return H;
    const int h = b.H[p];
    return h < 0 ? 0 : (h > b.Hmax ? b.Hmax : h);
}
__device__ __forceinline__ float problem_rho(const BatchDesc &b, int p, float rho) { return b.rho ? b.rho[p] : rho; }

struct RolloutArgs {
    NetDesc net;
    BatchDesc batch;
    const float *fwd;   // forward image (device)
    const float *raw;   // raw parameters (device), for the FP64 re-score
    const float *x0, *goal, *lo, *hi;
    const uint64_t *id;
    int n;
    const int *d_n;
    int H, M, d;
    float rho;
    uint64_t seed;
    unsigned long long *keys;  // [n] scratch
    float *ub, *best_u;
    double *inc_val;
    float *inc_u;
    int *status;
    // tensor-core path
    const uint8_t *tc_img;
    const float *tc_bias;
    int tc_bytes;        // bytes of the image the kernel loads (hi only for BF16)
    uint32_t tmem_cols;
    int stages;          // > 0: the image is streamed through a ring of `stages` buffers of stage_bytes
    int stage_bytes;
    size_t tc_img_stride;  // bytes between problems' tensor-core images (batched problems, streamed)
    // search-integrated bounds (nullable): per box the min / max over the samples of every hidden
    // pre-activation [n][H][sumh] and state [n][H+1][s], accumulated as order-preserving uint32 keys
    uint32_t *emp_pre_lo, *emp_pre_hi, *emp_x_lo, *emp_x_hi;
    float *costs;        // [n][M] (nullable): every sample's objective as the search computed it
    // BF16 rollouts: re-score in FP32 only the topk boxes of smallest BF16 ub (0: every box)
    int topk;
    unsigned long long *topk_t;  // [4] scratch: the selection threshold, then the number of boxes it picked
    int *topk_list;              // [n] scratch: the boxes the top-k selection picked (any order)
    // cross-entropy search (nullable): samples are cem_sample(.., cem_it, m, j, cem_mu[j], cem_sigma[j], ..) of
    // each box's [n][d] mean and spread instead of uniform draws
    const float *cem_mu, *cem_sigma;
    int cem_it;
    CostDesc cost;           // the state cost (kind 0: squared distance)
};

// one refit of the cross-entropy search (after a rollout of iteration `it` that wrote costs)
struct CemArgs {
    const float *lo, *hi;
    const uint64_t *id;
    int n;
    const int *d_n;
    int d, M, E, it;
    float jitter;
    uint64_t seed;
    const float *costs;       // [n][M]
    float *mu, *sigma;        // [n][d], refitted in place
    unsigned long long *best; // [n]: (order(f), it * M + m) of the best sample so far, ~0 before any
    float *ub, *best_u;       // [n], [n][d]
};

struct BoundArgs {
    NetDesc net;
    BatchDesc batch;
    const float *fwd, *bwd;
    const float *x0, *goal, *lo, *hi;
    int n;
    const int *d_n;
    int row0;                // the launch's first row within the caller's arrays (chunked calls; d_n counts from 0)
    int H, d;
    float rho;
    // interval bounds (written by k_ibp, read by k_crown / k_alpha_fwd)
    float *pre_lo, *pre_hi;  // [n][H][sumh]
    float *x_lo, *x_hi;      // [n][H+1][s]
    float *S;                // [n][H][sumh + s]: per row of each layer, sum_j |W_kj| max|a_j| over the input box
    float *lb_ibp;           // [n] (nullable)
    // CROWN
    const float *alpha;      // [n][H][sumh] (nullable: adaptive)
    float *A_pre;            // [n][H][sumh] (nullable): coefficient of each ReLU output before relaxation
    float *lb, *margin, *lin_coef, *lin_const;
    float *ustar;            // [n][d] (nullable)
    float *lb_best;          // [n] (nullable): running max
    // alpha
    float *grad_alpha;       // [n][H][sumh]
    int *status;
    // tensor-core CROWN
    const uint8_t *tcb_img;  // backward image (W_l^T, BF16 hi then lo)
    const float *tc_bias;    // biases padded to multiples of 16 (offsets tc_boff)
    float *mu;               // [n][d] coefficients of u (lin_coef or scratch)
    int t_stop;              // propagation early-stop step (0: back to the input); S == null: no margin
    uint32_t tmem_cols;
    int tc_rows;             // boxes per 128-row tile of the tensor-core CROWN (32, 64 or 128; the other rows idle)
    int stages;              // > 0: the backward image is streamed through `stages` ring buffers
    int stage_bytes;
    int stg_cols, stg_hid, stg_step;  // staged tensor-core CROWN: columns a thread takes, floats per area
    const uint8_t *ibp_img;  // tensor-core interval image (k_ibp_tc)
    CostDesc cost;           // the state cost (kind 0: squared distance)
};

// The pushing-with-obstacles state cost at step t on the box [xl, xu] of x_t, one warp per row (lane i owns
// coordinate i, s <= 32): lane i's coefficient aa of a linear lower bound aa . x + constant; returns the constant
// (rounded down, on every lane).  The norm by its tangent plane at the box centre, w ||x - g|| >= w ghat . (x - g)
// with |ghat| < 1 (the unit vector shrunk by 1e-5 against rounding); each keypoint penalty by penalty_lower.
__device__ __forceinline__ float obstacle_state_lin(const CostDesc &c, int t, int s, const float *xl, const float *xu,
                                                    const float *goal, int lane, float &aa)
{
    const float m = lane < s ? 0.5f * (xl[lane] + xu[lane]) - goal[lane] : 0.f;
    const float nm = sqrtf(warp_sum(m * m));
    float a_ = 0.f, cst = 0.f;
    if (nm > 0.f && lane < s) {
        a_ = c.w[t - 1] * (m / nm) * 0.99999f;
        cst = __fmul_rd(-a_, goal[lane]);
    }
    if (lane < s) {
        const int kp = lane >> 1;
        for (int o = 0; o < c.n_obs; ++o) {
            float a0, a1, b;
            if (penalty_lower(c, o, xl[2 * kp], xu[2 * kp], xl[2 * kp + 1], xu[2 * kp + 1], a0, a1, b)) {
                a_ += c.lam * ((lane & 1) ? a1 : a0);
                if (!(lane & 1)) cst = __fadd_rd(cst, __fmul_rd(c.lam, b));
            }
        }
    }
    aa = a_;
    return warp_sum_rd(cst);
}

// The pusher penalties at step t (1..H): the box of p_t = p_0 + u_0 + ... + u_{t-1} (directed rounding), then
// per obstacle the linear lower bound lam (a . p_t + b) = lam (a . p_0 + b) + lam a . (u_0 + ... + u_{t-1}):
// adds lam a to P[0..1] (the coefficient of every earlier action) and |lam a| to Pabs; returns the constant
// lam (a . p_0 + b), rounded down.  One thread.
__device__ __forceinline__ float pusher_lin(const CostDesc &c, int t, int k, const float *lo, const float *hi,
                                            float *P, float *Pabs)
{
    float l0 = c.p0x, l1 = c.p0y, u0 = c.p0x, u1 = c.p0y;
    for (int tau = 0; tau < t; ++tau) {
        l0 = __fadd_rd(l0, lo[tau * k]);
        l1 = __fadd_rd(l1, lo[tau * k + 1]);
        u0 = __fadd_ru(u0, hi[tau * k]);
        u1 = __fadd_ru(u1, hi[tau * k + 1]);
    }
    float cst = 0.f;
    for (int o = 0; o < c.n_obs; ++o) {
        float a0, a1, b;
        if (penalty_lower(c, o, l0, u0, l1, u1, a0, a1, b)) {
            P[0] += c.lam * a0;
            P[1] += c.lam * a1;
            Pabs[0] += fabsf(c.lam * a0);
            Pabs[1] += fabsf(c.lam * a1);
            cst = __fadd_rd(cst, __fmul_rd(c.lam, __fadd_rd(__fmaf_rd(a0, c.p0x, __fmul_rd(a1, c.p0y)), b)));
        }
    }
    return cst;
}

// The same linear lower bound as obstacle_state_lin for one box held by one thread (the tensor-core CROWN):
// coefficients aa[i] of x_t's coordinates i < s (xl, xu, goal: the box of x_t and the target, SP >= s values)
// and the constant (rounded down), the sums taken in index order.  |ghat| < 1 holds as there (the unit vector
// shrunk by 1e-5, far above the rounding of an s-term sum).
template <int SP>
__device__ __forceinline__ float obstacle_state_lin_row(const CostDesc &c, int t, int s, const float (&xl)[SP],
                                                        const float (&xu)[SP], const float *goal, float (&aa)[SP])
{
    float m[SP], ss = 0.f;
#pragma unroll
    for (int i = 0; i < SP; ++i) {
        m[i] = i < s ? 0.5f * (xl[i] + xu[i]) - goal[i] : 0.f;
        ss = fmaf(m[i], m[i], ss);
    }
    const float nm = sqrtf(ss);
    float cst = 0.f;
#pragma unroll
    for (int i = 0; i < SP; ++i) {
        float a_ = 0.f;
        if (nm > 0.f && i < s) {
            a_ = c.w[t - 1] * (m[i] / nm) * 0.99999f;
            cst = __fadd_rd(cst, __fmul_rd(-a_, goal[i]));
        }
        aa[i] = a_;
    }
#pragma unroll
    for (int kp = 0; kp < SP / 2; ++kp) {
        if (2 * kp >= s) break;
        for (int o = 0; o < c.n_obs; ++o) {
            float a0, a1, b;
            if (penalty_lower(c, o, xl[2 * kp], xu[2 * kp], xl[2 * kp + 1], xu[2 * kp + 1], a0, a1, b)) {
                aa[2 * kp] += c.lam * a0;
                aa[2 * kp + 1] += c.lam * a1;
                cst = __fadd_rd(cst, __fmul_rd(c.lam, b));
            }
        }
    }
    return cst;
}

struct AdamStep {
    float lr, bc1, bc2;
};

// Projected Adam ascent step (beta1 0.9, beta2 0.999, eps 1e-8), every operation rounded to nearest on its own
// (no contraction), so that the fused loop and the separate Adam launch agree bit for bit.
__device__ __forceinline__ float adam_update(float &alpha, float &m, float &v, float g, const AdamStep &s)
{
    const float mi = __fadd_rn(__fmul_rn(0.9f, m), __fmul_rn(0.1f, g));
    const float vi = __fadd_rn(__fmul_rn(0.999f, v), __fmul_rn(__fmul_rn(0.001f, g), g));
    m = mi;
    v = vi;
    const float mh = __fdiv_rn(mi, s.bc1), vh = __fdiv_rn(vi, s.bc2);
    const float x = __fadd_rn(alpha, __fdiv_rn(__fmul_rn(s.lr, mh), __fadd_rn(__fsqrt_rn(vh), 1e-8f)));
    alpha = fminf(fmaxf(x, 0.f), 1.f);
    return alpha;
}

// Adam bias corrections 1 - beta^step, formed on the host in FP64 exactly as for the separate Adam launches
constexpr int kAdamTable = 128;
struct AdamTable {
    float bc1[kAdamTable], bc2[kAdamTable];
};

// out[r][c] = act(sum_k in[r][k] * B[k][c] + bias[c]) for r < R, c < Np, where
// B is [Kp][Np] row-major (a forward image Wt_l, or a backward image W_l).
// Kp % 4 == 0 and Np % 4 == 0; bias may be null.
template <int R, int NT, int TR, int TN>
__device__ __forceinline__ void dense_rows(const float *__restrict__ in, int ldi, const float *__restrict__ B,
                                           const float *__restrict__ bias, int Kp, int Np, float *__restrict__ out,
                                           int ldo, bool relu)
{
    const int ngc = (Np + TN - 1) / TN;
    const int items = (R / TR) * ngc;
    for (int it = threadIdx.x; it < items; it += NT) {
        const int cg = it % ngc, rg = it / ngc;
        const int c0 = cg * TN, r0 = rg * TR;
        float acc[TR][TN];
        float bv[TN];
#pragma unroll
        for (int j = 0; j < TN; ++j) bv[j] = (bias && c0 + j < Np) ? bias[c0 + j] : 0.f;
#pragma unroll
        for (int i = 0; i < TR; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] = bv[j];
        const bool full = (c0 + TN <= Np);
        for (int k = 0; k < Kp; k += 4) {
            float4 xv[TR];
#pragma unroll
            for (int i = 0; i < TR; ++i) xv[i] = *reinterpret_cast<const float4 *>(in + (r0 + i) * ldi + k);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                float w[TN];
                const float *wr = B + (size_t)(k + kk) * Np + c0;
                if (full) {
#pragma unroll
                    for (int j = 0; j < TN; j += 4) {
                        float4 q = *reinterpret_cast<const float4 *>(wr + j);
                        w[j] = q.x;
                        w[j + 1] = q.y;
                        w[j + 2] = q.z;
                        w[j + 3] = q.w;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < TN; ++j) w[j] = (c0 + j < Np) ? wr[j] : 0.f;
                }
#pragma unroll
                for (int i = 0; i < TR; ++i) {
                    const float xs = kk == 0 ? xv[i].x : kk == 1 ? xv[i].y : kk == 2 ? xv[i].z : xv[i].w;
#pragma unroll
                    for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(xs, w[j], acc[i][j]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < TR; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j)
                if (c0 + j < Np) {
                    const float v = acc[i][j];
                    out[(r0 + i) * ldo + c0 + j] = relu ? fmaxf(v, 0.f) : v;
                }
    }
}

// Picks the register block so that the tile's items cover the threads.
template <int R, int NT>
__device__ __forceinline__ void dense_rows_auto(const float *in, int ldi, const float *B, const float *bias, int Kp,
                                                int Np, float *out, int ldo, bool relu)
{
    if (R >= 4 && (R / 4) * ((Np + 7) / 8) >= NT / 2)
        dense_rows<R, NT, (R >= 4 ? 4 : 1), 8>(in, ldi, B, bias, Kp, Np, out, ldo, relu);
    else if (R >= 2 && (R / 2) * ((Np + 3) / 4) >= NT / 2)
        dense_rows<R, NT, (R >= 2 ? 2 : 1), 4>(in, ldi, B, bias, Kp, Np, out, ldo, relu);
    else
        dense_rows<R, NT, 1, 4>(in, ldi, B, bias, Kp, Np, out, ldo, relu);
}

// host launchers (return the first CUDA error)
// variant < 0 picks by shared-memory size; rollout_fp32_variants() variants exist (the autotuner times them)
cudaError_t launch_rollout_fp32(const RolloutArgs &a, int variant, int num_sms, cudaStream_t st);
int rollout_fp32_variants();
cudaError_t launch_rollout_tc(RolloutArgs a, int split, int nslot_pref, int num_sms, cudaStream_t st);
// the synthetic objective sum 5 u^2 + cos(50 u): sampled search (uniform, or the cross-entropy mode with
// cem_mu / cem_sigma and costs), sound interval bound, FP64 incumbent
cudaError_t launch_synth_search(int d, const float *lo, const float *hi, const uint64_t *id, int n, const int *d_n,
                                int M, int it, uint64_t seed, const float *cem_mu, const float *cem_sigma,
                                unsigned long long *keys, float *costs, float *ub, float *best_u, cudaStream_t st);
cudaError_t launch_synth_bound(int d, const float *lo, const float *hi, int n, const int *d_n, float *lb,
                               cudaStream_t st);
cudaError_t launch_synth_incumbent(int d, const float *ub, const float *best_u, int n, const int *d_n,
                                   double *inc_val, float *inc_u, cudaStream_t st);
// cross-entropy search: start (mu, sigma, best) and one refit
cudaError_t launch_cem_init(const CemArgs &c, const float *warm_u, cudaStream_t st);
cudaError_t launch_cem_step(const CemArgs &c, cudaStream_t st);
bool rollout_tc_supported(const NetDesc &N, int split, int max_smem);
void k_fill_keys(unsigned long long *keys, int n, cudaStream_t st);
void launch_rollout_finalize(const RolloutArgs &a, cudaStream_t st);
// search-integrated bounds around an FP32 rollout (a.emp_* set): key init before, float conversion after
void launch_emp_init(const RolloutArgs &a, cudaStream_t st);
void launch_emp_finish(const RolloutArgs &a, cudaStream_t st);
void launch_incumbent(const RolloutArgs &a, cudaStream_t st);
cudaError_t launch_ibp(const BoundArgs &a, int num_sms, cudaStream_t st);
// interval bounds on tensor cores (split products with a computed margin; squared-distance cost, widths <= 256)
cudaError_t launch_ibp_tc(const BoundArgs &a, int num_sms, cudaStream_t st);
bool ibp_tc_supported(const NetDesc &N, int max_smem);
cudaError_t launch_crown(const BoundArgs &a, int num_sms, cudaStream_t st);
// Loads every instance launch_ibp / launch_crown may pick into the current device's context (lazy module loading
// would otherwise load, and allocate for, each one at its first launch).
cudaError_t preload_ibp_crown();
cudaError_t launch_crown_tc(BoundArgs a, int nslot_pref, int num_sms, cudaStream_t st);
bool crown_tc_supported(const NetDesc &N, int max_smem);
bool crown_tc_obstacles_supported(const NetDesc &N, int max_smem);
// CROWN with 3-term TF32 split products (a.tcb_img = the backward TF32 image; squared-distance cost, widths <= 256)
cudaError_t launch_crown_tf32(BoundArgs a, int num_sms, cudaStream_t st);
bool crown_tf32_supported(const NetDesc &N, int max_smem);
cudaError_t launch_alpha_fwd(const BoundArgs &a, int num_sms, cudaStream_t st);
cudaError_t launch_alpha_init(const BoundArgs &a, cudaStream_t st);
// the whole alpha optimisation of a tile of boxes in one CTA (needs the interval bounds of launch_ibp)
cudaError_t launch_alpha_fused(const BoundArgs &a, int steps, float lr, float *alpha_out, int variant, cudaStream_t st);
// interval bounds with one warp per box (any problem of the batch)
cudaError_t launch_ibp_warp(const BoundArgs &a, cudaStream_t st);
// d(bound)/d(box faces), one warp per box, after interval bounds and a CROWN pass that stored A_pre, u*, mu
// (lin_coef); GL, GU [n][Hmax][sumh] and GX [n][Hmax+1][s] are scratch
cudaError_t launch_box_grad_warp(const BoundArgs &a, float *GL, float *GU, float *GX, float *glo, float *ghi,
                                 cudaStream_t st);
// the whole alpha optimisation with one warp per box; alpha (written), m, v: [n][Hmax][sumh] device arrays;
// steps == 0: one bound with the adaptive slopes (alpha, m, v unused)
cudaError_t launch_alpha_warp(const BoundArgs &a, int steps, float lr, float *alpha, float *m, float *v,
                              cudaStream_t st);
void fill_adam_table(AdamTable &tab);
bool alpha_fused_fits(const NetDesc &N, int H, int d);
int alpha_fused_variants();
cudaError_t launch_fill(float *p, int n, float v, cudaStream_t st);
cudaError_t launch_adam(float *alpha, float *m, float *v, const float *grad, long long count, float lr, float bc1,
                        float bc2, cudaStream_t st);

struct BranchArgs {
    int d, n;
    const int *d_n;
    const float *lo, *hi, *lb, *ub;
    const uint64_t *id;
    const double *inc_val;   // [P]
    int n_pick;
    int n1;  // ceil(eta * n_pick), clamped to n_pick
    float *out_lo, *out_hi, *out_lb, *out_ub;
    uint64_t *out_id;
    uint8_t *keep;
    int *d_counts;
    int *dest;     // [n] scratch: destination code per row
    int *status;
    // several problems: one plan CTA per problem, output grouped by problem (children of every problem,
    // then the unpicked survivors of every problem)
    BatchDesc batch;
    int k;                   // action dimension: problem p splits only its first k * H_p coordinates
    const int *n_pick_dev;   // [P] per-problem pick quota (nullable: n_pick, n1)
    float eta;
    int cap_out;
    int *pcounts;            // [P][2] picked and unpicked survivors per problem
    int *poff;               // [P][2] first output row of the problem's children and of its unpicked rows
    int *out_prob;           // [cap_out] (nullable)
    // the paper's heuristics: pick_rule 1 fills the rest of the quota by the softmax race (pick_keys: [n]
    // scratch); split_dim (nullable) gives each pool row's dimension to split
    int pick_rule;
    float temperature;
    uint64_t pick_seed;
    float *pick_keys;
    const int *split_dim;
    int *out_split_dim;      // [cap_out] (nullable): unpicked rows keep theirs, children get -1 (not yet searched)
    const float *row_u;      // [n][d] (nullable): a vector per pool row (the best input of its search)
    float *out_row_u;        // [cap_out][d] (with row_u): unpicked rows keep theirs, children inherit the parent's
};
cudaError_t launch_split_dims(int d, const float *lo, const float *hi, const uint64_t *id, int n, const int *d_n,
                              uint64_t seed, const float *costs, int M, int top_k, int *split_dim, cudaStream_t st);
cudaError_t launch_prune_branch(const BranchArgs &a, cudaStream_t st);

}  // namespace bab
