// bound_warp.cu -- interval bounds and alpha-CROWN (Lemma 1's free lower
// slopes, optimised by projected Adam on the bound of Theorems 1-2) with one
// warp per box; every box may belong to a different problem (BatchDesc).
//
// Lane q of a box's warp owns neurons q, q + 32, ... of every layer: the
// coefficient vector of the backward pass and the activations of the adjoint
// forward pass live in registers, and each product A W_l (or W_l z) is a loop
// over the input index k in which the k-th input is broadcast with a shuffle
// and every lane adds its own outputs' terms.  Each output is therefore the
// sequential FMA sum over k from the bias (or 0) that dense_rows forms, and
// each per-box reduction is the same lane-strided partial sum plus warp tree
// of k_crown / k_alpha_fwd: the results are bit-identical to the separate
// bound, adjoint and Adam launches.  All `steps` rounds of a box run in the
// warp; the per-box arrays (interval bounds, margin helpers, slopes, Adam
// moments, coefficients before relaxation) are read from and written to
// global memory, where the L2 keeps them for small problems.
#include <cmath>

#include "bab_internal.cuh"
#include "kernels.cuh"

namespace bab {

namespace {

constexpr int kWarps = 8;  // warps (boxes in flight) per CTA
constexpr float kTwoU = 1.1920930376163597e-07f;  // 2^-23 (1 + 2^-20)

// out[p] (output j = lane + 32 p < Nn) = bias[j] + sum_{k < K} in_k B[k][j], in FMA order over k;
// in_k is held by lane k % 32 in slot k / 32.  Outputs j >= Nn are 0.
template <int P>
__device__ __forceinline__ void dense_warp(const float (&in)[P], int K, const float *__restrict__ B, int Nn,
                                           const float *__restrict__ bias, float (&out)[P])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int j = lane + 32 * p;
        out[p] = (bias && j < Nn) ? bias[j] : 0.f;
    }
    // K is a multiple of 4: four inputs per round, their weights loaded ahead of the FMA chain
    const float *Bj = B + lane;
#pragma unroll
    for (int pk = 0; pk < P; ++pk) {
        if (32 * pk >= K) break;
        const int kn = min(32, K - 32 * pk);
        for (int kl = 0; kl < kn; kl += 4) {
            float x[4], w[4][P];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                x[u] = __shfl_sync(0xFFFFFFFFu, in[pk], kl + u);
#pragma unroll
                for (int p = 0; p < P; ++p) w[u][p] = (lane + 32 * p < Nn) ? Bj[32 * p] : 0.f;
                Bj += Nn;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int p = 0; p < P; ++p)
                    if (lane + 32 * p < Nn) out[p] = fmaf(x[u], w[u][p], out[p]);
        }
    }
}

// out[p] (output j = lane + 32 p < Nn) = bias[j] + sum_{k < K} in_s[k] Wr[j ld + k], in FMA order over k (the
// same sum as dense_warp).  in_s: the warp's input vector in shared memory (K a multiple of 4); Wr: one padded
// row per output, ld = 4 mod 8 so that the float4 loads of a quarter warp hit distinct banks.
template <int P>
__device__ __forceinline__ void dense_rs(const float *__restrict__ in_s, int K, const float *__restrict__ Wr, int ld,
                                         int Nn, const float *__restrict__ bias, float (&out)[P])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int j = lane + 32 * p;
        out[p] = (bias && j < Nn) ? bias[j] : 0.f;
    }
    for (int k = 0; k < K; k += 4) {
        const float4 x = *reinterpret_cast<const float4 *>(in_s + k);
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const int j = lane + 32 * p;
            if (j < Nn) {
                const float4 w = *reinterpret_cast<const float4 *>(Wr + (size_t)j * ld + k);
                out[p] = fmaf(x.x, w.x, out[p]);
                out[p] = fmaf(x.y, w.y, out[p]);
                out[p] = fmaf(x.z, w.z, out[p]);
                out[p] = fmaf(x.w, w.w, out[p]);
            }
        }
    }
}

// Padded-row layout of one network in shared memory: per layer the forward rows (W_l row q, K = pad4(d_{l-1})),
// the backward rows (column c of W_l, K = pad4(d_l)) and the biases.
struct RowsLayout {
    int offF[kMaxLayers + 1], ldF[kMaxLayers + 1], offB[kMaxLayers + 1], ldB[kMaxLayers + 1], offb[kMaxLayers + 1];
    int floats;
};

__host__ __device__ inline int row_ld(int K) { return ((K + 7) & ~7) + 4; }

__host__ __device__ inline RowsLayout rows_layout(const NetDesc &N)
{
    RowsLayout R{};
    int o = 0;
    for (int l = 1; l <= N.L; ++l) {
        const int Kp = pad4(N.dims[l - 1]), Np = pad4(N.dims[l]);
        R.offF[l] = o;
        R.ldF[l] = row_ld(Kp);
        o += Np * R.ldF[l];
        R.offB[l] = o;
        R.ldB[l] = row_ld(Np);
        o += Kp * R.ldB[l];
        R.offb[l] = o;
        o += Np;
    }
    R.floats = (o + 3) & ~3;
    return R;
}

}  // namespace

// P: neurons per lane (every layer width <= 32 P).  ROWS: the products of the boxes whose problem is the round's
// read the network from shared memory in padded rows (dense_rs); other boxes, and ROWS = false, read the images
// from global memory with shuffle broadcasts (dense_warp).  Both sum in the same order.
// OBST: the pushing-with-obstacles cost (a separate instance, so that the squared-distance kernel carries none of
// its code or registers).
template <int P, bool ROWS, bool OBST>
__global__ void __launch_bounds__(kWarps * 32, P <= 2 ? 4 : (P <= 4 ? 2 : 1))
    k_alpha_warp(BoundArgs a, int steps, float lr, float *alpha_g, float *m_g, float *v_g, const AdamTable tab)
{
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    const NetDesc &N = a.net;
    const int s = N.s, k = N.k, L = N.L, Hm = a.batch.Hmax, d = a.d, sumh = N.sumh, sw = sumh + s, d4 = pad4(d);
    __shared__ RowsLayout R;
    if (threadIdx.x == 0) R = rows_layout(N);
    __syncthreads();
    float *rows = sm;
    float *p = sm + (ROWS ? R.floats : 0);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float *vin = p + (size_t)wib * (N.maxw_p + 2 * d4);  // the warp's product input
    float *mu = vin + N.maxw_p;                          // coefficients of u, per warp
    float *us = mu + d4;                                 // concretizing point u*, per warp

    const int nlive = live_count(a.n, a.d_n, a.row0);
    const size_t hs = (size_t)Hm * sumh;  // per-box stride of the [H][sumh] arrays
    const bool opt = steps > 0;           // steps == 0: one bound with the adaptive slopes, no adjoint
    constexpr bool obst = OBST;           // the pushing-with-obstacles cost (one problem, s <= 32)
    int loaded = -1;                      // the problem whose rows are in shared memory
    for (int base = blockIdx.x * kWarps; base < nlive; base += gridDim.x * kWarps) {
        // a round of kWarps boxes; the rows of its first box's problem serve every box of that problem
        const int pr = row_problem(a.batch, base);
        if (ROWS && pr != loaded) {
            __syncthreads();
            const float *F = a.fwd + (size_t)pr * N.img_floats, *Bw = a.bwd + (size_t)pr * N.img_floats;
            for (int l = 1; l <= L; ++l) {
                const int Kp = pad4(N.dims[l - 1]), Np = pad4(N.dims[l]);
                for (int i = threadIdx.x; i < Np * Kp; i += blockDim.x) {
                    const int q = i / Kp, c = i % Kp;
                    rows[R.offF[l] + q * R.ldF[l] + c] = Bw[N.bwd_w[l] + i];
                }
                for (int i = threadIdx.x; i < Kp * Np; i += blockDim.x) {
                    const int c = i / Np, q = i % Np;
                    rows[R.offB[l] + c * R.ldB[l] + q] = F[N.fwd_w[l] + i];
                }
                for (int i = threadIdx.x; i < Np; i += blockDim.x) rows[R.offb[l] + i] = F[N.fwd_b[l] + i];
            }
            __syncthreads();
            loaded = pr;
        }
        const int box = base + wib;
        if (box >= nlive) continue;
        // the box's problem: weights, start, goal, horizon and rho
        const int pb = row_problem(a.batch, box);
        const bool use_rows = ROWS && pb == loaded;
        const float *fwd = a.fwd + (size_t)pb * N.img_floats, *bwd = a.bwd + (size_t)pb * N.img_floats;
        // forward product of layer l: out[q] = b[q] + sum_c W[q][c] in[c]
        auto dense_f = [&](const float (&in)[P], int l, float (&out)[P]) {
            const int Kp = pad4(N.dims[l - 1]), Np = pad4(N.dims[l]);
            if (use_rows) {
#pragma unroll
                for (int q = 0; q < P; ++q)
                    if (lane + 32 * q < Kp) vin[lane + 32 * q] = in[q];
                __syncwarp();
                dense_rs<P>(vin, Kp, rows + R.offF[l], R.ldF[l], Np, rows + R.offb[l], out);
                __syncwarp();
            } else {
                dense_warp<P>(in, Kp, fwd + N.fwd_w[l], Np, fwd + N.fwd_b[l], out);
            }
        };
        // backward product of layer l: out[c] = sum_q in[q] W[q][c]
        auto dense_b = [&](const float (&in)[P], int l, float (&out)[P]) {
            const int Kp = pad4(N.dims[l - 1]), Np = pad4(N.dims[l]);
            if (use_rows) {
#pragma unroll
                for (int q = 0; q < P; ++q)
                    if (lane + 32 * q < Np) vin[lane + 32 * q] = in[q];
                __syncwarp();
                dense_rs<P>(vin, Np, rows + R.offB[l], R.ldB[l], Kp, nullptr, out);
                __syncwarp();
            } else {
                dense_warp<P>(in, Np, bwd + N.bwd_w[l], Kp, nullptr, out);
            }
        };
        const float *x0 = a.x0 + (size_t)pb * s, *goal = a.goal + (size_t)pb * s;
        const int H = problem_H(a.batch, pb, a.H), dp = k * H;
        const float rho = problem_rho(a.batch, pb, a.rho);
        const float *pl = a.pre_lo + box * hs, *ph = a.pre_hi + box * hs;
        const float *S = a.S + (size_t)box * Hm * sw;
        const float *xlo = a.x_lo + (size_t)box * (Hm + 1) * s, *xhi = a.x_hi + (size_t)box * (Hm + 1) * s;
        const float *blo = a.lo + (size_t)box * d, *bhi = a.hi + (size_t)box * d;
        float *al = opt ? alpha_g + box * hs : nullptr, *am = opt ? m_g + box * hs : nullptr;
        float *av = opt ? v_g + box * hs : nullptr, *Ap = opt ? a.A_pre + box * hs : nullptr;
        if (opt)
            for (size_t i = lane; i < (size_t)H * sumh; i += 32) {
                al[i] = (ph[i] >= -pl[i]) ? 1.f : 0.f;  // adaptive initial slopes
                am[i] = 0.f;
                av[i] = 0.f;
            }
        __syncwarp();
        float lb_best = -INFINITY;
        for (int step = 1; step <= (opt ? steps : 1); ++step) {
            // ------------------------------ bound (Theorems 1-2) ------------------------------
            float A[P], lam[P], tmp[P];
            float cst, mg = 0.f;
            // the pushing-with-obstacles cost: the pusher penalties' coefficient of every earlier action (2) and
            // the sum of its magnitudes (2), accumulated backward from step H (the same values on every lane)
            float Pu[4] = {0.f, 0.f, 0.f, 0.f};
            if (obst) {
                // its linear lower bound on x_H (lane i the coefficient of coordinate i < s <= 32), then the pusher
                // penalties at H
                float aa = 0.f;
                float c = obstacle_state_lin(a.cost, H, s, xlo + (size_t)H * s, xhi + (size_t)H * s, goal, lane, aa);
#pragma unroll
                for (int q = 0; q < P; ++q) lam[q] = (q == 0 && lane < s) ? aa : 0.f;
                cst = __fadd_rd(c, pusher_lin(a.cost, H, k, blo, bhi, Pu, Pu + 2));
            } else {
                float c = 0.f;
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const int i = lane + 32 * q;
                    float aa = 0.f;
                    if (i < s) {
                        const float g = goal[i];
                        const float Ls = __fsub_rd(xlo[(size_t)H * s + i], g), Us = __fsub_ru(xhi[(size_t)H * s + i], g);
                        const float m = 0.5f * (Ls + Us);
                        aa = 2.f * m;
                        c = __fadd_rd(c, __fmaf_rd(-aa, g, -__fmul_ru(m, m)));
                    }
                    lam[q] = aa;
                }
                cst = warp_sum_rd(c);
            }
            for (int t = H - 1; t >= 0; --t) {
                {
                    const int NpL = pad4(N.dims[L]);
                    const float *bL = bwd + N.bwd_b[L];
                    float c = 0.f, e = 0.f;
#pragma unroll
                    for (int q = 0; q < P; ++q) {
                        const int i = lane + 32 * q;
                        const float Av = i < s ? lam[q] : 0.f;
                        A[q] = Av;
                        if (i < s) {
                            c = __fmaf_rd(Av, bL[i], c);
                            e = __fmaf_ru(fabsf(Av), S[(size_t)t * sw + sumh + i], e);
                        }
                    }
                    c = warp_sum_rd(c);
                    e = warp_sum_ru(e);
                    cst = __fadd_rd(cst, c);
                    mg = __fmaf_ru(N.gam[L], e, mg);
                    dense_b(A, L, tmp);
#pragma unroll
                    for (int q = 0; q < P; ++q) A[q] = tmp[q];
                }
                for (int l = L - 1; l >= 1; --l) {
                    const int dl = N.dims[l];
                    const float *bl = bwd + N.bwd_b[l];
                    float c = 0.f, eg = 0.f, er = 0.f;
#pragma unroll
                    for (int q = 0; q < P; ++q) {
                        const int j = lane + 32 * q;
                        if (j < dl) {
                            const size_t idx = (size_t)t * sumh + N.hoff[l] + j;
                            const float zl = pl[idx], zu = ph[idx];
                            const float Av = A[q];
                            float D, ci;
                            if (opt) {
                                Ap[idx] = Av;
                                relax_select(zl, zu, Av, al[idx], true, D, ci);
                            } else {
                                relax_select(zl, zu, Av, 0.f, false, D, ci);
                            }
                            const float Apj = Av * D;
                            A[q] = Apj;
                            c = __fmaf_rd(Av, ci, c);
                            c = __fmaf_rd(Apj, bl[j], c);
                            eg = __fmaf_ru(fabsf(Apj), S[(size_t)t * sw + N.hoff[l] + j], eg);
                            if (D != 0.f && D != 1.f) er = __fmaf_ru(fabsf(Apj), fmaxf(-zl, zu), er);
                        }
                    }
                    c = warp_sum_rd(c);
                    eg = warp_sum_ru(eg);
                    er = warp_sum_ru(er);
                    cst = __fadd_rd(cst, c);
                    mg = __fadd_ru(mg, __fmaf_ru(N.gam[l], eg, __fmul_ru(kTwoU, er)));
                    dense_b(A, l, tmp);
#pragma unroll
                    for (int q = 0; q < P; ++q) A[q] = tmp[q];
                }
                if (obst) {
                    // mu_t = A_u + the pusher coefficient of the later steps (its rounding, H additions, in the
                    // margin), each action's term on lane j as in crown_rows; lam <- lam + A_x + the obstacle cost's
                    // coefficient at x_t; then the pusher penalties at t
#pragma unroll
                    for (int q = 0; q < P; ++q) {
                        const int i = lane + 32 * q;
                        if (i >= s && i < s + k) mu[t * k + (i - s)] = A[q];
                    }
                    __syncwarp();
                    float e = 0.f;
                    for (int j = lane; j < k; j += 32) {
                        const float Au = mu[t * k + j];
                        const float Pj = j < 2 ? Pu[j] : 0.f, Pa = j < 2 ? Pu[2 + j] : 0.f;
                        mu[t * k + j] = Au + Pj;
                        const float um = fmaxf(fabsf(blo[t * k + j]), fabsf(bhi[t * k + j]));
                        e = __fmaf_ru(__fmul_ru(__fmul_ru((float)(H + 2), kTwoU), __fadd_ru(fabsf(Au), Pa)), um, e);
                    }
                    __syncwarp();
                    float aa = 0.f, c = 0.f;
                    if (t >= 1)
                        c = obstacle_state_lin(a.cost, t, s, xlo + (size_t)t * s, xhi + (size_t)t * s, goal, lane, aa);
                    if (lane < s) {
                        const float Ax = A[0], lo_ = lam[0];
                        const float B = t >= 1 ? fmaxf(fabsf(xlo[(size_t)t * s + lane]), fabsf(xhi[(size_t)t * s + lane]))
                                               : fabsf(x0[lane]);
                        lam[0] = (lo_ + Ax) + aa;
                        const float mag = __fadd_ru(__fadd_ru(fabsf(lo_), fabsf(Ax)), fabsf(aa));
                        e = __fmaf_ru(__fmul_ru(kTwoU, mag), B, e);
                    }
                    e = warp_sum_ru(e);
                    if (t >= 1) c = __fadd_rd(c, pusher_lin(a.cost, t, k, blo, bhi, Pu, Pu + 2));
                    cst = __fadd_rd(cst, c);
                    mg = __fadd_ru(mg, e);
                    continue;
                }
                // A is on [x_t | u_t]: mu_t = A_u; lam <- lam + A_x (+ tangent of ||x_t - g||^2 for t >= 1)
                float c = 0.f, e = 0.f;
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const int i = lane + 32 * q;
                    if (i >= s && i < s + k) mu[t * k + (i - s)] = A[q];
                    if (i < s) {
                        const float Ax = A[q], lo_ = lam[q];
                        float aa = 0.f, B;
                        if (t >= 1) {
                            const float g = goal[i];
                            const float xl = xlo[(size_t)t * s + i], xu = xhi[(size_t)t * s + i];
                            const float Ls = __fsub_rd(xl, g), Us = __fsub_ru(xu, g);
                            const float m = 0.5f * (Ls + Us);
                            aa = 2.f * m;
                            c = __fadd_rd(c, __fmaf_rd(-aa, g, -__fmul_ru(m, m)));
                            B = fmaxf(fabsf(xl), fabsf(xu));
                        } else {
                            B = fabsf(x0[i]);
                        }
                        lam[q] = (lo_ + Ax) + aa;
                        const float mag = __fadd_ru(__fadd_ru(fabsf(lo_), fabsf(Ax)), fabsf(aa));
                        e = __fmaf_ru(__fmul_ru(kTwoU, mag), B, e);
                    }
                }
                c = warp_sum_rd(c);
                e = warp_sum_ru(e);
                cst = __fadd_rd(cst, c);
                mg = __fadd_ru(mg, e);
            }
            __syncwarp();
            // lam . x0, then Theorem 2 in box form
            float lbv;
            {
                float c = 0.f, val = 0.f, e = 0.f;
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const int i = lane + 32 * q;
                    if (i < s) c = __fmaf_rd(lam[q], x0[i], c);
                }
                c = __fadd_rd(cst, warp_sum_rd(c));
                for (int j = lane; j < dp; j += 32) {
                    const float m_ = mu[j];
                    const float lo = blo[j], hi = bhi[j];
                    float u_s, vj;
                    if (rho > 0.f) {
                        const float uc = -m_ / (2.f * rho);
                        if (uc >= lo && uc <= hi) {
                            u_s = uc;
                            vj = __fdiv_rd(-__fmul_ru(m_, m_), 4.f * rho);
                        } else {
                            u_s = uc < lo ? lo : hi;
                            vj = __fmaf_rd(m_, u_s, __fmul_rd(rho, __fmul_rd(u_s, u_s)));
                            const float du = __fmul_ru(kTwoU, fabsf(uc));
                            e = __fmaf_ru(__fmul_ru(rho, du), du, e);
                        }
                    } else {
                        u_s = m_ >= 0.f ? lo : hi;
                        vj = __fmul_rd(m_, u_s);
                    }
                    val = __fadd_rd(val, vj);
                    us[j] = u_s;
                }
                val = warp_sum_rd(val);
                e = warp_sum_ru(e);
                const float raw = __fadd_rd(c, val);
                const float marg = __fadd_ru(mg, e);
                lbv = __fsub_rd(raw, marg);
            }
            lb_best = fmaxf(lb_best, lbv);
            __syncwarp();
            if (!opt) break;
            // ------------------ adjoint: relaxed network forward from x_0 and u*, then Adam ------------------
            AdamStep ast;
            ast.lr = lr;
            if (step <= kAdamTable) {
                ast.bc1 = tab.bc1[step - 1];
                ast.bc2 = tab.bc2[step - 1];
            } else {
                ast.bc1 = (float)(1.0 - pow(0.9, (double)step));
                ast.bc2 = (float)(1.0 - pow(0.999, (double)step));
            }
            float x[P];
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const int i = lane + 32 * q;
                x[q] = i < s ? x0[i] : 0.f;
            }
            for (int t = 0; t < H; ++t) {
                float Z[P];
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const int c = lane + 32 * q;
                    Z[q] = c < s ? x[q] : (c < s + k ? us[t * k + (c - s)] : 0.f);
                }
                for (int l = 1; l <= L; ++l) {
                    dense_f(Z, l, tmp);
                    if (l < L) {
                        const int dl = N.dims[l];
#pragma unroll
                        for (int q = 0; q < P; ++q) {
                            const int j = lane + 32 * q;
                            if (j < dl) {
                                const size_t idx = (size_t)t * sumh + N.hoff[l] + j;
                                const float z = tmp[q];
                                const float zl = pl[idx], zu = ph[idx], Av = Ap[idx];
                                float D, c;
                                relax_select(zl, zu, Av, al[idx], true, D, c);
                                const bool unstable = zl < 0.f && zu > 0.f;
                                const float g = (unstable && Av >= 0.f) ? Av * z : 0.f;
                                float alv = al[idx], mv = am[idx], vv = av[idx];
                                adam_update(alv, mv, vv, g, ast);
                                al[idx] = alv;
                                am[idx] = mv;
                                av[idx] = vv;
                                tmp[q] = fmaf(D, z, c);
                            }
                        }
                    }
#pragma unroll
                    for (int q = 0; q < P; ++q) Z[q] = tmp[q];
                }
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const int i = lane + 32 * q;
                    if (i < s) x[q] += Z[q];
                }
            }
            __syncwarp();
        }
        if (lane == 0) a.lb_best[box] = lb_best;
    }
}

template <int P>
static cudaError_t launch_warp_variant(const BoundArgs &a, int steps, float lr, float *alpha, float *m, float *v,
                                       cudaStream_t st)
{
    int dev, max_optin = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const size_t per_warp = (size_t)(a.net.maxw_p + 2 * pad4(a.d)) * kWarps * sizeof(float);
    const size_t with_rows = per_warp + (size_t)rows_layout(a.net).floats * sizeof(float);
    // the padded rows pay while a few CTAs still fit on an SM
    const bool rows = with_rows * 2 + 2048 <= (size_t)max_optin;
    const size_t smem = rows ? with_rows : per_warp;
    if (smem + 1024 > (size_t)max_optin) return cudaErrorInvalidConfiguration;
    const bool ob = a.cost.kind == 1;
    auto kern = rows ? (ob ? k_alpha_warp<P, true, true> : k_alpha_warp<P, true, false>)
                     : (ob ? k_alpha_warp<P, false, true> : k_alpha_warp<P, false, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kWarps * 32, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int need = (a.n + kWarps - 1) / kWarps;
    const int grid = need < nsm * occ ? need : nsm * occ;
    AdamTable tab;
    fill_adam_table(tab);
    kern<<<grid, kWarps * 32, smem, st>>>(a, steps, lr, alpha, m, v, tab);
    return cudaGetLastError();
}


// Interval bound propagation (outward-rounded FP32) through the H-step unrolled
// network, one warp per box: lane q holds the interval of inputs and outputs
// q, q + 32, ...; per output the three directed-rounding sums (lower, upper,
// and S = sum_j |W_kj| max|a_j|) run over the inputs in order from the bias, as
// in k_ibp, so the bounds are bit-identical to it.  Writes the pre-activation
// bounds, the state intervals, S and (nullable) the interval bound of the cost.
template <int P, bool WSMEM>
__global__ void __launch_bounds__(kWarps * 32, P <= 2 ? 4 : (P <= 4 ? 2 : 1)) k_ibp_warp(BoundArgs a)
{
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    const NetDesc &N = a.net;
    const int s = N.s, k = N.k, L = N.L, Hm = a.batch.Hmax, d = a.d, sumh = N.sumh, sw = sumh + s;
    const float *fwd = a.fwd;
    if (WSMEM) {
        for (int i = threadIdx.x; i < N.img_floats / 4; i += blockDim.x)
            smem4[i] = reinterpret_cast<const float4 *>(a.fwd)[i];
        fwd = sm;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nlive = live_count(a.n, a.d_n, a.row0);
    for (int box = blockIdx.x * kWarps + wib; box < nlive; box += gridDim.x * kWarps) {
        const int pb = row_problem(a.batch, box);
        if (!WSMEM) fwd = a.fwd + (size_t)pb * N.img_floats;
        const float *x0 = a.x0 + (size_t)pb * s, *goal = a.goal + (size_t)pb * s;
        const int H = problem_H(a.batch, pb, a.H);
        const float rho = problem_rho(a.batch, pb, a.rho);
        const float *blo = a.lo + (size_t)box * d, *bhi = a.hi + (size_t)box * d;
        float *pl = a.pre_lo + (size_t)box * Hm * sumh, *ph = a.pre_hi + (size_t)box * Hm * sumh;
        float *S = a.S + (size_t)box * Hm * sw;
        float *xlo = a.x_lo + (size_t)box * (Hm + 1) * s, *xhi = a.x_hi + (size_t)box * (Hm + 1) * s;
        float xl[P], xu[P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int i = lane + 32 * q;
            xl[q] = xu[q] = i < s ? x0[i] : 0.f;
            if (i < s) {
                xlo[i] = x0[i];
                xhi[i] = x0[i];
            }
        }
        float lbacc = 0.f;
        for (int t = 0; t < H; ++t) {
            float zl[P], zu[P];
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const int c = lane + 32 * q;
                zl[q] = c < s ? xl[q] : (c < s + k ? blo[t * k + (c - s)] : 0.f);
                zu[q] = c < s ? xu[q] : (c < s + k ? bhi[t * k + (c - s)] : 0.f);
            }
            if (rho > 0.f) {
                float v = 0.f;
                for (int j = lane; j < k; j += 32) v = __fadd_rd(v, sq_min_rd(blo[t * k + j], bhi[t * k + j]));
                v = warp_sum_rd(v);
                lbacc = __fadd_rd(lbacc, __fmul_rd(rho, v));
            }
            for (int l = 1; l <= L; ++l) {
                const int Kp = pad4(N.dims[l - 1]), Np = pad4(N.dims[l]), dl = N.dims[l];
                const float *W = fwd + N.fwd_w[l], *bias = fwd + N.fwd_b[l];
                float al_[P], ah_[P], as_[P];
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const int j = lane + 32 * q;
                    const float bj = j < Np ? bias[j] : 0.f;
                    al_[q] = ah_[q] = bj;
                    as_[q] = 0.f;
                }
                const float *Wk = W + lane;
#pragma unroll
                for (int pk = 0; pk < P; ++pk) {
                    if (32 * pk >= Kp) break;
                    const int kn = min(32, Kp - 32 * pk);
                    for (int kl = 0; kl < kn; ++kl) {
                        const float il = __shfl_sync(0xFFFFFFFFu, zl[pk], kl);
                        const float ih = __shfl_sync(0xFFFFFFFFu, zu[pk], kl);
                        const float am = fmaxf(fabsf(il), fabsf(ih));
#pragma unroll
                        for (int q = 0; q < P; ++q) {
                            if (lane + 32 * q < Np) {
                                const float w = Wk[32 * q];
                                const bool pos = w >= 0.f;
                                al_[q] = __fmaf_rd(w, pos ? il : ih, al_[q]);
                                ah_[q] = __fmaf_ru(w, pos ? ih : il, ah_[q]);
                                as_[q] = __fmaf_ru(fabsf(w), am, as_[q]);
                            }
                        }
                        Wk += Np;
                    }
                }
                const int soff = (l < L) ? N.hoff[l] : sumh;
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const int j = lane + 32 * q;
                    if (j < dl) {
                        S[(size_t)t * sw + soff + j] = as_[q];
                        if (l < L) {
                            pl[(size_t)t * sumh + N.hoff[l] + j] = al_[q];
                            ph[(size_t)t * sumh + N.hoff[l] + j] = ah_[q];
                        }
                    }
                    if (l < L && j < dl) {
                        zl[q] = fmaxf(al_[q], 0.f);
                        zu[q] = fmaxf(ah_[q], 0.f);
                    } else {
                        zl[q] = al_[q];
                        zu[q] = ah_[q];
                    }
                }
            }
            // x_{t+1} in [x_t] + [z_L]; interval bound of ||x_{t+1} - g||^2
            float v = 0.f;
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const int i = lane + 32 * q;
                if (i < s) {
                    const float nl = __fadd_rd(xl[q], zl[q]), nh = __fadd_ru(xu[q], zu[q]);
                    xl[q] = nl;
                    xu[q] = nh;
                    xlo[(size_t)(t + 1) * s + i] = nl;
                    xhi[(size_t)(t + 1) * s + i] = nh;
                    const float g = goal[i];
                    v = __fadd_rd(v, sq_min_rd(__fsub_rd(nl, g), __fsub_ru(nh, g)));
                }
            }
            v = warp_sum_rd(v);
            lbacc = __fadd_rd(lbacc, v);
        }
        if (a.lb_ibp && lane == 0) a.lb_ibp[box] = lbacc;
    }
}

template <int P>
static cudaError_t launch_ibp_variant(const BoundArgs &a, cudaStream_t st)
{
    int dev, max_optin = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const size_t img = (size_t)a.net.img_floats * sizeof(float);
    const bool wsmem = a.batch.P <= 1 && img + 1024 <= (size_t)max_optin;
    const size_t smem = wsmem ? img : 0;
    auto kern = wsmem ? k_ibp_warp<P, true> : k_ibp_warp<P, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kWarps * 32, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int need = (a.n + kWarps - 1) / kWarps;
    const int grid = need < nsm * occ ? need : nsm * occ;
    kern<<<grid, kWarps * 32, smem, st>>>(a);
    return cudaGetLastError();
}

static int lanes_needed(const NetDesc &N)
{
    int maxw = 0;
    for (int l = 0; l <= N.L; ++l) maxw = N.dims[l] > maxw ? N.dims[l] : maxw;
    // every layer's width and the input row [x | u] must fit the lanes' slots
    const int need = pad4(maxw) > pad4(N.s + N.k) ? pad4(maxw) : pad4(N.s + N.k);
    return need <= 32 ? 1 : need <= 64 ? 2 : need <= 128 ? 4 : need <= 256 ? 8 : 0;
}

cudaError_t launch_ibp_warp(const BoundArgs &a, cudaStream_t st)
{
    if (a.n <= 0) return cudaSuccess;
    switch (lanes_needed(a.net)) {
        case 1: return launch_ibp_variant<1>(a, st);
        case 2: return launch_ibp_variant<2>(a, st);
        case 4: return launch_ibp_variant<4>(a, st);
        case 8: return launch_ibp_variant<8>(a, st);
        default: return cudaErrorInvalidConfiguration;
    }
}

cudaError_t launch_alpha_warp(const BoundArgs &a, int steps, float lr, float *alpha, float *m, float *v,
                              cudaStream_t st)
{
    if (a.n <= 0) return cudaSuccess;
    switch (lanes_needed(a.net)) {
        case 1: return launch_warp_variant<1>(a, steps, lr, alpha, m, v, st);
        case 2: return launch_warp_variant<2>(a, steps, lr, alpha, m, v, st);
        case 4: return launch_warp_variant<4>(a, steps, lr, alpha, m, v, st);
        case 8: return launch_warp_variant<8>(a, steps, lr, alpha, m, v, st);
        default: return cudaErrorInvalidConfiguration;
    }
}

// out_l[p] / out_h[p] (output c = lane + 32 p < Nn) = sum_{j < K} of W[j][c] times gl_j or gh_j, the factor
// picked by the sign of W[j][c] (W+ gl + W- gh, and W+ gh + W- gl): the transposed step of an interval
// product.  B is a backward image W_l [Kp][Np] (rows j = the layer's outputs).
template <int P>
__device__ __forceinline__ void dense_sign_warp(const float (&gl)[P], const float (&gh)[P], int K,
                                                const float *__restrict__ B, int Nn, float (&out_l)[P],
                                                float (&out_h)[P])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int p = 0; p < P; ++p) out_l[p] = out_h[p] = 0.f;
    const float *Bj = B + lane;
#pragma unroll
    for (int pk = 0; pk < P; ++pk) {
        if (32 * pk >= K) break;
        const int kn = min(32, K - 32 * pk);
        for (int kl = 0; kl < kn; ++kl) {
            const float xl = __shfl_sync(0xFFFFFFFFu, gl[pk], kl), xh = __shfl_sync(0xFFFFFFFFu, gh[pk], kl);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                if (lane + 32 * p < Nn) {
                    const float w = Bj[32 * p];
                    const bool pos = w >= 0.f;
                    out_l[p] = fmaf(w, pos ? xl : xh, out_l[p]);
                    out_h[p] = fmaf(w, pos ? xh : xl, out_h[p]);
                }
            }
            Bj += Nn;
        }
    }
}

// Gradient of the bound with respect to the box faces (the derivative oracle_box_grad defines), one warp per
// box, from the interval bounds and a CROWN pass that stored A_pre, u* and mu:
//   1. the relaxed network forward from x_0 and u*: each unstable neuron whose upper chord was selected
//      (A < 0) gets dLB/du = A l (l - z~)/(u - l)^2 and dLB/dl = A u (z~ - u)/(u - l)^2, each cost tangent
//      dLB/dx_lo = dLB/dx_hi = x~ - g - m;
//   2. those sensitivities run back through the interval bounds' steps (transposed sign-split products, the
//      ReLU passing a derivative where its end is positive, the residual x_{t+1} = x_t + z_L) to the box;
//   3. the concretization adds mu_j + 2 rho lo_j (hi_j) where u*_j sits on that face.
// GL, GU: [n][Hmax][sumh] scratch, GX: [n][Hmax+1][s] scratch.
template <int P, bool WSMEM>
__global__ void __launch_bounds__(kWarps * 32, P <= 2 ? 4 : (P <= 4 ? 2 : 1))
    k_box_grad_warp(BoundArgs a, float *GL, float *GU, float *GX, float *grad_lo, float *grad_hi)
{
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    const NetDesc &N = a.net;
    const int s = N.s, k = N.k, L = N.L, Hm = a.batch.Hmax, d = a.d, sumh = N.sumh;
    const float *fwd = a.fwd, *bwd = a.bwd;
    if (WSMEM) {
        for (int i = threadIdx.x; i < N.img_floats / 4; i += blockDim.x) {
            smem4[i] = reinterpret_cast<const float4 *>(a.fwd)[i];
            reinterpret_cast<float4 *>(sm + N.img_floats)[i] = reinterpret_cast<const float4 *>(a.bwd)[i];
        }
        fwd = sm;
        bwd = sm + N.img_floats;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nlive = live_count(a.n, a.d_n, a.row0);
    const size_t hs = (size_t)Hm * sumh;
    const bool has_alpha = a.alpha != nullptr;
    for (int box = blockIdx.x * kWarps + wib; box < nlive; box += gridDim.x * kWarps) {
        const int pb = row_problem(a.batch, box);
        if (!WSMEM) {
            fwd = a.fwd + (size_t)pb * N.img_floats;
            bwd = a.bwd + (size_t)pb * N.img_floats;
        }
        const float *x0 = a.x0 + (size_t)pb * s, *goal = a.goal + (size_t)pb * s;
        const int H = problem_H(a.batch, pb, a.H), dp = k * H;
        const float rho = problem_rho(a.batch, pb, a.rho);
        const float *pl = a.pre_lo + box * hs, *ph = a.pre_hi + box * hs, *Ap = a.A_pre + box * hs;
        const float *al = has_alpha ? a.alpha + box * hs : nullptr;
        const float *xlo = a.x_lo + (size_t)box * (Hm + 1) * s, *xhi = a.x_hi + (size_t)box * (Hm + 1) * s;
        const float *us = a.ustar + (size_t)box * d, *mu = a.lin_coef + (size_t)box * d;
        const float *blo = a.lo + (size_t)box * d, *bhi = a.hi + (size_t)box * d;
        float *gl_ = GL + box * hs, *gu_ = GU + box * hs, *gx = GX + (size_t)box * (Hm + 1) * s;
        float *glo = grad_lo + (size_t)box * d, *ghi = grad_hi + (size_t)box * d;

        // ---- 1. relaxed network forward from x_0 and u*, with the bound's sensitivities ----
        float x[P], Z[P], tmp[P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int i = lane + 32 * q;
            x[q] = i < s ? x0[i] : 0.f;
        }
        for (int t = 0; t < H; ++t) {
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const int c = lane + 32 * q;
                Z[q] = c < s ? x[q] : (c < s + k ? us[t * k + (c - s)] : 0.f);
            }
            for (int l = 1; l <= L; ++l) {
                dense_warp<P>(Z, pad4(N.dims[l - 1]), fwd + N.fwd_w[l], pad4(N.dims[l]), fwd + N.fwd_b[l], tmp);
                if (l < L) {
                    const int dl = N.dims[l];
#pragma unroll
                    for (int q = 0; q < P; ++q) {
                        const int j = lane + 32 * q;
                        if (j < dl) {
                            const size_t idx = (size_t)t * sumh + N.hoff[l] + j;
                            const float z = tmp[q], zl = pl[idx], zu = ph[idx], A = Ap[idx];
                            float D, c;
                            relax_select(zl, zu, A, has_alpha ? al[idx] : 0.f, has_alpha, D, c);
                            float gL = 0.f, gU = 0.f;
                            if (zl < 0.f && zu > 0.f && A < 0.f) {
                                const float w = zu - zl, w2 = w * w;
                                gU = A * zl * (zl - z) / w2;
                                gL = A * zu * (z - zu) / w2;
                            }
                            gl_[idx] = gL;
                            gu_[idx] = gU;
                            tmp[q] = fmaf(D, z, c);
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < P; ++q) Z[q] = tmp[q];
            }
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const int i = lane + 32 * q;
                if (i < s) {
                    x[q] += Z[q];
                    const float g = goal[i];
                    const float Ls = __fsub_rd(xlo[(size_t)(t + 1) * s + i], g);
                    const float Us = __fsub_ru(xhi[(size_t)(t + 1) * s + i], g);
                    const float m = 0.5f * (Ls + Us);
                    gx[(size_t)(t + 1) * s + i] = (x[q] - g) - m;
                }
            }
        }
        __syncwarp();

        // ---- 2. back through the interval bounds to the box ----
        float Gxl[P], Gxh[P], Gl[P], Gh[P], Al[P], Ah[P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int i = lane + 32 * q;
            Gxl[q] = Gxh[q] = i < s ? gx[(size_t)H * s + i] : 0.f;
        }
        for (int t = H - 1; t >= 0; --t) {
#pragma unroll
            for (int q = 0; q < P; ++q) {
                Gl[q] = Gxl[q];
                Gh[q] = Gxh[q];
            }
            for (int l = L; l >= 1; --l) {
                if (l < L) {
                    const int dl = N.dims[l];
#pragma unroll
                    for (int q = 0; q < P; ++q) {
                        const int j = lane + 32 * q;
                        Gl[q] = Gh[q] = 0.f;
                        if (j < dl) {
                            const size_t idx = (size_t)t * sumh + N.hoff[l] + j;
                            Gl[q] = (pl[idx] > 0.f ? Al[q] : 0.f) + gl_[idx];
                            Gh[q] = (ph[idx] > 0.f ? Ah[q] : 0.f) + gu_[idx];
                        }
                    }
                }
                dense_sign_warp<P>(Gl, Gh, pad4(N.dims[l]), bwd + N.bwd_w[l], pad4(N.dims[l - 1]), Al, Ah);
            }
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const int c = lane + 32 * q;
                if (c >= s && c < s + k) {
                    glo[t * k + (c - s)] = Al[q];
                    ghi[t * k + (c - s)] = Ah[q];
                }
                if (c < s) {
                    const float tg = t >= 1 ? gx[(size_t)t * s + c] : 0.f;
                    Gxl[q] = Gxl[q] + Al[q] + tg;
                    Gxh[q] = Gxh[q] + Ah[q] + tg;
                }
            }
        }
        __syncwarp();

        // ---- 3. the concretization's own dependence on the faces ----
        for (int j = lane; j < d; j += 32) {
            if (j >= dp) {
                glo[j] = ghi[j] = 0.f;
                continue;
            }
            const float m_ = mu[j], lo = blo[j], hi = bhi[j];
            bool at_lo, at_hi;
            if (rho > 0.f) {
                const float uc = -m_ / (2.f * rho);
                at_lo = uc <= lo;
                at_hi = !at_lo && uc >= hi;
            } else {
                at_lo = m_ >= 0.f;
                at_hi = !at_lo;
            }
            (void)us;
            if (at_lo) glo[j] += m_ + 2.f * rho * lo;
            if (at_hi) ghi[j] += m_ + 2.f * rho * hi;
        }
    }
}

template <int P>
static cudaError_t launch_box_grad_variant(const BoundArgs &a, float *GL, float *GU, float *GX, float *glo,
                                           float *ghi, cudaStream_t st)
{
    int dev, max_optin = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const size_t img = 2 * (size_t)a.net.img_floats * sizeof(float);
    const bool wsmem = a.batch.P <= 1 && img + 1024 <= (size_t)max_optin;
    const size_t smem = wsmem ? img : 0;
    auto kern = wsmem ? k_box_grad_warp<P, true> : k_box_grad_warp<P, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kWarps * 32, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int need = (a.n + kWarps - 1) / kWarps;
    const int grid = need < nsm * occ ? need : nsm * occ;
    kern<<<grid, kWarps * 32, smem, st>>>(a, GL, GU, GX, glo, ghi);
    return cudaGetLastError();
}

cudaError_t launch_box_grad_warp(const BoundArgs &a, float *GL, float *GU, float *GX, float *glo, float *ghi,
                                 cudaStream_t st)
{
    if (a.n <= 0) return cudaSuccess;
    switch (lanes_needed(a.net)) {
        case 1: return launch_box_grad_variant<1>(a, GL, GU, GX, glo, ghi, st);
        case 2: return launch_box_grad_variant<2>(a, GL, GU, GX, glo, ghi, st);
        case 4: return launch_box_grad_variant<4>(a, GL, GU, GX, glo, ghi, st);
        case 8: return launch_box_grad_variant<8>(a, GL, GU, GX, glo, ghi, st);
        default: return cudaErrorInvalidConfiguration;
    }
}

}  // namespace bab
