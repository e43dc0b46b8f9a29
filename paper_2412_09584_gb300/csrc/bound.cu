// bound.cu -- lower bounds of the planning objective over boxes.
//
//   k_ibp        interval bound propagation (outward-rounded FP32) through the
//                H-step unrolled network: the pre-activation bounds that
//                Lemma 1 (Appendix B.1) needs, the state intervals, and, per
//                row k of every layer, S_k = sum_j |W_kj| max|a_j| over the
//                layer's input box (used to bound the rounding error of the
//                backward products).
//   k_crown      Theorem 1 backward propagation of the tangent-linearised cost
//                through all H steps, then Theorem 2 in box form.  Constant
//                terms are accumulated with downward rounding (so they are
//                lower bounds by construction); the rounding error of the
//                coefficient vectors (the products A W_l, the relaxation
//                products, the state-coefficient updates) is bounded a
//                posteriori and subtracted as `margin`.
//   k_alpha_fwd  forward pass of the relaxed network from x_0 and the
//                concretizing point u*, giving dLB/dalpha = A_j z~_j.
//   k_adam       projected Adam ascent on alpha.
//
// A CTA owns RB boxes (rows); the network image lives in shared memory when
// it fits (otherwise it is read through L2); the rows move through the layers
// as register-blocked FP32 products (dense_rows), and each per-row reduction
// is one warp with shuffles.
#include <cmath>

#include "bab_internal.cuh"
#include "kernels.cuh"

namespace bab {

constexpr int RB = 28;  // boxes per CTA: 4096 boxes make 147 CTAs, one wave on 152 SMs (32 left 24 SMs idle)
constexpr int NT = 512;
constexpr float kTwoU = 1.1920930376163597e-07f;  // 2^-23 (1 + 2^-20): twice the unit roundoff, rounded up

// ---------------------------------------------------------------------------
// IBP
// ---------------------------------------------------------------------------
// Paired FP32 FMA with directed rounding: (a.x b.x + c.x, a.y b.y + c.y), each rounded down (RD) or up (RU);
// per element the same result as the scalar __fmaf_rd / __fmaf_ru.
__device__ __forceinline__ unsigned long long ffma2_rd(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long d;
    asm("fma.rm.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long ffma2_ru(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long d;
    asm("fma.rp.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long pack2f(float x, float y)
{
    return (unsigned long long)__float_as_uint(x) | ((unsigned long long)__float_as_uint(y) << 32);
}
__device__ __forceinline__ float half2f(unsigned long long v, int e)
{
    return __uint_as_float((uint32_t)(e ? v >> 32 : v));
}

// Where a layer's outputs go: the interval bounds and S of step t to global memory (rows < nlive, columns < dl;
// no pre-activation bounds for the output layer), and the next layer's input (ReLU of the bounds, or the bounds
// of the output layer themselves) to the tile's shared-memory buffers.
struct IbpSink {
    float *pre_lo, *pre_hi, *S;  // at (box0 * H + t) of the [n][H][...] arrays
    size_t rstride_h, rstride_s; // per row: H * sumh, H * (sumh + s)
    int hoff, soff, dl, nrows;
    bool hidden;
};

// One layer of interval bounds for RB rows, TR rows x TN columns per thread: per output the three directed-
// rounding sums (lower, upper, and S = sum_k |W_jk| max|a_k|) over the inputs in order from the bias, the
// endpoint of each input picked by the sign of the weight; two adjacent columns run as one paired FMA.
template <int TR, int TN>
__device__ __forceinline__ void ibp_dense(const float *__restrict__ alo, const float *__restrict__ ahi, int ld,
                                          const float *__restrict__ Wt, const float *__restrict__ bias, int Kp, int Np,
                                          float *__restrict__ zlo, float *__restrict__ zhi, const IbpSink &o)
{
    static_assert(TN % 2 == 0, "column pairs");
    constexpr int TP = TN / 2;
    const int ngc = (Np + TN - 1) / TN;
    const int items = (RB / TR) * ngc;
    for (int it = threadIdx.x; it < items; it += NT) {
        const int cg = it % ngc, rg = it / ngc;
        const int c0 = cg * TN, r0 = rg * TR;
        unsigned long long accl[TR][TP], acch[TR][TP], accs[TR][TP];
#pragma unroll
        for (int jp = 0; jp < TP; ++jp) {
            const int j = c0 + 2 * jp;
            const unsigned long long b2 = pack2f(j < Np ? bias[j] : 0.f, j + 1 < Np ? bias[j + 1] : 0.f);
#pragma unroll
            for (int i = 0; i < TR; ++i) {
                accl[i][jp] = acch[i][jp] = b2;
                accs[i][jp] = 0ull;
            }
        }
        const bool full = (c0 + TN <= Np);
        for (int k = 0; k < Kp; k += 4) {
            float4 l4[TR], h4[TR];
#pragma unroll
            for (int i = 0; i < TR; ++i) {
                l4[i] = *reinterpret_cast<const float4 *>(alo + (r0 + i) * ld + k);
                h4[i] = *reinterpret_cast<const float4 *>(ahi + (r0 + i) * ld + k);
            }
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                float w[TN];
                const float *wr = Wt + (size_t)(k + kk) * Np + c0;
                if (full && TN % 4 == 0) {
                    // whole 16-byte groups (Np and c0 are multiples of 4)
#pragma unroll
                    for (int j = 0; j < TN; j += 4) {
                        const float4 q = *reinterpret_cast<const float4 *>(wr + j);
                        w[j] = q.x;
                        w[j + 1] = q.y;
                        w[j + 2] = q.z;
                        w[j + 3] = q.w;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < TN; ++j) w[j] = (c0 + j < Np) ? wr[j] : 0.f;
                }
                bool pos[TN];
                unsigned long long w2[TP], a2[TP];
#pragma unroll
                for (int jp = 0; jp < TP; ++jp) {
                    pos[2 * jp] = w[2 * jp] >= 0.f;
                    pos[2 * jp + 1] = w[2 * jp + 1] >= 0.f;
                    w2[jp] = pack2f(w[2 * jp], w[2 * jp + 1]);
                    a2[jp] = pack2f(fabsf(w[2 * jp]), fabsf(w[2 * jp + 1]));
                }
#pragma unroll
                for (int i = 0; i < TR; ++i) {
                    const float al = kk == 0 ? l4[i].x : kk == 1 ? l4[i].y : kk == 2 ? l4[i].z : l4[i].w;
                    const float ah = kk == 0 ? h4[i].x : kk == 1 ? h4[i].y : kk == 2 ? h4[i].z : h4[i].w;
                    const float am = fmaxf(fabsf(al), fabsf(ah));
                    const unsigned long long m2 = pack2f(am, am);
#pragma unroll
                    for (int jp = 0; jp < TP; ++jp) {
                        const bool p0 = pos[2 * jp], p1 = pos[2 * jp + 1];
                        accl[i][jp] = ffma2_rd(w2[jp], pack2f(p0 ? al : ah, p1 ? al : ah), accl[i][jp]);
                        acch[i][jp] = ffma2_ru(w2[jp], pack2f(p0 ? ah : al, p1 ? ah : al), acch[i][jp]);
                        accs[i][jp] = ffma2_ru(a2[jp], m2, accs[i][jp]);
                    }
                }
            }
        }
        // write the rows' bounds and S, and the next layer's input
#pragma unroll
        for (int i = 0; i < TR; ++i) {
            const int r = r0 + i;
            const bool live = r < o.nrows;
#pragma unroll
            for (int jp = 0; jp < TP; ++jp)
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int j = c0 + 2 * jp + e;
                    if (j >= Np) continue;
                    const float zl = half2f(accl[i][jp], e), zh = half2f(acch[i][jp], e);
                    if (live && j < o.dl) {
                        o.S[r * o.rstride_s + o.soff + j] = half2f(accs[i][jp], e);
                        if (o.hidden) {
                            o.pre_lo[r * o.rstride_h + o.hoff + j] = zl;
                            o.pre_hi[r * o.rstride_h + o.hoff + j] = zh;
                        }
                    }
                    const bool relu = o.hidden && j < o.dl;
                    zlo[r * ld + j] = relu ? fmaxf(zl, 0.f) : zl;
                    zhi[r * ld + j] = relu ? fmaxf(zh, 0.f) : zh;
                }
        }
    }
}

template <bool WSMEM>
__global__ void __launch_bounds__(NT) k_ibp(BoundArgs a)
{
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    const NetDesc &N = a.net;
    const int s = N.s, k = N.k, L = N.L, d = a.d, H = a.H, sumh = N.sumh;
    const int ld = N.maxw_p, s4 = pad4(s);
    const float *img = a.fwd;
    float *p = sm;
    if (WSMEM) {
        for (int i = threadIdx.x; i < N.img_floats / 4; i += NT) smem4[i] = reinterpret_cast<const float4 *>(a.fwd)[i];
        img = sm;
        p += N.img_floats;
    }
    float *blo[2], *bhi[2];
    blo[0] = p; p += RB * ld;
    bhi[0] = p; p += RB * ld;
    blo[1] = p; p += RB * ld;
    bhi[1] = p; p += RB * ld;
    float *xl = p; p += RB * s4;
    float *xu = p; p += RB * s4;
    float *lbacc = p; p += RB;
    float *pbx = p; p += 4 * RB;  // pusher position box per row (obstacle cost): lo x, lo y, hi x, hi y

    const int nlive = live_count(a.n, a.d_n, a.row0);
    const int box0 = blockIdx.x * RB;
    if (box0 >= nlive) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int Kp1 = pad4(s + k);

    for (int i = threadIdx.x; i < RB * s; i += NT) {
        const int r = i / s, c = i % s;
        xl[r * s4 + c] = a.x0[c];
        xu[r * s4 + c] = a.x0[c];
        if (box0 + r < nlive && a.x_lo) {
            a.x_lo[(size_t)(box0 + r) * (H + 1) * s + c] = a.x0[c];
            a.x_hi[(size_t)(box0 + r) * (H + 1) * s + c] = a.x0[c];
        }
    }
    for (int r = threadIdx.x; r < RB; r += NT) {
        lbacc[r] = 0.f;
        pbx[4 * r] = pbx[4 * r + 2] = a.cost.p0x;
        pbx[4 * r + 1] = pbx[4 * r + 3] = a.cost.p0y;
    }
    __syncthreads();

    for (int t = 0; t < H; ++t) {
        for (int i = threadIdx.x; i < RB * Kp1; i += NT) {
            const int r = i / Kp1, c = i % Kp1;
            const int box = box0 + r;
            float vl = 0.f, vh = 0.f;
            if (c < s) {
                vl = xl[r * s4 + c];
                vh = xu[r * s4 + c];
            } else if (c < s + k && box < nlive) {
                vl = a.lo[(size_t)box * d + t * k + (c - s)];
                vh = a.hi[(size_t)box * d + t * k + (c - s)];
            }
            blo[0][r * ld + c] = vl;
            bhi[0][r * ld + c] = vh;
        }
        if (a.cost.kind == 1)
            for (int r = threadIdx.x; r < RB; r += NT)
                if (box0 + r < nlive) {
                    const float *ul = a.lo + (size_t)(box0 + r) * d + t * k, *uh = a.hi + (size_t)(box0 + r) * d + t * k;
                    pbx[4 * r] = __fadd_rd(pbx[4 * r], ul[0]);
                    pbx[4 * r + 1] = __fadd_rd(pbx[4 * r + 1], ul[1]);
                    pbx[4 * r + 2] = __fadd_ru(pbx[4 * r + 2], uh[0]);
                    pbx[4 * r + 3] = __fadd_ru(pbx[4 * r + 3], uh[1]);
                }
        if (a.rho > 0.f) {
            for (int r = warp; r < RB; r += NT / 32) {
                const int box = box0 + r;
                float v = 0.f;
                if (box < nlive)
                    for (int j = lane; j < k; j += 32)
                        v = __fadd_rd(v, sq_min_rd(a.lo[(size_t)box * d + t * k + j], a.hi[(size_t)box * d + t * k + j]));
                v = warp_sum_rd(v);
                if (lane == 0) lbacc[r] = __fadd_rd(lbacc[r], __fmul_rd(a.rho, v));
            }
        }
        __syncthreads();
        int cur = 0;
        for (int l = 1; l <= L; ++l) {
            const int Kp = pad4(N.dims[l - 1]), Np = pad4(N.dims[l]), dl = N.dims[l];
            // 2 rows x 4 columns per thread: a 16-row tile of a 128-wide layer is then one item per thread
            // (2 x 8 left half the threads idle: 21% slower on both the pushing and manipulation networks)
            IbpSink o;
            const size_t base = (size_t)box0 * H + t;
            o.pre_lo = a.pre_lo + base * sumh;
            o.pre_hi = a.pre_hi + base * sumh;
            o.S = a.S + base * (sumh + s);
            o.rstride_h = (size_t)H * sumh;
            o.rstride_s = (size_t)H * (sumh + s);
            o.hoff = l < L ? N.hoff[l] : 0;
            o.soff = l < L ? N.hoff[l] : sumh;
            o.dl = dl;
            o.nrows = nlive - box0;
            o.hidden = l < L;
            // (an output layer of 8 or 16 columns: 1 x 2 tiles, twice the threads of 1 x 4 on its K-long sums)
            if (Np >= 64)
                ibp_dense<2, 4>(blo[cur], bhi[cur], ld, img + N.fwd_w[l], img + N.fwd_b[l], Kp, Np, blo[cur ^ 1],
                                bhi[cur ^ 1], o);
            else if (Np >= 32)
                ibp_dense<1, 4>(blo[cur], bhi[cur], ld, img + N.fwd_w[l], img + N.fwd_b[l], Kp, Np, blo[cur ^ 1],
                                bhi[cur ^ 1], o);
            else
                ibp_dense<1, 2>(blo[cur], bhi[cur], ld, img + N.fwd_w[l], img + N.fwd_b[l], Kp, Np, blo[cur ^ 1],
                                bhi[cur ^ 1], o);
            __syncthreads();
            cur ^= 1;
        }
        // x_{t+1} in [x_t] + [z_L]; interval bound of ||x_{t+1} - g||^2
        for (int r = warp; r < RB; r += NT / 32) {
            const int box = box0 + r;
            float v = 0.f;
            for (int i = lane; i < s; i += 32) {
                const float nl = __fadd_rd(xl[r * s4 + i], blo[cur][r * ld + i]);
                const float nh = __fadd_ru(xu[r * s4 + i], bhi[cur][r * ld + i]);
                xl[r * s4 + i] = nl;
                xu[r * s4 + i] = nh;
                if (box < nlive && a.x_lo) {
                    a.x_lo[((size_t)box * (H + 1) + t + 1) * s + i] = nl;
                    a.x_hi[((size_t)box * (H + 1) + t + 1) * s + i] = nh;
                }
                const float g = a.goal[i];
                if (a.cost.kind == 0) {
                    v = __fadd_rd(v, sq_min_rd(__fsub_rd(nl, g), __fsub_ru(nh, g)));
                } else {
                    // distance from g to the interval, rounded down, squared rounded down
                    const float e = fmaxf(fmaxf(__fsub_rd(nl, g), __fsub_rd(g, nh)), 0.f);
                    v = __fmaf_rd(e, e, v);
                }
            }
            v = warp_sum_rd(v);
            if (a.cost.kind == 1) {
                // w_t times the distance from g to the box, then the penalties at their minima (each rounded down)
                __syncwarp();
                float pen = 0.f;
                const int nq = s / 2 + 1;
                for (int q = lane; q < a.cost.n_obs * nq; q += 32) {
                    const int o = q / nq, kp = q % nq - 1;
                    pen = __fadd_rd(pen, kp < 0 ? penalty_min_rd(a.cost, o, pbx[4 * r], pbx[4 * r + 2], pbx[4 * r + 1],
                                                                 pbx[4 * r + 3])
                                                : penalty_min_rd(a.cost, o, xl[r * s4 + 2 * kp], xu[r * s4 + 2 * kp],
                                                                 xl[r * s4 + 2 * kp + 1], xu[r * s4 + 2 * kp + 1]));
                }
                pen = warp_sum_rd(pen);
                v = __fadd_rd(__fmul_rd(a.cost.w[t], __fsqrt_rd(v)), pen);
            }
            if (lane == 0) lbacc[r] = __fadd_rd(lbacc[r], v);
        }
        __syncthreads();
    }
    if (a.lb_ibp)
        for (int r = threadIdx.x; r < RB; r += NT)
            if (box0 + r < nlive) a.lb_ibp[box0 + r] = lbacc[r];
}

// ---------------------------------------------------------------------------
// CROWN and its adjoint over a tile of rows.  The per-box arrays are reached
// through a RowsView whose pointers start at the tile's first box, so the same
// code runs on the global arrays (k_crown, k_alpha_fwd) and on copies held in
// shared memory for a whole alpha optimisation (k_alpha_fused).
// ---------------------------------------------------------------------------
struct RowsView {
    const float *lo, *hi;            // [rows][d]
    const float *pre_lo, *pre_hi;    // [rows][H][sumh]
    const float *x_lo, *x_hi;        // [rows][H+1][s]
    const float *S;                  // [rows][H][sumh + s]
    float *alpha;                    // [rows][H][sumh] (nullable: adaptive slopes)
    float *A_pre;                    // [rows][H][sumh] (nullable)
    float *ustar, *lin_coef;         // [rows][d] (nullable)
    float *lb, *margin, *lin_const, *lb_best;  // [rows] (lb required, the rest nullable)
    float *grad;                     // [rows][H][sumh]: adjoint output (nullable when Adam is fused)
    float *adam_m, *adam_v;          // [rows][H][sumh]: fused Adam moments (nullable)
};

__device__ __forceinline__ RowsView global_view(const BoundArgs &a, int box0)
{
    const size_t b = (size_t)box0, hs = (size_t)a.H * a.net.sumh;
    RowsView v;
    v.lo = a.lo + b * a.d;
    v.hi = a.hi + b * a.d;
    v.pre_lo = a.pre_lo + b * hs;
    v.pre_hi = a.pre_hi + b * hs;
    v.x_lo = a.x_lo + b * (a.H + 1) * a.net.s;
    v.x_hi = a.x_hi + b * (a.H + 1) * a.net.s;
    v.S = a.S + b * a.H * (a.net.sumh + a.net.s);
    v.alpha = a.alpha ? const_cast<float *>(a.alpha) + b * hs : nullptr;
    v.A_pre = a.A_pre ? a.A_pre + b * hs : nullptr;
    v.ustar = a.ustar ? a.ustar + b * a.d : nullptr;
    v.lin_coef = a.lin_coef ? a.lin_coef + b * a.d : nullptr;
    v.lb = a.lb + b;
    v.margin = a.margin ? a.margin + b : nullptr;
    v.lin_const = a.lin_const ? a.lin_const + b : nullptr;
    v.lb_best = a.lb_best ? a.lb_best + b : nullptr;
    v.grad = a.grad_alpha ? a.grad_alpha + b * hs : nullptr;
    v.adam_m = v.adam_v = nullptr;
    return v;
}

// shared-memory floats of crown_rows / fwd_rows scratch
__host__ __device__ inline size_t crown_rows_floats(const NetDesc &N, int rb, int d)
{
    return 2 * (size_t)rb * N.maxw_p + (size_t)rb * pad4(N.s) + (size_t)rb * pad4(d) + 2 * rb + 4 * rb;
}
__host__ __device__ inline size_t fwd_rows_floats(const NetDesc &N, int rb)
{
    return 2 * (size_t)rb * N.maxw_p + (size_t)rb * pad4(N.s);
}

// Theorem 1 backward propagation of the tangent-linearised cost through all H
// steps, then Theorem 2 in box form, for rows 0 .. nrows-1 of the view (rows
// nrows .. RBT-1 are padding).  img: backward image; p: crown_rows_floats of
// shared memory.
template <int RBT, int NTT>
__device__ void crown_rows(const BoundArgs &a, const float *img, float *p, const RowsView &v, int nrows)
{
    const NetDesc &N = a.net;
    const int s = N.s, k = N.k, L = N.L, d = a.d, H = a.H, sumh = N.sumh, sw = sumh + s;
    const int ld = N.maxw_p, s4 = pad4(s), d4 = pad4(d);
    float *Ab[2];
    Ab[0] = p; p += RBT * ld;
    Ab[1] = p; p += RBT * ld;
    float *lam = p; p += RBT * s4;
    float *mu = p; p += RBT * d4;
    float *cst = p; p += RBT;
    float *mg = p; p += RBT;
    float *Pu = p; p += 4 * RBT;  // obstacle cost: per row the pusher coefficient of the actions (2) and its |sum| (2)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool obst = a.cost.kind == 1;
    const bool has_alpha = v.alpha != nullptr;
    const int ts = a.t_stop;              // early stop: propagate back to x_ts only
    const bool with_margin = v.S != nullptr;

    // early stop: the cost terms at steps 1 .. ts on their intervals, no coefficient of u before ts
    if (ts > 0) {
        for (int i = threadIdx.x; i < RBT * d4; i += NTT) mu[i] = 0.f;
        for (int r = warp; r < RBT; r += NTT / 32) {
            float c = 0.f;
            if (r < nrows)
                for (int q = lane; q < ts * s; q += 32) {
                    const int t = 1 + q / s, i = q % s;
                    const float g = a.goal[i];
                    const size_t xi = ((size_t)r * (H + 1) + t) * s + i;
                    c = __fadd_rd(c, sq_min_rd(__fsub_rd(v.x_lo[xi], g), __fsub_ru(v.x_hi[xi], g)));
                }
            c = warp_sum_rd(c);
            if (lane == 0) cst[r] = c;
        }
    }
    // tangent of ||x_H - g||^2: coefficient 2m, constant -(2 m g + m^2)
    for (int r = warp; r < RBT; r += NTT / 32) {
        if (obst) {
            // the obstacle cost at step H: its linear lower bound on x_H, and the pusher penalties at H
            float aa = 0.f, c = 0.f;
            if (r < nrows && H > ts) {
                const size_t xi = ((size_t)r * (H + 1) + H) * s;
                c = obstacle_state_lin(a.cost, H, s, v.x_lo + xi, v.x_hi + xi, a.goal, lane, aa);
            }
            if (lane < s) lam[r * s4 + lane] = aa;
            if (lane == 0) {
                Pu[4 * r] = Pu[4 * r + 1] = Pu[4 * r + 2] = Pu[4 * r + 3] = 0.f;
                if (r < nrows) c = __fadd_rd(c, pusher_lin(a.cost, H, k, v.lo + (size_t)r * d, v.hi + (size_t)r * d,
                                                           Pu + 4 * r, Pu + 4 * r + 2));
                cst[r] = c;
                mg[r] = 0.f;
            }
            continue;
        }
        float c = 0.f;
        for (int i = lane; i < s; i += 32) {
            float aa = 0.f;
            if (r < nrows && H > ts) {
                const float g = a.goal[i];
                const size_t xi = ((size_t)r * (H + 1) + H) * s + i;
                const float Ls = __fsub_rd(v.x_lo[xi], g), Us = __fsub_ru(v.x_hi[xi], g);
                const float m = 0.5f * (Ls + Us);
                aa = 2.f * m;
                c = __fadd_rd(c, __fmaf_rd(-aa, g, -__fmul_ru(m, m)));
            }
            lam[r * s4 + i] = aa;
        }
        c = warp_sum_rd(c);
        if (lane == 0) {
            cst[r] = ts > 0 ? __fadd_rd(cst[r], c) : c;
            mg[r] = 0.f;
        }
    }
    __syncthreads();

    for (int t = H - 1; t >= ts; --t) {
        // last layer: A = lam on z_L (rows of W_L), constant lam . b_L
        {
            const int NpL = pad4(N.dims[L]);
            const float *bL = img + N.bwd_b[L];
            for (int r = warp; r < RBT; r += NTT / 32) {
                float c = 0.f, e = 0.f;
                for (int q = lane; q < NpL; q += 32) {
                    const float A = q < s ? lam[r * s4 + q] : 0.f;
                    Ab[0][r * ld + q] = A;
                    if (q < s && r < nrows) {
                        c = __fmaf_rd(A, bL[q], c);
                        if (with_margin) e = __fmaf_ru(fabsf(A), v.S[((size_t)r * H + t) * sw + sumh + q], e);
                    }
                }
                c = warp_sum_rd(c);
                e = warp_sum_ru(e);
                if (lane == 0) {
                    cst[r] = __fadd_rd(cst[r], c);
                    mg[r] = __fmaf_ru(N.gam[L], e, mg[r]);
                }
            }
            __syncthreads();
            dense_rows_auto<RBT, NTT>(Ab[0], ld, img + N.bwd_w[L], nullptr, NpL, pad4(N.dims[L - 1]), Ab[1], ld, false);
            __syncthreads();
        }
        int cur = 1;
        for (int l = L - 1; l >= 1; --l) {
            const int dl = N.dims[l], Npl = pad4(dl);
            const float *bl = img + N.bwd_b[l];
            for (int r = warp; r < RBT; r += NTT / 32) {
                float c = 0.f, eg = 0.f, er = 0.f;
                if (r < nrows) {
                    const size_t base = ((size_t)r * H + t);
                    for (int q = lane; q < dl; q += 32) {
                        const size_t idx = base * sumh + N.hoff[l] + q;
                        const float zl = v.pre_lo[idx], zu = v.pre_hi[idx];
                        const float A = Ab[cur][r * ld + q];
                        if (v.A_pre) v.A_pre[idx] = A;
                        float D, ci;
                        relax_select(zl, zu, A, has_alpha ? v.alpha[idx] : 0.f, has_alpha, D, ci);
                        const float Ap = A * D;
                        Ab[cur][r * ld + q] = Ap;
                        c = __fmaf_rd(A, ci, c);
                        c = __fmaf_rd(Ap, bl[q], c);
                        if (with_margin) {
                            eg = __fmaf_ru(fabsf(Ap), v.S[base * sw + N.hoff[l] + q], eg);
                            if (D != 0.f && D != 1.f) er = __fmaf_ru(fabsf(Ap), fmaxf(-zl, zu), er);
                        }
                    }
                } else {
                    for (int q = lane; q < dl; q += 32) Ab[cur][r * ld + q] = 0.f;
                }
                c = warp_sum_rd(c);
                eg = warp_sum_ru(eg);
                er = warp_sum_ru(er);
                if (lane == 0) {
                    cst[r] = __fadd_rd(cst[r], c);
                    mg[r] = __fadd_ru(mg[r], __fmaf_ru(N.gam[l], eg, __fmul_ru(kTwoU, er)));
                }
            }
            __syncthreads();
            dense_rows_auto<RBT, NTT>(Ab[cur], ld, img + N.bwd_w[l], nullptr, Npl, pad4(N.dims[l - 1]), Ab[cur ^ 1],
                                      ld, false);
            __syncthreads();
            cur ^= 1;
        }
        // A is on [x_t | u_t]: mu_t = A_u; lam <- lam + A_x (+ tangent of ||x_t - g||^2 for t >= 1)
        for (int r = warp; r < RBT; r += NTT / 32) {
            float c = 0.f, e = 0.f;
            if (obst) {
                // mu_t = A_u + the pusher coefficient of the later steps; its rounding (H additions) in the margin
                const float *lo_r = v.lo + (size_t)r * d, *hi_r = v.hi + (size_t)r * d;
                for (int j = lane; j < k; j += 32) {
                    const float Au = Ab[cur][r * ld + s + j];
                    const float Pj = j < 2 ? Pu[4 * r + j] : 0.f, Pa = j < 2 ? Pu[4 * r + 2 + j] : 0.f;
                    mu[r * d4 + t * k + j] = Au + Pj;
                    if (with_margin && r < nrows) {
                        const float um = fmaxf(fabsf(lo_r[t * k + j]), fabsf(hi_r[t * k + j]));
                        e = __fmaf_ru(__fmul_ru(__fmul_ru((float)(H + 2), kTwoU), __fadd_ru(fabsf(Au), Pa)), um, e);
                    }
                }
                float aa = 0.f;
                if (t > ts && t >= 1 && r < nrows) {
                    const size_t xi = ((size_t)r * (H + 1) + t) * s;
                    c = obstacle_state_lin(a.cost, t, s, v.x_lo + xi, v.x_hi + xi, a.goal, lane, aa);
                }
                if (lane < s) {
                    const float Ax = Ab[cur][r * ld + lane];
                    const float lo_ = lam[r * s4 + lane];
                    const size_t xi = ((size_t)r * (H + 1) + t) * s + lane;
                    const float B = (t >= 1 && r < nrows) ? fmaxf(fabsf(v.x_lo[xi]), fabsf(v.x_hi[xi])) : fabsf(a.x0[lane]);
                    lam[r * s4 + lane] = (lo_ + Ax) + aa;
                    const float mag = __fadd_ru(__fadd_ru(fabsf(lo_), fabsf(Ax)), fabsf(aa));
                    if (with_margin) e = __fmaf_ru(__fmul_ru(kTwoU, mag), B, e);
                }
                e = warp_sum_ru(e);
                if (lane == 0) {
                    if (t >= 1 && r < nrows)
                        c = __fadd_rd(c, pusher_lin(a.cost, t, k, lo_r, hi_r, Pu + 4 * r, Pu + 4 * r + 2));
                    cst[r] = __fadd_rd(cst[r], c);
                    mg[r] = __fadd_ru(mg[r], e);
                }
                continue;
            }
            for (int j = lane; j < k; j += 32) mu[r * d4 + t * k + j] = Ab[cur][r * ld + s + j];
            for (int i = lane; i < s; i += 32) {
                const float Ax = Ab[cur][r * ld + i];
                const float lo_ = lam[r * s4 + i];
                float aa = 0.f, B = fabsf(a.x0[i]);
                if (t >= 1 && r < nrows) {
                    // the updated coefficient multiplies x_t (concretized on its interval at an early stop)
                    const size_t xi = ((size_t)r * (H + 1) + t) * s + i;
                    const float xl = v.x_lo[xi], xu = v.x_hi[xi];
                    B = fmaxf(fabsf(xl), fabsf(xu));
                    if (t > ts) {
                        const float g = a.goal[i];
                        const float Ls = __fsub_rd(xl, g), Us = __fsub_ru(xu, g);
                        const float m = 0.5f * (Ls + Us);
                        aa = 2.f * m;
                        c = __fadd_rd(c, __fmaf_rd(-aa, g, -__fmul_ru(m, m)));
                    }
                }
                const float ln = (lo_ + Ax) + aa;
                lam[r * s4 + i] = ln;
                const float mag = __fadd_ru(__fadd_ru(fabsf(lo_), fabsf(Ax)), fabsf(aa));
                if (with_margin) e = __fmaf_ru(__fmul_ru(kTwoU, mag), B, e);
            }
            c = warp_sum_rd(c);
            e = warp_sum_ru(e);
            if (lane == 0) {
                cst[r] = __fadd_rd(cst[r], c);
                mg[r] = __fadd_ru(mg[r], e);
            }
        }
        __syncthreads();
    }

    // lam . x0, then Theorem 2 in box form: sum_j min_{u in [lo, hi]} mu_j u + rho u^2
    for (int r = warp; r < nrows; r += NTT / 32) {
        float c = 0.f, val = 0.f, e = 0.f;
        if (ts == 0) {
            for (int i = lane; i < s; i += 32) c = __fmaf_rd(lam[r * s4 + i], a.x0[i], c);
        } else {
            // early stop: the coefficient of x_ts on that state's interval (Theorem 2, box form)
            for (int i = lane; i < s; i += 32) {
                const size_t xi = ((size_t)r * (H + 1) + ts) * s + i;
                const float li = lam[r * s4 + i];
                c = __fadd_rd(c, fminf(__fmul_rd(li, v.x_lo[xi]), __fmul_rd(li, v.x_hi[xi])));
            }
        }
        c = __fadd_rd(cst[r], warp_sum_rd(c));
        for (int j = lane; j < d; j += 32) {
            const float m_ = mu[r * d4 + j];
            const float lo = v.lo[(size_t)r * d + j], hi = v.hi[(size_t)r * d + j];
            float us, vj;
            if (a.rho > 0.f) {
                const float uc = -m_ / (2.f * a.rho);
                if (uc >= lo && uc <= hi) {
                    us = uc;
                    vj = __fdiv_rd(-__fmul_ru(m_, m_), 4.f * a.rho);
                } else {
                    us = uc < lo ? lo : hi;
                    vj = __fmaf_rd(m_, us, __fmul_rd(a.rho, __fmul_rd(us, us)));
                    // the face choice can be off only when uc is within rounding of the face:
                    // the minimum then lies below q(us) by at most rho (2u uc)^2
                    const float du = __fmul_ru(kTwoU, fabsf(uc));
                    e = __fmaf_ru(__fmul_ru(a.rho, du), du, e);
                }
            } else {
                us = m_ >= 0.f ? lo : hi;
                vj = __fmul_rd(m_, us);
            }
            val = __fadd_rd(val, vj);
            if (v.ustar) v.ustar[(size_t)r * d + j] = us;
            if (v.lin_coef) v.lin_coef[(size_t)r * d + j] = m_;
        }
        val = warp_sum_rd(val);
        e = warp_sum_ru(e);
        if (lane == 0) {
            const float raw = __fadd_rd(c, val);
            const float marg = __fadd_ru(mg[r], e);
            const float lbv = __fsub_rd(raw, marg);
            v.lb[r] = lbv;
            if (v.margin) v.margin[r] = marg;
            if (v.lin_const) v.lin_const[r] = c;
            if (v.lb_best) v.lb_best[r] = fmaxf(v.lb_best[r], lbv);
        }
    }
}

// alpha gradient: forward pass of the relaxed network from x_0 and u*;
// dLB/dalpha_j = A_j z~_j for an unstable neuron whose coefficient A_j >= 0
// selects the lower line, 0 otherwise.  With `adam` the projected Adam step is
// applied to each slope as soon as its gradient is known (its own slope is
// not needed again in this pass); otherwise the gradient goes to v.grad.
template <int RBT, int NTT>
__device__ void fwd_rows(const BoundArgs &a, const float *img, float *p, const RowsView &v, int nrows,
                         const AdamStep *adam)
{
    const NetDesc &N = a.net;
    const int s = N.s, k = N.k, L = N.L, d = a.d, H = a.H, sumh = N.sumh;
    const int ld = N.maxw_p, s4 = pad4(s);
    float *Z[2];
    Z[0] = p; p += RBT * ld;
    Z[1] = p; p += RBT * ld;
    float *xs = p; p += RBT * s4;
    const bool has_alpha = v.alpha != nullptr;
    const int Kp1 = pad4(s + k);
    for (int i = threadIdx.x; i < RBT * s; i += NTT) xs[(i / s) * s4 + i % s] = a.x0[i % s];
    __syncthreads();
    for (int t = 0; t < H; ++t) {
        for (int i = threadIdx.x; i < RBT * Kp1; i += NTT) {
            const int r = i / Kp1, c = i % Kp1;
            float val = 0.f;
            if (c < s) val = xs[r * s4 + c];
            else if (c < s + k && r < nrows) val = v.ustar[(size_t)r * d + t * k + (c - s)];
            Z[0][r * ld + c] = val;
        }
        __syncthreads();
        int cur = 0;
        for (int l = 1; l <= L; ++l) {
            dense_rows_auto<RBT, NTT>(Z[cur], ld, img + N.fwd_w[l], img + N.fwd_b[l], pad4(N.dims[l - 1]),
                                      pad4(N.dims[l]), Z[cur ^ 1], ld, false);
            __syncthreads();
            cur ^= 1;
            if (l < L) {
                const int dl = N.dims[l];
                for (int i = threadIdx.x; i < RBT * dl; i += NTT) {
                    const int r = i / dl, q = i % dl;
                    if (r >= nrows) continue;
                    const size_t idx = ((size_t)r * H + t) * sumh + N.hoff[l] + q;
                    const float z = Z[cur][r * ld + q];
                    const float zl = v.pre_lo[idx], zu = v.pre_hi[idx], A = v.A_pre[idx];
                    float D, c;
                    relax_select(zl, zu, A, has_alpha ? v.alpha[idx] : 0.f, has_alpha, D, c);
                    const bool unstable = zl < 0.f && zu > 0.f;
                    const float g = (unstable && A >= 0.f) ? A * z : 0.f;
                    if (adam) adam_update(v.alpha[idx], v.adam_m[idx], v.adam_v[idx], g, *adam);
                    else v.grad[idx] = g;
                    Z[cur][r * ld + q] = fmaf(D, z, c);
                }
                __syncthreads();
            }
        }
        for (int i = threadIdx.x; i < RBT * s; i += NTT) {
            const int r = i / s, c = i % s;
            xs[r * s4 + c] += Z[cur][r * ld + c];
        }
        __syncthreads();
    }
}

template <bool WSMEM>
__global__ void __launch_bounds__(NT) k_crown(BoundArgs a)
{
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    const NetDesc &N = a.net;
    const float *img = a.bwd;
    float *p = sm;
    if (WSMEM) {
        for (int i = threadIdx.x; i < N.img_floats / 4; i += NT) smem4[i] = reinterpret_cast<const float4 *>(a.bwd)[i];
        img = sm;
        p += N.img_floats;
    }
    const int nlive = live_count(a.n, a.d_n, a.row0);
    const int box0 = blockIdx.x * RB;
    if (box0 >= nlive) return;
    const int nrows = min(RB, nlive - box0);
    crown_rows<RB, NT>(a, img, p, global_view(a, box0), nrows);
}

template <bool WSMEM>
__global__ void __launch_bounds__(NT) k_alpha_fwd(BoundArgs a)
{
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    const NetDesc &N = a.net;
    const float *img = a.fwd;
    float *p = sm;
    if (WSMEM) {
        for (int i = threadIdx.x; i < N.img_floats / 4; i += NT) smem4[i] = reinterpret_cast<const float4 *>(a.fwd)[i];
        img = sm;
        p += N.img_floats;
    }
    const int nlive = live_count(a.n, a.d_n, a.row0);
    const int box0 = blockIdx.x * RB;
    if (box0 >= nlive) return;
    const int nrows = min(RB, nlive - box0);
    fwd_rows<RB, NT>(a, img, p, global_view(a, box0), nrows, nullptr);
}

// ---------------------------------------------------------------------------
// Fused alpha-CROWN: the whole optimisation of a tile of RBT boxes in one CTA.
// Both network images and every per-box array (interval bounds, margin
// helpers, slopes, Adam moments, coefficients before relaxation, u*) stay in
// shared memory for all `steps` (bound, adjoint + Adam) rounds; only the best
// bound (and the final slopes, when asked for) go back to global memory.  The
// arithmetic is that of k_crown, k_alpha_fwd and k_adam, step for step.
// ---------------------------------------------------------------------------
__host__ __device__ inline size_t fused_box_floats(const NetDesc &N, int H, int d)
{
    const size_t hs = (size_t)H * N.sumh;
    return 6 * hs + (size_t)H * (N.sumh + N.s) + 2 * (size_t)(H + 1) * N.s + 3 * (size_t)d + 2;
}

template <int RBT, int NTT>
__global__ void __launch_bounds__(NTT) k_alpha_fused(BoundArgs a, int steps, float lr, float *alpha_out,
                                                     const AdamTable tab)
{
    __shared__ float bc_sh[2];
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    const NetDesc &N = a.net;
    const int H = a.H, d = a.d, s = N.s;
    const size_t hs = (size_t)H * N.sumh, hw = (size_t)H * (N.sumh + s), xs_ = (size_t)(H + 1) * s;
    const int nlive = live_count(a.n, a.d_n, a.row0);
    const int box0 = blockIdx.x * RBT;
    if (box0 >= nlive) return;
    const int nrows = min(RBT, nlive - box0);

    float *p = sm;
    const float *fwd = p;
    for (int i = threadIdx.x; i < N.img_floats / 4; i += NTT) smem4[i] = reinterpret_cast<const float4 *>(a.fwd)[i];
    p += N.img_floats;
    const float *bwd = p;
    for (int i = threadIdx.x; i < N.img_floats / 4; i += NTT)
        reinterpret_cast<float4 *>(p)[i] = reinterpret_cast<const float4 *>(a.bwd)[i];
    p += N.img_floats;
    RowsView v;
    float *pl = p; p += RBT * hs;
    float *ph = p; p += RBT * hs;
    v.alpha = p; p += RBT * hs;
    v.adam_m = p; p += RBT * hs;
    v.adam_v = p; p += RBT * hs;
    v.A_pre = p; p += RBT * hs;
    float *Sv = p; p += RBT * hw;
    float *xl = p; p += RBT * xs_;
    float *xu = p; p += RBT * xs_;
    float *blo = p; p += (size_t)RBT * d;
    float *bhi = p; p += (size_t)RBT * d;
    v.ustar = p; p += (size_t)RBT * d;
    v.lb = p; p += RBT;
    v.lb_best = p; p += RBT;
    float *scratch = sm + ((p - sm + 3) & ~(ptrdiff_t)3);  // float4-aligned for dense_rows
    v.pre_lo = pl;
    v.pre_hi = ph;
    v.S = Sv;
    v.x_lo = xl;
    v.x_hi = xu;
    v.lo = blo;
    v.hi = bhi;
    v.lin_coef = nullptr;
    v.margin = v.lin_const = nullptr;
    v.grad = nullptr;

    const size_t b = (size_t)box0;
    for (size_t i = threadIdx.x; i < (size_t)nrows * hs; i += NTT) {
        const float zl = a.pre_lo[b * hs + i], zu = a.pre_hi[b * hs + i];
        pl[i] = zl;
        ph[i] = zu;
        v.alpha[i] = (zu >= -zl) ? 1.f : 0.f;  // adaptive initial slopes
        v.adam_m[i] = 0.f;
        v.adam_v[i] = 0.f;
    }
    for (size_t i = threadIdx.x; i < (size_t)nrows * hw; i += NTT) Sv[i] = a.S[b * hw + i];
    for (size_t i = threadIdx.x; i < (size_t)nrows * xs_; i += NTT) {
        xl[i] = a.x_lo[b * xs_ + i];
        xu[i] = a.x_hi[b * xs_ + i];
    }
    for (size_t i = threadIdx.x; i < (size_t)nrows * d; i += NTT) {
        blo[i] = a.lo[b * d + i];
        bhi[i] = a.hi[b * d + i];
    }
    for (int r = threadIdx.x; r < RBT; r += NTT) v.lb_best[r] = -INFINITY;
    __syncthreads();

    for (int step = 1; step <= steps; ++step) {
        crown_rows<RBT, NTT>(a, bwd, scratch, v, nrows);
        __syncthreads();
        AdamStep st;
        st.lr = lr;
        if (step <= kAdamTable) {
            st.bc1 = tab.bc1[step - 1];
            st.bc2 = tab.bc2[step - 1];
        } else {
            // beyond the table: one thread forms the constants (FP64 is slow on this part)
            if (threadIdx.x == 0) {
                bc_sh[0] = (float)(1.0 - pow(0.9, (double)step));
                bc_sh[1] = (float)(1.0 - pow(0.999, (double)step));
            }
            __syncthreads();
            st.bc1 = bc_sh[0];
            st.bc2 = bc_sh[1];
        }
        fwd_rows<RBT, NTT>(a, fwd, scratch, v, nrows, &st);
        __syncthreads();
    }
    for (int r = threadIdx.x; r < nrows; r += NTT) a.lb_best[box0 + r] = v.lb_best[r];
    if (alpha_out)
        for (size_t i = threadIdx.x; i < (size_t)nrows * hs; i += NTT) alpha_out[b * hs + i] = v.alpha[i];
}

__global__ void k_alpha_init(BoundArgs a)
{
    const int nlive = live_count(a.n, a.d_n, a.row0);
    const long long total = (long long)nlive * a.H * a.net.sumh;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
        const_cast<float *>(a.alpha)[i] = (a.pre_hi[i] >= -a.pre_lo[i]) ? 1.f : 0.f;
}

__global__ void k_adam(float *alpha, float *m, float *v, const float *g, long long count, float lr, float bc1, float bc2)
{
    AdamStep st;
    st.lr = lr;
    st.bc1 = bc1;
    st.bc2 = bc2;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
        float al = alpha[i], mi = m[i], vi = v[i];
        adam_update(al, mi, vi, g[i], st);
        alpha[i] = al;
        m[i] = mi;
        v[i] = vi;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int max_optin_smem()
{
    int dev, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v - 1024;
}

template <typename K>
static cudaError_t launch_rows_kernel(K kern_smem, K kern_glob, size_t img_bytes, size_t rest_bytes, int n,
                                      const BoundArgs &a, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int budget = max_optin_smem();
    const bool wsmem = img_bytes + rest_bytes <= (size_t)budget;
    const size_t smem = (wsmem ? img_bytes : 0) + rest_bytes;
    if (smem > (size_t)budget) return cudaErrorInvalidConfiguration;
    K kern = wsmem ? kern_smem : kern_glob;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<(n + RB - 1) / RB, NT, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_ibp(const BoundArgs &a, int, cudaStream_t st)
{
    const NetDesc &N = a.net;
    size_t rest = (4 * (size_t)RB * N.maxw_p + 2 * (size_t)RB * pad4(N.s) + 5 * (size_t)RB) * sizeof(float);
    return launch_rows_kernel(k_ibp<true>, k_ibp<false>, (size_t)N.img_floats * 4, rest, a.n, a, st);
}

cudaError_t launch_crown(const BoundArgs &a, int, cudaStream_t st)
{
    const NetDesc &N = a.net;
    size_t rest = crown_rows_floats(N, RB, a.d) * sizeof(float);
    return launch_rows_kernel(k_crown<true>, k_crown<false>, (size_t)N.img_floats * 4, rest, a.n, a, st);
}

cudaError_t preload_ibp_crown()
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_ibp<true>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_ibp<false>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_crown<true>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_crown<false>);
    return e;
}

cudaError_t launch_alpha_fwd(const BoundArgs &a, int, cudaStream_t st)
{
    const NetDesc &N = a.net;
    size_t rest = fwd_rows_floats(N, RB) * sizeof(float);
    return launch_rows_kernel(k_alpha_fwd<true>, k_alpha_fwd<false>, (size_t)N.img_floats * 4, rest, a.n, a, st);
}

static size_t fused_smem(const NetDesc &N, int rb, int H, int d)
{
    const size_t rows = crown_rows_floats(N, rb, d), fw = fwd_rows_floats(N, rb);
    return (2 * (size_t)N.img_floats + (size_t)rb * fused_box_floats(N, H, d) + 4 + (rows > fw ? rows : fw)) *
           sizeof(float);
}

template <int RBT, int NTT>
static cudaError_t launch_fused_variant(const BoundArgs &a, int steps, float lr, float *alpha_out, cudaStream_t st)
{
    const size_t smem = fused_smem(a.net, RBT, a.H, a.d);
    if (smem > (size_t)max_optin_smem()) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(k_alpha_fused<RBT, NTT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    AdamTable tab;
    fill_adam_table(tab);
    k_alpha_fused<RBT, NTT><<<(a.n + RBT - 1) / RBT, NTT, smem, st>>>(a, steps, lr, alpha_out, tab);
    return cudaGetLastError();
}

int alpha_fused_variants() { return 3; }

bool alpha_fused_fits(const NetDesc &N, int H, int d)
{
    return fused_smem(N, 2, H, d) <= (size_t)max_optin_smem();
}

// variant 0: 2 boxes x 64 threads per CTA; 1: 4 x 128; 2: 8 x 256; < 0: the most boxes that fit in shared memory,
// at most 4.  Returns cudaErrorInvalidConfiguration when the tile does not fit.
cudaError_t launch_alpha_fused(const BoundArgs &a, int steps, float lr, float *alpha_out, int variant, cudaStream_t st)
{
    if (a.n <= 0) return cudaSuccess;
    if (variant < 0) variant = fused_smem(a.net, 4, a.H, a.d) <= (size_t)max_optin_smem() ? 1 : 0;
    switch (variant) {
        case 0: return launch_fused_variant<2, 64>(a, steps, lr, alpha_out, st);
        case 1: return launch_fused_variant<4, 128>(a, steps, lr, alpha_out, st);
        default: return launch_fused_variant<8, 256>(a, steps, lr, alpha_out, st);
    }
}

__global__ void k_fill_f32(float *p, int n, float v)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}

cudaError_t launch_fill(float *p, int n, float v, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_fill_f32<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, st>>>(p, n, v);
    return cudaGetLastError();
}

cudaError_t launch_alpha_init(const BoundArgs &a, cudaStream_t st)
{
    if (a.n <= 0) return cudaSuccess;
    k_alpha_init<<<1024, 256, 0, st>>>(a);
    return cudaGetLastError();
}

void fill_adam_table(AdamTable &tab)
{
    for (int i = 0; i < kAdamTable; ++i) {
        tab.bc1[i] = (float)(1.0 - std::pow(0.9, i + 1));
        tab.bc2[i] = (float)(1.0 - std::pow(0.999, i + 1));
    }
}

cudaError_t launch_adam(float *alpha, float *m, float *v, const float *grad, long long count, float lr, float bc1,
                        float bc2, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    long long blocks = (count + 255) / 256;
    k_adam<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(alpha, m, v, grad, count, lr, bc1, bc2);
    return cudaGetLastError();
}

}  // namespace bab
