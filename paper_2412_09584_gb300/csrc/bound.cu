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
#include "bab_internal.cuh"
#include "kernels.cuh"

namespace bab {

constexpr int RB = 16;
constexpr int NT = 256;
constexpr float kTwoU = 1.1920930376163597e-07f;  // 2^-23 (1 + 2^-20): twice the unit roundoff, rounded up

// ---------------------------------------------------------------------------
// IBP
// ---------------------------------------------------------------------------
template <int TR, int TN>
__device__ __forceinline__ void ibp_dense(const float *__restrict__ alo, const float *__restrict__ ahi, int ld,
                                          const float *__restrict__ Wt, const float *__restrict__ bias, int Kp, int Np,
                                          float *__restrict__ zlo, float *__restrict__ zhi, float *__restrict__ Sout)
{
    const int ngc = (Np + TN - 1) / TN;
    const int items = (RB / TR) * ngc;
    for (int it = threadIdx.x; it < items; it += NT) {
        const int cg = it % ngc, rg = it / ngc;
        const int c0 = cg * TN, r0 = rg * TR;
        float accl[TR][TN], acch[TR][TN], accs[TR][TN];
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const float bj = (c0 + j < Np) ? bias[c0 + j] : 0.f;
#pragma unroll
            for (int i = 0; i < TR; ++i) {
                accl[i][j] = bj;
                acch[i][j] = bj;
                accs[i][j] = 0.f;
            }
        }
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
#pragma unroll
                for (int j = 0; j < TN; ++j) w[j] = (c0 + j < Np) ? Wt[(size_t)(k + kk) * Np + c0 + j] : 0.f;
#pragma unroll
                for (int i = 0; i < TR; ++i) {
                    const float al = kk == 0 ? l4[i].x : kk == 1 ? l4[i].y : kk == 2 ? l4[i].z : l4[i].w;
                    const float ah = kk == 0 ? h4[i].x : kk == 1 ? h4[i].y : kk == 2 ? h4[i].z : h4[i].w;
                    const float am = fmaxf(fabsf(al), fabsf(ah));
#pragma unroll
                    for (int j = 0; j < TN; ++j) {
                        const bool pos = w[j] >= 0.f;
                        accl[i][j] = __fmaf_rd(w[j], pos ? al : ah, accl[i][j]);
                        acch[i][j] = __fmaf_ru(w[j], pos ? ah : al, acch[i][j]);
                        accs[i][j] = __fmaf_ru(fabsf(w[j]), am, accs[i][j]);
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < TR; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j)
                if (c0 + j < Np) {
                    zlo[(r0 + i) * ld + c0 + j] = accl[i][j];
                    zhi[(r0 + i) * ld + c0 + j] = acch[i][j];
                    Sout[(r0 + i) * ld + c0 + j] = accs[i][j];
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
    float *Sb = p; p += RB * ld;
    float *xl = p; p += RB * s4;
    float *xu = p; p += RB * s4;
    float *lbacc = p; p += RB;

    const int nlive = live_count(a.n, a.d_n);
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
    for (int r = threadIdx.x; r < RB; r += NT) lbacc[r] = 0.f;
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
            if (Np >= 64)
                ibp_dense<2, 8>(blo[cur], bhi[cur], ld, img + N.fwd_w[l], img + N.fwd_b[l], Kp, Np, blo[cur ^ 1],
                                bhi[cur ^ 1], Sb);
            else
                ibp_dense<1, 4>(blo[cur], bhi[cur], ld, img + N.fwd_w[l], img + N.fwd_b[l], Kp, Np, blo[cur ^ 1],
                                bhi[cur ^ 1], Sb);
            __syncthreads();
            cur ^= 1;
            const int soff = (l < L) ? N.hoff[l] : sumh;
            for (int i = threadIdx.x; i < RB * dl; i += NT) {
                const int r = i / dl, c = i % dl;
                const int box = box0 + r;
                const float zl = blo[cur][r * ld + c], zh = bhi[cur][r * ld + c];
                if (box < nlive) {
                    const size_t base = ((size_t)box * H + t);
                    a.S[base * (sumh + s) + soff + c] = Sb[r * ld + c];
                    if (l < L) {
                        a.pre_lo[base * sumh + N.hoff[l] + c] = zl;
                        a.pre_hi[base * sumh + N.hoff[l] + c] = zh;
                    }
                }
                if (l < L) {
                    blo[cur][r * ld + c] = fmaxf(zl, 0.f);
                    bhi[cur][r * ld + c] = fmaxf(zh, 0.f);
                }
            }
            __syncthreads();
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
                v = __fadd_rd(v, sq_min_rd(__fsub_rd(nl, g), __fsub_ru(nh, g)));
            }
            v = warp_sum_rd(v);
            if (lane == 0) lbacc[r] = __fadd_rd(lbacc[r], v);
        }
        __syncthreads();
    }
    if (a.lb_ibp)
        for (int r = threadIdx.x; r < RB; r += NT)
            if (box0 + r < nlive) a.lb_ibp[box0 + r] = lbacc[r];
}

template <bool WSMEM>
__global__ void __launch_bounds__(NT) k_crown(BoundArgs a)
{
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    const NetDesc &N = a.net;
    const int s = N.s, k = N.k, L = N.L, d = a.d, H = a.H, sumh = N.sumh, sw = sumh + s;
    const int ld = N.maxw_p, s4 = pad4(s), d4 = pad4(d);
    const float *img = a.bwd;
    float *p = sm;
    if (WSMEM) {
        for (int i = threadIdx.x; i < N.img_floats / 4; i += NT) smem4[i] = reinterpret_cast<const float4 *>(a.bwd)[i];
        img = sm;
        p += N.img_floats;
    }
    float *Ab[2];
    Ab[0] = p; p += RB * ld;
    Ab[1] = p; p += RB * ld;
    float *lam = p; p += RB * s4;
    float *mu = p; p += RB * d4;
    float *cst = p; p += RB;
    float *mg = p; p += RB;

    const int nlive = live_count(a.n, a.d_n);
    const int box0 = blockIdx.x * RB;
    if (box0 >= nlive) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool has_alpha = a.alpha != nullptr;

    // tangent of ||x_H - g||^2: coefficient 2m, constant -(2 m g + m^2)
    for (int r = warp; r < RB; r += NT / 32) {
        const int box = box0 + r;
        float c = 0.f;
        for (int i = lane; i < s; i += 32) {
            float aa = 0.f;
            if (box < nlive) {
                const float g = a.goal[i];
                const size_t xi = ((size_t)box * (H + 1) + H) * s + i;
                const float Ls = __fsub_rd(a.x_lo[xi], g), Us = __fsub_ru(a.x_hi[xi], g);
                const float m = 0.5f * (Ls + Us);
                aa = 2.f * m;
                c = __fadd_rd(c, __fmaf_rd(-aa, g, -__fmul_ru(m, m)));
            }
            lam[r * s4 + i] = aa;
        }
        c = warp_sum_rd(c);
        if (lane == 0) {
            cst[r] = c;
            mg[r] = 0.f;
        }
    }
    __syncthreads();

    for (int t = H - 1; t >= 0; --t) {
        // last layer: A = lam on z_L (rows of W_L), constant lam . b_L
        {
            const int NpL = pad4(N.dims[L]);
            const float *bL = img + N.bwd_b[L];
            for (int r = warp; r < RB; r += NT / 32) {
                const int box = box0 + r;
                float c = 0.f, e = 0.f;
                for (int q = lane; q < NpL; q += 32) {
                    const float A = q < s ? lam[r * s4 + q] : 0.f;
                    Ab[0][r * ld + q] = A;
                    if (q < s && box < nlive) {
                        c = __fmaf_rd(A, bL[q], c);
                        e = __fmaf_ru(fabsf(A), a.S[((size_t)box * H + t) * sw + sumh + q], e);
                    }
                }
                c = warp_sum_rd(c);
                e = warp_sum_ru(e);
                if (lane == 0) {
                    cst[r] = __fadd_rd(cst[r], c);
                    mg[r] = __fmaf_ru(gamma_fp32(NpL), e, mg[r]);
                }
            }
            __syncthreads();
            dense_rows_auto<RB, NT>(Ab[0], ld, img + N.bwd_w[L], nullptr, NpL, pad4(N.dims[L - 1]), Ab[1], ld, false);
            __syncthreads();
        }
        int cur = 1;
        for (int l = L - 1; l >= 1; --l) {
            const int dl = N.dims[l], Npl = pad4(dl);
            const float *bl = img + N.bwd_b[l];
            for (int r = warp; r < RB; r += NT / 32) {
                const int box = box0 + r;
                float c = 0.f, eg = 0.f, er = 0.f;
                if (box < nlive) {
                    const size_t base = ((size_t)box * H + t);
                    for (int q = lane; q < dl; q += 32) {
                        const size_t idx = base * sumh + N.hoff[l] + q;
                        const float zl = a.pre_lo[idx], zu = a.pre_hi[idx];
                        const float A = Ab[cur][r * ld + q];
                        if (a.A_pre) a.A_pre[idx] = A;
                        float D, ci;
                        relax_select(zl, zu, A, has_alpha ? a.alpha[idx] : 0.f, has_alpha, D, ci);
                        const float Ap = A * D;
                        Ab[cur][r * ld + q] = Ap;
                        c = __fmaf_rd(A, ci, c);
                        c = __fmaf_rd(Ap, bl[q], c);
                        eg = __fmaf_ru(fabsf(Ap), a.S[base * sw + N.hoff[l] + q], eg);
                        if (D != 0.f && D != 1.f) er = __fmaf_ru(fabsf(Ap), fmaxf(-zl, zu), er);
                    }
                } else {
                    for (int q = lane; q < dl; q += 32) Ab[cur][r * ld + q] = 0.f;
                }
                c = warp_sum_rd(c);
                eg = warp_sum_ru(eg);
                er = warp_sum_ru(er);
                if (lane == 0) {
                    cst[r] = __fadd_rd(cst[r], c);
                    mg[r] = __fadd_ru(mg[r], __fmaf_ru(gamma_fp32(Npl), eg, __fmul_ru(kTwoU, er)));
                }
            }
            __syncthreads();
            dense_rows_auto<RB, NT>(Ab[cur], ld, img + N.bwd_w[l], nullptr, Npl, pad4(N.dims[l - 1]), Ab[cur ^ 1], ld,
                                    false);
            __syncthreads();
            cur ^= 1;
        }
        // A is on [x_t | u_t]: mu_t = A_u; lam <- lam + A_x (+ tangent of ||x_t - g||^2 for t >= 1)
        for (int r = warp; r < RB; r += NT / 32) {
            const int box = box0 + r;
            float c = 0.f, e = 0.f;
            for (int j = lane; j < k; j += 32) mu[r * d4 + t * k + j] = Ab[cur][r * ld + s + j];
            for (int i = lane; i < s; i += 32) {
                const float Ax = Ab[cur][r * ld + i];
                const float lo_ = lam[r * s4 + i];
                float aa = 0.f, B;
                if (t >= 1 && box < nlive) {
                    const float g = a.goal[i];
                    const size_t xi = ((size_t)box * (H + 1) + t) * s + i;
                    const float xl = a.x_lo[xi], xu = a.x_hi[xi];
                    const float Ls = __fsub_rd(xl, g), Us = __fsub_ru(xu, g);
                    const float m = 0.5f * (Ls + Us);
                    aa = 2.f * m;
                    c = __fadd_rd(c, __fmaf_rd(-aa, g, -__fmul_ru(m, m)));
                    B = fmaxf(fabsf(xl), fabsf(xu));
                } else {
                    B = fabsf(a.x0[i]);
                }
                const float ln = (lo_ + Ax) + aa;
                lam[r * s4 + i] = ln;
                const float mag = __fadd_ru(__fadd_ru(fabsf(lo_), fabsf(Ax)), fabsf(aa));
                e = __fmaf_ru(__fmul_ru(kTwoU, mag), B, e);
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
    for (int r = warp; r < RB; r += NT / 32) {
        const int box = box0 + r;
        if (box >= nlive) continue;
        float c = 0.f, v = 0.f, e = 0.f;
        for (int i = lane; i < s; i += 32) c = __fmaf_rd(lam[r * s4 + i], a.x0[i], c);
        c = __fadd_rd(cst[r], warp_sum_rd(c));
        for (int j = lane; j < d; j += 32) {
            const float m_ = mu[r * d4 + j];
            const float lo = a.lo[(size_t)box * d + j], hi = a.hi[(size_t)box * d + j];
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
            v = __fadd_rd(v, vj);
            if (a.ustar) a.ustar[(size_t)box * d + j] = us;
            if (a.lin_coef) a.lin_coef[(size_t)box * d + j] = m_;
        }
        v = warp_sum_rd(v);
        e = warp_sum_ru(e);
        if (lane == 0) {
            const float raw = __fadd_rd(c, v);
            const float marg = __fadd_ru(mg[r], e);
            const float lbv = __fsub_rd(raw, marg);
            a.lb[box] = lbv;
            if (a.margin) a.margin[box] = marg;
            if (a.lin_const) a.lin_const[box] = c;
            if (a.lb_best) a.lb_best[box] = fmaxf(a.lb_best[box], lbv);
        }
    }
}

// ---------------------------------------------------------------------------
// alpha gradient: forward pass of the relaxed network from x_0 and u*
// ---------------------------------------------------------------------------
template <bool WSMEM>
__global__ void __launch_bounds__(NT) k_alpha_fwd(BoundArgs a)
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
    float *Z[2];
    Z[0] = p; p += RB * ld;
    Z[1] = p; p += RB * ld;
    float *xs = p; p += RB * s4;

    const int nlive = live_count(a.n, a.d_n);
    const int box0 = blockIdx.x * RB;
    if (box0 >= nlive) return;
    const bool has_alpha = a.alpha != nullptr;
    const int Kp1 = pad4(s + k);
    for (int i = threadIdx.x; i < RB * s; i += NT) xs[(i / s) * s4 + i % s] = a.x0[i % s];
    __syncthreads();
    for (int t = 0; t < H; ++t) {
        for (int i = threadIdx.x; i < RB * Kp1; i += NT) {
            const int r = i / Kp1, c = i % Kp1;
            const int box = box0 + r;
            float v = 0.f;
            if (c < s) v = xs[r * s4 + c];
            else if (c < s + k && box < nlive) v = a.ustar[(size_t)box * d + t * k + (c - s)];
            Z[0][r * ld + c] = v;
        }
        __syncthreads();
        int cur = 0;
        for (int l = 1; l <= L; ++l) {
            dense_rows_auto<RB, NT>(Z[cur], ld, img + N.fwd_w[l], img + N.fwd_b[l], pad4(N.dims[l - 1]),
                                    pad4(N.dims[l]), Z[cur ^ 1], ld, false);
            __syncthreads();
            cur ^= 1;
            if (l < L) {
                const int dl = N.dims[l];
                for (int i = threadIdx.x; i < RB * dl; i += NT) {
                    const int r = i / dl, q = i % dl;
                    const int box = box0 + r;
                    if (box >= nlive) continue;
                    const size_t idx = ((size_t)box * H + t) * sumh + N.hoff[l] + q;
                    const float z = Z[cur][r * ld + q];
                    const float zl = a.pre_lo[idx], zu = a.pre_hi[idx], A = a.A_pre[idx];
                    float D, c;
                    relax_select(zl, zu, A, has_alpha ? a.alpha[idx] : 0.f, has_alpha, D, c);
                    const bool unstable = zl < 0.f && zu > 0.f;
                    a.grad_alpha[idx] = (unstable && A >= 0.f) ? A * z : 0.f;
                    Z[cur][r * ld + q] = fmaf(D, z, c);
                }
                __syncthreads();
            }
        }
        for (int i = threadIdx.x; i < RB * s; i += NT) {
            const int r = i / s, c = i % s;
            xs[r * s4 + c] += Z[cur][r * ld + c];
        }
        __syncthreads();
    }
}

__global__ void k_alpha_init(BoundArgs a)
{
    const int nlive = live_count(a.n, a.d_n);
    const long long total = (long long)nlive * a.H * a.net.sumh;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
        const_cast<float *>(a.alpha)[i] = (a.pre_hi[i] >= -a.pre_lo[i]) ? 1.f : 0.f;
}

__global__ void k_adam(float *alpha, float *m, float *v, const float *g, long long count, float lr, float bc1, float bc2)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = 0.9f * m[i] + 0.1f * gi;
        const float vi = 0.999f * v[i] + 0.001f * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / bc1, vh = vi / bc2;
        float x = alpha[i] + lr * mh / (sqrtf(vh) + 1e-8f);
        alpha[i] = fminf(fmaxf(x, 0.f), 1.f);
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
    size_t rest = (5 * (size_t)RB * N.maxw_p + 2 * (size_t)RB * pad4(N.s) + RB) * sizeof(float);
    return launch_rows_kernel(k_ibp<true>, k_ibp<false>, (size_t)N.img_floats * 4, rest, a.n, a, st);
}

cudaError_t launch_crown(const BoundArgs &a, int, cudaStream_t st)
{
    const NetDesc &N = a.net;
    size_t rest = (2 * (size_t)RB * N.maxw_p + (size_t)RB * pad4(N.s) + (size_t)RB * pad4(a.d) + 2 * RB) * sizeof(float);
    return launch_rows_kernel(k_crown<true>, k_crown<false>, (size_t)N.img_floats * 4, rest, a.n, a, st);
}

cudaError_t launch_alpha_fwd(const BoundArgs &a, int, cudaStream_t st)
{
    const NetDesc &N = a.net;
    size_t rest = (2 * (size_t)RB * N.maxw_p + (size_t)RB * pad4(N.s)) * sizeof(float);
    return launch_rows_kernel(k_alpha_fwd<true>, k_alpha_fwd<false>, (size_t)N.img_floats * 4, rest, a.n, a, st);
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

cudaError_t launch_adam(float *alpha, float *m, float *v, const float *grad, long long count, float lr, float bc1,
                        float bc2, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    long long blocks = (count + 255) / 256;
    k_adam<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(alpha, m, v, grad, count, lr, bc1, bc2);
    return cudaGetLastError();
}

}  // namespace bab
