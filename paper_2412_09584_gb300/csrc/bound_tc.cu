// bound_tc.cu -- backward CROWN (Appendix B.1, Theorem 1) with the per-layer
// products A' W_l on tcgen05 tensor cores, 3-term BF16 split, FP32 accumulate.
//
// A tile is one 128-row MMA holding up to 128 boxes, one per TMEM lane: tc_rows of them (32, 64 or 128; spread
// over the four lane quadrants), fewer when the batch would otherwise leave SMs idle, since the per-box work of
// each layer step (interval-bound loads, relaxation, margin) and not the MMAs bounds the kernel.  Per time step t = H-1 .. 0 the coefficient row
// of each box runs backward through the network:
//
//   lam (coefficient of x_{t+1})  --x W_L^T-->  coefficient on a_{L-1}
//   relax (Lemma 1)               --x W_{L-1}^T--> ...  --x W_1^T-->  [x_t | u_t]
//
// Each product is an MMA chain D[box][j] = sum_k A'[box][k] W_l[k][j] with A'
// (the relaxed coefficients, BF16 hi/lo) in TMEM and W_l^T (BF16 hi/lo) in
// shared memory, loaded once by the bulk copy engine.  The epilogue warps read
// the FP32 accumulator rows from TMEM, apply Lemma 1 with the interval bounds
// of bab_bound_ibp (outward-rounded slope and intercept), add the constant
// terms rounded down, accumulate the rounding-error margin rounded up, and
// write the next A' back to TMEM.  The margin for a split product is
// (3.1 * 2^-16 + gamma_K) sum_k |A'_k| S_k: the BF16 hi/lo representation of
// both operands and the dropped lo*lo term cost at most 3.1 * 2^-16 of
// |A'_k| |W_kj| per term, and gamma_K (unit 2^-23, allowing a truncating
// accumulator) covers the FP32 sum; S_k = sum_j |W_kj| max|a_j| comes from IBP.
//
// Warp roles are those of k_rollout_tc: per slot 8 epilogue warps (primary
// and helper of each TMEM lane quadrant, splitting the columns of hidden
// layers) and one MMA issuer warp, plus a producer warp when the backward
// image is streamed.  Every wait is bounded in time.
#include <cuda_bf16.h>

#include "bab_internal.cuh"
#include "kernels.cuh"
#include "tc_ptx.cuh"

namespace bab {

namespace {

constexpr uint64_t kWaitNs = 2000000000ull;
constexpr int kEpi = 8;
constexpr int kMaxStages = 8;  // ring buffers when the backward image is streamed
constexpr float kTwoU = 1.1920930376163597e-07f;  // 2^-23 (1 + 2^-20)

__device__ __forceinline__ uint32_t pack2(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo)
{
    hi = pack2(a, b);
    lo = pack2(a - __uint_as_float(hi << 16), b - __uint_as_float(hi & 0xFFFF0000u));
}

// Per-thread asynchronous copies global -> shared (16 or 4 bytes), grouped; the issuing thread alone reads what
// it copied, after waiting for its group, so no barrier is involved.
__device__ __forceinline__ void cp16(float *dst, const float *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(dst)), "l"(__cvta_generic_to_global(src))
                 : "memory");
}
__device__ __forceinline__ void cp4(float *dst, const float *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(tc::smem_u32(dst)), "l"(__cvta_generic_to_global(src))
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int NG>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(NG) : "memory");
}
// n floats; 16-byte copies when both ends and n allow it
__device__ __forceinline__ void cp_row(float *dst, const float *src, int n, bool vec)
{
    if (vec)
        for (int c = 0; c < n; c += 4) cp16(dst + c, src + c);
    else
        for (int c = 0; c < n; ++c) cp4(dst + c, src + c);
}

__device__ __forceinline__ bool wwait(uint64_t *bar, uint32_t phase, volatile int *abort)
{
    return __all_sync(0xFFFFFFFFu, tc::mbar_wait(bar, phase, abort, kWaitNs));
}
__device__ __forceinline__ void abort_all(int *status, volatile int *abort)
{
    set_status(status, BAB_ERR_TIMEOUT);
    *abort = 1;
}

// tangent of s^2 at the midpoint of the interval of s = x - g (outward-rounded ends)
__device__ __forceinline__ void tangent(float xl, float xu, float g, float &coef, float &cterm)
{
    const float Ls = __fsub_rd(xl, g), Us = __fsub_ru(xu, g);
    const float m = 0.5f * (Ls + Us);
    coef = 2.f * m;
    cterm = __fmaf_rd(-coef, g, -__fmul_ru(m, m));
}

}  // namespace

// SP: padded state width (16 or 32).  STREAM: the backward image does not fit
// in shared memory; a producer warp streams it one K-atom (64 inputs of a
// layer's product, hi and lo halves) at a time through a ring of a.stages
// buffers in the MMA issuer's order (NSLOT = 1).
// OBST: the pushing-with-obstacles cost (Appendix D.4; a separate instance): the norm's tangent plane and the
// penalties' affine underestimators on each state's box (obstacle_state_lin_row), the pusher penalties' coefficients
// carried to every earlier action, as crown_rows does for the CUDA-core CROWN.
// STG: each epilogue thread copies the interval bounds, margin helpers and slopes of its columns of the next
// hidden layer (and, for the primary, the next step's output-layer helpers and state box) into its own shared
// memory area with cp.async while the tensor core runs the current product, instead of loading them from global
// memory column by column when it needs them (resident image, one slot).
template <int NSLOT, int SP, bool STREAM, bool OBST = false, bool STG = false>
__global__ void __launch_bounds__((NSLOT * (kEpi + 1) + (STREAM ? 1 : 0)) * 32, 1) k_crown_tc(BoundArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    const NetDesc &N = a.net;
    uint8_t *wimg = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float *bias = reinterpret_cast<float *>(wimg + (STREAM ? (size_t)a.stages * a.stage_bytes : (size_t)N.tcb_bytes));
    float *pair = bias + N.tc_bias_floats;  // [NSLOT][128][2]: helper warps' (constant, margin) partials
    // STG areas (16-byte aligned): per column half h and box slot b of the tile, [zl | zu | S | alpha] of
    // a.stg_cols floats each (a.stg_hid floats in all, an odd number of 16-byte units, so that the lanes of a warp
    // reading their areas at one offset hit distinct banks); then per box slot [2][S_L | xl | xu] of SP floats
    // each, double-buffered by the parity of t (a.stg_step floats)
    float *stg = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(pair + NSLOT * 256) + 15) & ~uintptr_t(15));
    __shared__ uint64_t bar_w, bar_a[NSLOT], bar_d[NSLOT], bar_p[NSLOT * 4], bar_fin;
    __shared__ uint64_t bar_full[kMaxStages], bar_empty[kMaxStages];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mma_warp = NSLOT * kEpi;
    const int L = N.L, s = N.s, k = N.k, H = a.H, d = a.d, sumh = N.sumh, sw = N.sumh + N.s;
    volatile int *abort = &abort_flag;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        tc::mbar_init(&bar_w, 1);
        tc::mbar_init(&bar_fin, 1);
        for (int i = 0; i < NSLOT; ++i) {
            tc::mbar_init(&bar_a[i], kEpi);
            tc::mbar_init(&bar_d[i], 1);
            for (int q = 0; q < 4; ++q) tc::mbar_init(&bar_p[i * 4 + q], 1);
        }
        for (int i = 0; i < kMaxStages; ++i) {
            tc::mbar_init(&bar_full[i], 1);
            tc::mbar_init(&bar_empty[i], 1);
        }
        tc::mbar_init_fence();
    }
    if (warp == mma_warp) tc::tmem_alloc(&tmem_base, a.tmem_cols);
    for (int i = threadIdx.x; i < N.tc_bias_floats; i += blockDim.x) bias[i] = a.tc_bias[i];
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (!STREAM) {
        if (threadIdx.x == mma_warp * 32) {
            tc::mbar_arrive_expect_tx(&bar_w, (uint32_t)N.tcb_bytes);
            for (uint32_t off = 0; off < (uint32_t)N.tcb_bytes; off += 32768u)
                tc::bulk_g2s(wimg + off, a.tcb_img + off, min(32768u, (uint32_t)N.tcb_bytes - off), &bar_w);
        }
        if (warp < mma_warp + NSLOT && !wwait(&bar_w, 0, abort) && lane == 0) abort_all(a.status, abort);
    }

    const int nlive = live_count(a.n, a.d_n, a.row0);
    // a tile is one 128-row MMA; it holds tc_rows boxes (fewer than 128 when the batch is small, so that the
    // per-box work spreads over more SMs: the MMAs are a small part of each layer step)
    const int bpt = a.tc_rows;
    const int ntiles = (nlive + bpt - 1) / bpt;
    const int G = gridDim.x * NSLOT;
    const uint32_t tb = tmem_base;
    const int Dc = N.tcb_dcols, Ac = N.tcb_acols;
    const int slot_cols = Dc + 2 * Ac;
    const bool has_alpha = a.alpha != nullptr;

    if (warp < mma_warp) {
        const int slot = warp / kEpi, qw = warp % kEpi, quad = qw & 3;
        const bool primary = qw < 4;
        const int r = 32 * quad + lane;
        const uint32_t dcol = tb + ((uint32_t)(32 * quad) << 16) + slot * slot_cols;
        const uint32_t acol_h = dcol + Dc, acol_l = acol_h + Ac;
        uint32_t phD = 0, phP = 0;
        // the tile's boxes spread evenly over the four lane quadrants (bpt / 4 lanes of each), so that every
        // epilogue warp has boxes to work on
        const int rq = bpt >> 2, lq = r & 31;
        const int bslot = lq < rq ? quad * rq + lq : 0;
        // STG: this thread's hidden-layer area (one per box slot and column half) and its box slot's step area
        const int CW = a.stg_cols;
        float *hz = stg + (size_t)((primary ? 0 : bpt) + bslot) * a.stg_hid;
        float *sa = stg + (size_t)2 * bpt * a.stg_hid + (size_t)bslot * a.stg_step;
        const bool s_vec = (sw & 3) == 0 && (reinterpret_cast<uintptr_t>(a.S) & 15) == 0;
        const bool a_vec = (reinterpret_cast<uintptr_t>(a.alpha) & 15) == 0;
        for (int tile = blockIdx.x * NSLOT + slot; tile < ntiles && !*abort; tile += G) {
            const int box = tile * bpt + (r >> 5) * rq + lq;
            const bool valid = lq < rq && box < nlive;
            float lam[SP];
            float cst = 0.f, mg = 0.f;  // constant (rounded down), margin (rounded up): this warp's share
            float Pu[4] = {0.f, 0.f, 0.f, 0.f};  // obstacle cost: pusher coefficient of the actions (2), its |sum| (2)
            const float *lo_b = a.lo + (size_t)(valid ? box : 0) * d, *hi_b = a.hi + (size_t)(valid ? box : 0) * d;
            bool ok = true;
            // this thread's columns [cb, ce) of hidden layer l: the primary and helper warps of a quadrant split
            // a width that is a multiple of 64, else the primary takes them all
            auto cols = [&](int l, int &cb, int &ce) {
                const int dl = N.dims[l];
                cb = primary ? 0 : dl / 2;
                ce = (dl % 64 == 0) ? cb + dl / 2 : (primary ? dl : 0);
            };
            // STG copies: hidden layer l of step t (one group), and the primary's step-t helpers (one group)
            auto stage_hidden = [&](int t, int l) {
                if (!STG || !valid) return;
                int cb, ce;
                cols(l, cb, ce);
                if (ce > cb) {
                    const size_t ib = ((size_t)box * H + t) * sumh + N.hoff[l] + cb;
                    cp_row(hz, a.pre_lo + ib, ce - cb, true);
                    cp_row(hz + CW, a.pre_hi + ib, ce - cb, true);
                    cp_row(hz + 2 * CW, a.S + ((size_t)box * H + t) * sw + N.hoff[l] + cb, ce - cb, s_vec);
                    if (has_alpha) cp_row(hz + 3 * CW, a.alpha + ib, ce - cb, a_vec);
                }
                cp_commit();
            };
            auto stage_step = [&](int t) {
                if (!STG || !valid || !primary) return;
                float *p = sa + (t & 1) * 3 * SP;
                cp_row(p, a.S + ((size_t)box * H + t) * sw + sumh, s, false);
                if (t >= 1) {
                    cp_row(p + SP, a.x_lo + ((size_t)box * (H + 1) + t) * s, s, false);
                    cp_row(p + 2 * SP, a.x_hi + ((size_t)box * (H + 1) + t) * s, s, false);
                }
                cp_commit();
            };
            stage_step(H - 1);
            stage_hidden(H - 1, L - 1);
            if (primary && OBST) {
                // the obstacle cost's linear lower bound on x_H, then the pusher penalties at H
                float xl[SP], xu[SP];
#pragma unroll
                for (int i = 0; i < SP; ++i) {
                    const size_t xi = ((size_t)box * (H + 1) + H) * s + i;
                    xl[i] = (i < s && valid) ? a.x_lo[xi] : 0.f;
                    xu[i] = (i < s && valid) ? a.x_hi[xi] : 0.f;
                }
                float c = obstacle_state_lin_row<SP>(a.cost, H, s, xl, xu, a.goal, lam);
                if (valid) c = __fadd_rd(c, pusher_lin(a.cost, H, k, lo_b, hi_b, Pu, Pu + 2));
                cst = valid ? c : 0.f;
            } else if (primary) {
                // tangent of ||x_H - g||^2
#pragma unroll
                for (int i = 0; i < SP; ++i) {
                    lam[i] = 0.f;
                    if (i < s && valid) {
                        const size_t xi = ((size_t)box * (H + 1) + H) * s + i;
                        float cf, ct;
                        tangent(a.x_lo[xi], a.x_hi[xi], a.goal[i], cf, ct);
                        lam[i] = cf;
                        cst = __fadd_rd(cst, ct);
                    }
                }
            }
            for (int t = H - 1; t >= 0 && ok; --t) {
                const size_t rowb = ((size_t)box * H + t);
                const float *sx = sa + (t & 1) * 3 * SP;  // STG: the step's [S_L | xl | xu]
                // ---- last layer: A = lam on z_L; constant lam . b_L; product lam W_L^T ----
                if (primary) {
                    const float *bL = bias + N.tc_boff[L];
                    float e = 0.f;
                    uint32_t ph[8], pl[8];
#pragma unroll
                    for (int c16 = 0; c16 < SP / 16; ++c16) {
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const int i0 = c16 * 16 + 2 * q;
                            const float v0 = (i0 < s) ? lam[i0] : 0.f, v1 = (i0 + 1 < s) ? lam[i0 + 1] : 0.f;
                            split2(v0, v1, ph[q], pl[q]);
                        }
                        tc::tmem_st8(acol_h + c16 * 8, ph);
                        tc::tmem_st8(acol_l + c16 * 8, pl);
                    }
                    if (STG) cp_wait<1>();  // the step's group (the hidden layer's may still be in flight)
#pragma unroll
                    for (int i = 0; i < SP; ++i)
                        if (i < s && valid) {
                            cst = __fmaf_rd(lam[i], bL[i], cst);
                            e = __fmaf_ru(fabsf(lam[i]), STG ? sx[i] : a.S[rowb * sw + sumh + i], e);
                        }
                    mg = __fmaf_ru(N.gam_tc[L], e, mg);
                    tc::tmem_wait_st();
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&bar_a[slot]);
                // ---- hidden layers l = L-1 .. 1: relax the coefficient on a_l, product with W_l^T ----
                for (int l = L - 1; l >= 1; --l) {
                    if (!wwait(&bar_d[slot], phD, abort)) {
                        if (lane == 0) abort_all(a.status, abort);
                        ok = false;
                        break;
                    }
                    phD ^= 1;
                    tc::fence_after_sync();
                    int c_beg, c_end;
                    cols(l, c_beg, c_end);
                    const float *bl = bias + N.tc_boff[l];
                    const float gK = N.gam_tc[l];
                    float eg = 0.f, er = 0.f;
                    if (STG) cp_wait<0>();
                    for (int c0 = c_beg; c0 < c_end; c0 += 16) {
                        uint32_t v[16];
                        tc::tmem_ld16(dcol + c0, v);
                        tc::tmem_wait_ld();
                        const size_t ib = rowb * sumh + N.hoff[l] + c0;
                        uint32_t ph[8], pl[8];
#pragma unroll
                        for (int q4 = 0; q4 < 4; ++q4) {
                            float4 zl4 = make_float4(0.f, 0.f, 0.f, 0.f), zu4 = zl4, al4 = zl4, s4 = zl4;
                            if (valid) {
                                if (STG) {
                                    const int o = c0 - c_beg + 4 * q4;
                                    zl4 = *reinterpret_cast<const float4 *>(hz + o);
                                    zu4 = *reinterpret_cast<const float4 *>(hz + CW + o);
                                    s4 = *reinterpret_cast<const float4 *>(hz + 2 * CW + o);
                                    if (has_alpha) al4 = *reinterpret_cast<const float4 *>(hz + 3 * CW + o);
                                } else {
                                    zl4 = *reinterpret_cast<const float4 *>(a.pre_lo + ib + 4 * q4);
                                    zu4 = *reinterpret_cast<const float4 *>(a.pre_hi + ib + 4 * q4);
                                    if (has_alpha) al4 = *reinterpret_cast<const float4 *>(a.alpha + ib + 4 * q4);
                                    const float *Sr = a.S + rowb * sw + N.hoff[l] + c0 + 4 * q4;
                                    s4 = make_float4(Sr[0], Sr[1], Sr[2], Sr[3]);
                                }
                            }
                            const float zlv[4] = {zl4.x, zl4.y, zl4.z, zl4.w}, zuv[4] = {zu4.x, zu4.y, zu4.z, zu4.w};
                            const float alv[4] = {al4.x, al4.y, al4.z, al4.w}, sv[4] = {s4.x, s4.y, s4.z, s4.w};
                            float ap[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int j = 4 * q4 + e;
                                const float A = valid ? __uint_as_float(v[j]) : 0.f;
                                float D, c;
                                relax_select(zlv[e], zuv[e], A, alv[e], has_alpha, D, c);
                                const float Ap = A * D;
                                ap[e] = Ap;
                                if (valid) {
                                    if (a.A_pre) a.A_pre[ib + j] = A;
                                    cst = __fmaf_rd(A, c, cst);
                                    cst = __fmaf_rd(Ap, bl[c0 + j], cst);
                                    eg = __fmaf_ru(fabsf(Ap), sv[e], eg);
                                    if (D != 0.f && D != 1.f) er = __fmaf_ru(fabsf(Ap), fmaxf(-zlv[e], zuv[e]), er);
                                }
                            }
                            split2(ap[0], ap[1], ph[2 * q4], pl[2 * q4]);
                            split2(ap[2], ap[3], ph[2 * q4 + 1], pl[2 * q4 + 1]);
                        }
                        tc::tmem_st8(acol_h + c0 / 2, ph);
                        tc::tmem_st8(acol_l + c0 / 2, pl);
                    }
                    // the next hidden layer's data (this thread is done with its area), or the next step's
                    if (l > 1) {
                        stage_hidden(t, l - 1);
                    } else if (t >= 1) {
                        stage_step(t - 1);
                        stage_hidden(t - 1, L - 1);
                    }
                    mg = __fadd_ru(mg, __fmaf_ru(gK, eg, __fmul_ru(kTwoU, er)));
                    tc::tmem_wait_st();
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&bar_a[slot]);
                }
                if (!ok) break;
                // ---- coefficient on [x_t | u_t]: mu_t, and lam <- lam + A_x (+ tangent of x_t) ----
                if (!wwait(&bar_d[slot], phD, abort)) {
                    if (lane == 0) abort_all(a.status, abort);
                    ok = false;
                    break;
                }
                phD ^= 1;
                tc::fence_after_sync();
                if (primary) {
                    float ax[SP + 16];
                    const int K1 = N.tcb_N[1];
#pragma unroll
                    for (int c16 = 0; c16 < (SP + 16) / 16; ++c16) {
                        if (c16 * 16 >= K1) break;
                        uint32_t v[16];
                        tc::tmem_ld16(dcol + c16 * 16, v);
                        tc::tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 16; ++j) ax[c16 * 16 + j] = __uint_as_float(v[j]);
                    }
                    float e = 0.f;
                    if (valid) {
#pragma unroll
                        for (int j = 0; j < SP + 16; ++j)
                            if (j >= s && j < s + k) {
                                const int ja = j - s;
                                float m_ = ax[j];
                                if (OBST) {
                                    // mu_t = A_u + the pusher coefficient of the later steps (H additions)
                                    const float Pj = ja < 2 ? Pu[ja] : 0.f, Pa = ja < 2 ? Pu[2 + ja] : 0.f;
                                    const float um = fmaxf(fabsf(lo_b[t * k + ja]), fabsf(hi_b[t * k + ja]));
                                    e = __fmaf_ru(__fmul_ru(__fmul_ru((float)(H + 2), kTwoU), __fadd_ru(fabsf(m_), Pa)), um, e);
                                    m_ = m_ + Pj;
                                }
                                a.mu[(size_t)box * d + t * k + ja] = m_;
                            }
                    }
                    // the state box of x_t (t >= 1)
                    auto xbox = [&](int i, float &xl, float &xu) {
                        const size_t xi = ((size_t)box * (H + 1) + t) * s + i;
                        xl = STG ? sx[SP + i] : a.x_lo[xi];
                        xu = STG ? sx[2 * SP + i] : a.x_hi[xi];
                    };
                    float aao[SP];  // obstacle cost: its coefficient of x_t
                    if (OBST) {
                        float c = 0.f;
                        if (t >= 1 && valid) {
                            float xlt[SP], xut[SP];
#pragma unroll
                            for (int i = 0; i < SP; ++i) {
                                xlt[i] = xut[i] = 0.f;
                                if (i < s) xbox(i, xlt[i], xut[i]);
                            }
                            c = obstacle_state_lin_row<SP>(a.cost, t, s, xlt, xut, a.goal, aao);
                            c = __fadd_rd(c, pusher_lin(a.cost, t, k, lo_b, hi_b, Pu, Pu + 2));
                            cst = __fadd_rd(cst, c);
                        } else {
#pragma unroll
                            for (int i = 0; i < SP; ++i) aao[i] = 0.f;
                        }
                    }
#pragma unroll
                    for (int i = 0; i < SP; ++i) {
                        if (i < s) {
                            float aa = 0.f, B;
                            if (t >= 1 && valid) {
                                float xl, xu;
                                xbox(i, xl, xu);
                                if (OBST) {
                                    aa = aao[i];
                                } else {
                                    float ct;
                                    tangent(xl, xu, a.goal[i], aa, ct);
                                    cst = __fadd_rd(cst, ct);
                                }
                                B = fmaxf(fabsf(xl), fabsf(xu));
                            } else {
                                B = fabsf(a.x0[i]);
                            }
                            const float lo_ = lam[i], Ax = ax[i];
                            lam[i] = (lo_ + Ax) + aa;
                            const float mag = __fadd_ru(__fadd_ru(fabsf(lo_), fabsf(Ax)), fabsf(aa));
                            e = __fmaf_ru(__fmul_ru(kTwoU, mag), B, e);
                        }
                    }
                    if (valid) mg = __fadd_ru(mg, e);
                }
            }
            if (!ok) break;
            // ---- combine with the helper's share, concretize (Theorem 2, box form), write ----
            float *pp = pair + ((size_t)slot * 128 + r) * 2;
            if (!primary) {
                pp[0] = cst;
                pp[1] = mg;
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&bar_p[slot * 4 + quad]);
            } else {
                if (!wwait(&bar_p[slot * 4 + quad], phP, abort)) {
                    if (lane == 0) abort_all(a.status, abort);
                    break;
                }
                phP ^= 1;
                cst = __fadd_rd(cst, pp[0]);
                mg = __fadd_ru(mg, pp[1]);
                if (valid) {
                    float c = 0.f, vsum = 0.f, e = 0.f;
#pragma unroll
                    for (int i = 0; i < SP; ++i)
                        if (i < s) c = __fmaf_rd(lam[i], a.x0[i], c);
                    c = __fadd_rd(cst, c);
                    // eight actions at a time: their coefficients and bounds loaded before any result is stored
                    for (int j0 = 0; j0 < d; j0 += 8) {
                        float mv[8], lv[8], hv[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const size_t e8 = (size_t)box * d + (j0 + q < d ? j0 + q : j0);
                            mv[q] = a.mu[e8];
                            lv[q] = a.lo[e8];
                            hv[q] = a.hi[e8];
                        }
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            if (j0 + q >= d) break;
                            const int j = j0 + q;
                            const float m_ = mv[q], lo = lv[q], hi = hv[q];
                            float us, vj;
                            if (a.rho > 0.f) {
                                const float uc = -m_ / (2.f * a.rho);
                                if (uc >= lo && uc <= hi) {
                                    us = uc;
                                    vj = __fdiv_rd(-__fmul_ru(m_, m_), 4.f * a.rho);
                                } else {
                                    us = uc < lo ? lo : hi;
                                    vj = __fmaf_rd(m_, us, __fmul_rd(a.rho, __fmul_rd(us, us)));
                                    const float du = __fmul_ru(kTwoU, fabsf(uc));
                                    e = __fmaf_ru(__fmul_ru(a.rho, du), du, e);
                                }
                            } else {
                                us = m_ >= 0.f ? lo : hi;
                                vj = __fmul_rd(m_, us);
                            }
                            vsum = __fadd_rd(vsum, vj);
                            if (a.ustar) a.ustar[(size_t)box * d + j] = us;
                            if (a.lin_coef && a.lin_coef != a.mu) a.lin_coef[(size_t)box * d + j] = m_;
                        }
                    }
                    const float raw = __fadd_rd(c, vsum);
                    const float marg = __fadd_ru(mg, e);
                    const float lbv = __fsub_rd(raw, marg);
                    a.lb[box] = lbv;
                    if (a.margin) a.margin[box] = marg;
                    if (a.lin_const) a.lin_const[box] = c;
                    if (a.lb_best) a.lb_best[box] = fmaxf(a.lb_best[box], lbv);
                }
            }
        }
        if (STG) cp_wait<0>();  // no copy may land after the shared memory is released
    } else if (warp < mma_warp + NSLOT && lane == 0) {
        // ---------------------- MMA issuer of slot (warp - mma_warp) ----------------------
        const int sl = warp - mma_warp;
        const int gi = blockIdx.x * NSLOT + sl;
        const long long cnt = gi < ntiles ? (ntiles - 1 - gi) / G + 1 : 0;
        long long left = cnt * H * L;
        int l = L;
        uint32_t phA = 0, ncommit = 0, ring_it = 0;
        const uint32_t dcol = tb + sl * slot_cols;
        const uint32_t ah = dcol + Dc, al = ah + Ac;
        while (left > 0 && !*abort) {
            if (!tc::mbar_wait(&bar_a[sl], phA, abort, kWaitNs)) {
                abort_all(a.status, abort);
                break;
            }
            phA ^= 1;
            tc::fence_after_sync();
            const int Kl = N.tcb_K[l], Nl = N.tcb_N[l];
            const uint32_t idesc = tc::idesc_bf16_f32(128, Nl);
            if (!STREAM) {
                // operands stepped with 32-bit adds on precomputed descriptor words, one K-atom unrolled
                const int nks = Kl / 16;
                const uint32_t atom = (uint32_t)Nl * 8u;
                uint32_t qh = tc::desc_sw128_lo(tc::smem_u32(wimg + N.tcb_hi[l]));
                uint32_t ql = tc::desc_sw128_lo(tc::smem_u32(wimg + N.tcb_lo[l]));
                uint32_t th = ah, tl = al;
                for (int ks0 = 0; ks0 < nks; ks0 += 4, qh += atom, ql += atom, th += 32u, tl += 32u) {
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        if (ks0 + kk >= nks) break;
                        const uint64_t dh = tc::desc_join(qh + 2u * kk);
                        tc::mma_ts(dcol, th + 8u * kk, dh, idesc, ks0 + kk > 0 ? 1u : 0u);
                        tc::mma_ts(dcol, th + 8u * kk, tc::desc_join(ql + 2u * kk), idesc, 1u);
                        tc::mma_ts(dcol, tl + 8u * kk, dh, idesc, 1u);
                    }
                }
            } else {
                bool ok = true;
                for (int at = 0; at < (Kl + 63) / 64; ++at, ++ring_it) {
                    const uint32_t st = ring_it % (uint32_t)a.stages, ph = (ring_it / (uint32_t)a.stages) & 1u;
                    if (!tc::mbar_wait(&bar_full[st], ph, abort, kWaitNs)) {
                        abort_all(a.status, abort);
                        ok = false;
                        break;
                    }
                    const uint32_t qh = tc::desc_sw128_lo(tc::smem_u32(wimg + (size_t)st * a.stage_bytes));
                    const uint32_t ql = qh + (uint32_t)Nl * 8u;  // the lo half follows the hi half in the buffer
                    const uint32_t th = ah + 32u * at, tl = al + 32u * at;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const int ks = 4 * at + kk;
                        if (ks >= Kl / 16) break;
                        const uint64_t dh = tc::desc_join(qh + 2u * kk);
                        tc::mma_ts(dcol, th + 8u * kk, dh, idesc, ks > 0 ? 1u : 0u);
                        tc::mma_ts(dcol, th + 8u * kk, tc::desc_join(ql + 2u * kk), idesc, 1u);
                        tc::mma_ts(dcol, tl + 8u * kk, dh, idesc, 1u);
                    }
                    tc::mma_commit(&bar_empty[st]);  // the buffer is free once these MMAs have read it
                }
                if (!ok) break;
            }
            tc::mma_commit(&bar_d[sl]);
            ++ncommit;
            l = (l == 1) ? L : l - 1;
            --left;
        }
        if (*abort) {
            // every issued MMA must finish before the TMEM and the ring are released
            volatile int never = 0;
            tc::mma_commit(&bar_fin);
            tc::mbar_wait(&bar_fin, 0, &never, kWaitNs);
        }
    } else if (STREAM && warp == mma_warp + NSLOT && lane == 0) {
        // ------------- producer: the backward image's atoms in the issuer's order (l = L .. 1) -------------
        const long long cnt = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / G + 1 : 0;
        uint32_t it = 0;
        bool ok = true;
        for (long long q = 0; q < cnt * H && ok && !*abort; ++q) {
            for (int l = L; l >= 1 && ok; --l) {
                const int Kl = N.tcb_K[l], Nl = N.tcb_N[l];
                const uint32_t atom = (uint32_t)Nl * 128u;
                for (int at = 0; at < (Kl + 63) / 64; ++at, ++it) {
                    const uint32_t st = it % (uint32_t)a.stages, ph = (it / (uint32_t)a.stages) & 1u;
                    if (!tc::mbar_wait(&bar_empty[st], ph ^ 1u, abort, kWaitNs)) {
                        abort_all(a.status, abort);
                        ok = false;
                        break;
                    }
                    uint8_t *dst = wimg + (size_t)st * a.stage_bytes;
                    tc::mbar_arrive_expect_tx(&bar_full[st], 2u * atom);
                    tc::bulk_g2s(dst, a.tcb_img + N.tcb_hi[l] + (size_t)at * atom, atom, &bar_full[st]);
                    tc::bulk_g2s(dst + atom, a.tcb_img + N.tcb_lo[l] + (size_t)at * atom, atom, &bar_full[st]);
                }
            }
        }
        // copies still in flight must land before the shared memory is released
        volatile int never = 0;
        const uint32_t inflight = it < (uint32_t)a.stages ? it : (uint32_t)a.stages;
        for (uint32_t j = 0; j < inflight; ++j) {
            const uint32_t i2 = it - 1 - j, st = i2 % (uint32_t)a.stages;
            tc::mbar_wait(&bar_full[st], (i2 / (uint32_t)a.stages) & 1u, &never, kWaitNs);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == mma_warp) {
        __syncwarp();
        tc::fence_after_sync();
        tc::tmem_dealloc(tb, a.tmem_cols);
    }
}

// ---------------------------------------------------------------------------------------------------------------
// Feature-major tensor-core CROWN.  The same backward pass with every product transposed,
//
//   D[i][b] = sum_j W_l[j][i] A'[b][j]      M = 128 feature rows (the layer's inputs, one per TMEM lane),
//                                           N = 32 boxes (a tile), K = d_l,
//
// A = the backward image in shared memory (a layer with fewer than 128 inputs: the rows past them read the
// image's next bytes and their accumulator lanes are ignored), B = the tile's relaxed coefficients A'[b][j],
// written to shared memory by the epilogue as BF16 hi and lo halves (K-major, 128-byte swizzle).  With WQ
// epilogue warps per TMEM lane quadrant (2 or 4), warp (quadrant q, share h) lane `lane` owns feature
// j = 32 q + lane of the tile's boxes 32/WQ h .. 32/WQ (h + 1) - 1: every lane works,
// and a warp's interval-bound loads for one box are 128 contiguous bytes, issued for the next layer while the
// tensor core runs the current product.  Each thread keeps, per box, partial sums over its features of the
// constant (rounded down) and of the rounding-error margin (rounded up); a warp shuffle and the four quadrant
// warps reduce them per box at the end of the tile.  The state lanes (j < s) carry the coefficient of the state
// from step to step, the action lanes (s <= j < s + k) write mu.  Squared-distance cost.
// TF = false: 3-term BF16 split products; TF = true: 3-term TF32 split products (kind::tf32, K = 8 per
// instruction, twice the operand bytes).  MB = 1: every width at most 128, tiles of 32 boxes; MB = 2: widths up
// to 256 as two 128-row feature blocks (two M = 128 products per K step into two accumulators, the second skipped
// for layers with at most 128 inputs), tiles of 16 boxes, warp (quadrant q, block mb, share h) owning feature
// j = 128 mb + 32 q + lane.  The backward image stays resident in shared memory for BF16 with one block; otherwise
// a producer warp streams it through a ring of K blocks (64-wide BF16 or 32-wide TF32, each with the rows of every
// feature block, hi then lo) in the issuer's order.
// ---------------------------------------------------------------------------------------------------------------
constexpr int kNB = 32;  // boxes per tile (the MMA's N) of the one-block kernels: 128 features at most
// Tile shape of k_crown_tcf with MB 128-row feature blocks: 32 / MB boxes, K up to 128 MB, the B operand's halves.
template <int MB>
struct TcfShape {
    static constexpr int KNB = 32 / MB;                      // boxes per tile
    static constexpr uint32_t kHalfBf = 2 * MB * KNB * 128;  // BF16 half of the B operand: 64-wide K blocks
    static constexpr uint32_t kHalfTf = 4 * MB * KNB * 128;  // TF32 half: 32-wide K blocks
    static constexpr uint32_t kRingHalf = MB * 128 * 128;    // ring stage: one K block of the image, MB x 128 rows
    static constexpr uint32_t kRingStage = 2 * kRingHalf;    // of the hi halves, then as many of the lo halves
};
constexpr int kRingMaxStages = 6;

// byte offset of element (box n, k) in the K-major 128-byte-swizzled B operand of KNB rows: BF16 (64 elements per
// 128-byte block) or TF32 (32 per block)
template <int KNB>
__device__ __forceinline__ uint32_t bop_off(int n, int k)
{
    const int kb = k >> 6, w = k & 63;
    return (uint32_t)(kb * KNB * 128 + (n >> 3) * 1024 + (n & 7) * 128 + ((((w * 2) >> 4) ^ (n & 7)) << 4) +
                      ((w * 2) & 15));
}
template <int KNB>
__device__ __forceinline__ uint32_t bop_off_tf(int n, int k)
{
    const int kb = k >> 5, w = k & 31;
    return (uint32_t)(kb * KNB * 128 + (n >> 3) * 1024 + (n & 7) * 128 + (((w >> 2) ^ (n & 7)) << 4) + ((w & 3) << 2));
}
// element (box n, k) of the split B operand in the kernel's arithmetic: BF16 hi = bf16(v), lo = bf16(v - hi), or TF32
// hi = tf32(v), lo = tf32(v - hi) (v - hi is exact in FP32); the lo halves `half` bytes after the hi halves
template <bool TF, int KNB>
__device__ __forceinline__ void st_split(uint8_t *bop, uint32_t half, int n, int k, float v)
{
    if (TF) {
        const uint32_t off = bop_off_tf<KNB>(n, k);
        const float h = tc::tf32_rna(v);
        *reinterpret_cast<float *>(bop + off) = h;
        *reinterpret_cast<float *>(bop + half + off) = tc::tf32_rna(v - h);
    } else {
        const uint32_t off = bop_off<KNB>(n, k);
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
        *reinterpret_cast<__nv_bfloat16 *>(bop + off) = h;
        *reinterpret_cast<__nv_bfloat16 *>(bop + half + off) = l;
    }
}

// Lemma 1's relaxation without branches (the lanes of a warp hold different neurons).  The upper slope of an
// unstable neuron is a fast quotient bounded upward: any slope at least u / (u - l) gives a valid upper line
// through (l, 0), and the quotient of __fdividef over the denominator rounded down (den in [1e-30, 1e36], so
// within 2 ulp wherever the quotient is a normal number), scaled up by 2^-20, raised to at least 2^-99 and capped
// at 1, is one: a quotient below 2^-126, whose rounding the bound does not cover, means a chord below 2^-126.
// Slope 1 where the quotient could be inexact otherwise (huge denominator, tiny numerator).
__device__ __forceinline__ void relax_nb(float zl, float zu, float A, float alpha_j, bool has_alpha, float &D, float &c)
{
    const bool on = zl >= 0.f, off = zu <= 0.f;
    const float den = __fsub_rd(zu, zl);
    const bool fast = den < 1e36f && zu > 1e-30f;
    const float du =
        fast ? fminf(fmaxf(__fmul_ru(__fdividef(zu, den), 1.00000095367431640625f), 0x1p-99f), 1.f) : 1.f;
    const float lower = has_alpha ? alpha_j : (zu >= -zl ? 1.f : 0.f);
    const bool up = !on && !off && A < 0.f;
    D = on ? 1.f : (off ? 0.f : (up ? du : lower));
    c = up ? __fmul_ru(du, -zl) : 0.f;
}

__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void tmem_ld_bpt(uint32_t taddr, uint32_t (&r)[16]) { tc::tmem_ld16(taddr, r); }
__device__ __forceinline__ void tmem_ld_bpt(uint32_t taddr, uint32_t (&r)[8]) { tc::tmem_ld8(taddr, r); }

template <bool ALPHA, int WQ, bool TF, int MB>
__global__ void __launch_bounds__((4 * WQ * MB + 1 + (TF || MB == 2 ? 1 : 0)) * 32, 1) k_crown_tcf(BoundArgs a)
{
    using S = TcfShape<MB>;
    constexpr int KNB = S::KNB;                           // boxes per tile
    constexpr int NE = 4 * WQ * MB, BPT = KNB / WQ;       // epilogue warps, boxes per epilogue thread
    constexpr bool STRM = TF || MB == 2;                  // the image streamed through a ring (else resident)
    constexpr uint32_t kHalf = TF ? S::kHalfTf : S::kHalfBf;
    extern __shared__ uint8_t smem_raw[];
    const NetDesc &N = a.net;
    // the resident image, or the ring of a.stages stages
    uint8_t *wimg = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *bop = wimg + (STRM ? (size_t)a.stages * S::kRingStage : (((size_t)N.tcb_bytes + 1023) & ~size_t(1023)));
    float *bias = reinterpret_cast<float *>(bop + 2 * kHalf);
    float *red = bias + ((N.tc_bias_floats + 3) & ~3);  // [2 tile parities][4 MB quadrants][KNB][2]
    float *small = red + 2 * 4 * MB * KNB * 2;          // [WQ][32 lanes][2 step parities][3][BPT]
    __shared__ uint64_t bar_w, bar_a, bar_d, bar_r, bar_fin;
    __shared__ uint64_t bar_full[STRM ? kRingMaxStages : 1], bar_empty[STRM ? kRingMaxStages : 1];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int L = N.L, s = N.s, k = N.k, H = a.H, d = a.d, sumh = N.sumh, sw = N.sumh + N.s;
    volatile int *abort = &abort_flag;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        tc::mbar_init(&bar_w, 1);
        tc::mbar_init(&bar_a, NE);
        tc::mbar_init(&bar_d, 1);
        tc::mbar_init(&bar_r, NE);
        tc::mbar_init(&bar_fin, 1);
        if (STRM)
            for (int i = 0; i < a.stages; ++i) {
                tc::mbar_init(&bar_full[i], 1);
                tc::mbar_init(&bar_empty[i], 1);
            }
        tc::mbar_init_fence();
    }
    if (warp == NE) tc::tmem_alloc(&tmem_base, 32);
    for (int i = threadIdx.x; i < N.tc_bias_floats; i += blockDim.x) bias[i] = a.tc_bias[i];
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (!STRM) {
        if (threadIdx.x == NE * 32) {
            tc::mbar_arrive_expect_tx(&bar_w, (uint32_t)N.tcb_bytes);
            for (uint32_t off = 0; off < (uint32_t)N.tcb_bytes; off += 32768u)
                tc::bulk_g2s(wimg + off, a.tcb_img + off, min(32768u, (uint32_t)N.tcb_bytes - off), &bar_w);
        }
        if (!wwait(&bar_w, 0, abort) && lane == 0) abort_all(a.status, abort);
    }

    const int nlive = live_count(a.n, a.d_n, a.row0);
    const int ntiles = (nlive + KNB - 1) / KNB;
    const uint32_t tb = tmem_base;

    if (warp < NE) {
        // lane quadrant q, feature block mb, share h of the tile's boxes: feature j of boxes BPT h .. BPT h + BPT - 1
        const int q = warp & 3, mb = MB == 2 ? (warp >> 2) & 1 : 0, h = warp >> (MB == 2 ? 3 : 2);
        const int j = 128 * mb + 32 * q + lane, qd = 4 * mb + q;
        const uint32_t dcol = tb + ((uint32_t)(32 * q) << 16) + (uint32_t)(KNB * mb + BPT * h);
        float *sm = small + (size_t)(h * 32 + lane) * (2 * 3 * BPT);
        const bool state = j < s;
        uint32_t phD = 0, phR = 0;
        int par = 0;
        for (int tile = blockIdx.x; tile < ntiles && !*abort; tile += gridDim.x, par ^= 1) {
            const int box0 = tile * KNB + BPT * h;
            float lam[BPT], cp[BPT], mp[BPT];
            float pzl[BPT], pzu[BPT], pS[BPT], pal[BPT];
            bool ok = true;
            // feature j of hidden layer l at step t for the thread's boxes: interval bounds, margin helper, slope;
            // and the layer after it into L2 (lane L: box L % 16, arrays L / 16 and 2 + L / 16)
            auto prefetch = [&](int t, int l) {
                const int t2 = l > 1 ? t : t - 1, l2 = l > 1 ? l - 1 : L - 1;
                if (t2 >= 0 && box0 + (lane % BPT) < nlive) {
                    const size_t rb = (size_t)(box0 + (lane % BPT)) * H + t2;
                    const size_t ib = rb * sumh + N.hoff[l2];
                    prefetch_l2((lane / BPT) % 2 == 0 ? a.pre_lo + ib : a.pre_hi + ib);
                    if ((lane / BPT) % 2 == 0) prefetch_l2(a.S + rb * sw + N.hoff[l2]);
                    else if (ALPHA) prefetch_l2(a.alpha + ib);
                }
                const bool fj = j < N.dims[l];
#pragma unroll
                for (int bi = 0; bi < BPT; ++bi) {
                    const bool v = fj && box0 + bi < nlive;
                    const size_t rb = (size_t)(box0 + bi) * H + t;
                    const size_t ib = rb * sumh + N.hoff[l] + j;
                    pzl[bi] = v ? a.pre_lo[ib] : 0.f;
                    pzu[bi] = v ? a.pre_hi[ib] : 0.f;
                    pS[bi] = v ? a.S[rb * sw + N.hoff[l] + j] : 0.f;
                    if (ALPHA) pal[bi] = v ? a.alpha[ib] : 0.f;
                }
            };
            // state lanes: the output layer's margin helper at step t and the box of x_t, copied ahead of use
            auto stage_step = [&](int t) {
                if (!state) return;
                float *p = sm + (t & 1) * 3 * BPT;
                for (int bi = 0; bi < BPT && box0 + bi < nlive; ++bi) {
                    const size_t b = (size_t)(box0 + bi);
                    cp4(p + bi, a.S + (b * H + t) * sw + sumh + j);
                    if (t >= 1) {
                        cp4(p + BPT + bi, a.x_lo + (b * (H + 1) + t) * s + j);
                        cp4(p + 2 * BPT + bi, a.x_hi + (b * (H + 1) + t) * s + j);
                    }
                }
                cp_commit();
            };
#pragma unroll
            for (int bi = 0; bi < BPT; ++bi) {
                lam[bi] = cp[bi] = mp[bi] = 0.f;
                if (state && box0 + bi < nlive) {
                    // tangent of ||x_H - g||^2
                    const size_t xi = ((size_t)(box0 + bi) * (H + 1) + H) * s + j;
                    float ct;
                    tangent(a.x_lo[xi], a.x_hi[xi], a.goal[j], lam[bi], ct);
                    cp[bi] = ct;
                }
            }
            stage_step(H - 1);
            prefetch(H - 1, L - 1);
            for (int t = H - 1; t >= 0 && ok; --t) {
                const float *sx = sm + (t & 1) * 3 * BPT;
                // ---- output layer: B = lam (zero up to K), constant lam . b_L, margin of the product ----
                if (q == 0 && j < (TF ? N.tf_K[L] : N.tcb_K[L])) {
                    float bL = 0.f;
                    if (state) {
                        cp_wait<0>();
                        bL = bias[N.tc_boff[L] + j];
                    }
                    const float gL = TF ? N.gam_tf[L] : N.gam_tc[L];
#pragma unroll
                    for (int bi = 0; bi < BPT; ++bi) {
                        const float v = state ? lam[bi] : 0.f;
                        st_split<TF, KNB>(bop, kHalf, BPT * h + bi, j, v);
                        if (state && box0 + bi < nlive) {
                            cp[bi] = __fmaf_rd(v, bL, cp[bi]);
                            mp[bi] = __fmaf_ru(__fmul_ru(gL, fabsf(v)), sx[bi], mp[bi]);
                        }
                    }
                }
                tc::fence_proxy_async_smem();
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&bar_a);
                // ---- hidden layers l = L-1 .. 1: relax the coefficient on a_l, B = A' for the product with W_l ----
                for (int l = L - 1; l >= 1; --l) {
                    if (!wwait(&bar_d, phD, abort)) {
                        if (lane == 0) abort_all(a.status, abort);
                        ok = false;
                        break;
                    }
                    phD ^= 1;
                    tc::fence_after_sync();
                    uint32_t v[BPT];
                    tmem_ld_bpt(dcol, v);
                    tc::tmem_wait_ld();
                    if (j < N.dims[l]) {
                        const float bj = bias[N.tc_boff[l] + j], gK = TF ? N.gam_tf[l] : N.gam_tc[l];
#pragma unroll
                        for (int bi = 0; bi < BPT; ++bi) {
                            const bool vb = box0 + bi < nlive;
                            const float A = vb ? __uint_as_float(v[bi]) : 0.f;
                            float D, c;
                            relax_nb(pzl[bi], pzu[bi], A, ALPHA ? pal[bi] : 0.f, ALPHA, D, c);
                            const float Ap = A * D;
                            if (vb) {
                                if (a.A_pre) a.A_pre[((size_t)(box0 + bi) * H + t) * sumh + N.hoff[l] + j] = A;
                                cp[bi] = __fmaf_rd(A, c, cp[bi]);
                                cp[bi] = __fmaf_rd(Ap, bj, cp[bi]);
                                mp[bi] = __fmaf_ru(__fmul_ru(gK, fabsf(Ap)), pS[bi], mp[bi]);
                                if (D != 0.f && D != 1.f)
                                    mp[bi] = __fmaf_ru(__fmul_ru(kTwoU, fabsf(Ap)), fmaxf(-pzl[bi], pzu[bi]), mp[bi]);
                            }
                            st_split<TF, KNB>(bop, kHalf, BPT * h + bi, j, Ap);
                        }
                    }
                    tc::fence_proxy_async_smem();
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&bar_a);
                    // the next layer's data, loaded while the tensor core runs this product
                    if (l > 1) {
                        prefetch(t, l - 1);
                    } else if (t >= 1) {
                        stage_step(t - 1);
                        prefetch(t - 1, L - 1);
                    }
                }
                if (!ok) break;
                // ---- coefficient on [x_t | u_t]: state lanes update lam (+ tangent of x_t), action lanes write mu ----
                if (!wwait(&bar_d, phD, abort)) {
                    if (lane == 0) abort_all(a.status, abort);
                    ok = false;
                    break;
                }
                phD ^= 1;
                tc::fence_after_sync();
                uint32_t v[BPT];
                tmem_ld_bpt(dcol, v);
                tc::tmem_wait_ld();
                if (state) {
#pragma unroll
                    for (int bi = 0; bi < BPT; ++bi) {
                        if (box0 + bi >= nlive) continue;
                        float aa = 0.f, B;
                        if (t >= 1) {
                            const float xl = sx[BPT + bi], xu = sx[2 * BPT + bi];
                            float ct;
                            tangent(xl, xu, a.goal[j], aa, ct);
                            cp[bi] = __fadd_rd(cp[bi], ct);
                            B = fmaxf(fabsf(xl), fabsf(xu));
                        } else {
                            B = fabsf(a.x0[j]);
                        }
                        const float lo_ = lam[bi], Ax = __uint_as_float(v[bi]);
                        lam[bi] = (lo_ + Ax) + aa;
                        const float mag = __fadd_ru(__fadd_ru(fabsf(lo_), fabsf(Ax)), fabsf(aa));
                        mp[bi] = __fmaf_ru(__fmul_ru(kTwoU, mag), B, mp[bi]);
                    }
                } else if (j < s + k) {
#pragma unroll
                    for (int bi = 0; bi < BPT; ++bi)
                        if (box0 + bi < nlive) a.mu[(size_t)(box0 + bi) * d + t * k + (j - s)] = __uint_as_float(v[bi]);
                }
            }
            if (!ok) break;
            // ---- per box: the constant with lam . x_0, summed over the warp's features, then over the quadrants ----
#pragma unroll
            for (int bi = 0; bi < BPT; ++bi) {
                if (state && box0 + bi < nlive) cp[bi] = __fmaf_rd(lam[bi], a.x0[j], cp[bi]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    cp[bi] = __fadd_rd(cp[bi], __shfl_xor_sync(0xFFFFFFFFu, cp[bi], o));
                    mp[bi] = __fadd_ru(mp[bi], __shfl_xor_sync(0xFFFFFFFFu, mp[bi], o));
                }
            }
            float *rp = red + (size_t)par * 4 * MB * KNB * 2 + ((size_t)qd * KNB + BPT * h) * 2;
            if (lane == 0)
#pragma unroll
                for (int bi = 0; bi < BPT; ++bi) {
                    rp[2 * bi] = cp[bi];
                    rp[2 * bi + 1] = mp[bi];
                }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&bar_r);
            if (warp != 0) continue;
            // ---- warp 0: concretize (Theorem 2, box form) box `lane` of the tile and write ----
            if (!wwait(&bar_r, phR, abort)) {
                if (lane == 0) abort_all(a.status, abort);
                break;
            }
            phR ^= 1;
            const int box = tile * KNB + lane;
            if (lane < KNB && box < nlive) {
            const float *rr = red + (size_t)par * 4 * MB * KNB * 2 + (size_t)lane * 2;
            float c = rr[0], mg = rr[1];
            for (int q2 = 1; q2 < 4 * MB; ++q2) {
                c = __fadd_rd(c, rr[(size_t)q2 * KNB * 2]);
                mg = __fadd_ru(mg, rr[(size_t)q2 * KNB * 2 + 1]);
            }
            float vsum = 0.f, e = 0.f;
            for (int j0 = 0; j0 < d; j0 += 8) {
                float mv[8], lv[8], hv[8];
#pragma unroll
                for (int qq = 0; qq < 8; ++qq) {
                    const size_t e8 = (size_t)box * d + (j0 + qq < d ? j0 + qq : j0);
                    mv[qq] = a.mu[e8];
                    lv[qq] = a.lo[e8];
                    hv[qq] = a.hi[e8];
                }
#pragma unroll
                for (int qq = 0; qq < 8; ++qq) {
                    if (j0 + qq >= d) break;
                    const int jj = j0 + qq;
                    const float m_ = mv[qq], lo = lv[qq], hi = hv[qq];
                    float us, vj;
                    if (a.rho > 0.f) {
                        const float uc = -m_ / (2.f * a.rho);
                        if (uc >= lo && uc <= hi) {
                            us = uc;
                            vj = __fdiv_rd(-__fmul_ru(m_, m_), 4.f * a.rho);
                        } else {
                            us = uc < lo ? lo : hi;
                            vj = __fmaf_rd(m_, us, __fmul_rd(a.rho, __fmul_rd(us, us)));
                            const float du = __fmul_ru(kTwoU, fabsf(uc));
                            e = __fmaf_ru(__fmul_ru(a.rho, du), du, e);
                        }
                    } else {
                        us = m_ >= 0.f ? lo : hi;
                        vj = __fmul_rd(m_, us);
                    }
                    vsum = __fadd_rd(vsum, vj);
                    if (a.ustar) a.ustar[(size_t)box * d + jj] = us;
                    if (a.lin_coef && a.lin_coef != a.mu) a.lin_coef[(size_t)box * d + jj] = m_;
                }
            }
            const float raw = __fadd_rd(c, vsum);
            const float marg = __fadd_ru(mg, e);
            const float lbv = __fsub_rd(raw, marg);
            a.lb[box] = lbv;
            if (a.margin) a.margin[box] = marg;
            if (a.lin_const) a.lin_const[box] = c;
            if (a.lb_best) a.lb_best[box] = fmaxf(a.lb_best[box], lbv);
            }
        }
        cp_wait<0>();  // no copy may land after the shared memory is released
    } else if (warp == NE && lane == 0) {
        // ---------------------- MMA issuer ----------------------
        const long long cnt = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
        long long left = cnt * H * L;
        int l = L;
        uint32_t phA = 0;
        const uint32_t idesc = TF ? tc::idesc_tf32_f32(128, KNB) : tc::idesc_bf16_f32(128, KNB);
        const uint32_t bh = tc::desc_sw128_lo(tc::smem_u32(bop)), bl = tc::desc_sw128_lo(tc::smem_u32(bop + kHalf));
        uint32_t ring_it = 0;
        bool ok = true;
        while (left > 0 && !*abort) {
            if (!tc::mbar_wait(&bar_a, phA, abort, kWaitNs)) {
                abort_all(a.status, abort);
                break;
            }
            phA ^= 1;
            tc::fence_after_sync();
            if (STRM) {
                // K = 16 (BF16) or 8 (TF32) per instruction, four instructions per 128-byte K block from the ring,
                // for each feature block that has rows (the layer's inputs beyond 128 need the second); each stage
                // is released once its MMAs are done
                const int nks = TF ? N.tf_K[l] / 8 : N.tcb_K[l] / 16;
                const int mbl = (MB == 2 && N.dims[l - 1] > 128) ? 2 : 1;
                for (int kb = 0; kb < (nks + 3) / 4; ++kb, ++ring_it) {
                    const uint32_t st = ring_it % (uint32_t)a.stages, ph = (ring_it / (uint32_t)a.stages) & 1u;
                    if (!tc::mbar_wait(&bar_full[st], ph, abort, kWaitNs)) {
                        abort_all(a.status, abort);
                        ok = false;
                        break;
                    }
                    const uint32_t a0 = tc::desc_sw128_lo(tc::smem_u32(wimg + (size_t)st * S::kRingStage));
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const int ks = 4 * kb + kk;
                        if (ks >= nks) break;
                        const uint32_t bo = (uint32_t)(kb * KNB * 8 + kk * 2);
                        const uint64_t Bh = tc::desc_join(bh + bo), Bl = tc::desc_join(bl + bo);
#pragma unroll
                        for (int m = 0; m < MB; ++m) {
                            if (m >= mbl) break;
                            // feature block m: rows 128 m .. 128 m + 127 of the stage's hi and lo halves
                            const uint32_t ah = a0 + (uint32_t)m * (128u * 128u >> 4) + 2u * kk;
                            const uint64_t Ah = tc::desc_join(ah), Al = tc::desc_join(ah + (S::kRingHalf >> 4));
                            const uint32_t dm = tb + (uint32_t)(m * KNB);
                            if (TF) {
                                tc::mma_ss_tf32(dm, Ah, Bh, idesc, ks > 0 ? 1u : 0u);
                                tc::mma_ss_tf32(dm, Al, Bh, idesc, 1u);
                                tc::mma_ss_tf32(dm, Ah, Bl, idesc, 1u);
                            } else {
                                tc::mma_ss(dm, Ah, Bh, idesc, ks > 0 ? 1u : 0u);
                                tc::mma_ss(dm, Al, Bh, idesc, 1u);
                                tc::mma_ss(dm, Ah, Bl, idesc, 1u);
                            }
                        }
                    }
                    tc::mma_commit(&bar_empty[st]);
                }
                if (!ok) break;
            } else {
                const int nks = N.tcb_K[l] / 16, Nl = N.tcb_N[l];
                const uint32_t ah = tc::desc_sw128_lo(tc::smem_u32(wimg + N.tcb_hi[l]));
                const uint32_t al = tc::desc_sw128_lo(tc::smem_u32(wimg + N.tcb_lo[l]));
                for (int ks = 0; ks < nks; ++ks) {
                    // 16-byte units: K-block ks / 4 of the operand, then 32 bytes per K = 16 step inside it
                    const uint32_t ao = (uint32_t)((ks >> 2) * Nl * 8 + (ks & 3) * 2);
                    const uint32_t bo = (uint32_t)((ks >> 2) * KNB * 8 + (ks & 3) * 2);
                    const uint64_t Ah = tc::desc_join(ah + ao), Bh = tc::desc_join(bh + bo);
                    tc::mma_ss(tb, Ah, Bh, idesc, ks > 0 ? 1u : 0u);
                    tc::mma_ss(tb, tc::desc_join(al + ao), Bh, idesc, 1u);
                    tc::mma_ss(tb, Ah, tc::desc_join(bl + bo), idesc, 1u);
                }
            }
            tc::mma_commit(&bar_d);
            l = (l == 1) ? L : l - 1;
            --left;
        }
        if (*abort) {
            volatile int never = 0;
            tc::mma_commit(&bar_fin);
            tc::mbar_wait(&bar_fin, 0, &never, kWaitNs);
        }
    } else if (STRM && warp == NE + 1 && lane == 0) {
        // ---------- producer: the image's K blocks in the issuer's order (t = H-1 .. 0, l = L .. 1) ----------
        // BF16: block kb of layer l's hi rows at tcb_hi[l] + kb rows, its lo rows at tcb_lo[l] + kb rows; TF32: the
        // two halves of block kb back to back at tf_off[l] + 2 kb rows (rows = the layer's tcb_N[l] x 128 bytes)
        const long long cnt = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
        uint32_t it = 0;
        bool ok = true;
        for (long long q = 0; q < cnt * H && ok && !*abort; ++q) {
            for (int l = L; l >= 1 && ok; --l) {
                const uint32_t rows = (uint32_t)N.tcb_N[l] * 128u;  // bytes of one half of a block
                const int nb = TF ? (N.tf_K[l] / 8 + 3) / 4 : (N.tcb_K[l] / 16 + 3) / 4;
                for (int kb = 0; kb < nb; ++kb, ++it) {
                    const uint32_t st = it % (uint32_t)a.stages, ph = (it / (uint32_t)a.stages) & 1u;
                    if (!tc::mbar_wait(&bar_empty[st], ph ^ 1u, abort, kWaitNs)) {
                        abort_all(a.status, abort);
                        ok = false;
                        break;
                    }
                    uint8_t *dst = wimg + (size_t)st * S::kRingStage;
                    const uint8_t *src_h = TF ? a.tcb_img + N.tf_off[l] + (size_t)kb * 2 * rows
                                              : a.tcb_img + N.tcb_hi[l] + (size_t)kb * rows;
                    const uint8_t *src_l = TF ? src_h + rows : a.tcb_img + N.tcb_lo[l] + (size_t)kb * rows;
                    tc::mbar_arrive_expect_tx(&bar_full[st], 2u * rows);
                    tc::bulk_g2s(dst, src_h, rows, &bar_full[st]);
                    tc::bulk_g2s(dst + S::kRingHalf, src_l, rows, &bar_full[st]);
                }
            }
        }
        // copies still in flight must land before the shared memory is released
        volatile int never = 0;
        const uint32_t inflight = it < (uint32_t)a.stages ? it : (uint32_t)a.stages;
        for (uint32_t j2 = 0; j2 < inflight; ++j2) {
            const uint32_t i2 = it - 1 - j2, st = i2 % (uint32_t)a.stages;
            tc::mbar_wait(&bar_full[st], (i2 / (uint32_t)a.stages) & 1u, &never, kWaitNs);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == NE) {
        __syncwarp();
        tc::fence_after_sync();
        tc::tmem_dealloc(tb, 32);
    }
}

// shared memory of k_crown_tcf beyond the resident image or the ring: mb feature blocks, BF16 or TF32 halves
static size_t crown_tcf_extra(const NetDesc &N, bool tf = false, int mb = 1)
{
    const size_t knb = (size_t)(32 / mb), half = (tf ? 4 : 2) * (size_t)mb * knb * 128;
    return 1024 + 1024 + 2 * half + ((size_t)((N.tc_bias_floats + 3) & ~3) + 2 * 4 * (size_t)mb * knb * 2 + 32 * 2 * 3 * knb) * 4;
}

// feature blocks of 128 rows the feature-major kernel needs: 1 (every width <= 128), 2 (<= 256), else 0
static int crown_tcf_blocks(const NetDesc &N)
{
    int w = 0;
    for (int l = 0; l <= N.L; ++l) w = N.dims[l] > w ? N.dims[l] : w;
    return w <= 128 ? 1 : (w <= 256 ? 2 : 0);
}

// ring stages of a streamed feature-major kernel that fit beside the rest of its shared memory
static int crown_ring_stages(const NetDesc &N, bool tf, int mb, int max_smem)
{
    const size_t extra = crown_tcf_extra(N, tf, mb), stage = 2 * (size_t)mb * 128 * 128;
    if (extra >= (size_t)max_smem) return 0;
    const int st = (int)(((size_t)max_smem - extra) / stage);
    return st > kRingMaxStages ? kRingMaxStages : st;
}

// the streamed feature-major kernels (TF32 halves, or BF16 halves with two feature blocks): squared-distance cost,
// hidden widths multiples of 32, every width at most 256, s <= 32, at least two ring stages
static bool crown_tcf_streamed_ok(const NetDesc &N, bool tf, int max_smem)
{
    const int mb = crown_tcf_blocks(N);
    return mb >= 1 && N.tc_ok && N.L >= 2 && N.s <= 32 && (tf ? N.tf_K[N.L] : N.tcb_K[N.L]) <= 32 &&
           crown_ring_stages(N, tf, mb, max_smem) >= 2;
}

// 3-term TF32 split CROWN
bool crown_tf32_supported(const NetDesc &N, int max_smem) { return crown_tcf_streamed_ok(N, true, max_smem); }

// A streamed feature-major launch: TF32 halves (one or two feature blocks) or BF16 halves with two feature blocks;
// 16 epilogue warps and 8 boxes a thread either way (4 warps per quadrant with one block, 2 with two).
static cudaError_t launch_crown_tcf_streamed(BoundArgs a, bool tf, int num_sms, int max_smem, cudaStream_t st)
{
    const NetDesc &N = a.net;
    const int mb = crown_tcf_blocks(N);
    a.stages = crown_ring_stages(N, tf, mb, max_smem);
    a.stage_bytes = 2 * mb * 128 * 128;
    const size_t smem = (size_t)a.stages * a.stage_bytes + crown_tcf_extra(N, tf, mb);
    const int knb = 32 / mb;
    const int ntiles = (a.n + knb - 1) / knb;
    const int grid = ntiles < num_sms ? ntiles : num_sms;
    void (*kern)(BoundArgs);
    if (mb == 1) kern = a.alpha ? k_crown_tcf<true, 4, true, 1> : k_crown_tcf<false, 4, true, 1>;
    else if (tf) kern = a.alpha ? k_crown_tcf<true, 2, true, 2> : k_crown_tcf<false, 2, true, 2>;
    else kern = a.alpha ? k_crown_tcf<true, 2, false, 2> : k_crown_tcf<false, 2, false, 2>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 18 * 32, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_crown_tf32(BoundArgs a, int num_sms, cudaStream_t st)
{
    if (a.n <= 0) return cudaSuccess;
    int dev, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (a.cost.kind != 0 || !crown_tf32_supported(a.net, max_smem)) return cudaErrorNotSupported;
    return launch_crown_tcf_streamed(a, true, num_sms, max_smem, st);
}

// The feature-major kernel: squared-distance cost, every width at most 128 (the MMA's 128 rows), the image resident
bool crown_tcf_supported(const NetDesc &N, int max_smem)
{
    for (int l = 0; l <= N.L; ++l)
        if (N.dims[l] > 128) return false;
    return N.tc_ok && N.L >= 2 && N.s <= 32 && N.tcb_K[N.L] <= 32 &&
           (size_t)N.tcb_bytes + crown_tcf_extra(N) <= (size_t)max_smem;
}

static size_t crown_tc_extra(const NetDesc &N, int nslot)
{
    return (size_t)N.tc_bias_floats * 4 + (size_t)nslot * 128 * 2 * 4 + 1024;
}

// one ring buffer: the largest K-atom of a backward product (N_l x 64 BF16), hi and lo halves
static size_t crown_tc_stage(const NetDesc &N)
{
    size_t b = 0;
    for (int l = 1; l <= N.L; ++l) b = (size_t)N.tcb_N[l] * 128 > b ? (size_t)N.tcb_N[l] * 128 : b;
    return 2 * b;
}

static bool crown_tc_resident(const NetDesc &N, int nslot, int max_smem)
{
    return (size_t)N.tcb_bytes + crown_tc_extra(N, nslot) + 1024 <= (size_t)max_smem;
}

// The obstacle cost runs only with the backward image resident in shared memory.
bool crown_tc_obstacles_supported(const NetDesc &N, int max_smem) { return crown_tc_resident(N, 1, max_smem); }

bool crown_tc_supported(const NetDesc &N, int max_smem)
{
    if (!N.tc_ok || N.L < 2 || N.s > 32 || pad16(N.s + N.k) > 48) return false;
    return crown_tc_resident(N, 1, max_smem) || 2 * crown_tc_stage(N) + crown_tc_extra(N, 1) + 1024 <= (size_t)max_smem;
}

// Staged launches: the floats of the per-thread areas for tiles of bpt boxes (a.stg_* set as a side effect).
static size_t crown_tc_stg_floats(const NetDesc &N, int bpt, bool alpha, BoundArgs &a)
{
    int cols = 0;
    for (int l = 1; l < N.L; ++l) {
        const int dl = N.dims[l], c = dl % 64 == 0 ? dl / 2 : dl;
        cols = c > cols ? c : cols;
    }
    int hid = (alpha ? 4 : 3) * cols + 4;
    if ((hid / 4) % 2 == 0) hid += 4;
    a.stg_cols = cols;
    a.stg_hid = hid;
    a.stg_step = 6 * pad16(N.s) + 4;
    return (size_t)2 * bpt * hid + (size_t)bpt * a.stg_step;
}

template <int NSLOT, int SP, bool STREAM, bool OBST, bool STG>
static cudaError_t launch_variant(const BoundArgs &a, int grid, size_t smem, cudaStream_t st)
{
    auto kern = k_crown_tc<NSLOT, SP, STREAM, OBST, STG>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, (NSLOT * (kEpi + 1) + (STREAM ? 1 : 0)) * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <int SP>
static cudaError_t launch_shape(const BoundArgs &a, int nslot, bool stream, bool stg, int grid, size_t smem,
                                cudaStream_t st)
{
    if (a.cost.kind == 1) {
        // the obstacle cost: resident backward image only (the caller checks crown_tc_obstacles_supported)
        if (stream) return cudaErrorNotSupported;
        if (stg) return launch_variant<1, SP, false, true, true>(a, grid, smem, st);
        return nslot == 2 ? launch_variant<2, SP, false, true, false>(a, grid, smem, st)
                          : launch_variant<1, SP, false, true, false>(a, grid, smem, st);
    }
    if (stream) return launch_variant<1, SP, true, false, false>(a, grid, smem, st);
    if (stg) return launch_variant<1, SP, false, false, true>(a, grid, smem, st);
    return nslot == 2 ? launch_variant<2, SP, false, false, false>(a, grid, smem, st)
                      : launch_variant<1, SP, false, false, false>(a, grid, smem, st);
}

// variant: 3 or 4 feature-major with 8 or 16 epilogue warps (widths up to 256: the streamed two-block kernel for
// either; fall back to 0 where it does not apply), 0 staged (one slot, a multiple of 4 up to
// 32 boxes per tile, the fewest that spread the batch over the SMs; falls back to 1 when the areas do not fit),
// 1 or 2 unstaged tiles per CTA, -1 the first of 4, 0, 1 that applies
cudaError_t launch_crown_tc(BoundArgs a, int variant, int num_sms, cudaStream_t st)
{
    const NetDesc &N = a.net;
    if (a.n <= 0) return cudaSuccess;
    int dev, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if ((variant == -1 || variant == 3 || variant == 4) && a.cost.kind == 0 && crown_tcf_blocks(N) == 2 &&
        crown_tcf_streamed_ok(N, false, max_smem))
        return launch_crown_tcf_streamed(a, false, num_sms, max_smem, st);
    if ((variant == -1 || variant == 3 || variant == 4) && a.cost.kind == 0 && crown_tcf_supported(N, max_smem)) {
        const size_t smem = (size_t)N.tcb_bytes + crown_tcf_extra(N);
        const int ntiles = (a.n + kNB - 1) / kNB;
        const int grid = ntiles < num_sms ? ntiles : num_sms;
        const int wq = variant == 3 ? 2 : 4;  // epilogue warps per TMEM lane quadrant
        auto kern = wq == 2 ? (a.alpha ? k_crown_tcf<true, 2, false, 1> : k_crown_tcf<false, 2, false, 1>)
                            : (a.alpha ? k_crown_tcf<true, 4, false, 1> : k_crown_tcf<false, 4, false, 1>);
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, (4 * wq + 1) * 32, smem, st>>>(a);
        return cudaGetLastError();
    }
    if (variant == 3 || variant == 4) variant = 0;
    const int slot_cols = N.tcb_dcols + 2 * N.tcb_acols;
    const int SP = pad16(N.s);
    int cols = 32;
    while (cols < slot_cols) cols *= 2;
    if (variant == -1 || variant == 0) {
        int bpt = (a.n + num_sms - 1) / num_sms;
        bpt = (bpt + 3) & ~3;
        bpt = bpt < 4 ? 4 : (bpt > 32 ? 32 : bpt);
        const bool resident = crown_tc_resident(N, 1, max_smem);
        for (; resident && bpt >= 4; bpt -= 4) {
            const size_t smem = (size_t)N.tcb_bytes + crown_tc_extra(N, 1) + 16 +
                                4 * crown_tc_stg_floats(N, bpt, a.alpha != nullptr, a);
            if (smem + 1024 > (size_t)max_smem) continue;
            a.tc_rows = bpt;
            a.tmem_cols = (uint32_t)cols;
            a.stages = 0;
            const int ntiles = (a.n + bpt - 1) / bpt;
            const int grid = ntiles < num_sms ? ntiles : num_sms;
            if (SP == 16) return launch_shape<16>(a, 1, false, true, grid, smem, st);
            if (SP == 32) return launch_shape<32>(a, 1, false, true, grid, smem, st);
            return cudaErrorInvalidConfiguration;
        }
    }
    a.stg_cols = a.stg_hid = a.stg_step = 0;
    // boxes per tile: 128 when the tiles at least fill the SMs, else 64 or 32
    a.tc_rows = 128;
    while (a.tc_rows > 32 && (a.n + a.tc_rows - 1) / a.tc_rows < num_sms) a.tc_rows /= 2;
    if ((a.n + a.tc_rows - 1) / a.tc_rows > num_sms && a.tc_rows < 128) a.tc_rows *= 2;
    const int ntiles = (a.n + a.tc_rows - 1) / a.tc_rows;
    int nslot = (ntiles > num_sms && 2 * slot_cols <= 512) ? 2 : 1;
    if (variant == 1 || variant == 2) nslot = variant;
    const bool stream = !crown_tc_resident(N, nslot, max_smem) && !crown_tc_resident(N, 1, max_smem);
    if (!stream && !crown_tc_resident(N, nslot, max_smem)) nslot = 1;
    if (stream) nslot = 1;
    cols = 32;
    while (cols < nslot * slot_cols) cols *= 2;
    if (cols > 512) return cudaErrorInvalidConfiguration;
    a.tmem_cols = (uint32_t)cols;
    size_t smem;
    if (stream) {
        a.stage_bytes = (int)crown_tc_stage(N);
        const size_t room = (size_t)max_smem - 1024 - crown_tc_extra(N, 1);
        int stages = (int)(room / a.stage_bytes);
        stages = stages > kMaxStages ? kMaxStages : stages;
        if (stages < 2) return cudaErrorInvalidConfiguration;
        a.stages = stages;
        smem = (size_t)stages * a.stage_bytes + crown_tc_extra(N, 1);
    } else {
        a.stages = 0;
        smem = (size_t)N.tcb_bytes + crown_tc_extra(N, nslot);
    }
    int grid = (ntiles + nslot - 1) / nslot;
    grid = grid < num_sms ? grid : num_sms;
    if (SP == 16) return launch_shape<16>(a, nslot, stream, false, grid, smem, st);
    if (SP == 32) return launch_shape<32>(a, nslot, stream, false, grid, smem, st);
    return cudaErrorInvalidConfiguration;
}

}  // namespace bab
