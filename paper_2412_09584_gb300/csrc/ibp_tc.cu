// ibp_tc.cu -- interval bound propagation on tcgen05 tensor cores (the intermediate bounds that Lemma 1 of
// Appendix B.1 relaxes), an alternative to the directed-rounding FP32 kernel k_ibp.
//
// Each layer input is taken in centre-radius form, [l, u] inside [c - r, c + r], and the products
//
//   zc = W c,   zr = |W| r,   zs = |W| (|c| + r)
//
// run feature-major: the layer's outputs on the MMA's 128 rows (one or two row blocks), a tile's boxes on its
// columns, K = the layer's inputs.  W c and |W| r are 3-term split products (hi x hi + lo x hi + hi x lo), zs a
// single product of the hi halves, in one of two precisions:
//
//   BF16 halves (kind::f16): 32 boxes a tile, eps = gamma_split(K) = 3.1 * 2^-16 + K 2^-23 / (1 - K 2^-23),
//     K = d_{l-1} rounded up to 16, and zs within 2^-6 of the exact |W| (|c| + r) (each BF16 half within 2^-9 of
//     its value, the FP32 sum within K 2^-23);
//   TF32 halves (kind::tf32): 16 boxes a tile, eps = gamma_tf32(K) = 3.1 * 2^-22 + K 2^-23 / (1 - K 2^-23),
//     K rounded up to 8, and zs within 2^-9 (each TF32 half within 2^-11).
//
// Their rounding is bounded, not directed: each split product is within eps of sum |terms|, and both sums of
// |terms| are at most S' = |W| (|c| + r), which zs bounds from above once scaled by 1 + 2^-6 (1 + 2^-9 for TF32).
// So
//
//   lower = zc + b - zr - eps S',   upper = zc + b + zr + eps S'   (each addition rounded outward),
//
// contains W a + b for every a in [c - r, c + r]; S' (at least sum_j |W_kj| max|a_j|) is what CROWN's margin reads.
// The weights (W and |W|, hi and lo halves) exceed shared memory at every size of interest, so a producer warp
// streams them one 64 KB stage (one 128-row block x 64 BF16 or 32 TF32 inputs of the four images: 128-byte rows)
// at a time through a ring, in the MMA issuer's order; the tile's operands c (hi, lo), r (hi, lo) and |c| + r stay
// in shared memory, 16 KB each in either precision.  Epilogue warp (row block mb, lane quadrant q) lane `lane` owns
// output j = 128 mb + 32 q + lane of every box of the tile, or, in a layer of one row block, output 32 q + lane of
// half the tile's boxes.  Squared-distance cost; the interval of the cost (lb_ibp) comes from a separate pass.
// Every wait is bounded in time.
#include <cuda_bf16.h>

#include "bab_internal.cuh"
#include "ibp_tc.cuh"
#include "kernels.cuh"
#include "tc_ptx.cuh"

namespace bab {

namespace {

constexpr uint64_t kWaitNs = 2000000000ull;
constexpr int kEpiW = 8;                 // epilogue warps: 2 row blocks x 4 lane quadrants
constexpr int kStages = 2;               // ring stages
constexpr uint32_t kStageBytes = 65536;  // W hi | W lo | |W| hi | |W| lo, 16 KB each (128 rows x 128 bytes)
constexpr uint32_t kOpBytes = 16384;     // one B operand: K <= 256 inputs of a tile's boxes in 128-byte row blocks

// per precision: boxes a tile (the MMA's N), inputs a 128-byte row, and the factor that lifts zs above S'
template <bool TF> struct IbpCfg {
    static constexpr int NB = 32, KR = 64, ES = 2;
    static constexpr float kS_up = 1.015625f;  // 1 + 2^-6
};
template <> struct IbpCfg<true> {
    static constexpr int NB = 16, KR = 32, ES = 4;
    static constexpr float kS_up = 1.001953125f;  // 1 + 2^-9
};

__device__ __forceinline__ bool wwait_(uint64_t *bar, uint32_t phase, volatile int *abort)
{
    return __all_sync(0xFFFFFFFFu, tc::mbar_wait(bar, phase, abort, kWaitNs));
}
__device__ __forceinline__ void abort_(int *status, volatile int *abort)
{
    set_status(status, BAB_ERR_TIMEOUT);
    *abort = 1;
}

// byte offset of element (box n, input k) in a K-major 128-byte-swizzled B operand of NB rows: KR inputs a row
template <bool TF> __device__ __forceinline__ uint32_t op_off(int n, int k)
{
    constexpr int NB = IbpCfg<TF>::NB, KR = IbpCfg<TF>::KR, ES = IbpCfg<TF>::ES;
    const int kb = k / KR, w = (k % KR) * ES;
    return (uint32_t)(kb * NB * 128 + (n >> 3) * 1024 + (n & 7) * 128 + (((w >> 4) ^ (n & 7)) << 4) + (w & 15));
}

// the operands of one input (interval [l, u]) for box n: c in hi and lo halves, r in hi and lo, |c| + r rounded up
// in FP32 and then to the nearest hi value (the five B operands follow one another, kOpBytes apart)
template <bool TF> __device__ __forceinline__ void put_input(uint8_t *ops, int n, int k, float l, float u)
{
    const float c = 0.5f * __fadd_rn(l, u);
    const float r = fmaxf(__fsub_ru(u, c), __fsub_ru(c, l));
    const float m = __fadd_ru(fabsf(c), r);
    const uint32_t o = op_off<TF>(n, k);
    if constexpr (TF) {
        const float ch = tc::tf32_rna(c), rh = tc::tf32_rna(r);
        *reinterpret_cast<float *>(ops + o) = ch;
        *reinterpret_cast<float *>(ops + kOpBytes + o) = tc::tf32_rna(c - ch);
        *reinterpret_cast<float *>(ops + 2 * kOpBytes + o) = rh;
        *reinterpret_cast<float *>(ops + 3 * kOpBytes + o) = tc::tf32_rna(r - rh);
        *reinterpret_cast<float *>(ops + 4 * kOpBytes + o) = tc::tf32_rna(m);
    } else {
        const __nv_bfloat16 ch = __float2bfloat16_rn(c), rh = __float2bfloat16_rn(r);
        const __nv_bfloat16 cl = __float2bfloat16_rn(c - __bfloat162float(ch)),
                            rl = __float2bfloat16_rn(r - __bfloat162float(rh));
        *reinterpret_cast<__nv_bfloat16 *>(ops + o) = ch;
        *reinterpret_cast<__nv_bfloat16 *>(ops + kOpBytes + o) = cl;
        *reinterpret_cast<__nv_bfloat16 *>(ops + 2 * kOpBytes + o) = rh;
        *reinterpret_cast<__nv_bfloat16 *>(ops + 3 * kOpBytes + o) = rl;
        *reinterpret_cast<__nv_bfloat16 *>(ops + 4 * kOpBytes + o) = __float2bfloat16_rn(m);
    }
}

template <bool TF> __device__ __forceinline__ void mma_(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    if constexpr (TF)
        tc::mma_ss_tf32(d, a, b, idesc, acc);
    else
        tc::mma_ss(d, a, b, idesc, acc);
}

// input blocks of layer l (64 BF16 or 32 TF32 inputs each): its image has one 64 KB stage per row block and block
template <bool TF> __device__ __forceinline__ int n_ka(const NetDesc &N, int l)
{
    return TF ? ibp_tf_ka(N.dims[l - 1]) : N.ibp_ka[l];
}

}  // namespace

template <bool TF> __global__ void __launch_bounds__((kEpiW + 2) * 32, 1) k_ibp_tc(BoundArgs a)
{
    constexpr int kNB = IbpCfg<TF>::NB, kHalf = kNB / 2;
    extern __shared__ uint8_t smem_raw[];
    const NetDesc &N = a.net;
    uint8_t *ring = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *ops = ring + kStages * kStageBytes;                         // c hi, c lo, r hi, r lo, |c| + r
    float *xs = reinterpret_cast<float *>(ops + 5 * kOpBytes);         // [kNB][2][32]: the tile's state boxes
    __shared__ uint64_t bar_a, bar_d, bar_fin, bar_full[kStages], bar_empty[kStages];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int L = N.L, s = N.s, k = N.k, H = a.H, d = a.d, sumh = N.sumh, sw = N.sumh + N.s;
    volatile int *abort = &abort_flag;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        tc::mbar_init(&bar_a, kEpiW);
        tc::mbar_init(&bar_d, 1);
        tc::mbar_init(&bar_fin, 1);
        for (int i = 0; i < kStages; ++i) {
            tc::mbar_init(&bar_full[i], 1);
            tc::mbar_init(&bar_empty[i], 1);
        }
        tc::mbar_init_fence();
    }
    if (warp == kEpiW) tc::tmem_alloc(&tmem_base, 256);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();

    const int nlive = live_count(a.n, a.d_n, a.row0);
    const int ntiles = (nlive + kNB - 1) / kNB;
    const uint32_t tb = tmem_base;
    const int K1 = TF ? pad8(N.dims[0]) : pad16(N.dims[0]);

    if (warp < kEpiW) {
        // ------------------------------- epilogue -------------------------------
        const int mb = warp >> 2, q = warp & 3, j = 128 * mb + 32 * q + lane;
        uint32_t phD = 0;
        // A layer of one row block (at most 128 outputs) has its tile split by boxes: warp (mb, q) then owns output
        // 32 q + lane of the tile's boxes kHalf mb .. kHalf mb + kHalf - 1 (both warp sets busy); with two row blocks
        // each warp takes all the tile's boxes of its block's outputs.  The first layer's inputs and the state boxes (at most 128 and 32 wide) are
        // always split by boxes.
        const int j1 = 32 * q + lane, nb1 = kHalf * mb;
        // layer 1's input of step t for the warp's boxes: [x_t | u_t] (the state boxes from xs), zero padded
        auto layer1_inputs = [&](int box0, int t) {
            if (j1 >= K1) return;
            for (int n = nb1; n < nb1 + kHalf; ++n) {
                const int box = box0 + n;
                float l = 0.f, u = 0.f;
                if (j1 < s) {
                    l = xs[(n * 2) * 32 + j1];
                    u = xs[(n * 2 + 1) * 32 + j1];
                } else if (j1 < s + k && box < nlive) {
                    l = a.lo[(size_t)box * d + t * k + (j1 - s)];
                    u = a.hi[(size_t)box * d + t * k + (j1 - s)];
                }
                put_input<TF>(ops, n, j1, l, u);
            }
        };
        auto handoff = [&]() {
            tc::fence_proxy_async_smem();
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&bar_a);
        };
        for (int tile = blockIdx.x; tile < ntiles && !*abort; tile += gridDim.x) {
            const int box0 = tile * kNB;
            if (j1 < s)
                for (int n = nb1; n < nb1 + kHalf; ++n) {
                    xs[(n * 2) * 32 + j1] = xs[(n * 2 + 1) * 32 + j1] = a.x0[j1];
                    if (box0 + n < nlive) {
                        a.x_lo[(size_t)(box0 + n) * (H + 1) * s + j1] = a.x0[j1];
                        a.x_hi[(size_t)(box0 + n) * (H + 1) * s + j1] = a.x0[j1];
                    }
                }
            layer1_inputs(box0, 0);
            handoff();
            bool ok = true;
            for (int t = 0; t < H && ok; ++t) {
                for (int l = 1; l <= L && ok; ++l) {
                    if (!wwait_(&bar_d, phD, abort)) {
                        if (lane == 0) abort_(a.status, abort);
                        ok = false;
                        break;
                    }
                    phD ^= 1;
                    tc::fence_after_sync();
                    const int dl = N.dims[l];
                    const bool one = N.ibp_mb[l] == 1;
                    const int jo = one ? j1 : j, nbeg = one ? nb1 : 0, nend = one ? nb1 + kHalf : kNB;
                    const uint32_t dl_ = tb + ((uint32_t)(32 * q) << 16) + (one ? 0u : (uint32_t)(3 * kNB * mb));
                    const bool fj = jo < dl;
                    const float bj = fj ? __ldg(a.fwd + N.fwd_b[l] + jo) : 0.f;
                    const float eps = TF ? gamma_tf32(pad8(N.dims[l - 1])) : N.gam_ibp[l];
                    for (int c8 = nbeg / 8; c8 < nend / 8; ++c8) {
                        uint32_t vc[8], vr[8], vs[8];
                        tc::tmem_ld8(dl_ + 8 * c8, vc);
                        tc::tmem_ld8(dl_ + kNB + 8 * c8, vr);
                        tc::tmem_ld8(dl_ + 2 * kNB + 8 * c8, vs);
                        tc::tmem_wait_ld();
                        if (!fj) continue;
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int n = 8 * c8 + e, box = box0 + n;
                            const float Sp = __fmul_ru(__uint_as_float(vs[e]), IbpCfg<TF>::kS_up);
                            const float rad = __fadd_ru(__uint_as_float(vr[e]), __fmul_ru(eps, Sp));
                            const float zb = __uint_as_float(vc[e]);
                            const float lo = __fsub_rd(__fadd_rd(zb, bj), rad);
                            const float hi = __fadd_ru(__fadd_ru(zb, bj), rad);
                            const size_t rb = (size_t)box * H + t;
                            if (l < L) {
                                if (box < nlive) {
                                    a.pre_lo[rb * sumh + N.hoff[l] + jo] = lo;
                                    a.pre_hi[rb * sumh + N.hoff[l] + jo] = hi;
                                    a.S[rb * sw + N.hoff[l] + jo] = Sp;
                                }
                                put_input<TF>(ops, n, jo, fmaxf(lo, 0.f), fmaxf(hi, 0.f));
                            } else {
                                // x_{t+1} in [x_t] + [z_L] (the output layer has one row block: jo = j1 < s)
                                const float nl = __fadd_rd(xs[(n * 2) * 32 + jo], lo);
                                const float nh = __fadd_ru(xs[(n * 2 + 1) * 32 + jo], hi);
                                xs[(n * 2) * 32 + jo] = nl;
                                xs[(n * 2 + 1) * 32 + jo] = nh;
                                if (box < nlive) {
                                    a.S[rb * sw + sumh + jo] = Sp;
                                    a.x_lo[((size_t)box * (H + 1) + t + 1) * s + jo] = nl;
                                    a.x_hi[((size_t)box * (H + 1) + t + 1) * s + jo] = nh;
                                }
                            }
                        }
                    }
                    if (l == L && t + 1 < H) layer1_inputs(box0, t + 1);
                    if (l < L || t + 1 < H) handoff();
                }
            }
            if (!ok) break;
        }
    } else if (warp == kEpiW && lane == 0) {
        // ---------------------- MMA issuer ----------------------
        const int cnt = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
        const uint32_t idesc = TF ? tc::idesc_tf32_f32(128, kNB) : tc::idesc_bf16_f32(128, kNB);
        const uint32_t opd = tc::desc_sw128_lo(tc::smem_u32(ops)), ringd = tc::desc_sw128_lo(tc::smem_u32(ring));
        constexpr uint32_t kOp16 = kOpBytes / 16, kImg16 = 16384 / 16, kStage16 = kStageBytes / 16;
        uint32_t phA = 0, it = 0;
        bool ok = true;
        for (int c = 0; c < cnt && ok; ++c)
            for (int t = 0; t < H && ok; ++t)
                for (int l = 1; l <= L && ok; ++l) {
                    if (!tc::mbar_wait(&bar_a, phA, abort, kWaitNs)) {
                        abort_(a.status, abort);
                        ok = false;
                        break;
                    }
                    phA ^= 1;
                    tc::fence_after_sync();
                    const int nks = TF ? pad8(N.dims[l - 1]) / 8 : pad16(N.dims[l - 1]) / 16, nka = n_ka<TF>(N, l);
                    for (int mb = 0; mb < N.ibp_mb[l] && ok; ++mb) {
                        const uint32_t dzc = tb + (uint32_t)(3 * kNB * mb), dzr = dzc + kNB, dzs = dzc + 2 * kNB;
                        for (int ka = 0; ka < nka; ++ka, ++it) {
                            const uint32_t st = it % kStages, ph = (it / kStages) & 1u;
                            if (!tc::mbar_wait(&bar_full[st], ph, abort, kWaitNs)) {
                                abort_(a.status, abort);
                                ok = false;
                                break;
                            }
                            const uint32_t wh = ringd + st * kStage16, wl = wh + kImg16, ah = wh + 2 * kImg16,
                                           al = wh + 3 * kImg16;
                            const uint32_t ob = opd + (uint32_t)ka * (kNB * 8);
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const int ks = 4 * ka + kk;
                                if (ks >= nks) break;
                                const uint32_t acc = ks > 0 ? 1u : 0u, o = 2u * kk;
                                const uint64_t Wh = tc::desc_join(wh + o), Ah = tc::desc_join(ah + o);
                                const uint64_t ch = tc::desc_join(ob + o), rh = tc::desc_join(ob + 2 * kOp16 + o);
                                mma_<TF>(dzc, Wh, ch, idesc, acc);
                                mma_<TF>(dzc, tc::desc_join(wl + o), ch, idesc, 1u);
                                mma_<TF>(dzc, Wh, tc::desc_join(ob + kOp16 + o), idesc, 1u);
                                mma_<TF>(dzr, Ah, rh, idesc, acc);
                                mma_<TF>(dzr, tc::desc_join(al + o), rh, idesc, 1u);
                                mma_<TF>(dzr, Ah, tc::desc_join(ob + 3 * kOp16 + o), idesc, 1u);
                                mma_<TF>(dzs, Ah, tc::desc_join(ob + 4 * kOp16 + o), idesc, acc);
                            }
                            tc::mma_commit(&bar_empty[st]);  // the stage is free once these MMAs have read it
                        }
                    }
                    if (ok) tc::mma_commit(&bar_d);
                }
        if (*abort) {
            volatile int never = 0;
            tc::mma_commit(&bar_fin);
            tc::mbar_wait(&bar_fin, 0, &never, kWaitNs);
        }
    } else if (warp == kEpiW + 1 && lane == 0) {
        // ------------- producer: the interval image's stages in the issuer's order -------------
        const int cnt = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
        uint32_t it = 0;
        bool ok = true;
        for (int c = 0; c < cnt && ok && !*abort; ++c)
            for (int t = 0; t < H && ok; ++t) {
                const uint8_t *img = a.ibp_img;  // the layers' stages follow one another in either image
                for (int l = 1; l <= L && ok; ++l) {
                    const int nblk = N.ibp_mb[l] * n_ka<TF>(N, l);
                    for (int blk = 0; blk < nblk; ++blk, ++it) {
                        const uint32_t st = it % kStages, ph = (it / kStages) & 1u;
                        if (!tc::mbar_wait(&bar_empty[st], ph ^ 1u, abort, kWaitNs)) {
                            abort_(a.status, abort);
                            ok = false;
                            break;
                        }
                        const uint8_t *src = img + (size_t)blk * kStageBytes;
                        uint8_t *dst = ring + (size_t)st * kStageBytes;
                        tc::mbar_arrive_expect_tx(&bar_full[st], kStageBytes);
                        tc::bulk_g2s(dst, src, 32768u, &bar_full[st]);
                        tc::bulk_g2s(dst + 32768, src + 32768, 32768u, &bar_full[st]);
                    }
                    img += (size_t)nblk * kStageBytes;
                }
            }
        // copies still in flight must land before the shared memory is released
        volatile int never = 0;
        const uint32_t inflight = it < kStages ? it : kStages;
        for (uint32_t jj = 0; jj < inflight; ++jj) {
            const uint32_t i2 = it - 1 - jj, st = i2 % kStages;
            tc::mbar_wait(&bar_full[st], (i2 / kStages) & 1u, &never, kWaitNs);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == kEpiW) {
        __syncwarp();
        tc::fence_after_sync();
        tc::tmem_dealloc(tb, 256);
    }
}

// The interval bound of the squared-distance objective from the state boxes: per step the minimum of rho u^2 over
// the actions' intervals, then of ||x_{t+1} - g||^2 over the next state's box, each rounded down (the sums k_ibp
// forms beside its products), one warp per box.
__global__ void k_lb_from_boxes(BoundArgs a)
{
    const int lane = threadIdx.x & 31;
    const int box = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int nlive = live_count(a.n, a.d_n, a.row0);
    if (box >= nlive) return;
    const int s = a.net.s, k = a.net.k, H = a.H, d = a.d;
    float acc = 0.f;
    for (int t = 0; t < H; ++t) {
        if (a.rho > 0.f) {
            float v = 0.f;
            for (int j = lane; j < k; j += 32)
                v = __fadd_rd(v, sq_min_rd(a.lo[(size_t)box * d + t * k + j], a.hi[(size_t)box * d + t * k + j]));
            v = warp_sum_rd(v);
            acc = __fadd_rd(acc, __fmul_rd(a.rho, v));
        }
        float v = 0.f;
        for (int i = lane; i < s; i += 32) {
            const size_t xi = ((size_t)box * (H + 1) + t + 1) * s + i;
            const float g = a.goal[i];
            v = __fadd_rd(v, sq_min_rd(__fsub_rd(a.x_lo[xi], g), __fsub_ru(a.x_hi[xi], g)));
        }
        v = warp_sum_rd(v);
        acc = __fadd_rd(acc, v);
    }
    if (lane == 0) a.lb_ibp[box] = acc;
}

template <bool TF> static size_t ibp_tc_smem()
{
    return 1024 + (size_t)kStages * kStageBytes + 5 * (size_t)kOpBytes + (size_t)IbpCfg<TF>::NB * 2 * 32 * 4;
}

bool ibp_tc_supported(const NetDesc &N, int max_smem)
{
    return N.ibp_ok && ibp_tc_smem<false>() <= (size_t)max_smem && ibp_tc_smem<true>() <= (size_t)max_smem;
}

template <bool TF> static cudaError_t launch_ibp_tc_(const BoundArgs &a, int num_sms, cudaStream_t st)
{
    if (a.n <= 0) return cudaSuccess;
    const size_t smem = ibp_tc_smem<TF>();
    cudaError_t e = cudaFuncSetAttribute(k_ibp_tc<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    constexpr int kNB = IbpCfg<TF>::NB;
    const int ntiles = (a.n + kNB - 1) / kNB;
    k_ibp_tc<TF><<<ntiles < num_sms ? ntiles : num_sms, (kEpiW + 2) * 32, smem, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess || !a.lb_ibp) return e;
    k_lb_from_boxes<<<(a.n + 7) / 8, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_ibp_tc(const BoundArgs &a, int num_sms, cudaStream_t st) { return launch_ibp_tc_<false>(a, num_sms, st); }

cudaError_t launch_ibp_tc_tf32(const BoundArgs &a, int num_sms, cudaStream_t st)
{
    return launch_ibp_tc_<true>(a, num_sms, st);
}

}  // namespace bab
