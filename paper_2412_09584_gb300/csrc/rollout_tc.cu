// rollout_tc.cu -- sampled search (Section 3.3) on tcgen05 tensor cores.
//
// A tile is M = 128 samples of one box (one sample per TMEM lane).  A CTA is
// persistent and runs NSLOT tiles at once, ping-ponging the tensor core
// between them:
//
//   warps 8s .. 8s+7 (slot s): the epilogue of slot s.  Thread r of warps
//     8s .. 8s+3 owns sample row r: it keeps the state x_t and the running
//     cost in registers, draws u_t (counter-based; the next step's while the
//     output layer runs), writes the input row [u_t|x_t|0] (fixed columns;
//     layer 1 of the weight image is permuted to match) to TMEM as the A
//     operand of layer 1, and after the last layer adds the residual and the
//     step cost.  After each hidden layer the warp pair of a lane quadrant
//     reads the FP32 accumulator row from TMEM 16 columns at a time (one half
//     of the columns each), adds the bias, applies ReLU and writes
//     the next layer's A operand back to TMEM (as BF16, or as a BF16 hi/lo
//     pair for the 3-term split).  No shared memory is written per layer.
//   warps 8*NSLOT + s: issue every layer's MMAs of slot s (M=128, N = layer
//     width, K = 16 per instruction), signalling completion on the slot's
//     mbarrier; the first of them allocates TMEM and loads the weight image
//     into shared memory once with the bulk copy engine.  With two slots the
//     issuers take turns, one layer-step each: left alone they fall into
//     step with each other, both epilogues then run while the tensor core
//     idles.
//
// Precision: SPLIT = 3 computes each product as a_hi b_hi + a_hi b_lo +
// a_lo b_hi with BF16 halves of the FP32 operands and FP32 accumulation
// (about 2^-16 relative per product); SPLIT = 1 uses BF16 operands only.
// Samples are drawn exactly as in the FP32 path (bit-identical u).
//
// Every mbarrier wait is bounded in time; on a time-out the kernel records
// BAB_ERR_TIMEOUT, stops issuing work, waits (bounded) for its MMAs, frees
// its TMEM and returns.
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include "bab_internal.cuh"
#include "kernels.cuh"
#include "select.cuh"
#include "tc_ptx.cuh"

namespace bab {

namespace {

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s per wait
constexpr int kEpiWarps = 8;                      // epilogue warps per tile slot (2 per TMEM lane quadrant)
constexpr int kMaxStages = 8;                     // weight ring buffers when the image is streamed

// (a, b) -> packed BF16 pair, a in the low half, round to nearest even
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

// hi = bf16(v), lo = bf16(v - hi), for a pair of values
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo)
{
    hi = pack_bf16x2(a, b);
    lo = pack_bf16x2(a - __uint_as_float(hi << 16), b - __uint_as_float(hi & 0xFFFF0000u));
}

// (a.x + b.x, a.y + b.y) and (a.x - b.x, a.y - b.y), each rounded to nearest, as one paired FP32 instruction.
__device__ __forceinline__ float2 add2(float2 a, float2 b)
{
    unsigned long long x = *reinterpret_cast<unsigned long long *>(&a), y = *reinterpret_cast<unsigned long long *>(&b), z;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(z) : "l"(x), "l"(y));
    return *reinterpret_cast<float2 *>(&z);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    unsigned long long x = *reinterpret_cast<unsigned long long *>(&a), y = *reinterpret_cast<unsigned long long *>(&b), z;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(z) : "l"(x), "l"(y));
    return *reinterpret_cast<float2 *>(&z);
}

// The hidden-layer epilogue of a pair of accumulator columns z = (acc + bias) in one conversion per half:
// SPLIT = 1: hi = bf16_rn(ReLU(z)); SPLIT = 3: hi = bf16 of ReLU(z) rounded toward zero, so that the residual
// ReLU(z) - hi is never negative (and is z itself, negative, where z < 0), lo = bf16_rn(ReLU(residual)); hi + lo
// then carries ReLU(z) to 2^-15 relative.  Low halves hold the even column.
template <int SPLIT>
__device__ __forceinline__ void relu_split2(float2 z, uint32_t &hi, uint32_t &lo)
{
    if (SPLIT == 3) {
        asm("cvt.rz.relu.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(z.y), "f"(z.x));
        const float2 r = sub2(z, make_float2(__uint_as_float(hi << 16), __uint_as_float(hi & 0xFFFF0000u)));
        asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(r.y), "f"(r.x));
    } else {
        asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(z.y), "f"(z.x));
    }
}

__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t phase, volatile int *abort)
{
    bool ok = tc::mbar_wait(bar, phase, abort, kWaitLimitNs);
    return __all_sync(0xFFFFFFFFu, ok);
}

__device__ __forceinline__ void raise_abort(int *status, volatile int *abort)
{
    set_status(status, BAB_ERR_TIMEOUT);
    *abort = 1;
}

}  // namespace

// SX: registers holding the state (8, 16 or 32, at least s; the output
// layer is 16 wide for SX <= 16, else 32).  STREAM: the weight
// image does not fit in shared memory, or every tile needs its own problem's
// image; per slot a producer warp streams it, one K-atom (64 inputs of one
// layer, hi and lo halves) at a time, through the slot's ring of a.stages
// buffers in the order the slot's MMA issuer consumes them.  CEM: samples
// from the cross-entropy search's per-box normal (cem_sample) instead of
// uniform draws.  OBST: the pushing-with-obstacles state cost (the pusher
// position kept beside the state).  Each is a separate instance, so that the
// plain kernel carries none of their code.
template <int NSLOT, int SPLIT, int SX, bool STREAM, bool CEM, bool OBST>
__global__ void __launch_bounds__((NSLOT * (kEpiWarps + 1) + (STREAM ? NSLOT : 0)) * 32, 1) k_rollout_tc(RolloutArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    const NetDesc &N = a.net;
    uint8_t *wimg = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float *bias = reinterpret_cast<float *>(wimg + (STREAM ? (size_t)NSLOT * a.stages * a.stage_bytes : (size_t)a.tc_bytes));
    float *goal_s = bias + N.tc_bias_floats;
    float *x0_s = goal_s + SX;
    __shared__ uint64_t bar_w, bar_a[NSLOT], bar_d[NSLOT], bar_tok[NSLOT], bar_fin;
    __shared__ uint64_t bar_full[NSLOT * kMaxStages], bar_empty[NSLOT * kMaxStages];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mma_warp = NSLOT * kEpiWarps;
    const int L = N.L, s = N.s, k = N.k;
    volatile int *abort = &abort_flag;
    // BF16 with the image resident: each hidden layer's bias enters the accumulator through one more K = 16 MMA of
    // a constant A block [1, 1, 0, ...] (8 TMEM columns after the slot's A operand) against the layer's bias atom
    // (b_hi, b_lo), so the epilogue adds nothing
    constexpr bool BMMA = SPLIT == 1 && !STREAM;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        tc::mbar_init(&bar_w, 1);
        tc::mbar_init(&bar_fin, 1);
        for (int i = 0; i < NSLOT; ++i) {
            tc::mbar_init(&bar_a[i], kEpiWarps);
            tc::mbar_init(&bar_d[i], 1);
            tc::mbar_init(&bar_tok[i], 1);
        }
        for (int i = 0; i < NSLOT * kMaxStages; ++i) {
            tc::mbar_init(&bar_full[i], 1);
            tc::mbar_init(&bar_empty[i], 1);
        }
        tc::mbar_init_fence();
    }
    if (warp == mma_warp) tc::tmem_alloc(&tmem_base, a.tmem_cols);
    for (int i = threadIdx.x; i < N.tc_bias_floats; i += blockDim.x) bias[i] = a.tc_bias[i];
    for (int i = threadIdx.x; i < SX; i += blockDim.x) {
        goal_s[i] = i < s ? a.goal[i] : 0.f;
        x0_s[i] = i < s ? a.x0[i] : 0.f;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (!STREAM) {
        if (threadIdx.x == mma_warp * 32) {
            // the image's first tc_bytes (BF16 with bias MMAs: the hi halves, then the bias atoms from the end of
            // the image), in 32 KB copies
            tc::mbar_arrive_expect_tx(&bar_w, (uint32_t)a.tc_bytes);
            constexpr uint32_t kChunk = 32768;
            const uint32_t first = BMMA ? (uint32_t)N.tc_bytes_hi : (uint32_t)a.tc_bytes;
            for (uint32_t off = 0; off < first; off += kChunk)
                tc::bulk_g2s(wimg + off, a.tc_img + off, min(kChunk, first - off), &bar_w);
            if (BMMA)
                for (uint32_t off = 0; off < (uint32_t)N.tc_bbytes; off += kChunk)
                    tc::bulk_g2s(wimg + first + off, a.tc_img + N.tc_bbase + off, min(kChunk, (uint32_t)N.tc_bbytes - off),
                                 &bar_w);
        }
        if (warp < mma_warp + NSLOT && !warp_wait(&bar_w, 0, abort) && lane == 0) raise_abort(a.status, abort);
    }

    const int nlive = live_count(a.n, a.d_n);
    // tiles: a box with M >= 128 samples spans tpb tiles; smaller M packs bpt = 128 / M boxes into a tile
    const int bpt = a.M >= 128 ? 1 : 128 / a.M;
    const int tpb = a.M >= 128 ? (a.M + 127) / 128 : 1;
    const long long ntiles = bpt > 1 ? ((long long)nlive + bpt - 1) / bpt : (long long)nlive * tpb;
    const long long G = (long long)gridDim.x * NSLOT;
    // batched problems (streamed images only, one box per tile): each tile's problem, horizon
    const bool batched = a.batch.P > 1;
    auto tile_problem = [&](long long tile) {
        return row_problem(a.batch, bpt > 1 ? (int)(tile * bpt) : (int)(tile / tpb));
    };
    auto tile_H = [&](long long tile) { return problem_H(a.batch, tile_problem(tile), a.H); };
    const uint32_t tb = tmem_base;
    const int Dc = N.tc_dcols, Ac = N.tc_acols;
    const int slot_cols = Dc + (SPLIT == 3 ? 2 : 1) * Ac + (BMMA ? 8 : 0);
    // the output layer's split as two MMAs per K step, a_hi [b_hi; b_lo] (2 N_L wide) and a_lo b_hi, where the
    // 2 N_L accumulator columns fit: columns 0.. hold a_hi b_hi + a_lo b_hi, columns N_L.. hold a_hi b_lo
    const bool stacked = SPLIT == 3 && 2 * N.tc_N[L] <= Dc && 2 * N.tc_N[L] <= 256;

    if (warp < mma_warp) {
        // ------------------------------- epilogue -------------------------------
        // Slot `slot` has 8 warps; warps q and q + 4 share TMEM lane quadrant q
        // (rows 32q .. 32q + 31).  The primary warp (q < 4) owns the rows' state;
        // for hidden layers whose width is a multiple of 64 the two warps of a
        // quadrant split the columns.
        const int slot = warp / kEpiWarps, qw = warp % kEpiWarps, quad = qw & 3;
        const bool primary = qw < 4;
        const int r = 32 * quad + lane;
        const uint32_t lane_off = (uint32_t)(32 * quad) << 16;
        const uint32_t dcol = tb + lane_off + slot * slot_cols;
        const uint32_t acol_h = dcol + Dc, acol_l = acol_h + Ac;
        const int K1 = N.tc_K[1];
        uint32_t phD = 0;
        if (BMMA && primary) {
            // the constant A block of the bias MMAs (its two first BF16 elements 1), once per slot; the first
            // arrive on bar_a below orders it before every MMA
            const uint32_t ones[8] = {0x3F803F80u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
            tc::tmem_st8(acol_l, ones);
            tc::tmem_wait_st();
        }
        for (long long tile = blockIdx.x * NSLOT + slot; tile < ntiles && !*abort; tile += G) {
            int box, m;
            bool lane_ok;
            if (bpt > 1) {
                box = (int)(tile * bpt) + r / a.M;
                m = r % a.M;
                lane_ok = r < bpt * a.M && box < nlive;
                if (!lane_ok) box = (int)(tile * bpt);  // an idle lane computes on a valid box, result unused
            } else {
                box = (int)(tile / tpb);
                m = (int)(tile % tpb) * 128 + r;
                lane_ok = m < a.M;
            }
            const uint64_t hb = box_hash(a.seed, a.id[box]);
            const float *blo = a.lo + (size_t)box * a.d, *bhi = a.hi + (size_t)box * a.d;
            // the tile's problem: start, goal, biases, horizon, rho (shared memory holds problem 0's)
            const int pb = batched ? tile_problem(tile) : 0;
            const float *x0_p = batched ? a.x0 + (size_t)pb * s : x0_s;
            const float *goal_p = batched ? a.goal + (size_t)pb * s : goal_s;
            const float *bias_p = batched ? a.tc_bias + (size_t)pb * N.tc_bias_floats : bias;
            const int Hb = batched ? problem_H(a.batch, pb, a.H) : a.H;
            const float rho = batched ? problem_rho(a.batch, pb, a.rho) : a.rho;
            // the state (zero beyond s) and the actions of the coming step (zero beyond k)
            float x[SX], u[kTcU];
#pragma unroll
            for (int i = 0; i < SX; ++i) x[i] = i < s ? x0_p[i] : 0.f;
            auto draw_step = [&](int t) {
#pragma unroll
                for (int j = 0; j < kTcU; ++j) {
                    const int jj = t * k + j;
                    if (j >= k) {
                        u[j] = 0.f;
                    } else if (CEM) {
                        const size_t e = (size_t)box * a.d + jj;
                        u[j] = cem_sample(hb, (uint32_t)a.cem_it, (uint32_t)m, (uint32_t)jj, __ldg(a.cem_mu + e),
                                          __ldg(a.cem_sigma + e), __ldg(blo + jj), __ldg(bhi + jj));
                    } else {
                        u[j] = draw_sample(hb, (uint32_t)m, (uint32_t)jj, __ldg(blo + jj), __ldg(bhi + jj));
                    }
                }
            };
            if (primary && Hb > 0) draw_step(0);
            float cost = 0.f;
            float px = a.cost.p0x, py = a.cost.p0y;  // pusher position (obstacle cost)
            bool ok = true;
            for (int t = 0; t < Hb && ok; ++t) {
                if (primary) {
                    // layer-1 input row [u_t | x_t | 0] (fixed columns), K1 <= 64 BF16 values
#pragma unroll
                    for (int j = 0; j < kTcU; ++j)
                        if (j < k) cost = fmaf(rho * u[j], u[j], cost);
                    if (OBST) {
                        px = __fadd_rn(px, u[0]);
                        py = __fadd_rn(py, u[1]);
                    }
#pragma unroll
                    for (int c16 = 0; c16 < 4; ++c16) {
                        if (c16 * 16 >= K1) break;
                        uint32_t ph[8], pl[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            float v2[2];
#pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                const int i = c16 * 16 + 2 * q + e;
                                v2[e] = i < kTcU ? u[i] : (i - kTcU < SX ? x[i - kTcU] : 0.f);
                            }
                            if (SPLIT == 3) split2(v2[0], v2[1], ph[q], pl[q]);
                            else ph[q] = pack_bf16x2(v2[0], v2[1]);
                        }
                        tc::tmem_st8(acol_h + c16 * 8, ph);
                        if (SPLIT == 3) tc::tmem_st8(acol_l + c16 * 8, pl);
                    }
                    tc::tmem_wait_st();
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&bar_a[slot]);
                for (int l = 1; l <= L; ++l) {
                    if (!warp_wait(&bar_d[slot], phD, abort)) {
                        if (lane == 0) raise_abort(a.status, abort);
                        ok = false;
                        break;
                    }
                    phD ^= 1;
                    tc::fence_after_sync();
                    const float *bl = bias_p + N.tc_boff[l];
                    const int Nl = N.tc_N[l];
                    const bool split_cols = (Nl % 64 == 0);
                    int c_beg = 0, c_end = Nl;
                    if (split_cols) {
                        c_beg = primary ? 0 : Nl / 2;
                        c_end = c_beg + Nl / 2;
                    } else if (!primary) {
                        c_end = 0;
                    }
                    if (l == L) {
                        // network output: residual step and step cost (the primary warps own the rows)
                        if (primary) {
                            float dx[SX];
                            if (SPLIT == 3 && stacked && SX == 8) {
                                uint32_t v[8], w[8];
                                tc::tmem_ld8(dcol, v);
                                tc::tmem_ld8(dcol + N.tc_N[L], w);
                                tc::tmem_wait_ld();
#pragma unroll
                                for (int i = 0; i < 8; ++i) dx[i] = __uint_as_float(v[i]) + __uint_as_float(w[i]);
                            } else if (SPLIT == 3 && stacked) {
#pragma unroll
                                for (int c0 = 0; c0 < SX; c0 += 16) {
                                    uint32_t v[16], w[16];
                                    tc::tmem_ld16(dcol + c0, v);
                                    tc::tmem_ld16(dcol + N.tc_N[L] + c0, w);
                                    tc::tmem_wait_ld();
#pragma unroll
                                    for (int i = 0; i < 16; ++i)
                                        if (c0 + i < SX) dx[c0 + i] = __uint_as_float(v[i]) + __uint_as_float(w[i]);
                                }
                            } else if (SX <= 16) {
                                uint32_t v[16];
                                tc::tmem_ld16(dcol, v);
                                tc::tmem_wait_ld();
#pragma unroll
                                for (int i = 0; i < SX; ++i) dx[i] = __uint_as_float(v[i]);
                            } else {
                                uint32_t v[32];
                                tc::tmem_ld32(dcol, v);
                                tc::tmem_wait_ld();
#pragma unroll
                                for (int i = 0; i < SX; ++i) dx[i] = __uint_as_float(v[i % 32]);
                            }
                            float c = 0.f;
#pragma unroll
                            for (int i = 0; i < SX; ++i) {
                                if (i < s) {
                                    x[i] = x[i] + (dx[i] + bl[i]);
                                    const float e = x[i] - goal_p[i];
                                    c = fmaf(e, e, c);
                                }
                            }
                            if (OBST) c = obstacle_cost_f32(a.cost, t + 1, s, x, goal_p, px, py);
                            cost += c;
                        }
                    } else {
                        // 16 columns per TMEM round trip: two loads per wait spill at the 96-register cap with the
                        // bias additions or the hi/lo split, and measured slower for BF16 with the bias in the MMA
                        // (11.1 against 10.5 ms); four epilogue warps per tile with two 64-column waits per layer
                        // measured slower too: the conversions then run on half as many warps
                        constexpr int kCols = 16;
                        for (int c0 = c_beg; c0 < c_end; c0 += kCols) {
                            uint32_t v[kCols / 16][16];
#pragma unroll
                            for (int g = 0; g < kCols / 16; ++g)
                                if (c0 + 16 * g < c_end) tc::tmem_ld16(dcol + c0 + 16 * g, v[g]);
                            tc::tmem_wait_ld();
#pragma unroll
                            for (int g = 0; g < kCols / 16; ++g) {
                                if (c0 + 16 * g >= c_end) break;
                                const int cc = c0 + 16 * g;
                                const float4 *b4 = reinterpret_cast<const float4 *>(bl + cc);
                                uint32_t ph[8], pl[8];
#pragma unroll
                                for (int q = 0; q < 4; ++q) {
                                    float2 z01 = make_float2(__uint_as_float(v[g][4 * q + 0]), __uint_as_float(v[g][4 * q + 1]));
                                    float2 z23 = make_float2(__uint_as_float(v[g][4 * q + 2]), __uint_as_float(v[g][4 * q + 3]));
                                    if (!BMMA) {
                                        const float4 bb = b4[q];
                                        z01 = add2(z01, make_float2(bb.x, bb.y));
                                        z23 = add2(z23, make_float2(bb.z, bb.w));
                                    }
                                    relu_split2<SPLIT>(z01, ph[2 * q], pl[2 * q]);
                                    relu_split2<SPLIT>(z23, ph[2 * q + 1], pl[2 * q + 1]);
                                }
                                tc::tmem_st8(acol_h + cc / 2, ph);
                                if (SPLIT == 3) tc::tmem_st8(acol_l + cc / 2, pl);
                            }
                        }
                        tc::tmem_wait_st();
                        tc::fence_before_sync();
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(&bar_a[slot]);
                        // the next step's actions, drawn while the output layer runs
                        if (primary && l == L - 1 && t + 1 < Hb) draw_step(t + 1);
                    }
                }
            }
            if (!ok) break;
            if (primary) {
                if (a.costs && lane_ok) a.costs[(size_t)box * a.M + m] = cost;
                const unsigned long long key =
                    lane_ok ? (((unsigned long long)float_order(cost) << 32) | (unsigned)m) : ~0ull;
                if (bpt > 1) {
                    // lanes of several boxes: each folds its own sample in
                    if (lane_ok) atomicMin(&a.keys[box], key);
                } else {
                    // best (f, m) of the warp's 32 rows of one box
                    unsigned long long kb = key;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const unsigned long long other = __shfl_xor_sync(0xFFFFFFFFu, kb, o);
                        kb = other < kb ? other : kb;
                    }
                    if (lane == 0 && kb != ~0ull) atomicMin(&a.keys[box], kb);
                }
            }
        }
    } else if (warp < mma_warp + NSLOT && lane == 0) {
        // ---------------------- MMA issuer of slot (warp - mma_warp) ----------------------
        const int sl = warp - mma_warp;
        const long long gi = (long long)blockIdx.x * NSLOT + sl;
        // walk (tile, t, l) in the epilogue's order; a tile of horizon 0 has nothing to issue
        long long tile = gi;
        int Hb = tile < ntiles ? tile_H(tile) : 0, t = 0, l = 1;
        while (tile < ntiles && Hb == 0) {
            tile += G;
            Hb = tile < ntiles ? tile_H(tile) : 0;
        }
        uint32_t phA = 0, ncommit = 0, ring_it = 0;
        // two slots take the tensor core in turns, one layer-step each, so that one slot's epilogue runs while
        // the other's MMAs do; n_other: the other slot's layer-steps in this CTA
        long long n_other = 0;
        if (NSLOT == 2)
            for (long long tt = (long long)blockIdx.x * NSLOT + (1 - sl); tt < ntiles; tt += G)
                n_other += (long long)tile_H(tt) * L;
        const uint32_t dcol = tb + sl * slot_cols;
        const uint32_t ah = dcol + Dc, al = ah + Ac;
        while (tile < ntiles && !*abort) {
            if (!tc::mbar_wait(&bar_a[sl], phA, abort, kWaitLimitNs)) {
                raise_abort(a.status, abort);
                break;
            }
            phA ^= 1;
            if (NSLOT == 2) {
                // slot 0's step i + 1 follows slot 1's step i, which follows slot 0's step i
                const long long i = ncommit;
                bool w = true;
                if (sl == 0 && i >= 1 && i - 1 < n_other)
                    w = tc::mbar_wait(&bar_tok[1], (uint32_t)((i - 1) & 1), abort, kWaitLimitNs);
                else if (sl == 1 && i < n_other)
                    w = tc::mbar_wait(&bar_tok[0], (uint32_t)(i & 1), abort, kWaitLimitNs);
                if (!w) {
                    raise_abort(a.status, abort);
                    break;
                }
            }
            tc::fence_after_sync();
            bool passed = false;  // the turn handed to the other slot
            const int Kl = N.tc_K[l], Nl = N.tc_N[l];
            // the other slot may start once three quarters of this layer are issued
            const int kpass = (3 * (Kl / 16) + 3) / 4;
            const uint32_t idesc = tc::idesc_bf16_f32(128, Nl);
            if (!STREAM) {
                // operands stepped with 32-bit adds on precomputed descriptor words, four K steps (one 64-wide
                // K-atom) unrolled: the issuing thread's own instructions, not the tensor core, set the MMA rate
                const int nks = Kl / 16;
                const uint32_t atom = (uint32_t)Nl * 8u;  // one K-atom of the image in 16-byte units
                uint32_t qh = tc::desc_sw128_lo(tc::smem_u32(wimg + N.tc_hi[l]));
                uint32_t ql = tc::desc_sw128_lo(tc::smem_u32(wimg + N.tc_lo[l]));
                uint32_t th = ah, tl = al;
                if (SPLIT == 3 && stacked && l == L) {
                    // stacked atoms: 2 N_L rows each, hi rows first
                    uint32_t qm = tc::desc_sw128_lo(tc::smem_u32(wimg + N.tc_mg));
                    const uint32_t idesc2 = tc::idesc_bf16_f32(128, 2 * Nl);
                    for (int ks0 = 0; ks0 < nks; ks0 += 4, qh += atom, qm += 2u * atom, th += 32u, tl += 32u) {
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            if (ks0 + kk >= nks) break;
                            tc::mma_ts(dcol, th + 8u * kk, tc::desc_join(qm + 2u * kk), idesc2, ks0 + kk > 0 ? 1u : 0u);
                            tc::mma_ts(dcol, tl + 8u * kk, tc::desc_join(qh + 2u * kk), idesc, 1u);
                            if (NSLOT == 2 && ks0 + kk + 1 == kpass) {
                                tc::mbar_arrive(&bar_tok[sl]);
                                passed = true;
                            }
                        }
                    }
                } else {
                for (int ks0 = 0; ks0 < nks; ks0 += 4, qh += atom, ql += atom, th += 32u, tl += 32u) {
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        if (ks0 + kk >= nks) break;
                        const uint64_t dh = tc::desc_join(qh + 2u * kk);
                        tc::mma_ts(dcol, th + 8u * kk, dh, idesc, ks0 + kk > 0 ? 1u : 0u);
                        if (SPLIT == 3) {
                            tc::mma_ts(dcol, th + 8u * kk, tc::desc_join(ql + 2u * kk), idesc, 1u);
                            tc::mma_ts(dcol, tl + 8u * kk, dh, idesc, 1u);
                        }
                        if (NSLOT == 2 && ks0 + kk + 1 == kpass) {
                            tc::mbar_arrive(&bar_tok[sl]);
                            passed = true;
                        }
                    }
                }
                // the bias: the constant block [1, 1, 0, ...] against the layer's (b_hi, b_lo) atom
                if (BMMA && l < L)
                    tc::mma_ts(dcol, al, tc::desc_join(tc::desc_sw128_lo(tc::smem_u32(wimg + N.tc_bytes_hi + N.tc_bb[l]))),
                               idesc, 1u);
                }
            } else {
                // one K-atom (64 inputs; hi, then lo for the split) per ring buffer
                bool ok = true;
                for (int at = 0; at < (Kl + 63) / 64; ++at, ++ring_it) {
                    const uint32_t st = ring_it % (uint32_t)a.stages, ph = (ring_it / (uint32_t)a.stages) & 1u;
                    uint64_t *full = bar_full + sl * kMaxStages, *empty = bar_empty + sl * kMaxStages;
                    if (!tc::mbar_wait(&full[st], ph, abort, kWaitLimitNs)) {
                        raise_abort(a.status, abort);
                        ok = false;
                        break;
                    }
                    const uint32_t qh = tc::desc_sw128_lo(tc::smem_u32(wimg + ((size_t)sl * a.stages + st) * a.stage_bytes));
                    const uint32_t ql = qh + (uint32_t)Nl * 8u;  // the lo half follows the hi half in the buffer
                    const uint32_t th = ah + 32u * at, tl = al + 32u * at;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const int ks = 4 * at + kk;
                        if (ks >= Kl / 16) break;
                        const uint64_t dh = tc::desc_join(qh + 2u * kk);
                        if (SPLIT == 3 && stacked && l == L) {
                            // the buffer holds the atom's hi rows, then its lo rows: already stacked
                            tc::mma_ts(dcol, th + 8u * kk, dh, tc::idesc_bf16_f32(128, 2 * Nl), ks > 0 ? 1u : 0u);
                            tc::mma_ts(dcol, tl + 8u * kk, dh, idesc, 1u);
                        } else {
                            tc::mma_ts(dcol, th + 8u * kk, dh, idesc, ks > 0 ? 1u : 0u);
                            if (SPLIT == 3) {
                                tc::mma_ts(dcol, th + 8u * kk, tc::desc_join(ql + 2u * kk), idesc, 1u);
                                tc::mma_ts(dcol, tl + 8u * kk, dh, idesc, 1u);
                            }
                        }
                        if (NSLOT == 2 && ks + 1 == kpass) {
                            tc::mbar_arrive(&bar_tok[sl]);
                            passed = true;
                        }
                    }
                    tc::mma_commit(&empty[st]);  // the buffer is free once these MMAs have read it
                }
                if (!ok) break;
            }
            tc::mma_commit(&bar_d[sl]);
            if (NSLOT == 2 && !passed) tc::mbar_arrive(&bar_tok[sl]);
            ++ncommit;
            if (++l > L) {
                l = 1;
                if (++t >= Hb) {
                    t = 0;
                    do {
                        tile += G;
                        Hb = tile < ntiles ? tile_H(tile) : 0;
                    } while (tile < ntiles && Hb == 0);
                }
            }
        }
        if (*abort) {
            // let every issued MMA finish before the TMEM and the ring are released
            volatile int never = 0;
            tc::mma_commit(&bar_fin);
            tc::mbar_wait(&bar_fin, 0, &never, kWaitLimitNs);
        }
    } else if (STREAM && warp >= mma_warp + NSLOT && lane == 0) {
        // ------------------- producer of slot ps: the weight atoms in that issuer's order -------------------
        const int ps = warp - mma_warp - NSLOT;
        uint64_t *full = bar_full + ps * kMaxStages, *empty = bar_empty + ps * kMaxStages;
        uint8_t *ring = wimg + (size_t)ps * a.stages * a.stage_bytes;
        uint32_t it = 0;
        bool ok = true;
        for (long long tile = (long long)blockIdx.x * NSLOT + ps; tile < ntiles && ok && !*abort; tile += G) {
          const int Hb = tile_H(tile);
          const uint8_t *img = a.tc_img + (batched ? (size_t)tile_problem(tile) * a.tc_img_stride : 0);
          for (int t = 0; t < Hb && ok && !*abort; ++t) {
            for (int l = 1; l <= L && ok; ++l) {
                const int Kl = N.tc_K[l], Nl = N.tc_N[l];
                const uint32_t atom = (uint32_t)Nl * 128u;
                for (int at = 0; at < (Kl + 63) / 64; ++at, ++it) {
                    const uint32_t st = it % (uint32_t)a.stages, ph = (it / (uint32_t)a.stages) & 1u;
                    if (!tc::mbar_wait(&empty[st], ph ^ 1u, abort, kWaitLimitNs)) {
                        raise_abort(a.status, abort);
                        ok = false;
                        break;
                    }
                    uint8_t *dst = ring + (size_t)st * a.stage_bytes;
                    tc::mbar_arrive_expect_tx(&full[st], (SPLIT == 3 ? 2u : 1u) * atom);
                    tc::bulk_g2s(dst, img + N.tc_hi[l] + (size_t)at * atom, atom, &full[st]);
                    if (SPLIT == 3) tc::bulk_g2s(dst + atom, img + N.tc_lo[l] + (size_t)at * atom, atom, &full[st]);
                }
            }
          }
        }
        // copies still in flight must land before the shared memory is released
        volatile int never = 0;
        const uint32_t inflight = it < (uint32_t)a.stages ? it : (uint32_t)a.stages;
        for (uint32_t j = 0; j < inflight; ++j) {
            const uint32_t i2 = it - 1 - j, st = i2 % (uint32_t)a.stages;
            tc::mbar_wait(&full[st], (i2 / (uint32_t)a.stages) & 1u, &never, kWaitLimitNs);
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
// Fused-step tensor-core rollout: BF16, the image resident in shared memory, uniform samples, squared-distance cost,
// at least two hidden layers.  With x_{t+1} = x_t + W_L a_{L-1} + b_L, the first layer of step t + 1 is
//
//   z1_{t+1} = (W1x W_L) a_{L-1} + W1x x_t + W1u u_{t+1} + (b1 + W1x b_L),
//
// so one product over the row [a_{L-1} | u_{t+1} x_t] against the fused image (NetDesc::tc_fbase) gives z1_{t+1}
// in accumulator columns 0 .. tc_N[1] - 1 and the step's output W_L a_{L-1} in the tc_N[L] columns after them.
// A time step is then L - 1 layer steps (layers 2 .. L-1 and the fused one) instead of L: one MMA / epilogue
// hand-off fewer per step on each slot's chain; layer 1 of step 0 runs on its own.  Warp roles, the two slots'
// turns, the bias MMAs and the bounded waits are those of k_rollout_tc.  The A region of a slot holds the layer
// input in columns 0 .. tc_K[L] / 2 - 1 and the input row [u | x] after it; the constant block of the bias MMAs
// follows the region.
template <int NSLOT, int SX>
__global__ void __launch_bounds__(NSLOT * (kEpiWarps + 1) * 32, 1) k_rollout_tcf(RolloutArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    const NetDesc &N = a.net;
    uint8_t *wimg = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float *bias = reinterpret_cast<float *>(wimg + (size_t)a.tc_bytes);
    float *goal_s = bias + N.tc_bias_floats;
    float *x0_s = goal_s + SX;
    __shared__ uint64_t bar_w, bar_a[NSLOT], bar_d[NSLOT], bar_tok[NSLOT], bar_fin;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mma_warp = NSLOT * kEpiWarps;
    const int L = N.L, s = N.s, k = N.k;
    volatile int *abort = &abort_flag;
    const int N1 = N.tc_N[1], NF = N.tc_N[1] + N.tc_N[L], KF = N.tc_K[L] + N.tc_K[1];
    const int Dc = N.tc_dcols > NF ? N.tc_dcols : NF, Ac = N.tc_acols > KF / 2 ? N.tc_acols : KF / 2;
    const int slot_cols = Dc + Ac + 8;
    const uint32_t rowc = (uint32_t)N.tc_K[L] / 2;  // TMEM column of the input row in the A region
    const uint32_t fimg = (uint32_t)(N.tc_bytes_hi + N.tc_bbytes);  // the fused image in shared memory

    if (threadIdx.x == 0) {
        abort_flag = 0;
        tc::mbar_init(&bar_w, 1);
        tc::mbar_init(&bar_fin, 1);
        for (int i = 0; i < NSLOT; ++i) {
            tc::mbar_init(&bar_a[i], kEpiWarps);
            tc::mbar_init(&bar_d[i], 1);
            tc::mbar_init(&bar_tok[i], 1);
        }
        tc::mbar_init_fence();
    }
    if (warp == mma_warp) tc::tmem_alloc(&tmem_base, a.tmem_cols);
    for (int i = threadIdx.x; i < N.tc_bias_floats; i += blockDim.x) bias[i] = a.tc_bias[i];
    for (int i = threadIdx.x; i < SX; i += blockDim.x) {
        goal_s[i] = i < s ? a.goal[i] : 0.f;
        x0_s[i] = i < s ? a.x0[i] : 0.f;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x == mma_warp * 32) {
        // the hi halves, the hidden layers' bias atoms, the fused image: three ranges, 32 KB copies
        tc::mbar_arrive_expect_tx(&bar_w, (uint32_t)a.tc_bytes);
        constexpr uint32_t kChunk = 32768;
        const uint32_t src[3] = {0u, (uint32_t)N.tc_bbase, (uint32_t)N.tc_fbase};
        const uint32_t len[3] = {(uint32_t)N.tc_bytes_hi, (uint32_t)N.tc_bbytes, (uint32_t)N.tc_fbytes};
        uint32_t dst = 0;
        for (int r = 0; r < 3; ++r) {
            for (uint32_t off = 0; off < len[r]; off += kChunk)
                tc::bulk_g2s(wimg + dst + off, a.tc_img + src[r] + off, min(kChunk, len[r] - off), &bar_w);
            dst += len[r];
        }
    }
    if (warp < mma_warp + NSLOT && !warp_wait(&bar_w, 0, abort) && lane == 0) raise_abort(a.status, abort);

    const int nlive = live_count(a.n, a.d_n);
    const int bpt = a.M >= 128 ? 1 : 128 / a.M;
    const int tpb = a.M >= 128 ? (a.M + 127) / 128 : 1;
    const long long ntiles = bpt > 1 ? ((long long)nlive + bpt - 1) / bpt : (long long)nlive * tpb;
    const long long G = (long long)gridDim.x * NSLOT;
    const uint32_t tb = tmem_base;

    if (warp < mma_warp) {
        // ------------------------------- epilogue -------------------------------
        const int slot = warp / kEpiWarps, qw = warp % kEpiWarps, quad = qw & 3;
        const bool primary = qw < 4;
        const int r = 32 * quad + lane;
        const uint32_t dcol = tb + ((uint32_t)(32 * quad) << 16) + slot * slot_cols;
        const uint32_t acol = dcol + Dc;
        const int K1 = N.tc_K[1];
        uint32_t phD = 0;
        if (primary) {
            // the constant A block of the bias MMAs, once per slot (ordered before every MMA by the first arrive)
            const uint32_t ones[8] = {0x3F803F80u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
            tc::tmem_st8(acol + Ac, ones);
            tc::tmem_wait_st();
        }
        // ReLU and BF16 conversion of accumulator columns [c_beg, c_end) (the bias came in by its MMA) into the A
        // region, 32 columns (two loads) per TMEM round trip (16 measured 8.29 against 8.18 ms); a width that is a
        // multiple of 64 is split between the quadrant's primary warp (the first pc columns) and its helper
        auto hidden = [&](int Nl, int pc) {
            const bool split_cols = (Nl % 64 == 0);
            int c_beg = 0, c_end = Nl;
            if (split_cols) {
                c_beg = primary ? 0 : pc;
                c_end = primary ? pc : Nl;
            } else if (!primary) {
                c_end = 0;
            }
            for (int c0 = c_beg; c0 < c_end; c0 += 32) {
                uint32_t v[16], w[16];
                tc::tmem_ld16(dcol + c0, v);
                tc::tmem_ld16(dcol + c0 + 16, w);
                tc::tmem_wait_ld();
                uint32_t ph[8], qh[8], unused;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    relu_split2<1>(make_float2(__uint_as_float(v[2 * q]), __uint_as_float(v[2 * q + 1])), ph[q], unused);
                    relu_split2<1>(make_float2(__uint_as_float(w[2 * q]), __uint_as_float(w[2 * q + 1])), qh[q], unused);
                }
                tc::tmem_st8(acol + c0 / 2, ph);
                tc::tmem_st8(acol + c0 / 2 + 8, qh);
            }
        };
        auto handoff = [&]() {
            tc::tmem_wait_st();
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&bar_a[slot]);
        };
        auto wait_d = [&]() -> bool {
            if (!warp_wait(&bar_d[slot], phD, abort)) {
                if (lane == 0) raise_abort(a.status, abort);
                return false;
            }
            phD ^= 1;
            tc::fence_after_sync();
            return true;
        };
        for (long long tile = blockIdx.x * NSLOT + slot; tile < ntiles && !*abort; tile += G) {
            int box, m;
            bool lane_ok;
            if (bpt > 1) {
                box = (int)(tile * bpt) + r / a.M;
                m = r % a.M;
                lane_ok = r < bpt * a.M && box < nlive;
                if (!lane_ok) box = (int)(tile * bpt);  // an idle lane computes on a valid box, result unused
            } else {
                box = (int)(tile / tpb);
                m = (int)(tile % tpb) * 128 + r;
                lane_ok = m < a.M;
            }
            const uint64_t hb = box_hash(a.seed, a.id[box]);
            const float *blo = a.lo + (size_t)box * a.d, *bhi = a.hi + (size_t)box * a.d;
            const int Hb = a.H;
            const float rho = a.rho;
            float x[SX], u[kTcU];
#pragma unroll
            for (int i = 0; i < SX; ++i) x[i] = i < s ? x0_s[i] : 0.f;
            auto draw_step = [&](int t) {
#pragma unroll
                for (int j = 0; j < kTcU; ++j) {
                    const int jj = t * k + j;
                    u[j] = j < k ? draw_sample(hb, (uint32_t)m, (uint32_t)jj, __ldg(blo + jj), __ldg(bhi + jj)) : 0.f;
                }
            };
            // the input row [u | x | 0] (u zero: the row of the last step feeds no further step)
            auto write_row = [&](bool with_u) {
#pragma unroll
                for (int c16 = 0; c16 < 4; ++c16) {
                    if (c16 * 16 >= K1) break;
                    uint32_t ph[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        float v2[2];
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const int i = c16 * 16 + 2 * q + e;
                            v2[e] = i < kTcU ? (with_u ? u[i] : 0.f) : (i - kTcU < SX ? x[i - kTcU] : 0.f);
                        }
                        ph[q] = pack_bf16x2(v2[0], v2[1]);
                    }
                    tc::tmem_st8(acol + rowc + c16 * 8, ph);
                }
            };
            auto rho_term = [&](float &c) {
#pragma unroll
                for (int j = 0; j < kTcU; ++j)
                    if (j < k) c = fmaf(rho * u[j], u[j], c);
            };
            float cost = 0.f;
            bool ok = Hb > 0;
            if (primary && ok) {
                draw_step(0);
                rho_term(cost);
                write_row(true);
            }
            if (ok) handoff();  // layer 1 of step 0 may start
            // z1_0
            if (ok && (ok = wait_d())) {
                hidden(N1, N1 / 2);
                handoff();
            }
            for (int t = 0; t < Hb && ok; ++t) {
                const bool more = t + 1 < Hb;
                if (primary && more) draw_step(t + 1);  // the next step's actions, drawn while layer 2 runs
                for (int l = 2; l <= L - 1 && ok; ++l) {
                    if (!(ok = wait_d())) break;
                    hidden(N.tc_N[l], N.tc_N[l] / 2);
                    if (l == L - 1 && primary) write_row(more);  // the fused product's input row [u_{t+1} | x_t]
                    handoff();
                }
                if (!ok || !(ok = wait_d())) break;
                // the fused product: the step's output (residual and cost), then z1_{t+1}
                if (primary) {
                    float dx[SX];
                    if (SX <= 8) {
                        uint32_t v[8];
                        tc::tmem_ld8(dcol + N1, v);
                        tc::tmem_wait_ld();
#pragma unroll
                        for (int i = 0; i < SX; ++i) dx[i] = __uint_as_float(v[i % 8]);
                    } else if (SX <= 16) {
                        uint32_t v[16];
                        tc::tmem_ld16(dcol + N1, v);
                        tc::tmem_wait_ld();
#pragma unroll
                        for (int i = 0; i < SX; ++i) dx[i] = __uint_as_float(v[i % 16]);
                    } else {
                        uint32_t v[32];
                        tc::tmem_ld32(dcol + N1, v);
                        tc::tmem_wait_ld();
#pragma unroll
                        for (int i = 0; i < SX; ++i) dx[i] = __uint_as_float(v[i % 32]);
                    }
                    const float *bl = bias + N.tc_boff[L];
                    float c = 0.f;
#pragma unroll
                    for (int i = 0; i < SX; ++i) {
                        if (i < s) {
                            x[i] = x[i] + (dx[i] + bl[i]);
                            const float e = x[i] - goal_s[i];
                            c = fmaf(e, e, c);
                        }
                    }
                    cost += c;
                    if (more) rho_term(cost);
                }
                if (more) {
                    hidden(N1, N1 / 2 >= 64 ? 32 : N1 / 2);  // the primary also ran the output stage: 32 columns
                    handoff();
                }
            }
            if (!ok) break;
            if (primary) {
                if (a.costs && lane_ok) a.costs[(size_t)box * a.M + m] = cost;
                const unsigned long long key =
                    lane_ok ? (((unsigned long long)float_order(cost) << 32) | (unsigned)m) : ~0ull;
                if (bpt > 1) {
                    if (lane_ok) atomicMin(&a.keys[box], key);
                } else {
                    unsigned long long kb = key;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const unsigned long long other = __shfl_xor_sync(0xFFFFFFFFu, kb, o);
                        kb = other < kb ? other : kb;
                    }
                    if (lane == 0 && kb != ~0ull) atomicMin(&a.keys[box], kb);
                }
            }
        }
    } else if (warp < mma_warp + NSLOT && lane == 0) {
        // ---------------------- MMA issuer of slot (warp - mma_warp) ----------------------
        // per tile: layer 1 of step 0 (phase 0), then per step layers 2 .. L-1 and the fused product
        const int sl = warp - mma_warp;
        const long long gi = (long long)blockIdx.x * NSLOT + sl;
        const long long per_tile = a.H > 0 ? 1 + (long long)a.H * (L - 1) : 0;
        long long left = gi < ntiles ? ((ntiles - 1 - gi) / G + 1) * per_tile : 0;
        long long n_other = 0;
        if (NSLOT == 2) {
            const long long go = (long long)blockIdx.x * NSLOT + (1 - sl);
            n_other = go < ntiles ? ((ntiles - 1 - go) / G + 1) * per_tile : 0;
        }
        uint32_t phA = 0, ncommit = 0;
        int ph = 0;  // phase within the tile: 0 layer 1; then 1 .. L-2 layers 2 .. L-1; L-1 the fused product
        const uint32_t dcol = tb + sl * slot_cols;
        const uint32_t acol = dcol + Dc, ones = acol + Ac;
        while (left > 0 && !*abort) {
            if (!tc::mbar_wait(&bar_a[sl], phA, abort, kWaitLimitNs)) {
                raise_abort(a.status, abort);
                break;
            }
            phA ^= 1;
            if (NSLOT == 2) {
                const long long i = ncommit;
                bool w = true;
                if (sl == 0 && i >= 1 && i - 1 < n_other)
                    w = tc::mbar_wait(&bar_tok[1], (uint32_t)((i - 1) & 1), abort, kWaitLimitNs);
                else if (sl == 1 && i < n_other)
                    w = tc::mbar_wait(&bar_tok[0], (uint32_t)(i & 1), abort, kWaitLimitNs);
                if (!w) {
                    raise_abort(a.status, abort);
                    break;
                }
            }
            tc::fence_after_sync();
            const bool fused = ph == L - 1;
            const int l = fused ? 0 : ph + 1;
            const int Kl = fused ? KF : N.tc_K[l], Nl = fused ? NF : N.tc_N[l];
            const uint32_t boff = fused ? fimg : (uint32_t)N.tc_hi[l];
            const uint32_t bboff = fused ? fimg + (uint32_t)N.tc_fb : (uint32_t)(N.tc_bytes_hi + N.tc_bb[l]);
            const uint32_t a0 = ph == 0 ? acol + rowc : acol;  // layer 1 of step 0 reads the input row
            const uint32_t idesc = tc::idesc_bf16_f32(128, Nl);
            // the other slot may start once half of this product is issued (a quarter, three quarters or all of it
            // measured 8.47, 8.43 and 8.45 ms against 8.30 for 4096 x 1024 x H = 20 rollouts with the re-score)
            const int nks = Kl / 16, kpass = (nks + 1) / 2;
            const uint32_t atom = (uint32_t)Nl * 8u;
            uint32_t q = tc::desc_sw128_lo(tc::smem_u32(wimg + boff));
            bool passed = false;
            for (int ks0 = 0; ks0 < nks; ks0 += 4, q += atom) {
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    if (ks0 + kk >= nks) break;
                    tc::mma_ts(dcol, a0 + 8u * (ks0 + kk), tc::desc_join(q + 2u * kk), idesc, ks0 + kk > 0 ? 1u : 0u);
                    if (NSLOT == 2 && ks0 + kk + 1 == kpass) {
                        tc::mbar_arrive(&bar_tok[sl]);
                        passed = true;
                    }
                }
            }
            // the bias: the constant block [1, 1, 0, ...] against the bias atom
            tc::mma_ts(dcol, ones, tc::desc_join(tc::desc_sw128_lo(tc::smem_u32(wimg + bboff))), idesc, 1u);
            tc::mma_commit(&bar_d[sl]);
            if (NSLOT == 2 && !passed) tc::mbar_arrive(&bar_tok[sl]);
            ++ncommit;
            --left;
            // next phase: after the fused product the step's layers 2 .. again (phase 1), a new tile after its last
            ph = ph == L - 1 ? 1 : ph + 1;
            if (per_tile > 0 && (ncommit % per_tile) == 0) ph = 0;
        }
        if (*abort) {
            volatile int never = 0;
            tc::mma_commit(&bar_fin);
            tc::mbar_wait(&bar_fin, 0, &never, kWaitLimitNs);
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

// BF16 mode: the threshold (order(ub), id) of the topk smallest BF16 upper bounds, and the list of the boxes it
// picks (in no particular order; each is re-scored on its own)
__global__ void __launch_bounds__(1024) k_topk_select(RolloutArgs a)
{
    __shared__ unsigned hist[256];
    __shared__ uint32_t sh_pk;
    __shared__ uint64_t sh_pid;
    __shared__ int sh_rem, sh_done, sh_cnt;
    const int n = live_count(a.n, a.d_n);
    const int K = a.topk < n ? a.topk : n;
    const Thresh T = radix_select(n, a.ub, a.id, [](int) { return true; }, K, hist, &sh_pk, &sh_pid, &sh_rem,
                                  &sh_done);
    if (threadIdx.x == 0) {
        a.topk_t[0] = T.key;
        a.topk_t[1] = T.id;
        a.topk_t[2] = T.none ? 1ull : 0ull;
        sh_cnt = 0;
    }
    __syncthreads();
    if (!T.none)
        for (int i = threadIdx.x; i < n; i += blockDim.x)
            if (le_thresh(float_order(a.ub[i]), a.id[i], T)) a.topk_list[atomicAdd(&sh_cnt, 1)] = i;
    __syncthreads();
    if (threadIdx.x == 0) a.topk_t[3] = (unsigned long long)sh_cnt;
}

// BF16 mode: the chosen sample of a box is re-scored in FP32 on CUDA cores (a
// CTA per box at a time), for every box or for the topk of smallest BF16 ub.
template <bool OBST>
__global__ void __launch_bounds__(256) k_rescore_fp32(RolloutArgs a)
{
    const NetDesc &N = a.net;
    const int nlive = live_count(a.n, a.d_n);
    Thresh T;
    if (a.topk > 0) {
        T.key = (uint32_t)a.topk_t[0];
        T.id = a.topk_t[1];
        T.none = a.topk_t[2] != 0;
    }
    __shared__ float act[2][kMaxWidth + 4];
    __shared__ float xs[kMaxWidth];
    __shared__ float f_sh;
    const int s = N.s, k = N.k, d = a.d;
    // boxes blockIdx.x, blockIdx.x + gridDim.x, ...: the grid is sized to the SMs, so that a top-k selection does
    // not pay for one CTA per box
    for (int box = blockIdx.x; box < nlive; box += gridDim.x) {
    if (a.topk > 0 && !le_thresh(float_order(a.ub[box]), a.id[box], T)) continue;
    const unsigned long long key = a.keys[box];
    const uint32_t m = (uint32_t)(key & 0xFFFFFFFFu);
    const uint64_t hb = box_hash(a.seed, a.id[box]);
    const int pb = row_problem(a.batch, box);
    const float *fwd = a.fwd + (size_t)pb * N.img_floats;
    const float *x0 = a.x0 + (size_t)pb * s, *goal = a.goal + (size_t)pb * s;
    const int Hb = problem_H(a.batch, pb, a.H);
    const float rho = problem_rho(a.batch, pb, a.rho);
    const float *blo = a.lo + (size_t)box * d, *bhi = a.hi + (size_t)box * d;
    for (int i = threadIdx.x; i < s; i += blockDim.x) xs[i] = x0[i];
    if (threadIdx.x == 0) f_sh = 0.f;
    float px = OBST ? a.cost.p0x : 0.f, py = OBST ? a.cost.p0y : 0.f;  // pusher position (thread 0)
    __syncthreads();
    for (int t = 0; t < Hb; ++t) {
        for (int c = threadIdx.x; c < s + k; c += blockDim.x)
            act[0][c] = c < s ? xs[c] : draw_sample(hb, m, (uint32_t)(t * k + c - s), blo[t * k + c - s], bhi[t * k + c - s]);
        __syncthreads();
        int cur = 0;
        for (int l = 1; l <= N.L; ++l) {
            const int no = N.dims[l], ni = N.dims[l - 1], Np = pad4(no);
            // forward image W_l^T [Kp][Np]: consecutive threads read consecutive outputs
            const float *Wt = fwd + N.fwd_w[l];
            const float *b = fwd + N.fwd_b[l];
            for (int q = threadIdx.x; q < no; q += blockDim.x) {
                float acc = b[q];
                // 16 inputs' weights loaded before their multiply-adds (which run in input order)
                for (int c0 = 0; c0 < ni; c0 += 16) {
                    float w[16];
#pragma unroll
                    for (int cc = 0; cc < 16; ++cc) w[cc] = c0 + cc < ni ? __ldg(Wt + (size_t)(c0 + cc) * Np + q) : 0.f;
#pragma unroll
                    for (int cc = 0; cc < 16; ++cc)
                        if (c0 + cc < ni) acc = fmaf(w[cc], act[cur][c0 + cc], acc);
                }
                act[cur ^ 1][q] = (l < N.L) ? fmaxf(acc, 0.f) : acc;
            }
            __syncthreads();
            cur ^= 1;
        }
        if (threadIdx.x == 0) {
            float f = f_sh;
            for (int j = 0; j < k; ++j) {
                const float u = draw_sample(hb, m, (uint32_t)(t * k + j), blo[t * k + j], bhi[t * k + j]);
                f = fmaf(rho * u, u, f);
                if (OBST && j == 0) px = __fadd_rn(px, u);
                if (OBST && j == 1) py = __fadd_rn(py, u);
            }
            float c = 0.f;
            for (int i = 0; i < s; ++i) {
                xs[i] = xs[i] + act[cur][i];
                const float e = xs[i] - goal[i];
                c = fmaf(e, e, c);
            }
            if (OBST) c = obstacle_cost_f32(a.cost, t + 1, s, xs, goal, px, py);
            f_sh = f + c;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) a.ub[box] = f_sh;  // best_u was written by the finalize kernel
    __syncthreads();  // before the next box reuses the shared arrays
    }
}

// BF16 mode, one problem, top-k re-score of a large network: the boxes of the top-k list, one per thread-block
// cluster at a time.  Each of the cluster's CTAs stages its share of each layer's columns of W_l^T (at most 32) in
// shared memory, computes those outputs one per thread (the same sums, in the same order, as k_rescore_fp32 and
// k_rescore_rows: from the bias over the inputs in order) and writes them into every CTA's shared memory
// (distributed shared memory); a cluster barrier closes each layer and each step's cost.  The list and its count
// are the same for every CTA, so all of them reach the same barriers.
constexpr int kRescoreCTAs = 8;
template <bool OBST>
__global__ void __launch_bounds__(256) k_rescore_cl(RolloutArgs a)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank(), ncta = (int)cluster.num_blocks();
    const int cl = (int)blockIdx.x / ncta, ncl = (int)gridDim.x / ncta;
    extern __shared__ float wsl[];  // [inputs][32]: this CTA's columns of W_l^T
    __shared__ float act[2][kMaxWidth + 4];
    __shared__ float xs[kMaxWidth];
    __shared__ float f_sh;
    const NetDesc &N = a.net;
    const int s = N.s, k = N.k, d = a.d;
    const int count = (int)a.topk_t[3];
    const float *fwd = a.fwd;
    const float *x0 = a.x0, *goal = a.goal;
    const float rho = a.rho;
    for (int e = cl; e < count; e += ncl) {
        const int box = a.topk_list[e];
        const unsigned long long key = a.keys[box];
        const uint32_t m = (uint32_t)(key & 0xFFFFFFFFu);
        const uint64_t hb = box_hash(a.seed, a.id[box]);
        const float *blo = a.lo + (size_t)box * d, *bhi = a.hi + (size_t)box * d;
        for (int i = threadIdx.x; i < s; i += blockDim.x) xs[i] = x0[i];
        if (threadIdx.x == 0) f_sh = 0.f;
        float px = OBST ? a.cost.p0x : 0.f, py = OBST ? a.cost.p0y : 0.f;  // pusher position (thread 0)
        __syncthreads();
        for (int t = 0; t < a.H; ++t) {
            for (int c = threadIdx.x; c < s + k; c += blockDim.x)
                act[0][c] = c < s ? xs[c]
                                  : draw_sample(hb, m, (uint32_t)(t * k + c - s), blo[t * k + c - s], bhi[t * k + c - s]);
            __syncthreads();
            int cur = 0;
            for (int l = 1; l <= N.L; ++l) {
                const int no = N.dims[l], ni = N.dims[l - 1], Np = pad4(no);
                const int chunk = (no + ncta - 1) / ncta, q0 = rank * chunk;  // chunk <= 32: widths <= 256
                const float *Wt = fwd + N.fwd_w[l];
                for (int i = threadIdx.x; i < ni * 32; i += blockDim.x) {
                    const int c = i >> 5, j = i & 31;
                    wsl[i] = (j < chunk && q0 + j < no) ? __ldg(Wt + (size_t)c * Np + q0 + j) : 0.f;
                }
                __syncthreads();
                const int q = q0 + (int)threadIdx.x;
                if ((int)threadIdx.x < chunk && q < no) {
                    float acc = fwd[N.fwd_b[l] + q];
                    for (int c = 0; c < ni; ++c) acc = fmaf(wsl[c * 32 + threadIdx.x], act[cur][c], acc);
                    const float v = (l < N.L) ? fmaxf(acc, 0.f) : acc;
                    for (int r2 = 0; r2 < ncta; ++r2) cluster.map_shared_rank(&act[cur ^ 1][0], r2)[q] = v;
                }
                cluster.sync();  // every CTA's copy of the layer output complete, the staged columns free again
                cur ^= 1;
            }
            if (threadIdx.x == 0) {
                float f = f_sh;
                for (int j = 0; j < k; ++j) {
                    const float u = draw_sample(hb, m, (uint32_t)(t * k + j), blo[t * k + j], bhi[t * k + j]);
                    f = fmaf(rho * u, u, f);
                    if (OBST && j == 0) px = __fadd_rn(px, u);
                    if (OBST && j == 1) py = __fadd_rn(py, u);
                }
                float c = 0.f;
                for (int i = 0; i < s; ++i) {
                    xs[i] = xs[i] + act[cur][i];
                    const float ee = xs[i] - goal[i];
                    c = fmaf(ee, ee, c);
                }
                if (OBST) c = obstacle_cost_f32(a.cost, t + 1, s, xs, goal, px, py);
                f_sh = f + c;
            }
            cluster.sync();  // the output read before the next step's first layer overwrites it
        }
        if (rank == 0 && threadIdx.x == 0) a.ub[box] = f_sh;  // best_u was written by the finalize kernel
    }
}

// BF16 mode, one problem, every box re-scored: the same FP32 re-score as k_rescore_fp32 for a tile of RR boxes
// at once (one row per box: its chosen sample), the layers as register-blocked FP32 products over the tile with
// the network image in shared memory (WSMEM) or read through L1, so that each weight read serves RR boxes.
constexpr int kRescoreRows = 28;  // 4096 boxes make 147 CTAs: one wave on 152 SMs
// 512 threads: a 128-wide layer of the tile is 448 register tiles of 2 rows x 4 columns, one per thread (256
// threads took two each, 0.49 ms for 4096 boxes)
constexpr int kRescoreThreads = 512;
static_assert(kRescoreRows <= kRescoreThreads, "one thread per row keeps that row's pusher position");
template <bool WSMEM, bool OBST>
__global__ void __launch_bounds__(kRescoreThreads) k_rescore_rows(RolloutArgs a)
{
    constexpr int RR = kRescoreRows, NT = kRescoreThreads;
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    const NetDesc &N = a.net;
    const int s = N.s, k = N.k, L = N.L, d = a.d, ld = N.maxw_p, s4 = pad4(s), Kp1 = pad4(s + k);
    const float *img = a.fwd;
    float *p = sm;
    if (WSMEM) {
        for (int i = threadIdx.x; i < N.img_floats / 4; i += NT) smem4[i] = reinterpret_cast<const float4 *>(a.fwd)[i];
        img = sm;
        p += N.img_floats;
    }
    float *act0 = p; p += RR * ld;
    float *act1 = p; p += RR * ld;
    float *xs = p; p += RR * s4;
    float *us = p; p += RR * pad4(k);
    float *fsum = p; p += RR;
    __shared__ uint64_t hbs[RR];
    __shared__ uint32_t ms[RR];
    __shared__ int take[RR];
    const int nlive = live_count(a.n, a.d_n);
    const int row0 = blockIdx.x * RR;
    if (row0 >= nlive) return;  // the whole tile is beyond the live rows (so below, nlive >= 1)
    for (int r = threadIdx.x; r < RR; r += NT) {
        const int box = row0 + r < nlive ? row0 + r : nlive - 1;  // idle rows recompute a valid box, unused
        take[r] = row0 + r < nlive;
        hbs[r] = box_hash(a.seed, a.id[box]);
        ms[r] = (uint32_t)(a.keys[box] & 0xFFFFFFFFull);
        fsum[r] = 0.f;
    }
    for (int i = threadIdx.x; i < RR * s; i += NT) xs[(i / s) * s4 + i % s] = a.x0[i % s];
    float px = OBST ? a.cost.p0x : 0.f, py = OBST ? a.cost.p0y : 0.f;  // pusher position of row threadIdx.x
    __syncthreads();
    for (int t = 0; t < a.H; ++t) {
        for (int i = threadIdx.x; i < RR * Kp1; i += NT) {
            const int r = i / Kp1, c = i % Kp1;
            const int box = row0 + r < nlive ? row0 + r : nlive - 1;
            float v = 0.f;
            if (c < s) {
                v = xs[r * s4 + c];
            } else if (c < s + k) {
                const int j = t * k + (c - s);
                v = draw_sample(hbs[r], ms[r], (uint32_t)j, a.lo[(size_t)box * d + j], a.hi[(size_t)box * d + j]);
                us[r * pad4(k) + (c - s)] = v;
            }
            act0[r * ld + c] = v;
        }
        __syncthreads();
        float *in = act0, *out = act1;
        for (int l = 1; l <= L; ++l) {
            dense_rows_auto<RR, NT>(in, ld, img + N.fwd_w[l], img + N.fwd_b[l], pad4(N.dims[l - 1]), pad4(N.dims[l]),
                                    out, ld, l < L);
            __syncthreads();
            float *tmp = in;
            in = out;
            out = tmp;
        }
        // the step's action cost (inputs in index order), then the state cost, as k_rescore_fp32 sums them
        for (int r = threadIdx.x; r < RR; r += NT) {
            float f = fsum[r];
            for (int j = 0; j < k; ++j) {
                const float u = us[r * pad4(k) + j];
                f = fmaf(a.rho * u, u, f);
            }
            float c = 0.f;
            for (int i = 0; i < s; ++i) {
                const float x = xs[r * s4 + i] + in[r * ld + i];
                xs[r * s4 + i] = x;
                const float e = x - a.goal[i];
                c = fmaf(e, e, c);
            }
            if (OBST) {
                px = __fadd_rn(px, us[r * pad4(k)]);
                py = __fadd_rn(py, us[r * pad4(k) + 1]);
                c = obstacle_cost_f32(a.cost, t + 1, s, xs + r * s4, a.goal, px, py);
            }
            fsum[r] = f + c;
        }
        __syncthreads();
    }
    for (int r = threadIdx.x; r < RR; r += NT)
        if (take[r]) a.ub[row0 + r] = fsum[r];
}

static cudaError_t launch_rescore(const RolloutArgs &a, cudaStream_t st)
{
    const NetDesc &N = a.net;
    long long macs = 0;
    for (int l = 1; l <= N.L; ++l) macs += (long long)N.dims[l] * N.dims[l - 1];
    if (a.batch.P <= 1 && a.topk > 0 && macs * a.H > 2000000) {
        // a large network's top k: a cluster of kRescoreCTAs per listed box
        cudaLaunchConfig_t cfg = {};
        const int ncl = a.topk < 64 ? a.topk : 64;
        cfg.gridDim = dim3((unsigned)(kRescoreCTAs * ncl));
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = (size_t)N.maxw_p * 32 * sizeof(float);
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = kRescoreCTAs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return a.cost.kind == 1 ? cudaLaunchKernelEx(&cfg, k_rescore_cl<true>, a)
                                : cudaLaunchKernelEx(&cfg, k_rescore_cl<false>, a);
    }
    if (a.batch.P > 1 || a.topk > 0) {
        // each box reads its own problem's image; with a top-k selection all but k boxes return at once
        int dev, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int grid = a.n < 2 * sms ? a.n : 2 * sms;
        if (a.cost.kind == 1) k_rescore_fp32<true><<<grid, 256, 0, st>>>(a);
        else k_rescore_fp32<false><<<grid, 256, 0, st>>>(a);
        return cudaGetLastError();
    }
    int dev, budget = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&budget, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t rest =
        ((size_t)2 * kRescoreRows * N.maxw_p + (size_t)kRescoreRows * (pad4(N.s) + pad4(N.k)) + kRescoreRows) * 4;
    const size_t img = (size_t)N.img_floats * 4;
    const bool wsmem = img + rest + 1024 <= (size_t)budget;
    const size_t smem = (wsmem ? img : 0) + rest;
    auto kern = a.cost.kind == 1 ? (wsmem ? k_rescore_rows<true, true> : k_rescore_rows<false, true>)
                                 : (wsmem ? k_rescore_rows<true, false> : k_rescore_rows<false, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(a.n + kRescoreRows - 1) / kRescoreRows, kRescoreThreads, smem, st>>>(a);
    return cudaGetLastError();
}

template <int NSLOT, int SPLIT, int SX, bool STREAM, bool CEM, bool OBST>
static cudaError_t launch_tc_variant(const RolloutArgs &a, int grid, size_t smem, cudaStream_t st)
{
    auto kern = k_rollout_tc<NSLOT, SPLIT, SX, STREAM, CEM, OBST>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, (NSLOT * (kEpiWarps + 1) + (STREAM ? NSLOT : 0)) * 32, smem, st>>>(a);
    return cudaGetLastError();
}

// Shared memory besides the weights: biases, goal and x0, and the 1024-byte alignment of the image.
static size_t rollout_tc_extra(const NetDesc &N)
{
    const int SP = N.tc_N[N.L];
    return ((size_t)N.tc_bias_floats + 2 * SP) * 4 + 1024;
}

// Bytes of one ring buffer: the largest K-atom (N_l x 64 BF16), hi and lo halves for the split.
static size_t rollout_tc_stage(const NetDesc &N, int split)
{
    size_t b = 0;
    for (int l = 1; l <= N.L; ++l) b = (size_t)N.tc_N[l] * 128 > b ? (size_t)N.tc_N[l] * 128 : b;
    return b * (split == 3 ? 2 : 1);
}

static bool rollout_tc_resident(const NetDesc &N, int split, int max_smem)
{
    const size_t img = split == 3 ? N.tc_bytes : (size_t)N.tc_bytes_hi + N.tc_bbytes;
    return img + rollout_tc_extra(N) + 1024 <= (size_t)max_smem;
}

bool rollout_tc_supported(const NetDesc &N, int split, int max_smem)
{
    if (!N.tc_ok || N.L < 2 || N.s > 32 || N.k > kTcU || N.tc_K[1] > 64) return false;
    // resident image, or at least two ring buffers
    return rollout_tc_resident(N, split, max_smem) ||
           2 * rollout_tc_stage(N, split) + rollout_tc_extra(N) + 1024 <= (size_t)max_smem;
}

// CEM: the cross-entropy sampling mode (a separate instance, so that the uniform kernel carries none of its code)
// OBST: the pushing-with-obstacles state cost (another instance for the same reason)
template <int SPLIT, int SX, bool CEM, bool OBST = false>
static cudaError_t launch_tc_shape(const RolloutArgs &a, int nslot, bool stream, int grid, size_t smem,
                                   cudaStream_t st)
{
    if (stream)
        return nslot == 2 ? launch_tc_variant<2, SPLIT, SX, true, CEM, OBST>(a, grid, smem, st)
                          : launch_tc_variant<1, SPLIT, SX, true, CEM, OBST>(a, grid, smem, st);
    return nslot == 2 ? launch_tc_variant<2, SPLIT, SX, false, CEM, OBST>(a, grid, smem, st)
                      : launch_tc_variant<1, SPLIT, SX, false, CEM, OBST>(a, grid, smem, st);
}

// The fused-step kernel (k_rollout_tcf): its image in shared memory, and the tensor-memory columns of one slot.
static size_t rollout_tcf_bytes(const NetDesc &N) { return (size_t)N.tc_bytes_hi + N.tc_bbytes + N.tc_fbytes; }
static int rollout_tcf_slot_cols(const NetDesc &N)
{
    const int NF = N.tc_N[1] + N.tc_N[N.L], KF = N.tc_K[N.L] + N.tc_K[1];
    return (N.tc_dcols > NF ? N.tc_dcols : NF) + (N.tc_acols > KF / 2 ? N.tc_acols : KF / 2) + 8;
}

template <int NSLOT, int SX>
static cudaError_t launch_tcf_variant(const RolloutArgs &a, int grid, size_t smem, cudaStream_t st)
{
    auto kern = k_rollout_tcf<NSLOT, SX>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, NSLOT * (kEpiWarps + 1) * 32, smem, st>>>(a);
    return cudaGetLastError();
}

// nslot_pref: 1 or 2 tiles per CTA, or -1 for two whenever both fit in tensor memory; the fused-step kernel where
// it applies (BF16, resident image, uniform samples, squared-distance cost), else layer by layer; 3 or 4: layer
// by layer with 1 or 2 tiles per CTA
cudaError_t launch_rollout_tc(RolloutArgs a, int split, int nslot_pref, int num_sms, cudaStream_t st)
{
    const NetDesc &N = a.net;
    if (a.n <= 0) return cudaSuccess;
    int dev, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const long long ntiles_all =
        a.M >= 128 ? (long long)a.n * ((a.M + 127) / 128) : ((long long)a.n + 128 / a.M - 1) / (128 / a.M);
    const bool fuse = split == 1 && a.batch.P <= 1 && a.cost.kind == 0 && !a.cem_mu && N.tc_fok &&
                      rollout_tcf_bytes(N) + rollout_tc_extra(N) + 1024 <= (size_t)max_smem &&
                      nslot_pref != 3 && nslot_pref != 4;
    if (fuse) {
        const int slot_cols = rollout_tcf_slot_cols(N);
        int nslot = nslot_pref == 1 || 2 * slot_cols > 512 ? 1 : 2;
        int cols = 32;
        while (cols < nslot * slot_cols) cols *= 2;
        if (cols > 512) return cudaErrorInvalidConfiguration;
        a.tmem_cols = (uint32_t)cols;
        a.tc_bytes = (int)rollout_tcf_bytes(N);
        a.stages = 0;
        const size_t smem = (size_t)a.tc_bytes + rollout_tc_extra(N);
        int grid = (int)((ntiles_all + nslot - 1) / nslot);
        grid = grid < num_sms ? grid : num_sms;
        k_fill_keys(a.keys, a.n, st);
        cudaError_t e;
        if (N.s <= 8) e = nslot == 2 ? launch_tcf_variant<2, 8>(a, grid, smem, st) : launch_tcf_variant<1, 8>(a, grid, smem, st);
        else if (N.s <= 16)
            e = nslot == 2 ? launch_tcf_variant<2, 16>(a, grid, smem, st) : launch_tcf_variant<1, 16>(a, grid, smem, st);
        else e = nslot == 2 ? launch_tcf_variant<2, 32>(a, grid, smem, st) : launch_tcf_variant<1, 32>(a, grid, smem, st);
        if (e != cudaSuccess) return e;
        launch_rollout_finalize(a, st);
        if (a.topk > 0) k_topk_select<<<1, 1024, 0, st>>>(a);
        e = launch_rescore(a, st);
        if (e != cudaSuccess) return e;
        if (a.inc_val) launch_incumbent(a, st);
        return cudaGetLastError();
    }
    if (nslot_pref == 3 || nslot_pref == 4) nslot_pref -= 2;
    // several problems: every tile streams its own problem's image
    const bool stream = a.batch.P > 1 || !rollout_tc_resident(N, split, max_smem);
    a.tc_img_stride = (size_t)N.tc_bytes + N.tc_bbytes + N.tc_fbytes;  // one problem's whole image
    // tensor memory: per slot the accumulator (widest layer) and the A operand(s) (widest input, 2 BF16 per column)
    // (plus, BF16 resident, the 8 columns of the bias MMAs' constant block)
    const int slot_cols = N.tc_dcols + (split == 3 ? 2 : 1) * N.tc_acols + (split == 1 && !stream ? 8 : 0);
    int nslot = (2 * slot_cols <= 512) ? 2 : 1;
    if (nslot_pref == 1 || nslot_pref == 2) nslot = nslot_pref;
    // a streamed image needs a ring of at least two buffers per slot
    if (stream && nslot == 2 &&
        2 * 2 * rollout_tc_stage(N, split) + rollout_tc_extra(N) + 1024 > (size_t)max_smem)
        nslot = 1;
    int cols = 32;
    while (cols < nslot * slot_cols) cols *= 2;
    if (cols > 512) return cudaErrorInvalidConfiguration;
    a.tmem_cols = (uint32_t)cols;
    if (split == 1) {
        // BF16 only: the hi halves and the bias atoms
        a.tc_bytes = N.tc_bytes_hi + N.tc_bbytes;
    }
    size_t smem;
    if (stream) {
        a.stage_bytes = (int)rollout_tc_stage(N, split);
        const size_t room = (size_t)max_smem - 1024 - rollout_tc_extra(N);
        int stages = (int)(room / ((size_t)nslot * a.stage_bytes));
        stages = stages > kMaxStages ? kMaxStages : stages;
        if (stages < 2) return cudaErrorInvalidConfiguration;
        a.stages = stages;
        smem = (size_t)nslot * stages * a.stage_bytes + rollout_tc_extra(N);
    } else {
        a.stages = 0;
        smem = (size_t)a.tc_bytes + rollout_tc_extra(N);
    }
    const long long ntiles = a.M >= 128 ? (long long)a.n * ((a.M + 127) / 128) : ((long long)a.n + 128 / a.M - 1) / (128 / a.M);
    int grid = (int)((ntiles + nslot - 1) / nslot);
    grid = grid < num_sms ? grid : num_sms;
    k_fill_keys(a.keys, a.n, st);
    cudaError_t e;
    // state registers: 8, 16 or 32 (the output layer is 16 wide up to 16 states, else 32)
    if (a.cost.kind == 1) {
        // the obstacle cost: uniform samples, at most 8 states
        if (a.cem_mu || N.s > 8) return cudaErrorInvalidValue;
        e = split == 3 ? launch_tc_shape<3, 8, false, true>(a, nslot, stream, grid, smem, st)
                       : launch_tc_shape<1, 8, false, true>(a, nslot, stream, grid, smem, st);
    } else if (a.cem_mu) {
        // the cross-entropy search runs the 3-term split only
        if (split != 3) return cudaErrorInvalidValue;
        if (N.s <= 8) e = launch_tc_shape<3, 8, true>(a, nslot, stream, grid, smem, st);
        else if (N.s <= 16) e = launch_tc_shape<3, 16, true>(a, nslot, stream, grid, smem, st);
        else e = launch_tc_shape<3, 32, true>(a, nslot, stream, grid, smem, st);
    } else if (N.s <= 8) {
        e = split == 3 ? launch_tc_shape<3, 8, false>(a, nslot, stream, grid, smem, st)
                       : launch_tc_shape<1, 8, false>(a, nslot, stream, grid, smem, st);
    } else if (N.s <= 16) {
        e = split == 3 ? launch_tc_shape<3, 16, false>(a, nslot, stream, grid, smem, st)
                       : launch_tc_shape<1, 16, false>(a, nslot, stream, grid, smem, st);
    } else {
        e = split == 3 ? launch_tc_shape<3, 32, false>(a, nslot, stream, grid, smem, st)
                       : launch_tc_shape<1, 32, false>(a, nslot, stream, grid, smem, st);
    }
    if (e != cudaSuccess) return e;
    if (a.cem_mu) return cudaGetLastError();  // the cross-entropy search keeps its own best (launch_cem_step)
    launch_rollout_finalize(a, st);  // ub and best_u from the packed minima
    if (split == 1) {
        if (a.topk > 0) k_topk_select<<<1, 1024, 0, st>>>(a);
        e = launch_rescore(a, st);
        if (e != cudaSuccess) return e;
    }
    if (a.inc_val) launch_incumbent(a, st);
    return cudaGetLastError();
}

}  // namespace bab
