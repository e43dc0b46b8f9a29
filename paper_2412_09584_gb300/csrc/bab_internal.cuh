// bab_internal.cuh -- device-side types and helpers shared by the libbab kernels.
//
// Network images.  The context keeps the dynamics network N (Section 3,
// Formulation; Appendix B.1, Definition) in three device layouts, every
// segment padded to a multiple of 4 floats (16 bytes) so that rows can be
// moved as float4:
//   raw : as loaded, W_l row-major [d_l][d_{l-1}] then b_l      (FP64 re-score)
//   fwd : per layer Wt_l [Kp][Np] (= W_l^T, zero padded), then b_l [Np]
//         (forward products a_l = W_l a_{l-1} + b_l over a tile of rows)
//   bwd : per layer W_l [Np][Kp] (zero padded), then b_l [Np]
//         (backward products A <- A W_l over a tile of rows)
// with Kp = pad4(d_{l-1}), Np = pad4(d_l).  The input layer's activation row
// is [x (s) | u (k) | 0 ...].
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bab.h"

namespace bab {

constexpr int kMaxLayers = BAB_MAX_LAYERS;
constexpr int kMaxWidth = BAB_MAX_WIDTH;

__host__ __device__ constexpr int pad4(int x) { return (x + 3) & ~3; }
// Tensor-core rollout input row: the action u_t in columns 0 .. kTcU - 1 (zero padded), the state x_t from
// column kTcU on, so that both sit at fixed positions; layer 1 of the forward image is permuted to match.
constexpr int kTcU = 8;

struct NetDesc {
    int L, s, k, sumh, maxw_p;                // maxw_p = pad4(max width)
    int dims[kMaxLayers + 1];
    int hoff[kMaxLayers + 1];                 // offset of hidden layer l in the [sumh] vector
    int raw_w[kMaxLayers + 1], raw_b[kMaxLayers + 1];
    int fwd_w[kMaxLayers + 1], fwd_b[kMaxLayers + 1];
    int bwd_w[kMaxLayers + 1], bwd_b[kMaxLayers + 1];
    int img_floats;                           // floats in the fwd (= bwd) image
    int raw_floats;
    // tensor-core image: per layer the BF16 hi halves of W_l (N_l x K_l, 128-byte
    // swizzled K-major), all layers first, then the lo halves; N_l = pad16(d_l),
    // K_l = pad16(d_{l-1}); FP32 biases padded to N_l
    int tc_ok;
    int tc_K[kMaxLayers + 1], tc_N[kMaxLayers + 1];
    int tc_hi[kMaxLayers + 1], tc_lo[kMaxLayers + 1];  // byte offsets in the image
    int tc_mg;  // byte offset of the output layer stacked per K-atom as [hi rows; lo rows] (after the lo halves)
    // BF16 bias atoms of the hidden layers l < L: one K-atom of N_l rows whose row n holds b_hi[n], b_lo[n] (the
    // BF16 halves of b_l) at K 0 and 1, so that one K = 16 MMA against an A block of [1, 1, 0, ...] adds the bias
    // to the accumulator.  They follow everything else in the image (at tc_bbase, tc_bbytes long; tc_bb[l]
    // relative to it); the BF16 kernel copies them into shared memory right after the hi halves.
    int tc_bb[kMaxLayers + 1];
    int tc_bbase, tc_bbytes;
    // Fused step (BF16): the output layer of step t and layer 1 of step t + 1 as one product over the row
    // [a_{L-1} | u_{t+1} x_t] (K = tc_K[L] + tc_K[1]) with N = tc_N[1] + tc_N[L] rows: [W1x W_L | W1 (input-row
    // layout)] for z1_{t+1}, then [W_L | 0] for the step's output; its bias atom (b1 + W1x b_L, then 0) after it.
    // At tc_fbase in the image, tc_fbytes long (bias atom at tc_fb relative to tc_fbase); tc_fok: it applies.
    int tc_fbase, tc_fbytes, tc_fb, tc_fok;
    int tc_boff[kMaxLayers + 1];                       // float offsets in the bias vector
    int tc_bytes, tc_bytes_hi, tc_bias_floats;
    int tc_dcols, tc_acols;                            // TMEM columns: accumulator, A operand
    // backward tensor-core image: per layer B = W_l^T as pad16(d_{l-1}) rows of pad16(d_l)
    // (the product A' W_l over a tile of boxes), hi halves of all layers, then lo halves
    int tcb_K[kMaxLayers + 1], tcb_N[kMaxLayers + 1];
    int tcb_hi[kMaxLayers + 1], tcb_lo[kMaxLayers + 1];
    int tcb_bytes, tcb_dcols, tcb_acols;
    // rounding-error factors of the backward products, formed once on the host (FP64 is slow on the device):
    // gam[l] = gamma_fp32(pad4(d_l)) for an FP32 product over K = pad4(d_l) terms,
    // gam_tc[l] = gamma_split(tcb_K[l]) for a 3-term BF16 split product
    float gam[kMaxLayers + 1];
    float gam_tc[kMaxLayers + 1];
    // tensor-core interval image (k_ibp_tc): per layer l, per 128-row block mb of its outputs and 64-wide block
    // ka of its inputs, one 64 KB stage [W hi | W lo | |W| hi | |W| lo], each 128 rows x 128 bytes (swizzled
    // K-major, rows past d_l zero); ibp_mb[l], ibp_ka[l] the block counts, ibp_off[l] the layer's first stage;
    // gam_ibp[l] = gamma_split(pad16(d_{l-1})); ibp_ok: every width at most 256
    int ibp_ok, ibp_bytes;
    int ibp_mb[kMaxLayers + 1], ibp_ka[kMaxLayers + 1], ibp_off[kMaxLayers + 1];
    float gam_ibp[kMaxLayers + 1];
    // backward TF32 image (3-term TF32 split products): per layer l, K = tf_K[l] = d_l rounded up to 8, in blocks
    // of 32 (128 bytes a row); block kb at tf_off[l] + 2 kb tcb_N[l] 128 bytes: tcb_N[l] rows of the hi halves, then
    // as many of the lo halves (swizzled K-major); gam_tf[l] = gamma_tf32(tf_K[l])
    int tf_K[kMaxLayers + 1], tf_off[kMaxLayers + 1], tf_bytes;
    float gam_tf[kMaxLayers + 1];
};

__host__ __device__ constexpr int pad16(int x) { return (x + 15) & ~15; }
__host__ __device__ constexpr int pad8(int x) { return (x + 7) & ~7; }

// ---------------------------------------------------------------------------
// Counter-based sampling: SplitMix64 output function (Steele, Lea and Flood,
// OOPSLA 2014), chained over (seed, box id, sample index m, coordinate j).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__device__ __forceinline__ uint64_t box_hash(uint64_t seed, uint64_t id) { return splitmix64(seed ^ splitmix64(id)); }

// Identifier of child c (0: lower, 1: upper half) of box `id`: 2 id + c while id < 2^62 (the binary path from the
// root box, id 1, through 62 splits), deeper 2^62 + (splitmix64(2 id + c) >> 2): the path continues as a hash so
// that the search can go arbitrarily deep (two boxes then share an identifier with probability about 2^-62).
__device__ __forceinline__ uint64_t child_id(uint64_t id, int c)
{
    if (id < (1ull << 62)) return 2 * id + (uint64_t)c;
    return (1ull << 62) | (splitmix64(2 * id + (uint64_t)c) >> 2);
}

// u = lo + (hi - lo) * r in FP32, one rounding per operation (no contraction).
__device__ __forceinline__ float draw_sample(uint64_t hbox, uint32_t m, uint32_t j, float lo, float hi)
{
    uint64_t h = splitmix64(hbox ^ (((uint64_t)m << 32) | (uint64_t)j));
    float r = __fmul_rn(__ull2float_rn(h >> 40), 5.9604644775390625e-08f);  // 2^-24, exact
    return __fadd_rn(lo, __fmul_rn(__fsub_rn(hi, lo), r));
}

// The normal draw of the cross-entropy search for (box key hbox, iteration it, sample m, coordinate j): the
// Irwin-Hall sum of four 24-bit uniforms, z = (r0 + r1 + r2 + r3 - 2) sqrt(3) (mean 0, variance 1, |z| <= 2
// sqrt(3)); the uniforms come from a SplitMix64 chain of the box key plus a stream constant, the iteration,
// then (m << 32 | 4 j + c).  FP32 left to right, one rounding per operation.  Sample 0 of iteration 0 is the
// mean itself (z = 0).
__device__ __forceinline__ float cem_normal(uint64_t hbox, uint32_t it, uint32_t m, uint32_t j)
{
    if (it == 0 && m == 0) return 0.f;
    uint64_t h = splitmix64(hbox + 0x632BE59BD9B4E019ull);
    h = splitmix64(h ^ (uint64_t)it);
    float acc = 0.f;
#pragma unroll
    for (uint32_t c = 0; c < 4; ++c) {
        const uint64_t hc = splitmix64(h ^ (((uint64_t)m << 32) | (uint64_t)(4u * j + c)));
        acc = __fadd_rn(acc, __fmul_rn(__ull2float_rn(hc >> 40), 5.9604644775390625e-08f));
    }
    return __fmul_rn(__fsub_rn(acc, 2.f), 1.7320508f);
}

// The search sample: mu + sigma z clipped to [lo, hi], in FP32.
__device__ __forceinline__ float cem_sample(uint64_t hbox, uint32_t it, uint32_t m, uint32_t j, float mu, float sigma,
                                            float lo, float hi)
{
    const float v = __fadd_rn(mu, __fmul_rn(sigma, cem_normal(hbox, it, m, j)));
    return fminf(fmaxf(v, lo), hi);
}

// Natural logarithm of a positive normal float from basic operations only, each rounded once (no
// contraction): x = 2^e m, m in [sqrt(1/2), sqrt(2)), log x = e ln 2 + 2 atanh(z), z = (m - 1)/(m + 1), by the
// atanh series to z^13.  The same steps in any IEEE arithmetic give the same bits; the softmax pick-out relies
// on that to agree with other implementations.
__device__ __forceinline__ float log_det(float x)
{
    const uint32_t b = __float_as_uint(x);
    int e = (int)((b >> 23) & 0xFFu) - 127;
    float m = __uint_as_float((b & 0x007FFFFFu) | 0x3F800000u);
    if (m > 1.41421356f) {
        m = __fmul_rn(m, 0.5f);
        e += 1;
    }
    const float z = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float z2 = __fmul_rn(z, z);
    float pp = 0.0769230769f;                                 // 1/13
    pp = __fadd_rn(__fmul_rn(pp, z2), 0.0909090909f);        // 1/11
    pp = __fadd_rn(__fmul_rn(pp, z2), 0.111111111f);         // 1/9
    pp = __fadd_rn(__fmul_rn(pp, z2), 0.142857143f);         // 1/7
    pp = __fadd_rn(__fmul_rn(pp, z2), 0.2f);                 // 1/5
    pp = __fadd_rn(__fmul_rn(pp, z2), 0.333333333f);         // 1/3
    pp = __fadd_rn(__fmul_rn(pp, z2), 1.0f);
    float t = __fmul_rn(z, pp);
    t = __fadd_rn(t, t);
    return __fadd_rn(__fmul_rn(__int2float_rn(e), 0.693147181f), t);
}

// Race key of the softmax pick-out (Section 3.1, Eq. lf_pick): s / T + log(-log U) with s the min-max scaled
// lower bound and U in (0, 1) from SplitMix64 of (seed, id); the k smallest keys draw k candidates without
// replacement with probabilities proportional to exp(-s / T).
__device__ __forceinline__ float pick_key(float lb, float lb_min, float lb_max, float temperature, uint64_t seed,
                                          uint64_t id)
{
    const float span = __fsub_rn(lb_max, lb_min);
    const float sc = span > 0.f ? __fdiv_rn(__fsub_rn(lb, lb_min), span) : 0.f;
    const uint64_t h = splitmix64(seed ^ splitmix64(id));
    const float uu = __fmul_rn(__fadd_rn(__ull2float_rn(h >> 41), 0.5f), 1.1920928955078125e-07f);  // 2^-23
    const float E = -log_det(uu);
    return __fadd_rn(__fdiv_rn(sc, temperature), log_det(E));
}

// Order-preserving map of a float to uint32 (NaN canonicalised to the top).
__device__ __forceinline__ uint32_t float_order(float f)
{
    if (f != f) return 0xFFFFFFFFu;
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float float_unorder(uint32_t k)
{
    if (k == 0xFFFFFFFFu) return __int_as_float(0x7FC00000);
    uint32_t b = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
    return __uint_as_float(b);
}

// gamma_n = n u / (1 - n u), u = 2^-24: the classical bound on the relative
// error of an n-term FP32 sum or dot product in any order (Higham, "Accuracy
// and Stability of Numerical Algorithms", 2nd ed., Section 3.1), rounded up.
__host__ __device__ __forceinline__ float gamma_fp32(int n)
{
    const double u = 5.9604644775390625e-08;
    double g = n * u / (1.0 - n * u);
    return (float)(g * (1.0 + 1e-6));
}

// Error factor of one 3-term BF16 split product of K terms with FP32 accumulation: 3.1 * 2^-16 for the
// BF16 hi/lo representation of both operands and the dropped lo x lo term, plus gamma_K with unit 2^-23
// (allowing a truncating accumulator), rounded up.
__host__ __device__ __forceinline__ float gamma_split(int K)
{
    const double u = 1.1920928955078125e-07;  // 2^-23
    return (float)(3.1 * 1.52587890625e-05 + K * u / (1.0 - K * u)) * 1.000001f;
}

// The same bound for a 3-term TF32 split (11 significant bits per half, so each operand's representation error
// and the dropped lo x lo term are at most about 2^-22 of |a| |b| each).
__host__ __device__ __forceinline__ float gamma_tf32(int K)
{
    const double u = 1.1920928955078125e-07;  // 2^-23
    return (float)(3.1 * 2.384185791015625e-07 + K * u / (1.0 - K * u)) * 1.000001f;
}

__device__ __forceinline__ int live_count(int n, const int *d_n)
{
    if (!d_n) return n;
    int v = *d_n;
    return v < n ? (v < 0 ? 0 : v) : n;
}
// The live rows of a launch that covers rows off .. off + n - 1 of the caller's arrays (a call processed in
// chunks under a scratch limit): the device count minus the offset, clamped to [0, n].
__device__ __forceinline__ int live_count(int n, const int *d_n, int off)
{
    if (!d_n) return n;
    int v = *d_n - off;
    return v < n ? (v < 0 ? 0 : v) : n;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}
// Sum with every addition rounded up: an upper bound of the exact sum of
// nonnegative terms.
__device__ __forceinline__ float warp_sum_ru(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __fadd_ru(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    return v;
}
__device__ __forceinline__ float warp_sum_rd(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __fadd_rd(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    return v;
}

// min over s in [lo, hi] of s^2, rounded down.
__device__ __forceinline__ float sq_min_rd(float lo, float hi)
{
    if (lo > 0.f) return __fmul_rd(lo, lo);
    if (hi < 0.f) return __fmul_rd(hi, hi);
    return 0.f;
}

// Lemma 1 (Appendix B.1) with outward rounding: slope D and intercept c of
// the selected linear bound of ReLU on [zl, zu] for coefficient A (the lower
// bound where A >= 0, the upper where A < 0).  The upper chord is replaced by
// a line that lies above it on [zl, zu]: slope rounded up, intercept -D zl
// rounded up.
__device__ __forceinline__ void relax_select(float zl, float zu, float A, float alpha_j, bool has_alpha, float &D,
                                             float &c)
{
    if (zl >= 0.f) {
        D = 1.f;
        c = 0.f;
    } else if (zu <= 0.f) {
        D = 0.f;
        c = 0.f;
    } else if (A >= 0.f) {
        D = has_alpha ? alpha_j : (zu >= -zl ? 1.f : 0.f);
        c = 0.f;
    } else {
        D = __fdiv_ru(zu, __fsub_rd(zu, zl));
        c = __fmul_ru(D, -zl);
    }
}

// Device status codes written by kernels (sticky, first error wins).
__device__ __forceinline__ void set_status(int *status, int code)
{
    if (status) atomicCAS(status, 0, code);
}

}  // namespace bab
