// api.cu -- the extern "C" entry points of libbab (declared in include/bab.h):
// argument checks, the context (network images, scratch, device status), and
// the kernel launches of each call.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "bab_internal.cuh"
#include "ibp_tc.cuh"
#include "kernels.cuh"

using namespace bab;

struct bab_ctx {
    int device = 0;
    int num_sms = 1;
    int n_problems = 1;
    int max_smem = 0;
    NetDesc net{};
    float *d_raw = nullptr, *d_fwd = nullptr, *d_bwd = nullptr;
    uint8_t *d_tc = nullptr, *d_tcb = nullptr;
    uint8_t *d_ibp = nullptr;    // the tensor-core interval image, BF16 halves (problem 0)
    uint8_t *d_ibp_tf = nullptr; // the tensor-core interval image, TF32 halves (problem 0)
    uint8_t *d_tf = nullptr;     // the backward TF32 image (problem 0)
    int interval_precision = 0;  // bab_set_interval_precision: BAB_PREC_FP32 (0), BAB_PREC_BF16X3 or BAB_PREC_TF32X3
    float *d_tc_bias = nullptr;
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    int *d_status = nullptr;
    // launch variants chosen by bab_autotune (-1: built-in heuristic)
    int tune_rollout_fp32 = -1;
    int tune_alpha_fused = -1;  // -2: the unfused loop of bound, adjoint and Adam launches
    int tune_rollout_tc = -1;   // tiles per CTA (3, 4: 1 or 2 without the fused step)
    int tune_crown_tc = -1;     // 3, 4 feature-major, 0 staged, 1 or 2 tiles per CTA, -1 the first that applies
    int rescore_topk = 0;       // BF16 rollouts: FP32 re-score of the topk smallest ub (0: every box)
    size_t scratch_limit = 0;   // bab_set_scratch_limit: bound calls chunk their boxes to stay within it (0: none)
    CostDesc cost{};            // the state cost (bab_set_cost); kind 0 by default
    int cost_H = 0;             // horizon its weights cover
    float *d_cost_w = nullptr;  // its weights w_t on the device
    char err[512] = {0};
};

namespace {

uint16_t bf16_rn_host(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7FFFFFFFu) > 0x7F800000u) return (uint16_t)((u >> 16) | 0x40u);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
float bf16_to_f32_host(uint16_t h)
{
    uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// f rounded to TF32 (10 stored mantissa bits, to nearest, ties away from zero): add half a unit of the 13th bit
// to the magnitude, clear the 13 low bits (finite inputs)
float tf32_rna_host(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;
    std::memcpy(&f, &u, 4);
    return f;
}

// One BF16 element (row n, input kk) of a 128-byte swizzled K-major operand of Nr rows at byte offset base.
void put_bf16(std::vector<uint8_t> &img, size_t base, int Nr, int n, int kk, float v)
{
    const int kb = kk / 64, within = kk % 64;
    const size_t off = base + (size_t)kb * Nr * 128 + (size_t)n * 128 + (size_t)((((within * 2) / 16) ^ (n % 8)) * 16) +
                       (size_t)((within * 2) % 16);
    const uint16_t h = bf16_rn_host(v);
    std::memcpy(&img[off], &h, 2);
}

// The fused step's BF16 image (see NetDesc::tc_fbase): with x_{t+1} = x_t + W_L a + b_L,
//   z1_{t+1} = (W1x W_L) a + W1x x_t + W1u u_{t+1} + (b1 + W1x b_L),
// rows 0 .. d_1 - 1 over the row [a | input row of layer 1], rows tc_N[1] + i the step's output W_L a (its bias
// b_L is added in FP32 by the epilogue, as in the unfused kernel).  Products and sums in double, then BF16.
void build_fused_image(const NetDesc &N, const float *params, std::vector<uint8_t> &img)
{
    const int L = N.L, s = N.s, NF = N.tc_N[1] + N.tc_N[L], kin = N.dims[L - 1], ni1 = N.dims[0], d1 = N.dims[1];
    const float *W1 = params + N.raw_w[1], *b1 = params + N.raw_b[1];
    const float *WL = params + N.raw_w[L], *bL = params + N.raw_b[L];
    const size_t base = (size_t)N.tc_fbase;
    for (int n = 0; n < d1; ++n) {
        for (int kk = 0; kk < kin; ++kk) {
            double c = 0.0;
            for (int i = 0; i < s; ++i) c += (double)W1[(size_t)n * ni1 + i] * (double)WL[(size_t)i * kin + kk];
            put_bf16(img, base, NF, n, kk, (float)c);
        }
        for (int kk0 = 0; kk0 < ni1; ++kk0) {
            const int kk = kk0 < s ? kTcU + kk0 : kk0 - s;  // the input row: u_t first, then x_t
            put_bf16(img, base, NF, n, N.tc_K[L] + kk, W1[(size_t)n * ni1 + kk0]);
        }
        double b = (double)b1[n];
        for (int i = 0; i < s; ++i) b += (double)W1[(size_t)n * ni1 + i] * (double)bL[i];
        const uint16_t bh = bf16_rn_host((float)b);
        const uint16_t bl = bf16_rn_host((float)(b - (double)bf16_to_f32_host(bh)));
        const size_t offb = base + (size_t)N.tc_fb + (size_t)n * 128 + (size_t)((0 ^ (n % 8)) * 16);
        std::memcpy(&img[offb], &bh, 2);
        std::memcpy(&img[offb + 2], &bl, 2);
    }
    for (int i = 0; i < s; ++i)
        for (int kk = 0; kk < kin; ++kk) put_bf16(img, base, NF, N.tc_N[1] + i, kk, WL[(size_t)i * kin + kk]);
}

// The tensor-core interval image (see NetDesc::ibp_off): W_l as the A operand of the feature-major products
// (rows = the layer's outputs, K = its inputs in the network's own order), BF16 hi and lo halves of W and |W|.
void build_ibp_tc_image(NetDesc &N, const float *params, std::vector<uint8_t> &img)
{
    const int L = N.L;
    bool ok = N.tc_ok && N.s <= 32 && N.dims[0] <= 128;  // the state boxes and the first layer's inputs: one block
    for (int l = 0; l <= L; ++l) ok = ok && N.dims[l] <= 256;
    int off = 0;
    for (int l = 1; l <= L; ++l) {
        N.ibp_mb[l] = (N.dims[l] + 127) / 128;
        N.ibp_ka[l] = (pad16(N.dims[l - 1]) + 63) / 64;
        N.ibp_off[l] = off;
        off += N.ibp_mb[l] * N.ibp_ka[l] * 65536;
        N.gam_ibp[l] = gamma_split(pad16(N.dims[l - 1]));
    }
    N.ibp_ok = ok ? 1 : 0;
    N.ibp_bytes = ok ? off : 0;
    img.assign((size_t)N.ibp_bytes, 0);
    if (!ok) return;
    for (int l = 1; l <= L; ++l) {
        const int no = N.dims[l], ni = N.dims[l - 1];
        const float *W = params + N.raw_w[l];
        for (int n = 0; n < no; ++n)
            for (int kk = 0; kk < ni; ++kk) {
                const float w = W[(size_t)n * ni + kk], a = std::fabs(w);
                const int mb = n / 128, row = n % 128, ka = kk / 64, within = kk % 64;
                const size_t stage = (size_t)N.ibp_off[l] + ((size_t)mb * N.ibp_ka[l] + ka) * 65536;
                const size_t o = (size_t)row * 128 + (size_t)((((within * 2) / 16) ^ (row % 8)) * 16) + (size_t)((within * 2) % 16);
                const uint16_t wh = bf16_rn_host(w), wl = bf16_rn_host(w - bf16_to_f32_host(wh));
                const uint16_t ah = bf16_rn_host(a), al = bf16_rn_host(a - bf16_to_f32_host(ah));
                std::memcpy(&img[stage + o], &wh, 2);
                std::memcpy(&img[stage + 16384 + o], &wl, 2);
                std::memcpy(&img[stage + 32768 + o], &ah, 2);
                std::memcpy(&img[stage + 49152 + o], &al, 2);
            }
    }
}

// The TF32 interval image (layout in ibp_tc.cuh): the same four A operands as the BF16 one, as TF32 halves (each
// rounded to nearest, ties away), 32 inputs a 128-byte row.  Empty unless the BF16 one is built (N.ibp_ok).
void build_ibp_tf_image(const NetDesc &N, const float *params, std::vector<uint8_t> &img)
{
    img.clear();
    if (!N.ibp_ok) return;
    std::vector<size_t> off(N.L + 2, 0);
    for (int l = 1; l <= N.L; ++l) off[l + 1] = off[l] + (size_t)N.ibp_mb[l] * ibp_tf_ka(N.dims[l - 1]) * 65536;
    img.assign(off[N.L + 1], 0);
    for (int l = 1; l <= N.L; ++l) {
        const int no = N.dims[l], ni = N.dims[l - 1], nka = ibp_tf_ka(ni);
        const float *W = params + N.raw_w[l];
        for (int n = 0; n < no; ++n)
            for (int kk = 0; kk < ni; ++kk) {
                const float w = W[(size_t)n * ni + kk], a = std::fabs(w);
                const int mb = n / 128, row = n % 128, ka = kk / 32, within = kk % 32;
                const size_t stage = off[l] + ((size_t)mb * nka + ka) * 65536;
                const size_t o = (size_t)row * 128 + (size_t)((((within * 4) / 16) ^ (row % 8)) * 16) + (size_t)((within * 4) % 16);
                const float wh = tf32_rna_host(w), wl = tf32_rna_host(w - wh);
                const float ah = tf32_rna_host(a), al = tf32_rna_host(a - ah);
                std::memcpy(&img[stage + o], &wh, 4);
                std::memcpy(&img[stage + 16384 + o], &wl, 4);
                std::memcpy(&img[stage + 32768 + o], &ah, 4);
                std::memcpy(&img[stage + 49152 + o], &al, 4);
            }
    }
}

// Tensor-core layout of the network (see NetDesc) and its BF16 hi/lo image.
void build_tc_image(NetDesc &N, const float *params, std::vector<uint8_t> &img, std::vector<float> &bias)
{
    const int L = N.L;
    bool ok = N.s <= 32 && N.k <= kTcU && pad16(kTcU + N.s) <= 64;
    for (int l = 1; l < L; ++l) ok = ok && (N.dims[l] % 32 == 0);
    int hi = 0, dcols = 16, acols = 8, bo = 0;
    for (int l = 1; l <= L; ++l) {
        // layer 1 reads the input row [u_t (kTcU columns) | x_t]
        N.tc_K[l] = pad16(l == 1 ? kTcU + N.s : N.dims[l - 1]);
        N.tc_N[l] = pad16(N.dims[l]);
        N.tc_hi[l] = hi;
        hi += ((N.tc_K[l] + 63) / 64) * N.tc_N[l] * 128;
        N.tc_boff[l] = bo;
        bo += N.tc_N[l];
        dcols = N.tc_N[l] > dcols ? N.tc_N[l] : dcols;
        acols = N.tc_K[l] / 2 > acols ? N.tc_K[l] / 2 : acols;
    }
    for (int l = 1; l <= L; ++l) N.tc_lo[l] = hi + N.tc_hi[l];
    N.tc_bytes_hi = hi;
    N.tc_mg = 2 * hi;
    N.tc_bytes = 2 * hi + ((N.tc_K[L] + 63) / 64) * 2 * N.tc_N[L] * 128;
    // the hidden layers' bias atoms after all of that (tc_bytes, what the split kernels load, excludes them)
    int bb = 0;
    for (int l = 1; l < L; ++l) {
        N.tc_bb[l] = bb;
        bb += N.tc_N[l] * 128;
    }
    N.tc_bbase = N.tc_bytes;
    N.tc_bbytes = bb;
    N.tc_bias_floats = bo;
    N.tc_dcols = dcols;
    N.tc_acols = acols;
    N.tc_ok = ok ? 1 : 0;
    // the fused step's image after the bias atoms
    const int NF = N.tc_N[1] + N.tc_N[L], KF = N.tc_K[L] + N.tc_K[1];
    N.tc_fok = ok && L >= 3 && NF <= 256 ? 1 : 0;
    N.tc_fbase = N.tc_bbase + N.tc_bbytes;
    N.tc_fb = ((KF + 63) / 64) * NF * 128;
    N.tc_fbytes = N.tc_fok ? N.tc_fb + NF * 128 : 0;
    img.assign((size_t)N.tc_bytes + N.tc_bbytes + N.tc_fbytes, 0);
    bias.assign((size_t)bo, 0.f);
    for (int l = 1; l <= L; ++l) {
        const int no = N.dims[l], ni = N.dims[l - 1], Nl = N.tc_N[l];
        const float *W = params + N.raw_w[l], *b = params + N.raw_b[l];
        for (int n = 0; n < no; ++n) {
            bias[N.tc_boff[l] + n] = b[n];
            if (l < L) {
                // bias atom: K 0 and 1 of row n (chunk 0, at its swizzled position)
                const uint16_t bh = bf16_rn_host(b[n]);
                const uint16_t bl = bf16_rn_host(b[n] - bf16_to_f32_host(bh));
                const size_t offb = (size_t)N.tc_bbase + N.tc_bb[l] + (size_t)n * 128 + (size_t)((0 ^ (n % 8)) * 16);
                std::memcpy(&img[offb], &bh, 2);
                std::memcpy(&img[offb + 2], &bl, 2);
            }
            for (int kk0 = 0; kk0 < ni; ++kk0) {
                const float w = W[(size_t)n * ni + kk0];
                const uint16_t h = bf16_rn_host(w);
                const uint16_t lo = bf16_rn_host(w - bf16_to_f32_host(h));
                // column of input kk0 in the tensor-core row (layer 1: state after the action block)
                const int kk = l == 1 ? (kk0 < N.s ? kTcU + kk0 : kk0 - N.s) : kk0;
                const int kb = kk / 64, within = kk % 64;
                const size_t off = (size_t)kb * Nl * 128 + (size_t)n * 128 + (size_t)((((within * 2) / 16) ^ (n % 8)) * 16) +
                                   (size_t)((within * 2) % 16);
                std::memcpy(&img[N.tc_hi[l] + off], &h, 2);
                std::memcpy(&img[N.tc_lo[l] + off], &lo, 2);
                if (l == L) {
                    // stacked copy: K-atom kb holds rows n (hi) and N_L + n (lo); (N_L + n) % 8 = n % 8
                    const size_t offm = off + (size_t)kb * Nl * 128;
                    std::memcpy(&img[N.tc_mg + offm], &h, 2);
                    std::memcpy(&img[N.tc_mg + offm + (size_t)Nl * 128], &lo, 2);
                }
            }
        }
    }
    if (N.tc_fok) build_fused_image(N, params, img);
}

// Backward tensor-core image: B_l = W_l^T (rows n < d_{l-1}, K = d_l), BF16 hi then lo, 128-byte swizzled.
void build_tcb_image(NetDesc &N, const float *params, std::vector<uint8_t> &img)
{
    const int L = N.L;
    int hi = 0, dcols = 16, acols = 8;
    for (int l = 1; l <= L; ++l) {
        N.tcb_K[l] = pad16(N.dims[l]);
        N.tcb_N[l] = pad16(N.dims[l - 1]);
        N.tcb_hi[l] = hi;
        hi += ((N.tcb_K[l] + 63) / 64) * N.tcb_N[l] * 128;
        dcols = N.tcb_N[l] > dcols ? N.tcb_N[l] : dcols;
        acols = N.tcb_K[l] / 2 > acols ? N.tcb_K[l] / 2 : acols;
    }
    for (int l = 1; l <= L; ++l) {
        N.tcb_lo[l] = hi + N.tcb_hi[l];
        N.gam_tc[l] = gamma_split(N.tcb_K[l]);
    }
    N.tcb_bytes = 2 * hi;
    N.tcb_dcols = dcols;
    N.tcb_acols = acols;
    img.assign((size_t)N.tcb_bytes, 0);
    for (int l = 1; l <= L; ++l) {
        const int no = N.dims[l], ni = N.dims[l - 1], Nl = N.tcb_N[l];
        const float *W = params + N.raw_w[l];
        for (int n = 0; n < ni; ++n)
            for (int kk = 0; kk < no; ++kk) {
                const float w = W[(size_t)kk * ni + n];
                const uint16_t h = bf16_rn_host(w);
                const uint16_t lo = bf16_rn_host(w - bf16_to_f32_host(h));
                const int kb = kk / 64, within = kk % 64;
                const size_t off = (size_t)kb * Nl * 128 + (size_t)n * 128 +
                                   (size_t)((((within * 2) / 16) ^ (n % 8)) * 16) + (size_t)((within * 2) % 16);
                std::memcpy(&img[N.tcb_hi[l] + off], &h, 2);
                std::memcpy(&img[N.tcb_lo[l] + off], &lo, 2);
            }
    }
}

// Backward TF32 image: the operand of build_tcb_image with 32-bit elements, for 3-term TF32 split products.  Layer
// l: K = d_l rounded up to 8 in blocks of 32 (128 bytes a row); block kb holds tcb_N[l] rows of the hi halves, then
// as many rows of the lo halves (hi = tf32(w), lo = tf32(w - hi)), swizzled K-major.  Needs build_tcb_image first.
void build_tf_image(NetDesc &N, const float *params, std::vector<uint8_t> &img)
{
    const int L = N.L;
    int off = 0;
    for (int l = 1; l <= L; ++l) {
        N.tf_K[l] = pad8(N.dims[l]);
        N.tf_off[l] = off;
        N.gam_tf[l] = gamma_tf32(N.tf_K[l]);
        off += ((N.tf_K[l] + 31) / 32) * 2 * N.tcb_N[l] * 128;
    }
    N.tf_bytes = off;
    img.assign((size_t)off, 0);
    for (int l = 1; l <= L; ++l) {
        const int no = N.dims[l], ni = N.dims[l - 1], Nl = N.tcb_N[l];
        const float *W = params + N.raw_w[l];
        for (int n = 0; n < ni; ++n)
            for (int kk = 0; kk < no; ++kk) {
                const float w = W[(size_t)kk * ni + n];
                const float h = tf32_rna_host(w), lo = tf32_rna_host(w - h);
                const int kb = kk / 32, within = kk % 32;
                const size_t off2 = (size_t)N.tf_off[l] + (size_t)kb * 2 * Nl * 128 + (size_t)n * 128 +
                                    (size_t)((((within * 4) / 16) ^ (n % 8)) * 16) + (size_t)((within * 4) % 16);
                std::memcpy(&img[off2], &h, 4);
                std::memcpy(&img[off2 + (size_t)Nl * 128], &lo, 4);
            }
    }
}

int fail(bab_ctx *c, int code, const char *fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

int cuda_fail(bab_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, e == cudaErrorMemoryAllocation ? BAB_ERR_OOM : BAB_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

// Grow the context scratch to at least `bytes` (synchronises the device when it reallocates).
int ensure_scratch(bab_ctx *c, size_t bytes)
{
    if (bytes <= c->scratch_bytes) return BAB_OK;
    size_t want = bytes + bytes / 4 + (1u << 20);
    if (c->scratch) {
        cudaDeviceSynchronize();
        cudaFree(c->scratch);
        c->scratch = nullptr;
        c->scratch_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&c->scratch, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(c, e, "scratch allocation");
    }
    c->scratch_bytes = want;
    return BAB_OK;
}

struct Carver {
    char *base;
    size_t off = 0;
    template <typename T>
    T *take(size_t count)
    {
        off = (off + 255) & ~size_t(255);
        T *p = reinterpret_cast<T *>(base + off);
        off += count * sizeof(T);
        return p;
    }
};

size_t bound_scratch_bytes(const NetDesc &N, int n, int H, int d, bool alpha)
{
    size_t nh = (size_t)n * H * N.sumh, nx = (size_t)n * (H + 1) * N.s, ns = (size_t)n * H * (N.sumh + N.s);
    size_t f = 2 * nh + 2 * nx + ns + (alpha ? (2 * nh + (size_t)n * d + 2 * (size_t)n) : 0);
    return f * sizeof(float) + 16 * 256;
}

// Boxes per pass of a bound call whose scratch is `fixed` bytes plus `per_row` bytes a box: all n without a
// limit or when they fit it, else as many as fit (0 when not even one box does).  Every box is bounded
// independently, so consecutive passes give the same bits as one.
int chunk_rows(const bab_ctx *c, size_t fixed, size_t per_row, int n)
{
    if (c->scratch_limit == 0 || fixed + (size_t)n * per_row <= c->scratch_limit) return n;
    if (fixed + per_row > c->scratch_limit) return 0;
    const size_t r = (c->scratch_limit - fixed) / per_row;
    return r < (size_t)n ? (int)r : n;
}

int check_problem(bab_ctx *c, const float *x0, const float *goal, int H, float rho, const float *lo, const float *hi,
                  int n)
{
    if (!c) return BAB_ERR_INVALID_ARG;
    c->err[0] = 0;
    if (!x0 || !goal) return fail(c, BAB_ERR_INVALID_ARG, "x0 and goal are required");
    if (H < 1 || H > (1 << 20)) return fail(c, BAB_ERR_SHAPE, "horizon %d out of range", H);
    if (n < 0) return fail(c, BAB_ERR_SHAPE, "n = %d < 0", n);
    if (n > 0 && (!lo || !hi)) return fail(c, BAB_ERR_INVALID_ARG, "lo and hi are required");
    if (!(rho >= 0.f) || !std::isfinite(rho)) return fail(c, BAB_ERR_INVALID_ARG, "rho must be finite and >= 0");
    if (c->net.L < 1) return fail(c, BAB_ERR_INVALID_ARG, "the context holds no network (bab_context_create)");
    if (c->cost.kind != 0 && H > c->cost_H)
        return fail(c, BAB_ERR_INVALID_ARG, "the cost weights cover horizons up to %d (H = %d)", c->cost_H, H);
    long long d = (long long)c->net.k * H;
    if (d > (1 << 24)) return fail(c, BAB_ERR_SHAPE, "action dimension k*H too large");
    return BAB_OK;
}

// The paths without the obstacle cost refuse it.
int refuse_obstacles(bab_ctx *c, const char *what)
{
    if (c->cost.kind != 0) return fail(c, BAB_ERR_UNSUPPORTED, "%s does not support the obstacle cost", what);
    return BAB_OK;
}

// The tensor-core CROWN carries the obstacle cost when its backward image is resident in shared memory.
int check_tc_obstacles(bab_ctx *c, const char *what)
{
    if (c->cost.kind != 0 && !crown_tc_obstacles_supported(c->net, c->max_smem))
        return fail(c, BAB_ERR_UNSUPPORTED, "%s carries the obstacle cost only with its weights in shared memory", what);
    return BAB_OK;
}

BoundArgs make_bound_args(bab_ctx *c, const float *x0, const float *goal, int H, float rho, const float *lo,
                          const float *hi, int n, const int *d_n, int row0 = 0)
{
    BoundArgs a{};
    a.row0 = row0;
    a.cost = c->cost;
    a.net = c->net;
    a.fwd = c->d_fwd;
    a.bwd = c->d_bwd;
    a.x0 = x0;
    a.goal = goal;
    a.lo = lo;
    a.hi = hi;
    a.n = n;
    a.d_n = d_n;
    a.H = H;
    a.d = c->net.k * H;
    a.rho = rho;
    a.status = c->d_status;
    a.batch.P = 1;
    a.batch.Hmax = H;
    return a;
}

// IBP into the scratch (or the caller's arrays); fills the interval fields of `a`.
int run_ibp(bab_ctx *c, BoundArgs &a, Carver &cv, float *pre_lo, float *pre_hi, float *x_lo, float *x_hi,
            float *lb_ibp, cudaStream_t st)
{
    const NetDesc &N = c->net;
    size_t nh = (size_t)a.n * a.H * N.sumh, nx = (size_t)a.n * (a.H + 1) * N.s;
    a.pre_lo = pre_lo ? pre_lo : cv.take<float>(nh);
    a.pre_hi = pre_hi ? pre_hi : cv.take<float>(nh);
    a.x_lo = x_lo ? x_lo : cv.take<float>(nx);
    a.x_hi = x_hi ? x_hi : cv.take<float>(nx);
    a.S = cv.take<float>((size_t)a.n * a.H * (N.sumh + N.s));
    a.lb_ibp = lb_ibp;
    const bool tc = c->interval_precision != BAB_PREC_FP32 && a.batch.P <= 1 && a.cost.kind == 0;
    const bool tf = c->interval_precision == BAB_PREC_TF32X3;
    a.ibp_img = tf ? c->d_ibp_tf : c->d_ibp;
    cudaError_t e = !tc ? launch_ibp(a, c->num_sms, st)
                        : (tf ? launch_ibp_tc_tf32(a, c->num_sms, st) : launch_ibp_tc(a, c->num_sms, st));
    if (e != cudaSuccess) return cuda_fail(c, e, "interval bounds kernel");
    return BAB_OK;
}

}  // namespace

extern "C" {

int bab_version(void) { return 1 * 10000 + 0 * 100 + 0; }

}  // extern "C"

namespace {

// P problems of one architecture: params holds P packed parameter vectors back to back.  The tensor-core
// images are built for problem 0 only (the batched calls run on CUDA cores).
int load_impl(bab_ctx **out, int P, int n_layers, const int *dims, const float *params, int state_dim,
              int action_dim, unsigned flags)
{
    if (!out || !dims || !params) return BAB_ERR_INVALID_ARG;
    *out = nullptr;
    if (P < 1 || P > (1 << 20)) return BAB_ERR_SHAPE;
    if (flags != 0) return BAB_ERR_INVALID_ARG;
    if (n_layers < 1 || n_layers > kMaxLayers) return BAB_ERR_SHAPE;
    if (state_dim < 1 || action_dim < 1 || dims[0] != state_dim + action_dim || dims[n_layers] != state_dim)
        return BAB_ERR_SHAPE;
    for (int l = 0; l <= n_layers; ++l)
        if (dims[l] < 1 || dims[l] > kMaxWidth) return BAB_ERR_SHAPE;

    bab_ctx *c = new bab_ctx();
    c->n_problems = P;
    NetDesc &N = c->net;
    N.L = n_layers;
    N.s = state_dim;
    N.k = action_dim;
    int maxw = 0, h = 0, raw = 0, img = 0;
    for (int l = 0; l <= n_layers; ++l) {
        N.dims[l] = dims[l];
        maxw = dims[l] > maxw ? dims[l] : maxw;
    }
    N.maxw_p = pad4(maxw);
    for (int l = 1; l <= n_layers; ++l) {
        N.hoff[l] = h;
        if (l < n_layers) h += dims[l];
        N.raw_w[l] = raw;
        raw += dims[l] * dims[l - 1];
        N.raw_b[l] = raw;
        raw += dims[l];
        const int Kp = pad4(dims[l - 1]), Np = pad4(dims[l]);
        N.fwd_w[l] = N.bwd_w[l] = img;
        img += Kp * Np;
        N.fwd_b[l] = N.bwd_b[l] = img;
        img += Np;
    }
    N.sumh = h;
    N.raw_floats = raw;
    N.img_floats = img;
    for (int l = 1; l <= n_layers; ++l) N.gam[l] = gamma_fp32(pad4(dims[l]));
    for (size_t i = 0; i < (size_t)P * raw; ++i)
        if (!std::isfinite(params[i])) {
            delete c;
            return BAB_ERR_NUMERIC;
        }

    std::vector<float> fwd((size_t)P * img, 0.f), bwd((size_t)P * img, 0.f);
    for (int pr = 0; pr < P; ++pr) {
        const float *prm = params + (size_t)pr * raw;
        float *fw = fwd.data() + (size_t)pr * img, *bw = bwd.data() + (size_t)pr * img;
        for (int l = 1; l <= n_layers; ++l) {
            const int no = dims[l], ni = dims[l - 1], Kp = pad4(ni), Np = pad4(no);
            const float *W = prm + N.raw_w[l], *b = prm + N.raw_b[l];
            for (int q = 0; q < no; ++q)
                for (int p = 0; p < ni; ++p) {
                    fw[N.fwd_w[l] + p * Np + q] = W[q * ni + p];  // Wt [Kp][Np]
                    bw[N.bwd_w[l] + q * Kp + p] = W[q * ni + p];  // W  [Np][Kp]
                }
            for (int q = 0; q < no; ++q) fw[N.fwd_b[l] + q] = bw[N.bwd_b[l] + q] = b[q];
        }
    }
    // tensor-core forward images (BF16 hi / lo) of every problem, back to back; backward image of problem 0
    std::vector<uint8_t> tc_img;
    std::vector<float> tc_bias;
    for (int pr = 0; pr < P; ++pr) {
        std::vector<uint8_t> im;
        std::vector<float> bi;
        build_tc_image(N, params + (size_t)pr * raw, im, bi);
        tc_img.insert(tc_img.end(), im.begin(), im.end());
        tc_bias.insert(tc_bias.end(), bi.begin(), bi.end());
    }
    std::vector<uint8_t> tcb_img, ibp_img, ibp_tf_img, tf_img;
    build_tcb_image(N, params, tcb_img);
    build_tf_image(N, params, tf_img);
    build_ibp_tc_image(N, params, ibp_img);
    build_ibp_tf_image(N, params, ibp_tf_img);
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_tc, tc_img.size());
    if (e == cudaSuccess) e = cudaMalloc(&c->d_tcb, tcb_img.size());
    if (e == cudaSuccess) e = cudaMemcpy(c->d_tcb, tcb_img.data(), tcb_img.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_tf, tf_img.size());
    if (e == cudaSuccess) e = cudaMemcpy(c->d_tf, tf_img.data(), tf_img.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !ibp_img.empty()) e = cudaMalloc(&c->d_ibp, ibp_img.size());
    if (e == cudaSuccess && !ibp_img.empty())
        e = cudaMemcpy(c->d_ibp, ibp_img.data(), ibp_img.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !ibp_tf_img.empty()) e = cudaMalloc(&c->d_ibp_tf, ibp_tf_img.size());
    if (e == cudaSuccess && !ibp_tf_img.empty())
        e = cudaMemcpy(c->d_ibp_tf, ibp_tf_img.data(), ibp_tf_img.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_tc_bias, sizeof(float) * tc_bias.size());
    if (e == cudaSuccess) e = cudaMemcpy(c->d_tc, tc_img.data(), tc_img.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_tc_bias, tc_bias.data(), sizeof(float) * tc_bias.size(), cudaMemcpyHostToDevice);
    const size_t nraw = (size_t)P * raw, nimg = (size_t)P * img;
    if (e == cudaSuccess) e = cudaMalloc(&c->d_raw, sizeof(float) * nraw);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_fwd, sizeof(float) * nimg);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_bwd, sizeof(float) * nimg);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(c->d_raw, params, sizeof(float) * nraw, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_fwd, fwd.data(), sizeof(float) * nimg, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_bwd, bwd.data(), sizeof(float) * nimg, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int));
    if (e != cudaSuccess) {
        int code = e == cudaErrorMemoryAllocation ? BAB_ERR_OOM : BAB_ERR_CUDA;
        cudaGetLastError();
        bab_destroy(c);
        return code;
    }
    *out = c;
    return BAB_OK;
}

}  // namespace

extern "C" {

int bab_load_dynamics(bab_ctx **out, int n_layers, const int *dims, const float *params, int state_dim, int action_dim,
                      unsigned flags)
{
    return load_impl(out, 1, n_layers, dims, params, state_dim, action_dim, flags);
}

int bab_load_dynamics_batch(bab_ctx **out, int n_problems, int n_layers, const int *dims, const float *params,
                            int state_dim, int action_dim, unsigned flags)
{
    return load_impl(out, n_problems, n_layers, dims, params, state_dim, action_dim, flags);
}

int bab_set_cost(bab_ctx *c, int kind, int H, const float *w, float lambda, int n_obs, const float *obstacles,
                 const float *p0)
{
    if (!c) return BAB_ERR_INVALID_ARG;
    c->err[0] = 0;
    if (kind == BAB_COST_SQUARED) {
        c->cost = CostDesc{};
        return BAB_OK;
    }
    if (kind != BAB_COST_PUSHING_OBSTACLES) return fail(c, BAB_ERR_INVALID_ARG, "unknown cost kind %d", kind);
    if (c->net.L >= 1 && (c->net.k != 2 || c->net.s % 2 != 0 || c->net.s > 32))
        return fail(c, BAB_ERR_UNSUPPORTED, "the obstacle cost needs planar keypoints (s even, at most 32 states: its "
                                            "relaxation gives one warp lane to each coordinate) and a planar pusher (k = 2)");
    if (H < 1 || H > (1 << 20) || !w || !p0 || n_obs < 0 || n_obs > kMaxObstacles || (n_obs > 0 && !obstacles))
        return fail(c, BAB_ERR_INVALID_ARG, "bad horizon, weights, obstacles (at most %d) or pusher start", kMaxObstacles);
    if (!(lambda >= 0.f) || !std::isfinite(lambda)) return fail(c, BAB_ERR_INVALID_ARG, "lambda must be finite and >= 0");
    for (int t = 0; t < H; ++t)
        if (!(w[t] >= 0.f) || !std::isfinite(w[t])) return fail(c, BAB_ERR_INVALID_ARG, "weights must be finite and >= 0");
    float *dw = nullptr;
    cudaError_t e = cudaMalloc(&dw, sizeof(float) * H);
    if (e == cudaSuccess) e = cudaMemcpy(dw, w, sizeof(float) * H, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(dw);
        return cuda_fail(c, e, "cost weights");
    }
    cudaFree(c->d_cost_w);
    c->d_cost_w = dw;
    CostDesc cd{};
    cd.kind = 1;
    cd.n_obs = n_obs;
    cd.lam = lambda;
    for (int o = 0; o < n_obs; ++o) {
        cd.ox[o] = obstacles[3 * o];
        cd.oy[o] = obstacles[3 * o + 1];
        cd.os[o] = obstacles[3 * o + 2];
    }
    cd.p0x = p0[0];
    cd.p0y = p0[1];
    cd.w = dw;
    c->cost = cd;
    c->cost_H = H;
    return BAB_OK;
}

int bab_context_create(bab_ctx **out)
{
    if (!out) return BAB_ERR_INVALID_ARG;
    *out = nullptr;
    bab_ctx *c = new bab_ctx();
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(c->d_status);
        delete c;
        return e == cudaErrorMemoryAllocation ? BAB_ERR_OOM : BAB_ERR_CUDA;
    }
    *out = c;
    return BAB_OK;
}

int bab_synth_search(bab_ctx *c, int d, const float *lo, const float *hi, const uint64_t *id, int n, const int *d_n,
                     int samples, uint64_t seed, int iters, int elites, float jitter, const float *warm_u, float *ub,
                     float *best_u, double *inc_val, float *inc_u, void *stream)
{
    if (!c) return BAB_ERR_INVALID_ARG;
    c->err[0] = 0;
    if (d < 1 || d > (1 << 20) || n < 0) return fail(c, BAB_ERR_SHAPE, "bad d or n");
    if (samples < 1 || samples > BAB_CEM_MAX_SAMPLES) return fail(c, BAB_ERR_SHAPE, "samples must be in [1, 4096]");
    if (iters < 0 || (iters > 0 && (elites < 1 || elites > samples)))
        return fail(c, BAB_ERR_INVALID_ARG, "need iters >= 0 and, for the cross-entropy search, 1 <= elites <= samples");
    if ((long long)(iters > 0 ? iters : 1) * samples >= (1ll << 32)) return fail(c, BAB_ERR_SHAPE, "too many samples");
    if (iters > 0 && (!(jitter >= 0.f) || !std::isfinite(jitter)))
        return fail(c, BAB_ERR_INVALID_ARG, "jitter must be finite and >= 0");
    if (n > 0 && (!lo || !hi || !id || !ub || !best_u)) return fail(c, BAB_ERR_INVALID_ARG, "null array");
    if ((inc_val == nullptr) != (inc_u == nullptr)) return fail(c, BAB_ERR_INVALID_ARG, "inc_val and inc_u go together");
    if (n == 0) return BAB_OK;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t kb = al((size_t)n * 8), cb = al((size_t)n * samples * 4), db = al((size_t)n * d * 4);
    int rc = ensure_scratch(c, iters > 0 ? kb + cb + 2 * db + kb : kb);
    if (rc) return rc;
    char *sp = static_cast<char *>(c->scratch);
    auto *keys = reinterpret_cast<unsigned long long *>(sp);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (iters == 0) {
        e = launch_synth_search(d, lo, hi, id, n, d_n, samples, 0, seed, nullptr, nullptr, keys, nullptr, ub, best_u, st);
    } else {
        CemArgs g{};
        g.lo = lo;
        g.hi = hi;
        g.id = id;
        g.n = n;
        g.d_n = d_n;
        g.d = d;
        g.M = samples;
        g.E = elites;
        g.jitter = jitter;
        g.seed = seed;
        g.costs = reinterpret_cast<float *>(sp + kb);
        g.mu = reinterpret_cast<float *>(sp + kb + cb);
        g.sigma = reinterpret_cast<float *>(sp + kb + cb + db);
        g.best = reinterpret_cast<unsigned long long *>(sp + kb + cb + 2 * db);
        g.ub = ub;
        g.best_u = best_u;
        e = launch_cem_init(g, warm_u, st);
        for (int it = 0; it < iters && e == cudaSuccess; ++it) {
            g.it = it;
            e = launch_synth_search(d, lo, hi, id, n, d_n, samples, it, seed, g.mu, g.sigma, keys,
                                    const_cast<float *>(g.costs), ub, best_u, st);
            if (e == cudaSuccess) e = launch_cem_step(g, st);
        }
    }
    if (e == cudaSuccess && inc_val) e = launch_synth_incumbent(d, ub, best_u, n, d_n, inc_val, inc_u, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "synthetic-objective search kernels");
    return BAB_OK;
}

int bab_synth_bound(bab_ctx *c, int d, const float *lo, const float *hi, int n, const int *d_n, float *lb, void *stream)
{
    if (!c) return BAB_ERR_INVALID_ARG;
    c->err[0] = 0;
    if (d < 1 || n < 0) return fail(c, BAB_ERR_SHAPE, "bad d or n");
    if (n > 0 && (!lo || !hi || !lb)) return fail(c, BAB_ERR_INVALID_ARG, "null array");
    cudaError_t e = launch_synth_bound(d, lo, hi, n, d_n, lb, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "synthetic-objective bound kernel");
    return BAB_OK;
}

int bab_destroy(bab_ctx *c)
{
    if (!c) return BAB_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    cudaFree(c->d_raw);
    cudaFree(c->d_fwd);
    cudaFree(c->d_bwd);
    cudaFree(c->d_tc);
    cudaFree(c->d_tcb);
    cudaFree(c->d_ibp);
    cudaFree(c->d_ibp_tf);
    cudaFree(c->d_tf);
    cudaFree(c->d_tc_bias);
    cudaFree(c->scratch);
    cudaFree(c->d_status);
    cudaFree(c->d_cost_w);
    delete c;
    return BAB_OK;
}

const char *bab_last_error(const bab_ctx *c) { return c ? c->err : "null context"; }

int bab_status(bab_ctx *c, void *stream)
{
    if (!c) return BAB_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int v = 0;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpy(&v, c->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(c, e, "status read");
    return v;
}

}  // extern "C"

namespace {
int rollout_impl(bab_ctx *c, const float *x0, const float *goal, int H, float rho, const float *lo, const float *hi,
                 const uint64_t *id, int n, const int *d_n, int samples, uint64_t seed, int precision, float *ub,
                 float *best_u, double *inc_val, float *inc_u, float *costs, void *stream);
// the head of a rollout call's scratch: the per-box keys, the top-k list, the selection words
size_t rollout_keys_bytes(int n) { return ((size_t)n * sizeof(unsigned long long) + 255) & ~size_t(255); }
size_t rollout_list_bytes(int n) { return ((size_t)n * sizeof(int) + 255) & ~size_t(255); }
size_t rollout_head_bytes(int n) { return rollout_keys_bytes(n) + rollout_list_bytes(n) + 512; }
}  // namespace

extern "C" {

int bab_rollout(bab_ctx *c, const float *x0, const float *goal, int H, float rho, const float *lo, const float *hi,
                const uint64_t *id, int n, const int *d_n, int samples, uint64_t seed, int precision, float *ub,
                float *best_u, double *inc_val, float *inc_u, void *stream)
{
    return rollout_impl(c, x0, goal, H, rho, lo, hi, id, n, d_n, samples, seed, precision, ub, best_u, inc_val, inc_u,
                        nullptr, stream);
}

}  // extern "C"

namespace {
int rollout_impl(bab_ctx *c, const float *x0, const float *goal, int H, float rho, const float *lo, const float *hi,
                 const uint64_t *id, int n, const int *d_n, int samples, uint64_t seed, int precision, float *ub,
                 float *best_u, double *inc_val, float *inc_u, float *costs, void *stream)
{
    int rc = check_problem(c, x0, goal, H, rho, lo, hi, n);
    if (rc) return rc;
    if (samples < 1) return fail(c, BAB_ERR_SHAPE, "samples must be >= 1");
    if (n > 0 && (!id || !ub)) return fail(c, BAB_ERR_INVALID_ARG, "id and ub are required");
    if ((inc_val == nullptr) != (inc_u == nullptr)) return fail(c, BAB_ERR_INVALID_ARG, "inc_val and inc_u go together");
    if (inc_val && !best_u) return fail(c, BAB_ERR_INVALID_ARG, "the incumbent update needs best_u");
    if (precision != BAB_PREC_FP32 && precision != BAB_PREC_BF16X3 && precision != BAB_PREC_BF16)
        return fail(c, BAB_ERR_INVALID_ARG, "unknown precision %d", precision);
    const int split = precision == BAB_PREC_BF16X3 ? 3 : 1;
    if (c->cost.kind != 0 && precision != BAB_PREC_FP32 && c->net.s > 8)
        return refuse_obstacles(c, "tensor-core rollouts with more than 8 states");
    if (precision != BAB_PREC_FP32 && !rollout_tc_supported(c->net, split, c->max_smem))
        return fail(c, BAB_ERR_UNSUPPORTED, "tensor-core rollout needs hidden widths that are multiples of 32, "
                                            "s <= 32, s + k <= 64 and a weight image that fits in shared memory");
    if (n == 0) return BAB_OK;
    const size_t key_bytes = rollout_keys_bytes(n);
    rc = ensure_scratch(c, rollout_head_bytes(n));
    if (rc) return rc;
    RolloutArgs a{};
    a.cost = c->cost;
    a.topk = precision == BAB_PREC_BF16 ? c->rescore_topk : 0;
    a.topk_list = reinterpret_cast<int *>(static_cast<char *>(c->scratch) + key_bytes);
    a.topk_t = reinterpret_cast<unsigned long long *>(static_cast<char *>(c->scratch) + key_bytes + rollout_list_bytes(n));
    a.net = c->net;
    a.batch.P = 1;
    a.batch.Hmax = H;
    a.fwd = c->d_fwd;
    a.raw = c->d_raw;
    a.x0 = x0;
    a.goal = goal;
    a.lo = lo;
    a.hi = hi;
    a.id = id;
    a.n = n;
    a.d_n = d_n;
    a.H = H;
    a.M = samples;
    a.d = c->net.k * H;
    a.rho = rho;
    a.seed = seed;
    a.keys = reinterpret_cast<unsigned long long *>(c->scratch);
    a.ub = ub;
    a.best_u = best_u;
    a.inc_val = inc_val;
    a.inc_u = inc_u;
    a.status = c->d_status;
    a.tc_img = c->d_tc;
    a.tc_bias = c->d_tc_bias;
    a.tc_bytes = c->net.tc_bytes;
    a.costs = costs;
    cudaError_t e = precision == BAB_PREC_FP32 ? launch_rollout_fp32(a, c->tune_rollout_fp32, c->num_sms, (cudaStream_t)stream)
                                               : launch_rollout_tc(a, split, c->tune_rollout_tc, c->num_sms, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "rollout kernels");
    return BAB_OK;
}
}  // namespace

extern "C" {

int bab_split_dims(bab_ctx *c, int d, const float *lo, const float *hi, const uint64_t *id, int n, const int *d_n,
                   uint64_t seed, const float *costs, int samples, int top_k, int *split_dim, void *stream)
{
    if (!c) return BAB_ERR_INVALID_ARG;
    c->err[0] = 0;
    if (d < 1 || n < 0 || samples < 1) return fail(c, BAB_ERR_SHAPE, "bad d, n or samples");
    if (top_k < 1 || top_k > 64 || top_k > samples) return fail(c, BAB_ERR_INVALID_ARG, "top_k must be in [1, min(64, samples)]");
    if (n > 0 && (!lo || !hi || !id || !costs || !split_dim)) return fail(c, BAB_ERR_INVALID_ARG, "null array");
    cudaError_t e = launch_split_dims(d, lo, hi, id, n, d_n, seed, costs, samples, top_k, split_dim, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "split-dimension kernel");
    return BAB_OK;
}

int bab_rollout_split(bab_ctx *c, const float *x0, const float *goal, int H, float rho, const float *lo, const float *hi,
                      const uint64_t *id, int n, const int *d_n, int samples, uint64_t seed, int precision,
                      float top_pct, float *ub, float *best_u, double *inc_val, float *inc_u, float *costs,
                      int *split_dim, void *stream)
{
    if (!c) return BAB_ERR_INVALID_ARG;
    if (!(top_pct > 0.f && top_pct <= 100.f)) return fail(c, BAB_ERR_INVALID_ARG, "top_pct must be in (0, 100]");
    if (n > 0 && !split_dim) return fail(c, BAB_ERR_INVALID_ARG, "split_dim is required");
    int top_k = (int)std::ceil((double)top_pct / 100.0 * samples);
    top_k = top_k < 1 ? 1 : (top_k > 64 ? 64 : top_k);
    if (top_k > samples) top_k = samples;
    float *cst = costs;
    if (!cst && n > 0) {
        // costs in the scratch after the rollout's own keys, top-k list and threshold
        int rc = ensure_scratch(c, rollout_head_bytes(n) + (size_t)n * samples * sizeof(float) + 256);
        if (rc) return rc;
        cst = reinterpret_cast<float *>(static_cast<char *>(c->scratch) + rollout_head_bytes(n));
    }
    int rc = rollout_impl(c, x0, goal, H, rho, lo, hi, id, n, d_n, samples, seed, precision, ub, best_u, inc_val, inc_u,
                          cst, stream);
    if (rc) return rc;
    return bab_split_dims(c, c->net.k * H, lo, hi, id, n, d_n, seed, cst, samples, top_k, split_dim, stream);
}

int bab_rollout_cem(bab_ctx *c, const float *x0, const float *goal, int H, float rho, const float *lo, const float *hi,
                    const uint64_t *id, int n, const int *d_n, int samples, int iters, int elites, float jitter,
                    uint64_t seed, int precision, const float *warm_u, float *ub, float *best_u, double *inc_val,
                    float *inc_u, void *stream)
{
    int rc = check_problem(c, x0, goal, H, rho, lo, hi, n);
    if (rc) return rc;
    if (samples < 1 || samples > BAB_CEM_MAX_SAMPLES) return fail(c, BAB_ERR_SHAPE, "samples must be in [1, 4096]");
    if (iters < 1 || elites < 1 || elites > samples)
        return fail(c, BAB_ERR_INVALID_ARG, "need iters >= 1 and 1 <= elites <= samples");
    if (!(jitter >= 0.f) || !std::isfinite(jitter)) return fail(c, BAB_ERR_INVALID_ARG, "jitter must be finite and >= 0");
    if (n > 0 && (!id || !ub || !best_u)) return fail(c, BAB_ERR_INVALID_ARG, "id, ub and best_u are required");
    if ((inc_val == nullptr) != (inc_u == nullptr)) return fail(c, BAB_ERR_INVALID_ARG, "inc_val and inc_u go together");
    if (precision != BAB_PREC_FP32 && precision != BAB_PREC_BF16X3)
        return fail(c, BAB_ERR_UNSUPPORTED, "the cross-entropy search runs in FP32 or BF16x3 (precision %d)", precision);
    if (precision == BAB_PREC_BF16X3 && (rc = refuse_obstacles(c, "the tensor-core cross-entropy search")) != BAB_OK)
        return rc;
    if ((long long)iters * samples >= (1ll << 32)) return fail(c, BAB_ERR_SHAPE, "iters * samples must be < 2^32");
    if (precision == BAB_PREC_BF16X3 && !rollout_tc_supported(c->net, 3, c->max_smem))
        return fail(c, BAB_ERR_UNSUPPORTED, "tensor-core rollout not available for this network");
    if (n == 0) return BAB_OK;
    const int d = c->net.k * H;
    // scratch: rollout keys, top-k threshold, costs [n][M], mu and sigma [n][d], best keys [n]
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t kb = al((size_t)n * 8), cb = al((size_t)n * samples * 4), db = al((size_t)n * d * 4);
    rc = ensure_scratch(c, kb + 512 + cb + 2 * db + kb);
    if (rc) return rc;
    char *sp = static_cast<char *>(c->scratch);
    float *costs = reinterpret_cast<float *>(sp + kb + 512);
    CemArgs g{};
    g.lo = lo;
    g.hi = hi;
    g.id = id;
    g.n = n;
    g.d_n = d_n;
    g.d = d;
    g.M = samples;
    g.E = elites;
    g.jitter = jitter;
    g.seed = seed;
    g.costs = costs;
    g.mu = reinterpret_cast<float *>(sp + kb + 512 + cb);
    g.sigma = reinterpret_cast<float *>(sp + kb + 512 + cb + db);
    g.best = reinterpret_cast<unsigned long long *>(sp + kb + 512 + cb + 2 * db);
    g.ub = ub;
    g.best_u = best_u;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = launch_cem_init(g, warm_u, st);
    RolloutArgs a{};
    a.cost = c->cost;
    a.net = c->net;
    a.batch.P = 1;
    a.batch.Hmax = H;
    a.fwd = c->d_fwd;
    a.raw = c->d_raw;
    a.x0 = x0;
    a.goal = goal;
    a.lo = lo;
    a.hi = hi;
    a.id = id;
    a.n = n;
    a.d_n = d_n;
    a.H = H;
    a.M = samples;
    a.d = d;
    a.rho = rho;
    a.seed = seed;
    a.keys = reinterpret_cast<unsigned long long *>(sp);
    a.topk_t = reinterpret_cast<unsigned long long *>(sp + kb);
    a.ub = ub;
    a.best_u = best_u;
    a.inc_val = inc_val;
    a.inc_u = inc_u;
    a.status = c->d_status;
    a.tc_img = c->d_tc;
    a.tc_bias = c->d_tc_bias;
    a.tc_bytes = c->net.tc_bytes;
    a.costs = costs;
    a.cem_mu = g.mu;
    a.cem_sigma = g.sigma;
    for (int it = 0; it < iters && e == cudaSuccess; ++it) {
        a.cem_it = it;
        g.it = it;
        e = precision == BAB_PREC_FP32 ? launch_rollout_fp32(a, c->tune_rollout_fp32, c->num_sms, st)
                                       : launch_rollout_tc(a, 3, c->tune_rollout_tc, c->num_sms, st);
        if (e == cudaSuccess) e = launch_cem_step(g, st);
    }
    if (e == cudaSuccess && inc_val) {
        launch_incumbent(a, st);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "cross-entropy search kernels");
    return BAB_OK;
}

int bab_rollout_search_bounds(bab_ctx *c, const float *x0, const float *goal, int H, float rho, const float *lo,
                              const float *hi, const uint64_t *id, int n, const int *d_n, int samples, uint64_t seed,
                              float *ub, float *best_u, double *inc_val, float *inc_u, float *pre_lo, float *pre_hi,
                              float *x_lo, float *x_hi, void *stream)
{
    int rc = check_problem(c, x0, goal, H, rho, lo, hi, n);
    if (rc) return rc;
    if (samples < 1) return fail(c, BAB_ERR_SHAPE, "samples must be >= 1");
    if (n > 0 && (!id || !ub || !pre_lo || !pre_hi || !x_lo || !x_hi))
        return fail(c, BAB_ERR_INVALID_ARG, "id, ub and the four bound arrays are required");
    if ((inc_val == nullptr) != (inc_u == nullptr)) return fail(c, BAB_ERR_INVALID_ARG, "inc_val and inc_u go together");
    if (inc_val && !best_u) return fail(c, BAB_ERR_INVALID_ARG, "the incumbent update needs best_u");
    if (n == 0) return BAB_OK;
    rc = ensure_scratch(c, (size_t)n * sizeof(unsigned long long) + 256);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    RolloutArgs a{};
    a.cost = c->cost;
    a.net = c->net;
    a.batch.P = 1;
    a.batch.Hmax = H;
    a.fwd = c->d_fwd;
    a.raw = c->d_raw;
    a.x0 = x0;
    a.goal = goal;
    a.lo = lo;
    a.hi = hi;
    a.id = id;
    a.n = n;
    a.d_n = d_n;
    a.H = H;
    a.M = samples;
    a.d = c->net.k * H;
    a.rho = rho;
    a.seed = seed;
    a.keys = reinterpret_cast<unsigned long long *>(c->scratch);
    a.ub = ub;
    a.best_u = best_u;
    a.inc_val = inc_val;
    a.inc_u = inc_u;
    a.status = c->d_status;
    a.emp_pre_lo = reinterpret_cast<uint32_t *>(pre_lo);
    a.emp_pre_hi = reinterpret_cast<uint32_t *>(pre_hi);
    a.emp_x_lo = reinterpret_cast<uint32_t *>(x_lo);
    a.emp_x_hi = reinterpret_cast<uint32_t *>(x_hi);
    launch_emp_init(a, st);
    cudaError_t e = launch_rollout_fp32(a, c->tune_rollout_fp32, c->num_sms, st);
    if (e == cudaSuccess) {
        launch_emp_finish(a, st);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "search-bound rollout kernels");
    return BAB_OK;
}

int bab_bound_crown_given(bab_ctx *c, const float *x0, const float *goal, int H, float rho, const float *lo,
                          const float *hi, int n, const int *d_n, const float *pre_lo, const float *pre_hi,
                          const float *x_lo, const float *x_hi, int t_stop, float *lb, void *stream)
{
    int rc = check_problem(c, x0, goal, H, rho, lo, hi, n);
    if (rc) return rc;
    rc = refuse_obstacles(c, "CROWN with given bounds and early stop");
    if (rc) return rc;
    if (t_stop < 0 || t_stop > H) return fail(c, BAB_ERR_INVALID_ARG, "t_stop must be in [0, horizon]");
    if (n > 0 && (!lb || !pre_lo || !pre_hi || !x_lo || !x_hi))
        return fail(c, BAB_ERR_INVALID_ARG, "lb and the four bound arrays are required");
    if (n == 0) return BAB_OK;
    BoundArgs a = make_bound_args(c, x0, goal, H, rho, lo, hi, n, d_n);
    a.pre_lo = const_cast<float *>(pre_lo);
    a.pre_hi = const_cast<float *>(pre_hi);
    a.x_lo = const_cast<float *>(x_lo);
    a.x_hi = const_cast<float *>(x_hi);
    a.S = nullptr;  // given bounds: an estimate, no rounding margin
    a.t_stop = t_stop;
    a.lb = lb;
    cudaError_t e = launch_crown(a, c->num_sms, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "CROWN kernel");
    return BAB_OK;
}

int bab_update_incumbent(bab_ctx *c, const float *x0, const float *goal, int H, float rho, const float *ub,
                         const float *best_u, int n, const int *d_n, double *inc_val, float *inc_u, void *stream)
{
    if (!c) return BAB_ERR_INVALID_ARG;
    c->err[0] = 0;
    if (!x0 || !goal || !inc_val || !inc_u) return fail(c, BAB_ERR_INVALID_ARG, "x0, goal, inc_val and inc_u are required");
    if (H < 1 || H > (1 << 20) || n < 0) return fail(c, BAB_ERR_SHAPE, "bad horizon or n");
    if (!(rho >= 0.f) || !std::isfinite(rho)) return fail(c, BAB_ERR_INVALID_ARG, "rho must be finite and >= 0");
    if (n > 0 && (!ub || !best_u)) return fail(c, BAB_ERR_INVALID_ARG, "ub and best_u are required");
    if (n == 0) return BAB_OK;
    RolloutArgs a{};
    a.cost = c->cost;
    a.net = c->net;
    a.batch.P = 1;
    a.batch.Hmax = H;
    a.raw = c->d_raw;
    a.x0 = x0;
    a.goal = goal;
    a.n = n;
    a.d_n = d_n;
    a.H = H;
    a.d = c->net.k * H;
    a.rho = rho;
    a.ub = const_cast<float *>(ub);
    a.best_u = const_cast<float *>(best_u);
    a.inc_val = inc_val;
    a.inc_u = inc_u;
    a.status = c->d_status;
    launch_incumbent(a, (cudaStream_t)stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "incumbent kernel");
    return BAB_OK;
}

int bab_bound_ibp(bab_ctx *c, const float *x0, const float *goal, int H, float rho, const float *lo, const float *hi,
                  int n, const int *d_n, float *lb_ibp, float *pre_lo, float *pre_hi, float *x_lo, float *x_hi,
                  void *stream)
{
    int rc = check_problem(c, x0, goal, H, rho, lo, hi, n);
    if (rc) return rc;
    if ((pre_lo == nullptr) != (pre_hi == nullptr) || (x_lo == nullptr) != (x_hi == nullptr))
        return fail(c, BAB_ERR_INVALID_ARG, "bound arrays come in lo/hi pairs");
    if (n == 0) return BAB_OK;
    rc = ensure_scratch(c, bound_scratch_bytes(c->net, n, H, c->net.k * H, false));
    if (rc) return rc;
    BoundArgs a = make_bound_args(c, x0, goal, H, rho, lo, hi, n, d_n);
    Carver cv{reinterpret_cast<char *>(c->scratch)};
    return run_ibp(c, a, cv, pre_lo, pre_hi, x_lo, x_hi, lb_ibp, (cudaStream_t)stream);
}

// The CROWN launch of a bound precision (the tensor-core ones need a.mu set by the caller).
static cudaError_t launch_crown_prec(bab_ctx *c, BoundArgs &a, int precision, cudaStream_t st)
{
    if (precision == BAB_PREC_FP32) return launch_crown(a, c->num_sms, st);
    a.tc_bias = c->d_tc_bias;
    if (precision == BAB_PREC_TF32X3) {
        a.tcb_img = c->d_tf;
        return launch_crown_tf32(a, c->num_sms, st);
    }
    a.tcb_img = c->d_tcb;
    return launch_crown_tc(a, c->tune_crown_tc, c->num_sms, st);
}

// Whether `precision` is a bound precision this context can run (else fails with BAB_ERR_UNSUPPORTED).
static int check_crown_precision(bab_ctx *c, int precision, const char *what)
{
    int rc;
    if (precision == BAB_PREC_BF16X3) {
        if ((rc = check_tc_obstacles(c, what)) != BAB_OK) return rc;
        if (!crown_tc_supported(c->net, c->max_smem))
            return fail(c, BAB_ERR_UNSUPPORTED, "tensor-core CROWN needs hidden widths that are multiples of 32, "
                                                "s <= 32, s + k <= 48 and a weight image that fits in shared memory");
        return BAB_OK;
    }
    if (precision == BAB_PREC_TF32X3) {
        if (c->cost.kind != 0) return fail(c, BAB_ERR_UNSUPPORTED, "%s in TF32x3 takes the squared-distance cost", what);
        if (!crown_tf32_supported(c->net, c->max_smem))
            return fail(c, BAB_ERR_UNSUPPORTED, "TF32x3 CROWN needs hidden widths that are multiples of 32 and every "
                                                "width at most 256, s <= 32");
        return BAB_OK;
    }
    if (precision != BAB_PREC_FP32) return fail(c, BAB_ERR_UNSUPPORTED, "bound precision %d not available", precision);
    return BAB_OK;
}

// One pass of bab_bound_crown over rows row0 .. row0 + n - 1 (pointers already offset to row0).
static int bound_crown_pass(bab_ctx *c, const float *x0, const float *goal, int H, float rho, const float *lo,
                            const float *hi, int n, const int *d_n, int row0, const float *alpha, int precision,
                            float *lb, float *margin, float *lin_coef, float *lin_const, void *stream)
{
    const bool tc = precision != BAB_PREC_FP32;
    int rc = ensure_scratch(c, bound_scratch_bytes(c->net, n, H, c->net.k * H, tc));
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    BoundArgs a = make_bound_args(c, x0, goal, H, rho, lo, hi, n, d_n, row0);
    Carver cv{reinterpret_cast<char *>(c->scratch)};
    rc = run_ibp(c, a, cv, nullptr, nullptr, nullptr, nullptr, nullptr, st);
    if (rc) return rc;
    a.alpha = alpha;
    a.lb = lb;
    a.margin = margin;
    a.lin_coef = lin_coef;
    a.lin_const = lin_const;
    if (tc) a.mu = lin_coef ? lin_coef : cv.take<float>((size_t)n * a.d);
    cudaError_t e = launch_crown_prec(c, a, precision, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "CROWN kernel");
    return BAB_OK;
}

int bab_bound_crown(bab_ctx *c, const float *x0, const float *goal, int H, float rho, const float *lo, const float *hi,
                    int n, const int *d_n, const float *alpha, int precision, float *lb, float *margin,
                    float *lin_coef, float *lin_const, void *stream)
{
    int rc = check_problem(c, x0, goal, H, rho, lo, hi, n);
    if (rc) return rc;
    if (n > 0 && !lb) return fail(c, BAB_ERR_INVALID_ARG, "lb is required");
    if ((rc = check_crown_precision(c, precision, "the tensor-core CROWN")) != BAB_OK) return rc;
    const bool tc = precision != BAB_PREC_FP32;
    if (n == 0) return BAB_OK;
    const int d = c->net.k * H;
    const size_t per_row = bound_scratch_bytes(c->net, 1, H, d, tc) - 16 * 256 + (tc && !lin_coef ? (size_t)d * 4 : 0);
    const int rows = chunk_rows(c, 16 * 256 + 256, per_row, n);
    if (rows == 0) return fail(c, BAB_ERR_OOM, "one box needs more scratch than the limit");
    for (int r0 = 0; r0 < n; r0 += rows) {
        const int m = n - r0 < rows ? n - r0 : rows;
        const size_t ro = (size_t)r0;
        rc = bound_crown_pass(c, x0, goal, H, rho, lo + ro * d, hi + ro * d, m, d_n, r0,
                              alpha ? alpha + ro * H * c->net.sumh : nullptr, precision, lb + ro,
                              margin ? margin + ro : nullptr, lin_coef ? lin_coef + ro * d : nullptr,
                              lin_const ? lin_const + ro : nullptr, stream);
        if (rc) return rc;
    }
    return BAB_OK;
}

int bab_alpha_init(bab_ctx *c, const float *x0, const float *goal, int H, float rho, const float *lo, const float *hi,
                   int n, const int *d_n, float *alpha, void *stream)
{
    int rc = check_problem(c, x0, goal, H, rho, lo, hi, n);
    if (rc) return rc;
    if (n > 0 && !alpha) return fail(c, BAB_ERR_INVALID_ARG, "alpha is required");
    if (n == 0) return BAB_OK;
    rc = ensure_scratch(c, bound_scratch_bytes(c->net, n, H, c->net.k * H, false));
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    BoundArgs a = make_bound_args(c, x0, goal, H, rho, lo, hi, n, d_n);
    Carver cv{reinterpret_cast<char *>(c->scratch)};
    rc = run_ibp(c, a, cv, nullptr, nullptr, nullptr, nullptr, nullptr, st);
    if (rc) return rc;
    a.alpha = alpha;
    cudaError_t e = launch_alpha_init(a, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "alpha init kernel");
    return BAB_OK;
}

}  // extern "C"

namespace {

// Bound at alpha and its gradient (interval bounds, CROWN storing the pre-relaxation coefficients and the
// concretizing point, forward pass of the relaxed network).  `a` keeps the scratch pointers for the caller.
int alpha_grad_core(bab_ctx *c, BoundArgs &a, Carver &cv, int precision, const float *alpha, float *lb,
                    float *lb_best, float *grad_alpha, cudaStream_t st)
{
    const int n = a.n, H = a.H, d = a.d;
    int rc = run_ibp(c, a, cv, nullptr, nullptr, nullptr, nullptr, nullptr, st);
    if (rc) return rc;
    const size_t nh = (size_t)n * H * c->net.sumh;
    a.alpha = alpha;
    a.A_pre = cv.take<float>(nh);
    a.ustar = cv.take<float>((size_t)n * d);
    a.grad_alpha = grad_alpha ? grad_alpha : cv.take<float>(nh);
    a.lb = lb ? lb : cv.take<float>(n);
    a.lb_best = lb_best;
    if (precision != BAB_PREC_FP32) a.mu = cv.take<float>((size_t)n * d);
    cudaError_t e = launch_crown_prec(c, a, precision, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "CROWN kernel");
    e = launch_alpha_fwd(a, c->num_sms, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "alpha adjoint kernel");
    return BAB_OK;
}

int check_bound_precision(bab_ctx *c, int precision) { return check_crown_precision(c, precision, "the alpha step"); }

}  // namespace

extern "C" {

int bab_alpha_grad(bab_ctx *c, const float *x0, const float *goal, int H, float rho, const float *lo, const float *hi,
                   int n, const int *d_n, const float *alpha, int precision, float *lb, float *grad_alpha, void *stream)
{
    int rc = check_problem(c, x0, goal, H, rho, lo, hi, n);
    if (rc) return rc;
    if (precision == BAB_PREC_BF16X3 && (rc = check_tc_obstacles(c, "the tensor-core alpha gradient")) != BAB_OK)
        return rc;
    if (n > 0 && (!alpha || !lb || !grad_alpha)) return fail(c, BAB_ERR_INVALID_ARG, "alpha, lb and grad are required");
    rc = check_bound_precision(c, precision);
    if (rc) return rc;
    if (n == 0) return BAB_OK;
    rc = ensure_scratch(c, bound_scratch_bytes(c->net, n, H, c->net.k * H, true) +
                               (size_t)n * c->net.k * H * sizeof(float) + 256);
    if (rc) return rc;
    BoundArgs a = make_bound_args(c, x0, goal, H, rho, lo, hi, n, d_n);
    Carver cv{reinterpret_cast<char *>(c->scratch)};
    return alpha_grad_core(c, a, cv, precision, alpha, lb, nullptr, grad_alpha, (cudaStream_t)stream);
}

int bab_alpha_step(bab_ctx *c, const float *x0, const float *goal, int H, float rho, const float *lo, const float *hi,
                   int n, const int *d_n, float *alpha, float *adam_m, float *adam_v, int step, float lr,
                   int precision, float *lb, float *lb_best, float *grad_alpha, void *stream)
{
    int rc = check_problem(c, x0, goal, H, rho, lo, hi, n);
    if (rc) return rc;
    if (precision == BAB_PREC_BF16X3 && (rc = check_tc_obstacles(c, "the tensor-core alpha step")) != BAB_OK)
        return rc;
    if (n > 0 && (!alpha || !adam_m || !adam_v)) return fail(c, BAB_ERR_INVALID_ARG, "alpha, m and v are required");
    if (step < 1) return fail(c, BAB_ERR_INVALID_ARG, "step counts from 1");
    if (!(lr >= 0.f) || !std::isfinite(lr)) return fail(c, BAB_ERR_INVALID_ARG, "bad learning rate");
    rc = check_bound_precision(c, precision);
    if (rc) return rc;
    if (n == 0) return BAB_OK;
    const int d = c->net.k * H;
    rc = ensure_scratch(c, bound_scratch_bytes(c->net, n, H, d, true) + (size_t)n * d * sizeof(float) + 256);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    BoundArgs a = make_bound_args(c, x0, goal, H, rho, lo, hi, n, d_n);
    Carver cv{reinterpret_cast<char *>(c->scratch)};
    rc = alpha_grad_core(c, a, cv, precision, alpha, lb, lb_best, grad_alpha, st);
    if (rc) return rc;
    const size_t nh = (size_t)n * H * c->net.sumh;
    const double bc1 = 1.0 - std::pow(0.9, step), bc2 = 1.0 - std::pow(0.999, step);
    cudaError_t e = launch_adam(alpha, adam_m, adam_v, a.grad_alpha, (long long)nh, lr, (float)bc1, (float)bc2, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "Adam kernel");
    return BAB_OK;
}

// One pass of bab_box_grad over rows row0 .. row0 + n - 1 (pointers already offset to row0).
static int box_grad_pass(bab_ctx *c, const float *x0, const float *goal, int H, float rho, const float *lo,
                         const float *hi, int n, const int *d_n, int row0, const float *alpha, float *lb,
                         float *grad_lo, float *grad_hi, void *stream)
{
    const NetDesc &N = c->net;
    const int d = N.k * H;
    const size_t nh = (size_t)n * H * N.sumh, nx = (size_t)n * (H + 1) * N.s;
    int rc = ensure_scratch(c, bound_scratch_bytes(N, n, H, d, true) + (3 * nh + nx + 2 * (size_t)n * d) * sizeof(float) +
                               8 * 256);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    BoundArgs a = make_bound_args(c, x0, goal, H, rho, lo, hi, n, d_n, row0);
    Carver cv{reinterpret_cast<char *>(c->scratch)};
    rc = run_ibp(c, a, cv, nullptr, nullptr, nullptr, nullptr, nullptr, st);
    if (rc) return rc;
    a.alpha = alpha;
    a.A_pre = cv.take<float>(nh);
    a.ustar = cv.take<float>((size_t)n * d);
    a.lin_coef = cv.take<float>((size_t)n * d);
    a.lb = lb;
    cudaError_t e = launch_crown(a, c->num_sms, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "CROWN kernel");
    float *GL = cv.take<float>(nh), *GU = cv.take<float>(nh), *GX = cv.take<float>(nx);
    e = launch_box_grad_warp(a, GL, GU, GX, grad_lo, grad_hi, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "box gradient kernel");
    return BAB_OK;
}

int bab_box_grad(bab_ctx *c, const float *x0, const float *goal, int H, float rho, const float *lo, const float *hi,
                 int n, const int *d_n, const float *alpha, float *lb, float *grad_lo, float *grad_hi, void *stream)
{
    int rc = check_problem(c, x0, goal, H, rho, lo, hi, n);
    if (rc) return rc;
    rc = refuse_obstacles(c, "the box gradient");
    if (rc) return rc;
    if (n > 0 && (!lb || !grad_lo || !grad_hi)) return fail(c, BAB_ERR_INVALID_ARG, "lb, grad_lo and grad_hi are required");
    if (n == 0) return BAB_OK;
    const NetDesc &N = c->net;
    const int d = N.k * H;
    const size_t per_row = bound_scratch_bytes(N, 1, H, d, true) - 16 * 256 +
                           (3 * (size_t)H * N.sumh + (size_t)(H + 1) * N.s + 2 * (size_t)d) * sizeof(float);
    const int rows = chunk_rows(c, 16 * 256 + 8 * 256, per_row, n);
    if (rows == 0) return fail(c, BAB_ERR_OOM, "one box needs more scratch than the limit");
    for (int r0 = 0; r0 < n; r0 += rows) {
        const int m = n - r0 < rows ? n - r0 : rows;
        const size_t ro = (size_t)r0;
        rc = box_grad_pass(c, x0, goal, H, rho, lo + ro * d, hi + ro * d, m, d_n, r0,
                           alpha ? alpha + ro * H * N.sumh : nullptr, lb + ro, grad_lo + ro * d, grad_hi + ro * d,
                           stream);
        if (rc) return rc;
    }
    return BAB_OK;
}

// One pass of bab_alpha_optimize over rows row0 .. row0 + n - 1 (pointers already offset to row0).
static int alpha_optimize_pass(bab_ctx *c, const float *x0, const float *goal, int H, float rho, const float *lo,
                               const float *hi, int n, const int *d_n, int row0, int steps, float lr, int precision,
                               float *alpha, float *lb_best, void *stream)
{
    const int d = c->net.k * H;
    const size_t nh = (size_t)n * H * c->net.sumh;
    int rc = ensure_scratch(c, bound_scratch_bytes(c->net, n, H, d, true) + (3 * nh + (size_t)n * d) * sizeof(float) +
                               4 * 256);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    BoundArgs a = make_bound_args(c, x0, goal, H, rho, lo, hi, n, d_n, row0);
    Carver cv{reinterpret_cast<char *>(c->scratch)};
    // interval bounds do not depend on alpha: once for all steps
    rc = run_ibp(c, a, cv, nullptr, nullptr, nullptr, nullptr, nullptr, st);
    if (rc) return rc;
    const int fv = c->tune_alpha_fused;
    if (precision == BAB_PREC_FP32 && fv >= 0 && fv < 3) {
        // the whole loop in one launch, a tile of boxes with all its state in shared memory
        if (!alpha_fused_fits(c->net, H, d)) return fail(c, BAB_ERR_UNSUPPORTED, "fused alpha tile does not fit");
        a.lb_best = lb_best;
        cudaError_t e = launch_alpha_fused(a, steps, lr, alpha, fv, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "fused alpha kernel");
        return BAB_OK;
    }
    float *al = alpha ? alpha : cv.take<float>(nh);
    float *m = cv.take<float>(nh), *v = cv.take<float>(nh);
    if (precision == BAB_PREC_FP32 && (fv == -1 || fv == 3)) {
        // the whole loop in one launch, one warp per box
        a.A_pre = cv.take<float>(nh);
        a.lb_best = lb_best;
        cudaError_t e = launch_alpha_warp(a, steps, lr, al, m, v, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "warp alpha kernel");
        return BAB_OK;
    }
    a.A_pre = cv.take<float>(nh);
    a.ustar = cv.take<float>((size_t)n * d);
    a.grad_alpha = cv.take<float>(nh);
    a.lb = cv.take<float>(n);
    a.mu = cv.take<float>((size_t)n * d);
    a.alpha = al;
    cudaError_t e = launch_alpha_init(a, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(m, 0, nh * sizeof(float), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(v, 0, nh * sizeof(float), st);
    if (e == cudaSuccess) e = launch_fill(lb_best, n, -INFINITY, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "alpha set-up");
    a.lb_best = lb_best;
    for (int step = 1; step <= steps; ++step) {
        e = launch_crown_prec(c, a, precision, st);
        if (e == cudaSuccess) e = launch_alpha_fwd(a, c->num_sms, st);
        const double bc1 = 1.0 - std::pow(0.9, step), bc2 = 1.0 - std::pow(0.999, step);
        if (e == cudaSuccess) e = launch_adam(al, m, v, a.grad_alpha, (long long)nh, lr, (float)bc1, (float)bc2, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "alpha step");
    }
    return BAB_OK;
}

int bab_alpha_optimize(bab_ctx *c, const float *x0, const float *goal, int H, float rho, const float *lo,
                       const float *hi, int n, const int *d_n, int steps, float lr, int precision, float *alpha,
                       float *lb_best, void *stream)
{
    int rc = check_problem(c, x0, goal, H, rho, lo, hi, n);
    if (rc) return rc;
    if (precision == BAB_PREC_BF16X3 && (rc = check_tc_obstacles(c, "the tensor-core alpha optimisation")) != BAB_OK)
        return rc;
    if (n > 0 && !lb_best) return fail(c, BAB_ERR_INVALID_ARG, "lb_best is required");
    if (steps < 1 || steps > 100000) return fail(c, BAB_ERR_INVALID_ARG, "steps must be in [1, 100000]");
    if (!(lr >= 0.f) || !std::isfinite(lr)) return fail(c, BAB_ERR_INVALID_ARG, "bad learning rate");
    rc = check_bound_precision(c, precision);
    if (rc) return rc;
    if (n == 0) return BAB_OK;
    const int d = c->net.k * H;
    const size_t per_row = bound_scratch_bytes(c->net, 1, H, d, true) - 16 * 256 +
                           (3 * (size_t)H * c->net.sumh + (size_t)d) * sizeof(float);
    const int rows = chunk_rows(c, 16 * 256 + 4 * 256, per_row, n);
    if (rows == 0) return fail(c, BAB_ERR_OOM, "one box needs more scratch than the limit");
    for (int r0 = 0; r0 < n; r0 += rows) {
        const int m = n - r0 < rows ? n - r0 : rows;
        const size_t ro = (size_t)r0;
        rc = alpha_optimize_pass(c, x0, goal, H, rho, lo + ro * d, hi + ro * d, m, d_n, r0, steps, lr, precision,
                                 alpha ? alpha + ro * H * c->net.sumh : nullptr, lb_best + ro, stream);
        if (rc) return rc;
    }
    return BAB_OK;
}

}  // extern "C"

namespace {
int prune_branch_impl(bab_ctx *c, int d, const float *lo, const float *hi, const float *lb, const float *ub,
                      const uint64_t *id, int n, const int *d_n, const double *inc_val, int n_pick, float eta,
                      int split_rule, int pick_rule, float temperature, uint64_t pick_seed, const int *split_dim,
                      int *out_split_dim, const float *row_u, float *out_row_u, int cap_out, float *out_lo,
                      float *out_hi, float *out_lb, float *out_ub, uint64_t *out_id, uint8_t *keep, int *d_counts,
                      void *stream);
}  // namespace

extern "C" {

int bab_prune_branch(bab_ctx *c, int d, const float *lo, const float *hi, const float *lb, const float *ub,
                     const uint64_t *id, int n, const int *d_n, const double *inc_val, int n_pick, float eta,
                     int split_rule, int cap_out, float *out_lo, float *out_hi, float *out_lb, float *out_ub,
                     uint64_t *out_id, uint8_t *keep, int *d_counts, void *stream)
{
    if (c && split_rule != BAB_SPLIT_WIDEST) return fail(c, BAB_ERR_UNSUPPORTED, "split rule %d", split_rule);
    return prune_branch_impl(c, d, lo, hi, lb, ub, id, n, d_n, inc_val, n_pick, eta, split_rule, BAB_PICK_LB, 1.f, 0,
                             nullptr, nullptr, nullptr, nullptr, cap_out, out_lo, out_hi, out_lb, out_ub, out_id, keep,
                             d_counts, stream);
}

int bab_prune_branch_heuristic(bab_ctx *c, int d, const float *lo, const float *hi, const float *lb, const float *ub,
                               const uint64_t *id, int n, const int *d_n, const double *inc_val, int n_pick,
                               float eta, int pick_rule, float temperature, uint64_t pick_seed, const int *split_dim,
                               int cap_out, float *out_lo, float *out_hi, float *out_lb, float *out_ub,
                               uint64_t *out_id, int *out_split_dim, const float *row_u, float *out_row_u,
                               uint8_t *keep, int *d_counts, void *stream)
{
    if (!c) return BAB_ERR_INVALID_ARG;
    if (pick_rule != BAB_PICK_LB && pick_rule != BAB_PICK_SOFTMAX) return fail(c, BAB_ERR_INVALID_ARG, "pick rule %d", pick_rule);
    if (!(temperature > 0.f) || !std::isfinite(temperature)) return fail(c, BAB_ERR_INVALID_ARG, "temperature must be > 0");
    if ((row_u == nullptr) != (out_row_u == nullptr))
        return fail(c, BAB_ERR_INVALID_ARG, "row_u and out_row_u go together");
    return prune_branch_impl(c, d, lo, hi, lb, ub, id, n, d_n, inc_val, n_pick, eta, BAB_SPLIT_WIDEST, pick_rule,
                             temperature, pick_seed, split_dim, out_split_dim, row_u, out_row_u, cap_out, out_lo,
                             out_hi, out_lb, out_ub, out_id, keep, d_counts, stream);
}

}  // extern "C"

namespace {
int prune_branch_impl(bab_ctx *c, int d, const float *lo, const float *hi, const float *lb, const float *ub,
                      const uint64_t *id, int n, const int *d_n, const double *inc_val, int n_pick, float eta,
                      int split_rule, int pick_rule, float temperature, uint64_t pick_seed, const int *split_dim,
                      int *out_split_dim, const float *row_u, float *out_row_u, int cap_out, float *out_lo,
                      float *out_hi, float *out_lb, float *out_ub, uint64_t *out_id, uint8_t *keep, int *d_counts,
                      void *stream)
{
    if (!c) return BAB_ERR_INVALID_ARG;
    c->err[0] = 0;
    if (d < 1 || n < 0 || n_pick < 0) return fail(c, BAB_ERR_SHAPE, "bad d, n or n_pick");
    if (!(eta >= 0.f && eta <= 1.f)) return fail(c, BAB_ERR_INVALID_ARG, "eta must be in [0, 1]");
    if (split_rule != BAB_SPLIT_WIDEST) return fail(c, BAB_ERR_UNSUPPORTED, "split rule %d", split_rule);
    if (!inc_val || !d_counts) return fail(c, BAB_ERR_INVALID_ARG, "inc_val and d_counts are required");
    if (n > 0 && (!lo || !hi || !lb || !ub || !id || !keep || !out_lo || !out_hi || !out_lb || !out_ub || !out_id))
        return fail(c, BAB_ERR_INVALID_ARG, "null array");
    if ((long long)cap_out < (long long)n + n_pick) return fail(c, BAB_ERR_SHAPE, "cap_out must be >= n + n_pick");
    const size_t rows = ((size_t)(n > 0 ? n : 1) + 63) / 64 * 64;
    int rc = ensure_scratch(c, rows * (sizeof(int) + sizeof(float)) + 1024);
    if (rc) return rc;
    BranchArgs a{};
    a.batch.P = 1;
    a.cap_out = cap_out;
    a.eta = eta;
    a.poff = reinterpret_cast<int *>(c->scratch) + rows;
    a.pick_rule = pick_rule;
    a.temperature = temperature;
    a.pick_seed = pick_seed;
    a.pick_keys = reinterpret_cast<float *>(reinterpret_cast<int *>(c->scratch) + rows + 64);
    a.split_dim = split_dim;
    a.out_split_dim = out_split_dim;
    a.row_u = row_u;
    a.out_row_u = out_row_u;
    a.d = d;
    a.n = n;
    a.d_n = d_n;
    a.lo = lo;
    a.hi = hi;
    a.lb = lb;
    a.ub = ub;
    a.id = id;
    a.inc_val = inc_val;
    a.n_pick = n_pick;
    int n1 = (int)std::ceil((double)eta * n_pick);
    a.n1 = n1 > n_pick ? n_pick : n1;
    a.out_lo = out_lo;
    a.out_hi = out_hi;
    a.out_lb = out_lb;
    a.out_ub = out_ub;
    a.out_id = out_id;
    a.keep = keep;
    a.d_counts = d_counts;
    a.dest = reinterpret_cast<int *>(c->scratch);
    a.status = c->d_status;
    cudaError_t e = launch_prune_branch(a, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "prune/branch kernels");
    return BAB_OK;
}
}  // namespace

extern "C" {

// ---------------------------------------------------------------------------
// Batched problems (one launch per kernel for every problem of the context)
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

int check_batch(bab_ctx *c, const float *x0, const float *goal, const int *horizon, const float *rho, int max_horizon,
                int d_stride, const float *lo, const float *hi, const int *prob, int n)
{
    if (!c) return BAB_ERR_INVALID_ARG;
    c->err[0] = 0;
    if (c->cost.kind != 0) return refuse_obstacles(c, "batched problems");
    if (!x0 || !goal || !horizon) return fail(c, BAB_ERR_INVALID_ARG, "x0, goal and horizon are required");
    if (max_horizon < 1 || max_horizon > (1 << 20)) return fail(c, BAB_ERR_SHAPE, "max_horizon out of range");
    if (n < 0) return fail(c, BAB_ERR_SHAPE, "n = %d < 0", n);
    if ((long long)d_stride < (long long)c->net.k * max_horizon || d_stride > (1 << 24))
        return fail(c, BAB_ERR_SHAPE, "d_stride must be >= action_dim * max_horizon");
    if (n > 0 && (!lo || !hi)) return fail(c, BAB_ERR_INVALID_ARG, "lo and hi are required");
    if (c->n_problems > 1 && n > 0 && !prob) return fail(c, BAB_ERR_INVALID_ARG, "prob is required");
    (void)rho;
    return BAB_OK;
}

BatchDesc make_batch(bab_ctx *c, const int *prob, const int *horizon, const float *rho, int max_horizon)
{
    BatchDesc b{};
    b.prob = prob;
    b.H = horizon;
    b.rho = rho;
    b.P = c->n_problems;
    b.Hmax = max_horizon;
    return b;
}

}  // namespace

extern "C" {

int bab_rollout_batch(bab_ctx *c, const float *x0, const float *goal, const int *horizon, const float *rho,
                      int max_horizon, int d_stride, const float *lo, const float *hi, const uint64_t *id,
                      const int *prob, int n, const int *d_n, int samples, uint64_t seed, int precision, float *ub,
                      float *best_u, double *inc_val, float *inc_u, void *stream)
{
    int rc = check_batch(c, x0, goal, horizon, rho, max_horizon, d_stride, lo, hi, prob, n);
    if (rc) return rc;
    if (samples < 1) return fail(c, BAB_ERR_SHAPE, "samples must be >= 1");
    if (precision != BAB_PREC_FP32 && precision != BAB_PREC_BF16X3 && precision != BAB_PREC_BF16)
        return fail(c, BAB_ERR_INVALID_ARG, "unknown precision %d", precision);
    const int split = precision == BAB_PREC_BF16X3 ? 3 : 1;
    if (precision != BAB_PREC_FP32 && (!rollout_tc_supported(c->net, split, c->max_smem) ||
                                       (c->n_problems > 1 && samples < 128)))
        return fail(c, BAB_ERR_UNSUPPORTED, "tensor-core rollout of batched problems needs a supported network "
                                            "and >= 128 samples per box");
    if (n > 0 && (!id || !ub)) return fail(c, BAB_ERR_INVALID_ARG, "id and ub are required");
    if ((inc_val == nullptr) != (inc_u == nullptr)) return fail(c, BAB_ERR_INVALID_ARG, "inc_val and inc_u go together");
    if (inc_val && !best_u) return fail(c, BAB_ERR_INVALID_ARG, "the incumbent update needs best_u");
    if (n == 0) return BAB_OK;
    rc = ensure_scratch(c, (size_t)n * sizeof(unsigned long long) + 256);
    if (rc) return rc;
    RolloutArgs a{};
    a.cost = c->cost;
    a.net = c->net;
    a.batch = make_batch(c, prob, horizon, rho, max_horizon);
    a.fwd = c->d_fwd;
    a.raw = c->d_raw;
    a.x0 = x0;
    a.goal = goal;
    a.lo = lo;
    a.hi = hi;
    a.id = id;
    a.n = n;
    a.d_n = d_n;
    a.H = max_horizon;
    a.M = samples;
    a.d = d_stride;
    a.rho = 0.f;
    a.seed = seed;
    a.keys = reinterpret_cast<unsigned long long *>(c->scratch);
    a.ub = ub;
    a.best_u = best_u;
    a.inc_val = inc_val;
    a.inc_u = inc_u;
    a.status = c->d_status;
    a.tc_img = c->d_tc;
    a.tc_bias = c->d_tc_bias;
    a.tc_bytes = c->net.tc_bytes;
    cudaError_t e = precision == BAB_PREC_FP32
                        ? launch_rollout_fp32(a, c->tune_rollout_fp32, c->num_sms, (cudaStream_t)stream)
                        : launch_rollout_tc(a, split, c->tune_rollout_tc, c->num_sms, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "batched rollout kernels");
    return BAB_OK;
}

int bab_bound_batch(bab_ctx *c, const float *x0, const float *goal, const int *horizon, const float *rho,
                    int max_horizon, int d_stride, const float *lo, const float *hi, const int *prob, int n,
                    const int *d_n, int alpha_steps, float lr, float *lb, float *lb_ibp, void *stream)
{
    int rc = check_batch(c, x0, goal, horizon, rho, max_horizon, d_stride, lo, hi, prob, n);
    if (rc) return rc;
    if (n > 0 && !lb) return fail(c, BAB_ERR_INVALID_ARG, "lb is required");
    if (alpha_steps < 0 || alpha_steps > 100000) return fail(c, BAB_ERR_INVALID_ARG, "alpha_steps out of range");
    if (!(lr >= 0.f) || !std::isfinite(lr)) return fail(c, BAB_ERR_INVALID_ARG, "bad learning rate");
    if (n == 0) return BAB_OK;
    const NetDesc &N = c->net;
    const size_t nh = (size_t)n * max_horizon * N.sumh, nx = (size_t)n * (max_horizon + 1) * N.s;
    const size_t ns = (size_t)n * max_horizon * (N.sumh + N.s);
    const size_t floats = 2 * nh + 2 * nx + ns + (alpha_steps > 0 ? 4 * nh : 0);
    rc = ensure_scratch(c, floats * sizeof(float) + 16 * 256);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    BoundArgs a = make_bound_args(c, x0, goal, max_horizon, 0.f, lo, hi, n, d_n);
    a.d = d_stride;
    a.batch = make_batch(c, prob, horizon, rho, max_horizon);
    Carver cv{reinterpret_cast<char *>(c->scratch)};
    a.pre_lo = cv.take<float>(nh);
    a.pre_hi = cv.take<float>(nh);
    a.x_lo = cv.take<float>(nx);
    a.x_hi = cv.take<float>(nx);
    a.S = cv.take<float>(ns);
    a.lb_ibp = lb_ibp;
    cudaError_t e = launch_ibp_warp(a, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "batched interval bounds");
    float *al = nullptr, *m = nullptr, *v = nullptr;
    if (alpha_steps > 0) {
        al = cv.take<float>(nh);
        m = cv.take<float>(nh);
        v = cv.take<float>(nh);
        a.A_pre = cv.take<float>(nh);
    }
    a.lb_best = lb;
    e = launch_alpha_warp(a, alpha_steps, lr, al, m, v, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "batched bound kernel");
    return BAB_OK;
}

int bab_prune_branch_batch(bab_ctx *c, int d_stride, const int *horizon, int max_horizon, const float *lo,
                           const float *hi, const float *lb, const float *ub, const uint64_t *id, const int *prob,
                           int n, const int *d_n, const double *inc_val, const int *n_pick, int max_pick_total,
                           float eta, int split_rule, int cap_out, float *out_lo, float *out_hi, float *out_lb,
                           float *out_ub, uint64_t *out_id, int *out_prob, uint8_t *keep, int *d_counts,
                           int *d_pcounts, void *stream)
{
    if (!c) return BAB_ERR_INVALID_ARG;
    c->err[0] = 0;
    const int P = c->n_problems;
    if (n < 0 || max_pick_total < 0 || max_horizon < 1) return fail(c, BAB_ERR_SHAPE, "bad n, max_pick_total or max_horizon");
    if ((long long)d_stride < (long long)c->net.k * max_horizon) return fail(c, BAB_ERR_SHAPE, "d_stride too small");
    if (!(eta >= 0.f && eta <= 1.f)) return fail(c, BAB_ERR_INVALID_ARG, "eta must be in [0, 1]");
    if (split_rule != BAB_SPLIT_WIDEST) return fail(c, BAB_ERR_UNSUPPORTED, "split rule %d", split_rule);
    if (!inc_val || !d_counts || !n_pick || !horizon) return fail(c, BAB_ERR_INVALID_ARG, "inc_val, n_pick, horizon and d_counts are required");
    if (n > 0 && (!lo || !hi || !lb || !ub || !id || !keep || !out_lo || !out_hi || !out_lb || !out_ub || !out_id ||
                  (P > 1 && !prob)))
        return fail(c, BAB_ERR_INVALID_ARG, "null array");
    if ((long long)cap_out < (long long)n + max_pick_total)
        return fail(c, BAB_ERR_SHAPE, "cap_out must be >= n + max_pick_total");
    const size_t nrow = (size_t)(n > 0 ? n : 1);
    const size_t dest_ints = (nrow + 63) / 64 * 64;
    int rc = ensure_scratch(c, (dest_ints + 4 * (size_t)P) * sizeof(int) + 1024);
    if (rc) return rc;
    BranchArgs a{};
    a.batch = make_batch(c, prob, horizon, nullptr, max_horizon);
    a.k = c->net.k;
    a.d = d_stride;
    a.n = n;
    a.d_n = d_n;
    a.lo = lo;
    a.hi = hi;
    a.lb = lb;
    a.ub = ub;
    a.id = id;
    a.inc_val = inc_val;
    a.n_pick_dev = n_pick;
    a.eta = eta;
    a.cap_out = cap_out;
    a.out_lo = out_lo;
    a.out_hi = out_hi;
    a.out_lb = out_lb;
    a.out_ub = out_ub;
    a.out_id = out_id;
    a.out_prob = out_prob;
    a.keep = keep;
    a.d_counts = d_counts;
    a.dest = reinterpret_cast<int *>(c->scratch);
    a.poff = a.dest + dest_ints;
    a.pcounts = d_pcounts ? d_pcounts : a.poff + 2 * P;
    a.status = c->d_status;
    cudaError_t e = launch_prune_branch(a, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "batched prune/branch kernels");
    return BAB_OK;
}

int bab_set_variant(bab_ctx *c, int kernel, int variant)
{
    if (!c) return BAB_ERR_INVALID_ARG;
    c->err[0] = 0;
    switch (kernel) {
        case BAB_KERNEL_ROLLOUT_FP32:
            if (variant < -1 || variant >= rollout_fp32_variants()) break;
            c->tune_rollout_fp32 = variant;
            return BAB_OK;
        case BAB_KERNEL_ALPHA_FUSED:
            if (variant < -2 || variant > 3) break;
            c->tune_alpha_fused = variant;
            return BAB_OK;
        case BAB_KERNEL_ROLLOUT_TC:
            if (variant < -1 || variant == 0 || variant > 4) break;
            c->tune_rollout_tc = variant;
            return BAB_OK;
        case BAB_KERNEL_CROWN_TC:
            if (variant < -1 || variant > 4) break;
            c->tune_crown_tc = variant;
            return BAB_OK;
        default:
            return fail(c, BAB_ERR_INVALID_ARG, "unknown kernel %d", kernel);
    }
    return fail(c, BAB_ERR_INVALID_ARG, "variant %d out of range for kernel %d", variant, kernel);
}

int bab_set_interval_precision(bab_ctx *c, int precision)
{
    if (!c) return BAB_ERR_INVALID_ARG;
    c->err[0] = 0;
    if (precision == BAB_PREC_FP32) {
        c->interval_precision = precision;
        return BAB_OK;
    }
    if (precision != BAB_PREC_BF16X3 && precision != BAB_PREC_TF32X3)
        return fail(c, BAB_ERR_INVALID_ARG, "interval precision %d unknown", precision);
    if (c->n_problems > 1 || !ibp_tc_supported(c->net, c->max_smem))
        return fail(c, BAB_ERR_UNSUPPORTED, "tensor-core interval bounds need one network with every width at most 256");
    c->interval_precision = precision;
    return BAB_OK;
}

int bab_set_scratch_limit(bab_ctx *c, size_t bytes)
{
    if (!c) return BAB_ERR_INVALID_ARG;
    c->err[0] = 0;
    c->scratch_limit = bytes;
    if (bytes > 0 && c->scratch_bytes > bytes) {
        // give back a larger scratch now; the next call allocates what it needs within the limit
        cudaDeviceSynchronize();
        cudaFree(c->scratch);
        c->scratch = nullptr;
        c->scratch_bytes = 0;
    }
    return BAB_OK;
}

int bab_set_rescore_topk(bab_ctx *c, int k)
{
    if (!c) return BAB_ERR_INVALID_ARG;
    c->err[0] = 0;
    if (k < 0) return fail(c, BAB_ERR_INVALID_ARG, "k must be >= 0");
    c->rescore_topk = k;
    return BAB_OK;
}

int bab_get_variant(bab_ctx *c, int kernel, int *variant)
{
    if (!c || !variant) return BAB_ERR_INVALID_ARG;
    switch (kernel) {
        case BAB_KERNEL_ROLLOUT_FP32: *variant = c->tune_rollout_fp32; return BAB_OK;
        case BAB_KERNEL_ALPHA_FUSED: *variant = c->tune_alpha_fused; return BAB_OK;
        case BAB_KERNEL_ROLLOUT_TC: *variant = c->tune_rollout_tc; return BAB_OK;
        case BAB_KERNEL_CROWN_TC: *variant = c->tune_crown_tc; return BAB_OK;
        default: return fail(c, BAB_ERR_INVALID_ARG, "unknown kernel %d", kernel);
    }
}

}  // extern "C"

namespace {

// Mean milliseconds of `reps` runs of fn after one warm-up run; a negative value if fn fails.
template <typename F>
float time_call(cudaStream_t st, int reps, F fn)
{
    if (fn() != BAB_OK) return -1.f;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1.f;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return -1.f;
    }
    float ms = -1.f;
    bool ok = cudaEventRecord(e0, st) == cudaSuccess;
    for (int i = 0; i < reps && ok; ++i) ok = fn() == BAB_OK;
    ok = ok && cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
         cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ok ? ms / reps : -1.f;
}

// Times each candidate (set(v) then the call) and keeps the fastest; the setting is left at the winner,
// or at `fallback` when every candidate failed.
template <typename Set, typename F>
int pick_fastest(bab_ctx *c, cudaStream_t st, const std::vector<int> &cands, int fallback, Set set, F fn)
{
    int best = fallback;
    float best_ms = -1.f;
    for (int v : cands) {
        set(v);
        const float ms = time_call(st, 3, fn);
        if (ms >= 0.f && (best_ms < 0.f || ms < best_ms)) {
            best_ms = ms;
            best = v;
        }
        c->err[0] = 0;
    }
    set(best);
    return best;
}

}  // namespace

extern "C" {

int bab_autotune(bab_ctx *c, const float *x0, const float *goal, int H, float rho, const float *lo, const float *hi,
                 const uint64_t *id, int n, int samples, int alpha_steps, void *stream)
{
    if (c && c->cost.kind != 0) return refuse_obstacles(c, "the autotuner");
    int rc = check_problem(c, x0, goal, H, rho, lo, hi, n);
    if (rc) return rc;
    if (n < 1 || !id) return fail(c, BAB_ERR_INVALID_ARG, "autotuning needs at least one box and its id");
    if (samples < 1) return fail(c, BAB_ERR_SHAPE, "samples must be >= 1");
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) == cudaSuccess && cap != cudaStreamCaptureStatusNone)
        return fail(c, BAB_ERR_INVALID_ARG, "bab_autotune cannot run inside a stream capture");
    const int d = c->net.k * H;
    float *buf = nullptr;
    const size_t floats = (size_t)n * (d + 2);
    cudaError_t e = cudaMalloc(&buf, floats * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(c, e, "autotune buffers");
    float *ub = buf, *lb = buf + n, *best_u = buf + 2 * (size_t)n;
    const uint64_t seed = 0x5eedull;

    pick_fastest(c, st, {0, 1, 2}, -1, [&](int v) { c->tune_rollout_fp32 = v; },
                 [&] { return bab_rollout(c, x0, goal, H, rho, lo, hi, id, n, nullptr, samples, seed, BAB_PREC_FP32, ub,
                                          best_u, nullptr, nullptr, stream); });
    const bool tc = c->net.tc_ok && rollout_tc_supported(c->net, 3, c->max_smem);
    if (tc)
        pick_fastest(c, st, {1, 2}, -1, [&](int v) { c->tune_rollout_tc = v; },
                     [&] { return bab_rollout(c, x0, goal, H, rho, lo, hi, id, n, nullptr, samples, seed,
                                              BAB_PREC_BF16X3, ub, best_u, nullptr, nullptr, stream); });
    if (crown_tc_supported(c->net, c->max_smem))
        pick_fastest(c, st, {4, 3, 0, 1, 2}, -1, [&](int v) { c->tune_crown_tc = v; },
                     [&] { return bab_bound_crown(c, x0, goal, H, rho, lo, hi, n, nullptr, nullptr, BAB_PREC_BF16X3, lb,
                                                  nullptr, nullptr, nullptr, stream); });
    if (alpha_steps > 0) {
        std::vector<int> cands{-2, 3};
        if (alpha_fused_fits(c->net, H, d))
            for (int v = 0; v < alpha_fused_variants(); ++v) cands.push_back(v);
        pick_fastest(c, st, cands, -1, [&](int v) { c->tune_alpha_fused = v; },
                     [&] { return bab_alpha_optimize(c, x0, goal, H, rho, lo, hi, n, nullptr, alpha_steps, 0.1f,
                                                     BAB_PREC_FP32, nullptr, lb, stream); });
    }
    e = cudaStreamSynchronize(st);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(c, e, "autotune");
    c->err[0] = 0;
    return BAB_OK;
}

}  // extern "C"
