// synth.cu -- the paper's synthetic objective (Section 4, synthetic example),
// f(u) = sum_i 5 u_i^2 + cos(50 u_i) over boxes of [-1, 1]^d, as a second
// objective for the same branch-and-bound machinery (search, bound, prune,
// pick-out, bisect):
//
//   k_synth_search     one thread per sample: uniform draws (the counter
//                      sampler of the rollouts) or the cross-entropy mode
//                      (cem_sample of the box's mean and spread); f in FP32;
//                      per box the packed minimum (order(f), m), every sample's
//                      value to costs when asked.
//   k_synth_finalize   ub and the argmin sample re-drawn.
//   k_synth_bound      one warp per box: the sum over coordinates of the exact
//                      minima of 5 u^2 over [lo, hi] and of cos(50 u) over
//                      [50 lo, 50 hi] (-1 when an odd multiple of pi lies in
//                      the interval, else the smaller end value), rounded
//                      outward: directed rounding for the products and the sum,
//                      and the interval's ends widened before cosf, whose error
//                      (2 ulp) is covered by subtracting 2^-21 per coordinate.
//   k_synth_incumbent  the best row's input re-evaluated in FP64.
#include "bab_internal.cuh"
#include "kernels.cuh"

namespace bab {

constexpr double kPi = 3.14159265358979323846;

struct SynthArgs {
    int d, n, M, it;
    const int *d_n;
    const float *lo, *hi;
    const uint64_t *id;
    uint64_t seed;
    const float *cem_mu, *cem_sigma;  // nullable: uniform draws
    unsigned long long *keys;          // [n]
    float *costs;                      // [n][M] (nullable)
    float *ub, *best_u;
    double *inc_val;
    float *inc_u;
};

__device__ __forceinline__ float synth_term(float u)
{
    return __fadd_rn(__fmul_rn(__fmul_rn(5.f, u), u), cosf(__fmul_rn(50.f, u)));
}

__global__ void __launch_bounds__(256) k_synth_search(SynthArgs a)
{
    const int n = live_count(a.n, a.d_n);
    const int tpb = (a.M + 255) / 256;
    const int box = blockIdx.x / tpb;
    if (box >= n) return;
    const int m = (blockIdx.x % tpb) * 256 + threadIdx.x;
    const uint64_t hb = box_hash(a.seed, a.id[box]);
    const size_t row = (size_t)box * a.d;
    unsigned long long key = ~0ull;
    if (m < a.M) {
        float f = 0.f;
        for (int j = 0; j < a.d; ++j) {
            const float l = a.lo[row + j], h = a.hi[row + j];
            const float u = a.cem_mu ? cem_sample(hb, (uint32_t)a.it, (uint32_t)m, (uint32_t)j, a.cem_mu[row + j],
                                                  a.cem_sigma[row + j], l, h)
                                     : draw_sample(hb, (uint32_t)m, (uint32_t)j, l, h);
            f = __fadd_rn(f, synth_term(u));
        }
        if (a.costs) a.costs[(size_t)box * a.M + m] = f;
        key = ((unsigned long long)float_order(f) << 32) | (unsigned)m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long k2 = __shfl_xor_sync(0xFFFFFFFFu, key, o);
        key = k2 < key ? k2 : key;
    }
    if ((threadIdx.x & 31) == 0 && key != ~0ull) atomicMin(&a.keys[box], key);
}

__global__ void k_synth_finalize(SynthArgs a)
{
    const int n = live_count(a.n, a.d_n);
    const int box = blockIdx.x;
    if (box >= n) return;
    const unsigned long long key = a.keys[box];
    const uint32_t m = (uint32_t)(key & 0xFFFFFFFFu);
    if (threadIdx.x == 0) a.ub[box] = float_unorder((uint32_t)(key >> 32));
    const uint64_t hb = box_hash(a.seed, a.id[box]);
    const size_t row = (size_t)box * a.d;
    for (int j = threadIdx.x; j < a.d; j += blockDim.x)
        a.best_u[row + j] = draw_sample(hb, m, (uint32_t)j, a.lo[row + j], a.hi[row + j]);
}

__global__ void __launch_bounds__(256) k_synth_bound(int d, const float *lo, const float *hi, int n_, const int *d_n,
                                                     float *lb)
{
    const int n = live_count(n_, d_n);
    const int box = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (box >= n) return;
    const size_t row = (size_t)box * d;
    float acc = 0.f;
    for (int j = lane; j < d; j += 32) {
        const float l = lo[row + j], h = hi[row + j];
        const float m = (l <= 0.f && h >= 0.f) ? 0.f : fminf(fabsf(l), fabsf(h));
        const float sq = __fmul_rd(5.f, __fmul_rd(m, m));
        const float ca = __fmul_rd(50.f, l), cb = __fmul_ru(50.f, h);
        const double k = ceil(((double)ca / kPi - 1.0) * 0.5);  // smallest k with (2k + 1) pi >= ca
        float cm;
        if ((2.0 * k + 1.0) * kPi <= (double)cb)
            cm = -1.f;
        else
            cm = __fsub_rd(fminf(cosf(ca), cosf(cb)), 4.76837158203125e-07f);  // 2^-21
        acc = __fadd_rd(acc, __fadd_rd(sq, cm));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = __fadd_rd(acc, __shfl_xor_sync(0xFFFFFFFFu, acc, o));
    if (lane == 0) lb[box] = acc;
}

// The row of smallest ub (lowest index on ties) re-evaluated in FP64; it becomes the incumbent if better.
__global__ void __launch_bounds__(256) k_synth_incumbent(SynthArgs a)
{
    __shared__ unsigned long long red[8];
    __shared__ double part[8];
    const int n = live_count(a.n, a.d_n);
    unsigned long long best = ~0ull;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        best = min(best, ((unsigned long long)float_order(a.ub[i]) << 32) | (unsigned)i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xFFFFFFFFu, best, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    best = red[0];
    for (int w = 1; w < 8; ++w) best = min(best, red[w]);
    if (best == ~0ull) return;
    const int row = (int)(best & 0xFFFFFFFFu);
    const float *u = a.best_u + (size_t)row * a.d;
    double f = 0.0;
    for (int j = threadIdx.x; j < a.d; j += blockDim.x) {
        const double v = u[j];
        f += 5.0 * v * v + cos(50.0 * v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xFFFFFFFFu, f, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = f;
    __syncthreads();
    double tot = 0.0;
    for (int w = 0; w < 8; ++w) tot += part[w];
    const bool better = tot < *a.inc_val;
    __syncthreads();
    if (better) {
        for (int j = threadIdx.x; j < a.d; j += blockDim.x) a.inc_u[j] = u[j];
        if (threadIdx.x == 0) *a.inc_val = tot;
    }
}

cudaError_t launch_synth_search(int d, const float *lo, const float *hi, const uint64_t *id, int n, const int *d_n,
                                int M, int it, uint64_t seed, const float *cem_mu, const float *cem_sigma,
                                unsigned long long *keys, float *costs, float *ub, float *best_u, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    SynthArgs a{};
    a.d = d;
    a.n = n;
    a.d_n = d_n;
    a.M = M;
    a.it = it;
    a.lo = lo;
    a.hi = hi;
    a.id = id;
    a.seed = seed;
    a.cem_mu = cem_mu;
    a.cem_sigma = cem_sigma;
    a.keys = keys;
    a.costs = costs;
    a.ub = ub;
    a.best_u = best_u;
    if (!cem_mu) k_fill_keys(keys, n, st);
    const int tpb = (M + 255) / 256;
    k_synth_search<<<(unsigned)((long long)n * tpb), 256, 0, st>>>(a);
    if (!cem_mu) k_synth_finalize<<<n, 128, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_synth_bound(int d, const float *lo, const float *hi, int n, const int *d_n, float *lb, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_synth_bound<<<(n + 7) / 8, 256, 0, st>>>(d, lo, hi, n, d_n, lb);
    return cudaGetLastError();
}

cudaError_t launch_synth_incumbent(int d, const float *ub, const float *best_u, int n, const int *d_n, double *inc_val,
                                   float *inc_u, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    SynthArgs a{};
    a.d = d;
    a.n = n;
    a.d_n = d_n;
    a.ub = const_cast<float *>(ub);
    a.best_u = const_cast<float *>(best_u);
    a.inc_val = inc_val;
    a.inc_u = inc_u;
    k_synth_incumbent<<<1, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace bab
