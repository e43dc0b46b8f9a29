// cem.cu -- the cross-entropy search of Section 3.3 (batch_search with CEM,
// warm-started from the parent's best input), around the rollout kernels.
//
// Per box the search distribution is a diagonal normal (mu, sigma) over the
// box.  An iteration is one rollout launch in CEM mode (samples
// cem_sample(mu, sigma), every sample's objective written to costs) and one
// k_cem_step: rank the samples by (objective, index), keep the best sample so
// far, and refit mu and sigma to the E best.  Every quantity is formed in
// FP32 with one rounding per operation in a fixed order, so the search takes
// the same decisions as any implementation of the same definition.
#include "bab_internal.cuh"
#include "kernels.cuh"

namespace bab {

// mu = the warm start clipped to the box (or the box centre), sigma = (hi - lo) / 2, no best yet
__global__ void k_cem_init(CemArgs c, const float *warm)
{
    const int n = live_count(c.n, c.d_n);
    const size_t tot = (size_t)n * c.d;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += stride) {
        const float lo = c.lo[e], hi = c.hi[e];
        c.mu[e] = warm ? fminf(fmaxf(warm[e], lo), hi) : __fmul_rn(0.5f, __fadd_rn(lo, hi));
        c.sigma[e] = __fmul_rn(0.5f, __fsub_rn(hi, lo));
    }
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)n; i += stride) c.best[i] = ~0ull;
}

// One CTA per box: bitonic sort of the keys (order(f), m) in shared memory (NaN last, ties by m), the best
// sample so far (a strictly smaller objective replaces it, so ties keep the earlier iteration), then the refit
// of every coordinate to the E best samples in rank order.
__global__ void __launch_bounds__(256) k_cem_step(CemArgs c)
{
    extern __shared__ unsigned long long key[];
    const int n = live_count(c.n, c.d_n);
    const int box = blockIdx.x;
    if (box >= n) return;
    int P2 = 1;
    while (P2 < c.M) P2 <<= 1;
    for (int m = threadIdx.x; m < P2; m += blockDim.x) {
        unsigned long long kk = ~0ull;
        if (m < c.M) {
            const float f = __fadd_rn(c.costs[(size_t)box * c.M + m], 0.f);  // -0 -> +0, so equal values tie
            kk = ((unsigned long long)float_order(f) << 32) | (unsigned)m;
        }
        key[m] = kk;
    }
    __syncthreads();
    for (int kk = 2; kk <= P2; kk <<= 1)
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P2; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const unsigned long long x = key[i], y = key[l];
                    if ((x > y) == ((i & kk) == 0)) {
                        key[i] = y;
                        key[l] = x;
                    }
                }
            }
            __syncthreads();
        }
    const uint64_t hb = box_hash(c.seed, c.id[box]);
    const uint32_t it = (uint32_t)c.it;
    const unsigned long long k0 = key[0];
    const uint32_t m0 = (uint32_t)(k0 & 0xFFFFFFFFu);
    const unsigned long long prev = c.best[box];
    const bool take = prev == ~0ull || (uint32_t)(k0 >> 32) < (uint32_t)(prev >> 32);
    const size_t row = (size_t)box * c.d;
    if (take) {
        if (threadIdx.x == 0) {
            c.best[box] = (k0 & 0xFFFFFFFF00000000ull) | (unsigned)(it * (uint32_t)c.M + m0);
            c.ub[box] = __fadd_rn(c.costs[(size_t)box * c.M + m0], 0.f);
        }
        for (int j = threadIdx.x; j < c.d; j += blockDim.x)
            c.best_u[row + j] = cem_sample(hb, it, m0, (uint32_t)j, c.mu[row + j], c.sigma[row + j], c.lo[row + j],
                                           c.hi[row + j]);
    }
    __syncthreads();
    const float Ef = (float)c.E;
    for (int j = threadIdx.x; j < c.d; j += blockDim.x) {
        const float mu = c.mu[row + j], sg = c.sigma[row + j], lo = c.lo[row + j], hi = c.hi[row + j];
        float sum = 0.f;
        for (int q = 0; q < c.E; ++q)
            sum = __fadd_rn(sum, cem_sample(hb, it, (uint32_t)(key[q] & 0xFFFFFFFFu), (uint32_t)j, mu, sg, lo, hi));
        const float mean = __fdiv_rn(sum, Ef);
        float acc = 0.f;
        for (int q = 0; q < c.E; ++q) {
            const float dv =
                __fsub_rn(cem_sample(hb, it, (uint32_t)(key[q] & 0xFFFFFFFFu), (uint32_t)j, mu, sg, lo, hi), mean);
            acc = fmaf(dv, dv, acc);
        }
        c.mu[row + j] = mean;
        c.sigma[row + j] = __fadd_rn(__fsqrt_rn(__fdiv_rn(acc, Ef)), c.jitter);
    }
}

cudaError_t launch_cem_init(const CemArgs &c, const float *warm_u, cudaStream_t st)
{
    if (c.n <= 0) return cudaSuccess;
    const size_t tot = (size_t)c.n * c.d;
    int grid = (int)((tot + 255) / 256);
    grid = grid > 4096 ? 4096 : grid;
    k_cem_init<<<grid, 256, 0, st>>>(c, warm_u);
    return cudaGetLastError();
}

cudaError_t launch_cem_step(const CemArgs &c, cudaStream_t st)
{
    if (c.n <= 0) return cudaSuccess;
    int P2 = 1;
    while (P2 < c.M) P2 <<= 1;
    k_cem_step<<<c.n, 256, (size_t)P2 * sizeof(unsigned long long), st>>>(c);
    return cudaGetLastError();
}

}  // namespace bab
