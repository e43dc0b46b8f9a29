// rollout.cu -- sampled search (Section 3.3, batch_search with uniform samples)
// and the FP64 incumbent re-score (the incumbent update of Algorithm 2).
//
// k_rollout_fp32: a persistent kernel.  A tile is R samples of one box; a CTA
// keeps the whole forward network image in shared memory for all H steps and
// all of its tiles, and carries the R states x_t and running costs in shared
// memory.  Per step it draws u_t (counter-based, so nothing is read from
// memory), runs the L dense layers as register-blocked FP32 products over the
// tile, adds the residual, and reduces the per-row cost with warp shuffles.
// A tile's best (f, m) is folded into its box with a 64-bit atomicMin on
// (order(f) << 32 | m), which keeps the lowest m among equal values.
#include <cooperative_groups.h>

#include "bab_internal.cuh"
#include "kernels.cuh"

namespace bab {

__device__ __forceinline__ unsigned long long umin64(unsigned long long a, unsigned long long b) { return a < b ? a : b; }

template <int R, int NT, bool WSMEM, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_rollout_fp32(RolloutArgs a)
{
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    const NetDesc &N = a.net;
    const int s = N.s, k = N.k, L = N.L, d = a.d;
    const int ld = N.maxw_p;
    const float *img = a.fwd;
    float *p = sm;
    if (WSMEM) {
        for (int i = threadIdx.x; i < N.img_floats / 4; i += NT)
            smem4[i] = reinterpret_cast<const float4 *>(a.fwd)[i];
        img = sm;
        p += N.img_floats;
    }
    float *act0 = p; p += R * ld;
    float *act1 = p; p += R * ld;
    float *xs = p; p += R * pad4(s);
    float *us = p; p += R * pad4(k);
    float *blo = p; p += pad4(d);
    float *bhi = p; p += pad4(d);
    float *cost = p; p += R;
    float *goal = p; p += pad4(s);
    float *ps = p; p += 2 * R;  // pusher position per row (obstacle cost)
    __shared__ unsigned long long red[NT / 32];

    const int nlive = live_count(a.n, a.d_n);
    const int tpb = (a.M + R - 1) / R;
    const long long ntiles = (long long)nlive * tpb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int Kp1 = pad4(s + k);
    const bool emit = a.emp_pre_lo != nullptr;
    const int Hm = a.batch.Hmax;

    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int box = (int)(tile / tpb);
        const int m0 = (int)(tile % tpb) * R;
        const int rv = a.M - m0 < R ? a.M - m0 : R;  // rows holding real samples
        // the box's problem: its weights, start, goal, horizon and rho
        const int pb = row_problem(a.batch, box);
        if (!WSMEM) img = a.fwd + (size_t)pb * N.img_floats;
        const int Hb = problem_H(a.batch, pb, a.H), db = k * Hb;
        const float rho = problem_rho(a.batch, pb, a.rho);
        const float *x0 = a.x0 + (size_t)pb * s;
        __syncthreads();  // previous tile fully consumed
        for (int i = threadIdx.x; i < s; i += NT) goal[i] = a.goal[(size_t)pb * s + i];
        for (int j = threadIdx.x; j < db; j += NT) {
            blo[j] = a.lo[(size_t)box * d + j];
            bhi[j] = a.hi[(size_t)box * d + j];
        }
        for (int i = threadIdx.x; i < R * s; i += NT) xs[(i / s) * pad4(s) + i % s] = x0[i % s];
        for (int r = threadIdx.x; r < R; r += NT) {
            cost[r] = 0.f;
            ps[2 * r] = a.cost.p0x;
            ps[2 * r + 1] = a.cost.p0y;
        }
        const uint64_t hb = box_hash(a.seed, a.id[box]);
        __syncthreads();
        for (int t = 0; t < Hb; ++t) {
            // input rows [x_t | u_t | 0]
            for (int i = threadIdx.x; i < R * Kp1; i += NT) {
                const int r = i / Kp1, c = i % Kp1;
                float v;
                if (c < s) {
                    v = xs[r * pad4(s) + c];
                } else if (c < s + k) {
                    const int j = t * k + (c - s);
                    v = a.cem_mu ? cem_sample(hb, (uint32_t)a.cem_it, (uint32_t)(m0 + r), (uint32_t)j,
                                              a.cem_mu[(size_t)box * d + j], a.cem_sigma[(size_t)box * d + j], blo[j],
                                              bhi[j])
                                 : draw_sample(hb, (uint32_t)(m0 + r), (uint32_t)j, blo[j], bhi[j]);
                    us[r * pad4(k) + (c - s)] = v;
                } else {
                    v = 0.f;
                }
                act0[r * ld + c] = v;
            }
            __syncthreads();
            float *in = act0, *out = act1;
            for (int l = 1; l <= L; ++l) {
                const int Kp = pad4(N.dims[l - 1]), Np = pad4(N.dims[l]);
                dense_rows_auto<R, NT>(in, ld, img + N.fwd_w[l], img + N.fwd_b[l], Kp, Np, out, ld, l < L && !emit);
                __syncthreads();
                if (emit && l < L) {
                    // search-integrated bounds: the tile's extremes of each pre-activation, then the ReLU
                    const int dl = N.dims[l];
                    for (int c = threadIdx.x; c < Np; c += NT) {
                        float mn = INFINITY, mx = -INFINITY;
                        for (int r = 0; r < R; ++r) {
                            const float v = out[r * ld + c];
                            if (r < rv) {
                                mn = fminf(mn, v);
                                mx = fmaxf(mx, v);
                            }
                            out[r * ld + c] = fmaxf(v, 0.f);
                        }
                        if (c < dl) {
                            const size_t e = ((size_t)box * Hm + t) * N.sumh + N.hoff[l] + c;
                            atomicMin(&a.emp_pre_lo[e], float_order(mn));
                            atomicMax(&a.emp_pre_hi[e], float_order(mx));
                        }
                    }
                    __syncthreads();
                }
                float *tmp = in; in = out; out = tmp;
            }
            // `in` holds the network output: residual step and the step cost of each row (one thread per row,
            // state terms then action terms in index order, so the value has a plain sequential definition)
            for (int r = threadIdx.x; r < R; r += NT) {
                float c = 0.f;
                if (a.cost.kind == 0) {
                    for (int i = 0; i < s; ++i) {
                        const float x = xs[r * pad4(s) + i] + in[r * ld + i];
                        xs[r * pad4(s) + i] = x;
                        const float e = x - goal[i];
                        c = fmaf(e, e, c);
                    }
                } else {
                    // the pusher moves by u_t, then the state cost at t + 1 (Appendix D.4)
                    ps[2 * r] = __fadd_rn(ps[2 * r], us[r * pad4(k)]);
                    ps[2 * r + 1] = __fadd_rn(ps[2 * r + 1], us[r * pad4(k) + 1]);
                    for (int i = 0; i < s; ++i) xs[r * pad4(s) + i] = __fadd_rn(xs[r * pad4(s) + i], in[r * ld + i]);
                    c = obstacle_cost_f32(a.cost, t + 1, s, xs + r * pad4(s), goal, ps[2 * r], ps[2 * r + 1]);
                }
                for (int j = 0; j < k; ++j) {
                    const float u = us[r * pad4(k) + j];
                    c = fmaf(rho * u, u, c);
                }
                cost[r] += c;
            }
            __syncthreads();
            if (emit) {
                // search-integrated bounds of the state x_{t+1}
                for (int i = threadIdx.x; i < s; i += NT) {
                    float mn = INFINITY, mx = -INFINITY;
                    for (int r = 0; r < rv; ++r) {
                        const float v = xs[r * pad4(s) + i];
                        mn = fminf(mn, v);
                        mx = fmaxf(mx, v);
                    }
                    const size_t e = ((size_t)box * (Hm + 1) + t + 1) * s + i;
                    atomicMin(&a.emp_x_lo[e], float_order(mn));
                    atomicMax(&a.emp_x_hi[e], float_order(mx));
                }
            }
        }
        if (a.costs)
            for (int r = threadIdx.x; r < rv; r += NT) a.costs[(size_t)box * a.M + m0 + r] = cost[r];
        // best (f, m) of the tile
        unsigned long long best = ~0ull;
        for (int r = threadIdx.x; r < R; r += NT)
            if (m0 + r < a.M) best = umin64(best, ((unsigned long long)float_order(cost[r]) << 32) | (unsigned)(m0 + r));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = umin64(best, __shfl_xor_sync(0xFFFFFFFFu, best, o));
        if (lane == 0) red[warp] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long b = red[0];
            for (int w = 1; w < NT / 32; ++w) b = umin64(b, red[w]);
            atomicMin(&a.keys[box], b);
        }
    }
}

__global__ void k_fill_u64(unsigned long long *p, int n, unsigned long long v)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// ub[i] and best_u[i] from the packed per-box minimum; the argmin sample is re-drawn.
__global__ void k_rollout_finalize(RolloutArgs a)
{
    const int nlive = live_count(a.n, a.d_n);
    const int box = blockIdx.x;
    if (box >= nlive) return;
    const unsigned long long key = a.keys[box];
    const uint32_t m = (uint32_t)(key & 0xFFFFFFFFu);
    if (threadIdx.x == 0) a.ub[box] = float_unorder((uint32_t)(key >> 32));
    if (!a.best_u) return;
    const uint64_t hb = box_hash(a.seed, a.id[box]);
    const int db = a.net.k * problem_H(a.batch, row_problem(a.batch, box), a.H);
    for (int j = threadIdx.x; j < a.d; j += blockDim.x)
        a.best_u[(size_t)box * a.d + j] =
            j < db ? draw_sample(hb, m, (uint32_t)j, a.lo[(size_t)box * a.d + j], a.hi[(size_t)box * a.d + j]) : 0.f;
}

// Incumbent update: the box with the smallest ub (lowest index on ties) has its best_u re-evaluated in FP64; if the
// value beats *inc_val, it becomes the incumbent.  The FP64 rate of one SM (about one multiply-add per clock) sets
// the pace of a one-CTA evaluation, so a large network's row is evaluated by a cluster of kIncCTAs CTAs (a small
// one's by a cluster of one, which leaves the other SMs to the bounds that run beside it): every CTA keeps the whole
// layer input in its shared memory, computes its share of each layer's outputs (each output's sum split over ks
// lanes, strided over the inputs, and added across them by shuffles) and writes them into every CTA's shared memory
// (distributed shared memory); a cluster barrier closes each layer and each step's cost.  The control flow depends
// only on values every CTA of the cluster computes alike, so all of them reach the same barriers.
constexpr int kIncCTAs = 16;  // a non-portable cluster size; 8 where the GPU cannot place 16

__global__ void __launch_bounds__(256) k_incumbent_fp64(RolloutArgs a)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank(), ncta = (int)cluster.num_blocks();
    const NetDesc &N = a.net;
    const int nlive = live_count(a.n, a.d_n);
    // one cluster per problem: its rows, weights, start, goal, horizon, rho and incumbent
    const int pb = blockIdx.x / ncta;
    const float *raw = a.raw + (size_t)pb * N.raw_floats;
    const float *x0 = a.x0 + (size_t)pb * N.s, *goal = a.goal + (size_t)pb * N.s;
    const int Hb = problem_H(a.batch, pb, a.H);
    const float rho = problem_rho(a.batch, pb, a.rho);
    double *inc_val = a.inc_val + pb;
    float *inc_u = a.inc_u + (size_t)pb * a.d;
    __shared__ unsigned long long red[8];
    __shared__ double act[2][kMaxWidth + 4];
    __shared__ double xs[kMaxWidth];
    __shared__ double f_sh;
    __shared__ int row_sh;
    const int lane = threadIdx.x & 31;
    unsigned long long best = ~0ull;
    for (int i = threadIdx.x; i < nlive; i += blockDim.x)
        if (row_problem(a.batch, i) == pb)
            best = umin64(best, ((unsigned long long)float_order(a.ub[i]) << 32) | (unsigned)i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = umin64(best, __shfl_xor_sync(0xFFFFFFFFu, best, o));
    if (lane == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = red[0];
        for (int w = 1; w < 8; ++w) b = umin64(b, red[w]);
        row_sh = (b == ~0ull) ? -1 : (int)(b & 0xFFFFFFFFu);
        f_sh = 0.0;
    }
    __syncthreads();
    const int row = row_sh;
    if (row < 0) return;  // the same in every CTA of the cluster
    const float *u = a.best_u + (size_t)row * a.d;
    const int s = N.s, k = N.k;
    double px = (double)a.cost.p0x, py = (double)a.cost.p0y;  // pusher position (obstacle cost; thread 0)
    for (int i = threadIdx.x; i < s; i += blockDim.x) xs[i] = (double)x0[i];
    __syncthreads();
    for (int t = 0; t < Hb; ++t) {
        for (int c = threadIdx.x; c < s + k; c += blockDim.x)
            act[0][c] = c < s ? xs[c] : (double)u[t * k + (c - s)];
        __syncthreads();
        int cur = 0;
        for (int l = 1; l <= N.L; ++l) {
            const int no = N.dims[l], ni = N.dims[l - 1];
            const float *W = raw + N.raw_w[l];
            const float *b = raw + N.raw_b[l];
            // this CTA's outputs q0 .. q0 + chunk - 1 (chunk <= 256, the widest layer): cp >= chunk slots of ks
            // lanes each (ks a power of two, at most 32, cp ks <= 256 threads)
            const int chunk = (no + ncta - 1) / ncta, q0 = rank * chunk;
            int cp = 1;
            while (cp < chunk) cp *= 2;
            const int ks = 256 / cp > 32 ? 32 : 256 / cp;
            const int ql = (int)threadIdx.x / ks, sl = (int)threadIdx.x % ks, q = q0 + ql;
            const bool mine = ql < chunk && q < no;
            double part = 0.0;
            if (mine)
                for (int c = sl; c < ni; c += ks) part = fma((double)W[(size_t)q * ni + c], act[cur][c], part);
            for (int o = ks / 2; o > 0; o >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
            if (mine && sl == 0) {
                double v = (double)b[q] + part;
                if (l < N.L && v < 0.0) v = 0.0;
                for (int r2 = 0; r2 < ncta; ++r2) cluster.map_shared_rank(&act[cur ^ 1][0], r2)[q] = v;
            }
            cluster.sync();  // every CTA's copy of the layer output complete
            cur ^= 1;
        }
        if (threadIdx.x == 0) {
            double f = f_sh;
            for (int i = 0; i < s; ++i) xs[i] += act[cur][i];
            if (a.cost.kind == 0) {
                for (int i = 0; i < s; ++i) {
                    const double e = xs[i] - (double)goal[i];
                    f += e * e;
                }
            } else {
                px += (double)u[t * k];
                py += (double)u[t * k + 1];
                f += obstacle_cost_f64(a.cost, t + 1, s, xs, goal, px, py);
            }
            for (int j = 0; j < k; ++j) {
                const double uu = (double)u[t * k + j];
                f += (double)rho * uu * uu;
            }
            f_sh = f;
        }
        cluster.sync();  // the output read before the next step's first layer overwrites it
    }
    if (rank != 0) return;
    if (threadIdx.x == 0) row_sh = (f_sh < *inc_val) ? 1 : 0;
    __syncthreads();
    if (row_sh) {
        for (int j = threadIdx.x; j < a.d; j += blockDim.x) inc_u[j] = u[j];
        if (threadIdx.x == 0) *inc_val = f_sh;
    }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static size_t rollout_smem_bytes(const NetDesc &N, int R, int d, bool wsmem)
{
    size_t f = (wsmem ? (size_t)N.img_floats : 0) + 2 * (size_t)R * N.maxw_p + (size_t)R * pad4(N.s) +
               (size_t)R * pad4(N.k) + 2 * (size_t)pad4(d) + R + pad4(N.s) + 2 * (size_t)R;
    return f * sizeof(float);
}

template <int R, int NT, int MINB>
static cudaError_t launch_fp32_variant(const RolloutArgs &a, int num_sms, size_t budget, cudaStream_t st)
{
    // several problems: every tile reads its own problem's image through L1 / L2
    bool wsmem = a.batch.P <= 1 && rollout_smem_bytes(a.net, R, a.d, true) <= budget;
    size_t smem = rollout_smem_bytes(a.net, R, a.d, wsmem);
    if (smem > budget) return cudaErrorInvalidConfiguration;
    auto kern = wsmem ? k_rollout_fp32<R, NT, true, MINB> : k_rollout_fp32<R, NT, false, MINB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const long long ntiles = (long long)a.n * ((a.M + R - 1) / R);
    const long long slots = (long long)num_sms * occ;
    const int grid = (int)(ntiles < slots ? ntiles : slots);
    kern<<<grid, NT, smem, st>>>(a);
    return cudaGetLastError();
}

int rollout_fp32_variants() { return 3; }

// variant 0: 64 samples x 256 threads per CTA, one CTA per SM (large networks, weights in shared memory);
// variant 1: 64 x 256 with at most 128 registers (two or more CTAs per SM for small networks);
// variant 2: 32 x 128, at most 128 registers.
cudaError_t launch_rollout_fp32(const RolloutArgs &a, int variant, int num_sms, cudaStream_t st)
{
    int dev;
    cudaGetDevice(&dev);
    int max_optin = 0;
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t budget = (size_t)max_optin - 1024;  // room for static shared memory
    if (rollout_smem_bytes(a.net, 64, a.d, false) > budget) return cudaErrorInvalidConfiguration;
    if (a.n <= 0) return cudaSuccess;
    if (variant < 0) {
        // default: the register-capped variant once two CTAs' shared memory fits on an SM
        variant = rollout_smem_bytes(a.net, 64, a.d, true) * 2 + 2048 <= (size_t)max_optin ? 1 : 0;
    }
    k_fill_keys(a.keys, a.n, st);
    cudaError_t e;
    switch (variant) {
        case 1: e = launch_fp32_variant<64, 256, 2>(a, num_sms, budget, st); break;
        case 2: e = launch_fp32_variant<32, 128, 4>(a, num_sms, budget, st); break;
        default: e = launch_fp32_variant<64, 256, 1>(a, num_sms, budget, st); break;
    }
    if (e != cudaSuccess) return e;
    if (a.cem_mu) return cudaGetLastError();  // the cross-entropy search keeps its own best (launch_cem_step)
    launch_rollout_finalize(a, st);
    if (a.inc_val) launch_incumbent(a, st);
    return cudaGetLastError();
}

// Search-integrated bounds: key arrays start at the identities of min / max; after the rollout the keys turn
// back into floats in place, and x_0 (known exactly) is written.
__global__ void k_emp_init(uint32_t *lo, uint32_t *hi, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        lo[i] = 0xFFFFFFFFu;
        hi[i] = 0u;
    }
}

__global__ void k_emp_finish(uint32_t *lo, uint32_t *hi, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        lo[i] = __float_as_uint(float_unorder(lo[i]));
        hi[i] = __float_as_uint(float_unorder(hi[i]));
    }
}

__global__ void k_emp_x0(const RolloutArgs a)
{
    const int nlive = live_count(a.n, a.d_n), s = a.net.s, Hm = a.batch.Hmax;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)nlive * s;
         i += (long long)gridDim.x * blockDim.x) {
        const long long box = i / s;
        const int c = (int)(i % s);
        const float v = a.x0[(size_t)row_problem(a.batch, (int)box) * s + c];
        a.emp_x_lo[(size_t)box * (Hm + 1) * s + c] = __float_as_uint(v);
        a.emp_x_hi[(size_t)box * (Hm + 1) * s + c] = __float_as_uint(v);
    }
}

void launch_emp_init(const RolloutArgs &a, cudaStream_t st)
{
    const long long nh = (long long)a.n * a.batch.Hmax * a.net.sumh, nx = (long long)a.n * (a.batch.Hmax + 1) * a.net.s;
    if (nh > 0) k_emp_init<<<1024, 256, 0, st>>>(a.emp_pre_lo, a.emp_pre_hi, nh);
    k_emp_init<<<1024, 256, 0, st>>>(a.emp_x_lo, a.emp_x_hi, nx);
}

void launch_emp_finish(const RolloutArgs &a, cudaStream_t st)
{
    const long long nh = (long long)a.n * a.batch.Hmax * a.net.sumh, nx = (long long)a.n * (a.batch.Hmax + 1) * a.net.s;
    if (nh > 0) k_emp_finish<<<1024, 256, 0, st>>>(a.emp_pre_lo, a.emp_pre_hi, nh);
    k_emp_finish<<<1024, 256, 0, st>>>(a.emp_x_lo, a.emp_x_hi, nx);
    k_emp_x0<<<256, 256, 0, st>>>(a);
}

void k_fill_keys(unsigned long long *keys, int n, cudaStream_t st)
{
    if (n > 0) k_fill_u64<<<(n + 255) / 256, 256, 0, st>>>(keys, n, ~0ull);
}

void launch_rollout_finalize(const RolloutArgs &a, cudaStream_t st)
{
    if (a.n > 0) k_rollout_finalize<<<a.n, 128, 0, st>>>(a);
}

void launch_incumbent(const RolloutArgs &a, cudaStream_t st)
{
    if (a.n <= 0) return;
    // a cluster of kIncCTAs (else 8) for rows of more than 2 M multiply-adds (at about one FP64 multiply-add per
    // clock, a millisecond on one SM), else one CTA per problem
    const NetDesc &N = a.net;
    long long macs = 0;
    for (int l = 1; l <= N.L; ++l) macs += (long long)N.dims[l] * N.dims[l - 1];
    int ncta = macs * a.H > 2000000 ? kIncCTAs : 1;
    // whether this GPU places a 16-CTA cluster of the kernel (non-portable size): decided at the first large launch,
    // which runs eagerly before any graph capture, and kept (one device per process)
    static int big_ok = -1;
    if (ncta > 8 && big_ok < 0) {
        big_ok = 0;
        if (cudaFuncSetAttribute(k_incumbent_fp64, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
            cudaLaunchConfig_t q = {};
            q.gridDim = dim3((unsigned)ncta);
            q.blockDim = dim3(256);
            cudaLaunchAttribute qa[1];
            qa[0].id = cudaLaunchAttributeClusterDimension;
            qa[0].val.clusterDim.x = (unsigned)ncta;
            qa[0].val.clusterDim.y = 1;
            qa[0].val.clusterDim.z = 1;
            q.attrs = qa;
            q.numAttrs = 1;
            int nclusters = 0;
            big_ok = cudaOccupancyMaxActiveClusters(&nclusters, k_incumbent_fp64, &q) == cudaSuccess && nclusters >= 1;
        }
        cudaGetLastError();
    }
    if (ncta > 8 && !big_ok) ncta = 8;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ncta * (a.batch.P > 1 ? a.batch.P : 1)));
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)ncta;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_incumbent_fp64, a);
}

}  // namespace bab
