// branch.cu -- Pruner, batch_pick_out and batch_split of Algorithm 2
// (Section 3 overview and Section 3.1), bit-exact and deterministic.
//
//   k_branch_plan   one CTA: the FP64 prune test, the pick-out selection (exact
//                   k-th smallest of the composite keys (order(ub), id) and
//                   (order(lb), id) by 8-bit radix selection), and the stable
//                   ranks of picked and unpicked survivors (warp ballots).
//   k_branch_write  one warp per pool row: the widest coordinate (warp
//                   argmax, lowest index on ties), the FP32 midpoint, and the
//                   coalesced writes of two children or of the unpicked row.
#include "bab_internal.cuh"
#include "kernels.cuh"
#include "select.cuh"

namespace bab {

constexpr int kPlanThreads = 1024;
constexpr int kPickFlag = 1 << 30;

__global__ void __launch_bounds__(kPlanThreads) k_branch_plan(BranchArgs a)
{
    __shared__ unsigned hist[256];
    __shared__ uint32_t sh_pk;
    __shared__ uint64_t sh_pid;
    __shared__ int sh_rem, sh_done;
    __shared__ int wsum[2][kPlanThreads / 32];
    __shared__ int red[kPlanThreads / 32];
    const int n = live_count(a.n, a.d_n);
    // this CTA's problem and its rows
    const int pb = blockIdx.x;
    const BatchDesc &B = a.batch;
    auto mine = [&](int i) { return B.prob == nullptr || row_problem(B, i) == pb; };
    const double inc = a.inc_val[pb];
    int n_pick = a.n_pick, n1 = a.n1;
    if (a.n_pick_dev) {
        n_pick = a.n_pick_dev[pb] < 0 ? 0 : a.n_pick_dev[pb];
        n1 = (int)ceil((double)a.eta * n_pick);
        n1 = n1 > n_pick ? n_pick : n1;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // prune (strict, in FP64; a NaN bound is kept and latched as BAB_ERR_NUMERIC)
    int cnt = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (!mine(i)) continue;
        const float lbi = a.lb[i];
        if (lbi != lbi) set_status(a.status, BAB_ERR_NUMERIC);
        const uint8_t k = !((double)lbi > inc);
        a.keep[i] = k;
        cnt += k;
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
    if (lane == 0) red[warp] = cnt;
    __syncthreads();
    int ns = 0;
    for (int w = 0; w < kPlanThreads / 32; ++w) ns += red[w];
    __syncthreads();

    const bool all = ns <= n_pick;
    Thresh T1, T2;
    T1.none = T2.none = true;
    // the rest of the quota is chosen on the lower bound, or on its softmax race key (pick_rule 1)
    const float *key2 = a.pick_rule == 1 ? a.pick_keys : a.lb;
    if (!all) {
        const uint8_t *keep = a.keep;
        T1 = radix_select(n, a.ub, a.id, [&](int i) { return mine(i) && keep[i] != 0; }, n1, hist, &sh_pk, &sh_pid,
                          &sh_rem, &sh_done);
        const float *ub = a.ub;
        const uint64_t *ids = a.id;
        auto cand = [&](int i) { return mine(i) && keep[i] != 0 && !le_thresh(float_order(ub[i]), ids[i], T1); };
        if (a.pick_rule == 1) {
            // min-max scaling over the candidates' (non-NaN) lower bounds, then each candidate's race key
            float mn = INFINITY, mx = -INFINITY;
            for (int i = threadIdx.x; i < n; i += blockDim.x)
                if (cand(i) && a.lb[i] == a.lb[i]) {
                    mn = fminf(mn, a.lb[i]);
                    mx = fmaxf(mx, a.lb[i]);
                }
            for (int o = 16; o > 0; o >>= 1) {
                mn = fminf(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
                mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
            }
            __shared__ float rmn[kPlanThreads / 32], rmx[kPlanThreads / 32];
            if (lane == 0) {
                rmn[warp] = mn;
                rmx[warp] = mx;
            }
            __syncthreads();
            mn = INFINITY;
            mx = -INFINITY;
            for (int w = 0; w < kPlanThreads / 32; ++w) {
                mn = fminf(mn, rmn[w]);
                mx = fmaxf(mx, rmx[w]);
            }
            for (int i = threadIdx.x; i < n; i += blockDim.x)
                if (cand(i)) {
                    const float v = a.lb[i];
                    a.pick_keys[i] = v == v ? pick_key(v, mn, mx, a.temperature, a.pick_seed, ids[i]) : v;
                }
            __syncthreads();
        }
        T2 = radix_select(n, key2, a.id, cand, n_pick - n1, hist, &sh_pk, &sh_pid, &sh_rem, &sh_done);
    }

    // stable ranks of picked and unpicked survivors
    int base_p = 0, base_r = 0;
    const unsigned lt = (1u << lane) - 1u;
    for (int c0 = 0; c0 < n; c0 += blockDim.x) {
        const int i = c0 + threadIdx.x;
        bool kp = false, pk = false;
        const bool own = i < n && mine(i);
        if (own) {
            kp = a.keep[i] != 0;
            const bool by_ub = le_thresh(float_order(a.ub[i]), a.id[i], T1);
            pk = kp && (all || by_ub || le_thresh(float_order(key2[i]), a.id[i], T2));
        }
        const bool rs = kp && !pk;
        const unsigned bp = __ballot_sync(0xFFFFFFFFu, pk), br = __ballot_sync(0xFFFFFFFFu, rs);
        if (lane == 0) {
            wsum[0][warp] = __popc(bp);
            wsum[1][warp] = __popc(br);
        }
        __syncthreads();
        int op = 0, orr = 0, tp = 0, tr = 0;
        for (int w = 0; w < kPlanThreads / 32; ++w) {
            if (w < warp) {
                op += wsum[0][w];
                orr += wsum[1][w];
            }
            tp += wsum[0][w];
            tr += wsum[1][w];
        }
        if (own) {
            if (pk) a.dest[i] = (base_p + op + __popc(bp & lt)) | kPickFlag;
            else if (rs) a.dest[i] = base_r + orr + __popc(br & lt);
            else a.dest[i] = -1;
        }
        base_p += tp;
        base_r += tr;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (gridDim.x == 1) {
            a.d_counts[0] = 2 * base_p;
            a.d_counts[1] = base_r;
            a.d_counts[2] = 2 * base_p + base_r;
            a.poff[0] = 0;
            a.poff[1] = 2 * base_p;
            if (a.pcounts) {
                a.pcounts[0] = base_p;
                a.pcounts[1] = base_r;
            }
        } else {
            a.pcounts[2 * pb] = base_p;
            a.pcounts[2 * pb + 1] = base_r;
        }
    }
}

// Several problems: output offsets of each problem's children and unpicked rows, and the totals.
__global__ void k_branch_offsets(BranchArgs a)
{
    if (threadIdx.x != 0) return;
    const int P = a.batch.P;
    long long tp = 0, tr = 0;
    for (int p = 0; p < P; ++p) {
        tp += a.pcounts[2 * p];
        tr += a.pcounts[2 * p + 1];
    }
    long long cp = 0, cr = 2 * tp;
    for (int p = 0; p < P; ++p) {
        a.poff[2 * p] = (int)cp;
        a.poff[2 * p + 1] = (int)cr;
        cp += 2 * a.pcounts[2 * p];
        cr += a.pcounts[2 * p + 1];
    }
    if (2 * tp + tr > a.cap_out) set_status(a.status, BAB_ERR_SHAPE);  // rows beyond cap_out are dropped
    a.d_counts[0] = (int)(2 * tp);
    a.d_counts[1] = (int)tr;
    a.d_counts[2] = (int)(2 * tp + tr);
}

__global__ void k_branch_write(BranchArgs a)
{
    const int n = live_count(a.n, a.d_n);
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (row >= n) return;
    const int dst = a.dest[row];
    if (dst < 0) return;
    const int d = a.d;
    const int pb = row_problem(a.batch, row);
    const int dp = a.batch.H ? a.k * problem_H(a.batch, pb, 0) : d;  // coordinates the problem uses
    const float *lo = a.lo + (size_t)row * d, *hi = a.hi + (size_t)row * d;
    const uint64_t id = a.id[row];
    if (!(dst & kPickFlag)) {
        const size_t o = (size_t)a.poff[2 * pb + 1] + dst;
        if (o >= (size_t)a.cap_out) return;
        if (a.out_prob && lane == 0) a.out_prob[o] = pb;
        if (a.out_split_dim && lane == 0) a.out_split_dim[o] = a.split_dim ? a.split_dim[row] : -1;
        for (int j = lane; j < d; j += 32) {
            a.out_lo[o * d + j] = lo[j];
            a.out_hi[o * d + j] = hi[j];
        }
        if (a.out_row_u)
            for (int j = lane; j < d; j += 32) a.out_row_u[o * d + j] = a.row_u[(size_t)row * d + j];
        if (lane == 0) {
            a.out_id[o] = id;
            a.out_lb[o] = a.lb[row];
            a.out_ub[o] = a.ub[row];
        }
        return;
    }
    // widest coordinate, lowest index on ties
    float wb = -1.f;
    int jb = 0x7FFFFFFF;
    const int given = a.split_dim ? a.split_dim[row] : -1;  // the sample-imbalance choice, when given
    for (int j = lane; j < dp && !(given >= 0 && given < dp); j += 32) {
        const float w = __fsub_rn(hi[j], lo[j]);
        if (w > wb) {
            wb = w;
            jb = j;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float w2 = __shfl_xor_sync(0xFFFFFFFFu, wb, o);
        const int j2 = __shfl_xor_sync(0xFFFFFFFFu, jb, o);
        if (w2 > wb || (w2 == wb && j2 < jb)) {
            wb = w2;
            jb = j2;
        }
    }
    if (given >= 0 && given < dp) jb = given;
    if (jb >= dp) jb = 0;  // a problem without coordinates (H_p = 0) splits nothing meaningful
    const float mid = __fmul_rn(0.5f, __fadd_rn(lo[jb], hi[jb]));
    const size_t o0 = (size_t)a.poff[2 * pb] + 2 * (size_t)(dst & ~kPickFlag);
    if (o0 + 1 >= (size_t)a.cap_out) return;
    if (a.out_prob && lane == 0) a.out_prob[o0] = a.out_prob[o0 + 1] = pb;
    if (a.out_split_dim && lane == 0) a.out_split_dim[o0] = a.out_split_dim[o0 + 1] = -1;
    for (int j = lane; j < d; j += 32) {
        const float l = lo[j], h = hi[j];
        a.out_lo[o0 * d + j] = l;
        a.out_hi[o0 * d + j] = (j == jb) ? mid : h;
        a.out_lo[(o0 + 1) * d + j] = (j == jb) ? mid : l;
        a.out_hi[(o0 + 1) * d + j] = h;
    }
    if (a.out_row_u)
        for (int j = lane; j < d; j += 32) {
            const float v = a.row_u[(size_t)row * d + j];
            a.out_row_u[o0 * d + j] = v;
            a.out_row_u[(o0 + 1) * d + j] = v;
        }
    if (lane == 0) {
        a.out_id[o0] = child_id(id, 0);
        a.out_id[o0 + 1] = child_id(id, 1);
        a.out_lb[o0] = a.out_lb[o0 + 1] = a.lb[row];
        a.out_ub[o0] = a.out_ub[o0 + 1] = a.ub[row];
    }
}

// The splitting heuristic of Section 3.1, one warp per box: the top_k samples of smallest (cost, m) (selected
// in increasing order, each the smallest key above the previous), their coordinates re-drawn from the counter
// sampler, per dimension the counts below / above the midpoint and the score (hi - lo) |n_lo - n_up|; the
// largest score (lowest j on ties), or the widest dimension when no dimension is imbalanced.
__global__ void __launch_bounds__(256) k_split_dims(int d, const float *lo, const float *hi, const uint64_t *id,
                                                    int n, const int *d_n, uint64_t seed, const float *costs, int M,
                                                    int top_k, int *split_dim)
{
    __shared__ int tops[8][64];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int box = blockIdx.x * 8 + wib;
    if (box >= live_count(n, d_n)) return;
    const float *c = costs + (size_t)box * M;
    unsigned long long prev = 0;
    for (int q = 0; q < top_k; ++q) {
        unsigned long long best = ~0ull;
        for (int m = lane; m < M; m += 32) {
            const unsigned long long key = ((unsigned long long)float_order(c[m]) << 32) | (unsigned)m;
            if ((q == 0 || key > prev) && key < best) best = key;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xFFFFFFFFu, best, o);
            best = other < best ? other : best;
        }
        prev = best;
        if (lane == 0) tops[wib][q] = (int)(best & 0xFFFFFFFFu);
    }
    __syncwarp();
    const uint64_t hb = box_hash(seed, id[box]);
    const float *bl = lo + (size_t)box * d, *bh = hi + (size_t)box * d;
    float sb = 0.f;
    int jb = 0x7FFFFFFF;
    for (int j = lane; j < d; j += 32) {
        const float mid = __fmul_rn(0.5f, __fadd_rn(bl[j], bh[j]));
        int nlo = 0, nup = 0;
        for (int q = 0; q < top_k; ++q) {
            const float u = draw_sample(hb, (uint32_t)tops[wib][q], (uint32_t)j, bl[j], bh[j]);
            nlo += u <= mid;
            nup += u >= mid;
        }
        const float sc = __fmul_rn(__fsub_rn(bh[j], bl[j]), (float)abs(nlo - nup));
        if (sc > sb) {
            sb = sc;
            jb = j;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xFFFFFFFFu, sb, o);
        const int j2 = __shfl_xor_sync(0xFFFFFFFFu, jb, o);
        if (s2 > sb || (s2 == sb && j2 < jb)) {
            sb = s2;
            jb = j2;
        }
    }
    if (!(sb > 0.f)) {
        // no imbalance: the widest dimension, lowest index on ties
        float wb = -1.f;
        jb = 0x7FFFFFFF;
        for (int j = lane; j < d; j += 32) {
            const float w = __fsub_rn(bh[j], bl[j]);
            if (w > wb) {
                wb = w;
                jb = j;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float w2 = __shfl_xor_sync(0xFFFFFFFFu, wb, o);
            const int j2 = __shfl_xor_sync(0xFFFFFFFFu, jb, o);
            if (w2 > wb || (w2 == wb && j2 < jb)) {
                wb = w2;
                jb = j2;
            }
        }
    }
    if (lane == 0) split_dim[box] = jb;
}

cudaError_t launch_split_dims(int d, const float *lo, const float *hi, const uint64_t *id, int n, const int *d_n,
                              uint64_t seed, const float *costs, int M, int top_k, int *split_dim, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    if (top_k < 1 || top_k > 64 || top_k > M) return cudaErrorInvalidValue;
    k_split_dims<<<(n + 7) / 8, 256, 0, st>>>(d, lo, hi, id, n, d_n, seed, costs, M, top_k, split_dim);
    return cudaGetLastError();
}

cudaError_t launch_prune_branch(const BranchArgs &a, cudaStream_t st)
{
    const int P = a.batch.P > 1 ? a.batch.P : 1;
    k_branch_plan<<<P, kPlanThreads, 0, st>>>(a);
    if (P > 1) k_branch_offsets<<<1, 32, 0, st>>>(a);
    if (a.n > 0) k_branch_write<<<(a.n + 7) / 8, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace bab
