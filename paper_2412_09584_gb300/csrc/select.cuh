// select.cuh -- exact k-th smallest composite key (order(value), id) over a
// filtered set of rows, by 8-bit radix selection in one CTA (12 passes at
// most: 4 bytes of the order-preserving value key, then 8 bytes of the id).
// Used by the pick-out of bab_prune_branch and the top-k re-score of BF16
// rollouts.
#pragma once

#include "bab_internal.cuh"

namespace bab {

struct Thresh {
    uint32_t key;
    uint64_t id;
    bool none;  // nothing selected
};

__device__ __forceinline__ bool le_thresh(uint32_t key, uint64_t id, const Thresh &T)
{
    return !T.none && (key < T.key || (key == T.key && id <= T.id));
}

__device__ __forceinline__ uint32_t row_key(const float *v, int i) { return float_order(v[i]); }

// 96-bit composite digit `pass` (0 = most significant byte of the key).
__device__ __forceinline__ uint32_t digit_of(uint32_t key, uint64_t id, int pass)
{
    return pass < 4 ? (key >> (24 - 8 * pass)) & 0xFFu : (uint32_t)(id >> (56 - 8 * (pass - 4))) & 0xFFu;
}

__device__ __forceinline__ bool prefix_match(uint32_t key, uint64_t id, uint32_t pk, uint64_t pid, int pass)
{
    if (pass == 0) return true;
    if (pass <= 4) {
        const int sh = 32 - 8 * pass;
        return sh == 0 ? key == pk : (key >> sh) == (pk >> sh);
    }
    if (key != pk) return false;
    const int sh = 64 - 8 * (pass - 4);
    return (id >> sh) == (pid >> sh);
}

// The kth smallest (1-based) composite key among the rows accepted by `filt`.
template <typename Filt>
__device__ Thresh radix_select(int n, const float *val, const uint64_t *ids, Filt filt, int kth, unsigned *hist,
                               uint32_t *sh_pk, uint64_t *sh_pid, int *sh_rem, int *sh_done)
{
    Thresh T;
    T.none = kth <= 0;
    if (T.none) return T;
    if (threadIdx.x == 0) {
        *sh_pk = 0;
        *sh_pid = 0;
        *sh_rem = kth;
        *sh_done = 0;
    }
    __syncthreads();
    for (int pass = 0; pass < 12; ++pass) {
        for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        const uint32_t pk = *sh_pk;
        const uint64_t pid = *sh_pid;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            if (!filt(i)) continue;
            const uint32_t key = row_key(val, i);
            const uint64_t id = ids[i];
            if (prefix_match(key, id, pk, pid, pass)) atomicAdd(&hist[digit_of(key, id, pass)], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int rem = *sh_rem;
            unsigned cum = 0;
            int D = 255;
            for (int b = 0; b < 256; ++b) {
                if (cum + hist[b] >= (unsigned)rem) {
                    D = b;
                    break;
                }
                cum += hist[b];
            }
            rem -= (int)cum;
            if (pass < 4) {
                *sh_pk = pk | ((uint32_t)D << (24 - 8 * pass));
            } else {
                *sh_pid = pid | ((uint64_t)D << (56 - 8 * (pass - 4)));
            }
            *sh_rem = rem;
            // key resolved and every row with that key is needed: take all ties
            if (pass == 3 && hist[D] == (unsigned)rem) {
                *sh_pid = ~0ull;
                *sh_done = 1;
            }
        }
        __syncthreads();
        if (*sh_done) break;
    }
    T.key = *sh_pk;
    T.id = *sh_pid;
    __syncthreads();
    return T;
}

}  // namespace bab
