// ibp_tc.cuh -- the TF32 interval image's layout and the launch of the tensor-core interval kernel with 3-term TF32
// split products (the BF16 image and its launch are described with NetDesc and in kernels.cuh).
//
// TF32 interval image: per layer l, per 128-row block mb of its outputs and 32-wide block ka of its inputs, one
// 64 KB stage of four 16 KB K-major 128-byte-swizzled A operands (W hi, W lo, |W| hi, |W| lo as TF32 halves, rows
// past d_l and inputs past d_{l-1} zero), stages in (l, mb, ka) order, the layers back to back.
#pragma once

#include "bab_internal.cuh"
#include "kernels.cuh"

namespace bab {

// 32-input blocks of a layer with K inputs (K rounded up to the TF32 k-step of 8)
__host__ __device__ constexpr int ibp_tf_ka(int K) { return (pad8(K) + 31) / 32; }

// k_ibp_tc with W c and |W| r as 3-term TF32 split products: a.ibp_img is the TF32 interval image
cudaError_t launch_ibp_tc_tf32(const BoundArgs &a, int num_sms, cudaStream_t st);

}  // namespace bab
