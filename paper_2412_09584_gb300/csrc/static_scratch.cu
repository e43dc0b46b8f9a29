// static_scratch.cu -- bab_bound_crown_static: the CROWN lower bound of
// bab_bound_crown, for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need a bound:
// a plugin whose enqueue step runs inside a host framework that owns all
// device memory and forbids allocation there, or a real-time planning loop
// that may not allocate (or synchronise the device, as cudaFree does) once
// it has started.  This entry point takes no context: the network comes in as
// a device pointer, and every byte of working memory (the padded weight
// images, the interval bounds and the rounding-error helpers) lives in one
// file-scope __device__ array of BAB_STATIC_SCRATCH_BYTES.  A GPU holds the
// array from the moment this file's module is loaded on it (the first call
// there) until the process exits.
//
// Host code cannot use the array's name as a device address, so the first
// call on each device (with that device current) asks the runtime for the
// array's device address once with cudaGetSymbolAddress and keeps it; the
// same call also loads the kernels the entry point launches.  With CUDA's
// lazy module loading both steps may allocate device memory, so a caller
// makes one warm-up call per device (n = 0 does nothing else) before the
// section that must not allocate, and before any stream capture.
// All calls share the array, so calls whose GPU work overlaps (for example
// on two streams) race.  Every word the kernels read is written earlier in
// the same call, so nothing needs clearing.
#include <cstring>
#include <mutex>

#include "bab_internal.cuh"
#include "kernels.cuh"

namespace {

__device__ __align__(256) unsigned char g_static_scratch[BAB_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

__global__ void k_pack_images(bab::NetDesc N, const float *__restrict__ params, float *__restrict__ fwd,
                              float *__restrict__ bwd);

// Device address of g_static_scratch on the current device, looked up once per device; the first lookup also
// loads the kernels this entry point launches.
int static_scratch_address(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return BAB_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return BAB_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        cudaFuncAttributes fa;
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_pack_images);
        if (e == cudaSuccess) e = bab::preload_ibp_crown();
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return BAB_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return BAB_OK;
}

// Layout of the padded forward / backward network images (as the context builds them).
bool make_net_desc(bab::NetDesc &N, int L, const int *dims, int s, int k)
{
    using namespace bab;
    std::memset(&N, 0, sizeof(N));
    if (L < 1 || L > kMaxLayers || s < 1 || k < 1 || dims[0] != s + k || dims[L] != s) return false;
    int maxw = 0, h = 0, raw = 0, img = 0;
    for (int l = 0; l <= L; ++l) {
        if (dims[l] < 1 || dims[l] > kMaxWidth) return false;
        N.dims[l] = dims[l];
        maxw = dims[l] > maxw ? dims[l] : maxw;
    }
    N.L = L;
    N.s = s;
    N.k = k;
    N.maxw_p = pad4(maxw);
    for (int l = 1; l <= L; ++l) {
        N.hoff[l] = h;
        if (l < L) h += dims[l];
        N.raw_w[l] = raw;
        raw += dims[l] * dims[l - 1];
        N.raw_b[l] = raw;
        raw += dims[l];
        N.fwd_w[l] = N.bwd_w[l] = img;
        img += pad4(dims[l - 1]) * pad4(dims[l]);
        N.fwd_b[l] = N.bwd_b[l] = img;
        img += pad4(dims[l]);
    }
    N.sumh = h;
    N.raw_floats = raw;
    N.img_floats = img;
    for (int l = 1; l <= L; ++l) N.gam[l] = gamma_fp32(pad4(dims[l]));
    return true;
}

// Fill both images from the packed parameters: every image word is written
// (zero padding included), one thread per word.
__global__ void k_pack_images(bab::NetDesc N, const float *__restrict__ params, float *__restrict__ fwd,
                              float *__restrict__ bwd)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N.img_floats; i += gridDim.x * blockDim.x) {
        int l = 1;
        while (l < N.L && i >= N.fwd_w[l + 1]) ++l;
        const int no = N.dims[l], ni = N.dims[l - 1], Kp = bab::pad4(ni), Np = bab::pad4(no);
        const float *W = params + N.raw_w[l], *b = params + N.raw_b[l];
        float vf = 0.f, vb = 0.f;
        if (i < N.fwd_b[l]) {
            const int local = i - N.fwd_w[l];
            const int p = local / Np, q = local % Np;  // forward image: [Kp][Np]
            if (p < ni && q < no) vf = W[(size_t)q * ni + p];
            const int qb = local / Kp, pb = local % Kp;  // backward image: [Np][Kp]
            if (qb < no && pb < ni) vb = W[(size_t)qb * ni + pb];
        } else {
            const int q = i - N.fwd_b[l];
            if (q < no) vf = vb = b[q];
        }
        fwd[i] = vf;
        bwd[i] = vb;
    }
}

}  // namespace

extern "C" int bab_bound_crown_static(int n_layers, const int *dims, const float *params, int state_dim,
                                      int action_dim, const float *x0, const float *goal, int horizon, float rho,
                                      const float *lo, const float *hi, int n, float *lb, float *margin,
                                      void *stream)
{
    using namespace bab;
    if (!dims || !params || !x0 || !goal) return BAB_ERR_INVALID_ARG;
    NetDesc N;
    if (!make_net_desc(N, n_layers, dims, state_dim, action_dim)) return BAB_ERR_SHAPE;
    if (horizon < 1 || horizon > (1 << 20) || n < 0) return BAB_ERR_SHAPE;
    if (!(rho >= 0.f) || rho != rho || rho > 3.0e38f) return BAB_ERR_INVALID_ARG;
    if (n > 0 && (!lo || !hi || !lb)) return BAB_ERR_INVALID_ARG;

    // working set, each piece 256-byte aligned: per box 4 (H (3 sumh + s) + 2 (H + 1) s) bytes (at most about
    // 2^20 * 2^12 * 4, so no product below can wrap), plus the two images and five alignment pads; the box count
    // is checked against the room left before any total is formed
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t img = up((size_t)N.img_floats * sizeof(float));
    const size_t per_box = 4 * ((size_t)horizon * (3 * (size_t)N.sumh + N.s) + 2 * ((size_t)horizon + 1) * N.s);
    const size_t cap = (size_t)BAB_STATIC_SCRATCH_BYTES;
    if (2 * img + 5 * 256 > cap || (size_t)n > (cap - 2 * img - 5 * 256) / per_box) return BAB_ERR_SHAPE;
    const size_t nh = (size_t)n * horizon * N.sumh, nx = (size_t)n * (horizon + 1) * N.s;

    // the address lookup (and, on a device's first call, the module loading) comes before the n = 0 return,
    // so that a call with n = 0 is the warm-up
    void *base = nullptr;
    int rc = static_scratch_address(&base);
    if (rc != BAB_OK) return rc;
    if (n == 0) return BAB_OK;
    char *p = static_cast<char *>(base);
    float *fwd = reinterpret_cast<float *>(p);
    p += img;
    float *bwd = reinterpret_cast<float *>(p);
    p += img;
    BoundArgs a{};
    a.pre_lo = reinterpret_cast<float *>(p);
    p += up(nh * 4);
    a.pre_hi = reinterpret_cast<float *>(p);
    p += up(nh * 4);
    a.x_lo = reinterpret_cast<float *>(p);
    p += up(nx * 4);
    a.x_hi = reinterpret_cast<float *>(p);
    p += up(nx * 4);
    a.S = reinterpret_cast<float *>(p);

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_pack_images<<<(N.img_floats + 255) / 256, 256, 0, st>>>(N, params, fwd, bwd);
    a.net = N;
    a.fwd = fwd;
    a.bwd = bwd;
    a.x0 = x0;
    a.goal = goal;
    a.lo = lo;
    a.hi = hi;
    a.n = n;
    a.d_n = nullptr;
    a.H = horizon;
    a.d = N.k * horizon;
    a.rho = rho;
    a.lb = lb;
    a.margin = margin;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_ibp(a, 0, st);
    if (e == cudaSuccess) e = launch_crown(a, 0, st);
    if (e != cudaSuccess) return BAB_ERR_CUDA;
    return BAB_OK;
}
