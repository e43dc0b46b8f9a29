// cost.cuh -- the state cost of the planning objective, c(x_t) for t = 1..H
// (Section 3, Eq. trajop), plus rho ||u_t||^2 handled by the callers:
//
//   kind 0  ||x_t - g||^2 (the default);
//   kind 1  the pushing-with-obstacles cost (Appendix D.4, Eq. pushing_cost):
//           w_t ||x_t - g|| + lambda sum_o [ReLU(s_o - ||p_t - p_o||)
//           + sum_i ReLU(s_o - ||x_t^(i) - p_o||)], the state holding s / 2
//           planar keypoints x_t^(i) = (x_{t,2i}, x_{t,2i+1}), the action the
//           planar pusher motion (k = 2), p_t = p_0 + u_0 + ... + u_{t-1}.
//
// Device pieces: the FP32 value in the order the search ranks by, the FP64
// value (incumbent), the interval minimum rounded down (interval bound), and
// the linear lower bound of an obstacle penalty on a box (CROWN).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace bab {

constexpr int kMaxObstacles = 8;

struct CostDesc {
    int kind;       // 0: squared distance; 1: pushing with obstacles
    int n_obs;
    float lam;
    float ox[kMaxObstacles], oy[kMaxObstacles], os[kMaxObstacles];
    float p0x, p0y;
    const float *w;  // device [H]: w[t - 1] = w_t
};

// FP32 state cost of kind 1 at step t: w_t sqrt(sum_i (x_i - g_i)^2) (squares by fused multiply-adds), then per
// obstacle in order lambda ReLU(s_o - d) for the pusher and each keypoint in order, d = sqrt(dx dx + dy dy) (dy dy
// rounded first), each added by a fused multiply-add.
__device__ __forceinline__ float obstacle_cost_f32(const CostDesc &c, int t, int s, const float *x, const float *goal,
                                                   float px, float py)
{
    float ss = 0.f;
    for (int i = 0; i < s; ++i) {
        const float e = __fsub_rn(x[i], goal[i]);
        ss = fmaf(e, e, ss);
    }
    float v = __fmul_rn(c.w[t - 1], __fsqrt_rn(ss));
    for (int o = 0; o < c.n_obs; ++o)
        for (int q = -1; 2 * q + 1 < s; ++q) {
            const float dx = __fsub_rn(q < 0 ? px : x[2 * q], c.ox[o]);
            const float dy = __fsub_rn(q < 0 ? py : x[2 * q + 1], c.oy[o]);
            const float r = __fsub_rn(c.os[o], __fsqrt_rn(fmaf(dx, dx, __fmul_rn(dy, dy))));
            v = fmaf(c.lam, r > 0.f ? r : 0.f, v);
        }
    return v;
}

// FP64 state cost of kind 1 at step t
__device__ __forceinline__ double obstacle_cost_f64(const CostDesc &c, int t, int s, const double *x,
                                                    const float *goal, double px, double py)
{
    double ss = 0.0;
    for (int i = 0; i < s; ++i) {
        const double e = x[i] - (double)goal[i];
        ss += e * e;
    }
    double v = (double)c.w[t - 1] * sqrt(ss);
    for (int o = 0; o < c.n_obs; ++o)
        for (int q = -1; 2 * q + 1 < s; ++q) {
            const double dx = (q < 0 ? px : x[2 * q]) - (double)c.ox[o];
            const double dy = (q < 0 ? py : x[2 * q + 1]) - (double)c.oy[o];
            const double r = (double)c.os[o] - sqrt(dx * dx + dy * dy);
            v += (double)c.lam * (r > 0.0 ? r : 0.0);
        }
    return v;
}

// lambda ReLU(size - (largest distance from (cx, cy) to the box)), rounded down: the minimum of a penalty term
__device__ __forceinline__ float penalty_min_rd(const CostDesc &c, int o, float l0, float u0, float l1, float u1)
{
    // the largest offsets along each axis, rounded up: max(u - c, c - l)
    const float a = fmaxf(__fsub_ru(u0, c.ox[o]), __fsub_ru(c.ox[o], l0));
    const float b = fmaxf(__fsub_ru(u1, c.oy[o]), __fsub_ru(c.oy[o], l1));
    const float md = __fsqrt_ru(__fmaf_ru(a, a, __fmul_ru(b, b)));
    const float r = __fsub_rd(c.os[o], md);
    return r > 0.f ? __fmul_rd(c.lam, r) : 0.f;
}

// A linear lower bound a . q + b of ReLU(size - ||q - c_o||) over the box [l0, u0] x [l1, u1]: a is the gradient of
// the concave size - ||q - c_o|| at the box centre (0 at c_o), b the smallest vertex offset h(v) - a . v (h rounded
// down, a . v rounded up, so b is rounded down); used only where it is positive at the box centre (returns true),
// otherwise the bound is 0.  Valid for any a: h is concave, so a function below it at the vertices stays below it.
__device__ __forceinline__ bool penalty_lower(const CostDesc &c, int o, float l0, float u0, float l1, float u1,
                                              float &a0, float &a1, float &b)
{
    const float mx = 0.5f * (l0 + u0), my = 0.5f * (l1 + u1);
    const float dx = mx - c.ox[o], dy = my - c.oy[o];
    const float nd = sqrtf(dx * dx + dy * dy);
    const float g0 = nd > 0.f ? -dx / nd : 0.f, g1 = nd > 0.f ? -dy / nd : 0.f;
    float bb = INFINITY;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const float vx = (v & 1) ? u0 : l0, vy = (v & 2) ? u1 : l1;
        const float ex = fmaxf(__fsub_ru(vx, c.ox[o]), __fsub_ru(c.ox[o], vx));  // |vx - cx| rounded up
        const float ey = fmaxf(__fsub_ru(vy, c.oy[o]), __fsub_ru(c.oy[o], vy));
        const float dist = __fsqrt_ru(__fmaf_ru(ex, ex, __fmul_ru(ey, ey)));
        const float h = __fsub_rd(c.os[o], dist);
        const float av = __fmaf_ru(g0, vx, __fmul_ru(g1, vy));
        bb = fminf(bb, __fsub_rd(h, av));
    }
    if (g0 * mx + g1 * my + bb > 0.f) {
        a0 = g0;
        a1 = g1;
        b = bb;
        return true;
    }
    a0 = a1 = b = 0.f;
    return false;
}

}  // namespace bab
