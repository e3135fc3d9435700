// Helpers of the MAP iteration shared by the single-request driver (map.cu)
// and the batched engine (engine.cu): QGGMRF potential and derivatives
// (eq. 15-17), clique weights, scalar slots and deterministic FP64 block sums.
#pragma once

#include "device_common.cuh"

namespace mbir {

constexpr int kRedThreads = 256;

struct PriorParams {
    float p, q, T, sigma0;
    float inv_s2;        // 1 / sigma_noise^2
    float kappa0_base;   // 2 / (p T^(2-p)) : kappa(0) * sigma^2
};

// scalar slots (doubles)
enum {
    S_GG = 0, S_GGP, S_GDP, S_GGPREV, S_BETA, S_GD, S_QQ, S_CURV, S_ALPHA, S_EE, S_PRIOR, S_BAD,
    S_COUNT = 16
};

__device__ __forceinline__ double block_sum(double v, double* sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
    return r;   // valid in thread 0
}

// QGGMRF potential (eq. 15) and its derivatives, in FP32 through log2/exp2.
// rho'(d) = sign(d) |d|^(p-1) / s^p * u/(1+u) * (1 + (q-p)/(p(1+u))),
// u = |d/(T s)|^(q-p); kappa = rho'(d)/d (limit 2/(p s^2 T^(2-p)) at d = 0).
__device__ __forceinline__ void qggmrf(const PriorParams& pr, float d, float s, float* drho, float* kappa,
                                       float* rho)
{
    float ad = fabsf(d);
    float ls = log2f(s);
    float r = ad / (pr.T * s);
    if (!(r > 1e-12f)) {
        if (drho) *drho = 0.0f;
        if (kappa) *kappa = pr.kappa0_base / (s * s);
        if (rho) *rho = 0.0f;
        return;
    }
    float la = log2f(ad);
    float u = exp2f((pr.q - pr.p) * log2f(r));
    float f = u / (1.0f + u);
    float corr = 1.0f + (pr.q - pr.p) / (pr.p * (1.0f + u));
    float base = exp2f((pr.p - 2.0f) * la - pr.p * ls);   // |d|^(p-2) / s^p
    float kap = base * f * corr;
    if (kappa) *kappa = kap;
    if (drho) *drho = kap * d;
    if (rho) *rho = base * ad * ad * f / pr.p;
}

static __constant__ int c_nb_dr[8] = {-1, -1, -1, 0, 0, 1, 1, 1};
static __constant__ int c_nb_dc[8] = {-1, 0, 1, -1, 1, -1, 0, 1};

__device__ __forceinline__ float nb_weight(int dr, int dc)
{
    const float be = 1.0f / (4.0f + 4.0f / 1.41421356237309515f);
    return (dr == 0 || dc == 0) ? be : be * 0.70710678118654752f;
}

}  // namespace mbir
