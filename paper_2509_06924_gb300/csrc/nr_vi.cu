// nr_vi.cu -- variational inference for a co-fitted slab model on the GPU,
// many independent restarts at once (arXiv 2509.06924, Sec. 2.4; the LED
// co-fit of Sec. 4.2 runs 100 restarts of a multivariate normal q in an
// unconstrained space, optimised by Adam).
//
// phi of one restart: mu [P] and the lower triangle of the Cholesky factor L,
// packed row by row ((i, j <= i) at i (i + 1) / 2 + j) with log L_ii on the
// diagonal.  One iteration with a standard-normal draw e (an input):
//   vi_sample: u = mu + L e, and the part of the ELBO estimate that does not
//              involve the likelihood, e^T e / 2 + sum_i log L_ii + P/2 log 2 pi
//              (one warp per restart);
//   the co-fit sampler's log pi(u) and gradient g (gather, mixed gradient
//   kernel, pull-back);
//   vi_adam:   the gradient of the single-sample negative ELBO (Eqs. 22-24,
//              e held fixed: d/d mu = -g, d/d L_ij = -g_i e_j,
//              d/d log L_ii = -g_i e_i L_ii - 1) and one Adam step of every
//              entry of phi (one block per restart, the moments and the step
//              in FP32 arithmetic on FP64 storage); the ELBO estimate
//              log pi(u) + (the part above) is written per restart.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "nr_internal.h"

namespace nrimpl {
namespace {

constexpr unsigned kMask = 0xffffffffu;
constexpr double kHalfLog2Pi = 0.91893853320467274178032973640562; // ln(2 pi) / 2

__global__ void vi_sample_kernel(const double *phi, const double *eps, int R, int P, int64_t nphi, double *u,
                                 double *part, int32_t *t_dev, double beta1, double beta2, double *bias)
{
    const int warps = blockDim.x >> 5;
    const int r = blockIdx.x * warps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    // the iteration counter lives on the device, so a captured iteration
    // advances it on every replay; vi_adam (later in the stream) reads the
    // Adam bias corrections 1 / (1 - beta^t) formed here once per iteration
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int t = *t_dev + 1;
        *t_dev = t;
        bias[0] = 1.0 / (1.0 - pow(beta1, (double)t));
        bias[1] = 1.0 / (1.0 - pow(beta2, (double)t));
    }
    if (r >= R) return;
    const double *mu = phi + (int64_t)r * nphi;
    const double *tri = mu + P;
    const double *e = eps + (int64_t)r * P;
    double acc = 0.0;
    for (int i = lane; i < P; i += 32) {
        const double *row = tri + (int64_t)i * (i + 1) / 2;
        double ui = mu[i] + exp(row[i]) * e[i];
        for (int j = 0; j < i; ++j) ui += row[j] * e[j];
        u[(int64_t)r * P + i] = ui;
        acc += 0.5 * e[i] * e[i] + row[i] + kHalfLog2Pi;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kMask, acc, o);
    if (lane == 0) part[r] = acc;
}

// One block per restart.  The restart's gradient and draw are staged as
// floats in shared memory (when P <= kAdamStageP), and the moments and the
// step are formed in FP32 arithmetic: phi, m and v keep their FP64 storage,
// so phi accumulates its updates at full precision, while the update itself
// (a heuristic scaling of the gradient, whose own error is ~1e-5) needs no
// more than FP32.  In FP64 the square root and division alone bound this
// kernel on GB300's FP64 rate.
constexpr int kAdamStageP = 4096;

__global__ void vi_adam_kernel(double *phi, double *m, double *v, const double *eps, const double *g,
                               const double *logp, const double *part, int P, int64_t nphi, const double *bias,
                               float lr, float beta1, float beta2, float eps_adam, bool stage, double *elbo)
{
    extern __shared__ float sh_ge[]; // g_r [P], eps_r [P]
    const int r = blockIdx.x;
    const double *gr = g + (int64_t)r * P, *er = eps + (int64_t)r * P;
    if (stage) {
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            sh_ge[i] = (float)gr[i];
            sh_ge[P + i] = (float)er[i];
        }
        __syncthreads();
    }
    auto gi = [&](int i) { return stage ? sh_ge[i] : (float)gr[i]; };
    auto ej = [&](int j) { return stage ? sh_ge[P + j] : (float)er[j]; };
    const float c0 = (float)bias[0], c1 = (float)bias[1];
    double *phr = phi + (int64_t)r * nphi, *mr = m + (int64_t)r * nphi, *vr = v + (int64_t)r * nphi;
    for (int64_t p = threadIdx.x; p < nphi; p += blockDim.x) {
        float grad;
        if (p < P) {
            grad = -gi((int)p);
        } else {
            // packed triangle index -> (i, j): i (i + 1) / 2 <= q < (i + 1) (i + 2) / 2
            const int64_t q = p - P;
            int i = (int)((sqrtf(8.f * (float)q + 1.f) - 1.f) * 0.5f); // corrected below
            while ((int64_t)(i + 1) * (i + 2) / 2 <= q) ++i;
            while ((int64_t)i * (i + 1) / 2 > q) --i;
            const int j = (int)(q - (int64_t)i * (i + 1) / 2);
            grad = (i == j) ? -gi(i) * ej(i) * expf((float)phr[p]) - 1.f : -gi(i) * ej(j);
        }
        const float mm = fmaf(beta1, (float)mr[p], (1.f - beta1) * grad);
        const float vv = fmaf(beta2, (float)vr[p], (1.f - beta2) * grad * grad);
        mr[p] = mm;
        vr[p] = vv;
        phr[p] -= (double)(lr * (mm * c0) / (sqrtf(vv * c1) + eps_adam));
    }
    if (threadIdx.x == 0 && elbo) elbo[r] = logp[r] + part[r];
}

} // namespace

cudaError_t launch_vi_sample(const double *phi, const double *eps, int R, int P, double *u, double *part,
                             int32_t *t_dev, double beta1, double beta2, double *bias, cudaStream_t st)
{
    if (R == 0) return cudaSuccess;
    const int64_t nphi = (int64_t)P + (int64_t)P * (P + 1) / 2;
    vi_sample_kernel<<<(R + 3) / 4, 128, 0, st>>>(phi, eps, R, P, nphi, u, part, t_dev, beta1, beta2, bias);
    return cudaGetLastError();
}

cudaError_t launch_vi_adam(double *phi, double *m, double *v, const double *eps, const double *g,
                           const double *logp, const double *part, int R, int P, const double *bias, double lr,
                           double beta1, double beta2, double eps_adam, double *elbo, cudaStream_t st)
{
    const int64_t nphi = (int64_t)P + (int64_t)P * (P + 1) / 2;
    if (R == 0 || nphi == 0) return cudaSuccess;
    const bool stage = P <= kAdamStageP;
    const size_t smem = stage ? sizeof(float) * 2 * (size_t)P : 0;
    vi_adam_kernel<<<R, 256, smem, st>>>(phi, m, v, eps, g, logp, part, P, nphi, bias, (float)lr, (float)beta1,
                                         (float)beta2, (float)eps_adam, stage, elbo);
    return cudaGetLastError();
}

} // namespace nrimpl
