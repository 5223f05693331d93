// nr_hmc.cu -- on-device Hamiltonian Monte Carlo over many chains of a
// co-fitted slab model (arXiv 2509.06924, Sec. 2.3: leapfrog integration,
// Eq. 7, then the Metropolis-Hastings acceptance of Eq. 8).
//
// A chain's free parameters theta_k carry uniform box priors [lo_k, hi_k]
// (as in Tables 1-4) and are sampled in unconstrained coordinates u
// (Sec. 2.3.1 advises such a change of variables for bounded parameters):
//   theta_k = lo_k + (hi_k - lo_k) s_k,  s_k = 1 / (1 + e^-u_k),
//   log pi(u) = sum_c loglik_c(theta) + sum_k [log s_k + log(1 - s_k)]
// (prior density times Jacobian).  Every contrast c of a chain is one stack
// of the likelihood batch; its packed slots either copy a free parameter
// (tied across contrasts) or hold a fixed value.
//
// The likelihood and its gradient come from the mixed gradient kernel.  The
// kernels here are the glue of a step, all chain-parallel and FP64 (the
// arrays are tiny next to the likelihood):
//   cofit_gather: u -> packed parameters of every stack (and the chain's
//                 resolution scale f for its stacks, when one is sampled);
//   cofit_stage:  one warp per chain pulls the packed gradient back to u
//                 (tied slots summed, chain rule through the sigmoid, prior
//                 term), reduces log pi, and applies the leapfrog stage:
//                 momentum draw and H0 at the start, kicks and drifts, and
//                 H1 with the accept/reject at the end.
// No kernel waits on another CTA and there is no device-side random number
// generation: the standard-normal and uniform draws are inputs.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "nr_internal.h"

namespace nrimpl {
namespace {

constexpr unsigned kFullMask = 0xffffffffu;

__global__ void cofit_gather_kernel(const double *u, int C, int P, int NS, const int32_t *src, const double *val,
                                    const double *lo, const double *hi, double *params, int res_param, int NC,
                                    double *dq_scale)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)C * NS) return;
    const int c = (int)(i / NS), slot = (int)(i - (int64_t)c * NS);
    if (res_param >= 0 && slot < NC) {
        // the chain's resolution scale, for each of its NC stacks
        const double s = 1.0 / (1.0 + exp(-u[(int64_t)c * P + res_param]));
        dq_scale[(int64_t)c * NC + slot] = lo[res_param] + (hi[res_param] - lo[res_param]) * s;
    }
    const int k = src[slot];
    double v = val[slot];
    if (k >= 0) {
        const double s = 1.0 / (1.0 + exp(-u[(int64_t)c * P + k]));
        v = lo[k] + (hi[k] - lo[k]) * s;
    }
    params[i] = v;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
    return v;
}

// One warp per chain.  stage: kStageLogp (log pi and gradient only),
// kStageFirst (momentum draw, H0, half kick, drift), kStageMid (kick, drift),
// kStageLast (half kick, H1, accept / reject).
__global__ void cofit_stage_kernel(CofitStageArgs a)
{
    const int warps = blockDim.x >> 5;
    const int c = blockIdx.x * warps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= a.C) return;
    const int P = a.P;
    double *u = a.u + (int64_t)c * P;
    const double *gpk = a.gpk + (int64_t)c * a.NS;
    // log pi: the contrasts' log-likelihoods plus the prior/Jacobian terms
    double lp = 0.0, kin0 = 0.0, kin1 = 0.0;
    for (int i = lane; i < a.n_contrast; i += 32) lp += a.ll[(int64_t)c * a.n_contrast + i];
    for (int k = lane; k < P; k += 32) {
        const double uk = u[k];
        const double s = 1.0 / (1.0 + exp(-uk));
        const double au = fabs(uk);
        lp += -au - 2.0 * log1p(exp(-au));
        double gt = 0.0;
        for (int t = a.tie_ptr[k]; t < a.tie_ptr[k + 1]; ++t) gt += gpk[a.tie_slot[t]];
        if (k == a.res_param) {
            // d loglik / d f = (d loglik / d ln f) / f, summed over the contrasts
            const double f = a.lo[k] + (a.hi[k] - a.lo[k]) * s;
            double gr = 0.0;
            for (int i = 0; i < a.n_contrast; ++i) gr += a.gres[(int64_t)c * a.n_contrast + i];
            gt += gr / f;
        }
        const double g = gt * (a.hi[k] - a.lo[k]) * s * (1.0 - s) + (1.0 - 2.0 * s);
        if (a.stage == kStageLogp) {
            if (a.grad_out) a.grad_out[(int64_t)c * P + k] = g;
            continue;
        }
        double *pm = a.mom + (int64_t)c * P;
        const double im = a.inv_mass[k];
        double pk;
        if (a.stage == kStageFirst) {
            pk = a.z[(int64_t)c * P + k] / sqrt(im);
            kin0 += 0.5 * pk * pk * im;
            a.u0[(int64_t)c * P + k] = uk;
        } else {
            pk = pm[k];
        }
        const double kick = (a.stage == kStageMid) ? a.eps : 0.5 * a.eps;
        pk += kick * g;
        if (a.stage == kStageLast) {
            kin1 += 0.5 * pk * pk * im;
        } else {
            u[k] = uk + a.eps * im * pk;
        }
        pm[k] = pk;
    }
    lp = warp_sum(lp);
    if (a.stage == kStageLogp) {
        if (lane == 0 && a.logp_out) a.logp_out[c] = lp;
        return;
    }
    if (a.stage == kStageFirst) {
        kin0 = warp_sum(kin0);
        if (lane == 0) {
            a.H0[c] = -lp + kin0;
            a.logp0[c] = lp;
        }
        return;
    }
    if (a.stage == kStageLast) {
        kin1 = warp_sum(kin1);
        const double H1 = -lp + kin1;
        // accept iff log U < H0 - H1; a NaN on either side rejects
        const bool acc = a.log_unif[c] < a.H0[c] - H1;
        if (!acc)
            for (int k = lane; k < P; k += 32) u[k] = a.u0[(int64_t)c * P + k];
        if (lane == 0) {
            if (a.accepted) a.accepted[c] = acc ? 1 : 0;
            if (a.logp_out) a.logp_out[c] = acc ? lp : a.logp0[c];
        }
    }
}

} // namespace

cudaError_t launch_cofit_gather(const double *u, int C, int P, int NS, const int32_t *src, const double *val,
                                const double *lo, const double *hi, double *params, int res_param, int NC,
                                double *dq_scale, cudaStream_t st)
{
    const int64_t n = (int64_t)C * NS;
    if (n == 0) return cudaSuccess;
    cofit_gather_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(u, C, P, NS, src, val, lo, hi, params,
                                                                     res_param, NC, dq_scale);
    return cudaGetLastError();
}

cudaError_t launch_cofit_stage(const CofitStageArgs &a, cudaStream_t st)
{
    if (a.C == 0) return cudaSuccess;
    const int warps = 4;
    cofit_stage_kernel<<<(a.C + warps - 1) / warps, 32 * warps, 0, st>>>(a);
    return cudaGetLastError();
}

} // namespace nrimpl
