// nr_profile.cu -- SLD and absorption depth profiles of a batch of stacks.
//
// The paper's figures draw the scattering-length-density profile through
// the film with posterior bands (Sec. 4.1, quartz; Sec. 4.2, LED device):
// one profile per posterior sample, evaluated on a common depth grid.  With
// Gaussian interfacial roughness every interface is an error-function step,
//   rho(z) = rho_0 + sum_j (rho_{j+1} - rho_j) (1 + erf((z - z_j) / (sqrt(2) sigma_j))) / 2,
// z_j = d_1 + ... + d_j the depth of interface j (z_0 = 0), and the same for
// the absorption iota(z) (iota_0 = 0).  sigma_j = 0 is the sharp step, which
// takes the deeper medium's value at z = z_j.
//
// One CTA per stack (grid-stride over stacks): thread j stages interface j
// (depth as a float pair, steps, 1/(sqrt(2) sigma)) in shared memory, then
// the threads sweep the depth grid, two outputs per thread, with coalesced
// stores.  z - z_j is formed as (z - z_hi) - z_lo, exact near the interface
// (where the error function is steep) and FP32-accurate elsewhere.
#include <cuda_runtime.h>

#include <cstdint>

#include "nr_internal.h"

namespace nrimpl {
namespace {

constexpr int kProfileBlock = 256;

__global__ void __launch_bounds__(kProfileBlock)
nr_profile_kernel(const double *params, const int64_t *par_off, const int32_t *n_layers, int n_stacks,
                  const float *z, int nz, float *rho_out, float *iota_out, int32_t *status)
{
    // interface j: (depth hi, depth lo, 1/(sqrt(2) sigma) or 0, SLD step); absorption step
    __shared__ float4 s_if[NR_MAX_LAYERS + 1];
    __shared__ float s_di[NR_MAX_LAYERS + 1];
    __shared__ float s_r0;
    const int tid = threadIdx.x;
    for (int s = blockIdx.x; s < n_stacks; s += gridDim.x) {
        const int n = n_layers[s];
        const double *p = params + par_off[s];
        __syncthreads(); // the previous stack's entries are no longer read
        if (tid <= n) {
            const int j = tid;
            double depth = 0.0;
            for (int i = 0; i < j; ++i) depth += p[i];
            const double rj = p[n + j], rj1 = p[n + j + 1];
            const double ij = j >= 1 ? p[2 * n + 2 + j - 1] : 0.0, ij1 = p[2 * n + 2 + j];
            const double sg = p[3 * n + 3 + j];
            const float zh = (float)depth;
            // inverse width 0 marks a sharp step (sigma = 0)
            const float sgf = (float)sg;
            s_if[j] = make_float4(zh, (float)(depth - (double)zh), sgf > 0.f ? 1.f / (1.41421356237f * sgf) : 0.f,
                                  (float)(rj1 - rj));
            s_di[j] = (float)(ij1 - ij);
            bool bad = !isfinite(depth) || !isfinite(rj) || !isfinite(rj1) || !isfinite(ij) || !isfinite(ij1) ||
                       !isfinite(sg) || sg < 0.0;
            if (j == 0) s_r0 = (float)rj;
            if (bad) atomicOr(status, NR_FLAG_NONFINITE_PARAM);
        }
        __syncthreads();
        const float r0 = s_r0;
        float *ro = rho_out ? rho_out + (int64_t)s * nz : nullptr;
        float *io = iota_out ? iota_out + (int64_t)s * nz : nullptr;
        // two depths per thread share each interface entry and overlap their
        // error functions
        for (int i0 = tid; i0 < nz; i0 += 2 * kProfileBlock) {
            const int i1 = i0 + kProfileBlock;
            const bool two = i1 < nz;
            const float z0 = z[i0], z1 = two ? z[i1] : z0;
            float r_0 = r0, r_1 = r0, a_0 = 0.f, a_1 = 0.f;
            for (int j = 0; j <= n; ++j) {
                const float4 f = s_if[j];
                const float t0 = (z0 - f.x) - f.y, t1 = (z1 - f.x) - f.y;
                float st0, st1;
                if (f.z > 0.f) {
                    st0 = 0.5f * (1.f + erff(t0 * f.z));
                    st1 = 0.5f * (1.f + erff(t1 * f.z));
                } else {
                    st0 = t0 >= 0.f ? 1.f : 0.f;
                    st1 = t1 >= 0.f ? 1.f : 0.f;
                }
                r_0 = fmaf(f.w, st0, r_0);
                r_1 = fmaf(f.w, st1, r_1);
                if (io) {
                    const float di = s_di[j];
                    a_0 = fmaf(di, st0, a_0);
                    a_1 = fmaf(di, st1, a_1);
                }
            }
            if (ro) {
                ro[i0] = r_0;
                if (two) ro[i1] = r_1;
            }
            if (io) {
                io[i0] = a_0;
                if (two) io[i1] = a_1;
            }
        }
    }
}

} // namespace

cudaError_t launch_profile(const double *params, const int64_t *par_off, const int32_t *n_layers, int n_stacks,
                           const float *z, int nz, float *rho_out, float *iota_out, int32_t *status, int sms,
                           cudaStream_t st)
{
    if (n_stacks == 0 || nz == 0) return cudaSuccess;
    const int grid = n_stacks < 8 * sms ? n_stacks : 8 * sms;
    nr_profile_kernel<<<grid, kProfileBlock, 0, st>>>(params, par_off, n_layers, n_stacks, z, nz, rho_out,
                                                      iota_out, status);
    return cudaGetLastError();
}

} // namespace nrimpl
