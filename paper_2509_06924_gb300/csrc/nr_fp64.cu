// nr_fp64.cu -- the plain FP64 path: the same forward model (Abeles /
// Parratt with Nevot-Croce roughness, Sec. 2.1; Gauss-Hermite smearing,
// Sec. 3; Gaussian likelihood, Sec. 2.1 / Eq. 25) written directly in
// complex double, one thread per (stack, Q point) looping over nodes and
// layers.  It is the baseline the mixed path is measured against, and its
// gradient is the central difference of the log-likelihood, each parameter
// stepped by h_p = eps^(1/3) max(|theta_p|, typ_p) (typ = 1 A, 1e-6 A^-2,
// 1e-8 A^-2, 1 A, 1, 1e-7 for d, rho, iota, sigma, scale, bkg; the
// pre-scaling advice of Sec. 2.3.1).  Perturbation p of a stack is launched
// as grid row p: row 0 is the unperturbed point, rows 2i+1 / 2i+2 step
// parameter i up / down (up / twice up for an absorption at its bound).
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

#include "nr_internal.h"

namespace nrimpl {
namespace {

constexpr double kPiD = 3.141592653589793238462643383279502884;

struct cd {
    double x, y;
};
__device__ __forceinline__ cd mk(double x, double y) { return cd{x, y}; }
__device__ __forceinline__ cd operator+(cd a, cd b) { return mk(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cd operator-(cd a, cd b) { return mk(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ cd operator*(cd a, cd b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ cd cdiv(cd a, cd b)
{
    const double d = b.x * b.x + b.y * b.y;
    return mk((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ cd cexp_d(cd a)
{
    double s, c;
    sincos(a.y, &s, &c);
    const double m = exp(a.x);
    return mk(m * c, m * s);
}
// principal square root, Im(z) >= 0 assumed
__device__ __forceinline__ cd csqrt_d(cd z)
{
    const double m = hypot(z.x, z.y);
    const double t = sqrt(0.5 * (fabs(z.x) + m));
    if (t == 0.0) return mk(0.0, 0.0);
    if (z.x >= 0.0) return mk(t, z.y / (2.0 * t));
    return mk(fabs(z.y) / (2.0 * t), copysign(t, z.y));
}

__device__ __forceinline__ double typ_of(int i, int n)
{
    if (i < n) return 1.0;
    if (i < 2 * n + 2) return 1e-6;
    if (i < 3 * n + 3) return 1e-8;
    if (i < 4 * n + 4) return 1.0;
    if (i == 4 * n + 4) return 1.0;
    return 1e-7;
}
__device__ __forceinline__ double step_of(double theta, int i, int n)
{
    return 6.0554544523933395e-06 /* cbrt(DBL_EPSILON) */ * fmax(fabs(theta), typ_of(i, n));
}
// Absorptions are bounded below by 0, and at iota = 0 below a critical edge
// the principal branch makes the derivative one-sided: there the difference
// is taken forward, f'(t) = (-3 f(t) + 4 f(t+h) - f(t+2h)) / (2h).
__device__ __forceinline__ bool one_sided(double theta, int i, int n)
{
    return i >= 2 * n + 2 && i < 3 * n + 3 && theta < step_of(theta, i, n);
}

// Reflectivity |r(q)|^2 of a stack by the Parratt recursion.
__device__ double reflect_fp64(const double *p, int n, int pi, double h, double q)
{
    auto par = [&](int i) { return i == pi ? p[i] + h : p[i]; };
    const double k0 = 0.5 * q;
    const double rho0 = par(n);
    auto kz = [&](int j) -> cd {
        if (j == 0) return mk(k0, 0.0);
        const double re = k0 * k0 - 4.0 * kPiD * (par(n + j) - rho0);
        const double im = 4.0 * kPiD * par(2 * n + 2 + j - 1);
        return csqrt_d(mk(re, im));
    };
    cd kb = kz(n + 1);
    cd X = mk(0.0, 0.0);
    for (int j = n; j >= 0; --j) {
        const cd ka = kz(j);
        const cd S = ka + kb;
        cd r = mk(0.0, 0.0);
        if (S.x != 0.0 || S.y != 0.0) {
            const double sg = par(3 * n + 3 + j);
            const cd w = ka * kb * mk(-2.0 * sg * sg, 0.0);
            r = cdiv(ka - kb, S) * cexp_d(w);
        }
        if (j == n) {
            X = r;
        } else {
            const double d = par(j);  // thickness of layer j+1
            const cd E = cexp_d(kb * mk(0.0, 2.0 * d));
            const cd Y = X * E;
            X = cdiv(r + Y, mk(1.0, 0.0) + r * Y);
        }
        kb = ka;
    }
    return X.x * X.x + X.y * X.y;
}

template <int MODE>
__global__ void __launch_bounds__(kFp64Block) nr_fp64_kernel(const KernelArgs ka, const QuadConst qc)
{
    __shared__ double sh[kFp64Block / 32];
    const WorkItem wi = ka.items[blockIdx.x];
    if constexpr (NR_DEBUG) {
        if (!item_in_bounds(ka, wi, 0)) { // uniform per block
            if (threadIdx.x == 0) atomicOr(ka.status, NR_FLAG_DEBUG_BOUNDS);
            return;
        }
    }
    const StackInfo si = ka.stacks[wi.stack];
    const int n = si.n;
    const int pert = blockIdx.y;
    const int npar = 4 * n + 6;
    if (pert >= (MODE == kGrad ? 2 * npar + 1 : 1)) return; // uniform per block
    const double *p = ka.params + si.par_off;
    int pi = -1;
    double h = 0.0;
    if (pert > 0) {
        pi = (pert - 1) >> 1;
        h = step_of(p[pi], pi, n);
        if (((pert - 1) & 1) != 0) h = one_sided(p[pi], pi, n) ? 2.0 * h : -h;
    }
    const int qi = wi.q_lo + threadIdx.x;
    double term = 0.0;
    if (qi < wi.q_hi) {  // a stack with an empty dataset still gets one (empty) item
        const double Q = (double)ka.q[si.q_begin + qi];
        const double dQ = (double)ka.dq[si.q_begin + qi];
        double S = 0.0;
        for (int k = 0; k < qc.K; ++k) {
            const double qk = Q + dQ * qc.gd[k];
            if (!(qk > 0.0)) {
                atomicOr(ka.status, NR_FLAG_BAD_Q);
                S = __longlong_as_double(0x7ff8000000000000ll);
                break;
            }
            S += qc.wd[k] * reflect_fp64(p, n, pi, h, qk);
        }
        const double scale = pi == 4 * n + 4 ? p[4 * n + 4] + h : p[4 * n + 4];
        const double bkg = pi == 4 * n + 5 ? p[4 * n + 5] + h : p[4 * n + 5];
        const double m = scale * S + bkg;
        if constexpr (MODE == kModel) {
            ka.r_out[si.out_off + qi] = (float)m;
        } else {
            const double Ro = (double)ka.r_obs[si.q_begin + qi];
            const double e = (double)ka.r_err[si.q_begin + qi];
            if (!(e > 0.0)) atomicOr(ka.status, NR_FLAG_BAD_ERR);
            const double res = (m - Ro) / e;
            term = res * res + log(2.0 * kPiD * e * e);
        }
    }
    if constexpr (MODE != kModel) {
        for (int o = 16; o > 0; o >>= 1) term += __shfl_xor_sync(0xffffffffu, term, o);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = term;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < kFp64Block / 32; ++w) s += sh[w];
            // one slot per (chunk, perturbation); the finalize kernel sums the
            // chunks of a stack in order, so the result is reproducible
            ka.ll_pert[(si.part_base + wi.chunk) * ka.n_pert + pert] = s;
        }
    }
}

// loglik = -1/2 sum; gradient by central differences.
template <int MODE>
__global__ void nr_fp64_finalize(const KernelArgs ka, int n_stacks)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_stacks) return;
    const StackInfo si = ka.stacks[s];
    const int n = si.n;
    const double *lp = ka.ll_pert + si.part_base * ka.n_pert;
    auto total = [&](int pert) {
        double acc = 0.0;
        for (int c = 0; c < si.n_chunks; ++c) acc += lp[(int64_t)c * ka.n_pert + pert];
        return acc;
    };
    if (ka.ll_out) ka.ll_out[s] = -0.5 * total(0);
    if (MODE != kGrad || ka.grad_out == nullptr) return;
    const double *p = ka.params + si.par_off;
    for (int i = 0; i < 4 * n + 6; ++i) {
        const double h = step_of(p[i], i, n);
        if (one_sided(p[i], i, n)) {
            const double up = (p[i] + h) - p[i];
            ka.grad_out[si.par_off + i] =
                -0.5 * (-3.0 * total(0) + 4.0 * total(2 * i + 1) - total(2 * i + 2)) / (2.0 * up);
        } else {
            // the actually represented steps, for an exact central quotient
            const double up = (p[i] + h) - p[i], dn = p[i] - (p[i] - h);
            ka.grad_out[si.par_off + i] = -0.5 * (total(2 * i + 1) - total(2 * i + 2)) / (up + dn);
        }
    }
}

} // namespace

cudaError_t launch_fp64(int mode, const KernelArgs &a, const QuadConst &qc, cudaStream_t st)
{
    if (a.n_items == 0) return cudaSuccess;
    dim3 grid(a.n_items, mode == kGrad ? a.n_pert : 1);
    switch (mode) {
    case kModel: nr_fp64_kernel<kModel><<<grid, kFp64Block, 0, st>>>(a, qc); break;
    case kLoglik: nr_fp64_kernel<kLoglik><<<grid, kFp64Block, 0, st>>>(a, qc); break;
    default: nr_fp64_kernel<kGrad><<<grid, kFp64Block, 0, st>>>(a, qc); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_fp64_finalize(int mode, int n_stacks, const KernelArgs &a, cudaStream_t st)
{
    if (n_stacks == 0 || mode == kModel) return cudaSuccess;
    const int blocks = (n_stacks + 127) / 128;
    if (mode == kGrad)
        nr_fp64_finalize<kGrad><<<blocks, 128, 0, st>>>(a, n_stacks);
    else
        nr_fp64_finalize<kLoglik><<<blocks, 128, 0, st>>>(a, n_stacks);
    return cudaGetLastError();
}

} // namespace nrimpl
