// nr_internal.h -- structures shared by the host API (nr_api.cpp) and the
// CUDA kernels (nr_mixed.cu, nr_pair.cu, nr_fp64.cu, ...) of the reflectivity library.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "nr.h"

namespace nrimpl {

// kGradRes: kGrad plus d loglik / d ln(resolution scale) per stack
enum Mode : int { kModel = 0, kLoglik = 1, kGrad = 2, kGradRes = 3 };
__host__ __device__ inline bool is_grad_mode(int mode) { return mode == kGrad || mode == kGradRes; }

// Lanes that share one Q point's smearing sum in the mixed kernels; a tile
// therefore holds at most (threads per CTA) / kSubLanes Q points.
constexpr int kSubLanes = 4;

// One stack of the batch, as the kernels see it.
struct StackInfo {
    int64_t par_off;   // first packed parameter
    int64_t out_off;   // first r_out element
    int64_t q_begin;   // first point of the stack's dataset in q/dq/r_obs/r_err
    int64_t part_base; // first partial-sum slot (doubles) when n_chunks > 1
    int32_t n;         // layers
    int32_t nq;        // dataset length
    int32_t n_chunks;  // work items of this stack
    int32_t pad;
};

// A contiguous range of Q points of one stack: the unit a CTA takes from the
// work queue.
struct WorkItem {
    int32_t stack;
    int32_t q_lo;  // first Q index within the dataset
    int32_t q_hi;  // one past the last
    int32_t chunk; // index among the stack's items (partial-sum slot)
};

// Entries of the kernels' sin / cos table (a power of two)
constexpr int kSinCosTabN = 128;

// Quadrature rule as the kernels use it: node offset q = Q + dQ * g_k with
// g_k = x_k / (2 sqrt(ln 2)) as a float pair (hi + lo) and as a double, and
// weight w_k / sqrt(pi).
struct QuadConst {
    float g_hi[NR_MAX_QUAD];
    float g_lo[NR_MAX_QUAD];
    float w[NR_MAX_QUAD];
    double gd[NR_MAX_QUAD];
    double wd[NR_MAX_QUAD];
    // cos(2 pi i / N) at [i], sin at [N + i], i < N = kSinCosTabN, correctly
    // rounded: the table of the kernels' sin / cos (nr_device.cuh, cis_tab)
    float cs_tab[2 * kSinCosTabN];
    int32_t K;
};

// The library's K-point Gauss-Hermite rule in the kernels' form (nr_api.cpp;
// host).  Returns false for K outside [1, NR_MAX_QUAD].
bool make_quad_const(int K, QuadConst &qc);

struct KernelArgs {
    const double *params;
    const float *q;
    const float *dq;
    const float *r_obs;
    const float *r_err;
    const StackInfo *stacks;
    const WorkItem *items;
    int32_t n_items;
    int32_t tile_q;      // Q points per CTA tile (mixed kernels)
    float *r_out;
    double *ll_out;
    double *grad_out;
    double *res_out;     // [n_stacks] d loglik / d ln(dQ scale) (kGradRes)
    double *partials;    // per-chunk raw sums of chunked stacks
    int32_t *stack_done; // per-stack arrival counters (self-resetting)
    int32_t *ticket;     // [2]: next work item, finished CTAs (self-resetting)
    int32_t *status;     // sticky NR_FLAG_* word
    const double *dq_scale; // [n_stacks] factor of every dQ of the stack's dataset (NULL: 1)
    // FP64 plain path only
    double *ll_pert;     // [(chunk slots) * n_pert] partial chi^2 sums per perturbation
    int32_t n_pert;      // 1, or 2 * max(4n+6) + 1 for central differences
    int32_t n_stacks;    // stacks of the batch (checked by NR_DEBUG builds)
};

// NR_DEBUG builds check on the device every work item a kernel takes (stack
// index, layer count against the launch's bucket, Q range, chunk index) and
// every interior-edge queue slot; a failed check sets NR_FLAG_DEBUG_BOUNDS in
// the status word and skips the access instead of trapping.  Release builds
// (NR_DEBUG 0) trust the plan, which the host builds from validated metadata.
#ifndef NR_DEBUG
#define NR_DEBUG 0
#endif
#ifdef __CUDACC__
// NR_DEBUG: does work item `wi` lie inside the batch?  Its stack index, the
// stack's layer count against the launch's capacity (nmax = 1: exactly one
// layer; 0: any count up to NR_MAX_LAYERS), its Q range within the stack's
// dataset and its chunk among the stack's items.  The stack record is read
// only once the index is known to be inside the array.
__device__ __forceinline__ bool item_in_bounds(const KernelArgs &ka, const WorkItem &wi, int nmax)
{
    if (wi.stack < 0 || wi.stack >= ka.n_stacks) return false;
    const StackInfo si = ka.stacks[wi.stack];
    const bool n_ok = nmax == 1 ? si.n == 1 : si.n >= 0 && si.n <= (nmax ? nmax : NR_MAX_LAYERS);
    return n_ok && wi.q_lo >= 0 && wi.q_lo <= wi.q_hi && wi.q_hi <= si.nq && wi.chunk >= 0 &&
           wi.chunk < si.n_chunks;
}
#endif

// ---- launchers (nr_mixed.cu) ----
// Mixed-precision kernels.  `nmax` is the register-array capacity bucket of
// the launch (every stack of the launch has n <= nmax; nmax = 1 means exactly
// one layer); 0 selects the runtime-n forward kernel (model / loglik modes).
// allow_pair = false keeps the one-evaluation kernel where the paired kernel
// (nr_pair.cu) would otherwise run (the autotuner times both).
int mixed_block_threads(int mode, int nmax);
// most Q points per CTA tile of a launch (quadrature order K)
int mixed_tile_q(int mode, int nmax, int K, bool allow_pair = true);
size_t mixed_dyn_smem(int mode, int nmax);
cudaError_t mixed_occupancy(int mode, int nmax, int K, int *blocks_per_sm, bool allow_pair = true);
cudaError_t launch_mixed(int mode, int nmax, int grid, const KernelArgs &a, const QuadConst &qc,
                         cudaStream_t st, bool allow_pair = true);
bool mixed_bucket_ok(int mode, int nmax);

// ---- paired kernel (nr_pair.cu): two evaluations per thread ----
// Used by launch_mixed / mixed_occupancy / mixed_tile_q when K >= 3 for the
// 1- and 2-layer gradient buckets and the 1-layer forward (model, loglik)
// bucket.
bool pair_eligible(int mode, int nmax, int K);
int pair_block_threads();
cudaError_t pair_occupancy(int mode, int nmax, int K, int *blocks_per_sm);
cudaError_t launch_pair(int mode, int nmax, int grid, const KernelArgs &a, const QuadConst &qc, cudaStream_t st);

// ---- launchers (nr_fp64.cu) ----
constexpr int kFp64Block = 128;
cudaError_t launch_fp64(int mode, const KernelArgs &a, const QuadConst &qc, cudaStream_t st);
cudaError_t launch_fp64_finalize(int mode, int n_stacks, const KernelArgs &a, cudaStream_t st);

// ---- SLD profiles (nr_profile.cu) ----
cudaError_t launch_profile(const double *params, const int64_t *par_off, const int32_t *n_layers, int n_stacks,
                           const float *z, int nz, float *rho_out, float *iota_out, int32_t *status, int sms,
                           cudaStream_t st);

// ---- co-fit samplers (nr_hmc.cu) ----
enum CofitStage : int { kStageLogp = 0, kStageFirst = 1, kStageMid = 2, kStageLast = 3 };
struct CofitStageArgs {
    int32_t C, P, NS, n_contrast; // chains, free parameters, packed slots per chain, contrasts per chain
    int32_t stage;
    double eps;                   // leapfrog step
    double *u;                    // [C x P] unconstrained position (updated)
    const double *ll;             // [C x n_contrast] log-likelihoods of the stacks
    const double *gpk;            // [C x NS] packed likelihood gradient
    const int32_t *tie_ptr;       // [P + 1] CSR over the slots that copy parameter k
    const int32_t *tie_slot;
    const double *lo, *hi;        // [P] prior bounds
    const double *inv_mass;       // [P]
    const double *z;              // [C x P] standard-normal momentum draws
    const double *log_unif;       // [C] log of the uniform acceptance draws
    double *mom;                  // [C x P] momentum (workspace)
    double *u0;                   // [C x P] starting position (workspace)
    double *H0, *logp0;           // [C] (workspace)
    int32_t res_param;            // free parameter scaling every dQ (-1: none)
    const double *gres;           // [C x n_contrast] d loglik / d ln f of the stacks (res_param >= 0)
    double *logp_out;             // [C] log pi of the resulting state (may be NULL)
    double *grad_out;             // [C x P] d log pi / du (kStageLogp; may be NULL)
    int32_t *accepted;            // [C] 1 accepted, 0 rejected (may be NULL)
};
// res_param >= 0: also dq_scale[c * NC + i] = theta_res of chain c (its NC stacks)
cudaError_t launch_cofit_gather(const double *u, int C, int P, int NS, const int32_t *src, const double *val,
                                const double *lo, const double *hi, double *params, int res_param, int NC,
                                double *dq_scale, cudaStream_t st);
cudaError_t launch_cofit_stage(const CofitStageArgs &a, cudaStream_t st);
// variational inference (nr_vi.cu)
// vi_sample advances the device iteration counter and writes the Adam bias
// corrections 1 / (1 - beta1^t), 1 / (1 - beta2^t) to bias[0..1]
cudaError_t launch_vi_sample(const double *phi, const double *eps, int R, int P, double *u, double *part,
                             int32_t *t_dev, double beta1, double beta2, double *bias, cudaStream_t st);
cudaError_t launch_vi_adam(double *phi, double *m, double *v, const double *eps, const double *g,
                           const double *logp, const double *part, int R, int P, const double *bias, double lr,
                           double beta1, double beta2, double eps_adam, double *elbo, cudaStream_t st);

// Raw per-stack sums of the mixed gradient kernels, and the stride of a
// chunk's partial-sum slot: [accD (n) | accUr (n+1) | accUi (n+1) |
// accS (n+1) | llsum | gscale | gbkg | gres].
__host__ __device__ inline int n_slot(int n) { return 4 * n + 7; }

} // namespace nrimpl
