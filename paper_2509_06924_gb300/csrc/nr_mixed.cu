// nr_mixed.cu -- batched reflectivity, log-likelihood and its exact gradient
// in complex FP32 with double-float guards, for sm_103a, one evaluation per
// thread.  The two-evaluations-per-thread kernels of nr_pair.cu run instead
// wherever they apply (K >= 3, gradient buckets up to 20 layers, both forward
// buckets); this kernel serves K < 3, the 32- and 64-layer gradient buckets,
// and builds with NR_PAIR=0, and the autotuner may pick it per bucket.
//
// Work decomposition.  A work item is a range of Q points of one stack.  A
// persistent CTA takes items from a queue (atomic ticket, cost-sorted on the
// host) and sweeps the item in tiles of TQ Q points x K quadrature nodes: one
// thread per (Q point, node) evaluation, the K threads of a Q point adjacent.
// The stack's parameters are staged once per item in shared memory (FP64 ->
// float pairs).  Per evaluation (Sec. 2.1 forward model, Sec. 3 smearing):
//   a1  node   q = Q + dQ x_k / (2 sqrt(ln 2))             double-float
//   a3  k_j = sqrt(k_0^2 - 4pi(rho_j - rho_0) + 4pi i iota_j)
//              k_0^2 - c_j in double-float, sqrt + one Newton step where a
//              layer phase needs it
//   a4  r_j = 4pi(drho_j + i diota_j) / (k_j + k_{j+1})^2 * exp(-2 k_j k_{j+1} s_j^2)
//              cancellation-free numerator (exactly k_j^2 - k_{j+1}^2)
//   a5  E_j = exp(2 i k_j d_j): phase 2 Re(k_j) d_j in double-float reduced
//              mod 2 pi before the FP32 sincos
//   a6  Parratt recursion from the backing up: X_n = r_n,
//       X_j = (r_j + X_{j+1} E_{j+1}) / (1 + r_j X_{j+1} E_{j+1}), R = |X_0|^2
//   a8  smearing: the K node values of a Q point meet in shared memory (one
//       barrier per tile, buffers alternate between tiles),
//   a9  m = scale S + bkg; loglik terms in a float pair, FP64 per item,
//   a10 dl/dm seeds the adjoint of every node,
//   a7  adjoint: a top-down sweep over the interfaces using the stored X_j
//       (and, for 1-2 layers, every stored intermediate; deeper stacks
//       recompute k_j, r_j, E_j), accumulating per-thread partial gradients.
// At the end of an item the CTA reduces its partials (warp shuffles, then a
// fixed-order cross-warp sum in FP64).  Stacks split over several items meet
// through per-chunk partial slots; the last arriving CTA sums them in chunk
// order, so results are bitwise reproducible.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "nr_device.cuh"
#include "nr_internal.h"

namespace nrimpl {
namespace {

// CTAs per SM the compiler is asked to fit (register cap) for the 1-layer
// gradient bucket and the forward kernels; overridable at build time.
#ifndef NR_MINB_GRAD1
#define NR_MINB_GRAD1 6
#endif
#ifndef NR_MINB_FWD
#define NR_MINB_FWD 4
#endif
// threads per CTA and CTAs per SM of the 1-layer forward (model / loglik)
// kernel; the rolled forward kernel keeps 256 threads and NR_MINB_FWD
#ifndef NR_BLOCK_FWD1
#define NR_BLOCK_FWD1 128
#endif
#ifndef NR_MINB_FWD1
#define NR_MINB_FWD1 8
#endif
// threads per CTA of the 1-layer gradient kernel
#ifndef NR_BLOCK_GRAD1
#define NR_BLOCK_GRAD1 128
#endif
// CTAs per SM of the 2- and 4-layer gradient buckets
#ifndef NR_MINB_SMALL
#define NR_MINB_SMALL 3
#endif
// gradient buckets of at least this many layers run 128-thread CTAs
#ifndef NR_DEEP_BLOCK128
#define NR_DEEP_BLOCK128 16
#endif
// unroll factor of the rolled (deep) forward and adjoint sweeps
#ifndef NR_DEEP_UNROLL
#define NR_DEEP_UNROLL 2
#endif
constexpr int kDeepUnroll = NR_DEEP_UNROLL;


// --------------------------------------------------------------- traits ---
template <int MODE, int NMAX>
struct Traits {
    static constexpr bool kGradMode = MODE == kGrad || MODE == kGradRes;
    static constexpr bool RES = MODE == kGradRes;               // + d loglik / d ln(dQ scale)
    static constexpr int NM = NMAX > 0 ? NMAX : NR_MAX_LAYERS; // smem capacity
    // deep gradient buckets run 128-thread CTAs so that their per-thread
    // state in shared memory still leaves room for several CTAs per SM
    static constexpr int BLOCK = !kGradMode ? (NMAX == 1 ? NR_BLOCK_FWD1 : 256)
                                 : NMAX == 1 ? NR_BLOCK_GRAD1 : NMAX >= NR_DEEP_BLOCK128 ? 128 : 256;
    static constexpr bool STORE = kGradMode && NMAX <= 2;     // keep all intermediates
    static constexpr bool UNROLL = NMAX >= 1 && NMAX <= 4;    // register arrays, unrolled sweeps
    static constexpr bool SMEM_ACC = kGradMode && !UNROLL;    // partials in shared memory
    static constexpr bool X_SMEM = kGradMode && !UNROLL;      // X_j in shared memory
    static constexpr int NACC = kGradMode ? 4 * NM + 3 : 0;   // partial gradients per thread
    static constexpr int NRAW = 4 * NM + 7;
    static constexpr int WARPS = BLOCK / 32;
    // interior-edge work queue per warp: unrolled kernels drain it after each
    // tile's sweep, rolled ones inside the sweep
    static constexpr int EQ_CAP = !kGradMode ? 1 : UNROLL ? 32 * NM + 32 : 64;
#ifndef NR_DEEP_REGS
#define NR_DEEP_REGS 96
#endif
    // register caps: rolled deep kernels are held to NR_DEEP_REGS per thread
    static constexpr int MINB = !kGradMode ? (NMAX == 1 ? NR_MINB_FWD1 : NR_MINB_FWD) : NMAX == 1 ? NR_MINB_GRAD1 : NMAX <= 4 ? NR_MINB_SMALL
                                : 65536 / (BLOCK * NR_DEEP_REGS);
    // Q points staged in shared memory per super-tile (several tiles)
    static constexpr int CAPQ = SMEM_ACC ? 96 : 256;
    static_assert(CAPQ >= BLOCK / kSubLanes, "a super-tile holds at least one tile");
    static constexpr size_t DYN = (SMEM_ACC ? (size_t)NACC * BLOCK * 4 : 0) +
                                  (X_SMEM ? (size_t)(NM + 1) * BLOCK * 8 : 0);
};

// ---------------------------------------------------------------- kernel --
template <int MODE, int NMAX, int KC>
__global__ void __launch_bounds__(Traits<MODE, NMAX>::BLOCK, Traits<MODE, NMAX>::MINB)
nr_mixed_kernel(const KernelArgs ka, const QuadConst qc)
{
    using T = Traits<MODE, NMAX>;
    constexpr int NM = T::NM;
    constexpr int BLOCK = T::BLOCK;
    constexpr bool GRAD = T::kGradMode;
    constexpr bool RES = T::RES;
    constexpr bool LIK = MODE != kModel;
    constexpr int EQ = T::EQ_CAP;

    __shared__ StackSmem<NM> sm;
    __shared__ float sh_cs[2 * kTabN];                   // cos, sin at multiples of 2 pi / kTabN
    __shared__ __align__(16) float sh_wR[2][2 * BLOCK]; // w_k R per (Q slot, node), double-buffered
    // the super-tile's data per Q point: (Q/2, dQ/2, R_obs, 1/err), and the
    // (residual, smeared R) pairs its tiles leave for the likelihood sums
    __shared__ float4 sh_qd[T::CAPQ];
    __shared__ float2 sh_rs[LIK ? T::CAPQ : 1];
    __shared__ double sh_red[T::WARPS][32];
    __shared__ double sh_redd[T::WARPS][4];
    __shared__ double sh_raw[T::NRAW];
    __shared__ int sh_item;
    __shared__ int sh_last;
    // interior-edge queue per warp: k_{j-1}, k_j, k_{j+1}, Z, Xbar_{j-1} and
    // the medium j; the rolled sweeps keep the node k_0 in place of the three
    // wavevectors (smaller entries, more CTAs per SM); the resolution mode
    // adds the factor that turns the entry's conj(kbar)/k into d/d ln f
    constexpr int EQF = (T::SMEM_ACC ? 3 : 5) + (RES ? 1 : 0); // RES: + k_0 dk_0/dln f
    __shared__ float2 sh_eq[GRAD ? T::WARPS : 1][EQF][EQ];
    __shared__ int sh_eqj[GRAD ? T::WARPS : 1][EQ];
    extern __shared__ __align__(16) float sh_dyn[]; // [NACC][BLOCK] partials, then [NM+1][BLOCK] X_j
    float *sh_acc = sh_dyn;
    float2 *sh_X = reinterpret_cast<float2 *>(sh_dyn + (T::SMEM_ACC ? T::NACC * BLOCK : 0));

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int K = KC > 0 ? KC : qc.K; // KC: quadrature order fixed at compile time (0: runtime)
    // node stride of a Q slot in sh_wR: K rounded up to whole float4s (the
    // padding stays 0), so a slot's values are read 4 at a time
    const int KP = (K + 3) & ~3;
    const int TQ = ka.tile_q;
    const int qslot = tid / K;
    const int kn = tid - qslot * K;
    const bool lane_on = qslot < TQ;
    const float g_hi = lane_on ? qc.g_hi[kn] : 0.f;
    const float g_lo = lane_on ? qc.g_lo[kn] : 0.f;
    const float wk = lane_on ? qc.w[kn] : 0.f;
    // the warp's Q slots for the smearing sums and the lanes per slot
    // (sgl depends on K only, so a Q point's sum has the same order in every
    // warp and tile shape)
    const int qs0 = (warp * 32) / K;
    const int nslots = (31 + K - 1) / K + 1; // most slots any warp touches
    const int sgl = nslots <= 1 ? 32 : nslots <= 2 ? 16 : nslots <= 4 ? 8 : nslots <= 8 ? 4 : nslots <= 16 ? 2 : 1;
    // widest node offset |g_k|: the nodes of a Q point lie within Q/2 +- |dQ/2| g_max
    const float g_max = fmaxf(fabsf(qc.g_hi[0]), fabsf(qc.g_hi[K - 1]));

    for (int i = tid; i < 4 * BLOCK; i += BLOCK) (&sh_wR[0][0])[i] = 0.f; // padding stays 0
    for (int i = tid; i < 2 * kTabN; i += BLOCK) sh_cs[i] = qc.cs_tab[i];   // read after the item barrier

    for (;;) {
        if (tid == 0) sh_item = atomicAdd(&ka.ticket[0], 1);
        __syncthreads();
        const int item = sh_item;
        if (item >= ka.n_items) break;
        const WorkItem wi = ka.items[item];
        if constexpr (NR_DEBUG) {
            if (!item_in_bounds(ka, wi, NMAX)) { // uniform over the block
                if (tid == 0) atomicOr(ka.status, NR_FLAG_DEBUG_BOUNDS);
                __syncthreads(); // every thread has read sh_item
                continue;
            }
        }
        const StackInfo si = ka.stacks[wi.stack];
        // the 1-layer bucket holds exactly-1-layer stacks: n is a constant there
        const int n = (NMAX == 1 && NR_EXACT1) ? 1 : si.n;
        const double *p = ka.params + si.par_off;
        stage_stack<NM>(sm, p, n, tid, ka.status);

        // per-thread partial gradients (FP32; reduced in FP64 per item)
        float accr[GRAD && !T::SMEM_ACC ? T::NACC : 1];
        if constexpr (GRAD) {
            if constexpr (T::SMEM_ACC) {
                for (int i = 0; i < T::NACC; ++i) sh_acc[i * BLOCK + tid] = 0.f;
            } else {
#pragma unroll
                for (int i = 0; i < T::NACC; ++i) accr[i] = 0.f;
            }
        }
        constexpr int oD = 0, oUr = NM, oUi = 2 * NM + 1, oS = 3 * NM + 2;
        auto acc_add = [&](int idx, float v) __attribute__((always_inline)) {
            if constexpr (GRAD) {
                if constexpr (T::SMEM_ACC) sh_acc[idx * BLOCK + tid] += v;
                else accr[idx] += v;
            }
        };
        // acc[idx] += a b + c d, fused into the accumulator
        auto acc_fma2 = [&](int idx, float a, float b, float c, float d) __attribute__((always_inline)) {
            if constexpr (GRAD) {
                if constexpr (T::SMEM_ACC) {
                    float *ap = sh_acc + idx * BLOCK + tid;
                    *ap = fmaf(a, b, fmaf(c, d, *ap));
                } else {
                    accr[idx] = fmaf(a, b, fmaf(c, d, accr[idx]));
                }
            }
        };
        // medium j (runtime) -> its u accumulators
        auto acc_u = [&](int j, float2 v) __attribute__((always_inline)) {
            if constexpr (GRAD) {
                if constexpr (T::SMEM_ACC) {
                    acc_add(oUr + j - 1, v.x);
                    acc_add(oUi + j - 1, v.y);
                } else {
#pragma unroll
                    for (int t = 1; t <= NM; ++t)
                        if (t == j) {
                            accr[oUr + t - 1] += v.x;
                            accr[oUi + t - 1] += v.y;
                        }
                }
            }
        };
        float gres_acc = 0.f; // per-thread d loglik / d ln(dQ scale) (RES)
        int eq_cnt = 0; // entries in this warp's interior-edge queue (warp-uniform)
        // drain `cnt` <= 32 queued entries, one per lane, then shift the rest down
        auto eq_drain = [&](int cnt) {
            if constexpr (T::SMEM_ACC) {
                gres_acc += eq_drain_smem<EQ, RES>(sh_eq[warp], sh_eqj[warp], sm.med, sm.lay, n, lane, cnt,
                                                   sh_acc + oUr * BLOCK + tid, BLOCK, (oUi - oUr) * BLOCK);
            } else if (lane < cnt) {
                const int j = sh_eqj[warp][lane];
                const float2 ub = edge_ubar(sh_eq[warp][0][lane], sh_eq[warp][1][lane], sh_eq[warp][2][lane],
                                            sm.lay[j - 1].w, sm.lay[j].w, 0.5f * sm.lay[j].x, sh_eq[warp][3][lane],
                                            j == n, sh_eq[warp][4][lane]);
                // conj(kbar)/k_j = 2 conj(ubar)
                acc_u(j, make_float2(2.f * ub.x, -2.f * ub.y));
                if constexpr (RES) gres_acc = fmaf(2.f * ub.x, sh_eq[warp][EQF - 1][lane].x, gres_acc);
            }
            __syncwarp();
            const int rest = eq_cnt - cnt;
            for (int e = lane; e < rest; e += 32) {
                const int src = cnt + e;
#pragma unroll
                for (int f = 0; f < EQF; ++f) sh_eq[warp][f][e] = sh_eq[warp][f][src];
                sh_eqj[warp][e] = sh_eqj[warp][src];
            }
            __syncwarp();
            eq_cnt = rest;
        };

        // per-thread sums of the loglik terms, d/dscale, d/dbkg
        float ll_hi = 0.f, ll_lo = 0.f, gsc_acc = 0.f, gbk_acc = 0.f;

        // Q data are staged per super-tile (span Q points, a whole number of
        // tiles) by all threads at once, as (Q/2, dQ/2, R_obs, 1/err).  The tiles of a super-tile leave one
        // (residual, S) pair per Q point in sh_rs; the likelihood terms of a
        // super-tile are summed with full warps when the next one is staged
        // (and after the last tile), not by one lane per Q point per tile.
        const float *qp = ka.q + si.q_begin, *dqp = ka.dq + si.q_begin;
        const float fsc = ka.dq_scale ? (float)ka.dq_scale[wi.stack] : 1.f; // resolution scale of the stack
        const float *rop = ka.r_obs + si.q_begin, *rep = ka.r_err + si.q_begin;
        const int span = (T::CAPQ / TQ) * TQ;
        int sb = wi.q_lo;     // first Q point of the staged super-tile
        int s_next = wi.q_lo; // first Q point of the next one
        int s_cnt = 0;        // staged Q points whose pairs await summation
        auto consume = [&](int i) __attribute__((always_inline)) {
            if constexpr (LIK) {
                const float2 rs = sh_rs[i];
                const float Re = __ldg(rep + sb + i);
                if (!(Re > 0.f)) atomicOr(ka.status, NR_FLAG_BAD_ERR);
                float t1, t2;
                two_sum(ll_hi, fmaf(rs.x, rs.x, kLog2Pi + 2.f * logf(Re)), t1, t2);
                ll_hi = t1;
                ll_lo += t2;
                if constexpr (GRAD) {
                    const float dldm = -(rs.x * fabsf(sh_qd[i].w));
                    gsc_acc = fmaf(dldm, rs.y, gsc_acc);
                    gbk_acc += dldm;
                }
            }
        };
        auto restage = [&](int q0) {
            __syncthreads(); // the previous super-tile's reads and pairs are complete
            for (int i = tid; i < span; i += BLOCK) {
                if (i < s_cnt) consume(i);
                const int qa = q0 + i;
                // past the last Q point: a harmless node whose residual, and
                // so adjoint seed, is 0 (1/err = 0)
                float4 v = make_float4(0.05f, 0.f, 0.f, 0.f);
                if (qa < wi.q_hi) {
                    v.x = 0.5f * __ldg(qp + qa);
                    v.y = 0.5f * fsc * __ldg(dqp + qa);
                    if (LIK) {
                        v.z = __ldg(rop + qa);
                        v.w = rcp_approx(__ldg(rep + qa));
                    }
                    if constexpr (GRAD) {
                        // can a node of this Q point reach the interior-edge band
                        // |k_j|^2 < f k_0^2 of a layer (k_0^2 within c_j / (1 +- f))?
                        // The sign of 1/err carries the answer (negative: yes).
                        const float a = fabsf(v.y) * g_max;
                        const float lo = fmaxf(v.x - a, 0.f), hi = v.x + a;
                        const float k2lo = lo * lo * (1.f - 1.5f * kEdgeFrac);
                        const float k2hi = hi * hi * (1.f + 1.5f * kEdgeFrac);
                        bool e = false;
                        for (int j = 1; j <= n; ++j) {
                            const float c = sm.med[j].x;
                            e |= c > 0.f && c < k2hi && c > k2lo;
                        }
                        if (e && v.w > 0.f) v.w = -v.w;
                    }
                }
                sh_qd[i] = v;
            }
            sb = q0;
            s_next = q0 + span;
            s_cnt = min(span, wi.q_hi - q0);
            __syncthreads();
        };
        __syncthreads();

        const float scale = sm.scale, bkg = sm.bkg;
        const float wks = wk * scale;
        int buf = 0;
        for (int q0 = wi.q_lo; q0 < wi.q_hi; q0 += TQ, buf ^= 1) {
            if (q0 == s_next) restage(q0);
            const int qi = q0 + qslot;
            // this lane's super-tile entry (idle lanes past the last Q slot
            // read slot 0 and write nothing)
            const int si_q = q0 - sb + (lane_on ? qslot : 0);
            const bool act = lane_on && qi < wi.q_hi;
            const float4 qd = sh_qd[si_q];
            // a1: node position k_0 = q/2 in double-float (Q and dQ are staged
            // halved, exactly), k_0^2
            float k0h, k0l;
            {
                const float th = __fmul_rn(qd.y, g_hi);
                float tl = fmaf(qd.y, g_hi, -th);
                tl = fmaf(qd.y, g_lo, tl);
                float s, e;
                two_sum(qd.x, th, s, e);
                e = __fadd_rn(e, tl);
                fast_two_sum(s, e, k0h, k0l);
            }
            const bool qok = k0h > 0.f;
            if (act && !qok) atomicOr(ka.status, NR_FLAG_BAD_Q);
            float p_hi, p_lo;
            k0_square(k0h, k0l, p_hi, p_lo);

            // a3-a6 forward, from the backing upwards
            Kz kst[T::STORE ? NM + 2 : 1];
            float2 rst[T::STORE ? NM + 1 : 1], Gst[T::STORE ? NM + 1 : 1];
            float2 Est[T::STORE ? NM + 2 : 1], Dst[T::STORE ? NM + 1 : 1], Yst[T::STORE ? NM + 1 : 1];
            float2 Xr[GRAD && T::UNROLL ? NM + 1 : 1];
            auto Xput = [&](int j, float2 v) __attribute__((always_inline)) {
                if constexpr (GRAD) {
                    if constexpr (T::X_SMEM) sh_X[j * BLOCK + tid] = v;
                    else Xr[j] = v;
                }
            };
            auto Xget = [&](int j) __attribute__((always_inline)) -> float2 {
                if constexpr (T::X_SMEM) return sh_X[j * BLOCK + tid];
                else if constexpr (GRAD) return Xr[j];
                else return make_float2(0.f, 0.f);
            };
            Kz kbelow = medium_kz<false>(p_hi, p_lo, sm.med[n + 1]);
            float2 Xbelow = make_float2(0.f, 0.f);
            // TOP: j == 0 (fronting), BOT: j == n (last interface)
            auto fwd_step = [&](int j, auto TOP, auto BOT) __attribute__((always_inline)) {
                const bool top = pos_flag(TOP, j == 0), bot = pos_flag(BOT, j == n);
                Kz kj;
                if (top) {
                    kj.re = k0h; kj.im = 0.f; kj.lo = k0l;
                } else {
                    kj = medium_kz<true>(p_hi, p_lo, sm.med[j]);
                }
                float2 Gj, kkj;
                // k_0 is real: the real-k_a form there
                const float4 Ij = sm.itf[j];
                const float2 rj = top ? fresnel_nc<true>(kc(kj), kc(kbelow), Ij, Gj, kkj, sh_cs)
                                      : fresnel_nc<false>(kc(kj), kc(kbelow), Ij, Gj, kkj, sh_cs);
                float2 Xj;
                if (bot) {
                    Xj = rj;
                    if constexpr (T::STORE) kst[j + 1] = kbelow;
                } else {
                    const float2 Ej = layer_phase(kbelow, sm.lay[j + 1], sh_cs);
                    const float2 Yj = cmul(Xbelow, Ej);
                    float2 Dj;
                    Xj = mobius(rj, Yj, Dj);
                    if constexpr (T::STORE) { Est[j + 1] = Ej; Dst[j] = Dj; Yst[j] = Yj; }
                }
                if constexpr (T::STORE) { kst[j] = kj; rst[j] = rj; Gst[j] = Gj; }
                Xput(j, Xj);
                Xbelow = Xj;
                kbelow = kj;
            };
            if constexpr (T::UNROLL) {
#pragma unroll
                for (int j = NM; j >= 0; --j)
                    if (j <= n) fwd_step(j, Pos<kRt>{}, Pos<kRt>{});
            } else {
                fwd_step(n, Pos<kRt>{}, Pos<kYes>{});
#pragma unroll kDeepUnroll
                for (int j = n - 1; j >= 1; --j) fwd_step(j, Pos<kNo>{}, Pos<kNo>{});
                if (n >= 1) fwd_step(0, Pos<kYes>{}, Pos<kNo>{});
            }
            float R = Xbelow.x * Xbelow.x + Xbelow.y * Xbelow.y;
            if (!qok) R = __int_as_float(0x7fffffff);

            // a8-a10: smearing sum, model, likelihood, adjoint seed.  Every
            // lane of a Q point forms the same sum from shared memory, so the
            // seed needs no second barrier.
            // (a lane past the item's last Q point adds a finite value to
            // a slot whose sum is never used)
            if (lane_on) sh_wR[buf][qslot * KP + kn] = wk * R;
            __syncthreads();
            float Rb = 0.f;
            // smearing sums of the Q slots this warp touches: sgl lanes per
            // slot add strided nodes, a shuffle tree finishes, and every lane
            // picks its own slot's sum (same order in every warp)
            float S;
            {
                const int g = lane / sgl, part = lane - g * sgl;
                const int slot = qs0 + g;
                float ps = 0.f;
                if (slot < TQ) {
                    const float4 *row = reinterpret_cast<const float4 *>(&sh_wR[buf][slot * KP]);
                    auto add4 = [&](int c) __attribute__((always_inline)) {
                        const float4 v = row[c];
                        ps += (v.x + v.y) + (v.z + v.w);
                    };
                    if constexpr (KC > 0) {
                        // compile-time trip count: the strided float4s of this part
                        constexpr int NSL = (31 + KC - 1) / KC + 1;
                        constexpr int SGL = NSL <= 1 ? 32 : NSL <= 2 ? 16 : NSL <= 4 ? 8 : NSL <= 8 ? 4
                                                                                : NSL <= 16 ? 2 : 1;
#pragma unroll
                        for (int i = 0; i < ((KC + 3) / 4 + SGL - 1) / SGL; ++i)
                            if (part + i * SGL < (KC + 3) / 4) add4(part + i * SGL);
                    } else {
                        for (int c = part; c < KP / 4; c += sgl) add4(c);
                    }
                }
                for (int o = 1; o < sgl; o <<= 1) ps += __shfl_xor_sync(kFull, ps, o);
                S = __shfl_sync(kFull, ps, ((qslot - qs0) * sgl) & 31);
            }
            if constexpr (MODE == kModel) {
                if (act && kn == 0) ka.r_out[si.out_off + qi] = fmaf(scale, S, bkg);
            } else {
                const float m = fmaf(scale, S, bkg);
                const float ie = fabsf(qd.w);
                const float res = (m - qd.z) * ie; // (m - R) / err
                if (act && kn == 0) sh_rs[si_q] = make_float2(res, S);
                if constexpr (GRAD) Rb = wks * -(res * ie); // w_k scale dl/dm (0 on idle lanes)
            }
            if constexpr (GRAD) {
                // a7: adjoint sweep from the fronting down to the backing
                float2 Xb = cscale(Xget(0), 2.f * Rb);
                float2 kbar = make_float2(0.f, 0.f); // adjoint of k_j (j >= 1)
                Kz kj;
                kj.re = k0h; kj.im = 0.f; kj.lo = k0l;
                float2 Xb_up = make_float2(0.f, 0.f);  // adjoint of X_{j-1}
                Kz kjm1 = kj;                          // k_{j-1} (unrolled queue entries)
                const float edge_u = kEdgeFrac * k0h * k0h;
                // resolution mode: every k_j depends on the node k_0 (dk_j/dk_0 =
                // k_0/k_j, dk_0/dk_0 = 1) and dk_0/d ln f = (dQ/2) g_k, so
                // d loglik/d ln f gains (dQ/2) g_k [Re kbar_0 + k_0 sum_j Re(conj(kbar_j)/k_j)]
                const float wres = RES ? qd.y * g_hi : 0.f;
                float res_sum = 0.f, res_k0 = 0.f;
                auto acc_u_nonedge = [&](int idx, float re, float im) __attribute__((always_inline)) {
                    acc_add(oUr + idx, re);
                    acc_add(oUi + idx, im);
                    if constexpr (RES) res_sum += re;
                };
                // EDG: the warp's tile may hold interior-edge evaluations (else
                // the edge test and its queue are compiled out of the sweep)
                auto adj_step = [&](int j, auto TOP, auto BOT, auto EDG) __attribute__((always_inline)) {
                    const bool top = pos_flag(TOP, j == 0), bot = pos_flag(BOT, j == n);
                    const float4 Ij = sm.itf[j];
                    const float4 Lj1 = sm.lay[j + 1]; // layer j+1 (zeros past the last layer)
                    const float2 Xb_in = Xb;
                    float2 Zj = make_float2(0.f, 0.f);
                    Kz kj1;
                    float2 rj, Gj, kkj;
                    if constexpr (T::STORE) {
                        kj1 = kst[j + 1];
                        rj = rst[j];
                        Gj = Gst[j];
                    } else {
                        const float4 Mj1 = sm.med[j + 1];
                        kj1 = bot ? medium_kz<false>(p_hi, p_lo, Mj1) : medium_kz<true>(p_hi, p_lo, Mj1);
                        rj = top ? fresnel_nc<true>(kc(kj), kc(kj1), Ij, Gj, kkj, sh_cs)
                                 : fresnel_nc<false>(kc(kj), kc(kj1), Ij, Gj, kkj, sh_cs);
                    }
                    float2 kbar1 = make_float2(0.f, 0.f);
                    float2 rb;
                    if (!bot) {
                        const float2 X1 = Xget(j + 1);
                        float2 Ej1, Dj, Y;
                        if constexpr (T::STORE) {
                            Ej1 = Est[j + 1];
                            Dj = Dst[j];
                            Y = Yst[j];
                        } else {
                            Ej1 = layer_phase(kj1, Lj1, sh_cs);
                            Y = cmul(X1, Ej1);
                            const float2 rY = cmul(rj, Y);
                            const float dx = 1.f + rY.x, dy = rY.y;
                            const float inv = rcp_approx(fmaf(dx, dx, dy * dy));
                            Dj = make_float2(dx * inv, -dy * inv);
                        }
                        Zj = Y;
                        // dX/dr = (1 - Y^2) D^2, dX/dY = (1 - r^2) D^2: both
                        // adjoints share V = conj(D^2) Xbar
                        const float2 V = cmulc(Dj, cmulc(Dj, Xb));
                        rb = cmulc(one_minus_sq(Y), V);
                        const float2 Yb = cmulc(one_minus_sq(rj), V);
                        Xb = cmulc(Ej1, Yb);
                        // Y = X_{j+1} E_{j+1}: dY/dd = 2 i k Y and dY/dk = 2 i d Y.
                        // With U = conj(Y) Ybar the d_{j+1} sum takes
                        // Re(k) Im(U) - Im(k) Re(U) (halved) and kbar_{j+1} = -2 i d U.
                        const float2 U = cmulc(Y, Yb);
                        acc_fma2(oD + j, kj1.re, U.y, -kj1.im, U.x);
                        const float dd = Lj1.x;
                        kbar1 = make_float2(dd * U.y, -dd * U.x);
                    } else {
                        rb = Xb;
                    }
                    // dr/dk_j = k_{j+1} P and dr/dk_{j+1} = k_j M with
                    // P = 2G + s r, M = s r - 2G.  With rr = conj(rbar) r
                    // (also the roughness term) and g = conj(G) rbar:
                    // conj(M) rbar = s conj(rr) - 2g, conj(P) rbar = s conj(rr) + 2g
                    const float sj = Ij.z;
                    const float2 rr = cmulc(rb, rj);             // accS += Re(rr k_j k_{j+1})
                    const float2 gg = cmulc(Gj, rb);
                    const float2 sr = make_float2(sj * rr.x, -sj * rr.y);
                    const float2 H = make_float2(fmaf(-2.f, gg.x, sr.x), fmaf(-2.f, gg.y, sr.y)); // conj(M) rbar
                    const bool k_real = top;                     // k_0 is real
                    if (k_real) kbar1 = make_float2(fmaf(kj.re, H.x, kbar1.x), fmaf(kj.re, H.y, kbar1.y));
                    else kbar1 = cfmac(kc(kj), H, kbar1);
                    // k_j k_{j+1} (the recomputing sweeps have it from fresnel_nc)
                    if constexpr (T::STORE)
                        kkj = k_real ? make_float2(kj.re * kj1.re, kj.re * kj1.im) : cmul(kc(kj), kc(kj1));
                    acc_fma2(oS + j, rr.x, kkj.x, -rr.y, kkj.y);
                    if (RES && top) {
                        // kbar_0 = conj(k_1) conj(P) rbar (the fronting has no phase)
                        const float2 H2 = make_float2(fmaf(2.f, gg.x, sr.x), fmaf(2.f, gg.y, sr.y));
                        res_k0 = fmaf(kj1.re, H2.x, kj1.im * H2.y);
                    }
                    if (!top) {
                        const float2 H2 = make_float2(fmaf(2.f, gg.x, sr.x), fmaf(2.f, gg.y, sr.y)); // conj(P) rbar
                        kbar = cfmac(kc(kj1), H2, kbar);
                        // k_j complete: accumulate conj(kbar) / k_j, or queue
                        // the interior-edge evaluation for this lane
                        const float m2 = fmaf(kj.re, kj.re, kj.im * kj.im);
                        const bool edge = decltype(EDG)::value && act && m2 < edge_u;
                        const unsigned em = decltype(EDG)::value ? __ballot_sync(kFull, edge) : 0u;
                        if (em) {
                            if (edge) {
                                const int slot = queue_slot<EQ>(eq_cnt + __popc(em & ((1u << lane) - 1u)), ka.status);
                                if constexpr (RES) sh_eq[warp][EQF - 1][slot] = make_float2(k0h * wres, 0.f);
                                if constexpr (T::SMEM_ACC) {
                                    sh_eq[warp][0][slot] = make_float2(k0h, k0l);
                                    sh_eq[warp][1][slot] = Zj;
                                    sh_eq[warp][2][slot] = Xb_up;
                                } else {
                                    sh_eq[warp][0][slot] = kc(kjm1);
                                    sh_eq[warp][1][slot] = kc(kj);
                                    sh_eq[warp][2][slot] = kc(kj1);
                                    sh_eq[warp][3][slot] = Zj;
                                    sh_eq[warp][4][slot] = Xb_up;
                                }
                                sh_eqj[warp][slot] = j;
                            }
                            eq_cnt = queue_count<EQ>(eq_cnt + __popc(em));
                            if constexpr (!T::UNROLL) {
                                if (eq_cnt >= 32) {
                                    __syncwarp();
                                    eq_drain(32);
                                }
                            }
                        }
                        if (!edge) {
                            const float2 kq = cmul(kbar, kc(kj));
                            const float inv = m2 > 0.f ? rcp_approx(m2) : 0.f;
                            acc_u_nonedge(j - 1, kq.x * inv, -kq.y * inv);
                        }
                    }
                    Xb_up = Xb_in;
                    kbar = kbar1;
                    kjm1 = kj;
                    kj = kj1;
                    if (bot) { // backing medium n+1: its k is complete as well
                        const float2 kk = cmul(kbar, kc(kj));
                        const float m2 = fmaf(kj.re, kj.re, kj.im * kj.im);
                        const float inv = m2 > 0.f ? rcp_approx(m2) : 0.f;
                        acc_u_nonedge(j, kk.x * inv, -kk.y * inv);
                    }
                };
                auto sweep = [&](auto EDG) __attribute__((always_inline)) {
                    if constexpr (T::UNROLL) {
#pragma unroll
                        for (int j = 0; j <= NM; ++j)
                            if (j <= n) adj_step(j, Pos<kRt>{}, Pos<kRt>{}, EDG);
                        // drain full batches of the interior-edge queue
                        if constexpr (decltype(EDG)::value) {
                            while (eq_cnt >= 32) {
                                __syncwarp();
                                eq_drain(32);
                            }
                        }
                    } else {
                        if (n >= 1) adj_step(0, Pos<kYes>{}, Pos<kNo>{}, EDG);
#pragma unroll kDeepUnroll
                        for (int j = 1; j <= n - 1; ++j) adj_step(j, Pos<kNo>{}, Pos<kNo>{}, EDG);
                        adj_step(n, Pos<kRt>{}, Pos<kYes>{}, EDG);
                    }
                };
                // the staged sign of 1/err marks Q points whose nodes may reach
                // an interior-edge band (warp-uniform choice)
                if (__any_sync(kFull, act && qd.w < 0.f)) sweep(std::true_type{});
                else sweep(std::false_type{});
                if constexpr (RES) gres_acc = fmaf(wres, fmaf(k0h, res_sum, res_k0), gres_acc);
            }
        }

        if constexpr (LIK) {
            if constexpr (GRAD) {
                if (eq_cnt > 0) {
                    __syncwarp();
                    eq_drain(eq_cnt);
                }
            }
            // ---- CTA reduction of the item's partial sums into sh_raw ----
            __syncthreads();
            for (int i = tid; i < s_cnt; i += BLOCK) consume(i);
            if constexpr (GRAD && !T::SMEM_ACC) {
                static_assert(T::NACC <= 32, "register partials exceed one reduction batch");
#pragma unroll
                for (int t = 0; t < T::NACC; ++t) {
                    float v = accr[t];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
                    if (lane == 0) sh_red[warp][t] = (double)v;
                }
                __syncthreads();
                if (tid < T::NACC) {
                    const int t = tid;
                    // accumulator slot -> raw index for this stack's n (-1: unused)
                    const int i = t < NM ? (t < n ? t : -1)
                                  : t < 2 * NM + 1 ? (t - NM <= n ? n + (t - NM) : -1)
                                  : t < 3 * NM + 2 ? (t - 2 * NM - 1 <= n ? 2 * n + 1 + (t - 2 * NM - 1) : -1)
                                                   : (t - 3 * NM - 2 <= n ? 3 * n + 2 + (t - 3 * NM - 2) : -1);
                    if (i >= 0) {
                        double s = 0.0;
                        for (int w = 0; w < T::WARPS; ++w) s += sh_red[w][t];
                        sh_raw[i] = s;
                    }
                }
                __syncthreads();
            }
            const int nraw = (GRAD && T::SMEM_ACC) ? 4 * n + 3 : 0;
            for (int base = 0; base < nraw; base += 32) {
                const int cnt = min(32, nraw - base);
                for (int c = 0; c < cnt; ++c) {
                    const int i = base + c;
                    const int idx = i < n ? i
                                    : i < 2 * n + 1 ? NM + (i - n)
                                    : i < 3 * n + 2 ? 2 * NM + 1 + (i - 2 * n - 1)
                                                    : 3 * NM + 2 + (i - 3 * n - 2);
                    float v = 0.f;
                    if constexpr (GRAD && T::SMEM_ACC) v = sh_acc[idx * BLOCK + tid];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
                    if (lane == 0) sh_red[warp][c] = (double)v;
                }
                __syncthreads();
                if (tid < cnt) {
                    double s = 0.0;
                    for (int w = 0; w < T::WARPS; ++w) s += sh_red[w][tid];
                    sh_raw[base + tid] = s;
                }
                __syncthreads();
            }
            {   // per-thread loglik (float pair), d/dscale, d/dbkg, d/d ln(dQ scale):
                // warp sums stay on the FP32 pipe, FP64 only across warps
                float h = ll_hi, l = ll_lo, a1 = gsc_acc, a2 = gbk_acc, a3 = gres_acc;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float h2 = __shfl_xor_sync(kFull, h, o), l2 = __shfl_xor_sync(kFull, l, o);
                    float s, e;
                    two_sum(h, h2, s, e);
                    h = s;
                    l = __fadd_rn(__fadd_rn(l, l2), e);
                    a1 += __shfl_xor_sync(kFull, a1, o);
                    a2 += __shfl_xor_sync(kFull, a2, o);
                    if constexpr (RES) a3 += __shfl_xor_sync(kFull, a3, o);
                }
                if (lane == 0) {
                    sh_redd[warp][0] = (double)h + (double)l;
                    sh_redd[warp][1] = a1;
                    sh_redd[warp][2] = a2;
                    sh_redd[warp][3] = a3;
                }
            }
            __syncthreads();
            if (tid < (RES ? 4 : 3)) {
                double s = 0.0;
                for (int w = 0; w < T::WARPS; ++w) s += sh_redd[w][tid];
                sh_raw[4 * n + 3 + tid] = s;
            }
            __syncthreads();
            const int nout = GRAD ? 4 * n + (RES ? 7 : 6) : 1;
            const int off0 = GRAD ? 0 : 4 * n + 3; // loglik mode: llsum only
            if (si.n_chunks == 1) {
                finalize_stack<MODE>(sh_raw, n, p, wi.stack, si.par_off, ka.ll_out, ka.grad_out, ka.res_out,
                                     tid, BLOCK);
            } else {
                double *slot = ka.partials + si.part_base + (int64_t)wi.chunk * n_slot(n);
                for (int i = tid; i < nout; i += BLOCK) slot[off0 + i] = sh_raw[off0 + i];
                __threadfence();
                __syncthreads();
                if (tid == 0) {
                    const int prev = atomicAdd(&ka.stack_done[wi.stack], 1);
                    sh_last = prev == si.n_chunks - 1;
                }
                __syncthreads();
                if (sh_last) {
                    __threadfence();
                    for (int i = tid; i < nout; i += BLOCK) {
                        double s = 0.0;
                        for (int c = 0; c < si.n_chunks; ++c)
                            s += __ldcg(ka.partials + si.part_base + (int64_t)c * n_slot(n) + off0 + i);
                        sh_raw[off0 + i] = s;
                    }
                    __syncthreads();
                    finalize_stack<MODE>(sh_raw, n, p, wi.stack, si.par_off, ka.ll_out, ka.grad_out,
                                         ka.res_out, tid, BLOCK);
                    if (tid == 0) ka.stack_done[wi.stack] = 0;
                }
            }
        }
        __syncthreads(); // sm / sh_raw / sh_item / sh_wR reused by the next item
    }
    // last CTA out resets the queue for the next launch
    if (tid == 0) {
        __threadfence();
        const int done = atomicAdd(&ka.ticket[1], 1);
        if (done == (int)gridDim.x - 1) {
            ka.ticket[0] = 0;
            ka.ticket[1] = 0;
            __threadfence();
        }
    }
}

template <int MODE, int NMAX, int KC>
cudaError_t set_smem_attr()
{
    using T = Traits<MODE, NMAX>;
    // the default cap on dynamic shared memory is 48 KB less the static use
    if (T::DYN > 0)
        return cudaFuncSetAttribute(nr_mixed_kernel<MODE, NMAX, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)T::DYN);
    return cudaSuccess;
}

template <int MODE, int NMAX, int KC>
cudaError_t launch_k(int grid, const KernelArgs &a, const QuadConst &qc, cudaStream_t st)
{
    using T = Traits<MODE, NMAX>;
    static bool attr_done = false; // per process: the attribute belongs to the function
    if (!attr_done) {
        cudaError_t e = set_smem_attr<MODE, NMAX, KC>();
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    nr_mixed_kernel<MODE, NMAX, KC><<<grid, T::BLOCK, T::DYN, st>>>(a, qc);
    return cudaGetLastError();
}

template <int MODE, int NMAX, int KC>
cudaError_t occupancy_k(int *blocks)
{
    using T = Traits<MODE, NMAX>;
    cudaError_t e = set_smem_attr<MODE, NMAX, KC>();
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, nr_mixed_kernel<MODE, NMAX, KC>, T::BLOCK,
                                                         T::DYN);
}

// The 1-layer kernels are also compiled for the workloads' quadrature orders
// (17 and 21 nodes), which turns the per-tile index arithmetic into constants.
template <int MODE, int NMAX>
cudaError_t launch_one(int grid, int K, const KernelArgs &a, const QuadConst &qc, cudaStream_t st)
{
    if constexpr (NMAX == 1) {
        if (K == 21) return launch_k<MODE, NMAX, 21>(grid, a, qc, st);
        if (K == 17) return launch_k<MODE, NMAX, 17>(grid, a, qc, st);
    }
    return launch_k<MODE, NMAX, 0>(grid, a, qc, st);
}

template <int MODE, int NMAX>
cudaError_t occupancy_one(int K, int *blocks)
{
    if constexpr (NMAX == 1) {
        if (K == 21) return occupancy_k<MODE, NMAX, 21>(blocks);
        if (K == 17) return occupancy_k<MODE, NMAX, 17>(blocks);
    }
    return occupancy_k<MODE, NMAX, 0>(blocks);
}

#define NR_GRAD_BUCKETS(X) X(1) X(2) X(4) X(8) X(12) X(16) X(20) X(32) X(64)

} // namespace

bool mixed_bucket_ok(int mode, int nmax)
{
    if (is_grad_mode(mode)) {
#define X(B) if (nmax == B) return true;
        NR_GRAD_BUCKETS(X)
#undef X
        return false;
    }
    return nmax == 0 || nmax == 1 || nmax == 64; // 64: runtime n, stacks deeper than 20 layers
}

int mixed_tile_q(int mode, int nmax, int K, bool allow_pair)
{
    if (allow_pair && pair_eligible(mode, nmax, K)) {
        const int slots = 2 * pair_block_threads(); // two evaluations per thread
        return std::min(slots / K, slots / kSubLanes);
    }
    const int block = mixed_block_threads(mode, nmax);
    return std::min(block / K, block / kSubLanes);
}

int mixed_block_threads(int mode, int nmax)
{
    if (!is_grad_mode(mode)) return nmax == 1 ? Traits<kModel, 1>::BLOCK : Traits<kModel, 0>::BLOCK;
#define X(B) if (nmax == B) return Traits<kGrad, B>::BLOCK;
    NR_GRAD_BUCKETS(X)
#undef X
    return 0;
}

size_t mixed_dyn_smem(int mode, int nmax)
{
    if (!is_grad_mode(mode)) return 0;
#define X(B) if (nmax == B) return Traits<kGrad, B>::DYN;
    NR_GRAD_BUCKETS(X)
#undef X
    return 0;
}

cudaError_t mixed_occupancy(int mode, int nmax, int K, int *blocks, bool allow_pair)
{
    if (allow_pair && pair_eligible(mode, nmax, K)) return pair_occupancy(mode, nmax, K, blocks);
    switch (mode) {
    case kModel:
        return nmax == 1 ? occupancy_one<kModel, 1>(K, blocks) : occupancy_one<kModel, 0>(K, blocks);
    case kLoglik:
        return nmax == 1 ? occupancy_one<kLoglik, 1>(K, blocks) : occupancy_one<kLoglik, 0>(K, blocks);
    case kGradRes:
#define X(B) if (nmax == B) return occupancy_one<kGradRes, B>(K, blocks);
        NR_GRAD_BUCKETS(X)
#undef X
        break;
    default:
#define X(B) if (nmax == B) return occupancy_one<kGrad, B>(K, blocks);
        NR_GRAD_BUCKETS(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_mixed(int mode, int nmax, int grid, const KernelArgs &a, const QuadConst &qc,
                         cudaStream_t st, bool allow_pair)
{
    const int K = qc.K;
    if (allow_pair && pair_eligible(mode, nmax, K)) return launch_pair(mode, nmax, grid, a, qc, st);
    switch (mode) {
    case kModel:
        return nmax == 1 ? launch_one<kModel, 1>(grid, K, a, qc, st) : launch_one<kModel, 0>(grid, K, a, qc, st);
    case kLoglik:
        return nmax == 1 ? launch_one<kLoglik, 1>(grid, K, a, qc, st)
                         : launch_one<kLoglik, 0>(grid, K, a, qc, st);
    case kGradRes:
#define X(B) if (nmax == B) return launch_one<kGradRes, B>(grid, K, a, qc, st);
        NR_GRAD_BUCKETS(X)
#undef X
        break;
    default:
#define X(B) if (nmax == B) return launch_one<kGrad, B>(grid, K, a, qc, st);
        NR_GRAD_BUCKETS(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

} // namespace nrimpl
