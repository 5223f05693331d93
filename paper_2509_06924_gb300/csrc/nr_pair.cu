// nr_pair.cu -- the kernels of the gradient buckets up to 20 layers and of
// both forward buckets (model, log-likelihood) with two evaluations per
// thread in paired FP32 arithmetic (sm_100-family add/mul/fma.rn.f32x2).
//
// The mixed-precision gradient evaluation is bound by instruction issue, not
// by the FP32 pipes: about 60 % of the issued instructions are FP32 adds,
// multiplies and FMAs, and the rest (selects, compares, special functions,
// shared-memory and shuffle traffic) keeps the FMA pipes half idle.  A
// paired instruction performs one FP32 operation for each of two independent
// evaluations at the cost of one issue slot.  So every thread here carries
// two (Q point, quadrature node) evaluations and the forward model, smearing
// seed and adjoint of both run as one stream of paired operations: the FP32
// work takes half the issue slots, as does the per-thread overhead (loop
// control, staged per-stack constants, edge tests of the tile).  Per-stack
// constants enter as a scalar replicated to both halves (free on the
// hardware), negated operands are free as well; nothing is swapped between
// the halves, which would cost moves.
//
// The forward modes run the same code up to the smearing sum (model: write
// scale S + bkg; log-likelihood: the residual terms) and no adjoint.
// Everything else follows the one-evaluation-per-thread kernel (nr_mixed.cu)
// step for step, with the same double-float guards, the same split between
// stored intermediates (1-2 layers keep all of them in registers) and
// rolled sweeps that recompute them (deeper stacks), and the same interior
// critical-edge treatment: evaluations whose k_j falls in the edge band are
// queued per warp and drained by the scalar edge adjoint, one entry per
// lane.  A thread carries two adjacent evaluation slots of its tile.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "nr_device.cuh"
#include "nr_internal.h"

// threads per CTA, and CTAs per SM asked of the compiler (register cap) for
// the 1- and the 2-layer kernels: the paired kernels are latency-bound at
// low occupancy, and the 2-layer kernel spills beyond 3 CTAs
#ifndef NR_PAIR_BLOCK
#define NR_PAIR_BLOCK 128
#endif
#ifndef NR_PAIR_MINB1
#define NR_PAIR_MINB1 5
#endif
#ifndef NR_PAIR_MINB2
#define NR_PAIR_MINB2 3
#endif
// CTAs per SM asked of the rolled (4-20 layer bucket) gradient kernels; their
// shared-memory partials and X_j usually set the occupancy first
#ifndef NR_PAIR_MINB_DEEP
#define NR_PAIR_MINB_DEEP 4
#endif
// gradient buckets [NR_PAIR_DEEP_FROM, 20] run the rolled paired kernel
// (NR_PAIR_DEEP_FROM 0: none).  The 32- and 64-layer buckets keep the
// one-evaluation kernel: two evaluations' X_j and partials per thread would
// leave room for one 128-thread CTA per SM at 32 layers, and none at 64.
#ifndef NR_PAIR_DEEP_FROM
#define NR_PAIR_DEEP_FROM 4
#endif
// 1: the runtime-n forward bucket (model / loglik of stacks with n != 1)
// runs the paired kernel too
#ifndef NR_PAIR_FWD_ANY
#define NR_PAIR_FWD_ANY 1
#endif
// CTAs per SM of the forward (model / loglik) kernels
#ifndef NR_PAIR_MINB_FWD
#define NR_PAIR_MINB_FWD 8
#endif
// 0: every bucket keeps the one-evaluation kernel
#ifndef NR_PAIR
#define NR_PAIR 1
#endif

namespace nrimpl {
namespace {

constexpr int kPairBlock = NR_PAIR_BLOCK;
#ifndef NR_PAIR_DEEP_UNROLL
#define NR_PAIR_DEEP_UNROLL 1
#endif
constexpr int kPairDeepUnroll = NR_PAIR_DEEP_UNROLL; // unroll of the rolled sweeps

// ---------------------------------------------------- paired FP32 values --
// f2 holds one FP32 value of each of the thread's two evaluations.
using f2 = float2;
struct b2 {
    bool x, y;
};

__device__ __forceinline__ f2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 pneg(f2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ f2 padd(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 psub(f2 a, f2 b) { return __fadd2_rn(a, pneg(b)); }
__device__ __forceinline__ f2 pmul(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 pfma(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 pabs(f2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ f2 pmax(f2 a, f2 b) { return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }
__device__ __forceinline__ f2 psel(b2 c, f2 a, f2 b) { return make_float2(c.x ? a.x : b.x, c.y ? a.y : b.y); }
__device__ __forceinline__ f2 prcp(f2 a) { return make_float2(rcp_approx(a.x), rcp_approx(a.y)); }
__device__ __forceinline__ f2 prsqrt(f2 a) { return make_float2(rsqrt_approx(a.x), rsqrt_approx(a.y)); }
__device__ __forceinline__ f2 pex2(f2 a) { return make_float2(ex2_approx(a.x), ex2_approx(a.y)); }
__device__ __forceinline__ void psincos(f2 a, f2 &s, f2 &c)
{
    sincos_approx(a.x, s.x, c.x);
    sincos_approx(a.y, s.y, c.y);
}
__device__ __forceinline__ float half(f2 a, int h) { return h ? a.y : a.x; }
// cis_tab (nr_device.cuh) on both halves: (cos, sin) as a complex pair
__device__ __forceinline__ void pcis_tab(f2 ph, f2 pl, const float *tab, f2 &cs, f2 &sn)
{
    const f2 t = pfma(ph, bc(kTabScale), bc(kRoundMagic));
    const f2 nt = padd(t, bc(-kRoundMagic));
    const int i0 = __float_as_int(t.x) & (kTabN - 1), i1 = __float_as_int(t.y) & (kTabN - 1);
    const f2 tc = make_float2(tab[i0], tab[i1]), ts = make_float2(tab[kTabN + i0], tab[kTabN + i1]);
    f2 x = pfma(pneg(nt), bc(kTabStepHi), ph);
    x = pfma(pneg(nt), bc(kTabStepLo), x);
    x = padd(x, pl);
    const f2 z = pmul(x, x);
    const f2 sx = pfma(pmul(x, z), bc(-1.f / 6.f), x);
    const f2 cx = pfma(z, bc(-kTabCosC), bc(1.f));
    cs = pfma(tc, cx, pneg(pmul(ts, sx)));
    sn = pfma(ts, cx, pmul(tc, sx));
}

// error-free transformations on both halves (every paired add rounds once)
__device__ __forceinline__ void two_sum2(f2 a, f2 b, f2 &s, f2 &e)
{
    s = padd(a, b);
    const f2 bb = psub(s, a);
    e = padd(psub(a, psub(s, bb)), psub(b, bb));
}
__device__ __forceinline__ void fast_two_sum2(f2 a, f2 b, f2 &s, f2 &e)
{
    s = padd(a, b);
    e = psub(b, psub(s, a));
}

// complex numbers of both evaluations
struct c2 {
    f2 re, im;
};
__device__ __forceinline__ c2 czero() { return c2{bc(0.f), bc(0.f)}; }
__device__ __forceinline__ c2 cadd2(c2 a, c2 b) { return c2{padd(a.re, b.re), padd(a.im, b.im)}; }
__device__ __forceinline__ c2 cmul2(c2 a, c2 b)
{
    return c2{pfma(a.re, b.re, pneg(pmul(a.im, b.im))), pfma(a.re, b.im, pmul(a.im, b.re))};
}
// conj(a) * b
__device__ __forceinline__ c2 cmulc2(c2 a, c2 b)
{
    return c2{pfma(a.re, b.re, pmul(a.im, b.im)), pfma(a.re, b.im, pneg(pmul(a.im, b.re)))};
}
__device__ __forceinline__ c2 csqr2(c2 a)
{
    return c2{pmul(psub(a.re, a.im), padd(a.re, a.im)), pmul(padd(a.re, a.re), a.im)};
}
// 1 - a^2
__device__ __forceinline__ c2 one_minus_sq2(c2 a)
{
    return c2{pfma(pneg(a.re), a.re, pfma(a.im, a.im, bc(1.f))), pmul(bc(-2.f), pmul(a.re, a.im))};
}
// conj(a) * b + c
__device__ __forceinline__ c2 cfmac2(c2 a, c2 b, c2 c)
{
    return c2{pfma(a.re, b.re, pfma(a.im, b.im, c.re)), pfma(a.re, b.im, pfma(pneg(a.im), b.re, c.im))};
}

// wavevector of both evaluations (value + low word of Re k, as Kz)
struct Kz2 {
    f2 re, im, lo;
};
__device__ __forceinline__ c2 kc2(const Kz2 &k) { return c2{k.re, k.im}; }

// principal sqrt of u + i a (u = uh + ul, a >= 0 the stack's 4 pi iota,
// a2 = a^2), as kz_sqrt
template <bool REFINE>
__device__ __forceinline__ Kz2 kz_sqrt2(f2 uh, f2 ul, float a, float a2)
{
    const f2 au = pabs(uh);
    const f2 m2 = pfma(uh, uh, bc(a2));
    const f2 m = pmul(m2, prsqrt(pmax(m2, bc(1e-37f))));
    const f2 H = padd(au, m);                             // |u| + |z| = 2 t^2
    const f2 i2t = prsqrt(pmax(padd(H, H), bc(4e-30f))); // 1 / (2 t)
    const f2 t = pmul(H, i2t);
    const f2 small = pmul(bc(a), i2t);
    const b2 prop{uh.x >= 0.f, uh.y >= 0.f};
    Kz2 k;
    if constexpr (REFINE) {
        const f2 e = padd(pfma(pneg(t), t, au), pfma(small, small, psel(prop, ul, pneg(ul))));
        const f2 corr = pmul(e, i2t);
        k.re = psel(prop, t, small);
        k.im = psel(prop, small, padd(t, corr));
        k.lo = psel(prop, corr, bc(0.f));
    } else {
        k.re = psel(prop, t, small);
        k.im = psel(prop, small, t);
        k.lo = bc(0.f);
    }
    return k;
}

// k of medium j >= 1 from k_0^2 = (p_hi + p_lo) and the staged medium entry
template <bool REFINE>
__device__ __forceinline__ Kz2 medium_kz2(f2 p_hi, f2 p_lo, float4 m)
{
    if constexpr (REFINE) {
        f2 uh, ul;
        two_sum2(p_hi, bc(-m.x), uh, ul);
        ul = padd(ul, padd(p_lo, bc(-m.y)));
        fast_two_sum2(uh, ul, uh, ul);
        return kz_sqrt2<true>(uh, ul, m.z, m.w);
    } else {
        const f2 u = padd(padd(p_hi, bc(-m.x)), padd(p_lo, bc(-m.y)));
        return kz_sqrt2<false>(u, bc(0.f), m.z, m.w);
    }
}

// E = exp(2 i k d), phase in double-float (as layer_phase).  TAB: the table
// sin / cos (NR_SINCOS_TABLE), else the special-function unit's.
template <bool TAB>
__device__ __forceinline__ c2 layer_phase2(const Kz2 &k, float4 L, const float *tab)
{
    const f2 ph = pmul(k.re, bc(L.x));
    f2 pl = pfma(k.re, bc(L.x), pneg(ph));
    pl = pfma(k.re, bc(L.y), pl);
    pl = pfma(k.lo, bc(L.x), pl);
    const f2 amp = pex2(pmul(k.im, bc(L.z)));
    f2 s, c;
    if constexpr (TAB && NR_SINCOS_TABLE) {
        pcis_tab(ph, pl, tab, c, s);
    } else {
        const f2 nt = padd(pfma(ph, bc(kInv2Pi), bc(kRoundMagic)), bc(-kRoundMagic));
        f2 red = pfma(pneg(nt), bc(kTwoPiHi), ph);
        red = pfma(pneg(nt), bc(kTwoPiLo), red);
        red = padd(red, pl);
        psincos(red, s, c);
    }
    return c2{pmul(amp, c), pmul(amp, s)};
}

// r_j with Nevot-Croce roughness, G = exp(s k_a k_b) / S^2 and kk = k_a k_b
// (as fresnel_nc).  A vanishing S (k_a = k_b = 0) gives G = r = 0.
template <bool REAL_A, bool TAB>
__device__ __forceinline__ c2 fresnel_nc2(c2 ka, c2 kb, float4 I, c2 &G, c2 &kk, const float *tab)
{
    const f2 Sx = padd(ka.re, kb.re);
    const f2 Sy = REAL_A ? kb.im : padd(ka.im, kb.im);
    const f2 n2 = pfma(Sx, Sx, pmul(Sy, Sy));
    const f2 inv = prcp(pmax(n2, bc(1e-30f)));
    const c2 iS2 = csqr2(c2{pmul(Sx, inv), pneg(pmul(Sy, inv))});
    kk = REAL_A ? c2{pmul(ka.re, kb.re), pmul(ka.re, kb.im)} : cmul2(ka, kb);
    const f2 amp = pex2(pmul(bc(I.w), kk.re));
    f2 sn, cs;
    if constexpr (TAB && NR_NC_TABLE) pcis_tab(pmul(bc(I.z), kk.im), bc(0.f), tab, cs, sn);
    else psincos(pmul(bc(I.z), kk.im), sn, cs);
    G = cmul2(c2{pmul(amp, cs), pmul(amp, sn)}, iS2);
    return cmul2(c2{bc(I.x), bc(I.y)}, G);
}

// X = (r + Y) / (1 + r Y); D = 1 / (1 + r Y)
__device__ __forceinline__ c2 mobius2(c2 r, c2 Y, c2 &D)
{
    const c2 rY = cmul2(r, Y);
    const f2 dx = padd(bc(1.f), rY.re), dy = rY.im;
    const f2 inv = prcp(pfma(dx, dx, pmul(dy, dy)));
    D = c2{pmul(dx, inv), pneg(pmul(dy, inv))};
    return cmul2(cadd2(r, Y), D);
}

// Drains `cnt` queued interior-edge entries of one warp (one per lane) into
// the lane-pair partials of the rolled kernels (acc points at this lane
// pair's slot of medium 1's Re partial; stride between partials `stride`,
// Re -> Im distance `im_off`).  Lanes 2i and 2i+1 share a slot: the even
// lanes add first, then the odd ones, so the order of the additions is
// fixed.  Called by whole warps; kept out of line (rare path).
template <int EQ, bool RES>
__device__ __noinline__ float eq_drain_lanepair(float2 (*q)[EQ], const int *qj, const float4 *med, const float4 *lay,
                                                int n, int lane, int cnt, float *acc, int stride, int im_off)
{
    float res = 0.f; // the resolution-mode term of the entry (factor in q[3])
    const bool on = lane < cnt;
    int j = 1;
    float2 ub = make_float2(0.f, 0.f);
    if (on) {
        j = qj[lane];
        ub = edge_entry_ubar(q[0][lane], q[1][lane], q[2][lane], j, n, med, lay);
        if constexpr (RES) res = 2.f * ub.x * q[3][lane].x;
    }
    for (int parity = 0; parity < 2; ++parity) {
        if (on && (lane & 1) == parity) {
            // conj(kbar)/k_j = 2 conj(ubar)
            acc[(j - 1) * stride] += 2.f * ub.x;
            acc[(j - 1) * stride + im_off] += -2.f * ub.y;
        }
        __syncwarp();
    }
    return res;
}

// ---------------------------------------------------------------- traits --
// STORE (1-2 layer gradients): unrolled sweeps, every forward intermediate
// and the partial gradients in registers.  ROLL (the 4-20 layer buckets,
// i.e. 3-20 layers): rolled sweeps
// peeled at the first and last steps; X_j (both halves) and the partial
// gradients in shared memory, the latter one float per lane pair (both
// halves of lanes 2i and 2i+1 summed: half the storage, which lets the
// 12-layer bucket run 4 CTAs per SM); k, r and E recomputed in the adjoint;
// edge entries keep the node k_0.
template <int MODE, int NMAX>
struct PairTraits {
    static constexpr bool GRAD = MODE == kGrad || MODE == kGradRes;
    static constexpr bool ROLL = GRAD && NMAX > 2;
    // rolled forward sweep: the rolled gradient kernels and the runtime-n
    // forward kernel (NMAX = 0, any layer count)
    static constexpr bool RFWD = ROLL || NMAX == 0;
    static constexpr int NACC = 4 * NMAX + 3;
    static constexpr int MINB = !GRAD ? NR_PAIR_MINB_FWD : NMAX == 1 ? NR_PAIR_MINB1
                                : NMAX == 2 ? NR_PAIR_MINB2 : NR_PAIR_MINB_DEEP;
    // ROLL: partials per lane pair (kPairBlock / 2 floats per index), then X_j
    static constexpr size_t DYN = ROLL ? (size_t)NACC * (kPairBlock / 2) * 4 + (size_t)(NMAX + 1) * kPairBlock * 16
                                       : 0;
};

// ---------------------------------------------------------------- kernel --
template <int MODE, int NMAX, int KC>
__global__ void __launch_bounds__(kPairBlock, PairTraits<MODE, NMAX>::MINB)
nr_pair_kernel(const KernelArgs ka, const QuadConst qc)
{
    using PT = PairTraits<MODE, NMAX>;
    constexpr bool GRAD = PT::GRAD;
    constexpr bool ROLL = PT::ROLL;
    constexpr bool LIK = MODE != kModel;
    // sin / cos by table for the model and the gradient; the log-likelihood
    // alone keeps the special-function unit's (its sum over Q points
    // averages their error: within 5e-6 of the oracle on every workload)
    constexpr bool TAB = MODE != kLoglik;
    static_assert(GRAD ? (NMAX >= 1 && NMAX <= NR_MAX_LAYERS) : (NMAX == 1 || NMAX == 0),
                  "paired kernel: gradient buckets, 1-layer and runtime-n forward");
    constexpr int NM = NMAX > 0 ? NMAX : NR_MAX_LAYERS; // shared-memory capacity in layers
    constexpr int BLOCK = kPairBlock;
    constexpr int WARPS = BLOCK / 32;
    constexpr bool RES = MODE == kGradRes;
    constexpr int NACC = PT::NACC;
    constexpr int NRAW = 4 * NM + 7;
    constexpr int CAPQ = ROLL ? 96 : 256;
    // a warp's STORE tile queues at most 64 n interior-edge entries and keeps
    // fewer than 32 between tiles; the rolled sweeps drain at 32 after each
    // half's entries of a step
    constexpr int EQ = ROLL ? 64 : 64 * NM + 32;
    // STORE: k_{j-1}, k_j, k_{j+1}, Z, Xbar_{j-1}; ROLL: node k_0, Z,
    // Xbar_{j-1}; (+ k_0 dk_0/d ln f)
    constexpr int EQF = (ROLL ? 3 : 5) + (RES ? 1 : 0);
    static_assert(CAPQ >= 2 * BLOCK / kSubLanes, "a super-tile holds at least one tile");

    __shared__ StackSmem<NM> sm;
    __shared__ float sh_cs[2 * kTabN]; // cos, sin at multiples of 2 pi / kTabN
    // w_k R per (Q slot, node), double-buffered.  TQ KP <= 4 BLOCK for any K >= 3;
    // the rolled kernels, short of shared memory, take the exact maximum
    // over K >= 3 (408 at K = 5: 51 Q points x 8)
    constexpr int WRN = ROLL ? 416 : 4 * BLOCK;
    __shared__ __align__(16) float sh_wR[2][WRN];
    __shared__ float4 sh_qd[CAPQ];                      // (Q/2, dQ/2, R_obs, 1/err) per staged Q point
    __shared__ float2 sh_rs[LIK ? CAPQ : 1];            // (residual, S) per staged Q point
    __shared__ double sh_red[WARPS][32];
    __shared__ double sh_redd[WARPS][4];
    __shared__ double sh_raw[NRAW];
    __shared__ int sh_item;
    __shared__ int sh_last;
    __shared__ float2 sh_eq[GRAD ? WARPS : 1][EQF][GRAD ? EQ : 1];
    __shared__ int sh_eqj[GRAD ? WARPS : 1][GRAD ? EQ : 1];
    // ROLL: [NACC][BLOCK/2] partial gradients (one float per lane pair), then
    // [NM+1][BLOCK] X_j pairs
    constexpr int HALF = BLOCK / 2;
    extern __shared__ __align__(16) float sh_dyn[];
    float *sh_acc = sh_dyn;
    float4 *sh_X = reinterpret_cast<float4 *>(sh_dyn + (ROLL ? NACC * HALF : 0));

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int K = KC > 0 ? KC : qc.K; // K >= 3 (the host's choice of this kernel)
    const int KP = (K + 3) & ~3;      // node stride of a Q slot in sh_wR (whole float4s)
    const int TQ = ka.tile_q;
    // Warp-local tiles: when every warp's 64 evaluation slots hold whole Q
    // points and the CTA tile is exactly those (TQ = warps x floor(64/K), no
    // slot lost against the CTA-wide layout, e.g. K = 21: 4 x 3 Q points),
    // each warp owns its Q slots and the smearing exchange needs only a warp
    // barrier.  Otherwise the thread carries tile slots 2 tid + h and the
    // exchange takes a CTA barrier.
    const int tqw = 64 / K;
    const bool wloc = TQ == WARPS * tqw;
    int qslot[2], kn[2];
    bool lane_on[2];
    f2 g_hi, g_lo, wk;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int e = wloc ? 2 * lane + h : 2 * tid + h;
        const int ls = e / K;
        kn[h] = e - ls * K;
        qslot[h] = wloc ? warp * tqw + ls : ls;
        lane_on[h] = wloc ? ls < tqw : ls < TQ;
        const float gh = lane_on[h] ? qc.g_hi[kn[h]] : 0.f;
        const float gl = lane_on[h] ? qc.g_lo[kn[h]] : 0.f;
        const float w = lane_on[h] ? qc.w[kn[h]] : 0.f;
        if (h == 0) { g_hi.x = gh; g_lo.x = gl; wk.x = w; }
        else { g_hi.y = gh; g_lo.y = gl; wk.y = w; }
    }
    // smearing sums: the warp's 64 evaluations touch Q slots qs0.. (at most
    // nslots of them; exactly tqw with warp-local tiles, and only those are
    // summed); sgl lanes per slot (depends on K only)
    const int qs0 = wloc ? warp * tqw : (warp * 64) / K;
    const int qs_end = wloc ? qs0 + tqw : TQ;
    const int nslots = (63 + K - 1) / K + 1;
    const int sgl = nslots <= 1 ? 32 : nslots <= 2 ? 16 : nslots <= 4 ? 8 : nslots <= 8 ? 4 : nslots <= 16 ? 2 : 1;
    const float g_max = fmaxf(fabsf(qc.g_hi[0]), fabsf(qc.g_hi[K - 1]));

    for (int i = tid; i < 2 * WRN; i += BLOCK) (&sh_wR[0][0])[i] = 0.f; // padding stays 0
    for (int i = tid; i < 2 * kTabN; i += BLOCK) sh_cs[i] = qc.cs_tab[i];  // read after the item barrier

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
        const int n = (NMAX == 1 && NR_EXACT1) ? 1 : si.n;
        const double *p = ka.params + si.par_off;
        stage_stack<NM>(sm, p, n, tid, ka.status);

        f2 accr[ROLL ? 1 : NACC];
        if constexpr (ROLL) {
            for (int i = tid; i < NACC * HALF; i += BLOCK) sh_acc[i] = 0.f;
        } else {
#pragma unroll
            for (int i = 0; i < NACC; ++i) accr[i] = bc(0.f);
        }
        constexpr int oD = 0, oUr = NM, oUi = 2 * NM + 1, oS = 3 * NM + 2;
        // ROLL: the lane pair's partial idx += t (t: this lane's both halves);
        // called by whole warps
        auto acc_lanepair = [&](int idx, float t) __attribute__((always_inline)) {
            t += __shfl_xor_sync(kFull, t, 1);
            if (!(lane & 1)) sh_acc[idx * HALF + (tid >> 1)] += t;
        };
        // partial gradient idx += v (both halves)
        auto acc_add = [&](int idx, f2 v) __attribute__((always_inline)) {
            if constexpr (ROLL) acc_lanepair(idx, v.x + v.y);
            else accr[idx] = padd(accr[idx], v);
        };
        // partial gradient idx += a b + c d
        auto acc_fma2 = [&](int idx, f2 a, f2 b, f2 c, f2 d) __attribute__((always_inline)) {
            if constexpr (ROLL) {
                const f2 t = pfma(a, b, pmul(c, d));
                acc_lanepair(idx, t.x + t.y);
            } else {
                accr[idx] = pfma(a, b, pfma(c, d, accr[idx]));
            }
        };
        f2 gres_acc = bc(0.f);
        int eq_cnt = 0; // entries in this warp's interior-edge queue (warp-uniform)
        // drain `cnt` <= 32 queued entries, one per lane (scalar edge adjoint)
        auto eq_drain = [&](int cnt) {
            if constexpr (ROLL) {
                const float r = eq_drain_lanepair<EQ, RES>(sh_eq[warp], sh_eqj[warp], sm.med, sm.lay, n, lane, cnt,
                                                           sh_acc + oUr * HALF + (tid >> 1), HALF,
                                                           (oUi - oUr) * HALF);
                if constexpr (RES) gres_acc.x += r;
            } else if (lane < cnt) {
                const int j = sh_eqj[warp][lane];
                const float2 ub = edge_ubar(sh_eq[warp][0][lane], sh_eq[warp][1][lane], sh_eq[warp][2][lane],
                                            sm.lay[j - 1].w, sm.lay[j].w, 0.5f * sm.lay[j].x, sh_eq[warp][3][lane],
                                            j == n, sh_eq[warp][4][lane]);
                // conj(kbar)/k_j = 2 conj(ubar)
#pragma unroll
                for (int t = 1; t <= NM; ++t)
                    if (t == j) {
                        accr[oUr + t - 1].x += 2.f * ub.x;
                        accr[oUi + t - 1].x += -2.f * ub.y;
                    }
                if constexpr (RES) gres_acc.x = fmaf(2.f * ub.x, sh_eq[warp][EQF - 1][lane].x, gres_acc.x);
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

        // per-thread sums of the loglik terms, d/dscale, d/dbkg (per Q point)
        float ll_hi = 0.f, ll_lo = 0.f, gsc_acc = 0.f, gbk_acc = 0.f;
        const float *qp = ka.q + si.q_begin, *dqp = ka.dq + si.q_begin;
        const float fsc = ka.dq_scale ? (float)ka.dq_scale[wi.stack] : 1.f; // resolution scale of the stack
        const float *rop = ka.r_obs + si.q_begin, *rep = ka.r_err + si.q_begin;
        const int span = (CAPQ / TQ) * TQ;
        int sb = wi.q_lo, s_next = wi.q_lo, s_cnt = 0;
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
                float4 v = make_float4(0.05f, 0.f, 0.f, 0.f); // past the end: a harmless node, 1/err = 0
                if (qa < wi.q_hi) {
                    v.x = 0.5f * __ldg(qp + qa);
                    v.y = 0.5f * fsc * __ldg(dqp + qa);
                    if constexpr (LIK) {
                        v.z = __ldg(rop + qa);
                        v.w = rcp_approx(__ldg(rep + qa));
                    }
                    if constexpr (GRAD) {
                        // may a node of this Q point reach an interior-edge
                        // band?  (negative 1/err: yes)
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
        const f2 wks = pmul(wk, bc(scale));
        int buf = 0;
        for (int q0 = wi.q_lo; q0 < wi.q_hi; q0 += TQ, buf ^= 1) {
            if (q0 == s_next) restage(q0);
            int qi[2], si_q[2];
            bool act[2];
            float4 qd[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                qi[h] = q0 + qslot[h];
                si_q[h] = q0 - sb + (lane_on[h] ? qslot[h] : 0);
                act[h] = lane_on[h] && qi[h] < wi.q_hi;
                qd[h] = sh_qd[si_q[h]];
            }
            const f2 Qh = make_float2(qd[0].x, qd[1].x), dQh = make_float2(qd[0].y, qd[1].y);
            // a1: node position k_0 = q/2 in double-float, k_0^2
            f2 k0h, k0l;
            {
                const f2 th = pmul(dQh, g_hi);
                f2 tl = pfma(dQh, g_hi, pneg(th));
                tl = pfma(dQh, g_lo, tl);
                f2 s, e;
                two_sum2(Qh, th, s, e);
                e = padd(e, tl);
                fast_two_sum2(s, e, k0h, k0l);
            }
            const b2 qok{k0h.x > 0.f, k0h.y > 0.f};
            if ((act[0] && !qok.x) || (act[1] && !qok.y)) atomicOr(ka.status, NR_FLAG_BAD_Q);
            const f2 p_hi = pmul(k0h, k0h);
            f2 p_lo = pfma(k0h, k0h, pneg(p_hi));
            p_lo = pfma(padd(k0h, k0h), k0l, p_lo);

            // a3-a6 forward from the backing up (STORE keeps every
            // intermediate; ROLL keeps X_j in shared memory)
            Kz2 kst[ROLL ? 1 : NM + 2];
            c2 rst[ROLL ? 1 : NM + 1], Gst[ROLL ? 1 : NM + 1], Est[ROLL ? 1 : NM + 2], Dst[ROLL ? 1 : NM + 1],
                Yst[ROLL ? 1 : NM + 1];
            Kz2 kbelow = medium_kz2<false>(p_hi, p_lo, sm.med[n + 1]);
            c2 Xbelow = czero();
            auto fwd_step = [&](int j, auto TOP, auto BOT) __attribute__((always_inline)) {
                const bool top = pos_flag(TOP, j == 0), bot = pos_flag(BOT, j == n);
                Kz2 kj;
                if (top) kj = Kz2{k0h, bc(0.f), k0l};
                else kj = medium_kz2<true>(p_hi, p_lo, sm.med[j]);
                c2 Gj, kkj;
                const float4 Ij = sm.itf[j];
                const c2 rj = top ? fresnel_nc2<true, TAB>(kc2(kj), kc2(kbelow), Ij, Gj, kkj, sh_cs)
                                  : fresnel_nc2<false, TAB>(kc2(kj), kc2(kbelow), Ij, Gj, kkj, sh_cs);
                c2 Xj;
                if (bot) {
                    Xj = rj;
                    if constexpr (!ROLL) kst[j + 1] = kbelow;
                } else {
                    const c2 Ej = layer_phase2<TAB>(kbelow, sm.lay[j + 1], sh_cs);
                    const c2 Yj = cmul2(Xbelow, Ej);
                    c2 Dj;
                    Xj = mobius2(rj, Yj, Dj);
                    if constexpr (!ROLL) {
                        Est[j + 1] = Ej;
                        Dst[j] = Dj;
                        Yst[j] = Yj;
                    }
                }
                if constexpr (ROLL) {
                    sh_X[j * BLOCK + tid] = make_float4(Xj.re.x, Xj.re.y, Xj.im.x, Xj.im.y);
                } else {
                    kst[j] = kj;
                    rst[j] = rj;
                    Gst[j] = Gj;
                }
                Xbelow = Xj;
                kbelow = kj;
            };
            if constexpr (PT::RFWD) {
                fwd_step(n, Pos<kRt>{}, Pos<kYes>{});
#pragma unroll kPairDeepUnroll
                for (int j = n - 1; j >= 1; --j) fwd_step(j, Pos<kNo>{}, Pos<kNo>{});
                if (n >= 1) fwd_step(0, Pos<kYes>{}, Pos<kNo>{});
            } else {
#pragma unroll
                for (int j = NM; j >= 0; --j)
                    if (j <= n) fwd_step(j, Pos<kRt>{}, Pos<kRt>{});
            }
            f2 R = pfma(Xbelow.re, Xbelow.re, pmul(Xbelow.im, Xbelow.im));
            if (!qok.x) R.x = __int_as_float(0x7fffffff);
            if (!qok.y) R.y = __int_as_float(0x7fffffff);

            // a8-a10: smearing sum, model, residual, adjoint seed
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (lane_on[h]) sh_wR[buf][qslot[h] * KP + kn[h]] = half(wk, h) * half(R, h);
            if (wloc) __syncwarp();
            else __syncthreads();
            f2 S;
            {
                const int g = lane / sgl, part = lane - g * sgl;
                const int slot = qs0 + g;
                float ps = 0.f;
                if (slot < qs_end) {
                    const float4 *row = reinterpret_cast<const float4 *>(&sh_wR[buf][slot * KP]);
                    auto add4 = [&](int c) __attribute__((always_inline)) {
                        const float4 v = row[c];
                        ps += (v.x + v.y) + (v.z + v.w);
                    };
                    if constexpr (KC > 0) {
                        constexpr int NSL = (63 + KC - 1) / KC + 1;
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
                S.x = __shfl_sync(kFull, ps, ((qslot[0] - qs0) * sgl) & 31);
                S.y = __shfl_sync(kFull, ps, ((qslot[1] - qs0) * sgl) & 31);
            }
            if constexpr (MODE == kModel) {
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    if (act[h] && kn[h] == 0) ka.r_out[si.out_off + qi[h]] = fmaf(scale, half(S, h), bkg);
            } else {
                const f2 ie = make_float2(fabsf(qd[0].w), fabsf(qd[1].w));
                const f2 res = pmul(psub(pfma(bc(scale), S, bc(bkg)), make_float2(qd[0].z, qd[1].z)), ie);
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    if (act[h] && kn[h] == 0) sh_rs[si_q[h]] = make_float2(half(res, h), half(S, h));
                if constexpr (GRAD) {
                    const f2 Rb = pmul(wks, pneg(pmul(res, ie))); // w_k scale dl/dm (0 on idle slots)

                    // a7: adjoint sweep from the fronting down to the backing
                    c2 Xb = c2{pmul(Xbelow.re, padd(Rb, Rb)), pmul(Xbelow.im, padd(Rb, Rb))}; // X_0
                    c2 kbar = czero();
                    Kz2 kj = Kz2{k0h, bc(0.f), k0l};
                    c2 Xb_up = czero();
                    Kz2 kjm1 = kj;
                    const f2 edge_u = pmul(bc(kEdgeFrac), pmul(k0h, k0h));
                    const f2 wres = RES ? pmul(dQh, g_hi) : bc(0.f);
                    f2 res_sum = bc(0.f), res_k0 = bc(0.f);
                    auto adj_step = [&](int j, auto TOP, auto BOT, auto EDG) __attribute__((always_inline)) {
                        const bool top = pos_flag(TOP, j == 0), bot = pos_flag(BOT, j == n);
                        const float4 Ij = sm.itf[j];
                        const float4 Lj1 = sm.lay[j + 1];
                        const c2 Xb_in = Xb;
                        c2 Zj = czero();
                        Kz2 kj1;
                        c2 rj, Gj, kkj;
                        if constexpr (ROLL) {
                            const float4 Mj1 = sm.med[j + 1];
                            kj1 = bot ? medium_kz2<false>(p_hi, p_lo, Mj1) : medium_kz2<true>(p_hi, p_lo, Mj1);
                            rj = top ? fresnel_nc2<true, TAB>(kc2(kj), kc2(kj1), Ij, Gj, kkj, sh_cs)
                                     : fresnel_nc2<false, TAB>(kc2(kj), kc2(kj1), Ij, Gj, kkj, sh_cs);
                        } else {
                            kj1 = kst[j + 1];
                            rj = rst[j];
                            Gj = Gst[j];
                            kkj = top ? c2{pmul(kj.re, kj1.re), pmul(kj.re, kj1.im)} : cmul2(kc2(kj), kc2(kj1));
                        }
                        c2 kbar1 = czero();
                        c2 rb;
                        if (!bot) {
                            c2 Ej1, Dj, Y;
                            if constexpr (ROLL) {
                                const float4 x1 = sh_X[(j + 1) * BLOCK + tid];
                                Ej1 = layer_phase2<TAB>(kj1, Lj1, sh_cs);
                                Y = cmul2(c2{make_float2(x1.x, x1.y), make_float2(x1.z, x1.w)}, Ej1);
                                const c2 rY = cmul2(rj, Y);
                                const f2 dx = padd(bc(1.f), rY.re), dy = rY.im;
                                const f2 inv = prcp(pfma(dx, dx, pmul(dy, dy)));
                                Dj = c2{pmul(dx, inv), pneg(pmul(dy, inv))};
                            } else {
                                Ej1 = Est[j + 1];
                                Dj = Dst[j];
                                Y = Yst[j];
                            }
                            Zj = Y;
                            const c2 V = cmulc2(Dj, cmulc2(Dj, Xb));
                            rb = cmulc2(one_minus_sq2(Y), V);
                            const c2 Yb = cmulc2(one_minus_sq2(rj), V);
                            Xb = cmulc2(Ej1, Yb);
                            const c2 U = cmulc2(Y, Yb);
                            acc_fma2(oD + j, kj1.re, U.im, pneg(kj1.im), U.re);
                            kbar1 = c2{pmul(bc(Lj1.x), U.im), pneg(pmul(bc(Lj1.x), U.re))};
                        } else {
                            rb = Xb;
                        }
                        const c2 rr = cmulc2(rb, rj);
                        const c2 gg = cmulc2(Gj, rb);
                        const c2 sr = c2{pmul(bc(Ij.z), rr.re), pneg(pmul(bc(Ij.z), rr.im))};
                        const c2 Hm = c2{pfma(bc(-2.f), gg.re, sr.re), pfma(bc(-2.f), gg.im, sr.im)}; // conj(M) rbar
                        if (top) kbar1 = c2{pfma(kj.re, Hm.re, kbar1.re), pfma(kj.re, Hm.im, kbar1.im)};
                        else kbar1 = cfmac2(kc2(kj), Hm, kbar1);
                        acc_fma2(oS + j, rr.re, kkj.re, pneg(rr.im), kkj.im);
                        const c2 Hp = c2{pfma(bc(2.f), gg.re, sr.re), pfma(bc(2.f), gg.im, sr.im)}; // conj(P) rbar
                        if (RES && top) res_k0 = pfma(kj1.re, Hp.re, pmul(kj1.im, Hp.im));
                        if (!top) {
                            kbar = cfmac2(kc2(kj1), Hp, kbar);
                            // k_j complete: accumulate conj(kbar) / k_j, or queue the
                            // interior-edge evaluation
                            const f2 m2 = pfma(kj.re, kj.re, pmul(kj.im, kj.im));
                            b2 edge{false, false};
                            if constexpr (decltype(EDG)::value) {
                                edge = b2{act[0] && m2.x < edge_u.x, act[1] && m2.y < edge_u.y};
#pragma unroll
                                for (int h = 0; h < 2; ++h) {
                                    const bool eh = h ? edge.y : edge.x;
                                    const unsigned em = __ballot_sync(kFull, eh);
                                    if (em) {
                                        if (eh) {
                                            const int slot =
                                                queue_slot<EQ>(eq_cnt + __popc(em & ((1u << lane) - 1u)), ka.status);
                                            if constexpr (RES)
                                                sh_eq[warp][EQF - 1][slot] = make_float2(half(k0h, h) * half(wres, h), 0.f);
                                            if constexpr (ROLL) {
                                                sh_eq[warp][0][slot] = make_float2(half(k0h, h), half(k0l, h));
                                                sh_eq[warp][1][slot] = make_float2(half(Zj.re, h), half(Zj.im, h));
                                                sh_eq[warp][2][slot] = make_float2(half(Xb_up.re, h), half(Xb_up.im, h));
                                            } else {
                                                sh_eq[warp][0][slot] = make_float2(half(kjm1.re, h), half(kjm1.im, h));
                                                sh_eq[warp][1][slot] = make_float2(half(kj.re, h), half(kj.im, h));
                                                sh_eq[warp][2][slot] = make_float2(half(kj1.re, h), half(kj1.im, h));
                                                sh_eq[warp][3][slot] = make_float2(half(Zj.re, h), half(Zj.im, h));
                                                sh_eq[warp][4][slot] = make_float2(half(Xb_up.re, h), half(Xb_up.im, h));
                                            }
                                            sh_eqj[warp][slot] = j;
                                        }
                                        eq_cnt = queue_count<EQ>(eq_cnt + __popc(em));
                                        if constexpr (ROLL) {
                                            if (eq_cnt >= 32) {
                                                __syncwarp();
                                                eq_drain(32);
                                            }
                                        }
                                    }
                                }
                            }
                            const c2 kq = cmul2(kbar, kc2(kj));
                            f2 inv = prcp(pmax(m2, bc(1e-30f)));
                            if constexpr (decltype(EDG)::value) inv = psel(edge, bc(0.f), inv);
                            const f2 ur = pmul(kq.re, inv), ui = pneg(pmul(kq.im, inv));
                            acc_add(oUr + j - 1, ur);
                            acc_add(oUi + j - 1, ui);
                            if constexpr (RES) res_sum = padd(res_sum, ur);
                        }
                        Xb_up = Xb_in;
                        kbar = kbar1;
                        kjm1 = kj;
                        kj = kj1;
                        if (bot) { // backing medium n+1
                            const c2 kk = cmul2(kbar, kc2(kj));
                            const f2 m2 = pfma(kj.re, kj.re, pmul(kj.im, kj.im));
                            const f2 inv = prcp(pmax(m2, bc(1e-30f)));
                            const f2 ur = pmul(kk.re, inv), ui = pneg(pmul(kk.im, inv));
                            acc_add(oUr + j, ur);
                            acc_add(oUi + j, ui);
                            if constexpr (RES) res_sum = padd(res_sum, ur);
                        }
                    };
                    auto sweep = [&](auto EDG) __attribute__((always_inline)) {
                        if constexpr (ROLL) {
                            if (n >= 1) adj_step(0, Pos<kYes>{}, Pos<kNo>{}, EDG);
#pragma unroll kPairDeepUnroll
                            for (int j = 1; j <= n - 1; ++j) adj_step(j, Pos<kNo>{}, Pos<kNo>{}, EDG);
                            adj_step(n, Pos<kRt>{}, Pos<kYes>{}, EDG);
                        } else {
#pragma unroll
                            for (int j = 0; j <= NM; ++j)
                                if (j <= n) adj_step(j, Pos<kRt>{}, Pos<kRt>{}, EDG);
                        }
                        if constexpr (decltype(EDG)::value) {
                            while (eq_cnt >= 32) {
                                __syncwarp();
                                eq_drain(32);
                            }
                        }
                    };
                    // the staged sign of 1/err marks Q points whose nodes may reach an
                    // interior-edge band (warp-uniform choice)
                    if (__any_sync(kFull, (act[0] && qd[0].w < 0.f) || (act[1] && qd[1].w < 0.f)))
                        sweep(std::true_type{});
                    else
                        sweep(std::false_type{});
                    if constexpr (RES) gres_acc = pfma(wres, pfma(k0h, res_sum, res_k0), gres_acc);
                } // GRAD
            } // LIK
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
            static_assert(ROLL || NACC <= 32, "register partials exceed one reduction batch");
            if constexpr (GRAD && !ROLL) {
#pragma unroll
                for (int t = 0; t < NACC; ++t) {
                    float v = accr[t].x + accr[t].y;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
                    if (lane == 0) sh_red[warp][t] = (double)v;
                }
                __syncthreads();
                if (tid < NACC) {
                    const int t = tid;
                    // accumulator slot -> raw index for this stack's n (-1: unused)
                    const int i = t < NM ? (t < n ? t : -1)
                                  : t < 2 * NM + 1 ? (t - NM <= n ? n + (t - NM) : -1)
                                  : t < 3 * NM + 2 ? (t - 2 * NM - 1 <= n ? 2 * n + 1 + (t - 2 * NM - 1) : -1)
                                                   : (t - 3 * NM - 2 <= n ? 3 * n + 2 + (t - 3 * NM - 2) : -1);
                    if (i >= 0) {
                        double s = 0.0;
                        for (int w = 0; w < WARPS; ++w) s += sh_red[w][t];
                        sh_raw[i] = s;
                    }
                }
                __syncthreads();
            } // GRAD && !ROLL
            if constexpr (ROLL) { // shared-memory partials, 32 raw sums at a time
                const int nraw = 4 * n + 3;
                for (int base = 0; base < nraw; base += 32) {
                    const int cnt = min(32, nraw - base);
                    for (int c = 0; c < cnt; ++c) {
                        const int i = base + c;
                        const int idx = i < n ? i
                                        : i < 2 * n + 1 ? NM + (i - n)
                                        : i < 3 * n + 2 ? 2 * NM + 1 + (i - 2 * n - 1)
                                                        : 3 * NM + 2 + (i - 3 * n - 2);
                        float v = tid < HALF ? sh_acc[idx * HALF + tid] : 0.f;
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
                        if (lane == 0) sh_red[warp][c] = (double)v;
                    }
                    __syncthreads();
                    if (tid < cnt) {
                        double sum = 0.0;
                        for (int w = 0; w < WARPS; ++w) sum += sh_red[w][tid];
                        sh_raw[base + tid] = sum;
                    }
                    __syncthreads();
                }
            }
            {   // loglik (float pair), d/dscale, d/dbkg, d/d ln(dQ scale)
                float h = ll_hi, l = ll_lo, a1 = gsc_acc, a2 = gbk_acc, a3 = gres_acc.x + gres_acc.y;
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
                for (int w = 0; w < WARPS; ++w) s += sh_redd[w][tid];
                sh_raw[4 * n + 3 + tid] = s;
            }
            __syncthreads();
            const int nout = GRAD ? 4 * n + (RES ? 7 : 6) : 1;
            const int off0 = GRAD ? 0 : 4 * n + 3; // loglik mode: llsum only
            if (si.n_chunks == 1) {
                finalize_stack<MODE>(sh_raw, n, p, wi.stack, si.par_off, ka.ll_out, ka.grad_out, ka.res_out, tid,
                                     BLOCK);
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
                    finalize_stack<MODE>(sh_raw, n, p, wi.stack, si.par_off, ka.ll_out, ka.grad_out, ka.res_out,
                                         tid, BLOCK);
                    if (tid == 0) ka.stack_done[wi.stack] = 0;
                }
            }
        } // LIK
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
cudaError_t pair_smem_attr()
{
    // the default cap on dynamic shared memory is 48 KB less the static use
    constexpr size_t dyn = PairTraits<MODE, NMAX>::DYN;
    if (dyn > 0)
        return cudaFuncSetAttribute(nr_pair_kernel<MODE, NMAX, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)dyn);
    return cudaSuccess;
}

template <int MODE, int NMAX, int KC>
cudaError_t pair_launch_k(int grid, const KernelArgs &a, const QuadConst &qc, cudaStream_t st)
{
    static bool attr_done = false; // per process: the attribute belongs to the function
    if (!attr_done) {
        const cudaError_t e = pair_smem_attr<MODE, NMAX, KC>();
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    nr_pair_kernel<MODE, NMAX, KC><<<grid, kPairBlock, PairTraits<MODE, NMAX>::DYN, st>>>(a, qc);
    return cudaGetLastError();
}

template <int MODE, int NMAX, int KC>
cudaError_t pair_occupancy_k(int *blocks)
{
    const cudaError_t e = pair_smem_attr<MODE, NMAX, KC>();
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, nr_pair_kernel<MODE, NMAX, KC>, kPairBlock,
                                                         PairTraits<MODE, NMAX>::DYN);
}

// the 1-layer kernels are also compiled for the workloads' quadrature
// orders (17 and 21 nodes); for deeper stacks the fixed count gains about 1%
// and doubles the build time
template <int MODE, int NMAX>
cudaError_t pair_launch_one(int grid, const KernelArgs &a, const QuadConst &qc, cudaStream_t st)
{
    if constexpr (NMAX == 1) {
        if (qc.K == 21) return pair_launch_k<MODE, NMAX, 21>(grid, a, qc, st);
        if (qc.K == 17) return pair_launch_k<MODE, NMAX, 17>(grid, a, qc, st);
    }
    return pair_launch_k<MODE, NMAX, 0>(grid, a, qc, st);
}

template <int MODE, int NMAX>
cudaError_t pair_occupancy_one(int K, int *blocks)
{
    if constexpr (NMAX == 1) {
        if (K == 21) return pair_occupancy_k<MODE, NMAX, 21>(blocks);
        if (K == 17) return pair_occupancy_k<MODE, NMAX, 17>(blocks);
    }
    return pair_occupancy_k<MODE, NMAX, 0>(blocks);
}

} // namespace

// gradient buckets of the paired kernels
#define NR_PAIR_GRAD_BUCKETS(X) X(1) X(2) X(4) X(8) X(12) X(16) X(20)

bool pair_eligible(int mode, int nmax, int K)
{
    if (!NR_PAIR || K < 3) return false;
    if (!is_grad_mode(mode)) return nmax == 1 || (NR_PAIR_FWD_ANY && nmax == 0);
    if (nmax <= 2) return nmax >= 1;
    return NR_PAIR_DEEP_FROM > 0 && nmax >= NR_PAIR_DEEP_FROM && nmax <= 20;
}

int pair_block_threads() { return kPairBlock; }

cudaError_t pair_occupancy(int mode, int nmax, int K, int *blocks)
{
    if (mode == kModel) return nmax == 1 ? pair_occupancy_one<kModel, 1>(K, blocks)
                                         : pair_occupancy_one<kModel, 0>(K, blocks);
    if (mode == kLoglik) return nmax == 1 ? pair_occupancy_one<kLoglik, 1>(K, blocks)
                                          : pair_occupancy_one<kLoglik, 0>(K, blocks);
    if (mode == kGradRes) {
#define X(B) if (nmax == B) return pair_occupancy_one<kGradRes, B>(K, blocks);
        NR_PAIR_GRAD_BUCKETS(X)
#undef X
    } else {
#define X(B) if (nmax == B) return pair_occupancy_one<kGrad, B>(K, blocks);
        NR_PAIR_GRAD_BUCKETS(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_pair(int mode, int nmax, int grid, const KernelArgs &a, const QuadConst &qc, cudaStream_t st)
{
    if (mode == kModel) return nmax == 1 ? pair_launch_one<kModel, 1>(grid, a, qc, st)
                                         : pair_launch_one<kModel, 0>(grid, a, qc, st);
    if (mode == kLoglik) return nmax == 1 ? pair_launch_one<kLoglik, 1>(grid, a, qc, st)
                                          : pair_launch_one<kLoglik, 0>(grid, a, qc, st);
    if (mode == kGradRes) {
#define X(B) if (nmax == B) return pair_launch_one<kGradRes, B>(grid, a, qc, st);
        NR_PAIR_GRAD_BUCKETS(X)
#undef X
    } else {
#define X(B) if (nmax == B) return pair_launch_one<kGrad, B>(grid, a, qc, st);
        NR_PAIR_GRAD_BUCKETS(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

} // namespace nrimpl
