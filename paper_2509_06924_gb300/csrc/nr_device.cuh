// nr_device.cuh -- device code shared by the mixed-precision kernels
// (nr_mixed.cu: one evaluation per thread; nr_pair.cu: two per thread):
// constants, the FP32 primitives with double-float guards, the scalar forward
// model pieces and the interior-edge adjoint (used by both kernels' edge
// queues), and the per-stack staging and output conversion.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "nr_internal.h"

namespace nrimpl {
namespace {

constexpr float kInv2Pi = 0.159154943091895335769f;
constexpr float kTwoPiHi = 6.28318548202514648438f;      // float(2 pi)
constexpr float kTwoPiLo = -1.74845553146951715e-07f;    // 2 pi - kTwoPiHi
constexpr float kRoundMagic = 12582912.0f;               // 1.5 * 2^23: x + M - M rounds x to an integer
constexpr double kFourPiD = 12.566370614359172953850573533118;
constexpr double kLog2ED = 1.4426950408889634073599246810019; // log2(e)
constexpr float kLog2Pi = 1.83787706640934548356f;       // ln(2 pi)
constexpr unsigned kFull = 0xffffffffu;

// |k_j|^2 < kEdgeFrac k_0^2 selects the interior-edge treatment of the adjoint
#ifndef NR_EDGE_FRAC
#define NR_EDGE_FRAC 0.04f
#endif
constexpr float kEdgeFrac = NR_EDGE_FRAC;

// 1: Nevot-Croce phase and |u + i a| are computed without data-dependent
// branches (a few more XU operations, straight-line code)
#ifndef NR_BRANCHFREE
#define NR_BRANCHFREE 1
#endif
// 1: the 1-layer kernels treat n as the compile-time constant 1
#ifndef NR_EXACT1
#define NR_EXACT1 1
#endif

// Position of a sweep step, known at compile time or tested at run time: the
// rolled sweeps peel their first and last steps so that the steps between
// them carry no branches on j.
enum : int { kNo = 0, kYes = 1, kRt = 2 };
template <int V>
using Pos = std::integral_constant<int, V>;
template <class P>
__device__ __forceinline__ bool pos_flag(P, bool rt)
{
    return P::value == kRt ? rt : P::value == kYes;
}

// ------------------------------------------------------------ primitives --
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// 2^x; exp(y) is taken as 2^(y log2 e) with log2 e folded into the staged
// per-stack constants
__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void sincos_approx(float x, float &sn, float &cs)
{
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(sn) : "f"(x));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(cs) : "f"(x));
}
// sin / cos of the layer phases and of the Nevot-Croce factors.
// NR_SINCOS_TABLE 1: a 128-entry table of cos / sin at multiples of 2 pi / 128
// (correctly rounded on the host, staged in shared memory) and two short
// polynomials for the remainder |x| <= pi / 128 (sin: x - x^3 / 6, below
// 1e-10; cos: 1 - c x^2 with c the minimax coefficient on that interval,
// below 2.6e-9, where the Taylor c = 1/2 leaves a one-sided 1.5e-8),
// combined by the angle-addition formula: about 1e-7 absolute, on the FMA
// pipe plus one shared load.  0: the special-function unit's sin.approx /
// cos.approx (about 5e-7 absolute over [-pi, pi]).  Near a waveguide
// resonance the gradient amplifies the phase error by 10^2 - 10^3, which
// the table keeps within the tolerance where the special-function unit did
// not.
#ifndef NR_SINCOS_TABLE
#define NR_SINCOS_TABLE 1
#endif
// the same choice for the Nevot-Croce factors (their phase is usually small,
// but the special-function unit's error there is absolute too)
#ifndef NR_NC_TABLE
#define NR_NC_TABLE NR_SINCOS_TABLE
#endif

constexpr int kTabN = kSinCosTabN;
static_assert(kTabN == 128, "reduction constants are for 128 entries");
constexpr float kTabScale = 20.3718318939209f;        // 128 / (2 pi)
constexpr float kTabStepHi = 0.04908738657832146f;    // float(2 pi / 128)
constexpr float kTabStepLo = -1.3659808839605603e-09f; // 2 pi / 128 - kTabStepHi
// c of cos x ~ 1 - c x^2 minimising the largest error over |x| <= pi / 128
constexpr float kTabCosC = 0.4999791979789734f;

// (cos, sin) of ph + pl (pl a low-order correction, |pl| << 1): reduction
// by multiples of 2 pi / 128 (the multiple rounded with the 1.5 * 2^23
// addition, whose low mantissa bits are then the table index), remainder
// polynomials sin x ~ x - x^3 / 6, cos x ~ 1 - kTabCosC x^2.  tab: cos at
// [i], sin at [kTabN + i].
__device__ __forceinline__ float2 cis_tab(float ph, float pl, const float *tab)
{
    const float t = fmaf(ph, kTabScale, kRoundMagic);
    const float nt = __fadd_rn(t, -kRoundMagic);
    const int i = __float_as_int(t) & (kTabN - 1);
    const float2 cs = make_float2(tab[i], tab[kTabN + i]);
    float x = fmaf(-nt, kTabStepHi, ph);
    x = fmaf(-nt, kTabStepLo, x);
    x = __fadd_rn(x, pl);
    const float z = x * x;
    const float sn = fmaf(x * z, -1.f / 6.f, x);
    const float cn = fmaf(z, -kTabCosC, 1.f);
    return make_float2(fmaf(cs.x, cn, -cs.y * sn), fmaf(cs.y, cn, cs.x * sn));
}

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// Error-free transformations (Knuth TwoSum, Dekker FastTwoSum); the _rn
// intrinsics keep the compiler from fusing or reassociating them.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fadd_rn(s, -a);
    e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fadd_rn(b, -__fadd_rn(s, -a));
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 cmulc(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float2 csqr(float2 a)
{
    return make_float2((a.x - a.y) * (a.x + a.y), 2.f * a.x * a.y);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// 1 - a^2
__device__ __forceinline__ float2 one_minus_sq(float2 a)
{
    return make_float2(fmaf(-a.x, a.x, fmaf(a.y, a.y, 1.f)), -2.f * a.x * a.y);
}
// conj(a) * b + c, four fused multiply-adds
__device__ __forceinline__ float2 cfmac(float2 a, float2 b, float2 c)
{
    return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(-a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 cdiv(float2 a, float2 b)
{
    const float inv = rcp_approx(fmaf(b.x, b.x, b.y * b.y));
    return cscale(cmulc(b, a), inv);
}

// z-component of the wavevector in one medium: value (re, im) plus the low
// word of Re k when the wave propagates (double-float real part).
struct Kz {
    float re, im, lo;
};
__device__ __forceinline__ float2 kc(const Kz &k) { return make_float2(k.re, k.im); }

// Principal sqrt of u + i a (u = uh + ul double-float, a >= 0; aa = (a, a^2))
// from two rsqrt: t = sqrt((|u| + |z|) / 2) is the dominant component and
// a / (2 t) the other.  With REFINE, one Newton step on the dominant
// component makes Re k good to double-float accuracy for propagating waves
// (a layer phase needs it) and Im k good to FP32 accuracy for evanescent ones.
template <bool REFINE>
__device__ __forceinline__ Kz kz_sqrt(float uh, float ul, float2 aa)
{
    const float a = aa.x;
    const float au = fabsf(uh);
    float m = au;
    if (NR_BRANCHFREE || a != 0.f) {
        const float m2 = fmaf(uh, uh, aa.y);
        m = m2 * rsqrt_approx(fmaxf(m2, 1e-37f));
    }
    // H = |u| + |z| = 2 t^2; rsqrt(2 H) = 1 / (2 t) exactly as 0.5 rsqrt(H / 2)
    const float H = au + m;
    const float i2t = rsqrt_approx(fmaxf(H + H, 4e-30f)); // 1 / (2 t)
    const float t = H * i2t;
    const float small = a * i2t;
    const bool prop = uh >= 0.f;
    Kz k;
    if constexpr (REFINE) {
        // residual of big^2 - small^2 = |u| and its Newton correction
        const float e = fmaf(-t, t, au) + fmaf(small, small, prop ? ul : -ul);
        const float corr = e * i2t;
        k.re = prop ? t : small;
        k.im = prop ? small : t + corr;
        k.lo = prop ? corr : 0.f;
    } else {
        k.re = prop ? t : small;
        k.im = prop ? small : t;
        k.lo = 0.f;
    }
    return k;
}

// k of medium j >= 1 from k_0^2 = (p_hi + p_lo) and c_j = 4 pi (rho_j - rho_0).
// Without REFINE (the backing medium: no phase) u is formed in FP32, where
// p_hi - c_hi is exact near the critical edge (Sterbenz) and the low words
// keep the rest to FP32 accuracy.
template <bool REFINE>
__device__ __forceinline__ Kz medium_kz(float p_hi, float p_lo, float4 m)
{
    const float2 c = make_float2(m.x, m.y), a = make_float2(m.z, m.w);
    if constexpr (REFINE) {
        float uh, ul;
        two_sum(p_hi, -c.x, uh, ul);
        ul = __fadd_rn(ul, __fadd_rn(p_lo, -c.y));
        fast_two_sum(uh, ul, uh, ul);
        return kz_sqrt<true>(uh, ul, a);
    } else {
        const float u = (p_hi - c.x) + (p_lo - c.y);
        return kz_sqrt<false>(u, 0.f, a);
    }
}

// E = exp(2 i k d).  The real phase 2 Re(k) d is formed in double-float and
// reduced modulo 2 pi (Cody-Waite, two-word 2 pi; the multiple of 2 pi is
// rounded with the 1.5 * 2^23 addition) before the FP32 sincos.
// L = (2 d as (hi, lo), ea = -2 d log2(e), -): |E| = 2^(Im(k) ea).
__device__ __forceinline__ float2 layer_phase(const Kz &k, float4 L, const float *tab)
{
    const float2 d2 = make_float2(L.x, L.y);
    const float ea = L.z;
    const float t = k.re, tl = k.lo;
    const float ph = __fmul_rn(t, d2.x);
    float pl = fmaf(t, d2.x, -ph);
    pl = fmaf(t, d2.y, pl);
    pl = fmaf(tl, d2.x, pl);
    const float amp = ex2_approx(k.im * ea);
#if NR_SINCOS_TABLE
    const float2 e = cis_tab(ph, pl, tab);
    return make_float2(amp * e.x, amp * e.y);
#else
    const float nt = __fadd_rn(fmaf(ph, kInv2Pi, kRoundMagic), -kRoundMagic);
    float red = fmaf(-nt, kTwoPiHi, ph);
    red = fmaf(-nt, kTwoPiLo, red);
    red += pl;
    float s, c;
    sincos_approx(red, s, c);
    return make_float2(amp * c, amp * s);
#endif
}

// r_j with Nevot-Croce roughness; also returns G = exp(s k_a k_b) / S^2 with
// S = k_a + k_b (the adjoint needs it) and kk = k_a k_b: r = N G.  I = (N, s,
// sl = s log2(e)).  REAL_A:
// k_a is real (the fronting medium), its imaginary part is not read.
template <bool REAL_A>
__device__ __forceinline__ float2 fresnel_nc(float2 ka, float2 kb, float4 I, float2 &G, float2 &kk, const float *tab)
{
    const float2 N = make_float2(I.x, I.y);
    const float s = I.z, sl = I.w;
    const float Sx = ka.x + kb.x, Sy = REAL_A ? kb.y : ka.y + kb.y;
    const float n2 = fmaf(Sx, Sx, Sy * Sy);
    const float inv = n2 > 0.f ? rcp_approx(n2) : 0.f;
    const float2 iS = make_float2(Sx * inv, -Sy * inv); // 1/S
    const float2 iS2 = csqr(iS);                         // 1/S^2
    kk = REAL_A ? make_float2(ka.x * kb.x, ka.x * kb.y) : cmul(ka, kb);
    const float amp = ex2_approx(sl * kk.x);
    float2 F = make_float2(amp, 0.f);
    const float wi = s * kk.y;
    if (NR_BRANCHFREE || wi != 0.f) {
#if NR_NC_TABLE
        const float2 e = cis_tab(wi, 0.f, tab);
        F = make_float2(amp * e.x, amp * e.y);
#else
        float sn, cs;
        sincos_approx(wi, sn, cs);
        F = make_float2(amp * cs, amp * sn);
#endif
    }
    G = cmul(F, iS2);
    return cmul(N, G);
}

// X = (r + Y) / (1 + r Y); D = 1 / (1 + r Y).
__device__ __forceinline__ float2 mobius(float2 r, float2 Y, float2 &D)
{
    const float2 rY = cmul(r, Y);
    const float dx = 1.f + rY.x, dy = rY.y;
    const float inv = rcp_approx(fmaf(dx, dx, dy * dy));
    D = make_float2(dx * inv, -dy * inv);
    return cmul(cadd(r, Y), D);
}

// ------------------------------------------------- interior critical edges --
// Near the critical edge of an interior layer (k_j -> 0) the Parratt form is
// 0/0 (r_{j-1} -> 1, r_j -> -1, E_j -> 1) and the plain adjoint forms d/dk_j
// as a sum of large terms that cancel before dividing by k_j, which costs
// FP32 all its digits.  The reflectivity is an even function of every
// interior k_j (the rough Fresnel coefficients obey r(-k) = 1/r(k)), so it
// depends on u_j = k_j^2 only.  These evaluations take dX_{j-1}/du_j through
// the layer's symmetrised characteristic matrix
//   Lambda = I_{j-1} P_j I_j * (rho+_{j-1} rho+_j) / (2 k_j),
// with rho+_{j-1} = (a + k) e^{a k s1^2}, rho+_j = (k + b) e^{k b s2^2}; its
// entries are (ab +- u) sinh(k g)/k + (a +- b) cosh(k g) with
// g = a s1^2 +- b s2^2 -+ i d (a = k_{j-1}, b = k_{j+1}), all even in k_j,
// differentiated in u analytically (no cancellation):
//   X_{j-1} = (L10 + L11 Z) / (L00 + L01 Z),  Z = X_{j+1} E_{j+1}
// (Z = 0 for the bottom layer, where only L00 and L10 are needed).
struct Hyp {
    float2 ch, shc, g; // cosh(x), sinh(x)/x, (x cosh x - sinh x)/x^3, all times e^-m
};

__device__ __forceinline__ Hyp hyp_scaled(float2 x, float m)
{
    float sn, cs;
    __sincosf(x.y, &sn, &cs);
    const float ep = __expf(x.x - m), em = __expf(-x.x - m);
    Hyp h;
    h.ch = make_float2(0.5f * (ep + em) * cs, 0.5f * (ep - em) * sn);
    const float r2 = fmaf(x.x, x.x, x.y * x.y);
    if (r2 < 0.25f) {
        // Taylor series in x^2 (truncation < 1e-10 for |x| < 1/2), scaled
        const float2 x2 = csqr(x);
        const float sc = __expf(-m);
        float2 t = cadd(make_float2(1.f, 0.f), cscale(x2, 1.f / 72.f));
        t = cadd(make_float2(1.f, 0.f), cscale(cmul(x2, t), 1.f / 42.f));
        t = cadd(make_float2(1.f, 0.f), cscale(cmul(x2, t), 1.f / 20.f));
        t = cadd(make_float2(1.f, 0.f), cscale(cmul(x2, t), 1.f / 6.f));
        h.shc = cscale(t, sc);
        float2 v = make_float2(1.f / 3991680.f, 0.f);
        v = cadd(make_float2(1.f / 45360.f, 0.f), cmul(x2, v));
        v = cadd(make_float2(1.f / 840.f, 0.f), cmul(x2, v));
        v = cadd(make_float2(1.f / 30.f, 0.f), cmul(x2, v));
        v = cadd(make_float2(1.f / 3.f, 0.f), cmul(x2, v));
        h.g = cscale(v, sc);
    } else {
        const float2 sh = make_float2(0.5f * (ep - em) * cs, 0.5f * (ep + em) * sn);
        const float2 ix = cdiv(make_float2(1.f, 0.f), x);
        h.shc = cmul(sh, ix);
        h.g = cmul(csub(cmul(x, h.ch), sh), cmul(ix, csqr(ix)));
    }
    return h;
}

// Returns ubar = conj(dX_{j-1}/du_j) * Xbar_{j-1}.
__device__ __forceinline__ float2 edge_ubar(float2 a, float2 k, float2 b, float s1, float s2, float d, float2 Z,
                                            bool zzero, float2 Xbar_up)
{
    const float2 u = csqr(k);
    const float2 ab = cmul(a, b);
    const float2 sp = cadd(cscale(a, s1 * s1), cscale(b, s2 * s2));
    const float2 sq = csub(cscale(a, s1 * s1), cscale(b, s2 * s2));
    // common scale e^-m, m >= max |Re(k g)| over the exponents
    float m = fmaxf(fabsf(fmaf(k.x, sp.x, -k.y * sp.y)), fabsf(fmaf(k.x, sq.x, -k.y * sq.y)));
    m += fabsf(k.y * d);
    // entry i: 0 chi (L00), 1 phi (L10), 2 nu (L01), 3 psi (L11); streamed
    // into den = L00 + L01 Z, dden, xn = L10 + L11 Z, dxn
    float2 den = make_float2(0.f, 0.f), dden = den, xn = den, dxn = den;
    const int ne = zzero ? 2 : 4;
#pragma unroll 1
    for (int i = 0; i < ne; ++i) {
        const bool plus = (i == 0 || i == 3);                   // (ab+u) S + (a+b) C
        const float2 base = plus ? sp : sq;
        const float2 g = make_float2(base.x, (i == 0 || i == 2) ? base.y - d : base.y + d);
        const Hyp h = hyp_scaled(cmul(k, g), m);
        const float2 g2 = csqr(g);
        const float2 S = cmul(g, h.shc);                        // sinh(kg)/k
        const float2 dC = cscale(cmul(g2, h.shc), 0.5f);        // d cosh(kg)/du
        const float2 dS = cscale(cmul(cmul(g2, g), h.g), 0.5f); // d (sinh(kg)/k)/du
        const float2 f = plus ? cadd(ab, u) : csub(u, ab);      // (ab+u) or -(ab-u)
        const float2 cfac = plus ? cadd(a, b) : csub(a, b);     // (a+b) or (a-b)
        const float2 L = cadd(cmul(f, S), cmul(cfac, h.ch));
        const float2 dL = cadd(S, cadd(cmul(f, dS), cmul(cfac, dC)));
        const float2 w = (i >= 2) ? Z : make_float2(1.f, 0.f);
        if (i == 0 || i == 2) {
            den = cadd(den, cmul(w, L));
            dden = cadd(dden, cmul(w, dL));
        } else {
            xn = cadd(xn, cmul(w, L));
            dxn = cadd(dxn, cmul(w, dL));
        }
    }
    const float2 X = cdiv(xn, den);
    const float2 dXdu = cdiv(csub(dxn, cmul(X, dden)), den);
    return cmulc(dXdu, Xbar_up);
}

// k_0^2 = (p_hi + p_lo) from k_0 = (k0h + k0l), double-float
__device__ __forceinline__ void k0_square(float k0h, float k0l, float &p_hi, float &p_lo)
{
    p_hi = __fmul_rn(k0h, k0h);
    p_lo = fmaf(k0h, k0h, -p_hi);
    p_lo = fmaf(2.f * k0h, k0l, p_lo);
}

// One queued interior-edge evaluation: the entry keeps the node k_0 (hi, lo),
// Z and Xbar_{j-1}; k_{j-1}, k_j and k_{j+1} are formed again from the node
// exactly as the sweeps form them.
__device__ __forceinline__ float2 edge_entry_ubar(float2 node, float2 Z, float2 Xbu, int j, int n,
                                                  const float4 *med, const float4 *lay)
{
    float p_hi, p_lo;
    k0_square(node.x, node.y, p_hi, p_lo);
    const Kz ka = j == 1 ? Kz{node.x, 0.f, node.y} : medium_kz<true>(p_hi, p_lo, med[j - 1]);
    const Kz kj = medium_kz<true>(p_hi, p_lo, med[j]);
    const Kz kb = j == n ? medium_kz<false>(p_hi, p_lo, med[j + 1]) : medium_kz<true>(p_hi, p_lo, med[j + 1]);
    return edge_ubar(kc(ka), kc(kj), kc(kb), lay[j - 1].w, lay[j].w, 0.5f * lay[j].x, Z, j == n, Xbu);
}

// Drains `cnt` queued interior-edge entries of one warp (one per lane) into
// per-thread partials kept in shared memory (acc points at this thread's
// slot of medium 1's Re-accumulator; stride between accumulators `stride`,
// Re -> Im distance `im_off`; med, lay: the staged stack entries).  Kept out
// of line so that the rolled sweep it is called from keeps its register budget.
template <int EQ, bool RES>
__device__ __noinline__ float eq_drain_smem(float2 (*q)[EQ], const int *qj, const float4 *med, const float4 *lay,
                                            int n, int lane, int cnt, float *acc, int stride, int im_off)
{
    float res = 0.f; // the resolution-mode term of the entry (factor in q[3])
    if (lane < cnt) {
        const int j = qj[lane];
        const float2 ub = edge_entry_ubar(q[0][lane], q[1][lane], q[2][lane], j, n, med, lay);
        // conj(kbar)/k_j = 2 conj(ubar)
        acc[(j - 1) * stride] += 2.f * ub.x;
        acc[(j - 1) * stride + im_off] += -2.f * ub.y;
        if constexpr (RES) res = 2.f * ub.x * q[3][lane].x;
    }
    return res;
}

// Slot of a new interior-edge queue entry, and the queue's count after an
// append: NR_DEBUG builds flag a slot past the CAP-entry queue and keep it
// (and the count) inside, so an overflow corrupts entries, not memory.
template <int CAP>
__device__ __forceinline__ int queue_slot(int slot, int32_t *status)
{
    if constexpr (NR_DEBUG) {
        if (slot >= CAP) {
            atomicOr(status, NR_FLAG_DEBUG_BOUNDS);
            return CAP - 1;
        }
    }
    return slot;
}
template <int CAP>
__device__ __forceinline__ int queue_count(int cnt)
{
    if constexpr (NR_DEBUG) return cnt < CAP ? cnt : CAP;
    return cnt;
}

// Per-stack parameters staged in shared memory, one 16-byte entry per
// medium, interface and layer (a sweep step reads each with one load).
template <int NM>
struct StackSmem {
    float4 med[NM + 2]; // medium j = 1..n+1: 4 pi (rho_j - rho_0) as (hi, lo), 4 pi iota_j, its square
    float4 itf[NM + 1]; // interface j = 0..n: 4 pi (rho_{j+1} - rho_j) + 4 pi i (iota_j - iota_{j+1}),
                        // s_j = -2 sigma_j^2, s_j log2(e)
    float4 lay[NM + 2]; // layer j = 1..n: 2 d_j as (hi, lo), -2 d_j log2(e); sigma_j (j = 0..n)
    float scale, bkg;
};

__device__ __forceinline__ float2 split_double(double v)
{
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

template <int NM>
__device__ void stage_stack(StackSmem<NM> &sm, const double *p, int n, int tid, int32_t *status)
{
    // Thread j stages medium j / interface j / layer j.
    if (tid <= n + 1) {
        const int j = tid;
        const double rho0 = p[n];
        bool bad = false;
        float4 lay = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j >= 1) {
            const double rj = p[n + j];
            const double ij = p[2 * n + 2 + j - 1];
            const float2 c = split_double(kFourPiD * (rj - rho0));
            sm.med[j] = make_float4(c.x, c.y, (float)(kFourPiD * ij), (float)(kFourPiD * kFourPiD * ij * ij));
            bad |= !isfinite(rj) || !isfinite(ij);
            if (j <= n) {
                const double dj = p[j - 1];
                const float2 d2 = split_double(2.0 * dj);
                lay.x = d2.x;
                lay.y = d2.y;
                lay.z = (float)(-2.0 * kLog2ED * dj);
                bad |= !isfinite(dj);
            }
        } else {
            bad |= !isfinite(rho0);
        }
        if (j <= n) {
            const double iot_j = j >= 1 ? p[2 * n + 2 + j - 1] : 0.0;
            const double iot_j1 = p[2 * n + 2 + j];
            const double sig = p[3 * n + 3 + j];
            sm.itf[j] = make_float4((float)(kFourPiD * (p[n + j + 1] - p[n + j])),
                                    (float)(kFourPiD * (iot_j - iot_j1)), (float)(-2.0 * sig * sig),
                                    (float)(-2.0 * kLog2ED * sig * sig));
            lay.w = (float)sig;
            bad |= !isfinite(sig);
        }
        sm.lay[j] = lay;
        if (j == 0) {
            sm.scale = (float)p[4 * n + 4];
            sm.bkg = (float)p[4 * n + 5];
            bad |= !isfinite(p[4 * n + 4]) || !isfinite(p[4 * n + 5]);
        }
        if (bad) atomicOr(status, NR_FLAG_NONFINITE_PARAM);
    }
}

// Convert a stack's raw sums into outputs (loglik, packed gradient).
//   raw: [accD (n) | accUr (n+1) | accUi (n+1) | accS (n+1) | llsum | gscale | gbkg | gres]
template <int MODE>
__device__ void finalize_stack(const double *raw, int n, const double *p, int s, int64_t par_off,
                               double *ll_out, double *grad_out, double *res_out, int tid, int nthreads)
{
    if (tid == 0 && ll_out) ll_out[s] = -0.5 * raw[4 * n + 3];
    if (MODE == kGradRes && tid == 0 && res_out) res_out[s] = raw[4 * n + 6];
    if (!is_grad_mode(MODE) || grad_out == nullptr) return;
    const double twoPi = 6.283185307179586476925286766559;
    double *g = grad_out + par_off;
    for (int i = tid; i < 4 * n + 6; i += nthreads) {
        double v;
        if (i < n) {
            v = 2.0 * raw[i];                                  // d_j
        } else if (i == n) {                                   // rho_0 = -sum rho_j
            double acc = 0.0;
            for (int j = 1; j <= n + 1; ++j) acc += raw[n + j - 1];
            v = twoPi * acc;
        } else if (i < 2 * n + 2) {
            v = -twoPi * raw[n + (i - n) - 1];                 // rho_j, j >= 1
        } else if (i < 3 * n + 3) {
            v = -twoPi * raw[2 * n + 1 + (i - (2 * n + 2))];   // iota_j
        } else if (i < 4 * n + 4) {
            const int j = i - (3 * n + 3);
            v = -4.0 * p[3 * n + 3 + j] * raw[3 * n + 2 + j];  // sigma_j
        } else {
            v = raw[i];                                        // scale, bkg
        }
        g[i] = v;
    }
}

} // namespace
} // namespace nrimpl
