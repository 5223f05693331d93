// nr_mixed.cu -- the fast path: batched reflectivity, log-likelihood and its
// exact gradient in complex FP32 with double-float guards, for sm_103a.
//
// Work decomposition.  A work item is a range of Q points of one stack.  A
// persistent CTA takes items from a queue (atomic ticket, cost-sorted on the
// host) and sweeps the item in tiles of TQ Q points x K quadrature nodes: one
// thread per (Q point, node) evaluation, the K threads of a Q point adjacent.
// The stack's parameters are staged once per item in shared memory (FP64 ->
// float pairs).  Per evaluation (Sec. 2.1 forward model, Sec. 3 smearing):
//   a1  node   q = Q + dQ x_k / (2 sqrt(ln 2))             double-float
//   a3  k_j = sqrt(k_0^2 - 4pi(rho_j - rho_0) + 4pi i iota_j)
//              k_0^2 - c_j in double-float, sqrt + one Newton step
//   a4  r_j = 4pi(drho_j + i diota_j) / (k_j + k_{j+1})^2 * exp(-2 k_j k_{j+1} s_j^2)
//              cancellation-free numerator (exactly k_j^2 - k_{j+1}^2)
//   a5  E_j = exp(2 i k_j d_j): phase 2 Re(k_j) d_j in double-float reduced
//              mod 2 pi before the FP32 sincos
//   a6  Parratt recursion from the backing up: X_n = r_n,
//       X_j = (r_j + X_{j+1} E_{j+1}) / (1 + r_j X_{j+1} E_{j+1}), R = |X_0|^2
//   a8  smearing: the K node values of a Q point meet in shared memory,
//   a9  m = scale S + bkg; loglik term accumulated in FP64,
//   a10 dl/dm seeds the adjoint of every node,
//   a7  adjoint: a top-down sweep over the interfaces using the stored X_j
//       (and, for 1-2 layers, every stored intermediate; deeper stacks
//       recompute k_j, r_j, E_j), accumulating per-thread partial gradients.
// At the end of an item the CTA reduces its partials (warp shuffles, then a
// fixed-order cross-warp sum in FP64).  Stacks split over several items meet
// through per-chunk partial slots; the last arriving CTA sums them in chunk
// order, so results are bitwise reproducible.
#include <cuda_runtime.h>

#include <cstdint>

#include "nr_internal.h"

namespace nrimpl {
namespace {

constexpr float kInv2Pi = 0.159154943091895335769f;
constexpr float kTwoPiHi = 6.28318548202514648438f;      // float(2 pi)
constexpr float kTwoPiLo = -1.74845553146951715e-07f;    // 2 pi - kTwoPiHi
constexpr double kFourPiD = 12.566370614359172953850573533118;
constexpr float kLog2Pi = 1.83787706640934548356f;       // ln(2 pi)
// |k_j|^2 < kEdgeFrac k_0^2 selects the interior-edge guard of the adjoint
#ifndef NR_EDGE_FRAC
#define NR_EDGE_FRAC 0.04f
#endif
constexpr float kEdgeFrac = NR_EDGE_FRAC;

// CTAs per SM the compiler is asked to fit (register cap) for the 1-layer
// gradient bucket and the forward kernels; overridable at build time.
#ifndef NR_MINB_GRAD1
#define NR_MINB_GRAD1 4
#endif
#ifndef NR_MINB_FWD
#define NR_MINB_FWD 4
#endif

// ------------------------------------------------------------ primitives --
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
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
// Re(conj(a) * b)
__device__ __forceinline__ float redot(float2 a, float2 b) { return fmaf(a.x, b.x, a.y * b.y); }

// z-component of the wavevector in one medium: value (re, im) plus the low
// word of Re k when the wave propagates (double-float real part).
struct Kz {
    float re, im, lo;
};
__device__ __forceinline__ float2 kc(const Kz &k) { return make_float2(k.re, k.im); }

// Principal sqrt of u + i a (u = uh + ul double-float, a >= 0): FP32 root
// from one rsqrt, then one Newton step on the dominant component, which makes
// Re k good to double-float accuracy for propagating waves (the phase needs
// it) and Im k good to FP32 accuracy for evanescent ones.
__device__ __forceinline__ Kz kz_sqrt(float uh, float ul, float a)
{
    const float au = fabsf(uh);
    float m = au;
    if (a != 0.f) {
        const float m2 = fmaf(uh, uh, a * a);
        m = m2 * rsqrt_approx(fmaxf(m2, 1e-37f));
    }
    const float h = fmaxf(0.5f * (au + m), 1e-30f);
    const float rt = rsqrt_approx(h);
    const float t = h * rt;     // sqrt(h)
    const float i2t = 0.5f * rt; // 1 / (2 sqrt(h))
    const float small = a * i2t;
    const bool prop = uh >= 0.f;
    const float sgn = prop ? 1.f : -1.f;
    // residual of big^2 - small^2 = |u| and its Newton correction
    const float e = fmaf(-t, t, sgn * uh) + fmaf(small, small, sgn * ul);
    const float corr = e * i2t;
    Kz k;
    k.re = prop ? t : small;
    k.im = prop ? small : t + corr;
    k.lo = prop ? corr : 0.f;
    return k;
}

// k of medium j >= 1 from k_0^2 = (p_hi + p_lo) and c_j = 4 pi (rho_j - rho_0).
__device__ __forceinline__ Kz medium_kz(float p_hi, float p_lo, float2 c, float a)
{
    float uh, ul;
    two_sum(p_hi, -c.x, uh, ul);
    ul = __fadd_rn(ul, __fadd_rn(p_lo, -c.y));
    fast_two_sum(uh, ul, uh, ul);
    return kz_sqrt(uh, ul, a);
}

// E = exp(2 i k d).  The real phase 2 Re(k) d is formed in double-float and
// reduced modulo 2 pi (Cody-Waite, two-word 2 pi) before the FP32 sincos.
__device__ __forceinline__ float2 layer_phase(const Kz &k, float2 d)
{
    const float t = 2.f * k.re, tl = 2.f * k.lo;
    const float ph = __fmul_rn(t, d.x);
    float pl = fmaf(t, d.x, -ph);
    pl = fmaf(t, d.y, pl);
    pl = fmaf(tl, d.x, pl);
    const float nt = rintf(ph * kInv2Pi);
    float red = fmaf(-nt, kTwoPiHi, ph);
    red = fmaf(-nt, kTwoPiLo, red);
    red += pl;
    float s, c;
    __sincosf(red, &s, &c);
    const float amp = __expf(-2.f * k.im * d.x);
    return make_float2(amp * c, amp * s);
}

// r_j with Nevot-Croce roughness; also returns G = exp(s k_a k_b) / S^2 with
// S = k_a + k_b (the adjoint needs it): r = N G.
__device__ __forceinline__ float2 fresnel_nc(float2 ka, float2 kb, float2 N, float s, float2 &G)
{
    const float Sx = ka.x + kb.x, Sy = ka.y + kb.y;
    const float n2 = fmaf(Sx, Sx, Sy * Sy);
    const float inv = n2 > 0.f ? rcp_approx(n2) : 0.f;
    const float2 iS = make_float2(Sx * inv, -Sy * inv); // 1/S
    const float2 iS2 = csqr(iS);                         // 1/S^2
    const float2 kk = cmul(ka, kb);
    const float amp = __expf(s * kk.x);
    float2 F = make_float2(amp, 0.f);
    const float wi = s * kk.y;
    if (wi != 0.f) {
        float sn, cs;
        __sincosf(wi, &sn, &cs);
        F = make_float2(amp * cs, amp * sn);
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
// Near the critical edge of an interior layer (k_j -> 0) the plain adjoint
// forms d/dk_j as a sum of large terms that cancel and then divides by k_j,
// which costs FP32 all its digits.  The reflectivity is an even function of
// every interior k_j (the rough Fresnel coefficients obey r(-k) = 1/r(k)),
// so it depends on u_j = k_j^2 only.  This guard evaluates dX_{j-1}/du_j
// through the layer's symmetrised characteristic matrix
//   Lambda = I_{j-1} P_j I_j * (rho+_{j-1} rho+_j) / (2 k_j),
// whose entries are (ab +- u) sinh(k g)/k + (a +- b) cosh(k g) with
// g = a s1^2 +- b s2^2 +- i d (a = k_{j-1}, b = k_{j+1}), all even in k_j,
// and differentiates them in u analytically (no cancellation):
//   X_{j-1} = (L10 + L11 Z) / (L00 + L01 Z),  Z = X_{j+1} E_{j+1}.
// Returns ubar = conj(dX_{j-1}/du_j) * Xbar_{j-1}.
__device__ __forceinline__ float2 cdiv(float2 a, float2 b)
{
    const float inv = rcp_approx(fmaf(b.x, b.x, b.y * b.y));
    return cscale(cmulc(b, a), inv);
}

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

template <bool INL>
__device__ float2 edge_ubar_impl(float2 a, float2 k, float2 b, float s1, float s2, float d, float2 Z,
                                         float2 Xbar_up)
{
    const float2 u = csqr(k);
    const float2 ab = cmul(a, b);
    const float2 sp = cadd(cscale(a, s1 * s1), cscale(b, s2 * s2));
    const float2 sq = csub(cscale(a, s1 * s1), cscale(b, s2 * s2));
    // common scale e^-m, m = max |Re(k g)| over the four exponents
    float m = fmaxf(fabsf(fmaf(k.x, sp.x, -k.y * sp.y)), fabsf(fmaf(k.x, sq.x, -k.y * sq.y)));
    m += fabsf(k.y * d);
    // entry i: 0 chi (L00), 1 nu (L01), 2 phi (L10), 3 psi (L11); streamed into
    // den = L00 + L01 Z, dden = L00' + L01' Z, xn = L10 + L11 Z, dxn = L10' + L11' Z
    float2 den = make_float2(0.f, 0.f), dden = den, xn = den, dxn = den;
#pragma unroll 1
    for (int i = 0; i < 4; ++i) {
        const bool plus = (i == 0 || i == 3);
        const float2 base = plus ? sp : sq;
        const float2 g = make_float2(base.x, (i == 0 || i == 1) ? base.y - d : base.y + d);
        const Hyp h = hyp_scaled(cmul(k, g), m);
        const float2 g2 = csqr(g);
        const float2 S = cmul(g, h.shc);                        // sinh(kg)/k
        const float2 dC = cscale(cmul(g2, h.shc), 0.5f);        // d cosh(kg)/du
        const float2 dS = cscale(cmul(cmul(g2, g), h.g), 0.5f); // d (sinh(kg)/k)/du
        const float sgn = plus ? 1.f : -1.f;                    // (ab+u) or -(ab-u)
        const float2 f = plus ? cadd(ab, u) : csub(u, ab);
        const float2 cfac = plus ? cadd(a, b) : csub(a, b);     // (a+b) or (a-b)
        const float2 L = cadd(cmul(f, S), cmul(cfac, h.ch));
        const float2 dL = cadd(cscale(S, 1.f), cadd(cmul(f, dS), cmul(cfac, dC)));
        (void)sgn;
        const float2 w = (i == 1 || i == 3) ? Z : make_float2(1.f, 0.f);
        if (i < 2) {
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
__device__ __noinline__ float2 edge_ubar_call(float2 a, float2 k, float2 b, float s1, float s2, float d, float2 Z,
                                              float2 Xbar_up)
{
    return edge_ubar_impl<false>(a, k, b, s1, s2, d, Z, Xbar_up);
}
__device__ __forceinline__ float2 edge_ubar_inline(float2 a, float2 k, float2 b, float s1, float s2, float d,
                                                   float2 Z, float2 Xbar_up)
{
    return edge_ubar_impl<true>(a, k, b, s1, s2, d, Z, Xbar_up);
}

// --------------------------------------------------------------- traits ---
template <int MODE, int NMAX>
struct Traits {
    static constexpr bool kGradMode = MODE == kGrad;
    static constexpr int NM = NMAX > 0 ? NMAX : NR_MAX_LAYERS; // smem capacity
    // per-thread partials live in shared memory for NMAX >= 8; the block
    // shrinks for deep buckets so that they still fit
    static constexpr int BLOCK = !kGradMode ? 256 : NMAX >= 32 ? 128 : 256;
    static constexpr bool STORE = kGradMode && NMAX <= 2;     // keep all intermediates
    static constexpr bool SMEM_ACC = kGradMode && NMAX >= 8;  // per-thread partials in smem
    static constexpr bool UNROLL = NMAX >= 1 && NMAX <= 20;   // register arrays
    static constexpr int NACC = kGradMode ? 4 * NM + 3 : 0;   // partial gradients per thread
    static constexpr int NRAW = 4 * NM + 6;
    static constexpr int WARPS = BLOCK / 32;
    // the 1-layer bucket runs the interior-edge guard after the adjoint sweep
    // (inlined, little else live); deeper buckets call it in the sweep
    static constexpr bool EDGE_DEFER = kGradMode && NMAX == 1;
    // shallow gradient buckets: cap registers so that 4 CTAs fit on an SM
    static constexpr int MINB = !kGradMode ? NR_MINB_FWD : NMAX == 1 ? NR_MINB_GRAD1 : NMAX <= 20 ? 2 : 4;
};

// Per-stack parameters staged in shared memory.
template <int NM>
struct StackSmem {
    float2 c[NM + 2];  // 4 pi (rho_j - rho_0) as (hi, lo), j = 1..n+1
    float a[NM + 2];   // 4 pi iota_j, j = 1..n+1
    float2 N[NM + 1];  // 4 pi (rho_{j+1} - rho_j) + 4 pi i (iota_j - iota_{j+1})
    float s[NM + 1];   // -2 sigma_j^2
    float sg[NM + 1];  // sigma_j
    float2 d[NM + 2];  // thickness (hi, lo), j = 1..n
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
        if (j >= 1) {
            const double rj = p[n + j];
            const double ij = p[2 * n + 2 + j - 1];
            sm.c[j] = split_double(kFourPiD * (rj - rho0));
            sm.a[j] = (float)(kFourPiD * ij);
            bad |= !isfinite(rj) || !isfinite(ij);
            if (j <= n) {
                const double dj = p[j - 1];
                sm.d[j] = split_double(dj);
                bad |= !isfinite(dj);
            }
        } else {
            bad |= !isfinite(rho0);
        }
        if (j <= n) {
            const double iot_j = j >= 1 ? p[2 * n + 2 + j - 1] : 0.0;
            const double iot_j1 = p[2 * n + 2 + j];
            const double sig = p[3 * n + 3 + j];
            sm.N[j] = make_float2((float)(kFourPiD * (p[n + j + 1] - p[n + j])),
                                  (float)(kFourPiD * (iot_j - iot_j1)));
            sm.s[j] = (float)(-2.0 * sig * sig);
            sm.sg[j] = (float)sig;
            bad |= !isfinite(sig);
        }
        if (j == 0) {
            sm.scale = (float)p[4 * n + 4];
            sm.bkg = (float)p[4 * n + 5];
            bad |= !isfinite(p[4 * n + 4]) || !isfinite(p[4 * n + 5]);
        }
        if (bad) atomicOr(status, NR_FLAG_NONFINITE_PARAM);
    }
}

// Convert a stack's raw sums into outputs (loglik, packed gradient).
//   raw: [accD (n) | accUr (n+1) | accUi (n+1) | accS (n+1) | llsum | gscale | gbkg]
template <int MODE>
__device__ void finalize_stack(const double *raw, int n, const double *p, int s, int64_t par_off,
                               double *ll_out, double *grad_out, int tid, int nthreads)
{
    if (tid == 0 && ll_out) ll_out[s] = -0.5 * raw[4 * n + 3];
    if (MODE != kGrad || grad_out == nullptr) return;
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

// ---------------------------------------------------------------- kernel --
template <int MODE, int NMAX>
__global__ void __launch_bounds__(Traits<MODE, NMAX>::BLOCK, Traits<MODE, NMAX>::MINB)
nr_mixed_kernel(const KernelArgs ka, const QuadConst qc)
{
    using T = Traits<MODE, NMAX>;
    constexpr int NM = T::NM;
    constexpr int BLOCK = T::BLOCK;
    constexpr bool GRAD = T::kGradMode;
    constexpr bool LIK = MODE != kModel;

    __shared__ StackSmem<NM> sm;
    __shared__ float sh_wR[2][BLOCK];   // w_k R per evaluation, double-buffered by tile
    __shared__ float sh_seed[2][BLOCK]; // scale * dl/dm per Q slot
    __shared__ double sh_red[T::WARPS][32];
    __shared__ double sh_redd[T::WARPS][4];
    __shared__ double sh_raw[T::NRAW];
    __shared__ int sh_item;
    __shared__ int sh_last;
    extern __shared__ float sh_acc[]; // [NACC][BLOCK] per-thread partials when SMEM_ACC

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int K = qc.K;
    const int TQ = ka.tile_q;
    const int qslot = tid / K;
    const int kn = tid - qslot * K;
    const bool lane_on = qslot < TQ;
    const float g_hi = lane_on ? qc.g_hi[kn] : 0.f;
    const float g_lo = lane_on ? qc.g_lo[kn] : 0.f;
    const float wk = lane_on ? qc.w[kn] : 0.f;
    // per-Q lanes: kSubLanes threads per Q slot of the tile
    const int qgrp = tid / kSubLanes, qpart = tid - qgrp * kSubLanes;
    const bool qlane = qgrp < TQ;
    const int qwarps = (TQ * kSubLanes + 31) / 32;

    for (;;) {
        if (tid == 0) sh_item = atomicAdd(&ka.ticket[0], 1);
        __syncthreads();
        const int item = sh_item;
        if (item >= ka.n_items) break;
        const WorkItem wi = ka.items[item];
        const StackInfo si = ka.stacks[wi.stack];
        const int n = si.n;
        const double *p = ka.params + si.par_off;
        stage_stack<NM>(sm, p, n, tid, ka.status);

        // per-thread partial gradients (FP32; reduced in FP64 per item)
        float accr[GRAD && !T::SMEM_ACC ? T::NACC : 1];
        if constexpr (GRAD) {
            if constexpr (T::SMEM_ACC) {
                for (int i = 0; i < 4 * n + 3; ++i) {
                    const int idx = i < n ? i
                                    : i < 2 * n + 1 ? NM + (i - n)
                                    : i < 3 * n + 2 ? 2 * NM + 1 + (i - 2 * n - 1)
                                                    : 3 * NM + 2 + (i - 3 * n - 2);
                    sh_acc[idx * BLOCK + tid] = 0.f;
                }
            } else {
#pragma unroll
                for (int i = 0; i < T::NACC; ++i) accr[i] = 0.f;
            }
        }
        auto acc_add = [&](int idx, float v) __attribute__((always_inline)) {
            if constexpr (GRAD) {
                if constexpr (T::SMEM_ACC) sh_acc[idx * BLOCK + tid] += v;
                else accr[idx] += v;
            }
        };
        constexpr int oD = 0, oUr = NM, oUi = 2 * NM + 1, oS = 3 * NM + 2;
        // per-Q-lane sums: loglik terms as a float pair, d/dscale, d/dbkg
        float ll_hi = 0.f, ll_lo = 0.f, gsc_acc = 0.f, gbk_acc = 0.f;

        // software pipeline: inputs of the next tile are loaded while the
        // current one computes
        const float *qp = ka.q + si.q_begin, *dqp = ka.dq + si.q_begin;
        const float *rop = ka.r_obs + si.q_begin, *rep = ka.r_err + si.q_begin;
        float Qn = 0.1f, dQn = 0.f, Ron = 0.f, Ren = 1.f;
        {
            const int qi = wi.q_lo + qslot;
            if (lane_on && qi < wi.q_hi) { Qn = __ldg(qp + qi); dQn = __ldg(dqp + qi); }
            const int qj = wi.q_lo + qgrp;
            if (LIK && qlane && qpart == 0 && qj < wi.q_hi) { Ron = __ldg(rop + qj); Ren = __ldg(rep + qj); }
        }
        __syncthreads();

        const float scale = sm.scale, bkg = sm.bkg;
        int buf = 0;
        for (int q0 = wi.q_lo; q0 < wi.q_hi; q0 += TQ, buf ^= 1) {
            const int qi = q0 + qslot;
            const bool act = lane_on && qi < wi.q_hi;
            const float Qv = Qn, dQv = dQn;
            float Ro = Ron, ie = 0.f, lterm = 0.f;
            if (LIK && qlane && qpart == 0) {
                if (!(Ren > 0.f) && q0 + qgrp < wi.q_hi) atomicOr(ka.status, NR_FLAG_BAD_ERR);
                ie = 1.0f / Ren;
                lterm = kLog2Pi + 2.f * logf(Ren);
            }
            {   // prefetch the next tile
                const int q1 = q0 + TQ;
                Qn = 0.1f; dQn = 0.f;
                if (lane_on && q1 + qslot < wi.q_hi) { Qn = __ldg(qp + q1 + qslot); dQn = __ldg(dqp + q1 + qslot); }
                if (LIK && qlane && qpart == 0 && q1 + qgrp < wi.q_hi) {
                    Ron = __ldg(rop + q1 + qgrp);
                    Ren = __ldg(rep + q1 + qgrp);
                }
            }
            // a1: node position in double-float, k_0 = q/2, k_0^2
            float qh, ql;
            {
                const float th = __fmul_rn(dQv, g_hi);
                float tl = fmaf(dQv, g_hi, -th);
                tl = fmaf(dQv, g_lo, tl);
                float s, e;
                two_sum(Qv, th, s, e);
                e = __fadd_rn(e, tl);
                fast_two_sum(s, e, qh, ql);
            }
            const bool qok = qh > 0.f;
            if (act && !qok) atomicOr(ka.status, NR_FLAG_BAD_Q);
            const float k0h = 0.5f * qh, k0l = 0.5f * ql;
            const float p_hi = __fmul_rn(k0h, k0h);
            float p_lo = fmaf(k0h, k0h, -p_hi);
            p_lo = fmaf(2.f * k0h, k0l, p_lo);

            // a3-a6 forward, from the backing upwards
            Kz kst[T::STORE ? NM + 2 : 1];
            float2 rst[T::STORE ? NM + 1 : 1], Gst[T::STORE ? NM + 1 : 1];
            float2 Est[T::STORE ? NM + 2 : 1], Dst[T::STORE ? NM + 1 : 1];
            float2 X[GRAD ? NM + 1 : 1];
            Kz kbelow = medium_kz(p_hi, p_lo, sm.c[n + 1], sm.a[n + 1]);
            float2 Xbelow = make_float2(0.f, 0.f);
            auto fwd_step = [&](int j) __attribute__((always_inline)) {
                Kz kj;
                if (j == 0) {
                    kj.re = k0h; kj.im = 0.f; kj.lo = k0l;
                } else {
                    kj = medium_kz(p_hi, p_lo, sm.c[j], sm.a[j]);
                }
                float2 Gj;
                const float2 rj = fresnel_nc(kc(kj), kc(kbelow), sm.N[j], sm.s[j], Gj);
                float2 Xj;
                if (j == n) {
                    Xj = rj;
                    if constexpr (T::STORE) kst[j + 1] = kbelow;
                } else {
                    const float2 Ej = layer_phase(kbelow, sm.d[j + 1]);
                    float2 Dj;
                    Xj = mobius(rj, cmul(Xbelow, Ej), Dj);
                    if constexpr (T::STORE) { Est[j + 1] = Ej; Dst[j] = Dj; }
                }
                if constexpr (T::STORE) { kst[j] = kj; rst[j] = rj; Gst[j] = Gj; }
                if constexpr (GRAD) X[j] = Xj;
                Xbelow = Xj;
                kbelow = kj;
            };
            if constexpr (T::UNROLL) {
#pragma unroll
                for (int j = NM; j >= 0; --j)
                    if (j <= n) fwd_step(j);
            } else {
#pragma unroll 1
                for (int j = n; j >= 0; --j) fwd_step(j);
            }
            float R = Xbelow.x * Xbelow.x + Xbelow.y * Xbelow.y;
            if (!qok) R = __int_as_float(0x7fffffff);

            // a8-a10: smearing sum per Q point (kSubLanes lanes each), model,
            // likelihood, adjoint seed
            sh_wR[buf][tid] = act ? wk * R : 0.f;
            __syncthreads();
            if (warp < qwarps) {
                float S = 0.f;
                if (qlane)
                    for (int k = qpart; k < K; k += kSubLanes) S += sh_wR[buf][qgrp * K + k];
                S += __shfl_xor_sync(0xffffffffu, S, 1);
                S += __shfl_xor_sync(0xffffffffu, S, 2);
                const int qj = q0 + qgrp;
                if (qlane && qpart == 0) {
                    float seed = 0.f;
                    if (qj < wi.q_hi) {
                        const float m = fmaf(scale, S, bkg);
                        if constexpr (MODE == kModel) {
                            ka.r_out[si.out_off + qj] = m;
                        } else {
                            const float res = (m - Ro) * ie;
                            float t1, t2;
                            two_sum(ll_hi, fmaf(res, res, lterm), t1, t2);
                            ll_hi = t1;
                            ll_lo += t2;
                            if constexpr (GRAD) {
                                const float dldm = -res * ie;
                                gsc_acc = fmaf(dldm, S, gsc_acc);
                                gbk_acc += dldm;
                                seed = scale * dldm;
                            }
                        }
                    }
                    if constexpr (GRAD) sh_seed[buf][qgrp] = seed;
                }
            }
            if constexpr (GRAD) {
                __syncthreads();
                const float Rb = act ? wk * sh_seed[buf][qslot] : 0.f;

                // a7: adjoint sweep from the fronting down to the backing
                float2 Xb = cscale(X[0], 2.f * Rb);
                float2 kbar = make_float2(0.f, 0.f); // adjoint of k_j (j >= 1)
                Kz kj;
                kj.re = k0h; kj.im = 0.f; kj.lo = k0l;
                Kz kjm1 = kj;                          // k_{j-1}
                float2 Xb_up = make_float2(0.f, 0.f);  // adjoint of X_{j-1}
                const float edge_u = kEdgeFrac * k0h * k0h;
                // deferred guard inputs (1-layer bucket: only medium 1 can be interior)
                bool edge_pending = false;
                float2 e_a, e_k, e_b, e_Z, e_Xb;
                auto adj_step = [&](int j) __attribute__((always_inline)) {
                    const float2 Xb_in = Xb;
                    float2 Zj = make_float2(0.f, 0.f);
                    Kz kj1;
                    float2 rj, Gj;
                    if constexpr (T::STORE) {
                        kj1 = kst[j + 1];
                        rj = rst[j];
                        Gj = Gst[j];
                    } else {
                        kj1 = medium_kz(p_hi, p_lo, sm.c[j + 1], sm.a[j + 1]);
                        rj = fresnel_nc(kc(kj), kc(kj1), sm.N[j], sm.s[j], Gj);
                    }
                    float2 kbar1 = make_float2(0.f, 0.f);
                    float2 rb;
                    if (j < n) {
                        float2 Ej1, Dj, Y;
                        if constexpr (T::STORE) {
                            Ej1 = Est[j + 1];
                            Dj = Dst[j];
                            Y = cmul(X[j + 1], Ej1);
                        } else {
                            Ej1 = layer_phase(kj1, sm.d[j + 1]);
                            Y = cmul(X[j + 1], Ej1);
                            const float2 rY = cmul(rj, Y);
                            const float dx = 1.f + rY.x, dy = rY.y;
                            const float inv = rcp_approx(fmaf(dx, dx, dy * dy));
                            Dj = make_float2(dx * inv, -dy * inv);
                        }
                        Zj = Y;
                        const float2 D2 = csqr(Dj);
                        const float2 one = make_float2(1.f, 0.f);
                        const float2 dXdr = cmul(csub(one, csqr(Y)), D2);
                        const float2 dXdY = cmul(csub(one, csqr(rj)), D2);
                        rb = cmulc(dXdr, Xb);
                        const float2 Yb = cmulc(dXdY, Xb);
                        const float2 Eb = cmulc(X[j + 1], Yb);
                        const float2 Xb1 = cmulc(Ej1, Yb);
                        const float2 iE = make_float2(-Ej1.y, Ej1.x);
                        acc_add(oD + j, redot(Eb, cmul(kc(kj1), iE)));           // d_{j+1}
                        kbar1 = cscale(cmulc(iE, Eb), 2.f * sm.d[j + 1].x);
                        Xb = Xb1;
                    } else {
                        rb = Xb;
                    }
                    const float2 T1 = cscale(Gj, 2.f);
                    const float2 T2 = cscale(rj, sm.s[j]);
                    const float2 dr_dkj = cmul(kc(kj1), cadd(T1, T2));
                    const float2 dr_dkj1 = cmul(kc(kj), csub(T2, T1));
                    kbar1 = cadd(kbar1, cmulc(dr_dkj1, rb));
                    acc_add(oS + j, redot(rb, cmul(rj, cmul(kc(kj), kc(kj1)))));
                    if (j >= 1) {
                        kbar = cadd(kbar, cmulc(dr_dkj, rb));
                        // k_j complete: accumulate conj(kbar) / k_j
                        const float m2 = fmaf(kj.re, kj.re, kj.im * kj.im);
                        if (m2 < edge_u) {
                            // interior critical edge: conj(kbar)/k_j = 2 conj(ubar)
                            if constexpr (T::EDGE_DEFER) {
                                edge_pending = true;
                                e_a = kc(kjm1); e_k = kc(kj); e_b = kc(kj1); e_Z = Zj; e_Xb = Xb_up;
                            } else {
                                const float2 ub = edge_ubar_call(kc(kjm1), kc(kj), kc(kj1), sm.sg[j - 1],
                                                                 sm.sg[j], sm.d[j].x, Zj, Xb_up);
                                acc_add(oUr + j - 1, 2.f * ub.x);
                                acc_add(oUi + j - 1, -2.f * ub.y);
                            }
                        } else {
                            const float2 kk = cmul(kbar, kc(kj));
                            const float inv = m2 > 0.f ? rcp_approx(m2) : 0.f;
                            acc_add(oUr + j - 1, kk.x * inv);
                            acc_add(oUi + j - 1, -kk.y * inv);
                        }
                    }
                    Xb_up = Xb_in;
                    kbar = kbar1;
                    kjm1 = kj;
                    kj = kj1;
                    if (j == n) { // backing medium n+1: its k is complete as well
                        const float2 kk = cmul(kbar, kc(kj));
                        const float m2 = fmaf(kj.re, kj.re, kj.im * kj.im);
                        const float inv = m2 > 0.f ? rcp_approx(m2) : 0.f;
                        acc_add(oUr + j, kk.x * inv);
                        acc_add(oUi + j, -kk.y * inv);
                    }
                };
                if constexpr (T::UNROLL) {
#pragma unroll
                    for (int j = 0; j <= NM; ++j)
                        if (j <= n) adj_step(j);
                } else {
#pragma unroll 1
                    for (int j = 0; j <= n; ++j) adj_step(j);
                }
                if constexpr (T::EDGE_DEFER) {
                    if (edge_pending) {
                        const float2 ub = edge_ubar_inline(e_a, e_k, e_b, sm.sg[0], sm.sg[1], sm.d[1].x, e_Z, e_Xb);
                        acc_add(oUr + 0, 2.f * ub.x);
                        acc_add(oUi + 0, -2.f * ub.y);
                    }
                }
            }
            // no end-of-tile barrier: the next tile uses the other buffers
        }

        if constexpr (LIK) {
            // ---- CTA reduction of the item's partial sums into sh_raw ----
            __syncthreads();
            if constexpr (GRAD && !T::SMEM_ACC) {
                static_assert(T::NACC <= 32, "register partials exceed one reduction batch");
#pragma unroll
                for (int t = 0; t < T::NACC; ++t) {
                    float v = accr[t];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
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
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
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
            if (warp < qwarps) {   // loglik, d/dscale, d/dbkg live in the per-Q lanes
                double a0 = (double)ll_hi + (double)ll_lo, a1 = gsc_acc, a2 = gbk_acc;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
                    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
                    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
                }
                if (lane == 0) {
                    sh_redd[warp][0] = a0;
                    sh_redd[warp][1] = a1;
                    sh_redd[warp][2] = a2;
                }
            }
            __syncthreads();
            if (tid < 3) {
                double s = 0.0;
                for (int w = 0; w < qwarps; ++w) s += sh_redd[w][tid];
                sh_raw[4 * n + 3 + tid] = s;
            }
            __syncthreads();
            const int nout = GRAD ? 4 * n + 6 : 1;
            const int off0 = GRAD ? 0 : 4 * n + 3; // loglik mode: llsum only
            if (si.n_chunks == 1) {
                finalize_stack<MODE>(sh_raw, n, p, wi.stack, si.par_off, ka.ll_out, ka.grad_out, tid,
                                     BLOCK);
            } else {
                double *slot = ka.partials + si.part_base + (int64_t)wi.chunk * (4 * n + 6);
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
                            s += __ldcg(ka.partials + si.part_base + (int64_t)c * (4 * n + 6) + off0 + i);
                        sh_raw[off0 + i] = s;
                    }
                    __syncthreads();
                    finalize_stack<MODE>(sh_raw, n, p, wi.stack, si.par_off, ka.ll_out, ka.grad_out,
                                         tid, BLOCK);
                    if (tid == 0) ka.stack_done[wi.stack] = 0;
                }
            }
        }
        __syncthreads(); // sm / sh_raw / sh_item reused by the next item
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

template <int MODE, int NMAX>
cudaError_t launch_one(int grid, const KernelArgs &a, const QuadConst &qc, cudaStream_t st)
{
    using T = Traits<MODE, NMAX>;
    const size_t dyn = T::SMEM_ACC ? (size_t)T::NACC * T::BLOCK * sizeof(float) : 0;
    static bool attr_done = false; // per-process; the attribute is per function
    if (!attr_done && dyn > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(nr_mixed_kernel<MODE, NMAX>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    nr_mixed_kernel<MODE, NMAX><<<grid, T::BLOCK, dyn, st>>>(a, qc);
    return cudaGetLastError();
}

template <int MODE, int NMAX>
cudaError_t occupancy_one(int *blocks)
{
    using T = Traits<MODE, NMAX>;
    const size_t dyn = T::SMEM_ACC ? (size_t)T::NACC * T::BLOCK * sizeof(float) : 0;
    if (dyn > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(nr_mixed_kernel<MODE, NMAX>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, nr_mixed_kernel<MODE, NMAX>, T::BLOCK,
                                                         dyn);
}

#define NR_GRAD_BUCKETS(X) X(1) X(2) X(4) X(8) X(12) X(16) X(20) X(32) X(64)

} // namespace

bool mixed_bucket_ok(int mode, int nmax)
{
    if (mode == kGrad) {
#define X(B) if (nmax == B) return true;
        NR_GRAD_BUCKETS(X)
#undef X
        return false;
    }
    return nmax == 0 || nmax == 1;
}

int mixed_block_threads(int mode, int nmax)
{
    return mode != kGrad ? 256 : nmax >= 32 ? 128 : 256;
}

size_t mixed_dyn_smem(int mode, int nmax)
{
    if (mode != kGrad || nmax < 8) return 0;
    return (size_t)(4 * nmax + 3) * mixed_block_threads(mode, nmax) * sizeof(float);
}

cudaError_t mixed_occupancy(int mode, int nmax, int *blocks)
{
    switch (mode) {
    case kModel:
        return nmax == 1 ? occupancy_one<kModel, 1>(blocks) : occupancy_one<kModel, 0>(blocks);
    case kLoglik:
        return nmax == 1 ? occupancy_one<kLoglik, 1>(blocks) : occupancy_one<kLoglik, 0>(blocks);
    default:
#define X(B) if (nmax == B) return occupancy_one<kGrad, B>(blocks);
        NR_GRAD_BUCKETS(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_mixed(int mode, int nmax, int grid, const KernelArgs &a, const QuadConst &qc,
                         cudaStream_t st)
{
    switch (mode) {
    case kModel:
        return nmax == 1 ? launch_one<kModel, 1>(grid, a, qc, st) : launch_one<kModel, 0>(grid, a, qc, st);
    case kLoglik:
        return nmax == 1 ? launch_one<kLoglik, 1>(grid, a, qc, st)
                         : launch_one<kLoglik, 0>(grid, a, qc, st);
    default:
#define X(B) if (nmax == B) return launch_one<kGrad, B>(grid, a, qc, st);
        NR_GRAD_BUCKETS(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

} // namespace nrimpl
