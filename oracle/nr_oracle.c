/*
 * nr_oracle.c -- TEST INFRASTRUCTURE ONLY: the plain, slow CPU oracle for the
 * batched neutron-reflectivity forward model, its Gaussian log-likelihood and
 * the exact gradient of that log-likelihood.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg load
 * this file (through oracle/__init__.py).  It shares no code, header, table
 * or constant with the CUDA library; it is compiled by gcc only.
 *
 * Precision: `double` by default; compiled with -DNR_ORACLE_LONG it runs the
 * same source in `long double` (80-bit on x86-64, binary128 on aarch64), the
 * reference the tests use for the double build itself.
 *
 * What it computes (arXiv 2509.06924):
 *  - slab model theta = {thick, SLD, rough, scale, bkg} of the refjax
 *    parameter dictionary (Sec. 3), extended with an absorption (imaginary
 *    SLD) per layer and for the backing medium;
 *  - reflectivity by the Abeles characteristic-matrix formalism named in
 *    Sec. 2.1, with Gaussian interfacial roughness (Sec. 3 dictionary,
 *    supplement Sec. S2 figure caption) taken in the Nevot-Croce form;
 *  - Gaussian resolution smearing in Q with a pointwise FWHM dQ (Sec. 3
 *    smearing kernels, Sec. 4.1 "pointwise FWHM"), evaluated by K-point
 *    Gauss-Hermite quadrature;
 *  - model m = scale * S + bkg (theta_NR of Sec. 2.1; Tables 2 and 4);
 *  - Gaussian likelihood with per-point standard deviations (Sec. 2.1,
 *    text after Eq. 2), whose data term is the chi^2 of Eq. 25:
 *      loglik = -1/2 sum_i [ ((m_i - R_i)/e_i)^2 + ln(2 pi e_i^2) ];
 *  - the gradient of loglik w.r.t. every packed parameter, by forward-mode
 *    dual numbers (one pass per parameter), the exact derivative the paper
 *    obtains by automatic differentiation (Sec. 2.1, Fig. 1; Sec. 3);
 *  - the derivative of loglik w.r.t. the resolution, taken as a common scale
 *    f of every dQ_i (dQ_i -> f dQ_i, derivative in ln f at f = 1): the
 *    quantity a fit of a shared smearing percentage needs (Sec. 4.2, the
 *    LED fit's smearing parameter); one more dual pass, seeded on the node
 *    positions, dq_k / d ln f = sqrt(2) sigma_Q x_k;
 *  - the SLD profile of a stack through its depth z, the curve drawn with
 *    posterior bands in the paper's figures (Sec. 4.1 quartz, Sec. 4.2 LED):
 *    rho(z) = rho_0 + sum_j (rho_{j+1} - rho_j) (1 + erf((z - z_j) /
 *    (sqrt(2) sigma_j))) / 2, interface j at depth z_j = d_1 + ... + d_j
 *    (z_0 = 0), each step smoothed by the Gaussian roughness of that
 *    interface; the same for the absorption iota(z).
 *
 * Readings where the paper is silent (the paper prints no reflectivity
 * equation):
 *  - media 0 (fronting) .. n+1 (backing); k_0 = q/2 and, for j >= 1,
 *    k_j = sqrt(k_0^2 - 4 pi (rho_j - rho_0) + 4 pi i iota_j), principal
 *    root (Im k_j >= 0), time factor exp(-i omega t);
 *  - r_j = (k_j - k_{j+1}) / (k_j + k_{j+1}) * exp(-2 k_j k_{j+1} sigma_j^2),
 *    sigma_j the roughness of the interface below medium j;
 *  - Abeles: beta_0 = 0, beta_j = k_j d_j,
 *    C_j = [[e^{-i b}, r_j e^{-i b}], [r_j e^{i b}, e^{i b}]],
 *    M = C_0 C_1 ... C_n, amplitude r = M_10 / M_00, R = |r|^2;
 *  - smearing: sigma_Q = dQ / (2 sqrt(2 ln 2)),
 *    S(Q) = sum_k (w_k / sqrt(pi)) R(Q + sqrt(2) sigma_Q x_k), with (x_k, w_k)
 *    the Gauss-Hermite rule for the weight exp(-x^2);
 *  - SLDs are absolute (A^-2, e.g. 2.07e-6 for Si).
 *
 * Packed parameter layout of one stack with n layers (4n+6 values):
 *   d[n] | rho[n+2] (fronting, layers, backing) | iota[n+1] (layers, backing)
 *   | sigma[n+1] (interfaces top to bottom) | scale | bkg
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifdef NR_ORACLE_LONG
typedef long double real;
typedef long double _Complex cplx;
#define R_SQRT sqrtl
#define R_LOG logl
#define R_FABS fabsl
#define R_CBRT cbrtl
#define R_ERF erfl
#define C_SQRT csqrtl
#define C_EXP cexpl
#define C_RE creall
#define C_IM cimagl
#define C_CONJ conjl
#define R_PI 3.141592653589793238462643383279502884L
#define R_LN2 0.693147180559945309417232121458176568L
#else
typedef double real;
typedef double _Complex cplx;
#define R_SQRT sqrt
#define R_LOG log
#define R_FABS fabs
#define R_CBRT cbrt
#define R_ERF erf
#define C_SQRT csqrt
#define C_EXP cexp
#define C_RE creal
#define C_IM cimag
#define C_CONJ conj
#define R_PI 3.141592653589793238462643383279502884
#define R_LN2 0.693147180559945309417232121458176568
#endif

#define ORACLE_MAX_LAYERS 64
#define ORACLE_MAX_QUAD 64

enum { OR_OK = 0, OR_EINVAL = -1, OR_EDOMAIN = -2 };

/* ------------------------------------------------------------------------ */
/* First-order dual numbers over the complex type: value v and the derivative
 * t along one parameter direction.  Each rule below is the textbook
 * derivative of the operation.                                              */
/* ------------------------------------------------------------------------ */
typedef struct { cplx v, t; } dual;

static dual dl(cplx v, cplx t) { dual r; r.v = v; r.t = t; return r; }
static dual dconst(cplx v) { return dl(v, 0); }
static dual dadd(dual a, dual b) { return dl(a.v + b.v, a.t + b.t); }
static dual dsub(dual a, dual b) { return dl(a.v - b.v, a.t - b.t); }
static dual dmul(dual a, dual b) { return dl(a.v * b.v, a.t * b.v + a.v * b.t); }
static dual dscale(dual a, cplx s) { return dl(a.v * s, a.t * s); }
static dual ddiv(dual a, dual b)
{
    cplx q = a.v / b.v;
    return dl(q, (a.t - q * b.t) / b.v);
}
static dual dexp(dual a)
{
    cplx e = C_EXP(a.v);
    return dl(e, e * a.t);
}
/* principal square root; the caller guarantees Im(a.v) >= +0 */
static dual dsqrt(dual a)
{
    cplx s = C_SQRT(a.v);
    return dl(s, s != 0 ? a.t / (2 * s) : 0);
}
/* |a|^2 as a real-valued dual: d|a|^2 = 2 Re(conj(a) da) */
static dual dabs2(dual a)
{
    real v = C_RE(a.v) * C_RE(a.v) + C_IM(a.v) * C_IM(a.v);
    real t = 2 * C_RE(C_CONJ(a.v) * a.t);
    return dl(v, t);
}

/* A stack's parameters as duals (tangent 1 on the seeded parameter). */
typedef struct {
    int n;
    dual d[ORACLE_MAX_LAYERS + 2];     /* d[j], j = 1..n (index 0 unused)       */
    dual rho[ORACLE_MAX_LAYERS + 2];   /* rho[j], j = 0..n+1                    */
    dual iota[ORACLE_MAX_LAYERS + 2];  /* iota[j], j = 0..n+1 (iota[0] = 0)     */
    dual sig[ORACLE_MAX_LAYERS + 1];   /* sigma[j], j = 0..n                    */
    dual scale, bkg;
} stack_t_;

/* Unpack the 4n+6 packed values; `seed` < 0 means no derivative direction. */
static void unpack(int n, const double *p, int seed, stack_t_ *s)
{
    int idx = 0;
    s->n = n;
#define NEXT(dst) do { (dst) = dl((real)p[idx], idx == seed ? 1 : 0); ++idx; } while (0)
    s->d[0] = dconst(0);
    for (int j = 1; j <= n; ++j) NEXT(s->d[j]);
    for (int j = 0; j <= n + 1; ++j) NEXT(s->rho[j]);
    s->iota[0] = dconst(0);
    for (int j = 1; j <= n + 1; ++j) NEXT(s->iota[j]);
    for (int j = 0; j <= n; ++j) NEXT(s->sig[j]);
    NEXT(s->scale);
    NEXT(s->bkg);
#undef NEXT
}

/* z-components of the wavevector in every medium at momentum transfer q
 * (with tangent qt: q itself may carry the derivative direction). */
static void wavevectors(const stack_t_ *s, real q, real qt, dual *k)
{
    const int n = s->n;
    real k0 = q / 2, k0t = qt / 2;
    k[0] = dl(k0, k0t);
    for (int j = 1; j <= n + 1; ++j) {
        /* k0^2 - 4 pi (rho_j - rho_0) + 4 pi i iota_j ; adding +0.0 to the
         * imaginary part turns a -0.0 into +0.0 so that csqrt stays on the
         * principal branch for non-absorbing media. */
        dual drho = dsub(s->rho[j], s->rho[0]);
        cplx re_v = k0 * k0 - 4 * R_PI * C_RE(drho.v);
        real im_v = 4 * R_PI * C_RE(s->iota[j].v) + (real)0.0;
        cplx v = re_v + im_v * I;
        cplx t = 2 * k0 * k0t - 4 * R_PI * drho.t + 4 * R_PI * s->iota[j].t * I;
        k[j] = dsqrt(dl(v, t));
    }
}

/* Fresnel coefficient of interface j with Nevot-Croce roughness. */
static dual fresnel(const stack_t_ *s, const dual *k, int j)
{
    dual num = dsub(k[j], k[j + 1]);
    dual den = dadd(k[j], k[j + 1]);
    if (den.v == 0) return dconst(0); /* both media at k = 0: identical media */
    dual r0 = ddiv(num, den);
    /* exp(-2 k_j k_{j+1} sigma_j^2) */
    dual s2 = dmul(s->sig[j], s->sig[j]);
    dual arg = dscale(dmul(dmul(k[j], k[j + 1]), s2), -2);
    return dmul(r0, dexp(arg));
}

/* Complex reflection amplitude of the stack at q.
 * form 0: Abeles characteristic-matrix product (the definition);
 * form 1: Parratt recursion from the backing upwards (cross-check). */
static dual amplitude(const stack_t_ *s, real q, real qt, int form)
{
    const int n = s->n;
    dual k[ORACLE_MAX_LAYERS + 2];
    dual r[ORACLE_MAX_LAYERS + 1];
    wavevectors(s, q, qt, k);
    for (int j = 0; j <= n; ++j) r[j] = fresnel(s, k, j);

    if (form == 0) {
        dual M00 = dconst(1), M01 = dconst(0), M10 = dconst(0), M11 = dconst(1);
        for (int j = 0; j <= n; ++j) {
            dual beta = (j == 0) ? dconst(0) : dmul(k[j], s->d[j]);
            dual em = dexp(dscale(beta, -I)); /* e^{-i beta} */
            dual ep = dexp(dscale(beta, I));  /* e^{+i beta} */
            dual C00 = em, C01 = dmul(r[j], em), C10 = dmul(r[j], ep), C11 = ep;
            dual N00 = dadd(dmul(M00, C00), dmul(M01, C10));
            dual N01 = dadd(dmul(M00, C01), dmul(M01, C11));
            dual N10 = dadd(dmul(M10, C00), dmul(M11, C10));
            dual N11 = dadd(dmul(M10, C01), dmul(M11, C11));
            M00 = N00; M01 = N01; M10 = N10; M11 = N11;
        }
        return ddiv(M10, M00);
    }
    /* Parratt: X_n = r_n; X_j = (r_j + X_{j+1} E_{j+1}) / (1 + r_j X_{j+1} E_{j+1}),
     * E_j = exp(2 i k_j d_j). */
    dual X = r[n];
    for (int j = n - 1; j >= 0; --j) {
        dual E = dexp(dscale(dmul(k[j + 1], s->d[j + 1]), 2 * I));
        dual Y = dmul(X, E);
        X = ddiv(dadd(r[j], Y), dadd(dconst(1), dmul(r[j], Y)));
    }
    return X;
}

/* ------------------------------------------------------------------------ */
/* Gauss-Hermite rule for the weight exp(-x^2): nodes are the roots of the
 * degree-K Hermite polynomial, found by scanning for sign changes and
 * bisecting, then polished by Newton; weights are the Christoffel numbers
 * 1 / sum_{j<K} psi_j(x)^2 of the orthonormal Hermite polynomials psi_j.   */
/* ------------------------------------------------------------------------ */
/* psi_0 .. psi_K at x (orthonormal w.r.t. exp(-x^2)); returns psi_K, writes
 * psi_K'(x) = sqrt(2K) psi_{K-1}(x) and sum_{j<K} psi_j^2. */
static real hermite_orthonormal(int K, real x, real *deriv, real *christoffel_sum)
{
    real pm1 = 0, p = 1 / R_SQRT(R_SQRT(R_PI)), sum = 0;
    for (int j = 0; j < K; ++j) {
        sum += p * p;
        real pn = x * R_SQRT((real)2 / (j + 1)) * p - R_SQRT((real)j / (j + 1)) * pm1;
        pm1 = p;
        p = pn;
    }
    if (deriv) *deriv = R_SQRT((real)2 * K) * pm1;
    if (christoffel_sum) *christoffel_sum = sum;
    return p;
}

static int gauss_hermite(int K, real *x, real *w)
{
    if (K < 1 || K > ORACLE_MAX_QUAD) return OR_EINVAL;
    const real lim = R_SQRT((real)2 * K + 1) + 1; /* all roots lie inside */
    const int grid = 40001; /* odd: x = 0 (a root for odd K) is never a grid point */
    int found = 0;
    real xa = -lim, fa = hermite_orthonormal(K, xa, NULL, NULL);
    for (int g = 1; g <= grid && found < K; ++g) {
        real xb = -lim + 2 * lim * g / grid;
        real fb = hermite_orthonormal(K, xb, NULL, NULL);
        if ((fa < 0) != (fb < 0)) {
            real lo = xa, hi = xb, flo = fa;
            for (int it = 0; it < 200; ++it) {
                real mid = (lo + hi) / 2;
                if (mid == lo || mid == hi) break;
                real fm = hermite_orthonormal(K, mid, NULL, NULL);
                if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else { hi = mid; }
            }
            real root = (lo + hi) / 2;
            for (int it = 0; it < 3; ++it) { /* Newton polish */
                real dp, f = hermite_orthonormal(K, root, &dp, NULL);
                if (dp != 0) root -= f / dp;
            }
            x[found++] = root;
        }
        xa = xb;
        fa = fb;
    }
    if (found != K) return OR_EDOMAIN;
    for (int i = 0; i < K; ++i) {
        real cs;
        hermite_orthonormal(K, x[i], NULL, &cs);
        w[i] = 1 / cs;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Smeared model, likelihood, gradient.                                     */
/* ------------------------------------------------------------------------ */
typedef struct { int K; real x[ORACLE_MAX_QUAD]; real w[ORACLE_MAX_QUAD]; } quad_t_;

static int make_quad(int K, quad_t_ *qd)
{
    qd->K = K;
    return gauss_hermite(K, qd->x, qd->w);
}

/* m(Q) = scale * S(Q) + bkg as a real-valued dual.  res_seed: the tangent
 * is the derivative in ln f of the resolution scale f (dQ -> f dQ, f = 1). */
static int smeared_model(const stack_t_ *s, real Q, real dQ, const quad_t_ *qd, int form, int res_seed,
                         dual *m)
{
    dual S = dconst(0);
    if (dQ == 0) {
        if (!(Q > 0)) return OR_EDOMAIN;
        S = dabs2(amplitude(s, Q, 0, form));
    } else {
        real sigQ = dQ / (2 * R_SQRT(2 * R_LN2));
        for (int k = 0; k < qd->K; ++k) {
            real step = R_SQRT((real)2) * sigQ * qd->x[k];
            real qk = Q + step;
            if (!(qk > 0)) return OR_EDOMAIN;
            dual R = dabs2(amplitude(s, qk, res_seed ? step : 0, form));
            S = dadd(S, dscale(R, qd->w[k] / R_SQRT(R_PI)));
        }
    }
    *m = dadd(dmul(s->scale, S), s->bkg);
    return OR_OK;
}

static int loglik_dual(const stack_t_ *s, int nq, const double *Q, const double *dQ,
                       const double *Robs, const double *err, const quad_t_ *qd, int res_seed, dual *ll)
{
    dual acc = dconst(0);
    for (int i = 0; i < nq; ++i) {
        if (!(err[i] > 0)) return OR_EDOMAIN;
        dual m;
        int st = smeared_model(s, Q[i], dQ[i], qd, 0, res_seed, &m);
        if (st) return st;
        real e = err[i];
        dual res = dscale(dsub(m, dconst(Robs[i])), 1 / e);
        dual term = dadd(dmul(res, res), dconst(R_LOG(2 * R_PI * e * e)));
        acc = dadd(acc, term);
    }
    *ll = dscale(acc, -0.5);
    return OR_OK;
}

static int check_stack(int n, const double *p)
{
    if (n < 0 || n > ORACLE_MAX_LAYERS) return OR_EINVAL;
    for (int i = 0; i < 4 * n + 6; ++i)
        if (!isfinite(p[i])) return OR_EINVAL;
    return OR_OK;
}

/* ======================================================================== */
/* Exported entry points (all arrays are host memory, doubles).             */
/* ======================================================================== */

int oracle_real_bytes(void) { return (int)sizeof(real); }

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Gauss-Hermite nodes and weights for exp(-x^2). */
int oracle_gauss_hermite(int K, double *x, double *w)
{
    real xr[ORACLE_MAX_QUAD], wr[ORACLE_MAX_QUAD];
    int st = gauss_hermite(K, xr, wr);
    if (st) return st;
    for (int i = 0; i < K; ++i) { x[i] = (double)xr[i]; w[i] = (double)wr[i]; }
    return OR_OK;
}

/* Unsmeared complex amplitude r(q) of one stack (form 0 Abeles, 1 Parratt). */
int oracle_amplitude(int n, const double *params, int nq, const double *q, int form,
                     double *re, double *im)
{
    if (check_stack(n, params)) return OR_EINVAL;
    stack_t_ s;
    unpack(n, params, -1, &s);
    for (int i = 0; i < nq; ++i) {
        if (!(q[i] > 0)) return OR_EDOMAIN;
        dual r = amplitude(&s, q[i], 0, form);
        re[i] = (double)C_RE(r.v);
        im[i] = (double)C_IM(r.v);
    }
    return OR_OK;
}

/* Derivative of the unsmeared reflectivity R(q) = |r|^2 w.r.t. packed
 * parameter `seed`, together with R itself. */
int oracle_reflectivity_unsmeared_d(int n, const double *params, int nq, const double *q,
                                    int seed, double *R, double *dR)
{
    if (check_stack(n, params)) return OR_EINVAL;
    stack_t_ s;
    unpack(n, params, seed, &s);
    for (int i = 0; i < nq; ++i) {
        if (!(q[i] > 0)) return OR_EDOMAIN;
        dual v = dabs2(amplitude(&s, q[i], 0, 0));
        R[i] = (double)C_RE(v.v);
        if (dR) dR[i] = (double)C_RE(v.t);
    }
    return OR_OK;
}

/* Smeared model m_i = scale * S(Q_i) + bkg of one stack; form as above. */
int oracle_model(int n, const double *params, int nq, const double *Q, const double *dQ,
                 int K, int form, double *m)
{
    if (check_stack(n, params)) return OR_EINVAL;
    quad_t_ qd;
    if (make_quad(K, &qd)) return OR_EINVAL;
    stack_t_ s;
    unpack(n, params, -1, &s);
    for (int i = 0; i < nq; ++i) {
        dual v;
        int st = smeared_model(&s, Q[i], dQ[i], &qd, form, 0, &v);
        if (st) return st;
        m[i] = (double)C_RE(v.v);
    }
    return OR_OK;
}

/* Log-likelihood of one stack, and (if grad != NULL) its gradient w.r.t.
 * all 4n+6 packed parameters by one dual pass per parameter. */
int oracle_loglik_grad(int n, const double *params, int nq, const double *Q, const double *dQ,
                       const double *Robs, const double *err, int K, double *ll, double *grad)
{
    if (check_stack(n, params)) return OR_EINVAL;
    quad_t_ qd;
    if (make_quad(K, &qd)) return OR_EINVAL;
    stack_t_ s;
    dual v;
    unpack(n, params, -1, &s);
    int st = loglik_dual(&s, nq, Q, dQ, Robs, err, &qd, 0, &v);
    if (st) return st;
    *ll = (double)C_RE(v.v);
    if (grad) {
        for (int p = 0; p < 4 * n + 6; ++p) {
            unpack(n, params, p, &s);
            st = loglik_dual(&s, nq, Q, dQ, Robs, err, &qd, 0, &v);
            if (st) return st;
            grad[p] = (double)C_RE(v.t);
        }
    }
    return OR_OK;
}

/* d loglik / d ln f of one stack, f a common scale of every dQ_i (f = 1). */
int oracle_loglik_grad_res(int n, const double *params, int nq, const double *Q, const double *dQ,
                           const double *Robs, const double *err, int K, double *gres)
{
    if (check_stack(n, params)) return OR_EINVAL;
    quad_t_ qd;
    if (make_quad(K, &qd)) return OR_EINVAL;
    stack_t_ s;
    dual v;
    unpack(n, params, -1, &s);
    int st = loglik_dual(&s, nq, Q, dQ, Robs, err, &qd, 1, &v);
    if (st) return st;
    *gres = (double)C_RE(v.t);
    return OR_OK;
}

/* SLD and absorption profiles of one stack at nz depths z (A); either output
 * may be NULL.  sigma_j = 0 gives the sharp step (value of the deeper medium
 * at z = z_j itself, the erf's sign convention at 0). */
int oracle_sld_profile(int n, const double *params, int nz, const double *z, double *rho, double *iota)
{
    if (check_stack(n, params)) return OR_EINVAL;
    const double *d = params, *r = params + n, *io = params + 2 * n + 2, *sg = params + 3 * n + 3;
    for (int i = 0; i < nz; ++i) {
        real zr = (real)z[i], depth = 0, vr = (real)r[0], vi = 0;
        for (int j = 0; j <= n; ++j) {
            if (j >= 1) depth += (real)d[j - 1];
            real step;
            if (sg[j] > 0) step = (1 + R_ERF((zr - depth) / (R_SQRT((real)2) * (real)sg[j]))) / 2;
            else step = zr >= depth ? 1 : 0;
            real io_j = j >= 1 ? (real)io[j - 1] : 0, io_j1 = (real)io[j];
            vr += ((real)r[j + 1] - (real)r[j]) * step;
            vi += (io_j1 - io_j) * step;
        }
        if (rho) rho[i] = (double)vr;
        if (iota) iota[i] = (double)vi;
    }
    return OR_OK;
}

/* Batch driver over many stacks (OpenMP over stacks when available).
 * mode 0: smeared model into out_m (offsets: prefix over stacks of the
 *         dataset lengths); mode 1: loglik; mode 2: loglik and gradient
 *         (packed like params); mode 3: loglik, gradient and, in out_m (one
 *         value per stack), d loglik / d ln f of the resolution scale.
 *         Returns 0, or the first failing status. */
int oracle_batch(int mode, int n_stacks, const int32_t *n_layers, const double *params,
                 const int32_t *dataset, int n_datasets, const int64_t *q_off,
                 const double *Q, const double *dQ, const double *Robs, const double *err,
                 int K, int n_threads, double *out_m, double *out_ll, double *out_grad)
{
    if (n_stacks < 0 || n_datasets < 0) return OR_EINVAL;
    int64_t *par_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_stacks + 1));
    int64_t *out_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_stacks + 1));
    if (!par_off || !out_off) { free(par_off); free(out_off); return OR_EINVAL; }
    par_off[0] = 0;
    out_off[0] = 0;
    int bad = 0;
    for (int s = 0; s < n_stacks; ++s) {
        if (n_layers[s] < 0 || n_layers[s] > ORACLE_MAX_LAYERS) bad = 1;
        if (dataset[s] < 0 || dataset[s] >= n_datasets) { bad = 1; break; }
        par_off[s + 1] = par_off[s] + 4 * (int64_t)n_layers[s] + 6;
        out_off[s + 1] = out_off[s] + (q_off[dataset[s] + 1] - q_off[dataset[s]]);
    }
    if (bad) { free(par_off); free(out_off); return OR_EINVAL; }
    int status = OR_OK;
#ifdef _OPENMP
    /* a thread count for this call only (a global setting would outlive it) */
    const int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (int s = 0; s < n_stacks; ++s) {
        const int n = n_layers[s];
        const double *p = params + par_off[s];
        const int64_t q0 = q_off[dataset[s]];
        const int nq = (int)(q_off[dataset[s] + 1] - q0);
        int st;
        if (mode == 0) {
            st = oracle_model(n, p, nq, Q + q0, dQ + q0, K, 0, out_m + out_off[s]);
        } else {
            st = oracle_loglik_grad(n, p, nq, Q + q0, dQ + q0, Robs + q0, err + q0, K,
                                    out_ll + s, mode >= 2 ? out_grad + par_off[s] : NULL);
            if (!st && mode == 3)
                st = oracle_loglik_grad_res(n, p, nq, Q + q0, dQ + q0, Robs + q0, err + q0, K, out_m + s);
        }
        if (st) {
#ifdef _OPENMP
#pragma omp critical
#endif
            status = st;
        }
    }
    free(par_off);
    free(out_off);
    return status;
}
