/*
 * tf_oracle.c -- plain, slow CPU oracle for the twofold exp/log library.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, __graft_entry__.smoke() and
 * the CPU-baseline leg of bench.py may load this library.  The product path
 * (the CUDA kernels behind tf_*) never calls it and shares no code with it.
 *
 * What it computes is the plain definition of a twofold function, written in
 * IEEE binary128 (_Float128) with glibc's binary128 libm as the library step:
 *
 *   For a twofold argument x = x0 + x1 the twofold result z0 + z1 approximates
 *   f(x0 + x1); the main part z0 is f(x0) rounded to double, and z1 assesses
 *   the deviation f(x0 + x1) - z0 (paper, "Twofold exponent" > "Method
 *   summary"; "Twofold logarithm" > "Newton inversion", last part).  The main
 *   part must be the correctly rounded f(x0) (read: the standard library the
 *   paper wants z0 to reproduce bitwise is taken to be a correctly rounded one).
 *
 *   For tadd/tmul the main part is the plain floating-point operation on x0 and
 *   y0 (paper, "Overview": z0 = x0 (+) y0 equals the ordinary sum) and z1
 *   assesses the deviation from the exact sum or product of the twofolds.
 *
 * Per element the oracle returns
 *   Z0    : f(x0) rounded to nearest double (ties to even, IEEE subnormals/overflow),
 *           or to nearest float for float twofolds (tfo_eval2 with f32 = 1),
 *   G     : the ideal deviation F - Z0, F = f(x0 + x1), as a pair of doubles
 *           Gh + Gl (about 106 bits of G),
 *   A     : |F| rounded to double (the scale for relative errors),
 *   flags : FL_AMBIG if f(x0) lies within 2^-50 ulp of a rounding midpoint (the
 *           binary128 value cannot be trusted to decide Z0; the Python side
 *           re-decides these with a 250-bit decimal evaluation), FL_EXACT if
 *           z1 is fixed by the special-value rules below and Gh holds it exactly.
 *
 * F is formed without rounding x0 + x1 (which alone would cost up to
 * |x| 2^-113 ~ 2^-103.5 relative for exp):
 *   exp   : F = e^x0 + e^x0 * expm1(x1)
 *   expm1 : F = expm1(x0) + e^x0 * expm1(x1)
 *   log   : F = log(y0) + log1p(y1 / y0)
 *   log1p : F = log1p(y0) + log1p(y1 / (1 + y0))
 *   add   : F = (x0 + y0) + (x1 + y1)         (binary128, see ox_add)
 *   mul   : F = (x0 + x1) (y0 + y1)           (binary128, see ox_mul)
 *
 * Special values (the paper's "avoid NaN when z0 = v0 = infinity" remark in
 * the texp/texpm1 algorithm summary, and "Domain errors" after the tlog
 * algorithms, read as follows):
 *   - NaN x0, or x0 outside the domain of log/log1p: z0 = z1 = NaN.
 *   - NaN x1 (y1) with a numeric z0: z1 = NaN.
 *   - z0 = +-Inf (overflow, infinite argument, log(0), log1p(-1)), or z0 = 0
 *     from exp underflow / exp(-Inf), or expm1(-Inf) = -1: z1 = 0.
 *   - x1 = +Inf: z1 = +Inf (exp, expm1, log, log1p); x1 = -Inf: F = 0 (exp),
 *     F = -1 (expm1), NaN (log, log1p).
 *   - A twofold log argument with y0 + y1 < 0 gives z1 = NaN, = 0 gives -Inf.
 *
 * Build: gcc -O2 -fPIC -shared -ffp-contract=off -fno-fast-math
 *        -frounding-math [-fopenmp] tf_oracle.c -lm
 * (-ffp-contract=off matters: GCC contracts a*b+c into an FMA by default on
 * aarch64, which would change the plain double tadd/tmul main parts.)
 */
#define _GNU_SOURCE 1
/* TFO_PLANT=k compiles a deliberately wrong oracle (k = 1..10) so that the tests
   can show their pins catch that kind of mistake.  Never set in normal builds. */
#ifndef TFO_PLANT
#define TFO_PLANT 0
#endif
#define __STDC_WANT_IEC_60559_TYPES_EXT__ 1
#include <math.h>
#include <float.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef _Float128 Q;

enum { K_EXP = 0, K_EXPM1 = 1, K_LOG = 2, K_LOG1P = 3, K_ADD = 4, K_MUL = 5 };
enum { FL_AMBIG = 1u, FL_EXACT = 2u };


static Q qabs(Q a) { return a < 0 ? -a : a; }

/* Round a binary128 value to the nearest double and flag values that lie within
 * 2^-50 of a double spacing from a rounding midpoint. */
static double rn_double(Q F, int *ambig)
{
#if TFO_PLANT == 4
    double d = (double)F;           /* planted: round toward zero instead of to nearest */
    if (isfinite(d) && qabs((Q)d) > qabs(F)) d = nextafter(d, 0.0);
#else
    double d = (double)F;           /* one IEEE rounding (subnormal and overflow aware) */
#endif
    *ambig = 0;
    if (isnan(d) || isinf(F))
        return d;
    Q a = qabs(F);
    if (a == 0)
        return d;
    double ad = fabs(d);
    if (isinf(ad))
        ad = DBL_MAX;
    Q r = a - (Q)ad;                 /* exact: both within a factor 2 or ad == 0 */
    Q spacing, mid;
    if (r >= 0) {
        double up = nextafter(ad, INFINITY);
        spacing = isinf(up) ? (Q)ldexp(1.0, 971) : (Q)up - (Q)ad;
        mid = r - spacing / 2;
    } else {
        double dn = nextafter(ad, 0.0);
        spacing = (Q)ad - (Q)dn;
        mid = -r - spacing / 2;
    }
    if (qabs(mid) <= spacing * (Q)0x1p-50)
        *ambig = 1;
    return d;
}

/* Round a binary128 value to the nearest float (returned as a double) and flag
 * values within 2^-50 of a float spacing from a rounding midpoint.  The
 * binary128 -> binary32 conversion is one IEEE rounding. */
static double rn_float(Q F, int *ambig)
{
#if TFO_PLANT == 10
    float f = (float)(double)F;     /* planted: round through double, then toward zero */
    if (isfinite(f) && qabs((Q)f) > qabs(F)) f = nextafterf(f, 0.0f);
#else
    float f = (float)F;
#endif
    *ambig = 0;
    if (isnan(f) || isinf(F))
        return (double)f;
    Q a = qabs(F);
    if (a == 0)
        return (double)f;
    float af = fabsf(f);
    if (isinf(af))
        af = FLT_MAX;
    Q r = a - (Q)af;
    Q spacing, mid;
    if (r >= 0) {
        float up = nextafterf(af, INFINITY);
        spacing = isinf(up) ? (Q)ldexp(1.0, 104) : (Q)up - (Q)af;
        mid = r - spacing / 2;
    } else {
        float dn = nextafterf(af, 0.0f);
        spacing = (Q)af - (Q)dn;
        mid = -r - spacing / 2;
    }
    if (qabs(mid) <= spacing * (Q)0x1p-50)
        *ambig = 1;
    return (double)f;
}

/* The main part: F rounded to the twofold's format (f32: binary32, else binary64). */
static double rn_main(Q F, int *ambig, int f32)
{
    return f32 ? rn_float(F, ambig) : rn_double(F, ambig);
}

static void put_g(Q G, double *Gh, double *Gl)
{
    double h = (double)G;
    *Gh = h;
    *Gl = (isfinite(h)) ? (double)(G - (Q)h) : 0.0;
}

static void set_exact(double z1, double *Gh, double *Gl, unsigned *fl)
{
    *Gh = z1;
    *Gl = 0.0;
    *fl |= FL_EXACT;
}

/* ---- unary twofold functions --------------------------------------------------- */

static void ox_exp(double x0, double x1, double *Z0, double *Gh, double *Gl, double *A, unsigned *fl, int f32)
{
    int amb = 0;
    *fl = 0; *A = 0;
    if (isnan(x0)) { *Z0 = NAN; set_exact(NAN, Gh, Gl, fl); return; }
    Q E = expf128((Q)x0);                          /* e^x0; exp(-Inf) = 0, exp(+Inf) = Inf */
    *Z0 = rn_main(E, &amb, f32);
    if (amb) *fl |= FL_AMBIG;
    if (isnan(x1)) { set_exact(NAN, Gh, Gl, fl); return; }
    if (*Z0 == 0.0 || isinf(*Z0)) { set_exact(0.0, Gh, Gl, fl); return; }
    if (isinf(x1) && x1 > 0) { set_exact(INFINITY, Gh, Gl, fl); return; }
    Q U = isinf(x1) ? -E : E * expm1f128((Q)x1);  /* e^x0 (e^x1 - 1) */
#if TFO_PLANT == 1
    U = 0;                                         /* planted: drop the x1 term */
#elif TFO_PLANT == 7
    U = expf128((Q)(x0 + x1)) - E;                 /* planted: round x0 + x1 to double first */
#endif
    Q G = (E - (Q)*Z0) + U;                        /* E - Z0 is exact (Sterbenz) */
    put_g(G, Gh, Gl);
    *A = (double)qabs(E + U);
}

static void ox_expm1(double x0, double x1, double *Z0, double *Gh, double *Gl, double *A, unsigned *fl, int f32)
{
    int amb = 0;
    *fl = 0; *A = 0;
    if (isnan(x0)) { *Z0 = NAN; set_exact(NAN, Gh, Gl, fl); return; }
    Q M = expm1f128((Q)x0);
    *Z0 = rn_main(M, &amb, f32);
    if (amb) *fl |= FL_AMBIG;
    if (isnan(x1)) { set_exact(NAN, Gh, Gl, fl); return; }
    if (isinf(*Z0) || (isinf(x0) && x0 < 0)) { set_exact(0.0, Gh, Gl, fl); return; }
    if (isinf(x1) && x1 > 0) { set_exact(INFINITY, Gh, Gl, fl); return; }
    Q E = expf128((Q)x0);
    Q U = isinf(x1) ? -E : E * expm1f128((Q)x1);  /* e^x0 (e^x1 - 1) */
    if (isnan(U)) {
        /* e^x0 underflowed to 0 while e^x1 overflowed: the product is undefined,
           so take expm1 at the binary128 sum x0 + x1 (exact here: both parts
           are huge) */
        Q F = expm1f128((Q)x0 + (Q)x1);
        put_g(F - (Q)*Z0, Gh, Gl);
        *A = (double)qabs(F);
        return;
    }
    /* (e^x0 - 1) - Z0: below x0 = -1 the binary128 expm1 has dropped the low bits
       of e^x0, so form it as e^x0 - (1 + Z0), with 1 + Z0 exact. */
    Q D = (x0 < -1.0) ? E - ((Q)1 + (Q)*Z0) : M - (Q)*Z0;
    Q G = D + U;
    put_g(G, Gh, Gl);
    *A = (double)qabs(M + U);
}

/* log1p(q) of the binary128 ratio q = y1/w, with the log(0) / domain rules. Returns
   0 and sets *special when the answer is fixed exactly. */
static Q corr_log1p(double y1, Q w, Q base, double Z0, int *special, double *zs)
{
    *special = 0;
    if (isinf(y1)) { *special = 1; *zs = (y1 > 0) ? INFINITY : NAN; return 0; }
#if TFO_PLANT == 2
    Q q = -(Q)y1 / w;                              /* planted: wrong sign */
#else
    Q q = (Q)y1 / w;
#endif
    if (q < -1) { *special = 1; *zs = NAN; return 0; }
    if (q == -1) { *special = 1; *zs = -INFINITY; return 0; }
    (void)base; (void)Z0;
    return log1pf128(q);
}

static void ox_log(double y0, double y1, double *Z0, double *Gh, double *Gl, double *A, unsigned *fl, int f32)
{
    int amb = 0, sp = 0;
    double zs = 0;
    *fl = 0; *A = 0;
    if (isnan(y0) || y0 < 0) { *Z0 = NAN; set_exact(NAN, Gh, Gl, fl); return; }
    Q L = logf128((Q)y0);                          /* log(+-0) = -Inf, log(+Inf) = +Inf */
    *Z0 = rn_main(L, &amb, f32);
    if (amb) *fl |= FL_AMBIG;
    if (isnan(y1)) { set_exact(NAN, Gh, Gl, fl); return; }
    if (isinf(*Z0)) { set_exact(0.0, Gh, Gl, fl); return; }
    Q P;
    Q s = (Q)y0 + (Q)y1;
    if (!isinf(y1) && (s - (Q)y0) == (Q)y1 && (Q)y1 < -(Q)y0 / 2) {
        /* y0 + y1 is exact in binary128 and far from y0: take log of it directly
           (avoids the 1/(1+q) sensitivity of log1p near q = -1). */
        if (s < 0) { set_exact(NAN, Gh, Gl, fl); return; }
        if (s == 0) { set_exact(-INFINITY, Gh, Gl, fl); return; }
        P = logf128(s) - L;
    } else {
        P = corr_log1p(y1, (Q)y0, L, *Z0, &sp, &zs);
        if (sp) { set_exact(zs, Gh, Gl, fl); return; }
    }
    Q G = (L - (Q)*Z0) + P;
    put_g(G, Gh, Gl);
    *A = (double)qabs(L + P);
}

static void ox_log1p(double y0, double y1, double *Z0, double *Gh, double *Gl, double *A, unsigned *fl, int f32)
{
    int amb = 0, sp = 0;
    double zs = 0;
    *fl = 0; *A = 0;
    if (isnan(y0) || y0 < -1.0) { *Z0 = NAN; set_exact(NAN, Gh, Gl, fl); return; }
    Q L = log1pf128((Q)y0);                        /* log1p(-1) = -Inf */
    *Z0 = rn_main(L, &amb, f32);
    if (amb) *fl |= FL_AMBIG;
    if (isnan(y1)) { set_exact(NAN, Gh, Gl, fl); return; }
    if (isinf(*Z0)) { set_exact(0.0, Gh, Gl, fl); return; }
    /* w = 1 + y0 held exactly as the binary128 pair wh + wl (Knuth's TwoSum):
       1 + y0 alone would drop a tiny y0, and 1 + y0 + y1 can cancel to it. */
    Q wh = (Q)1 + (Q)y0;
    Q bv = wh - (Q)1;
    Q wl = ((Q)1 - (wh - bv)) + ((Q)y0 - bv);
#if TFO_PLANT == 3
    Q w = (Q)y0;                                   /* planted: wrong base for log1p */
#else
    Q w = wh;
#endif
    Q P;
    if (!isinf(y1) && (Q)y1 < -w / 2) {
        /* y1 cancels most of 1 + y0: s = 1 + y0 + y1 with one rounding (wh + y1
           is exact by Sterbenz) and log(s) directly, not log1p of a ratio near -1. */
        Q s = (wh + (Q)y1) + wl;
        if (s < 0) { set_exact(NAN, Gh, Gl, fl); return; }
        if (s == 0) { set_exact(-INFINITY, Gh, Gl, fl); return; }
        Q Fs = logf128(s);
        Q G = Fs - (Q)*Z0;
        put_g(G, Gh, Gl);
        *A = (double)qabs(Fs);
        return;
    } else {
        P = corr_log1p(y1, w, L, *Z0, &sp, &zs);
        if (sp) { set_exact(zs, Gh, Gl, fl); return; }
    }
    Q G = (L - (Q)*Z0) + P;
    put_g(G, Gh, Gl);
    *A = (double)qabs(L + P);
}

/* ---- twofold add / mul ------------------------------------------------------------ */

static void ox_add(double x0, double x1, double y0, double y1,
                   double *Z0, double *Gh, double *Gl, double *A, unsigned *fl)
{
    volatile double s = x0 + y0;                   /* the plain double sum (no contraction) */
    *fl = 0; *A = 0;
    *Z0 = s;
    if (isnan(s) || isnan(x1) || isnan(y1)) { set_exact(NAN, Gh, Gl, fl); return; }
    if (isinf(s)) { set_exact(0.0, Gh, Gl, fl); return; }
    if (isinf(x1) || isinf(y1)) { volatile double t = x1 + y1; set_exact(t, Gh, Gl, fl); return; }
    double big = fabs(x0) >= fabs(y0) ? x0 : y0;
    double sml = fabs(x0) >= fabs(y0) ? y0 : x0;
#if TFO_PLANT == 6
    Q t = ((Q)s - (Q)big) + (Q)sml;                /* planted: transposed operands */
#else
    Q t = ((Q)big - (Q)s) + (Q)sml;                /* exact rounding error of s */
#endif
    Q G = (t + (Q)x1) + (Q)y1;
    put_g(G, Gh, Gl);
    *A = (double)qabs((Q)s + G);
}

static void ox_mul(double x0, double x1, double y0, double y1,
                   double *Z0, double *Gh, double *Gl, double *A, unsigned *fl)
{
    volatile double p = x0 * y0;                   /* the plain double product */
    *fl = 0; *A = 0;
    *Z0 = p;
    if (isnan(p) || isnan(x1) || isnan(y1)) { set_exact(NAN, Gh, Gl, fl); return; }
    if (isinf(p)) { set_exact(0.0, Gh, Gl, fl); return; }
    if (isinf(x1) || isinf(y1)) {
        volatile double a = x0 * y1, b = x1 * y0;
        volatile double t = a + b;
        set_exact(t, Gh, Gl, fl);
        return;
    }
    Q e = (Q)x0 * (Q)y0 - (Q)p;                     /* exact: 106-bit product, p close */
#if TFO_PLANT == 5
    Q G = e + ((Q)x0 * (Q)y1) + (Q)x1 * (Q)y1;    /* planted: drop x1*y0 */
#else
    Q G = e + ((Q)x0 * (Q)y1 + (Q)x1 * (Q)y0) + (Q)x1 * (Q)y1;
#endif
    put_g(G, Gh, Gl);
    *A = (double)qabs((Q)p + G);
}

/* ---- exported entry points ----------------------------------------------------------- */

int tfo_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void tfo_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

int tfo_eval2(int kind, int f32, int64_t n, const double *x0, const double *x1,
              const double *y0, const double *y1,
              double *Z0, double *Gh, double *Gl, double *A, unsigned *flags);

/* Unary: kind in {0 exp, 1 expm1, 2 log, 3 log1p}; x1 may be NULL (dotted argument).
   Binary: kind in {4 add, 5 mul}; x = x0 + x1, y = y0 + y1 (x1, y1 may be NULL). */
int tfo_eval(int kind, int64_t n, const double *x0, const double *x1,
             const double *y0, const double *y1,
             double *Z0, double *Gh, double *Gl, double *A, unsigned *flags)
{
    return tfo_eval2(kind, 0, n, x0, x1, y0, y1, Z0, Gh, Gl, A, flags);
}

/* As tfo_eval; f32 = 1 evaluates float twofolds (unary kinds only): the
   arguments are floats held in doubles, Z0 = f(x0) rounded to float, and
   G = F - Z0 as before. */
int tfo_eval2(int kind, int f32, int64_t n, const double *x0, const double *x1,
              const double *y0, const double *y1,
              double *Z0, double *Gh, double *Gl, double *A, unsigned *flags)
{
    if (n < 0 || kind < 0 || kind > 5 || (f32 && kind >= K_ADD)) return -1;
    if (kind >= K_ADD && !y0) return -1;
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; i++) {
        double a1 = x1 ? x1[i] : 0.0;
        switch (kind) {
        case K_EXP:   ox_exp(x0[i], a1, &Z0[i], &Gh[i], &Gl[i], &A[i], &flags[i], f32); break;
        case K_EXPM1: ox_expm1(x0[i], a1, &Z0[i], &Gh[i], &Gl[i], &A[i], &flags[i], f32); break;
        case K_LOG:   ox_log(x0[i], a1, &Z0[i], &Gh[i], &Gl[i], &A[i], &flags[i], f32); break;
        case K_LOG1P: ox_log1p(x0[i], a1, &Z0[i], &Gh[i], &Gl[i], &A[i], &flags[i], f32); break;
        case K_ADD:   ox_add(x0[i], a1, y0[i], y1 ? y1[i] : 0.0, &Z0[i], &Gh[i], &Gl[i], &A[i], &flags[i]); break;
        case K_MUL:   ox_mul(x0[i], a1, y0[i], y1 ? y1[i] : 0.0, &Z0[i], &Gh[i], &Gl[i], &A[i], &flags[i]); break;
        }
    }
    return 0;
}

/* Chains of twofold operations (the on-the-fly error tracking of the paper's
   "Overview": the state carries its deviation through a whole computation).
   For each chain, the exact result of its operations applied in order to the
   exact initial state s0 + s1, evaluated in binary128 on the exact operands:
       add: s + (a0 + a1)   mul: s (a0 + a1)   exp: e^s   log: log s
   returned as Fh + Fl (about 106 bits), and the condition sum K of the chain:
   if every operation makes a relative error of at most eps and the later
   operations propagate it exactly, the final relative error is at most
   eps K.  The relative-error gain of one operation on its input state is
   |s| / |s + a| (add), 1 (mul), |s| (exp), 1 / |log s| (log), and
   K = sum over steps t of the product of the gains after step t, accumulated
   as k <- gain k + 1.  Layout as tf_chain (include/tf.h): operation t of
   chain c is entry step_base[t] + c.  An unknown op code leaves the state. */
int tfo_chain(int64_t n_chains, const uint8_t *ops, const double *a0, const double *a1,
              const int64_t *step_base, const int32_t *len, const double *s0, const double *s1,
              double *Fh, double *Fl, double *K)
{
    if (n_chains < 0) return -1;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t c = 0; c < n_chains; c++) {
        Q s = (Q)s0[c] + (Q)s1[c];
        double k = 0.0;
        for (int32_t t = 0; t < len[c]; t++) {
            int64_t i = step_base[t] + c;
            Q a = (Q)a0[i] + (Q)a1[i];
            double g = 1.0;
            switch (ops[i]) {
            case 0: { Q r = s + a; g = (double)(qabs(s) / qabs(r)); s = r; break; }
#if TFO_PLANT == 8
            case 1: s = s * (Q)a0[i]; break;            /* planted: drop the operand tail */
#else
            case 1: s = s * a; break;
#endif
            case 2: g = (double)qabs(s); s = expf128(s); break;
            case 3: { Q r = logf128(s); g = (double)(1 / qabs(r)); s = r; break; }
            default: k -= 1.0; break;   /* no operation, no error */
            }
#if TFO_PLANT == 9
            k = k + 1.0;                                 /* planted: ignore the gains */
#else
            k = g * k + 1.0;
#endif
        }
        put_g(s, &Fh[c], &Fl[c]);
        K[c] = k;
    }
    return 0;
}

/* The binary128 library values themselves, for pinning the oracle against an
   independent evaluation: out[2i] + out[2i+1] = f(x[i]) to about 106 bits. */
int tfo_libq(int kind, int64_t n, const double *x, double *out)
{
    if (n < 0) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        Q v;
        switch (kind) {
        case K_EXP: v = expf128((Q)x[i]); break;
        case K_EXPM1: v = expm1f128((Q)x[i]); break;
        case K_LOG: v = logf128((Q)x[i]); break;
        case K_LOG1P: v = log1pf128((Q)x[i]); break;
        default: v = (Q)NAN;
        }
        put_g(v, &out[2 * i], &out[2 * i + 1]);
    }
    return 0;
}
