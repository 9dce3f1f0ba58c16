/*
 * elbm_oracle.c -- plain, slow FP64 CPU oracle of the essentially entropic
 * lattice Boltzmann step (Atif, Kolluru & Ansumali, "Essentially entropic
 * lattice Boltzmann model: Theory and simulations", arXiv:2203.12946).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the
 * CPU-baseline leg of the benchmark load this library.  The CUDA library never
 * links, loads or calls it, and the two share no source, header, table or
 * constant generator.
 *
 * Every function follows one passage of the paper, named in its comment by
 * section and equation.  Loops are deliberately straightforward: one node at a
 * time, one population at a time, in the order in which the paper states the
 * algorithm (Appendix D).  All arithmetic is IEEE double; nothing is fused or
 * reordered beyond what the formulas say.
 *
 * Two parts have no passage in the paper and say so where they are defined:
 * the uniform body force (an exact-difference term added after the collision)
 * and the adjoint of the step (node Jacobians by central differences), both
 * used to check gradients.
 *
 * Readings where the paper is ambiguous:
 *  R1  the product-form equilibrium carries one factor Upsilon_a per axis
 *      (Sec. I, D2Q9/D3Q27 equilibrium), and with theta0 = 1/3 the exponent
 *      c_ia/sqrt(3 theta0) is c_ia in {-1, 0, 1};
 *  R2  velocity order: lexicographic over (c_1, ..., c_D) in {-1,0,1}^D with
 *      the last axis varying fastest, so opp(i) = Q-1-i;
 *  R3  the Omega^+ denominators of the b coefficient (Eq. qaud_tight_coeff)
 *      are 4 + k x, 4 + 2 k x, 4 + 3 k x with k = alpha_Lower * beta, as the
 *      lower-bound split of Appendix C gives (4/alpha_Lower + beta x); the
 *      printed k = alpha_Lower is kept as b_variant = 1;
 *  R4  h and alpha_Higher use the same conjugate root form as alpha_Lower,
 *      2c/(b + sqrt(b^2 - 4ac)) (Eq. alphaLowerSoln);
 *  R5  the near-equilibrium cutoff is the strict test |x|max < 1e-3;
 *  R6  positivity clamp (Appendix D): if after alpha = (1+alpha_max)/2 the
 *      path length still exceeds alpha_max (only possible when alpha_max < 1),
 *      alpha = alpha_max/2;
 *  R7  with the cutoff disabled, a node with x == 0 exactly (all sums zero)
 *      takes the near-equilibrium limit alpha = 2;
 *  R12 alpha_Iterate1 (Sec. IV) keeps alpha_Lower where its Newton step cannot
 *      be taken: 1 + alpha_Lower x_i <= 0 for some i (the mirror state at
 *      alpha_Lower is not positive, so its entropy is undefined) or
 *      dF/dalpha <= 0 there.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_QMAX 27
#define OR_CUTOFF 1e-3

enum { OR_MODE_HIGHER = 0, OR_MODE_LOWER = 1, OR_MODE_LBGK = 2, OR_MODE_ITERATE1 = 3 };
enum { OR_BRANCH_CUTOFF = 0, OR_BRANCH_SOLVED = 1, OR_BRANCH_CLAMPED = 2 };

/* ------------------------------------------------------------------------ */
/* Lattice: D1Q3 and its tensor products D2Q9, D3Q27 (Sec. I).               */
/* D1Q3 weights read off the explicit equilibrium at u = 0: f_{+-1} = rho/6, */
/* f_0 = 4 rho/6.  Product weights make w_i of DdQ3^d the product over axes. */
/* ------------------------------------------------------------------------ */
static const double OR_W1[3] = {1.0 / 6.0, 4.0 / 6.0, 1.0 / 6.0}; /* c = -1, 0, +1 */

int or_lattice(int D, int *c, double *w)
{
    int Q = 1, i, a;
    if (D < 1 || D > 3) return -1;
    for (a = 0; a < D; a++) Q *= 3;
    for (i = 0; i < Q; i++) {
        int r = i;
        w[i] = 1.0;
        for (a = D - 1; a >= 0; a--) {
            int digit = r % 3;
            r /= 3;
            c[i * D + a] = digit - 1;
            w[i] *= OR_W1[digit];
        }
    }
    return Q;
}

/* Sec. I: entropic equilibrium, Upsilon_a = 2 - sqrt(1 + 3 u_a^2) and        */
/* z_a = (2 u_a + sqrt(1 + 3 u_a^2)) / (1 - u_a);                              */
/* f_i^eq = w_i rho prod_a Upsilon_a z_a^{c_ia}.                                */
void or_equilibrium(int D, double rho, const double *u, double *feq)
{
    int c[OR_QMAX * 3];
    double w[OR_QMAX], Y[3], z[3];
    int Q = or_lattice(D, c, w), i, a;
    for (a = 0; a < D; a++) {
        double s = sqrt(1.0 + 3.0 * u[a] * u[a]);
        Y[a] = 2.0 - s;
        z[a] = (2.0 * u[a] + s) / (1.0 - u[a]);
    }
    for (i = 0; i < Q; i++) {
        double p = w[i] * rho;
        for (a = 0; a < D; a++) {
            p *= Y[a];
            if (c[i * D + a] == 1) p *= z[a];
            else if (c[i * D + a] == -1) p /= z[a];
        }
        feq[i] = p;
    }
}

/* Sec. I: rho = <f, 1>, rho u = <f, c>. */
void or_moments(int D, const double *f, double *rho, double *u)
{
    int c[OR_QMAX * 3];
    double w[OR_QMAX];
    int Q = or_lattice(D, c, w), i, a;
    double r = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (i = 0; i < Q; i++) {
        r += f[i];
        for (a = 0; a < D; a++) m[a] += f[i] * c[i * D + a];
    }
    *rho = r;
    for (a = 0; a < D; a++) u[a] = m[a] / r;
}

/* Eq. hdef: H[f] = <f, log(f/w) - 1>. */
double or_H(int Q, const double *f, const double *w)
{
    double H = 0.0;
    int i;
    for (i = 0; i < Q; i++) H += f[i] * (log(f[i] / w[i]) - 1.0);
    return H;
}

/* Eq. xdef: x_i = f_i^eq / f_i - 1. */
void or_departure(int Q, const double *f, const double *feq, double *x)
{
    int i;
    for (i = 0; i < Q; i++) x[i] = feq[i] / f[i] - 1.0;
}

/* ------------------------------------------------------------------------ */
/* Path length: Sec. III (alpha_Lower, alpha_Higher, h), Appendix C and the  */
/* implementation steps of Appendix D, including the positivity clamp.      */
/* ------------------------------------------------------------------------ */
typedef struct {
    double alpha;        /* path length applied by the collision            */
    double alpha_lower;  /* Eq. alphaLowerSoln (NaN when not evaluated)     */
    double h;            /* positive root of Eq. gaplhah0 (upper bound)     */
    double alpha_higher; /* positive root of Eq. qaud_tight                 */
    double xabsmax;      /* max_i |x_i|                                     */
    double xmin;         /* min_i x_i                                       */
    double alpha_max;    /* -1/(beta x_min), +inf when x_min >= 0           */
    double a1, b1, c1;   /* Eq. alphaLowerCoeffs                            */
    double a2, a, b, c;  /* Eq. a2def and Eq. qaud_tight_coeff              */
    int branch;          /* OR_BRANCH_*                                     */
} or_alpha_info;

/* Positive root of -alpha^2 a + alpha b - c, in the conjugate form of       */
/* Eq. alphaLowerSoln: 2c / (b + sqrt(b^2 - 4ac)).                           */
static double or_root(double a, double b, double c)
{
    return 2.0 * c / (b + sqrt(b * b - 4.0 * a * c));
}

double or_alpha_iterate1(int Q, const double *f, const double *feq, double alpha_lower);
static double or_dF(int Q, const double *f, const double *x, double alpha);

int or_alpha(int Q, const double *f, const double *feq, double beta, int cutoff,
             int b_variant, int mode, or_alpha_info *out)
{
    double x[OR_QMAX];
    int i;
    or_alpha_info r;
    const double nan = NAN;

    r.alpha_lower = r.h = r.alpha_higher = nan;
    r.a1 = r.b1 = r.c1 = r.a2 = r.a = r.b = r.c = nan;

    /* Appendix D, step 1: departures and their extremes. */
    or_departure(Q, f, feq, x);
    r.xabsmax = 0.0;
    r.xmin = x[0];
    for (i = 0; i < Q; i++) {
        if (fabs(x[i]) > r.xabsmax) r.xabsmax = fabs(x[i]);
        if (x[i] < r.xmin) r.xmin = x[i];
    }
    r.alpha_max = (r.xmin < 0.0) ? -1.0 / (beta * r.xmin) : INFINITY;

    if (mode == OR_MODE_LBGK) {
        /* Standard LBGK: constant alpha = 2 (Sec. I). */
        r.alpha = 2.0;
        r.branch = OR_BRANCH_CUTOFF;
        *out = r;
        return 0;
    }

    if (cutoff && r.xabsmax < OR_CUTOFF) {
        /* Appendix D: near equilibrium, alpha = 2. */
        r.alpha = 2.0;
        r.branch = OR_BRANCH_CUTOFF;
    } else {
        double a1 = 0.0, b1 = 0.0, c1 = 0.0;
        /* Eq. alphaLowerCoeffs: a1 = <f, x^3/2>_{Omega-}, b1 = <f, x^2/2>,  */
        /* c1 = <f, 2x^2/(2+x)>;  Omega- = {x < 0} (Eq. decompose).          */
        for (i = 0; i < Q; i++) {
            if (x[i] < 0.0) a1 += f[i] * x[i] * x[i] * x[i] / 2.0;
            b1 += f[i] * x[i] * x[i] / 2.0;
            c1 += f[i] * 2.0 * x[i] * x[i] / (2.0 + x[i]);
        }
        r.a1 = a1;
        r.b1 = b1;
        r.c1 = c1;
        if (b1 == 0.0) {
            /* R7: x == 0 exactly; the near-equilibrium limit. */
            r.alpha = 2.0;
            r.branch = OR_BRANCH_CUTOFF;
        } else {
            /* Eq. alphaLowerSoln. */
            double aL = or_root(a1, b1, c1);
            r.alpha_lower = aL;
            if (mode == OR_MODE_LOWER) {
                r.alpha = aL;
            } else if (mode == OR_MODE_ITERATE1) {
                /* Sec. IV: one Newton step of Eq. deltaH_ from alpha_Lower (R12). */
                int ok = 1;
                for (i = 0; i < Q; i++)
                    if (1.0 + aL * x[i] <= 0.0) ok = 0;
                if (ok && or_dF(Q, f, x, aL) <= 0.0) ok = 0;
                r.alpha = ok ? or_alpha_iterate1(Q, f, feq, aL) : aL;
            } else {
                double b = 0.0, c = 0.0, a2 = 0.0, a = 0.0, h;
                double k = (b_variant == 1) ? aL : aL * beta; /* R3 */
                /* Eq. qaud_tight_coeff, b and c. */
                b = b1;
                for (i = 0; i < Q; i++) {
                    if (x[i] >= 0.0) {
                        double xi = x[i];
                        b -= f[i] * (2.0 * aL * beta * beta * xi * xi * xi / 15.0) *
                             (2.0 / (4.0 + k * xi) + 1.0 / (4.0 + 2.0 * k * xi) +
                              2.0 / (4.0 + 3.0 * k * xi));
                    }
                }
                for (i = 0; i < Q; i++) {
                    double xi = x[i];
                    c += f[i] * (60.0 * xi * xi + 60.0 * xi * xi * xi + 11.0 * xi * xi * xi * xi) /
                         (60.0 + 90.0 * xi + 36.0 * xi * xi + 3.0 * xi * xi * xi);
                }
                /* Eq. a2def: a2 = beta^2 <f, x^3/6>_{Omega-}. */
                for (i = 0; i < Q; i++)
                    if (x[i] < 0.0) a2 += f[i] * x[i] * x[i] * x[i] / 6.0;
                a2 *= beta * beta;
                /* h: positive root of Eq. gaplhah0 (R4). */
                h = or_root(a2, b, c);
                /* Eq. qaud_tight_coeff, a with the upper bound h. */
                for (i = 0; i < Q; i++) {
                    if (x[i] < 0.0) {
                        double xi = x[i], x3 = xi * xi * xi;
                        a += f[i] * (x3 / 6.0 - h * beta * x3 * xi / 12.0 +
                                     h * h * beta * beta * x3 * xi * xi / 20.0 -
                                     h * h * h * beta * beta * beta * x3 * x3 / 5.0);
                    }
                }
                a *= beta * beta;
                r.b = b;
                r.c = c;
                r.a2 = a2;
                r.h = h;
                r.a = a;
                /* Positive root of Eq. qaud_tight (R4). */
                r.alpha_higher = or_root(a, b, c);
                r.alpha = r.alpha_higher;
            }
            r.branch = OR_BRANCH_SOLVED;
        }
    }

    /* Appendix D, positivity: alpha_max = -1/(beta x_min). */
    if (r.alpha > r.alpha_max) {
        r.alpha = (1.0 + r.alpha_max) / 2.0;
        if (r.alpha > r.alpha_max) r.alpha = r.alpha_max / 2.0; /* R6 */
        r.branch = OR_BRANCH_CLAMPED;
    }
    *out = r;
    return 0;
}

/* Eq. fstar_def: f* = f + alpha beta (f^eq - f). */
void or_relax(int Q, const double *f, const double *feq, double alpha, double beta, double *fstar)
{
    int i;
    for (i = 0; i < Q; i++) fstar[i] = f[i] + alpha * beta * (feq[i] - f[i]);
}

/* ------------------------------------------------------------------------ */
/* Entropy changes (Appendix A and Eq. deltaH3).                             */
/* ------------------------------------------------------------------------ */

/* Eq. deltaH3 with xhat = alpha beta x:                                     */
/* H[f*] - H[f] = <f, (1+xhat) log(1+xhat)> - alpha beta <f, x log(1+x)>.    */
double or_deltaH_star(int Q, const double *f, const double *x, double alpha, double beta)
{
    double s1 = 0.0, s2 = 0.0;
    int i;
    for (i = 0; i < Q; i++) {
        double xh = alpha * beta * x[i];
        s1 += f[i] * (1.0 + xh) * log1p(xh);
        s2 += f[i] * x[i] * log1p(x[i]);
    }
    return s1 - alpha * beta * s2;
}

/* g(y) = (1+y) log(1+y) - y, with g(-1) = 1.  Near y = 0 the direct form     */
/* cancels (absolute error ~1e-16 |y| against a value ~y^2/2), so for         */
/* |y| < 0.1 the Taylor series sum_{k>=2} (-1)^k y^k / (k (k-1)) is summed     */
/* through k = 20 (dropped remainder below 1e-19 relative).                  */
static double or_g(double y)
{
    if (y <= -1.0) return 1.0;
    if (fabs(y) < 0.1) {
        double s = 0.0;
        int k;
        for (k = 20; k >= 2; k--) s = s * y + ((k % 2 == 0) ? 1.0 : -1.0) / ((double)k * (k - 1));
        return s * y * y;
    }
    return (1.0 + y) * log1p(y) - y;
}

/* Eq. deltaH_ (mirror state, beta = 1), with <f, x> = 0 (Appendix A) used  */
/* to subtract alpha <f, x> from the first sum:                              */
/* F(alpha) = sum_i f_i [ g(alpha x_i) - alpha x_i log(1 + x_i) ].          */
static double or_F(int Q, const double *f, const double *x, double alpha)
{
    double s = 0.0;
    int i;
    for (i = 0; i < Q; i++) s += f[i] * (or_g(alpha * x[i]) - alpha * x[i] * log1p(x[i]));
    return s;
}

/* dF/dalpha = sum_i f_i x_i [ log(1 + alpha x_i) - log(1 + x_i) ]. */
static double or_dF(int Q, const double *f, const double *x, double alpha)
{
    double s = 0.0;
    int i;
    for (i = 0; i < Q; i++) s += f[i] * x[i] * (log1p(alpha * x[i]) - log1p(x[i]));
    return s;
}

double or_mirror_F(int Q, const double *f, const double *x, double alpha)
{
    return or_F(Q, f, x, alpha);
}

/* Sec. II-III: alpha_ELBM, the non-trivial root of H[f_mirror] = H[f]       */
/* (Eq. entropy_conserve), by Newton iteration safeguarded with bisection on  */
/* the bracket (1, -1/x_min) (F(1) < 0; F convex in alpha).                  */
/* status: 0 converged, 1 no root inside the positivity polytope (the        */
/* indeterminate case of Sec. II), 2 x == 0 (alpha = 2), 3 no convergence.   */
double or_alpha_elbm(int Q, const double *f, const double *feq, double alpha0,
                     int *iters_out, int *status_out)
{
    double x[OR_QMAX], xmin, lo, hi, al;
    int i, it, status = 3;
    or_departure(Q, f, feq, x);
    xmin = x[0];
    for (i = 0; i < Q; i++)
        if (x[i] < xmin) xmin = x[i];
    if (iters_out) *iters_out = 0;
    if (!(xmin < 0.0)) {
        if (status_out) *status_out = 2;
        return 2.0;
    }
    lo = 1.0;
    hi = -1.0 / xmin;
    if (or_F(Q, f, x, hi) < 0.0) {
        if (status_out) *status_out = 1;
        return NAN;
    }
    al = alpha0;
    if (!(al > lo && al < hi)) al = 0.5 * (lo + hi);
    for (it = 1; it <= 100; it++) {
        double F = or_F(Q, f, x, al), dF = or_dF(Q, f, x, al), next;
        if (F < 0.0) lo = al;
        else hi = al;
        next = al - F / dF;
        if (F == 0.0 || fabs(next - al) <= 1e-14 * al) {
            /* Newton step below the tolerance: converged. */
            al = next;
            status = 0;
            break;
        }
        if (!(next > lo && next < hi)) next = 0.5 * (lo + hi); /* bisection safeguard */
        if (hi - lo <= 1e-14 * al) {
            al = 0.5 * (lo + hi);
            status = 0;
            break;
        }
        al = next;
    }
    if (iters_out) *iters_out = it;
    if (status_out) *status_out = status;
    return al;
}

/* Sec. IV (lid-driven cavity): alpha_Iterate1, one Newton step of Eq.       */
/* deltaH_ started from alpha_Lower.                                         */
double or_alpha_iterate1(int Q, const double *f, const double *feq, double alpha_lower)
{
    double x[OR_QMAX];
    or_departure(Q, f, feq, x);
    return alpha_lower - or_F(Q, f, x, alpha_lower) / or_dF(Q, f, x, alpha_lower);
}

/* ------------------------------------------------------------------------ */
/* Field operations on a periodic grid.  Layout: structure of arrays,        */
/* f[i * N + n] with n = (z * ny + y) * nx + x; axis 0 of c_i is x, axis 1 y, */
/* axis 2 z.  D = 2 uses nz = 1.                                             */
/* ------------------------------------------------------------------------ */

static int64_t or_wrap(int64_t v, int64_t n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

static int or_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* Eq. advection: f_i(x + c_i, t + 1) = f*_i(x, t), evaluated as a pull:     */
/* fout_i(x) = fin_i(x - c_i) with periodic wrap.                            */
void or_stream(int D, int64_t nx, int64_t ny, int64_t nz, const double *fin, double *fout, int nthreads)
{
    int c[OR_QMAX * 3];
    double w[OR_QMAX];
    int Q = or_lattice(D, c, w);
    int64_t N = nx * ny * nz, z;
    or_set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (z = 0; z < nz; z++) {
        int64_t y, xx;
        int i;
        for (y = 0; y < ny; y++)
            for (xx = 0; xx < nx; xx++) {
                int64_t n = (z * ny + y) * nx + xx;
                for (i = 0; i < Q; i++) {
                    int64_t sx = or_wrap(xx - c[i * D + 0], nx);
                    int64_t sy = or_wrap(y - c[i * D + 1], ny);
                    int64_t sz = (D == 3) ? or_wrap(z - c[i * D + 2], nz) : 0;
                    fout[(int64_t)i * N + n] = fin[(int64_t)i * N + (sz * ny + sy) * nx + sx];
                }
            }
    }
}

/* Collide every node in place (Eq. fstar_def with alpha from Appendix D).  */
/* Optional per-node outputs: alpha, branch, and H[f*] - H[f] (Eq. deltaH3, */
/* evaluated as the direct difference of Eq. hdef).                          */
void or_collide(int D, int64_t N, double beta, int cutoff, int b_variant, int mode, double *f,
                double *alpha_out, int8_t *branch_out, double *dH_out, int nthreads)
{
    int c[OR_QMAX * 3];
    double w[OR_QMAX];
    int Q = or_lattice(D, c, w);
    int64_t n;
    or_set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (n = 0; n < N; n++) {
        double fn[OR_QMAX], feq[OR_QMAX], fs[OR_QMAX], rho, u[3];
        or_alpha_info info;
        int i;
        for (i = 0; i < Q; i++) fn[i] = f[(int64_t)i * N + n];
        or_moments(D, fn, &rho, u);
        or_equilibrium(D, rho, u, feq);
        or_alpha(Q, fn, feq, beta, cutoff, b_variant, mode, &info);
        or_relax(Q, fn, feq, info.alpha, beta, fs);
        for (i = 0; i < Q; i++) f[(int64_t)i * N + n] = fs[i];
        if (alpha_out) alpha_out[n] = info.alpha;
        if (branch_out) branch_out[n] = (int8_t)info.branch;
        if (dH_out) dH_out[n] = or_H(Q, fs, w) - or_H(Q, fn, w);
    }
}

/* Path length of every node of a (pre-collision) field without relaxing.  */
void or_alpha_field(int D, int64_t N, double beta, int cutoff, int b_variant, int mode,
                    const double *f, double *alpha_out, int8_t *branch_out,
                    double *alpha_elbm_out, int nthreads)
{
    int c[OR_QMAX * 3];
    double w[OR_QMAX];
    int Q = or_lattice(D, c, w);
    int64_t n;
    or_set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (n = 0; n < N; n++) {
        double fn[OR_QMAX], feq[OR_QMAX], rho, u[3];
        or_alpha_info info;
        int i;
        for (i = 0; i < Q; i++) fn[i] = f[(int64_t)i * N + n];
        or_moments(D, fn, &rho, u);
        or_equilibrium(D, rho, u, feq);
        or_alpha(Q, fn, feq, beta, cutoff, b_variant, mode, &info);
        if (alpha_out) alpha_out[n] = info.alpha;
        if (branch_out) branch_out[n] = (int8_t)info.branch;
        if (alpha_elbm_out) {
            int it, st;
            double a0 = (info.alpha_lower == info.alpha_lower) ? info.alpha_lower : 2.0;
            alpha_elbm_out[n] = or_alpha_elbm(Q, fn, feq, a0, &it, &st);
        }
    }
}

/* One time step: stream (Eq. advection) then collide (Eq. fstar_def).      */
/* The stored state is post-collision; fin and fout must not alias.         */
/* Uniform body force (the paper has none; used by the gradient workload).      */
/* Exact-difference forcing applied after the collision:                       */
/*   f_i += f^eq_i(rho, u + F/rho) - f^eq_i(rho, u),                           */
/* rho, u the node's moments (which the collision conserves).  Mass is          */
/* unchanged and the momentum grows by exactly F per step.                      */
void or_force_node(int D, const double *force, double *f)
{
    double rho, u[3], v[3], feq0[OR_QMAX], feq1[OR_QMAX];
    int Q = 1, a, i;
    for (a = 0; a < D; a++) Q *= 3;
    or_moments(D, f, &rho, u);
    for (a = 0; a < D; a++) v[a] = u[a] + force[a] / rho;
    or_equilibrium(D, rho, u, feq0);
    or_equilibrium(D, rho, v, feq1);
    for (i = 0; i < Q; i++) f[i] += feq1[i] - feq0[i];
}

void or_force(int D, int64_t N, const double *force, double *f, int nthreads)
{
    int Q = 1, a;
    int64_t n;
    for (a = 0; a < D; a++) Q *= 3;
    or_set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (n = 0; n < N; n++) {
        double fn[OR_QMAX];
        int i;
        for (i = 0; i < Q; i++) fn[i] = f[(int64_t)i * N + n];
        or_force_node(D, force, fn);
        for (i = 0; i < Q; i++) f[(int64_t)i * N + n] = fn[i];
    }
}

void or_step(int D, int64_t nx, int64_t ny, int64_t nz, double beta, int cutoff, int b_variant,
             int mode, const double *fin, double *fout, double *alpha_out, int8_t *branch_out,
             double *dH_out, int nthreads)
{
    or_stream(D, nx, ny, nz, fin, fout, nthreads);
    or_collide(D, nx * ny * nz, beta, cutoff, b_variant, mode, fout, alpha_out, branch_out, dH_out,
               nthreads);
}

/* Initial state f = f^eq(rho, u) at every node; u is D x N (SoA). */
void or_init_equilibrium(int D, int64_t N, const double *rho, const double *u, double *f)
{
    int c[OR_QMAX * 3];
    double w[OR_QMAX];
    int Q = or_lattice(D, c, w);
    int64_t n;
    for (n = 0; n < N; n++) {
        double un[3], feq[OR_QMAX];
        int i, a;
        for (a = 0; a < D; a++) un[a] = u[(int64_t)a * N + n];
        or_equilibrium(D, rho[n], un, feq);
        for (i = 0; i < Q; i++) f[(int64_t)i * N + n] = feq[i];
    }
}

/* rho and u of every node (u is D x N, SoA). */
void or_moments_field(int D, int64_t N, const double *f, double *rho, double *u)
{
    int c[OR_QMAX * 3];
    double w[OR_QMAX];
    int Q = or_lattice(D, c, w);
    int64_t n;
    for (n = 0; n < N; n++) {
        double fn[OR_QMAX], r, un[3];
        int i, a;
        for (i = 0; i < Q; i++) fn[i] = f[(int64_t)i * N + n];
        or_moments(D, fn, &r, un);
        rho[n] = r;
        for (a = 0; a < D; a++) u[(int64_t)a * N + n] = un[a];
    }
}

/* Global H = sum over nodes of Eq. hdef. */
double or_H_total(int D, int64_t N, const double *f)
{
    int c[OR_QMAX * 3];
    double w[OR_QMAX];
    int Q = or_lattice(D, c, w);
    int64_t n;
    double H = 0.0;
    for (n = 0; n < N; n++) {
        double fn[OR_QMAX];
        int i;
        for (i = 0; i < Q; i++) fn[i] = f[(int64_t)i * N + n];
        H += or_H(Q, fn, w);
    }
    return H;
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Adjoint (reverse-mode derivative) of the step, for checking a hand-written */
/* backward pass.  The paper defines no adjoint; this is the chain rule       */
/* applied to the step above, with each node's Jacobian-transpose product     */
/* taken by central differences of the node collision in FP64 (relative step  */
/* eps on each population).  Streaming is a permutation, so its adjoint is    */
/* the inverse permutation: pull by c_i becomes push by c_i.                  */
/* ------------------------------------------------------------------------ */

/* One node: f (pre-collision, Q values) -> f* (Eq. fstar_def with alpha). */
static void or_collide_node(int D, const double *f, double beta, int cutoff, int b_variant, int mode,
                            const double *force, double *fs)
{
    double feq[OR_QMAX], rho, u[3];
    or_alpha_info info;
    int Q = 1, a;
    for (a = 0; a < D; a++) Q *= 3;
    or_moments(D, f, &rho, u);
    or_equilibrium(D, rho, u, feq);
    or_alpha(Q, f, feq, beta, cutoff, b_variant, mode, &info);
    or_relax(Q, f, feq, info.alpha, beta, fs);
    if (force) or_force_node(D, force, fs);
}

/* h_j = sum_i g_i d f*_i / d f_j at one node, by central differences. */
void or_collide_vjp(int D, const double *f, const double *g, double beta, int cutoff, int b_variant, int mode,
                    const double *force, double eps, double *h)
{
    double fp[OR_QMAX], fm[OR_QMAX], sp[OR_QMAX], sm[OR_QMAX];
    int Q = 1, a, i, j;
    for (a = 0; a < D; a++) Q *= 3;
    for (j = 0; j < Q; j++) {
        double d = eps * f[j], acc = 0.0;
        memcpy(fp, f, sizeof(double) * Q);
        memcpy(fm, f, sizeof(double) * Q);
        fp[j] += d;
        fm[j] -= d;
        or_collide_node(D, fp, beta, cutoff, b_variant, mode, force, sp);
        or_collide_node(D, fm, beta, cutoff, b_variant, mode, force, sm);
        for (i = 0; i < Q; i++) acc += g[i] * (sp[i] - sm[i]);
        h[j] = acc / (2.0 * d);
    }
}

/* dL/df^t from dL/df^{t+1}, where f^{t+1} = collide(stream(f^t)) (fields SoA). */
void or_step_adjoint(int D, int64_t nx, int64_t ny, int64_t nz, double beta, int cutoff, int b_variant, int mode,
                     const double *force, const double *f_t, const double *g_next, double *g_t, double eps,
                     int nthreads)
{
    int c[OR_QMAX * 3];
    double w[OR_QMAX];
    int Q = or_lattice(D, c, w);
    int64_t N = nx * ny * nz, z;
    double *F = (double *)malloc(sizeof(double) * (size_t)Q * (size_t)N);
    if (!F) return;
    or_stream(D, nx, ny, nz, f_t, F, nthreads);
    or_set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (z = 0; z < nz; z++) {
        int64_t y, xx;
        for (y = 0; y < ny; y++)
            for (xx = 0; xx < nx; xx++) {
                int64_t n = (z * ny + y) * nx + xx;
                double fn[OR_QMAX], gn[OR_QMAX], h[OR_QMAX];
                int i;
                for (i = 0; i < Q; i++) {
                    fn[i] = F[(int64_t)i * N + n];
                    gn[i] = g_next[(int64_t)i * N + n];
                }
                or_collide_vjp(D, fn, gn, beta, cutoff, b_variant, mode, force, eps, h);
                /* F_i(x) = f^t_i(x - c_i): the adjoint sends h_i(x) back to x - c_i */
                for (i = 0; i < Q; i++) {
                    int64_t sx = or_wrap(xx - c[i * D + 0], nx);
                    int64_t sy = or_wrap(y - c[i * D + 1], ny);
                    int64_t sz = (D == 3) ? or_wrap(z - c[i * D + 2], nz) : 0;
                    g_t[(int64_t)i * N + (sz * ny + sy) * nx + sx] = h[i];
                }
            }
    }
    free(F);
}

/* Kinetic energy L = 1/2 sum_x rho |u|^2 of a field and its gradient          */
/* dL/df_i = c_i . u - |u|^2 / 2 at every node.                               */
/* d/dF of sum_x <g_next(x), f^{t+1}(x)> for one forced step, by central        */
/* differences in each force component (dF_out: D values).                     */
void or_step_force_vjp(int D, int64_t nx, int64_t ny, int64_t nz, double beta, int cutoff, int b_variant,
                       int mode, const double *force, const double *f_t, const double *g_next, double eps,
                       double *dF_out, int nthreads)
{
    int Q = 1, a, b;
    int64_t N = nx * ny * nz, n;
    double *F;
    for (a = 0; a < D; a++) Q *= 3;
    F = (double *)malloc(sizeof(double) * (size_t)Q * (size_t)N);
    if (!F) return;
    or_stream(D, nx, ny, nz, f_t, F, nthreads);
    for (b = 0; b < D; b++) {
        double acc = 0.0;
        or_set_threads(nthreads);
#pragma omp parallel for schedule(static) reduction(+ : acc)
        for (n = 0; n < N; n++) {
            double fn[OR_QMAX], sp[OR_QMAX], sm[OR_QMAX], fp_[3], fm_[3];
            int i, k;
            for (i = 0; i < Q; i++) fn[i] = F[(int64_t)i * N + n];
            for (k = 0; k < 3; k++) fp_[k] = fm_[k] = (k < D) ? force[k] : 0.0;
            fp_[b] += eps;
            fm_[b] -= eps;
            or_collide_node(D, fn, beta, cutoff, b_variant, mode, fp_, sp);
            or_collide_node(D, fn, beta, cutoff, b_variant, mode, fm_, sm);
            for (i = 0; i < Q; i++) acc += g_next[(int64_t)i * N + n] * (sp[i] - sm[i]) / (2.0 * eps);
        }
        dF_out[b] = acc;
    }
    free(F);
}

double or_kinetic_energy(int D, int64_t N, const double *f, double *grad)
{
    int c[OR_QMAX * 3];
    double w[OR_QMAX];
    int Q = or_lattice(D, c, w);
    int64_t n;
    double L = 0.0;
    for (n = 0; n < N; n++) {
        double fn[OR_QMAX], rho, u[3], uu = 0.0;
        int i, a;
        for (i = 0; i < Q; i++) fn[i] = f[(int64_t)i * N + n];
        or_moments(D, fn, &rho, u);
        for (a = 0; a < D; a++) uu += u[a] * u[a];
        L += 0.5 * rho * uu;
        if (grad)
            for (i = 0; i < Q; i++) {
                double cu = 0.0;
                for (a = 0; a < D; a++) cu += c[i * D + a] * u[a];
                grad[(int64_t)i * N + n] = cu - 0.5 * uu;
            }
    }
    return L;
}
