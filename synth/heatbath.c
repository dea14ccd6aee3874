/*
 * Seeded quenched U(1) gauge fields for the 2D Wilson plaquette action.
 *
 * Input generator only: this file holds none of the solver's arithmetic.  It
 * produces the gauge configurations that both the CPU oracle and the CUDA path
 * read (the paper generates its beta = 6.0 configurations with QCDLAB; these
 * seeded fields stand in for them, Section 2 "Methods").
 *
 * Action S = beta * sum_P (1 - Re U_P),
 *   U_P(x,t) = U_x(x,t) U_t(x+1,t) conj(U_x(x,t+1)) conj(U_t(x,t)),
 * periodic in both directions (the fermion's antiperiodic t boundary belongs to
 * the Dirac operator, not to the gauge field).
 *
 * Update: exact heatbath.  With A the sum of the two staples of a link, the
 * link's conditional density is p(U) ~ exp(beta Re(U A)); writing
 * U = exp(i theta) conj(A)/|A| makes theta a von Mises variate with
 * kappa = beta |A|, drawn by the Best-Fisher (1979) rejection method.
 * Sweep order: checkerboard (x+t parity), direction x first, then t.  Links of
 * one direction and one parity share no staple, so each sub-sweep is parallel.
 * Cold start (all links 1).
 *
 * Reproducibility across machines: the random numbers come from a counter-based
 * splitmix64 hash keyed by (seed, sweep, direction, link, attempt), and the
 * floating-point work uses only +, -, *, /, sqrt and ldexp (the exponential in
 * the rejection test is a Cody-Waite reduced Taylor series written here), built
 * with -ffp-contract=off, so x86-64 and aarch64 produce bit-identical fields.
 *
 * Layout of the output: double[L_t][L_x][2 (mu: 0 = x, 1 = t)][2 (re, im)],
 * i.e. complex128[L_t][L_x][2].
 */
#include <stdint.h>
#include <math.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static inline uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* uniform double in (0, 1) from a 64-bit key and a counter */
static inline double uniform01(uint64_t key, uint64_t ctr) {
    uint64_t z = mix64(key ^ mix64(ctr));
    return ((double)(z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

/* exp(x) from arithmetic only: x = n ln2 + r, |r| <= ln2/2, Taylor to r^17. */
static double det_exp(double x) {
    if (x < -745.0) return 0.0;
    if (x > 709.0) return HUGE_VAL;
    const double ln2_hi = 6.93147180369123816490e-01;
    const double ln2_lo = 1.90821492927058770002e-10;
    const double inv_ln2 = 1.44269504088896338700e+00;
    double t = x * inv_ln2;
    double n = (t >= 0.0) ? (double)(int64_t)(t + 0.5) : -(double)(int64_t)(0.5 - t);
    double r = (x - n * ln2_hi) - n * ln2_lo;
    double p = 1.0;
    for (int k = 17; k >= 1; --k) p = 1.0 + p * r / (double)k;
    return ldexp(p, (int)n);
}

/* One von Mises draw on the circle with concentration kappa around angle 0,
 * returned as (cos theta, sin theta).  Best & Fisher, Appl. Statist. 28 (1979)
 * 152.  The proposal's cos(pi u) is drawn as cos(2 phi) of a uniform point
 * (a, b) in the unit disc, so no trigonometric function is needed. */
static void vonmises(double kappa, uint64_t key, uint64_t ctr0, double* c_out, double* s_out) {
    if (kappa < 1e-8) { /* uniform angle */
        for (uint64_t att = 0;; ++att) {
            double a = 2.0 * uniform01(key, ctr0 + 8 * att) - 1.0;
            double b = 2.0 * uniform01(key, ctr0 + 8 * att + 1) - 1.0;
            double q = a * a + b * b;
            if (q > 0.0 && q <= 1.0) {
                *c_out = (a * a - b * b) / q;
                *s_out = 2.0 * a * b / q;
                return;
            }
        }
    }
    double tau = 1.0 + sqrt(1.0 + 4.0 * kappa * kappa);
    double rho = (tau - sqrt(2.0 * tau)) / (2.0 * kappa);
    double r = (1.0 + rho * rho) / (2.0 * rho);
    for (uint64_t att = 0;; ++att) {
        uint64_t c = ctr0 + 8 * att;
        double a = 2.0 * uniform01(key, c) - 1.0;
        double b = 2.0 * uniform01(key, c + 1) - 1.0;
        double q = a * a + b * b;
        if (!(q > 0.0 && q <= 1.0)) continue;
        double z = (a * a - b * b) / q;
        double f = (1.0 + r * z) / (r + z);
        double cc = kappa * (r - f);
        double u2 = uniform01(key, c + 2);
        int accept = (cc * (2.0 - cc) - u2 > 0.0);
        if (!accept) accept = (cc >= u2 * det_exp(cc - 1.0)); /* log(c/u2)+1-c >= 0 */
        if (!accept) continue;
        double u3 = uniform01(key, c + 3);
        double s = 1.0 - f * f;
        s = (s > 0.0) ? sqrt(s) : 0.0;
        *c_out = f;
        *s_out = (u3 < 0.5) ? -s : s;
        return;
    }
}

static inline void cmul(double ar, double ai, double br, double bi, double* cr, double* ci) {
    double pr = ar * br;
    double qr = ai * bi;
    double pi = ar * bi;
    double qi = ai * br;
    *cr = pr - qr;
    *ci = pi + qi;
}

/* Fill U (layout above) with a thermalised field.  Returns 0 on success. */
int synth_heatbath(double* U, int Lx, int Lt, double beta, int sweeps, uint64_t seed, int nthreads) {
    if (Lx < 2 || Lt < 2 || (Lx & 1) || (Lt & 1) || sweeps < 0 || beta < 0.0) return -1;
    const long V = (long)Lx * Lt;
    for (long i = 0; i < 2 * V; ++i) { U[2 * i] = 1.0; U[2 * i + 1] = 0.0; }
    const uint64_t key = mix64(seed ^ 0x5CA1AB1E0DDBA11ULL);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    for (int sw = 0; sw < sweeps; ++sw) {
        for (int mu = 0; mu < 2; ++mu) {
            for (int par = 0; par < 2; ++par) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
                for (long s = 0; s < V; ++s) {
                    const int x = (int)(s % Lx), t = (int)(s / Lx);
                    if (((x + t) & 1) != par) continue;
                    const int xp = (x + 1) % Lx, xm = (x + Lx - 1) % Lx;
                    const int tp = (t + 1) % Lt, tm = (t + Lt - 1) % Lt;
#define LNK(xx, tt, m, ri) U[(((long)(tt) * Lx + (xx)) * 2 + (m)) * 2 + (ri)]
                    double ar, ai, pr, pi_, qr, qi;
                    if (mu == 0) {
                        /* A = U_t(x+1,t) conj(U_x(x,t+1)) conj(U_t(x,t))
                         *   + conj(U_x(x,t-1)) conj(U_t(x+1,t-1)) U_t(x,t-1) */
                        cmul(LNK(xp, t, 1, 0), LNK(xp, t, 1, 1), LNK(x, tp, 0, 0), -LNK(x, tp, 0, 1), &pr, &pi_);
                        cmul(pr, pi_, LNK(x, t, 1, 0), -LNK(x, t, 1, 1), &ar, &ai);
                        cmul(LNK(x, tm, 0, 0), -LNK(x, tm, 0, 1), LNK(xp, tm, 1, 0), -LNK(xp, tm, 1, 1), &pr, &pi_);
                        cmul(pr, pi_, LNK(x, tm, 1, 0), LNK(x, tm, 1, 1), &qr, &qi);
                    } else {
                        /* A = U_x(x,t+1) conj(U_t(x+1,t)) conj(U_x(x,t))
                         *   + conj(U_x(x-1,t+1)) conj(U_t(x-1,t)) U_x(x-1,t) */
                        cmul(LNK(x, tp, 0, 0), LNK(x, tp, 0, 1), LNK(xp, t, 1, 0), -LNK(xp, t, 1, 1), &pr, &pi_);
                        cmul(pr, pi_, LNK(x, t, 0, 0), -LNK(x, t, 0, 1), &ar, &ai);
                        cmul(LNK(xm, tp, 0, 0), -LNK(xm, tp, 0, 1), LNK(xm, t, 1, 0), -LNK(xm, t, 1, 1), &pr, &pi_);
                        cmul(pr, pi_, LNK(xm, t, 0, 0), LNK(xm, t, 0, 1), &qr, &qi);
                    }
                    ar = ar + qr;
                    ai = ai + qi;
                    double n2 = ar * ar + ai * ai;
                    double nrm = sqrt(n2);
                    double c, sn;
                    /* counter: (sweep, mu, link) then 8 slots per rejection attempt */
                    uint64_t ctr = ((((uint64_t)sw * 2u + (uint64_t)mu) << 24) | (uint64_t)s) << 24;
                    vonmises(beta * nrm, key, ctr, &c, &sn);
                    double ur, ui;
                    if (nrm > 0.0) {
                        /* U = exp(i theta) conj(A)/|A| */
                        cmul(c, sn, ar / nrm, -ai / nrm, &ur, &ui);
                    } else {
                        ur = c; ui = sn;
                    }
                    LNK(x, t, mu, 0) = ur;
                    LNK(x, t, mu, 1) = ui;
#undef LNK
                }
            }
        }
    }
    return 0;
}

/* Test hook: n von Mises draws (cos, sin) with concentration kappa. */
int synth_vonmises(double kappa, long n, uint64_t seed, double* cs) {
    const uint64_t key = mix64(seed ^ 0x5CA1AB1E0DDBA11ULL);
    for (long i = 0; i < n; ++i) vonmises(kappa, key, (uint64_t)i << 24, &cs[2 * i], &cs[2 * i + 1]);
    return 0;
}

/* Test hook: the arithmetic-only exponential. */
double synth_exp(double x) { return det_exp(x); }
