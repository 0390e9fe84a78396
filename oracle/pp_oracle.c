/*
 * pp_oracle.c -- plain, slow, FP64 CPU oracle for the pair-number hot path of
 * "Pulse shape optimization for electron-positron production in rotating
 * fields" (Fillion-Gourdeau, Hebenstreit, Gagnon, MacLean; arXiv 1704.08919).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file: it is used by tests/, by __graft_entry__.smoke() and by the
 * cpu_baseline / reference legs of bench.py.  It shares no source, header,
 * table or helper with the CUDA library.
 *
 * Every routine follows a passage of the paper, step by step, in FP64 with no
 * blocking, fusion or reordering:
 *   - B-spline spectral model ............ Sec. III, Eqs. (coeff_basis_E/phi),
 *                                           Cox-de Boor recursion, clamped knots
 *   - multimode field, potential, fluence . Sec. III, Eqs. (field), (energy);
 *                                           DE renormalisation, Sec. IV.B;
 *                                           Hann envelope, Eqs. (hann),
 *                                           (vector_potential)
 *   - momentum-space Dirac equation ...... Sec. II.A, Eqs. (kin_mom), (free_spin1),
 *                                           (wf_init), (dirac_eq_mom)
 *   - pair density ....................... Sec. II.A, Eq. (pair_prod_homo)
 *   - total density (momentum integral) .. Sec. II.A last paragraph, Eq. (opt_prob)
 *   - quantum kinetic equation (6 comp.) . Sec. II.B, Eqs. (qke), (matrix)
 *   - its adjoint and the gradient ........ Sec. IV.A, Eqs. (eom2), (adj), (grad)
 *   - differential evolution ............. Sec. IV.B, DE/rand/1/bin steps 1-4
 *
 * Compile with -ffp-contract=off so that every product and sum is rounded as
 * written.  Units: m = e = c = hbar = 1 (so e*E is written E).
 */
#define _GNU_SOURCE
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef double complex cplx;

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_DEGENERATE 4

/* ------------------------------------------------------------------------- */
/* B-spline basis, Sec. III                                                  */
/* ------------------------------------------------------------------------- */

/* Clamped knot vector: `order` copies of w_min, equidistant interior
 * breakpoints, `order` copies of w_max.  n = K - order + 2 breakpoints
 * (including both ends), K + order knots in total (N_s = n + k - 2). */
static int knot_vector(int K, int order, double wmin, double wmax, double *t)
{
    int n = K - order + 2;
    if (n < 2)
        return ORC_ERR_ARG;
    for (int i = 0; i < order; i++)
        t[i] = wmin;
    for (int i = 1; i < n - 1; i++)
        t[order - 1 + i] = wmin + (wmax - wmin) * (double)i / (double)(n - 1);
    for (int i = 0; i < order; i++)
        t[K + i] = wmax;
    return ORC_OK;
}

/* B_i(w), i = 0..K-1, by the Cox-de Boor recursion of Sec. III.  The order-1
 * functions are indicators of [t_i, t_{i+1}); reading: the last non-empty
 * interval is closed on the right so that the basis does not vanish at w_max.
 * Terms with a zero-length denominator are zero. */
int orc_bspline_basis(int K, int order, double wmin, double wmax, double w, double *B)
{
    if (K < 1 || order < 1 || K < order || !(wmax > wmin) || !B)
        return ORC_ERR_ARG;
    int nk = K + order;
    double *t = malloc(sizeof(double) * nk);
    double *b = malloc(sizeof(double) * nk);
    knot_vector(K, order, wmin, wmax, t);
    int last = -1; /* index of the last non-empty interval */
    for (int i = 0; i < nk - 1; i++)
        if (t[i] < t[i + 1])
            last = i;
    for (int i = 0; i < nk - 1; i++) {
        int inside = (t[i] <= w && w < t[i + 1]);
        if (i == last && w == t[i + 1])
            inside = 1;
        b[i] = inside ? 1.0 : 0.0;
    }
    for (int r = 2; r <= order; r++) {
        for (int i = 0; i < nk - r; i++) {
            double left = 0.0, right = 0.0;
            double d1 = t[i + r - 1] - t[i];
            double d2 = t[i + r] - t[i + 1];
            if (d1 > 0.0)
                left = (w - t[i]) / d1 * b[i];
            if (d2 > 0.0)
                right = (t[i + r] - w) / d2 * b[i + 1];
            b[i] = left + right;
        }
    }
    for (int i = 0; i < K; i++)
        B[i] = b[i];
    free(t);
    free(b);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Spectral sampling and field synthesis, Sec. III                           */
/* ------------------------------------------------------------------------- */

/* Modes Omega_j = j * dOmega, dOmega = 2 pi / T, for every integer j >= 1 with
 * w_min <= Omega_j <= w_max (the j = 0 DC term is removed).  Returns the number
 * of modes and the first j. */
int orc_mode_range(double wmin, double wmax, double T, int *j_first)
{
    double dw = 2.0 * M_PI / T;
    int j0 = (int)ceil(wmin / dw - 1e-12);
    if (j0 < 1)
        j0 = 1;
    int j1 = (int)floor(wmax / dw + 1e-12);
    if (j_first)
        *j_first = j0;
    return j1 >= j0 ? j1 - j0 + 1 : 0;
}

/* Parameter layout of one candidate: [a^E_x (K), a^phi_x (K), a^E_y (K), a^phi_y (K)].
 * Fills Omega[M], amp[2][M] = E~_l(Omega_j), phase[2][M] = phi_l(Omega_j). */
int orc_spectrum(const double *params, int K, int order, double wmin, double wmax, double T,
                 double *Omega, double *amp, double *phase)
{
    int j0;
    int M = orc_mode_range(wmin, wmax, T, &j0);
    if (M <= 0)
        return -ORC_ERR_ARG;
    double dw = 2.0 * M_PI / T;
    double *B = malloc(sizeof(double) * K);
    for (int m = 0; m < M; m++) {
        double W = (double)(j0 + m) * dw;
        Omega[m] = W;
        int rc = orc_bspline_basis(K, order, wmin, wmax, W, B);
        if (rc) {
            free(B);
            return -rc;
        }
        for (int l = 0; l < 2; l++) {
            const double *aE = params + (2 * l) * K;
            const double *aP = params + (2 * l + 1) * K;
            double e = 0.0, p = 0.0;
            for (int i = 0; i < K; i++) {
                e += aE[i] * B[i];
                p += aP[i] * B[i];
            }
            amp[l * M + m] = e;
            phase[l * M + m] = p;
        }
    }
    free(B);
    return M;
}

/* Field of Eq. (field) with g = 1 over one period t in [-T/2, T/2], the
 * potential A_l(t) = -int_{-T/2}^t E_l, and the global renormalisation of the
 * DE update (Sec. IV.B) to the fluence U of Eq. (energy).  Without the DC term
 * the potential is periodic, so A(-T/2) = A(T/2) = 0.  The fluence of the
 * unscaled field over one period is (T/2) sum_{l,j} E~_{l,j}^2 (orthogonality
 * of the modes); the field is scaled by s = sqrt(U / U_raw).
 *
 * Output: A[c][2][ld] (row 0 = A_x, row 1 = A_y) on the half-step grid
 * t_k = -T/2 + k*T/(2 n_steps), k = 0..2 n_steps; E likewise (may be NULL);
 * scale[c] = s (may be NULL).  A zero-fluence candidate gets A = E = 0,
 * scale = 0 and makes the call return ORC_ERR_DEGENERATE. */
int orc_synth_field(const double *params, int ncand, int K, int order, double wmin, double wmax,
                    double T, double U, int n_steps, int ld, double *A, double *E, double *scale)
{
    if (ncand < 0 || n_steps < 1 || ld < 2 * n_steps + 1 || !(T > 0) || !(U > 0))
        return ORC_ERR_ARG;
    int M = orc_mode_range(wmin, wmax, T, NULL);
    if (M <= 0)
        return ORC_ERR_ARG;
    double *Om = malloc(sizeof(double) * M);
    double *amp = malloc(sizeof(double) * 2 * M);
    double *ph = malloc(sizeof(double) * 2 * M);
    int status = ORC_OK;
    int nsamp = 2 * n_steps + 1;
    double h = T / (2.0 * n_steps);
    double ti = -0.5 * T;
    for (int c = 0; c < ncand; c++) {
        int rc = orc_spectrum(params + (size_t)c * 4 * K, K, order, wmin, wmax, T, Om, amp, ph);
        if (rc < 0) {
            status = -rc;
            break;
        }
        double Uraw = 0.0;
        for (int q = 0; q < 2 * M; q++)
            Uraw += amp[q] * amp[q];
        Uraw *= 0.5 * T;
        double s = Uraw > 0.0 ? sqrt(U / Uraw) : 0.0;
        if (!(Uraw > 0.0))
            status = ORC_ERR_DEGENERATE;
        if (scale)
            scale[c] = s;
        for (int l = 0; l < 2; l++) {
            double *Arow = A + ((size_t)c * 2 + l) * ld;
            double *Erow = E ? E + ((size_t)c * 2 + l) * ld : NULL;
            for (int k = 0; k < nsamp; k++) {
                double t = ti + (double)k * h;
                double a = 0.0, e = 0.0;
                for (int m = 0; m < M; m++) {
                    double Ej = amp[l * M + m], Pj = ph[l * M + m], W = Om[m];
                    e += Ej * cos(W * t - Pj);
                    a += Ej * (sin(W * t - Pj) - sin(W * ti - Pj)) / W;
                }
                Arow[k] = -s * a;
                if (Erow)
                    Erow[k] = s * e;
            }
        }
    }
    free(Om);
    free(amp);
    free(ph);
    return status;
}

/* ------------------------------------------------------------------------- */
/* The Hann envelope of Eq. (hann): g(t) = cos^2(Omega_T t), Omega_T = pi / T. */
/* ------------------------------------------------------------------------- */

/* The antiderivative F of g(t) cos(W t - P) of Eq. (vector_potential),
 * F = 1/4 [2 sin(W t - P)/W + sin((2 Omega_T - W) t + P)/(2 Omega_T - W)
 *          + sin((2 Omega_T + W) t - P)/(2 Omega_T + W)],
 * with the middle term written as (sin(d t + P) - sin P)/d, d = 2 Omega_T - W,
 * which differs from the paper's by a constant (absorbed by A_{l,0}) and has the
 * regular limit t cos P at d = 0 (the mode W = 2 Omega_T). */
static double hann_F(double W, double P, double OT, double t)
{
    double d = 2.0 * OT - W;
    double mid = fabs(d) > 1e-12 * W ? (sin(d * t + P) - sin(P)) / d : t * cos(P);
    return 0.25 * (2.0 * sin(W * t - P) / W + mid + sin((2.0 * OT + W) * t - P) / (2.0 * OT + W));
}

/* Field of Eq. (field) with the Hann envelope: E_l = s g(t) sum_j E_{l,j}
 * cos(Omega_j t - Phi_{l,j}), A_l(t) = s sum_j E_{l,j} [F_{l,j}(t_f) - F_{l,j}(t)] (the paper's
 * gauge A(t_f) = 0), Ed = dE/dt; on the half-step grid of orc_synth_field.  With
 * normalize = 1, s = sqrt(U / U_raw), U_raw = int E^2 dt of the unit-scale field over
 * one period, evaluated by the rectangle rule on the 2 n_steps grid points of the
 * period (exact: E^2 is a trigonometric polynomial of degree < 2 n_steps); with
 * normalize = 0, s = 1.  scale[c] (may be NULL) receives s, or U_raw when
 * normalize = 0.  E and Ed may be NULL. */
int orc_synth_hann(const double *params, int ncand, int K, int order, double wmin, double wmax,
                   double T, double U, int normalize, int n_steps, int ld, double *A, double *E,
                   double *Ed, double *scale)
{
    if (ncand < 0 || n_steps < 1 || ld < 2 * n_steps + 1 || !(T > 0) || !A)
        return ORC_ERR_ARG;
    int M = orc_mode_range(wmin, wmax, T, NULL);
    if (M <= 0)
        return ORC_ERR_ARG;
    double *Om = malloc(sizeof(double) * M);
    double *amp = malloc(sizeof(double) * 2 * M);
    double *ph = malloc(sizeof(double) * 2 * M);
    int nsamp = 2 * n_steps + 1, status = ORC_OK;
    double h = T / (2.0 * n_steps), ti = -0.5 * T, tf = 0.5 * T, OT = M_PI / T;
    double *e1 = malloc(sizeof(double) * nsamp);
    for (int c = 0; c < ncand && status == ORC_OK; c++) {
        int rc = orc_spectrum(params + (size_t)c * 4 * K, K, order, wmin, wmax, T, Om, amp, ph);
        if (rc < 0) {
            status = -rc;
            break;
        }
        /* fluence of the unit-scale field: rectangle rule over one period */
        double Uraw = 0.0;
        for (int l = 0; l < 2; l++)
            for (int k = 0; k < 2 * n_steps; k++) {
                double t = ti + (double)k * h, g = cos(OT * t), e = 0.0;
                g = g * g;
                for (int m = 0; m < M; m++)
                    e += amp[l * M + m] * cos(Om[m] * t - ph[l * M + m]);
                Uraw += (g * e) * (g * e);
            }
        Uraw *= h;
        double s = normalize ? (Uraw > 0.0 ? sqrt(U / Uraw) : 0.0) : 1.0;
        if (normalize && !(Uraw > 0.0))
            status = ORC_ERR_DEGENERATE;
        if (scale)
            scale[c] = normalize ? s : Uraw;
        for (int l = 0; l < 2; l++) {
            double *Ar = A + ((size_t)c * 2 + l) * ld;
            double *Er = E ? E + ((size_t)c * 2 + l) * ld : NULL;
            double *Dr = Ed ? Ed + ((size_t)c * 2 + l) * ld : NULL;
            for (int k = 0; k < nsamp; k++) {
                double t = ti + (double)k * h;
                double cg = cos(OT * t), g = cg * cg, gp = -OT * sin(2.0 * OT * t);
                double a = 0.0, sum_c = 0.0, sum_s = 0.0;
                for (int m = 0; m < M; m++) {
                    double Ej = amp[l * M + m], Pj = ph[l * M + m], W = Om[m];
                    a += Ej * (hann_F(W, Pj, OT, tf) - hann_F(W, Pj, OT, t));
                    sum_c += Ej * cos(W * t - Pj);
                    sum_s += Ej * W * sin(W * t - Pj);
                }
                Ar[k] = s * a;
                e1[k] = s * g * sum_c;
                if (Er)
                    Er[k] = e1[k];
                if (Dr)
                    Dr[k] = s * (gp * sum_c - g * sum_s);
            }
        }
    }
    free(Om), free(amp), free(ph), free(e1);
    return status;
}

/* dF/dP of hann_F (P the phase), with the middle term in the same regular form. */
static double hann_dF_dP(double W, double P, double OT, double t)
{
    double d = 2.0 * OT - W;
    double mid = fabs(d) > 1e-12 * W ? (cos(d * t + P) - cos(P)) / d : -t * sin(P);
    return 0.25 * (-2.0 * cos(W * t - P) / W + mid - cos((2.0 * OT + W) * t - P) / (2.0 * OT + W));
}

/* Chain rule of the un-normalised Hann-envelope field (orc_synth_hann with
 * normalize = 0) for one candidate: gA, gE, gEd = dJ/d(samples) ([2][ld]) ->
 * grad[4K]; and the fluence U (rectangle rule over one period, as orc_synth_hann)
 * with dU[4K].  Each output may be NULL.  With theta = W t - P the samples depend
 * on (E_j, P_j) through A = E_j (F(t_f) - F(t)), E = g E_j cos theta,
 * Ed = E_j (g' cos theta - g W sin theta). */
int orc_synth_vjp_hann(const double *params, int K, int order, double wmin, double wmax, double T,
                       int n_steps, int ld, const double *gA, const double *gE, const double *gEd,
                       double *grad, double *U_out, double *dU)
{
    int M = orc_mode_range(wmin, wmax, T, NULL);
    if (M <= 0 || n_steps < 1 || ld < 2 * n_steps + 1)
        return ORC_ERR_ARG;
    double *Om = malloc(sizeof(double) * M);
    double *amp = malloc(sizeof(double) * 2 * M);
    double *ph = malloc(sizeof(double) * 2 * M);
    double *B = malloc(sizeof(double) * K);
    double *Ek = malloc(sizeof(double) * 2 * (size_t)(2 * n_steps));
    int rc = orc_spectrum(params, K, order, wmin, wmax, T, Om, amp, ph);
    if (rc < 0) {
        free(Om), free(amp), free(ph), free(B), free(Ek);
        return -rc;
    }
    double h = T / (2.0 * n_steps), ti = -0.5 * T, tf = 0.5 * T, OT = M_PI / T;
    /* the field on the 2 n_steps points of the period, for the fluence */
    double U = 0.0;
    for (int l = 0; l < 2; l++)
        for (int k = 0; k < 2 * n_steps; k++) {
            double t = ti + (double)k * h, cg = cos(OT * t), e = 0.0;
            for (int m = 0; m < M; m++)
                e += amp[l * M + m] * cos(Om[m] * t - ph[l * M + m]);
            Ek[l * 2 * n_steps + k] = cg * cg * e;
            U += Ek[l * 2 * n_steps + k] * Ek[l * 2 * n_steps + k];
        }
    U *= h;
    if (U_out)
        *U_out = U;
    if (grad)
        for (int i = 0; i < 4 * K; i++)
            grad[i] = 0.0;
    if (dU)
        for (int i = 0; i < 4 * K; i++)
            dU[i] = 0.0;
    for (int m = 0; m < M; m++) {
        double W = Om[m];
        orc_bspline_basis(K, order, wmin, wmax, W, B);
        for (int l = 0; l < 2; l++) {
            double Ej = amp[l * M + m], Pj = ph[l * M + m];
            double dE = 0.0, dP = 0.0, uE = 0.0, uP = 0.0;
            double Ff = hann_F(W, Pj, OT, tf), Pf = hann_dF_dP(W, Pj, OT, tf);
            for (int k = 0; k <= 2 * n_steps; k++) {
                double t = ti + (double)k * h;
                double cg = cos(OT * t), g = cg * cg, gp = -OT * sin(2.0 * OT * t);
                double ck = cos(W * t - Pj), sk = sin(W * t - Pj);
                if (grad) {
                    double ga = gA[l * ld + k], ge = gE[l * ld + k], gd = gEd[l * ld + k];
                    dE += ga * (Ff - hann_F(W, Pj, OT, t)) + ge * (g * ck) + gd * (gp * ck - g * W * sk);
                    dP += ga * (Ej * (Pf - hann_dF_dP(W, Pj, OT, t))) + ge * (g * Ej * sk)
                          + gd * (Ej * (gp * sk + g * W * ck));
                }
                if (dU && k < 2 * n_steps) {
                    double e = Ek[l * 2 * n_steps + k];
                    uE += 2.0 * h * e * (g * ck);
                    uP += 2.0 * h * e * (g * Ej * sk);
                }
            }
            for (int i = 0; i < K; i++) {
                if (grad) {
                    grad[2 * l * K + i] += B[i] * dE;
                    grad[(2 * l + 1) * K + i] += B[i] * dP;
                }
                if (dU) {
                    dU[2 * l * K + i] += B[i] * uE;
                    dU[(2 * l + 1) * K + i] += B[i] * uP;
                }
            }
        }
    }
    free(Om), free(amp), free(ph), free(B), free(Ek);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* A test field: E(t) = E0 exp(-t^2/tau^2) (cos w t, sin w t, 0), A(t0) = 0,  */
/* A(t) = -int_{t0}^t E.  The integral has no elementary closed form; it is  */
/* accumulated interval by interval with 10-point Gauss-Legendre quadrature. */
/* ------------------------------------------------------------------------- */

/* Gauss-Legendre nodes/weights on [-1,1] by Newton iteration on P_n. */
static void gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < n; i++) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16)
                break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

static void gauss_rot_E(double E0, double w, double tau, double t, double *ex, double *ey)
{
    double g = E0 * exp(-(t * t) / (tau * tau));
    *ex = g * cos(w * t);
    *ey = g * sin(w * t);
}

/* Samples k = 0..nsamp-1 at t = t0 + k h.  A[2][nsamp]; E, Edot likewise or NULL. */
void orc_gaussian_rotating_field(double E0, double w, double tau, double t0, double h, int nsamp,
                                 double *A, double *E, double *Edot)
{
    double gx[10], gw[10];
    gauss_legendre(10, gx, gw);
    double ax = 0.0, ay = 0.0;
    for (int k = 0; k < nsamp; k++) {
        double t = t0 + (double)k * h;
        if (k > 0) {
            double a = t0 + (double)(k - 1) * h, mid = a + 0.5 * h;
            double sx = 0.0, sy = 0.0;
            for (int q = 0; q < 10; q++) {
                double ex, ey;
                gauss_rot_E(E0, w, tau, mid + 0.5 * h * gx[q], &ex, &ey);
                sx += gw[q] * ex;
                sy += gw[q] * ey;
            }
            ax -= 0.5 * h * sx;
            ay -= 0.5 * h * sy;
        }
        A[k] = ax;
        A[nsamp + k] = ay;
        double ex, ey;
        gauss_rot_E(E0, w, tau, t, &ex, &ey);
        if (E) {
            E[k] = ex;
            E[nsamp + k] = ey;
        }
        if (Edot) {
            double dg = -2.0 * t / (tau * tau);
            Edot[k] = dg * ex - w * ey;
            Edot[nsamp + k] = dg * ey + w * ex;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Momentum-space Dirac equation, Sec. II.A                                  */
/* ------------------------------------------------------------------------- */

/* Dirac representation: alpha_i = sigma_x (x) sigma_i, beta = sigma_z (x) 1. */
static void kron2(const cplx a[2][2], const cplx b[2][2], cplx out[4][4])
{
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++)
            for (int k = 0; k < 2; k++)
                for (int l = 0; l < 2; l++)
                    out[2 * i + k][2 * j + l] = a[i][j] * b[k][l];
}

typedef struct {
    cplx alpha[3][4][4];
    cplx beta[4][4];
} dirac_mats;

static void make_dirac_mats(dirac_mats *D)
{
    const cplx s0[2][2] = {{1, 0}, {0, 1}};
    const cplx sx[2][2] = {{0, 1}, {1, 0}};
    const cplx sy[2][2] = {{0, -I}, {I, 0}};
    const cplx sz[2][2] = {{1, 0}, {0, -1}};
    kron2(sx, sx, D->alpha[0]);
    kron2(sx, sy, D->alpha[1]);
    kron2(sx, sz, D->alpha[2]);
    kron2(sz, s0, D->beta);
}

/* H(P) = alpha . P + beta m, Eq. (dirac_eq_mom) with P = p - A(t), Eq. (kin_mom). */
static void hamiltonian(const dirac_mats *D, const double P[3], cplx H[4][4])
{
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++)
            H[i][j] = D->alpha[0][i][j] * P[0] + D->alpha[1][i][j] * P[1] +
                      D->alpha[2][i][j] * P[2] + D->beta[i][j];
}

/* dpsi/dt = -i H psi */
static void dirac_rhs(const cplx H[4][4], const cplx psi[4], cplx out[4])
{
    for (int i = 0; i < 4; i++) {
        cplx acc = 0;
        for (int j = 0; j < 4; j++)
            acc += H[i][j] * psi[j];
        out[i] = -I * acc;
    }
}

/* sigma . P as a 2x2 matrix */
static void sigma_dot(const double P[3], cplx S[2][2])
{
    S[0][0] = P[2];
    S[0][1] = P[0] - I * P[1];
    S[1][0] = P[0] + I * P[1];
    S[1][1] = -P[2];
}

/* Adiabatic free spinors of Eq. (free_spin1) at kinetic momentum P:
 * u_s = [(w+m) xi_s ; (sigma.P) xi_s] / sqrt(w+m),
 * v_s = [-(sigma.P) eta_s ; (w+m) eta_s] / sqrt(w+m),
 * xi_1 = eta_2 = (1,0), xi_2 = eta_1 = (0,1); s = 0,1 here for s = 1,2. */
void orc_spinors(const double P[3], double _Complex u[2][4], double _Complex v[2][4])
{
    double w = sqrt(P[0] * P[0] + P[1] * P[1] + P[2] * P[2] + 1.0);
    double nrm = 1.0 / sqrt(w + 1.0);
    cplx S[2][2];
    sigma_dot(P, S);
    const cplx xi[2][2] = {{1, 0}, {0, 1}};
    const cplx eta[2][2] = {{0, 1}, {1, 0}};
    for (int s = 0; s < 2; s++) {
        for (int a = 0; a < 2; a++) {
            cplx sx = S[a][0] * xi[s][0] + S[a][1] * xi[s][1];
            cplx se = S[a][0] * eta[s][0] + S[a][1] * eta[s][1];
            u[s][a] = (w + 1.0) * xi[s][a] * nrm;
            u[s][2 + a] = sx * nrm;
            v[s][a] = -se * nrm;
            v[s][2 + a] = (w + 1.0) * eta[s][a] * nrm;
        }
    }
}

static double pdot2(const double P[3])
{
    return P[0] * P[0] + P[1] * P[1] + P[2] * P[2];
}

/* One momentum mode, both spins.  A[0][k], A[1][k] (row stride ld) are the
 * potential samples at t_i + k dt/2.  Classical RK4 on Eq. (dirac_eq_mom)
 * over n_steps steps of size dt; the stage times t_n, t_n + dt/2, t_n + dt use
 * samples 2n, 2n+1, 2n+2.  Initial state psi_s = v_s(P_in), Eq. (wf_init).
 * Returns f(t_f, p) of Eq. (pair_prod_homo):
 *   spin_sum = 0: sum_s sum_s' |u_s'^out+ psi_s|^2 / (2 w_out 2 w_in)   (full trace)
 *   spin_sum = 1: sum_s        |u_s^out+  psi_s|^2 / (2 w_out 2 w_in)   (same-s only)
 * If psi_out is given it receives psi_s(t_f) (s-major, 8 complex). */
double orc_dirac_mode(const double *A, int ld, int n_steps, double dt, const double p[3],
                      int spin_sum, double _Complex *psi_out)
{
    dirac_mats D;
    make_dirac_mats(&D);
    const double *Ax = A, *Ay = A + ld;
    double Pin[3] = {p[0] - Ax[0], p[1] - Ay[0], p[2]};
    double Pout[3] = {p[0] - Ax[2 * n_steps], p[1] - Ay[2 * n_steps], p[2]};
    double win = sqrt(pdot2(Pin) + 1.0), wout = sqrt(pdot2(Pout) + 1.0);
    cplx uin[2][4], vin[2][4], uout[2][4], vout[2][4];
    orc_spinors(Pin, uin, vin);
    orc_spinors(Pout, uout, vout);
    double f = 0.0;
    for (int s = 0; s < 2; s++) {
        cplx psi[4];
        for (int a = 0; a < 4; a++)
            psi[a] = vin[s][a];
        for (int n = 0; n < n_steps; n++) {
            double P0[3] = {p[0] - Ax[2 * n], p[1] - Ay[2 * n], p[2]};
            double P1[3] = {p[0] - Ax[2 * n + 1], p[1] - Ay[2 * n + 1], p[2]};
            double P2[3] = {p[0] - Ax[2 * n + 2], p[1] - Ay[2 * n + 2], p[2]};
            cplx H0[4][4], H1[4][4], H2[4][4];
            hamiltonian(&D, P0, H0);
            hamiltonian(&D, P1, H1);
            hamiltonian(&D, P2, H2);
            cplx k1[4], k2[4], k3[4], k4[4], tmp[4];
            dirac_rhs(H0, psi, k1);
            for (int a = 0; a < 4; a++)
                tmp[a] = psi[a] + 0.5 * dt * k1[a];
            dirac_rhs(H1, tmp, k2);
            for (int a = 0; a < 4; a++)
                tmp[a] = psi[a] + 0.5 * dt * k2[a];
            dirac_rhs(H1, tmp, k3);
            for (int a = 0; a < 4; a++)
                tmp[a] = psi[a] + dt * k3[a];
            dirac_rhs(H2, tmp, k4);
            for (int a = 0; a < 4; a++)
                psi[a] = psi[a] + dt / 6.0 * (k1[a] + 2.0 * k2[a] + 2.0 * k3[a] + k4[a]);
        }
        if (psi_out)
            for (int a = 0; a < 4; a++)
                psi_out[4 * s + a] = psi[a];
        for (int s2 = 0; s2 < 2; s2++) {
            if (spin_sum == 1 && s2 != s)
                continue;
            cplx amp = 0;
            for (int a = 0; a < 4; a++)
                amp += conj(uout[s2][a]) * psi[a];
            f += creal(amp * conj(amp)) / (2.0 * wout * 2.0 * win);
        }
    }
    return f;
}

/* ------------------------------------------------------------------------- */
/* Second-order split operator (Sec. II.A: the paper propagates the Dirac    */
/* equation with "a simple split-operator method with a second order         */
/* convergence"; the splitting is not given).  Reading: Strang splitting of  */
/* H(t) = H_0 + V(t) into the free Hamiltonian H_0 = alpha.p + beta and the  */
/* coupling to the field V(t) = -alpha.A(t), the latter at t_n + dt/2:        */
/*   psi_{n+1} = e^{-i H_0 dt/2} e^{-i V(t_n + dt/2) dt} e^{-i H_0 dt/2} psi_n */
/* Both parts square to multiples of the identity (H_0^2 = (p^2 + 1) 1,      */
/* V^2 = |A|^2 1 for A in the x-y plane), so each factor is exactly          */
/* cos(k tau) - i sin(k tau) K / k, and free propagation (A = 0) is exact.   */
/* ------------------------------------------------------------------------- */

/* U = exp(-i K tau) for Hermitian K with K^2 = k2 * 1. */
static void expm_squared_scalar(cplx K[4][4], double k2, double tau, cplx U[4][4])
{
    double k = sqrt(k2);
    double c = cos(k * tau);
    double sk = k > 0.0 ? sin(k * tau) / k : tau;
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++)
            U[i][j] = (i == j ? c : 0.0) - I * sk * K[i][j];
}

static void matvec4(cplx U[4][4], const cplx x[4], cplx y[4])
{
    for (int i = 0; i < 4; i++) {
        cplx acc = 0;
        for (int j = 0; j < 4; j++)
            acc += U[i][j] * x[j];
        y[i] = acc;
    }
}

/* f(t_f, p) as orc_dirac_mode (full spin trace), propagated with the split
 * operator; *norm_dev receives max_s | |psi_s(t_f)|^2 / |psi_s(t_0)|^2 - 1 |. */
double orc_dirac_split_mode(const double *A, int ld, int n_steps, double dt, const double p[3],
                            double *norm_dev)
{
    dirac_mats D;
    make_dirac_mats(&D);
    const double *Ax = A, *Ay = A + ld;
    double Pin[3] = {p[0] - Ax[0], p[1] - Ay[0], p[2]};
    double Pout[3] = {p[0] - Ax[2 * n_steps], p[1] - Ay[2 * n_steps], p[2]};
    double win = sqrt(pdot2(Pin) + 1.0), wout = sqrt(pdot2(Pout) + 1.0);
    cplx uin[2][4], vin[2][4], uout[2][4], vout[2][4];
    orc_spinors(Pin, uin, vin);
    orc_spinors(Pout, uout, vout);
    cplx H0[4][4], UB[4][4];
    hamiltonian(&D, p, H0);
    expm_squared_scalar(H0, pdot2(p) + 1.0, 0.5 * dt, UB);
    double f = 0.0, dev = 0.0;
    for (int s = 0; s < 2; s++) {
        cplx psi[4], tmp[4];
        for (int a = 0; a < 4; a++)
            psi[a] = vin[s][a];
        double n0 = 0.0;
        for (int a = 0; a < 4; a++)
            n0 += creal(psi[a] * conj(psi[a]));
        for (int n = 0; n < n_steps; n++) {
            double ax = Ax[2 * n + 1], ay = Ay[2 * n + 1];
            cplx V[4][4], UA[4][4];
            for (int i = 0; i < 4; i++)
                for (int j = 0; j < 4; j++)
                    V[i][j] = -(D.alpha[0][i][j] * ax + D.alpha[1][i][j] * ay);
            expm_squared_scalar(V, ax * ax + ay * ay, dt, UA);
            matvec4(UB, psi, tmp);
            matvec4(UA, tmp, psi);
            matvec4(UB, psi, tmp);
            for (int a = 0; a < 4; a++)
                psi[a] = tmp[a];
        }
        double n1 = 0.0;
        for (int a = 0; a < 4; a++)
            n1 += creal(psi[a] * conj(psi[a]));
        if (fabs(n1 / n0 - 1.0) > dev)
            dev = fabs(n1 / n0 - 1.0);
        for (int s2 = 0; s2 < 2; s2++) {
            cplx amp = 0;
            for (int a = 0; a < 4; a++)
                amp += conj(uout[s2][a]) * psi[a];
            f += creal(amp * conj(amp)) / (2.0 * wout * 2.0 * win);
        }
    }
    if (norm_dev)
        *norm_dev = dev;
    return f;
}

/* ------------------------------------------------------------------------- */
/* Fourth-order Magnus integrator (the paper's outlook, Sec. V.C.2, names a   */
/* fourth-order scheme for the Dirac equation as the next step).  With the    */
/* samples H_0 = H(t_n), H_h = H(t_n + dt/2), H_1 = H(t_n + dt):               */
/*   Omega = -i dt/6 (H_0 + 4 H_h + H_1) + dt^2/12 [H_0, H_1],                */
/*   psi_{n+1} = exp(Omega) psi_n,                                            */
/* the two-term Magnus expansion with Simpson's rule for the first integral   */
/* and the endpoint form of the commutator term (fourth order, unitary).      */
/* ------------------------------------------------------------------------- */

static void matmul4(cplx X[4][4], cplx Y[4][4], cplx Z[4][4])
{
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            cplx acc = 0;
            for (int k = 0; k < 4; k++)
                acc += X[i][k] * Y[k][j];
            Z[i][j] = acc;
        }
}

/* exp(X) by its Taylor series, summed until the terms stop changing the sum
 * (|X| < 1 here, so at most ~25 terms). */
static void expm_taylor(cplx X[4][4], cplx E[4][4])
{
    cplx term[4][4], next[4][4];
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            E[i][j] = (i == j) ? 1.0 : 0.0;
            term[i][j] = E[i][j];
        }
    for (int k = 1; k < 60; k++) {
        matmul4(term, X, next);
        double mx = 0.0;
        for (int i = 0; i < 4; i++)
            for (int j = 0; j < 4; j++) {
                term[i][j] = next[i][j] / (double)k;
                E[i][j] += term[i][j];
                if (cabs(term[i][j]) > mx)
                    mx = cabs(term[i][j]);
            }
        if (mx < 1e-30)
            break;
    }
}

/* f(t_f, p) as orc_dirac_mode (full spin trace), propagated with the
 * fourth-order Magnus step; *norm_dev as in orc_dirac_split_mode. */
double orc_dirac_magnus_mode(const double *A, int ld, int n_steps, double dt, const double p[3],
                             double *norm_dev)
{
    dirac_mats D;
    make_dirac_mats(&D);
    const double *Ax = A, *Ay = A + ld;
    double Pin[3] = {p[0] - Ax[0], p[1] - Ay[0], p[2]};
    double Pout[3] = {p[0] - Ax[2 * n_steps], p[1] - Ay[2 * n_steps], p[2]};
    double win = sqrt(pdot2(Pin) + 1.0), wout = sqrt(pdot2(Pout) + 1.0);
    cplx uin[2][4], vin[2][4], uout[2][4], vout[2][4];
    orc_spinors(Pin, uin, vin);
    orc_spinors(Pout, uout, vout);
    cplx psi[2][4];
    for (int s = 0; s < 2; s++)
        for (int a = 0; a < 4; a++)
            psi[s][a] = vin[s][a];
    for (int n = 0; n < n_steps; n++) {
        double P0[3] = {p[0] - Ax[2 * n], p[1] - Ay[2 * n], p[2]};
        double Ph[3] = {p[0] - Ax[2 * n + 1], p[1] - Ay[2 * n + 1], p[2]};
        double P1[3] = {p[0] - Ax[2 * n + 2], p[1] - Ay[2 * n + 2], p[2]};
        cplx H0[4][4], Hh[4][4], H1[4][4], C01[4][4], C10[4][4], Om[4][4], U[4][4];
        hamiltonian(&D, P0, H0);
        hamiltonian(&D, Ph, Hh);
        hamiltonian(&D, P1, H1);
        matmul4(H0, H1, C01);
        matmul4(H1, H0, C10);
        for (int i = 0; i < 4; i++)
            for (int j = 0; j < 4; j++)
                Om[i][j] = -I * dt / 6.0 * (H0[i][j] + 4.0 * Hh[i][j] + H1[i][j]) +
                           dt * dt / 12.0 * (C01[i][j] - C10[i][j]);
        expm_taylor(Om, U);
        for (int s = 0; s < 2; s++) {
            cplx tmp[4];
            matvec4(U, psi[s], tmp);
            for (int a = 0; a < 4; a++)
                psi[s][a] = tmp[a];
        }
    }
    double f = 0.0, dev = 0.0;
    for (int s = 0; s < 2; s++) {
        double n0 = 0.0, n1 = 0.0;
        for (int a = 0; a < 4; a++) {
            n0 += creal(vin[s][a] * conj(vin[s][a]));
            n1 += creal(psi[s][a] * conj(psi[s][a]));
        }
        if (fabs(n1 / n0 - 1.0) > dev)
            dev = fabs(n1 / n0 - 1.0);
        for (int s2 = 0; s2 < 2; s2++) {
            cplx amp = 0;
            for (int a = 0; a < 4; a++)
                amp += conj(uout[s2][a]) * psi[s][a];
            f += creal(amp * conj(amp)) / (2.0 * wout * 2.0 * win);
        }
    }
    if (norm_dev)
        *norm_dev = dev;
    return f;
}

/* ------------------------------------------------------------------------- */
/* 6-component quantum kinetic equation, Sec. II.B, Eqs. (qke), (matrix)      */
/* The paper's field plane (e2,e3) with out-of-plane axis e1 maps onto this   */
/* file's (x,y) plane with out-of-plane z (a cyclic relabelling).             */
/* ------------------------------------------------------------------------- */

static void qke_matrix(const double P[3], const double E[2], const double Ed[2], double N[6][6])
{
    double w2 = pdot2(P) + 1.0, w = sqrt(w2);
    double EE = E[0] * E[0] + E[1] * E[1];
    double EP = E[0] * P[0] + E[1] * P[1];
    double X = w2 * EE - EP * EP;
    double eperp = sqrt(1.0 + P[2] * P[2]);
    double cross = E[0] * Ed[1] - E[1] * Ed[0];
    double Q = sqrt(X) / w2;
    double R = X > 0.0 ? eperp * w * cross / X : 0.0;
    memset(N, 0, sizeof(double) * 36);
    N[0][1] = -Q;
    N[1][0] = Q;
    N[1][2] = -2.0 * w;
    N[1][3] = R;
    N[2][1] = 2.0 * w;
    N[2][4] = -R;
    N[3][1] = -R;
    N[3][4] = 2.0 * w;
    N[4][2] = R;
    N[4][3] = -2.0 * w;
    N[4][5] = Q;
    N[5][4] = -Q;
}

static void mat6_vec(const double N[6][6], const double x[6], double y[6])
{
    for (int i = 0; i < 6; i++) {
        double acc = 0.0;
        for (int j = 0; j < 6; j++)
            acc += N[i][j] * x[j];
        y[i] = acc;
    }
}

/* chi moves on the unit sphere (N is skew), but RK4 does not keep |chi| = 1:
 * its amplification per step, |1 + z + ... + z^4/24| at z = i theta, is below
 * one for theta < 2 sqrt(2) and above it beyond, so where the field is too
 * strong for the step the discrete chi grows without bound and f = 1 - chi_1
 * leaves the physical range [0, 2].  A density whose |chi(t_f)|^2 exceeds
 * 1 + QKE_GROWTH_TOL is reported as NaN (the step is too coarse for the field),
 * so that an optimiser never climbs on that artefact. */
#define QKE_GROWTH_TOL 1e-3

static double qke_density(const double chi[6])
{
    double nrm = 0.0;
    for (int i = 0; i < 6; i++)
        nrm += chi[i] * chi[i];
    if (!(nrm <= 1.0 + QKE_GROWTH_TOL))
        return NAN;
    return 1.0 - chi[0];
}

/* f = 1 - chi_1(t_f) by classical RK4 with chi(t_i) = (1,0,0,0,0,0).  A, E,
 * Edot are [2][ld] half-step samples as in orc_dirac_mode. */
double orc_qke6_mode(const double *A, const double *E, const double *Edot, int ld, int n_steps,
                     double dt, const double p[3])
{
    double chi[6] = {1, 0, 0, 0, 0, 0};
    for (int n = 0; n < n_steps; n++) {
        double Nm[3][6][6];
        for (int q = 0; q < 3; q++) {
            int k = 2 * n + q;
            double P[3] = {p[0] - A[k], p[1] - A[ld + k], p[2]};
            double Ek[2] = {E[k], E[ld + k]};
            double Edk[2] = {Edot[k], Edot[ld + k]};
            qke_matrix(P, Ek, Edk, Nm[q]);
        }
        double k1[6], k2[6], k3[6], k4[6], tmp[6];
        mat6_vec(Nm[0], chi, k1);
        for (int i = 0; i < 6; i++)
            tmp[i] = chi[i] + 0.5 * dt * k1[i];
        mat6_vec(Nm[1], tmp, k2);
        for (int i = 0; i < 6; i++)
            tmp[i] = chi[i] + 0.5 * dt * k2[i];
        mat6_vec(Nm[1], tmp, k3);
        for (int i = 0; i < 6; i++)
            tmp[i] = chi[i] + dt * k3[i];
        mat6_vec(Nm[2], tmp, k4);
        for (int i = 0; i < 6; i++)
            chi[i] = chi[i] + dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    }
    return qke_density(chi);
}

/* ------------------------------------------------------------------------- */
/* Many modes in parallel (std threads over the mode list)                   */
/* ------------------------------------------------------------------------- */

typedef struct {
    const double *A, *E, *Edot;
    int ld, n_steps, spin_sum, kind;
    double dt;
    const double *p;
    int nm, stride;
    int first;
    double *out;
    double *aux;
} mode_job;

static void *mode_worker(void *arg)
{
    mode_job *J = arg;
    for (int m = J->first; m < J->nm; m += J->stride) {
        if (J->kind == 0)
            J->out[m] = orc_dirac_mode(J->A, J->ld, J->n_steps, J->dt, J->p + 3 * m, J->spin_sum, NULL);
        else if (J->kind == 2)
            J->out[m] = orc_dirac_split_mode(J->A, J->ld, J->n_steps, J->dt, J->p + 3 * m,
                                             J->aux ? J->aux + m : NULL);
        else if (J->kind == 3)
            J->out[m] = orc_dirac_magnus_mode(J->A, J->ld, J->n_steps, J->dt, J->p + 3 * m,
                                              J->aux ? J->aux + m : NULL);
        else
            J->out[m] = orc_qke6_mode(J->A, J->E, J->Edot, J->ld, J->n_steps, J->dt, J->p + 3 * m);
    }
    return NULL;
}

static int resolve_threads(int nthreads)
{
    if (nthreads <= 0) {
        long c = sysconf(_SC_NPROCESSORS_ONLN);
        nthreads = c > 0 ? (int)c : 1;
    }
    return nthreads;
}

int orc_num_threads(int nthreads)
{
    return resolve_threads(nthreads);
}

static void run_modes(mode_job *tmpl, int nthreads)
{
    nthreads = resolve_threads(nthreads);
    if (nthreads > tmpl->nm)
        nthreads = tmpl->nm > 0 ? tmpl->nm : 1;
    pthread_t *th = malloc(sizeof(pthread_t) * nthreads);
    mode_job *jobs = malloc(sizeof(mode_job) * nthreads);
    for (int i = 0; i < nthreads; i++) {
        jobs[i] = *tmpl;
        jobs[i].first = i;
        jobs[i].stride = nthreads;
        pthread_create(&th[i], NULL, mode_worker, &jobs[i]);
    }
    for (int i = 0; i < nthreads; i++)
        pthread_join(th[i], NULL);
    free(th);
    free(jobs);
}

/* f(p) for a list of momenta p[nm][3] (Dirac, Eq. pair_prod_homo). */
int orc_dirac_modes(const double *A, int ld, int n_steps, double dt, const double *p, int nm,
                    int spin_sum, double *n_out, int nthreads)
{
    if (!A || !p || !n_out || nm < 0 || n_steps < 1 || ld < 2 * n_steps + 1)
        return ORC_ERR_ARG;
    mode_job J = {A, NULL, NULL, ld, n_steps, spin_sum, 0, dt, p, nm, 1, 0, n_out, NULL};
    run_modes(&J, nthreads);
    return ORC_OK;
}

/* f(p) for a list of momenta with the fourth-order Magnus step. */
int orc_dirac_magnus_modes(const double *A, int ld, int n_steps, double dt, const double *p, int nm,
                           double *n_out, double *norm_dev, int nthreads)
{
    if (!A || !p || !n_out || nm < 0 || n_steps < 1 || ld < 2 * n_steps + 1)
        return ORC_ERR_ARG;
    mode_job J = {A, NULL, NULL, ld, n_steps, 0, 3, dt, p, nm, 1, 0, n_out, norm_dev};
    run_modes(&J, nthreads);
    return ORC_OK;
}

/* f(p) for a list of momenta with the split operator; norm_dev[m] may be NULL. */
int orc_dirac_split_modes(const double *A, int ld, int n_steps, double dt, const double *p, int nm,
                          double *n_out, double *norm_dev, int nthreads)
{
    if (!A || !p || !n_out || nm < 0 || n_steps < 1 || ld < 2 * n_steps + 1)
        return ORC_ERR_ARG;
    mode_job J = {A, NULL, NULL, ld, n_steps, 0, 2, dt, p, nm, 1, 0, n_out, norm_dev};
    run_modes(&J, nthreads);
    return ORC_OK;
}

/* f(p) = 1 - chi_1 for a list of momenta (quantum kinetic equation). */
int orc_qke6_modes(const double *A, const double *E, const double *Edot, int ld, int n_steps,
                   double dt, const double *p, int nm, double *f_out, int nthreads)
{
    if (!A || !E || !Edot || !p || !f_out || nm < 0 || n_steps < 1 || ld < 2 * n_steps + 1)
        return ORC_ERR_ARG;
    mode_job J = {A, E, Edot, ld, n_steps, 0, 1, dt, p, nm, 1, 0, f_out, NULL};
    run_modes(&J, nthreads);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Local search, Sec. IV.A: the field without renormalisation and with its   */
/* time derivative, the adjoint of the QKE forward solve (Eqs. (eom2), (adj), */
/* (grad)) and the chain rule back to the B-spline parameters.               */
/* ------------------------------------------------------------------------- */

/* Field of Eq. (field) with g = 1 and no renormalisation (the local search
 * holds the fluence through the augmented Lagrangian's penalty instead): A and
 * E as orc_synth_field gives them with s = 1, Ed = dE/dt, all [c][2][ld] on the
 * half-step grid.  U_out[c] (may be NULL) = the fluence of Eq. (energy) over one
 * period, (T/2) sum_{l,j} E_{l,j}^2 (orthogonality of the modes). */
int orc_synth_raw(const double *params, int ncand, int K, int order, double wmin, double wmax,
                  double T, int n_steps, int ld, double *A, double *E, double *Ed, double *U_out)
{
    if (ncand < 0 || n_steps < 1 || ld < 2 * n_steps + 1 || !(T > 0) || !A)
        return ORC_ERR_ARG;
    int M = orc_mode_range(wmin, wmax, T, NULL);
    if (M <= 0)
        return ORC_ERR_ARG;
    double *Om = malloc(sizeof(double) * M);
    double *amp = malloc(sizeof(double) * 2 * M);
    double *ph = malloc(sizeof(double) * 2 * M);
    int status = ORC_OK;
    double h = T / (2.0 * n_steps), ti = -0.5 * T;
    for (int c = 0; c < ncand && status == ORC_OK; c++) {
        int rc = orc_spectrum(params + (size_t)c * 4 * K, K, order, wmin, wmax, T, Om, amp, ph);
        if (rc < 0) {
            status = -rc;
            break;
        }
        if (U_out) {
            double U = 0.0;
            for (int q = 0; q < 2 * M; q++)
                U += amp[q] * amp[q];
            U_out[c] = 0.5 * T * U;
        }
        for (int l = 0; l < 2; l++) {
            double *Ar = A + ((size_t)c * 2 + l) * ld;
            double *Er = E ? E + ((size_t)c * 2 + l) * ld : NULL;
            double *Dr = Ed ? Ed + ((size_t)c * 2 + l) * ld : NULL;
            for (int k = 0; k <= 2 * n_steps; k++) {
                double t = ti + (double)k * h;
                double a = 0.0, e = 0.0, d = 0.0;
                for (int m = 0; m < M; m++) {
                    double Ej = amp[l * M + m], Pj = ph[l * M + m], W = Om[m];
                    e += Ej * cos(W * t - Pj);
                    a += Ej * (sin(W * t - Pj) - sin(W * ti - Pj)) / W;
                    d -= Ej * W * sin(W * t - Pj);
                }
                Ar[k] = -a;
                if (Er)
                    Er[k] = e;
                if (Dr)
                    Dr[k] = d;
            }
        }
    }
    free(Om);
    free(amp);
    free(ph);
    return status;
}

/* The fluence U of the un-normalised field and its gradient with respect to
 * the 4K parameters: dU/da^E_{l,i} = T sum_j E_{l,j} B_i(Omega_j), zero for the
 * phase weights. */
int orc_fluence_raw(const double *params, int K, int order, double wmin, double wmax, double T,
                    double *U_out, double *dU)
{
    int M = orc_mode_range(wmin, wmax, T, NULL);
    if (M <= 0 || !U_out || !dU)
        return ORC_ERR_ARG;
    double *Om = malloc(sizeof(double) * M);
    double *amp = malloc(sizeof(double) * 2 * M);
    double *ph = malloc(sizeof(double) * 2 * M);
    double *B = malloc(sizeof(double) * K);
    int rc = orc_spectrum(params, K, order, wmin, wmax, T, Om, amp, ph);
    if (rc < 0) {
        free(Om), free(amp), free(ph), free(B);
        return -rc;
    }
    double U = 0.0;
    for (int q = 0; q < 2 * M; q++)
        U += amp[q] * amp[q];
    *U_out = 0.5 * T * U;
    for (int i = 0; i < 4 * K; i++)
        dU[i] = 0.0;
    for (int m = 0; m < M; m++) {
        orc_bspline_basis(K, order, wmin, wmax, Om[m], B);
        for (int l = 0; l < 2; l++)
            for (int i = 0; i < K; i++)
                dU[2 * l * K + i] += T * amp[l * M + m] * B[i];
    }
    free(Om), free(amp), free(ph), free(B);
    return ORC_OK;
}

/* The three coefficients of the QKE matrix of Eq. (matrix) at one sample,
 * N = Q S_Q + R S_R + 2 omega S_W (S_* the constant 0/+-1 patterns), and their
 * partial derivatives with respect to the in-plane kinetic momentum P, the
 * field E and its derivative Ed.  X = 0 (E = 0) gives Q = R = 0 and zero
 * derivatives, as qke_matrix does for R. */
typedef struct {
    double Q, R, w;
    double dQ_dP[2], dR_dP[2], dw_dP[2], dQ_dE[2], dR_dE[2], dR_dEd[2];
} qke_coef;

static void qke_coef_eval(const double P[3], const double E[2], const double Ed[2], qke_coef *c)
{
    memset(c, 0, sizeof(*c));
    double w2 = pdot2(P) + 1.0, w = sqrt(w2);
    double EE = E[0] * E[0] + E[1] * E[1];
    double EP = E[0] * P[0] + E[1] * P[1];
    double X = w2 * EE - EP * EP;
    double eperp = sqrt(1.0 + P[2] * P[2]);
    double cr = E[0] * Ed[1] - E[1] * Ed[0];
    double dcr_dE[2] = {Ed[1], -Ed[0]}, dcr_dEd[2] = {-E[1], E[0]};
    c->w = w;
    for (int a = 0; a < 2; a++)
        c->dw_dP[a] = P[a] / w;
    if (!(X > 0.0))
        return;
    double sX = sqrt(X);
    c->Q = sX / w2;
    c->R = eperp * w * cr / X;
    for (int a = 0; a < 2; a++) {
        double dX_dP = 2.0 * P[a] * EE - 2.0 * EP * E[a];
        double dX_dE = 2.0 * w2 * E[a] - 2.0 * EP * P[a];
        c->dQ_dP[a] = dX_dP / (2.0 * sX * w2) - sX * 2.0 * P[a] / (w2 * w2);
        c->dQ_dE[a] = dX_dE / (2.0 * sX * w2);
        c->dR_dP[a] = eperp * cr * (c->dw_dP[a] / X - w * dX_dP / (X * X));
        c->dR_dE[a] = eperp * w * (dcr_dE[a] / X - cr * dX_dE / (X * X));
        c->dR_dEd[a] = eperp * w * dcr_dEd[a] / X;
    }
}

/* y_j = sum_i N[i][j] x_i */
static void mat6_tvec(const double N[6][6], const double x[6], double y[6])
{
    for (int j = 0; j < 6; j++) {
        double acc = 0.0;
        for (int i = 0; i < 6; i++)
            acc += N[i][j] * x[i];
        y[j] = acc;
    }
}

/* One stage k = N y of the forward solve contributes kb (x) y to the adjoint of
 * N; its projections on S_Q, S_R and 2 S_W are the adjoints of Q, R and omega,
 * which the chain rule sends to the sample's A (through P = p - A), E and Ed. */
static void coef_adjoint(const qke_coef *c, const double kb[6], const double y[6], int k, int ld,
                         double *gA, double *gE, double *gEd)
{
    double Qb = -kb[0] * y[1] + kb[1] * y[0] + kb[4] * y[5] - kb[5] * y[4];
    double Rb = kb[1] * y[3] - kb[2] * y[4] - kb[3] * y[1] + kb[4] * y[2];
    double wb = 2.0 * (-kb[1] * y[2] + kb[2] * y[1] + kb[3] * y[4] - kb[4] * y[3]);
    for (int l = 0; l < 2; l++) {
        gA[l * ld + k] -= Qb * c->dQ_dP[l] + Rb * c->dR_dP[l] + wb * c->dw_dP[l];
        gE[l * ld + k] += Qb * c->dQ_dE[l] + Rb * c->dR_dE[l];
        gEd[l * ld + k] += Rb * c->dR_dEd[l];
    }
}

static void qke_sample(const double *A, const double *E, const double *Ed, int ld, int k,
                       const double p[3], qke_coef *c, double N[6][6])
{
    double P[3] = {p[0] - A[k], p[1] - A[ld + k], p[2]};
    double Ek[2] = {E[k], E[ld + k]};
    double Edk[2] = {Ed[k], Ed[ld + k]};
    qke_coef_eval(P, Ek, Edk, c);
    qke_matrix(P, Ek, Edk, N);
}

/* f = 1 - chi_1(t_f) of one mode by the RK4 of orc_qke6_mode and the gradient
 * of weight * f with respect to every sample of A, E and Ed, ADDED to gA, gE,
 * gEd ([2][ld] each).  The adjoint lambda of Eq. (adj) (final value
 * lambda_1 = -1, the others 0, here scaled by the weight) is carried backwards
 * through the RK4 steps as the exact adjoint of the discrete forward map, and
 * the inner product <chi, grad N lambda> of Eq. (grad) is taken stage by stage,
 * so the result is the exact derivative of the discrete objective. */
double orc_qke6_adjoint_mode(const double *A, const double *E, const double *Ed, int ld,
                             int n_steps, double dt, const double p[3], double weight, double *gA,
                             double *gE, double *gEd)
{
    double (*chi)[6] = malloc(sizeof(double[6]) * (size_t)(n_steps + 1));
    memset(chi[0], 0, sizeof(double[6]));
    chi[0][0] = 1.0;
    for (int n = 0; n < n_steps; n++) {
        double N0[6][6], Nh[6][6], N1[6][6], k1[6], k2[6], k3[6], k4[6], y[6];
        qke_coef c;
        qke_sample(A, E, Ed, ld, 2 * n, p, &c, N0);
        qke_sample(A, E, Ed, ld, 2 * n + 1, p, &c, Nh);
        qke_sample(A, E, Ed, ld, 2 * n + 2, p, &c, N1);
        mat6_vec(N0, chi[n], k1);
        for (int i = 0; i < 6; i++)
            y[i] = chi[n][i] + 0.5 * dt * k1[i];
        mat6_vec(Nh, y, k2);
        for (int i = 0; i < 6; i++)
            y[i] = chi[n][i] + 0.5 * dt * k2[i];
        mat6_vec(Nh, y, k3);
        for (int i = 0; i < 6; i++)
            y[i] = chi[n][i] + dt * k3[i];
        mat6_vec(N1, y, k4);
        for (int i = 0; i < 6; i++)
            chi[n + 1][i] = chi[n][i] + dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    }
    double f = qke_density(chi[n_steps]);
    double bar[6] = {-weight, 0, 0, 0, 0, 0};  /* d(weight f)/d chi(t_f) */
    for (int n = n_steps - 1; n >= 0; n--) {
        double N0[6][6], Nh[6][6], N1[6][6], k1[6], k2[6], k3[6], y2[6], y3[6], y4[6];
        qke_coef c0, ch, c1;
        qke_sample(A, E, Ed, ld, 2 * n, p, &c0, N0);
        qke_sample(A, E, Ed, ld, 2 * n + 1, p, &ch, Nh);
        qke_sample(A, E, Ed, ld, 2 * n + 2, p, &c1, N1);
        const double *x = chi[n];
        mat6_vec(N0, x, k1);
        for (int i = 0; i < 6; i++)
            y2[i] = x[i] + 0.5 * dt * k1[i];
        mat6_vec(Nh, y2, k2);
        for (int i = 0; i < 6; i++)
            y3[i] = x[i] + 0.5 * dt * k2[i];
        mat6_vec(Nh, y3, k3);
        for (int i = 0; i < 6; i++)
            y4[i] = x[i] + dt * k3[i];
        double kb1[6], kb2[6], kb3[6], kb4[6], xb[6], yb[6];
        for (int i = 0; i < 6; i++) {
            kb1[i] = dt / 6.0 * bar[i];
            kb2[i] = 2.0 * dt / 6.0 * bar[i];
            kb3[i] = 2.0 * dt / 6.0 * bar[i];
            kb4[i] = dt / 6.0 * bar[i];
            xb[i] = bar[i];
        }
        /* k4 = N1 y4, y4 = x + dt k3 */
        coef_adjoint(&c1, kb4, y4, 2 * n + 2, ld, gA, gE, gEd);
        mat6_tvec(N1, kb4, yb);
        for (int i = 0; i < 6; i++) {
            xb[i] += yb[i];
            kb3[i] += dt * yb[i];
        }
        /* k3 = Nh y3, y3 = x + dt/2 k2 */
        coef_adjoint(&ch, kb3, y3, 2 * n + 1, ld, gA, gE, gEd);
        mat6_tvec(Nh, kb3, yb);
        for (int i = 0; i < 6; i++) {
            xb[i] += yb[i];
            kb2[i] += 0.5 * dt * yb[i];
        }
        /* k2 = Nh y2, y2 = x + dt/2 k1 */
        coef_adjoint(&ch, kb2, y2, 2 * n + 1, ld, gA, gE, gEd);
        mat6_tvec(Nh, kb2, yb);
        for (int i = 0; i < 6; i++) {
            xb[i] += yb[i];
            kb1[i] += 0.5 * dt * yb[i];
        }
        /* k1 = N0 x */
        coef_adjoint(&c0, kb1, x, 2 * n, ld, gA, gE, gEd);
        mat6_tvec(N0, kb1, yb);
        for (int i = 0; i < 6; i++)
            bar[i] = xb[i] + yb[i];
    }
    free(chi);
    return f;
}

typedef struct {
    const double *A, *E, *Ed, *p, *w;
    int ld, n_steps, nm, first, stride;
    double dt;
    double *f, *gA, *gE, *gEd;  /* private [2][ld] accumulators */
} grad_job;

static void *grad_worker(void *arg)
{
    grad_job *J = arg;
    for (int m = J->first; m < J->nm; m += J->stride)
        J->f[m] = orc_qke6_adjoint_mode(J->A, J->E, J->Ed, J->ld, J->n_steps, J->dt, J->p + 3 * m,
                                        J->w[m], J->gA, J->gE, J->gEd);
    return NULL;
}

/* J = sum_m w[m] f(p_m) (Eq. (opt_prob) with the QKE f) for one field and the
 * gradient of J with respect to its samples: gA, gE, gEd ([2][ld], overwritten).
 * f_out[m] (may be NULL) receives each f.  Threads accumulate privately and
 * their sums are added in thread order. */
int orc_qke6_grad(const double *A, const double *E, const double *Ed, int ld, int n_steps,
                  double dt, const double *p, const double *w, int nm, double *f_out,
                  double *J_out, double *gA, double *gE, double *gEd, int nthreads)
{
    if (!A || !E || !Ed || !p || !w || !J_out || !gA || !gE || !gEd || nm < 0 || n_steps < 1 ||
        ld < 2 * n_steps + 1)
        return ORC_ERR_ARG;
    nthreads = resolve_threads(nthreads);
    if (nthreads > nm)
        nthreads = nm > 0 ? nm : 1;
    size_t G = (size_t)2 * ld;
    double *f = malloc(sizeof(double) * (nm > 0 ? nm : 1));
    double *acc = calloc((size_t)nthreads * 3 * G, sizeof(double));
    pthread_t *th = malloc(sizeof(pthread_t) * nthreads);
    grad_job *jobs = malloc(sizeof(grad_job) * nthreads);
    for (int i = 0; i < nthreads; i++) {
        grad_job j = {A, E, Ed, p, w, ld, n_steps, nm, i, nthreads, dt, f,
                      acc + (size_t)i * 3 * G, acc + (size_t)i * 3 * G + G,
                      acc + (size_t)i * 3 * G + 2 * G};
        jobs[i] = j;
        pthread_create(&th[i], NULL, grad_worker, &jobs[i]);
    }
    for (int i = 0; i < nthreads; i++)
        pthread_join(th[i], NULL);
    memset(gA, 0, sizeof(double) * G);
    memset(gE, 0, sizeof(double) * G);
    memset(gEd, 0, sizeof(double) * G);
    for (int i = 0; i < nthreads; i++)
        for (size_t q = 0; q < G; q++) {
            gA[q] += jobs[i].gA[q];
            gE[q] += jobs[i].gE[q];
            gEd[q] += jobs[i].gEd[q];
        }
    double J = 0.0;
    for (int m = 0; m < nm; m++)
        J += w[m] * f[m];
    *J_out = J;
    if (f_out)
        memcpy(f_out, f, sizeof(double) * nm);
    free(f), free(acc), free(th), free(jobs);
    return ORC_OK;
}

/* Chain rule from the samples back to the parameters of one candidate (the
 * field of orc_synth_raw): given gA, gE, gEd = dJ/d(samples) ([2][ld]),
 * grad[4K] = dJ/d[a^E_x, a^phi_x, a^E_y, a^phi_y].  With theta = Omega_j t - Phi_j
 * the samples depend on (E_{l,j}, Phi_{l,j}) through
 *   A = -E_j (sin theta_k - sin theta_i)/Omega_j, E = E_j cos theta_k,
 *   Ed = -E_j Omega_j sin theta_k,
 * and E_{l,j}, Phi_{l,j} are the B-spline sums of Eqs. (coeff_basis_E/phi). */
int orc_synth_vjp(const double *params, int K, int order, double wmin, double wmax, double T,
                  int n_steps, int ld, const double *gA, const double *gE, const double *gEd,
                  double *grad)
{
    int M = orc_mode_range(wmin, wmax, T, NULL);
    if (M <= 0 || n_steps < 1 || ld < 2 * n_steps + 1 || !grad)
        return ORC_ERR_ARG;
    double *Om = malloc(sizeof(double) * M);
    double *amp = malloc(sizeof(double) * 2 * M);
    double *ph = malloc(sizeof(double) * 2 * M);
    double *B = malloc(sizeof(double) * K);
    int rc = orc_spectrum(params, K, order, wmin, wmax, T, Om, amp, ph);
    if (rc < 0) {
        free(Om), free(amp), free(ph), free(B);
        return -rc;
    }
    for (int i = 0; i < 4 * K; i++)
        grad[i] = 0.0;
    double h = T / (2.0 * n_steps), ti = -0.5 * T;
    for (int m = 0; m < M; m++) {
        double W = Om[m];
        orc_bspline_basis(K, order, wmin, wmax, W, B);
        for (int l = 0; l < 2; l++) {
            double Ej = amp[l * M + m], Pj = ph[l * M + m];
            double si = sin(W * ti - Pj), ci = cos(W * ti - Pj);
            double dE = 0.0, dP = 0.0;
            for (int k = 0; k <= 2 * n_steps; k++) {
                double t = ti + (double)k * h;
                double sk = sin(W * t - Pj), ck = cos(W * t - Pj);
                double ga = gA[l * ld + k], ge = gE[l * ld + k], gd = gEd[l * ld + k];
                dE += ga * (-(sk - si) / W) + ge * ck + gd * (-W * sk);
                dP += ga * (Ej * (ck - ci) / W) + ge * (Ej * sk) + gd * (Ej * W * ck);
            }
            for (int i = 0; i < K; i++) {
                grad[2 * l * K + i] += B[i] * dE;
                grad[(2 * l + 1) * K + i] += B[i] * dP;
            }
        }
    }
    free(Om), free(amp), free(ph), free(B);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Momentum integral, Eq. (opt_prob): N = int_D d^3p f                        */
/* ------------------------------------------------------------------------- */

/* Trapezoid weights of a linspace(a, b, n) axis (endpoints included).  With
 * mirror = 1 the axis is the non-negative half [0, b] of the symmetric axis
 * [-b, b] and the weights are those of the trapezoid rule on the full axis:
 * a point p > 0 stands for +p and -p (twice its half-axis weight) and p = 0 is
 * an interior point of the full axis (weight d = twice its half-axis d/2).
 * Both cases double the half-axis weight.  A single-point axis has weight 1. */
void orc_trapz_weights(int n, double a, double b, int mirror, double *w)
{
    if (n == 1) {
        w[0] = 1.0;
        return;
    }
    double d = (b - a) / (double)(n - 1);
    for (int i = 0; i < n; i++) {
        w[i] = (i == 0 || i == n - 1) ? 0.5 * d : d;
        if (mirror)
            w[i] = 2.0 * w[i];
    }
}

static double axis_point(int i, int n, double a, double b)
{
    return n == 1 ? a : a + (b - a) * (double)i / (double)(n - 1);
}

/* Pair number N[c] = sum_p w(p) f_c(p) over the grid p = (x_i, y_j, z_k),
 * x fastest (n_p[c][k][j][i]).  Candidate c uses n_steps[c] steps and the
 * potential rows A + c*2*ld.  n_out may be NULL.  The sum is taken serially
 * in grid order, so the result does not depend on the thread count. */
int orc_pair_number(const double *A, int ncand, int ld, const int *n_steps, double dt, int nx,
                    int ny, int nz, double x0, double x1, double y0, double y1, double z0,
                    double z1, int mirror_z, int spin_sum, double *n_out, double *N_out,
                    int nthreads)
{
    if (!A || !n_steps || !N_out || ncand < 0 || nx < 1 || ny < 1 || nz < 1)
        return ORC_ERR_ARG;
    int nm = nx * ny * nz;
    double *p = malloc(sizeof(double) * 3 * nm);
    double *wgt = malloc(sizeof(double) * nm);
    double *wx = malloc(sizeof(double) * nx), *wy = malloc(sizeof(double) * ny),
           *wz = malloc(sizeof(double) * nz);
    orc_trapz_weights(nx, x0, x1, 0, wx);
    orc_trapz_weights(ny, y0, y1, 0, wy);
    orc_trapz_weights(nz, z0, z1, mirror_z, wz);
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                int m = (k * ny + j) * nx + i;
                p[3 * m + 0] = axis_point(i, nx, x0, x1);
                p[3 * m + 1] = axis_point(j, ny, y0, y1);
                p[3 * m + 2] = axis_point(k, nz, z0, z1);
                wgt[m] = wx[i] * wy[j] * wz[k];
            }
    double *nbuf = malloc(sizeof(double) * nm);
    int status = ORC_OK;
    for (int c = 0; c < ncand; c++) {
        if (n_steps[c] < 1 || ld < 2 * n_steps[c] + 1) {
            status = ORC_ERR_ARG;
            break;
        }
        orc_dirac_modes(A + (size_t)c * 2 * ld, ld, n_steps[c], dt, p, nm, spin_sum, nbuf, nthreads);
        double N = 0.0;
        for (int m = 0; m < nm; m++)
            N += wgt[m] * nbuf[m];
        N_out[c] = N;
        if (n_out)
            memcpy(n_out + (size_t)c * nm, nbuf, sizeof(double) * nm);
    }
    free(p);
    free(wgt);
    free(wx);
    free(wy);
    free(wz);
    free(nbuf);
    return status;
}

/* ------------------------------------------------------------------------- */
/* Differential evolution, DE/rand/1/bin, Sec. IV.B                          */
/* ------------------------------------------------------------------------- */

/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the k-th output (k = 0,1,..)
 * of the generator seeded with `seed` is mix(seed + (k+1) * gamma). */
uint64_t orc_splitmix64_at(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Random-number slots of individual i in generation g: the stream key is
 * splitmix64_at(splitmix64_at(seed, g), i); slots 0..61 feed the rejection
 * draws of the three donors, slot 62 the forced index R, slot 64 + j the
 * crossover number of coordinate j. */
#define DE_SLOT_R 62
#define DE_SLOT_CROSS 64
#define DE_MAX_DRAWS 62

static double u01(uint64_t x)
{
    return (double)(x >> 11) * 0x1.0p-53;
}

static int below(uint64_t x, int n)
{
    return (int)(((x >> 32) * (uint64_t)n) >> 32);
}

/* Steps 1-3 of DE/rand/1/bin for every individual i:
 *  1. three distinct donors a, b, c, all different from i;
 *  2. mutation u = a + F (b - c);
 *  3. binomial crossover: y_j = u_j if r_j <= CR or j == R, else x_ij.
 * Coordinates taken from u are brought back into bounds: periodic ones
 * (phases) are wrapped into [lo, hi), the others clipped to [lo, hi].
 * The paper does not say how the donors are drawn; here each is drawn by
 * rejection from at most 62 random slots, and if the slots run out (possible
 * only for tiny populations) the trial is a copy of the parent.
 * pop[NP][D] -> trial[NP][D].  Returns ORC_ERR_ARG when NP < 4. */
int orc_de_propose(const double *pop, int NP, int D, const double *lo, const double *hi,
                   const uint8_t *periodic, double F, double CR, uint64_t seed, uint64_t gen,
                   double *trial)
{
    if (NP < 4 || D < 1 || D > 4096 || !pop || !trial || !lo || !hi)
        return ORC_ERR_ARG;
    uint64_t gkey = orc_splitmix64_at(seed, gen);
    for (int i = 0; i < NP; i++) {
        uint64_t key = orc_splitmix64_at(gkey, (uint64_t)i);
        int r[3] = {-1, -1, -1};
        int slot = 0, found_all = 1;
        for (int q = 0; q < 3 && found_all; q++) {
            found_all = 0;
            while (slot < DE_MAX_DRAWS) {
                int cand = below(orc_splitmix64_at(key, (uint64_t)slot++), NP);
                int clash = (cand == i);
                for (int z = 0; z < q; z++)
                    clash |= (cand == r[z]);
                if (!clash) {
                    r[q] = cand;
                    found_all = 1;
                    break;
                }
            }
        }
        if (!found_all) {
            /* the donor draws ran out of random slots: the trial is the parent */
            memcpy(trial + (size_t)i * D, pop + (size_t)i * D, sizeof(double) * D);
            continue;
        }
        int R = below(orc_splitmix64_at(key, DE_SLOT_R), D);
        const double *xa = pop + (size_t)r[0] * D, *xb = pop + (size_t)r[1] * D,
                     *xc = pop + (size_t)r[2] * D, *xi = pop + (size_t)i * D;
        double *y = trial + (size_t)i * D;
        for (int j = 0; j < D; j++) {
            double rj = u01(orc_splitmix64_at(key, (uint64_t)(DE_SLOT_CROSS + j)));
            if (rj <= CR || j == R) {
                double diff = xb[j] - xc[j];
                double step = F * diff;
                double u = xa[j] + step;
                if (periodic && periodic[j]) {
                    double period = hi[j] - lo[j];
                    double off = fmod(u - lo[j], period);
                    if (off < 0.0)
                        off = off + period;
                    u = lo[j] + off;
                    if (u >= hi[j])
                        u = lo[j];
                } else {
                    if (u < lo[j])
                        u = lo[j];
                    if (u > hi[j])
                        u = hi[j];
                }
                y[j] = u;
            } else {
                y[j] = xi[j];
            }
        }
    }
    return ORC_OK;
}

/* Step 4, read for maximisation of N: x is replaced by y when N(y) >= N(x)
 * (ties go to the trial).  A NaN trial fitness never replaces. */
int orc_de_select(double *pop, double *fit, const double *trial, const double *trial_fit, int NP,
                  int D)
{
    if (NP < 1 || D < 1 || !pop || !fit || !trial || !trial_fit)
        return ORC_ERR_ARG;
    for (int i = 0; i < NP; i++) {
        if (trial_fit[i] >= fit[i]) {
            memcpy(pop + (size_t)i * D, trial + (size_t)i * D, sizeof(double) * D);
            fit[i] = trial_fit[i];
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Host mirror of the library's entry points                                 */
/* ------------------------------------------------------------------------- */

/* pp_oracle_* take the arguments of the CUDA library's pp_synth_field,
 * pp_pair_number, pp_de_propose, pp_de_select and pp_de_step, in the same order
 * and with the same meaning, but every array is a HOST pointer, the work is done
 * here on the CPU in FP64 and `stream` is ignored (the call returns when done).
 * The two structs below have the layout of the library's pulse model and
 * momentum grid; they are declared here again because the oracle shares no
 * header with the library.  Return values use the library's codes for the
 * cases the oracle detects: 0 = OK, 1 = invalid argument, 4 = zero-fluence
 * pulse. */
typedef struct {
    int32_t K;
    int32_t order;
    double w_min;
    double w_max;
    double T;
    double fluence;
    int32_t n_steps;
    int32_t envelope; /* 0: g(t) = 1; 1: Hann envelope, Eq. (hann) */
} orc_field_spec;

typedef struct {
    int32_t nx, ny, nz;
    double x0, x1, y0, y1, z0, z1;
    int32_t mirror_z;
} orc_grid;

enum { ORC_RK4 = 0, ORC_MAGNUS4 = 1, ORC_SPLIT2 = 2 };

/* Eqs. (field), (energy), (hann), (vector_potential): as orc_synth_field
 * (envelope 0) or orc_synth_hann with renormalisation (envelope 1). */
int pp_oracle_synth_field(const double *params, int32_t ncand, const orc_field_spec *spec, double *A,
                          int32_t ld, double *E, double *scale, void *stream)
{
    (void)stream;
    if (!spec || (ncand > 0 && (!params || !A)) || (spec->envelope != 0 && spec->envelope != 1))
        return ORC_ERR_ARG;
    if (spec->envelope == 1)
        return orc_synth_hann(params, ncand, spec->K, spec->order, spec->w_min, spec->w_max, spec->T,
                              spec->fluence, 1, spec->n_steps, ld, A, E, NULL, scale);
    return orc_synth_field(params, ncand, spec->K, spec->order, spec->w_min, spec->w_max, spec->T,
                           spec->fluence, spec->n_steps, ld, A, E, scale);
}

/* Eq. (opt_prob) with the full spin trace of Eq. (pair_prod_homo): every mode
 * integrated in FP64 with the requested scheme (classical RK4, the fourth-order
 * Magnus step or the split operator); `precision` is checked and otherwise
 * ignored (the oracle is FP64 throughout).  N = sum_p w(p) f(p) in grid order. */
int pp_oracle_pair_number(const double *A, int32_t ncand, int32_t ld, const int32_t *n_steps, double dt,
                          const orc_grid *grid, int32_t precision, int32_t scheme, double *N, double *n_p,
                          void *stream)
{
    (void)stream;
    if (!grid || ncand < 0 || (ncand > 0 && (!A || !N)) || !(dt > 0.0) || precision < 0 || precision > 2 ||
        scheme < ORC_RK4 || scheme > ORC_SPLIT2 || grid->nx < 1 || grid->ny < 1 || grid->nz < 1)
        return ORC_ERR_ARG;
    const int nx = grid->nx, ny = grid->ny, nz = grid->nz, nm = nx * ny * nz;
    double *p = malloc(sizeof(double) * 3 * (size_t)nm), *wgt = malloc(sizeof(double) * (size_t)nm);
    double *wx = malloc(sizeof(double) * nx), *wy = malloc(sizeof(double) * ny), *wz = malloc(sizeof(double) * nz);
    double *nbuf = malloc(sizeof(double) * (size_t)nm);
    orc_trapz_weights(nx, grid->x0, grid->x1, 0, wx);
    orc_trapz_weights(ny, grid->y0, grid->y1, 0, wy);
    orc_trapz_weights(nz, grid->z0, grid->z1, grid->mirror_z, wz);
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                const int m = (k * ny + j) * nx + i;
                p[3 * m + 0] = axis_point(i, nx, grid->x0, grid->x1);
                p[3 * m + 1] = axis_point(j, ny, grid->y0, grid->y1);
                p[3 * m + 2] = axis_point(k, nz, grid->z0, grid->z1);
                wgt[m] = wx[i] * wy[j] * wz[k];
            }
    int status = ORC_OK;
    for (int c = 0; c < ncand && status == ORC_OK; c++) {
        const int ns = n_steps ? n_steps[c] : (ld - 1) / 2;
        if (ns < 1 || ld < 2 * ns + 1) {
            status = ORC_ERR_ARG;
            break;
        }
        const double *Ac = A + (size_t)c * 2 * ld;
        if (scheme == ORC_RK4)
            status = orc_dirac_modes(Ac, ld, ns, dt, p, nm, 0, nbuf, 0);
        else if (scheme == ORC_MAGNUS4)
            status = orc_dirac_magnus_modes(Ac, ld, ns, dt, p, nm, nbuf, NULL, 0);
        else
            status = orc_dirac_split_modes(Ac, ld, ns, dt, p, nm, nbuf, NULL, 0);
        double s = 0.0;
        for (int m = 0; m < nm; m++)
            s += wgt[m] * nbuf[m];
        N[c] = s;
        if (n_p)
            memcpy(n_p + (size_t)c * nm, nbuf, sizeof(double) * (size_t)nm);
    }
    free(p);
    free(wgt);
    free(wx);
    free(wy);
    free(wz);
    free(nbuf);
    return status;
}

/* Sec. IV.B, steps 1-3 (orc_de_propose). */
int pp_oracle_de_propose(const double *pop, int32_t NP, int32_t D, const double *lo, const double *hi,
                         const uint8_t *periodic, double F, double CR, uint64_t seed, uint64_t generation,
                         double *trial, void *stream)
{
    (void)stream;
    return orc_de_propose(pop, NP, D, lo, hi, periodic, F, CR, seed, generation, trial);
}

/* Sec. IV.B, step 4 (orc_de_select). */
int pp_oracle_de_select(double *pop, double *fit, const double *trial, const double *trial_fit, int32_t NP,
                        int32_t D, void *stream)
{
    (void)stream;
    return orc_de_select(pop, fit, trial, trial_fit, NP, D);
}

/* One generation of Sec. IV.B: propose, synthesise the trials (Sec. III),
 * score them (Sec. II.A, Eq. (opt_prob)), select.  D = 4 K; the trials take
 * spec->n_steps steps of dt = T / n_steps.  trial_out [NP][D] and
 * trial_fit_out [NP] receive the proposals and their pair numbers (may be NULL). */
int pp_oracle_de_step(double *pop, double *fit, int32_t NP, const orc_field_spec *spec, const orc_grid *grid,
                      int32_t precision, int32_t scheme, const double *lo, const double *hi, const uint8_t *periodic,
                      double F, double CR, uint64_t seed, uint64_t generation, double *trial_out,
                      double *trial_fit_out, void *stream)
{
    (void)stream;
    if (!spec || !grid || !pop || !fit || NP < 4 || spec->n_steps < 1 || !(spec->T > 0.0))
        return ORC_ERR_ARG;
    const int D = 4 * spec->K, ld = 2 * spec->n_steps + 1;
    double *trial = malloc(sizeof(double) * (size_t)NP * D), *tfit = malloc(sizeof(double) * (size_t)NP);
    double *A = malloc(sizeof(double) * (size_t)NP * 2 * ld);
    int status = orc_de_propose(pop, NP, D, lo, hi, periodic, F, CR, seed, generation, trial);
    if (status == ORC_OK)
        status = pp_oracle_synth_field(trial, NP, spec, A, ld, NULL, NULL, NULL);
    if (status == ORC_OK)
        status = pp_oracle_pair_number(A, NP, ld, NULL, spec->T / spec->n_steps, grid, precision, scheme, tfit,
                                       NULL, NULL);
    if (status == ORC_OK) {
        if (trial_out)
            memcpy(trial_out, trial, sizeof(double) * (size_t)NP * D);
        if (trial_fit_out)
            memcpy(trial_fit_out, tfit, sizeof(double) * (size_t)NP);
        status = orc_de_select(pop, fit, trial, tfit, NP, D);
    }
    free(trial);
    free(tfit);
    free(A);
    return status;
}
