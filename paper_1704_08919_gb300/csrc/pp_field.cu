// pp_field.cu -- pulse synthesis: B-spline spectral parameters -> A(t), E(t)
// (Sec. III of arXiv 1704.08919, Eqs. (coeff_basis_E), (coeff_basis_phi),
// (field), (energy); global renormalisation to U_const at every DE update,
// Sec. IV.B).
//
// With g(t) = 1 and the DC term removed, on the half-step grid
//     t_k = -T/2 + k h,  h = T / (2 n),  Omega_j = j 2 pi / T,
// the phases are Omega_j t_k = -j pi + pi j k / n, so with z_k = exp(i pi k / n)
//     E_l(t_k) = Re sum_j C_j z_k^j,         C_j = s E~_j e^{-i Phi_j} (-1)^j
//     A_l(t_k) = -Im sum_j D_j (z_k^j - 1),  D_j = C_j / Omega_j
// (A = -int_{-T/2}^t E, so A(-T/2) = 0 and, by periodicity, A(T/2) = 0).
// Each sum is evaluated by Horner's rule in z_k after factoring z_k^{j_first};
// z_k comes from sincospi of an exactly reduced argument.  The fluence of the
// unit-scale field over one period is (T/2) sum_{l,j} E~_{l,j}^2, and
// s = sqrt(U_const / that).
#include <math.h>

#include <vector>

#include "pp_internal.cuh"

namespace {

constexpr int kMaxK = 64;
constexpr int kMaxOrder = 8;

// Cox-de Boor recursion on the clamped knot vector (order copies of w_min,
// equidistant interior breakpoints, order copies of w_max); order-1 indicators
// of [t_i, t_{i+1}) with the last non-empty interval closed on the right.
__device__ void bspline_basis(int K, int order, double wmin, double wmax, double w, double *B)
{
    double t[kMaxK + kMaxOrder];
    double b[kMaxK + kMaxOrder];
    const int nk = K + order;
    const int nbrk = K - order + 2;
    for (int i = 0; i < order; ++i) {
        t[i] = wmin;
        t[K + i] = wmax;
    }
    for (int i = 1; i < nbrk - 1; ++i)
        t[order - 1 + i] = wmin + (wmax - wmin) * (double)i / (double)(nbrk - 1);
    int last = -1;
    for (int i = 0; i < nk - 1; ++i)
        if (t[i] < t[i + 1])
            last = i;
    for (int i = 0; i < nk - 1; ++i) {
        bool inside = (t[i] <= w && w < t[i + 1]) || (i == last && w == t[i + 1]);
        b[i] = inside ? 1.0 : 0.0;
    }
    for (int r = 2; r <= order; ++r) {
        for (int i = 0; i < nk - r; ++i) {
            double d1 = t[i + r - 1] - t[i], d2 = t[i + r] - t[i + 1];
            double left = d1 > 0.0 ? (w - t[i]) / d1 * b[i] : 0.0;
            double right = d2 > 0.0 ? (t[i + r] - w) / d2 * b[i + 1] : 0.0;
            b[i] = left + right;
        }
    }
    for (int i = 0; i < K; ++i)
        B[i] = b[i];
}

// Block-wide sum of one value per thread (blockDim.x a power of two <= 256).
__device__ double block_sum(double v)
{
    __shared__ double red[256];
    __syncthreads();  // red may still be read by a previous call
    red[threadIdx.x] = v;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    return red[0];
}

// One block per candidate: spectrum at every mode, fluence, scale, and the
// Horner coefficients cf[l][m] = C, cf[l][M + m] = D for mode j = j0 + m
// (cf: this candidate's 4 M coefficients; scale_out: its scale slot or NULL).
__device__ void spectrum_block(const double *__restrict__ prm, int K, int order, double wmin, double wmax,
                               double T, double U, int j0, int M, double2 *__restrict__ cf,
                               double *__restrict__ scale_out, unsigned int *__restrict__ status, int normalize)
{
    const double dw = 2.0 * M_PI / T;
    double ssq = 0.0;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const int j = j0 + m;
        const double W = (double)j * dw;
        double B[kMaxK];
        bspline_basis(K, order, wmin, wmax, W, B);
        for (int l = 0; l < 2; ++l) {
            double e = 0.0, ph = 0.0;
            for (int i = 0; i < K; ++i) {
                e += prm[(2 * l) * K + i] * B[i];
                ph += prm[(2 * l + 1) * K + i] * B[i];
            }
            ssq += e * e;
            double sn, cs;
            sincos(ph, &sn, &cs);
            const double sg = (j & 1) ? -1.0 : 1.0;
            // unit-scale C_j = E~ e^{-i Phi} (-1)^j ; the scale is applied below
            cf[(size_t)l * 2 * M + m] = make_double2(sg * e * cs, -sg * e * sn);
            cf[(size_t)l * 2 * M + M + m] = make_double2(sg * e * cs / W, -sg * e * sn / W);
        }
    }
    const double Uraw = 0.5 * T * block_sum(ssq);
    // normalize = 0: the un-normalised field (s = 1) and scale_out receives its fluence
    const double s = normalize ? (Uraw > 0.0 ? sqrt(U / Uraw) : 0.0) : 1.0;
    if (threadIdx.x == 0) {
        if (normalize && !(Uraw > 0.0))
            pp_flag(status, PP_FLAG_DEGENERATE);
        if (scale_out)
            *scale_out = normalize ? s : Uraw;
    }
    for (int q = threadIdx.x; q < 4 * M; q += blockDim.x) {
        const double2 v = cf[q];
        cf[q] = make_double2(s * v.x, s * v.y);
    }
}

// The Hann envelope of Eq. (hann), g(t) = cos^2(pi t / T) = 1/2 + 1/2 cos(dOmega t),
// keeps the field a trigonometric polynomial on the same harmonic grid: mode j feeds
// harmonics j and j +- 1 with weights 1/2 and 1/4.  With the (-1)^j phase factor of
// the stored coefficients, C'_j = C_j / 2 - C_{j-1} / 4 - C_{j+1} / 4 for the
// harmonics j0 - 1 .. j1 + 1 (Mp = M + 2 of them, starting at j0p = j0 - 1).  A
// harmonic j = 0 (when j0 = 1) is the DC part of E: D'_0 = 0 and the samples add
// its potential c0 (t_f - t) (the gauge A(t_f) = 0 of Eq. (vector_potential)).  The
// fluence is (T/2) sum_{j >= 1} |C'_j|^2 + T c0^2.  Layout as spectrum_block, with
// Mp in place of M (cf: 4 Mp coefficients).
__device__ void hann_spectrum_block(const double *__restrict__ prm, int K, int order, double wmin, double wmax,
                                    double T, double U, int j0, int M, double2 *__restrict__ cf,
                                    double *__restrict__ scale_out, unsigned int *__restrict__ status,
                                    int normalize)
{
    const int Mp = M + 2, j0p = j0 - 1;
    const double dw = 2.0 * M_PI / T;
    // unit-scale C_j of mode j = j0 + m into slot m + 1 of the D region (slots 0 and M+1 zero)
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const int j = j0 + m;
        double B[kMaxK];
        bspline_basis(K, order, wmin, wmax, (double)j * dw, B);
        for (int l = 0; l < 2; ++l) {
            double e = 0.0, ph = 0.0;
            for (int i = 0; i < K; ++i) {
                e += prm[(2 * l) * K + i] * B[i];
                ph += prm[(2 * l + 1) * K + i] * B[i];
            }
            double sn, cs;
            sincos(ph, &sn, &cs);
            const double sg = (j & 1) ? -1.0 : 1.0;
            cf[(size_t)l * 2 * Mp + Mp + m + 1] = make_double2(sg * e * cs, -sg * e * sn);
        }
    }
    if (threadIdx.x < 2) {
        cf[(size_t)threadIdx.x * 2 * Mp + Mp] = make_double2(0.0, 0.0);
        cf[(size_t)threadIdx.x * 2 * Mp + Mp + M + 1] = make_double2(0.0, 0.0);
    }
    __syncthreads();
    double ssq = 0.0;
    for (int q = threadIdx.x; q < 2 * Mp; q += blockDim.x) {
        const int l = q / Mp, m = q % Mp;
        const double2 *u = cf + (size_t)l * 2 * Mp + Mp;  // untransformed, slot m = harmonic j0p + m
        const double2 cm = u[m], cl = m > 0 ? u[m - 1] : make_double2(0.0, 0.0),
                      cr = m + 1 < Mp ? u[m + 1] : make_double2(0.0, 0.0);
        const double2 v = make_double2(0.5 * cm.x - 0.25 * cl.x - 0.25 * cr.x, 0.5 * cm.y - 0.25 * cl.y - 0.25 * cr.y);
        cf[(size_t)l * 2 * Mp + m] = v;
        ssq += (j0p + m == 0) ? 2.0 * v.x * v.x : v.x * v.x + v.y * v.y;
    }
    // block_sum's barriers also order the C' writes above before the reads below
    const double Uraw = 0.5 * T * block_sum(ssq);
    const double s = normalize ? (Uraw > 0.0 ? sqrt(U / Uraw) : 0.0) : 1.0;
    if (threadIdx.x == 0) {
        if (normalize && !(Uraw > 0.0))
            pp_flag(status, PP_FLAG_DEGENERATE);
        if (scale_out)
            *scale_out = normalize ? s : Uraw;
    }
    for (int q = threadIdx.x; q < 2 * Mp; q += blockDim.x) {
        const int l = q / Mp, m = q % Mp;
        double2 *c = cf + (size_t)l * 2 * Mp;
        const double2 v = make_double2(s * c[m].x, s * c[m].y);
        const double W = (double)(j0p + m) * dw;
        c[m] = v;
        c[Mp + m] = W > 0.0 ? make_double2(v.x / W, v.y / W) : make_double2(0.0, 0.0);
    }
}

__global__ void spectrum_kernel(const double *__restrict__ params, int K, int order, double wmin,
                                double wmax, double T, double U, int j0, int M,
                                double2 *__restrict__ coef, double *__restrict__ scale_out,
                                unsigned int *__restrict__ status, int normalize)
{
    const int c = blockIdx.x;
    spectrum_block(params + (size_t)c * 4 * K, K, order, wmin, wmax, T, U, j0, M, coef + (size_t)c * 4 * M,
                   scale_out ? scale_out + c : nullptr, status, normalize);
}

__global__ void hann_spectrum_kernel(const double *__restrict__ params, int K, int order, double wmin,
                                     double wmax, double T, double U, int j0, int M,
                                     double2 *__restrict__ coef, double *__restrict__ scale_out,
                                     unsigned int *__restrict__ status, int normalize)
{
    const int c = blockIdx.x;
    hann_spectrum_block(params + (size_t)c * 4 * K, K, order, wmin, wmax, T, U, j0, M,
                        coef + (size_t)c * 4 * (M + 2), scale_out ? scale_out + c : nullptr, status, normalize);
}

// Samples: grid (ceil(nsamp / 256), ncand, 2 polarisations).  Horner's rule in
// FP64 with explicit fused multiply-adds, per complex step z (x) + X_m:
// (xr zc - xi zs + Xr, xr zs + xi zc + Xi).  WANT_E / WANT_ED compile the
// accumulations of E and dE/dt in only when the caller asked for them.
template <bool WANT_E, bool WANT_ED>
__global__ void samples_kernel(const double2 *__restrict__ coef, int M, int j0, int n_steps,
                               int ld, double *__restrict__ A, double *__restrict__ E, double dw,
                               double *__restrict__ Ed, double T)
{
    extern __shared__ double2 sc[];  // [2M]: C then D
    __shared__ double s_d0i;
    const int c = blockIdx.y, l = blockIdx.z;
    const double2 *cf = coef + ((size_t)c * 2 + l) * 2 * M;
    for (int q = threadIdx.x; q < 2 * M; q += blockDim.x)
        sc[q] = cf[q];
    __syncthreads();
    if (threadIdx.x == 0) {  // Im of the sum of D_j (the z = 1 value), the same for every sample
        double d0i = 0.0;
        for (int m = M - 1; m >= 0; --m)
            d0i += sc[M + m].y;
        s_d0i = d0i;
    }
    __syncthreads();
    const int nsamp = 2 * n_steps + 1;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nsamp)
        return;
    // z = exp(i pi k / n), zj0 = z^{j0}; arguments reduced exactly modulo 2n
    const long long two_n = 2ll * n_steps;
    double zs, zc, js, jc;
    sincospi((double)(k % two_n) / (double)n_steps, &zs, &zc);
    sincospi((double)(((long long)k * j0) % two_n) / (double)n_steps, &js, &jc);
    // Horner: sum_{m=0}^{M-1} X_m z^m
    double cr = 0.0, ci = 0.0, dr = 0.0, di = 0.0, gr = 0.0, gi = 0.0;
    for (int m = M - 1; m >= 0; --m) {
        const double2 D = sc[M + m];
        const double tr = fma(dr, zc, fma(-di, zs, D.x));
        di = fma(dr, zs, fma(di, zc, D.y));
        dr = tr;
        if constexpr (WANT_E) {
            const double2 C = sc[m];
            const double ur = fma(cr, zc, fma(-ci, zs, C.x));
            ci = fma(cr, zs, fma(ci, zc, C.y));
            cr = ur;
        }
        if constexpr (WANT_ED) {  // dE/dt: coefficients i Omega_j C_j
            const double2 C = sc[m];
            const double W = (double)(j0 + m) * dw;
            const double vr = fma(gr, zc, fma(-gi, zs, -W * C.y));
            gi = fma(gr, zs, fma(gi, zc, W * C.x));
            gr = vr;
        }
    }
    // multiply by z^{j0}
    const double Di = fma(dr, js, di * jc);
    double *Arow = A + ((size_t)c * 2 + l) * ld;
    double a = -(Di - s_d0i);
    if (j0 == 0)  // DC harmonic (Hann envelope): potential c0 (t_f - t_k)
        a += sc[0].x * ((double)(2 * n_steps - k) * (T / (2.0 * n_steps)));
    Arow[k] = a;
    if constexpr (WANT_E)
        E[((size_t)c * 2 + l) * ld + k] = fma(cr, jc, -ci * js);
    if constexpr (WANT_ED)
        Ed[((size_t)c * 2 + l) * ld + k] = fma(gr, jc, -gi * js);
}

// ---- chain rule of the un-normalised synthesis (the local search's gradient):
// with theta_k = Omega_j t_k - Phi_j = pi j k / n - (j pi + Phi_j), the samples
// depend on (E_j, Phi_j) through A = -E_j (sin theta_k - sin theta_0) / Omega_j,
// E = E_j cos theta_k, Ed = -E_j Omega_j sin theta_k.  One block per (mode j,
// polarisation l, candidate): dEP = (dJ/dE_j, dJ/dPhi_j) from dJ/d(samples)
// g[c][q][k], q = (A_x, A_y, E_x, E_y, Ed_x, Ed_y).
constexpr int kVjpThreads = 256;
constexpr int kVjpResync = 32;
__global__ void __launch_bounds__(kVjpThreads) vjp_modes_kernel(
    const double *__restrict__ params, int K, int order, double wmin, double wmax, double T, int j0,
    int n_steps, const double *__restrict__ g, int ldg, double2 *__restrict__ dEP)
{
    __shared__ double sh[3];
    __shared__ double red[2][kVjpThreads];
    const int m = blockIdx.x, l = blockIdx.y, c = blockIdx.z, M = gridDim.x;
    const int j = j0 + m;
    const double W = (double)j * (2.0 * M_PI / T);
    if (threadIdx.x == 0) {
        double B[kMaxK];
        bspline_basis(K, order, wmin, wmax, W, B);
        const double *prm = params + (size_t)c * 4 * K;
        double e = 0.0, ph = 0.0;
        for (int i = 0; i < K; ++i) {
            e += prm[(2 * l) * K + i] * B[i];
            ph += prm[(2 * l + 1) * K + i] * B[i];
        }
        double sn, cs;
        sincos(ph, &sn, &cs);
        const double sg = (j & 1) ? -1.0 : 1.0;
        sh[0] = e;
        sh[1] = sg * cs;  // cos(j pi + Phi)
        sh[2] = sg * sn;  // sin(j pi + Phi)
    }
    __syncthreads();
    const double Ej = sh[0], cb = sh[1], sb = sh[2];
    const double si = -sb, ci = cb;  // theta_0 = -(j pi + Phi)
    const double *gA = g + ((size_t)c * 6 + l) * ldg;
    const double *gE = g + ((size_t)c * 6 + 2 + l) * ldg;
    const double *gD = g + ((size_t)c * 6 + 4 + l) * ldg;
    const long long two_n = 2ll * n_steps;
    // (sin, cos)(pi j k / n) by rotation from sample to sample (stride kVjpThreads),
    // recomputed exactly every kVjpResync samples
    double sr, cr;
    sincospi((double)(((long long)j * kVjpThreads) % two_n) / (double)n_steps, &sr, &cr);
    const double iW = 1.0 / W, EjiW = Ej / W, EjW = Ej * W;
    double dE = 0.0, dP = 0.0, sa = 0.0, ca = 1.0;
    int it = 0;
    for (int k = threadIdx.x; k <= 2 * n_steps; k += kVjpThreads, ++it) {
        if (it % kVjpResync == 0)
            sincospi((double)(((long long)j * k) % two_n) / (double)n_steps, &sa, &ca);
        const double ck = ca * cb + sa * sb, sk = sa * cb - ca * sb;
        const double ga = gA[k], ge = gE[k], gd = gD[k];
        dE += ga * (-(sk - si) * iW) + ge * ck + gd * (-W * sk);
        dP += ga * ((ck - ci) * EjiW) + ge * (Ej * sk) + gd * (EjW * ck);
        const double sn = fma(sa, cr, ca * sr);
        ca = fma(ca, cr, -sa * sr);
        sa = sn;
    }
    red[0][threadIdx.x] = dE;
    red[1][threadIdx.x] = dP;
    __syncthreads();
    for (int h = kVjpThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            red[0][threadIdx.x] += red[0][threadIdx.x + h];
            red[1][threadIdx.x] += red[1][threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        dEP[((size_t)c * 2 + l) * M + m] = make_double2(red[0][0], red[1][0]);
}

// One block per candidate, one thread per parameter o = (2l + kind) K + i:
// grad_o = sum_j B_i(Omega_j) dEP[l][j].{E or Phi}; the un-normalised fluence
// U = (T/2) sum E_{l,j}^2 and dU_o = T sum_j E_{l,j} B_i(Omega_j) (0 for phases).
__global__ void vjp_params_kernel(const double *__restrict__ params, int K, int order, double wmin,
                                  double wmax, double T, int j0, int M, const double2 *__restrict__ dEP,
                                  double *__restrict__ grad, double *__restrict__ U_out,
                                  double *__restrict__ dU)
{
    const int c = blockIdx.x;
    const double *prm = params + (size_t)c * 4 * K;
    const double dw = 2.0 * M_PI / T;
    for (int o = threadIdx.x; o < 4 * K; o += blockDim.x) {
        const int l = o / (2 * K), kind = (o / K) % 2, i = o % K;
        double acc = 0.0, accU = 0.0;
        for (int m = 0; m < M; ++m) {
            double B[kMaxK];
            bspline_basis(K, order, wmin, wmax, (double)(j0 + m) * dw, B);
            const double2 v = dEP[((size_t)c * 2 + l) * M + m];
            acc += B[i] * (kind ? v.y : v.x);
            if (!kind) {
                double e = 0.0;
                for (int q = 0; q < K; ++q)
                    e += prm[(2 * l) * K + q] * B[q];
                accU += e * B[i];
            }
        }
        if (grad)
            grad[(size_t)c * 4 * K + o] = acc;
        if (dU)
            dU[(size_t)c * 4 * K + o] = kind ? 0.0 : T * accU;
    }
    if (threadIdx.x == 0 && U_out) {
        double u = 0.0;
        for (int m = 0; m < M; ++m) {
            double B[kMaxK];
            bspline_basis(K, order, wmin, wmax, (double)(j0 + m) * dw, B);
            for (int l = 0; l < 2; ++l) {
                double e = 0.0;
                for (int q = 0; q < K; ++q)
                    e += prm[(2 * l) * K + q] * B[q];
                u += e * e;
            }
        }
        U_out[c] = 0.5 * T * u;
    }
}

// ---- chain rule of the Hann-envelope synthesis.  The samples are linear in the
// harmonic coefficients C'_j of hann_spectrum_kernel (s = 1):
//   E = Re sum_j C'_j z^j,  Ed = Re sum_j i W_j C'_j z^j,
//   A = -Im sum_{j>=1} C'_j (z^j - 1) / W_j + Re(C'_0) (t_f - t),   z = exp(i pi k / n),
// so dJ/dC'_j is a sum over samples; the transpose of C'_j = C_j/2 - C_{j-1}/4 -
// C_{j+1}/4 gives dJ/dC_j, and C_j = (-1)^j E~_j e^{-i Phi_j} gives dJ/dE~_j, dJ/dPhi_j.
// The fluence (T/2) sum_{j>=1} |C'_j|^2 + T Re(C'_0)^2 goes the same way.

// One block per (harmonic slot, polarisation, candidate): gH = (dJ/dRe C'_j, dJ/dIm C'_j).
__global__ void __launch_bounds__(kVjpThreads) hann_vjp_harmonics_kernel(
    double T, int j0p, int n_steps, const double *__restrict__ g, int ldg, double2 *__restrict__ gH)
{
    __shared__ double red[2][kVjpThreads];
    const int m = blockIdx.x, l = blockIdx.y, c = blockIdx.z, Mp = gridDim.x;
    const int j = j0p + m;
    const double W = (double)j * (2.0 * M_PI / T), h = T / (2.0 * n_steps);
    const double *gA = g + ((size_t)c * 6 + l) * ldg;
    const double *gE = g + ((size_t)c * 6 + 2 + l) * ldg;
    const double *gD = g + ((size_t)c * 6 + 4 + l) * ldg;
    const long long two_n = 2ll * n_steps;
    double sr, cr;  // rotation by kVjpThreads samples, as in vjp_modes_kernel
    sincospi((double)(((long long)j * kVjpThreads) % two_n) / (double)n_steps, &sr, &cr);
    const double iW = j ? 1.0 / W : 0.0;
    double gre = 0.0, gim = 0.0, sz = 0.0, cz = 1.0;
    int it = 0;
    for (int k = threadIdx.x; k <= 2 * n_steps; k += kVjpThreads, ++it) {
        const double ga = gA[k], ge = gE[k], gd = gD[k];
        if (j == 0) {
            gre += ga * ((double)(2 * n_steps - k) * h) + ge;
        } else {
            if (it % kVjpResync == 0)
                sincospi((double)(((long long)j * k) % two_n) / (double)n_steps, &sz, &cz);
            gre += ga * (-sz * iW) + ge * cz + gd * (-W * sz);
            gim += ga * (-(cz - 1.0) * iW) + ge * (-sz) + gd * (-W * cz);
            const double sn = fma(sz, cr, cz * sr);
            cz = fma(cz, cr, -sz * sr);
            sz = sn;
        }
    }
    red[0][threadIdx.x] = gre;
    red[1][threadIdx.x] = gim;
    __syncthreads();
    for (int hh = kVjpThreads / 2; hh > 0; hh >>= 1) {
        if (threadIdx.x < hh) {
            red[0][threadIdx.x] += red[0][threadIdx.x + hh];
            red[1][threadIdx.x] += red[1][threadIdx.x + hh];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        gH[((size_t)c * 2 + l) * Mp + m] = make_double2(red[0][0], red[1][0]);
}

// One block per candidate: unit-scale spectrum, the harmonics C', the fluence U,
// and per mode (dJ/dE~, dJ/dPhi) (if gH is given) and (dU/dE~, dU/dPhi).
// Work arrays (global, per candidate): cp[2][M+2] padded C, ch[2][M+2] = C'.
__global__ void hann_vjp_modes_kernel(const double *__restrict__ params, int K, int order, double wmin,
                                      double wmax, double T, int j0, int M, const double2 *__restrict__ gH,
                                      double2 *__restrict__ cpad, double2 *__restrict__ chh,
                                      double2 *__restrict__ eph, double2 *__restrict__ dEP,
                                      double2 *__restrict__ dUP, double *__restrict__ U_out)
{
    const int c = blockIdx.x, Mp = M + 2, j0p = j0 - 1;
    const double *prm = params + (size_t)c * 4 * K;
    const double dw = 2.0 * M_PI / T;
    double2 *cp = cpad + (size_t)c * 2 * Mp, *hc = chh + (size_t)c * 2 * Mp;
    double2 *ep = eph + (size_t)c * 2 * M;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const int j = j0 + m;
        double B[kMaxK];
        bspline_basis(K, order, wmin, wmax, (double)j * dw, B);
        for (int l = 0; l < 2; ++l) {
            double e = 0.0, ph = 0.0;
            for (int i = 0; i < K; ++i) {
                e += prm[(2 * l) * K + i] * B[i];
                ph += prm[(2 * l + 1) * K + i] * B[i];
            }
            double sn, cs;
            sincos(ph, &sn, &cs);
            const double sg = (j & 1) ? -1.0 : 1.0;
            cp[l * Mp + m + 1] = make_double2(sg * e * cs, -sg * e * sn);
            ep[l * M + m] = make_double2(e, ph);
        }
    }
    if (threadIdx.x < 2) {
        cp[threadIdx.x * Mp] = make_double2(0.0, 0.0);
        cp[threadIdx.x * Mp + M + 1] = make_double2(0.0, 0.0);
    }
    __syncthreads();
    double ssq = 0.0;
    for (int q = threadIdx.x; q < 2 * Mp; q += blockDim.x) {
        const int l = q / Mp, m = q % Mp;
        const double2 *u = cp + l * Mp;
        const double2 cm = u[m], cl = m > 0 ? u[m - 1] : make_double2(0.0, 0.0),
                      cr = m + 1 < Mp ? u[m + 1] : make_double2(0.0, 0.0);
        const double2 v = make_double2(0.5 * cm.x - 0.25 * cl.x - 0.25 * cr.x, 0.5 * cm.y - 0.25 * cl.y - 0.25 * cr.y);
        hc[q] = v;
        ssq += (j0p + m == 0) ? 2.0 * v.x * v.x : v.x * v.x + v.y * v.y;
    }
    // block_sum's barriers also order the C' writes above before the reads below
    const double usum = block_sum(ssq);
    if (threadIdx.x == 0 && U_out)
        U_out[c] = 0.5 * T * usum;
    // dU/dC'_j: T C'_j (j >= 1), 2 T Re C'_0 (j = 0); transposed to the modes
    for (int q = threadIdx.x; q < 2 * M; q += blockDim.x) {
        const int l = q / M, m = q % M;
        auto uH = [&](int s) -> double2 {
            const double2 v = hc[l * Mp + s];
            return (j0p + s == 0) ? make_double2(2.0 * T * v.x, 0.0) : make_double2(T * v.x, T * v.y);
        };
        const double2 a = uH(m + 1), b = uH(m), d = uH(m + 2);
        const double ure = 0.5 * a.x - 0.25 * b.x - 0.25 * d.x, uim = 0.5 * a.y - 0.25 * b.y - 0.25 * d.y;
        const double2 eq = ep[l * M + m];
        const double sg = ((j0 + m) & 1) ? -1.0 : 1.0;
        double sn, cs;
        sincos(eq.y, &sn, &cs);
        dUP[(size_t)c * 2 * M + q] = make_double2(sg * (ure * cs - uim * sn), sg * eq.x * (-ure * sn - uim * cs));
        if (gH) {
            const double2 *gh = gH + ((size_t)c * 2 + l) * Mp;
            const double gre = 0.5 * gh[m + 1].x - 0.25 * gh[m].x - 0.25 * gh[m + 2].x;
            const double gim = 0.5 * gh[m + 1].y - 0.25 * gh[m].y - 0.25 * gh[m + 2].y;
            dEP[(size_t)c * 2 * M + q] = make_double2(sg * (gre * cs - gim * sn), sg * eq.x * (-gre * sn - gim * cs));
        }
    }
}

// B-spline sums of the per-mode derivatives: grad_o and dU_o (U already written).
__global__ void hann_vjp_params_kernel(int K, int order, double wmin, double wmax, double T, int j0, int M,
                                       const double2 *__restrict__ dEP, const double2 *__restrict__ dUP,
                                       double *__restrict__ grad, double *__restrict__ dU)
{
    const int c = blockIdx.x;
    const double dw = 2.0 * M_PI / T;
    for (int o = threadIdx.x; o < 4 * K; o += blockDim.x) {
        const int l = o / (2 * K), kind = (o / K) % 2, i = o % K;
        double acc = 0.0, accU = 0.0;
        for (int m = 0; m < M; ++m) {
            double B[kMaxK];
            bspline_basis(K, order, wmin, wmax, (double)(j0 + m) * dw, B);
            if (grad) {
                const double2 v = dEP[((size_t)c * 2 + l) * M + m];
                acc += B[i] * (kind ? v.y : v.x);
            }
            const double2 u = dUP[((size_t)c * 2 + l) * M + m];
            accU += B[i] * (kind ? u.y : u.x);
        }
        if (grad)
            grad[(size_t)c * 4 * K + o] = acc;
        if (dU)
            dU[(size_t)c * 4 * K + o] = accU;
    }
}

// ---- batches of candidates with their own pulse length and step count (same K,
// order, band and fluence): per-candidate spectrum descriptors.
struct SynthCand {
    double T;
    int n_steps;
    int j0, M;    // harmonic band of the samples (the mode band widened by one each side
                  // with the Hann envelope)
    int j0m, Mm;  // mode band of the spectrum
    int env;      // 0: g = 1, 1: Hann
    long long coef_off;  // into the coefficient buffer, 4 M double2 per candidate
};

__global__ void spectrum_batch_kernel(const double *__restrict__ params, int K, int order, double wmin,
                                      double wmax, double U, const SynthCand *__restrict__ sc,
                                      double2 *__restrict__ coef, unsigned int *__restrict__ status)
{
    const int c = blockIdx.x;
    const SynthCand d = sc[c];
    const double *prm = params + (size_t)c * 4 * K;
    if (d.env)
        hann_spectrum_block(prm, K, order, wmin, wmax, d.T, U, d.j0m, d.Mm, coef + d.coef_off, nullptr, status, 1);
    else
        spectrum_block(prm, K, order, wmin, wmax, d.T, U, d.j0m, d.Mm, coef + d.coef_off, nullptr, status, 1);
}

__global__ void samples_batch_kernel(const double2 *__restrict__ coef, const SynthCand *__restrict__ sc,
                                     int ld, double *__restrict__ A)
{
    extern __shared__ double2 scf[];
    const int c = blockIdx.y, l = blockIdx.z;
    const SynthCand d = sc[c];
    const int nsamp = 2 * d.n_steps + 1;
    if (blockIdx.x * blockDim.x >= nsamp)
        return;  // the whole block is past this candidate's samples
    const double2 *cf = coef + d.coef_off + (size_t)l * 2 * d.M;
    for (int q = threadIdx.x; q < 2 * d.M; q += blockDim.x)
        scf[q] = cf[q];
    __syncthreads();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nsamp)
        return;
    const int M = d.M;
    const long long two_n = 2ll * d.n_steps;
    double zs, zc, js, jc;
    sincospi((double)(k % two_n) / (double)d.n_steps, &zs, &zc);
    sincospi((double)(((long long)k * d.j0) % two_n) / (double)d.n_steps, &js, &jc);
    double dr = 0.0, di = 0.0, d0i = 0.0;
    for (int m = M - 1; m >= 0; --m) {
        const double2 D = scf[M + m];
        const double tr = fma(dr, zc, fma(-di, zs, D.x));
        di = fma(dr, zs, fma(di, zc, D.y));
        dr = tr;
        d0i += D.y;
    }
    const double Di = fma(dr, js, di * jc);
    double a = -(Di - d0i);
    if (d.j0 == 0)  // DC harmonic of the Hann envelope: potential c0 (t_f - t_k)
        a += scf[0].x * ((double)(2 * d.n_steps - k) * (d.T / (2.0 * d.n_steps)));
    A[((size_t)c * 2 + l) * ld + k] = a;
}

}  // namespace

namespace pp {

// Device descriptors for a batch of pulse lengths (pp_batch): built once on the host.
int synth_batch_prepare(int ncand, const pp_field_spec *specs, void **d_desc, void **d_coef,
                        int *max_M)
{
    std::vector<SynthCand> h(ncand);
    long long off = 0;
    int mm = 0;
    for (int c = 0; c < ncand; ++c) {
        const double dw = 2.0 * M_PI / specs[c].T;
        int j0 = (int)ceil(specs[c].w_min / dw - 1e-12);
        if (j0 < 1)
            j0 = 1;
        const int j1 = (int)floor(specs[c].w_max / dw + 1e-12);
        const int env = specs[c].envelope == 1;
        h[c].T = specs[c].T;
        h[c].n_steps = specs[c].n_steps;
        h[c].j0m = j0;
        h[c].Mm = j1 - j0 + 1;
        h[c].env = env;
        h[c].j0 = env ? j0 - 1 : j0;
        h[c].M = env ? h[c].Mm + 2 : h[c].Mm;
        h[c].coef_off = off;
        off += 4ll * h[c].M;
        mm = h[c].M > mm ? h[c].M : mm;
    }
    cudaError_t e = cudaMalloc(d_desc, sizeof(SynthCand) * (size_t)ncand);
    if (e == cudaSuccess)
        e = cudaMalloc(d_coef, sizeof(double2) * (size_t)(off > 0 ? off : 1));
    if (e == cudaSuccess)
        e = cudaMemcpy(*d_desc, h.data(), sizeof(SynthCand) * (size_t)ncand, cudaMemcpyHostToDevice);
    if (e != cudaSuccess)
        return cuda_fail(e, "batch synthesis descriptors");
    *max_M = mm;
    return PP_OK;
}

int launch_synth_batch(const double *params, int ncand, const pp_field_spec *spec0, const void *d_desc,
                       void *d_coef, int max_M, int max_nsamp, int ld, double *A, cudaStream_t stream)
{
    unsigned int *status = status_word();
    if (!status)
        return fail(PP_ERR_CUDA, "status word unavailable");
    spectrum_batch_kernel<<<ncand, 128, 0, stream>>>(params, spec0->K, spec0->order, spec0->w_min,
                                                     spec0->w_max, spec0->fluence,
                                                     (const SynthCand *)d_desc, (double2 *)d_coef,
                                                     status);
    dim3 g((max_nsamp + 255) / 256, ncand, 2);
    samples_batch_kernel<<<g, 256, 2 * max_M * sizeof(double2), stream>>>(
        (const double2 *)d_coef, (const SynthCand *)d_desc, ld, A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e, "batch synthesis launch");
    return PP_OK;
}

namespace {
int mode_band(const pp_field_spec *spec, int *j0_out)
{
    const double dw = 2.0 * M_PI / spec->T;
    int j0 = (int)ceil(spec->w_min / dw - 1e-12);
    if (j0 < 1)
        j0 = 1;
    const int j1 = (int)floor(spec->w_max / dw + 1e-12);
    *j0_out = j0;
    return j1 - j0 + 1;
}
}  // namespace

int launch_synth(const double *params, int ncand, const pp_field_spec *spec, int normalize, double *A,
                 int ld, double *E, double *Ed, double *scale, cudaStream_t stream)
{
    int j0;
    const int M = mode_band(spec, &j0);
    const bool hann = spec->envelope == 1;
    const int Ms = hann ? M + 2 : M, j0s = hann ? j0 - 1 : j0;  // harmonics actually synthesised
    void *coef = nullptr;
    int rc = scratch(SCR_COEF, (size_t)ncand * 4 * Ms * sizeof(double2), &coef);
    if (rc)
        return rc;
    if (ncand == 0)
        return PP_OK;
    unsigned int *status = status_word();
    if (!status)
        return fail(PP_ERR_CUDA, "status word unavailable");
    if (hann)
        hann_spectrum_kernel<<<ncand, 128, 0, stream>>>(params, spec->K, spec->order, spec->w_min, spec->w_max,
                                                        spec->T, spec->fluence, j0, M, (double2 *)coef, scale,
                                                        status, normalize);
    else
        spectrum_kernel<<<ncand, 128, 0, stream>>>(params, spec->K, spec->order, spec->w_min, spec->w_max,
                                                   spec->T, spec->fluence, j0, M, (double2 *)coef, scale, status,
                                                   normalize);
    const int nsamp = 2 * spec->n_steps + 1;
    dim3 g((nsamp + 255) / 256, ncand, 2);
    auto kern = E ? (Ed ? samples_kernel<true, true> : samples_kernel<true, false>)
                  : (Ed ? samples_kernel<false, true> : samples_kernel<false, false>);
    kern<<<g, 256, 2 * Ms * sizeof(double2), stream>>>((const double2 *)coef, Ms, j0s, spec->n_steps, ld, A, E,
                                                       2.0 * M_PI / spec->T, Ed, spec->T);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e, "synthesis kernel launch");
    return PP_OK;
}

int launch_synth_field(const double *params, int ncand, const pp_field_spec *spec, double *A, int ld,
                       double *E, double *scale, cudaStream_t stream)
{
    return launch_synth(params, ncand, spec, 1, A, ld, E, nullptr, scale, stream);
}

int launch_synth_vjp(const double *params, int ncand, const pp_field_spec *spec, const double *g, int ldg,
                     double *grad, double *U, double *dU, cudaStream_t stream)
{
    int j0;
    const int M = mode_band(spec, &j0);
    if (spec->envelope == 1) {
        const int Mp = M + 2;
        // gH, cpad, chh: 2 Mp each; eph, dEP, dUP: 2 M each (per candidate)
        void *buf = nullptr;
        int rc = scratch(SCR_VJP, (size_t)ncand * (6 * Mp + 6 * M) * sizeof(double2), &buf);
        if (rc || ncand == 0)
            return rc;
        double2 *gH = (double2 *)buf, *cpad = gH + (size_t)ncand * 2 * Mp, *chh = cpad + (size_t)ncand * 2 * Mp;
        double2 *eph = chh + (size_t)ncand * 2 * Mp, *dEP = eph + (size_t)ncand * 2 * M,
                *dUP = dEP + (size_t)ncand * 2 * M;
        if (grad)
            hann_vjp_harmonics_kernel<<<dim3(Mp, 2, ncand), kVjpThreads, 0, stream>>>(spec->T, j0 - 1, spec->n_steps,
                                                                                    g, ldg, gH);
        hann_vjp_modes_kernel<<<ncand, 128, 0, stream>>>(params, spec->K, spec->order, spec->w_min, spec->w_max,
                                                         spec->T, j0, M, grad ? gH : nullptr, cpad, chh, eph, dEP,
                                                         dUP, U);
        if (grad || dU)
            hann_vjp_params_kernel<<<ncand, 128, 0, stream>>>(spec->K, spec->order, spec->w_min, spec->w_max,
                                                              spec->T, j0, M, dEP, dUP, grad, dU);
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? PP_OK : cuda_fail(e, "synthesis chain-rule launch");
    }
    void *dep = nullptr;
    int rc = scratch(SCR_VJP, (size_t)ncand * 2 * M * sizeof(double2), &dep);
    if (rc || ncand == 0)
        return rc;
    if (grad)
        vjp_modes_kernel<<<dim3(M, 2, ncand), kVjpThreads, 0, stream>>>(params, spec->K, spec->order,
                                                                        spec->w_min, spec->w_max, spec->T, j0,
                                                                        spec->n_steps, g, ldg, (double2 *)dep);
    vjp_params_kernel<<<ncand, 128, 0, stream>>>(params, spec->K, spec->order, spec->w_min, spec->w_max, spec->T,
                                                 j0, M, (const double2 *)dep, grad, U, dU);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PP_OK : cuda_fail(e, "synthesis chain-rule launch");
}

}  // namespace pp
