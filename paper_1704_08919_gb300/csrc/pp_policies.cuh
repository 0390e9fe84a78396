// pp_policies.cuh -- the per-mode propagation of the pair-number kernels
// (Sec. II.A of arXiv 1704.08919: Eqs. (kin_mom), (free_spin1), (wf_init),
// (dirac_eq_mom), (pair_prod_homo); Eq. (opt_prob)): the stepping policies
// (RK4, fourth-order Magnus, second-order split operator; FP64, FP32 and FP32
// with compensated state), the table builder and the work-item body shared by
// the uniform kernel (pp_propagate.cu) and the persistent batch kernel
// (pp_batch.cu).  Included by those two files only (internal linkage).
#pragma once

#include <math.h>
#include <string.h>

#include "pp_internal.cuh"

namespace {

// Modes per partial sum of the momentum integral: the per-CTA sums are formed
// over fixed groups of kGroup consecutive modes, so N does not depend on the
// launch configuration (threads per CTA, tile length) the tuner picks.
constexpr int kGroup = 128;

struct alignas(32) dbl4 {
    double x, y, z, w;
};
template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
    using type = float4;
};
template <>
struct Vec4<double> {
    using type = dbl4;
};

// e = -i (h . sigma) z for a 2-vector z = (z0r, z0i, z1r, z1i).
template <typename T>
__device__ __forceinline__ void rot(T hx, T hy, T hz, const T z[4], T e[4])
{
    e[0] = fma(hy, -z[2], fma(hx, z[3], hz * z[1]));
    e[1] = fma(hy, -z[3], fma(hx, -z[2], -hz * z[0]));
    e[2] = fma(hz, -z[3], fma(hy, z[0], hx * z[1]));
    e[3] = fma(hz, z[2], fma(hy, z[1], -hx * z[0]));
}

// acc += -i (h . sigma) z
template <typename T>
__device__ __forceinline__ void rot_acc(T hx, T hy, T hz, const T z[4], T acc[4])
{
    acc[0] = fma(hy, -z[2], fma(hx, z[3], fma(hz, z[1], acc[0])));
    acc[1] = fma(hy, -z[3], fma(hx, -z[2], fma(-hz, z[0], acc[1])));
    acc[2] = fma(hz, -z[3], fma(hy, z[0], fma(hx, z[1], acc[2])));
    acc[3] = fma(hz, z[2], fma(hy, z[1], fma(-hx, z[0], acc[3])));
}

// Node i of linspace(a, b, n), rounded exactly as a + ((b - a) * i) / (n - 1).
__device__ __forceinline__ double axis_node(int i, int n, double a, double b)
{
    if (n == 1)
        return a;
    return __dadd_rn(a, __ddiv_rn(__dmul_rn(__dsub_rn(b, a), (double)i), (double)(n - 1)));
}

__device__ __forceinline__ double axis_weight(int i, int n, double a, double b, int mirror)
{
    if (n == 1)
        return 1.0;
    double d = __ddiv_rn(__dsub_rn(b, a), (double)(n - 1));
    double w = (i == 0 || i == n - 1) ? __dmul_rn(0.5, d) : d;
    return mirror ? __dmul_rn(2.0, w) : w;
}

// Normalised eigenvectors of h . sigma (h_z = eps_perp >= 1 > 0), FP64.
// negative: (-(hx - i hy), w + hz) / sqrt(2 w (w + hz)); positive: (w + hz, hx + i hy) / same.
__device__ __forceinline__ void eig_neg(double hx, double hy, double hz, double v[4])
{
    double w = sqrt(hx * hx + hy * hy + hz * hz);
    double nr = 1.0 / sqrt(2.0 * w * (w + hz));
    v[0] = -hx * nr;
    v[1] = hy * nr;
    v[2] = (w + hz) * nr;
    v[3] = 0.0;
}

__device__ __forceinline__ double proj_pos2(double hx, double hy, double hz, const double p[4])
{
    double w = sqrt(hx * hx + hy * hy + hz * hz);
    double nr = 1.0 / sqrt(2.0 * w * (w + hz));
    double u0 = (w + hz) * nr, u2 = hx * nr, u3 = hy * nr;  // u1 = 0
    double re = u0 * p[0] + u2 * p[2] + u3 * p[3];
    double im = u0 * p[1] + u2 * p[3] - u3 * p[2];
    return re * re + im * im;
}

// ---------------------------------------------------------------- stepping policies
// A policy supplies the per-step table entry (Entry), the tile length, the
// per-thread state and the RK4 step.  Table entry n holds the potential of
// step n scaled for the stages: (dt/3) A(t_{n+1/2}) and (dt/6) A(t_{n+1}).

// Scalar policy: T = double (parity path) or float (COMP: compensated state).
template <typename T, bool COMP>
struct ScalarPolicy {
    using Entry = typename Vec4<T>::type;

    __device__ static Entry make_entry(double ax3, double ay3, double ax6, double ay6)
    {
        Entry e;
        e.x = (T)ax3;
        e.y = (T)ay3;
        e.z = (T)ax6;
        e.w = (T)ay6;
        return e;
    }

    struct State {
        T hi[2][4], lo[2][4];
        T px3, py3, px6, py6, ez3, ez6, q6x, q6y;
    };

    __device__ static void init(State &st, const double v[2][4], double px, double py, double eperp,
                                double d3, double d6, double ax0, double ay0)
    {
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                st.hi[s][q] = (T)v[s][q];
                st.lo[s][q] = (T)(v[s][q] - (double)st.hi[s][q]);
            }
        st.px3 = (T)(d3 * px);
        st.py3 = (T)(d3 * py);
        st.px6 = (T)(d6 * px);
        st.py6 = (T)(d6 * py);
        st.ez3 = (T)(d3 * eperp);
        st.ez6 = (T)(d6 * eperp);
        st.q6x = st.px6 - (T)(d6 * ax0);
        st.q6y = st.py6 - (T)(d6 * ay0);
    }

    __device__ static __forceinline__ void step(State &st, const Entry &e)
    {
        const T q3x = st.px3 - e.x, q3y = st.py3 - e.y;
        const T n6x = st.px6 - e.z, n6y = st.py6 - e.w;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const T a6 = s ? -st.q6y : st.q6y;
            const T a3 = s ? -q3y : q3y;
            const T b6 = s ? -n6y : n6y;
            T e1[4], e2[4], y[4], S[4];
            rot(st.q6x, a6, st.ez6, st.hi[s], e1);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                y[q] = fma((T)3, e1[q], st.hi[s][q]);
            rot(q3x, a3, st.ez3, y, e2);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                y[q] = fma((T)1.5, e2[q], st.hi[s][q]);
                S[q] = e1[q] + e2[q];
            }
            rot(q3x, a3, st.ez3, y, e2);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                y[q] = fma((T)3, e2[q], st.hi[s][q]);
                S[q] = S[q] + e2[q];
                if (COMP)
                    S[q] = S[q] + st.lo[s][q];
            }
            rot_acc(n6x, b6, st.ez6, y, S);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (COMP) {
                    const T h = st.hi[s][q] + S[q];
                    st.lo[s][q] = S[q] - (h - st.hi[s][q]);
                    st.hi[s][q] = h;
                } else {
                    st.hi[s][q] = st.hi[s][q] + S[q];
                }
            }
        }
        st.q6x = n6x;
        st.q6y = n6y;
    }

    __device__ static void psi(const State &st, int s, double out[4], double, double, double,
                               double)
    {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            out[q] = COMP ? (double)st.hi[s][q] + (double)st.lo[s][q] : (double)st.hi[s][q];
    }
};

// Packed FP32 policy: both spin channels in one 64-bit register pair per state
// component (low half: s = +1, high half: s = -1), advanced together by the
// sm_100+ packed instructions fma/add/sub/mul.rn.f32x2.  Channel s = -1 sees
// h_y -> -h_y, so the table carries (A_x, A_x) and (A_y, -A_y) pairs; every
// coefficient is also formed with the opposite sign, because the real form of
// -i h.sigma has both signs of each coefficient.  Compensated (two-float) state.
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk2(float a, float b)
{
    f2 d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ void unpk2(f2 v, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2 ffma2(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 fadd2(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fsub2(f2 a, f2 b)
{
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fmul2(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Scaled h at one time point, with both signs: (hx, -hx, hy, -hy) as channel pairs.
struct H2 {
    f2 x, nx, y, ny;
};

// e = -i (h . sigma) z for both channels (see rot()).
__device__ __forceinline__ void rot2(const H2 &h, f2 hz, f2 nhz, const f2 z[4], f2 e[4])
{
    e[0] = ffma2(h.ny, z[2], ffma2(h.x, z[3], fmul2(hz, z[1])));
    e[1] = ffma2(h.ny, z[3], ffma2(h.nx, z[2], fmul2(nhz, z[0])));
    e[2] = ffma2(nhz, z[3], ffma2(h.y, z[0], fmul2(h.x, z[1])));
    e[3] = ffma2(hz, z[2], ffma2(h.y, z[1], fmul2(h.nx, z[0])));
}

__device__ __forceinline__ void rot2_acc(const H2 &h, f2 hz, f2 nhz, const f2 z[4], f2 acc[4])
{
    acc[0] = ffma2(h.ny, z[2], ffma2(h.x, z[3], ffma2(hz, z[1], acc[0])));
    acc[1] = ffma2(h.ny, z[3], ffma2(h.nx, z[2], ffma2(nhz, z[0], acc[1])));
    acc[2] = ffma2(nhz, z[3], ffma2(h.y, z[0], ffma2(h.x, z[1], acc[2])));
    acc[3] = ffma2(hz, z[2], ffma2(h.y, z[1], ffma2(h.nx, z[0], acc[3])));
}

struct alignas(32) PackedEntry {
    f2 ax3, ay3, ax6, ay6;  // (dt/3)(A_x, A_x), (dt/3)(A_y, -A_y), (dt/6)(...), (dt/6)(...)
};

template <bool COMP>
struct PackedPolicy {
    using Entry = PackedEntry;

    __device__ static Entry make_entry(double ax3, double ay3, double ax6, double ay6)
    {
        Entry e;
        const float a = (float)ax3, b = (float)ay3, c = (float)ax6, d = (float)ay6;
        e.ax3 = pk2(a, a);
        e.ay3 = pk2(b, -b);
        e.ax6 = pk2(c, c);
        e.ay6 = pk2(d, -d);
        return e;
    }

    struct State {
        f2 hi[4], lo[4];
        f2 px3, py3, px6, py6, ez3, nez3, ez6, nez6;
        H2 h6;  // (dt/6) h at the current time t_n
    };

    __device__ static __forceinline__ H2 make_h(f2 px, f2 py, f2 ax, f2 ay)
    {
        H2 h;
        h.x = fsub2(px, ax);
        h.nx = fsub2(ax, px);
        h.y = fsub2(py, ay);
        h.ny = fsub2(ay, py);
        return h;
    }

    __device__ static void init(State &st, const double v[2][4], double px, double py, double eperp,
                                double d3, double d6, double ax0, double ay0)
    {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float h0 = (float)v[0][q], h1 = (float)v[1][q];
            st.hi[q] = pk2(h0, h1);
            st.lo[q] = pk2((float)(v[0][q] - (double)h0), (float)(v[1][q] - (double)h1));
        }
        const float x3 = (float)(d3 * px), y3 = (float)(d3 * py);
        const float x6 = (float)(d6 * px), y6 = (float)(d6 * py);
        const float z3 = (float)(d3 * eperp), z6 = (float)(d6 * eperp);
        st.px3 = pk2(x3, x3);
        st.py3 = pk2(y3, -y3);
        st.px6 = pk2(x6, x6);
        st.py6 = pk2(y6, -y6);
        st.ez3 = pk2(z3, z3);
        st.nez3 = pk2(-z3, -z3);
        st.ez6 = pk2(z6, z6);
        st.nez6 = pk2(-z6, -z6);
        const float a = (float)(d6 * ax0), b = (float)(d6 * ay0);
        st.h6 = make_h(st.px6, st.py6, pk2(a, a), pk2(b, -b));
    }

    __device__ static __forceinline__ void step(State &st, const Entry &e)
    {
        const f2 three = pk2(3.0f, 3.0f), half3 = pk2(1.5f, 1.5f);
        const H2 h3 = make_h(st.px3, st.py3, e.ax3, e.ay3);
        const H2 hn = make_h(st.px6, st.py6, e.ax6, e.ay6);
        f2 e1[4], e2[4], y[4], S[4];
        rot2(st.h6, st.ez6, st.nez6, st.hi, e1);
        #pragma unroll
        for (int q = 0; q < 4; ++q)
            y[q] = ffma2(three, e1[q], st.hi[q]);
        rot2(h3, st.ez3, st.nez3, y, e2);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            y[q] = ffma2(half3, e2[q], st.hi[q]);
            S[q] = fadd2(e1[q], e2[q]);
        }
        rot2(h3, st.ez3, st.nez3, y, e2);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            y[q] = ffma2(three, e2[q], st.hi[q]);
            S[q] = fadd2(S[q], e2[q]);
            if (COMP)
                S[q] = fadd2(S[q], st.lo[q]);
        }
        rot2_acc(hn, st.ez6, st.nez6, y, S);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const f2 h = fadd2(st.hi[q], S[q]);
            if (COMP)
                st.lo[q] = fsub2(S[q], fsub2(h, st.hi[q]));
            st.hi[q] = h;
        }
        st.h6 = hn;
    }

    __device__ static void psi(const State &st, int s, double out[4], double, double, double,
                               double)
    {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float h0, h1, l0, l1;
            unpk2(st.hi[q], h0, h1);
            unpk2(st.lo[q], l0, l1);
            if (!COMP)
                l0 = l1 = 0.0f;
            out[q] = s ? (double)h1 + (double)l1 : (double)h0 + (double)l0;
        }
    }
};

// cos(th) - 1 and sin(th)/th as polynomials in t = th^2 for th <= 0.2: FP32
// keeps terms through th^6 / th^4 (the rest is below 1e-9 relative), FP64
// through th^12 (the rest is below 1e-17 relative).  Beyond th = 0.2 the FP32
// truncation grows as th^6 / 5040 per step (8e-7 at 0.4, 5e-5 at 0.8) and the
// step stops being unitary, so the Magnus policy only uses these polynomials on
// tiles of steps whose bound on th stays within kSeriesLimit.
constexpr double kSeriesLimit = 0.2;
// Most halvings of th in the wide-range Magnus step (the scale 2^-2k stays a
// normal number in both precisions); th up to kSeriesLimit 2^60 ~ 2e17.
constexpr int kMaxHalvings = 60;
template <typename T>
struct TrigSeries;
template <>
struct TrigSeries<float> {
    __device__ static __forceinline__ float cm1(float t)
    {
        return t * fmaf(t, fmaf(t, -1.0f / 720.0f, 1.0f / 24.0f), -0.5f);
    }
    __device__ static __forceinline__ float sinc(float t)
    {
        return fmaf(t, fmaf(t, 1.0f / 120.0f, -1.0f / 6.0f), 1.0f);
    }
};
template <>
struct TrigSeries<double> {
    __device__ static __forceinline__ double cm1(double t)
    {
        double r = 1.0 / 479001600.0;
        r = fma(t, r, -1.0 / 3628800.0);
        r = fma(t, r, 1.0 / 40320.0);
        r = fma(t, r, -1.0 / 720.0);
        r = fma(t, r, 1.0 / 24.0);
        r = fma(t, r, -0.5);
        return t * r;
    }
    __device__ static __forceinline__ double sinc(double t)
    {
        double r = 1.0 / 6227020800.0;
        r = fma(t, r, -1.0 / 39916800.0);
        r = fma(t, r, 1.0 / 362880.0);
        r = fma(t, r, -1.0 / 5040.0);
        r = fma(t, r, 1.0 / 120.0);
        r = fma(t, r, -1.0 / 6.0);
        return fma(t, r, 1.0);
    }
};

// tan(th) / th as a cubic in t = th^2 for th <= kSeriesLimit (t <= 0.04): the
// Taylor series 1 + t/3 + 2t^2/15 + 17t^3/315 + 62t^4/2835 with its t^4 term
// economised by the Chebyshev polynomial T_4 on [0, 0.04] (t^4 replaced by
// t^4 - (0.02)^4 T_4(t/0.02 - 1)/8, a cubic): coefficients 1 - 4.4e-10 (rounded to
// 1 in FP32), 29531281/88593750, 94469/708750, 3949/70875; relative error below
// 1.4e-9 on the range (1.8e-9 with the constant term rounded).
struct TanSeries {
    __device__ static __forceinline__ float tanc(float t)
    {
        float r = 5.571781305e-02f;
        r = fmaf(t, r, 1.332895944e-01f);
        r = fmaf(t, r, 3.333336832e-01f);
        return fmaf(t, r, 1.0f);
    }
};

// Fourth-order Magnus policy.  One step applies exp(-i dt h_eff . sigma) with
//     h_eff = (h_0 + 4 h_{1/2} + h_1) / 6 - (dt/6) h_0 x h_1,
// the 2-level form of Omega = -i dt/6 (H_0 + 4 H_h + H_1) + dt^2/12 [H_0, H_1]
// ([a.sigma, b.sigma] = 2i (a x b).sigma).  With H = dt h_eff and th = |H|:
// exp(-i H.sigma) = cos th - i (sin th / th) H.sigma; the increment
// (cos th - 1) psi - i (sin th / th) H.sigma psi uses the even polynomials of
// TrigSeries where th <= kSeriesLimit, and their argument-halved form elsewhere.
// Table entry: (dt Abar_x, dt Abar_y, D_x, D_y, C, th_max, 4^-k, k) with Abar = (A_0 + 4 A_h + A_1)/6,
// D_x = dt^2/6 (A0x - A1x), D_y = dt^2/6 (A1y - A0y), C = dt^2/6 (A0x A1y - A0y A1x),
// which makes dt h_eff for spin channel s:
//     x = (dt p_x - dt Abar_x) - s eps D_y
//     y = s (dt p_y - dt Abar_y) - eps D_x
//     z = dt eps + s (D_y p_x + D_x p_y - C)
// and th_max bounds |dt h_eff| over every mode of the grid and both channels:
// with P_x = max |p_x|, P_y = max |p_y|, E = max eps over the grid,
//     th_max^2 = (dt P_x + |dt Abar_x| + E |D_y|)^2 + (dt P_y + |dt Abar_y| + E |D_x|)^2
//              + (dt E + |D_y| P_x + |D_x| P_y + |C|)^2.
// A candidate with any th_max > kSeriesLimit takes the wide-range step (in a kernel
// of its own) for all its steps; step n halves th k_n times, k_n the least k with th_max 2^-k <= kSeriesLimit
// (0 where the bound is inside the range), the same for every mode, so the
// threads of a warp never diverge.
// FP32 series steps are taken in tracked form: (cos th)^-1 exp(-i H.sigma) =
// 1 - i (tan th / th) H.sigma, which drops the cos th - 1 term and its
// polynomial (24 instead of 30 FP32 instructions per channel and step).  The
// state then grows by 1 / cos th per step; the exact evolution is unitary, so the
// projection is divided by the squared norm, and rescale() (between shared-memory tiles) scales
// each channel by a power of two, which is exact: the result does not depend on
// where the rescaling happens.
template <typename T, bool COMP>
struct MagnusPolicy {
    struct alignas(sizeof(T) * 8) Entry {
        T ax, ay, dx, dy, c, pad0, pad1, pad2;
    };

    __device__ static Entry make_entry6(double dt, double a0x, double a0y, double ahx, double ahy,
                                        double a1x, double a1y, const pp_grid &g)
    {
        Entry e;
        const double d6 = dt * dt / 6.0;
        const double ax = dt * (a0x + 4.0 * ahx + a1x) / 6.0;
        const double ay = dt * (a0y + 4.0 * ahy + a1y) / 6.0;
        const double dx = d6 * (a0x - a1x), dy = d6 * (a1y - a0y);
        const double c = d6 * (a0x * a1y - a0y * a1x);
        e.ax = (T)ax;
        e.ay = (T)ay;
        e.dx = (T)dx;
        e.dy = (T)dy;
        e.c = (T)c;
        // bound on th = |dt h_eff| over the grid (see above)
        const double Px = fmax(fabs(g.x0), fabs(g.x1)), Py = fmax(fabs(g.y0), fabs(g.y1));
        const double Pz = fmax(fabs(g.z0), fabs(g.z1)), E = sqrt(1.0 + Pz * Pz);
        const double bx = dt * Px + fabs(ax) + E * fabs(dy);
        const double by = dt * Py + fabs(ay) + E * fabs(dx);
        const double bz = dt * E + fabs(dy) * Px + fabs(dx) * Py + fabs(c);
        double th = sqrt(bx * bx + by * by + bz * bz);
        e.pad0 = (T)th;
        int k = 0;
        while (th > kSeriesLimit && k < kMaxHalvings) {
            th *= 0.5;
            ++k;
        }
        e.pad1 = (T)ldexp(1.0, -2 * k);
        e.pad2 = (T)k;
        return e;
    }

    // True if the step of this entry may leave the range of TrigSeries.
    __device__ static __forceinline__ bool beyond_series(const Entry &e) { return e.pad0 > (T)kSeriesLimit; }

    struct State {
        T hi[2][4], lo[2][4];
        T dtpx, dtpy, dteps, eps, px, py;
    };

    __device__ static void init(State &st, const double v[2][4], double px, double py, double eperp,
                                double dt)
    {
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                st.hi[s][q] = (T)v[s][q];
                st.lo[s][q] = (T)(v[s][q] - (double)st.hi[s][q]);
            }
        st.dtpx = (T)(dt * px);
        st.dtpy = (T)(dt * py);
        st.dteps = (T)(dt * eperp);
        st.eps = (T)eperp;
        st.px = (T)px;
        st.py = (T)py;
    }

    // WIDE = false: cos th - 1 and sin th / th from TrigSeries (th <= kSeriesLimit).
    // WIDE = true: th is halved k = e.pad2 times (th^2 scaled by e.pad1 = 4^-k) into
    // the series range, the series gives c = cos a - 1 and S = sin a / a there, and k
    // double-angle steps restore th: sin 2a / 2a = S (1 + c) and
    // cos 2a - 1 = 2 c (c + 2).  With k = 0 this is the series path exactly.
    template <bool WIDE>
    __device__ static __forceinline__ void step_impl(State &st, const Entry &e)
    {
        const T u = st.dtpx - e.ax, v = st.dtpy - e.ay;
        const T w = fma(e.dy, st.px, fma(e.dx, st.py, -e.c));
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const T Hx = s ? fma(st.eps, e.dy, u) : fma(-st.eps, e.dy, u);
            const T Hy = s ? fma(-st.eps, e.dx, -v) : fma(-st.eps, e.dx, v);
            const T Hz = s ? st.dteps - w : st.dteps + w;
            const T t2 = fma(Hz, Hz, fma(Hy, Hy, Hx * Hx));
            T cm1, sc;
            if constexpr (WIDE) {
                const T tr = t2 * e.pad1;
                const int k = (int)e.pad2;
                cm1 = TrigSeries<T>::cm1(tr);
                sc = TrigSeries<T>::sinc(tr);
                for (int i = 0; i < k; ++i) {
                    sc = fma(sc, cm1, sc);
                    cm1 = (T)2 * fma(cm1, cm1, (T)2 * cm1);
                }
            } else {
                cm1 = TrigSeries<T>::cm1(t2);
                sc = TrigSeries<T>::sinc(t2);
            }
            const T gx = sc * Hx, gy = sc * Hy, gz = sc * Hz;
            const T *z = st.hi[s];
            if (COMP) {
                T D[4];
                D[0] = fma(gz, z[1], fma(gx, z[3], fma(-gy, z[2], cm1 * z[0])));
                D[1] = fma(-gz, z[0], fma(-gx, z[2], fma(-gy, z[3], cm1 * z[1])));
                D[2] = fma(gx, z[1], fma(gy, z[0], fma(-gz, z[3], cm1 * z[2])));
                D[3] = fma(-gx, z[0], fma(gy, z[1], fma(gz, z[2], cm1 * z[3])));
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const T Dl = D[q] + st.lo[s][q];
                    const T h = st.hi[s][q] + Dl;
                    st.lo[s][q] = Dl - (h - st.hi[s][q]);
                    st.hi[s][q] = h;
                }
            } else {
                // uncompensated: the increment is accumulated straight into the state
                T nz[4];
                nz[0] = fma(gz, z[1], fma(gx, z[3], fma(-gy, z[2], fma(cm1, z[0], z[0]))));
                nz[1] = fma(-gz, z[0], fma(-gx, z[2], fma(-gy, z[3], fma(cm1, z[1], z[1]))));
                nz[2] = fma(gx, z[1], fma(gy, z[0], fma(-gz, z[3], fma(cm1, z[2], z[2]))));
                nz[3] = fma(-gx, z[0], fma(gy, z[1], fma(gz, z[2], fma(cm1, z[3], z[3]))));
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    st.hi[s][q] = nz[q];
            }
        }
    }

    // The FP32 series step in tracked form (see above).
    __device__ static __forceinline__ void step_tracked(State &st, const Entry &e)
    {
        const T u = st.dtpx - e.ax, v = st.dtpy - e.ay;
        const T w = fma(e.dy, st.px, fma(e.dx, st.py, -e.c));
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const T Hx = s ? fma(st.eps, e.dy, u) : fma(-st.eps, e.dy, u);
            const T Hy = s ? fma(-st.eps, e.dx, -v) : fma(-st.eps, e.dx, v);
            const T Hz = s ? st.dteps - w : st.dteps + w;
            const T t2 = fma(Hz, Hz, fma(Hy, Hy, Hx * Hx));
            const T tc = TanSeries::tanc(t2);
            const T gx = tc * Hx, gy = tc * Hy, gz = tc * Hz;
            const T *z = st.hi[s];
            if (COMP) {
                T D[4];
                D[0] = fma(gz, z[1], fma(gx, z[3], -gy * z[2]));
                D[1] = fma(-gz, z[0], fma(-gx, z[2], -gy * z[3]));
                D[2] = fma(gx, z[1], fma(gy, z[0], -gz * z[3]));
                D[3] = fma(-gx, z[0], fma(gy, z[1], gz * z[2]));
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const T Dl = D[q] + st.lo[s][q];
                    const T h = st.hi[s][q] + Dl;
                    st.lo[s][q] = Dl - (h - st.hi[s][q]);
                    st.hi[s][q] = h;
                }
            } else {
                T nz[4];
                nz[0] = fma(gz, z[1], fma(gx, z[3], fma(-gy, z[2], z[0])));
                nz[1] = fma(-gz, z[0], fma(-gx, z[2], fma(-gy, z[3], z[1])));
                nz[2] = fma(gx, z[1], fma(gy, z[0], fma(-gz, z[3], z[2])));
                nz[3] = fma(-gx, z[0], fma(gy, z[1], fma(gz, z[2], z[3])));
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    st.hi[s][q] = nz[q];
            }
        }
    }

    static constexpr bool kTracked = sizeof(T) == 4;

    __device__ static __forceinline__ void step(State &st, const Entry &e)
    {
        if constexpr (kTracked)
            step_tracked(st, e);
        else
            step_impl<false>(st, e);
    }
    __device__ static __forceinline__ void step_wide(State &st, const Entry &e) { step_impl<true>(st, e); }

    // Scales each channel by the power of two 2^-floor(log2(|psi|^2) / 2) (exact).
    __device__ static __forceinline__ void rescale(State &st)
    {
        if constexpr (kTracked) {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const float n2 = fmaf(st.hi[s][3], st.hi[s][3],
                                      fmaf(st.hi[s][2], st.hi[s][2],
                                           fmaf(st.hi[s][1], st.hi[s][1], st.hi[s][0] * st.hi[s][0])));
                const int e2 = ((__float_as_int(n2) >> 23) & 0xff) - 127;  // n2 is a normal number
                const float f = __int_as_float((127 - (e2 >> 1)) << 23);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    st.hi[s][q] *= f;
                    st.lo[s][q] *= f;
                }
            }
        }
    }

    __device__ static void psi(const State &st, int s, double out[4], double, double, double,
                               double)
    {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            out[q] = COMP ? (double)st.hi[s][q] + (double)st.lo[s][q] : (double)st.hi[s][q];
    }
};

// Second-order split-operator policy: Strang splitting of h_s . sigma into the
// free part h0 = (p_x, s p_y, eps) and the coupling v = (-A_x, -s A_y, 0) at
// t_{n+1/2}:  psi <- e^{-i h0.sigma dt/2} e^{-i v.sigma dt} e^{-i h0.sigma dt/2} psi.
// Neighbouring free half steps are merged: the prologue applies one free half
// step (FP64), every step applies the coupling factor and then the full free
// factor, and the epilogue undoes one free half step (FP64).  Both factors are
// exact: e^{-i k.sigma tau} = cos(|k| tau) - i sin(|k| tau) k.sigma / |k|.  The
// coupling factor does not depend on the mode, so the table holds it:
// (cos(|A| dt) - 1, -A_x sin(|A| dt)/|A|, -A_y sin(|A| dt)/|A|).
template <typename T, bool COMP>
struct SplitPolicy {
    struct alignas(sizeof(T) * 4) Entry {
        T cm1, wx, wy, pad;
    };

    __device__ static Entry make_entry2(double dt, double ahx, double ahy)
    {
        const double a = sqrt(ahx * ahx + ahy * ahy), th = a * dt;
        const double sn = a > 0.0 ? sin(th) / a : dt;
        const double sh = sin(0.5 * th);
        Entry e;
        e.cm1 = (T)(-2.0 * sh * sh);
        e.wx = (T)(-sn * ahx);
        e.wy = (T)(-sn * ahy);
        e.pad = (T)0;
        return e;
    }

    struct State {
        T hi[2][4], lo[2][4];
        T c0m1, gx, gy, gz;  // e^{-i h0.sigma dt} = (1 + c0m1) - i (g . sigma)
    };

    // out = c psi + sg rot(h, psi), i.e. (c - i sg h.sigma) psi, in FP64
    __device__ static void apply_free(double c, double sg, double hx, double hy, double hz,
                                      const double in[4], double out[4])
    {
        double r[4];
        rot<double>(hx, hy, hz, in, r);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            out[q] = c * in[q] + sg * r[q];
    }

    __device__ static void init(State &st, const double v[2][4], double px, double py, double eperp,
                                double dt)
    {
        const double w0 = sqrt(px * px + py * py + eperp * eperp);
        const double sh = sin(0.5 * w0 * dt), ch = cos(0.5 * w0 * dt);
        const double sg = sin(w0 * dt) / w0;
        st.c0m1 = (T)(-2.0 * sh * sh);
        st.gx = (T)(sg * px);
        st.gy = (T)(sg * py);
        st.gz = (T)(sg * eperp);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            double w[4];
            apply_free(ch, sh / w0, px, s ? -py : py, eperp, v[s], w);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                st.hi[s][q] = (T)w[q];
                st.lo[s][q] = (T)(w[q] - (double)st.hi[s][q]);
            }
        }
    }

    __device__ static __forceinline__ void step(State &st, const Entry &e)
    {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const T wy = s ? -e.wy : e.wy;
            const T gy = s ? -st.gy : st.gy;
            const T *z = st.hi[s];
            T D[4], y[4];
            D[0] = fma(e.wx, z[3], fma(-wy, z[2], e.cm1 * z[0]));
            D[1] = fma(-e.wx, z[2], fma(-wy, z[3], e.cm1 * z[1]));
            D[2] = fma(e.wx, z[1], fma(wy, z[0], e.cm1 * z[2]));
            D[3] = fma(-e.wx, z[0], fma(wy, z[1], e.cm1 * z[3]));
#pragma unroll
            for (int q = 0; q < 4; ++q)
                y[q] = z[q] + D[q];
            if (COMP) {
                D[0] = fma(st.gz, y[1], fma(st.gx, y[3], fma(-gy, y[2], fma(st.c0m1, y[0], D[0]))));
                D[1] = fma(-st.gz, y[0], fma(-st.gx, y[2], fma(-gy, y[3], fma(st.c0m1, y[1], D[1]))));
                D[2] = fma(st.gx, y[1], fma(gy, y[0], fma(-st.gz, y[3], fma(st.c0m1, y[2], D[2]))));
                D[3] = fma(-st.gx, y[0], fma(gy, y[1], fma(st.gz, y[2], fma(st.c0m1, y[3], D[3]))));
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const T Dl = D[q] + st.lo[s][q];
                    const T h = st.hi[s][q] + Dl;
                    st.lo[s][q] = Dl - (h - st.hi[s][q]);
                    st.hi[s][q] = h;
                }
            } else {
                // uncompensated: the free factor is applied to y = psi + D_v directly
                T nz[4];
                nz[0] = fma(st.gz, y[1], fma(st.gx, y[3], fma(-gy, y[2], fma(st.c0m1, y[0], y[0]))));
                nz[1] = fma(-st.gz, y[0], fma(-st.gx, y[2], fma(-gy, y[3], fma(st.c0m1, y[1], y[1]))));
                nz[2] = fma(st.gx, y[1], fma(gy, y[0], fma(-st.gz, y[3], fma(st.c0m1, y[2], y[2]))));
                nz[3] = fma(-st.gx, y[0], fma(gy, y[1], fma(st.gz, y[2], fma(st.c0m1, y[3], y[3]))));
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    st.hi[s][q] = nz[q];
            }
        }
    }

    __device__ static void psi(const State &st, int s, double out[4], double px, double py,
                               double eperp, double dt)
    {
        double w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            w[q] = COMP ? (double)st.hi[s][q] + (double)st.lo[s][q] : (double)st.hi[s][q];
        // undo one free half step: e^{+i h0.sigma dt/2} = ch + i (sh / w0) h0.sigma
        const double w0 = sqrt(px * px + py * py + eperp * eperp);
        apply_free(cos(0.5 * w0 * dt), -sin(0.5 * w0 * dt) / w0, px, s ? -py : py, eperp, w, out);
    }
};

// Table builders: RK4 policies take (dt/3) A_{n+1/2} and (dt/6) A_{n+1};
// the Magnus policy the Simpson mean and the commutator coefficients; the
// split policy dt A_{n+1/2}.
template <class P>
__device__ __forceinline__ typename P::Entry table_entry(const P *, const double *Ax,
                                                         const double *Ay, int n, double dt,
                                                         const pp_grid &)
{
    const double d3 = dt / 3.0, d6 = dt / 6.0;
    return P::make_entry(d3 * Ax[2 * n + 1], d3 * Ay[2 * n + 1], d6 * Ax[2 * n + 2],
                         d6 * Ay[2 * n + 2]);
}
template <typename T, bool C>
__device__ __forceinline__ typename MagnusPolicy<T, C>::Entry
table_entry(const MagnusPolicy<T, C> *, const double *Ax, const double *Ay, int n, double dt,
            const pp_grid &g)
{
    return MagnusPolicy<T, C>::make_entry6(dt, Ax[2 * n], Ay[2 * n], Ax[2 * n + 1], Ay[2 * n + 1],
                                           Ax[2 * n + 2], Ay[2 * n + 2], g);
}
template <typename T, bool C>
__device__ __forceinline__ typename SplitPolicy<T, C>::Entry
table_entry(const SplitPolicy<T, C> *, const double *Ax, const double *Ay, int n, double dt,
            const pp_grid &)
{
    return SplitPolicy<T, C>::make_entry2(dt, Ax[2 * n + 1], Ay[2 * n + 1]);
}

// State initialisation: the RK4 policies take the stage scales dt/3 and dt/6.
template <class P>
__device__ __forceinline__ void policy_init(typename P::State &st, const double v[2][4], double px,
                                            double py, double eperp, double dt, double ax0,
                                            double ay0, int)
{
    P::init(st, v, px, py, eperp, dt / 3.0, dt / 6.0, ax0, ay0);
}

template <class P>
struct UsesDtInit {
    static constexpr bool value = false;
};
template <typename T, bool C>
struct UsesDtInit<MagnusPolicy<T, C>> {
    static constexpr bool value = true;
};
template <typename T, bool C>
struct UsesDtInit<SplitPolicy<T, C>> {
    static constexpr bool value = true;
};

// Policies whose series steps let the state's norm grow (rescale between tiles).
template <class P>
struct TracksNorm {
    static constexpr bool value = false;
};
template <bool C>
struct TracksNorm<MagnusPolicy<float, C>> {
    static constexpr bool value = MagnusPolicy<float, C>::kTracked;
};

// Policies whose step has a series range (beyond_series, step_wide).
template <class P>
struct HasSeriesGuard {
    static constexpr bool value = false;
};
template <typename T, bool C>
struct HasSeriesGuard<MagnusPolicy<T, C>> {
    static constexpr bool value = true;
};

// Table of candidate c (grid (blocks, candidates), 256 threads).  For policies with
// a series range, wide_flags[c] (zeroed before the launch) is set when any step of
// the candidate leaves it; the propagation then runs that candidate in the
// wide-range kernel instead.
template <class P>
__global__ void build_table_kernel(const double *__restrict__ A, int ld, int ns_uniform,
                                   const int *__restrict__ ns_array, int padded, double dt,
                                   pp_grid g, typename P::Entry *__restrict__ table,
                                   int *__restrict__ wide_flags)
{
    int c = blockIdx.y;
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    int ns = ns_array ? ns_array[c] : ns_uniform;
    const double *Ax = A + (size_t)c * 2 * ld, *Ay = Ax + ld;
    bool big = false;
    if (n < padded) {
        typename P::Entry e;
        if (n < ns) {
            e = table_entry((const P *)nullptr, Ax, Ay, n, dt, g);
            if constexpr (HasSeriesGuard<P>::value)
                big = P::beyond_series(e);
        } else {
            memset(&e, 0, sizeof e);
        }
        table[(size_t)c * padded + n] = e;
    }
    if constexpr (HasSeriesGuard<P>::value) {
        if (__syncthreads_or(big) && threadIdx.x == 0)
            atomicOr(wide_flags + c, 1);
    }
}

// The candidate's kernel: a policy with a series range runs each candidate in
// exactly one of its two kernels (WIDE = wide_flags[c] != 0).
template <class P, bool WIDE>
__device__ __forceinline__ bool takes_candidate(const int *__restrict__ wide_flags, int c)
{
    if constexpr (HasSeriesGuard<P>::value)
        return (wide_flags[c] != 0) == WIDE;
    else
        return !WIDE;
}

// One work item: the modes [blk * THREADS, (blk + 1) * THREADS) of candidate c.
// The caller owns the shared-memory buffers and the two mbarriers; tile_base
// is the number of tiles this CTA has consumed before (the barrier phases run
// on across items).  Returns false if a bounded wait gave up.
template <class P, int THREADS, int TILE_BYTES>
struct ItemSmem {
    using V = typename P::Entry;
    static constexpr int TILE = TILE_BYTES / (int)sizeof(V);
    __align__(128) V buf[2][TILE];
    __align__(8) uint64_t bar[2];
    double red[THREADS / 32];
};

template <class P, int THREADS, int TILE_BYTES, bool WIDE>
__device__ __forceinline__ bool process_item(ItemSmem<P, THREADS, TILE_BYTES> &sm, int blk,
                                             const pp_grid &g, int ns,
                                             const typename P::Entry *__restrict__ trow,
                                             const double *__restrict__ Ax,
                                             const double *__restrict__ Ay, double dt,
                                             double *__restrict__ n_out,
                                             double *__restrict__ part_out, long long wait_limit,
                                             int skip_copies, unsigned int *__restrict__ status,
                                             int tile_base)
{
    using V = typename P::Entry;
    constexpr int TILE = TILE_BYTES / (int)sizeof(V);
    static_assert(THREADS % kGroup == 0, "CTA size must be a multiple of the partial-sum group");
    const int tid = threadIdx.x;
    const int nmodes = g.nx * g.ny * g.nz;
    const int m = blk * THREADS + tid;
    const bool active = m < nmodes;
    const int ntiles = (ns + TILE - 1) / TILE;

    int issued = 0;  // meaningful in thread 0 only
    if (tid == 0 && !skip_copies) {
        for (int t = 0; t < 2 && t < ntiles; ++t) {
            const int k = tile_base + t;
            mbar_arrive_expect_tx(&sm.bar[k & 1], TILE * (uint32_t)sizeof(V));
            bulk_copy_g2s(sm.buf[k & 1], trow + (size_t)t * TILE, TILE * (uint32_t)sizeof(V),
                          &sm.bar[k & 1]);
            ++issued;
        }
    }

    // ---- this thread's momentum mode and FP64 initial state
    int ix = 0, iy = 0, iz = 0;
    if (active) {
        ix = m % g.nx;
        iy = (m / g.nx) % g.ny;
        iz = m / (g.nx * g.ny);
    }
    const double px = axis_node(ix, g.nx, g.x0, g.x1);
    const double py = axis_node(iy, g.ny, g.y0, g.y1);
    const double pz = axis_node(iz, g.nz, g.z0, g.z1);
    const double eperp = sqrt(1.0 + pz * pz);

    typename P::State st;
    {
        const double Pinx = px - Ax[0], Piny = py - Ay[0];
        double v[2][4];
        eig_neg(Pinx, Piny, eperp, v[0]);
        eig_neg(Pinx, -Piny, eperp, v[1]);
        if constexpr (UsesDtInit<P>::value)
            P::init(st, v, px, py, eperp, dt);
        else
            policy_init<P>(st, v, px, py, eperp, dt, Ax[0], Ay[0], 0);
    }

    bool timed_out = false;
    int t_fail = 0;
    for (int t = 0; t < ntiles; ++t) {
        const int k = tile_base + t;
        const int b = k & 1;
        const uint32_t par = (k >> 1) & 1;
        bool ok = mbar_wait_bounded(&sm.bar[b], par, wait_limit);
        ok = __syncthreads_and(ok);
        if (!ok) {
            timed_out = true;
            t_fail = t;
            break;
        }
        const int nst = min(TILE, ns - t * TILE);
        if (active) {
            const V *tb = sm.buf[b];
            if constexpr (WIDE) {
                for (int kk = 0; kk < nst; ++kk)
                    P::step_wide(st, tb[kk]);
            } else {
#pragma unroll 2
                for (int kk = 0; kk < nst; ++kk)
                    P::step(st, tb[kk]);
                if constexpr (TracksNorm<P>::value)
                    P::rescale(st);
            }
        }
        __syncthreads();  // every thread is done with buf[b]
        if (tid == 0 && !skip_copies && t + 2 < ntiles) {
            mbar_arrive_expect_tx(&sm.bar[b], TILE * (uint32_t)sizeof(V));
            bulk_copy_g2s(sm.buf[b], trow + (size_t)(t + 2) * TILE, TILE * (uint32_t)sizeof(V),
                          &sm.bar[b]);
            ++issued;
        }
    }

    if (timed_out) {
        // Drain every copy this CTA issued (bounded) before shared memory is reused or released.
        if (tid == 0) {
            pp_flag(status, PP_FLAG_TIMEOUT);
            // copies t_fail <= t < issued were never consumed: wait for each in order
            for (int t = t_fail; t < issued; ++t) {
                const int k = tile_base + t;
                mbar_wait_bounded(&sm.bar[k & 1], (k >> 1) & 1, 1ll << 24);
            }
        }
        __syncthreads();
    }

    // ---- FP64 projection onto the positive-energy states at t_end
    double f = 0.0;
    if (active) {
        const double Poutx = px - Ax[2 * ns], Pouty = py - Ay[2 * ns];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            double psi[4];
            P::psi(st, s, psi, px, py, eperp, dt);
            double fs = proj_pos2(Poutx, s ? -Pouty : Pouty, eperp, psi);
            if constexpr (TracksNorm<P>::value)  // the state's norm grew in the series steps
                fs /= psi[0] * psi[0] + psi[1] * psi[1] + psi[2] * psi[2] + psi[3] * psi[3];
            f += fs;
        }
        if (timed_out)
            f = __longlong_as_double(0x7ff8000000000000ll);
        if (n_out)
            n_out[m] = f;
    }
    double wf = 0.0;
    if (active) {
        double w = __dmul_rn(__dmul_rn(axis_weight(ix, g.nx, g.x0, g.x1, 0),
                                       axis_weight(iy, g.ny, g.y0, g.y1, 0)),
                             axis_weight(iz, g.nz, g.z0, g.z1, g.mirror_z));
        wf = w * f;
    }
    // fixed-order reduction over groups of kGroup modes
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        wf += __shfl_down_sync(0xffffffffu, wf, off);
    if ((tid & 31) == 0)
        sm.red[tid >> 5] = wf;
    __syncthreads();
    constexpr int kGroups = THREADS / kGroup;
    const int ngroups = (nmodes + kGroup - 1) / kGroup;
    if (tid < kGroups) {
        const int gidx = blk * kGroups + tid;
        if (gidx < ngroups) {
            double acc = 0.0;
#pragma unroll
            for (int w = 0; w < kGroup / 32; ++w)
                acc += sm.red[tid * (kGroup / 32) + w];
            part_out[gidx] = acc;
        }
    }
    __syncthreads();  // sm.red is reused by the next item
    return !timed_out;
}


}  // namespace
