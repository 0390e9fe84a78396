// pp_qke.cu -- the 6-component quantum kinetic equation of Sec. II.B of
// arXiv 1704.08919 (Eqs. (qke), (matrix); f = 1 - chi_1) and its adjoint
// (Sec. IV.A, Eqs. (eom2), (adj), (grad)): the pair density of every momentum
// mode and the gradient of J = sum_p w(p) f(p) with respect to every sample of
// A, E and dE/dt, for the local search.
//
// Per mode, chi' = N(t) chi with the skew-symmetric
//   N = Q S_Q + R S_R + 2 omega S_W,  omega = sqrt(1 + P^2),  P = p - A(t),
//   X = omega^2 |E|^2 - (E.P)^2,  Q = sqrt(X) / omega^2,
//   R = eps_perp omega (E x Ed)_z / X      (Q = R = 0 where X = 0),
// integrated by classical RK4 on the half-step sample grid (N at t_n, t_{n+1/2},
// t_{n+1}).  The state is carried as delta = chi - e_1 (delta(t_i) = 0), the same
// RK4 iterates, so that f = -delta_1 keeps its relative precision when f is small.
// RK4 does not keep |chi| = 1: past |N| dt = 2 sqrt(2) it amplifies, and near a
// zero of E, where R ~ |Ed| / |E|, that happens at any practical step; a mode
// whose |chi(t_f)|^2 exceeds 1 + 1e-3 reports f = NaN.
//
// The gradient is the exact adjoint of the discrete forward map: the adjoint
// state (final value -w(p) e_1, i.e. lambda_1(t_f) = -1 of Eq. (adj) times the
// quadrature weight) runs backwards through the transposed RK4 stages, and each
// stage k = N y contributes kb (x) y to the adjoint of N, whose projections on
// S_Q, S_R, S_W are the adjoints of Q, R, omega -- the inner product
// <chi, grad N lambda> of Eq. (grad) taken stage by stage.  The forward states
// are kept at every S-th step (checkpoints in HBM) and recomputed a segment at a
// time into per-thread shared-memory slots for the backward sweep.  Each sample's six sensitivities
// are summed over the CTA's modes (warp shuffles, then warps in fixed order) into
// a per-CTA row; a second kernel sums the rows in fixed order.
#include <math.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "pp_policies.cuh"

namespace {

constexpr int kQThreads = 256;
constexpr int kQWarps = kQThreads / 32;

// Mode-independent values of one sample: A, E, dE/dt, |E|^2, (E x Ed)_z.
template <typename T>
struct alignas(sizeof(T) * 8) QkeS {
    T ax, ay, ex, ey, edx, edy, ee, cr;
};

template <typename T>
struct Coef {
    T Q, R, W2;  // W2 = 2 omega
};

// Reciprocal square root.  FP32: the special-function unit's approximation
// (rsqrtf, at most 2 ulp), one instruction instead of a square root and a
// division; its error is far below the FP32 RK4 rounding of the state.  The
// forward, recomputed and adjoint sweeps all call this one function, so the
// recomputed trajectory is the forward one bit for bit.
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return 1.0 / sqrt(x); }

template <typename T>
__device__ __forceinline__ Coef<T> coef_at(const QkeS<T> &s, T px, T py, T pz2, T eperp)
{
    const T Px = px - s.ax, Py = py - s.ay;
    const T w2 = ((Px * Px + Py * Py) + pz2) + T(1);
    const T iw = rsq(w2);
    const T EP = s.ex * Px + s.ey * Py;
    const T X = w2 * s.ee - EP * EP;
    Coef<T> c;
    c.W2 = T(2) * (w2 * iw);
    if (X > T(0)) {
        const T rX = rsq(X);
        c.Q = (X * rX) * (iw * iw);
        c.R = eperp * (w2 * iw) * s.cr * (rX * rX);
    } else {
        c.Q = T(0);
        c.R = T(0);
    }
    return c;
}

// The mode-dependent quantities of one sample that both the coefficients and
// their derivatives need.
template <typename T>
struct Basics {
    T Px, Py, w2, iw, EP, X, rX;  // rX = 1/sqrt(X) where X > 0, else 0
};

template <typename T>
__device__ __forceinline__ Basics<T> basics(const QkeS<T> &s, T px, T py, T pz2)
{
    Basics<T> b;
    b.Px = px - s.ax;
    b.Py = py - s.ay;
    b.w2 = ((b.Px * b.Px + b.Py * b.Py) + pz2) + T(1);
    b.iw = rsq(b.w2);
    b.EP = s.ex * b.Px + s.ey * b.Py;
    b.X = b.w2 * s.ee - b.EP * b.EP;
    b.rX = b.X > T(0) ? rsq(b.X) : T(0);
    return b;
}

// the same values as coef_at, from precomputed basics
template <typename T>
__device__ __forceinline__ Coef<T> coef_from(const Basics<T> &b, const QkeS<T> &s, T eperp)
{
    Coef<T> c;
    c.W2 = T(2) * (b.w2 * b.iw);
    if (b.X > T(0)) {
        c.Q = (b.X * b.rX) * (b.iw * b.iw);
        c.R = eperp * (b.w2 * b.iw) * s.cr * (b.rX * b.rX);
    } else {
        c.Q = T(0);
        c.R = T(0);
    }
    return c;
}

// out = N (e_1 + v) (ONE) or N v; Q (1 + v_0) is formed as Q + Q v_0 in one FMA,
// which also keeps the low bits of the small v_0.
template <bool ONE, typename T>
__device__ __forceinline__ void nmul(const Coef<T> &c, const T v[6], T out[6])
{
    out[0] = -c.Q * v[1];
    const T q1 = ONE ? fma(c.Q, v[0], c.Q) : c.Q * v[0];
    out[1] = fma(c.R, v[3], fma(-c.W2, v[2], q1));
    out[2] = fma(c.W2, v[1], -c.R * v[4]);
    out[3] = fma(c.W2, v[4], -c.R * v[1]);
    out[4] = fma(c.Q, v[5], fma(-c.W2, v[3], c.R * v[2]));
    out[5] = -c.Q * v[4];
}

// out = base - N v, each component one chain of FMAs (N as in nmul).
template <typename T>
__device__ __forceinline__ void nmul_sub(const Coef<T> &c, const T v[6], const T base[6], T out[6])
{
    out[0] = fma(c.Q, v[1], base[0]);
    out[1] = fma(-c.R, v[3], fma(c.W2, v[2], fma(-c.Q, v[0], base[1])));
    out[2] = fma(c.R, v[4], fma(-c.W2, v[1], base[2]));
    out[3] = fma(-c.W2, v[4], fma(c.R, v[1], base[3]));
    out[4] = fma(-c.Q, v[5], fma(c.W2, v[3], fma(-c.R, v[2], base[4])));
    out[5] = fma(c.Q, v[4], base[5]);
}

// One RK4 step of delta: chi = e_1 + delta.
template <typename T>
__device__ __forceinline__ void rk4_step(T d[6], const Coef<T> &c0, const Coef<T> &ch, const Coef<T> &c1, T dt)
{
    const T hd = T(0.5) * dt, sx = dt / T(6);
    T k1[6], k2[6], k3[6], k4[6], y[6];
    nmul<true>(c0, d, k1);
#pragma unroll
    for (int i = 0; i < 6; ++i)
        y[i] = d[i] + hd * k1[i];
    nmul<true>(ch, y, k2);
#pragma unroll
    for (int i = 0; i < 6; ++i)
        y[i] = d[i] + hd * k2[i];
    nmul<true>(ch, y, k3);
#pragma unroll
    for (int i = 0; i < 6; ++i)
        y[i] = d[i] + dt * k3[i];
    nmul<true>(c1, y, k4);
#pragma unroll
    for (int i = 0; i < 6; ++i)
        d[i] = d[i] + sx * (((k1[i] + T(2) * k2[i]) + T(2) * k3[i]) + k4[i]);
}

// Adjoints of (Q, R, omega) from one stage k = N (e_1 + y) with stage adjoint kb,
// accumulated term by term: acc[0] += Qb, acc[1] += Rb, acc[2] += wb / 2 (the
// factor 2 of N's omega entries is applied once per sample, in sens_from).
template <typename T>
__device__ __forceinline__ void coef_adj(const T kb[6], const T y[6], T acc[3])
{
    T a = fma(kb[1], y[0], acc[0] + kb[1]);
    a = fma(-kb[0], y[1], a);
    a = fma(kb[4], y[5], a);
    acc[0] = fma(-kb[5], y[4], a);
    a = fma(kb[1], y[3], acc[1]);
    a = fma(-kb[2], y[4], a);
    a = fma(kb[4], y[2], a);
    acc[1] = fma(-kb[3], y[1], a);
    a = fma(kb[2], y[1], acc[2]);
    a = fma(-kb[1], y[2], a);
    a = fma(kb[3], y[4], a);
    acc[2] = fma(-kb[4], y[3], a);
}

// Sensitivities (A_x, A_y, E_x, E_y, Ed_x, Ed_y) of one sample from the
// adjoints (Qb, Rb, wb / 2) of its coefficients, as coef_adj accumulates them.
template <typename T>
__device__ __forceinline__ void sample_sens(const QkeS<T> &s, T px, T py, T pz2, T eperp, const T ab[3], T out[6])
{
    const T Px = px - s.ax, Py = py - s.ay;
    const T w2 = ((Px * Px + Py * Py) + pz2) + T(1);
    const T iw = rsq(w2), w = w2 * iw, iw2 = iw * iw;
    const T EP = s.ex * Px + s.ey * Py;
    const T X = w2 * s.ee - EP * EP;
    const T P[2] = {Px, Py}, E[2] = {s.ex, s.ey};
    const T dcr_dE[2] = {s.edy, -s.edx}, dcr_dEd[2] = {-s.ey, s.ex};
    const T Qb = ab[0], Rb = ab[1], wb = ab[2] + ab[2];
    const bool pos = X > T(0);
    const T rX = pos ? rsq(X) : T(0);
    const T sX = X * rX, iX = rX * rX;
    const T hq = T(0.5) * rX * iw2;  // dQ/dX = 1 / (2 sqrt(X) omega^2)
    const T cx = s.cr * iX;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const T dw_dP = P[a] * iw;
        T dQ_dP = 0, dQ_dE = 0, dR_dP = 0, dR_dE = 0, dR_dEd = 0;
        if (pos) {
            const T dX_dP = T(2) * P[a] * s.ee - T(2) * EP * E[a];
            const T dX_dE = T(2) * w2 * E[a] - T(2) * EP * P[a];
            dQ_dP = dX_dP * hq - sX * T(2) * P[a] * (iw2 * iw2);
            dQ_dE = dX_dE * hq;
            // grouped so that no 1/X^2 is formed on its own (FP32 range)
            dR_dP = eperp * cx * (dw_dP - w * (dX_dP * iX));
            dR_dE = eperp * w * iX * (dcr_dE[a] - s.cr * (dX_dE * iX));
            dR_dEd = eperp * w * dcr_dEd[a] * iX;
        }
        out[a] = -((Qb * dQ_dP + Rb * dR_dP) + wb * dw_dP);
        out[2 + a] = Qb * dQ_dE + Rb * dR_dE;
        out[4 + a] = Rb * dR_dEd;
    }
}

// f = 1 - chi_1 = -delta_1, or NaN where RK4 let |chi|^2 = 1 + 2 delta_1 + |delta|^2
// grow past 1 + 1e-3 (a step too coarse for the field: the discrete chi is no
// longer a rotation and f has left its physical range).
constexpr double kGrowthTol = 1e-3;

template <typename T>
__device__ __forceinline__ double density(const T d[6])
{
    T g = T(2) * d[0];
#pragma unroll
    for (int i = 0; i < 6; ++i)
        g += d[i] * d[i];
    return (double)g <= kGrowthTol ? -(double)d[0] : __longlong_as_double(0x7ff8000000000000ll);
}

// Per-mode terms of one sample's sensitivities, from precomputed basics and the
// adjoints (Qb, Rb, wb / 2).  Writing dX/dP_a = 2 (P_a |E|^2 - (E.P) E_a) and
// dX/dE_a = 2 (omega^2 E_a - (E.P) P_a), the chain rule through Q = sqrt(X)/omega^2,
// R = eps_perp omega cr / X and omega gives, per mode,
//   dJ/dA_a  = -(mu P_a) + nu E_a,
//   dJ/dE_a  = (2 kappa omega^2) E_a - (nu P_a) + gam dcr/dE_a,
//   dJ/dEd_a = gam dcr/dEd_a,
// with kappa = Qb hq - Rb R / X, hq = dQ/dX = 1 / (2 sqrt(X) omega^2),
// gam = Rb eps_perp omega / X, beta = wb / omega + Rb R / omega^2 - 2 Qb sqrt(X) / omega^4,
// mu = 2 kappa |E|^2 + beta and nu = 2 kappa (E.P).  E, Ed and cr are the same for
// every mode, so only the seven mode-dependent factors are summed over the modes:
//   out = (mu P_x, mu P_y, nu, 2 kappa omega^2, nu P_x, nu P_y, gam),
// and sample_sens_from_sums applies the sample's constants once.  R is divided by
// X before it meets dX (FP32 range near zeros of E).  Where X <= 0, rX = 0 makes
// every Q and R term vanish, as in sample_sens.
constexpr int kSensTerms = 7;

template <typename T>
__device__ __forceinline__ void sens_from(const Basics<T> &b, const QkeS<T> &s, T eperp, const T ab[3], T out[7])
{
    const T w = b.w2 * b.iw, iw2 = b.iw * b.iw;
    const T sX = b.X * b.rX, iX = b.rX * b.rX;
    const T Qb = ab[0], Rb = ab[1], wb = ab[2] + ab[2];
    const T ewX = eperp * w * iX;     // R / cr
    const T RbR = Rb * (ewX * s.cr);  // Rb R
    const T gam = Rb * ewX;
    const T beta = (wb * b.iw + RbR * iw2) - T(2) * Qb * sX * (iw2 * iw2);
    const T k2 = Qb * (b.rX * iw2) - T(2) * (RbR * iX);  // 2 kappa
    const T mu = fma(k2, s.ee, beta), nu = k2 * b.EP;
    out[0] = mu * b.Px;
    out[1] = mu * b.Py;
    out[2] = nu;
    out[3] = k2 * b.w2;
    out[4] = nu * b.Px;
    out[5] = nu * b.Py;
    out[6] = gam;
}

// The sensitivity i of a sample (E, Ed) from the sums over modes u[0..6] of sens_from.
__device__ __forceinline__ double sample_sens_from_sums(int i, double ex, double ey, double edx, double edy,
                                                        const double u[7])
{
    switch (i) {
    case 0: return -u[0] + ex * u[2];
    case 1: return -u[1] + ey * u[2];
    case 2: return (ex * u[3] - u[4]) + edy * u[6];
    case 3: return (ey * u[3] - u[5]) - edx * u[6];
    case 4: return -ey * u[6];
    default: return ex * u[6];
    }
}

// Sums v[0..15] over the warp by halving exchanges (16 shuffles instead of 80):
// afterwards lanes L and L^1 hold the total of value (L >> 1) & 15.
template <typename T>
__device__ __forceinline__ T warp_sum16(T v[16], int lane)
{
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int o = 16 >> r, w = 8 >> r;
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < w; ++i) {
            const T send = up ? v[i] : v[i + w];
            const T keep = up ? v[i + w] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

struct ModeGeom {
    double px, py, pz, w;
    bool active;
};

__device__ __forceinline__ ModeGeom mode_geom(const pp_grid &g, int m)
{
    ModeGeom r;
    const int nmodes = g.nx * g.ny * g.nz;
    r.active = m < nmodes;
    int ix = 0, iy = 0, iz = 0;
    if (r.active) {
        ix = m % g.nx;
        iy = (m / g.nx) % g.ny;
        iz = m / (g.nx * g.ny);
    }
    r.px = axis_node(ix, g.nx, g.x0, g.x1);
    r.py = axis_node(iy, g.ny, g.y0, g.y1);
    r.pz = axis_node(iz, g.nz, g.z0, g.z1);
    r.w = r.active ? __dmul_rn(__dmul_rn(axis_weight(ix, g.nx, g.x0, g.x1, 0), axis_weight(iy, g.ny, g.y0, g.y1, 0)),
                               axis_weight(iz, g.nz, g.z0, g.z1, g.mirror_z))
                   : 0.0;
    return r;
}

// fixed-order CTA sum of one double per thread; the result is valid in thread 0
__device__ __forceinline__ double cta_sum(double v, double *red)
{
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kQWarps; ++w)
            s += red[w];
    __syncthreads();
    return s;
}

// table[c][k] from A, E, Ed ([c][2][ld] FP64)
template <typename T>
__global__ void qke_table_kernel(const double *__restrict__ A, const double *__restrict__ E,
                                 const double *__restrict__ Ed, int ld, int nsamp, int ldt, QkeS<T> *__restrict__ tab)
{
    const int c = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nsamp)
        return;
    const size_t r0 = (size_t)c * 2 * ld, r1 = r0 + ld;
    const double ex = E[r0 + k], ey = E[r1 + k], dx = Ed[r0 + k], dy = Ed[r1 + k];
    QkeS<T> s;
    s.ax = (T)A[r0 + k];
    s.ay = (T)A[r1 + k];
    s.ex = (T)ex;
    s.ey = (T)ey;
    s.edx = (T)dx;
    s.edy = (T)dy;
    s.ee = (T)(ex * ex + ey * ey);
    s.cr = (T)(ex * dy - ey * dx);
    tab[(size_t)c * ldt + k] = s;
}

// Forward only: f(p) of every mode and per-CTA partial sums of w f.
template <typename T>
__global__ void __launch_bounds__(kQThreads) qke_forward_kernel(const QkeS<T> *__restrict__ tab, int ldt, int n_steps,
                                                                double dt, pp_grid g, double *__restrict__ n_out,
                                                                double *__restrict__ part)
{
    constexpr int kTile = 32;  // steps per staged tile
    __shared__ double red[kQWarps];
    __shared__ QkeS<T> seg[2 * kTile + 1];
    const int c = blockIdx.y, blk = blockIdx.x;
    const int nmodes = g.nx * g.ny * g.nz;
    const int m = blk * kQThreads + threadIdx.x;
    const ModeGeom mg = mode_geom(g, m);
    const T px = (T)mg.px, py = (T)mg.py, pz2 = (T)(mg.pz * mg.pz), eperp = (T)sqrt(1.0 + mg.pz * mg.pz);
    const QkeS<T> *tr = tab + (size_t)c * ldt;
    T d[6] = {0, 0, 0, 0, 0, 0};
    Coef<T> c0 = coef_at(tr[0], px, py, pz2, eperp);
    for (int n0 = 0; n0 < n_steps; n0 += kTile) {
        const int cnt = min(kTile, n_steps - n0);
        __syncthreads();
        if (threadIdx.x < 2 * cnt + 1)
            seg[threadIdx.x] = tr[2 * n0 + threadIdx.x];
        __syncthreads();
        for (int q = 0; q < cnt; ++q) {
            const Coef<T> ch = coef_at(seg[2 * q + 1], px, py, pz2, eperp);
            const Coef<T> c1 = coef_at(seg[2 * q + 2], px, py, pz2, eperp);
            rk4_step(d, c0, ch, c1, (T)dt);
            c0 = c1;
        }
    }
    const double f = density(d);
    if (mg.active && n_out)
        n_out[(size_t)c * nmodes + m] = f;
    const double s = cta_sum(mg.active ? mg.w * f : 0.0, red);
    if (threadIdx.x == 0)
        part[(size_t)c * gridDim.x + blk] = s;
}

// Per-thread asynchronous copies of one 4- or 8-byte value global -> shared
// (cp.async), one commit group per step, so that a thread can wait for its own
// copies without a barrier.
template <typename T>
__device__ __forceinline__ void cp_async_value(T *smem, const T *gmem)
{
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "cp.async copies 4, 8 or 16 bytes");
    const unsigned int sa = (unsigned int)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"((int)sizeof(T))
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Forward with checkpoints, then the backward sweep segment by segment.
// ckpt[c][seg][6][nmp] (T), part[c][blk][6][ldg] (FP64), partJ[c][blk].
// S = 1: every step's state is kept, and the backward sweep reads it back through
// a per-thread ring of kQRing shared-memory slots filled kQRing - 1 steps ahead by
// cp.async (no recomputation).  S > 1: one state per S steps, and each segment is
// recomputed into per-thread shared-memory slots before its backward steps.
// The steps are handled in groups of q_group_steps: the samples of a group are
// staged into shared memory once, and the sample sensitivities of a whole group
// are summed over the CTA's warps once, so a group costs five barriers whatever S
// is, and J and the gradient do not depend on S.  FP32: 2 CTAs per SM with up to
// 128 registers (no spills; 3 CTAs per SM at 80 registers spilled in the backward
// step and measured 2.9% slower).
// steps per group: 64 in FP32, 32 in FP64 (static shared memory stays under 48 KB)
template <typename T>
constexpr int q_group_steps() { return sizeof(T) == 4 ? 64 : 32; }
constexpr int kQRing = 4;
template <typename T, int S>
__global__ void __launch_bounds__(kQThreads, sizeof(T) == 4 ? 2 : 1) qke_adjoint_kernel(const QkeS<T> *__restrict__ tab, int ldt, int n_steps,
                                                                double dt_d, pp_grid g, T *__restrict__ ckpt, int nmp,
                                                                double *__restrict__ part, int ldg,
                                                                double *__restrict__ partJ)
{
    constexpr int GS = q_group_steps<T>();  // steps per group
    static_assert(GS % S == 0, "a group holds whole segments");
    constexpr int kQGroup = GS / S;  // segments per group
    __shared__ double red[kQWarps];
    __shared__ T sb[kQWarps][2 * GS][kSensTerms];       // per-warp sums of the terms
    __shared__ double usum[2 * GS][kSensTerms];         // their sums over the warps
    __shared__ QkeS<T> seg[2 * GS + 1];  // the samples of the current group (broadcast reads)
    // per-thread state slots, sst[(q * 6 + i) * kQThreads + tid]: the segment's
    // recomputed states (S > 1) or the prefetch ring (S = 1, slot q = step % kQRing)
    extern __shared__ __align__(16) unsigned char qke_dyn[];
    T *sst = reinterpret_cast<T *>(qke_dyn);
    const int c = blockIdx.y, blk = blockIdx.x, nblk = gridDim.x;
    const int m = blk * kQThreads + threadIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const ModeGeom mg = mode_geom(g, m);
    const T px = (T)mg.px, py = (T)mg.py, pz2 = (T)(mg.pz * mg.pz), eperp = (T)sqrt(1.0 + mg.pz * mg.pz);
    const T dt = (T)dt_d, hd = T(0.5) * dt, sx = dt / T(6);
    const QkeS<T> *tr = tab + (size_t)c * ldt;
    const int nseg = (n_steps + S - 1) / S;
    const int mm = min(m, nmp - 1);  // inactive threads store into a valid slot they own alone
    T *ck = ckpt + (size_t)c * nseg * 6 * nmp;
    auto stage = [&](int n0, int cnt) {  // samples 2 n0 .. 2 (n0 + cnt) into shared memory
        __syncthreads();
        for (int k = threadIdx.x; k < 2 * cnt + 1; k += kQThreads)
            seg[k] = tr[2 * n0 + k];
        __syncthreads();
    };
    const int ngrp = (nseg + kQGroup - 1) / kQGroup;

    // ---- phase A: forward, keeping the state at the start of every segment
    T d[6] = {0, 0, 0, 0, 0, 0};
    {
        Coef<T> c0 = coef_at(tr[0], px, py, pz2, eperp);
        for (int gr = 0; gr < ngrp; ++gr) {
            const int g0 = gr * kQGroup, n0g = g0 * S;
            stage(n0g, min(GS, n_steps - n0g));
            for (int s = g0; s < min(g0 + kQGroup, nseg); ++s) {
                if (mg.active)
#pragma unroll
                    for (int i = 0; i < 6; ++i)
                        ck[((size_t)s * 6 + i) * nmp + mm] = d[i];
                const int so = (s - g0) * S, cnt = min(S, n_steps - s * S);
                for (int q = 0; q < cnt; ++q) {
                    const Coef<T> ch = coef_at(seg[2 * (so + q) + 1], px, py, pz2, eperp);
                    const Coef<T> c1 = coef_at(seg[2 * (so + q) + 2], px, py, pz2, eperp);
                    rk4_step(d, c0, ch, c1, dt);
                    c0 = c1;
                }
            }
        }
    }
    {
        const double s = cta_sum(mg.active ? mg.w * density(d) : 0.0, red);
        if (threadIdx.x == 0)
            partJ[(size_t)c * nblk + blk] = s;
    }

    // ---- phase B: backward
    double *prow = part + ((size_t)c * nblk + blk) * 6 * ldg;
    T bar[6] = {(T)(-mg.w), 0, 0, 0, 0, 0};
    T pend[3] = {0, 0, 0};  // coefficient adjoints of the sample at the top of the next step
    Coef<T> c1 = coef_at(tr[2 * n_steps], px, py, pz2, eperp);
    Basics<T> b1 = basics(tr[2 * n_steps], px, py, pz2);  // of the sample at the top of the step
    // S = 1: this thread's stored state at the start of step n into ring slot n % kQRing
    auto prefetch = [&](int n) {
        if (n >= 0) {
            T *dst = sst + (size_t)(n % kQRing) * 6 * kQThreads + threadIdx.x;
            const T *src = ck + (size_t)n * 6 * nmp + mm;
#pragma unroll
            for (int i = 0; i < 6; ++i)
                cp_async_value(dst + i * kQThreads, src + (size_t)i * nmp);
        }
        cp_async_commit();  // one group per step, empty below step 0
    };
    if constexpr (S == 1)
        for (int n = n_steps - 1; n > n_steps - kQRing; --n)
            prefetch(n);
    for (int gr = ngrp - 1; gr >= 0; --gr) {
        const int g0 = gr * kQGroup, n0g = g0 * S, cntg = min(GS, n_steps - n0g);
        stage(n0g, cntg);
        for (int s = min(g0 + kQGroup, nseg) - 1; s >= g0; --s) {
            const int so = (s - g0) * S, cnt = min(S, n_steps - s * S);
            const T *xs = sst;  // the states x_q of this segment: xs[(q * 6 + i) * kQThreads + tid]
            if constexpr (S == 1) {
                prefetch(s - (kQRing - 1));
                cp_async_wait<kQRing - 1>();  // this thread's copy of step s has landed
                xs = sst + (size_t)(s % kQRing) * 6 * kQThreads;
            } else {
#pragma unroll
                for (int i = 0; i < 6; ++i)
                    d[i] = mg.active ? ck[((size_t)s * 6 + i) * nmp + mm] : T(0);
                // the segment's states x_0 .. x_{cnt-1}; x_cnt (the next checkpoint) is not needed
                Coef<T> c0 = coef_at(seg[2 * so], px, py, pz2, eperp);
#pragma unroll 1
                for (int q = 0;; ++q) {
#pragma unroll
                    for (int i = 0; i < 6; ++i)
                        sst[(q * 6 + i) * kQThreads + threadIdx.x] = d[i];
                    if (q + 1 >= cnt)
                        break;
                    const Coef<T> ch = coef_at(seg[2 * (so + q) + 1], px, py, pz2, eperp);
                    const Coef<T> cn = coef_at(seg[2 * (so + q) + 2], px, py, pz2, eperp);
                    rk4_step(d, c0, ch, cn, dt);
                    c0 = cn;
                }
            }
#pragma unroll 1
            for (int q = cnt - 1; q >= 0; --q) {
                {
                    const QkeS<T> e0 = seg[2 * (so + q)], eh = seg[2 * (so + q) + 1], e1 = seg[2 * (so + q) + 2];
                    const Basics<T> bh = basics(eh, px, py, pz2);
                    const Basics<T> b0 = basics(e0, px, py, pz2);
                    const Coef<T> c0 = coef_from(b0, e0, eperp);
                    const Coef<T> ch = coef_from(bh, eh, eperp);
                    T x[6];
#pragma unroll
                    for (int i = 0; i < 6; ++i)
                        x[i] = xs[(q * 6 + i) * kQThreads + threadIdx.x];
                    T k1[6], k2[6], k3[6], y2[6], y3[6], y4[6];
                    nmul<true>(c0, x, k1);
#pragma unroll
                    for (int i = 0; i < 6; ++i)
                        y2[i] = x[i] + hd * k1[i];
                    nmul<true>(ch, y2, k2);
#pragma unroll
                    for (int i = 0; i < 6; ++i)
                        y3[i] = x[i] + hd * k2[i];
                    nmul<true>(ch, y3, k3);
#pragma unroll
                    for (int i = 0; i < 6; ++i)
                        y4[i] = x[i] + dt * k3[i];
                    T kb1[6], kb2[6], kb3[6], kb4[6], xb[6], yb[6];
#pragma unroll
                    for (int i = 0; i < 6; ++i) {
                        kb1[i] = sx * bar[i];
                        kb2[i] = T(2) * sx * bar[i];
                        kb3[i] = kb2[i];
                        kb4[i] = kb1[i];
                        xb[i] = bar[i];
                    }
                    // k4 = N1 (e1 + y4): completes the sample 2n+2
                    coef_adj(kb4, y4, pend);
                    nmul<false>(c1, kb4, yb);
#pragma unroll
                    for (int i = 0; i < 6; ++i) {
                        xb[i] -= yb[i];
                        kb3[i] -= dt * yb[i];
                    }
                    T hacc[3] = {0, 0, 0};
                    coef_adj(kb3, y3, hacc);  // k3 = Nh (e1 + y3)
                    nmul<false>(ch, kb3, yb);
#pragma unroll
                    for (int i = 0; i < 6; ++i) {
                        xb[i] -= yb[i];
                        kb2[i] -= hd * yb[i];
                    }
                    coef_adj(kb2, y2, hacc);  // k2 = Nh (e1 + y2)
                    nmul<false>(ch, kb2, yb);
#pragma unroll
                    for (int i = 0; i < 6; ++i) {
                        xb[i] -= yb[i];
                        kb1[i] -= hd * yb[i];
                    }
                    T nacc[3] = {0, 0, 0};
                    coef_adj(kb1, x, nacc);  // k1 = N0 (e1 + x)
                    nmul_sub(c0, kb1, xb, bar);
                    // emit samples 2n+2 (terms 0..6, slot 2q+1) and 2n+1 (terms 7..13, slot 2q)
                    T o[16];
                    sens_from(b1, e1, eperp, pend, o);
                    sens_from(bh, eh, eperp, hacc, o + kSensTerms);
#pragma unroll
                    for (int i = 2 * kSensTerms; i < 16; ++i)
                        o[i] = T(0);
                    const T tot = warp_sum16(o, lane);
                    const int vi = (lane >> 1) & 15;
                    if ((lane & 1) == 0 && vi < 2 * kSensTerms)
                        sb[warp][vi < kSensTerms ? 2 * (so + q) + 1 : 2 * (so + q)]
                          [vi < kSensTerms ? vi : vi - kSensTerms] = tot;
#pragma unroll
                    for (int i = 0; i < 3; ++i)
                        pend[i] = nacc[i];
                    c1 = c0;
                    b1 = b0;
                }
            }
        }
        __syncthreads();
        // sample 2 n0g + 1 + kk: each of its seven terms summed over the warps in
        // fixed order (FP64), then its six sensitivities from the sample's E and Ed
        for (int t = threadIdx.x; t < 2 * cntg * kSensTerms; t += kQThreads) {
            const int j = t / (2 * cntg), kk = t % (2 * cntg);
            double acc = (double)sb[0][kk][j];
            for (int w = 1; w < kQWarps; ++w)
                acc += (double)sb[w][kk][j];
            usum[kk][j] = acc;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < 2 * cntg * 6; t += kQThreads) {
            const int i = t / (2 * cntg), kk = t % (2 * cntg);
            const QkeS<T> &e = seg[kk + 1];
            prow[(size_t)i * ldg + 2 * n0g + 1 + kk] =
                sample_sens_from_sums(i, (double)e.ex, (double)e.ey, (double)e.edx, (double)e.edy, usum[kk]);
        }
        __syncthreads();
    }
    // sample 0 (t_i): only the first step's k1 stage reaches it
    {
        T o[6];
        sample_sens(tr[0], px, py, pz2, eperp, pend, o);
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const T v = warp_sum(o[i]);
            if (lane == 0)
                sb[warp][0][i] = v;
        }
        __syncthreads();
        if (threadIdx.x < 6) {
            double acc = 0.0;
            for (int w = 0; w < kQWarps; ++w)
                acc += (double)sb[w][0][threadIdx.x];
            prow[(size_t)threadIdx.x * ldg] = acc;
        }
    }
}

// out[c][...] = sum over blocks of part[c][blk][...] (fixed order); n per candidate.
__global__ void sum_blocks_kernel(const double *__restrict__ part, int nblk, long long n, double *__restrict__ out)
{
    const int c = blockIdx.y;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const double *p = part + (size_t)c * nblk * n + i;
    double acc = 0.0;
    for (int b = 0; b < nblk; ++b)
        acc += p[(size_t)b * n];
    out[(size_t)c * n + i] = acc;
}

inline unsigned nbk(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

template <typename T>
int build_table(const double *A, const double *E, const double *Ed, int ncand, int ld, int n_steps, void **tab,
                int *ldt_out, cudaStream_t st)
{
    const int nsamp = 2 * n_steps + 1;
    const int ldt = (nsamp + 31) / 32 * 32;
    int rc = pp::scratch(pp::SCR_QKE_TABLE, sizeof(QkeS<T>) * (size_t)ldt * ncand, tab);
    if (rc)
        return rc;
    qke_table_kernel<T><<<dim3(nbk(nsamp), ncand), 256, 0, st>>>(A, E, Ed, ld, nsamp, ldt, (QkeS<T> *)*tab);
    *ldt_out = ldt;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PP_OK : pp::cuda_fail(e, "QKE table");
}

template <typename T>
int forward(const double *A, const double *E, const double *Ed, int ncand, int ld, int n_steps, double dt,
            const pp_grid *g, double *N, double *n_p, cudaStream_t st)
{
    void *tab = nullptr, *part = nullptr;
    int ldt = 0;
    int rc = build_table<T>(A, E, Ed, ncand, ld, n_steps, &tab, &ldt, st);
    const int nmodes = g->nx * g->ny * g->nz;
    const int nblk = (nmodes + kQThreads - 1) / kQThreads;
    if (!rc)
        rc = pp::scratch(pp::SCR_QKE_PART, sizeof(double) * (size_t)nblk * ncand, &part);
    if (rc)
        return rc;
    qke_forward_kernel<T><<<dim3(nblk, ncand), kQThreads, 0, st>>>((const QkeS<T> *)tab, ldt, n_steps, dt, *g, n_p,
                                                                   (double *)part);
    sum_blocks_kernel<<<dim3(1, ncand), 32, 0, st>>>((const double *)part, nblk, 1, N);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PP_OK : pp::cuda_fail(e, "QKE forward launch");
}

// Per-candidate scratch of the adjoint that keeps one state per S steps: the
// states and the per-CTA partial rows.
template <typename T>
size_t adjoint_bytes(int S, int n_steps, int nmodes, int ldg)
{
    const int nblk = (nmodes + kQThreads - 1) / kQThreads;
    const size_t ck = sizeof(T) * 6 * (size_t)((n_steps + S - 1) / S) * nmodes;
    const size_t pr = sizeof(double) * 6 * (size_t)nblk * ldg;
    return ck + pr;
}

int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 1;
    return std::max(1, n);
}

// Relative duration of a launch of n equal CTAs, ctas_per_sm at a time on each of
// sms SMs: every full wave costs 1; a last partial wave costs 1 if some SM runs
// more than one CTA of it, else kLoneWave (a CTA alone on its SM runs faster:
// measured 0.61 for the FP32 adjoint at 2 CTAs per SM).
constexpr double kLoneWave = 0.61;
double launch_cost(long long n, int ctas_per_sm, int sms)
{
    const long long slots = (long long)ctas_per_sm * sms;
    const long long full = n / slots, r = n % slots;
    return (double)full + (r == 0 ? 0.0 : (r > sms || ctas_per_sm == 1 ? 1.0 : kLoneWave));
}

// Candidates per launch: at most budget / per (one at least), chosen to minimise
// the summed launch_cost of the launches (ties: the larger chunk, fewer launches).
int wave_chunk(int ncand, size_t per, size_t budget, int nblk, int ctas_per_sm, int sms)
{
    const int cap = (int)std::max<size_t>(1, std::min<size_t>((size_t)ncand, budget / std::max<size_t>(per, 1)));
    int best = cap;
    double best_cost = 1e300;
    for (int c = cap; c >= 1; --c) {
        const int nfull = ncand / c, rest = ncand % c;
        const double cost = nfull * launch_cost((long long)c * nblk, ctas_per_sm, sms) +
                            (rest ? launch_cost((long long)rest * nblk, ctas_per_sm, sms) : 0.0);
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = c;
        }
    }
    return best;
}

// Scratch of an adjoint launch sequence with one state per S steps, chunk candidates per launch.
struct AdjointScratch {
    void *ck = nullptr, *part = nullptr, *pj = nullptr;
};

template <typename T, int S>
int adjoint_scratch(int n_steps, int nmodes, int ldg, int chunk, AdjointScratch *a)
{
    const int nblk = (nmodes + kQThreads - 1) / kQThreads;
    const int nseg = (n_steps + S - 1) / S;
    int rc = pp::scratch(pp::SCR_QKE_CKPT, sizeof(T) * 6 * (size_t)nseg * nmodes * chunk, &a->ck);
    if (!rc)
        rc = pp::scratch(pp::SCR_QKE_PART, sizeof(double) * 6 * (size_t)nblk * ldg * chunk, &a->part);
    if (!rc)
        rc = pp::scratch(pp::SCR_QKE_X, sizeof(double) * (size_t)nblk * chunk, &a->pj);
    return rc;
}

template <typename T, int S>
int run_adjoint(const void *tab, int ldt, int ncand, int n_steps, double dt, const pp_grid *g, int chunk,
                const AdjointScratch &a, double *J, double *gs, int ldg, cudaStream_t st)
{
    void *ck = a.ck, *part = a.part, *pj = a.pj;
    const int nmodes = g->nx * g->ny * g->nz;
    const int nblk = (nmodes + kQThreads - 1) / kQThreads;
    const size_t dyn = sizeof(T) * (S == 1 ? kQRing : S) * 6 * kQThreads;
    cudaError_t ea = cudaFuncSetAttribute(qke_adjoint_kernel<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)dyn);
    if (ea != cudaSuccess)
        return pp::cuda_fail(ea, "QKE adjoint shared memory");
    for (int c0 = 0; c0 < ncand; c0 += chunk) {
        const int nc = std::min(chunk, ncand - c0);
        qke_adjoint_kernel<T, S><<<dim3(nblk, nc), kQThreads, dyn, st>>>(
            (const QkeS<T> *)tab + (size_t)c0 * ldt, ldt, n_steps, dt, *g, (T *)ck, nmodes, (double *)part, ldg,
            (double *)pj);
        sum_blocks_kernel<<<dim3(nbk(6ll * ldg), nc), 256, 0, st>>>((const double *)part, nblk, 6ll * ldg,
                                                                    gs + (size_t)c0 * 6 * ldg);
        sum_blocks_kernel<<<dim3(1, nc), 32, 0, st>>>((const double *)pj, nblk, 1, J + c0);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PP_OK : pp::cuda_fail(e, "QKE adjoint launch");
}

// State budget: bytes set by pp_set_qke_state_budget, or -1 for the default, half
// of the device's memory.
std::atomic<int64_t> g_state_budget{-1};

size_t state_budget()
{
    const int64_t b = g_state_budget.load();
    if (b >= 0)
        return (size_t)b;
    size_t free_b = 0, total = 0;
    if (cudaMemGetInfo(&free_b, &total) != cudaSuccess) {
        cudaGetLastError();
        return (size_t)8 << 30;
    }
    return total / 2;
}

// Every step's state is kept (no recomputation) when the states of enough
// candidates to fill the GPU once (2 CTAs per SM for FP32, 1 for FP64) fit the
// budget and can be allocated; otherwise one state per SR steps.
template <typename T, int SR>
int gradient(const double *A, const double *E, const double *Ed, int ncand, int ld, int n_steps, double dt,
             const pp_grid *g, double *J, double *gs, int ldg, cudaStream_t st)
{
    void *tab = nullptr;
    int ldt = 0;
    int rc = build_table<T>(A, E, Ed, ncand, ld, n_steps, &tab, &ldt, st);
    if (rc)
        return rc;
    const int nmodes = g->nx * g->ny * g->nz;
    const int nblk = (nmodes + kQThreads - 1) / kQThreads;
    const size_t budget = state_budget();
    const int sms = sm_count(), per_sm = sizeof(T) == 4 ? 2 : 1;
    const int wave = std::min(ncand, (sms * per_sm + nblk - 1) / nblk);
    AdjointScratch a;
    const size_t per1 = adjoint_bytes<T>(1, n_steps, nmodes, ldg);
    if (per1 * (size_t)wave <= budget) {
        const int chunk = wave_chunk(ncand, per1, budget, nblk, per_sm, sms);
        if (adjoint_scratch<T, 1>(n_steps, nmodes, ldg, chunk, &a) == PP_OK)
            return run_adjoint<T, 1>(tab, ldt, ncand, n_steps, dt, g, chunk, a, J, gs, ldg, st);
        cudaGetLastError();  // the kept states did not fit in free memory: recompute instead
        pp::clear_error();
    }
    const size_t perR = adjoint_bytes<T>(SR, n_steps, nmodes, ldg);
    const int chunk = wave_chunk(ncand, perR, budget, nblk, per_sm, sms);
    rc = adjoint_scratch<T, SR>(n_steps, nmodes, ldg, chunk, &a);
    if (rc)
        return rc;
    return run_adjoint<T, SR>(tab, ldt, ncand, n_steps, dt, g, chunk, a, J, gs, ldg, st);
}

}  // namespace

namespace pp {

int launch_qke_pair_number(const double *A, const double *E, const double *Ed, int ncand, int ld, int n_steps,
                           double dt, const pp_grid *g, int precision, double *N, double *n_p, cudaStream_t st)
{
    if (precision == PP_FP64)
        return forward<double>(A, E, Ed, ncand, ld, n_steps, dt, g, N, n_p, st);
    return forward<float>(A, E, Ed, ncand, ld, n_steps, dt, g, N, n_p, st);
}

// J[c] and gs[c][6][ldg] = dJ/d(A_x, A_y, E_x, E_y, Ed_x, Ed_y samples)
int launch_qke_gradient(const double *A, const double *E, const double *Ed, int ncand, int ld, int n_steps,
                        double dt, const pp_grid *g, int precision, double *J, double *gs, int ldg, cudaStream_t st)
{
    if (precision == PP_FP64)
        return gradient<double, 4>(A, E, Ed, ncand, ld, n_steps, dt, g, J, gs, ldg, st);
    return gradient<float, 8>(A, E, Ed, ncand, ld, n_steps, dt, g, J, gs, ldg, st);
}

}  // namespace pp

using namespace pp;

namespace {

int check_raw_spec(const pp_field_spec *spec)
{
    if (!spec)
        return fail(PP_ERR_INVALID_ARG, "field spec is NULL");
    pp_field_spec s = *spec;
    s.fluence = 1.0;  // not used without renormalisation
    return check_spec(&s);
}

int check_precision(int precision)
{
    if (precision != PP_FP64 && precision != PP_FP32 && precision != PP_FP32_FAST)
        return fail(PP_ERR_INVALID_ARG, "precision must be PP_FP64, PP_FP32 or PP_FP32_FAST");
    return PP_OK;
}

int check_samples(int ncand, int ld, int n_steps, double dt)
{
    if (ncand < 0 || ncand > 65535)
        return fail(PP_ERR_INVALID_ARG, "ncand must be in [0, 65535]");
    if (n_steps < 1 || n_steps > (1 << 28) || ld < 2 * n_steps + 1)
        return fail(PP_ERR_INVALID_ARG, "need 1 <= n_steps <= 2^28 and ld >= 2 n_steps + 1");
    if (!(dt > 0.0) || !isfinite(dt))
        return fail(PP_ERR_INVALID_ARG, "dt must be positive");
    return PP_OK;
}

struct GpuObjective {
    const pp_field_spec *spec;
    const pp_grid *grid;
    int precision;
    double U_const;
    cudaStream_t st;
    double *dx = nullptr, *dJ = nullptr, *dg = nullptr, *dU = nullptr, *ddU = nullptr;
    int cap = 0;
    std::vector<double> hU, hdU;
};

// The search's batched objective: J, grad J from the QKE adjoint on the GPU,
// C = U_const - U, grad C = -grad U.
int gpu_objective(void *ctx, int32_t count, const double *x, double *J, double *gJ, double *C, double *gC)
{
    GpuObjective *o = (GpuObjective *)ctx;
    const int D = 4 * o->spec->K;
    if (count > o->cap) {
        cudaFree(o->dx);
        cudaFree(o->dJ);
        cudaFree(o->dg);
        cudaFree(o->dU);
        cudaFree(o->ddU);
        o->dx = o->dJ = o->dg = o->dU = o->ddU = nullptr;
        cudaError_t e = cudaMalloc(&o->dx, sizeof(double) * (size_t)count * D);
        if (e == cudaSuccess)
            e = cudaMalloc(&o->dJ, sizeof(double) * count);
        if (e == cudaSuccess)
            e = cudaMalloc(&o->dg, sizeof(double) * (size_t)count * D);
        if (e == cudaSuccess)
            e = cudaMalloc(&o->dU, sizeof(double) * count);
        if (e == cudaSuccess)
            e = cudaMalloc(&o->ddU, sizeof(double) * (size_t)count * D);
        if (e != cudaSuccess)
            return cuda_fail(e, "local-search buffers");
        o->cap = count;
    }
    cudaError_t e = cudaMemcpyAsync(o->dx, x, sizeof(double) * (size_t)count * D, cudaMemcpyHostToDevice, o->st);
    if (e != cudaSuccess)
        return cuda_fail(e, "local-search upload");
    int rc = pp_qke_gradient(o->dx, count, o->spec, o->grid, o->precision, o->dJ, o->dg, o->dU, o->ddU, o->st);
    if (rc)
        return rc;
    o->hU.resize(count);
    o->hdU.resize((size_t)count * D);
    e = cudaMemcpyAsync(J, o->dJ, sizeof(double) * count, cudaMemcpyDeviceToHost, o->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(gJ, o->dg, sizeof(double) * (size_t)count * D, cudaMemcpyDeviceToHost, o->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(o->hU.data(), o->dU, sizeof(double) * count, cudaMemcpyDeviceToHost, o->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(o->hdU.data(), o->ddU, sizeof(double) * (size_t)count * D, cudaMemcpyDeviceToHost, o->st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(o->st);
    if (e != cudaSuccess)
        return cuda_fail(e, "local-search download");
    if ((rc = pp_sync_status(o->st)))
        return rc;
    for (int q = 0; q < count; ++q) {
        C[q] = o->U_const - o->hU[q];
        for (int i = 0; i < D; ++i)
            gC[(size_t)q * D + i] = -o->hdU[(size_t)q * D + i];
    }
    return PP_OK;
}

}  // namespace

extern "C" {

int pp_synth_field_raw(const double *params, int32_t ncand, const pp_field_spec *spec, double *A, double *E,
                       double *Ed, int32_t ld, double *U, void *stream)
{
    clear_error();
    int rc = check_raw_spec(spec);
    if (rc)
        return rc;
    if (ncand < 0 || ncand > 65535)
        return fail(PP_ERR_INVALID_ARG, "ncand must be in [0, 65535]");
    if (ncand > 0 && (!params || !A))
        return fail(PP_ERR_INVALID_ARG, "params and A must not be NULL");
    if (ld < 2 * spec->n_steps + 1)
        return fail(PP_ERR_INVALID_ARG, "ld must be >= 2 n_steps + 1");
    return launch_synth(params, ncand, spec, 0, A, ld, E, Ed, U, (cudaStream_t)stream);
}

int pp_synth_vjp(const double *params, int32_t ncand, const pp_field_spec *spec, const double *g, int32_t ldg,
                 double *grad, double *U, double *dU, void *stream)
{
    clear_error();
    int rc = check_raw_spec(spec);
    if (rc)
        return rc;
    if (ncand < 0 || ncand > 65535)
        return fail(PP_ERR_INVALID_ARG, "ncand must be in [0, 65535]");
    if (ncand > 0 && (!params || (grad && !g)))
        return fail(PP_ERR_INVALID_ARG, "params (and g when grad is wanted) must not be NULL");
    if (grad && ldg < 2 * spec->n_steps + 1)
        return fail(PP_ERR_INVALID_ARG, "ldg must be >= 2 n_steps + 1");
    return launch_synth_vjp(params, ncand, spec, g, ldg, grad, U, dU, (cudaStream_t)stream);
}

int pp_qke_pair_number(const double *A, const double *E, const double *Ed, int32_t ncand, int32_t ld,
                       int32_t n_steps, double dt, const pp_grid *grid, int32_t precision, double *N, double *n_p,
                       void *stream)
{
    clear_error();
    int rc = check_samples(ncand, ld, n_steps, dt);
    if (!rc)
        rc = check_grid(grid);
    if (!rc)
        rc = check_precision(precision);
    if (rc)
        return rc;
    if (ncand == 0)
        return PP_OK;
    if (!A || !E || !Ed || !N)
        return fail(PP_ERR_INVALID_ARG, "A, E, Ed and N must not be NULL");
    return launch_qke_pair_number(A, E, Ed, ncand, ld, n_steps, dt, grid, precision, N, n_p, (cudaStream_t)stream);
}

int pp_qke_sample_gradient(const double *A, const double *E, const double *Ed, int32_t ncand, int32_t ld,
                           int32_t n_steps, double dt, const pp_grid *grid, int32_t precision, double *J, double *g,
                           int32_t ldg, void *stream)
{
    clear_error();
    int rc = check_samples(ncand, ld, n_steps, dt);
    if (!rc)
        rc = check_grid(grid);
    if (!rc)
        rc = check_precision(precision);
    if (rc)
        return rc;
    if (ncand == 0)
        return PP_OK;
    if (!A || !E || !Ed || !J || !g)
        return fail(PP_ERR_INVALID_ARG, "A, E, Ed, J and g must not be NULL");
    if (ldg < 2 * n_steps + 1)
        return fail(PP_ERR_INVALID_ARG, "ldg must be >= 2 n_steps + 1");
    return launch_qke_gradient(A, E, Ed, ncand, ld, n_steps, dt, grid, precision, J, g, ldg, (cudaStream_t)stream);
}

int64_t pp_set_qke_state_budget(int64_t bytes)
{
    return g_state_budget.exchange(bytes < 0 ? -1 : bytes);
}

int pp_qke_gradient(const double *params, int32_t ncand, const pp_field_spec *spec, const pp_grid *grid,
                    int32_t precision, double *J, double *gJ, double *U, double *dU, void *stream)
{
    clear_error();
    int rc = check_raw_spec(spec);
    if (!rc)
        rc = check_grid(grid);
    if (!rc)
        rc = check_precision(precision);
    if (rc)
        return rc;
    if (ncand < 0 || ncand > 65535)
        return fail(PP_ERR_INVALID_ARG, "ncand must be in [0, 65535]");
    if (ncand == 0)
        return PP_OK;
    if (!params || !J)
        return fail(PP_ERR_INVALID_ARG, "params and J must not be NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const int n = spec->n_steps, ld = 2 * n + 1;
    void *fld = nullptr, *gs = nullptr;
    rc = scratch(SCR_QKE_FIELD, sizeof(double) * 3 * 2 * (size_t)ld * ncand, &fld);
    if (!rc && gJ)
        rc = scratch(SCR_QKE_G, sizeof(double) * 6 * (size_t)ld * ncand, &gs);
    if (rc)
        return rc;
    double *A = (double *)fld, *E = A + 2 * (size_t)ld * ncand, *Ed = E + 2 * (size_t)ld * ncand;
    if ((rc = launch_synth(params, ncand, spec, 0, A, ld, E, Ed, nullptr, st)))
        return rc;
    const double dt = spec->T / n;
    if (gJ) {
        if ((rc = launch_qke_gradient(A, E, Ed, ncand, ld, n, dt, grid, precision, J, (double *)gs, ld, st)))
            return rc;
    } else if ((rc = launch_qke_pair_number(A, E, Ed, ncand, ld, n, dt, grid, precision, J, nullptr, st))) {
        return rc;
    }
    if (gJ || U || dU)
        return launch_synth_vjp(params, ncand, spec, (const double *)gs, ld, gJ, U, dU, st);
    return PP_OK;
}

int pp_local_search(double *x, int32_t nstart, const pp_field_spec *spec, const pp_grid *grid, int32_t precision,
                    double U_const, const pp_al_options *opt, double *J_out, double *C_out, double *lam_out,
                    int32_t *evals_out, int32_t *outer_out, int32_t *status_out, void *stream)
{
    clear_error();
    int rc = check_raw_spec(spec);
    if (!rc)
        rc = check_grid(grid);
    if (!rc)
        rc = check_precision(precision);
    if (rc)
        return rc;
    if (!(U_const > 0.0) || !isfinite(U_const))
        return fail(PP_ERR_INVALID_ARG, "U_const must be positive");
    GpuObjective o;
    o.spec = spec;
    o.grid = grid;
    o.precision = precision;
    o.U_const = U_const;
    o.st = (cudaStream_t)stream;
    rc = pp_al_search(4 * spec->K, nstart, x, gpu_objective, &o, opt, J_out, C_out, lam_out, evals_out, outer_out,
                      status_out);
    cudaFree(o.dx);
    cudaFree(o.dJ);
    cudaFree(o.dg);
    cudaFree(o.dU);
    cudaFree(o.ddU);
    return rc;
}

}  // extern "C"
