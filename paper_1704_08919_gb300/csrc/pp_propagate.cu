// pp_propagate.cu -- per-mode Dirac propagation, projection and momentum sum
// (Sec. II.A of arXiv 1704.08919: Eqs. (kin_mom), (free_spin1), (wf_init),
// (dirac_eq_mom), (pair_prod_homo); Eq. (opt_prob)).
//
// Reduction used on the GPU.  For a field in the x-y plane the Hermitian
// operator O = p_z gamma^5 + sigma_z (x) sigma_z (gamma^5 = sigma_x (x) 1 in the
// Dirac representation) commutes with H(t) = alpha.(p - A(t)) + beta at every
// t, and O^2 = (1 + p_z^2) 1.  Each eigenspace of O (eigenvalue s eps_perp,
// eps_perp = sqrt(1 + p_z^2), s = +-1) is invariant and holds one positive- and
// one negative-energy state; in a fixed orthonormal basis of that eigenspace H
// acts as the 2x2 matrix h_s . sigma with
//     h_s(t) = (P_x(t), s P_y(t), eps_perp),   P = p - A(t).
// So the 4-spinor equation for both spins is two 2-level equations.  RK4 is a
// polynomial in dt H, so it commutes with the constant change of basis: RK4 on
// the two 2-level systems produces exactly the RK4 iterates of the 4-spinor
// equation.  The negative-energy subspace at t_0 is spanned by the two
// negative eigenvectors |-, h_s(t_0)>, and the full spin trace of Eq.
// (pair_prod_homo) is
//     f(p) = sum_s |<+, h_s(t_end) | U_s |-, h_s(t_0)>|^2.
//
// RK4 in increment form (one step, M_t = -i h(t).sigma, z = dt/6):
//     e1 = z M_n psi,             y1 = psi + 3 e1
//     e2 = 2z M_{n+1/2} y1,       y2 = psi + 1.5 e2
//     e3 = 2z M_{n+1/2} y2,       y3 = psi + 3 e3
//     psi <- psi + (e1 + e2 + e3 + z M_{n+1} y3)
// which is the classical psi + dt/6 (k1 + 2 k2 + 2 k3 + k4).  In the FP32 path
// the state is a two-float (hi, lo) pair and the increment is added with
// Fast2Sum, so the O(1) state does not lose the small increments' low bits;
// the initial state, the projection and the momentum sum are FP64.
#include <math.h>

#include "pp_internal.cuh"

namespace {

constexpr int kThreads = 256;

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

// Steps per shared-memory tile: 8 KiB per buffer in both precisions.
template <typename T>
struct TileSteps {
    static constexpr int value = 8192 / (int)sizeof(typename Vec4<T>::type);
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

// Table entry of step n: ((dt/3) A(t_{n+1/2}), (dt/6) A(t_{n+1})), zero past n_steps.
template <typename T>
__global__ void build_table_kernel(const double *__restrict__ A, int ld, int ns_uniform,
                                   const int *__restrict__ ns_array, int padded, double dt,
                                   typename Vec4<T>::type *__restrict__ table)
{
    int c = blockIdx.y;
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= padded)
        return;
    int ns = ns_array ? ns_array[c] : ns_uniform;
    const double *Ax = A + (size_t)c * 2 * ld, *Ay = Ax + ld;
    typename Vec4<T>::type e;
    if (n < ns) {
        double d3 = dt / 3.0, d6 = dt / 6.0;
        e.x = (T)(d3 * Ax[2 * n + 1]);
        e.y = (T)(d3 * Ay[2 * n + 1]);
        e.z = (T)(d6 * Ax[2 * n + 2]);
        e.w = (T)(d6 * Ay[2 * n + 2]);
    } else {
        e.x = e.y = e.z = e.w = (T)0;
    }
    table[(size_t)c * padded + n] = e;
}

template <typename T, bool COMP>
__global__ void __launch_bounds__(kThreads)
    propagate_kernel(const double *__restrict__ A, int ld, int ns_uniform,
                     const int *__restrict__ ns_array, const typename Vec4<T>::type *__restrict__ table,
                     int padded, double dt, pp_grid g, double *__restrict__ n_p,
                     double *__restrict__ partial, long long wait_limit, int skip_copies,
                     unsigned int *__restrict__ status)
{
    using V = typename Vec4<T>::type;
    constexpr int TILE = TileSteps<T>::value;
    __shared__ __align__(128) V buf[2][TILE];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ double red[kThreads / 32];

    const int c = blockIdx.y;
    const int tid = threadIdx.x;
    const int nmodes = g.nx * g.ny * g.nz;
    const int m = blockIdx.x * kThreads + tid;
    const bool active = m < nmodes;
    const int ns = ns_array ? ns_array[c] : ns_uniform;
    const int ntiles = (ns + TILE - 1) / TILE;
    const V *trow = table + (size_t)c * padded;
    const double *Ax = A + (size_t)c * 2 * ld, *Ay = Ax + ld;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    int issued = 0;  // meaningful in thread 0 only
    if (tid == 0 && !skip_copies) {
        for (int t = 0; t < 2 && t < ntiles; ++t) {
            mbar_arrive_expect_tx(&bar[t], TILE * (uint32_t)sizeof(V));
            bulk_copy_g2s(buf[t], trow + (size_t)t * TILE, TILE * (uint32_t)sizeof(V), &bar[t]);
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
    const double d3 = dt / 3.0, d6 = dt / 6.0;

    T hi[2][4], lo[2][4];
    {
        double Pinx = px - Ax[0], Piny = py - Ay[0];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            double v[4];
            eig_neg(Pinx, s ? -Piny : Piny, eperp, v);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                hi[s][q] = (T)v[q];
                lo[s][q] = (T)(v[q] - (double)hi[s][q]);
            }
        }
    }
    const T px3 = (T)(d3 * px), py3 = (T)(d3 * py);
    const T px6 = (T)(d6 * px), py6 = (T)(d6 * py);
    const T ez3 = (T)(d3 * eperp), ez6 = (T)(d6 * eperp);
    T q6x = px6 - (T)(d6 * Ax[0]);
    T q6y = py6 - (T)(d6 * Ay[0]);

    bool timed_out = false;
    int t_fail = 0;
    for (int t = 0; t < ntiles; ++t) {
        const int b = t & 1;
        const uint32_t par = (t >> 1) & 1;
        bool ok = mbar_wait_bounded(&bar[b], par, wait_limit);
        ok = __syncthreads_and(ok);
        if (!ok) {
            timed_out = true;
            t_fail = t;
            break;
        }
        const int nst = min(TILE, ns - t * TILE);
        if (active) {
            const V *tb = buf[b];
#pragma unroll 2
            for (int k = 0; k < nst; ++k) {
                const V e = tb[k];
                const T q3x = px3 - e.x, q3y = py3 - e.y;
                const T n6x = px6 - e.z, n6y = py6 - e.w;
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const T a6 = s ? -q6y : q6y;
                    const T a3 = s ? -q3y : q3y;
                    const T b6 = s ? -n6y : n6y;
                    T e1[4], e2[4], y[4], S[4];
                    rot(q6x, a6, ez6, hi[s], e1);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        y[q] = fma((T)3, e1[q], hi[s][q]);
                    rot(q3x, a3, ez3, y, e2);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        y[q] = fma((T)1.5, e2[q], hi[s][q]);
                        S[q] = e1[q] + e2[q];
                    }
                    rot(q3x, a3, ez3, y, e2);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        y[q] = fma((T)3, e2[q], hi[s][q]);
                        S[q] = S[q] + e2[q];
                        if (COMP)
                            S[q] = S[q] + lo[s][q];
                    }
                    rot_acc(n6x, b6, ez6, y, S);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (COMP) {
                            const T h = hi[s][q] + S[q];
                            lo[s][q] = S[q] - (h - hi[s][q]);
                            hi[s][q] = h;
                        } else {
                            hi[s][q] = hi[s][q] + S[q];
                        }
                    }
                }
                q6x = n6x;
                q6y = n6y;
            }
        }
        __syncthreads();  // every thread is done with buf[b]
        if (tid == 0 && !skip_copies && t + 2 < ntiles) {
            mbar_arrive_expect_tx(&bar[b], TILE * (uint32_t)sizeof(V));
            bulk_copy_g2s(buf[b], trow + (size_t)(t + 2) * TILE, TILE * (uint32_t)sizeof(V), &bar[b]);
            ++issued;
        }
    }

    if (timed_out) {
        // Drain every copy this CTA issued (bounded) before shared memory is released.
        if (tid == 0) {
            pp_flag(status, PP_FLAG_TIMEOUT);
            // copies t_fail <= t < issued were never consumed: wait for each in order
            for (int t = t_fail; t < issued; ++t)
                mbar_wait_bounded(&bar[t & 1], (t >> 1) & 1, 1ll << 24);
        }
        __syncthreads();
    }

    // ---- FP64 projection onto the positive-energy states at t_end
    double f = 0.0;
    if (active) {
        double Poutx = px - Ax[2 * ns], Pouty = py - Ay[2 * ns];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            double psi[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                psi[q] = COMP ? (double)hi[s][q] + (double)lo[s][q] : (double)hi[s][q];
            f += proj_pos2(Poutx, s ? -Pouty : Pouty, eperp, psi);
        }
        if (timed_out)
            f = __longlong_as_double(0x7ff8000000000000ll);
        if (n_p)
            n_p[(size_t)c * nmodes + m] = f;
    }
    double wf = 0.0;
    if (active) {
        double w = __dmul_rn(__dmul_rn(axis_weight(ix, g.nx, g.x0, g.x1, 0),
                                       axis_weight(iy, g.ny, g.y0, g.y1, 0)),
                             axis_weight(iz, g.nz, g.z0, g.z1, g.mirror_z));
        wf = w * f;
    }
    // fixed-order block reduction
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        wf += __shfl_down_sync(0xffffffffu, wf, off);
    if ((tid & 31) == 0)
        red[tid >> 5] = wf;
    __syncthreads();
    if (tid == 0) {
        double acc = 0.0;
        for (int w = 0; w < kThreads / 32; ++w)
            acc += red[w];
        partial[(size_t)c * gridDim.x + blockIdx.x] = acc;
    }
}

// N[c] = sum of the per-block partials of candidate c, in a fixed order.
__global__ void finalize_kernel(const double *__restrict__ partial, int nblk, double *__restrict__ N,
                                unsigned int *__restrict__ status)
{
    __shared__ double red[256];
    int c = blockIdx.x;
    double acc = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x)
        acc += partial[(size_t)c * nblk + i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double v = red[0];
        if (!isfinite(v))
            pp_flag(status, PP_FLAG_NONFINITE);
        N[c] = v;
    }
}

template <typename T, bool COMP>
int run(const double *A, int ncand, int ld, const int32_t *ns_host, double dt, const pp_grid *grid,
        double *N, double *n_p, cudaStream_t stream)
{
    using V = typename Vec4<T>::type;
    constexpr int TILE = TileSteps<T>::value;
    int max_ns = 0;
    bool uniform = true;
    int ns0 = ns_host ? ns_host[0] : (ld - 1) / 2;
    for (int c = 0; c < ncand; ++c) {
        int ns = ns_host ? ns_host[c] : ns0;
        max_ns = ns > max_ns ? ns : max_ns;
        uniform &= (ns == ns0);
    }
    const int padded = ((max_ns + TILE - 1) / TILE) * TILE;
    unsigned int *status = pp::status_word();
    if (!status)
        return pp::fail(PP_ERR_CUDA, "status word unavailable");
    const int nmodes = grid->nx * grid->ny * grid->nz;
    const int nblk = (nmodes + kThreads - 1) / kThreads;

    void *table = nullptr, *partial = nullptr, *nsdev = nullptr;
    int rc = pp::scratch(pp::SCR_TABLE, (size_t)ncand * padded * sizeof(V), &table);
    if (rc)
        return rc;
    rc = pp::scratch(pp::SCR_PARTIAL, (size_t)ncand * nblk * sizeof(double) + 256 * sizeof(int) +
                                          (size_t)ncand * sizeof(int),
                     &partial);
    if (rc)
        return rc;
    const int *ns_array = nullptr;
    if (!uniform) {
        nsdev = (char *)partial + (size_t)ncand * nblk * sizeof(double);
        nsdev = (void *)(((uintptr_t)nsdev + 255) & ~(uintptr_t)255);
        cudaError_t e = cudaMemcpyAsync(nsdev, ns_host, sizeof(int) * ncand, cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess)
            return pp::cuda_fail(e, "copy of n_steps");
        ns_array = (const int *)nsdev;
    }
    dim3 tg((padded + 255) / 256, ncand);
    build_table_kernel<T><<<tg, 256, 0, stream>>>(A, ld, ns0, ns_array, padded, dt, (V *)table);
    dim3 pg(nblk, ncand);
    pp::profile_mark_start(stream);
    propagate_kernel<T, COMP><<<pg, kThreads, 0, stream>>>(A, ld, ns0, ns_array, (const V *)table,
                                                             padded, dt, *grid, n_p, (double *)partial,
                                                             (long long)pp::wait_limit(), pp::skip_copies(), status);
    pp::profile_mark_stop(stream);
    finalize_kernel<<<ncand, 256, 0, stream>>>((const double *)partial, nblk, N, status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return pp::cuda_fail(e, "pair-number kernel launch");
    return PP_OK;
}

}  // namespace

namespace pp {

int launch_pair_number(const double *A, int ncand, int ld, const int32_t *n_steps_host, double dt,
                       const pp_grid *grid, int precision, double *N, double *n_p, cudaStream_t stream)
{
    if (precision == PP_FP64)
        return run<double, false>(A, ncand, ld, n_steps_host, dt, grid, N, n_p, stream);
    return run<float, true>(A, ncand, ld, n_steps_host, dt, grid, N, n_p, stream);
}

}  // namespace pp
