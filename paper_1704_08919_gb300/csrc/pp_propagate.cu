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
#include <map>
#include <mutex>

#include "pp_policies.cuh"

namespace {

// WIDE = false: the candidates whose steps stay in the policy's series range (all
// candidates for policies without one); WIDE = true: the others (see
// build_table_kernel).  A CTA of the other kind returns at once.
template <class P, int THREADS, int TILE_BYTES, bool WIDE>
__global__ void __launch_bounds__(THREADS)
    propagate_kernel(const double *__restrict__ A, int ld, int ns_uniform,
                     const int *__restrict__ ns_array, const typename P::Entry *__restrict__ table,
                     int padded, double dt, pp_grid g, double *__restrict__ n_p,
                     double *__restrict__ partial, long long wait_limit, int skip_copies,
                     unsigned int *__restrict__ status, const int *__restrict__ wide_flags)
{
    __shared__ ItemSmem<P, THREADS, TILE_BYTES> sm;
    const int c = blockIdx.y;
    if (!takes_candidate<P, WIDE>(wide_flags, c))
        return;
    const int nmodes = g.nx * g.ny * g.nz;
    const int ngroups = (nmodes + kGroup - 1) / kGroup;
    const int ns = ns_array ? ns_array[c] : ns_uniform;
    const double *Ax = A + (size_t)c * 2 * ld;
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    process_item<P, THREADS, TILE_BYTES, WIDE>(sm, blockIdx.x, g, ns, table + (size_t)c * padded, Ax,
                                         Ax + ld, dt, n_p ? n_p + (size_t)c * nmodes : nullptr,
                                         partial + (size_t)c * ngroups, wait_limit, skip_copies,
                                         status, 0);
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

template <class P, int THREADS, int TILE_BYTES>
int run(const double *A, int ncand, int ld, const int32_t *ns_host, double dt, const pp_grid *grid,
        double *N, double *n_p, cudaStream_t stream)
{
    using V = typename P::Entry;
    constexpr int TILE = TILE_BYTES / (int)sizeof(V);
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
    const int nblk = (nmodes + THREADS - 1) / THREADS;
    const int ngroups = (nmodes + kGroup - 1) / kGroup;

    void *table = nullptr, *partial = nullptr, *nsdev = nullptr;
    int rc = pp::scratch(pp::SCR_TABLE, (size_t)ncand * padded * sizeof(V), &table);
    if (rc)
        return rc;
    rc = pp::scratch(pp::SCR_PARTIAL, (size_t)ncand * ngroups * sizeof(double) + 512 * sizeof(int) +
                                          2 * (size_t)ncand * sizeof(int),
                     &partial);
    if (rc)
        return rc;
    // after the partial sums: the per-candidate wide flags, then (uneven) n_steps
    int *flags = (int *)(((uintptr_t)((char *)partial + (size_t)ncand * ngroups * sizeof(double)) + 255) &
                         ~(uintptr_t)255);
    const int *ns_array = nullptr;
    if (!uniform) {
        nsdev = (void *)(((uintptr_t)(flags + ncand) + 255) & ~(uintptr_t)255);
        cudaError_t e = cudaMemcpyAsync(nsdev, ns_host, sizeof(int) * ncand, cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess)
            return pp::cuda_fail(e, "copy of n_steps");
        ns_array = (const int *)nsdev;
    }
    cudaError_t ez = cudaMemsetAsync(flags, 0, sizeof(int) * ncand, stream);
    if (ez != cudaSuccess)
        return pp::cuda_fail(ez, "wide-flag reset");
    dim3 tg((padded + 255) / 256, ncand);
    build_table_kernel<P><<<tg, 256, 0, stream>>>(A, ld, ns0, ns_array, padded, dt, *grid, (V *)table, flags);
    dim3 pg(nblk, ncand);
    pp::profile_mark_start(stream);
    propagate_kernel<P, THREADS, TILE_BYTES, false><<<pg, THREADS, 0, stream>>>(
        A, ld, ns0, ns_array, (const V *)table, padded, dt, *grid, n_p, (double *)partial,
        (long long)pp::wait_limit(), pp::skip_copies(), status, flags);
    if constexpr (HasSeriesGuard<P>::value)
        propagate_kernel<P, THREADS, TILE_BYTES, true><<<pg, THREADS, 0, stream>>>(
            A, ld, ns0, ns_array, (const V *)table, padded, dt, *grid, n_p, (double *)partial,
            (long long)pp::wait_limit(), pp::skip_copies(), status, flags);
    pp::profile_mark_stop(stream);
    finalize_kernel<<<ncand, 256, 0, stream>>>((const double *)partial, ngroups, N, status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return pp::cuda_fail(e, "pair-number kernel launch");
    return PP_OK;
}

// ---------------------------------------------------------------- no-allocation variant
// Scratch of pp_pair_number_static: a fixed device array in this file, held by
// every GPU that loads the library until the process exits.  It holds, in
// order, the per-step table, the per-block partial sums, the per-candidate
// wide-range flags (cleared by each call before use) and (for uneven step
// counts) a copy of n_steps; each call writes every byte it later reads, and
// calls that overlap on the GPU race on it.
constexpr size_t kStaticScratchBytes = (size_t)16 << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of g_static_scratch on the current device, looked up once per
// device (host code must not use the symbol itself as a device address).
unsigned char *static_scratch_address()
{
    constexpr int kMaxDev = 64;
    static unsigned char *addr[kMaxDev] = {};
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev)
        return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess)
            return nullptr;
        addr[dev] = (unsigned char *)p;
    }
    return addr[dev];
}

template <class P, int THREADS, int TILE_BYTES>
int run_static(const double *A, int ncand, int ld, const int32_t *ns_host, double dt,
               const pp_grid *grid, double *N, double *n_p, cudaStream_t stream)
{
    using V = typename P::Entry;
    constexpr int TILE = TILE_BYTES / (int)sizeof(V);
    int max_ns = 0;
    bool uniform = true;
    const int ns0 = ns_host ? ns_host[0] : (ld - 1) / 2;
    for (int c = 0; c < ncand; ++c) {
        const int ns = ns_host ? ns_host[c] : ns0;
        max_ns = ns > max_ns ? ns : max_ns;
        uniform &= (ns == ns0);
    }
    const int padded = ((max_ns + TILE - 1) / TILE) * TILE;
    const int nmodes = grid->nx * grid->ny * grid->nz;
    const int nblk = (nmodes + THREADS - 1) / THREADS;
    const int ngroups = (nmodes + kGroup - 1) / kGroup;
    const size_t table_bytes = align256((size_t)ncand * padded * sizeof(V));
    const size_t part_bytes = align256((size_t)ncand * ngroups * sizeof(double));
    const size_t flag_bytes = align256((size_t)ncand * sizeof(int));
    const size_t ns_bytes = uniform ? 0 : align256((size_t)ncand * sizeof(int));
    const size_t need = table_bytes + part_bytes + flag_bytes + ns_bytes;
    if (need > kStaticScratchBytes)
        return pp::fail(PP_ERR_INVALID_ARG,
                        "this call needs %zu bytes of scratch; the static scratch holds %zu "
                        "(use fewer candidates, steps or modes, or pp_pair_number)",
                        need, kStaticScratchBytes);
    unsigned char *base = static_scratch_address();
    if (!base)
        return pp::fail(PP_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
    unsigned int *status = pp::status_word();
    if (!status)
        return pp::fail(PP_ERR_CUDA, "status word unavailable");
    V *table = (V *)base;
    double *partial = (double *)(base + table_bytes);
    int *flags = (int *)(base + table_bytes + part_bytes);
    const int *ns_array = nullptr;
    if (!uniform) {
        int *nsdev = (int *)(base + table_bytes + part_bytes + flag_bytes);
        cudaError_t e = cudaMemcpyAsync(nsdev, ns_host, sizeof(int) * ncand, cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess)
            return pp::cuda_fail(e, "copy of n_steps");
        ns_array = nsdev;
    }
    cudaError_t ez = cudaMemsetAsync(flags, 0, sizeof(int) * ncand, stream);
    if (ez != cudaSuccess)
        return pp::cuda_fail(ez, "wide-flag reset");
    dim3 tg((padded + 255) / 256, ncand);
    build_table_kernel<P><<<tg, 256, 0, stream>>>(A, ld, ns0, ns_array, padded, dt, *grid, table, flags);
    dim3 pg(nblk, ncand);
    propagate_kernel<P, THREADS, TILE_BYTES, false><<<pg, THREADS, 0, stream>>>(
        A, ld, ns0, ns_array, table, padded, dt, *grid, n_p, partial, (long long)pp::wait_limit(),
        pp::skip_copies(), status, flags);
    if constexpr (HasSeriesGuard<P>::value)
        propagate_kernel<P, THREADS, TILE_BYTES, true><<<pg, THREADS, 0, stream>>>(
            A, ld, ns0, ns_array, table, padded, dt, *grid, n_p, partial, (long long)pp::wait_limit(),
            pp::skip_copies(), status, flags);
    finalize_kernel<<<ncand, 256, 0, stream>>>(partial, ngroups, N, status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return pp::cuda_fail(e, "pair-number kernel launch");
    return PP_OK;
}

// ---------------------------------------------------------------- launch configurations
// (threads per CTA, bytes per shared-memory tile buffer).  FP32 paths may use
// any of them (chosen by pp_tune_pair_number, else kDefault*); FP64 paths use
// configuration 0.  The arithmetic does not depend on the configuration.
constexpr int kNumConfigs = 6;
constexpr int kCfgThreads[kNumConfigs] = {256, 128, 512, 256, 128, 512};
constexpr int kCfgTileBytes[kNumConfigs] = {8192, 8192, 8192, 32768, 32768, 32768};

using LaunchFn = int (*)(const double *, int, int, const int32_t *, double, const pp_grid *, double *,
                         double *, cudaStream_t);

template <class P, bool ALL>
struct ConfigTable {
    LaunchFn run_fn[kNumConfigs];
    LaunchFn static_fn[kNumConfigs];
    ConfigTable()
    {
        if constexpr (ALL) {
            run_fn[0] = &run<P, 256, 8192>;
            run_fn[1] = &run<P, 128, 8192>;
            run_fn[2] = &run<P, 512, 8192>;
            run_fn[3] = &run<P, 256, 32768>;
            run_fn[4] = &run<P, 128, 32768>;
            run_fn[5] = &run<P, 512, 32768>;
            static_fn[0] = &run_static<P, 256, 8192>;
            static_fn[1] = &run_static<P, 128, 8192>;
            static_fn[2] = &run_static<P, 512, 8192>;
            static_fn[3] = &run_static<P, 256, 32768>;
            static_fn[4] = &run_static<P, 128, 32768>;
            static_fn[5] = &run_static<P, 512, 32768>;
        } else {
            for (int k = 0; k < kNumConfigs; ++k) {
                run_fn[k] = &run<P, 256, 8192>;
                static_fn[k] = &run_static<P, 256, 8192>;
            }
        }
    }
};

// Policy by (precision, scheme).
struct PolicySlot {
    const LaunchFn *run_fn;
    const LaunchFn *static_fn;
    bool tunable;
    int default_cfg;
};

const PolicySlot &policy_slot(int precision, int scheme)
{
    static const ConfigTable<ScalarPolicy<double, false>, true> d_rk4;  // tunable: small FP64 grids
    static const ConfigTable<MagnusPolicy<double, false>, false> d_mag;
    static const ConfigTable<SplitPolicy<double, false>, false> d_spl;
    static const ConfigTable<PackedPolicy<true>, true> f_rk4;
    static const ConfigTable<MagnusPolicy<float, true>, true> f_mag;
    static const ConfigTable<SplitPolicy<float, true>, true> f_spl;
    static const ConfigTable<PackedPolicy<false>, true> x_rk4;
    static const ConfigTable<MagnusPolicy<float, false>, true> x_mag;
    static const ConfigTable<SplitPolicy<float, false>, true> x_spl;
    // defaults from timing the 64-candidate workload on GB300 (see the tuner)
    static const PolicySlot slots[3][3] = {
        {{d_rk4.run_fn, d_rk4.static_fn, true, 0}, {d_mag.run_fn, d_mag.static_fn, false, 0},
         {d_spl.run_fn, d_spl.static_fn, false, 0}},
        {{f_rk4.run_fn, f_rk4.static_fn, true, 0}, {f_mag.run_fn, f_mag.static_fn, true, 2},
         {f_spl.run_fn, f_spl.static_fn, true, 0}},
        {{x_rk4.run_fn, x_rk4.static_fn, true, 0}, {x_mag.run_fn, x_mag.static_fn, true, 0},
         {x_spl.run_fn, x_spl.static_fn, true, 3}},
    };
    return slots[precision][scheme];
}

// Tuned configurations, keyed by the workload shape.
struct TuneKey {
    int precision, scheme, ncand, nmodes, max_ns;
    bool operator<(const TuneKey &o) const
    {
        if (precision != o.precision) return precision < o.precision;
        if (scheme != o.scheme) return scheme < o.scheme;
        if (ncand != o.ncand) return ncand < o.ncand;
        if (nmodes != o.nmodes) return nmodes < o.nmodes;
        return max_ns < o.max_ns;
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tuned;

TuneKey make_key(int precision, int scheme, int ncand, int ld, const int32_t *ns, const pp_grid *g)
{
    int max_ns = 0;
    for (int c = 0; c < ncand; ++c) {
        const int v = ns ? ns[c] : (ld - 1) / 2;
        max_ns = v > max_ns ? v : max_ns;
    }
    return TuneKey{precision, scheme, ncand, g->nx * g->ny * g->nz, max_ns};
}

int chosen_config(int precision, int scheme, int ncand, int ld, const int32_t *ns, const pp_grid *g)
{
    const PolicySlot &slot = policy_slot(precision, scheme);
    if (!slot.tunable)
        return 0;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(make_key(precision, scheme, ncand, ld, ns, g));
    return it == g_tuned.end() ? slot.default_cfg : it->second;
}

}  // namespace

namespace pp {

int launch_pair_number(const double *A, int ncand, int ld, const int32_t *n_steps_host, double dt,
                       const pp_grid *grid, int precision, int scheme, double *N, double *n_p,
                       cudaStream_t stream)
{
    const int cfg = chosen_config(precision, scheme, ncand, ld, n_steps_host, grid);
    return policy_slot(precision, scheme).run_fn[cfg](A, ncand, ld, n_steps_host, dt, grid, N, n_p,
                                                      stream);
}

int launch_pair_number_static(const double *A, int ncand, int ld, const int32_t *n_steps_host,
                              double dt, const pp_grid *grid, int precision, int scheme, double *N,
                              double *n_p, cudaStream_t stream)
{
    const int cfg = chosen_config(precision, scheme, ncand, ld, n_steps_host, grid);
    return policy_slot(precision, scheme).static_fn[cfg](A, ncand, ld, n_steps_host, dt, grid, N,
                                                         n_p, stream);
}

size_t static_scratch_bytes() { return kStaticScratchBytes; }

int num_launch_configs() { return kNumConfigs; }

int tune_pair_number(const double *A, int ncand, int ld, const int32_t *n_steps_host, double dt,
                     const pp_grid *grid, int precision, int scheme, double *N, int32_t *chosen,
                     float *config_ms, cudaStream_t stream)
{
    const PolicySlot &slot = policy_slot(precision, scheme);
    const int ncfg = slot.tunable ? kNumConfigs : 1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e1);
    if (e != cudaSuccess)
        return cuda_fail(e, "tuner event");
    int best = slot.default_cfg;
    float best_ms = 3.0e38f;
    int rc = PP_OK;
    for (int k = 0; k < ncfg && rc == PP_OK; ++k) {
        // one untimed launch (table build, caches), then one timed launch
        rc = slot.run_fn[k](A, ncand, ld, n_steps_host, dt, grid, N, nullptr, stream);
        if (rc)
            break;
        cudaEventRecord(e0, stream);
        rc = slot.run_fn[k](A, ncand, ld, n_steps_host, dt, grid, N, nullptr, stream);
        cudaEventRecord(e1, stream);
        if (rc)
            break;
        float ms = 0.0f;
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "tuner timing");
            break;
        }
        if (config_ms)
            config_ms[k] = ms;
        if (ms < best_ms) {
            best_ms = ms;
            best = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc)
        return rc;
    if (slot.tunable) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[make_key(precision, scheme, ncand, ld, n_steps_host, grid)] = best;
    }
    if (chosen)
        *chosen = best;
    return PP_OK;
}

void clear_tuning()
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned.clear();
}

void launch_config(int k, int *threads, int *tile_bytes)
{
    *threads = kCfgThreads[k];
    *tile_bytes = kCfgTileBytes[k];
}

}  // namespace pp
