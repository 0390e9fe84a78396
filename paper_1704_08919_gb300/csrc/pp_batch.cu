// pp_batch.cu -- uneven batches: candidates with their own pulse length, step
// count and momentum grid scored in one persistent launch, and whole DE
// generations captured in a CUDA graph (the pp_batch_* entry points).
//
// Work is split into items (candidate c, block of THREADS modes).  The items are
// listed longest first (by step count, then candidate and block) and handed out
// by an atomic counter to a grid sized to fill the GPU once, so long and short
// candidates share the machine without a tail of idle SMs.  Each item runs the
// same per-mode body as the uniform kernel (pp_policies.cuh); the mbarrier
// phases of a CTA run on from item to item.  Partial sums are kept per
// candidate in fixed groups of 128 modes, so N is bitwise what pp_pair_number
// gives for that candidate alone.
#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "pp_policies.cuh"

namespace {

struct BatchCand {
    pp_grid g;
    int ns;
    int ngroups;
    long long table_off;  // table entries before this candidate's row
    long long n_off;      // n(p) values before this candidate's
    long long part_off;   // partial sums before this candidate's
};

// As build_table_kernel, per slot with its own grid and step count; wide_flags[c]
// (zeroed before the launch) marks slots that leave the policy's series range.
template <class P>
__global__ void build_table_batch_kernel(const double *__restrict__ A, int ld,
                                         const BatchCand *__restrict__ cands, int row_quantum, double dt,
                                         typename P::Entry *__restrict__ table, int *__restrict__ wide_flags)
{
    const int c = blockIdx.y;
    const BatchCand d = cands[c];
    const int padded = ((d.ns + row_quantum - 1) / row_quantum) * row_quantum;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const double *Ax = A + (size_t)c * 2 * ld, *Ay = Ax + ld;
    bool big = false;
    if (n < padded) {
        typename P::Entry e;
        if (n < d.ns) {
            e = table_entry((const P *)nullptr, Ax, Ay, n, dt, d.g);
            if constexpr (HasSeriesGuard<P>::value)
                big = P::beyond_series(e);
        } else {
            memset(&e, 0, sizeof e);
        }
        table[d.table_off + n] = e;
    }
    if constexpr (HasSeriesGuard<P>::value) {
        if (__syncthreads_or(big) && threadIdx.x == 0)
            atomicOr(wide_flags + c, 1);
    }
}

// WIDE selects the slots this launch takes (see takes_candidate); items of the
// other kind are drawn from the queue and skipped.
template <class P, int THREADS, int TILE_BYTES, bool WIDE>
__global__ void __launch_bounds__(THREADS)
    propagate_batch_kernel(const double *__restrict__ A, int ld, const BatchCand *__restrict__ cands,
                           const int2 *__restrict__ work, int nwork, int *__restrict__ counter,
                           const typename P::Entry *__restrict__ table, double dt,
                           double *__restrict__ n_p, double *__restrict__ partial,
                           long long wait_limit, int skip_copies, unsigned int *__restrict__ status,
                           const int *__restrict__ wide_flags)
{
    using V = typename P::Entry;
    constexpr int TILE = TILE_BYTES / (int)sizeof(V);
    __shared__ ItemSmem<P, THREADS, TILE_BYTES> sm;
    __shared__ int s_item;
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    int tile_base = 0;
    for (;;) {
        if (threadIdx.x == 0)
            s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;  // process_item synchronises before s_item is written again
        if (it >= nwork)
            break;
        const int2 w = work[it];
        if (!takes_candidate<P, WIDE>(wide_flags, w.x)) {
            __syncthreads();  // every thread has read s_item before thread 0 draws again
            continue;
        }
        const BatchCand d = cands[w.x];
        const double *Ax = A + (size_t)w.x * 2 * ld;
        const bool ok = process_item<P, THREADS, TILE_BYTES, WIDE>(
            sm, w.y, d.g, d.ns, table + d.table_off, Ax, Ax + ld, dt, n_p ? n_p + d.n_off : nullptr,
            partial + d.part_off, wait_limit, skip_copies, status, tile_base);
        if (!ok)
            break;  // barrier phases are unknown after a wait gave up: this CTA stops
        tile_base += (d.ns + TILE - 1) / TILE;
    }
}

// N[c] from the partial groups of candidate c, in the same fixed order as the
// uniform path.
__global__ void finalize_batch_kernel(const double *__restrict__ partial,
                                      const BatchCand *__restrict__ cands, double *__restrict__ N,
                                      unsigned int *__restrict__ status)
{
    __shared__ double red[256];
    const int c = blockIdx.x;
    const BatchCand d = cands[c];
    double acc = 0.0;
    for (int i = threadIdx.x; i < d.ngroups; i += blockDim.x)
        acc += partial[d.part_off + i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double v = red[0];
        if (!isfinite(v))
            pp_flag(status, PP_FLAG_NONFINITE);
        N[c] = v;
    }
}

constexpr int kNumBatchConfigs = 6;
constexpr int kBCfgThreads[kNumBatchConfigs] = {256, 128, 512, 256, 128, 512};

// Everything a launch needs that depends on the policy and configuration.
struct BatchLaunch {
    const double *A;
    int ld;
    const BatchCand *cands;
    const int2 *work;
    int nwork;
    int *counter;
    void *table;
    int row_quantum;
    int ncand;
    int max_padded;
    double dt;
    double *n_p;
    double *partial;
    double *N;
    int grid_ctas;
};

using BatchFn = int (*)(const BatchLaunch &, cudaStream_t);
using OccFn = int (*)(int *);

template <class P, int THREADS, int TILE_BYTES>
int run_batch(const BatchLaunch &L, cudaStream_t stream)
{
    unsigned int *status = pp::status_word();
    if (!status)
        return pp::fail(PP_ERR_CUDA, "status word unavailable");
    // counter[0], counter[1]: the work counters of the two launches; counter[2 + c]: wide flags
    cudaError_t e = cudaMemsetAsync(L.counter, 0, sizeof(int) * (2 + (size_t)L.ncand), stream);
    if (e != cudaSuccess)
        return pp::cuda_fail(e, "batch work counter reset");
    int *flags = L.counter + 2;
    dim3 tg((L.max_padded + 255) / 256, L.ncand);
    build_table_batch_kernel<P><<<tg, 256, 0, stream>>>(L.A, L.ld, L.cands, L.row_quantum, L.dt,
                                                       (typename P::Entry *)L.table, flags);
    propagate_batch_kernel<P, THREADS, TILE_BYTES, false><<<L.grid_ctas, THREADS, 0, stream>>>(
        L.A, L.ld, L.cands, L.work, L.nwork, L.counter, (const typename P::Entry *)L.table, L.dt,
        L.n_p, L.partial, (long long)pp::wait_limit(), pp::skip_copies(), status, flags);
    if constexpr (HasSeriesGuard<P>::value)
        propagate_batch_kernel<P, THREADS, TILE_BYTES, true><<<L.grid_ctas, THREADS, 0, stream>>>(
            L.A, L.ld, L.cands, L.work, L.nwork, L.counter + 1, (const typename P::Entry *)L.table, L.dt,
            L.n_p, L.partial, (long long)pp::wait_limit(), pp::skip_copies(), status, flags);
    finalize_batch_kernel<<<L.ncand, 256, 0, stream>>>(L.partial, L.cands, L.N, status);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return pp::cuda_fail(e, "batch kernel launch");
    return PP_OK;
}

template <class P, int THREADS, int TILE_BYTES>
int occupancy(int *blocks)
{
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks, propagate_batch_kernel<P, THREADS, TILE_BYTES, false>, THREADS, 0);
    return e == cudaSuccess ? PP_OK : pp::cuda_fail(e, "occupancy query");
}

struct BatchTable {
    BatchFn run[kNumBatchConfigs];
    OccFn occ[kNumBatchConfigs];
    int entry_bytes;
    bool tunable;
    int default_cfg;
};

template <class P>
BatchTable make_batch_table(bool all, int default_cfg)
{
    BatchTable t;
    t.entry_bytes = (int)sizeof(typename P::Entry);
    t.tunable = all;
    t.default_cfg = default_cfg;
    if (all) {
        t.run[0] = &run_batch<P, 256, 8192>;
        t.run[1] = &run_batch<P, 128, 8192>;
        t.run[2] = &run_batch<P, 512, 8192>;
        t.run[3] = &run_batch<P, 256, 32768>;
        t.run[4] = &run_batch<P, 128, 32768>;
        t.run[5] = &run_batch<P, 512, 32768>;
        t.occ[0] = &occupancy<P, 256, 8192>;
        t.occ[1] = &occupancy<P, 128, 8192>;
        t.occ[2] = &occupancy<P, 512, 8192>;
        t.occ[3] = &occupancy<P, 256, 32768>;
        t.occ[4] = &occupancy<P, 128, 32768>;
        t.occ[5] = &occupancy<P, 512, 32768>;
    } else {
        for (int k = 0; k < kNumBatchConfigs; ++k) {
            t.run[k] = &run_batch<P, 256, 8192>;
            t.occ[k] = &occupancy<P, 256, 8192>;
        }
    }
    return t;
}

const BatchTable &batch_table(int precision, int scheme)
{
    static const BatchTable t[3][3] = {
        {make_batch_table<ScalarPolicy<double, false>>(false, 0),
         make_batch_table<MagnusPolicy<double, false>>(false, 0),
         make_batch_table<SplitPolicy<double, false>>(false, 0)},
        {make_batch_table<PackedPolicy<true>>(true, 0), make_batch_table<MagnusPolicy<float, true>>(true, 2),
         make_batch_table<SplitPolicy<float, true>>(true, 0)},
        {make_batch_table<PackedPolicy<false>>(true, 0),
         make_batch_table<MagnusPolicy<float, false>>(true, 0),
         make_batch_table<SplitPolicy<float, false>>(true, 3)},
    };
    return t[precision][scheme];
}

}  // namespace

// ---------------------------------------------------------------- the batch object
struct pp_batch {
    int dev = 0;
    int ncand = 0, precision = 0, scheme = 0;
    int ld = 0, max_ns = 0, max_padded = 0, row_quantum = 1;
    double dt = 0.0;
    int K = 0;
    std::vector<pp_field_spec> specs;
    std::vector<pp_grid> grids;
    std::vector<int> ns;
    long long total_modes = 0;
    int cfg = 0;
    int grid_ctas[kNumBatchConfigs] = {};
    // device buffers, all allocated by pp_batch_create
    BatchCand *d_cands = nullptr;
    int2 *d_work[3] = {nullptr, nullptr, nullptr};  // per CTA size 128, 256, 512
    int nwork[3] = {0, 0, 0};
    int *d_counter = nullptr;
    void *d_table = nullptr;
    double *d_partial = nullptr;
    void *d_synth_desc = nullptr, *d_coef = nullptr;
    int max_M = 0;
    double *d_A = nullptr, *d_trial = nullptr, *d_tfit = nullptr;
    unsigned long long *d_gen = nullptr;
    // captured DE loop
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<char> graph_key;
};

namespace {

int threads_slot(int threads) { return threads == 128 ? 0 : (threads == 256 ? 1 : 2); }

template <typename T>
void key_push(std::vector<char> &k, const T &v)
{
    const char *p = (const char *)&v;
    k.insert(k.end(), p, p + sizeof(T));
}

void batch_free(pp_batch *b)
{
    if (!b)
        return;
    if (b->graph_exec)
        cudaGraphExecDestroy(b->graph_exec);
    if (b->graph)
        cudaGraphDestroy(b->graph);
    void *ptrs[] = {b->d_cands, b->d_work[0], b->d_work[1], b->d_work[2], b->d_counter, b->d_table,
                    b->d_partial, b->d_synth_desc, b->d_coef, b->d_A, b->d_trial, b->d_tfit, b->d_gen};
    for (void *p : ptrs)
        if (p)
            cudaFree(p);
    delete b;
}

BatchLaunch launch_args(const pp_batch *b, const double *A, double *N, double *n_p, int cfg)
{
    const int slot = threads_slot(kBCfgThreads[cfg]);
    BatchLaunch L;
    L.A = A;
    L.ld = b->ld;
    L.cands = b->d_cands;
    L.work = b->d_work[slot];
    L.nwork = b->nwork[slot];
    L.counter = b->d_counter;
    L.table = b->d_table;
    L.row_quantum = b->row_quantum;
    L.ncand = b->ncand;
    L.max_padded = b->max_padded;
    L.dt = b->dt;
    L.n_p = n_p;
    L.partial = b->d_partial;
    L.N = N;
    L.grid_ctas = b->grid_ctas[cfg];
    return L;
}

int batch_pair_number(const pp_batch *b, const double *A, double *N, double *n_p, int cfg,
                      cudaStream_t stream)
{
    return batch_table(b->precision, b->scheme).run[cfg](launch_args(b, A, N, n_p, cfg), stream);
}

int batch_de_generation(pp_batch *b, double *pop, double *fit, const double *lo, const double *hi,
                        const uint8_t *periodic, double F, double CR, uint64_t seed, cudaStream_t st)
{
    const int D = 4 * b->K;
    int rc = pp::launch_de_propose_devgen(pop, b->ncand, D, lo, hi, periodic, F, CR, seed, b->d_gen,
                                          b->d_trial, st);
    if (!rc)
        rc = pp::launch_synth_batch(b->d_trial, b->ncand, &b->specs[0], b->d_synth_desc, b->d_coef,
                                    b->max_M, 2 * b->max_ns + 1, b->ld, b->d_A, st);
    if (!rc)
        rc = batch_pair_number(b, b->d_A, b->d_tfit, nullptr, b->cfg, st);
    if (!rc)
        rc = pp::launch_de_select(pop, fit, b->d_trial, b->d_tfit, b->ncand, D, st);
    if (!rc)
        rc = pp::launch_de_advance(b->d_gen, st);
    return rc;
}

}  // namespace

using namespace pp;

extern "C" {

int pp_batch_create(int32_t ncand, const pp_field_spec *specs, const pp_grid *grids, int32_t precision,
                    int32_t scheme, double dt, pp_batch **out)
{
    clear_error();
    if (!out)
        return fail(PP_ERR_INVALID_ARG, "out must not be NULL");
    *out = nullptr;
    if (ncand < 4 || ncand > 65535 || !specs || !grids)
        return fail(PP_ERR_INVALID_ARG, "need 4 <= ncand <= 65535 and non-NULL specs and grids");
    if (precision != PP_FP64 && precision != PP_FP32 && precision != PP_FP32_FAST)
        return fail(PP_ERR_INVALID_ARG, "precision must be PP_FP64, PP_FP32 or PP_FP32_FAST");
    if (scheme != PP_RK4 && scheme != PP_MAGNUS4 && scheme != PP_SPLIT2)
        return fail(PP_ERR_INVALID_ARG, "scheme must be PP_RK4, PP_MAGNUS4 or PP_SPLIT2");
    if (!(dt > 0.0) || !isfinite(dt))
        return fail(PP_ERR_INVALID_ARG, "dt must be positive and finite");
    for (int c = 0; c < ncand; ++c) {
        const pp_field_spec &s = specs[c];
        if (s.K != specs[0].K || s.order != specs[0].order || s.w_min != specs[0].w_min ||
            s.w_max != specs[0].w_max || s.fluence != specs[0].fluence || s.envelope != specs[0].envelope)
            return fail(PP_ERR_INVALID_ARG, "candidate %d: K, order, band, fluence and envelope must match "
                                            "candidate 0", c);
        if (s.envelope != 0 && s.envelope != 1)
            return fail(PP_ERR_NOT_IMPLEMENTED, "envelope must be 0 (none) or 1 (Hann)");
        if (s.K < s.order || s.K > 64 || s.order < 1 || s.order > 8 || !(s.T > 0.0) || s.n_steps < 1)
            return fail(PP_ERR_INVALID_ARG, "candidate %d: bad pulse model", c);
        if (fabs(s.T / s.n_steps - dt) > 1e-12 * dt)
            return fail(PP_ERR_INVALID_ARG, "candidate %d: T / n_steps must equal dt", c);
        const double dw = 2.0 * M_PI / s.T;
        int j0 = (int)ceil(s.w_min / dw - 1e-12);
        if (j0 < 1)
            j0 = 1;
        const int j1 = (int)floor(s.w_max / dw + 1e-12);
        const int max_modes = s.envelope ? 1534 : 1536;
        if (j1 < j0 || j1 - j0 + 1 > max_modes)
            return fail(PP_ERR_INVALID_ARG, "candidate %d: 1 to %d modes must lie in the band", c, max_modes);
        const pp_grid &g = grids[c];
        if (g.nx < 1 || g.ny < 1 || g.nz < 1 || (long long)g.nx * g.ny * g.nz > (1ll << 30))
            return fail(PP_ERR_INVALID_ARG, "candidate %d: bad grid sizes", c);
        if ((g.nx > 1 && !(g.x1 > g.x0)) || (g.ny > 1 && !(g.y1 > g.y0)) || (g.nz > 1 && !(g.z1 > g.z0)) ||
            (g.mirror_z && g.z0 != 0.0))
            return fail(PP_ERR_INVALID_ARG, "candidate %d: bad grid bounds", c);
    }
    pp_batch *b = new pp_batch();
    cudaGetDevice(&b->dev);
    b->ncand = ncand;
    b->precision = precision;
    b->scheme = scheme;
    b->dt = dt;
    b->K = specs[0].K;
    b->specs.assign(specs, specs + ncand);
    b->grids.assign(grids, grids + ncand);
    b->ns.resize(ncand);
    for (int c = 0; c < ncand; ++c) {
        b->ns[c] = specs[c].n_steps;
        b->max_ns = std::max(b->max_ns, b->ns[c]);
    }
    b->ld = 2 * b->max_ns + 1;
    const BatchTable &tab = batch_table(precision, scheme);
    b->row_quantum = 32768 / tab.entry_bytes;  // the longest tile of any configuration
    b->cfg = tab.default_cfg;

    // candidate descriptors
    std::vector<BatchCand> hc(ncand);
    long long toff = 0, noff = 0, poff = 0;
    for (int c = 0; c < ncand; ++c) {
        const int padded = ((b->ns[c] + b->row_quantum - 1) / b->row_quantum) * b->row_quantum;
        b->max_padded = std::max(b->max_padded, padded);
        const long long nm = (long long)grids[c].nx * grids[c].ny * grids[c].nz;
        hc[c].g = grids[c];
        hc[c].ns = b->ns[c];
        hc[c].ngroups = (int)((nm + kGroup - 1) / kGroup);
        hc[c].table_off = toff;
        hc[c].n_off = noff;
        hc[c].part_off = poff;
        toff += padded;
        noff += nm;
        poff += hc[c].ngroups;
    }
    b->total_modes = noff;
    cudaError_t e = cudaMalloc(&b->d_cands, sizeof(BatchCand) * ncand);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_cands, hc.data(), sizeof(BatchCand) * ncand, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMalloc(&b->d_table, (size_t)toff * tab.entry_bytes);
    if (e == cudaSuccess)
        e = cudaMalloc(&b->d_partial, sizeof(double) * (size_t)poff);
    if (e == cudaSuccess)
        e = cudaMalloc(&b->d_counter, sizeof(int) * (2 + (size_t)ncand));
    // work lists (longest candidates first) for each CTA size
    const int sizes[3] = {128, 256, 512};
    std::vector<int> order(ncand);
    for (int c = 0; c < ncand; ++c)
        order[c] = c;
    std::stable_sort(order.begin(), order.end(), [&](int a, int z) { return b->ns[a] > b->ns[z]; });
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        std::vector<int2> w;
        for (int c : order) {
            const long long nm = (long long)grids[c].nx * grids[c].ny * grids[c].nz;
            const int nb = (int)((nm + sizes[k] - 1) / sizes[k]);
            for (int blk = 0; blk < nb; ++blk)
                w.push_back(make_int2(c, blk));
        }
        b->nwork[k] = (int)w.size();
        e = cudaMalloc(&b->d_work[k], sizeof(int2) * w.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(b->d_work[k], w.data(), sizeof(int2) * w.size(), cudaMemcpyHostToDevice);
    }
    // DE buffers
    if (e == cudaSuccess)
        e = cudaMalloc(&b->d_A, sizeof(double) * 2 * (size_t)b->ld * ncand);
    if (e == cudaSuccess)
        e = cudaMalloc(&b->d_trial, sizeof(double) * 4 * (size_t)b->K * ncand);
    if (e == cudaSuccess)
        e = cudaMalloc(&b->d_tfit, sizeof(double) * ncand);
    if (e == cudaSuccess)
        e = cudaMalloc(&b->d_gen, sizeof(unsigned long long));
    if (e == cudaSuccess)
        e = cudaMemset(b->d_gen, 0, sizeof(unsigned long long));
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_fail(e, "batch allocation");
    }
    int rc = synth_batch_prepare(ncand, specs, &b->d_synth_desc, &b->d_coef, &b->max_M);
    // persistent grid sizes
    int sms = 0;
    if (!rc && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->dev) != cudaSuccess)
        rc = fail(PP_ERR_CUDA, "multiprocessor count");
    for (int k = 0; k < kNumBatchConfigs && !rc; ++k) {
        int blocks = 0;
        rc = tab.occ[k](&blocks);
        const int nwork = b->nwork[threads_slot(kBCfgThreads[k])];
        b->grid_ctas[k] = std::max(1, std::min(nwork, sms * std::max(blocks, 1)));
    }
    if (rc) {
        batch_free(b);
        return rc;
    }
    *out = b;
    return PP_OK;
}

void pp_batch_destroy(pp_batch *b) { batch_free(b); }

int pp_batch_info(const pp_batch *b, int32_t *ld, int64_t *total_modes, int32_t *config)
{
    clear_error();
    if (!b)
        return fail(PP_ERR_INVALID_ARG, "batch is NULL");
    if (ld)
        *ld = b->ld;
    if (total_modes)
        *total_modes = b->total_modes;
    if (config)
        *config = b->cfg;
    return PP_OK;
}

int pp_batch_synth(pp_batch *b, const double *params, double *A, void *stream)
{
    clear_error();
    if (!b || !params || !A)
        return fail(PP_ERR_INVALID_ARG, "batch, params and A must not be NULL");
    return launch_synth_batch(params, b->ncand, &b->specs[0], b->d_synth_desc, b->d_coef, b->max_M,
                              2 * b->max_ns + 1, b->ld, A, (cudaStream_t)stream);
}

int pp_batch_pair_number(pp_batch *b, const double *A, double *N, double *n_p, void *stream)
{
    clear_error();
    if (!b || !A || !N)
        return fail(PP_ERR_INVALID_ARG, "batch, A and N must not be NULL");
    return batch_pair_number(b, A, N, n_p, b->cfg, (cudaStream_t)stream);
}

int pp_batch_tune(pp_batch *b, const double *A, double *N, int32_t *chosen_config, float *config_ms,
                  void *stream)
{
    clear_error();
    if (!b || !A || !N)
        return fail(PP_ERR_INVALID_ARG, "batch, A and N must not be NULL");
    const BatchTable &tab = batch_table(b->precision, b->scheme);
    const int ncfg = tab.tunable ? kNumBatchConfigs : 1;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e1);
    if (e != cudaSuccess)
        return cuda_fail(e, "tuner event");
    int best = tab.default_cfg, rc = PP_OK;
    float best_ms = 3.0e38f;
    for (int k = 0; k < ncfg && !rc; ++k) {
        rc = batch_pair_number(b, A, N, nullptr, k, st);
        if (rc)
            break;
        cudaEventRecord(e0, st);
        rc = batch_pair_number(b, A, N, nullptr, k, st);
        cudaEventRecord(e1, st);
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
    if (b->cfg != best && b->graph_exec) {  // the captured loop used the old configuration
        cudaGraphExecDestroy(b->graph_exec);
        cudaGraphDestroy(b->graph);
        b->graph_exec = nullptr;
        b->graph = nullptr;
        b->graph_key.clear();
    }
    b->cfg = best;
    if (chosen_config)
        *chosen_config = best;
    return PP_OK;
}

int pp_batch_set_generation(pp_batch *b, uint64_t generation, void *stream)
{
    clear_error();
    if (!b)
        return fail(PP_ERR_INVALID_ARG, "batch is NULL");
    return launch_de_set_generation(b->d_gen, generation, (cudaStream_t)stream);
}

int pp_batch_de_step(pp_batch *b, double *pop, double *fit, const double *lo, const double *hi,
                     const uint8_t *periodic, double F, double CR, uint64_t seed, void *stream)
{
    clear_error();
    if (!b || !pop || !fit || !lo || !hi)
        return fail(PP_ERR_INVALID_ARG, "batch, pop, fit, lo, hi must not be NULL");
    if (!(CR >= 0.0 && CR <= 1.0) || !isfinite(F))
        return fail(PP_ERR_INVALID_ARG, "CR must be in [0, 1] and F finite");
    return batch_de_generation(b, pop, fit, lo, hi, periodic, F, CR, seed, (cudaStream_t)stream);
}

int pp_batch_de_run(pp_batch *b, double *pop, double *fit, const double *lo, const double *hi,
                    const uint8_t *periodic, double F, double CR, uint64_t seed, int32_t generations,
                    void *stream)
{
    clear_error();
    if (!b || !pop || !fit || !lo || !hi)
        return fail(PP_ERR_INVALID_ARG, "batch, pop, fit, lo, hi must not be NULL");
    if (!(CR >= 0.0 && CR <= 1.0) || !isfinite(F))
        return fail(PP_ERR_INVALID_ARG, "CR must be in [0, 1] and F finite");
    if (generations < 1 || generations > 100000)
        return fail(PP_ERR_INVALID_ARG, "generations must be in [1, 100000]");
    std::vector<char> key;
    key_push(key, pop);
    key_push(key, fit);
    key_push(key, lo);
    key_push(key, hi);
    key_push(key, periodic);
    key_push(key, F);
    key_push(key, CR);
    key_push(key, seed);
    key_push(key, generations);
    key_push(key, b->cfg);
    if (!b->graph_exec || key != b->graph_key) {
        if (b->graph_exec) {
            cudaGraphExecDestroy(b->graph_exec);
            cudaGraphDestroy(b->graph);
            b->graph_exec = nullptr;
            b->graph = nullptr;
        }
        cudaStream_t cap = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess)
            return cuda_fail(e, "capture stream");
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        int rc = e == cudaSuccess ? PP_OK : cuda_fail(e, "begin capture");
        for (int g = 0; g < generations && !rc; ++g)
            rc = batch_de_generation(b, pop, fit, lo, hi, periodic, F, CR, seed, cap);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cap, &graph);
        if (!rc && e != cudaSuccess)
            rc = cuda_fail(e, "end capture");
        if (!rc) {
            e = cudaGraphInstantiate(&b->graph_exec, graph, 0);
            if (e != cudaSuccess)
                rc = cuda_fail(e, "graph instantiate");
        }
        cudaStreamDestroy(cap);
        if (rc) {
            if (graph)
                cudaGraphDestroy(graph);
            b->graph_exec = nullptr;
            return rc;
        }
        b->graph = graph;
        b->graph_key = key;
    }
    cudaError_t e = cudaGraphLaunch(b->graph_exec, (cudaStream_t)stream);
    return e == cudaSuccess ? PP_OK : cuda_fail(e, "graph launch");
}

}  // extern "C"

// ---------------------------------------------------------------- per-candidate grids
// pp_pair_number with a grid per candidate: one persistent launch of the batch
// kernel over (candidate, block of modes) items, longest first, with the
// descriptors, work list, step tables and partial sums in library scratch.
int pp_pair_number_grids(const double *A, int32_t ncand, int32_t ld, const int32_t *n_steps, double dt,
                         const pp_grid *grids, int32_t n_grids, int32_t precision, int32_t scheme, double *N,
                         double *n_p, void *stream)
{
    clear_error();
    if (n_grids == 1)
        return pp_pair_number(A, ncand, ld, n_steps, dt, grids, precision, scheme, N, n_p, stream);
    if (ncand < 0 || ncand > 65535)
        return fail(PP_ERR_INVALID_ARG, "ncand must be in [0, 65535]");
    if (n_grids != ncand)
        return fail(PP_ERR_INVALID_ARG, "n_grids (%d) must be 1 or ncand (%d)", n_grids, ncand);
    if (ncand == 0)
        return PP_OK;
    if (!A || !N || !grids)
        return fail(PP_ERR_INVALID_ARG, "A, N and grids must not be NULL");
    if (!(dt > 0.0) || !isfinite(dt))
        return fail(PP_ERR_INVALID_ARG, "dt must be positive and finite");
    if (precision != PP_FP64 && precision != PP_FP32 && precision != PP_FP32_FAST)
        return fail(PP_ERR_INVALID_ARG, "precision must be PP_FP64, PP_FP32 or PP_FP32_FAST");
    if (scheme != PP_RK4 && scheme != PP_MAGNUS4 && scheme != PP_SPLIT2)
        return fail(PP_ERR_INVALID_ARG, "scheme must be PP_RK4, PP_MAGNUS4 or PP_SPLIT2");
    if (ld < 3)
        return fail(PP_ERR_INVALID_ARG, "ld must be >= 3");
    for (int c = 0; c < ncand; ++c) {
        if (check_grid(grids + c)) {
            const std::string why = pp_last_error();
            return fail(PP_ERR_INVALID_ARG, "candidate %d: %s", c, why.c_str());
        }
        const long long ns = n_steps ? n_steps[c] : (ld - 1) / 2;
        if (ns < 1 || 2 * ns + 1 > ld)
            return fail(PP_ERR_INVALID_ARG, "candidate %d: n_steps %lld needs 2 n_steps + 1 <= ld (%d)", c, ns, ld);
    }
    const BatchTable &tab = batch_table(precision, scheme);
    const int cfg = tab.default_cfg;
    const int threads = kBCfgThreads[cfg];
    const int row_quantum = 32768 / tab.entry_bytes;
    std::vector<BatchCand> hc(ncand);
    std::vector<int> order(ncand);
    long long toff = 0, noff = 0, poff = 0;
    int max_padded = 0;
    for (int c = 0; c < ncand; ++c) {
        const int ns = n_steps ? n_steps[c] : (ld - 1) / 2;
        const int padded = ((ns + row_quantum - 1) / row_quantum) * row_quantum;
        const long long nm = (long long)grids[c].nx * grids[c].ny * grids[c].nz;
        max_padded = std::max(max_padded, padded);
        hc[c].g = grids[c];
        hc[c].ns = ns;
        hc[c].ngroups = (int)((nm + kGroup - 1) / kGroup);
        hc[c].table_off = toff;
        hc[c].n_off = noff;
        hc[c].part_off = poff;
        toff += padded;
        noff += nm;
        poff += hc[c].ngroups;
        order[c] = c;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int z) { return hc[a].ns > hc[z].ns; });
    std::vector<int2> work;
    for (int c : order) {
        const long long nm = (long long)grids[c].nx * grids[c].ny * grids[c].nz;
        for (int blk = 0; blk < (int)((nm + threads - 1) / threads); ++blk)
            work.push_back(make_int2(c, blk));
    }
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_work = al(sizeof(BatchCand) * ncand);
    const size_t o_table = o_work + al(sizeof(int2) * work.size());
    const size_t o_part = o_table + al((size_t)toff * tab.entry_bytes);
    const size_t o_count = o_part + al(sizeof(double) * (size_t)poff);
    const size_t total = o_count + al(sizeof(int) * (2 + (size_t)ncand));
    void *base = nullptr;
    int rc = scratch(SCR_GRIDS, total, &base);
    if (rc)
        return rc;
    char *b = (char *)base;
    cudaStream_t st = (cudaStream_t)stream;
    // from pageable host memory: each call returns once its source has been staged
    cudaError_t e = cudaMemcpyAsync(b, hc.data(), sizeof(BatchCand) * ncand, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + o_work, work.data(), sizeof(int2) * work.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "grid descriptors");
    int dev = 0, sms = 0, blocks = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fail(PP_ERR_CUDA, "multiprocessor count");
    if ((rc = tab.occ[cfg](&blocks)))
        return rc;
    BatchLaunch L;
    L.A = A;
    L.ld = ld;
    L.cands = (const BatchCand *)b;
    L.work = (const int2 *)(b + o_work);
    L.nwork = (int)work.size();
    L.counter = (int *)(b + o_count);
    L.table = b + o_table;
    L.row_quantum = row_quantum;
    L.ncand = ncand;
    L.max_padded = max_padded;
    L.dt = dt;
    L.n_p = n_p;
    L.partial = (double *)(b + o_part);
    L.N = N;
    L.grid_ctas = std::max(1, std::min((int)work.size(), sms * std::max(blocks, 1)));
    return tab.run[cfg](L, st);
}
