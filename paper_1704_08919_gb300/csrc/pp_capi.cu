// pp_capi.cu -- the extern "C" entry points of libpp (declared in include/pp.h):
// host-side validation, error reporting, the device status word, the private
// per-device scratch area and the one-call DE generation.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "pp_internal.cuh"

// The status word: one per device, in this translation unit; other units get
// its device address from pp::status_word() and receive it as a kernel argument.
__device__ unsigned int g_pp_status = 0;

namespace pp {

namespace {
thread_local char t_msg[512] = "";
std::mutex g_mu;
constexpr int kMaxDevices = 64;
void *g_buf[kMaxDevices][SCR_NSLOTS] = {};
size_t g_cap[kMaxDevices][SCR_NSLOTS] = {};
int64_t g_wait_limit = 1ll << 26;
int g_skip_copies = 0;
}  // namespace

int fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_msg, sizeof t_msg, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(PP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void clear_error() { t_msg[0] = 0; }

int scratch(int slot, size_t bytes, void **ptr)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return fail(PP_ERR_CUDA, "device index %d out of range", dev);
    if (bytes == 0)
        bytes = 256;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_cap[dev][slot] < bytes) {
        if (g_buf[dev][slot]) {
            e = cudaDeviceSynchronize();
            if (e != cudaSuccess)
                return cuda_fail(e, "scratch growth sync");
            cudaFree(g_buf[dev][slot]);
            g_buf[dev][slot] = nullptr;
            g_cap[dev][slot] = 0;
        }
        size_t cap = (bytes + 4095) & ~(size_t)4095;
        e = cudaMalloc(&g_buf[dev][slot], cap);
        if (e != cudaSuccess) {
            g_buf[dev][slot] = nullptr;
            return cuda_fail(e, "scratch cudaMalloc");
        }
        g_cap[dev][slot] = cap;
    }
    *ptr = g_buf[dev][slot];
    return PP_OK;
}

int release_scratch()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return fail(PP_ERR_CUDA, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess)
        return cuda_fail(e, "scratch release sync");
    for (int slot = 0; slot < SCR_NSLOTS; ++slot) {
        if (g_buf[dev][slot])
            cudaFree(g_buf[dev][slot]);
        g_buf[dev][slot] = nullptr;
        g_cap[dev][slot] = 0;
    }
    return PP_OK;
}

unsigned int *status_word()
{
    static unsigned int *addr[kMaxDevices] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_pp_status) != cudaSuccess)
            return nullptr;
        addr[dev] = (unsigned int *)p;
    }
    return addr[dev];
}

namespace {
bool g_prof_on = false;
std::vector<cudaEvent_t> g_prof_events;  // start, stop, start, stop, ...
size_t g_prof_used = 0;

cudaEvent_t prof_event()
{
    if (g_prof_used == g_prof_events.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess)
            return nullptr;
        g_prof_events.push_back(e);
    }
    return g_prof_events[g_prof_used++];
}
}  // namespace

void profile_mark_start(cudaStream_t stream)
{
    if (!g_prof_on)
        return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_prof_used % 2 != 0)
        return;
    cudaEvent_t e = prof_event();
    if (e)
        cudaEventRecord(e, stream);
}

void profile_mark_stop(cudaStream_t stream)
{
    if (!g_prof_on)
        return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_prof_used % 2 != 1)
        return;
    cudaEvent_t e = prof_event();
    if (e)
        cudaEventRecord(e, stream);
}

int64_t wait_limit() { return g_wait_limit; }
int skip_copies() { return g_skip_copies; }

int check_grid(const pp_grid *g)
{
    if (!g)
        return fail(PP_ERR_INVALID_ARG, "grid is NULL");
    if (g->nx < 1 || g->ny < 1 || g->nz < 1)
        return fail(PP_ERR_INVALID_ARG, "grid sizes must be >= 1 (got %d x %d x %d)", g->nx, g->ny, g->nz);
    if ((long long)g->nx * g->ny * g->nz > (1ll << 30))
        return fail(PP_ERR_INVALID_ARG, "grid has more than 2^30 modes");
    const double v[6] = {g->x0, g->x1, g->y0, g->y1, g->z0, g->z1};
    for (double x : v)
        if (!isfinite(x))
            return fail(PP_ERR_INVALID_ARG, "grid bounds must be finite");
    if ((g->nx > 1 && !(g->x1 > g->x0)) || (g->ny > 1 && !(g->y1 > g->y0)) ||
        (g->nz > 1 && !(g->z1 > g->z0)))
        return fail(PP_ERR_INVALID_ARG, "grid bounds must be increasing");
    if (g->mirror_z && g->z0 != 0.0)
        return fail(PP_ERR_INVALID_ARG, "mirror_z requires z0 == 0");
    return PP_OK;
}

int check_spec(const pp_field_spec *s)
{
    if (!s)
        return fail(PP_ERR_INVALID_ARG, "field spec is NULL");
    if (s->order < 1 || s->order > 8)
        return fail(PP_ERR_INVALID_ARG, "order must be in [1, 8] (got %d)", s->order);
    if (s->K < s->order || s->K > 64)
        return fail(PP_ERR_INVALID_ARG, "K must be in [order, 64] (got %d)", s->K);
    if (!(s->T > 0.0) || !isfinite(s->T))
        return fail(PP_ERR_INVALID_ARG, "T must be positive");
    if (!(s->fluence > 0.0) || !isfinite(s->fluence))
        return fail(PP_ERR_INVALID_ARG, "fluence must be positive");
    if (!(s->w_max > s->w_min) || !(s->w_min >= 0.0) || !isfinite(s->w_max))
        return fail(PP_ERR_INVALID_ARG, "band must satisfy 0 <= w_min < w_max");
    if (s->n_steps < 1 || s->n_steps > (1 << 28))
        return fail(PP_ERR_INVALID_ARG, "n_steps must be in [1, 2^28]");
    if (s->envelope != 0 && s->envelope != 1)
        return fail(PP_ERR_NOT_IMPLEMENTED, "envelope must be 0 (none) or 1 (Hann)");
    const double dw = 2.0 * M_PI / s->T;
    int j0 = (int)ceil(s->w_min / dw - 1e-12);
    if (j0 < 1)
        j0 = 1;
    const int j1 = (int)floor(s->w_max / dw + 1e-12);
    if (j1 < j0)
        return fail(PP_ERR_INVALID_ARG, "no mode j*2pi/T (j >= 1) lies in [w_min, w_max]");
    // the sample kernels stage 2 (M + 2 with the envelope) coefficients in 48 KB of shared memory
    const int max_modes = s->envelope ? 1534 : 1536;
    if (j1 - j0 + 1 > max_modes)
        return fail(PP_ERR_INVALID_ARG, "more than %d modes in the band", max_modes);
    return PP_OK;
}

}  // namespace pp

using namespace pp;

extern "C" {

const char *pp_last_error(void) { return t_msg; }

int pp_version(void) { return 100; }

int pp_release_scratch(void)
{
    clear_error();
    return release_scratch();
}

int64_t pp_set_wait_limit(int64_t limit)
{
    int64_t old = g_wait_limit;
    g_wait_limit = limit > 0 ? limit : (1ll << 26);
    return old;
}

int pp_set_skip_copies(int skip)
{
    int old = g_skip_copies;
    g_skip_copies = skip ? 1 : 0;
    return old;
}

int pp_profile_begin(void)
{
    clear_error();
    std::lock_guard<std::mutex> lk(g_mu);
    g_prof_used = 0;
    g_prof_on = true;
    return PP_OK;
}

int pp_profile_end(double *total_ms, int64_t *launches)
{
    clear_error();
    std::lock_guard<std::mutex> lk(g_mu);
    g_prof_on = false;
    double tot = 0.0;
    int64_t n = 0;
    for (size_t i = 0; i + 1 < g_prof_used; i += 2) {
        cudaError_t e = cudaEventSynchronize(g_prof_events[i + 1]);
        float ms = 0.0f;
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&ms, g_prof_events[i], g_prof_events[i + 1]);
        if (e != cudaSuccess)
            return cuda_fail(e, "profile event");
        tot += ms;
        ++n;
    }
    g_prof_used = 0;
    if (total_ms)
        *total_ms = tot;
    if (launches)
        *launches = n;
    return PP_OK;
}

int pp_sync_status(void *stream)
{
    clear_error();
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "stream synchronize");
    unsigned int st = 0, zero = 0;
    e = cudaMemcpyFromSymbol(&st, g_pp_status, sizeof st);
    if (e == cudaSuccess)
        e = cudaMemcpyToSymbol(g_pp_status, &zero, sizeof zero);
    if (e != cudaSuccess)
        return cuda_fail(e, "status word read");
    if (st & PP_FLAG_TIMEOUT)
        return fail(PP_ERR_TIMEOUT, "a bounded device wait gave up; affected results are NaN");
    if (st & PP_FLAG_NONFINITE)
        return fail(PP_ERR_NONFINITE, "a non-finite value reached N");
    if (st & PP_FLAG_DEGENERATE)
        return fail(PP_ERR_DEGENERATE_FIELD, "a candidate had zero fluence (its field was set to 0)");
    return PP_OK;
}

int pp_synth_field(const double *params, int32_t ncand, const pp_field_spec *spec, double *A,
                   int32_t ld, double *E, double *scale, void *stream)
{
    clear_error();
    int rc = check_spec(spec);
    if (rc)
        return rc;
    if (ncand < 0)
        return fail(PP_ERR_INVALID_ARG, "ncand must be >= 0");
    if (ncand > 0 && (!params || !A))
        return fail(PP_ERR_INVALID_ARG, "params and A must not be NULL");
    if ((long long)ld < 2ll * spec->n_steps + 1)
        return fail(PP_ERR_INVALID_ARG, "ld (%d) < 2 n_steps + 1 (%d)", ld, 2 * spec->n_steps + 1);
    return launch_synth_field(params, ncand, spec, A, ld, E, scale, (cudaStream_t)stream);
}

int pp_pair_number(const double *A, int32_t ncand, int32_t ld, const int32_t *n_steps, double dt,
                   const pp_grid *grid, int32_t precision, int32_t scheme, double *N, double *n_p,
                   void *stream)
{
    clear_error();
    int rc = check_grid(grid);
    if (rc)
        return rc;
    if (ncand < 0 || ncand > 65535)
        return fail(PP_ERR_INVALID_ARG, "ncand must be in [0, 65535]");
    if (ncand == 0)
        return PP_OK;
    if (!A || !N)
        return fail(PP_ERR_INVALID_ARG, "A and N must not be NULL");
    if (!(dt > 0.0) || !isfinite(dt))
        return fail(PP_ERR_INVALID_ARG, "dt must be positive and finite");
    if (precision != PP_FP64 && precision != PP_FP32 && precision != PP_FP32_FAST)
        return fail(PP_ERR_INVALID_ARG, "precision must be PP_FP64, PP_FP32 or PP_FP32_FAST");
    if (scheme != PP_RK4 && scheme != PP_MAGNUS4 && scheme != PP_SPLIT2)
        return fail(PP_ERR_INVALID_ARG, "scheme must be PP_RK4, PP_MAGNUS4 or PP_SPLIT2");
    if (ld < 3)
        return fail(PP_ERR_INVALID_ARG, "ld must be >= 3");
    for (int c = 0; c < ncand; ++c) {
        long long ns = n_steps ? n_steps[c] : (ld - 1) / 2;
        if (ns < 1 || 2 * ns + 1 > ld)
            return fail(PP_ERR_INVALID_ARG, "candidate %d: n_steps %lld needs 2 n_steps + 1 <= ld (%d)", c, ns, ld);
    }
    return launch_pair_number(A, ncand, ld, n_steps, dt, grid, precision, scheme, N, n_p,
                              (cudaStream_t)stream);
}

int pp_pair_number_static(const double *A, int32_t ncand, int32_t ld, const int32_t *n_steps,
                          double dt, const pp_grid *grid, int32_t precision, int32_t scheme,
                          double *N, double *n_p, void *stream)
{
    clear_error();
    int rc = check_grid(grid);
    if (rc)
        return rc;
    if (ncand < 0 || ncand > 65535)
        return fail(PP_ERR_INVALID_ARG, "ncand must be in [0, 65535]");
    if (ncand == 0)
        return PP_OK;
    if (!A || !N)
        return fail(PP_ERR_INVALID_ARG, "A and N must not be NULL");
    if (!(dt > 0.0) || !isfinite(dt))
        return fail(PP_ERR_INVALID_ARG, "dt must be positive and finite");
    if (precision != PP_FP64 && precision != PP_FP32 && precision != PP_FP32_FAST)
        return fail(PP_ERR_INVALID_ARG, "precision must be PP_FP64, PP_FP32 or PP_FP32_FAST");
    if (scheme != PP_RK4 && scheme != PP_MAGNUS4 && scheme != PP_SPLIT2)
        return fail(PP_ERR_INVALID_ARG, "scheme must be PP_RK4, PP_MAGNUS4 or PP_SPLIT2");
    if (ld < 3)
        return fail(PP_ERR_INVALID_ARG, "ld must be >= 3");
    for (int c = 0; c < ncand; ++c) {
        long long ns = n_steps ? n_steps[c] : (ld - 1) / 2;
        if (ns < 1 || 2 * ns + 1 > ld)
            return fail(PP_ERR_INVALID_ARG, "candidate %d: n_steps %lld needs 2 n_steps + 1 <= ld (%d)", c, ns, ld);
    }
    return launch_pair_number_static(A, ncand, ld, n_steps, dt, grid, precision, scheme, N, n_p,
                                     (cudaStream_t)stream);
}

size_t pp_static_scratch_bytes(void) { return static_scratch_bytes(); }

int pp_tune_pair_number(const double *A, int32_t ncand, int32_t ld, const int32_t *n_steps,
                        double dt, const pp_grid *grid, int32_t precision, int32_t scheme,
                        double *N, int32_t *chosen_config, float *config_ms, void *stream)
{
    clear_error();
    int rc = check_grid(grid);
    if (rc)
        return rc;
    if (ncand < 1 || ncand > 65535)
        return fail(PP_ERR_INVALID_ARG, "ncand must be in [1, 65535]");
    if (!A || !N)
        return fail(PP_ERR_INVALID_ARG, "A and N must not be NULL");
    if (!(dt > 0.0) || !isfinite(dt))
        return fail(PP_ERR_INVALID_ARG, "dt must be positive and finite");
    if (precision != PP_FP64 && precision != PP_FP32 && precision != PP_FP32_FAST)
        return fail(PP_ERR_INVALID_ARG, "precision must be PP_FP64, PP_FP32 or PP_FP32_FAST");
    if (scheme != PP_RK4 && scheme != PP_MAGNUS4 && scheme != PP_SPLIT2)
        return fail(PP_ERR_INVALID_ARG, "scheme must be PP_RK4, PP_MAGNUS4 or PP_SPLIT2");
    if (ld < 3)
        return fail(PP_ERR_INVALID_ARG, "ld must be >= 3");
    for (int c = 0; c < ncand; ++c) {
        long long ns = n_steps ? n_steps[c] : (ld - 1) / 2;
        if (ns < 1 || 2 * ns + 1 > ld)
            return fail(PP_ERR_INVALID_ARG, "candidate %d: n_steps %lld needs 2 n_steps + 1 <= ld (%d)", c, ns, ld);
    }
    return tune_pair_number(A, ncand, ld, n_steps, dt, grid, precision, scheme, N, chosen_config,
                            config_ms, (cudaStream_t)stream);
}

int pp_num_launch_configs(void) { return num_launch_configs(); }

size_t pp_packed_bf16_bytes(int32_t rows, int32_t cols)
{
    if (rows < 1 || cols < 1)
        return 0;
    const size_t r = ((size_t)rows + 127) / 128 * 128, c = ((size_t)cols + 63) / 64 * 64;
    return r * c * 2;
}

int pp_pack_bf16(const float *X, int32_t rows, int32_t cols, int32_t ldx, int32_t transpose, void *P,
                 void *stream)
{
    clear_error();
    if (!X || !P || rows < 1 || cols < 1)
        return fail(PP_ERR_INVALID_ARG, "X and P must not be NULL; rows, cols >= 1");
    const int src_cols = transpose ? rows : cols;
    if (ldx < src_cols)
        return fail(PP_ERR_INVALID_ARG, "ldx smaller than the stored row length");
    const int rp = (rows + 127) / 128 * 128, cp = (cols + 63) / 64 * 64;
    return launch_pack_bf16(X, rows, cols, ldx, transpose ? 1 : 0, P, rp, cp, (cudaStream_t)stream);
}

int pp_gemm_bf16(const void *A, const void *B, float *D, int32_t M, int32_t N, int32_t K, int32_t ldd,
                 void *stream)
{
    clear_error();
    if (!A || !B || !D)
        return fail(PP_ERR_INVALID_ARG, "A, B and D must not be NULL");
    if (M < 128 || M % 128 || N < 16 || N > 256 || N % 16 || K < 64 || K % 64 || ldd < N)
        return fail(PP_ERR_INVALID_ARG, "need M %% 128 == 0, 16 <= N <= 256 with N %% 16 == 0, "
                                        "K %% 64 == 0 and ldd >= N (got M=%d N=%d K=%d ldd=%d)",
                    M, N, K, ldd);
    return launch_gemm_bf16(A, B, D, M, N, K, ldd, (cudaStream_t)stream);
}

int pp_launch_config(int32_t k, int32_t *threads_per_cta, int32_t *tile_bytes)
{
    clear_error();
    if (k < 0 || k >= num_launch_configs() || !threads_per_cta || !tile_bytes)
        return fail(PP_ERR_INVALID_ARG, "configuration index out of range or NULL output");
    int t = 0, b = 0;
    launch_config(k, &t, &b);
    *threads_per_cta = t;
    *tile_bytes = b;
    return PP_OK;
}

void pp_clear_tuning(void) { clear_tuning(); }

int pp_de_propose(const double *pop, int32_t NP, int32_t D, const double *lo, const double *hi,
                  const uint8_t *periodic, double F, double CR, uint64_t seed, uint64_t generation,
                  double *trial, void *stream)
{
    clear_error();
    if (NP < 4)
        return fail(PP_ERR_INVALID_ARG, "DE needs NP >= 4 (got %d)", NP);
    if (D < 1 || D > 4096)
        return fail(PP_ERR_INVALID_ARG, "D must be in [1, 4096]");
    if (!pop || !lo || !hi || !trial)
        return fail(PP_ERR_INVALID_ARG, "pop, lo, hi and trial must not be NULL");
    if (!(CR >= 0.0 && CR <= 1.0) || !isfinite(F))
        return fail(PP_ERR_INVALID_ARG, "CR must be in [0, 1] and F finite");
    return launch_de_propose(pop, NP, D, lo, hi, periodic, F, CR, seed, generation, trial,
                             (cudaStream_t)stream);
}

int pp_de_select(double *pop, double *fit, const double *trial, const double *trial_fit, int32_t NP,
                 int32_t D, void *stream)
{
    clear_error();
    if (NP < 1 || D < 1)
        return fail(PP_ERR_INVALID_ARG, "NP and D must be >= 1");
    if (!pop || !fit || !trial || !trial_fit)
        return fail(PP_ERR_INVALID_ARG, "pointers must not be NULL");
    return launch_de_select(pop, fit, trial, trial_fit, NP, D, (cudaStream_t)stream);
}

int pp_de_step(double *pop, double *fit, int32_t NP, const pp_field_spec *spec, const pp_grid *grid,
               int32_t precision, int32_t scheme, const double *lo, const double *hi, const uint8_t *periodic,
               double F, double CR, uint64_t seed, uint64_t generation, double *trial_out,
               double *trial_fit_out, void *stream)
{
    clear_error();
    int rc = check_spec(spec);
    if (!rc)
        rc = check_grid(grid);
    if (rc)
        return rc;
    if (NP < 4 || NP > 65535)
        return fail(PP_ERR_INVALID_ARG, "NP must be in [4, 65535]");
    if (!pop || !fit || !lo || !hi)
        return fail(PP_ERR_INVALID_ARG, "pop, fit, lo, hi must not be NULL");
    if (precision != PP_FP64 && precision != PP_FP32 && precision != PP_FP32_FAST)
        return fail(PP_ERR_INVALID_ARG, "precision must be PP_FP64, PP_FP32 or PP_FP32_FAST");
    if (scheme != PP_RK4 && scheme != PP_MAGNUS4 && scheme != PP_SPLIT2)
        return fail(PP_ERR_INVALID_ARG, "scheme must be PP_RK4, PP_MAGNUS4 or PP_SPLIT2");
    if (!(CR >= 0.0 && CR <= 1.0) || !isfinite(F))
        return fail(PP_ERR_INVALID_ARG, "CR must be in [0, 1] and F finite");
    cudaStream_t st = (cudaStream_t)stream;
    const int D = 4 * spec->K;
    const int ld = 2 * spec->n_steps + 1;
    double *trial = trial_out, *tfit = trial_fit_out, *A = nullptr;
    void *p = nullptr;
    if (!trial) {
        if ((rc = scratch(SCR_TRIAL, (size_t)NP * D * sizeof(double), &p)))
            return rc;
        trial = (double *)p;
    }
    if (!tfit) {
        if ((rc = scratch(SCR_TFIT, (size_t)NP * sizeof(double), &p)))
            return rc;
        tfit = (double *)p;
    }
    if ((rc = scratch(SCR_A, (size_t)NP * 2 * ld * sizeof(double), &p)))
        return rc;
    A = (double *)p;
    if ((rc = launch_de_propose(pop, NP, D, lo, hi, periodic, F, CR, seed, generation, trial, st)))
        return rc;
    if ((rc = launch_synth_field(trial, NP, spec, A, ld, nullptr, nullptr, st)))
        return rc;
    if ((rc = launch_pair_number(A, NP, ld, nullptr, spec->T / spec->n_steps, grid, precision, scheme,
                                 tfit, nullptr, st)))
        return rc;
    return launch_de_select(pop, fit, trial, tfit, NP, D, st);
}

}  // extern "C"
