/*
 * pp.h -- C ABI of libpp: GPU scoring of candidate laser pulses by the
 * electron-positron pair number they produce, after
 * F. Fillion-Gourdeau, F. Hebenstreit, D. Gagnon, S. MacLean,
 * "Pulse shape optimization for electron-positron production in rotating
 * fields", arXiv 1704.08919.
 *
 * Units: m = e = c = hbar = 1 (so e*E is written E; E = 1 is the Schwinger field).
 *
 * Conventions shared by every entry point:
 *  - Array arguments marked (device) are caller-owned device pointers in the
 *    current CUDA context; (host) pointers are read before the call returns.
 *    Nothing is retained after a call returns.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  All GPU work
 *    is enqueued on it asynchronously; a PP_OK return means "validated and
 *    launched", not "finished".
 *  - Argument errors are detected on the host before anything is launched and
 *    return PP_ERR_INVALID_ARG; pp_last_error() then describes the problem.
 *  - Errors that only the device can see (a bounded wait that gave up, a
 *    non-finite result, a zero-fluence pulse) are recorded in a device status
 *    word and returned by pp_sync_status().
 *  - The library keeps a private per-device scratch area (the per-step field
 *    table of pp_pair_number, the per-block partial sums, the QKE forward states,
 *    the screening buffers).  It grows on demand with cudaMalloc after a device
 *    synchronisation; call an entry point once with the largest sizes before
 *    capturing it in a CUDA graph.  Because the scratch is per device, work that
 *    uses it must be ordered on one stream per device at a time (two streams
 *    running such calls concurrently would share it).  pp_pair_number_static
 *    uses a fixed device array of its own, also one per device, so the same
 *    ordering applies to it; a pp_batch and a pp_mlp own their buffers.
 *  - Calls are thread-compatible: concurrent calls on different host threads
 *    must use different devices.
 */
#ifndef PP_H
#define PP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PP_OK = 0,
    PP_ERR_INVALID_ARG = 1,      /* bad size, null pointer, bad option: nothing launched */
    PP_ERR_CUDA = 2,             /* a CUDA runtime call failed (message in pp_last_error) */
    PP_ERR_NONFINITE = 3,        /* a NaN or Inf reached N (device-detected) */
    PP_ERR_DEGENERATE_FIELD = 4, /* a candidate had zero fluence and was set to A = 0 */
    PP_ERR_TIMEOUT = 5,          /* a bounded device wait gave up (the kernel returned early) */
    PP_ERR_NOT_IMPLEMENTED = 6
} pp_status;

typedef enum {
    PP_FP64 = 0,     /* FP64 throughout (the parity path) */
    PP_FP32 = 1,     /* FP32 propagation with compensated (two-float) state accumulation;
                        FP64 initial state, projection and momentum sum */
    PP_FP32_FAST = 2 /* as PP_FP32 but with plain FP32 accumulation of the state: about 27%
                        faster; N stays within ~2e-6 of FP64 on the DE-batch workload while
                        single n(p) values lose accuracy (a rounding walk of ~1e-6 in the
                        transition amplitude): n_p is written in this mode but is not accurate
                        mode by mode, and no flag marks it; use PP_FP32 or PP_FP64 where n(p)
                        itself matters */
} pp_precision;
/* Note on the FP32 paths.  A recipe that keeps the time coordinate and the
 * dynamical phase in FP64 has no counterpart here: the propagation runs on two
 * 2-level systems in the lab frame, time is an index into a table of potential
 * samples synthesised in FP64 at exact grid times, and the initial state, the
 * projection and the momentum sum are FP64. */

/* Time integrator of the momentum-space Dirac equation (all on the same grid:
 * step dt, potential samples at t_n, t_n + dt/2, t_n + dt).
 *  PP_RK4     classical fourth-order Runge-Kutta (the integrator of the paper's
 *             kinetic equation, Sec. II.B, applied to the Dirac equation); the
 *             parity path against the CPU oracle.
 *  PP_MAGNUS4 fourth-order Magnus step exp(Omega), Omega = -i dt/6 (H_0 + 4 H_h +
 *             H_1) + dt^2/12 [H_0, H_1]: unitary; the fourth-order scheme the
 *             paper's outlook (Sec. V.C.2) calls for.  On each 2-level system the
 *             step is exp(-i th n.sigma) with th = |dt h_eff|, from even
 *             polynomials in th that hold (to FP32/FP64 rounding) for th <= 0.2:
 *             in FP32 the step is taken as (cos th)^-1 exp(-i th n.sigma) =
 *             1 - i tan th n.sigma (tan th / th one polynomial) and the state's
 *             norm, which then grows, is divided out at the projection (power-of-
 *             two rescaling between tiles keeps it in range exactly); in FP64
 *             cos th - 1 and sin th / th are used.  The step table bounds th per
 *             step over the whole momentum grid (corner momenta and the step's
 *             potential terms); a candidate with any step beyond 0.2 takes, for all
 *             its steps, an argument-halved form instead (th halved k times into
 *             the range, cos th - 1 and sin th / th there, k double-angle steps
 *             back), which is exact for th up to 0.2 * 2^60 and costs about 2k more
 *             instructions per step.  The workloads here stay near th = 0.11-0.14
 *             (dt ~ 0.02, |p| <= 2.5), where only the polynomials run.
 *  PP_SPLIT2  second-order Strang split operator, the paper's own integrator
 *             (Sec. II.A): free part alpha.p + beta (two half steps), coupling
 *             -alpha.A(t_n + dt/2) (one full step), each factor an exact
 *             exponential; unitary. */
typedef enum { PP_RK4 = 0, PP_MAGNUS4 = 1, PP_SPLIT2 = 2 } pp_scheme;

/* Pulse model of Sec. III of the paper.
 *  K        B-spline coefficients per amplitude and per phase and polarisation (N_s).
 *  order    B-spline order k (k = 4: cubic; the paper's tables use k = 3).
 *  w_min, w_max  spectral band [omega_min, omega_max] (angular frequency).
 *  T        pulse length = period 2 pi / dOmega; t runs over [-T/2, T/2].
 *  fluence  U_const of Eq. (energy): every pulse is rescaled to int E^2 dt = U_const.
 *  n_steps  RK4 steps over [-T/2, T/2] (dt = T / n_steps); the potential is
 *           sampled on the half-step grid, 2 n_steps + 1 samples.
 *  envelope 0: g(t) = 1 (DC removed, so A(-T/2) = A(T/2) = 0 with A(-T/2) = 0 as
 *           the gauge); 1: the Hann envelope of Eq. (hann), g(t) = cos^2(pi t / T),
 *           with A of Eq. (vector_potential) in the paper's gauge A(T/2) = 0
 *           (A(-T/2) is then in general not 0) and the fluence of the enveloped
 *           field.  Every entry point that takes a pp_field_spec accepts both;
 *           other values return PP_ERR_NOT_IMPLEMENTED. */
typedef struct {
    int32_t K;
    int32_t order;
    double w_min;
    double w_max;
    double T;
    double fluence;
    int32_t n_steps;
    int32_t envelope;
} pp_field_spec;

/* Uniform momentum grid: nx x ny x nz linspace nodes (end points included) over
 * [x0,x1] x [y0,y1] x [z0,z1].  mirror_z = 1 declares [z0,z1] = [0, zmax] to be
 * the non-negative half of the symmetric window [-zmax, zmax]: the pair density
 * is even in p_z for fields in the x-y plane, and the p_z weights are doubled. */
typedef struct {
    int32_t nx, ny, nz;
    double x0, x1, y0, y1, z0, z1;
    int32_t mirror_z;
} pp_grid;

/* Field synthesis: parameters -> vector potential (Sec. III, Eqs. (coeff_basis_E),
 * (coeff_basis_phi), (field), (energy); renormalisation to U_const at every
 * update, Sec. IV.B).
 *  params (device) [ncand][4K] FP64, per candidate [a^E_x(K), a^phi_x(K), a^E_y(K), a^phi_y(K)].
 *  spec   (host)   pulse model.
 *  A      (device) [ncand][2][ld] FP64 output, row 0 = A_x, row 1 = A_y, sample k at
 *                  t_k = -T/2 + k T / (2 n_steps), k = 0 .. 2 n_steps; ld >= 2 n_steps + 1.
 *  E      (device) same layout for E = -dA/dt, or NULL.
 *  scale  (device) [ncand] the factor s applied to the unit-weight spectrum, or NULL.
 * A zero-fluence candidate produces A = E = 0, s = 0 and sets PP_ERR_DEGENERATE_FIELD
 * in the status word.  Errors: INVALID_ARG (K < order, order < 1 or > 8, K > 64,
 * empty band or more than 1536 modes in it (1534 with the envelope), T <= 0,
 * fluence <= 0, n_steps < 1, ld too small, null A or params). */
int pp_synth_field(const double *params, int32_t ncand, const pp_field_spec *spec, double *A,
                   int32_t ld, double *E, double *scale, void *stream);

/* Pair number of each candidate field (Sec. II.A, Eqs. (kin_mom), (free_spin1),
 * (wf_init), (dirac_eq_mom), (pair_prod_homo); Eq. (opt_prob)).
 * For every momentum p of the grid and both spin states, the momentum-space
 * Dirac equation i d/dt psi = [alpha.(p - A(t)) + beta] psi is integrated with
 * the chosen scheme (step dt; times t_n, t_n + dt/2, t_n + dt take samples
 * 2n, 2n+1, 2n+2 of A) from the negative-energy state at p - A(t_0);
 * f(p) = sum over both spins of the squared projections onto the positive-
 * energy states at p - A(t_end) (the full spin trace); N = sum_p w(p) f(p)
 * with trapezoid weights per axis.
 *  A       (device) [ncand][2][ld] FP64 potential samples as written by pp_synth_field.
 *  n_steps (host)   [ncand] steps per candidate (each 2 n_steps[c] + 1 <= ld), or
 *                   NULL: every candidate takes (ld - 1) / 2 steps.
 *  dt      step size (> 0).
 *  grid    (host)   momentum grid shared by all candidates (a grid per candidate:
 *                   pp_pair_number_grids; with pulse models per candidate as well:
 *                   the pp_batch_* calls).
 *  precision PP_FP64, PP_FP32 or PP_FP32_FAST.
 *  scheme  PP_RK4, PP_MAGNUS4 or PP_SPLIT2.
 *  N       (device) [ncand] FP64 output.
 *  n_p     (device) [ncand][nz][ny][nx] FP64 output (x fastest), or NULL.
 * The sum over p is taken in a fixed order: results are bitwise reproducible
 * run to run.  Errors: INVALID_ARG (sizes, null pointers, dt <= 0, bad precision
 * or scheme). */
int pp_pair_number(const double *A, int32_t ncand, int32_t ld, const int32_t *n_steps, double dt,
                   const pp_grid *grid, int32_t precision, int32_t scheme, double *N, double *n_p,
                   void *stream);

/* Pair numbers with a momentum grid per candidate: pp_pair_number's arguments
 * with grids (host) [n_grids] and n_grids = 1 (one grid shared by all candidates:
 * exactly pp_pair_number) or n_grids = ncand (candidate c on grids[c]).  Per-
 * candidate grids run as one persistent launch of the uneven-batch kernel
 * (pp_batch_pair_number): CTAs take (candidate, block of modes) items, longest
 * candidates first; N[c] is bitwise what pp_pair_number gives for candidate c on
 * its own grid, and n_p (device, or NULL) holds the candidates' n(p) arrays
 * concatenated in candidate order (candidate c's nz*ny*nx values, x fastest).  The
 * descriptors, work list, step tables and partial sums live in library scratch
 * (grown with cudaMalloc on demand); the descriptors are copied from host memory
 * on `stream` in the call.  The launch configuration is the batch kernel's default
 * for the precision and scheme.  Errors: as pp_pair_number, and INVALID_ARG when
 * n_grids is neither 1 nor ncand or a grid is invalid (its index named). */
int pp_pair_number_grids(const double *A, int32_t ncand, int32_t ld, const int32_t *n_steps, double dt,
                         const pp_grid *grids, int32_t n_grids, int32_t precision, int32_t scheme, double *N,
                         double *n_p, void *stream);

/* Launch-configuration tuner of the propagation kernel.  FP32 paths can run the
 * kernel with pp_num_launch_configs() launch configurations (threads per CTA x
 * shared-memory tile length; pp_launch_config describes configuration k); the
 * results do not depend on the configuration (the momentum sum uses fixed
 * groups of 128 modes).  pp_tune_pair_number runs pp_pair_number's work once
 * per configuration (plus one untimed launch each) on the caller's inputs,
 * times it with CUDA events on `stream`, waits for the stream, and records the
 * fastest configuration for this workload shape (precision, scheme, ncand,
 * number of modes, largest n_steps); later pp_pair_number, pp_de_step and
 * pp_pair_number_static calls with that shape use it, others use a built-in
 * default.  N receives the pair numbers of the last run.  config_ms (host,
 * pp_num_launch_configs() floats, or NULL) receives each configuration's time;
 * chosen_config (host, or NULL) the winner.  FP64 paths have one configuration.
 * pp_clear_tuning() forgets every tuned shape.  Errors as pp_pair_number. */
int pp_tune_pair_number(const double *A, int32_t ncand, int32_t ld, const int32_t *n_steps,
                        double dt, const pp_grid *grid, int32_t precision, int32_t scheme,
                        double *N, int32_t *chosen_config, float *config_ms, void *stream);
int pp_num_launch_configs(void);
int pp_launch_config(int32_t k, int32_t *threads_per_cta, int32_t *tile_bytes);
void pp_clear_tuning(void);

/* ---- Uneven batches (candidates with their own pulse length, step count and
 * momentum grid) and captured DE loops.  A pp_batch fixes, per population slot
 * c, the pulse model specs[c] (same K, order, band, fluence and envelope for all slots;
 * T and n_steps per slot with T / n_steps = dt) and the momentum grid grids[c],
 * plus the precision and scheme.  pp_batch_create allocates every device
 * buffer the batch needs (the step table, partial sums, work lists, potential,
 * trial vectors and a device-resident DE generation counter); nothing later
 * allocates, so the DE loop can be captured in a CUDA graph.
 *  pp_batch_synth        params (device [ncand][4K]) -> A (device [ncand][2][ld],
 *                        ld from pp_batch_info; slot c fills 2 n_steps[c] + 1 samples).
 *  pp_batch_pair_number  A -> N (device [ncand]) and n_p (device, the slots'
 *                        n(p) arrays concatenated in slot order, or NULL).  One
 *                        persistent launch: CTAs take (slot, block of modes)
 *                        items, longest slots first, from an atomic counter.
 *                        N[c] is bitwise what pp_pair_number gives for slot c.
 *  pp_batch_tune         times every launch configuration on A, keeps the fastest
 *                        for this batch (waits for the stream).
 *  pp_batch_de_step      one DE generation (propose, synthesise, score, select) on
 *                        pop (device [ncand][4K]) and fit (device [ncand]); the
 *                        generation number comes from the device counter, which
 *                        the step then advances (pp_batch_set_generation sets it).
 *  pp_batch_de_run       `generations` DE generations as one CUDA graph launch on
 *                        `stream`: captured on first use (and again whenever an
 *                        argument or the tuned configuration changes), then
 *                        relaunched; generations continue from the device counter.
 *                        Results are bitwise those of as many pp_batch_de_step calls.
 * Errors: PP_ERR_INVALID_ARG for inconsistent specs, grids or arguments,
 * PP_ERR_CUDA for allocation or capture failures.  A batch belongs to the device
 * that was current at creation; calls on it must not overlap on the GPU. */
typedef struct pp_batch pp_batch;
int pp_batch_create(int32_t ncand, const pp_field_spec *specs, const pp_grid *grids, int32_t precision,
                    int32_t scheme, double dt, pp_batch **out);
void pp_batch_destroy(pp_batch *batch);
int pp_batch_info(const pp_batch *batch, int32_t *ld, int64_t *total_modes, int32_t *config);
int pp_batch_synth(pp_batch *batch, const double *params, double *A, void *stream);
int pp_batch_pair_number(pp_batch *batch, const double *A, double *N, double *n_p, void *stream);
int pp_batch_tune(pp_batch *batch, const double *A, double *N, int32_t *chosen_config,
                  float *config_ms, void *stream);
int pp_batch_set_generation(pp_batch *batch, uint64_t generation, void *stream);
int pp_batch_de_step(pp_batch *batch, double *pop, double *fit, const double *lo, const double *hi,
                     const uint8_t *periodic, double F, double CR, uint64_t seed, void *stream);
int pp_batch_de_run(pp_batch *batch, double *pop, double *fit, const double *lo, const double *hi,
                    const uint8_t *periodic, double F, double CR, uint64_t seed, int32_t generations,
                    void *stream);

/* ---- BF16 tensor-core GEMM (tcgen05, FP32 accumulation in tensor memory): the
 * dense contractions of the surrogate network.  Not in the paper.
 * Operands are BF16 matrices in the packed tile layout: 128-row x 64-column
 * tiles, each a contiguous 16 KiB block of 8 x 8 core matrices (K-major, no
 * swizzle), rows padded to 128 and columns to 64 with zeros;
 * pp_packed_bf16_bytes(rows, cols) is the size of a packed matrix.
 * pp_pack_bf16 packs the FP32 matrix X (rows x cols, row-major with leading
 * dimension ldx; with transpose = 1, X is stored cols x rows and packed
 * transposed) into P (device), rounding to nearest.
 * pp_gemm_bf16 computes D[M][N] = A[M][K] . B[N][K]^T into FP32 D (device,
 * row-major, leading dimension ldd) from packed A (M x K) and B (N x K):
 * M % 128 == 0, 16 <= N <= 256 with N % 16 == 0, K % 64 == 0, ldd >= N.  Columns
 * N .. ldd - 1 of D are not written.  The accumulation order over K is fixed
 * (64-wide chunks in order), so results are reproducible run to run.  Errors:
 * PP_ERR_INVALID_ARG for the shape conditions or NULL pointers; a stalled copy
 * on the device surfaces as PP_ERR_TIMEOUT through pp_sync_status. */
size_t pp_packed_bf16_bytes(int32_t rows, int32_t cols);
int pp_pack_bf16(const float *X, int32_t rows, int32_t cols, int32_t ldx, int32_t transpose, void *P,
                 void *stream);
int pp_gemm_bf16(const void *A, const void *B, float *D, int32_t M, int32_t N, int32_t K, int32_t ldd,
                 void *stream);

/* ---- Surrogate network for screened DE (not in the paper): an MLP
 * d_in -> H -> H -> H -> 1 with GELU activations predicting a normalised log10 N
 * from normalised pulse parameters, trained on the GPU by its own forward and
 * backward kernels (hidden layers on the tensor cores via pp_gemm_bf16; FP32
 * master weights, biases, activations and Adam).  Parameters are one FP32 vector
 * [W1 (H x d_in), b1, W2 (H x H), b2, W3 (H x H), b3, w4 (H), b4].
 *  pp_mlp_create       allocates everything for batches up to max_batch
 *                      (1 <= d_in <= 256, H = 128 or 256: whole 128-row GEMM tiles).
 *  pp_mlp_set_params / pp_mlp_get_params  copy the parameter vector (host or device
 *                      pointer); set_params also resets Adam.
 *  pp_mlp_forward      y (device [B]) for inputs X (device FP32 [B][d_in]).
 *  pp_mlp_loss_grad    loss = mean (y - t)^2 (device float, or NULL) and its
 *                      gradient (device FP32 [n_params], or NULL).
 *  pp_mlp_train_step   one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on that loss.
 *  pp_mlp_features     FP64 parameter vectors (device [B][D]) -> network inputs
 *                      (x - lo) / (hi - lo) - 1/2 as FP32 (device [B][D]). */
typedef struct pp_mlp pp_mlp;
int pp_mlp_create(int32_t d_in, int32_t hidden, int32_t max_batch, pp_mlp **out);
void pp_mlp_destroy(pp_mlp *mlp);
int64_t pp_mlp_num_params(const pp_mlp *mlp);
int pp_mlp_set_params(pp_mlp *mlp, const float *params, void *stream);

/* He initialisation on the device: every weight of a block with fan-in f is
 * sqrt(2/f) z, z a standard normal from the Box-Muller transform of SplitMix64
 * outputs 2i and 2i+1 (i = the parameter's index, generator seeded with seed);
 * biases are zero.  Resets the Adam moments and step count. */
int pp_mlp_init(pp_mlp *mlp, uint64_t seed, void *stream);
int pp_mlp_get_params(const pp_mlp *mlp, float *params, void *stream);
int pp_mlp_forward(pp_mlp *mlp, const float *X, int32_t B, float *y, void *stream);
int pp_mlp_loss_grad(pp_mlp *mlp, const float *X, const float *t, int32_t B, float *loss, float *grad,
                     void *stream);
int pp_mlp_train_step(pp_mlp *mlp, const float *X, const float *t, int32_t B, float lr, float *loss,
                      void *stream);
int pp_mlp_features(const double *params, int32_t B, int32_t D, const double *lo, const double *hi,
                    float *X, void *stream);

/* Mini-batch training: `epochs` passes over the n rows of X (device FP32
 * [n][d_in]) and t (device FP32 [n]), in slices of `batch` rows (the last one
 * ragged), one pp_mlp_train_step per slice, the learning rate following a cosine
 * from lr0 (first step) to lr1 (last step).  epoch_loss (device FP32 [epochs],
 * or NULL) receives the loss of each epoch's last slice.
 * Row order: seed = 0 visits the rows in the order given, every epoch.  Any other
 * seed visits, in epoch e, rows pi_e(0), pi_e(1), ..., pi_e(n - 1), where pi_e is
 * a bijection of [0, n): a 4-round Feistel network on b-bit integers (b the least
 * even number with 2^b >= n, halves of b/2 bits; round i maps (L, R) to
 * (R, L xor (out(k_i, R) mod 2^(b/2))) with k_i = out(seed, 4 e + i), out(s, k) the
 * k-th SplitMix64 output of seed s as in pp_de_propose), applied again while the
 * value is >= n.  The rows of each slice are gathered into buffers of the network;
 * nothing is allocated. */
int pp_mlp_fit(pp_mlp *h, const float *X, const float *t, int32_t n, int32_t batch, int32_t epochs,
               float lr0, float lr1, uint64_t seed, float *epoch_loss, void *stream);

/* Training targets from pair numbers: t[i] = (log10(max(N[i], floor)) - shift)
 * / scale for device FP64 N[n] into device FP32 t[n]; floor > 0, scale != 0. */
int pp_mlp_log_targets(const double *N, int32_t n, double floor_value, double shift, double scale, float *t,
                       void *stream);

/* Screening modes of pp_de_screened_step. */
enum pp_screen_mode {
    PP_SCREEN_PER_INDIVIDUAL = 0, /* each individual's best-predicted proposal */
    PP_SCREEN_GLOBAL = 1          /* the NP best-predicted of all R NP proposals */
};

/* Surrogate-screened DE generation (an extension; the paper's DE scores every
 * trial exactly).  For each individual R DE/rand/1/bin trials are proposed
 * (trial r of generation g uses the counter-RNG key of generation R g + r in
 * pp_de_propose's scheme; proposal k = r NP + i belongs to individual i), the
 * network predicts all R NP of them and NP are kept for exact scoring
 * (pp_synth_field, pp_pair_number), so a generation costs NP exact evaluations
 * as plain DE does:
 *  PP_SCREEN_PER_INDIVIDUAL: row i is individual i's best-predicted proposal
 *    (first maximum); selection as pp_de_select.  With R = 1 this is pp_de_step.
 *  PP_SCREEN_GLOBAL: rows are the NP best-predicted proposals of all R NP in
 *    order (ties to the lower k, NaN predictions last); individual i takes the
 *    exactly best of its kept proposals, if any, when that N >= its fitness.
 * The exact pair number alone decides selection.  trial_out (device [NP][4K]),
 * trial_fit_out (device [NP]), pred_out (device FP32 [R NP]) and kept_out
 * (device int32 [NP], the k of each row) receive the scored trials, their pair
 * numbers, all predictions and the kept indices; each may be NULL.  Needs
 * 4 <= NP <= 65535, 1 <= R <= 64, R NP at most the network's max_batch (rounded
 * up to 128) and a network input size of 4K. */
int pp_de_screened_step(double *pop, double *fit, int32_t NP, const pp_field_spec *spec,
                        const pp_grid *grid, int32_t precision, int32_t scheme, const double *lo,
                        const double *hi, const uint8_t *periodic, double F, double CR, uint64_t seed,
                        uint64_t generation, int32_t R, int32_t mode, pp_mlp *mlp, double *trial_out,
                        double *trial_fit_out, float *pred_out, int32_t *kept_out, void *stream);

/* pp_pair_number without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory --
 * for example a host application whose device memory is fully reserved by its
 * own allocator, or that forbids allocation once it is running, or code called
 * back from another runtime in which a cudaMalloc (with its implicit device
 * synchronisation) is not allowed.  The caller still supplies A, N and n_p.
 * Arguments, results and errors are those of pp_pair_number, computed by the
 * same kernels; the scratch (the per-step field table, the per-block partial
 * sums and, for uneven step counts, a copy of n_steps) lives in a fixed device
 * array of pp_static_scratch_bytes() = 16 MiB inside the library, which every
 * GPU that loads the library holds until the process exits.
 *  - A call whose scratch would exceed that size returns PP_ERR_INVALID_ARG
 *    with the required size in pp_last_error(); it needs about
 *    ncand * (padded n_steps * E + ceil(modes/128) * 8 B), with a table entry
 *    of E = 32 B per step for PP_MAGNUS4 and PP_RK4 in FP32 (16 B for
 *    PP_SPLIT2; twice these in FP64) and n_steps padded to the kernel's tile
 *    (256 to 1024 steps), e.g. 64 candidates of 4096 steps, or 16 candidates
 *    of 16384 steps, with PP_MAGNUS4 in FP32.
 *  - The first call on each device looks up the device address of the array
 *    (a one-time set-up with that device current); make that first call before
 *    any stream capture.
 *  - Every call shares the array and leaves its contents behind; each call
 *    writes all the scratch it reads, so nothing must be cleared, but calls
 *    whose work overlaps on the GPU (other streams, other host threads) race on
 *    it: serialise them.
 *  - Nothing in this call allocates: no cudaMalloc, cudaFree or allocating
 *    library routine.  It calls no kernel-timing hook. */
int pp_pair_number_static(const double *A, int32_t ncand, int32_t ld, const int32_t *n_steps,
                          double dt, const pp_grid *grid, int32_t precision, int32_t scheme,
                          double *N, double *n_p, void *stream);

/* Size in bytes of the fixed scratch array used by pp_pair_number_static. */
size_t pp_static_scratch_bytes(void);

/* DE/rand/1/bin trial vectors (Sec. IV.B, steps 1-3).  For each individual i:
 * three distinct donors r1, r2, r3 != i; u = x_r1 + F (x_r2 - x_r3); binomial
 * crossover with a forced index R.  Coordinates taken from u are wrapped into
 * [lo, hi) where periodic[j] = 1 (phases) and clipped to [lo, hi] elsewhere.
 * Random numbers come from SplitMix64 (Steele, Lea, Flood 2014): the key of
 * individual i in generation `generation` is out(out(seed, generation), i)
 * with out(s, k) the k-th output of the generator seeded with s; slots 0..61
 * of that key serve the donor draws (rejection), slot 62 the index R and slot
 * 64 + j the crossover number of coordinate j.  The result is bit-identical to
 * the sequential definition.
 *  pop (device) [NP][D]; lo, hi (device) [D]; periodic (device) [D] or NULL;
 *  trial (device) [NP][D] output.  NP >= 4, 1 <= D <= 4096, 0 <= CR <= 1. */
int pp_de_propose(const double *pop, int32_t NP, int32_t D, const double *lo, const double *hi,
                  const uint8_t *periodic, double F, double CR, uint64_t seed, uint64_t generation,
                  double *trial, void *stream);

/* Greedy selection for maximisation (Sec. IV.B, step 4): row i of pop and fit[i]
 * are replaced by the trial when trial_fit[i] >= fit[i] (ties go to the trial;
 * a NaN trial never replaces).  All pointers (device). */
int pp_de_select(double *pop, double *fit, const double *trial, const double *trial_fit,
                 int32_t NP, int32_t D, void *stream);

/* One DE generation on the device: propose (pp_de_propose) -> synthesise the
 * trial pulses (pp_synth_field) -> score them (pp_pair_number) -> select
 * (pp_de_select).  pop [NP][4 spec->K] and fit [NP] (device) are updated in
 * place; lo, hi, periodic as in pp_de_propose (device); trial_out (device,
 * [NP][4K]) and trial_fit_out (device, [NP]) receive the scored trials or may
 * be NULL.  The potential buffer and the trials live in library scratch. */
int pp_de_step(double *pop, double *fit, int32_t NP, const pp_field_spec *spec,
               const pp_grid *grid, int32_t precision, int32_t scheme, const double *lo, const double *hi,
               const uint8_t *periodic, double F, double CR, uint64_t seed, uint64_t generation,
               double *trial_out, double *trial_fit_out, void *stream);

/* Waits for `stream`, returns and clears the device status word:
 * PP_OK, PP_ERR_TIMEOUT, PP_ERR_NONFINITE or PP_ERR_DEGENERATE_FIELD (the most
 * severe one seen since the last call), or PP_ERR_CUDA if the wait failed. */
int pp_sync_status(void *stream);

/* Frees the library's scratch on the current device (it only grows otherwise: the
 * QKE adjoint, for instance, keeps up to its state budget, by default half of
 * the device's memory).  Synchronises the
 * device first; the next call that needs scratch allocates it again.  Do not call
 * it while a CUDA graph that uses the scratch may still be launched. */
int pp_release_scratch(void);

/* Test hooks for the bounded device waits (failure detection without a GPU fault).
 * pp_set_wait_limit: iteration limit of every mbarrier wait in the propagation
 *   kernel's main loop (default 1 << 26 polls; 0 restores the default).  Returns
 *   the previous limit.
 * pp_set_skip_copies: when nonzero, the propagation kernel issues none of its
 *   tile copies, so its first wait is on a barrier that nothing completes; the
 *   wait runs out after the limit, the kernel records PP_ERR_TIMEOUT, writes NaN
 *   for the affected candidates and returns.  No copy is ever in flight on that
 *   path.  Returns the previous setting. */
int64_t pp_set_wait_limit(int64_t limit);
int pp_set_skip_copies(int skip);

/* Kernel timing for the propagation kernel (the hot loop of pp_pair_number and
 * pp_de_step).  pp_profile_begin() makes every later launch of that kernel, on
 * the calling host thread's device, bracket itself with a pair of CUDA events
 * recorded on its own stream.  pp_profile_end() waits for the recorded events,
 * writes the summed kernel time in milliseconds and the number of launches, and
 * stops the recording.  Both return PP_OK or PP_ERR_CUDA. */
int pp_profile_begin(void);
int pp_profile_end(double *total_ms, int64_t *launches);

/* The fused multiply-add rate this GPU sustains, in flop/s (2 per FMA), for
 * precision PP_FP64 or PP_FP32 (PP_FP32_FAST is the same): a kernel of eight
 * independent FMA chains per thread and nothing else, a multiple of the SM count
 * in CTAs, timed with CUDA events on `stream` after one untimed launch (about 6 ms
 * for FP64 and 12 ms for FP32 on a GB300): a measured denominator for the
 * roofline fractions of the ALU-bound kernels.  Synchronous: waits for its own
 * events.
 * Errors: PP_ERR_INVALID_ARG (precision, NULL output), PP_ERR_CUDA. */
int pp_fma_rate(int32_t precision, double *flop_per_s, void *stream);

/* Message of the last error on the calling host thread ("" if none). */
const char *pp_last_error(void);

/* Library version, major * 10000 + minor * 100 + patch. */
int pp_version(void);

/* ---- Local search of Sec. IV.A: augmented Lagrangian, BFGS, multistart ----
 * Maximise J subject to C = U_const - U = 0 by minimising
 *   L = -J - lambda C + C^2 / (2 mu)
 * with BFGS (Nocedal & Wright Algorithm 6.1; inverse update Eq. 6.17, first-step
 * scaling Eq. 6.20) and a strong-Wolfe line search (their Algorithms 3.5 and
 * 3.6: c1 = 1e-4, c2 = 0.9, first trial step min(1, 1/|grad L|) on the first
 * iteration of each inner minimisation and 1 after it, doubling while
 * bracketing up to 1e3, 20 bracketing and 30 zoom evaluations, cubic
 * interpolation kept inside the middle 80% of the bracket, else bisection);
 * after each inner minimisation lambda <- lambda - C / mu and mu <- xi mu
 * (steps 2-4), until |C| <= ctol or `outer` inner minimisations have run.
 * BFGS restarts from the identity at every inner minimisation and whenever
 * -H grad L is not a descent direction; updates with y.s <= 0 are skipped. */
typedef struct {
    double mu0;       /* initial penalty parameter, > 0 */
    double xi;        /* penalty factor per outer iteration, 0 < xi < 1 */
    int32_t outer;    /* maximum inner minimisations, >= 1 */
    int32_t max_iter; /* maximum BFGS iterations per inner minimisation */
    double gtol;      /* an inner minimisation stops when max |grad L| <= gtol */
    double ctol;      /* the search stops when |C| <= ctol */
} pp_al_options;

/* Batched objective for pp_al_search: for the `count` host points x[count][n]
 * fill J[count], gJ[count][n], C[count], gC[count][n] (host).  Returns PP_OK or
 * a pp_status code, which ends the search with that code. */
typedef int (*pp_objective_fn)(void *ctx, int32_t count, const double *x, double *J, double *gJ,
                               double *C, double *gC);

/* Multistart augmented-Lagrangian search (step 5) on the host: all nstart
 * starts x[nstart][n] (host, overwritten with the results) advance in lockstep
 * and every round evaluates the pending points of all active starts with one
 * call of fn.  Per start (each may be NULL): J_out, C_out at the result,
 * lam_out the final multiplier, evals_out the objective evaluations,
 * outer_out the inner minimisations run, status_out 0 = |C| <= ctol reached,
 * 1 = `outer` exhausted, 2 = L or its gradient is not finite where an inner
 * minimisation starts (the start ends there).  A non-finite value or slope at
 * a trial step counts as a failed sufficient-decrease test.  Each start's
 * iterates do not depend on the others. */
int pp_al_search(int32_t n, int32_t nstart, double *x, pp_objective_fn fn, void *ctx,
                 const pp_al_options *opt, double *J_out, double *C_out, double *lam_out,
                 int32_t *evals_out, int32_t *outer_out, int32_t *status_out);

/* ---- The 6-component quantum kinetic equation and its adjoint (Sec. II.B,
 * Eqs. (qke), (matrix); Sec. IV.A, Eqs. (eom2), (adj), (grad)) ----
 *
 * pp_synth_field_raw: the field of Eq. (field) (envelope per spec->envelope)
 *   WITHOUT the DE renormalisation (the local search keeps the fluence through its
 *   penalty): A, E and Ed = dE/dt ([ncand][2][ld] device FP64, half-step grid as in
 *   pp_synth_field; E, Ed and U may be NULL); U[c] = the fluence of Eq. (energy)
 *   over one period: (T/2) sum_{l,j} E_{l,j}^2 for g = 1, and for the Hann
 *   envelope (T/2) sum_{l,j>=1} |C'_{l,j}|^2 + T sum_l (C'_{l,0})^2 over the
 *   enveloped harmonics C'.  spec->fluence is not used.
 * pp_synth_vjp: the chain rule of that synthesis (both envelopes).  g
 *   ([ncand][6][ldg] device) holds dJ/d(samples) in the order A_x, A_y, E_x, E_y,
 *   Ed_x, Ed_y; grad ([ncand][4K] device) receives dJ/dparams.  U and dU
 *   ([ncand][4K]) receive the fluence and its gradient.  Each output may be NULL
 *   (g is read only for grad).
 * pp_qke_pair_number: J[c] = sum_p w(p) f(p), f = 1 - chi_1(t_f) by classical
 *   RK4 of the QKE on the half-step grid of (A, E, Ed) ([ncand][2][ld] device),
 *   chi(t_i) = e_1; n_p as in pp_pair_number (may be NULL).  FP64 or FP32 state
 *   (PP_FP32 and PP_FP32_FAST are the same here); J and the sums are FP64.
 * pp_qke_sample_gradient: J[c] and g[c][6][ldg] = dJ/d(every sample of A_x, A_y,
 *   E_x, E_y, Ed_x, Ed_y): the exact derivative of the discrete J, computed by
 *   the adjoint of the RK4 map (adjoint final value lambda_1 = -1 of Eq. (adj)
 *   scaled by w(p), the inner product of Eq. (grad) taken stage by stage).  The
 *   forward states are kept in device scratch for the backward sweep: every
 *   step's state when the states of enough candidates to fill the GPU once fit
 *   within the state budget (pp_set_qke_state_budget, by default half of the
 *   device's memory), else every 4th (FP64) or 8th (FP32) step's, the others
 *   recomputed.  Candidates are processed in chunks whose work buffers fit the
 *   budget (one candidate per chunk at least), sized so that partial waves of
 *   CTAs cost least.  J and g do not depend on either choice.
 * pp_qke_gradient: params -> raw field -> J[c], gJ[c][4K] = dJ/dparams (may be
 *   NULL: J only), U[c] and dU[c][4K] (each may be NULL); all device pointers.
 * pp_local_search: the multistart search of pp_al_search with this objective:
 *   maximise J subject to U = U_const from the host starts x[nstart][4K]
 *   (overwritten with the results); each round evaluates all pending points
 *   of all starts with one pp_qke_gradient call on `stream`.
 * Errors: PP_ERR_INVALID_ARG for bad sizes, pointers or options, PP_ERR_CUDA
 * for a failed launch or allocation; device flags surface through pp_sync_status. */
int pp_synth_field_raw(const double *params, int32_t ncand, const pp_field_spec *spec, double *A, double *E,
                       double *Ed, int32_t ld, double *U, void *stream);
int pp_synth_vjp(const double *params, int32_t ncand, const pp_field_spec *spec, const double *g, int32_t ldg,
                 double *grad, double *U, double *dU, void *stream);
int pp_qke_pair_number(const double *A, const double *E, const double *Ed, int32_t ncand, int32_t ld,
                       int32_t n_steps, double dt, const pp_grid *grid, int32_t precision, double *N, double *n_p,
                       void *stream);
int pp_qke_sample_gradient(const double *A, const double *E, const double *Ed, int32_t ncand, int32_t ld,
                           int32_t n_steps, double dt, const pp_grid *grid, int32_t precision, double *J, double *g,
                           int32_t ldg, void *stream);
int pp_qke_gradient(const double *params, int32_t ncand, const pp_field_spec *spec, const pp_grid *grid,
                    int32_t precision, double *J, double *gJ, double *U, double *dU, void *stream);

/* Device bytes the QKE adjoint (pp_qke_sample_gradient, pp_qke_gradient,
 * pp_local_search) may use for kept forward states and per-CTA partial rows.
 * A negative value selects the default, half of the device's memory; 0 selects
 * the recomputing variant with one candidate per launch.  If the kept states do
 * not fit in free device memory, the adjoint recomputes instead.  The scratch
 * stays allocated until pp_release_scratch.  Host-only setting for every device,
 * read at each call.  Returns the previous setting (-1: the default). */
int64_t pp_set_qke_state_budget(int64_t bytes);
int pp_local_search(double *x, int32_t nstart, const pp_field_spec *spec, const pp_grid *grid, int32_t precision,
                    double U_const, const pp_al_options *opt, double *J_out, double *C_out, double *lam_out,
                    int32_t *evals_out, int32_t *outer_out, int32_t *status_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PP_H */
