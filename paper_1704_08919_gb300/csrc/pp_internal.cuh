// pp_internal.cuh -- private declarations shared by the libpp translation units
// (status word, scratch, launch helpers, inline-PTX wrappers for mbarriers and
// 1-D bulk copies on sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pp.h"

// ---------------------------------------------------------------- device status word
// Bits set by kernels with atomicOr on the word whose device address
// pp::status_word() returns; collected and cleared by pp_sync_status.
#define PP_FLAG_TIMEOUT 1u
#define PP_FLAG_NONFINITE 2u
#define PP_FLAG_DEGENERATE 4u

__device__ __forceinline__ void pp_flag(unsigned int *status, unsigned int bit) { atomicOr(status, bit); }

// ---------------------------------------------------------------- host helpers
namespace pp {

// Thread-local error message; returns `code` for convenient `return fail(...)`.
int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);
void clear_error();

// Per-device grow-only scratch buffers (slot index -> pointer).  Growth
// synchronises the device, frees the old buffer and allocates a new one.
enum ScratchSlot {
    SCR_TABLE = 0, SCR_PARTIAL, SCR_A, SCR_TRIAL, SCR_TFIT, SCR_COEF,
    SCR_SCREEN_PROPS, SCR_SCREEN_X, SCR_SCREEN_Y, SCR_SCREEN_KEPT,
    SCR_VJP, SCR_QKE_TABLE, SCR_QKE_CKPT, SCR_QKE_PART, SCR_QKE_G, SCR_QKE_FIELD, SCR_QKE_X, SCR_GRIDS, SCR_RATE,
    SCR_NSLOTS
};
int scratch(int slot, size_t bytes, void **ptr);
int release_scratch();  // frees every slot of the current device (after a device synchronisation)

// Argument checks shared by the entry points (pp_capi.cu); they record the message.
int check_grid(const pp_grid *g);
int check_spec(const pp_field_spec *s);

// Device address of the status word of the current device (nullptr on failure).
unsigned int *status_word();

// Kernel-timing hooks around the propagation kernel (no-ops unless profiling).
void profile_mark_start(cudaStream_t stream);
void profile_mark_stop(cudaStream_t stream);

int64_t wait_limit();
int skip_copies();

// Launch the propagation for one precision (pp_propagate.cu).
int launch_pair_number(const double *A, int ncand, int ld, const int32_t *n_steps_host, double dt,
                       const pp_grid *grid, int precision, int scheme, double *N, double *n_p,
                       cudaStream_t stream);

// The same with the fixed static scratch of pp_propagate.cu instead of
// allocated scratch (pp_pair_number_static); static_scratch_bytes() is its size.
int launch_pair_number_static(const double *A, int ncand, int ld, const int32_t *n_steps_host,
                              double dt, const pp_grid *grid, int precision, int scheme, double *N,
                              double *n_p, cudaStream_t stream);
size_t static_scratch_bytes();

// Launch-configuration tuner of the propagation kernel (pp_propagate.cu).
int num_launch_configs();
void launch_config(int k, int *threads, int *tile_bytes);
int tune_pair_number(const double *A, int ncand, int ld, const int32_t *n_steps_host, double dt,
                     const pp_grid *grid, int precision, int scheme, double *N, int32_t *chosen,
                     float *config_ms, cudaStream_t stream);
void clear_tuning();

// Field synthesis launch without argument re-validation (pp_field.cu).
int launch_synth_field(const double *params, int ncand, const pp_field_spec *spec, double *A,
                       int ld, double *E, double *scale, cudaStream_t stream);

// Synthesis with a choice of renormalisation (normalize = 0: s = 1 and `scale`
// receives the fluence) and the time derivative Ed (may be NULL) (pp_field.cu).
int launch_synth(const double *params, int ncand, const pp_field_spec *spec, int normalize, double *A,
                 int ld, double *E, double *Ed, double *scale, cudaStream_t stream);
// Chain rule of the un-normalised synthesis: g[c][6][ldg] = dJ/d(A_x, A_y, E_x, E_y,
// Ed_x, Ed_y samples) -> grad[c][4K] (may be NULL: then g is not read); U[c], dU[c][4K]
// the fluence and its gradient (each may be NULL).
int launch_synth_vjp(const double *params, int ncand, const pp_field_spec *spec, const double *g, int ldg,
                     double *grad, double *U, double *dU, cudaStream_t stream);

// QKE forward and adjoint (pp_qke.cu).
int launch_qke_pair_number(const double *A, const double *E, const double *Ed, int ncand, int ld, int n_steps,
                           double dt, const pp_grid *g, int precision, double *N, double *n_p, cudaStream_t st);
int launch_qke_gradient(const double *A, const double *E, const double *Ed, int ncand, int ld, int n_steps,
                        double dt, const pp_grid *g, int precision, double *J, double *gs, int ldg, cudaStream_t st);

// DE launches (pp_de.cu).
int launch_de_propose(const double *pop, int NP, int D, const double *lo, const double *hi,
                      const uint8_t *periodic, double F, double CR, uint64_t seed, uint64_t gen,
                      double *trial, cudaStream_t stream);
int launch_de_select(double *pop, double *fit, const double *trial, const double *trial_fit,
                     int NP, int D, cudaStream_t stream);
// DE with a device-resident generation counter (captured loops, pp_batch).
int launch_de_propose_devgen(const double *pop, int NP, int D, const double *lo, const double *hi,
                             const uint8_t *periodic, double F, double CR, uint64_t seed,
                             const unsigned long long *gen_dev, double *trial, cudaStream_t stream);
int launch_de_advance(unsigned long long *gen_dev, cudaStream_t stream);
int launch_de_set_generation(unsigned long long *gen_dev, uint64_t v, cudaStream_t stream);

// BF16 tensor-core GEMM and operand packing (pp_gemm.cu).
int launch_gemm_bf16(const void *A, const void *B, float *D, int M, int N, int K, int ldd,
                     cudaStream_t stream);
int launch_pack_bf16(const float *X, int rows, int cols, int ldx, int trans, void *P, int rows_pad,
                     int cols_pad, cudaStream_t stream);

// Batch synthesis (pp_field.cu): per-candidate pulse lengths.
int synth_batch_prepare(int ncand, const pp_field_spec *specs, void **d_desc, void **d_coef,
                        int *max_M);
int launch_synth_batch(const double *params, int ncand, const pp_field_spec *spec0, const void *d_desc,
                       void *d_coef, int max_M, int max_nsamp, int ld, double *A, cudaStream_t stream);

}  // namespace pp

// ---------------------------------------------------------------- inline PTX (sm_90+)
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// Make barrier initialisation visible to the asynchronous (bulk-copy) proxy.
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

// Non-blocking test of phase `parity`; true once that phase has completed.
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: polls at most `limit` times; false if the phase never completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int64_t limit)
{
    for (int64_t it = 0; it < limit; ++it) {
        if (mbar_test_wait(bar, parity))
            return true;
        if (it > 64)
            __nanosleep(32);
    }
    return false;
}

// 1-D bulk copy global -> shared (TMA engine), completion counted on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
