// pp_de.cu -- DE/rand/1/bin on the device (Sec. IV.B of arXiv 1704.08919,
// steps 1-4), with counter-based SplitMix64 random numbers so that every
// individual's draws are independent of launch shape and bit-identical to the
// sequential definition.
#include <math.h>

#include "pp_internal.cuh"

namespace {

// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the k-th output (k = 0, 1, ...)
// of the generator seeded with s is mix(s + (k + 1) * golden_gamma).
__device__ __forceinline__ uint64_t sm64_at(uint64_t s, uint64_t k)
{
    uint64_t z = s + (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

constexpr int kSlotR = 62;      // forced crossover index R
constexpr int kSlotCross = 64;  // + j: crossover number of coordinate j
constexpr int kMaxDraws = 62;   // donor rejection draws use slots 0..61

__device__ __forceinline__ double u01(uint64_t x) { return (double)(x >> 11) * 0x1.0p-53; }

__device__ __forceinline__ int below(uint64_t x, int n)
{
    return (int)(((x >> 32) * (uint64_t)n) >> 32);
}

// One block per individual: thread 0 draws the donors and R, all threads build
// the trial coordinates.  Floating-point steps use explicit round-to-nearest
// intrinsics so that no multiply-add is contracted.
__global__ void de_propose_kernel(const double *__restrict__ pop, int NP, int D,
                                  const double *__restrict__ lo, const double *__restrict__ hi,
                                  const uint8_t *__restrict__ periodic, double F, double CR,
                                  uint64_t seed, uint64_t gen, double *__restrict__ trial,
                                  const unsigned long long *__restrict__ gen_dev)
{
    __shared__ int sr[4];  // r1, r2, r3, R (r1 = -1 on failure)
    const int i = blockIdx.x;
    if (gen_dev)
        gen = *gen_dev;
    const uint64_t key = sm64_at(sm64_at(seed, gen), (uint64_t)i);
    if (threadIdx.x == 0) {
        int r[3] = {-1, -1, -1};
        int slot = 0;
        bool okall = true;
        for (int q = 0; q < 3 && okall; ++q) {
            bool found = false;
            while (slot < kMaxDraws) {
                int cand = below(sm64_at(key, (uint64_t)slot++), NP);
                bool clash = (cand == i);
                for (int z = 0; z < q; ++z)
                    clash |= (cand == r[z]);
                if (!clash) {
                    r[q] = cand;
                    found = true;
                    break;
                }
            }
            okall = found;
        }
        sr[0] = okall ? r[0] : -1;
        sr[1] = r[1];
        sr[2] = r[2];
        sr[3] = below(sm64_at(key, kSlotR), D);
    }
    __syncthreads();
    const int r1 = sr[0], r2 = sr[1], r3 = sr[2], R = sr[3];
    double *y = trial + (size_t)i * D;
    const double *xi = pop + (size_t)i * D;
    if (r1 < 0) {  // rejection ran out of slots (probability < 1e-30): keep the parent
        for (int j = threadIdx.x; j < D; j += blockDim.x)
            y[j] = xi[j];
        return;
    }
    const double *xa = pop + (size_t)r1 * D, *xb = pop + (size_t)r2 * D, *xc = pop + (size_t)r3 * D;
    for (int j = threadIdx.x; j < D; j += blockDim.x) {
        const double rj = u01(sm64_at(key, (uint64_t)(kSlotCross + j)));
        if (rj <= CR || j == R) {
            double u = __dadd_rn(xa[j], __dmul_rn(F, __dsub_rn(xb[j], xc[j])));
            if (periodic && periodic[j]) {
                const double period = __dsub_rn(hi[j], lo[j]);
                double off = fmod(__dsub_rn(u, lo[j]), period);
                if (off < 0.0)
                    off = __dadd_rn(off, period);
                u = __dadd_rn(lo[j], off);
                if (u >= hi[j])
                    u = lo[j];
            } else {
                u = u < lo[j] ? lo[j] : u;
                u = u > hi[j] ? hi[j] : u;
            }
            y[j] = u;
        } else {
            y[j] = xi[j];
        }
    }
}

// Advances a device-resident generation counter (used by captured DE loops).
__global__ void de_advance_kernel(unsigned long long *gen_dev)
{
    if (threadIdx.x == 0 && blockIdx.x == 0)
        *gen_dev += 1ull;
}

__global__ void de_set_generation_kernel(unsigned long long *gen_dev, unsigned long long v)
{
    if (threadIdx.x == 0 && blockIdx.x == 0)
        *gen_dev = v;
}

// One block per individual; the decision is read before any write.
__global__ void de_select_kernel(double *__restrict__ pop, double *__restrict__ fit,
                                 const double *__restrict__ trial, const double *__restrict__ tfit,
                                 int D)
{
    const int i = blockIdx.x;
    const bool take = tfit[i] >= fit[i];
    __syncthreads();
    if (!take)
        return;
    for (int j = threadIdx.x; j < D; j += blockDim.x)
        pop[(size_t)i * D + j] = trial[(size_t)i * D + j];
    if (threadIdx.x == 0)
        fit[i] = tfit[i];
}

}  // namespace

namespace pp {

int launch_de_propose(const double *pop, int NP, int D, const double *lo, const double *hi,
                      const uint8_t *periodic, double F, double CR, uint64_t seed, uint64_t gen,
                      double *trial, cudaStream_t stream)
{
    de_propose_kernel<<<NP, 64, 0, stream>>>(pop, NP, D, lo, hi, periodic, F, CR, seed, gen, trial,
                                             nullptr);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PP_OK : cuda_fail(e, "DE propose launch");
}

int launch_de_propose_devgen(const double *pop, int NP, int D, const double *lo, const double *hi,
                             const uint8_t *periodic, double F, double CR, uint64_t seed,
                             const unsigned long long *gen_dev, double *trial, cudaStream_t stream)
{
    de_propose_kernel<<<NP, 64, 0, stream>>>(pop, NP, D, lo, hi, periodic, F, CR, seed, 0, trial,
                                             gen_dev);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PP_OK : cuda_fail(e, "DE propose launch");
}

int launch_de_advance(unsigned long long *gen_dev, cudaStream_t stream)
{
    de_advance_kernel<<<1, 32, 0, stream>>>(gen_dev);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PP_OK : cuda_fail(e, "DE generation advance");
}

int launch_de_set_generation(unsigned long long *gen_dev, uint64_t v, cudaStream_t stream)
{
    de_set_generation_kernel<<<1, 32, 0, stream>>>(gen_dev, v);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PP_OK : cuda_fail(e, "DE generation set");
}

int launch_de_select(double *pop, double *fit, const double *trial, const double *trial_fit, int NP,
                     int D, cudaStream_t stream)
{
    de_select_kernel<<<NP, 64, 0, stream>>>(pop, fit, trial, trial_fit, D);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PP_OK : cuda_fail(e, "DE select launch");
}

}  // namespace pp
