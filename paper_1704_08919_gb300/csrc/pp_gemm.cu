// pp_gemm.cu -- BF16 GEMM on the fifth-generation tensor cores (tcgen05, TMEM),
// FP32 accumulation: the dense contractions of the surrogate network.
//
//   D[M][N] (FP32, row-major, leading dimension ldd) = A[M][K] . B[N][K]^T
//
// Operands live in global memory in a packed BF16 layout: tiles of 128 rows x
// 64 columns, each stored contiguously as 16 row groups x 8 column groups of
// 8 x 8 "core matrices" (one core matrix = 8 rows of 16 bytes), which is the
// K-major layout without swizzle that tcgen05.mma reads from shared memory.  A
// tile is therefore one 16 KiB block and reaches shared memory with a single
// 1-D bulk copy.  Element (r, c) of a packed R x C matrix (R, C padded to 128 and
// 64) sits at byte
//   ((r / 128) * (C / 64) + c / 64) * 16384 + ((r % 128) / 8) * 1024
//     + ((c % 64) / 8) * 128 + (r % 8) * 16 + (c % 8) * 2.
// In shared memory the core matrices adjacent along K are 128 B apart (the
// descriptor's leading-dimension offset) and the row groups 1024 B apart (its
// stride offset).
//
// Persistent, warp-specialised kernel: one CTA per SM (at most one per 128-row
// tile of D) walks the tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...; each tile
// is the full width of D (N <= 256), so every A tile crosses from L2 once.
//   warp 0      producer: lane 0 streams the A tile and the one or two B tiles of
//               every 64-wide K chunk into a ring with bulk copies; when all of B
//               fits in 128 KiB (K <= 512, or K <= 256 for N > 128) it loads B once
//               per CTA and the ring carries A alone;
//   warp 1      owns TMEM (two 256-column FP32 accumulators) and issues: lane 0
//               issues 4 MMAs (K = 16 each) per chunk into the accumulator of the
//               tile, commits each stage back to the producer and each finished
//               tile to the epilogue;
//   warps 2..9  epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (the quadrant
//               tcgen05.ld allows it) over one half of the columns, stages 32 x 32
//               blocks through shared memory and writes whole row segments of D,
//               then hands the accumulator back, so the next tile's MMAs overlap
//               this tile's stores.
// Every wait is bounded; a wait that gives up records PP_ERR_TIMEOUT, and the
// issuing lanes wait (bounded) for their copies and MMAs in flight before TMEM is
// freed.
#include <cuda_bf16.h>
#include <stdint.h>

#include "pp_internal.cuh"

namespace {

constexpr int kBM = 128;        // rows per CTA (MMA M)
constexpr int kKC = 64;         // K per chunk
constexpr int kTileBytes = kBM * kKC * 2;  // one packed 128 x 64 tile

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);            // start address
    d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;         // leading byte offset: next core matrix along K
    d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;        // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                               // descriptor version for sm_100 family
    return d;                                             // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: D F32, A and B BF16, both K-major, M x N.
__device__ __forceinline__ uint32_t instr_desc(int M, int N)
{
    uint32_t d = 0;
    d |= 1u << 4;                      // D format: F32
    d |= 1u << 7;                      // A format: BF16
    d |= 1u << 10;                     // B format: BF16
    d |= (uint32_t)(N >> 3) << 17;     // N / 8
    d |= (uint32_t)(M >> 4) << 24;     // M / 16
    return d;
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i)
        v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
                 : "memory");
}

constexpr int kBN = 256;                      // D columns per tile (all of N)
constexpr int kEpiWarps = 8;                  // two per TMEM lane quadrant, one per column half
constexpr int kEpiPitch = 33;                 // floats per staged row: conflict-free columns and rows
constexpr int kEpiBytes = kEpiWarps * 32 * kEpiPitch * 4;
constexpr int kBarBytes = 256;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr uint32_t kTmemCols = 2 * kBN;       // double-buffered accumulator
constexpr int kMaxResidentB = 8;              // B tiles kept resident (128 KiB): K <= 512, or K <= 256 for N > 128

// Shared-memory plan, one CTA per SM.  Streaming B (RB = false): a ring of 4 stages x
// (A tile + two B tiles, 48 KiB).  Resident B (RB = true, when all of B fits): the B
// tiles of every chunk, loaded once per CTA, then a ring of 4 A tiles.  Both: the
// epilogue's staging blocks and the barriers.
template <bool RB>
struct GemmPlan {
    static constexpr int stages = 4;
    static constexpr int stage_bytes = RB ? kTileBytes : 3 * kTileBytes;
    static constexpr int ring_off = RB ? kMaxResidentB * kTileBytes : 0;
    static constexpr int epi_off = ring_off + stages * stage_bytes;
    static constexpr int bar_off = epi_off + kEpiBytes;
    static constexpr int smem_bytes = bar_off + kBarBytes + 1024;
    static_assert(smem_bytes <= 232448, "shared memory per CTA");
};

template <bool RB>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_bf16_kernel(const uint8_t *__restrict__ A, const uint8_t *__restrict__ B, float *__restrict__ D,
                     int M, int N, int K, int ldd, long long wait_limit, unsigned int *__restrict__ status,
                     int skip_copies)
{
    using Plan = GemmPlan<RB>;
    constexpr int kStages = Plan::stages;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *bres = smem;                           // resident B: chunk ch's tiles at ch * nb tiles
    uint8_t *ring = smem + Plan::ring_off;
    float *stage_all = (float *)(smem + Plan::epi_off);
    uint64_t *full = (uint64_t *)(smem + Plan::bar_off);  // [kStages] copies landed
    uint64_t *empty = full + kStages;                     // [kStages] stage's MMAs done
    uint64_t *tfull = empty + kStages;                    // [2] accumulator complete
    uint64_t *tempty = tfull + 2;                         // [2] accumulator read out
    uint64_t *bfull = tempty + 2;                         // resident B landed
    uint32_t *s_taddr = (uint32_t *)(bfull + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = M / kBM, nchunks = K / kKC;
    const int nb = N > 128 ? 2 : 1;  // packed B row tiles per chunk
    const uint32_t stage_tx = (uint32_t)(RB ? 1 : 1 + nb) * kTileBytes;

    if (warp == 1)
        tmem_alloc(s_taddr, kTmemCols);
    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&tfull[i], 1);
            mbar_init(&tempty[i], kEpiWarps);
        }
        mbar_init(bfull, 1);
        mbar_fence_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *s_taddr;

    bool ok = true;
    // drain bookkeeping of the issuing lanes: chunks copied, chunks committed and tiles
    // committed, each in ring order, so the last round of every barrier follows from the count
    long long n_copied = 0, n_committed = 0;
    int n_tiles_done = 0;
    bool b_loaded = false;

    if (warp == 0) {
        if (lane == 0) {
            if (RB && !skip_copies && blockIdx.x < ntiles) {
                b_loaded = true;
                mbar_arrive_expect_tx(bfull, (uint32_t)(nchunks * nb) * kTileBytes);
                for (int ch = 0; ch < nchunks; ++ch)
                    for (int j = 0; j < nb; ++j)
                        bulk_copy_g2s(bres + (ch * nb + j) * kTileBytes, B + ((size_t)j * nchunks + ch) * kTileBytes,
                                      kTileBytes, bfull);
            }
            long long g = 0;  // chunk counter over all tiles of this CTA
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                for (int ch = 0; ch < nchunks; ++ch, ++g) {
                    const int st = (int)(g % kStages);
                    const long long round = g / kStages;
                    if (round > 0 && !mbar_wait_bounded(&empty[st], (uint32_t)((round - 1) & 1), wait_limit)) {
                        ok = false;
                        break;
                    }
                    if (skip_copies)  // test hook: nothing is issued, so the consumers' waits give up
                        continue;
                    uint8_t *sa = ring + st * Plan::stage_bytes;
                    ++n_copied;
                    mbar_arrive_expect_tx(&full[st], stage_tx);
                    bulk_copy_g2s(sa, A + ((size_t)t * nchunks + ch) * kTileBytes, kTileBytes, &full[st]);
                    if (!RB)
                        for (int j = 0; j < nb; ++j)
                            bulk_copy_g2s(sa + (1 + j) * kTileBytes, B + ((size_t)j * nchunks + ch) * kTileBytes,
                                          kTileBytes, &full[st]);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = instr_desc(kBM, N);
            if (RB && blockIdx.x < ntiles && !mbar_wait_bounded(bfull, 0, wait_limit))
                ok = false;
            long long g = 0;
            int tc = 0;  // tiles of this CTA so far
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tc) {
                const int buf = tc & 1, use = tc >> 1;
                if (use > 0 && !mbar_wait_bounded(&tempty[buf], (uint32_t)((use - 1) & 1), wait_limit)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dtm = taddr + (uint32_t)(buf * kBN);
                for (int ch = 0; ch < nchunks; ++ch, ++g) {
                    const int st = (int)(g % kStages);
                    const long long round = g / kStages;
                    if (!mbar_wait_bounded(&full[st], (uint32_t)(round & 1), wait_limit)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(ring + st * Plan::stage_bytes);
                    // B rows 128..255 follow rows 0..127 at +16 KiB (16 row groups)
                    const uint32_t sb = RB ? smem_u32(bres + ch * nb * kTileBytes) : sa + kTileBytes;
#pragma unroll
                    for (int k = 0; k < kKC / 16; ++k) {
                        // K = 16 spans two core matrices along K: advance by 2 x 128 B per step
                        mma_bf16(dtm, smem_desc(sa + k * 256), smem_desc(sb + k * 256), idesc,
                                 (ch > 0 || k > 0) ? 1u : 0u);
                    }
                    mma_commit(&empty[st]);
                    ++n_committed;
                }
                if (!ok)
                    break;
                mma_commit(&tfull[buf]);
                ++n_tiles_done;
            }
        }
    } else {
        const int quad = warp & 3;                     // TMEM lanes 32 quad .. 32 quad + 31
        const int cbeg = ((warp - 2) >> 2) * (kBN / 2);  // this warp's column half
        const int cend = min(N, cbeg + kBN / 2);
        float *stg = stage_all + (warp - 2) * 32 * kEpiPitch;
        const bool vec = ((uintptr_t)D % 16 == 0) && (ldd % 4 == 0);
        int tc = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++tc) {
            const int buf = tc & 1, use = tc >> 1;
            const bool got = __all_sync(0xffffffffu, mbar_wait_bounded(&tfull[buf], (uint32_t)(use & 1), wait_limit));
            if (!got) {
                ok = false;
                break;
            }
            tc_fence_after();
            const int row0 = t * kBM + quad * 32;
            const uint32_t tl = taddr + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * kBN);
            for (int c0 = cbeg; c0 < cend; c0 += 32) {
                const int w = min(32, cend - c0);  // 16 or 32 columns
                float v[32];
                tmem_ld16(tl + (uint32_t)c0, v);
                if (w > 16)
                    tmem_ld16(tl + (uint32_t)c0 + 16, v + 16);
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (j < w)
                        stg[lane * kEpiPitch + j] = v[j];
                __syncwarp();
                // w / 4 lanes per row, 16 bytes each: every store instruction writes whole rows
                const int lpr = w >> 2, rpi = 32 / lpr;
                const int cc = (lane % lpr) * 4;
                for (int r = lane / lpr; r < 32; r += rpi) {
                    const float *src = stg + r * kEpiPitch + cc;
                    float *dst = D + (size_t)(row0 + r) * ldd + c0 + cc;
                    if (vec) {
                        *reinterpret_cast<float4 *>(dst) = make_float4(src[0], src[1], src[2], src[3]);
                    } else {
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            dst[i] = src[i];
                    }
                }
                __syncwarp();
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&tempty[buf]);
        }
    }

    ok = __syncthreads_and(ok);
    if (!ok) {
        // drain (bounded) every copy issued and every MMA committed before TMEM is freed
        // (stage st last held chunk st + kStages r, r = (n - 1 - st) / kStages, when n > st)
        if (tid == 0) {
            pp_flag(status, PP_FLAG_TIMEOUT);
            for (int st = 0; st < kStages && st < n_copied; ++st)
                mbar_wait_bounded(&full[st], (uint32_t)(((n_copied - 1 - st) / kStages) & 1), 1ll << 24);
            if (b_loaded)
                mbar_wait_bounded(bfull, 0, 1ll << 24);
        }
        if (tid == 32) {
            for (int st = 0; st < kStages && st < n_committed; ++st)
                mbar_wait_bounded(&empty[st], (uint32_t)(((n_committed - 1 - st) / kStages) & 1), 1ll << 24);
            for (int i = 0; i < 2 && i < n_tiles_done; ++i)
                mbar_wait_bounded(&tfull[i], (uint32_t)(((n_tiles_done - 1 - i) / 2) & 1), 1ll << 24);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        tmem_dealloc(taddr, kTmemCols);
}

// Packs an FP32 matrix (rows x cols, leading dimension ldx; transposed if trans)
// into the BF16 tile layout above, zero-padding to rows_pad x cols_pad.
__global__ void pack_bf16_kernel(const float *__restrict__ X, int rows, int cols, int ldx, int trans,
                                 int rows_pad, int cols_pad, uint16_t *__restrict__ P)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)rows_pad * cols_pad;
    if (i >= total)
        return;
    const int r = (int)(i / cols_pad), c = (int)(i % cols_pad);
    float v = 0.0f;
    if (r < rows && c < cols)
        v = trans ? X[(size_t)c * ldx + r] : X[(size_t)r * ldx + c];
    const size_t off = ((size_t)(r / kBM) * (cols_pad / kKC) + c / kKC) * (kTileBytes / 2) +
                       ((r % kBM) / 8) * 512 + ((c % kKC) / 8) * 64 + (r % 8) * 8 + (c % 8);
    P[off] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

}  // namespace

namespace pp {

int launch_gemm_bf16(const void *A, const void *B, float *D, int M, int N, int K, int ldd,
                     cudaStream_t stream)
{
    static bool attr_set[64] = {};
    static int sms[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(gemm_bf16_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             GemmPlan<false>::smem_bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(gemm_bf16_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     GemmPlan<true>::smem_bytes);
        if (e != cudaSuccess)
            return cuda_fail(e, "GEMM shared-memory attribute");
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess)
            return cuda_fail(e, "SM count");
        sms[dev] = n;
        attr_set[dev] = true;
    }
    unsigned int *status = status_word();
    if (!status)
        return fail(PP_ERR_CUDA, "status word unavailable");
    const int ntiles = M / kBM;
    const int grid = (dev >= 0 && dev < 64 && sms[dev] > 0 && sms[dev] < ntiles) ? sms[dev] : ntiles;
    // B resident in shared memory when all its tiles fit: every CTA then reads B once
    const bool resident = (K / kKC) * (N > 128 ? 2 : 1) <= kMaxResidentB;
    if (resident)
        gemm_bf16_kernel<true><<<grid, kThreads, GemmPlan<true>::smem_bytes, stream>>>(
            (const uint8_t *)A, (const uint8_t *)B, D, M, N, K, ldd, (long long)wait_limit(), status, skip_copies());
    else
        gemm_bf16_kernel<false><<<grid, kThreads, GemmPlan<false>::smem_bytes, stream>>>(
            (const uint8_t *)A, (const uint8_t *)B, D, M, N, K, ldd, (long long)wait_limit(), status, skip_copies());
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PP_OK : cuda_fail(e, "GEMM launch");
}

int launch_pack_bf16(const float *X, int rows, int cols, int ldx, int trans, void *P, int rows_pad,
                     int cols_pad, cudaStream_t stream)
{
    const long long total = (long long)rows_pad * cols_pad;
    pack_bf16_kernel<<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(X, rows, cols, ldx, trans, rows_pad,
                                                                           cols_pad, (uint16_t *)P);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PP_OK : cuda_fail(e, "pack launch");
}

}  // namespace pp
