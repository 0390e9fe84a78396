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
// One CTA of 128 threads computes a 128 x 128 block of D (the last column block
// may be narrower): warp 0 allocates its TMEM columns, thread 0 issues 4 MMAs
// (K = 16 each) per 64-wide K chunk from a 3-stage ring of bulk copies, each warp
// then reads its 32 TMEM lanes with tcgen05.ld and writes its rows of D.
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

// Shared-memory plan: a ring of kStages stages x (A tile 16 KiB + B tile 16 KiB) and
// the barriers; two CTAs fit on an SM.
constexpr int kStages = 3;
constexpr int kBN = 128;                      // columns per CTA (one packed B tile)
constexpr int kStageBytes = 2 * kTileBytes;
constexpr int kSmemBytes = kStages * kStageBytes + 1024 + 128;

// One CTA: rows [128 mt, 128 mt + 128) x columns [128 nt, 128 nt + nc), nc = min(128, N - 128 nt).
// Thread 0 keeps kStages chunks in flight: after issuing chunk ch's MMAs it waits for
// chunk ch-1's MMAs to finish reading their stage and refills that stage with chunk
// ch-1+kStages, so the tensor pipe always has the next chunk queued.
__global__ void __launch_bounds__(128, 2)
    gemm_bf16_kernel(const uint8_t *__restrict__ A, const uint8_t *__restrict__ B, float *__restrict__ D,
                     int M, int N, int K, int ldd, long long wait_limit, unsigned int *__restrict__ status,
                     int skip_copies)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const bool vec = ((uintptr_t)D % 16 == 0) && (ldd % 4 == 0);
    uint64_t *full = (uint64_t *)(smem + kStages * kStageBytes);  // [kStages] copies landed
    uint64_t *done = full + kStages;                              // [kStages] MMAs of a stage finished
    uint32_t *s_taddr = (uint32_t *)(done + kStages);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mt = blockIdx.x, nt = blockIdx.y;
    const int nc = min(kBN, N - nt * kBN);  // a multiple of 16 in [16, 128]
    const int nchunks = K / kKC;
    const uint32_t ncols = nc <= 32 ? 32 : (nc <= 64 ? 64 : 128);

    if (warp == 0)
        tmem_alloc(s_taddr, ncols);
    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&done[i], 1);
        }
        mbar_fence_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *s_taddr;

    int last_issue[kStages], last_commit[kStages];  // thread 0's bookkeeping for the drain
    for (int i = 0; i < kStages; ++i)
        last_issue[i] = last_commit[i] = -1;
    auto issue_copy = [&](int ch, int st) {
        if (skip_copies)  // test hook: nothing is issued, so the first wait gives up
            return;
        uint8_t *sa = smem + st * kStageBytes;
        last_issue[st] = ch;
        mbar_arrive_expect_tx(&full[st], 2u * kTileBytes);
        bulk_copy_g2s(sa, A + ((size_t)mt * nchunks + ch) * kTileBytes, kTileBytes, &full[st]);
        bulk_copy_g2s(sa + kTileBytes, B + ((size_t)nt * nchunks + ch) * kTileBytes, kTileBytes, &full[st]);
    };

    bool ok = true;
    if (tid == 0) {
        const uint32_t idesc = instr_desc(kBM, nc);
        for (int ch = 0; ch < kStages && ch < nchunks; ++ch)
            issue_copy(ch, ch);
        for (int ch = 0; ch < nchunks && ok; ++ch) {
            const int st = ch % kStages;
            if (!mbar_wait_bounded(&full[st], (ch / kStages) & 1, wait_limit)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + st * kStageBytes);
            const uint32_t sb = sa + kTileBytes;
#pragma unroll
            for (int k = 0; k < kKC / 16; ++k) {
                // K = 16 spans two core matrices along K: advance by 2 x 128 B per step
                mma_bf16(taddr, smem_desc(sa + k * 256), smem_desc(sb + k * 256), idesc,
                         (ch > 0 || k > 0) ? 1u : 0u);
            }
            mma_commit(&done[st]);
            last_commit[st] = ch;
            const int prev = ch - 1;
            if (prev >= 0 && prev + kStages < nchunks) {
                const int pst = prev % kStages;
                if (!mbar_wait_bounded(&done[pst], (prev / kStages) & 1, wait_limit)) {
                    ok = false;
                    break;
                }
                issue_copy(prev + kStages, pst);
            }
        }
        if (ok) {
            // the last commit covers every earlier MMA of this thread
            const int last = nchunks - 1;
            ok = mbar_wait_bounded(&done[last % kStages], (last / kStages) & 1, wait_limit);
        }
        if (!ok) {
            pp_flag(status, PP_FLAG_TIMEOUT);
            // drain (bounded) every copy issued and every MMA committed before TMEM is freed
            for (int st = 0; st < kStages; ++st) {
                if (last_issue[st] >= 0)
                    mbar_wait_bounded(&full[st], (last_issue[st] / kStages) & 1, 1ll << 24);
                if (last_commit[st] >= 0)
                    mbar_wait_bounded(&done[st], (last_commit[st] / kStages) & 1, 1ll << 24);
            }
        }
    }
    ok = __syncthreads_and(ok);
    tc_fence_after();
    if (ok) {
        const int row = mt * kBM + warp * 32 + lane;
        float *drow = D + (size_t)row * ldd + (size_t)nt * kBN;
        for (int c0 = 0; c0 < nc; c0 += 16) {
            float v[16];
            tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (row < M) {
                if (vec) {  // 16-byte stores: a thread's 16 columns are 64 contiguous bytes
                    float4 *d4 = reinterpret_cast<float4 *>(drow + c0);
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        d4[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        drow[c0 + i] = v[i];
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        tmem_dealloc(taddr, ncols);
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

int gemm_smem_bytes() { return kSmemBytes; }

int launch_gemm_bf16(const void *A, const void *B, float *D, int M, int N, int K, int ldd,
                     cudaStream_t stream)
{
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kSmemBytes);
        if (e != cudaSuccess)
            return cuda_fail(e, "GEMM shared-memory attribute");
        attr_set[dev] = true;
    }
    unsigned int *status = status_word();
    if (!status)
        return fail(PP_ERR_CUDA, "status word unavailable");
    gemm_bf16_kernel<<<dim3(M / kBM, (N + kBN - 1) / kBN), 128, kSmemBytes, stream>>>(
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
