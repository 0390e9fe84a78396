// pp_mlp.cu -- the surrogate network of the screened DE: a multilayer
// perceptron d_in -> H -> H -> H -> 1 with GELU activations that predicts the
// (normalised) log10 of the pair number from normalised pulse parameters.
// The three hidden layers run on the tensor cores (pp_gemm.cu: BF16 operands,
// FP32 accumulation); biases, activations, the output unit, the loss and Adam
// run on the CUDA cores in FP32.  Not part of the paper.
//
// Parameters (one flat FP32 vector, this order):
//   W1 [H][d_in], b1 [H], W2 [H][H], b2 [H], W3 [H][H], b3 [H], w4 [H], b4 [1].
// Forward, for a batch X [B][d_in] (B padded to a multiple of 128 with zero rows):
//   Z1 = X W1^T + b1, A1 = gelu(Z1), Z2 = A1 W2^T + b2, A2 = gelu(Z2),
//   Z3 = A2 W3^T + b3, A3 = gelu(Z3), y = A3 w4 + b4,
// gelu(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2.  Loss: mean over the valid
// rows of (y - t)^2.  Backward: dy = 2 (y - t) / B_valid; dW = dZ^T A, db = sum
// of dZ over rows, dA = dZ W, dZ = dA gelu'(Z), gelu'(z) = Phi(z) + z phi(z).
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "pp_internal.cuh"

namespace {

constexpr int kRows = 128;  // batch rows are padded to this

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad(float z)
{
    const float Phi = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
    const float phi = 0.39894228040143268f * expf(-0.5f * z * z);
    return Phi + z * phi;
}

// Packed BF16 offset of element (r, c) in a matrix with cols_pad columns (see pp_gemm.cu).
__device__ __forceinline__ size_t packed_off(int r, int c, int cols_pad)
{
    return ((size_t)(r / 128) * (cols_pad / 64) + c / 64) * 8192 + ((r % 128) / 8) * 512 + ((c % 64) / 8) * 64 +
           (r % 8) * 8 + (c % 8);
}

// Z (B x H) += bias; A = gelu(Z); Ap = packed BF16 of A.  Rows >= nvalid are zeroed.
__global__ void bias_gelu_pack_kernel(float *__restrict__ Z, const float *__restrict__ bias, int B, int H,
                                      int nvalid, float *__restrict__ A, uint16_t *__restrict__ Ap)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)B * H)
        return;
    const int r = (int)(i / H), c = (int)(i % H);
    float z = Z[i] + bias[c];
    float a = gelu(z);
    if (r >= nvalid) {
        z = 0.0f;
        a = 0.0f;
    }
    Z[i] = z;
    A[i] = a;
    Ap[packed_off(r, c, H)] = __bfloat16_as_ushort(__float2bfloat16_rn(a));
}

// y[r] = A3[r] . w4 + b4, one warp per row.
__global__ void output_kernel(const float *__restrict__ A, const float *__restrict__ w4, const float *__restrict__ b4,
                              int B, int H, float *__restrict__ y)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= B)
        return;
    float acc = 0.0f;
    for (int c = lane; c < H; c += 32)
        acc = fmaf(A[(size_t)warp * H + c], w4[c], acc);
    for (int off = 16; off > 0; off >>= 1)
        acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0)
        y[warp] = acc + b4[0];
}

// loss = mean (y - t)^2 over the valid rows (fixed-order single-block sum);
// dy = 2 (y - t) / nvalid (0 on padded rows).
__global__ void loss_kernel(const float *__restrict__ y, const float *__restrict__ t, int B, int nvalid,
                            float *__restrict__ dy, float *__restrict__ loss)
{
    __shared__ float red[256];
    float acc = 0.0f;
    for (int r = threadIdx.x; r < B; r += blockDim.x) {
        const float e = r < nvalid ? y[r] - t[r] : 0.0f;
        dy[r] = 2.0f * e / (float)nvalid;
        acc += e * e;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss)
        *loss = red[0] / (float)nvalid;
}

// dA3 = dy w4^T; dZ3 = dA3 gelu'(Z3)  (B x H)
__global__ void output_backward_kernel(const float *__restrict__ dy, const float *__restrict__ w4,
                                       const float *__restrict__ Z, int B, int H, float *__restrict__ dZ)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)B * H)
        return;
    const int r = (int)(i / H), c = (int)(i % H);
    dZ[i] = dy[r] * w4[c] * gelu_grad(Z[i]);
}

// dZ = dA gelu'(Z) in place on dA
__global__ void gelu_backward_kernel(float *__restrict__ dA, const float *__restrict__ Z, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        dA[i] *= gelu_grad(Z[i]);
}

// out[c] = sum_r X[r][c] (column sums over B rows, fixed order per column)
__global__ void colsum_kernel(const float *__restrict__ X, int B, int H, float *__restrict__ out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= H)
        return;
    float acc = 0.0f;
    for (int r = 0; r < B; ++r)
        acc += X[(size_t)r * H + c];
    out[c] = acc;
}

// dw4[c] = sum_r dy[r] A3[r][c]; db4 = sum_r dy[r]
__global__ void output_grad_kernel(const float *__restrict__ dy, const float *__restrict__ A, int B, int H,
                                   float *__restrict__ dw4, float *__restrict__ db4)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < H) {
        float acc = 0.0f;
        for (int r = 0; r < B; ++r)
            acc = fmaf(dy[r], A[(size_t)r * H + c], acc);
        dw4[c] = acc;
    }
    if (c == 0) {
        float acc = 0.0f;
        for (int r = 0; r < B; ++r)
            acc += dy[r];
        db4[0] = acc;
    }
}

// copies an FP32 D (rows x ldd) block into a flat gradient slice (rows x cols)
__global__ void copy_block_kernel(const float *__restrict__ D, int rows, int cols, int ldd,
                                  float *__restrict__ out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)rows * cols)
        return;
    out[i] = D[(size_t)(i / cols) * ldd + i % cols];
}

// Adam (Kingma, Ba 2015) with bias correction; step is the 1-based step number.
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, long long n, float lr, float b1, float b2, float eps,
                            float c1, float c2)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// FP64 parameter vectors -> normalised FP32 network inputs: (x - lo) / (hi - lo) - 1/2
__global__ void features_kernel(const double *__restrict__ P, int B, int D, const double *__restrict__ lo,
                                const double *__restrict__ hi, int ldx, float *__restrict__ X)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)B * D)
        return;
    const int r = (int)(i / D), c = (int)(i % D);
    X[(size_t)r * ldx + c] = (float)((P[i] - lo[c]) / (hi[c] - lo[c]) - 0.5);
}

// trial[i] = props[r*][i] with r* = argmax_r y[r NP + i] (first maximum);
// kept[i] = r* NP + i
__global__ void pick_best_kernel(const double *__restrict__ props, const float *__restrict__ y, int R, int NP,
                                 int D, double *__restrict__ trial, int32_t *__restrict__ kept)
{
    const int i = blockIdx.x;
    int best = 0;
    float bv = y[i];
    for (int r = 1; r < R; ++r) {
        const float v = y[(size_t)r * NP + i];
        if (v > bv) {
            bv = v;
            best = r;
        }
    }
    for (int j = threadIdx.x; j < D; j += blockDim.x)
        trial[(size_t)i * D + j] = props[((size_t)best * NP + i) * D + j];
    if (threadIdx.x == 0)
        kept[i] = best * NP + i;
}

__device__ __forceinline__ float rank_key(float v) { return isnan(v) ? -INFINITY : v; }

// Global top-NP of the n = R NP predictions: element k has rank
// #{j : y_j > y_k or (y_j = y_k and j < k)} (NaN ranks as -inf); the element of
// rank r < NP goes to row r of trial and kept[r] = k.
constexpr int kRankThreads = 256;
__global__ void __launch_bounds__(kRankThreads) rank_top_kernel(const double *__restrict__ props,
                                                                const float *__restrict__ y, int n, int NP,
                                                                int D, double *__restrict__ trial,
                                                                int32_t *__restrict__ kept)
{
    __shared__ float tile[kRankThreads];
    const int k = blockIdx.x * kRankThreads + threadIdx.x;
    const float yk = k < n ? rank_key(y[k]) : 0.0f;
    int rank = 0;
    for (int j0 = 0; j0 < n; j0 += kRankThreads) {
        const int j = j0 + threadIdx.x;
        tile[threadIdx.x] = j < n ? rank_key(y[j]) : -INFINITY;
        __syncthreads();
        const int m = min(kRankThreads, n - j0);
        for (int q = 0; q < m; ++q) {
            const float v = tile[q];
            rank += (v > yk) || (v == yk && j0 + q < k);
        }
        __syncthreads();
    }
    if (k < n && rank < NP) {
        kept[rank] = k;
        for (int c = 0; c < D; ++c)
            trial[(size_t)rank * D + c] = props[(size_t)k * D + c];
    }
}

// Selection after global screening: individual i takes the best exactly scored
// trial among those whose parent (kept[r] mod NP) is i (first maximum, NaN never
// chosen) when its pair number is >= fit[i].  One block per individual.
__global__ void group_select_kernel(double *__restrict__ pop, double *__restrict__ fit,
                                    const double *__restrict__ trial, const double *__restrict__ tfit,
                                    const int32_t *__restrict__ kept, int NP, int D)
{
    __shared__ int s_best;
    const int i = blockIdx.x;
    if (threadIdx.x == 0) {
        int best = -1;
        double bv = 0.0;
        for (int r = 0; r < NP; ++r) {
            const double v = tfit[r];
            if (kept[r] % NP != i || isnan(v))
                continue;
            if (best < 0 || v > bv) {
                best = r;
                bv = v;
            }
        }
        s_best = (best >= 0 && bv >= fit[i]) ? best : -1;
    }
    __syncthreads();
    const int r = s_best;
    if (r < 0)
        return;
    for (int j = threadIdx.x; j < D; j += blockDim.x)
        pop[(size_t)i * D + j] = trial[(size_t)r * D + j];
    if (threadIdx.x == 0)
        fit[i] = tfit[r];
}

// SplitMix64 output k of the generator seeded with s (Steele, Lea, Flood 2014).
__host__ __device__ __forceinline__ uint64_t mlp_sm64_at(uint64_t s, uint64_t k)
{
    uint64_t z = s + (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Row order of one training epoch: a bijection of [0, n) from a 4-round Feistel
// network on b-bit integers (b the least even number with 2^b >= n; halves of
// hb = b/2 bits; round i maps (L, R) to (R, L xor (out(k_i, R) mod 2^hb)), out =
// SplitMix64), applied again while the value is >= n (cycle walking: the walk
// stays on the cycle through x, which returns below n within 2^b steps).
struct RowShuffle {
    uint64_t k[4];
    int hb;
    long long n;
};

__device__ __forceinline__ long long shuffled_row(const RowShuffle &r, long long x)
{
    const uint64_t mask = (1ull << r.hb) - 1ull;
    const long long dom = 1ll << (2 * r.hb);
    for (long long it = 0; it < dom; ++it) {
        uint64_t L = (uint64_t)x >> r.hb, R = (uint64_t)x & mask;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint64_t F = mlp_sm64_at(r.k[i], R) & mask;
            const uint64_t nL = R;
            R = L ^ F;
            L = nL;
        }
        x = (long long)((L << r.hb) | R);
        if (x < r.n)
            break;
    }
    return x;
}

// Mini-batch rows r0 .. r0 + rows - 1 of an epoch into the staging buffers.
__global__ void gather_rows_kernel(const float *__restrict__ X, const float *__restrict__ t, int din,
                                   RowShuffle sh, long long r0, int rows, float *__restrict__ Xs,
                                   float *__restrict__ ts)
{
    const int i = blockIdx.x;
    if (i >= rows)
        return;
    const long long src = shuffled_row(sh, r0 + i);
    for (int j = threadIdx.x; j < din; j += blockDim.x)
        Xs[(size_t)i * din + j] = X[(size_t)src * din + j];
    if (threadIdx.x == 0)
        ts[i] = t[src];
}

// He initialisation: parameter i of a weight block with fan-in f is
// sqrt(2/f) times a standard normal from the Box-Muller transform of outputs
// 2i and 2i+1; biases are zero.  Blocks: [W1 | b1 | W2 | b2 | W3 | b3 | w4 | b4].
__global__ void he_init_kernel(float *__restrict__ p, long long n, long long oW1, long long ob1,
                               long long oW2, long long ob2, long long oW3, long long ob3, long long ow4,
                               long long ob4, int din, int H, uint64_t seed)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    int fan = 0;
    if (i >= oW1 && i < ob1)
        fan = din;
    else if ((i >= oW2 && i < ob2) || (i >= oW3 && i < ob3) || (i >= ow4 && i < ob4))
        fan = H;
    if (!fan) {
        p[i] = 0.0f;
        return;
    }
    const double u1 = ((double)(mlp_sm64_at(seed, 2 * (uint64_t)i) >> 11) + 1.0) * 0x1.0p-53;  // (0, 1]
    const double u2 = (double)(mlp_sm64_at(seed, 2 * (uint64_t)i + 1) >> 11) * 0x1.0p-53;
    const double z = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
    p[i] = (float)(z * sqrt(2.0 / fan));
}

// t = (log10(max(N, floor)) - shift) / scale
__global__ void log_targets_kernel(const double *__restrict__ N, int n, double floor_, double shift,
                                   double scale, float *__restrict__ t)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const double v = N[i];
        t[i] = (float)((log10(v > floor_ ? v : floor_) - shift) / scale);
    }
}

inline unsigned nb(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

struct pp_mlp {
    int dev = 0, din = 0, H = 0, dinp = 0, bmax = 0;
    long long nparam = 0;
    long long off_W1, off_b1, off_W2, off_b2, off_W3, off_b3, off_w4, off_b4;
    float *p = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
    long long step = 0;
    // packed weights
    void *W1p = nullptr, *W2p = nullptr, *W3p = nullptr, *W2Tp = nullptr, *W3Tp = nullptr;
    // activations (bmax rows)
    float *X = nullptr, *Z1 = nullptr, *Z2 = nullptr, *Z3 = nullptr, *A1 = nullptr, *A2 = nullptr,
          *A3 = nullptr, *y = nullptr, *dy = nullptr, *dZ = nullptr, *dA = nullptr, *D = nullptr;
    void *Xp = nullptr, *A1p = nullptr, *A2p = nullptr, *Tp1 = nullptr, *Tp2 = nullptr;
    // shuffled mini-batches of pp_mlp_fit (bmax rows)
    float *Xs = nullptr, *ts = nullptr;
};

namespace {

size_t packed_bytes(int r, int c) { return (size_t)((r + 127) / 128 * 128) * ((c + 63) / 64 * 64) * 2; }

void mlp_free(pp_mlp *h)
{
    if (!h)
        return;
    void *ptrs[] = {h->p, h->m, h->v, h->g, h->W1p, h->W2p, h->W3p, h->W2Tp, h->W3Tp, h->X, h->Z1, h->Z2,
                    h->Z3, h->A1, h->A2, h->A3, h->y, h->dy, h->dZ, h->dA, h->D, h->Xp, h->A1p, h->A2p,
                    h->Tp1, h->Tp2, h->Xs, h->ts};
    for (void *q : ptrs)
        if (q)
            cudaFree(q);
    delete h;
}

int repack_weights(pp_mlp *h, cudaStream_t st)
{
    const int H = h->H;
    int rc = pp::launch_pack_bf16(h->p + h->off_W1, H, h->din, h->din, 0, h->W1p, H, h->dinp, st);
    if (!rc)
        rc = pp::launch_pack_bf16(h->p + h->off_W2, H, H, H, 0, h->W2p, H, H, st);
    if (!rc)
        rc = pp::launch_pack_bf16(h->p + h->off_W3, H, H, H, 0, h->W3p, H, H, st);
    if (!rc)  // W^T for dA = dZ W: B operand [in][out]
        rc = pp::launch_pack_bf16(h->p + h->off_W2, H, H, H, 1, h->W2Tp, H, H, st);
    if (!rc)
        rc = pp::launch_pack_bf16(h->p + h->off_W3, H, H, H, 1, h->W3Tp, H, H, st);
    return rc;
}

// Forward on X (rows x din, already in h->X, rows padded to Bp); y into h->y.
int forward(pp_mlp *h, int Bp, int nvalid, cudaStream_t st)
{
    const int H = h->H;
    const long long BH = (long long)Bp * H;
    int rc = pp::launch_pack_bf16(h->X, Bp, h->dinp, h->dinp, 0, h->Xp, Bp, h->dinp, st);
    if (!rc)
        rc = pp::launch_gemm_bf16(h->Xp, h->W1p, h->Z1, Bp, H, h->dinp, H, st);
    if (rc)
        return rc;
    bias_gelu_pack_kernel<<<nb(BH), 256, 0, st>>>(h->Z1, h->p + h->off_b1, Bp, H, nvalid, h->A1,
                                                  (uint16_t *)h->A1p);
    rc = pp::launch_gemm_bf16(h->A1p, h->W2p, h->Z2, Bp, H, H, H, st);
    if (rc)
        return rc;
    bias_gelu_pack_kernel<<<nb(BH), 256, 0, st>>>(h->Z2, h->p + h->off_b2, Bp, H, nvalid, h->A2,
                                                  (uint16_t *)h->A2p);
    rc = pp::launch_gemm_bf16(h->A2p, h->W3p, h->Z3, Bp, H, H, H, st);
    if (rc)
        return rc;
    bias_gelu_pack_kernel<<<nb(BH), 256, 0, st>>>(h->Z3, h->p + h->off_b3, Bp, H, nvalid, h->A3,
                                                  (uint16_t *)h->A2p /* scratch: A3 is not re-packed */);
    output_kernel<<<nb((long long)Bp * 32), 256, 0, st>>>(h->A3, h->p + h->off_w4, h->p + h->off_b4, Bp, H, h->y);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PP_OK : pp::cuda_fail(e, "surrogate forward");
}

// Backward after forward; gradient into h->g.
int backward(pp_mlp *h, const float *t, int Bp, int nvalid, float *loss, cudaStream_t st)
{
    const int H = h->H;
    const long long BH = (long long)Bp * H;
    loss_kernel<<<1, 256, 0, st>>>(h->y, t, Bp, nvalid, h->dy, loss);
    output_grad_kernel<<<nb(H, 128), 128, 0, st>>>(h->dy, h->A3, Bp, H, h->g + h->off_w4, h->g + h->off_b4);
    output_backward_kernel<<<nb(BH), 256, 0, st>>>(h->dy, h->p + h->off_w4, h->Z3, Bp, H, h->dZ);  // dZ3
    // layer 3: dW3 = dZ3^T A2, db3, dA2 = dZ3 W3
    int rc = pp::launch_pack_bf16(h->dZ, H, Bp, H, 1, h->Tp1, H, Bp, st);   // dZ3^T (H x Bp)
    if (!rc)
        rc = pp::launch_pack_bf16(h->A2, H, Bp, H, 1, h->Tp2, H, Bp, st);   // A2^T (H x Bp)
    if (!rc)
        rc = pp::launch_gemm_bf16(h->Tp1, h->Tp2, h->D, H, H, Bp, H, st);
    if (rc)
        return rc;
    copy_block_kernel<<<nb((long long)H * H), 256, 0, st>>>(h->D, H, H, H, h->g + h->off_W3);
    colsum_kernel<<<nb(H, 128), 128, 0, st>>>(h->dZ, Bp, H, h->g + h->off_b3);
    rc = pp::launch_pack_bf16(h->dZ, Bp, H, H, 0, h->Tp1, Bp, H, st);       // dZ3 (Bp x H)
    if (!rc)
        rc = pp::launch_gemm_bf16(h->Tp1, h->W3Tp, h->dA, Bp, H, H, H, st);  // dA2
    if (rc)
        return rc;
    gelu_backward_kernel<<<nb(BH), 256, 0, st>>>(h->dA, h->Z2, BH);          // dZ2 in dA
    // layer 2: dW2 = dZ2^T A1, db2, dA1 = dZ2 W2
    rc = pp::launch_pack_bf16(h->dA, H, Bp, H, 1, h->Tp1, H, Bp, st);
    if (!rc)
        rc = pp::launch_pack_bf16(h->A1, H, Bp, H, 1, h->Tp2, H, Bp, st);
    if (!rc)
        rc = pp::launch_gemm_bf16(h->Tp1, h->Tp2, h->D, H, H, Bp, H, st);
    if (rc)
        return rc;
    copy_block_kernel<<<nb((long long)H * H), 256, 0, st>>>(h->D, H, H, H, h->g + h->off_W2);
    colsum_kernel<<<nb(H, 128), 128, 0, st>>>(h->dA, Bp, H, h->g + h->off_b2);
    rc = pp::launch_pack_bf16(h->dA, Bp, H, H, 0, h->Tp1, Bp, H, st);
    if (!rc)
        rc = pp::launch_gemm_bf16(h->Tp1, h->W2Tp, h->dZ, Bp, H, H, H, st);  // dA1 in dZ
    if (rc)
        return rc;
    gelu_backward_kernel<<<nb(BH), 256, 0, st>>>(h->dZ, h->Z1, BH);          // dZ1
    // layer 1: dW1 = dZ1^T X, db1
    rc = pp::launch_pack_bf16(h->dZ, H, Bp, H, 1, h->Tp1, H, Bp, st);
    if (!rc)
        rc = pp::launch_pack_bf16(h->X, h->dinp, Bp, h->dinp, 1, h->Tp2, h->dinp, Bp, st);  // X^T
    if (!rc)
        rc = pp::launch_gemm_bf16(h->Tp1, h->Tp2, h->D, H, h->dinp, Bp, h->dinp, st);
    if (rc)
        return rc;
    copy_block_kernel<<<nb((long long)H * h->din), 256, 0, st>>>(h->D, H, h->din, h->dinp, h->g + h->off_W1);
    colsum_kernel<<<nb(H, 128), 128, 0, st>>>(h->dZ, Bp, H, h->g + h->off_b1);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PP_OK : pp::cuda_fail(e, "surrogate backward");
}

int stage_inputs(pp_mlp *h, const float *X, int B, cudaStream_t st)
{
    const int Bp = (B + kRows - 1) / kRows * kRows;
    cudaError_t e = cudaMemsetAsync(h->X, 0, sizeof(float) * (size_t)Bp * h->dinp, st);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(h->X, sizeof(float) * h->dinp, X, sizeof(float) * h->din, sizeof(float) * h->din,
                              B, cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? PP_OK : pp::cuda_fail(e, "surrogate input staging");
}

}  // namespace

using namespace pp;

extern "C" {

int pp_mlp_create(int32_t d_in, int32_t hidden, int32_t max_batch, pp_mlp **out)
{
    clear_error();
    if (!out)
        return fail(PP_ERR_INVALID_ARG, "out must not be NULL");
    *out = nullptr;
    // hidden is a whole number of 128-row GEMM tiles: it is the M of the weight-gradient
    // products and the K (and packed width) of the hidden layers
    if (d_in < 1 || d_in > 256 || (hidden != 128 && hidden != 256) || max_batch < 1 || max_batch > (1 << 20))
        return fail(PP_ERR_INVALID_ARG, "need 1 <= d_in <= 256, hidden = 128 or 256, 1 <= max_batch <= 2^20");
    pp_mlp *h = new pp_mlp();
    cudaGetDevice(&h->dev);
    h->din = d_in;
    h->H = hidden;
    h->dinp = (d_in + 63) / 64 * 64;
    if (h->dinp > 256) {
        delete h;
        return fail(PP_ERR_INVALID_ARG, "d_in too large");
    }
    h->bmax = (max_batch + kRows - 1) / kRows * kRows;
    const long long H = hidden;
    h->off_W1 = 0;
    h->off_b1 = H * d_in;
    h->off_W2 = h->off_b1 + H;
    h->off_b2 = h->off_W2 + H * H;
    h->off_W3 = h->off_b2 + H;
    h->off_b3 = h->off_W3 + H * H;
    h->off_w4 = h->off_b3 + H;
    h->off_b4 = h->off_w4 + H;
    h->nparam = h->off_b4 + 1;
    const size_t BH = (size_t)h->bmax * hidden;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **pp_, size_t bytes) {
        if (e == cudaSuccess)
            e = cudaMalloc(pp_, bytes);
        if (e == cudaSuccess)
            e = cudaMemset(*pp_, 0, bytes);
    };
    alloc((void **)&h->p, sizeof(float) * h->nparam);
    alloc((void **)&h->m, sizeof(float) * h->nparam);
    alloc((void **)&h->v, sizeof(float) * h->nparam);
    alloc((void **)&h->g, sizeof(float) * h->nparam);
    alloc(&h->W1p, packed_bytes(hidden, h->dinp));
    alloc(&h->W2p, packed_bytes(hidden, hidden));
    alloc(&h->W3p, packed_bytes(hidden, hidden));
    alloc(&h->W2Tp, packed_bytes(hidden, hidden));
    alloc(&h->W3Tp, packed_bytes(hidden, hidden));
    alloc((void **)&h->X, sizeof(float) * (size_t)h->bmax * h->dinp);
    float **acts[] = {&h->Z1, &h->Z2, &h->Z3, &h->A1, &h->A2, &h->A3, &h->dZ, &h->dA};
    for (float **a : acts)
        alloc((void **)a, sizeof(float) * BH);
    alloc((void **)&h->D, sizeof(float) * (size_t)std::max(BH, (size_t)hidden * hidden));
    alloc((void **)&h->y, sizeof(float) * h->bmax);
    alloc((void **)&h->dy, sizeof(float) * h->bmax);
    alloc(&h->Xp, packed_bytes(h->bmax, h->dinp));
    alloc(&h->A1p, packed_bytes(h->bmax, hidden));
    alloc(&h->A2p, packed_bytes(h->bmax, hidden));
    const size_t tp = std::max(packed_bytes(h->bmax, hidden), packed_bytes(hidden, h->bmax));
    alloc(&h->Tp1, tp);
    alloc(&h->Tp2, std::max(tp, packed_bytes(h->dinp, h->bmax)));
    alloc((void **)&h->Xs, sizeof(float) * (size_t)h->bmax * h->din);
    alloc((void **)&h->ts, sizeof(float) * h->bmax);
    if (e != cudaSuccess) {
        mlp_free(h);
        return cuda_fail(e, "surrogate allocation");
    }
    *out = h;
    return PP_OK;
}

void pp_mlp_destroy(pp_mlp *h) { mlp_free(h); }

int64_t pp_mlp_num_params(const pp_mlp *h) { return h ? h->nparam : 0; }

int pp_mlp_set_params(pp_mlp *h, const float *params, void *stream)
{
    clear_error();
    if (!h || !params)
        return fail(PP_ERR_INVALID_ARG, "handle and params must not be NULL");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(h->p, params, sizeof(float) * h->nparam, cudaMemcpyDefault, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(h->m, 0, sizeof(float) * h->nparam, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(h->v, 0, sizeof(float) * h->nparam, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "surrogate parameters");
    h->step = 0;
    return repack_weights(h, st);
}

int pp_mlp_init(pp_mlp *h, uint64_t seed, void *stream)
{
    clear_error();
    if (!h)
        return fail(PP_ERR_INVALID_ARG, "network handle is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    he_init_kernel<<<nb(h->nparam), 256, 0, st>>>(h->p, h->nparam, h->off_W1, h->off_b1, h->off_W2, h->off_b2,
                                                   h->off_W3, h->off_b3, h->off_w4, h->off_b4, h->din, h->H,
                                                   seed);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemsetAsync(h->m, 0, sizeof(float) * h->nparam, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(h->v, 0, sizeof(float) * h->nparam, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "surrogate initialisation");
    h->step = 0;
    return repack_weights(h, st);
}

int pp_mlp_get_params(const pp_mlp *h, float *params, void *stream)
{
    clear_error();
    if (!h || !params)
        return fail(PP_ERR_INVALID_ARG, "handle and params must not be NULL");
    cudaError_t e = cudaMemcpyAsync(params, h->p, sizeof(float) * h->nparam, cudaMemcpyDefault,
                                    (cudaStream_t)stream);
    return e == cudaSuccess ? PP_OK : cuda_fail(e, "surrogate parameters");
}

int pp_mlp_forward(pp_mlp *h, const float *X, int32_t B, float *y, void *stream)
{
    clear_error();
    if (!h || !X || !y || B < 1 || B > h->bmax)
        return fail(PP_ERR_INVALID_ARG, "need a handle, X, y and 1 <= B <= max_batch");
    cudaStream_t st = (cudaStream_t)stream;
    const int Bp = (B + kRows - 1) / kRows * kRows;
    int rc = stage_inputs(h, X, B, st);
    if (!rc)
        rc = forward(h, Bp, B, st);
    if (rc)
        return rc;
    cudaError_t e = cudaMemcpyAsync(y, h->y, sizeof(float) * B, cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? PP_OK : cuda_fail(e, "surrogate output");
}

int pp_mlp_loss_grad(pp_mlp *h, const float *X, const float *t, int32_t B, float *loss, float *grad,
                     void *stream)
{
    clear_error();
    if (!h || !X || !t || B < 1 || B > h->bmax)
        return fail(PP_ERR_INVALID_ARG, "need a handle, X, t and 1 <= B <= max_batch");
    cudaStream_t st = (cudaStream_t)stream;
    const int Bp = (B + kRows - 1) / kRows * kRows;
    int rc = stage_inputs(h, X, B, st);
    if (!rc)
        rc = forward(h, Bp, B, st);
    if (!rc) {
        // targets on padded rows are never read (dy = 0 there)
        rc = backward(h, t, Bp, B, loss, st);
    }
    if (rc)
        return rc;
    if (grad) {
        cudaError_t e = cudaMemcpyAsync(grad, h->g, sizeof(float) * h->nparam, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess)
            return cuda_fail(e, "surrogate gradient");
    }
    return PP_OK;
}

int pp_mlp_train_step(pp_mlp *h, const float *X, const float *t, int32_t B, float lr, float *loss,
                      void *stream)
{
    int rc = pp_mlp_loss_grad(h, X, t, B, loss, nullptr, stream);
    if (rc)
        return rc;
    cudaStream_t st = (cudaStream_t)stream;
    h->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f - powf(b1, (float)h->step), c2 = 1.0f - powf(b2, (float)h->step);
    adam_kernel<<<nb(h->nparam), 256, 0, st>>>(h->p, h->g, h->m, h->v, h->nparam, lr, b1, b2, eps, c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e, "Adam");
    return repack_weights(h, st);
}

int pp_mlp_fit(pp_mlp *h, const float *X, const float *t, int32_t n, int32_t batch, int32_t epochs,
               float lr0, float lr1, uint64_t seed, float *epoch_loss, void *stream)
{
    clear_error();
    if (!h || !X || !t || n < 1 || batch < 1 || batch > h->bmax || epochs < 1)
        return fail(PP_ERR_INVALID_ARG, "need a network, X and t, n >= 1, 1 <= batch <= max_batch, epochs >= 1");
    if (!(lr0 >= 0.0f) || !(lr1 >= 0.0f))
        return fail(PP_ERR_INVALID_ARG, "learning rates must be non-negative");
    cudaStream_t st = (cudaStream_t)stream;
    RowShuffle sh;
    sh.n = n;
    sh.hb = 0;
    while ((1ll << (2 * sh.hb)) < (long long)n)
        ++sh.hb;
    const long long per = (n + (long long)batch - 1) / batch, total = per * epochs;
    long long k = 0;
    for (int e = 0; e < epochs; ++e) {
        for (int i = 0; i < 4; ++i)
            sh.k[i] = mlp_sm64_at(seed, 4 * (uint64_t)e + (uint64_t)i);
        for (long long b = 0; b < per; ++b, ++k) {
            const int r0 = (int)(b * batch), rows = (int)std::min<long long>(batch, n - r0);
            // cosine schedule from lr0 (first step) to lr1 (last step)
            const double c = total > 1 ? 0.5 * (1.0 + cos(M_PI * (double)k / (double)(total - 1))) : 1.0;
            const float lr = (float)(lr1 + (lr0 - lr1) * c);
            float *loss = (epoch_loss && b == per - 1) ? epoch_loss + e : nullptr;
            const float *Xb = X + (size_t)r0 * h->din, *tb = t + r0;
            if (seed != 0) {
                gather_rows_kernel<<<rows, 64, 0, st>>>(X, t, h->din, sh, r0, rows, h->Xs, h->ts);
                cudaError_t eg = cudaGetLastError();
                if (eg != cudaSuccess)
                    return cuda_fail(eg, "mini-batch gather");
                Xb = h->Xs;
                tb = h->ts;
            }
            const int rc = pp_mlp_train_step(h, Xb, tb, rows, lr, loss, stream);
            if (rc)
                return rc;
        }
    }
    return PP_OK;
}

int pp_mlp_log_targets(const double *N, int32_t n, double floor_value, double shift, double scale, float *t,
                       void *stream)
{
    clear_error();
    if (!N || !t || n < 0 || !(floor_value > 0.0) || !(scale != 0.0) || !isfinite(shift) || !isfinite(scale))
        return fail(PP_ERR_INVALID_ARG, "need N and t, n >= 0, floor > 0, finite shift and non-zero scale");
    if (n == 0)
        return PP_OK;
    log_targets_kernel<<<nb(n), 256, 0, (cudaStream_t)stream>>>(N, n, floor_value, shift, scale, t);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PP_OK : cuda_fail(e, "log targets");
}

int pp_de_screened_step(double *pop, double *fit, int32_t NP, const pp_field_spec *spec,
                        const pp_grid *grid, int32_t precision, int32_t scheme, const double *lo,
                        const double *hi, const uint8_t *periodic, double F, double CR, uint64_t seed,
                        uint64_t generation, int32_t R, int32_t mode, pp_mlp *mlp, double *trial_out,
                        double *trial_fit_out, float *pred_out, int32_t *kept_out, void *stream)
{
    clear_error();
    int rc = check_spec(spec);
    if (!rc)
        rc = check_grid(grid);
    if (rc)
        return rc;
    if (!pop || !fit || !lo || !hi || !mlp)
        return fail(PP_ERR_INVALID_ARG, "pop, fit, lo, hi and mlp must not be NULL");
    if (precision != PP_FP64 && precision != PP_FP32 && precision != PP_FP32_FAST)
        return fail(PP_ERR_INVALID_ARG, "precision must be PP_FP64, PP_FP32 or PP_FP32_FAST");
    if (scheme != PP_RK4 && scheme != PP_MAGNUS4 && scheme != PP_SPLIT2)
        return fail(PP_ERR_INVALID_ARG, "scheme must be PP_RK4, PP_MAGNUS4 or PP_SPLIT2");
    const int D = 4 * spec->K;
    if (NP < 4 || NP > 65535 || R < 1 || R > 64 || (long long)R * NP > mlp->bmax || D != mlp->din)
        return fail(PP_ERR_INVALID_ARG, "need NP >= 4, 1 <= R <= 64, R NP <= the network's max_batch "
                                        "and 4K equal to its input size");
    if (!(CR >= 0.0 && CR <= 1.0) || !isfinite(F))
        return fail(PP_ERR_INVALID_ARG, "CR must be in [0, 1] and F finite");
    if (mode != PP_SCREEN_PER_INDIVIDUAL && mode != PP_SCREEN_GLOBAL)
        return fail(PP_ERR_INVALID_ARG, "mode must be PP_SCREEN_PER_INDIVIDUAL or PP_SCREEN_GLOBAL");
    cudaStream_t st = (cudaStream_t)stream;
    void *props = nullptr, *X = nullptr, *y = nullptr, *trial = nullptr, *tfit = nullptr, *A = nullptr;
    void *kept = nullptr;
    const int ld = 2 * spec->n_steps + 1;
    rc = scratch(SCR_SCREEN_PROPS, sizeof(double) * (size_t)R * NP * D, &props);
    if (!rc)
        rc = scratch(SCR_SCREEN_X, sizeof(float) * (size_t)R * NP * D, &X);
    if (!rc)
        rc = scratch(SCR_SCREEN_Y, sizeof(float) * (size_t)R * NP, &y);
    if (!rc && !trial_out)
        rc = scratch(SCR_TRIAL, sizeof(double) * (size_t)NP * D, &trial);
    if (!rc && !trial_fit_out)
        rc = scratch(SCR_TFIT, sizeof(double) * (size_t)NP, &tfit);
    if (!rc)
        rc = scratch(SCR_A, sizeof(double) * 2 * (size_t)ld * NP, &A);
    if (!rc && !kept_out)
        rc = scratch(SCR_SCREEN_KEPT, sizeof(int32_t) * (size_t)NP, &kept);
    if (rc)
        return rc;
    int32_t *kp = kept_out ? kept_out : (int32_t *)kept;
    double *tr = trial_out ? trial_out : (double *)trial;
    double *tf = trial_fit_out ? trial_fit_out : (double *)tfit;
    // R proposals per individual, each from its own counter-RNG stream (generation R g + r)
    for (int r = 0; r < R && !rc; ++r)
        rc = launch_de_propose(pop, NP, D, lo, hi, periodic, F, CR, seed, generation * (uint64_t)R + r,
                               (double *)props + (size_t)r * NP * D, st);
    if (rc)
        return rc;
    features_kernel<<<nb((long long)R * NP * D), 256, 0, st>>>((const double *)props, R * NP, D, lo, hi, D,
                                                                (float *)X);
    rc = pp_mlp_forward(mlp, (const float *)X, R * NP, (float *)y, stream);
    if (rc)
        return rc;
    if (pred_out) {
        cudaError_t e = cudaMemcpyAsync(pred_out, y, sizeof(float) * (size_t)R * NP, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess)
            return cuda_fail(e, "screening predictions");
    }
    if (mode == PP_SCREEN_PER_INDIVIDUAL)
        pick_best_kernel<<<NP, 64, 0, st>>>((const double *)props, (const float *)y, R, NP, D, tr, kp);
    else
        rank_top_kernel<<<nb((long long)R * NP, kRankThreads), kRankThreads, 0, st>>>(
            (const double *)props, (const float *)y, R * NP, NP, D, tr, kp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e, "screening pick");
    if ((rc = launch_synth_field(tr, NP, spec, (double *)A, ld, nullptr, nullptr, st)))
        return rc;
    if ((rc = launch_pair_number((double *)A, NP, ld, nullptr, spec->T / spec->n_steps, grid, precision,
                                 scheme, tf, nullptr, st)))
        return rc;
    if (mode == PP_SCREEN_PER_INDIVIDUAL)
        return launch_de_select(pop, fit, tr, tf, NP, D, st);
    group_select_kernel<<<NP, 64, 0, st>>>(pop, fit, tr, tf, kp, NP, D);
    e = cudaGetLastError();
    return e == cudaSuccess ? PP_OK : cuda_fail(e, "screening selection");
}

int pp_mlp_features(const double *params, int32_t B, int32_t D, const double *lo, const double *hi,
                    float *X, void *stream)
{
    clear_error();
    if (!params || !lo || !hi || !X || B < 1 || D < 1)
        return fail(PP_ERR_INVALID_ARG, "bad arguments");
    features_kernel<<<nb((long long)B * D), 256, 0, (cudaStream_t)stream>>>(params, B, D, lo, hi, D, X);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PP_OK : cuda_fail(e, "features");
}

}  // extern "C"
