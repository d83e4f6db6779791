// rad_mlp.cu -- the learned surrogate's network: a ReLU MLP with BF16 weights
// (FP32 master copy), BF16 GEMM operands and FP32 accumulation, trained with
// MSE and Adam, entirely on the device (C ABI in include/rad_mlp.h).
//
// GEMMs run on the tensor cores (mma.sync m16n8k16 BF16 -> FP32) in one kernel
// template whose operands may be stored K-contiguous or not: ldmatrix (or
// ldmatrix.trans) reads them from shared memory in the fragment layout, so the
// forward (X W^T), input-gradient (G W) and weight-gradient (G^T X) products
// all read their operands in place.  Tiles: 128 x 128 x 32 per 256-thread
// block, cp.async double buffering, epilogue fused (bias, ReLU, ReLU mask of
// the backward pass, FP32 and/or BF16 output).  Products with few output
// tiles and a long K (the input gradient of the wide output layer: 128 x 512
// outputs over K = 393,216) split K across blocks: each slice writes raw FP32
// partial sums and one reduction kernel adds the slices in a fixed order and
// applies the epilogue, so the result does not depend on scheduling.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "rad_mlp.h"

namespace {

typedef __nv_bfloat16 bf16;

constexpr int TM = 128, TN = 128, TK = 32;   // block tile
constexpr int kGemmThreads = 256;
constexpr int kSplitTargetBlocks = 2 * 152;  // two resident blocks on each of 152 SMs
constexpr int kMinSplitTiles = 8;            // K tiles per slice at least

struct Epilogue {
    const float* bias;      // [N] or null
    const float* mask;      // [M][N] (z of the backward pass: keep where > 0) or null
    float* out_f32;         // [M][N] or null
    bf16* out_bf16;         // [M][N] or null
    int relu;               // apply ReLU before the BF16 store
};

// Number of K slices for an M x N x K product: enough blocks to fill the GPU
// twice over when the output alone gives too few, each slice kMinSplitTiles
// K tiles or more.
int split_count(int M, int N, int K)
{
    const int blocks = (M / TM) * (N / TN), nk = K / TK;
    if (blocks >= kSplitTargetBlocks / 2) return 1;
    const int want = (kSplitTargetBlocks + blocks - 1) / blocks;
    return std::max(1, std::min(want, nk / kMinSplitTiles));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// C[M][N] = op(A) op(B) with op(A) [M][K], op(B)^T [N][K].
//   AK: A stored [M][K] (row m at A + m lda); else stored [K][M] (row k at A + k lda).
//   BKC: B stored [N][K] (row n at B + n ldb); else stored [K][N].
// M, N multiples of 128, K a multiple of 32, leading dimensions multiples of 8.
template <bool AK, bool BKC>
__global__ void __launch_bounds__(kGemmThreads) gemm_bf16_kernel(const bf16* __restrict__ A,
                                                                 const bf16* __restrict__ B, int M,
                                                                 int N, int K, int lda, int ldb,
                                                                 Epilogue ep, float* partial)
{
    constexpr int A_ROWS = AK ? TM : TK, A_COLS = (AK ? TK : TM) + 8;
    constexpr int B_ROWS = BKC ? TN : TK, B_COLS = (BKC ? TK : TN) + 8;
    __shared__ __align__(16) bf16 As[2][A_ROWS][A_COLS];
    __shared__ __align__(16) bf16 Bs[2][B_ROWS][B_COLS];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;           // 2 x 4 warps, 64 x 32 each
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;

    auto load_stage = [&](int st, int k0) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = tid + h * kGemmThreads;     // 512 chunks of 16 B per operand
            if (AK) {
                const int r = c >> 2, col = (c & 3) * 8;
                cp_async16(&As[st][r][col], A + (size_t)(m0 + r) * lda + k0 + col);
            } else {
                const int r = c >> 4, col = (c & 15) * 8;
                cp_async16(&As[st][r][col], A + (size_t)(k0 + r) * lda + m0 + col);
            }
            if (BKC) {
                const int r = c >> 2, col = (c & 3) * 8;
                cp_async16(&Bs[st][r][col], B + (size_t)(n0 + r) * ldb + k0 + col);
            } else {
                const int r = c >> 4, col = (c & 15) * 8;
                cp_async16(&Bs[st][r][col], B + (size_t)(k0 + r) * ldb + n0 + col);
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };

    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;

    // K tiles of this block's slice (the whole K range when gridDim.z == 1)
    const int nk_all = K / TK, S = gridDim.z, z = blockIdx.z;
    const int kt0 = (int)((int64_t)nk_all * z / S), kt1 = (int)((int64_t)nk_all * (z + 1) / S);
    const int nk = kt1 - kt0;
    load_stage(0, kt0 * TK);
    const int r8 = lane & 7, j4 = lane >> 3;
    for (int kt = 0; kt < nk; ++kt) {
        const int st = kt & 1;
        if (kt + 1 < nk) {
            load_stage(st ^ 1, (kt0 + kt + 1) * TK);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; kk += 16) {
            uint32_t a[4][4], b[2][4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int mb = wm * 64 + i * 16;
                if (AK) ldsm_x4(a[i], &As[st][mb + r8 + 8 * (j4 & 1)][kk + 8 * (j4 >> 1)]);
                else ldsm_x4_t(a[i], &As[st][kk + r8 + 8 * (j4 >> 1)][mb + 8 * (j4 & 1)]);
            }
#pragma unroll
            for (int jp = 0; jp < 2; ++jp) {
                const int nb = wn * 32 + jp * 16;
                if (BKC) ldsm_x4(b[jp], &Bs[st][nb + r8 + 8 * (j4 >> 1)][kk + 8 * (j4 & 1)]);
                else ldsm_x4_t(b[jp], &Bs[st][kk + r8 + 8 * (j4 & 1)][nb + 8 * (j4 >> 1)]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    mma_bf16(acc[i][j], a[i], b[j >> 1][2 * (j & 1)], b[j >> 1][2 * (j & 1) + 1]);
        }
        __syncthreads();
    }

    if (partial) {   // split K: raw partial sums of slice z, epilogue in splitk_reduce
        float* P = partial + (size_t)z * M * N;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int hlf = 0; hlf < 2; ++hlf) {
                    const int m = m0 + wm * 64 + i * 16 + (lane >> 2) + 8 * hlf;
                    const int n = n0 + wn * 32 + j * 8 + 2 * (lane & 3);
                    *reinterpret_cast<float2*>(P + (size_t)m * N + n) =
                        make_float2(acc[i][j][2 * hlf], acc[i][j][2 * hlf + 1]);
                }
        return;
    }
    // epilogue
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int hlf = 0; hlf < 2; ++hlf) {
                const int m = m0 + wm * 64 + i * 16 + (lane >> 2) + 8 * hlf;
                const int n = n0 + wn * 32 + j * 8 + 2 * (lane & 3);
                float v0 = acc[i][j][2 * hlf], v1 = acc[i][j][2 * hlf + 1];
                if (ep.bias) {
                    v0 += ep.bias[n];
                    v1 += ep.bias[n + 1];
                }
                const size_t o = (size_t)m * N + n;
                if (ep.mask) {
                    v0 = ep.mask[o] > 0.0f ? v0 : 0.0f;
                    v1 = ep.mask[o + 1] > 0.0f ? v1 : 0.0f;
                }
                if (ep.out_f32) *reinterpret_cast<float2*>(ep.out_f32 + o) = make_float2(v0, v1);
                if (ep.out_bf16) {
                    if (ep.relu) {
                        v0 = fmaxf(v0, 0.0f);
                        v1 = fmaxf(v1, 0.0f);
                    }
                    *reinterpret_cast<__nv_bfloat162*>(ep.out_bf16 + o) = __floats2bfloat162_rn(v0, v1);
                }
            }
}

// Sum of the S slices' partials in slice order, then the epilogue of the
// unsplit kernel (four consecutive outputs per thread; N is a multiple of 128).
__global__ void splitk_reduce(const float* __restrict__ partial, int S, int M, int N, Epilogue ep)
{
    const int64_t MN = (int64_t)M * N, n4 = MN / 4;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n4;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = 4 * q;
        float4 v = *reinterpret_cast<const float4*>(partial + o);
        for (int s = 1; s < S; ++s) {
            const float4 p = *reinterpret_cast<const float4*>(partial + s * MN + o);
            v.x += p.x;
            v.y += p.y;
            v.z += p.z;
            v.w += p.w;
        }
        float r[4] = {v.x, v.y, v.z, v.w};
        const int n = (int)(o % N);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (ep.bias) r[c] += ep.bias[n + c];
            if (ep.mask) r[c] = ep.mask[o + c] > 0.0f ? r[c] : 0.0f;
        }
        if (ep.out_f32) *reinterpret_cast<float4*>(ep.out_f32 + o) = make_float4(r[0], r[1], r[2], r[3]);
        if (ep.out_bf16) {
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (ep.relu) r[c] = fmaxf(r[c], 0.0f);
            __nv_bfloat162* d = reinterpret_cast<__nv_bfloat162*>(ep.out_bf16 + o);
            d[0] = __floats2bfloat162_rn(r[0], r[1]);
            d[1] = __floats2bfloat162_rn(r[2], r[3]);
        }
    }
}

// C = op(A) op(B) with the fused epilogue.  work: FP32 scratch of at least
// split_count(M, N, K) * M * N floats, or null to run unsplit.
template <bool AK, bool BKC>
cudaError_t gemm(const bf16* A, const bf16* B, int M, int N, int K, int lda, int ldb,
                 const Epilogue& ep, cudaStream_t st, float* work = nullptr)
{
    if (M % TM || N % TN || K % TK || lda % 8 || ldb % 8) return cudaErrorInvalidValue;
    const int S = work ? split_count(M, N, K) : 1;
    dim3 grid(N / TN, M / TM, S);
    gemm_bf16_kernel<AK, BKC><<<grid, kGemmThreads, 0, st>>>(A, B, M, N, K, lda, ldb, ep,
                                                             S > 1 ? work : nullptr);
    if (S > 1) {
        const int64_t n4 = (int64_t)M * N / 4;
        const int blocks = (int)std::min<int64_t>((n4 + 255) / 256, 4 * 152);
        splitk_reduce<<<blocks, 256, 0, st>>>(work, S, M, N, ep);
    }
    return cudaGetLastError();
}

__global__ void to_bf16_rows(const float* x, bf16* y, int rows_valid, int rows, int cols)
{
    const int64_t n = (int64_t)rows * cols;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / cols);
        y[i] = __float2bfloat16_rn(r < rows_valid ? x[i] : 0.0f);
    }
}

// MSE over the valid rows: g = 2 (y - t) / (rows_valid * cols) (FP32 and BF16),
// loss accumulated in FP64.
__global__ void mse_grad(const float* y, const float* t, float* g, bf16* gb, double* loss,
                         int rows_valid, int rows, int cols)
{
    const int64_t n = (int64_t)rows * cols;
    const double inv = 1.0 / ((double)rows_valid * cols);
    double part = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / cols);
        float gi = 0.0f;
        if (r < rows_valid) {
            const float d = y[i] - t[i];
            part += (double)d * d;
            gi = (float)(2.0 * inv) * d;
        }
        g[i] = gi;
        gb[i] = __float2bfloat16_rn(gi);
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0 && part != 0.0) atomicAdd(loss, part * inv);
}

// db[n] = sum over rows of g[r][n]
__global__ void column_sums(const float* g, float* db, int rows, int cols)
{
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < cols; n += gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int r = 0; r < rows; ++r) s += g[(size_t)r * cols + n];
        db[n] = s;
    }
}

// Adam on the FP32 master weights; refreshes the BF16 copy.
__global__ void adam_update(float* w, bf16* wb, float* m, float* v, const float* g, int64_t n,
                            float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        if (wb) wb[i] = __float2bfloat16_rn(wi);
    }
}

__global__ void f32_to_bf16(const float* x, bf16* y, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

int grid_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 4096); }

bool is_dev(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

struct rad_mlp {
    int L = 0;                      // layers
    std::vector<int> w;             // widths [L + 1]
    int max_rows = 0;               // max batch rounded up to 128
    cudaStream_t st = nullptr;
    // parameters: per layer, [out][in]
    std::vector<float*> W, b, Wm, Wv, bm, bv, dW, db;
    std::vector<bf16*> Wb;
    int64_t step = 0;
    // activations: h[l] bf16 [rows][w[l]] (h[0] = input), z[l] fp32 [rows][w[l]] (l >= 1)
    std::vector<bf16*> h;
    std::vector<float*> z;
    float* t = nullptr;             // targets [rows][w[L]]
    float* g = nullptr;             // output gradient fp32 [rows][w[L]]
    std::vector<bf16*> gb;          // layer gradients bf16: gb[l] [rows][w[l]] for l >= 1
    double* loss = nullptr;
    float* xin = nullptr;           // staging for host inputs [rows][w[0]]
    float* work = nullptr;          // split-K partial sums (largest split product)
};

#define MCU(call)                                            \
    do {                                                     \
        if ((call) != cudaSuccess) return RAD_MLP_ECUDA;     \
    } while (0)

static int round128(int n) { return (n + 127) / 128 * 128; }

extern "C" {

int rad_mlp_init(rad_mlp** out, const int32_t* widths, int32_t n_layers, int32_t max_batch,
                 void* stream)
{
    if (!out || !widths || n_layers < 1 || n_layers > 16 || max_batch < 1) return RAD_MLP_EINVAL;
    *out = nullptr;
    for (int l = 0; l <= n_layers; ++l)
        if (widths[l] < 128 || widths[l] % 128) return RAD_MLP_EINVAL;
    rad_mlp* m = new (std::nothrow) rad_mlp();
    if (!m) return RAD_MLP_ENOMEM;
    m->L = n_layers;
    m->w.assign(widths, widths + n_layers + 1);
    m->max_rows = round128(max_batch);
    m->st = (cudaStream_t)stream;
    auto bail = [&](int rc) {
        rad_mlp_destroy(m);
        return rc;
    };
#define MAL(ptr, bytes)                                                          \
    do {                                                                         \
        cudaError_t e_ = cudaMalloc(&(ptr), (bytes));                            \
        if (e_ != cudaSuccess) return bail(e_ == cudaErrorMemoryAllocation ? RAD_MLP_ENOMEM : RAD_MLP_ECUDA); \
        cudaMemset((ptr), 0, (bytes));                                           \
    } while (0)
    const int R = m->max_rows;
    m->W.assign(n_layers, nullptr);
    m->b = m->Wm = m->Wv = m->bm = m->bv = m->dW = m->db = m->W;
    m->Wb.assign(n_layers, nullptr);
    m->h.assign(n_layers + 1, nullptr);
    m->z.assign(n_layers + 1, nullptr);
    m->gb.assign(n_layers + 1, nullptr);
    for (int l = 0; l < n_layers; ++l) {
        const size_t np = (size_t)m->w[l + 1] * m->w[l];
        MAL(m->W[l], np * 4);
        MAL(m->Wm[l], np * 4);
        MAL(m->Wv[l], np * 4);
        MAL(m->dW[l], np * 4);
        MAL(m->Wb[l], np * 2);
        MAL(m->b[l], (size_t)m->w[l + 1] * 4);
        MAL(m->bm[l], (size_t)m->w[l + 1] * 4);
        MAL(m->bv[l], (size_t)m->w[l + 1] * 4);
        MAL(m->db[l], (size_t)m->w[l + 1] * 4);
    }
    for (int l = 0; l <= n_layers; ++l) {
        MAL(m->h[l], (size_t)R * m->w[l] * 2);
        if (l >= 1) {
            MAL(m->z[l], (size_t)R * m->w[l] * 4);
            MAL(m->gb[l], (size_t)R * m->w[l] * 2);
        }
    }
    MAL(m->t, (size_t)R * m->w[n_layers] * 4);
    MAL(m->g, (size_t)R * m->w[n_layers] * 4);
    MAL(m->loss, sizeof(double));
    MAL(m->xin, (size_t)R * m->w[0] * 4);
    // split-K scratch: the forward and input-gradient products are R rows wide
    // (the weight gradient reduces over R itself and never splits)
    size_t work = 0;
    for (int l = 0; l < n_layers; ++l) {
        const int in = m->w[l], outw = m->w[l + 1];
        for (int rows = 128; rows <= R; rows += 128) {
            work = std::max(work, (size_t)split_count(rows, outw, in) * rows * outw);
            if (l > 0) work = std::max(work, (size_t)split_count(rows, in, outw) * rows * in);
        }
    }
    MAL(m->work, work * 4);
#undef MAL
    if (cudaDeviceSynchronize() != cudaSuccess) return bail(RAD_MLP_ECUDA);
    *out = m;
    return RAD_MLP_OK;
}

int rad_mlp_set_layer(rad_mlp* m, int32_t layer, const float* W, const float* b)
{
    if (!m || layer < 0 || layer >= m->L || !W || !b) return RAD_MLP_EINVAL;
    const size_t np = (size_t)m->w[layer + 1] * m->w[layer];
    MCU(cudaMemcpyAsync(m->W[layer], W, np * 4, cudaMemcpyDefault, m->st));
    MCU(cudaMemcpyAsync(m->b[layer], b, (size_t)m->w[layer + 1] * 4, cudaMemcpyDefault, m->st));
    f32_to_bf16<<<grid_for(np), 256, 0, m->st>>>(m->W[layer], m->Wb[layer], (int64_t)np);
    MCU(cudaGetLastError());
    // a new parameter set restarts the optimiser
    MCU(cudaMemsetAsync(m->Wm[layer], 0, np * 4, m->st));
    MCU(cudaMemsetAsync(m->Wv[layer], 0, np * 4, m->st));
    MCU(cudaMemsetAsync(m->bm[layer], 0, (size_t)m->w[layer + 1] * 4, m->st));
    MCU(cudaMemsetAsync(m->bv[layer], 0, (size_t)m->w[layer + 1] * 4, m->st));
    m->step = 0;
    MCU(cudaStreamSynchronize(m->st));
    return RAD_MLP_OK;
}

int rad_mlp_get_layer(rad_mlp* m, int32_t layer, float* W, float* b, float* dW, float* db)
{
    if (!m || layer < 0 || layer >= m->L) return RAD_MLP_EINVAL;
    const size_t np = (size_t)m->w[layer + 1] * m->w[layer];
    const size_t nb = (size_t)m->w[layer + 1] * 4;
    if (W) MCU(cudaMemcpyAsync(W, m->W[layer], np * 4, cudaMemcpyDefault, m->st));
    if (b) MCU(cudaMemcpyAsync(b, m->b[layer], nb, cudaMemcpyDefault, m->st));
    if (dW) MCU(cudaMemcpyAsync(dW, m->dW[layer], np * 4, cudaMemcpyDefault, m->st));
    if (db) MCU(cudaMemcpyAsync(db, m->db[layer], nb, cudaMemcpyDefault, m->st));
    MCU(cudaStreamSynchronize(m->st));
    return RAD_MLP_OK;
}

static int forward(rad_mlp* m, int32_t batch, const float* x)
{
    const int R = round128(batch);
    const float* xd = x;
    if (!is_dev(x)) {
        MCU(cudaMemcpyAsync(m->xin, x, (size_t)batch * m->w[0] * 4, cudaMemcpyHostToDevice, m->st));
        xd = m->xin;
    }
    to_bf16_rows<<<grid_for((int64_t)R * m->w[0]), 256, 0, m->st>>>(xd, m->h[0], batch, R, m->w[0]);
    MCU(cudaGetLastError());
    for (int l = 0; l < m->L; ++l) {
        const bool last = l == m->L - 1;
        Epilogue ep{m->b[l], nullptr, m->z[l + 1], last ? nullptr : m->h[l + 1], 1};
        // z = h W^T + b: A = h [R][in], B = W [out][in]
        MCU((gemm<true, true>(m->h[l], m->Wb[l], R, m->w[l + 1], m->w[l], m->w[l], m->w[l], ep, m->st,
                              m->work)));
    }
    return RAD_MLP_OK;
}

int rad_mlp_forward(rad_mlp* m, int32_t batch, const float* x, float* y)
{
    if (!m || batch < 1 || batch > m->max_rows || !x || !y) return RAD_MLP_EINVAL;
    int rc = forward(m, batch, x);
    if (rc) return rc;
    MCU(cudaMemcpyAsync(y, m->z[m->L], (size_t)batch * m->w[m->L] * 4, cudaMemcpyDefault, m->st));
    MCU(cudaStreamSynchronize(m->st));
    return RAD_MLP_OK;
}

int rad_mlp_gradients(rad_mlp* m, int32_t batch, const float* x, const float* t, double* loss)
{
    if (!m || batch < 1 || batch > m->max_rows || !x || !t) return RAD_MLP_EINVAL;
    const int R = round128(batch);
    int rc = forward(m, batch, x);
    if (rc) return rc;
    const int L = m->L, wo = m->w[L];
    MCU(cudaMemcpyAsync(m->t, t, (size_t)batch * wo * 4, cudaMemcpyDefault, m->st));
    MCU(cudaMemsetAsync(m->loss, 0, sizeof(double), m->st));
    mse_grad<<<grid_for((int64_t)R * wo), 256, 0, m->st>>>(m->z[L], m->t, m->g, m->gb[L], m->loss,
                                                           batch, R, wo);
    MCU(cudaGetLastError());
    for (int l = L - 1; l >= 0; --l) {
        const int in = m->w[l], outw = m->w[l + 1];
        // dW = G^T H: A = G stored [R][out] (M = out contiguous), B = H stored [R][in]
        Epilogue ew{nullptr, nullptr, m->dW[l], nullptr, 0};
        MCU((gemm<false, false>(m->gb[l + 1], m->h[l], outw, in, R, outw, in, ew, m->st)));
        // db of the output layer: column sums of the FP32 output gradient (the
        // hidden layers' bias gradients follow below, from the FP32 masked products)
        if (l == L - 1) {
            column_sums<<<grid_for(outw), 256, 0, m->st>>>(m->g, m->db[l], R, outw);
            MCU(cudaGetLastError());
        }
        if (l > 0) {
            // G_prev = (G W) * [z_l > 0]: A = G [R][out] (K = out contiguous), B = W [out][in]
            // stored [K][N]; the FP32 product lands in z_l's buffer for the bias sum
            Epilogue eg{nullptr, m->z[l], m->z[l], m->gb[l], 0};
            MCU((gemm<true, false>(m->gb[l + 1], m->Wb[l], R, in, outw, outw, in, eg, m->st,
                                   m->work)));
        }
    }
    // bias gradients of the hidden layers: column sums of the FP32 masked products
    for (int l = L - 2; l >= 0; --l) {
        column_sums<<<grid_for(m->w[l + 1]), 256, 0, m->st>>>(m->z[l + 1], m->db[l], R, m->w[l + 1]);
        MCU(cudaGetLastError());
    }
    if (loss) MCU(cudaMemcpyAsync(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->st));
    MCU(cudaStreamSynchronize(m->st));
    return RAD_MLP_OK;
}

int rad_mlp_adam(rad_mlp* m, float lr, float beta1, float beta2, float eps)
{
    if (!m || !(lr > 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f))
        return RAD_MLP_EINVAL;
    m->step += 1;
    const float c1 = 1.0f - std::pow(beta1, (float)m->step);
    const float c2 = 1.0f - std::pow(beta2, (float)m->step);
    for (int l = 0; l < m->L; ++l) {
        const int64_t np = (int64_t)m->w[l + 1] * m->w[l];
        adam_update<<<grid_for(np), 256, 0, m->st>>>(m->W[l], m->Wb[l], m->Wm[l], m->Wv[l], m->dW[l],
                                                     np, lr, beta1, beta2, eps, c1, c2);
        adam_update<<<grid_for(m->w[l + 1]), 256, 0, m->st>>>(m->b[l], nullptr, m->bm[l], m->bv[l],
                                                              m->db[l], m->w[l + 1], lr, beta1,
                                                              beta2, eps, c1, c2);
        MCU(cudaGetLastError());
    }
    return RAD_MLP_OK;
}

int rad_mlp_gemm(int32_t AK, int32_t BK, int32_t M, int32_t N, int32_t K, const void* A,
                      const void* B, float* C)
{
    if (M < 1 || N < 1 || K < 1 || M % TM || N % TN || K % TK || !A || !B || !C)
        return RAD_MLP_EINVAL;
    Epilogue ep{nullptr, nullptr, C, nullptr, 0};
    const bf16* a = static_cast<const bf16*>(A);
    const bf16* b = static_cast<const bf16*>(B);
    // split-K scratch from the stream-ordered pool of the default stream
    float* work = nullptr;
    const int S = split_count(M, N, K);
    if (S > 1 && cudaMallocAsync(&work, (size_t)S * M * N * 4, nullptr) != cudaSuccess) {
        cudaGetLastError();
        return RAD_MLP_ENOMEM;
    }
    cudaError_t e;
    const int lda = AK ? K : M, ldb = BK ? K : N;
    if (AK && BK) e = gemm<true, true>(a, b, M, N, K, lda, ldb, ep, nullptr, work);
    else if (AK) e = gemm<true, false>(a, b, M, N, K, lda, ldb, ep, nullptr, work);
    else if (BK) e = gemm<false, true>(a, b, M, N, K, lda, ldb, ep, nullptr, work);
    else e = gemm<false, false>(a, b, M, N, K, lda, ldb, ep, nullptr, work);
    if (work) cudaFreeAsync(work, nullptr);
    if (e == cudaErrorInvalidValue) return RAD_MLP_EINVAL;
    return e == cudaSuccess ? RAD_MLP_OK : RAD_MLP_ECUDA;
}

void rad_mlp_destroy(rad_mlp* m)
{
    if (!m) return;
    if (m->st) cudaStreamSynchronize(m->st);
    for (auto* vv : {&m->W, &m->b, &m->Wm, &m->Wv, &m->bm, &m->bv, &m->dW, &m->db, &m->z})
        for (float* p : *vv)
            if (p) cudaFree(p);
    for (auto* vv : {&m->Wb, &m->h, &m->gb})
        for (bf16* p : *vv)
            if (p) cudaFree(p);
    for (void* p : {(void*)m->t, (void*)m->g, (void*)m->loss, (void*)m->xin, (void*)m->work})
        if (p) cudaFree(p);
    delete m;
}

}  // extern "C"
