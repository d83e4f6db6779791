// rad_mlp.cu -- the learned surrogate's network: a ReLU MLP with BF16 weights
// (FP32 master copy), BF16 GEMM operands and FP32 accumulation, trained with
// MSE and Adam, entirely on the device (C ABI in include/rad_mlp.h).
//
// GEMMs run on the 5th-generation tensor cores: one persistent kernel computes
// C = A B^T for K-contiguous BF16 operands A [M][K], B [N][K], one block of ten
// warps per SM taking 128 x 128 output tiles in turn:
//   * warp 0, one lane: TMA (cp.async.bulk.tensor.2d) loads of 128 x 64 tiles
//     of A and B in the 128-byte-swizzled layout into a five-stage ring,
//     completion on mbarriers;
//   * warp 1, one lane: four tcgen05.mma (kind::f16, BF16 x BF16 -> FP32,
//     M 128, N 128, K 16) per stage into one of two 128-column accumulators in
//     tensor memory (tiles alternate); tcgen05.commit frees the stage and,
//     after a tile's last stage, hands the accumulator to the epilogue;
//   * warps 2-9: tcgen05.ld of 32 accumulator rows x 64 columns each, a
//     transpose through shared memory into row-contiguous groups, the fused
//     epilogue (bias, ReLU, ReLU mask of the backward pass, FP32 and/or BF16
//     output) and coalesced global stores, after which the accumulator goes
//     back to warp 1 -- so a tile's epilogue overlaps the next tile's loads
//     and MMAs.
// Products with few output tiles and a long K (the input gradient of the wide
// output layer: 128 x 512 outputs over K = 393,216) split K across blocks:
// each slice writes raw FP32 partial sums and one reduction kernel adds the
// slices in a fixed order and applies the epilogue, so the result does not
// depend on scheduling.  The forward product X W^T reads its operands in
// place; the input gradient G W reads a BF16 copy of W^T (refreshed with W),
// the weight gradient G^T H reads transposed copies of G and H made per step.
// Every wait on an mbarrier is bounded; on expiry the block raises an error
// word, drains what it issued and releases its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>
#include <new>
#include <vector>

#include "rad_internal.cuh"
#include "rad_mlp.h"

namespace {

typedef __nv_bfloat16 bf16;
using rad::smem_addr;

constexpr int BM = 128, BN = 128, BK = 64;   // block tile; BK x 2 B = one 128-byte swizzle row
constexpr int kStages = 5;                   // TMA -> MMA pipeline depth
constexpr int kEpiWarps = 8;                 // epilogue warps: two per 32 TMEM lanes, each
                                             // storing half of the tile's columns
constexpr int kGemmThreads = (2 + kEpiWarps) * 32;   // TMA warp, MMA warp, epilogue warps
constexpr uint32_t kTileBytes = BM * BK * 2;               // 16 KB per operand per stage
constexpr uint32_t kStageBytes = 2 * kTileBytes;
constexpr uint32_t kTmemCols = 2 * BN;                     // two FP32 128 x 128 accumulators
constexpr size_t kEpiBytes = kEpiWarps * 32 * 32 * sizeof(float);   // transpose staging
constexpr size_t kGemmSmem = kStages * kStageBytes + kEpiBytes + 1024 /* alignment */ +
                             256 /* barriers */;
constexpr int kMinSplitTiles = 4;            // K tiles (of 64) per slice at least

// Streaming multiprocessors of the current device (the persistent GEMM runs one
// block on each).
int device_sms()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
        cudaGetLastError();
        return 1;
    }
    return n;
}

// tcgen05 instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1),
// A and B BF16 (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N / 8 in bits 17-22, M / 16 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

// Text of the last failure of a rad_mlp_* call on this host thread.
thread_local char g_last_error[256] = "";

int fail(int rc, const char* what, cudaError_t e = cudaSuccess)
{
    if (e != cudaSuccess)
        snprintf(g_last_error, sizeof g_last_error, "%s: %s", what, cudaGetErrorString(e));
    else
        snprintf(g_last_error, sizeof g_last_error, "%s", what);
    return rc;
}

// Raised (bit rad::kErrTimeout) by a GEMM block whose bounded wait expired.
__device__ int g_gemm_err;

int* gemm_err_word()
{
    void* p = nullptr;
    return cudaGetSymbolAddress(&p, g_gemm_err) == cudaSuccess ? static_cast<int*>(p) : nullptr;
}

// Reads and clears the error word (after the stream has been synchronised).
bool gemm_timed_out()
{
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_gemm_err, sizeof(int)) != cudaSuccess) return true;
    if (v) {
        const int zero = 0;
        cudaMemcpyToSymbol(g_gemm_err, &zero, sizeof(int));
    }
    return v != 0;
}

struct Epilogue {
    const float* bias;      // [N] or null
    const float* mask;      // [M][N] (z of the backward pass: keep where > 0) or null
    float* out_f32;         // [M][N] or null
    bf16* out_bf16;         // [M][N] or null
    int relu;               // apply ReLU before the BF16 store
};

// Number of K slices for an M x N x K product: enough tiles to fill the GPU
// twice over when the output alone gives too few, each slice kMinSplitTiles
// K tiles or more.
int split_count(int M, int N, int K)
{
    const int blocks = (M / BM) * (N / BN), nk = K / BK, target = 2 * device_sms();
    if (blocks >= target / 2) return 1;
    const int want = (target + blocks - 1) / blocks;
    return std::max(1, std::min(want, nk / kMinSplitTiles));
}

// Shared-memory matrix descriptor of a K-major operand tile stored by TMA with
// 128-byte swizzling: rows of 128 B, 8-row groups 1024 B apart (stride byte
// offset), leading byte offset unused for this layout (1), descriptor version
// 1 (bit 46), layout SWIZZLE_128B (2 in bits 61-63).  The tile base is 1024-B
// aligned; the k-th 16-element slice starts 32 k bytes further.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) |
           ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

// Arrives on bar once every tcgen05.mma this thread issued before has completed.
__device__ __forceinline__ void umma_commit(uint64_t* bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// Output tile t of C = A B^T (split into S slices along K): slice z, row tile
// mi, column tile ni, K tiles [kt0, kt1).  Column tiles vary fastest, so the
// blocks working at the same time share their A tile in L2.
struct TileCoord {
    int z, m0, n0, kt0, kt1;
};

__device__ __forceinline__ TileCoord tile_coord(int t, int M, int N, int K, int S)
{
    const int mt = M / BM, ntl = N / BN, nk_all = K / BK;
    const int z = t / (mt * ntl), rem = t - z * mt * ntl;
    TileCoord c;
    c.z = z;
    c.m0 = (rem / ntl) * BM;
    c.n0 = (rem % ntl) * BN;
    c.kt0 = (int)((int64_t)nk_all * z / S);
    c.kt1 = (int)((int64_t)nk_all * (z + 1) / S);
    return c;
}

// C = A B^T, persistent: block b takes output tiles b, b + gridDim.x, ...
// Warp 0 (one lane) streams A and B tiles by TMA into a kStages-deep ring of
// shared-memory stages; warp 1 (one lane) issues the tcgen05 MMAs of a tile
// into one of two TMEM accumulators and commits it; warps 2-9 drain the other
// accumulator through the epilogue (two warps per 32-row quarter, 64 columns
// each), so that a tile's epilogue overlaps the next tile's loads and MMAs.  A and B come through the tensor maps (K
// innermost, box 64 x 128, 128-byte swizzle).  Every wait is bounded: an
// expired wait raises the block's abort flag and err_word, every role leaves
// its loop, the TMA warp waits for its loads in flight and the MMA warp for its
// MMAs before the accumulators are released.
__global__ void __launch_bounds__(kGemmThreads, 1) umma_gemm_kernel(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M,
    int N, int K, int S, Epilogue ep, float* partial, int* err_word)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float* epi = reinterpret_cast<float*>(base + kStages * kStageBytes);
    uint64_t* full = reinterpret_cast<uint64_t*>(base + kStages * kStageBytes + kEpiBytes);
    uint64_t* empty = full + kStages;
    uint64_t* tfull = empty + kStages;    // [2] accumulator b holds a finished tile
    uint64_t* tempty = tfull + 2;         // [2] accumulator b has been drained
    uint64_t* mdone = tempty + 2;         // every MMA issued by this block is done
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mdone + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles = (M / BM) * (N / BN) * S;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            rad::mbar_init(&full[s], 1);
            rad::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            rad::mbar_init(&tfull[b], 1);
            rad::mbar_init(&tempty[b], kEpiWarps);
        }
        rad::mbar_init(mdone, 1);
        *abort_flag = 0;
        rad::fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer: stage use counter `it` runs across tiles
            uint32_t it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
                const TileCoord tc = tile_coord(t, M, N, K, S);
                for (int kt = tc.kt0; kt < tc.kt1; ++kt, ++it) {
                    const int s = (int)(it % kStages);
                    const uint32_t u = it / kStages;
                    if (it >= (uint32_t)kStages &&
                        !rad::mbar_wait_bounded(&empty[s], (u - 1) & 1, abort_flag, err_word)) {
                        ok = false;
                        break;
                    }
                    rad::mbar_arrive_expect_tx(&full[s], kStageBytes);
                    unsigned char* st = base + s * kStageBytes;
                    tma_load_2d(st, &tmA, kt * BK, tc.m0, &full[s]);
                    tma_load_2d(st + kTileBytes, &tmB, kt * BK, tc.n0, &full[s]);
                }
            }
            if (!ok || *abort_flag) {
                // never leave with a copy in flight: wait (bounded) for the last
                // kStages issued loads to land
                for (uint32_t j = it > (uint32_t)kStages ? it - kStages : 0; j < it; ++j)
                    rad::mbar_drain(&full[j % kStages], (j / kStages) & 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer: tile i of this block goes to accumulator i & 1
            uint32_t it = 0, i = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++i) {
                const TileCoord tc = tile_coord(t, M, N, K, S);
                const int ab = (int)(i & 1);
                const uint32_t use = i >> 1;
                if (use >= 1 &&
                    !rad::mbar_wait_bounded(&tempty[ab], (use - 1) & 1, abort_flag, err_word))
                    break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(ab * BN);
                for (int kt = tc.kt0; kt < tc.kt1; ++kt, ++it) {
                    const int s = (int)(it % kStages);
                    const uint32_t u = it / kStages;
                    if (!rad::mbar_wait_bounded(&full[s], u & 1, abort_flag, err_word)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = smem_addr(base + s * kStageBytes);
                    const uint32_t b0 = a0 + kTileBytes;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk)
                        umma_bf16(d, sw128_desc(a0 + 32 * kk), sw128_desc(b0 + 32 * kk),
                                  (kt > tc.kt0 || kk > 0) ? 1u : 0u);
                    umma_commit(&empty[s]);
                }
                if (ok) umma_commit(&tfull[ab]);
            }
            // completes once every MMA issued above is done (also after an abort)
            umma_commit(mdone);
            rad::mbar_drain(mdone, 0);
        }
    } else {
        // ---- epilogue: warp w may read TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31,
        // the accumulator rows of that quarter; warps 2-5 take columns 0-63 and
        // warps 6-9 columns 64-127.  Each 32 x 32 block goes TMEM ->
        // registers (one row per lane) -> this warp's staging (float4 slots
        // XOR-swizzled by row, conflict-free both ways) -> registers (four
        // consecutive columns per lane, eight lanes per row), so every global
        // access of a warp covers four whole 128-byte row segments.
        const int lg = warp & 3, cbase = ((warp - 2) >> 2) * (BN / 2);
        float* stage = epi + (warp - 2) * 32 * 32;
        const int qi = lane & 7, ri = lane >> 3;
        uint32_t i = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++i) {
            const TileCoord tc = tile_coord(t, M, N, K, S);
            const int ab = (int)(i & 1);
            const bool ready = rad::mbar_wait_bounded(&tfull[ab], (i >> 1) & 1, abort_flag, err_word);
            // tcgen05.ld below is warp-collective: the whole warp goes on or stops
            if (!__all_sync(0xffffffffu, ready && !*abort_flag)) break;
            tc_fence_after();
#pragma unroll 1
            for (int c0 = cbase; c0 < cbase + BN / 2; c0 += 32) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(ab * BN + c0), v);
                float4* srow = reinterpret_cast<float4*>(stage + lane * 32);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    srow[j ^ (lane & 7)] =
                        make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                __syncwarp();
#pragma unroll 2
                for (int k = 0; k < 8; ++k) {
                    const int r = 4 * k + ri;
                    float4 x = reinterpret_cast<const float4*>(stage + r * 32)[qi ^ (r & 7)];
                    const int n = tc.n0 + c0 + 4 * qi;
                    const size_t o = (size_t)(tc.m0 + lg * 32 + r) * N + n;
                    if (partial) {
                        *reinterpret_cast<float4*>(partial + (size_t)tc.z * M * N + o) = x;
                        continue;
                    }
                    if (ep.bias) {
                        const float4 b = *reinterpret_cast<const float4*>(ep.bias + n);
                        x.x += b.x;
                        x.y += b.y;
                        x.z += b.z;
                        x.w += b.w;
                    }
                    if (ep.mask) {
                        const float4 q = *reinterpret_cast<const float4*>(ep.mask + o);
                        x.x = q.x > 0.0f ? x.x : 0.0f;
                        x.y = q.y > 0.0f ? x.y : 0.0f;
                        x.z = q.z > 0.0f ? x.z : 0.0f;
                        x.w = q.w > 0.0f ? x.w : 0.0f;
                    }
                    if (ep.out_f32) *reinterpret_cast<float4*>(ep.out_f32 + o) = x;
                    if (ep.out_bf16) {
                        if (ep.relu) {
                            x.x = fmaxf(x.x, 0.0f);
                            x.y = fmaxf(x.y, 0.0f);
                            x.z = fmaxf(x.z, 0.0f);
                            x.w = fmaxf(x.w, 0.0f);
                        }
                        const __nv_bfloat162 lo = __floats2bfloat162_rn(x.x, x.y);
                        const __nv_bfloat162 hi = __floats2bfloat162_rn(x.z, x.w);
                        *reinterpret_cast<uint2*>(ep.out_bf16 + o) =
                            make_uint2(*reinterpret_cast<const uint32_t*>(&lo),
                                       *reinterpret_cast<const uint32_t*>(&hi));
                    }
                }
                __syncwarp();
            }
            // this warp's reads of the accumulator are complete: hand it back
            tc_fence_before();
            __syncwarp();
            if (lane == 0) rad::mbar_arrive(&tempty[ab]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
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

// out [cols][rows] = in [rows][cols]^T (BF16), 32 x 32 tiles through shared memory.
__global__ void transpose_bf16(const bf16* __restrict__ in, bf16* __restrict__ out, int rows,
                               int cols)
{
    __shared__ bf16 t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        if (r < rows && c < cols) t[i][threadIdx.x] = in[(size_t)r * cols + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[(size_t)c * rows + r] = t[threadIdx.x][i];
    }
}

cudaError_t transpose(const bf16* in, bf16* out, int rows, int cols, cudaStream_t st)
{
    dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
    transpose_bf16<<<grid, block, 0, st>>>(in, out, rows, cols);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) fail(RAD_MLP_ECUDA, "transpose: launch", e);
    return e;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// Row-major BF16 [rows][ld] viewed as rows x cols, K (= cols) innermost; box
// 64 x 128, 128-byte swizzle.
bool make_map(CUtensorMap* map, const bf16* ptr, int rows, int cols, int ld)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(bf16)};
    const cuuint32_t box[2] = {BK, BM};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(ptr), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// C [M][N] = A [M][K] B [N][K]^T with the fused epilogue.  work: FP32 scratch
// of at least split_count(M, N, K) * M * N floats, or null to run unsplit.
cudaError_t gemm_tn(const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K,
                    const Epilogue& ep, cudaStream_t st, float* work, int* err_word)
{
    if (M % BM || N % BN || K % BK || K < BK || lda % 8 || ldb % 8 || lda < K || ldb < K ||
        (reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) % 16 || !err_word) {
        fail(RAD_MLP_EINVAL, "gemm: shape, leading dimension or alignment not supported");
        return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaFuncSetAttribute(umma_gemm_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kGemmSmem);
    if (e != cudaSuccess) {
        fail(RAD_MLP_ECUDA, "gemm: shared-memory attribute", e);
        return e;
    }
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, M, K, lda) || !make_map(&mb, B, N, K, ldb)) {
        fail(RAD_MLP_EINVAL, "gemm: tensor map encoding failed");
        return cudaErrorInvalidValue;
    }
    const int S = work ? split_count(M, N, K) : 1;
    const int tiles = (M / BM) * (N / BN) * S, sms = device_sms();
    umma_gemm_kernel<<<std::min(tiles, sms), kGemmThreads, kGemmSmem, st>>>(
        ma, mb, M, N, K, S, ep, S > 1 ? work : nullptr, err_word);
    if (S > 1) {
        const int64_t n4 = (int64_t)M * N / 4;
        const int blocks = (int)std::min<int64_t>((n4 + 255) / 256, 4 * sms);
        splitk_reduce<<<blocks, 256, 0, st>>>(work, S, M, N, ep);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) fail(RAD_MLP_ECUDA, "gemm: launch", e);
    return e;
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

// Input transform of rad_mlp_predict: h0 = BF16((log10(max(x, floor)) - mu) / sd)
// per feature (padded rows zero).
__global__ void log_standardise_rows(const float* __restrict__ x, bf16* __restrict__ y,
                                     const float* __restrict__ mu, const float* __restrict__ sd,
                                     float floor_v, int rows_valid, int rows, int cols)
{
    const int64_t n = (int64_t)rows * cols;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / cols), c = (int)(i - (int64_t)r * cols);
        float v = 0.0f;
        if (r < rows_valid) v = (log10f(fmaxf(x[i], floor_v)) - mu[c]) / sd[c];
        y[i] = __float2bfloat16_rn(v);
    }
}

// Output transform of rad_mlp_predict: y = 10^(z sd + mu) per feature.
__global__ void exp10_affine_rows(const float* __restrict__ z, float* __restrict__ y,
                                  const float* __restrict__ mu, const float* __restrict__ sd,
                                  int rows_valid, int cols)
{
    const int64_t n = (int64_t)rows_valid * cols;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % cols);
        y[i] = exp10f(fmaf(z[i], sd[c], mu[c]));
    }
}

// MSE over the valid rows, loss = sum (y - t)^2 / (rows_valid * cols), and its
// gradient g = 2 (y - t) / (rows_valid * cols) (FP32 and BF16; zero on padded rows).
// In 32 x 32 tiles, also writing BF16 G^T [cols][rows]
// (the weight-gradient operand) through shared memory; each block's share of
// the loss (FP32 within the block) goes to part[block] and is summed in FP64,
// in a fixed order, by loss_sum.
__global__ void __launch_bounds__(256) mse_tile(const float* __restrict__ y,
                                                const float* __restrict__ t,
                                                float* __restrict__ g, bf16* __restrict__ gb,
                                                bf16* __restrict__ gbt,
                                                double* __restrict__ part, float scale,
                                                int rows_valid, int rows, int cols)
{
    // scale = 2 / (rows_valid * cols), rounded once on the host: this kernel
    // issues no FP64 arithmetic (the FP64 pipe is 1/64 of FP32 here), only
    // the per-block share is widened
    __shared__ bf16 tr[32][33];
    __shared__ float red[8];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32, c = c0 + threadIdx.x;
    // rows threadIdx.y + 8 q of the tile: all loads first, then the stores
    float d[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int r = r0 + threadIdx.y + 8 * q;
        const size_t k = (size_t)r * cols + c;
        d[q] = (r < rows_valid && c < cols) ? y[k] - t[k] : 0.0f;
    }
    float acc = 0.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = threadIdx.y + 8 * q, r = r0 + i;
        const float gi = scale * d[q];
        acc = fmaf(d[q], d[q], acc);
        const bf16 h = __float2bfloat16_rn(gi);
        if (r < rows && c < cols) {
            const size_t k = (size_t)r * cols + c;
            g[k] = gi;
            gb[k] = h;
        }
        tr[i][threadIdx.x] = h;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) red[threadIdx.y] = acc;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        float b = 0.0f;
        for (int w = 0; w < 8; ++w) b += red[w];
        part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = (double)b;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = threadIdx.y + 8 * q, cc = c0 + i, r = r0 + threadIdx.x;
        if (r < rows && cc < cols) gbt[(size_t)cc * rows + r] = tr[threadIdx.x][i];
    }
}

// loss = sum of the n block shares / (rows_valid * cols), one block, fixed order.
__global__ void loss_sum(const double* part, int64_t n, double inv, double* loss)
{
    __shared__ double red[256];
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a += part[i];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0] * inv;
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

// The same Adam step for a weight matrix W [rows][cols] in 32 x 32 tiles, also
// writing the BF16 copy of W and, through shared memory, of W^T [cols][rows]:
// one pass over the optimiser state instead of a second one for the transpose.
__global__ void __launch_bounds__(256) adam_tile(float* __restrict__ w, bf16* __restrict__ wb,
                                                 bf16* __restrict__ wbt, float* __restrict__ m,
                                                 float* __restrict__ v,
                                                 const float* __restrict__ g, int rows, int cols,
                                                 float lr, float b1, float b2, float eps, float c1,
                                                 float c2)
{
    __shared__ bf16 t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const int c = c0 + threadIdx.x;
    // rows threadIdx.y + 8 q of the tile: all loads first, then the update
    float gq[4], mq[4], vq[4], wq[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int r = r0 + threadIdx.y + 8 * q;
        const bool in = r < rows && c < cols;
        const size_t k = (size_t)r * cols + c;
        gq[q] = in ? g[k] : 0.0f;
        mq[q] = in ? m[k] : 0.0f;
        vq[q] = in ? v[k] : 0.0f;
        wq[q] = in ? w[k] : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = threadIdx.y + 8 * q, r = r0 + i;
        const float gi = gq[q];
        const float mi = b1 * mq[q] + (1.0f - b1) * gi;
        const float vi = b2 * vq[q] + (1.0f - b2) * gi * gi;
        const float wi = wq[q] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        const bf16 h = __float2bfloat16_rn(wi);
        if (r < rows && c < cols) {
            const size_t k = (size_t)r * cols + c;
            m[k] = mi;
            v[k] = vi;
            w[k] = wi;
            wb[k] = h;
        }
        t[i][threadIdx.x] = h;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = threadIdx.y + 8 * q, cc = c0 + i, r = r0 + threadIdx.x;
        if (r < rows && cc < cols) wbt[(size_t)cc * rows + r] = t[threadIdx.x][i];
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
    std::vector<bf16*> Wb;          // BF16 copy of W [out][in] (forward operand)
    std::vector<bf16*> Wbt;         // BF16 copy of W^T [in][out] (input-gradient operand)
    int64_t step = 0;
    // activations: h[l] bf16 [rows][w[l]] (h[0] = input), z[l] fp32 [rows][w[l]] (l >= 1)
    std::vector<bf16*> h;
    std::vector<float*> z;
    float* t = nullptr;             // targets [rows][w[L]]
    float* g = nullptr;             // output gradient fp32 [rows][w[L]]
    std::vector<bf16*> gb;          // layer gradients bf16: gb[l] [rows][w[l]] for l >= 1
    double* loss = nullptr;
    double* loss_part = nullptr;    // per-block loss shares of mse_tile
    float* xin = nullptr;           // staging for host inputs [rows][w[0]]
    float* work = nullptr;          // split-K partial sums (largest split product)
    float* in_mu = nullptr;         // rad_mlp_predict transforms [w[0]], [w[L]] (null: unset)
    float* in_sd = nullptr;
    float* out_mu = nullptr;
    float* out_sd = nullptr;
    float floor_v = 0.0f;
    float* ypred = nullptr;         // predict output staging [rows][w[L]]
    bf16* gt = nullptr;             // G^T [w][rows] for the weight gradient (largest layer)
    bf16* ht = nullptr;             // H^T [w][rows]
    int* err = nullptr;             // GEMM timeout word
};

#define MCU(call)                                                                  \
    do {                                                                           \
        const cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess)                                                     \
            return e_ == cudaErrorInvalidValue ? fail(RAD_MLP_EINVAL, #call, e_)   \
                                               : fail(RAD_MLP_ECUDA, #call, e_);   \
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
    m->Wbt.assign(n_layers, nullptr);
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
        MAL(m->Wbt[l], np * 2);
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
    MAL(m->loss_part, (size_t)(R / 32) * ((m->w[n_layers] + 31) / 32) * sizeof(double));
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
    int wmax = 0;
    for (int l = 0; l <= n_layers; ++l) wmax = std::max(wmax, m->w[l]);
    MAL(m->gt, (size_t)wmax * R * 2);
    MAL(m->ht, (size_t)wmax * R * 2);
#undef MAL
    m->err = gemm_err_word();
    if (!m->err) return bail(RAD_MLP_ECUDA);
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
    MCU(transpose(m->Wb[layer], m->Wbt[layer], m->w[layer + 1], m->w[layer], m->st));
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

static int forward(rad_mlp* m, int32_t batch, const float* x, bool transform = false)
{
    const int R = round128(batch);
    const float* xd = x;
    if (!is_dev(x)) {
        MCU(cudaMemcpyAsync(m->xin, x, (size_t)batch * m->w[0] * 4, cudaMemcpyHostToDevice, m->st));
        xd = m->xin;
    }
    if (transform)
        log_standardise_rows<<<grid_for((int64_t)R * m->w[0]), 256, 0, m->st>>>(
            xd, m->h[0], m->in_mu, m->in_sd, m->floor_v, batch, R, m->w[0]);
    else
        to_bf16_rows<<<grid_for((int64_t)R * m->w[0]), 256, 0, m->st>>>(xd, m->h[0], batch, R, m->w[0]);
    MCU(cudaGetLastError());
    for (int l = 0; l < m->L; ++l) {
        const bool last = l == m->L - 1;
        Epilogue ep{m->b[l], nullptr, m->z[l + 1], last ? nullptr : m->h[l + 1], 1};
        // z = h W^T + b: A = h [R][in], B = W [out][in]
        MCU(gemm_tn(m->h[l], m->w[l], m->Wb[l], m->w[l], R, m->w[l + 1], m->w[l], ep, m->st,
                    m->work, m->err));
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
    return gemm_timed_out() ? RAD_MLP_ETIMEOUT : RAD_MLP_OK;
}

int rad_mlp_set_transform(rad_mlp* m, const float* in_mu, const float* in_sd, const float* out_mu,
                          const float* out_sd, float floor_value)
{
    if (!m || !in_mu || !in_sd || !out_mu || !out_sd || !(floor_value > 0.0f))
        return fail(RAD_MLP_EINVAL, "rad_mlp_set_transform: null statistics or floor <= 0");
    const int wi = m->w[0], wo = m->w[m->L];
    if (!m->in_mu) {
        MCU(cudaMalloc(&m->in_mu, (size_t)wi * 4));
        MCU(cudaMalloc(&m->in_sd, (size_t)wi * 4));
        MCU(cudaMalloc(&m->out_mu, (size_t)wo * 4));
        MCU(cudaMalloc(&m->out_sd, (size_t)wo * 4));
        MCU(cudaMalloc(&m->ypred, (size_t)m->max_rows * wo * 4));
    }
    MCU(cudaMemcpyAsync(m->in_mu, in_mu, (size_t)wi * 4, cudaMemcpyDefault, m->st));
    MCU(cudaMemcpyAsync(m->in_sd, in_sd, (size_t)wi * 4, cudaMemcpyDefault, m->st));
    MCU(cudaMemcpyAsync(m->out_mu, out_mu, (size_t)wo * 4, cudaMemcpyDefault, m->st));
    MCU(cudaMemcpyAsync(m->out_sd, out_sd, (size_t)wo * 4, cudaMemcpyDefault, m->st));
    MCU(cudaStreamSynchronize(m->st));
    m->floor_v = floor_value;
    return RAD_MLP_OK;
}

int rad_mlp_predict(rad_mlp* m, int32_t batch, const float* x, float* y)
{
    if (!m || batch < 1 || batch > m->max_rows || !x || !y) return RAD_MLP_EINVAL;
    if (!m->in_mu) return fail(RAD_MLP_EINVAL, "rad_mlp_predict: no transform set");
    int rc = forward(m, batch, x, true);
    if (rc) return rc;
    const int wo = m->w[m->L];
    float* yd = is_dev(y) ? y : m->ypred;
    exp10_affine_rows<<<grid_for((int64_t)batch * wo), 256, 0, m->st>>>(m->z[m->L], yd, m->out_mu,
                                                                       m->out_sd, batch, wo);
    MCU(cudaGetLastError());
    if (yd != y)
        MCU(cudaMemcpyAsync(y, yd, (size_t)batch * wo * 4, cudaMemcpyDeviceToHost, m->st));
    MCU(cudaStreamSynchronize(m->st));
    return gemm_timed_out() ? RAD_MLP_ETIMEOUT : RAD_MLP_OK;
}

// Forward, MSE and backward, enqueued on the stream (no host synchronisation).
static int backward(rad_mlp* m, int32_t batch, const float* x, const float* t)
{
    const int R = round128(batch);
    int rc = forward(m, batch, x);
    if (rc) return rc;
    const int L = m->L, wo = m->w[L];
    // device targets are read in place (mse_tile touches only the batch's rows)
    const float* td = t;
    if (!is_dev(t)) {
        MCU(cudaMemcpyAsync(m->t, t, (size_t)batch * wo * 4, cudaMemcpyHostToDevice, m->st));
        td = m->t;
    }
    {
        const dim3 grid((wo + 31) / 32, R / 32);
        mse_tile<<<grid, dim3(32, 8), 0, m->st>>>(m->z[L], td, m->g, m->gb[L], m->gt, m->loss_part,
                                                  (float)(2.0 / ((double)batch * wo)), batch, R,
                                                  wo);
        loss_sum<<<1, 256, 0, m->st>>>(m->loss_part, (int64_t)grid.x * grid.y,
                                       1.0 / ((double)batch * wo), m->loss);
        MCU(cudaGetLastError());
    }
    for (int l = L - 1; l >= 0; --l) {
        const int in = m->w[l], outw = m->w[l + 1];
        // dW = G^T H over the batch: both operands transposed to batch-contiguous
        // copies, G^T [out][R] and H^T [in][R]
        Epilogue ew{nullptr, nullptr, m->dW[l], nullptr, 0};
        if (l < L - 1) MCU(transpose(m->gb[l + 1], m->gt, R, outw, m->st));   // output layer: mse_tile
        MCU(transpose(m->h[l], m->ht, R, in, m->st));
        MCU(gemm_tn(m->gt, R, m->ht, R, outw, in, R, ew, m->st, nullptr, m->err));
        // db of the output layer: column sums of the FP32 output gradient (the
        // hidden layers' bias gradients follow below, from the FP32 masked products)
        if (l == L - 1) {
            column_sums<<<grid_for(outw), 256, 0, m->st>>>(m->g, m->db[l], R, outw);
            MCU(cudaGetLastError());
        }
        if (l > 0) {
            // G_prev = (G W) * [z_l > 0]: A = G [R][out], B = W^T [in][out] (both
            // out-contiguous); the FP32 product lands in z_l's buffer for the bias sum
            Epilogue eg{nullptr, m->z[l], m->z[l], m->gb[l], 0};
            MCU(gemm_tn(m->gb[l + 1], outw, m->Wbt[l], outw, R, in, outw, eg, m->st, m->work,
                        m->err));
        }
    }
    // bias gradients of the hidden layers: column sums of the FP32 masked products
    for (int l = L - 2; l >= 0; --l) {
        column_sums<<<grid_for(m->w[l + 1]), 256, 0, m->st>>>(m->z[l + 1], m->db[l], R, m->w[l + 1]);
        MCU(cudaGetLastError());
    }
    return RAD_MLP_OK;
}

static int finish(rad_mlp* m, double* loss)
{
    if (loss) MCU(cudaMemcpyAsync(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->st));
    MCU(cudaStreamSynchronize(m->st));
    return gemm_timed_out() ? RAD_MLP_ETIMEOUT : RAD_MLP_OK;
}

int rad_mlp_gradients(rad_mlp* m, int32_t batch, const float* x, const float* t, double* loss)
{
    if (!m || batch < 1 || batch > m->max_rows || !x || !t) return RAD_MLP_EINVAL;
    const int rc = backward(m, batch, x, t);
    return rc ? rc : finish(m, loss);
}

// One Adam step of every layer from the stored gradients, enqueued.
static int adam_enqueue(rad_mlp* m, float lr, float beta1, float beta2, float eps)
{
    m->step += 1;
    const float c1 = 1.0f - std::pow(beta1, (float)m->step);
    const float c2 = 1.0f - std::pow(beta2, (float)m->step);
    for (int l = 0; l < m->L; ++l) {
        const int rows = m->w[l + 1], cols = m->w[l];
        adam_tile<<<dim3((cols + 31) / 32, (rows + 31) / 32), dim3(32, 8), 0, m->st>>>(
            m->W[l], m->Wb[l], m->Wbt[l], m->Wm[l], m->Wv[l], m->dW[l], rows, cols, lr, beta1, beta2,
            eps, c1, c2);
        adam_update<<<grid_for(m->w[l + 1]), 256, 0, m->st>>>(m->b[l], nullptr, m->bm[l], m->bv[l],
                                                              m->db[l], m->w[l + 1], lr, beta1,
                                                              beta2, eps, c1, c2);
        MCU(cudaGetLastError());
    }
    return RAD_MLP_OK;
}

static bool adam_args_ok(float lr, float beta1, float beta2)
{
    return lr > 0.0f && beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f;
}

int rad_mlp_adam(rad_mlp* m, float lr, float beta1, float beta2, float eps)
{
    if (!m || !adam_args_ok(lr, beta1, beta2)) return RAD_MLP_EINVAL;
    return adam_enqueue(m, lr, beta1, beta2, eps);
}

int rad_mlp_train_step(rad_mlp* m, int32_t batch, const float* x, const float* t, float lr,
                       float beta1, float beta2, float eps, double* loss)
{
    if (!m || batch < 1 || batch > m->max_rows || !x || !t || !adam_args_ok(lr, beta1, beta2))
        return RAD_MLP_EINVAL;
    int rc = backward(m, batch, x, t);
    if (!rc) rc = adam_enqueue(m, lr, beta1, beta2, eps);
    return rc ? rc : finish(m, loss);
}

int rad_mlp_gemm(int32_t a_kcontig, int32_t b_kcontig, int32_t M, int32_t N, int32_t K, const void* A,
                 const void* B, float* C)
{
    if (M < 1 || N < 1 || K < 1 || M % BM || N % BN || K % BK || !A || !B || !C)
        return fail(RAD_MLP_EINVAL, "rad_mlp_gemm: M, N must be multiples of 128 and K of 64");
    // the kernels load A and B by TMA and write C directly: host memory is
    // refused here instead of faulting inside a launch
    if (!is_dev(A) || !is_dev(B) || !is_dev(C))
        return fail(RAD_MLP_EINVAL, "rad_mlp_gemm: A, B and C must be device or managed memory");
    int* err = gemm_err_word();
    if (!err) return fail(RAD_MLP_ECUDA, "rad_mlp_gemm: error word");
    Epilogue ep{nullptr, nullptr, C, nullptr, 0};
    const bf16* a = static_cast<const bf16*>(A);
    const bf16* b = static_cast<const bf16*>(B);
    // scratch from the default stream's stream-ordered pool: split-K partials
    // and K-contiguous copies of operands stored the other way round
    const int S = split_count(M, N, K);
    const size_t part = S > 1 ? (size_t)S * M * N * 4 : 0;
    const size_t at = a_kcontig ? 0 : (size_t)M * K * 2, bt = b_kcontig ? 0 : (size_t)N * K * 2;
    unsigned char* scratch = nullptr;
    if (part + at + bt &&
        cudaMallocAsync(reinterpret_cast<void**>(&scratch), part + at + bt, nullptr) != cudaSuccess) {
        return fail(RAD_MLP_ENOMEM, "rad_mlp_gemm: scratch", cudaGetLastError());
    }
    float* work = part ? reinterpret_cast<float*>(scratch) : nullptr;
    cudaError_t e = cudaSuccess;
    if (!a_kcontig) {       // A stored [K][M]
        bf16* t = reinterpret_cast<bf16*>(scratch + part);
        e = transpose(a, t, K, M, nullptr);
        a = t;
    }
    if (e == cudaSuccess && !b_kcontig) {       // B stored [K][N]
        bf16* t = reinterpret_cast<bf16*>(scratch + part + at);
        e = transpose(b, t, K, N, nullptr);
        b = t;
    }
    if (e == cudaSuccess) e = gemm_tn(a, K, b, K, M, N, K, ep, nullptr, work, err);
    if (scratch) cudaFreeAsync(scratch, nullptr);
    if (e == cudaErrorInvalidValue) return RAD_MLP_EINVAL;
    return e == cudaSuccess ? RAD_MLP_OK : RAD_MLP_ECUDA;
}

int rad_mlp_check(void)
{
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail(RAD_MLP_ECUDA, "rad_mlp_check", e);
    return gemm_timed_out() ? fail(RAD_MLP_ETIMEOUT, "a GEMM block's bounded wait expired")
                            : RAD_MLP_OK;
}

const char* rad_mlp_last_error(void) { return g_last_error; }

void rad_mlp_destroy(rad_mlp* m)
{
    if (!m) return;
    if (m->st) cudaStreamSynchronize(m->st);
    for (auto* vv : {&m->W, &m->b, &m->Wm, &m->Wv, &m->bm, &m->bv, &m->dW, &m->db, &m->z})
        for (float* p : *vv)
            if (p) cudaFree(p);
    for (auto* vv : {&m->Wb, &m->Wbt, &m->h, &m->gb})
        for (bf16* p : *vv)
            if (p) cudaFree(p);
    for (void* p : {(void*)m->in_mu, (void*)m->in_sd, (void*)m->out_mu, (void*)m->out_sd,
                    (void*)m->ypred})
        if (p) cudaFree(p);
    for (void* p : {(void*)m->t, (void*)m->g, (void*)m->loss, (void*)m->loss_part, (void*)m->xin,
                    (void*)m->work,
                    (void*)m->gt, (void*)m->ht})
        if (p) cudaFree(p);
    delete m;
}

}  // extern "C"
