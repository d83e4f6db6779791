// rad_internal.cuh -- structures and sm_103a device helpers shared by the
// kernels of the radiation-spectrum library (not part of the public ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

struct rad_ctx;   // the radiation context (rad_api.cu)

namespace rad {

// ---------------------------------------------------------------------------
// trajectory ring layout
// ---------------------------------------------------------------------------
// Both rings are tile-major: element (tile, slot, c, p) of particle column
// col = 8 tile + p sits at ((tile * ring + slot) * comps + c) * 8 + p, so the
// chunk of consecutive slots the kernels stage is one contiguous block.
// comps is 10, or 11 when sample selectors are defined (the flags word); the
// precise-phase FP32 path adds dr's lo part as components 11-13 (comps 14).
// FP32 split path: slab[tile][slot][c][p] float, c = 0..9 (10) =
//   dr (3)   : r_m - r_a, the offset from the block's FP64 anchor position
//   beta (3) : beta_m
//   bdot (3) : betadot_m (differenced in FP64 before the rounding)
//   g (1)    : 1/gamma_m^2 = 1/(1 + ubar^2)
//   flags (1): selector bits of the sample (bit i: inside selector i), stored as
//              the float with those bits (FP32 ring) or as an exact double (FP64)
// anc32[tile][blk][c][p] float, c = 0..5: r_a as hi (3) + lo (3) FP32 pairs at
//   the anchor samples a = K * blk (ring of ring/K blocks, tile-major like the
//   samples, so a chunk's anchors are one contiguous block too).
// FP64 path: slab64[tile][slot][c][p] double with c = r (3, absolute unwrapped),
// beta (3), bdot (3), g (1), flags (1).
constexpr int kComps = 11;     // components at most (10 + the selector flags)
constexpr int kCompsPlain = 10;   // without selectors
constexpr int kCompsPrec = 14;    // precise-phase FP32 ring: + flags + the lo part of dr
constexpr int kTileP = 8;      // particles per tile: one warp each
constexpr int kChunk32 = 32;   // samples per TMA chunk, FP32 ring
constexpr int kChunk64 = 16;   // samples per TMA chunk, FP64 ring
constexpr int kComputeWarps = 8;
constexpr int kBlockThreads = (kComputeWarps + 1) * 32;  // + one TMA producer warp
constexpr int kMaxSpecies = 32;

// error word bits
constexpr int kErrTimeout = 1;
constexpr int kErrNaN = 2;

// One unit of accumulation work: a window, a direction, a tile of the
// frequency grid and a run of particle tiles of one species.
struct WorkItem {
    int32_t win;      // window index
    int32_t dir;      // direction index (into the context's directions)
    int32_t ftile;    // frequency tile index within the window's grid
    int32_t sp;       // species index
    int32_t tile0;    // first particle tile (column / 8)
    int32_t ntiles;   // number of particle tiles
    int32_t row;      // output row of the direction in the window's [dirs][len] block
    int32_t kmul;     // FP32 path: phases anchored every K << kmul samples (K: the ring's)
    int32_t prec;     // FP32 path, precise-phase build for chosen items: 1 = this item
};

// Per-window constants the accumulation kernels read.
struct WinDev {
    int64_t s0, s1;      // sample range
    int32_t grid_off;    // offset of the frequency grid in the frequency arrays
    int32_t grid_len;    // frequencies in the grid
    int64_t out_off;     // offset of the window's [dirs][len] block in the accumulators
    int32_t sel;         // selector bit the samples must have, or -1 (all samples)
    int32_t pad_;
};

// A sample selector evaluated at ingest (positions as handed over, ubar).
constexpr int kMaxSelectors = 32;
struct SelectorDev {
    int32_t kind;        // 1: box, 2: cone
    int32_t pad_;
    double lo[3], hi[3]; // box: lo <= x < hi per component
    double axis[3];      // cone: unit axis
    double cos_lo, cos_hi;  // cone: cos(angle(ubar, axis)) in [cos_lo, cos_hi]
};

struct SpeciesDev {
    double qdt;          // q * dt
    int32_t col0;        // first column of the species in the ring
    int32_t count;       // particles
};

// ---------------------------------------------------------------------------
// float-float (double-single) helpers: error-free transformations of FP32
// arithmetic (Dekker/Knuth), used where FP64 accuracy is needed without the
// FP64 pipe
// ---------------------------------------------------------------------------
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff two_prod(float a, float b)
{
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ ff two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z))};
}

// ---------------------------------------------------------------------------
// mbarrier / TMA helpers (inline PTX, sm_90+ forms valid on sm_103a)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: spins with a growing back-off for at most 2^18 polls.  A
// poll that fails costs about 4 us on GB300 (the try_wait's own suspension
// plus the back-off; 2^22 polls measured 17 s), so a wait expires after
// about a second, while every wait of a working kernel ends within
// microseconds.  On expiry it raises the block's abort flag and the device
// error word, and returns false; callers then carry on without waiting
// (results are flagged invalid) so that no thread is left behind at a barrier.
constexpr uint32_t kMaxPolls = 1u << 18;

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  volatile int* s_abort, int* err_word)
{
    if (mbar_try_wait(bar, parity)) return true;
    for (uint32_t it = 0; it < kMaxPolls; ++it) {
        if (*s_abort) return false;
        if (mbar_try_wait(bar, parity)) return true;
        __nanosleep(it < 64 ? 32 : 256);
    }
    *s_abort = 1;
    atomicOr(err_word, kErrTimeout);
    return false;
}

// Orders this thread's earlier generic-proxy accesses to shared memory before
// later async-proxy (bulk copy) writes to it.
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bounded wait for a block's own copies still in flight before it exits: it
// polls at most kMaxPolls times and never raises flags.
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity)
{
    for (uint32_t it = 0; it < kMaxPolls; ++it) {
        if (mbar_try_wait(bar, parity)) return;
        __nanosleep(256);
    }
}

// 1-D bulk copy (TMA) of `bytes` contiguous bytes into shared memory,
// completion on `bar`.  Both addresses 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes),
        "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void named_barrier_sync(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}


// ---------------------------------------------------------------------------
// kernel parameter blocks and launchers
// ---------------------------------------------------------------------------
struct IngestParams {
    const double* x;        // [n_steps][3][n_in]
    const double* u;        // [n_steps][3][n_in]
    int64_t n_in;           // particles on the input axis
    int32_t n_steps;
    int64_t step0;          // absolute step of the first state in x/u
    double dt;
    double box_L;           // 0: no unwrapping
    double* x_prev;         // [3][ncols] raw x of the previous call
    double* r_prev;         // [3][ncols] image count n of the previous call (r = x + L n)
    double* u_prev;         // [3][ncols] u of the previous call
    float* slab32;          // FP32 ring or nullptr
    double* slab64;         // FP64 ring or nullptr
    float* anc32;           // FP32 path: tile-major anchor ring (r_a as hi + lo)
    int64_t ncols;
    int64_t ring;           // samples in the ring
    int32_t comps;          // ring components per sample (10, or 11 with selector flags)
    int32_t K;              // anchor interval (FP32 path)
    int64_t nblk;           // anchor blocks in the ring
    int32_t n_species;
    int64_t in_off[kMaxSpecies + 1];
    int32_t col_off[kMaxSpecies];
    int32_t check;          // flag non-finite inputs
    int* err_word;
    const SelectorDev* sel; // selectors (device) or nullptr
    int32_t n_sel;
    int32_t nsub;           // sub-samples per PIC sample (<= 1: none)
    // particle range of this launch and layout of x/u (zero: all particles,
    // x/u holding every particle): particles first .. first + count - 1 are
    // processed; particle i is column i - xoff of x/u, whose particle axis
    // has stride ld
    int64_t first;
    int64_t count;
    int64_t ld;
    int64_t xoff;
    // time segments (one thread per particle and segment): segment 0 starts at
    // step0, segment g >= 1 at seg_first + (g - 1) seg_len (calls 1 + j seg_len:
    // anchor-aligned samples); wind [n_seg - 1][3][count] receives each
    // segment's change of the image count.  n_seg <= 1: one thread per particle.
    int64_t seg_first;
    int32_t seg_len;
    int32_t n_seg;
    int32_t* wind;
    double* state_out;      // [9][count]: the last segment's carry-over state,
                            // stored to x_prev/r_prev/u_prev after the launch
};

struct Accum32Params {
    const WorkItem* items;
    int32_t n_items;
    int* counter;             // dynamic item counter (zeroed before the launch)
    const WinDev* wins;
    const SpeciesDev* species;
    const float* dirs32;      // [D][12]: n, e1, e2, n - (float)n
    const float* omega;       // [n_freq] rad per unit time
    const float* nu_hi;       // [n_freq] (omega / 2 pi) hi part
    const float* nu_lo;       // [n_freq] lo part
    const float* slab32;      // tile-major FP32 ring
    const float* anc32;       // tile-major anchor ring
    int64_t ring;
    int64_t nblk;
    int32_t comps;            // ring components per sample (10, or 11 with selector flags)
    float dt_hi, dt_lo;       // dt as a float-float pair
    double* acc;              // incoherent [n_out]; coherent [n_out][4]
    int* err_word;
    // failure-detection test hook (0: off): block 0's producer first waits on
    // a barrier nothing arrives on, so that its bounded wait expires
    int32_t fault_stall;
};

struct Accum64Params {
    const WorkItem* items;
    int32_t n_items;
    const WinDev* wins;
    const SpeciesDev* species;
    const double* dirs64;     // [D][9]: n, e1, e2
    const double* omega;      // [n_freq]
    const double* slab64;     // tile-major FP64 ring
    int64_t ring;
    int32_t comps;            // ring components per sample (10, or 11 with selector flags)
    double dt;
    double* acc;
    int* err_word;
    int32_t fault_stall;      // as in Accum32Params
};

cudaError_t launch_ingest(const IngestParams& p, cudaStream_t st);
// The two builds of the ingest kernel (common ring, precise-phase ring); a
// kernel function pointer compares equal to the set when it is either build.
struct IngestKernels {
    const void* plain;
    const void* precise;
};
inline bool operator==(const void* f, const IngestKernels& k) { return f == k.plain || f == k.precise; }
IngestKernels ingest_kernel_ptr();

// Stream a radiation context orders its work on (for in-library callers that
// hand it device buffers from another stream).
cudaStream_t ctx_stream(const rad_ctx* c);
// Particles a radiation context takes per call, and the step it expects next.
int64_t ctx_particles(const rad_ctx* c);
int64_t ctx_next_step(const rad_ctx* c);
// FP32 kernel variant: frequencies per thread, of which np by the FMA-pipe
// polynomial, anchor interval K, coherent sum, minimum resident blocks per SM.
struct Accum32Config {
    int ft, np, K;
    bool coh;
    int mb;
    bool band = false;   // items with anchor blocks of K << kmul (8 SFU frequencies per thread)
    int pm = 0;          // precise offset phase (8 SFU frequencies, K 32): 0 none, 1 every
                         // item, 2 the items whose WorkItem.prec is set
};
bool accum32_ft8_sfu(const Accum32Params* p, const Accum32Config& cfg, int grid,
                     cudaStream_t st, cudaError_t* err, int* nb);
bool accum32_band(const Accum32Params* p, const Accum32Config& cfg, int grid,
                  cudaStream_t st, cudaError_t* err, int* nb);
bool accum32_precise(const Accum32Params* p, const Accum32Config& cfg, int grid,
                     cudaStream_t st, cudaError_t* err, int* nb);
bool accum32_ft8_mix(const Accum32Params* p, const Accum32Config& cfg, int grid,
                     cudaStream_t st, cudaError_t* err, int* nb);
bool accum32_ft16(const Accum32Params* p, const Accum32Config& cfg, int grid,
                  cudaStream_t st, cudaError_t* err, int* nb);
bool accum32_ft4(const Accum32Params* p, const Accum32Config& cfg, int grid,
                 cudaStream_t st, cudaError_t* err, int* nb);
// launch (p != nullptr) or occupancy query; false if the variant is not built
bool accum32_dispatch(const Accum32Params* p, const Accum32Config& cfg, int grid,
                      cudaStream_t st, cudaError_t* err, int* nb);
cudaError_t launch_accum64(const Accum64Params& p, bool coh, int grid, cudaStream_t st);
int accum64_blocks_per_sm(bool coh);
int accum64_ft();

}  // namespace rad
