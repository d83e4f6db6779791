// rad_accum32.cuh -- FP32 split-phase accumulation of the far-field amplitude
// (kernel template; instantiated by rad_accum32_*.cu).
//
// For every work item (window, direction n, frequency tile, run of particle
// tiles) the block evaluates, for each particle j and frequency w_k,
//   A_{j,k} = sum_{m in window} q V_m exp(i w_k phi_m) dt        (Sec. 2.2)
//   V = n x ((n - beta) x betadot) / (1 - n.beta)^2,  phi = t_m - n.r_m,
// then the window-close reduction: incoherent sum_j |A_j|^2 or coherent
// sum_j A_j, added in FP64 to the accumulators.
//
// Design (GB300):
// * V is perpendicular to n, so it is carried as two components on an
//   orthonormal basis (e1, e2) of the plane normal to n:
//     e_i . [n x ((n-beta) x betadot)] = -(e_i.beta)(n.betadot) - (e_i.betadot) kappa,
//   kappa = 1 - n.beta evaluated as (g + (e1.beta)^2 + (e2.beta)^2)/(1 + n.beta)
//   when n.beta > 0 (no cancellation at high gamma), else directly.
//   |A|^2 = |A.e1|^2 + |A.e2|^2: two complex accumulators per (j, n, w).
// * Phase split: phi_m = phi_ref + dphi_m.  phi_ref is the retarded time at
//   the block's anchor sample a = K floor(m/K) plus the centre h of the
//   block's offsets (half the offset of its last sample), carried as a
//   float-float (hi + lo FP32) pair with FP64-class accuracy; it enters once
//   per K samples through the float-float product nu_k * phi_ref
//   (nu = w / 2 pi) reduced modulo one turn exactly.
//   dphi_m = (m - a) dt - h - n.(r_m - r_a) is formed with compensated
//   (error-free) FP32 arithmetic from the ring's FP32 offsets and rounded
//   once, so |dphi| is at most half the block's phase range (K dt (1 - n.beta)
//   / 2: tiny towards the head-on directions) and the per-update phase is one
//   FP32 FMA:
//   theta = fma(w_k, dphi_m, Theta_k).  GB300's FP64 pipe is 1/64 of FP32
//   and its latency stalls the warps, so the kernel issues no FP64 at all.
// * e^{i theta}: by the special-function unit (__sincosf) for the first FT-NP
//   frequencies of each thread; for the last NP (MIX variant) by an FMA-pipe
//   polynomial -- Cody-Waite reduction of theta/2 by multiples of pi, minimax
//   sin (degree 9) and cos (degree 8) on [-pi/2, pi/2], double angle -- so
//   both the MUFU and the FMA pipes carry the transcendental work.
// * Builds beside the common one: per-item anchor blocks of K << kmul samples
//   (BAND: longer blocks for lower frequency tiles under a phase budget), and
//   the precise phase (PM: nu dphi in float-float from a ring that carries the
//   position offsets' lo parts, reduced to one turn before the special-function
//   unit; for every item or per item).
// * The trajectory ring is tile-major ([tile][slot][comp][8 particles]), so a
//   chunk of 32 samples x 10 components (11 with selector flags, 14 for the
//   precise phase) x 8 particles is one contiguous block (its anchor positions
//   another), staged into shared memory by bulk
//   TMA copies (cp.async.bulk).  Warp specialisation: a producer warp issues
//   the copies and turns each chunk into geometry and reference phases in
//   shared memory (double-buffered, mbarrier hand-off); eight compute warps,
//   one particle per warp, FT frequencies per lane (stride 32: coalesced
//   output), turn each anchor block's phi_ref into their own anchor phases
//   (about 12 FP32 operations per frequency per block, so short blocks cost
//   the compute warps little and the producer nothing) and run the update loop.
// * Persistent grid with a dynamic longest-first schedule: the producer of each
//   block takes the next item of a list sorted by decreasing cost from an atomic
//   counter and describes every chunk it hands over (item, tile, sample range,
//   first/last flags), so the compute warps need no schedule of their own.
#pragma once

#include "rad_internal.cuh"

namespace rad {

// FMA-pipe e^{i theta} constants (fit_sincos.py: minimax on [-pi/2, pi/2]).
constexpr float kS3 = -1.666665673e-01f, kS5 = 8.333017118e-03f, kS7 = -1.980661473e-04f,
                kS9 = 2.600054813e-06f;
constexpr float kC2 = -4.999993145e-01f, kC4 = 4.166398942e-02f, kC6 = -1.385592739e-03f,
                kC8 = 2.319438681e-05f;
constexpr float kPiHi = 3.141592741e+00f, kPiLo = -8.742277657e-08f;
constexpr float kInvPi = 0.318309886183790671538f;
constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23: x + kMagic - kMagic = rint(x)

// cos(2 h) and sin(2 h) / 2 for the half angle h (|h| < 2^22 pi).
__device__ __forceinline__ void poly_cis_half(float h, float& c2, float& s2half)
{
    const float t = fmaf(h, kInvPi, kMagic);
    const float k = t - kMagic;
    float y = fmaf(k, -kPiHi, h);
    y = fmaf(k, -kPiLo, y);
    const float y2 = y * y;
    float p = fmaf(y2, kS9, kS7);
    p = fmaf(y2, p, kS5);
    p = fmaf(y2, p, kS3);
    const float y3 = y * y2;
    const float s = fmaf(y3, p, y);
    float q = fmaf(y2, kC8, kC6);
    q = fmaf(y2, q, kC4);
    q = fmaf(y2, q, kC2);
    const float c = fmaf(y2, q, 1.0f);
    c2 = fmaf(c, c, -(s * s));
    s2half = c * s;
}

// frac(nu phi_ref) in turns, in [-1, 1]: the float-float product of nu (hi, lo)
// and phi_ref (hi, lo) with its integer part removed exactly on the FP32 pipe
// (no round instruction next to the sin/cos of the update loop): adding and
// removing 1.5 * 2^23 rounds to an integer for |x| < 2^22 and to a float within
// a few ulp of x above; either difference is exact (Sterbenz), and the second
// pass brings a large-|x| remainder into [-1/2, 1/2].
__device__ __forceinline__ float anchor_turns(float nh, float nl, float2 an)
{
    // __fmul_rn / __fadd_rn: the rounded product pr must not be re-formed as a
    // fused multiply-add inside the sums below (pe holds its rounding error)
    const float pr = __fmul_rn(nh, an.x);
    const float pe = fmaf(nh, an.x, -pr);
    const float tl = fmaf(nl, an.x, fmaf(nh, an.y, pe));
    float fr = __fsub_rn(pr, __fsub_rn(__fadd_rn(pr, kMagic), kMagic));
    fr = __fsub_rn(fr, __fsub_rn(__fadd_rn(fr, kMagic), kMagic));
    return __fadd_rn(fr, tl);
}

// Shared-memory slot of lane l's j-th float4 of frequencies: l * FT/4 + j, with j
// flipped for every other group of four lanes when a lane has two or more slots,
// so that the eight lanes of one 128-bit access phase cover all 32 banks.
template <int FT>
__device__ __forceinline__ int nu_slot(int lane, int j)
{
    static_assert(FT % 4 == 0, "frequencies per thread come in float4 slots");
    return lane * (FT / 4) + (FT / 4 > 1 ? (j ^ ((lane >> 2) & 1)) : j);
}

// What the producer tells the compute warps about the chunk in a buffer.
struct ChunkMeta {
    int64_t out_off;       // the item's output block
    int32_t ii;            // item index (-1: no more work)
    int32_t lo, hi;        // samples [lo, hi) of the chunk inside the window
    int32_t flags;         // kFirstOfTile | kLastOfTile | kFirstOfItem | kLastOfItem
    int32_t real;          // particles of this tile that exist (0..8)
    int32_t grid_len, ftile, row;   // row: the direction's output row in the window
    int32_t kmul;          // anchor blocks of K << kmul samples
};
constexpr int kFirstOfTile = 1, kLastOfTile = 2, kFirstOfItem = 4, kLastOfItem = 8;

template <int FT, int K, bool COH, int PM = 0>
struct Smem32 {
    float tbuf[2][kChunk32][PM ? kCompsPrec : kComps][kTileP];     // bulk-copy destinations
                                                      // (producer only; a chunk fills comps rows)
    float tanc[2][kChunk32 / K][6][kTileP];           // the chunk's anchor positions (hi, lo)
    float4 geo[2][kComputeWarps][kChunk32 + 1];       // V1, V2, dphi per particle and sample
    // the item's nu = w / 2 pi as float-float (hi, lo): lane l's FT values as
    // FT/4 float4 slots at nu_slot<FT>(l, j)
    float4 nu[2][2][32 * FT / 4];
    float4 nup[2][32 * FT / 4];                       // the producer's copy for the current item
    float2 anc[2][kComputeWarps][kChunk32 / K];       // phi_ref (hi, lo) per particle, block
    float csh[kComputeWarps][kChunk32 / K];           // centre of each block's offset range
    float2 cof[kComputeWarps][kChunk32 / K];          // n . (r_a - r_A) per ring anchor block
    float red[kComputeWarps][FT][32];                 // window-close partials
    double run[(COH ? 4 : 1) * FT * 32];              // per-item particle sums (FP64)
    ChunkMeta meta[2];
    uint64_t tfull[2];                                // bulk copy landed
    uint64_t gfull[2];                                // geometry of a chunk ready
    uint64_t gempty[2];                               // compute warps done with a chunk
    uint64_t cbar;                                    // compute-warp barrier (bounded)
    int abort_flag;
};

// Barrier among the compute warps with a bounded wait: unlike bar.sync it
// cannot hang if a warp has left after a device-side timeout.
__device__ __forceinline__ void compute_sync(uint64_t* bar, uint32_t& phase, int lane,
                                             volatile int* abort_flag, int* err_word)
{
    __syncwarp();
    if (lane == 0) mbar_arrive(bar);
    mbar_wait_bounded(bar, phase & 1, abort_flag, err_word);
    ++phase;
}

template <int FT, int NP, int K, bool COH, int PM = 0>
constexpr size_t smem32_bytes()
{
    return sizeof(Smem32<FT, K, COH, PM>) + 128;
}

// The producer's walk over (item, tile, chunk): items come from an atomic
// counter (items are sorted by decreasing cost, so this is a dynamic
// longest-first schedule); every tile of an item; every 32-sample chunk the
// item's window touches.  All lanes of the producer warp hold the same state.
struct ChunkCursor {
    int ii, t, ntiles;
    int64_t c, c0, c1;
    bool valid;
    __device__ void load_item(const Accum32Params& p, int lane)
    {
        int v = 0;
        if (lane == 0) v = atomicAdd(p.counter, 1);
        ii = __shfl_sync(0xffffffffu, v, 0);
        valid = ii < p.n_items;
        if (!valid) return;
        const WorkItem it = p.items[ii];
        const WinDev w = p.wins[it.win];
        ntiles = it.ntiles;
        c0 = w.s0 / kChunk32;
        c1 = (w.s1 - 1) / kChunk32;
        t = 0;
        c = c0;
    }
    __device__ void next(const Accum32Params& p, int lane)
    {
        if (++c <= c1) return;
        c = c0;
        if (++t < ntiles) return;
        load_item(p, lane);
    }
};

// BAND: the work items may take anchor blocks of K << kmul samples (a separate
// build, so that the common build keeps its blocks at the compile-time K).
// PM: the precise offset phase (nu * dphi in float-float, reduced to one turn
// before the special-function unit) for no item (0), every item (1) or the
// items that ask for it (2); 1 and 2 read a ring that carries dr's lo part.
template <int FT, int NP, int K, bool COH, int MB, bool BAND = false, int PM = 0>
__global__ void __launch_bounds__(kBlockThreads, MB) accum32_kernel(const Accum32Params p)
{
    static_assert(NP >= 0 && NP < FT, "polynomial frequencies per thread");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    auto& S = *reinterpret_cast<Smem32<FT, K, COH, PM>*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    // one chunk of the ring: 32 samples x comps components x 8 particles
    const int cstride = p.comps * kTileP;
    const uint32_t kBytes = (uint32_t)(kChunk32 * cstride * sizeof(float));
    constexpr int kNRun = (COH ? 4 : 1) * FT * 32;
    constexpr int NS = FT - NP;   // SFU frequencies per thread
    static_assert(K == 8 || K == 16 || K == 32, "ring anchor interval");
    constexpr int kLog2K = K == 8 ? 3 : (K == 16 ? 4 : 5);

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;

    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&S.tfull[b], 1);
            mbar_init(&S.gfull[b], 1);
            mbar_init(&S.gempty[b], kComputeWarps);
        }
        mbar_init(&S.cbar, kComputeWarps);
        S.abort_flag = 0;
        fence_mbar_init();
    }
    for (int v = tid; v < kNRun; v += blockDim.x) S.run[v] = 0.0;
    __syncthreads();
    volatile int* abort_flag = &S.abort_flag;

    // ---------------------------------------------------------------- producer
    // Lane 0 streams the chunks (samples and anchor positions) in with bulk
    // copies one chunk ahead; the whole warp turns each landed chunk into the
    // per-sample geometry (V1, V2, dphi) and the per-anchor-block reference
    // phases phi_ref of the 8 particles, for the compute warps.  FP32 only: the
    // quantities that need FP64 accuracy use float-float (error-free) arithmetic.
    if (warp == kComputeWarps) {
        constexpr int NB = kChunk32 / K;                      // anchor blocks per chunk
        constexpr uint32_t kAncBytes = sizeof(S.tanc[0]);
        // cur is the chunk being turned into geometry; nxt, one chunk ahead, is
        // the only cursor that advances (and so the only one that takes items
        // from the counter): each item is fetched exactly once.
        if (p.fault_stall && blockIdx.x == 0) {
            // test hook: buffer 1 is released only after chunk 1 has been
            // produced, so nothing arrives during this wait and it expires
            mbar_wait_bounded(&S.gempty[1], 0, abort_flag, p.err_word);
        }
        ChunkCursor cur;
        cur.load_item(p, lane);
        bool pending[2] = {false, false};     // copy issued, not yet seen landed
        uint32_t pend_parity[2] = {0, 0};
        uint32_t uses[2] = {0, 0};            // copies issued into each buffer
        auto issue = [&](const ChunkCursor& q, int buf) {
            if (lane == 0 && !*abort_flag) {
                pending[buf] = true;
                pend_parity[buf] = uses[buf] & 1;
                const WorkItem it = p.items[q.ii];
                const int64_t tile = p.species[it.sp].col0 / kTileP + it.tile0 + q.t;
                const int64_t slot = (q.c * kChunk32) % p.ring;
                const int64_t blk = (q.c * NB) % p.nblk;
                const float* src = p.slab32 + (tile * p.ring + slot) * cstride;
                const float* asrc = p.anc32 + (tile * p.nblk + blk) * (6 * kTileP);
                fence_proxy_async();
                mbar_arrive_expect_tx(&S.tfull[buf], kBytes + kAncBytes);
                bulk_load(&S.tbuf[buf][0][0][0], src, kBytes, &S.tfull[buf]);
                bulk_load(&S.tanc[buf][0][0][0], asrc, kAncBytes, &S.tfull[buf]);
            }
            ++uses[buf];
        };
        if (cur.valid) issue(cur, 0);
        int item_loaded = -1;
        float n0 = 0, n1 = 0, n2 = 0, e10 = 0, e11 = 0, e12 = 0, e20 = 0, e21 = 0, e22 = 0;
        float nl0 = 0, nl1 = 0, nl2 = 0, qdt = 0;
        int64_t s0 = 0, s1 = 0, out_off = 0;
        int selb = -1;
        int grid_len = 0, ftile = 0, row = 0, count = 0, tile0 = 0, kmul = 0;
        uint32_t L = 0;
        for (; cur.valid; ++L) {
            const int buf = L & 1;
            ChunkCursor nxt = cur;
            nxt.next(p, lane);
            if (nxt.valid) issue(nxt, buf ^ 1);   // chunk L+1 into the other buffer
            if (cur.ii != item_loaded) {
                item_loaded = cur.ii;
                const WorkItem it = p.items[cur.ii];
                const WinDev w = p.wins[it.win];
                const float* dv = p.dirs32 + 12 * it.dir;
                n0 = dv[0]; n1 = dv[1]; n2 = dv[2];
                e10 = dv[3]; e11 = dv[4]; e12 = dv[5];
                e20 = dv[6]; e21 = dv[7]; e22 = dv[8];
                nl0 = dv[9]; nl1 = dv[10]; nl2 = dv[11];
                qdt = (float)p.species[it.sp].qdt;
                count = p.species[it.sp].count;
                s0 = w.s0;
                s1 = w.s1;
                selb = w.sel;
                out_off = w.out_off;
                grid_len = w.grid_len;
                ftile = it.ftile;
                row = it.row;
                kmul = BAND ? it.kmul : 0;
                tile0 = it.tile0;
#pragma unroll
                for (int j = 0; j < FT / 4; ++j) {
                    float h[4], l[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int k = it.ftile * (32 * FT) + lane + 32 * (4 * j + q);
                        const int kk = w.grid_off + (k < w.grid_len ? k : 0);
                        h[q] = p.nu_hi[kk];
                        l[q] = p.nu_lo[kk];
                    }
                    const int slot = nu_slot<FT>(lane, j);
                    S.nup[0][slot] = make_float4(h[0], h[1], h[2], h[3]);
                    S.nup[1][slot] = make_float4(l[0], l[1], l[2], l[3]);
                }
            }
            // after an abort, produce nothing more: the compute warps may still
            // read this buffer, and its copy may not have landed
            if (L >= 2 &&
                !mbar_wait_bounded(&S.gempty[buf], ((L - 2) >> 1) & 1, abort_flag, p.err_word))
                break;
            if (!mbar_wait_bounded(&S.tfull[buf], (L >> 1) & 1, abort_flag, p.err_word)) break;
            pending[buf] = false;
            const int64_t c = cur.c;
            // samples [lo, hi) of this chunk that lie in the window
            const int64_t cs = c * kChunk32;
            const int lo = (int)((s0 > cs ? s0 : cs) - cs);
            const int hi = (int)((s1 < cs + kChunk32 ? s1 : cs + kChunk32) - cs);
            // Anchor blocks.  The ring holds anchor positions r_a every K samples;
            // an item takes its phases in blocks of KE = K << kmul samples (a
            // longer block for a lower-frequency tile, chosen by the host under
            // the phase-rounding budget), anchored at the first ring anchor A of
            // the block.  For kmul > 0 the offsets of the later ring anchors
            // from A enter the sample offsets as C = n . (r_a - r_A), formed in
            // float-float from the anchors' hi/lo pairs (the differences are
            // short, so the hi parts subtract exactly).
            const int ks = kLog2K + kmul, KE = 1 << ks;
            if (kmul > 0 && lane < kTileP * NB) {
                const int pp = lane & (kTileP - 1), b = lane >> 3;
                const int bA = (b >> kmul) << kmul;
                float sh = 0.0f, e = 0.0f;
                const float nh[3] = {n0, n1, n2}, nlo[3] = {nl0, nl1, nl2};
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const ff dh = two_sum(S.tanc[buf][b][q][pp], -S.tanc[buf][bA][q][pp]);
                    const float dl = dh.lo + (S.tanc[buf][b][3 + q][pp] - S.tanc[buf][bA][3 + q][pp]);
                    const ff d = two_prod(nh[q], dh.hi);
                    const float dd = fmaf(nh[q], dl, fmaf(nlo[q], dh.hi, d.lo));
                    const ff u = two_sum(sh, d.hi);
                    sh = u.hi;
                    e = e + (u.lo + dd);
                }
                const float chi = sh + e;
                S.cof[pp][b] = make_float2(chi, e - (chi - sh));
            }
            __syncwarp();
            // anchor reference phase of (particle pp, block B):
            //   phi_ref = A dt + h - n . r_A,  A = 32 c + KE B   (float-float),
            // h the centre of the block's offsets (A dt - n . r_A + offset = phi_m):
            // the offsets (m - A) dt - n . (r_m - r_A) rise monotonically in m
            // (dphi / dt = 1 - n . beta > 0), so h is the mean of the offsets of
            // the block's first and last samples inside the window, and every
            // offset minus h is at most half the block's phase range -- small
            // where 1 - n . beta is small.  Any h gives the same phi_m; h is taken
            // from samples of the window only, so that the result does not depend
            // on what the ring holds outside it (a block outside the window, or a
            // non-finite offset, takes the range's bound).
            if (lane < kTileP * (NB >> kmul)) {
                const int pp = lane & (kTileP - 1), B = lane >> 3;
                const int bl = B * KE, bA = B << kmul;
                const int mlo = lo > bl ? lo : bl;
                const int mhi = hi - 1 < bl + KE - 1 ? hi - 1 : bl + KE - 1;
                float h = 0.5f * (float)(KE - 1) * p.dt_hi;
                if (mlo <= mhi) {
                    const float* t0 = &S.tbuf[buf][0][0][0] + mlo * cstride + pp;
                    const float* t1 = &S.tbuf[buf][0][0][0] + mhi * cstride + pp;
                    float o0 = (float)(mlo - bl) * p.dt_hi -
                               (n0 * t0[0] + n1 * t0[kTileP] + n2 * t0[2 * kTileP]);
                    float o1 = (float)(mhi - bl) * p.dt_hi -
                               (n0 * t1[0] + n1 * t1[kTileP] + n2 * t1[2 * kTileP]);
                    if (kmul > 0) {
                        o0 -= S.cof[pp][mlo >> kLog2K].x;
                        o1 -= S.cof[pp][mhi >> kLog2K].x;
                    }
                    const float hh = 0.5f * (o0 + o1);
                    if (fabsf(hh) <= (float)KE * p.dt_hi) h = hh;
                }
                S.csh[pp][B] = h;
                const float ta = (float)(c * kChunk32 + bl);
                ff t = two_prod(ta, p.dt_hi);
                float e = fmaf(ta, p.dt_lo, t.lo);
                const ff th = two_sum(t.hi, h);
                float sh = th.hi;
                e = e + th.lo;
                const float nh[3] = {n0, n1, n2}, nlo[3] = {nl0, nl1, nl2};
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const float rh = S.tanc[buf][bA][q][pp], rl = S.tanc[buf][bA][3 + q][pp];
                    const ff d = two_prod(nh[q], rh);
                    const float dl = fmaf(nh[q], rl, fmaf(nlo[q], rh, d.lo));
                    const ff u = two_sum(sh, -d.hi);
                    sh = u.hi;
                    e = e + (u.lo - dl);
                }
                const float hi = sh + e;
                S.anc[buf][pp][B] = make_float2(hi, e - (hi - sh));
            }
            __syncwarp();
            // geometry: round r handles sample 4 r + lane / 8 of particle lane % 8
#pragma unroll 2
            for (int r = 0; r < kChunk32 / 4; ++r) {
                const int sm = 4 * r + (lane >> 3), pp = lane & (kTileP - 1);
                const float* tb = &S.tbuf[buf][0][0][0] + sm * cstride + pp;
                const float b0 = tb[3 * kTileP], b1 = tb[4 * kTileP], b2 = tb[5 * kTileP];
                const float d0 = tb[6 * kTileP], d1 = tb[7 * kTileP], d2 = tb[8 * kTileP];
                const float g = tb[9 * kTileP];
                const float bn = n0 * b0 + n1 * b1 + n2 * b2;
                const float p1 = e10 * b0 + e11 * b1 + e12 * b2;
                const float p2 = e20 * b0 + e21 * b1 + e22 * b2;
                const float dn = n0 * d0 + n1 * d1 + n2 * d2;
                const float q1 = e10 * d0 + e11 * d1 + e12 * d2;
                const float q2 = e20 * d0 + e21 * d1 + e22 * d2;
                const float kap = bn > 0.0f ? (g + p1 * p1 + p2 * p2) / (1.0f + bn) : 1.0f - bn;
                const float inv = qdt / (kap * kap);
                float V1 = -(p1 * dn + q1 * kap) * inv;
                float V2 = -(p2 * dn + q2 * kap) * inv;
                if (selb >= 0 && !((__float_as_uint(tb[10 * kTileP]) >> selb) & 1u)) V1 = V2 = 0.0f;
                // dphi = (sm mod KE) dt - h - n . dr (- C), compensated
                const float ti = (float)(sm & (KE - 1));
                const ff t = two_prod(ti, p.dt_hi);
                float e = fmaf(ti, p.dt_lo, t.lo);
                const ff th = two_sum(t.hi, -S.csh[pp][sm >> ks]);
                float sh = th.hi;
                e = e + th.lo;
                if (kmul > 0) {
                    const float2 cf = S.cof[pp][sm >> kLog2K];
                    const ff u = two_sum(sh, -cf.x);
                    sh = u.hi;
                    e = e + (u.lo - cf.y);
                }
                const float dr[3] = {tb[0], tb[kTileP], tb[2 * kTileP]};
                const float nh[3] = {n0, n1, n2}, nlo[3] = {nl0, nl1, nl2};
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const ff d = two_prod(nh[q], dr[q]);
                    float dl = fmaf(nlo[q], dr[q], d.lo);
                    if (PM) dl = fmaf(nh[q], tb[(11 + q) * kTileP], dl);   // n . dr_lo
                    const ff u = two_sum(sh, -d.hi);
                    sh = u.hi;
                    e = e + (u.lo - dl);
                }
                const float dh = sh + e;
                S.geo[buf][pp][sm] = make_float4(V1, V2, dh, PM ? e - (dh - sh) : 0.0f);
            }
            __syncwarp();
            // the item's frequencies (nu hi, lo) for the compute warps, which turn
            // them and the anchors' phi_ref into their anchor phases themselves
#pragma unroll
            for (int j = 0; j < FT / 4; ++j) {
                const int slot = lane * (FT / 4) + j;
                S.nu[buf][0][slot] = S.nup[0][slot];
                S.nu[buf][1][slot] = S.nup[1][slot];
            }
            if (lane == 0) {
                ChunkMeta& M = S.meta[buf];
                M.out_off = out_off;
                M.ii = cur.ii;
                M.lo = lo;
                M.hi = hi;
                M.flags = (c == cur.c0 ? kFirstOfTile : 0) | (c == cur.c1 ? kLastOfTile : 0) |
                          (c == cur.c0 && cur.t == 0 ? kFirstOfItem : 0) |
                          (c == cur.c1 && cur.t == cur.ntiles - 1 ? kLastOfItem : 0);
                const int base = (tile0 + cur.t) * kTileP;
                M.real = count - base < 0 ? 0 : (count - base > kTileP ? kTileP : count - base);
                M.grid_len = grid_len;
                M.ftile = ftile;
                M.row = row;
                M.kmul = kmul;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.gfull[buf]);
            cur = nxt;
        }
        // tell the compute warps there is no more work
        {
            const int buf = L & 1;
            if (L >= 2) mbar_wait_bounded(&S.gempty[buf], ((L - 2) >> 1) & 1, abort_flag, p.err_word);
            if (lane == 0) {
                S.meta[buf].ii = -1;
                mbar_arrive(&S.gfull[buf]);
            }
        }
        // never leave the block with a copy in flight (only possible after an abort)
        if (lane == 0) {
            for (int b = 0; b < 2; ++b)
                if (pending[b]) mbar_drain(&S.tfull[b], pend_parity[b]);
        }
        return;
    }

    // ---------------------------------------------------------------- compute
    float om[FT];   // omega (SFU), omega / 2 (polynomial) or nu_hi = omega / 2 pi (precise)
    float nlo[FT];  // precise: nu_lo
    float a1r[FT], a1i[FT], a2r[FT], a2i[FT], th[FT];
#pragma unroll
    for (int i = 0; i < FT; ++i) om[i] = nlo[i] = a1r[i] = a1i[i] = a2r[i] = a2i[i] = th[i] = 0.0f;
    bool iprec = PM == 1;   // the current item's phases are precise
    uint32_t cphase = 0;
    for (uint32_t L = 0;; ++L) {
        const int buf = L & 1;
        mbar_wait_bounded(&S.gfull[buf], (L >> 1) & 1, abort_flag, p.err_word);
        const int ii = S.meta[buf].ii;
        if (ii < 0 || *abort_flag) break;
        const int flags = S.meta[buf].flags;
        const int lo = S.meta[buf].lo, hi = S.meta[buf].hi;
        const int ks = kLog2K + (BAND ? S.meta[buf].kmul : 0);   // blocks of 1 << ks samples
        if (flags & kFirstOfItem) {
            const WorkItem it = p.items[ii];
            const WinDev w = p.wins[it.win];
            if (PM == 2) iprec = it.prec != 0;
#pragma unroll
            for (int i = 0; i < FT; ++i) {
                const int k = it.ftile * (32 * FT) + lane + 32 * i;
                if (PM != 0 && (PM == 1 || iprec)) {
                    om[i] = (k < w.grid_len) ? p.nu_hi[w.grid_off + k] : 0.0f;
                    nlo[i] = (k < w.grid_len) ? p.nu_lo[w.grid_off + k] : 0.0f;
                } else {
                    const float wk = (k < w.grid_len) ? p.omega[w.grid_off + k] : 0.0f;
                    om[i] = (i < NS) ? wk : 0.5f * wk;
                }
            }
        }
        if (flags & kFirstOfTile) {
#pragma unroll
            for (int i = 0; i < FT; ++i) a1r[i] = a1i[i] = a2r[i] = a2i[i] = 0.0f;
        }
        // update loop, one anchor block at a time; the next sample's geometry
        // is loaded while the current one is accumulated.  P: precise phase (a
        // compile-time constant unless the build chooses it per item)
        const bool P = PM == 1 || (PM == 2 && iprec);
#pragma unroll 1
        for (int b = lo >> ks; (b << ks) < hi; ++b) {
            const int l0 = lo > (b << ks) ? lo : (b << ks);
            const int l1 = hi < ((b + 1) << ks) ? hi : ((b + 1) << ks);
            // anchor phases Theta_k = frac(nu_k phi_ref) turns: float-float
            // product, exact reduction to one turn; in radians (halved for
            // the polynomial frequencies) unless the phase is precise
            const float2 an = S.anc[buf][warp][b];
#pragma unroll
            for (int j = 0; j < FT / 4; ++j) {
                const int slot = nu_slot<FT>(lane, j);
                const float4 h4 = S.nu[buf][0][slot], l4 = S.nu[buf][1][slot];
                const float nh[4] = {h4.x, h4.y, h4.z, h4.w}, nl[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int i = 4 * j + q;
                    th[i] = P ? anchor_turns(nh[q], nl[q], an)
                              : anchor_turns(nh[q], nl[q], an) *
                                    (i < NS ? 6.28318530717958647f : 3.14159265358979323f);
                }
            }
            float4 gg = S.geo[buf][warp][l0];
#pragma unroll 1
            for (int l = l0; l < l1; ++l) {
                const float4 gn = S.geo[buf][warp][(l + 1) & (kChunk32 - 1)];
#pragma unroll
                for (int i = 0; i < NS; ++i) {
                    float tt;
                    if (P) {
                        // turns: nu dphi = p + (p's rounding error) + nu_lo dphi_hi
                        // + nu_hi dphi_lo (+ Theta); p's integer part removed exactly
                        const float pr = __fmul_rn(om[i], gg.z);
                        float c = fmaf(om[i], gg.z, -pr);
                        c = fmaf(nlo[i], gg.z, c);
                        c = fmaf(om[i], gg.w, c);
                        c = __fadd_rn(c, th[i]);
                        const float r = __fsub_rn(__fadd_rn(pr, kMagic), kMagic);
                        tt = __fmul_rn(__fadd_rn(__fsub_rn(pr, r), c), 6.28318530717958647f);
                    } else {
                        tt = fmaf(om[i], gg.z, th[i]);
                    }
                    float sn, cs_;
                    __sincosf(tt, &sn, &cs_);
                    a1r[i] = fmaf(gg.x, cs_, a1r[i]);
                    a1i[i] = fmaf(gg.x, sn, a1i[i]);
                    a2r[i] = fmaf(gg.y, cs_, a2r[i]);
                    a2i[i] = fmaf(gg.y, sn, a2i[i]);
                }
                if (NP > 0) {
                    const float v1d = gg.x + gg.x, v2d = gg.y + gg.y;
#pragma unroll
                    for (int i = NS; i < FT; ++i) {
                        const float hh = fmaf(om[i], gg.z, th[i]);
                        float cs_, snh;
                        poly_cis_half(hh, cs_, snh);
                        a1r[i] = fmaf(gg.x, cs_, a1r[i]);
                        a1i[i] = fmaf(v1d, snh, a1i[i]);
                        a2r[i] = fmaf(gg.y, cs_, a2r[i]);
                        a2i[i] = fmaf(v2d, snh, a2i[i]);
                    }
                }
                gg = gn;
            }
        }
        // copy what the window close needs before the buffer is handed back
        const bool real_particle = warp < S.meta[buf].real;
        const int64_t out_off = S.meta[buf].out_off;
        const int glen = S.meta[buf].grid_len, ftile = S.meta[buf].ftile, row = S.meta[buf].row;
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.gempty[buf]);

        if (flags & kLastOfTile) {
            // ---- window close for this tile: reduce over the block's 8 particles
            if (!COH) {
#pragma unroll
                for (int i = 0; i < FT; ++i) {
                    const float pw = a1r[i] * a1r[i] + a1i[i] * a1i[i] + a2r[i] * a2r[i] +
                                     a2i[i] * a2i[i];
                    S.red[warp][i][lane] = real_particle ? pw : 0.0f;
                }
                compute_sync(&S.cbar, cphase, lane, abort_flag, p.err_word);
                for (int v = tid; v < FT * 32; v += kComputeWarps * 32) {
                    double s = 0.0;
#pragma unroll
                    for (int q = 0; q < kComputeWarps; ++q) s += (double)S.red[q][v >> 5][v & 31];
                    S.run[v] += s;
                }
                compute_sync(&S.cbar, cphase, lane, abort_flag, p.err_word);
            } else {
#pragma unroll
                for (int comp = 0; comp < 4; ++comp) {
#pragma unroll
                    for (int i = 0; i < FT; ++i) {
                        const float val = comp == 0 ? a1r[i] : comp == 1 ? a1i[i]
                                        : comp == 2 ? a2r[i] : a2i[i];
                        S.red[warp][i][lane] = real_particle ? val : 0.0f;
                    }
                    compute_sync(&S.cbar, cphase, lane, abort_flag, p.err_word);
                    for (int v = tid; v < FT * 32; v += kComputeWarps * 32) {
                        double s = 0.0;
#pragma unroll
                        for (int q = 0; q < kComputeWarps; ++q)
                            s += (double)S.red[q][v >> 5][v & 31];
                        S.run[v * 4 + comp] += s;
                    }
                    compute_sync(&S.cbar, cphase, lane, abort_flag, p.err_word);
                }
            }
        }
        if (flags & kLastOfItem) {
            // ---- item done: add the particle sums to the FP64 accumulators
            for (int v = tid; v < FT * 32; v += kComputeWarps * 32) {
                const int k = ftile * (32 * FT) + (v & 31) + 32 * (v >> 5);
                if (k < glen) {
                    const int64_t o = out_off + (int64_t)row * glen + k;
                    if (!COH) {
                        atomicAdd(p.acc + o, S.run[v]);
                    } else {
#pragma unroll
                        for (int comp = 0; comp < 4; ++comp)
                            atomicAdd(p.acc + 4 * o + comp, S.run[v * 4 + comp]);
                    }
                }
                if (!COH) {
                    S.run[v] = 0.0;
                } else {
#pragma unroll
                    for (int comp = 0; comp < 4; ++comp) S.run[v * 4 + comp] = 0.0;
                }
            }
        }
    }
}

template <int FT, int NP, int K, bool COH, int MB, bool BAND = false, int PM = 0>
cudaError_t launch32_one(const Accum32Params& p, int grid, cudaStream_t st)
{
    auto kern = accum32_kernel<FT, NP, K, COH, MB, BAND, PM>;
    const size_t smem = smem32_bytes<FT, NP, K, COH, PM>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kBlockThreads, smem, st>>>(p);
    return cudaGetLastError();
}

template <int FT, int NP, int K, bool COH, int MB, bool BAND = false, int PM = 0>
int blocks32_one()
{
    int nb = 0;
    const size_t smem = smem32_bytes<FT, NP, K, COH, PM>();
    if (cudaFuncSetAttribute(accum32_kernel<FT, NP, K, COH, MB, BAND, PM>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, accum32_kernel<FT, NP, K, COH, MB, BAND, PM>,
                                                      kBlockThreads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

// One instantiation family: (FT, NP, MB) for every K and both summation modes.
#define RAD_ACCUM32_FAMILY(FT, NP, MB)                                                       \
    if (cfg.ft == FT && cfg.np == NP && cfg.mb == MB) {                                      \
        if (cfg.K == 8) { if (cfg.coh) FN(FT, NP, 8, true, MB); else FN(FT, NP, 8, false, MB); } \
        if (cfg.K == 16) { if (cfg.coh) FN(FT, NP, 16, true, MB); else FN(FT, NP, 16, false, MB); } \
        if (cfg.K == 32) { if (cfg.coh) FN(FT, NP, 32, true, MB); else FN(FT, NP, 32, false, MB); } \
    }
}  // namespace rad
