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
// * Phase split: phi_m = phi_ref + dphi_m.  phi_ref is the FP64 retarded time
//   at the block's anchor sample a = K floor(m/K), shifted to the middle of the
//   block's phase range; it enters once per K samples through the float-float
//   product nu_k * phi_ref (nu = w / 2 pi, both as hi+lo FP32 pairs) reduced
//   modulo one turn exactly.  dphi_m = (m - a - (K-1)) dt - n.(r_m - r_a) is
//   formed in FP64 from the ring's FP32 offsets and rounded once, so the
//   per-update phase is one FP32 FMA: theta = fma(w_k, dphi_m, Theta_k).
// * e^{i theta}: by the special-function unit (__sincosf) for the first FT-NP
//   frequencies of each thread; for the last NP (MIX variant) by an FMA-pipe
//   polynomial -- Cody-Waite reduction of theta/2 by multiples of pi, minimax
//   sin (degree 9) and cos (degree 8) on [-pi/2, pi/2], double angle -- so
//   both the MUFU and the FMA pipes carry the transcendental work.
// * The trajectory ring is tile-major ([tile][slot][comp][8 particles]), so a
//   chunk of 32 samples x 10 components x 8 particles is one contiguous 10 KB
//   block, staged into shared memory by a bulk TMA copy (cp.async.bulk) from a
//   dedicated producer warp, double-buffered on mbarriers.  Each compute warp
//   owns one particle; each lane FT frequencies (stride 32: coalesced output).
// * Persistent grid: block b takes items b, b + gridDim.x, ... from a list
//   sorted by decreasing cost.
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

// Constants of the work item every compute warp is on; kept in shared memory
// (re-read where used) so that the update loop holds only its accumulators.
struct ItemSmem {
    double nd[3];          // n (FP64) for the phase offsets
    int64_t s0, s1;        // window
    int64_t out_off;
    float n[3], e1[3], e2[3];
    float qdt;
    int32_t grid_off, grid_len;
    int32_t count, tile0, ntiles, ftile, dir, tilebase;
};

template <int FT, int K, bool COH>
struct Smem32 {
    float tbuf[2][kChunk32][kComps][kTileP];   // 2 x 10240 B, bulk-copy destinations
    float4 geo[kComputeWarps][kChunk32];        // V1, V2, dphi per sample
    float2 anc[kComputeWarps][kChunk32 / K];    // phi_ref as hi + lo
    float ths[kComputeWarps][kChunk32 / K][FT][32];  // anchor phases per block
    float red[kComputeWarps][FT][32];           // window-close partials
    double run[(COH ? 4 : 1) * FT * 32];        // per-item particle sums (FP64)
    ItemSmem item;
    uint64_t full[2];
    uint64_t empty[2];
    int abort_flag;
};

template <int FT, int NP, int K, bool COH>
constexpr size_t smem32_bytes()
{
    return sizeof(Smem32<FT, K, COH>) + 128;
}

template <int FT, int NP, int K, bool COH, int MB>
__global__ void __launch_bounds__(kBlockThreads, MB) accum32_kernel(const Accum32Params p)
{
    static_assert(NP >= 0 && NP < FT, "polynomial frequencies per thread");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    auto& S = *reinterpret_cast<Smem32<FT, K, COH>*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    constexpr uint32_t kBytes = sizeof(S.tbuf[0]);
    constexpr int kNRun = (COH ? 4 : 1) * FT * 32;
    constexpr int NS = FT - NP;   // SFU frequencies per thread

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;

    if (tid == 0) {
        mbar_init(&S.full[0], 1);
        mbar_init(&S.full[1], 1);
        mbar_init(&S.empty[0], kComputeWarps);
        mbar_init(&S.empty[1], kComputeWarps);
        S.abort_flag = 0;
        fence_mbar_init();
    }
    for (int v = tid; v < kNRun; v += blockDim.x) S.run[v] = 0.0;
    __syncthreads();
    volatile int* abort_flag = &S.abort_flag;

    // ------------------------------------------------------------------ producer
    if (warp == kComputeWarps) {
        if (lane != 0) return;
        uint32_t L = 0;
        for (int ii = blockIdx.x; ii < p.n_items; ii += gridDim.x) {
            const WorkItem it = p.items[ii];
            const WinDev w = p.wins[it.win];
            const int64_t c0 = w.s0 / kChunk32, c1 = (w.s1 - 1) / kChunk32;
            const int64_t tilebase = p.species[it.sp].col0 / kTileP;
            for (int t = 0; t < it.ntiles; ++t) {
                const int64_t tile = tilebase + it.tile0 + t;
                for (int64_t c = c0; c <= c1; ++c, ++L) {
                    const int buf = L & 1;
                    if (L >= 2) mbar_wait_bounded(&S.empty[buf], ((L - 2) >> 1) & 1, abort_flag,
                                                  p.err_word);
                    if (*abort_flag) continue;
                    mbar_arrive_expect_tx(&S.full[buf], kBytes);
                    const int64_t slot = (c * kChunk32) % p.ring;
                    const float* src = p.slab32 + (tile * p.ring + slot) * (kComps * kTileP);
                    bulk_load(&S.tbuf[buf][0][0][0], src, kBytes, &S.full[buf]);
                }
            }
        }
        // never leave the block with a copy in flight
        if (L >= 1) mbar_wait_bounded(&S.full[(L - 1) & 1], ((L - 1) >> 1) & 1, abort_flag,
                                      p.err_word);
        if (L >= 2) mbar_wait_bounded(&S.full[(L - 2) & 1], ((L - 2) >> 1) & 1, abort_flag,
                                      p.err_word);
        return;
    }

    // ------------------------------------------------------------------ compute
    uint32_t L = 0;
    for (int ii = blockIdx.x; ii < p.n_items; ii += gridDim.x) {
        if (tid == 0) {
            const WorkItem it = p.items[ii];
            const WinDev w = p.wins[it.win];
            const SpeciesDev spd = p.species[it.sp];
            ItemSmem& I = S.item;
            for (int q = 0; q < 3; ++q) {
                I.nd[q] = p.dirs64[3 * it.dir + q];
                I.n[q] = p.dirs32[9 * it.dir + q];
                I.e1[q] = p.dirs32[9 * it.dir + 3 + q];
                I.e2[q] = p.dirs32[9 * it.dir + 6 + q];
            }
            I.s0 = w.s0;
            I.s1 = w.s1;
            I.out_off = w.out_off;
            I.qdt = (float)spd.qdt;
            I.grid_off = w.grid_off;
            I.grid_len = w.grid_len;
            I.count = spd.count;
            I.tile0 = it.tile0;
            I.ntiles = it.ntiles;
            I.ftile = it.ftile;
            I.dir = it.dir;
            I.tilebase = spd.col0 / kTileP;
        }
        named_barrier_sync(1, kComputeWarps * 32);
        const int kbase = S.item.ftile * (32 * FT) + lane;
        float om[FT];   // omega (SFU) or omega / 2 (polynomial)
#pragma unroll
        for (int i = 0; i < FT; ++i) {
            const int k = kbase + 32 * i;
            const float wk = (k < S.item.grid_len) ? p.omega[S.item.grid_off + k] : 0.0f;
            om[i] = (i < NS) ? wk : 0.5f * wk;
        }
        const int ntiles = S.item.ntiles;

        for (int t = 0; t < ntiles; ++t) {
            float a1r[FT], a1i[FT], a2r[FT], a2i[FT], th[FT];
#pragma unroll
            for (int i = 0; i < FT; ++i) a1r[i] = a1i[i] = a2r[i] = a2i[i] = th[i] = 0.0f;
            const int64_t c0 = S.item.s0 / kChunk32, c1 = (S.item.s1 - 1) / kChunk32;

            for (int64_t c = c0; c <= c1; ++c, ++L) {
                const int buf = L & 1;
                mbar_wait_bounded(&S.full[buf], (L >> 1) & 1, abort_flag, p.err_word);
                // ---- geometry of sample m = 32 c + lane for this warp's particle
                {
                    const ItemSmem& I = S.item;
                    const float* tb = &S.tbuf[buf][lane][0][warp];
                    const float b0 = tb[3 * kTileP], b1 = tb[4 * kTileP], b2 = tb[5 * kTileP];
                    const float bn = I.n[0] * b0 + I.n[1] * b1 + I.n[2] * b2;
                    const float p1 = I.e1[0] * b0 + I.e1[1] * b1 + I.e1[2] * b2;
                    const float p2 = I.e2[0] * b0 + I.e2[1] * b1 + I.e2[2] * b2;
                    const float d0 = tb[6 * kTileP], d1 = tb[7 * kTileP], d2 = tb[8 * kTileP];
                    const float dn = I.n[0] * d0 + I.n[1] * d1 + I.n[2] * d2;
                    const float q1 = I.e1[0] * d0 + I.e1[1] * d1 + I.e1[2] * d2;
                    const float q2 = I.e2[0] * d0 + I.e2[1] * d1 + I.e2[2] * d2;
                    const float g = tb[9 * kTileP];
                    const float kap = bn > 0.0f ? (g + p1 * p1 + p2 * p2) / (1.0f + bn) : 1.0f - bn;
                    const float inv = I.qdt / (kap * kap);
                    const float V1 = -(p1 * dn + q1 * kap) * inv;
                    const float V2 = -(p2 * dn + q2 * kap) * inv;
                    const int64_t m = c * kChunk32 + lane;
                    const int64_t a = m - (m & (K - 1));
                    const double dphi = (double)(m - a - (K - 1)) * p.dt -
                                        (I.nd[0] * (double)tb[0] + I.nd[1] * (double)tb[kTileP] +
                                         I.nd[2] * (double)tb[2 * kTileP]);
                    S.geo[warp][lane] = make_float4(V1, V2, (float)dphi, 0.0f);
                    if ((lane & (K - 1)) == 0) {
                        const int64_t col = (int64_t)(I.tilebase + I.tile0 + t) * kTileP + warp;
                        const int64_t blk = (a / K) % p.nblk;
                        const double* ra = p.anchors + blk * 3 * p.ncols + col;
                        const double phi_ref = (double)(a + K - 1) * p.dt -
                                               (I.nd[0] * ra[0] + I.nd[1] * ra[p.ncols] +
                                                I.nd[2] * ra[2 * p.ncols]);
                        const float hi = (float)phi_ref;
                        const float lo = (float)(phi_ref - (double)hi);
                        S.anc[warp][lane / K] = make_float2(hi, lo);
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&S.empty[buf]);

                // ---- anchor phases Theta_k = 2 pi frac(nu_k phi_ref) of the chunk's
                // anchor blocks (float-float product, exact reduction to one turn);
                // halved for the polynomial frequencies
                const int64_t cs = c * kChunk32;
                const int lo = (int)((S.item.s0 > cs ? S.item.s0 : cs) - cs);
                const int hi = (int)((S.item.s1 < cs + kChunk32 ? S.item.s1 : cs + kChunk32) - cs);
#pragma unroll 1
                for (int b = lo / K; b * K < hi; ++b) {
                    const float2 an = S.anc[warp][b];
                    const int goff = S.item.grid_off, glen = S.item.grid_len;
#pragma unroll
                    for (int i = 0; i < FT; ++i) {
                        const int k = kbase + 32 * i;
                        const int kk = goff + (k < glen ? k : 0);
                        const float nh = __ldg(p.nu_hi + kk), nl = __ldg(p.nu_lo + kk);
                        const float pr = nh * an.x;
                        const float pe = fmaf(nh, an.x, -pr);
                        const float tl = fmaf(nl, an.x, fmaf(nh, an.y, pe));
                        const float fr = pr - rintf(pr);
                        S.ths[warp][b][i][lane] =
                            (fr + tl) * (i < NS ? 6.28318530717958647f : 3.14159265358979323f);
                    }
                }
                __syncwarp();

                // ---- update loop over the chunk's samples inside the window, one
                // anchor block at a time; the next sample's geometry is loaded
                // while the current one is being accumulated
#pragma unroll 1
                for (int b = lo / K; b * K < hi; ++b) {
                    const int l0 = lo > b * K ? lo : b * K;
                    const int l1 = hi < b * K + K ? hi : b * K + K;
#pragma unroll
                    for (int i = 0; i < FT; ++i) th[i] = S.ths[warp][b][i][lane];
                    float4 gg = S.geo[warp][l0];
#pragma unroll 1
                    for (int l = l0; l < l1; ++l) {
                        const float4 gn = S.geo[warp][(l + 1) & (kChunk32 - 1)];
#pragma unroll
                        for (int i = 0; i < NS; ++i) {
                            const float tt = fmaf(om[i], gg.z, th[i]);
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
                __syncwarp();
            }

            // ---- window close for this tile: reduce over the block's 8 particles
            const bool real_particle = (S.item.tile0 + t) * kTileP + warp < S.item.count;
            if (!COH) {
#pragma unroll
                for (int i = 0; i < FT; ++i) {
                    const float pw = a1r[i] * a1r[i] + a1i[i] * a1i[i] + a2r[i] * a2r[i] +
                                     a2i[i] * a2i[i];
                    S.red[warp][i][lane] = real_particle ? pw : 0.0f;
                }
                named_barrier_sync(1, kComputeWarps * 32);
                for (int v = tid; v < FT * 32; v += kComputeWarps * 32) {
                    double s = 0.0;
#pragma unroll
                    for (int q = 0; q < kComputeWarps; ++q) s += (double)S.red[q][v >> 5][v & 31];
                    S.run[v] += s;
                }
                named_barrier_sync(1, kComputeWarps * 32);
            } else {
#pragma unroll
                for (int comp = 0; comp < 4; ++comp) {
#pragma unroll
                    for (int i = 0; i < FT; ++i) {
                        const float val = comp == 0 ? a1r[i] : comp == 1 ? a1i[i]
                                        : comp == 2 ? a2r[i] : a2i[i];
                        S.red[warp][i][lane] = real_particle ? val : 0.0f;
                    }
                    named_barrier_sync(1, kComputeWarps * 32);
                    for (int v = tid; v < FT * 32; v += kComputeWarps * 32) {
                        double s = 0.0;
#pragma unroll
                        for (int q = 0; q < kComputeWarps; ++q)
                            s += (double)S.red[q][v >> 5][v & 31];
                        S.run[v * 4 + comp] += s;
                    }
                    named_barrier_sync(1, kComputeWarps * 32);
                }
            }
        }

        // ---- item done: add the particle sums to the FP64 accumulators
        {
            const ItemSmem& I = S.item;
            for (int v = tid; v < FT * 32; v += kComputeWarps * 32) {
                const int k = I.ftile * (32 * FT) + (v & 31) + 32 * (v >> 5);
                if (k < I.grid_len) {
                    const int64_t o = I.out_off + (int64_t)I.dir * I.grid_len + k;
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
        // everyone is done with S.item before thread 0 overwrites it
        named_barrier_sync(1, kComputeWarps * 32);
    }
}

template <int FT, int NP, int K, bool COH, int MB>
cudaError_t launch32_one(const Accum32Params& p, int grid, cudaStream_t st)
{
    auto kern = accum32_kernel<FT, NP, K, COH, MB>;
    const size_t smem = smem32_bytes<FT, NP, K, COH>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kBlockThreads, smem, st>>>(p);
    return cudaGetLastError();
}

template <int FT, int NP, int K, bool COH, int MB>
int blocks32_one()
{
    int nb = 0;
    const size_t smem = smem32_bytes<FT, NP, K, COH>();
    if (cudaFuncSetAttribute(accum32_kernel<FT, NP, K, COH, MB>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, accum32_kernel<FT, NP, K, COH, MB>,
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
