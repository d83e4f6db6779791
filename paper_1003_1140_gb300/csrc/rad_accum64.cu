// rad_accum64.cu -- FP64 accumulation of the far-field amplitude.
//
// Same sum as the FP32 split path (Sec. 2.2, Jackson retarded-time
// integrand), evaluated in FP64 throughout: phi_m = m dt - n.r_m from the
// ring's absolute FP64 positions, theta = w_k phi_m, e^{i theta} by CUDA's
// double-precision sincos, FP64 accumulators and FP64 particle sums.  This is
// the GPU reference against which the FP32 split path is judged; on GB300 it
// is bound by the FP64 pipe.  Trajectory chunks (16 samples x 11 components
// x 8 particles, FP64; one contiguous 11 KB block of the tile-major ring) are
// staged by bulk TMA copies exactly as in the FP32 path.
#include "rad_internal.cuh"

namespace rad {

template <int FT, bool COH>
struct Smem64 {
    double tbuf[2][kChunk64][kComps][kTileP];   // 2 x 11264 B
    double geo[kComputeWarps][kChunk64][4];     // V1, V2, phi, pad
    double red[kComputeWarps][FT][32];
    double run[(COH ? 4 : 1) * FT * 32];
    uint64_t full[2];
    uint64_t empty[2];
    int abort_flag;
};

template <int FT, bool COH>
__global__ void __launch_bounds__(kBlockThreads, 1)
    accum64_kernel(const Accum64Params p)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    auto& S = *reinterpret_cast<Smem64<FT, COH>*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int cstride = p.comps * kTileP;   // one sample's components x 8 particles
    const uint32_t kBytes = (uint32_t)(kChunk64 * cstride * sizeof(double));
    constexpr int kNRun = (COH ? 4 : 1) * FT * 32;
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

    if (warp == kComputeWarps) {
        if (lane != 0) return;
        if (p.fault_stall && blockIdx.x == 0) {
            // test hook: buffer 1 is released only after its first chunk has
            // been issued, so nothing arrives during this wait and it expires
            mbar_wait_bounded(&S.empty[1], 0, abort_flag, p.err_word);
        }
        bool pending[2] = {false, false};   // a copy was issued into the buffer
        uint32_t pend_parity[2] = {0, 0};   // phase parity of its latest copy
        uint32_t L = 0;
        for (int ii = blockIdx.x; ii < p.n_items; ii += gridDim.x) {
            const WorkItem it = p.items[ii];
            const WinDev w = p.wins[it.win];
            const int64_t c0 = w.s0 / kChunk64, c1 = (w.s1 - 1) / kChunk64;
            const int64_t tilebase = p.species[it.sp].col0 / kTileP;
            for (int t = 0; t < it.ntiles; ++t) {
                const int64_t tile = tilebase + it.tile0 + t;
                for (int64_t c = c0; c <= c1; ++c, ++L) {
                    const int buf = L & 1;
                    if (L >= 2) mbar_wait_bounded(&S.empty[buf], ((L - 2) >> 1) & 1, abort_flag,
                                                  p.err_word);
                    if (*abort_flag) continue;
                    pending[buf] = true;
                    pend_parity[buf] = (L >> 1) & 1;
                    mbar_arrive_expect_tx(&S.full[buf], kBytes);
                    const int64_t slot = (c * kChunk64) % p.ring;
                    const double* src = p.slab64 + (tile * p.ring + slot) * cstride;
                    bulk_load(&S.tbuf[buf][0][0][0], src, kBytes, &S.full[buf]);
                }
            }
        }
        // never leave the block with a copy in flight, also after an abort
        // (bounded; the latest copy into a buffer is the last phase it completes)
        for (int b = 0; b < 2; ++b)
            if (pending[b]) mbar_drain(&S.full[b], pend_parity[b]);
        return;
    }

    uint32_t L = 0;
    for (int ii = blockIdx.x; ii < p.n_items; ii += gridDim.x) {
        const WorkItem it = p.items[ii];
        const WinDev w = p.wins[it.win];
        const SpeciesDev spd = p.species[it.sp];
        const int kbase = it.ftile * (32 * FT) + lane;
        double om[FT];
#pragma unroll
        for (int i = 0; i < FT; ++i) {
            const int k = kbase + 32 * i;
            om[i] = (k < w.grid_len) ? p.omega[w.grid_off + k] : 0.0;
        }
        const int64_t c0 = w.s0 / kChunk64, c1 = (w.s1 - 1) / kChunk64;

        for (int t = 0; t < it.ntiles; ++t) {
            const bool real_particle = (it.tile0 + t) * kTileP + warp < spd.count;
            double a1r[FT], a1i[FT], a2r[FT], a2i[FT];
#pragma unroll
            for (int i = 0; i < FT; ++i) a1r[i] = a1i[i] = a2r[i] = a2i[i] = 0.0;

            for (int64_t c = c0; c <= c1; ++c, ++L) {
                const int buf = L & 1;
                mbar_wait_bounded(&S.full[buf], (L >> 1) & 1, abort_flag, p.err_word);
                if (lane < kChunk64) {
                    const double* dv = p.dirs64 + 9 * it.dir;
                    const double n0 = __ldg(dv + 0), n1 = __ldg(dv + 1), n2 = __ldg(dv + 2);
                    const double e10 = __ldg(dv + 3), e11 = __ldg(dv + 4), e12 = __ldg(dv + 5);
                    const double e20 = __ldg(dv + 6), e21 = __ldg(dv + 7), e22 = __ldg(dv + 8);
                    const double* tb = &S.tbuf[buf][0][0][0] + lane * cstride + warp;
                    const double r0 = tb[0 * kTileP], r1 = tb[1 * kTileP], r2 = tb[2 * kTileP];
                    const double b0 = tb[3 * kTileP], b1 = tb[4 * kTileP], b2 = tb[5 * kTileP];
                    const double d0 = tb[6 * kTileP], d1 = tb[7 * kTileP], d2 = tb[8 * kTileP];
                    const double g = tb[9 * kTileP];
                    const double bn = n0 * b0 + n1 * b1 + n2 * b2;
                    const double p1 = e10 * b0 + e11 * b1 + e12 * b2;
                    const double p2 = e20 * b0 + e21 * b1 + e22 * b2;
                    const double dn = n0 * d0 + n1 * d1 + n2 * d2;
                    const double q1 = e10 * d0 + e11 * d1 + e12 * d2;
                    const double q2 = e20 * d0 + e21 * d1 + e22 * d2;
                    const double kap = bn > 0.0 ? (g + p1 * p1 + p2 * p2) / (1.0 + bn) : 1.0 - bn;
                    const double inv = spd.qdt / (kap * kap);
                    const int64_t m = c * kChunk64 + lane;
                    const bool keep = w.sel < 0 ||
                                      ((((uint32_t)tb[10 * kTileP]) >> w.sel) & 1u);
                    S.geo[warp][lane][0] = keep ? -(p1 * dn + q1 * kap) * inv : 0.0;
                    S.geo[warp][lane][1] = keep ? -(p2 * dn + q2 * kap) * inv : 0.0;
                    S.geo[warp][lane][2] = (double)m * p.dt - (n0 * r0 + n1 * r1 + n2 * r2);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&S.empty[buf]);

                const int64_t cs = c * kChunk64;
                const int lo = (int)((w.s0 > cs ? w.s0 : cs) - cs);
                const int hi = (int)((w.s1 < cs + kChunk64 ? w.s1 : cs + kChunk64) - cs);
                for (int l = lo; l < hi; ++l) {
                    const double V1 = S.geo[warp][l][0], V2 = S.geo[warp][l][1];
                    const double ph = S.geo[warp][l][2];
#pragma unroll
                    for (int i = 0; i < FT; ++i) {
                        double sn, cs_;
                        sincos(om[i] * ph, &sn, &cs_);
                        a1r[i] = fma(V1, cs_, a1r[i]);
                        a1i[i] = fma(V1, sn, a1i[i]);
                        a2r[i] = fma(V2, cs_, a2r[i]);
                        a2i[i] = fma(V2, sn, a2i[i]);
                    }
                }
                __syncwarp();
            }

            if (!COH) {
#pragma unroll
                for (int i = 0; i < FT; ++i) {
                    const double pw = a1r[i] * a1r[i] + a1i[i] * a1i[i] + a2r[i] * a2r[i] +
                                      a2i[i] * a2i[i];
                    S.red[warp][i][lane] = real_particle ? pw : 0.0;
                }
                named_barrier_sync(1, kComputeWarps * 32);
                for (int v = tid; v < FT * 32; v += kComputeWarps * 32) {
                    double s = 0.0;
#pragma unroll
                    for (int q = 0; q < kComputeWarps; ++q) s += S.red[q][v >> 5][v & 31];
                    S.run[v] += s;
                }
                named_barrier_sync(1, kComputeWarps * 32);
            } else {
#pragma unroll
                for (int comp = 0; comp < 4; ++comp) {
#pragma unroll
                    for (int i = 0; i < FT; ++i) {
                        const double val = comp == 0 ? a1r[i] : comp == 1 ? a1i[i]
                                         : comp == 2 ? a2r[i] : a2i[i];
                        S.red[warp][i][lane] = real_particle ? val : 0.0;
                    }
                    named_barrier_sync(1, kComputeWarps * 32);
                    for (int v = tid; v < FT * 32; v += kComputeWarps * 32) {
                        double s = 0.0;
#pragma unroll
                        for (int q = 0; q < kComputeWarps; ++q) s += S.red[q][v >> 5][v & 31];
                        S.run[v * 4 + comp] += s;
                    }
                    named_barrier_sync(1, kComputeWarps * 32);
                }
            }
        }

        for (int v = tid; v < FT * 32; v += kComputeWarps * 32) {
            const int k = it.ftile * (32 * FT) + (v & 31) + 32 * (v >> 5);
            if (k < w.grid_len) {
                const int64_t o = w.out_off + (int64_t)it.row * w.grid_len + k;
                if (!COH) {
                    atomicAdd(p.acc + o, S.run[v]);
                } else {
#pragma unroll
                    for (int comp = 0; comp < 4; ++comp) atomicAdd(p.acc + 4 * o + comp, S.run[v * 4 + comp]);
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

template <int FT, bool COH>
static cudaError_t launch64_one(const Accum64Params& p, int grid, cudaStream_t st)
{
    auto kern = accum64_kernel<FT, COH>;
    const size_t smem = sizeof(Smem64<FT, COH>) + 128;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kBlockThreads, smem, st>>>(p);
    return cudaGetLastError();
}

template <int FT, bool COH>
static int blocks64_one()
{
    int nb = 0;
    const size_t smem = sizeof(Smem64<FT, COH>) + 128;
    cudaFuncSetAttribute(accum64_kernel<FT, COH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, accum64_kernel<FT, COH>, kBlockThreads,
                                                  smem);
    return nb;
}

constexpr int kFT64 = 4;

cudaError_t launch_accum64(const Accum64Params& p, bool coh, int grid, cudaStream_t st)
{
    if (p.n_items == 0) return cudaSuccess;
    return coh ? launch64_one<kFT64, true>(p, grid, st) : launch64_one<kFT64, false>(p, grid, st);
}

int accum64_blocks_per_sm(bool coh)
{
    return coh ? blocks64_one<kFT64, true>() : blocks64_one<kFT64, false>();
}

int accum64_ft() { return kFT64; }

}  // namespace rad
