// rad_ingest.cu -- per-step ingest: leapfrog states -> trajectory ring.
//
// Sec. 2.2 integrates E_ret exp(i w phi') over the particle history.  This
// kernel turns the states the PIC hands over (call s: x_s, u_{s-1/2}) into
// the samples the accumulation needs, one call late: sample m = s - 1 uses
//   r_m       = unwrapped x_m (minimum image in a periodic box),
//   beta_m    = ubar / sqrt(1 + ubar^2),  ubar = (u_{m-1/2} + u_{m+1/2}) / 2,
//   betadot_m = (beta_{m+1/2} - beta_{m-1/2}) / dt,
//   g_m       = 1/gamma_m^2 = 1 / (1 + ubar^2).
// A thread walks one particle through one time segment of the launch's steps,
// keeping the previous raw position, the image count n (the unwrapped position
// is r = x + L n) and u_{s-3/2} in registers; the per-particle state arrays
// carry them between launches.  Segments after the first start at
// anchor-aligned samples; their starting image count is the launch's initial
// count plus the integer changes of the earlier segments (wind_kernel), so the
// split in time changes no result.
#include "rad_internal.cuh"

namespace rad {

// Whole box lengths in a displacement d, rint(d / L): the change of the image
// count (its nearest periodic image is d - L rint(d / L)).  A particle that did
// not cross the boundary has |d| <= L/2, where that is 0 exactly; only a
// crossing pays for the FP64 division, which this GPU runs on its 1/64-rate
// FP64 pipe.  Same value in every case.
__device__ __forceinline__ double image_jump(double d, double L, double half_L)
{
    if (!(L > 0.0) || fabs(d) <= half_L) return 0.0;
    return rint(d / L);
}

// Calls [s_begin, s_end) of segment g of the launch.
__device__ __forceinline__ void segment_range(const IngestParams& p, int g, int64_t& s_begin,
                                              int64_t& s_end)
{
    const int64_t end = p.step0 + p.n_steps;
    if (p.n_seg <= 1) {
        s_begin = p.step0;
        s_end = end;
        return;
    }
    s_begin = g == 0 ? p.step0 : p.seg_first + (int64_t)(g - 1) * p.seg_len;
    const int64_t e = p.seg_first + (int64_t)g * p.seg_len;
    s_end = e < end ? e : end;
}

// Change of the image count over each segment but the last (box_L > 0).
__global__ void __launch_bounds__(256) wind_kernel(const IngestParams p)
{
    const int64_t cnt = p.count ? p.count : p.n_in - p.first;
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= cnt * (p.n_seg - 1)) return;
    const int g = (int)(q / cnt);
    const int64_t k = q - (int64_t)g * cnt, i = p.first + k;
    const int64_t ld = p.ld ? p.ld : p.n_in;
    const int64_t xi = i - p.xoff;
    int sp = 0;
    while (sp + 1 < p.n_species && i >= p.in_off[sp + 1]) ++sp;
    const int64_t col = p.col_off[sp] + (i - p.in_off[sp]);
    int64_t s_begin, s_end;
    segment_range(p, g, s_begin, s_end);
    const double half_L = 0.5 * p.box_L;
    double xp[3];
    bool have = true;
    if (s_begin > p.step0) {
        for (int c = 0; c < 3; ++c) xp[c] = p.x[(s_begin - 1 - p.step0) * 3 * ld + c * ld + xi];
    } else if (p.step0 > 0) {
        for (int c = 0; c < 3; ++c) xp[c] = p.x_prev[c * p.ncols + col];
    } else {
        have = false;                       // call 0 has no predecessor
    }
    int32_t dn[3] = {0, 0, 0};
    for (int64_t s = s_begin; s < s_end; ++s) {
        for (int c = 0; c < 3; ++c) {
            const double xn = p.x[(s - p.step0) * 3 * ld + c * ld + xi];
            if (have) dn[c] -= (int32_t)image_jump(xn - xp[c], p.box_L, half_L);
            xp[c] = xn;
        }
        have = true;
    }
    for (int c = 0; c < 3; ++c) p.wind[((int64_t)g * 3 + c) * cnt + k] = dn[c];
}

// Selector bits of a sample: box tests on the position as handed over, cone
// tests on cos(angle(ubar, axis)) = ubar.axis / |ubar|, in FP64 without
// contraction (the oracle takes the same decisions bit for bit).
__device__ uint32_t selector_bits(const IngestParams& p, const double x[3], const double ub[3])
{
    uint32_t bits = 0;
    for (int i = 0; i < p.n_sel; ++i) {
        const SelectorDev& S = p.sel[i];
        bool in = false;
        if (S.kind == 1) {
            in = x[0] >= S.lo[0] && x[0] < S.hi[0] && x[1] >= S.lo[1] && x[1] < S.hi[1] &&
                 x[2] >= S.lo[2] && x[2] < S.hi[2];
        } else if (S.kind == 2) {
            const double par = __dadd_rn(__dadd_rn(__dmul_rn(ub[0], S.axis[0]), __dmul_rn(ub[1], S.axis[1])),
                                         __dmul_rn(ub[2], S.axis[2]));
            const double nrm = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(ub[0], ub[0]), __dmul_rn(ub[1], ub[1])),
                                                    __dmul_rn(ub[2], ub[2])));
            const double cs = __ddiv_rn(par, nrm);
            in = cs >= S.cos_lo && cs <= S.cos_hi;
        }
        bits |= (in ? 1u : 0u) << i;
    }
    return bits;
}

// 64-thread blocks (launch_ingest), at least 8 resident per SM: the FP64-bound
// loop needs the warps to hide its latency more than it needs registers.
// PRING: the ring is the precise-phase one (comps >= kCompsPrec), which also
// takes the lo part of each position offset -- a build of its own, so that the
// FP64-bound common build carries none of that work.
template <bool PRING>
__global__ void __launch_bounds__(64, 8) ingest_kernel(const IngestParams p)
{
    const int64_t cnt = p.count ? p.count : p.n_in - p.first;
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int nseg = p.n_seg > 1 ? p.n_seg : 1;
    if (q >= cnt * nseg) return;
    const int g = (int)(q / cnt);                // time segment
    const int64_t k = q - (int64_t)g * cnt;
    const int64_t i = p.first + k;
    const int64_t ld = p.ld ? p.ld : p.n_in;    // input particle stride
    const int64_t xi = i - p.xoff;              // input column of particle i
    int64_t s_begin, s_end;
    segment_range(p, g, s_begin, s_end);
    const int n_loc = (int)(s_end - s_begin);   // calls of this thread
    const int64_t t0 = s_begin - p.step0;       // its first input row
    int sp = 0;
    while (sp + 1 < p.n_species && i >= p.in_off[sp + 1]) ++sp;
    const int64_t col = p.col_off[sp] + (i - p.in_off[sp]);
    const int64_t nc = p.ncols;
    const int64_t tile = col / kTileP, pp = col % kTileP;

    double xp[3], off[3], rp[3], up[3], ra[3];   // off = L n (n the image count), exact
    const double half_L = 0.5 * p.box_L;
    const bool box = p.box_L > 0.0;
    bool have_state = s_begin > 0;
    // ring slot, position in the anchor block and anchor block of the next
    // sample m (nsub = 1), advanced by counters instead of 64-bit divisions
    int64_t m_next = s_begin > 0 ? s_begin - 1 : 0;
    // (nblk is 0 for an FP64 ring, which has no anchors)
    int64_t slot_n = m_next % p.ring, kpos_n = m_next % p.K;
    int64_t blk_n = p.nblk > 0 ? (m_next / p.K) % p.nblk : 0;
    if (have_state) {
        for (int c = 0; c < 3; ++c) {
            // image count at the launch start, plus the earlier segments' changes
            double n0 = p.step0 > 0 ? p.r_prev[c * nc + col] : 0.0;
            for (int h = 0; h < g; ++h) n0 += (double)p.wind[((int64_t)h * 3 + c) * cnt + k];
            off[c] = box ? p.box_L * n0 : 0.0;
            if (g == 0) {
                xp[c] = p.x_prev[c * nc + col];
                up[c] = p.u_prev[c * nc + col];
            } else {
                xp[c] = p.x[(t0 - 1) * 3 * ld + c * ld + xi];
                up[c] = p.u[(t0 - 1) * 3 * ld + c * ld + xi];
            }
            rp[c] = xp[c] + off[c];
        }
    }
    bool have_anchor = false;
    bool bad = false;

    // the next step's inputs are loaded while this step is being processed
    double xq[3], uq[3];
    for (int c = 0; c < 3; ++c) {
        xq[c] = n_loc > 0 ? p.x[t0 * 3 * ld + c * ld + xi] : 0.0;
        uq[c] = n_loc > 0 ? p.u[t0 * 3 * ld + c * ld + xi] : 0.0;
    }
    for (int t = 0; t < n_loc; ++t) {
        const int64_t s = s_begin + t;
        double xn[3], un[3], rn[3];
        for (int c = 0; c < 3; ++c) {
            xn[c] = xq[c];
            un[c] = uq[c];
        }
        if (t + 1 < n_loc) {
            const double* xs = p.x + (t0 + t + 1) * 3 * ld;
            const double* us = p.u + (t0 + t + 1) * 3 * ld;
            for (int c = 0; c < 3; ++c) {
                xq[c] = xs[c * ld + xi];
                uq[c] = us[c * ld + xi];
            }
        }
        if (p.check) {
            for (int c = 0; c < 3; ++c) bad |= !isfinite(xn[c]) || !isfinite(un[c]);
        }
        if (s == 0) {
            for (int c = 0; c < 3; ++c) {
                xp[c] = xn[c];
                off[c] = 0.0;
                rp[c] = xn[c];
                up[c] = un[c];
            }
            continue;
        }
        // unwrapped position of this call: r = x + L n, n counting box crossings
        // (L n, exact, changes only at a crossing)
        for (int c = 0; c < 3; ++c) {
            const double jump = image_jump(xn[c] - xp[c], p.box_L, half_L);
            if (jump != 0.0) off[c] -= p.box_L * jump;      // exact: integer multiples of L
            rn[c] = xn[c] + off[c];
        }

        // sample m = s - 1: r_m = rp, u_{m-1/2} = up, u_{m+1/2} = un
        const int64_t m = s - 1;
        const int64_t slot = slot_n, kpos = kpos_n, blk = blk_n;
        if (++slot_n == p.ring) slot_n = 0;
        if (++kpos_n == p.K) {
            kpos_n = 0;
            if (++blk_n == p.nblk) blk_n = 0;
        }
        if (p.nsub > 1) {
            // Sub-cycling (Sec. 2.2: tracked particles sub-cycled at
            // dt_synth <= dt_sim / 10): n sub-samples per PIC sample at
            // tau = (k + 1/2)/n - 1/2, u(tau) = ubar + tau du linear in time
            // between the half-step states, betadot the exact derivative of
            // u/gamma(u) for that u, r(tau) = r_m + dt * Simpson integral of
            // beta over [0, tau].  Sub-sample M = m n + k lives in ring slot
            // M mod ring; the samples' selector flags are those of sample m.
            double ub[3], du[3], b0[3];
            for (int c = 0; c < 3; ++c) {
                ub[c] = 0.5 * (up[c] + un[c]);
                du[c] = un[c] - up[c];
            }
            const double g0 = sqrt(1.0 + (ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2]));
            for (int c = 0; c < 3; ++c) b0[c] = ub[c] / g0;
            const uint32_t flags = p.n_sel ? selector_bits(p, xp, ub) : 0xffffffffu;
            for (int k = 0; k < p.nsub; ++k) {
                const double tau = (k + 0.5) / p.nsub - 0.5;
                double uk[3], uh[3], bk[3], bh[3], bd[3], rk[3];
                for (int c = 0; c < 3; ++c) {
                    uk[c] = ub[c] + tau * du[c];
                    uh[c] = ub[c] + 0.5 * tau * du[c];
                }
                const double gk2 = 1.0 + (uk[0] * uk[0] + uk[1] * uk[1] + uk[2] * uk[2]);
                const double gk = sqrt(gk2);
                const double gh = sqrt(1.0 + (uh[0] * uh[0] + uh[1] * uh[1] + uh[2] * uh[2]));
                const double udot_u = (uk[0] * du[0] + uk[1] * du[1] + uk[2] * du[2]) / p.dt;
                for (int c = 0; c < 3; ++c) {
                    bk[c] = uk[c] / gk;
                    bh[c] = uh[c] / gh;
                    bd[c] = (du[c] / p.dt) / gk - uk[c] * udot_u / (gk2 * gk);
                    rk[c] = rp[c] + p.dt * (tau / 6.0) * (b0[c] + 4.0 * bh[c] + bk[c]);
                }
                const int64_t M = m * p.nsub + k;
                const int64_t sl = M % p.ring;
                if (p.slab32) {
                    float* an = p.anc32 + (tile * p.nblk + (M / p.K) % p.nblk) * (6 * kTileP) + pp;
                    if ((M % p.K) == 0 || !have_anchor) {
                        if ((M % p.K) == 0) {
                            for (int c = 0; c < 3; ++c) {
                                const float hi = (float)rk[c];
                                const float lo = (float)(rk[c] - (double)hi);
                                an[c * kTileP] = hi;
                                an[(3 + c) * kTileP] = lo;
                                ra[c] = (double)hi + (double)lo;
                            }
                        } else {
                            for (int c = 0; c < 3; ++c)
                                ra[c] = (double)an[c * kTileP] + (double)an[(3 + c) * kTileP];
                        }
                        have_anchor = true;
                    }
                    float* o = p.slab32 + (tile * p.ring + sl) * (p.comps * kTileP) + pp;
                    for (int c = 0; c < 3; ++c) {
                        const double d = rk[c] - ra[c];
                        const float dh = (float)d;
                        o[c * kTileP] = dh;
                        if (PRING) o[(11 + c) * kTileP] = (float)(d - (double)dh);
                        o[(3 + c) * kTileP] = (float)bk[c];
                        o[(6 + c) * kTileP] = (float)bd[c];
                    }
                    o[9 * kTileP] = (float)(1.0 / gk2);
                    if (p.comps > kCompsPlain) o[10 * kTileP] = __uint_as_float(flags);
                } else {
                    double* o = p.slab64 + (tile * p.ring + sl) * (p.comps * kTileP) + pp;
                    for (int c = 0; c < 3; ++c) {
                        o[c * kTileP] = rk[c];
                        o[(3 + c) * kTileP] = bk[c];
                        o[(6 + c) * kTileP] = bd[c];
                    }
                    o[9 * kTileP] = 1.0 / gk2;
                    if (p.comps > kCompsPlain) o[10 * kTileP] = (double)flags;
                }
            }
        } else if (p.slab32) {
            // FP32 ring: the only cancellation-prone quantities are differenced
            // in FP64 -- du = u_{m+1/2} - u_{m-1/2} and r_m - r_anchor -- and the
            // rest is evaluated in FP32 through the rearrangement
            //   beta_+ - beta_- = du/g_+ - u_- (du.(u_+ + u_-)) / (g_+ g_- (g_+ + g_-)),
            // which has no cancellation for the magnetic (du perpendicular to u)
            // and weakly parallel accelerations a frozen-field push produces.
            // anchor position r_a as an FP32 hi + lo pair; dr is taken relative
            // to exactly hi + lo, the value the accumulation kernel sees
            float* an = p.anc32 + (tile * p.nblk + blk) * (6 * kTileP) + pp;
            if (kpos == 0) {
                for (int c = 0; c < 3; ++c) {
                    const float hi = (float)rp[c];
                    const float lo = (float)(rp[c] - (double)hi);
                    an[c * kTileP] = hi;
                    an[(3 + c) * kTileP] = lo;
                    ra[c] = (double)hi + (double)lo;
                }
                have_anchor = true;
            } else if (!have_anchor) {
                for (int c = 0; c < 3; ++c) ra[c] = (double)an[c * kTileP] + (double)an[(3 + c) * kTileP];
                have_anchor = true;
            }
            float um[3], uq[3], du[3], ub[3];
            for (int c = 0; c < 3; ++c) {
                um[c] = (float)up[c];
                uq[c] = (float)un[c];
                du[c] = (float)(un[c] - up[c]);
                ub[c] = 0.5f * (um[c] + uq[c]);
            }
            const float gm = sqrtf(1.0f + (um[0] * um[0] + um[1] * um[1] + um[2] * um[2]));
            const float gq = sqrtf(1.0f + (uq[0] * uq[0] + uq[1] * uq[1] + uq[2] * uq[2]));
            const float gb2 = 1.0f + (ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2]);
            const float igb = rsqrtf(gb2);
            const float dus = du[0] * (uq[0] + um[0]) + du[1] * (uq[1] + um[1]) +
                              du[2] * (uq[2] + um[2]);
            const float igq = 1.0f / gq;
            const float corr = dus / (gq * gm * (gq + gm));
            const float idt = (float)(1.0 / p.dt);
            float* o = p.slab32 + (tile * p.ring + slot) * (p.comps * kTileP) + pp;
            for (int c = 0; c < 3; ++c) {
                const double d = rp[c] - ra[c];
                const float dh = (float)d;
                o[c * kTileP] = dh;
                // precise-phase ring: the rounding of the offset as its lo part
                if (PRING) o[(11 + c) * kTileP] = (float)(d - (double)dh);
            }
            o[3 * kTileP] = ub[0] * igb;
            o[4 * kTileP] = ub[1] * igb;
            o[5 * kTileP] = ub[2] * igb;
            o[6 * kTileP] = (du[0] * igq - um[0] * corr) * idt;
            o[7 * kTileP] = (du[1] * igq - um[1] * corr) * idt;
            o[8 * kTileP] = (du[2] * igq - um[2] * corr) * idt;
            o[9 * kTileP] = 1.0f / gb2;
            if (p.comps > kCompsPlain) {
                double ubd[3] = {__dmul_rn(0.5, __dadd_rn(up[0], un[0])),
                                 __dmul_rn(0.5, __dadd_rn(up[1], un[1])),
                                 __dmul_rn(0.5, __dadd_rn(up[2], un[2]))};
                o[10 * kTileP] = __uint_as_float(p.n_sel ? selector_bits(p, xp, ubd) : 0xffffffffu);
            }
        } else {
            double ub[3];
            for (int c = 0; c < 3; ++c) ub[c] = 0.5 * (up[c] + un[c]);
            const double gm = sqrt(1.0 + (up[0] * up[0] + up[1] * up[1] + up[2] * up[2]));
            const double gp = sqrt(1.0 + (un[0] * un[0] + un[1] * un[1] + un[2] * un[2]));
            const double gb2 = 1.0 + (ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2]);
            const double gb = sqrt(gb2);
            double* o = p.slab64 + (tile * p.ring + slot) * (p.comps * kTileP) + pp;
            o[0 * kTileP] = rp[0];
            o[1 * kTileP] = rp[1];
            o[2 * kTileP] = rp[2];
            for (int c = 0; c < 3; ++c) {
                o[(3 + c) * kTileP] = ub[c] / gb;
                o[(6 + c) * kTileP] = (un[c] / gp - up[c] / gm) / p.dt;
            }
            o[9 * kTileP] = 1.0 / gb2;
            if (p.comps > kCompsPlain) {
                double ubd[3] = {__dmul_rn(0.5, __dadd_rn(up[0], un[0])),
                                 __dmul_rn(0.5, __dadd_rn(up[1], un[1])),
                                 __dmul_rn(0.5, __dadd_rn(up[2], un[2]))};
                o[10 * kTileP] = (double)(p.n_sel ? selector_bits(p, xp, ubd) : 0xffffffffu);
            }
        }
        for (int c = 0; c < 3; ++c) {
            xp[c] = xn[c];
            rp[c] = rn[c];
            up[c] = un[c];
        }
    }
    if (g == nseg - 1) {                        // the launch's last segment carries the state on
        if (nseg > 1) {
            // segment 0 may still be reading the state arrays: stage it
            for (int c = 0; c < 3; ++c) {
                p.state_out[c * cnt + k] = xp[c];
                p.state_out[(3 + c) * cnt + k] = box ? off[c] / p.box_L : 0.0;   // exact
                p.state_out[(6 + c) * cnt + k] = up[c];
            }
        } else {
            for (int c = 0; c < 3; ++c) {
                p.x_prev[c * nc + col] = xp[c];
                p.r_prev[c * nc + col] = box ? off[c] / p.box_L : 0.0;
                p.u_prev[c * nc + col] = up[c];
            }
        }
    }
    if (bad) atomicOr(p.err_word, kErrNaN);
}

// The staged carry-over state of a segmented launch into the state arrays.
__global__ void store_state(const IngestParams p)
{
    const int64_t cnt = p.count ? p.count : p.n_in - p.first;
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= cnt) return;
    const int64_t i = p.first + k;
    int sp = 0;
    while (sp + 1 < p.n_species && i >= p.in_off[sp + 1]) ++sp;
    const int64_t col = p.col_off[sp] + (i - p.in_off[sp]);
    for (int c = 0; c < 3; ++c) {
        p.x_prev[c * p.ncols + col] = p.state_out[c * cnt + k];
        p.r_prev[c * p.ncols + col] = p.state_out[(3 + c) * cnt + k];
        p.u_prev[c * p.ncols + col] = p.state_out[(6 + c) * cnt + k];
    }
}

IngestKernels ingest_kernel_ptr()
{
    return {reinterpret_cast<const void*>(&ingest_kernel<false>),
            reinterpret_cast<const void*>(&ingest_kernel<true>)};
}

cudaError_t launch_ingest(const IngestParams& p, cudaStream_t st)
{
    const int64_t cnt = p.count ? p.count : p.n_in - p.first;
    if (cnt <= 0 || p.n_steps == 0) return cudaSuccess;
    IngestParams q = p;
    q.n_seg = 1;
    // time segments only when the particles alone leave the GPU idle: with
    // 32,768 or more one thread per particle already keeps the FP64 pipes of
    // all SMs busy, and the segments' extra pass only adds work (measured)
    constexpr int64_t kSegMaxParticles = 32768;
    if (p.wind && p.state_out && p.seg_len > 0 && cnt < kSegMaxParticles) {
        // boundaries at calls 1 + j seg_len strictly inside (step0, step0 + n_steps)
        // at most kMaxSeg segments (each thread sums the earlier segments' counts):
        // longer batches get longer segments, still multiples of seg_len
        constexpr int64_t kMaxSeg = 256;
        const int64_t end = p.step0 + p.n_steps;
        int64_t len = p.seg_len;
        const int64_t span = p.n_steps / (kMaxSeg - 1) + 1;
        if (span > len) len = (span + p.seg_len - 1) / p.seg_len * p.seg_len;
        const int64_t j0 = p.step0 < 1 ? 0 : (p.step0 - 1) / len + 1;
        const int64_t first = 1 + j0 * len;
        if (first < end) {
            q.seg_len = (int32_t)len;
            q.seg_first = first;
            q.n_seg = (int32_t)(1 + (end - first + len - 1) / len);
        }
    }
    // one thread per particle, small blocks: the kernel is bound by its FP64
    // work per SM, so the blocks must spread evenly over all 152 SMs (256-thread
    // blocks left 65,536 particles at two blocks on most SMs and one on the rest,
    // and a 16,384-particle share on 64 SMs)
    const int threads = 64;
    if (q.n_seg > 1 && q.box_L > 0.0) {
        const int64_t nw = cnt * (q.n_seg - 1);
        wind_kernel<<<(unsigned)((nw + 255) / 256), 256, 0, st>>>(q);
    }
    const int64_t blocks = (cnt * q.n_seg + threads - 1) / threads;
    if (q.slab32 && q.comps >= kCompsPrec)
        ingest_kernel<true><<<(unsigned)blocks, threads, 0, st>>>(q);
    else
        ingest_kernel<false><<<(unsigned)blocks, threads, 0, st>>>(q);
    if (q.n_seg > 1) store_state<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(q);
    return cudaGetLastError();
}

}  // namespace rad
