// rad_accum32_band.cu -- instantiations of the FP32 split-phase kernel whose
// work items take anchor blocks of K << kmul samples (the anchor interval per
// frequency band under a phase budget): 8 SFU frequencies per thread, 2 or 3
// blocks per SM, ring anchor interval 8 or 16 (a ring anchored every 32 samples
// already has the longest block); see rad_accum32.cuh.
#include "rad_accum32.cuh"

namespace rad {

#define FN(FT, NP, K, COH, MB)                                                 \
    do {                                                                       \
        if (p) *err = launch32_one<FT, NP, K, COH, MB, true>(*p, grid, st);    \
        else *nb = blocks32_one<FT, NP, K, COH, MB, true>();                   \
        return true;                                                           \
    } while (0)

#define RAD_ACCUM32_BAND(MB)                                                         \
    if (cfg.mb == MB) {                                                              \
        if (cfg.K == 8) { if (cfg.coh) FN(8, 0, 8, true, MB); else FN(8, 0, 8, false, MB); }   \
        if (cfg.K == 16) { if (cfg.coh) FN(8, 0, 16, true, MB); else FN(8, 0, 16, false, MB); } \
    }

bool accum32_band(const Accum32Params* p, const Accum32Config& cfg, int grid,
                  cudaStream_t st, cudaError_t* err, int* nb)
{
    if (cfg.ft != 8 || cfg.np != 0) return false;
    RAD_ACCUM32_BAND(2)
    RAD_ACCUM32_BAND(3)
    return false;
}

}  // namespace rad
