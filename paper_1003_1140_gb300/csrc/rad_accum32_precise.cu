// rad_accum32_precise.cu -- instantiations of the FP32 split-phase kernel with
// the precise offset phase (nu dphi in float-float, reduced to one turn before
// the special-function unit): 8 SFU frequencies per thread, ring anchor
// interval 32, 2 or 3 blocks per SM; see rad_accum32.cuh.
#include "rad_accum32.cuh"

namespace rad {

#define FN(COH, MB)                                                                  \
    do {                                                                             \
        if (p) *err = launch32_one<8, 0, 32, COH, MB, false, true>(*p, grid, st);    \
        else *nb = blocks32_one<8, 0, 32, COH, MB, false, true>();                   \
        return true;                                                                 \
    } while (0)

bool accum32_precise(const Accum32Params* p, const Accum32Config& cfg, int grid,
                     cudaStream_t st, cudaError_t* err, int* nb)
{
    if (cfg.ft != 8 || cfg.np != 0 || cfg.K != 32) return false;
    if (cfg.mb == 2) { if (cfg.coh) FN(true, 2); else FN(false, 2); }
    if (cfg.mb == 3) { if (cfg.coh) FN(true, 3); else FN(false, 3); }
    return false;
}

}  // namespace rad
