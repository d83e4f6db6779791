// rad_accum32_precise.cu -- instantiations of the FP32 split-phase kernel with
// the precise offset phase (nu dphi in float-float, reduced to one turn before
// the special-function unit) for every work item or for the items that ask for
// it: 8 SFU frequencies per thread, ring anchor interval 32, 2 or 3 blocks per
// SM; see rad_accum32.cuh.
#include "rad_accum32.cuh"

namespace rad {

#define FN(COH, MB, PM)                                                              \
    do {                                                                             \
        if (p) *err = launch32_one<8, 0, 32, COH, MB, false, PM>(*p, grid, st);      \
        else *nb = blocks32_one<8, 0, 32, COH, MB, false, PM>();                     \
        return true;                                                                 \
    } while (0)

bool accum32_precise(const Accum32Params* p, const Accum32Config& cfg, int grid,
                     cudaStream_t st, cudaError_t* err, int* nb)
{
    if (cfg.ft != 8 || cfg.np != 0 || cfg.K != 32) return false;
    if (cfg.pm == 1) {
        if (cfg.mb == 2) { if (cfg.coh) FN(true, 2, 1); else FN(false, 2, 1); }
        if (cfg.mb == 3) { if (cfg.coh) FN(true, 3, 1); else FN(false, 3, 1); }
    }
    if (cfg.pm == 2) {
        if (cfg.mb == 2) { if (cfg.coh) FN(true, 2, 2); else FN(false, 2, 2); }
        if (cfg.mb == 3) { if (cfg.coh) FN(true, 3, 2); else FN(false, 3, 2); }
    }
    return false;
}

}  // namespace rad
