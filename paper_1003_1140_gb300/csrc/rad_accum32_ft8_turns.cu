// rad_accum32_ft8_turns.cu -- instantiations of the FP32 accumulation kernel
// with the turns-reduced SFU phase: 8 frequencies per thread, 2 or 3 blocks
// per SM, every anchor interval and both summation modes.
#include "rad_accum32.cuh"

namespace rad {

#define FNT(FT, K, COH, MB)                                                     \
    do {                                                                        \
        if (p) *err = launch32_one<FT, 0, K, COH, MB, true>(*p, grid, st);      \
        else *nb = blocks32_one<FT, 0, K, COH, MB, true>();                     \
        return true;                                                            \
    } while (0)

bool accum32_ft8_turns(const Accum32Params* p, const Accum32Config& cfg, int grid,
                       cudaStream_t st, cudaError_t* err, int* nb)
{
    RAD_ACCUM32_FAMILY_TURNS(8, 2)
    RAD_ACCUM32_FAMILY_TURNS(8, 3)
    return false;
}

}  // namespace rad
