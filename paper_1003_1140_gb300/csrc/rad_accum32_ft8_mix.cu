// rad_accum32_ft8_mix.cu -- instantiations of the FP32 split-phase kernel
// for the (frequencies per thread, polynomial frequencies, blocks per SM)
// families (8,2,2), (8,2,3), (8,1,2) and (8,1,3); see rad_accum32.cuh.
#include "rad_accum32.cuh"

namespace rad {

#define FN(FT, NP, K, COH, MB)                                            \
    do {                                                                  \
        if (p) *err = launch32_one<FT, NP, K, COH, MB>(*p, grid, st);     \
        else *nb = blocks32_one<FT, NP, K, COH, MB>();                    \
        return true;                                                      \
    } while (0)

bool accum32_ft8_mix(const Accum32Params* p, const Accum32Config& cfg, int grid,
                     cudaStream_t st, cudaError_t* err, int* nb)
{
    RAD_ACCUM32_FAMILY(8,2,2)
    RAD_ACCUM32_FAMILY(8,2,3)
    RAD_ACCUM32_FAMILY(8,1,2)
    RAD_ACCUM32_FAMILY(8,1,3)
    return false;
}

}  // namespace rad
