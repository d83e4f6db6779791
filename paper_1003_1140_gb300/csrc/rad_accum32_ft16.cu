// rad_accum32_ft16.cu -- instantiations of the FP32 split-phase kernel
// for the (frequencies per thread, polynomial frequencies, blocks per SM)
// families (16,0,2) and (16,4,2); see rad_accum32.cuh.
#include "rad_accum32.cuh"

namespace rad {

#define FN(FT, NP, K, COH, MB)                                            \
    do {                                                                  \
        if (p) *err = launch32_one<FT, NP, K, COH, MB>(*p, grid, st);     \
        else *nb = blocks32_one<FT, NP, K, COH, MB>();                    \
        return true;                                                      \
    } while (0)

bool accum32_ft16(const Accum32Params* p, const Accum32Config& cfg, int grid,
                     cudaStream_t st, cudaError_t* err, int* nb)
{
    RAD_ACCUM32_FAMILY(16,0,2)
    RAD_ACCUM32_FAMILY(16,4,2)
    return false;
}

}  // namespace rad
