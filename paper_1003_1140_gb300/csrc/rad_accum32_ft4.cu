// rad_accum32_ft4.cu -- instantiations of the FP32 split-phase kernel with 4
// frequencies per thread at 4 resident blocks per SM (fewer registers per
// thread, more warps to hide the special-function unit's latency), SFU only;
// see rad_accum32.cuh.
#include "rad_accum32.cuh"

namespace rad {

#define FN(FT, NP, K, COH, MB)                                            \
    do {                                                                  \
        if (p) *err = launch32_one<FT, NP, K, COH, MB>(*p, grid, st);     \
        else *nb = blocks32_one<FT, NP, K, COH, MB>();                    \
        return true;                                                      \
    } while (0)

bool accum32_ft4(const Accum32Params* p, const Accum32Config& cfg, int grid,
                 cudaStream_t st, cudaError_t* err, int* nb)
{
    RAD_ACCUM32_FAMILY(4,0,4)
    return false;
}

}  // namespace rad
