// Kernel instance: mixed-precision root iterations, 2 new limb samples per lane per
// iteration, compiled for 4 CTAs per SM.
#include "kernels.cuh"

namespace tw {
TW_DEFINE_LAUNCHER_OCC(1, 2, 4)
}
