// Kernel instance: FP64 root iterations, 2 new limb samples per lane per
// iteration, compiled for 4 CTAs per SM.
#include "kernels.cuh"

namespace tw {
TW_DEFINE_LAUNCHER_OCC(0, 2, 4)
}
