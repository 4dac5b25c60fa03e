// Kernel instance: FP64 root iterations, repair pass of crossings that failed
// the slope test (four warps per position, one sample per lane).
#include "kernels.cuh"

namespace tw {
TW_DEFINE_REPAIR_LAUNCHER(0)
}
