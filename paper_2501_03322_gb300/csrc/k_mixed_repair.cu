// Kernel instance: mixed-precision root iterations, repair pass of crossings that failed
// the slope test (two samples per lane).
#include "kernels.cuh"

namespace tw {
TW_DEFINE_REPAIR_LAUNCHER(1)
}
