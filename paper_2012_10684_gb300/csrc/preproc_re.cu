// Pre-processing kernel instantiations for radii 14.
#include "preproc.cuh"

namespace tsl {
namespace pre {
TSL_PREPROC_INSTANTIATE(14)
}  // namespace pre
}  // namespace tsl
