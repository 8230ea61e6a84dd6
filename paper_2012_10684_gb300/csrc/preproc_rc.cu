// Pre-processing kernel instantiations for radii 11, 12.
#include "preproc.cuh"

namespace tsl {
namespace pre {
TSL_PREPROC_INSTANTIATE(11)
TSL_PREPROC_INSTANTIATE(12)
}  // namespace pre
}  // namespace tsl
