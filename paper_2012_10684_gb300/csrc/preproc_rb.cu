// Pre-processing kernel instantiations for radii 8, 9, 10.
#include "preproc.cuh"

namespace tsl {
namespace pre {
TSL_PREPROC_INSTANTIATE(8)
TSL_PREPROC_INSTANTIATE(9)
TSL_PREPROC_INSTANTIATE(10)
}  // namespace pre
}  // namespace tsl
