// Pre-processing kernel instantiations for radii 0, 1, 2, 3, 4, 5, 6, 7.
#include "preproc.cuh"

namespace tsl {
namespace pre {
TSL_PREPROC_INSTANTIATE(0)
TSL_PREPROC_INSTANTIATE(1)
TSL_PREPROC_INSTANTIATE(2)
TSL_PREPROC_INSTANTIATE(3)
TSL_PREPROC_INSTANTIATE(4)
TSL_PREPROC_INSTANTIATE(5)
TSL_PREPROC_INSTANTIATE(6)
TSL_PREPROC_INSTANTIATE(7)
}  // namespace pre
}  // namespace tsl
