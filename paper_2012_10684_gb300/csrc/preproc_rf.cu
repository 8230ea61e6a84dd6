// Pre-processing kernel instantiations for radii 15.
#include "preproc.cuh"

namespace tsl {
namespace pre {
TSL_PREPROC_INSTANTIATE(15)
}  // namespace pre
}  // namespace tsl
