// Pre-processing kernel instantiations for radii 13.
#include "preproc.cuh"

namespace tsl {
namespace pre {
TSL_PREPROC_INSTANTIATE(13)
}  // namespace pre
}  // namespace tsl
