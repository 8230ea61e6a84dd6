// Radius dispatch of the pre-processing and morphology kernel (preproc.cuh).
#include "preproc.cuh"

namespace tsl {
namespace pre {
#define TSL_PREPROC_DECLARE(R)                                              \
    extern template cudaError_t prepare_r<R>();                             \
    extern template cudaError_t launch_r<R>(const PreArgs&, cudaStream_t);
TSL_PREPROC_DECLARE(0) TSL_PREPROC_DECLARE(1) TSL_PREPROC_DECLARE(2) TSL_PREPROC_DECLARE(3)
TSL_PREPROC_DECLARE(4) TSL_PREPROC_DECLARE(5) TSL_PREPROC_DECLARE(6) TSL_PREPROC_DECLARE(7)
TSL_PREPROC_DECLARE(8) TSL_PREPROC_DECLARE(9) TSL_PREPROC_DECLARE(10) TSL_PREPROC_DECLARE(11)
TSL_PREPROC_DECLARE(12) TSL_PREPROC_DECLARE(13) TSL_PREPROC_DECLARE(14) TSL_PREPROC_DECLARE(15)

namespace {
template <int... Rs>
struct RadiusTable;
template <>
struct RadiusTable<> {
    static cudaError_t prepare() { return cudaSuccess; }
    static cudaError_t launch(int, const PreArgs&, cudaStream_t) { return cudaErrorInvalidValue; }
};
template <int R0, int... Rs>
struct RadiusTable<R0, Rs...> {
    static cudaError_t prepare() {
        cudaError_t e = prepare_r<R0>();
        return e != cudaSuccess ? e : RadiusTable<Rs...>::prepare();
    }
    static cudaError_t launch(int r, const PreArgs& a, cudaStream_t s) {
        return r == R0 ? launch_r<R0>(a, s) : RadiusTable<Rs...>::launch(r, a, s);
    }
};
using Radii = RadiusTable<0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15>;

}  // namespace
}  // namespace pre

int preproc_tile_w() { return pre::kTW; }
int preproc_tile_h() { return pre::kTH; }

cudaError_t preproc_prepare() { return pre::Radii::prepare(); }

cudaError_t launch_preprocess(const PreArgs& a, cudaStream_t s) {
    if (a.radius < 0 || a.radius > kPreMaxRadius) return cudaErrorInvalidValue;
    if ((long long)a.ntx * a.nty * a.nz > 0x7fffffffll) return cudaErrorInvalidValue;
    return pre::Radii::launch(a.radius, a, s);
}

}  // namespace tsl
