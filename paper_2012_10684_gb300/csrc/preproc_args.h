// Arguments of the pre-processing and morphology kernel (preproc.cuh):
// CT numbers to 8-bit levels, flat disk erosion/dilation per slice,
// chest-mask subtraction, 256-level histograms. Ops follow tsallis_morph_op.
#pragma once
#include <cstdint>

namespace tsl {

constexpr int kPreMaxRadius = 15;
struct PreArgs {
    const int16_t* vol;     // [nz][ny][nx]
    int16_t* out;           // [nz][ny][nx] levels 0..255, or null
    int* hist;              // [nz][256] (per_slice) or [256], zeroed by the caller, or null
    int nx, ny, nz;
    int background, hu_min, hu_max;
    int D;                  // hu_max - hu_min
    unsigned long long magic;   // floor(n / (2D)) == umulhi(n, magic) >> shift for every n the map forms
    int shift;
    int op, radius, per_slice;
    int ntx, nty;           // tiles per slice in x and y
    unsigned* check;        // checked build: first failing index check (checked.cuh)
};

}  // namespace tsl
