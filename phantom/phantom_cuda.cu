/* Device build of the phantom generator: one thread per voxel row segment.
 * The descriptor's capsule and CSR pointers must be device pointers. */
#include "phantom.h"
#include <cuda_runtime.h>

__global__ void ph_generate_kernel(ph_desc d, int16_t* __restrict__ out) {
    int64_t z = blockIdx.y;
    int64_t nrow = d.ny * d.nx;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nrow;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t y = i / d.nx, x = i - y * d.nx;
        out[z * nrow + i] = ph_voxel(&d, z, y, x);
    }
}

extern "C" int ph_generate_cuda(const ph_desc* h_desc, int16_t* d_out, void* stream) {
    if (!h_desc || !d_out || h_desc->nx <= 0 || h_desc->ny <= 0 || h_desc->nz <= 0) return 1;
    if (h_desc->nx > 16384 || h_desc->ny > 16384 || h_desc->nz > 65535) return 1;
    int64_t nrow = h_desc->nx * h_desc->ny;
    int gx = (int)((nrow + 255) / 256);
    if (gx > 1024) gx = 1024;
    dim3 grid(gx, (unsigned)h_desc->nz);
    ph_generate_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(*h_desc, d_out);
    return cudaGetLastError() == cudaSuccess ? 0 : 4;
}
