// Internal interface between the C-ABI layer (api.cu) and the kernel
// translation units. Host-side only declarations plus the argument structs
// that are passed by value to the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tsl {

constexpr int kMaxLevels = 4096;  // largest 1-D histogram

// Scratch header that lives at the start of a context's device scratch.
// It starts zeroed and every launch leaves it as it found it (the last block
// to finish resets the ticket and done counters and bumps the epoch), so no
// memset is needed between launches and CUDA-graph replays are safe.
struct ScratchHeader {
    unsigned int ticket;  // next work item
    unsigned int done;    // blocks that have finished
    int epoch;            // launches so far; ready flags are compared to epoch + 1
    int err;              // a device wait ran out or an arrival was skipped
    int pad[12];
};

enum Phase : int { kPhaseHist = 1, kPhaseSearch = 2, kPhaseBin = 4 };

// One work item of a batch: a histogram group and a tile of it.
struct WorkItem {
    int group;  // histogram group
    int tile;   // tile index within the group; bit 31 set for a binarise tile
};

// A group (one histogram): voxel range and where its mask goes.
struct GroupDesc {
    const int16_t* vol;
    uint8_t* mask;
    long long nvox;
    int ntiles;
    int pad;
};

struct SegArgs {
    const int16_t* vol;     // uniform groups: group g starts at vol + g * group_vox
    uint8_t* mask;
    long long group_vox;
    int ngroups;
    int ntiles;             // tiles per group (uniform groups)
    int tile_vox;           // voxels per tile, multiple of 8
    int lag;                // binarise tiles of group s - lag follow histogram tiles of group s
    unsigned int nticket;   // number of work items
    const GroupDesc* groups;   // non-null: batch with an explicit work list
    const WorkItem* worklist;
    int lo, L;
    float q;
    int polarity;
    int bin_shift;          // threshold applies to level >> bin_shift (2-D grey levels)
    int phases;
    unsigned int flags;
    unsigned long long timeout_ns;
    ScratchHeader* hdr;
    int* arrive;            // [ngroups]
    int* ready;             // [ngroups]
    int* tmo;               // [ngroups]: epoch + 1 when a wait on the group ran out
    int* ghist;             // [ngroups][L]: histogram target (scratch or caller's)
    const int* t_in;        // binarise-only: caller's thresholds
    int* t_out;
    float* phi_out;
    int* status;
    float* curve;           // optional [ngroups][L-1]
};

// Kernel launchers (seg1d.cu).
cudaError_t launch_segment1d(const SegArgs& a, int grid, int copies, cudaStream_t s);
cudaError_t launch_search1d(const int32_t* hist, long long nh, int L, float q, int32_t* t, float* phi,
                            int32_t* status, float* curve, cudaStream_t s);
int segment1d_threads();
int segment1d_smem_bytes(int L, int copies);
cudaError_t segment1d_occupancy(int copies, int L, int* blocks_per_sm);

}  // namespace tsl
