// Checked build (compiled with -DTSALLIS_CHECKED, into its own library): the
// kernels test computed indices against the extents of the buffers they
// address. A failed test records its site number in *check (the first
// failure wins) and the access it guards is skipped; the host reads and
// clears the word with tsallis_check_status. This stands in for a memory
// sanitizer on GPUs where none may run. In normal builds every test is the
// constant true and compiles away.
#pragma once

namespace tsl {

#ifdef TSALLIS_CHECKED
constexpr bool kCheckedBuild = true;
__device__ __forceinline__ bool in_range(long long i, long long n, unsigned* check, unsigned site) {
    if (i >= 0 && i < n) return true;
    if (check) atomicCAS(check, 0u, site);
    return false;
}
#else
constexpr bool kCheckedBuild = false;
__device__ __forceinline__ bool in_range(long long, long long, unsigned*, unsigned) { return true; }
#endif

// Site numbers (reported by tsallis_check_status).
enum CheckSite : unsigned {
    kSiteSegGroup = 101,      // tile kernel: work item's group
    kSiteSegTile = 102,       // tile kernel: work item's tile within its group
    kSiteSegQueue = 103,      // tile kernel: binarise queue position
    kSitePreStage = 201,      // pre-processing: shared tile word being staged
    kSitePreVol = 202,        // pre-processing: voxel read
    kSitePreWindow = 203,     // pre-processing: rows/words a disk run reads
    kSitePreMid = 204,        // pre-processing: intermediate word written
    kSitePreOut = 205,        // pre-processing: output voxel written
    kSitePreHist = 206,       // pre-processing: histogram level
    kSite2dTables = 301,      // 2-D search: table entries of a pair
    kSite2dCell = 302,        // 2-D window: candidate cell
    kSite2dBrute = 303,       // 2-D brute force: histogram row
    kSiteSpecSlice = 401,     // predicted first pass: job's slice
    kSiteSpecPatch = 402,     // predicted first pass: listed position rewritten
    kSiteSpecQueue = 403,     // predicted first pass: second-pass queue position
    kSitePipeChunk = 501,     // pipelined per-slice kernel: chunk's slice
    kSitePipePatch = 502,     // pipelined per-slice kernel: listed position rewritten
};

}  // namespace tsl
