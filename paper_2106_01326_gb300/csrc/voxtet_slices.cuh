// voxtet_slices.cuh -- host interface of the slice-unit kernel (voxtet_slices.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "voxtet_device.cuh"

namespace voxtet {

constexpr int kSuBlock = 128;   // threads per block, and tets per tile (one per thread)
constexpr int kSuSlices = 32;   // most z-slices of a tet's box this kernel takes (5 blocks per SM)
constexpr int kSuSlicesSmall = 16;  // the smaller capacity: less shared memory, 7 blocks per SM
constexpr int kSuRows = 1024;   // most x-rows per slice of a tet's box this kernel takes

// Enqueue the slice-unit kernel for p on `stream`: variant = (strided << 3) | (strict << 2) |
// (cull << 1) | clamp; slices = the most z-slices a tet may span in it (kSuSlicesSmall or
// kSuSlices).  Tets it leaves to the span kernel are listed at the back of p.tetq (count in
// the header's listq_count); the caller launches the span kernel in list mode after it.
// Returns VOXTET_OK or VOXTET_ERR_CUDA.
int launch_slices(const Params &p, int variant, int slices, int sms, cudaStream_t stream);

// Shared memory of one block of the slice-unit kernel with that slice capacity.
size_t slices_smem_bytes(int slices);

}  // namespace voxtet
