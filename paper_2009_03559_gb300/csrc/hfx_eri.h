// Host-side interface of the ERI kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>
#include "hfx_internal.cuh"

namespace hfx {

struct EriLaunch;

// Group sizes (lanes per quartet): 1 (a thread) or 32 (a warp).  Precision passes `prec`:
// 0 every quartet in FP64; 1 and 2 the FP64 and FP32 shares of a mixed-precision class.
int eri_group_size(int cls);  // default for a class: 1 or 32
bool eri_group_size_valid(int gs);
size_t eri_smem_bytes(int cls, int gs, int streams = 0, int prec = 0);
int eri_block_size();
cudaError_t eri_prepare();
int eri_blocks_per_sm(int cls, int mode, int gs, int prec, bool batch, int streams = 0);
// Streams of the warp kernel (primitive quartets run at a time): 0 = the class default;
// the value a launch with `streams` uses; whether a class has that variant.
int eri_streams(int cls, int streams);
bool eri_streams_valid(int cls, int streams);
int eri_groups_per_block(int gs);

}  // namespace hfx

namespace hfx {
cudaError_t eri_launch(const EriLaunch& L, int cls, int mode, int grid, cudaStream_t stream, int gs, int prec,
                       bool batch, int streams = 0);
}
