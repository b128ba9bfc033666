// Host-side interface of the ERI kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>
#include "hfx_internal.cuh"

namespace hfx {

struct EriLaunch;

int eri_group_size(int cls);
size_t eri_smem_bytes(int cls, bool g32);
int eri_block_size();
cudaError_t eri_prepare();
int eri_blocks_per_sm(int cls, int mode, bool g32, bool mixed, bool batch);

}  // namespace hfx

namespace hfx {
cudaError_t eri_launch(const EriLaunch& L, int cls, int mode, int grid, cudaStream_t stream, bool g32, bool mixed,
                       bool batch);
}
