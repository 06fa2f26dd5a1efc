// Batched transfer launch with the level orders of the stage (k_levels.cu): the level pairs
// of the coarsening rule run with compile-time orders, any other pair with the orders read
// at run time.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

namespace pmg {

cudaError_t transfer_batch_launch_pair(const void* table, int restrict_, int Pf, int Pc, int nctas, int threads,
                                       size_t smem, cudaStream_t st);

}  // namespace pmg
