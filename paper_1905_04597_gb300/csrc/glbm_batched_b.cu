// Heterogeneous-batch step kernels, levels 5 6.
#include "glbm_batched.cuh"

template cudaError_t glbm_batched_level<5>(const BatchArgs &, bool, cudaStream_t);
template cudaError_t glbm_batched_level<6>(const BatchArgs &, bool, cudaStream_t);
