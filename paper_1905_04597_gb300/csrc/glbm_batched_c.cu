// Heterogeneous-batch step kernels, levels 7 8.
#include "glbm_batched.cuh"

template cudaError_t glbm_batched_level<7>(const BatchArgs &, bool, cudaStream_t);
template cudaError_t glbm_batched_level<8>(const BatchArgs &, bool, cudaStream_t);
