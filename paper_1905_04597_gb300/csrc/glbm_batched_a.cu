// Heterogeneous-batch step kernels, levels 1 2 3 4.
#include "glbm_batched.cuh"

template cudaError_t glbm_batched_level<1>(const BatchArgs &, bool, cudaStream_t);
template cudaError_t glbm_batched_level<2>(const BatchArgs &, bool, cudaStream_t);
template cudaError_t glbm_batched_level<3>(const BatchArgs &, bool, cudaStream_t);
template cudaError_t glbm_batched_level<4>(const BatchArgs &, bool, cudaStream_t);
