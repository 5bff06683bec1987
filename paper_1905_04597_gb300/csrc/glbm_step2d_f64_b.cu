// FP64 instantiations of the fused 2D stream-collide kernel, levels 6 7 8.
#include "glbm_step2d_launch.cuh"

template cudaError_t glbm_step2d_level<6, double>(int, const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_level<7, double>(int, const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_level<8, double>(int, const Step2DArgs &, int, cudaStream_t);
