// FP32-deviation instantiations of the fused 2D stream-collide kernel, levels 7 8.
#include "glbm_step2d_launch.cuh"

template cudaError_t glbm_step2d_level<7, float>(int, const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_level<8, float>(int, const Step2DArgs &, int, cudaStream_t);
