// FP32-deviation instantiations of the fused 2D stream-collide kernel, levels 5 6.
#include "glbm_step2d_launch.cuh"

template cudaError_t glbm_step2d_level<5, float>(int, const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_level<6, float>(int, const Step2DArgs &, int, cudaStream_t);
