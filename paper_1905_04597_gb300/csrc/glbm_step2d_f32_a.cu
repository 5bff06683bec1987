// FP32-deviation instantiations of the fused 2D stream-collide kernel, levels 1 2 3 4.
#include "glbm_step2d_launch.cuh"

template cudaError_t glbm_step2d_level<1, float>(int, const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_level<2, float>(int, const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_level<3, float>(int, const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_level<4, float>(int, const Step2DArgs &, int, cudaStream_t);
