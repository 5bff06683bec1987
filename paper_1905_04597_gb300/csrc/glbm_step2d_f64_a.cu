// FP64 instantiations of the fused 2D stream-collide kernel, levels 1 2 3 4 5.
#include "glbm_step2d_launch.cuh"

template cudaError_t glbm_step2d_level<1, double>(int, const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_level<2, double>(int, const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_level<3, double>(int, const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_level<4, double>(int, const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_level<5, double>(int, const Step2DArgs &, int, cudaStream_t);
