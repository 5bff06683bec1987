// 2N+2-hierarchy instantiations of the fused 2D step (float), levels 1 2 3 4.
#include "glbm_step2d_zv.cuh"

template cudaError_t glbm_step2d_zv_level<1, float>(int, int, const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_zv_level<2, float>(int, int, const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_zv_level<3, float>(int, int, const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_zv_level<4, float>(int, int, const Step2DArgs &, int, cudaStream_t);
