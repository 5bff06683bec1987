// 2N+2-hierarchy instantiations of the fused 2D step (float), levels 5 6 7 8.
#include "glbm_step2d_zv.cuh"

template cudaError_t glbm_step2d_zv_level<5, float>(int, int, const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_zv_level<6, float>(int, int, const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_zv_level<7, float>(int, int, const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_zv_level<8, float>(int, int, const Step2DArgs &, int, cudaStream_t);
