// 2N+2-hierarchy instantiations of the fused 2D step (double), levels 6 7 8.
#include "glbm_step2d_zv.cuh"

template cudaError_t glbm_step2d_zv_level<6, double>(int, int, const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_zv_level<7, double>(int, int, const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_zv_level<8, double>(int, int, const Step2DArgs &, int, cudaStream_t);
