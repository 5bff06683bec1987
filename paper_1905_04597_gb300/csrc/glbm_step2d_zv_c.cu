// 2N+2-hierarchy instantiations of the fused 2D step (double), levels 1 2 3 4 5.
#include "glbm_step2d_zv.cuh"

template cudaError_t glbm_step2d_zv_level<1, double>(int, int, const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_zv_level<2, double>(int, int, const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_zv_level<3, double>(int, int, const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_zv_level<4, double>(int, int, const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_zv_level<5, double>(int, int, const Step2DArgs &, int, cudaStream_t);
