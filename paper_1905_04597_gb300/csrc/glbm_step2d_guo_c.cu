// Instantiations of the fused 2D step with Guo's force (float, kind GLBM_GUOK_X1), levels 1-8.
#include "glbm_step2d_guo.cuh"

template cudaError_t glbm_step2d_guo_level<1, float, GLBM_GUOK_X1>(const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_guo_level<2, float, GLBM_GUOK_X1>(const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_guo_level<3, float, GLBM_GUOK_X1>(const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_guo_level<4, float, GLBM_GUOK_X1>(const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_guo_level<5, float, GLBM_GUOK_X1>(const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_guo_level<6, float, GLBM_GUOK_X1>(const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_guo_level<7, float, GLBM_GUOK_X1>(const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_guo_level<8, float, GLBM_GUOK_X1>(const Step2DArgs &, int, cudaStream_t);
