// Instantiations of the fused 2D step with Guo's force (double, kind GLBM_GUOK_ZV), levels 1-8.
#include "glbm_step2d_guo.cuh"

template cudaError_t glbm_step2d_guo_level<1, double, GLBM_GUOK_ZV>(const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_guo_level<2, double, GLBM_GUOK_ZV>(const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_guo_level<3, double, GLBM_GUOK_ZV>(const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_guo_level<4, double, GLBM_GUOK_ZV>(const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_guo_level<5, double, GLBM_GUOK_ZV>(const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_guo_level<6, double, GLBM_GUOK_ZV>(const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_guo_level<7, double, GLBM_GUOK_ZV>(const Step2DArgs &, int, cudaStream_t);
template cudaError_t glbm_step2d_guo_level<8, double, GLBM_GUOK_ZV>(const Step2DArgs &, int, cudaStream_t);
