// 2N+2-hierarchy instantiations of the fused 2D step (double), levels 9 10 11 12 13 (D1Q3 x D1Q(2N+2) only).
#include "glbm_step2d_zv.cuh"

template cudaError_t glbm_step2d_zv_level<9, double>(int, int, const Step2DArgsHi &, int, cudaStream_t);
template cudaError_t glbm_step2d_zv_level<10, double>(int, int, const Step2DArgsHi &, int, cudaStream_t);
template cudaError_t glbm_step2d_zv_level<11, double>(int, int, const Step2DArgsHi &, int, cudaStream_t);
template cudaError_t glbm_step2d_zv_level<12, double>(int, int, const Step2DArgsHi &, int, cudaStream_t);
template cudaError_t glbm_step2d_zv_level<13, double>(int, int, const Step2DArgsHi &, int, cudaStream_t);
