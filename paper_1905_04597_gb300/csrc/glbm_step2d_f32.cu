// FP32-deviation instantiations of the fused 2D stream-collide kernel.
#include "glbm_step2d.cuh"

cudaError_t glbm_launch_step2d_f32(int N, const Step2DArgs &a, int n_inst, cudaStream_t s)
{
    return launch_step2d<float>(N, a, n_inst, s);
}
