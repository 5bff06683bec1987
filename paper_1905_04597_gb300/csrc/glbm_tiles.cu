// Tile-shape candidates and the per-level dispatch of the uniform 2D step.
#include "glbm_tiles.h"

template <int N, typename T>
static int copy_shapes(TileShape *out)
{
    for (int i = 0; i < Tiles<N, T>::count; ++i) out[i] = Tiles<N, T>::shape[i];
    return Tiles<N, T>::count;
}

template <typename T>
static int shapes_of(int N, TileShape *out)
{
    switch (N) {
    case 1: return copy_shapes<1, T>(out);
    case 2: return copy_shapes<2, T>(out);
    case 3: return copy_shapes<3, T>(out);
    case 4: return copy_shapes<4, T>(out);
    case 5: return copy_shapes<5, T>(out);
    case 6: return copy_shapes<6, T>(out);
    case 7: return copy_shapes<7, T>(out);
    case 8: return copy_shapes<8, T>(out);
    default: return 0;
    }
}

int glbm_tile_shapes(int N, int prec, TileShape *out)
{
    return prec == GLBM_FP64 ? shapes_of<double>(N, out) : shapes_of<float>(N, out);
}

template <typename T>
static cudaError_t launch_level(int N, int shape, const Step2DArgs &a, int n_inst, cudaStream_t s)
{
    switch (N) {
    case 1: return glbm_step2d_level<1, T>(shape, a, n_inst, s);
    case 2: return glbm_step2d_level<2, T>(shape, a, n_inst, s);
    case 3: return glbm_step2d_level<3, T>(shape, a, n_inst, s);
    case 4: return glbm_step2d_level<4, T>(shape, a, n_inst, s);
    case 5: return glbm_step2d_level<5, T>(shape, a, n_inst, s);
    case 6: return glbm_step2d_level<6, T>(shape, a, n_inst, s);
    case 7: return glbm_step2d_level<7, T>(shape, a, n_inst, s);
    case 8: return glbm_step2d_level<8, T>(shape, a, n_inst, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t glbm_launch_step2d_f32(int N, int shape, const Step2DArgs &a, int n_inst,
                                   cudaStream_t s)
{
    return launch_level<float>(N, shape, a, n_inst, s);
}

cudaError_t glbm_launch_step2d_f64(int N, int shape, const Step2DArgs &a, int n_inst,
                                   cudaStream_t s)
{
    return launch_level<double>(N, shape, a, n_inst, s);
}
