// Tile-shape candidates and the per-level dispatch of the 2N+2 lattices (the
// kernels are instantiated in glbm_step2d_zv_a.cu .. _f.cu).
#include "glbm_tiles_zv.h"

template <typename T, int KIND>
static int shapes_zv(int N, TileShape *out)
{
    switch (N) {
    case 1: return glbm_zv_copy_shapes<1, T, KIND>(out);
    case 2: return glbm_zv_copy_shapes<2, T, KIND>(out);
    case 3: return glbm_zv_copy_shapes<3, T, KIND>(out);
    case 4: return glbm_zv_copy_shapes<4, T, KIND>(out);
    case 5: return glbm_zv_copy_shapes<5, T, KIND>(out);
    case 6: return glbm_zv_copy_shapes<6, T, KIND>(out);
    case 7: return glbm_zv_copy_shapes<7, T, KIND>(out);
    case 8: return glbm_zv_copy_shapes<8, T, KIND>(out);
    case 9: return glbm_zv_copy_shapes<9, T, KIND>(out);
    case 10: return glbm_zv_copy_shapes<10, T, KIND>(out);
    case 11: return glbm_zv_copy_shapes<11, T, KIND>(out);
    case 12: return glbm_zv_copy_shapes<12, T, KIND>(out);
    case 13: return glbm_zv_copy_shapes<13, T, KIND>(out);
    default: return 0;
    }
}

int glbm_tile_shapes_zv(int N, int kind, int prec, TileShape *out)
{
    if (kind == GLBM_ZVK_X1)
        return prec == GLBM_FP64 ? shapes_zv<double, GLBM_ZVK_X1>(N, out)
                                 : shapes_zv<float, GLBM_ZVK_X1>(N, out);
    return prec == GLBM_FP64 ? shapes_zv<double, GLBM_ZVK_XY>(N, out)
                             : shapes_zv<float, GLBM_ZVK_XY>(N, out);
}

template <typename T>
static cudaError_t launch_zv(int N, int kind, int shape, const Step2DArgs &a, int n_inst,
                             cudaStream_t s)
{
    switch (N) {
    case 1: return glbm_step2d_zv_level<1, T>(kind, shape, a, n_inst, s);
    case 2: return glbm_step2d_zv_level<2, T>(kind, shape, a, n_inst, s);
    case 3: return glbm_step2d_zv_level<3, T>(kind, shape, a, n_inst, s);
    case 4: return glbm_step2d_zv_level<4, T>(kind, shape, a, n_inst, s);
    case 5: return glbm_step2d_zv_level<5, T>(kind, shape, a, n_inst, s);
    case 6: return glbm_step2d_zv_level<6, T>(kind, shape, a, n_inst, s);
    case 7: return glbm_step2d_zv_level<7, T>(kind, shape, a, n_inst, s);
    case 8: return glbm_step2d_zv_level<8, T>(kind, shape, a, n_inst, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t glbm_launch_step2d_zv(int N, int kind, int prec, int shape, const Step2DArgs &a,
                                  int n_inst, cudaStream_t s)
{
    return prec == GLBM_FP64 ? launch_zv<double>(N, kind, shape, a, n_inst, s)
                             : launch_zv<float>(N, kind, shape, a, n_inst, s);
}

template <typename T>
static cudaError_t launch_zv_hi(int N, int shape, const Step2DArgsHi &a, int n_inst, cudaStream_t s)
{
    switch (N) {
    case 9: return glbm_step2d_zv_level<9, T>(GLBM_ZVK_X1, shape, a, n_inst, s);
    case 10: return glbm_step2d_zv_level<10, T>(GLBM_ZVK_X1, shape, a, n_inst, s);
    case 11: return glbm_step2d_zv_level<11, T>(GLBM_ZVK_X1, shape, a, n_inst, s);
    case 12: return glbm_step2d_zv_level<12, T>(GLBM_ZVK_X1, shape, a, n_inst, s);
    case 13: return glbm_step2d_zv_level<13, T>(GLBM_ZVK_X1, shape, a, n_inst, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t glbm_launch_step2d_zv_hi(int N, int prec, int shape, const Step2DArgsHi &a,
                                     int n_inst, cudaStream_t s)
{
    return prec == GLBM_FP64 ? launch_zv_hi<double>(N, shape, a, n_inst, s)
                             : launch_zv_hi<float>(N, shape, a, n_inst, s);
}
