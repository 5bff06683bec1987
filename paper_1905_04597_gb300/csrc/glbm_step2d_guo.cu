// Per-level dispatch of the fused 2D step with Guo's force (the kernels are
// instantiated in glbm_step2d_guo_a.cu .. _f.cu).
#include "glbm_tiles_guo.h"

template <typename T, int KIND>
static cudaError_t launch_guo(int N, const Step2DArgs &a, int n_inst, cudaStream_t s)
{
    switch (N) {
    case 1: return glbm_step2d_guo_level<1, T, KIND>(a, n_inst, s);
    case 2: return glbm_step2d_guo_level<2, T, KIND>(a, n_inst, s);
    case 3: return glbm_step2d_guo_level<3, T, KIND>(a, n_inst, s);
    case 4: return glbm_step2d_guo_level<4, T, KIND>(a, n_inst, s);
    case 5: return glbm_step2d_guo_level<5, T, KIND>(a, n_inst, s);
    case 6: return glbm_step2d_guo_level<6, T, KIND>(a, n_inst, s);
    case 7: return glbm_step2d_guo_level<7, T, KIND>(a, n_inst, s);
    case 8: return glbm_step2d_guo_level<8, T, KIND>(a, n_inst, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
static cudaError_t launch_guo_kind(int N, int kind, const Step2DArgs &a, int n_inst, cudaStream_t s)
{
    switch (kind) {
    case GLBM_GUOK_ISO: return launch_guo<T, GLBM_GUOK_ISO>(N, a, n_inst, s);
    case GLBM_GUOK_X1: return launch_guo<T, GLBM_GUOK_X1>(N, a, n_inst, s);
    case GLBM_GUOK_ZV: return launch_guo<T, GLBM_GUOK_ZV>(N, a, n_inst, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t glbm_launch_step2d_guo(int N, int kind, int prec, const Step2DArgs &a, int n_inst,
                                   cudaStream_t s)
{
    return prec == GLBM_FP64 ? launch_guo_kind<double>(N, kind, a, n_inst, s)
                             : launch_guo_kind<float>(N, kind, a, n_inst, s);
}

template <typename T, int KIND>
static int shape_guo(int N, TileShape *out)
{
    switch (N) {
    case 1: *out = guo_shape<1, T, KIND>(); return 1;
    case 2: *out = guo_shape<2, T, KIND>(); return 1;
    case 3: *out = guo_shape<3, T, KIND>(); return 1;
    case 4: *out = guo_shape<4, T, KIND>(); return 1;
    case 5: *out = guo_shape<5, T, KIND>(); return 1;
    case 6: *out = guo_shape<6, T, KIND>(); return 1;
    case 7: *out = guo_shape<7, T, KIND>(); return 1;
    case 8: *out = guo_shape<8, T, KIND>(); return 1;
    default: return 0;
    }
}

template <typename T>
static int shape_guo_kind(int N, int kind, TileShape *out)
{
    switch (kind) {
    case GLBM_GUOK_ISO: return shape_guo<T, GLBM_GUOK_ISO>(N, out);
    case GLBM_GUOK_X1: return shape_guo<T, GLBM_GUOK_X1>(N, out);
    case GLBM_GUOK_ZV: return shape_guo<T, GLBM_GUOK_ZV>(N, out);
    default: return 0;
    }
}

int glbm_tile_shape_guo(int N, int kind, int prec, TileShape *out)
{
    return prec == GLBM_FP64 ? shape_guo_kind<double>(N, kind, out)
                             : shape_guo_kind<float>(N, kind, out);
}
