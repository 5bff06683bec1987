// Anisotropic tensor products (Sec. 4 builds a 2D lattice as the product of any
// two 1D levels): D1Q3 along x (level 1) times the level-N Gaussian lattice
// along y, the form the paper uses for its channel flows. One-node tiles,
// both precisions, and packed pair tiles in FP32; the candidate shapes of each
// level are TilesX1 of glbm_tiles.h.
#include "glbm_step2d_launch.cuh"

template <int N, typename T, int I = 0>
static cudaError_t launch_x1_shape(int shape, const Step2DArgs &a, int n_inst, cudaStream_t s)
{
    if constexpr (I < TilesX1<N, T>::count) {
        if (shape == I) {
            constexpr TileShape t = TilesX1<N, T>::shape[I];
            const dim3 grid((a.Lx + 32 * t.V - 1) / (32 * t.V), (a.Ly + t.R - 1) / t.R, n_inst);
            const cudaError_t e = launch_wall_rho<N, T, 1, 0, 0>(a, n_inst, s);
            if (e != cudaSuccess) return e;
            if constexpr (t.V == 2) {
                static_assert(sizeof(T) == 4, "pair tiles store FP32 deviations");
                return launch_serialized(k_step2d_pair<N, t.G, t.R, 1>, grid, dim3(32 * t.G * t.R), s, a);
            } else {
                return launch_serialized(k_step2d<N, T, t.G, t.R, 1>, grid, dim3(32 * t.G * t.R), s, a);
            }
        }
        return launch_x1_shape<N, T, I + 1>(shape, a, n_inst, s);
    } else {
        return cudaErrorInvalidValue;
    }
}

template <typename T>
static cudaError_t launch_x1(int N, int shape, const Step2DArgs &a, int n_inst, cudaStream_t s)
{
    switch (N) {
    case 1: return launch_x1_shape<1, T>(shape, a, n_inst, s);
    case 2: return launch_x1_shape<2, T>(shape, a, n_inst, s);
    case 3: return launch_x1_shape<3, T>(shape, a, n_inst, s);
    case 4: return launch_x1_shape<4, T>(shape, a, n_inst, s);
    case 5: return launch_x1_shape<5, T>(shape, a, n_inst, s);
    case 6: return launch_x1_shape<6, T>(shape, a, n_inst, s);
    case 7: return launch_x1_shape<7, T>(shape, a, n_inst, s);
    case 8: return launch_x1_shape<8, T>(shape, a, n_inst, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t glbm_launch_step2d_x1(int N, int prec, int shape, const Step2DArgs &a, int n_inst,
                                  cudaStream_t s)
{
    return prec == GLBM_FP64 ? launch_x1<double>(N, shape, a, n_inst, s)
                             : launch_x1<float>(N, shape, a, n_inst, s);
}

template <int N, typename T>
static int copy_x1(TileShape *out)
{
    for (int i = 0; i < TilesX1<N, T>::count; ++i) out[i] = TilesX1<N, T>::shape[i];
    return TilesX1<N, T>::count;
}

template <typename T>
static int shapes_x1(int N, TileShape *out)
{
    switch (N) {
    case 1: return copy_x1<1, T>(out);
    case 2: return copy_x1<2, T>(out);
    case 3: return copy_x1<3, T>(out);
    case 4: return copy_x1<4, T>(out);
    case 5: return copy_x1<5, T>(out);
    case 6: return copy_x1<6, T>(out);
    case 7: return copy_x1<7, T>(out);
    case 8: return copy_x1<8, T>(out);
    default: return 0;
    }
}

int glbm_tile_shapes_x1(int N, int prec, TileShape *out)
{
    return prec == GLBM_FP64 ? shapes_x1<double>(N, out) : shapes_x1<float>(N, out);
}
