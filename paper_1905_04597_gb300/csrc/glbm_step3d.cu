// Tile shapes and launches of the 3D step (glbm_step3d.cuh), levels 1..3
// (D3Q27, D3Q125, D3Q343), FP32 deviations and FP64.
#include "glbm_step2d_launch.cuh"
#include "glbm_step3d.cuh"

template <int N, typename T>
struct Tiles3D;

#define GLBM_TILES_3D(N_, T_, ...)                                     \
    template <>                                                        \
    struct Tiles3D<N_, T_> {                                           \
        static constexpr TileShape shape[] = {__VA_ARGS__};            \
        static constexpr int count = sizeof(shape) / sizeof(shape[0]); \
        static_assert(count <= GLBM_MAX_TILES, "too many shapes");     \
    };
// {G, R, V}: the (2N+1)^2 velocity rows of a node divide evenly among G warps
// where the list allows it; one-node tiles. Entry 0 is the fastest measured on
// GB300 (256 x 64 x 32, walls, about 400 MB per step).
GLBM_TILES_3D(1, float, {1, 8, 1}, {1, 4, 1}, {3, 2, 1}, {3, 4, 1})
GLBM_TILES_3D(2, float, {5, 1, 1}, {5, 2, 1}, {5, 4, 1}, {3, 2, 1})
GLBM_TILES_3D(3, float, {7, 1, 1}, {5, 1, 1}, {7, 2, 1})
GLBM_TILES_3D(1, double, {1, 4, 1}, {3, 2, 1})
GLBM_TILES_3D(2, double, {5, 1, 1}, {5, 2, 1})
GLBM_TILES_3D(3, double, {7, 1, 1}, {10, 1, 1})
#undef GLBM_TILES_3D

template <int N, typename T, int I = 0>
static cudaError_t launch_3d_shape(int shape, const Step3DArgs &a, int n_inst, cudaStream_t s)
{
    if constexpr (I < Tiles3D<N, T>::count) {
        if (shape == I) {
            constexpr TileShape t = Tiles3D<N, T>::shape[I];
            const dim3 grid((a.Lx + 31) / 32, (a.Ly + t.R - 1) / t.R, a.Lz * n_inst);
            return launch_serialized(k_step3d<N, T, t.G, t.R>, grid, dim3(32 * t.G * t.R), s, a);
        }
        return launch_3d_shape<N, T, I + 1>(shape, a, n_inst, s);
    } else {
        return cudaErrorInvalidValue;
    }
}

template <typename T>
static cudaError_t launch_3d(int N, int shape, const Step3DArgs &a, int n_inst, cudaStream_t s)
{
    switch (N) {
    case 1: return launch_3d_shape<1, T>(shape, a, n_inst, s);
    case 2: return launch_3d_shape<2, T>(shape, a, n_inst, s);
    case 3: return launch_3d_shape<3, T>(shape, a, n_inst, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t glbm_launch_step3d(int N, int prec, int shape, const Step3DArgs &a, int n_inst,
                               cudaStream_t s)
{
    return prec == GLBM_FP64 ? launch_3d<double>(N, shape, a, n_inst, s)
                             : launch_3d<float>(N, shape, a, n_inst, s);
}

template <int N, typename T>
static int copy_3d(TileShape *out)
{
    for (int i = 0; i < Tiles3D<N, T>::count; ++i) out[i] = Tiles3D<N, T>::shape[i];
    return Tiles3D<N, T>::count;
}

int glbm_tile_shapes_3d(int N, int prec, TileShape *out)
{
    const bool f64 = prec == GLBM_FP64;
    switch (N) {
    case 1: return f64 ? copy_3d<1, double>(out) : copy_3d<1, float>(out);
    case 2: return f64 ? copy_3d<2, double>(out) : copy_3d<2, float>(out);
    case 3: return f64 ? copy_3d<3, double>(out) : copy_3d<3, float>(out);
    default: return 0;
    }
}
