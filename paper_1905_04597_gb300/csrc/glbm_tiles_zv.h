// Candidate tile shapes of the fused 2D step on the 2N+2 hierarchy (Sec. 4:
// the zero velocity removed), per level N, precision and kind: GLBM_ZVK_X1
// (D1Q3 along x times the level-N 2N+2 axis along y) or GLBM_ZVK_XY (the 2N+2
// axis on both). In FP32 both kinds also have packed pair tiles (V = 2).
#pragma once
#include "glbm_internal.h"

// Combinations without candidates (D2Q(2N+2)^2 above level 8) have none.
template <int N, typename T, int KIND>
struct TilesZv {
    static constexpr TileShape shape[1] = {{1, 1, 1}};
    static constexpr int count = 0;
};

#define GLBM_TILES_ZV(N_, T_, K_, ...)                                 \
    template <>                                                        \
    struct TilesZv<N_, T_, K_> {                                       \
        static constexpr TileShape shape[] = {__VA_ARGS__};            \
        static constexpr int count = sizeof(shape) / sizeof(shape[0]); \
        static_assert(count <= GLBM_MAX_TILES, "too many shapes");     \
    };
// {G, R, V}: the 2N+2 velocity rows divide evenly among G warps where the
// list allows it. Entry 0 is the fastest measured on
// GB300 (1024 x 200 channels for X1, 512 x 256 for XY, walls).
GLBM_TILES_ZV(1, float, GLBM_ZVK_X1, {1, 8, 2}, {1, 4, 2}, {1, 16, 1}, {1, 8, 1}, {1, 4, 1})
GLBM_TILES_ZV(2, float, GLBM_ZVK_X1, {1, 4, 2}, {1, 8, 2}, {1, 8, 1}, {1, 4, 1}, {1, 16, 1})
GLBM_TILES_ZV(3, float, GLBM_ZVK_X1, {1, 4, 2}, {2, 4, 2}, {1, 8, 1}, {1, 4, 1}, {2, 4, 1})
GLBM_TILES_ZV(4, float, GLBM_ZVK_X1, {2, 2, 2}, {1, 4, 2}, {1, 8, 1}, {1, 4, 1}, {2, 2, 1})
GLBM_TILES_ZV(5, float, GLBM_ZVK_X1, {2, 2, 2}, {1, 2, 2}, {1, 4, 1}, {2, 2, 1}, {1, 2, 1})
GLBM_TILES_ZV(6, float, GLBM_ZVK_X1, {2, 2, 2}, {1, 2, 2}, {1, 4, 1}, {2, 2, 1}, {1, 2, 1})
GLBM_TILES_ZV(7, float, GLBM_ZVK_X1, {2, 2, 2}, {4, 1, 2}, {1, 4, 1}, {2, 2, 1}, {2, 4, 1})
GLBM_TILES_ZV(8, float, GLBM_ZVK_X1, {2, 2, 2}, {3, 1, 2}, {2, 2, 1}, {1, 4, 1}, {3, 2, 1})
// levels 9..13 (the paper's G-D1Q22 x D1Q3 .. G-D1Q28 x D1Q3, Sec. 5.4)
GLBM_TILES_ZV(9, float, GLBM_ZVK_X1, {4, 1, 2}, {2, 2, 2}, {2, 2, 1}, {1, 4, 1})
GLBM_TILES_ZV(10, float, GLBM_ZVK_X1, {2, 2, 2}, {2, 1, 2}, {2, 2, 1}, {1, 4, 1})
GLBM_TILES_ZV(11, float, GLBM_ZVK_X1, {2, 2, 2}, {3, 1, 2}, {2, 2, 1}, {4, 1, 1})
GLBM_TILES_ZV(12, float, GLBM_ZVK_X1, {2, 2, 2}, {2, 1, 2}, {2, 2, 1}, {1, 4, 1})
GLBM_TILES_ZV(13, float, GLBM_ZVK_X1, {2, 2, 2}, {4, 1, 2}, {2, 2, 1}, {4, 1, 1})
GLBM_TILES_ZV(1, double, GLBM_ZVK_X1, {1, 4, 1}, {1, 8, 1})
GLBM_TILES_ZV(2, double, GLBM_ZVK_X1, {1, 4, 1}, {1, 8, 1})
GLBM_TILES_ZV(3, double, GLBM_ZVK_X1, {1, 4, 1}, {2, 2, 1})
GLBM_TILES_ZV(4, double, GLBM_ZVK_X1, {1, 4, 1}, {2, 2, 1})
GLBM_TILES_ZV(5, double, GLBM_ZVK_X1, {1, 4, 1}, {2, 2, 1})
GLBM_TILES_ZV(6, double, GLBM_ZVK_X1, {2, 2, 1}, {1, 4, 1})
GLBM_TILES_ZV(7, double, GLBM_ZVK_X1, {2, 2, 1}, {1, 2, 1})
GLBM_TILES_ZV(8, double, GLBM_ZVK_X1, {2, 2, 1}, {3, 2, 1})
GLBM_TILES_ZV(9, double, GLBM_ZVK_X1, {1, 4, 1}, {2, 2, 1})
GLBM_TILES_ZV(10, double, GLBM_ZVK_X1, {1, 4, 1}, {2, 2, 1})
GLBM_TILES_ZV(11, double, GLBM_ZVK_X1, {2, 2, 1}, {4, 1, 1})
GLBM_TILES_ZV(12, double, GLBM_ZVK_X1, {1, 4, 1}, {2, 2, 1})
GLBM_TILES_ZV(13, double, GLBM_ZVK_X1, {2, 2, 1}, {4, 1, 1})
GLBM_TILES_ZV(1, float, GLBM_ZVK_XY, {1, 8, 2}, {1, 4, 2}, {1, 16, 1}, {1, 8, 1}, {1, 4, 1})
GLBM_TILES_ZV(2, float, GLBM_ZVK_XY, {1, 4, 2}, {2, 4, 2}, {1, 4, 1}, {2, 4, 1}, {1, 8, 1})
GLBM_TILES_ZV(3, float, GLBM_ZVK_XY, {2, 2, 2}, {2, 4, 2}, {2, 4, 1}, {2, 2, 1}, {1, 4, 1})
GLBM_TILES_ZV(4, float, GLBM_ZVK_XY, {2, 4, 1}, {2, 2, 1}, {5, 1, 1}, {2, 2, 2}, {5, 1, 2})
GLBM_TILES_ZV(5, float, GLBM_ZVK_XY, {4, 1, 2}, {3, 1, 2}, {4, 1, 1}, {3, 1, 1}, {3, 2, 1})
GLBM_TILES_ZV(6, float, GLBM_ZVK_XY, {2, 2, 1}, {7, 1, 1}, {4, 1, 1}, {7, 1, 2}, {2, 2, 2})
GLBM_TILES_ZV(7, float, GLBM_ZVK_XY, {4, 1, 2}, {8, 1, 2}, {8, 1, 1}, {4, 1, 1}, {4, 2, 1})
GLBM_TILES_ZV(8, float, GLBM_ZVK_XY, {6, 1, 1}, {9, 1, 1}, {3, 2, 1}, {9, 1, 2}, {6, 1, 2})
GLBM_TILES_ZV(1, double, GLBM_ZVK_XY, {1, 4, 1}, {1, 8, 1})
GLBM_TILES_ZV(2, double, GLBM_ZVK_XY, {1, 4, 1}, {2, 2, 1})
GLBM_TILES_ZV(3, double, GLBM_ZVK_XY, {2, 2, 1}, {1, 4, 1})
GLBM_TILES_ZV(4, double, GLBM_ZVK_XY, {2, 2, 1}, {5, 1, 1})
GLBM_TILES_ZV(5, double, GLBM_ZVK_XY, {3, 1, 1}, {4, 1, 1})
GLBM_TILES_ZV(6, double, GLBM_ZVK_XY, {4, 1, 1}, {7, 1, 1})
GLBM_TILES_ZV(7, double, GLBM_ZVK_XY, {8, 1, 1}, {4, 1, 1})
GLBM_TILES_ZV(8, double, GLBM_ZVK_XY, {6, 1, 1}, {9, 1, 1})
#undef GLBM_TILES_ZV

template <int N, typename T, int KIND>
int glbm_zv_copy_shapes(TileShape *out)
{
    for (int i = 0; i < TilesZv<N, T, KIND>::count; ++i) out[i] = TilesZv<N, T, KIND>::shape[i];
    return TilesZv<N, T, KIND>::count;
}
