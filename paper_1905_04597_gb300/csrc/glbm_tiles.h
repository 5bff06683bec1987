// Candidate tile shapes of the fused 2D step, per level N and precision. A
// CTA covers 32 V columns x R node rows: each thread owns V x-adjacent nodes
// (V = 1: the one-node tile of glbm_step2d.cuh; V = 2: the packed pair tile of
// glbm_step2d_pair.cuh, FP32 only), and each node's 2N+1 velocity rows are
// dealt to G warps, so a thread keeps V ceil((2N+1)/G) (2N+1) populations in
// registers and a CTA has 32 G R threads. Entry 0 is the shape used until a
// context is autotuned. R and V only regroup nodes into CTAs and threads; G
// also sets how the partial moments are grouped before their compensated sum,
// so shapes with different G can differ in the last bits of a result.
#pragma once
#include "glbm_internal.h"

template <int N, typename T>
struct Tiles;

#define GLBM_TILES(N_, T_, ...)                                        \
    template <>                                                        \
    struct Tiles<N_, T_> {                                             \
        static constexpr TileShape shape[] = {__VA_ARGS__};            \
        static constexpr int count = sizeof(shape) / sizeof(shape[0]); \
        static_assert(count <= GLBM_MAX_TILES, "too many shapes");     \
    };

// FP32 deviations: {G, R, V}. Entry 0 of each level is the fastest measured on
// GB300 for 512 x 256 lattices with walls (the autotuner re-times them for a
// given context).
GLBM_TILES(1, float, {1, 16, 2}, {1, 8, 2}, {1, 16, 1}, {1, 8, 1}, {1, 4, 1})
GLBM_TILES(2, float, {1, 4, 2}, {1, 8, 2}, {1, 8, 1}, {1, 4, 1}, {1, 16, 1})
GLBM_TILES(3, float, {2, 2, 2}, {1, 4, 1}, {1, 2, 1}, {1, 8, 1}, {2, 4, 1}, {1, 2, 2}, {2, 4, 2})
GLBM_TILES(4, float, {3, 1, 2}, {2, 2, 2}, {3, 2, 2}, {1, 4, 1}, {1, 2, 1}, {2, 2, 1}, {2, 4, 1},
           {3, 2, 1})
GLBM_TILES(5, float, {4, 1, 2}, {3, 1, 2}, {4, 2, 2}, {3, 2, 1}, {2, 2, 1}, {2, 1, 1}, {2, 4, 1},
           {4, 2, 1})
GLBM_TILES(6, float, {4, 2, 1}, {2, 2, 1}, {4, 1, 2}, {5, 1, 2}, {7, 1, 2}, {2, 1, 1}, {3, 1, 1},
           {3, 2, 1})
GLBM_TILES(7, float, {5, 1, 2}, {5, 1, 1}, {4, 1, 1}, {3, 1, 1}, {3, 2, 1}, {2, 2, 1}, {4, 2, 1},
           {4, 1, 2})
GLBM_TILES(8, float, {6, 1, 1}, {4, 1, 1}, {4, 2, 1}, {3, 1, 1}, {3, 2, 1}, {5, 1, 1}, {6, 1, 2},
           {9, 1, 2})
// FP64 (one-node tiles)
GLBM_TILES(1, double, {1, 8, 1}, {1, 4, 1})
GLBM_TILES(2, double, {1, 4, 1}, {1, 8, 1}, {2, 4, 1})
GLBM_TILES(3, double, {1, 4, 1}, {2, 2, 1}, {2, 4, 1})
GLBM_TILES(4, double, {2, 2, 1}, {3, 2, 1}, {2, 4, 1})
GLBM_TILES(5, double, {3, 1, 1}, {3, 2, 1}, {4, 1, 1})
GLBM_TILES(6, double, {4, 1, 1}, {4, 2, 1}, {5, 1, 1})
GLBM_TILES(7, double, {4, 1, 1}, {5, 1, 1}, {6, 1, 1})
GLBM_TILES(8, double, {6, 1, 1}, {5, 1, 1}, {9, 1, 1})

#undef GLBM_TILES

// Anisotropic products D1Q3 (x) times level N (y), the channel lattices of Sec. 5.
template <int N, typename T>
struct TilesX1;

#define GLBM_TILES_X1(N_, T_, ...)                                     \
    template <>                                                        \
    struct TilesX1<N_, T_> {                                           \
        static constexpr TileShape shape[] = {__VA_ARGS__};            \
        static constexpr int count = sizeof(shape) / sizeof(shape[0]); \
    };
// {G, R, V}: 3 (2N+1) populations per node, a few rows per CTA; V = 2 pairs.
// Entry 0 of each level is the fastest measured on GB300 (1024 x 200, walls).
GLBM_TILES_X1(1, float, {1, 8, 2}, {1, 4, 2}, {1, 8, 1}, {1, 4, 1}, {1, 16, 1})
GLBM_TILES_X1(2, float, {1, 8, 2}, {1, 4, 2}, {1, 8, 1}, {1, 4, 1}, {1, 16, 1})
GLBM_TILES_X1(3, float, {1, 4, 2}, {1, 2, 2}, {1, 8, 1}, {1, 4, 1}, {1, 16, 1})
GLBM_TILES_X1(4, float, {1, 4, 2}, {1, 2, 2}, {2, 2, 2}, {1, 8, 1}, {1, 4, 1}, {1, 2, 1})
GLBM_TILES_X1(5, float, {2, 2, 2}, {1, 2, 2}, {2, 1, 2}, {1, 4, 1}, {1, 8, 1}, {1, 2, 1})
GLBM_TILES_X1(6, float, {2, 2, 2}, {1, 2, 2}, {2, 1, 2}, {1, 4, 1}, {1, 8, 1}, {1, 2, 1})
GLBM_TILES_X1(7, float, {2, 2, 2}, {2, 1, 2}, {3, 1, 2}, {1, 4, 1}, {1, 2, 1}, {2, 4, 1})
GLBM_TILES_X1(8, float, {2, 2, 2}, {2, 1, 2}, {3, 1, 2}, {1, 4, 1}, {1, 2, 1}, {2, 4, 1})
GLBM_TILES_X1(1, double, {1, 8, 1}, {1, 4, 1})
GLBM_TILES_X1(2, double, {1, 8, 1}, {1, 4, 1})
GLBM_TILES_X1(3, double, {1, 4, 1}, {1, 8, 1})
GLBM_TILES_X1(4, double, {1, 4, 1}, {1, 2, 1})
GLBM_TILES_X1(5, double, {1, 4, 1}, {1, 2, 1})
GLBM_TILES_X1(6, double, {1, 4, 1}, {2, 2, 1})
GLBM_TILES_X1(7, double, {1, 4, 1}, {2, 2, 1})
GLBM_TILES_X1(8, double, {1, 2, 1}, {2, 2, 1})
#undef GLBM_TILES_X1
