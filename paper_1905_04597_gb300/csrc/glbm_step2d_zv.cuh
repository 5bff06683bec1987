// Fused 2D step on the 2N+2 hierarchy (Sec. 4: the zero velocity removed,
// Eqs. maineq01_noball - maineq04_noball): the one-node tile of
// glbm_step2d.cuh (and in FP32 the pair tile of glbm_step2d_pair.cuh) with
// the 2N+2 axis along y (kind GLBM_ZVK_X1: D1Q3 along x,
// the form of the paper's channel models G-D1Q6 x D1Q3 and G-D1Q8 x D1Q3) or
// along both axes (kind GLBM_ZVK_XY, the fully symmetric lattices).
#pragma once
#include "glbm_step2d_launch.cuh"
#include "glbm_tiles_zv.h"

template <int N, typename T, int KIND, int I = 0>
cudaError_t launch_zv_shape(int shape, const Step2DArgsOf<N> &a, int n_inst, cudaStream_t s)
{
    if constexpr (I < TilesZv<N, T, KIND>::count) {
        if (shape == I) {
            constexpr TileShape t = TilesZv<N, T, KIND>::shape[I];
            constexpr int NXL = KIND == GLBM_ZVK_X1 ? 1 : N;
            constexpr int ZX = KIND == GLBM_ZVK_X1 ? 0 : 1;
            const dim3 grid((a.Lx + 32 * t.V - 1) / (32 * t.V), (a.Ly + t.R - 1) / t.R, n_inst);
            const cudaError_t e = launch_wall_rho<N, T, NXL, 1, ZX>(a, n_inst, s);
            if (e != cudaSuccess) return e;
            if constexpr (t.V == 2) {
                static_assert(sizeof(T) == 4, "pair tiles store FP32 deviations");
                return launch_serialized(k_step2d_pair<N, t.G, t.R, NXL, 1, ZX>, grid,
                                         dim3(32 * t.G * t.R), s, a);
            } else {
                return launch_serialized(k_step2d<N, T, t.G, t.R, NXL, 1, ZX>, grid,
                                         dim3(32 * t.G * t.R), s, a);
            }
        }
        return launch_zv_shape<N, T, KIND, I + 1>(shape, a, n_inst, s);
    } else {
        return cudaErrorInvalidValue;
    }
}

template <int N, typename T>
cudaError_t glbm_step2d_zv_level(int kind, int shape, const Step2DArgsOf<N> &a, int n_inst,
                                 cudaStream_t s)
{
    return kind == GLBM_ZVK_X1 ? launch_zv_shape<N, T, GLBM_ZVK_X1>(shape, a, n_inst, s)
                               : launch_zv_shape<N, T, GLBM_ZVK_XY>(shape, a, n_inst, s);
}
