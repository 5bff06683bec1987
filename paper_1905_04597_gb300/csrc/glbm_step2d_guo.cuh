// The fused 2D step with the force of Guo, Zheng and Shi (2002) in place of the
// paper's linearised force (Step2D with GUO set). One tile shape per level and
// lattice kind: the first one-node entry of the kind's candidate list, whose
// linearised counterpart is measured there; the autotuner has nothing to
// choose. Kinds: GLBM_GUOK_ISO (the level-N lattice on both axes),
// GLBM_GUOK_X1 (D1Q3 along x times level N along y) and GLBM_GUOK_ZV (D1Q3
// along x times the level-N 2N+2 axis along y).
#pragma once
#include "glbm_step2d_launch.cuh"
#include "glbm_tiles_guo.h"

template <int N, typename T, int KIND>
cudaError_t glbm_step2d_guo_level(const Step2DArgs &a, int n_inst, cudaStream_t s)
{
    constexpr TileShape t = guo_shape<N, T, KIND>();
    constexpr int NXL = KIND == GLBM_GUOK_ISO ? N : 1;
    constexpr int ZY = KIND == GLBM_GUOK_ZV ? 1 : 0;
    const dim3 grid((a.Lx + 31) / 32, (a.Ly + t.R - 1) / t.R, n_inst);
    const cudaError_t e = launch_wall_rho<N, T, NXL, ZY, 0>(a, n_inst, s);
    if (e != cudaSuccess) return e;
    return launch_serialized(k_step2d<N, T, t.G, t.R, NXL, ZY, 0, true>, grid, dim3(32 * t.G * t.R),
                             s, a);
}
