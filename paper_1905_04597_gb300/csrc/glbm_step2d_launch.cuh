// Launch of the uniform fused 2D step by tile shape (glbm_tiles.h): one-node
// tiles for both precisions, packed pair tiles for FP32 deviations.
#pragma once
#include "glbm_step2d_pair.cuh"
#include "glbm_tiles.h"

template <int N, int G, int R, int NXL = N, int ZY = 0, int ZX = 0>
__global__ void __launch_bounds__(32 * G * R)
    k_step2d_pair(const __grid_constant__ Step2DArgsOf<N> a)
{
    using S = Step2DPair<N, G, R, NXL, ZY, ZX>;
    __shared__ __align__(16) typename S::Smem sm;
    const int inst = blockIdx.z;
    const bool df = a.bands != nullptr;  // dataflow chunk (glbm_internal.h)
    if (df) {
        df_launch_next();
        if (a.node > 0) {
            constexpr int V = AxisVel<N, ZY>::VMAX;
            const int y0 = blockIdx.y * R;
            df_wait_rows(a.bands, a.status, inst, y0 - V, y0 + R - 1 + V, a.Ly, R,
                         a.bc != GLBM_BC_WALLS, (unsigned)a.node * gridDim.x);
        }
    } else {
        wait_prior_grid();
    }
    const bool live = !step_halted(a.status);  // needed only at the stores
    const float *fin = static_cast<const float *>(a.fin) + (long long)inst * a.inst_stride;
    float *fout = static_cast<float *>(a.fout) + (long long)inst * a.inst_stride;
    // the step clock: the launch counter (read before any CTA of this launch
    // can advance it), or the chunk's base plus this step's index
    const unsigned clk = df ? __ldcg(a.status + ST_BASE) + (unsigned)a.node : __ldcg(a.step_ctr);
    const unsigned seed = hash32(clk * 0x632BE5ABu + inst);
    const float *rwg =
        a.rw ? static_cast<const float *>(a.rw) + (long long)inst * 2 * a.pitch : nullptr;
    if constexpr (NXL == N && ZX == ZY)
        S::run(a.tab, a.tab, a.ip[inst], a.Lx, a.Ly, a.pitch, (int)a.plane, a.bc, fin, fout,
               blockIdx.x * S::TW, blockIdx.y * R, sm, a.status, seed, rwg, live);
    else
        S::run(a.tab, a.tabx, a.ip[inst], a.Lx, a.Ly, a.pitch, (int)a.plane, a.bc, fin, fout,
               blockIdx.x * S::TW, blockIdx.y * R, sm, a.status, seed, rwg, live);
    if (df) {
        df_tile_done(a.bands, inst);
        if (live) finish_step_df(a.status, a.node_done + a.node);
    } else if (live) {
        finish_step(a.status);
    }
}

// Launch with programmatic stream serialization (see wait_prior_grid), except
// the first step of a dataflow chunk, which waits for all work before it.
template <class TY>
inline bool programmatic(const Step2DArgsT<TY> &a)
{
    return !(a.bands && a.node == 0);
}
template <typename Args>
inline bool programmatic(const Args &)
{
    return true;
}

template <typename Args>
inline cudaError_t launch_serialized(void (*kern)(Args), dim3 grid, dim3 block, cudaStream_t s,
                                     const Args &a)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = programmatic(a) ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

// The wall-density launch that precedes a step whose arguments carry a
// wall-density buffer (Step2DArgs::rw); nothing otherwise.
template <int N, typename T, int NXL, int ZY, int ZX, class Args>
inline cudaError_t launch_wall_rho(const Args &a, int n_inst, cudaStream_t s)
{
    if (!a.rw || a.bc != GLBM_BC_WALLS) return cudaSuccess;
    constexpr int NV = Step2D<N, T, 1, 1, NXL, ZY, ZX>::NV;
    return launch_serialized(k_wall_rho<N, T, NXL, ZY, ZX>, dim3((a.Lx + 31) / 32, n_inst, 2),
                             dim3(32 * NV), s, a);
}

// Launch of tile shape number I of level N.
template <int N, typename T, int I = 0>
cudaError_t launch_step2d_shape(int shape, const Step2DArgs &a, int n_inst, cudaStream_t s)
{
    if constexpr (I < Tiles<N, T>::count) {
        if (shape == I) {
            constexpr TileShape t = Tiles<N, T>::shape[I];
            constexpr int G = t.G, R = t.R, TW = 32 * t.V;
            const dim3 grid((a.Lx + TW - 1) / TW, (a.Ly + R - 1) / R, n_inst);
            const cudaError_t e = launch_wall_rho<N, T, N, 0, 0>(a, n_inst, s);
            if (e != cudaSuccess) return e;
            if constexpr (t.V == 2) {
                static_assert(sizeof(T) == 4, "pair tiles store FP32 deviations");
                return launch_serialized(k_step2d_pair<N, G, R>, grid, dim3(32 * G * R), s, a);
            } else {
                return launch_serialized(k_step2d<N, T, G, R>, grid, dim3(32 * G * R), s, a);
            }
        }
        return launch_step2d_shape<N, T, I + 1>(shape, a, n_inst, s);
    } else {
        return cudaErrorInvalidValue;
    }
}

template <int N, typename T>
cudaError_t glbm_step2d_level(int shape, const Step2DArgs &a, int n_inst, cudaStream_t s)
{
    return launch_step2d_shape<N, T>(shape, a, n_inst, s);
}
