// Heterogeneous batches: many independent channel instances of different
// level, size, relaxation time, walls and force advance one step together.
// The work list holds every (instance, x0, y0) tile, grouped by level; a step
// is one launch per level present, each CTA taking one tile of that level and
// running the fused stream-collide tile (one-node or packed pair) with the
// level's tile shape. All launches of a step are captured in one CUDA graph, and only
// the step's last launch advances the dither counter.
#pragma once
#include "glbm_step2d_pair.cuh"
#include "glbm_tiles.h"

template <int N, int G, int R>
__global__ void __launch_bounds__(32 * G * R)
    k_step2d_items(const __grid_constant__ BatchArgs a, int first, int advance)
{
    using S = Step2D<N, float, G, R>;
    __shared__ typename S::Smem sm;
    const bool live = !step_halted(a.status);  // needed only at the stores
    const int4 it = a.items[first + blockIdx.x];  // (instance, x0, y0, N)
    const InstParams &ip = a.ip[it.x];
    const float *fin = static_cast<const float *>(a.fin) + ip.off;
    float *fout = static_cast<float *>(a.fout) + ip.off;
    const unsigned seed = hash32(__ldcg(a.step_ctr) * 0x632BE5ABu + (unsigned)it.x);
    S::run(a.tab[N - 1], a.tab[N - 1], ip, ip.Lx, ip.Ly, ip.pitch, (int)ip.plane, ip.bc, fin, fout,
           it.y, it.z, sm, a.status, seed, nullptr, live);
    if (advance && live) finish_step(a.status);
}

template <int N, int G, int R>
__global__ void __launch_bounds__(32 * G * R)
    k_step2d_pair_items(const __grid_constant__ BatchArgs a, int first, int advance)
{
    using S = Step2DPair<N, G, R>;
    __shared__ __align__(16) typename S::Smem sm;
    const bool live = !step_halted(a.status);  // needed only at the stores
    const int4 it = a.items[first + blockIdx.x];  // (instance, x0, y0, N)
    const InstParams &ip = a.ip[it.x];
    const float *fin = static_cast<const float *>(a.fin) + ip.off;
    float *fout = static_cast<float *>(a.fout) + ip.off;
    const unsigned seed = hash32(__ldcg(a.step_ctr) * 0x632BE5ABu + (unsigned)it.x);
    S::run(a.tab[N - 1], a.tab[N - 1], ip, ip.Lx, ip.Ly, ip.pitch, (int)ip.plane, ip.bc, fin, fout,
           it.y, it.z, sm, a.status, seed, nullptr, live);
    if (advance && live) finish_step(a.status);
}

template <int N, int I = 0>
cudaError_t launch_items_shape(const BatchArgs &a, int first, int count, bool advance,
                               cudaStream_t s)
{
    if constexpr (I < Tiles<N, float>::count) {
        if (a.shape[N] == I) {
            constexpr TileShape t = Tiles<N, float>::shape[I];
            constexpr int G = t.G, R = t.R;
            if constexpr (t.V == 2)
                k_step2d_pair_items<N, G, R><<<count, 32 * G * R, 0, s>>>(a, first, advance ? 1 : 0);
            else
                k_step2d_items<N, G, R><<<count, 32 * G * R, 0, s>>>(a, first, advance ? 1 : 0);
            return cudaGetLastError();
        }
        return launch_items_shape<N, I + 1>(a, first, count, advance, s);
    } else {
        return cudaErrorInvalidValue;
    }
}

template <int N>
cudaError_t glbm_batched_level(const BatchArgs &a, bool advance, cudaStream_t s)
{
    const int first = a.group[N], count = a.group[N + 1] - a.group[N];
    if (count <= 0) return cudaSuccess;
    return launch_items_shape<N>(a, first, count, advance, s);
}
