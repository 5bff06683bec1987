// Heterogeneous batches: many independent channel instances of different
// level, size, relaxation time, walls and force advance one step together.
// The work list holds every (instance, x0, y0) tile, grouped by level; a step
// is one launch per level present, each CTA taking one tile of that level and
// running the fused stream-collide tile (glbm_step2d.cuh) with the tile shape
// tuned for the level. All launches of a step are captured in one CUDA graph,
// and only the step's last launch advances the dither counter.
#include "glbm_step2d.cuh"

template <int N>
__global__ void __launch_bounds__(32 * Tile2D<N, float>::G * Tile2D<N, float>::R)
    k_step2d_items(const __grid_constant__ BatchArgs a, int first, int advance)
{
    constexpr int G = Tile2D<N, float>::G, R = Tile2D<N, float>::R;
    using S = Step2D<N, float, G, R>;
    __shared__ typename S::Smem sm;
    const int4 it = a.items[first + blockIdx.x];  // (instance, x0, y0, N)
    const InstParams &ip = a.ip[it.x];
    const float *fin = static_cast<const float *>(a.fin) + ip.off;
    float *fout = static_cast<float *>(a.fout) + ip.off;
    const unsigned seed = hash32(__ldcg(a.step_ctr) * 0x632BE5ABu + (unsigned)it.x);
    S::run(a.tab[N - 1], ip, ip.Lx, ip.Ly, ip.pitch, (int)ip.plane, ip.bc, fin, fout, it.y, it.z, sm,
           a.status, seed);
    if (advance) advance_launch_counter(a.step_ctr, a.done_ctr);
}

int glbm_batched_rows(int N)
{
    switch (N) {
    case 1: return Tile2D<1, float>::R;
    case 2: return Tile2D<2, float>::R;
    case 3: return Tile2D<3, float>::R;
    case 4: return Tile2D<4, float>::R;
    case 5: return Tile2D<5, float>::R;
    case 6: return Tile2D<6, float>::R;
    case 7: return Tile2D<7, float>::R;
    case 8: return Tile2D<8, float>::R;
    default: return 1;
    }
}

template <int N>
static cudaError_t launch_level(const BatchArgs &a, bool last, cudaStream_t s)
{
    const int first = a.group[N], count = a.group[N + 1] - a.group[N];
    if (count <= 0) return cudaSuccess;
    constexpr int threads = 32 * Tile2D<N, float>::G * Tile2D<N, float>::R;
    k_step2d_items<N><<<count, threads, 0, s>>>(a, first, last ? 1 : 0);
    return cudaGetLastError();
}

int glbm_batched_launches(const BatchArgs &a)
{
    int n = 0;
    for (int N = 1; N <= GLBM_MAXN; ++N) n += a.group[N + 1] > a.group[N] ? 1 : 0;
    return n;
}

cudaError_t glbm_launch_batched_f32(const BatchArgs &a, cudaStream_t s)
{
    int lowest = 0;  // the last level launched advances the counter
    for (int N = 1; N <= GLBM_MAXN && !lowest; ++N)
        if (a.group[N + 1] > a.group[N]) lowest = N;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = launch_level<8>(a, lowest == 8, s);
    if (e == cudaSuccess) e = launch_level<7>(a, lowest == 7, s);
    if (e == cudaSuccess) e = launch_level<6>(a, lowest == 6, s);
    if (e == cudaSuccess) e = launch_level<5>(a, lowest == 5, s);
    if (e == cudaSuccess) e = launch_level<4>(a, lowest == 4, s);
    if (e == cudaSuccess) e = launch_level<3>(a, lowest == 3, s);
    if (e == cudaSuccess) e = launch_level<2>(a, lowest == 2, s);
    if (e == cudaSuccess) e = launch_level<1>(a, lowest == 1, s);
    return e;
}
