// Launch sequence of one heterogeneous-batch step: one launch per level
// present, highest level first (the kernels are in glbm_batched.cuh).
#include "glbm_internal.h"

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
    if (e == cudaSuccess) e = glbm_batched_level<8>(a, lowest == 8, s);
    if (e == cudaSuccess) e = glbm_batched_level<7>(a, lowest == 7, s);
    if (e == cudaSuccess) e = glbm_batched_level<6>(a, lowest == 6, s);
    if (e == cudaSuccess) e = glbm_batched_level<5>(a, lowest == 5, s);
    if (e == cudaSuccess) e = glbm_batched_level<4>(a, lowest == 4, s);
    if (e == cudaSuccess) e = glbm_batched_level<3>(a, lowest == 3, s);
    if (e == cudaSuccess) e = glbm_batched_level<2>(a, lowest == 2, s);
    if (e == cudaSuccess) e = glbm_batched_level<1>(a, lowest == 1, s);
    return e;
}

cudaError_t glbm_launch_batched_level(int N, const BatchArgs &a, bool advance, cudaStream_t s)
{
    switch (N) {
    case 1: return glbm_batched_level<1>(a, advance, s);
    case 2: return glbm_batched_level<2>(a, advance, s);
    case 3: return glbm_batched_level<3>(a, advance, s);
    case 4: return glbm_batched_level<4>(a, advance, s);
    case 5: return glbm_batched_level<5>(a, advance, s);
    case 6: return glbm_batched_level<6>(a, advance, s);
    case 7: return glbm_batched_level<7>(a, advance, s);
    case 8: return glbm_batched_level<8>(a, advance, s);
    default: return cudaErrorInvalidValue;
    }
}
