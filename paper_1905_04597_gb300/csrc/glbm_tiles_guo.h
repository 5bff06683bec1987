// Tile shape of the fused 2D step with Guo's force, per level, precision and
// lattice kind: the first one-node (V = 1) entry of the kind's candidate list.
#pragma once
#include "glbm_tiles.h"
#include "glbm_tiles_zv.h"

template <int N, typename T, int KIND>
struct GuoList;
template <int N, typename T>
struct GuoList<N, T, GLBM_GUOK_ISO> : Tiles<N, T> {};
template <int N, typename T>
struct GuoList<N, T, GLBM_GUOK_X1> : TilesX1<N, T> {};
template <int N, typename T>
struct GuoList<N, T, GLBM_GUOK_ZV> : TilesZv<N, T, GLBM_ZVK_X1> {};

// index of the first one-node (V = 1) shape of a candidate list
template <class L>
constexpr int first_one_node()
{
    for (int i = 0; i < L::count; ++i)
        if (L::shape[i].V == 1) return i;
    return -1;
}

template <int N, typename T, int KIND>
constexpr TileShape guo_shape()
{
    using L = GuoList<N, T, KIND>;
    static_assert(first_one_node<L>() >= 0, "no one-node tile for this level");
    return L::shape[first_one_node<L>()];
}
