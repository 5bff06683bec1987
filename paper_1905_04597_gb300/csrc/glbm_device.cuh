// Device helpers shared by the libglbm kernels: table access by precision,
// Horner evaluation of the equilibrium polynomials, compensated addition.
#pragma once
#include "glbm_internal.h"
#include "../../include/glbm.h"

template <typename T>
struct TabAcc;

template <>
struct TabAcc<double> {
    static constexpr bool HILO = false;
    template <class Tab>
    static __device__ __forceinline__ double C1lo(const Tab &, int) { return 0.0; }
    template <class Tab>
    static __device__ __forceinline__ double W(const Tab &t, int i) { return t.W[i]; }
    template <class Tab>
    static __device__ __forceinline__ double WN(const Tab &t, int i) { return t.WN[i]; }
    template <class Tab>
    static __device__ __forceinline__ double Ce(const Tab &t, int n, int i) { return t.Ce[n][i]; }
    template <class Tab>
    static __device__ __forceinline__ double Co(const Tab &t, int n, int i) { return t.Co[n][i]; }
};

template <>
struct TabAcc<float> {
    static constexpr bool HILO = true;
    template <class Tab>
    static __device__ __forceinline__ float C1lo(const Tab &t, int n) { return t.Co1lo[n]; }
    template <class Tab>
    static __device__ __forceinline__ float W(const Tab &t, int i) { return t.Wf[i]; }
    template <class Tab>
    static __device__ __forceinline__ float WN(const Tab &t, int i) { return t.WNf[i]; }
    template <class Tab>
    static __device__ __forceinline__ float Ce(const Tab &t, int n, int i) { return t.Cef[n][i]; }
    template <class Tab>
    static __device__ __forceinline__ float Co(const Tab &t, int n, int i) { return t.Cof[n][i]; }
};

// Programmatic dependent launch: the uniform step kernels are launched with
// programmatic stream serialization (launch_serialized), so a launch's CTAs
// are scheduled while the previous step's grid drains. This wait holds them
// until that grid has completed and its writes are visible (a no-op for a
// launch without a programmatic dependency); it precedes every global access.
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Product rounded on its own (never contracted into a following addition), so
// that the one-node and the packed pair tiles round alike.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// Deviation of the level-N equilibrium from the rest weights, for one |n|:
// Ae_n(v) (even powers >= 2) and Bo_n(v) (odd powers / u), v = u^2, so that
// E_{+n}(u) - W_n = Ae + u Bo and E_{-n}(u) - W_n = Ae - u Bo. On the 2N+2
// hierarchy (Z = 1) n is the magnitude index m of the velocities +-(2m+1).
template <int N, typename T, int Z = 0, class Tab>
__device__ __forceinline__ void eq_parts(const Tab &t, int n, T v, T &ae, T &bo)
{
    using A = TabAcc<T>;
    T a = A::Ce(t, n, N);
#pragma unroll
    for (int i = N - 1; i >= 1; --i) a = fma(a, v, A::Ce(t, n, i));
    ae = mul_rn(a, v);
    if (n == 0 && !Z) {
        bo = T(0);  // E_0 is even in u
    } else if (A::HILO) {
        // linear coefficient as hi + lo: the low part joins before the high part
        T b = A::Co(t, n, N - 1);
        if (N >= 2) {
#pragma unroll
            for (int i = N - 2; i >= 1; --i) b = fma(b, v, A::Co(t, n, i));
            b = fma(b, v, A::C1lo(t, n));
        } else {
            b = A::C1lo(t, n);
        }
        bo = b + A::Co(t, n, 0);
    } else {
        T b = A::Co(t, n, N - 1);
#pragma unroll
        for (int i = N - 2; i >= 0; --i) b = fma(b, v, A::Co(t, n, i));
        bo = b;
    }
}

// d[i] = E_i(u) - W_i for every velocity index i of the axis (i = n + N on
// the 2N+1 hierarchy).
template <int N, typename T, int Z = 0, class Tab>
__device__ __forceinline__ void eq_dev_all(const Tab &t, T u, T (&d)[2 * N + 1 + Z])
{
    using AV = AxisVel<N, Z>;
    const T v = u * u;
#pragma unroll
    for (int n = 0; n <= N; ++n) {
        T ae, bo;
        eq_parts<N, T, Z>(t, n, v, ae, bo);
        if (n == 0 && !Z) {
            d[N] = ae;
        } else {
            d[AV::ipos(n)] = fma(u, bo, ae);
            d[AV::ineg(n)] = fma(-u, bo, ae);
        }
    }
}

// E_n(u) - W_n for a single n (compile-time after unrolling).
template <int N, typename T, class Tab>
__device__ __forceinline__ T eq_dev_one(const Tab &t, T u, int n)
{
    const int an = n < 0 ? -n : n;
    T ae, bo;
    eq_parts<N, T>(t, an, u * u, ae, bo);
    if (an == 0) return ae;
    return n > 0 ? fma(u, bo, ae) : fma(-u, bo, ae);
}

// Knuth's two-sum: s + x is added to (s, c) with the rounding error of the
// addition carried in c (compensated summation of the FP32 moments).
__device__ __forceinline__ void acc2(float &s, float &c, float x)
{
    const float t = s + x;
    const float bp = t - s;
    const float err = (s - (t - bp)) + (x - bp);
    s = t;
    c += err;
}
__device__ __forceinline__ void acc2(double &s, double &c, double x)
{
    (void)c;
    s += x;
}

// 32-bit integer hash (xorshift-multiply), used to draw the dither of the
// FP32 stores from (launch, instance, node).
__device__ __forceinline__ unsigned hash32(unsigned x)
{
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// Dither for the FP32 store of `ref + inc`: u times the power of two of ref's
// exponent (0 for zero and subnormal ref), with u uniform in [-2^-24, 2^-24),
// i.e. uniform in [-1/2, 1/2) units in the last place of `ref`. Adding it to
// the increment before the final rounding makes the rounding error zero-mean,
// so a steady state does not repeat the same rounding error at every step
// (whose effect on slowly relaxing moments would grow like 1/omega).
__device__ __forceinline__ float dither_ulp(float ref, float u)
{
    return u * __int_as_float(__float_as_int(ref) & 0x7F800000);
}

// A draw u in [-2^-24, 2^-24) from the random word r (the signed word times
// 2^-55). Each (launch, node, velocity row) draws two, a and b; the row's
// velocity columns take a, b, -a, -b in turn, so every population's dither is
// uniform and fresh at every launch while the draw costs nothing per population.
__device__ __forceinline__ float dither_unit(unsigned r)
{
    return (float)(int)r * 0x1p-55f;
}
__device__ __forceinline__ unsigned dither_word_b(unsigned hrow)
{
    return hrow * 0x9E3779B9u;
}
template <class U>
__device__ __forceinline__ U dither_pick(int ix, U a, U b, U na, U nb)
{
    switch (ix & 3) {
    case 0: return a;
    case 1: return b;
    case 2: return na;
    default: return nb;
    }
}

__device__ __forceinline__ int wrap_index(int i, int L)
{
    i %= L;
    return i < 0 ? i + L : i;
}

// i mod L for a column or row index shifted by at most one period (-L <= i <
// 2L): two selects instead of a division. `one_wrap` (L larger than the
// largest shift, uniform across the launch) selects it; otherwise the
// remainder is taken.
__device__ __forceinline__ int wrap_shift(int i, int L, bool one_wrap)
{
    if (one_wrap) return i < 0 ? i + L : (i >= L ? i - L : i);
    return wrap_index(i, L);
}
