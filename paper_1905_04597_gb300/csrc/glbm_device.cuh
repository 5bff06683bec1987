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

// Whether an earlier step left the positivity domain (status word ST_HALT):
// then the launches of later steps store nothing and do not count, so the
// state stays at the end of the failing step. Read after wait_prior_grid;
// uniform over the grid. The step kernels read it at entry but use it only at
// their stores, so that it delays none of their loads.
__device__ __forceinline__ bool step_halted(const unsigned *status)
{
    return __ldcg(status + ST_HALT) != 0u;
}

// Called by every CTA of a step's last launch: the last CTA to finish advances
// the launch counter that seeds the FP32 dither of the next step (every CTA
// read it before finishing) and the count of completed steps, and sets the
// halt word when a node of this or an earlier step left the positivity
// domain (flag_unstable fences each flag before its CTA reaches the count).
__device__ __forceinline__ void finish_step(unsigned *status)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned total = gridDim.x * gridDim.y * gridDim.z;
        if (atomicAdd(status + ST_DONE, 1u) == total - 1u) {
            status[ST_DONE] = 0u;
            atomicAdd(status + ST_CLOCK, 1u);
            atomicAdd(status + ST_STEPS, 1u);
            if (atomicOr(status + ST_FLAGS, 0u) & 1u) atomicExch(status + ST_HALT, 1u);
        }
    }
}

// Load of a population by the step tiles: an ordinary (weak, L1-cached) load,
// not the read-only path, because in a dataflow chunk (below) another grid may
// still have been writing the input when this one started; the band counts'
// acquire orders those writes before the load. (Measured on GB300: within 1 %
// of the read-only path when the steps do not overlap.)
template <typename T>
__device__ __forceinline__ T ld_pop(const T *p)
{
    return __ldca(p);
}

// ---- dataflow stepping (GLBM_DF_CHUNK, glbm_internal.h) -------------------

// Let the next launch of the stream start its CTAs now (their waits below
// keep them off data that is not ready).
__device__ __forceinline__ void df_launch_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait (bounded) until every band of rows [r0, r1] of instance `inst` counts at
// least `need` finished tiles. Rows outside 0..Ly-1 wrap (periodic along y) or
// clamp (walls). Warp 0 polls, one row per lane per pass; after half a second
// a lane gives up, sets ST_TIMEOUT and ST_HALT (so no later step stores, and
// the host reports the timeout), and the CTA goes on. Every thread of the CTA
// calls it; the barrier at the end orders the acquire before every thread's
// loads.
__device__ __forceinline__ void df_wait_rows(const unsigned *bands, unsigned *status, int inst,
                                             int r0, int r1, int Ly, int R, bool periodic,
                                             unsigned need)
{
    if (threadIdx.x < 32) {
        const int nb = gridDim.y;
        for (int r = r0 + (int)threadIdx.x; r <= r1; r += 32) {
            int row = r;
            if (periodic) {
                row %= Ly;
                if (row < 0) row += Ly;
            } else {
                row = row < 0 ? 0 : (row >= Ly ? Ly - 1 : row);
            }
            const unsigned *c = bands + (long long)inst * nb + row / R;
            if (ld_acquire(c) >= need) continue;
            const unsigned long long t0 = global_ns();
            bool gave_up = false;
            while (ld_acquire(c) < need) {
                // a halted run stores nothing more: stop waiting
                if (ld_acquire(status + ST_HALT) != 0u) {
                    gave_up = true;
                    break;
                }
                __nanosleep(256);
                if (global_ns() - t0 > 500000000ull) {  // 0.5 s
                    atomicOr(status + ST_FLAGS, (unsigned)ST_TIMEOUT);
                    atomicExch(status + ST_HALT, 1u);
                    gave_up = true;
                    break;
                }
            }
            if (gave_up) break;
        }
    }
    __syncthreads();
}

// This CTA's tile of band blockIdx.y of instance `inst` has finished its step:
// after the barrier, one thread adds one to the band count with release
// semantics, which publishes every thread's stores of the CTA (the barrier
// orders them before the release). A fence by every thread would hold each
// warp until its stores land.
__device__ __forceinline__ void df_tile_done(unsigned *bands, int inst)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned *c = bands + (long long)inst * gridDim.y + blockIdx.y;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(c) : "memory");
    }
}

// finish_step of a dataflow launch: its CTAs count in their own word of the
// chunk (launches overlap), the last one advances the clocks.
__device__ __forceinline__ void finish_step_df(unsigned *status, unsigned *done)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned total = gridDim.x * gridDim.y * gridDim.z;
        if (atomicAdd(done, 1u) == total - 1u) {
            atomicAdd(status + ST_CLOCK, 1u);
            atomicAdd(status + ST_STEPS, 1u);
            if (atomicOr(status + ST_FLAGS, 0u) & ST_UNSTABLE) atomicExch(status + ST_HALT, 1u);
        }
    }
}

// A node left the positivity domain: set the status flag, visible device-wide
// before this thread goes on (so before its CTA's finish_step count), the
// only path that pays for a fence.
__device__ __forceinline__ void flag_unstable(unsigned *status)
{
    atomicOr(status + ST_FLAGS, 1u);
    __threadfence();
}

// Product rounded on its own (never contracted into a following addition), so
// that the one-node and the packed pair tiles round alike.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

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
// Second and third random words of a node word, for the stochastic rounding
// of its velocity components (decorrelated from the row words).
__device__ __forceinline__ unsigned dither_word_ux(unsigned hnode) { return hnode * 0x27D4EB2Du; }
__device__ __forceinline__ unsigned dither_word_uy(unsigned hnode) { return hnode * 0x165667B1u; }
__device__ __forceinline__ unsigned dither_word_uz(unsigned hnode) { return hnode * 0xD3A2646Du; }
// Words of the stochastic rounding of a node's equilibrium polynomials, one
// per axis, and a draw in [-2^-23, 2^-23) (two ulps at dither_ulp's scale).
__device__ __forceinline__ unsigned dither_word_ex(unsigned hnode) { return hnode * 0x4CF5AD43u; }
__device__ __forceinline__ unsigned dither_word_ey(unsigned hnode) { return hnode * 0x2545F491u; }
__device__ __forceinline__ unsigned dither_word_ez(unsigned hnode) { return hnode * 0x6A09E667u; }
__device__ __forceinline__ float dither_unit2(unsigned r) { return (float)(int)r * 0x1p-54f; }
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

// Deviation of the level-N equilibrium from the rest weights, for one |n|:
// Ae_n(v) (even powers >= 2) and Bo_n(v) (odd powers / u), v = u^2, so that
// E_{+n}(u) - W_n = Ae + u Bo and E_{-n}(u) - W_n = Ae - u Bo. On the 2N+2
// hierarchy (Z = 1) n is the magnitude index m of the velocities +-(2m+1).
// FP32 keeps Bo in two parts, bo + b0 with b0 the constant (linear)
// coefficient's high part: eq_pm adds u b0 inside the final fused rounding,
// so each value E_{+-n} - W_n is rounded once (a rounded Bo would give a
// fixed relative error of the momentum at each u). FP64: bo = Bo, b0 = 0.
template <int N, typename T, int Z = 0, class Tab>
__device__ __forceinline__ void eq_parts(const Tab &t, int n, T v, T &ae, T &bo, T &b0)
{
    using A = TabAcc<T>;
    T a = A::Ce(t, n, N);
#pragma unroll
    for (int i = N - 1; i >= 1; --i) a = fma(a, v, A::Ce(t, n, i));
    ae = mul_rn(a, v);
    b0 = T(0);
    if (n == 0 && !Z) {
        bo = T(0);  // E_0 is even in u
    } else if (A::HILO) {
        // linear coefficient as hi + lo: the low part joins the higher powers
        T b = A::Co(t, n, N - 1);
        if (N >= 2) {
#pragma unroll
            for (int i = N - 2; i >= 1; --i) b = fma(b, v, A::Co(t, n, i));
            b = fma(b, v, A::C1lo(t, n));
        } else {
            b = A::C1lo(t, n);
        }
        bo = b;
        b0 = A::Co(t, n, 0);
    } else {
        T b = A::Co(t, n, N - 1);
#pragma unroll
        for (int i = N - 2; i >= 0; --i) b = fma(b, v, A::Co(t, n, i));
        bo = b;
    }
}

// E_{+n}(u) - W_n and E_{-n}(u) - W_n from the parts of eq_parts.
template <typename T>
__device__ __forceinline__ void eq_pm(T u, T ae, T bo, T b0, T &plus, T &minus)
{
    if (TabAcc<T>::HILO) {
        plus = fma(u, b0, fma(u, bo, ae));
        minus = fma(-u, b0, fma(-u, bo, ae));
    } else {
        plus = fma(u, bo, ae);
        minus = fma(-u, bo, ae);
    }
}

// FP32 E_{+n}(u) - W_n and E_{-n}(u) - W_n (or E_{+-(2m+1)} on the 2N+2
// hierarchy, n = m) with a stochastic final rounding. Each value is
// a v + (+-u bo) + (+-u b0) with a the even Horner value (Ae = a v) and bo,
// b0 the odd parts of eq_parts; it is rounded once, after a dither that spans
// two ulps of |a v| + |u b0| (a bound of both values up to one binade, so the
// dither covers a power-of-two number of their ulps and the rounding is
// zero-mean). r is a draw in [-2^-23, 2^-23) shared by every n of the axis,
// taken with opposite signs for +n and -n. Deterministic roundings of E - W
// would repeat at every step of a steady flow and act as fixed sources of
// mass and momentum; with the dither they are noise. single: the zero velocity
// of a 2N+1 axis (plus = minus = Ae).
template <int N, int Z = 0, class Tab>
__device__ __forceinline__ void eq_pm_sr(const Tab &t, int n, float u, float v, float r,
                                         float &plus, float &minus)
{
    using A = TabAcc<float>;
    float a = A::Ce(t, n, N);
#pragma unroll
    for (int i = N - 1; i >= 1; --i) a = fmaf(a, v, A::Ce(t, n, i));
    const float av = a * v;
    if (n == 0 && !Z) {  // E_0 is even in u
        plus = minus = fmaf(a, v, dither_ulp(av, r));
        return;
    }
    float b = A::Co(t, n, N - 1);  // odd part without the linear coefficient's high part
    if (N >= 2) {
#pragma unroll
        for (int i = N - 2; i >= 1; --i) b = fmaf(b, v, A::Co(t, n, i));
        b = fmaf(b, v, A::C1lo(t, n));
    } else {
        b = A::C1lo(t, n);
    }
    const float b0 = A::Co(t, n, 0);
    const float del = dither_ulp(fabsf(av) + fabsf(u * b0), r);
    const float sd = fmaf(u, b, del);
    plus = fmaf(u, b0, fmaf(a, v, sd));
    minus = fmaf(-u, b0, fmaf(a, v, -sd));
}

// d[i] = E_i(u) - W_i of every velocity index of the axis in FP32, rounded
// stochastically (eq_pm_sr) with the axis draw r.
template <int N, int Z = 0, class Tab>
__device__ __forceinline__ void eq_dev_all_sr(const Tab &t, float u, float r,
                                              float (&d)[2 * N + 1 + Z])
{
    using AV = AxisVel<N, Z>;
    const float v = u * u;
#pragma unroll
    for (int n = 0; n <= N; ++n) {
        float dp, dm;
        eq_pm_sr<N, Z>(t, n, u, v, r, dp, dm);
        if (n == 0 && !Z) {
            d[N] = dp;
        } else {
            d[AV::ipos(n)] = dp;
            d[AV::ineg(n)] = dm;
        }
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
        T ae, bo, b0;
        eq_parts<N, T, Z>(t, n, v, ae, bo, b0);
        if (n == 0 && !Z) {
            d[N] = ae;
        } else {
            eq_pm(u, ae, bo, b0, d[AV::ipos(n)], d[AV::ineg(n)]);
        }
    }
}

// Two FP32 lanes in one 64-bit register pair, with the two-lane instructions
// of sm_100 and later (add/sub/mul/fma .f32x2): each lane rounds exactly like
// the scalar instruction. The pair tile packs two nodes per thread, the
// one-node tile two velocity columns of one node.
typedef unsigned long long f32x2;  // two FP32 lanes; low word: node x, or the lower column

__device__ __forceinline__ f32x2 pk2(float a, float b)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float lo2(f32x2 v)
{
    float a;
    asm("{ .reg .f32 t; mov.b64 {%0, t}, %1; }" : "=f"(a) : "l"(v));
    return a;
}
__device__ __forceinline__ float hi2(f32x2 v)
{
    float b;
    asm("{ .reg .f32 t; mov.b64 {t, %0}, %1; }" : "=f"(b) : "l"(v));
    return b;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Knuth's two-sum on both lanes (the packed form of acc2).
__device__ __forceinline__ void acc2x2(f32x2 &s, f32x2 &c, f32x2 x)
{
    const f32x2 t = add2(s, x);
    const f32x2 bp = sub2(t, s);
    const f32x2 err = add2(sub2(s, sub2(t, bp)), sub2(x, bp));
    s = t;
    c = add2(c, err);
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
