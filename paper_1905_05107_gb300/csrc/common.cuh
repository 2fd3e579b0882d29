// Shared device helpers of the GB300 ISMA library: device-side iteration
// state, Philox4x32-10, warp/block reductions and the double-float scalar
// used for the small dense algebra of the FP32 path.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#include "../../include/pod.h"

#define POD_WARP 32

// ---------------------------------------------------------------------------
// Device-resident state of one ISMA run.  Every kernel of an iteration reads
// its sizes (t, r_cur, g) from here, so an iteration is a fixed launch
// sequence that can be captured once in a CUDA graph and replayed.
// ---------------------------------------------------------------------------
struct DevState {
    int t;          // index of the next round (0 = first GET UPDATE)
    int r_cur;      // modes carried by U
    int g;          // distinct columns drawn this round
    int done;       // 1: converged, S empty or max_iter reached
    int remaining;  // |S|
    int status;     // pod_status raised on the device (0 = ok)
    int r_new;      // modes kept by this round's merge
    int rounds_run; // rounds completed
    int done_next;  // stop decision of the current round, applied at its end
    int sweeps;     // Jacobi sweeps of the last core SVD
    double measure; // last convergence measure
    double sin_max;
    double cos_min;
    long long core_cycles[6];   // last core SVD: clock64 deltas of its phases
    int robust;     // redo this round's first CholeskyQR pass with a compensated
                    // Gram: set by the plain Cholesky when it dropped a column its
                    // Gram could not resolve, or by the QR2 pass when G2 is far from I
    int robust_rounds;   // rounds that needed it
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64-bit
// multiplies with a Weyl key schedule.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += W0;
        k.y += W1;
    }
    return c;
}

// 64-bit uniform of draw j, round t, stream s: (x0 << 32) | x1.
__device__ __forceinline__ uint64_t philox_u64(uint64_t seed, uint32_t j, uint32_t t, uint32_t s) {
    uint4 r = philox4x32_10(make_uint4(j, t, s, 0u),
                            make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    return ((uint64_t)r.x << 32) | (uint64_t)r.y;
}

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------
template <typename V>
__device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename V>
__device__ __forceinline__ V warp_max(V v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        V u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    return v;
}

// Block-wide sum in a fixed order (deterministic); `red` needs 32 slots.
template <typename V>
__device__ V block_sum(V v, V *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    V s = 0;
    if (wid == 0) {
        s = lane < nw ? red[lane] : (V)0;
        s = warp_sum(s);
        if (lane == 0) red[0] = s;
    }
    __syncthreads();
    s = red[0];
    __syncthreads();
    return s;
}

template <typename V>
__device__ V block_max(V v, V *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_max(v);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        V s = lane < nw ? red[lane] : red[0];
        s = warp_max(s);
        if (lane == 0) red[0] = s;
    }
    __syncthreads();
    V s = red[0];
    __syncthreads();
    return s;
}

// ---------------------------------------------------------------------------
// Double-float scalar: an unevaluated sum hi + lo of two floats (about 44
// significant bits).  GB300 runs FP64 about 58x slower than FP32, so the
// small dense algebra of the FP32 path (Cholesky, triangular inverses, the
// Rayleigh finish of the core SVD) runs in this type on the FP32 pipes.
// Error-free transformations: Knuth's TwoSum and the FMA-based TwoProduct.
// ---------------------------------------------------------------------------
struct dfloat {
    float hi, lo;
};

__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {
    float s = a + b;
    float e = b - (s - a);
    return {s, e};
}
__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
    dfloat s = df_two_sum(a.hi, b.hi);
    dfloat t = df_two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = df_fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return df_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}
// a / b: approximate quotient q1 (2 ulp), then one correction from the exact
// residual a - b q1, giving ~2^-44 relative accuracy without IEEE division.
__device__ __forceinline__ dfloat operator/(dfloat a, dfloat b) {
    const float rb = __frcp_rn(b.hi);
    const float q1 = a.hi * rb;
    const dfloat r = a - b * dfloat{q1, 0.f};
    const float q2 = r.hi * rb;
    return df_fast_two_sum(q1, q2);
}

// Accumulator of a sum of products (a dot product) over X.  X = double: FMA.
// X = dfloat: the compensated dot product "Dot2" of Ogita, Rump and Oishi
// (SIAM J. Sci. Comput. 26, 2005): the rounded sum s is carried with TwoSum,
// the rounding errors of the sums and of the products (TwoProduct, plus the
// low-part cross terms of the double-float operands) are collected in c; the
// result s + c is as accurate as a sum taken in twice the working precision,
// with a dependent chain of about eight FP32 operations per term instead of
// the ~20 of a double-float add.  Two accumulators per loop (even and odd
// terms) let the chains overlap.
template <typename X> struct Acc;
template <> struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double get() const { return s; }
};
template <> struct Acc<dfloat> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(dfloat a, dfloat b) {
        const float p = a.hi * b.hi;
        const float e = fmaf(a.hi, b.hi, -p) + fmaf(a.hi, b.lo, a.lo * b.hi);
        const float t = s + p;
        const float bb = t - s;
        c += ((s - (t - bb)) + (p - bb)) + e;
        s = t;
    }
    __device__ __forceinline__ dfloat get() const { return df_fast_two_sum(s, c); }
};

// Scalar traits: the small dense algebra is written once over X = double
// (FP64 path) or X = dfloat (FP32 path).
template <typename X> struct XOps;
template <> struct XOps<double> {
    __device__ static double from(double d) { return d; }
    __device__ static double from_f(float f) { return (double)f; }
    __device__ static double to(double x) { return x; }
    __device__ static double sqrt_(double x) { return sqrt(x); }
    __device__ static double zero() { return 0.0; }
    __device__ static double one() { return 1.0; }
};
template <> struct XOps<dfloat> {
    __device__ static dfloat from(double d) {
        float hi = (float)d;
        return {hi, (float)(d - (double)hi)};
    }
    __device__ static dfloat from_f(float f) { return {f, 0.f}; }
    __device__ static double to(dfloat x) { return (double)x.hi + (double)x.lo; }
    __device__ static dfloat sqrt_(dfloat a) {
        if (!(a.hi > 0.f)) return {0.f, 0.f};
        const float rs = rsqrtf(a.hi);
        const float s = a.hi * rs;                       // sqrt(a.hi), ~2 ulp
        const dfloat r = a - dfloat{s, 0.f} * dfloat{s, 0.f};
        return df_fast_two_sum(s, 0.5f * r.hi * rs);     // one Newton step from the exact residual
    }
    __device__ static dfloat zero() { return {0.f, 0.f}; }
    __device__ static dfloat one() { return {1.f, 0.f}; }
};

template <> struct XOps<float> {
    __device__ static float from(double d) { return (float)d; }
    __device__ static float from_f(float f) { return f; }
    __device__ static double to(float x) { return (double)x; }
    __device__ static float sqrt_(float x) { return sqrtf(x); }
    __device__ static float zero() { return 0.f; }
    __device__ static float one() { return 1.f; }
};

__device__ __forceinline__ bool x_gt(float a, float b) { return a > b; }
__device__ __forceinline__ bool x_gt(double a, double b) { return a > b; }
__device__ __forceinline__ bool x_gt(dfloat a, dfloat b) {
    return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo);
}
__device__ __forceinline__ float x_hi(float a) { return a; }
__device__ __forceinline__ float x_hi(double a) { return (float)a; }
__device__ __forceinline__ float x_hi(dfloat a) { return a.hi; }
// Rotation arithmetic of the Jacobi sweeps: fast reciprocals on the FP32
// path (a rotation need not be exact, only applied consistently to the
// columns and to V), IEEE on the FP64 path.
__device__ __forceinline__ float j_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double j_div(double a, double b) { return a / b; }
__device__ __forceinline__ float j_rsqrt(float a) { return rsqrtf(a); }
__device__ __forceinline__ double j_rsqrt(double a) { return 1.0 / sqrt(a); }

__device__ __forceinline__ double x_shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ dfloat x_shfl_xor(dfloat v, int o) {
    return {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

// ---------------------------------------------------------------------------
// Host-side error plumbing
// ---------------------------------------------------------------------------
#define POD_CUDA_TRY(expr)                                         \
    do {                                                           \
        cudaError_t _e = (expr);                                   \
        if (_e != cudaSuccess) return POD_ECUDA;                   \
    } while (0)

#define POD_TRY(expr)                                              \
    do {                                                           \
        pod_status _s = (expr);                                    \
        if (_s != POD_OK) return _s;                               \
    } while (0)

static inline int pod_ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// CTAs per first-level group of the in-kernel partial sums (tall_reduce)
constexpr int RED_GROUP = 16;

// Sum of FP64 partials inside the kernel: the last CTA to arrive in each
// group of RED_GROUP CTAs sums that group's partials; the last group to
// finish sums the group results.  Orders are fixed by block index; arrival
// counters are reset by the CTAs that consumed them.  Returns true on the CTA
// that wrote the final sums.
__device__ inline bool tall_reduce(const double *part, double *gsum, double *out, int count, int64_t stride,
                            unsigned *counters, int *s_flag) {
    const int tid = threadIdx.x;
    const int grid = gridDim.x;
    const int ngroups = (grid + RED_GROUP - 1) / RED_GROUP;
    const int grp = blockIdx.x / RED_GROUP;
    const int gsize = min(RED_GROUP, grid - grp * RED_GROUP);
    __threadfence();
    __syncthreads();
    if (tid == 0) *s_flag = (atomicAdd(&counters[grp], 1u) == (unsigned)(gsize - 1));
    __syncthreads();
    if (!*s_flag) return false;
    __threadfence();
    for (int e = tid; e < count; e += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < gsize; ++b) s += __ldcg(part + (int64_t)(grp * RED_GROUP + b) * stride + e);
        gsum[(int64_t)grp * stride + e] = s;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        counters[grp] = 0;
        *s_flag = (atomicAdd(&counters[ngroups], 1u) == (unsigned)(ngroups - 1));
    }
    __syncthreads();
    if (!*s_flag) return false;
    __threadfence();
    for (int e = tid; e < count; e += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < ngroups; ++b) s += __ldcg(gsum + (int64_t)b * stride + e);
        out[e] = s;
    }
    if (tid == 0) counters[ngroups] = 0;
    return true;   // this CTA wrote out (the last to arrive)
}
