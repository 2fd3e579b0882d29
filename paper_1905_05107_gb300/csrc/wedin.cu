// Quality of the converged solution (Sec. 3.3, Eq. 7): after the closing
// refinement the approximate top-k triplets are U~_k (the refined modes),
// sigma~_k and V~_k = (A^T U) K (K from the refinement SVD).  This file forms
//   |S|_F^2 = |A^T U~_k - V~_k Sigma~_k|_F^2   (n x k, from Y = A^T U in FP64)
//   |R|_F^2 = |A V~_k - U~_k Sigma~_k|_F^2     (m x k, one pass over A)
// The right-hand side of Eq. 7 follows on the host with omega estimated from
// sigma~_k and sigma~_{k+1}.  R is a small difference of large terms, so the
// FP32 path accumulates A V~_k with exact products (TwoProduct) summed by
// TwoSum, against V~_k held as double-float.
#include "pod_internal.h"

namespace {

constexpr int WT = 256;      // threads per CTA (one row or column each)
constexpr int WCH = 128;     // columns of A per shared-memory chunk of V~
constexpr int WKB = 32;      // modes per pass over A

// V~_k = Y K[:, :k] (FP64 and double-float copies) and the partial |S|^2:
// S = Y V_R[:, :k] - V~_k diag(sigma).  Y: n x r, ld n; K, V_R: r x r, ld r.
__global__ void __launch_bounds__(WT) k_wedin_v(WedinArgs a) {
    __shared__ double red[32];
    __shared__ int s_flag;
    const int64_t j = (int64_t)blockIdx.x * WT + threadIdx.x;
    double s2 = 0.0;
    if (j < a.n) {
        for (int l = 0; l < a.k; ++l) {
            double v = 0.0, y = 0.0;
            for (int q = 0; q < a.r; ++q) {
                const double yq = a.Y[(int64_t)q * a.n + j];
                v = fma(yq, a.K[q * a.r + l], v);
                y = fma(yq, a.VR[q * a.r + l], y);
            }
            const double sres = y - v * a.sigma[l];
            s2 = fma(sres, sres, s2);
            a.Vk[(int64_t)l * a.n + j] = v;
            const float hi = (float)v;
            a.Vkf[(int64_t)l * a.n + j] = make_float2(hi, (float)(v - (double)hi));
        }
    }
    s2 = block_sum<double>(s2, red);
    if (threadIdx.x == 0) a.part_s[blockIdx.x] = s2;
    tall_reduce(a.part_s, a.gsum_s, a.out, 1, 1, a.counters_v, &s_flag);
}

// Partial |R|^2 over the rows of this CTA for modes [l0, l0 + kb).
template <typename T>
__global__ void __launch_bounds__(WT) k_wedin_r(WedinArgs a, const T *__restrict__ A, const T *__restrict__ U,
                                               int l0, int kb) {
    __shared__ double red[32];
    __shared__ int s_flag;
    __shared__ float2 vs[WCH * WKB];   // V~ chunk, entry (c, l) at c * WKB + l
    const int64_t i = (int64_t)blockIdx.x * WT + threadIdx.x;
    const bool row = i < a.m;
    float ahi[WKB], alo[WKB];
    double ad[WKB];
#pragma unroll
    for (int l = 0; l < WKB; ++l) {
        ahi[l] = 0.f;
        alo[l] = 0.f;
        ad[l] = 0.0;
    }
    for (int64_t j0 = 0; j0 < a.n; j0 += WCH) {
        const int nch = (int)(a.n - j0 < WCH ? a.n - j0 : WCH);
        __syncthreads();
        for (int e = threadIdx.x; e < nch * WKB; e += WT) {
            const int c = e / WKB, l = e - c * WKB;
            vs[e] = l < kb ? a.Vkf[(int64_t)(l0 + l) * a.n + j0 + c] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        if (!row) continue;
        for (int c = 0; c < nch; ++c) {
            const T x = A[(j0 + c) * a.lda + i];
            if constexpr (sizeof(T) == 4) {
#pragma unroll
                for (int l = 0; l < WKB; ++l) {
                    const float2 v = vs[c * WKB + l];
                    const float p = x * v.x;
                    float e = fmaf(x, v.x, -p);
                    e = fmaf(x, v.y, e);
                    const dfloat t = df_two_sum(ahi[l], p);
                    ahi[l] = t.hi;
                    alo[l] += t.lo + e;
                }
            } else {
#pragma unroll
                for (int l = 0; l < WKB; ++l) {
                    const float2 v = vs[c * WKB + l];
                    ad[l] = fma((double)x, (double)v.x + (double)v.y, ad[l]);
                }
            }
        }
    }
    double r2 = 0.0;
    if (row) {
#pragma unroll
        for (int l = 0; l < WKB; ++l) {
            if (l < kb) {
                const double av = sizeof(T) == 4 ? (double)ahi[l] + (double)alo[l] : ad[l];
                const double res = av - (double)U[(int64_t)(l0 + l) * a.m + i] * a.sigma[l0 + l];
                r2 = fma(res, res, r2);
            }
        }
    }
    r2 = block_sum<double>(r2, red);
    if (threadIdx.x == 0) a.part_r[blockIdx.x] = r2;
    tall_reduce(a.part_r, a.gsum_r, a.out + 1 + (l0 / WKB), 1, 1, a.counters_r, &s_flag);
}

}  // namespace

int wedin_grid_n(int64_t n) { return (int)((n + WT - 1) / WT); }
int wedin_grid_m(int64_t m) { return (int)((m + WT - 1) / WT); }
int wedin_passes(int k) { return (k + WKB - 1) / WKB; }

template <typename T>
pod_status launch_wedin(const WedinArgs &a, const T *A, const T *U, cudaStream_t s) {
    k_wedin_v<<<wedin_grid_n(a.n), WT, 0, s>>>(a);
    POD_CUDA_TRY(cudaGetLastError());
    for (int l0 = 0; l0 < a.k; l0 += WKB) {
        const int kb = a.k - l0 < WKB ? a.k - l0 : WKB;
        k_wedin_r<T><<<wedin_grid_m(a.m), WT, 0, s>>>(a, A, U, l0, kb);
        POD_CUDA_TRY(cudaGetLastError());
    }
    return POD_OK;
}

template pod_status launch_wedin<float>(const WedinArgs &, const float *, const float *, cudaStream_t);
template pod_status launch_wedin<double>(const WedinArgs &, const double *, const double *, cudaStream_t);
