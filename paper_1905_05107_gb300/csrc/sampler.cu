// Column norms, integer sampling weights, Philox draws and de-duplication:
// the probability and draw steps of ISMA (Algorithm 1: GET UPDATE's I_s, I_c,
// S <- S \ I_c; Sec. 3.1 sampling strategies; Eq. 2 column-norm weights).
#include "pod_internal.h"

// ---------------------------------------------------------------------------
// s_j = sum_i a_ij^2.  FP32 data: each square is split exactly into
// p + e (TwoProduct) and summed with TwoSum into a (hi, lo) pair per thread,
// so every thread's partial carries ~44 bits; partials are then combined in
// FP64 in a fixed order.  One CTA per column (grid-stride over columns);
// float4 loads when the column start is 16-byte aligned.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_colnorms(const T *__restrict__ A, int64_t m, int64_t n,
                                                  int64_t lda, double *__restrict__ s) {
    __shared__ double red[32];
    for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
        const T *col = A + j * lda;
        double part;
        if constexpr (sizeof(T) == 4) {
            dfloat acc{0.f, 0.f};
            int64_t i = threadIdx.x * 4;
            const bool vec = ((reinterpret_cast<uintptr_t>(col) & 15) == 0);
            if (vec) {
                const int64_t m4 = m & ~(int64_t)3;
                for (; i < m4; i += (int64_t)blockDim.x * 4) {
                    float4 v = *reinterpret_cast<const float4 *>(col + i);
                    float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        float p = vv[u] * vv[u];
                        float e = fmaf(vv[u], vv[u], -p);
                        dfloat t = df_two_sum(acc.hi, p);
                        acc.hi = t.hi;
                        acc.lo += t.lo + e;
                    }
                }
                for (int64_t q = m4 + threadIdx.x; q < m; q += blockDim.x) {
                    float v = col[q];
                    float p = v * v, e = fmaf(v, v, -p);
                    dfloat t = df_two_sum(acc.hi, p);
                    acc.hi = t.hi;
                    acc.lo += t.lo + e;
                }
            } else {
                for (int64_t q = threadIdx.x; q < m; q += blockDim.x) {
                    float v = col[q];
                    float p = v * v, e = fmaf(v, v, -p);
                    dfloat t = df_two_sum(acc.hi, p);
                    acc.hi = t.hi;
                    acc.lo += t.lo + e;
                }
            }
            part = (double)acc.hi + (double)acc.lo;
        } else {
            double acc = 0.0;
            for (int64_t q = threadIdx.x; q < m; q += blockDim.x) acc = fma(col[q], col[q], acc);
            part = acc;
        }
        double tot = block_sum<double>(part, red);
        if (threadIdx.x == 0) s[j] = tot;
    }
}

pod_status launch_colnorms(const void *A, int dtype, int64_t m, int64_t n, int64_t lda,
                           double *s, cudaStream_t st) {
    if (n <= 0) return POD_OK;
    int grid = (int)(n < 65535 ? n : 65535);
    if (dtype == POD_F32)
        k_colnorms<float><<<grid, 256, 0, st>>>((const float *)A, m, n, lda, s);
    else
        k_colnorms<double><<<grid, 256, 0, st>>>((const double *)A, m, n, lda, s);
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}

// ---------------------------------------------------------------------------
// Block-wide inclusive scan (1024 threads max) of uint64 / int values.
// ---------------------------------------------------------------------------
template <typename V>
__device__ V block_inclusive_scan(V v, V *warp_tot) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        V u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    __syncthreads();
    if (lane == 31) warp_tot[wid] = v;
    __syncthreads();
    if (wid == 0) {
        V w = lane < nw ? warp_tot[lane] : (V)0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            V u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += u;
        }
        if (lane < nw) warp_tot[lane] = w;
    }
    __syncthreads();
    if (wid > 0) v += warp_tot[wid - 1];
    return v;
}

// ---------------------------------------------------------------------------
// Integer weights over the remaining set S.
//   mode 0 (L2N):  value_j = s_j            (Eq. 2)
//   mode 1 (UNF):  value_j = 1
//   mode 2 (ORT):  value_j = ort_j          (Eq. 6)
//   mode 3 (given): w_j supplied by the caller (pod_sample)
// w_j = floor(value_j / max_{S} value * 2^L), L = 62 - ceil(log2(n+1)); if
// every w_j is 0 on S the weights become 1 on S (uniform fallback).
// Then c Philox draws, binary search of the inclusive prefix sums, distinct
// draws in ascending order, S <- S \ I_c.  One CTA of 1024 threads.
// ---------------------------------------------------------------------------


__global__ void __launch_bounds__(1024) k_sample(SampleArgs a) {
    __shared__ uint64_t red64[32];
    __shared__ double redd[32];
    __shared__ int redi[32];
    __shared__ int s_g;
    DevState *st = a.st;
    if (st && st->done) return;
    const int t = st ? st->t : a.t_fixed;
    const int64_t n = a.n;

    if (st && a.s) {
        // a column norm that is not finite means a NaN or an infinity in A:
        // the run stops with POD_ENAN before any merge uses the column
        int bad = 0;
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x) bad |= !isfinite(a.s[j]);
        if (__syncthreads_or(bad)) {
            if (threadIdx.x == 0) {
                st->status = POD_ENAN;
                st->done = 1;
            }
            return;
        }
    }

    if (a.replay_idx) {
        // frozen draws: round t merges replay list t
        if (t >= a.replay_T) {
            if (threadIdx.x == 0 && st) {
                st->done = 1;
                st->g = 0;
            }
            return;
        }
        const int b = a.replay_off[t], e = a.replay_off[t + 1];
        for (int j = b + threadIdx.x; j < e; j += blockDim.x) a.flags[a.replay_idx[j]] = 1;
    } else {
        const int mode = (t == 0) ? a.mode_round0 : a.mode;
        if (mode != 3) {
            double vmax = 0.0;
            for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
                if (!a.mask[j]) continue;
                double v = mode == 0 ? a.s[j] : (mode == 1 ? 1.0 : a.ort[j]);
                vmax = v > vmax ? v : vmax;
            }
            vmax = block_max<double>(vmax, redd);
            for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
                uint64_t wj = 0;
                if (a.mask[j] && vmax > 0.0) {
                    double v = mode == 0 ? a.s[j] : (mode == 1 ? 1.0 : a.ort[j]);
                    wj = (uint64_t)floor(ldexp(v / vmax, a.L));
                }
                a.w[j] = wj;
            }
        } else {
            for (int64_t j = threadIdx.x; j < n; j += blockDim.x)
                if (!a.mask[j]) a.w[j] = 0;
        }
        __syncthreads();
        // prefix sums in chunks of blockDim
        uint64_t carry = 0;
        for (int64_t base = 0; base < n; base += blockDim.x) {
            int64_t j = base + threadIdx.x;
            uint64_t v = j < n ? a.w[j] : 0;
            uint64_t inc = block_inclusive_scan<uint64_t>(v, red64);
            if (j < n) a.cdf[j] = carry + inc;
            __syncthreads();
            uint64_t chunk_tot = red64[((blockDim.x + 31) >> 5) - 1];
            __syncthreads();
            carry += chunk_tot;
        }
        uint64_t total = carry;
        if (total == 0) {
            // uniform over S
            carry = 0;
            for (int64_t base = 0; base < n; base += blockDim.x) {
                int64_t j = base + threadIdx.x;
                uint64_t v = (j < n && a.mask[j]) ? 1 : 0;
                if (j < n) a.w[j] = v;
                uint64_t inc = block_inclusive_scan<uint64_t>(v, red64);
                if (j < n) a.cdf[j] = carry + inc;
                __syncthreads();
                uint64_t chunk_tot = red64[((blockDim.x + 31) >> 5) - 1];
                __syncthreads();
                carry += chunk_tot;
            }
            total = carry;
        }
        __syncthreads();
        if (total > 0) {
            for (int j = threadIdx.x; j < a.c; j += blockDim.x) {
                uint64_t u = philox_u64(a.seed, (uint32_t)j, (uint32_t)t, (uint32_t)a.stream_id);
                uint64_t v = __umul64hi(u, total);
                // smallest i with cdf[i] > v
                int64_t lo = 0, hi = n - 1;
                while (lo < hi) {
                    int64_t mid = (lo + hi) >> 1;
                    if (a.cdf[mid] > v) hi = mid; else lo = mid + 1;
                }
                a.draws[j] = (int32_t)lo;
                a.flags[lo] = 1;
            }
        }
    }
    __syncthreads();
    // ascending distinct draws, S <- S \ I_c, clear flags
    int carry = 0;
    for (int64_t base = 0; base < n; base += blockDim.x) {
        int64_t j = base + threadIdx.x;
        int f = (j < n) ? (int)a.flags[j] : 0;
        int inc = block_inclusive_scan<int>(f, redi);
        if (f) {
            a.idx[carry + inc - 1] = (int32_t)j;
            a.flags[j] = 0;
            a.mask[j] = 0;
        }
        __syncthreads();
        int chunk_tot = redi[((blockDim.x + 31) >> 5) - 1];
        __syncthreads();
        carry += chunk_tot;
    }
    if (threadIdx.x == 0) s_g = carry;
    __syncthreads();
    const int g = s_g;
    // remaining |S|
    int cnt = 0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) cnt += a.mask[j] ? 1 : 0;
    cnt = block_sum<int>(cnt, redi);
    if (a.hist_idx && st) {
        for (int j = threadIdx.x; j < g; j += blockDim.x) a.hist_idx[(int64_t)t * a.c + j] = a.idx[j];
    }
    if (threadIdx.x == 0) {
        if (st) {
            st->g = g;
            st->remaining = cnt;
            if (a.hist_g) a.hist_g[t] = g;
        }
        if (a.g_out) *a.g_out = g;
    }
}

int weight_bits(int64_t n) {
    int b = 0;
    while (((int64_t)1 << b) < n + 1) ++b;   // ceil(log2(n + 1))
    return 62 - b;
}

pod_status launch_sample(const SampleArgs &a, cudaStream_t st) {
    k_sample<<<1, 1024, 0, st>>>(a);
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}

// ---------------------------------------------------------------------------
// ORT values (Eq. 6): ort_j = max(0, s_j - |U^T a_j|^2) from Y = A^T U.
// ---------------------------------------------------------------------------
__global__ void k_ort_values(const double *__restrict__ s, const double *__restrict__ Y, int64_t n,
                             int ldy, const DevState *st, const uint8_t *__restrict__ mask,
                             double *__restrict__ ort) {
    if (st->done) return;
    const int r = st->r_cur;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        if (!mask[j]) { ort[j] = 0.0; continue; }
        double q = 0.0;
        for (int l = 0; l < r; ++l) {
            double y = Y[(int64_t)l * n + j];
            q += y * y;
        }
        double v = s[j] - q;
        ort[j] = v > 0.0 ? v : 0.0;
    }
}

pod_status launch_ort_values(const double *s, const double *Y, int64_t n, int ldy,
                             const DevState *st, const uint8_t *mask, double *ort, cudaStream_t stream) {
    int grid = pod_ceil_div(n, 256);
    k_ort_values<<<grid, 256, 0, stream>>>(s, Y, n, ldy, st, mask, ort);
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}
