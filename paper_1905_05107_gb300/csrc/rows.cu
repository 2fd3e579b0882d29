// Row sampling of ISMA with rows = 1 (ICRS): Algorithm 1, GET UPDATE with
// rows, and SAMPLE AND SCALE UNIQUE ROWS; Sec. 3.1 row strategies.
//   q_i = |d^i|^2 over the sampled columns (L2), or |u^i|^2 over the first k
//         modes (leverage scores, rounds after the first);
//   w_i = floor(q_i / max q * 2^L), L = 62 - ceil(log2(m + 1)) (uniform if all 0);
//   w draws of Philox(j, t, 1, 0): smallest i with prefix_i > floor(u W / 2^64);
//   distinct rows I_r ascending with counts t_hat; row l of W is d^{I_r[l]}
//   scaled by sqrt(t_hat_l W / (w w_{I_r[l]}))  (q = w_i / W is the quantised
//   probability actually used).
// The m-length passes run on the whole GPU (block partials plus one-block
// scans of the partials); W^T W is formed straight from the gathered rows
// (k_row_gram) and its eigenvectors come from the small kernel k_rows_small.
#include "pod_internal.h"

namespace {

constexpr int RB = 1024;   // rows per block of the m-length passes

template <typename T>
__global__ void __launch_bounds__(RB) k_row_values(RowArgs<T> a) {
    const DevState *st = a.st;
    if (st->done) return;
    __shared__ double red[32];
    const int g = st->g, r = st->r_cur, t = st->t;
    const bool ls = a.row_strategy == POD_ROW_LS && t > 0 && r > 0;
    const int kk = r < a.k ? r : a.k;
    const int64_t i = (int64_t)blockIdx.x * RB + threadIdx.x;
    double v = 0.0;
    if (i < a.m) {
        if (ls) {
            for (int l = 0; l < kk; ++l) {
                const double x = (double)a.U[(int64_t)l * a.ldu + i];
                v += x * x;
            }
            v /= (double)kk;
        } else {
            for (int j = 0; j < g; ++j) {
                const double x = (double)a.A[(int64_t)a.idx[j] * a.lda + i];
                v += x * x;
            }
        }
        a.val[i] = v;
    }
    v = block_max<double>(v, red);
    if (threadIdx.x == 0) a.bmax[blockIdx.x] = v;
}

// weights and per-block sums (every block re-reduces the block maxima)
template <typename T>
__global__ void __launch_bounds__(RB) k_row_weights(RowArgs<T> a) {
    const DevState *st = a.st;
    if (st->done) return;
    __shared__ double redd[32];
    __shared__ unsigned long long red64[32];
    double vmax = 0.0;
    for (int b = threadIdx.x; b < a.nblocks; b += RB) vmax = a.bmax[b] > vmax ? a.bmax[b] : vmax;
    vmax = block_max<double>(vmax, redd);
    const int64_t i = (int64_t)blockIdx.x * RB + threadIdx.x;
    uint64_t w = 0;
    if (i < a.m) {
        if (vmax > 0.0) w = (uint64_t)floor(ldexp(a.val[i] / vmax, a.L));
        else w = 1;   // every weight zero: uniform over the rows
        a.w[i] = w;
    }
    const unsigned long long s = block_sum<unsigned long long>((unsigned long long)w, red64);
    if (threadIdx.x == 0) a.bsum[blockIdx.x] = s;
}

// one block: exclusive offsets of the block sums (and the total)
template <typename T>
__global__ void __launch_bounds__(RB) k_row_offsets(RowArgs<T> a, int write_total) {
    const DevState *st = a.st;
    if (st->done) return;
    __shared__ unsigned long long warp_tot[32];
    unsigned long long carry = 0;
    for (int base = 0; base < a.nblocks; base += RB) {
        const int b = base + threadIdx.x;
        unsigned long long v = b < a.nblocks ? a.bsum[b] : 0ull;
        // inclusive warp scan, then across warps
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        unsigned long long x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        __syncthreads();
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        if (wid == 0) {
            unsigned long long w = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warp_tot[lane] = w;
        }
        __syncthreads();
        const unsigned long long incl = x + (wid > 0 ? warp_tot[wid - 1] : 0ull);
        if (b < a.nblocks) a.boff[b] = carry + incl - v;
        const unsigned long long tot = warp_tot[31];
        __syncthreads();
        carry += tot;
    }
    if (threadIdx.x == 0 && write_total) a.total[0] = carry;
}

// inclusive prefix sums of the weights
template <typename T>
__global__ void __launch_bounds__(RB) k_row_cdf(RowArgs<T> a) {
    const DevState *st = a.st;
    if (st->done) return;
    __shared__ unsigned long long warp_tot[32];
    const int64_t i = (int64_t)blockIdx.x * RB + threadIdx.x;
    unsigned long long v = i < a.m ? a.w[i] : 0ull;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long w = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    if (i < a.m) a.cdf[i] = a.boff[blockIdx.x] + x + (wid > 0 ? warp_tot[wid - 1] : 0ull);
}

// w draws; counts per row
template <typename T>
__global__ void k_row_draws(RowArgs<T> a) {
    const DevState *st = a.st;
    if (st->done) return;
    const uint64_t total = a.total[0];
    const int t = st->t;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < a.wdraws; j += gridDim.x * blockDim.x) {
        const uint64_t u = philox_u64(a.seed, (uint32_t)j, (uint32_t)t, 1u);
        const uint64_t v = __umul64hi(u, total);
        int64_t lo = 0, hi = a.m - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (a.cdf[mid] > v) hi = mid; else lo = mid + 1;
        }
        atomicAdd(&a.cnt[lo], 1u);
    }
}

// per-block counts of drawn rows
template <typename T>
__global__ void __launch_bounds__(RB) k_row_nzcount(RowArgs<T> a) {
    const DevState *st = a.st;
    if (st->done) return;
    __shared__ unsigned long long red64[32];
    const int64_t i = (int64_t)blockIdx.x * RB + threadIdx.x;
    const unsigned long long f = (i < a.m && a.cnt[i] > 0) ? 1ull : 0ull;
    const unsigned long long s = block_sum<unsigned long long>(f, red64);
    if (threadIdx.x == 0) a.bsum[blockIdx.x] = s;
}

// distinct rows ascending with their counts and scales; clears the counts
template <typename T>
__global__ void __launch_bounds__(RB) k_row_compact(RowArgs<T> a) {
    const DevState *st = a.st;
    if (st->done) return;
    __shared__ int warp_tot[32];
    const int64_t i = (int64_t)blockIdx.x * RB + threadIdx.x;
    const unsigned c = i < a.m ? a.cnt[i] : 0u;
    const int f = c > 0 ? 1 : 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = f;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    if (f) {
        const int64_t pos = (int64_t)a.boff[blockIdx.x] + x - 1 + (wid > 0 ? warp_tot[wid - 1] : 0);
        a.rows[pos] = (int32_t)i;
        a.rcnt[pos] = (int32_t)c;
        // sqrt(t_hat * W / (w * w_i)) with q_i = w_i / W the quantised probability
        const double total = (double)a.total[0];
        a.rscale[pos] = sqrt((double)c * total / ((double)a.wdraws * (double)a.w[i]));
        a.cnt[i] = 0u;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        // number of distinct rows: offset of the last block + its count
        a.h[0] = (int32_t)(a.boff[blockIdx.x] + a.bsum[blockIdx.x]);
    }
}

// G_W = W^T W without materialising W: each CTA gathers its share of the h
// scaled rows (row l of W = d^{I_r[l]} * scale_l; with all_rows, W = D: all
// m rows, unit scale, for the literal truncation of the new block) into
// shared memory and
// forms its partial Gram; the partials are summed in a fixed order in FP64.
// FP32 data: the eigenvectors of a Gram formed in FP32 lose accuracy as
// sigma_1^2 / (sigma_r^2 - sigma_{r+1}^2), so every product is split exactly
// (TwoProduct) and summed with TwoSum into a (hi, lo) pair; FP64 data uses
// FP64 FMAs.  Upper triangle, ld cmax.
template <typename T>
__global__ void __launch_bounds__(256) k_row_gram(RowArgs<T> a) {
    const DevState *st = a.st;
    if (st->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Ws = reinterpret_cast<T *>(smem_raw);   // column j at j * lds
    __shared__ int s_flag;
    const int g = st->g;
    const int64_t h = a.all_rows ? a.m : (int64_t)a.h[0];
    const int rp = a.rows_per, lds = a.lds;
    const int64_t r0 = (int64_t)blockIdx.x * rp;
    const int nr = (int)max((int64_t)0, min((int64_t)rp, h - r0));
    if (a.all_rows) {
        for (int e = threadIdx.x; e < nr * g; e += blockDim.x) {
            const int j = e / nr, l = e - j * nr;
            Ws[j * lds + l] = a.A[(int64_t)a.idx[j] * a.lda + r0 + l];
        }
    } else {
        for (int e = threadIdx.x; e < nr * g; e += blockDim.x) {
            const int j = e / nr, l = e - j * nr;
            Ws[j * lds + l] = (T)((double)a.A[(int64_t)a.idx[j] * a.lda + a.rows[r0 + l]] * a.rscale[r0 + l]);
        }
    }
    __syncthreads();
    const int cm = a.cmax;
    double *out = a.part + (int64_t)blockIdx.x * cm * cm;
    for (int e = threadIdx.x; e < g * cm; e += blockDim.x) {
        const int p = e / cm, q = e - p * cm;
        double v = 0.0;
        if (q >= p && q < g) {
            const T *x = Ws + p * lds, *y = Ws + q * lds;
            if constexpr (sizeof(T) == 4) {
                dfloat acc{0.f, 0.f};
                for (int l = 0; l < nr; ++l) {
                    const float pr = x[l] * y[l];
                    const float er = fmaf(x[l], y[l], -pr);
                    const dfloat s = df_two_sum(acc.hi, pr);
                    acc.hi = s.hi;
                    acc.lo += s.lo + er;
                }
                v = (double)acc.hi + (double)acc.lo;
            } else {
                double acc = 0.0;
                for (int l = 0; l < nr; ++l) acc = fma(x[l], y[l], acc);
                v = acc;
            }
        }
        out[e] = v;
    }
    tall_reduce(a.part, a.gsum, a.GW, g * cm, (int64_t)cm * cm, a.gcounters, &s_flag);
}

}  // namespace

template <typename T>
pod_status launch_rows(const RowArgs<T> &a, cudaStream_t s, int sms) {
    const int nb = a.nblocks;
    k_row_values<T><<<nb, RB, 0, s>>>(a);
    k_row_weights<T><<<nb, RB, 0, s>>>(a);
    k_row_offsets<T><<<1, RB, 0, s>>>(a, 1);
    k_row_cdf<T><<<nb, RB, 0, s>>>(a);
    int dg = (a.wdraws + 255) / 256;
    if (dg > 4 * sms) dg = 4 * sms;
    if (dg < 1) dg = 1;
    k_row_draws<T><<<dg, 256, 0, s>>>(a);
    k_row_nzcount<T><<<nb, RB, 0, s>>>(a);
    k_row_offsets<T><<<1, RB, 0, s>>>(a, 0);
    k_row_compact<T><<<nb, RB, 0, s>>>(a);
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}

template <typename T>
pod_status launch_row_gram(const RowArgs<T> &a, cudaStream_t s) {
    const size_t smem = (size_t)a.lds * a.cmax * sizeof(T);
    POD_CUDA_TRY(cudaFuncSetAttribute(k_row_gram<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_row_gram<T><<<a.ggrid, 256, smem, s>>>(a);
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}

int row_blocks(int64_t m) { return (int)((m + RB - 1) / RB); }

RowGramPlan row_gram_plan(int dtype, int64_t wdraws, int cmax, int sms) {
    RowGramPlan p{};
    const size_t es = dtype == POD_F32 ? 4 : 8;
    const int max_rows = (int)((96 * 1024) / ((size_t)cmax * es)) - 1;   // shared-memory cap per CTA
    int64_t grid = 2 * sms;
    if ((wdraws + grid - 1) / grid > max_rows) grid = (wdraws + max_rows - 1) / max_rows;
    if (grid > (wdraws + 15) / 16) grid = (wdraws + 15) / 16;
    if (grid < 1) grid = 1;
    p.grid = (int)grid;
    p.rows_per = (int)((wdraws + grid - 1) / grid);
    p.lds = p.rows_per | 1;   // odd column stride: conflict-free shared loads across columns
    p.groups = (grid + RED_GROUP - 1) / RED_GROUP;
    return p;
}

template pod_status launch_rows<float>(const RowArgs<float> &, cudaStream_t, int);
template pod_status launch_rows<double>(const RowArgs<double> &, cudaStream_t, int);
template pod_status launch_row_gram<float>(const RowArgs<float> &, cudaStream_t);
template pod_status launch_row_gram<double>(const RowArgs<double> &, cudaStream_t);
