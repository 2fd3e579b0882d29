// Tall-skinny passes of BLOCK MERGE (Algorithm 2) over the m rows:
//   TALL_PROJ   : P  = U^T C                              (U_1^T U_2, Eq. 8)
//   TALL_CGS    : Z  = C - U P;  P2 = U^T Z;  G = Z^T Z    (U_t, second projection)
//   TALL_QR2    : W  = (C - U P - U P2) M1;  G2 = W^T W     (second CholeskyQR pass)
//   TALL_UPDATE : U <- U X + C Y                          (U = [U_1 U_o] U_E, truncated)
// plus Y = A^T U (closing refinement of Algorithm 1, ORT probabilities) and
// the sign-reference dots.
//
// Every CTA walks row slabs of `bm` rows (grid-stride), stages the slab of U
// and of the gathered columns of C in shared memory (row-major, so one row of
// a slab is contiguous), and accumulates the small products with 4x4
// register tiles.  FP32 data: the per-slab tile sums are FP32 and are flushed
// into FP64 accumulators after every slab; the CTA's FP64 partial is written
// to `part`, and a separate kernel sums the partials in a fixed order, so
// results are bit-for-bit reproducible.
#include "pod_internal.h"

namespace {

__host__ __device__ inline int round4(int x) { return (x + 3) & ~3; }

template <typename T>
__device__ __forceinline__ void ld4(const T *p, T (&v)[4]) {
    if constexpr (sizeof(T) == 4) {
        float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
        double2 a = *reinterpret_cast<const double2 *>(p);
        double2 b = *reinterpret_cast<const double2 *>(p + 2);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
}

// Stage rows [i0, i0 + bm) of `ncols` columns into dst (row-major, ld),
// zero-filling rows >= rows and columns ncols..round4(ncols)-1.
template <typename T, typename ColFn>
__device__ void load_slab(T *dst, int ld, int ncols, int bm, int rows, int64_t i0, ColFn col) {
    const int nc4 = round4(ncols);
    for (int e = threadIdx.x; e < nc4 * bm; e += blockDim.x) {
        const int c = e / bm, i = e - c * bm;
        T v = (T)0;
        if (c < ncols && i < rows) v = col(c)[i0 + i];
        dst[i * ld + c] = v;
    }
}

// acc[p][q] += sum_{i < rows} X[i][p] Y[i][q] for p < na, q < nb (4x4 tiles;
// tiles with ti > tj are skipped when sym).  acc is FP64 (ld ldacc), red is
// scratch of blockDim.x * 16 T.  Ends with __syncthreads.
template <typename T>
__device__ void acc_xty(const T *X, int ldx, int na, const T *Y, int ldy, int nb, int rows, bool sym,
                        double *acc, int ldacc, T *red) {
    const int bd = blockDim.x, tid = threadIdx.x;
    const int ta = (na + 3) >> 2, tb = (nb + 3) >> 2;
    const int nT = ta * tb;
    if (nT == 0 || rows <= 0) return;
    if (nT * 2 > bd) {
        for (int tile = tid; tile < nT; tile += bd) {
            const int ti = tile / tb, tj = tile - ti * tb;
            if (sym && ti > tj) continue;
            T a[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) a[e] = (T)0;
            for (int i = 0; i < rows; ++i) {
                T x[4], y[4];
                ld4(X + i * ldx + 4 * ti, x);
                ld4(Y + i * ldy + 4 * tj, y);
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) a[u * 4 + v] = fma(x[u], y[v], a[u * 4 + v]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[(4 * ti + u) * ldacc + 4 * tj + v] += (double)a[u * 4 + v];
        }
        __syncthreads();
        return;
    }
    const int RG = bd / nT;
    const int tile = tid % nT, grp = tid / nT;
    const int ti = tile / tb, tj = tile - ti * tb;
    T a[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) a[e] = (T)0;
    if (grp < RG && !(sym && ti > tj)) {
        for (int i = grp; i < rows; i += RG) {
            T x[4], y[4];
            ld4(X + i * ldx + 4 * ti, x);
            ld4(Y + i * ldy + 4 * tj, y);
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) a[u * 4 + v] = fma(x[u], y[v], a[u * 4 + v]);
        }
    }
    if (grp < RG) {
#pragma unroll
        for (int e = 0; e < 16; ++e) red[(grp * nT + tile) * 16 + e] = a[e];
    }
    __syncthreads();
    for (int e = tid; e < nT * 16; e += bd) {
        const int t2 = e >> 4, uv = e & 15;
        const int i2 = t2 / tb, j2 = t2 - i2 * tb;
        if (sym && i2 > j2) continue;
        T s = (T)0;
        for (int g2 = 0; g2 < RG; ++g2) s += red[(g2 * nT + t2) * 16 + uv];
        acc[(4 * i2 + (uv >> 2)) * ldacc + 4 * j2 + (uv & 3)] += (double)s;
    }
    __syncthreads();
}

struct Layout {
    int ldu, ldc;       // smem leading dims of the U and C slabs
    int r4, c4;
};

__device__ __forceinline__ Layout layout_of(int rmax, int cmax) {
    Layout L;
    L.r4 = round4(rmax);
    L.c4 = round4(cmax);
    L.ldu = L.r4 + 4;
    L.ldc = L.c4 + 4;
    return L;
}

template <typename T>
__global__ void __launch_bounds__(256) k_tall(int kind, TallArgs<T> a) {
    const DevState *st = a.st;
    if (st->done) return;
    const int r = st->r_cur, g = st->g, rn = st->r_new;
    const Layout L = layout_of(a.rmax, a.cmax);
    const int bm = a.bm;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Us = reinterpret_cast<T *>(smem_raw);                 // bm x ldu
    T *Cs = Us + (size_t)bm * L.ldu;                         // bm x ldc
    T *Ws = Cs + (size_t)bm * L.ldc;                         // bm x max(ldc, ldu)
    const int ldw = L.ldc > L.ldu ? L.ldc : L.ldu;
    const size_t sq = (size_t)(L.r4 + L.c4) * (L.r4 + L.c4);
    T *S1 = Ws + (size_t)bm * ldw;                           // small operand 1
    T *S2 = S1 + sq;                                         // small operand 2
    T *S3 = S2 + sq;                                         // small operand 3 (c4 x c4)
    double *acc1 = reinterpret_cast<double *>(S3 + (size_t)L.c4 * L.c4);
    double *acc2 = acc1 + (size_t)L.r4 * L.c4;
    T *red = reinterpret_cast<T *>(acc2 + (size_t)L.c4 * L.c4);

    const int tid = threadIdx.x, bd = blockDim.x;
    auto ucol = [&](int l) { return a.U + (int64_t)l * a.ldu; };
    auto ccol = [&](int j) { return a.A + (int64_t)(a.idx ? a.idx[j] : j) * a.lda; };

    // small operands -> shared (as T); accumulators -> 0
    if (kind == TALL_CGS || kind == TALL_QR2) {
        for (int e = tid; e < L.r4 * L.c4; e += bd) {
            const int l = e / L.c4, j = e - l * L.c4;
            S1[e] = (l < r && j < g) ? (T)a.P[l * a.cmax + j] : (T)0;
            if (kind == TALL_QR2) S2[e] = (l < r && j < g) ? (T)a.P2[l * a.cmax + j] : (T)0;
        }
    }
    if (kind == TALL_QR2) {
        for (int e = tid; e < L.c4 * L.c4; e += bd) {
            const int l = e / L.c4, j = e - l * L.c4;
            S3[e] = (l < g && j < g && l <= j) ? (T)a.M1[l * a.cmax + j] : (T)0;
        }
    }
    if (kind == TALL_UPDATE) {
        // X: r x rn (ld r4), Y: g x rn (ld r4)
        for (int e = tid; e < L.r4 * L.r4; e += bd) {
            const int l = e / L.r4, q = e - l * L.r4;
            S1[e] = (l < r && q < rn) ? (T)a.Xm[l * a.rmax + q] : (T)0;
        }
        for (int e = tid; e < L.c4 * L.r4; e += bd) {
            const int j = e / L.r4, q = e - j * L.r4;
            S2[e] = (j < g && q < rn) ? (T)a.Ym[j * a.rmax + q] : (T)0;
        }
    }
    if (kind != TALL_UPDATE) {
        for (int e = tid; e < L.r4 * L.c4; e += bd) acc1[e] = 0.0;
        for (int e = tid; e < L.c4 * L.c4; e += bd) acc2[e] = 0.0;
    }
    __syncthreads();

    for (int64_t i0 = (int64_t)blockIdx.x * bm; i0 < a.m; i0 += (int64_t)gridDim.x * bm) {
        const int rows = (int)((a.m - i0) < bm ? (a.m - i0) : bm);
        load_slab<T>(Us, L.ldu, r, bm, rows, i0, ucol);
        if (kind != TALL_UPDATE || g > 0) load_slab<T>(Cs, L.ldc, g, bm, rows, i0, ccol);
        __syncthreads();
        if (kind == TALL_PROJ) {
            acc_xty<T>(Us, L.ldu, r, Cs, L.ldc, g, rows, false, acc1, L.c4, red);
        } else if (kind == TALL_CGS || kind == TALL_QR2) {
            // Z = C - U P  (then - U P2 for the QR2 pass), in place in Cs
            if (r > 0) {
                for (int e = tid; e < rows * g; e += bd) {
                    const int i = e / g, j = e - i * g;
                    T z = Cs[i * L.ldc + j];
                    for (int l = 0; l < r; ++l) z = fma(-Us[i * L.ldu + l], S1[l * L.c4 + j], z);
                    if (kind == TALL_QR2) {
                        T z2 = (T)0;
                        for (int l = 0; l < r; ++l) z2 = fma(Us[i * L.ldu + l], S2[l * L.c4 + j], z2);
                        z -= z2;
                    }
                    Cs[i * L.ldc + j] = z;
                }
                __syncthreads();
            }
            if (kind == TALL_CGS) {
                if (r > 0) acc_xty<T>(Us, L.ldu, r, Cs, L.ldc, g, rows, false, acc1, L.c4, red);
                acc_xty<T>(Cs, L.ldc, g, Cs, L.ldc, g, rows, true, acc2, L.c4, red);
            } else {
                // W = Z M1 (M1 upper triangular)
                for (int e = tid; e < rows * g; e += bd) {
                    const int i = e / g, j = e - i * g;
                    T w = (T)0;
                    for (int l = 0; l <= j; ++l) w = fma(Cs[i * L.ldc + l], S3[l * L.c4 + j], w);
                    Ws[i * L.ldc + j] = w;
                }
                for (int e = tid; e < rows * (L.c4 - g); e += bd) {
                    const int i = e / (L.c4 - g), j = g + (e - i * (L.c4 - g));
                    Ws[i * L.ldc + j] = (T)0;
                }
                __syncthreads();
                acc_xty<T>(Ws, L.ldc, g, Ws, L.ldc, g, rows, true, acc2, L.c4, red);
            }
        } else {
            // U_new rows = U X + C Y  -> Ws (bm x ldu), then coalesced write-back
            for (int e = tid; e < rows * rn; e += bd) {
                const int i = e / rn, q = e - i * rn;
                T u = (T)0;
                for (int l = 0; l < r; ++l) u = fma(Us[i * L.ldu + l], S1[l * L.r4 + q], u);
                for (int j = 0; j < g; ++j) u = fma(Cs[i * L.ldc + j], S2[j * L.r4 + q], u);
                Ws[i * L.ldu + q] = u;
            }
            __syncthreads();
            for (int e = tid; e < rows * rn; e += bd) {
                const int q = e / rows, i = e - q * rows;
                a.U[(int64_t)q * a.ldu + i0 + i] = Ws[i * L.ldu + q];
            }
            __syncthreads();
        }
    }
    if (kind == TALL_UPDATE) return;
    // write this CTA's FP64 partial
    double *out = a.part + (int64_t)blockIdx.x * a.part_stride;
    if (kind == TALL_PROJ) {
        for (int e = tid; e < r * g; e += bd) {
            const int l = e / g, j = e - l * g;
            out[l * a.cmax + j] = acc1[l * L.c4 + j];
        }
    } else if (kind == TALL_CGS) {
        for (int e = tid; e < r * g; e += bd) {
            const int l = e / g, j = e - l * g;
            out[l * a.cmax + j] = acc1[l * L.c4 + j];
        }
        double *outG = out + (int64_t)a.rmax * a.cmax;
        for (int e = tid; e < g * g; e += bd) {
            const int p = e / g, q = e - p * g;
            if (p <= q) outG[p * a.cmax + q] = acc2[p * L.c4 + q];
        }
    } else {
        for (int e = tid; e < g * g; e += bd) {
            const int p = e / g, q = e - p * g;
            if (p <= q) out[p * a.cmax + q] = acc2[p * L.c4 + q];
        }
    }
}

// ---------------------------------------------------------------------------
// Y = A^T U.  CTA (blockIdx.x, blockIdx.y) owns nb columns of A and a range
// of rows; writes its FP64 partial of the nb x r block of Y.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_atu(AtuArgs<T> a, int nb, int bm) {
    const DevState *st = a.st;
    if (st->done) return;
    const int r = st->r_cur;
    const int64_t j0 = (int64_t)blockIdx.x * nb;
    const int ncols = (int)((a.n - j0) < nb ? (a.n - j0) : nb);
    const int split = gridDim.y;
    const int64_t rows_per = ((a.m + split - 1) / split + bm - 1) / bm * bm;
    const int64_t ib = (int64_t)blockIdx.y * rows_per;
    const int64_t ie = (ib + rows_per) < a.m ? (ib + rows_per) : a.m;
    const int nb4 = round4(nb), r4 = round4(r);
    const int ldas = nb4 + 4, ldus = r4 + 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *As = reinterpret_cast<T *>(smem_raw);
    T *Us = As + (size_t)bm * ldas;
    double *acc = reinterpret_cast<double *>(Us + (size_t)bm * ldus);
    T *red = reinterpret_cast<T *>(acc + (size_t)nb4 * r4);
    const int tid = threadIdx.x, bd = blockDim.x;
    for (int e = tid; e < nb4 * r4; e += bd) acc[e] = 0.0;
    bool any = true;
    if (a.mask) {
        any = false;
        for (int c = 0; c < ncols; ++c) any |= a.mask[j0 + c] != 0;
    }
    __syncthreads();
    if (any && r > 0) {
        auto acol = [&](int c) {
            const bool live = !a.mask || a.mask[j0 + c];
            return live ? a.A + (j0 + c) * a.lda : (const T *)nullptr;
        };
        auto ucol = [&](int l) { return a.U + (int64_t)l * a.ldu; };
        for (int64_t i0 = ib; i0 < ie; i0 += bm) {
            const int rows = (int)((ie - i0) < bm ? (ie - i0) : bm);
            // A slab: masked-out columns are zero and not read
            for (int e = tid; e < nb4 * bm; e += bd) {
                const int c = e / bm, i = e - c * bm;
                T v = (T)0;
                if (c < ncols && i < rows) {
                    const T *p = acol(c);
                    if (p) v = p[i0 + i];
                }
                As[i * ldas + c] = v;
            }
            load_slab<T>(Us, ldus, r, bm, rows, i0, ucol);
            __syncthreads();
            acc_xty<T>(As, ldas, ncols, Us, ldus, r, rows, false, acc, r4, red);
        }
    }
    double *out = a.part + (int64_t)blockIdx.y * a.n * a.rmax;
    for (int e = tid; e < ncols * r; e += bd) {
        const int l = e / ncols, c = e - l * ncols;
        out[(int64_t)l * a.n + j0 + c] = acc[c * r4 + l];
    }
}

// sign-reference dots: d_l = sum_i U_il z_i
template <typename T>
__global__ void __launch_bounds__(256) k_sign_dots(const T *U, int64_t m, int64_t ldu, int r,
                                                   uint64_t seed, double *part) {
    __shared__ double red[32];
    for (int l = 0; l < r; ++l) {
        double acc = 0.0;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
             i += (int64_t)gridDim.x * blockDim.x) {
            uint4 x = philox4x32_10(make_uint4((uint32_t)i, 0u, 3u, 0u),
                                    make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
            double z = (double)(int32_t)x.x * (1.0 / 2147483648.0);
            acc += (double)U[(int64_t)l * ldu + i] * z;
        }
        acc = block_sum<double>(acc, red);
        if (threadIdx.x == 0) part[(int64_t)blockIdx.x * r + l] = acc;
    }
}

}  // namespace

TallPlan tall_plan(int dtype, int64_t m, int rmax, int cmax, int num_sms) {
    TallPlan p;
    const size_t es = dtype == POD_F32 ? 4 : 8;
    const int r4 = round4(rmax), c4 = round4(cmax);
    const int ldu = r4 + 4, ldc = c4 + 4;
    const int ldw = ldc > ldu ? ldc : ldu;
    const size_t small_t = (size_t)(r4 + c4) * (r4 + c4) * 2 + (size_t)c4 * c4;
    const size_t accs = ((size_t)r4 * c4 + (size_t)c4 * c4) * 8;
    const size_t red = 256 * 16 * es;
    // two CTAs per SM when the slab allows it
    int bm = 128;
    for (; bm > 16; bm >>= 1) {
        size_t tot = (size_t)bm * (ldu + ldc + (size_t)ldw) * es + small_t * es + accs + red;
        if (tot <= 110 * 1024) break;
    }
    p.bm = bm;
    const size_t base = (size_t)bm * (ldu + ldc + (size_t)ldw) * es + small_t * es + accs + red;
    for (int k = 0; k < 4; ++k) p.smem[k] = base;
    const int64_t slabs = (m + bm - 1) / bm;
    int64_t grid = 2 * (int64_t)num_sms;
    if (grid > slabs) grid = slabs;
    if (grid < 1) grid = 1;
    p.grid = (int)grid;
    return p;
}

template <typename T>
pod_status launch_tall(TallKind kind, const TallArgs<T> &a, const TallPlan &plan, cudaStream_t st) {
    const size_t smem = plan.smem[kind];
    POD_CUDA_TRY(cudaFuncSetAttribute(k_tall<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_tall<T><<<plan.grid, 256, smem, st>>>((int)kind, a);
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}

AtuPlan atu_plan(int dtype, int64_t m, int64_t n, int rmax, int num_sms) {
    AtuPlan p;
    const size_t es = dtype == POD_F32 ? 4 : 8;
    p.nb = 32;
    p.bm = 128;
    const int nb4 = round4(p.nb), r4 = round4(rmax);
    for (;;) {
        p.smem = (size_t)p.bm * ((nb4 + 4) + (r4 + 4)) * es + (size_t)nb4 * r4 * 8 + 256 * 16 * es;
        if (p.smem <= 200 * 1024 || p.bm <= 16) break;
        p.bm >>= 1;
    }
    const int64_t cb = (n + p.nb - 1) / p.nb;
    int64_t split = (2 * (int64_t)num_sms + cb - 1) / cb;
    const int64_t max_split = (m + p.bm - 1) / p.bm;
    if (split > max_split) split = max_split;
    if (split < 1) split = 1;
    if (split > 64) split = 64;
    p.split = (int)split;
    p.grid = dim3((unsigned)cb, (unsigned)split, 1);
    return p;
}

template <typename T>
pod_status launch_atu(const AtuArgs<T> &a, const AtuPlan &plan, cudaStream_t st) {
    POD_CUDA_TRY(cudaFuncSetAttribute(k_atu<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem));
    k_atu<T><<<plan.grid, 256, plan.smem, st>>>(a, plan.nb, plan.bm);
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}

template <typename T>
pod_status launch_sign_dots(const T *U, int64_t m, int64_t ldu, int r, uint64_t seed, double *part,
                            int grid, cudaStream_t st) {
    k_sign_dots<T><<<grid, 256, 0, st>>>(U, m, ldu, r, seed, part);
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}

template pod_status launch_tall<float>(TallKind, const TallArgs<float> &, const TallPlan &, cudaStream_t);
template pod_status launch_tall<double>(TallKind, const TallArgs<double> &, const TallPlan &, cudaStream_t);
template pod_status launch_atu<float>(const AtuArgs<float> &, const AtuPlan &, cudaStream_t);
template pod_status launch_atu<double>(const AtuArgs<double> &, const AtuPlan &, cudaStream_t);
template pod_status launch_sign_dots<float>(const float *, int64_t, int64_t, int, uint64_t, double *, int, cudaStream_t);
template pod_status launch_sign_dots<double>(const double *, int64_t, int64_t, int, uint64_t, double *, int, cudaStream_t);
