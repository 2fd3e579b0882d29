// Small dense algebra of BLOCK MERGE (Algorithm 2) and of the closing
// refinement of Algorithm 1, one CTA per problem:
//   * fixed-order sums of the tall passes' FP64 partials;
//   * CholeskyQR2 factors (Cholesky with pivot dropping, triangular inverses);
//   * the core E = [[Sigma_1, U_1^T C], [0, R]] (Eq. 8) and its SVD (Eq. 9);
//   * truncation to r and to the non-zero singular values, the convergence
//     measures of Algorithm 1, and the update coefficients X, Y with
//     U_new = U X + C Y.
// The FP64 storage path computes in FP64.  The FP32 path computes the
// triangular factors in double-float (X = dfloat), runs the one-sided Jacobi
// sweeps of the core in FP32, and finishes with a double-float Rayleigh step
// sigma_i = |E v_i| on the top-r right vectors plus a CholeskyQR of E V_r, so
// the singular values are second-order accurate in the FP32 rotation error.
#include "pod_internal.h"

namespace {

constexpr int SMALL_THREADS = 1024;

__device__ __forceinline__ double unit_roundoff(int dtype) {
    return dtype == POD_F32 ? 5.9604644775390625e-08 : 1.1102230246251565e-16;
}
__device__ __forceinline__ double round_to(int dtype, double v) {
    return dtype == POD_F32 ? (double)(float)v : v;
}

// ---------------------------------------------------------------------------
// In-place upper Cholesky with pivot dropping.  On entry the upper triangle
// of W (n x n, ld) holds a symmetric Gram matrix; on exit W holds R with
// R^T R = G on the kept indices.  A pivot d <= thr marks its index as
// numerically dependent: R's row is zero (Algorithm 2 drops the matching
// zero singular values of E).
// ---------------------------------------------------------------------------
template <typename X>
__device__ void chol_drop(X *W, int ld, int n, X thr, X *s_piv) {
    const int tid = threadIdx.x, bd = blockDim.x;
    for (int k = 0; k < n; ++k) {
        if (tid == 0) {
            X d = W[k * ld + k];
            *s_piv = x_gt(d, thr) ? XOps<X>::sqrt_(d) : XOps<X>::zero();
        }
        __syncthreads();
        const X piv = *s_piv;
        const bool keep = x_hi(piv) > 0.f;
        for (int j = k + tid; j < n; j += bd) {
            X v = XOps<X>::zero();
            if (keep) v = (j == k) ? piv : W[k * ld + j] / piv;
            W[k * ld + j] = v;
        }
        __syncthreads();
        if (keep) {
            const int w = n - k - 1;
            for (int e = tid; e < w * w; e += bd) {
                const int i = k + 1 + e / w, j = k + 1 + e % w;
                if (i <= j) W[i * ld + j] = W[i * ld + j] - W[k * ld + i] * W[k * ld + j];
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < n * n; e += bd) {
        const int i = e / n, j = e % n;
        if (i > j) W[i * ld + j] = XOps<X>::zero();
    }
    __syncthreads();
}

// M = R^{-1} for upper triangular R (zero rows of dropped indices give zero
// rows and columns of M).  Row-oriented back substitution: M starts as I.
template <typename X>
__device__ void tri_inv(const X *R, int ldr, int n, X *M, int ldm) {
    const int tid = threadIdx.x, bd = blockDim.x;
    for (int e = tid; e < n * n; e += bd) {
        const int i = e / n, j = e % n;
        M[i * ldm + j] = (i == j && x_hi(R[i * ldr + i]) != 0.f) ? XOps<X>::one() : XOps<X>::zero();
    }
    __syncthreads();
    for (int k = n - 1; k >= 0; --k) {
        const X d = R[k * ldr + k];
        if (x_hi(d) != 0.f) {
            for (int j = k + tid; j < n; j += bd) M[k * ldm + j] = M[k * ldm + j] / d;
            __syncthreads();
            for (int e = tid; e < k * (n - k); e += bd) {
                const int i = e / (n - k), j = k + e % (n - k);
                M[i * ldm + j] = M[i * ldm + j] - R[i * ldr + k] * M[k * ldm + j];
            }
        }
        __syncthreads();
    }
}

// A <- A B for upper triangular A, B (in place in A; columns descending).
template <typename X>
__device__ void trmm_inplace_left(X *A, int lda, const X *B, int ldb, int n) {
    const int tid = threadIdx.x, bd = blockDim.x;
    for (int j = n - 1; j >= 0; --j) {
        for (int i = tid; i <= j; i += bd) {
            X s = XOps<X>::zero();
            for (int l = i; l <= j; ++l) s = s + A[i * lda + l] * B[l * ldb + j];
            A[i * lda + j] = s;
        }
        __syncthreads();
    }
}

// B <- A B for upper triangular A, B (in place in B; rows ascending).
template <typename X>
__device__ void trmm_inplace_right(const X *A, int lda, X *B, int ldb, int n) {
    const int tid = threadIdx.x, bd = blockDim.x;
    for (int i = 0; i < n; ++i) {
        for (int j = i + tid; j < n; j += bd) {
            X s = XOps<X>::zero();
            for (int l = i; l <= j; ++l) s = s + A[i * lda + l] * B[l * ldb + j];
            B[i * ldb + j] = s;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// One-sided (Hestenes) Jacobi on the columns of B (nrow x ncol, column-major,
// ld ldb): rotate column pairs until every pair is orthogonal to tol
// (|b_p . b_q| <= tol |b_p| |b_q|).  Parallel ordering: round-robin
// tournament, one warp per pair, all pairs of a round disjoint.  Optionally
// accumulates the rotations into V (ncol x ncol, column-major, ld ldv).
// Bounded by max_sweeps.  Returns sweeps run.
// ---------------------------------------------------------------------------
template <typename J>
__device__ int jacobi_cols(J *B, int ldb, int nrow, int ncol, J *V, int ldv, J tol, int max_sweeps,
                           int *s_flag) {
    const int N = ncol + (ncol & 1);
    const int npairs = N / 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    int sweep = 0;
    if (ncol < 2) return 0;
    for (; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) *s_flag = 0;
        __syncthreads();
        for (int rnd = 0; rnd < N - 1; ++rnd) {
            for (int pr = warp; pr < npairs; pr += nw) {
                int p, q;
                if (pr == 0) {
                    p = N - 1;
                    q = rnd;
                } else {
                    p = (rnd + pr) % (N - 1);
                    q = (rnd - pr + N - 1) % (N - 1);
                }
                if (p >= ncol || q >= ncol) continue;
                if (p > q) { int tmp = p; p = q; q = tmp; }
                J *bp = B + (size_t)p * ldb, *bq = B + (size_t)q * ldb;
                J a = 0, b = 0, c = 0;
                for (int i = lane; i < nrow; i += 32) {
                    J x = bp[i], y = bq[i];
                    a = fma(x, x, a);
                    b = fma(y, y, b);
                    c = fma(x, y, c);
                }
                a = warp_sum(a);
                b = warp_sum(b);
                c = warp_sum(c);
                if (a > (J)0 && b > (J)0 && fabs(c) > tol * sqrt(a) * sqrt(b)) {
                    J zeta = (b - a) / (c + c);
                    J t;
                    if (fabs(zeta) > (J)1e15)
                        t = (J)0.5 / zeta;
                    else
                        t = (zeta >= (J)0 ? (J)1 : (J)-1) / (fabs(zeta) + sqrt((J)1 + zeta * zeta));
                    J cs = (J)1 / sqrt((J)1 + t * t), sn = cs * t;
                    for (int i = lane; i < nrow; i += 32) {
                        J x = bp[i], y = bq[i];
                        bp[i] = cs * x - sn * y;
                        bq[i] = sn * x + cs * y;
                    }
                    if (V) {
                        J *vp = V + (size_t)p * ldv, *vq = V + (size_t)q * ldv;
                        for (int i = lane; i < ncol; i += 32) {
                            J x = vp[i], y = vq[i];
                            vp[i] = cs * x - sn * y;
                            vq[i] = sn * x + cs * y;
                        }
                    }
                    if (lane == 0) *s_flag = 1;
                }
            }
            __syncthreads();
        }
        const int rotated = *s_flag;
        __syncthreads();
        if (!rotated) break;
    }
    return sweep;
}

// rank of each of n keys in descending order (ties by index) -> order[rank] = i
template <typename K>
__device__ void sort_desc(const K *key, int n, int *order) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const K ki = key[i];
        int rank = 0;
        for (int j = 0; j < n; ++j) {
            const K kj = key[j];
            rank += (x_gt(kj, ki) || (!x_gt(ki, kj) && !x_gt(kj, ki) && j < i)) ? 1 : 0;
        }
        order[rank] = i;
    }
    __syncthreads();
}

// bump allocator over dynamic shared memory
struct Carve {
    unsigned char *p;
    template <typename V>
    __device__ V *take(size_t count) {
        V *r = reinterpret_cast<V *>(p);
        p += ((count * sizeof(V) + 15) / 16) * 16;
        return r;
    }
};

}  // namespace

// ---------------------------------------------------------------------------
// Fixed-order sum of FP64 partials.
// ---------------------------------------------------------------------------
__global__ void k_reduce(const double *__restrict__ part, int nparts, int64_t stride, int64_t count,
                         double *__restrict__ out, const DevState *st) {
    if (st && st->done) return;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int p = 0; p < nparts; ++p) s += part[(int64_t)p * stride + e];
        out[e] = s;
    }
}

pod_status launch_reduce(const double *part, int nparts, int64_t stride, int64_t count, double *out,
                         const DevState *st, cudaStream_t s) {
    if (count <= 0) return POD_OK;
    int grid = pod_ceil_div(count, 256);
    if (grid > 1024) grid = 1024;
    k_reduce<<<grid, 256, 0, s>>>(part, nparts, stride, count, out, st);
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}

// ---------------------------------------------------------------------------
// First CholeskyQR pass: Ptot = fl(P) + fl(P2), R1 = chol(Z^T Z) with pivot
// dropping, M1 = fl(R1^{-1}) (the matrix the tall pass applies), and
// R1p = M1^{-1} (the exact inverse of what was applied, used in E).
// ---------------------------------------------------------------------------
template <typename X>
__global__ void __launch_bounds__(SMALL_THREADS) k_small_chol(SmallArgs a) {
    DevState *st = a.st;
    if (st->done) return;
    const int r = st->r_cur, g = st->g, nc = r + g;
    const int ld = a.cmax;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Carve cv{smem_raw};
    X *W = cv.take<X>((size_t)ld * ld);
    X *M = cv.take<X>((size_t)ld * ld);
    X *Q = cv.take<X>((size_t)ld * ld);
    __shared__ double red[32];
    __shared__ X s_piv;
    const int tid = threadIdx.x, bd = blockDim.x;
    const double *P2 = a.PG;
    const double *G = a.PG + (int64_t)a.rmax * a.cmax;

    double cmax2 = 0.0;
    for (int j = tid; j < g; j += bd) {
        double cn = G[j * ld + j];
        for (int l = 0; l < r; ++l) {
            double pt = round_to(a.dtype, a.P[l * ld + j]) + round_to(a.dtype, P2[l * ld + j]);
            a.Ptot[l * ld + j] = pt;
            cn += pt * pt;
        }
        cmax2 = cn > cmax2 ? cn : cmax2;
    }
    cmax2 = block_max<double>(cmax2, red);
    const double s0 = r > 0 ? a.sigma[0] : 0.0;
    const double scale = cmax2 > s0 * s0 ? cmax2 : s0 * s0;
    const double eps = nc * unit_roundoff(a.dtype);
    const X thr = XOps<X>::from(eps * eps * scale);

    for (int e = tid; e < g * g; e += bd) {
        const int i = e / g, j = e % g;
        W[i * ld + j] = XOps<X>::from(i <= j ? G[i * ld + j] : 0.0);
    }
    __syncthreads();
    chol_drop<X>(W, ld, g, thr, &s_piv);
    tri_inv<X>(W, ld, g, M, ld);
    // round M1 to the storage type: that is the matrix the QR2 pass applies
    for (int e = tid; e < g * g; e += bd) {
        const int i = e / g, j = e % g;
        double v = round_to(a.dtype, XOps<X>::to(M[i * ld + j]));
        a.M1[i * ld + j] = v;
        M[i * ld + j] = XOps<X>::from(v);
    }
    __syncthreads();
    tri_inv<X>(M, ld, g, Q, ld);
    for (int e = tid; e < g * g; e += bd) {
        const int i = e / g, j = e % g;
        a.R1p[i * ld + j] = XOps<X>::to(Q[i * ld + j]);
    }
}

size_t small_chol_smem(int cmax) { return 3 * (size_t)cmax * cmax * 8 + 64; }

pod_status launch_small_chol(const SmallArgs &a, cudaStream_t s) {
    const size_t smem = small_chol_smem(a.cmax);
    if (smem > 220 * 1024) return POD_EUNSUPPORTED;
    if (a.dtype == POD_F32) {
        POD_CUDA_TRY(cudaFuncSetAttribute(k_small_chol<dfloat>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_small_chol<dfloat><<<1, SMALL_THREADS, smem, s>>>(a);
    } else {
        POD_CUDA_TRY(cudaFuncSetAttribute(k_small_chol<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_small_chol<double><<<1, SMALL_THREADS, smem, s>>>(a);
    }
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}

// ---------------------------------------------------------------------------
// Second CholeskyQR pass, the core E and its SVD, truncation, convergence,
// and the update coefficients.
// ---------------------------------------------------------------------------
struct CoreLayout {
    size_t phaseA;   // 4 g x g X matrices
    size_t phaseB;   // Jacobi: B and V (J), keys, order
    size_t phaseC;   // finish
    size_t total;
};

__host__ __device__ inline size_t al16(size_t b) { return (b + 15) / 16 * 16; }

__host__ __device__ inline CoreLayout core_layout(int rmax, int cmax, int jsize) {
    CoreLayout L;
    const int nmax = rmax + cmax;
    L.phaseA = 4 * al16((size_t)cmax * cmax * 8);
    L.phaseB = 2 * al16((size_t)nmax * nmax * jsize) + al16((size_t)nmax * 8) + al16((size_t)nmax * 4);
    // Vh, Bd, UE: nmax x rmax X; Gb, Mb: rmax x rmax X; Bsin: nmax x rmax J; sig: rmax X
    L.phaseC = 3 * al16((size_t)nmax * rmax * 8) + 2 * al16((size_t)rmax * rmax * 8) +
               al16((size_t)nmax * rmax * jsize) + al16((size_t)rmax * 8) + al16((size_t)rmax * 4);
    const size_t bc = L.phaseB + L.phaseC;
    L.total = (L.phaseA > bc ? L.phaseA : bc) + 64;
    return L;
}

size_t core_smem_bytes(int rmax, int cmax, int dtype) {
    return core_layout(rmax, cmax, dtype == POD_F32 ? 4 : 8).total;
}

template <typename X, typename J>
__global__ void __launch_bounds__(SMALL_THREADS) k_core(SmallArgs a) {
    DevState *st = a.st;
    if (st->done) return;
    const int r = st->r_cur, g = st->g, nc = r + g, t = st->t;
    const int ld = a.cmax, nmax = a.rmax + a.cmax, lde = nmax;
    const int tid = threadIdx.x, bd = blockDim.x;
    const CoreLayout CL = core_layout(a.rmax, a.cmax, (int)sizeof(J));
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ X s_piv;
    __shared__ int s_flag;
    __shared__ double red[32];
    __shared__ int s_rnew;
    __shared__ double s_measure, s_sin, s_cos;
    __shared__ int s_bad;
    const double u = unit_roundoff(a.dtype);
    if (tid == 0) s_bad = 0;

    // ---- phase A: R2 = chol(G2), M2 = R2^{-1}, R = R2 R1p, Rinv = M1 M2
    {
        Carve cv{smem_raw};
        X *W = cv.take<X>((size_t)ld * ld);
        X *M2 = cv.take<X>((size_t)ld * ld);
        X *Rr = cv.take<X>((size_t)ld * ld);
        X *Mi = cv.take<X>((size_t)ld * ld);
        double dmax = 0.0;
        for (int j = tid; j < g; j += bd) dmax = a.G2[j * ld + j] > dmax ? a.G2[j * ld + j] : dmax;
        dmax = block_max<double>(dmax, red);
        const double eps = nc * u;
        const X thr = XOps<X>::from(eps * eps * dmax);
        for (int e = tid; e < g * g; e += bd) {
            const int i = e / g, j = e % g;
            W[i * ld + j] = XOps<X>::from(i <= j ? a.G2[i * ld + j] : 0.0);
            Rr[i * ld + j] = XOps<X>::from(a.R1p[i * ld + j]);
            Mi[i * ld + j] = XOps<X>::from(a.M1[i * ld + j]);
        }
        __syncthreads();
        chol_drop<X>(W, ld, g, thr, &s_piv);
        tri_inv<X>(W, ld, g, M2, ld);
        trmm_inplace_right<X>(W, ld, Rr, ld, g);     // Rr <- R2 R1p
        trmm_inplace_left<X>(Mi, ld, M2, ld, g);     // Mi <- M1 M2
        // E (column-major, ld lde) and Rinv (kept in Ym's scratch: the E buffer tail)
        double *Rinv = a.E + (size_t)lde * lde;
        for (int e = tid; e < nc * nc; e += bd) {
            const int q = e / nc, p = e % nc;   // column q, row p
            double v = 0.0;
            if (p < r) {
                if (q < r) v = (p == q) ? a.sigma[p] : 0.0;
                else v = a.Ptot[p * ld + (q - r)];
            } else if (q >= r) {
                v = XOps<X>::to(Rr[(p - r) * ld + (q - r)]);
            }
            if (!isfinite(v)) s_bad = 1;
            a.E[(size_t)q * lde + p] = v;
        }
        for (int e = tid; e < g * g; e += bd) {
            const int i = e / g, j = e % g;
            Rinv[i * ld + j] = XOps<X>::to(Mi[i * ld + j]);
        }
        __syncthreads();
    }

    // ---- phase B: Jacobi on the columns of E
    Carve cv{smem_raw};
    J *B = cv.take<J>((size_t)nmax * nmax);
    J *V = cv.take<J>((size_t)nmax * nmax);
    double *key = cv.take<double>(nmax);
    int *order = cv.take<int>(nmax);
    X *Vh = cv.take<X>((size_t)nmax * a.rmax);
    X *Bd = cv.take<X>((size_t)nmax * a.rmax);
    X *UE = cv.take<X>((size_t)nmax * a.rmax);
    X *Gb = cv.take<X>((size_t)a.rmax * a.rmax);
    X *Mb = cv.take<X>((size_t)a.rmax * a.rmax);
    J *Bs = cv.take<J>((size_t)nmax * a.rmax);
    X *sig = cv.take<X>(a.rmax);
    int *ord2 = cv.take<int>(a.rmax);
    const bool with_v = sizeof(J) == 4;
    for (int e = tid; e < nc * nc; e += bd) {
        const int q = e / nc, p = e % nc;
        B[q * nc + p] = (J)a.E[(size_t)q * lde + p];
        if (with_v) V[q * nc + p] = (p == q) ? (J)1 : (J)0;
    }
    __syncthreads();
    const J eps_j = sizeof(J) == 4 ? (J)1.1920928955078125e-07 : (J)2.220446049250313e-16;
    const J tol = (J)2 * sqrt((J)nc) * eps_j;
    jacobi_cols<J>(B, nc, nc, nc, with_v ? V : nullptr, nc, tol, sizeof(J) == 4 ? 20 : 30, &s_flag);
    for (int i = tid; i < nc; i += bd) {
        double s = 0.0;
        for (int p = 0; p < nc; ++p) s += (double)B[i * nc + p] * (double)B[i * nc + p];
        key[i] = s;
    }
    __syncthreads();
    sort_desc<double>(key, nc, order);
    const int rsel = a.r < nc ? a.r : nc;

    // ---- phase C: top-r left vectors and singular values
    if (with_v) {
        // v_s = normalised V[:, order[s]] (X); b_s = E v_s; sigma_s = |b_s|
        for (int s = tid >> 5; s < rsel; s += bd >> 5) {
            const int col = order[s];
            X nrm = XOps<X>::zero();
            for (int i = (tid & 31); i < nc; i += 32) {
                X v = XOps<X>::from((double)V[col * nc + i]);
                nrm = nrm + v * v;
            }
            // warp sum in X via shuffles of the two halves
            for (int o = 16; o > 0; o >>= 1) nrm = nrm + x_shfl_xor(nrm, o);
            nrm = XOps<X>::sqrt_(nrm);
            for (int i = (tid & 31); i < nc; i += 32)
                Vh[s * nc + i] = XOps<X>::from((double)V[col * nc + i]) / nrm;
        }
        __syncthreads();
        for (int e = tid; e < nc * rsel; e += bd) {
            const int s = e / nc, p = e % nc;
            X acc = XOps<X>::zero();
            for (int q = 0; q < nc; ++q) acc = acc + XOps<X>::from(a.E[(size_t)q * lde + p]) * Vh[s * nc + q];
            Bd[s * nc + p] = acc;
        }
        __syncthreads();
        for (int s = tid; s < rsel; s += bd) {
            X acc = XOps<X>::zero();
            for (int p = 0; p < nc; ++p) acc = acc + Bd[s * nc + p] * Bd[s * nc + p];
            sig[s] = XOps<X>::sqrt_(acc);
        }
        __syncthreads();
        sort_desc<X>(sig, rsel, ord2);
        // Gram of the re-ordered columns, CholeskyQR
        for (int e = tid; e < rsel * rsel; e += bd) {
            const int i = e / rsel, j = e % rsel;
            X acc = XOps<X>::zero();
            if (i <= j) {
                const X *bi = Bd + ord2[i] * nc, *bj = Bd + ord2[j] * nc;
                for (int p = 0; p < nc; ++p) acc = acc + bi[p] * bj[p];
            }
            Gb[i * a.rmax + j] = acc;
        }
        __syncthreads();
        {
            const double s0 = XOps<X>::to(sig[ord2[0]]);
            const double e2 = (nc * u) * (nc * u) * s0 * s0;
            chol_drop<X>(Gb, a.rmax, rsel, XOps<X>::from(e2), &s_piv);
        }
        tri_inv<X>(Gb, a.rmax, rsel, Mb, a.rmax);
        for (int e = tid; e < nc * rsel; e += bd) {
            const int s = e / nc, p = e % nc;
            X acc = XOps<X>::zero();
            for (int l = 0; l <= s; ++l) acc = acc + Bd[ord2[l] * nc + p] * Mb[l * a.rmax + s];
            UE[s * nc + p] = acc;
        }
        __syncthreads();
        // singular values in the new order (reuse Vh's first column as scratch)
        for (int s = tid; s < rsel; s += bd) Vh[s] = sig[ord2[s]];
        __syncthreads();
        for (int s = tid; s < rsel; s += bd) sig[s] = Vh[s];
        __syncthreads();
    } else {
        for (int e = tid; e < nc * rsel; e += bd) {
            const int s = e / nc, p = e % nc;
            const double nrm = sqrt(key[order[s]]);
            UE[s * nc + p] = XOps<X>::from(nrm > 0.0 ? (double)B[order[s] * nc + p] / nrm : 0.0);
        }
        for (int s = tid; s < rsel; s += bd) sig[s] = XOps<X>::from(sqrt(key[order[s]]));
        __syncthreads();
    }

    // truncation: keep min(r, #sigma > nc u sigma_1)
    if (tid == 0) {
        const double s0 = XOps<X>::to(sig[0]);
        const double thr = nc * u * s0;
        int keep = 0;
        for (int s = 0; s < rsel; ++s)
            if (XOps<X>::to(sig[s]) > thr) ++keep;
        if (!(s0 == s0) || !isfinite(s0)) s_bad = 1;
        s_rnew = keep;
        s_measure = 1.0;
        s_sin = 1.0;
        s_cos = 0.0;
    }
    __syncthreads();
    const int rn = s_rnew;

    // convergence measures between the previous and the merged top-k modes
    const int k = a.k;
    const bool comparable = t > 0 && r >= k && rn >= k;
    if (comparable) {
        const int nr = nc - k;
        if (a.criterion == POD_SUBSPACE) {
            for (int e = tid; e < nr * k; e += bd) {
                const int cidx = e / nr, p = e % nr;
                Bs[cidx * nr + p] = (J)XOps<X>::to(UE[cidx * nc + k + p]);
            }
            __syncthreads();
            jacobi_cols<J>(Bs, nr, nr, k, nullptr, 0, (J)2 * sqrt((J)(nr > 1 ? nr : 1)) * eps_j,
                           sizeof(J) == 4 ? 20 : 30, &s_flag);
            double mx = 0.0;
            for (int cidx = tid; cidx < k; cidx += bd) {
                double s = 0.0;
                for (int p = 0; p < nr; ++p) s += (double)Bs[cidx * nr + p] * (double)Bs[cidx * nr + p];
                mx = s > mx ? s : mx;
            }
            mx = block_max<double>(mx, red);
            if (tid == 0) {
                s_sin = sqrt(mx);
                s_measure = s_sin;
            }
        } else {
            double mn = 1e300;
            for (int i = tid; i < k; i += bd) {
                double c = fabs(XOps<X>::to(UE[i * nc + i]));
                mn = c < mn ? c : mn;
            }
            mn = -block_max<double>(-mn, red);
            if (tid == 0) {
                s_cos = mn;
                s_measure = 1.0 - mn;
            }
        }
        __syncthreads();
    }

    // Y = Rinv U_E[r:, :rn] (g x rn), X = U_E[:r, :rn] - Ptot Y (r x rn)
    {
        const double *Rinv = a.E + (size_t)lde * lde;
        for (int e = tid; e < g * rn; e += bd) {
            const int j = e / rn, q = e % rn;
            X acc = XOps<X>::zero();
            for (int l = j; l < g; ++l) acc = acc + XOps<X>::from(Rinv[j * ld + l]) * UE[q * nc + r + l];
            Bd[j * a.rmax + q] = acc;   // Bd reused as Y (g x rn, ld rmax)
        }
        __syncthreads();
        for (int e = tid; e < g * rn; e += bd) {
            const int j = e / rn, q = e % rn;
            a.Ym[j * a.rmax + q] = XOps<X>::to(Bd[j * a.rmax + q]);
        }
        for (int e = tid; e < r * rn; e += bd) {
            const int l = e / rn, q = e % rn;
            X acc = UE[q * nc + l];
            for (int j = 0; j < g; ++j) acc = acc - XOps<X>::from(a.Ptot[l * ld + j]) * Bd[j * a.rmax + q];
            a.Xm[l * a.rmax + q] = XOps<X>::to(acc);
        }
        for (int s = tid; s < rn; s += bd) a.sigma[s] = XOps<X>::to(sig[s]);
    }
    __syncthreads();
    if (tid == 0) {
        st->r_new = rn;
        st->measure = s_measure;
        st->sin_max = s_sin;
        st->cos_min = s_cos;
        if (a.hist_measure) a.hist_measure[t] = s_measure;
        bool converged = false;
        if (comparable) {
            if (a.criterion == POD_SUBSPACE) converged = s_sin <= a.tol;
            else converged = s_cos >= a.tol;
        }
        int dn = converged || st->remaining == 0 || (a.max_iter > 0 && t >= a.max_iter);
        if (s_bad) {
            st->status = POD_ENAN;
            dn = 1;
        }
        st->done_next = dn;
    }
}

pod_status launch_core(const SmallArgs &a, cudaStream_t s) {
    const size_t smem = core_smem_bytes(a.rmax, a.cmax, a.core_f64 ? POD_F64 : POD_F32);
    if (smem > 220 * 1024) return POD_EUNSUPPORTED;
    if (a.dtype == POD_F32 && !a.core_f64) {
        POD_CUDA_TRY(cudaFuncSetAttribute(k_core<dfloat, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_core<dfloat, float><<<1, SMALL_THREADS, smem, s>>>(a);
    } else {
        POD_CUDA_TRY(cudaFuncSetAttribute(k_core<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_core<double, double><<<1, SMALL_THREADS, smem, s>>>(a);
    }
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}

// ---------------------------------------------------------------------------
// End of a round: r_cur <- r_new, t <- t + 1, apply the stop decision.
// ---------------------------------------------------------------------------
__global__ void k_finish(DevState *st) {
    if (threadIdx.x != 0 || st->done) return;
    st->r_cur = st->r_new;
    st->t += 1;
    st->rounds_run += 1;
    if (st->done_next) st->done = 1;
}

pod_status launch_finish(DevState *st, cudaStream_t s);
pod_status launch_finish(DevState *st, cudaStream_t s) {
    k_finish<<<1, 32, 0, s>>>(st);
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}

// ---------------------------------------------------------------------------
// Refinement (closing lines of Algorithm 1): with Y = A^T U (n x r),
// CholeskyQR2 gives Y = Q R; SVD(R) = U_R S_R V_R^T by one-sided Jacobi in
// FP64 with accumulated V_R; outputs sigma = S_R, VR (U <- U V_R) and
// K = R^{-1} U_R (V <- Y K = Q U_R).  r <= 128, one CTA.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(SMALL_THREADS) k_refine_chol(RefineArgs a) {
    const int r = a.r;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Carve cv{smem_raw};
    double *W = cv.take<double>((size_t)r * r);
    double *M = cv.take<double>((size_t)r * r);
    __shared__ double s_piv;
    __shared__ double red[32];
    const int tid = threadIdx.x, bd = blockDim.x;
    double dmax = 0.0;
    for (int j = tid; j < r; j += bd) dmax = a.G[j * r + j] > dmax ? a.G[j * r + j] : dmax;
    dmax = block_max<double>(dmax, red);
    for (int e = tid; e < r * r; e += bd) {
        const int i = e / r, j = e % r;
        W[e] = i <= j ? a.G[i * r + j] : 0.0;
    }
    __syncthreads();
    const double eps = r * 1.1102230246251565e-16;
    chol_drop<double>(W, r, r, eps * eps * dmax, &s_piv);
    tri_inv<double>(W, r, r, M, r);
    for (int e = tid; e < r * r; e += bd) {
        a.M1[e] = M[e];
        a.R1p[e] = W[e];
    }
}

__global__ void __launch_bounds__(SMALL_THREADS) k_refine_svd(RefineArgs a) {
    const int r = a.r;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Carve cv{smem_raw};
    double *W = cv.take<double>((size_t)r * r);   // R2 -> R (row-major upper)
    double *M2 = cv.take<double>((size_t)r * r);
    double *B = cv.take<double>((size_t)r * r);   // column-major copy of R for Jacobi
    double *V = cv.take<double>((size_t)r * r);
    double *key = cv.take<double>(r);
    int *order = cv.take<int>(r);
    double *R1 = cv.take<double>((size_t)r * r);
    __shared__ double s_piv;
    __shared__ int s_flag;
    __shared__ double red[32];
    const int tid = threadIdx.x, bd = blockDim.x;
    double dmax = 0.0;
    for (int j = tid; j < r; j += bd) dmax = a.G2[j * r + j] > dmax ? a.G2[j * r + j] : dmax;
    dmax = block_max<double>(dmax, red);
    for (int e = tid; e < r * r; e += bd) {
        const int i = e / r, j = e % r;
        W[e] = i <= j ? a.G2[i * r + j] : 0.0;
        R1[e] = a.R1p[e];
    }
    __syncthreads();
    const double eps = r * 1.1102230246251565e-16;
    chol_drop<double>(W, r, r, eps * eps * dmax, &s_piv);
    tri_inv<double>(W, r, r, M2, r);
    trmm_inplace_right<double>(W, r, R1, r, r);   // R1 <- R2 R1  (= R)
    // Rinv = M1 M2 -> M2 (in place on the left factor copy)
    double *Mi = W;   // reuse
    for (int e = tid; e < r * r; e += bd) Mi[e] = a.M1[e];
    __syncthreads();
    trmm_inplace_left<double>(Mi, r, M2, r, r);   // Mi <- M1 M2 (= R^{-1})
    for (int e = tid; e < r * r; e += bd) {
        const int q = e / r, p = e % r;   // B column-major: column q
        B[q * r + p] = R1[p * r + q];
        V[q * r + p] = (p == q) ? 1.0 : 0.0;
    }
    __syncthreads();
    jacobi_cols<double>(B, r, r, r, V, r, 2.0 * sqrt((double)r) * 2.220446049250313e-16, 40, &s_flag);
    for (int i = tid; i < r; i += bd) {
        double s = 0.0;
        for (int p = 0; p < r; ++p) s += B[i * r + p] * B[i * r + p];
        key[i] = s;
    }
    __syncthreads();
    sort_desc<double>(key, r, order);
    // sigma_s, V_R[:, s], U_R[:, s] = B[:, order[s]] / sigma_s, K = Rinv U_R
    for (int s = tid; s < r; s += bd) a.sigma[s] = sqrt(key[order[s]]);
    for (int e = tid; e < r * r; e += bd) {
        const int l = e / r, s = e % r;
        a.VR[l * r + s] = V[order[s] * r + l];
    }
    for (int e = tid; e < r * r; e += bd) {
        const int j = e / r, s = e % r;
        const double sg = sqrt(key[order[s]]);
        double acc = 0.0;
        if (sg > 0.0)
            for (int l = j; l < r; ++l) acc += Mi[j * r + l] * B[order[s] * r + l] / sg;
        a.K[j * r + s] = acc;
    }
}

pod_status launch_refine_chol(const RefineArgs &a, cudaStream_t s) {
    const size_t smem = 2 * al16((size_t)a.r * a.r * 8) + 64;
    POD_CUDA_TRY(cudaFuncSetAttribute(k_refine_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_refine_chol<<<1, SMALL_THREADS, smem, s>>>(a);
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}

pod_status launch_refine_svd(const RefineArgs &a, cudaStream_t s) {
    const size_t smem = 5 * al16((size_t)a.r * a.r * 8) + al16((size_t)a.r * 8) + al16((size_t)a.r * 4) + 64;
    if (smem > 220 * 1024) return POD_EUNSUPPORTED;
    POD_CUDA_TRY(cudaFuncSetAttribute(k_refine_svd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_refine_svd<<<1, SMALL_THREADS, smem, s>>>(a);
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}
