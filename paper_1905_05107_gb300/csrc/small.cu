// Small dense algebra of BLOCK MERGE (Algorithm 2) and of the closing
// refinement of Algorithm 1, one CTA per problem:
//   * fixed-order sums of the tall passes' FP64 partials;
//   * CholeskyQR2 factors (Cholesky with pivot dropping, triangular inverses);
//   * the core E = [[Sigma_1, U_1^T C], [0, R]] (Eq. 8) and its SVD (Eq. 9);
//   * truncation to r and to the non-zero singular values, the convergence
//     measures of Algorithm 1, and the update coefficients X, Y with
//     U_new = U X + W Y (W = Z M1 stored by the QR2 pass), or U X + C Y
//     for the row-block stage of ICRS.
// The FP64 storage path computes in FP64.  The FP32 path computes the
// triangular factors in double-float (X = dfloat), runs the one-sided Jacobi
// sweeps of the core in FP32, and finishes with a double-float Rayleigh step
// sigma_i = |E v_i| on the top-r right vectors plus a CholeskyQR of E V_r, so
// the singular values are second-order accurate in the FP32 rotation error.
#include "pod_internal.h"

namespace {

// The one-CTA Cholesky kernels take a barrier per elimination step; with
// O(n^2 / 4) work per step, 8 warps finish a step sooner than 32.
constexpr int CHOL_THREADS = 256;
// k_small_chol: up to 1024 threads for the blocked factorisation's trailing
// updates and block products (1024 when g > 64, else 512)
constexpr int CHOL1_MAX_THREADS = 1024;
constexpr int CORE_THREADS = 512;

__device__ __forceinline__ double unit_roundoff(int dtype) {
    return dtype == POD_F32 ? 5.9604644775390625e-08 : 1.1102230246251565e-16;
}
__device__ __forceinline__ double round_to(int dtype, double v) {
    return dtype == POD_F32 ? (double)(float)v : v;
}

// ---------------------------------------------------------------------------
// Upper Cholesky with pivot dropping, one barrier per pivot.  W (n x n, ld)
// holds a symmetric Gram matrix in its upper triangle and is overwritten;
// R (ld) receives the factor with R^T R = G on the kept indices.  A pivot
// d <= thr (or d <= thrv[k], per index, when thrv is given) marks its index
// as numerically dependent: R's row is zero (Algorithm 2 drops the matching
// zero singular values of E).  Every thread forms the pivot's square root
// and reciprocals itself (no broadcast step).  Threads are laid out as NC
// columns (a power of two, at least min(n, blockDim)) by blockDim / NC row
// phases, fixed for the whole factorisation, so the inner loops carry no
// index division; step k writes row k of R and updates rows i > k, which
// read only row k.  piv3 is unused (kept for the callers' layouts).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int col_lanes(int n, int bd) {
    int nc = 32;
    while (nc < n && nc < bd) nc <<= 1;
    return nc > bd ? bd : nc;
}

template <typename X>
__device__ void chol_drop(X *W, int ldw, int n, X thr, X *R, int ldr, X *piv3, const X *thrv = nullptr) {
    (void)piv3;
    const int tid = threadIdx.x, bd = blockDim.x;
    for (int e = tid; e < n * n; e += bd) {
        const int i = e / n, j = e % n;
        if (i > j) R[i * ldr + j] = XOps<X>::zero();
    }
    const int NC = col_lanes(n, bd), RS = bd / NC;
    const int jt = tid & (NC - 1), it = tid / NC;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        const X d = W[k * ldw + k];
        const bool keep = x_gt(d, thrv ? thrv[k] : thr);
        X p = XOps<X>::zero(), inv_p = XOps<X>::zero(), inv_d = XOps<X>::zero();
        if (keep) {
            p = XOps<X>::sqrt_(d);
            inv_p = XOps<X>::one() / p;
            inv_d = inv_p * inv_p;
        }
        if (it < RS)
            for (int j = k + jt; j < n; j += NC) {
                const X wkj = W[k * ldw + j];
                if (it == 0) R[k * ldr + j] = keep ? (j == k ? p : wkj * inv_p) : XOps<X>::zero();
                if (!keep || j == k) continue;
                const X rkj = wkj * inv_d;
                for (int i = k + 1 + it; i <= j; i += RS) W[i * ldw + j] = W[i * ldw + j] - W[k * ldw + i] * rkj;
            }
        __syncthreads();
    }
}

// M = R^{-1} for upper triangular R, one barrier per row (zero pivots of
// dropped indices give zero rows and columns of M).  Mw is a work array;
// row k of M is the scaled row k of Mw, written while the rows above are
// updated from the unscaled row.  Same fixed thread layout as chol_drop.
template <typename X>
__device__ void tri_inv(const X *R, int ldr, int n, X *Mw, int ldw, X *M, int ldm, X *dinv) {
    const int tid = threadIdx.x, bd = blockDim.x;
    for (int e = tid; e < n * n; e += bd) {
        const int i = e / n, j = e % n;
        Mw[i * ldw + j] = (i == j) ? XOps<X>::one() : XOps<X>::zero();
        M[i * ldm + j] = XOps<X>::zero();
    }
    for (int k = tid; k < n; k += bd) {
        const X d = R[k * ldr + k];
        dinv[k] = x_hi(d) != 0.f ? XOps<X>::one() / d : XOps<X>::zero();
    }
    const int NC = col_lanes(n, bd), RS = bd / NC;
    const int jt = tid & (NC - 1), it = tid / NC;
    __syncthreads();
    for (int k = n - 1; k >= 0; --k) {
        const X inv = dinv[k];
        if (x_hi(inv) != 0.f && it < RS)
            for (int j = k + jt; j < n; j += NC) {
                const X mkj = Mw[k * ldw + j] * inv;
                if (it == 0) M[k * ldm + j] = mkj;
                for (int i = it; i < k; i += RS) Mw[i * ldw + j] = Mw[i * ldw + j] - R[i * ldr + k] * mkj;
            }
        __syncthreads();
    }
}

// C = A B for upper triangular A, B (all entries in parallel).
template <typename X>
__device__ void trmm_upper(const X *A, int lda, const X *B, int ldb, int n, X *C, int ldc) {
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        X s = XOps<X>::zero();
        for (int l = i; l <= j; ++l) s = s + A[i * lda + l] * B[l * ldb + j];
        C[i * ldc + j] = s;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// One-sided (Hestenes) Jacobi on the columns of B (nrow x ncol, column-major,
// ld ldb) with the rotations accumulated into V (ncol x ncol, ld ldv; V must
// hold I on entry).  Round-robin tournament ordering; a group of LP lanes
// rotates one column pair (MAXE elements per lane), so a round is
// ceil(ncol/2) disjoint pairs and one barrier.  Only the warps that hold
// pairs take part: they synchronise on hardware barrier 1 and the function
// returns at once on the other threads (the caller's next __syncthreads
// joins them).  Squared column norms are kept in alpha and updated
// analytically after each rotation (alpha_p - t g, alpha_q + t g), then
// recomputed exactly at every sweep; only b_p . b_q is reduced per pair.
// A pair is rotated while g^2 > tol^2 alpha_p alpha_q.  Bounded by
// max_sweeps.  On return alpha holds exact squared norms (on the working
// threads; visible to all after the caller's barrier).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bar_sync_1(int nthreads) {
    asm volatile("bar.sync 1, %0;\n" ::"r"(nthreads) : "memory");
}

template <typename J, int LP, int MAXE>
__device__ int jacobi_lp(J *B, int ldb, int nrow, int ncol, J *V, int ldv, J *alpha, J tol, int max_sweeps,
                         int *s_flag) {
    // nrow, ncol <= LP * MAXE
    constexpr int PPW = 32 / LP;   // pairs per warp
    const int N = ncol + (ncol & 1), npairs = N / 2, M = N - 1;
    int nwarps = (npairs + PPW - 1) / PPW;
    if (nwarps > (int)(blockDim.x >> 5)) nwarps = blockDim.x >> 5;   // then warps take several pairs
    if (nwarps < 1) nwarps = 1;
    const int nwork = 32 * nwarps;
    const int tid = threadIdx.x;
    if (tid >= nwork) return 0;
    const int lane = tid & 31, sub = lane / LP, lp = lane % LP, warp = tid >> 5;
    const J tol2 = tol * tol;
    // a sweep whose largest relative off-diagonal g^2 / (alpha_p alpha_q) stays
    // below loose2 leaves every pair below tol after its own rotations
    // (quadratic convergence), so the all-quiet check sweep is skipped
    const J loose2 = (J)16 * tol;
    int sweep = 0;
    for (;; ++sweep) {
        for (int c = tid; c < ncol; c += nwork) {
            J s = 0;
            for (int i = 0; i < nrow; ++i) s = fma(B[(size_t)c * ldb + i], B[(size_t)c * ldb + i], s);
            alpha[c] = s;
        }
        if (tid == 0) *s_flag = 0;
        bar_sync_1(nwork);
        if (sweep >= max_sweeps || ncol < 2) break;
        for (int rnd = 0; rnd < M; ++rnd) {
          for (int pr0 = warp * PPW; pr0 < npairs; pr0 += nwork / LP) {
            const int pr = pr0 + sub;
            int p = 0, q = 0;
            bool valid = pr < npairs;
            if (valid) {
                if (pr == 0) {
                    p = M;
                    q = rnd;
                } else {
                    p = rnd + pr;
                    if (p >= M) p -= M;
                    q = rnd - pr + M;
                    if (q >= M) q -= M;
                }
                if (p >= ncol || q >= ncol) valid = false;
                if (p > q) { int tmp = p; p = q; q = tmp; }
            }
            J *bp = B + (size_t)p * ldb, *bq = B + (size_t)q * ldb;
            J *vp = V + (size_t)p * ldv, *vq = V + (size_t)q * ldv;
            J x[MAXE], y[MAXE];
            J g0 = 0, g1 = 0;
#pragma unroll
            for (int e = 0; e < MAXE; ++e) {
                const int i = lp + LP * e;
                const bool in = valid && i < nrow;
                x[e] = in ? bp[i] : (J)0;
                y[e] = in ? bq[i] : (J)0;
                if (e & 1) g1 = fma(x[e], y[e], g1);
                else g0 = fma(x[e], y[e], g0);
            }
            J g = g0 + g1;
#pragma unroll
            for (int o = LP / 2; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o, LP);
            if (valid) {
                const J a = alpha[p], b = alpha[q];
                if (a > (J)0 && b > (J)0 && g * g > loose2 * loose2 * a * b && lp == 0) s_flag[1] = 1;
                if (a > (J)0 && b > (J)0 && g * g > tol2 * a * b) {
                    const J zeta = j_div(b - a, g + g);
                    const J az = fabs(zeta);
                    J t;
                    if (az > (J)1e15) {
                        t = j_div((J)0.5, zeta);
                    } else {
                        const J w = (J)1 + zeta * zeta;
                        t = j_div((J)1, az + w * j_rsqrt(w));
                        if (zeta < (J)0) t = -t;
                    }
                    const J cs = j_rsqrt((J)1 + t * t), sn = cs * t;
#pragma unroll
                    for (int e = 0; e < MAXE; ++e) {
                        const int i = lp + LP * e;
                        if (i < nrow) {
                            bp[i] = cs * x[e] - sn * y[e];
                            bq[i] = sn * x[e] + cs * y[e];
                        }
                        if (i < ncol) {
                            const J vx = vp[i], vy = vq[i];
                            vp[i] = cs * vx - sn * vy;
                            vq[i] = sn * vx + cs * vy;
                        }
                    }
                    if (lp == 0) {
                        alpha[p] = a - t * g;
                        alpha[q] = b + t * g;
                        *s_flag = 1;
                    }
                }
            }
          }
            bar_sync_1(nwork);
        }
        const int rotated = s_flag[0], big = s_flag[1];
        bar_sync_1(nwork);
        if (tid == 0) s_flag[1] = 0;
        if (!rotated) break;
        if (!big) {
            ++sweep;
            for (int c = tid; c < ncol; c += nwork) {
                J s = 0;
                for (int i = 0; i < nrow; ++i) s = fma(B[(size_t)c * ldb + i], B[(size_t)c * ldb + i], s);
                alpha[c] = s;
            }
            break;
        }
    }
    return sweep;
}

// Half-warp pairs: 4 elements per lane up to 64 columns, 10 up to 160, 20 up
// to 320.
template <typename J>
__device__ int jacobi_hw(J *B, int ldb, int nrow, int ncol, J *V, int ldv, J *alpha, J tol, int max_sweeps,
                         int *s_flag) {
    if (nrow <= 64 && ncol <= 64) return jacobi_lp<J, 16, 4>(B, ldb, nrow, ncol, V, ldv, alpha, tol, max_sweeps, s_flag);
    if (nrow <= 160 && ncol <= 160)
        return jacobi_lp<J, 16, 10>(B, ldb, nrow, ncol, V, ldv, alpha, tol, max_sweeps, s_flag);
    return jacobi_lp<J, 16, 20>(B, ldb, nrow, ncol, V, ldv, alpha, tol, max_sweeps, s_flag);
}

// Lean FP32 variant for n_c <= 64, same ordering, thresholds and stopping
// rule as jacobi_lp.  B (and V) have leading dimension 64 with zero rows
// beyond nrow, so four lanes hold a column pair as four 16-byte row groups
// each, with no bounds tests; the pairs of a warp take their row groups in
// rotated order so that each 8-lane phase of a 16-byte access touches all 32
// banks once; each lane group keeps its pair indices in registers and
// advances them by one per round; the rotation uses reciprocal square roots
// only (an FP32 rotation orthogonal to a few ulp is all the double-float
// finish needs).  V is rotated only when WITHV.  (Four lanes per pair
// measured faster than 8 or 16 on 60-column cores, and 16-byte row groups
// than 4-byte rows.)
constexpr int LEAN_LD = 64;     // smallest leading dimension of the lean layout
constexpr int LEAN_MAX = 160;   // widest core the lean layout serves

// leading dimension of the lean layout for cores up to nmax wide
__host__ __device__ inline int lean_ld(int nmax) {
    return nmax <= 64 ? 64 : (nmax <= 96 ? 96 : (nmax <= 128 ? 128 : 160));
}

template <bool WITHV, int LD>
__device__ int jacobi_lean(float *B, int ncol, float *V, float *alpha, float tol, int max_sweeps, int *s_flag,
                           int keep_top = 0) {
    // keep_top > 0: only the keep_top rows of largest norm are used afterwards,
    // so from the third sweep on a pair whose squared norms are both below an
    // eighth of the keep_top-th largest counts as converged (the rows among
    // the rest need not be orthogonal to one another; every pair touching a
    // leading row still is).  A Gershgorin test at the end confirms that the
    // trailing rows hide no direction above the leading ones, else the sweeps
    // go on over every pair.
    __shared__ float s_thr;
    constexpr int LP = 4, PPW = 8;
    constexpr int KG = LD / 16;   // 16-row groups of a row; each lane holds one float4 of each
    const int N = ncol + (ncol & 1), npairs = N / 2, M = N - 1;
    const int nwork = 32 * ((npairs + PPW - 1) / PPW);
    const int tid = threadIdx.x;
    if (tid >= nwork) return 0;
    const int lane = tid & 31, lp = lane % LP, sub = lane / LP, pr = (tid >> 5) * PPW + sub;
    const bool active = pr < npairs;
    // float4 index of this lane's part of row group k: rows 16 ((k + sub) mod
    // KG) + 4 lp .. + 3 (rows start on bank 0 since LD is a multiple of 32
    // floats; the rotation by sub puts the two pairs of an 8-lane phase 16
    // banks apart)
    int off[KG];
#pragma unroll
    for (int k = 0; k < KG; ++k) off[k] = 4 * ((k + sub) % KG) + lp;
    const float tol2 = tol * tol, loose = 16.f * tol, loose2 = loose * loose;
    const int max_sweeps0 = max_sweeps;
    int sweep = 0;
    for (;;) {   // a second pass only when the guard below turns the skipping off
    for (;; ++sweep) {
        for (int c = tid; c < ncol; c += nwork) {
            const float4 *bc = reinterpret_cast<const float4 *>(B + (size_t)c * LD);
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int i = 0; i < LD / 4; i += 2) {
                const float4 u0 = bc[i], u1 = bc[i + 1];
                s0 = fmaf(u0.x, u0.x, fmaf(u0.y, u0.y, fmaf(u0.z, u0.z, fmaf(u0.w, u0.w, s0))));
                s1 = fmaf(u1.x, u1.x, fmaf(u1.y, u1.y, fmaf(u1.z, u1.z, fmaf(u1.w, u1.w, s1))));
            }
            alpha[c] = s0 + s1;
        }
        if (tid == 0) {
            s_flag[0] = 0;
            s_thr = 0.f;   // no pair skipped unless a rank below sets it (a NaN norm matches no rank)
        }
        bar_sync_1(nwork);
        if (sweep >= max_sweeps || ncol < 2) break;
        if (keep_top > 0 && keep_top < ncol) {
            if (tid < 32) {
                // the keep_top-th largest squared norm (ranks with ties by index)
                for (int c = tid; c < ncol; c += 32) {
                    const float ac = alpha[c];
                    int rank = 0;
                    for (int j = 0; j < ncol; ++j) {
                        const float aj = alpha[j];
                        rank += (aj > ac || (aj == ac && j < c)) ? 1 : 0;
                    }
                    if (rank == keep_top - 1) s_thr = sweep >= 2 ? 0.125f * ac : 0.f;
                }
            }
            bar_sync_1(nwork);
        }
        const float thr = (keep_top > 0 && keep_top < ncol) ? s_thr : 0.f;
        // round 0 of the tournament: pair 0 = (M, 0), pair k = (k, M - k)
        int pa = pr == 0 ? M : pr, qa = pr == 0 ? 0 : M - pr;
        for (int rnd = 0; rnd < M; ++rnd) {
            const int p = active ? min(pa, qa) : 0, q = active ? max(pa, qa) : 0;
            const bool valid = active && q < ncol;
            float4 *bp = reinterpret_cast<float4 *>(B + (size_t)p * LD);
            float4 *bq = reinterpret_cast<float4 *>(B + (size_t)(valid ? q : p) * LD);
            float4 x[KG], y[KG];
#pragma unroll
            for (int k = 0; k < KG; ++k) {
                x[k] = bp[off[k]];
                y[k] = bq[off[k]];
            }
            const float a = alpha[p], b = alpha[valid ? q : p];
            float g0 = 0.f, g1 = 0.f;
#pragma unroll
            for (int k = 0; k < KG; ++k) {
                g0 = fmaf(x[k].x, y[k].x, g0);
                g1 = fmaf(x[k].y, y[k].y, g1);
                g0 = fmaf(x[k].z, y[k].z, g0);
                g1 = fmaf(x[k].w, y[k].w, g1);
            }
            float g = g0 + g1;
            g += __shfl_xor_sync(0xffffffffu, g, 2, LP);
            g += __shfl_xor_sync(0xffffffffu, g, 1, LP);
            if (valid && (a >= thr || b >= thr)) {
                const float ab = a * b, g2 = g * g;
                if (ab > 0.f && g2 > loose2 * ab && lp == 0) s_flag[1] = 1;
                if (ab > 0.f && g2 > tol2 * ab) {
                    // the rotation with |theta| <= pi/4 that makes b_p . b_q
                    // zero: with d = alpha_q - alpha_p, h = 2 g, r = |(d, h)|:
                    // cos 2theta = |d| / r, cos theta = sqrt((1 + cos 2theta) / 2),
                    // sin theta = sign(d) h / (2 r cos theta), t = tan theta
                    const float d = b - a, h = g + g;
                    const float ir = rsqrtf(fmaf(d, d, h * h));
                    const float y2 = fmaf(0.5f * fabsf(d), ir, 0.5f);
                    const float iy = rsqrtf(y2);
                    const float cs = y2 * iy;
                    const float sn = copysignf(1.f, d) * (0.5f * h) * (ir * iy);
                    const float t = sn * iy;
#pragma unroll
                    for (int k = 0; k < KG; ++k) {
                        bp[off[k]] = make_float4(fmaf(cs, x[k].x, -sn * y[k].x), fmaf(cs, x[k].y, -sn * y[k].y),
                                                 fmaf(cs, x[k].z, -sn * y[k].z), fmaf(cs, x[k].w, -sn * y[k].w));
                        bq[off[k]] = make_float4(fmaf(sn, x[k].x, cs * y[k].x), fmaf(sn, x[k].y, cs * y[k].y),
                                                 fmaf(sn, x[k].z, cs * y[k].z), fmaf(sn, x[k].w, cs * y[k].w));
                    }
                    if (WITHV) {
                        float4 *vp = reinterpret_cast<float4 *>(V + (size_t)p * LD);
                        float4 *vq = reinterpret_cast<float4 *>(V + (size_t)q * LD);
#pragma unroll
                        for (int k = 0; k < KG; ++k) {
                            const float4 vx = vp[off[k]], vy = vq[off[k]];
                            vp[off[k]] = make_float4(fmaf(cs, vx.x, -sn * vy.x), fmaf(cs, vx.y, -sn * vy.y),
                                                     fmaf(cs, vx.z, -sn * vy.z), fmaf(cs, vx.w, -sn * vy.w));
                            vq[off[k]] = make_float4(fmaf(sn, vx.x, cs * vy.x), fmaf(sn, vx.y, cs * vy.y),
                                                     fmaf(sn, vx.z, cs * vy.z), fmaf(sn, vx.w, cs * vy.w));
                        }
                    }
                    if (lp == 0) {
                        alpha[p] = fmaf(-t, g, a);
                        alpha[q] = fmaf(t, g, b);
                        s_flag[0] = 1;
                    }
                }
            }
            if (pr == 0) {
                qa = rnd + 1;
            } else {
                pa = pa + 1 == M ? 0 : pa + 1;
                qa = qa + 1 == M ? 0 : qa + 1;
            }
            bar_sync_1(nwork);
        }
        const int rotated = s_flag[0], big = s_flag[1];
        bar_sync_1(nwork);
        if (tid == 0) s_flag[1] = 0;
        if (!rotated) break;
        if (!big) {
            ++sweep;
            for (int c = tid; c < ncol; c += nwork) {
                const float *bc = B + (size_t)c * LD;
                float s0 = 0.f;
                for (int i = 0; i < LD; ++i) s0 = fmaf(bc[i], bc[i], s0);
                alpha[c] = s0;
            }
            break;
        }
    }
    // guard: the trailing rows, not orthogonalised among themselves, must
    // not hold a direction above the keep_top-th leading row.  Gershgorin:
    // every eigenvalue of their Gram lies below max_i (alpha_i + sum_j
    // |b_i . b_j|); if that reaches the keep_top-th largest alpha, the
    // sweeps go on over every pair
    if (keep_top > 0 && keep_top < ncol) {
        __shared__ int s_top[LD];
        __shared__ float s_amin;
        __shared__ int s_bad;
        bar_sync_1(nwork);   // the final norms are in
        if (tid == 0) s_bad = 0;
        for (int c = tid; c < ncol; c += nwork) {
            const float ac = alpha[c];
            int rank = 0;
            for (int j = 0; j < ncol; ++j) {
                const float aj = alpha[j];
                rank += (aj > ac || (aj == ac && j < c)) ? 1 : 0;
            }
            s_top[c] = rank < keep_top;
            if (rank == keep_top - 1) s_amin = ac;
        }
        bar_sync_1(nwork);
        // |b_i . b_j| of the trailing pairs into Dm (V's storage, unused
        // without WITHV), spread over the threads; then each trailing row's
        // radius in a fixed order
        float *Dm = V;
        for (int e = tid; e < ncol * ncol; e += nwork) {
            const int i = e / ncol, j = e - i * ncol;
            if (i >= j || s_top[i] || s_top[j]) continue;
            const float4 *bi = reinterpret_cast<const float4 *>(B + (size_t)i * LD);
            const float4 *bj = reinterpret_cast<const float4 *>(B + (size_t)j * LD);
            float d0 = 0.f, d1 = 0.f;
#pragma unroll
            for (int k = 0; k < LD / 4; k += 2) {
                const float4 x0 = bi[k], y0 = bj[k], x1 = bi[k + 1], y1 = bj[k + 1];
                d0 = fmaf(x0.x, y0.x, fmaf(x0.y, y0.y, fmaf(x0.z, y0.z, fmaf(x0.w, y0.w, d0))));
                d1 = fmaf(x1.x, y1.x, fmaf(x1.y, y1.y, fmaf(x1.z, y1.z, fmaf(x1.w, y1.w, d1))));
            }
            const float d = fabsf(d0 + d1);
            Dm[i * LD + j] = d;
            Dm[j * LD + i] = d;
        }
        bar_sync_1(nwork);
        for (int i = tid; i < ncol; i += nwork) {
            if (s_top[i]) continue;
            float rad = 0.f;
            for (int j = 0; j < ncol; ++j)
                if (j != i && !s_top[j]) rad += Dm[i * LD + j];
            if (alpha[i] + rad >= s_amin) s_bad = 1;
        }
        bar_sync_1(nwork);
        if (s_bad) {
            // sweep every pair from here on; when the skipping used up the
            // sweep budget, the full sweeps get a budget of their own
            if (sweep >= max_sweeps) max_sweeps = sweep + max_sweeps0;
            keep_top = 0;
            continue;
        }
    }
    break;
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

// Largest singular value of B (nrow x k), the square root of the largest
// eigenvalue lambda_1 of the k x k matrix M = B^T B:
//  * M from B stored row by row (Bt[p k + i] = B[p][i]: consecutive threads
//    read consecutive entries);
//  * P = M / trace(M), then repeated squaring P <- P^2 / trace(P^2): after s
//    squarings P is M^(2^s) normalised, whose eigenvalues are
//    (lambda_i / lambda_1)^(2^s) relative to the top one, so P approaches the
//    projector on the top eigenvector; it stops when trace(P^2) > 1 - eps
//    (one eigenvalue left) or after SQ_MAX squarings (M^16384);
//  * x = the column of P with the largest diagonal, refined by SQ_APPLY
//    products with P (each worth 2^s power steps), then the Rayleigh quotient
//    x^T M x / x^T x with the original M: a lower bound of lambda_1 whose
//    error is (lambda_1 - lambda_j) times the square of x's residual
//    components, clamped to [trace(M) / k, trace(M)], bounds any lambda_1 of
//    M obeys.  A degenerate top eigenvalue needs no separation: any vector of
//    its eigenspace gives it exactly.
// The power iteration this replaces (16 plain steps) under-read sin(theta)
// by up to 1.4e-3 when the top two singular values of B were close; a
// Lanczos version with full reorthogonalisation was exact but cost ~4 k
// thousand cycles per core.
// Work arrays: M, P, P2 k^2 each, x and y k each.  Called by the whole CTA;
// the result is valid in every thread.
constexpr int SQ_MAX = 14;
constexpr int SQ_APPLY = 4;

template <typename J>
__device__ void sq_matmul(const J *A, J *C, int k) {
    // C = A A for symmetric A (k x k, row-major); four partial sums per entry
    const int tid = threadIdx.x, bd = blockDim.x;
    for (int e = tid; e < k * k; e += bd) {
        const int i = e / k, j = e - i * k;
        J v0 = 0, v1 = 0, v2 = 0, v3 = 0;
        int t = 0;
        for (; t + 4 <= k; t += 4) {
            v0 = fma(A[i * k + t], A[t * k + j], v0);
            v1 = fma(A[i * k + t + 1], A[(t + 1) * k + j], v1);
            v2 = fma(A[i * k + t + 2], A[(t + 2) * k + j], v2);
            v3 = fma(A[i * k + t + 3], A[(t + 3) * k + j], v3);
        }
        for (; t < k; ++t) v0 = fma(A[i * k + t], A[t * k + j], v0);
        C[e] = (v0 + v1) + (v2 + v3);
    }
}

// Sum of v[i * stride] over i < k by warp 0 (lane partials, then a fixed
// shuffle tree), the same value returned to every thread.  Called by the
// whole CTA; ends with a barrier.
template <typename J>
__device__ J warp0_sum(const J *v, int k, int stride) {
    __shared__ J s_sum;
    const int tid = threadIdx.x;
    if (tid < 32) {
        J part = 0;
        for (int i = tid; i < k; i += 32) part += v[(size_t)i * stride];
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (tid == 0) s_sum = part;
    }
    __syncthreads();
    const J r = s_sum;
    __syncthreads();
    return r;
}

template <typename J>
__device__ double top_singular_value(const J *Bt, int nrow, int k, J *M, J *P, J *P2, J *x, J *y, double *red_d) {
    const int tid = threadIdx.x, bd = blockDim.x;
    J *red = reinterpret_cast<J *>(red_d);
    for (int e = tid; e < k * k; e += bd) {
        const int i = e / k, j = e - i * k;
        J v0 = 0, v1 = 0;
        int p = 0;
        for (; p + 2 <= nrow; p += 2) {
            v0 = fma(Bt[p * k + i], Bt[p * k + j], v0);
            v1 = fma(Bt[(p + 1) * k + i], Bt[(p + 1) * k + j], v1);
        }
        if (p < nrow) v0 = fma(Bt[p * k + i], Bt[p * k + j], v0);
        M[e] = v0 + v1;
    }
    __syncthreads();
    const J tr = warp0_sum<J>(M, k, k + 1);
    if (!(tr > (J)0)) return 0.0;   // B = 0 (or not finite); every thread the same
    const J eps = sizeof(J) == 4 ? (J)1e-6 : (J)1e-13;
    const J itr = (J)1 / tr;
    for (int e = tid; e < k * k; e += bd) P[e] = M[e] * itr;
    __syncthreads();
    J *cur = P, *nxt = P2;
    for (int sq = 0; sq < SQ_MAX; ++sq) {
        sq_matmul<J>(cur, nxt, k);
        __syncthreads();
        const J t2 = warp0_sum<J>(nxt, k, k + 1);   // trace(cur^2) = sum of squared eigenvalues
        if (!(t2 > (J)0)) break;                    // (every thread the same)
        const J it2 = (J)1 / t2;
        for (int e = tid; e < k * k; e += bd) nxt[e] *= it2;
        __syncthreads();
        J *sw = cur;
        cur = nxt;
        nxt = sw;
        if (t2 > (J)1 - eps) break;                           // one eigenvalue left
    }
    // x = the column of cur with the largest diagonal (the first of equal
    // ones), found by warp 0
    __shared__ int s_imax;
    if (tid < 32) {
        J best = -1;
        int bi = k;
        for (int i = tid; i < k; i += 32) {
            const J v = cur[i * k + i];
            if (v > best) {
                best = v;
                bi = i;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const J ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if (tid == 0) s_imax = bi < k ? bi : 0;
    }
    __syncthreads();
    const int imax = s_imax;
    for (int i = tid; i < k; i += bd) x[i] = cur[i * k + imax];
    __syncthreads();
    for (int it = 0; it < SQ_APPLY; ++it) {
        for (int i = tid; i < k; i += bd) {
            J v = 0;
            for (int t = 0; t < k; ++t) v = fma(cur[i * k + t], x[t], v);
            y[i] = v;
        }
        __syncthreads();
        // |y|^2 (every thread the same)
        __shared__ J s_n2;
        if (tid < 32) {
            J part = 0;
            for (int t = tid; t < k; t += 32) part = fma(y[t], y[t], part);
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            if (tid == 0) s_n2 = part;
        }
        __syncthreads();
        const J n2 = s_n2;
        const J in = n2 > (J)0 ? (J)1 / sqrt(n2) : (J)0;
        __syncthreads();
        for (int i = tid; i < k; i += bd) x[i] = y[i] * in;
        __syncthreads();
    }
    // Rayleigh quotient with the original M
    J num = 0;
    for (int i = tid; i < k; i += bd) {
        J v = 0;
        for (int t = 0; t < k; ++t) v = fma(M[i * k + t], x[t], v);
        num = fma(x[i], v, num);
    }
    num = block_sum<J>(num, red);
    __shared__ J s_xx;
    if (tid < 32) {
        J part = 0;
        for (int t = tid; t < k; t += 32) part = fma(x[t], x[t], part);
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (tid == 0) s_xx = part;
    }
    __syncthreads();
    const J xx = s_xx;
    J lam = xx > (J)0 ? num / xx : (J)0;
    const J lower = tr / (J)k;
    lam = lam < lower ? lower : (lam > tr ? tr : lam);
    return sqrt((double)lam);
}

__host__ __device__ inline size_t al16x(size_t b) { return (b + 15) / 16 * 16; }

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
// Blocked forms of chol_drop and tri_inv for the first CholeskyQR kernel
// (CB-row blocks: a few barriers per block instead of one per row).
// ---------------------------------------------------------------------------
constexpr int CB = 8;

// Right-looking Cholesky with the pivot drops of chol_drop (a pivot not
// above its floor (thrv[k], else thr) gives a zero row of R).  W: upper
// triangle (ld ldw), updated in place; R: upper triangular factor (ld ldr).
// Warp 0 forms each CB-row panel of R (row k: W[k][j] minus the panel rows
// above it, divided by the pivot), then all threads subtract the panel's
// rank-CB product from the trailing upper triangle of W.
template <typename X>
__device__ void chol_drop_blk(X *W, int ldw, int n, X thr, X *R, int ldr, const X *thrv) {
    const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31;
    for (int e = tid; e < n * n; e += bd) {
        const int i = e / n, j = e - i * n;
        if (i > j) R[i * ldr + j] = XOps<X>::zero();
    }
    __syncthreads();
    for (int k0 = 0; k0 < n; k0 += CB) {
        const int k1 = k0 + CB < n ? k0 + CB : n;
        if (tid < 32) {
            for (int k = k0; k < k1; ++k) {
                X d = W[k * ldw + k];
                for (int l = k0; l < k; ++l) d = d - R[l * ldr + k] * R[l * ldr + k];
                const bool keep = x_gt(d, thrv ? thrv[k] : thr);
                X p = XOps<X>::zero(), inv_p = XOps<X>::zero();
                if (keep) {
                    p = XOps<X>::sqrt_(d);
                    inv_p = XOps<X>::one() / p;
                }
                for (int j = k + lane; j < n; j += 32) {
                    X w = W[k * ldw + j];
                    for (int l = k0; l < k; ++l) w = w - R[l * ldr + k] * R[l * ldr + j];
                    R[k * ldr + j] = keep ? (j == k ? p : w * inv_p) : XOps<X>::zero();
                }
                __syncwarp();
            }
        }
        __syncthreads();
        const int nt = n - k1;
        for (int e = tid; e < nt * nt; e += bd) {
            const int i = k1 + e / nt, j = k1 + e % nt;
            if (i > j) continue;
            X w = W[i * ldw + j];
            for (int l = k0; l < k1; ++l) w = w - R[l * ldr + i] * R[l * ldr + j];
            W[i * ldw + j] = w;
        }
        __syncthreads();
    }
}

// M = R^{-1} for upper triangular R (zero pivots of dropped indices give
// zero rows and columns of M): the CB x CB diagonal blocks by back
// substitution (a thread per column), then the blocks at block distance
// 1, 2, ...: M_IJ = -M_II (sum_{K = I+1..J} R_IK M_KJ).  T: scratch of
// ceil(n / CB) CB^2 entries.
template <typename X>
__device__ void tri_inv_blk(const X *R, int ldr, int n, X *M, int ldm, X *T, X *dinv) {
    const int tid = threadIdx.x, bd = blockDim.x;
    const int nb = (n + CB - 1) / CB;
    for (int e = tid; e < n * n; e += bd) {
        const int i = e / n, j = e - i * n;
        M[i * ldm + j] = XOps<X>::zero();
    }
    for (int k = tid; k < n; k += bd) {
        const X d = R[k * ldr + k];
        dinv[k] = x_hi(d) != 0.f ? XOps<X>::one() / d : XOps<X>::zero();
    }
    __syncthreads();
    for (int j = tid; j < n; j += bd) {
        const int i0 = (j / CB) * CB;
        M[j * ldm + j] = dinv[j];
        for (int i = j - 1; i >= i0; --i) {
            X sum = XOps<X>::zero();
            for (int l = i + 1; l <= j; ++l) sum = sum + R[i * ldr + l] * M[l * ldm + j];
            M[i * ldm + j] = XOps<X>::zero() - sum * dinv[i];
        }
    }
    __syncthreads();
    for (int dl = 1; dl < nb; ++dl) {
        const int np = nb - dl;
        for (int e = tid; e < np * CB * CB; e += bd) {
            const int bi = e / (CB * CB), rem = e - bi * CB * CB;
            const int i = bi * CB + rem / CB, j = (bi + dl) * CB + rem % CB;
            X sum = XOps<X>::zero();
            if (i < n && j < n)
                for (int l = (bi + 1) * CB; l <= j; ++l) sum = sum + R[i * ldr + l] * M[l * ldm + j];
            T[e] = sum;
        }
        __syncthreads();
        for (int e = tid; e < np * CB * CB; e += bd) {
            const int bi = e / (CB * CB), rem = e - bi * CB * CB, ii = rem / CB, jj = rem % CB;
            const int i = bi * CB + ii, j = (bi + dl) * CB + jj;
            if (i >= n || j >= n) continue;
            const int iend = (bi + 1) * CB < n ? (bi + 1) * CB : n;
            X sum = XOps<X>::zero();
            for (int l = i; l < iend; ++l) sum = sum + M[i * ldm + l] * T[bi * CB * CB + (l - bi * CB) * CB + jj];
            M[i * ldm + j] = XOps<X>::zero() - sum;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// First CholeskyQR pass: Ptot = fl(P) + fl(P2), R1 = chol(Z^T Z) with pivot
// dropping, M1 = fl(R1^{-1}) (the matrix the tall pass applies), and
// R1p = M1^{-1} (the exact inverse of what was applied, used in E).
// ---------------------------------------------------------------------------
//
// XC is the arithmetic of the Cholesky and of M1: FP32 in the plain pass of
// FP32 data, whose Gram is only FP32-accurate anyway (M1 is rounded to FP32
// before use, so an FP32 inverse costs no accuracy: both errors are
// O(u kappa)); X (double-float or FP64) in the compensated rerun and for FP64
// data.  R1p, the inverse of the applied M1, is always formed in X.
struct Chol1Layout {
    size_t xc, x;      // one ld x ld array of XC / of X (16-byte multiples)
    size_t main;       // the larger of 3 xc and 2 x
    size_t t;          // the blocked inverse's scratch (ceil(ld / CB) CB^2 X)
    size_t vec;        // one length-ld X vector
    size_t total;
};
__host__ __device__ inline Chol1Layout chol1_layout(int ld, int xs, int xcs) {
    Chol1Layout L;
    L.xc = al16x((size_t)ld * ld * xcs);
    L.x = al16x((size_t)ld * ld * xs);
    L.main = 3 * L.xc > 2 * L.x ? 3 * L.xc : 2 * L.x;
    if (L.main < L.x) L.main = L.x;   // the column-norm squares (ld^2 doubles)
    L.t = al16x((size_t)((ld + CB - 1) / CB) * CB * CB * xs);
    L.vec = al16x((size_t)ld * xs);
    L.total = L.main + L.t + 2 * L.vec + 64;
    return L;
}

template <typename X, typename XC>
__global__ void __launch_bounds__(CHOL1_MAX_THREADS) k_small_chol(SmallArgs a) {
    DevState *st = a.st;
    if (st->done) return;
    if (a.cond && !st->robust) return;
    const int r = st->r_cur, g = st->g, nc = r + g;
    const int ld = a.cmax;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // layout (chol1_layout): the XC stage's three ld x ld XC arrays (W, R,
    // M), or the X stage's two ld x ld X arrays (M1, its inverse), over the
    // same bytes; then the blocked inverse's scratch, dinv and the pivot
    // floors
    const Chol1Layout CL = chol1_layout(ld, (int)sizeof(X), (int)sizeof(XC));
    unsigned char *base = a.gws_chol ? a.gws_chol : smem_raw;
    XC *Wc = reinterpret_cast<XC *>(base), *Rc = reinterpret_cast<XC *>(base + CL.xc);
    XC *Mc = reinterpret_cast<XC *>(base + 2 * CL.xc);
    X *R = reinterpret_cast<X *>(base), *Mx = reinterpret_cast<X *>(base + CL.x);
    unsigned char *tb = base + CL.main;   // blocked-inverse scratch
    X *dinv = reinterpret_cast<X *>(base + CL.main + CL.t);
    X *thrv_x = reinterpret_cast<X *>(base + CL.main + CL.t + CL.vec);
    __shared__ double red[32];
    XC *dinvc = reinterpret_cast<XC *>(dinv), *thrv = reinterpret_cast<XC *>(thrv_x);
    const int tid = threadIdx.x, bd = blockDim.x;
    const double *P2 = a.PG;
    const double *G = a.PG + (int64_t)a.rmax * a.cmax;

    // Ptot over all (l, j) at once (the global loads spread over the CTA),
    // then the squared column norms of the block from the squares kept at
    // the base of the work area (ld^2 8-byte entries; with r g beyond that,
    // per column)
    double *sq = reinterpret_cast<double *>(base);
    const bool spread = r * g <= ld * ld;
    if (spread)
        for (int e = tid; e < r * g; e += bd) {
            const int l = e / g, j = e - l * g;
            const double pt = round_to(a.dtype, a.P[l * ld + j]) + round_to(a.dtype, P2[l * ld + j]);
            a.Ptot[l * ld + j] = pt;
            sq[e] = pt * pt;
        }
    __syncthreads();
    double cmax2 = 0.0;
    for (int j = tid; j < g; j += bd) {
        double cn = G[j * ld + j];
        for (int l = 0; l < r; ++l) {
            if (spread) {
                cn += sq[l * g + j];
            } else {
                const double pt = round_to(a.dtype, a.P[l * ld + j]) + round_to(a.dtype, P2[l * ld + j]);
                a.Ptot[l * ld + j] = pt;
                cn += pt * pt;
            }
        }
        cmax2 = cn > cmax2 ? cn : cmax2;
    }
    cmax2 = block_max<double>(cmax2, red);
    const double s0 = r > 0 ? a.sigma[0] : 0.0;
    const double scale = cmax2 > s0 * s0 ? cmax2 : s0 * s0;
    // Pivot floors.  FP32 storage: a direction whose pivot d_j is dropped
    // hides at most sqrt(d_j) of the block, so the floor is (8u)^2 scale
    // (8 u sigma_1), which the compensated Gram of the rerun resolves.  The
    // plain FP32 Gram is off by up to ~ 8 u G_jj in the pivot of column j,
    // so there the floor for column j is also at least 8 u G_jj (smaller
    // pivots are rounding noise).  FP64 storage: (n_c u)^2 scale.
    const double u = unit_roundoff(a.dtype);
    const bool f32 = a.dtype == POD_F32;
    const double eps = f32 ? 8.0 * u : nc * u;
    const double floor_abs = eps * eps * scale;
    const XC thr = XOps<XC>::from(floor_abs);
    const bool plain32 = f32 && !a.cond;
    for (int j = tid; j < g; j += bd) {
        const double tj = 8.0 * u * G[j * ld + j];
        thrv[j] = XOps<XC>::from(plain32 && tj > floor_abs ? tj : floor_abs);
    }
    for (int e = tid; e < g * g; e += bd) {
        const int i = e / g, j = e % g;
        Wc[i * ld + j] = XOps<XC>::from(i <= j ? G[i * ld + j] : 0.0);
    }
    __syncthreads();
    chol_drop_blk<XC>(Wc, ld, g, thr, Rc, ld, thrv);
    if (!a.cond) {
        // a column the plain FP32 pass dropped under its noise floor
        // 8 u G_jj may hide more than 8 u sigma_1: the round then takes the
        // compensated rerun.  The QR2 pass adds its own test on G2 and counts
        // the round.
        int flag = 0;
        if (plain32)
            for (int j = tid; j < g; j += bd)
                if (x_hi(Rc[j * ld + j]) == 0.f && 8.0 * u * G[j * ld + j] > floor_abs) flag = 1;
        flag = __syncthreads_or(flag);
        if (tid == 0) st->robust = flag;
    }
    tri_inv_blk<XC>(Rc, ld, g, Mc, ld, reinterpret_cast<XC *>(tb), dinvc);
    // round M1 to the storage type: that is the matrix the QR2 pass applies;
    // its X copy goes to R's array (over Wc and Rc, no longer needed; R ends
    // where Mc starts)
    for (int e = tid; e < g * g; e += bd) {
        const int i = e / g, j = e % g;
        const double v = round_to(a.dtype, XOps<XC>::to(Mc[i * ld + j]));
        a.M1[i * ld + j] = v;
        R[i * ld + j] = XOps<X>::from(v);
    }
    __syncthreads();
    tri_inv_blk<X>(R, ld, g, Mx, ld, reinterpret_cast<X *>(tb), dinv);
    for (int e = tid; e < g * g; e += bd) {
        const int i = e / g, j = e % g;
        a.R1p[i * ld + j] = XOps<X>::to(Mx[i * ld + j]);
    }
}

size_t small_chol_smem(int cmax, int dtype, int cond) {
    const int xs = 8, xcs = (dtype == POD_F32 && !cond) ? 4 : 8;
    return chol1_layout(cmax, xs, xcs).total;
}

pod_status launch_small_chol(const SmallArgs &a0, cudaStream_t s) {
    // shared memory when this form's layout fits, else the global scratch
    SmallArgs a = a0;
    size_t smem = small_chol_smem(a.cmax, a.dtype, a.cond);
    if (smem <= 220 * 1024) {
        a.gws_chol = nullptr;
    } else {
        if (!a.gws_chol) return POD_EUNSUPPORTED;
        smem = 64;
    }
    const int nthr = a.cmax > 64 ? CHOL1_MAX_THREADS : 512;
    if (a.dtype == POD_F32 && !a.cond) {
        POD_CUDA_TRY(cudaFuncSetAttribute(k_small_chol<dfloat, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_small_chol<dfloat, float><<<1, nthr, smem, s>>>(a);
    } else if (a.dtype == POD_F32) {
        POD_CUDA_TRY(cudaFuncSetAttribute(k_small_chol<dfloat, dfloat>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_small_chol<dfloat, dfloat><<<1, nthr, smem, s>>>(a);
    } else {
        POD_CUDA_TRY(cudaFuncSetAttribute(k_small_chol<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_small_chol<double, double><<<1, nthr, smem, s>>>(a);
    }
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}

// ---------------------------------------------------------------------------
// Second CholeskyQR pass, the core E and its SVD, truncation, convergence,
// and the update coefficients.
//
// The SVD of E runs one-sided Jacobi on the rows of E (the columns of E^T),
// accumulating the rotations: E^T V = W Sigma, so V holds U_E.  (On E's
// columns the same matrices needed about 40% more sweeps.)  FP64 path: all
// in FP64, U_E = V, sigma = column norms.  FP32 path: sweeps in FP32, then
// the top-r columns of V are re-orthonormalised by a double-float
// CholeskyQR (leading spans kept) and sigma_i = |E^T q_i| in double-float:
// a Rayleigh quotient, second-order accurate in the FP32 rotation error.
// ---------------------------------------------------------------------------
struct CoreLayout {
    size_t keep;     // E, Rinv, Ptot as X (persist across phases)
    size_t phaseA;   // 6 g x g X matrices
    size_t phaseB;   // Jacobi: B and V (J), alpha (J), order (int)
    size_t phaseC;   // finish
    size_t total;
};

__host__ __device__ inline CoreLayout core_layout(int rmax, int cmax, int jsize) {
    CoreLayout L;
    const int nmax = rmax + cmax;
    L.keep = al16x((size_t)nmax * nmax * 8) + al16x((size_t)cmax * cmax * 8) + al16x((size_t)rmax * cmax * 8);
    // FP32 path: 3 X + 8 float g x g arrays; FP64 path: 5 X arrays
    L.phaseA = jsize == 4 ? 3 * al16x((size_t)cmax * cmax * 8) + 8 * al16x((size_t)cmax * cmax * 4)
                          : 5 * al16x((size_t)cmax * cmax * 8);
    // B, V: leading dimension lean_ld(nmax) (zero-padded rows) on the lean
    // FP32 path (n_c <= 160)
    const size_t jb = (jsize == 4 && nmax <= LEAN_MAX) ? (size_t)lean_ld(nmax) * nmax : (size_t)nmax * nmax;
    L.phaseB = 2 * al16x(jb * jsize) + al16x((size_t)nmax * jsize) + al16x((size_t)nmax * 4);
    // Vr, Q, Yt: nmax x rmax X; Gb, Rb, Mw, Mb: rmax x rmax X; Bs: nmax x rmax J;
    // BtB, Psq: rmax^2 J each; xv, yv: rmax J; sig: rmax X; ord2: rmax int
    L.phaseC = 3 * al16x((size_t)nmax * rmax * 8) + 4 * al16x((size_t)rmax * rmax * 8) +
               al16x((size_t)nmax * rmax * jsize) + 2 * al16x((size_t)rmax * rmax * jsize) + 2 * al16x((size_t)rmax * jsize) +
               al16x((size_t)rmax * 8) + al16x((size_t)rmax * 4);
    const size_t bc = L.phaseB + L.phaseC;
    L.total = L.keep + (L.phaseA > bc ? L.phaseA : bc) + 64;
    return L;
}

size_t core_smem_bytes(int rmax, int cmax, int dtype) {
    return core_layout(rmax, cmax, dtype == POD_F32 ? 4 : 8).total;
}

size_t core_jacobi_bytes(int rmax, int cmax, int dtype) {
    return core_layout(rmax, cmax, dtype == POD_F32 ? 4 : 8).phaseB + 64;
}

template <typename X, typename J>
__global__ void __launch_bounds__(CORE_THREADS) k_core(SmallArgs a) {
    DevState *st = a.st;
    if (st->done) return;
    const int r = st->r_cur, g = st->g, nc = r + g, t = st->t;
    const int ld = a.cmax, nmax = a.rmax + a.cmax;
    const int tid = threadIdx.x, bd = blockDim.x;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_flag[2];
    __shared__ double red[32];
    __shared__ int s_rnew;
    __shared__ double s_measure, s_sin, s_cos;
    __shared__ int s_bad;
    __shared__ X piv3[3];
    __shared__ X dinv[256];
    const double u = unit_roundoff(a.dtype);
    long long clk[6];
    clk[0] = clock64();
    if (tid == 0) s_bad = 0;
    const CoreLayout CL = core_layout(a.rmax, a.cmax, (int)sizeof(J));
    // wide cores: everything but the Jacobi arrays in global scratch
    unsigned char *gbase = a.gws_core;
    Carve keep{gbase ? gbase : smem_raw};
    X *Ex = keep.take<X>((size_t)nmax * nmax);    // E, column-major, ld nc
    X *Rinv = keep.take<X>((size_t)ld * ld);      // g x g, ld cmax
    X *Ptx = keep.take<X>((size_t)a.rmax * ld);   // r x g, ld cmax
    unsigned char *work = (gbase ? gbase : smem_raw) + CL.keep;

    // ---- phase A: R2 = chol(G2), M2 = R2^{-1}, R = R2 R1p, Rinv = M1 M2, E
    if (sizeof(J) == 4) {
        // FP32 path.  G2 = W^T W with W = Z M1 nearly orthonormal, so when
        // |G2 - I| < 0.1 on the kept indices, R2 and R2^{-1} come from Newton
        // steps R <- R + T(G2 - R^T R) (T: upper triangle, diagonal halved)
        // and X <- X (2I - R2 X) from I, each step a parallel triangular
        // product; otherwise a double-float Cholesky.  R = R2 R1p and
        // R^{-1} = M1 M2 need only FP32 relative accuracy.
        Carve cv{work};
        X *W = cv.take<X>((size_t)ld * ld);
        X *R2x = cv.take<X>((size_t)ld * ld);
        X *M2x = cv.take<X>((size_t)ld * ld);
        float *Gf = cv.take<float>((size_t)ld * ld);
        float *R2f = cv.take<float>((size_t)ld * ld);
        float *M2f = cv.take<float>((size_t)ld * ld);
        float *T1 = cv.take<float>((size_t)ld * ld);
        float *R1f = cv.take<float>((size_t)ld * ld);
        float *M1f = cv.take<float>((size_t)ld * ld);
        float *Rf = cv.take<float>((size_t)ld * ld);
        float *Rif = cv.take<float>((size_t)ld * ld);
        double dev = 0.0, dmax = 0.0;
        for (int e = tid; e < g * g; e += bd) {
            const int i = e / g, j = e % g;
            const double gij = i <= j ? a.G2[i * ld + j] : a.G2[j * ld + i];
            Gf[i * ld + j] = (float)gij;
            R1f[i * ld + j] = (float)a.R1p[i * ld + j];
            M1f[i * ld + j] = (float)a.M1[i * ld + j];
            const bool kept = a.G2[i * ld + i] != 0.0 && a.G2[j * ld + j] != 0.0;
            if (kept) {
                const double d = fabs(gij - (i == j ? 1.0 : 0.0));
                dev = d > dev ? d : dev;
            }
            if (i == j) dmax = gij > dmax ? gij : dmax;
        }
        for (int e = tid; e < r * g; e += bd) {
            const int l = e / g, j = e % g;
            Ptx[l * ld + j] = XOps<X>::from(a.Ptot[l * ld + j]);
        }
        dev = block_max<double>(dev, red);
        dmax = block_max<double>(dmax, red);
        // Newton steps from I.  For R2 (R <- R + T(G2 - R^T R)) the error
        // contracts by ~2 dev per step (linear), after n steps ~(2 dev)^(n+1);
        // for M2 (X <- X (2I - R2 X)) it squares, ~(2 dev)^(2^n).  Each takes
        // the fewest steps that reach u; beyond dev = 1.5e-2 the double-float
        // Cholesky runs instead.
        int nitR = 0, nitM = 0;
        {
            const double d = 2.0 * dev;
            double pr = d * d, pm = d * d;
            nitR = 1;
            while (pr > u && nitR < 4) { pr *= d; ++nitR; }
            nitM = 1;
            while (pm > u && nitM < 4) { pm *= pm; ++nitM; }
            if (pr > u) nitR = 0;
        }
        if (nitR > 0) {
            const int nit = nitR;
            // step 1 for R2 from R2 = I (on the kept indices): T1 = G2 - I
            for (int e = tid; e < g * g; e += bd) {
                const int i = e / g, j = e % g;
                const bool kept = Gf[i * ld + i] != 0.f && Gf[j * ld + j] != 0.f;
                float v = 0.f;
                if (i <= j && kept) {
                    const float t = Gf[i * ld + j] - (i == j ? 1.f : 0.f);
                    v = (i == j ? 1.f : 0.f) + (i == j ? 0.5f * t : t);
                }
                R2f[i * ld + j] = v;
            }
            __syncthreads();
            for (int it = 1; it < nit; ++it) {
                // T1 = G2 - R2^T R2 (upper part)
                for (int e = tid; e < g * g; e += bd) {
                    const int i = e / g, j = e % g;
                    float v = 0.f;
                    if (i <= j) {
                        float acc = Gf[i * ld + j];
                        for (int l = 0; l <= i; ++l) acc = fmaf(-R2f[l * ld + i], R2f[l * ld + j], acc);
                        v = acc;
                    }
                    T1[i * ld + j] = v;
                }
                __syncthreads();
                for (int e = tid; e < g * g; e += bd) {
                    const int i = e / g, j = e % g;
                    if (i <= j && Gf[i * ld + i] != 0.f && Gf[j * ld + j] != 0.f)
                        R2f[i * ld + j] += (i == j) ? 0.5f * T1[i * ld + j] : T1[i * ld + j];
                }
                __syncthreads();
            }
            // M2 = R2^{-1}: X <- X (2I - R2 X) from X = I (first step 2I - R2),
            // the iterates alternating between M2f and the unused M2x storage
            float *Ma = M2f, *Mb = reinterpret_cast<float *>(M2x);
            for (int e = tid; e < g * g; e += bd) {
                const int i = e / g, j = e % g;
                float v = 0.f;
                if (i <= j) v = (i == j && Gf[i * ld + i] != 0.f ? 2.f : 0.f) - R2f[i * ld + j];
                Ma[i * ld + j] = v;
            }
            __syncthreads();
            for (int it = 1; it < nitM; ++it) {
                // T1 = 2I - R2 Ma ; Mb = Ma T1   (all upper triangular)
                for (int e = tid; e < g * g; e += bd) {
                    const int i = e / g, j = e % g;
                    float v = 0.f;
                    if (i <= j) {
                        float acc = 0.f;
                        for (int l = i; l <= j; ++l) acc = fmaf(R2f[i * ld + l], Ma[l * ld + j], acc);
                        v = (i == j && Gf[i * ld + i] != 0.f ? 2.f : 0.f) - acc;
                    }
                    T1[i * ld + j] = v;
                }
                __syncthreads();
                for (int e = tid; e < g * g; e += bd) {
                    const int i = e / g, j = e % g;
                    float v = 0.f;
                    if (i <= j)
                        for (int l = i; l <= j; ++l) v = fmaf(Ma[i * ld + l], T1[l * ld + j], v);
                    Mb[i * ld + j] = v;
                }
                __syncthreads();
                float *tmp = Ma;
                Ma = Mb;
                Mb = tmp;
            }
            M2f = Ma;
        } else {
            const double eps = nc * u;
            const X thr = XOps<X>::from(eps * eps * dmax);
            for (int e = tid; e < g * g; e += bd) {
                const int i = e / g, j = e % g;
                W[i * ld + j] = XOps<X>::from(i <= j ? a.G2[i * ld + j] : 0.0);
            }
            __syncthreads();
            chol_drop<X>(W, ld, g, thr, R2x, ld, piv3);
            tri_inv<X>(R2x, ld, g, W, ld, M2x, ld, dinv);
            for (int e = tid; e < g * g; e += bd) {
                const int i = e / g, j = e % g;
                R2f[i * ld + j] = x_hi(R2x[i * ld + j]);
                M2f[i * ld + j] = x_hi(M2x[i * ld + j]);
            }
            __syncthreads();
        }
        // R = R2 R1p, Rinv = M1 M2
        for (int e = tid; e < g * g; e += bd) {
            const int i = e / g, j = e % g;
            float v = 0.f, w = 0.f;
            if (i <= j)
                for (int l = i; l <= j; ++l) {
                    v = fmaf(R2f[i * ld + l], R1f[l * ld + j], v);
                    w = fmaf(M1f[i * ld + l], M2f[l * ld + j], w);
                }
            Rf[i * ld + j] = v;
            Rif[i * ld + j] = w;
        }
        __syncthreads();
        // Rinv keeps R2^{-1} alone when the update applies it to the stored W
        for (int e = tid; e < g * g; e += bd) {
            const int i = e / g, j = e % g;
            Rinv[i * ld + j] = XOps<X>::from_f(a.wq ? M2f[i * ld + j] : Rif[i * ld + j]);
        }
        for (int e = tid; e < nc * nc; e += bd) {
            const int q = e / nc, p = e % nc;   // column q, row p
            X v = XOps<X>::zero();
            if (p < r) {
                if (q < r) v = (p == q) ? XOps<X>::from(a.sigma[p]) : XOps<X>::zero();
                else v = Ptx[p * ld + (q - r)];
            } else if (q >= r) {
                v = XOps<X>::from_f(Rf[(p - r) * ld + (q - r)]);
            }
            if (!isfinite(x_hi(v))) s_bad = 1;
            Ex[q * nc + p] = v;
        }
        __syncthreads();
    } else {
        Carve cv{work};
        X *W = cv.take<X>((size_t)ld * ld);
        X *R2 = cv.take<X>((size_t)ld * ld);
        X *M2 = cv.take<X>((size_t)ld * ld);
        X *R1 = cv.take<X>((size_t)ld * ld);
        X *M1 = cv.take<X>((size_t)ld * ld);
        X *Rr = W;   // W is free once M2 is formed
        double dmax = 0.0;
        for (int j = tid; j < g; j += bd) dmax = a.G2[j * ld + j] > dmax ? a.G2[j * ld + j] : dmax;
        dmax = block_max<double>(dmax, red);
        const double eps = nc * u;
        const X thr = XOps<X>::from(eps * eps * dmax);
        for (int e = tid; e < g * g; e += bd) {
            const int i = e / g, j = e % g;
            W[i * ld + j] = XOps<X>::from(i <= j ? a.G2[i * ld + j] : 0.0);
            R1[i * ld + j] = XOps<X>::from(a.R1p[i * ld + j]);
            M1[i * ld + j] = XOps<X>::from(a.M1[i * ld + j]);
        }
        for (int e = tid; e < r * g; e += bd) {
            const int l = e / g, j = e % g;
            Ptx[l * ld + j] = XOps<X>::from(a.Ptot[l * ld + j]);
        }
        __syncthreads();
        chol_drop<X>(W, ld, g, thr, R2, ld, piv3);
        tri_inv<X>(R2, ld, g, W, ld, M2, ld, dinv);
        trmm_upper<X>(R2, ld, R1, ld, g, Rr, ld);     // R = R2 R1p
        if (a.wq) {
            for (int e = tid; e < g * g; e += bd) Rinv[(e / g) * ld + e % g] = M2[(e / g) * ld + e % g];
        } else {
            trmm_upper<X>(M1, ld, M2, ld, g, Rinv, ld);   // Rinv = M1 M2
        }
        for (int e = tid; e < nc * nc; e += bd) {
            const int q = e / nc, p = e % nc;   // column q, row p
            X v = XOps<X>::zero();
            if (p < r) {
                if (q < r) v = (p == q) ? XOps<X>::from(a.sigma[p]) : XOps<X>::zero();
                else v = Ptx[p * ld + (q - r)];
            } else if (q >= r) {
                v = Rr[(p - r) * ld + (q - r)];
            }
            if (!isfinite(x_hi(v))) s_bad = 1;
            Ex[q * nc + p] = v;
        }
        __syncthreads();
    }

    // ---- phase B: Jacobi on the rows of E: B = E^T (column p = row p of E)
    // (wide cores: B, V in shared memory when they fit, else in global scratch)
    Carve cvB{(gbase && a.jac_smem) ? smem_raw : work};
    const bool lean = sizeof(J) == 4 && nmax <= LEAN_MAX;
    const int ldj = lean ? lean_ld(nmax) : nc;   // leading dimension of B and V
    J *B = cvB.take<J>(lean ? (size_t)ldj * nmax : (size_t)nmax * nmax);
    J *V = cvB.take<J>(lean ? (size_t)ldj * nmax : (size_t)nmax * nmax);
    J *alpha = cvB.take<J>(nmax);
    int *order = cvB.take<int>(nmax);
    Carve cv = (gbase && a.jac_smem) ? Carve{work} : cvB;
    X *Vr = cv.take<X>((size_t)nmax * a.rmax);
    X *Q = cv.take<X>((size_t)nmax * a.rmax);
    X *Yt = cv.take<X>((size_t)nmax * a.rmax);
    X *Gb = cv.take<X>((size_t)a.rmax * a.rmax);
    X *Rb = cv.take<X>((size_t)a.rmax * a.rmax);
    X *Mw = cv.take<X>((size_t)a.rmax * a.rmax);
    X *Mb = cv.take<X>((size_t)a.rmax * a.rmax);
    J *Bs = cv.take<J>((size_t)nmax * a.rmax);
    J *BtB = cv.take<J>((size_t)a.rmax * a.rmax);
    J *Psq = cv.take<J>((size_t)a.rmax * a.rmax);
    J *xv = cv.take<J>(a.rmax);
    J *yv = cv.take<J>(a.rmax);
    X *sig = cv.take<X>(a.rmax);
    int *ord2 = cv.take<int>(a.rmax);
    const bool f32 = sizeof(J) == 4;
    // lean path: B scaled by a power of two to max |B_ij| in [1/2, 1), so the
    // FP32 squared norms and their products stay clear of overflow and
    // underflow (rotations and the directions the finish uses are unchanged)
    double jscale = 1.0;
    if (lean) {
        double mx = 0.0;
        for (int e = tid; e < nc * nc; e += bd) mx = fmax(mx, fabs((double)x_hi(Ex[e])));
        mx = block_max<double>(mx, red);
        if (mx > 0.0 && isfinite(mx)) {
            int ex;
            frexp(mx, &ex);
            jscale = ldexp(1.0, -ex);
        }
    }
    for (int e = tid; e < nc * ldj; e += bd) {
        const int col = e / ldj, i = e % ldj;   // B column col = row col of E; entry i = E[col][i]
        J v = (J)0;
        if (i < nc) v = f32 ? (J)((double)x_hi(Ex[i * nc + col]) * jscale) : (J)XOps<X>::to(Ex[i * nc + col]);
        B[col * ldj + i] = v;
        V[col * ldj + i] = (i == col) ? (J)1 : (J)0;
    }
    __syncthreads();
    const J eps_j = f32 ? (J)1.1920928955078125e-07 : (J)2.220446049250313e-16;
    // FP64: n eps, above the rounding error of the computed b_p . b_q, so
    // that the sweeps end; FP32: the double-float finish below carries the
    // accuracy and a tighter rotation threshold pays off
    const J tol = f32 ? (J)2 * sqrt((J)nc) * eps_j : (J)nc * eps_j;
    clk[1] = clock64();
    if (tid == 0) s_flag[1] = 0;
    int nsweeps;
    if constexpr (sizeof(J) == 4) {
        if (lean) {
            float *Bf = reinterpret_cast<float *>(B), *Vf = reinterpret_cast<float *>(V);
            float *af = reinterpret_cast<float *>(alpha);
            const float tf = (float)tol;
            const int keep = a.wq ? (a.r < nc ? a.r : nc) : 0;
            switch (ldj) {
                case 64:
                    nsweeps = a.tape ? jacobi_lean<true, 64>(Bf, nc, Vf, af, tf, 20, s_flag)
                                     : jacobi_lean<false, 64>(Bf, nc, Vf, af, tf, 20, s_flag, keep);
                    break;
                case 96:
                    nsweeps = a.tape ? jacobi_lean<true, 96>(Bf, nc, Vf, af, tf, 20, s_flag)
                                     : jacobi_lean<false, 96>(Bf, nc, Vf, af, tf, 20, s_flag, keep);
                    break;
                case 128:
                    nsweeps = a.tape ? jacobi_lean<true, 128>(Bf, nc, Vf, af, tf, 20, s_flag)
                                     : jacobi_lean<false, 128>(Bf, nc, Vf, af, tf, 20, s_flag, keep);
                    break;
                default:
                    nsweeps = a.tape ? jacobi_lean<true, 160>(Bf, nc, Vf, af, tf, 20, s_flag)
                                     : jacobi_lean<false, 160>(Bf, nc, Vf, af, tf, 20, s_flag, keep);
                    break;
            }
        } else {
            nsweeps = jacobi_hw<J>(B, nc, nc, nc, V, nc, alpha, tol, 20, s_flag);
        }
    } else {
        nsweeps = jacobi_hw<J>(B, nc, nc, nc, V, nc, alpha, tol, 30, s_flag);
    }
    __syncthreads();
    clk[2] = clock64();
    sort_desc<J>(alpha, nc, order);
    const int rsel = a.r < nc ? a.r : nc;

    // ---- phase C: top-r left vectors of E and singular values
    if (f32) {
        // The rotated rows b_s = E^T v_s = sigma_s w_s give the left vectors
        // u_s = E b_s / sigma_s^2 (a power step that damps the FP32 rotation
        // error of direction j by sigma_j / sigma_s).  Vr_s = E b_s in
        // double-float, orthonormalised by CholeskyQR (leading spans kept);
        // then sigma_s = |E^T q_s| (Rayleigh quotient).
        // E is upper triangular (diag(Sigma) and P in its first r rows, R in
        // the rest): row p < r holds sigma_p at column p and P at columns >= r,
        // row p >= r holds R at columns >= p
        for (int e = tid; e < nc * rsel; e += bd) {
            const int s = e / nc, p = e % nc;
            const J *bs = B + (size_t)order[s] * ldj;
            Acc<X> a0, a1;
            if (p < r) a0.add(Ex[p * nc + p], XOps<X>::from_f((float)bs[p]));
            int j = p < r ? r : p;
            for (; j + 1 < nc; j += 2) {
                a0.add(Ex[j * nc + p], XOps<X>::from_f((float)bs[j]));
                a1.add(Ex[(j + 1) * nc + p], XOps<X>::from_f((float)bs[j + 1]));
            }
            if (j < nc) a0.add(Ex[j * nc + p], XOps<X>::from_f((float)bs[j]));
            Vr[s * nc + p] = a0.get() + a1.get();
        }
        __syncthreads();
        // Vr transposed into Yt (free until the Rayleigh products), so that
        // the threads of a warp (consecutive j) read consecutive entries
        X *VrT = Yt;
        for (int e = tid; e < nc * rsel; e += bd) {
            const int s2 = e / nc, p = e % nc;
            VrT[p * rsel + s2] = Vr[e];
        }
        __syncthreads();
        const int rm = a.rmax;
        for (int e = tid; e < rsel * rsel; e += bd) {
            const int i = e / rsel, j = e % rsel;
            Acc<X> a0, a1;
            if (i <= j) {
                int p = 0;
                for (; p + 1 < nc; p += 2) {
                    a0.add(VrT[p * rsel + i], VrT[p * rsel + j]);
                    a1.add(VrT[(p + 1) * rsel + i], VrT[(p + 1) * rsel + j]);
                }
                if (p < nc) a0.add(VrT[p * rsel + i], VrT[p * rsel + j]);
            }
            Gb[i * rm + j] = a0.get() + a1.get();
        }
        __syncthreads();
        // CholeskyQR of Vr.  Its columns are nearly orthogonal (the rotated
        // rows' couplings are below the Jacobi threshold and the power step
        // only damps them), so with D = diag(Gb) and Gs = D^{-1/2} Gb D^{-1/2}
        // = I + F the factor Rs of Gs and Rs^{-1} come from Newton steps from
        // I, as in phase A, to the double-float unit (2^-44); a larger |F|
        // takes the Cholesky.  Mb = D^{-1/2} Rs^{-1}, so Q = Vr Mb.
        double fm = 0.0;
        for (int e = tid; e < rsel * rsel; e += bd) {
            const int i = e / rsel, j = e % rsel;
            if (i < j) {
                const double di = XOps<X>::to(Gb[i * rm + i]), dj = XOps<X>::to(Gb[j * rm + j]);
                if (di > 1e-60 && dj > 1e-60) fm = fmax(fm, fabs(XOps<X>::to(Gb[i * rm + j])) / sqrt(di * dj));
            }
        }
        for (int i = tid; i < rsel; i += bd) {
            const X d = Gb[i * rm + i];
            dinv[i] = XOps<X>::to(d) > 1e-60 ? XOps<X>::one() / XOps<X>::sqrt_(d) : XOps<X>::zero();
        }
        fm = block_max<double>(fm, red);
        const double ud = 5.684341886080802e-14;   // 2^-44
        int nR = 0, nM = 0;
        {
            const double d = 2.0 * fm;
            double pr = d * d, pm = d * d;
            nR = 1;
            while (pr > ud && nR < 4) { pr *= d; ++nR; }
            nM = 1;
            while (pm > ud && nM < 4) { pm *= pm; ++nM; }
            if (pr > ud) nR = 0;
        }
        if (nR > 0) {
            auto kept = [&](int i) { return x_hi(dinv[i]) != 0.f; };
            for (int e = tid; e < rsel * rsel; e += bd) {
                const int i = e / rsel, j = e % rsel;
                if (i <= j) Gb[i * rm + j] = kept(i) && kept(j) ? Gb[i * rm + j] * dinv[i] * dinv[j] : XOps<X>::zero();
            }
            __syncthreads();
            // Rs = I + T(Gs - I), then Rs <- Rs + T(Gs - Rs^T Rs)
            for (int e = tid; e < rsel * rsel; e += bd) {
                const int i = e / rsel, j = e % rsel;
                X v = XOps<X>::zero();
                if (i <= j && kept(i) && kept(j)) {
                    const X t = Gb[i * rm + j] - (i == j ? XOps<X>::one() : XOps<X>::zero());
                    v = i == j ? XOps<X>::one() + t * XOps<X>::from(0.5) : t;
                }
                Rb[i * rm + j] = v;
            }
            __syncthreads();
            for (int it = 1; it < nR; ++it) {
                for (int e = tid; e < rsel * rsel; e += bd) {
                    const int i = e / rsel, j = e % rsel;
                    X v = XOps<X>::zero();
                    if (i <= j) {
                        v = Gb[i * rm + j];
                        for (int l = 0; l <= i; ++l) v = v - Rb[l * rm + i] * Rb[l * rm + j];
                    }
                    Mw[i * rm + j] = v;
                }
                __syncthreads();
                for (int e = tid; e < rsel * rsel; e += bd) {
                    const int i = e / rsel, j = e % rsel;
                    if (i <= j && kept(i) && kept(j))
                        Rb[i * rm + j] = Rb[i * rm + j] + (i == j ? Mw[i * rm + j] * XOps<X>::from(0.5) : Mw[i * rm + j]);
                }
                __syncthreads();
            }
            // Rs^{-1}: X <- X (2I - Rs X) from X = I, alternating Mb / Gb
            X *Ma = Mb, *Mc = Gb;
            for (int e = tid; e < rsel * rsel; e += bd) {
                const int i = e / rsel, j = e % rsel;
                X v = XOps<X>::zero();
                if (i <= j) v = (i == j && kept(i) ? XOps<X>::from(2.0) : XOps<X>::zero()) - Rb[i * rm + j];
                Ma[i * rm + j] = v;
            }
            __syncthreads();
            for (int it = 1; it < nM; ++it) {
                for (int e = tid; e < rsel * rsel; e += bd) {
                    const int i = e / rsel, j = e % rsel;
                    X v = XOps<X>::zero();
                    if (i <= j) {
                        X acc = XOps<X>::zero();
                        for (int l = i; l <= j; ++l) acc = acc + Rb[i * rm + l] * Ma[l * rm + j];
                        v = (i == j && kept(i) ? XOps<X>::from(2.0) : XOps<X>::zero()) - acc;
                    }
                    Mw[i * rm + j] = v;
                }
                __syncthreads();
                for (int e = tid; e < rsel * rsel; e += bd) {
                    const int i = e / rsel, j = e % rsel;
                    X v = XOps<X>::zero();
                    if (i <= j)
                        for (int l = i; l <= j; ++l) v = v + Ma[i * rm + l] * Mw[l * rm + j];
                    Mc[i * rm + j] = v;
                }
                __syncthreads();
                X *tmp = Ma;
                Ma = Mc;
                Mc = tmp;
            }
            for (int e = tid; e < rsel * rsel; e += bd) {
                const int i = e / rsel, j = e % rsel;
                Mb[i * rm + j] = i <= j ? dinv[i] * Ma[i * rm + j] : XOps<X>::zero();
            }
            __syncthreads();
        } else {
            chol_drop<X>(Gb, rm, rsel, XOps<X>::from(1e-60), Rb, rm, piv3);
            tri_inv<X>(Rb, rm, rsel, Mw, rm, Mb, rm, dinv);
        }
        for (int e = tid; e < nc * rsel; e += bd) {
            const int s = e / nc, p = e % nc;
            Acc<X> a0, a1;
            int l = 0;
            for (; l + 1 <= s; l += 2) {
                a0.add(Vr[l * nc + p], Mb[l * a.rmax + s]);
                a1.add(Vr[(l + 1) * nc + p], Mb[(l + 1) * a.rmax + s]);
            }
            if (l <= s) a0.add(Vr[l * nc + p], Mb[l * a.rmax + s]);
            Q[s * nc + p] = a0.get() + a1.get();
        }
        __syncthreads();
        // Q transposed into Vr (no longer read): the threads of a warp take
        // consecutive s of one column j of E (one broadcast E entry, Q
        // entries side by side)
        X *QT = Vr;
        for (int e = tid; e < nc * rsel; e += bd) {
            const int s2 = e / nc, p = e % nc;
            QT[p * rsel + s2] = Q[e];
        }
        __syncthreads();
        for (int e = tid; e < nc * rsel; e += bd) {
            const int j = e / rsel, s = e % rsel;
            // column j of E: sigma_j alone for j < r, rows 0..j otherwise
            X acc = XOps<X>::zero();
            if (j < r) {
                acc = Ex[j * nc + j] * QT[j * rsel + s];
            } else {
                Acc<X> a0, a1;
                int p = 0;
                for (; p + 1 <= j; p += 2) {
                    a0.add(Ex[j * nc + p], QT[p * rsel + s]);
                    a1.add(Ex[j * nc + p + 1], QT[(p + 1) * rsel + s]);
                }
                if (p <= j) a0.add(Ex[j * nc + p], QT[p * rsel + s]);
                acc = a0.get() + a1.get();
            }
            Yt[s * nc + j] = acc;
        }
        __syncthreads();
        for (int s = tid; s < rsel; s += bd) {
            X acc = XOps<X>::zero();
            for (int j = 0; j < nc; ++j) acc = acc + Yt[s * nc + j] * Yt[s * nc + j];
            sig[s] = XOps<X>::sqrt_(acc);
        }
        __syncthreads();
        sort_desc<X>(sig, rsel, ord2);
        for (int e = tid; e < nc * rsel; e += bd) {
            const int s = e / nc, p = e % nc;
            Vr[s * nc + p] = Q[ord2[s] * nc + p];
        }
        for (int s = tid; s < rsel; s += bd) Yt[s] = sig[ord2[s]];
        __syncthreads();
        for (int e = tid; e < nc * rsel; e += bd) Q[e] = Vr[e];
        for (int s = tid; s < rsel; s += bd) sig[s] = Yt[s];
        __syncthreads();
    } else {
        for (int e = tid; e < nc * rsel; e += bd) {
            const int s = e / nc, p = e % nc;
            Q[s * nc + p] = XOps<X>::from((double)V[order[s] * ldj + p]);
        }
        for (int s = tid; s < rsel; s += bd) sig[s] = XOps<X>::from(sqrt((double)alpha[order[s]]));
        __syncthreads();
    }
    clk[3] = clock64();
    // truncation: keep min(r, #sigma > nc u sigma_1)
    if (tid == 0) {
        const double s0 = rsel > 0 ? XOps<X>::to(sig[0]) : 0.0;
        const double thr = nc * u * s0;
        int keepn = 0;
        for (int s = 0; s < rsel; ++s)
            if (XOps<X>::to(sig[s]) > thr) ++keepn;
        if (!isfinite(s0)) s_bad = 1;
        s_rnew = keepn;
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
                Bs[p * k + cidx] = (J)XOps<X>::to(Q[cidx * nc + k + p]);   // B row by row
            }
            __syncthreads();
            // P^2 goes to Bs once B^T B is formed (B is no longer read then)
            const double smax = top_singular_value<J>(Bs, nr, k, BtB, Psq, Bs, xv, yv, red);
            if (tid == 0) {
                s_sin = smax;
                s_measure = smax;
            }
        } else {
            double mn = 1e300;
            for (int i = tid; i < k; i += bd) {
                double c = fabs(XOps<X>::to(Q[i * nc + i]));
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
    clk[4] = clock64();
    if (a.tape && a.tape->core && t < a.tape->cap) {
        // merge record for the adjoint: sizes, every singular value and left
        // vector of E (refined ones for the first rsel), E, Ptot, R^{-1}
        const TapeLayout TL = tape_layout(a.rmax, a.cmax);
        double *tp = a.tape->core + (int64_t)t * TL.stride;
        if (tid == 0) {
            tp[0] = r;
            tp[1] = g;
            tp[2] = rn;
            tp[3] = nc;
        }
        for (int s = tid; s < nc; s += bd)
            tp[TL.sig + s] = s < rsel ? XOps<X>::to(sig[s]) : sqrt((double)alpha[order[s]]) / jscale;
        for (int e = tid; e < nc * nc; e += bd) {
            const int q = e / nc, p = e % nc;
            tp[TL.E + (int64_t)q * nmax + p] = XOps<X>::to(Ex[q * nc + p]);
            tp[TL.UE + (int64_t)q * nmax + p] =
                q < rsel ? XOps<X>::to(Q[q * nc + p]) : (double)V[(size_t)order[q] * ldj + p];
        }
        for (int e = tid; e < r * g; e += bd) {
            const int l = e / g, j = e % g;
            tp[TL.Ptot + l * ld + j] = XOps<X>::to(Ptx[l * ld + j]);
        }
        for (int e = tid; e < g * g; e += bd) {
            const int i = e / g, j = e % g;
            double v = 0.0;
            if (!a.wq) {
                v = XOps<X>::to(Rinv[i * ld + j]);
            } else if (i <= j) {   // R^{-1} = M1 R2^{-1}
                for (int l = i; l <= j; ++l) v = fma(a.M1[i * ld + l], XOps<X>::to(Rinv[l * ld + j]), v);
            }
            tp[TL.Rinv + i * ld + j] = v;
        }
    }
    // wq: Y = R2^{-1} U_E[r:, :rn], X = U_E[:r, :rn]; otherwise
    // Y = R^{-1} U_E[r:, :rn] (g x rn), X = U_E[:r, :rn] - Ptot Y (r x rn)
    // (Q transposed into Vr, free here: the threads of a warp, consecutive
    // q, read consecutive entries)
    X *QTc = Vr;
    for (int e = tid; e < nc * rsel; e += bd) {
        const int s2 = e / nc, p = e % nc;
        QTc[p * rsel + s2] = Q[e];
    }
    __syncthreads();
    for (int e = tid; e < g * rn; e += bd) {
        const int j = e / rn, q = e % rn;
        X acc = XOps<X>::zero();
        for (int l = j; l < g; ++l) acc = acc + Rinv[j * ld + l] * QTc[(r + l) * rsel + q];
        Yt[j * a.rmax + q] = acc;
    }
    __syncthreads();
    for (int e = tid; e < g * rn; e += bd) {
        const int j = e / rn, q = e % rn;
        a.Ym[j * a.rmax + q] = XOps<X>::to(Yt[j * a.rmax + q]);
    }
    for (int e = tid; e < r * rn; e += bd) {
        const int l = e / rn, q = e % rn;
        X acc = QTc[l * rsel + q];
        if (!a.wq)
            for (int j = 0; j < g; ++j) acc = acc - Ptx[l * ld + j] * Yt[j * a.rmax + q];
        a.Xm[l * a.rmax + q] = XOps<X>::to(acc);
    }
    for (int s = tid; s < rn; s += bd) a.sigma[s] = XOps<X>::to(sig[s]);
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
        st->sweeps = nsweeps;
        clk[5] = clock64();
        for (int i = 0; i < 5; ++i) st->core_cycles[i] = clk[i + 1] - clk[i];
        st->core_cycles[5] = clk[5] - clk[0];
    }
}

pod_status launch_core(const SmallArgs &a, cudaStream_t s) {
    const bool f64 = a.core_f64 || a.dtype == POD_F64;
    size_t smem = core_smem_bytes(a.rmax, a.cmax, f64 ? POD_F64 : POD_F32);
    if (a.gws_core) smem = a.jac_smem ? core_jacobi_bytes(a.rmax, a.cmax, f64 ? POD_F64 : POD_F32) : 64;
    if (smem > 220 * 1024) return POD_EUNSUPPORTED;
    if (!f64) {
        POD_CUDA_TRY(cudaFuncSetAttribute(k_core<dfloat, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_core<dfloat, float><<<1, CORE_THREADS, smem, s>>>(a);
    } else {
        POD_CUDA_TRY(cudaFuncSetAttribute(k_core<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_core<double, double><<<1, CORE_THREADS, smem, s>>>(a);
    }
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}


// ---------------------------------------------------------------------------
// Refinement (closing lines of Algorithm 1): with Y = A^T U (n x r),
// CholeskyQR2 gives Y = Q R; SVD(R) = U_R S_R V_R^T by one-sided Jacobi in
// FP64 on the columns of R with accumulated V_R; outputs sigma = S_R,
// VR (U <- U V_R) and K = R^{-1} U_R (V <- Y K = Q U_R).  One CTA.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(CHOL_THREADS) k_refine_chol(RefineArgs a) {
    const int r = a.r;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Carve cv{a.gws ? a.gws : smem_raw};
    double *W = cv.take<double>((size_t)r * r);
    double *R = cv.take<double>((size_t)r * r);
    double *Mw = cv.take<double>((size_t)r * r);
    double *M = cv.take<double>((size_t)r * r);
    __shared__ double red[32];
    __shared__ double piv3[3];
    __shared__ double dinv[256];
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
    chol_drop<double>(W, r, r, eps * eps * dmax, R, r, piv3);
    tri_inv<double>(R, r, r, Mw, r, M, r, dinv);
    for (int e = tid; e < r * r; e += bd) {
        a.M1[e] = M[e];
        a.R1p[e] = R[e];
    }
}

__global__ void __launch_bounds__(CORE_THREADS) k_refine_svd(RefineArgs a) {
    const int r = a.r;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Carve cv{a.gws ? a.gws : smem_raw};
    double *W = cv.take<double>((size_t)r * r);
    double *R2 = cv.take<double>((size_t)r * r);
    double *M2 = cv.take<double>((size_t)r * r);
    double *R1 = cv.take<double>((size_t)r * r);
    double *Rr = cv.take<double>((size_t)r * r);   // R = R2 R1
    double *Mi = cv.take<double>((size_t)r * r);   // R^{-1} = M1 M2
    double *B = cv.take<double>((size_t)r * r);
    double *V = cv.take<double>((size_t)r * r);
    double *alpha = cv.take<double>(r);
    int *order = cv.take<int>(r);
    __shared__ int s_flag[2];
    __shared__ double red[32];
    __shared__ double piv3[3];
    __shared__ double dinv[256];
    const int tid = threadIdx.x, bd = blockDim.x;
    if (tid == 0) s_flag[1] = 0;
    double dmax = 0.0;
    for (int j = tid; j < r; j += bd) dmax = a.G2[j * r + j] > dmax ? a.G2[j * r + j] : dmax;
    dmax = block_max<double>(dmax, red);
    for (int e = tid; e < r * r; e += bd) {
        const int i = e / r, j = e % r;
        W[e] = i <= j ? a.G2[i * r + j] : 0.0;
        R1[e] = a.R1p[e];
        Mi[e] = a.M1[e];
    }
    __syncthreads();
    const double eps = r * 1.1102230246251565e-16;
    chol_drop<double>(W, r, r, eps * eps * dmax, R2, r, piv3);
    tri_inv<double>(R2, r, r, W, r, M2, r, dinv);
    trmm_upper<double>(R2, r, R1, r, r, Rr, r);
    trmm_upper<double>(Mi, r, M2, r, r, W, r);   // W <- R^{-1}
    for (int e = tid; e < r * r; e += bd) {
        const int q = e / r, p = e % r;   // B column-major: column q of R
        B[q * r + p] = Rr[p * r + q];
        V[q * r + p] = (p == q) ? 1.0 : 0.0;
    }
    __syncthreads();
    // threshold n eps: above the rounding error of the computed dot products
    jacobi_hw<double>(B, r, r, r, V, r, alpha, (double)r * 2.220446049250313e-16, 40, s_flag);
    __syncthreads();
    sort_desc<double>(alpha, r, order);
    // sigma_s, V_R[:, s], U_R[:, s] = B[:, order[s]] / sigma_s, K = R^{-1} U_R
    for (int s = tid; s < r; s += bd) a.sigma[s] = sqrt(alpha[order[s]]);
    for (int e = tid; e < r * r; e += bd) {
        const int l = e / r, s = e % r;
        a.VR[l * r + s] = V[order[s] * r + l];
    }
    for (int e = tid; e < r * r; e += bd) {
        const int j = e / r, s = e % r;
        const double sg = sqrt(alpha[order[s]]);
        double acc = 0.0;
        if (sg > 0.0)
            for (int l = j; l < r; ++l) acc += W[j * r + l] * B[order[s] * r + l] / sg;
        a.K[j * r + s] = acc;
    }
}

// ---------------------------------------------------------------------------
// ICRS (Algorithm 1, GET UPDATE with rows): the top right singular vectors
// V_r of the scaled row block W are the top eigenvectors of G_W = W^T W
// (g x g, FP64, ld cmax).  A Cholesky factorisation of the index-reversed
// Gram, J G_W J = R^T R (J the reversal), gives the upper triangular
// R_hat = J R^T J with G_W = R_hat R_hat^T, so the left singular vectors of
// R_hat are the wanted eigenvectors: the core SVD kernel (k_core) computes
// them as the merge of the block R_hat into an empty basis.  Its inputs are
// set up here: R1p = R_hat, G2 = I (second CholeskyQR factor R2 = I) and
// M1 = I, so that the core's block-coefficient output Y = R^{-1} U_E is U_E
// itself, and the state stc = {r_cur 0, g}.
// ---------------------------------------------------------------------------
template <typename X>
__global__ void __launch_bounds__(CHOL_THREADS) k_rows_chol(RowsSmallArgs a) {
    DevState *st = a.st;
    const int g = st->g, done = st->done, t = st->t;
    const int tid = threadIdx.x, bd = blockDim.x;
    if (tid == 0) {
        DevState s{};
        s.done = done;
        s.t = t;
        s.r_cur = 0;
        s.g = g;
        s.remaining = st->remaining;
        *a.stc = s;
    }
    if (done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Carve cv{smem_raw};
    X *W = cv.take<X>((size_t)g * g);
    X *R = cv.take<X>((size_t)g * g);
    __shared__ double red[32];
    __shared__ X piv3[3];
    const int cm = a.cmax;
    double dmax = 0.0;
    for (int j = tid; j < g; j += bd) dmax = a.GW[j * cm + j] > dmax ? a.GW[j * cm + j] : dmax;
    dmax = block_max<double>(dmax, red);
    for (int e = tid; e < g * g; e += bd) {
        const int i = e / g, j = e % g;   // reversed indices: (i, j) <- (g-1-j, g-1-i), upper part
        W[e] = XOps<X>::from(i <= j ? a.GW[(g - 1 - j) * cm + (g - 1 - i)] : 0.0);
    }
    __syncthreads();
    const double eps = g * unit_roundoff(a.dtype);
    chol_drop<X>(W, g, g, XOps<X>::from(eps * eps * dmax), R, g, piv3);
    for (int e = tid; e < g * g; e += bd) {
        const int i = e / g, j = e % g;
        a.R1p[i * cm + j] = i <= j ? XOps<X>::to(R[(g - 1 - j) * g + (g - 1 - i)]) : 0.0;
        a.G2[i * cm + j] = i == j ? 1.0 : 0.0;
        a.M1[i * cm + j] = i == j ? 1.0 : 0.0;
    }
}

// End of the ICRS block step: the round's block width becomes the number of
// kept right vectors; a non-finite value seen by the core is reported.
__global__ void k_rows_setg(DevState *st, const DevState *stc) {
    if (threadIdx.x != 0 || st->done) return;
    st->g = stc->r_new;
    if (stc->status != 0) st->status = stc->status;
}

size_t rows_small_smem(int cmax) { return 2 * al16x((size_t)cmax * cmax * 8) + 64; }

pod_status launch_rows_chol(const RowsSmallArgs &a, cudaStream_t s) {
    const size_t smem = rows_small_smem(a.cmax);
    if (smem > 220 * 1024) return POD_EUNSUPPORTED;
    if (a.dtype == POD_F32 && !a.core_f64) {
        POD_CUDA_TRY(cudaFuncSetAttribute(k_rows_chol<dfloat>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_rows_chol<dfloat><<<1, CHOL_THREADS, smem, s>>>(a);
    } else {
        POD_CUDA_TRY(cudaFuncSetAttribute(k_rows_chol<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_rows_chol<double><<<1, CHOL_THREADS, smem, s>>>(a);
    }
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}

pod_status launch_rows_setg(DevState *st, const DevState *stc, cudaStream_t s) {
    k_rows_setg<<<1, 32, 0, s>>>(st, stc);
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}

size_t refine_gws_bytes(int r) {
    return 8 * al16x((size_t)r * r * 8) + al16x((size_t)r * 8) + al16x((size_t)r * 4) + 64;
}

pod_status launch_refine_chol(const RefineArgs &a, cudaStream_t s) {
    const size_t smem = a.gws ? 64 : 4 * al16x((size_t)a.r * a.r * 8) + 64;
    if (smem > 220 * 1024) return POD_EUNSUPPORTED;
    POD_CUDA_TRY(cudaFuncSetAttribute(k_refine_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_refine_chol<<<1, CHOL_THREADS, smem, s>>>(a);
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}

pod_status launch_refine_svd(const RefineArgs &a, cudaStream_t s) {
    const size_t smem = a.gws ? 64 : 8 * al16x((size_t)a.r * a.r * 8) + al16x((size_t)a.r * 8) + al16x((size_t)a.r * 4) + 64;
    if (smem > 220 * 1024) return POD_EUNSUPPORTED;
    POD_CUDA_TRY(cudaFuncSetAttribute(k_refine_svd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_refine_svd<<<1, CORE_THREADS, smem, s>>>(a);
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}
