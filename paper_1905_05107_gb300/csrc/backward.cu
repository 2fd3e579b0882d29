// Adjoint of the truncated POD computed by ISMA with the draws of the
// forward run held fixed (pod_backward).
//
// Round t of Algorithm 1 maps (U_t, Sigma_t, A) to (U_{t+1}, Sigma_{t+1}): with
// X = [U_t Sigma_t, C_t] (C_t = A[:, I_t]) and its thin SVD X = U~ S~ V~^T,
// U_{t+1} = U~[:, :r'], Sigma_{t+1} = S~[:r'] (Algorithm 2 with the direct merge,
// Eqs. 8-9).  In the implicit form of the forward, U~ = [U_t, C_t] T_c with
// T_c = [[U_E[:r] - Ptot R^{-1} U_E[r:]], [R^{-1} U_E[r:]]] and V~ = V_E =
// E^T U_E S~^{-1}.  The SVD adjoint (no V~ output) is
//   Xbar = U~ [(F o (J - J^T)) S~ + diag(sbar)] V~^T + (I - U~ U~^T) Ubar S~^{-1} V~^T,
// J = U~^T Ubar, F_ij = 1 / (s_j^2 - s_i^2) (broadened near degeneracy), with
// Ubar, sbar extended by zeros beyond r'.  Then Ubar_t = Xbar[:, :r] Sigma_t,
// sbar_t,i = u_t,i^T Xbar[:, i] and Cbar_t = Xbar[:, r:] adds into dA[:, I_t].
// Everything m-long is expressed as row mixes of [U_t, C_t, Ubar] with small
// coefficient matrices; the Gram [U_t, C_t]^T [U_t, C_t, Ubar] gives J and
// sbar_t.  The closing refinement (SVD of B = U_T^T A: U_fin = U_T V_R) adds
// dA += U_fin M_B K^T Y^T and Ubar_T = (Ubar_fin + A Y K M_B^T) V_R^T, with
// M_B = (F o (J_B - J_B^T)) S + diag(sbar), J_B = U_fin^T Ubar_fin, Y = A^T U_T.
#include "pod_internal.h"

namespace {

constexpr int BT = 256;

// --------------------------------------------------------------- tape copy
template <typename T>
__global__ void k_tape_u(const TapePtrs *tp, const DevState *st, const T *U, int64_t m, int rmax) {
    if (st->done) return;
    const int t = st->t, r = st->r_cur;
    if (!tp->U || t >= tp->cap || r <= 0) return;
    T *dst = reinterpret_cast<T *>(tp->U) + (int64_t)t * m * rmax;
    const int64_t total = m * r;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = U[e];
}

// ------------------------------------------- Gram of up to three column blocks
// G = [blocks < nleft]^T [all blocks], compensated sums (TwoProduct + TwoSum)
// for FP32 data, FP64 FMAs for FP64 data; per-CTA partials summed in a fixed
// order (tall_reduce).  Output row-major (nl x nt).
template <typename T>
__global__ void __launch_bounds__(BT) k_bwd_gram(BwdGram a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Ws = reinterpret_cast<T *>(smem_raw);
    __shared__ int s_flag;
    int nt = 0, nl = 0;
    for (int b = 0; b < 3; ++b) {
        nt += a.ncol[b];
        if (b < a.nleft) nl += a.ncol[b];
    }
    const int rp = a.rows_per, lds = a.lds;
    const int64_t r0 = (int64_t)blockIdx.x * rp;
    const int nr = (int)max((int64_t)0, min((int64_t)rp, a.m - r0));
    int cbase = 0;
    for (int b = 0; b < 3; ++b) {
        const T *p = reinterpret_cast<const T *>(a.ptr[b]);
        for (int e = threadIdx.x; e < nr * a.ncol[b]; e += blockDim.x) {
            const int j = e / nr, l = e - j * nr;
            const int64_t col = a.idx[b] ? (int64_t)a.idx[b][j] : (int64_t)j;
            Ws[(cbase + j) * lds + l] = p[col * a.ld[b] + r0 + l];
        }
        cbase += a.ncol[b];
    }
    __syncthreads();
    double *out = a.part + (int64_t)blockIdx.x * nl * nt;
    for (int e = threadIdx.x; e < nl * nt; e += blockDim.x) {
        const int i = e / nt, j = e - i * nt;
        const T *x = Ws + i * lds, *y = Ws + j * lds;
        double v;
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
        out[e] = v;
    }
    tall_reduce(a.part, a.gsum, a.out, nl * nt, (int64_t)nl * nt, a.counters, &s_flag);
}

// ------------------------------------------------------- row mix of blocks
// out_o[i, q] (+)= sum_b sum_l in_b[i, l] coef[(l_b + l) * qtot + (q_o + q)]
template <typename T>
__global__ void __launch_bounds__(BT) k_rowmix(RowMix a) {
    constexpr int RT = 64;   // rows per CTA
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int ptot = 0, qtot = 0;
    for (int b = 0; b < 3; ++b) ptot += a.pin[b];
    for (int o = 0; o < 2; ++o) qtot += a.qout[o];
    T *tile = reinterpret_cast<T *>(smem_raw);          // ptot x RT
    T *cf = tile + (size_t)ptot * RT;                    // ptot x qtot
    const int64_t i0 = (int64_t)blockIdx.x * RT;
    const int nr = (int)min((int64_t)RT, a.m - i0);
    int cb = 0;
    for (int b = 0; b < 3; ++b) {
        const T *p = reinterpret_cast<const T *>(a.in[b]);
        for (int e = threadIdx.x; e < a.pin[b] * RT; e += blockDim.x) {
            const int j = e / RT, l = e - j * RT;
            T v = (T)0;
            if (l < nr) {
                const int64_t col = a.idx_in[b] ? (int64_t)a.idx_in[b][j] : (int64_t)j;
                v = p[col * a.ldi[b] + i0 + l];
            }
            tile[(cb + j) * RT + l] = v;
        }
        cb += a.pin[b];
    }
    for (int e = threadIdx.x; e < ptot * qtot; e += blockDim.x) cf[e] = (T)a.coef[e];
    __syncthreads();
    const int row = threadIdx.x % RT, grp = threadIdx.x / RT, ngrp = blockDim.x / RT;
    if (row >= nr) return;
    int qb = 0;
    for (int o = 0; o < 2; ++o) {
        T *po = reinterpret_cast<T *>(a.out[o]);
        for (int q = grp; q < a.qout[o]; q += ngrp) {
            T acc = (T)0;
            for (int l = 0; l < ptot; ++l) acc = fma(tile[l * RT + row], cf[l * qtot + qb + q], acc);
            const int64_t col = a.idx_out[o] ? (int64_t)a.idx_out[o][q] : (int64_t)q;
            T *dst = po + col * a.ldo[o] + i0 + row;
            *dst = a.acc_out[o] ? *dst + acc : acc;
        }
        qb += a.qout[o];
    }
}

// ------------------------------------------------------------------ A Y
// out (m x r, ld m) = A Y with Y n x r FP64 (ld n); A rows streamed once per
// pass of up to 32 columns of Y, products accumulated in double-float.
template <typename T>
__global__ void __launch_bounds__(BT) k_az(const T *__restrict__ A, int64_t m, int64_t n, int64_t lda,
                                          const double *__restrict__ Y, int r, int l0, T *__restrict__ out) {
    constexpr int CH = 128, KB = 32;
    __shared__ float2 ys[CH * KB];
    const int64_t i = (int64_t)blockIdx.x * BT + threadIdx.x;
    const bool row = i < m;
    const int kb = r - l0 < KB ? r - l0 : KB;
    float ahi[KB], alo[KB];
    double ad[KB];
#pragma unroll
    for (int l = 0; l < KB; ++l) {
        ahi[l] = alo[l] = 0.f;
        ad[l] = 0.0;
    }
    for (int64_t j0 = 0; j0 < n; j0 += CH) {
        const int nch = (int)(n - j0 < CH ? n - j0 : CH);
        __syncthreads();
        for (int e = threadIdx.x; e < nch * KB; e += BT) {
            const int c = e / KB, l = e - c * KB;
            float2 v = make_float2(0.f, 0.f);
            if (l < kb) {
                const double d = Y[(int64_t)(l0 + l) * n + j0 + c];
                v.x = (float)d;
                v.y = (float)(d - (double)v.x);
            }
            ys[e] = v;
        }
        __syncthreads();
        if (!row) continue;
        for (int c = 0; c < nch; ++c) {
            const T x = A[(j0 + c) * lda + i];
            if constexpr (sizeof(T) == 4) {
#pragma unroll
                for (int l = 0; l < KB; ++l) {
                    const float2 v = ys[c * KB + l];
                    const float p = x * v.x;
                    float e = fmaf(x, v.x, -p);
                    e = fmaf(x, v.y, e);
                    const dfloat t = df_two_sum(ahi[l], p);
                    ahi[l] = t.hi;
                    alo[l] += t.lo + e;
                }
            } else {
#pragma unroll
                for (int l = 0; l < KB; ++l) {
                    const float2 v = ys[c * KB + l];
                    ad[l] = fma((double)x, (double)v.x + (double)v.y, ad[l]);
                }
            }
        }
    }
    if (!row) return;
#pragma unroll
    for (int l = 0; l < KB; ++l)
        if (l < kb) out[(int64_t)(l0 + l) * m + i] = (T)(sizeof(T) == 4 ? (double)ahi[l] + (double)alo[l] : ad[l]);
}

// ------------------------------------------------------------ dA (+)= L R^T
template <typename T>
__global__ void __launch_bounds__(BT) k_outer(T *dA, int64_t m, int64_t n, int64_t lda, const T *L, int r,
                                             const double *R, int acc) {
    constexpr int CN = 32;
    __shared__ T rs[CN * 64];
    const int64_t i = (int64_t)blockIdx.x * BT + threadIdx.x;
    const int64_t j0 = (int64_t)blockIdx.y * CN;
    const int ncol = (int)min((int64_t)CN, n - j0);
    for (int e = threadIdx.x; e < ncol * r; e += BT) {
        const int c = e / r, l = e - c * r;
        rs[c * 64 + l] = (T)R[(int64_t)l * n + j0 + c];
    }
    __syncthreads();
    if (i >= m) return;
    T lr[64];
#pragma unroll
    for (int l = 0; l < 64; ++l) lr[l] = l < r ? L[(int64_t)l * m + i] : (T)0;
    for (int c = 0; c < ncol; ++c) {
        T v = (T)0;
#pragma unroll
        for (int l = 0; l < 64; ++l)
            if (l < r) v = fma(lr[l], rs[c * 64 + l], v);
        T *dst = dA + (j0 + c) * lda + i;
        *dst = acc ? *dst + v : v;
    }
}

// Broadened 1 / (b - a): (b - a) / ((b - a)^2 + eta^2).
__device__ __forceinline__ double inv_gap(double a, double b, double eta) {
    const double d = b - a;
    return d / (d * d + eta * eta);
}

// ------------------------------------------- refinement adjoint (one CTA)
__global__ void __launch_bounds__(BT) k_bwd_refine_small(BwdRefine a) {
    const int r = a.r, k = a.k, tid = threadIdx.x, bd = blockDim.x;
    double *MB = a.work;                 // r x r
    double *MK = a.work + r * r;         // r x r: M_B^T V_R^T
    const double s0 = a.S[0];
    const double eta = 1e-12 * s0 * s0;
    for (int e = tid; e < r * r; e += bd) {
        const int i = e / r, j = e - i * r;
        // J_B = U_fin^T Ubar_fin (Ubar_fin = Ubar_out diag(sign), zero beyond k)
        auto J = [&](int p, int q) {
            if (q >= k) return 0.0;
            const double sg = a.dots[q] < 0.0 ? -1.0 : 1.0;
            return a.G[p * a.ldg + a.goff + q] * sg;
        };
        double v;
        if (i == j) {
            v = (a.dsigma && i < k) ? a.dsigma[i] : 0.0;
        } else {
            const double si = a.S[i], sj = a.S[j];
            v = inv_gap(si * si, sj * sj, eta) * (J(i, j) - J(j, i)) * sj;
        }
        MB[i * r + j] = v;
    }
    __syncthreads();
    // coefL = M_B K^T (U_fin -> L_ref); MK = M_B^T V_R^T
    for (int e = tid; e < r * r; e += bd) {
        const int l = e / r, q = e - l * r;
        double c1 = 0.0, c2 = 0.0;
        for (int j = 0; j < r; ++j) {
            c1 = fma(MB[l * r + j], a.K[q * r + j], c1);
            c2 = fma(MB[j * r + l], a.VR[q * r + j], c2);
        }
        a.coefL[l * r + q] = c1;
        MK[l * r + q] = c2;
    }
    __syncthreads();
    // coefT: rows [0, k) from Ubar_out (sign V_R^T), rows [k, k + r) from A Y
    // (K M_B^T V_R^T)
    for (int e = tid; e < (k + r) * r; e += bd) {
        const int l = e / r, q = e - l * r;
        double v;
        if (l < k) {
            v = (a.dots[l] < 0.0 ? -1.0 : 1.0) * a.VR[q * r + l];
        } else {
            const int ll = l - k;
            v = 0.0;
            for (int j = 0; j < r; ++j) v = fma(a.K[ll * r + j], MK[j * r + q], v);
        }
        a.coefT[l * r + q] = v;
    }
}

// --------------------------------------------- merge adjoint (one CTA)
__global__ void __launch_bounds__(BT) k_bwd_merge_small(BwdMerge a) {
    const double *rec = a.rec;
    const TapeLayout TL = tape_layout(a.rmax, a.cmax);
    const int r = (int)rec[0], g = (int)rec[1], rp = (int)rec[2], nc = (int)rec[3];
    const int nmax = a.rmax + a.cmax, ld = a.cmax, nt = r + g + rp;
    const double *sig = rec + TL.sig, *E = rec + TL.E, *UE = rec + TL.UE;
    const double *Ptot = rec + TL.Ptot, *Rinv = rec + TL.Rinv;
    const int tid = threadIdx.x, bd = blockDim.x;
    double *Tc = a.work;                       // (r + g) x nc
    double *VE = Tc + (size_t)nc * nc;         // nc x nc, VE[q * nc + s] = V_E[q][s]
    double *J = VE + (size_t)nc * nc;          // nc x rp
    double *N1 = J + (size_t)nc * nc;          // nc x nc
    double *Q1 = N1 + (size_t)nc * nc;         // nc x nc
    double *H = Q1 + (size_t)nc * nc;          // (r + g) x nc
    const double s0 = nc > 0 ? sig[0] : 0.0;
    const double u = a.dtype == POD_F32 ? 5.9604644775390625e-08 : 1.1102230246251565e-16;
    const double thr = nc * u * s0;   // the forward's drop rule for sigma
    const double eta = 1e-12 * s0 * s0;
    auto inv = [&](int s) { return sig[s] > thr ? 1.0 / sig[s] : 0.0; };
    // T_c rows r.. : R^{-1} U_E[r:, s]
    for (int e = tid; e < g * nc; e += bd) {
        const int j = e / nc, s = e - j * nc;
        double v = 0.0;
        for (int l = j; l < g; ++l) v = fma(Rinv[j * ld + l], UE[(size_t)s * nmax + r + l], v);
        Tc[(size_t)(r + j) * nc + s] = v;
    }
    // V_E[q][s] = (E^T u_s)_q / sigma_s
    for (int e = tid; e < nc * nc; e += bd) {
        const int q = e / nc, s = e - q * nc;
        double v = 0.0;
        for (int p = 0; p < nc; ++p) v = fma(E[(size_t)q * nmax + p], UE[(size_t)s * nmax + p], v);
        VE[(size_t)q * nc + s] = v * inv(s);
    }
    __syncthreads();
    // T_c rows < r : U_E[:r, s] - Ptot R^{-1} U_E[r:, s]
    for (int e = tid; e < r * nc; e += bd) {
        const int p = e / nc, s = e - p * nc;
        double v = UE[(size_t)s * nmax + p];
        for (int j = 0; j < g; ++j) v = fma(-Ptot[p * ld + j], Tc[(size_t)(r + j) * nc + s], v);
        Tc[(size_t)p * nc + s] = v;
    }
    __syncthreads();
    // J = T_c^T [U_t, C_t]^T Ubar = T_c^T G[:, r + g:]
    for (int e = tid; e < nc * rp; e += bd) {
        const int s = e / rp, j = e - s * rp;
        double v = 0.0;
        for (int p = 0; p < r + g; ++p) v = fma(Tc[(size_t)p * nc + s], a.G[(size_t)p * nt + r + g + j], v);
        J[(size_t)s * rp + j] = v;
    }
    __syncthreads();
    auto Je = [&](int i, int j) { return j < rp ? J[(size_t)i * rp + j] : 0.0; };
    for (int e = tid; e < nc * nc; e += bd) {
        const int i = e / nc, j = e - i * nc;
        double v = 0.0;
        if (i == j) {
            v = i < rp ? a.sbar[i] : 0.0;
        } else {
            v = inv_gap(sig[i] * sig[i], sig[j] * sig[j], eta) * (Je(i, j) - Je(j, i)) * sig[j];
        }
        if (j < rp) v -= Je(i, j) * inv(j);
        N1[e] = v;
    }
    __syncthreads();
    // Q1 = N1 V_E^T
    for (int e = tid; e < nc * nc; e += bd) {
        const int i = e / nc, c = e - i * nc;
        double v = 0.0;
        for (int j = 0; j < nc; ++j) v = fma(N1[(size_t)i * nc + j], VE[(size_t)c * nc + j], v);
        Q1[e] = v;
    }
    __syncthreads();
    // H = T_c Q1
    for (int e = tid; e < (r + g) * nc; e += bd) {
        const int p = e / nc, c = e - p * nc;
        double v = 0.0;
        for (int i = 0; i < nc; ++i) v = fma(Tc[(size_t)p * nc + i], Q1[(size_t)i * nc + c], v);
        H[e] = v;
    }
    __syncthreads();
    // coefficients of [U_t, C_t, Ubar] -> [Ubar_t (scaled by Sigma_t), Cbar_t];
    // K2[j][c] = V_E[c][j] / sigma_j
    const int qt = r + g;
    for (int e = tid; e < nt * qt; e += bd) {
        const int l = e / qt, c = e - l * qt;
        const double scale = c < r ? E[(size_t)c * nmax + c] : 1.0;   // Sigma_t on E's diagonal
        double v;
        if (l < r + g) v = H[(size_t)l * nc + c];
        else v = VE[(size_t)c * nc + (l - r - g)] * inv(l - r - g);
        a.coef[e] = v * scale;
    }
    // sbar_t,i = u_t,i^T Xbar[:, i]
    for (int i = tid; i < r; i += bd) {
        double v = 0.0;
        for (int p = 0; p < r + g; ++p) v = fma(a.G[(size_t)i * nt + p], H[(size_t)p * nc + i], v);
        for (int j = 0; j < rp; ++j) v = fma(a.G[(size_t)i * nt + r + g + j], VE[(size_t)i * nc + j] * inv(j), v);
        a.sbar_out[i] = v;
    }
}

}  // namespace

template <typename T>
pod_status launch_tape_u(const TapePtrs *tp, const DevState *st, const T *U, int64_t m, int rmax, cudaStream_t s) {
    int grid = (int)((m * rmax + BT - 1) / BT);
    if (grid > 1024) grid = 1024;
    k_tape_u<T><<<grid, BT, 0, s>>>(tp, st, U, m, rmax);
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}

BwdGramPlan bwd_gram_plan(int dtype, int64_t m, int ncols, int sms) {
    BwdGramPlan p{};
    const size_t es = dtype == POD_F32 ? 4 : 8;
    int rows = (int)((64 * 1024) / ((size_t)(ncols > 0 ? ncols : 1) * es)) - 1;
    if (rows > 512) rows = 512;
    if (rows < 16) rows = 16;
    int64_t grid = (m + rows - 1) / rows;
    if (grid < 2 * sms) {
        grid = 2 * sms;
        rows = (int)((m + grid - 1) / grid);
        if (rows < 1) rows = 1;
        grid = (m + rows - 1) / rows;
    }
    p.grid = (int)grid;
    p.rows_per = rows;
    p.lds = rows | 1;
    p.groups = (p.grid + RED_GROUP - 1) / RED_GROUP;
    p.smem = (size_t)p.lds * ncols * es;
    return p;
}

template <typename T>
pod_status launch_bwd_gram(const BwdGram &a, const BwdGramPlan &p, cudaStream_t s) {
    if (p.smem > 200 * 1024) return POD_EUNSUPPORTED;
    POD_CUDA_TRY(cudaFuncSetAttribute(k_bwd_gram<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
    k_bwd_gram<T><<<p.grid, BT, p.smem, s>>>(a);
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}

template <typename T>
pod_status launch_rowmix(const RowMix &a, cudaStream_t s) {
    int ptot = 0, qtot = 0;
    for (int b = 0; b < 3; ++b) ptot += a.pin[b];
    for (int o = 0; o < 2; ++o) qtot += a.qout[o];
    const size_t smem = ((size_t)ptot * 64 + (size_t)ptot * qtot) * sizeof(T);
    if (smem > 200 * 1024) return POD_EUNSUPPORTED;
    if (a.m <= 0 || qtot == 0) return POD_OK;
    POD_CUDA_TRY(cudaFuncSetAttribute(k_rowmix<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_rowmix<T><<<(unsigned)((a.m + 63) / 64), BT, smem, s>>>(a);
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}

template <typename T>
pod_status launch_az(const T *A, int64_t m, int64_t n, int64_t lda, const double *Y, int r, T *out, cudaStream_t s) {
    for (int l0 = 0; l0 < r; l0 += 32) {
        k_az<T><<<(unsigned)((m + BT - 1) / BT), BT, 0, s>>>(A, m, n, lda, Y, r, l0, out);
        POD_CUDA_TRY(cudaGetLastError());
    }
    return POD_OK;
}

template <typename T>
pod_status launch_outer(T *dA, int64_t m, int64_t n, int64_t lda, const T *L, int r, const double *R, int acc,
                        cudaStream_t s) {
    if (r > 64) return POD_EUNSUPPORTED;
    dim3 grid((unsigned)((m + BT - 1) / BT), (unsigned)((n + 31) / 32), 1);
    k_outer<T><<<grid, BT, 0, s>>>(dA, m, n, lda, L, r, R, acc);
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}

pod_status launch_bwd_refine_small(const BwdRefine &a, cudaStream_t s) {
    k_bwd_refine_small<<<1, BT, 0, s>>>(a);
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}

pod_status launch_bwd_merge_small(const BwdMerge &a, cudaStream_t s) {
    k_bwd_merge_small<<<1, BT, 0, s>>>(a);
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}

#define POD_BWD_INST(T)                                                                                          \
    template pod_status launch_tape_u<T>(const TapePtrs *, const DevState *, const T *, int64_t, int, cudaStream_t); \
    template pod_status launch_bwd_gram<T>(const BwdGram &, const BwdGramPlan &, cudaStream_t);                \
    template pod_status launch_rowmix<T>(const RowMix &, cudaStream_t);                                         \
    template pod_status launch_az<T>(const T *, int64_t, int64_t, int64_t, const double *, int, T *, cudaStream_t); \
    template pod_status launch_outer<T>(T *, int64_t, int64_t, int64_t, const T *, int, const double *, int,     \
                                        cudaStream_t);
POD_BWD_INST(float)
POD_BWD_INST(double)
