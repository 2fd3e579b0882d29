// Internal declarations shared by the translation units of the library.
#pragma once

#include "common.cuh"

// ---------------------------------------------------------------- sampler.cu
struct SampleArgs {
    int64_t n;
    int c;
    int L;                     // weight bits
    int mode_round0, mode;     // value source for round 0 and later rounds
    uint64_t seed;
    int stream_id;
    const double *s;           // column squared norms
    const double *ort;         // ORT values
    uint64_t *w;               // n weights (scratch, or input for mode 3)
    uint64_t *cdf;             // n prefix sums (scratch)
    uint8_t *mask;             // n, S membership
    uint8_t *flags;            // n scratch, zero on entry and on exit
    int32_t *draws;            // c raw draws
    int32_t *idx;              // c sorted distinct
    DevState *st;              // nullptr for the stand-alone entry point
    int32_t *g_out;            // stand-alone: distinct count
    int t_fixed;               // stand-alone: round index
    // replay of frozen index lists
    const int32_t *replay_idx;
    const int32_t *replay_off;
    int replay_T;
    // history
    int32_t *hist_idx;
    int32_t *hist_g;
};
pod_status launch_sample(const SampleArgs &a, cudaStream_t st);
pod_status launch_colnorms(const void *A, int dtype, int64_t m, int64_t n, int64_t lda,
                           double *s, cudaStream_t st);
pod_status launch_ort_values(const double *s, const double *Y, int64_t n, int ldy,
                             const DevState *st, const uint8_t *mask, double *ort,
                             cudaStream_t stream);
int weight_bits(int64_t n);

// ------------------------------------------------------------------- tall.cu
// Operands of the tall-skinny passes.  C columns are A + (idx ? idx[j] : j) * lda.
// Sizes are read on the device: r = st->r_cur (columns of U), g = st->g
// (columns of C), rn = st->r_new (columns written by the update).
template <typename T>
struct TallArgs {
    int64_t m;
    const T *A;
    int64_t lda;
    const int32_t *idx;
    T *U;
    int64_t ldu;
    const DevState *st;
    int rmax, cmax;         // capacities (layout)
    int bm;                 // rows per slab
    double *part;           // partials [gridDim.x][part_stride]
    int64_t part_stride;
    double *gsum;           // group sums [ceil(grid / 16)][part_stride]
    double *out;            // final sum (part_stride doubles)
    unsigned *counters;     // arrival counters (ceil(grid / 16) + 1), zero between launches
    int vec;                // 1: 16-byte copies are legal for every operand
    const double *P;        // r x g, ld cmax
    const double *P2;       // r x g, ld cmax
    const double *M1;       // g x g, ld cmax (upper triangular)
    const double *Xm;       // r x rn, ld rmax
    const double *Ym;       // g x rn, ld rmax
    unsigned char *gscratch;   // wide plans: per-CTA slices of gstride bytes (else null)
    int64_t gstride;
    int cond;               // 1: run only when st->robust is set (and then with a
                            // compensated Gram in the CGS pass); the QR2 pass with
                            // cond = 0 sets st->robust from its G2
    T *Wout;                // CGS pass: Z = C - U P stored here; QR2 pass (reading that Z
    int64_t ldw;            // as its C operand): W = (Z - U P2) M1 stored over it, the block
                            // the UPDATE pass then combines (m x g, ld ldw; or null)
    int defer;              // 1: write this CTA's partial and return; k_sum_parts sums
    unsigned *finish;       // UPDATE of a round: arrival counter; the last CTA ends the
                            // round (r_cur <- r_new, t + 1, the stop decision), or null
};

// Fixed-order sums of the tall passes' per-CTA FP64 partials, spread over
// many CTAs (one row of outputs and 32 columns per CTA).  The used entries:
// a rectangle (rows l < r_cur, columns j < g, at offset 0) and/or an upper
// triangle (p <= q < g, at tri_off), both with leading dimension ld.
struct SumParts {
    const double *part;
    int64_t stride;         // doubles per partial
    int nparts;
    double *out;
    int ld;
    int rect, tri;
    int rows_rect;          // grid rows reserved for the rectangle (its capacity)
    int64_t tri_off;
    const DevState *st;
    DevState *check;        // QR2: flag the round from |G2 - I| (or null)
    unsigned *counter;      // arrival counter of the check, zero between launches
    unsigned long long *devmax;   // running max |G2 - I| (bits of a double >= 0), zero between launches
};
pod_status launch_sum_parts(const SumParts &a, int cols_cap, cudaStream_t s);

enum TallKind { TALL_PROJ = 0, TALL_CGS = 1, TALL_QR2 = 2, TALL_UPDATE = 3 };

struct TallPlan {
    int grid;
    int bm;                 // slab rows of the PROJ pass (see bm_k)
    int groups;
    size_t smem;            // the largest of smem_k
    int wide;               // some kind keeps coefficient tiles and FP64 accumulators in global scratch
    int64_t gstride;        // bytes of scratch per CTA (wide kinds)
    int bm_k[4];            // per TallKind: slab rows,
    size_t smem_k[4];       //   dynamic shared memory,
    int wide_k[4];          //   whether it uses the global scratch,
    int threads_k[4];       //   threads per CTA
};

TallPlan tall_plan(int dtype, int64_t m, int rmax, int cmax, int num_sms);
template <typename T>
pod_status launch_tall(TallKind kind, const TallArgs<T> &a, const TallPlan &plan, cudaStream_t st);

// Y = A^T U (n x r, column-major with leading dimension n), optionally only
// for columns in `mask`.  Partials over `split` row ranges, reduced by the
// caller with launch_reduce.
template <typename T>
struct AtuArgs {
    int64_t m, n;
    const T *A;
    int64_t lda;
    const T *U;
    int64_t ldu;
    const DevState *st;     // r = st->r_cur
    const uint8_t *mask;    // may be null
    int rmax;               // partial stride is n * rmax
    int ldy;                // unused (Y is column-major, ld n)
    double *part;           // [split][n * r], column l at l * n
    double *Y;              // result, column-major n x r (ld n)
    unsigned *counters;     // one per column block, zero between launches
    int vec;                // 1: 16-byte copies are legal
};
struct AtuPlan {
    int nb, split, bm;
    size_t smem;
    dim3 grid;
};
AtuPlan atu_plan(int dtype, int64_t m, int64_t n, int rmax, int num_sms);
template <typename T>
pod_status launch_atu(const AtuArgs<T> &a, const AtuPlan &plan, cudaStream_t st);

// d_l = sum_i U_il z_i with z_i = int32(Philox(i, 0, 3, 0).x0) / 2^31.
template <typename T>
pod_status launch_sign_dots(const T *U, int64_t m, int64_t ldu, int r, uint64_t seed,
                            double *part, int grid, cudaStream_t st);

// ------------------------------------------------------------------- rows.cu
// Row sampling of ICRS (Algorithm 1, SAMPLE AND SCALE UNIQUE ROWS) and the
// Gram G_W = W^T W of the scaled row block.
template <typename T>
struct RowArgs {
    int64_t m;
    const T *A;
    int64_t lda;
    const int32_t *idx;     // sampled columns (g = st->g of them)
    const T *U;             // current modes (leverage scores)
    int64_t ldu;
    const DevState *st;
    int k;
    int row_strategy;
    int L;                  // weight bits for m rows
    int nblocks;            // ceil(m / 1024)
    int wdraws;             // row draws w
    int cmax;
    uint64_t seed;
    double *val;            // m row values
    double *bmax;           // nblocks
    uint64_t *w;            // m integer weights
    unsigned long long *bsum, *boff;   // nblocks
    unsigned long long *total;         // 1
    uint64_t *cdf;          // m
    unsigned *cnt;          // m, zero between rounds
    int32_t *rows, *rcnt;   // wdraws
    double *rscale;         // wdraws
    int32_t *h;             // distinct rows
    // Gram pass: ggrid CTAs of rows_per rows (shared column stride lds)
    int ggrid, rows_per, lds;
    int all_rows;           // 1: W = D (all m rows, unit scale)
    double *part;           // ggrid x cmax^2
    double *gsum;           // (groups + 1) x cmax^2
    unsigned *gcounters;    // groups + 1, zero between launches
    double *GW;             // cmax x cmax, upper triangle
};
struct RowGramPlan {
    int grid, rows_per, lds, groups;
};
RowGramPlan row_gram_plan(int dtype, int64_t wdraws, int cmax, int sms);
template <typename T>
pod_status launch_rows(const RowArgs<T> &a, cudaStream_t s, int sms);
template <typename T>
pod_status launch_row_gram(const RowArgs<T> &a, cudaStream_t s);
int row_blocks(int64_t m);

// ----------------------------------------------------------------- xty_tc.cu
// D = X^T Y on the tensor cores for FP32 data (see xty_tc.cu): the projection
// U^T C of BLOCK MERGE (X gathered from A or dense) and A^T U.
struct XtyTcArgs {
    int64_t m;              // rows (the reduction)
    int64_t ncols;          // X columns when not gathered
    int gather;             // 1: X = columns idx[0 .. st->g) of the matrix X (ld ldx)
    const int32_t *idx;
    const float *X;         // set by launch_xty_tc
    int64_t ldx;
    const DevState *st;     // done flag; st->r_cur Y columns when ny_from_state; st->g
    int ny_from_state, ny;
    int mtiles, maxcover;   // set by launch_xty_tc from the plan
    int deferred;           // 1: per-CTA slots part[b * part_stride + yc * ldo_y + xc], summed elsewhere
    double *part;
    int64_t part_stride;
    double *out;            // local sums: out[yc * ldo_y + xc * ldo_x]
    int64_t ldo_y, ldo_x;
    unsigned *counters;     // one per M-tile, zero between launches
    int *err;               // set to POD_ETIMEOUT when a bounded wait expires
    uint32_t spin;          // polls before a pipeline wait gives up (0: default)
};
struct XtyTcPlan {
    int mode, nt, grid, mtiles, maxcover;
    size_t smem, part_doubles;
};
int xty_tc_mode_ok(int mode);
int xty_tc_supported(int dtype, int64_t m, int64_t ldx, int ny_max, const void *X, const void *Y);
XtyTcPlan xty_tc_plan(int mode, int64_t m, int64_t ncols_max, int ny_max, int sms, int deferred);
pod_status launch_xty_tc(const XtyTcArgs &a, const XtyTcPlan &plan, const float *X, int64_t ldx, int64_t xcols,
                         const float *Y, int64_t ycols, cudaStream_t s);


// ------------------------------------------------------------------ wedin.cu
// Eq. 7 residual norms after the refinement (see wedin.cu).
struct WedinArgs {
    int64_t m, n, lda;
    int k, r;
    const double *Y, *K, *VR, *sigma;   // Y = A^T U (n x r), refinement K and V_R (r x r)
    double *Vk;                         // n x k
    float2 *Vkf;                        // n x k, double-float copy
    double *part_s, *gsum_s, *part_r, *gsum_r;
    double *out;                        // [0] = |S|^2, [1 + p] = |R|^2 of pass p
    unsigned *counters_v, *counters_r;  // zero between launches
};
int wedin_grid_n(int64_t n);
int wedin_grid_m(int64_t m);
int wedin_passes(int k);
template <typename T>
pod_status launch_wedin(const WedinArgs &a, const T *A, const T *U, cudaStream_t s);

// --------------------------------------------------------- backward tape
// Where the forward records what pod_backward needs: the basis U_t entering
// every round (m x rmax, storage type) and a per-round record of the merge
// core.  Device-resident so the host can grow the buffers between batches of
// rounds without re-capturing the round graph.
struct TapePtrs {
    void *U;        // cap slots of m * rmax elements
    double *core;   // cap records of tape_layout(...).stride doubles
    int cap;
};
// Record of round t (doubles): [0] r_t, [1] g_t, [2] r_new, [3] n_c; then
// sig (nmax: all singular values of E, descending), E (nmax x nmax, column-
// major, ld nmax), UE (nmax x nmax: left singular vector s at s * nmax),
// Ptot (rmax x cmax, ld cmax), Rinv (cmax x cmax, ld cmax).
struct TapeLayout {
    int64_t sig, E, UE, Ptot, Rinv, stride;
};
__host__ __device__ inline TapeLayout tape_layout(int rmax, int cmax) {
    const int64_t nmax = rmax + cmax;
    TapeLayout L;
    L.sig = 8;
    L.E = L.sig + nmax;
    L.UE = L.E + nmax * nmax;
    L.Ptot = L.UE + nmax * nmax;
    L.Rinv = L.Ptot + (int64_t)rmax * cmax;
    L.stride = L.Rinv + (int64_t)cmax * cmax;
    return L;
}
template <typename T>
pod_status launch_tape_u(const TapePtrs *tp, const DevState *st, const T *U, int64_t m, int rmax, cudaStream_t s);

// ---------------------------------------------------------- backward.cu
struct BwdGram {            // G = [blocks < nleft]^T [blocks], row-major nl x nt
    const void *ptr[3];
    int64_t ld[3];
    const int32_t *idx[3];  // column gather (or null)
    int ncol[3];
    int nleft;
    int64_t m;
    int rows_per, lds;
    double *part, *gsum, *out;
    unsigned *counters;     // groups + 1, zero between launches
};
struct BwdGramPlan {
    int grid, rows_per, lds, groups;
    size_t smem;
};
BwdGramPlan bwd_gram_plan(int dtype, int64_t m, int ncols, int sms);
template <typename T>
pod_status launch_bwd_gram(const BwdGram &a, const BwdGramPlan &p, cudaStream_t s);
struct RowMix {             // out_o[i, q] (+)= sum_b in_b[i, :] coef[rows of b][cols of o]
    int64_t m;
    const void *in[3];
    int64_t ldi[3];
    const int32_t *idx_in[3];
    int pin[3];
    void *out[2];
    int64_t ldo[2];
    const int32_t *idx_out[2];
    int qout[2];
    int acc_out[2];
    const double *coef;     // (sum pin) x (sum qout), row-major
};
template <typename T>
pod_status launch_rowmix(const RowMix &a, cudaStream_t s);
template <typename T>
pod_status launch_az(const T *A, int64_t m, int64_t n, int64_t lda, const double *Y, int r, T *out, cudaStream_t s);
template <typename T>
pod_status launch_outer(T *dA, int64_t m, int64_t n, int64_t lda, const T *L, int r, const double *R, int acc,
                        cudaStream_t s);
struct BwdRefine {
    int r, k;
    const double *G;        // r x (r + k): U_fin^T [U_fin, Ubar_out]
    int ldg, goff;
    const double *S, *VR, *K, *dots, *dsigma;   // dsigma may be null
    double *work;           // 2 r^2
    double *coefL;          // r x r
    double *coefT;          // (k + r) x r
};
pod_status launch_bwd_refine_small(const BwdRefine &a, cudaStream_t s);
struct BwdMerge {
    const double *rec;      // tape record of the round
    int rmax, cmax, dtype;
    const double *G;        // (r + g) x (r + g + r')
    const double *sbar;     // r' incoming singular-value adjoints
    double *work;           // 6 nmax^2
    double *coef;           // (r + g + r') x (r + g)
    double *sbar_out;       // r
};
pod_status launch_bwd_merge_small(const BwdMerge &a, cudaStream_t s);

// ------------------------------------------------------------------ small.cu
pod_status launch_reduce(const double *part, int nparts, int64_t stride, int64_t count,
                         double *out, const DevState *st, cudaStream_t s);

struct SmallArgs {
    DevState *st;
    int cond;               // 1: run only when st->robust is set
    int dtype;              // storage type (rounding of coefficients)
    int core_f64;           // arithmetic of the core SVD
    int64_t m;
    int k, r, c, rmax, cmax;   // r: truncation rank (<= rmax, the layout capacity)
    int criterion;
    double tol;
    int max_iter;
    double *sigma;          // r_cur values (in) / r_new values (out)
    const double *P;        // r x g (ld cmax): U^T C
    const double *PG;       // cgs partial sums: P2 (r x g, ld cmax) then G (g x g, ld cmax)
    const double *G2;       // second CholeskyQR Gram (g x g, ld cmax)
    double *Ptot;           // r x g, ld cmax
    double *M1;             // g x g, ld cmax
    double *R1p;            // g x g, ld cmax
    double *E;              // nc x nc scratch (column-major, ld rmax + cmax)
    const struct TapePtrs *tape;   // per-round merge record for pod_backward (or null)
    unsigned char *gws_core;       // wide cores: global scratch (core_gws_bytes), else null
    int jac_smem;                  // wide cores: 1 = Jacobi arrays still in shared memory
    unsigned char *gws_chol;       // wide first-CholeskyQR kernel: global scratch, else null
    double *Xm;             // r x rn, ld rmax
    double *Ym;             // g x rn, ld rmax
    int wq;                 // 1: the UPDATE combines U and the stored W = Z M1, so
                            // Xm = U_E[:r, :rn], Ym = R2^{-1} U_E[r:, :rn];
                            // 0: it combines U and C, Xm = U_E[:r] - Ptot Ym,
                            // Ym = R^{-1} U_E[r:]
    double *hist_measure;   // per-round measure
};
pod_status launch_small_chol(const SmallArgs &a, cudaStream_t s);
pod_status launch_core(const SmallArgs &a, cudaStream_t s);
size_t core_smem_bytes(int rmax, int cmax, int dtype);
size_t core_jacobi_bytes(int rmax, int cmax, int dtype);   // shared memory of the Jacobi arrays alone
size_t small_chol_smem(int cmax, int dtype, int cond);   // bytes of k_small_chol's work area


// refinement QR(A^T U), SVD(R)
struct RefineArgs {
    int r;                  // modes
    int dtype;
    const double *G;        // r x r, ld r: Y^T Y
    const double *G2;       // r x r, ld r: second CholeskyQR Gram
    double *M1, *R1p;       // r x r, ld r
    double *sigma;          // out: r
    double *VR;             // out: r x r (ld r), U <- U VR
    double *K;              // out: r x r (ld r), V <- Y K
    unsigned char *gws;     // wide refinements: global scratch (refine_gws_bytes), else null
};
pod_status launch_refine_chol(const RefineArgs &a, cudaStream_t s);
size_t refine_gws_bytes(int r);   // bytes of the refinement kernels' work arrays

// ICRS: from G_W = W^T W (g x g, ld cmax) the inputs of a core SVD whose
// left singular vectors are the eigenvectors of G_W (R1p = R_hat with
// G_W = R_hat R_hat^T, G2 = M1 = I) and its state stc = {r_cur 0, g};
// afterwards k_rows_setg sets the round's block width to the kept count.
struct RowsSmallArgs {
    DevState *st, *stc;
    int dtype, core_f64, cmax;
    const double *GW;
    double *R1p, *G2, *M1;
};
pod_status launch_rows_chol(const RowsSmallArgs &a, cudaStream_t s);
pod_status launch_rows_setg(DevState *st, const DevState *stc, cudaStream_t s);
size_t rows_small_smem(int cmax);
pod_status launch_refine_svd(const RefineArgs &a, cudaStream_t s);
