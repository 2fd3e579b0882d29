// C ABI of the library (include/pod.h): context life cycle, the ISMA
// iteration driver (Algorithm 1), the closing refinement and the step-level
// entry points.  One round of Algorithm 1 is a fixed sequence of kernels
// whose sizes live in device memory (DevState); it is captured once into a
// CUDA graph and replayed, and the host reads the 80-byte state only between
// batches of rounds.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "pod_internal.h"



namespace {

constexpr int ROW_KERNELS = 8;   // launches of launch_rows

template <typename T>
__global__ void k_write_modes(const T *U, int64_t m, int r_cur, int k, const double *sigma,
                              const double *dots, T *U_out, double *sigma_out) {
    const int64_t total = m * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(e / m);
        const int64_t i = e - (int64_t)l * m;
        T v = (T)0;
        if (l < r_cur) v = dots[l] < 0.0 ? -U[(int64_t)l * m + i] : U[(int64_t)l * m + i];
        U_out[(int64_t)l * m + i] = v;
    }
    if (blockIdx.x == 0)
        for (int l = threadIdx.x; l < k; l += blockDim.x) sigma_out[l] = l < r_cur ? sigma[l] : 0.0;
}

// V_out[:, l] = sign_l * (Y K)[:, l]; Y column-major n x r (ld n), K r x r (ld r)
template <typename T>
__global__ void k_write_v(const double *Y, const double *K, int64_t n, int r, int k, const double *dots,
                          T *V_out) {
    const int64_t total = n * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(e / n);
        const int64_t j = e - (int64_t)l * n;
        double v = 0.0;
        if (l < r) {
            for (int q = 0; q < r; ++q) v += Y[(int64_t)q * n + j] * K[q * r + l];
            if (dots[l] < 0.0) v = -v;
        }
        V_out[(int64_t)l * n + j] = (T)v;
    }
}

__global__ void k_set_state(DevState *st, int r_cur, int g, int r_new, int t, int remaining) {
    if (threadIdx.x == 0) {
        DevState s{};
        s.t = t;
        s.r_cur = r_cur;
        s.g = g;
        s.r_new = r_new;
        s.remaining = remaining;
        *st = s;
    }
}

// C = U diag(sigma): the scaled left factor of a block (Algorithm 3's merge input)
template <typename T>
__global__ void k_scale_cols(const T *U, int64_t m, int r, const double *sigma, T *C) {
    const int64_t total = m * r;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(e / m);
        C[e] = (T)((double)U[e] * sigma[l]);
    }
}

int device_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 148;
    return sms > 0 ? sms : 148;
}

template <typename V>
pod_status dalloc(V **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    if (cudaMalloc((void **)p, count * sizeof(V)) != cudaSuccess) {
        cudaGetLastError();
        return POD_ENOMEM;
    }
    return POD_OK;
}

}  // namespace

struct pod_ctx {
    pod_params p;
    const void *A;
    cudaStream_t stream;
    int rmax, cmax, nmax;
    int rtrunc;         // truncation rank of a merge (<= rmax)
    int core_f64;
    int sms;
    TallPlan plan;
    AtuPlan aplan;
    // device buffers
    void *U;
    double *sigma, *s, *ort, *Y;
    uint8_t *mask, *flags;
    uint64_t *w, *cdf;
    int32_t *draws, *idx, *hist_idx, *hist_g;
    double *hist_measure;
    DevState *st, *aux;
    double *part, *part_atu;
    double *P, *PG, *G2, *Ptot, *M1, *R1p, *E, *Xm, *Ym, *gsum;
    unsigned *counters, *atu_counters;
    size_t part_cap, gsum_cap, counters_cap;   // doubles / doubles / counters allocated
    int vec;            // 16-byte copies legal for A and U
    double *rG, *rG2, *rM1, *rR1p, *rsig, *rVR, *rK, *dots, *part_sign;
    int32_t *replay_idx, *replay_off;
    int replay_T;
    // ICRS (rows = 1): row sampling buffers, the Gram G_W of the scaled row
    // block, the coefficients V_r and the new block C = D V_r
    int wdraws, rnb;
    RowGramPlan gplan;
    double *r_val, *r_bmax, *r_rscale, *GW, *rYm, *part_w, *gsum_w;
    double *wR1p, *wG2, *wM1, *wsig, *wX;
    unsigned long long *r_bsum, *r_boff, *r_total;
    uint64_t *r_w, *r_cdf;
    unsigned *r_cnt, *counters_w;
    int32_t *r_rows, *r_rcnt, *r_h;
    void *Cbuf;
    void *Wbuf;      // W = Z M1 of the current round (m x cmax, ld m), from the QR2 pass
    unsigned *sum_counter;   // arrival counter of the QR2 sums' G2 check
    unsigned *upd_counter;   // arrival counter of the UPDATE pass (end of the round)
    unsigned long long *g2dev;   // running max |G2 - I| of the QR2 sums
    // wide sizes: global scratch for the tall passes, the core, the first
    // CholeskyQR kernel and the refinement when their shared memory would not fit
    unsigned char *tall_gs, *core_gs, *chol_gs, *refine_gs, *ytall_gs;
    int jac_smem;
    // pod_backward tape (keep_tape = 1): host copy of the device TapePtrs
    TapePtrs tape_h;
    TapePtrs *tape_d;
    bool modes_done;
    // tensor-core contractions (precision TF32X3, BF16X3, BF16): A^T U
    // (local sums into Y) and the round's U^T C (deferred sums, ICS only)
    int use_tc, use_tc_proj;
    uint32_t tc_spin;   // pipeline-wait bound of the tensor-core kernels (0: default)
    XtyTcPlan tcplan, pplan;
    double *tc_part;
    unsigned *tc_counters;
    // host
    DevState *hstate;   // pinned mirror
    cudaGraphExec_t graph;
    bool graph_ready, graph_failed;
    bool poisoned;
    bool refined;
    int refined_r;
    int sign_grid;
    // kernel launches issued (host count) and per-launch event marks
    long long launches;
    int graph_kernels;
    cudaEvent_t *prof_ev;
    int prof_n, prof_cap;
};

static void mark(pod_ctx *c) {
    c->launches += 1;
    if (c->prof_ev && c->prof_n < c->prof_cap) cudaEventRecord(c->prof_ev[c->prof_n++], c->stream);
}

static void ctx_free(pod_ctx *c) {
    if (!c) return;
    if (c->graph_ready) cudaGraphExecDestroy(c->graph);
    void *bufs[] = {c->U, c->sigma, c->s, c->ort, c->Y, c->mask, c->flags, c->w, c->cdf, c->draws,
                    c->idx, c->hist_idx, c->hist_g, c->hist_measure, c->st, c->aux, c->part,
                    c->part_atu, c->P, c->PG, c->G2, c->Ptot, c->M1, c->R1p, c->E, c->Xm, c->Ym,
                    c->rG, c->rG2, c->rM1, c->rR1p, c->rsig, c->rVR, c->rK, c->dots, c->part_sign,
                    c->replay_idx, c->replay_off, c->gsum, c->counters, c->atu_counters,
                    c->r_val, c->r_bmax, c->r_rscale, c->GW, c->rYm, c->part_w, c->gsum_w, c->r_bsum,
                    c->r_boff, c->r_total, c->r_w, c->r_cdf, c->r_cnt, c->counters_w, c->r_rows,
                    c->r_rcnt, c->r_h, c->Cbuf, c->Wbuf, c->sum_counter, c->upd_counter, c->g2dev, c->wR1p, c->wG2, c->wM1, c->wsig, c->wX,
                    c->tc_part, c->tc_counters, c->tall_gs, c->core_gs, c->chol_gs, c->refine_gs, c->ytall_gs};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (c->tape_h.U) cudaFree(c->tape_h.U);
    if (c->tape_h.core) cudaFree(c->tape_h.core);
    if (c->tape_d) cudaFree(c->tape_d);
    if (c->hstate) cudaFreeHost(c->hstate);
    free(c);
}

static pod_status check_params(const pod_params *p) {
    if (!p) return POD_EINVAL;
    if (p->m <= 0 || p->n <= 0 || p->lda < p->m) return POD_EINVAL;
    if (p->n > 0x7fffffffLL) return POD_EINVAL;
    if (p->k < 1 || p->k > p->m || p->k > p->n) return POD_EINVAL;
    if (p->c < 1) return POD_EINVAL;
    const int r = p->r > 0 ? p->r : p->k;
    if (r < p->k) return POD_EINVAL;
    if (p->dtype != POD_F32 && p->dtype != POD_F64) return POD_EINVAL;
    if (p->col_strategy < POD_L2N || p->col_strategy > POD_ORT) return POD_EINVAL;
    if (p->criterion != POD_SUBSPACE && p->criterion != POD_MODES) return POD_EINVAL;
    if (p->core < POD_CORE_AUTO || p->core > POD_CORE_F64) return POD_EINVAL;
    if (p->rows != 0 && p->rows != 1) return POD_EINVAL;
    if (p->row_strategy != POD_ROW_L2N && p->row_strategy != POD_ROW_LS) return POD_EINVAL;
    if (p->w < 0) return POD_EINVAL;
    if (p->block_trunc != 0 && p->block_trunc != 1) return POD_EINVAL;
    if (p->precision < POD_PREC_F32 || p->precision > POD_PREC_TF32X3) return POD_EINVAL;
    if (p->keep_tape != 0 && p->keep_tape != 1) return POD_EINVAL;
    if (p->precision != POD_PREC_F32 && p->dtype != POD_F32) return POD_EUNSUPPORTED;
    if (p->keep_tape && (p->rows || p->block_trunc)) return POD_EUNSUPPORTED;
    if (p->reserved != 0) return POD_EINVAL;
    if (p->c > 256 || (p->r > 0 ? p->r : p->k) > 256) return POD_EUNSUPPORTED;
    if (p->c + (p->r > 0 ? p->r : p->k) > 320) return POD_EUNSUPPORTED;   // Jacobi holds n_c <= 320
    if (!(p->tol == p->tol)) return POD_EINVAL;
    return POD_OK;
}

// Default row draws of ICRS: Eq. 5 with epsilon = delta = 0.6, at most m.
static int64_t default_row_draws(int64_t k, int64_t m) {
    const double eps = 0.6, delta = 0.6;
    const double v = ceil((double)(k * k) * pow(1.0 + sqrt(log(2.0 / delta)), 2.0) / pow(eps, 4.0));
    const int64_t w = (int64_t)v;
    return w < m ? w : m;
}

template <typename T>
static TallArgs<T> tall_args(pod_ctx *c, double *part, int64_t stride) {
    TallArgs<T> a{};
    a.m = c->p.m;
    a.A = (const T *)c->A;
    a.lda = c->p.lda;
    a.idx = c->idx;
    a.U = (T *)c->U;
    a.ldu = c->p.m;
    a.st = c->st;
    a.rmax = c->rmax;
    a.cmax = c->cmax;
    a.bm = c->plan.bm;
    a.part = part;
    a.part_stride = stride;
    a.gsum = c->gsum;
    a.counters = c->counters;
    a.vec = c->vec;
    a.out = nullptr;
    a.P = c->P;
    a.P2 = c->PG;
    a.M1 = c->M1;
    a.Xm = c->Xm;
    a.Ym = c->Ym;
    a.gscratch = c->plan.wide ? c->tall_gs : nullptr;
    a.gstride = c->plan.gstride;
    return a;
}

static SmallArgs small_args(pod_ctx *c) {
    SmallArgs s{};
    s.st = c->st;
    s.dtype = c->p.dtype;
    s.core_f64 = c->core_f64;
    s.m = c->p.m;
    s.k = c->p.k;
    s.r = c->rtrunc;
    s.c = c->p.c;
    s.rmax = c->rmax;
    s.cmax = c->cmax;
    s.criterion = c->p.criterion;
    s.tol = c->p.tol;
    s.max_iter = c->p.max_iter;
    s.sigma = c->sigma;
    s.P = c->P;
    s.PG = c->PG;
    s.G2 = c->G2;
    s.Ptot = c->Ptot;
    s.M1 = c->M1;
    s.R1p = c->R1p;
    s.E = c->E;
    s.Xm = c->Xm;
    s.Ym = c->Ym;
    s.hist_measure = c->hist_measure;
    s.gws_core = c->core_gs;
    s.jac_smem = c->jac_smem;
    s.gws_chol = c->chol_gs;
    return s;
}

// Make the tape hold at least `slots` rounds (U_t and the merge record);
// grows by doubling, keeping what was recorded.  Host side, between batches.
static pod_status tape_reserve(pod_ctx *c, int slots) {
    if (!c->p.keep_tape || slots <= c->tape_h.cap) return POD_OK;
    int cap = c->tape_h.cap > 0 ? c->tape_h.cap : 4;
    while (cap < slots) cap *= 2;
    const size_t es = c->p.dtype == POD_F32 ? 4 : 8;
    const size_t ubytes = (size_t)c->p.m * c->rmax * es;
    const int64_t stride = tape_layout(c->rmax, c->cmax).stride;
    void *U = nullptr;
    double *core = nullptr;
    if (cudaMalloc(&U, ubytes * cap) != cudaSuccess || cudaMalloc((void **)&core, (size_t)stride * cap * 8) != cudaSuccess) {
        cudaGetLastError();
        if (U) cudaFree(U);
        return POD_ENOMEM;
    }
    cudaStream_t s = c->stream;
    TapePtrs nt{U, core, cap};
    if (c->tape_h.cap > 0) {
        POD_CUDA_TRY(cudaMemcpyAsync(U, c->tape_h.U, ubytes * c->tape_h.cap, cudaMemcpyDeviceToDevice, s));
        POD_CUDA_TRY(cudaMemcpyAsync(core, c->tape_h.core, (size_t)stride * c->tape_h.cap * 8, cudaMemcpyDeviceToDevice, s));
    }
    POD_CUDA_TRY(cudaMemcpyAsync(c->tape_d, &nt, sizeof(TapePtrs), cudaMemcpyHostToDevice, s));
    POD_CUDA_TRY(cudaStreamSynchronize(s));
    if (c->tape_h.U) cudaFree(c->tape_h.U);
    if (c->tape_h.core) cudaFree(c->tape_h.core);
    c->tape_h = nt;
    return POD_OK;
}

// Y = A^T U (n x r_cur of state st): tensor cores (split TF32, split BF16 or
// BF16 products) when the context runs at a tensor-core precision, FP32 SIMT
// otherwise.
template <typename T>
static pod_status enqueue_atu(pod_ctx *c, const DevState *st, const uint8_t *mask, cudaStream_t s) {
    if (c->use_tc) {
        XtyTcArgs xa{};
        xa.m = c->p.m;
        xa.ncols = c->p.n;
        xa.st = st;
        xa.ny_from_state = 1;
        xa.part = c->tc_part;
        xa.out = c->Y;
        xa.ldo_y = c->p.n;
        xa.ldo_x = 1;
        xa.counters = c->tc_counters;
        xa.err = &c->st->status;
        xa.spin = c->tc_spin;
        return launch_xty_tc(xa, c->tcplan, (const float *)c->A, c->p.lda, c->p.n, (const float *)c->U, c->rmax, s);
    }
    AtuArgs<T> aa{};
    aa.m = c->p.m;
    aa.n = c->p.n;
    aa.A = (const T *)c->A;
    aa.lda = c->p.lda;
    aa.U = (const T *)c->U;
    aa.ldu = c->p.m;
    aa.st = st;
    aa.mask = mask;
    aa.ldy = (int)c->p.n;
    aa.rmax = c->rmax;
    aa.part = c->part_atu;
    aa.Y = c->Y;
    aa.counters = c->atu_counters;
    aa.vec = c->vec;
    return launch_atu<T>(aa, c->aplan, s);
}

// One round of Algorithm 1 (probabilities, draws, GET UPDATE, BLOCK MERGE,
// convergence test) as a fixed launch sequence.
template <typename T>
static pod_status enqueue_round(pod_ctx *c) {
    cudaStream_t s = c->stream;
    if (c->p.keep_tape) {
        POD_TRY(launch_tape_u<T>(c->tape_d, c->st, (const T *)c->U, c->p.m, c->rmax, s));
        mark(c);
    }
    const int64_t sPG = (int64_t)c->rmax * c->cmax + (int64_t)c->cmax * c->cmax;
    if (c->p.col_strategy == POD_ORT) {
        POD_TRY(enqueue_atu<T>(c, c->st, c->mask, s));
        mark(c);
        POD_TRY(launch_ort_values(c->s, c->Y, c->p.n, (int)c->p.n, c->st, c->mask, c->ort, s));
        mark(c);
    }
    SampleArgs sa{};
    sa.n = c->p.n;
    sa.c = c->p.c;
    sa.L = weight_bits(c->p.n);
    sa.mode_round0 = 0;
    sa.mode = c->p.col_strategy == POD_L2N ? 0 : (c->p.col_strategy == POD_UNF ? 1 : 2);
    sa.seed = c->p.seed;
    sa.stream_id = 0;
    sa.s = c->s;
    sa.ort = c->ort;
    sa.w = c->w;
    sa.cdf = c->cdf;
    sa.mask = c->mask;
    sa.flags = c->flags;
    sa.draws = c->draws;
    sa.idx = c->idx;
    sa.st = c->st;
    sa.replay_idx = c->replay_idx;
    sa.replay_off = c->replay_off;
    sa.replay_T = c->replay_T;
    sa.hist_idx = c->hist_idx;
    sa.hist_g = c->hist_g;
    POD_TRY(launch_sample(sa, s));
    mark(c);

    TallArgs<T> ta = tall_args<T>(c, c->part, (int64_t)c->rmax * c->cmax);
    if (c->p.rows || c->p.block_trunc) {
        // GET UPDATE with rows (ICRS): W from sampled rows of D, V_r from
        // W^T W; or the literal truncation of the new block (W = D, all rows,
        // unit scale); the merge then takes the materialised block C = D V_r
        RowArgs<T> ra{};
        ra.m = c->p.m;
        ra.A = (const T *)c->A;
        ra.lda = c->p.lda;
        ra.idx = c->idx;
        ra.U = (const T *)c->U;
        ra.ldu = c->p.m;
        ra.st = c->st;
        ra.k = c->p.k;
        ra.row_strategy = c->p.row_strategy;
        ra.L = weight_bits(c->p.m);
        ra.nblocks = c->rnb;
        ra.wdraws = c->wdraws;
        ra.cmax = c->cmax;
        ra.seed = c->p.seed;
        ra.val = c->r_val;
        ra.bmax = c->r_bmax;
        ra.w = c->r_w;
        ra.bsum = c->r_bsum;
        ra.boff = c->r_boff;
        ra.total = c->r_total;
        ra.cdf = c->r_cdf;
        ra.cnt = c->r_cnt;
        ra.rows = c->r_rows;
        ra.rcnt = c->r_rcnt;
        ra.rscale = c->r_rscale;
        ra.h = c->r_h;
        ra.ggrid = c->gplan.grid;
        ra.rows_per = c->gplan.rows_per;
        ra.lds = c->gplan.lds;
        ra.part = c->part_w;
        ra.gsum = c->gsum_w;
        ra.gcounters = c->counters_w;
        ra.GW = c->GW;
        ra.all_rows = c->p.rows ? 0 : 1;
        if (c->p.rows) {
            POD_TRY(launch_rows<T>(ra, s, c->sms));
            c->launches += ROW_KERNELS - 1;
            mark(c);
        }
        POD_TRY(launch_row_gram<T>(ra, s));
        mark(c);
        RowsSmallArgs rs{};
        rs.st = c->st;
        rs.stc = c->aux + 5;
        rs.dtype = c->p.dtype;
        rs.core_f64 = c->core_f64;
        rs.cmax = c->cmax;
        rs.GW = c->GW;
        rs.R1p = c->wR1p;
        rs.G2 = c->wG2;
        rs.M1 = c->wM1;
        POD_TRY(launch_rows_chol(rs, s));
        mark(c);
        SmallArgs sw = small_args(c);
        sw.st = c->aux + 5;
        sw.r = c->rmax;
        sw.G2 = c->wG2;
        sw.M1 = c->wM1;
        sw.R1p = c->wR1p;
        sw.sigma = c->wsig;
        sw.Xm = c->wX;
        sw.Ym = c->rYm;
        sw.hist_measure = nullptr;
        POD_TRY(launch_core(sw, s));
        mark(c);
        TallArgs<T> ca = tall_args<T>(c, c->part, 0);
        ca.st = c->aux + 5;
        ca.U = (T *)c->Cbuf;
        ca.Ym = c->rYm;
        POD_TRY(launch_tall<T>(TALL_UPDATE, ca, c->plan, s));
        mark(c);
        POD_TRY(launch_rows_setg(c->st, c->aux + 5, s));
        mark(c);
        ta.A = (const T *)c->Cbuf;
        ta.idx = nullptr;
        ta.lda = c->p.m;
        ta.vec = (c->p.m * (int64_t)sizeof(T)) % 16 == 0;
    }
    ta.Wout = (T *)c->Wbuf;
    ta.ldw = c->p.m;
    // the three passes leave their per-CTA partials to k_sum_parts, which
    // spreads the fixed-order sums over many CTAs (one CTA summing all
    // partials was 40% of a pass)
    ta.defer = 1;
    SumParts sp{};
    sp.part = c->part;
    sp.nparts = c->plan.grid;
    sp.ld = c->cmax;
    sp.rows_rect = c->rmax;
    sp.st = c->st;
    ta.out = c->P;
    if (c->use_tc_proj && !(c->p.rows || c->p.block_trunc)) {
        // U^T C on the tensor cores, the sampled columns read in place
        XtyTcArgs xa{};
        xa.m = c->p.m;
        xa.gather = 1;
        xa.idx = c->idx;
        xa.st = c->st;
        xa.ny_from_state = 1;
        xa.deferred = 1;
        xa.part = c->part;
        xa.part_stride = ta.part_stride;
        xa.ldo_y = c->cmax;
        xa.ldo_x = 1;
        xa.err = &c->st->status;
        xa.spin = c->tc_spin;
        POD_TRY(launch_xty_tc(xa, c->pplan, (const float *)c->A, c->p.lda, c->p.n, (const float *)c->U, c->rmax, s));
        mark(c);
        sp.nparts = c->pplan.grid;
    } else {
        POD_TRY(launch_tall<T>(TALL_PROJ, ta, c->plan, s));
        mark(c);
    }
    sp.stride = ta.part_stride;
    sp.out = c->P;
    sp.rect = 1;
    sp.tri = 0;
    POD_TRY(launch_sum_parts(sp, c->cmax, s));
    mark(c);
    sp.nparts = c->plan.grid;
    ta.part_stride = sPG;
    ta.out = c->PG;
    POD_TRY(launch_tall<T>(TALL_CGS, ta, c->plan, s));
    mark(c);
    sp.stride = sPG;
    sp.out = c->PG;
    sp.rect = 1;
    sp.tri = 1;
    sp.tri_off = (int64_t)c->rmax * c->cmax;
    POD_TRY(launch_sum_parts(sp, c->cmax, s));
    mark(c);
    SmallArgs sm = small_args(c);
    sm.tape = c->p.keep_tape ? c->tape_d : nullptr;
    sm.wq = 1;
    POD_TRY(launch_small_chol(sm, s));
    mark(c);
    // QR2 reads the Z that the CGS pass stored in Wbuf and writes W over it
    TallArgs<T> qa = ta;
    qa.A = (const T *)c->Wbuf;
    qa.idx = nullptr;
    qa.lda = c->p.m;
    qa.vec = (c->p.m * (int64_t)sizeof(T)) % 16 == 0;
    qa.part_stride = (int64_t)c->cmax * c->cmax;
    qa.out = c->G2;
    POD_TRY(launch_tall<T>(TALL_QR2, qa, c->plan, s));
    mark(c);
    sp.stride = qa.part_stride;
    sp.out = c->G2;
    sp.rect = 0;
    sp.tri = 1;
    sp.tri_off = 0;
    sp.check = c->st;
    sp.counter = c->sum_counter;
    sp.devmax = c->g2dev;
    POD_TRY(launch_sum_parts(sp, c->cmax, s));
    mark(c);
    ta.defer = 0;
    // when G2 is far from I (flagged by the QR2 pass itself) the residual
    // block was too ill-conditioned for an FP32 first Gram: redo CGS with a
    // compensated Gram, the Cholesky and QR2; otherwise these return at once
    {
        TallArgs<T> tr = ta;
        tr.cond = 1;
        SmallArgs sr = sm;
        sr.cond = 1;
        tr.part_stride = sPG;
        tr.out = c->PG;
        POD_TRY(launch_tall<T>(TALL_CGS, tr, c->plan, s));
        mark(c);
        POD_TRY(launch_small_chol(sr, s));
        mark(c);
        TallArgs<T> qr = qa;   // reads the Z the rerun of CGS stored again
        qr.cond = 1;
        qr.defer = 0;
        POD_TRY(launch_tall<T>(TALL_QR2, qr, c->plan, s));
        mark(c);
    }
    POD_TRY(launch_core(sm, s));
    mark(c);
    {
        // U <- U X + W Y with the W the QR2 pass stored (the one whose Gram gave R2)
        TallArgs<T> ua = ta;
        ua.A = (const T *)c->Wbuf;
        ua.idx = nullptr;
        ua.lda = c->p.m;
        ua.Wout = nullptr;
        ua.vec = (c->p.m * (int64_t)sizeof(T)) % 16 == 0;
        ua.finish = c->upd_counter;   // its last CTA also ends the round
        POD_TRY(launch_tall<T>(TALL_UPDATE, ua, c->plan, s));
        mark(c);
    }
    return POD_OK;
}

static pod_status enqueue_round_any(pod_ctx *c) {
    return c->p.dtype == POD_F32 ? enqueue_round<float>(c) : enqueue_round<double>(c);
}

static pod_status build_graph(pod_ctx *c) {
    if (c->graph_ready || c->graph_failed) return POD_OK;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        cudaGetLastError();
        c->graph_failed = true;
        return POD_OK;
    }
    const long long before = c->launches;
    pod_status st = enqueue_round_any(c);
    c->graph_kernels = (int)(c->launches - before);
    c->launches = before;
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (st != POD_OK || e != cudaSuccess || !g) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        c->graph_failed = true;
        return st == POD_EUNSUPPORTED ? st : POD_OK;
    }
    if (cudaGraphInstantiate(&c->graph, g, 0) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        c->graph_failed = true;
        return POD_OK;
    }
    cudaGraphDestroy(g);
    c->graph_ready = true;
    return POD_OK;
}

static pod_status read_state(pod_ctx *c) {
    POD_CUDA_TRY(cudaMemcpyAsync(c->hstate, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
    POD_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return POD_OK;
}

template <typename T>
static pod_status run_refine(pod_ctx *c) {
    cudaStream_t s = c->stream;
    const int r = c->hstate->r_cur;
    const int64_t m = c->p.m, n = c->p.n;
    if (r == 0) return POD_OK;
    if (c->p.keep_tape) {
        // U_T, the basis the refinement starts from, for pod_backward
        const int T_ = c->hstate->rounds_run;
        POD_TRY(tape_reserve(c, T_ + 1));
        POD_CUDA_TRY(cudaMemcpyAsync((T *)c->tape_h.U + (int64_t)T_ * m * c->rmax, c->U, (size_t)m * r * sizeof(T),
                                     cudaMemcpyDeviceToDevice, s));
    }
    // Y = A^T U
    k_set_state<<<1, 32, 0, s>>>(c->aux + 0, r, 0, 0, 1, 1);
    mark(c);
    POD_TRY(enqueue_atu<T>(c, c->aux + 0, nullptr, s));
    mark(c);
    // G = Y^T Y, CholeskyQR2 on the n x r matrix Y (FP64 tall passes)
    TallPlan yplan = tall_plan(POD_F64, n, r, r, c->sms);
    TallArgs<double> ya{};
    ya.m = n;
    ya.A = c->Y;
    ya.lda = n;
    ya.idx = nullptr;
    ya.U = c->Y;
    ya.ldu = n;
    ya.rmax = r;
    ya.cmax = r;
    ya.bm = yplan.bm;
    ya.part = c->part;
    ya.part_stride = (int64_t)r * r;
    ya.gsum = c->gsum;
    ya.counters = c->counters;
    ya.vec = (n % 2) == 0;
    ya.gscratch = yplan.wide ? c->ytall_gs : nullptr;
    ya.gstride = yplan.gstride;
    if (yplan.wide && !c->ytall_gs) return POD_EUNSUPPORTED;
    if ((size_t)yplan.grid * r * r > c->part_cap || (size_t)(yplan.groups + 1) * r * r > c->gsum_cap ||
        (size_t)yplan.groups + 1 > c->counters_cap)
        return POD_EUNSUPPORTED;
    k_set_state<<<1, 32, 0, s>>>(c->aux + 1, r, r, 0, 1, 1);
    mark(c);
    ya.st = c->aux + 1;
    ya.out = c->rG;
    POD_TRY(launch_tall<double>(TALL_PROJ, ya, yplan, s));
    mark(c);
    RefineArgs ra{};
    ra.r = r;
    ra.dtype = c->p.dtype;
    ra.G = c->rG;
    ra.G2 = c->rG2;
    ra.M1 = c->rM1;
    ra.R1p = c->rR1p;
    ra.sigma = c->rsig;
    ra.VR = c->rVR;
    ra.K = c->rK;
    ra.gws = c->refine_gs;
    POD_TRY(launch_refine_chol(ra, s));
    mark(c);
    k_set_state<<<1, 32, 0, s>>>(c->aux + 2, 0, r, 0, 1, 1);
    mark(c);
    ya.st = c->aux + 2;
    ya.M1 = c->rM1;
    ya.out = c->rG2;
    POD_TRY(launch_tall<double>(TALL_QR2, ya, yplan, s));
    mark(c);
    POD_TRY(launch_refine_svd(ra, s));
    mark(c);
    // U <- U V_R (in place)
    k_set_state<<<1, 32, 0, s>>>(c->aux + 3, r, 0, r, 1, 1);
    mark(c);
    TallArgs<T> ua = tall_args<T>(c, c->part, 0);
    ua.st = c->aux + 3;
    ua.rmax = r;
    ua.cmax = c->cmax;
    ua.Xm = c->rVR;
    ua.Ym = c->Ym;
    TallPlan uplan = tall_plan(c->p.dtype, m, r, c->cmax, c->sms);
    ua.bm = uplan.bm;
    ua.gscratch = uplan.wide ? c->tall_gs : nullptr;   // (r, cmax) needs no more than the round's plan
    ua.gstride = uplan.gstride;
    POD_TRY(launch_tall<T>(TALL_UPDATE, ua, uplan, s));
    mark(c);
    POD_CUDA_TRY(cudaMemcpyAsync(c->sigma, c->rsig, r * sizeof(double), cudaMemcpyDeviceToDevice, s));
    c->refined = true;
    c->refined_r = r;
    return POD_OK;
}

template <typename T>
static pod_status write_modes(pod_ctx *c, void *U_dev, double *sigma_dev, void *V_dev) {
    cudaStream_t s = c->stream;
    const int r = c->hstate->r_cur, k = c->p.k;
    const int64_t m = c->p.m, n = c->p.n;
    if (r > 0) {
        POD_TRY(launch_sign_dots<T>((const T *)c->U, m, m, r, c->p.seed, c->part_sign, c->sign_grid, s));
        POD_TRY(launch_reduce(c->part_sign, c->sign_grid, r, r, c->dots, nullptr, s));
        c->launches += 2;
    }
    int grid = (int)((m * k + 255) / 256);
    if (grid > 4 * c->sms) grid = 4 * c->sms;
    if (grid < 1) grid = 1;
    k_write_modes<T><<<grid, 256, 0, s>>>((const T *)c->U, m, r, k, c->sigma, c->dots, (T *)U_dev, sigma_dev);
    POD_CUDA_TRY(cudaGetLastError());
    c->launches += 1;
    if (V_dev) {
        int gv = (int)((n * k + 255) / 256);
        if (gv > 4 * c->sms) gv = 4 * c->sms;
        if (gv < 1) gv = 1;
        k_write_v<T><<<gv, 256, 0, s>>>(c->Y, c->rK, n, c->refined ? c->refined_r : 0, k, c->dots, (T *)V_dev);
        POD_CUDA_TRY(cudaGetLastError());
        c->launches += 1;
    }
    return POD_OK;
}

// Adjoint of the truncated POD with the draws of the forward run held fixed:
// the refinement first (when it ran), then the merges in reverse order, each
// as a Gram pass, a one-CTA coefficient kernel and a row-mix pass that writes
// the next basis adjoint and adds the sampled columns' adjoint into dA.
template <typename T>
static pod_status run_backward(pod_ctx *c, const void *dU_dev, const double *dsigma_dev, void *dA_dev,
                               int32_t accumulate) {
    cudaStream_t s = c->stream;
    POD_TRY(read_state(c));
    const int T_ = c->hstate->rounds_run;
    const int k = c->p.k, rmax = c->rmax, cmax = c->cmax, nmax = rmax + cmax;
    const int64_t m = c->p.m, n = c->p.n, lda = c->p.lda;
    const int rT = c->hstate->r_cur;
    if (T_ + 1 > c->tape_h.cap) return POD_EUNSUPPORTED;
    if (rT < 1) return POD_ESTATE;
    const TapeLayout TL = tape_layout(rmax, cmax);
    // per-round sizes from the tape
    double *meta = (double *)malloc((size_t)(T_ > 0 ? T_ : 1) * 4 * sizeof(double));
    if (!meta) return POD_ENOMEM;
    if (T_ > 0 && cudaMemcpy2DAsync(meta, 4 * sizeof(double), c->tape_h.core, TL.stride * sizeof(double),
                                    4 * sizeof(double), T_, cudaMemcpyDeviceToHost, s) != cudaSuccess) {
        cudaGetLastError();
        free(meta);
        return POD_ECUDA;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        free(meta);
        return POD_ECUDA;
    }
    const int es = (int)sizeof(T);
    const int maxcols = rmax + cmax + rmax;
    BwdGramPlan gp = bwd_gram_plan(c->p.dtype, m, maxcols > rmax + k ? maxcols : rmax + k, c->sms);
    T *GU[2] = {nullptr, nullptr}, *AY = nullptr, *Lref = nullptr;
    double *G = nullptr, *part = nullptr, *gsum = nullptr, *coef = nullptr, *work = nullptr, *sb[2] = {nullptr, nullptr};
    double *coefL = nullptr, *coefT = nullptr;
    unsigned *cnt = nullptr;
    const size_t gmax = (size_t)(rmax + cmax) * maxcols > (size_t)rmax * (rmax + k) ? (size_t)(rmax + cmax) * maxcols
                                                                                   : (size_t)rmax * (rmax + k);
    pod_status st = POD_OK;
#define BALLOC(ptr, cnt_) if (st == POD_OK) st = dalloc(&(ptr), (size_t)(cnt_))
    BALLOC(GU[0], (size_t)m * rmax);
    BALLOC(GU[1], (size_t)m * rmax);
    BALLOC(AY, (size_t)m * rmax);
    BALLOC(Lref, (size_t)m * rmax);
    BALLOC(G, gmax);
    BALLOC(part, (size_t)gp.grid * gmax);
    BALLOC(gsum, (size_t)(gp.groups + 1) * gmax);
    BALLOC(coef, (size_t)maxcols * maxcols);
    BALLOC(work, (size_t)6 * nmax * nmax + 2 * rmax * rmax);
    BALLOC(sb[0], rmax > k ? rmax : k);
    BALLOC(sb[1], rmax > k ? rmax : k);
    BALLOC(coefL, (size_t)rmax * rmax);
    BALLOC(coefT, (size_t)(k + rmax) * rmax);
    BALLOC(cnt, gp.groups + 1);
#undef BALLOC
    if (st == POD_OK && cudaMemsetAsync(cnt, 0, (gp.groups + 1) * sizeof(unsigned), s) != cudaSuccess) st = POD_ECUDA;
    auto gram = [&](const void *p0, int64_t ld0, const int32_t *i0, int n0, const void *p1, int64_t ld1,
                    const int32_t *i1, int n1, const void *p2, int64_t ld2, int n2, int nleft) {
        BwdGram ga{};
        ga.ptr[0] = p0; ga.ld[0] = ld0; ga.idx[0] = i0; ga.ncol[0] = n0;
        ga.ptr[1] = p1; ga.ld[1] = ld1; ga.idx[1] = i1; ga.ncol[1] = n1;
        ga.ptr[2] = p2; ga.ld[2] = ld2; ga.idx[2] = nullptr; ga.ncol[2] = n2;
        ga.nleft = nleft;
        ga.m = m;
        ga.rows_per = gp.rows_per;
        ga.lds = gp.lds;
        ga.part = part;
        ga.gsum = gsum;
        ga.out = G;
        ga.counters = cnt;
        c->launches += 1;
        return launch_bwd_gram<T>(ga, gp, s);
    };
    const T *Ufin = (const T *)c->U;
    // ------------------------------------------------ refinement
    if (st == POD_OK) {
        if (c->refined) {
            const int r = c->refined_r;
            st = gram(Ufin, m, nullptr, r, dU_dev, m, nullptr, k, nullptr, 0, 0, 1);
            BwdRefine br{};
            br.r = r;
            br.k = k;
            br.G = G;
            br.ldg = r + k;
            br.goff = r;
            br.S = c->rsig;
            br.VR = c->rVR;
            br.K = c->rK;
            br.dots = c->dots;
            br.dsigma = dsigma_dev;
            br.work = work;
            br.coefL = coefL;
            br.coefT = coefT;
            if (st == POD_OK) st = launch_bwd_refine_small(br, s);
            if (st == POD_OK) st = launch_az<T>((const T *)c->A, m, n, lda, c->Y, r, AY, s);
            RowMix rm{};
            rm.m = m;
            rm.in[0] = Ufin; rm.ldi[0] = m; rm.pin[0] = r;
            rm.out[0] = Lref; rm.ldo[0] = m; rm.qout[0] = r;
            rm.coef = coefL;
            if (st == POD_OK) st = launch_rowmix<T>(rm, s);
            if (st == POD_OK) st = launch_outer<T>((T *)dA_dev, m, n, lda, Lref, r, c->Y, accumulate, s);
            RowMix rt{};
            rt.m = m;
            rt.in[0] = dU_dev; rt.ldi[0] = m; rt.pin[0] = k;
            rt.in[1] = AY; rt.ldi[1] = m; rt.pin[1] = r;
            rt.out[0] = GU[0]; rt.ldo[0] = m; rt.qout[0] = r;
            rt.coef = coefT;
            if (st == POD_OK) st = launch_rowmix<T>(rt, s);
            if (st == POD_OK && cudaMemsetAsync(sb[0], 0, rmax * sizeof(double), s) != cudaSuccess) st = POD_ECUDA;
            c->launches += 5;
        } else {
            // U_fin = U_T: only the sign fix lies between the rounds and the output
            double *hc = (double *)calloc((size_t)k * rT, sizeof(double));
            double *hd = (double *)malloc((size_t)rT * sizeof(double));
            double *hs = (double *)calloc((size_t)rT, sizeof(double));
            if (!hc || !hd || !hs) st = POD_ENOMEM;
            if (st == POD_OK && (cudaMemcpy(hd, c->dots, rT * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
                                 (dsigma_dev && cudaMemcpy(hs, dsigma_dev, (k < rT ? k : rT) * sizeof(double),
                                                           cudaMemcpyDeviceToHost) != cudaSuccess)))
                st = POD_ECUDA;
            if (st == POD_OK) {
                for (int l = 0; l < k && l < rT; ++l) hc[l * rT + l] = hd[l] < 0.0 ? -1.0 : 1.0;
                if (cudaMemcpy(coefT, hc, (size_t)k * rT * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
                    cudaMemcpy(sb[0], hs, rT * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
                    st = POD_ECUDA;
            }
            free(hc);
            free(hd);
            free(hs);
            RowMix rt{};
            rt.m = m;
            rt.in[0] = dU_dev; rt.ldi[0] = m; rt.pin[0] = k;
            rt.out[0] = GU[0]; rt.ldo[0] = m; rt.qout[0] = rT;
            rt.coef = coefT;
            if (st == POD_OK) st = launch_rowmix<T>(rt, s);
            if (st == POD_OK && !accumulate &&
                cudaMemset2DAsync(dA_dev, (size_t)lda * es, 0, (size_t)m * es, (size_t)n, s) != cudaSuccess)
                st = POD_ECUDA;
        }
    }
    // ------------------------------------------------ merges, last to first
    int cur = 0;
    for (int t = T_ - 1; t >= 0 && st == POD_OK; --t) {
        const int r = (int)meta[4 * t + 0], g = (int)meta[4 * t + 1], rp = (int)meta[4 * t + 2];
        const T *Ut = (const T *)c->tape_h.U + (int64_t)t * m * rmax;
        const int32_t *idx = c->hist_idx + (int64_t)t * c->p.c;
        st = gram(Ut, m, nullptr, r, c->A, lda, idx, g, GU[cur], m, rp, 2);
        BwdMerge bm{};
        bm.rec = c->tape_h.core + (int64_t)t * TL.stride;
        bm.rmax = rmax;
        bm.cmax = cmax;
        bm.dtype = c->p.dtype;
        bm.G = G;
        bm.sbar = sb[cur];
        bm.work = work;
        bm.coef = coef;
        bm.sbar_out = sb[cur ^ 1];
        if (st == POD_OK) st = launch_bwd_merge_small(bm, s);
        RowMix rm{};
        rm.m = m;
        rm.in[0] = Ut; rm.ldi[0] = m; rm.pin[0] = r;
        rm.in[1] = c->A; rm.ldi[1] = lda; rm.idx_in[1] = idx; rm.pin[1] = g;
        rm.in[2] = GU[cur]; rm.ldi[2] = m; rm.pin[2] = rp;
        rm.out[0] = GU[cur ^ 1]; rm.ldo[0] = m; rm.qout[0] = r;
        rm.out[1] = dA_dev; rm.ldo[1] = lda; rm.idx_out[1] = idx; rm.qout[1] = g; rm.acc_out[1] = 1;
        rm.coef = coef;
        if (st == POD_OK) st = launch_rowmix<T>(rm, s);
        c->launches += 2;
        cur ^= 1;
    }
    if (st == POD_OK && cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        st = POD_ECUDA;
    }
    cudaStreamSynchronize(s);
    void *bufs[] = {GU[0], GU[1], AY, Lref, G, part, gsum, coef, work, sb[0], sb[1], coefL, coefT, cnt};
    for (void *b : bufs)
        if (b) cudaFree(b);
    free(meta);
    return st;
}

extern "C" {

const char *pod_strerror(pod_status s) {
    switch (s) {
        case POD_OK: return "ok";
        case POD_EINVAL: return "invalid argument";
        case POD_ENOMEM: return "out of memory";
        case POD_ECUDA: return "CUDA runtime error";
        case POD_ERANK: return "Cholesky breakdown";
        case POD_ETIMEOUT: return "bounded device wait gave up";
        case POD_ENAN: return "non-finite value in the core";
        case POD_ESTATE: return "call not valid in the context's state";
        case POD_EUNSUPPORTED: return "unsupported size or option in this build";
    }
    return "unknown status";
}

pod_status pod_init(pod_ctx **ctx_out, const pod_params *p, const void *A_dev, void *stream) {
    if (!ctx_out) return POD_EINVAL;
    *ctx_out = nullptr;
    POD_TRY(check_params(p));
    if (!A_dev) return POD_EINVAL;
    pod_ctx *c = (pod_ctx *)calloc(1, sizeof(pod_ctx));
    if (!c) return POD_ENOMEM;
    c->p = *p;
    c->A = A_dev;
    c->stream = (cudaStream_t)stream;
    c->rmax = p->r > 0 ? p->r : p->k;
    c->cmax = p->c;
    c->nmax = c->rmax + c->cmax;
    c->rtrunc = c->rmax;
    c->core_f64 = p->core == POD_CORE_F64 || (p->core == POD_CORE_AUTO && p->dtype == POD_F64);
    c->sms = device_sms();
    c->plan = tall_plan(p->dtype, p->m, c->rmax, c->cmax, c->sms);
    c->aplan = atu_plan(p->dtype, p->m, p->n, c->rmax, c->sms);
    {
        const size_t esz = p->dtype == POD_F32 ? 4 : 8;
        c->vec = ((uintptr_t)A_dev % 16 == 0) && ((p->lda * esz) % 16 == 0) && ((p->m * esz) % 16 == 0);
    }
    if (p->rows) {
        c->wdraws = (int)(p->w > 0 ? p->w : default_row_draws(p->k, p->m));   // draws with replacement: w may exceed m
        c->rnb = row_blocks(p->m);
        c->gplan = row_gram_plan(p->dtype, c->wdraws, c->cmax, c->sms);
    } else if (p->block_trunc) {
        c->gplan = row_gram_plan(p->dtype, p->m, c->cmax, c->sms);
    }
    if (p->precision != POD_PREC_F32) {
        if (!xty_tc_supported(p->dtype, p->m, p->lda, c->rmax, A_dev, A_dev)) {
            free(c);
            return POD_EUNSUPPORTED;
        }
        c->use_tc = 1;
        c->tcplan = xty_tc_plan(p->precision, p->m, p->n, c->rmax, c->sms, 0);
        c->pplan = xty_tc_plan(p->precision, p->m, c->cmax, c->rmax, c->sms, 1);
        // the deferred partials use the round's partial buffer (plan.grid slots)
        c->use_tc_proj = c->pplan.grid <= c->plan.grid;
    }
    if ((p->rows || p->block_trunc) && rows_small_smem(c->cmax) > 220 * 1024) {
        free(c);
        return POD_EUNSUPPORTED;
    }
    const bool wide_core = core_smem_bytes(c->rmax, c->cmax, c->core_f64 ? POD_F64 : POD_F32) > 220 * 1024;
    // global scratch when one of the forms this context runs (plain, the
    // compensated rerun) does not fit in shared memory
    const size_t chol_bytes = small_chol_smem(c->cmax, p->dtype, 1) > small_chol_smem(c->cmax, p->dtype, 0)
                                  ? small_chol_smem(c->cmax, p->dtype, 1) : small_chol_smem(c->cmax, p->dtype, 0);
    const bool wide_chol = chol_bytes > 220 * 1024;
    const bool wide_refine = refine_gws_bytes(c->rmax) > 220 * 1024;
    c->jac_smem = wide_core && core_jacobi_bytes(c->rmax, c->cmax, c->core_f64 ? POD_F64 : POD_F32) <= 200 * 1024;
    if (wide_core && (p->rows || p->block_trunc)) {
        free(c);
        return POD_EUNSUPPORTED;
    }
    if (c->plan.smem > 227 * 1024) {
        free(c);
        return POD_EUNSUPPORTED;
    }
    const size_t es = p->dtype == POD_F32 ? 4 : 8;
    const int64_t m = p->m, n = p->n;
    const int rm = c->rmax, cm = c->cmax, nm = c->nmax;
    pod_status st = POD_OK;
#define ALLOC(ptr, cnt) if (st == POD_OK) st = dalloc(&(ptr), (size_t)(cnt))
    unsigned char *Ub = nullptr;
    ALLOC(Ub, (size_t)m * rm * es);
    c->U = Ub;
    unsigned char *Wb = nullptr;
    ALLOC(Wb, (size_t)m * cm * es);
    c->Wbuf = Wb;
    ALLOC(c->sum_counter, 1);
    ALLOC(c->upd_counter, 1);
    ALLOC(c->g2dev, 1);
    ALLOC(c->sigma, rm);
    ALLOC(c->s, n);
    ALLOC(c->ort, n);
    ALLOC(c->Y, (size_t)n * rm);
    ALLOC(c->mask, n);
    ALLOC(c->flags, n);
    ALLOC(c->w, n);
    ALLOC(c->cdf, n);
    ALLOC(c->draws, cm);
    ALLOC(c->idx, cm);
    ALLOC(c->hist_idx, (size_t)(n + 1) * cm);
    ALLOC(c->hist_g, n + 1);
    ALLOC(c->hist_measure, n + 1);
    ALLOC(c->st, 1);
    ALLOC(c->aux, 6);
    {
        // the round's tall passes and the refinement's Gram of Y = A^T U
        // (n x r, FP64) share the partial buffers: size them for both
        const TallPlan yp = tall_plan(POD_F64, n, rm, rm, c->sms);
        c->part_cap = (size_t)c->plan.grid * ((size_t)rm * cm + (size_t)cm * cm);
        if ((size_t)yp.grid * rm * rm > c->part_cap) c->part_cap = (size_t)yp.grid * rm * rm;
        c->gsum_cap = (size_t)(c->plan.groups + 1) * ((size_t)rm * cm + (size_t)cm * cm);
        if ((size_t)(yp.groups + 1) * rm * rm > c->gsum_cap) c->gsum_cap = (size_t)(yp.groups + 1) * rm * rm;
        c->counters_cap = 64 + (c->plan.groups > yp.groups ? c->plan.groups : yp.groups);
    }
    ALLOC(c->part, c->part_cap);
    ALLOC(c->part_atu, (size_t)c->aplan.split * n * rm);
    ALLOC(c->P, (size_t)rm * cm);
    ALLOC(c->gsum, c->gsum_cap);
    ALLOC(c->counters, c->counters_cap);
    ALLOC(c->atu_counters, (size_t)c->aplan.grid.x + 64);
    ALLOC(c->PG, (size_t)rm * cm + (size_t)cm * cm);
    ALLOC(c->G2, (size_t)cm * cm);
    ALLOC(c->Ptot, (size_t)rm * cm);
    ALLOC(c->M1, (size_t)cm * cm);
    ALLOC(c->R1p, (size_t)cm * cm);
    ALLOC(c->E, (size_t)nm * nm + (size_t)cm * cm);
    ALLOC(c->Xm, (size_t)rm * rm);
    ALLOC(c->Ym, (size_t)cm * rm);
    ALLOC(c->rG, (size_t)rm * rm);
    ALLOC(c->rG2, (size_t)rm * rm);
    ALLOC(c->rM1, (size_t)rm * rm);
    ALLOC(c->rR1p, (size_t)rm * rm);
    ALLOC(c->rsig, rm);
    ALLOC(c->rVR, (size_t)rm * rm);
    ALLOC(c->rK, (size_t)rm * rm);
    ALLOC(c->dots, rm);
    c->sign_grid = 2 * c->sms;
    ALLOC(c->part_sign, (size_t)c->sign_grid * rm);
    if (p->rows) {
        const int nb = c->rnb;
        ALLOC(c->r_val, m);
        ALLOC(c->r_bmax, nb);
        ALLOC(c->r_bsum, nb);
        ALLOC(c->r_boff, nb);
        ALLOC(c->r_total, 1);
        ALLOC(c->r_w, m);
        ALLOC(c->r_cdf, m);
        ALLOC(c->r_cnt, m);
        ALLOC(c->r_rows, c->wdraws);
        ALLOC(c->r_rcnt, c->wdraws);
        ALLOC(c->r_rscale, c->wdraws);
        ALLOC(c->r_h, 1);
    }
    if (p->keep_tape) ALLOC(c->tape_d, 1);
    if (c->plan.wide) ALLOC(c->tall_gs, (size_t)c->plan.grid * c->plan.gstride);
    if (wide_core) ALLOC(c->core_gs, core_smem_bytes(c->rmax, c->cmax, c->core_f64 ? POD_F64 : POD_F32));
    if (wide_chol) ALLOC(c->chol_gs, chol_bytes);
    if (wide_refine) ALLOC(c->refine_gs, refine_gws_bytes(c->rmax));
    {
        const TallPlan yp = tall_plan(POD_F64, n, rm, rm, c->sms);
        if (yp.wide) ALLOC(c->ytall_gs, (size_t)yp.grid * yp.gstride);
    }
    if (c->use_tc) {
        ALLOC(c->tc_part, c->tcplan.part_doubles);
        ALLOC(c->tc_counters, c->tcplan.mtiles);
    }
    if (p->rows || p->block_trunc) {
        unsigned char *Cb = nullptr;
        ALLOC(Cb, (size_t)m * rm * es);
        c->Cbuf = Cb;
        ALLOC(c->GW, (size_t)cm * cm);
        ALLOC(c->rYm, (size_t)cm * rm);
        ALLOC(c->wR1p, (size_t)cm * cm);
        ALLOC(c->wG2, (size_t)cm * cm);
        ALLOC(c->wM1, (size_t)cm * cm);
        ALLOC(c->wsig, rm);
        ALLOC(c->wX, (size_t)rm * rm);
        ALLOC(c->part_w, (size_t)c->gplan.grid * cm * cm);
        ALLOC(c->gsum_w, (size_t)(c->gplan.groups + 1) * cm * cm);
        ALLOC(c->counters_w, c->gplan.groups + 1);
    }
#undef ALLOC
    if (st == POD_OK && cudaMallocHost((void **)&c->hstate, sizeof(DevState)) != cudaSuccess) {
        cudaGetLastError();
        st = POD_ENOMEM;
    }
    if (st != POD_OK) {
        ctx_free(c);
        return st;
    }
    cudaStream_t s = c->stream;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemsetAsync(c->U, 0, (size_t)m * rm * es, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->sigma, 0, rm * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->mask, 1, n, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->flags, 0, n, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ort, 0, n * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->part, 0, (size_t)c->plan.grid * ((size_t)rm * cm + (size_t)cm * cm) * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->P, 0, (size_t)rm * cm * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->PG, 0, ((size_t)rm * cm + (size_t)cm * cm) * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->hist_g, 0, (n + 1) * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->counters, 0, c->counters_cap * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->atu_counters, 0, (c->aplan.grid.x + 64) * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->sum_counter, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->upd_counter, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->g2dev, 0, sizeof(unsigned long long), s);
    if (p->rows) {
        if (e == cudaSuccess) e = cudaMemsetAsync(c->r_cnt, 0, (size_t)m * sizeof(unsigned), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->r_h, 0, sizeof(int32_t), s);
    }
    if (p->rows || p->block_trunc)
        if (e == cudaSuccess) e = cudaMemsetAsync(c->counters_w, 0, (c->gplan.groups + 1) * sizeof(unsigned), s);
    if (c->use_tc && e == cudaSuccess) e = cudaMemsetAsync(c->tc_counters, 0, c->tcplan.mtiles * sizeof(unsigned), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx_free(c);
        return POD_ECUDA;
    }
    if (p->keep_tape) {
        const TapePtrs z{nullptr, nullptr, 0};
        if (cudaMemcpy(c->tape_d, &z, sizeof(TapePtrs), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            ctx_free(c);
            return POD_ECUDA;
        }
        const int64_t est = 2 * ((n + p->c - 1) / p->c) + 4;
        pod_status ts = tape_reserve(c, (int)(est < n + 1 ? est : n + 1));
        if (ts != POD_OK) {
            ctx_free(c);
            return ts;
        }
    }
    k_set_state<<<1, 32, 0, s>>>(c->st, 0, 0, 0, 0, (int)n);
    mark(c);
    pod_status ls = launch_colnorms(A_dev, p->dtype, m, n, p->lda, c->s, s);
    mark(c);
    if (ls == POD_OK && cudaGetLastError() != cudaSuccess) ls = POD_ECUDA;
    if (ls != POD_OK) {
        ctx_free(c);
        return ls;
    }
    memset(c->hstate, 0, sizeof(DevState));
    c->hstate->remaining = (int)n;
    *ctx_out = c;
    return POD_OK;
}

pod_status pod_iterate(pod_ctx *c, int32_t max_steps, int32_t *done, double *sin_max, int32_t *steps_run) {
    if (!c) return POD_EINVAL;
    if (c->poisoned) return POD_ESTATE;
    if (max_steps <= 0) return POD_EINVAL;
    if (c->refined) return POD_ESTATE;
    pod_status st = build_graph(c);
    if (st != POD_OK) return st;
    const int before = c->hstate->rounds_run;
    int launched = 0;
    while (launched < max_steps && !c->hstate->done) {
        int chunk = (c->hstate->remaining + c->p.c - 1) / c->p.c;
        if (chunk < 1) chunk = 1;
        if (chunk > 64) chunk = 64;
        if (chunk > max_steps - launched) chunk = max_steps - launched;
        if (c->p.keep_tape) {
            st = tape_reserve(c, c->hstate->t + chunk + 1);
            if (st != POD_OK) return st;
        }
        for (int i = 0; i < chunk; ++i) {
            if (c->graph_ready) {
                if (cudaGraphLaunch(c->graph, c->stream) != cudaSuccess) {
                    cudaGetLastError();
                    c->poisoned = true;
                    return POD_ECUDA;
                }
                c->launches += c->graph_kernels;
            } else {
                st = enqueue_round_any(c);
                if (st != POD_OK) {
                    if (st == POD_ECUDA) c->poisoned = true;
                    return st;
                }
            }
        }
        launched += chunk;
        st = read_state(c);
        if (st != POD_OK) {
            c->poisoned = true;
            return st;
        }
        if (c->hstate->status != 0) break;
    }
    if (done) *done = c->hstate->done;
    if (sin_max) *sin_max = c->hstate->measure;
    if (steps_run) *steps_run = c->hstate->rounds_run - before;
    if (c->hstate->status != 0) {
        c->poisoned = true;   // POD_ENAN, POD_ERANK, POD_ETIMEOUT: the run's state is not usable
        return (pod_status)c->hstate->status;
    }
    return POD_OK;
}

pod_status pod_modes(pod_ctx *c, void *U_dev, double *sigma_dev, void *V_dev) {
    if (!c || !U_dev || !sigma_dev) return POD_EINVAL;
    if (c->poisoned) return POD_ESTATE;
    if (V_dev && !c->p.refine) return POD_EINVAL;
    pod_status st = read_state(c);
    if (st != POD_OK) {
        c->poisoned = true;
        return st;
    }
    if (c->p.refine && !c->refined) {
        st = c->p.dtype == POD_F32 ? run_refine<float>(c) : run_refine<double>(c);
        if (st == POD_OK) st = read_state(c);
        if (st == POD_OK && c->hstate->status != 0) st = (pod_status)c->hstate->status;
        if (st != POD_OK) {
            if (st == POD_ECUDA || st == POD_ETIMEOUT || st == POD_ENAN) c->poisoned = true;
            return st;
        }
    }
    st = c->p.dtype == POD_F32 ? write_modes<float>(c, U_dev, sigma_dev, V_dev)
                               : write_modes<double>(c, U_dev, sigma_dev, V_dev);
    if (st == POD_ECUDA) c->poisoned = true;
    if (st == POD_OK) c->modes_done = true;
    return st;
}

pod_status pod_get_trace(pod_ctx *c, int32_t t, int32_t *idx_host, int32_t *g_host, double *measure_host) {
    if (!c) return POD_EINVAL;
    if (c->poisoned) return POD_ESTATE;
    pod_status st = read_state(c);
    if (st != POD_OK) return st;
    if (t < 0 || t >= c->hstate->rounds_run) return POD_EINVAL;
    int32_t g = 0;
    POD_CUDA_TRY(cudaMemcpy(&g, c->hist_g + t, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (g_host) *g_host = g;
    if (idx_host && g > 0)
        POD_CUDA_TRY(cudaMemcpy(idx_host, c->hist_idx + (int64_t)t * c->p.c, g * sizeof(int32_t),
                                cudaMemcpyDeviceToHost));
    if (measure_host)
        POD_CUDA_TRY(cudaMemcpy(measure_host, c->hist_measure + t, sizeof(double), cudaMemcpyDeviceToHost));
    return POD_OK;
}

pod_status pod_replay_indices(pod_ctx *c, const int32_t *idx_host, const int32_t *offsets_host, int32_t T) {
    if (!c || !idx_host || !offsets_host || T < 0 || T > c->p.n) return POD_EINVAL;
    if (c->poisoned || c->graph_ready || c->hstate->rounds_run > 0) return POD_ESTATE;
    const int32_t total = offsets_host[T];
    if (offsets_host[0] != 0 || total < 0) return POD_EINVAL;
    for (int t = 0; t < T; ++t) {
        const int len = offsets_host[t + 1] - offsets_host[t];
        if (len < 0 || len > c->p.c) return POD_EINVAL;
    }
    for (int i = 0; i < total; ++i)
        if (idx_host[i] < 0 || idx_host[i] >= c->p.n) return POD_EINVAL;
    if (c->replay_idx) cudaFree(c->replay_idx);
    if (c->replay_off) cudaFree(c->replay_off);
    c->replay_idx = nullptr;
    c->replay_off = nullptr;
    POD_TRY(dalloc(&c->replay_idx, total > 0 ? total : 1));
    POD_TRY(dalloc(&c->replay_off, T + 1));
    if (total > 0)
        POD_CUDA_TRY(cudaMemcpy(c->replay_idx, idx_host, total * sizeof(int32_t), cudaMemcpyHostToDevice));
    POD_CUDA_TRY(cudaMemcpy(c->replay_off, offsets_host, (T + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
    c->replay_T = T;
    return POD_OK;
}

pod_status pod_backward(pod_ctx *c, const void *dU_dev, const double *dsigma_dev, void *dA_dev,
                        int32_t accumulate) {
    if (!c || !dU_dev || !dA_dev) return POD_EINVAL;
    if (c->poisoned) return POD_ESTATE;
    if (!c->p.keep_tape || !c->modes_done) return POD_ESTATE;
    pod_status st = c->p.dtype == POD_F32 ? run_backward<float>(c, dU_dev, dsigma_dev, dA_dev, accumulate)
                                          : run_backward<double>(c, dU_dev, dsigma_dev, dA_dev, accumulate);
    if (st == POD_ECUDA) c->poisoned = true;
    return st;
}

pod_status pod_last_rows(pod_ctx *c, int32_t *rows_host, int32_t *counts_host, int32_t cap, int32_t *h) {
    if (!c || !h) return POD_EINVAL;
    if (c->poisoned) return POD_ESTATE;
    if (!c->p.rows) return POD_ESTATE;
    int32_t hh = 0;
    POD_CUDA_TRY(cudaMemcpyAsync(&hh, c->r_h, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    POD_CUDA_TRY(cudaStreamSynchronize(c->stream));
    *h = hh;
    if (hh > cap) return POD_EINVAL;
    if (hh > 0 && rows_host)
        POD_CUDA_TRY(cudaMemcpyAsync(rows_host, c->r_rows, (size_t)hh * 4, cudaMemcpyDeviceToHost, c->stream));
    if (hh > 0 && counts_host)
        POD_CUDA_TRY(cudaMemcpyAsync(counts_host, c->r_rcnt, (size_t)hh * 4, cudaMemcpyDeviceToHost, c->stream));
    POD_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return POD_OK;
}

pod_status pod_wedin(pod_ctx *c, double *out4) {
    if (!c || !out4) return POD_EINVAL;
    if (c->poisoned) return POD_ESTATE;
    if (!c->refined) return POD_ESTATE;
    const int k = c->p.k, r = c->refined_r;
    if (r < k + 1) return POD_EUNSUPPORTED;
    cudaStream_t s = c->stream;
    const int64_t m = c->p.m, n = c->p.n;
    const int gn = wedin_grid_n(n), gm = wedin_grid_m(m), passes = wedin_passes(k);
    const int grn = (gn + RED_GROUP - 1) / RED_GROUP, grm = (gm + RED_GROUP - 1) / RED_GROUP;
    // workspace for this call (released before returning)
    double *Vk = nullptr, *part = nullptr, *out = nullptr;
    float2 *Vkf = nullptr;
    unsigned *cnt = nullptr;
    pod_status st = dalloc(&Vk, (size_t)n * k);
    if (st == POD_OK) st = dalloc(&Vkf, (size_t)n * k);
    const size_t np = (size_t)gn + grn + 1 + gm + grm + 1;
    if (st == POD_OK) st = dalloc(&part, np);
    if (st == POD_OK) st = dalloc(&out, 1 + passes);
    if (st == POD_OK) st = dalloc(&cnt, (size_t)grn + 1 + grm + 1);
    double host[2 + 64] = {0};
    double sig2[2] = {0, 0};
    if (st == POD_OK) {
        WedinArgs a{};
        a.m = m;
        a.n = n;
        a.lda = c->p.lda;
        a.k = k;
        a.r = r;
        a.Y = c->Y;
        a.K = c->rK;
        a.VR = c->rVR;
        a.sigma = c->sigma;
        a.Vk = Vk;
        a.Vkf = Vkf;
        a.part_s = part;
        a.gsum_s = part + gn;
        a.part_r = part + gn + grn + 1;
        a.gsum_r = a.part_r + gm;
        a.out = out;
        a.counters_v = cnt;
        a.counters_r = cnt + grn + 1;
        cudaError_t e = cudaMemsetAsync(cnt, 0, ((size_t)grn + 1 + grm + 1) * sizeof(unsigned), s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            st = POD_ECUDA;
        }
        if (st == POD_OK)
            st = c->p.dtype == POD_F32 ? launch_wedin<float>(a, (const float *)c->A, (const float *)c->U, s)
                                       : launch_wedin<double>(a, (const double *)c->A, (const double *)c->U, s);
        c->launches += 1 + passes;
        if (st == POD_OK && passes + 1 <= 64) {
            if (cudaMemcpyAsync(host, out, (1 + passes) * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaMemcpyAsync(sig2, c->sigma + (k - 1), 2 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                cudaGetLastError();
                st = POD_ECUDA;
            }
        } else if (st == POD_OK) {
            st = POD_EUNSUPPORTED;
        }
    }
    cudaStreamSynchronize(s);
    cudaFree(Vk);
    cudaFree(Vkf);
    cudaFree(part);
    cudaFree(out);
    cudaFree(cnt);
    if (st != POD_OK) return st;
    double r2 = 0.0;
    for (int p = 0; p < passes; ++p) r2 += host[1 + p];
    const double s2 = host[0];
    const double sk = sig2[0], sk1 = sig2[1];
    const double gap = fabs(sk - sk1);
    const double omega = gap < sk ? gap : sk;
    out4[0] = sqrt(r2 + s2) / omega;
    out4[1] = sqrt(r2);
    out4[2] = sqrt(s2);
    out4[3] = omega;
    return POD_OK;
}

pod_status pod_row_draws(pod_ctx *c, int32_t *w) {
    if (!c || !w) return POD_EINVAL;
    *w = c->p.rows ? c->wdraws : 0;
    return POD_OK;
}

static pod_status reset_state(pod_ctx *c) {
    cudaStream_t s = c->stream;
    const size_t es = c->p.dtype == POD_F32 ? 4 : 8;
    const int64_t m = c->p.m, n = c->p.n;
    cudaError_t e = cudaMemsetAsync(c->U, 0, (size_t)m * c->rmax * es, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->sigma, 0, c->rmax * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->mask, 1, n, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ort, 0, n * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->hist_g, 0, (n + 1) * sizeof(int32_t), s);
    if (e == cudaSuccess && c->p.rows) e = cudaMemsetAsync(c->r_h, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return POD_ECUDA;
    }
    k_set_state<<<1, 32, 0, s>>>(c->st, 0, 0, 0, 0, (int)n);
    mark(c);
    POD_TRY(launch_colnorms(c->A, c->p.dtype, m, n, c->p.lda, c->s, s));
    mark(c);
    memset(c->hstate, 0, sizeof(DevState));
    c->hstate->remaining = (int)n;
    c->refined = false;
    c->refined_r = 0;
    c->modes_done = false;
    return POD_OK;
}

pod_status pod_reset(pod_ctx *c, const void *A_dev) {
    if (!c) return POD_EINVAL;
    if (c->poisoned) return POD_ESTATE;
    if (A_dev && A_dev != c->A) {
        c->A = A_dev;
        if (c->graph_ready) cudaGraphExecDestroy(c->graph);
        c->graph_ready = false;
        c->graph_failed = false;
    }
    pod_status st = reset_state(c);
    if (st == POD_ECUDA) c->poisoned = true;
    return st;
}

pod_status pod_round_timings(pod_ctx *c, float *ms_host, int32_t cap, int32_t *count) {
    if (!c || !ms_host || cap <= 0 || !count) return POD_EINVAL;
    if (c->poisoned) return POD_ESTATE;
    if (c->refined) return POD_ESTATE;
    *count = 0;
    const int nev = 24;
    cudaEvent_t ev[nev];
    for (int i = 0; i < nev; ++i)
        if (cudaEventCreate(&ev[i]) != cudaSuccess) {
            cudaGetLastError();
            for (int j = 0; j < i; ++j) cudaEventDestroy(ev[j]);
            return POD_ECUDA;
        }
    c->prof_ev = ev;
    c->prof_cap = nev;
    c->prof_n = 1;
    cudaEventRecord(ev[0], c->stream);
    pod_status st = enqueue_round_any(c);
    const int n = c->prof_n;
    c->prof_ev = nullptr;
    c->prof_cap = 0;
    c->prof_n = 0;
    if (st == POD_OK) st = read_state(c);
    if (st == POD_OK) {
        int k = 0;
        for (int i = 1; i < n && k < cap; ++i, ++k) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[i - 1], ev[i]);
            ms_host[k] = ms;
        }
        *count = k;
    }
    for (int i = 0; i < nev; ++i) cudaEventDestroy(ev[i]);
    if (st == POD_OK && c->hstate->status != 0) st = (pod_status)c->hstate->status;
    return st;
}

pod_status pod_refine_timings(pod_ctx *c, float *ms_host, int32_t cap, int32_t *count) {
    if (!c || !ms_host || cap <= 0 || !count) return POD_EINVAL;
    if (c->poisoned) return POD_ESTATE;
    if (!c->p.refine || c->refined) return POD_ESTATE;
    *count = 0;
    pod_status st = read_state(c);
    if (st != POD_OK) {
        c->poisoned = true;
        return st;
    }
    const int nev = 16;
    cudaEvent_t ev[nev];
    for (int i = 0; i < nev; ++i)
        if (cudaEventCreate(&ev[i]) != cudaSuccess) {
            cudaGetLastError();
            for (int j = 0; j < i; ++j) cudaEventDestroy(ev[j]);
            return POD_ECUDA;
        }
    c->prof_ev = ev;
    c->prof_cap = nev;
    c->prof_n = 1;
    cudaEventRecord(ev[0], c->stream);
    st = c->p.dtype == POD_F32 ? run_refine<float>(c) : run_refine<double>(c);
    const int n = c->prof_n;
    c->prof_ev = nullptr;
    c->prof_cap = 0;
    c->prof_n = 0;
    if (st == POD_OK) st = read_state(c);
    if (st == POD_OK) {
        int k = 0;
        for (int i = 1; i < n && k < cap; ++i, ++k) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[i - 1], ev[i]);
            ms_host[k] = ms;
        }
        *count = k;
    }
    for (int i = 0; i < nev; ++i) cudaEventDestroy(ev[i]);
    if (st == POD_OK && c->hstate->status != 0) st = (pod_status)c->hstate->status;
    if (st != POD_OK) c->poisoned = true;
    return st;
}

pod_status pod_core_stats(pod_ctx *c, int32_t *sweeps, int64_t *cycles) {
    if (!c) return POD_EINVAL;
    if (c->poisoned) return POD_ESTATE;
    pod_status st = read_state(c);
    if (st != POD_OK) return st;
    if (sweeps) *sweeps = c->hstate->sweeps;
    if (cycles)
        for (int i = 0; i < 6; ++i) cycles[i] = c->hstate->core_cycles[i];
    return POD_OK;
}

pod_status pod_robust_rounds(pod_ctx *c, int32_t *robust_rounds) {
    if (!c || !robust_rounds) return POD_EINVAL;
    if (c->poisoned) return POD_ESTATE;
    POD_TRY(read_state(c));
    *robust_rounds = c->hstate->robust_rounds;
    return POD_OK;
}

pod_status pod_set_wait_limit(pod_ctx *c, uint32_t polls) {
    if (!c) return POD_EINVAL;
    if (c->poisoned) return POD_ESTATE;
    c->tc_spin = polls;
    return POD_OK;
}

pod_status pod_counters(pod_ctx *c, int64_t *kernel_launches, int32_t *rounds) {
    if (!c) return POD_EINVAL;
    if (kernel_launches) *kernel_launches = c->launches;
    if (rounds) *rounds = c->hstate->rounds_run;
    return POD_OK;
}

void pod_destroy(pod_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    cudaGetLastError();
    ctx_free(c);
}

pod_status pod_colnorms(const void *A_dev, int32_t dtype, int64_t m, int64_t n, int64_t lda, double *s_dev,
                        void *stream) {
    if (!A_dev || !s_dev || m <= 0 || n <= 0 || lda < m) return POD_EINVAL;
    if (dtype != POD_F32 && dtype != POD_F64) return POD_EINVAL;
    return launch_colnorms(A_dev, dtype, m, n, lda, s_dev, (cudaStream_t)stream);
}

pod_status pod_atu(const void *A_dev, int32_t dtype, int64_t m, int64_t n, int64_t lda, const void *U_dev, int32_t r,
                   double *Y_dev, int32_t precision, void *stream) {
    if (!A_dev || !U_dev || !Y_dev || m <= 0 || n <= 0 || lda < m || r <= 0) return POD_EINVAL;
    if (dtype != POD_F32 && dtype != POD_F64) return POD_EINVAL;
    if (precision < POD_PREC_F32 || precision > POD_PREC_TF32X3) return POD_EINVAL;
    const bool tc = precision != POD_PREC_F32;
    if (tc && !xty_tc_supported(dtype, m, lda, r, A_dev, U_dev)) return POD_EUNSUPPORTED;
    if (!tc && r > 256) return POD_EUNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    const int sms = device_sms();
    DevState *stt = nullptr;
    double *part = nullptr;
    unsigned *cnt = nullptr;
    pod_status st = dalloc(&stt, 1);
    XtyTcPlan tp{};
    AtuPlan ap{};
    size_t ncnt = 0;
    if (tc) {
        tp = xty_tc_plan(precision, m, n, r, sms, 0);
        if (st == POD_OK) st = dalloc(&part, tp.part_doubles);
        ncnt = (size_t)tp.mtiles;
    } else {
        ap = atu_plan(dtype, m, n, r, sms);
        if (st == POD_OK) st = dalloc(&part, (size_t)ap.split * n * r);
        ncnt = (size_t)ap.grid.x + 64;
    }
    if (st == POD_OK) st = dalloc(&cnt, ncnt);
    if (st == POD_OK && cudaMemsetAsync(cnt, 0, ncnt * sizeof(unsigned), s) != cudaSuccess) st = POD_ECUDA;
    if (st == POD_OK) {
        k_set_state<<<1, 32, 0, s>>>(stt, r, 0, 0, 0, 1);
        if (tc) {
            XtyTcArgs xa{};
            xa.m = m;
            xa.ncols = n;
            xa.st = stt;
            xa.ny_from_state = 1;
            xa.part = part;
            xa.out = Y_dev;
            xa.ldo_y = n;
            xa.ldo_x = 1;
            xa.counters = cnt;
            xa.err = &stt->status;
            st = launch_xty_tc(xa, tp, (const float *)A_dev, lda, n, (const float *)U_dev, r, s);
        } else if (dtype == POD_F32) {
            AtuArgs<float> aa{};
            aa.m = m;
            aa.n = n;
            aa.A = (const float *)A_dev;
            aa.lda = lda;
            aa.U = (const float *)U_dev;
            aa.ldu = m;
            aa.st = stt;
            aa.ldy = (int)n;
            aa.rmax = r;
            aa.part = part;
            aa.Y = Y_dev;
            aa.counters = cnt;
            aa.vec = ((uintptr_t)A_dev % 16 == 0) && ((uintptr_t)U_dev % 16 == 0) && ((lda * 4) % 16 == 0) &&
                     ((m * 4) % 16 == 0);
            st = launch_atu<float>(aa, ap, s);
        } else {
            AtuArgs<double> aa{};
            aa.m = m;
            aa.n = n;
            aa.A = (const double *)A_dev;
            aa.lda = lda;
            aa.U = (const double *)U_dev;
            aa.ldu = m;
            aa.st = stt;
            aa.ldy = (int)n;
            aa.rmax = r;
            aa.part = part;
            aa.Y = Y_dev;
            aa.counters = cnt;
            aa.vec = ((uintptr_t)A_dev % 16 == 0) && ((uintptr_t)U_dev % 16 == 0) && ((lda * 8) % 16 == 0) &&
                     ((m * 8) % 16 == 0);
            st = launch_atu<double>(aa, ap, s);
        }
    }
    int status = 0;
    if (st == POD_OK && (cudaMemcpyAsync(&status, &stt->status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                         cudaStreamSynchronize(s) != cudaSuccess)) {
        cudaGetLastError();
        st = POD_ECUDA;
    }
    cudaStreamSynchronize(s);
    cudaFree(stt);
    cudaFree(part);
    cudaFree(cnt);
    if (st == POD_OK && status != 0) st = (pod_status)status;
    return st;
}

pod_status pod_sample(const uint64_t *w_dev, uint8_t *mask_dev, int64_t n, int32_t c, uint64_t seed, int32_t t,
                      int32_t stream_id, int32_t *idx_dev, int32_t *g_dev, void *stream) {
    if (!w_dev || !mask_dev || !idx_dev || !g_dev || n <= 0 || c <= 0 || t < 0 || stream_id < 0)
        return POD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t *w = nullptr, *cdf = nullptr;
    uint8_t *flags = nullptr;
    int32_t *draws = nullptr;
    POD_CUDA_TRY(cudaMallocAsync((void **)&w, n * sizeof(uint64_t), s));
    POD_CUDA_TRY(cudaMallocAsync((void **)&cdf, n * sizeof(uint64_t), s));
    POD_CUDA_TRY(cudaMallocAsync((void **)&flags, n, s));
    POD_CUDA_TRY(cudaMallocAsync((void **)&draws, c * sizeof(int32_t), s));
    POD_CUDA_TRY(cudaMemcpyAsync(w, w_dev, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    POD_CUDA_TRY(cudaMemsetAsync(flags, 0, n, s));
    SampleArgs a{};
    a.n = n;
    a.c = c;
    a.mode_round0 = 3;
    a.mode = 3;
    a.seed = seed;
    a.stream_id = stream_id;
    a.w = w;
    a.cdf = cdf;
    a.mask = mask_dev;
    a.flags = flags;
    a.draws = draws;
    a.idx = idx_dev;
    a.st = nullptr;
    a.g_out = g_dev;
    a.t_fixed = t;
    pod_status st = launch_sample(a, s);
    cudaFreeAsync(w, s);
    cudaFreeAsync(cdf, s);
    cudaFreeAsync(flags, s);
    cudaFreeAsync(draws, s);
    return st;
}

pod_status pod_incremental(const pod_params *p, const void *A_host, int32_t blocks, void *U_dev, double *sigma_dev,
                           void *stream) {
    POD_TRY(check_params(p));
    if (!A_host || !U_dev || !sigma_dev || blocks < 1 || blocks > p->n) return POD_EINVAL;
    if (p->keep_tape) return POD_EUNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t m = p->m, n = p->n;
    const size_t es = p->dtype == POD_F32 ? 4 : 8;
    const int r = p->r > 0 ? p->r : p->k;
    const int64_t ldb = (m + 3) & ~(int64_t)3;   // 16-byte column starts
    int64_t maxw = 0;
    for (int b = 0; b < blocks; ++b) {
        const int64_t w = (b + 1) * n / blocks - b * n / blocks;
        maxw = w > maxw ? w : maxw;
    }
    void *buf[2] = {nullptr, nullptr}, *Cb = nullptr, *Ua[2] = {nullptr, nullptr};
    double *sa[2] = {nullptr, nullptr}, *dots = nullptr, *part = nullptr;
    pod_ctx *cache[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    int64_t cache_w[2][2] = {{0, 0}, {0, 0}};
    cudaStream_t cs = nullptr;
    cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
    pod_status st = POD_OK;
    const int sms = device_sms();
    const int sgrid = 2 * sms;
    auto dalloc_bytes = [&](void **q, size_t bytes) {
        if (st == POD_OK && cudaMalloc(q, bytes) != cudaSuccess) {
            cudaGetLastError();
            st = POD_ENOMEM;
        }
    };
    dalloc_bytes(&buf[0], (size_t)ldb * maxw * es);
    dalloc_bytes(&buf[1], (size_t)ldb * maxw * es);
    dalloc_bytes(&Cb, (size_t)m * r * es);
    dalloc_bytes(&Ua[0], (size_t)m * r * es);
    dalloc_bytes(&Ua[1], (size_t)m * r * es);
    if (st == POD_OK) st = dalloc(&sa[0], r);
    if (st == POD_OK) st = dalloc(&sa[1], r);
    if (st == POD_OK) st = dalloc(&dots, r);
    if (st == POD_OK) st = dalloc(&part, (size_t)sgrid * r);
    if (st == POD_OK && (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess ||
                         cudaEventCreateWithFlags(&ev_copied[0], cudaEventDisableTiming) != cudaSuccess ||
                         cudaEventCreateWithFlags(&ev_copied[1], cudaEventDisableTiming) != cudaSuccess ||
                         cudaEventCreateWithFlags(&ev_free[0], cudaEventDisableTiming) != cudaSuccess ||
                         cudaEventCreateWithFlags(&ev_free[1], cudaEventDisableTiming) != cudaSuccess)) {
        cudaGetLastError();
        st = POD_ECUDA;
    }
    // copy of block b (host columns [b n / t, (b + 1) n / t)) into buf[b % 2]
    auto copy_block = [&](int b) {
        if (st != POD_OK) return;
        const int64_t j0 = b * n / blocks, w = (b + 1) * n / blocks - j0;
        const int q = b & 1;
        if (b >= 2 && cudaStreamWaitEvent(cs, ev_free[q], 0) != cudaSuccess) st = POD_ECUDA;
        if (st == POD_OK &&
            cudaMemcpy2DAsync(buf[q], ldb * es, (const char *)A_host + (size_t)j0 * p->lda * es, p->lda * es, m * es,
                              w, cudaMemcpyHostToDevice, cs) != cudaSuccess)
            st = POD_ECUDA;
        if (st == POD_OK && cudaEventRecord(ev_copied[q], cs) != cudaSuccess) st = POD_ECUDA;
        if (st != POD_OK) cudaGetLastError();
    };
    copy_block(0);
    int racc = 0, cur = 0;
    for (int b = 0; b < blocks && st == POD_OK; ++b) {
        const int q = b & 1;
        const int64_t w = (b + 1) * n / blocks - b * n / blocks;
        if (cudaStreamWaitEvent(s, ev_copied[q], 0) != cudaSuccess) {
            cudaGetLastError();
            st = POD_ECUDA;
            break;
        }
        if (b + 1 < blocks) copy_block(b + 1);   // streams while this block is processed
        // ISMA on the block: same parameters, r modes kept, no refinement
        const int wi = (cache_w[q][0] == w || cache_w[q][0] == 0) ? 0 : 1;
        pod_ctx *cb = cache[q][wi];
        if (!cb) {
            pod_params pb = *p;
            pb.n = w;
            pb.lda = ldb;
            pb.k = r;
            pb.refine = 0;
            st = pod_init(&cb, &pb, buf[q], stream);
            if (st != POD_OK) break;
            cache[q][wi] = cb;
            cache_w[q][wi] = w;
        } else {
            st = pod_reset(cb, buf[q]);
            if (st != POD_OK) break;
        }
        int32_t done = 0, steps = 0;
        while (st == POD_OK && !done) {
            st = pod_iterate(cb, 1 << 20, &done, nullptr, &steps);
            if (steps == 0) break;
        }
        if (st != POD_OK) break;
        if (cudaEventRecord(ev_free[q], s) != cudaSuccess) {
            cudaGetLastError();
            st = POD_ECUDA;
            break;
        }
        const int rb = cb->hstate->r_cur;
        if (rb == 0) continue;
        int grid = (int)((m * rb + 255) / 256);
        if (grid > 4 * sms) grid = 4 * sms;
        if (p->dtype == POD_F32)
            k_scale_cols<float><<<grid, 256, 0, s>>>((const float *)cb->U, m, rb, cb->sigma, (float *)Cb);
        else
            k_scale_cols<double><<<grid, 256, 0, s>>>((const double *)cb->U, m, rb, cb->sigma, (double *)Cb);
        if (cudaGetLastError() != cudaSuccess) {
            st = POD_ECUDA;
            break;
        }
        // BLOCK MERGE of the running factors with the block's (Algorithm 3)
        int32_t rn = 0;
        st = pod_block_merge(p->dtype, m, racc > 0 ? Ua[cur] : nullptr, racc > 0 ? sa[cur] : nullptr, racc, Cb, m,
                             rb, r, p->core, Ua[cur ^ 1], sa[cur ^ 1], &rn, stream);
        if (st != POD_OK) break;
        racc = rn;
        cur ^= 1;
    }
    if (st == POD_OK) {
        // the first k modes with the sign convention of pod_modes
        const int k = p->k;
        if (racc > 0) {
            if (p->dtype == POD_F32)
                st = launch_sign_dots<float>((const float *)Ua[cur], m, m, racc, p->seed, part, sgrid, s);
            else
                st = launch_sign_dots<double>((const double *)Ua[cur], m, m, racc, p->seed, part, sgrid, s);
            if (st == POD_OK) st = launch_reduce(part, sgrid, racc, racc, dots, nullptr, s);
        }
        int grid = (int)((m * k + 255) / 256);
        if (grid > 4 * sms) grid = 4 * sms;
        if (st == POD_OK) {
            if (p->dtype == POD_F32)
                k_write_modes<float><<<grid, 256, 0, s>>>((const float *)Ua[cur], m, racc, k, sa[cur], dots,
                                                          (float *)U_dev, sigma_dev);
            else
                k_write_modes<double><<<grid, 256, 0, s>>>((const double *)Ua[cur], m, racc, k, sa[cur], dots,
                                                           (double *)U_dev, sigma_dev);
            if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) st = POD_ECUDA;
        }
    }
    if (st != POD_OK) cudaGetLastError();
    if (s) cudaStreamSynchronize(s);
    if (cs) {
        cudaStreamSynchronize(cs);
        cudaStreamDestroy(cs);
    }
    for (int i = 0; i < 2; ++i) {
        if (ev_copied[i]) cudaEventDestroy(ev_copied[i]);
        if (ev_free[i]) cudaEventDestroy(ev_free[i]);
        for (int j = 0; j < 2; ++j)
            if (cache[i][j]) pod_destroy(cache[i][j]);
    }
    void *bufs[] = {buf[0], buf[1], Cb, Ua[0], Ua[1], sa[0], sa[1], dots, part};
    for (void *b : bufs)
        if (b) cudaFree(b);
    return st;
}

pod_status pod_block_merge(int32_t dtype, int64_t m, const void *U1_dev, const double *s1_dev, int32_t r1,
                           const void *C_dev, int64_t ldc, int32_t g, int32_t r, int32_t core, void *U_out_dev,
                           double *s_out_dev, int32_t *r_out_host, void *stream) {
    if ((dtype != POD_F32 && dtype != POD_F64) || m <= 0 || r1 < 0 || g < 1 || r < 1 || ldc < m) return POD_EINVAL;
    if (!C_dev || !U_out_dev || !s_out_dev || !r_out_host || (r1 > 0 && (!U1_dev || !s1_dev))) return POD_EINVAL;
    if (core < POD_CORE_AUTO || core > POD_CORE_F64) return POD_EINVAL;
    pod_params p{};
    p.m = m;
    p.n = g;
    p.lda = ldc;
    p.k = 1;
    p.c = g;
    p.r = r > r1 ? r : r1;
    p.dtype = dtype;
    p.core = core;
    p.tol = -1.0;
    p.col_strategy = POD_UNF;
    pod_ctx *c = nullptr;
    pod_status st = pod_init(&c, &p, C_dev, stream);
    if (st != POD_OK) return st;
    cudaStream_t s = c->stream;
    const size_t es = dtype == POD_F32 ? 4 : 8;
    // state: U1 carried (r1 modes), all g columns drawn this round (replay of 0..g-1)
    if (r1 > 0) {
        if (cudaMemcpy2DAsync(c->U, m * es, U1_dev, m * es, m * es, r1, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(c->sigma, s1_dev, r1 * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            cudaGetLastError();
            pod_destroy(c);
            return POD_ECUDA;
        }
    }
    c->rtrunc = r;   // truncation rank of this merge
    int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)g);
    int32_t off[2] = {0, g};
    if (!idx) {
        pod_destroy(c);
        return POD_ENOMEM;
    }
    for (int j = 0; j < g; ++j) idx[j] = j;
    st = pod_replay_indices(c, idx, off, 1);
    free(idx);
    if (st == POD_OK) {
        k_set_state<<<1, 32, 0, s>>>(c->st, r1, 0, 0, 0, 1);
        c->graph_failed = true;   // run eagerly
        st = enqueue_round_any(c);
    }
    if (st == POD_OK) st = read_state(c);
    if (st == POD_OK && c->hstate->status != 0) st = (pod_status)c->hstate->status;
    if (st == POD_OK) {
        const int rn = c->hstate->r_cur;
        *r_out_host = rn;
        if (cudaMemcpyAsync(U_out_dev, c->U, (size_t)m * rn * es, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(s_out_dev, c->sigma, rn * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            st = POD_ECUDA;
        }
    }
    pod_destroy(c);
    return st;
}

}  // extern "C"
