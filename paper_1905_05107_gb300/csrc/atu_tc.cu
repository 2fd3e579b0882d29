// Y = A^T U on the 5th-generation tensor cores (tcgen05), FP32 data: the
// dense contraction of the closing refinement (Algorithm 1's QR(A^T U)) and
// of the ORT probabilities (Eq. 6).  A is m x n column-major, U is m x r
// (ld m), Y is n x r column-major (ld n), K = m is the reduction.
//
// FP32 accuracy from TF32 tensor cores (split TF32, "3xTF32"): every operand
// x is split exactly into hi = x with the low 13 mantissa bits cleared (a TF32
// value) and lo = x - hi; A^T U ~ hi_A^T hi_U + hi_A^T lo_U + lo_A^T hi_U, the
// dropped lo_A^T lo_U term being ~2^-21 relative.
//
// CTA (M-tile of 128 columns of A) x (split of the K range):
//   warp 0      TMA producer: 32-row slabs of A (128 x 32 FP32) and of U
//               (N x 32) into a 4-stage ring, 128-byte swizzled (the layout
//               the MMA descriptors read); also allocates / frees TMEM
//   warp 1      one thread issues tcgen05.mma (M = 128, N, K = 8) for the
//               three split products, accumulating in TMEM; commits free a
//               stage and, every 2 slabs, hand an accumulator to the epilogue
//   warps 4-7   split each landed stage in place (hi) and into a lo copy
//   warps 8-11  drain each 64-row accumulator group from TMEM into double-
//               float registers (TwoSum; two TMEM buffers alternate), then write the CTA's
//               FP64 partial; the last CTA of an M-tile sums the splits in a
//               fixed order into Y.
// Every wait is bounded: on expiry the CTA records POD_ETIMEOUT, stops
// issuing work, waits for its own MMAs and copies, frees TMEM and returns.
#include <cuda.h>

#include "pod_internal.h"

namespace {

constexpr int TC_STAGES = 4;
constexpr int TC_KC = 32;                    // rows of A per slab (128 bytes)
// Slabs per TMEM accumulation group.  The tensor cores' FP32 accumulation
// does not round to nearest: over 512 rows (192 MMAs into one accumulator) a
// relative bias of ~1e-5 appeared in A^T U; two slabs (24 MMAs) keep it near
// 1e-6, and the epilogue continues the sum in double-float.
constexpr int TC_GROUP = 2;
constexpr int TC_THREADS = 384;
constexpr uint32_t TC_SPIN = 1u << 24;       // default bound of a wait: try_wait polls

__device__ __forceinline__ uint32_t sa(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(sa(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(sa(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(sa(b)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(sa(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait (at most `limit` polls) for the phase with the given parity;
// false on expiry or when another thread of the CTA has already given up.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, volatile int *abort_flag, uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it) {
        if (mbar_test(b, parity)) return true;
        if (*abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
}

__device__ __forceinline__ void tma_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];\n" ::
            "r"(sa(dst)),
        "l"(map), "r"(sa(bar)), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile stored with the
// 128-byte swizzle: rows of 128 bytes, 8-row core groups 1024 bytes apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
    d |= (uint64_t)1 << 16;                             // leading byte offset (unused here)
    d |= (uint64_t)(1024 >> 4) << 32;                   // stride byte offset
    d |= (uint64_t)1 << 46;                             // descriptor version
    d |= (uint64_t)2 << 61;                             // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void mma_tf32(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(sa(b))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// 32 TMEM columns of this warp's 32 lanes -> 32 registers per thread.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void bar_named(int id, int n) { asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(n) : "memory"); }

template <int NT>
struct TcLayout {
    static constexpr int A_BYTES = 128 * TC_KC * 4;   // 16 KB
    static constexpr int B_BYTES = NT * TC_KC * 4;
    static constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;   // hi and lo of both
    static constexpr int TMEM_COLS = 2 * NT <= 32 ? 32 : (2 * NT <= 64 ? 64 : 128);
    static constexpr size_t SMEM = 1024 + (size_t)TC_STAGES * STAGE + 256;
};

template <int NT>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_atu_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapU, AtuTcArgs a) {
    using L = TcLayout<NT>;
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + (size_t)TC_STAGES * L::STAGE);
    uint64_t *full = bars, *ready = bars + TC_STAGES, *freed = bars + 2 * TC_STAGES;
    uint64_t *accf = bars + 3 * TC_STAGES, *drained = accf + 2, *done = accf + 4;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    __shared__ int s_last;
    __shared__ int s_issued;   // slabs whose copies the producer started

    const DevState *st = a.st;
    if (st->done) return;
    const int r = st->r_cur;
    if (r <= 0) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // bound of the pipeline waits (the waits for this CTA's own copies and
    // MMAs after an abort always keep the default bound)
    const uint32_t lim = a.spin ? a.spin : TC_SPIN;
    const int mt = blockIdx.x, sp = blockIdx.y, splits = gridDim.y;
    const int64_t nslab_all = (a.m + TC_KC - 1) / TC_KC;
    const int64_t per = (nslab_all + splits - 1) / splits;
    const int64_t s0 = (int64_t)sp * per;
    const int64_t s1 = s0 + per < nslab_all ? s0 + per : nslab_all;
    const int nslab = s1 > s0 ? (int)(s1 - s0) : 0;
    const int ngroups = (nslab + TC_GROUP - 1) / TC_GROUP;

    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&ready[s], 128);
            mbar_init(&freed[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&drained[b], 128);
        }
        mbar_init(done, 1);
        s_abort = 0;
        s_issued = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(sa(&s_tmem)),
                     "r"((uint32_t)L::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    auto stageA = [&](int s) { return base + (size_t)s * L::STAGE; };
    auto stageAlo = [&](int s) { return base + (size_t)s * L::STAGE + L::A_BYTES; };
    auto stageB = [&](int s) { return base + (size_t)s * L::STAGE + 2 * L::A_BYTES; };
    auto stageBlo = [&](int s) { return base + (size_t)s * L::STAGE + 2 * L::A_BYTES + L::B_BYTES; };

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            for (int kc = 0; kc < nslab && !s_abort; ++kc) {
                const int s = kc % TC_STAGES;
                if (kc >= TC_STAGES && !mbar_wait(&freed[s], ((kc / TC_STAGES) - 1) & 1, &s_abort, lim)) break;
                mbar_expect_tx(&full[s], L::A_BYTES + L::B_BYTES);
                const int x = (int)((s0 + kc) * TC_KC);
                tma_2d(stageA(s), &mapA, &full[s], x, mt * 128);
                tma_2d(stageB(s), &mapU, &full[s], x, 0);
                s_issued = kc + 1;
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            // D format F32, A and B TF32, both K-major, N, M = 128
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NT >> 3) << 17) |
                                   ((uint32_t)(128 >> 4) << 24);
            for (int kc = 0; kc < nslab && !s_abort; ++kc) {
                const int s = kc % TC_STAGES;
                const int g = kc / TC_GROUP, b = g & 1;
                const bool first = (kc % TC_GROUP) == 0;
                if (first && g >= 2 && !mbar_wait(&drained[b], ((g >> 1) - 1) & 1, &s_abort, lim)) break;
                if (!mbar_wait(&ready[s], (kc / TC_STAGES) & 1, &s_abort, lim)) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * NT);
                const uint32_t ah = sa(stageA(s)), al = sa(stageAlo(s));
                const uint32_t bh = sa(stageB(s)), bl = sa(stageBlo(s));
#pragma unroll
                for (int kk = 0; kk < TC_KC / 8; ++kk) {   // K = 8 TF32 = 32 bytes per MMA
                    const uint32_t off = (uint32_t)kk * 32u;
                    mma_tf32(d, desc_sw128(ah + off), desc_sw128(bh + off), idesc, (first && kk == 0) ? 0u : 1u);
                    mma_tf32(d, desc_sw128(ah + off), desc_sw128(bl + off), idesc, 1u);
                    mma_tf32(d, desc_sw128(al + off), desc_sw128(bh + off), idesc, 1u);
                }
                mma_commit(&freed[s]);
                if ((kc % TC_GROUP) == TC_GROUP - 1 || kc == nslab - 1) mma_commit(&accf[b]);
            }
            // every MMA issued by this thread has completed once `done` flips
            // (waited for even after an abort: TMEM must not be freed earlier)
            mma_commit(done);
            int never = 0;
            mbar_wait(done, 0, &never, TC_SPIN);
        }
    } else if (warp >= 4 && warp < 8) {
        // ------------------------------------------------ split hi / lo
        const int t = tid - 128;
        for (int kc = 0; kc < nslab && !s_abort; ++kc) {
            const int s = kc % TC_STAGES;
            if (!mbar_wait(&full[s], (kc / TC_STAGES) & 1, &s_abort, lim)) break;
            float4 *ah = reinterpret_cast<float4 *>(stageA(s));
            float4 *al = reinterpret_cast<float4 *>(stageAlo(s));
            float4 *bh = reinterpret_cast<float4 *>(stageB(s));
            float4 *bl = reinterpret_cast<float4 *>(stageBlo(s));
            auto split = [](float4 *h, float4 *lo, int e) {
                float4 v = h[e], hv, lv;
                hv.x = __uint_as_float(__float_as_uint(v.x) & 0xFFFFE000u);
                hv.y = __uint_as_float(__float_as_uint(v.y) & 0xFFFFE000u);
                hv.z = __uint_as_float(__float_as_uint(v.z) & 0xFFFFE000u);
                hv.w = __uint_as_float(__float_as_uint(v.w) & 0xFFFFE000u);
                lv.x = v.x - hv.x;
                lv.y = v.y - hv.y;
                lv.z = v.z - hv.z;
                lv.w = v.w - hv.w;
                h[e] = hv;
                lo[e] = lv;
            };
            for (int e = t; e < L::A_BYTES / 16; e += 128) split(ah, al, e);
            for (int e = t; e < L::B_BYTES / 16; e += 128) split(bh, bl, e);
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            mbar_arrive(&ready[s]);
        }
    } else if (warp >= 8) {
        // ------------------------------------------------ epilogue
        const int q = warp - 8;                    // TMEM lane quadrant
        const int row = q * 32 + lane;             // row of the M-tile
        float ahi[NT], alo[NT];
#pragma unroll
        for (int c = 0; c < NT; ++c) ahi[c] = alo[c] = 0.f;
        for (int g = 0; g < ngroups && !s_abort; ++g) {
            const int b = g & 1;
            if (!mbar_wait(&accf[b], (g >> 1) & 1, &s_abort, lim)) break;
            tc_fence_after();
#pragma unroll
            for (int c0 = 0; c0 < NT; c0 += 32) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * NT + c0), v);
#pragma unroll
                for (int c = 0; c < 32; ++c)
                    if (c0 + c < NT) {
                        const dfloat t = df_two_sum(ahi[c0 + c], v[c]);
                        ahi[c0 + c] = t.hi;
                        alo[c0 + c] += t.lo;
                    }
            }
            tc_fence_before();
            mbar_arrive(&drained[b]);
        }
        // this CTA's partial (column-major within the tile: coalesced)
        double *part = a.part + ((size_t)mt * gridDim.y + sp) * (128 * NT);
#pragma unroll
        for (int c = 0; c < NT; ++c) part[(size_t)c * 128 + row] = (double)ahi[c] + (double)alo[c];
        __threadfence();
        bar_named(1, 128);
        if (tid == 256) s_last = atomicAdd(&a.counters[mt], 1u) == (unsigned)(gridDim.y - 1);
        bar_named(1, 128);
        if (s_last) {
            __threadfence();
            const double *pt = a.part + (size_t)mt * gridDim.y * (128 * NT);
            const int64_t j = (int64_t)mt * 128 + row;
            for (int c = 0; c < r && c < NT; ++c) {
                double sum = 0.0;
                for (int p = 0; p < (int)gridDim.y; ++p) sum += __ldcg(pt + (size_t)p * (128 * NT) + (size_t)c * 128 + row);
                if (j < a.n) a.Y[(int64_t)c * a.n + j] = sum;
            }
            if (tid == 256) a.counters[mt] = 0;
        }
    }

    tc_fence_before();
    __syncthreads();
    if (s_abort) {
        // stop: let the copies still in flight land (bounded) before the CTA
        // exits; the slabs after the last one the split warps took are the
        // only ones whose copies can be outstanding
        if (tid == 0) {
            *a.err = POD_ETIMEOUT;
            const int issued = s_issued;
            for (int kc = issued > TC_STAGES ? issued - TC_STAGES : 0; kc < issued; ++kc) {
                int never = 0;
                mbar_wait(&full[kc % TC_STAGES], (kc / TC_STAGES) & 1, &never, TC_SPIN);
            }
        }
        __syncthreads();
    }
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"((uint32_t)L::TMEM_COLS)
                     : "memory");
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 2-D FP32 tensor (rows inner) with a box of 32 rows x `box_cols` columns.
bool make_map(CUtensorMap *map, const float *ptr, int64_t rows, int64_t cols, int64_t ld, int box_cols) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {(cuuint32_t)TC_KC, (cuuint32_t)box_cols};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)ptr, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int atu_tc_supported(int dtype, int64_t m, int64_t lda, int rmax, const void *A, const void *U) {
    return dtype == POD_F32 && rmax >= 1 && rmax <= 64 && (m % 4) == 0 && (lda % 4) == 0 &&
           ((uintptr_t)A % 16) == 0 && ((uintptr_t)U % 16) == 0 && m <= 0x7fffffffLL;
}

AtuTcPlan atu_tc_plan(int64_t m, int64_t n, int rmax, int sms) {
    AtuTcPlan p{};
    p.nt = rmax <= 32 ? 32 : 64;
    p.mtiles = (int)((n + 127) / 128);
    const int64_t nslab = (m + TC_KC - 1) / TC_KC;
    int splits = sms / (p.mtiles > 0 ? p.mtiles : 1);
    if (splits < 1) splits = 1;
    if (splits > nslab) splits = (int)nslab;
    p.splits = splits;
    p.smem = p.nt == 32 ? TcLayout<32>::SMEM : TcLayout<64>::SMEM;
    p.part_doubles = (size_t)p.mtiles * splits * 128 * p.nt;
    return p;
}

pod_status launch_atu_tc(const AtuTcArgs &a, const AtuTcPlan &plan, const float *A, const float *U, cudaStream_t s) {
    CUtensorMap mA, mU;
    if (!make_map(&mA, A, a.m, a.n, a.lda, 128) || !make_map(&mU, U, a.m, a.rmax, a.m, plan.nt))
        return POD_EUNSUPPORTED;
    dim3 grid((unsigned)plan.mtiles, (unsigned)plan.splits, 1);
    if (plan.nt == 32) {
        POD_CUDA_TRY(cudaFuncSetAttribute(k_atu_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem));
        k_atu_tc<32><<<grid, TC_THREADS, plan.smem, s>>>(mA, mU, a);
    } else {
        POD_CUDA_TRY(cudaFuncSetAttribute(k_atu_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem));
        k_atu_tc<64><<<grid, TC_THREADS, plan.smem, s>>>(mA, mU, a);
    }
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}
