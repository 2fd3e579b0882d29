// D = X^T Y on the 5th-generation tensor cores (tcgen05) for FP32 data, the
// reduction over the m rows of two tall column-major matrices:
//   * U^T C of BLOCK MERGE (Algorithm 2, U_1^T U_2; Eq. 8), X = the sampled
//     columns C = A[:, I_c] read in place (gathered) or the ICRS block D V_r,
//     Y = U;
//   * A^T U of the closing refinement (Algorithm 1, QR(A^T U)) and of the ORT
//     probabilities (Eq. 6), X = A, Y = U.
// Products of FP32 data on tensor cores, three precisions:
//   POD_PREC_TF32X3  x = hi + lo exactly, hi = x with the low 13 mantissa
//                    bits cleared (TF32), lo = x - hi; hi_X hi_Y + hi_X lo_Y +
//                    lo_X hi_Y (kind::tf32, K = 8): FP32-level products
//   POD_PREC_BF16X3  x ~ b0 + b1, b0 = bf16(x), b1 = bf16(x - b0) (rounded to
//                    nearest); b0 b0 + b0 b1 + b1 b0 (kind::f16, K = 16):
//                    about 2^-16 relative per product
//   POD_PREC_BF16    b0 b0 alone: about 2^-8 relative per product
// FP32 accumulation in TMEM over groups of 64 rows (the tensor cores' FP32
// accumulation does not round to nearest: over 512 rows a relative bias of
// ~1e-5 appeared in A^T U, 64 rows keep it near 1e-6), double-float across
// groups in the epilogue, FP64 partials summed in a fixed order.
//
// Work: the X columns form M-tiles of 128 (the MMA's M), the rows slabs of
// 32 (TF32) or 64 (BF16) rows; the (M-tile, slab) items, M-tile major, are
// cut into gridDim.x equal contiguous ranges, one per CTA, so every SM gets
// the same number of slabs whatever the tile count.  A range that crosses an
// M-tile boundary yields one partial per M-tile it touches.
//
// CTA roles (512 threads):
//   warp 0      producer: TMA copies of each slab into a ring, 128-byte
//               swizzled (the layout the MMA descriptors read): X as one box
//               of 128 columns (dense) or four sampled columns per
//               tile::gather4 copy (gathered; one copy per lane), Y as one box; also
//               allocates / frees TMEM
//   warp 1      one thread issues the MMAs (M = 128, N = NT) into one of two
//               TMEM accumulators, commits free a stage and, at the end of a
//               64-row group, hand the accumulator to the epilogue
//   warps 4-7   split (TF32: hi and lo tiles) or convert (BF16:
//               from the raw FP32 ring into a bf16 ring) each landed slab
//   warps 8-15  drain each group's accumulator into double-float registers
//               (two warps per TMEM lane quadrant, half of the columns each,
//               so that the running sums stay in registers), write the CTA's
//               FP64 partials; the last CTA of an M-tile sums the partials of
//               that tile in a fixed order (or, deferred, the partials are
//               left to a separate summing kernel)
// Every pipeline wait is bounded: on expiry the CTA records POD_ETIMEOUT,
// stops issuing work, waits (with the default bound) for its own copies and
// MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include "pod_internal.h"

namespace {

constexpr int XT_THREADS = 512;
constexpr int XT_TM = 128;                   // X columns per M-tile
constexpr uint32_t XT_SPIN = 1u << 24;       // default bound of a wait: try_wait polls
constexpr int XT_SMEM_BUDGET = 200 * 1024;   // ring bytes per CTA

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

// Four columns c0..c3 of a 2-D tensor map with a box of 32 rows x 1 column
// (tile::gather4): 4 x 128 bytes into four consecutive 128-byte rows at dst,
// swizzled as the map says; rows x .. x + 31 (x a multiple of 32).
__device__ __forceinline__ void tma_gather4(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int c0, int c1,
                                            int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6, %7}], [%2];\n" ::"r"(sa(dst)),
        "l"(map), "r"(sa(bar)), "r"(x), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
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

template <int MODE>
__device__ __forceinline__ void mma_issue(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    if constexpr (MODE == POD_PREC_TF32X3) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::
                "r"(dt),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::
                "r"(dt),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
    }
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

// 16 TMEM columns of this warp's 32 lanes -> 16 registers per thread.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void bar_named(int id, int n) { asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(n) : "memory"); }

// Ring layout of one (MODE, NT): a raw FP32 ring the copies land in and a
// ring of operand tiles the converter fills (TF32 hi and lo; bf16 b0, and b1
// for X3).  A raw stage is free again once converted, before its MMAs run.
template <int MODE, int NT>
struct XtLayout {
    static constexpr int KROWS = MODE == POD_PREC_TF32X3 ? 32 : 64;   // rows per slab (128 bytes of K)
    static constexpr int BOXES = KROWS / 32;                  // 32-row FP32 boxes per slab
    static constexpr int PRODUCTS = MODE == POD_PREC_BF16 ? 1 : 3;
    static constexpr int GROUP = 64 / KROWS;                  // slabs per TMEM accumulation group
    static constexpr int XB32 = XT_TM * 128;                  // one 32-row FP32 box of X
    static constexpr int YB32 = NT * 128;
    static constexpr int RAW = BOXES * (XB32 + YB32);         // FP32 bytes of a slab
    // converted stage: X hi / b0 at 0, X lo / b1, Y hi / b0, Y lo / b1
    static constexpr int CX = XT_TM * 128, CY = NT * 128;     // one converted operand tile
    static constexpr int NCONV = PRODUCTS == 1 ? 1 : 2;       // tiles per operand
    static constexpr int CONV = NCONV * (CX + CY);
    static constexpr int CS = 2 * RAW + 2 * CONV <= XT_SMEM_BUDGET ? 2 : 1;
    static constexpr int RS = 4 * RAW + CS * CONV <= XT_SMEM_BUDGET ? 4 : (3 * RAW + CS * CONV <= XT_SMEM_BUDGET ? 3 : 2);
    static constexpr int RAW_BYTES = RS * RAW;
    static constexpr int CONV_BYTES = CS * CONV;
    static constexpr int TMEM_COLS = 2 * NT <= 32 ? 32 : (2 * NT <= 64 ? 64 : (2 * NT <= 128 ? 128 : 256));
    static constexpr size_t SMEM = 1024 + (size_t)RAW_BYTES + CONV_BYTES + 256;
    // offsets inside a stage / conversion tile
    static constexpr int X_HI = 0;
    static constexpr int X_LO = CX;
    static constexpr int Y_HI = NCONV * CX;
    static constexpr int Y_LO = NCONV * CX + CY;
};

// Owner CTA of work item i when W items are cut into G equal contiguous ranges
// [floor(b W / G), floor((b + 1) W / G)).
__host__ __device__ inline int64_t item_owner(int64_t i, int64_t W, int64_t G) { return ((i + 1) * G - 1) / W; }

template <int MODE, int NT>
__global__ void __launch_bounds__(XT_THREADS, 1)
    k_xty_tc(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapY, XtyTcArgs a) {
    using L = XtLayout<MODE, NT>;
    extern __shared__ __align__(1024) unsigned char xt_smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(((uintptr_t)xt_smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *rawb = base;
    unsigned char *convb = base + L::RAW_BYTES;
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + L::RAW_BYTES + L::CONV_BYTES);
    uint64_t *full = bars, *rfree = bars + L::RS, *ready = bars + 2 * L::RS, *cfree = ready + L::CS;
    uint64_t *accf = cfree + L::CS, *drained = accf + 2, *done = accf + 4;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    __shared__ int s_last;
    __shared__ int s_issued;   // slabs whose copies the producer started

    const DevState *st = a.st;
    if (st && st->done) return;
    const int ny = a.ny_from_state ? st->r_cur : a.ny;
    const int64_t ncols = a.gather ? (int64_t)st->g : a.ncols;
    if (ny <= 0 || ncols <= 0) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t lim = a.spin ? a.spin : XT_SPIN;
    // work items (M-tile, slab), M-tile major; this CTA's range
    const int64_t nslab = (a.m + L::KROWS - 1) / L::KROWS;
    const int64_t W = (int64_t)a.mtiles * nslab, G = gridDim.x;
    const int64_t lo = (int64_t)blockIdx.x * W / G, hi = ((int64_t)blockIdx.x + 1) * W / G;
    const int nit = (int)(hi - lo);
    if (nit <= 0) return;
    // slab kc of this CTA: item lo + kc; a new accumulation group starts at
    // the first slab of the range, of each M-tile, and every GROUP slabs
    auto mt_of = [&](int kc) { return (int)((lo + kc) / nslab); };
    auto group_start = [&](int kc) {
        if (kc == 0) return true;
        const int64_t it = lo + kc;
        const int64_t seg0 = (it / nslab) * nslab > lo ? (it / nslab) * nslab : lo;
        return ((it - seg0) % L::GROUP) == 0;
    };

    if (tid == 0) {
        for (int s = 0; s < L::RS; ++s) {
            // the producer's expect_tx arrival (the copies complete by bytes)
            mbar_init(&full[s], 1);
            mbar_init(&rfree[s], 128);   // the converter's threads
        }
        for (int s = 0; s < L::CS; ++s) {
            mbar_init(&ready[s], 128);
            mbar_init(&cfree[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&drained[b], 256);
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

    auto raw_stage = [&](int s) {
        return rawb + (size_t)s * L::RAW;
    };
    // operand tiles the MMA reads for slab stage cs
    auto op_stage = [&](int cs) { return convb + (size_t)cs * L::CONV; };

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        int gcol[4];   // gathered: the columns of this lane's group of four (M-tile rows 4 lane ..)
        int cur_mt = -1, ncol_mt = 0, ngrp = 0;
        for (int kc = 0; kc < nit; ++kc) {
            const int s = kc % L::RS;
            // lane 0 decides, the warp follows (every lane reaches the shuffle)
            int go = 1;
            if (lane == 0) {
                go = s_abort ? 0 : 1;
                if (go && kc >= L::RS) go = mbar_wait(&rfree[s], ((kc / L::RS) - 1) & 1, &s_abort, lim) ? 1 : 0;
            }
            go = __shfl_sync(0xffffffffu, go, 0);
            if (!go) break;
            const int mt = mt_of(kc);
            const int x = (int)(((lo + kc) % nslab) * L::KROWS);
            if (a.gather && mt != cur_mt) {
                cur_mt = mt;
                const int64_t c0 = (int64_t)mt * XT_TM;
                ncol_mt = ncols - c0 < XT_TM ? (int)(ncols - c0) : XT_TM;
                ngrp = (ncol_mt + 3) / 4;
                // rows past the last column repeat the group's first column
                // (their products are never read)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int j = 4 * lane + q;
                    gcol[q] = lane < ngrp ? a.idx[c0 + (j < ncol_mt ? j : 4 * lane)] : 0;
                }
            }
            unsigned char *stg = raw_stage(s);
            const uint32_t xbytes = a.gather ? (uint32_t)ngrp * 512u * L::BOXES : (uint32_t)L::XB32 * L::BOXES;
            if (lane == 0) mbar_expect_tx(&full[s], xbytes + (uint32_t)L::YB32 * L::BOXES);
            __syncwarp();
#pragma unroll
            for (int bx = 0; bx < L::BOXES; ++bx) {
                unsigned char *xdst = stg + bx * L::XB32;
                unsigned char *ydst = stg + L::BOXES * L::XB32 + bx * L::YB32;
                if (a.gather) {
                    // sampled columns 4 lane .. 4 lane + 3: their 32 rows
                    // (128 bytes each) into tile rows 4 lane .. by one TMA
                    // gather (128-byte swizzle; rows beyond m read as 0)
                    if (lane < ngrp)
                        tma_gather4(xdst + lane * 512, &mapX, &full[s], x + 32 * bx, gcol[0], gcol[1], gcol[2], gcol[3]);
                } else if (lane == 0) {
                    tma_2d(xdst, &mapX, &full[s], x + 32 * bx, mt * XT_TM);
                }
                if (lane == 0) tma_2d(ydst, &mapY, &full[s], x + 32 * bx, 0);
            }
            if (lane == 0) s_issued = kc + 1;
            __syncwarp();
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t fmt = MODE == POD_PREC_TF32X3 ? 2u : 1u;   // TF32 / BF16 operands
            const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(NT >> 3) << 17) |
                                   ((uint32_t)(XT_TM >> 4) << 24);
            int gi = -1;
            for (int kc = 0; kc < nit && !s_abort; ++kc) {
                const int cs = kc % L::CS;
                const bool first = group_start(kc);
                if (first) ++gi;
                const int b = gi & 1;
                if (first && gi >= 2 && !mbar_wait(&drained[b], ((gi >> 1) - 1) & 1, &s_abort, lim)) break;
                if (!mbar_wait(&ready[cs], (kc / L::CS) & 1, &s_abort, lim)) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * NT);
                unsigned char *op = op_stage(cs);
                const uint32_t xh = sa(op + L::X_HI), xl = sa(op + L::X_LO);
                const uint32_t yh = sa(op + L::Y_HI), yl = sa(op + L::Y_LO);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {   // 32 bytes of K per MMA
                    const uint32_t off = (uint32_t)kk * 32u;
                    mma_issue<MODE>(d, desc_sw128(xh + off), desc_sw128(yh + off), idesc, (first && kk == 0) ? 0u : 1u);
                    if constexpr (L::PRODUCTS == 3) {
                        mma_issue<MODE>(d, desc_sw128(xh + off), desc_sw128(yl + off), idesc, 1u);
                        mma_issue<MODE>(d, desc_sw128(xl + off), desc_sw128(yh + off), idesc, 1u);
                    }
                }
                mma_commit(&cfree[cs]);
                if (kc == nit - 1 || group_start(kc + 1)) mma_commit(&accf[b]);
            }
            // every MMA issued by this thread has completed once `done` flips
            // (waited for even after an abort: TMEM must not be freed earlier)
            mma_commit(done);
            int never = 0;
            mbar_wait(done, 0, &never, XT_SPIN);
        }
    } else if (warp >= 4 && warp < 8) {
        // ------------------------------------------------ split / convert
        const int t = tid - 128;
        for (int kc = 0; kc < nit; ++kc) {
            if (s_abort) break;
            const int s = kc % L::RS;
            if (!mbar_wait(&full[s], (kc / L::RS) & 1, &s_abort, lim)) break;
            const int cs = kc % L::CS;
            if (kc >= L::CS && !mbar_wait(&cfree[cs], ((kc / L::CS) - 1) & 1, &s_abort, lim)) break;
            const unsigned char *stg = raw_stage(s);
            unsigned char *cv = convb + (size_t)cs * L::CONV;
            // row j of a tile (one X or Y column, 64 K values): FP32 chunk
            // c of box bx at j*128 + ((c ^ (j & 7)) << 4); bf16 chunk q
            // (rows 8q .. 8q+7) at j*128 + ((q ^ (j & 7)) << 4)
            auto convert_row = [&](const unsigned char *raw0, int boxbytes, unsigned char *d0, unsigned char *d1, int j) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const unsigned char *rb = raw0 + (q >> 2) * boxbytes + j * 128;
                    const int c = 2 * (q & 3);
                    const float4 u0 = *reinterpret_cast<const float4 *>(rb + (((c) ^ (j & 7)) << 4));
                    const float4 u1 = *reinterpret_cast<const float4 *>(rb + (((c + 1) ^ (j & 7)) << 4));
                    const float v[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
                    __nv_bfloat162 h[4], l[4];
#pragma unroll
                    for (int p = 0; p < 4; ++p) {
                        const __nv_bfloat16 a0 = __float2bfloat16_rn(v[2 * p]);
                        const __nv_bfloat16 a1 = __float2bfloat16_rn(v[2 * p + 1]);
                        h[p] = __halves2bfloat162(a0, a1);
                        if (d1) {
                            const float r0 = v[2 * p] - __bfloat162float(a0);
                            const float r1 = v[2 * p + 1] - __bfloat162float(a1);
                            l[p] = __halves2bfloat162(__float2bfloat16_rn(r0), __float2bfloat16_rn(r1));
                        }
                    }
                    const int dst = j * 128 + ((q ^ (j & 7)) << 4);
                    *reinterpret_cast<uint4 *>(d0 + dst) = *reinterpret_cast<const uint4 *>(h);
                    if (d1) *reinterpret_cast<uint4 *>(d1 + dst) = *reinterpret_cast<const uint4 *>(l);
                }
            };
            // TF32: row j's eight 16-byte chunks split into hi (low 13
            // mantissa bits cleared) and lo = x - hi, at the same swizzled
            // positions
            auto split_row = [&](const unsigned char *raw0, unsigned char *d0, unsigned char *d1, int j) {
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int off = j * 128 + ((c ^ (j & 7)) << 4);
                    const float4 v = *reinterpret_cast<const float4 *>(raw0 + off);
                    float4 hv, lv;
                    hv.x = __uint_as_float(__float_as_uint(v.x) & 0xFFFFE000u);
                    hv.y = __uint_as_float(__float_as_uint(v.y) & 0xFFFFE000u);
                    hv.z = __uint_as_float(__float_as_uint(v.z) & 0xFFFFE000u);
                    hv.w = __uint_as_float(__float_as_uint(v.w) & 0xFFFFE000u);
                    lv.x = v.x - hv.x;
                    lv.y = v.y - hv.y;
                    lv.z = v.z - hv.z;
                    lv.w = v.w - hv.w;
                    *reinterpret_cast<float4 *>(d0 + off) = hv;
                    *reinterpret_cast<float4 *>(d1 + off) = lv;
                }
            };
            constexpr bool two = L::PRODUCTS == 3;
            if constexpr (MODE == POD_PREC_TF32X3) {
                split_row(stg, cv + L::X_HI, cv + L::X_LO, t);
                if (t < NT) split_row(stg + L::XB32, cv + L::Y_HI, cv + L::Y_LO, t);
            } else {
                convert_row(stg, L::XB32, cv + L::X_HI, two ? cv + L::X_LO : nullptr, t);
                if (t < NT)
                    convert_row(stg + L::BOXES * L::XB32, L::YB32, cv + L::Y_HI, two ? cv + L::Y_LO : nullptr,
                                t);
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            mbar_arrive(&rfree[s]);
            mbar_arrive(&ready[cs]);
        }
    } else if (warp >= 8) {
        // ------------------------------------------------ epilogue
        constexpr int NH = NT / 2;                 // columns per epilogue warp
        const int q = warp & 3;                    // TMEM lane quadrant (warp % 4)
        const int c0 = ((warp - 8) >> 2) * NH;     // this warp's first column
        const int row = q * 32 + lane;             // row of the M-tile
        float ahi[NH], alo[NH];
#pragma unroll
        for (int c = 0; c < NH; ++c) ahi[c] = alo[c] = 0.f;
        int gi = -1;
        for (int kc = 0; kc < nit; ++kc) {
            if (!group_start(kc)) continue;
            ++gi;
            const int b = gi & 1;
            // a warp-uniform decision: tcgen05.ld is a whole-warp operation
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&accf[b], (gi >> 1) & 1, &s_abort, lim));
            if (!ok) break;
            tc_fence_after();
            const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * NT + c0);
            float v[NH];
            if constexpr (NH == 32) tmem_ld32(ta, v);
            else tmem_ld16(ta, v);
#pragma unroll
            for (int c = 0; c < NH; ++c) {
                const dfloat t2 = df_two_sum(ahi[c], v[c]);
                ahi[c] = t2.hi;
                alo[c] += t2.lo;
            }
            tc_fence_before();
            mbar_arrive(&drained[b]);
            // end of this CTA's part of an M-tile: store its partial (plain
            // stores; the arrival bookkeeping follows the loop)
            int kend = kc + 1;
            while (kend < nit && !group_start(kend)) ++kend;
            const int mt = mt_of(kc);
            if (kend < nit && mt_of(kend) == mt) continue;
            const int64_t xc = (int64_t)mt * XT_TM + row;
            if (a.deferred) {
                double *slot = a.part + (int64_t)blockIdx.x * a.part_stride;
#pragma unroll
                for (int c = 0; c < NH; ++c)
                    if (c0 + c < ny && xc < ncols) slot[(int64_t)(c0 + c) * a.ldo_y + xc] = (double)ahi[c] + (double)alo[c];
            } else {
                const int64_t bf = item_owner((int64_t)mt * nslab, W, G);
                double *part = a.part + ((int64_t)mt * a.maxcover + (blockIdx.x - bf)) * (XT_TM * NT);
#pragma unroll
                for (int c = 0; c < NH; ++c) part[(size_t)(c0 + c) * XT_TM + row] = (double)ahi[c] + (double)alo[c];
            }
#pragma unroll
            for (int c = 0; c < NH; ++c) ahi[c] = alo[c] = 0.f;
        }
        // every epilogue warp runs what follows the same way, aborted or not
        const int mt0 = mt_of(0), mt1 = mt_of(nit - 1);
        if (a.deferred) {
            // this CTA covers one M-tile (the plan makes the grid a multiple
            // of the tiles); the other tiles' entries of its slot hold zeros
            double *slot = a.part + (int64_t)blockIdx.x * a.part_stride;
            for (int omt = 0; omt < a.mtiles; ++omt) {
                if (omt >= mt0 && omt <= mt1) continue;
                const int64_t oc = (int64_t)omt * XT_TM + row;
                for (int c = c0; c < c0 + NH && c < ny; ++c)
                    if (oc < ncols) slot[(int64_t)c * a.ldo_y + oc] = 0.0;
            }
        } else {
            for (int mt = mt0; mt <= mt1; ++mt) {
                const int64_t bf = item_owner((int64_t)mt * nslab, W, G);
                const int64_t bl = item_owner((int64_t)mt * nslab + nslab - 1, W, G);
                __threadfence();
                bar_named(1, 256);
                if (tid == 256) s_last = atomicAdd(&a.counters[mt], 1u) == (unsigned)(bl - bf);
                bar_named(1, 256);
                if (s_last) {
                    __threadfence();
                    const int64_t xc = (int64_t)mt * XT_TM + row;
                    const double *pt = a.part + (int64_t)mt * a.maxcover * (XT_TM * NT);
                    for (int c = c0; c < c0 + NH && c < ny; ++c) {
                        double sum = 0.0;
                        for (int p = 0; p <= (int)(bl - bf); ++p)
                            sum += __ldcg(pt + (size_t)p * (XT_TM * NT) + (size_t)c * XT_TM + row);
                        if (xc < ncols) a.out[(int64_t)c * a.ldo_y + xc * a.ldo_x] = sum;
                    }
                    if (tid == 256) a.counters[mt] = 0;
                }
                bar_named(1, 256);   // s_last is reused for the next tile
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (s_abort) {
        // stop: let the copies still in flight land (bounded) before the CTA
        // exits; the slabs after the last one the converter took are the only
        // ones whose copies can be outstanding
        if (tid == 0) {
            if (a.err) *a.err = POD_ETIMEOUT;
            const int issued = s_issued;
            for (int kc = issued > L::RS ? issued - L::RS : 0; kc < issued; ++kc) {
                int never = 0;
                mbar_wait(&full[kc % L::RS], (kc / L::RS) & 1, &never, XT_SPIN);
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

// 2-D FP32 tensor (rows inner, ld between columns) with a box of 32 rows x
// `box_cols` columns, 128-byte swizzle; rows or columns beyond the tensor
// read as zeros.
bool make_map(CUtensorMap *map, const float *ptr, int64_t rows, int64_t cols, int64_t ld, int box_cols) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {32u, (cuuint32_t)box_cols};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)ptr, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int MODE, int NT>
size_t smem_of() { return XtLayout<MODE, NT>::SMEM; }

template <int MODE, int NT>
pod_status launch_one(const CUtensorMap &mX, const CUtensorMap &mY, const XtyTcArgs &a, const XtyTcPlan &p,
                      cudaStream_t s) {
    const size_t smem = XtLayout<MODE, NT>::SMEM;
    POD_CUDA_TRY(cudaFuncSetAttribute(k_xty_tc<MODE, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_xty_tc<MODE, NT><<<p.grid, XT_THREADS, smem, s>>>(mX, mY, a);
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}

int krows_of(int mode) { return mode == POD_PREC_TF32X3 ? 32 : 64; }

}  // namespace

int xty_tc_mode_ok(int mode) {
    return mode == POD_PREC_TF32X3 || mode == POD_PREC_BF16X3 || mode == POD_PREC_BF16;
}

int xty_tc_supported(int dtype, int64_t m, int64_t ldx, int ny_max, const void *X, const void *Y) {
    return dtype == POD_F32 && ny_max >= 1 && ny_max <= 64 && (m % 4) == 0 && (ldx % 4) == 0 &&
           ((uintptr_t)X % 16) == 0 && ((uintptr_t)Y % 16) == 0 && m <= 0x7fffffffLL;
}

XtyTcPlan xty_tc_plan(int mode, int64_t m, int64_t ncols_max, int ny_max, int sms, int deferred) {
    XtyTcPlan p{};
    p.mode = mode;
    p.nt = ny_max <= 32 ? 32 : 64;
    p.mtiles = (int)((ncols_max + XT_TM - 1) / XT_TM);
    const int64_t nslab = (m + krows_of(mode) - 1) / krows_of(mode);
    const int64_t W = (int64_t)p.mtiles * nslab;
    int64_t G = sms;
    // deferred sums: one M-tile per CTA (the grid a multiple of the tiles)
    if (deferred) G = (int64_t)p.mtiles * (sms / p.mtiles > 0 ? sms / p.mtiles : 1);
    if (G > W) G = W;
    if (G < 1) G = 1;
    p.grid = (int)G;
    // partial slots per M-tile in local-sum mode
    int maxcover = 1;
    for (int mt = 0; mt < p.mtiles; ++mt) {
        const int64_t bf = item_owner((int64_t)mt * nslab, W, G), bl = item_owner((int64_t)mt * nslab + nslab - 1, W, G);
        if (bl - bf + 1 > maxcover) maxcover = (int)(bl - bf + 1);
    }
    p.maxcover = maxcover;
    p.part_doubles = (size_t)p.mtiles * maxcover * XT_TM * p.nt;
    const bool b3 = mode == POD_PREC_BF16X3, b1 = mode == POD_PREC_BF16;
    if (p.nt == 32)
        p.smem = b3 ? smem_of<POD_PREC_BF16X3, 32>() : (b1 ? smem_of<POD_PREC_BF16, 32>() : smem_of<POD_PREC_TF32X3, 32>());
    else
        p.smem = b3 ? smem_of<POD_PREC_BF16X3, 64>() : (b1 ? smem_of<POD_PREC_BF16, 64>() : smem_of<POD_PREC_TF32X3, 64>());
    return p;
}

pod_status launch_xty_tc(const XtyTcArgs &a0, const XtyTcPlan &plan, const float *X, int64_t ldx, int64_t xcols,
                         const float *Y, int64_t ycols, cudaStream_t s) {
    XtyTcArgs a = a0;
    a.mtiles = plan.mtiles;
    a.maxcover = plan.maxcover;
    CUtensorMap mX, mY;
    a.X = X;
    a.ldx = ldx;
    // dense X: boxes of 128 columns; gathered X: one-column boxes (tile::gather4)
    if (!make_map(&mY, Y, a.m, ycols, a.m, plan.nt)) return POD_EUNSUPPORTED;
    if (!make_map(&mX, X, a.m, xcols, ldx, a.gather ? 1 : XT_TM)) return POD_EUNSUPPORTED;
    const int mode = plan.mode;
    if (plan.nt == 32) {
        if (mode == POD_PREC_TF32X3) return launch_one<POD_PREC_TF32X3, 32>(mX, mY, a, plan, s);
        if (mode == POD_PREC_BF16X3) return launch_one<POD_PREC_BF16X3, 32>(mX, mY, a, plan, s);
        return launch_one<POD_PREC_BF16, 32>(mX, mY, a, plan, s);
    }
    if (mode == POD_PREC_TF32X3) return launch_one<POD_PREC_TF32X3, 64>(mX, mY, a, plan, s);
    if (mode == POD_PREC_BF16X3) return launch_one<POD_PREC_BF16X3, 64>(mX, mY, a, plan, s);
    return launch_one<POD_PREC_BF16, 64>(mX, mY, a, plan, s);
}
