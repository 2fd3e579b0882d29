// Tall-skinny passes of BLOCK MERGE (Algorithm 2) over the m rows:
//   TALL_PROJ   : P  = U^T C                              (U_1^T U_2, Eq. 8)
//   TALL_CGS    : Z  = C - U P;  P2 = U^T Z;  G = Z^T Z    (U_t, second projection;
//                 Z is stored)
//   TALL_QR2    : W  = (Z - U P2) M1;  G2 = W^T W          (second CholeskyQR pass;
//                 W is stored over Z)
//   TALL_UPDATE : U <- U X + W Y                          (U = [U_1 U_o] U_E, truncated;
//                 U_o = W R2^{-1}; the ICRS row stage combines C instead of W)
// plus Y = A^T U (closing refinement of Algorithm 1, ORT probabilities) and
// the sign-reference dots.
//
// Each CTA walks row slabs of `bm` rows.  Slabs of U and of the gathered
// columns A[:, idx[j]] are copied column-major into shared memory with
// cp.async (16-byte copies when every column start is 16-byte aligned),
// double-buffered so the next slab streams in while the current one is
// used.  Every product is a 4x4 register tile fed by 128-bit shared loads:
// the row-space products (C - U P, Z - U P2, Z M1, U X + W Y) tile 4 rows x 4
// output columns (the triangular Z M1 with each tile's k-range split in two
// and balanced across the threads), the Gram-type products (U^T C, Z^T Z)
// tile 4 x 4 outputs over 4-row chunks.  Each kind of pass has its own
// shared-memory layout, slab height and thread count (tall_plan).  FP32 tile
// sums are added into running sums after every
// slab (double-float slots for FP32 data, FP64 for FP64 data).  Each CTA
// writes its FP64 partial; in a round's PROJ, CGS and QR2 passes those are
// summed by k_sum_parts (many CTAs, fixed order), elsewhere inside the kernel:
// the last CTA to finish in each group of 16 sums its group, the last group
// sums the groups, in a fixed order, using atomic arrival counters only (no
// waiting).  Either way the sums are bit-reproducible.  The UPDATE pass of a
// round also ends the round in its last CTA.
#include "pod_internal.h"

namespace {

constexpr int TALL_THREADS = 256;       // k_atu; k_tall when two CTAs share an SM
constexpr int TALL_MAX_THREADS = 512;   // k_tall with one CTA per SM (tall_plan picks)

__host__ __device__ inline int round4(int x) { return (x + 3) & ~3; }

template <typename T>
__device__ __forceinline__ void lds4(const T *p, T (&v)[4]) {
    if constexpr (sizeof(T) == 4) {
        float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
        double2 a = *reinterpret_cast<const double2 *>(p);
        double2 b = *reinterpret_cast<const double2 *>(p + 2);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
}
template <typename T>
__device__ __forceinline__ void sts4(T *p, const T (&v)[4]) {
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
        *reinterpret_cast<double2 *>(p + 2) = make_double2(v[2], v[3]);
    }
}

// ---------------------------------------------------------------- cp.async
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void *smem, const void *gmem, int src_bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(s), "l"(gmem), "n"(BYTES), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Slab layout in shared memory: column-major with leading dimension ld = bm,
// the 4-element row chunks of column c XOR-swizzled by (c / 4) mod 8 (masked
// to the chunks a column has): chunk q of column c sits at chunk q ^ sw(c).
// The 4 x 4 tiles give consecutive threads columns 4 apart, so without the
// swizzle (or with the old 4-element pad) a warp's 16-byte loads fell on two
// bank groups (16-way conflicts); with it they cover all eight.
__host__ __device__ inline int sw_mask(int bm) { return (bm >> 2) - 1 < 7 ? (bm >> 2) - 1 : 7; }
// position of row i (0 <= i < bm) of column c inside that column
__device__ __forceinline__ int swz(int c, int i, int mask) {
    return ((((i >> 2) ^ ((c >> 2) & mask)) << 2) | (i & 3));
}

// Copy rows [i0, i0 + bm) of `ncols` columns into dst (the swizzled slab
// layout above, ld), zero-filling rows at or beyond `mend`.  vec: 16-byte
// copies are legal.  `live(c)` false makes column c read as zeros (nothing
// is fetched).
template <typename T, typename ColFn, typename LiveFn>
__device__ __forceinline__ void issue_slab(T *dst, int ld, int ncols, int bm, int64_t i0, int64_t mend,
                                           bool vec, ColFn col, LiveFn live) {
    constexpr int V = 16 / sizeof(T);
    if (vec) {
        const int chunks = bm / V;
        for (int e = threadIdx.x; e < ncols * chunks; e += blockDim.x) {
            const int c = e / chunks, q = e - c * chunks;
            const int64_t row = i0 + (int64_t)q * V;
            const int64_t left = mend - row;
            int bytes = left >= V ? 16 : (left > 0 ? (int)left * (int)sizeof(T) : 0);
            if (!live(c)) bytes = 0;
            const T *src = col(c) + (bytes > 0 ? row : 0);
            cp_async16(dst + (size_t)c * ld + swz(c, q * V, sw_mask(bm)), src, bytes);
        }
    } else {
        for (int e = threadIdx.x; e < ncols * bm; e += blockDim.x) {
            const int c = e / bm, q = e - c * bm;
            const int64_t row = i0 + q;
            const int bytes = (row < mend && live(c)) ? (int)sizeof(T) : 0;
            const T *src = col(c) + (bytes > 0 ? row : 0);
            cp_async_small<sizeof(T)>(dst + (size_t)c * ld + swz(c, q, sw_mask(bm)), src, bytes);
        }
    }
}

struct AllLive {
    __device__ bool operator()(int) const { return true; }
};

// ------------------------------------------------------------ micro-kernels
// Cross-slab accumulators of the Gram-type products.  FP32 data: each 8-byte
// slot holds a double-float (hi, lo) pair updated with TwoSum (FP32 pipes;
// an FP64 add per output and slab cost as much FP64-pipe time as the slab's
// FP32 products, FP64 running ~58x slower than FP32 here); FP64 data: a
// plain double.  acc_read gives the slot's value as a double.
__device__ __forceinline__ void acc_add(double *slot, float s) {
    float2 *p = reinterpret_cast<float2 *>(slot);
    const float2 v = *p;
    const dfloat t = df_two_sum(v.x, s);
    const dfloat n = df_fast_two_sum(t.hi, t.lo + v.y);
    *p = make_float2(n.hi, n.lo);
}
__device__ __forceinline__ void acc_add(double *slot, double s) { *slot += s; }
template <typename T>
__device__ __forceinline__ double acc_read(const double *slot) {
    if constexpr (sizeof(T) == 4) {
        const float2 v = *reinterpret_cast<const float2 *>(slot);
        return (double)v.x + (double)v.y;
    } else {
        return *slot;
    }
}

// Index of tile (ti, tj), ti <= tj, in the row-major enumeration of the
// upper triangle of a tb x tb tile grid (the order tile_of decodes).
__host__ __device__ inline size_t tri_tile(int ti, int tj, int tb) {
    return (size_t)ti * tb - (size_t)ti * (ti - 1) / 2 + (size_t)(tj - ti);
}

// Accumulator slot of output (p, q) of an na x nb product (sym: p <= q of an
// nb x nb Gram).  Outputs are grouped in 4x4 tiles (row-major over the tile
// grid, or over its upper triangle when sym) and stored element-major: slot
// e * nT + tile, e = 4 (p mod 4) + (q mod 4), nT = the number of tiles, so
// the threads of a warp, which hold consecutive tiles, touch consecutive
// slots.
__device__ __forceinline__ double *gram_slot(double *acc, int na, int nb, bool sym, int p, int q) {
    const int tb = (nb + 3) >> 2;
    const int nT = sym ? tb * (tb + 1) / 2 : ((na + 3) >> 2) * tb;
    const size_t tile = sym ? tri_tile(p >> 2, q >> 2, tb) : (size_t)(p >> 2) * tb + (q >> 2);
    return acc + (size_t)((p & 3) * 4 + (q & 3)) * nT + tile;
}

// acc[p][q] += sum_i X[p][i] Y[q][i] over the bm rows of a slab (X, Y
// column-major with leading dimension ld; p < na, q < nb).  Tiles of 4x4
// outputs over 4-row chunks; tiles with ti > tj skipped when sym.  acc slots
// (as in acc_add) laid out as gram_slot gives; red holds blockDim*16 T.  Ends
// with a barrier.
// Tile t of the output grid: row-major over ta x tb tiles, or over the upper
// triangle (ti <= tj) of a tb x tb grid when sym.
__device__ __forceinline__ void tile_of(int t, int tb, bool sym, int &ti, int &tj) {
    if (!sym) {
        ti = t / tb;
        tj = t - ti * tb;
        return;
    }
    int i = 0, rem = t;
    while (rem >= tb - i) {
        rem -= tb - i;
        ++i;
    }
    ti = i;
    tj = i + rem;
}

template <typename T>
__device__ void gram_acc(const T *X, int na, const T *Y, int nb, int ld, int bm, bool sym, double *acc,
                         T *red) {
    const int tid = threadIdx.x, bd = blockDim.x;
    const int msk = sw_mask(bm);
    const int ta = (na + 3) >> 2, tb = (nb + 3) >> 2;
    // only the tiles that are computed (the upper triangle when sym) share out the threads
    const int nT = sym ? tb * (tb + 1) / 2 : ta * tb;
    const int chunks = bm >> 2;
    if (nT == 0) return;
    if (nT * 2 > bd) {
        for (int tile = tid; tile < nT; tile += bd) {
            int ti, tj;
            tile_of(tile, tb, sym, ti, tj);
            T a[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) a[e] = (T)0;
#pragma unroll 2
            for (int rc = 0; rc < chunks; ++rc) {
                T x[4][4], y[4][4];
#pragma unroll
                for (int u = 0; u < 4; ++u) lds4(X + (size_t)(4 * ti + u) * ld + ((rc ^ (ti & msk)) << 2), x[u]);
#pragma unroll
                for (int v = 0; v < 4; ++v) lds4(Y + (size_t)(4 * tj + v) * ld + ((rc ^ (tj & msk)) << 2), y[v]);
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v)
#pragma unroll
                        for (int w = 0; w < 4; ++w) a[u * 4 + v] = fma(x[u][w], y[v][w], a[u * 4 + v]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc_add(&acc[(size_t)(u * 4 + v) * nT + tile], a[u * 4 + v]);
        }
        __syncthreads();
        return;
    }
    const int RG = bd / nT;
    const int tile = tid % nT, grp = tid / nT;
    int ti, tj;
    tile_of(tile, tb, sym, ti, tj);
    T a[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) a[e] = (T)0;
    if (grp < RG) {
#pragma unroll 2
        for (int rc = grp; rc < chunks; rc += RG) {
            T x[4][4], y[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u) lds4(X + (size_t)(4 * ti + u) * ld + ((rc ^ (ti & msk)) << 2), x[u]);
#pragma unroll
            for (int v = 0; v < 4; ++v) lds4(Y + (size_t)(4 * tj + v) * ld + ((rc ^ (tj & msk)) << 2), y[v]);
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v)
#pragma unroll
                    for (int w = 0; w < 4; ++w) a[u * 4 + v] = fma(x[u][w], y[v][w], a[u * 4 + v]);
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) red[(e * RG + grp) * nT + tile] = a[e];
    }
    __syncthreads();
    for (int e = tid; e < nT * 16; e += bd) {
        const int uv = e / nT, t2 = e - uv * nT;
        T s = (T)0;
        for (int g2 = 0; g2 < RG; ++g2) s += red[(uv * RG + g2) * nT + t2];
        acc_add(&acc[e], s);
    }
    __syncthreads();
}

// As gram_acc for a symmetric X^T X with every product split exactly
// (TwoProduct) and summed with TwoSum: the tile sums carry ~44 bits before the
// FP64 flush.  Used for the first CholeskyQR Gram when the plain FP32 one
// proved too inexact (ill-conditioned residual blocks).  Its acc slots are
// plain doubles (FP64 running sums), laid out as gram_slot gives for sym.
// Ends with a barrier.
template <typename T>
__device__ void gram_acc_comp(const T *X, int na, int ld, int bm, double *acc) {
    const int ta = (na + 3) >> 2, nT = ta * ta, nTs = ta * (ta + 1) / 2, chunks = bm >> 2;
    const int msk = sw_mask(bm);
    for (int tile = threadIdx.x; tile < nT; tile += blockDim.x) {
        const int ti = tile / ta, tj = tile - ti * ta;
        if (ti > tj) continue;
        if constexpr (sizeof(T) == 4) {
            float hi[16], lo[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) hi[e] = lo[e] = 0.f;
            for (int rc = 0; rc < chunks; ++rc) {
                float x[4][4], y[4][4];
#pragma unroll
                for (int u = 0; u < 4; ++u) lds4(X + (size_t)(4 * ti + u) * ld + ((rc ^ (ti & msk)) << 2), x[u]);
#pragma unroll
                for (int v = 0; v < 4; ++v) lds4(X + (size_t)(4 * tj + v) * ld + ((rc ^ (tj & msk)) << 2), y[v]);
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v)
#pragma unroll
                        for (int w = 0; w < 4; ++w) {
                            const float p = x[u][w] * y[v][w];
                            const float e = fmaf(x[u][w], y[v][w], -p);
                            const dfloat s = df_two_sum(hi[u * 4 + v], p);
                            hi[u * 4 + v] = s.hi;
                            lo[u * 4 + v] += s.lo + e;
                        }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    acc[(size_t)(u * 4 + v) * nTs + tri_tile(ti, tj, ta)] += (double)hi[u * 4 + v] + (double)lo[u * 4 + v];
        } else {
            double a[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) a[e] = 0.0;
            for (int rc = 0; rc < chunks; ++rc) {
                double x[4][4], y[4][4];
#pragma unroll
                for (int u = 0; u < 4; ++u) lds4(X + (size_t)(4 * ti + u) * ld + ((rc ^ (ti & msk)) << 2), x[u]);
#pragma unroll
                for (int v = 0; v < 4; ++v) lds4(X + (size_t)(4 * tj + v) * ld + ((rc ^ (tj & msk)) << 2), y[v]);
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v)
#pragma unroll
                        for (int w = 0; w < 4; ++w) a[u * 4 + v] = fma(x[u][w], y[v][w], a[u * 4 + v]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[(size_t)(u * 4 + v) * nTs + tri_tile(ti, tj, ta)] += a[u * 4 + v];
        }
    }
    __syncthreads();
}

// Offset of row k of an upper-triangular matrix stored with its rows trimmed
// to whole 4-column chunks: row k holds columns 4 floor(k / 4) .. n4 - 1.
__host__ __device__ inline size_t tri_row_off(int k, int n4) {
    const int a = k >> 2, b = k & 3;
    return (size_t)4 * a * n4 - (size_t)8 * a * (a - 1) + (size_t)b * (n4 - 4 * a);
}

// Row-space products on a slab, tiled 4 rows x 4 output columns:
// a1 = A1 S1 (K1 terms), a2 = A2 S2 (K2 terms); A1, A2 column-major (ld);
// S1, S2 row-major with leading dimensions ls1, ls2; tri: S1 is upper
// triangular with trimmed rows (tri_row_off with n4 = ls1; terms k > column
// skipped).  store(rc, cj, a1, a2) consumes the tile of row chunk rc and
// column chunk cj.
template <typename T, typename Store>
__device__ __forceinline__ void rowspace_tiles(int bm, int N, const T *A1, int K1, const T *S1, int ls1,
                                               const T *A2, int K2, const T *S2, int ls2, int ld, bool tri,
                                               Store store) {
    const int chunks = bm >> 2, tn = (N + 3) >> 2, msk = sw_mask(bm);
    for (int tile = threadIdx.x; tile < chunks * tn; tile += blockDim.x) {
        const int rc = tile % chunks, cj = tile / chunks;
        T a1[4][4], a2[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) a1[u][v] = a2[u][v] = (T)0;
        const int k1end = tri ? min(K1, 4 * cj + 4) : K1;
        size_t soff = 4 * cj;   // S1 offset of (k, 4 cj)
#pragma unroll 4
        for (int k = 0; k < k1end; ++k) {
            T x[4], s[4];
            lds4(A1 + (size_t)k * ld + ((rc ^ ((k >> 2) & msk)) << 2), x);
            lds4(S1 + soff, s);
            // trimmed rows: row k is ls1 - 4 floor(k / 4) long and starts at column 4 floor(k / 4)
            soff += tri ? (size_t)(ls1 - 4 * (k >> 2) - ((k & 3) == 3 ? 4 : 0)) : (size_t)ls1;
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) a1[u][v] = fma(x[u], s[v], a1[u][v]);
        }
#pragma unroll 4
        for (int k = 0; k < K2; ++k) {
            T x[4], s[4];
            lds4(A2 + (size_t)k * ld + ((rc ^ ((k >> 2) & msk)) << 2), x);
            lds4(S2 + (size_t)k * ls2 + 4 * cj, s);
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) a2[u][v] = fma(x[u], s[v], a2[u][v]);
        }
        store(rc, cj, a1, a2);
    }
}

// W = A S for upper triangular S with trimmed rows (tri_row_off, n4 = ls),
// with the work balanced over the threads: output tile (rc, cj) takes the
// k-steps 0 .. K(cj) - 1, K(cj) = min(4 cj + 4, N), cut at m(cj) =
// min(2 cj + 2, K(cj)); thread (rc, cj) forms the first part of tile
// (rc, cj) and the second part of tile (rc, tn - 1 - cj), about 2 tn + 2
// steps for every thread (one tile per thread in rowspace_tiles: the thread
// of the last column did 4 tn).  The second parts meet their first parts
// through red (element-major, tiles x 16 T).  Needs chunks x tn <=
// blockDim.x.  store(rc, cj, w) consumes each tile; ends with a barrier.
template <typename T, typename Store>
__device__ __forceinline__ void rowspace_tri_bal(int bm, int N, const T *A, const T *S, int ls, int ld, T *red,
                                                 Store store) {
    const int chunks = bm >> 2, tn = (N + 3) >> 2, msk = sw_mask(bm), nt = chunks * tn;
    const int t = threadIdx.x;
    T a[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) a[u][v] = (T)0;
    auto part = [&](int rc, int cj, int k0, int k1, T (&acc)[4][4]) {
        size_t soff = tri_row_off(k0, ls) + 4 * cj - 4 * (k0 >> 2);
#pragma unroll 4
        for (int k = k0; k < k1; ++k) {
            T x[4], sv[4];
            lds4(A + (size_t)k * ld + ((rc ^ ((k >> 2) & msk)) << 2), x);
            lds4(S + soff, sv);
            soff += (size_t)(ls - 4 * (k >> 2) - ((k & 3) == 3 ? 4 : 0));
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(x[u], sv[v], acc[u][v]);
        }
    };
    const int rc = t % chunks, cj = t / chunks;
    if (t < nt) {
        const int K = min(4 * cj + 4, N), m = min(2 * cj + 2, K);
        part(rc, cj, 0, m, a);
        const int cj2 = tn - 1 - cj;
        const int K2 = min(4 * cj2 + 4, N), m2 = min(2 * cj2 + 2, K2);
        T b[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) b[u][v] = (T)0;
        part(rc, cj2, m2, K2, b);
        const int t2 = cj2 * chunks + rc;
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) red[(size_t)(u * 4 + v) * nt + t2] = b[u][v];
    }
    __syncthreads();
    if (t < nt) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) a[u][v] += red[(size_t)(u * 4 + v) * nt + t];
        store(rc, cj, a);
    }
    __syncthreads();
}

struct SmemPlan {
    int ld;          // slab leading dimension (= bm; the slabs are swizzled, not padded)
    int r4, c4;
    size_t buf;      // one slab buffer (r4 + c4 columns), elements
    size_t ws;       // W buffer, elements (QR2 pass)
    size_t s1, s2, s3;   // coefficient tiles, elements
    size_t acc1, acc2;   // FP64 accumulators (doubles)
};

// Shared-memory layout of one pass: only what that kind uses.
//   PROJ    acc1 = P (r4 x c4)
//   CGS     S1 = P (r4 x c4); acc1 = P2 (r4 x c4); acc2 = Z^T Z (upper tiles)
//   QR2     W slab; S2 = P2 (r4 x c4), S3 = M1 (trimmed rows); acc2 = W^T W (upper tiles)
//   UPDATE  S1 = X (r4 x r4), S2 = Y (c4 x r4)
__host__ __device__ inline SmemPlan smem_plan(int rmax, int cmax, int bm, int kind) {
    SmemPlan p;
    p.ld = bm;
    p.r4 = round4(rmax);
    p.c4 = round4(cmax);
    const size_t tb = (size_t)p.c4 / 4, tri = tb * (tb + 1) / 2 * 16;
    p.buf = (size_t)(p.r4 + p.c4) * p.ld;
    p.ws = kind == TALL_QR2 ? (size_t)p.c4 * p.ld : 0;
    p.s1 = kind == TALL_CGS ? (size_t)p.r4 * p.c4 : (kind == TALL_UPDATE ? (size_t)p.r4 * p.r4 : 0);
    p.s2 = kind == TALL_QR2 || kind == TALL_UPDATE ? (size_t)p.c4 * p.r4 : 0;
    p.s3 = kind == TALL_QR2 ? tri_row_off(p.c4, p.c4) : 0;   // M1, trimmed rows
    p.acc1 = kind == TALL_PROJ || kind == TALL_CGS ? (size_t)p.r4 * p.c4 : 0;
    p.acc2 = kind == TALL_CGS || kind == TALL_QR2 ? tri : 0;
    return p;
}

template <typename T>
__host__ __device__ inline size_t smem_bytes(const SmemPlan &p, int threads) {
    return (2 * p.buf + p.ws + p.s1 + p.s2 + p.s3) * sizeof(T) + (p.acc1 + p.acc2) * 8 +
           (size_t)threads * 16 * sizeof(T) + 64;
}
// Wide plans keep only the slab buffers and the reduction tile in shared
// memory; the coefficient tiles S1..S3 and the FP64 accumulators live in the
// CTA's slice of global scratch (L2-resident).
template <typename T>
__host__ __device__ inline size_t smem_bytes_wide(const SmemPlan &p, int threads) {
    return (2 * p.buf + p.ws) * sizeof(T) + (size_t)threads * 16 * sizeof(T) + 64;
}
template <typename T>
__host__ __device__ inline size_t gscratch_bytes(const SmemPlan &p) {
    return (((p.s1 + p.s2 + p.s3) * sizeof(T) + 15) / 16) * 16 + (p.acc1 + p.acc2) * 8;
}

// The second CholeskyQR Gram must be near I on its kept indices; if not, the
// first pass lost accuracy (an ill-conditioned residual block): flag the
// round for the compensated rerun (or'ed with the first Cholesky's drop
// test).  Run by one whole CTA on the final G2.
__device__ void g2_check(const double *G2, int g, int cmax, DevState *st) {
    const int tid = threadIdx.x, bd = blockDim.x;
    double dev = 0.0;
    for (int e = tid; e < g * g; e += bd) {
        const int i = e / g, j = e - i * g;
        if (i > j) continue;
        const double gii = __ldcg(G2 + i * cmax + i), gjj = __ldcg(G2 + j * cmax + j);
        if (gii == 0.0 || gjj == 0.0) continue;   // dropped index
        const double d = fabs(__ldcg(G2 + i * cmax + j) - (i == j ? 1.0 : 0.0));
        dev = (d != d) ? 1e300 : (d > dev ? d : dev);
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double y = __shfl_xor_sync(0xffffffffu, dev, o);
        dev = y > dev ? y : dev;
    }
    __shared__ double wmax[TALL_MAX_THREADS / 32];
    if ((tid & 31) == 0) wmax[tid >> 5] = dev;
    __syncthreads();
    if (tid == 0) {
        double mx = 0.0;
        for (int w = 0; w < (bd >> 5); ++w) mx = wmax[w] > mx ? wmax[w] : mx;
        const int rb = st->robust || mx > 0.1;
        st->robust = rb;
        st->robust_rounds += rb;
    }
}

// Sums of the deferred partials: CTA (x, y) owns output row y (rectangle
// rows first, then triangle rows) and columns 32x .. 32x + 31; warp w adds
// partials w, w + 8, w + 16, ... in that order (four loads in flight), and
// the eight warp sums are added in warp order: a fixed order, so results
// are reproducible run to run.  With a check, the last CTA to arrive
// inspects the finished G2.
constexpr int SUM_THREADS = 256;
__global__ void __launch_bounds__(SUM_THREADS) k_sum_parts(SumParts a) {
    const DevState *st = a.st;
    if (st->done) return;
    const int r = st->r_cur, g = st->g;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int row = blockIdx.y, c0 = 0;
    int64_t off = 0;
    bool act;
    if (a.rect && row < a.rows_rect) {
        act = row < r;
        off = (int64_t)row * a.ld;
    } else {
        row -= a.rect ? a.rows_rect : 0;
        act = a.tri && row < g;
        off = a.tri_off + (int64_t)row * a.ld;
        c0 = row;
    }
    const int j = blockIdx.x * 32 + lane;
    const bool live = act && j >= c0 && j < g;
    __shared__ double red[SUM_THREADS / 32][32];
    if (act && blockIdx.x * 32 + 31 >= c0 && blockIdx.x * 32 < g) {
        double s = 0.0;
        if (live) {
            const double *p0 = a.part + off + j;
            int b = w;
            for (; b + 24 < a.nparts; b += 32) {
                const double v0 = __ldcg(p0 + (int64_t)b * a.stride), v1 = __ldcg(p0 + (int64_t)(b + 8) * a.stride);
                const double v2 = __ldcg(p0 + (int64_t)(b + 16) * a.stride), v3 = __ldcg(p0 + (int64_t)(b + 24) * a.stride);
                s += v0;
                s += v1;
                s += v2;
                s += v3;
            }
            for (; b < a.nparts; b += 8) s += __ldcg(p0 + (int64_t)b * a.stride);
        }
        red[w][lane] = s;
        __syncthreads();
        if (w == 0) {
            double dev = 0.0;
            if (live) {
                double t = 0.0;
                for (int k = 0; k < SUM_THREADS / 32; ++k) t += red[k][lane];
                a.out[off + j] = t;
                // |G2 - I| on the kept indices: a dropped index has a zero row,
                // column and diagonal
                if (a.check) {
                    const double d = j == row ? (t == 0.0 ? 0.0 : fabs(t - 1.0)) : fabs(t);
                    dev = d != d ? 1e300 : d;
                }
            }
            if (a.check) {
                for (int o = 16; o > 0; o >>= 1) dev = fmax(dev, __shfl_xor_sync(0xffffffffu, dev, o));
                if (lane == 0 && dev > 0.0) atomicMax(a.devmax, (unsigned long long)__double_as_longlong(dev));
            }
        }
    }
    if (a.check) {
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            const unsigned total = gridDim.x * gridDim.y;
            if (atomicAdd(a.counter, 1u) == total - 1) {
                // the last CTA: every row's deviation is in
                __threadfence();
                *a.counter = 0;
                const double mx = __longlong_as_double((long long)atomicExch(a.devmax, 0ull));
                DevState *sw = a.check;
                const int rb = sw->robust || mx > 0.1;   // or'ed with the first Cholesky's drop test
                sw->robust = rb;
                sw->robust_rounds += rb;
            }
        }
    }
}

template <typename T, int KIND>
__global__ void __launch_bounds__(TALL_MAX_THREADS) k_tall(TallArgs<T> a) {
    const DevState *st = a.st;
    if (st->done) return;
    if (a.cond && !st->robust) return;
    const int r = st->r_cur, g = st->g, rn = st->r_new;
    const int bm = a.bm;
    const SmemPlan L = smem_plan(a.rmax, a.cmax, bm, KIND);
    const int ld = L.ld, msk = sw_mask(bm);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *buf0 = reinterpret_cast<T *>(smem_raw);
    T *buf1 = buf0 + L.buf;
    T *Ws = buf1 + L.buf;
    T *S1, *S2, *S3, *red;
    double *acc1, *acc2;
    if (a.gscratch) {
        unsigned char *gs = a.gscratch + (int64_t)blockIdx.x * a.gstride;
        S1 = reinterpret_cast<T *>(gs);
        S2 = S1 + L.s1;
        S3 = S2 + L.s2;
        acc1 = reinterpret_cast<double *>(gs + (((L.s1 + L.s2 + L.s3) * sizeof(T) + 15) / 16) * 16);
        acc2 = acc1 + L.acc1;
        red = Ws + L.ws;
    } else {
        S1 = Ws + L.ws;
        S2 = S1 + L.s1;
        S3 = S2 + L.s2;
        acc1 = reinterpret_cast<double *>(S3 + L.s3);
        acc2 = acc1 + L.acc1;
        red = reinterpret_cast<T *>(acc2 + L.acc2);
    }
    int *s_flag = reinterpret_cast<int *>(red + blockDim.x * 16);
    const int tid = threadIdx.x, bd = blockDim.x;
    const int r4 = round4(r), g4 = round4(g), rn4 = round4(rn);
    const bool vec = a.vec != 0;
    const bool load_c = KIND != TALL_UPDATE || g > 0;
    auto ucol = [&](int l) { return a.U + (int64_t)l * a.ldu; };
    auto ccol = [&](int j) { return a.A + (int64_t)(a.idx ? a.idx[j] : j) * a.lda; };

    // zero the padding columns of both buffers once; small operands -> shared
    for (int b = 0; b < 2; ++b) {
        T *Ub = b ? buf1 : buf0;
        T *Cb = Ub + (size_t)L.r4 * ld;
        for (int e = tid; e < (r4 - r) * ld; e += bd) Ub[(size_t)r * ld + e] = (T)0;
        for (int e = tid; e < (g4 - g) * ld; e += bd) Cb[(size_t)g * ld + e] = (T)0;
    }
    if (KIND == TALL_CGS || KIND == TALL_QR2) {
        for (int e = tid; e < r4 * g4; e += bd) {
            const int l = e / g4, j = e - l * g4;
            if (KIND == TALL_CGS) S1[e] = (l < r && j < g) ? (T)a.P[l * a.cmax + j] : (T)0;
            else S2[e] = (l < r && j < g) ? (T)a.P2[l * a.cmax + j] : (T)0;
        }
    }
    if (KIND == TALL_QR2) {
        // M1 with trimmed rows (tri_row_off, n4 = g4)
        for (int e = tid; e < g4 * g4; e += bd) {
            const int l = e / g4, j = e - l * g4;
            if (j < 4 * (l >> 2)) continue;
            S3[tri_row_off(l, g4) + j - 4 * (l >> 2)] = (l < g && j < g && l <= j) ? (T)a.M1[l * a.cmax + j] : (T)0;
        }
        for (int e = tid; e < (g4 - g) * ld; e += bd) Ws[(size_t)g * ld + e] = (T)0;
    }
    if (KIND == TALL_UPDATE) {
        for (int e = tid; e < r4 * rn4; e += bd) {
            const int l = e / rn4, q = e - l * rn4;
            S1[e] = (l < r && q < rn) ? (T)a.Xm[l * a.rmax + q] : (T)0;
        }
        for (int e = tid; e < g4 * rn4; e += bd) {
            const int j = e / rn4, q = e - j * rn4;
            S2[e] = (j < g && q < rn) ? (T)a.Ym[j * a.rmax + q] : (T)0;
        }
    }
    if (KIND != TALL_UPDATE) {
        for (int e = tid; e < (int)L.acc1; e += bd) acc1[e] = 0.0;
        for (int e = tid; e < (int)L.acc2; e += bd) acc2[e] = 0.0;
    }

    const int64_t step = (int64_t)gridDim.x * bm;
    int64_t i0 = (int64_t)blockIdx.x * bm;
    if (i0 < a.m) {
        issue_slab<T>(buf0, ld, r, bm, i0, a.m, vec, ucol, AllLive{});
        if (load_c) issue_slab<T>(buf0 + (size_t)L.r4 * ld, ld, g, bm, i0, a.m, vec, ccol, AllLive{});
    }
    cp_async_commit();
    int b = 0;
    for (; i0 < a.m; i0 += step, b ^= 1) {
        T *Us = b ? buf1 : buf0;
        T *Cs = Us + (size_t)L.r4 * ld;
        const int64_t inext = i0 + step;
        if (inext < a.m) {
            T *Un = b ? buf0 : buf1;
            issue_slab<T>(Un, ld, r, bm, inext, a.m, vec, ucol, AllLive{});
            if (load_c) issue_slab<T>(Un + (size_t)L.r4 * ld, ld, g, bm, inext, a.m, vec, ccol, AllLive{});
        }
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        if (KIND == TALL_PROJ) {
            gram_acc<T>(Us, r, Cs, g, ld, bm, false, acc1, red);
        } else if (KIND == TALL_CGS) {
            // Z is also stored (a.Wout) for the QR2 pass, which then only
            // removes U P2
            const int64_t rows_left = a.m - i0;
            if (r > 0) {
                const bool zvec = (a.ldw * (int64_t)sizeof(T)) % 16 == 0;
                rowspace_tiles<T>(bm, g, Us, r, S1, g4, Us, 0, S2, g4, ld, false,
                                  [&](int rc, int cj, T (&a1)[4][4], T (&)[4][4]) {
#pragma unroll
                                      for (int v = 0; v < 4; ++v) {
                                          T *p = Cs + (size_t)(4 * cj + v) * ld + ((rc ^ (cj & msk)) << 2);
                                          T z[4];
                                          lds4(p, z);
#pragma unroll
                                          for (int u = 0; u < 4; ++u) z[u] -= a1[u][v];
                                          sts4(p, z);
                                          const int q = 4 * cj + v;
                                          if (!a.Wout || q >= g) continue;
                                          T *dst = a.Wout + (int64_t)q * a.ldw + i0 + 4 * rc;
                                          if (zvec && rows_left >= 4 * rc + 4) {
                                              sts4(dst, z);
                                          } else {
#pragma unroll
                                              for (int u = 0; u < 4; ++u)
                                                  if (4 * rc + u < rows_left) dst[u] = z[u];
                                          }
                                      }
                                  });
                __syncthreads();
                gram_acc<T>(Us, r, Cs, g, ld, bm, false, acc1, red);
            } else if (a.Wout) {
                const int nrow = rows_left < bm ? (int)rows_left : bm;
                for (int e = tid; e < g * bm; e += bd) {
                    const int j = e / bm, i = e - j * bm;
                    if (i < nrow) a.Wout[(int64_t)j * a.ldw + i0 + i] = Cs[(size_t)j * ld + swz(j, i, msk)];
                }
            }
            if (a.cond) gram_acc_comp<T>(Cs, g, ld, bm, acc2);
            else gram_acc<T>(Cs, g, Cs, g, ld, bm, true, acc2, red);
        } else if (KIND == TALL_QR2) {
            // the C operand is Z = C - U P as the CGS pass stored it
            if (r > 0) {
                rowspace_tiles<T>(bm, g, Us, r, S2, g4, Us, 0, S2, g4, ld, false,
                                  [&](int rc, int cj, T (&a2)[4][4], T (&)[4][4]) {
#pragma unroll
                                      for (int v = 0; v < 4; ++v) {
                                          T *p = Cs + (size_t)(4 * cj + v) * ld + ((rc ^ (cj & msk)) << 2);
                                          T z[4];
                                          lds4(p, z);
#pragma unroll
                                          for (int u = 0; u < 4; ++u) z[u] -= a2[u][v];
                                          sts4(p, z);
                                      }
                                  });
                __syncthreads();
            }
            auto store_w = [&](int rc, int cj, T (&a1)[4][4]) {
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    T w[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) w[u] = a1[u][v];
                    sts4(Ws + (size_t)(4 * cj + v) * ld + ((rc ^ (cj & msk)) << 2), w);
                }
            };
            if ((bm >> 2) * ((g + 3) >> 2) <= bd) {
                rowspace_tri_bal<T>(bm, g, Cs, S3, g4, ld, red, store_w);
            } else {
                rowspace_tiles<T>(bm, g, Cs, g, S3, g4, Cs, 0, S3, g4, ld, true,
                                  [&](int rc, int cj, T (&a1)[4][4], T (&)[4][4]) { store_w(rc, cj, a1); });
                __syncthreads();
            }
            if (a.Wout) {
                // W itself for the UPDATE pass: Q = W R2^{-1} is then formed from
                // the very W whose Gram gave R2 (explicit CholeskyQR2)
                const int64_t left = a.m - i0;
                const int nrow = left < bm ? (int)left : bm;
                for (int e = tid; e < g * bm; e += bd) {
                    const int j = e / bm, i = e - j * bm;
                    if (i < nrow) a.Wout[(int64_t)j * a.ldw + i0 + i] = Ws[(size_t)j * ld + swz(j, i, msk)];
                }
            }
            gram_acc<T>(Ws, g, Ws, g, ld, bm, true, acc2, red);
        } else {
            const int64_t rows_left = a.m - i0;
            rowspace_tiles<T>(bm, rn, Us, r, S1, rn4, Cs, g, S2, rn4, ld, false,
                              [&](int rc, int cj, T (&a1)[4][4], T (&a2)[4][4]) {
#pragma unroll
                                  for (int v = 0; v < 4; ++v) {
                                      const int q = 4 * cj + v;
                                      if (q >= rn) continue;
                                      T o[4];
#pragma unroll
                                      for (int u = 0; u < 4; ++u) o[u] = a1[u][v] + a2[u][v];
                                      T *dst = a.U + (int64_t)q * a.ldu + i0 + 4 * rc;
                                      if (vec && rows_left >= 4 * rc + 4) {
                                          sts4(dst, o);
                                      } else {
#pragma unroll
                                          for (int u = 0; u < 4; ++u)
                                              if (4 * rc + u < rows_left) dst[u] = o[u];
                                      }
                                  }
                              });
        }
        __syncthreads();
    }
    cp_async_wait<0>();
    // a CTA whose first slab lies beyond m never entered the loop: its
    // accumulators were zeroed by all threads with no barrier since
    __syncthreads();
    if (KIND == TALL_UPDATE) {
        if (a.finish) {
            // end of the round, by the last CTA to finish its rows (every CTA
            // read the round's sizes before arriving)
            __threadfence();
            __syncthreads();
            if (tid == 0 && atomicAdd(a.finish, 1u) == gridDim.x - 1) {
                *a.finish = 0;
                DevState *sw = const_cast<DevState *>(st);
                sw->r_cur = sw->r_new;
                sw->t += 1;
                sw->rounds_run += 1;
                if (sw->done_next) sw->done = 1;
            }
        }
        return;
    }
    // this CTA's FP64 partial, then the in-kernel fixed-order sum
    double *out = a.part + (int64_t)blockIdx.x * a.part_stride;
    if (KIND == TALL_PROJ) {
        for (int e = tid; e < r * g; e += bd) {
            const int l = e / g, j = e - l * g;
            out[l * a.cmax + j] = acc_read<T>(gram_slot(acc1, r, g, false, l, j));
        }
    } else if (KIND == TALL_CGS) {
        for (int e = tid; e < r * g; e += bd) {
            const int l = e / g, j = e - l * g;
            out[l * a.cmax + j] = acc_read<T>(gram_slot(acc1, r, g, false, l, j));
        }
        double *outG = out + (int64_t)a.rmax * a.cmax;
        for (int e = tid; e < g * g; e += bd) {
            const int p = e / g, q = e - p * g;
            // the compensated Gram of the rerun keeps FP64 running sums
            if (p <= q) outG[p * a.cmax + q] = a.cond ? *gram_slot(acc2, g, g, true, p, q)
                                                       : acc_read<T>(gram_slot(acc2, g, g, true, p, q));
        }
    } else {
        for (int e = tid; e < g * g; e += bd) {
            const int p = e / g, q = e - p * g;
            if (p <= q) out[p * a.cmax + q] = acc_read<T>(gram_slot(acc2, g, g, true, p, q));
        }
    }
    if (a.defer) return;   // summed by k_sum_parts
    const bool last = tall_reduce(a.part, a.gsum, a.out, (int)a.part_stride, a.part_stride, a.counters, s_flag);
    if (KIND == TALL_QR2 && !a.cond && last) {
        __threadfence();
        g2_check(a.out, g, a.cmax, const_cast<DevState *>(st));
    }
}

// ---------------------------------------------------------------------------
// Y = A^T U.  CTA (blockIdx.x, blockIdx.y) owns nb columns of A and a range
// of rows; its FP64 partial of the nb x r block of Y is summed over the
// row ranges by the last CTA of the column block to arrive.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(TALL_THREADS) k_atu(AtuArgs<T> a, int nb, int bm) {
    const DevState *st = a.st;
    if (st->done) return;
    const int r = st->r_cur;
    const int64_t j0 = (int64_t)blockIdx.x * nb;
    const int ncols = (int)((a.n - j0) < nb ? (a.n - j0) : nb);
    const int split = gridDim.y;
    const int64_t rows_per = ((a.m + split - 1) / split + bm - 1) / bm * bm;
    const int64_t ib = (int64_t)blockIdx.y * rows_per;
    const int64_t ie = (ib + rows_per) < a.m ? (ib + rows_per) : a.m;
    const int nb4 = round4(nb), r4 = round4(a.rmax);
    const int ld = bm;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *buf0 = reinterpret_cast<T *>(smem_raw);
    const size_t bsz = (size_t)(nb4 + r4) * ld;
    T *buf1 = buf0 + bsz;
    double *acc = reinterpret_cast<double *>(buf1 + bsz);
    T *red = reinterpret_cast<T *>(acc + (size_t)nb4 * r4);
    int *s_flag = reinterpret_cast<int *>(red + TALL_THREADS * 16);
    const int tid = threadIdx.x, bd = blockDim.x;
    const bool vec = a.vec != 0;
    for (int e = tid; e < nb4 * r4; e += bd) acc[e] = 0.0;
    bool any = true;
    if (a.mask) {
        any = false;
        for (int c = 0; c < ncols; ++c) any |= a.mask[j0 + c] != 0;
    }
    for (int bb = 0; bb < 2; ++bb) {
        T *Ab = bb ? buf1 : buf0;
        T *Ub = Ab + (size_t)nb4 * ld;
        for (int e = tid; e < (nb4 - ncols) * ld; e += bd) Ab[(size_t)ncols * ld + e] = (T)0;
        for (int e = tid; e < (round4(r) - r) * ld; e += bd) Ub[(size_t)r * ld + e] = (T)0;
    }
    __syncthreads();
    if (any && r > 0 && ib < ie) {
        auto acol = [&](int c) { return a.A + (j0 + c) * a.lda; };
        auto ucol = [&](int l) { return a.U + (int64_t)l * a.ldu; };
        auto live = [&](int c) { return a.mask == nullptr || a.mask[j0 + c] != 0; };
        auto issue = [&](T *dst, int64_t i0) {
            issue_slab<T>(dst, ld, ncols, bm, i0, ie, vec, acol, live);
            issue_slab<T>(dst + (size_t)nb4 * ld, ld, r, bm, i0, ie, vec, ucol, AllLive{});
        };
        issue(buf0, ib);
        cp_async_commit();
        int b = 0;
        for (int64_t i0 = ib; i0 < ie; i0 += bm, b ^= 1) {
            T *As = b ? buf1 : buf0;
            if (i0 + bm < ie) issue(b ? buf0 : buf1, i0 + bm);
            cp_async_commit();
            cp_async_wait<1>();
            __syncthreads();
            gram_acc<T>(As, ncols, As + (size_t)nb4 * ld, r, ld, bm, false, acc, red);
        }
        cp_async_wait<0>();
    }
    __syncthreads();
    // partial: column-major n x r (ld n) per row range
    double *out = a.part + (int64_t)blockIdx.y * a.n * a.rmax;
    for (int e = tid; e < ncols * r; e += bd) {
        const int l = e / ncols, c = e - l * ncols;
        out[(int64_t)l * a.n + j0 + c] = acc_read<T>(gram_slot(acc, ncols, r, false, c, l));
    }
    // the last of the `split` CTAs of this column block sums them
    __threadfence();
    __syncthreads();
    if (tid == 0) *s_flag = (atomicAdd(&a.counters[blockIdx.x], 1u) == (unsigned)(split - 1));
    __syncthreads();
    if (!*s_flag) return;
    __threadfence();
    for (int e = tid; e < ncols * r; e += bd) {
        const int l = e / ncols, c = e - l * ncols;
        double s = 0.0;
        for (int y = 0; y < split; ++y)
            s += __ldcg(a.part + (int64_t)y * a.n * a.rmax + (int64_t)l * a.n + j0 + c);
        a.Y[(int64_t)l * a.n + j0 + c] = s;
    }
    if (tid == 0) a.counters[blockIdx.x] = 0;
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

template <typename T, int KIND>
pod_status launch_kind(const TallArgs<T> &a0, const TallPlan &plan, cudaStream_t st) {
    // each kind has its own slab height and shared-memory layout
    TallArgs<T> a = a0;
    a.bm = plan.bm_k[KIND];
    if (!plan.wide_k[KIND]) a.gscratch = nullptr;
    const size_t smem = plan.smem_k[KIND];
    POD_CUDA_TRY(cudaFuncSetAttribute(k_tall<T, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int threads = plan.threads_k[KIND] ? plan.threads_k[KIND] : TALL_THREADS;
    k_tall<T, KIND><<<plan.grid, threads, smem, st>>>(a);
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}

}  // namespace

pod_status launch_sum_parts(const SumParts &a, int cols_cap, cudaStream_t s) {
    const int rows = (a.rect ? a.rows_rect : 0) + (a.tri ? cols_cap : 0);
    dim3 grid((unsigned)((cols_cap + 31) / 32), (unsigned)rows);
    k_sum_parts<<<grid, SUM_THREADS, 0, s>>>(a);
    POD_CUDA_TRY(cudaGetLastError());
    return POD_OK;
}


// Threads of a one-CTA-per-SM pass: enough that each of its tile loops
// (row-space tiles of a slab, Gram tiles) takes one round, within 256..512.
static int tall_threads_for(int kind, int bm, int rmax, int cmax) {
    const int rt = round4(rmax) / 4, ct = round4(cmax) / 4, ch = bm / 4;
    int tiles = 0;
    auto mx = [&](int t) { tiles = t > tiles ? t : tiles; };
    if (kind == TALL_PROJ) mx(rt * ct);
    if (kind == TALL_CGS) {
        mx(ch * ct);
        mx(rt * ct);
        mx(ct * (ct + 1) / 2);
    }
    if (kind == TALL_QR2) {
        mx(ch * ct);
        mx(ct * (ct + 1) / 2);
    }
    if (kind == TALL_UPDATE) mx(ch * rt);
    int th = (tiles + 31) / 32 * 32;
    return th < TALL_THREADS ? TALL_THREADS : (th > TALL_MAX_THREADS ? TALL_MAX_THREADS : th);
}

TallPlan tall_plan(int dtype, int64_t m, int rmax, int cmax, int num_sms) {
    TallPlan p{};
    const bool f32 = dtype == POD_F32;
    auto bytes_for = [&](int bm, int kind, int th) {
        SmemPlan L = smem_plan(rmax, cmax, bm, kind);
        return f32 ? smem_bytes<float>(L, th) : smem_bytes<double>(L, th);
    };
    auto wide_for = [&](int bm, int kind) {
        SmemPlan L = smem_plan(rmax, cmax, bm, kind);
        return f32 ? smem_bytes_wide<float>(L, TALL_THREADS) : smem_bytes_wide<double>(L, TALL_THREADS);
    };
    // two resident CTAs per SM (16 warps) when every kind fits in 110 KB with
    // slabs of at least 32 rows and 256 threads; else one CTA per SM, each
    // kind with the tallest slab whose layout fits in 220 KB and as many
    // threads as its tile loops can use (tall_threads_for); a kind that does
    // not fit even with 16-row slabs keeps its coefficient tiles and
    // accumulators in global scratch (wide, 256 threads)
    int per_sm = 2;
    for (int k = 0; k < 4 && per_sm == 2; ++k) {
        int bm = 0;
        for (int b = 128; b >= 32 && !bm; b >>= 1)
            if (bytes_for(b, k, TALL_THREADS) <= 110 * 1024) bm = b;
        if (!bm) per_sm = 1;
        p.bm_k[k] = bm;
        p.smem_k[k] = bm ? bytes_for(bm, k, TALL_THREADS) : 0;
        p.threads_k[k] = TALL_THREADS;
    }
    if (per_sm == 1) {
        for (int k = 0; k < 4; ++k) {
            int bm = 0, th = TALL_THREADS;
            for (int b = 128; b >= 16 && !bm; b >>= 1) {
                th = tall_threads_for(k, b, rmax, cmax);
                if (bytes_for(b, k, th) <= 220 * 1024) bm = b;
            }
            p.wide_k[k] = 0;
            if (bm) {
                p.bm_k[k] = bm;
                p.smem_k[k] = bytes_for(bm, k, th);
                p.threads_k[k] = th;
                continue;
            }
            bm = 16;
            for (int b = 64; b >= 16; b >>= 1)
                if (wide_for(b, k) <= 200 * 1024) {
                    bm = b;
                    break;
                }
            SmemPlan L = smem_plan(rmax, cmax, bm, k);
            p.bm_k[k] = bm;
            p.smem_k[k] = wide_for(bm, k);
            p.threads_k[k] = TALL_THREADS;
            p.wide_k[k] = 1;
            const int64_t gs = (int64_t)(f32 ? gscratch_bytes<float>(L) : gscratch_bytes<double>(L));
            if (gs > p.gstride) p.gstride = gs;
        }
    }
    p.bm = p.bm_k[TALL_PROJ];
    p.smem = 0;
    p.wide = 0;
    for (int k = 0; k < 4; ++k) {
        if (p.smem_k[k] > p.smem) p.smem = p.smem_k[k];
        p.wide |= p.wide_k[k];
    }
    // CTAs: at most one per slab of the tallest kind, so that every CTA of
    // every kind has rows (idle CTAs would only add zero partials)
    int bmx = 16;
    for (int k = 0; k < 4; ++k)
        if (p.bm_k[k] > bmx) bmx = p.bm_k[k];
    const int64_t slabs = (m + bmx - 1) / bmx;
    int64_t grid = (int64_t)per_sm * num_sms;
    if (grid > slabs) grid = slabs;
    if (grid < 1) grid = 1;
    p.grid = (int)grid;
    p.groups = (p.grid + RED_GROUP - 1) / RED_GROUP;
    return p;
}

template <typename T>
pod_status launch_tall(TallKind kind, const TallArgs<T> &a, const TallPlan &plan, cudaStream_t st) {
    if (plan.smem > 227 * 1024) return POD_EUNSUPPORTED;
    switch (kind) {
        case TALL_PROJ: return launch_kind<T, TALL_PROJ>(a, plan, st);
        case TALL_CGS: return launch_kind<T, TALL_CGS>(a, plan, st);
        case TALL_QR2: return launch_kind<T, TALL_QR2>(a, plan, st);
        default: return launch_kind<T, TALL_UPDATE>(a, plan, st);
    }
}

AtuPlan atu_plan(int dtype, int64_t m, int64_t n, int rmax, int num_sms) {
    AtuPlan p{};
    const size_t es = dtype == POD_F32 ? 4 : 8;
    p.nb = 32;
    p.bm = 128;
    const int nb4 = round4(p.nb), r4 = round4(rmax);
    for (;;) {
        p.smem = 2 * (size_t)(nb4 + r4) * p.bm * es + (size_t)nb4 * r4 * 8 + TALL_THREADS * 16 * es + 64;
        if (p.smem <= 110 * 1024 || p.bm <= 16) break;
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
    k_atu<T><<<plan.grid, TALL_THREADS, plan.smem, st>>>(a, plan.nb, plan.bm);
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
