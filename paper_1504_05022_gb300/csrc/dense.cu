// Stage 3, bin group 5, for the rows whose products cover a large part of B's
// column range (and, in the precise method, for every bin-37 row): an accumulator
// over column slices instead of the merge of Section 4.1.
//
// B's columns are cut into K slices of W columns (W a multiple of 32, at most
// DENSE_W_MAX, K W >= ncols).  A slice of a row is one CTA.  The counting pass marks
// the columns of the row's products in the slice in a shared bitmap and counts its
// bits, and may leave the bitmap in device memory.  The fill pass reads it back (or marks
// the columns again when it was not kept), ranks the bitmap (set bits before each word),
// and adds every product into a compact buffer of sums, one per column of the result,
// at its column's rank: clearing and writing out cost the slice's entries, not its
// width, and the sums come out in column order.  There are no misses, no merges and no
// capacity to outgrow (a slice with more entries than the buffer is done in pieces).
// The part of each B row that falls in slice s is read from a table of per-row slice
// boundaries, built once per call, and is cut into chunks of consecutive entries that
// the warps share out.
//
// Because the rows are counted first, they need no temporary result rows: their sizes
// go into the row counts of C with the other rows', and the values are written
// straight into C once its row pointers exist (the kept bitmaps, W / 8 bytes per
// (row, slice), are the only temporary, and an optional one).  The same launch recomputes the values
// for a values-only replay.
#include "internal.h"
#include "common.cuh"

#include <algorithm>

namespace spg {

// ---- per-B-row slice boundaries ----

__global__ void k_dense_bounds(DevCSR B, int K, int W, int32_t *bnd) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B.nrows * (K + 1)) return;
    const int64_t k = i / (K + 1);
    const int s = (int)(i - k * (K + 1));
    const int64_t rs = B.rp[k];
    const int n = (int)(B.rp[k + 1] - rs);
    int v;
    if (s == 0) v = 0;
    else if (s == K) v = n;
    else v = lower_bound_i32(B.col + rs, n, (int32_t)((int64_t)s * W));
    bnd[i] = v;
}

cudaError_t launch_dense_bounds(const DevCSR &B, int K, int W, int32_t *bnd, cudaStream_t st) {
    const int64_t n = B.nrows * (K + 1);
    if (n <= 0 || K <= 1) return cudaSuccess;
    k_dense_bounds<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(B, K, W, bnd);
    return cudaGetLastError();
}

// ---- which bin-37 rows are dense ----
// One warp per row: u_i from the stage-1 prefix, and for u_i > 512 the row's column
// range [lo, hi) (first and last column of every touched B row).  The row is dense when
// u_i >= dmin (dmin > 0), else when div u_i >= hi - lo: its products cover at least a
// div-th of the columns they can reach, so the dense accumulator's O(hi - lo) clearing
// and write-out are small beside them.
__global__ void k_dense_mark(DevCSR A, DevCSR B, const int64_t *__restrict__ S, int64_t dmin, int div,
                             uint8_t *flag, int32_t *lo, int32_t *hi) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= A.nrows) return;
    const int64_t a0 = A.rp[row], a1 = A.rp[row + 1];
    const int64_t u = S[a1] - S[a0];
    if (u <= BIN_MERGE_MIN_U) {
        if (lane == 0) flag[row] = 0;
        return;
    }
    int32_t cmin = INT32_MAX, cmax = -1;
    for (int64_t e = a0 + lane; e < a1; e += 32) {
        const int32_t k = A.col[e];
        const int64_t rs = B.rp[k], re = B.rp[k + 1];
        if (re > rs) {
            cmin = min(cmin, B.col[rs]);
            cmax = max(cmax, B.col[re - 1]);
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        cmin = min(cmin, __shfl_xor_sync(SPG_FULL, cmin, d));
        cmax = max(cmax, __shfl_xor_sync(SPG_FULL, cmax, d));
    }
    if (lane == 0) {
        const int64_t span = (int64_t)cmax - cmin + 1;  // u > 0, so some B row is not empty
        flag[row] = (uint8_t)(dmin > 0 ? u >= dmin : (int64_t)div * u >= span);
        lo[row] = cmin;
        hi[row] = cmax + 1;
    }
}

cudaError_t launch_dense_mark(const DevCSR &A, const DevCSR &B, const int64_t *S, int64_t dmin, int div,
                              uint8_t *flag, int32_t *lo, int32_t *hi, cudaStream_t st) {
    if (A.nrows <= 0) return cudaSuccess;
    if (div < 1) return cudaErrorInvalidValue;
    const int64_t threads = A.nrows * 32;
    k_dense_mark<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(A, B, S, dmin, div, flag, lo, hi);
    return cudaGetLastError();
}

// ---- selection of the dense rows among the bin-37 rows ----
// Bucket g = 63 - floor(log2 u) (the leading zeros of u) for a dense row, so that
// larger rows come first; DENSE_BUCKETS for the others.  order[0..nd) lists the
// dense items, order[nd..n37) the rest.

constexpr int DENSE_BUCKETS = 64;

__global__ void k_dense_select_count(const int32_t *bin_rows, int64_t m, const BinSummary *summary, const int64_t *u,
                                     const uint8_t *flag, int32_t *cls_of, int32_t *count) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n37 = summary->bin_count[BIN_MERGE];
    if (j >= n37) return;
    const int32_t row = bin_rows[m - n37 + j];
    const int64_t uu = u[row];
    const int g = flag[row] ? __clzll((long long)uu) : DENSE_BUCKETS;
    cls_of[j] = g;
    atomicAdd(&count[g], 1);
}

__global__ void k_dense_select_starts(const int32_t *count, int32_t *start, int32_t *cursor, BinSummary *summary) {
    if (threadIdx.x == 0) {
        int32_t s = 0;
        for (int g = 0; g <= DENSE_BUCKETS; ++g) {
            start[g] = s;
            cursor[g] = 0;
            if (g == DENSE_BUCKETS) summary->dense_count = s;
            s += count[g];
        }
    }
}

__global__ void k_dense_select_scatter(const int32_t *bin_rows, int64_t m, const BinSummary *summary,
                                       const int32_t *cls_of, const int32_t *start, int32_t *cursor,
                                       const int32_t *lo, const int32_t *hi, int32_t *order, int32_t *rows,
                                       int32_t *rlo, int32_t *rhi) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n37 = summary->bin_count[BIN_MERGE];
    if (j >= n37) return;
    const int g = cls_of[j];
    const int32_t pos = start[g] + atomicAdd(&cursor[g], 1);
    order[pos] = (int32_t)j;
    if (g < DENSE_BUCKETS) {
        const int32_t row = bin_rows[m - n37 + j];
        rows[pos] = row;
        rlo[pos] = lo[row];
        rhi[pos] = hi[row];
    }
}

int64_t dense_select_scratch(int64_t m) { return 3 * (DENSE_BUCKETS + 1) + m; }

cudaError_t launch_dense_select(const int32_t *bin_rows, int64_t m, BinSummary *summary, const int64_t *u,
                                const uint8_t *flag, const int32_t *lo, const int32_t *hi, int32_t *scratch,
                                int32_t *order, int32_t *rows, int32_t *rlo, int32_t *rhi, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    int32_t *count = scratch, *start = count + DENSE_BUCKETS + 1, *cursor = start + DENSE_BUCKETS + 1,
            *cls_of = cursor + DENSE_BUCKETS + 1;
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int32_t) * (DENSE_BUCKETS + 1), st);
    if (e != cudaSuccess) return e;
    const unsigned g = (unsigned)((m + 255) / 256);
    k_dense_select_count<<<g, 256, 0, st>>>(bin_rows, m, summary, u, flag, cls_of, count);
    k_dense_select_starts<<<1, 32, 0, st>>>(count, start, cursor, summary);
    k_dense_select_scatter<<<g, 256, 0, st>>>(bin_rows, m, summary, cls_of, start, cursor, lo, hi, order, rows, rlo,
                                              rhi);
    return cudaGetLastError();
}

// ---- the product expansion shared by the count and fill kernels ----
// Walks the A entries of `row` in windows of WIN (<= NT); wbs holds 2 WIN entries (the
// parts' starts, then their lengths).  Where the window's parts -- the selected B rows'
// entries inside slice s -- average DENSE_FLAT_BELOW products or more, they are cut into
// chunks of DENSE_CH entries and warp w takes the w-th contiguous range of the chunks, its
// lanes a chunk's entries 32 at a time.  Shorter parts (the slices of a wide B cut most
// sparse rows into parts of a few entries, which would leave most lanes idle) form one
// flat sequence of products: the threads take consecutive products and find each one's
// part by a binary search of the window's scan.  Either way consecutive lanes read
// consecutive entries of one B row (coalesced, distinct ascending columns).
// f(p, ok) gets DENSE_UN entry positions p[] of B and which of them are valid; every lane
// of a warp makes the same calls (so f may use warp-wide intrinsics).  Ends with a barrier.
constexpr int DENSE_CH = 256;
constexpr int DENSE_UN = 4;
constexpr int DENSE_FLAT_BELOW = 32;  // windows whose parts average fewer products go flat

template <int NT, int WIN, typename F>
SPG_DEV void dense_expand(const DevCSR &A, const DevCSR &B, const DenseArgs &D, int row, int s, int64_t *wbs,
                          int64_t *cscan, int64_t *scan64, F f) {
    const int64_t a0 = A.rp[row], a1 = A.rp[row + 1];
    const int K1 = D.K + 1;
    for (int64_t e = a0; e < a1; e += WIN) {
        const int nW = (int)min((int64_t)WIN, a1 - e);
        int64_t len = 0;
        if (threadIdx.x < nW) {
            const int32_t k = A.col[e + threadIdx.x];
            const int64_t rs = B.rp[k];
            int64_t bs, be;
            if (D.K > 1) {
                const int32_t *bk = D.bnd + (int64_t)k * K1 + s;
                bs = rs + bk[0];
                be = rs + bk[1];
            } else {
                bs = rs;
                be = B.rp[k + 1];
            }
            wbs[threadIdx.x] = bs;
            wbs[WIN + threadIdx.x] = be - bs;
            len = be - bs;
        }
        int64_t tot;
        const int64_t ex = block_exclusive_scan<NT, int64_t, false>(len, scan64, tot);
        if (threadIdx.x < nW) cscan[threadIdx.x] = ex;
        __syncthreads();
        if (tot >= (int64_t)DENSE_FLAT_BELOW * nW) {
            // long parts on average: warp w takes the w-th contiguous range of the window's
            // chunks of DENSE_CH entries, its lanes a chunk's entries 32 at a time
            constexpr int NW = NT / 32;
            const int lane = lane_id(), wid = warp_id();
            const int64_t nch = threadIdx.x < nW ? (wbs[WIN + threadIdx.x] + DENSE_CH - 1) / DENSE_CH : 0;
            int64_t tc;
            const int64_t exc = block_exclusive_scan<NT, int64_t, false>(nch, scan64, tc);
            if (threadIdx.x < nW) cscan[threadIdx.x] = exc;  // now the first chunk of each part
            __syncthreads();
            const int64_t c0 = tc * wid / NW, c1 = tc * (wid + 1) / NW;
            int t = 0;
            if (c0 < c1) t = find_segment_i64(cscan, nW, c0);
            for (int64_t c = c0; c < c1; ++c) {
                while (t + 1 < nW && cscan[t + 1] <= c) ++t;  // warp-uniform: skips parts without chunks
                const int64_t off = (c - cscan[t]) * DENSE_CH;
                const int64_t p0 = wbs[t] + off;
                const int n = (int)min((int64_t)DENSE_CH, wbs[WIN + t] - off);
                // the trip count is the same for every lane (f may be warp-collective)
                for (int i0 = 0; i0 < n; i0 += 32 * DENSE_UN) {
                    const int i = i0 + lane;
                    int64_t p[DENSE_UN];
                    bool ok[DENSE_UN];
#pragma unroll
                    for (int u = 0; u < DENSE_UN; ++u) {
                        ok[u] = i + 32 * u < n;
                        p[u] = p0 + i + 32 * u;
                    }
                    f(p, ok);
                }
            }
        } else {
            // short parts on average: one flat sequence of products; the trip count is the
            // same for every lane (f may be warp-collective)
            for (int64_t q0 = 0; q0 < tot; q0 += (int64_t)NT * DENSE_UN) {
                int64_t p[DENSE_UN];
                bool ok[DENSE_UN];
#pragma unroll
                for (int u = 0; u < DENSE_UN; ++u) {
                    const int64_t q = q0 + (int64_t)u * NT + threadIdx.x;
                    ok[u] = q < tot;
                    p[u] = 0;
                    if (ok[u]) {
                        const int t = find_segment_i64(cscan, nW, q);  // the last part starting at or before q
                        p[u] = wbs[t] + (q - cscan[t]);
                    }
                }
                f(p, ok);
            }
        }
        __syncthreads();  // the window's tables are reused
    }
}

// ---- the column bitmap of a (row, slice) ----
// Sets bit x - lo of Bm for every column x of the row's products in the slice.  The 32
// lanes of an access read consecutive entries of one B row (ascending columns), so lanes
// whose columns share a word are neighbours: an OR over each such run of lanes leaves one
// shared atomic per word touched instead of one per product.  Ends with a barrier.

SPG_DEV void bitmap_set_warp(uint32_t *Bm, int x, bool ok) {
    const int lane = lane_id();
    const int w = ok ? (x >> 5) : -1 - lane;  // invalid lanes form runs of their own
    uint32_t bits = ok ? (1u << (x & 31)) : 0u;
    // sparse columns (no two neighbours in one word): one atomic per lane, no combining
    const int prev_w = __shfl_up_sync(SPG_FULL, w, 1);  // every lane takes part in the shuffle
    const bool shared_word = lane > 0 && prev_w == w;
    if (!__any_sync(SPG_FULL, shared_word)) {
        if (ok) atomicOr(&Bm[w], bits);
        return;
    }
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t nb = __shfl_down_sync(SPG_FULL, bits, d);
        const int nw = __shfl_down_sync(SPG_FULL, w, d);
        if (lane + d < 32 && nw == w) bits |= nb;
    }
    const int pw = __shfl_up_sync(SPG_FULL, w, 1);
    if (ok && (lane == 0 || pw != w)) atomicOr(&Bm[w], bits);
}

template <int NT>
SPG_DEV bool dense_bitmap(const DevCSR &A, const DevCSR &B, const DenseArgs &D, int row, int s, int64_t lo,
                          int span, uint32_t *Bm, int64_t *wbs, int64_t *cscan, int64_t *scan64) {
    const int nq = (((span + 31) >> 5) + 3) >> 2;  // 16-byte groups of bitmap words
    uint4 *b4 = reinterpret_cast<uint4 *>(Bm);
    for (int q = threadIdx.x; q < nq; q += NT) b4[q] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    bool bad = false;
    dense_expand<NT, NT>(A, B, D, row, s, wbs, cscan, scan64, [&](const int64_t *p, const bool *ok) {
        int32_t c[DENSE_UN];
#pragma unroll
        for (int u = 0; u < DENSE_UN; ++u)
            if (ok[u]) c[u] = __ldg(B.col + p[u]);
#pragma unroll
        for (int u = 0; u < DENSE_UN; ++u) {
            const int x = ok[u] ? (int)(c[u] - lo) : 0;
            const bool in = ok[u] && (unsigned)x < (unsigned)span;
            if (ok[u] && !in) bad = true;  // cannot happen: the slice boundaries select the columns
            bitmap_set_warp(Bm, x, in);
        }
    });
    return bad;
}

// ---- pass 1: the number of columns of every (row, slice) ----
// Shared memory: the slice's column bitmap (one bit per column), then its popcount.

// The next (item, slice) of a CTA: blockIdx.x, then + gridDim.x (a grid that covers the
// items takes one each), or, with a work counter, the counter's next ticket (a persistent
// grid over a count read on the device).  All threads call it; its barrier ends the
// previous item's use of shared memory.
SPG_DEV int64_t dense_next(unsigned long long *counter, int64_t cur, bool first, int64_t *s_b) {
    __syncthreads();
    if (counter == nullptr) return first ? (int64_t)blockIdx.x : cur + gridDim.x;
    if (threadIdx.x == 0) *s_b = (int64_t)atomicAdd(counter, 1ull);
    __syncthreads();
    return *s_b;
}

// Starts moving `bytes` (a multiple of 16) at p (16-byte aligned) from memory into L2; the
// copy completes on its own, nothing waits for it.
SPG_DEV void prefetch_l2(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

SPG_DEV int64_t dense_items(const DenseArgs &D) { return (D.dev_n != nullptr ? *D.dev_n : D.n) * (int64_t)D.K; }

// The columns of slice s that row d of the dense items can reach: [lo, lo + span).
SPG_DEV int dense_span(const DevCSR &B, const DenseArgs &D, int64_t d, int s, int64_t &lo) {
    lo = max((int64_t)s * D.W, (int64_t)D.clo[d]);
    return (int)(min(min((int64_t)(s + 1) * D.W, B.ncols), (int64_t)D.chi[d]) - lo);
}

// FLAGS: narrow slices count with one flag byte per column (a plain store of 1 per product:
// every writer stores the same value, so no atomics are needed); wide ones with the bitmap.
template <int NT, bool FLAGS>
SPG_DEV void dense_count_item(const DevCSR &A, const DevCSR &B, const DenseArgs &D, int64_t b, int64_t *err) {
    extern __shared__ __align__(16) uint32_t dc_bm[];
    __shared__ int64_t wbs[2 * NT], cscan[NT], scan64[NT / 32 + 1];  // part starts, then part lengths
    __shared__ int32_t scan32[NT / 32 + 1];
    const int64_t d = b / D.K;
    const int s = (int)(b - d * D.K);
    int64_t lo;
    const int span = dense_span(B, D, d, s, lo);
    if (span <= 0) {
        if (threadIdx.x == 0) D.cnt[b] = 0;
        return;
    }
    bool bad = false;
    int n = 0;
    if constexpr (FLAGS) {
        const int nq = ((span + 31) >> 5) << 1;  // 16-byte groups of flags, whole 32-column words
        uint4 *f4 = reinterpret_cast<uint4 *>(dc_bm);
        for (int q = threadIdx.x; q < nq; q += NT) f4[q] = make_uint4(0u, 0u, 0u, 0u);
        __syncthreads();
        volatile uint8_t *fl = reinterpret_cast<uint8_t *>(dc_bm);
        dense_expand<NT, NT>(A, B, D, D.rows[d], s, wbs, cscan, scan64, [&](const int64_t *p, const bool *ok) {
            int32_t c[DENSE_UN];
#pragma unroll
            for (int u = 0; u < DENSE_UN; ++u)
                if (ok[u]) c[u] = __ldg(B.col + p[u]);
#pragma unroll
            for (int u = 0; u < DENSE_UN; ++u) {
                if (!ok[u]) continue;
                const int x = (int)(c[u] - lo);
                if ((unsigned)x >= (unsigned)span) {  // cannot happen: the slice boundaries select the columns
                    bad = true;
                    continue;
                }
                fl[x] = 1;
            }
        });
        for (int q = threadIdx.x; q < nq; q += NT) {
            const uint4 v = f4[q];
            n += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
        }
        if (D.keep != nullptr) {
            // the flags as a bitmap (32 columns per word, whole 16-byte groups), for the fill
            uint32_t *kb = D.keep + b * (int64_t)D.keep_words;
            const int nw = (span + 31) >> 5;
            for (int w = threadIdx.x; w < ((nw + 3) & ~3); w += NT) {
                uint32_t m = 0;
                if (w < nw) {
                    const uint4 lo4 = f4[2 * w], hi4 = f4[2 * w + 1];
                    const uint32_t q[8] = {lo4.x, lo4.y, lo4.z, lo4.w, hi4.x, hi4.y, hi4.z, hi4.w};
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        // byte j of q[k] (0 or 1) is column 4k + j
                        const uint32_t y = q[k];
                        m |= ((y & 1u) | ((y >> 7) & 2u) | ((y >> 14) & 4u) | ((y >> 21) & 8u)) << (4 * k);
                    }
                }
                kb[w] = m;
            }
        }
    } else {
        bad = dense_bitmap<NT>(A, B, D, D.rows[d], s, lo, span, dc_bm, wbs, cscan, scan64);
        const int nw = (span + 31) >> 5;
        for (int w = threadIdx.x; w < nw; w += NT) n += __popc(dc_bm[w]);
        if (D.keep != nullptr) {
            // the bitmap, in whole 16-byte groups (the words past the span were cleared), for the fill
            const uint4 *b4 = reinterpret_cast<const uint4 *>(dc_bm);
            uint4 *k4 = reinterpret_cast<uint4 *>(D.keep + b * (int64_t)D.keep_words);
            for (int q = threadIdx.x; q < (nw + 3) >> 2; q += NT) k4[q] = b4[q];
        }
    }
    n = block_reduce_sum<NT, int>(n, scan32);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch((unsigned long long *)err, 5ull);
    if (threadIdx.x == 0) D.cnt[b] = n;
}

template <int NT, bool FLAGS>
__global__ void __launch_bounds__(NT)
k_dense_count(DevCSR A, DevCSR B, DenseArgs D, int64_t *err) {
    __shared__ int64_t s_b;
    unsigned long long *q = D.dev_n != nullptr ? D.queue : nullptr;
    const int64_t nb = dense_items(D);
    for (int64_t b = dense_next(q, 0, true, &s_b); b < nb; b = dense_next(q, b, false, &s_b))
        dense_count_item<NT, FLAGS>(A, B, D, b, err);
}

// One thread per dense item: the slices' offsets inside the row and the row's length.
__global__ void k_dense_rows(MergeItems it, DenseArgs D) {
    const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= D.n) return;
    int32_t acc = 0;
    for (int s = 0; s < D.K; ++s) {
        D.soff[d * D.K + s] = acc;
        acc += D.cnt[d * D.K + s];
    }
    const int j = D.items[d];
    it.len[j] = acc;
    it.src_len[j] = 0;
    it.home_cap[j] = 0;
    it.home_col[j] = nullptr;
    it.home_val[j] = nullptr;
    it.child[j] = ITEM_DENSE;
}

// ---- pass 2: the values, written into C ----
// Shared memory: the slice's column bitmap Bm and its rank directory Rd (Rd[w] = set bits
// in the words before w), then a compact buffer V of vcap sums.  A product's column x has
// the position Rd[x >> 5] + popc(bits of its word below x) among the slice's columns, so
// V holds one sum per column of the result, in column order: clearing and writing out
// cost the slice's entries, not its width.  When a slice has more entries than V holds,
// its word range is cut into pieces of at most vcap entries (the rank directory gives
// the cuts) and the products are gone through once per piece.
//
// The columns of one B row are distinct, so while the whole CTA works on a single B-row
// part no two threads add into the same sum and plain adds suffice; parts of at least
// DENSE_LONG products are done that way, one after another (a barrier between two
// parts), each product one fused multiply-add.  The shorter parts are shared out to the
// warps in chunks and added with shared fp64 atomics, before the long ones.
constexpr int DENSE_FILL_WIN = 512;  // A entries per window
constexpr int DENSE_LONG = 512;

__host__ __device__ inline int dense_nw4(int W) { return ((W + 31) / 32 + 4) & ~3; }

// The product loop of a fill: every product of row `row` in slice s whose column offset x
// lies in [x0, x1) is passed to add(x, a * b) (short parts, by the warps) or add_plain
// (long parts, the whole CTA on one part).  Ends with a barrier.
template <int NT, typename Fa, typename Fp>
SPG_DEV bool dense_products(const DevCSR &A, const DevCSR &B, const DenseArgs &D, int row, int s, int64_t lo,
                            int x0, int x1, int64_t *wbs, int64_t *cscan, val_t *wa, int32_t *wlen, int32_t *lidx,
                            int64_t *scan64, Fa add, Fp add_plain) {
    constexpr int WIN = DENSE_FILL_WIN;
    bool bad = false;
    const int64_t a0 = A.rp[row], a1 = A.rp[row + 1];
    const int K1 = D.K + 1;
    for (int64_t e = a0; e < a1; e += WIN) {
        const int nW = (int)min((int64_t)WIN, a1 - e);
        // products of the short parts (low 40 bits) and the count of long parts (above)
        int64_t packed = 0;
        if (threadIdx.x < nW) {
            const int32_t k = A.col[e + threadIdx.x];
            const int64_t rs = B.rp[k];
            int64_t bs, be;
            if (D.K > 1) {
                const int32_t *bk = D.bnd + (int64_t)k * K1 + s;
                bs = rs + bk[0];
                be = rs + bk[1];
            } else {
                bs = rs;
                be = B.rp[k + 1];
            }
            const int64_t len = be - bs;
            wbs[threadIdx.x] = bs;
            wlen[threadIdx.x] = (int32_t)len;  // a B row has at most ncols < 2^31 entries
            wa[threadIdx.x] = A.val[e + threadIdx.x];
            packed = len >= DENSE_LONG ? (int64_t(1) << 40) : len;
        }
        int64_t ptot;
        const int64_t ex = block_exclusive_scan<NT, int64_t, false>(packed, scan64, ptot);
        if (threadIdx.x < nW) {
            cscan[threadIdx.x] = ex & ((int64_t(1) << 40) - 1);
            if (packed >> 40) lidx[ex >> 40] = threadIdx.x;
        }
        const int64_t tshort = ptot & ((int64_t(1) << 40) - 1);
        const int nlong = (int)(ptot >> 40);
        __syncthreads();
        const int nshort = nW - nlong;
        if (tshort >= (int64_t)DENSE_FLAT_BELOW * (nshort > 0 ? nshort : 1)) {
            // short parts averaging DENSE_FLAT_BELOW products or more: warp w takes the w-th
            // contiguous range of their chunks of DENSE_CH entries, shared atomics
            constexpr int NW = NT / 32;
            const int lane = lane_id(), wid = warp_id();
            const int64_t nch = (threadIdx.x < nW && wlen[threadIdx.x] < DENSE_LONG)
                                    ? ((int64_t)wlen[threadIdx.x] + DENSE_CH - 1) / DENSE_CH : 0;
            int64_t tc;
            const int64_t exc = block_exclusive_scan<NT, int64_t, false>(nch, scan64, tc);
            if (threadIdx.x < nW) cscan[threadIdx.x] = exc;  // now the first chunk of each part
            __syncthreads();
            const int64_t c0 = tc * wid / NW, c1 = tc * (wid + 1) / NW;
            int t = 0;
            if (c0 < c1) t = find_segment_i64(cscan, nW, c0);
            for (int64_t c = c0; c < c1; ++c) {
                while (t + 1 < nW && cscan[t + 1] <= c) ++t;  // warp-uniform: skips parts without chunks
                const int64_t off = (c - cscan[t]) * DENSE_CH;
                const int64_t p0 = wbs[t] + off;
                const int n = (int)min((int64_t)DENSE_CH, (int64_t)wlen[t] - off);
                const val_t av = wa[t];
                for (int i = lane; i < n; i += 32 * DENSE_UN) {
                    int32_t cc[DENSE_UN];
                    val_t v[DENSE_UN];
#pragma unroll
                    for (int u = 0; u < DENSE_UN; ++u)
                        if (i + 32 * u < n) cc[u] = __ldg(B.col + p0 + i + 32 * u);
#pragma unroll
                    for (int u = 0; u < DENSE_UN; ++u)
                        if (i + 32 * u < n) v[u] = __ldg(B.val + p0 + i + 32 * u);
#pragma unroll
                    for (int u = 0; u < DENSE_UN; ++u) {
                        if (i + 32 * u >= n) continue;
                        const int x = (int)(cc[u] - lo);
                        if (x < x0 || x >= x1) continue;
                        if (!add(x, av * v[u])) bad = true;
                    }
                }
            }
        } else {
            // shorter ones: one flat sequence of their products (long parts add none to the
            // scan), consecutive threads on consecutive products, shared atomics
            for (int64_t q0 = 0; q0 < tshort; q0 += (int64_t)NT * DENSE_UN) {
                int64_t pp[DENSE_UN];
                int tt[DENSE_UN];
#pragma unroll
                for (int u = 0; u < DENSE_UN; ++u) {
                    const int64_t q = q0 + (int64_t)u * NT + threadIdx.x;
                    tt[u] = -1;
                    if (q < tshort) {
                        const int t = find_segment_i64(cscan, nW, q);  // the last part starting at or before q
                        tt[u] = t;
                        pp[u] = wbs[t] + (q - cscan[t]);
                    }
                }
                int32_t cc[DENSE_UN];
                val_t v[DENSE_UN];
#pragma unroll
                for (int u = 0; u < DENSE_UN; ++u)
                    if (tt[u] >= 0) cc[u] = __ldg(B.col + pp[u]);
#pragma unroll
                for (int u = 0; u < DENSE_UN; ++u)
                    if (tt[u] >= 0) v[u] = __ldg(B.val + pp[u]);
#pragma unroll
                for (int u = 0; u < DENSE_UN; ++u) {
                    if (tt[u] < 0) continue;
                    const int x = (int)(cc[u] - lo);
                    if (x < x0 || x >= x1) continue;
                    if (!add(x, wa[tt[u]] * v[u])) bad = true;
                }
            }
        }
        __syncthreads();
        // long parts: one at a time, the whole CTA, plain adds.  A round is NT * DENSE_UN
        // consecutive entries of one part; the loads of the next two rounds are in flight
        // while a round is added (they touch no shared memory, so they may cross the
        // barrier between two parts)
        if (nlong > 0) {
            constexpr int RND = NT * DENSE_UN;
            int32_t c0[DENSE_UN], c1[DENSE_UN], c2[DENSE_UN];
            val_t v0[DENSE_UN], v1[DENSE_UN], v2[DENSE_UN];
            int j0 = 0, o0 = 0, j1, o1, j2, o2;
            auto load = [&](int32_t (&cc)[DENSE_UN], val_t (&vv)[DENSE_UN], int j, int i0) {
                if (j >= nlong) return;
                const int t = lidx[j];
                const int64_t p0 = wbs[t] + i0;
                const int n = wlen[t] - i0;
#pragma unroll
                for (int u = 0; u < DENSE_UN; ++u)
                    if ((int)threadIdx.x + NT * u < n) cc[u] = __ldg(B.col + p0 + threadIdx.x + NT * u);
#pragma unroll
                for (int u = 0; u < DENSE_UN; ++u)
                    if ((int)threadIdx.x + NT * u < n) vv[u] = __ldg(B.val + p0 + threadIdx.x + NT * u);
            };
            auto after = [&](int j, int i0, int &nj, int &ni) {
                if (j >= nlong) {
                    nj = nlong;
                    ni = 0;
                } else if (i0 + RND < wlen[lidx[j]]) {
                    nj = j;
                    ni = i0 + RND;
                } else {
                    nj = j + 1;
                    ni = 0;
                }
            };
            load(c0, v0, j0, o0);
            after(j0, o0, j1, o1);
            load(c1, v1, j1, o1);
            while (j0 < nlong) {
                after(j1, o1, j2, o2);
                load(c2, v2, j2, o2);
                {
                    const int t = lidx[j0];
                    const int n = wlen[t] - o0;
                    const val_t av = wa[t];
#pragma unroll
                    for (int u = 0; u < DENSE_UN; ++u) {
                        if ((int)threadIdx.x + NT * u >= n) continue;
                        const int x = (int)(c0[u] - lo);
                        if (x < x0 || x >= x1) continue;
                        if (!add_plain(x, av * v0[u])) bad = true;
                    }
                }
                if (j1 != j0) __syncthreads();  // the next part may add into the same columns
#pragma unroll
                for (int u = 0; u < DENSE_UN; ++u) {
                    c0[u] = c1[u];
                    v0[u] = v1[u];
                    c1[u] = c2[u];
                    v1[u] = v2[u];
                }
                j0 = j1;
                o0 = o1;
                j1 = j2;
                o1 = o2;
            }
        }
        __syncthreads();  // the window's tables are reused
    }
    return bad;
}

// REPLAY: values-only replay; C's columns are already in place, so the bitmap is built
// from the slice's known entries of C and only the values are written.
// WIDE: the single-pass form for slices narrow enough to hold one sum per column of the
// slice (W sums, W flag bytes, then the flags as a bitmap with its rank directory for the
// write-out): every product adds into its column's sum and marks its flag in one pass,
// and the write-out walks the slice's columns.  It reads the products once instead of
// twice, which pays where slices are dense (products well above their width).
template <int NT, bool REPLAY, bool WIDE>
SPG_DEV void dense_fill_item(const DevCSR &A, const DevCSR &B, const DenseArgs &D, int64_t b, const int64_t *c_rp,
                             int32_t *c_col, val_t *c_val, int64_t *err, int vcap, int cmin, int cmax) {
    constexpr int WIN = DENSE_FILL_WIN;
    extern __shared__ __align__(16) unsigned char df_smem[];
    __shared__ int64_t wbs[2 * WIN], cscan[WIN], scan64[NT / 32 + 1];  // part starts, then part lengths
    __shared__ val_t wa[WIN];
    __shared__ int32_t wlen[WIN], lidx[WIN], scan32[NT / 32 + 1];
    const int expected = D.cnt[b];
    if (expected <= cmin || expected > cmax) return;  // empty, or another launch's item
    const int64_t d = b / D.K;
    const int s = (int)(b - d * D.K);
    const int row = D.rows[d];
    // the slice's columns that the row can reach (non-empty: the slice has columns of the row)
    int64_t lo;
    const int span = dense_span(B, D, d, s, lo);
    const int nwords = (span + 31) >> 5;
    const int nw4 = dense_nw4(D.W);
    const int64_t o = c_rp[row] + D.soff[b];  // the slice's first entry in C
    bool bad = false;
    if constexpr (WIDE) {
        val_t *V = reinterpret_cast<val_t *>(df_smem);
        uint8_t *flag = reinterpret_cast<uint8_t *>(V + D.W);
        uint32_t *Bm = reinterpret_cast<uint32_t *>(flag + D.W);  // D.W is a multiple of 32
        int32_t *Rd = reinterpret_cast<int32_t *>(Bm + nw4);
        {
            // V's first span sums, in whole 16-byte groups (W sums fill a multiple of 16 bytes)
            uint4 *z4 = reinterpret_cast<uint4 *>(V);
            const int nz = (int)((span * sizeof(val_t) + 15) / 16);
            for (int q = threadIdx.x; q < nz; q += NT) z4[q] = make_uint4(0u, 0u, 0u, 0u);
            uint4 *f4 = reinterpret_cast<uint4 *>(flag);  // whole 32-column words, as read below
            if (!REPLAY)
                for (int q = threadIdx.x; q < 2 * nwords; q += NT) f4[q] = make_uint4(0u, 0u, 0u, 0u);
        }
        __syncthreads();
        volatile uint8_t *fl = flag;
        bad = dense_products<NT>(
            A, B, D, row, s, lo, 0, span, wbs, cscan, wa, wlen, lidx, scan64,
            [&](int x, val_t v) {
                atomicAdd(&V[x], v);
                if (!REPLAY) fl[x] = 1;
                return true;
            },
            [&](int x, val_t v) {
                V[x] += v;
                if (!REPLAY) fl[x] = 1;
                return true;
            });
        if (REPLAY) {
            // the slice's entries of C, in place since the product: their values
            for (int t = threadIdx.x; t < expected; t += NT) {
                const int x = (int)(c_col[o + t] - lo);
                if ((unsigned)x < (unsigned)span) c_val[o + t] = V[x];
                else bad = true;  // C's columns were changed since the product
            }
            if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch((unsigned long long *)err, 6ull);
            return;
        }
        // flags -> bitmap (32 columns per word), then its rank directory
        for (int w = threadIdx.x; w < nwords; w += NT) {
            const uint4 *f4 = reinterpret_cast<const uint4 *>(flag + 32 * w);
            const uint4 lo4 = f4[0], hi4 = f4[1];
            const uint32_t q[8] = {lo4.x, lo4.y, lo4.z, lo4.w, hi4.x, hi4.y, hi4.z, hi4.w};
            uint32_t m = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                // byte j of q[k] (0 or 1) is column 4k + j
                const uint32_t y = q[k];
                m |= ((y & 1u) | ((y >> 7) & 2u) | ((y >> 14) & 4u) | ((y >> 21) & 8u)) << (4 * k);
            }
            Bm[w] = m;
        }
        __syncthreads();
        const int tot = bitmap_rank<NT>(Bm, Rd, nwords, scan32);
        if (__syncthreads_or(bad || tot != expected)) {  // the counting pass saw other columns: cannot happen
            if (threadIdx.x == 0) atomicExch((unsigned long long *)err, 6ull);
            return;
        }
        // column order: consecutive threads take consecutive columns, so a warp's stores
        // land in one contiguous run of C
        for (int x = threadIdx.x; x < span; x += NT) {
            const uint32_t wd = Bm[x >> 5];  // the same word for the whole warp
            if (wd == 0u) continue;
            if ((wd >> (x & 31)) & 1u) {
                const int64_t pos = o + Rd[x >> 5] + __popc(wd & ((1u << (x & 31)) - 1u));
                if (!SPG_IN(pos < o + expected, 112)) continue;  // the slice's entries of C
                c_col[pos] = (int32_t)(lo + x);
                c_val[pos] = V[x];
            }
        }
        return;
    }
    uint32_t *Bm = reinterpret_cast<uint32_t *>(df_smem);
    int32_t *Rd = reinterpret_cast<int32_t *>(Bm + nw4);
    val_t *V = reinterpret_cast<val_t *>(Rd + nw4);
    // ---- the slice's columns: bitmap and rank directory ----
    if (REPLAY) {
        uint4 *b4 = reinterpret_cast<uint4 *>(Bm);
        for (int q = threadIdx.x; q < (nwords + 3) >> 2; q += NT) b4[q] = make_uint4(0u, 0u, 0u, 0u);
        __syncthreads();
        for (int t0 = 0; t0 < expected; t0 += NT) {  // whole warps: the bitmap update is warp-wide
            const int t = t0 + (int)threadIdx.x;
            const int x = t < expected ? (int)(c_col[o + t] - lo) : 0;
            const bool in = t < expected && (unsigned)x < (unsigned)span;
            if (t < expected && !in) bad = true;  // C's columns were changed since the product
            bitmap_set_warp(Bm, x, in);
        }
        __syncthreads();
    } else if (D.keep != nullptr) {
        // the bitmap the counting pass left for this (row, slice)
        const uint4 *k4 = reinterpret_cast<const uint4 *>(D.keep + b * (int64_t)D.keep_words);
        uint4 *b4 = reinterpret_cast<uint4 *>(Bm);
        for (int q = threadIdx.x; q < (nwords + 3) >> 2; q += NT) b4[q] = __ldg(k4 + q);
        __syncthreads();
    } else {
        bad = dense_bitmap<NT>(A, B, D, row, s, lo, span, Bm, wbs, cscan, scan64);
    }
    const int tot = bitmap_rank<NT>(Bm, Rd, nwords, scan32);
    if (__syncthreads_or(bad || tot != expected)) {  // the counting pass saw other columns: cannot happen
        if (threadIdx.x == 0) atomicExch((unsigned long long *)err, 6ull);
        return;
    }
    auto rank_at = [&](int w) { return w < nwords ? Rd[w] : tot; };
    // ---- pieces of at most vcap entries, each summed in V and written out ----
    for (int w0 = 0; w0 < nwords;) {
        // the last word end w1 with rank_at(w1) - Rd[w0] <= vcap (a word holds <= 32 <= vcap entries)
        const int e0 = Rd[w0];
        int w1 = nwords;  // the rest of the slice, when it fits
        if (tot - e0 > vcap) {
            int lo_ = w0 + 1, hi = nwords;
            while (lo_ < hi) {
                const int mid = (lo_ + hi + 1) >> 1;
                if (rank_at(mid) - e0 <= vcap) lo_ = mid; else hi = mid - 1;
            }
            w1 = lo_;
        }
        const int n = rank_at(w1) - e0;
        const int x0 = w0 << 5, x1 = min(span, w1 << 5);
        for (int k = threadIdx.x; k < n; k += NT) V[k] = val_t(0);
        __syncthreads();
        auto pos_of = [&](int x) {
            const uint32_t wd = Bm[x >> 5];
            return ((wd >> (x & 31)) & 1u) ? Rd[x >> 5] + __popc(wd & ((1u << (x & 31)) - 1u)) - e0 : -1;
        };
        bad = dense_products<NT>(
            A, B, D, row, s, lo, x0, x1, wbs, cscan, wa, wlen, lidx, scan64,
            [&](int x, val_t v) {
                const int q = pos_of(x);
                if (q < 0) return false;  // a column the bitmap does not hold: cannot happen
                if (SPG_IN(q < n, 109)) atomicAdd(&V[q], v);
                return true;
            },
            [&](int x, val_t v) {
                const int q = pos_of(x);
                if (q < 0) return false;
                if (SPG_IN(q < n, 109)) V[q] += v;
                return true;
            });
        if (__syncthreads_or(bad)) {
            if (threadIdx.x == 0) atomicExch((unsigned long long *)err, 6ull);
            return;
        }
        // write-out: the sums in column order (contiguous), and the columns word by word
        // (a thread takes a 16-byte group of words when the piece starts on one)
        if (SPG_IN(e0 + n <= expected, 111))
            for (int k = threadIdx.x; k < n; k += NT) c_val[o + e0 + k] = V[k];
        if (!REPLAY) {
            auto put = [&](int w, uint32_t bits, int r) {
                if (!SPG_IN(r + __popc(bits) <= expected, 110)) return;  // the slice's entries of C
                int64_t q = o + r;
                while (bits) {
                    const int t = __ffs(bits) - 1;
                    bits &= bits - 1u;
                    c_col[q++] = (int32_t)(lo + ((int64_t)w << 5) + t);
                }
            };
            if ((w0 & 3) == 0) {
                for (int g = (w0 >> 2) + (int)threadIdx.x; g < (w1 + 3) >> 2; g += NT) {
                    const int w = g << 2;
                    const uint4 bv = *reinterpret_cast<const uint4 *>(Bm + w);
                    if ((bv.x | bv.y | bv.z | bv.w) == 0u) continue;
                    const int4 rv = *reinterpret_cast<const int4 *>(Rd + w);  // entries past w1 are not used
                    put(w, bv.x, rv.x);
                    if (w + 1 < w1) put(w + 1, bv.y, rv.y);
                    if (w + 2 < w1) put(w + 2, bv.z, rv.z);
                    if (w + 3 < w1) put(w + 3, bv.w, rv.w);
                }
            } else {
                for (int w = w0 + (int)threadIdx.x; w < w1; w += NT) put(w, Bm[w], Rd[w]);
            }
        }
        __syncthreads();  // V is reused by the next piece
        w0 = w1;
    }
}

// Items whose count lies in (cmin, cmax]; with a work counter the grid is persistent.
template <int NT, int MINB, bool REPLAY, bool WIDE>
__global__ void __launch_bounds__(NT, MINB)
k_dense_fill(DevCSR A, DevCSR B, DenseArgs D, const int64_t *c_rp, int32_t *c_col, val_t *c_val, int64_t *err,
             const int64_t *gate, int vcap, unsigned long long *counter, int cmin, int cmax) {
    __shared__ int64_t s_b, s_nx;
    if (gated(gate)) return;
    const int64_t nb = dense_items(D);
    int64_t b = dense_next(counter, 0, true, &s_b);
    while (b < nb) {
        // the CTA's next item is taken one item ahead, so that its kept bitmap (written by the
        // counting pass, long out of L2) is on its way into L2 while this item is filled
        if (threadIdx.x == 0) {
            const int64_t nx = counter != nullptr ? (int64_t)atomicAdd(counter, 1ull) : b + gridDim.x;
            s_nx = nx;
            if (!REPLAY && D.keep != nullptr && nx < nb) {
                const int c = D.cnt[nx];
                if (c > cmin && c <= cmax) prefetch_l2(D.keep + nx * (int64_t)D.keep_words, 4u * (uint32_t)D.keep_words);
            }
        }
        dense_fill_item<NT, REPLAY, WIDE>(A, B, D, b, c_rp, c_col, c_val, err, vcap, cmin, cmax);
        __syncthreads();  // s_nx is visible and the item's shared memory is free
        b = s_nx;
        __syncthreads();  // every thread has read s_nx before thread 0 overwrites it
    }
}

// One thread per dense item (precise method): the slices' offsets inside the row and the
// row's size nnz(c_i), the sum of its slices' counts.
__global__ void k_dense_rowsum(DenseArgs D, int32_t *nnzc) {
    const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = D.dev_n != nullptr ? *D.dev_n : D.n;
    if (d >= n) return;
    int32_t acc = 0;
    for (int s = 0; s < D.K; ++s) {
        D.soff[d * D.K + s] = acc;
        acc += D.cnt[d * D.K + s];
    }
    nnzc[D.rows[d]] = acc;
}

constexpr int DENSE_COUNT_NT = 256;
constexpr int DENSE_COUNT_FLAGS_MAX = 32768;
constexpr int DENSE_FILL_NT = 512;
constexpr int DENSE_FILL_TWO_MIN = 4096;  // smallest sum buffer worth a second CTA per SM

// Bytes of a fill CTA's bitmap and rank directory for slices of W columns.
static int dense_index_bytes(int W) { return (int)(2 * sizeof(int32_t) * (size_t)dense_nw4(W)); }

int dense_fill_smem_bytes(int W) {
    // the index, and room for at least one word's entries in V
    return dense_index_bytes(W) + 32 * (int)sizeof(val_t);
}

// The single-pass form: one sum and one flag byte per column of the slice, and the index.
int dense_fill_wide_bytes(int W) { return (int)((sizeof(val_t) + 1) * (size_t)W) + dense_index_bytes(W); }

// Largest dynamic shared memory of a fill CTA when `per_sm` of them share an SM
// (228 KB per SM, 1 KB of it reserved per CTA, at most 227 KB per CTA).
int dense_fill_max_dynamic(int per_sm) {
    const int per_cta = std::min(227 * 1024, 228 * 1024 / per_sm - 1024);
    return per_cta - dense_fill_static_smem();
}

int dense_fill_static_smem() {
    return (int)(DENSE_FILL_WIN * (3 * sizeof(int64_t) + sizeof(val_t) + 2 * sizeof(int32_t)) +
                 (DENSE_FILL_NT / 32 + 1) * 12 + 64);
}

int dense_keep_words(int W) {
    if (dense_fill_wide_bytes(W) <= dense_fill_max_dynamic(1)) return 0;
    return dense_nw4(W);  // a multiple of 4: every item's bitmap starts on a 16-byte boundary
}

cudaError_t launch_dense_count(const DevCSR &A, const DevCSR &B, const DenseArgs &D, int64_t *err, cudaStream_t st) {
    if (D.n <= 0) return cudaSuccess;
    const int64_t nb = D.n * D.K;
    if (nb > INT32_MAX || D.W % 32 != 0 || (int64_t)D.K * D.W < B.ncols) return cudaErrorInvalidValue;
    // flag bytes for slices of up to DENSE_COUNT_FLAGS_MAX columns, else the bitmap
    const bool flags = D.W <= DENSE_COUNT_FLAGS_MAX;
    if (D.keep != nullptr && (D.keep_words < dense_nw4(D.W) || D.keep_words % 4 != 0))
        return cudaErrorInvalidValue;
    const int smem = flags ? D.W : (int)(sizeof(uint32_t) * dense_nw4(D.W));
    auto kern = flags ? k_dense_count<DENSE_COUNT_NT, true> : k_dense_count<DENSE_COUNT_NT, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int64_t grid = nb;
    if (D.dev_n != nullptr) {  // persistent grid over the items counted on the device
        if (D.queue == nullptr) return cudaErrorInvalidValue;
        e = cudaMemsetAsync(D.queue, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
        grid = persistent_blocks((const void *)kern, DENSE_COUNT_NT, smem, nb);
        if (grid <= 0) return cudaErrorInvalidValue;
    }
    kern<<<(unsigned)grid, DENSE_COUNT_NT, smem, st>>>(A, B, D, err);
    return cudaGetLastError();
}

cudaError_t launch_dense_rowsum(const DenseArgs &D, int32_t *nnzc, cudaStream_t st) {
    if (D.n <= 0) return cudaSuccess;
    k_dense_rowsum<<<(unsigned)((D.n + 127) / 128), 128, 0, st>>>(D, nnzc);
    return cudaGetLastError();
}

cudaError_t launch_dense_rows(const MergeItems &it, const DenseArgs &D, cudaStream_t st) {
    if (D.n <= 0) return cudaSuccess;
    k_dense_rows<<<(unsigned)((D.n + 127) / 128), 128, 0, st>>>(it, D);
    return cudaGetLastError();
}

cudaError_t launch_dense_fill(const DevCSR &A, const DevCSR &B, const DenseArgs &D, const int64_t *c_rp,
                              int32_t *c_col, val_t *c_val, int64_t *err, cudaStream_t st, bool replay,
                              const int64_t *gate) {
    if (D.n <= 0) return cudaSuccess;
    const int64_t nb = D.n * D.K;
    if (nb > INT32_MAX || D.W % 32 != 0 || (int64_t)D.K * D.W < B.ncols) return cudaErrorInvalidValue;
    if (D.keep != nullptr && (D.keep_words < dense_nw4(D.W) || D.keep_words % 4 != 0)) return cudaErrorInvalidValue;
    // one launch: a grid over the items, or a persistent grid taking them from counter q
    auto go = [&](auto kern, int smem, int vcap, unsigned long long *q, int cmin, int cmax) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        int64_t grid = nb;
        if (q != nullptr) {
            e = cudaMemsetAsync(q, 0, sizeof(unsigned long long), st);
            if (e != cudaSuccess) return e;
            grid = persistent_blocks((const void *)kern, DENSE_FILL_NT, smem, nb);
            if (grid <= 0) return cudaErrorInvalidValue;
        }
        kern<<<(unsigned)grid, DENSE_FILL_NT, smem, st>>>(A, B, D, c_rp, c_col, c_val, err, gate, vcap, q, cmin,
                                                           cmax);
        return cudaGetLastError();
    };
    if (D.dev_n != nullptr && D.queue == nullptr) return cudaErrorInvalidValue;
    const int index = dense_index_bytes(D.W);
    if (dense_fill_wide_bytes(D.W) <= dense_fill_max_dynamic(1)) {
        // single-pass form (two CTAs per SM when two slices fit an SM's shared memory)
        const int smem = dense_fill_wide_bytes(D.W);
        const int vcap = (smem - index) / (int)sizeof(val_t);
        unsigned long long *q = D.dev_n != nullptr ? D.queue + 1 : nullptr;
        if (smem <= dense_fill_max_dynamic(2))
            return replay ? go(k_dense_fill<DENSE_FILL_NT, 2, true, true>, smem, vcap, q, 0, INT32_MAX)
                          : go(k_dense_fill<DENSE_FILL_NT, 2, false, true>, smem, vcap, q, 0, INT32_MAX);
        return replay ? go(k_dense_fill<DENSE_FILL_NT, 1, true, true>, smem, vcap, q, 0, INT32_MAX)
                      : go(k_dense_fill<DENSE_FILL_NT, 1, false, true>, smem, vcap, q, 0, INT32_MAX);
    }
    // compact form: the index, then as many sums as the rest of the CTA's shared memory holds.
    // With work counters, the items whose slices have at most vcap2 entries run at two CTAs per
    // SM (half the shared memory each), the others at one
    const int smem1 = dense_fill_max_dynamic(1) & ~15, smem2 = dense_fill_max_dynamic(2) & ~15;
    const int vcap1 = (smem1 - index) / (int)sizeof(val_t), vcap2 = (smem2 - index) / (int)sizeof(val_t);
    if (vcap1 < 32) return cudaErrorInvalidValue;
    if (D.queue != nullptr && vcap2 >= DENSE_FILL_TWO_MIN) {
        cudaError_t e = replay ? go(k_dense_fill<DENSE_FILL_NT, 2, true, false>, smem2, vcap2, D.queue + 1, 0, vcap2)
                               : go(k_dense_fill<DENSE_FILL_NT, 2, false, false>, smem2, vcap2, D.queue + 1, 0, vcap2);
        if (e != cudaSuccess) return e;
        return replay ? go(k_dense_fill<DENSE_FILL_NT, 1, true, false>, smem1, vcap1, D.queue + 2, vcap2, INT32_MAX)
                      : go(k_dense_fill<DENSE_FILL_NT, 1, false, false>, smem1, vcap1, D.queue + 2, vcap2, INT32_MAX);
    }
    unsigned long long *q = D.dev_n != nullptr ? D.queue + 1 : nullptr;
    return replay ? go(k_dense_fill<DENSE_FILL_NT, 1, true, false>, smem1, vcap1, q, 0, INT32_MAX)
                  : go(k_dense_fill<DENSE_FILL_NT, 1, false, false>, smem1, vcap1, q, 0, INT32_MAX);
}

}  // namespace spg
