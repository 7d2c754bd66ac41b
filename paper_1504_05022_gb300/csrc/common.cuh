// Device helpers shared by the SpGEMM kernels: warp/block scans, merge-path
// partitioning and the in-place merges used by the bin-37 merge kernel.
#pragma once

#include <cstdint>
#include <climits>
#include <cuda_runtime.h>

#include "internal.h"

#define SPG_DEV __device__ __forceinline__
#define SPG_FULL 0xffffffffu

namespace spg {

// Sentinel key used to pad sorting networks; real column indices are < ncols <= INT_MAX.
constexpr int32_t KEY_PAD = INT_MAX;

SPG_DEV int lane_id() { return threadIdx.x & 31; }

// ---- the bounds-checked build ----
// Built with SPGEMM_CHECK, SPG_IN(cond, code) records `code` in this translation unit's
// status word when cond is false (the first code recorded stays) and yields false, so that
// the caller skips the access; the kernel carries on (no trap) and the host reads the words
// with spgemm_check_status.  Without SPGEMM_CHECK it is `true` and costs nothing.
#ifdef SPGEMM_CHECK
static __device__ unsigned long long spg_check_word;
SPG_DEV bool spg_in(bool ok, int code) {
    if (!ok) atomicCAS(&spg_check_word, 0ull, (unsigned long long)code);
    return ok;
}
#define SPG_IN(cond, code) (::spg::spg_in((cond), (code)))
static cudaError_t spg_read_check_word(unsigned long long *out, bool reset) {
    cudaError_t e = cudaMemcpyFromSymbol(out, spg_check_word, sizeof(*out));
    if (e == cudaSuccess && reset) {
        const unsigned long long zero = 0;
        e = cudaMemcpyToSymbol(spg_check_word, &zero, sizeof(zero));
    }
    return e;
}
static const int spg_check_registered = register_check_reader(spg_read_check_word);
#else
#define SPG_IN(cond, code) (true)
#endif

// The rows of a RowSet: host-known, or a range of `rows` whose ends are read here.
SPG_DEV void rowset_range(const RowSet &R, const int32_t *&rows, int64_t &n) {
    if (R.dev_lo != nullptr) {
        const int64_t lo = *R.dev_lo;
        rows = R.rows + lo;
        n = *R.dev_hi - lo;
    } else {
        rows = R.rows;
        n = R.n;
    }
}

// Walks of a row's split tree in column order (left child first), without a stack, so a
// tree of any depth is walked: the first leaf under x, and the leaf after x under root
// (-1 after the last).  Leaves are the items with child < 0.
SPG_DEV int split_first_leaf(const MergeItems &it, int x) {
    while (it.child[x] >= 0) x = it.child[x];
    return x;
}
SPG_DEV int split_next_leaf(const MergeItems &it, int root, int x) {
    while (x != root) {
        const int p = it.parent[x];
        if (x == it.child[p]) return split_first_leaf(it, x + 1);  // a left child: its right sibling
        x = p;
    }
    return -1;
}

// True when a gate word is set: the launch must write nothing.
SPG_DEV bool gated(const int64_t *gate) { return gate != nullptr && *gate != 0; }
SPG_DEV int warp_id() { return threadIdx.x >> 5; }

template <typename T>
SPG_DEV T warp_inclusive_scan(T v) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T n = __shfl_up_sync(SPG_FULL, v, d);
        if (lane_id() >= d) v += n;
    }
    return v;
}

template <typename T>
SPG_DEV T warp_reduce_sum(T v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(SPG_FULL, v, d);
    return v;
}

// Block-wide exclusive scan.  `scratch` needs NT/32 + 1 elements of T.  Every
// thread of the block must call it.  Returns the exclusive prefix; `total`
// receives the block sum.  With TRAILING_SYNC it ends with a barrier so scratch
// can be reused at once; without it the caller must pass a barrier before the
// next scan that uses the same scratch.
template <int NT, typename T, bool TRAILING_SYNC = true>
SPG_DEV T block_exclusive_scan(T v, T *scratch, T &total) {
    constexpr int NW = NT / 32;
    const int lane = lane_id(), wid = warp_id();
    T inc = warp_inclusive_scan(v);
    if (lane == 31) scratch[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        T w = (lane < NW) ? scratch[lane] : T(0);
        T winc = warp_inclusive_scan(w);
        if (lane < NW) scratch[lane] = winc - w;
        if (lane == NW - 1) scratch[NW] = winc;
    }
    __syncthreads();
    T res = scratch[wid] + inc - v;
    total = scratch[NW];
    if (TRAILING_SYNC) __syncthreads();
    return res;
}

template <int NT, typename T>
SPG_DEV T block_reduce_sum(T v, T *scratch) {
    constexpr int NW = NT / 32;
    v = warp_reduce_sum(v);
    if (lane_id() == 0) scratch[warp_id()] = v;
    __syncthreads();
    T s = T(0);
    if (threadIdx.x == 0) {
        for (int w = 0; w < NW; ++w) s += scratch[w];
        scratch[NW] = s;
    }
    __syncthreads();
    s = scratch[NW];
    __syncthreads();
    return s;
}

// Number of elements of the sorted array a[0..n) that are < key.
SPG_DEV int lower_bound_i32(const int32_t *a, int n, int32_t key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Number of elements of the sorted array a[0..n) that are <= key.
SPG_DEV int upper_bound_i32(const int32_t *a, int n, int32_t key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] <= key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Largest t in [0, n) with s[t] <= x, for a non-decreasing s with s[0] <= x.
SPG_DEV int find_segment_i64(const int64_t *s, int n, int64_t x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (s[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

SPG_DEV int find_segment_i32(const int32_t *s, int n, int32_t x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (s[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Merge path (Green, McColl & Bader): for the stable merge of a[0..na) and
// b[0..nb) in which a's element goes first on equal keys, returns how many of
// the first `diag` outputs come from a.
SPG_DEV int merge_path(const int32_t *a, int na, const int32_t *b, int nb, int diag) {
    int lo = diag > nb ? diag - nb : 0;
    int hi = diag < na ? diag : na;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] <= b[diag - 1 - mid]) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Lockstep lower_bound of up to IPT keys in the sorted array a[0..n): pos[k]
// receives the number of entries < key[k].  The IPT searches are independent,
// so their shared-memory loads overlap.
template <int IPT>
SPG_DEV void lower_bound_multi(const int32_t *a, int n, const int32_t (&key)[IPT], int cnt, int (&pos)[IPT]) {
    int hi[IPT];
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
        pos[k] = 0;
        hi[k] = (k < cnt) ? n : 0;
    }
    for (int step = 32 - __clz(n); step > 0; --step) {
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            if (pos[k] < hi[k]) {
                const int mid = (pos[k] + hi[k]) >> 1;
                if (a[mid] < key[k]) pos[k] = mid + 1; else hi[k] = mid;
            }
        }
    }
}

// Rank directory of a bitmap: Rd[w] = number of set bits in Bm[0..w) for w <
// nwords; returns the total.  Each thread takes a run of consecutive words, a whole
// number of 16-byte groups (Bm and Rd 16-byte aligned), read and written as vectors
// (the last, partial group of the bitmap word by word).  scan32 needs NT/32 + 1 ints
// and must not be reused before the next barrier after this call.  All threads
// call; ends with a barrier.
template <int NT>
SPG_DEV int bitmap_rank(const uint32_t *Bm, int32_t *Rd, int nwords, int32_t *scan32) {
    const int per = ((nwords + NT - 1) / NT + 3) & ~3;
    const int w0 = threadIdx.x * per;
    const int w1 = min(nwords, w0 + per);
    int sum = 0;
    for (int w = w0; w < w1; w += 4) {
        if (w + 4 <= w1) {
            const uint4 b = *reinterpret_cast<const uint4 *>(Bm + w);
            sum += __popc(b.x) + __popc(b.y) + __popc(b.z) + __popc(b.w);
        } else {
            for (int k = w; k < w1; ++k) sum += __popc(Bm[k]);
        }
    }
    int tot;
    int ex = block_exclusive_scan<NT, int, false>(sum, scan32, tot);
    for (int w = w0; w < w1; w += 4) {
        if (w + 4 <= w1) {
            const uint4 b = *reinterpret_cast<const uint4 *>(Bm + w);
            const int c0 = __popc(b.x), c1 = __popc(b.y), c2 = __popc(b.z);
            *reinterpret_cast<int4 *>(Rd + w) = make_int4(ex, ex + c0, ex + c0 + c1, ex + c0 + c1 + c2);
            ex += c0 + c1 + c2 + __popc(b.w);
        } else {
            for (int k = w; k < w1; ++k) {
                Rd[k] = ex;
                ex += __popc(Bm[k]);
            }
        }
    }
    __syncthreads();
    return tot;
}

// Rank of bit x (set) of a bitmap with rank directory Rd.
SPG_DEV int bitmap_pos(const uint32_t *Bm, const int32_t *Rd, int x) {
    return Rd[x >> 5] + __popc(Bm[x >> 5] & ((1u << (x & 31)) - 1u));
}

// In-place merge of two disjoint sorted sequences: x (keys xk, values xv,
// length nx) lives at the front of an array with room for nx + ny entries; y
// (yk, yv, length ny) lives elsewhere.  Afterwards xk/xv[0 .. nx+ny) hold the
// merged sequence.  The output is produced in chunks of NT*IPT entries from the
// right end: an x entry only moves right, so a chunk never overwrites an x entry
// that a chunk to its left still has to read.  Every thread of the block must
// call it; it ends with a barrier.
template <int NT, int IPT>
SPG_DEV void merge_inplace_rtl(int32_t *xk, val_t *xv, int nx, const int32_t *yk, const val_t *yv,
                               int ny) {
    if (ny == 0) return;
    const int n = nx + ny;
    constexpr int CH = NT * IPT;
    for (int hi = n; hi > 0; hi -= CH) {
        const int lo = hi > CH ? hi - CH : 0;
        int32_t rk[IPT];
        val_t rv[IPT];
        const int d0 = lo + threadIdx.x * IPT;
        int cnt = 0;
        if (d0 < hi) {
            int i = merge_path(xk, nx, yk, ny, d0);
            int j = d0 - i;
            cnt = min(IPT, hi - d0);
#pragma unroll
            for (int t = 0; t < IPT; ++t) {
                if (t < cnt) {
                    bool takex = (i < nx) && (j >= ny || xk[i] <= yk[j]);
                    if (takex) { rk[t] = xk[i]; rv[t] = xv[i]; ++i; }
                    else { rk[t] = yk[j]; rv[t] = yv[j]; ++j; }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < IPT; ++t) {
            if (t < cnt) { xk[d0 + t] = rk[t]; xv[d0 + t] = rv[t]; }
        }
        __syncthreads();
    }
}

// Out-of-place stable merge of a and b into out (na + nb entries).  All threads call.
template <int NT>
SPG_DEV void merge_into(const int32_t *ak, const val_t *av, int na, const int32_t *bk,
                        const val_t *bv, int nb, int32_t *ok, val_t *ov) {
    const int n = na + nb;
    const int ipt = (n + NT - 1) / NT;
    const int d0 = threadIdx.x * ipt;
    if (d0 < n) {
        const int d1 = min(n, d0 + ipt);
        int i = merge_path(ak, na, bk, nb, d0);
        int j = d0 - i;
        for (int d = d0; d < d1; ++d) {
            bool takea = (i < na) && (j >= nb || ak[i] <= bk[j]);
            if (takea) { ok[d] = ak[i]; ov[d] = av[i]; ++i; }
            else { ok[d] = bk[j]; ov[d] = bv[j]; ++j; }
        }
    }
    __syncthreads();
}

}  // namespace spg
