// Stage 3, bin group 5 (u_i > 512): the merge method of Section 4.1 with the
// result's membership kept as a bitmap over the item's column range.
//
// One CTA per work item (a row, or a column slice of a row).  The result
// sequence R (sorted, duplicate-free keys Rk with values Rv) lives in shared
// memory, and next to it a bitmap Bm of the columns R holds plus a rank
// directory Rd (Rd[w] = number of R entries in the words before w).  The
// paper's sub-steps of the parallel insert become:
//   (1) fuse: a product whose column is in R finds its position as
//       Rd[w] + popc(Bm[w] below its bit) -- two shared loads instead of a
//       binary search -- and is added with a shared atomicAdd;
//   (2)-(3) products whose column is not in R are appended, unsorted, to a
//       miss buffer (warp-aggregated slots, no block barrier);
//   (4) when the miss buffer is full, the misses are merged into R by rank:
//       their bits are set, Rd is rebuilt by one block scan, every old entry
//       moves (right to left, in chunks) to its rank in the union, and every
//       new column takes its rank; duplicate misses add into the same entry.
// A batch of products therefore costs one block barrier, and the merge work
// is paid once per miss buffer instead of once per batch.  Capacity, the
// checkpoint at overflow and the progressive relaunch are those of k_merge:
// a batch never exceeds the free capacity, so a merge can always complete.
// Used when the columns of B fit the bitmap (ncols <= BM_MAX_COLS) and long
// rows are split; level-1 launches use k_merge.
#include "internal.h"
#include "common.cuh"

#include <algorithm>

namespace spg {

constexpr int BM_IPT = 4;          // products per thread per batch: batch <= NT * 4

struct BmSmem {
    double *Rv, *Mv, *wa;
    int64_t *wbs, *wscan;
    int32_t *Rk, *Mk, *Rd;
    uint32_t *Bm;
};

// Shared-memory layout: R (cap), the miss buffer (miss), the window of W A
// entries, the bitmap and its rank directory (nwords + 1).
__host__ __device__ inline size_t bm_layout(int cap, int nwords, int miss, int W, unsigned char *base, BmSmem *s) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = (off + bytes + 15) & ~size_t(15);
        return base ? base + o : nullptr;
    };
    unsigned char *p;
    p = take(sizeof(double) * cap);            if (s) s->Rv = (double *)p;
    p = take(sizeof(double) * miss);           if (s) s->Mv = (double *)p;
    p = take(sizeof(double) * W);              if (s) s->wa = (double *)p;
    p = take(sizeof(int64_t) * W);             if (s) s->wbs = (int64_t *)p;
    p = take(sizeof(int64_t) * (W + 1));       if (s) s->wscan = (int64_t *)p;
    p = take(sizeof(int32_t) * cap);           if (s) s->Rk = (int32_t *)p;
    p = take(sizeof(int32_t) * miss);          if (s) s->Mk = (int32_t *)p;
    p = take(sizeof(int32_t) * (nwords + 1));  if (s) s->Rd = (int32_t *)p;
    p = take(sizeof(uint32_t) * nwords);       if (s) s->Bm = (uint32_t *)p;
    return off;
}

// Position of column c (already in the bitmap) in R.
SPG_DEV int bm_pos(const BmSmem &s, int32_t c, int32_t lo) { return bitmap_pos(s.Bm, s.Rd, c - lo); }

// Rebuilds the rank directory of words [0, nwords); returns the number of set
// bits.  All threads call; ends with a barrier.
template <int NT>
SPG_DEV int bm_rank(const BmSmem &s, int nwords, int32_t *scan32) {
    return bitmap_rank<NT>(s.Bm, s.Rd, nwords, scan32);
}

// Merges the nm buffered misses into R (length rlen) by rank; returns the new
// length.  All threads call, after a barrier that made the buffer visible; ends
// with a barrier.
template <int NT>
SPG_DEV int bm_merge_misses(const BmSmem &s, int rlen, int nm, int32_t lo, int nwords, int32_t *scan32,
                            int32_t *nmiss_shared) {
    for (int m = threadIdx.x; m < nm; m += NT) {
        const int x = s.Mk[m] - lo;
        atomicOr(&s.Bm[x >> 5], 1u << (x & 31));
    }
    __syncthreads();
    // every thread has read the buffer count before this barrier: the counter can restart
    if (threadIdx.x == 0) *nmiss_shared = 0;
    const int fnew = bm_rank<NT>(s, nwords, scan32);
    // old entries move right (to their rank in the union), a chunk at a time from
    // the right end.  A chunk's targets lie at or beyond its own old positions, so
    // they never overwrite an entry that a chunk to its left still has to read;
    // only the chunk's own reads must finish before its writes (one barrier).
    constexpr int CH = NT * 4;
    for (int hi = rlen; hi > 0; hi -= CH) {
        const int base = hi > CH ? hi - CH : 0;
        int32_t kk[4];
        double vv[4];
        int np[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {  // entry base + q*NT + thread: consecutive lanes, consecutive words
            const int p = base + q * NT + threadIdx.x;
            np[q] = -1;
            if (p < hi) {
                kk[q] = s.Rk[p];
                vv[q] = s.Rv[p];
                const int t = bm_pos(s, kk[q], lo);
                if (t != p) np[q] = t;
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (np[q] >= 0) {
                s.Rk[np[q]] = kk[q];
                s.Rv[np[q]] = vv[q];
            }
        }
    }
    __syncthreads();
    // new columns: key and a zero value (duplicate misses write the same), then the sums
    for (int m = threadIdx.x; m < nm; m += NT) {
        const int32_t c = s.Mk[m];
        const int t = bm_pos(s, c, lo);
        s.Rk[t] = c;
        s.Rv[t] = 0.0;
    }
    __syncthreads();
    for (int m = threadIdx.x; m < nm; m += NT) atomicAdd(&s.Rv[bm_pos(s, s.Mk[m], lo)], s.Mv[m]);
    __syncthreads();
    return fnew;
}

template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
k_merge_bm(StageArgs a, MergeItems it, MergeLaunch L) {
    extern __shared__ __align__(16) unsigned char bm_smem[];
    __shared__ int64_t scan64[NT / 32 + 1];
    __shared__ int32_t scan32[NT / 32 + 1];
    __shared__ int32_t s_nmiss;
    constexpr int W = NT;
    BmSmem s;
    const int kb = L.batch;
    const int mcap = L.bm_miss;
    bm_layout(L.cap, L.bm_words, mcap, W, bm_smem, &s);

    const int64_t w = blockIdx.x;
    const int j = L.work ? L.work[w] : (int)(L.work_base + w);
    const int row = it.row[j];
    const int32_t clo = it.clo[j], chi = it.chi[j];
    const bool filtered = (clo > 0) || (chi < INT32_MAX);
    const int32_t lo = clo > 0 ? clo : 0;  // bitmap origin
    const int64_t hicol = min((int64_t)chi, a.B.ncols);
    const int nwords = hicol > lo ? (int)((hicol - lo + 31) >> 5) : 1;
    const int64_t a0 = a.A.rp[row], a1 = a.A.rp[row + 1];
    int rlen = it.src_len[j];
    int64_t e = a0 + it.ck_entry[j];
    int64_t off = it.ck_off[j];

    // where this launch writes the item: its home if large enough, else a fresh
    // slot; without a pool the item's capacity is that of its home
    int32_t *dst_col = it.home_col[j];
    double *dst_val = it.home_val[j];
    int64_t dst_cap = it.home_cap[j];
    int cap = L.cap;
    if (dst_cap < cap) {
        if (L.pool_col != nullptr) {
            dst_col = L.pool_col + w * L.pool_cap;
            dst_val = L.pool_val + w * L.pool_cap;
            dst_cap = L.pool_cap;
        } else {
            cap = (int)dst_cap;
        }
    }
    if (nwords > L.bm_words || rlen > cap) {  // cannot happen: slices fit the bitmap; relaunches fit R
        if (threadIdx.x == 0) atomicExch((unsigned long long *)L.err, 1ull);
        return;
    }
    // reload the item's sequence (empty for a fresh row; half of the parent's for a split child)
    for (int t = threadIdx.x; t < nwords; t += NT) s.Bm[t] = 0u;
    if (threadIdx.x == 0) s_nmiss = 0;
    __syncthreads();
    {
        const int32_t *sc = it.src_col[j];
        const double *sv = it.src_val[j];
        for (int t = threadIdx.x; t < rlen; t += NT) {
            const int32_t c = sc[t];
            s.Rk[t] = c;
            s.Rv[t] = sv[t];
            const int x = c - lo;
            if ((unsigned)x < (unsigned)(nwords << 5)) atomicOr(&s.Bm[x >> 5], 1u << (x & 31));
            else atomicExch((unsigned long long *)L.err, 5ull);  // cannot happen: slices hold their own columns
        }
    }
    __syncthreads();
    bm_rank<NT>(s, nwords, scan32);
    int nmiss = 0;

    bool overflow = false;
    while (e < a1 && !overflow) {
        __syncthreads();  // the previous window's entries are no longer read
        // ---- window: the next W entries of the A row and their (column-filtered) B-row ranges ----
        const int nW = (int)min((int64_t)W, a1 - e);
        int64_t len = 0;
        if (threadIdx.x < nW) {
            const int64_t idx = e + threadIdx.x;
            const int32_t kk = a.A.col[idx];
            const int64_t rs = a.B.rp[kk];
            int64_t be = a.B.rp[kk + 1];
            int64_t bs = rs + (threadIdx.x == 0 ? off : 0);
            if (filtered) {
                const int n = (int)(be - rs);
                if (clo > 0) {
                    const int64_t lb = rs + lower_bound_i32(a.B.col + rs, n, clo);
                    bs = bs > lb ? bs : lb;
                }
                if (chi < INT32_MAX) be = rs + lower_bound_i32(a.B.col + rs, n, chi);
            }
            s.wbs[threadIdx.x] = bs;
            s.wa[threadIdx.x] = a.A.val[idx];
            len = be > bs ? be - bs : 0;
        }
        int64_t total;
        const int64_t ex = block_exclusive_scan<NT, int64_t, false>(len, scan64, total);
        if (threadIdx.x < nW) s.wscan[threadIdx.x] = ex;
        if (threadIdx.x == 0) s.wscan[nW] = total;
        __syncthreads();

        int64_t p0 = 0;
        while (p0 < total) {
            const int need = (int)min((int64_t)kb, total - p0);
            if (nmiss + need > mcap) {  // room in the miss buffer first
                rlen = bm_merge_misses<NT>(s, rlen, nmiss, lo, nwords, scan32, &s_nmiss);
                nmiss = 0;
            }
            int avail = cap - rlen - nmiss;
            const int tf = find_segment_i64(s.wscan, nW, p0);
            const int tl = find_segment_i64(s.wscan, nW, p0 + need - 1);
            const int nruns = tl - tf + 1;
            // (0) each thread expands products threadIdx.x + k*NT of the batch into
            // registers: consecutive lanes read consecutive B entries (coalesced)
            int cnt = need > (int)threadIdx.x ? min(BM_IPT, (need - (int)threadIdx.x + NT - 1) / NT) : 0;
            int32_t key[BM_IPT];
            double val[BM_IPT];
            {
                int te[BM_IPT], to[BM_IPT];
#pragma unroll
                for (int k = 0; k < BM_IPT; ++k) {
                    if (k < cnt) {
                        const int64_t pos = p0 + threadIdx.x + k * NT;
                        const int t = tf + find_segment_i64(s.wscan + tf, nruns, pos);
                        te[k] = t;
                        to[k] = (int)(pos - s.wscan[t]);
                    }
                }
#pragma unroll
                for (int k = 0; k < BM_IPT; ++k)
                    if (k < cnt) key[k] = __ldg(a.B.col + s.wbs[te[k]] + to[k]);
#pragma unroll
                for (int k = 0; k < BM_IPT; ++k)
                    if (k < cnt) val[k] = __ldg(a.B.val + s.wbs[te[k]] + to[k]);
#pragma unroll
                for (int k = 0; k < BM_IPT; ++k)
                    if (k < cnt) val[k] *= s.wa[te[k]];
            }
            // (1) which products' columns are in R (position from the rank directory)
            int rpos[BM_IPT];
            unsigned miss = 0;
#pragma unroll
            for (int k = 0; k < BM_IPT; ++k) {
                rpos[k] = -1;
                if (k < cnt) {
                    const int x = key[k] - lo;
                    if ((unsigned)x >= (unsigned)(nwords << 5)) {  // a column outside [0, ncols): bad input
                        atomicExch((unsigned long long *)L.err, 5ull);
                        continue;
                    }
                    const uint32_t wd = s.Bm[x >> 5];
                    if ((wd >> (x & 31)) & 1u) rpos[k] = s.Rd[x >> 5] + __popc(wd & ((1u << (x & 31)) - 1u));
                    else miss |= 1u << k;
                }
            }
            int nb = need;
            if (avail < need) {
                // the batch fits if its actual misses fit the free capacity (its hits take none)
                int cm = block_reduce_sum<NT, int>(__popc(miss), scan32);
                if (cm > avail && nmiss > 0) {
                    rlen = bm_merge_misses<NT>(s, rlen, nmiss, lo, nwords, scan32, &s_nmiss);
                    nmiss = 0;
                    avail = cap - rlen;
                    miss = 0;  // the bitmap changed: look the products up again
#pragma unroll
                    for (int k = 0; k < BM_IPT; ++k) {
                        rpos[k] = -1;
                        if (k < cnt) {
                            const int x = key[k] - lo;
                            if ((unsigned)x >= (unsigned)(nwords << 5)) continue;
                            const uint32_t wd = s.Bm[x >> 5];
                            if ((wd >> (x & 31)) & 1u) rpos[k] = s.Rd[x >> 5] + __popc(wd & ((1u << (x & 31)) - 1u));
                            else miss |= 1u << k;
                        }
                    }
                    cm = block_reduce_sum<NT, int>(__popc(miss), scan32);
                }
                if (cm > avail) {
                    if (avail < (kb >> 2) || avail <= 0) {
                        // checkpoint at product p0 of this window (offset counted in the full B row)
                        const int t = find_segment_i64(s.wscan, nW, p0);
                        if (threadIdx.x == 0) {
                            const int32_t kk = a.A.col[e + t];
                            it.ck_entry[j] = (e + t) - a0;
                            it.ck_off[j] = s.wbs[t] + (p0 - s.wscan[t]) - a.B.rp[kk];
                        }
                        overflow = true;
                        break;
                    }
                    // only the first `avail` products: each adds at most one new column
                    nb = avail;
                    cnt = nb > (int)threadIdx.x ? min(BM_IPT, (nb - (int)threadIdx.x + NT - 1) / NT) : 0;
#pragma unroll
                    for (int k = 0; k < BM_IPT; ++k)
                        if (k >= cnt) rpos[k] = -1;
                    miss &= (1u << cnt) - 1u;
                }
            }
            // fuse the hits
#pragma unroll
            for (int k = 0; k < BM_IPT; ++k)
                if (rpos[k] >= 0) atomicAdd(&s.Rv[rpos[k]], val[k]);
            // (2)-(3) append the misses to the buffer: one shared atomic per warp
            {
                const int nm = __popc(miss);
                const int inc = warp_inclusive_scan(nm);
                const int wtot = __shfl_sync(SPG_FULL, inc, 31);
                int slot = 0;
                if (lane_id() == 31 && wtot > 0) slot = atomicAdd(&s_nmiss, wtot);
                slot = __shfl_sync(SPG_FULL, slot, 31) + inc - nm;
#pragma unroll
                for (int k = 0; k < BM_IPT; ++k) {
                    if ((miss >> k) & 1u) {
                        s.Mk[slot] = key[k];
                        s.Mv[slot] = val[k];
                        ++slot;
                    }
                }
            }
            __syncthreads();
            nmiss = s_nmiss;
            p0 += nb;
        }
        if (!overflow) {
            e += nW;
            off = 0;
        }
    }
    // (4) the last buffered misses
    if (nmiss > 0) {
        rlen = bm_merge_misses<NT>(s, rlen, nmiss, lo, nwords, scan32, &s_nmiss);
        nmiss = 0;
    }
    if (rlen > dst_cap) {  // cannot happen: dst_cap >= cap >= rlen
        if (threadIdx.x == 0) atomicExch((unsigned long long *)L.err, 1ull);
        return;
    }
    for (int t = threadIdx.x; t < rlen; t += NT) {
        dst_col[t] = s.Rk[t];
        dst_val[t] = s.Rv[t];
    }
    if (threadIdx.x == 0) {
        it.home_col[j] = dst_col;
        it.home_val[j] = dst_val;
        it.home_cap[j] = dst_cap;
        if (overflow) {
            it.src_col[j] = dst_col;
            it.src_val[j] = dst_val;
            it.src_len[j] = (int32_t)rlen;
            const int slot = atomicAdd(L.ovf_count, 1);
            L.ovf_list[slot] = j;
        } else {
            it.len[j] = (int32_t)rlen;
        }
    }
}

// Threads per CTA (same rule as k_merge).
static int bm_threads(int cap, int wide_above) {
    if (wide_above <= 0) wide_above = 2048;
    return cap <= 512 ? 128 : (cap <= wide_above ? 256 : 512);
}

int merge_bm_smem_bytes(int cap, int nwords, int miss, int wide_above) {
    return (int)bm_layout(cap, nwords, miss, bm_threads(cap, wide_above), nullptr, nullptr);
}

int merge_bm_max_cap(int nwords, int miss, int smem_limit, int wide_above) {
    int cap = 256;
    while (merge_bm_smem_bytes(cap + 256, nwords, miss, wide_above) <= smem_limit) cap += 256;
    return cap;
}

template <int NT, int MINB>
static cudaError_t launch_bm_nt(const StageArgs &a, const MergeItems &s, const MergeLaunch &L, int smem,
                                cudaStream_t st) {
    auto kern = k_merge_bm<NT, MINB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)L.nwork, NT, smem, st>>>(a, s, L);
    return cudaGetLastError();
}

cudaError_t launch_merge_bm(const StageArgs &a, const MergeItems &s, const MergeLaunch &L, cudaStream_t st) {
    if (L.nwork <= 0) return cudaSuccess;
    const int nt = bm_threads(L.cap, L.wide_above);
    // every batch fits the miss buffer and the free capacity; batch >= 32 keeps the loops progressing
    if (L.level1 || L.bm_words <= 0 || L.batch > nt * BM_IPT || L.batch < 32 ||
        L.bm_miss < L.batch || (!L.bm_sliced && (int64_t)L.bm_words * 32 < a.B.ncols))
        return cudaErrorInvalidValue;
    const int smem = merge_bm_smem_bytes(L.cap, L.bm_words, L.bm_miss, L.wide_above);
    if (nt == 128) return launch_bm_nt<128, 4>(a, s, L, smem, st);
    if (nt == 256) return launch_bm_nt<256, 2>(a, s, L, smem, st);
    return launch_bm_nt<512, 1>(a, s, L, smem, st);
}

}  // namespace spg
