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
// is paid once per miss buffer instead of once per batch.  A batch is admitted
// when its actual new columns fit the free capacity (its hits take none), so a
// merge can always complete.  The checkpoint at overflow and the progressive
// relaunch are those of k_merge.
// The index has two forms.  Flat (B with at most BM_MAX_COLS columns): one bit
// per column of the item's range.  Two-level (wider B, up to BM2_MAX_COLS): a
// level-1 bitmap marks the occupied 32-column words, and a word table in word
// order holds each occupied word's bits, its index and the rank of its first
// entry; a lookup is then four shared loads (two rounds).  Long rows must be
// split; level-1 launches use k_merge.
#include "internal.h"
#include "common.cuh"

#include <algorithm>
#include <type_traits>

namespace spg {

constexpr int BM_IPT = 4;          // products per thread per batch: batch <= NT * 4

struct BmSmem {
    val_t *Rv, *Mv, *wa;
    int64_t *wbs, *wscan;
    int32_t *Rk, *Mk;
};

// Flat index: a bitmap over the item's columns and its rank directory.
struct FlatIndex {
    uint32_t *Bm;
    int32_t *Rd;
    int nwords;
    SPG_DEV int span() const { return nwords << 5; }
    // position of column offset x in R, or -1
    SPG_DEV int lookup(int x) const {
        const uint32_t wd = Bm[x >> 5];
        if (!((wd >> (x & 31)) & 1u)) return -1;
        return Rd[x >> 5] + __popc(wd & ((1u << (x & 31)) - 1u));
    }
    // the index of the sorted keys Rk[0..rlen) (column offsets key - lo)
    template <int NT>
    SPG_DEV void build(const int32_t *Rk, int rlen, int32_t lo, int32_t *scan32) {
        for (int t = threadIdx.x; t < nwords; t += NT) Bm[t] = 0u;
        __syncthreads();
        for (int t = threadIdx.x; t < rlen; t += NT) {
            const int x = Rk[t] - lo;
            atomicOr(&Bm[x >> 5], 1u << (x & 31));
        }
        __syncthreads();
        bitmap_rank<NT>(Bm, Rd, nwords, scan32);
    }
    // adds the columns of the nm misses; returns the number of columns.  The first
    // barrier is passed before `after_first_barrier` runs.  Ends with a barrier.
    template <int NT, typename F>
    SPG_DEV int add(const int32_t *Mk, int nm, int32_t lo, int32_t *scan32, F after_first_barrier) {
        for (int m = threadIdx.x; m < nm; m += NT) {
            const int x = Mk[m] - lo;
            atomicOr(&Bm[x >> 5], 1u << (x & 31));
        }
        __syncthreads();
        after_first_barrier();
        return bitmap_rank<NT>(Bm, Rd, nwords, scan32);
    }
};

// Two-level index: level-1 bits L1 over 32-column words (rank directory L1r),
// and the table of occupied words in word order: bits Wb, word index Wi and the
// rank Wr of the word's first entry.  T is scratch (zero between calls).
struct TwoIndex {
    uint32_t *L1, *T, *Wb;
    int32_t *L1r, *Wi, *Wr;
    int nw1;   // level-1 words
    int nocc;  // occupied words
    SPG_DEV int span() const { return nw1 << 10; }
    SPG_DEV int word_rank(int w) const {
        return L1r[w >> 5] + __popc(L1[w >> 5] & ((1u << (w & 31)) - 1u));
    }
    SPG_DEV int lookup(int x) const {
        const int w = x >> 5;
        const uint32_t l = L1[w >> 5];
        if (!((l >> (w & 31)) & 1u)) return -1;
        const int k = L1r[w >> 5] + __popc(l & ((1u << (w & 31)) - 1u));
        const uint32_t bits = Wb[k];
        if (!((bits >> (x & 31)) & 1u)) return -1;
        return Wr[k] + __popc(bits & ((1u << (x & 31)) - 1u));
    }
    template <int NT>
    SPG_DEV void build(const int32_t *Rk, int rlen, int32_t lo, int32_t *scan32) {
        for (int t = threadIdx.x; t < nw1; t += NT) {
            L1[t] = 0u;
            T[t] = 0u;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < rlen; t += NT) {
            const int w = (Rk[t] - lo) >> 5;
            atomicOr(&L1[w >> 5], 1u << (w & 31));
        }
        __syncthreads();
        nocc = bitmap_rank<NT>(L1, L1r, nw1, scan32);
        for (int k = threadIdx.x; k < nocc; k += NT) Wb[k] = 0u;
        __syncthreads();
        for (int t = threadIdx.x; t < rlen; t += NT) {
            const int x = Rk[t] - lo;
            const int k = word_rank(x >> 5);
            Wi[k] = x >> 5;
            atomicOr(&Wb[k], 1u << (x & 31));
        }
        __syncthreads();
        bitmap_rank<NT>(Wb, Wr, nocc, scan32);
    }
    template <int NT, typename F>
    SPG_DEV int add(const int32_t *Mk, int nm, int32_t lo, int32_t *scan32, F after_first_barrier) {
        // (a) words of the misses
        for (int m = threadIdx.x; m < nm; m += NT) {
            const int w = (Mk[m] - lo) >> 5;
            atomicOr(&T[w >> 5], 1u << (w & 31));
        }
        __syncthreads();
        after_first_barrier();
        // (b) level 1 takes them; T keeps only the words not occupied before
        for (int i = threadIdx.x; i < nw1; i += NT) {
            const uint32_t t = T[i], l = L1[i];
            T[i] = t & ~l;
            L1[i] = l | t;
        }
        __syncthreads();
        const int nocc_new = bitmap_rank<NT>(L1, L1r, nw1, scan32);
        // (c) old table entries move right to their new index, a chunk at a time from
        //     the right end (their targets lie at or beyond their old indices)
        constexpr int CH = NT * 4;
        for (int hi = nocc; hi > 0; hi -= CH) {
            const int base = hi > CH ? hi - CH : 0;
            uint32_t bb[4];
            int ww[4], nk[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = base + q * NT + threadIdx.x;
                nk[q] = -1;
                if (k < hi) {
                    bb[q] = Wb[k];
                    ww[q] = Wi[k];
                    const int t = word_rank(ww[q]);
                    if (t != k) nk[q] = t;
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (nk[q] >= 0) {
                    Wb[nk[q]] = bb[q];
                    Wi[nk[q]] = ww[q];
                }
            }
        }
        __syncthreads();
        // (d) new words start empty
        for (int i = threadIdx.x; i < nw1; i += NT) {
            uint32_t b = T[i];
            T[i] = 0u;
            while (b) {
                const int t = __ffs(b) - 1;
                b &= b - 1u;
                const int w = (i << 5) + t;
                const int k = word_rank(w);
                Wb[k] = 0u;
                Wi[k] = w;
            }
        }
        __syncthreads();
        // (e) the misses' bits, then the entry ranks of all words
        for (int m = threadIdx.x; m < nm; m += NT) {
            const int x = Mk[m] - lo;
            atomicOr(&Wb[word_rank(x >> 5)], 1u << (x & 31));
        }
        __syncthreads();
        nocc = nocc_new;
        return bitmap_rank<NT>(Wb, Wr, nocc, scan32);
    }
};

// Shared-memory layout: R (cap), the miss buffer (miss), the window of W A
// entries, then the index: flat (nwords = bitmap words) or two-level (nwords =
// level-1 words, plus a word table of cap entries).
__host__ __device__ inline size_t bm_layout(int cap, int nwords, int miss, int W, bool two, unsigned char *base,
                                            BmSmem *s, FlatIndex *fi, TwoIndex *ti) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = (off + bytes + 15) & ~size_t(15);
        return base ? base + o : nullptr;
    };
    const int nw4 = (nwords + 4) & ~3;
    unsigned char *p;
    p = take(sizeof(val_t) * cap);            if (s) s->Rv = (val_t *)p;
    p = take(sizeof(val_t) * miss);           if (s) s->Mv = (val_t *)p;
    p = take(sizeof(val_t) * W);              if (s) s->wa = (val_t *)p;
    p = take(sizeof(int64_t) * W);             if (s) s->wbs = (int64_t *)p;
    p = take(sizeof(int64_t) * (W + 1));       if (s) s->wscan = (int64_t *)p;
    p = take(sizeof(int32_t) * cap);           if (s) s->Rk = (int32_t *)p;
    p = take(sizeof(int32_t) * miss);          if (s) s->Mk = (int32_t *)p;
    if (!two) {
        p = take(sizeof(int32_t) * nw4);       if (fi) fi->Rd = (int32_t *)p;
        p = take(sizeof(uint32_t) * nw4);      if (fi) fi->Bm = (uint32_t *)p;
    } else {
        const int cap4 = (cap + 4) & ~3;
        p = take(sizeof(int32_t) * nw4);       if (ti) ti->L1r = (int32_t *)p;
        p = take(sizeof(uint32_t) * nw4);      if (ti) ti->L1 = (uint32_t *)p;
        p = take(sizeof(uint32_t) * nw4);      if (ti) ti->T = (uint32_t *)p;
        p = take(sizeof(int32_t) * cap4);      if (ti) ti->Wr = (int32_t *)p;
        p = take(sizeof(uint32_t) * cap4);     if (ti) ti->Wb = (uint32_t *)p;
        p = take(sizeof(int32_t) * cap4);      if (ti) ti->Wi = (int32_t *)p;
    }
    return off;
}

// Merges the nm buffered misses into R (length rlen) by rank; returns the new
// length.  All threads call, after a barrier that made the buffer visible; ends
// with a barrier.
template <int NT, typename Index>
SPG_DEV int bm_merge_misses(const BmSmem &s, Index &ix, int rlen, int nm, int32_t lo, int32_t *scan32,
                            int32_t *nmiss_shared) {
    // every thread has read the buffer count before the index's first barrier:
    // the counter can restart after it
    const int fnew = ix.template add<NT>(s.Mk, nm, lo, scan32, [&] {
        if (threadIdx.x == 0) *nmiss_shared = 0;
    });
    // old entries move right (to their rank in the union), a chunk at a time from
    // the right end.  A chunk's targets lie at or beyond its own old positions, so
    // they never overwrite an entry that a chunk to its left still has to read;
    // only the chunk's own reads must finish before its writes (one barrier).
    constexpr int CH = NT * 4;
    for (int hi = rlen; hi > 0; hi -= CH) {
        const int base = hi > CH ? hi - CH : 0;
        int32_t kk[4];
        val_t vv[4];
        int np[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {  // entry base + q*NT + thread: consecutive lanes, consecutive words
            const int p = base + q * NT + threadIdx.x;
            np[q] = -1;
            if (p < hi) {
                kk[q] = s.Rk[p];
                vv[q] = s.Rv[p];
                const int t = ix.lookup(kk[q] - lo);
                if (t != p) np[q] = t;
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (np[q] >= 0 && SPG_IN(np[q] < fnew, 108)) {
                s.Rk[np[q]] = kk[q];
                s.Rv[np[q]] = vv[q];
            }
        }
    }
    __syncthreads();
    // new columns: key and a zero value (duplicate misses write the same), then the sums
    for (int m = threadIdx.x; m < nm; m += NT) {
        const int32_t c = s.Mk[m];
        const int t = ix.lookup(c - lo);
        if (!SPG_IN(t >= 0 && t < fnew, 108)) continue;
        s.Rk[t] = c;
        s.Rv[t] = 0.0;
    }
    __syncthreads();
    for (int m = threadIdx.x; m < nm; m += NT) {
        const int t = ix.lookup(s.Mk[m] - lo);
        if (SPG_IN(t >= 0 && t < fnew, 108)) atomicAdd(&s.Rv[t], s.Mv[m]);
    }
    __syncthreads();
    return fnew;
}

template <int NT, int MINB, bool TWO>
__global__ void __launch_bounds__(NT, MINB)
k_merge_bm(StageArgs a, MergeItems it, MergeLaunch L) {
    extern __shared__ __align__(16) unsigned char bm_smem[];
    __shared__ int64_t scan64[NT / 32 + 1];
    __shared__ int32_t scan32[NT / 32 + 1];
    __shared__ int32_t s_nmiss;
    constexpr int W = NT;
    using Index = typename std::conditional<TWO, TwoIndex, FlatIndex>::type;
    BmSmem s;
    FlatIndex fi{};
    TwoIndex ti{};
    const int kb = L.batch;
    const int mcap = L.bm_miss;
    bm_layout(L.cap, L.bm_words, mcap, W, TWO, bm_smem, &s, &fi, &ti);

    const int64_t w = blockIdx.x;
    const int j = L.work ? L.work[w] : (int)(L.work_base + w);
    const int row = it.row[j];
    const int32_t clo = it.clo[j], chi = it.chi[j];
    const bool filtered = (clo > 0) || (chi < INT32_MAX);
    const int32_t lo = clo > 0 ? clo : 0;  // bitmap origin
    const int64_t hicol = min((int64_t)chi, a.B.ncols);
    const int nwords = hicol > lo ? (int)((hicol - lo + 31) >> 5) : 1;
    const int nunits = TWO ? (nwords + 31) >> 5 : nwords;  // index words of this item
    const int64_t a0 = a.A.rp[row], a1 = a.A.rp[row + 1];
    int rlen = it.src_len[j];
    int64_t e = a0 + it.ck_entry[j];
    int64_t off = it.ck_off[j];

    // where this launch writes the item: its home if large enough, else a fresh
    // slot; without a pool the item's capacity is that of its home
    int32_t *dst_col = it.home_col[j];
    val_t *dst_val = it.home_val[j];
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
    if (nunits > L.bm_words || rlen > cap) {  // cannot happen: items fit the index; relaunches fit R
        if (threadIdx.x == 0) atomicExch((unsigned long long *)L.err, 1ull);
        return;
    }
    fi.nwords = nwords;
    ti.nw1 = nunits;
    ti.nocc = 0;
    Index &ix = *[&] {
        if constexpr (TWO) return &ti; else return &fi;
    }();
    const int span = ix.span();
    // reload the item's sequence (empty for a fresh row; half of the parent's for a split child)
    if (threadIdx.x == 0) s_nmiss = 0;
    bool bad = false;
    {
        const int32_t *sc = it.src_col[j];
        const val_t *sv = it.src_val[j];
        for (int t = threadIdx.x; t < rlen; t += NT) {
            const int32_t c = sc[t];
            if ((unsigned)(c - lo) >= (unsigned)span) bad = true;  // cannot happen: items hold their own columns
            s.Rk[t] = c;
            s.Rv[t] = sv[t];
        }
    }
    if (__syncthreads_or(bad)) {
        if (threadIdx.x == 0) atomicExch((unsigned long long *)L.err, 5ull);
        return;
    }
    ix.template build<NT>(s.Rk, rlen, lo, scan32);
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
                rlen = bm_merge_misses<NT>(s, ix, rlen, nmiss, lo, scan32, &s_nmiss);
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
            val_t val[BM_IPT];
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
                    if ((unsigned)x >= (unsigned)span) {  // a column outside [0, ncols): bad input
                        atomicExch((unsigned long long *)L.err, 5ull);
                        continue;
                    }
                    rpos[k] = ix.lookup(x);
                    if (rpos[k] < 0) miss |= 1u << k;
                }
            }
            int nb = need;
            if (avail < need) {
                // the batch fits if its actual misses fit the free capacity (its hits take none)
                int cm = block_reduce_sum<NT, int>(__popc(miss), scan32);
                if (cm > avail && nmiss > 0) {
                    rlen = bm_merge_misses<NT>(s, ix, rlen, nmiss, lo, scan32, &s_nmiss);
                    nmiss = 0;
                    avail = cap - rlen;
                    miss = 0;  // the bitmap changed: look the products up again
#pragma unroll
                    for (int k = 0; k < BM_IPT; ++k) {
                        rpos[k] = -1;
                        if (k < cnt) {
                            const int x = key[k] - lo;
                            if ((unsigned)x >= (unsigned)span) continue;
                            rpos[k] = ix.lookup(x);
                            if (rpos[k] < 0) miss |= 1u << k;
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
                if (rpos[k] >= 0 && SPG_IN(rpos[k] < rlen, 107)) atomicAdd(&s.Rv[rpos[k]], val[k]);
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
                        if (SPG_IN(slot < mcap, 106)) {
                            s.Mk[slot] = key[k];
                            s.Mv[slot] = val[k];
                        }
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
        rlen = bm_merge_misses<NT>(s, ix, rlen, nmiss, lo, scan32, &s_nmiss);
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

int merge_bm_smem_bytes(int cap, int nwords, int miss, int wide_above, bool two) {
    return (int)bm_layout(cap, nwords, miss, bm_threads(cap, wide_above), two, nullptr, nullptr, nullptr, nullptr);
}

int merge_bm_max_cap(int nwords, int miss, int smem_limit, int wide_above, bool two) {
    int cap = 256;
    while (merge_bm_smem_bytes(cap + 256, nwords, miss, wide_above, two) <= smem_limit) cap += 256;
    return cap;
}

template <int NT, int MINB, bool TWO>
static cudaError_t launch_bm_nt(const StageArgs &a, const MergeItems &s, const MergeLaunch &L, int smem,
                                cudaStream_t st) {
    auto kern = k_merge_bm<NT, MINB, TWO>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)L.nwork, NT, smem, st>>>(a, s, L);
    return cudaGetLastError();
}

template <bool TWO>
static cudaError_t launch_bm(const StageArgs &a, const MergeItems &s, const MergeLaunch &L, int nt, int smem,
                             cudaStream_t st) {
    if (nt == 128) return launch_bm_nt<128, 4, TWO>(a, s, L, smem, st);
    if (nt == 256) return launch_bm_nt<256, 2, TWO>(a, s, L, smem, st);
    return launch_bm_nt<512, 1, TWO>(a, s, L, smem, st);
}

cudaError_t launch_merge_bm(const StageArgs &a, const MergeItems &s, const MergeLaunch &L, cudaStream_t st) {
    if (L.nwork <= 0) return cudaSuccess;
    const int nt = bm_threads(L.cap, L.wide_above);
    // the index must cover B's columns: bm_words bitmap words (flat) or level-1 words (two-level)
    const int64_t span = L.bm_two ? (int64_t)L.bm_words * 1024 : (int64_t)L.bm_words * 32;
    if (L.level1 || L.bm_words <= 0 || L.batch > nt * BM_IPT || L.batch < 32 || L.bm_miss < L.batch ||
        span < a.B.ncols)
        return cudaErrorInvalidValue;
    const int smem = merge_bm_smem_bytes(L.cap, L.bm_words, L.bm_miss, L.wide_above, L.bm_two != 0);
    return L.bm_two ? launch_bm<true>(a, s, L, nt, smem, st) : launch_bm<false>(a, s, L, nt, smem, st);
}

}  // namespace spg
