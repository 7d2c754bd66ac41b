// Stage 3, bin group 5 (u_i > 512): the merge method of Section 4.1 with
// progressive reallocation and a level-1 sequence.
//
// One CTA per row.  The row's result sequence R (sorted, duplicate-free) lives
// in shared memory with a capacity `cap` fixed per launch.  The A row is walked
// in windows of W entries; the products of a window are consumed in batches.
// For each batch the four sub-steps of the paper's parallel insert are done for
// many B rows at once:
//   (1) every product binary-searches R and a small pending sorted set N; a hit
//       is fused into the existing entry;
//   (2) a block scan over the misses gives their compacted positions;
//   (3) the misses -- still one sorted run per B row -- are merged pairwise by
//       merge path into one sorted sequence and equal columns are fused;
//   (4) that sequence is merged into N, and N into R when N is full, in place,
//       right to left, with merge path.
// The batch never exceeds the free capacity, so a merge can always complete.
// When the free capacity gets too small the CTA records a checkpoint (the A
// entry and the offset inside its B row), writes R to global memory and queues
// the row; the host allocates 2x larger homes and relaunches with 2x larger
// shared memory, and the row reloads R and resumes (progressive reallocation).
// Rows that outgrow the largest shared-memory capacity run in level-1 mode: the
// shared sequence is a level-1 sequence that is union-merged into a global
// sequence whenever it fills up, and once more before the row ends.
//
// Fusion in (1) uses shared-memory atomicAdd, so the order in which several
// products of one batch are added to one existing entry is not fixed; every
// other sum is taken in a fixed order.
#include "internal.h"
#include "common.cuh"
#include "scan.cuh"

#include <algorithm>

namespace spg {

constexpr int MERGE_MAX_IPT = 4;   // products per thread per batch: batch <= NT * 4
constexpr int MERGE_TN_MAX = 2048; // pending-set capacity

struct MergeSmem {
    val_t *Rv, *Nv, *Sav, *Sbv, *wa;
    int64_t *wbs, *wscan;
    int32_t *Rk, *Nk, *Sak, *Sbk, *pf, *runoff;
};

__host__ __device__ inline int merge_tn(int cap) { return cap < MERGE_TN_MAX ? cap : MERGE_TN_MAX; }

// Shared-memory layout of one CTA: result R (cap), pending set N, two batch
// buffers, the compaction prefix, and the window of W A entries (W = threads).
__host__ __device__ inline size_t merge_layout(int cap, int kb, int W, unsigned char *base, MergeSmem *s) {
    const int tn = merge_tn(cap);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = (off + bytes + 15) & ~size_t(15);
        return base ? base + o : nullptr;
    };
    unsigned char *p;
    p = take(sizeof(val_t) * cap);       if (s) s->Rv = (val_t *)p;
    p = take(sizeof(val_t) * tn);        if (s) s->Nv = (val_t *)p;
    p = take(sizeof(val_t) * kb);        if (s) s->Sav = (val_t *)p;
    p = take(sizeof(val_t) * kb);        if (s) s->Sbv = (val_t *)p;
    p = take(sizeof(val_t) * W);         if (s) s->wa = (val_t *)p;
    p = take(sizeof(int64_t) * W);        if (s) s->wbs = (int64_t *)p;
    p = take(sizeof(int64_t) * (W + 1));  if (s) s->wscan = (int64_t *)p;
    p = take(sizeof(int32_t) * cap);      if (s) s->Rk = (int32_t *)p;
    p = take(sizeof(int32_t) * tn);       if (s) s->Nk = (int32_t *)p;
    p = take(sizeof(int32_t) * kb);       if (s) s->Sak = (int32_t *)p;
    p = take(sizeof(int32_t) * kb);       if (s) s->Sbk = (int32_t *)p;
    p = take(sizeof(int32_t) * (kb + 1)); if (s) s->pf = (int32_t *)p;
    p = take(sizeof(int32_t) * (W + 2));  if (s) s->runoff = (int32_t *)p;
    return off;
}

// Threads per CTA for a launch with result capacity `cap`: 128 up to 512 entries,
// 256 up to `wide_above` entries (0 = 2048), 512 beyond.
inline int merge_threads(int cap, int wide_above) {
    if (wide_above <= 0) wide_above = 2048;
    return cap <= 512 ? 128 : (cap <= wide_above ? 256 : 512);
}

int merge_smem_bytes(int cap, int batch, int wide_above) {
    return (int)merge_layout(cap, batch, merge_threads(cap, wide_above), nullptr, nullptr);
}

int merge_max_cap(int batch, int smem_limit, int wide_above) {
    int cap = 256;
    while (merge_smem_bytes(cap + 256, std::min(batch, 4 * merge_threads(cap + 256, wide_above)), wide_above) <=
           smem_limit)
        cap += 256;
    return cap;
}

// One level of the pairwise merge of sorted runs.  The runs of the current level
// are groups of `stride` original runs: run r spans [off(r*stride), off((r+1)*stride))
// with off(i) = runoff[min(i, nr0)], so the offsets never need rewriting between
// levels.  Runs 2p and 2p+1 are merged into the same range of dk/dv.  All threads
// call; ends with a barrier.
template <int NT>
SPG_DEV void merge_level(const int32_t *sk, const val_t *sv, const int32_t *runoff, int nr0, int stride, int n,
                         int32_t *dk, val_t *dv) {
    const int ipt = (n + NT - 1) / NT;
    int d = threadIdx.x * ipt;
    const int dend = min(n, d + ipt);
    if (d < dend) {
        const int nruns = (nr0 + stride - 1) / stride;
        const int npairs = (nruns + 1) >> 1;
        const int pstride = 2 * stride;
        int lo = 0, hi = npairs - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (runoff[min(mid * pstride, nr0)] <= d) lo = mid; else hi = mid - 1;
        }
        int p = lo;
        while (d < dend) {
            const int as = runoff[min(p * pstride, nr0)];
            const int am = runoff[min(p * pstride + stride, nr0)];
            const int ae = runoff[min(p * pstride + pstride, nr0)];
            const int i = merge_path(sk + as, am - as, sk + am, ae - am, d - as);
            int ia = as + i, ib = am + (d - as - i);
            const int stop = min(dend, ae);
            while (d < stop) {
                const bool ta = ia < am && (ib >= ae || sk[ia] <= sk[ib]);
                if (ta) { dk[d] = sk[ia]; dv[d] = sv[ia]; ++ia; }
                else { dk[d] = sk[ib]; dv[d] = sv[ib]; ++ib; }
                ++d;
            }
            ++p;
        }
    }
    __syncthreads();
}

// Fuses runs of equal keys of the sorted k/v[0..n) into ok/ov (in order, sums
// taken left to right).  Returns the number of distinct keys.  All threads call.
template <int NT>
SPG_DEV int compress_runs(const int32_t *k, const val_t *v, int n, int32_t *ok, val_t *ov,
                          int32_t *scan32) {
    const int ipt = (n + NT - 1) / NT;
    const int q0 = threadIdx.x * ipt;
    const int q1 = min(n, q0 + ipt);
    int cnt = 0;
    for (int q = q0; q < q1; ++q)
        if (q == 0 || k[q] != k[q - 1]) ++cnt;
    int tot;
    int o = block_exclusive_scan<NT, int, false>(cnt, scan32, tot);
    for (int q = q0; q < q1; ++q) {
        if (q == 0 || k[q] != k[q - 1]) {
            const int32_t key = k[q];
            val_t s = v[q];
            for (int r = q + 1; r < n && k[r] == key; ++r) s += v[r];
            ok[o] = key;
            ov[o] = s;
            ++o;
        }
    }
    __syncthreads();
    return tot;
}

// Level-1 flush: Z = X u Y with equal keys fused, X global (nx), Y in shared
// memory (ny), Z global.  Streams X through the batch buffers in tiles; each
// step consumes every key <= a limit from both inputs.  Returns |Z|.
template <int NT>
SPG_DEV int64_t union_stream(const int32_t *xk, const val_t *xv, int64_t nx, const int32_t *yk,
                             const val_t *yv, int ny, int32_t *zk, val_t *zv, const MergeSmem &s,
                             int kb, int32_t *scan32) {
    const int T = kb / 2;
    int64_t xa = 0, zo = 0;
    int ya = 0;
    while (xa < nx || ya < ny) {
        const int nxt = (int)min((int64_t)T, nx - xa);
        for (int t = threadIdx.x; t < nxt; t += NT) {
            s.Sak[t] = xk[xa + t];
            s.Sav[t] = xv[xa + t];
        }
        __syncthreads();
        int32_t lim = (xa + nxt < nx) ? s.Sak[nxt - 1] : KEY_PAD;
        int yb = ya + upper_bound_i32(yk + ya, ny - ya, lim);
        if (yb - ya > T) {
            yb = ya + T;
            lim = yk[yb - 1];
        }
        const int xc = upper_bound_i32(s.Sak, nxt, lim);
        merge_into<NT>(s.Sak, s.Sav, xc, yk + ya, yv + ya, yb - ya, s.Sbk, s.Sbv);
        const int nz = compress_runs<NT>(s.Sbk, s.Sbv, xc + (yb - ya), zk + zo, zv + zo, scan32);
        zo += nz;
        xa += xc;
        ya = yb;
    }
    return zo;
}

template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
k_merge(StageArgs a, MergeItems it, MergeLaunch L) {
    extern __shared__ __align__(16) unsigned char merge_smem[];
    __shared__ int64_t scan64[NT / 32 + 1];
    __shared__ int32_t scan32[NT / 32 + 1];
    constexpr int W = NT;
    MergeSmem s;
    const int kb = L.batch;
    const int tn = merge_tn(L.cap);
    merge_layout(L.cap, kb, W, merge_smem, &s);

    const int64_t w = blockIdx.x;
    const int j = L.work ? L.work[w] : (int)(L.work_base + w);
    const int row = it.row[j];
    const int32_t clo = it.clo[j], chi = it.chi[j];
    const bool filtered = (clo > 0) || (chi < INT32_MAX);
    const int64_t a0 = a.A.rp[row], a1 = a.A.rp[row + 1];
    int rlen = it.src_len[j];
    int64_t e = a0 + it.ck_entry[j];
    int64_t off = it.ck_off[j];

    // reload the item's sequence (empty for a fresh row; half of the parent's for a split child)
    {
        const int32_t *sc = it.src_col[j];
        const val_t *sv = it.src_val[j];
        for (int t = threadIdx.x; t < rlen; t += NT) {
            s.Rk[t] = sc[t];
            s.Rv[t] = sv[t];
        }
    }
    // where this launch writes the item: its home if large enough, else a fresh
    // slot; without a pool the item's capacity is that of its home
    int32_t *dst_col = it.home_col[j];
    val_t *dst_val = it.home_val[j];
    int64_t dst_cap = it.home_cap[j];
    int cap = L.cap;
    if (!L.level1 && dst_cap < cap) {
        if (L.pool_col != nullptr) {
            dst_col = L.pool_col + w * L.pool_cap;
            dst_val = L.pool_val + w * L.pool_cap;
            dst_cap = L.pool_cap;
        } else {
            cap = (int)dst_cap;
        }
    }
    // level-1 global sequence: ping-pong between g0 and g1
    int32_t *g0k = nullptr, *g1k = nullptr;
    val_t *g0v = nullptr, *g1v = nullptr;
    int64_t glen = 0;
    if (L.level1) {
        const int64_t go = L.g_off[w], gc = L.g_cap[w];
        g0k = L.g_col + go;
        g0v = L.g_val + go;
        g1k = L.g_col + go + gc;
        g1v = L.g_val + go + gc;
    }
    int nlen = 0;
    __syncthreads();

    bool overflow = false;
    while (e < a1 && !overflow) {
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
                    const int64_t lo = rs + lower_bound_i32(a.B.col + rs, n, clo);
                    bs = bs > lo ? bs : lo;
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
            int avail = cap - rlen - nlen;
            if (avail < need) {
                if (L.level1) {
                    // flush the level-1 sequence into the global sequence
                    if (nlen > 0) {
                        merge_inplace_rtl<NT, 4>(s.Rk, s.Rv, rlen, s.Nk, s.Nv, nlen);
                        rlen += nlen;
                        nlen = 0;
                    }
                    glen = union_stream<NT>(g0k, g0v, glen, s.Rk, s.Rv, rlen, g1k, g1v, s, kb, scan32);
                    int32_t *tk = g0k; g0k = g1k; g1k = tk;
                    val_t *tv = g0v; g0v = g1v; g1v = tv;
                    rlen = 0;
                    avail = cap;
                } else if (avail < (kb >> 2) || avail <= 0) {
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
            }
            const int nb = min(need, avail);
            const int tf = find_segment_i64(s.wscan, nW, p0);
            const int tl = find_segment_i64(s.wscan, nW, p0 + nb - 1);
            const int nruns = tl - tf + 1;
            // (0) each thread expands IPT consecutive products of the batch into registers
            const int ipt = (nb + NT - 1) / NT;
            const int q0 = threadIdx.x * ipt;
            const int cnt = max(0, min(ipt, nb - q0));
            int32_t key[MERGE_MAX_IPT];
            val_t val[MERGE_MAX_IPT];
            if (cnt > 0) {
                // all addresses first, then all loads: one L2 round trip per batch, not IPT
                int te[MERGE_MAX_IPT], to[MERGE_MAX_IPT];  // window entry and offset in its B range
                int64_t pos = p0 + q0;
                int t = tf + find_segment_i64(s.wscan + tf, nruns, pos);
#pragma unroll
                for (int k = 0; k < MERGE_MAX_IPT; ++k) {
                    if (k < cnt) {
                        while (t + 1 < nW && s.wscan[t + 1] <= pos) ++t;
                        te[k] = t;
                        to[k] = (int)(pos - s.wscan[t]);
                        ++pos;
                    }
                }
#pragma unroll
                for (int k = 0; k < MERGE_MAX_IPT; ++k)
                    if (k < cnt) key[k] = __ldg(a.B.col + s.wbs[te[k]] + to[k]);
#pragma unroll
                for (int k = 0; k < MERGE_MAX_IPT; ++k)
                    if (k < cnt) val[k] = __ldg(a.B.val + s.wbs[te[k]] + to[k]);
#pragma unroll
                for (int k = 0; k < MERGE_MAX_IPT; ++k)
                    if (k < cnt) val[k] *= s.wa[te[k]];
            }
            // (1) fuse products whose column is already in R or N (lockstep binary searches)
            unsigned miss = 0;
            int pos[MERGE_MAX_IPT];
            if (rlen > 0) {
                lower_bound_multi<MERGE_MAX_IPT>(s.Rk, rlen, key, cnt, pos);
#pragma unroll
                for (int k = 0; k < MERGE_MAX_IPT; ++k) {
                    if (k < cnt) {
                        if (pos[k] < rlen && s.Rk[pos[k]] == key[k]) atomicAdd(&s.Rv[pos[k]], val[k]);
                        else miss |= 1u << k;
                    }
                }
            } else {
                miss = (1u << cnt) - 1u;
            }
            if (nlen > 0 && miss != 0) {
                int32_t k2[MERGE_MAX_IPT];
#pragma unroll
                for (int k = 0; k < MERGE_MAX_IPT; ++k) k2[k] = (miss >> k) & 1u ? key[k] : INT_MIN;
                lower_bound_multi<MERGE_MAX_IPT>(s.Nk, nlen, k2, cnt, pos);
#pragma unroll
                for (int k = 0; k < MERGE_MAX_IPT; ++k) {
                    if ((miss >> k) & 1u) {
                        if (pos[k] < nlen && s.Nk[pos[k]] == key[k]) {
                            atomicAdd(&s.Nv[pos[k]], val[k]);
                            miss &= ~(1u << k);
                        }
                    }
                }
            }
            // (2) compact the misses into Sb, keeping one run per B row
            int nnew;
            int o = block_exclusive_scan<NT, int, false>(__popc(miss), scan32, nnew);
#pragma unroll
            for (int k = 0; k < MERGE_MAX_IPT; ++k) {
                if (k < cnt) {
                    s.pf[q0 + k] = o;
                    if ((miss >> k) & 1u) {
                        s.Sbk[o] = key[k];
                        s.Sbv[o] = val[k];
                        ++o;
                    }
                }
            }
            if (threadIdx.x == 0) s.pf[nb] = nnew;
            __syncthreads();
            for (int r = threadIdx.x; r <= nruns; r += NT) {
                const int q = (r == 0) ? 0 : (r == nruns ? nb : (int)(s.wscan[tf + r] - p0));
                s.runoff[r] = s.pf[q];
            }
            __syncthreads();
            if (nnew > 0) {
                // (3) pairwise merge-path merges of the runs, then fuse equal columns
                int32_t *ck = s.Sbk, *okk = s.Sak;
                val_t *cv = s.Sbv, *ovv = s.Sav;
                for (int stride = 1; stride < nruns; stride *= 2) {
                    merge_level<NT>(ck, cv, s.runoff, nruns, stride, nnew, okk, ovv);
                    int32_t *tk = ck; ck = okk; okk = tk;
                    val_t *tv = cv; cv = ovv; ovv = tv;
                }
                const int nn = compress_runs<NT>(ck, cv, nnew, okk, ovv, scan32);
                // (4) in-place merges into N, and N into R
                if (nlen + nn > tn) {
                    if (nlen > 0) {
                        merge_inplace_rtl<NT, 4>(s.Rk, s.Rv, rlen, s.Nk, s.Nv, nlen);
                        rlen += nlen;
                        nlen = 0;
                    }
                    if (nn > tn) {
                        merge_inplace_rtl<NT, 4>(s.Rk, s.Rv, rlen, okk, ovv, nn);
                        rlen += nn;
                    } else {
                        for (int t = threadIdx.x; t < nn; t += NT) {
                            s.Nk[t] = okk[t];
                            s.Nv[t] = ovv[t];
                        }
                        nlen = nn;
                        __syncthreads();
                    }
                } else {
                    merge_inplace_rtl<NT, 4>(s.Nk, s.Nv, nlen, okk, ovv, nn);
                    nlen += nn;
                }
            }
            p0 += nb;
        }
        if (!overflow) {
            e += nW;
            off = 0;
        }
    }
    // fold the pending set into R
    if (nlen > 0) {
        merge_inplace_rtl<NT, 4>(s.Rk, s.Rv, rlen, s.Nk, s.Nv, nlen);
        rlen += nlen;
        nlen = 0;
    }
    int64_t final_len;
    int32_t *fin_col;
    val_t *fin_val;
    int64_t fin_cap;
    if (L.level1) {
        glen = union_stream<NT>(g0k, g0v, glen, s.Rk, s.Rv, rlen, g1k, g1v, s, kb, scan32);
        final_len = glen;
        fin_col = g1k;
        fin_val = g1v;
        fin_cap = L.g_cap[w];
    } else {
        if (rlen > dst_cap) {  // cannot happen: dst_cap >= cap >= rlen
            if (threadIdx.x == 0) atomicExch((unsigned long long *)L.err, 1ull);
            return;
        }
        for (int t = threadIdx.x; t < rlen; t += NT) {
            dst_col[t] = s.Rk[t];
            dst_val[t] = s.Rv[t];
        }
        final_len = rlen;
        fin_col = dst_col;
        fin_val = dst_val;
        fin_cap = dst_cap;
    }
    if (threadIdx.x == 0) {
        it.home_col[j] = fin_col;
        it.home_val[j] = fin_val;
        it.home_cap[j] = fin_cap;
        if (overflow) {
            it.src_col[j] = fin_col;
            it.src_val[j] = fin_val;
            it.src_len[j] = (int32_t)final_len;
            const int slot = atomicAdd(L.ovf_count, 1);
            L.ovf_list[slot] = j;
        } else {
            it.len[j] = (int32_t)final_len;
        }
    }
}

__global__ void k_merge_init(const int32_t *rows37, int64_t n37, const int64_t *ctil_rp, int32_t *ctil_col,
                             val_t *ctil_val, MergeItems it) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n37) return;
    const int row = rows37[j];
    const int64_t o = ctil_rp[row];
    it.row[j] = row;
    it.clo[j] = 0;
    it.chi[j] = INT32_MAX;
    it.src_col[j] = ctil_col + o;
    it.src_val[j] = ctil_val + o;
    it.src_len[j] = 0;
    it.home_col[j] = ctil_col + o;
    it.home_val[j] = ctil_val + o;
    it.home_cap[j] = ctil_rp[row + 1] - o;
    it.len[j] = 0;
    it.ck_entry[j] = 0;
    it.ck_off[j] = 0;
    it.child[j] = -1;
    it.parent[j] = -1;
}

cudaError_t launch_merge_init(const int32_t *rows37, int64_t n37, const int64_t *ctil_rp, int32_t *ctil_col,
                              val_t *ctil_val, const MergeItems &it, cudaStream_t st) {
    if (n37 <= 0) return cudaSuccess;
    k_merge_init<<<(unsigned)((n37 + 255) / 256), 256, 0, st>>>(rows37, n37, ctil_rp, ctil_col, ctil_val, it);
    return cudaGetLastError();
}

// Splits an overflowed item at the median column of its dumped sequence.  Both
// children resume from the parent's checkpoint and only take products inside
// their column range.  The left child keeps the parent's home, where its half
// already sits at the start; the right child gets slot i of `pool`, and
// k_split_copy moves the right half there, so no two items share memory.
__global__ void k_split(const int32_t *ovf, int64_t n, int64_t first_new, MergeItems it, int32_t *pool_col,
                        val_t *pool_val, int64_t pool_cap) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = ovf[i];
    const int plen = it.src_len[p];
    const int mid = plen / 2;
    const int32_t mkey = it.src_col[p][mid];
    const int64_t l = first_new + 2 * i, r = l + 1;
    for (int c = 0; c < 2; ++c) {
        const int64_t q = c == 0 ? l : r;
        it.row[q] = it.row[p];
        it.clo[q] = c == 0 ? it.clo[p] : mkey;
        it.chi[q] = c == 0 ? mkey : it.chi[p];
        it.len[q] = 0;
        it.ck_entry[q] = it.ck_entry[p];
        it.ck_off[q] = it.ck_off[p];
        it.child[q] = -1;
        it.parent[q] = p;
    }
    it.src_col[l] = it.src_col[p];
    it.src_val[l] = it.src_val[p];
    it.src_len[l] = mid;
    it.home_col[l] = it.home_col[p];
    it.home_val[l] = it.home_val[p];
    it.home_cap[l] = it.home_cap[p];
    it.src_col[r] = pool_col + i * pool_cap;
    it.src_val[r] = pool_val + i * pool_cap;
    it.src_len[r] = plen - mid;
    it.home_col[r] = pool_col + i * pool_cap;
    it.home_val[r] = pool_val + i * pool_cap;
    it.home_cap[r] = pool_cap;
    it.child[p] = (int32_t)l;
    it.len[p] = 0;
}

// One CTA per split: copies the right half of the parent's sequence into the right child's slot.
__global__ void k_split_copy(const int32_t *ovf, int64_t first_new, MergeItems it) {
    const int64_t i = blockIdx.x;
    const int p = ovf[i];
    const int64_t r = first_new + 2 * i + 1;
    const int plen = it.src_len[p];
    const int mid = plen / 2;
    const int32_t *sc = it.src_col[p] + mid;
    const val_t *sv = it.src_val[p] + mid;
    int32_t *dc = it.home_col[r];
    val_t *dv = it.home_val[r];
    for (int t = threadIdx.x; t < plen - mid; t += blockDim.x) {
        dc[t] = sc[t];
        dv[t] = sv[t];
    }
}

cudaError_t launch_split(const int32_t *ovf, int64_t n, int64_t first_new, const MergeItems &it,
                         int32_t *pool_col, val_t *pool_val, int64_t pool_cap, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_split<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ovf, n, first_new, it, pool_col, pool_val, pool_cap);
    k_split_copy<<<(unsigned)n, 256, 0, st>>>(ovf, first_new, it);
    return cudaGetLastError();
}

// Sum of the leaf lengths under item j (its column slices).
SPG_DEV int64_t leaf_total(const MergeItems &it, int j) {
    int64_t tot = 0;
    for (int x = split_first_leaf(it, j); x >= 0; x = split_next_leaf(it, j, x)) tot += it.len[x];
    return tot;
}

__global__ void k_finalize37(int64_t n37, MergeItems it, int32_t *nnzc, int64_t *err) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n37) return;
    const int64_t tot = leaf_total(it, (int)j);
    if (tot < 0 || tot > INT32_MAX) atomicExch((unsigned long long *)err, 2ull);
    nnzc[it.row[j]] = tot < 0 ? 0 : (int32_t)tot;
}

cudaError_t launch_finalize37(int64_t n37, const MergeItems &it, int32_t *nnzc, int64_t *err, cudaStream_t st) {
    if (n37 <= 0) return cudaSuccess;
    k_finalize37<<<(unsigned)((n37 + 127) / 128), 128, 0, st>>>(n37, it, nnzc, err);
    return cudaGetLastError();
}

__global__ void k_level1_caps(MergeItems it, const int32_t *work, int64_t nwork, const int64_t *u,
                              int64_t ncols, int64_t *g_cap) {
    int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nwork) return;
    const int j = work[w];
    int64_t c = u[it.row[j]];
    if (c > ncols) c = ncols;
    g_cap[w] = c < 1 ? 1 : c;
}

struct LoadCap2 {
    const int64_t *cap;
    SPG_DEV int64_t operator()(int64_t i) const { return 2 * cap[i]; }
};
struct StoreOff {
    int64_t *out;
    SPG_DEV void operator()(int64_t i, int64_t v) const { out[i] = v; }
};

cudaError_t launch_level1_sizes(const MergeItems &it, const int32_t *work, int64_t nwork,
                                const int64_t *u, int64_t ncols, int64_t *g_cap, int64_t *g_off,
                                int64_t *partial, int64_t *total, cudaStream_t st) {
    if (nwork > 0)
        k_level1_caps<<<(unsigned)((nwork + 255) / 256), 256, 0, st>>>(it, work, nwork, u, ncols, g_cap);
    return device_exclusive_scan(nwork, LoadCap2{g_cap}, StoreOff{g_off}, partial, total, st);
}

template <int NT, int MINB>
static cudaError_t launch_merge_nt(const StageArgs &a, const MergeItems &s, const MergeLaunch &L, int smem,
                                  cudaStream_t st) {
    auto kern = k_merge<NT, MINB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)L.nwork, NT, smem, st>>>(a, s, L);
    return cudaGetLastError();
}

cudaError_t launch_merge(const StageArgs &a, const MergeItems &s, const MergeLaunch &L, cudaStream_t st) {
    if (L.nwork <= 0) return cudaSuccess;
    if (L.bm_words > 0 && !L.level1) return launch_merge_bm(a, s, L, st);
    const int nt = merge_threads(L.cap, L.wide_above);
    // batch >= 32 keeps every loop of the kernel progressing (the level-1 stream takes batch/2 per step)
    if (L.batch > nt * MERGE_MAX_IPT || L.batch < 32 || L.batch > L.cap) return cudaErrorInvalidValue;
    const int smem = merge_smem_bytes(L.cap, L.batch, L.wide_above);
    if (nt == 128) return launch_merge_nt<128, 4>(a, s, L, smem, st);
    if (nt == 256) return launch_merge_nt<256, 2>(a, s, L, smem, st);
    return launch_merge_nt<512, 1>(a, s, L, smem, st);
}

int merge_batch_limit(int cap, int wide_above) { return MERGE_MAX_IPT * merge_threads(cap, wide_above); }

}  // namespace spg
