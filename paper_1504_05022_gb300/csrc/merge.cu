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

namespace spg {

constexpr int MERGE_NT = 256;
constexpr int MERGE_W = 256;       // A entries per window (one per thread)
constexpr int MERGE_MAX_IPT = 8;   // batch <= MERGE_NT * MERGE_MAX_IPT
constexpr int MERGE_TN_MAX = 1024; // pending-set capacity

struct MergeSmem {
    double *Rv, *Nv, *Sav, *Sbv, *wa;
    int64_t *wbs, *wscan;
    int32_t *Rk, *Nk, *Sak, *Sbk, *pf, *runoff;
};

SPG_DEV size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline int merge_tn(int cap) { return cap < MERGE_TN_MAX ? cap : MERGE_TN_MAX; }

__host__ __device__ inline size_t merge_layout(int cap, int kb, unsigned char *base, MergeSmem *s) {
    const int tn = merge_tn(cap);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = (off + bytes + 15) & ~size_t(15);
        return base ? base + o : nullptr;
    };
    unsigned char *p;
    p = take(sizeof(double) * cap);           if (s) s->Rv = (double *)p;
    p = take(sizeof(double) * tn);            if (s) s->Nv = (double *)p;
    p = take(sizeof(double) * kb);            if (s) s->Sav = (double *)p;
    p = take(sizeof(double) * kb);            if (s) s->Sbv = (double *)p;
    p = take(sizeof(double) * MERGE_W);       if (s) s->wa = (double *)p;
    p = take(sizeof(int64_t) * MERGE_W);      if (s) s->wbs = (int64_t *)p;
    p = take(sizeof(int64_t) * (MERGE_W + 1)); if (s) s->wscan = (int64_t *)p;
    p = take(sizeof(int32_t) * cap);          if (s) s->Rk = (int32_t *)p;
    p = take(sizeof(int32_t) * tn);           if (s) s->Nk = (int32_t *)p;
    p = take(sizeof(int32_t) * kb);           if (s) s->Sak = (int32_t *)p;
    p = take(sizeof(int32_t) * kb);           if (s) s->Sbk = (int32_t *)p;
    p = take(sizeof(int32_t) * (kb + 1));     if (s) s->pf = (int32_t *)p;
    p = take(sizeof(int32_t) * (MERGE_W + 2)); if (s) s->runoff = (int32_t *)p;
    return off;
}

int merge_smem_bytes(int cap, int batch) { return (int)merge_layout(cap, batch, nullptr, nullptr); }

int merge_max_cap(int batch, int smem_limit) {
    int cap = 256;
    while (merge_smem_bytes(cap + 256, batch) <= smem_limit) cap += 256;
    return cap;
}

// One level of the pairwise merge of `nruns` sorted runs: run r occupies
// [runoff[r], runoff[r+1]) of sk/sv; runs 2p and 2p+1 are merged into the same
// range of dk/dv.  All threads call; ends with a barrier.
template <int NT>
SPG_DEV void merge_level(const int32_t *sk, const double *sv, const int32_t *runoff, int nruns, int n,
                         int32_t *dk, double *dv) {
    const int ipt = (n + NT - 1) / NT;
    int d = threadIdx.x * ipt;
    const int dend = min(n, d + ipt);
    if (d < dend) {
        const int npairs = (nruns + 1) >> 1;
        int lo = 0, hi = npairs - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (runoff[2 * mid] <= d) lo = mid; else hi = mid - 1;
        }
        int p = lo;
        while (d < dend) {
            const int as = runoff[2 * p];
            const int am = runoff[min(2 * p + 1, nruns)];
            const int ae = runoff[min(2 * p + 2, nruns)];
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
SPG_DEV int compress_runs(const int32_t *k, const double *v, int n, int32_t *ok, double *ov,
                          int32_t *scan32) {
    const int ipt = (n + NT - 1) / NT;
    const int q0 = threadIdx.x * ipt;
    const int q1 = min(n, q0 + ipt);
    int cnt = 0;
    for (int q = q0; q < q1; ++q)
        if (q == 0 || k[q] != k[q - 1]) ++cnt;
    int tot;
    int o = block_exclusive_scan<NT>(cnt, scan32, tot);
    for (int q = q0; q < q1; ++q) {
        if (q == 0 || k[q] != k[q - 1]) {
            const int32_t key = k[q];
            double s = v[q];
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
SPG_DEV int64_t union_stream(const int32_t *xk, const double *xv, int64_t nx, const int32_t *yk,
                             const double *yv, int ny, int32_t *zk, double *zv, const MergeSmem &s,
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

template <int NT>
__global__ void __launch_bounds__(NT, 1)
k_merge(StageArgs a, MergeState st, MergeLaunch L, const int64_t *__restrict__ u) {
    extern __shared__ __align__(16) unsigned char merge_smem[];
    __shared__ int64_t scan64[NT / 32 + 1];
    __shared__ int32_t scan32[NT / 32 + 1];
    MergeSmem s;
    const int cap = L.cap;
    const int kb = L.batch;
    const int tn = merge_tn(cap);
    merge_layout(cap, kb, merge_smem, &s);

    const int64_t w = blockIdx.x;
    const int j = L.work ? L.work[w] : (int)w;
    const int row = L.rows37[j];
    const int64_t a0 = a.A.rp[row], a1 = a.A.rp[row + 1];
    int32_t *home_col = st.loc_col[j];
    double *home_val = st.loc_val[j];
    const int64_t home_cap = st.loc_cap[j];
    int rlen = st.len[j];
    int64_t e = a0 + st.ck_entry[j];
    int64_t off = st.ck_off[j];

    // reload the dumped sequence (empty for a fresh row)
    for (int t = threadIdx.x; t < rlen; t += NT) {
        s.Rk[t] = home_col[t];
        s.Rv[t] = home_val[t];
    }
    // where this launch writes the row: its home if large enough, else a fresh slot
    int32_t *dst_col = home_col;
    double *dst_val = home_val;
    int64_t dst_cap = home_cap;
    if (!L.level1 && home_cap < cap && L.pool_col != nullptr) {
        dst_col = L.pool_col + w * L.pool_cap;
        dst_val = L.pool_val + w * L.pool_cap;
        dst_cap = L.pool_cap;
    }
    // level-1 global sequence (ping-pong)
    int32_t *gk[2] = {nullptr, nullptr};
    double *gv[2] = {nullptr, nullptr};
    int gcur = 0;
    int64_t glen = 0;
    if (L.level1) {
        const int64_t go = L.g_off[w], gc = L.g_cap[w];
        gk[0] = L.g_col + go;
        gv[0] = L.g_val + go;
        gk[1] = L.g_col + go + gc;
        gv[1] = L.g_val + go + gc;
    }
    int nlen = 0;
    __syncthreads();

    bool overflow = false;
    while (e < a1 && !overflow) {
        const int nW = (int)min((int64_t)MERGE_W, a1 - e);
        int64_t len = 0;
        if (threadIdx.x < nW) {
            const int64_t idx = e + threadIdx.x;
            const int32_t kk = a.A.col[idx];
            int64_t bs = a.B.rp[kk];
            int64_t bl = a.B.rp[kk + 1] - bs;
            if (threadIdx.x == 0) {
                bs += off;
                bl -= off;
            }
            s.wbs[threadIdx.x] = bs;
            s.wa[threadIdx.x] = a.A.val[idx];
            len = bl;
        }
        int64_t total;
        const int64_t ex = block_exclusive_scan<NT>(len, scan64, total);
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
                    glen = union_stream<NT>(gk[gcur], gv[gcur], glen, s.Rk, s.Rv, rlen, gk[gcur ^ 1],
                                            gv[gcur ^ 1], s, kb, scan32);
                    gcur ^= 1;
                    rlen = 0;
                    avail = cap;
                } else if (avail < (kb >> 2) || avail <= 0) {
                    // checkpoint at product p0 of this window
                    const int t = find_segment_i64(s.wscan, nW, p0);
                    if (threadIdx.x == 0) {
                        st.ck_entry[j] = (e + t) - a0;
                        st.ck_off[j] = (t == 0 ? off : 0) + (p0 - s.wscan[t]);
                    }
                    overflow = true;
                    break;
                }
            }
            const int nb = min(need, avail);
            // (0) expand the batch [p0, p0 + nb) into Sa, one run per B row
            const int tf = find_segment_i64(s.wscan, nW, p0);
            const int tl = find_segment_i64(s.wscan, nW, p0 + nb - 1);
            const int nruns = tl - tf + 1;
            for (int q = threadIdx.x; q < nb; q += NT) {
                const int64_t pos = p0 + q;
                const int t = tf + find_segment_i64(s.wscan + tf, nruns, pos);
                const int64_t bidx = s.wbs[t] + (pos - s.wscan[t]);
                s.Sak[q] = a.B.col[bidx];
                s.Sav[q] = s.wa[t] * a.B.val[bidx];
            }
            for (int r = threadIdx.x; r <= nruns; r += NT)
                s.runoff[r] = (r == 0) ? 0 : (r == nruns ? nb : (int)(s.wscan[tf + r] - p0));
            __syncthreads();
            // (1) fuse products whose column is already in R or N
            const int ipt = (nb + NT - 1) / NT;
            const int q0 = threadIdx.x * ipt;
            unsigned newmask = 0;
            int cntnew = 0;
            for (int k = 0; k < MERGE_MAX_IPT; ++k) {
                const int q = q0 + k;
                if (k < ipt && q < nb) {
                    const int32_t key = s.Sak[q];
                    bool found = false;
                    if (rlen > 0) {
                        const int pos = lower_bound_i32(s.Rk, rlen, key);
                        if (pos < rlen && s.Rk[pos] == key) {
                            atomicAdd(&s.Rv[pos], s.Sav[q]);
                            found = true;
                        }
                    }
                    if (!found && nlen > 0) {
                        const int pos = lower_bound_i32(s.Nk, nlen, key);
                        if (pos < nlen && s.Nk[pos] == key) {
                            atomicAdd(&s.Nv[pos], s.Sav[q]);
                            found = true;
                        }
                    }
                    if (!found) {
                        newmask |= 1u << k;
                        ++cntnew;
                    }
                }
            }
            // (2) compact the misses into Sb, keeping one run per B row
            int nnew;
            int o = block_exclusive_scan<NT>(cntnew, scan32, nnew);
            for (int k = 0; k < MERGE_MAX_IPT; ++k) {
                const int q = q0 + k;
                if (k < ipt && q < nb) {
                    s.pf[q] = o;
                    if (newmask & (1u << k)) {
                        s.Sbk[o] = s.Sak[q];
                        s.Sbv[o] = s.Sav[q];
                        ++o;
                    }
                }
            }
            if (threadIdx.x == 0) s.pf[nb] = nnew;
            __syncthreads();
            for (int r = threadIdx.x; r <= nruns; r += NT) s.runoff[r] = s.pf[s.runoff[r]];
            __syncthreads();
            if (nnew > 0) {
                // (3) pairwise merge-path merges of the runs, then fuse equal columns
                int32_t *ck = s.Sbk, *okk = s.Sak;
                double *cv = s.Sbv, *ovv = s.Sav;
                int nr = nruns;
                while (nr > 1) {
                    merge_level<NT>(ck, cv, s.runoff, nr, nnew, okk, ovv);
                    const int np = (nr + 1) >> 1;
                    int v = 0;
                    if (threadIdx.x <= np) v = (threadIdx.x == np) ? nnew : s.runoff[2 * threadIdx.x];
                    __syncthreads();
                    if (threadIdx.x <= np) s.runoff[threadIdx.x] = v;
                    __syncthreads();
                    nr = np;
                    int32_t *tk = ck; ck = okk; okk = tk;
                    double *tv = cv; cv = ovv; ovv = tv;
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
    double *fin_val;
    int64_t fin_cap;
    if (L.level1) {
        glen = union_stream<NT>(gk[gcur], gv[gcur], glen, s.Rk, s.Rv, rlen, gk[gcur ^ 1], gv[gcur ^ 1], s,
                                kb, scan32);
        gcur ^= 1;
        final_len = glen;
        fin_col = gk[gcur];
        fin_val = gv[gcur];
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
        st.loc_col[j] = fin_col;
        st.loc_val[j] = fin_val;
        st.loc_cap[j] = fin_cap;
        st.len[j] = (int32_t)final_len;
        if (overflow) {
            const int slot = atomicAdd(L.ovf_count, 1);
            L.ovf_list[slot] = j;
        } else {
            st.done[j] = 1;
            a.nnzc[row] = (int32_t)final_len;
        }
    }
}

__global__ void k_level1_caps(const int32_t *rows37, const int32_t *work, int64_t nwork,
                              const int64_t *u, int64_t ncols, int64_t *g_cap) {
    int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nwork) return;
    const int j = work ? work[w] : (int)w;
    int64_t c = u[rows37[j]];
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

cudaError_t launch_level1_sizes(const int32_t *rows37, const int32_t *work, int64_t nwork,
                                const int64_t *u, int64_t ncols, int64_t *g_cap, int64_t *g_off,
                                int64_t *partial, int64_t *total, cudaStream_t st) {
    if (nwork > 0)
        k_level1_caps<<<(unsigned)((nwork + 255) / 256), 256, 0, st>>>(rows37, work, nwork, u, ncols, g_cap);
    return device_exclusive_scan(nwork, LoadCap2{g_cap}, StoreOff{g_off}, partial, total, st);
}

cudaError_t launch_merge(const StageArgs &a, const MergeState &s, const MergeLaunch &L,
                         const int64_t *u, cudaStream_t st) {
    if (L.nwork <= 0) return cudaSuccess;
    // batch >= 32 keeps every loop of the kernel progressing (the level-1 stream takes batch/2 per step)
    if (L.batch > MERGE_NT * MERGE_MAX_IPT || L.batch < 32 || L.batch > L.cap) return cudaErrorInvalidValue;
    const int smem = merge_smem_bytes(L.cap, L.batch);
    cudaError_t e = cudaFuncSetAttribute(k_merge<MERGE_NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_merge<MERGE_NT><<<(unsigned)L.nwork, MERGE_NT, smem, st>>>(a, s, L, u);
    return cudaGetLastError();
}

}  // namespace spg
