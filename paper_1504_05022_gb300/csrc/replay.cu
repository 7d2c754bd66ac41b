// Values-only replay of a finished product: C's structure is known (its row
// pointers and columns, and for long rows the column slices of the split tree),
// so recomputing C's values for new values of A and B needs only sub-step (1) of
// the merge method of Section 4.1 -- every product is fused into the already
// known, sorted result sequence, by a bitmap rank when B's columns fit the bitmap
// and by binary search otherwise.  Rows of bins 2..36 are recomputed by
// the heap and bitonic-ESC kernels writing straight into C.  Nothing here
// allocates or synchronises with the host, so a replay can be captured in a CUDA
// graph.
#include "internal.h"
#include "common.cuh"

namespace spg {

constexpr int REPLAY_IPT = 4;

// One CTA per leaf: preload the leaf's known columns with zero values, fuse all
// products of its column range, write the values back into C.
template <int NT>
__global__ void __launch_bounds__(NT, 2048 / NT / 2)
k_replay(StageArgs a, ReplayLeaves lv, const int32_t *__restrict__ order, int32_t *__restrict__ c_col,
         val_t *__restrict__ c_val, int64_t *err) {
    extern __shared__ __align__(16) unsigned char rsmem[];
    __shared__ int64_t scan64[NT / 32 + 1];
    constexpr int W = NT;
    const int q = order[blockIdx.x];
    const int row = lv.row[q];
    const int32_t clo = lv.clo[q], chi = lv.chi[q];
    const bool filtered = (clo > 0) || (chi < INT32_MAX);
    const int64_t coff = lv.c_off[q];
    const int len = lv.len[q];
    if (len > lv.cap) {  // cannot happen for split plans: every leaf fits its class
        if (threadIdx.x == 0) atomicExch((unsigned long long *)err, 4ull);
        return;
    }
    val_t *Rv = reinterpret_cast<val_t *>(rsmem);
    val_t *wa = Rv + lv.cap;
    int64_t *wbs = reinterpret_cast<int64_t *>(wa + W);
    int64_t *wscan = wbs + W;
    int32_t *Rk = reinterpret_cast<int32_t *>(wscan + W + 1);
    for (int t = threadIdx.x; t < len; t += NT) {
        Rk[t] = c_col[coff + t];
        Rv[t] = 0.0;
    }
    bool bad = false;
    const int64_t a0 = a.A.rp[row], a1 = a.A.rp[row + 1];
    for (int64_t e = a0; e < a1; e += W) {
        const int nW = (int)min((int64_t)W, a1 - e);
        int64_t blen = 0;
        if (threadIdx.x < nW) {
            const int64_t idx = e + threadIdx.x;
            const int32_t kk = a.A.col[idx];
            const int64_t rs = a.B.rp[kk];
            int64_t bs = rs, be = a.B.rp[kk + 1];
            if (filtered) {
                const int n = (int)(be - rs);
                if (clo > 0) bs = rs + lower_bound_i32(a.B.col + rs, n, clo);
                if (chi < INT32_MAX) be = rs + lower_bound_i32(a.B.col + rs, n, chi);
            }
            wbs[threadIdx.x] = bs;
            wa[threadIdx.x] = a.A.val[idx];
            blen = be > bs ? be - bs : 0;
        }
        int64_t total;
        const int64_t ex = block_exclusive_scan<NT, int64_t, false>(blen, scan64, total);
        if (threadIdx.x < nW) wscan[threadIdx.x] = ex;
        if (threadIdx.x == 0) wscan[nW] = total;
        __syncthreads();
        for (int64_t p0 = 0; p0 < total; p0 += (int64_t)NT * REPLAY_IPT) {
            const int nb = (int)min((int64_t)NT * REPLAY_IPT, total - p0);
            const int ipt = (nb + NT - 1) / NT;
            const int q0 = threadIdx.x * ipt;
            const int cnt = max(0, min(ipt, nb - q0));
            int32_t key[REPLAY_IPT];
            val_t val[REPLAY_IPT];
            if (cnt > 0) {
                int te[REPLAY_IPT], to[REPLAY_IPT];
                int64_t pos = p0 + q0;
                int t = find_segment_i64(wscan, nW, pos);
#pragma unroll
                for (int k = 0; k < REPLAY_IPT; ++k) {
                    if (k < cnt) {
                        while (t + 1 < nW && wscan[t + 1] <= pos) ++t;
                        te[k] = t;
                        to[k] = (int)(pos - wscan[t]);
                        ++pos;
                    }
                }
#pragma unroll
                for (int k = 0; k < REPLAY_IPT; ++k)
                    if (k < cnt) key[k] = __ldg(a.B.col + wbs[te[k]] + to[k]);
#pragma unroll
                for (int k = 0; k < REPLAY_IPT; ++k)
                    if (k < cnt) val[k] = wa[te[k]] * __ldg(a.B.val + wbs[te[k]] + to[k]);
            }
            int posr[REPLAY_IPT];
            lower_bound_multi<REPLAY_IPT>(Rk, len, key, cnt, posr);
#pragma unroll
            for (int k = 0; k < REPLAY_IPT; ++k) {
                if (k < cnt) {
                    if (posr[k] < len && Rk[posr[k]] == key[k]) atomicAdd(&Rv[posr[k]], val[k]);
                    else bad = true;  // the structure of A or B changed since the product was planned
                }
            }
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < len; t += NT) c_val[coff + t] = Rv[t];
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch((unsigned long long *)err, 3ull);
}

// Bitmap form: the leaf's known columns are entered in a bitmap over its column
// range with a rank directory, so a product finds its position in O(1) (two
// shared loads) instead of a binary search; used when B's columns fit the bitmap.
template <int NT>
__global__ void __launch_bounds__(NT, 2048 / NT / 2)
k_replay_bm(StageArgs a, ReplayLeaves lv, const int32_t *__restrict__ order, int nwords_max,
            int32_t *__restrict__ c_col, val_t *__restrict__ c_val, int64_t *err) {
    extern __shared__ __align__(16) unsigned char rsmem[];
    __shared__ int64_t scan64[NT / 32 + 1];
    __shared__ int32_t scan32[NT / 32 + 1];
    constexpr int W = NT;
    const int q = order[blockIdx.x];
    const int row = lv.row[q];
    const int32_t clo = lv.clo[q], chi = lv.chi[q];
    const bool filtered = (clo > 0) || (chi < INT32_MAX);
    const int32_t lo = clo > 0 ? clo : 0;
    const int64_t hicol = min((int64_t)chi, a.B.ncols);
    const int nwords = hicol > lo ? (int)((hicol - lo + 31) >> 5) : 1;
    const int64_t coff = lv.c_off[q];
    const int len = lv.len[q];
    if (len > lv.cap || nwords > nwords_max) {  // cannot happen: leaves fit their class and the bitmap
        if (threadIdx.x == 0) atomicExch((unsigned long long *)err, 4ull);
        return;
    }
    val_t *Rv = reinterpret_cast<val_t *>(rsmem);
    val_t *wa = Rv + lv.cap;
    int64_t *wbs = reinterpret_cast<int64_t *>(wa + W);
    int64_t *wscan = wbs + W;
    int32_t *Rd = reinterpret_cast<int32_t *>(wscan + W + 1 + 1);  // 16-byte aligned (W is a multiple of 32)
    uint32_t *Bm = reinterpret_cast<uint32_t *>(Rd + ((nwords_max + 4) & ~3));
    for (int t = threadIdx.x; t < nwords; t += NT) Bm[t] = 0u;
    __syncthreads();
    bool bad = false;
    for (int t = threadIdx.x; t < len; t += NT) {
        const int x = c_col[coff + t] - lo;
        Rv[t] = 0.0;
        if ((unsigned)x < (unsigned)(nwords << 5)) atomicOr(&Bm[x >> 5], 1u << (x & 31));
        else bad = true;
    }
    __syncthreads();
    bitmap_rank<NT>(Bm, Rd, nwords, scan32);
    const int64_t a0 = a.A.rp[row], a1 = a.A.rp[row + 1];
    for (int64_t e = a0; e < a1; e += W) {
        const int nW = (int)min((int64_t)W, a1 - e);
        int64_t blen = 0;
        if (threadIdx.x < nW) {
            const int64_t idx = e + threadIdx.x;
            const int32_t kk = a.A.col[idx];
            const int64_t rs = a.B.rp[kk];
            int64_t bs = rs, be = a.B.rp[kk + 1];
            if (filtered) {
                const int n = (int)(be - rs);
                if (clo > 0) bs = rs + lower_bound_i32(a.B.col + rs, n, clo);
                if (chi < INT32_MAX) be = rs + lower_bound_i32(a.B.col + rs, n, chi);
            }
            wbs[threadIdx.x] = bs;
            wa[threadIdx.x] = a.A.val[idx];
            blen = be > bs ? be - bs : 0;
        }
        int64_t total;
        const int64_t ex = block_exclusive_scan<NT, int64_t, false>(blen, scan64, total);
        if (threadIdx.x < nW) wscan[threadIdx.x] = ex;
        if (threadIdx.x == 0) wscan[nW] = total;
        __syncthreads();
        for (int64_t p0 = 0; p0 < total; p0 += (int64_t)NT * REPLAY_IPT) {
            const int nb = (int)min((int64_t)NT * REPLAY_IPT, total - p0);
            const int tf = find_segment_i64(wscan, nW, p0);
            const int tl = find_segment_i64(wscan, nW, p0 + nb - 1);
            // products threadIdx.x + k*NT: consecutive lanes read consecutive B entries
            const int cnt = nb > (int)threadIdx.x ? min(REPLAY_IPT, (nb - (int)threadIdx.x + NT - 1) / NT) : 0;
            if (cnt > 0) {
                int te[REPLAY_IPT], to[REPLAY_IPT];
                int32_t key[REPLAY_IPT];
                val_t val[REPLAY_IPT];
#pragma unroll
                for (int k = 0; k < REPLAY_IPT; ++k) {
                    if (k < cnt) {
                        const int64_t pos = p0 + threadIdx.x + k * NT;
                        const int t = tf + find_segment_i64(wscan + tf, tl - tf + 1, pos);
                        te[k] = t;
                        to[k] = (int)(pos - wscan[t]);
                    }
                }
#pragma unroll
                for (int k = 0; k < REPLAY_IPT; ++k)
                    if (k < cnt) key[k] = __ldg(a.B.col + wbs[te[k]] + to[k]);
#pragma unroll
                for (int k = 0; k < REPLAY_IPT; ++k)
                    if (k < cnt) val[k] = wa[te[k]] * __ldg(a.B.val + wbs[te[k]] + to[k]);
#pragma unroll
                for (int k = 0; k < REPLAY_IPT; ++k) {
                    if (k < cnt) {
                        const int x = key[k] - lo;
                        if ((unsigned)x < (unsigned)(nwords << 5) && ((Bm[x >> 5] >> (x & 31)) & 1u))
                            atomicAdd(&Rv[bitmap_pos(Bm, Rd, x)], val[k]);
                        else
                            bad = true;  // the structure of A or B changed since the product was planned
                    }
                }
            }
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < len; t += NT) c_val[coff + t] = Rv[t];
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch((unsigned long long *)err, 3ull);
}

int replay_threads(int cap) { return cap <= 1024 ? 128 : (cap <= 4096 ? 256 : 512); }

int replay_bm_smem_bytes(int cap, int nwords_max) {
    const int W = replay_threads(cap);
    return (int)(sizeof(val_t) * (cap + W) + sizeof(int64_t) * (2 * W + 2) +
                 sizeof(int32_t) * ((nwords_max + 4) & ~3) + sizeof(uint32_t) * nwords_max + 64);
}

int replay_smem_bytes(int cap) {
    const int W = replay_threads(cap);
    return (int)(sizeof(val_t) * (cap + W) + sizeof(int64_t) * (2 * W + 1) + sizeof(int32_t) * cap + 64);
}

template <int NT>
static cudaError_t launch_replay_nt(const StageArgs &a, const ReplayLeaves &lv, const int32_t *order, int64_t n,
                                   int32_t *c_col, val_t *c_val, int64_t *err, int smem, cudaStream_t st) {
    auto kern = k_replay<NT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)n, NT, smem, st>>>(a, lv, order, c_col, c_val, err);
    return cudaGetLastError();
}

template <int NT>
static cudaError_t launch_replay_bm_nt(const StageArgs &a, const ReplayLeaves &lv, const int32_t *order, int64_t n,
                                      int nwords, int32_t *c_col, val_t *c_val, int64_t *err, int smem,
                                      cudaStream_t st) {
    auto kern = k_replay_bm<NT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)n, NT, smem, st>>>(a, lv, order, nwords, c_col, c_val, err);
    return cudaGetLastError();
}

cudaError_t launch_replay(const StageArgs &a, ReplayLeaves lv, const int32_t *order, int64_t n, int cap,
                          int32_t *c_col, val_t *c_val, int64_t *err, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    lv.cap = cap;
    if (a.B.ncols > 0 && a.B.ncols <= BM_MAX_COLS) {
        const int nwords = (int)((a.B.ncols + 31) / 32);
        const int smem = replay_bm_smem_bytes(cap, nwords);
        int optin = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (smem <= optin) {
            switch (replay_threads(cap)) {
                case 128: return launch_replay_bm_nt<128>(a, lv, order, n, nwords, c_col, c_val, err, smem, st);
                case 256: return launch_replay_bm_nt<256>(a, lv, order, n, nwords, c_col, c_val, err, smem, st);
                default: return launch_replay_bm_nt<512>(a, lv, order, n, nwords, c_col, c_val, err, smem, st);
            }
        }
    }
    const int smem = replay_smem_bytes(cap);
    switch (replay_threads(cap)) {
        case 128: return launch_replay_nt<128>(a, lv, order, n, c_col, c_val, err, smem, st);
        case 256: return launch_replay_nt<256>(a, lv, order, n, c_col, c_val, err, smem, st);
        default: return launch_replay_nt<512>(a, lv, order, n, c_col, c_val, err, smem, st);
    }
}

// ---- leaf table: the column slices of every bin-37 row, with their offsets in C ----

template <bool SCATTER>
__global__ void k_replay_leaves(int64_t n37, MergeItems it, const int64_t *c_rp, const int32_t *class_cap,
                                int ncls, int32_t *count, const int32_t *start, int32_t *cursor, ReplayLeaves lv,
                                int32_t *order, int64_t *err) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n37) return;
    int64_t off = c_rp[it.row[j]];
    for (int x = split_first_leaf(it, (int)j); x >= 0; x = split_next_leaf(it, (int)j, x)) {
        if (it.child[x] == ITEM_DENSE) continue;  // replayed by the dense-slice kernel
        const int len = it.len[x];
        int g = ncls - 1;
        for (int k = 0; k < ncls; ++k)
            if (len <= class_cap[k]) {
                g = k;
                break;
            }
        if (!SCATTER) {
            atomicAdd(&count[g], 1);
        } else {
            const int slot = start[g] + atomicAdd(&cursor[g], 1);
            lv.row[slot] = it.row[x];
            lv.clo[slot] = it.clo[x];
            lv.chi[slot] = it.chi[x];
            lv.c_off[slot] = off;
            lv.len[slot] = len;
            order[slot] = slot;
        }
        off += len;
    }
}

cudaError_t launch_replay_leaves(int64_t n37, const MergeItems &it, const int64_t *c_rp, const int32_t *class_cap,
                                 int ncls, int32_t *count, int32_t *start, int32_t *cursor, const ReplayLeaves &lv,
                                 int32_t *order, int64_t *err, bool scatter, cudaStream_t st) {
    if (n37 <= 0) return cudaSuccess;
    const unsigned g = (unsigned)((n37 + 127) / 128);
    if (scatter)
        k_replay_leaves<true><<<g, 128, 0, st>>>(n37, it, c_rp, class_cap, ncls, count, start, cursor, lv, order, err);
    else
        k_replay_leaves<false><<<g, 128, 0, st>>>(n37, it, c_rp, class_cap, ncls, count, start, cursor, lv, order,
                                                  err);
    return cudaGetLastError();
}

}  // namespace spg
