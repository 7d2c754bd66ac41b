// Stage 4 (Section 4.1, "arranging data"): the sizes nnz(c_i) are summed by an
// exclusive prefix sum into C.row_ptr (int64), C is allocated by the host, and
// the rows are copied from the temporary matrix C~ into C.  Rows of bin 1 hold a
// single product, which is computed here directly; rows of bin 0 need nothing.
// Bins 2..36 are copied by one warp per row, bin 37 by one CTA per row (all
// column slices of a split row, in column order).
#include "internal.h"
#include "scan.cuh"

namespace spg {

struct LoadNnzc {
    const int32_t *nnzc;
    SPG_DEV int64_t operator()(int64_t i) const { return (int64_t)nnzc[i]; }
};
struct StoreRp {
    int64_t *rp;
    SPG_DEV void operator()(int64_t i, int64_t v) const { rp[i] = v; }
};

cudaError_t launch_row_scan(int64_t m, const int32_t *nnzc, int64_t *c_rp, int64_t *partial,
                            cudaStream_t st) {
    return device_exclusive_scan(m, LoadNnzc{nnzc}, StoreRp{c_rp}, partial, c_rp + m, st);
}

constexpr int ARR_NT = 256;

// A warp per row; the warps stride over the rows (one pass when the grid covers them).
__global__ void __launch_bounds__(ARR_NT)
k_arrange_short(StageArgs a, RowSet R, const uint8_t *__restrict__ bin,
                const int64_t *__restrict__ c_rp, int32_t *__restrict__ c_col, val_t *__restrict__ c_val) {
    if (gated(a.gate)) return;
    const int32_t *rows;
    int64_t nrows;
    rowset_range(R, rows, nrows);
    const int lane = threadIdx.x & 31;
    for (int64_t wg = ((int64_t)blockIdx.x * ARR_NT + threadIdx.x) >> 5; wg < nrows;
         wg += (int64_t)gridDim.x * (ARR_NT / 32)) {
        const int row = rows[wg];
        const int64_t o = c_rp[row];
        if (bin[row] == 1) {
            // exactly one A entry of this row selects a B row of length 1
            const int64_t a0 = a.A.rp[row], a1 = a.A.rp[row + 1];
            for (int64_t base = a0; base < a1; base += 32) {
                const int64_t p = base + lane;
                int64_t b0 = 0;
                bool hit = false;
                if (p < a1) {
                    const int32_t j = a.A.col[p];
                    b0 = a.B.rp[j];
                    hit = (a.B.rp[j + 1] - b0) > 0;
                }
                const unsigned m = __ballot_sync(SPG_FULL, hit);
                if (m) {
                    if (lane == __ffs(m) - 1 && SPG_IN(o < c_rp[row + 1], 103)) {
                        c_col[o] = a.B.col[b0];
                        c_val[o] = a.A.val[p] * a.B.val[b0];
                    }
                    break;
                }
            }
            continue;
        }
        const int64_t n = c_rp[row + 1] - o;
        const int64_t src = a.ctil_rp[row];
        if (!SPG_IN(src + n <= a.ctil_rp[row + 1], 104)) continue;  // C~ holds the row
        for (int64_t t = lane; t < n; t += 32) {
            c_col[o + t] = a.ctil_col[src + t];
            c_val[o + t] = a.ctil_val[src + t];
        }
    }
}

cudaError_t launch_arrange_short(const StageArgs &a, const int32_t *rows, int64_t nrows,
                                 const uint8_t *bin, const int64_t *c_rp, int32_t *c_col,
                                 val_t *c_val, cudaStream_t st) {
    return launch_arrange_short_set(a, host_rows(rows, nrows), bin, c_rp, c_col, c_val, st);
}

cudaError_t launch_arrange_short_set(const StageArgs &a, const RowSet &R, const uint8_t *bin, const int64_t *c_rp,
                                     int32_t *c_col, val_t *c_val, cudaStream_t st) {
    if (R.n <= 0) return cudaSuccess;
    const int64_t need = (R.n * 32 + ARR_NT - 1) / ARR_NT;
    const int64_t grid = R.dev_lo ? persistent_blocks((const void *)k_arrange_short, ARR_NT, 0, need) : need;
    if (grid <= 0) return cudaErrorInvalidValue;
    k_arrange_short<<<(unsigned)grid, ARR_NT, 0, st>>>(a, R, bin, c_rp, c_col, c_val);
    return cudaGetLastError();
}

// One thread: whether C (c_rp[m] entries) fits the cap entries allocated for it.
__global__ void k_gate(const int64_t *c_rp, int64_t m, int64_t cap, int64_t *gate, int64_t *err) {
    const bool over = c_rp[m] > cap;
    *gate = over ? 1 : 0;
    if (over) atomicExch((unsigned long long *)err, 8ull);
}

// A C that does not fit becomes the empty matrix (all row pointers 0), so that nothing
// downstream -- a chained product reading it as its B -- reads beyond its arrays.
__global__ void k_gate_clear(int64_t *c_rp, int64_t m, const int64_t *gate) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= m && *gate != 0) c_rp[i] = 0;
}

cudaError_t launch_gate(int64_t *c_rp, int64_t m, int64_t cap, int64_t *gate, int64_t *err, cudaStream_t st) {
    k_gate<<<1, 1, 0, st>>>(c_rp, m, cap, gate, err);
    k_gate_clear<<<(unsigned)((m + 1 + 255) / 256), 256, 0, st>>>(c_rp, m, gate);
    return cudaGetLastError();
}

// One CTA per bin-37 row: its leaves (column slices) are visited in column order
// (a walk of the split tree, left child first) and copied back to back.
// Rows of the dense-slice kernels are already in C.
__global__ void __launch_bounds__(ARR_NT)
k_arrange_long(MergeItems it, const int64_t *__restrict__ c_rp, int32_t *__restrict__ c_col,
               val_t *__restrict__ c_val) {
    constexpr int LEAF_BUF = 128;
    __shared__ int leaves[LEAF_BUF];
    __shared__ int nleaves, cursor;
    const int j = blockIdx.x;
    if (it.child[j] == ITEM_DENSE) return;  // written into C by the dense-slice kernel
    int64_t o = c_rp[it.row[j]];
    if (threadIdx.x == 0) cursor = split_first_leaf(it, j);
    __syncthreads();
    while (true) {
        if (threadIdx.x == 0) {
            int n = 0, x = cursor;
            while (x >= 0 && n < LEAF_BUF) {
                leaves[n++] = x;
                x = split_next_leaf(it, j, x);
            }
            cursor = x;
            nleaves = n;
        }
        __syncthreads();
        const int nl = nleaves;
        if (nl == 0) break;
        for (int l = 0; l < nl; ++l) {
            const int x = leaves[l];
            const int64_t n = it.len[x];
            const int32_t *sc = it.home_col[x];
            const val_t *sv = it.home_val[x];
            if (!SPG_IN(o + n <= c_rp[it.row[j] + 1], 105)) break;  // the leaves fill the row of C exactly
            for (int64_t t = threadIdx.x; t < n; t += ARR_NT) {
                c_col[o + t] = sc[t];
                c_val[o + t] = sv[t];
            }
            o += n;
        }
        __syncthreads();
    }
}

cudaError_t launch_arrange_long(const MergeItems &it, int64_t n37, const int64_t *c_rp, int32_t *c_col,
                                val_t *c_val, cudaStream_t st) {
    if (n37 <= 0) return cudaSuccess;
    k_arrange_long<<<(unsigned)n37, ARR_NT, 0, st>>>(it, c_rp, c_col, c_val);
    return cudaGetLastError();
}

}  // namespace spg
