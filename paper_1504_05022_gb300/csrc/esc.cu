// Stage 3, bin group 4 (u_i = 33..512): the bitonic ESC method of Section 4.1
// (expand, sort, compress).  With N = 32 it also serves rows of the heap bins
// (u_i <= 32) when the heap kernel is limited to shorter rows (heap_max_u).
//
// One warp per row.  The warp expands the row's u_i products into a per-warp
// shared-memory array padded to N = 32*E entries (64, 128, 256 or 512, the bin's
// upper edge) with the sentinel column INT_MAX, loads E consecutive entries per
// lane into registers, and sorts the N entries with a bitonic network: element
// i = lane*E + e, so compare-exchange distances below E stay inside a thread
// and larger ones are one __shfl_xor_sync per key and value.  Compression is a
// segmented inclusive scan over equal columns (in registers, then across lanes
// with shuffles); the last entry of each run carries the run's sum and is
// written to C~ at the position given by a warp scan of run ends.
#include "internal.h"
#include "common.cuh"

namespace spg {

constexpr int ESC_WARPS = 4;

// COUNT: the counting pass of the precise method (Section 3.1): the same expansion and sort
// on the columns alone, and nnz(c_i) = the number of distinct columns, written to a.nnzc.
// The warps stride over the rows (one pass when the grid covers them).
template <int E, bool COUNT>
__global__ void __launch_bounds__(ESC_WARPS * 32)
k_esc(StageArgs a, RowSet R) {
    constexpr int N = 32 * E;
    __shared__ int32_t sk[ESC_WARPS][N];
    __shared__ val_t sv[ESC_WARPS][COUNT ? 1 : N];
    __shared__ int64_t sbs[ESC_WARPS][32];
    __shared__ int32_t soff[ESC_WARPS][33];
    __shared__ val_t sa[ESC_WARPS][32];
    const int lane = lane_id(), w = warp_id();
    if (!COUNT && gated(a.gate)) return;
    const int32_t *rows;
    int64_t nrows;
    rowset_range(R, rows, nrows);
    int32_t *wk = sk[w];
    val_t *wv = sv[w];
    for (int64_t t = (int64_t)blockIdx.x * ESC_WARPS + w; t < nrows; t += (int64_t)gridDim.x * ESC_WARPS) {
        const int row = rows[t];  // the whole warp takes the same rows

        // ---- expand ----
        int filled = 0;
        const int64_t a0 = a.A.rp[row], a1 = a.A.rp[row + 1];
        for (int64_t base = a0; base < a1; base += 32) {
            const int64_t p = base + lane;
            int32_t len = 0;
            int64_t bs = 0;
            val_t av = 0.0;
            if (p < a1) {
                const int32_t j = a.A.col[p];
                bs = a.B.rp[j];
                len = (int32_t)(a.B.rp[j + 1] - bs);
                if (!COUNT) av = a.A.val[p];
            }
            const int32_t inc = warp_inclusive_scan(len);
            sbs[w][lane] = bs;
            sa[w][lane] = av;
            soff[w][lane] = inc - len;
            if (lane == 31) soff[w][32] = inc;
            __syncwarp();
            const int total = soff[w][32];
            for (int pos = lane; pos < total; pos += 32) {
                const int e = find_segment_i32(soff[w], 32, pos);
                const int64_t q = sbs[w][e] + (pos - soff[w][e]);
                const int dst = filled + pos;
                if (dst < N) {
                    wk[dst] = a.B.col[q];
                    if (!COUNT) wv[dst] = sa[w][e] * a.B.val[q];
                }
            }
            filled += total;
            __syncwarp();
        }
        for (int pos = filled + lane; pos < N; pos += 32) {
            wk[pos] = KEY_PAD;
            if (!COUNT) wv[pos] = 0.0;
        }
        __syncwarp();

        int32_t key[E];
        val_t val[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            key[e] = wk[lane * E + e];
            val[e] = COUNT ? val_t(0) : wv[lane * E + e];
        }
        __syncwarp();  // the next row's expansion reuses the warp's arrays

        // ---- bitonic sort, ascending on i = lane*E + e ----
#pragma unroll
        for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                if (j >= E) {
                    const int lj = j / E;
                    const bool lower = (lane & lj) == 0;
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int32_t pk = __shfl_xor_sync(SPG_FULL, key[e], lj);
                        const val_t pv = COUNT ? val_t(0) : __shfl_xor_sync(SPG_FULL, val[e], lj);
                        const bool up = ((lane * E + e) & k) == 0;
                        const bool take = (lower == up) ? (pk < key[e]) : (pk > key[e]);
                        if (take) {
                            key[e] = pk;
                            if (!COUNT) val[e] = pv;
                        }
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        if ((e & j) == 0) {
                            const int e2 = e | j;
                            const bool up = ((lane * E + e) & k) == 0;
                            const bool sw = up ? (key[e] > key[e2]) : (key[e] < key[e2]);
                            if (sw) {
                                const int32_t tk = key[e];
                                key[e] = key[e2];
                                key[e2] = tk;
                                if (!COUNT) {
                                    const val_t tv = val[e];
                                    val[e] = val[e2];
                                    val[e2] = tv;
                                }
                            }
                        }
                    }
                }
            }
        }

        if constexpr (COUNT) {
            // distinct columns: entries that differ from their predecessor (the pad excluded)
            const int32_t prev_last_c = __shfl_up_sync(SPG_FULL, key[E - 1], 1);
            int cnt = 0;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int32_t pk = e > 0 ? key[e - 1] : (lane > 0 ? prev_last_c : -1);
                cnt += (key[e] != KEY_PAD && key[e] != pk) ? 1 : 0;
            }
            cnt = warp_reduce_sum(cnt);
            if (lane == 0) a.nnzc[row] = cnt;
        } else {
            // ---- compress: segmented sums over runs of equal columns ----
#pragma unroll
            for (int e = 1; e < E; ++e)
                if (key[e] == key[e - 1]) val[e] += val[e - 1];
            const int32_t first = key[0], last = key[E - 1];
            int32_t prev_last = __shfl_up_sync(SPG_FULL, last, 1);
            const bool cont = (lane > 0) && (prev_last == first);
            // R = running sum of the run that ends this lane; flag = a run starts in this lane
            val_t R = val[E - 1];
            bool f = !((first == last) && cont);
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const val_t Rn = __shfl_up_sync(SPG_FULL, R, d);
                const bool fn = __shfl_up_sync(SPG_FULL, (int)f, d) != 0;
                if (lane >= d && !f) {
                    R += Rn;
                    f = fn;
                }
            }
            const val_t carry = __shfl_up_sync(SPG_FULL, R, 1);
            if (cont) {
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if (key[e] == first) val[e] += carry;
            }
            int32_t next_first = __shfl_down_sync(SPG_FULL, first, 1);
            if (lane == 31) next_first = KEY_PAD;  // nothing follows; the pad never ends a run
            int cnt = 0;
            unsigned tails = 0;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int32_t nk = (e + 1 < E) ? key[e + 1] : next_first;
                const bool tail = (key[e] != KEY_PAD) && (key[e] != nk || (e == E - 1 && lane == 31));
                if (tail) {
                    tails |= 1u << e;
                    ++cnt;
                }
            }
            const int inc = warp_inclusive_scan(cnt);
            const int total = __shfl_sync(SPG_FULL, inc, 31);
            int o = inc - cnt;
            const int64_t base = a.ctil_rp[row];
            if (!SPG_IN(base + total <= a.ctil_rp[row + 1], 102)) tails = 0;  // the row's space in C~ (or C)
#pragma unroll
            for (int e = 0; e < E; ++e) {
                if (tails & (1u << e)) {
                    a.ctil_col[base + o] = key[e];
                    a.ctil_val[base + o] = val[e];
                    ++o;
                }
            }
            if (lane == 0) a.nnzc[row] = total;
        }
    }
}

cudaError_t launch_esc(const StageArgs &a, const int32_t *rows, int64_t nrows, int bin,
                       cudaStream_t st) {
    return launch_esc_set(a, host_rows(rows, nrows), bin, false, st);
}

template <int E, bool COUNT>
static cudaError_t esc_go(const StageArgs &a, const RowSet &R, cudaStream_t st) {
    const int64_t need = (R.n + ESC_WARPS - 1) / ESC_WARPS;
    const int64_t grid = R.dev_lo ? persistent_blocks((const void *)k_esc<E, COUNT>, ESC_WARPS * 32, 0, need) : need;
    if (grid <= 0) return cudaErrorInvalidValue;
    k_esc<E, COUNT><<<(unsigned)grid, ESC_WARPS * 32, 0, st>>>(a, R);
    return cudaGetLastError();
}

cudaError_t launch_esc_set(const StageArgs &a, const RowSet &R, int bin, bool count_only, cudaStream_t st) {
    if (R.n <= 0) return cudaSuccess;
    switch (bin) {
        case 32: return count_only ? esc_go<1, true>(a, R, st) : esc_go<1, false>(a, R, st);  // u <= 32
        case 33: return count_only ? esc_go<2, true>(a, R, st) : esc_go<2, false>(a, R, st);
        case 34: return count_only ? esc_go<4, true>(a, R, st) : esc_go<4, false>(a, R, st);
        case 35: return count_only ? esc_go<8, true>(a, R, st) : esc_go<8, false>(a, R, st);
        case 36: return count_only ? esc_go<16, true>(a, R, st) : esc_go<16, false>(a, R, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace spg
