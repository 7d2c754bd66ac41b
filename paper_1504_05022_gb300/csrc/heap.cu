// Stage 3, bin group 3 (u_i = 2..32): the heap method of Section 4.1.
//
// One thread per row.  The thread collects all u_i candidate products of its
// row into an implicit max-heap (keyed by column) in shared memory, then runs
// a heapsort-like delete-max loop.  The sorted, duplicate-free result grows
// downwards in the tail of the same array: a popped root whose column equals
// the first entry of the result is fused into it (values added), otherwise it
// is prepended.  Heap slot s of thread t lives at [s * NT + t], so the threads of
// a warp touch 32 consecutive words and never conflict on a bank.
#include "internal.h"
#include "common.cuh"

namespace spg {

// The grid strides over the rows: one pass when it covers them (rows known on the host),
// several when it is a persistent grid over a range read on the device.
template <int NT>
__global__ void __launch_bounds__(NT)
k_heap(StageArgs a, RowSet R, int slots) {
    extern __shared__ val_t heap_smem[];
    val_t *hv = heap_smem;
    int32_t *hk = reinterpret_cast<int32_t *>(heap_smem + (size_t)slots * NT);
    if (gated(a.gate)) return;
    const int32_t *rows;
    int64_t nrows;
    rowset_range(R, rows, nrows);
#define HK(s) hk[(s) * NT + threadIdx.x]
#define HV(s) hv[(s) * NT + threadIdx.x]
    for (int64_t t = (int64_t)blockIdx.x * NT + threadIdx.x; t < nrows; t += (int64_t)gridDim.x * NT) {
        const int row = rows[t];
        // collect the candidate entries a_ij * b_jk (the expansion of Algorithm 1)
        int n = 0;
        const int64_t a0 = a.A.rp[row], a1 = a.A.rp[row + 1];
        for (int64_t p = a0; p < a1; ++p) {
            const int32_t j = a.A.col[p];
            const val_t av = a.A.val[p];
            const int64_t b0 = a.B.rp[j], b1 = a.B.rp[j + 1];
            for (int64_t q = b0; q < b1 && n < slots; ++q) {
                HK(n) = a.B.col[q];
                HV(n) = av * a.B.val[q];
                ++n;
            }
        }
        // heapify (max-heap on the column index)
        for (int s = n / 2 - 1; s >= 0; --s) {
            int c = s;
            const int32_t k = HK(c);
            const val_t v = HV(c);
            while (true) {
                int l = 2 * c + 1;
                if (l >= n) break;
                int r = l + 1;
                int m = (r < n && HK(r) > HK(l)) ? r : l;
                if (HK(m) <= k) break;
                HK(c) = HK(m);
                HV(c) = HV(m);
                c = m;
            }
            HK(c) = k;
            HV(c) = v;
        }
        // delete-max with duplicate fusion; the result occupies [rs, n) ascending
        int hn = n, rs = n;
        while (hn > 0) {
            const int32_t key = HK(0);
            const val_t val = HV(0);
            --hn;
            if (hn > 0) {
                const int32_t k = HK(hn);
                const val_t v = HV(hn);
                int c = 0;
                while (true) {
                    int l = 2 * c + 1;
                    if (l >= hn) break;
                    int r = l + 1;
                    int m = (r < hn && HK(r) > HK(l)) ? r : l;
                    if (HK(m) <= k) break;
                    HK(c) = HK(m);
                    HV(c) = HV(m);
                    c = m;
                }
                HK(c) = k;
                HV(c) = v;
            }
            if (rs < n && HK(rs) == key) {
                HV(rs) += val;
            } else {
                --rs;
                HK(rs) = key;
                HV(rs) = val;
            }
        }
        const int cnt = n - rs;
        const int64_t o = a.ctil_rp[row];
        if (!SPG_IN(o + cnt <= a.ctil_rp[row + 1], 101)) continue;  // the row's space in C~ (or C)
        for (int r = 0; r < cnt; ++r) {
            a.ctil_col[o + r] = HK(rs + r);
            a.ctil_val[o + r] = HV(rs + r);
        }
        a.nnzc[row] = cnt;
    }
#undef HK
#undef HV
}

cudaError_t launch_heap(const StageArgs &a, const int32_t *rows, int64_t nrows, int slots, int nt,
                        cudaStream_t st) {
    return launch_heap_set(a, host_rows(rows, nrows), slots, nt, st);
}

cudaError_t launch_heap_set(const StageArgs &a, const RowSet &R, int slots, int nt, cudaStream_t st) {
    if (R.n <= 0) return cudaSuccess;
    const size_t smem = (size_t)slots * nt * (sizeof(val_t) + sizeof(int32_t));
    const int64_t need = (R.n + nt - 1) / nt;
    auto go = [&](auto kern) -> cudaError_t {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        const int64_t grid = R.dev_lo ? persistent_blocks((const void *)kern, nt, smem, need) : need;
        if (grid <= 0) return cudaErrorInvalidValue;
        kern<<<(unsigned)grid, nt, smem, st>>>(a, R, slots);
        return cudaGetLastError();
    };
    switch (nt) {
        case 64: return go(k_heap<64>);
        case 128: return go(k_heap<128>);
        case 256: return go(k_heap<256>);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace spg
