// The merge evaluation of Section 4.2 ("Evaluating GPU Merge algorithms"): merging two
// sorted sequences of length l into one of length 2l, many independent groups (the paper
// uses 2^25 elements in all), with 32-bit keys and no value, a 32-bit value or a 64-bit
// value.  Three of the paper's five algorithms, each in shared memory on one CTA per group:
//   ranking merge   every element's output position is its index plus its rank in the other
//                   sequence (a binary search); out of place;
//   merge path      each thread finds where its share of the output starts on the merge
//                   path (a co-rank binary search), then merges its share sequentially;
//   bitonic merge   the last stage of a bitonic sort: the second sequence reversed, then
//                   log2(2l) compare-exchange steps in place.
// Ties: an element of the first sequence precedes an equal one of the second (ranking merge
// and merge path); the bitonic network does not keep that order.
#include "internal.h"
#include "common.cuh"

#include <type_traits>

namespace spg {

template <int VB>
struct MicroVal {
    using T = typename std::conditional<VB == 8, double, uint32_t>::type;
};

// Number of elements of the sorted a[0..n) that are < key (strict) or <= key.
template <bool STRICT>
SPG_DEV int micro_rank(const int32_t *a, int n, int32_t key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const bool before = STRICT ? a[mid] < key : a[mid] <= key;
        if (before) lo = mid + 1; else hi = mid;
    }
    return lo;
}

template <int NT, int VB, int METHOD>
__global__ void __launch_bounds__(NT)
k_merge_micro(const int32_t *__restrict__ keys, const void *__restrict__ vals, int l, int32_t *__restrict__ okeys,
              void *__restrict__ ovals) {
    using V = typename MicroVal<VB>::T;
    extern __shared__ __align__(16) unsigned char mm_smem[];
    const int n = 2 * l;
    int32_t *sk = reinterpret_cast<int32_t *>(mm_smem);
    V *sv = reinterpret_cast<V *>(mm_smem + ((sizeof(int32_t) * n + 15) & ~size_t(15)));
    const int64_t base = (int64_t)blockIdx.x * n;
    const V *gv = reinterpret_cast<const V *>(vals);
    V *ov = reinterpret_cast<V *>(ovals);
    // load the group; the bitonic merge takes the second sequence reversed
    for (int i = threadIdx.x; i < n; i += NT) {
        const int d = (METHOD == 2 && i >= l) ? n - 1 - (i - l) : i;
        sk[d] = keys[base + i];
        if (VB) sv[d] = gv[base + i];
    }
    __syncthreads();
    if (METHOD == 0) {  // ranking merge
        for (int i = threadIdx.x; i < n; i += NT) {
            const int32_t k = sk[i];
            const int pos = i < l ? i + micro_rank<true>(sk + l, l, k) : (i - l) + micro_rank<false>(sk, l, k);
            okeys[base + pos] = k;
            if (VB) ov[base + pos] = sv[i];
        }
    } else if (METHOD == 1) {  // merge path
        const int per = (n + NT - 1) / NT;
        const int d0 = min(n, (int)threadIdx.x * per), d1 = min(n, d0 + per);
        if (d0 < d1) {
            // co-rank: i elements of the first sequence and d0 - i of the second come before output d0
            int lo = max(0, d0 - l), hi = min(d0, l);
            while (lo < hi) {
                const int i = (lo + hi) >> 1;
                if (sk[i] <= sk[l + d0 - i - 1]) lo = i + 1; else hi = i;
            }
            int ia = lo, ib = d0 - lo;
            for (int d = d0; d < d1; ++d) {
                const bool take_a = ib >= l || (ia < l && sk[ia] <= sk[l + ib]);
                const int src = take_a ? ia++ : l + ib++;
                okeys[base + d] = sk[src];
                if (VB) ov[base + d] = sv[src];
            }
        }
    } else {  // bitonic merge of the bitonic sequence a ++ reverse(b)
        for (int stride = l; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < l; t += NT) {
                const int i = 2 * stride * (t / stride) + (t % stride), j = i + stride;
                const int32_t ki = sk[i], kj = sk[j];
                if (ki > kj) {
                    sk[i] = kj;
                    sk[j] = ki;
                    if (VB) {
                        const V vi = sv[i];
                        sv[i] = sv[j];
                        sv[j] = vi;
                    }
                }
            }
            __syncthreads();
        }
        for (int i = threadIdx.x; i < n; i += NT) {
            okeys[base + i] = sk[i];
            if (VB) ov[base + i] = sv[i];
        }
    }
}

int merge_micro_smem(int l, int value_bytes) {
    const size_t kb = ((sizeof(int32_t) * 2 * (size_t)l) + 15) & ~size_t(15);
    return (int)(kb + (size_t)value_bytes * 2 * l);
}

template <int NT, int VB>
static cudaError_t micro_launch(int method, const int32_t *keys, const void *vals, int64_t groups, int l,
                                int32_t *okeys, void *ovals, cudaStream_t st) {
    const int smem = merge_micro_smem(l, VB);
    auto kern = method == 0 ? k_merge_micro<NT, VB, 0> : (method == 1 ? k_merge_micro<NT, VB, 1>
                                                                      : k_merge_micro<NT, VB, 2>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)groups, NT, smem, st>>>(keys, vals, l, okeys, ovals);
    return cudaGetLastError();
}

template <int NT>
static cudaError_t micro_vb(int method, int vb, const int32_t *keys, const void *vals, int64_t groups, int l,
                            int32_t *okeys, void *ovals, cudaStream_t st) {
    if (vb == 0) return micro_launch<NT, 0>(method, keys, vals, groups, l, okeys, ovals, st);
    if (vb == 4) return micro_launch<NT, 4>(method, keys, vals, groups, l, okeys, ovals, st);
    return micro_launch<NT, 8>(method, keys, vals, groups, l, okeys, ovals, st);
}

cudaError_t launch_merge_micro(int method, int threads, int value_bytes, const int32_t *keys, const void *vals,
                               int64_t n, int l, int32_t *okeys, void *ovals, cudaStream_t st) {
    const int64_t groups = n / (2 * (int64_t)l);
    switch (threads) {
        case 64: return micro_vb<64>(method, value_bytes, keys, vals, groups, l, okeys, ovals, st);
        case 128: return micro_vb<128>(method, value_bytes, keys, vals, groups, l, okeys, ovals, st);
        case 256: return micro_vb<256>(method, value_bytes, keys, vals, groups, l, okeys, ovals, st);
        case 512: return micro_vb<512>(method, value_bytes, keys, vals, groups, l, okeys, ovals, st);
        default: return micro_vb<1024>(method, value_bytes, keys, vals, groups, l, okeys, ovals, st);
    }
}

}  // namespace spg
