// Device-wide exclusive prefix sum by reduce-then-scan: three launches
// (per-tile sums, one-block scan of the tile sums, per-tile scan with offsets).
// No block waits on another block, so nothing here can hang.
#pragma once

#include "common.cuh"

namespace spg {

constexpr int SCAN_NT = 256;
constexpr int SCAN_IPT = 8;
constexpr int SCAN_TILE = SCAN_NT * SCAN_IPT;

// Load: int64 operator()(int64 i) const; valid for 0 <= i < n.
template <typename Load>
__global__ void __launch_bounds__(SCAN_NT) k_scan_reduce(int64_t n, Load load, int64_t *partial) {
    __shared__ int64_t scratch[SCAN_NT / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
        int64_t i = base + k * SCAN_NT + threadIdx.x;
        if (i < n) s += load(i);
    }
    s = block_reduce_sum<SCAN_NT>(s, scratch);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// One block of NT threads scans partial[0..nb) in place (exclusive) and writes
// the grand total to *total.
template <int NT>
__global__ void __launch_bounds__(NT) k_scan_partials(int64_t nb, int64_t *partial, int64_t *total) {
    __shared__ int64_t scratch[NT / 32 + 1];
    int64_t carry = 0;
    for (int64_t base = 0; base < nb; base += NT) {
        int64_t i = base + threadIdx.x;
        int64_t v = (i < nb) ? partial[i] : 0;
        int64_t tot;
        int64_t ex = block_exclusive_scan<NT>(v, scratch, tot);
        if (i < nb) partial[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

// Store: void operator()(int64 i, int64 exclusive_prefix) const.
template <typename Load, typename Store>
__global__ void __launch_bounds__(SCAN_NT) k_scan_down(int64_t n, Load load, const int64_t *partial,
                                                       Store store) {
    __shared__ int64_t tile[SCAN_TILE];
    __shared__ int64_t scratch[SCAN_NT / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
        int64_t i = base + k * SCAN_NT + threadIdx.x;
        tile[k * SCAN_NT + threadIdx.x] = (i < n) ? load(i) : 0;
    }
    __syncthreads();
    int64_t v[SCAN_IPT];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
        v[k] = tile[threadIdx.x * SCAN_IPT + k];
        s += v[k];
    }
    int64_t tot;
    int64_t pre = block_exclusive_scan<SCAN_NT>(s, scratch, tot) + partial[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
        tile[threadIdx.x * SCAN_IPT + k] = pre;
        pre += v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
        int64_t i = base + k * SCAN_NT + threadIdx.x;
        if (i < n) store(i, tile[k * SCAN_NT + threadIdx.x]);
    }
}

inline int64_t scan_blocks(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE; }

// Enqueues the three kernels.  partial must hold scan_blocks(n) int64 (>= 1);
// total receives the sum (device pointer).  n may be 0.
template <typename Load, typename Store>
inline cudaError_t device_exclusive_scan(int64_t n, Load load, Store store, int64_t *partial,
                                         int64_t *total, cudaStream_t st) {
    int64_t nb = scan_blocks(n);
    if (nb > 0) {
        k_scan_reduce<Load><<<(unsigned)nb, SCAN_NT, 0, st>>>(n, load, partial);
    }
    k_scan_partials<1024><<<1, 1024, 0, st>>>(nb, partial, total);
    if (nb > 0) {
        k_scan_down<Load, Store><<<(unsigned)nb, SCAN_NT, 0, st>>>(n, load, partial, store);
    }
    return cudaGetLastError();
}

}  // namespace spg
