// Stage 1 (upper bound, Algorithm 2) and stage 2 (binning and C~ sizing,
// Algorithm 3) of the SpGEMM framework, plus input widening and validation.
//
// Stage 1 is computed as one exclusive prefix sum S over the nonzeros of A of
// the lengths of the B rows they select: u_i = S[A.rp[i+1]] - S[A.rp[i]].  Every
// nonzero costs the same work, so a hub row of A cannot unbalance the kernel the
// way one-thread-per-row (the paper's launch shape) would.
//
// Stage 2 runs on the GPU instead of a CPU core (the paper's choice, Section 4.1)
// and without atomics: per-block 38-bin histograms built with warp match/popc,
// one scan over the (bin, block) counts, and a stable scatter that keeps rows
// in ascending order inside every bin.
#include "internal.h"
#include "scan.cuh"

#include <mutex>
#include <vector>

namespace spg {

int persistent_blocks(const void *kern, int nt, size_t smem, int64_t cap) {
    static std::mutex mu;
    static std::vector<int> sms;  // SM count per device
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    int nsm = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        if ((int)sms.size() <= dev) sms.resize(dev + 1, 0);
        if (sms[dev] == 0 && cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return 0;
        nsm = sms[dev];
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int64_t g = (int64_t)nsm * per_sm;
    return (int)(cap > 0 && cap < g ? cap : g);
}

__global__ void k_widen_rowptr(const int32_t *in, int64_t *out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int64_t)in[i];
}

cudaError_t launch_widen_rowptr(const int32_t *in, int64_t *out, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_widen_rowptr<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, out, n);
    return cudaGetLastError();
}

// One warp per row: row_ptr monotone and within [0, nnz], columns in range and
// strictly ascending.  Writes 1 into *status on the first violation found.
__global__ void k_validate(DevCSR M, int64_t *status) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w > M.nrows) return;
    if (w == M.nrows) {
        if (lane == 0 && (M.rp[0] != 0 || M.rp[M.nrows] != M.nnz)) *status = 1;
        return;
    }
    const int64_t s = M.rp[w], e = M.rp[w + 1];
    bool bad = (s > e) || (s < 0) || (e > M.nnz);
    if (!bad) {
        for (int64_t p = s + lane; p < e; p += 32) {
            int32_t c = M.col[p];
            if (c < 0 || c >= M.ncols) bad = true;
            if (p + 1 < e && M.col[p + 1] <= c) bad = true;
        }
    }
    if (__any_sync(SPG_FULL, bad) && lane == 0) *status = 1;
}

cudaError_t launch_validate(const DevCSR &M, int64_t *status, cudaStream_t st) {
    int64_t warps = M.nrows + 1;
    int64_t threads = warps * 32;
    k_validate<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(M, status);
    return cudaGetLastError();
}

// ---------------- stage 1 ----------------

struct BRowLen {
    const int32_t *acol;
    const int64_t *brp;
    SPG_DEV int64_t operator()(int64_t j) const {
        int32_t k = acol[j];
        return brp[k + 1] - brp[k];
    }
};

struct StoreI64 {
    int64_t *out;
    SPG_DEV void operator()(int64_t i, int64_t v) const { out[i] = v; }
};

int64_t bound_partial_size(int64_t nnzA) { return scan_blocks(nnzA) + 1; }

cudaError_t launch_bound(const DevCSR &A, const DevCSR &B, int64_t *S, int64_t *partial,
                         cudaStream_t st) {
    return device_exclusive_scan(A.nnz, BRowLen{A.col, B.rp}, StoreI64{S}, partial, S + A.nnz, st);
}

// ---------------- stage 2 ----------------

constexpr int BIN_NT = 256;
constexpr int BIN_IPT = 4;
constexpr int BIN_ROWS = BIN_NT * BIN_IPT;
constexpr int BIN_NW = BIN_NT / 32;

int64_t bin_blocks(int64_t m) { return (m + BIN_ROWS - 1) / BIN_ROWS; }

// Algorithm 3: bin 0 (u = 0), bin 1 (u = 1), bins 2..32 (u = 2..32, one bin per
// size), bins 33..36 (33-64, 65-128, 129-256, 257-512), bin 37 (u > 512).
SPG_DEV int bin_of(int64_t u) {
    if (u <= 32) return (int)u;
    if (u <= 64) return 33;
    if (u <= 128) return 34;
    if (u <= 256) return 35;
    if (u <= 512) return 36;
    return 37;
}

// Size of row i in C~.  Hybrid (Algorithm 3): u_i for bins 0..36, a fixed
// initial size (256) for bin 37.  Upper bound: u_i.  Learned: u_i for bins
// 0..36, the predicted size (never above u_i) for bin 37.  Bin-37 rows computed
// by the dense-slice kernels take none in every policy, and the precise method
// has no C~ at all.
SPG_DEV int64_t cap_of(int64_t u, int b, int64_t i, const CapPolicy &P) {
    if (P.policy == POLICY_PRECISE) return 0;  // counted first, then computed straight into C
    if (b == BIN_MERGE && P.dense != nullptr && P.dense[i]) return 0;  // written straight into C
    if (P.policy == POLICY_UPPER_BOUND) return u;
    if (P.policy == POLICY_LEARNED && P.pred_cap != nullptr && b == BIN_MERGE) {
        int64_t c = P.pred_cap[i];
        if (c > P.cap_max) c = P.cap_max;  // longer rows are split into column slices anyway
        return c < u ? (c < 1 ? 1 : c) : u;
    }
    if (b == BIN_MERGE) return P.initial_cap < u ? P.initial_cap : u;
    return u;
}

__global__ void __launch_bounds__(BIN_NT)
k_bin_count(int64_t m, const int64_t *arp, const int64_t *S, CapPolicy P, int64_t *u_out,
            uint8_t *bin_out, int32_t *nnzc, int32_t *hist, int64_t *cap_partial, int64_t nblk) {
    __shared__ int32_t whist[BIN_NW][NUM_BINS];
    __shared__ int64_t scratch[BIN_NW + 1];
    const int lane = lane_id(), wid = warp_id();
    for (int t = threadIdx.x; t < BIN_NW * NUM_BINS; t += BIN_NT) (&whist[0][0])[t] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * BIN_ROWS;
    int64_t capsum = 0;
#pragma unroll
    for (int k = 0; k < BIN_IPT; ++k) {
        const int64_t i = base + k * BIN_NT + threadIdx.x;
        const bool valid = i < m;
        int b = 255;
        if (valid) {
            int64_t u = S[arp[i + 1]] - S[arp[i]];
            b = bin_of(u);
            u_out[i] = u;
            bin_out[i] = (uint8_t)b;
            nnzc[i] = (b <= 1) ? (int32_t)u : 0;
            capsum += cap_of(u, b, i, P);
        }
        unsigned peers = __match_any_sync(SPG_FULL, b);
        if (valid && lane == __ffs(peers) - 1) whist[wid][b] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x < NUM_BINS) {
        int32_t h = 0;
#pragma unroll
        for (int w = 0; w < BIN_NW; ++w) h += whist[w][threadIdx.x];
        hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = h;
    }
    capsum = block_reduce_sum<BIN_NT>(capsum, scratch);
    if (threadIdx.x == 0) cap_partial[blockIdx.x] = capsum;
}

// One block: exclusive scan of the bin-major (bin, block) histogram and of the
// per-block C~ sizes; writes the host summary and C~.rp[m].
__global__ void __launch_bounds__(1024)
k_bin_scan(int64_t m, int32_t *hist, int64_t nblk, int64_t *cap_partial, int64_t *ctil_rp,
           const int64_t *sum_u, BinSummary *summary) {
    __shared__ int64_t scratch[1024 / 32 + 1];
    __shared__ int64_t bstart[NUM_BINS + 1];
    const int64_t nh = (int64_t)NUM_BINS * nblk;
    int64_t carry = 0;
    for (int64_t base = 0; base < nh; base += 1024) {
        int64_t i = base + threadIdx.x;
        int64_t v = (i < nh) ? hist[i] : 0;
        int64_t tot;
        int64_t ex = block_exclusive_scan<1024>(v, scratch, tot);
        if (i < nh) {
            hist[i] = (int32_t)(carry + ex);
            if (i % nblk == 0) bstart[i / nblk] = carry + ex;
        }
        carry += tot;
    }
    carry = 0;
    for (int64_t base = 0; base < nblk; base += 1024) {
        int64_t i = base + threadIdx.x;
        int64_t v = (i < nblk) ? cap_partial[i] : 0;
        int64_t tot;
        int64_t ex = block_exclusive_scan<1024>(v, scratch, tot);
        if (i < nblk) cap_partial[i] = carry + ex;
        carry += tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bstart[NUM_BINS] = m;
        if (nblk == 0)
            for (int b = 0; b < NUM_BINS; ++b) bstart[b] = 0;
        ctil_rp[m] = carry;
        summary->sum_cap = carry;
        summary->sum_u = *sum_u;
    }
    __syncthreads();
    if (threadIdx.x < NUM_BINS) summary->bin_count[threadIdx.x] = bstart[threadIdx.x + 1] - bstart[threadIdx.x];
    if (threadIdx.x <= NUM_BINS) summary->bin_start[threadIdx.x] = bstart[threadIdx.x];
}

__global__ void __launch_bounds__(BIN_NT)
k_bin_scatter(int64_t m, const int64_t *u_in, const uint8_t *bin_in, CapPolicy P,
              const int32_t *hist_off, const int64_t *cap_off, int64_t nblk, int32_t *bin_rows,
              int64_t *ctil_rp) {
    __shared__ int32_t wcnt[BIN_NW][NUM_BINS];
    __shared__ int32_t run[NUM_BINS];
    __shared__ int64_t scratch[BIN_NW + 1];
    const int lane = lane_id(), wid = warp_id();
    if (threadIdx.x < NUM_BINS) run[threadIdx.x] = 0;
    const int64_t base = (int64_t)blockIdx.x * BIN_ROWS;
    int64_t capcarry = cap_off[blockIdx.x];
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int k = 0; k < BIN_IPT; ++k) {
        for (int t = threadIdx.x; t < BIN_NW * NUM_BINS; t += BIN_NT) (&wcnt[0][0])[t] = 0;
        __syncthreads();
        const int64_t i = base + k * BIN_NT + threadIdx.x;
        const bool valid = i < m;
        int b = valid ? (int)bin_in[i] : 255;
        unsigned peers = __match_any_sync(SPG_FULL, b);
        int rank = __popc(peers & lt_mask);
        if (valid && lane == __ffs(peers) - 1) wcnt[wid][b] = __popc(peers);
        __syncthreads();
        int64_t cap = 0;
        if (valid) {
            int pos = run[b] + rank;
            for (int w = 0; w < wid; ++w) pos += wcnt[w][b];
            bin_rows[(int64_t)hist_off[(int64_t)b * nblk + blockIdx.x] + pos] = (int32_t)i;
            cap = cap_of(u_in[i], b, i, P);
        }
        int64_t tot;
        int64_t ex = block_exclusive_scan<BIN_NT>(cap, scratch, tot);
        if (valid) ctil_rp[i] = capcarry + ex;
        capcarry += tot;
        if (threadIdx.x < NUM_BINS) {
            int32_t s = 0;
#pragma unroll
            for (int w = 0; w < BIN_NW; ++w) s += wcnt[w][threadIdx.x];
            run[threadIdx.x] += s;
        }
        __syncthreads();
    }
}

// The rows of C~ laid out again from the stored u_i and bins under policy P (the learned
// sizes are known only after the binning): ctil_rp[0..m] and the total into *total.
struct LoadCap {
    const int64_t *u;
    const uint8_t *bin;
    CapPolicy P;
    SPG_DEV int64_t operator()(int64_t i) const { return cap_of(u[i], (int)bin[i], i, P); }
};

cudaError_t launch_cap_rescan(int64_t m, const int64_t *u, const uint8_t *bin, CapPolicy P, int64_t *ctil_rp,
                              int64_t *partial, int64_t *total, cudaStream_t st) {
    cudaError_t e = device_exclusive_scan(m, LoadCap{u, bin, P}, StoreI64{ctil_rp}, partial, total, st);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(ctil_rp + m, total, sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
}

cudaError_t launch_binning(int64_t m, const int64_t *arp, const int64_t *S,
                           const int64_t *sum_u_ptr, CapPolicy P, int64_t *u, uint8_t *bin, int32_t *nnzc, int32_t *bin_rows,
                           int64_t *ctil_rp, int32_t *hist, int64_t *cap_partial,
                           BinSummary *summary, cudaStream_t st) {
    const int64_t nblk = bin_blocks(m);
    if (nblk > 0)
        k_bin_count<<<(unsigned)nblk, BIN_NT, 0, st>>>(m, arp, S, P, u, bin, nnzc, hist, cap_partial,
                                                        nblk);
    k_bin_scan<<<1, 1024, 0, st>>>(m, hist, nblk, cap_partial, ctil_rp, sum_u_ptr, summary);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (nblk > 0)
        k_bin_scatter<<<(unsigned)nblk, BIN_NT, 0, st>>>(m, u, bin, P, hist, cap_partial, nblk,
                                                          bin_rows, ctil_rp);
    return cudaGetLastError();
}

}  // namespace spg
