// Batched products: many independent C_i = A_i * B_i computed as one product of
// block-diagonal matrices, diag(A_1..A_n) * diag(B_1..B_n) = diag(A_1 B_1 .. A_n B_n).
// The concatenation gives A_i's columns an offset of sum_{j<i} k_j, so they
// select B_i's rows; B_i's columns keep their own numbering (0 .. n_i - 1): a
// row of C_i only ever combines rows of B_i, so no row mixes columns of two
// pairs, and the concatenated C holds every C_i with its own column numbers.
// Every stage of the framework runs once over the rows of all pairs (one launch
// per bin for the whole batch).  The split step only rebases each C_i's row
// pointers; its columns and values are views into the concatenated C.
#include "internal.h"
#include "common.cuh"

namespace spg {

SPG_DEV int find_pair(const int64_t *off, int64_t npairs, int64_t x) {
    // largest i with off[i] <= x
    int64_t lo = 0, hi = npairs - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (off[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return (int)lo;
}

SPG_DEV int64_t rp_at(const void *rp, int bits, int64_t i) {
    return bits == 64 ? static_cast<const int64_t *>(rp)[i] : (int64_t) static_cast<const int32_t *>(rp)[i];
}

// Row pointers of the concatenated A (rows of all pairs) and B.
__global__ void k_concat_rp(const PairDesc *d, int64_t npairs, const int64_t *moff, const int64_t *koff, int64_t M,
                            int64_t K, int64_t annz, int64_t bnnz, int64_t *a_rp, int64_t *b_rp) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < M) {
        const int i = find_pair(moff, npairs, r);
        a_rp[r] = d[i].annz_off + rp_at(d[i].a_rp, d[i].a_bits, r - d[i].moff);
    } else if (r == M) {
        a_rp[M] = annz;
    }
    if (r < K) {
        const int i = find_pair(koff, npairs, r);
        b_rp[r] = d[i].bnnz_off + rp_at(d[i].b_rp, d[i].b_bits, r - d[i].koff);
    } else if (r == K) {
        b_rp[K] = bnnz;
    }
}

// Entries of the concatenated A (columns shifted into the pair's block) and B.
__global__ void k_concat_entries(const PairDesc *d, int64_t npairs, const int64_t *annz_off, const int64_t *bnnz_off,
                                 int64_t annz, int64_t bnnz, int32_t *a_col, val_t *a_val, int32_t *b_col,
                                 val_t *b_val, int values_only) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < annz) {
        const int i = find_pair(annz_off, npairs, t);
        const int64_t l = t - d[i].annz_off;
        if (!values_only) a_col[t] = d[i].a_col[l] + (int32_t)d[i].koff;
        a_val[t] = d[i].a_val[l];
    }
    if (t < bnnz) {
        const int i = find_pair(bnnz_off, npairs, t);
        const int64_t l = t - d[i].bnnz_off;
        if (!values_only) b_col[t] = d[i].b_col[l];
        b_val[t] = d[i].b_val[l];
    }
}

cudaError_t launch_concat(const PairDesc *d, int64_t npairs, const int64_t *moff, const int64_t *koff,
                          const int64_t *annz_off, const int64_t *bnnz_off, int64_t M, int64_t K, int64_t annz,
                          int64_t bnnz, int64_t *a_rp, int32_t *a_col, val_t *a_val, int64_t *b_rp, int32_t *b_col,
                          val_t *b_val, bool values_only, cudaStream_t st) {
    if (npairs <= 0) return cudaSuccess;
    if (!values_only) {
        const int64_t rmax = (M > K ? M : K) + 1;
        k_concat_rp<<<(unsigned)((rmax + 255) / 256), 256, 0, st>>>(d, npairs, moff, koff, M, K, annz, bnnz, a_rp,
                                                                   b_rp);
    }
    const int64_t emax = annz > bnnz ? annz : bnnz;
    if (emax > 0)
        k_concat_entries<<<(unsigned)((emax + 255) / 256), 256, 0, st>>>(d, npairs, annz_off, bnnz_off, annz, bnnz,
                                                                        a_col, a_val, b_col, b_val,
                                                                        values_only ? 1 : 0);
    return cudaGetLastError();
}

// C_i's row pointers, rebased to 0; pair i occupies rp_out[moff_i + i .. moff_i + i + m_i].
__global__ void k_split_out(const PairDesc *d, int64_t npairs, const int64_t *c_rp, int64_t M, int64_t *rp_out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < M + npairs) {
        // entry t of the rebased row-pointer array: pair i holds m_i + 1 entries starting at moff_i + i
        int64_t lo = 0, hi = npairs - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (d[mid].moff + mid <= t) lo = mid; else hi = mid - 1;
        }
        const int i = (int)lo;
        const int64_t r = t - (d[i].moff + i);
        rp_out[t] = c_rp[d[i].moff + r] - c_rp[d[i].moff];
    }
}

cudaError_t launch_split_out(const PairDesc *d, int64_t npairs, const int64_t *c_rp, int64_t M, int64_t *rp_out,
                             cudaStream_t st) {
    const int64_t n = M + npairs;
    if (n <= 0) return cudaSuccess;
    k_split_out<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d, npairs, c_rp, M, rp_out);
    return cudaGetLastError();
}

// Per pair i: prod[i] = sum over the entries a_ik of A_i of nnz(b_k*), the
// products of the pair (Algorithm 2 summed over its rows), and clow[i] = sum
// over the rows of A_i of max_k nnz(b_k*), a lower bound of nnz(C_i) (a row of
// C contains every column of each B row it merges).  Grid (PAIR_BLOCKS, npairs),
// a warp per row; columns outside [0, k_i) are skipped (they are rejected later
// when inputs are checked).  prod and clow must be zeroed.
constexpr int PAIR_BLOCKS = 64;

__global__ void k_pair_products(const PairDesc *d, unsigned long long *prod, unsigned long long *clow) {
    __shared__ int64_t sh[2][256 / 32];
    const PairDesc q = d[blockIdx.y];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t s = 0, lo = 0;
    for (int64_t r = (int64_t)blockIdx.x * 8 + wid; r < q.m; r += (int64_t)PAIR_BLOCKS * 8) {
        const int64_t a0 = rp_at(q.a_rp, q.a_bits, r), a1 = rp_at(q.a_rp, q.a_bits, r + 1);
        int64_t rs = 0, rm = 0;
        for (int64_t e = a0 + lane; e < a1; e += 32) {
            const int32_t k = q.a_col[e];
            if (k >= 0 && k < q.k) {
                const int64_t len = rp_at(q.b_rp, q.b_bits, k + 1) - rp_at(q.b_rp, q.b_bits, k);
                rs += len;
                rm = len > rm ? len : rm;
            }
        }
        s += rs;
        for (int o = 16; o > 0; o >>= 1) {
            const int64_t x = __shfl_xor_sync(SPG_FULL, rm, o);
            rm = x > rm ? x : rm;
        }
        lo += rm;  // the same on every lane
    }
    s = warp_reduce_sum(s);
    if (lane == 0) {
        sh[0][wid] = s;
        sh[1][wid] = lo;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t ts = 0, tl = 0;
        for (int w = 0; w < 8; ++w) {
            ts += sh[0][w];
            tl += sh[1][w];
        }
        if (ts) atomicAdd(prod + blockIdx.y, (unsigned long long)ts);
        if (tl) atomicAdd(clow + blockIdx.y, (unsigned long long)tl);
    }
}

cudaError_t launch_pair_products(const PairDesc *d, int64_t npairs, int64_t *prod, int64_t *clow,
                                 cudaStream_t st) {
    if (npairs <= 0) return cudaSuccess;
    if (npairs > 65535) return cudaErrorInvalidValue;  // grid.y limit; the caller then uses one wave
    cudaError_t e = cudaMemsetAsync(prod, 0, sizeof(int64_t) * npairs, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(clow, 0, sizeof(int64_t) * npairs, st);
    if (e != cudaSuccess) return e;
    k_pair_products<<<dim3(PAIR_BLOCKS, (unsigned)npairs), 256, 0, st>>>(
        d, reinterpret_cast<unsigned long long *>(prod), reinterpret_cast<unsigned long long *>(clow));
    return cudaGetLastError();
}

// out[i] = c_rp[moff_i] (first entry of C_i in the concatenation), out[np] = c_rp[M].
__global__ void k_gather_first(const PairDesc *d, int64_t npairs, const int64_t *c_rp, int64_t M, int64_t *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < npairs) out[i] = c_rp[d[i].moff];
    else if (i == npairs) out[npairs] = c_rp[M];
}

cudaError_t launch_gather_first(const PairDesc *d, int64_t npairs, const int64_t *c_rp, int64_t M, int64_t *out,
                                cudaStream_t st) {
    k_gather_first<<<(unsigned)((npairs + 256) / 256), 256, 0, st>>>(d, npairs, c_rp, M, out);
    return cudaGetLastError();
}

}  // namespace spg
