// Learned preallocation: per-row features, a small MLP (forward, gradient,
// Adam), and the prediction of each bin-37 row's temporary size and launch
// class.  Not in the paper: it replaces the fixed 256-entry start of the
// progressive allocation (Section 4.1) by a predicted size, while the exact
// progressive path stays the fallback for any row predicted too small.
//
// Parameter vector (float32): W1[32x8] b1[32] W2[32x32] b2[32] W3[17x32] b3[17]
// then mu[8] sigma[8].  out = W3 relu(W2 relu(W1 (x-mu)/sigma + b1) + b2) + b3;
// out[0..15] are size-class logits, out[16] regresses log2(1 + nnz(c_i)).
#include "spgemm.h"
#include "internal.h"
#include "common.cuh"

#include <new>

namespace spg {

constexpr int MLP_IN = SPGEMM_MLP_FEATURES;
constexpr int MLP_HID = SPGEMM_MLP_HIDDEN;
constexpr int MLP_CLS = SPGEMM_MLP_CLASSES;
constexpr int MLP_OUT = MLP_CLS + 1;
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + MLP_HID * MLP_IN;
constexpr int OFF_W2 = OFF_B1 + MLP_HID;
constexpr int OFF_B2 = OFF_W2 + MLP_HID * MLP_HID;
constexpr int OFF_W3 = OFF_B2 + MLP_HID;
constexpr int OFF_B3 = OFF_W3 + MLP_OUT * MLP_HID;
constexpr int OFF_MU = OFF_B3 + MLP_OUT;
constexpr int OFF_SG = OFF_MU + MLP_IN;
static_assert(OFF_MU == SPGEMM_MLP_NUM_PARAMS, "parameter layout");
static_assert(OFF_SG + MLP_IN == SPGEMM_MLP_NUM_TOTAL, "parameter layout");
// per-sample record kept between the forward/backward pass and the reduction
constexpr int REC = MLP_IN + 2 * MLP_HID + MLP_HID + MLP_HID + MLP_OUT;  // xh, h1, h2, dz1, dz2, dout
constexpr int R_XH = 0, R_H1 = MLP_IN, R_H2 = R_H1 + MLP_HID, R_DZ1 = R_H2 + MLP_HID,
              R_DZ2 = R_DZ1 + MLP_HID, R_DOUT = R_DZ2 + MLP_HID;

// ---------------- features ----------------

// One warp per row: the 8 features (log2(1+.) of nnz(a_i*), u_i, min/max/mean/std
// of the selected B-row lengths, the column span of the selected B rows, ncols(B)).
__global__ void k_row_features(DevCSR A, DevCSR B, const int64_t *__restrict__ S, int64_t u_min,
                               const uint8_t *__restrict__ skip, float *__restrict__ X) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= A.nrows) return;
    const int64_t a0 = A.rp[row], a1 = A.rp[row + 1];
    // with the stage-1 prefix S given, only rows with u_i > u_min (bin 37) need features, and
    // not the dense-slice rows
    if (S != nullptr && S[a1] - S[a0] <= u_min) return;
    if (skip != nullptr && skip[row]) return;
    double sum_len = 0.0, sg = 0.0, sg2 = 0.0;
    float gmin = 3.4e38f, gmax = -3.4e38f;
    int32_t cmin = INT_MAX, cmax = -1;
    for (int64_t p = a0 + lane; p < a1; p += 32) {
        const int32_t k = A.col[p];
        const int64_t b0 = B.rp[k], b1 = B.rp[k + 1];
        const int64_t len = b1 - b0;
        const float g = log2f(1.f + (float)len);
        sum_len += (double)len;
        sg += (double)g;
        sg2 += (double)g * (double)g;
        gmin = fminf(gmin, g);
        gmax = fmaxf(gmax, g);
        if (len > 0) {
            cmin = min(cmin, B.col[b0]);
            cmax = max(cmax, B.col[b1 - 1]);
        }
    }
    for (int d = 16; d > 0; d >>= 1) {
        sum_len += __shfl_xor_sync(SPG_FULL, sum_len, d);
        sg += __shfl_xor_sync(SPG_FULL, sg, d);
        sg2 += __shfl_xor_sync(SPG_FULL, sg2, d);
        gmin = fminf(gmin, __shfl_xor_sync(SPG_FULL, gmin, d));
        gmax = fmaxf(gmax, __shfl_xor_sync(SPG_FULL, gmax, d));
        cmin = min(cmin, __shfl_xor_sync(SPG_FULL, cmin, d));
        cmax = max(cmax, __shfl_xor_sync(SPG_FULL, cmax, d));
    }
    if (lane == 0) {
        const double n = (double)(a1 - a0);
        float *x = X + row * MLP_IN;
        x[0] = log2f(1.f + (float)n);
        x[1] = log2f(1.f + (float)sum_len);
        if (n > 0) {
            const double mean = sg / n;
            const double var = sg2 / n - mean * mean;
            x[2] = gmin;
            x[3] = gmax;
            x[4] = (float)mean;
            x[5] = (float)sqrt(var > 0.0 ? var : 0.0);
            x[6] = cmax >= 0 ? log2f(1.f + (float)(cmax - cmin + 1)) : 0.f;
        } else {
            x[2] = x[3] = x[4] = x[5] = x[6] = 0.f;
        }
        x[7] = log2f(1.f + (float)B.ncols);
    }
}

cudaError_t launch_row_features(const DevCSR &A, const DevCSR &B, float *X, cudaStream_t st, const int64_t *S,
                                int64_t u_min, const uint8_t *skip) {
    if (A.nrows <= 0) return cudaSuccess;
    const int64_t threads = A.nrows * 32;
    k_row_features<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(A, B, S, u_min, skip, X);
    return cudaGetLastError();
}

// ---------------- MLP ----------------

SPG_DEV void mlp_forward_one(const float *P, const float *x, float *xh, float *h1, float *h2, float *out) {
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) xh[i] = (x[i] - P[OFF_MU + i]) / P[OFF_SG + i];
#pragma unroll 4
    for (int o = 0; o < MLP_HID; ++o) {
        float z = P[OFF_B1 + o];
#pragma unroll
        for (int i = 0; i < MLP_IN; ++i) z = fmaf(P[OFF_W1 + o * MLP_IN + i], xh[i], z);
        h1[o] = z > 0.f ? z : 0.f;
    }
#pragma unroll 4
    for (int o = 0; o < MLP_HID; ++o) {
        float z = P[OFF_B2 + o];
#pragma unroll 8
        for (int i = 0; i < MLP_HID; ++i) z = fmaf(P[OFF_W2 + o * MLP_HID + i], h1[i], z);
        h2[o] = z > 0.f ? z : 0.f;
    }
#pragma unroll 1
    for (int o = 0; o < MLP_OUT; ++o) {
        float z = P[OFF_B3 + o];
#pragma unroll 8
        for (int i = 0; i < MLP_HID; ++i) z = fmaf(P[OFF_W3 + o * MLP_HID + i], h2[i], z);
        out[o] = z;
    }
}

__global__ void k_mlp_forward(const float *__restrict__ params, const float *__restrict__ X, int64_t n,
                              float *__restrict__ out) {
    __shared__ float P[SPGEMM_MLP_NUM_TOTAL];
    for (int t = threadIdx.x; t < SPGEMM_MLP_NUM_TOTAL; t += blockDim.x) P[t] = params[t];
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float xh[MLP_IN], h1[MLP_HID], h2[MLP_HID], o[MLP_OUT];
    mlp_forward_one(P, X + s * MLP_IN, xh, h1, h2, o);
#pragma unroll
    for (int k = 0; k < MLP_OUT; ++k) out[s * MLP_OUT + k] = o[k];
}

// Forward and backward of one sample per thread; records activations and deltas
// for the reduction kernel and accumulates the summed loss.
__global__ void k_mlp_fwd_bwd(const float *__restrict__ params, const float *__restrict__ X,
                              const int32_t *__restrict__ cls, const float *__restrict__ y, int64_t n,
                              float *__restrict__ rec, double *__restrict__ loss) {
    __shared__ float P[SPGEMM_MLP_NUM_TOTAL];
    __shared__ double lsum[8];
    for (int t = threadIdx.x; t < SPGEMM_MLP_NUM_TOTAL; t += blockDim.x) P[t] = params[t];
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (s < n) {
        float xh[MLP_IN], h1[MLP_HID], h2[MLP_HID], o[MLP_OUT];
        mlp_forward_one(P, X + s * MLP_IN, xh, h1, h2, o);
        float mx = o[0];
#pragma unroll
        for (int k = 1; k < MLP_CLS; ++k) mx = fmaxf(mx, o[k]);
        float se = 0.f;
#pragma unroll
        for (int k = 0; k < MLP_CLS; ++k) se += expf(o[k] - mx);
        const int c = cls[s];
        const float r = o[MLP_CLS] - y[s];
        l = (double)(logf(se) + mx - o[c]) + 0.5 * (double)r * (double)r;
        float *R = rec + s * REC;
        float dout[MLP_OUT];
#pragma unroll
        for (int k = 0; k < MLP_CLS; ++k) dout[k] = expf(o[k] - mx) / se - (k == c ? 1.f : 0.f);
        dout[MLP_CLS] = r;
        float dz2[MLP_HID];
#pragma unroll 4
        for (int i = 0; i < MLP_HID; ++i) {
            float d = 0.f;
            for (int k = 0; k < MLP_OUT; ++k) d = fmaf(dout[k], P[OFF_W3 + k * MLP_HID + i], d);
            dz2[i] = h2[i] > 0.f ? d : 0.f;
        }
#pragma unroll 4
        for (int i = 0; i < MLP_HID; ++i) {
            float d = 0.f;
#pragma unroll 8
            for (int k = 0; k < MLP_HID; ++k) d = fmaf(dz2[k], P[OFF_W2 + k * MLP_HID + i], d);
            R[R_DZ1 + i] = h1[i] > 0.f ? d : 0.f;
        }
#pragma unroll
        for (int i = 0; i < MLP_IN; ++i) R[R_XH + i] = xh[i];
#pragma unroll
        for (int i = 0; i < MLP_HID; ++i) {
            R[R_H1 + i] = h1[i];
            R[R_H2 + i] = h2[i];
            R[R_DZ2 + i] = dz2[i];
        }
#pragma unroll
        for (int k = 0; k < MLP_OUT; ++k) R[R_DOUT + k] = dout[k];
    }
    // block sum of the loss, one atomic per block
    for (int d = 16; d > 0; d >>= 1) l += __shfl_xor_sync(SPG_FULL, l, d);
    if ((threadIdx.x & 31) == 0) lsum[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += lsum[w];
        atomicAdd(loss, t);
    }
}

// One block per output neuron of a layer: gradient row (weights and bias) summed
// over all samples.  Blocks 0..31: layer 1, 32..63: layer 2, 64..80: layer 3.
__global__ void k_mlp_grad_reduce(const float *__restrict__ rec, int64_t n, float *__restrict__ grad) {
    const int b = blockIdx.x;
    int o, nin, din, ain, gw, gb;
    if (b < MLP_HID) {  // layer 1
        o = b; nin = MLP_IN; din = R_DZ1; ain = R_XH; gw = OFF_W1; gb = OFF_B1;
    } else if (b < 2 * MLP_HID) {  // layer 2
        o = b - MLP_HID; nin = MLP_HID; din = R_DZ2; ain = R_H1; gw = OFF_W2; gb = OFF_B2;
    } else {  // layer 3
        o = b - 2 * MLP_HID; nin = MLP_HID; din = R_DOUT; ain = R_H2; gw = OFF_W3; gb = OFF_B3;
    }
    float acc[MLP_HID + 1];
#pragma unroll
    for (int i = 0; i <= MLP_HID; ++i) acc[i] = 0.f;
    for (int64_t s = threadIdx.x; s < n; s += blockDim.x) {
        const float *R = rec + s * REC;
        const float d = R[din + o];
        if (d != 0.f) {
#pragma unroll
            for (int i = 0; i < MLP_HID; ++i)
                if (i < nin) acc[i] = fmaf(d, R[ain + i], acc[i]);
            acc[MLP_HID] += d;
        }
    }
    __shared__ float red[MLP_HID + 1][8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i <= MLP_HID; ++i) {
        float v = acc[i];
        for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(SPG_FULL, v, d);
        if (lane == 0) red[i][w] = v;
    }
    __syncthreads();
    if (threadIdx.x <= MLP_HID) {
        const int i = threadIdx.x;
        float v = 0.f;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v += red[i][k];
        if (i < nin) grad[gw + o * nin + i] = v;
        else if (i == MLP_HID) grad[gb + o] = v;
    }
}

__global__ void k_mlp_adam(float *__restrict__ params, const float *__restrict__ grad, float *__restrict__ m,
                           float *__restrict__ v, int n, float lr, float b1, float b2, float eps, float scale,
                           float bc1, float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = grad[i] * scale;
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    params[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// Plan-side prediction for every row: predicted home size (>= min_cap, <= u_i)
// from the regression head, times `margin`, rounded up to 32; u_i itself when it is
// within a factor `margin` of that size.
__global__ void k_mlp_predict_caps(const float *__restrict__ params, const float *__restrict__ X, int64_t m,
                                   const int64_t *__restrict__ u, const int64_t *__restrict__ arp,
                                   const int64_t *__restrict__ S, int64_t u_min, uint8_t *__restrict__ skip,
                                   float margin, int32_t min_cap, int32_t *__restrict__ pred_cap,
                                   int64_t promote_min) {
    __shared__ float P[SPGEMM_MLP_NUM_TOTAL];
    for (int t = threadIdx.x; t < SPGEMM_MLP_NUM_TOTAL; t += blockDim.x) P[t] = params[t];
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= m) return;
    // the row's bound u_i (Algorithm 2), when known
    const int64_t uu = S != nullptr ? S[arp[s + 1]] - S[arp[s]] : (u != nullptr ? u[s] : -1);
    // outside bin 37, or a dense-slice row: no prediction needed
    if ((S != nullptr && uu <= u_min) || (skip != nullptr && skip[s])) {
        pred_cap[s] = 0;
        return;
    }
    float xh[MLP_IN], h1[MLP_HID], h2[MLP_HID], o[MLP_OUT];
    mlp_forward_one(P, X + s * MLP_IN, xh, h1, h2, o);
    float reg = fminf(fmaxf(o[MLP_CLS], 0.f), 30.f);
    double nnz = exp2((double)reg) - 1.0;
    if (promote_min > 0 && skip != nullptr && nnz >= (double)promote_min) {
        // the network's choice of kernel: a row this long goes to the dense-slice kernels
        skip[s] = 1;
        pred_cap[s] = 0;
        return;
    }
    double c = ceil(nnz * (double)margin / 32.0) * 32.0;
    int64_t cap = (int64_t)c;
    if (cap < min_cap) cap = min_cap;
    if (uu >= 0) {
        // a bound within a factor `margin` of the sized prediction is taken instead: the row
        // can then never outgrow its slot, for at most `margin` times the prediction's space
        if ((double)uu <= (double)cap * (double)margin) cap = uu;
        if (cap > uu) cap = uu;
    }
    if (cap > INT32_MAX) cap = INT32_MAX;
    pred_cap[s] = (int32_t)cap;
}

cudaError_t launch_predict_caps(const float *params, const float *X, int64_t m, const int64_t *u, float margin,
                                int32_t min_cap, int32_t *pred_cap, cudaStream_t st, const int64_t *arp,
                                const int64_t *S, int64_t u_min, uint8_t *skip, int64_t promote_min) {
    if (m <= 0) return cudaSuccess;
    k_mlp_predict_caps<<<(unsigned)((m + 127) / 128), 128, 0, st>>>(params, X, m, u, arp, S, u_min, skip, margin,
                                                                     min_cap, pred_cap, promote_min);
    return cudaGetLastError();
}

// Launch-class partition of the bin-37 rows by predicted size: class g holds
// the rows whose predicted size is at most class_cap[g] (the smallest such g).
// The dense-slice rows go to slot ncls, after the classes.
// Bin 37 is the last segment of bin_rows; its size is read from the stage-2
// summary on the device, so no host round trip is needed.  The order inside a
// class is not fixed (atomics); it only affects scheduling, not C.
__global__ void k_class_count(const int32_t *bin_rows, int64_t m, const BinSummary *summary,
                              const int32_t *pred_cap, const int32_t *class_cap, int ncls, const uint8_t *dense,
                              int32_t *cls_of, int32_t *count) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n37 = summary->bin_count[BIN_MERGE];
    if (j >= n37) return;
    const int32_t row = bin_rows[m - n37 + j];
    const int32_t c = pred_cap[row];
    int g = ncls - 1;
    for (int k = 0; k < ncls; ++k)
        if (c <= class_cap[k]) {
            g = k;
            break;
        }
    if (dense != nullptr && dense[row]) g = ncls;
    cls_of[j] = g;
    atomicAdd(&count[g], 1);
}

__global__ void k_class_starts(const int32_t *count, int ncls, int32_t *start, int32_t *cursor,
                               BinSummary *summary) {
    if (threadIdx.x == 0) {
        int32_t s = 0;
        for (int g = 0; g <= ncls; ++g) {
            start[g] = s;
            cursor[g] = 0;
            if (g < ncls) summary->class_count[g] = count[g];
            s += count[g];
        }
    }
}

__global__ void k_class_scatter(int64_t m, const BinSummary *summary, const int32_t *cls_of, const int32_t *start,
                                int32_t *cursor, int32_t *order) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= summary->bin_count[BIN_MERGE]) return;
    const int g = cls_of[j];
    order[start[g] + atomicAdd(&cursor[g], 1)] = (int32_t)j;
}

cudaError_t launch_class_partition_tail(const int32_t *bin_rows, int64_t m, BinSummary *summary,
                                        const int32_t *pred_cap, const int32_t *class_cap, int ncls,
                                        const uint8_t *dense, int32_t *scratch, int32_t *order, cudaStream_t st) {
    if (m <= 0 || ncls > 31) return m <= 0 ? cudaSuccess : cudaErrorInvalidValue;
    int32_t *count = scratch, *start = scratch + 32, *cursor = scratch + 64, *cls_of = scratch + 96;
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int32_t) * 32, st);
    if (e != cudaSuccess) return e;
    const unsigned g = (unsigned)((m + 255) / 256);
    k_class_count<<<g, 256, 0, st>>>(bin_rows, m, summary, pred_cap, class_cap, ncls, dense, cls_of, count);
    k_class_starts<<<1, 32, 0, st>>>(count, ncls, start, cursor, summary);
    k_class_scatter<<<g, 256, 0, st>>>(m, summary, cls_of, start, cursor, order);
    return cudaGetLastError();
}

}  // namespace spg

// ---------------- C ABI of the predictor ----------------

using namespace spg;

struct spgemm_predictor {
    int device;
    float *params;  // device copy of the SPGEMM_MLP_NUM_TOTAL values
};

extern "C" spgemm_status spgemm_predictor_create(const float *host_params, int64_t n, spgemm_predictor **out) {
    if (!out || !host_params || n != SPGEMM_MLP_NUM_TOTAL) return SPGEMM_ERR_INVALID_ARG;
    *out = nullptr;
    spgemm_predictor *p = new (std::nothrow) spgemm_predictor();
    if (!p) return SPGEMM_ERR_OOM;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return SPGEMM_ERR_CUDA;
    }
    cudaError_t e = cudaMalloc(&p->params, sizeof(float) * SPGEMM_MLP_NUM_TOTAL);
    if (e != cudaSuccess) {
        delete p;
        return e == cudaErrorMemoryAllocation ? SPGEMM_ERR_OOM : SPGEMM_ERR_CUDA;
    }
    e = cudaMemcpy(p->params, host_params, sizeof(float) * SPGEMM_MLP_NUM_TOTAL, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(p->params);
        delete p;
        return SPGEMM_ERR_CUDA;
    }
    *out = p;
    return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_predictor_free(spgemm_predictor *p) {
    if (!p) return SPGEMM_OK;
    cudaFree(p->params);
    delete p;
    return SPGEMM_OK;
}

namespace spg {
const float *predictor_params(const void *pred) {
    return pred ? static_cast<const spgemm_predictor *>(pred)->params : nullptr;
}
}  // namespace spg

static spgemm_status widen_in(const spgemm_csr_in *M, DevCSR &D, int64_t **tmp, cudaStream_t st) {
    D.nrows = M->nrows;
    D.ncols = M->ncols;
    D.nnz = M->nnz;
    D.col = M->col_idx;
    D.val = M->val;
    *tmp = nullptr;
    if (M->rowptr_bits == 64) {
        D.rp = static_cast<const int64_t *>(M->row_ptr);
        return SPGEMM_OK;
    }
    if (cudaMallocAsync(reinterpret_cast<void **>(tmp), sizeof(int64_t) * (M->nrows + 1), st) != cudaSuccess)
        return SPGEMM_ERR_OOM;
    if (launch_widen_rowptr(static_cast<const int32_t *>(M->row_ptr), *tmp, M->nrows + 1, st) != cudaSuccess)
        return SPGEMM_ERR_CUDA;
    D.rp = *tmp;
    return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_row_features(const spgemm_csr_in *A, const spgemm_csr_in *B, float *X,
                                             spgemm_stream_t stream) {
    if (!A || !B || (!X && A->nrows > 0)) return SPGEMM_ERR_INVALID_ARG;
    if (A->ncols != B->nrows) return SPGEMM_ERR_SHAPE;
    if ((A->rowptr_bits != 32 && A->rowptr_bits != 64) || (B->rowptr_bits != 32 && B->rowptr_bits != 64))
        return SPGEMM_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    DevCSR a, b;
    int64_t *ta = nullptr, *tb = nullptr;
    spgemm_status s = widen_in(A, a, &ta, st);
    if (s == SPGEMM_OK) s = widen_in(B, b, &tb, st);
    if (s == SPGEMM_OK && launch_row_features(a, b, X, st) != cudaSuccess) s = SPGEMM_ERR_CUDA;
    if (ta) cudaFreeAsync(ta, st);
    if (tb) cudaFreeAsync(tb, st);
    return s;
}

extern "C" spgemm_status spgemm_mlp_forward(const float *params, const float *X, int64_t n, float *out,
                                            spgemm_stream_t stream) {
    if (n < 0 || !params || (n > 0 && (!X || !out))) return SPGEMM_ERR_INVALID_ARG;
    if (n == 0) return SPGEMM_OK;
    k_mlp_forward<<<(unsigned)((n + 127) / 128), 128, 0, reinterpret_cast<cudaStream_t>(stream)>>>(params, X, n,
                                                                                                 out);
    return cudaGetLastError() == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
}

extern "C" spgemm_status spgemm_mlp_loss_grad(const float *params, const float *X, const int32_t *cls,
                                              const float *y, int64_t n, float *work, float *grad, double *loss,
                                              spgemm_stream_t stream) {
    if (n < 0 || !params || !grad || !loss || (n > 0 && (!X || !cls || !y || !work)))
        return SPGEMM_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(loss, 0, sizeof(double), st) != cudaSuccess) return SPGEMM_ERR_CUDA;
    if (n == 0) {
        if (cudaMemsetAsync(grad, 0, sizeof(float) * SPGEMM_MLP_NUM_PARAMS, st) != cudaSuccess)
            return SPGEMM_ERR_CUDA;
        return SPGEMM_OK;
    }
    k_mlp_fwd_bwd<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(params, X, cls, y, n, work, loss);
    k_mlp_grad_reduce<<<2 * MLP_HID + MLP_OUT, 256, 0, st>>>(work, n, grad);
    return cudaGetLastError() == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
}

extern "C" int64_t spgemm_mlp_work_floats(int64_t n) { return n * (int64_t)REC; }

extern "C" spgemm_status spgemm_mlp_adam(float *params, const float *grad, float *m, float *v, int64_t step,
                                         float lr, float grad_scale, spgemm_stream_t stream) {
    if (!params || !grad || !m || !v || step < 1) return SPGEMM_ERR_INVALID_ARG;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
    k_mlp_adam<<<(SPGEMM_MLP_NUM_PARAMS + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        params, grad, m, v, SPGEMM_MLP_NUM_PARAMS, lr, b1, b2, eps, grad_scale, bc1, bc2);
    return cudaGetLastError() == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
}
