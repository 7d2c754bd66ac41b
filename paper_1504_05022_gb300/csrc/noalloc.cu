// An allocation-free variant of stage 4's prefix sum (row sizes -> int64 row
// pointers) for callers that must not allocate device memory.
//
// The scan's per-tile partial sums live in a file-scope __device__ array of a
// fixed size instead of a buffer from the library's pool.  In host code that
// array's name is only a host-side stand-in, so the device address is looked up
// once per device with cudaGetSymbolAddress and passed to the kernels.
#include "spgemm.h"
#include "internal.h"
#include "scan.cuh"

#include <mutex>
#include <utility>
#include <vector>

namespace {

// One partial sum per scan tile of SCAN_TILE (2048) rows, plus one spare slot.
constexpr int64_t kRowPtrScratchTiles = 32768;
constexpr int64_t kRowPtrMaxRows = kRowPtrScratchTiles * spg::SCAN_TILE;  // 67,108,864 rows

static __device__ __align__(256) int64_t g_rowptr_scratch[kRowPtrScratchTiles + 1];

std::mutex g_scratch_mu;
std::vector<std::pair<int, int64_t *>> g_scratch_addr;  // device -> address of g_rowptr_scratch

// Resolves the scratch array's device address for the current device (once per device).
cudaError_t scratch_address(int device, int64_t **out) {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    for (auto &d : g_scratch_addr)
        if (d.first == device) {
            *out = d.second;
            return cudaSuccess;
        }
    int64_t *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&ptr, g_rowptr_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr.emplace_back(device, ptr);
    *out = ptr;
    return cudaSuccess;
}

struct LoadRowSize {
    const int32_t *size;
    SPG_DEV int64_t operator()(int64_t i) const { return (int64_t)size[i]; }
};

struct StoreRowPtr {
    int64_t *rp;
    SPG_DEV void operator()(int64_t i, int64_t v) const { rp[i] = v; }
};

}  // namespace

extern "C" spgemm_status spgemm_rowptr_scan_noalloc(const int32_t *row_nnz, int64_t m, int64_t *row_ptr,
                                                    spgemm_stream_t stream) {
    if (m < 0 || row_ptr == nullptr || (m > 0 && row_nnz == nullptr)) return SPGEMM_ERR_INVALID_ARG;
    if (m > kRowPtrMaxRows) return SPGEMM_ERR_SHAPE;
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return SPGEMM_ERR_CUDA;
    int64_t *scratch = nullptr;
    e = scratch_address(device, &scratch);
    if (e != cudaSuccess) return SPGEMM_ERR_CUDA;
    // Every partial slot the scan reads is written by the same call first, so the
    // scratch needs no clearing between calls.
    e = spg::device_exclusive_scan(m, LoadRowSize{row_nnz}, StoreRowPtr{row_ptr}, scratch, row_ptr + m,
                                   reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
}

extern "C" int64_t spgemm_rowptr_scan_noalloc_max_rows(void) { return kRowPtrMaxRows; }
