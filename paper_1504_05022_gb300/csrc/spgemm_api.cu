// C ABI and host orchestration of the four-stage SpGEMM framework (Section 4.1).
//
// The host side decides which per-bin kernels run (only non-empty bins), sizes
// and allocates the temporary matrix C~ and the result C, and drives the
// progressive relaunch loop of bin 37.  Device memory comes from a
// library-owned stream-ordered pool (cudaMallocAsync), so every buffer is
// ordered on the plan's stream and its high-water mark is the peak memory of
// a call.
#include "spgemm.h"
#include "internal.h"

#include <algorithm>
#include <chrono>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

using namespace spg;

namespace {

struct DevicePool {
    int device;
    cudaMemPool_t pool;
};

std::mutex g_pool_mu;
std::vector<DevicePool> g_pools;

cudaError_t get_pool(int device, cudaMemPool_t *out) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (auto &p : g_pools)
        if (p.device == device) {
            *out = p.pool;
            return cudaSuccess;
        }
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool;
    cudaError_t e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t thr = UINT64_MAX;  // keep freed blocks for reuse by later calls
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    if (e != cudaSuccess) return e;
    g_pools.push_back({device, pool});
    *out = pool;
    return cudaSuccess;
}

// Small pinned host blocks for the few device->host size reads of a call, mapped into the
// device's address space: a kernel stores the sizes there, so the reads do not go through a
// copy engine and never queue behind large copies that other streams have in flight (a
// caller copying one result to the host while the next product runs).
std::mutex g_pin_mu;
std::vector<void *> g_pinned_free;
constexpr size_t PIN_BYTES = 4096;

void *get_pinned() {
    {
        std::lock_guard<std::mutex> lk(g_pin_mu);
        if (!g_pinned_free.empty()) {
            void *p = g_pinned_free.back();
            g_pinned_free.pop_back();
            return p;
        }
    }
    void *p = nullptr;
    if (cudaHostAlloc(&p, PIN_BYTES, cudaHostAllocMapped) != cudaSuccess) return nullptr;
    return p;
}

static_assert(sizeof(BinSummary) <= PIN_BYTES, "the stage-2 summary is read through one pinned block");

__global__ void k_read_bytes(const unsigned char *__restrict__ src, unsigned char *dst, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

__global__ void k_read_words2(const int64_t *a, const int64_t *b, int64_t *dst) {
    if (threadIdx.x == 0) {
        dst[0] = *a;
        dst[1] = *b;
    }
}

// Auxiliary streams (created once, kept for the process): the learned launch classes of
// bin 37 run on them concurrently, so one class's tail of long CTAs overlaps the next class
// instead of idling the SMs, and the dense-slice kernels run beside the merge kernels.  Each
// stream a plan runs on gets aux streams of its own (up to MAX_AUX_OWNERS streams per device,
// beyond which the last set is shared), so plans on different streams stay independent.
constexpr int NUM_AUX_STREAMS = 5;
constexpr int DENSE_AUX = NUM_AUX_STREAMS - 1;  // the dense-slice kernels; the others take the launch classes
constexpr size_t MAX_AUX_OWNERS = 16;
struct AuxSet {
    int device;
    cudaStream_t owner;
    std::vector<cudaStream_t> s;
};
std::mutex g_aux_mu;
std::vector<AuxSet> g_aux;

cudaStream_t aux_stream(int device, cudaStream_t owner, int i) {
    std::lock_guard<std::mutex> lk(g_aux_mu);
    AuxSet *set = nullptr;
    size_t on_device = 0;
    for (auto &a : g_aux) {
        if (a.device != device) continue;
        ++on_device;
        set = &a;  // the device's last set, unless the owner has one
        if (a.owner == owner) break;
    }
    if (set == nullptr || (set->owner != owner && on_device < MAX_AUX_OWNERS)) {
        g_aux.push_back(AuxSet{device, owner, {}});
        set = &g_aux.back();
    }
    while ((int)set->s.size() < NUM_AUX_STREAMS) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
        set->s.push_back(st);
    }
    return set->s[i % NUM_AUX_STREAMS];
}

void put_pinned(void *p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pinned_free.push_back(p);
}

spgemm_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return SPGEMM_OK;
    if (e == cudaErrorMemoryAllocation) return SPGEMM_ERR_OOM;
    return SPGEMM_ERR_CUDA;
}

struct Timer {
    int kind;
    cudaEvent_t a, b;
};

// Heap-kernel launches: bins 2..32 split into ranges sized to their widest heap.
const int kHeapRanges[][2] = {{2, 8}, {9, 16}, {17, 24}, {25, 32}};

// Bytes of one stored entry (int32 column + value).
constexpr int64_t ENTRY_BYTES = sizeof(int32_t) + sizeof(val_t);

// Lifetimes of plan allocations.
constexpr int LIFE_SYMBOLIC = 0;  // released when spgemm_symbolic returns
constexpr int LIFE_NUMERIC = 1;   // released when spgemm_numeric returns
constexpr int LIFE_PLAN = 2;      // released by spgemm_free

}  // namespace

struct spgemm_plan {
    int device = 0;
    cudaStream_t st = nullptr;
    spgemm_opts opts{};
    cudaMemPool_t pool = nullptr;
    DevCSR A{}, B{};
    std::vector<void *> allocs;
    // temporaries: freed when the stage that needs them is over (symbolic: stage-1
    // prefix and binning scratch; numeric: C~, merge pools and lists)
    struct Temp {
        void *ptr;
        int64_t bytes;
        int life;
    };
    std::vector<Temp> temps;
    int64_t bytes_ctilde = 0;
    int64_t bytes_held = 0;  // device bytes the plan holds now
    int64_t bytes_peak = 0;  // largest bytes_held so far
    // stage 1-2 buffers
    int64_t *S = nullptr, *u = nullptr, *ctil_rp = nullptr, *scan_partial = nullptr;
    uint8_t *bin = nullptr;
    int32_t *bin_rows = nullptr, *nnzc = nullptr, *ctil_col_i = nullptr;
    int32_t *ctil_col = nullptr;
    val_t *ctil_val = nullptr;
    BinSummary *d_summary = nullptr;
    int64_t *d_err = nullptr;
    // products sized on the device: stage-2 scratch and dense-selection scratch kept with the
    // plan, and the work counters of the persistent dense kernels
    int32_t *d_hist = nullptr, *d_select = nullptr;
    int64_t *d_capp = nullptr;
    unsigned long long *d_queue = nullptr;
    BinSummary h_summary{};
    int64_t bin_start[NUM_BINS + 1] = {0};
    // bin 37 work items
    MergeItems items{};
    int64_t n_items = 0, items_cap = 0;
    // learned preallocation
    int32_t *pred_cap = nullptr;      // predicted temporary size per row
    int32_t *class_order = nullptr;   // bin-37 item indices grouped by launch class
    int32_t class_caps[NUM_LAUNCH_CLASSES] = {0};
    int capmax = 0, batch = 0, wide_above = 2048, bm_words = 0, bm_miss = 0, bm_two = 0;
    // dense column slices for the longest bin-37 rows (off when dense_K == 0)
    int dense_K = 0, dense_W = 0;
    int64_t dense_min_u = 0;              // > 0: absolute threshold on u_i; 0: the row's column range
    int64_t dense_n = 0;                  // dense bin-37 rows
    uint8_t *dense_flag = nullptr;        // per row: 1 = dense-slice row (symbolic only)
    int32_t *dense_lo = nullptr, *dense_hi = nullptr;  // per row: column range (symbolic only)
    int32_t *dense_order = nullptr;       // bin-37 items: the dense ones (larger first), then the rest
    int32_t *dense_rows = nullptr;        // rows of the dense items
    int32_t *dense_clo = nullptr, *dense_chi = nullptr;  // and their column ranges
    int32_t *dense_bnd = nullptr;         // per B row, K + 1 slice boundaries (K > 1)
    int32_t *dense_cnt = nullptr, *dense_soff = nullptr;
    uint32_t *dense_keep = nullptr;  // the counting pass's column bitmaps, kept for the fill (numeric only)
    int dense_keep_words = 0;        // words per (row, slice) of dense_keep
    cudaEvent_t dense_count_done = nullptr;  // the counts' stream reached the end of the counting pass
    DenseArgs dense_args() const {
        DenseArgs D{dense_order, dense_rows, dense_clo, dense_chi, dense_n, dense_K, dense_W, dense_bnd,
                    dense_cnt, dense_soff};
        D.queue = d_queue;
        D.keep = dense_keep;
        D.keep_words = dense_keep_words;
        return D;
    }
    // batched plans: the pairs and the concatenation offsets
    int64_t npairs = 0;
    PairDesc *d_pairs = nullptr;
    std::vector<PairDesc> h_pairs;
    int64_t *d_moff = nullptr, *d_koff = nullptr, *d_annz_off = nullptr, *d_bnnz_off = nullptr;
    int64_t *cat_a_rp = nullptr, *cat_b_rp = nullptr;
    int32_t *cat_a_col = nullptr, *cat_b_col = nullptr;
    val_t *cat_a_val = nullptr, *cat_b_val = nullptr;
    int64_t *split_rp = nullptr;
    std::vector<spgemm_csr_out> batch_out;
    // batched plans in waves: groups of pairs computed one after another, each a
    // batched sub-plan of its own made by spgemm_batched_numeric
    bool wave_mode = false;
    std::vector<spgemm_csr_in> wave_A, wave_B;
    std::vector<int64_t> wave_order;  // pairs by descending product count: wave_A[q] = A[wave_order[q]]
    std::vector<int64_t> wave_start;  // first position (in wave_order) of each wave, then npairs
    std::vector<spgemm_plan *> waves;
    // values-only replay
    bool replay_ready = false;
    ReplayLeaves leaves{};
    int32_t *leaf_order = nullptr;
    int64_t leaf_count[NUM_REPLAY_CLASSES] = {0};
    int leaf_cap[NUM_REPLAY_CLASSES] = {0};
    // result
    bool numeric_done = false;
    spgemm_csr_out C{};
    spgemm_stats stats{};
    std::vector<Timer> timers;
    void *pinned = nullptr;
    int smem_optin = 0;

    cudaError_t alloc(void **p, size_t bytes, int life = LIFE_PLAN) {
        if (bytes == 0) bytes = 16;
        if (opts.max_bytes > 0 && bytes_held + (int64_t)bytes > opts.max_bytes) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
        const auto t0 = std::chrono::steady_clock::now();
        cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, st);
        stats.alloc_host_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        stats.allocs += 1;
        if (e != cudaSuccess) {
            *p = nullptr;
            cudaGetLastError();
            return e;
        }
        if (life == LIFE_PLAN) allocs.push_back(*p);
        else temps.push_back(Temp{*p, (int64_t)bytes, life});
        bytes_held += (int64_t)bytes;
        bytes_peak = std::max(bytes_peak, bytes_held);
        return cudaSuccess;
    }
    template <typename T>
    cudaError_t alloc_n(T **p, int64_t n, int life = LIFE_PLAN) {
        return alloc(reinterpret_cast<void **>(p), sizeof(T) * (size_t)std::max<int64_t>(n, 1), life);
    }
    // Frees (stream-ordered) every temporary whose life ends at or before `life`.
    void release_temps(int life) {
        size_t k = 0;
        for (auto &t : temps) {
            if (t.life <= life) {
                cudaFreeAsync(t.ptr, st);
                bytes_held -= t.bytes;
            } else {
                temps[k++] = t;
            }
        }
        temps.resize(k);
    }
    void time_begin(int kind) {
        if (!opts.record_timing) return;
        Timer t{kind, nullptr, nullptr};
        cudaEventCreate(&t.a);
        cudaEventCreate(&t.b);
        cudaEventRecord(t.a, st);
        timers.push_back(t);
    }
    void time_end() {
        if (!opts.record_timing || timers.empty()) return;
        cudaEventRecord(timers.back().b, st);
    }
    void count(int kind, int n = 1) { stats.launches[kind] += n; }
    // two 8-byte device words with one synchronisation
    cudaError_t d2h2(int64_t *dst, const int64_t *src0, const int64_t *src1) {
        int64_t *pin = static_cast<int64_t *>(pinned);
        void *dev = nullptr;
        cudaError_t e = cudaHostGetDevicePointer(&dev, pinned, 0);
        if (e == cudaSuccess) {
            k_read_words2<<<1, 32, 0, st>>>(src0, src1, static_cast<int64_t *>(dev));
            e = cudaGetLastError();
            count(SPGEMM_K_OTHER);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        dst[0] = pin[0];
        dst[1] = pin[1];
        return cudaSuccess;
    }
    cudaError_t d2h(void *dst, const void *src, size_t bytes) {
        cudaError_t e;
        void *dev = nullptr;
        if (bytes <= PIN_BYTES && (e = cudaHostGetDevicePointer(&dev, pinned, 0)) == cudaSuccess) {
            k_read_bytes<<<1, 256, 0, st>>>(static_cast<const unsigned char *>(src), static_cast<unsigned char *>(dev),
                                            (int)bytes);
            e = cudaGetLastError();
            count(SPGEMM_K_OTHER);
        } else {
            e = bytes <= PIN_BYTES ? e : cudaErrorInvalidValue;  // the pinned block holds PIN_BYTES
        }
        if (e != cudaSuccess) return e;
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        std::memcpy(dst, pinned, bytes);
        return cudaSuccess;
    }
    void release() {
        if (dense_count_done) {
            cudaStreamWaitEvent(st, dense_count_done, 0);
            cudaEventDestroy(dense_count_done);
            dense_count_done = nullptr;
        }
        for (spgemm_plan *w : waves) {
            if (w) {
                w->release();
                delete w;
            }
        }
        waves.clear();
        for (auto &t : timers) {
            if (t.a) cudaEventDestroy(t.a);
            if (t.b) cudaEventDestroy(t.b);
        }
        timers.clear();
        for (void *p : allocs) cudaFreeAsync(p, st);
        allocs.clear();
        for (auto &t : temps) cudaFreeAsync(t.ptr, st);
        temps.clear();
        bytes_held = 0;
        put_pinned(pinned);
        pinned = nullptr;
    }
};

// Largest shared-memory result capacity of the merge kernel for the plan's batch size, and
// the dense column slices (always sized for the precise method, which computes every bin-37
// row with them).
static void merge_limits(spgemm_plan *p) {
    const bool force_dense = p->opts.alloc_policy == SPGEMM_ALLOC_PRECISE;
    // leave room for the kernel's static shared memory
    const int smem_limit = (p->smem_optin > 0 ? p->smem_optin : 227 * 1024) - 1024;
    int batch = p->opts.merge_batch > 0 ? p->opts.merge_batch : 2048;
    batch = std::max(32, std::min(batch, 2048));
    p->wide_above = p->opts.merge_wide_above > 0 ? p->opts.merge_wide_above : 2048;
    int capmax = merge_max_cap(batch, smem_limit, p->wide_above);
    // the bitmap kernel when B's columns fit its bitmap and long rows are split
    p->bm_words = 0;
    p->bm_miss = 0;
    p->bm_two = 0;
    if (p->opts.merge_kernel != SPGEMM_MERGE_PATH && p->opts.long_rows == SPGEMM_LONG_ROWS_SPLIT && p->B.ncols > 0 &&
        p->B.ncols <= BM2_MAX_COLS) {
        // flat bitmap up to BM_MAX_COLS columns, the two-level index beyond
        p->bm_two = p->B.ncols > BM_MAX_COLS ? 1 : 0;
        p->bm_words = p->bm_two ? (int)((p->B.ncols + 1023) / 1024) : (int)((p->B.ncols + 31) / 32);
        const int miss = p->opts.merge_miss > 0 ? p->opts.merge_miss : 4096;
        p->bm_miss = std::max(batch, std::min(miss, 16384));
        capmax = merge_bm_max_cap(p->bm_words, p->bm_miss, smem_limit, p->wide_above, p->bm_two != 0);
    }
    if (p->opts.smem_cap_max > 0) capmax = std::min(capmax, std::max(256, p->opts.smem_cap_max));
    p->batch = batch;
    p->capmax = capmax;
    // dense column slices: B's columns cut into equal slices of at most DENSE_W_MAX columns
    // (a multiple of 32); a fill CTA holds the slice's bitmap and rank directory and a
    // compact buffer of sums, one per column of the result; dense_span narrows the slices
    p->dense_K = 0;
    p->dense_W = 0;
    p->dense_min_u = 0;
    if ((force_dense || (p->opts.dense_min_u >= 0 && p->opts.merge_kernel != SPGEMM_MERGE_PATH &&
                         p->opts.long_rows == SPGEMM_LONG_ROWS_SPLIT)) &&
        p->B.ncols > 0) {
        const int64_t n = p->B.ncols;
        int wmax = DENSE_W_MAX;
        if (p->opts.dense_span > 0) wmax = std::min(wmax, std::max(1024, p->opts.dense_span & ~31));
        const int64_t k0 = (n + wmax - 1) / wmax;
        if (k0 <= DENSE_MAX_SLICES && dense_fill_smem_bytes(wmax) <= dense_fill_max_dynamic(1)) {
            const int64_t w = ((n + k0 - 1) / k0 + 31) & ~int64_t(31);
            p->dense_W = (int)w;
            p->dense_K = (int)((n + w - 1) / w);
            p->dense_min_u = p->opts.dense_min_u > 0 ? (int64_t)p->opts.dense_min_u : 0;
            if (force_dense) p->dense_min_u = BIN_MERGE_MIN_U + 1;  // every bin-37 row
        }
    }
    // learned launch classes: 256, 512, ..., 8192, the largest capacity, and "beyond it"
    for (int g = 0; g < NUM_LAUNCH_CLASSES - 1; ++g) p->class_caps[g] = std::min(256 << g, capmax);
    p->class_caps[NUM_LAUNCH_CLASSES - 2] = capmax;
    p->class_caps[NUM_LAUNCH_CLASSES - 1] = INT32_MAX;
}

extern "C" {

spgemm_status spgemm_opts_init(spgemm_opts *o) {
    if (!o) return SPGEMM_ERR_INVALID_ARG;
    std::memset(o, 0, sizeof(*o));
    o->alloc_policy = SPGEMM_ALLOC_HYBRID;
    o->initial_cap = 256;
    o->predictor_margin = 1.0;
    return SPGEMM_OK;
}

const char *spgemm_status_string(spgemm_status s) {
    switch (s) {
        case SPGEMM_OK: return "success";
        case SPGEMM_ERR_INVALID_ARG: return "invalid argument";
        case SPGEMM_ERR_SHAPE: return "shape mismatch or unsupported dimension";
        case SPGEMM_ERR_UNSORTED: return "input CSR is malformed (unsorted/duplicate/out-of-range columns)";
        case SPGEMM_ERR_OOM: return "device out of memory";
        case SPGEMM_ERR_CUDA: return "CUDA error";
        case SPGEMM_ERR_TIMEOUT: return "bounded device wait timed out";
        case SPGEMM_ERR_INTERNAL: return "internal error";
    }
    return "unknown status";
}

}  // extern "C"

namespace {

spgemm_status check_in(const spgemm_csr_in *M) {
    if (!M) return SPGEMM_ERR_INVALID_ARG;
    if (M->nrows < 0 || M->ncols < 0 || M->nnz < 0) return SPGEMM_ERR_INVALID_ARG;
    if (M->nrows > INT32_MAX || M->ncols > INT32_MAX) return SPGEMM_ERR_SHAPE;
    if (M->rowptr_bits != 32 && M->rowptr_bits != 64) return SPGEMM_ERR_INVALID_ARG;
    if (M->rowptr_bits == 32 && M->nnz > INT32_MAX) return SPGEMM_ERR_INVALID_ARG;
    if (!M->row_ptr) return SPGEMM_ERR_INVALID_ARG;
    if (M->nnz > 0 && (!M->col_idx || !M->val)) return SPGEMM_ERR_INVALID_ARG;
    return SPGEMM_OK;
}

#define SPG_TRY(expr)                                  \
    do {                                               \
        cudaError_t _e = (expr);                       \
        if (_e != cudaSuccess) {                       \
            status = from_cuda(_e);                    \
            goto fail;                                 \
        }                                              \
    } while (0)

StageArgs stage_args(spgemm_plan *p) {
    StageArgs a;
    a.A = p->A;
    a.B = p->B;
    a.ctil_rp = p->ctil_rp;
    a.ctil_col = p->ctil_col;
    a.ctil_val = p->ctil_val;
    a.nnzc = p->nnzc;
    return a;
}

// Rows of bins lo..hi: host-known from the stage-2 summary, or (dev) a range of bin_rows whose
// ends the kernels read from the device copy of the summary.
RowSet bin_range(const spgemm_plan *p, int lo, int hi, bool dev) {
    if (dev)
        return RowSet{p->bin_rows, p->A.nrows, &p->d_summary->bin_start[lo], &p->d_summary->bin_start[hi + 1]};
    return host_rows(p->bin_rows + p->bin_start[lo], p->bin_start[hi + 1] - p->bin_start[lo]);
}

// Stage 3, bins 2..36 (bin groups 3 and 4): the heap kernel for bins 2..heap_max_u
// (one launch per range, sized to the range's widest heap), the bitonic ESC kernel
// with 32 slots for the rest of bins up to 32, and ESC for bins 33..36.  With dev the
// bin sizes are read on the device (persistent grids; every launch is made).
cudaError_t launch_short_bins(spgemm_plan *p, const StageArgs &a, bool account, bool dev = false) {
    cudaError_t e = cudaSuccess;
    const int hmax = (p->opts.heap_max_u >= 2 && p->opts.heap_max_u <= 32) ? p->opts.heap_max_u : 32;
    const int heap_nt = p->opts.heap_block > 0 ? p->opts.heap_block : 128;
    auto run = [&](int kind, auto &&launch) {
        if (account) p->time_begin(kind);
        e = launch();
        if (account) {
            p->time_end();
            p->count(kind);
        }
        return e;
    };
    for (auto &r : kHeapRanges) {
        const int lo = r[0], hi = std::min(r[1], hmax);
        if (lo > hi) continue;
        const RowSet R = bin_range(p, lo, hi, dev);
        if (R.n > 0 && run(SPGEMM_K_HEAP, [&] { return launch_heap_set(a, R, hi, heap_nt, p->st); }) != cudaSuccess)
            return e;
    }
    if (hmax < 32) {
        const RowSet R = bin_range(p, hmax + 1, 32, dev);
        if (R.n > 0 && run(SPGEMM_K_ESC, [&] { return launch_esc_set(a, R, 32, false, p->st); }) != cudaSuccess)
            return e;
    }
    for (int b = BIN_ESC_LO; b <= BIN_ESC_HI; ++b) {
        const RowSet R = bin_range(p, b, b, dev);
        if (R.n > 0 && run(SPGEMM_K_ESC, [&] { return launch_esc_set(a, R, b, false, p->st); }) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

}  // namespace

// Creates a plan bound to the current device, the library's memory pool and `stream`.
static spgemm_status plan_begin(const spgemm_opts *opts, spgemm_stream_t stream, spgemm_plan **out) {
    *out = nullptr;
    spgemm_opts o;
    if (opts) o = *opts; else spgemm_opts_init(&o);
    if (o.alloc_policy < 0 || o.alloc_policy > 3 || o.initial_cap < 1) return SPGEMM_ERR_INVALID_ARG;
    if (o.alloc_policy == SPGEMM_ALLOC_LEARNED && o.predictor == nullptr) return SPGEMM_ERR_INVALID_ARG;
    spgemm_plan *p = new (std::nothrow) spgemm_plan();
    if (!p) return SPGEMM_ERR_OOM;
    p->opts = o;
    p->st = reinterpret_cast<cudaStream_t>(stream);
    spgemm_status status = SPGEMM_OK;
    {
        SPG_TRY(cudaGetDevice(&p->device));
        SPG_TRY(get_pool(p->device, &p->pool));
        SPG_TRY(cudaDeviceGetAttribute(&p->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
        p->pinned = get_pinned();
        if (!p->pinned) {
            status = SPGEMM_ERR_OOM;
            goto fail;
        }
    }
    *out = p;
    return SPGEMM_OK;
fail:
    p->release();
    delete p;
    return status;
}

static void plan_abort(spgemm_plan *p) {
    cudaStreamSynchronize(p->st);
    p->release();
    delete p;
}

// Stages 1 and 2 on the plan's A and B (int64 row pointers on the device).
static spgemm_status plan_symbolic_core(spgemm_plan *p) {
    spgemm_status status = SPGEMM_OK;
    const spgemm_opts &o = p->opts;
    const int64_t m = p->A.nrows, nnzA = p->A.nnz;
    int64_t nblk;
    CapPolicy pol{};
    {
        SPG_TRY(p->alloc_n(&p->d_summary, 1));
        SPG_TRY(p->alloc_n(&p->d_err, 1));
        SPG_TRY(cudaMemsetAsync(p->d_summary, 0, sizeof(BinSummary), p->st));
        SPG_TRY(cudaMemsetAsync(p->d_err, 0, sizeof(int64_t), p->st));
        if (o.check_inputs) {
            // the check's result is read before any kernel indexes B through A's columns
            p->time_begin(SPGEMM_K_OTHER);
            SPG_TRY(launch_validate(p->A, &p->d_summary->status, p->st));
            SPG_TRY(launch_validate(p->B, &p->d_summary->status, p->st));
            p->time_end();
            p->count(SPGEMM_K_OTHER, 2);
            int64_t bad = 0;
            SPG_TRY(p->d2h(&bad, &p->d_summary->status, sizeof(int64_t)));
            if (bad != 0) {
                status = SPGEMM_ERR_UNSORTED;
                goto fail;
            }
        }
        // ---- stage 1: upper bound ----
        SPG_TRY(p->alloc_n(&p->S, nnzA + 1, LIFE_SYMBOLIC));
        {
            int64_t nb = std::max<int64_t>(bound_partial_size(nnzA), bin_blocks(m) + 1);
            SPG_TRY(p->alloc_n(&p->scan_partial, nb + 1));
        }
        p->time_begin(SPGEMM_K_BOUND);
        SPG_TRY(launch_bound(p->A, p->B, p->S, p->scan_partial, p->st));
        p->time_end();
        p->count(SPGEMM_K_BOUND, 3);
        merge_limits(p);
        if (o.alloc_policy == SPGEMM_ALLOC_PRECISE && p->dense_K == 0 && p->B.ncols > 0) {
            status = SPGEMM_ERR_SHAPE;  // B too wide for the column slices of the precise method
            goto fail;
        }
        if (p->dense_K > 0) {
            // which bin-37 rows go to the dense-slice kernels, and their column ranges
            SPG_TRY(p->alloc_n(&p->dense_flag, m, LIFE_SYMBOLIC));
            SPG_TRY(p->alloc_n(&p->dense_lo, m, LIFE_SYMBOLIC));
            SPG_TRY(p->alloc_n(&p->dense_hi, m, LIFE_SYMBOLIC));
            SPG_TRY(launch_dense_mark(p->A, p->B, p->S, p->dense_min_u,
                                      o.dense_span_div > 0 ? o.dense_span_div : 8, p->dense_flag, p->dense_lo,
                                      p->dense_hi, p->st));
            p->count(SPGEMM_K_OTHER);
        }
        // ---- stage 2: binning ----
        nblk = bin_blocks(m);
        SPG_TRY(p->alloc_n(&p->u, m));
        SPG_TRY(p->alloc_n(&p->bin, m));
        SPG_TRY(p->alloc_n(&p->nnzc, m));
        SPG_TRY(p->alloc_n(&p->bin_rows, m));
        SPG_TRY(p->alloc_n(&p->ctil_rp, m + 1));
        {
            int32_t *hist = nullptr;
            int64_t *capp = nullptr;
            SPG_TRY(p->alloc_n(&hist, (int64_t)NUM_BINS * nblk, LIFE_SYMBOLIC));
            SPG_TRY(p->alloc_n(&capp, nblk, LIFE_SYMBOLIC));
            pol.policy = o.alloc_policy;
            pol.initial_cap = o.initial_cap;
            pol.pred_cap = nullptr;  // learned: bin-37 sizes are set after the prediction below
            pol.cap_max = p->capmax;
            pol.dense = p->dense_flag;
            p->time_begin(SPGEMM_K_BIN);
            SPG_TRY(launch_binning(m, p->A.rp, p->S, p->S + nnzA, pol, p->u, p->bin, p->nnzc, p->bin_rows,
                                   p->ctil_rp, hist, capp, p->d_summary, p->st));
            p->time_end();
            p->count(SPGEMM_K_BIN, nblk > 0 ? 3 : 1);
        }
        // the bin sizes first: without bin-37 rows the learned launch classes and the slice
        // selection have nothing to do, and their launches are skipped
        SPG_TRY(p->d2h(&p->h_summary, p->d_summary, sizeof(BinSummary)));
        if (p->h_summary.bin_count[BIN_MERGE] > 0 && (o.alloc_policy == SPGEMM_ALLOC_LEARNED || p->dense_K > 0)) {
            if (o.alloc_policy == SPGEMM_ALLOC_LEARNED) {
                // features and predicted temporary sizes of the bin-37 rows, then the rows of C~
                // laid out again with those sizes (the binning above sized bin 37 as hybrid)
                float *X = nullptr;
                SPG_TRY(p->alloc_n(&X, m * SPGEMM_MLP_FEATURES, LIFE_SYMBOLIC));
                SPG_TRY(p->alloc_n(&p->pred_cap, m, LIFE_SYMBOLIC));
                p->time_begin(SPGEMM_K_OTHER);
                SPG_TRY(launch_row_features(p->A, p->B, X, p->st, p->S, BIN_MERGE_MIN_U, p->dense_flag));
                SPG_TRY(launch_predict_caps(predictor_params(o.predictor), X, m, nullptr,
                                            (float)(o.predictor_margin > 0 ? o.predictor_margin : 1.0),
                                            o.initial_cap, p->pred_cap, p->st, p->A.rp, p->S, BIN_MERGE_MIN_U,
                                            p->dense_flag, p->dense_K > 0 ? (int64_t)o.dense_pred_min : 0));
                pol.pred_cap = p->pred_cap;
                SPG_TRY(launch_cap_rescan(m, p->u, p->bin, pol, p->ctil_rp, p->scan_partial, &p->d_summary->sum_cap,
                                          p->st));
                p->time_end();
                p->count(SPGEMM_K_OTHER, 5);
            }
            if (o.alloc_policy == SPGEMM_ALLOC_LEARNED) {
                // group the bin-37 rows by the shared-memory class their predicted size needs
                int32_t *ccap = nullptr, *scratch = nullptr;
                SPG_TRY(p->alloc_n(&ccap, NUM_LAUNCH_CLASSES));
                SPG_TRY(cudaMemcpyAsync(ccap, p->class_caps, sizeof(p->class_caps), cudaMemcpyHostToDevice, p->st));
                SPG_TRY(p->alloc_n(&scratch, 96 + m, LIFE_SYMBOLIC));
                SPG_TRY(p->alloc_n(&p->class_order, m, LIFE_NUMERIC));
                SPG_TRY(launch_class_partition_tail(p->bin_rows, m, p->d_summary, p->pred_cap, ccap,
                                                    NUM_LAUNCH_CLASSES, p->dense_flag, scratch, p->class_order, p->st));
                p->count(SPGEMM_K_OTHER, 3);
            }
            if (p->dense_K > 0) {
                // the bin-37 rows for the dense-slice kernels, larger first, then the others
                int32_t *scratch = nullptr;
                SPG_TRY(p->alloc_n(&scratch, dense_select_scratch(m), LIFE_SYMBOLIC));
                SPG_TRY(p->alloc_n(&p->dense_order, m));
                SPG_TRY(p->alloc_n(&p->dense_rows, m));
                SPG_TRY(p->alloc_n(&p->dense_clo, m));
                SPG_TRY(p->alloc_n(&p->dense_chi, m));
                SPG_TRY(launch_dense_select(p->bin_rows, m, p->d_summary, p->u, p->dense_flag, p->dense_lo, p->dense_hi,
                                            scratch, p->dense_order, p->dense_rows, p->dense_clo, p->dense_chi, p->st));
                p->count(SPGEMM_K_OTHER, 3);
            }
            SPG_TRY(p->d2h(&p->h_summary, p->d_summary, sizeof(BinSummary)));  // class and slice counts
        }
        p->bin_start[0] = 0;
        for (int b = 0; b < NUM_BINS; ++b) p->bin_start[b + 1] = p->bin_start[b] + p->h_summary.bin_count[b];
        for (int b = 0; b < NUM_BINS; ++b) p->stats.bin_count[b] = p->h_summary.bin_count[b];
        p->stats.sum_u = p->h_summary.sum_u;
        p->stats.nnz_ctilde = p->h_summary.sum_cap;
        p->dense_n = p->dense_K > 0 ? p->h_summary.dense_count : 0;
        p->stats.rows_dense = p->dense_n;
        p->stats.dense_slices = p->dense_n > 0 ? p->dense_K : 0;
        if (p->dense_n > 0) {
            // kept for values-only replay: the slice boundaries, counts and offsets
            if (p->dense_K > 1) {
                SPG_TRY(p->alloc_n(&p->dense_bnd, p->B.nrows * (p->dense_K + 1)));
                SPG_TRY(launch_dense_bounds(p->B, p->dense_K, p->dense_W, p->dense_bnd, p->st));
                p->count(SPGEMM_K_OTHER);
            }
            SPG_TRY(p->alloc_n(&p->dense_cnt, p->dense_n * p->dense_K));
            SPG_TRY(p->alloc_n(&p->dense_soff, p->dense_n * p->dense_K));
            SPG_TRY(p->alloc_n(&p->d_queue, 3));  // work counters of the fill launches
        }
        // C~ (hybrid: u_i for bins 0..36, 256 for bin 37)
        SPG_TRY(p->alloc_n(&p->ctil_col, p->h_summary.sum_cap, LIFE_NUMERIC));
        SPG_TRY(p->alloc_n(&p->ctil_val, p->h_summary.sum_cap, LIFE_NUMERIC));
        p->bytes_ctilde += p->h_summary.sum_cap * ENTRY_BYTES;
        p->release_temps(LIFE_SYMBOLIC);
        p->dense_flag = nullptr;
        p->dense_lo = p->dense_hi = nullptr;
    }
    return SPGEMM_OK;
fail:
    return status;
}

// Widens an int32 row-pointer array into a plan-owned int64 copy when needed.
static cudaError_t plan_widen(spgemm_plan *p, const spgemm_csr_in *M, DevCSR &D) {
    D.nrows = M->nrows;
    D.ncols = M->ncols;
    D.nnz = M->nnz;
    D.col = M->col_idx;
    D.val = M->val;
    if (M->rowptr_bits == 64) {
        D.rp = static_cast<const int64_t *>(M->row_ptr);
        return cudaSuccess;
    }
    int64_t *rp = nullptr;
    cudaError_t e = p->alloc_n(&rp, M->nrows + 1);
    if (e != cudaSuccess) return e;
    e = launch_widen_rowptr(static_cast<const int32_t *>(M->row_ptr), rp, M->nrows + 1, p->st);
    p->count(SPGEMM_K_OTHER);
    D.rp = rp;
    return e;
}

extern "C" spgemm_status spgemm_symbolic(const spgemm_csr_in *A_in, const spgemm_csr_in *B_in,
                                         const spgemm_opts *opts, spgemm_stream_t stream,
                                         spgemm_plan **plan_out, int64_t *upper_bound_nnz_out) {
    if (!plan_out) return SPGEMM_ERR_INVALID_ARG;
    *plan_out = nullptr;
    spgemm_status status = check_in(A_in);
    if (status != SPGEMM_OK) return status;
    status = check_in(B_in);
    if (status != SPGEMM_OK) return status;
    if (A_in->ncols != B_in->nrows) return SPGEMM_ERR_SHAPE;
    spgemm_plan *p = nullptr;
    status = plan_begin(opts, stream, &p);
    if (status != SPGEMM_OK) return status;
    {
        SPG_TRY(plan_widen(p, A_in, p->A));
        SPG_TRY(plan_widen(p, B_in, p->B));
        status = plan_symbolic_core(p);
        if (status != SPGEMM_OK) goto fail;
    }
    if (upper_bound_nnz_out) *upper_bound_nnz_out = p->h_summary.sum_u;
    *plan_out = p;
    return SPGEMM_OK;
fail:
    plan_abort(p);
    return status;
}

namespace {

template <typename T>
cudaError_t grow_array(spgemm_plan *p, T **arr, int64_t old_n, int64_t new_cap) {
    T *n = nullptr;
    cudaError_t e = p->alloc_n(&n, new_cap);
    if (e != cudaSuccess) return e;
    if (old_n > 0 && *arr) {
        e = cudaMemcpyAsync(n, *arr, sizeof(T) * old_n, cudaMemcpyDeviceToDevice, p->st);
        if (e != cudaSuccess) return e;
    }
    *arr = n;
    return cudaSuccess;
}

// Makes room for `need` work items (keeps the first n_items).
cudaError_t reserve_items(spgemm_plan *p, int64_t need) {
    if (need <= p->items_cap) return cudaSuccess;
    const int64_t nc = std::max(need, p->items_cap + p->items_cap / 2);
    MergeItems &it = p->items;
    const int64_t n = p->n_items;
    cudaError_t e;
    if ((e = grow_array(p, &it.row, n, nc)) != cudaSuccess) return e;
    if ((e = grow_array(p, &it.clo, n, nc)) != cudaSuccess) return e;
    if ((e = grow_array(p, &it.chi, n, nc)) != cudaSuccess) return e;
    if ((e = grow_array(p, &it.src_col, n, nc)) != cudaSuccess) return e;
    if ((e = grow_array(p, &it.src_val, n, nc)) != cudaSuccess) return e;
    if ((e = grow_array(p, &it.src_len, n, nc)) != cudaSuccess) return e;
    if ((e = grow_array(p, &it.home_col, n, nc)) != cudaSuccess) return e;
    if ((e = grow_array(p, &it.home_val, n, nc)) != cudaSuccess) return e;
    if ((e = grow_array(p, &it.home_cap, n, nc)) != cudaSuccess) return e;
    if ((e = grow_array(p, &it.len, n, nc)) != cudaSuccess) return e;
    if ((e = grow_array(p, &it.ck_entry, n, nc)) != cudaSuccess) return e;
    if ((e = grow_array(p, &it.ck_off, n, nc)) != cudaSuccess) return e;
    if ((e = grow_array(p, &it.child, n, nc)) != cudaSuccess) return e;
    if ((e = grow_array(p, &it.parent, n, nc)) != cudaSuccess) return e;
    p->items_cap = nc;
    return cudaSuccess;
}

// Products per batch of a bin-37 launch with capacity `cap`: the plan's batch and
// at most what the CTA's threads hold; the merge-path form (and level-1) also at
// most the capacity, while the bitmap form admits a larger batch whenever its
// actual new columns fit.
int launch_batch(const spgemm_plan *p, int cap, bool level1) {
    const int b = std::min(p->batch, merge_batch_limit(cap, p->wide_above));
    return (p->bm_words > 0 && !level1) ? b : std::min(b, cap);
}

// Progressive rounds (Section 4.1): runs `nwork` work items (work_in, or the
// items work_base.. when work_in is null) at capacity `cap`; items that
// overflow are relaunched with twice the capacity in a fresh pool slot, and at
// the largest shared-memory capacity an overflowing item is split by column
// (default) or finished with a level-1 sequence.  With split_first the items have
// already overflowed at the largest capacity and go straight to that step.  With
// first_in_home the listed items are fresh rows whose homes in C~ hold `cap`
// entries, as the items work_base.. of a first round do.
spgemm_status run_progressive(spgemm_plan *p, const int32_t *work_in, int64_t work_base, int64_t nwork, int cap,
                              bool split_first, int32_t *ovf_count, bool first_in_home = false) {
    spgemm_status status = SPGEMM_OK;
    if (nwork <= 0) return SPGEMM_OK;
    StageArgs a = stage_args(p);
    const int capmax = p->capmax;
    const bool use_level1 = p->opts.long_rows == SPGEMM_LONG_ROWS_LEVEL1;
    const bool learned = p->opts.alloc_policy == SPGEMM_ALLOC_LEARNED;
    int32_t *list[2] = {nullptr, nullptr};
    int64_t list_cap = nwork;
    int64_t *g_cap = nullptr, *g_off = nullptr, *g_partial = nullptr, *g_total = nullptr;
    const int32_t *work = work_in;
    int which = 0;
    bool level1 = false;
    bool pending_split = split_first;
    if (pending_split && use_level1) {
        level1 = true;
        pending_split = false;
    }
    {
        SPG_TRY(p->alloc_n(&list[0], list_cap, LIFE_NUMERIC));
        SPG_TRY(p->alloc_n(&list[1], list_cap, LIFE_NUMERIC));
        while (nwork > 0) {
            int64_t novf = 0;
            const int32_t *ovf_items = nullptr;
            if (pending_split) {
                novf = nwork;
                ovf_items = work;
                pending_split = false;
            } else {
                if (nwork > list_cap) {  // more work items than the overflow lists can hold
                    list_cap = nwork;
                    SPG_TRY(p->alloc_n(&list[which], list_cap, LIFE_NUMERIC));
                    SPG_TRY(p->alloc_n(&list[which ^ 1], list_cap, LIFE_NUMERIC));
                }
                MergeLaunch L{};
                L.wide_above = p->wide_above;
                L.bm_words = p->bm_words;
                L.bm_miss = p->bm_miss;
                L.bm_two = p->bm_two;
                L.work = work;
                L.work_base = work_base;
                L.nwork = nwork;
                L.cap = cap;
                L.batch = launch_batch(p, cap, level1);
                L.level1 = level1 ? 1 : 0;
                L.ovf_list = list[which];
                L.ovf_count = ovf_count;
                L.err = p->d_err;
                const bool fresh = first_in_home && work == work_in;
                if (!level1 && work == nullptr && work_base > 0) {
                    // split round: every child already has a home (set by the split)
                } else if (fresh) {
                    // first round over fresh rows: their homes in C~ are large enough
                } else if (!level1 && p->opts.alloc_policy != SPGEMM_ALLOC_UPPER_BOUND &&
                           (work != nullptr || cap > p->opts.initial_cap || learned)) {
                    SPG_TRY(p->alloc_n(&L.pool_col, nwork * (int64_t)cap, LIFE_NUMERIC));
                    SPG_TRY(p->alloc_n(&L.pool_val, nwork * (int64_t)cap, LIFE_NUMERIC));
                    L.pool_cap = cap;
                    p->bytes_ctilde += nwork * (int64_t)cap * ENTRY_BYTES;
                }
                if (level1) {
                    SPG_TRY(p->alloc_n(&g_cap, nwork, LIFE_NUMERIC));
                    SPG_TRY(p->alloc_n(&g_off, nwork, LIFE_NUMERIC));
                    SPG_TRY(p->alloc_n(&g_partial, nwork / 2048 + 2, LIFE_NUMERIC));
                    SPG_TRY(p->alloc_n(&g_total, 1, LIFE_NUMERIC));
                    SPG_TRY(launch_level1_sizes(p->items, work, nwork, p->u, p->B.ncols, g_cap, g_off, g_partial,
                                                g_total, p->st));
                    p->count(SPGEMM_K_OTHER, 4);
                    int64_t gtot = 0;
                    SPG_TRY(p->d2h(&gtot, g_total, sizeof(int64_t)));
                    SPG_TRY(p->alloc_n(&L.g_col, gtot, LIFE_NUMERIC));
                    SPG_TRY(p->alloc_n(&L.g_val, gtot, LIFE_NUMERIC));
                    p->bytes_ctilde += gtot * ENTRY_BYTES;
                    L.g_cap = g_cap;
                    L.g_off = g_off;
                    p->stats.rows_level1 += nwork;
                }
                SPG_TRY(cudaMemsetAsync(ovf_count, 0, sizeof(int32_t), p->st));
                p->time_begin(SPGEMM_K_MERGE);
                SPG_TRY(launch_merge(a, p->items, L, p->st));
                p->time_end();
                p->count(SPGEMM_K_MERGE);
                p->stats.merge_rounds += 1;
                p->stats.item_rounds += nwork;
                int32_t n = 0;
                SPG_TRY(p->d2h(&n, ovf_count, sizeof(int32_t)));
                novf = n;
                if (novf > 0 && level1) {
                    status = SPGEMM_ERR_INTERNAL;
                    goto fail;
                }
                if (((work == nullptr && work_base == 0) || fresh) && !learned) p->stats.rows_relaunched = novf;
                if (novf == 0) break;
                ovf_items = list[which];
                if (cap < capmax) {
                    cap = std::min(capmax, cap * 2);
                    work = list[which];
                    work_base = 0;
                    nwork = novf;
                    which ^= 1;
                    continue;
                }
                if (use_level1) {
                    level1 = true;
                    work = list[which];
                    work_base = 0;
                    nwork = novf;
                    which ^= 1;
                    continue;
                }
            }
            // split every overflowed item at the median column of its sequence
            SPG_TRY(reserve_items(p, p->n_items + 2 * novf));
            int32_t *scol = nullptr;
            val_t *sval = nullptr;
            SPG_TRY(p->alloc_n(&scol, novf * (int64_t)capmax, LIFE_NUMERIC));
            SPG_TRY(p->alloc_n(&sval, novf * (int64_t)capmax, LIFE_NUMERIC));
            p->bytes_ctilde += novf * (int64_t)capmax * ENTRY_BYTES;
            p->time_begin(SPGEMM_K_OTHER);
            SPG_TRY(launch_split(ovf_items, novf, p->n_items, p->items, scol, sval, capmax, p->st));
            p->time_end();
            p->count(SPGEMM_K_OTHER, 2);
            p->stats.rows_split += novf;
            cap = capmax;
            work = nullptr;
            work_base = p->n_items;
            nwork = 2 * novf;
            p->n_items += nwork;
        }
    }
    return SPGEMM_OK;
fail:
    return status;
}

// The column bitmaps that the slices' counting pass leaves for the fill (opts.dense_keep):
// only where the count builds bitmaps and the fill is the compact form, never by default in
// the precise method, and only while they take at most a quarter of the free device memory.
// Released with the other numeric temporaries; without them the fill marks the columns again.
static void alloc_dense_keep(spgemm_plan *p) {
    p->dense_keep = nullptr;
    p->dense_keep_words = 0;
    const int want = p->opts.dense_keep;
    const int kw = p->dense_K > 0 ? dense_keep_words(p->dense_W) : 0;
    if (p->dense_n == 0 || kw == 0 || want < 0 || (want == 0 && p->opts.alloc_policy == SPGEMM_ALLOC_PRECISE))
        return;
    const int64_t words = p->dense_n * p->dense_K * (int64_t)kw;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if ((uint64_t)words * sizeof(uint32_t) > free_b / 4) return;
    if (p->alloc_n(&p->dense_keep, words, LIFE_NUMERIC) != cudaSuccess) {
        p->dense_keep = nullptr;
        return;
    }
    p->dense_keep_words = kw;
}

// Dense-slice rows: their column counts, launched first in stage 3 on their own
// stream (unless every kernel is timed), beside the heap, ESC and merge kernels; the
// event joins them before the row sizes are finalised.
static spgemm_status launch_dense_counts(spgemm_plan *p) {
    spgemm_status status = SPGEMM_OK;
    if (p->dense_n == 0 || p->h_summary.bin_count[BIN_MERGE] == 0) return SPGEMM_OK;
    {
        cudaStream_t ds = p->st;
        if (!p->opts.record_timing) {
            ds = aux_stream(p->device, p->st, DENSE_AUX);
            if (ds == nullptr) return SPGEMM_ERR_CUDA;
            cudaEvent_t go = nullptr;
            SPG_TRY(cudaEventCreateWithFlags(&go, cudaEventDisableTiming));
            cudaError_t e = cudaEventRecord(go, p->st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(ds, go, 0);
            cudaEventDestroy(go);
            SPG_TRY(e);
            SPG_TRY(cudaEventCreateWithFlags(&p->dense_count_done, cudaEventDisableTiming));
        }
        p->time_begin(SPGEMM_K_MERGE);
        SPG_TRY(launch_dense_count(p->A, p->B, p->dense_args(), p->d_err, ds));
        p->time_end();
        p->count(SPGEMM_K_MERGE);
        if (p->dense_count_done) SPG_TRY(cudaEventRecord(p->dense_count_done, ds));
    }
    return SPGEMM_OK;
fail:
    return status;
}

// Bin group 5: the merge kernel over all bin-37 rows.  Plain policies start
// every row at the initial capacity and go through the progressive rounds.  The
// learned policy launches each predicted size class with homes of the predicted
// size; a row that outgrows its prediction continues at twice its class's
// capacity (and so on up to the largest one), and rows predicted beyond the
// largest capacity that reach it are split at once.
spgemm_status run_bin37(spgemm_plan *p) {
    spgemm_status status = SPGEMM_OK;
    const int64_t n37 = p->h_summary.bin_count[BIN_MERGE];
    if (n37 == 0) return SPGEMM_OK;
    const int32_t *rows37 = p->bin_rows + p->bin_start[BIN_MERGE];
    StageArgs a = stage_args(p);
    int32_t *ovf_count = nullptr;
    const int capmax = p->capmax;
    const bool learned = p->opts.alloc_policy == SPGEMM_ALLOC_LEARNED;
    cudaEvent_t dense_done = p->dense_count_done;
    p->dense_count_done = nullptr;
    {
        SPG_TRY(reserve_items(p, n37));
        p->n_items = n37;
        SPG_TRY(p->alloc_n(&ovf_count, 1, LIFE_NUMERIC));
        SPG_TRY(launch_merge_init(rows37, n37, p->ctil_rp, p->ctil_col, p->ctil_val, p->items, p->st));
        p->count(SPGEMM_K_OTHER);
        if (!learned) {
            int cap;
            if (p->opts.alloc_policy == SPGEMM_ALLOC_UPPER_BOUND) cap = capmax;
            else cap = std::min(capmax, std::max(32, (int)p->opts.initial_cap));
            if (p->dense_n == 0) {
                status = run_progressive(p, nullptr, 0, n37, cap, false, ovf_count);
            } else if (n37 > p->dense_n) {
                // the other rows, listed after the dense ones
                status = run_progressive(p, p->dense_order + p->dense_n, 0, n37 - p->dense_n, cap, false, ovf_count,
                                         true);
            }
            if (status != SPGEMM_OK) goto fail;
        } else {
            // capacity levels of the fallback: 512, 1024, ... below the largest, then the largest
            std::vector<int> lv;
            for (int c = 512; c < capmax; c *= 2) lv.push_back(c);
            lv.push_back(capmax);
            const int nlv = (int)lv.size();
            const int SPLIT = nlv;  // target index of rows that overflow at the largest capacity
            auto level_of = [&](int c) {
                for (int k = 0; k < nlv; ++k)
                    if (lv[k] >= c) return k;
                return nlv - 1;
            };
            std::vector<int32_t *> lists(nlv + 1, nullptr);
            int32_t *counts = nullptr;
            for (int k = 0; k <= nlv; ++k) SPG_TRY(p->alloc_n(&lists[k], n37, LIFE_NUMERIC));
            SPG_TRY(p->alloc_n(&counts, nlv + 1, LIFE_NUMERIC));
            SPG_TRY(cudaMemsetAsync(counts, 0, sizeof(int32_t) * (nlv + 1), p->st));
            // the classes are independent: without per-kernel timing they run on auxiliary
            // streams, largest capacity first, and the plan's stream waits for all of them
            const bool concurrent = !p->opts.record_timing;
            cudaEvent_t ready = nullptr;
            std::vector<cudaEvent_t> joins;
            if (concurrent) {
                SPG_TRY(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
                joins.push_back(ready);
                SPG_TRY(cudaEventRecord(ready, p->st));
            }
            int64_t class_off[NUM_LAUNCH_CLASSES + 1] = {0};
            for (int g = 0; g < NUM_LAUNCH_CLASSES; ++g) class_off[g + 1] = class_off[g] + p->h_summary.class_count[g];
            int nlaunched = 0;
            for (int gi = NUM_LAUNCH_CLASSES - 1; gi >= 0; --gi) {
                const int g = concurrent ? gi : NUM_LAUNCH_CLASSES - 1 - gi;
                const int64_t cnt = p->h_summary.class_count[g];
                const int64_t off = class_off[g];
                if (cnt == 0) continue;
                cudaStream_t cs = p->st;
                if (concurrent) {
                    cs = aux_stream(p->device, p->st, nlaunched % DENSE_AUX);
                    if (cs == nullptr) {
                        status = SPGEMM_ERR_CUDA;
                        goto fail;
                    }
                    SPG_TRY(cudaStreamWaitEvent(cs, ready, 0));
                }
                ++nlaunched;
                const bool beyond = p->class_caps[g] == INT32_MAX;
                const int ccap = std::min(capmax, beyond ? capmax : p->class_caps[g]);
                const int tgt = beyond ? SPLIT : level_of(std::min(2 * ccap, capmax));
                MergeLaunch L{};
                L.wide_above = p->wide_above;
                L.bm_words = p->bm_words;
                L.bm_miss = p->bm_miss;
                L.bm_two = p->bm_two;
                L.work = p->class_order + off;
                L.nwork = cnt;
                L.cap = ccap;
                L.batch = launch_batch(p, ccap, false);
                L.ovf_list = lists[tgt];
                L.ovf_count = counts + tgt;
                L.err = p->d_err;
                p->time_begin(SPGEMM_K_MERGE);
                SPG_TRY(launch_merge(a, p->items, L, cs));
                p->time_end();
                p->count(SPGEMM_K_MERGE);
                p->stats.merge_rounds += 1;
                p->stats.item_rounds += cnt;
                if (concurrent) {
                    cudaEvent_t done = nullptr;
                    SPG_TRY(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
                    joins.push_back(done);
                    SPG_TRY(cudaEventRecord(done, cs));
                    SPG_TRY(cudaStreamWaitEvent(p->st, done, 0));
                }
            }
            for (cudaEvent_t ev : joins) cudaEventDestroy(ev);  // released once their work is done
            std::vector<int32_t> hc(nlv + 1, 0);
            SPG_TRY(p->d2h(hc.data(), counts, sizeof(int32_t) * (nlv + 1)));
            int64_t fell = 0;
            for (int k = 0; k < nlv; ++k) fell += hc[k];
            p->stats.rows_fallback = fell;  // rows whose result outgrew the predicted size
            p->stats.rows_relaunched = fell;
            // levels below the largest capacity, in ascending order: each launch's
            // overflow lands on a higher level
            bool stale = false;  // a level was launched since hc was read
            for (int k = 0; k + 1 < nlv; ++k) {
                int32_t nk = hc[k];
                if (stale) SPG_TRY(p->d2h(&nk, counts + k, sizeof(int32_t)));
                if (nk == 0) continue;
                stale = true;
                const int tgt = level_of(std::min(2 * lv[k], capmax));
                MergeLaunch L{};
                L.wide_above = p->wide_above;
                L.bm_words = p->bm_words;
                L.bm_miss = p->bm_miss;
                L.bm_two = p->bm_two;
                L.work = lists[k];
                L.nwork = nk;
                L.cap = lv[k];
                L.batch = launch_batch(p, lv[k], false);
                L.ovf_list = lists[tgt];
                L.ovf_count = counts + tgt;
                L.err = p->d_err;
                SPG_TRY(p->alloc_n(&L.pool_col, (int64_t)nk * lv[k], LIFE_NUMERIC));
                SPG_TRY(p->alloc_n(&L.pool_val, (int64_t)nk * lv[k], LIFE_NUMERIC));
                L.pool_cap = lv[k];
                p->bytes_ctilde += (int64_t)nk * lv[k] * ENTRY_BYTES;
                p->time_begin(SPGEMM_K_MERGE);
                SPG_TRY(launch_merge(a, p->items, L, p->st));
                p->time_end();
                p->count(SPGEMM_K_MERGE);
                p->stats.merge_rounds += 1;
                p->stats.item_rounds += nk;
            }
            if (stale) SPG_TRY(p->d2h(hc.data(), counts, sizeof(int32_t) * (nlv + 1)));
            status = run_progressive(p, lists[nlv - 1], 0, hc[nlv - 1], capmax, false, ovf_count);
            if (status != SPGEMM_OK) goto fail;
            status = run_progressive(p, lists[SPLIT], 0, hc[SPLIT], capmax, true, ovf_count);
            if (status != SPGEMM_OK) goto fail;
        }
        if (dense_done) {
            SPG_TRY(cudaStreamWaitEvent(p->st, dense_done, 0));
            cudaEventDestroy(dense_done);
            dense_done = nullptr;
        }
        SPG_TRY(launch_dense_rows(p->items, p->dense_args(), p->st));
        if (p->dense_n > 0) p->count(SPGEMM_K_MERGE);
        // the error word is read with nnz(C), after the row scan
        SPG_TRY(launch_finalize37(n37, p->items, p->nnzc, p->d_err, p->st));
        p->count(SPGEMM_K_OTHER);
    }
    return status;
fail:
    if (dense_done) {
        cudaStreamWaitEvent(p->st, dense_done, 0);
        cudaEventDestroy(dense_done);
    }
    return status;
}

}  // namespace

static spgemm_status run_precise(spgemm_plan *p, spgemm_csr_out *C_out);

extern "C" spgemm_status spgemm_numeric(spgemm_plan *p, spgemm_csr_out *C_out) {
    if (!p || !C_out || p->wave_mode) return SPGEMM_ERR_INVALID_ARG;
    if (p->numeric_done) {
        *C_out = p->C;
        return SPGEMM_OK;
    }
    if (p->opts.alloc_policy == SPGEMM_ALLOC_PRECISE) return run_precise(p, C_out);
    spgemm_status status = SPGEMM_OK;
    const int64_t m = p->A.nrows;
    StageArgs a = stage_args(p);
    {
        // ---- stage 3: the dense-slice rows' counts, then bin groups 3 (heap) and 4 (bitonic ESC) ----
        if (p->h_summary.bin_count[BIN_MERGE] > 0) alloc_dense_keep(p);
        status = launch_dense_counts(p);
        if (status != SPGEMM_OK) goto fail;
        SPG_TRY(launch_short_bins(p, a, true));
        // ---- stage 3: bin group 5 (merge, progressive) ----
        status = run_bin37(p);
        if (status != SPGEMM_OK) goto fail;
        // ---- stage 4: arrange ----
        SPG_TRY(p->alloc_n(&p->C.row_ptr, m + 1));
        p->time_begin(SPGEMM_K_SCAN);
        SPG_TRY(launch_row_scan(m, p->nnzc, p->C.row_ptr, p->scan_partial, p->st));
        p->time_end();
        p->count(SPGEMM_K_SCAN, 3);
        int64_t nnzC = 0;
        {
            // nnz(C) and the device error word of stage 3, with one synchronisation
            int64_t both[2] = {0, 0};
            SPG_TRY(p->d2h2(both, p->C.row_ptr + m, p->d_err));
            nnzC = both[0];
            if (both[1] != 0) {
                status = SPGEMM_ERR_INTERNAL;
                goto fail;
            }
        }
        SPG_TRY(p->alloc_n(&p->C.col_idx, nnzC));
        SPG_TRY(p->alloc_n(&p->C.val, nnzC));
        cudaEvent_t fill_done = nullptr;
        if (p->dense_n > 0) {
            // the dense-slice rows write their values straight into C, beside the copy of
            // the other rows (their own stream unless every kernel is timed)
            cudaStream_t ds = p->st;
            if (!p->opts.record_timing) {
                ds = aux_stream(p->device, p->st, DENSE_AUX);
                if (ds == nullptr) {
                    status = SPGEMM_ERR_CUDA;
                    goto fail;
                }
                cudaEvent_t go = nullptr;
                SPG_TRY(cudaEventCreateWithFlags(&go, cudaEventDisableTiming));
                cudaError_t e = cudaEventRecord(go, p->st);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(ds, go, 0);
                cudaEventDestroy(go);
                SPG_TRY(e);
                SPG_TRY(cudaEventCreateWithFlags(&fill_done, cudaEventDisableTiming));
            }
            p->time_begin(SPGEMM_K_MERGE);
            cudaError_t e = launch_dense_fill(p->A, p->B, p->dense_args(), p->C.row_ptr, p->C.col_idx, p->C.val,
                                              p->d_err, ds);
            if (e == cudaSuccess && fill_done) e = cudaEventRecord(fill_done, ds);
            p->time_end();
            p->count(SPGEMM_K_MERGE);
            if (e != cudaSuccess) {
                if (fill_done) cudaEventDestroy(fill_done);
                status = from_cuda(e);
                goto fail;
            }
        }
        p->time_begin(SPGEMM_K_ARRANGE);
        {
            const int64_t s0 = p->bin_start[1], s1 = p->bin_start[BIN_MERGE];
            SPG_TRY(launch_arrange_short(a, p->bin_rows + s0, s1 - s0, p->bin, p->C.row_ptr, p->C.col_idx,
                                         p->C.val, p->st));
            if (s1 > s0) p->count(SPGEMM_K_ARRANGE);
            const int64_t n37 = p->h_summary.bin_count[BIN_MERGE];
            SPG_TRY(launch_arrange_long(p->items, n37, p->C.row_ptr, p->C.col_idx, p->C.val, p->st));
            if (n37 > 0) p->count(SPGEMM_K_ARRANGE);
        }
        p->time_end();
        if (fill_done) {
            SPG_TRY(cudaStreamWaitEvent(p->st, fill_done, 0));
            cudaEventDestroy(fill_done);
        }
        p->C.nrows = m;
        p->C.ncols = p->B.ncols;
        p->C.nnz = nnzC;
        p->stats.nnz_c = nnzC;
        p->stats.bytes_ctilde = p->bytes_ctilde;
        p->numeric_done = true;
        p->release_temps(LIFE_NUMERIC);
        p->dense_keep = nullptr;  // released above: a values-only replay marks the columns from C
        p->dense_keep_words = 0;
        *C_out = p->C;
    }
    return SPGEMM_OK;
fail:
    return status;
}

extern "C" spgemm_status spgemm_merge_micro(int32_t method, int32_t threads, int32_t value_bytes,
                                            const int32_t *keys, const void *vals, int64_t n, int32_t l,
                                            int32_t *out_keys, void *out_vals, spgemm_stream_t stream) {
    if (method < 0 || method > 2 || !keys || !out_keys || n <= 0 || l < 1 || (l & (l - 1)) != 0)
        return SPGEMM_ERR_INVALID_ARG;
    if (threads != 64 && threads != 128 && threads != 256 && threads != 512 && threads != 1024)
        return SPGEMM_ERR_INVALID_ARG;
    if (value_bytes != 0 && value_bytes != 4 && value_bytes != 8) return SPGEMM_ERR_INVALID_ARG;
    if (value_bytes != 0 && (!vals || !out_vals)) return SPGEMM_ERR_INVALID_ARG;
    if (n % (2 * (int64_t)l) != 0 || n / (2 * (int64_t)l) > INT32_MAX) return SPGEMM_ERR_INVALID_ARG;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return from_cuda(e);
    if (merge_micro_smem(l, value_bytes) > optin - 1024) return SPGEMM_ERR_INVALID_ARG;
    e = launch_merge_micro(method, threads, value_bytes, keys, vals, n, l, out_keys, out_vals,
                           reinterpret_cast<cudaStream_t>(stream));
    return from_cuda(e);
}

namespace spg {
static std::vector<CheckReader> &check_readers() {
    static std::vector<CheckReader> readers;
    return readers;
}
int register_check_reader(CheckReader read) {
    check_readers().push_back(read);
    return 0;
}
}  // namespace spg

extern "C" spgemm_status spgemm_check_status(int64_t *code_out, int32_t reset) {
    if (!code_out) return SPGEMM_ERR_INVALID_ARG;
#ifdef SPGEMM_CHECK
    int64_t first = 0;
    for (spg::CheckReader read : spg::check_readers()) {
        unsigned long long w = 0;
        cudaError_t e = read(&w, reset != 0);
        if (e != cudaSuccess) return from_cuda(e);
        if (first == 0 && w != 0) first = (int64_t)w;
    }
    *code_out = first;
#else
    (void)reset;
    *code_out = -1;
#endif
    return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_pool_trim(int32_t device, int64_t keep_bytes) {
    if (device < 0 || keep_bytes < 0) return SPGEMM_ERR_INVALID_ARG;
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        for (auto &q : g_pools)
            if (q.device == device) pool = q.pool;
    }
    if (pool == nullptr) return SPGEMM_OK;
    return from_cuda(cudaMemPoolTrimTo(pool, (size_t)keep_bytes));
}

extern "C" spgemm_status spgemm_free(spgemm_plan *p) {
    if (!p) return SPGEMM_OK;
    p->release();
    delete p;
    return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_plan_stats(spgemm_plan *p, spgemm_stats *out) {
    if (!p || !out) return SPGEMM_ERR_INVALID_ARG;
    if (!p->timers.empty()) {
        cudaError_t e = cudaStreamSynchronize(p->st);
        if (e != cudaSuccess) return from_cuda(e);
        for (int k = 0; k < SPGEMM_K_COUNT; ++k) p->stats.kernel_ms[k] = 0.f;
        for (auto &t : p->timers) {
            float ms = 0.f;
            if (t.a && t.b && cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) p->stats.kernel_ms[t.kind] += ms;
        }
    }
    p->stats.peak_bytes = p->bytes_peak;
    p->stats.held_bytes = p->bytes_held;
    *out = p->stats;
    for (spgemm_plan *w : p->waves) {  // wave mode: sums over the waves
        spgemm_stats ws;
        spgemm_status st = spgemm_plan_stats(w, &ws);
        if (st != SPGEMM_OK) return st;
        for (int b = 0; b < NUM_BINS; ++b) out->bin_count[b] += ws.bin_count[b];
        out->nnz_ctilde += ws.nnz_ctilde;
        out->nnz_c += ws.nnz_c;
        out->merge_rounds += ws.merge_rounds;
        out->item_rounds += ws.item_rounds;
        out->rows_relaunched += ws.rows_relaunched;
        out->rows_level1 += ws.rows_level1;
        out->rows_split += ws.rows_split;
        out->rows_fallback += ws.rows_fallback;
        out->bytes_ctilde += ws.bytes_ctilde;
        out->held_bytes += ws.held_bytes;
        out->rows_dense += ws.rows_dense;
        out->dense_slices = std::max(out->dense_slices, ws.dense_slices);
        out->alloc_host_ms += ws.alloc_host_ms;
        out->allocs += ws.allocs;
        for (int k = 0; k < SPGEMM_K_COUNT; ++k) {
            out->launches[k] += ws.launches[k];
            out->kernel_ms[k] += ws.kernel_ms[k];
        }
    }
    return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_batched_waves(spgemm_plan *p, int64_t *n) {
    if (!p || !n) return SPGEMM_ERR_INVALID_ARG;
    *n = p->wave_mode ? (int64_t)p->wave_start.size() - 1 : 1;
    return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_batched_wave(spgemm_plan *p, int64_t i, spgemm_plan **sub, int64_t *first_pair) {
    if (!p || !sub || i < 0) return SPGEMM_ERR_INVALID_ARG;
    if (!p->wave_mode) {
        if (i != 0) return SPGEMM_ERR_INVALID_ARG;
        *sub = p;
        if (first_pair) *first_pair = 0;
        return SPGEMM_OK;
    }
    if (i >= (int64_t)p->waves.size()) return SPGEMM_ERR_INVALID_ARG;
    *sub = p->waves[i];
    if (first_pair) *first_pair = p->wave_start[i];
    return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_batched_wave_pairs(spgemm_plan *p, int64_t *order) {
    if (!p || !order) return SPGEMM_ERR_INVALID_ARG;
    for (int64_t q = 0; q < p->npairs; ++q) order[q] = p->wave_mode ? p->wave_order[q] : q;
    return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_plan_arrays_get(spgemm_plan *p, spgemm_plan_arrays *out) {
    if (!p || !out || p->wave_mode) return SPGEMM_ERR_INVALID_ARG;
    out->nrows = p->A.nrows;
    out->u = p->u;
    out->bin = p->bin;
    out->bin_rows = p->bin_rows;
    out->bin_start = p->bin_start;
    out->ctilde_row_ptr = p->ctil_rp;
    out->row_nnz = p->nnzc;
    return SPGEMM_OK;
}

// ---------------------------------------------------------------------------
// Batched products: block-diagonal concatenation, one pipeline for all pairs.
// ---------------------------------------------------------------------------

extern "C" spgemm_status spgemm_batched_symbolic(int64_t npairs, const spgemm_csr_in *A, const spgemm_csr_in *B,
                                                 const spgemm_opts *opts, spgemm_stream_t stream,
                                                 spgemm_plan **plan_out, int64_t *upper_bound_nnz_out) {
    if (!plan_out || npairs < 1 || !A || !B) return SPGEMM_ERR_INVALID_ARG;
    *plan_out = nullptr;
    std::vector<PairDesc> hd((size_t)npairs);
    std::vector<int64_t> moff(npairs), koff(npairs), aoff(npairs), boff(npairs);
    int64_t M = 0, K = 0, N = 0, annz = 0, bnnz = 0;
    for (int64_t i = 0; i < npairs; ++i) {
        spgemm_status st = check_in(&A[i]);
        if (st != SPGEMM_OK) return st;
        st = check_in(&B[i]);
        if (st != SPGEMM_OK) return st;
        if (A[i].ncols != B[i].nrows) return SPGEMM_ERR_SHAPE;
        PairDesc &d = hd[i];
        d.a_rp = A[i].row_ptr;
        d.b_rp = B[i].row_ptr;
        d.a_col = A[i].col_idx;
        d.b_col = B[i].col_idx;
        d.a_val = A[i].val;
        d.b_val = B[i].val;
        d.a_bits = A[i].rowptr_bits;
        d.b_bits = B[i].rowptr_bits;
        d.m = A[i].nrows;
        d.k = A[i].ncols;
        d.n = B[i].ncols;
        d.moff = moff[i] = M;
        d.koff = koff[i] = K;
        d.annz_off = aoff[i] = annz;
        d.bnnz_off = boff[i] = bnnz;
        d.annz = A[i].nnz;
        d.bnnz = B[i].nnz;
        M += d.m;
        K += d.k;
        N = std::max(N, d.n);  // B_i keeps its own column numbers
        annz += d.annz;
        bnnz += d.bnnz;
    }
    if (M > INT32_MAX || K > INT32_MAX || N > INT32_MAX) return SPGEMM_ERR_SHAPE;
    spgemm_plan *p = nullptr;
    spgemm_status status = plan_begin(opts, stream, &p);
    if (status != SPGEMM_OK) return status;
    {
        p->npairs = npairs;
        p->h_pairs = hd;
        SPG_TRY(p->alloc_n(&p->d_pairs, npairs));
        SPG_TRY(p->alloc_n(&p->d_moff, npairs));
        SPG_TRY(p->alloc_n(&p->d_koff, npairs));
        SPG_TRY(p->alloc_n(&p->d_annz_off, npairs));
        SPG_TRY(p->alloc_n(&p->d_bnnz_off, npairs));
        // pageable sources: the copies are staged before the calls return
        SPG_TRY(cudaMemcpyAsync(p->d_pairs, hd.data(), sizeof(PairDesc) * npairs, cudaMemcpyHostToDevice, p->st));
        SPG_TRY(cudaMemcpyAsync(p->d_moff, moff.data(), sizeof(int64_t) * npairs, cudaMemcpyHostToDevice, p->st));
        SPG_TRY(cudaMemcpyAsync(p->d_koff, koff.data(), sizeof(int64_t) * npairs, cudaMemcpyHostToDevice, p->st));
        SPG_TRY(cudaMemcpyAsync(p->d_annz_off, aoff.data(), sizeof(int64_t) * npairs, cudaMemcpyHostToDevice, p->st));
        SPG_TRY(cudaMemcpyAsync(p->d_bnnz_off, boff.data(), sizeof(int64_t) * npairs, cudaMemcpyHostToDevice, p->st));
        const int64_t budget = p->opts.wave_mproducts < 0 ? INT64_MAX
                               : (int64_t)(p->opts.wave_mproducts > 0 ? p->opts.wave_mproducts : 1024) * 1000000;
        if (npairs > 1 && npairs <= 65535 && budget < INT64_MAX) {
            // products and a lower bound of nnz(C_i) of every pair, then waves
            int64_t *d_prod = nullptr, *d_clow = nullptr;
            SPG_TRY(p->alloc_n(&d_prod, npairs, LIFE_SYMBOLIC));
            SPG_TRY(p->alloc_n(&d_clow, npairs, LIFE_SYMBOLIC));
            SPG_TRY(launch_pair_products(p->d_pairs, npairs, d_prod, d_clow, p->st));
            p->count(SPGEMM_K_OTHER);
            std::vector<int64_t> prod(npairs), clow(npairs);
            SPG_TRY(cudaStreamSynchronize(p->st));
            SPG_TRY(cudaMemcpy(prod.data(), d_prod, sizeof(int64_t) * npairs, cudaMemcpyDeviceToHost));
            SPG_TRY(cudaMemcpy(clow.data(), d_clow, sizeof(int64_t) * npairs, cudaMemcpyDeviceToHost));
            // largest pairs first: they run while few results are resident.  A wave grows
            // while its products (which bound its temporary entries) fit the budget and do
            // not exceed the entries of the results still to come (sum of the lower bounds
            // of the later pairs), so the peak stays near the size of all results; waves
            // of up to WAVE_MIN products are always allowed, which bounds their number.
            constexpr int64_t WAVE_MIN = 32 * 1000000LL;
            std::vector<int64_t> order(npairs);
            for (int64_t i = 0; i < npairs; ++i) order[i] = i;
            std::stable_sort(order.begin(), order.end(),
                             [&](int64_t x, int64_t y) { return prod[x] > prod[y]; });
            std::vector<int64_t> after(npairs + 1, 0);  // after[q] = sum of clow over positions >= q
            for (int64_t q = npairs - 1; q >= 0; --q) after[q] = after[q + 1] + clow[order[q]];
            std::vector<int64_t> starts{0};
            int64_t acc = 0, total = 0;
            for (int64_t q = 0; q < npairs; ++q) {
                const int64_t pq = prod[order[q]];
                const int64_t grown = acc + pq;
                if (acc > 0 && (grown > budget || (grown > WAVE_MIN && grown > after[q + 1]))) {
                    starts.push_back(q);
                    acc = 0;
                }
                acc += pq;
                total += pq;
            }
            starts.push_back(npairs);
            if (starts.size() > 2) {
                p->wave_mode = true;
                p->wave_order = order;
                for (int64_t q = 0; q < npairs; ++q) {
                    p->wave_A.push_back(A[order[q]]);
                    p->wave_B.push_back(B[order[q]]);
                }
                p->wave_start = starts;
                p->h_summary.sum_u = total;
                p->stats.sum_u = total;
                p->release_temps(LIFE_SYMBOLIC);
                if (upper_bound_nnz_out) *upper_bound_nnz_out = total;
                *plan_out = p;
                return SPGEMM_OK;
            }
        }
        SPG_TRY(p->alloc_n(&p->cat_a_rp, M + 1));
        SPG_TRY(p->alloc_n(&p->cat_b_rp, K + 1));
        SPG_TRY(p->alloc_n(&p->cat_a_col, annz));
        SPG_TRY(p->alloc_n(&p->cat_a_val, annz));
        SPG_TRY(p->alloc_n(&p->cat_b_col, bnnz));
        SPG_TRY(p->alloc_n(&p->cat_b_val, bnnz));
        p->time_begin(SPGEMM_K_OTHER);
        SPG_TRY(launch_concat(p->d_pairs, npairs, p->d_moff, p->d_koff, p->d_annz_off, p->d_bnnz_off, M, K, annz, bnnz,
                              p->cat_a_rp, p->cat_a_col, p->cat_a_val, p->cat_b_rp, p->cat_b_col, p->cat_b_val, false,
                              p->st));
        p->time_end();
        p->count(SPGEMM_K_OTHER, 2);
        p->A = DevCSR{M, K, annz, p->cat_a_rp, p->cat_a_col, p->cat_a_val};
        p->B = DevCSR{K, N, bnnz, p->cat_b_rp, p->cat_b_col, p->cat_b_val};
        status = plan_symbolic_core(p);
        if (status != SPGEMM_OK) goto fail;
    }
    if (upper_bound_nnz_out) *upper_bound_nnz_out = p->h_summary.sum_u;
    *plan_out = p;
    return SPGEMM_OK;
fail:
    plan_abort(p);
    return status;
}

// Wave mode: every wave is a batched product of its own, made, computed and
// stripped of its temporaries before the next one starts.
static spgemm_status batched_numeric_waves(spgemm_plan *p, spgemm_csr_out *C_out) {
    spgemm_opts o = p->opts;
    o.wave_mproducts = -1;
    int64_t held_before = 0;
    for (spgemm_plan *w : p->waves) held_before += w->bytes_held;
    const int nw = (int)p->wave_start.size() - 1;
    std::vector<spgemm_csr_out> outs(p->npairs);
    for (int w = 0; w < nw; ++w) {
        const int64_t s0 = p->wave_start[w], n = p->wave_start[w + 1] - s0;
        spgemm_status st = SPGEMM_OK;
        if (w >= (int)p->waves.size()) {
            spgemm_plan *sub = nullptr;
            st = spgemm_batched_symbolic(n, p->wave_A.data() + s0, p->wave_B.data() + s0, &o,
                                         reinterpret_cast<spgemm_stream_t>(p->st), &sub, nullptr);
            if (st != SPGEMM_OK) return st;
            p->waves.push_back(sub);
            st = spgemm_batched_numeric(sub, outs.data() + s0);
            if (st != SPGEMM_OK) return st;
            p->bytes_peak = std::max(p->bytes_peak, held_before + sub->bytes_peak);
            held_before += sub->bytes_held;
        } else {
            st = spgemm_batched_numeric(p->waves[w], outs.data() + s0);  // finished earlier
            if (st != SPGEMM_OK) return st;
        }
    }
    p->batch_out.resize(p->npairs);
    for (int64_t q = 0; q < p->npairs; ++q) p->batch_out[p->wave_order[q]] = outs[q];
    for (int64_t i = 0; i < p->npairs; ++i) C_out[i] = p->batch_out[i];
    p->numeric_done = true;
    return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_batched_numeric(spgemm_plan *p, spgemm_csr_out *C_out) {
    if (!p || !C_out || p->npairs < 1) return SPGEMM_ERR_INVALID_ARG;
    if (!p->batch_out.empty()) {
        for (int64_t i = 0; i < p->npairs; ++i) C_out[i] = p->batch_out[i];
        return SPGEMM_OK;
    }
    if (p->wave_mode) return batched_numeric_waves(p, C_out);
    spgemm_csr_out whole;
    spgemm_status status = spgemm_numeric(p, &whole);
    if (status != SPGEMM_OK) return status;
    {
        const int64_t M = p->A.nrows, np = p->npairs;
        SPG_TRY(p->alloc_n(&p->split_rp, M + np));
        p->time_begin(SPGEMM_K_OTHER);
        SPG_TRY(launch_split_out(p->d_pairs, np, whole.row_ptr, M, p->split_rp, p->st));
        p->time_end();
        p->count(SPGEMM_K_OTHER);
        // C_i's first entry in the concatenation: read every pair's first row pointer once
        std::vector<int64_t> first(np + 1);
        int64_t *d_first = nullptr;
        SPG_TRY(p->alloc_n(&d_first, np + 1));
        SPG_TRY(launch_gather_first(p->d_pairs, np, whole.row_ptr, M, d_first, p->st));
        SPG_TRY(cudaStreamSynchronize(p->st));
        SPG_TRY(cudaMemcpy(first.data(), d_first, sizeof(int64_t) * (np + 1), cudaMemcpyDeviceToHost));
        p->batch_out.resize(np);
        for (int64_t i = 0; i < np; ++i) {
            const PairDesc &d = p->h_pairs[i];
            spgemm_csr_out &c = p->batch_out[i];
            c.nrows = d.m;
            c.ncols = d.n;
            c.nnz = first[i + 1] - first[i];
            c.row_ptr = p->split_rp + d.moff + i;
            c.col_idx = whole.col_idx + first[i];
            c.val = whole.val + first[i];
            C_out[i] = c;
        }
    }
    return SPGEMM_OK;
fail:
    return status;
}

// ---------------------------------------------------------------------------
// Values-only replay (capturable): same structure, new values of A and B.
// ---------------------------------------------------------------------------

static spgemm_status prepare_replay(spgemm_plan *p) {
    spgemm_status status = SPGEMM_OK;
    const int64_t n37 = p->h_summary.bin_count[BIN_MERGE];
    if (p->opts.alloc_policy == SPGEMM_ALLOC_PRECISE) {
        // every bin-37 row is a dense-slice row, replayed by the fill kernel
        p->replay_ready = true;
        return SPGEMM_OK;
    }
    // rows finished with a level-1 sequence can be longer than any shared-memory slice
    if (p->stats.rows_level1 > 0) return SPGEMM_ERR_INVALID_ARG;
    {
        const int64_t nleaves = p->n_items - p->stats.rows_split - p->dense_n;
        int32_t *scratch = nullptr, *ccap = nullptr;
        const int caps[NUM_REPLAY_CLASSES] = {1024, 4096, std::max(4096, p->capmax)};
        for (int g = 0; g < NUM_REPLAY_CLASSES; ++g) p->leaf_cap[g] = caps[g];
        SPG_TRY(p->alloc_n(&ccap, NUM_REPLAY_CLASSES));
        SPG_TRY(cudaMemcpyAsync(ccap, caps, sizeof(caps), cudaMemcpyHostToDevice, p->st));
        SPG_TRY(p->alloc_n(&scratch, 96));
        SPG_TRY(cudaMemsetAsync(scratch, 0, sizeof(int32_t) * 96, p->st));
        ReplayLeaves &lv = p->leaves;
        SPG_TRY(p->alloc_n(&lv.row, nleaves));
        SPG_TRY(p->alloc_n(&lv.clo, nleaves));
        SPG_TRY(p->alloc_n(&lv.chi, nleaves));
        SPG_TRY(p->alloc_n(&lv.c_off, nleaves));
        SPG_TRY(p->alloc_n(&lv.len, nleaves));
        SPG_TRY(p->alloc_n(&p->leaf_order, nleaves));
        int32_t *count = scratch, *start = scratch + 32, *cursor = scratch + 64;
        SPG_TRY(launch_replay_leaves(n37, p->items, p->C.row_ptr, ccap, NUM_REPLAY_CLASSES, count, start, cursor, lv,
                                     p->leaf_order, p->d_err, false, p->st));
        int32_t hc[NUM_REPLAY_CLASSES] = {0};
        SPG_TRY(p->d2h(hc, count, sizeof(hc)));
        int32_t hs[NUM_REPLAY_CLASSES];
        int32_t acc = 0;
        for (int g = 0; g < NUM_REPLAY_CLASSES; ++g) {
            hs[g] = acc;
            p->leaf_count[g] = hc[g];
            acc += hc[g];
        }
        if (acc != nleaves) return SPGEMM_ERR_INTERNAL;
        SPG_TRY(cudaMemcpyAsync(start, hs, sizeof(hs), cudaMemcpyHostToDevice, p->st));
        SPG_TRY(launch_replay_leaves(n37, p->items, p->C.row_ptr, ccap, NUM_REPLAY_CLASSES, count, start, cursor, lv,
                                     p->leaf_order, p->d_err, true, p->st));
        SPG_TRY(cudaStreamSynchronize(p->st));
        p->replay_ready = true;
    }
    return SPGEMM_OK;
fail:
    return status;
}

extern "C" spgemm_status spgemm_numeric_replay(spgemm_plan *p) {
    if (!p || !p->numeric_done) return SPGEMM_ERR_INVALID_ARG;
    if (p->wave_mode) {
        for (spgemm_plan *w : p->waves) {
            spgemm_status st = spgemm_numeric_replay(w);
            if (st != SPGEMM_OK) return st;
        }
        return SPGEMM_OK;
    }
    spgemm_status status = SPGEMM_OK;
    if (!p->replay_ready) {
        status = prepare_replay(p);
        if (status != SPGEMM_OK) return status;
    }
    {
        if (p->npairs > 0) {
            // refresh the concatenated values from the pairs' inputs
            SPG_TRY(launch_concat(p->d_pairs, p->npairs, p->d_moff, p->d_koff, p->d_annz_off, p->d_bnnz_off,
                                  p->A.nrows, p->B.nrows, p->A.nnz, p->B.nnz, p->cat_a_rp, p->cat_a_col,
                                  p->cat_a_val, p->cat_b_rp, p->cat_b_col, p->cat_b_val, true, p->st));
        }
        // bins 2..36: the heap and bitonic-ESC kernels write straight into C
        StageArgs a = stage_args(p);
        a.ctil_rp = p->C.row_ptr;
        a.ctil_col = p->C.col_idx;
        a.ctil_val = p->C.val;
        SPG_TRY(launch_short_bins(p, a, false));
        // bin 1: the single product of each row
        {
            const int64_t s0 = p->bin_start[1], s1 = p->bin_start[2];
            SPG_TRY(launch_arrange_short(a, p->bin_rows + s0, s1 - s0, p->bin, p->C.row_ptr, p->C.col_idx, p->C.val,
                                         p->st));
        }
        // bin 37: every leaf fuses its products into its known columns
        int64_t off = 0;
        for (int g = 0; g < NUM_REPLAY_CLASSES; ++g) {
            if (p->leaf_count[g] > 0)
                SPG_TRY(launch_replay(a, p->leaves, p->leaf_order + off, p->leaf_count[g], p->leaf_cap[g],
                                      p->C.col_idx, p->C.val, p->d_err, p->st));
            off += p->leaf_count[g];
        }
        if (p->dense_n > 0)
            SPG_TRY(launch_dense_fill(p->A, p->B, p->dense_args(), p->C.row_ptr, p->C.col_idx, p->C.val, p->d_err,
                                      p->st, true));
    }
    return SPGEMM_OK;
fail:
    return status;
}

extern "C" spgemm_status spgemm_plan_check(spgemm_plan *p) {
    if (!p) return SPGEMM_ERR_INVALID_ARG;
    for (spgemm_plan *w : p->waves) {
        spgemm_status st = spgemm_plan_check(w);
        if (st != SPGEMM_OK) return st;
    }
    if (p->wave_mode) return SPGEMM_OK;
    int64_t err = 0;
    cudaError_t e = p->d2h(&err, p->d_err, sizeof(int64_t));
    if (e != cudaSuccess) return from_cuda(e);
    return err == 0 ? SPGEMM_OK : SPGEMM_ERR_INTERNAL;
}

// ---------------------------------------------------------------------------
// CUDA graph of values-only replays (e.g. both products of a Galerkin chain).
// ---------------------------------------------------------------------------

struct spgemm_graph {
    cudaStream_t st;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

extern "C" spgemm_status spgemm_graph_create(spgemm_plan *const *plans, int64_t n, spgemm_graph **out) {
    if (!plans || n < 1 || !out) return SPGEMM_ERR_INVALID_ARG;
    *out = nullptr;
    cudaStream_t st = plans[0]->st;
    if (st == nullptr) return SPGEMM_ERR_INVALID_ARG;  // the legacy default stream cannot be captured
    for (int64_t i = 0; i < n; ++i) {
        if (!plans[i] || !plans[i]->numeric_done || plans[i]->st != st) return SPGEMM_ERR_INVALID_ARG;
        // build the slice tables and set kernel attributes outside the capture
        spgemm_status s = spgemm_numeric_replay(plans[i]);
        if (s != SPGEMM_OK) return s;
    }
    spgemm_graph *g = new (std::nothrow) spgemm_graph();
    if (!g) return SPGEMM_ERR_OOM;
    g->st = st;
    g->graph = nullptr;
    g->exec = nullptr;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    spgemm_status status = e == cudaSuccess ? SPGEMM_OK : from_cuda(e);
    for (int64_t i = 0; status == SPGEMM_OK && i < n; ++i) status = spgemm_numeric_replay(plans[i]);
    e = cudaStreamEndCapture(st, &g->graph);
    if (status == SPGEMM_OK && e != cudaSuccess) status = from_cuda(e);
    if (status == SPGEMM_OK) {
        e = cudaGraphInstantiate(&g->exec, g->graph, 0);
        if (e != cudaSuccess) status = from_cuda(e);
    }
    if (status != SPGEMM_OK) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return status;
    }
    *out = g;
    return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_graph_launch(spgemm_graph *g) {
    if (!g) return SPGEMM_ERR_INVALID_ARG;
    return from_cuda(cudaGraphLaunch(g->exec, g->st));
}

extern "C" spgemm_status spgemm_graph_free(spgemm_graph *g) {
    if (!g) return SPGEMM_OK;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return SPGEMM_OK;
}

// Galerkin triple product Ac = R * (A * P) (the order the paper finds faster for
// its method, Section 5.2): two plans on one stream; *plan_rap owns Ac.
extern "C" spgemm_status spgemm_galerkin(const spgemm_csr_in *R, const spgemm_csr_in *A, const spgemm_csr_in *P,
                                         const spgemm_opts *opts, spgemm_stream_t stream, spgemm_plan **plan_ap,
                                         spgemm_plan **plan_rap, spgemm_csr_out *Ac) {
    if (!R || !A || !P || !plan_ap || !plan_rap || !Ac) return SPGEMM_ERR_INVALID_ARG;
    *plan_ap = *plan_rap = nullptr;
    if (R->ncols != A->nrows || A->ncols != P->nrows) return SPGEMM_ERR_SHAPE;
    spgemm_plan *p1 = nullptr, *p2 = nullptr;
    spgemm_status s = spgemm_symbolic(A, P, opts, stream, &p1, nullptr);
    if (s != SPGEMM_OK) return s;
    spgemm_csr_out ap;
    s = spgemm_numeric(p1, &ap);
    if (s != SPGEMM_OK) {
        spgemm_free(p1);
        return s;
    }
    spgemm_csr_in apin{ap.nrows, ap.ncols, ap.nnz, ap.row_ptr, 64, ap.col_idx, ap.val};
    s = spgemm_symbolic(R, &apin, opts, stream, &p2, nullptr);
    if (s == SPGEMM_OK) s = spgemm_numeric(p2, Ac);
    if (s != SPGEMM_OK) {
        spgemm_free(p2);
        spgemm_free(p1);
        return s;
    }
    *plan_ap = p1;
    *plan_rap = p2;
    return SPGEMM_OK;
}

// ---------------------------------------------------------------------------
// The precise method (Section 3.1): count every row, allocate C exactly, compute
// every row straight into it.  The same passes serve the products sized on the
// device (spgemm_dplan_*), with the bin sizes read by the kernels.
// ---------------------------------------------------------------------------

// The dense-slice arguments of a plan; with dev, the number of items is read on the device
// (the plan's bin-37 count) and the kernels take work from the plan's counters.
static DenseArgs dense_args_of(const spgemm_plan *p, bool dev) {
    DenseArgs D = p->dense_args();
    if (dev) {
        D.n = p->A.nrows;  // every row may be in bin 37: the arrays hold n K entries
        D.dev_n = &p->d_summary->dense_count;
        D.queue = p->d_queue;
        D.keep = nullptr;  // tables sized for every row: no room kept for bitmaps
        D.keep_words = 0;
    }
    return D;
}

// Counting pass: nnz(c_i) of bins 2..36 by a warp sort of their columns, and of bin 37 by the
// dense-slice count; bins 0 and 1 were sized by stage 2.
static cudaError_t precise_count(spgemm_plan *p, bool dev) {
    StageArgs a = stage_args(p);
    const bool acc = !dev;
    auto run = [&](int kind, auto &&launch) -> cudaError_t {
        if (acc) p->time_begin(kind);
        cudaError_t e = launch();
        if (acc) {
            p->time_end();
            p->count(kind);
        }
        return e;
    };
    cudaError_t e;
    const RowSet r32 = bin_range(p, BIN_HEAP_LO, BIN_HEAP_HI, dev);
    if (r32.n > 0 && (e = run(SPGEMM_K_ESC, [&] { return launch_esc_set(a, r32, 32, true, p->st); })) != cudaSuccess)
        return e;
    for (int b = BIN_ESC_LO; b <= BIN_ESC_HI; ++b) {
        const RowSet R = bin_range(p, b, b, dev);
        if (R.n > 0 && (e = run(SPGEMM_K_ESC, [&] { return launch_esc_set(a, R, b, true, p->st); })) != cudaSuccess)
            return e;
    }
    if (p->dense_K > 0 && (dev || p->dense_n > 0)) {
        const DenseArgs D = dense_args_of(p, dev);
        if ((e = run(SPGEMM_K_MERGE, [&] { return launch_dense_count(p->A, p->B, D, p->d_err, p->st); })) != cudaSuccess)
            return e;
        if ((e = run(SPGEMM_K_OTHER, [&] { return launch_dense_rowsum(D, p->nnzc, p->st); })) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Fill pass: every row computed straight into C (whose row pointers exist); nothing is
// written when the gate word is set.
static cudaError_t precise_fill(spgemm_plan *p, bool dev, const int64_t *gate) {
    StageArgs a = stage_args(p);
    a.ctil_rp = p->C.row_ptr;
    a.ctil_col = p->C.col_idx;
    a.ctil_val = p->C.val;
    a.gate = gate;
    cudaError_t e = launch_short_bins(p, a, !dev, dev);
    if (e != cudaSuccess) return e;
    // bin 1: the single product of each row
    const RowSet r1 = bin_range(p, 1, 1, dev);
    if (!dev) p->time_begin(SPGEMM_K_ARRANGE);
    e = launch_arrange_short_set(a, r1, p->bin, p->C.row_ptr, p->C.col_idx, p->C.val, p->st);
    if (!dev) {
        p->time_end();
        if (r1.n > 0) p->count(SPGEMM_K_ARRANGE);
    }
    if (e != cudaSuccess) return e;
    if (p->dense_K > 0 && (dev || p->dense_n > 0)) {
        if (!dev) p->time_begin(SPGEMM_K_MERGE);
        e = launch_dense_fill(p->A, p->B, dense_args_of(p, dev), p->C.row_ptr, p->C.col_idx, p->C.val, p->d_err, p->st,
                              false, gate);
        if (!dev) {
            p->time_end();
            p->count(SPGEMM_K_MERGE);
        }
    }
    return e;
}

static spgemm_status run_precise(spgemm_plan *p, spgemm_csr_out *C_out) {
    spgemm_status status = SPGEMM_OK;
    const int64_t m = p->A.nrows;
    {
        alloc_dense_keep(p);
        SPG_TRY(precise_count(p, false));
        SPG_TRY(p->alloc_n(&p->C.row_ptr, m + 1));
        p->time_begin(SPGEMM_K_SCAN);
        SPG_TRY(launch_row_scan(m, p->nnzc, p->C.row_ptr, p->scan_partial, p->st));
        p->time_end();
        p->count(SPGEMM_K_SCAN, 3);
        int64_t both[2] = {0, 0};
        SPG_TRY(p->d2h2(both, p->C.row_ptr + m, p->d_err));  // nnz(C), the one size the method reads back
        if (both[1] != 0) {
            status = SPGEMM_ERR_INTERNAL;
            goto fail;
        }
        const int64_t nnzC = both[0];
        SPG_TRY(p->alloc_n(&p->C.col_idx, nnzC));
        SPG_TRY(p->alloc_n(&p->C.val, nnzC));
        SPG_TRY(precise_fill(p, false, nullptr));
        p->C.nrows = m;
        p->C.ncols = p->B.ncols;
        p->C.nnz = nnzC;
        p->stats.nnz_c = nnzC;
        p->stats.bytes_ctilde = p->bytes_ctilde;
        p->numeric_done = true;
        p->release_temps(LIFE_NUMERIC);
        p->dense_keep = nullptr;  // released above: a values-only replay marks the columns from C
        p->dense_keep_words = 0;
        *C_out = p->C;
    }
    return SPGEMM_OK;
fail:
    return status;
}

// ---------------------------------------------------------------------------
// Products sized on the device: the precise method with every size kept in device
// memory, enqueued without allocation or read-back (capturable in a CUDA graph).
// ---------------------------------------------------------------------------

struct spgemm_dplan {
    spgemm_plan *p = nullptr;
    spgemm_csr_in A_in{}, B_in{};  // the borrowed inputs (int32 row pointers are widened each run)
    int64_t *a_rp64 = nullptr, *b_rp64 = nullptr;
    int64_t c_cap = 0;
    int64_t *gate = nullptr;
    int64_t *d_first = nullptr;     // batched: first entry of each C_i in the concatenated C
    int64_t nnz_cat_a = 0, nnz_cat_b = 0;
};

// Allocates every buffer of a device-sized plan whose A and B (DevCSR sizes) are set.
static spgemm_status dplan_buffers(spgemm_dplan *d) {
    spgemm_plan *p = d->p;
    spgemm_status status = SPGEMM_OK;
    const int64_t m = p->A.nrows, nnzA = p->A.nnz;
    const int64_t nblk = bin_blocks(m);
    {
        merge_limits(p);
        if (p->dense_K == 0 && p->B.ncols > 0) return SPGEMM_ERR_SHAPE;
        SPG_TRY(p->alloc_n(&p->d_summary, 1));
        SPG_TRY(p->alloc_n(&p->d_err, 1));
        SPG_TRY(p->alloc_n(&d->gate, 1));
        SPG_TRY(p->alloc_n(&p->d_queue, 3));
        SPG_TRY(p->alloc_n(&p->S, nnzA + 1));
        SPG_TRY(p->alloc_n(&p->scan_partial, std::max(bound_partial_size(nnzA), bin_blocks(m) + 1) + 1));
        SPG_TRY(p->alloc_n(&p->u, m));
        SPG_TRY(p->alloc_n(&p->bin, m));
        SPG_TRY(p->alloc_n(&p->nnzc, m));
        SPG_TRY(p->alloc_n(&p->bin_rows, m));
        SPG_TRY(p->alloc_n(&p->ctil_rp, m + 1));
        SPG_TRY(p->alloc_n(&p->d_hist, (int64_t)NUM_BINS * nblk));
        SPG_TRY(p->alloc_n(&p->d_capp, nblk));
        if (p->dense_K > 0) {
            SPG_TRY(p->alloc_n(&p->dense_flag, m));
            SPG_TRY(p->alloc_n(&p->dense_lo, m));
            SPG_TRY(p->alloc_n(&p->dense_hi, m));
            SPG_TRY(p->alloc_n(&p->d_select, dense_select_scratch(m)));
            SPG_TRY(p->alloc_n(&p->dense_order, m));
            SPG_TRY(p->alloc_n(&p->dense_rows, m));
            SPG_TRY(p->alloc_n(&p->dense_clo, m));
            SPG_TRY(p->alloc_n(&p->dense_chi, m));
            if (p->dense_K > 1) SPG_TRY(p->alloc_n(&p->dense_bnd, p->B.nrows * (p->dense_K + 1)));
            SPG_TRY(p->alloc_n(&p->dense_cnt, m * p->dense_K));
            SPG_TRY(p->alloc_n(&p->dense_soff, m * p->dense_K));
        }
        SPG_TRY(p->alloc_n(&p->C.row_ptr, m + 1));
        SPG_TRY(p->alloc_n(&p->C.col_idx, d->c_cap));
        SPG_TRY(p->alloc_n(&p->C.val, d->c_cap));
        SPG_TRY(cudaStreamSynchronize(p->st));  // the buffers exist before any capture
        p->C.nrows = m;
        p->C.ncols = p->B.ncols;
        p->C.nnz = -1;
    }
    return SPGEMM_OK;
fail:
    return status;
}

// One product, stages 1-4, every size on the device.
static cudaError_t dplan_enqueue(spgemm_dplan *d) {
    spgemm_plan *p = d->p;
    const int64_t m = p->A.nrows;
    cudaError_t e;
#define DP_TRY(x)                            \
    do {                                     \
        if ((e = (x)) != cudaSuccess) return e; \
    } while (0)
    DP_TRY(cudaMemsetAsync(p->d_summary, 0, sizeof(BinSummary), p->st));
    DP_TRY(cudaMemsetAsync(p->d_err, 0, sizeof(int64_t), p->st));
    if (p->npairs > 0) {
        DP_TRY(launch_concat(p->d_pairs, p->npairs, p->d_moff, p->d_koff, p->d_annz_off, p->d_bnnz_off, p->A.nrows,
                             p->B.nrows, p->A.nnz, p->B.nnz, p->cat_a_rp, p->cat_a_col, p->cat_a_val, p->cat_b_rp,
                             p->cat_b_col, p->cat_b_val, false, p->st));
    } else {
        if (d->a_rp64)
            DP_TRY(launch_widen_rowptr(static_cast<const int32_t *>(d->A_in.row_ptr), d->a_rp64, m + 1, p->st));
        if (d->b_rp64 && d->b_rp64 != d->a_rp64)
            DP_TRY(launch_widen_rowptr(static_cast<const int32_t *>(d->B_in.row_ptr), d->b_rp64, p->B.nrows + 1,
                                       p->st));
    }
    // stage 1 and the column ranges of the bin-37 rows (all of them dense-slice rows)
    DP_TRY(launch_bound(p->A, p->B, p->S, p->scan_partial, p->st));
    if (p->dense_K > 0)
        DP_TRY(launch_dense_mark(p->A, p->B, p->S, p->dense_min_u, 8, p->dense_flag, p->dense_lo, p->dense_hi, p->st));
    // stage 2: bins (no C~ to size)
    CapPolicy pol{};
    pol.policy = POLICY_PRECISE;
    pol.initial_cap = 1;
    pol.dense = p->dense_flag;
    DP_TRY(launch_binning(m, p->A.rp, p->S, p->S + p->A.nnz, pol, p->u, p->bin, p->nnzc, p->bin_rows, p->ctil_rp,
                          p->d_hist, p->d_capp, p->d_summary, p->st));
    if (p->dense_K > 0) {
        DP_TRY(launch_dense_select(p->bin_rows, m, p->d_summary, p->u, p->dense_flag, p->dense_lo, p->dense_hi,
                                   p->d_select, p->dense_order, p->dense_rows, p->dense_clo, p->dense_chi, p->st));
        if (p->dense_K > 1) DP_TRY(launch_dense_bounds(p->B, p->dense_K, p->dense_W, p->dense_bnd, p->st));
    }
    // stage 3, counting pass; stage 4, row pointers; then the fill pass straight into C
    DP_TRY(precise_count(p, true));
    DP_TRY(launch_row_scan(m, p->nnzc, p->C.row_ptr, p->scan_partial, p->st));
    DP_TRY(launch_gate(p->C.row_ptr, m, d->c_cap, d->gate, p->d_err, p->st));
    DP_TRY(precise_fill(p, true, d->gate));
    if (p->npairs > 0) {
        DP_TRY(launch_split_out(p->d_pairs, p->npairs, p->C.row_ptr, m, p->split_rp, p->st));
        DP_TRY(launch_gather_first(p->d_pairs, p->npairs, p->C.row_ptr, m, d->d_first, p->st));
    }
#undef DP_TRY
    return cudaSuccess;
}

static spgemm_status dplan_begin(const spgemm_opts *opts, spgemm_stream_t stream, int64_t c_cap, spgemm_dplan **out) {
    *out = nullptr;
    if (c_cap < 0) return SPGEMM_ERR_INVALID_ARG;
    spgemm_opts o;
    if (opts) o = *opts; else spgemm_opts_init(&o);
    o.alloc_policy = SPGEMM_ALLOC_PRECISE;
    o.predictor = nullptr;
    o.record_timing = 0;
    o.check_inputs = 0;
    spgemm_dplan *d = new (std::nothrow) spgemm_dplan();
    if (!d) return SPGEMM_ERR_OOM;
    spgemm_status st = plan_begin(&o, stream, &d->p);
    if (st != SPGEMM_OK) {
        delete d;
        return st;
    }
    d->c_cap = c_cap;
    *out = d;
    return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_dplan_free(spgemm_dplan *d) {
    if (!d) return SPGEMM_OK;
    if (d->p) spgemm_free(d->p);
    delete d;
    return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_dplan_create(const spgemm_csr_in *A_in, const spgemm_csr_in *B_in, int64_t c_cap,
                                             const spgemm_opts *opts, spgemm_stream_t stream, spgemm_dplan **out,
                                             spgemm_csr_out *C) {
    if (!out || !C) return SPGEMM_ERR_INVALID_ARG;
    *out = nullptr;
    spgemm_status status = check_in(A_in);
    if (status != SPGEMM_OK) return status;
    status = check_in(B_in);
    if (status != SPGEMM_OK) return status;
    if (A_in->ncols != B_in->nrows) return SPGEMM_ERR_SHAPE;
    spgemm_dplan *d = nullptr;
    status = dplan_begin(opts, stream, c_cap, &d);
    if (status != SPGEMM_OK) return status;
    spgemm_plan *p = d->p;
    {
        d->A_in = *A_in;
        d->B_in = *B_in;
        auto side = [&](const spgemm_csr_in *M, DevCSR &D, int64_t **rp64) -> cudaError_t {
            D = DevCSR{M->nrows, M->ncols, M->nnz, static_cast<const int64_t *>(M->row_ptr), M->col_idx, M->val};
            if (M->rowptr_bits == 64) return cudaSuccess;
            cudaError_t e = p->alloc_n(rp64, M->nrows + 1);
            D.rp = *rp64;
            return e;
        };
        SPG_TRY(side(A_in, p->A, &d->a_rp64));
        if (B_in->row_ptr == A_in->row_ptr && B_in->rowptr_bits == A_in->rowptr_bits) {
            p->B = DevCSR{B_in->nrows, B_in->ncols, B_in->nnz, p->A.rp, B_in->col_idx, B_in->val};
            d->b_rp64 = d->a_rp64;
        } else {
            SPG_TRY(side(B_in, p->B, &d->b_rp64));
        }
        status = dplan_buffers(d);
        if (status != SPGEMM_OK) goto fail;
    }
    *C = p->C;
    *out = d;
    return SPGEMM_OK;
fail:
    cudaStreamSynchronize(p->st);
    spgemm_dplan_free(d);
    return status;
}

extern "C" spgemm_status spgemm_dplan_batched_create(int64_t npairs, const spgemm_csr_in *A, const spgemm_csr_in *B,
                                                     int64_t c_cap, const spgemm_opts *opts, spgemm_stream_t stream,
                                                     spgemm_dplan **out, spgemm_csr_out *C) {
    if (!out || !C || npairs < 1 || !A || !B) return SPGEMM_ERR_INVALID_ARG;
    *out = nullptr;
    std::vector<PairDesc> hd((size_t)npairs);
    std::vector<int64_t> moff(npairs), koff(npairs), aoff(npairs), boff(npairs);
    int64_t M = 0, K = 0, N = 0, annz = 0, bnnz = 0;
    for (int64_t i = 0; i < npairs; ++i) {
        spgemm_status st = check_in(&A[i]);
        if (st != SPGEMM_OK) return st;
        st = check_in(&B[i]);
        if (st != SPGEMM_OK) return st;
        if (A[i].ncols != B[i].nrows) return SPGEMM_ERR_SHAPE;
        PairDesc &q = hd[i];
        q.a_rp = A[i].row_ptr;
        q.b_rp = B[i].row_ptr;
        q.a_col = A[i].col_idx;
        q.b_col = B[i].col_idx;
        q.a_val = A[i].val;
        q.b_val = B[i].val;
        q.a_bits = A[i].rowptr_bits;
        q.b_bits = B[i].rowptr_bits;
        q.m = A[i].nrows;
        q.k = A[i].ncols;
        q.n = B[i].ncols;
        q.moff = moff[i] = M;
        q.koff = koff[i] = K;
        q.annz_off = aoff[i] = annz;
        q.bnnz_off = boff[i] = bnnz;
        q.annz = A[i].nnz;
        q.bnnz = B[i].nnz;
        M += q.m;
        K += q.k;
        N = std::max(N, q.n);
        annz += q.annz;
        bnnz += q.bnnz;
    }
    if (M > INT32_MAX || K > INT32_MAX || N > INT32_MAX) return SPGEMM_ERR_SHAPE;
    spgemm_dplan *d = nullptr;
    spgemm_status status = dplan_begin(opts, stream, c_cap, &d);
    if (status != SPGEMM_OK) return status;
    spgemm_plan *p = d->p;
    {
        p->npairs = npairs;
        p->h_pairs = hd;
        SPG_TRY(p->alloc_n(&p->d_pairs, npairs));
        SPG_TRY(p->alloc_n(&p->d_moff, npairs));
        SPG_TRY(p->alloc_n(&p->d_koff, npairs));
        SPG_TRY(p->alloc_n(&p->d_annz_off, npairs));
        SPG_TRY(p->alloc_n(&p->d_bnnz_off, npairs));
        SPG_TRY(cudaMemcpyAsync(p->d_pairs, hd.data(), sizeof(PairDesc) * npairs, cudaMemcpyHostToDevice, p->st));
        SPG_TRY(cudaMemcpyAsync(p->d_moff, moff.data(), sizeof(int64_t) * npairs, cudaMemcpyHostToDevice, p->st));
        SPG_TRY(cudaMemcpyAsync(p->d_koff, koff.data(), sizeof(int64_t) * npairs, cudaMemcpyHostToDevice, p->st));
        SPG_TRY(cudaMemcpyAsync(p->d_annz_off, aoff.data(), sizeof(int64_t) * npairs, cudaMemcpyHostToDevice, p->st));
        SPG_TRY(cudaMemcpyAsync(p->d_bnnz_off, boff.data(), sizeof(int64_t) * npairs, cudaMemcpyHostToDevice, p->st));
        SPG_TRY(cudaStreamSynchronize(p->st));  // pageable sources
        SPG_TRY(p->alloc_n(&p->cat_a_rp, M + 1));
        SPG_TRY(p->alloc_n(&p->cat_b_rp, K + 1));
        SPG_TRY(p->alloc_n(&p->cat_a_col, annz));
        SPG_TRY(p->alloc_n(&p->cat_a_val, annz));
        SPG_TRY(p->alloc_n(&p->cat_b_col, bnnz));
        SPG_TRY(p->alloc_n(&p->cat_b_val, bnnz));
        SPG_TRY(p->alloc_n(&p->split_rp, M + npairs));
        SPG_TRY(p->alloc_n(&d->d_first, npairs + 1));
        p->A = DevCSR{M, K, annz, p->cat_a_rp, p->cat_a_col, p->cat_a_val};
        p->B = DevCSR{K, N, bnnz, p->cat_b_rp, p->cat_b_col, p->cat_b_val};
        status = dplan_buffers(d);
        if (status != SPGEMM_OK) goto fail;
    }
    *C = p->C;
    *out = d;
    return SPGEMM_OK;
fail:
    cudaStreamSynchronize(p->st);
    spgemm_dplan_free(d);
    return status;
}

extern "C" spgemm_status spgemm_dplan_run(spgemm_dplan *d) {
    if (!d || !d->p) return SPGEMM_ERR_INVALID_ARG;
    return from_cuda(dplan_enqueue(d));
}

extern "C" spgemm_status spgemm_dplan_result(spgemm_dplan *d, spgemm_csr_out *C_out) {
    if (!d || !d->p || !C_out) return SPGEMM_ERR_INVALID_ARG;
    spgemm_plan *p = d->p;
    const int64_t m = p->A.nrows;
    int64_t both[2] = {0, 0};
    cudaError_t e = p->d2h2(both, p->C.row_ptr + m, p->d_err);
    if (e != cudaSuccess) return from_cuda(e);
    if (both[1] == 8) return SPGEMM_ERR_OOM;  // nnz(C) exceeded the capacity: C was left empty
    if (both[1] != 0) return SPGEMM_ERR_INTERNAL;
    p->C.nnz = both[0];
    if (p->npairs == 0) {
        *C_out = p->C;
        return SPGEMM_OK;
    }
    const int64_t np = p->npairs;
    std::vector<int64_t> first(np + 1);
    e = cudaMemcpy(first.data(), d->d_first, sizeof(int64_t) * (np + 1), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return from_cuda(e);
    for (int64_t i = 0; i < np; ++i) {
        const PairDesc &q = p->h_pairs[i];
        spgemm_csr_out &c = C_out[i];
        c.nrows = q.m;
        c.ncols = q.n;
        c.nnz = first[i + 1] - first[i];
        c.row_ptr = p->split_rp + q.moff + i;
        c.col_idx = p->C.col_idx + first[i];
        c.val = p->C.val + first[i];
    }
    return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_dplan_bytes(spgemm_dplan *d, int64_t *bytes) {
    if (!d || !d->p || !bytes) return SPGEMM_ERR_INVALID_ARG;
    *bytes = d->p->bytes_held;
    return SPGEMM_OK;
}

extern "C" spgemm_status spgemm_dplan_graph_create(spgemm_dplan *const *plans, int64_t n, spgemm_graph **out) {
    if (!plans || n < 1 || !out) return SPGEMM_ERR_INVALID_ARG;
    *out = nullptr;
    for (int64_t i = 0; i < n; ++i)
        if (!plans[i] || !plans[i]->p) return SPGEMM_ERR_INVALID_ARG;
    cudaStream_t st = plans[0]->p->st;
    if (st == nullptr) return SPGEMM_ERR_INVALID_ARG;  // the legacy default stream cannot be captured
    for (int64_t i = 0; i < n; ++i) {
        if (plans[i]->p->st != st) return SPGEMM_ERR_INVALID_ARG;
        // one run outside the capture sets the kernels' attributes
        spgemm_status s = from_cuda(dplan_enqueue(plans[i]));
        if (s != SPGEMM_OK) return s;
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return from_cuda(e);
    spgemm_graph *g = new (std::nothrow) spgemm_graph();
    if (!g) return SPGEMM_ERR_OOM;
    g->st = st;
    g->graph = nullptr;
    g->exec = nullptr;
    e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    spgemm_status status = e == cudaSuccess ? SPGEMM_OK : from_cuda(e);
    for (int64_t i = 0; status == SPGEMM_OK && i < n; ++i) status = from_cuda(dplan_enqueue(plans[i]));
    e = cudaStreamEndCapture(st, &g->graph);
    if (status == SPGEMM_OK && e != cudaSuccess) status = from_cuda(e);
    if (status == SPGEMM_OK) {
        e = cudaGraphInstantiate(&g->exec, g->graph, 0);
        if (e != cudaSuccess) status = from_cuda(e);
    }
    if (status != SPGEMM_OK) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return status;
    }
    *out = g;
    return SPGEMM_OK;
}
