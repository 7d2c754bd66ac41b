// Internal interfaces between the host orchestrator (spgemm_api.cu) and the
// kernel translation units.  Not part of the public C ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace spg {

// Value type of A, B and C: double in the default build, float in the single-precision
// build (compiled with SPGEMM_FLOAT, the same entry points).
#ifdef SPGEMM_FLOAT
using val_t = float;
#else
using val_t = double;
#endif

constexpr int NUM_BINS = 38;
constexpr int BIN_HEAP_LO = 2, BIN_HEAP_HI = 32;  // bin group 3 (Section 4.1)
constexpr int BIN_ESC_LO = 33, BIN_ESC_HI = 36;   // bin group 4
constexpr int BIN_MERGE = 37;                     // bin group 5
constexpr int64_t BIN_MERGE_MIN_U = 512;          // bin 37 holds the rows with u_i > 512 (Algorithm 3)

enum AllocPolicy { POLICY_HYBRID = 0, POLICY_UPPER_BOUND = 1, POLICY_LEARNED = 2, POLICY_PRECISE = 3 };

// CSR with int64 row pointers (int32 inputs are widened once per call).
struct DevCSR {
    int64_t nrows, ncols, nnz;
    const int64_t *rp;
    const int32_t *col;
    const val_t *val;
};

// Host-visible summary written by stage 2 (copied back in one transfer).
constexpr int NUM_LAUNCH_CLASSES = 8;  // learned: shared-memory classes of bin-37 rows

struct BinSummary {
    int64_t bin_count[NUM_BINS];
    int64_t sum_cap;   // nnz(C~) of the initial allocation
    int64_t sum_u;     // sum u_i
    int64_t status;    // validation result (0 = ok)
    int64_t pad;
    int64_t class_count[NUM_LAUNCH_CLASSES];  // learned: bin-37 rows per launch class
    int64_t dense_count;                      // bin-37 rows computed by the dense-slice kernels
    int64_t bin_start[NUM_BINS + 1];          // offsets of the bins in bin_rows (for launches sized on the device)
};

// Rows of one stage-3 launch.  With dev_lo == nullptr they are rows[0..n), n known on the
// host.  Otherwise they are rows[*dev_lo .. *dev_hi), both ends read on the device, so the
// launch needs no read-back: it runs a fixed (persistent) grid that strides over the range,
// and n is only an upper bound of its length (it caps the grid).
struct RowSet {
    const int32_t *rows;
    int64_t n;
    const int64_t *dev_lo = nullptr;
    const int64_t *dev_hi = nullptr;
};
inline RowSet host_rows(const int32_t *rows, int64_t n) { return RowSet{rows, n, nullptr, nullptr}; }

// Blocks of a persistent launch of `kern` (NT threads, smem dynamic bytes): as many as are
// resident on all SMs at once, at most `cap` (> 0).
int persistent_blocks(const void *kern, int nt, size_t smem, int64_t cap);

struct CapPolicy {
    int policy;
    int64_t initial_cap;
    const int32_t *pred_cap;  // learned per-row temporary row sizes (POLICY_LEARNED), may be null
    int64_t cap_max;          // learned: a bin-37 row's home never exceeds the largest shared capacity
    const uint8_t *dense;     // per row, 1: a dense-slice row (no C~ space); null: none
};

// ---- stage 0/1/2 (stage12.cu) ----
cudaError_t launch_widen_rowptr(const int32_t *in, int64_t *out, int64_t n, cudaStream_t st);
cudaError_t launch_validate(const DevCSR &M, int64_t *status, cudaStream_t st);
// S[j] = sum_{t<j} nnz(b_{A.col[t]*}), S[nnzA] = sum u (Algorithm 2 as a prefix sum).
cudaError_t launch_bound(const DevCSR &A, const DevCSR &B, int64_t *S, int64_t *partial,
                         cudaStream_t st);
int64_t bound_partial_size(int64_t nnzA);
// Binning scratch sizes for m rows.
int64_t bin_blocks(int64_t m);
cudaError_t launch_binning(int64_t m, const int64_t *arp, const int64_t *S,
                           const int64_t *sum_u_ptr, CapPolicy P, int64_t *u, uint8_t *bin, int32_t *nnzc, int32_t *bin_rows,
                           int64_t *ctil_rp, int32_t *hist, int64_t *cap_partial,
                           BinSummary *summary, cudaStream_t st);

// C~ row offsets again from u and the bins under P (ctil_rp[0..m]; the total into *total)
cudaError_t launch_cap_rescan(int64_t m, const int64_t *u, const uint8_t *bin, CapPolicy P, int64_t *ctil_rp,
                              int64_t *partial, int64_t *total, cudaStream_t st);

// ---- learned preallocation (predictor.cu) ----
// Row features (warp per row).  With the stage-1 prefix S, rows with u_i <= u_min are
// skipped, and so are the rows flagged in `skip` (when given).
cudaError_t launch_row_features(const DevCSR &A, const DevCSR &B, float *X, cudaStream_t st,
                                const int64_t *S = nullptr, int64_t u_min = 0, const uint8_t *skip = nullptr);
// Predicted temporary size per row (0 for rows skipped through arp/S/u_min/skip).  With
// promote_min > 0, a row whose predicted nnz(c_i) is at least promote_min is flagged in
// skip (a dense-slice row) instead.
cudaError_t launch_predict_caps(const float *params, const float *X, int64_t m, const int64_t *u, float margin,
                                int32_t min_cap, int32_t *pred_cap, cudaStream_t st, const int64_t *arp = nullptr,
                                const int64_t *S = nullptr, int64_t u_min = 0, uint8_t *skip = nullptr,
                                int64_t promote_min = 0);
// Groups the bin-37 items (tail of bin_rows, size read from summary) by launch
// class; items of flagged (dense-slice) rows go after the last class; scratch: 96 + m
// int32; order: item indices grouped by class; counts go to summary->class_count.
cudaError_t launch_class_partition_tail(const int32_t *bin_rows, int64_t m, BinSummary *summary,
                                        const int32_t *pred_cap, const int32_t *class_cap, int ncls,
                                        const uint8_t *dense, int32_t *scratch, int32_t *order, cudaStream_t st);
const float *predictor_params(const void *pred);

// ---- stage 3 ----
// The status words of the bounds-checked build: every translation unit built with
// SPGEMM_CHECK registers the reader of its word (spgemm_check_status reads them all).
using CheckReader = cudaError_t (*)(unsigned long long *word, bool reset);
int register_check_reader(CheckReader read);

struct StageArgs {
    DevCSR A, B;
    const int64_t *ctil_rp;
    int32_t *ctil_col;
    val_t *ctil_val;
    int32_t *nnzc;
    const int64_t *gate = nullptr;  // when set and *gate != 0, the kernels write nothing (C too small)
};

cudaError_t launch_heap(const StageArgs &a, const int32_t *rows, int64_t nrows, int slots, int nt,
                        cudaStream_t st);
cudaError_t launch_heap_set(const StageArgs &a, const RowSet &R, int slots, int nt, cudaStream_t st);
cudaError_t launch_esc(const StageArgs &a, const int32_t *rows, int64_t nrows, int bin,
                       cudaStream_t st);
// count_only: nnz(c_i) of every row into a.nnzc and nothing else (the counting pass of the
// precise method, Section 3.1); bin 32 stands for any u_i <= 32
cudaError_t launch_esc_set(const StageArgs &a, const RowSet &R, int bin, bool count_only, cudaStream_t st);

// Bin-37 work items.  Item j < n37 is the j-th row of bin 37 with the full
// column range.  An item whose sequence outgrows the largest shared-memory
// capacity is split at the median column of that sequence into two child items
// with column ranges [clo, mkey) and [mkey, chi); the leaves of a row, read in
// column order, concatenate to the row of C.
struct MergeItems {
    int32_t *row;        // row of C
    int32_t *clo;        // first column of the item's range
    int32_t *chi;        // end of the range (exclusive); INT32_MAX = unbounded
    int32_t **src_col;   // sorted sequence to reload when the item (re)starts
    val_t **src_val;
    int32_t *src_len;
    int32_t **home_col;  // where the item's sequence is written
    val_t **home_val;
    int64_t *home_cap;
    int32_t *len;        // final length (leaves)
    int64_t *ck_entry;   // checkpoint: A-entry index relative to the row start
    int64_t *ck_off;     //             and offset inside that entry's full B row
    int32_t *child;      // -1 for a leaf, else the left child (the right one is child + 1)
    int32_t *parent;     // the item it was split from; -1 for a row's own item
};

struct MergeLaunch {
    const int32_t *work;     // items to process (nullptr: items work_base .. work_base + nwork - 1)
    int64_t work_base;
    int64_t nwork;
    int cap;                 // shared-memory result capacity for this launch
    int batch;               // products per batch
    int level1;              // 1: level-1 mode (global result + shared level-1 sequence)
    int32_t *pool_col;       // per-work-item homes of capacity pool_cap (may be null)
    val_t *pool_val;
    int64_t pool_cap;
    const int64_t *g_off;    // level-1: per-work-item offset of two global buffers
    const int64_t *g_cap;    //          and their capacity
    int32_t *g_col;
    val_t *g_val;
    int32_t *ovf_list;       // items that overflowed
    int32_t *ovf_count;
    int64_t *err;            // device error word
    int wide_above;          // capacities above this use 512-thread CTAs (0 = 2048)
    int bm_words;            // > 0: bitmap kernel; flat: bitmap words, two-level: level-1 words
    int bm_two;              // 1: two-level index
    int bm_miss;             // bitmap kernel: miss-buffer entries
};

int merge_smem_bytes(int cap, int batch, int wide_above);
// Bitmap form of the bin-37 kernel (merge_bm.cu): a flat bitmap index for B with at
// most BM_MAX_COLS columns, a two-level index up to BM2_MAX_COLS.
constexpr int64_t BM_MAX_COLS = 131072;
constexpr int64_t BM2_MAX_COLS = (int64_t)1 << 22;
int merge_bm_smem_bytes(int cap, int nwords, int miss, int wide_above, bool two);
int merge_bm_max_cap(int nwords, int miss, int smem_limit, int wide_above, bool two);
cudaError_t launch_merge_bm(const StageArgs &a, const MergeItems &s, const MergeLaunch &L, cudaStream_t st);
int merge_batch_limit(int cap, int wide_above);
int merge_max_cap(int batch, int smem_limit, int wide_above);
cudaError_t launch_merge(const StageArgs &a, const MergeItems &it, const MergeLaunch &L, cudaStream_t st);
cudaError_t launch_merge_init(const int32_t *rows37, int64_t n37, const int64_t *ctil_rp, int32_t *ctil_col,
                              val_t *ctil_val, const MergeItems &it, cudaStream_t st);
// splits the items listed in ovf (count n) into children first_new + 2i, first_new + 2i + 1;
// right child i gets slot i of the pool (n slots of pool_cap entries)
cudaError_t launch_split(const int32_t *ovf, int64_t n, int64_t first_new, const MergeItems &it,
                         int32_t *pool_col, val_t *pool_val, int64_t pool_cap, cudaStream_t st);
// nnz(c_i) of every bin-37 row = summed lengths of its leaves
cudaError_t launch_finalize37(int64_t n37, const MergeItems &it, int32_t *nnzc, int64_t *err, cudaStream_t st);
// level-1 buffer sizing: per work item cap = min(u_row, ncols_B) (two buffers each)
cudaError_t launch_level1_sizes(const MergeItems &it, const int32_t *work, int64_t nwork,
                                const int64_t *u, int64_t ncols, int64_t *g_cap, int64_t *g_off,
                                int64_t *partial, int64_t *total, cudaStream_t st);

// ---- dense column slices for the longest bin-37 rows (dense.cu) ----
constexpr int32_t ITEM_DENSE = -2;  // MergeItems.child of a row computed by the dense-slice kernels
constexpr int DENSE_MAX_SLICES = 64;
constexpr int DENSE_W_MAX = 131072;  // widest slice: its bitmap and rank directory take 32 KB
struct DenseArgs {
    const int32_t *items;  // dense items (indices into MergeItems), larger rows first
    const int32_t *rows;   // their rows of A
    const int32_t *clo;    // and the column range [clo, chi) that each row's products can reach
    const int32_t *chi;
    int64_t n;             // number of dense items
    int K;                 // column slices of B
    int W;                 // slice width (a multiple of 32); slice s holds columns [s W, (s + 1) W)
    const int32_t *bnd;    // K > 1: per B row, K + 1 offsets of the slices' first entries in the row
    int32_t *cnt;          // n K columns per (row, slice)
    int32_t *soff;         // n K offsets of the slices inside their row of C
    const int64_t *dev_n = nullptr;  // when set: the number of dense items is *dev_n (<= n), read on
                                     // the device; the kernels run persistent grids over (item, slice)
    unsigned long long *queue = nullptr;  // three work counters (count, fill, fill of the heavy items),
                                          // zeroed by the launchers; needed with dev_n
    uint32_t *keep = nullptr;  // when set (bitmap counts, compact fills only): keep_words words per
    int keep_words = 0;        // (row, slice), where the count leaves the slice's column bitmap and
                               // the fill reads it back instead of marking the columns again
};
cudaError_t launch_dense_bounds(const DevCSR &B, int K, int W, int32_t *bnd, cudaStream_t st);
// per row: flag (1 = dense-slice row: bin 37, and u_i >= dmin if dmin > 0, else div u_i >= the
// width of its column range) and, for bin-37 rows, the column range [lo, hi)
cudaError_t launch_dense_mark(const DevCSR &A, const DevCSR &B, const int64_t *S, int64_t dmin, int div,
                              uint8_t *flag, int32_t *lo, int32_t *hi, cudaStream_t st);
int64_t dense_select_scratch(int64_t m);
// order[0..nd) = items of the flagged bin-37 rows (larger u first), order[nd..n37) = the rest;
// rows, rlo, rhi [0..nd) = their rows and column ranges; nd goes to summary->dense_count
cudaError_t launch_dense_select(const int32_t *bin_rows, int64_t m, BinSummary *summary, const int64_t *u,
                                const uint8_t *flag, const int32_t *lo, const int32_t *hi, int32_t *scratch,
                                int32_t *order, int32_t *rows, int32_t *rlo, int32_t *rhi, cudaStream_t st);
// counts the columns of every (row, slice) into D.cnt (reads no work-item table, so it
// may run beside the merge launches)
cudaError_t launch_dense_count(const DevCSR &A, const DevCSR &B, const DenseArgs &D, int64_t *err, cudaStream_t st);
// Words per (row, slice) of a kept column bitmap for slices of W columns, or 0 when the count
// does not build bitmaps for such slices or the fill does not read them (the single-pass form).
int dense_keep_words(int W);
// slice offsets inside the rows, and the dense items' lengths in the work-item table
cudaError_t launch_dense_rows(const MergeItems &it, const DenseArgs &D, cudaStream_t st);
// precise method: slice offsets inside the rows, and nnz(c_i) of every dense row into nnzc
cudaError_t launch_dense_rowsum(const DenseArgs &D, int32_t *nnzc, cudaStream_t st);
// accumulates every (row, slice) and writes it into C at c_rp[row] + soff; replay: values
// only, into the entries whose columns are already in C
cudaError_t launch_dense_fill(const DevCSR &A, const DevCSR &B, const DenseArgs &D, const int64_t *c_rp,
                              int32_t *c_col, val_t *c_val, int64_t *err, cudaStream_t st, bool replay = false,
                              const int64_t *gate = nullptr);
int dense_fill_smem_bytes(int W);
int dense_fill_wide_bytes(int W);  // the single-pass form (fits for narrow slices only)
int dense_fill_static_smem();
int dense_fill_max_dynamic(int per_sm);

// ---- the merge evaluation of Section 4.2 (merge_micro.cu) ----
// method 0 ranking merge, 1 merge path, 2 bitonic merge; groups of 2l keys (two sorted runs)
int merge_micro_smem(int l, int value_bytes);
cudaError_t launch_merge_micro(int method, int threads, int value_bytes, const int32_t *keys, const void *vals,
                               int64_t n, int l, int32_t *okeys, void *ovals, cudaStream_t st);

// ---- values-only replay (replay.cu) ----
struct ReplayLeaves {
    int32_t *row, *clo, *chi;
    int64_t *c_off;   // first entry of the leaf in C
    int32_t *len;
    int cap;          // shared-memory capacity of a launch (set by launch_replay)
};
constexpr int NUM_REPLAY_CLASSES = 3;
cudaError_t launch_replay(const StageArgs &a, ReplayLeaves lv, const int32_t *order, int64_t n, int cap,
                          int32_t *c_col, val_t *c_val, int64_t *err, cudaStream_t st);
cudaError_t launch_replay_leaves(int64_t n37, const MergeItems &it, const int64_t *c_rp, const int32_t *class_cap,
                                 int ncls, int32_t *count, int32_t *start, int32_t *cursor, const ReplayLeaves &lv,
                                 int32_t *order, int64_t *err, bool scatter, cudaStream_t st);

// ---- batched products (batched.cu): block-diagonal concatenation ----
struct PairDesc {
    const void *a_rp, *b_rp;
    const int32_t *a_col, *b_col;
    const val_t *a_val, *b_val;
    int32_t a_bits, b_bits;
    int64_t m, k, n;             // A_i is m x k, B_i is k x n
    int64_t moff, koff;          // row offset of A_i and B_i in the concatenation
    int64_t annz_off, bnnz_off;  // entry offsets
    int64_t annz, bnnz;
};
cudaError_t launch_concat(const PairDesc *d, int64_t npairs, const int64_t *moff, const int64_t *koff,
                          const int64_t *annz_off, const int64_t *bnnz_off, int64_t M, int64_t K, int64_t annz,
                          int64_t bnnz, int64_t *a_rp, int32_t *a_col, val_t *a_val, int64_t *b_rp, int32_t *b_col,
                          val_t *b_val, bool values_only, cudaStream_t st);
cudaError_t launch_gather_first(const PairDesc *d, int64_t npairs, const int64_t *c_rp, int64_t M, int64_t *out,
                                cudaStream_t st);
cudaError_t launch_pair_products(const PairDesc *d, int64_t npairs, int64_t *prod, int64_t *clow,
                                 cudaStream_t st);
cudaError_t launch_split_out(const PairDesc *d, int64_t npairs, const int64_t *c_rp, int64_t M, int64_t *rp_out,
                             cudaStream_t st);

// ---- stage 4 (arrange.cu) ----
cudaError_t launch_row_scan(int64_t m, const int32_t *nnzc, int64_t *c_rp, int64_t *partial,
                            cudaStream_t st);
cudaError_t launch_arrange_short(const StageArgs &a, const int32_t *rows, int64_t nrows,
                                 const uint8_t *bin, const int64_t *c_rp, int32_t *c_col,
                                 val_t *c_val, cudaStream_t st);
cudaError_t launch_arrange_short_set(const StageArgs &a, const RowSet &R, const uint8_t *bin, const int64_t *c_rp,
                                     int32_t *c_col, val_t *c_val, cudaStream_t st);
// *gate = 1, *err = 8 and every c_rp[0..m] = 0 (C empty) when the result of m rows (c_rp[m]
// entries) exceeds cap entries, else *gate = 0
cudaError_t launch_gate(int64_t *c_rp, int64_t m, int64_t cap, int64_t *gate, int64_t *err, cudaStream_t st);
cudaError_t launch_arrange_long(const MergeItems &it, int64_t n37, const int64_t *c_rp, int32_t *c_col,
                                val_t *c_val, cudaStream_t st);

}  // namespace spg
