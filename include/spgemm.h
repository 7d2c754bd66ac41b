/*
 * spgemm.h -- C ABI of a GB300 (sm_103a) CSR SpGEMM library, C = A * B, FP64.
 *
 * The library implements the four-stage framework of Liu & Vinter, "A
 * Framework for General Sparse Matrix-Matrix Multiplication on GPUs and
 * Heterogeneous Processors" (JPDC 2015), Section 4.1:
 *   stage 1  per-row upper bound u_i of the intermediate products (Algorithm 2);
 *   stage 2  binning of rows by u_i into 38 bins and allocation of the
 *            temporary matrix C~ with the hybrid policy (Algorithm 3) --
 *            computed on the GPU here, without atomics;
 *   stage 3  per-bin insert-and-accumulate: heap method (bins u = 2..32),
 *            bitonic expand-sort-compress (u = 33..512), merge method with
 *            progressive reallocation and a level-1 sequence (u > 512);
 *   stage 4  prefix sum of the row sizes and compaction of C~ into C.
 *
 * All pointers inside spgemm_csr_in / spgemm_csr_out are DEVICE pointers on the
 * device that is current when spgemm_symbolic is called.  No function throws;
 * every function returns an spgemm_status.  A plan is used by one host thread at
 * a time.  Everything a plan launches is ordered on the stream given to
 * spgemm_symbolic.
 */
#ifndef SPGEMM_H
#define SPGEMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL means the legacy default stream. */
typedef struct CUstream_st *spgemm_stream_t;

typedef enum spgemm_status {
    SPGEMM_OK = 0,
    SPGEMM_ERR_INVALID_ARG = 1, /* NULL where a pointer is required, negative size, bad option */
    SPGEMM_ERR_SHAPE = 2,       /* A.ncols != B.nrows, or a dimension beyond the supported range */
    SPGEMM_ERR_UNSORTED = 3,    /* check_inputs: a row's column indices are not strictly ascending,
                                   out of range, or row_ptr is not a valid prefix array */
    SPGEMM_ERR_OOM = 4,         /* a device allocation failed; the plan stays freeable */
    SPGEMM_ERR_CUDA = 5,        /* a CUDA runtime call or launch failed */
    SPGEMM_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up */
    SPGEMM_ERR_INTERNAL = 7     /* an internal consistency check failed */
} spgemm_status;

/* Value type of A, B and C.  The default library (libspgemm.so) computes in double; the
   single-precision library (libspgemm_f32.so, built from the same sources with SPGEMM_FLOAT
   defined) has the same entry points with float values (the paper's SpSGEMM). */
#ifdef SPGEMM_FLOAT
typedef float spgemm_value_t;
#else
typedef double spgemm_value_t;
#endif

/*
 * Input matrix in CSR format (Section 2.1): row_ptr has nrows+1 entries with
 * row_ptr[0] = 0 and row_ptr[nrows] = nnz; row i holds col_idx/val entries
 * row_ptr[i] .. row_ptr[i+1]-1 with column indices strictly ascending (the
 * sorted-column assumption of Section 3.2; duplicates are not allowed).
 * row_ptr is int32 (rowptr_bits = 32) or int64 (rowptr_bits = 64).
 * Requirements: 0 <= nrows, ncols <= 2^31 - 1.  Borrowed: the arrays must stay
 * valid and unchanged until the work enqueued by spgemm_numeric has completed.
 * A value stored as 0.0 is still a structural entry.
 */
typedef struct spgemm_csr_in {
    int64_t nrows;
    int64_t ncols;
    int64_t nnz;
    const void *row_ptr;
    int32_t rowptr_bits;
    const int32_t *col_idx;
    const spgemm_value_t *val;
} spgemm_csr_in;

/*
 * Result matrix C in CSR format, owned by the plan: valid from the completion
 * of spgemm_numeric's work on the plan's stream until spgemm_free.  row_ptr is
 * always int64 (nrows+1 entries); each row's columns are strictly ascending.
 * Every (i, j) with a structural a_ik and b_kj is present, also when the sum
 * cancels to 0.0 (Section 3.1).
 */
typedef struct spgemm_csr_out {
    int64_t nrows;
    int64_t ncols;
    int64_t nnz;
    int64_t *row_ptr;
    int32_t *col_idx;
    spgemm_value_t *val;
} spgemm_csr_out;

/* Memory pre-allocation policy for the temporary matrix C~ (Section 3.1). */
typedef enum spgemm_alloc_policy {
    /* The paper's hybrid method: rows with u_i <= 512 get u_i slots, longer rows
       start at initial_cap slots and grow x2 per relaunch (Section 4.1). */
    SPGEMM_ALLOC_HYBRID = 0,
    /* Every row gets u_i slots (the upper-bound method of Section 3.1); long rows
       still run in shared memory and use the level-1 sequence when too long. */
    SPGEMM_ALLOC_UPPER_BOUND = 1,
    /* Rows are sized from a learned prediction of nnz(c_i) (see
       spgemm_predictor_*); a row whose result exceeds its prediction falls back
       to the exact path, so C is unchanged. */
    SPGEMM_ALLOC_LEARNED = 2,
    /* The precise method (Section 3.1): a counting pass first computes nnz(c_i) of every
       row -- a warp sort of the row's columns for u_i <= 512, the dense column-slice count for
       longer rows -- then C is allocated exactly and every row is computed straight into it
       (heap / bitonic ESC for u_i <= 512, the dense column slices for the rest): no temporary
       matrix C~ and no relaunch, at the price of a second pass over the products.  B's columns
       must fit 64 slices of 131,072 columns (8,388,608 columns); a wider B returns
       SPGEMM_ERR_SHAPE. */
    SPGEMM_ALLOC_PRECISE = 3
} spgemm_alloc_policy;

/* Rows whose result outgrows the largest shared-memory capacity (bin 37). */
typedef enum spgemm_long_rows {
    /* Split the row at the median column of its merged sequence into two column
       slices that resume independently (default; slices run on separate SMs). */
    SPGEMM_LONG_ROWS_SPLIT = 0,
    /* The paper's level-1 sequence (Section 4.1): shared memory holds a level-1
       sequence that is merged into a global sequence whenever it fills up. */
    SPGEMM_LONG_ROWS_LEVEL1 = 1
} spgemm_long_rows;

/* Form of the bin-37 merge kernel (Section 4.1, merge method). */
typedef enum spgemm_merge_kernel {
    /* Bitmap form when long rows are split and B has at most 4,194,304 columns, else
       the merge-path form (default). */
    SPGEMM_MERGE_AUTO = 0,
    /* Merge-path form: every batch's new columns are sorted by pairwise merge-path
       merges and merged into a pending set, then into the result, in place. */
    SPGEMM_MERGE_PATH = 1,
    /* Bitmap form: an index over the item's column range gives each product's
       position in the result in O(1) -- a bitmap with a rank directory for B with at
       most 131,072 columns, else a two-level index (occupied 32-column words, then
       their bits) up to 4,194,304 columns; new columns are buffered and merged into
       the result by rank when the buffer fills (same eligibility as AUTO). */
    SPGEMM_MERGE_BITMAP = 2
} spgemm_merge_kernel;

/* Options; initialise with spgemm_opts_init and change fields as needed. */
typedef struct spgemm_opts {
    int32_t alloc_policy;    /* spgemm_alloc_policy */
    int32_t initial_cap;     /* first temporary row size of bin 37 (paper: 256) */
    int32_t check_inputs;    /* 1: validate A and B on the device (one pass) */
    int32_t record_timing;   /* 1: time every kernel with CUDA events (spgemm_plan_stats) */
    int32_t merge_batch;     /* products per batch in the bin-37 merge kernel (0 = auto) */
    int32_t smem_cap_max;    /* largest result capacity held in shared memory (0 = auto) */
    int32_t heap_block;      /* threads per block of the heap kernel (0 = auto) */
    int32_t long_rows;       /* spgemm_long_rows: handling of rows beyond shared memory */
    int32_t wave_mproducts;  /* batched products: largest number of products (in millions) that
                                one wave of pairs may hold; pairs are grouped in order into waves
                                computed one after another, each releasing its temporaries
                                before the next (0 = 1024, negative = one wave) */
    int32_t heap_max_u;      /* rows with u_i <= heap_max_u use the heap kernel; the longer rows
                                of bins 2..32 use the bitonic ESC kernel with 32 slots
                                (0 = 32, the paper's split; 2..32 allowed) */
    int32_t merge_wide_above; /* bin-37 launches with a result capacity above this use 512-thread
                                 CTAs, smaller ones 256 (128 up to 512 entries); 0 = 2048 */
    int32_t merge_kernel;    /* spgemm_merge_kernel: form of the bin-37 kernel */
    int32_t merge_miss;      /* bitmap form: products whose column is new are buffered up to this
                                many entries before they are merged into the result (0 = 4096) */
    int32_t dense_min_u;     /* bin-37 rows with u_i >= this are computed by the dense-slice
                                kernels instead of the merge kernel: B's columns are cut into
                                slices, one CTA per (row, slice), after a pass that counts the
                                columns of every slice; the rows are then written straight into C.
                                0 = a bin-37 row is dense when dense_span_div * u_i >= the width of
                                the column range its products can reach (first to last column of
                                the B rows it selects); negative = never.  Off with SPGEMM_MERGE_PATH,
                                SPGEMM_LONG_ROWS_LEVEL1 and when B needs more than 64 slices */
    int32_t dense_span;      /* widest dense slice in columns (0 = 131,072, at least 1,024).  A slice
                                narrow enough for one sum and one flag per column in shared memory
                                (about 21,900 columns in double) is filled in one pass over its
                                products; a wider one keeps a bitmap of its columns, its rank
                                directory and one sum per column of the result */
    int32_t dense_span_div;  /* with dense_min_u = 0: the divisor of the rule above (0 = 8) */
    const void *predictor;   /* spgemm_predictor* for SPGEMM_ALLOC_LEARNED, else NULL; it must
                                not be freed before spgemm_symbolic (or spgemm_galerkin) has
                                returned, since its weights are read by that call's kernels */
    double predictor_margin; /* predicted size is multiplied by this before rounding up */
    int32_t dense_pred_min;  /* learned policy: a bin-37 row whose predicted nnz(c_i) is at least this
                                is computed by the dense-slice kernels (the network's choice of
                                kernel as well as of size); 0 = off */
    int32_t dense_keep;      /* slices too wide for the single-pass fill (about 21,900 columns in
                                double, 40,000 in float), which the compact form fills: the counting
                                pass leaves every (row, slice)'s column bitmap in device memory (ceil(W / 32) + 1 words, rounded up to 4, per
                                (row, slice), released when spgemm_numeric returns) and the fill reads
                                it back instead of marking the columns again from the products.
                                0 = kept by the hybrid, upper-bound and learned policies when the
                                bitmaps take at most a quarter of the free device memory, never by the
                                precise policy (whose peak stays C plus O(rows) tables); positive = the
                                same test under every policy; negative = never.  Products sized on the
                                device never keep them (their tables are sized for every row) */
    int64_t max_bytes;       /* device bytes the plan may hold at once (0 = no limit): an allocation
                                that would exceed it fails as if the device were full and the call
                                returns SPGEMM_ERR_OOM (the kept bitmaps of dense_keep are skipped
                                instead).  A failed spgemm_symbolic leaves nothing allocated; a
                                failed spgemm_numeric leaves its temporaries with the plan until
                                spgemm_free releases them */
} spgemm_opts;

/* Fills *opts with the defaults (hybrid policy, initial_cap 256, no checks). */
spgemm_status spgemm_opts_init(spgemm_opts *opts);

typedef struct spgemm_plan spgemm_plan;

/*
 * Stages 1 and 2.  Computes u_i for every row of A (Algorithm 2), bins the
 * rows (Algorithm 3) and allocates C~.  Enqueues on `stream` and synchronises it
 * once to read the 38 bin sizes (the host decides which per-bin kernels to
 * launch, Section 4.1).  On success *plan_out owns the temporaries and, if
 * upper_bound_nnz_out is not NULL, receives sum_i u_i = nnz(C^) = flops/2.
 * On error *plan_out is set to NULL and nothing stays allocated.
 */
spgemm_status spgemm_symbolic(const spgemm_csr_in *A, const spgemm_csr_in *B,
                              const spgemm_opts *opts, spgemm_stream_t stream,
                              spgemm_plan **plan_out, int64_t *upper_bound_nnz_out);

/*
 * Stages 3 and 4.  Runs the per-bin kernels (including the progressive
 * relaunches of bin 37), scans the row sizes, allocates C and compacts C~ into
 * it.  Synchronises the plan's stream when it needs a size on the host (each
 * progressive round, and nnz(C) before C is allocated).  On success *C_out
 * describes C, owned by the plan.  Calling it twice returns the same C.
 */
spgemm_status spgemm_numeric(spgemm_plan *plan, spgemm_csr_out *C_out);

/* Releases every device buffer of the plan (stream-ordered on its stream) and
   the plan itself.  NULL is accepted. */
spgemm_status spgemm_free(spgemm_plan *plan);

/* Every plan allocates from one stream-ordered memory pool per device, which keeps the
   blocks freed by earlier plans for reuse (no release threshold), so a process that ran a
   large product keeps holding that device memory.  This returns the pool's unused memory
   on `device` to the system, keeping at most keep_bytes (cudaMemPoolTrimTo).  Synchronise
   the streams of the plans freed on that device first: blocks whose stream-ordered free has
   not run yet are still in use.  SPGEMM_ERR_INVALID_ARG for a negative device or
   keep_bytes; no-op for a device the library has not allocated on. */
spgemm_status spgemm_pool_trim(int32_t device, int64_t keep_bytes);

/* The bounds-checked build (libspgemm_check.so: the same sources with SPGEMM_CHECK defined).
   Its kernels check the indices of their result writes and shared-memory scatters; an index
   outside its array records a site code (the first one recorded stays) and the access is
   skipped, without a trap, so the context stays usable.  *code_out = 0 when no check failed
   since the last reset, the first code recorded otherwise, and -1 in a build without the
   checks.  reset != 0 clears the record.  Synchronise the device first; SPGEMM_ERR_INVALID_ARG
   for a NULL code_out. */
spgemm_status spgemm_check_status(int64_t *code_out, int32_t reset);

/* Static English text for a status code. */
const char *spgemm_status_string(spgemm_status status);

/* Kernel classes reported by spgemm_plan_stats. */
typedef enum spgemm_kernel_id {
    SPGEMM_K_BOUND = 0,     /* stage 1: upper bound (prefix sum of B-row lengths over A) */
    SPGEMM_K_BIN = 1,       /* stage 2: histogram, scan and scatter of the 38 bins */
    SPGEMM_K_HEAP = 2,      /* stage 3, bins 2..32 */
    SPGEMM_K_ESC = 3,       /* stage 3, bins 33..36 */
    SPGEMM_K_MERGE = 4,     /* stage 3, bin 37 (all progressive rounds and level-1) */
    SPGEMM_K_SCAN = 5,      /* stage 4: prefix sum of nnz(c_i) */
    SPGEMM_K_ARRANGE = 6,   /* stage 4: copy of C~ into C (and the u_i = 1 rows) */
    SPGEMM_K_OTHER = 7,     /* validation, predictor, bookkeeping */
    SPGEMM_K_COUNT = 8
} spgemm_kernel_id;

typedef struct spgemm_stats {
    int64_t bin_count[38];      /* rows per bin (Algorithm 3) */
    int64_t sum_u;              /* sum of u_i = number of products */
    int64_t nnz_ctilde;         /* entries allocated for C~ in stage 2 */
    int64_t nnz_c;              /* nnz(C), after spgemm_numeric */
    int64_t merge_rounds;       /* launches of the bin-37 kernel (progressive rounds) */
    int64_t rows_relaunched;    /* bin-37 rows that overflowed at least once */
    int64_t rows_level1;        /* bin-37 rows finished with a level-1 sequence */
    int64_t rows_split;         /* column splits of long rows (SPGEMM_LONG_ROWS_SPLIT) */
    int64_t rows_fallback;      /* rows recomputed because a prediction was too small */
    int64_t bytes_ctilde;       /* device bytes allocated for temporary rows (all rounds) */
    int64_t peak_bytes;         /* high-water mark of the device bytes held by the plan (temporaries
                                   and C) from spgemm_symbolic on */
    int32_t launches[SPGEMM_K_COUNT];  /* kernels launched per class */
    float kernel_ms[SPGEMM_K_COUNT];   /* summed event time per class (record_timing = 1) */
    int64_t held_bytes;         /* device bytes the plan holds now: stage-1/2 scratch is released
                                   when spgemm_symbolic returns and C~ with the merge pools when
                                   spgemm_numeric returns (stream-ordered), so after the product
                                   this is C plus the O(rows) tables that values-only replay uses */
    int64_t rows_dense;         /* bin-37 rows computed by the dense-slice kernels */
    int64_t dense_slices;       /* column slices of B used by them (0 when none) */
    int64_t item_rounds;        /* bin-37 work items summed over every launch of the bin-37 merge
                                   kernel: a row counts once per progressive round it runs in, and
                                   each half of a split row counts on its own */
    double alloc_host_ms;       /* host milliseconds spent in the plan's device allocations (from a
                                   stream-ordered pool: long when the pool must map new memory) */
    int64_t allocs;             /* device allocations made by the plan */
} spgemm_stats;

/* Copies the plan's counters into *out.  Timings are read after synchronising
   the plan's stream. */
spgemm_status spgemm_plan_stats(spgemm_plan *plan, spgemm_stats *out);

/*
 * Read-only views of a plan's intermediate arrays (device pointers owned by the
 * plan, valid until spgemm_free; bin_start is a host array inside the plan):
 *   u[m]             upper bound of each row of C (Algorithm 2, stage 1)
 *   bin[m]           bin of each row, 0..37 (Algorithm 3, stage 2)
 *   bin_rows[m]      row ids grouped by bin, ascending within each bin
 *   bin_start[39]    offsets of the 38 bins in bin_rows
 *   ctilde_row_ptr   m+1 offsets of the rows of C~ as first allocated (stage 2)
 *   row_nnz[m]       nnz(c_i); complete after spgemm_numeric (stage 3)
 */
typedef struct spgemm_plan_arrays {
    int64_t nrows;
    const int64_t *u;
    const uint8_t *bin;
    const int32_t *bin_rows;
    const int64_t *bin_start;
    const int64_t *ctilde_row_ptr;
    const int32_t *row_nnz;
} spgemm_plan_arrays;

spgemm_status spgemm_plan_arrays_get(spgemm_plan *plan, spgemm_plan_arrays *out);

/*
 * Batched products (not in the paper): npairs independent C_i = A_i * B_i (host
 * arrays of npairs descriptors of device matrices) computed as one product of
 * block-diagonal matrices, diag(A_1..A_n) * diag(B_1..B_n) = diag(A_1 B_1 ..
 * A_n B_n), so every stage -- including each per-bin kernel of stage 3 -- runs
 * once for the rows of all pairs.  B_i keeps its own column numbers (a row of
 * C_i only combines rows of B_i), so the concatenated C holds every C_i with its
 * own columns.  Requires sum m_i, sum k_i <= 2^31-1.  spgemm_batched_numeric
 * fills C_out[0..npairs) with views owned by the plan: each C_i has its own
 * int64 row pointers (starting at 0); its columns and values are slices of the
 * plan's concatenated result.  spgemm_free releases everything.  The inputs are
 * copied into the plan at symbolic time (their values are read again by
 * spgemm_numeric_replay).
 */
spgemm_status spgemm_batched_symbolic(int64_t npairs, const spgemm_csr_in *A, const spgemm_csr_in *B,
                                      const spgemm_opts *opts, spgemm_stream_t stream,
                                      spgemm_plan **plan_out, int64_t *upper_bound_nnz_out);
spgemm_status spgemm_batched_numeric(spgemm_plan *plan, spgemm_csr_out *C_out);

/*
 * Waves of a batched plan.  spgemm_batched_symbolic counts every pair's products
 * (Algorithm 2 summed over its rows) and a lower bound of nnz(C_i) (the sum over
 * rows of the longest B row they merge), orders the pairs by descending product
 * count and groups consecutive pairs of that order into waves.  A wave holds at
 * most opts->wave_mproducts million products (a larger pair is a wave of its
 * own), and beyond 32 million products it also stops growing once its products
 * (which bound its temporary entries) exceed the lower bounds of the pairs still
 * to come.  With more than one wave, spgemm_batched_numeric computes the waves
 * one after another, each as a batched product of its own whose temporaries are
 * released before the next wave starts: the largest pairs run while few results
 * are resident and no wave's temporaries outgrow the results that follow it, so
 * the peak stays near the size of all results.  C_out[i] is still the product of
 * pair i.  In this mode the inputs are read by
 * spgemm_batched_numeric and must stay valid until its work has completed, and
 * spgemm_plan_arrays_get is refused (read each wave's arrays instead).
 * spgemm_batched_waves gives the number of waves (1 without wave mode);
 * spgemm_batched_wave gives wave i's plan (borrowed, owned by the batched plan;
 * available after spgemm_batched_numeric; wave 0 of a single-wave plan is the
 * plan itself) and the position of its first pair in the wave order;
 * spgemm_batched_wave_pairs fills order[0..npairs) with the pair at each
 * position of that order (the identity without wave mode).
 */
spgemm_status spgemm_batched_waves(spgemm_plan *plan, int64_t *n_waves);
spgemm_status spgemm_batched_wave(spgemm_plan *plan, int64_t i, spgemm_plan **wave, int64_t *first_pair);
spgemm_status spgemm_batched_wave_pairs(spgemm_plan *plan, int64_t *order);

/*
 * Values-only replay (not in the paper): after spgemm_numeric (or
 * spgemm_batched_numeric), recomputes the values of C for new values of A and B
 * with the SAME structure (row pointers and columns unchanged), into the same C.
 * The known columns of each long row are preloaded and every product is fused
 * into them by binary search (sub-step 1 of the merge method, Section 4.1); bins
 * 2..36 rerun their heap / ESC kernels straight into C.  The first call on a plan
 * builds its slice table (allocates and synchronises once); later calls neither
 * allocate nor synchronise, so they can be captured in a CUDA graph.  A product
 * whose column is missing from C (the structure changed) makes spgemm_plan_check
 * return SPGEMM_ERR_INTERNAL.  Plans that used the level-1 sequence
 * (SPGEMM_LONG_ROWS_LEVEL1) are refused with SPGEMM_ERR_INVALID_ARG.
 */
spgemm_status spgemm_numeric_replay(spgemm_plan *plan);

/* Reads the plan's device error word (synchronises its stream). */
spgemm_status spgemm_plan_check(spgemm_plan *plan);

/*
 * CUDA graph of values-only replays: captures one spgemm_numeric_replay of each of
 * plans[0..n) in order (all plans must share one non-default stream and have
 * finished spgemm_numeric); spgemm_graph_launch enqueues the graph on that stream.
 * Creating the graph runs one replay of each plan first (outside the capture).
 * The graph stays valid while the plans live.
 */
typedef struct spgemm_graph spgemm_graph;
spgemm_status spgemm_graph_create(spgemm_plan *const *plans, int64_t n, spgemm_graph **out);
spgemm_status spgemm_graph_launch(spgemm_graph *graph);
spgemm_status spgemm_graph_free(spgemm_graph *graph);

/*
 * Galerkin triple product Ac = R * (A * P) as two products (the association the
 * paper measures as faster for its method, Section 5.2).  *plan_ap owns A*P,
 * *plan_rap owns Ac (described by *Ac); free both.  Both plans use `stream`, so
 * spgemm_graph_create on {*plan_ap, *plan_rap} captures the whole chain for new
 * values of R, A and P with unchanged structure.
 */
spgemm_status spgemm_galerkin(const spgemm_csr_in *R, const spgemm_csr_in *A, const spgemm_csr_in *P,
                              const spgemm_opts *opts, spgemm_stream_t stream, spgemm_plan **plan_ap,
                              spgemm_plan **plan_rap, spgemm_csr_out *Ac);

/*
 * Products sized on the device (not in the paper): the whole of C = A * B -- stages 1 to 4 --
 * enqueued with every size the method needs (bin counts, nnz(c_i), nnz(C)) kept in device
 * memory and none read back, so that the product can be enqueued again and again or captured
 * in a CUDA graph, for inputs whose structure changes from one run to the next.  It follows
 * the precise method (SPGEMM_ALLOC_PRECISE: count, then compute every row straight into C),
 * and each stage-3 launch is a persistent kernel: a fixed grid of as many CTAs as the SMs
 * hold, striding over a bin whose rows are listed on the device (warps and threads over the
 * rows of bins 2..36, a work counter over the (row, slice) items of bin 37).
 *
 * spgemm_dplan_create allocates everything at once for inputs of the given sizes: A and B
 * (or the npairs pairs of spgemm_dplan_batched_create, computed as one block-diagonal
 * product) are borrowed device matrices whose sizes (nrows, ncols, nnz, rowptr_bits) are
 * fixed, while their row pointers, columns and values may change between runs.  C gets room
 * for c_capacity entries; *C receives its device arrays (row_ptr with nrows + 1 entries, col
 * and val with c_capacity entries; C->nnz = -1 until a result is read).  C's arrays may be
 * the B of a later plan on the same stream (B.nnz = c_capacity), which chains two products.
 * Options: as for spgemm_symbolic; the allocation policy is always the precise method.
 *
 * spgemm_dplan_run enqueues the product on the plan's stream: no allocation, no host
 * synchronisation.  If nnz(C) exceeds c_capacity, nothing is written to C's columns and
 * values, and spgemm_dplan_result returns SPGEMM_ERR_OOM.  spgemm_dplan_result synchronises
 * the stream, reads nnz(C) and the device error word, and describes C (npairs descriptors for
 * a batched plan: each C_i with its own int64 row pointers starting at 0, its columns and
 * values views into the concatenated C).  spgemm_dplan_graph_create captures one run of each
 * of plans[0..n) in order (all on one created, non-default stream) into a CUDA graph; it runs
 * each plan once before the capture.  spgemm_graph_launch and spgemm_graph_free apply.
 * Errors: as spgemm_symbolic; SPGEMM_ERR_SHAPE also when B is too wide for the precise method.
 */
typedef struct spgemm_dplan spgemm_dplan;
spgemm_status spgemm_dplan_create(const spgemm_csr_in *A, const spgemm_csr_in *B, int64_t c_capacity,
                                  const spgemm_opts *opts, spgemm_stream_t stream, spgemm_dplan **out,
                                  spgemm_csr_out *C);
spgemm_status spgemm_dplan_batched_create(int64_t npairs, const spgemm_csr_in *A, const spgemm_csr_in *B,
                                          int64_t c_capacity, const spgemm_opts *opts, spgemm_stream_t stream,
                                          spgemm_dplan **out, spgemm_csr_out *C);
spgemm_status spgemm_dplan_run(spgemm_dplan *plan);
spgemm_status spgemm_dplan_result(spgemm_dplan *plan, spgemm_csr_out *C_out);
spgemm_status spgemm_dplan_graph_create(spgemm_dplan *const *plans, int64_t n, spgemm_graph **out);
spgemm_status spgemm_dplan_free(spgemm_dplan *plan);
/* Device bytes the plan holds (all of it allocated by spgemm_dplan_create). */
spgemm_status spgemm_dplan_bytes(spgemm_dplan *plan, int64_t *bytes);

/*
 * Allocation-free row-pointer scan (no counterpart in the paper).
 *
 * Computes row_ptr[0..m] from row sizes: row_ptr[i] = row_nnz[0] + ... +
 * row_nnz[i-1] (int64), row_ptr[m] = the total -- the prefix sum that stage 4
 * uses to lay out C -- without allocating any device memory.  It is meant for
 * callers that cannot call cudaMalloc: code whose device memory is owned by an
 * arena that forbids other allocations, code that must not risk the implicit
 * device synchronisation an allocation can cause, or code that has a fixed
 * memory budget decided up front.
 *
 * row_nnz: device array of m int32 sizes (each >= 0); row_ptr: device array of
 * m+1 int64 outputs.  Both are owned by the caller.  The work is enqueued on
 * `stream`; the call returns without waiting for it.
 *
 * The scan keeps its per-tile partial sums in one fixed device array that the
 * library holds on every GPU that loads it until the process exits (32769
 * int64 = 256 KiB), which limits m to spgemm_rowptr_scan_noalloc_max_rows()
 * (67,108,864); a larger m returns SPGEMM_ERR_SHAPE without launching anything.
 * NULL pointers or m < 0 return SPGEMM_ERR_INVALID_ARG.  The first call on a
 * device looks up that array's device address (once per device, with that
 * device current), so make the first call on each device before any stream
 * capture.  All calls on a device share the one array: calls whose work could
 * overlap on the GPU (different streams, or concurrent host threads) race and
 * must be serialised by the caller.  Nothing needs clearing between calls.
 */
spgemm_status spgemm_rowptr_scan_noalloc(const int32_t *row_nnz, int64_t m, int64_t *row_ptr,
                                         spgemm_stream_t stream);

/* Largest m accepted by spgemm_rowptr_scan_noalloc. */
int64_t spgemm_rowptr_scan_noalloc_max_rows(void);

/*
 * Learned preallocation (not in the paper; it replaces the fixed 256-entry start
 * of bin 37's progressive allocation, Section 4.1, by a predicted size).
 *
 * A small MLP maps 8 features of a row of C to SPGEMM_MLP_CLASSES size-class
 * logits (class of nnz(c_i): 0 for nnz <= 1, else ceil(log2 nnz), at most 15)
 * and a regression of log2(1 + nnz(c_i)).  Parameter vector (float32):
 *   W1[32x8] b1[32] W2[32x32] b2[32] W3[17x32] b3[17]   (SPGEMM_MLP_NUM_PARAMS)
 *   mu[8] sigma[8]                                      (input standardisation)
 * out = W3 relu(W2 relu(W1 (x - mu)/sigma + b1) + b2) + b3.
 * Features (float32, row-major [m][8]): log2(1+x) of nnz(a_i*), of u_i, the
 * min, max, mean and standard deviation of log2(1 + nnz(b_k*)) over the stored
 * a_ik, log2(1 + column span of the selected non-empty B rows), log2(1 + ncols(B)).
 * With SPGEMM_ALLOC_LEARNED, a bin-37 row gets a temporary row of
 * s = max(256, 32*ceil(margin * (2^reg - 1) / 32)) entries -- or u_i entries when
 * u_i <= margin * s, a bound it can never outgrow at little extra space -- and starts in
 * the shared-memory class that fits it; a row whose result outgrows that size
 * continues on the exact progressive path, so C does not depend on the prediction.
 */
#define SPGEMM_MLP_FEATURES 8
#define SPGEMM_MLP_HIDDEN 32
#define SPGEMM_MLP_CLASSES 16
#define SPGEMM_MLP_NUM_PARAMS 1905
#define SPGEMM_MLP_NUM_TOTAL 1921

typedef struct spgemm_predictor spgemm_predictor;

/* Copies SPGEMM_MLP_NUM_TOTAL host floats (n must equal it) to the current device. */
spgemm_status spgemm_predictor_create(const float *host_params, int64_t n, spgemm_predictor **out);
spgemm_status spgemm_predictor_free(spgemm_predictor *pred);

/* X[m][8] (device, float32) = the features of every row of C = A*B; enqueued on stream. */
spgemm_status spgemm_row_features(const spgemm_csr_in *A, const spgemm_csr_in *B, float *X,
                                  spgemm_stream_t stream);

/* out[n][17] (device) = MLP outputs for X[n][8] with device parameters `params`. */
spgemm_status spgemm_mlp_forward(const float *params, const float *X, int64_t n, float *out,
                                 spgemm_stream_t stream);

/* Floats of device workspace spgemm_mlp_loss_grad needs for n samples. */
int64_t spgemm_mlp_work_floats(int64_t n);

/* Summed loss over n samples, loss = CE(softmax(out[0..15]), cls) + 0.5 (out[16] - y)^2,
   into *loss (device double), and its gradient w.r.t. the SPGEMM_MLP_NUM_PARAMS
   trainable values into grad (device float, overwritten).  work: device floats of
   spgemm_mlp_work_floats(n). */
spgemm_status spgemm_mlp_loss_grad(const float *params, const float *X, const int32_t *cls,
                                   const float *y, int64_t n, float *work, float *grad, double *loss,
                                   spgemm_stream_t stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the trainable values with
   gradient grad * grad_scale; m and v are device moment buffers; step >= 1. */
spgemm_status spgemm_mlp_adam(float *params, const float *grad, float *m, float *v, int64_t step,
                              float lr, float grad_scale, spgemm_stream_t stream);

/*
 * The merge evaluation of Section 4.2 ("Evaluating GPU Merge algorithms"): merges groups
 * of two sorted runs into sorted sequences, with one CTA of `threads` threads (64, 128,
 * 256, 512 or 1024) per group, in shared memory.  method: 0 ranking merge, 1 merge path,
 * 2 bitonic merge (the last stage of a bitonic sort).  keys: n int32 device values, in
 * groups of 2l: keys[g 2l .. g 2l + l) and keys[g 2l + l .. (g + 1) 2l) each ascending.
 * vals: n device values of value_bytes (0: none and may be NULL, 4 or 8) that move with
 * their keys.  out_keys, out_vals: n each (out_vals ignored when value_bytes = 0).  l must
 * be a power of two with 2 l (4 + value_bytes) bytes of shared memory available, and n a
 * positive multiple of 2 l.  Equal keys: ranking merge and merge path put the first run's
 * element first; the bitonic network does not keep an order among them.  Enqueued on
 * `stream`; SPGEMM_ERR_INVALID_ARG for bad arguments.
 */
spgemm_status spgemm_merge_micro(int32_t method, int32_t threads, int32_t value_bytes, const int32_t *keys,
                                 const void *vals, int64_t n, int32_t l, int32_t *out_keys, void *out_vals,
                                 spgemm_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SPGEMM_H */
