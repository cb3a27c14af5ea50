/*
 * msgemm -- masked sparse matrix-matrix products on NVIDIA GB300 (sm_103a).
 *
 * The operation (Sec. 2 of "Parallel Algorithms for Masked Sparse
 * Matrix-Matrix Products"): C = M .* (A B) on a semiring, where only the
 * pattern of the mask M is used; its complemented form C = !M .* (A B) keeps
 * the entries the mask does NOT hold (Sec. 1; complement paragraphs of
 * Sec. 5.2 and 5.5).  An entry C_ij exists iff the mask allows (i, j) and at
 * least one k has both A_ik and B_kj stored (the SET state of the accumulator
 * interface, Sec. 5.1); entries whose numeric sum is zero are kept.  Output
 * rows have ascending column indices.  The product is one-phase (Sec. 6): the
 * output is written into room sized by the mask and then compacted, with no
 * separate symbolic pass.
 *
 * Conventions for every entry point
 *  - Matrices are CSR with int32 row pointers and column indices; within a row
 *    the column indices are strictly ascending (sorted, no duplicates);
 *    nnz < 2^31.  Input pointers are DEVICE pointers, borrowed for the call.
 *  - Values: float for MSGEMM_PLUS_TIMES_F32, int64_t for the two int64
 *    semirings.  PLUS_PAIR ignores input values (they may be NULL).  Under
 *    the plus-times semirings, NULL values make A or B of a masked product a
 *    pattern operand: every stored value is 1 (a 0/1 adjacency, as in the
 *    BFS step, needs no value array).  The gradients (msgemm_backward) need
 *    the values.  Mask values are never read.
 *  - Shapes: M is m x n, A is m x k, B is k x n; any of m, n, k may be 0.
 *  - Every call is asynchronous on the handle's stream and returns as soon as
 *    its work is enqueued, except where a call says it synchronises.  Errors
 *    found on the host are returned at once and leave no work enqueued.  Errors
 *    found by kernels (invalid input under validation, a bounded wait that
 *    ran out) set a device error word that msgemm_sync_status() reports.
 *  - Output arrays are allocated through the handle's allocation callback and
 *    then belong to the caller, who frees them (with the matching free).
 *  - A handle is not thread-safe; use one handle per host thread and stream.
 */
#ifndef MSGEMM_H
#define MSGEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MSGEMM_OK = 0,
    MSGEMM_ERR_INVALID = 1,      /* NULL pointer, negative size, bad option, bad rowptr/column */
    MSGEMM_ERR_SHAPE = 2,        /* operand shapes do not chain */
    MSGEMM_ERR_UNSORTED = 3,     /* a row is not strictly ascending (found by validation) */
    MSGEMM_ERR_UNSUPPORTED = 4,  /* combination the library does not implement */
    MSGEMM_ERR_OOM = 5,          /* the allocation callback returned NULL */
    MSGEMM_ERR_OVERFLOW = 6,     /* a size does not fit the int32 index space */
    MSGEMM_ERR_CUDA = 7,         /* a CUDA runtime call failed */
    MSGEMM_ERR_TIMEOUT = 8       /* a bounded device-side wait ran out */
} msgemm_status;

typedef enum {
    MSGEMM_PLUS_TIMES_F32 = 0,   /* (+, *) on float; accumulation in float */
    MSGEMM_PLUS_TIMES_I64 = 1,   /* (+, *) on int64_t, wrapping modulo 2^64 */
    MSGEMM_PLUS_PAIR_I64 = 2     /* (+, pair): every product counts 1; result int64_t */
} msgemm_semiring;

/* Accumulator families (Sec. 4-5) that the row binning may pick per row. */
typedef enum {
    MSGEMM_ACC_AUTO = 0,  /* per-row choice by the binning policy (default) */
    MSGEMM_ACC_MSA = 1,   /* masked sparse accumulator: dense states + values (Sec. 5.2) */
    MSGEMM_ACC_HASH = 2,  /* hash table keyed by the mask's columns (Sec. 5.3) */
    MSGEMM_ACC_MCA = 3,   /* mask-compressed accumulator indexed by rank in the mask row (Sec. 5.4) */
    MSGEMM_ACC_DOT = 4,   /* pull: masked inner products A_i* . B_*j (Sec. 4.1) */
    MSGEMM_ACC_HEAP = 5,  /* multiway merge of the rows of B with the mask row (Sec. 5.5,
                             Alg. 4 and 5), NInspect = 1; rows with at most 128 stored
                             entries in A_i*.  Complemented: NInspect = 0 */
    MSGEMM_ACC_HEAPDOT = 6 /* the same with NInspect unbounded (each row iterator walks to
                             its next mask column before it is queued) */
} msgemm_accumulator;

/* Options for msgemm_set_option. */
typedef enum {
    MSGEMM_OPT_FORCE_ACCUM = 1,   /* value: msgemm_accumulator.  Rows that do not fit the
                                     forced family's per-row shared-memory form use the
                                     column-tiled MSA; MCA and DOT do not exist for
                                     complemented masks, where AUTO is used instead. */
    MSGEMM_OPT_VALIDATE = 2,      /* value 0/1 (default 0): check every input on the device
                                     (row pointers, column range, strict order) before the
                                     product runs; synchronises once per call and returns
                                     MSGEMM_ERR_INVALID / MSGEMM_ERR_UNSORTED without running
                                     the product.  Without validation, out-of-range indices
                                     are undefined behaviour. */
    MSGEMM_OPT_DOT = 3,           /* value 0/1 (default 1): allow the pull (DOT) kernel in AUTO */
    MSGEMM_OPT_PROFILE = 4,       /* value 0/1 (default 0): record CUDA events around every
                                     phase and kernel launch of a call, on the handle's stream
                                     (read back with msgemm_profile_entry) */
    MSGEMM_OPT_TILE_INDEX = 5,    /* value 0/1 (default 1): heavy rows of wide products walk
                                     their column tiles through a tile index of B
                                     (rows(B) x (tiles + 1) ints, built per call, 4 GiB cap);
                                     0, or a product over the cap, uses per-entry cursors */
    MSGEMM_OPT_GRID = 6,          /* value 0/1/2 (default 1): heavy rows are processed as
                                     (row, column tile) items swept tile by tile over the whole
                                     GPU -- 1: complemented rows whose output is dense (room
                                     n - nnz(M_i*) each) and plain rows over the flop bound of
                                     MSGEMM_OPT_GRID_MIN_FLOPS, 2: every heavy row (tests),
                                     0: never (one CTA walks all tiles of a row); needs the
                                     tile index (or a single tile) */
    MSGEMM_OPT_WARP_SLAB = 7,     /* value 1024..24576, a multiple of 16 (default 4608): shared
                                     bytes per warp of the one-warp MCA and pull kinds; rows
                                     whose arrays do not fit go to the one-CTA kinds */
    MSGEMM_OPT_GRID_MIN_FLOPS = 8, /* value >= 0 (default 2^20): plain-mask rows with at least
                                     this many push products, in products wider than one
                                     column tile, are processed as (row, tile) items over the
                                     whole GPU (at most 4096 to 65536 such rows per call, by
                                     the product's width; the rest and every lighter row keep
                                     one CTA or warp per row) */
    MSGEMM_OPT_PHASES = 9,        /* value 1/2 (default 1), for msgemm_run, msgemm_run_batched
                                     and msgemm_autotune (Sec. 6).  1: one phase -- rows write
                                     to a temporary the size of the mask (plain) or of the
                                     per-row bounds (complemented), then a compaction copies
                                     them into C.  2: a symbolic pass counts each row's entries
                                     from the indices alone, C is allocated to its exact size
                                     (capacity == nnz; the call synchronises once more), and a
                                     numeric pass writes each row in place: no temporary, more
                                     work.  Two phases never use the (row, tile) grid kinds
                                     nor a CUDA graph (use_graph is ignored). */
    MSGEMM_OPT_HASH_KICKS = 10,   /* value 0..4096 (default 64): the hash rows (Sec. 5.3) place
                                     each mask column by two-choice (cuckoo) hashing, moving at
                                     most this many keys per insertion; a row whose insertion
                                     runs out retries with a second pair of hash functions, then
                                     falls back to linear probing.  0 = linear probing only.
                                     The result never depends on it (tests use 0 and 1 to run
                                     every build path). */
    MSGEMM_OPT_QTEAM_FLOPS = 11,  /* value 0..2^20 (default 1024): plain rows with at most 8 mask
                                     entries and at most this many push products take the
                                     mask-compressed accumulator (Sec. 5.4) on a team of eight
                                     lanes (four rows per warp, the mask row and its accumulators
                                     in registers) -- under AUTO and when MCA is forced; 0 = never */
    MSGEMM_OPT_HASH_SLAB = 12     /* value 1024..24576, a multiple of 16 (default 4608): shared
                                     bytes per warp of the one-warp hash kinds (their table is a
                                     power of two of 4-byte keys and accumulators); rows whose
                                     table does not fit go to the one-CTA hash kinds */
} msgemm_option;

/* Input CSR matrix (device pointers, borrowed). */
typedef struct {
    int32_t nrows, ncols;
    int64_t nnz;                 /* == rowptr[nrows]; must be < 2^31 */
    const int32_t *rowptr;       /* nrows + 1 entries */
    const int32_t *colidx;       /* nnz entries, strictly ascending per row */
    const void *values;          /* nnz entries, or NULL (plus-pair, masks, pattern operands) */
} msgemm_csr;

/* Output CSR matrix.  The library fills every field; the arrays come from the
 * handle's allocation callback and belong to the caller afterwards.
 * capacity is the room of colidx/values; the true entry count is *d_nnz
 * (a device int64) and rowptr[nrows] (device).  A call allocates each array
 * kind (row pointers, entry counts, and columns and values once for the
 * outputs sized by their mask and once for those sized after counting) in ONE
 * callback allocation for all its products, carved in 16-byte-aligned
 * slices: an array either is such an allocation (its callback's return
 * value: the first product it serves) or lies inside one.  The caller frees
 * exactly the pointers its callback returned. */
typedef struct {
    int32_t nrows, ncols;
    int32_t *rowptr;
    int32_t *colidx;
    void *values;
    int64_t capacity;
    int64_t *d_nnz;
} msgemm_csr_out;

/* Device memory callbacks: alloc returns a device pointer (256-byte aligned)
 * or NULL; free releases it.  Both are called on the host from inside
 * library calls, never from a kernel or a stream callback. */
typedef void *(*msgemm_alloc_fn)(size_t bytes, void *ctx);
typedef void (*msgemm_free_fn)(void *ptr, void *ctx);

typedef struct msgemm_handle msgemm_handle;

/* Creates a handle bound to the current CUDA device and to `stream` (a
 * cudaStream_t; NULL = the legacy default stream).  With alloc/free NULL the
 * library uses cudaMalloc/cudaFree.  Workspace (row scores, bins, temporary
 * output room, tile cursors) belongs to the handle and is reused; a free
 * callback must honour stream order (torch's caching allocator does). */
msgemm_status msgemm_create(msgemm_handle **handle, void *stream,
                            msgemm_alloc_fn alloc, msgemm_free_fn free_fn, void *ctx);

/* Rebinds the handle to another stream (synchronises the old one first). */
msgemm_status msgemm_set_stream(msgemm_handle *handle, void *stream);

msgemm_status msgemm_set_option(msgemm_handle *handle, msgemm_option option, int64_t value);

/* C = M .* (A B) (complement == 0) or C = !M .* (A B) (complement != 0),
 * Sec. 2.  Allocates C: rowptr (m + 1), colidx and values with
 * capacity = nnz(M) for a plain mask -- no host synchronisation -- and, for a
 * complemented mask, capacity = the exact entry count, which costs two
 * host synchronisations (one for the temporary room, one for the count).
 * Pipeline: row binning by flops and mask size, per-bin accumulator kernels
 * (MSA / hash / MCA / pull-dot with per-row tables in shared memory; a
 * column-tiled shared-memory MSA for rows too heavy for one table), then
 * compaction into canonical CSR. */
msgemm_status msgemm_run(msgemm_handle *handle, const msgemm_csr *M, int complement,
                         const msgemm_csr *A, const msgemm_csr *B, msgemm_semiring semiring,
                         msgemm_csr_out *C);

/* Gradients of l = sum_ij G_ij C_ij for C = M .* (A B), plus-times fp32:
 *   dA = pattern(A) .* (G B^T)   -> dA_vals[t] for A's t-th stored entry
 *   dB = pattern(B) .* (A^T G)   -> dB_vals[t] for B's t-th stored entry
 * G is m x n, fp32, stored on the pattern of C (any pattern contained in M's
 * gives the same result).  Both are masked products run by the same
 * accumulators: dA as pull (DOT) over rows of G and rows of B, dB as push over
 * rows of A^T (built by a transpose kernel) and rows of G.  dA_vals / dB_vals
 * are caller-allocated device float arrays of nnz(A) / nnz(B) entries; either
 * may be NULL to skip it.  Returns UNSUPPORTED for any other semiring. */
msgemm_status msgemm_backward(msgemm_handle *handle, const msgemm_csr *A, const msgemm_csr *B,
                              const msgemm_csr *G, msgemm_semiring semiring,
                              float *dA_vals, float *dB_vals);

/* A backward plan: the transposes msgemm_backward builds on every call (B^T
 * and A^T), built once for fixed patterns of A and B -- the usual case when
 * training values on a fixed sparsity pattern.  The plan keeps the two
 * transposed patterns with ascending rows and, for each of their entries,
 * the position of its value in A or B; msgemm_backward_planned then only
 * gathers the current values by those positions (one light kernel each)
 * before the two masked products, instead of counting, scanning, scattering
 * and sorting.  Results equal msgemm_backward's (same products, same
 * accumulators; the summation order inside an entry may differ, within the
 * fp32 bound).
 * The plan records A's and B's row-pointer and column arrays by address and
 * their sizes: the arrays must hold the same pattern while the plan is used
 * (planned calls with other addresses or sizes return MSGEMM_ERR_INVALID).
 * Its memory (about 12 bytes per stored entry of A and of B, plus the row
 * pointers) comes from the handle's allocation callback; destroy the plan
 * with the same handle, before the handle.  Planned calls on one plan share
 * its value arrays: run them on one stream.  Asynchronous on the handle's
 * stream. */
typedef struct msgemm_backward_plan msgemm_backward_plan;
msgemm_status msgemm_backward_plan_create(msgemm_handle *handle, const msgemm_csr *A, const msgemm_csr *B,
                                          msgemm_backward_plan **plan);
/* dA and dB as msgemm_backward (plus-times fp32) for the plan's patterns. */
msgemm_status msgemm_backward_planned(msgemm_handle *handle, msgemm_backward_plan *plan,
                                      const msgemm_csr *A, const msgemm_csr *B, const msgemm_csr *G,
                                      float *dA_vals, float *dB_vals);
void msgemm_backward_plan_destroy(msgemm_handle *handle, msgemm_backward_plan *plan);

/* nprod independent products C[p] = M[p] .* (A[p] B[p]) (or complemented per
 * complement[p], which may be NULL for all-plain), one semiring.  Binning,
 * accumulation and compaction for all products run as one pipeline: rows of
 * every product are binned together, and each accumulator kind is ONE
 * persistent kernel over the rows of that kind in all products (grid =
 * resident CTAs x SMs), so the launch count does not grow with nprod.
 * With use_graph != 0 and every mask plain (and neither validation nor
 * profiling on), the device part of the pipeline is captured into a CUDA
 * graph on first use and replayed while the arguments stay the same (the
 * same input pointers and sizes, the same handle options and workspace);
 * outputs may differ between replays: they are passed through a device table
 * uploaded before each replay.  Anything else runs eagerly.  The C[p] share
 * allocations (see msgemm_csr_out): four callback calls for a batch of plain
 * masks however many products it holds, two more when some mask is
 * complemented (those synchronise the host as in msgemm_run). */
msgemm_status msgemm_run_batched(msgemm_handle *handle, int nprod, const msgemm_csr *M,
                                 const int *complement, const msgemm_csr *A, const msgemm_csr *B,
                                 msgemm_semiring semiring, msgemm_csr_out *C, int use_graph);

/* Tunes the handle's binning policy on the given batch by timing it
 * (synchronises; every candidate computes the same result).  Starting with
 * the pull kernel off: for each row class carrying work (4 push-flop bands x
 * 4 mask-row bands), the accumulator family tried first (MSA, hash, MCA,
 * Heap or HeapDot), then the flop bound between warp and CTA rows, the warp
 * slab, the flop bound of the (row, tile) grid rows, and last the pull/push
 * ratio below which rows take the pull kernel (or pull kept off).  The
 * starting policy is kept when no candidate beats it.  With cache_path !=
 * NULL the tuned policy is stored there as JSON keyed by device name and
 * semiring, and read back instead of timing when the file already holds
 * that key (a malformed entry is ignored).  nprod == 0 only loads the
 * cache. */
msgemm_status msgemm_autotune(msgemm_handle *handle, int nprod, const msgemm_csr *M,
                              const int *complement, const msgemm_csr *A, const msgemm_csr *B,
                              msgemm_semiring semiring, const char *cache_path);

/* Betweenness centrality from a batch of sources (the application of Sec.
 * 8.3, Brandes' algorithm in matrix form over this library's products).
 * Forward: level 0 = the sources (one row per source), level d + 1 =
 * !visited .* (level_d A) on plus-times int64, so each entry carries sigma,
 * the number of shortest paths from its row's source; visited = levels
 * 0..d.  Backward, from the deepest level: W = (1 + delta) / sigma on level
 * d, T = level_{d-1} .* (W A^T) on plus-times fp32 (values at each entry's
 * own slot), delta = sigma T on level d-1.  centrality[v] (device, n
 * doubles, overwritten) = sum over the sources s != v of delta_s(v).  A is
 * n x n, an edge v -> w per stored entry (v, w); its values are ignored.
 * sources: device int32[nsrc], each in [0, n) (checked on the host).
 * *levels (host, optional) = number of BFS levels including level 0.
 * Synchronises once per level; allocates its workspace through the handle. */
msgemm_status msgemm_bc(msgemm_handle *handle, const msgemm_csr *A, const int32_t *sources, int nsrc,
                        double *centrality, int32_t *levels);

/* k-truss (the application of Sec. 8.2; k = 5 in its benchmark): the
 * largest subgraph of the symmetric n x n pattern A in which every edge lies
 * on at least k - 2 triangles of the subgraph.  Each round computes every
 * edge's support as A .* (A A) on plus-pair (values at each entry's own
 * slot) and drops the edges below k - 2; it stops when a round drops none.
 * Self loops are dropped first.  T (allocated like an output) = the truss's
 * pattern, values = each edge's support (int64).  *iterations (optional) =
 * rounds run; *products (optional) = products kept by the masks over all
 * rounds (the sum of the supports; masked flops = 2x).  Synchronises every
 * round. */
msgemm_status msgemm_ktruss(msgemm_handle *handle, const msgemm_csr *A, int64_t k, msgemm_csr_out *T,
                            int32_t *iterations, int64_t *products);

/* Transpose (CSR of A^T), value_bytes in {0, 4, 8}.  At is allocated like an
 * output (capacity nnz(A)).  Column indices within a row of A^T are in
 * arbitrary order unless sorted != 0, which adds a segmented sort pass
 * (bitonic per row) and gives strictly ascending rows.  Synchronises. */
msgemm_status msgemm_transpose(msgemm_handle *handle, const msgemm_csr *A, int value_bytes,
                               int sorted, msgemm_csr_out *At);

/* Transpose that allocates nothing.  The paper has no counterpart to this
 * entry point: it serves callers that cannot allocate device memory where
 * they need a transpose -- runtimes that hand out all device memory from
 * their own fixed pools and forbid any other allocation, hosts with no
 * device allocator to pass in, and latency-critical paths where cudaMalloc
 * (which may synchronise the device) is not acceptable.
 * It needs no handle.  Result as msgemm_transpose(A, value_bytes, sorted),
 * written into caller-owned device arrays: At_rowptr (ncols(A) + 1 entries),
 * At_colidx and At_values (nnz(A) entries; At_values unused when value_bytes
 * is 0).  Asynchronous on `stream` (a cudaStream_t; NULL = legacy default).
 * Its scratch (per-column cursors, scan tile sums) is one file-scope device
 * array of about 4 MiB that every GPU loading the library keeps until the
 * process exits; it bounds ncols(A) at 1,048,576 -- larger returns
 * MSGEMM_ERR_OVERFLOW before any work.  The first call on a device looks up
 * the array's device address with that device current; make that first call
 * before any stream capture.  Every call shares the array, which keeps the
 * previous call's contents (each call clears what it needs; the sort pass
 * reuses the cursor area for its list of long rows), so calls that overlap on
 * the GPU race: serialise them (one stream, or events).  The call returns
 * before the GPU work is done: the outputs are valid once `stream` reaches
 * this point, so synchronise the stream, or record an event on it and wait
 * for that, before reading them from another stream or from the host.
 * Entries whose column index lies outside [0, ncols(A)) are skipped (never
 * written anywhere); At_rowptr then counts only the entries in range. */
msgemm_status msgemm_transpose_noalloc(const msgemm_csr *A, int value_bytes, int sorted, int32_t *At_rowptr,
                                       int32_t *At_colidx, void *At_values, void *stream);

/* *d_sum (device, 8 bytes) = sum of C's values: int64 wrapping for the int64
 * semirings (the triangle count of Sec. 8.2 for C = L .* (L L) on plus-pair),
 * fp64 accumulation rounded into a double for plus-times fp32. */
msgemm_status msgemm_reduce_sum(msgemm_handle *handle, const msgemm_csr_out *C,
                                msgemm_semiring semiring, void *d_sum);

/* Synchronises the handle's stream and reports (then clears) the device error
 * word: MSGEMM_ERR_INVALID / _UNSORTED for a validation failure,
 * MSGEMM_ERR_TIMEOUT for a bounded wait that ran out, MSGEMM_ERR_CUDA for a
 * failed launch or copy. */
msgemm_status msgemm_sync_status(msgemm_handle *handle);

/* Copies a NUL-terminated description of the last error into buf. */
msgemm_status msgemm_last_error_detail(msgemm_handle *handle, char *buf, size_t len);

/* Per-kind row counts of the last msgemm_run / msgemm_run_batched binning
 * (synchronises): counts[kind] for kind < min(n, msgemm_num_kinds()). */
int msgemm_num_kinds(void);
msgemm_status msgemm_bin_counts(msgemm_handle *handle, int64_t *counts, int n);

/* Phase timings of the last call made with MSGEMM_OPT_PROFILE on (synchronises).
 * msgemm_profile_count returns the number of entries; entry idx gives the
 * phase name (NUL-terminated, truncated to len) and its device time in ms. */
int msgemm_profile_count(msgemm_handle *handle);
msgemm_status msgemm_profile_entry(msgemm_handle *handle, int idx, char *name, size_t len, float *ms);

/* Kind (msgemm row kind index, as counted by msgemm_bin_counts) of each row of
 * the last msgemm_run / msgemm_run_batched, copied to host memory `kinds`
 * (nrows bytes; rows of all products concatenated).  Synchronises. */
msgemm_status msgemm_last_row_kinds(msgemm_handle *handle, uint8_t *kinds, int64_t nrows);

/* Process-wide number of kernels this library has launched so far. */
int64_t msgemm_kernel_launches(void);

/* Frees the workspace and the handle (synchronises its stream). */
void msgemm_destroy(msgemm_handle *handle);

#ifdef __cplusplus
}
#endif
#endif /* MSGEMM_H */
