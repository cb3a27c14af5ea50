// Host-side launchers shared between the translation units.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

#include <atomic>

namespace msg {

// Kernels launched by this library (process-wide), for launch accounting.
extern std::atomic<long long> g_kernel_launches;
inline cudaError_t counted(cudaError_t e, int n = 1) {
    g_kernel_launches.fetch_add(n, std::memory_order_relaxed);
    return e;
}

struct RowLaunch;

// Per semiring (rows_f32.cu, rows_i64.cu, rows_pp.cu).
cudaError_t launch_bin_score_f32(const ProdSet &, const RowArrays &, const Policy &, long long *room, cudaStream_t, int nsm);
cudaError_t launch_bin_score_i64(const ProdSet &, const RowArrays &, const Policy &, long long *room, cudaStream_t, int nsm);
cudaError_t launch_bin_score_pp(const ProdSet &, const RowArrays &, const Policy &, long long *room, cudaStream_t, int nsm);
cudaError_t launch_kind_f32(int kind, const ProdSet &, const RowLaunch &, cudaStream_t, int nsm);
cudaError_t launch_kind_i64(int kind, const ProdSet &, const RowLaunch &, cudaStream_t, int nsm);
cudaError_t launch_kind_pp(int kind, const ProdSet &, const RowLaunch &, cudaStream_t, int nsm);

// Threads per CTA of each kind's kernel.
inline int kind_threads(int kind) {
    switch (kind) {
    case K_MSA_W: return 128;
    case K_MSA_T: case K_CMSA_T: return 512;
    case K_CMSA_G: case K_MSA_G: return 1024;
    default: return 256;
    }
}
inline bool kind_is_warp(int kind) {
    return kind == K_MSA_W || kind == K_HASH_W || kind == K_MCA_W || kind == K_DOT_W || kind == K_CHASH_W ||
           kind == K_HEAP_W || kind == K_HEAPDOT_W || kind == K_CHEAP_W;
}
// Dynamic shared memory of a kind's launch for a given slab.
inline size_t kind_smem(int kind, int slab) {
    return kind_is_warp(kind) ? (size_t)slab * (kind_threads(kind) / 32) : (size_t)slab;
}

// pipeline.cu
cudaError_t launch_bin_scatter(const RowArrays &, cudaStream_t, int nsm);
cudaError_t launch_scan_room(const RowArrays &, const long long *room, long long comp_base, long long *tile_buf,
                             long long *total, cudaStream_t, int nsm);
cudaError_t launch_count_tiles(const ProdSet &, const RowArrays &, long long ntiles, long long *tile_sums,
                               long long *tile_offs, long long *prod_totals, long long *chunk_start, cudaStream_t,
                               int nsm);
cudaError_t launch_compact(const ProdSet &, const RowArrays &, const TmpOut &, long long ntiles,
                           const long long *tile_offs, const long long *chunk_start, long long max_chunks,
                           int out_bytes, cudaStream_t, int nsm);
cudaError_t launch_row_offsets(const ProdSet &, const RowArrays &, long long ntiles, const long long *tile_offs,
                               cudaStream_t, int nsm);
cudaError_t launch_col_counts(const int *ci, long long nnz, int ncols, int *counts, cudaStream_t, int nsm);
cudaError_t launch_excl_scan_int(const int *in, long long n, int *out, long long *tile_buf, cudaStream_t, int nsm);
// Entries whose column is outside [0, ncols) are skipped (not transposed).
cudaError_t launch_transpose_fill(const int *rp, const int *ci, const void *v, int vbytes, int nrows,
                                  int ncols, int *cursor, int *tci, void *tv, const int *gate,
                                  cudaStream_t, int nsm);
cudaError_t launch_validate(const int *rp, const int *ci, int nrows, int ncols, long long nnz, unsigned *err,
                            cudaStream_t, int nsm);
cudaError_t launch_reduce_sum(int semiring, const void *vals, const long long *d_nnz, void *d_sum, cudaStream_t,
                              int nsm);
cudaError_t launch_sort_heavy(const RowArrays &, int kind, cudaStream_t);
// One product's B for the multi-product transpose (pull kernel).
struct BtDesc {
    const int *rp, *ci;
    const void *v;
    int nrows, ncols;
    long long nnz;
    long long co;   // first count slot (ncols + 1 slots per product)
    long long eo;   // first entry in the concatenation of all entries
    long long ro;   // first row in the concatenation of all rows
};
cudaError_t launch_bt_counts_multi(const BtDesc *d, int Q, long long total_nnz, int *counts, long long ncounts,
                                   cudaStream_t, int nsm);
cudaError_t launch_bt_fill_multi(const BtDesc *d, int Q, long long total_rows, int vbytes, int *cursor, int *tci,
                                 void *tv, const int *gate, cudaStream_t, int nsm);
cudaError_t launch_tile_bounds(const int *rp, const int *ci, int nrows, int T, int nt, int *tpos, const int *gate,
                               cudaStream_t, int nsm);
// scratch: nrows + 1 ints of device memory (a list of the long rows)
cudaError_t launch_segsort(const int *rp, int *ci, void *v, int vbytes, int nrows, int *scratch, cudaStream_t,
                           int nsm);

// apps.cu: elementwise steps of batched betweenness centrality and k-truss
cudaError_t launch_bc_sources(const int *src, int nsrc, int *rp, int *ci, long long *v, cudaStream_t, int nsm);
cudaError_t launch_bitmap_or(const int *rp, const int *ci, int nrows, long long wpr, unsigned *bm, cudaStream_t,
                             int nsm);
cudaError_t launch_bitmap_counts(const unsigned *bm, int nrows, long long wpr, int *cnt, cudaStream_t, int nsm);
cudaError_t launch_bitmap_cols(const unsigned *bm, int nrows, long long wpr, const int *rp, int *ci, cudaStream_t,
                               int nsm);
cudaError_t launch_bc_weight(const long long *sigma, const float *T, long long nnz, float *W, cudaStream_t, int nsm);
cudaError_t launch_bc_accum(const int *ci, const long long *sigma, const float *T, long long nnz, double *bc,
                            cudaStream_t, int nsm);
cudaError_t launch_filter_counts(const int *rp, const int *ci, int nrows, const long long *sup, long long thr, int *cnt,
                                 cudaStream_t, int nsm);
cudaError_t launch_filter_write(const int *rp, const int *ci, int nrows, const long long *sup, long long thr,
                                const int *nrp, int *nci, long long *nsup, cudaStream_t, int nsm);
cudaError_t launch_iota_i32(int *p, long long n, cudaStream_t, int nsm);
cudaError_t launch_gather_f32(const int *perm, const float *src, long long n, float *dst, cudaStream_t, int nsm);

constexpr int CTILE = 1024;        // rows per compaction tile
constexpr int CCH = 8192;          // output entries per compaction chunk
constexpr int STILE = 2048;        // elements per generic scan tile

}  // namespace msg
