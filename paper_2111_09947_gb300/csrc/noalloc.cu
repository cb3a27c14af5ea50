// Transpose that allocates nothing: msgemm_transpose_noalloc (declared in
// include/msgemm.h).
//
// Some callers cannot allocate device memory at the point where they need a
// transpose: runtimes that hand the library fixed memory pools and forbid any
// other allocation, embedded hosts that have no allocator to give, and
// latency-critical paths that cannot afford cudaMalloc (it may synchronise
// the device).  For them this entry point takes the input and
// the caller's output arrays and a stream, and keeps its scratch (the
// per-column cursors and the scan's tile sums) in the file-scope device array
// below, which every GPU that loads the library holds until the process exits.
#include <mutex>

#include "launch.h"

namespace msg {
namespace {

// Largest number of columns of A (rows of A^T) this entry point accepts.
constexpr long long NOALLOC_MAX_COLS = 1 << 20;
constexpr size_t NOALLOC_CURSOR_BYTES = ((size_t)(NOALLOC_MAX_COLS + 1) * sizeof(int) + 255) & ~size_t(255);
constexpr size_t NOALLOC_TILE_BYTES = (size_t)(NOALLOC_MAX_COLS / STILE + 4) * sizeof(long long);

// Scratch shared by every call: cursors first, then scan tile sums.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_CURSOR_BYTES + NOALLOC_TILE_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[MAX_DEVICES];   // device address of the array, per device
int g_nsm[MAX_DEVICES];

// Once per device, with that device current: the array's device address
// (the host-side symbol is only a stand-in and must not reach a kernel).
cudaError_t setup(int dev) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_scratch_addr[dev]) return cudaSuccess;
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    int nsm = 0;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g_nsm[dev] = nsm;
    g_scratch_addr[dev] = ptr;
    return cudaSuccess;
}

}  // namespace
}  // namespace msg

using namespace msg;

extern "C" msgemm_status msgemm_transpose_noalloc(const msgemm_csr *A, int value_bytes, int sorted,
                                                  int32_t *At_rowptr, int32_t *At_colidx, void *At_values,
                                                  void *stream) {
    if (!A || !At_rowptr || A->nrows < 0 || A->ncols < 0 || A->nnz < 0 || !A->rowptr)
        return MSGEMM_ERR_INVALID;
    if (value_bytes != 0 && value_bytes != 4 && value_bytes != 8) return MSGEMM_ERR_INVALID;
    if (A->nnz > 0 && (!A->colidx || !At_colidx || (value_bytes && (!A->values || !At_values))))
        return MSGEMM_ERR_INVALID;
    if (A->nnz >= (1LL << 31)) return MSGEMM_ERR_OVERFLOW;
    if ((long long)A->ncols > NOALLOC_MAX_COLS) return MSGEMM_ERR_OVERFLOW;   // beyond the scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return MSGEMM_ERR_CUDA;
    if (setup(dev) != cudaSuccess) return MSGEMM_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nsm = g_nsm[dev];
    unsigned char *base = static_cast<unsigned char *>(g_scratch_addr[dev]);
    int *cursor = reinterpret_cast<int *>(base);
    long long *tiles = reinterpret_cast<long long *>(base + NOALLOC_CURSOR_BYTES);
    const int n = A->ncols;
    // column counts (the cursors are cleared first: the array keeps the last
    // call's contents), their exclusive scan into At's row pointers, then the
    // scatter with the cursors restarted at those row pointers
    if (launch_col_counts(A->colidx, A->nnz, n, cursor, st, nsm) != cudaSuccess) return MSGEMM_ERR_CUDA;
    if (launch_excl_scan_int(cursor, n, At_rowptr, tiles, st, nsm) != cudaSuccess) return MSGEMM_ERR_CUDA;
    if (cudaMemcpyAsync(cursor, At_rowptr, sizeof(int) * ((size_t)n + 1), cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess)
        return MSGEMM_ERR_CUDA;
    if (launch_transpose_fill(A->rowptr, A->colidx, A->values, value_bytes, A->nrows, n, cursor, At_colidx,
                              At_values, nullptr, st, nsm) != cudaSuccess)
        return MSGEMM_ERR_CUDA;
    // the cursors (n + 1 ints) are free after the scatter: they hold the sort's row list
    if (sorted && launch_segsort(At_rowptr, At_colidx, At_values, value_bytes, n, cursor, st, nsm) != cudaSuccess)
        return MSGEMM_ERR_CUDA;
    return MSGEMM_OK;
}
