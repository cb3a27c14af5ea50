// Pipeline kernels that do not depend on the semiring: bucket scatter of the
// binned rows, scans, compaction of the one-phase output (Sec. 6: the output
// is first written into room sized by the mask, then copied out), the
// transpose used by the pull kernel and the backward products, input
// validation and the value reduction (triangle count, Sec. 8.2).
#include <algorithm>

#include "launch.h"

namespace msg {

std::atomic<long long> g_kernel_launches{0};

static int grid_cap(long long work_blocks, int nsm, int per_sm) {
    long long g = std::min<long long>(work_blocks, (long long)nsm * per_sm);
    return (int)std::max<long long>(1, g);
}

// ------------------------------------------------------------ bucket scatter
// perm holds the rows grouped by kind and, within a kind, by flops class
// heaviest first (the order the row kernels take them in); within a class the
// order is arbitrary.
constexpr int NSUB = NKIND * NCLS_FLOPS;
__global__ void __launch_bounds__(256) k_bin_scatter(const __grid_constant__ RowArrays ra) {
    __shared__ int off[NSUB + 1];
    __shared__ int loc[NSUB];
    __shared__ int base[NSUB];
    if (threadIdx.x == 0) {
        off[0] = 0;
        for (int k = 0; k < NSUB; ++k) off[k + 1] = off[k] + ra.sub_count[k];
        if (blockIdx.x == 0)
            for (int k = 0; k <= NKIND; ++k) ra.kind_off[k] = off[k * NCLS_FLOPS];
    }
    for (long long r0 = (long long)blockIdx.x * blockDim.x; r0 < ra.R; r0 += (long long)gridDim.x * blockDim.x) {
        for (int x = threadIdx.x; x < NSUB; x += blockDim.x) loc[x] = 0;
        __syncthreads();
        const long long r = r0 + threadIdx.x;
        int key = -1, rank = 0;
        if (r < ra.R) {
            const int k = ra.kind[r];
            if (k != K_EMPTY) {
                key = k * NCLS_FLOPS + flops_sub(ra.flops[r]);
                rank = atomicAdd(&loc[key], 1);
            }
        }
        __syncthreads();
        for (int x = threadIdx.x; x < NSUB; x += blockDim.x)
            if (loc[x]) base[x] = atomicAdd(&ra.sub_fill[x], loc[x]);
        __syncthreads();
        if (key >= 0) ra.perm[off[key] + base[key] + rank] = (int)r;
        __syncthreads();
    }
}

cudaError_t launch_bin_scatter(const RowArrays &ra, cudaStream_t st, int nsm) {
    if (ra.R == 0) return cudaSuccess;
    k_bin_scatter<<<grid_cap((ra.R + 255) / 256, nsm, 8), 256, 0, st>>>(ra); g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

// ------------------------------------------------------------ generic scans
// Block-wide exclusive scan of int64 values (256 threads).
__device__ __forceinline__ long long block_excl_scan_ll(long long v, long long *sh, long long *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) sh[w] = incl;
    __syncthreads();
    if (w == 0) {
        long long x = lane < nw ? sh[lane] : 0;
        long long xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long t = __shfl_up_sync(FULL, xi, o);
            if (lane >= o) xi += t;
        }
        if (lane < nw) sh[lane] = xi - x;
        if (lane == 31) sh[32] = xi;
    }
    __syncthreads();
    long long res = sh[w] + incl - v;
    *total = sh[32];
    __syncthreads();
    return res;
}

// Single-block exclusive scan in place over n values; *total = sum.
__global__ void __launch_bounds__(1024) k_scan_small_ll(long long *v, long long n, long long *total) {
    __shared__ long long sh[33];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long b = 0; b < n; b += blockDim.x) {
        const long long x = b + threadIdx.x;
        const long long val = x < n ? v[x] : 0;
        long long tot;
        const long long ex = block_excl_scan_ll(val, sh, &tot);
        if (x < n) v[x] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

// Tile sums of an int64 array (tiles of STILE elements, 256 threads).
__global__ void __launch_bounds__(256) k_tile_sums_ll(const long long *in, long long n, long long *sums, long long ntiles) {
    __shared__ long long sh[33];
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        long long s = 0;
        for (long long x = t * STILE + threadIdx.x; x < std::min(n, (t + 1) * STILE); x += blockDim.x) s += in[x];
        long long tot;
        block_excl_scan_ll(s, sh, &tot);
        if (threadIdx.x == 0) sums[t] = tot;
    }
}

// Complemented rows: tmpoff[r] = comp_base + exclusive prefix of room[] for
// rows with room > 0.
__global__ void __launch_bounds__(256) k_room_apply(const long long *room, long long *tmpoff, long long n,
                                                    const long long *tile_offs, long long comp_base, long long ntiles) {
    __shared__ long long sh[33];
    constexpr int PER = STILE / 256;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long long x0 = t * STILE + (long long)threadIdx.x * PER;
        long long v[PER];
        long long s = 0;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            v[u] = (x0 + u < n) ? room[x0 + u] : 0;
            s += v[u];
        }
        long long tot;
        long long ex = block_excl_scan_ll(s, sh, &tot) + tile_offs[t] + comp_base;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            if (x0 + u < n && v[u] > 0) tmpoff[x0 + u] = ex;
            ex += v[u];
        }
    }
}

cudaError_t launch_scan_room(const RowArrays &ra, const long long *room, long long comp_base, long long *tile_buf,
                             long long *total, cudaStream_t st, int nsm) {
    const long long n = ra.R;
    if (n == 0) return cudaMemsetAsync(total, 0, sizeof(long long), st);
    const long long nt = (n + STILE - 1) / STILE;
    k_tile_sums_ll<<<grid_cap(nt, nsm, 8), 256, 0, st>>>(room, n, tile_buf, nt); g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    k_scan_small_ll<<<1, 1024, 0, st>>>(tile_buf, nt, total); g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    k_room_apply<<<grid_cap(nt, nsm, 8), 256, 0, st>>>(room, ra.tmpoff, n, tile_buf, comp_base, nt); g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

// ------------------------------------------------------------ compaction
__device__ __forceinline__ int prod_of_tile(const ProdSet &ps, long long t) {
    if (ps.P == 1) return 0;
    int lo = 0, hi = ps.P - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ps.tab[mid].tile0 <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Sum of kept counts per compaction tile (CTILE rows of one product).
__global__ void __launch_bounds__(256) k_count_tiles(const __grid_constant__ ProdSet ps, const __grid_constant__ RowArrays ra,
                                                     long long ntiles, long long *sums) {
    __shared__ long long sh[33];
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const DevProd &P = prod_at(ps, prod_of_tile(ps, t));
        const long long lt = t - P.tile0;
        const long long r0 = P.row0 + lt * CTILE;
        const long long r1 = P.row0 + std::min<long long>(P.m, (lt + 1) * CTILE);
        long long s = 0;
        for (long long r = r0 + threadIdx.x; r < r1; r += blockDim.x) s += ra.cnt[r];
        long long tot;
        block_excl_scan_ll(s, sh, &tot);
        if (threadIdx.x == 0) sums[t] = tot;
    }
}

// Exclusive scan of tile sums, restarted per product; writes each product's
// entry count to *c_nnz, c_rp[m] and prod_totals[p].
__global__ void __launch_bounds__(1024) k_scan_tiles(const __grid_constant__ ProdSet ps, long long ntiles,
                                                     const long long *sums, long long *offs, long long *prod_base,
                                                     long long *prod_totals, long long *chunk_start) {
    __shared__ long long sh[33];
    __shared__ long long carry, ccarry;
    if (threadIdx.x == 0) carry = ccarry = 0;
    __syncthreads();
    for (long long b = 0; b < ntiles; b += blockDim.x) {
        const long long x = b + threadIdx.x;
        const long long val = x < ntiles ? sums[x] : 0;
        long long tot;
        const long long ex = block_excl_scan_ll(val, sh, &tot);
        if (x < ntiles) offs[x] = carry + ex;
        // copy chunks of a tile: at least one (it also writes the row pointers)
        const long long nch = x < ntiles ? std::max(1LL, (val + CCH - 1) / CCH) : 0;
        long long ctot;
        const long long cex = block_excl_scan_ll(nch, sh, &ctot);
        if (x < ntiles) chunk_start[x] = ccarry + cex;
        __syncthreads();
        if (threadIdx.x == 0) { carry += tot; ccarry += ctot; }
        __syncthreads();
    }
    if (threadIdx.x == 0) chunk_start[ntiles] = ccarry;
    for (int p = threadIdx.x; p < ps.P; p += blockDim.x) {
        const DevProd &P = prod_at(ps, p);
        const long long nt = (P.m + CTILE - 1) / CTILE;
        long long base = 0, total = 0;
        if (nt > 0) {
            base = offs[P.tile0];
            total = offs[P.tile0 + nt - 1] + sums[P.tile0 + nt - 1] - base;
        }
        prod_base[p] = base;
        prod_totals[p] = total;
        *P.c_nnz = total;
        P.c_rp[P.m] = (int)total;
    }
    __syncthreads();
    for (long long t = threadIdx.x; t < ntiles; t += blockDim.x) offs[t] -= prod_base[prod_of_tile(ps, t)];
}

cudaError_t launch_count_tiles(const ProdSet &ps, const RowArrays &ra, long long ntiles, long long *tile_sums,
                               long long *tile_offs, long long *prod_totals, long long *chunk_start, cudaStream_t st,
                               int nsm) {
    if (ntiles > 0) { k_count_tiles<<<grid_cap(ntiles, nsm, 8), 256, 0, st>>>(ps, ra, ntiles, tile_sums); g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }
    // prod_totals holds 2 * P entries: [0, P) bases, [P, 2P) totals
    k_scan_tiles<<<1, 1024, 0, st>>>(ps, ntiles, tile_sums, tile_offs, prod_totals, prod_totals + ps.P, chunk_start); g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

// Compaction: the output of a tile (CTILE rows of one product) is cut into
// chunks of CCH entries, one CTA per chunk.  The CTA rebuilds its tile's
// row offsets by a block scan of the kept counts (and the first chunk of the
// tile writes them into C's row pointers), then copies its output range:
// each output position finds its row by binary search over the offsets, so
// reads and writes stay coalesced whatever the row lengths.
template <int OUTB>
__global__ void __launch_bounds__(256) k_compact(const __grid_constant__ ProdSet ps, const __grid_constant__ RowArrays ra,
                                                 const __grid_constant__ TmpOut tmp, long long ntiles,
                                                 const long long *offs, const long long *chunk_start) {
    using V = typename std::conditional<OUTB == 4, unsigned, unsigned long long>::type;
    __shared__ long long sh[33];
    __shared__ int rowoff[CTILE + 1];
    __shared__ long long src0[CTILE];
    __shared__ long long s_tile;
    constexpr int PER = CTILE / 256;
    const long long nch = chunk_start[ntiles];
    for (long long ch = blockIdx.x; ch < nch; ch += gridDim.x) {
        if (threadIdx.x == 0) {
            long long lo = 0, hi = ntiles - 1;
            while (lo < hi) {
                const long long mid = (lo + hi + 1) >> 1;
                if (chunk_start[mid] <= ch) lo = mid; else hi = mid - 1;
            }
            s_tile = lo;
        }
        __syncthreads();
        const long long t = s_tile;
        const long long sub = ch - chunk_start[t];
        const DevProd &P = prod_at(ps, prod_of_tile(ps, t));
        const long long lt = t - P.tile0;
        const int i0 = (int)(lt * CTILE);
        const int i1 = (int)std::min<long long>(P.m, (lt + 1) * CTILE);
        int c[PER];
        long long s = 0;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int i = i0 + threadIdx.x * PER + u;
            c[u] = i < i1 ? ra.cnt[P.row0 + i] : 0;
            s += c[u];
        }
        long long tot;
        long long ex = block_excl_scan_ll(s, sh, &tot);
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int il = threadIdx.x * PER + u;
            if (i0 + il < i1) {
                rowoff[il] = (int)ex;
                src0[il] = ra.tmpoff[P.row0 + i0 + il];
                if (sub == 0) P.c_rp[i0 + il] = (int)(offs[t] + ex);
            }
            ex += c[u];
        }
        __syncthreads();
        const int nrow = i1 - i0;
        const long long base = offs[t];
        const long long o1 = std::min(tot, (sub + 1) * (long long)CCH);
        const V *src = static_cast<const V *>(tmp.v);
        V *dst = static_cast<V *>(P.c_v);
        for (long long o = sub * (long long)CCH + threadIdx.x; o < o1; o += blockDim.x) {
            int lo = 0, hi = nrow - 1;   // last row whose offset is <= o (it holds o)
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (rowoff[mid] <= o) lo = mid; else hi = mid - 1;
            }
            const long long so = src0[lo] + (o - rowoff[lo]);
            P.c_ci[base + o] = tmp.ci[so];
            dst[base + o] = src[so];
        }
        __syncthreads();
    }
}

cudaError_t launch_compact(const ProdSet &ps, const RowArrays &ra, const TmpOut &tmp, long long ntiles,
                           const long long *tile_offs, const long long *chunk_start, long long max_chunks,
                           int out_bytes, cudaStream_t st, int nsm) {
    if (ntiles == 0) return cudaSuccess;
    const int g = grid_cap(max_chunks, nsm, 8);
    if (out_bytes == 4) { k_compact<4><<<g, 256, 0, st>>>(ps, ra, tmp, ntiles, tile_offs, chunk_start); g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }
    else { k_compact<8><<<g, 256, 0, st>>>(ps, ra, tmp, ntiles, tile_offs, chunk_start); g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }
    return cudaGetLastError();
}

// Two-phase form (Sec. 6): after the symbolic launch, the row pointers of C
// and each row's final offset, from the per-row counts and the tiles' scanned
// offsets (one CTA per tile of CTILE rows).
__global__ void __launch_bounds__(256) k_row_offsets(const __grid_constant__ ProdSet ps,
                                                     const __grid_constant__ RowArrays ra, long long ntiles,
                                                     const long long *offs) {
    __shared__ long long sh[33];
    constexpr int PER = CTILE / 256;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const DevProd &P = prod_at(ps, prod_of_tile(ps, t));
        const long long lt = t - P.tile0;
        const int i0 = (int)(lt * CTILE);
        const int i1 = (int)std::min<long long>(P.m, (lt + 1) * CTILE);
        int c[PER];
        long long s = 0;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int i = i0 + threadIdx.x * PER + u;
            c[u] = i < i1 ? ra.cnt[P.row0 + i] : 0;
            s += c[u];
        }
        long long tot;
        long long ex = block_excl_scan_ll(s, sh, &tot);
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int i = i0 + threadIdx.x * PER + u;
            if (i < i1) {
                const long long o = offs[t] + ex;
                P.c_rp[i] = (int)o;
                ra.tmpoff[P.row0 + i] = o;
            }
            ex += c[u];
        }
        __syncthreads();
    }
}

cudaError_t launch_row_offsets(const ProdSet &ps, const RowArrays &ra, long long ntiles, const long long *tile_offs,
                               cudaStream_t st, int nsm) {
    if (ntiles == 0) return cudaSuccess;
    k_row_offsets<<<grid_cap(ntiles, nsm, 8), 256, 0, st>>>(ps, ra, ntiles, tile_offs);
    g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

// ------------------------------------------------------------ transpose
// Column indices outside [0, ncols) are skipped here and in the fill below,
// so a bad index never writes outside the counts/cursor array (ncols + 1).
__global__ void __launch_bounds__(256) k_col_counts(const int *ci, long long nnz, int ncols, int *counts) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nnz; t += (long long)gridDim.x * blockDim.x) {
        const int c = ci[t];
        if ((unsigned)c < (unsigned)ncols) atomicAdd(&counts[c], 1);
    }
}

cudaError_t launch_col_counts(const int *ci, long long nnz, int ncols, int *counts, cudaStream_t st, int nsm) {
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int) * ((size_t)ncols + 1), st);
    if (e != cudaSuccess || nnz == 0) return e;
    k_col_counts<<<grid_cap((nnz + 255) / 256, nsm, 8), 256, 0, st>>>(ci, nnz, ncols, counts); g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_tile_sums_int(const int *in, long long n, long long *sums, long long ntiles) {
    __shared__ long long sh[33];
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        long long s = 0;
        for (long long x = t * STILE + threadIdx.x; x < std::min(n, (t + 1) * STILE); x += blockDim.x) s += in[x];
        long long tot;
        block_excl_scan_ll(s, sh, &tot);
        if (threadIdx.x == 0) sums[t] = tot;
    }
}

__global__ void __launch_bounds__(256) k_scan_apply_int(const int *in, long long n, int *out, const long long *tile_offs,
                                                        long long ntiles, const long long *total) {
    __shared__ long long sh[33];
    constexpr int PER = STILE / 256;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long long x0 = t * STILE + (long long)threadIdx.x * PER;
        int v[PER];
        long long s = 0;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            v[u] = (x0 + u < n) ? in[x0 + u] : 0;
            s += v[u];
        }
        long long tot;
        long long ex = block_excl_scan_ll(s, sh, &tot) + tile_offs[t];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            if (x0 + u < n) out[x0 + u] = (int)ex;
            ex += v[u];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = (int)*total;
}

// out[0..n] = exclusive scan of in[0..n) followed by the total.
cudaError_t launch_excl_scan_int(const int *in, long long n, int *out, long long *tile_buf, cudaStream_t st, int nsm) {
    if (n == 0) return cudaMemsetAsync(out, 0, sizeof(int), st);
    const long long nt = (n + STILE - 1) / STILE;
    k_tile_sums_int<<<grid_cap(nt, nsm, 8), 256, 0, st>>>(in, n, tile_buf, nt); g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    k_scan_small_ll<<<1, 1024, 0, st>>>(tile_buf, nt, tile_buf + nt); g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    k_scan_apply_int<<<grid_cap(nt, nsm, 8), 256, 0, st>>>(in, n, out, tile_buf, nt, tile_buf + nt); g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

// Scatter of A's entries into the rows of A^T; cursor starts as a copy of
// the transpose's row pointers.  Rows of A^T come out in arbitrary order.
// With gate != NULL the kernel does nothing unless *gate is set.
template <int VB>
__global__ void __launch_bounds__(256) k_transpose_fill(const int *rp, const int *ci, const void *v, int nrows,
                                                        int ncols, int *cursor, int *tci, void *tv, const int *gate) {
    if (gate && *gate == 0) return;
    using V = typename std::conditional<VB == 4, unsigned, unsigned long long>::type;
    const int lane = threadIdx.x & 31;
    const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long i = gw; i < nrows; i += nw) {
        const int s = rp[i], e = rp[i + 1];
        for (int t = s + lane; t < e; t += 32) {
            const int c = ci[t];
            if ((unsigned)c >= (unsigned)ncols) continue;
            const int pos = atomicAdd(&cursor[c], 1);
            tci[pos] = (int)i;
            if (VB) static_cast<V *>(tv)[pos] = static_cast<const V *>(v)[t];
        }
    }
}

cudaError_t launch_transpose_fill(const int *rp, const int *ci, const void *v, int vbytes, int nrows, int ncols,
                                  int *cursor, int *tci, void *tv, const int *gate, cudaStream_t st, int nsm) {
    if (nrows == 0) return cudaSuccess;
    const int g = grid_cap(((long long)nrows + 7) / 8, nsm, 16);
    if (vbytes == 4) { k_transpose_fill<4><<<g, 256, 0, st>>>(rp, ci, v, nrows, ncols, cursor, tci, tv, gate); g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }
    else if (vbytes == 8) { k_transpose_fill<8><<<g, 256, 0, st>>>(rp, ci, v, nrows, ncols, cursor, tci, tv, gate); g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }
    else { k_transpose_fill<0><<<g, 256, 0, st>>>(rp, ci, nullptr, nrows, ncols, cursor, tci, nullptr, gate); g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }
    return cudaGetLastError();
}

// ------------------------------------------------------------ validation
// Row pointers non-decreasing from 0 to nnz, columns in [0, ncols) and
// strictly ascending within a row.  Failures set bits of *err.
__global__ void __launch_bounds__(256) k_validate(const int *rp, const int *ci, int nrows, int ncols, long long nnz,
                                                  unsigned *err) {
    const int lane = threadIdx.x & 31;
    const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    if (gw == 0 && lane == 0 && (rp[0] != 0 || rp[nrows] != nnz)) atomicOr(err, ERR_INVALID);
    for (long long i = gw; i < nrows; i += nw) {
        int s = rp[i], e = rp[i + 1];
        if (e < s || s < 0 || (long long)e > nnz) {
            if (lane == 0) atomicOr(err, ERR_INVALID);
            continue;   // never read entries through an invalid row pointer
        }
        bool bad = false, unsorted = false;
        for (int t = s + lane; t < e; t += 32) {
            const int c = ci[t];
            bad |= (c < 0 || c >= ncols);
            if (t > s) unsorted |= (ci[t - 1] >= c);
        }
        if (__any_sync(FULL, bad) && lane == 0) atomicOr(err, ERR_INVALID);
        if (__any_sync(FULL, unsorted) && lane == 0) atomicOr(err, ERR_UNSORTED);
    }
}

cudaError_t launch_validate(const int *rp, const int *ci, int nrows, int ncols, long long nnz, unsigned *err,
                            cudaStream_t st, int nsm) {
    k_validate<<<grid_cap(((long long)nrows + 7) / 8, nsm, 16), 256, 0, st>>>(rp, ci, nrows, ncols, nnz, err); g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

// ------------------------------------------------------------ value sum
template <int SR>
__global__ void __launch_bounds__(256) k_reduce_sum(const void *vals, const long long *d_nnz, void *out) {
    const long long n = *d_nnz;
    const int lane = threadIdx.x & 31;
    if (SR == MSGEMM_PLUS_TIMES_F32) {
        double s = 0.0;
        for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x)
            s += (double)static_cast<const float *>(vals)[x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
        if (lane == 0) atomicAdd(static_cast<double *>(out), s);
    } else {
        unsigned long long s = 0;
        for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x)
            s += static_cast<const unsigned long long *>(vals)[x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
        if (lane == 0) atomicAdd(static_cast<unsigned long long *>(out), s);
    }
}

cudaError_t launch_reduce_sum(int semiring, const void *vals, const long long *d_nnz, void *d_sum, cudaStream_t st,
                              int nsm) {
    cudaError_t e = cudaMemsetAsync(d_sum, 0, 8, st);
    if (e != cudaSuccess) return e;
    if (semiring == MSGEMM_PLUS_TIMES_F32) { k_reduce_sum<MSGEMM_PLUS_TIMES_F32><<<nsm * 4, 256, 0, st>>>(vals, d_nnz, d_sum); g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }
    else { k_reduce_sum<MSGEMM_PLUS_TIMES_I64><<<nsm * 4, 256, 0, st>>>(vals, d_nnz, d_sum); g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }
    return cudaGetLastError();
}

// ------------------------------------------------------------ heavy-row order
// Sorts a heavy kind's bucket by descending flops (single CTA bitonic sort,
// buckets of up to 4096 rows; larger buckets keep the binned order), so the
// dynamic row queue starts with the longest rows.
__global__ void __launch_bounds__(1024) k_sort_heavy(const __grid_constant__ RowArrays ra, int kind) {
    __shared__ long long key[4096];
    __shared__ int val[4096];
    const int n = ra.kind_count[kind];
    if (n <= 1 || n > 4096) return;
    const int off = ra.kind_off[kind];
    int N = 1;
    while (N < n) N <<= 1;
    for (int x = threadIdx.x; x < N; x += blockDim.x) {
        if (x < n) {
            val[x] = ra.perm[off + x];
            key[x] = -ra.flops[val[x]];
        } else {
            val[x] = -1;
            key[x] = LLONG_MAX;
        }
    }
    __syncthreads();
    for (int k = 2; k <= N; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int x = threadIdx.x; x < N / 2; x += blockDim.x) {
                const int lo = 2 * j * (x / j) + (x % j), hi = lo + j;
                const bool up = (lo & k) == 0;
                if ((key[lo] > key[hi]) == up) {
                    const long long tk = key[lo]; key[lo] = key[hi]; key[hi] = tk;
                    const int tv = val[lo]; val[lo] = val[hi]; val[hi] = tv;
                }
            }
            __syncthreads();
        }
    }
    for (int x = threadIdx.x; x < n; x += blockDim.x) ra.perm[off + x] = val[x];
}

cudaError_t launch_sort_heavy(const RowArrays &ra, int kind, cudaStream_t st) {
    k_sort_heavy<<<1, 1024, 0, st>>>(ra, kind); g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

}  // namespace msg

namespace msg {

// ------------------------------------------------------------ segmented sort
// Sorts every row of a CSR matrix by column, carrying VB-byte values, in
// place.  Bitonic network written with ascending comparators only (the first
// step of each merge compares i with i ^ (k - 1)), so positions past the row
// end act as +infinity without storage.  Rows up to 256 entries: one warp in
// shared memory; the warp pass lists longer rows, which 1024-thread CTAs
// then take from the list: up to SEG_SMEM entries in shared memory, longer
// ones on global memory.
constexpr int SEG_WARP = 256;
constexpr int SEG_SMEM = 16384;
constexpr int SEG_CTA = 1024;

template <int VB> struct ValT { using T = unsigned char; };
template <> struct ValT<4> { using T = unsigned; };
template <> struct ValT<8> { using T = unsigned long long; };

template <int VB, class KeyAt, class Swap>
__device__ __forceinline__ void bitonic_asc(int len, int tid, int nthreads, KeyAt key, Swap swp, bool cta) {
    int N = 1;
    while (N < len) N <<= 1;
    for (int k = 2; k <= N; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int x = tid; x < N / 2; x += nthreads) {
                const int i = 2 * j * (x / j) + (x % j);          // lower element of the pair
                const int p = (j == (k >> 1)) ? (i ^ (k - 1)) : (i + j);
                if (p < len && key(p) < key(i)) swp(i, p);
            }
            if (cta) __syncthreads(); else __syncwarp();
        }
    }
}

template <int VB>
__global__ void __launch_bounds__(256) k_segsort_warp(const int *rp, int *ci, void *v, int nrows, int *list) {
    using V = typename ValT<VB>::T;
    __shared__ int sk[8][SEG_WARP];
    __shared__ V sv[8][VB ? SEG_WARP : 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long gw = (long long)blockIdx.x * 8 + w, nw = (long long)gridDim.x * 8;
    for (long long i = gw; i < nrows; i += nw) {
        const int s = rp[i], len = rp[i + 1] - s;
        if (len > SEG_WARP && lane == 0) list[1 + atomicAdd(list, 1)] = (int)i;   // for k_segsort_cta
        if (len < 2 || len > SEG_WARP) continue;
        for (int x = lane; x < len; x += 32) {
            sk[w][x] = ci[s + x];
            if (VB) sv[w][x] = static_cast<const V *>(v)[s + x];
        }
        __syncwarp();
        bitonic_asc<VB>(len, lane, 32, [&](int a) { return sk[w][a]; },
                        [&](int a, int b) {
                            const int t = sk[w][a]; sk[w][a] = sk[w][b]; sk[w][b] = t;
                            if (VB) { const V u = sv[w][a]; sv[w][a] = sv[w][b]; sv[w][b] = u; }
                        }, false);
        for (int x = lane; x < len; x += 32) {
            ci[s + x] = sk[w][x];
            if (VB) static_cast<V *>(v)[s + x] = sv[w][x];
        }
        __syncwarp();
    }
}

template <int VB>
__global__ void __launch_bounds__(SEG_CTA) k_segsort_cta(const int *rp, int *ci, void *v, const int *list) {
    using V = typename ValT<VB>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    int *sk = reinterpret_cast<int *>(smem);
    V *sv = reinterpret_cast<V *>(smem + 4 * SEG_SMEM);
    const int nlist = list[0];
    for (int x0 = blockIdx.x; x0 < nlist; x0 += gridDim.x) {
        const long long i = list[1 + x0];
        const int s = rp[i], len = rp[i + 1] - s;
        if (len <= SEG_SMEM) {
            for (int x = threadIdx.x; x < len; x += blockDim.x) {
                sk[x] = ci[s + x];
                if (VB) sv[x] = static_cast<const V *>(v)[s + x];
            }
            __syncthreads();
            bitonic_asc<VB>(len, threadIdx.x, blockDim.x, [&](int a) { return sk[a]; },
                            [&](int a, int b) {
                                const int t = sk[a]; sk[a] = sk[b]; sk[b] = t;
                                if (VB) { const V u = sv[a]; sv[a] = sv[b]; sv[b] = u; }
                            }, true);
            for (int x = threadIdx.x; x < len; x += blockDim.x) {
                ci[s + x] = sk[x];
                if (VB) static_cast<V *>(v)[s + x] = sv[x];
            }
        } else {
            int *gk = ci + s;
            V *gv = VB ? static_cast<V *>(v) + s : nullptr;
            bitonic_asc<VB>(len, threadIdx.x, blockDim.x, [&](int a) { return gk[a]; },
                            [&](int a, int b) {
                                const int t = gk[a]; gk[a] = gk[b]; gk[b] = t;
                                if (VB) { const V u = gv[a]; gv[a] = gv[b]; gv[b] = u; }
                            }, true);
        }
        __syncthreads();
    }
}

template <int VB>
static cudaError_t segsort_t(const int *rp, int *ci, void *v, int nrows, int *list, cudaStream_t st, int nsm) {
    const size_t smem = 4 * SEG_SMEM + (VB ? (size_t)VB * SEG_SMEM : 0);
    // The shared-memory limit is a per-device attribute of the kernel: raised
    // once per device (bit d of the mask; racing threads may both set it,
    // which is harmless).
    static std::atomic<unsigned long long> attr_set{0};
    int dev = 0;
    cudaError_t ed = cudaGetDevice(&dev);
    if (ed != cudaSuccess) return ed;
    const unsigned long long bit = dev < 64 ? 1ULL << dev : 0ULL;
    if (!bit || !(attr_set.load(std::memory_order_acquire) & bit)) {
        cudaError_t e = cudaFuncSetAttribute(k_segsort_cta<VB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set.fetch_or(bit, std::memory_order_acq_rel);
    }
    cudaError_t e = cudaMemsetAsync(list, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    k_segsort_warp<VB><<<grid_cap(((long long)nrows + 7) / 8, nsm, 8), 256, 0, st>>>(rp, ci, v, nrows, list); g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    k_segsort_cta<VB><<<nsm, SEG_CTA, smem, st>>>(rp, ci, v, list); g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t launch_segsort(const int *rp, int *ci, void *v, int vbytes, int nrows, int *scratch, cudaStream_t st,
                           int nsm) {
    if (nrows == 0) return cudaSuccess;
    if (vbytes == 4) return segsort_t<4>(rp, ci, v, nrows, scratch, st, nsm);
    if (vbytes == 8) return segsort_t<8>(rp, ci, v, nrows, scratch, st, nsm);
    return segsort_t<0>(rp, ci, nullptr, nrows, scratch, st, nsm);
}

}  // namespace msg

namespace msg {

// ------------------------------------------------------------ multi-product transpose
// B^T for the pull kernel, for every product of a call at once: column
// counts of all B's go to one concatenated array (product q owns slots
// [co, co + ncols]), one exclusive scan turns it into row pointers that index
// a shared entry array, and one fill kernel scatters the entries.
__device__ __forceinline__ int bt_of(const BtDesc *d, int Q, long long x, bool by_rows) {
    int lo = 0, hi = Q - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((by_rows ? d[mid].ro : d[mid].eo) <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_col_counts_multi(const BtDesc *d, int Q, long long total, int *counts) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int q = bt_of(d, Q, e, false);
        atomicAdd(&counts[d[q].co + d[q].ci[e - d[q].eo]], 1);
    }
}

template <int VB>
__global__ void __launch_bounds__(256) k_transpose_fill_multi(const BtDesc *d, int Q, long long rows, int *cursor,
                                                              int *tci, void *tv, const int *gate) {
    if (gate && *gate == 0) return;
    using V = typename std::conditional<VB == 4, unsigned, unsigned long long>::type;
    const int lane = threadIdx.x & 31, grp = lane >> 3, gl = lane & 7;
    const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    // four rows per warp at a time: a row of at most eight entries is
    // scattered by its group of eight lanes, one entry per lane, so the four
    // rows' cursor atomics are in flight together; longer rows then take the
    // whole warp
    for (long long r0 = 4 * gw; r0 < rows; r0 += 4 * nw) {
        const long long r = r0 + grp;
        int q = 0, i = 0, s = 0, e = 0;
        if (r < rows) {
            q = bt_of(d, Q, r, true);
            i = (int)(r - d[q].ro);
            s = d[q].rp[i];
            e = d[q].rp[i + 1];
        }
        const bool lng = e - s > 8;
        if (!lng && s + gl < e) {
            const BtDesc &b = d[q];
            const int t = s + gl;
            const int pos = atomicAdd(&cursor[b.co + b.ci[t]], 1);
            tci[pos] = i;
            if (VB && b.v) static_cast<V *>(tv)[pos] = static_cast<const V *>(b.v)[t];   // none for a pattern B
        }
        unsigned todo = __ballot_sync(FULL, lng && gl == 0);
        while (todo) {
            const int u = __ffs(todo) - 1;
            todo &= todo - 1;
            const int qu = __shfl_sync(FULL, q, u), iu = __shfl_sync(FULL, i, u);
            const int su = __shfl_sync(FULL, s, u), eu = __shfl_sync(FULL, e, u);
            const BtDesc &b = d[qu];
            for (int t = su + lane; t < eu; t += 32) {
                const int pos = atomicAdd(&cursor[b.co + b.ci[t]], 1);
                tci[pos] = iu;
                if (VB && b.v) static_cast<V *>(tv)[pos] = static_cast<const V *>(b.v)[t];
            }
        }
    }
}

cudaError_t launch_bt_counts_multi(const BtDesc *d, int Q, long long total_nnz, int *counts, long long ncounts,
                                   cudaStream_t st, int nsm) {
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)ncounts, st);
    if (e != cudaSuccess || total_nnz == 0) return e;
    k_col_counts_multi<<<grid_cap((total_nnz + 255) / 256, nsm, 8), 256, 0, st>>>(d, Q, total_nnz, counts); g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t launch_bt_fill_multi(const BtDesc *d, int Q, long long total_rows, int vbytes, int *cursor, int *tci,
                                 void *tv, const int *gate, cudaStream_t st, int nsm) {
    if (total_rows == 0) return cudaSuccess;
    const int g = grid_cap((total_rows + 31) / 32, nsm, 16);
    if (vbytes == 4) { k_transpose_fill_multi<4><<<g, 256, 0, st>>>(d, Q, total_rows, cursor, tci, tv, gate); g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }
    else if (vbytes == 8) { k_transpose_fill_multi<8><<<g, 256, 0, st>>>(d, Q, total_rows, cursor, tci, tv, gate); g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }
    else { k_transpose_fill_multi<0><<<g, 256, 0, st>>>(d, Q, total_rows, cursor, tci, nullptr, gate); g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }
    return cudaGetLastError();
}

}  // namespace msg

namespace msg {

// ------------------------------------------------------------ tile index
// For every row k of B and column tile t (width T), the part of row k inside
// tile t as a pair of positions, (first position whose column is >= t * T,
// the same for t + 1; the row end if none), at tpos[t * nrows + k] (int2):
// one aligned 8-byte load gives both bounds.  Tile-major planes: kernels that
// sweep one tile for many rows read one plane.  One thread per row, the warp's 32 rows consecutive, planes
// in order: each lane advances a cursor through its (sorted) row -- linearly
// for short rows, by binary search from the cursor for long ones -- and the
// warp writes 32 consecutive slots of a plane at a time.
__global__ void __launch_bounds__(256) k_tile_bounds(const int *rp, const int *ci, int nrows, int T, int nt,
                                                     int *tpos, const int *gate) {
    // gate = per-kind row counts
    if (gate && gate[K_MSA_T] == 0 && gate[K_CMSA_T] == 0 && gate[K_CMSA_G] == 0 && gate[K_MSA_G] == 0) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k0 = (long long)blockIdx.x * blockDim.x; k0 < nrows; k0 += stride) {
        const long long k = k0 + threadIdx.x;
        const bool valid = k < nrows;
        int pos = valid ? rp[k] : 0;
        const int e = valid ? rp[k + 1] : 0;
        const bool longrow = e - pos > 64;
        int prev = pos;
        for (int t = 0; t <= nt; ++t) {
            if (valid) {
                if (t == nt) {
                    pos = e;
                } else {
                    const long long lo_col = (long long)t * T;
                    if (!longrow) {
                        while (pos < e && ci[pos] < lo_col) ++pos;
                    } else {
                        int lo = pos, hi = e;
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if (ci[mid] < lo_col) lo = mid + 1; else hi = mid;
                        }
                        pos = lo;
                    }
                }
                if (t > 0) reinterpret_cast<int2 *>(tpos)[(long long)(t - 1) * nrows + k] = make_int2(prev, pos);
                prev = pos;
            }
        }
    }
}

cudaError_t launch_tile_bounds(const int *rp, const int *ci, int nrows, int T, int nt, int *tpos, const int *gate,
                               cudaStream_t st, int nsm) {
    if (nrows == 0) return cudaSuccess;
    k_tile_bounds<<<grid_cap(((long long)nrows + 255) / 256, nsm, 16), 256, 0, st>>>(rp, ci, nrows, T, nt, tpos, gate); g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

}  // namespace msg
