// Elementwise kernels of the graph applications built on the library's masked
// products (capi.cu): batched betweenness centrality (msgemm_bc) -- the first
// frontier, the visited pattern of every level (a row-major bitmap turned
// into CSR for the complemented mask), the backward weights and the
// dependency sums -- and k-truss (msgemm_ktruss) -- the entry filter that
// drops self loops and edges below the support threshold.
#include "launch.h"

namespace msg {
namespace {

__global__ void __launch_bounds__(256) k_bc_sources(const int *src, int nsrc, int *rp, int *ci, long long *v) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= nsrc; i += gridDim.x * blockDim.x) {
        rp[i] = i;
        if (i < nsrc) {
            ci[i] = src[i];
            v[i] = 1;
        }
    }
}

// Bits of a CSR pattern into a row-major bitmap of wpr words per row; one
// warp per row.
__global__ void __launch_bounds__(256) k_bitmap_or(const int *rp, const int *ci, int nrows, long long wpr, unsigned *bm) {
    const int lane = threadIdx.x & 31;
    const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long i = gw; i < nrows; i += nw)
        for (int t = rp[i] + lane; t < rp[i + 1]; t += 32) {
            const int j = ci[t];
            atomicOr(&bm[i * wpr + (j >> 5)], 1u << (j & 31));
        }
}

// Set bits per bitmap row; one warp per row.
__global__ void __launch_bounds__(256) k_bitmap_counts(const unsigned *bm, int nrows, long long wpr, int *cnt) {
    const int lane = threadIdx.x & 31;
    const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long i = gw; i < nrows; i += nw) {
        int c = 0;
        for (long long w = lane; w < wpr; w += 32) c += __popc(bm[i * wpr + w]);
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
        if (lane == 0) cnt[i] = c;
    }
}

// Bitmap rows to ascending CSR columns at the scanned row pointers; one warp
// per row, 32 words per pass.
__global__ void __launch_bounds__(256) k_bitmap_cols(const unsigned *bm, int nrows, long long wpr, const int *rp, int *ci) {
    const int lane = threadIdx.x & 31;
    const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long i = gw; i < nrows; i += nw) {
        int base = rp[i];
        for (long long w0 = 0; w0 < wpr; w0 += 32) {
            const long long w = w0 + lane;
            unsigned bits = w < wpr ? bm[i * wpr + w] : 0u;
            const int c = __popc(bits);
            int incl = c;
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += t;
            }
            int o = base + incl - c;
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                ci[o++] = (int)(w * 32 + b);
            }
            base += __shfl_sync(FULL, incl, 31);
        }
    }
}

// Backward weight of a level's entries: (1 + delta) / sigma = 1 / sigma + T
// (T = 0 on the deepest level).
__global__ void __launch_bounds__(256) k_bc_weight(const long long *sigma, const float *T, long long nnz, float *W) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (long long)gridDim.x * blockDim.x)
        W[e] = (float)(1.0 / (double)sigma[e]) + (T ? T[e] : 0.0f);
}

// delta = sigma * T for a level's entries, summed into the column's vertex.
__global__ void __launch_bounds__(256) k_bc_accum(const int *ci, const long long *sigma, const float *T, long long nnz,
                                                  double *bc) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (long long)gridDim.x * blockDim.x) {
        const float t = T[e];
        if (t != 0.0f) atomicAdd(&bc[ci[e]], (double)sigma[e] * (double)t);
    }
}

// k-truss filter: entry e of row i is kept iff ci[e] != i and (no support
// array, or support[e] >= thr).  Counts per row, then the kept entries
// (and their supports) in order at the scanned row pointers; a warp per row.
__global__ void __launch_bounds__(256) k_filter_counts(const int *rp, const int *ci, int nrows, const long long *sup,
                                                       long long thr, int *cnt) {
    const int lane = threadIdx.x & 31;
    const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long i = gw; i < nrows; i += nw) {
        int c = 0;
        for (int t = rp[i] + lane; t < rp[i + 1]; t += 32) c += (ci[t] != i && (!sup || sup[t] >= thr)) ? 1 : 0;
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
        if (lane == 0) cnt[i] = c;
    }
}

__global__ void __launch_bounds__(256) k_filter_write(const int *rp, const int *ci, int nrows, const long long *sup,
                                                      long long thr, const int *nrp, int *nci, long long *nsup) {
    const int lane = threadIdx.x & 31;
    const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long i = gw; i < nrows; i += nw) {
        int base = nrp[i];
        for (int t0 = rp[i]; t0 < rp[i + 1]; t0 += 32) {
            const int t = t0 + lane;
            const bool k = t < rp[i + 1] && ci[t] != i && (!sup || sup[t] >= thr);
            const unsigned bal = __ballot_sync(FULL, k);
            if (k) {
                const int o = base + __popc(bal & ((1u << lane) - 1u));
                nci[o] = ci[t];
                if (nsup) nsup[o] = sup ? sup[t] : 0;
            }
            base += __popc(bal);
        }
    }
}

// p[e] = e: the position of every entry, carried through a transpose as its
// value so that the transpose's entries can later be filled by a gather.
__global__ void __launch_bounds__(256) k_iota(int *p, long long n) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        p[e] = (int)e;
}

// dst[e] = src[perm[e]] (coalesced writes, reads through L2).
__global__ void __launch_bounds__(256) k_gather_f32(const int *__restrict__ perm, const float *__restrict__ src,
                                                    long long n, float *__restrict__ dst) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        dst[e] = __ldg(src + __ldg(perm + e));
}

int blocks_for(long long work, int nsm, int per_sm) {
    const long long b = (work + 255) / 256;
    return (int)std::max(1LL, std::min(b, (long long)nsm * per_sm));
}

}  // namespace

cudaError_t launch_bc_sources(const int *src, int nsrc, int *rp, int *ci, long long *v, cudaStream_t st, int nsm) {
    k_bc_sources<<<blocks_for(nsrc + 1, nsm, 4), 256, 0, st>>>(src, nsrc, rp, ci, v);
    return counted(cudaGetLastError());
}
cudaError_t launch_bitmap_or(const int *rp, const int *ci, int nrows, long long wpr, unsigned *bm, cudaStream_t st,
                             int nsm) {
    if (nrows == 0) return cudaSuccess;
    k_bitmap_or<<<blocks_for((long long)nrows * 32, nsm, 16), 256, 0, st>>>(rp, ci, nrows, wpr, bm);
    return counted(cudaGetLastError());
}
cudaError_t launch_bitmap_counts(const unsigned *bm, int nrows, long long wpr, int *cnt, cudaStream_t st, int nsm) {
    if (nrows == 0) return cudaSuccess;
    k_bitmap_counts<<<blocks_for((long long)nrows * 32, nsm, 16), 256, 0, st>>>(bm, nrows, wpr, cnt);
    return counted(cudaGetLastError());
}
cudaError_t launch_bitmap_cols(const unsigned *bm, int nrows, long long wpr, const int *rp, int *ci, cudaStream_t st,
                               int nsm) {
    if (nrows == 0) return cudaSuccess;
    k_bitmap_cols<<<blocks_for((long long)nrows * 32, nsm, 16), 256, 0, st>>>(bm, nrows, wpr, rp, ci);
    return counted(cudaGetLastError());
}
cudaError_t launch_bc_weight(const long long *sigma, const float *T, long long nnz, float *W, cudaStream_t st, int nsm) {
    if (nnz == 0) return cudaSuccess;
    k_bc_weight<<<blocks_for(nnz, nsm, 16), 256, 0, st>>>(sigma, T, nnz, W);
    return counted(cudaGetLastError());
}
cudaError_t launch_bc_accum(const int *ci, const long long *sigma, const float *T, long long nnz, double *bc,
                            cudaStream_t st, int nsm) {
    if (nnz == 0) return cudaSuccess;
    k_bc_accum<<<blocks_for(nnz, nsm, 16), 256, 0, st>>>(ci, sigma, T, nnz, bc);
    return counted(cudaGetLastError());
}
cudaError_t launch_filter_counts(const int *rp, const int *ci, int nrows, const long long *sup, long long thr, int *cnt,
                                 cudaStream_t st, int nsm) {
    if (nrows == 0) return cudaSuccess;
    k_filter_counts<<<blocks_for((long long)nrows * 32, nsm, 16), 256, 0, st>>>(rp, ci, nrows, sup, thr, cnt);
    return counted(cudaGetLastError());
}
cudaError_t launch_filter_write(const int *rp, const int *ci, int nrows, const long long *sup, long long thr,
                                const int *nrp, int *nci, long long *nsup, cudaStream_t st, int nsm) {
    if (nrows == 0) return cudaSuccess;
    k_filter_write<<<blocks_for((long long)nrows * 32, nsm, 16), 256, 0, st>>>(rp, ci, nrows, sup, thr, nrp, nci, nsup);
    return counted(cudaGetLastError());
}
cudaError_t launch_iota_i32(int *p, long long n, cudaStream_t st, int nsm) {
    if (n == 0) return cudaSuccess;
    k_iota<<<blocks_for(n, nsm, 16), 256, 0, st>>>(p, n);
    return counted(cudaGetLastError());
}
cudaError_t launch_gather_f32(const int *perm, const float *src, long long n, float *dst, cudaStream_t st, int nsm) {
    if (n == 0) return cudaSuccess;
    k_gather_f32<<<blocks_for(n, nsm, 16), 256, 0, st>>>(perm, src, n, dst);
    return counted(cudaGetLastError());
}

}  // namespace msg
