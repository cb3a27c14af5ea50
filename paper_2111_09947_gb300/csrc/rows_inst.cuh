// Instantiation of the row kernels and the binning pass for one semiring.
// Included by exactly one translation unit per semiring with MSG_SR and
// MSG_SUFFIX defined, so the three semirings compile in parallel.
#pragma once

#include <mutex>

#include "bin.cuh"
#include "launch.h"
#include "rows.cuh"

namespace msg {
namespace {

using RowKernel = void (*)(ProdSet, RowLaunch);

// Grid of a persistent kernel: resident CTAs per SM x SMs.  The dynamic
// shared-memory limit (a per-device attribute of the kernel, raised for any
// size: static shared memory counts against the default 48 KB too) and the
// occupancy of the last size asked are cached per kernel and device.
template <RowKernel K>
cudaError_t go(const ProdSet &ps, const RowLaunch &L, int threads, size_t smem, cudaStream_t st, int nsm) {
    struct DevState {
        size_t attr = 0, occ_smem = ~size_t(0);
        int occ = 0;
    };
    static std::mutex mu;
    static DevState cache[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int occ = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        DevState spare;
        DevState &d = (dev >= 0 && dev < 64) ? cache[dev] : spare;
        if (smem > d.attr) {
            e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            d.attr = smem;
        }
        if (d.occ_smem != smem) {
            int nb = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, K, threads, smem);
            if (e != cudaSuccess) return e;
            d.occ = nb;
            d.occ_smem = smem;
        }
        occ = d.occ;
    }
    if (occ < 1) return cudaErrorInvalidConfiguration;
    K<<<occ * nsm, threads, smem, st>>>(ps, L); g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

}  // namespace

cudaError_t MSG_CAT(launch_bin_score_, MSG_SUFFIX)(const ProdSet &ps, const RowArrays &ra, const Policy &pol,
                                                   long long *room, cudaStream_t st, int nsm) {
    if (ra.R == 0) return cudaSuccess;
    // up to one warp per row; the kernel packs up to 32 rows per warp when rows outnumber warps
    const long long blocks = std::min<long long>((ra.R + 7) / 8, (long long)nsm * 16);
    k_bin_score<MSG_SR><<<(int)blocks, 256, 0, st>>>(ps, ra, pol, room); g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // rows longer than LONG_ROW entries, listed by the pass above
    k_bin_long<MSG_SR><<<nsm * 4, 256, 0, st>>>(ps, ra, pol, room); g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t MSG_CAT(launch_kind_, MSG_SUFFIX)(int kind, const ProdSet &ps, const RowLaunch &L, cudaStream_t st,
                                              int nsm) {
    const int th = kind_threads(kind);
    const size_t sm = kind_smem(kind, L.slab);
    switch (kind) {
    case K_MSA_W: return go<k_rows_w<MSG_SR, K_MSA_W>>(ps, L, th, sm, st, nsm);
    case K_HASH_W: return go<k_rows_w<MSG_SR, K_HASH_W>>(ps, L, th, sm, st, nsm);
    case K_MCA_W: return go<k_rows_w<MSG_SR, K_MCA_W>>(ps, L, th, sm, st, nsm);
    case K_DOT_W: return go<k_rows_w<MSG_SR, K_DOT_W>>(ps, L, th, sm, st, nsm);
    case K_CHASH_W: return go<k_rows_w<MSG_SR, K_CHASH_W>>(ps, L, th, sm, st, nsm);
    case K_HEAP_W: return go<k_rows_w<MSG_SR, K_HEAP_W>>(ps, L, th, sm, st, nsm);
    case K_HEAPDOT_W: return go<k_rows_w<MSG_SR, K_HEAPDOT_W>>(ps, L, th, sm, st, nsm);
    case K_CHEAP_W: return go<k_rows_w<MSG_SR, K_CHEAP_W>>(ps, L, th, sm, st, nsm);
    case K_MCA_Q: return go<k_rows_q<MSG_SR>>(ps, L, th, sm, st, nsm);
    case K_DOT_Q: return go<k_rows_dq<MSG_SR>>(ps, L, th, sm, st, nsm);
    case K_HASH_B: return go<k_rows_b<MSG_SR, K_HASH_B>>(ps, L, th, sm, st, nsm);
    case K_HASH_L: return go<k_rows_b<MSG_SR, K_HASH_L>>(ps, L, th, sm, st, nsm);
    case K_MCA_B: return go<k_rows_b<MSG_SR, K_MCA_B>>(ps, L, th, sm, st, nsm);
    case K_DOT_B: return go<k_rows_b<MSG_SR, K_DOT_B>>(ps, L, th, sm, st, nsm);
    case K_CHASH_B: return go<k_rows_b<MSG_SR, K_CHASH_B>>(ps, L, th, sm, st, nsm);
    case K_MSA_T: return go<k_rows_t<MSG_SR, false>>(ps, L, th, sm, st, nsm);
    case K_CMSA_T: return go<k_rows_t<MSG_SR, true>>(ps, L, th, sm, st, nsm);
    case K_CMSA_G: return go<k_rows_g<MSG_SR, true>>(ps, L, th, sm, st, nsm);
    case K_MSA_G: return go<k_rows_g<MSG_SR, false>>(ps, L, th, sm, st, nsm);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace msg
