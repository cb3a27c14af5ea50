// Row binning (the per-row choice of accumulator).
//
// The paper notes that unmasked flops and the per-row nonzeros of the mask
// and inputs are the natural proxies for choosing an algorithm per row, with
// a scan of the inputs to estimate flops (Sec. 6, remark on a hybrid), and
// its density study (Sec. 8.1) ranks the algorithms: pull (inner products)
// when the mask is much sparser than the inputs, MSA for small dimensions,
// hash for larger ones.  This pass computes, for every row i,
//   flops_i = sum over stored A_ik of nnz(B_k*)      (push work)
//   pull_i  = sum over mask entries j of nnz(B_*j)    (pull work)
// and picks a kind from the policy's preference list for the row's class,
// the first whose shared-memory form fits.
#pragma once

#include "common.cuh"

namespace msg {

template <int SR>
__device__ __forceinline__ int pick_family(const Policy &pol, int fam, bool warp, long long flops, int mnz, int anz, int n,
                           bool dot_ok, bool forced) {
    constexpr int acc = SrSizes<SR>::acc, in = SrSizes<SR>::in;
    constexpr bool sb = SrSizes<SR>::setbits;
    switch (fam) {
    case F_MSA:
        if (warp && pol.slab[K_MSA_W] > 0 && msa_bytes(n, acc) <= pol.slab[K_MSA_W]) return K_MSA_W;
        // the one-CTA form pays a CTA per row: unforced, only for CTA-sized
        // rows whose columns fit one shared-memory tile
        if (forced || (!warp && n <= pol.tileT[0])) return K_MSA_T;
        return -1;
    case F_HASH:
        if (warp && pol.slab[K_HASH_W] > 0 && hash_slots(mnz, acc, pol.slab[K_HASH_W])) return K_HASH_W;
        if (pol.slab[K_HASH_B] > 0 && hash_slots(mnz, acc, pol.slab[K_HASH_B])) return K_HASH_B;
        if (pol.slab[K_HASH_L] > 0 && hash_slots(mnz, acc, pol.slab[K_HASH_L])) return K_HASH_L;
        return -1;
    case F_MCA:
        if (warp && pol.slab[K_MCA_W] > 0 && mca_bytes(mnz, acc, sb) <= pol.slab[K_MCA_W]) return K_MCA_W;
        if (pol.slab[K_MCA_B] > 0 && mca_bytes(mnz, acc, sb) <= pol.slab[K_MCA_B]) return K_MCA_B;
        return -1;
    case F_HEAP:
    case F_HEAPDOT:
        // iterators live in registers: at most HEAP_MAX_ITERS stored entries in A_i*
        if ((warp || forced) && anz <= HEAP_MAX_ITERS) return fam == F_HEAP ? K_HEAP_W : K_HEAPDOT_W;
        return -1;
    case F_DOT:
        if (!dot_ok) return -1;
        if (warp && pol.slab[K_DOT_W] > 0 && dot_bytes(anz, mnz, in, acc, sb) <= pol.slab[K_DOT_W]) return K_DOT_W;
        if (pol.slab[K_DOT_B] > 0 && dot_bytes(anz, mnz, in, acc, sb) <= pol.slab[K_DOT_B]) return K_DOT_B;
        return -1;
    default:
        return -1;
    }
}

template <int SR>
__device__ __forceinline__ int choose_kind(const Policy &pol, long long flops, int mnz, int anz, int n, bool comp,
                           long long pull, bool dot_ok, bool index_ok) {
    constexpr int acc = SrSizes<SR>::acc;
    const bool warp = flops <= pol.warp_flops_max;
    if (comp) {
        const long long open = (long long)n - mnz;
        const long long bound = min(flops, open);
        if (flops == 0 || bound <= 0) return K_EMPTY;
        // heavy rows: the grid of (row, tile) items when the output is dense
        // (its room is then all open columns, at most 4x the bound)
        const int heavy = (pol.grid > 0 && index_ok && (n + pol.tileT[1] - 1) / pol.tileT[1] <= GRID_MAX_TILES &&
                           (pol.grid == 2 || pol.comp_grid_all || 4 * bound >= open)) ? K_CMSA_G : K_CMSA_T;
        if (pol.force == F_MSA) return heavy;
        if (pol.force == F_HEAP || pol.force == F_HEAPDOT)   // NInspect is 0 under a complement
            return anz <= HEAP_MAX_ITERS ? K_CHEAP_W : heavy;
        if (warp && pol.slab[K_CHASH_W] > 0 && chash_slots(bound, mnz, acc, pol.slab[K_CHASH_W])) return K_CHASH_W;
        if (pol.slab[K_CHASH_B] > 0 && chash_slots(bound, mnz, acc, pol.slab[K_CHASH_B])) return K_CHASH_B;
        return heavy;
    }
    if (flops == 0 || mnz == 0) return K_EMPTY;
    // the smallest rows: MCA on a team of eight (a family choice of MCA, or AUTO)
    if (pol.q_flops_max > 0 && mnz <= QMASK && flops <= pol.q_flops_max &&
        (pol.force == F_AUTO || pol.force == F_MCA))
        return K_MCA_Q;
    // heaviest rows of products wider than a tile: (row, tile) items over the GPU
    const bool grid_ok = pol.grid > 0 && !warp && index_ok && n > pol.tileT[0] &&
                         (n + pol.tileT[0] - 1) / pol.tileT[0] <= GRID_MAX_TILES;
    if (grid_ok && (pol.grid == 2 ? (pol.force == F_AUTO || pol.force == F_MSA) : flops >= pol.grid_min_flops))
        return K_MSA_G;
    // pull rows with tiny masks and little pull work: pull on a team of eight
    const bool dot_q = dot_ok && pol.q_flops_max > 0 && mnz <= QDMASK && pull <= pol.q_flops_max;
    if (pol.force != F_AUTO) {
        if (pol.force == F_DOT && dot_q) return K_DOT_Q;
        const int k = pick_family<SR>(pol, pol.force, warp, flops, mnz, anz, n, dot_ok, true);
        return k >= 0 ? k : K_MSA_T;
    }
    if (dot_ok && (double)pull * pol.dot_ratio < (double)flops) {
        if (dot_q) return K_DOT_Q;
        const int k = pick_family<SR>(pol, F_DOT, warp, flops, mnz, anz, n, dot_ok, false);
        if (k >= 0) return k;
    }
    const unsigned char *pref = pol.pref[row_class(flops, mnz)];
    for (int x = 0; x < 4 && pref[x] != F_AUTO; ++x) {
        const int k = pick_family<SR>(pol, pref[x], warp, flops, mnz, anz, n, dot_ok, false);
        if (k >= 0) return k;
    }
    return K_MSA_T;
}

// Kind, flops and temporary room of row r, and the per-CTA kind histogram.
template <int SR>
__device__ __forceinline__ void finish_row(const DevProd &P, const RowArrays &ra, const Policy &pol, long long *room,
                                           int *hist, int *hsub, long long r, int a0, int a1, int m0, int m1,
                                           bool dot_ok, long long f, long long pull) {
    const int mnz = m1 - m0;
    const bool index_ok = P.tpos != nullptr || P.n <= pol.tileT[1];
    int kind = choose_kind<SR>(pol, f, mnz, a1 - a0, P.n, P.complement != 0, pull, dot_ok, index_ok);
    if (kind == K_MSA_G && atomicAdd(ra.gplain, 1) >= pol.grid_cap) kind = K_MSA_T;   // piece tables are full
    ra.flops[r] = f;
    ra.kind[r] = (unsigned char)kind;
    ra.cnt[r] = 0;
    if (!P.complement) {
        ra.tmpoff[r] = P.tmp0 + m0;
        room[r] = 0;
    } else {
        room[r] = (kind == K_EMPTY) ? 0 : kind == K_CMSA_G ? (long long)(P.n - mnz) : min(f, (long long)(P.n - mnz));
    }
    atomicAdd(&hist[kind], 1);
    atomicAdd(&hsub[kind * NCLS_FLOPS + flops_sub(f)], 1);
    if (kind == K_DOT_W || kind == K_DOT_B || kind == K_DOT_Q) *ra.any_dot = 1;
}

__device__ __forceinline__ void flush_hist(const RowArrays &ra, const int *hist, const int *hsub) {
    for (int x = threadIdx.x; x < NKIND; x += blockDim.x)
        if (hist[x]) atomicAdd(&ra.kind_count[x], hist[x]);
    for (int x = threadIdx.x; x < NKIND * NCLS_FLOPS; x += blockDim.x)
        if (hsub[x]) atomicAdd(&ra.sub_count[x], hsub[x]);
}

// Sum over idx[q0..q1) of the row length rp[c + 1] - rp[c], by the whole warp
// with four entries per lane in flight (the row-pointer loads depend on the
// column loads, and long rows are latency-bound).
__device__ __forceinline__ long long warp_len_sum(const int *idx, const int *rp, int q0, int q1) {
    const int lane = lane_id();
    long long acc = 0;
    for (int b = q0; b < q1; b += 128) {
        int c[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int q = b + x * 32 + lane;
            c[x] = q < q1 ? __ldg(idx + q) : -1;
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
            if (c[x] >= 0) acc += __ldg(rp + c[x] + 1) - __ldg(rp + c[x]);
    }
    return warp_sum_ll(acc);
}

// Pull work of a row is only compared with its push work f (pull is picked
// when pull * ratio < f), so its sum may stop once pull * ratio >= f: the
// partial sum then gives the same decision.  Chunks of 128 as above.
__device__ __forceinline__ long long warp_len_sum_until(const int *idx, const int *rp, int q0, int q1, double ratio,
                                                        long long f) {
    const int lane = lane_id();
    long long total = 0;
    for (int b = q0; b < q1; b += 128) {
        int c[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int q = b + x * 32 + lane;
            c[x] = q < q1 ? __ldg(idx + q) : -1;
        }
        long long acc = 0;
#pragma unroll
        for (int x = 0; x < 4; ++x)
            if (c[x] >= 0) acc += __ldg(rp + c[x] + 1) - __ldg(rp + c[x]);
        total += warp_sum_ll(acc);
        if ((double)total * ratio >= (double)f) break;   // warp-uniform
    }
    return total;
}

// Flops, pull work, kind and temporary room of every row.  A warp takes up
// to 32 consecutive rows, one per lane: a row whose A row has at most
// SHORT_ROW entries is summed by its own lane, and so is its pull work over
// up to SHORT_ROW mask entries (the partial sum usually decides against pull
// after a few); rows with longer A rows, or whose pull work is still open,
// are then summed by the whole warp one at a time; rows beyond LONG_ROW
// entries go to a list that k_bin_long sums with a whole CTA each.  Every
// lane then picks its row's kind.
constexpr int SHORT_ROW = 32;
constexpr int LONG_ROW = 1024;

// (At most 64 registers: four CTAs per SM.  With the compiler's own choice
// the per-row policy code spilled, and the pass ran 40% slower.)
template <int SR>
__global__ void __launch_bounds__(256, 4) k_bin_score(const __grid_constant__ ProdSet ps, const __grid_constant__ RowArrays ra,
                                                   const __grid_constant__ Policy pol, long long *room) {
    __shared__ int hist[NKIND];
    __shared__ int hsub[NKIND * NCLS_FLOPS];
    for (int x = threadIdx.x; x < NKIND; x += blockDim.x) hist[x] = 0;
    for (int x = threadIdx.x; x < NKIND * NCLS_FLOPS; x += blockDim.x) hsub[x] = 0;
    block_sync();
    const int lane = lane_id();
    const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    // rows per warp and pass: 32, or fewer when there are few rows, so that
    // few long rows still spread over many warps
    const int W = (int)min(32LL, max(1LL, (ra.R + nw - 1) / nw));
    for (long long r0 = gw * W; r0 < ra.R; r0 += nw * W) {
        const long long r = r0 + lane;
        const bool valid = lane < W && r < ra.R;
        // the warp's rows are consecutive: when its first and last rows share
        // a product, so do all (two searches instead of one per lane); the
        // row kernels read the recorded product instead of searching again
        int p = 0;
        if (ps.P > 1) {
            const long long rl = min(r0 + W, ra.R) - 1;
            int pe = 0;
            if (lane < 2) pe = prod_of_row(ps, lane ? rl : r0);
            const int pf = __shfl_sync(FULL, pe, 0), pl = __shfl_sync(FULL, pe, 1);
            p = pf == pl ? pf : (valid ? prod_of_row(ps, r) : 0);
            if (valid && ra.prod) ra.prod[r] = p;
        }
        const DevProd &P = prod_at(ps, p);
        int a0 = 0, a1 = 0, m0 = 0, m1 = 0;
        if (valid) {
            const int i = (int)(r - P.row0);
            a0 = __ldg(P.a_rp + i); a1 = __ldg(P.a_rp + i + 1);
            m0 = __ldg(P.m_rp + i); m1 = __ldg(P.m_rp + i + 1);
        }
        const bool dot_ok = valid && !P.complement && P.bt_rp != nullptr && P.a_sorted && pol.allow_dot;
        const bool a_short = a1 - a0 <= SHORT_ROW;
        const bool is_huge = a1 - a0 > LONG_ROW || (dot_ok && m1 - m0 > LONG_ROW);
        long long f = 0, pull = 0;
        bool pull_open = false;   // pull work not yet decided by the lane's own partial sum
        if (valid && a_short && !is_huge) {
            for (int t = a0; t < a1; ++t) {
                const int k = __ldg(P.a_ci + t);
                f += __ldg(P.b_rp + k + 1) - __ldg(P.b_rp + k);
            }
            if (dot_ok) {
                // the lane sums up to SHORT_ROW mask entries and stops once the
                // partial sum rules pull out; rows still open go to the warp
                const int qe = min(m1, m0 + SHORT_ROW);
                bool decided = false;
                for (int q = m0; q < qe; ++q) {
                    const int j = __ldg(P.m_ci + q);
                    pull += __ldg(P.bt_rp + j + 1) - __ldg(P.bt_rp + j);
                    if ((double)pull * pol.dot_ratio >= (double)f) { decided = true; break; }   // no pull
                }
                pull_open = !decided && m1 - m0 > SHORT_ROW;
            }
        }
        if (valid && is_huge) ra.perm[atomicAdd(ra.nlong, 1)] = (int)r;   // to k_bin_long
        unsigned longs = __ballot_sync(FULL, valid && !is_huge && (!a_short || pull_open));
        while (longs) {
            const int u = __ffs(longs) - 1;
            longs &= longs - 1;
            const DevProd &Q = prod_at(ps, __shfl_sync(FULL, p, u));
            const int ua0 = __shfl_sync(FULL, a0, u), ua1 = __shfl_sync(FULL, a1, u);
            const int um0 = __shfl_sync(FULL, m0, u), um1 = __shfl_sync(FULL, m1, u);
            const bool udot = __shfl_sync(FULL, dot_ok, u);
            const bool ushort = __shfl_sync(FULL, a_short, u);
            const long long fl = __shfl_sync(FULL, f, u);
            const long long fu = ushort ? fl : warp_len_sum(Q.a_ci, Q.b_rp, ua0, ua1);
            const long long pu = udot ? warp_len_sum_until(Q.m_ci, Q.bt_rp, um0, um1, pol.dot_ratio, fu) : 0;
            if (lane == u) {
                f = fu;
                pull = pu;
            }
        }
        if (valid && !is_huge) finish_row<SR>(P, ra, pol, room, hist, hsub, r, a0, a1, m0, m1, dot_ok, f, pull);
    }
    block_sync();
    flush_hist(ra, hist, hsub);
}

// The listed rows (more than LONG_ROW entries), one CTA per row: each warp
// sums a share of the row, the CTA adds the shares.  The list lives in
// ra.perm, which k_bin_scatter fills only afterwards.
template <int SR>
__global__ void __launch_bounds__(256) k_bin_long(const __grid_constant__ ProdSet ps, const __grid_constant__ RowArrays ra,
                                                  const __grid_constant__ Policy pol, long long *room) {
    __shared__ int hist[NKIND];
    __shared__ int hsub[NKIND * NCLS_FLOPS];
    __shared__ long long part[2][8];
    __shared__ long long s_f;
    for (int x = threadIdx.x; x < NKIND; x += blockDim.x) hist[x] = 0;
    for (int x = threadIdx.x; x < NKIND * NCLS_FLOPS; x += blockDim.x) hsub[x] = 0;
    block_sync();
    const int nlong = *ra.nlong;
    const int w = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int x = blockIdx.x; x < nlong; x += gridDim.x) {
        const long long r = ra.perm[x];
        const DevProd &P = prod_at(ps, row_prod(ps, ra.prod, r));
        const int i = (int)(r - P.row0);
        const int a0 = __ldg(P.a_rp + i), a1 = __ldg(P.a_rp + i + 1);
        const int m0 = __ldg(P.m_rp + i), m1 = __ldg(P.m_rp + i + 1);
        const bool dot_ok = !P.complement && P.bt_rp != nullptr && P.a_sorted && pol.allow_dot;
        auto share = [&](int q0, int q1, int &s0, int &s1) {   // warp w's contiguous share
            const long long len = q1 - q0, per = (len + nwarp - 1) / nwarp;
            s0 = (int)min((long long)q1, q0 + per * w);
            s1 = (int)min((long long)q1, (long long)s0 + per);
        };
        int s0, s1;
        share(a0, a1, s0, s1);
        const long long f = warp_len_sum(P.a_ci, P.b_rp, s0, s1);
        if (lane_id() == 0) part[0][w] = f;
        block_sync();
        if (threadIdx.x == 0) {
            long long ft = 0;
            for (int q = 0; q < nwarp; ++q) ft += part[0][q];
            s_f = ft;
        }
        block_sync();
        const long long ft = s_f;
        long long pull = 0;
        if (dot_ok) {   // a warp whose share alone decides against pull stops early
            share(m0, m1, s0, s1);
            pull = warp_len_sum_until(P.m_ci, P.bt_rp, s0, s1, pol.dot_ratio, ft);
        }
        if (lane_id() == 0) part[1][w] = pull;
        block_sync();
        if (threadIdx.x == 0) {
            long long pt = 0;
            for (int q = 0; q < nwarp; ++q) pt += part[1][q];
            finish_row<SR>(P, ra, pol, room, hist, hsub, r, a0, a1, m0, m1, dot_ok, ft, pt);
        }
        block_sync();
    }
    block_sync();
    flush_hist(ra, hist, hsub);
}

}  // namespace msg
