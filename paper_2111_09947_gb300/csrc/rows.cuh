// Row accumulators of the masked SpGEMM (Sec. 4-5), one team per row.
//
// Every kernel here is persistent: it walks the rows the binning pass put in
// its kind's bucket, so the host never needs the bucket sizes.  Each row
// writes its kept entries, in ascending column order, to its slot range of
// the temporary output and its count to cnt[r]; compaction follows.
//
// Push kinds enumerate the products A_ik * B_kj of row i (Gustavson order,
// Sec. 4.2): the outer list is A_i*, the inner rows are B_k*.  The pull kind
// (DOT) enumerates pairs (mask entry j, entry k of column B_*j) and looks k up
// in the staged row A_i* (Sec. 4.1).
#pragma once

#include "common.cuh"

namespace msg {

constexpr unsigned long long EMPTY64 = ~0ULL;
constexpr unsigned EMPTY32 = 0xffffffffu;

// Launch parameters of one accumulator kernel.
struct GridTab {
    int *cnt, *off, *done;
    unsigned long long *next;
};

struct RowLaunch {
    RowArrays ra;
    TmpOut tmp;
    int slab;          // shared bytes per warp (_W) or per CTA (_B, _T)
    int tileT;         // column tile width of _T kinds
    int4 *cursors;     // _T kinds: one cursor per stored entry of A (global)
    int aligned;       // 1: write values only, at the mask entry's own slot (tmp + rank);
                       //    the output array is zeroed beforehand (gradient form)
    // grid kinds ([0] MSA_G, [1] CMSA_G): per (row of the kind, tile) entry
    // count and offset in the row, per-row completed items, item cursor;
    // tiles per row slot (the most of any product)
    GridTab g[2];
    int gnt;
    // int64 tiled kinds: high words, tileT per CTA (CTA b at tile_hi + b * tileT)
    unsigned *tile_hi;
    int tile_hi_slots;
    int *spec_off;     // grid kinds: raised by the first unsafe tile of a launch
    // two-phase form (Sec. 6): the symbolic launch counts each row's entries
    // and writes none (count_only); the numeric launch writes them straight
    // into the product's output arrays at the row's final offset (direct)
    int count_only;
    int direct;
    int hash_kicks;    // HASH kinds: moves allowed per cuckoo insertion; 0 = linear probing
};

// Where a row's entries go: the shared temporary output, or (two-phase
// numeric launch) the product's own output arrays.
__device__ __forceinline__ TmpOut out_of(const DevProd &P, const RowLaunch &L) {
    return L.direct ? TmpOut{P.c_ci, P.c_v} : L.tmp;
}

// This CTA's high-word array of the tiled kinds (null unless split int64);
// a grid larger than the workspace flags an error and gets null.
template <int SR>
__device__ __forceinline__ unsigned *tile_hi_of(const RowLaunch &L) {
    if constexpr (!TileAcc<SR>::split) {
        return nullptr;
    } else {
        if ((int)blockIdx.x >= L.tile_hi_slots || !L.tile_hi) return nullptr;
        return L.tile_hi + (size_t)blockIdx.x * L.tileT;
    }
}

template <int SR>
__device__ __forceinline__ typename Sr<SR>::in_t shfl_val(typename Sr<SR>::in_t v, int src) {
    if constexpr (Sr<SR>::vals) return __shfl_sync(FULL, v, src);
    else return v;
}

template <int SR>
__device__ __forceinline__ typename Sr<SR>::in_t shfl_val_mask(unsigned m, typename Sr<SR>::in_t v, int src) {
    if constexpr (Sr<SR>::vals) return __shfl_sync(m, v, src);
    else return v;
}
template <int SR>
__device__ __forceinline__ typename Sr<SR>::acc_t shfl_xor_acc(unsigned m, typename Sr<SR>::acc_t v, int o) {
    return __shfl_xor_sync(m, v, o);
}

__device__ __forceinline__ bool test_bit(const unsigned *w, int b) { return (w[b >> 5] >> (b & 31)) & 1u; }
__device__ __forceinline__ void set_bit_once(unsigned *w, int b) {
    unsigned m = 1u << (b & 31);
    if (!(w[b >> 5] & m)) atomicOr(&w[b >> 5], m);
}

// --------------------------------------------------------------- enumerators
// Inner range of outer entry t with inner row c: the whole row of the inner
// CSR (RowSeg) or the part of it inside one column tile (TileSeg, from the
// per-row tile index).
struct RowSeg {
    const int *irp;
    __device__ __forceinline__ void operator()(int c, int &s, int &e) const {
        s = __ldg(irp + c);
        e = __ldg(irp + c + 1);
    }
};
struct TileSeg {
    const int *tpos;   // row c, tile t: [x, y) of the int2 at tpos[t * stride + c]
    int stride, tile;
    __device__ __forceinline__ void operator()(int c, int &s, int &e) const {
        const int2 v = __ldg(reinterpret_cast<const int2 *>(tpos) + (long long)tile * stride + c);
        s = v.x;
        e = v.y;
    }
};

// Calls f(t, a_t, col, val) for every (outer position t in [o0, o1), inner
// entry q of the range seg gives for row oci[t]) pair, with col = ici[q],
// val = iv[q].  Outer entries are dealt to the team's warps round-robin
// (entry x goes to warp x mod nw), so every warp of a CTA-row gets work even
// for short outer lists; a warp's window holds its next 32 entries.  Within a
// window, ranges of LONG_SEG or more entries are walked one at a time by the
// whole warp (lanes stride the range, 4 loads in flight per lane); all
// shorter ranges are enumerated together: their products are numbered and
// each lane finds its range by a binary search over the window's prefix of
// lengths, so lanes stay busy whatever the mix of lengths.
#ifndef MSG_LONG_SEG
#define MSG_LONG_SEG 64
#endif
constexpr int LONG_SEG = MSG_LONG_SEG;
// Column of an empty product slot; below zero and, as a 32-bit key, neither
// a column (< 2^31) nor the empty-slot word 2^32 - 1.
constexpr int NO_PRODUCT = -2;

// The walk of one range [s, e) by the whole warp, chunks of 128 entries
// (4 loads per lane in flight), from chunk c0 in steps of cstep chunks.
// With WSYNC every lane calls f for every slot (column NO_PRODUCT: no
// product), so f may use warp-wide votes; otherwise only lanes holding a
// product call it.
template <int SR, bool WSYNC, bool PAT, class F>
__device__ __forceinline__ void walk_range_v(int t, typename Sr<SR>::in_t a, int s, int e, int c0, int cstep,
                                             const int *__restrict__ ici, const void *iv, F &f) {
    using in_t = typename Sr<SR>::in_t;
    const unsigned lane = (unsigned)lane_id(), ue = (unsigned)e;
    // unsigned 32-bit indices (e < 2^31, steps below 2^13: no wrap); the four
    // loads of a chunk share one address with immediate offsets
    for (unsigned q0 = (unsigned)s + 128u * (unsigned)c0 + lane; q0 - lane < ue; q0 += 128u * (unsigned)cstep) {
        const int *cp = ici + q0;
        int col[4];
        in_t bv[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            col[x] = NO_PRODUCT;
            bv[x] = in_t{};
            if (q0 + 32u * x < ue) {
                col[x] = __ldg(cp + 32 * x);
                if constexpr (Sr<SR>::vals)
                    bv[x] = PAT ? in_t(1) : __ldg(static_cast<const in_t *>(iv) + (q0 + 32u * x));
            }
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
            if (WSYNC || col[x] >= 0) f(t, a, col[x], bv[x]);
    }
}

// The walk, with the pattern test (no value array: every value 1) taken once
// per range instead of per entry.
template <int SR, bool WSYNC = false, class F>
__device__ __forceinline__ void walk_range(int t, typename Sr<SR>::in_t a, int s, int e, int c0, int cstep,
                                           const int *__restrict__ ici, const void *iv, F &f) {
    if (!Sr<SR>::vals || iv) walk_range_v<SR, WSYNC, false>(t, a, s, e, c0, cstep, ici, iv, f);
    else walk_range_v<SR, WSYNC, true>(t, a, s, e, c0, cstep, ici, iv, f);
}

// CTA teams: ranges of BIG_SEG or more entries (hub rows of B) are not walked
// by the warp that meets them but listed, and after the windows every warp
// takes chunks of every listed range, so one hub does not hold the team's
// next barrier; a full list falls back to the warp walk.
constexpr int BIG_SEG = 2048;
constexpr int BIG_LIST = 128;

template <int SR, bool CTA, bool OUTV, bool WSYNC = false, class Seg, class F>
__device__ __forceinline__ void enum_products(int o0, int o1, const int *__restrict__ oci, const void *ov,
                                              const Seg &seg, const int *__restrict__ ici, const void *iv, F &f) {
    using in_t = typename Sr<SR>::in_t;
    Team<CTA> team;
    const int lane = lane_id();
    const int nw = team.nwarps(), wq = team.warp();
    const int cnt = o1 - o0;
    __shared__ int s_nbig;
    __shared__ int s_big[CTA ? BIG_LIST : 1][3];
    __shared__ in_t s_biga[CTA ? BIG_LIST : 1];
    if constexpr (CTA) {
        if (threadIdx.x == 0) s_nbig = 0;
        block_sync();
    }
    for (int b0 = 0; wq + nw * b0 < cnt; b0 += 32) {
        const int t = o0 + wq + nw * (b0 + lane);
        int s = 0, e = 0;
        in_t av{};
        if (t < o1) {
            seg(__ldg(oci + t), s, e);
            if constexpr (OUTV) av = load_val<SR>(ov, t);
        }
        const int tbase = o0 + wq + nw * b0;   // outer position of lane 0's entry
        const int len = max(0, e - s);         // an unsorted row can give e < s in a tile index
        // long ranges: cooperative walk (CTA teams list the biggest)
        bool listed = false;
        if constexpr (CTA) {
            if (len >= BIG_SEG) {
                const int slot = atomicAdd(&s_nbig, 1);
                if (slot < BIG_LIST) {
                    s_big[slot][0] = t;
                    s_big[slot][1] = s;
                    s_big[slot][2] = e;
                    s_biga[slot] = av;
                    listed = true;
                }
            }
        }
        unsigned lmask = __ballot_sync(FULL, len >= LONG_SEG && !listed);
        while (lmask) {
            const int u = __ffs(lmask) - 1;
            lmask &= lmask - 1;
            const int su = __shfl_sync(FULL, s, u), eu = __shfl_sync(FULL, e, u);
            const in_t au = shfl_val<SR>(av, u);
            walk_range<SR, WSYNC>(tbase + nw * u, au, su, eu, 0, 1, ici, iv, f);
        }
        // short ranges: load-balanced flat enumeration, two products per lane
        // per pass (both searches and both loads in flight together)
        const int sl = len < LONG_SEG ? len : 0;
        const int incl = warp_incl_scan(sl);
        const int total = __shfl_sync(FULL, incl, 31);
        const int excl = incl - sl;
        for (int base = 0; base < total; base += 64) {
            const int p0 = base + lane, p1 = p0 + 32;
            int k0 = 0, k1 = 0;
#pragma unroll
            for (int st = 16; st > 0; st >>= 1) {
                const int c0 = __shfl_sync(FULL, incl, k0 + st - 1);
                const int c1 = __shfl_sync(FULL, incl, k1 + st - 1);
                if (c0 <= p0) k0 += st;
                if (c1 <= p1) k1 += st;
            }
            k0 &= 31;
            k1 &= 31;
            const int q0 = __shfl_sync(FULL, s, k0) + p0 - __shfl_sync(FULL, excl, k0);
            const int q1 = __shfl_sync(FULL, s, k1) + p1 - __shfl_sync(FULL, excl, k1);
            const in_t a0 = shfl_val<SR>(av, k0), a1 = shfl_val<SR>(av, k1);
            int col0 = NO_PRODUCT, col1 = NO_PRODUCT;
            in_t b0{}, b1{};
            if (p0 < total) {
                col0 = __ldg(ici + q0);
                b0 = load_val<SR>(iv, q0);
            }
            if (p1 < total) {
                col1 = __ldg(ici + q1);
                b1 = load_val<SR>(iv, q1);
            }
            if (WSYNC || p0 < total) f(tbase + nw * k0, a0, col0, b0);
            if (WSYNC || p1 < total) f(tbase + nw * k1, a1, col1, b1);
        }
    }
    if constexpr (CTA) {
        // listed ranges: their 128-entry chunks, concatenated, dealt to the
        // warps round-robin
        block_sync();
        const int nb = min(s_nbig, BIG_LIST);
        long long g = 0;   // chunks of the ranges before this one
        for (int i = 0; i < nb; ++i) {
            const int s0 = s_big[i][1], e0 = s_big[i][2];
            const int first = (int)(((long long)wq - g % nw + nw) % nw);
            walk_range<SR, WSYNC>(s_big[i][0], s_biga[i], s0, e0, first, nw, ici, iv, f);
            g += (e0 - s0 + 127) / 128;
        }
        block_sync();   // the list is reused by the team's next call
    }
}

// ------------------------------------------------------------------ gather
// Ordered output of the mask-ordered accumulators (HASH, MCA, DOT): entries
// of the mask row, in mask order, whose state is SET (Sec. 5.2 collects the
// output in the mask's own order, so it comes out sorted).  get(q, v)
// returns whether mask entry q is SET and its accumulated value in v.
template <int SR, bool CTA, class G>
__device__ __forceinline__ void gather_by(const int *mcols, int mnz, const G &get, long long tmp, const TmpOut &T,
                                          int *cnt_slot, int *scratch, int aligned, bool write) {
    using S = Sr<SR>;
    using acc_t = typename S::acc_t;
    using out_t = typename S::out_t;
    Team<CTA> team;
    const int lane = lane_id();
    out_t *tv = static_cast<out_t *>(T.v);
    if (aligned) {
        for (int q = team.tid(); q < mnz; q += team.size()) {
            acc_t v;
            if (get(q, v)) tv[tmp + q] = S::out(v);
        }
        return;
    }
    if (!CTA) {
        int base = 0;
        for (int r0 = 0; r0 < mnz; r0 += 32) {
            const int q = r0 + lane;
            acc_t v{};
            const bool keep = q < mnz && get(q, v);
            const unsigned bal = __ballot_sync(FULL, keep);
            if (keep && write) {
                const long long o = tmp + base + __popc(bal & lanemask_lt());
                T.ci[o] = mcols[q];
                tv[o] = S::out(v);
            }
            base += __popc(bal);
        }
        if (lane == 0) *cnt_slot = base;
    } else {
        const int nw = team.nwarps(), w = team.warp();
        const int seg = ((mnz + nw - 1) / nw + 31) & ~31;
        const int s0 = min(mnz, w * seg), s1 = min(mnz, s0 + seg);
        int c = 0;
        for (int r0 = s0; r0 < s1; r0 += 32) {
            const int q = r0 + lane;
            acc_t v{};
            c += __popc(__ballot_sync(FULL, q < s1 && get(q, v)));
        }
        int total;
        const int off = block_excl_scan(lane == 0 ? c : 0, scratch, &total);
        int base = __shfl_sync(FULL, off, 0);
        for (int r0 = s0; r0 < s1; r0 += 32) {
            const int q = r0 + lane;
            acc_t v{};
            const bool keep = q < s1 && get(q, v);
            const unsigned bal = __ballot_sync(FULL, keep);
            if (keep && write) {
                const long long o = tmp + base + __popc(bal & lanemask_lt());
                T.ci[o] = mcols[q];
                tv[o] = S::out(v);
            }
            base += __popc(bal);
        }
        if (threadIdx.x == 0) *cnt_slot = total;
    }
}

// Rank-indexed accumulators (MCA, DOT): acc[q] and SET bit q belong to mask
// entry q.
template <int SR, bool CTA>
__device__ __forceinline__ void gather_ranked(const int *mcols, int mnz, const typename Sr<SR>::acc_t *acc,
                                              const unsigned *sb, long long tmp, const TmpOut &T,
                                              int *cnt_slot, int *scratch, int aligned, bool write) {
    using acc_t = typename Sr<SR>::acc_t;
    auto get = [&](int q, acc_t &v) -> bool {
        v = acc[q];
        if constexpr (Sr<SR>::count_set) return v != 0;
        else return test_bit(sb, q);
    };
    gather_by<SR, CTA>(mcols, mnz, get, tmp, T, cnt_slot, scratch, aligned, write);
}

// Row context.
struct RowCtx {
    int i, n;
    int a0, a1, m0, m1;
    long long r, tmp, flops;
};

__device__ __forceinline__ RowCtx row_ctx(const DevProd &P, long long r, const RowArrays &ra) {
    RowCtx c;
    c.r = r;
    c.i = (int)(r - P.row0);
    c.n = P.n;
    c.a0 = __ldg(P.a_rp + c.i);
    c.a1 = __ldg(P.a_rp + c.i + 1);
    c.m0 = __ldg(P.m_rp + c.i);
    c.m1 = __ldg(P.m_rp + c.i + 1);
    c.tmp = ra.tmpoff[r];
    c.flops = ra.flops[r];
    return c;
}



// --------------------------------------------------------------- HASH rows
// Sec. 5.3: a table keyed by the mask's columns, no resizing; a product
// whose column is not a key is never evaluated (NOTALLOWED).  The paper's
// table probes linearly; here every key is placed by two-choice (cuckoo)
// hashing, so a lookup reads exactly two slots with no probe loop: on a warp,
// a linear probe runs as long as the longest chain among its 32 lanes, which
// made the probe loop most of the kernel's instructions.  The accumulator of
// a key lives in the key's own slot; for semirings with a separate SET state
// it is bit 31 of the key word (columns are below 2^31 - 1).  The gather walks
// the mask row in order and looks each column up again.
//
// Building: each mask column is inserted by atomic exchange, carrying any
// key it displaces to that key's other position (at most CUCKOO_KICKS moves
// per key).  If an insertion runs out of moves, the table is rebuilt with the
// second multiplier pair, and if that fails too, with linear probing (the
// paper's form) in the same layout; every form finds every key.
constexpr unsigned KEY_SET = 0x80000000u;

// Inserts the mask row's columns; returns true on failure (team-uniform).
template <bool CTA>
__device__ __forceinline__ bool cuckoo_build(unsigned *key, const CuckooHash &ch, const int *mcols, int mnz,
                                             int kicks) {
    Team<CTA> team;
    bool fail = false;
    for (int q = team.tid(); q < mnz; q += team.size()) {
        unsigned x = (unsigned)__ldg(mcols + q);
        unsigned pos = ch.h1(x);
        int it = 0;
        for (; it < kicks; ++it) {
            const unsigned y = atomicExch(&key[pos], x);
            if (y == EMPTY32) break;
            x = y;   // carry the displaced key to its other position
            unsigned a, b;
            ch.pos(y, a, b);
            pos = pos == a ? b : a;
        }
        if (it == kicks) fail = true;
    }
    team.sync();
    if constexpr (CTA) return __syncthreads_or(fail) != 0;
    else return __any_sync(FULL, fail);
}

template <bool CTA>
__device__ __forceinline__ void linear_build(unsigned *key, const CuckooHash &ch, const int *mcols, int mnz) {
    Team<CTA> team;
    for (int q = team.tid(); q < mnz; q += team.size()) {
        const unsigned x = (unsigned)__ldg(mcols + q);
        unsigned h = ch.h1(x);
        while (atomicCAS(&key[h], EMPTY32, x) != EMPTY32) h = h + 1 == ch.H ? 0u : h + 1;
    }
    team.sync();
}

template <bool CTA>
__device__ __forceinline__ void clear_keys(unsigned *key, unsigned H) {
    Team<CTA> team;
    for (unsigned h = team.tid(); h < H; h += team.size()) key[h] = EMPTY32;
    team.sync();
}

template <int SR, bool CTA>
__device__ __forceinline__ void row_hash(const DevProd &P, const RowCtx &c, const RowLaunch &L, unsigned char *slab, int *scratch) {
    using S = Sr<SR>;
    using acc_t = typename S::acc_t;
    using in_t = typename S::in_t;
    constexpr bool SETB = SrSizes<SR>::setbits;
    constexpr unsigned KMASK = SETB ? ~KEY_SET : ~0u;   // key bits of a slot word
    Team<CTA> team;
    const int mnz = c.m1 - c.m0;
    const unsigned H = (unsigned)hash_slots(mnz, (int)sizeof(acc_t), L.slab);
    unsigned *key = reinterpret_cast<unsigned *>(slab);
    acc_t *acc = reinterpret_cast<acc_t *>(slab + align8(4LL * H));
    const int *mcols = P.m_ci + c.m0;
    for (unsigned h = team.tid(); h < H; h += team.size()) {
        key[h] = EMPTY32;
        acc[h] = 0;
    }
    team.sync();
    CuckooHash ch = cuckoo_hash(CUCKOO_A, H);
    const int kicks = L.hash_kicks;
    bool linear = kicks <= 0;
    if (linear) {
        linear_build<CTA>(key, ch, mcols, mnz);
    } else if (cuckoo_build<CTA>(key, ch, mcols, mnz, kicks)) {
        clear_keys<CTA>(key, H);
        ch.c = CUCKOO_B;
        if (cuckoo_build<CTA>(key, ch, mcols, mnz, kicks)) {
            clear_keys<CTA>(key, H);
            linear_build<CTA>(key, ch, mcols, mnz);
            linear = true;
        }
    }
    // a hit: add the product into the slot; mark SET once (bit 31 of the key word)
    auto hit = [&](unsigned p, unsigned kw, in_t a, in_t b) {
        S::add(&acc[p], S::mul(a, b));
        if constexpr (SETB)
            if (!(kw & KEY_SET)) atomicOr(&key[p], KEY_SET);
    };
    // slot of a key known to be in the table
    auto slot_of = [&](unsigned x) -> unsigned {
        unsigned h, h2;
        ch.pos(x, h, h2);
        if (!linear) {
            return (ld_vol(&key[h]) & KMASK) == x ? h : h2;
        }
        while ((ld_vol(&key[h]) & KMASK) != x) h = h + 1 == H ? 0u : h + 1;
        return h;
    };
    if (!linear) {
        // called on every lane for every product slot (NO_PRODUCT: none), so the
        // lookup runs without a branch around it
        auto ins = [&](int, in_t a, int j, in_t b) {
            // NO_PRODUCT (2^32 - 2 as a key) equals neither a column nor an empty slot
            const unsigned x = (unsigned)j;
            unsigned p1, p2;
            ch.pos(x, p1, p2);
            const unsigned k1 = ld_vol(&key[p1]), k2 = ld_vol(&key[p2]);
            const bool f1 = (k1 & KMASK) == x, f2 = (k2 & KMASK) == x;
            if (f1 | f2) hit(f1 ? p1 : p2, f1 ? k1 : k2, a, b);
        };
        enum_products<SR, CTA, true, true>(c.a0, c.a1, P.a_ci, P.a_v, RowSeg{P.b_rp}, P.b_ci, P.b_v, ins);
    } else {
        auto ins = [&](int, in_t a, int j, in_t b) {
            unsigned h = ch.h1((unsigned)j);
            for (;;) {   // terminates: at least half of the slots are empty
                const unsigned kk = ld_vol(&key[h]);
                if ((kk & KMASK) == (unsigned)j) {
                    hit(h, kk, a, b);
                    return;
                }
                if (kk == EMPTY32) return;   // NOTALLOWED: product never evaluated
                h = h + 1 == H ? 0u : h + 1;
            }
        };
        enum_products<SR, CTA, true>(c.a0, c.a1, P.a_ci, P.a_v, RowSeg{P.b_rp}, P.b_ci, P.b_v, ins);
    }
    team.sync();
    auto get = [&](int q, acc_t &v) -> bool {
        const unsigned p = slot_of((unsigned)__ldg(mcols + q));
        v = ld_vol(&acc[p]);
        if constexpr (Sr<SR>::count_set) return v != 0;
        else return (ld_vol(&key[p]) & KEY_SET) != 0;
    };
    gather_by<SR, CTA>(mcols, mnz, get, c.tmp, out_of(P, L), L.ra.cnt + c.r, scratch, L.aligned, !L.count_only);
    team.sync();
}

// --------------------------------------------------------------- MCA rows
// Sec. 5.4: arrays of length nnz(m) indexed by the rank of j in the mask row;
// the rank comes from a binary search in the staged (sorted) mask row.
template <int SR, bool CTA>
__device__ __forceinline__ void row_mca(const DevProd &P, const RowCtx &c, const RowLaunch &L, unsigned char *slab, int *scratch) {
    using S = Sr<SR>;
    using acc_t = typename S::acc_t;
    using in_t = typename S::in_t;
    Team<CTA> team;
    const int mnz = c.m1 - c.m0;
    int *mcol = reinterpret_cast<int *>(slab);
    acc_t *acc = reinterpret_cast<acc_t *>(slab + align8(4LL * mnz));
    unsigned *sb = reinterpret_cast<unsigned *>(slab + align8(4LL * mnz) + align8((long long)mnz * sizeof(acc_t)));
    stage_async<4, CTA>(mcol, P.m_ci + c.m0, mnz);   // the mask row, in flight while the arrays clear
    for (int q = team.tid(); q < mnz; q += team.size()) acc[q] = 0;
    if constexpr (SrSizes<SR>::setbits)
        for (int w = team.tid(); w < (int)words32(mnz); w += team.size()) sb[w] = 0;
    stage_wait();
    team.sync();
    auto ins = [&](int, in_t a, int j, in_t b) {
        int lo = 0, hi = mnz;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (mcol[mid] < j) lo = mid + 1; else hi = mid;
        }
        if (lo < mnz && mcol[lo] == j) {
            S::add(&acc[lo], S::mul(a, b));
            if constexpr (SrSizes<SR>::setbits) set_bit_once(sb, lo);
        }
    };
    enum_products<SR, CTA, true>(c.a0, c.a1, P.a_ci, P.a_v, RowSeg{P.b_rp}, P.b_ci, P.b_v, ins);
    team.sync();
    gather_ranked<SR, CTA>(mcol, mnz, acc, sb, c.tmp, out_of(P, L), L.ra.cnt + c.r, scratch, L.aligned,
                           !L.count_only);
    team.sync();
}

// --------------------------------------------------------------- DOT rows
// Sec. 4.1 pull: for each mask entry (i, j), the sparse dot A_i* . B_*j.  A_i*
// is staged in shared memory; the pairs (j, k in column j of B) are
// enumerated and k is found in A_i* by binary search.
template <int SR, bool CTA>
__device__ __forceinline__ void row_dot(const DevProd &P, const RowCtx &c, const RowLaunch &L, unsigned char *slab, int *scratch) {
    using S = Sr<SR>;
    using acc_t = typename S::acc_t;
    using in_t = typename S::in_t;
    Team<CTA> team;
    const int mnz = c.m1 - c.m0, anz = c.a1 - c.a0;
    int *acol = reinterpret_cast<int *>(slab);
    in_t *aval = reinterpret_cast<in_t *>(slab + align8(4LL * anz));
    const long long avb = Sr<SR>::vals ? align8((long long)anz * sizeof(in_t)) : 0;
    acc_t *acc = reinterpret_cast<acc_t *>(slab + align8(4LL * anz) + avb);
    unsigned *sb = reinterpret_cast<unsigned *>(reinterpret_cast<unsigned char *>(acc) + align8((long long)mnz * sizeof(acc_t)));
    // the row A_i* (columns and values), in flight while the arrays clear
    stage_async<4, CTA>(acol, P.a_ci + c.a0, anz);
    if constexpr (Sr<SR>::vals) {
        if (P.a_v)
            stage_async<(int)sizeof(in_t), CTA>(aval, static_cast<const in_t *>(P.a_v) + c.a0, anz);
        else   // a pattern operand: every value 1
            for (int q = team.tid(); q < anz; q += team.size()) aval[q] = in_t(1);
    }
    for (int q = team.tid(); q < mnz; q += team.size()) acc[q] = 0;
    if constexpr (SrSizes<SR>::setbits)
        for (int w = team.tid(); w < (int)words32(mnz); w += team.size()) sb[w] = 0;
    stage_wait();
    team.sync();
    const int m0 = c.m0;
    auto ins = [&](int t, in_t, int k, in_t b) {
        int lo = 0, hi = anz;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (acol[mid] < k) lo = mid + 1; else hi = mid;
        }
        if (lo < anz && acol[lo] == k) {
            const int rk = t - m0;
            in_t a{};
            if constexpr (Sr<SR>::vals) a = aval[lo];
            S::add(&acc[rk], S::mul(a, b));
            if constexpr (SrSizes<SR>::setbits) set_bit_once(sb, rk);
        }
    };
    enum_products<SR, CTA, false>(c.m0, c.m1, P.m_ci, nullptr, RowSeg{P.bt_rp}, P.bt_ci, P.bt_v, ins);
    team.sync();
    gather_ranked<SR, CTA>(P.m_ci + c.m0, mnz, acc, sb, c.tmp, out_of(P, L), L.ra.cnt + c.r, scratch, L.aligned,
                           !L.count_only);
    team.sync();
}

// --------------------------------------------------------------- MSA_W rows
// Sec. 5.2 MSA per warp: dense values and two bit arrays (ALLOWED, SET) over
// all n columns.  Invariant between rows: everything zero; a row resets only
// the positions of its own mask entries (O(nnz(m)), not O(n)).
template <int SR>
__device__ __forceinline__ void row_msa_w(const DevProd &P, const RowCtx &c, const RowLaunch &L, unsigned char *slab) {
    using S = Sr<SR>;
    using acc_t = typename S::acc_t;
    using in_t = typename S::in_t;
    using out_t = typename S::out_t;
    const int lane = lane_id();
    const int n = c.n;
    acc_t *vals = reinterpret_cast<acc_t *>(slab);
    unsigned *allowed = reinterpret_cast<unsigned *>(slab + align8((long long)n * sizeof(acc_t)));
    unsigned *setw = allowed + words32(n);
    for (int q = c.m0 + lane; q < c.m1; q += 32) {
        const int j = __ldg(P.m_ci + q);
        atomicOr(&allowed[j >> 5], 1u << (j & 31));
    }
    __threadfence_block();
    __syncwarp();
    auto ins = [&](int, in_t a, int j, in_t b) {
        if (test_bit(allowed, j)) {
            S::add(&vals[j], S::mul(a, b));
            if constexpr (SrSizes<SR>::setbits) set_bit_once(setw, j);
        }
    };
    enum_products<SR, false, true>(c.a0, c.a1, P.a_ci, P.a_v, RowSeg{P.b_rp}, P.b_ci, P.b_v, ins);
    __threadfence_block();
    __syncwarp();
    const TmpOut T = out_of(P, L);
    out_t *tv = static_cast<out_t *>(T.v);
    int base = 0;
    if (L.aligned) {
        for (int q = c.m0 + lane; q < c.m1; q += 32) {
            const int j = __ldg(P.m_ci + q);
            bool keep;
            if constexpr (S::count_set) keep = vals[j] != 0;
            else keep = test_bit(setw, j);
            if (keep) tv[c.tmp + (q - c.m0)] = S::out(vals[j]);
        }
    } else
    for (int q0 = c.m0; q0 < c.m1; q0 += 32) {
        const int q = q0 + lane;
        int j = 0;
        bool keep = false;
        if (q < c.m1) {
            j = __ldg(P.m_ci + q);
            if constexpr (S::count_set) keep = vals[j] != 0;
            else keep = test_bit(setw, j);
        }
        const unsigned bal = __ballot_sync(FULL, keep);
        if (keep && !L.count_only) {
            const long long o = c.tmp + base + __popc(bal & lanemask_lt());
            T.ci[o] = j;
            tv[o] = S::out(vals[j]);
        }
        base += __popc(bal);
    }
    if (lane == 0) L.ra.cnt[c.r] = base;
    __threadfence_block();
    __syncwarp();
    for (int q = c.m0 + lane; q < c.m1; q += 32) {
        const int j = __ldg(P.m_ci + q);
        vals[j] = 0;
        allowed[j >> 5] = 0;
        setw[j >> 5] = 0;
    }
    __threadfence_block();
    __syncwarp();
}

// --------------------------------------------------------------- CHASH rows
// Complemented mask, hash keyed by the produced columns (Sec. 5.3 with the
// complement of Sec. 5.2): a product is dropped when its column is in the
// mask row (binary search in the staged sorted row); otherwise it is added
// under its column, inserting the key on first sight.  Capacity is a power of
// two >= 2 x min(flops, n - nnz(m)) so probing always ends.  The occupied
// slots are bitonic-sorted by column for the canonical ascending output.
template <int SR, bool CTA>
__device__ __forceinline__ void row_chash(const DevProd &P, const RowCtx &c, const RowLaunch &L, unsigned char *slab) {
    using S = Sr<SR>;
    using acc_t = typename S::acc_t;
    using in_t = typename S::in_t;
    using out_t = typename S::out_t;
    Team<CTA> team;
    const int mnz = c.m1 - c.m0;
    const long long bound = min(c.flops, (long long)(c.n - mnz));
    const long long H = pow2_at_least(2 * bound);
    const int logH = ilog2(H);
    const unsigned hmask = (unsigned)H - 1u;
    unsigned *keys = reinterpret_cast<unsigned *>(slab);
    acc_t *vals = reinterpret_cast<acc_t *>(slab + align8(4 * H));
    int *mcol = reinterpret_cast<int *>(slab + align8(4 * H) + align8(H * (long long)sizeof(acc_t)));
    stage_async<4, CTA>(mcol, P.m_ci + c.m0, mnz);   // the mask row, in flight while the table clears
    for (long long h = team.tid(); h < H; h += team.size()) {
        keys[h] = EMPTY32;
        vals[h] = 0;
    }
    stage_wait();
    team.sync();
    auto ins = [&](int, in_t a, int j, in_t b) {
        int lo = 0, hi = mnz;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (mcol[mid] < j) lo = mid + 1; else hi = mid;
        }
        if (lo < mnz && mcol[lo] == j) return;   // in the mask: NOTALLOWED under complement
        unsigned h = hash32((unsigned)j, logH);
        for (;;) {
            const unsigned k = keys[h];
            if (k == (unsigned)j) break;
            if (k == EMPTY32) {
                const unsigned prev = atomicCAS(&keys[h], EMPTY32, (unsigned)j);
                if (prev == EMPTY32 || prev == (unsigned)j) break;
            }
            h = (h + 1) & hmask;
        }
        S::add(&vals[h], S::mul(a, b));
    };
    enum_products<SR, CTA, true>(c.a0, c.a1, P.a_ci, P.a_v, RowSeg{P.b_rp}, P.b_ci, P.b_v, ins);
    team.sync();
    // bitonic sort of (key, value) over H slots, ascending; EMPTY sorts last
    for (long long kk = 2; kk <= H; kk <<= 1) {
        for (long long jj = kk >> 1; jj > 0; jj >>= 1) {
            for (long long x = team.tid(); x < H / 2; x += team.size()) {
                const long long lo = 2 * jj * (x / jj) + (x % jj);
                const long long hi = lo + jj;
                const bool up = (lo & kk) == 0;
                const unsigned kl = keys[lo], kh = keys[hi];
                if ((kl > kh) == up) {
                    keys[lo] = kh;
                    keys[hi] = kl;
                    const acc_t t = vals[lo];
                    vals[lo] = vals[hi];
                    vals[hi] = t;
                }
            }
            team.sync();
        }
    }
    // occupied slots form a sorted prefix; write it out
    const TmpOut T = out_of(P, L);
    out_t *tv = static_cast<out_t *>(T.v);
    int cntl = 0;
    for (long long x = team.tid(); x < H; x += team.size()) {
        const unsigned k = keys[x];
        if (k != EMPTY32) {
            if (!L.count_only) {
                T.ci[c.tmp + x] = (int)k;
                tv[c.tmp + x] = S::out(vals[x]);
            }
            ++cntl;
        }
    }
    // count = number of occupied slots
    if (!CTA) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cntl += __shfl_xor_sync(FULL, cntl, o);
        if (lane_id() == 0) L.ra.cnt[c.r] = cntl;
    } else {
        __shared__ int red;
        if (threadIdx.x == 0) red = 0;
        block_sync();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cntl += __shfl_xor_sync(FULL, cntl, o);
        if (lane_id() == 0) atomicAdd(&red, cntl);
        block_sync();
        if (threadIdx.x == 0) L.ra.cnt[c.r] = red;
    }
    team.sync();
}

// --------------------------------------------------------------- HEAP rows
// Sec. 5.5, Alg. 4 and 5: the row is the multiway merge of the rows B_k*
// (k in A_i*), consumed in ascending column order and intersected with the
// sorted mask row (or, complemented, with its complement) by a two-way merge.
// The priority queue of row iterators becomes a warp-wide tournament: lane l
// holds the iterators of stored entries l, l + 32, ... of A_i* in registers,
// and a warp minimum over their current columns is the queue's top.  All
// iterators at the top column are popped together; their products form the
// column's sum, and each is advanced and re-inserted by Alg. 5's procedure.
// NI is NInspect: 0 inserts at once; otherwise the iterator first walks
// towards the current mask entry, giving up after NI mask entries passed
// (Heap: 1, HeapDot: unbounded).  Complemented rows use NI = 0.  Output comes
// out ascending and compact.
template <int SR>
__device__ __forceinline__ typename Sr<SR>::acc_t warp_sum_acc(typename Sr<SR>::acc_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

template <int SR, int NI, bool COMP>
__device__ __forceinline__ void row_heap(const DevProd &P, const RowCtx &c, const RowLaunch &L) {
    using S = Sr<SR>;
    using acc_t = typename S::acc_t;
    using in_t = typename S::in_t;
    using out_t = typename S::out_t;
    const int lane = lane_id();
    const int m1 = c.m1;
    int pos[HEAP_PER_LANE], end[HEAP_PER_LANE], col[HEAP_PER_LANE];
    in_t av[HEAP_PER_LANE];
    int mq = c.m0;   // the mask iterator (warp-uniform)
    // Alg. 5 for iterator x: its column, or INT_MAX when it leaves the queue
    auto insert = [&](int x) {
        int p = pos[x];
        const int e = end[x];
        int cc = INT_MAX;
        if constexpr (NI == 0) {
            if (p < e) cc = __ldg(P.b_ci + p);
        } else {
            int mi = mq, left = NI;
            while (p < e && mi < m1) {
                const int bc = __ldg(P.b_ci + p), mc = __ldg(P.m_ci + mi);
                if (bc == mc) { cc = bc; break; }
                if (bc < mc) {
                    ++p;
                } else {
                    ++mi;
                    if (--left == 0) { cc = bc; break; }
                }
            }
        }
        pos[x] = p;
        col[x] = cc;
    };
#pragma unroll
    for (int x = 0; x < HEAP_PER_LANE; ++x) {
        const int t = c.a0 + lane + 32 * x;
        pos[x] = end[x] = 0;
        col[x] = INT_MAX;
        av[x] = in_t{};
        if (t < c.a1) {
            const int k = __ldg(P.a_ci + t);
            pos[x] = __ldg(P.b_rp + k);
            end[x] = __ldg(P.b_rp + k + 1);
            if constexpr (S::vals) av[x] = load_val<SR>(P.a_v, t);
            insert(x);
        }
    }
    const TmpOut T = out_of(P, L);
    out_t *tv = static_cast<out_t *>(T.v);
    int o = 0;
    for (;;) {
        int lm = INT_MAX;
#pragma unroll
        for (int x = 0; x < HEAP_PER_LANE; ++x) lm = min(lm, col[x]);
        const int top = __reduce_min_sync(FULL, lm);
        if (top == INT_MAX) break;   // queue empty
        // advance the mask iterator to its first entry >= top, 32 entries a step
        while (mq < m1 && __ldg(P.m_ci + mq) < top) {
            const int q = mq + lane;
            const int v = q < m1 ? __ldg(P.m_ci + q) : INT_MAX;
            const unsigned bal = __ballot_sync(FULL, v >= top);
            mq = bal ? mq + __ffs(bal) - 1 : min(m1, mq + 32);
        }
        if (!COMP && mq >= m1) break;   // mask exhausted: nothing more can be kept
        const bool in_mask = mq < m1 && __ldg(P.m_ci + mq) == top;
        const bool keep = COMP ? !in_mask : in_mask;
        acc_t s = 0;
#pragma unroll
        for (int x = 0; x < HEAP_PER_LANE; ++x) {
            if (col[x] == top) {
                if (keep) s += S::mul(av[x], load_val<SR>(P.b_v, pos[x]));
                ++pos[x];
                insert(x);
            }
        }
        if (keep) {
            s = warp_sum_acc<SR>(s);
            if (lane == 0 && !L.count_only) {
                if (!COMP && L.aligned) {
                    tv[c.tmp + (mq - c.m0)] = S::out(s);
                } else {
                    T.ci[c.tmp + o] = top;
                    tv[c.tmp + o] = S::out(s);
                }
            }
            ++o;
        }
    }
    if (lane == 0) L.ra.cnt[c.r] = o;
    __syncwarp();
}

// --------------------------------------------------------------- _T rows
// Sec. 5.2 MSA for rows too heavy for a per-row shared table, on one CTA.
// The column range is cut into tiles of T columns; a tile holds dense values
// and two bit arrays (ALLOWED -- or NOTALLOWED when complemented -- and SET)
// in shared memory.  B rows are sorted, so each stored A_ik keeps a cursor
// into B_k* that the next tile resumes from; the mask row is consumed tile by
// tile the same way.  Output comes out in ascending column order.  With a
// single tile the cursors are skipped.  Invariant between tiles and rows:
// values and bits are zero.
template <int SR, bool COMP>
__device__ __forceinline__ void row_msa_t(const DevProd &P, const RowCtx &c, const RowLaunch &L, unsigned char *slab, int *scratch) {
    using S = Sr<SR>;
    using acc_t = typename S::acc_t;
    using in_t = typename S::in_t;
    using out_t = typename S::out_t;
    using TA = TileAcc<SR>;
    using lo_t = typename TA::lo_t;
    Team<true> team;
    const int lane = lane_id();
    const int T = L.tileT;
    lo_t *vals = reinterpret_cast<lo_t *>(slab);
    unsigned *mbits = reinterpret_cast<unsigned *>(slab + align8((long long)T * sizeof(lo_t)));
    unsigned *setw = mbits + words32(T);
    unsigned *hi = tile_hi_of<SR>(L);
    if (TA::split && !hi) {   // uniform over the CTA
        if (threadIdx.x == 0) atomicOr(L.ra.err, ERR_INTERNAL);
        return;
    }
    const int n = c.n;
    const int ntiles = (n + T - 1) / T;
    // Column tiles come from the product's tile index when it has one (exact
    // range of every (row of B, tile)); otherwise from per-entry cursors:
    // cursor of stored entry t of A (product-local index) is cursors[abase + t].
    const bool use_index = P.tpos != nullptr;
    int4 *cur = L.cursors + P.abase;
    const TmpOut Tout = out_of(P, L);
    out_t *tv = static_cast<out_t *>(Tout.v);
    __shared__ int s_out;    // entries written so far in this row
    __shared__ int s_mpos;   // mask cursor
    if (threadIdx.x == 0) { s_out = 0; s_mpos = c.m0; }
    if (ntiles > 1 && !use_index) {
        for (int t = c.a0 + team.tid(); t < c.a1; t += team.size()) {
            const int k = __ldg(P.a_ci + t);
            const int s = __ldg(P.b_rp + k), e = __ldg(P.b_rp + k + 1);
            cur[t] = make_int4(s, e, s < e ? __ldg(P.b_ci + s) : INT_MAX, 0);
        }
    }
    cta_sync();
    for (int tile = 0; tile < ntiles; ++tile) {
        const int c0 = tile * T, c1 = min(n, c0 + T);
        const int mq0 = s_mpos;
        // mask entries of this tile: [mq0, mq1)
        int mq1;
        {
            int lo = mq0, hi = c.m1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(P.m_ci + mid) < c1) lo = mid + 1; else hi = mid;
            }
            mq1 = lo;
        }
        // In-tile guards: sorted rows keep every index inside [0, T); an
        // unsorted row (invalid input) is flagged and its stray entry skipped
        // rather than indexing outside the tile.
        for (int q = mq0 + team.tid(); q < mq1; q += team.size()) {
            const int jj = __ldg(P.m_ci + q) - c0;
            if ((unsigned)jj < (unsigned)T) atomicOr(&mbits[jj >> 5], 1u << (jj & 31));
            else atomicOr(L.ra.err, ERR_INTERNAL);
        }
        cta_sync();
        auto ins = [&](int jj, in_t a, in_t b) {
            if ((unsigned)jj >= (unsigned)T) {
                atomicOr(L.ra.err, ERR_INTERNAL);
                return;
            }
            const bool m = test_bit(mbits, jj);
            if (m != COMP) {   // plain: allowed iff in mask; complemented: iff not
                TA::add(vals, hi, jj, S::mul(a, b));
                if constexpr (COMP || SrSizes<SR>::setbits) set_bit_once(setw, jj);
            }
        };
        if (ntiles == 1) {
            auto f = [&](int, in_t a, int j, in_t b) { ins(j, a, b); };
            enum_products<SR, true, true>(c.a0, c.a1, P.a_ci, P.a_v, RowSeg{P.b_rp}, P.b_ci, P.b_v, f);
        } else if (use_index) {
            auto f = [&](int, in_t a, int j, in_t b) { ins(j - c0, a, b); };
            const TileSeg seg{P.tpos, P.tstride, tile};
            enum_products<SR, true, true>(c.a0, c.a1, P.a_ci, P.a_v, seg, P.b_ci, P.b_v, f);
        } else {
            // Contiguous windows of 32 entries per warp (coalesced cursor
            // loads).  Pass 1: every lane advances its own entry's segment
            // inside the tile, up to LS entries, so the many short segments
            // (low-degree k) proceed 32 at a time.  Pass 2: segments still
            // open (long rows of B) are walked by the whole warp; the next
            // column after the tile comes from the loaded chunk by shuffle.
            constexpr int LS = 3;
            for (int w0 = c.a0 + team.warp() * 32; w0 < c.a1; w0 += team.nwarps() * 32) {
                const int t = w0 + lane;
                int4 cu = make_int4(0, 0, INT_MAX, 0);
                in_t av{};
                if (t < c.a1) cu = cur[t];
                if (!__any_sync(FULL, cu.z < c1)) continue;
                if constexpr (Sr<SR>::vals) {
                    if (t < c.a1) av = load_val<SR>(P.a_v, t);
                }
                const int x0 = cu.x;
#pragma unroll 1
                for (int rep = 0; rep < LS; ++rep) {
                    const bool go = cu.z < c1;
                    if (!__any_sync(FULL, go)) break;
                    if (go) {
                        const in_t b = load_val<SR>(P.b_v, cu.x);
                        const int nx = cu.x + 1;
                        const int ncol = nx < cu.y ? __ldg(P.b_ci + nx) : INT_MAX;
                        ins(cu.z - c0, av, b);
                        cu.x = nx;
                        cu.z = ncol;
                    }
                }
                unsigned act = __ballot_sync(FULL, cu.z < c1);
                while (act) {
                    const int u = __ffs(act) - 1;
                    act &= act - 1;
                    const int pos = __shfl_sync(FULL, cu.x, u), end = __shfl_sync(FULL, cu.y, u);
                    const in_t au = shfl_val<SR>(av, u);
                    int stop = end, nextc = INT_MAX;
                    for (int q0 = pos; q0 < end; q0 += 128) {
                        int col[4];
                        in_t bv[4];
#pragma unroll
                        for (int x = 0; x < 4; ++x) {
                            const int q = q0 + x * 32 + lane;
                            col[x] = (q < end) ? __ldg(P.b_ci + q) : INT_MAX;
                            if (col[x] < c1) bv[x] = load_val<SR>(P.b_v, q);
                        }
                        bool done = false;
#pragma unroll
                        for (int x = 0; x < 4; ++x) {
                            if (!done) {
                                const bool ok = col[x] < c1;
                                if (ok) ins(col[x] - c0, au, bv[x]);
                                const unsigned okm = __ballot_sync(FULL, ok);
                                if (okm != FULL) {
                                    // sorted row: the ok lanes are a prefix; the
                                    // first other lane holds the next column
                                    const int first = __popc(okm);
                                    stop = q0 + x * 32 + first;
                                    nextc = __shfl_sync(FULL, col[x], first);
                                    done = true;
                                }
                            }
                        }
                        if (done) break;
                    }
                    if (lane == u) {
                        cu.x = stop;
                        cu.z = stop < end ? nextc : INT_MAX;
                    }
                }
                if (t < c.a1 && cu.x != x0) cur[t] = cu;
            }
        }
        cta_sync();
        // gather this tile in ascending column order
        int outbase = s_out;
        if (!COMP) {
            // over the tile's mask entries, in mask order (= ascending)
            const int cntm = mq1 - mq0;
            const int nw = team.nwarps(), w = team.warp();
            const int seg = ((cntm + nw - 1) / nw + 31) & ~31;
            const int s0 = mq0 + min(cntm, w * seg), s1 = mq0 + min(cntm, w * seg + seg);
            auto kept = [&](int jj) -> bool {
                if ((unsigned)jj >= (unsigned)T) return false;
                if constexpr (S::count_set) return vals[jj] != 0;
                else return test_bit(setw, jj);
            };
            int cw = 0;
            for (int r0 = s0; r0 < s1; r0 += 32) {
                const int q = r0 + lane;
                const bool keep = q < s1 && kept(__ldg(P.m_ci + q) - c0);
                if (L.aligned && keep) tv[c.tmp + (q - c.m0)] = S::out(TA::get(vals, hi, __ldg(P.m_ci + q) - c0));
                cw += __popc(__ballot_sync(FULL, keep));
            }
            int total;
            const int off = block_excl_scan(lane == 0 ? cw : 0, scratch, &total);
            int base = outbase + __shfl_sync(FULL, off, 0);
            for (int r0 = s0; r0 < s1; r0 += 32) {
                const int q = r0 + lane;
                int j = 0;
                bool keep = false;
                if (q < s1) {
                    j = __ldg(P.m_ci + q);
                    keep = kept(j - c0);
                }
                const unsigned bal = __ballot_sync(FULL, keep);
                if (keep && !L.aligned && !L.count_only) {
                    const long long o = c.tmp + base + __popc(bal & lanemask_lt());
                    Tout.ci[o] = j;
                    tv[o] = S::out(TA::get(vals, hi, j - c0));
                }
                base += __popc(bal);
            }
            cta_sync();
            for (int q = s0 + lane; q < s1; q += 32) {
                const int jj = __ldg(P.m_ci + q) - c0;
                if ((unsigned)jj >= (unsigned)T) continue;
                TA::clear(vals, hi, jj);
                mbits[jj >> 5] = 0;
                setw[jj >> 5] = 0;
            }
            if (threadIdx.x == 0) { s_out = outbase + total; s_mpos = mq1; }
        } else {
            // scan the SET bits of the tile; each thread owns a run of words
            const int nwords = (int)words32(c1 - c0);
            const int per = (nwords + team.size() - 1) / team.size();
            const int w0 = min(nwords, team.tid() * per), w1 = min(nwords, w0 + per);
            int cw = 0;
            for (int w = w0; w < w1; ++w) cw += __popc(setw[w]);
            int total;
            const int off = block_excl_scan(cw, scratch, &total);
            long long o = c.tmp + outbase + off;
            for (int w = w0; w < w1; ++w) {
                unsigned bits = setw[w];
                while (bits) {
                    const int b = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const int jj = w * 32 + b;
                    const auto v = S::out(TA::take(vals, hi, jj));
                    if (!L.count_only) {
                        Tout.ci[o] = c0 + jj;
                        tv[o] = v;
                    }
                    ++o;
                }
                setw[w] = 0;
            }
            cta_sync();
            for (int q = mq0 + team.tid(); q < mq1; q += team.size()) {
                const int jj = __ldg(P.m_ci + q) - c0;
                if ((unsigned)jj < (unsigned)T) mbits[jj >> 5] = 0;
            }
            if (threadIdx.x == 0) { s_out = outbase + total; s_mpos = mq1; }
        }
        cta_sync();
    }
    if (threadIdx.x == 0) L.ra.cnt[c.r] = s_out;
    cta_sync();
}

// ------------------------------------------------------------------ kernels
template <int SR, int KIND>
__global__ void __launch_bounds__(256) k_rows_w(const __grid_constant__ ProdSet ps, const __grid_constant__ RowLaunch L) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int wib = threadIdx.x >> 5;
    unsigned char *slab = smem + (size_t)wib * L.slab;
    const int count = L.ra.kind_count[KIND];
    const int off = L.ra.kind_off[KIND];
    if (KIND == K_MSA_W) {   // invariant: the dense arrays start zeroed
        for (int x = lane_id(); x < L.slab / 4; x += 32) reinterpret_cast<unsigned *>(slab)[x] = 0;
        __syncwarp();
    }
    // rows from a device counter, one per warp at a time (the bucket lists
    // heavy rows first): no warp is left with a tail of heavy rows
    for (;;) {
        int x = 0;
        if (lane_id() == 0) x = atomicAdd(&L.ra.kind_next[KIND], 1);
        x = __shfl_sync(FULL, x, 0);
        if (x >= count) break;
        const long long r = L.ra.perm[off + x];
        const DevProd &P = prod_at(ps, row_prod(ps, L.ra.prod, r));
        const RowCtx c = row_ctx(P, r, L.ra);
        if (KIND == K_HASH_W) row_hash<SR, false>(P, c, L, slab, nullptr);
        else if (KIND == K_MCA_W) row_mca<SR, false>(P, c, L, slab, nullptr);
        else if (KIND == K_DOT_W) row_dot<SR, false>(P, c, L, slab, nullptr);
        else if (KIND == K_MSA_W) row_msa_w<SR>(P, c, L, slab);
        else if (KIND == K_CHASH_W) row_chash<SR, false>(P, c, L, slab);
        else if (KIND == K_HEAP_W) row_heap<SR, 1, false>(P, c, L);
        else if (KIND == K_HEAPDOT_W) row_heap<SR, HEAP_INSPECT_ALL, false>(P, c, L);
        else if (KIND == K_CHEAP_W) row_heap<SR, 0, true>(P, c, L);
    }
}

// --------------------------------------------------------------- MCA, team of eight
// Sec. 5.4's mask-compressed accumulator for the smallest rows (at most QMASK
// mask entries and few push products, the bulk of the rows of a batch of
// small products): an eight-lane team per row, four rows per warp.  The mask
// row m sits in registers of every lane of the team, and so do the QMASK
// accumulators of its entries: a product's rank in m is the index of the mask
// column equal to its column, found by comparing with all of them (after a
// range test that rejects most products at once).  The team walks the rows of
// B one A entry at a time, its lanes striding B_k*; afterwards it sums its
// lanes' accumulators with shuffles and writes the SET entries in mask order.
// No shared memory and no barrier: the per-row fixed cost of the warp kinds
// (clearing, staging, gathering mask-sized arrays) is what dominates such rows.
template <int SR>
__global__ void __launch_bounds__(256) k_rows_q(const __grid_constant__ ProdSet ps, const __grid_constant__ RowLaunch L) {
    using S = Sr<SR>;
    using acc_t = typename S::acc_t;
    using in_t = typename S::in_t;
    using out_t = typename S::out_t;
    const int lane = lane_id(), g = lane >> 3, tl = lane & 7;
    const unsigned tmask = 0xffu << (8 * g);   // the team's lanes
    const int count = L.ra.kind_count[K_MCA_Q];
    const int off = L.ra.kind_off[K_MCA_Q];
    for (;;) {
        int x = 0;
        if (lane == 0) x = atomicAdd(&L.ra.kind_next[K_MCA_Q], 4);
        x = __shfl_sync(FULL, x, 0);
        if (x >= count) break;   // uniform over the warp
        const int xr = x + g;    // this team's row (none past the bucket's end)
        const bool have = xr < count;
        const long long r = have ? (long long)L.ra.perm[off + xr] : 0;
        const DevProd &P = prod_at(ps, have ? row_prod(ps, L.ra.prod, r) : 0);
        int a0 = 0, a1 = 0, m0 = 0, mnz = 0;
        long long tmp = 0;
        if (have) {
            const long long i = r - P.row0;
            a0 = __ldg(P.a_rp + i);
            a1 = __ldg(P.a_rp + i + 1);
            m0 = __ldg(P.m_rp + i);
            mnz = __ldg(P.m_rp + i + 1) - m0;
            tmp = L.ra.tmpoff[r];
        }
        // the mask row in registers; -1 (never a column) past its end
        const int mv = tl < mnz ? __ldg(P.m_ci + m0 + tl) : -1;
        int mk[QMASK];
#pragma unroll
        for (int q = 0; q < QMASK; ++q) mk[q] = __shfl_sync(FULL, mv, (g << 3) + q);
        const int mlo = mk[0];
        const int mhi = __shfl_sync(FULL, mv, (g << 3) + max(mnz - 1, 0));
        const unsigned mspan = (unsigned)(mhi - mlo);
        acc_t acc[QMASK];
#pragma unroll
        for (int q = 0; q < QMASK; ++q) acc[q] = 0;
        unsigned setm = 0;
        if (mnz > 0) {   // uniform over the team
            // A entries eight at a time: lane u holds entry a + u (its value
            // and the range of its row of B); the team then walks each row
            for (int a = a0; a < a1; a += QTEAM) {
                const int t = a + tl;
                int s = 0, e = 0;
                in_t av{};
                if (t < a1) {
                    const int k = __ldg(P.a_ci + t);
                    av = load_val<SR>(P.a_v, t);
                    s = __ldg(P.b_rp + k);
                    e = __ldg(P.b_rp + k + 1);
                }
                const int na = min(QTEAM, a1 - a);
                for (int u = 0; u < na; ++u) {   // uniform over the team
                    const int src = (g << 3) + u;
                    const int su = __shfl_sync(tmask, s, src), eu = __shfl_sync(tmask, e, src);
                    const in_t au = shfl_val_mask<SR>(tmask, av, src);
                    for (int q = su + tl; q < eu; q += QTEAM) {
                        const int j = __ldg(P.b_ci + q);
                        if ((unsigned)(j - mlo) > mspan) continue;   // outside the mask row's range
                        unsigned hitm = 0;
#pragma unroll
                        for (int w = 0; w < QMASK; ++w) hitm |= (j == mk[w]) ? (1u << w) : 0u;
                        if (hitm) {
                            const acc_t pv = S::mul(au, load_val<SR>(P.b_v, q));
#pragma unroll
                            for (int w = 0; w < QMASK; ++w)
                                if (hitm & (1u << w)) acc[w] += pv;
                            setm |= hitm;
                        }
                    }
                }
            }
        }
        // team sums (a fixed butterfly over the eight lanes)
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
#pragma unroll
            for (int w = 0; w < QMASK; ++w) acc[w] += shfl_xor_acc<SR>(FULL, acc[w], o);
            setm |= __shfl_xor_sync(FULL, setm, o);
        }
        acc_t v = 0;
#pragma unroll
        for (int w = 0; w < QMASK; ++w)
            if (w == tl) v = acc[w];
        const bool keep = have && tl < mnz && ((setm >> tl) & 1u);
        const unsigned bal = (__ballot_sync(FULL, keep) >> (8 * g)) & 0xffu;
        if (have) {
            const TmpOut T = out_of(P, L);
            out_t *tv = static_cast<out_t *>(T.v);
            if (L.aligned) {
                if (keep) tv[tmp + tl] = S::out(v);
            } else if (!L.count_only && keep) {
                const long long o = tmp + __popc(bal & ((1u << tl) - 1u));
                T.ci[o] = mv;
                tv[o] = S::out(v);
            }
            if (tl == 0) L.ra.cnt[r] = __popc(bal);
        }
    }
}

// --------------------------------------------------------------- DOT, team of eight
// Sec. 4.1's pull form for rows with at most QDMASK mask entries and little
// pull work (in a batch of small products: rows whose single mask entry meets
// a heavy row of A): an eight-lane team per row, four rows per warp.  For each
// mask entry j the team's lanes stride the column B_*j (row j of B^T); each
// entry k is found in the sorted row A_i* by a binary search in global memory
// (the row is read through L1 by all eight lanes; nothing is staged), and the
// products a_ik b_kj are summed per lane, then over the team by shuffles.
template <int SR>
__global__ void __launch_bounds__(256) k_rows_dq(const __grid_constant__ ProdSet ps, const __grid_constant__ RowLaunch L) {
    using S = Sr<SR>;
    using acc_t = typename S::acc_t;
    using out_t = typename S::out_t;
    const int lane = lane_id(), g = lane >> 3, tl = lane & 7;
    const unsigned tmask = 0xffu << (8 * g);   // the team's lanes
    const int count = L.ra.kind_count[K_DOT_Q];
    const int off = L.ra.kind_off[K_DOT_Q];
    for (;;) {
        int x = 0;
        if (lane == 0) x = atomicAdd(&L.ra.kind_next[K_DOT_Q], 4);
        x = __shfl_sync(FULL, x, 0);
        if (x >= count) break;   // uniform over the warp
        const int xr = x + g;
        const bool have = xr < count;
        const long long r = have ? (long long)L.ra.perm[off + xr] : 0;
        const DevProd &P = prod_at(ps, have ? row_prod(ps, L.ra.prod, r) : 0);
        int a0 = 0, a1 = 0, m0 = 0, mnz = 0;
        long long tmp = 0;
        if (have) {
            const long long i = r - P.row0;
            a0 = __ldg(P.a_rp + i);
            a1 = __ldg(P.a_rp + i + 1);
            m0 = __ldg(P.m_rp + i);
            mnz = __ldg(P.m_rp + i + 1) - m0;
            tmp = L.ra.tmpoff[r];
        }
        // mask entry w sits in slot w / 8 of lane w % 8 (up to QDMASK entries)
        int mv[QDMASK / QTEAM];
        acc_t v[QDMASK / QTEAM];
        unsigned setm = 0;   // bit s: this lane's slot s is SET
#pragma unroll
        for (int sl = 0; sl < QDMASK / QTEAM; ++sl) {
            const int w = sl * QTEAM + tl;
            mv[sl] = w < mnz ? __ldg(P.m_ci + m0 + w) : -1;
            v[sl] = 0;
        }
        for (int w = 0; w < mnz; ++w) {   // uniform over the team
            int jm = mv[0];
#pragma unroll
            for (int sl = 1; sl < QDMASK / QTEAM; ++sl)
                if ((w >> 3) == sl) jm = mv[sl];
            const int j = __shfl_sync(tmask, jm, (g << 3) + (w & 7));
            const int s = __ldg(P.bt_rp + j), e = __ldg(P.bt_rp + j + 1);
            acc_t part = 0;
            bool hit = false;
            for (int q = s + tl; q < e; q += QTEAM) {
                const int k = __ldg(P.bt_ci + q);
                int lo = a0, hi = a1;   // first entry of A_i* with column >= k
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (__ldg(P.a_ci + mid) < k) lo = mid + 1; else hi = mid;
                }
                if (lo < a1 && __ldg(P.a_ci + lo) == k) {
                    part += S::mul(load_val<SR>(P.a_v, lo), load_val<SR>(P.bt_v, q));
                    hit = true;
                }
            }
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) part += shfl_xor_acc<SR>(tmask, part, o);
            const bool any = (__ballot_sync(tmask, hit) & tmask) != 0;
            if (tl == (w & 7)) {
#pragma unroll
                for (int sl = 0; sl < QDMASK / QTEAM; ++sl)
                    if ((w >> 3) == sl) {
                        v[sl] = part;
                        if (any) setm |= 1u << sl;
                    }
            }
        }
        // SET entries in mask order: slot by slot, the team's lanes in order
        const TmpOut T = out_of(P, L);
        out_t *tv = static_cast<out_t *>(T.v);
        int base = 0;
#pragma unroll
        for (int sl = 0; sl < QDMASK / QTEAM; ++sl) {
            const bool keep = have && ((setm >> sl) & 1u);
            const unsigned bal = (__ballot_sync(FULL, keep) >> (8 * g)) & 0xffu;
            if (keep) {
                if (L.aligned) {
                    tv[tmp + sl * QTEAM + tl] = S::out(v[sl]);
                } else if (!L.count_only) {
                    const long long o = tmp + base + __popc(bal & ((1u << tl) - 1u));
                    T.ci[o] = mv[sl];
                    tv[o] = S::out(v[sl]);
                }
            }
            base += __popc(bal);
        }
        if (have && tl == 0) L.ra.cnt[r] = base;
    }
}

template <int SR, int KIND>
__global__ void __launch_bounds__(256, 4) k_rows_b(const __grid_constant__ ProdSet ps, const __grid_constant__ RowLaunch L) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int scratch[40];
    __shared__ int s_row;
    const int count = L.ra.kind_count[KIND];
    const int off = L.ra.kind_off[KIND];
    // rows from a device counter, heavy rows first (bucket order)
    for (;;) {
        block_sync();
        if (threadIdx.x == 0) s_row = atomicAdd(&L.ra.kind_next[KIND], 1);
        block_sync();
        const int x = s_row;
        if (x >= count) break;
        const long long r = L.ra.perm[off + x];
        const DevProd &P = prod_at(ps, row_prod(ps, L.ra.prod, r));
        const RowCtx c = row_ctx(P, r, L.ra);
        if (KIND == K_HASH_B || KIND == K_HASH_L) row_hash<SR, true>(P, c, L, smem, scratch);
        else if (KIND == K_MCA_B) row_mca<SR, true>(P, c, L, smem, scratch);
        else if (KIND == K_DOT_B) row_dot<SR, true>(P, c, L, smem, scratch);
        else if (KIND == K_CHASH_B) row_chash<SR, true>(P, c, L, smem);
    }
}

// One CTA per SM (the slab takes the SM's shared memory), so every thread may
// hold up to 128 registers.
template <int SR, bool COMP>
__global__ void __launch_bounds__(512, 1) k_rows_t(const __grid_constant__ ProdSet ps, const __grid_constant__ RowLaunch L) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int scratch[40];
    __shared__ int s_row;
    constexpr int KIND = COMP ? K_CMSA_T : K_MSA_T;
    const int count = L.ra.kind_count[KIND];
    const int off = L.ra.kind_off[KIND];
    {   // zero the tile arrays once
        unsigned *w = reinterpret_cast<unsigned *>(smem);
        for (int x = threadIdx.x; x < L.slab / 4; x += blockDim.x) w[x] = 0;
    }
    for (;;) {
        cta_sync();
        if (threadIdx.x == 0) s_row = atomicAdd(&L.ra.kind_next[KIND], 1);
        cta_sync();
        const int x = s_row;
        if (x >= count) break;
        const long long r = L.ra.perm[off + x];
        const DevProd &P = prod_at(ps, row_prod(ps, L.ra.prod, r));
        const RowCtx c = row_ctx(P, r, L.ra);
        row_msa_t<SR, COMP>(P, c, L, smem, scratch);
    }
}

// ------------------------------------------------------ MSA, grid of tiles
// Heavy rows as (row, column tile) items swept tile-major over the whole GPU:
// complemented rows with dense output (CMSA_G: their reachable columns are at
// least a quarter of those the mask leaves open), and plain rows with the
// most push work in products wider than one tile (MSA_G), which one CTA per
// row would leave most SMs idle for.  Items go out tile-major from a device
// counter: the CTAs of the whole GPU sweep one column tile at a time, so that
// tile's slice of B and of the tile index stays in L2 while every such row
// passes over it, instead of each row streaming all of B from HBM.  An item
// is Sec. 5.2's MSA on one tile and writes its entries, ascending, at the
// row's exact offset for the tile: for a plain mask the mask entries before
// the tile (the row's room is its mask row); complemented, the columns before
// the tile that the mask leaves open (room n - nnz(M_i*)).  The CTA that
// completes a row's last item (a device-scope count after a fence; nothing
// waits) packs the row's pieces to the front of its room.

// Insertion of product (j, a*b) into a grid item's tile.  Column state bits:
// bit 0 the mask (ALLOWED for a plain mask, NOTALLOWED when complemented),
// bit 1 SET; two bits per column in one word array, so a product reads one
// word to learn both.  A product is added when the mask allows it.
// TRACK: its column is marked SET on the column's first product.  Without
// TRACK nothing is marked, and *unsafe is raised by any product that could
// make a column's sum zero although the column is SET (a value not in
// (0, 2^31) -- for int64, also any carry into the high word): while no
// product does, SET <=> the column's sum is non-zero, and the gather reads the
// values instead of the bits.
template <int SR>
__device__ __forceinline__ bool grid_safe(typename Sr<SR>::acc_t v) {
    if constexpr (SR == MSGEMM_PLUS_TIMES_F32) return v > 0.0f;   // false for 0, negatives, NaN
    else if constexpr (SR == MSGEMM_PLUS_TIMES_I64) return (long long)v > 0 && v < (1ULL << 31);
    else return true;                                              // plus-pair: counts >= 1
}

// Position of tile column jj in the grid kinds' value arrays: its low five
// bits XORed with the next five, a permutation within every 32-column group
// (tile widths are multiples of 32).  A warp walking a sorted row of B meets
// columns at near-regular spacing, and spacings that share factors with 32
// put many lanes on few shared-memory banks; the swizzle spreads them.
__device__ __forceinline__ int vswz(int jj) { return jj ^ ((jj >> 5) & 31); }

template <int SR, bool COMP>
struct GridIns {
    using S = Sr<SR>;
    using TA = TileAcc<SR>;
    using lo_t = typename TA::lo_t;
    using in_t = typename S::in_t;
    lo_t *vals;
    unsigned *st;
    unsigned *hi;
    unsigned *err;
    int *unsafe;
    int c0, T;
    bool track;   // uniform over the CTA
    __device__ __forceinline__ void operator()(int, in_t a, int j, in_t b) const {
        const int jj = j - c0;
        if ((unsigned)jj >= (unsigned)T) {   // only an unsorted row of B gets here
            atomicOr(err, ERR_INTERNAL);
            return;
        }
        if (COMP && !track) {
            // speculative complemented tile: every product is added, with no
            // state read; the gather drops (and clears) the columns the mask
            // holds.  One shared access per product instead of two.
            const typename S::acc_t v = S::mul(a, b);
            if constexpr (TA::split) {
                const unsigned l = (unsigned)v;
                const unsigned old = atomicAdd(&vals[vswz(jj)], l);
                if (!grid_safe<SR>(v) || old + l < old) *unsafe = 1;
            } else {
                TA::add(vals, hi, vswz(jj), v);
                if (!grid_safe<SR>(v)) *unsafe = 1;
            }
            return;
        }
        const unsigned w = st[jj >> 4] >> (2 * (jj & 15));
        if ((w & 1u) != (COMP ? 1u : 0u)) {
            const typename S::acc_t v = S::mul(a, b);
            if (track) {
                TA::add(vals, hi, vswz(jj), v);
                if (!(w & 2u)) atomicOr(&st[jj >> 4], 2u << (2 * (jj & 15)));
            } else if constexpr (TA::split) {
                // int64: the low word only; a carry would need the high word
                const unsigned l = (unsigned)v;
                const unsigned old = atomicAdd(&vals[vswz(jj)], l);
                if (!grid_safe<SR>(v) || old + l < old) *unsafe = 1;
            } else {
                TA::add(vals, hi, vswz(jj), v);
                if (!grid_safe<SR>(v)) *unsafe = 1;
            }
        }
    }
};

// One item.  Entries are written ascending from obase; in the gradient form
// (aligned, plain masks) values go to their mask entry's own slot instead.
// For a dense tile (the row's push work per tile at least 8x the tile width,
// so reading every column's value at the gather is cheap) the products first
// run without SET bits; if any was unsafe (see GridIns) the tile's values are
// cleared and the products run again with them, and the launch stops
// speculating (values with signs, say).  Returns the entries written.
template <int SR, bool COMP>
__device__ __forceinline__ int grid_tile(const DevProd &P, const RowCtx &c, const RowLaunch &L, unsigned char *slab,
                                         int *scratch, int *s_unsafe, int *s_spec, int tile, int ntiles, int mq0,
                                         int mq1, long long obase) {
    using S = Sr<SR>;
    using out_t = typename S::out_t;
    using TA = TileAcc<SR>;
    using lo_t = typename TA::lo_t;
    Team<true> team;
    const int T = L.tileT;
    lo_t *vals = reinterpret_cast<lo_t *>(slab);
    unsigned *st = reinterpret_cast<unsigned *>(slab + align8((long long)T * sizeof(lo_t)));   // T / 16 words
    unsigned *hi = tile_hi_of<SR>(L);   // checked by the caller
    const int c0 = tile * T, c1 = min(c.n, c0 + T);
    if (threadIdx.x == 0) {
        *s_unsafe = 0;
        *s_spec = *(volatile int *)L.spec_off == 0;   // one read, shared by the CTA after the barrier
    }
    for (int q = mq0 + team.tid(); q < mq1; q += team.size()) {
        const int jj = __ldg(P.m_ci + q) - c0;
        if ((unsigned)jj < (unsigned)T) atomicOr(&st[jj >> 4], 1u << (2 * (jj & 15)));
        else atomicOr(L.ra.err, ERR_INTERNAL);
    }
    cta_sync();
    const bool dense = c.flops / ntiles >= 8LL * T;
    const bool speculate = dense && *s_spec;   // uniform over the CTA
    GridIns<SR, COMP> ins{vals, st, hi, L.ra.err, s_unsafe, c0, T, !speculate};
    bool tracked = !speculate;
    for (int pass = 0; pass < 2; ++pass) {   // pass 1 only after an unsafe product
        if (ntiles == 1) {
            enum_products<SR, true, true>(c.a0, c.a1, P.a_ci, P.a_v, RowSeg{P.b_rp}, P.b_ci, P.b_v, ins);
        } else {
            const TileSeg seg{P.tpos, P.tstride, tile};
            enum_products<SR, true, true>(c.a0, c.a1, P.a_ci, P.a_v, seg, P.b_ci, P.b_v, ins);
        }
        cta_sync();
        if (tracked || *s_unsafe == 0) break;   // uniform over the CTA
        if (threadIdx.x == 0) *(volatile int *)L.spec_off = 1;
        // clear the tile's values (low and high words) and run again with SET
        // bits; swizzled positions stay inside the last 32-column group
        for (int x = team.tid(); x < min(T, ((c1 - c0) + 31) & ~31); x += team.size()) {
            vals[x] = 0;
            if constexpr (TA::split) hi[x] = 0;
        }
        cta_sync();
        tracked = true;
        ins.track = true;
    }
    // gather the SET columns in ascending order; each thread owns a run of
    // state words (16 columns each), and clears them
    // speculative complemented tiles also added products to the columns the
    // mask holds (NOTALLOWED, bit 2b of the state word): those are dropped here
    auto nonzero_bits = [&](int w) -> unsigned {   // bit 2b set for column 16 w + b with a non-zero value
        unsigned m = 0;
        const int cend = min(16, (c1 - c0) - 16 * w);
        for (int b = 0; b < cend; ++b)
            if (vals[vswz(16 * w + b)] != 0) m |= 1u << (2 * b);
        return m;
    };
    auto set_bits = [&](int w) -> unsigned {   // bit 2b set for SET column 16 w + b
        if (tracked) return (st[w] >> 1) & 0x55555555u;
        const unsigned m = nonzero_bits(w);
        return COMP ? m & ~(st[w] & 0x55555555u) : m;
    };
    const int nwords = (c1 - c0 + 15) >> 4;
    const int per = (nwords + team.size() - 1) / team.size();
    const int w0 = min(nwords, team.tid() * per), w1 = min(nwords, w0 + per);
    int cw = 0;
    for (int w = w0; w < w1; ++w) cw += __popc(set_bits(w));
    int total;
    const int off = block_excl_scan(cw, scratch, &total);
    long long o = obase + off;
    out_t *tv = static_cast<out_t *>(L.tmp.v);
    for (int w = w0; w < w1; ++w) {
        unsigned bits = set_bits(w);
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            const int jj = w * 16 + (b >> 1);
            out_t v;
            if (tracked) {
                v = S::out(TA::take(vals, hi, vswz(jj)));
            } else {   // no carry reached the high word: the low word is the value
                v = S::out((typename S::acc_t)vals[vswz(jj)]);
                vals[vswz(jj)] = 0;
            }
            if (!COMP && L.aligned) {
                // the column's rank in the mask row (SET columns are mask columns)
                int lo = mq0, up = mq1;
                while (lo < up) {
                    const int mid = (lo + up) >> 1;
                    if (__ldg(P.m_ci + mid) < c0 + jj) lo = mid + 1; else up = mid;
                }
                tv[c.tmp + (lo - c.m0)] = v;
            } else {
                L.tmp.ci[o] = c0 + jj;
                tv[o] = v;
                ++o;
            }
        }
        if (COMP && !tracked) {   // clear the dropped columns' sums for the next item
            unsigned d = nonzero_bits(w) & st[w] & 0x55555555u;
            while (d) {
                const int b = __ffs(d) - 1;
                d &= d - 1;
                vals[vswz(w * 16 + (b >> 1))] = 0;
            }
        }
        st[w] = 0;
    }
    return total;
}

// Moves a row's tile pieces to the front of its room, in tile order.  Each
// piece moves left (its destination never passes its source), chunk by chunk,
// all reads of a chunk before its writes.  Pieces were written by other SMs:
// read through L2.
template <int SR>
__device__ __forceinline__ void grid_pack(const RowCtx &c, const RowLaunch &L, const GridTab &G, int x, int ntiles) {
    using out_t = typename Sr<SR>::out_t;
    out_t *tv = static_cast<out_t *>(L.tmp.v);
    int *tci = L.tmp.ci;
    long long dst = 0;
    for (int t = 0; t < ntiles; ++t) {
        const long long slot = (long long)x * L.gnt + t;
        const int nt = __ldcg(G.cnt + slot);
        const long long src = __ldcg(G.off + slot);
        if (src != dst) {
            for (int b = 0; b < nt; b += blockDim.x) {
                const int q = b + threadIdx.x;
                int col = 0;
                out_t v{};
                if (q < nt) {
                    col = __ldcg(tci + c.tmp + src + q);
                    v = __ldcg(tv + c.tmp + src + q);
                }
                block_sync();
                if (q < nt) {
                    tci[c.tmp + dst + q] = col;
                    tv[c.tmp + dst + q] = v;
                }
            }
        }
        dst += nt;
    }
    if (threadIdx.x == 0) L.ra.cnt[c.r] = (int)dst;
}

template <int SR, bool COMP>
__global__ void __launch_bounds__(1024, 1) k_rows_g(const __grid_constant__ ProdSet ps, const __grid_constant__ RowLaunch L) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int scratch[64];
    __shared__ long long s_item;
    __shared__ int s_mq[2];
    __shared__ int s_last;
    __shared__ int s_unsafe, s_spec;
    constexpr int KIND = COMP ? K_CMSA_G : K_MSA_G;
    const GridTab &G = L.g[COMP ? 1 : 0];
    const int count = L.ra.kind_count[KIND];
    const int off = L.ra.kind_off[KIND];
    const int T = L.tileT;
    // pieces need the temporary's room: never part of the two-phase form
    if ((TileAcc<SR>::split && !tile_hi_of<SR>(L)) || L.count_only || L.direct) {   // uniform over the CTA
        if (threadIdx.x == 0 && count > 0) atomicOr(L.ra.err, ERR_INTERNAL);
        return;
    }
    if (count == 0) return;
    {   // zero the tile arrays once; every item leaves them zeroed
        unsigned *w = reinterpret_cast<unsigned *>(smem);
        for (int x = threadIdx.x; x < L.slab / 4; x += blockDim.x) w[x] = 0;
    }
    const long long nitems = (long long)count * L.gnt;
    for (;;) {
        cta_sync();
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(G.next, 1ULL);
        cta_sync();
        const long long item = s_item;
        if (item >= nitems) break;
        const int tile = (int)(item / count), x = (int)(item % count);
        const long long r = L.ra.perm[off + x];
        const DevProd &P = prod_at(ps, row_prod(ps, L.ra.prod, r));
        const RowCtx c = row_ctx(P, r, L.ra);
        const int ntiles = (c.n + T - 1) / T;
        if (tile >= ntiles) continue;
        const int c0 = tile * T, c1 = min(c.n, c0 + T);
        if (threadIdx.x < 2) {   // first mask entry at or after the tile's start / end
            const int bound = threadIdx.x ? c1 : c0;
            int lo = c.m0, hi = c.m1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(P.m_ci + mid) < bound) lo = mid + 1; else hi = mid;
            }
            s_mq[threadIdx.x] = lo;
        }
        cta_sync();
        const int mq0 = s_mq[0], mq1 = s_mq[1];
        // the piece's offset in the row: mask entries before the tile (plain),
        // or columns before the tile the mask leaves open (complemented)
        const long long rel = COMP ? (long long)c0 - (mq0 - c.m0) : (long long)(mq0 - c.m0);
        const int cnt = grid_tile<SR, COMP>(P, c, L, smem, scratch, &s_unsafe, &s_spec, tile, ntiles, mq0, mq1,
                                            c.tmp + rel);
        __threadfence();   // this item's entries, before the row's completion count
        cta_sync();
        if (threadIdx.x == 0) {
            const long long slot = (long long)x * L.gnt + tile;
            G.cnt[slot] = cnt;
            G.off[slot] = (int)rel;
            __threadfence();
            s_last = atomicAdd(&G.done[x], 1) == ntiles - 1;
        }
        cta_sync();
        if (s_last && (COMP || !L.aligned)) {
            __threadfence();
            grid_pack<SR>(c, L, G, x, ntiles);
        }
    }
}

}  // namespace msg
